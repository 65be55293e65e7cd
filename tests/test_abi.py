"""CPU-side checks of the C ABI: the library builds, loads, and exports every
entry point that include/rt_cnop.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rt_cnop.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:rt_status|void|const char\*|int|size_t)\s+\**\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_and_binding_agree():
    import paper_2608_04085_b300 as rt
    assert _declared() == sorted(rt.EXPORTS)


def test_library_exports_every_declared_symbol():
    from paper_2608_04085_b300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_struct_sizes_match_header_layout():
    import paper_2608_04085_b300 as rt
    # rt_problem: 2 ints, 12 doubles, 2 ints, 2 doubles, 4 ints, 1 double
    assert ctypes.sizeof(rt.RtProblem) == 8 + 12 * 8 + 8 + 16 + 16 + 8
    assert rt.RtProblem.flux.offset == 140 and rt.RtProblem.flux_theta.offset == 144
    assert ctypes.sizeof(rt.RtOptions) == 32
    # cnop_params: 3 ints (+ pad), 4 doubles, a pointer, 2 ints, a double, 2 pointers, 2 ints
    # cnop_result: 3 ints (+ pad), a double, 5 pointers
    assert ctypes.sizeof(rt.CnopParams) == 16 + 32 + 8 + 8 + 8 + 16 + 8
    assert ctypes.sizeof(rt.CnopResult) == 16 + 8 + 40


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2608_04085_b300 as rt
    monkeypatch.setattr(rt, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(rt, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        rt.library()


def test_header_enums_match_binding_constants():
    import paper_2608_04085_b300 as rt
    src = open(os.path.join(ROOT, "include", "rt_cnop.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = dict((k, int(v)) for k, v in re.findall(r"\b(RT_[A-Z0-9_]+)\s*=\s*(\d+)", src))
    assert len(consts) >= 25
    for name, value in consts.items():
        assert getattr(rt, name) == value, name


def test_make_problem_fills_the_flux_fields():
    """A problem description without the flux fields gets HLLC (threshold 2);
    given ones pass through; a missing required field is an error."""
    import paper_2608_04085_b300 as rt
    import rt_inputs as I
    w = I.rt_box(8, 16, nsteps=3)
    d = {k: v for k, v in w.__dict__.items() if k not in ("flux", "flux_theta")}
    p = rt.make_problem(d)
    assert p.flux == rt.RT_FLUX_HLLC and p.flux_theta == 2.0
    assert p.perturb_ncomp == w.ncomp and p.nx == 8 and p.ny == 16
    q = rt.make_problem(w.replace(flux=I.FLUX_HYBRID, flux_theta=1.5))
    assert q.flux == rt.RT_FLUX_HYBRID and q.flux_theta == 1.5
    del d["gamma"]
    with pytest.raises(ValueError, match="gamma"):
        rt.make_problem(d)


def test_null_arguments_return_einval_without_a_gpu():
    """The ABI's error contract on the host: every entry point answers a null
    context or a missing argument with a status (never a crash), before any
    device call, so it holds on a machine without a GPU."""
    import paper_2608_04085_b300 as rt
    L = rt.library()
    h = ctypes.c_void_p()
    assert L.rt_init(None, 0, None, None, ctypes.byref(h)) == rt.RT_EINVAL and not h.value
    assert L.rt_init(None, 1, None, None, None) == rt.RT_EINVAL
    assert L.rt_forward(None, None, 0, None, None, None) == rt.RT_EINVAL
    assert L.rt_gradient(None, None, 0, None, None, None) == rt.RT_EINVAL
    assert L.rt_constraint(None, None, 0, None) == rt.RT_EINVAL
    assert L.rt_project(None, None, 0, None, 0) == rt.RT_EINVAL
    assert L.rt_get_state(None, 0, None) == rt.RT_EINVAL
    assert L.rt_get_dt(None, 0, None, 0, None) == rt.RT_EINVAL
    assert L.rt_forward_series(None, None, 0, 1, 1, None, None, None, None) == rt.RT_EINVAL
    assert L.rt_spectrum_x(None, None, 0, 0, None, None) == rt.RT_EINVAL
    assert L.rt_spectrum_2d(None, None, 0, 0, None) == rt.RT_EINVAL
    assert L.rt_reconstruct(None, None, 0, 0, 1.0, None, None, None) == rt.RT_EINVAL
    assert L.cnop_solve(None, None, None, 0, None, None) == rt.RT_EINVAL
    assert L.rt_set_kernel_timing(None, 1) == rt.RT_EINVAL
    assert L.rt_kernel_times(None, None, None, None) == rt.RT_EINVAL
    assert L.rt_fma_peak(None, None) == rt.RT_EINVAL
    assert L.rt_last_error(None) == b"null context"
    assert L.rt_num_instances(None) == 0 and L.rt_field_total(None) == 0
    assert L.rt_field_offset(None, 0) == 0 and L.rt_field_size(None, 0) == 0
    L.rt_destroy(None)
    f = ctypes.CDLL(rt.LIB_PATH).rt_objective_noalloc  # a private handle: no shared prototype changes
    f.argtypes = [ctypes.c_void_p] * 5
    f.restype = ctypes.c_int
    assert f(None, None, None, None, None) == rt.RT_EINVAL


C_USER = r"""
#include <stdlib.h>
#include "rt_cnop.h"
int main(void) {
  rt_problem p[2] = {{0}};
  rt_options o = {RT_FP32_STATE, RT_CKPT_AUTO, 0.0, 0, RT_STAGE_AUTO, 0, RT_LOADS_TMA};
  rt_ctx* ctx;
  if (rt_init(p, 2, &o, NULL, &ctx) != RT_OK) return 1;
  size_t n = rt_field_total(ctx);
  double J[2], eps[2] = {1e-4, 1e-4};
  double *v0 = calloc(n, sizeof(double)), *g = calloc(n, sizeof(double));
  rt_project(ctx, v0, 0, eps, 1);
  rt_gradient(ctx, v0, 0, J, g, NULL);
  cnop_params cp = {0};
  cp.max_iter = 5; cp.armijo_c = 1e-4; cp.eps = eps; cp.method = RT_CNOP_LBFGS;
  cnop_result cr = {0};
  cnop_solve(ctx, &cp, v0, 0, J, &cr);
  rt_destroy(ctx);
  free(v0); free(g);
  return 0;
}
"""


def test_header_is_plain_c_and_a_c_program_links(tmp_path):
    """include/rt_cnop.h compiles as strict C99 with warnings as errors, and a
    C caller links against the library (nothing is run)."""
    import shutil
    import subprocess
    from paper_2608_04085_b300 import build
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lib = build.build()
    src = tmp_path / "user.c"
    src.write_text(C_USER)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-L", os.path.dirname(lib), "-lrt_cnop", "-o", str(tmp_path / "user")],
                   check=True, capture_output=True)


def test_binding_passes_tensors_by_pointer():
    """Host torch tensors (pinned or not) reach the C ABI as host pointers to
    their own storage, CUDA tensors would carry RT_DEVICE_PTRS, and NumPy
    arrays pass as host pointers: no copy in the binding."""
    import numpy as np
    import torch
    import paper_2608_04085_b300 as rt
    ctx = rt.Context.__new__(rt.Context)  # no device needed for the marshalling
    ctx.total = 8
    t = torch.arange(8, dtype=torch.float64)
    p, flags, keep = ctx._arg(t)
    assert flags == 0 and p.value == t.data_ptr() and keep is t
    a = np.arange(8, dtype=np.float64)
    p, flags, keep = ctx._arg(a)
    assert flags == 0 and p.value == a.ctypes.data
    with pytest.raises(AssertionError):
        ctx._arg(torch.zeros(8, dtype=torch.float32))
