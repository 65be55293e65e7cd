"""B300 (sm_103a) library for conditional nonlinear optimal perturbations of
the 2D compressible Rayleigh-Taylor instability (arXiv 2608.04085).

This module is the thin Python binding of the C ABI declared in
``include/rt_cnop.h``: it only marshals arguments (ctypes structures, host
NumPy arrays or device tensor pointers) and raises on error statuses. Every
step of the computation runs in the CUDA library ``librt_cnop.so``; there is
no CPU fallback, and importing the binding fails loudly when that library has
not been built (``python -m paper_2608_04085_b300.build``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librt_cnop.so")

RT_OK, RT_EINVAL, RT_ENOMEM, RT_ECUDA, RT_ENONFINITE, RT_ETIMEOUT, RT_ENOTCONVERGED, RT_ESTATE, RT_EIO = range(9)
RT_BC_REFLECT, RT_BC_HYDROSTATIC = 0, 1
RT_LIM_MINMOD, RT_LIM_MC, RT_LIM_NONE = 0, 1, 2
RT_FLUX_HLLC, RT_FLUX_HLL, RT_FLUX_HYBRID = 0, 1, 2
RT_OBJ_KE, RT_OBJ_EK_ANOMALY_L2 = 0, 1
RT_FP64, RT_FP32_STATE = 0, 1
RT_CKPT_AUTO, RT_CKPT_STORE_ALL, RT_CKPT_SQRT, RT_CKPT_REVOLVE = 0, 1, 2, 3
RT_STAGE_AUTO, RT_STAGE_SWEEP, RT_STAGE_TILE, RT_STAGE_TILE8, RT_STAGE_TILE32 = 0, 1, 2, 3, 4
RT_LOADS_TMA, RT_LOADS_PLAIN = 0, 1
RT_DEVICE_PTRS, RT_REPLAY_DT, RT_GRAD_DT = 1, 2, 4
RT_CNOP_SPG, RT_CNOP_LBFGS = 0, 1
RT_RECON_X_MODES, RT_RECON_2D_POWER = 0, 1

_STATUS = {1: "RT_EINVAL", 2: "RT_ENOMEM", 3: "RT_ECUDA", 4: "RT_ENONFINITE", 5: "RT_ETIMEOUT",
           6: "RT_ENOTCONVERGED", 7: "RT_ESTATE", 8: "RT_EIO"}

#: every entry point declared in include/rt_cnop.h
EXPORTS = ("rt_init", "rt_destroy", "rt_last_error", "rt_num_instances", "rt_field_offset",
           "rt_field_size", "rt_field_total", "rt_forward", "rt_gradient", "rt_constraint",
           "rt_project", "rt_get_state", "rt_get_dt", "rt_set_kernel_timing", "rt_kernel_times", "rt_stage_kernel",
           "cnop_solve", "rt_objective_noalloc", "rt_forward_series", "rt_spectrum_x", "rt_spectrum_2d",
           "rt_reconstruct", "rt_fma_peak", "rt_revolve_plan", "rt_stage_tuning", "rt_adjoint_rows",
           "rt_tma_plan")


class RtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class RtProblem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("gamma", ctypes.c_double), ("g_y", ctypes.c_double),
                ("rho_heavy", ctypes.c_double), ("rho_light", ctypes.c_double),
                ("y_int", ctypes.c_double), ("h_s", ctypes.c_double),
                ("p_ref", ctypes.c_double), ("y_ref", ctypes.c_double),
                ("bc_y", ctypes.c_int), ("limiter", ctypes.c_int),
                ("cfl", ctypes.c_double), ("T", ctypes.c_double),
                ("nsteps", ctypes.c_int), ("perturb_ncomp", ctypes.c_int),
                ("objective", ctypes.c_int), ("flux", ctypes.c_int),
                ("flux_theta", ctypes.c_double)]

# rt_problem fields a problem description may leave out, with their values
_PROBLEM_DEFAULTS = {"flux": RT_FLUX_HLLC, "flux_theta": 2.0}


class RtOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("ckpt", ctypes.c_int),
                ("ckpt_hbm_cap_bytes", ctypes.c_double), ("max_steps", ctypes.c_int),
                ("stage_kernel", ctypes.c_int), ("y_slabs", ctypes.c_int), ("tile_loads", ctypes.c_int)]


class RtRunStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("segments", ctypes.c_int), ("bad_instance", ctypes.c_int),
                ("bad_step", ctypes.c_int), ("bad_cell", ctypes.c_longlong), ("cell_updates", ctypes.c_double),
                ("ms", ctypes.c_double), ("launches", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class CnopParams(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("gll_memory", ctypes.c_int), ("max_backtracks", ctypes.c_int),
                ("armijo_c", ctypes.c_double), ("alpha_min", ctypes.c_double), ("alpha_max", ctypes.c_double),
                ("h_loc", ctypes.c_double), ("eps", ctypes.POINTER(ctypes.c_double)),
                ("method", ctypes.c_int), ("lbfgs_memory", ctypes.c_int), ("chi_tol", ctypes.c_double),
                ("log_path", ctypes.c_char_p), ("checkpoint_path", ctypes.c_char_p),
                ("checkpoint_every", ctypes.c_int), ("resume", ctypes.c_int)]


class CnopResult(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("forward_evals", ctypes.c_int),
                ("gradient_evals", ctypes.c_int), ("ms", ctypes.c_double),
                ("C", ctypes.POINTER(ctypes.c_double)), ("chi", ctypes.POINTER(ctypes.c_double)),
                ("grad_norm", ctypes.POINTER(ctypes.c_double)), ("stop", ctypes.POINTER(ctypes.c_int)),
                ("J_history", ctypes.POINTER(ctypes.c_double))]


_lib = None


def library():
    """Load librt_cnop.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing; build it with "
                               "`python -m paper_2608_04085_b300.build` (there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
        L.rt_init.argtypes = [ctypes.POINTER(RtProblem), ip, ctypes.POINTER(RtOptions), vp, ctypes.POINTER(vp)]
        L.rt_init.restype = ip
        L.rt_destroy.argtypes = [vp]
        L.rt_destroy.restype = None
        L.rt_last_error.argtypes = [vp]
        L.rt_last_error.restype = ctypes.c_char_p
        L.rt_num_instances.argtypes = [vp]
        L.rt_num_instances.restype = ip
        for f in ("rt_field_offset", "rt_field_size"):
            getattr(L, f).argtypes = [vp, ip]
            getattr(L, f).restype = ctypes.c_size_t
        L.rt_field_total.argtypes = [vp]
        L.rt_field_total.restype = ctypes.c_size_t
        L.rt_forward.argtypes = [vp, vp, ip, dp, dp, ctypes.POINTER(RtRunStats)]
        L.rt_forward.restype = ip
        L.rt_gradient.argtypes = [vp, vp, ip, dp, vp, ctypes.POINTER(RtRunStats)]
        L.rt_gradient.restype = ip
        L.rt_constraint.argtypes = [vp, vp, ip, dp]
        L.rt_constraint.restype = ip
        L.rt_project.argtypes = [vp, vp, ip, dp, ip]
        L.rt_project.restype = ip
        L.rt_get_state.argtypes = [vp, ip, dp]
        L.rt_get_state.restype = ip
        L.rt_get_dt.argtypes = [vp, ip, dp, ip, ctypes.POINTER(ip)]
        L.rt_get_dt.restype = ip
        L.rt_stage_kernel.argtypes = [vp, dp]
        L.rt_stage_kernel.restype = ip
        L.rt_stage_tuning.argtypes = [vp, dp]
        L.rt_stage_tuning.restype = ip
        L.rt_adjoint_rows.argtypes = [vp, dp]
        L.rt_adjoint_rows.restype = ip
        L.rt_set_kernel_timing.argtypes = [vp, ip]
        L.rt_set_kernel_timing.restype = ip
        llp = ctypes.POINTER(ctypes.c_longlong)
        L.rt_kernel_times.argtypes = [vp, dp, llp, llp]
        L.rt_kernel_times.restype = ip
        L.rt_forward_series.argtypes = [vp, vp, ip, ip, ip, dp, dp, dp, ctypes.POINTER(ip)]
        L.rt_forward_series.restype = ip
        L.rt_spectrum_x.argtypes = [vp, vp, ip, ip, dp, ctypes.POINTER(ip)]
        L.rt_spectrum_x.restype = ip
        L.rt_spectrum_2d.argtypes = [vp, vp, ip, ip, dp]
        L.rt_spectrum_2d.restype = ip
        L.rt_reconstruct.argtypes = [vp, vp, ip, ip, ctypes.c_double, dp, vp, ctypes.POINTER(ip)]
        L.rt_reconstruct.restype = ip
        L.rt_fma_peak.argtypes = [dp, dp]
        L.rt_fma_peak.restype = ip
        L.rt_revolve_plan.argtypes = [ip, ip, ctypes.POINTER(ctypes.c_longlong), dp]
        L.rt_revolve_plan.restype = ip
        L.rt_tma_plan.argtypes = [vp, vp, ip, ip, vp, vp]
        L.rt_tma_plan.restype = ip
        L.cnop_solve.argtypes = [vp, ctypes.POINTER(CnopParams), vp, ip, dp, ctypes.POINTER(CnopResult)]
        L.cnop_solve.restype = ip
        _lib = L
    return _lib


def _field(w, name, alt=None, default=None):
    if isinstance(w, dict):
        if name in w:
            return w[name]
        if alt and alt in w:
            return w[alt]
        return default
    if hasattr(w, name):
        return getattr(w, name)
    if alt and hasattr(w, alt):
        return getattr(w, alt)
    return default


def make_problem(w) -> RtProblem:
    """rt_problem from any object or dict with the field names of rt_problem
    (``ncomp`` is accepted for ``perturb_ncomp``; ``flux`` and ``flux_theta``
    default to HLLC and 2)."""
    p = RtProblem()
    for name, _ in RtProblem._fields_:
        alt = "ncomp" if name == "perturb_ncomp" else None
        val = _field(w, name, alt, _PROBLEM_DEFAULTS.get(name))
        if val is None:
            raise ValueError(f"problem is missing field {name!r}")
        setattr(p, name, val)
    return p


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Context:
    """A batch of RT instances on the current CUDA device (see rt_init)."""

    def __init__(self, problems, precision=RT_FP64, ckpt=RT_CKPT_AUTO, ckpt_cap_bytes=0.0, max_steps=0,
                 stream=None, stage_kernel=RT_STAGE_AUTO, y_slabs=0, tile_loads=RT_LOADS_TMA):
        L = library()
        if not isinstance(problems, (list, tuple)):
            problems = [problems]
        self.problems = list(problems)
        arr = (RtProblem * len(problems))(*[make_problem(w) for w in problems])
        opt = RtOptions(precision, ckpt, float(ckpt_cap_bytes), int(max_steps), int(stage_kernel), int(y_slabs),
                        int(tile_loads))
        if stream is None:
            stream = self._torch_stream()
        self._stream = stream
        h = ctypes.c_void_p()
        st = L.rt_init(arr, len(problems), ctypes.byref(opt), ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if st != RT_OK:
            raise RtError(st, "rt_init failed (see stderr)")
        self._h = h
        self.n = L.rt_num_instances(h)
        self.total = L.rt_field_total(h)
        self.offsets = [L.rt_field_offset(h, i) for i in range(self.n)]
        self.sizes = [L.rt_field_size(h, i) for i in range(self.n)]

    @staticmethod
    def _torch_stream():
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return 0

    def _check(self, st, stats=None):
        if st != RT_OK:
            err = RtError(st, library().rt_last_error(self._h).decode())
            err.stats = stats.as_dict() if stats is not None else None
            raise err

    def _arg(self, a):
        """(pointer, flags, keepalive) for a host ndarray, a host (for example
        pinned) torch tensor, or a CUDA tensor; tensors are passed by pointer."""
        if hasattr(a, "data_ptr"):
            import torch
            assert a.dtype == torch.float64 and a.is_contiguous() and a.numel() == self.total
            return ctypes.c_void_p(a.data_ptr()), (RT_DEVICE_PTRS if a.is_cuda else 0), a
        a = np.ascontiguousarray(a, dtype=np.float64)
        assert a.size == self.total, (a.size, self.total)
        return a.ctypes.data_as(ctypes.c_void_p), 0, a

    def close(self):
        if getattr(self, "_h", None):
            library().rt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------ entry points
    def forward(self, v0, replay=False):
        """(J[n], J_ke[n], stats) of the forward map (rt_forward)."""
        p, flags, keep = self._arg(v0)
        J = np.zeros(self.n)
        Jke = np.zeros(self.n)
        st = RtRunStats()
        self._check(library().rt_forward(self._h, p, flags | (RT_REPLAY_DT if replay else 0), _dptr(J),
                                          _dptr(Jke), ctypes.byref(st)), st)
        del keep
        return J, Jke, st.as_dict()

    def gradient(self, v0, out=None, dt_grad=False):
        """(J[n], dJ/dv0, stats) (rt_gradient; dt_grad adds RT_GRAD_DT, the
        derivative through the step control). For a CUDA tensor input the
        gradient is a CUDA tensor, else a NumPy array."""
        p, flags, keep = self._arg(v0)
        if out is None:
            if flags & RT_DEVICE_PTRS:
                import torch
                out = torch.empty_like(v0)
            else:
                out = np.zeros(self.total)
        gp, gflags, gkeep = self._arg(out)
        assert gflags == flags, "v0 and the gradient must both be host or both be device arrays"
        J = np.zeros(self.n)
        st = RtRunStats()
        self._check(library().rt_gradient(self._h, p, flags | (RT_GRAD_DT if dt_grad else 0), _dptr(J), gp,
                                          ctypes.byref(st)), st)
        del keep, gkeep
        return J, out, st.as_dict()

    def constraint(self, v):
        p, flags, keep = self._arg(v)
        C = np.zeros(self.n)
        self._check(library().rt_constraint(self._h, p, flags, _dptr(C)))
        return C

    def project(self, v, eps, to_budget=False):
        """P(v) (Eq. projection), or the rescale onto C = eps; returns a new array."""
        if hasattr(v, "clone"):
            out = v.clone()
        else:
            out = np.array(v, dtype=np.float64, copy=True).ravel()
        p, flags, keep = self._arg(out)
        e = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, dtype=np.float64), (self.n,)))
        self._check(library().rt_project(self._h, p, flags, _dptr(e), int(bool(to_budget))))
        return out

    def state(self, inst=0):
        w = self.problems[inst]
        out = np.zeros((4, _field(w, "ny"), _field(w, "nx")))
        self._check(library().rt_get_state(self._h, inst, _dptr(out)))
        return out

    def dt(self, inst=0):
        n = ctypes.c_int(0)
        self._check(library().rt_get_dt(self._h, inst, None, 0, ctypes.byref(n)))
        out = np.zeros(max(n.value, 1))
        self._check(library().rt_get_dt(self._h, inst, _dptr(out), n.value, ctypes.byref(n)))
        return out[:n.value]

    def stage_kernel(self):
        """(variant in use, {"sweep", "tile8", "tile", "tile32": ms/step} from the
        autotuner; "tile" is the 16-row tile kernel)."""
        t = np.zeros(4)
        v = library().rt_stage_kernel(self._h, None)
        self._check(library().rt_stage_tuning(self._h, _dptr(t)))
        return v, {"sweep": t[0], "tile8": t[1], "tile": t[2], "tile32": t[3]}

    def adjoint_rows(self):
        """(adjoint tile height in use, {16: ms, 24: ms} per launch from the
        autotuner; zeros when it did not run)."""
        t = np.zeros(2)
        rows = library().rt_adjoint_rows(self._h, _dptr(t))
        return rows, {16: t[0], 24: t[1]}

    def set_kernel_timing(self, every):
        """Sample CUDA-event timings of every `every`-th time-step kernel launch."""
        self._check(library().rt_set_kernel_timing(self._h, int(every)))

    def kernel_times(self):
        """{'stage1'|'stage2'|'adjoint': (mean ms per sampled launch, samples, launches)}."""
        ms = np.zeros(3)
        sa = (ctypes.c_longlong * 3)()
        la = (ctypes.c_longlong * 3)()
        self._check(library().rt_kernel_times(self._h, _dptr(ms), sa, la))
        return {k: (ms[i], sa[i], la[i]) for i, k in enumerate(("stage1", "stage2", "adjoint"))}

    def series(self, v, every, max_samples=4096, replay=False):
        """KE(t) and h_mix(t) sampled every `every` steps of one forward run
        (rt_forward_series; at most max_samples per instance). Returns one
        dict per instance with arrays t, KE, h_mix."""
        p, flags, keep = self._arg(v)
        if replay:
            flags |= RT_REPLAY_DT
        shape = (self.n, int(max_samples))
        t, ke, h = np.zeros(shape), np.zeros(shape), np.zeros(shape)
        n = (ctypes.c_int * self.n)()
        self._check(library().rt_forward_series(self._h, p, flags, int(every), int(max_samples), _dptr(t),
                                                _dptr(ke), _dptr(h), n))
        return [{"t": t[i, :n[i]], "KE": ke[i, :n[i]], "h_mix": h[i, :n[i]]} for i in range(self.n)]

    def spectrum_x(self, v, inst=0):
        """(y_peak, E_n for n = 1 .. nx/2) of u_y (rt_spectrum_x, Eq. fourier_coeff)."""
        p, flags, keep = self._arg(v)
        E = np.zeros(_field(self.problems[inst], "nx") // 2)
        yp = ctypes.c_int()
        self._check(library().rt_spectrum_x(self._h, p, flags, int(inst), _dptr(E), ctypes.byref(yp)))
        return yp.value, E

    def spectrum_2d(self, v, inst=0):
        """Normalised 2D spectral energy E[ky, kx] of u_y (rt_spectrum_2d, App. B)."""
        p, flags, keep = self._arg(v)
        w = self.problems[inst]
        E = np.zeros((_field(w, "ny"), _field(w, "nx")))
        self._check(library().rt_spectrum_2d(self._h, p, flags, int(inst), _dptr(E)))
        return E

    def reconstruct(self, v, kind, param, eps):
        """Reduced seeds (rt_reconstruct): RT_RECON_X_MODES with param = count
        (five-mode seed) or RT_RECON_2D_POWER with param = energy fraction.
        Returns (field, kept modes per instance)."""
        p, flags, keep = self._arg(v)
        if hasattr(v, "clone"):
            out = v.clone()
        else:
            out = np.zeros(self.total)
        po, _, keep2 = self._arg(out)
        e = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, dtype=np.float64), (self.n,)))
        kept = (ctypes.c_int * self.n)()
        self._check(library().rt_reconstruct(self._h, p, flags, int(kind), float(param), _dptr(e), po, kept))
        return out, list(kept)

    def cnop(self, v_start, eps, iters, method=RT_CNOP_LBFGS, lbfgs_memory=10, gll_memory=10, armijo_c=1e-4,
             alpha_min=1e-30, alpha_max=1e30, max_backtracks=30, h_loc=0.0, chi_tol=0.0, log_path=None,
             checkpoint_path=None, checkpoint_every=0, resume=False, dt_grad=False, raise_on_stall=False):
        """CNOP search (cnop_solve): projected L-BFGS (the default) or spectral
        projected gradient. Returns (v, J, result); result holds the counts,
        the status and per-instance C, chi, grad_norm, stop and J_history
        (iterations + 1 rows)."""
        if hasattr(v_start, "clone"):
            v = v_start.clone()
        else:
            v = np.array(v_start, dtype=np.float64, copy=True).ravel()
        p, flags, keep = self._arg(v)
        if dt_grad:
            flags |= RT_GRAD_DT
        e = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, dtype=np.float64), (self.n,)))
        enc = lambda path: None if path is None else os.fsencode(path)
        prm = CnopParams(int(iters), int(gll_memory), int(max_backtracks), float(armijo_c), float(alpha_min),
                         float(alpha_max), float(h_loc), _dptr(e), int(method), int(lbfgs_memory),
                         float(chi_tol), enc(log_path), enc(checkpoint_path), int(checkpoint_every), int(bool(resume)))
        J = np.zeros(self.n)
        C, chi, gnorm = np.zeros(self.n), np.zeros(self.n), np.zeros(self.n)
        stop = np.zeros(self.n, dtype=np.int32)
        hist = np.full((int(iters) + 1, self.n), np.nan)
        res = CnopResult()
        res.C, res.chi, res.grad_norm, res.J_history = _dptr(C), _dptr(chi), _dptr(gnorm), _dptr(hist)
        res.stop = stop.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        st = library().cnop_solve(self._h, ctypes.byref(prm), p, flags, _dptr(J), ctypes.byref(res))
        if st != RT_OK and (raise_on_stall or st != RT_ENOTCONVERGED):
            self._check(st)
        out = {k: getattr(res, k) for k in ("iterations", "forward_evals", "gradient_evals", "ms")}
        return v, J, out | {"status": st, "C": C, "chi": chi, "grad_norm": gnorm, "stop": stop,
                            "J_history": hist[:res.iterations + 1]}


def revolve_plan(steps, slots):
    """(recomputed steps of the binomial schedule, Griewank-Walther minimum)
    for `steps` time steps and `slots` free checkpoint slots (rt_revolve_plan;
    host arithmetic, no device needed)."""
    n = ctypes.c_longlong(0)
    o = ctypes.c_double(0.0)
    st = library().rt_revolve_plan(int(steps), int(slots), ctypes.byref(n), ctypes.byref(o))
    if st != RT_OK:
        raise RtError(st, "rt_revolve_plan: steps and slots must be >= 0")
    return n.value, o.value


def fma_peak():
    """(FP32, FP64) FMA throughput of the current device in TFLOP/s (rt_fma_peak)."""
    f32, f64 = ctypes.c_double(), ctypes.c_double()
    st = library().rt_fma_peak(ctypes.byref(f32), ctypes.byref(f64))
    if st != RT_OK:
        raise RtError(st, "rt_fma_peak failed")
    return f32.value, f64.value


def field_layout(problems):
    """Offsets and sizes of each instance in the concatenated perturbation layout."""
    off, out = 0, []
    for w in problems:
        n = _field(w, "perturb_ncomp", "ncomp") * _field(w, "nx") * _field(w, "ny")
        out.append((off, n))
        off += n
    return out


def tma_plan(shapes, elem_bytes=4):
    """(group of each instance or -1, index within the group) of the TMA
    tile-load plan for device instances of grids shapes = [(nx, ny), ...] in
    slot order (rt_tma_plan; host arithmetic, no device needed)."""
    n = len(shapes)
    nx = np.ascontiguousarray([s[0] for s in shapes], dtype=np.int32)
    ny = np.ascontiguousarray([s[1] for s in shapes], dtype=np.int32)
    grp = np.zeros(n, dtype=np.int32)
    idx = np.zeros(n, dtype=np.int32)
    st = library().rt_tma_plan(nx.ctypes.data_as(ctypes.c_void_p), ny.ctypes.data_as(ctypes.c_void_p), n,
                               int(elem_bytes), grp.ctypes.data_as(ctypes.c_void_p),
                               idx.ctypes.data_as(ctypes.c_void_p))
    if st != RT_OK:
        raise RtError(st, "rt_tma_plan: element size must be 4 or 8")
    return grp.tolist(), idx.tolist()
