"""Fourier analysis and reduced seeds on the GPU (Sec. 3.5, Sec. 4.2
Eq. fourier_coeff, App. B) against the oracle's DFT definitions: the 1D
horizontal spectrum at y_peak, the 2D spectrum, the five-mode seed and the
90%-power seed, over a batch of uneven grids."""
import numpy as np
import pytest

import rt_inputs as I

pytestmark = pytest.mark.gpu


def _batch():
    ws = [I.rt_box(32, 48), I.rt_box(20, 36, ncomp=I.PERT_VY), I.paper_unit_square(24)]
    vs = []
    for k, w in enumerate(ws):
        # a smooth interface-localised packet plus noise, so the spectra are not flat
        x = (np.arange(w.nx) + 0.5) / w.nx
        y = (np.arange(w.ny) + 0.5) / w.ny
        pk = np.exp(-((y - 0.5) / 0.15) ** 2)[:, None] * np.cos(2 * np.pi * (3 + k) * x)[None, :]
        vs.append(pk[None] * np.ones((w.ncomp, 1, 1)) + 0.2 * I.gaussian_field(50 + k, w.ncomp, w.ny, w.nx))
    return ws, vs


def test_spectra_match_oracle():
    import oracle
    import paper_2608_04085_b300 as rt
    ws, vs = _batch()
    flat = np.concatenate([v.ravel() for v in vs])
    with rt.Context(ws, precision=rt.RT_FP64) as ctx:
        for i, w in enumerate(ws):
            yp, E = ctx.spectrum_x(flat, i)
            ryp, n, rE = oracle.spectrum(vs[i][-1])
            assert yp == ryp
            assert np.allclose(E, rE, rtol=1e-10, atol=1e-16)
            E2 = ctx.spectrum_2d(flat, i)
            assert np.allclose(E2, oracle.spectrum2d(vs[i][-1]), rtol=1e-10, atol=1e-16)
            assert E2.sum() == pytest.approx(1.0, rel=1e-13)


def test_reduced_seeds_match_oracle():
    import oracle
    import paper_2608_04085_b300 as rt
    ws, vs = _batch()
    flat = np.concatenate([v.ravel() for v in vs])
    eps = [1e-4, 1e-6, 1e-6]
    with rt.Context(ws, precision=rt.RT_FP64) as ctx:
        r5, kept5 = ctx.reconstruct(flat, rt.RT_RECON_X_MODES, 5, eps)
        r9, kept9 = ctx.reconstruct(flat, rt.RT_RECON_2D_POWER, 0.9, eps)
        offs, sizes = ctx.offsets, ctx.sizes
    for i, w in enumerate(ws):
        ref5, modes = oracle.five_modes(w, vs[i], eps[i])
        got5 = r5[offs[i]:offs[i] + sizes[i]]
        assert kept5[i] == sum(2 if 0 < m < w.nx // 2 else 1 for m in modes)
        assert np.allclose(got5, ref5.ravel(), rtol=1e-9, atol=1e-12 * np.abs(ref5).max())
        ref9, k9 = oracle.power_reconstruct(w, vs[i], eps[i], 0.9)
        got9 = r9[offs[i]:offs[i] + sizes[i]]
        assert kept9[i] == k9
        assert np.allclose(got9, ref9.ravel(), rtol=1e-9, atol=1e-12 * np.abs(ref9).max())
        assert oracle.constraint(w, got9) == pytest.approx(eps[i], rel=1e-12)


def test_power_seed_of_three_pairs_and_bad_arguments():
    import oracle
    import paper_2608_04085_b300 as rt
    w = I.rt_box(16, 12, ncomp=I.PERT_VY)
    j = np.arange(w.nx)[None, :]
    l = np.arange(w.ny)[:, None]
    a = np.sqrt([0.62, 0.30, 0.08])
    m1 = a[0] * np.cos(2 * np.pi * (3 * j / w.nx + 1 * l / w.ny))
    m2 = a[1] * np.sin(2 * np.pi * (5 * j / w.nx - 2 * l / w.ny))
    m3 = a[2] * np.cos(2 * np.pi * (1 * j / w.nx + 4 * l / w.ny) + 0.3)
    v = (m1 + m2 + m3).ravel()
    with rt.Context([w], precision=rt.RT_FP64) as ctx:
        r, kept = ctx.reconstruct(v, rt.RT_RECON_2D_POWER, 0.9, 1e-4)
        assert kept == [4]
        assert np.allclose(r, oracle.scale_to_budget(w, (m1 + m2)[None], 1e-4).ravel(), rtol=1e-9, atol=1e-13)
        for kind, param in ((rt.RT_RECON_2D_POWER, 0.0), (rt.RT_RECON_2D_POWER, 1.5), (rt.RT_RECON_X_MODES, 0),
                            (7, 1.0)):
            with pytest.raises(RuntimeError, match="RT_EINVAL"):
                ctx.reconstruct(v, kind, param, 1e-4)
        # the C ABI itself rejects an instance out of range
        E = np.zeros(w.nx * w.ny)
        st = rt.library().rt_spectrum_2d(ctx._h, v.ctypes.data, 0, 1, E.ctypes.data_as(rt.ctypes.POINTER(rt.ctypes.c_double)))
        assert st == rt.RT_EINVAL
