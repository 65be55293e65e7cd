"""Brute-force tangent-linear eigenproblem of a small steady stratified box,
the reference for the CNOP optimisers in the small-amplitude limit.

With g = 0 the unperturbed state is exactly steady, so at small amplitude
J_KE is the quadratic form v^T (M^T W_T M) v, M the tangent-linear map from
the perturbation to the final momenta (columns built one unit vector at a
time) and W_T = dA / rho_T. Its maximiser on {C = eps} is the leading
generalised eigenvector of (M^T W_T M, W_0), W_0 = rho0 dA.
"""
import numpy as np

import rt_inputs as I


def steady_case():
    # stratified, g = 0: the unperturbed state is exactly steady, so J_KE is a
    # pure quadratic form at small amplitude and its maximiser on {C = eps} is
    # the leading generalised eigenvector of (M^T W_T M, W_0).
    return I.rt_box(8, 24, g_y=0.0, nsteps=30, limiter=I.LIM_NONE)


def tlm_eigen(o, w):
    nv = w.ncomp * w.ny * w.nx
    zero = np.zeros((w.ncomp, w.ny, w.nx))
    base = o.forward(w, zero)
    dt = base["dt"]
    rho_T = base["U"][0]
    dx, dy = o.grid_spacing(w)
    cols = []
    for c in range(nv):
        e = np.zeros(nv)
        e[c] = 1.0
        _, dU = o.tangent_state(w, zero, e.reshape(zero.shape), dt)
        cols.append(dU[1:3].ravel())
    M = np.array(cols).T
    wT = np.tile((dx * dy / rho_T).ravel(), 2)
    rho0, _ = o.base_state(w)
    w0 = np.tile(np.repeat(rho0 * dx * dy, w.nx), w.ncomp)
    H = M.T @ (wT[:, None] * M)
    s = 1.0 / np.sqrt(w0)
    lam, V = np.linalg.eigh(s[:, None] * H * s[None, :])
    return lam[::-1], (s[:, None] * V)[:, ::-1], w0, dt
