"""Plain FP64 CPU oracle for the CNOP Rayleigh-Taylor hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product path (the
CUDA library and its Python binding) never imports, loads or calls it, and the
two share no code: the only common module is ``rt_inputs`` (seeded draws and
plain parameter values).

The time stepper, its tangent and its reverse sweep (with the dt sequence
frozen, and in a second form differentiated through the CFL step control) live
in ``rt_oracle.cpp``
(plain C++, FP64, built with ``-O2 -ffp-contract=off``); the CNOP pieces that
act on whole fields (constraint, projection, random start, spectral projected
gradient and projected L-BFGS with a non-monotone line search, 1D Fourier
spectrum, five-mode reconstruction) are plain NumPy here. Each function names the paper passage it
follows. ``branch_signature`` is a test aid: it records which side of every
kink of the scheme a run took, so that finite differences across a kink can be
told apart.

Parity status: every function below is pinned by a ``-m "not gpu"`` test
(``tests/test_oracle_*.py``) against closed forms, textbook solutions,
invariants or brute force. ``spg`` and ``lbfgs`` at finite amplitude have no
closed form; they are pinned there by the first-order (KKT) optimality
conditions of the maximisation on the energy ball, in the small-amplitude
limit by the leading eigenvector of the tangent-linear problem, and their cores
``projected_spg`` and ``projected_lbfgs`` / ``lbfgs_direction`` on analytic
objectives (the latter also against the dense BFGS update).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rt_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "librt_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C++ oracle into ``oracle/_build/librt_oracle.so``."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        cmd = ["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c++17", "-fopenmp",
               "-shared", "-fPIC", "-o", _LIB_PATH, _SRC]
        subprocess.check_call(cmd)
    return _LIB_PATH


class OParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("gamma", ctypes.c_double), ("g_y", ctypes.c_double),
                ("rho_h", ctypes.c_double), ("rho_l", ctypes.c_double),
                ("y_int", ctypes.c_double), ("h_s", ctypes.c_double),
                ("p_ref", ctypes.c_double), ("y_ref", ctypes.c_double),
                ("bc_y", ctypes.c_int), ("limiter", ctypes.c_int),
                ("cfl", ctypes.c_double), ("T", ctypes.c_double),
                ("nsteps", ctypes.c_int), ("ncomp", ctypes.c_int),
                ("objective", ctypes.c_int), ("flux", ctypes.c_int),
                ("flux_theta", ctypes.c_double)]


def _params(w) -> OParams:
    return OParams(w.nx, w.ny, w.x0, w.x1, w.y0, w.y1, w.gamma, w.g_y,
                   w.rho_heavy, w.rho_light, w.y_int, w.h_s, w.p_ref, w.y_ref,
                   w.bc_y, w.limiter, w.cfl, w.T, w.nsteps, w.ncomp, w.objective,
                   getattr(w, "flux", 0), getattr(w, "flux_theta", 2.0))


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(OParams)
        L.o_base_state.argtypes = [pp, dp, dp]
        L.o_cfl_wmin.argtypes = [pp, dp]
        L.o_cfl_wmin.restype = ctypes.c_double
        L.o_stage.argtypes = [pp, dp, ctypes.c_double, dp, dp]
        L.o_run_state.argtypes = [pp, dp, dp, ctypes.c_int]
        L.o_run_state.restype = ctypes.c_int
        L.o_inject.argtypes = [pp, dp, dp]
        L.o_forward.argtypes = [pp, dp, dp, ctypes.c_int, dp, ctypes.c_int, dp, dp, dp, dp]
        L.o_forward.restype = ctypes.c_int
        L.o_tangent.argtypes = [pp, dp, dp, dp, ctypes.c_int, dp, dp, dp]
        L.o_tangent_state.argtypes = [pp, dp, dp, dp, ctypes.c_int, dp, dp]
        L.o_gradient.argtypes = [pp, dp, dp, ctypes.c_int, dp, dp, dp]
        L.o_step_vjp.argtypes = [pp, dp, ctypes.c_double, dp, dp]
        L.o_tangent_dt.argtypes = [pp, dp, dp, ctypes.c_int, dp, dp, dp]
        L.o_tangent_dt.restype = ctypes.c_int
        L.o_gradient_dt.argtypes = [pp, dp, ctypes.c_int, dp, dp, dp]
        L.o_gradient_dt.restype = ctypes.c_int
        L.o_forward_signature.argtypes = [pp, dp, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_ulonglong)]
        L.o_set_threads.argtypes = [ctypes.c_int]
        L.o_set_threads.restype = None
        L.o_get_threads.restype = ctypes.c_int
        L.o_num_procs.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n):
    """Host threads of the oracle's row loops (OpenMP); results are bitwise
    the same for any count. The default is 1."""
    lib().o_set_threads(int(n))


def get_threads():
    return lib().o_get_threads()


def num_procs():
    """Processors available to this process (OpenMP's count)."""
    return lib().o_num_procs()


def grid_spacing(w):
    return (w.x1 - w.x0) / w.nx, (w.y1 - w.y0) / w.ny


def cell_centres(w):
    dx, dy = grid_spacing(w)
    x = w.x0 + (np.arange(w.nx) + 0.5) * dx
    y = w.y0 + (np.arange(w.ny) + 0.5) * dy
    return x, y


# ----------------------------------------------------------------- the stepper
def base_state(w):
    """Sec. 2.2, Eq. rho0: tanh density and hydrostatic pressure at cell centres."""
    rho0 = np.zeros(w.ny)
    p0 = np.zeros(w.ny)
    lib().o_base_state(ctypes.byref(_params(w)), _ptr(rho0), _ptr(p0))
    return rho0, p0


def inject(w, v):
    """Sec. 3.1: conserved initial state from the velocity perturbation v."""
    v = _f64(v)
    U = np.zeros((4, w.ny, w.nx))
    lib().o_inject(ctypes.byref(_params(w)), _ptr(v), _ptr(U))
    return U


def cfl_wmin(w, U):
    return lib().o_cfl_wmin(ctypes.byref(_params(w)), _ptr(_f64(U)))


def stage(w, U, dt, base=None):
    """One RK stage of the finite-volume scheme (stage 2 when base is given)."""
    out = np.zeros((4, w.ny, w.nx))
    b = None if base is None else _f64(base)
    lib().o_stage(ctypes.byref(_params(w)), _ptr(_f64(U)), float(dt), _ptr(b), _ptr(out))
    return out


def run_state(w, U, max_steps=10**7):
    """Advance an arbitrary conserved state with the step control of w."""
    U = _f64(U).copy()
    dts = np.zeros(max_steps if max_steps < 10**6 else 10**6)
    n = lib().o_run_state(ctypes.byref(_params(w)), _ptr(U), _ptr(dts), len(dts))
    return U, dts[:n].copy()


def forward(w, v, dt_replay=None, ek0=None, max_steps=400000):
    """Forward map F_t (Sec. 3.1) from perturbation v: returns a dict with the
    final state U, e_k, J_ke (total kinetic energy), J_pap (Eq. objective
    against ek0) and the time-step sequence dt."""
    v = _f64(v)
    U = np.zeros((4, w.ny, w.nx))
    ek = np.zeros((w.ny, w.nx))
    J = np.zeros(2)
    dts = np.zeros(max_steps)
    rep = None if dt_replay is None else _f64(dt_replay)
    n = lib().o_forward(ctypes.byref(_params(w)), _ptr(v), _ptr(rep),
                        0 if rep is None else len(rep), _ptr(dts), max_steps,
                        _ptr(None if ek0 is None else _f64(ek0)), _ptr(U), _ptr(ek), _ptr(J))
    dt = rep.copy() if rep is not None else dts[:n].copy()
    return {"U": U, "ek": ek, "J_ke": J[0], "J_pap": J[1], "dt": dt, "nsteps": n}


def branch_signature(w, v, dt_replay):
    """(hash, count) of every kink decision (limiter pick, Davis speed
    min/max, HLLC branch) of the forward run from v with the frozen step
    sequence dt_replay. Equal signatures at v + h d and v - h d mean the
    central difference along d straddles no kink."""
    dt = _f64(dt_replay)
    sig = (ctypes.c_ulonglong * 2)()
    lib().o_forward_signature(ctypes.byref(_params(w)), _ptr(_f64(v)), _ptr(dt), len(dt), sig)
    return int(sig[0]), int(sig[1])


def objective_value(w, out):
    return out["J_pap"] if w.objective == 1 else out["J_ke"]


def tangent(w, v, dv, dt, ek0=None):
    """J and its directional derivative along dv with the dt sequence frozen."""
    J = np.zeros(2)
    dJ = np.zeros(2)
    lib().o_tangent(ctypes.byref(_params(w)), _ptr(_f64(v)), _ptr(_f64(dv)), _ptr(_f64(dt)),
                    len(dt), _ptr(None if ek0 is None else _f64(ek0)), _ptr(J), _ptr(dJ))
    k = 1 if w.objective == 1 else 0
    return J[k], dJ[k]


def tangent_state(w, v, dv, dt):
    U = np.zeros((4, w.ny, w.nx))
    dU = np.zeros((4, w.ny, w.nx))
    lib().o_tangent_state(ctypes.byref(_params(w)), _ptr(_f64(v)), _ptr(_f64(dv)),
                          _ptr(_f64(dt)), len(dt), _ptr(U), _ptr(dU))
    return U, dU


def gradient(w, v, dt, ek0=None):
    """Sec. 3.4: exact discrete gradient of J (w.objective) with respect to v,
    dt sequence frozen. Returns (J, grad) with grad shaped like v."""
    v = _f64(v)
    J = np.zeros(2)
    g = np.zeros_like(v)
    lib().o_gradient(ctypes.byref(_params(w)), _ptr(v), _ptr(_f64(dt)), len(dt),
                     _ptr(None if ek0 is None else _f64(ek0)), _ptr(J), _ptr(g))
    return (J[1] if w.objective == 1 else J[0]), g


def tangent_dt(w, v, dv, ek0=None, max_steps=400000):
    """J and its directional derivative along dv with the CFL step control
    differentiated too (dt_n = cfl * min crossing time; the horizon-clipped
    last step dt = T - t). Returns (J, dJ, steps)."""
    J = np.zeros(2)
    dJ = np.zeros(2)
    n = lib().o_tangent_dt(ctypes.byref(_params(w)), _ptr(_f64(v)), _ptr(_f64(dv)), max_steps,
                           _ptr(None if ek0 is None else _f64(ek0)), _ptr(J), _ptr(dJ))
    k = 1 if w.objective == 1 else 0
    return J[k], dJ[k], n


def gradient_dt(w, v, ek0=None, max_steps=400000):
    """The gradient of J through the step control as well (the reverse of
    tangent_dt): readings in rt_oracle.cpp. Returns (J, grad, steps)."""
    v = _f64(v)
    J = np.zeros(2)
    g = np.zeros_like(v)
    n = lib().o_gradient_dt(ctypes.byref(_params(w)), _ptr(v), max_steps,
                            _ptr(None if ek0 is None else _f64(ek0)), _ptr(J), _ptr(g))
    return (J[1] if w.objective == 1 else J[0]), g, n


def value_and_gradient(w, v, ek0=None):
    """CFL-controlled forward, then the reverse sweep with that dt sequence."""
    out = forward(w, v, ek0=ek0)
    J, g = gradient(w, v, out["dt"], ek0=ek0)
    return J, g, out


def step_vjp(w, U, dt, lam):
    out = np.zeros((4, w.ny, w.nx))
    lib().o_step_vjp(ctypes.byref(_params(w)), _ptr(_f64(U)), float(dt), _ptr(_f64(lam)), _ptr(out))
    return out


def baseline_ek(w):
    """Sec. 2.3 / Eq. objective: e_k at the horizon of the unperturbed run."""
    out = forward(w, np.zeros((w.ncomp, w.ny, w.nx)))
    return out["ek"]


# ------------------------------------------------------------- CNOP, Sec. 3.4
def constraint(w, v):
    """Eq. constraint: C(v) = sum over cells and perturbed components of rho0 v^2 / 2 dx dy."""
    rho0, _ = base_state(w)
    dx, dy = grid_spacing(w)
    v = np.asarray(v, dtype=np.float64).reshape(w.ncomp, w.ny, w.nx)
    return float(np.sum(0.5 * rho0[None, :, None] * v * v) * dx * dy)


def project(w, v, eps):
    """Eq. projection: radial rescale onto C <= eps (identity inside the ball)."""
    C = constraint(w, v)
    if C <= eps:
        return np.array(v, dtype=np.float64, copy=True)
    return np.asarray(v, dtype=np.float64) * np.sqrt(eps / C)


def scale_to_budget(w, v, eps):
    """Rescale v so that C(v) = eps exactly (up to rounding)."""
    return np.asarray(v, dtype=np.float64) * np.sqrt(eps / constraint(w, v))


def random_start(w, xi, h_loc, eps):
    """Sec. 3.4: zero-mean Gaussian field localised at the interface with width
    h_loc, scaled to C = eps. Reading: envelope exp(-(y - y_int)^2 / (2 h_loc^2))."""
    _, y = cell_centres(w)
    env = np.exp(-((y - w.y_int) ** 2) / (2.0 * h_loc * h_loc))
    v = np.asarray(xi, dtype=np.float64).reshape(w.ncomp, w.ny, w.nx) * env[None, :, None]
    return scale_to_budget(w, v, eps)


def projected_spg(value, value_and_grad, proj, v_start, iters, memory=10, armijo=1e-4, alpha_min=1e-30,
                  alpha_max=1e30, max_backtracks=30, log=None, metric=None):
    """Spectral projected gradient ascent of value(v) over the set onto which
    proj projects, with the non-monotone Armijo backtracking line search of
    Grippo, Lampariello & Lucidi (Sec. 3.4): a trial is measured against the
    worst, i.e. smallest, of the last ``memory`` accepted values, so that J
    may dip temporarily.

    ``metric`` (an array like v, or None for the identity) is the diagonal of
    the inner product <a, b>_M = sum a M b in which the method steps: the
    ascent direction is the gradient's representer q = g / M, and the
    spectral step uses M-norms. With proj the exact projection in that inner
    product, the fixed points (d = 0) are the first-order (KKT) points of the
    constrained maximisation.

    Iteration k: d = proj(v + alpha q) - v; accept v + lam d once
    value(v + lam d) >= min_recent + armijo * lam * <g, d>, halving lam
    otherwise; then alpha = <s, s>_M / <s, y'> with s the step and
    y' = -(g_new - g_old) (the gradient change of the minimised objective
    -value), clipped to [alpha_min, alpha_max], and alpha_max when
    <s, y'> <= 0. The first alpha is ||v0||_M / ||q0||_M. The stationarity
    chi of App. A (with the gradient g) is recorded per iteration. Returns a
    dict with v, J, the history, the per-iteration records and the
    evaluation counts."""
    Mw = None if metric is None else np.asarray(metric, dtype=np.float64)

    def rep(g):
        return g if Mw is None else g / Mw

    def mdot(a, b):
        return float(np.sum(a * b)) if Mw is None else float(np.sum(a * Mw * b))

    def mnorm(a):
        return float(np.linalg.norm(a)) if Mw is None else float(np.sqrt(mdot(a, a)))

    v = proj(v_start)
    J, g = value_and_grad(v)
    evals, grads = 1, 1
    hist = [J]
    q = rep(g)
    alpha = mnorm(v) / max(mnorm(q), 1e-300)
    alpha = min(max(alpha, alpha_min), alpha_max)
    records = []
    for k in range(iters):
        d = proj(v + alpha * rep(g)) - v
        gd = float(np.sum(g * d))
        Jref = min(hist[-memory:])
        lam = 1.0
        accepted = False
        for _ in range(max_backtracks):
            vt = v + lam * d
            Jt = value(vt)
            evals += 1
            if Jt >= Jref + armijo * lam * gd:
                accepted = True
                break
            lam *= 0.5
        if not accepted:
            break
        Jn, gn = value_and_grad(vt)
        grads += 1
        s = vt - v
        yv = -(gn - g)
        sy = float(np.sum(s * yv))
        alpha = alpha_max if sy <= 0.0 else min(max(mdot(s, s) / sy, alpha_min), alpha_max)
        v, J, g = vt, Jn, gn
        hist.append(J)
        chi = float(np.max(np.abs(proj(v + g) - v)))
        records.append({"iter": k, "J": J, "lam": lam, "alpha": alpha, "chi": chi,
                        "grad_norm": float(np.linalg.norm(g))})
        if log is not None:
            log(records[-1])
    return {"v": v, "J": J, "history": hist, "records": records, "evals": evals, "grads": grads}


def spg(w, v_start, eps, iters, memory=10, armijo=1e-4, alpha_min=1e-30, alpha_max=1e30,
        max_backtracks=30, ek0=None, log=None):
    """Spectral projected gradient ascent (projected_spg) of the workload's
    objective over {C <= eps} with the radial projection of Eq. projection
    (Sec. 3.4), starting from P(v_start). It steps in the energy inner product
    of Eq. constraint, <a, b>_E = sum rho0 a b dx dy, in which the radial
    rescale is the exact projection onto the ball, so that its fixed points
    are the KKT points grad J = lambda grad C; with the Euclidean gradient
    instead they would be the points where grad J is parallel to v, which
    differ wherever rho0 varies."""
    def value(v):
        return objective_value(w, forward(w, v, ek0=ek0))

    def value_and_grad(v):
        J, g, _ = value_and_gradient(w, v, ek0)
        return J, g

    vs = np.asarray(v_start, dtype=np.float64)
    metric = constraint_normal(w, np.ones(vs.size)).reshape(vs.shape)
    return projected_spg(value, value_and_grad, lambda v: project(w, v, eps), v_start, iters, memory=memory,
                         armijo=armijo, alpha_min=alpha_min, alpha_max=alpha_max,
                         max_backtracks=max_backtracks, log=log, metric=metric)


# ------------------------------------- projected L-BFGS, Sec. 3.4 (Eq. projection)
def lbfgs_direction(g, pairs, gamma):
    """Two-loop recursion (Nocedal & Wright, Numerical Optimization, Alg. 7.4)
    for the ascent direction p = H g, H the limited-memory inverse-Hessian
    estimate of -J. ``pairs`` lists (s, y, rho) from oldest to newest, with
    y = -(g_new - g_old) and rho = 1 / <s, y>; a pair with rho = 0 (one that
    failed the curvature test) takes no part. The initial matrix is gamma I."""
    q = np.array(g, dtype=np.float64, copy=True)
    a = [0.0] * len(pairs)
    for j in range(len(pairs) - 1, -1, -1):
        s, y, rho = pairs[j]
        a[j] = rho * float(np.sum(s * q))
        q = q - a[j] * y
    r = gamma * q
    for j in range(len(pairs)):
        s, y, rho = pairs[j]
        b = rho * float(np.sum(y * r))
        r = r + (a[j] - b) * s
    return r


def projected_lbfgs(value, value_and_grad, proj, v_start, iters, m=10, memory=10, armijo=1e-4,
                    max_backtracks=30, normal=None, active=None, log=None):
    """Projected L-BFGS ascent with a non-monotone Armijo line search
    (Sec. 3.4), on any objective: ``value(v)`` -> J, ``value_and_grad(v)`` ->
    (J, dJ/dv), ``proj`` the radial projection P onto {C <= eps} of a
    constraint C homogeneous of degree 2, ``normal(v)`` = dC/dv and
    ``active(v)`` true when v lies on C = eps (both may be None: no
    constraint surface).

    At an iterate on the surface the search runs on it:
      - the model gradient is the gradient of J o P there,
        gh = g - (<g, v> / <n, v>) n, n = normal(v) (elsewhere gh = g);
      - the direction is made tangent to the surface,
        p <- p - (<n, p> / <n, n>) n, so that C(v + lam p) >= eps and P puts
        every trial point back on the surface.
    Iteration k, from v with model gradient gh:
      - p = H gh by ``lbfgs_direction`` over the pairs of the last m
        iterations; H0 = gamma I with gamma = <s, y> / <y, y> of the newest
        stored pair, or ||v|| / ||gh|| when none is stored; then tangent;
      - if <gh, p> <= 0 while pairs are stored, every pair is dropped and
        p = (||v|| / ||gh||) gh, then tangent (steepest-ascent restart);
      - trial points v(lam) = P(v + lam p), lam = 1, 1/2, 1/4, ...; the first
        with J(v(lam)) >= min(last ``memory`` accepted J) + armijo <gh, v(lam) - v>
        is taken (Grippo-Lampariello-Lucidi non-monotone rule). None within
        ``max_backtracks`` trials ends the run;
      - the pair (s, y) = (v_new - v, -(gh_new - gh)) is stored with
        rho = 1 / <s, y> if <s, y> > 0 and rho = 0 otherwise; the memory
        keeps the pairs of the last m iterations.
    Returns a dict with v, J, the accepted J history, per-iteration records
    and evaluation counts."""
    def on_surface(v):
        return normal is not None and active is not None and active(v)

    def model_gradient(v, g):
        if not on_surface(v):
            return g
        n = normal(v)
        return g - (float(np.sum(g * v)) / float(np.sum(n * v))) * n

    def tangent(v, p):
        if not on_surface(v):
            return p
        n = normal(v)
        return p - (float(np.sum(n * p)) / float(np.sum(n * n))) * n

    def steepest_gamma(v, g):
        return float(np.linalg.norm(v) / max(np.linalg.norm(g), 1e-300))

    def stationarity(v, g):
        # App. A: chi = ||P(v + dJ/dv) - v||_inf, with the gradient of J itself
        return float(np.max(np.abs(proj(v + g) - v))), float(np.linalg.norm(g))

    v = np.array(v_start, dtype=np.float64, copy=True)
    J, g = value_and_grad(v)
    chi0 = stationarity(v, g)
    g = model_gradient(v, g)
    evals, grads = 1, 1
    hist = [J]
    pairs = []
    records = []
    for k in range(iters):
        stored = [pr for pr in pairs if pr[2] > 0.0]
        if stored:
            s, y, _ = stored[-1]
            gamma = float(np.sum(s * y)) / float(np.sum(y * y))
        else:
            gamma = steepest_gamma(v, g)
        p = tangent(v, lbfgs_direction(g, pairs, gamma))
        restart = False
        if stored and float(np.sum(g * p)) <= 0.0:
            pairs = [(s, y, 0.0) for s, y, _ in pairs]
            p = tangent(v, steepest_gamma(v, g) * g)
            restart = True
        Jref = min(hist[-memory:])
        lam = 1.0
        accepted = False
        for _ in range(max_backtracks):
            vt = proj(v + lam * p)
            Jt = value(vt)
            evals += 1
            if Jt >= Jref + armijo * float(np.sum(g * (vt - v))):
                accepted = True
                break
            lam *= 0.5
        if not accepted:
            break
        Jn, gn = value_and_grad(vt)
        chi, gnorm = stationarity(vt, gn)
        gn = model_gradient(vt, gn)
        grads += 1
        s = vt - v
        y = -(gn - g)
        sy = float(np.sum(s * y))
        pairs.append((s, y, 1.0 / sy if sy > 0.0 else 0.0))
        if len(pairs) > m:
            pairs.pop(0)
        v, J, g = vt, Jn, gn
        hist.append(J)
        records.append({"iter": k, "J": J, "lam": lam, "gamma": gamma, "restart": restart, "sy": sy,
                        "chi": chi, "grad_norm": gnorm})
        if log is not None:
            log(records[-1])
    return {"v": v, "J": J, "history": hist, "records": records, "evals": evals, "grads": grads,
            "chi0": chi0[0], "grad_norm0": chi0[1]}


def constraint_normal(w, v):
    """dC/dv of Eq. constraint: rho0 v dx dy per perturbed component."""
    rho0, _ = base_state(w)
    dx, dy = grid_spacing(w)
    v = np.asarray(v, dtype=np.float64).reshape(w.ncomp, w.ny, w.nx)
    return rho0[None, :, None] * v * dx * dy


def lbfgs(w, v_start, eps, iters, m=10, memory=10, armijo=1e-4, max_backtracks=30, ek0=None, log=None):
    """The CNOP by projected L-BFGS (Sec. 3.4): ``projected_lbfgs`` on the
    workload's objective with the radial projection P onto {C <= eps}
    (Eq. projection), starting from P(v_start). The iterate counts as on the
    budget surface when C(v) >= eps (1 - 1e-10), i.e. P placed it there up
    to rounding."""
    def value(v):
        return objective_value(w, forward(w, v, ek0=ek0))

    def value_and_grad(v):
        J, g, _ = value_and_gradient(w, v, ek0)
        return J, g

    return projected_lbfgs(value, value_and_grad, lambda v: project(w, v, eps), project(w, v_start, eps),
                           iters, m=m, memory=memory, armijo=armijo, max_backtracks=max_backtracks,
                           normal=lambda v: constraint_normal(w, v),
                           active=lambda v: constraint(w, v) >= eps * (1.0 - 1e-10), log=log)


# ------------------------------- comparison diagnostics, Sec. 4.3 (Eqs. ke, hmix, hmix-f)
def kinetic_energy(w, U):
    """Total kinetic energy: sum over cells of e_k = rho |u|^2 / 2 = |m|^2 / (2 rho), times dx dy (Eq. ke)."""
    U = np.asarray(U, dtype=np.float64).reshape(4, w.ny, w.nx)
    dx, dy = grid_spacing(w)
    return float(np.sum(0.5 * (U[1] * U[1] + U[2] * U[2]) / U[0]) * dx * dy)


def mixing_width(w, U):
    """Eqs. hmix, hmix-f: f(y) = clip((<rho>_x - rho_l) / (rho_h - rho_l), 0, 1) and
    h_mix = integral of 4 f (1 - f) dy, the integral a midpoint sum over the rows."""
    U = np.asarray(U, dtype=np.float64).reshape(4, w.ny, w.nx)
    _, dy = grid_spacing(w)
    rho_mean = np.mean(U[0], axis=1)
    f = np.clip((rho_mean - w.rho_light) / (w.rho_heavy - w.rho_light), 0.0, 1.0)
    return float(np.sum(4.0 * f * (1.0 - f)) * dy)


def series(w, v, every):
    """KE(t) and h_mix(t) of the forward run from v, sampled at steps 0, every,
    2 every, ... and at the last step (Sec. 4.3, Figs. ek_growth, mixing_width).
    The state after k steps is the forward run replaying the first k time
    steps. Returns arrays step, t, KE, h_mix."""
    full = forward(w, v)
    dt = full["dt"]
    n = len(dt)
    steps = list(range(0, n, every))
    if steps[-1] != n:
        steps.append(n)
    out = {"step": [], "t": [], "KE": [], "h_mix": []}
    for k in steps:
        U = inject(w, v) if k == 0 else forward(w, v, dt_replay=dt[:k])["U"]
        t = 0.0
        for d in dt[:k]:
            t += d
        out["step"].append(k)
        out["t"].append(t)
        out["KE"].append(kinetic_energy(w, U))
        out["h_mix"].append(mixing_width(w, U))
    return {key: np.array(val) for key, val in out.items()}


# ------------------------------------------------- spectra, Sec. 4.2 Eq. fourier_coeff
def spectrum(vy):
    """Row y_peak of largest rms along x (ties: lowest row), its DFT u_n and the
    normalised energies E_n over the positive modes n = 1 .. nx/2."""
    vy = np.asarray(vy, dtype=np.float64)
    rms = np.sqrt(np.mean(vy * vy, axis=1))
    y_peak = int(np.argmax(rms))
    nx = vy.shape[1]
    j = np.arange(nx)
    n = np.arange(1, nx // 2 + 1)
    # plain DFT of the definition, u_n = sum_j u_j exp(-2 pi i n j / N)
    u_hat = np.array([np.sum(vy[y_peak] * np.exp(-2j * np.pi * m * j / nx)) for m in n])
    pw = np.abs(u_hat) ** 2
    return y_peak, n, pw / np.sum(pw)


def dft_matrix(n, sign=-1.0):
    """W[k, j] = exp(sign 2 pi i k j / n), the phase reduced exactly as (k j mod n)."""
    k = np.arange(n)
    return np.exp(sign * 2j * np.pi * (np.outer(k, k) % n) / n)


def spectrum2d(vy):
    """App. B: normalised two-dimensional spectral energy of a field [ny][nx]:
    F = sum_{l,j} u(x_j, y_l) exp(-2 pi i (n_x j / N_x + n_y l / N_y)) and
    E[n_y, n_x] = |F|^2 / sum |F|^2 over all modes (reading: the DFT runs over
    the whole grid, and the energies are normalised over every mode)."""
    vy = np.asarray(vy, dtype=np.float64)
    ny, nx = vy.shape
    F = dft_matrix(ny) @ vy @ dft_matrix(nx).T
    pw = np.abs(F) ** 2
    return pw / np.sum(pw)


def power_reconstruct(w, v, eps, frac=0.9):
    """App. B: the reconstruction that keeps the two-dimensional Fourier modes
    holding `frac` of the spectral energy of u_y. Reading: modes are ranked in
    conjugate pairs {(n_x, n_y), (-n_x, -n_y)} by the pair's energy, so the
    field stays real; the pairs are kept from the largest down until the kept
    energy reaches frac of the total, together with every pair whose energy
    ties the last one kept. That mode set is applied to every perturbed
    component, the inverse DFT's real part is taken and the result rescaled to
    C = eps. Returns (field, number of kept modes)."""
    v = np.asarray(v, dtype=np.float64).reshape(w.ncomp, w.ny, w.nx)
    ny, nx = w.ny, w.nx
    E = spectrum2d(v[-1])
    ky, kx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    cy, cx = (-ky) % ny, (-kx) % nx
    pair = np.where((cy == ky) & (cx == kx), E, E + E[cy, cx])
    rep = (ky * nx + kx) <= (cy * nx + cx)  # one representative per pair
    vals = np.sort(pair[rep])[::-1]
    csum = np.cumsum(vals)
    tau = vals[int(np.nonzero(csum >= frac * csum[-1])[0][0])]
    keep = pair >= tau
    Wy, Wx = dft_matrix(ny), dft_matrix(nx)
    iWy, iWx = dft_matrix(ny, +1.0) / ny, dft_matrix(nx, +1.0) / nx
    out = np.empty_like(v)
    for c in range(w.ncomp):
        F = Wy @ v[c] @ Wx.T
        out[c] = np.real(iWy @ (F * keep) @ iWx.T)
    return scale_to_budget(w, out, eps), int(np.sum(keep))


def five_modes(w, v, eps, count=5):
    """Sec. 3.5 / 4.2: keep the ``count`` positive horizontal modes with the
    largest E_n at y_peak (ties: lower n), apply that index set to every row
    and component, and rescale to C = eps."""
    v = np.asarray(v, dtype=np.float64).reshape(w.ncomp, w.ny, w.nx)
    _, n, E = spectrum(v[-1])
    order = np.argsort(-E, kind="stable")[:count]
    keep = set(int(n[o]) for o in order)
    nx = w.nx
    mask = np.zeros(nx, dtype=bool)
    for m in keep:
        mask[m % nx] = True
        mask[(-m) % nx] = True
    out = np.real(np.fft.ifft(np.fft.fft(v, axis=2) * mask[None, None, :], axis=2))
    return scale_to_budget(w, out, eps), sorted(keep)
