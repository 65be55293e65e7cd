"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds workload descriptions (plain parameter values) and seeded
random draws only. It contains none of the method's arithmetic: no base state,
no energy functional, no scaling to a budget, no envelope. Both the CPU oracle
and the CUDA path receive the arrays produced here as inputs.

Random numbers come from NumPy's ``Generator(PCG64(seed))`` standard normal
draws, so every array is reproducible from its seed on any machine.
"""
from __future__ import annotations

import dataclasses
import numpy as np

# Boundary, limiter, perturbation, objective and precision enums. The values
# match the C-ABI's enums; they are plain labels, not arithmetic.
BC_REFLECT, BC_HYDROSTATIC = 0, 1
LIM_MINMOD, LIM_MC, LIM_NONE = 0, 1, 2
PERT_VY, PERT_VXVY = 1, 2          # number of perturbed velocity components
OBJ_KE, OBJ_EK_ANOMALY_L2 = 0, 1
FP64, FP32_STATE = 0, 1
FLUX_HLLC, FLUX_HLL, FLUX_HYBRID = 0, 1, 2


@dataclasses.dataclass
class Workload:
    """One Rayleigh-Taylor problem: grid, gas, base state, boundary, scheme, horizon."""
    nx: int = 64
    ny: int = 192
    x0: float = -0.25
    x1: float = 0.25
    y0: float = -0.75
    y1: float = 0.75
    gamma: float = 1.4
    g_y: float = -0.1
    rho_heavy: float = 2.0
    rho_light: float = 1.0
    y_int: float = 0.0
    h_s: float = 0.01
    p_ref: float = 2.5
    y_ref: float = 0.0
    bc_y: int = BC_REFLECT
    limiter: int = LIM_MINMOD
    cfl: float = 0.4
    T: float = 2.0
    nsteps: int = 0                 # > 0: fixed step count, T ignored
    ncomp: int = PERT_VXVY
    objective: int = OBJ_KE
    flux: int = FLUX_HLLC
    flux_theta: float = 2.0         # hybrid: HLL where the face pressure ratio exceeds this

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def rt_box(nx: int, ny: int, **kw) -> Workload:
    """Athena-style RT box [-0.25,0.25]x[-0.75,0.75]: gamma 1.4, g_y -0.1,
    heavy (2) over light (1) fluid across a tanh interface of width 0.01 at
    y = 0, p = 2.5 at y = 0, periodic x, reflecting y."""
    return Workload(nx=nx, ny=ny, **kw)


def small_fixed_steps() -> Workload:
    """64x192 RT box, 500 CFL-0.4 steps, perturbation (vx, vy)."""
    return rt_box(64, 192, nsteps=500)


def single_256() -> Workload:
    """256x768 RT box to horizon T = 2.0."""
    return rt_box(256, 768, T=2.0)


def paper_unit_square(n: int, t_star: float = 2.0) -> Workload:
    """Unit-square configuration of the paper's parameter table: gamma 5/3,
    g = 1, rho 2 over 1 at y = 0.5 with h_s = 0.02, p(y = 1) = rho_h g L = 2,
    hydrostatic y boundary, u_y-only perturbation, squared e_k anomaly."""
    return Workload(nx=n, ny=n, x0=0.0, x1=1.0, y0=0.0, y1=1.0,
                    gamma=5.0 / 3.0, g_y=-1.0, rho_heavy=2.0, rho_light=1.0,
                    y_int=0.5, h_s=0.02, p_ref=2.0, y_ref=1.0,
                    bc_y=BC_HYDROSTATIC, T=t_star, ncomp=PERT_VY,
                    objective=OBJ_EK_ANOMALY_L2)


def gaussian_field(seed: int, ncomp: int, ny: int, nx: int) -> np.ndarray:
    """i.i.d. N(0,1) field of shape (ncomp, ny, nx), float64, C-contiguous."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.ascontiguousarray(rng.standard_normal((ncomp, ny, nx)))


def gaussian_batch(seeds, ncomp: int, ny: int, nx: int) -> np.ndarray:
    """Stack of ``gaussian_field`` draws, shape (len(seeds), ncomp, ny, nx)."""
    return np.stack([gaussian_field(s, ncomp, ny, nx) for s in seeds])


def directions(seed0: int, count: int, ncomp: int, ny: int, nx: int) -> np.ndarray:
    """``count`` seeded N(0,1) directions (seeds seed0 .. seed0+count-1)."""
    return gaussian_batch(range(seed0, seed0 + count), ncomp, ny, nx)


def uniform_cells(seed: int, shape, lo: float, hi: float) -> np.ndarray:
    """Seeded uniform values in [lo, hi), float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=shape)
