"""Seeded synthetic workloads for the sphere-in-channel problem.

This module holds only problem set-ups and random inputs: box, boundary
types, sphere, rheology parameters and the seeded initial noise.  It holds
none of the method's arithmetic, so both the CUDA path and its test oracle may
draw their inputs from it.

Units follow the paper's sphere study (Sec. "Sphere moving through Bingham
fluid"): body diameter D = 2r and inflow speed U = 1 are the reference scales,
so the Bingham number is Bi = tau0 * D / (mu * U).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

INFLOW, OUTFLOW, SLIP, NOSLIP = 0, 1, 2, 3
NEWTONIAN, BINGHAM, HB, POWERLAW, SMD = 0, 1, 2, 3, 4
CHANNEL_BC = (SLIP, SLIP, SLIP, SLIP, INFLOW, OUTFLOW)


@dataclass
class Workload:
    name: str
    n: int
    radius: float
    centre: tuple = (0.5, 0.5, 0.5)
    rho: float = 1.0
    mu: float = 1.0
    tau0: float = 1.0
    m: float = 1e3
    n_flow: float = 1.0
    model: int = BINGHAM
    cfl: float = 0.5
    steps: int = 10
    seed: int = 0
    noise: float = 1e-3
    u_in: tuple = (0.0, 0.0, 1.0)
    bc: tuple = CHANNEL_BC
    extra: dict = field(default_factory=dict)

    @property
    def h(self) -> float:
        return 1.0 / self.n

    @property
    def bingham(self) -> float:
        """Bi = tau0 D / (mu U) with D = 2r, U = |u_in|."""
        U = float(np.linalg.norm(self.u_in))
        return self.tau0 * 2.0 * self.radius / (self.mu * U)

    @property
    def cells(self) -> int:
        return self.n ** 3


def tau0_for_bingham(bi: float, radius: float, mu: float = 1.0, U: float = 1.0) -> float:
    return bi * mu * U / (2.0 * radius)


def sphere_channel_32() -> Workload:
    """32^3 box, sphere r = 0.125 at the centre, tau_y = 1, m = 1e3, 10 steps."""
    return Workload("sphere_channel_32_fp64", n=32, radius=0.125, tau0=1.0, m=1e3, steps=10)


def sphere_channel_128(bi: float = 1.0, herschel_bulkley: bool = False) -> Workload:
    """128^3 box, sphere r = 0.125; Bi in {0, 1, 10}, or HB n = 0.5, tau0 = 1."""
    if herschel_bulkley:
        return Workload("sphere_channel_128_hb", n=128, radius=0.125, tau0=1.0, m=1e3,
                        n_flow=0.5, model=HB, steps=20)
    model = NEWTONIAN if bi == 0 else BINGHAM
    return Workload(f"sphere_channel_128_bi{bi:g}", n=128, radius=0.125,
                    tau0=tau0_for_bingham(bi, 0.125), m=1e3, model=model, steps=20)


def sphere_channel_256() -> Workload:
    """256^3 box, sphere r = 0.1, Bi = 10, m = 1e4, 50 steps."""
    return Workload("sphere_channel_256_bi10", n=256, radius=0.1,
                    tau0=tau0_for_bingham(10.0, 0.1), m=1e4, steps=50)


def batched_sweep(seed: int = 0, count: int = 64) -> list:
    """Independent instances: N from {48, 64, 96}, r ~ U[0.08, 0.2], centre
    jittered by U[-0.05, 0.05] per axis, log10 Bi ~ U[-1, 2], m = 1e3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for q in range(count):
        n = int(rng.choice([48, 64, 96]))
        r = float(rng.uniform(0.08, 0.2))
        c = tuple(float(v) for v in 0.5 + rng.uniform(-0.05, 0.05, size=3))
        bi = float(10.0 ** rng.uniform(-1.0, 2.0))
        out.append(Workload(f"sweep_{q}", n=n, radius=r, centre=c,
                            tau0=tau0_for_bingham(bi, r), m=1e3, steps=20, seed=seed + 1 + q))
    return out


def initial_velocity(w: Workload) -> np.ndarray:
    """Inflow value plus i.i.d. U[-noise, noise] per component and cell,
    shape (3, n, n, n) in (component, z, y, x) order.  Covered cells are
    zeroed by the consumer, which owns the geometry."""
    rng = np.random.Generator(np.random.PCG64(w.seed))
    u = rng.uniform(-w.noise, w.noise, size=(3, w.n, w.n, w.n))
    for q in range(3):
        u[q] += w.u_in[q]
    return u


def body_force(w: Workload, sigma: float = 0.1) -> np.ndarray:
    """i.i.d. N(0, sigma^2) per component and cell, shape (3, n, n, n)."""
    rng = np.random.Generator(np.random.PCG64(w.seed + 1000))
    return rng.normal(0.0, sigma, size=(3, w.n, w.n, w.n))


def with_steps(w: Workload, steps: int) -> Workload:
    return replace(w, steps=steps)


# ---------------------------------------------------------------------------
# Taylor-Green vortex (Sec. "Spatio-temporal convergence study: Taylor-Green
# vortices", Eq. taylor-green): unit box in x and y, rho = U = L = 1,
# mu = 1 / Re.  The paper runs it with periodic sides; the same solution also
# satisfies slip walls at x, y in {0, 1} exactly (u_n = 0 and zero tangential
# stress there), and slip walls in z with a field uniform in z, so the box
# here has slip walls on all six sides.
# ---------------------------------------------------------------------------
TG_BC = (SLIP, SLIP, SLIP, SLIP, SLIP, SLIP)


def taylor_green(x, y, t, re=100.0):
    """(u, v, p) of Eq. taylor-green at points (x, y) and time t."""
    f = np.exp(-8.0 * np.pi ** 2 * t / re)
    u = np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) * f
    v = -np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y) * f
    p = 0.25 * (np.cos(4 * np.pi * x) + np.cos(4 * np.pi * y)) * f * f
    return u, v, p


def taylor_green_depth(n):
    """Cells in z: 8, or n/8 from 128 on, so that the multigrid hierarchies
    still coarsen to a small bottom level."""
    return max(8, n // 8)


def taylor_green_grid(n, nz=None):
    """Cells (n, n, nz) of size 1/n: the unit square in x, y, nz cells deep."""
    return (n, n, nz or taylor_green_depth(n)), 1.0 / n


def taylor_green_velocity(n, nz=None, t=0.0, re=100.0):
    """Cell-centred (u, v, w), shape (3, nz, n, n), at time t."""
    nz = nz or taylor_green_depth(n)
    c = (np.arange(n) + 0.5) / n
    Y, X = np.meshgrid(c, c, indexing="ij")
    u, v, _ = taylor_green(X, Y, t, re)
    out = np.zeros((3, nz, n, n))
    out[0] = u[None]
    out[1] = v[None]
    return out


# ---------------------------------------------------------------------------
# The paper's sphere set-up (Sec. "Sphere moving through Bingham fluid"):
# box [0, 4D] x [0, 4D] x [0, 6D] with u = U e_z on every side (the sphere
# falls at U through fluid at rest), sphere of diameter D at the centre.
# ---------------------------------------------------------------------------
def sphere_box(cells_per_d=16, bi=1.0, m=1e3, D=0.25):
    n = (4 * cells_per_d, 4 * cells_per_d, 6 * cells_per_d)
    r = 0.5 * D
    return Workload(f"sphere_box_{cells_per_d}perD_bi{bi:g}", n=n[0], radius=r, centre=(2 * D, 2 * D, 3 * D),
                    tau0=tau0_for_bingham(bi, r), m=m, model=BINGHAM if bi > 0 else NEWTONIAN, noise=0.0,
                    bc=(INFLOW,) * 6, extra={"shape": n, "h": D / cells_per_d})


# The paper's non-trivial body (Sec. "Non-trivial particle shape"): the
# union of a sphere of diameter D centred at (1.8, 1.8, 2.8) D and the cube
# with opposite corners (1.85, 1.85, 2.85) D and (2.5, 2.5, 3.5) D, in the
# sphere box [0, 4D]^2 x [0, 6D] with u = U e_z on every side.
SPHERE_CUBE_D = ((1.8, 1.8, 2.8), 0.5, (1.85, 1.85, 2.85), (2.5, 2.5, 3.5))


def sphere_cube_bodies(D=0.25):
    """(sphere (cx, cy, cz, r), cube (lo..., hi...)) in box units for diameter D."""
    c, r, lo, hi = SPHERE_CUBE_D
    return (tuple(D * v for v in c) + (D * r,), tuple(D * v for v in lo) + tuple(D * v for v in hi))


def sphere_box_grid(cells_per_d, D=0.25):
    """Cells (4N, 4N, 6N) of size D/N for N cells per diameter."""
    n = cells_per_d
    return (4 * n, 4 * n, 6 * n), D / n
