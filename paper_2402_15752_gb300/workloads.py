"""Seeded synthetic workloads: parameter sets and signed-distance fields.

This module only generates inputs.  It holds none of the method's arithmetic
(no relaxation times, no tanh profile, no equilibria): it returns the physical
parameters, in lattice units (dx = dt = 1), and the signed-distance field l(x)
of the initial interface (Eq. 2 of arXiv 2402.15752 turns it into phi on each
side of the comparison separately).  Both the CUDA path and the CPU oracle are
fed from here.

Random draws use numpy's PCG64 with seed 2402157520 + workload index.
Node coordinates are x = i, y = j (not cell centres).

Workloads (all in lattice units):

* ``droplet64``   -- static droplet, 64x64 periodic, R = 16 at (32, 32),
  W = 4, density and viscosity ratio 1, D1/D2 = 10, K_eq = 2, scalar 1 inside
  and 0 outside, 1000 steps.
* ``planar1024``  -- planar interface at x = 512 in a 1024x8 channel with
  bounce-back walls at the x ends and periodic y, D1/D2 = 100, K_eq = 3,
  20000 steps; the closed-form erfc solution applies in the bulk.
* ``bubble1024x2048`` -- rising bubble (phase 2) of radius 128 at (512, 512)
  in a 1024x2048 wall-bounded box, density ratio 1000 (rho 1 / 1e-3),
  viscosity ratio 100 (mu 0.1 / 1e-3, i.e. nu 0.1 liquid / 1.0 gas), sigma 0.01,
  mu = mu_lin(phi) exp(-beta T) with beta ~ U[0, 2], buoyancy g = 1e-6,
  T = c1 + c2 initialised as 1 - phi (tanh across the interface).
* ``batched`` -- 256 independent droplets for the batched runner: square
  periodic grids of side drawn uniformly from {64, 96, ..., 512}, radius
  U[0.15, 0.35] * side, centre jittered by U[-5, 5] nodes, density ratio
  U[1, 100], K_eq U[0.5, 5], D1/D2 U[1, 100]; 2000 steps.
* ``droplets8192`` -- 1 to 4 droplets in an 8192x8192 periodic box, radii
  U[10, 60] * 32, density ratio U[1, 100] (single-case scaling run).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2402157520
WORKLOAD_INDEX = {"droplet64": 0, "planar1024": 1, "bubble1024x2048": 2,
                  "batched": 3, "droplets8192": 4}


def rng(index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(index)))


# ---------------------------------------------------------------- geometry --
def grid(nx: int, ny: int):
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                       indexing="ij")
    return x, y


def sdf_droplet(nx, ny, xc, yc, R):
    """l = R - |x - x_c| : phase 1 inside the circle."""
    x, y = grid(nx, ny)
    return R - np.hypot(x - xc, y - yc)


def sdf_bubble(nx, ny, xc, yc, R):
    """l = |x - x_c| - R : phase 2 inside the circle."""
    return -sdf_droplet(nx, ny, xc, yc, R)


def sdf_droplets(nx, ny, centres, radii, periodic=True):
    """Union of droplets (max of the individual signed distances); periodic images."""
    x, y = grid(nx, ny)
    out = np.full((ny, nx), -np.inf)
    for (xc, yc), R in zip(centres, radii):
        dx = x - xc
        dy = y - yc
        if periodic:
            dx = dx - nx * np.round(dx / nx)
            dy = dy - ny * np.round(dy / ny)
        out = np.maximum(out, R - np.hypot(dx, dy))
    return out


def sdf_planar_x(nx, ny, x0):
    """l = x0 - x : phase 1 on the left of x = x0."""
    x, _ = grid(nx, ny)
    return x0 - x


def sdf_planar_y(nx, ny, y0):
    """l = y0 - y : phase 1 below y = y0."""
    _, y = grid(nx, ny)
    return y0 - y


# --------------------------------------------------------------- workloads --
BASE = dict(wall_x=0, wall_y=0, scalar_q=5, W=4.0, M=0.01, sigma=0.0,
            rho1=1.0, rho2=1.0, mu1=0.1, mu2=0.1, D1=0.1, D2=0.1, Keq=1.0, A=0.1,
            gx=0.0, gy=0.0, g_rho_ref=0.0, Fx=0.0, Fy=0.0, visc_model=0, visc_beta=0.0,
            scalar_model=0, grad_scheme=0)


@dataclass
class Workload:
    name: str
    params: dict
    sdf: np.ndarray
    c1_tilde: float
    c2_tilde: float
    steps: int
    info: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return int(self.params["nx"]) * int(self.params["ny"])


def droplet64(nx=64, ny=64, R=16.0, steps=1000, **over) -> Workload:
    p = dict(BASE, nx=nx, ny=ny, sigma=0.01, rho1=1.0, rho2=1.0, mu1=0.1, mu2=0.1,
             D1=0.1, D2=0.01, Keq=2.0)
    p.update(over)
    return Workload("droplet64", p, sdf_droplet(nx, ny, nx / 2, ny / 2, R), 1.0, 0.0, steps,
                    {"R": R})


def planar1024(nx=1024, ny=8, x0=None, steps=20000, **over) -> Workload:
    x0 = nx / 2 if x0 is None else x0
    p = dict(BASE, nx=nx, ny=ny, wall_x=1, wall_y=0, sigma=0.01, rho1=1.0, rho2=1.0,
             mu1=0.1, mu2=0.1, D1=0.1, D2=0.001, Keq=3.0)
    p.update(over)
    return Workload("planar1024", p, sdf_planar_x(nx, ny, x0), 1.0, 0.0, steps, {"x0": x0})


def bubble1024x2048(nx=1024, ny=2048, R=None, steps=10000, **over) -> Workload:
    """Rising bubble; smaller boxes keep the geometry in proportion.

    Defined for 10 000 steps.  At full size it goes non-finite between 13 000
    and 14 000 steps, in FP64 and FP32 alike: c1 + c2 builds up on the gas side
    of the bubble's lower interface (to 6.6 by then), and mu_lin exp(-beta T)
    takes tau_g there toward 1/2.  visc_beta=0 (or visc_model=0) runs 30 000
    steps."""
    R = 128.0 * nx / 1024 if R is None else R
    beta = float(rng(WORKLOAD_INDEX["bubble1024x2048"]).uniform(0.0, 2.0))
    p = dict(BASE, nx=nx, ny=ny, wall_x=1, wall_y=1, sigma=0.01,
             rho1=1.0, rho2=1e-3, mu1=0.1, mu2=1e-3,
             D1=0.01, D2=0.05, Keq=1.0 / 33.0,
             gx=0.0, gy=-1e-6, g_rho_ref=1.0, visc_model=2, visc_beta=beta)
    p.update(over)
    return Workload("bubble1024x2048", p, sdf_bubble(nx, ny, nx / 2, ny / 4, R), 0.0, 1.0,
                    steps, {"beta": beta, "R": R})


def droplets8192(nx=8192, ny=8192, steps=1000, **over) -> Workload:
    g = rng(WORKLOAD_INDEX["droplets8192"])
    scale = nx / 256.0
    n = int(g.integers(1, 5))
    radii = g.uniform(10.0, 60.0, size=n) * scale
    centres = g.uniform(0.0, 1.0, size=(n, 2)) * np.array([nx, ny])
    ratio = float(g.uniform(1.0, 100.0))
    p = dict(BASE, nx=nx, ny=ny, sigma=0.01, rho1=1.0, rho2=1.0 / ratio,
             mu1=0.1, mu2=0.1 / ratio, D1=0.1, D2=0.01, Keq=2.0)
    p.update(over)
    return Workload("droplets8192", p, sdf_droplets(nx, ny, centres, radii), 1.0, 0.0, steps,
                    {"radii": radii.tolist(), "centres": centres.tolist(), "rho_ratio": ratio})


def layered_poiseuille(nx=15, ny=150, G=1e-6, D=0.5, steps=200000, **over) -> Workload:
    """Layered two-phase channel flow with concentration-dependent viscosity
    (Sec. IV C 2): walls at both y ends (half-way bounce-back), periodic x,
    phase 1 (rho 10, mu 1) below the centre line, phase 2 (rho 1, mu 0.1) above,
    log mu = c1 log mu1 + c2 log mu2 (Eq. 48), K_eq = 1, D1 = D2, c1 = phi,
    c2 = 0, driven by the body force (G, 0)."""
    p = dict(BASE, nx=nx, ny=ny, wall_x=0, wall_y=1, sigma=0.01, rho1=10.0, rho2=1.0,
             mu1=1.0, mu2=0.1, D1=D, D2=D, Keq=1.0, Fx=G, visc_model=1)
    p.update(over)
    return Workload("layered_poiseuille", p, sdf_planar_y(nx, ny, (ny - 1) / 2.0), 1.0, 0.0, steps,
                    {"G": G})


def batched(n=256, sides=tuple(range(64, 513, 32)), steps=2000) -> list:
    """n independent droplet cases of uneven sizes (one Workload each)."""
    g = rng(WORKLOAD_INDEX["batched"])
    out = []
    for k in range(n):
        side = int(g.choice(sides))
        R = float(g.uniform(0.15, 0.35)) * side
        xc, yc = side / 2 + g.uniform(-5.0, 5.0, size=2)
        ratio = float(g.uniform(1.0, 100.0))
        K = float(g.uniform(0.5, 5.0))
        dratio = float(g.uniform(1.0, 100.0))
        # droplet (phase 1) the heavier phase; kinematic viscosity 0.1 in both
        p = dict(BASE, nx=side, ny=side, sigma=0.01, rho1=1.0, rho2=1.0 / ratio,
                 mu1=0.1, mu2=0.1 / ratio, D1=0.1, D2=0.1 / dratio, Keq=K)
        out.append(Workload("batched[%d]" % k, p, sdf_droplet(side, side, xc, yc, R), 1.0, 0.0,
                            steps, {"R": R, "centre": (float(xc), float(yc)), "rho_ratio": ratio,
                                    "Keq": K, "D_ratio": dratio}))
    return out


WORKLOADS = {"droplet64": droplet64, "planar1024": planar1024,
             "bubble1024x2048": bubble1024x2048, "droplets8192": droplets8192}


def get(name: str, **kw) -> Workload:
    return WORKLOADS[name](**kw)
