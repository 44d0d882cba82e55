"""Shared helpers of the GPU parity tests (import only from tests)."""
import numpy as np

import oracle
from paper_2402_15752_gb300 import Simulation

MAIN_FIELDS = ("phi", "ux", "uy", "p", "c1", "c2")


def field_scales(want: dict) -> dict:
    """Natural scale of each field of the oracle's solution.

    * phi, rho, mu: their maximum magnitude.
    * c1, c2: the maximum total scalar c1 + c2 (one scalar split over two phases).
    * ux, uy, p: u and p are the first and zeroth moments of the same flow
      populations g_i (Eq. 32), whose magnitude in the dense phase is set by
      both |p| / c_s and rho |u|.  Velocity is measured against
      max(max speed, max|p| / (rho_max c_s)) and pressure against
      max(max|p|, rho_max c_s max speed).  A velocity component that vanishes
      by symmetry, or a pressure that is uniform, is then not divided by its
      own roundoff.
    """
    cs = 1.0 / np.sqrt(3.0)
    speed = float(np.sqrt(want["ux"] ** 2 + want["uy"] ** 2).max())
    pmax = float(np.abs(want["p"]).max())
    rho_max = float(np.abs(want["rho"]).max())
    total = float(np.abs(want["c1"] + want["c2"]).max())
    sc = {k: float(np.abs(v).max()) for k, v in want.items()}
    u_scale = max(speed, pmax / (rho_max * cs))
    sc.update(ux=u_scale, uy=u_scale, p=max(pmax, rho_max * cs * speed), c1=total, c2=total)
    return {k: max(v, 1e-30) for k, v in sc.items()}


def rel_max_errors(got: dict, want: dict, names=MAIN_FIELDS) -> dict:
    """Per field: max |gpu - oracle| / (natural scale of the field)."""
    sc = field_scales(want)
    return {k: float(np.abs(np.asarray(got[k], dtype=np.float64) - want[k]).max() / sc[k])
            for k in names}


def run_oracle(params, init, steps):
    s = oracle.OracleSim(params)
    _apply_init(s, init)
    s.step(steps)
    return s


def run_gpu(params, init, steps, precision, chunks=None):
    sim = Simulation(params, precision=precision)
    _apply_init(sim, init)
    if chunks:
        for c in chunks:
            sim.step(c)
    else:
        sim.step(steps)
    return sim


def _apply_init(sim, init):
    kind = init[0]
    if kind == "sdf":
        sim.init(init[1], init[2], init[3])
    else:
        sim.init_fields(init[1], init[2], init[3])


def assert_parity(got, want, tol, names=MAIN_FIELDS, label=""):
    errs = rel_max_errors(got, want, names)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, "%s rel-max errors above %.1e: %s (all: %s)" % (label, tol, bad, errs)
    return errs
