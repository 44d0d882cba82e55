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


def own_max_errors(got: dict, want: dict, names=MAIN_FIELDS) -> dict:
    """Per field: max |gpu - oracle| / max |oracle| (the relative max error in
    its plain form, each field against its own maximum)."""
    return {k: float(np.abs(np.asarray(got[k], dtype=np.float64) - want[k]).max()
                     / max(float(np.abs(want[k]).max()), 1e-300)) for k in names}


# A field is compared against its own maximum unless that maximum is below this
# fraction of its natural scale.  The fields below it are the ones whose exact
# (continuum) value vanishes: the velocity of a flat interface or a static
# droplet at rest (spurious currents, 1-3 % of the flow-population scale), a
# velocity component that vanishes by symmetry, the pressure of a Poiseuille
# channel.  What FP32 storage of the populations can promise for a moment of
# them is a fraction of the populations' own scale (measured: at most 5.3e-7 of
# the natural scale after 1000 steps in every case); against a field that is
# itself below 5 % of that scale, 1e-5 of its own maximum asks for more digits
# than the stored populations carry.  Those fields are held to the tolerance
# against the natural scale, and their own-max error is printed.
OWN_MAX_FLOOR = 0.05


def assert_parity(got, want, tol, names=MAIN_FIELDS, label=""):
    """Relative max error per field at most `tol`, measured against the field's
    own maximum wherever that is at least OWN_MAX_FLOOR of its natural scale,
    and against the natural scale always.  Both forms are printed."""
    errs = rel_max_errors(got, want, names)
    own = own_max_errors(got, want, names)
    sc = field_scales(want)
    vanishing = {k for k in names if float(np.abs(want[k]).max()) < OWN_MAX_FLOOR * sc[k]}
    print("\n%s: field  own-max  natural-scale" % label)
    for k in names:
        print("  %-4s %.2e%s  %.2e" % (k, own[k], " (vanishing)" if k in vanishing else "", errs[k]))
    bad = {k: v for k, v in errs.items() if not v <= tol}
    bad.update({"%s(own max)" % k: own[k] for k in names if k not in vanishing and not own[k] <= tol})
    assert not bad, "%s rel-max errors above %.1e: %s (all: %s, own max: %s)" % (label, tol, bad, errs, own)
    return errs
