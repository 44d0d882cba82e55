"""16-bit population storage (bfloat16 / IEEE half, FP32 arithmetic) against
the FP64 oracle, the erfc closed form and the FP32 path, field by field.

Every stored population is rounded stochastically to the 16-bit grid, whose
spacing is 2u relative (u = 2^-8 for bfloat16, 2^-11 for half), so each step
adds zero-mean noise of up to 2u relative to every stored value.  Each is
stored as its offset from a base of the node that wrote it: f_i - b_i phi_w,
g_i - 3 b_i p_w (3 (b_0 - 1) p_w for i = 0; in half scaled by 2^10) and
h_k,i - bq_i c_k,w, with phi_w, p_w in FP32 and c_k,w rounded to half.
The bounds below are about twice the errors measured on these cases (printed
with -s); they state the accuracy of each storage, field by field.
"""
import math

import numpy as np
import pytest

from paper_2402_15752_gb300 import workloads as wl

from _parity import MAIN_FIELDS, field_scales, rel_max_errors, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

U = {"bf16": 2.0 ** -8, "fp16": 2.0 ** -11}  # unit roundoff of the stored format
STORAGES = ("bf16", "fp16")


def _report(label, errs):
    print("\n%-28s " % label + " ".join("%s=%.2e" % (k, v) for k, v in errs.items()))


# ------------------------------------------------------------ initial state --
@pytest.mark.parametrize("storage", STORAGES)
def test_initial_phase_field_is_within_one_rounding(storage):
    """Right after init phi is the sum of the stored populations: the rest
    population takes what the rounded moving ones leave of phi, so only its own
    rounding (of a value near (w_0 - b_0) phi, 1e-6) and the FP32 sums reach
    phi; the bound below, u w_0 / 2 + 1e-6, is the older offset encoding's."""
    w = wl.droplet64(nx=70, ny=45, R=12.0)
    sim = run_gpu(w.params, ("sdf", w.sdf, 1.0, 0.0), 0, storage)
    got = sim.fields(names=("phi", "c1", "c2"))
    phi0 = 0.5 + 0.5 * np.tanh(2.0 * w.sdf / w.params["W"])
    bound = U[storage] * (4.0 / 9.0) / 2.0 + 1e-6
    assert np.abs(got["phi"] - phi0).max() <= bound
    # c1 + c2 is the plain sum of 2 x 5 stored h values, each within u of w_i c
    c_err = np.abs((got["c1"] + got["c2"]) - phi0).max()
    assert c_err <= 2 * U[storage] + 1e-6


# ------------------------------------- planar interface, 1024 x 8, 20000 steps --
_PLANAR = {}


def _planar_oracle():
    """FP64 oracle of the planar case.  The initial state and the boundaries
    do not depend on y (periodic in y), so every row of the 1024 x 8 channel
    evolves like the single row of a 1024 x 1 channel; the oracle runs that."""
    if "oracle" not in _PLANAR:
        w = wl.planar1024(ny=1)
        _PLANAR["oracle"] = run_oracle(w.params, ("sdf", w.sdf, 1.0, 0.0), w.steps).fields()
    return _PLANAR["oracle"]


def _erfc_errors(f, p, steps):
    """max |c1/phi - exact| on the phase-1 side and |c2/(1-phi) - exact| on the
    phase-2 side, 3W away from the interface: two semi-infinite phases with a
    Henry jump c1 = K c2 (Eqs. 8, 9, 12)."""
    nx = f["phi"].shape[1]
    x0, D1, D2, K = nx / 2, p["D1"], p["D2"], p["Keq"]
    r = math.sqrt(D2 / D1)
    worst = 0.0
    for row in range(f["phi"].shape[0]):
        phi, c1, c2 = f["phi"][row], f["c1"][row], f["c2"][row]
        for i in range(nx):
            d = i - x0
            if d < -3 * p["W"]:
                exact = 1 - r / (K + r) * math.erfc((x0 - i) / (2 * math.sqrt(D1 * steps)))
                worst = max(worst, abs(c1[i] / phi[i] - exact))
            elif d > 3 * p["W"]:
                exact = 1 / (K + r) * math.erfc((i - x0) / (2 * math.sqrt(D2 * steps)))
                worst = max(worst, abs(c2[i] / (1 - phi[i]) - exact))
    return worst


# Bounds on each field's max error relative to its natural scale: about twice
# the measured error.  FP32 is here at 20x the step count of the 1e-5 parity
# cases; its error grows with the steps.
PLANAR_TOL = {
    "fp32": dict(phi=1.5e-4, c1=1.5e-4, c2=1.5e-4, rho=1.5e-4, mu=1.5e-4, erfc=3e-3),
    "bf16": dict(phi=5e-4, c1=7e-4, c2=5e-4, rho=1e-6, mu=1e-6, erfc=6e-3),
    "fp16": dict(phi=6e-5, c1=3e-4, c2=1e-4, rho=1e-6, mu=1e-6, erfc=6e-3),
}


@pytest.mark.parametrize("storage", ["fp32", "bf16", "fp16"])
def test_planar_interface_1024x8_per_storage(storage):
    w = wl.planar1024()  # 1024 x 8, x walls, D1/D2 = 100, K = 3, 20000 steps
    want_row = _planar_oracle()
    want = {k: np.repeat(v, 8, axis=0) for k, v in want_row.items()}
    sim = run_gpu(w.params, ("sdf", w.sdf, 1.0, 0.0), w.steps, storage)
    got = sim.fields()
    errs = rel_max_errors(got, want, MAIN_FIELDS + ("rho", "mu"))
    e_exact = _erfc_errors(got, w.params, w.steps)
    e_exact_oracle = _erfc_errors(want_row, w.params, w.steps)
    flow = {k: float(np.abs(got[k]).max()) for k in ("ux", "uy", "p")}
    _report("planar1024x8/%s" % storage, dict(errs, erfc=e_exact, erfc_oracle=e_exact_oracle))
    _report("planar1024x8/%s |flow|" % storage, flow)
    tol = PLANAR_TOL[storage]
    for k in ("phi", "c1", "c2", "rho", "mu"):
        assert errs[k] <= tol[k], (k, errs[k], tol[k])
    # no flow in the exact solution: what remains is rounding noise of the stored g
    for k, v in flow.items():
        assert v <= 1e-3, (k, v)
    assert e_exact <= tol["erfc"]


# ------------------------------------------------ droplet and bubble vs oracle --
def _droplet():
    w = wl.droplet64()
    return w.params, ("sdf", w.sdf, w.c1_tilde, w.c2_tilde), 1000


def _bubble_small():
    w = wl.bubble1024x2048(nx=96, ny=192)
    return w.params, ("sdf", w.sdf, w.c1_tilde, w.c2_tilde), 100


def _q9_walls():
    # D2Q9 scalar lattices (nine h bases per node), y walls, Eq. (48)
    # viscosity, body forces, a 40-wide ragged row
    w = wl.droplet64(nx=40, ny=33, R=9.0, scalar_q=9, visc_model=1, mu1=0.2, mu2=0.05, rho2=0.5,
                     Fx=2e-6, gy=-1e-6, g_rho_ref=0.75, wall_y=1)
    return w.params, ("sdf", w.sdf, 0.8, 0.4), 300


CASE_TOL = {  # about twice the measured error, relative to each field's natural scale
    "droplet64": {
        "bf16": dict(phi=8e-4, ux=0.035, uy=0.035, p=0.025, c1=8e-4, c2=4e-4, rho=1e-6, mu=1e-6),
        "fp16": dict(phi=1e-4, ux=4e-3, uy=4.5e-3, p=3e-3, c1=8e-5, c2=6e-5, rho=1e-6, mu=1e-6),
    },
    "bubble_small": {
        "bf16": dict(phi=1.4e-3, ux=0.032, uy=0.04, p=8.5e-3, c1=1e-5, c2=7e-4, rho=1.4e-3, mu=1.4e-3),
        "fp16": dict(phi=6e-4, ux=4.5e-3, uy=5.5e-3, p=1e-3, c1=2e-6, c2=1.3e-4, rho=6e-4, mu=6e-4),
    },
    "q9_walls": {
        "bf16": dict(phi=8e-4, ux=0.012, uy=0.013, p=9e-3, c1=5e-4, c2=2.5e-4, rho=4e-4, mu=1e-3),
        "fp16": dict(phi=9e-5, ux=1.5e-3, uy=1e-3, p=1e-3, c1=6e-5, c2=4e-5, rho=5e-5, mu=1.1e-4),
    },
}
_CASE_ORACLE = {}


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("name", ["droplet64", "bubble_small", "q9_walls"])
def test_case_fields_per_storage(name, storage):
    params, init, steps = {"droplet64": _droplet, "bubble_small": _bubble_small, "q9_walls": _q9_walls}[name]()
    if name not in _CASE_ORACLE:
        _CASE_ORACLE[name] = run_oracle(params, init, steps).fields()
    want = _CASE_ORACLE[name]
    got = run_gpu(params, init, steps, storage).fields()
    errs = rel_max_errors(got, want, MAIN_FIELDS + ("rho", "mu"))
    _report("%s/%s" % (name, storage), errs)
    tol = CASE_TOL[name][storage]
    bad = {k: v for k, v in errs.items() if not v <= tol[k]}
    assert not bad, (bad, tol)


# ------------------------------------------------------------ conservation --
CONS_TOL = {"bf16": (5e-6, 2e-6), "fp16": (1e-6, 2e-6)}  # (phi, c)


@pytest.mark.parametrize("storage", STORAGES)
def test_conserved_sums_wander_at_rounding_level(storage):
    """sum phi and sum (c1 + c2) are conserved by the method.  With 16-bit
    storage the rounding of each stored rest population changes a node's
    total; stochastic rounding makes that change zero on average, so the
    totals wander instead of drifting (static droplet, 2000 steps): a random
    walk of one rounding per node and step.  The rest populations are stored
    as offsets near 0 (base weights summing to exactly 1), so both walks are
    small (measured ~5e-7 over 2000 steps; with h stored whole sum c walked
    1.1e-3 in bfloat16)."""
    w = wl.droplet64()
    sim = run_gpu(w.params, ("sdf", w.sdf, w.c1_tilde, w.c2_tilde), 0, storage)
    s0 = sim.conserved()
    sim.step(2000)
    s1 = sim.conserved()
    rel = np.abs(s1 - s0) / np.abs(s0)
    _report("conservation/%s" % storage, {"phi": rel[0], "c": rel[1]})
    assert rel[0] <= CONS_TOL[storage][0] and rel[1] <= CONS_TOL[storage][1]


# -------------------------------- full-size rising bubble: 16-bit vs FP32 --
_BUBBLE = {}


def _bubble_fp32():
    w = wl.bubble1024x2048()
    init = ("sdf", w.sdf, w.c1_tilde, w.c2_tilde)
    if "fp32" not in _BUBBLE:
        _BUBBLE["fp32"] = run_gpu(w.params, init, w.steps, "fp32").fields()
    return w, init, _BUBBLE["fp32"]


def _gas_centroid(phi):
    gas = 1.0 - phi
    ys, xs = np.mgrid[0:phi.shape[0], 0:phi.shape[1]]
    a = gas.sum()
    return a, (gas * xs).sum() / a, (gas * ys).sum() / a


def test_bubble_1024x2048_fp16_against_fp32():
    """The rising bubble at full size (1024 x 2048 walls, density ratio 1000,
    exp(-beta T) viscosity), 10000 steps: half storage against FP32 storage on
    the GPU (the FP32 path itself matches the oracle to 1e-5)."""
    w, init, ref = _bubble_fp32()
    got = run_gpu(w.params, init, w.steps, "fp16").fields()
    errs = rel_max_errors(got, ref, MAIN_FIELDS + ("rho", "mu"))
    sc = field_scales(ref)
    rms = {k: float(np.sqrt(np.mean((got[k] - ref[k]) ** 2)) / sc[k]) for k in MAIN_FIELDS}
    _report("bubble1024x2048/fp16 max", errs)
    _report("bubble1024x2048/fp16 rms", rms)
    a0, x0, y0 = _gas_centroid(ref["phi"])
    a1, x1, y1 = _gas_centroid(got["phi"])
    print("gas centroid fp32 (%.3f, %.3f) area %.1f; fp16 (%.3f, %.3f) area %.1f"
          % (x0, y0, a0, x1, y1, a1))
    assert all(np.isfinite(v).all() for v in got.values())
    # the bubble has risen ~45 nodes; with half storage it is within 0.005 of FP32
    assert abs(x1 - x0) < 0.05 and abs(y1 - y0) < 0.05
    assert abs(a1 - a0) / a0 < 1e-4
    assert rms["phi"] < 7e-5 and rms["c1"] < 1.5e-6 and rms["c2"] < 6e-5
    assert rms["ux"] < 1e-4 and rms["uy"] < 1.2e-4 and rms["p"] < 1e-4


def test_bubble_1024x2048_bf16_against_fp32():
    """bfloat16 keeps 8 significant bits.  In the gas (rho = 1e-3) the velocity
    is the flow populations' first moment divided by rho; stored whole, g_i is
    dominated by its pressure part 3 w_i p (p ~ 1e-4 against rho u ~ 1e-6 there),
    and its rounding noise, amplified a thousandfold, blew the run up within a
    few thousand steps; so did the noise that 8-bit f put into phi, through
    the surface-tension force in the gas.  Stored relative to their writers'
    pressure and phase field, the same 10000 steps stay finite and track the
    FP32 run."""
    w, init, ref = _bubble_fp32()
    got = run_gpu(w.params, init, w.steps, "bf16").fields()
    assert all(np.isfinite(v).all() for v in got.values())
    errs = rel_max_errors(got, ref, MAIN_FIELDS + ("rho", "mu"))
    sc = field_scales(ref)
    rms = {k: float(np.sqrt(np.mean((got[k] - ref[k]) ** 2)) / sc[k]) for k in MAIN_FIELDS}
    _report("bubble1024x2048/bf16 max", errs)
    _report("bubble1024x2048/bf16 rms", rms)
    a0, x0, y0 = _gas_centroid(ref["phi"])
    a1, x1, y1 = _gas_centroid(got["phi"])
    print("gas centroid fp32 (%.3f, %.3f) area %.1f; bf16 (%.3f, %.3f) area %.1f"
          % (x0, y0, a0, x1, y1, a1))
    # measured: centroid within 0.012 nodes, area within 4e-5
    assert abs(x1 - x0) < 0.1 and abs(y1 - y0) < 0.1
    assert abs(a1 - a0) / a0 < 2e-4
    assert rms["phi"] < 1e-4 and rms["c1"] < 5e-6 and rms["c2"] < 3e-4
    assert rms["ux"] < 8e-4 and rms["uy"] < 8e-4 and rms["p"] < 8e-4


@pytest.mark.parametrize("storage", STORAGES)
def test_restart_from_macros_per_storage(storage):
    """lbm_init_macros with a velocity field and a rough pressure field, read
    back before any step, against the oracle's restart: every flow population
    is stored relative to the pressure of the node its slot is pulled from (the
    upstream node, or the node itself behind a wall), so u and p come back to
    16-bit rounding of the small remainders.  Subtracting the node's own
    pressure instead would leave errors of the order of its gradient, 1e-4
    against a speed of 1e-3."""
    import oracle
    from paper_2402_15752_gb300 import Simulation
    w = wl.droplet64(nx=70, ny=45, R=12.0, rho2=0.2, mu2=0.05, wall_y=1)
    g = np.random.default_rng(17)
    ny, nx = w.sdf.shape
    phi = 0.5 + 0.5 * np.tanh(2.0 * w.sdf / w.params["W"])
    yy, xx = np.mgrid[0:ny, 0:nx]
    ux = 1e-3 * np.sin(2 * np.pi * xx / nx) * np.cos(np.pi * yy / ny)
    uy = -1e-3 * np.cos(2 * np.pi * xx / nx) * np.sin(np.pi * yy / ny)
    p = 1e-4 * g.standard_normal((ny, nx))
    c1, c2 = 0.8 * phi, 0.3 * (1.0 - phi)
    o = oracle.OracleSim(w.params)
    o.init_macros(phi, ux, uy, p, c1, c2)
    want = o.fields()
    sim = Simulation(w.params, precision=storage)
    sim.init_macros(phi, ux, uy, p, c1, c2)
    got = sim.fields()
    errs = rel_max_errors(got, want, ("ux", "uy", "p"))
    _report("restart/%s" % storage, errs)
    tol = {"bf16": 0.03, "fp16": 5e-3}[storage]
    assert max(errs.values()) < tol, errs


# ------------------------------------------------------------- determinism --
@pytest.mark.parametrize("storage", STORAGES)
def test_checkpoint_and_graph_are_bit_identical(storage):
    w = wl.droplet64(nx=50, ny=41, R=11.0, rho2=0.3, mu2=0.04)
    init = ("sdf", w.sdf, 1.0, 0.2)
    a = run_gpu(w.params, init, 0, storage)
    a.step(40)  # graphs of 32 and 8 steps
    b = run_gpu(w.params, init, 0, storage, chunks=[1] * 40)
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    st = a.get_state()
    a.step(17)
    want = a.fields()
    a.set_state(st)
    a.step(17)
    got = a.fields()
    for k in want:
        assert np.array_equal(got[k], want[k]), k
