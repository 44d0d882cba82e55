"""Batched runner (lbm_batch_*): many independent FP32 lattices of uneven sizes
in one persistent launch.

Every node of a batched step evaluates the expressions of lbm_step in the same
order; the two kernels are compiled separately, so the compiler may fuse a
different set of multiply-adds, and the results agree to FP32 rounding rather
than bit for bit.  They are checked against the same lattices stepped one at a
time to the FP32 parity bar, 1e-5 of each field's natural scale (the measured
difference after 75 steps is ~1e-6, in the spurious-current velocity of a static
droplet; a stale read at a tile border would show at 1e-3 and above), and a few
cases against the FP64 oracle at 1e-5.  Within one tile width every tile height runs the same code and
must give the same bits.  The bounded waits are exercised by withholding one
tile's completion: the launch must come back with LBM_ERR_TIMEOUT, never hang.
"""
import json

import numpy as np
import pytest

from paper_2402_15752_gb300 import Batch, Simulation
from paper_2402_15752_gb300 import workloads as wl
from paper_2402_15752_gb300.lbm import LBM_ERR_NONFINITE, LBM_ERR_TIMEOUT, LBMError

from _parity import MAIN_FIELDS, assert_parity, rel_max_errors, run_oracle

pytestmark = pytest.mark.gpu


def _cases():
    """Uneven shapes (ragged against 32-node blocks and every tile width),
    periodic and wall boundaries, different physics per case."""
    out = []
    for k, (nx, ny, walls, extra) in enumerate([
            (64, 64, (0, 0), {}),
            (96, 70, (0, 0), dict(rho2=0.2, mu2=0.05)),
            (130, 45, (1, 0), dict(Keq=3.0, D2=0.01)),
            (37, 23, (0, 0), dict(rho2=0.5)),
            (200, 128, (1, 1), dict(gy=-1e-5, g_rho_ref=1.0, rho2=0.1, mu2=0.02)),
            (33, 97, (0, 1), dict(visc_model=2, visc_beta=0.7)),
            (160, 31, (0, 0), dict(Fx=1e-6)),
            (257, 66, (1, 1), dict(A=1.0, Keq=0.5))]):
        w = wl.droplet64(nx=nx, ny=ny, R=0.3 * min(nx, ny), wall_x=walls[0], wall_y=walls[1],
                         **extra)
        out.append(w)
    return out


def _sims(cases):
    sims = [Simulation(w.params, precision="fp32") for w in cases]
    for s, w in zip(sims, cases):
        s.init(w.sdf, 1.0, 0.25)
    return sims


BATCH_TOL = 1e-5


def _assert_same(a_sims, b_sims, label="", tol=BATCH_TOL):
    """Each case's fields agree to `tol` of their natural scale (0: bit for bit)."""
    worst = 0.0
    for k, (a, b) in enumerate(zip(a_sims, b_sims)):
        fa, fb = a.fields(), b.fields()
        if tol == 0.0:
            for name in fa:
                assert np.array_equal(fa[name], fb[name]), "%s case %d field %s" % (label, k, name)
            continue
        errs = rel_max_errors(fa, fb, MAIN_FIELDS + ("rho", "mu"))
        worst = max(worst, max(errs.values()))
        bad = {n: v for n, v in errs.items() if not v <= tol}
        assert not bad, "%s case %d: %s" % (label, k, bad)
    print("\n%s worst rel-max difference %.2e" % (label, worst))


def test_batch_matches_single_lattice_steps():
    cases = _cases()
    batched, alone = _sims(cases), _sims(cases)
    b = Batch(batched)
    b.step(75)  # two graph replays of 32 steps and an 11-step launch
    b.sync()
    for s in alone:
        s.step(75)
        s.sync()
    assert all(s.time == 75 for s in batched)
    _assert_same(batched, alone)
    b.close()


@pytest.mark.parametrize("tile_w", [32, 64, 128])
def test_every_tiling_matches_and_heights_give_the_same_bits(tile_w):
    cases = _cases()
    alone = _sims(cases)
    for s in alone:
        s.step(13)
    runs = []
    for tile_h in (4, 16, 64):
        batched = _sims(cases)
        b = Batch(batched)
        b.set_tiling(tile_w, tile_h)
        t = b.tiling()
        assert (t["tile_w"], t["tile_h"]) == (tile_w, tile_h) and t["tiles"] >= len(cases)
        b.step(13)
        b.sync()
        _assert_same(batched, alone, label="tiling %dx%d" % (tile_w, tile_h))
        runs.append(batched)
        b.close()
    for other in runs[1:]:
        _assert_same(other, runs[0], label="heights at width %d" % tile_w, tol=0.0)


def test_batch_is_deterministic():
    cases = _cases()
    a_sims, b_sims = _sims(cases), _sims(cases)
    a, b = Batch(a_sims), Batch(b_sims)
    a.step(40)
    b.step(40)
    _assert_same(a_sims, b_sims, label="two identical batches", tol=0.0)
    a.close()
    b.close()


def test_batched_cases_match_the_oracle():
    cases = _cases()[:4]
    sims = _sims(cases)
    b = Batch(sims)
    b.set_tiling(32, 8)
    b.step(300)
    b.sync()
    for s, w in zip(sims, cases):
        want = run_oracle(w.params, ("sdf", w.sdf, 1.0, 0.25), 300).fields()
        assert_parity(s.fields(), want, 1e-5, label=w.name)
    b.close()


def test_autotuner_picks_a_timed_candidate_and_caches_it(tmp_path):
    cases = _cases()
    batched, alone = _sims(cases), _sims(cases)
    b = Batch(batched)
    cache = str(tmp_path / "tiles.json")
    got = b.autotune(steps_per_trial=3, cache=cache)
    assert not got["cached"] and len(got["trials"]) == 12
    best = min(got["trials"], key=lambda r: r["ms_per_step"])
    assert (got["tile_w"], got["tile_h"]) == (best["tile_w"], best["tile_h"])
    assert all(r["ms_per_step"] > 0 for r in got["trials"])
    # the trial steps were real steps: 12 candidates x (2 + 3)
    steps = 12 * 5
    assert all(s.time == steps for s in batched)
    for s in alone:
        s.step(steps)
    _assert_same(batched, alone, label="after autotune")
    known = json.load(open(cache))
    assert known[b.signature()] == {"tile_w": got["tile_w"], "tile_h": got["tile_h"]}
    again = b.autotune(steps_per_trial=3, cache=cache)
    assert again["cached"] and again["tile_w"] == got["tile_w"]
    b.close()


def test_case_reinitialised_alone_keeps_the_batch_consistent():
    cases = _cases()[:3]
    batched, alone = _sims(cases), _sims(cases)
    b = Batch(batched)
    b.step(7)
    batched[1].init(cases[1].sdf, 0.5, 0.5)  # back to buffer 0 while the others are in 1
    alone[1].init(cases[1].sdf, 0.5, 0.5)
    for k in (0, 2):
        alone[k].step(7)
    b.step(5)
    b.sync()
    for s in alone:
        s.step(5)
    _assert_same(batched, alone, label="after a lone init")
    b.close()


def test_batch_fields_state_and_restart_match_the_per_case_calls():
    """lbm_batch_get_fields, lbm_batch_get_state / set_state and
    lbm_batch_init_macros over uneven shapes: the concatenated buffers hold
    exactly what the per-case calls give, a restored batch steps to the same
    bits, and a batch restarted in one call steps to the same bits as one
    whose cases were restarted one by one."""
    import torch
    cases = _cases()
    names6 = ("phi", "ux", "uy", "p", "c1", "c2")
    sims = _sims(cases)
    b = Batch(sims)
    b.step(7)  # odd: every case's state is in its second buffer
    cells = sum(w.params["nx"] * w.params["ny"] for w in cases)
    out = torch.empty(6 * cells, dtype=torch.float64, device="cuda")
    b.fields(names6, out)
    got = out.cpu().numpy()
    off = 0
    for s in sims:
        n = s.nx * s.ny
        f = s.fields(names=names6)
        for k, name in enumerate(names6):
            assert np.array_equal(got[off + k * n: off + (k + 1) * n].reshape(s.ny, s.nx), f[name]), name
        off += 6 * n
    # checkpoint, step, restore, step again: the same bits
    buf = b.get_state()
    assert buf.numel() == b.state_bytes() == sum(s.state_bytes() for s in sims)
    b.step(5)
    b.sync()
    first = [s.fields() for s in sims]
    b.set_state(buf)
    b.step(5)
    b.sync()
    for k, s in enumerate(sims):
        again = s.fields()
        for name in again:
            assert np.array_equal(again[name], first[k][name]), (k, name)
    # restart from the concatenated macros in one call, against case by case
    macros = out.clone()
    one, each = _sims(cases), _sims(cases)
    b1, b2 = Batch(one), Batch(each)
    b1.step(3)
    b2.step(3)
    b1.init_macros(macros)
    off = 0
    for s in each:
        n = s.nx * s.ny
        m = [macros[off + k * n: off + (k + 1) * n].view(s.ny, s.nx) for k in range(6)]
        s.init_macros(*m)
        off += 6 * n
    b1.step(4)
    b2.step(4)
    b1.sync()
    b2.sync()
    _assert_same(one, each, label="batch restart", tol=0.0)
    for bb in (b1, b2, b):
        bb.close()


def test_a_withheld_tile_times_out_instead_of_hanging():
    cases = _cases()[:3]
    sims = _sims(cases)
    b = Batch(sims)
    b.set_tiling(64, 8)
    b.set_wait_limit(2000, hold_tile=0)  # tile 0 never reports: its neighbours give up
    b.step(3)
    with pytest.raises(LBMError) as e:
        b.sync()
    assert e.value.code == LBM_ERR_TIMEOUT
    with pytest.raises(LBMError) as e:
        b.step(1)
    assert e.value.code == LBM_ERR_TIMEOUT
    # recovery: re-initialise, restore the default limit, rebuild the tiling
    for s, w in zip(sims, cases):
        s.init(w.sdf, 1.0, 0.25)
    b.set_wait_limit(1 << 21, hold_tile=-1)
    b.set_tiling(64, 8)
    b.step(4)
    b.sync()
    alone = _sims(cases)
    for s in alone:
        s.step(4)
    _assert_same(sims, alone, label="after recovery")
    b.close()


def test_non_finite_case_is_reported_by_the_batch():
    cases = _cases()[:2]
    sims = _sims(cases)
    bad = np.full((cases[1].params["ny"], cases[1].params["nx"]), 0.5)
    bad[3, 4] = np.nan
    sims[1].init_fields(bad, bad, bad)
    b = Batch(sims)
    b.step(2)
    with pytest.raises(LBMError) as e:
        b.sync()
    assert e.value.code == LBM_ERR_NONFINITE
    b.close()


def test_batch_rejects_mixed_cases():
    a = Simulation(wl.droplet64(nx=40, ny=40).params, precision="fp32")
    c = Simulation(wl.droplet64(nx=40, ny=40).params, precision="fp64")
    with pytest.raises(LBMError):
        Batch([a, c])
    with pytest.raises(LBMError):
        Batch([a, a])
    d = Simulation(wl.droplet64(nx=40, ny=40, scalar_q=9).params, precision="fp32")
    with pytest.raises(LBMError):
        Batch([a, d])
