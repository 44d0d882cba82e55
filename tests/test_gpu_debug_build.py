"""The debug build of the library (liblbm_debug.so, compiled with LBM_DEBUG=1):
its step, field and reduction kernels check every global load and store of the
workspace against the handle's workspace range; an access outside it is
skipped, recorded, and reported by lbm_sync as LBM_ERR_BOUNDS (nothing faults).

Small, odd and one-node-wide grids, periodic and walled, D2Q5 and D2Q9 scalars,
all four storage precisions and the batched runner run once through each build
(in child processes: the environment variable LBM_DEBUG selects the library):
* the debug build finds no access outside the workspace;
* it computes what the release build computes: to the parity bar of each
  precision, not bit for bit, since the checks change the compiled code
  around the arithmetic and with it the compiler's fusion of multiply-adds
  (and, in 16-bit storage, the value bits that seed the stochastic rounding);
  an access skipped by a failed check would read zero instead, an error of
  order one;
* with its checked range narrowed to half the workspace, a step is reported.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2402_15752_gb300.lbm import LBM_ERR_BOUNDS

from _debug_child import CASES, FIELDS, PRECISIONS
from _parity import MAIN_FIELDS, rel_max_errors

pytestmark = pytest.mark.gpu

# largest field difference, against each field's natural scale, and the
# relative difference of the conserved sums, after 40 steps
FIELD_TOL = {"fp64": 1e-11, "fp32": 1e-5, "fp16": 5e-3, "bf16": 5e-2}
SUM_TOL = {"fp64": 1e-12, "fp32": 1e-6, "fp16": 1e-3, "bf16": 1e-3}

HERE = os.path.dirname(os.path.abspath(__file__))
CHILD = os.path.join(HERE, "_debug_child.py")
LIMIT_KEYS = ("before_rc", "limit_rc", "after_rc", "cleared_rc")


def _run(out, debug, extra=()):
    env = dict(os.environ, LBM_DEBUG="1" if debug else "0")
    r = subprocess.run([sys.executable, CHILD, str(out), *extra], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    return dict(np.load(out))


@pytest.fixture(scope="module")
def runs(tmp_path_factory):
    from paper_2402_15752_gb300 import build
    build.build()
    build.build(debug=True)
    d = tmp_path_factory.mktemp("debug_build")
    return _run(d / "release.npz", False), _run(d / "debug.npz", True, ("limit",))


def test_the_builds_are_the_ones_selected(runs):
    rel, dbg = runs
    assert int(rel["debug"]) == 0
    assert int(dbg["debug"]) == 1


def test_debug_build_finds_no_access_outside_the_workspace(runs):
    _, dbg = runs
    codes = {k: int(v) for k, v in dbg.items() if k.endswith("_rc") and k not in LIMIT_KEYS}
    assert len(codes) == 6 * 4 + 1
    assert all(c == 0 for c in codes.values()), {k: c for k, c in codes.items() if c}


def test_debug_build_computes_what_the_release_build_does(runs):
    rel, dbg = runs
    worst = {}
    for case in CASES:
        for prec in PRECISIONS:
            key = "%s_%s_" % (case, prec)
            want = {k: rel[key + k] for k in FIELDS}
            got = {k: dbg[key + k] for k in FIELDS}
            errs = rel_max_errors(got, want, MAIN_FIELDS)
            assert max(errs.values()) <= FIELD_TOL[prec], (case, prec, errs)
            np.testing.assert_allclose(dbg[key + "sums"], rel[key + "sums"], rtol=SUM_TOL[prec], atol=0)
            worst[prec] = max(worst.get(prec, 0.0), max(errs.values()))
    for i in range(3):
        np.testing.assert_allclose(dbg["batch%d_phi" % i], rel["batch%d_phi" % i], rtol=0, atol=1e-5)
    print("\ndebug vs release build, worst field difference:",
          ", ".join("%s %.1e" % kv for kv in sorted(worst.items())))


def test_debug_build_reports_an_access_outside_its_range(runs):
    _, dbg = runs
    assert int(dbg["before_rc"]) == 0
    assert int(dbg["limit_rc"]) == 0
    assert int(dbg["after_rc"]) == LBM_ERR_BOUNDS
    # the report clears the check (the zeros the skipped loads read may have
    # made the state non-finite, which is reported next)
    assert int(dbg["cleared_rc"]) != LBM_ERR_BOUNDS
