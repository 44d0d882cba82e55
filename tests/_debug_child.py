"""Child process of test_gpu_debug_build.py: runs small cases through the library
that LBM_DEBUG selects (the debug build when LBM_DEBUG=1, else the release one)
and saves their fields, conserved sums and return codes to an .npz file.

usage: python _debug_child.py OUT.npz [limit]
  limit: also narrow one handle's checked range (debug build) and record what
  lbm_sync reports after a step.
"""
import ctypes
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

from paper_2402_15752_gb300 import Batch, Simulation, lbm  # noqa: E402
from paper_2402_15752_gb300 import workloads as wl  # noqa: E402

from _parity import run_gpu  # noqa: E402
from test_gpu_parity import _case  # noqa: E402

# tiny, odd and one-node-wide grids, periodic and walled, both scalar lattices
CASES = ["ragged_periodic", "ragged_walls", "strip_x", "strip_y_poiseuille", "narrow_x_walls",
         "q9_logc_force"]
PRECISIONS = ["fp32", "fp64", "bf16", "fp16"]
STEPS = 40
FIELDS = ("phi", "ux", "uy", "p", "c1", "c2", "rho")


def main(out, limit):
    L = lbm.load_library()
    res = {"debug": np.array(int(L.lbm_debug_build()))}
    for name in CASES:
        params, init, _ = _case(name)
        for prec in PRECISIONS:
            sim = run_gpu(params, init, STEPS, prec)
            rc = L.lbm_sync(sim._h)
            f = sim.fields()
            key = "%s_%s" % (name, prec)
            res[key + "_rc"] = np.array(rc)
            res[key + "_sums"] = sim.conserved()
            for k in FIELDS:
                res[key + "_" + k] = f[k]
            sim.close()
    # the batched runner over three uneven lattices
    sims = []
    for nx, ny, walls in ((37, 23, (0, 0)), (64, 40, (1, 0)), (45, 19, (1, 1))):
        w = wl.droplet64(nx=nx, ny=ny, R=0.3 * min(nx, ny), wall_x=walls[0], wall_y=walls[1])
        s = Simulation(w.params, precision="fp32")
        s.init(w.sdf, 1.0, 0.25)
        sims.append(s)
    b = Batch(sims)
    b.set_tiling(32, 8)
    b.step(STEPS)
    res["batch_rc"] = np.array(L.lbm_batch_sync(b._b))
    for i, s in enumerate(sims):
        res["batch%d_phi" % i] = s.fields()["phi"]
    b.close()
    for s in sims:
        s.close()
    if limit:
        params, init, _ = _case("ragged_periodic")
        sim = run_gpu(params, init, 1, "fp32")
        res["before_rc"] = np.array(L.lbm_sync(sim._h))
        nbytes = ctypes.c_size_t(sim.workspace.numel() * sim.workspace.element_size() // 2)
        res["limit_rc"] = np.array(L.lbm_debug_limit_workspace(sim._h, nbytes))
        L.lbm_step(sim._h, 1)
        res["after_rc"] = np.array(L.lbm_sync(sim._h))
        res["cleared_rc"] = np.array(L.lbm_sync(sim._h))  # the report clears the check
    np.savez(out, **res)


if __name__ == "__main__":
    main(sys.argv[1], len(sys.argv) > 2 and sys.argv[2] == "limit")
