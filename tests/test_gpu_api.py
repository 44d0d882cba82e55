"""GPU tests of the C ABI beyond field parity: conservation, checkpoints,
graph/plain equivalence, host/device read-back and error reporting."""
import ctypes

import numpy as np
import pytest

from paper_2402_15752_gb300 import Simulation, lbm
from paper_2402_15752_gb300 import workloads as wl

from _parity import run_oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-6)])
@pytest.mark.parametrize("name", ["droplet", "bubble"])
def test_conserved_sums(name, precision, tol):
    w = wl.droplet64(nx=70, ny=50, R=12.0) if name == "droplet" else wl.bubble1024x2048(nx=96, ny=192)
    sim = Simulation(w.params, precision=precision)
    sim.init(w.sdf, w.c1_tilde, w.c2_tilde)
    c0 = sim.conserved()
    ref = run_oracle(w.params, ("sdf", w.sdf, w.c1_tilde, w.c2_tilde), 0).conserved()
    assert np.allclose(c0, ref, rtol=1e-13 if precision == "fp64" else 1e-7, atol=0)
    sim.step(1000)
    c1 = sim.conserved()
    assert np.all(np.abs(c1 - c0) <= tol * np.abs(c0)), (c0, c1)
    if precision == "fp32":
        # the FP32 phase field is stored as integers: sum(phi) is conserved bit for bit
        assert c1[0] == c0[0]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpoint_resume_is_bit_identical(precision):
    w = wl.bubble1024x2048(nx=64, ny=96, R=10.0)
    a = Simulation(w.params, precision=precision)
    a.init(w.sdf, 0.0, 1.0)
    a.step(150)
    straight = None
    b = Simulation(w.params, precision=precision)
    b.init(w.sdf, 0.0, 1.0)
    b.step(75)
    state = b.get_state()
    dev_state = b.get_state(device=True)
    assert np.array_equal(state, dev_state.cpu().numpy())
    c = Simulation(w.params, precision=precision)
    c.set_state(state)
    c.step(75)
    straight = a.fields()
    resumed = c.fields()
    for k in straight:
        assert np.array_equal(straight[k], resumed[k]), k


def test_graph_and_plain_launches_agree_bitwise():
    w = wl.droplet64(nx=50, ny=41, R=10.0)
    a = Simulation(w.params, precision="fp32")
    a.init(w.sdf, 1.0, 0.0)
    a.step(97)  # three 32-step graphs + one plain step
    b = Simulation(w.params, precision="fp32")
    b.init(w.sdf, 1.0, 0.0)
    for _ in range(97):
        b.step(1)
    assert a.time == b.time == 97
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


def test_every_graph_length_matches_plain_launches():
    """A call of n steps replays captured graphs for the binary digits of n
    (32, 16, 8, 4, 2) and launches an odd last step plainly; the graphs are
    captured for both starting buffers.  63 steps (every graph length and a
    plain step, ending in the other buffer) and then 30 more (starting from
    that buffer) give the bits of 93 single steps."""
    w = wl.droplet64(nx=45, ny=38, R=9.0, rho2=0.4, mu2=0.05)
    a = Simulation(w.params, precision="fp32")
    a.init(w.sdf, 1.0, 0.2)
    a.step(63)
    a.step(30)
    b = Simulation(w.params, precision="fp32")
    b.init(w.sdf, 1.0, 0.2)
    for _ in range(93):
        b.step(1)
    assert a.time == b.time == 93
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


def test_host_and_device_readback_agree():
    w = wl.droplet64(nx=33, ny=65, R=8.0)
    sim = Simulation(w.params, precision="fp32")
    sim.init(w.sdf, 1.0, 0.5)
    sim.step(40)
    host = sim.fields()
    dev = sim.fields(device=True)
    f32 = sim.fields(dtype="f32")
    sub = sim.fields(names=("c2", "phi"))
    for k in host:
        assert np.array_equal(host[k], dev[k].cpu().numpy()), k
        assert np.array_equal(host[k].astype(np.float32), f32[k]), k
    assert list(sub) == ["phi", "c2"]
    assert np.array_equal(sub["c2"], host["c2"])


def test_page_locked_host_buffers_read_and_written_in_place():
    """Page-locked (mapped) host memory is read by the initialisation and written
    by the field evaluation in place; pageable memory goes through device
    staging and copies.  Both give the same bits, for every field set and both
    output types."""
    import torch
    w = wl.droplet64(nx=70, ny=37, R=9.0, rho2=0.3, mu2=0.04)
    sdf_pinned = torch.from_numpy(np.ascontiguousarray(w.sdf, dtype=np.float64)).pin_memory()
    a = Simulation(w.params, precision="fp32")
    a.init(sdf_pinned, 1.0, 0.3)        # read in place
    b = Simulation(w.params, precision="fp32")
    b.init(np.array(w.sdf), 1.0, 0.3)   # pageable: staged copy
    a.step(50)
    b.step(50)
    for dtype, tdt in (("f64", torch.float64), ("f32", torch.float32)):
        for names in (("phi", "ux", "uy", "p", "c1", "c2", "rho", "mu"), ("c2", "p")):
            out = torch.empty((len(names), 37, 70), dtype=tdt).pin_memory()
            got = a.fields(names=names, dtype=dtype, out=out.numpy())   # written in place
            want = b.fields(names=names, dtype=dtype)                    # staged
            for k in names:
                assert np.array_equal(got[k], want[k]), (dtype, names, k)


def test_init_from_device_fields():
    import torch
    w = wl.droplet64(nx=40, ny=40, R=9.0)
    phi = 0.5 + 0.5 * np.tanh(2 * w.sdf / 4.0)
    a = Simulation(w.params, precision="fp64")
    a.init_fields(phi, 0.7 * phi, 0.1 * (1 - phi))
    b = Simulation(w.params, precision="fp64")
    t = lambda v: torch.tensor(v, dtype=torch.float64, device="cuda")
    b.init_fields(t(phi), t(0.7 * phi), t(0.1 * (1 - phi)))
    a.step(20)
    b.step(20)
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


@pytest.mark.parametrize("W", [4.0, 5.0])
def test_init_profile_from_the_signed_distance(W):
    """lbm_init's profile phi = 1/2 + 1/2 tanh(2 l / W) (Eq. 2), c1 = c1~ phi,
    c2 = c2~ (1 - phi), read back before any step in FP64 storage, against
    numpy's FP64 tanh: across the interface band and the saturated bulk on both
    sides (|2 l / W| up to 24; beyond 20 the kernel skips the tanh, whose
    rounded value is +-1 there), to the rounding of the moments."""
    nx, ny = 160, 4
    l = np.tile((np.arange(nx) - 80.0) * 0.75, (ny, 1))
    p = dict(wl.BASE, nx=nx, ny=ny, W=W)
    sim = Simulation(p, precision="fp64")
    sim.init(l, 0.7, 0.2)
    f = sim.fields(names=("phi", "c1", "c2"))
    phi = 0.5 + 0.5 * np.tanh(2.0 * l / W)
    assert np.abs(2.0 * l / W).max() > 23 and (np.abs(2.0 * l / W) < 20).sum() > 40
    assert np.abs(f["phi"] - phi).max() < 2e-15
    assert np.abs(f["c1"] - 0.7 * phi).max() < 2e-15
    assert np.abs(f["c2"] - 0.2 * (1.0 - phi)).max() < 2e-15
    sim.close()


def test_nonfinite_state_is_reported():
    w = wl.droplet64(nx=32, ny=32, R=8.0)
    sim = Simulation(w.params, precision="fp32")
    phi = 0.5 + 0.5 * np.tanh(2 * w.sdf / 4.0)
    c1 = phi.copy()
    c1[5, 7] = np.nan
    sim.init_fields(phi, c1, 0 * phi)
    sim.step(3)
    with pytest.raises(lbm.LBMError) as e:
        sim.sync()
    assert e.value.code == lbm.LBM_ERR_NONFINITE
    with pytest.raises(lbm.LBMError) as e:
        sim.step(1)
    assert e.value.code == lbm.LBM_ERR_NONFINITE
    # a fresh init clears the condition
    sim.init(w.sdf, 1.0, 0.0)
    sim.step(3)
    sim.sync()


def test_argument_errors_are_codes_not_crashes():
    import torch
    L = lbm.load_library()
    p = lbm.make_params(dict(nx=16, ny=16), "fp32")
    need = L.lbm_workspace_bytes(ctypes.byref(p))
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p()
    rc = L.lbm_create(ctypes.byref(p), ctypes.c_void_p(ws.data_ptr()), need - 256, None, ctypes.byref(h))
    assert rc == lbm.LBM_ERR_WORKSPACE
    rc = L.lbm_create(ctypes.byref(p), ctypes.c_void_p(ws.data_ptr() + 8), need, None, ctypes.byref(h))
    assert rc == lbm.LBM_ERR_WORKSPACE
    host = np.zeros(need, dtype=np.uint8)
    rc = L.lbm_create(ctypes.byref(p), ctypes.c_void_p(host.ctypes.data), need, None, ctypes.byref(h))
    assert rc in (lbm.LBM_ERR_WORKSPACE,)
    rc = L.lbm_create(ctypes.byref(p), ctypes.c_void_p(ws.data_ptr()), need, None, ctypes.byref(h))
    assert rc == lbm.LBM_OK
    assert L.lbm_step(h, -1) == lbm.LBM_ERR_ARG
    assert L.lbm_get_fields(h, 0, ctypes.c_void_p(ws.data_ptr()), 1, 0) == lbm.LBM_ERR_ARG
    L.lbm_destroy(h)
    with pytest.raises(lbm.LBMError) as e:
        Simulation(dict(nx=8, ny=8, mu1=0.0))
    assert e.value.code == lbm.LBM_ERR_UNSTABLE_TAU
