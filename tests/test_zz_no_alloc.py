"""lbm_conserved_noalloc: conserved sums of a device-resident state for callers
that may not allocate device memory (a validator living inside an application
whose GPU memory belongs to another allocator, a process already out of device
memory checking a saved state).  It keeps its reduction scratch in a fixed
array inside the library, so it needs neither a handle nor a workspace.

Checked through the C ABI against the handle-based lbm_conserved, twice in a
row on two different states, to the tolerance the conservation tests use.
This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process (the first call
on a device sets up the scratch address).
"""
import ctypes

import numpy as np
import pytest

from paper_2402_15752_gb300 import Simulation, lbm
from paper_2402_15752_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _entry(L):
    fn = L.lbm_conserved_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(lbm.LBMParams), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_int32, ctypes.c_char_p, ctypes.c_size_t]
    return fn


CASES = {
    # wall-bounded bubble (both boundary kinds of the pull: walls in x and y)
    "bubble": lambda: (wl.bubble1024x2048(nx=96, ny=192).params, wl.bubble1024x2048(nx=96, ny=192)),
    # periodic droplet (wrap-around pulls at every edge)
    "droplet": lambda: (wl.droplet64().params, wl.droplet64()),
    # one-scalar model: the h2 planes are not part of the state's sums
    "bubble_one_scalar": lambda: (dict(wl.bubble1024x2048(nx=96, ny=192).params, scalar_model=1, Keq=1.0),
                                  wl.bubble1024x2048(nx=96, ny=192)),
}


@pytest.mark.parametrize("case,precision", [
    ("bubble", "fp32"), ("bubble", "fp64"), ("bubble", "bf16"), ("bubble", "fp16"),
    ("droplet", "fp32"), ("droplet", "bf16"), ("droplet", "fp16"),
    ("bubble_one_scalar", "fp32"), ("bubble_one_scalar", "fp64"),
])
def test_noalloc_sums_match_lbm_conserved_on_two_calls(case, precision):
    """Every storage the entry point accepts (FP64, FP32 with the fixed-point
    phase field, bfloat16 and half in paired 16-bit words with the f - w/2
    offset), both scalar models, walls and periodic wrap."""
    import torch
    params_dict, w = CASES[case]()
    sim = Simulation(params_dict, precision=precision)
    sim.init(w.sdf, w.c1_tilde, w.c2_tilde)
    fn = _entry(sim.L)
    params = lbm.make_params(params_dict, precision)
    err = ctypes.create_string_buffer(256)
    for steps in (0, 200):  # two calls in a row, on two different states
        sim.step(steps)
        want = sim.conserved()
        state = sim.get_state(device=True)
        host_out = (ctypes.c_double * 2)()
        rc = fn(ctypes.byref(params), state.data_ptr(), state.numel(), sim.stream.cuda_stream,
                ctypes.addressof(host_out), 0, err, len(err))
        assert rc == lbm.LBM_OK, err.value
        # same loads, possibly another summation order
        np.testing.assert_allclose([host_out[0], host_out[1]], want, rtol=1e-12, atol=0)
        dev_out = torch.zeros(2, dtype=torch.float64, device=sim.device)
        rc = fn(ctypes.byref(params), state.data_ptr(), state.numel(), sim.stream.cuda_stream,
                dev_out.data_ptr(), 1, err, len(err))
        assert rc == lbm.LBM_OK, err.value
        sim.stream.synchronize()
        np.testing.assert_allclose(dev_out.cpu().numpy(), want, rtol=1e-12, atol=0)
        if precision == "fp32":
            # the phase field is integer in FP32 runs: both reductions agree exactly
            assert host_out[0] == want[0]


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    L = lbm.load_library()
    fn = _entry(L)
    buf = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    err = ctypes.create_string_buffer(256)
    out = (ctypes.c_double * 2)()
    too_big = lbm.make_params(dict(nx=8193, ny=8192), "fp32")
    rc = fn(ctypes.byref(too_big), buf.data_ptr(), buf.numel(), None, ctypes.addressof(out), 0,
            err, len(err))
    assert rc == lbm.LBM_ERR_ARG
    assert b"limit" in err.value
    small = lbm.make_params(dict(nx=64, ny=64), "fp32")
    rc = fn(ctypes.byref(small), buf.data_ptr(), buf.numel(), None, ctypes.addressof(out), 0,
            err, len(err))
    assert rc == lbm.LBM_ERR_ARG  # buffer smaller than the state of a 64x64 grid
    big = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    rc = fn(ctypes.byref(small), big.data_ptr() + 4, big.numel() - 4, None, ctypes.addressof(out), 0,
            err, len(err))
    assert rc == lbm.LBM_ERR_ARG and b"aligned" in err.value  # an offset pointer is refused
    bad_q = lbm.make_params(dict(nx=64, ny=64, scalar_q=7), "fp32")
    rc = fn(ctypes.byref(bad_q), big.data_ptr(), big.numel(), None, ctypes.addressof(out), 0,
            err, len(err))
    assert rc == lbm.LBM_ERR_ARG and b"scalar_q" in err.value
