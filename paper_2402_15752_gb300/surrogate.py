"""Surrogate network: a residual CNN that advances the macroscopic fields of a
periodic lattice 16 time steps at a time, trained on trajectories of the
solver, with the solver as its judge and fallback.  Not in the paper.

* Network: six periodic 3x3 convolutions, 48 channels, ReLU between them,
  input and output (phi, ux, uy, p, C = c1 + c2) normalised per channel, and
  a residual connection: state(t + 16) = state(t) + net(state(t)).  BF16
  weights and activations, FP32 accumulation, FP32 master weights (Adam).
* Every arithmetic step runs in the library's kernels (include/lbm_nn.h):
  the convolutions and their gradients on the tensor cores, loss, Adam,
  packing.  This module allocates memory and sequences the calls.
* Data: trajectories of the solver's batched runner, snapshots every 16
  steps after a warm-up: buoyant droplets and rising bubbles under gravity
  (flow_cases: 1-4 separated drops, R ~ U[10, 60], density ratio ~ U[1, 100])
  or resting droplets (droplet_cases).
* Judge and fallback: every `judge_every` hops the solver is restarted from
  the state the hop started from (lbm_batch_init_macros, C split at the Henry
  equilibrium) and run 16 steps; if the network's hop differs from it by more
  than `tol` in phi or C (RMS, in units of the channel's spread), the solver
  reruns from the last accepted state and its result is kept.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import time

import numpy as np

from .batch import Batch
from .lbm import LBMError, Simulation, load_library
from . import workloads as wl

LAYERS = ((16, 48), (48, 48), (48, 48), (48, 48), (48, 48), (48, 16))
# Dilated layers: the receptive field reaches 21 nodes, past the ~9 nodes a
# sound wave travels in one 16-step hop (c_s = 1/sqrt(3)) and across the
# largest drops' radius.
DILATIONS = (1, 2, 4, 8, 4, 2)
HOP = 16
USED = 5
CHANNELS = ("phi", "ux", "uy", "p", "C")
FIELDS6 = ("phi", "ux", "uy", "p", "c1", "c2")
RELU, RESIDUAL, MASK = 0, 1, 2


def nn_lib():
    L = load_library()
    if getattr(L, "_nn_ready", False):
        return L
    vp, i32, i64, sz, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_float
    sig = {
        "lbm_nn_conv3x3": [vp, i32, vp, vp, i32, i32, vp, vp, vp, i32, i32, i32, i32, vp, vp],
        "lbm_nn_flip_weights": [vp, i32, i32, vp, vp],
        "lbm_nn_conv3x3_wgrad": [vp, i32, vp, i32, vp, vp, sz, i32, i32, i32, i32, vp, vp],
        "lbm_nn_bias_grad": [vp, i32, i64, vp, vp, vp],
        "lbm_nn_mse": [vp, vp, i32, i64, vp, vp, vp, vp],
        "lbm_nn_adam": [vp, vp, vp, vp, vp, vp, i64, f32, f32, f32, f32, i32, vp],
        "lbm_nn_pack": [vp, i32, i32, i32, vp, vp, vp, vp, vp],
        "lbm_nn_unpack": [vp, i32, i32, i32, vp, vp, vp, vp],
        "lbm_nn_unpack_macros": [vp, i32, i32, i32, vp, vp, vp, vp, vp],
        "lbm_nn_state_diff": [vp, vp, i32, i64, vp, vp, vp],
        "lbm_nn_to_bf16": [vp, i64, vp, vp],
        "lbm_nn_add_noise": [vp, i64, i32, f32, ctypes.c_uint32, vp],
        "lbm_nn_to_f32": [vp, i64, vp, vp],
        "lbm_nn_axpy": [vp, vp, f32, i64, vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.restype = ctypes.c_int
        fn.argtypes = args
    L.lbm_nn_wgrad_partial_bytes.restype = sz
    L.lbm_nn_wgrad_partial_bytes.argtypes = [i32, i32, i32, i32, i32, i32]
    L._nn_ready = True
    return L


def _ck(rc, what):
    if rc != 0:
        raise LBMError(rc, what)


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def bf16_bits(a: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 bit patterns, rounded to nearest even."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def to_device_bf16(a: np.ndarray, device):
    import torch
    bits = torch.from_numpy(bf16_bits(a).view(np.int16))
    return bits.to(device).view(torch.bfloat16)


class Net:
    """Parameters, optimiser state and scratch of the six-layer network."""

    def __init__(self, device, seed: int = 0, stream=None, dilations=DILATIONS):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.dil = tuple(int(d) for d in dilations)
        assert len(self.dil) == len(LAYERS)
        # bit 0 set by a convolution whose bounded wait on the tensor cores gave up
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)
        g = np.random.default_rng(seed)
        self.w32, self.b32, self.wb, self.wt = [], [], [], []
        self.mw, self.vw, self.mb, self.vb, self.gw, self.gb = [], [], [], [], [], []
        self.mask_w, self.mask_b = [], []
        for l, (ci, co) in enumerate(LAYERS):
            ci_r = 5 if l == 0 else ci
            co_r = 5 if l == 5 else co
            w = np.zeros((co, 9, ci), np.float32)
            w[:co_r, :, :ci_r] = g.standard_normal((co_r, 9, ci_r)) * math.sqrt(2.0 / (9 * ci_r))
            if l == 5:
                w *= 0.1  # start close to the identity map of the residual network
            mw = np.zeros((co, 9, ci), np.uint8)
            mw[:co_r, :, :ci_r] = 1
            mb = np.zeros(co, np.uint8)
            mb[:co_r] = 1
            self._add(w, np.zeros(co, np.float32), mw, mb)
        self.t = 0
        self.refresh()

    def _add(self, w, b, mw, mb):
        t, d = self.torch, self.device
        self.w32.append(t.from_numpy(w).to(d))
        self.b32.append(t.from_numpy(b).to(d))
        self.wb.append(to_device_bf16(w, d))
        self.wt.append(t.empty((w.shape[2], 9, w.shape[0]), dtype=t.bfloat16, device=d))
        self.mask_w.append(t.from_numpy(mw).to(d))
        self.mask_b.append(t.from_numpy(mb).to(d))
        for lst, shape in ((self.mw, w.shape), (self.vw, w.shape), (self.gw, w.shape),
                           (self.mb, b.shape), (self.vb, b.shape), (self.gb, b.shape)):
            lst.append(t.zeros(shape, dtype=t.float32, device=d))

    @property
    def s(self):
        return ctypes.c_void_p(self.stream.cuda_stream)

    def refresh(self):
        """Flipped (adjoint) weights for the backward pass, from the bf16 copies
        (layer 0's for the gradient with respect to the network's input)."""
        L = nn_lib()
        for l in range(6):
            ci, co = LAYERS[l]
            _ck(L.lbm_nn_flip_weights(_p(self.wb[l]), ci, co, _p(self.wt[l]), self.s), "flip")

    # -- save / load (FP32 master weights) --
    def check(self):
        """Raise if a convolution reported that a bounded wait gave up."""
        if int(self.status.item()) != 0:
            raise LBMError(-6, "surrogate convolution: a wait on the tensor cores timed out")

    def state_dict(self) -> dict:
        out = {"dilations": np.asarray(self.dil, dtype=np.int32)}
        for l in range(6):
            out["w%d" % l] = self.w32[l].cpu().numpy()
            out["b%d" % l] = self.b32[l].cpu().numpy()
        return out

    def load_state_dict(self, d: dict):
        t = self.torch
        for l in range(6):
            w = np.asarray(d["w%d" % l], dtype=np.float32)
            self.w32[l].copy_(t.from_numpy(w))
            self.b32[l].copy_(t.from_numpy(np.asarray(d["b%d" % l], dtype=np.float32)))
            self.wb[l].copy_(to_device_bf16(w, self.device))
        self.refresh()

    # -- passes --
    def forward(self, x32, x16, out32, acts, B, H, W):
        """out32 = x32 + net(x); acts: 5 bf16 buffers [B, H, W, 48] (kept for
        backward) or 2 (ping-pong, inference)."""
        L = nn_lib()
        cur = x16
        for l in range(5):
            ci, co = LAYERS[l]
            nxt = acts[l] if len(acts) == 5 else acts[l % 2]
            _ck(L.lbm_nn_conv3x3(_p(cur), ci, _p(self.wb[l]), _p(self.b32[l]), co, RELU, None, None,
                                 _p(nxt), B, H, W, self.dil[l], _p(self.status), self.s), "conv%d" % l)
            cur = nxt
        _ck(L.lbm_nn_conv3x3(_p(cur), 48, _p(self.wb[5]), _p(self.b32[5]), 16, RESIDUAL, _p(x32), None,
                             _p(out32), B, H, W, self.dil[5], _p(self.status), self.s), "conv5")

    def backward(self, x16, acts, dz16, dbuf, scratch, B, H, W, dx32=None):
        """Gradients of every weight and bias from dz16 = d loss / d out (bf16, 16 ch).
        With dx32 (a float state buffer), also the gradient with respect to the
        network's input: the residual path dz16 plus layer 0's adjoint
        convolution of its output gradient (the residual epilogue adds them)."""
        L = nn_lib()
        P = B * H * W
        wpart, bpart = scratch
        dz = dz16
        if dx32 is not None:
            _ck(L.lbm_nn_to_f32(_p(dz16), dx32.numel(), _p(dx32), self.s), "to_f32")
        for l in range(5, -1, -1):
            ci, co = LAYERS[l]
            a_l = x16 if l == 0 else acts[l - 1]
            nb = L.lbm_nn_wgrad_partial_bytes(ci, co, B, H, W, self.dil[l])
            _ck(L.lbm_nn_conv3x3_wgrad(_p(a_l), ci, _p(dz), co, _p(self.gw[l]), _p(wpart), nb, B, H, W,
                                       self.dil[l], _p(self.status), self.s), "wgrad%d" % l)
            _ck(L.lbm_nn_bias_grad(_p(dz), co, P, _p(self.gb[l]), _p(bpart), self.s), "bgrad%d" % l)
            if l > 0:
                nxt = dbuf[l % 2]
                _ck(L.lbm_nn_conv3x3(_p(dz), co, _p(self.wt[l]), None, ci, MASK, None, _p(a_l), _p(nxt),
                                     B, H, W, self.dil[l], _p(self.status), self.s), "dgrad%d" % l)
                dz = nxt
            elif dx32 is not None:
                _ck(L.lbm_nn_conv3x3(_p(dz), co, _p(self.wt[0]), None, ci, RESIDUAL, _p(dx32), None, _p(dx32),
                                     B, H, W, self.dil[0], _p(self.status), self.s), "dgrad0")

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        L = nn_lib()
        self.t += 1
        for l in range(6):
            _ck(L.lbm_nn_adam(_p(self.w32[l]), _p(self.gw[l]), _p(self.mw[l]), _p(self.vw[l]), _p(self.mask_w[l]),
                              _p(self.wb[l]), self.w32[l].numel(), lr, beta1, beta2, eps, self.t, self.s), "adam w")
            _ck(L.lbm_nn_adam(_p(self.b32[l]), _p(self.gb[l]), _p(self.mb[l]), _p(self.vb[l]), _p(self.mask_b[l]),
                              None, self.b32[l].numel(), lr, beta1, beta2, eps, self.t, self.s), "adam b")
        self.refresh()


class Workspace:
    """Device buffers for batches of B samples of H x W."""

    def __init__(self, B, H, W, device, train=True, dilations=DILATIONS):
        import torch
        t = torch
        self.B, self.H, self.W = B, H, W
        P = B * H * W
        self.x32 = t.zeros((B, H, W, 16), dtype=t.float32, device=device)
        self.y32 = t.zeros_like(self.x32)
        self.t32 = t.zeros_like(self.x32)
        self.x16 = t.zeros((B, H, W, 16), dtype=t.bfloat16, device=device)
        self.dz16 = t.zeros((B, H, W, 16), dtype=t.bfloat16, device=device)
        nacts = 5 if train else 2
        self.acts = [t.empty((B, H, W, 48), dtype=t.bfloat16, device=device) for _ in range(nacts)]
        self.dbuf = [t.empty((B, H, W, 48), dtype=t.bfloat16, device=device) for _ in range(2)] if train else None
        L = nn_lib()
        wbytes = max(L.lbm_nn_wgrad_partial_bytes(ci, co, B, H, W, d) for (ci, co), d in zip(LAYERS, dilations))
        self.scratch = (t.empty(wbytes // 4 + 1, dtype=t.float32, device=device),
                        t.empty(1024 * 48, dtype=t.float32, device=device))
        self.loss_part = t.empty(1024, dtype=t.float64, device=device)
        self.diff_part = t.empty(640 * B, dtype=t.float32, device=device)
        self.diff = t.empty(B * 10, dtype=t.float32, device=device)
        self.P = P


def droplet_cases(n, seed, side=256, radius=(10.0, 60.0)):
    """Seeded droplet cases of the surrogate's data: 1-4 droplets, radius
    U[10, 60], density ratio U[1, 100] (heavy droplets at density 1), K_eq
    U[0.5, 5], D1/D2 U[1, 100]; scalar 1 in the droplets."""
    g = np.random.default_rng(wl.SEED_BASE + 1000 + int(seed))
    out = []
    for _ in range(n):
        k = int(g.integers(1, 5))
        radii = g.uniform(radius[0], radius[1], size=k)
        centres = g.uniform(0.0, side, size=(k, 2))
        ratio = float(g.uniform(1.0, 100.0))
        p = dict(wl.BASE, nx=side, ny=side, sigma=0.01, rho1=1.0, rho2=1.0 / ratio, mu1=0.1,
                 mu2=0.1 / ratio, D1=0.1, D2=0.1 / float(g.uniform(1.0, 100.0)),
                 Keq=float(g.uniform(0.5, 5.0)))
        out.append(wl.Workload("surrogate", p, wl.sdf_droplets(side, side, centres, radii), 1.0, 0.0,
                               HOP, {"ratio": ratio}))
    return out


def _separated_circles(g, radii, side, gap, tries=200):
    """Centres drawn uniformly in the periodic box such that the circles stay at
    least `gap` nodes apart (periodic distance); a circle that finds no room is
    dropped (the first always stays).  Returns (centres, radii) of those kept.
    Touching inclusions at density ratios near 100 start with a thin neck whose
    curvature drives the scheme unstable."""
    centres, kept = [], []
    for R in radii:
        for _ in range(tries):
            c = g.uniform(0.0, side, size=2)
            clear = True
            for c2, R2 in zip(centres, kept):
                dd = np.abs(c - c2)
                dd = np.minimum(dd, side - dd)
                if float(np.hypot(dd[0], dd[1])) < R + R2 + gap:
                    clear = False
                    break
            if clear:
                centres.append(c)
                kept.append(float(R))
                break
    return np.array(centres), np.array(kept)


def flow_cases(n, seed, side=256, radius=(10.0, 60.0), g_range=(1e-6, 5e-6), gap=8.0):
    """Seeded cases with sustained motion: half of them 1-4 heavy droplets
    (phase 1) in a light fluid, half 1-4 light bubbles (phase 2) in a heavy
    liquid, radius U[10, 60], density ratio U[1, 100] (heavy phase at density
    1), K_eq U[0.5, 5], D1/D2 U[1, 100], periodic box, gravity U[1e-6, 5e-6]
    along -y; inclusions at least `gap` nodes apart.  The body force is the
    buoyancy (rho - rho_ref) g with rho_ref the
    box's mean density from the inclusions' area fraction, so the box as a whole
    is not accelerated: droplets sink and bubbles rise."""
    g = np.random.default_rng(wl.SEED_BASE + 2000 + int(seed))
    out = []
    for i in range(n):
        k = int(g.integers(1, 5))
        radii = g.uniform(radius[0], radius[1], size=k)
        centres, radii = _separated_circles(g, radii, side, gap)
        ratio = float(g.uniform(1.0, 100.0))
        rho1, rho2 = 1.0, 1.0 / ratio
        bubbles = bool(i % 2)
        sdf = wl.sdf_droplets(side, side, centres, radii)  # phase 1 inside the circles
        frac = min(1.0, float(np.pi * np.sum(radii ** 2)) / side ** 2)  # area of the circles
        if bubbles:
            sdf = -sdf  # phase 2 inside
            phi_mean = 1.0 - frac
        else:
            phi_mean = frac
        grav = float(g.uniform(*g_range))
        # kinematic viscosity 0.1 in the heavy phase and 0.1 min(ratio, 10) in the
        # light one: light bubbles at large density ratios need tau_g well above
        # 1/2 inside them to stay stable (as the rising-bubble workload does)
        p = dict(wl.BASE, nx=side, ny=side, sigma=0.01, rho1=rho1, rho2=rho2, mu1=0.1,
                 mu2=0.1 * min(ratio, 10.0) / ratio, D1=0.1, D2=0.1 / float(g.uniform(1.0, 100.0)),
                 Keq=float(g.uniform(0.5, 5.0)), gx=0.0, gy=-grav,
                 g_rho_ref=rho2 + (rho1 - rho2) * phi_mean)
        c1t, c2t = (0.0, 1.0) if bubbles else (1.0, 0.0)
        out.append(wl.Workload("surrogate-flow", p, sdf, c1t, c2t, HOP,
                               {"ratio": ratio, "bubbles": bubbles, "g": grav}))
    return out


def generate(cases, snapshots, device, warm=64, group=128):
    """Solver trajectories: fields (phi, ux, uy, p, c1, c2) as float planes,
    [n, snapshots, 6, H, W], one snapshot every HOP steps after `warm` steps."""
    import torch
    H, W = cases[0].params["ny"], cases[0].params["nx"]
    data = torch.empty((len(cases), snapshots, 6, H, W), dtype=torch.float32, device=device)
    for g0 in range(0, len(cases), group):
        part = cases[g0:g0 + group]
        sims = [Simulation(w.params, precision="fp32", device=device) for w in part]
        for s, w in zip(sims, part):
            s.init(w.sdf, w.c1_tilde, w.c2_tilde)
        b = Batch(sims)
        b.set_tiling(128, 32)
        b.step(warm)
        for k in range(snapshots):
            if k:
                b.step(HOP)
            for j, s in enumerate(sims):
                s.fields(names=FIELDS6, dtype="f32", device=True, out=data[g0 + j, k])
        b.sync()
        b.close()
        for s in sims:
            s.close()
    return data


def normalisation(data, samples=64):
    """Per-channel shift and scale of (phi, ux, uy, p, C) from a sample of
    snapshots (host statistics)."""
    n = data.shape[0]
    idx = np.linspace(0, n - 1, min(n, samples)).astype(int)
    host = data[idx].cpu().numpy()  # [s, snaps, 6, H, W]
    ch = [host[:, :, 0], host[:, :, 1], host[:, :, 2], host[:, :, 3], host[:, :, 4] + host[:, :, 5]]
    shift = np.array([float(c.mean()) for c in ch], dtype=np.float32)
    scale = np.array([1.0 / max(float(c.std()), 1e-12) for c in ch], dtype=np.float32)
    return shift, scale


class Surrogate:
    def __init__(self, net: Net, shift, scale):
        import torch
        self.net = net
        self.shift = torch.from_numpy(np.asarray(shift, np.float32)).to(net.device)
        self.scale = torch.from_numpy(np.asarray(scale, np.float32)).to(net.device)

    def save(self, path):
        d = self.net.state_dict()
        d["shift"] = self.shift.cpu().numpy()
        d["scale"] = self.scale.cpu().numpy()
        np.savez(path, **d)

    @classmethod
    def load(cls, path, device, stream=None):
        d = dict(np.load(path))
        net = Net(device, stream=stream, dilations=tuple(d.get("dilations", DILATIONS)))
        net.load_state_dict(d)
        return cls(net, d["shift"], d["scale"])

    def pack(self, fields6, ws, state32, act16=None):
        L = nn_lib()
        _ck(L.lbm_nn_pack(_p(fields6), ws.B, ws.H, ws.W, _p(self.shift), _p(self.scale), _p(state32),
                          _p(act16), self.net.s), "pack")

    def hop(self, ws):
        """ws.y32 = one network hop of ws.x32 (bf16 copy in ws.x16)."""
        self.net.forward(ws.x32, ws.x16, ws.y32, ws.acts, ws.B, ws.H, ws.W)

    def unpack(self, state32, ws, fields5):
        L = nn_lib()
        _ck(L.lbm_nn_unpack(_p(state32), ws.B, ws.H, ws.W, _p(self.shift), _p(self.scale), _p(fields5),
                            self.net.s), "unpack")


def train(sur: Surrogate, data, epochs=4, batch=16, lr=1e-3, seed=0, noise=0.03, log=print,
          pushforward=0.0):
    """Adam on the MSE of one hop over all consecutive snapshot pairs, with a
    cosine learning-rate decay.  The input state is corrupted by Gaussian noise
    of `noise` (normalised units) while the target stays the solver's: the
    network learns to pull a perturbed state back, which keeps its own
    autoregressive rollouts from drifting (input-noise training as in
    Sanchez-Gonzalez et al. 2020).  With pushforward = q > 0, from the second
    epoch on a fraction q of the batches starts one snapshot earlier: the
    network's own (untrained-through) prediction of the next snapshot is the
    input and the snapshot after it the target, so the network also learns
    from the errors it makes itself (the pushforward trick of Brandstetter,
    Worrall & Welling 2022)."""
    import torch
    net = sur.net
    n, S = data.shape[0], data.shape[1]
    H, W = data.shape[3], data.shape[4]
    ws = Workspace(batch, H, W, net.device, train=True, dilations=net.dil)
    L = nn_lib()
    pairs = np.array([(i, k) for i in range(n) for k in range(S - 1)])
    triples = np.array([(i, k) for i in range(n) for k in range(S - 2)])
    g = np.random.default_rng(seed)
    steps = epochs * (len(pairs) // batch)
    losses = torch.zeros(max(1, steps), dtype=torch.float64, device=net.device)
    ident = torch.zeros(8, dtype=torch.float64, device=net.device)
    step = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        order = g.permutation(len(pairs))
        lr_ep = lr * (0.5 * (1.0 + math.cos(math.pi * ep / max(1, epochs))))
        for b0 in range(0, len(order) - batch + 1, batch):
            push = pushforward > 0 and ep > 0 and len(triples) > 0 and g.random() < pushforward
            sel = triples[g.integers(0, len(triples), batch)] if push else pairs[order[b0:b0 + batch]]
            ii = torch.from_numpy(sel[:, 0]).to(net.device)
            kk = torch.from_numpy(sel[:, 1]).to(net.device)
            xf = data[ii, kk].contiguous()
            yf = data[ii, kk + (2 if push else 1)].contiguous()
            sur.pack(xf, ws, ws.x32, ws.x16 if (push or noise <= 0) else None)
            sur.pack(yf, ws, ws.t32)
            if push:
                # the network's own hop as the input (no gradient through it)
                net.forward(ws.x32, ws.x16, ws.y32, ws.acts, batch, H, W)
                ws.x32.copy_(ws.y32)
                _ck(L.lbm_nn_to_bf16(_p(ws.x32), ws.x32.numel(), _p(ws.x16), net.s), "to_bf16")
            elif noise > 0:
                _ck(L.lbm_nn_add_noise(_p(ws.x32), ws.P, USED, noise, (seed * 1000003 + step) & 0xffffffff,
                                       net.s), "noise")
                _ck(L.lbm_nn_to_bf16(_p(ws.x32), ws.x32.numel(), _p(ws.x16), net.s), "to_bf16")
            if step < 8:  # the loss of predicting no change, for reference
                _ck(L.lbm_nn_mse(_p(ws.x32), _p(ws.t32), USED, ws.P, None, _p(ws.loss_part),
                                 _p(ident[step:step + 1]), net.s), "mse")
            net.forward(ws.x32, ws.x16, ws.y32, ws.acts, batch, H, W)
            _ck(L.lbm_nn_mse(_p(ws.y32), _p(ws.t32), USED, ws.P, _p(ws.dz16), _p(ws.loss_part),
                             _p(losses[step:step + 1]), net.s), "mse")
            net.backward(ws.x16, ws.acts, ws.dz16, ws.dbuf, ws.scratch, batch, H, W)
            net.adam(lr_ep)
            step += 1
        if log:
            lh = losses[:step].cpu().numpy()
            per = max(1, len(order) // batch)
            net.check()
            log("epoch %d: loss %.4e (first %.4e, no-change baseline %.4e)  %.1f s"
                % (ep, lh[-per:].mean(), lh[0], float(ident[:min(step, 8)].mean()), time.perf_counter() - t0))
    train.identity_loss = float(ident[:min(step, 8)].mean())
    out = losses[:step].cpu().numpy()
    net.check()
    return out


class TwoHop:
    """Buffers and the gradient of the unrolled two-hop loss: from the state in
    ws.x32 / ws.x16 the network predicts hop 1 and, from its own prediction,
    hop 2; the loss is MSE(hop 1, ws.t32) + MSE(hop 2, t2) and its gradient
    flows through the second hop back into the first (the second hop's input
    gradient joins the first hop's output gradient).  Leaves the summed
    gradients in net.gw / net.gb."""

    def __init__(self, ws):
        import torch as t
        self.ws = ws
        self.acts2 = [t.empty_like(a) for a in ws.acts]
        self.out1 = t.empty_like(ws.x32)
        self.x1_16 = t.empty_like(ws.x16)
        self.t2 = t.empty_like(ws.t32)
        self.dz2 = t.empty_like(ws.dz16)
        self.dx = t.empty_like(ws.x32)
        self.g1 = t.empty_like(ws.x32)
        self.gw_acc = self.gb_acc = None

    def grads(self, net, loss1, loss2):
        L = nn_lib()
        ws, B, H, W = self.ws, self.ws.B, self.ws.H, self.ws.W
        if self.gw_acc is None:
            self.gw_acc = [g.clone() for g in net.gw]
            self.gb_acc = [g.clone() for g in net.gb]
        net.forward(ws.x32, ws.x16, self.out1, ws.acts, B, H, W)
        _ck(L.lbm_nn_to_bf16(_p(self.out1), self.out1.numel(), _p(self.x1_16), net.s), "to_bf16")
        net.forward(self.out1, self.x1_16, ws.y32, self.acts2, B, H, W)
        # hop 2: weight gradients and the gradient at its input
        _ck(L.lbm_nn_mse(_p(ws.y32), _p(self.t2), USED, ws.P, _p(self.dz2), _p(ws.loss_part), _p(loss2),
                         net.s), "mse")
        net.backward(self.x1_16, self.acts2, self.dz2, ws.dbuf, ws.scratch, B, H, W, dx32=self.dx)
        for l in range(6):
            self.gw_acc[l].copy_(net.gw[l])
            self.gb_acc[l].copy_(net.gb[l])
        # hop 1: its own loss gradient plus what flows back from hop 2
        _ck(L.lbm_nn_mse(_p(self.out1), _p(ws.t32), USED, ws.P, _p(ws.dz16), _p(ws.loss_part), _p(loss1),
                         net.s), "mse")
        _ck(L.lbm_nn_to_f32(_p(ws.dz16), self.g1.numel(), _p(self.g1), net.s), "to_f32")
        _ck(L.lbm_nn_axpy(_p(self.g1), _p(self.dx), 1.0, self.g1.numel(), net.s), "axpy")
        _ck(L.lbm_nn_to_bf16(_p(self.g1), self.g1.numel(), _p(ws.dz16), net.s), "to_bf16")
        net.backward(ws.x16, ws.acts, ws.dz16, ws.dbuf, ws.scratch, B, H, W)
        for l in range(6):
            _ck(L.lbm_nn_axpy(_p(net.gw[l]), _p(self.gw_acc[l]), 1.0, net.gw[l].numel(), net.s), "axpy")
            _ck(L.lbm_nn_axpy(_p(net.gb[l]), _p(self.gb_acc[l]), 1.0, net.gb[l].numel(), net.s), "axpy")


def train_unrolled(sur: Surrogate, data, epochs=4, batch=16, lr=1e-3, seed=0, noise=0.03, log=print):
    """Adam on the unrolled two-hop loss (TwoHop) over all snapshot triples,
    the input corrupted by noise as in `train`; cosine learning-rate decay."""
    import torch
    t = torch
    net = sur.net
    n, S = data.shape[0], data.shape[1]
    H, W = data.shape[3], data.shape[4]
    ws = Workspace(batch, H, W, net.device, train=True, dilations=net.dil)
    two = TwoHop(ws)
    L = nn_lib()
    triples = np.array([(i, k) for i in range(n) for k in range(S - 2)])
    g = np.random.default_rng(seed)
    steps = epochs * (len(triples) // batch)
    losses = t.zeros(max(1, steps), dtype=t.float64, device=net.device)
    loss2 = t.zeros(max(1, steps), dtype=t.float64, device=net.device)
    step = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        order = g.permutation(len(triples))
        lr_ep = lr * (0.5 * (1.0 + math.cos(math.pi * ep / max(1, epochs))))
        for b0 in range(0, len(order) - batch + 1, batch):
            sel = triples[order[b0:b0 + batch]]
            ii = t.from_numpy(sel[:, 0]).to(net.device)
            kk = t.from_numpy(sel[:, 1]).to(net.device)
            sur.pack(data[ii, kk].contiguous(), ws, ws.x32)
            sur.pack(data[ii, kk + 1].contiguous(), ws, ws.t32)
            sur.pack(data[ii, kk + 2].contiguous(), ws, two.t2)
            if noise > 0:
                _ck(L.lbm_nn_add_noise(_p(ws.x32), ws.P, USED, noise, (seed * 1000003 + step) & 0xffffffff,
                                       net.s), "noise")
            _ck(L.lbm_nn_to_bf16(_p(ws.x32), ws.x32.numel(), _p(ws.x16), net.s), "to_bf16")
            two.grads(net, losses[step:step + 1], loss2[step:step + 1])
            net.adam(lr_ep)
            step += 1
        if log:
            net.check()
            per = max(1, len(order) // batch)
            lh, l2 = losses[:step].cpu().numpy(), loss2[:step].cpu().numpy()
            log("epoch %d: hop-1 loss %.4e, hop-2 loss %.4e  %.1f s"
                % (ep, lh[-per:].mean(), l2[-per:].mean(), time.perf_counter() - t0))
    out = (losses[:step] + loss2[:step]).cpu().numpy()
    net.check()
    return out


def field_rms_errors(got5, want5):
    """Per channel: RMS of got - want over all nodes and cases, in the scales of
    field_errors."""
    got5, want5 = np.asarray(got5, np.float64), np.asarray(want5, np.float64)
    speed = float(np.sqrt(want5[:, 1] ** 2 + want5[:, 2] ** 2).max())
    scales = [float(np.abs(want5[:, 0]).max()), speed, speed, float(np.abs(want5[:, 3]).max()),
              float(np.abs(want5[:, 4]).max())]
    return {c: float(np.sqrt(np.mean((got5[:, k] - want5[:, k]) ** 2)) / max(scales[k], 1e-30))
            for k, c in enumerate(CHANNELS)}


def field_errors(got5, want5):
    """Per channel: max |got - want| / max |want| (phi, C) or / max speed (u) or
    / max |p|, on host arrays [B, 5, H, W]."""
    got5, want5 = np.asarray(got5, np.float64), np.asarray(want5, np.float64)
    speed = float(np.sqrt(want5[:, 1] ** 2 + want5[:, 2] ** 2).max())
    scales = [float(np.abs(want5[:, 0]).max()), speed, speed, float(np.abs(want5[:, 3]).max()),
              float(np.abs(want5[:, 4]).max())]
    return {c: float(np.abs(got5[:, k] - want5[:, k]).max() / max(scales[k], 1e-30))
            for k, c in enumerate(CHANNELS)}


# Channels the judge compares: phi and C = c1 + c2, the transported fields.  A
# solver restarted from macroscopic fields (populations at equilibrium) rebuilds
# the acoustic part of p and u within the hop, so on those channels a restarted
# solver differs from the continuing one by up to 0.15 channel spreads even
# from the exact state (measured, `evaluate`'s restart_rms) and far more from a
# state whose pressure the network got slightly wrong.
JUDGED = (0, 4)
# Judge tolerance (RMS over the lattice, in channel spreads).  A solver hop
# restarted from a state's fields differs from the solver continuing from its
# populations by up to 0.075 spreads in C on 256 x 256 buoyant drops and
# bubbles (the split of C at the Henry equilibrium, the equilibrium
# populations); the tolerance sits above that floor.
JUDGE_TOL = 0.1
# A network trained on 2000 buoyant droplet and bubble trajectories of 256 x 256
# (flow_cases, seed 0), 9 snapshots each after 1024 warm-up steps, 48 epochs,
# pushforward 0.8, dilations 1, 2, 4, 8, 4, 2: the defaults of `train`.
MODEL_FLOW256 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "surrogate_flow256_d8.npz")


def rollout(sur: Surrogate, sims, hops, judge_every=0, tol=0.1, keq=None, judged=JUDGED, batch=None):
    """Advance the lattices `sims` (one shape, FP32) by `hops` network hops of
    16 steps.  With judge_every = m > 0 every m-th hop is checked on the
    channels `judged` (phi and C by default): the solver
    restarts from the state that hop started from (lbm_init_macros) and runs
    16 steps.  If every case's network hop lies within `tol` of the solver's (RMS
    over the lattice, in units of each channel's spread) the network's state
    becomes the verified state; otherwise the solver takes over from the last
    verified state (from its own populations when it produced that state, else
    restarted from the state's fields), runs up to the current hop, and its
    result is the new verified state.  The lattices' own states are overwritten.
    `batch` (optional): a Batch over `sims` to step them with (kept open);
    without one a Batch is built and closed here.  Returns (fields [B, 5, H, W]
    on the device: phi, ux, uy, p, C; stats)."""
    import torch
    net = sur.net
    B = len(sims)
    H, W = sims[0].ny, sims[0].nx
    ws = Workspace(B, H, W, net.device, train=False, dilations=net.dil)
    L = nn_lib()
    f6 = torch.empty((B, 6, H, W), dtype=torch.float32, device=net.device)
    own = batch is None and judge_every
    if own:
        batch = Batch(sims)
    if batch is not None:
        batch.fields(FIELDS6, f6)
    else:
        for j, s in enumerate(sims):
            s.fields(names=FIELDS6, dtype="f32", device=True, out=f6[j])
    sur.pack(f6, ws, ws.x32, ws.x16)
    stats = {"judged": 0, "fallbacks": 0, "solver_steps": 0}
    if judge_every:
        keq_t = torch.tensor([float(s.params["Keq"]) if keq is None else keq[j] for j, s in enumerate(sims)],
                             dtype=torch.float32, device=net.device)
        macros = torch.empty((B, 6, H, W), dtype=torch.float64, device=net.device)
        lb32 = torch.empty_like(ws.x32)
        ver32 = ws.x32.clone()
        ver_k = 0
        # the verified state as the solver's own populations, while it is one the
        # solver produced (None once a network state has been accepted)
        pop_buf = batch.get_state()
        ver_pop = True

        def solver(steps, out32, state32=None, pops=False):
            if pops:
                batch.set_state(pop_buf)
            else:
                _ck(L.lbm_nn_unpack_macros(_p(state32), B, H, W, _p(sur.shift), _p(sur.scale), _p(keq_t),
                                           _p(macros), net.s), "unpack_macros")
                batch.init_macros(macros)
            batch.step(steps)
            batch.fields(FIELDS6, f6)
            sur.pack(f6, ws, out32)
            stats["solver_steps"] += steps

    for k in range(1, hops + 1):
        sur.hop(ws)
        if judge_every and k % judge_every == 0:
            solver(HOP, lb32, state32=ws.x32)
            _ck(L.lbm_nn_state_diff(_p(ws.y32), _p(lb32), B, H * W, _p(ws.diff_part), _p(ws.diff), net.s), "diff")
            rms_all = ws.diff.view(B, 5, 2)[:, :, 1].cpu().numpy()
            rms = rms_all[:, list(judged)]
            stats["judged"] += 1
            stats.setdefault("judged_rms_max", []).append(float(np.nanmax(rms)) if np.isfinite(rms).any() else float("inf"))
            stats.setdefault("judged_rms_channels", []).append(
                {c: float(np.nanmax(rms_all[:, k])) for k, c in enumerate(CHANNELS)})
            if np.all(np.isfinite(rms_all)) and float(rms.max()) <= tol:
                ver32.copy_(ws.y32)
                ver_pop = False
            else:
                # the solver takes over from the last verified state, with its own
                # populations where it produced that state
                stats["fallbacks"] += 1
                solver(HOP * (k - ver_k), ws.y32, state32=ver32, pops=ver_pop)
                ver32.copy_(ws.y32)
                batch.get_state(pop_buf)
                ver_pop = True
            ver_k = k
        ws.x32, ws.y32 = ws.y32, ws.x32
        _ck(L.lbm_nn_to_bf16(_p(ws.x32), ws.x32.numel(), _p(ws.x16), net.s), "to_bf16")
    if own:
        batch.close()
    out5 = torch.empty((B, 5, H, W), dtype=torch.float32, device=net.device)
    sur.unpack(ws.x32, ws, out5)
    return out5, stats


def conv_flops(B, H, W):
    """Multiply-adds x 2 of one network hop (padding channels included)."""
    return 2.0 * B * H * W * 9 * sum(ci * co for ci, co in LAYERS)


def evaluate(sur: Surrogate, cases, hops=8, judge_every=4, tol=0.1, warm=64):
    """Speed and error of the network against the solver on `cases` (one shape):
    the solver alone (batched runner, 16 * hops steps), the network alone (hops
    hops), and the judged hybrid.  Errors are each field's max difference from
    the solver's result relative to the field's scale (see field_errors)."""
    import torch
    dev = sur.net.device
    stream = sur.net.stream

    def fresh():
        sims = [Simulation(w.params, precision="fp32", device=dev) for w in cases]
        for s, w in zip(sims, cases):
            s.init(w.sdf, w.c1_tilde, w.c2_tilde)
        b = Batch(sims)
        b.set_tiling(128, 32)
        b.step(warm)
        b.sync()
        return sims, b

    def timed(fn):
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return r, e0.elapsed_time(e1) * 1e-3

    H, W = cases[0].params["ny"], cases[0].params["nx"]
    B = len(cases)
    # the solver alone
    sims, b = fresh()
    _, t_lb = timed(lambda: b.step(HOP * hops))
    f6 = torch.empty((B, 6, H, W), dtype=torch.float32, device=dev)
    b.fields(FIELDS6, f6)
    truth = f6.cpu().numpy()
    truth5 = np.concatenate([truth[:, :4], truth[:, 4:5] + truth[:, 5:6]], axis=1)
    b.close()
    # the judge's own floor: one solver hop restarted from the fields (populations
    # at equilibrium, C split at the Henry equilibrium) against the solver
    # continuing from its populations, RMS in channel spreads as the judge measures
    L = nn_lib()
    sims_r, br = fresh()
    wsr = Workspace(B, H, W, dev, train=False, dilations=sur.net.dil)
    br.fields(FIELDS6, f6)
    sur.pack(f6, wsr, wsr.x32)
    keq_t = torch.tensor([float(s.params["Keq"]) for s in sims_r], dtype=torch.float32, device=dev)
    macros = torch.empty((B, 6, H, W), dtype=torch.float64, device=dev)
    _ck(L.lbm_nn_unpack_macros(_p(wsr.x32), B, H, W, _p(sur.shift), _p(sur.scale), _p(keq_t), _p(macros),
                               sur.net.s), "unpack_macros")
    br.step(HOP)
    br.fields(FIELDS6, f6)
    sur.pack(f6, wsr, wsr.y32)
    br.init_macros(macros)
    br.step(HOP)
    br.fields(FIELDS6, f6)
    lb32 = torch.empty_like(wsr.x32)
    sur.pack(f6, wsr, lb32)
    _ck(L.lbm_nn_state_diff(_p(wsr.y32), _p(lb32), B, H * W, _p(wsr.diff_part), _p(wsr.diff), sur.net.s), "diff")
    restart_rms = wsr.diff.view(B, 5, 2)[:, :, 1].cpu().numpy()
    br.close()
    del sims_r, wsr
    # the network alone (one untimed call first: allocations, first launches);
    # the batch built with the lattices serves both the network and the hybrid,
    # as the solver's own batch serves the solver
    sims, b = fresh()
    b.fields(FIELDS6, f6)
    start = f6.cpu().numpy()
    start5 = np.concatenate([start[:, :4], start[:, 4:5] + start[:, 5:6]], axis=1)
    rollout(sur, sims, 1, batch=b)
    (out, _), t_nn = timed(lambda: rollout(sur, sims, hops, batch=b))
    out_np = out.cpu().numpy()
    err_nn = field_errors(out_np, truth5)
    rms_nn = field_rms_errors(out_np, truth5)
    rms_none = field_rms_errors(start5, truth5)
    # judged hybrid (one untimed call first, as for the network, on separate
    # lattices: the judge and the fallback step the solver's state)
    sims_w, bw = fresh()
    rollout(sur, sims_w, judge_every, judge_every=judge_every, tol=tol, batch=bw)
    bw.close()
    del sims_w
    (out_h, st), t_h = timed(lambda: rollout(sur, sims, hops, judge_every=judge_every, tol=tol, batch=b))
    b.close()
    err_h = field_errors(out_h.cpu().numpy(), truth5)
    cells = B * H * W
    mlups = lambda t: cells * HOP * hops / t / 1e6
    # the hop's convolutions alone: achieved tensor throughput
    ws = Workspace(B, H, W, dev, train=False, dilations=sur.net.dil)
    sur.hop(ws)
    _, t_hop = timed(lambda: [sur.hop(ws) for _ in range(hops)])
    sur.net.check()
    return {
        "cases": B, "shape": [H, W], "hops": hops, "steps_per_hop": HOP,
        "solver_s": t_lb, "network_s": t_nn, "hybrid_s": t_h,
        "solver_mlups": mlups(t_lb), "network_mlups_equiv": mlups(t_nn), "hybrid_mlups_equiv": mlups(t_h),
        "speedup_network": t_lb / t_nn, "speedup_hybrid": t_lb / t_h,
        "error_network": err_nn, "error_network_rms": rms_nn, "error_no_change_rms": rms_none,
        "error_hybrid": err_h, "judge": dict(st, every=judge_every, tol=tol),
        "restart_rms_max": float(restart_rms.max()),
        "restart_rms_max_judged": float(restart_rms[:, list(JUDGED)].max()),
        "restart_rms_mean": {c: float(restart_rms[:, k].mean()) for k, c in enumerate(CHANNELS)},
        "conv_tflops": conv_flops(B, H, W) * hops / t_hop / 1e12,
    }


def conv_bench(B=16, H=256, W=256, launches=20, dilation=1, kind="fwd"):
    """Time one 48 -> 48 convolution alone (CUDA events): the forward ReLU
    convolution (kind "fwd"), the masked adjoint ("dgrad") or the weight
    gradient ("wgrad"); returns (ms per launch, TFLOP/s)."""
    import torch
    L = nn_lib()
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev).manual_seed(0)
    x = torch.randn((B, H, W, 48), generator=g, device=dev).to(torch.bfloat16)
    w = (0.05 * torch.randn((48, 9, 48), generator=g, device=dev)).to(torch.bfloat16)
    b = torch.zeros(48, dtype=torch.float32, device=dev)
    y = torch.empty_like(x)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    nb = L.lbm_nn_wgrad_partial_bytes(48, 48, B, H, W, dilation)
    part = torch.empty(nb // 4 + 1, dtype=torch.float32, device=dev)
    dw = torch.empty((48, 9, 48), dtype=torch.float32, device=dev)

    def run():
        if kind == "fwd":
            rc = L.lbm_nn_conv3x3(_p(x), 48, _p(w), _p(b), 48, RELU, None, None, _p(y), B, H, W, dilation, _p(st), s)
        elif kind == "dgrad":
            rc = L.lbm_nn_conv3x3(_p(x), 48, _p(w), None, 48, MASK, None, _p(x), _p(y), B, H, W, dilation, _p(st), s)
        else:
            rc = L.lbm_nn_conv3x3_wgrad(_p(x), 48, _p(x), 48, _p(dw), _p(part), nb, B, H, W, dilation, _p(st), s)
        _ck(rc, "conv")

    for _ in range(3):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(launches):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / launches
    if int(st.item()) != 0:
        raise LBMError(-6, "conv-bench: a wait on the tensor cores timed out")
    return ms, 2.0 * B * H * W * 9 * 48 * 48 / ms / 1e9


def main():
    import torch
    ap = argparse.ArgumentParser(description="train or evaluate the surrogate network")
    ap.add_argument("command", choices=["train", "evaluate", "conv-bench"])
    ap.add_argument("--model", default=MODEL_FLOW256, help="evaluate: a saved model (.npz)")
    ap.add_argument("--eval-cases", type=int, default=64)
    ap.add_argument("--hops", type=int, default=8)
    ap.add_argument("--warm", type=int, default=1024, help="solver steps before the first snapshot")
    ap.add_argument("--trajectories", type=int, default=2000)
    ap.add_argument("--snapshots", type=int, default=9)
    ap.add_argument("--epochs", type=int, default=48)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--side", type=int, default=256)
    ap.add_argument("--out", default="surrogate.npz")
    ap.add_argument("--dilation", type=int, default=1, help="conv-bench: dilation of the timed convolution")
    ap.add_argument("--pushforward", type=float, default=0.8,
                    help="train: fraction of batches (from the second epoch) fed the network's own hop")
    ap.add_argument("--data", choices=["flow", "droplets"], default="flow",
                    help="cases: buoyant droplets and bubbles (flow) or resting droplets")
    ap.add_argument("--dilations", default=",".join(str(d) for d in DILATIONS),
                    help="train: dilation of each of the six layers")
    ap.add_argument("--noise", type=float, default=0.03, help="train: input noise (normalised units)")
    ap.add_argument("--unroll", type=int, choices=[1, 2], default=1,
                    help="train: hops per loss (2: the second from the network's own prediction)")
    ap.add_argument("--finetune", type=int, default=0,
                    help="train: epochs of two-hop unrolled training after the one-hop epochs")
    ap.add_argument("--seed", type=int, default=0, help="train: weights and batch order")
    ap.add_argument("--judge-every", type=int, default=4)
    ap.add_argument("--tol", type=float, default=JUDGE_TOL, help="judge tolerance (RMS, channel spreads)")
    args = ap.parse_args()
    dev = torch.device("cuda", 0)
    make_cases = flow_cases if args.data == "flow" else droplet_cases
    if args.command == "conv-bench":
        for kind in ("fwd", "dgrad", "wgrad"):
            ms, tf = conv_bench(kind=kind, dilation=args.dilation)
            print("conv 48->48 %s, dilation %d, batch 16 of 256 x 256: %.4f ms, %.1f TFLOP/s"
                  % (kind, args.dilation, ms, tf))
        return
    if args.command == "evaluate":
        sur = Surrogate.load(args.model, dev)
        print(json.dumps(evaluate(sur, make_cases(args.eval_cases, 7, args.side), hops=args.hops,
                                  judge_every=args.judge_every, tol=args.tol, warm=args.warm)))
        return
    t0 = time.perf_counter()
    data = generate(make_cases(args.trajectories, 0, args.side), args.snapshots, dev, warm=args.warm)
    torch.cuda.synchronize()
    print("data: %d trajectories x %d snapshots in %.1f s" % (args.trajectories, args.snapshots,
                                                             time.perf_counter() - t0), flush=True)
    shift, scale = normalisation(data)
    dil = tuple(int(v) for v in args.dilations.split(","))
    sur = Surrogate(Net(dev, seed=args.seed, dilations=dil), shift, scale)
    if args.unroll == 2:
        losses = train_unrolled(sur, data, epochs=args.epochs, batch=args.batch, lr=args.lr, noise=args.noise,
                                seed=args.seed)
        train.identity_loss = float("nan")
    else:
        losses = train(sur, data, epochs=args.epochs, batch=args.batch, lr=args.lr,
                       pushforward=args.pushforward, noise=args.noise, seed=args.seed)
    if args.finetune:
        identity = train.identity_loss
        losses = np.concatenate([losses, train_unrolled(sur, data, epochs=args.finetune, batch=args.batch,
                                                        lr=0.3 * args.lr, noise=args.noise, seed=args.seed + 1)])
        train.identity_loss = identity
    sur.save(args.out)
    print(json.dumps({"trajectories": args.trajectories, "epochs": args.epochs, "first_loss": float(losses[0]),
                      "last_loss": float(losses[-100:].mean()), "no_change_loss": train.identity_loss,
                      "seconds": time.perf_counter() - t0}), flush=True)
    del data
    torch.cuda.empty_cache()
    print(json.dumps(evaluate(sur, make_cases(args.eval_cases, 7, args.side), hops=args.hops,
                              judge_every=args.judge_every, tol=args.tol, warm=args.warm)))


if __name__ == "__main__":
    main()
