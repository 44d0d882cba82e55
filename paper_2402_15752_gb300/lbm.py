"""ctypes binding of liblbm (include/lbm.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels; PyTorch supplies
the device workspace (a uint8 CUDA tensor) and the CUDA stream.  There is no
CPU fallback: if liblbm.so is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# LBM_DEBUG=1 in the environment selects the debug build (liblbm_debug.so:
# every kernel access of the workspace checked, lbm_sync reports LBM_ERR_BOUNDS)
LIB_PATH = os.path.join(_PKG, "liblbm_debug.so" if os.environ.get("LBM_DEBUG") == "1" else "liblbm.so")

# ---- constants mirrored from include/lbm.h ----
LBM_OK = 0
LBM_ERR_ARG = -1
LBM_ERR_UNSTABLE_TAU = -2
LBM_ERR_WORKSPACE = -3
LBM_ERR_CUDA = -4
LBM_ERR_NONFINITE = -5
LBM_ERR_TIMEOUT = -6
LBM_ERR_BOUNDS = -7
ERROR_NAMES = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_UNSTABLE_TAU", -3: "LBM_ERR_WORKSPACE",
               -4: "LBM_ERR_CUDA", -5: "LBM_ERR_NONFINITE", -6: "LBM_ERR_TIMEOUT",
               -7: "LBM_ERR_BOUNDS"}

LBM_BC_PERIODIC, LBM_BC_WALL = 0, 1
LBM_FP64, LBM_FP32, LBM_FP32_BF16STORE, LBM_FP32_FP16STORE = 0, 1, 2, 3
# storage of the populations; the arithmetic is FP64 for "fp64", else FP32
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "bf16": LBM_FP32_BF16STORE, "fp16": LBM_FP32_FP16STORE}
LBM_VISC_LINEAR, LBM_VISC_LOG_C, LBM_VISC_EXP_T = 0, 1, 2
FIELDS = ("phi", "ux", "uy", "p", "c1", "c2", "rho", "mu")
FIELD_BITS = {name: 1 << i for i, name in enumerate(FIELDS)}
LBM_FIELD_ALL = 0xFF
LBM_OUT_F64, LBM_OUT_F32 = 0, 1


class LBMParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32),
        ("scalar_q", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("W", ctypes.c_double), ("M", ctypes.c_double), ("sigma", ctypes.c_double),
        ("rho1", ctypes.c_double), ("rho2", ctypes.c_double),
        ("mu1", ctypes.c_double), ("mu2", ctypes.c_double),
        ("D1", ctypes.c_double), ("D2", ctypes.c_double),
        ("Keq", ctypes.c_double), ("A", ctypes.c_double),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double), ("g_rho_ref", ctypes.c_double),
        ("Fx", ctypes.c_double), ("Fy", ctypes.c_double),
        ("visc_model", ctypes.c_int32), ("visc_beta", ctypes.c_double),
        ("scalar_model", ctypes.c_int32), ("grad_scheme", ctypes.c_int32),
    ]


class LBMError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__("%s (%d): %s" % (ERROR_NAMES.get(code, "?"), code, message))
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblbm.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("liblbm.so not found at %s: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    L = ctypes.CDLL(path)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    dp = ctypes.c_void_p  # pointers are passed as integers (host or device)
    P = ctypes.POINTER(LBMParams)
    sig = {
        "lbm_workspace_bytes": (sz, [P]),
        "lbm_create": (ctypes.c_int, [P, vp, sz, vp, ctypes.POINTER(vp)]),
        "lbm_init": (ctypes.c_int, [vp, dp, i32, ctypes.c_double, ctypes.c_double]),
        "lbm_init_fields": (ctypes.c_int, [vp, dp, dp, dp, i32]),
        "lbm_init_macros": (ctypes.c_int, [vp, dp, dp, dp, dp, dp, dp, i32]),
        "lbm_step": (ctypes.c_int, [vp, i64]),
        "lbm_get_fields": (ctypes.c_int, [vp, ctypes.c_uint32, dp, i32, i32]),
        "lbm_conserved": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_double)]),
        "lbm_sync": (ctypes.c_int, [vp]),
        "lbm_debug_build": (ctypes.c_int, []),
        "lbm_debug_limit_workspace": (ctypes.c_int, [vp, sz]),
        "lbm_state_bytes": (sz, [vp]),
        "lbm_get_state": (ctypes.c_int, [vp, dp, sz, i32]),
        "lbm_set_state": (ctypes.c_int, [vp, dp, sz, i32]),
        "lbm_time": (i64, [vp]),
        "lbm_destroy": (None, [vp]),
        "lbm_last_error": (ctypes.c_char_p, [vp]),
        "lbm_conserved_noalloc": (ctypes.c_int, [P, dp, sz, vp, dp, i32, ctypes.c_char_p, sz]),
        "lbm_batch_workspace_bytes": (sz, [ctypes.POINTER(vp), i32]),
        "lbm_batch_create": (ctypes.c_int, [ctypes.POINTER(vp), i32, vp, sz, ctypes.POINTER(vp)]),
        "lbm_batch_set_tiling": (ctypes.c_int, [vp, i32, i32]),
        "lbm_batch_tiling": (ctypes.c_int, [vp] + [ctypes.POINTER(i32)] * 4),
        "lbm_batch_step": (ctypes.c_int, [vp, i64]),
        "lbm_batch_sync": (ctypes.c_int, [vp]),
        "lbm_batch_autotune": (ctypes.c_int, [vp, i32, ctypes.POINTER(ctypes.c_double), i32,
                                              ctypes.POINTER(i32)]),
        "lbm_batch_set_wait_limit": (ctypes.c_int, [vp, i64, i32]),
        "lbm_batch_init_macros": (ctypes.c_int, [vp, vp, i32]),
        "lbm_batch_get_fields": (ctypes.c_int, [vp, ctypes.c_uint32, vp, i32, i32]),
        "lbm_batch_state_bytes": (sz, [vp]),
        "lbm_batch_get_state": (ctypes.c_int, [vp, vp, sz, i32]),
        "lbm_batch_set_state": (ctypes.c_int, [vp, vp, sz, i32]),
        "lbm_batch_destroy": (None, [vp]),
        "lbm_batch_last_error": (ctypes.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


DEFAULTS = dict(wall_x=0, wall_y=0, scalar_q=5, W=4.0, M=0.01, sigma=0.0,
                rho1=1.0, rho2=1.0, mu1=0.1, mu2=0.1, D1=0.1, D2=0.1, Keq=1.0, A=0.1,
                gx=0.0, gy=0.0, g_rho_ref=0.0, Fx=0.0, Fy=0.0, visc_model=0, visc_beta=0.0,
                scalar_model=0, grad_scheme=0)


def make_params(params: dict, precision: str = "fp32") -> LBMParams:
    """Plain parameter dict (lattice units) -> lbm_params."""
    q = dict(DEFAULTS)
    q.update(params)
    s = LBMParams()
    s.nx, s.ny = int(q["nx"]), int(q["ny"])
    s.bc_x = LBM_BC_WALL if q["wall_x"] else LBM_BC_PERIODIC
    s.bc_y = LBM_BC_WALL if q["wall_y"] else LBM_BC_PERIODIC
    s.scalar_q = int(q["scalar_q"])
    s.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    for k in ("W", "M", "sigma", "rho1", "rho2", "mu1", "mu2", "D1", "D2", "Keq", "A",
              "gx", "gy", "g_rho_ref", "Fx", "Fy", "visc_beta"):
        setattr(s, k, float(q[k]))
    s.visc_model = int(q["visc_model"])
    s.scalar_model = int(q["scalar_model"])
    s.grad_scheme = int(q["grad_scheme"])
    return s


def _check(L, h, rc):
    if rc != LBM_OK:
        msg = L.lbm_last_error(h)
        raise LBMError(rc, msg.decode() if msg else "")


def workspace_bytes(params: dict, precision: str = "fp32") -> int:
    L = load_library()
    p = make_params(params, precision)
    n = L.lbm_workspace_bytes(ctypes.byref(p))
    if n == 0:
        raise LBMError(LBM_ERR_ARG, L.lbm_last_error(None).decode())
    return int(n)


class Simulation:
    """One solver instance on one GPU.

    params    -- plain dict of lattice-unit parameters (see workloads.BASE)
    precision -- population storage: "fp64", "fp32", or "bf16"/"fp16" (16-bit
                 storage, FP32 arithmetic)
    device    -- torch device (default: current CUDA device)
    stream    -- torch.cuda.Stream (default: the current stream of the device)
    """

    def __init__(self, params: dict, precision: str = "fp32", device=None, stream=None):
        import torch
        self._torch = torch
        self.L = load_library()
        self.params = dict(DEFAULTS)
        self.params.update(params)
        self.precision = precision
        self.nx, self.ny = int(self.params["nx"]), int(self.params["ny"])
        self._p = make_params(self.params, precision)
        nbytes = self.L.lbm_workspace_bytes(ctypes.byref(self._p))
        if nbytes == 0:
            # validation failed: lbm_create reports the specific code before any GPU use
            rc = self.L.lbm_create(ctypes.byref(self._p), None, 0, None, ctypes.byref(ctypes.c_void_p()))
            raise LBMError(rc if rc != LBM_OK else LBM_ERR_ARG, self.L.lbm_last_error(None).decode())
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        rc = self.L.lbm_create(ctypes.byref(self._p), ctypes.c_void_p(self.workspace.data_ptr()),
                               ctypes.c_size_t(nbytes), ctypes.c_void_p(self.stream.cuda_stream),
                               ctypes.byref(h))
        if rc != LBM_OK:
            raise LBMError(rc, self.L.lbm_last_error(None).decode())
        self._h = h

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None):
            self.L.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers --
    def _host_grid(self, a) -> np.ndarray:
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        if a.shape != (self.ny, self.nx):
            a = np.ascontiguousarray(np.broadcast_to(a, (self.ny, self.nx)))
        return a

    def _ptr(self, a):
        """(pointer, on_device, keepalive) for a numpy array or a torch tensor."""
        t = self._torch
        if isinstance(a, t.Tensor):
            if a.is_cuda:
                a = a.to(t.float64).contiguous()
                assert a.numel() == self.nx * self.ny
                return a.data_ptr(), 1, a
            a = a.numpy()
        a = self._host_grid(a)
        return a.ctypes.data, 0, a

    # -- API --
    def init(self, sdf, c1_tilde: float, c2_tilde: float):
        p, dev, keep = self._ptr(sdf)
        _check(self.L, self._h, self.L.lbm_init(self._h, p, dev, float(c1_tilde), float(c2_tilde)))
        self._keep = keep

    def init_fields(self, phi, c1, c2):
        a, b, c = self._ptr(phi), self._ptr(c1), self._ptr(c2)
        if len({a[1], b[1], c[1]}) != 1:
            raise ValueError("phi, c1, c2 must all be on the host or all on the device")
        _check(self.L, self._h, self.L.lbm_init_fields(self._h, a[0], b[0], c[0], a[1]))
        self._keep = (a[2], b[2], c[2])

    def init_macros(self, phi, ux, uy, p, c1, c2):
        """Restart at the equilibria of all six macroscopic fields (host or device)."""
        a = [self._ptr(v) for v in (phi, ux, uy, p, c1, c2)]
        if len({v[1] for v in a}) != 1:
            raise ValueError("the six fields must all be on the host or all on the device")
        _check(self.L, self._h, self.L.lbm_init_macros(self._h, *[v[0] for v in a], a[0][1]))
        self._keep = tuple(v[2] for v in a)

    def step(self, n: int = 1):
        _check(self.L, self._h, self.L.lbm_step(self._h, int(n)))

    def sync(self):
        _check(self.L, self._h, self.L.lbm_sync(self._h))

    @property
    def time(self) -> int:
        return int(self.L.lbm_time(self._h))

    def fields(self, names=FIELDS, dtype="f64", device: bool = False, out=None) -> dict:
        """Macroscopic fields as (ny, nx) arrays: numpy on the host (synchronous)
        or torch tensors on the device (asynchronous on the stream)."""
        names = [n for n in FIELDS if n in names]
        mask = 0
        for n in names:
            mask |= FIELD_BITS[n]
        f64 = dtype in ("f64", "float64", np.float64)
        code = LBM_OUT_F64 if f64 else LBM_OUT_F32
        if device:
            t = self._torch
            if out is None:
                out = t.empty((len(names), self.ny, self.nx), device=self.device,
                              dtype=t.float64 if f64 else t.float32)
            _check(self.L, self._h, self.L.lbm_get_fields(self._h, mask, out.data_ptr(), 1, code))
        else:
            if out is None:
                out = np.empty((len(names), self.ny, self.nx), dtype=np.float64 if f64 else np.float32)
            _check(self.L, self._h, self.L.lbm_get_fields(self._h, mask, out.ctypes.data, 0, code))
        return {n: out[i] for i, n in enumerate(names)}

    def conserved(self) -> np.ndarray:
        out = (ctypes.c_double * 2)()
        _check(self.L, self._h, self.L.lbm_conserved(self._h, out))
        return np.array([out[0], out[1]])

    def state_bytes(self) -> int:
        return int(self.L.lbm_state_bytes(self._h))

    def get_state(self, device: bool = False):
        n = self.state_bytes()
        if device:
            buf = self._torch.empty(n, dtype=self._torch.uint8, device=self.device)
            _check(self.L, self._h, self.L.lbm_get_state(self._h, buf.data_ptr(), n, 1))
        else:
            buf = np.empty(n, dtype=np.uint8)
            _check(self.L, self._h, self.L.lbm_get_state(self._h, buf.ctypes.data, n, 0))
        return buf

    def set_state(self, buf):
        t = self._torch
        if isinstance(buf, t.Tensor) and buf.is_cuda:
            _check(self.L, self._h, self.L.lbm_set_state(self._h, buf.data_ptr(), buf.numel(), 1))
        else:
            b = np.ascontiguousarray(buf, dtype=np.uint8)
            _check(self.L, self._h, self.L.lbm_set_state(self._h, b.ctypes.data, b.size, 0))
