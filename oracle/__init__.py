"""FP64 CPU oracle of the phase-field lattice Boltzmann step (arXiv 2402.15752).

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct restatement of
the paper's algorithm (Sec. III; see ``oracle.c`` for the equation map) that
the CUDA library is checked against.  Only the test suite, the package smoke
check and the benchmark's CPU-baseline leg load it; the CUDA path never
imports it and shares no code with it.

Parameters are a plain ``dict`` (the keys of ``PARAM_FIELDS``), the same
plain-data description that the CUDA binding consumes with its own struct.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

FIELDS = ("phi", "ux", "uy", "p", "c1", "c2", "rho", "mu")

PARAM_FIELDS = (
    ("nx", ctypes.c_int), ("ny", ctypes.c_int),
    ("wall_x", ctypes.c_int), ("wall_y", ctypes.c_int),
    ("scalar_q", ctypes.c_int),
    ("W", ctypes.c_double), ("M", ctypes.c_double), ("sigma", ctypes.c_double),
    ("rho1", ctypes.c_double), ("rho2", ctypes.c_double),
    ("mu1", ctypes.c_double), ("mu2", ctypes.c_double),
    ("D1", ctypes.c_double), ("D2", ctypes.c_double),
    ("Keq", ctypes.c_double), ("A", ctypes.c_double),
    ("gx", ctypes.c_double), ("gy", ctypes.c_double), ("g_rho_ref", ctypes.c_double),
    ("Fx", ctypes.c_double), ("Fy", ctypes.c_double),
    ("visc_model", ctypes.c_int), ("visc_beta", ctypes.c_double),
    ("scalar_model", ctypes.c_int), ("grad_scheme", ctypes.c_int),
)


class OrcParams(ctypes.Structure):
    _fields_ = list(PARAM_FIELDS)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain C11, FP64, no FMA contraction;
    OpenMP for the per-node loops when the compiler has it, else serial)."""
    srcs = (_SRC, os.path.join(_HERE, "oracle.h"))
    if not force and os.path.exists(_LIB) and all(
            os.path.getmtime(_LIB) >= os.path.getmtime(s) for s in srcs):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
            "-o", _LIB + ".tmp", _SRC, "-lm"]
    if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
        subprocess.run(base, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.POINTER(OrcParams)]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_init.argtypes = [ctypes.c_void_p, dp, ctypes.c_double, ctypes.c_double]
        L.orc_init_fields.argtypes = [ctypes.c_void_p, dp, dp, dp]
        L.orc_init_macros.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp, dp]
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
        L.orc_get_fields.argtypes = [ctypes.c_void_p, dp]
        L.orc_conserved.argtypes = [ctypes.c_void_p, dp]
        L.orc_get_stencils.argtypes = [ctypes.c_void_p, dp]
        L.orc_taus.argtypes = [ctypes.c_void_p, dp]
        L.orc_cell_functions.argtypes = [ctypes.POINTER(OrcParams), dp, dp]
        L.orc_solve_scalars.argtypes = [ctypes.POINTER(OrcParams), dp, dp]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_threads.restype = ctypes.c_int
        _lib = L
        set_threads(1)  # serial unless a caller asks for more
    return _lib


def set_threads(n: int) -> int:
    """Host threads of the oracle's per-node loops (results do not depend on
    it); returns the number now in use (1 without OpenMP)."""
    L = lib()
    L.orc_set_threads(int(n))
    return int(L.orc_threads())


DEFAULTS = dict(wall_x=0, wall_y=0, scalar_q=5, W=4.0, M=0.01, sigma=0.0,
                rho1=1.0, rho2=1.0, mu1=0.1, mu2=0.1, D1=0.1, D2=0.1, Keq=1.0, A=0.1,
                gx=0.0, gy=0.0, g_rho_ref=0.0, Fx=0.0, Fy=0.0, visc_model=0, visc_beta=0.0,
                scalar_model=0, grad_scheme=0)


def make_params(p: dict) -> OrcParams:
    q = dict(DEFAULTS)
    q.update(p)
    s = OrcParams()
    for name, ctype in PARAM_FIELDS:
        v = q[name]
        setattr(s, name, int(v) if ctype is ctypes.c_int else float(v))
    return s


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleSim:
    """One FP64 CPU simulation; fields are (ny, nx) float64 arrays."""

    def __init__(self, params: dict):
        self.params = dict(DEFAULTS)
        self.params.update(params)
        self._p = make_params(self.params)
        self.nx, self.ny = int(self.params["nx"]), int(self.params["ny"])
        h = lib().orc_create(ctypes.byref(self._p))
        if not h:
            raise ValueError("oracle rejected the parameters")
        self._h = ctypes.c_void_p(h)

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    __del__ = close

    def _grid(self, a) -> np.ndarray:
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        if a.shape != (self.ny, self.nx):
            a = np.ascontiguousarray(np.broadcast_to(a, (self.ny, self.nx)))
        return a

    def init(self, sdf, c1_tilde: float, c2_tilde: float):
        s = self._grid(sdf)
        lib().orc_init(self._h, _dptr(s), float(c1_tilde), float(c2_tilde))

    def init_fields(self, phi, c1, c2):
        a, b, c = self._grid(phi), self._grid(c1), self._grid(c2)
        lib().orc_init_fields(self._h, _dptr(a), _dptr(b), _dptr(c))

    def init_macros(self, phi, ux, uy, p, c1, c2):
        """Restart at the equilibria of the six given fields."""
        a = [self._grid(v) for v in (phi, ux, uy, p, c1, c2)]
        lib().orc_init_macros(self._h, *[_dptr(v) for v in a])

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    def fields(self) -> dict:
        out = np.empty((len(FIELDS), self.ny, self.nx), dtype=np.float64)
        lib().orc_get_fields(self._h, _dptr(out))
        return {k: out[i] for i, k in enumerate(FIELDS)}

    def stencils(self) -> dict:
        out = np.empty((7, self.ny, self.nx), dtype=np.float64)
        lib().orc_get_stencils(self._h, _dptr(out))
        names = ("dphix", "dphiy", "lap", "dc1x", "dc1y", "dc2x", "dc2y")
        return {k: out[i] for i, k in enumerate(names)}

    def conserved(self) -> np.ndarray:
        out = np.zeros(2)
        lib().orc_conserved(self._h, _dptr(out))
        return out

    def taus(self) -> np.ndarray:
        out = np.zeros(3)
        lib().orc_taus(self._h, _dptr(out))
        return out


CELL_INPUTS = ("phi", "ux", "uy", "p", "c1", "c2", "dphix", "dphiy", "lap",
               "dc1x", "dc1y", "dc2x", "dc2y", "dtpux", "dtpuy",
               "dtc1ux", "dtc1uy", "dtc2ux", "dtc2uy")
CELL_OUTPUTS = ("feq", "F", "geq", "G", "h1eq", "h2eq", "H1", "H2", "Ht1", "Ht2")


def cell_functions(params: dict, cell: dict) -> dict:
    """Per-cell discrete distributions (Eqs. 24-25, 29-31, 35-36) for given macros."""
    p = make_params(dict(params, nx=1, ny=1))
    inp = np.array([float(cell.get(k, 0.0)) for k in CELL_INPUTS])
    out = np.zeros(90)
    lib().orc_cell_functions(ctypes.byref(p), _dptr(inp), _dptr(out))
    return {k: out[9 * i:9 * i + 9].copy() for i, k in enumerate(CELL_OUTPUTS)}


def solve_scalars(params: dict, phi: float, P1: float, P2: float):
    """Exact 2x2 solve of the implicit scalar moments (Eq. 37)."""
    p = make_params(dict(params, nx=1, ny=1))
    inp = np.array([phi, P1, P2], dtype=np.float64)
    out = np.zeros(2)
    lib().orc_solve_scalars(ctypes.byref(p), _dptr(inp), _dptr(out))
    return float(out[0]), float(out[1])
