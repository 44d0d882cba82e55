"""Batched runner: many independent FP32 lattices (Simulation objects) advanced
together by the library's persistent batched kernel (lbm_batch_* in lbm.h).

Argument marshalling only: the tile tables, the launch and the autotuner's
timing loop are in the library.  The autotuner's choice can be cached in a
JSON file keyed by the GPU and the batch's shapes.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os

from .lbm import FIELD_BITS, FIELDS, LBM_OK, LBM_OUT_F32, LBM_OUT_F64, LBMError, Simulation, load_library


def _check(L, b, rc):
    if rc != LBM_OK:
        msg = L.lbm_batch_last_error(b)
        raise LBMError(rc, msg.decode() if msg else "")


class Batch:
    """A batch over `sims` (all "fp32", one scalar_q, one device and stream).

    The Simulation objects stay usable for init, fields, conserved and state;
    step them through the batch.  Close the batch before the simulations."""

    def __init__(self, sims: list[Simulation]):
        import torch
        self._torch = torch
        self.L = load_library()
        self.sims = list(sims)
        n = len(self.sims)
        self._arr = (ctypes.c_void_p * n)(*[s._h.value for s in self.sims])
        nbytes = self.L.lbm_batch_workspace_bytes(self._arr, n)
        if nbytes == 0:
            raise LBMError(-1, self.L.lbm_batch_last_error(None).decode())
        dev = self.sims[0].device
        self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=dev)
        b = ctypes.c_void_p()
        rc = self.L.lbm_batch_create(self._arr, n, ctypes.c_void_p(self.workspace.data_ptr()),
                                     ctypes.c_size_t(nbytes), ctypes.byref(b))
        if rc != LBM_OK:
            raise LBMError(rc, self.L.lbm_batch_last_error(None).decode())
        self._b = b

    def close(self):
        if getattr(self, "_b", None):
            self.L.lbm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def cells(self) -> int:
        return sum(s.nx * s.ny for s in self.sims)

    def step(self, n: int = 1):
        _check(self.L, self._b, self.L.lbm_batch_step(self._b, int(n)))

    def sync(self):
        _check(self.L, self._b, self.L.lbm_batch_sync(self._b))

    def init_macros(self, macros):
        """Restart every case at the equilibria of its fields: `macros` is a
        contiguous FP64 device tensor holding, case after case, the six (ny, nx)
        fields phi, ux, uy, p, c1, c2 (shape [B, 6, ny, nx] when all cases share
        a shape).  Asynchronous on the stream."""
        assert macros.is_cuda and macros.dtype == self._torch.float64 and macros.is_contiguous()
        assert macros.numel() == 6 * self.cells
        _check(self.L, self._b, self.L.lbm_batch_init_macros(self._b, macros.data_ptr(), 1))

    def fields(self, names, out):
        """The selected fields of every case into the contiguous FP32 or FP64
        device tensor `out` (case after case, fields in the library's order;
        shape [B, k, ny, nx] when all cases share a shape).  Asynchronous."""
        names = [n for n in FIELDS if n in names]
        mask = 0
        for n in names:
            mask |= FIELD_BITS[n]
        t = self._torch
        assert out.is_cuda and out.is_contiguous() and out.numel() == len(names) * self.cells
        code = LBM_OUT_F64 if out.dtype == t.float64 else LBM_OUT_F32
        assert out.dtype in (t.float64, t.float32)
        _check(self.L, self._b, self.L.lbm_batch_get_fields(self._b, mask, out.data_ptr(), 1, code))
        return out

    def state_bytes(self) -> int:
        return int(self.L.lbm_batch_state_bytes(self._b))

    def get_state(self, out=None):
        """Every case's checkpoint into one device buffer (uint8, allocated when
        `out` is None).  Asynchronous on the stream."""
        n = self.state_bytes()
        if out is None:
            out = self._torch.empty(n, dtype=self._torch.uint8, device=self.sims[0].device)
        _check(self.L, self._b, self.L.lbm_batch_get_state(self._b, out.data_ptr(), out.numel(), 1))
        return out

    def set_state(self, buf):
        """Restore every case from a buffer written by get_state (asynchronous)."""
        _check(self.L, self._b, self.L.lbm_batch_set_state(self._b, buf.data_ptr(), buf.numel(), 1))

    def set_tiling(self, tile_w: int, tile_h: int):
        _check(self.L, self._b, self.L.lbm_batch_set_tiling(self._b, int(tile_w), int(tile_h)))

    def tiling(self) -> dict:
        v = [ctypes.c_int32() for _ in range(4)]
        _check(self.L, self._b, self.L.lbm_batch_tiling(self._b, *[ctypes.byref(x) for x in v]))
        return dict(tile_w=v[0].value, tile_h=v[1].value, tiles=v[2].value, ctas=v[3].value)

    def set_wait_limit(self, spin_limit: int, hold_tile: int = -1):
        _check(self.L, self._b, self.L.lbm_batch_set_wait_limit(self._b, int(spin_limit), int(hold_tile)))

    def signature(self) -> str:
        """Key of the autotuner cache: GPU, scalar lattice, and the multiset of shapes."""
        import torch
        props = torch.cuda.get_device_properties(self.sims[0].device)
        shapes = sorted((s.nx, s.ny, int(s.params["wall_x"]), int(s.params["wall_y"])) for s in self.sims)
        raw = json.dumps([props.name, props.multi_processor_count, int(self.sims[0].params["scalar_q"]), shapes])
        return hashlib.sha256(raw.encode()).hexdigest()[:16]

    def autotune(self, steps_per_trial: int = 20, cache: str | None = None) -> dict:
        """Pick the fastest tiling by timing each candidate (the trial steps are
        real steps of every case).  With `cache`, a JSON file, a choice stored for
        the same signature is applied without timing, and a new one is stored."""
        key = self.signature()
        if cache and os.path.exists(cache):
            with open(cache) as f:
                known = json.load(f)
            if key in known:
                self.set_tiling(known[key]["tile_w"], known[key]["tile_h"])
                return dict(known[key], cached=True)
        rows = 12
        table = (ctypes.c_double * (5 * rows))()
        written = ctypes.c_int32()
        _check(self.L, self._b, self.L.lbm_batch_autotune(self._b, int(steps_per_trial), table, rows,
                                                          ctypes.byref(written)))
        trials = [dict(tile_w=int(table[5 * r]), tile_h=int(table[5 * r + 1]),
                       ms_per_step=table[5 * r + 2], tiles=int(table[5 * r + 3]),
                       ctas=int(table[5 * r + 4])) for r in range(written.value)]
        choice = dict(self.tiling(), trials=trials, cached=False)
        if cache:
            known = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    known = json.load(f)
            known[key] = {"tile_w": choice["tile_w"], "tile_h": choice["tile_h"]}
            with open(cache, "w") as f:
                json.dump(known, f, indent=1, sort_keys=True)
        return choice
