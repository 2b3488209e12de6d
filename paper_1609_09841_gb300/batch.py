"""Batched half steps: many independent simulations per persistent launch.

``BatchPlan(sims, prec, state)`` takes a list of dicts with keys m, grid
(n1, n2, n3), h (h1, h2, h3), c and dt (the FULL time step).  ``step`` runs one
half step of every simulation (one kernel launch); ``run`` runs nhalf half
steps as one captured CUDA graph.  Argument marshalling only."""
import ctypes

from . import capi
from .hermite import PRECISIONS, STATES, _stream


class BatchPlan:
    def __init__(self, sims, prec="fp32", state="fp32"):
        self.sims = [dict(s) for s in sims]
        self.prec, self.state = prec, state
        n = len(sims)
        I3, D3 = ctypes.c_int * (3 * n), ctypes.c_double * (3 * n)
        handle = ctypes.c_void_p()
        capi.check(capi.lib.hermite_batch_plan(
            ctypes.byref(handle), n, (ctypes.c_int * n)(*[int(s["m"]) for s in sims]),
            I3(*[int(v) for s in sims for v in s["grid"]]), D3(*[float(v) for s in sims for v in s["h"]]),
            (ctypes.c_double * n)(*[float(s["c"]) for s in sims]), (ctypes.c_double * n)(*[float(s["dt"]) for s in sims]),
            PRECISIONS[prec], STATES[state]))
        self._h = handle

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan destroyed")
        return self._h

    def __len__(self):
        return len(self.sims)

    def shape(self, i):
        M = self.sims[i]["m"] + 1
        g = self.sims[i]["grid"]
        return (2, M, M, M, g[2], g[1], g[0])

    def dof(self, i):
        return capi.lib.hermite_batch_elems(self.handle, i)

    def empty(self, device="cuda"):
        import torch
        dt = torch.float64 if self.state == "fp64" else torch.float32
        return [torch.empty(self.shape(i), dtype=dt, device=device) for i in range(len(self))]

    def _ptrs(self, xs):
        if len(xs) != len(self):
            raise ValueError("one state per simulation")
        dt = "float64" if self.state == "fp64" else "float32"
        for i, x in enumerate(xs):
            if (tuple(x.shape) != self.shape(i) or not x.is_cuda or not x.is_contiguous()
                    or str(x.dtype).replace("torch.", "") != dt):
                raise ValueError(f"state {i}: expected contiguous {dt} device tensor of shape {self.shape(i)}")
        return (ctypes.c_void_p * len(xs))(*[x.data_ptr() for x in xs])

    def step(self, ins, outs, parity, stream=None):
        capi.check(capi.lib.hermite_batch_step(self.handle, self._ptrs(ins), self._ptrs(outs), int(parity),
                                               _stream(stream)))
        return outs

    def run(self, a, b, nhalf, stream=None):
        """nhalf half steps from the primal grid; returns the buffer set holding the result."""
        capi.check(capi.lib.hermite_batch_run(self.handle, self._ptrs(a), self._ptrs(b), int(nhalf), _stream(stream)))
        return a if nhalf % 2 == 0 else b

    def set_schedule(self, zchunk):
        capi.check(capi.lib.hermite_batch_set_schedule(self.handle, (ctypes.c_int * 3)(*[int(v) for v in zchunk])))

    def set_tiles(self, tile):
        """Tile shape index (0 or 1) per order 1, 2, 3."""
        capi.check(capi.lib.hermite_batch_set_tiles(self.handle, (ctypes.c_int * 3)(*[int(v) for v in tile])))

    @staticmethod
    def tile_shape(m, tile):
        """(tx, ty) of the batched kernel's tile shape `tile` of order m."""
        tx, ty = ctypes.c_int(), ctypes.c_int()
        capi.check(capi.lib.hermite_batch_tile_shape(int(m), int(tile), ctypes.byref(tx), ctypes.byref(ty)))
        return tx.value, ty.value

    def close(self):
        if self._h is not None:
            capi.lib.hermite_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
