"""Python front end of libhermite (argument marshalling only).

Device states are torch tensors (torch provides device memory and the current
CUDA stream); host states are numpy arrays or CPU tensors.  Every arithmetic
step of the half step runs in the CUDA library.
"""
import ctypes

import numpy as np

from . import capi

PRECISIONS = {"fp64": capi.HERMITE_FP64, "fp32": capi.HERMITE_FP32, "hybrid64": capi.HERMITE_HYBRID64,
              "hybriddf": capi.HERMITE_HYBRIDDF, "3xtf32": capi.HERMITE_3XTF32,
              "splitbf16": capi.HERMITE_SPLITBF16, "remainder": capi.HERMITE_REMAINDER}
STATES = {"fp64": capi.HERMITE_STATE_FP64, "fp32": capi.HERMITE_STATE_FP32}
VARIANTS = {"auto": capi.HERMITE_AUTO, "fused": capi.HERMITE_FUSED, "split": capi.HERMITE_SPLIT}


def stability_limit(m, q=4):
    """Largest c*(dt/2)/h with a stable half step of order m and q Taylor
    stages (q = 4 is RK4)."""
    return capi.lib.hermite_stability_limit_taylor(int(m), int(q))


def _ptr(x):
    """(address, is_device) of a contiguous torch tensor or numpy array."""
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("state arrays must be C-contiguous")
        return x.ctypes.data, False
    if not x.is_contiguous():
        raise ValueError("state tensors must be contiguous")
    return x.data_ptr(), x.is_cuda


def _is_fp64(x):
    """True for a float64 array or tensor, False for float32; anything else
    is rejected (the library reads exactly the plan's element type, so a
    buffer of another type would be read out of its bounds or misread)."""
    name = str(x.dtype).replace("torch.", "")
    if name == "float64":
        return True
    if name == "float32":
        return False
    raise ValueError(f"dtype {x.dtype}: expected float32 or float64")


def _need(x, dtype, count, what):
    """A contiguous device tensor of `dtype` (a torch dtype name) with at
    least `count` elements."""
    if str(x.dtype).replace("torch.", "") != dtype or not getattr(x, "is_cuda", False) or not x.is_contiguous():
        raise ValueError(f"{what}: expected a contiguous {dtype} device tensor")
    if x.numel() < count:
        raise ValueError(f"{what}: {x.numel()} elements, {count} needed")


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Plan:
    """A half-step plan: order m, periodic grid (n1, n2, n3), spacings h, wave
    speed c and FULL time step dt (each step advances dt / 2); q Taylor stages
    of the local evolution (4 = RK4, up to 3(2m+1))."""

    def __init__(self, m, grid, h, c, dt, prec="fp64", state="fp64", variant="auto", q=4):
        self.m, self.grid, self.h = int(m), tuple(int(v) for v in grid), tuple(float(v) for v in h)
        self.c, self.dt, self.prec, self.state, self.variant = float(c), float(dt), prec, state, variant
        handle = ctypes.c_void_p()
        capi.check(capi.lib.hermite_plan_taylor(ctypes.byref(handle), self.m, (ctypes.c_int * 3)(*self.grid),
                                                (ctypes.c_double * 3)(*self.h), self.c, self.dt,
                                                PRECISIONS[prec], STATES[state], VARIANTS[variant], int(q)))
        self._h = handle

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan destroyed")
        return self._h

    @property
    def shape(self):
        M = self.m + 1
        return (2, M, M, M, self.grid[2], self.grid[1], self.grid[0])

    @property
    def elems(self):
        return capi.lib.hermite_state_elems(self.handle)

    @property
    def torch_dtype(self):
        import torch
        return torch.float64 if self.state == "fp64" else torch.float32

    def empty(self, device="cuda"):
        import torch
        return torch.empty(self.shape, dtype=self.torch_dtype, device=device)

    def set_taylor_order(self, q):
        """Stages of the local Taylor evolution (4 = RK4, up to 3(2m+1))."""
        capi.check(capi.lib.hermite_set_taylor_order(self.handle, int(q)))

    @property
    def taylor_order(self):
        return capi.lib.hermite_taylor_order(self.handle)

    def schedule_count(self):
        return capi.lib.hermite_schedule_count(self.handle)

    def set_schedule(self, tile, zchunk):
        capi.check(capi.lib.hermite_set_schedule(self.handle, int(tile), int(zchunk)))

    def operator(self):
        P = 2 * self.m + 2
        out = (ctypes.c_double * (P * P))()
        capi.check(capi.lib.hermite_plan_operator(self.handle, out))
        return np.array(out).reshape(P, P)

    def _check(self, *xs):
        """Every x is a state of this plan: its shape and its element type."""
        for x in xs:
            if tuple(x.shape) != self.shape:
                raise ValueError(f"state shape {tuple(x.shape)} != {self.shape}")
            if _is_fp64(x) != (self.state == "fp64"):
                raise ValueError(f"state dtype {x.dtype} does not match the plan's {self.state} state")

    @staticmethod
    def _out_and_parity(x_in, x_out, parity):
        """(x_out, parity) of a call written f(x, y, parity) or f(x, parity),
        the second allocating the output like x."""
        if parity is None:
            if not isinstance(x_out, (int, np.integer)):
                raise TypeError("expected (x_in, x_out, parity) or (x_in, parity)")
            parity = x_out
            x_out = np.empty_like(x_in) if isinstance(x_in, np.ndarray) else x_in.new_empty(x_in.shape)
        return x_out, parity

    def step(self, x_in, x_out, parity=None, stream=None):
        """x_out = S_parity(x_in) (device tensors: enqueued; host arrays: synchronous).
        ``step(x, parity)`` allocates the output and returns it."""
        x_out, parity = self._out_and_parity(x_in, x_out, parity)
        self._check(x_in, x_out)
        pi, di = _ptr(x_in)
        po, do = _ptr(x_out)
        st = _stream(stream) if (di or do) else ctypes.c_void_p(int(stream or 0))
        capi.check(capi.lib.hermite_step(self.handle, ctypes.c_void_p(pi), ctypes.c_void_p(po), int(parity), st))
        return x_out

    def adjoint(self, g_out, g_in, parity=None, stream=None):
        """g_in = S_parity^T g_out (device tensors); ``adjoint(g, parity)``
        allocates g_in and returns it."""
        g_in, parity = self._out_and_parity(g_out, g_in, parity)
        self._check(g_out, g_in)
        capi.check(capi.lib.hermite_adjoint_step(self.handle, ctypes.c_void_p(_ptr(g_out)[0]),
                                                 ctypes.c_void_p(_ptr(g_in)[0]), int(parity), _stream(stream)))
        return g_in

    def step_dc(self, x_in, x_out, parity, stream=None):
        """x_out = (dS_parity/dc) x_in (device tensors)."""
        self._check(x_in, x_out)
        capi.check(capi.lib.hermite_step_dc(self.handle, ctypes.c_void_p(_ptr(x_in)[0]),
                                            ctypes.c_void_p(_ptr(x_out)[0]), int(parity), _stream(stream)))
        return x_out

    def device_status(self, stream=None):
        """Flags raised by the plan's kernels since the last call (0: none),
        then cleared; bit 0: a CTA gave up a bounded wait (a tensor-core CTA
        waiting for its MMAs, a staged CTA waiting for a plane's copy)."""
        out = ctypes.c_int()
        capi.check(capi.lib.hermite_device_status(self.handle, ctypes.byref(out), _stream(stream)))
        return out.value

    def dot(self, a, b, stream=None):
        """FP64 sum of a * b over every entry of two device states."""
        self._check(a, b)
        out = ctypes.c_double()
        capi.check(capi.lib.hermite_dot(self.handle, ctypes.c_void_p(_ptr(a)[0]), ctypes.c_void_p(_ptr(b)[0]),
                                        ctypes.byref(out), _stream(stream)))
        return out.value

    def record(self, x, idx, out, stream=None):
        """out[k] (FP64 device) = value of u at flat node idx[k] (int64 device)."""
        self._check(x)
        _need(idx, "int64", 0, "receiver indices")
        _need(out, "float64", idx.numel(), "receiver values")
        capi.check(capi.lib.hermite_record(self.handle, ctypes.c_void_p(_ptr(x)[0]), ctypes.c_void_p(idx.data_ptr()),
                                           int(idx.numel()), ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def inject(self, adj, idx, w, stream=None):
        """adj[u value at idx[k]] += w[k] (the transpose of record)."""
        self._check(adj)
        _need(idx, "int64", 0, "receiver indices")
        _need(w, "float64", idx.numel(), "receiver weights")
        capi.check(capi.lib.hermite_inject(self.handle, ctypes.c_void_p(_ptr(adj)[0]), ctypes.c_void_p(idx.data_ptr()),
                                           int(idx.numel()), ctypes.c_void_p(w.data_ptr()), _stream(stream)))
        return adj

    def error(self, x, ref, mask=0b111, stream=None):
        """(max_abs, max_rel, l2_abs, l2_rel) of x - ref (ref FP64, device tensors)."""
        self._check(x)
        if tuple(ref.shape) != self.shape or not _is_fp64(ref):
            raise ValueError(f"ref must be a float64 state of shape {self.shape}")
        out = (ctypes.c_double * 4)()
        rc = capi.lib.hermite_error(self.handle, ctypes.c_void_p(_ptr(x)[0]), ctypes.c_void_p(_ptr(ref)[0]),
                                    int(mask), out, _stream(stream))
        if rc not in (capi.HERMITE_OK, capi.HERMITE_ENONFINITE):
            capi.check(rc)
        return tuple(out), rc

    def close(self):
        if self._h is not None:
            capi.lib.hermite_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def adv_stability_limit(m, q=0):
    """Largest max_k |a_k| (dt/2)/h_k of a stable advection half step (q = 0:
    the whole series, limit 0.5)."""
    return capi.lib.hermite_adv_stability_limit(int(m), int(q))


class AdvectionPlan(Plan):
    """Half-step plan of the advection equation u_t = a . grad u (Eq. 1 is
    a = (1, 1, 1)): order m, periodic grid, spacings h, velocity a, FULL time
    step dt and q Taylor stages (0 = the whole series 3(2m+1), run by the fused
    kernel; fewer stages run the split pair)."""

    def __init__(self, m, grid, h, a, dt, q=0, prec="fp64", state="fp64", variant="auto"):
        self.m, self.grid, self.h = int(m), tuple(int(v) for v in grid), tuple(float(v) for v in h)
        self.a = tuple(float(v) for v in a)
        self.c, self.dt, self.prec, self.state, self.variant = 0.0, float(dt), prec, state, variant
        self.q = int(q) if q else 3 * (2 * self.m + 1)
        handle = ctypes.c_void_p()
        capi.check(capi.lib.hermite_adv_plan(ctypes.byref(handle), self.m, (ctypes.c_int * 3)(*self.grid),
                                             (ctypes.c_double * 3)(*self.h), (ctypes.c_double * 3)(*self.a),
                                             self.dt, int(q), PRECISIONS[prec], STATES[state], VARIANTS[variant]))
        self._h = handle

    @property
    def shape(self):
        M = self.m + 1
        return (M, M, M, self.grid[2], self.grid[1], self.grid[0])

    def error(self, x, ref, mask=0b101, stream=None):
        """(max_abs, max_rel, l2_abs, l2_rel) of x - ref (one field; mask bit 4:
        every derivative component, else values only)."""
        return super().error(x, ref, mask, stream)


def _d3(v):
    return (ctypes.c_double * 3)(*[float(x) for x in v])


def symbol_radius(m, h, c, dt, theta, q=4):
    """Spectral radius of the Fourier symbol of the wave half step at theta."""
    out = ctypes.c_double()
    capi.check(capi.lib.hermite_symbol_radius(int(m), int(q), float(c), _d3(h), float(dt), _d3(theta),
                                              ctypes.byref(out)))
    return out.value


def max_dt(m, h, c, q=4, npts=7):
    """Largest stable full step dt of the wave half step for spacings h (the
    symbol's spectral radius <= 1 on an npts^3 grid of theta)."""
    out = ctypes.c_double()
    capi.check(capi.lib.hermite_max_dt(int(m), int(q), float(c), _d3(h), int(npts), ctypes.byref(out)))
    return out.value


def adv_symbol_radius(m, h, a, dt, theta, q=0):
    """Spectral radius of the Fourier symbol of the advection half step."""
    out = ctypes.c_double()
    capi.check(capi.lib.hermite_adv_symbol_radius(int(m), int(q), _d3(a), _d3(h), float(dt), _d3(theta),
                                                  ctypes.byref(out)))
    return out.value


def adv_max_dt(m, h, a, q=0, npts=7):
    """Largest stable full step dt of the advection half step."""
    out = ctypes.c_double()
    capi.check(capi.lib.hermite_adv_max_dt(int(m), int(q), _d3(a), _d3(h), int(npts), ctypes.byref(out)))
    return out.value


def max_radius(m, h, c, dt, q=4, npts=7):
    """Largest spectral radius of the wave half step's symbol on an npts^3
    grid of theta."""
    out = ctypes.c_double()
    capi.check(capi.lib.hermite_max_radius(int(m), int(q), float(c), _d3(h), float(dt), int(npts),
                                           ctypes.byref(out)))
    return out.value


def adv_max_radius(m, h, a, dt, q=0, npts=7):
    """Largest spectral radius of the advection half step's symbol."""
    out = ctypes.c_double()
    capi.check(capi.lib.hermite_adv_max_radius(int(m), int(q), _d3(a), _d3(h), float(dt), int(npts),
                                               ctypes.byref(out)))
    return out.value
