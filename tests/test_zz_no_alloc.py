"""The allocation-free half step, hermite_step_split_static, against hermite_step.

hermite_step_split_static exists for callers that cannot allocate device memory
(another library owns it, or allocation must stay out of a time-critical
loop).  It keeps its workspace in a static device array of the library, so it
must give the same states as hermite_step (split variant) on consecutive calls:
the array keeps the previous call's contents, which must not leak into the
next result.  This file is collected last so that a run stopping at the first
failure has run every other test before it."""
import ctypes

import numpy as np
import pytest

import hermite_inputs as HI

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


@pytest.mark.parametrize("m,n,prec,state,tol", [
    (3, (40, 40, 12), "fp64", "fp64", 1e-12),   # one z-layer per slab: 12 slabs
    (2, (23, 17, 9), "fp64", "fp64", 1e-12),    # ragged tiles, one slab
    (2, (48, 40, 10), "fp32", "fp32", 2e-5),
])
def test_static_workspace_step_matches_hermite_step(torch_cuda, m, n, prec, state, tol):
    torch = torch_cuda
    from paper_1609_09841_gb300 import Plan, capi
    h = tuple(1.0 / v for v in n)
    plan = Plan(m, n, h, 1.0, 0.4 * min(h), prec=prec, state=state, variant="split")
    dtype = plan.torch_dtype
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (seed, parity) in enumerate(((70, 0), (71, 1))):   # two calls in a row
        x = torch.from_numpy(HI.random_state(m, n, seed=seed)).to(dtype).cuda()
        ref = torch.empty_like(x)
        plan.step(x, ref, parity)
        got = torch.full_like(x, float("nan"))
        rc = capi.lib.hermite_step_split_static(plan.handle, ctypes.c_void_p(x.data_ptr()),
                                                ctypes.c_void_p(got.data_ptr()), parity, stream)
        assert rc == capi.HERMITE_OK, capi.last_error()
        torch.cuda.synchronize()
        a, b = got.double().cpu().numpy(), ref.double().cpu().numpy()
        assert np.all(np.isfinite(a)), call
        assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(b)), call


def test_static_workspace_rejects_oversized_layer(torch_cuda):
    torch = torch_cuda
    from paper_1609_09841_gb300 import Plan, capi
    n = (64, 64, 4)           # one layer of m = 3 FP64 polynomials: 2*8^3*64*64*8 B = 32 MiB > 16 MiB
    h = tuple(1.0 / v for v in n)
    plan = Plan(3, n, h, 1.0, 0.4 * min(h))
    x = plan.empty()
    y = plan.empty()
    rc = capi.lib.hermite_step_split_static(plan.handle, ctypes.c_void_p(x.data_ptr()),
                                            ctypes.c_void_p(y.data_ptr()), 0, None)
    assert rc == capi.HERMITE_EINVAL
    msg = capi.last_error()
    assert "static workspace" in msg and str(capi.lib.hermite_static_workspace_bytes()) in msg


def test_static_workspace_rejects_host_buffers(torch_cuda):
    """Host buffers are refused before any launch, as hermite_step's device-only
    calls refuse them: a kernel given a host address would fault."""
    from paper_1609_09841_gb300 import Plan, capi
    n = (8, 8, 8)
    h = tuple(1.0 / v for v in n)
    plan = Plan(1, n, h, 1.0, 0.4 * min(h))
    x = np.zeros(plan.elems)
    y = np.zeros(plan.elems)
    dev = plan.empty()
    for a, b in ((x, y), (dev, y), (x, dev)):
        pa = a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr()
        pb = b.ctypes.data if isinstance(b, np.ndarray) else b.data_ptr()
        rc = capi.lib.hermite_step_split_static(plan.handle, ctypes.c_void_p(pa), ctypes.c_void_p(pb), 0, None)
        assert rc == capi.HERMITE_EINVAL, capi.last_error()
        assert "device buffers" in capi.last_error()
