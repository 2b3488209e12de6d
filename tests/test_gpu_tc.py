"""GPU parity of the tensor-core half step (HERMITE_3XTF32, HERMITE_SPLITBF16)
against the FP64 oracle, through the C ABI.

The z-pass (the mode product along x3 of the 1-D evolution-and-truncation
factors, Sec. 3.1 Alg. 1/2 with the evolution of Sec. 3.2 folded in) runs on
tcgen05 with FP32 accumulation, on operands split into tensor-core pieces:
3xTF32 keeps 2 x 11 = 22 significant bits of each operand and drops the
product of the two low pieces (relative size <= 2^-22); BF16 x 3 keeps
3 x 8 = 24 bits and drops the products of total order > 2 (<= 2^-24).  The
x- and y-passes are FP32 as in HERMITE_FP32.  The per-step error is
therefore of the FP32 arithmetic's order, and the tests hold it to the FP32
bar of tests/test_gpu_parity.py: relative max-norm <= 2e-5 against the
oracle's FP64 half step, on every component of both fields (the random
states scale component i by 0.5^|i|, so a wrong index or sign in a small
high-order component already shows as a relative error >= 2e-3)."""
import ctypes

import numpy as np
import pytest

import hermite_inputs as HI
from oracle import hermite as oracle

pytestmark = pytest.mark.gpu

TOL = 2e-5
# Several 8x4 (m = 1) or 8x2 tiles with ragged tails in x and y.
GRIDS = {1: (19, 13, 11), 2: (9, 7, 6), 3: (9, 6, 5)}
PRECS = ["3xtf32", "splitbf16"]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _plan(m, n, prec, state, c=1.0, lam=0.2):
    from paper_1609_09841_gb300 import Plan
    h = tuple(1.0 / v for v in n)
    dt = 2 * lam * min(h) / c
    return Plan(m, n, h, c, dt, prec=prec, state=state), h, dt


def _relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("state", ["fp32", "fp64"])
@pytest.mark.parametrize("m", [1, 2, 3])
@pytest.mark.parametrize("zchunk", [16, 2])
def test_tc_step_matches_oracle(torch_cuda, prec, state, m, zchunk):
    torch = torch_cuda
    n = GRIDS[m]
    plan, h, dt = _plan(m, n, prec, state, c=1.3)
    plan.set_schedule(0, zchunk)            # 2: several z-chunks, the last one partial
    x = HI.random_state(m, n, seed=40 + m)
    if state == "fp32":
        x = x.astype(np.float32).astype(np.float64)
    xd = torch.from_numpy(x).cuda().to(plan.torch_dtype)
    for parity in (0, 1):
        yd = torch.full_like(xd, float("nan"))
        plan.step(xd, yd, parity)
        ref = oracle.half_step(x, m, h, 1.3, dt, parity)
        got = yd.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got)), parity
        assert _relmax(got, ref) <= TOL, (parity, _relmax(got, ref))
    assert plan.device_status() == 0


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("m", [1, 2, 3])
def test_tc_adjoint_matches_oracle(torch_cuda, prec, m):
    torch = torch_cuda
    n = GRIDS[m]
    plan, h, dt = _plan(m, n, prec, "fp64", c=0.8)
    g = HI.random_state(m, n, seed=50 + m)
    gd = torch.from_numpy(g).cuda()
    for parity in (0, 1):
        out = torch.full_like(gd, float("nan"))
        plan.adjoint(gd, out, parity)
        ref = oracle.adjoint_half_step(g, m, h, 0.8, dt, parity)
        assert _relmax(out.cpu().numpy(), ref) <= TOL, parity


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n", [(1, 1, 1), (2, 2, 2), (1, 3, 2), (17, 1, 4)])
@pytest.mark.parametrize("m", [1, 3])
def test_tc_degenerate_grids(torch_cuda, prec, n, m):
    """Grids thinner than a tile, down to one node per dimension (every
    corner of a cell is the same node)."""
    torch = torch_cuda
    plan, h, dt = _plan(m, n, prec, "fp64")
    x = HI.random_state(m, n, seed=4)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    for parity in (0, 1):
        plan.step(xd, yd, parity)
        ref = oracle.half_step(x, m, h, 1.0, dt, parity)
        assert _relmax(yd.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("prec", PRECS)
def test_tc_host_buffers_equal_device_step(torch_cuda, prec):
    """Host buffers run the same kernel z-slab by z-slab (pipelined copies):
    bit for bit the device-buffer result."""
    torch = torch_cuda
    m, n = 2, (9, 8, 7)
    plan, h, dt = _plan(m, n, prec, "fp32")
    x = HI.random_state(m, n, seed=8).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    for parity in (0, 1):
        y_host = np.full_like(x, np.nan)
        plan.step(x, y_host, parity)
        plan.step(xd, yd, parity)
        torch.cuda.synchronize()
        assert np.array_equal(y_host, yd.cpu().numpy()), parity


@pytest.mark.parametrize("prec", PRECS)
def test_tc_fp64_state_equals_fp32_state(torch_cuda, prec):
    """An FP64 state is converted to FP32 on load and back on store (the store
    by integer operations, exact): the same results as the FP32 state."""
    torch = torch_cuda
    m, n = 3, (17, 10, 9)
    p32, h, dt = _plan(m, n, prec, "fp32")
    p64, _, _ = _plan(m, n, prec, "fp64")
    x = HI.random_state(m, n, seed=9).astype(np.float32)
    x32 = torch.from_numpy(x).cuda()
    x64 = x32.double()
    y32, y64 = torch.empty_like(x32), torch.empty_like(x64)
    for parity in (0, 1):
        p32.step(x32, y32, parity)
        p64.step(x64, y64, parity)
        assert torch.equal(y32.double(), y64), parity
