"""The remainder-form precision (HERMITE_REMAINDER) against the FP64 oracle.

Per half step on seeded random states (no smoothness: the remainders are as
large as the data, so the FP32 parts carry the FP32 arithmetic's error) the
result is held to the FP32 bar of tests/test_gpu_parity.py, 2e-5 relative
max-norm.  Its accuracy on resolved data, the reason it exists, is tested at
t = 1 in tests/test_gpu_precision.py (bar 1e-5)."""
import numpy as np
import pytest

import hermite_inputs as HI
from oracle import hermite as oracle

pytestmark = pytest.mark.gpu
GRIDS = {1: (19, 13, 11), 2: (9, 7, 6), 3: (9, 6, 5)}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _plan(m, n, c=1.0, lam=0.2):
    from paper_1609_09841_gb300 import Plan
    h = tuple(1.0 / v for v in n)
    dt = 2 * lam * min(h) / c
    return Plan(m, n, h, c, dt, prec="remainder", state="fp64"), h, dt


def _relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("m", [1, 2, 3])
@pytest.mark.parametrize("zchunk", [16, 2])
def test_remainder_step_matches_oracle(torch_cuda, m, zchunk):
    torch = torch_cuda
    n = GRIDS[m]
    plan, h, dt = _plan(m, n, c=1.3)
    plan.set_schedule(0, zchunk)
    x = HI.random_state(m, n, seed=60 + m)
    xd = torch.from_numpy(x).cuda()
    for parity in (0, 1):
        yd = torch.full_like(xd, float("nan"))
        plan.step(xd, yd, parity)
        ref = oracle.half_step(x, m, h, 1.3, dt, parity)
        assert _relmax(yd.cpu().numpy(), ref) <= 2e-5, parity


@pytest.mark.parametrize("n", [(1, 1, 1), (2, 2, 2), (1, 3, 2), (17, 1, 4)])
def test_remainder_degenerate_grids(torch_cuda, n):
    torch = torch_cuda
    plan, h, dt = _plan(3, n)
    x = HI.random_state(3, n, seed=5)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    for parity in (0, 1):
        plan.step(xd, yd, parity)
        assert _relmax(yd.cpu().numpy(), oracle.half_step(x, 3, h, 1.0, dt, parity)) <= 2e-5


def test_remainder_host_buffers_and_rules(torch_cuda):
    torch = torch_cuda
    from paper_1609_09841_gb300 import capi
    m, n = 2, (9, 8, 7)
    plan, h, dt = _plan(m, n)
    x = HI.random_state(m, n, seed=8)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    for parity in (0, 1):
        y_host = np.full_like(x, np.nan)
        plan.step(x, y_host, parity)
        plan.step(xd, yd, parity)
        torch.cuda.synchronize()
        assert np.array_equal(y_host, yd.cpu().numpy()), parity
    with pytest.raises(capi.HermiteError) as e:      # forward steps only
        plan.adjoint(xd, yd, 0)
    assert e.value.code == capi.HERMITE_EUNSUPPORTED
