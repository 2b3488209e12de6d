"""q-stage Hermite-Taylor evolution (Alg. 4 with q up to d(2m+1) = 3(2m+1))
on the GPU against the oracle's Taylor evolution with the same q."""
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


def _relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


CASES = [(1, 9), (2, 15), (2, 6), (3, 21), (3, 7)]


@pytest.mark.parametrize("m,q", CASES)
@pytest.mark.parametrize("variant", ["fused", "split"])
def test_taylor_q_fp64_matches_oracle(torch_cuda, m, q, variant):
    torch = torch_cuda
    from paper_1609_09841_gb300 import Plan
    n = GRIDS[m]
    h = tuple(1.0 / v for v in n)
    dt = 0.4 * min(h)
    plan = Plan(m, n, h, 1.1, dt, variant=variant)
    plan.set_taylor_order(q)
    assert plan.taylor_order == q
    x = HI.random_state(m, n, seed=90 + q)
    xd = torch.from_numpy(x).cuda()
    yd = torch.full_like(xd, float("nan"))
    for parity in (0, 1):
        plan.step(xd, yd, parity)
        ref = oracle.half_step(x, m, h, 1.1, dt, parity, evolve="taylor", q=q)
        assert _relmax(yd.cpu().numpy(), ref) <= 1e-12, parity
    if variant == "fused":
        for parity in (0, 1):
            plan.adjoint(xd, yd, parity)
            ref = oracle.adjoint_half_step(x, m, h, 1.1, dt, parity, evolve="taylor", q=q)
            assert _relmax(yd.cpu().numpy(), ref) <= 1e-12, parity


@pytest.mark.parametrize("m,q", CASES)
@pytest.mark.parametrize("state", ["fp32", "fp64"])
def test_taylor_q_fp32(torch_cuda, m, q, state):
    """FP32 arithmetic with the longer series: within the FP32 per-step
    tolerance of the parity tests against the FP64 oracle."""
    torch = torch_cuda
    from paper_1609_09841_gb300 import Plan
    n = GRIDS[m]
    h = tuple(1.0 / v for v in n)
    dt = 0.4 * min(h)
    plan = Plan(m, n, h, 1.0, dt, prec="fp32", state=state)
    plan.set_taylor_order(q)
    x = HI.random_state(m, n, seed=95 + q).astype(np.float32).astype(np.float64)
    xd = torch.from_numpy(x).cuda().to(plan.torch_dtype)
    yd = torch.empty_like(xd)
    for parity in (0, 1):
        plan.step(xd, yd, parity)
        ref = oracle.half_step(x, m, h, 1.0, dt, parity, evolve="taylor", q=q)
        assert _relmax(yd.double().cpu().numpy(), ref) <= 2e-5, parity



def test_full_series_runs_at_a_step_rk4_cannot_take(torch_cuda):
    """m = 2, q = 15 at lam = 0.41 (RK4's limit is 0.30): the first half steps
    match the oracle's q = 15 run and 200 half steps stay bounded."""
    torch = torch_cuda
    from paper_1609_09841_gb300 import Plan, stability_limit
    m, q, n = 2, 15, (12, 12, 12)
    h = (1.0 / 12,) * 3
    lam = 0.41
    assert stability_limit(m, 4) < lam <= stability_limit(m, q)
    dt = 2 * lam * h[0]
    plan = Plan(m, n, h, 1.0, dt, q=q)
    x = HI.random_state(m, n, seed=7)
    ref = oracle.run(x, m, h, 1.0, dt, 4, evolve="taylor", q=q)
    a = torch.from_numpy(x).cuda()
    b = torch.empty_like(a)
    for k in range(4):
        plan.step(a, b, k % 2)
        a, b = b, a
    assert _relmax(a.cpu().numpy(), ref) <= 1e-12
    amp0 = float(a.abs().max())
    for k in range(196):
        plan.step(a, b, k % 2)
        a, b = b, a
    assert torch.isfinite(a).all() and float(a.abs().max()) <= 2.0 * amp0
