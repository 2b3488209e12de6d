"""Device allocations made lazily by the calls (split workspace, host-step
staging buffers, reduction scratch, tensor-core status word) report
HERMITE_ENOMEM when they fail, and the plan works once memory is available
again (hermite_inject_alloc_failure, the library's testing hook)."""
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


@pytest.fixture(autouse=True)
def disarm():
    yield
    from paper_1609_09841_gb300 import capi
    capi.lib.hermite_inject_alloc_failure(0, 0)


def _expect_enomem(fn):
    from paper_1609_09841_gb300 import capi
    capi.lib.hermite_inject_alloc_failure(0, 1)
    with pytest.raises(capi.HermiteError) as e:
        fn()
    assert e.value.code == capi.HERMITE_ENOMEM
    capi.lib.hermite_inject_alloc_failure(0, 0)


@pytest.mark.parametrize("prec,state,variant,host", [("fp64", "fp64", "split", False), ("fp32", "fp32", "fused", True),
                                                     ("3xtf32", "fp32", "fused", False)])
def test_lazy_device_allocations_fail_then_recover(torch_cuda, prec, state, variant, host):
    torch = torch_cuda
    from paper_1609_09841_gb300 import Plan
    m, n = 2, (9, 8, 7)
    h = tuple(1.0 / v for v in n)
    plan = Plan(m, n, h, 1.0, 0.4 * min(h), prec=prec, state=state, variant=variant)
    x = HI.random_state(m, n, seed=3).astype(np.float64 if state == "fp64" else np.float32)
    if host:
        y = np.empty_like(x)
        _expect_enomem(lambda: plan.step(x, y, 0))          # staging buffers
        plan.step(x, y, 0)
        ref = torch.empty(plan.shape, dtype=plan.torch_dtype, device="cuda")
        plan.step(torch.from_numpy(x).cuda(), ref, 0)
        torch.cuda.synchronize()
        assert np.array_equal(y, ref.cpu().numpy())
    else:
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        _expect_enomem(lambda: plan.step(xd, yd, 0))        # workspace / status word
        plan.step(xd, yd, 0)
        torch.cuda.synchronize()
        assert torch.isfinite(yd).all()


def test_error_norm_scratch_fails_then_recovers(torch_cuda):
    torch = torch_cuda
    from paper_1609_09841_gb300 import Plan, capi
    n = (8, 8, 8)
    plan = Plan(1, n, (0.125,) * 3, 1.0, 0.05)
    a = torch.zeros(plan.shape, dtype=torch.float64, device="cuda")
    capi.lib.hermite_inject_alloc_failure(0, 1)
    with pytest.raises(capi.HermiteError) as e:
        plan.error(a, a)
    assert e.value.code == capi.HERMITE_ENOMEM
    capi.lib.hermite_inject_alloc_failure(0, 0)
    (mx, _, _, _), rc = plan.error(a, a + 1.0)
    assert rc == 0 and mx == 1.0
