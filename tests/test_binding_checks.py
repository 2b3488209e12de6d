"""The Python binding rejects buffers of the wrong element type or size
before the library sees them: the C ABI takes bare pointers and reads exactly
the plan's element type, so an FP32 buffer handed to an FP64 plan would be
read past its end.  Plans need no GPU, and these checks run before any call
that does."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1609_09841_gb300 as p
    return p


def _plan(pkg, state):
    n = (4, 4, 4)
    h = (0.25,) * 3
    prec = "fp64" if state == "fp64" else "fp32"
    return pkg.Plan(1, n, h, 1.0, 0.1, prec=prec, state=state)


@pytest.mark.parametrize("state,wrong", [("fp64", np.float32), ("fp32", np.float64), ("fp32", np.int32)])
def test_step_rejects_host_buffers_of_another_type(pkg, state, wrong):
    plan = _plan(pkg, state)
    x = np.zeros(plan.shape, wrong)
    y = np.zeros(plan.shape, wrong)
    with pytest.raises(ValueError):
        plan.step(x, y, 0)


def test_step_rejects_a_mixed_pair(pkg):
    plan = _plan(pkg, "fp64")
    with pytest.raises(ValueError):
        plan.step(np.zeros(plan.shape), np.zeros(plan.shape, np.float32), 0)


def test_advection_plan_checks_types_too(pkg):
    adv = pkg.AdvectionPlan(2, (4, 4, 4), (0.25,) * 3, (1.0, 1.0, 1.0), 0.2, prec="fp32", state="fp32")
    with pytest.raises(ValueError):
        adv.step(np.zeros(adv.shape), np.zeros(adv.shape), 0)


def test_error_wants_an_fp64_reference(pkg):
    torch = pytest.importorskip("torch")
    plan = _plan(pkg, "fp32")
    x = torch.zeros(plan.shape, dtype=torch.float32)
    with pytest.raises(ValueError):
        plan.error(x, torch.zeros(plan.shape, dtype=torch.float32))


def test_receivers_want_int64_indices_and_enough_room(pkg):
    torch = pytest.importorskip("torch")
    plan = _plan(pkg, "fp64")
    x = torch.zeros(plan.shape, dtype=torch.float64)
    with pytest.raises(ValueError):
        plan.record(x, torch.zeros(4, dtype=torch.int32), torch.zeros(4, dtype=torch.float64))
    with pytest.raises(ValueError):       # host tensors: the receiver calls take device buffers
        plan.record(x, torch.zeros(4, dtype=torch.int64), torch.zeros(4, dtype=torch.float64))
    with pytest.raises(ValueError):
        plan.inject(x, torch.zeros(4, dtype=torch.int64), torch.zeros(2, dtype=torch.float64))


@pytest.mark.gpu
def test_batch_states_must_match_the_plan_type(pkg):
    """A batched plan allocates its work list on the device, so this one
    needs a GPU; the float64 device tensors are rejected before any launch."""
    torch = pytest.importorskip("torch")
    from paper_1609_09841_gb300.batch import BatchPlan
    sims = [{"m": 1, "grid": (4, 4, 4), "h": (0.25,) * 3, "c": 1.0, "dt": 0.1}]
    bp = BatchPlan(sims, prec="fp32", state="fp32")
    x = [torch.zeros(bp.shape(0), dtype=torch.float64, device="cuda")]
    with pytest.raises(ValueError):
        bp.step(x, x, 0)
