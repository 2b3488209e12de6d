"""Differentiable receiver runs (discrete adjoint + checkpointing) on the GPU."""
import numpy as np
import pytest

import hermite_inputs as HI
from oracle import hermite as oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _oracle_traces(x0, m, h, c, dt, nhalf, idx):
    x, tr = x0, []
    for t in range(nhalf):
        x = oracle.half_step(x, m, h, c, dt, t % 2)
        tr.append(x[0, 0, 0, 0].reshape(-1)[idx])
    return np.array(tr)


def _oracle_grad_u0(m, h, c, dt, nhalf, idx, g, shape):
    adj = np.zeros(shape)
    for t in range(nhalf - 1, -1, -1):
        flat = adj[0, 0, 0, 0].reshape(-1)
        np.add.at(flat, idx, g[t])
        adj[0, 0, 0, 0] = flat.reshape(shape[-3:])
        adj = oracle.adjoint_half_step(adj, m, h, c, dt, t % 2)
    return adj


@pytest.mark.parametrize("every", [1, 5, 40])
def test_small_run_matches_oracle(torch_cuda, every):
    """FP64: traces, dL/du0 (oracle adjoint sweep) and dL/dc (central
    difference of the oracle's loss in c) on an 8 x 7 x 6 grid, m = 2,
    13 half steps, checkpoints every 1, 5 (ragged last segment) or 40
    (a single segment) half steps."""
    torch = torch_cuda
    from paper_1609_09841_gb300 import Plan
    from paper_1609_09841_gb300.adjoint import receiver_traces
    m, n = 2, (8, 7, 6)
    h = tuple(1.0 / v for v in n)
    c, dt, nhalf = 1.1, 0.3 * min(h), 13
    x0 = HI.gaussian_pulse(m, n, h, centre=(0.4, 0.5, 0.6), sigma=0.15)
    idx = HI.receiver_draw(2, n, count=6)
    target = np.random.default_rng(3).standard_normal((nhalf, 6)) * 0.01
    plan = Plan(m, n, h, c, dt)
    u0 = torch.from_numpy(x0).cuda().requires_grad_(True)
    ct = torch.tensor(c, dtype=torch.float64, requires_grad=True)
    tr = receiver_traces(plan, u0, nhalf, torch.from_numpy(idx).cuda(), every, ct)
    loss = ((tr - torch.from_numpy(target).cuda()) ** 2).sum()
    loss.backward()
    ref_tr = _oracle_traces(x0, m, h, c, dt, nhalf, idx)
    assert np.max(np.abs(tr.detach().cpu().numpy() - ref_tr)) <= 1e-12 * np.max(np.abs(ref_tr))
    g = 2 * (ref_tr - target)
    ref_grad = _oracle_grad_u0(m, h, c, dt, nhalf, idx, g, x0.shape)
    got = u0.grad.cpu().numpy()
    assert np.max(np.abs(got - ref_grad)) <= 1e-11 * np.max(np.abs(ref_grad))
    dc = 1e-4 * c
    lp = np.sum((_oracle_traces(x0, m, h, c + dc, dt, nhalf, idx) - target) ** 2)
    lm = np.sum((_oracle_traces(x0, m, h, c - dc, dt, nhalf, idx) - target) ** 2)
    fd = (lp - lm) / (2 * dc)
    assert abs(float(ct.grad) - fd) <= 1e-6 * abs(fd)


def _config5(torch, prec, state):
    from paper_1609_09841_gb300 import Plan
    m, n = 2, (64, 64, 64)
    h = (1 / 64,) * 3
    dt = 0.4 * h[0]
    plan = Plan(m, n, h, 1.0, dt, prec=prec, state=state)
    rng = np.random.default_rng(1609)
    centre = tuple(rng.uniform(0.3, 0.7, 3))
    x0 = HI.gaussian_pulse(m, n, h, centre=centre, sigma=0.05)
    shifted = HI.gaussian_pulse(m, n, h, centre=(centre[0] + 0.02, centre[1], centre[2]), sigma=0.05)
    idx = torch.from_numpy(HI.receiver_draw(5, n, 32)).cuda()
    return plan, x0, shifted, idx


def test_config5_gradient_fd_and_fp64(torch_cuda):
    """m = 2, 64^3, 300 half steps, 32 receivers, checkpoints every 20 half
    steps.  Loss: squared misfit against the traces of the pulse shifted by
    0.02 in x1.  The gradient with respect to u0 is checked against central
    finite differences along 16 seeded directions, for the FP64 path with
    step 1e-4 and for FP32 arithmetic with an FP64 state; and the FP32 and
    FP64 gradients are compared.

    The loss is quadratic in u0, so the central difference has no truncation
    error at any step.  With FP64 arithmetic the step 1e-4 leaves rounding
    far below the tolerance 1e-7.  With FP32 arithmetic each trace carries a
    rounding error of about 1e-7 of its size, which is not correlated between
    the two perturbed runs; a step of 1e-4 would drown the difference in that
    noise, so the FP32 check uses a step of the size of u0 itself (step 1.0
    on directions scaled to max|u0|) and a tolerance of 1e-3."""
    torch = torch_cuda
    from paper_1609_09841_gb300.adjoint import receiver_traces
    nhalf, every = 300, 20
    grads = {}
    for prec, eps, tol in (("fp64", 1e-4, 1e-7), ("fp32", 1.0, 1e-3)):
        plan, x0, shifted, idx = _config5(torch, prec, "fp64")
        with torch.no_grad():
            target = receiver_traces(plan, torch.from_numpy(shifted).cuda(), nhalf, idx, every)
        u0 = torch.from_numpy(x0).cuda().requires_grad_(True)

        def loss_of(u):
            return float(((receiver_traces(plan, u, nhalf, idx, every) - target) ** 2).sum())

        loss = ((receiver_traces(plan, u0, nhalf, idx, every) - target) ** 2).sum()
        loss.backward()
        grads[prec] = u0.grad.clone()
        gen = torch.Generator(device="cuda").manual_seed(16)
        for _ in range(16):
            v = torch.randn(u0.shape, dtype=torch.float64, device="cuda", generator=gen)
            v *= u0.detach().abs().max() / v.abs().max()
            fd = (loss_of(u0.detach() + eps * v) - loss_of(u0.detach() - eps * v)) / (2 * eps)
            ad = float((grads[prec] * v).sum())
            assert abs(fd - ad) <= tol * max(abs(ad), 1e-30), (prec, fd, ad)
    a, b = grads["fp32"], grads["fp64"]
    assert float((a - b).norm() / b.norm()) <= 1e-4


@pytest.mark.parametrize("every", [1, 4, 40])
def test_hermite_run_matches_oracle(torch_cuda, every):
    """HermiteRun (adjoint.run): the state after 11 half steps, the gradient
    of L = <x_n, w> with respect to x0 (the oracle's adjoint sweep of w) and
    dL/dc (central difference of the oracle's L in c), FP64, m = 2, on a
    9 x 7 x 6 grid, checkpoints every 1, 4 (ragged last segment) or 40 half
    steps."""
    torch = torch_cuda
    from paper_1609_09841_gb300 import Plan
    from paper_1609_09841_gb300.adjoint import run
    m, n = 2, (9, 7, 6)
    h = tuple(1.0 / v for v in n)
    c, dt, nhalf = 1.1, 0.3 * min(h), 11
    x0 = HI.random_state(m, n, seed=21)
    w = HI.random_state(m, n, seed=22)
    plan = Plan(m, n, h, c, dt)
    xt = torch.from_numpy(x0).cuda().requires_grad_(True)
    ct = torch.tensor(c, dtype=torch.float64, requires_grad=True)
    y = run(plan, xt, nhalf, every, ct)
    ((y * torch.from_numpy(w).cuda()).sum()).backward()

    ref = oracle.run(x0, m, h, c, dt, nhalf)
    assert np.max(np.abs(y.detach().cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    adj = w.copy()
    for t in range(nhalf - 1, -1, -1):
        adj = oracle.adjoint_half_step(adj, m, h, c, dt, t % 2)
    g = xt.grad.cpu().numpy()
    assert np.max(np.abs(g - adj)) <= 1e-12 * np.max(np.abs(adj))
    dc = 1e-4
    lp = float(np.sum(oracle.run(x0, m, h, c + dc, dt, nhalf) * w))
    lm = float(np.sum(oracle.run(x0, m, h, c - dc, dt, nhalf) * w))
    fd = (lp - lm) / (2 * dc)
    assert abs(float(ct.grad) - fd) <= 1e-6 * abs(fd)


def test_two_argument_step_and_adjoint(torch_cuda):
    """Plan.step(x, parity) and Plan.adjoint(g, parity) allocate their output
    and equal the three-argument calls."""
    torch = torch_cuda
    from paper_1609_09841_gb300 import Plan
    m, n = 1, (8, 8, 8)
    h = (1 / 8,) * 3
    plan = Plan(m, n, h, 1.0, 0.4 / 8)
    x = torch.from_numpy(HI.random_state(m, n, seed=23)).cuda()
    for parity in (0, 1):
        y = torch.empty_like(x)
        plan.step(x, y, parity)
        assert torch.equal(plan.step(x, parity), y)
        plan.adjoint(x, y, parity)
        assert torch.equal(plan.adjoint(x, parity), y)
    with pytest.raises(TypeError):
        plan.step(x, x)
