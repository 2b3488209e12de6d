"""Parity at the workloads' full sizes on sampled outputs: the GPU computes a
whole half step of a seeded random state, the oracle recomputes a random
sample of output nodes one by one from their 8 corners."""
import numpy as np
import pytest

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


def _gather_corners(x, m, nodes, parity):
    """u_loc of the cells centred at the given output nodes (index work only):
    shape (k, 2, P, P, P) from the device state x (torch, any float type)."""
    M = m + 1
    nz, ny, nx = x.shape[-3:]
    s = 0 if parity == 0 else -1
    k = len(nodes)
    U = np.empty((k, 2, 2 * M, 2 * M, 2 * M))
    for c in (0, 1):
        for b in (0, 1):
            for a in (0, 1):
                zi = (nodes[:, 0] + s + c) % nz
                yi = (nodes[:, 1] + s + b) % ny
                xi = (nodes[:, 2] + s + a) % nx
                import torch
                idx = [torch.as_tensor(v, device=x.device) for v in (zi, yi, xi)]
                vals = x[:, :, :, :, idx[0], idx[1], idx[2]].double().cpu().numpy()  # (2,M,M,M,k)
                U[:, :, c * M:(c + 1) * M, b * M:(b + 1) * M, a * M:(a + 1) * M] = vals.transpose(4, 0, 1, 2, 3)
    return U


def _sampled_parity(torch, plan, m, n, h, c, dt, dtype, variant_tol, seed=7, count=96):
    gen = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn(plan.shape, dtype=dtype, device="cuda", generator=gen)
    y = torch.empty_like(x)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for parity in (0, 1):
        plan.step(x, y, parity)
        torch.cuda.synchronize()
        nodes = np.stack([rng.integers(0, n[2], count), rng.integers(0, n[1], count),
                          rng.integers(0, n[0], count)], axis=1)
        # always include the corners of the grid (periodic wrap) and the last CTA tile
        nodes[:4] = [[0, 0, 0], [n[2] - 1, n[1] - 1, n[0] - 1], [0, n[1] - 1, 0], [n[2] - 1, 0, n[0] - 1]]
        U = _gather_corners(x, m, nodes, parity)
        ref = oracle.cell_map(U, m, h, c, dt / 2)                         # (k, 2, M, M, M)
        got = y[:, :, :, :, torch.as_tensor(nodes[:, 0], device="cuda"),
                torch.as_tensor(nodes[:, 1], device="cuda"),
                torch.as_tensor(nodes[:, 2], device="cuda")].double().cpu().numpy().transpose(4, 0, 1, 2, 3)
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        worst = max(worst, err)
    assert worst <= variant_tol, worst
    return worst


@pytest.mark.parametrize("variant", ["fused", "split"])
def test_config2_size_fp64_sampled(torch_cuda, variant):
    """m = 3, 128^3, c = 1, dt = 0.4 h (the FP64 GPU-vs-oracle workload)."""
    torch = torch_cuda
    from paper_1609_09841_gb300 import Plan
    m, n = 3, (128, 128, 128)
    h = (1 / 128,) * 3
    dt = 0.4 * h[0]
    plan = Plan(m, n, h, 1.0, dt, prec="fp64", state="fp64", variant=variant)
    _sampled_parity(torch, plan, m, n, h, 1.0, dt, torch.float64, 1e-12)


@pytest.mark.parametrize("state,schedule", [("fp32", None), ("fp64", None), ("fp32", (5, 64)), ("fp64", (5, 64))])
def test_metric_size_fp32_sampled(torch_cuda, state, schedule):
    """m = 3, 256^3 (the throughput workload) with FP32 arithmetic; the sample
    is compared with the FP64 oracle on the same (rounded) input.  Schedule
    (5, 64) is the 8x2-cell, 256-thread tile with z-chunk 64 that the bench's
    autotuner picks and times at this size."""
    torch = torch_cuda
    from paper_1609_09841_gb300 import Plan
    m, n = 3, (256, 256, 256)
    h = (1 / 256,) * 3
    dt = 0.4 * h[0]
    plan = Plan(m, n, h, 1.0, dt, prec="fp32", state=state)
    if schedule is not None:
        plan.set_schedule(*schedule)
    _sampled_parity(torch, plan, m, n, h, 1.0, dt, torch.float32 if state == "fp32" else torch.float64, 2e-5)
