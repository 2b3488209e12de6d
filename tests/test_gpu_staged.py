"""Staged schedules of the FP32 fused kernel (tiles 6 and 7: each node plane
copied into shared memory by the bulk tensor-copy engine, tiles whose window
wraps around the periodic boundary filled with plain loads).

The grids have row pitches the copy engine can address (nx a multiple of
16 bytes' worth of state elements), so that interior tiles take the copy and
the tiles at the x and y boundaries (and the ragged ones) the plain loads.
Each staged tile must equal tile 0 of the same plan bit for bit (the per-node
arithmetic of the fused tile does not depend on the tile shape) on forward
and adjoint half steps, match the oracle within the FP32 per-step bound of
tests/test_gpu_parity.py, and leave the plan's device status clear."""
import numpy as np
import pytest

import hermite_inputs as HI
from oracle import hermite as oracle

pytestmark = pytest.mark.gpu

# (m, grid): x and y with tiles of both kinds for every staged shape
GRIDS = [(1, (32, 20, 9)), (1, (24, 18, 5)), (2, (24, 12, 7)), (2, (16, 10, 6)), (3, (24, 12, 7)), (3, (16, 8, 5))]
STAGED = (6, 7)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _plan(m, n, state):
    from paper_1609_09841_gb300 import Plan
    h = tuple(1.0 / v for v in n)
    dt = 0.4 * min(h)
    return Plan(m, n, h, 1.0, dt, prec="fp32", state=state), h, dt


@pytest.mark.parametrize("state", ["fp32", "fp64"])
@pytest.mark.parametrize("m,n", GRIDS)
def test_staged_tiles_equal_tile0_and_oracle(torch_cuda, m, n, state):
    torch = torch_cuda
    plan, h, dt = _plan(m, n, state)
    assert plan.schedule_count() == 8
    x = HI.random_state(m, n, seed=70 + m)
    if state == "fp32":
        x = x.astype(np.float32).astype(np.float64)
    xd = torch.from_numpy(x).cuda().to(plan.torch_dtype)
    for parity in (0, 1):
        plan.set_schedule(0, 16)
        ref_fwd = torch.empty_like(xd)
        plan.step(xd, ref_fwd, parity)
        ref_adj = torch.empty_like(xd)
        plan.adjoint(xd, ref_adj, parity)
        want = oracle.half_step(x, m, h, 1.0, dt, parity)
        err = float(np.max(np.abs(ref_fwd.cpu().numpy().astype(np.float64) - want)) / np.max(np.abs(want)))
        assert err <= 2e-5
        for tile in STAGED:
            for zc in (1, 5, 16):
                plan.set_schedule(tile, zc)
                y = torch.full_like(xd, float("nan"))
                plan.step(xd, y, parity)
                assert torch.equal(y, ref_fwd), (tile, zc, parity)
                g = torch.full_like(xd, float("nan"))
                plan.adjoint(xd, g, parity)
                assert torch.equal(g, ref_adj), (tile, zc, parity, "adjoint")
    assert plan.device_status() == 0


def test_staged_tile_on_a_grid_the_copy_engine_cannot_address(torch_cuda):
    """nx = 21: no tensor map, every tile fills its window with plain loads."""
    torch = torch_cuda
    m, n = 3, (21, 10, 6)
    plan, h, dt = _plan(m, n, "fp32")
    x = torch.randn(plan.shape, dtype=torch.float32, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    plan.set_schedule(0, 16)
    ref = torch.empty_like(x)
    plan.step(x, ref, 1)
    for tile in STAGED:
        plan.set_schedule(tile, 4)
        y = torch.empty_like(x)
        plan.step(x, y, 1)
        assert torch.equal(y, ref), tile
    assert plan.device_status() == 0
