"""Batched half steps (one persistent launch per half step, CUDA-graph runs)."""
import json

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


SMALL = [  # uneven orders and grids, ragged tiles, one grid thinner than a tile
    {"m": 3, "grid": (9, 6, 5)}, {"m": 1, "grid": (19, 13, 11)}, {"m": 2, "grid": (9, 7, 6)},
    {"m": 1, "grid": (3, 2, 17)}, {"m": 3, "grid": (4, 4, 4)},
]


def _sims(spec, c=1.0, lam=0.2):
    out = []
    for s in spec:
        h = tuple(1.0 / v for v in s["grid"])
        out.append({"m": s["m"], "grid": s["grid"], "h": h, "c": c, "dt": 2 * lam * min(h) / c})
    return out


@pytest.mark.parametrize("zchunk,tiles", [((16, 16, 16), (0, 0, 0)), ((3, 2, 1), (0, 0, 0)),
                                         ((16, 16, 16), (1, 1, 1)), ((5, 1, 2), (1, 0, 1))])
def test_batch_step_matches_oracle_fp64(torch_cuda, zchunk, tiles):
    torch = torch_cuda
    from paper_1609_09841_gb300.batch import BatchPlan
    sims = _sims(SMALL, c=1.2)
    bp = BatchPlan(sims, prec="fp64", state="fp64")
    bp.set_schedule(zchunk)
    bp.set_tiles(tiles)
    xs = [HI.random_state(s["m"], s["grid"], seed=60 + i) for i, s in enumerate(sims)]
    a = [torch.from_numpy(x).cuda() for x in xs]
    b = [torch.full_like(t, float("nan")) for t in a]
    for parity in (0, 1):
        bp.step(a, b, parity)
        for i, s in enumerate(sims):
            ref = oracle.half_step(xs[i], s["m"], s["h"], s["c"], s["dt"], parity)
            got = b[i].cpu().numpy()
            assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), (i, parity)


@pytest.mark.parametrize("tiles", [(0, 0, 0), (1, 1, 1), (0, 1, 1)])
def test_batch_fp32_equals_single_plans_and_graph_run(torch_cuda, tiles):
    """FP32: each simulation of a batched step equals its own single-grid
    plan's step bit for bit (same per-cell arithmetic, whatever the tile
    shape), and a 7-half-step graph run equals 7 batched steps bit for bit."""
    torch = torch_cuda
    from paper_1609_09841_gb300 import Plan
    from paper_1609_09841_gb300.batch import BatchPlan
    sims = _sims(SMALL)
    bp = BatchPlan(sims, prec="fp32", state="fp32")
    bp.set_tiles(tiles)
    gen = torch.Generator(device="cuda").manual_seed(4)
    a = [torch.randn(bp.shape(i), dtype=torch.float32, device="cuda", generator=gen) for i in range(len(sims))]
    a0 = [t.clone() for t in a]
    b = [torch.empty_like(t) for t in a]
    bp.step(a, b, 0)
    for i, s in enumerate(sims):
        p = Plan(s["m"], s["grid"], s["h"], s["c"], s["dt"], prec="fp32", state="fp32")
        y = torch.empty_like(a[i])
        p.step(a[i], y, 0)
        assert torch.equal(y, b[i]), i
    x = [t.clone() for t in a0]
    y = [torch.empty_like(t) for t in a0]
    for k in range(7):
        bp.step(x, y, k % 2)
        x, y = y, x
    ga = [t.clone() for t in a0]
    gb = [torch.empty_like(t) for t in a0]
    res = bp.run(ga, gb, 7)
    torch.cuda.synchronize()
    assert res is gb
    for i in range(len(sims)):
        assert torch.equal(res[i], x[i]), i


def test_config4_batch_64_sims(torch_cuda):
    """64 seeded simulations (sides from {32,48,64,96} per dimension, m from
    {1,2,3}, Gaussian pulses), FP32, 200 half steps as one graph, with the
    autotuned tile shapes and z-chunks; every simulation equals its
    single-grid FP32 run bit for bit and stays finite."""
    torch = torch_cuda
    from paper_1609_09841_gb300 import Plan
    from paper_1609_09841_gb300.autotune import tune_batch
    from paper_1609_09841_gb300.batch import BatchPlan
    draw = HI.batch_draw(1609)
    sims = []
    for d in draw:
        hmin = min(d["h"])
        sims.append({"m": d["m"], "grid": d["n"], "h": d["h"], "c": 1.0, "dt": 0.4 * hmin})
    bp = BatchPlan(sims, prec="fp32", state="fp32")
    a = [torch.from_numpy(HI.gaussian_pulse(d["m"], d["n"], d["h"], d["centre"], d["sigma"])).float().cuda()
         for d in draw]
    b = [torch.empty_like(t) for t in a]
    tuned = tune_batch(bp, [t.clone() for t in a], b)
    res = bp.run(a, b, 200)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x, y = [t.clone() for t in a], [torch.empty_like(t) for t in a]
    bp.run(x, y, 200)            # captures and instantiates the graph of this buffer pair
    torch.cuda.synchronize()
    e0.record()
    bp.run(x, y, 200)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"config": 4, "sims": len(sims), "half_steps": 200, "tile": tuned["tile"],
                      "zchunk": tuned["zchunk"], "ms_200_half_steps": e0.elapsed_time(e1),
                      "tuning_ms_per_half_step": tuned["ms"]}))
    for i in (0, 17, 40, 63):
        s = sims[i]
        p = Plan(s["m"], s["grid"], s["h"], s["c"], s["dt"], prec="fp32", state="fp32")
        x = torch.from_numpy(HI.gaussian_pulse(draw[i]["m"], draw[i]["n"], draw[i]["h"], draw[i]["centre"],
                                               draw[i]["sigma"])).float().cuda()
        y = torch.empty_like(x)
        for k in range(200):
            p.step(x, y, k % 2)
            x, y = y, x
        assert torch.equal(x, res[i]), i
    assert all(bool(torch.isfinite(t).all()) for t in res)


def test_batch_plan_validation(torch_cuda):
    from paper_1609_09841_gb300 import capi
    from paper_1609_09841_gb300.batch import BatchPlan
    bad = _sims([{"m": 2, "grid": (8, 8, 8)}], lam=0.4)
    with pytest.raises(capi.HermiteError) as e:
        BatchPlan(bad)
    assert e.value.code == capi.HERMITE_EUNSTABLE
    bp = BatchPlan(_sims([{"m": 1, "grid": (8, 8, 8)}]))
    torch = torch_cuda
    x = bp.empty()
    with pytest.raises(capi.HermiteError):
        bp.step(x, x, 0)
