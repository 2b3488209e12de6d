"""The batched autotuner's search on the host: a stand-in plan records the
schedule it is given and a synthetic timer prices it, so the coordinate search
over (tile, z-chunk) per order runs without a GPU."""
import pytest


@pytest.fixture(scope="module")
def at():
    import __graft_entry__
    __graft_entry__.build()            # the package loads libhermite.so on import
    from paper_1609_09841_gb300 import autotune
    return autotune


class FakeBatchPlan:
    def __init__(self, orders):
        self.sims = [{"m": m} for m in orders]
        self.tiles, self.zchunk = None, None

    def set_tiles(self, tiles):
        self.tiles = list(tiles)

    def set_schedule(self, zchunk):
        self.zchunk = list(zchunk)


def separable_cost(at, best, present):
    """Sum over the orders present of a bowl around best[m] = (tile, zchunk)."""
    def cost(p):
        total = 0.0
        for m in present:
            t, z = p.tiles[m - 1], p.zchunk[m - 1]
            bt, bz = best[m]
            total += m * (1.0 + 0.3 * abs(t - bt) + abs(at.BATCH_ZCHUNKS.index(z) - at.BATCH_ZCHUNKS.index(bz)))
        return total
    return cost


@pytest.mark.parametrize("present", [(1, 2, 3), (3,), (1, 3)])
def test_tune_batch_finds_the_minimum_of_a_separable_cost(at, present):
    best = {1: (1, 48), 2: (0, 8), 3: (1, 96)}
    plan = FakeBatchPlan(present)
    res = at.tune_batch(plan, None, None, timer=separable_cost(at, best, present))
    for m in present:
        assert (res["tile"][m - 1], res["zchunk"][m - 1]) == best[m], m
    assert res["ms"] == pytest.approx(sum(present))
    # the choice is applied to the plan last
    assert plan.tiles == res["tile"] and plan.zchunk == res["zchunk"]


def test_tune_batch_times_the_start_triples_first_and_every_option_per_order(at):
    plan = FakeBatchPlan((1, 2, 3))
    res = at.tune_batch(plan, None, None, timer=lambda p: 1.0, sweeps=1)
    starts = [k for k in res["table"] if k.startswith("start")]
    assert len(starts) == len(at.BATCH_STARTS)
    per_order = [k for k in res["table"] if k.startswith("sweep 0 m=2")]
    # every (tile, zchunk) pair but the current choice
    assert len(per_order) == len(at.BATCH_TILES) * len(at.BATCH_ZCHUNKS) - 1
    # nothing beat the first start: it stays chosen, with the first shapes
    assert res["zchunk"] == list(at.BATCH_STARTS[0]) and res["tile"] == [0, 0, 0]


def test_tune_batch_leaves_orders_absent_from_the_batch_alone(at):
    plan = FakeBatchPlan((2,))
    res = at.tune_batch(plan, None, None, timer=separable_cost(at, {2: (1, 64)}, (2,)))
    assert res["tile"][1] == 1 and res["zchunk"][1] == 64
    assert res["tile"][0] == 0 and res["tile"][2] == 0
    assert not any(k.startswith("sweep 0 m=1") or k.startswith("sweep 0 m=3") for k in res["table"])
