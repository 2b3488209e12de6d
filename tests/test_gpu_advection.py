"""Advection half step (Eq. 1 with a constant velocity) on the GPU against
the FP64 oracle: fused Kronecker kernel (whole series) and split pair (any q),
FP64 and FP32, host buffers, the 150^3 workload of Table 1 and convergence."""
from math import pi

import numpy as np
import pytest

import hermite_inputs as HI
from oracle import advection as adv
from oracle import hermite as oh

pytestmark = pytest.mark.gpu
EPS32 = 2.0 ** -24

# several 32-cell tiles along x1 with a ragged tail, several rows along x2 and
# zchunks along x3
GRIDS = {1: (37, 19, 21), 2: (35, 11, 18), 3: (33, 7, 17)}
VEL = (1.0, -0.7, 0.45)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _setup(m, lam=0.35):
    n = GRIDS[m]
    h = tuple(1.0 / v for v in n)
    dt = 2 * lam * min(hk / abs(ak) for hk, ak in zip(h, VEL))
    return n, h, dt


def _relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _fp32_bound(m, h, a, dt, q, x):
    """First-order forward-error bound of the FP32 path relative to max|ref|:
    (k + 2) eps32 max_rows (|T1 E_q| |H (x) H (x) H|) |x| with k the length
    of the longest chain of roundings (three passes of P terms, plus four per
    Horner stage for the split pair)."""
    P = 2 * m + 2
    H = np.abs(oh.hermite_matrix(m))
    H3 = np.kron(np.kron(H, H), H)                 # [jz jy jx][tz ty tx]
    E = np.eye(P ** 3).reshape(P ** 3, P, P, P)
    Eq = adv.evolve_taylor(E, 0.5 * dt, a, h, q).reshape(P ** 3, -1).T
    M = m + 1
    keep = [(jz * P + jy) * P + jx for jz in range(M) for jy in range(M) for jx in range(M)]
    R = np.abs(Eq[keep]) @ H3
    k = 3 * P + (0 if q >= adv.full_q(m) else 4 * q)
    return (k + 2) * EPS32 * R.sum(axis=1).max() * np.max(np.abs(x))


@pytest.mark.parametrize("m", [1, 2, 3])
@pytest.mark.parametrize("variant", ["fused", "split"])
def test_fp64_whole_series_matches_oracle(torch_cuda, m, variant):
    torch = torch_cuda
    from paper_1609_09841_gb300 import AdvectionPlan
    n, h, dt = _setup(m)
    plan = AdvectionPlan(m, n, h, VEL, dt, variant=variant)
    x = HI.advection_random_state(m, n, seed=300 + m)
    xd = torch.from_numpy(x).cuda()
    yd = torch.full_like(xd, float("nan"))
    for parity in (0, 1):
        plan.step(xd, yd, parity)
        ref = adv.half_step(x, m, h, VEL, dt, parity)
        assert _relmax(yd.cpu().numpy(), ref) <= 1e-12, parity


@pytest.mark.parametrize("m,q", [(1, 2), (1, 5), (2, 4), (2, 9), (3, 3), (3, 10)])
def test_fp64_split_any_q_matches_oracle(torch_cuda, m, q):
    torch = torch_cuda
    from paper_1609_09841_gb300 import AdvectionPlan, adv_stability_limit
    lam = 0.8 * adv_stability_limit(m, q)
    n, h, dt = _setup(m, lam)
    plan = AdvectionPlan(m, n, h, VEL, dt, q=q)
    x = HI.advection_random_state(m, n, seed=310 + q)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    for parity in (0, 1):
        plan.step(xd, yd, parity)
        ref = adv.half_step(x, m, h, VEL, dt, parity, q=q)
        assert _relmax(yd.cpu().numpy(), ref) <= 1e-12, parity


@pytest.mark.parametrize("m,q", [(1, 0), (2, 0), (3, 0), (2, 6), (3, 12)])
@pytest.mark.parametrize("state", ["fp32", "fp64"])
def test_fp32_within_forward_error_bound(torch_cuda, m, q, state):
    torch = torch_cuda
    from paper_1609_09841_gb300 import AdvectionPlan, adv_stability_limit
    qq = q or adv.full_q(m)
    n, h, dt = _setup(m, 0.8 * adv_stability_limit(m, qq))
    plan = AdvectionPlan(m, n, h, VEL, dt, q=q, prec="fp32", state=state)
    x = HI.advection_random_state(m, n, seed=320 + m).astype(np.float32).astype(np.float64)
    xd = torch.from_numpy(x).cuda().to(plan.torch_dtype)
    yd = torch.empty_like(xd)
    bound = _fp32_bound(m, h, VEL, dt, qq, x)
    for parity in (0, 1):
        plan.step(xd, yd, parity)
        ref = adv.half_step(x, m, h, VEL, dt, parity, q=qq)
        err = float(np.max(np.abs(yd.double().cpu().numpy() - ref)))
        assert err <= bound, (err, bound)


@pytest.mark.parametrize("variant", ["fused", "split"])
@pytest.mark.parametrize("prec,state", [("fp64", "fp64"), ("fp32", "fp32")])
def test_host_buffers_equal_device_buffers(torch_cuda, variant, prec, state):
    torch = torch_cuda
    from paper_1609_09841_gb300 import AdvectionPlan
    m = 2
    n, h, dt = _setup(m, 0.25)
    q = 0 if variant == "fused" else 8
    plan = AdvectionPlan(m, n, h, VEL, dt, q=q, prec=prec, state=state, variant=variant)
    dtype = np.float64 if state == "fp64" else np.float32
    x = HI.advection_random_state(m, n, seed=5).astype(dtype)
    for parity in (0, 1):
        y = np.empty_like(x)
        plan.step(x, y, parity)
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        plan.step(xd, yd, parity)
        torch.cuda.synchronize()
        assert np.array_equal(y, yd.cpu().numpy())


def test_zchunk_and_degenerate_grids(torch_cuda):
    """Every schedule (CTA shape and zchunk) gives the same result; grids of
    one node per dimension and a single CTA tile agree with the oracle."""
    torch = torch_cuda
    from paper_1609_09841_gb300 import AdvectionPlan
    m = 2
    for n in [(1, 1, 1), (1, 5, 3), (4, 1, 1), (32, 4, 2)]:
        h = tuple(1.0 / v for v in n)
        dt = 0.6 * min(hk / abs(ak) for hk, ak in zip(h, VEL))
        plan = AdvectionPlan(m, n, h, VEL, dt)
        x = HI.advection_random_state(m, n, seed=11)
        xd = torch.from_numpy(x).cuda()
        ref = adv.half_step(x, m, h, VEL, dt, 1)
        for tile in range(plan.schedule_count()):
            outs = []
            for zc in (1, 2, 16):
                plan.set_schedule(tile, zc)
                yd = torch.empty_like(xd)
                plan.step(xd, yd, 1)
                outs.append(yd.cpu().numpy())
            for o in outs:
                assert _relmax(o, ref) <= 1e-12, (n, tile)
            assert np.array_equal(outs[0], outs[2])


def test_many_steps_match_oracle_run(torch_cuda):
    torch = torch_cuda
    from paper_1609_09841_gb300 import AdvectionPlan
    m, n = 3, (12, 10, 9)
    h = tuple(1.0 / v for v in n)
    dt = 0.9 * min(h)                         # lam = 0.45 with |a| <= 1
    plan = AdvectionPlan(m, n, h, VEL, dt)
    x = HI.advection_random_state(m, n, seed=21)
    ref = adv.run(x, m, h, VEL, dt, 12)
    a = torch.from_numpy(x).cuda()
    b = torch.empty_like(a)
    for k in range(12):
        plan.step(a, b, k % 2)
        a, b = b, a
    assert _relmax(a.cpu().numpy(), ref) <= 1e-11


def test_table1_workload_sampled(torch_cuda):
    """150^3, m = 3, the whole series, FP32 (the paper's precision): sampled
    z layers, including both periodic ends, against the oracle."""
    torch = torch_cuda
    from paper_1609_09841_gb300 import AdvectionPlan
    m, n = 3, (150, 150, 150)
    h = (1.0 / 150,) * 3
    a = (1.0, 1.0, 1.0)
    dt = 0.9 * h[0]
    plan = AdvectionPlan(m, n, h, a, dt, prec="fp32", state="fp32")
    x = HI.advection_random_state(m, n, seed=1500, dtype=np.float32)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    zs = [0, 1, 74, 148, 149]
    x64 = x.astype(np.float64)
    bound = _fp32_bound(m, h, a, dt, adv.full_q(m), x64)
    for parity in (0, 1):
        plan.step(xd, yd, parity)
        ref = adv.half_step(x64, m, h, a, dt, parity, z_cells=zs)
        got = yd.cpu().numpy().astype(np.float64)
        err = float(np.max(np.abs(got[..., zs, :, :] - ref[..., zs, :, :])))
        assert err <= bound, (err, bound)
        assert torch.isfinite(yd).all()


@pytest.mark.parametrize("m,n0", [(1, 16), (2, 12), (3, 8)])
def test_plane_wave_convergence_on_gpu(torch_cuda, m, n0):
    """Sec. 2: error O(h^(2m+1)) for a smooth solution; the FP64 GPU path on
    n0^3 and (2 n0)^3 grids, plane wave along (1, 1, 1) to t = 0.25."""
    torch = torch_cuda
    from paper_1609_09841_gb300 import AdvectionPlan
    errs = []
    for n in (n0, 2 * n0):
        h = (1.0 / n,) * 3
        dt = 0.5 * h[0]
        plan = AdvectionPlan(m, (n,) * 3, h, (1.0, 1.0, 1.0), dt)
        a = torch.from_numpy(HI.plane_wave(m, (n,) * 3, h)).cuda()
        b = torch.empty_like(a)
        for k in range(2 * int(round(0.25 / dt))):
            plan.step(a, b, k % 2)
            a, b = b, a
        exact = HI.plane_wave(m, (n,) * 3, h, phase=2 * pi * 0.75)
        errs.append(float(np.max(np.abs(a.cpu().numpy()[0, 0, 0] - exact[0, 0, 0]))))
    assert np.log2(errs[0] / errs[1]) >= 2 * m + 1 - 0.5, errs


@pytest.mark.parametrize("m", [1, 2, 3])
@pytest.mark.parametrize("prec,state", [("fp64", "fp64"), ("fp32", "fp32"), ("fp32", "fp64")])
def test_every_fused_schedule_matches_oracle(torch_cuda, m, prec, state):
    """Each compiled CTA shape of the fused kernel, on the ragged multi-tile
    grids, against the oracle (FP64 1e-12, FP32 the forward-error bound)."""
    torch = torch_cuda
    from paper_1609_09841_gb300 import AdvectionPlan
    n, h, dt = _setup(m, 0.4)
    plan = AdvectionPlan(m, n, h, VEL, dt, prec=prec, state=state)
    x = HI.advection_random_state(m, n, seed=330 + m)
    if prec == "fp32":
        x = x.astype(np.float32).astype(np.float64)
    xd = torch.from_numpy(x).cuda().to(plan.torch_dtype)
    ref = adv.half_step(x, m, h, VEL, dt, 0)
    bound = 1e-12 * np.max(np.abs(ref)) if prec == "fp64" else _fp32_bound(m, h, VEL, dt, adv.full_q(m), x)
    for tile in range(plan.schedule_count()):
        plan.set_schedule(tile, 5)
        yd = torch.empty_like(xd)
        plan.step(xd, yd, 0)
        err = float(np.max(np.abs(yd.double().cpu().numpy() - ref)))
        assert err <= bound, (tile, err, bound)
