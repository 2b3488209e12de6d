"""Accuracy of the mixed-precision variants at t = 1 (the precision workload):
m = 2, Gaussian pulse at (0.5, 0.5, 0.5) with sigma = 0.05, v0 = 0, c = 1,
dt = 0.4 h, run to t = 1.

* 16^3 (80 half steps): every GPU variant against the oracle's own run.
* 64^3 (320 half steps) and 256^3 (1280 half steps): the FP32-arithmetic
  variants against the FP64 GPU path (itself equal to the oracle to 1e-12 per
  half step, tests/test_gpu_parity.py).

Errors are relative max-norm (max|a-b| / max|b|) and relative L2 over every
component of both fields, and separately over the values (orders 0) of u and
of v; each test prints one JSON line per variant.

The hybrid modes (grade-0 contractions in FP64 or double-float, the rest in
FP32) and the remainder form (every factor applied to the one-sided Taylor
remainder, exact FP32 sums for the remainder and the grade-0 chain) must meet
the stated bar of 1e-5 relative at t = 1.  Measured, FP32
arithmetic meets it on the values of u at 64^3 and comes within 2x of it at
256^3, but the derivative components and v carry a rounding error that grows
linearly with the number of half steps (an O(eps32) perturbation of the
operator applied 320 / 1280 times): about 1.4e-4 at 64^3 and 8e-4 at 256^3 in
the relative max-norm over all components.  The assertions below are
regression guards at twice the measured errors, not the target."""
import json

import numpy as np
import pytest

import hermite_inputs as HI
from oracle import hermite as oracle

pytestmark = pytest.mark.gpu
GUARD = {16: 6e-5, 64: 3e-4, 256: 2e-3}     # twice the measured all-component max-norm error


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _run(torch, plan, x0, nhalf):
    x = (torch.from_numpy(x0).cuda() if isinstance(x0, np.ndarray) else x0).to(plan.torch_dtype, copy=True)
    y = torch.empty_like(x)
    for k in range(nhalf):
        plan.step(x, y, k % 2)
        x, y = y, x
    torch.cuda.synchronize()
    return x


def _setup(n1):
    m, n = 2, (n1,) * 3
    h = (1.0 / n1,) * 3
    dt = 0.4 * h[0]
    nhalf = int(round(1.0 / (dt / 2)))
    return m, n, h, dt, nhalf


VARIANTS = [("fp64", "fp64"), ("fp32", "fp64"), ("fp32", "fp32"), ("hybrid64", "fp64"), ("hybriddf", "fp64"),
            ("remainder", "fp64"), ("3xtf32", "fp32"), ("splitbf16", "fp32")]
BAR = 1e-5       # the stated bar for the mixed variants at t = 1
# The tensor-core variants (FP32 x- and y-passes, z-pass on tcgen05 with FP32
# accumulation) carry the FP32 arithmetic's error and more: the tensor cores'
# FP32 accumulation is not round-to-nearest, so its error does not average
# out over the half steps.  Their t = 1 errors are stated, not held to the
# bar; the guard only catches a broken kernel.
TC_GUARD = 1e-2


def _bound(prec, n1):
    if prec == "fp64":
        return 1e-12
    if prec == "fp32":
        return GUARD[n1]
    if prec in ("3xtf32", "splitbf16"):
        return TC_GUARD
    return BAR


def test_mixed_vs_oracle_16(torch_cuda):
    torch = torch_cuda
    from paper_1609_09841_gb300 import Plan
    m, n, h, dt, nhalf = _setup(16)
    x0 = HI.gaussian_pulse(m, n, h, sigma=0.05)
    ref = oracle.run(x0, m, h, 1.0, dt, nhalf)
    refd = torch.from_numpy(ref).cuda()
    for prec, state in VARIANTS:
        plan = Plan(m, n, h, 1.0, dt, prec=prec, state=state)
        out = _run(torch, plan, x0, nhalf)
        (mx, mrel, rms, l2rel), rc = plan.error(out, refd, 0b111)
        print(json.dumps({"grid": 16, "nhalf": nhalf, "prec": prec, "state": state, "vs": "oracle",
                          "max_rel": mrel, "l2_rel": l2rel}))
        assert rc == 0
        assert mrel <= _bound(prec, 16)


@pytest.mark.parametrize("n1", [64, 256])
def test_mixed_vs_fp64_gpu(torch_cuda, n1):
    torch = torch_cuda
    from paper_1609_09841_gb300 import Plan
    m, n, h, dt, nhalf = _setup(n1)
    x0 = torch.from_numpy(HI.gaussian_pulse(m, n, h, sigma=0.05)).cuda()
    ref_plan = Plan(m, n, h, 1.0, dt, prec="fp64", state="fp64")
    ref = _run(torch, ref_plan, x0, nhalf)
    for prec, state in VARIANTS[1:]:
        plan = Plan(m, n, h, 1.0, dt, prec=prec, state=state)
        out = _run(torch, plan, x0, nhalf)
        (mx, mrel, rms, l2rel), rc = plan.error(out, ref, 0b111)
        (mxu, mrelu, _, l2relu), _ = plan.error(out, ref, 0b001)
        (mxv, mrelv, _, l2relv), _ = plan.error(out, ref, 0b010)
        print(json.dumps({"grid": n1, "nhalf": nhalf, "prec": prec, "state": state, "vs": "fp64 gpu",
                          "max_rel": mrel, "l2_rel": l2rel, "u_values_max_rel": mrelu, "u_values_l2_rel": l2relu,
                          "v_values_max_rel": mrelv, "v_values_l2_rel": l2relv}))
        assert rc == 0
        assert mrel <= _bound(prec, n1)


def test_fp32_state_alone_misses_the_bar(torch_cuda):
    """Why the variants within the bar keep an FP64 state: the exact FP64
    half step, with only the state rounded to FP32 after every half step,
    already misses 1e-5 at t = 1 (64^3 here; the error grows with resolution:
    about 4e-5 / 9e-5 / 2e-4 at 64^3 / 128^3 / 256^3).  The rounding of the
    value components is a perturbation of size eps32 |u| at the grid scale,
    which the Laplacian terms of the next half steps amplify by 1/(k h)."""
    torch = torch_cuda
    from paper_1609_09841_gb300 import Plan
    m, n, h, dt, nhalf = _setup(64)
    x0 = torch.from_numpy(HI.gaussian_pulse(m, n, h, sigma=0.05)).cuda()
    plan = Plan(m, n, h, 1.0, dt, prec="fp64", state="fp64")
    ref = _run(torch, plan, x0, nhalf)
    a, b = x0.clone(), torch.empty_like(x0)
    for k in range(nhalf):
        plan.step(a, b, k % 2)
        a, b = b.float().double(), a
    (mx, mrel, _, _), rc = plan.error(a, ref, 0b111)
    print(json.dumps({"grid": 64, "fp64_state_rounded_to_fp32_each_half_step": mrel}))
    assert rc == 0 and mrel > BAR
