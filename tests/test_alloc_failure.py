"""Allocation failures are reported as HERMITE_ENOMEM and leave the library
usable: every host and device allocation goes through one gate, and
hermite_inject_alloc_failure(skip, count) makes the count allocations after
the next skip ones fail.  Plan creation allocates on the host only, so it is
tested here without a GPU; the device allocations are in
tests/test_gpu_alloc_failure.py."""
import ctypes

import pytest

from paper_1609_09841_gb300 import Plan, capi


@pytest.fixture(autouse=True)
def disarm():
    yield
    capi.lib.hermite_inject_alloc_failure(0, 0)


def _plan_rc(m=2, n=(8, 8, 8)):
    p = ctypes.c_void_p()
    h = (ctypes.c_double * 3)(*(1.0 / v for v in n))
    rc = capi.lib.hermite_plan(ctypes.byref(p), m, (ctypes.c_int * 3)(*n), h, 1.0, 0.4 / n[0], 0, 0, 1)
    return rc, p


def test_plan_creation_reports_enomem_then_recovers():
    assert capi.lib.hermite_inject_alloc_failure(0, 1) == 0
    rc, p = _plan_rc()
    assert rc == capi.HERMITE_ENOMEM and not p.value
    rc, p = _plan_rc()                       # the window is spent
    assert rc == capi.HERMITE_OK and p.value
    capi.lib.hermite_destroy(p)


def test_skip_counts_successful_allocations():
    assert capi.lib.hermite_inject_alloc_failure(2, 1) == 0
    plans = []
    for _ in range(2):                       # two plans allocate one block each
        rc, p = _plan_rc()
        assert rc == capi.HERMITE_OK
        plans.append(p)
    rc, p = _plan_rc()
    assert rc == capi.HERMITE_ENOMEM and not p.value
    for p in plans:
        capi.lib.hermite_destroy(p)


def test_advection_and_batched_plans_report_enomem():
    capi.lib.hermite_inject_alloc_failure(0, 1)
    p = ctypes.c_void_p()
    n = (ctypes.c_int * 3)(8, 8, 8)
    h = (ctypes.c_double * 3)(0.125, 0.125, 0.125)
    a = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    assert capi.lib.hermite_adv_plan(ctypes.byref(p), 1, n, h, a, 0.1, 0, 1, 1, 0) == capi.HERMITE_ENOMEM
    assert not p.value
    capi.lib.hermite_inject_alloc_failure(0, 1)
    one = (ctypes.c_int * 1)(2)
    c = (ctypes.c_double * 1)(1.0)
    dt = (ctypes.c_double * 1)(0.04)
    rc = capi.lib.hermite_batch_plan(ctypes.byref(p), 1, one, n, h, c, dt, 1, 1)
    assert rc == capi.HERMITE_ENOMEM and not p.value


def test_python_plan_raises_and_hook_rejects_negative():
    capi.lib.hermite_inject_alloc_failure(0, 1)
    with pytest.raises(capi.HermiteError) as e:
        Plan(1, (4, 4, 4), (0.25,) * 3, 1.0, 0.1)
    assert e.value.code == capi.HERMITE_ENOMEM
    assert capi.lib.hermite_inject_alloc_failure(-1, 1) == capi.HERMITE_EINVAL
