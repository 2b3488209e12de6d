"""Bounds checks of the debug build on the GPU.

* Every fused precision runs a half step through libhermite_debug.so on
  small ragged grids: no access is flagged, and the result equals the release
  library's bit for bit (the checks change no arithmetic).
* hermite_debug_selftest tells the kernels that the state holds half its
  elements: the loads and stores past that are flagged (bits 1 and 2) with
  the first offending offset at the half, and skipped -- on full-size
  buffers, so no access could leave them in any case.
* hermite_debug_wait_drill runs a half step whose awaited work (the plane
  copies of a staged FP32 schedule, the MMAs of the tensor-core kernel) is
  never issued: every bounded wait runs out, the status bit is set, and the
  next ordinary step gives the same bits as before the drill."""
import ctypes

import numpy as np
import pytest

import hermite_inputs as HI

pytestmark = pytest.mark.gpu
PRECS = {"fp64": (0, 0), "fp32": (1, 1), "hybriddf": (5, 0), "3xtf32": (2, 1), "remainder": (6, 0)}


@pytest.fixture(scope="module")
def libs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os, sys
    import __graft_entry__
    __graft_entry__.build()
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                    "paper_1609_09841_gb300"))
    import build as builder
    from paper_1609_09841_gb300 import capi
    return torch, capi, capi.load_library(builder.build(debug=True))


def _plan(lib, m, n, prec, state):
    p = ctypes.c_void_p()
    h = (ctypes.c_double * 3)(*(1.0 / v for v in n))
    rc = lib.hermite_plan(ctypes.byref(p), m, (ctypes.c_int * 3)(*n), h, 1.0, 0.4 / max(n), prec, state, 1)
    assert rc == 0
    return p


def _status(lib, p):
    f, first = ctypes.c_int(), ctypes.c_ulonglong()
    assert lib.hermite_debug_status(p, ctypes.byref(f), ctypes.byref(first), None) == 0
    return f.value, first.value


@pytest.mark.parametrize("name", list(PRECS))
@pytest.mark.parametrize("m,n", [(1, (19, 13, 11)), (3, (9, 6, 5)), (2, (1, 3, 2))])
def test_debug_build_flags_nothing_and_matches_release(libs, name, m, n):
    torch, capi, dbg = libs
    prec, state = PRECS[name]
    x = HI.random_state(m, n, seed=11)
    dt = torch.float64 if state == 0 else torch.float32
    xd = torch.from_numpy(x).to(dt).cuda()
    for parity in (0, 1):
        outs = []
        for lib in (capi.lib, dbg):
            p = _plan(lib, m, n, prec, state)
            y = torch.full_like(xd, float("nan"))
            assert lib.hermite_step(p, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(y.data_ptr()), parity, None) == 0
            torch.cuda.synchronize()
            if lib is dbg:
                assert _status(dbg, p) == (0, 2 ** 64 - 1)
            lib.hermite_destroy(p)
            outs.append(y.cpu().numpy())
        assert np.array_equal(outs[0], outs[1]), parity


@pytest.mark.parametrize("name", list(PRECS))
def test_debug_selftest_flags_and_skips_accesses_past_the_bound(libs, name):
    torch, capi, dbg = libs
    prec, state = PRECS[name]
    m, n = 2, (9, 8, 7)
    x = HI.random_state(m, n, seed=12)
    dt = torch.float64 if state == 0 else torch.float32
    xd = torch.from_numpy(x).to(dt).cuda()
    y = torch.full_like(xd, 7.0)
    p = _plan(dbg, m, n, prec, state)
    elems = dbg.hermite_state_elems(p)
    rc = dbg.hermite_debug_selftest(p, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(y.data_ptr()), 0, 0.5, None)
    assert rc == 0
    torch.cuda.synchronize()
    flags, first = _status(dbg, p)
    assert flags == 2 | 4 and first == elems // 2
    flat = y.flatten().cpu().numpy()
    assert np.all(flat[elems // 2:] == 7.0)        # stores past the bound were skipped
    assert _status(dbg, p) == (0, 2 ** 64 - 1)     # cleared by the read
    dbg.hermite_destroy(p)


@pytest.mark.parametrize("name,m,n,tile", [("fp32", 3, (24, 12, 8), 6), ("fp32", 2, (24, 12, 8), 7),
                                           ("3xtf32", 3, (16, 12, 8), 0)])
def test_wait_drill_sets_status_and_leaves_the_context_usable(libs, name, m, n, tile):
    """The drill's waits give up after a few polls and set bit 0 of the status
    word; nothing is left waiting, and the plan and the context keep working."""
    torch, capi, dbg = libs
    prec, state = PRECS[name]
    p = _plan(dbg, m, n, prec, state)
    assert dbg.hermite_set_schedule(p, tile, 4) == 0
    x = HI.random_state(m, n, seed=12)
    xd = torch.from_numpy(x).to(torch.float32).cuda()
    xp, yp = ctypes.c_void_p(xd.data_ptr()), None
    before = torch.empty_like(xd)
    assert dbg.hermite_step(p, xp, ctypes.c_void_p(before.data_ptr()), 0, None) == 0
    st = ctypes.c_int()
    assert dbg.hermite_device_status(p, ctypes.byref(st), None) == 0 and st.value == 0
    y = torch.empty_like(xd)
    yp = ctypes.c_void_p(y.data_ptr())
    assert dbg.hermite_debug_wait_drill(p, xp, yp, 0, None) == 0
    assert dbg.hermite_device_status(p, ctypes.byref(st), None) == 0 and st.value == 1
    after = torch.full_like(xd, float("nan"))
    assert dbg.hermite_step(p, xp, ctypes.c_void_p(after.data_ptr()), 0, None) == 0
    assert dbg.hermite_device_status(p, ctypes.byref(st), None) == 0 and st.value == 0
    assert torch.equal(before, after)
    dbg.hermite_destroy(p)


def test_wait_drill_rejects_plans_without_bounded_waits(libs):
    torch, capi, dbg = libs
    p = _plan(dbg, 2, (8, 8, 8), 1, 1)     # FP32, default tile 0: plain loads, no waits
    x = torch.zeros(2 * 27 * 512, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    rc = dbg.hermite_debug_wait_drill(p, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), 0, None)
    assert rc == capi.HERMITE_EINVAL
    dbg.hermite_destroy(p)
