"""Host-side tests of the C ABI (no GPU needed): the library loads, exports
every entry point declared in include/*.h, validates plans, and its exact
rational tables agree with the oracle's."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from oracle import hermite as oracle_hermite
from oracle import symbol

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1609_09841_gb300 import capi as c
    return c


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(hdr).read(), flags=re.S)
        for mt in re.finditer(r"\b(hermite_[a-z0-9_]+)\s*\(", src):
            names.add(mt.group(1))
    return names


def test_every_declared_symbol_is_exported(capi):
    names = _declared_functions()
    assert "hermite_step" in names and "hermite_plan" in names
    for name in sorted(names):
        assert hasattr(capi.lib, name), name


def _plan(capi, m=1, grid=(8, 8, 8), h=None, c=1.0, dt=None, prec=0, state=0, variant=0):
    h = h or tuple(1.0 / max(g, 1) for g in grid)
    dt = dt if dt is not None else 0.4 * min(h)
    p = ctypes.c_void_p()
    rc = capi.lib.hermite_plan(ctypes.byref(p), m, (ctypes.c_int * 3)(*grid), (ctypes.c_double * 3)(*h),
                               c, dt, prec, state, variant)
    return rc, p


@pytest.mark.parametrize("kw,code", [
    (dict(m=0), -1), (dict(m=4), -1), (dict(grid=(0, 4, 4)), -1), (dict(h=(0.1, -0.1, 0.1)), -1),
    (dict(c=0.0), -1), (dict(dt=0.0), -1), (dict(prec=7), -4), (dict(state=5), -1),
    (dict(prec=0, state=1), -4), (dict(variant=9), -1), (dict(dt=1.0), -5),
    (dict(grid=((1 << 20) + 1, 2, 2)), -1),
    (dict(grid=(1 << 20, 1 << 11, 1)), -1),    # 2^31 nodes in one x1-x2 plane: 32-bit in-plane offsets
])
def test_plan_rejects_bad_arguments(capi, kw, code):
    rc, p = _plan(capi, **kw)
    assert rc == code, capi.last_error()
    assert not p.value
    assert capi.last_error()


def test_plan_accepts_the_largest_plane(capi):
    """grid[0] * grid[1] = 2^31 - 2^20 nodes is below the limit; the plan
    allocates nothing on the device, so this needs no GPU."""
    rc, p = _plan(capi, grid=(1 << 20, (1 << 11) - 1, 1))
    assert rc == 0, capi.last_error()
    capi.lib.hermite_destroy(p)


def test_plan_accepts_and_reports_sizes(capi):
    rc, p = _plan(capi, m=2, grid=(5, 6, 7))
    assert rc == 0
    assert capi.lib.hermite_state_elems(p) == 2 * 27 * 5 * 6 * 7
    capi.lib.hermite_destroy(p)
    capi.lib.hermite_destroy(None)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_library_H_equals_oracle_exact_H(capi, m):
    rc, p = _plan(capi, m=m)
    assert rc == 0
    P = 2 * m + 2
    buf = (ctypes.c_double * (P * P))()
    assert capi.lib.hermite_plan_operator(p, buf) == 0
    capi.lib.hermite_destroy(p)
    ref = np.array([[float(v) for v in row] for row in oracle_hermite.hermite_matrix_exact(m)])
    assert np.array_equal(np.array(buf).reshape(P, P), ref)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_stability_table_agrees_with_symbol(capi, m):
    """The library's limit is stable by the oracle's symbol, 4% above it is
    not, and plans straddling it are accepted / rejected."""
    lim = capi.lib.hermite_stability_limit(m)
    assert symbol.max_spectral_radius(m, lim, npts=7) <= 1.0 + 1e-10
    assert symbol.max_spectral_radius(m, lim * 1.04, npts=9) > 1.0 + 1e-9
    h = 1.0 / 16
    assert _plan(capi, m=m, grid=(16,) * 3, dt=2 * lim * h * 0.999)[0] == 0
    assert _plan(capi, m=m, grid=(16,) * 3, dt=2 * lim * h * 1.01)[0] == -5


def test_step_without_gpu_fails_cleanly(capi):
    """On a machine without a CUDA device the step reports an error code
    instead of crashing (skipped when a GPU is present)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, p = _plan(capi)
    assert rc == 0
    a = np.zeros(capi.lib.hermite_state_elems(p))
    b = np.zeros_like(a)
    rc = capi.lib.hermite_step(p, a.ctypes.data_as(ctypes.c_void_p), b.ctypes.data_as(ctypes.c_void_p), 0, None)
    assert rc < 0
    capi.lib.hermite_destroy(p)


def test_schedule_validation(capi):
    rc, p = _plan(capi, m=3, prec=1, state=1)
    assert rc == 0
    count = capi.lib.hermite_schedule_count(p)
    assert count >= 2
    assert capi.lib.hermite_set_schedule(p, count - 1, 8) == 0
    assert capi.lib.hermite_set_schedule(p, count, 8) == -1
    assert capi.lib.hermite_set_schedule(p, 0, 0) == -1
    assert capi.lib.hermite_set_schedule(None, 0, 8) == -1
    capi.lib.hermite_destroy(p)


def test_batched_plan_rejected_by_single_calls_without_gpu(capi):
    """Argument checks of the batched plan that need no device."""
    p = ctypes.c_void_p()
    one = (ctypes.c_int * 1)(1)
    g = (ctypes.c_int * 3)(8, 8, 8)
    h = (ctypes.c_double * 3)(0.125, 0.125, 0.125)
    c = (ctypes.c_double * 1)(1.0)
    dt_bad = (ctypes.c_double * 1)(1.0)
    assert capi.lib.hermite_batch_plan(ctypes.byref(p), 0, one, g, h, c, dt_bad, 1, 1) == -1
    assert capi.lib.hermite_batch_plan(ctypes.byref(p), 1, one, g, h, c, dt_bad, 1, 1) == -5
    assert capi.lib.hermite_batch_plan(ctypes.byref(p), 1, one, g, h, c, dt_bad, 0, 1) == -4
    assert not p.value


def test_batch_tile_shapes_without_gpu(capi):
    """The batched kernel's two tile shapes per order, and the range checks of
    hermite_batch_tile_shape / hermite_batch_set_tiles."""
    want = {(1, 0): (16, 8), (1, 1): (8, 8), (2, 0): (16, 4), (2, 1): (8, 4), (3, 0): (8, 2), (3, 1): (4, 4)}
    tx, ty = ctypes.c_int(), ctypes.c_int()
    for (m, t), shape in want.items():
        assert capi.lib.hermite_batch_tile_shape(m, t, ctypes.byref(tx), ctypes.byref(ty)) == 0
        assert (tx.value, ty.value) == shape
    for m, t in ((0, 0), (4, 0), (1, -1), (2, 2)):
        assert capi.lib.hermite_batch_tile_shape(m, t, ctypes.byref(tx), ctypes.byref(ty)) == -1
    assert capi.lib.hermite_batch_set_tiles(None, (ctypes.c_int * 3)(0, 0, 0)) == -1
    rc, p = _plan(capi)
    assert rc == 0
    assert capi.lib.hermite_batch_set_tiles(p, (ctypes.c_int * 3)(0, 0, 0)) == -1   # not a batched plan
    capi.lib.hermite_destroy(p)


def test_taylor_order_validation(capi):
    rc, p = _plan(capi, m=2)
    assert rc == 0
    assert capi.lib.hermite_taylor_order(p) == 4
    assert capi.lib.hermite_set_taylor_order(p, 3) == -1
    assert capi.lib.hermite_set_taylor_order(p, 16) == -1          # 3(2m+1) = 15
    assert capi.lib.hermite_set_taylor_order(p, 15) == 0
    assert capi.lib.hermite_taylor_order(p) == 15
    capi.lib.hermite_destroy(p)
    rc, p = _plan(capi, m=2, prec=capi.HERMITE_HYBRIDDF, state=0)    # double-float hybrid
    assert rc == 0
    assert capi.lib.hermite_set_taylor_order(p, 6) == -4
    assert capi.lib.hermite_set_taylor_order(p, 4) == 0
    capi.lib.hermite_destroy(p)


Q_TABLE_CASES = [(1, q) for q in range(4, 10)] + [(2, q) for q in range(4, 16)] + [(3, 5), (3, 6), (3, 21)]


@pytest.mark.parametrize("m,q", Q_TABLE_CASES)
def test_taylor_stability_table_agrees_with_symbol(capi, m, q):
    """Each entry of the per-q table is stable by the oracle's symbol of the
    q-stage Taylor half step and 0.02 above it is not (entries are rounded
    down to two decimals, so 0.02 above is past the true limit)."""
    lim = capi.lib.hermite_stability_limit_taylor(m, q)
    assert lim > 0
    assert symbol.max_spectral_radius(m, lim, npts=7, evolve="taylor", q=q) <= 1.0 + 1e-10
    assert symbol.max_spectral_radius(m, lim + 0.02, npts=7, evolve="taylor", q=q) > 1.0 + 1e-9


def _plan_q(capi, m, q, dt, grid=(16, 16, 16), prec=0):
    h = tuple(1.0 / g for g in grid)
    p = ctypes.c_void_p()
    rc = capi.lib.hermite_plan_taylor(ctypes.byref(p), m, (ctypes.c_int * 3)(*grid), (ctypes.c_double * 3)(*h),
                                      1.0, dt, prec, 0, 0, q)
    return rc, p


def test_plan_taylor_checks_its_own_limit(capi):
    """A full-series plan accepts a step RK4 rejects; a lower q that is less
    stable rejects a step RK4 accepts; set_taylor_order checks the same."""
    h = 1.0 / 16
    assert capi.lib.hermite_stability_limit_taylor(2, 3) == 0.0
    assert capi.lib.hermite_stability_limit_taylor(2, 16) == 0.0
    assert capi.lib.hermite_stability_limit_taylor(2, 4) == capi.lib.hermite_stability_limit(2)
    big = 2 * 0.40 * h                      # lam = 0.40: above RK4's 0.30, below the full series' 0.42
    assert _plan_q(capi, 2, 4, big)[0] == -5
    rc, p = _plan_q(capi, 2, 15, big)
    assert rc == 0 and capi.lib.hermite_taylor_order(p) == 15
    assert capi.lib.hermite_set_taylor_order(p, 4) == -5    # would be unstable: refused, q kept
    assert capi.lib.hermite_taylor_order(p) == 15
    capi.lib.hermite_destroy(p)
    mid = 2 * 0.15 * h                      # lam = 0.15: fine for RK4 (0.26), not for m = 3, q = 5 (0.09)
    assert _plan_q(capi, 3, 5, mid)[0] == -5
    rc, p = _plan_q(capi, 3, 4, mid)
    assert rc == 0
    assert capi.lib.hermite_set_taylor_order(p, 5) == -5
    assert capi.lib.hermite_set_taylor_order(p, 21) == 0
    capi.lib.hermite_destroy(p)
    assert _plan_q(capi, 2, 6, 2 * 0.2 * h, prec=capi.HERMITE_HYBRID64)[0] == -4   # hybrid: q = 4 only
    assert _plan_q(capi, 2, 2, 2 * 0.2 * h)[0] == -1
