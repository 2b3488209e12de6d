"""C-ABI checks of the advection plans (no GPU needed): argument validation,
the stability table against the oracle's symbol, calls that advection plans
refuse."""
import ctypes

import pytest

from oracle import advection as adv


@pytest.fixture(scope="module")
def capi():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1609_09841_gb300 import capi as c
    return c


def _adv(capi, m=2, grid=(8, 8, 8), h=None, a=(1.0, 1.0, 1.0), dt=None, q=0, prec=0, state=0, variant=0):
    h = h or tuple(1.0 / max(g, 1) for g in grid)
    dt = dt if dt is not None else 0.5 * min(h)
    p = ctypes.c_void_p()
    rc = capi.lib.hermite_adv_plan(ctypes.byref(p), m, (ctypes.c_int * 3)(*grid), (ctypes.c_double * 3)(*h),
                                   (ctypes.c_double * 3)(*a), dt, q, prec, state, variant)
    return rc, p


@pytest.mark.parametrize("kw,code", [
    (dict(m=0), -1), (dict(m=4), -1), (dict(grid=(0, 4, 4)), -1), (dict(h=(0.1, 0.0, 0.1)), -1),
    (dict(a=(1.0, float("nan"), 0.0)), -1), (dict(dt=0.0), -1), (dict(q=-1), -1), (dict(q=16), -1),
    (dict(prec=2), -4), (dict(prec=3), -4), (dict(prec=0, state=1), -4), (dict(variant=7), -1),
    (dict(q=8, variant=1), -4), (dict(dt=1.0), -5), (dict(q=1), -5),
    (dict(grid=(1 << 20, 1 << 11, 1)), -1),    # 2^31 nodes in one x1-x2 plane
])
def test_adv_plan_rejects(capi, kw, code):
    rc, p = _adv(capi, **kw)
    assert rc == code and not p.value


def test_adv_plan_accepts_and_refuses_wave_only_calls(capi):
    rc, p = _adv(capi, m=2, grid=(6, 5, 4))
    assert rc == 0
    assert capi.lib.hermite_state_elems(p) == 27 * 6 * 5 * 4
    assert capi.lib.hermite_schedule_count(p) == 6     # fused: three CTA heights x two load depths
    assert capi.lib.hermite_set_schedule(p, 5, 4) == 0
    assert capi.lib.hermite_set_schedule(p, 6, 4) == -1
    assert capi.lib.hermite_set_taylor_order(p, 6) == -4
    assert capi.lib.hermite_adjoint_step(p, None, None, 0, None) == -4
    assert capi.lib.hermite_step_dc(p, None, None, 0, None) == -4
    assert capi.lib.hermite_step_split_static(p, None, None, 0, None) == -4
    capi.lib.hermite_destroy(p)
    rc, p = _adv(capi, a=(0.0, 0.0, 0.0), q=1)      # no motion: any q is stable
    assert rc == 0
    capi.lib.hermite_destroy(p)
    rc, p = _adv(capi, m=3, q=5, dt=2 * 0.05 / 8)    # lam = 0.05 <= 0.05
    assert rc == 0
    capi.lib.hermite_destroy(p)


def test_adv_whole_series_limit_is_half_a_cell(capi):
    """Sec. 2: half a cell per half step, for every order, with the whole series."""
    for m in (1, 2, 3):
        assert capi.lib.hermite_adv_stability_limit(m, 0) == 0.5
        assert capi.lib.hermite_adv_stability_limit(m, 3 * (2 * m + 1)) == 0.5
    h = 1.0 / 8
    assert _adv(capi, m=3, dt=2 * 0.5 * h)[0] == 0
    assert _adv(capi, m=3, dt=2 * 0.501 * h)[0] == -5


TABLE_CASES = [(1, q) for q in range(1, 10)] + [(2, q) for q in range(1, 16)] + [(3, q) for q in (3, 5, 8, 12, 21)]


@pytest.mark.parametrize("m,q", TABLE_CASES)
def test_adv_stability_table_agrees_with_symbol(capi, m, q):
    """Each entry is stable by the oracle's advection symbol along x1 and on
    the diagonal, and 0.02 above it one of the two is unstable."""
    lim = capi.lib.hermite_adv_stability_limit(m, q)
    if lim > 0:
        assert adv.max_spectral_radius(m, lim, q=q, npts=13, dims=1) <= 1.0 + 1e-10
        assert adv.max_spectral_radius(m, lim, q=q, npts=7, dims=3) <= 1.0 + 1e-10
    above = lim + 0.02
    assert max(adv.max_spectral_radius(m, above, q=q, npts=13, dims=1),
               adv.max_spectral_radius(m, above, q=q, npts=7, dims=3)) > 1.0 + 1e-9
