"""Host-side rules of the tensor-core precisions (no kernel runs): plan
arguments, schedules, Taylor order and the device status word."""
import pytest

PRECS = ["3xtf32", "splitbf16"]


def test_tc_plan_rules():
    from paper_1609_09841_gb300 import Plan, capi
    n = (8, 8, 8)
    h = (1 / 8,) * 3
    for prec in PRECS:
        with pytest.raises(capi.HermiteError) as e:
            Plan(2, n, h, 1.0, 0.4 / 8, prec=prec, variant="split")
        assert e.value.code == capi.HERMITE_EUNSUPPORTED
        with pytest.raises(capi.HermiteError) as e:
            Plan(2, n, h, 1.0, 0.4 / 8, prec=prec, q=6)
        assert e.value.code == capi.HERMITE_EUNSUPPORTED
        p = Plan(2, n, h, 1.0, 0.4 / 8, prec=prec, state="fp32")
        assert p.schedule_count() == 1
        assert capi.lib.hermite_set_taylor_order(p.handle, 5) == capi.HERMITE_EUNSUPPORTED
        assert p.device_status(stream=0) == 0    # nothing launched yet: no status word


def test_remainder_plan_rules():
    from paper_1609_09841_gb300 import Plan, capi
    n, h = (8, 8, 8), (1 / 8,) * 3
    for kw, code in (({"state": "fp32"}, capi.HERMITE_EUNSUPPORTED), ({"variant": "split"}, capi.HERMITE_EUNSUPPORTED),
                     ({"q": 6}, capi.HERMITE_EUNSUPPORTED)):
        with pytest.raises(capi.HermiteError) as e:
            Plan(2, n, h, 1.0, 0.4 / 8, prec="remainder", **kw)
        assert e.value.code == code, kw
    p = Plan(3, n, h, 1.0, 0.4 / 8, prec="remainder")
    assert p.schedule_count() == 3
