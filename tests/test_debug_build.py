"""The debug build (libhermite_debug.so, -DHERMITE_DEBUG) compiles, exports
the same C ABI and says that it is a debug build; the release library says it
is not and refuses the self-test and the wait drill.  The checks themselves run on the GPU
(tests/test_gpu_debug_build.py)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_library_builds_and_identifies_itself():
    sys.path.insert(0, os.path.join(ROOT, "paper_1609_09841_gb300"))
    import build as builder
    path = builder.build(debug=True)
    from paper_1609_09841_gb300 import capi
    dbg = capi.load_library(path)
    assert dbg.hermite_debug_build() == 1
    assert capi.lib.hermite_debug_build() == 0
    assert capi.lib.hermite_debug_selftest(None, None, None, 0, 0.5, None) == capi.HERMITE_EUNSUPPORTED
    assert capi.lib.hermite_debug_wait_drill(None, None, None, 0, None) == capi.HERMITE_EUNSUPPORTED
    assert dbg.hermite_debug_wait_drill(None, None, None, 0, None) == capi.HERMITE_EINVAL
