"""Hermite half step of the 3-D scalar wave equation on one GB300 (sm_103a).

``Plan`` wraps the C ABI of libhermite (include/hermite.h); the arithmetic
runs only in that CUDA library, which must be built (``build.build()``)."""
from .hermite import (AdvectionPlan, Plan, adv_max_dt, adv_stability_limit, adv_symbol_radius,  # noqa: F401
                      adv_max_radius, max_dt, max_radius, stability_limit, symbol_radius)
