"""Helpers shared by the GPU tests: contexts from workload parameters and comparison of
chain traces with the oracle's."""
import numpy as np

from paper_2403_03156_gb300 import fsmp

# log u is never below log(2^-54) = -37.4, so any log acceptance below -40 is a certain
# reject on both sides; such values (and -inf) compare equal.
LA_FLOOR = -40.0


def context(params, **kw):
    return fsmp.Context(params, **kw)


def compare_traces(gpu, orc, rel=1e-9):
    """Same decisions, same N and t0 path, log acceptance ratios equal to rel (floor 1)."""
    assert gpu.shape == orc.shape
    np.testing.assert_array_equal(gpu["flags"], orc["flags"])
    np.testing.assert_array_equal(gpu["N"], orc["N"])
    np.testing.assert_array_equal(gpu["k0"], orc["k0"])
    np.testing.assert_array_equal(gpu["jump"], orc["jump"])
    for f in ("la", "la0"):
        a, b = gpu[f], orc[f]
        nan_a, nan_b = np.isnan(a), np.isnan(b)
        np.testing.assert_array_equal(nan_a, nan_b)
        a = np.maximum(np.where(nan_a, 0.0, a), LA_FLOOR)
        b = np.maximum(np.where(nan_b, 0.0, b), LA_FLOOR)
        err = np.abs(a - b) / np.maximum(1.0, np.abs(b))
        assert err.max() <= rel, (f, err.max(), np.unravel_index(err.argmax(), err.shape))
    # The log uniforms each side compared its ratios with: the same Philox outputs, the same
    # u = ((x >> 11) + 0.5) 2^-53 and the same order of use within a step (u2 for t0, u7 for
    # the jump), up to the last-place rounding of the two libm logs. lu0 exists only where t0
    # was proposed.
    for f, where in (("lu", np.ones(orc.shape, bool)), ("lu0", (orc["flags"] & 1) != 0)):
        a, b = gpu[f][where], orc[f][where]
        assert np.all(np.isfinite(a)) and np.all(np.isfinite(b)), f
        err = np.abs(a - b) / np.maximum(np.abs(b), 1e-300)
        assert err.max(initial=0.0) <= 1e-15, (f, err.max(), np.unravel_index(err.argmax(), err.shape))
    return True
