"""fsmp_gelman_rubin (host code in the library; no GPU): the summary-based R equals the
textbook Gelman-Rubin statistic computed from raw sample chains, and its limits."""
import numpy as np
import pytest

from paper_2403_03156_gb300 import fsmp


def _lib_or_skip():
    try:
        return fsmp.load()
    except Exception as e:  # the library needs the CUDA runtime to load
        pytest.skip("library not loadable here: %s" % e)


def _summaries_from_chains(x):
    """Per-chain mean and population variance of raw samples x[m, n], as the kernels report."""
    s = np.zeros(len(x), fsmp.SUMMARY_DTYPE)
    s["mean_N"] = x.mean(1)
    s["var_N"] = x.var(1)
    s["mean_t0"] = x.mean(1)
    s["var_t0"] = x.var(1)
    s["n_samples"] = x.shape[1]
    return s


def _rhat_raw(x):
    m, n = x.shape
    W = x.var(1, ddof=1).mean()
    B = n * x.mean(1).var(ddof=1)
    return np.sqrt(((n - 1) / n * W + B / n) / W)


def test_rhat_matches_raw_chains():
    _lib_or_skip()
    rng = np.random.default_rng(0)
    for shift in (0.0, 0.3, 2.0):
        x = rng.normal(0, 1, (4, 500)) + shift * np.arange(4)[:, None]
        s = _summaries_from_chains(x)
        assert abs(fsmp.gelman_rubin(s, fsmp.RHAT_N) - _rhat_raw(x)) < 1e-12
        assert abs(fsmp.gelman_rubin(s, fsmp.RHAT_T0) - _rhat_raw(x)) < 1e-12


def test_rhat_limits():
    _lib_or_skip()
    rng = np.random.default_rng(1)
    same = np.tile(rng.normal(0, 1, 300), (3, 1))  # identical chains: B = 0
    assert abs(fsmp.gelman_rubin(_summaries_from_chains(same)) - np.sqrt(299 / 300)) < 1e-12
    mixed = rng.normal(0, 1, (8, 4000))  # independent chains of one distribution
    assert abs(fsmp.gelman_rubin(_summaries_from_chains(mixed)) - 1.0) < 0.01
    apart = rng.normal(0, 1, (4, 400)) + 5.0 * np.arange(4)[:, None]
    assert fsmp.gelman_rubin(_summaries_from_chains(apart)) > 1.1
    const = np.ones((3, 10))
    assert fsmp.gelman_rubin(_summaries_from_chains(const)) == 1.0
    with pytest.raises(fsmp.FsmpError):
        fsmp.gelman_rubin(_summaries_from_chains(const)[:1])
