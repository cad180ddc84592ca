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


def test_gelman_diag_matches_the_oracle_on_raw_chains():
    """fsmp_gelman_diag (the degrees-of-freedom corrected R with its upper confidence limit, from
    summaries) against the oracle's gelman_diag on the raw sample chains (numpy, scipy's F
    quantile), for every field it reads, at the paper's 90 % and at 95 %: chains of one
    distribution, chains apart, chains of unequal spread, few and many chains."""
    _lib_or_skip()
    from oracle import convergence
    rng = np.random.default_rng(21)
    fields = {fsmp.RHAT_N: ("mean_N", "var_N"), fsmp.RHAT_T0: ("mean_t0", "var_t0"),
              fsmp.RHAT_Q: ("mean_Q", "var_Q"), fsmp.RHAT_WT: ("mean_wt", "var_wt"),
              fsmp.RHAT_WE: ("mean_we", "var_we")}
    n_cases = 0
    for m in (2, 3, 4, 8, 16):
        for n in (10, 200, 3000):
            for spread in (0.0, 0.1, 1.0, 5.0):
                x = rng.normal(0, 1, (m, n)) * rng.uniform(0.5, 1.5, (m, 1)) + spread * rng.normal(0, 1, (m, 1))
                x = 3.0 * x + 40.0
                for field, (fm, fv) in fields.items():
                    s = np.zeros(m, fsmp.SUMMARY_DTYPE)
                    s[fm], s[fv], s["n_samples"] = x.mean(1), x.var(1), n
                    for conf in (0.9, 0.95):
                        r, u = fsmp.gelman_diag(s, field, conf)
                        r0, u0 = convergence.gelman_diag(x, conf)
                        assert abs(r - r0) <= 1e-9 * r0 and abs(u - u0) <= 1e-9 * u0, (m, n, spread, field, r, r0, u, u0)
                n_cases += 1
    # equal within-chain variances: the chi-square limit of the upper limit
    base = rng.normal(0, 1, 500)
    x = np.stack([base + c for c in (0.0, 0.1, -0.2)])
    s = np.zeros(3, fsmp.SUMMARY_DTYPE)
    s["mean_wt"], s["var_wt"], s["n_samples"] = x.mean(1), x.var(1), 500
    r, u = fsmp.gelman_diag(s, fsmp.RHAT_WT)
    r0, u0 = convergence.gelman_diag(x)
    assert abs(r - r0) <= 1e-9 * r0 and abs(u - u0) <= 1e-9 * u0
    with pytest.raises(fsmp.FsmpError):
        fsmp.gelman_diag(s, fsmp.RHAT_WT, 1.0)
    assert n_cases == 60
