"""Pins of the oracle's convergence diagnostics (Sec. 3.2, CPU only): the Wasserstein scalar of
a PE sequence with its dummy PE, and the Gelman-Rubin R with its upper confidence limit.

Sources other than the oracle itself: scipy's wasserstein_distance, closed forms of the
scalar's expectation in the prior-only limit of the chain (Eq. (pzmu) restricted to T: N
Poisson, positions iid proportional to phi), exact special cases of R, its invariance under
affine changes of units, and scipy's chi-square quantile for the F(m - 1, inf) limit."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import convergence
from paper_2403_03156_gb300 import workloads
from tests import model_ref

C1 = workloads.CONFIGS["plain_fp64_256x128"]["params"]


# ---------------------------------------------------------------- the Wasserstein scalar
def test_wasserstein1_matches_scipy(orc):
    """The 1-Wasserstein distance of two 1-D empirical distributions (unequal sizes, ties,
    negative values) against scipy.stats.wasserstein_distance."""
    rng = np.random.default_rng(7)
    for _ in range(300):
        a = rng.normal(0, 30, rng.integers(1, 40))
        b = rng.normal(5, 10, rng.integers(1, 40))
        if rng.random() < 0.3:  # ties
            a = np.round(a / 4) * 4
            b = np.round(b / 4) * 4
        assert abs(orc.wasserstein1(a, b) - stats.wasserstein_distance(a, b)) <= 1e-12 * max(1.0, abs(a).max())


def test_pe_wasserstein_has_the_dummy_pe(orc):
    """The scalar of a sequence is its distance, with a dummy PE at 0 added, to the dummy alone:
    0 for an empty sequence, |t| / 2 for one PE, scipy's distance otherwise."""
    assert orc.pe_wasserstein([]) == 0.0
    assert orc.pe_wasserstein([7.5]) == pytest.approx(3.75, abs=1e-15)
    rng = np.random.default_rng(3)
    for n in (2, 5, 40, 384):
        v = rng.uniform(0, 1000, n)
        want = stats.wasserstein_distance(np.r_[0.0, v], [0.0])
        assert abs(orc.pe_wasserstein(v) - want) <= 1e-12 * want


def _prior_only_batch(n_chains, n_steps, burn_in, T_lo, T_hi, lam0, n=64):
    return dict(samples=np.zeros(n * n_chains, np.float32), offsets=np.arange(n_chains + 1, dtype=np.int32) * n,
                lambda0=np.full(n_chains, lam0), t_origin_ns=np.zeros(n_chains),
                T_lo=np.full(n_chains, T_lo, np.int32), T_hi=np.full(n_chains, T_hi, np.int32),
                seed=11, index_base=0, n_steps=n_steps, burn_in=burn_in)


def _check(per_chain, exact, k=4.0, floor=2e-3):
    m = per_chain.mean()
    se = per_chain.std(ddof=1) / math.sqrt(len(per_chain))
    assert abs(m - exact) <= k * se + floor, (m, exact, se)


def test_wasserstein_scalar_prior_only_closed_form(orc):
    """Delta nu := 0, t0 fixed: N ~ Poisson(lambda0 Phi_T) truncated at n_cap and the PE times
    iid proportional to phi on T, so the time scalar sum_k t_k / (N + 1) has expectation
    E[N / (N + 1)] E[t], and the component scalar of the dynode model is 0. The chains'
    post-burn-in means of the scalar must match (4 SE over 64 independent chains)."""
    params = dict(C1, prior_only=1, sample_t0=0, t0_lo=30.0, t0_hi=30.0, n_cap=12)
    T_lo, T_hi, lam0 = 100, 180, 3.0
    s, tr = orc.run_batch(params, _prior_only_batch(64, 8000, 500, T_lo, T_hi, lam0), orc.MODE_INCREMENTAL,
                          n_threads=8, trace=True)
    g = params["grid_ns"]
    j = np.arange(T_lo, T_hi)
    ph = model_ref.phi(params, (j - 120) * g)
    mu = lam0 * ph.sum() * g
    pN = stats.poisson.pmf(np.arange(13), mu)
    pN /= pN.sum()
    Et = (ph * j * g).sum() / ph.sum()
    _check(s["mean_wt"], Et * (pN * np.arange(13) / np.arange(1, 14)).sum(), floor=0.05)
    assert np.all(s["mean_we"] == 0.0) and np.all(s["var_we"] == 0.0)
    # the summary is the mean of the per-step scalar after burn-in
    np.testing.assert_allclose(s["mean_wt"], tr["wt"][:, 500:].mean(1), rtol=1e-12)


def test_component_scalar_prior_only_closed_form(orc):
    """The same with the paper's MCP mixture (Table tbl:mgm): a PE's component e ~ G
    independently of its time (the marked process of Eq. (mcp-pzmu)), so the component scalar
    sum_k e_k / (N + 1) has expectation E[N / (N + 1)] sum_e e G(e)."""
    from tests.test_oracle_mcp_pins import _paper_mixture
    mix = _paper_mixture()
    params = dict(C1, **mix, prior_only=1, sample_t0=0, t0_lo=30.0, t0_hi=30.0, n_cap=16)
    T_lo, T_hi, lam0 = 100, 180, 2.0
    s, _ = orc.run_batch(params, _prior_only_batch(64, 8000, 500, T_lo, T_hi, lam0), orc.MODE_INCREMENTAL,
                         n_threads=8)
    g = params["grid_ns"]
    mu = lam0 * model_ref.phi(params, (np.arange(T_lo, T_hi) - 120) * g).sum() * g
    pN = stats.poisson.pmf(np.arange(17), mu)
    pN /= pN.sum()
    Ee = (np.arange(5) * np.array(mix["mix_G"])).sum()
    _check(s["mean_we"], Ee * (pN * np.arange(17) / np.arange(1, 18)).sum(), floor=0.01)


# ---------------------------------------------------------------- Gelman-Rubin with its upper limit
def test_rhat_invariant_under_units(orc):
    """R and its upper limit do not depend on the units of the scalar: x -> a x + b leaves both
    unchanged (a wrong centring of the covariance term of var(V), or a B taken on another
    scale than W, breaks this)."""
    rng = np.random.default_rng(5)
    for m, n in ((2, 50), (4, 300), (8, 1000)):
        for _ in range(5):
            x = rng.normal(0, 1, (m, n)) * rng.uniform(0.5, 2.0, (m, 1)) + rng.normal(0, 0.3, (m, 1))
            r, u = convergence.gelman_diag(x)
            for a, b in ((3.7, 1e3), (-0.01, -42.0), (1e4, 5e5)):
                r2, u2 = convergence.gelman_diag(a * x + b)
                assert abs(r2 - r) <= 1e-9 * r and abs(u2 - u) <= 1e-9 * u


def test_rhat_exact_when_chains_agree(orc):
    """Chains that are permutations of one sample have equal means (B = 0) and equal
    within-chain variances, so var(V) = 0, the degrees-of-freedom factor is 1 and R = its
    upper limit = sqrt((n - 1) / n)."""
    rng = np.random.default_rng(9)
    base = rng.normal(0, 1, 200)
    x = np.stack([rng.permutation(base) for _ in range(5)])
    r, u = convergence.gelman_diag(x)
    assert abs(r - math.sqrt(199 / 200)) < 1e-12 and abs(u - r) < 1e-12


def test_rhat_chi_square_limit(orc):
    """Chains that are shifted copies of one sample have equal within-chain variances, so W is
    known exactly and the F(m - 1, 2 W^2 m / var(s2)) quantile of the upper limit becomes the
    F(m - 1, inf) = chi2(m - 1) / (m - 1) quantile (scipy's chi2): a tiny perturbation that
    makes var(s2) positive (F with ~1e15 degrees of freedom) gives the same limit."""
    rng = np.random.default_rng(11)
    base = rng.normal(0, 1, 400)
    x = np.stack([base + c for c in (0.0, 0.05, -0.03, 0.02)])
    r, u = convergence.gelman_diag(x)
    xp = x + rng.normal(0, 1e-7, x.shape)
    r2, u2 = convergence.gelman_diag(xp)
    assert u > r and abs(u2 - u) <= 1e-6 * u and abs(r2 - r) <= 1e-6 * r


def test_rhat_limits_and_ordering(orc):
    """Independent chains of one distribution: R and its upper limit near 1; chains apart: both
    above 1.1; the upper limit never below R and growing with the confidence; W = 0 limits."""
    rng = np.random.default_rng(13)
    same = rng.normal(0, 1, (8, 20000))
    r, u = convergence.gelman_diag(same)
    assert abs(r - 1.0) < 0.01 and r <= u < 1.02
    apart = rng.normal(0, 1, (4, 500)) + 2.0 * np.arange(4)[:, None]
    r, u = convergence.gelman_diag(apart)
    assert 1.1 < r < u
    for _ in range(50):
        x = rng.normal(0, 1, (int(rng.integers(2, 9)), int(rng.integers(5, 400)))) + rng.normal(0, 0.2, (1, 1))
        r, u90 = convergence.gelman_diag(x, 0.9)
        _, u95 = convergence.gelman_diag(x, 0.95)
        assert r <= u90 <= u95
    assert convergence.gelman_diag(np.ones((3, 10))) == (1.0, 1.0)
    assert convergence.gelman_diag(np.vstack([np.ones(10), 2 * np.ones(10)])) == (math.inf, math.inf)
