"""Convergence diagnostics of the FSMP chains on raw samples (numpy / scipy): the Gelman-Rubin
potential scale reduction R with its upper confidence limit, as the paper's convergence check
of Sec. 3.2 uses it on t0, N and the Wasserstein scalars of the PE sequences.

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only ``tests/`` and ``bench.py``'s CPU legs
may import it; the CUDA product path never does.

The statistic follows Gelman and Rubin (1992, Statistical Science 7, 457-472, Sec. 3) with the
degrees-of-freedom correction of Brooks and Gelman (1998, J. Comp. Graph. Stat. 7, 434-455,
Sec. 3.2): for m chains of n samples of one scalar, with chain means xbar_j and within-chain
variances s2_j (n - 1 in the denominator),
  W = mean_j s2_j,   B = n var_j(xbar_j),
  V = (n - 1) / n W + (1 + 1 / m) B / n,
  var(V) = [(n - 1)^2 var(s2) / m + (1 + 1 / m)^2 2 B^2 / (m - 1)
            + 2 (n - 1)(1 + 1 / m) (n / m)(cov(s2, xbar^2) - 2 xbarbar cov(s2, xbar))] / n^2,
  d = 2 V^2 / var(V),
  R = sqrt((d + 3) / (d + 1) [(n - 1) / n + (1 + 1 / m)(B / W) / n]),
and the upper limit replaces B / W by B / W times the F(m - 1, 2 W^2 m / var(s2)) quantile at
(1 + confidence) / 2. The paper plots the "90 % upper confidence limit"; the reading taken is
confidence = 0.9. Sample variances and covariances across chains use m - 1.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import stats


def gelman_diag_from_moments(xbar, s2, n, confidence=0.9):
    """(R, upper limit) from the chains' means xbar[m], within-chain variances s2[m] (n - 1
    denominators) and the common number of samples n. W = 0 gives (1, 1) when the means agree
    and (inf, inf) when they do not."""
    xbar = np.asarray(xbar, np.float64)
    s2 = np.asarray(s2, np.float64)
    m = len(xbar)
    if m < 2 or n < 2:
        raise ValueError("need m >= 2 chains of n >= 2 samples")
    W = float(s2.mean())
    B = float(n * xbar.var(ddof=1))
    if not W > 0.0:
        return (1.0, 1.0) if B == 0.0 else (math.inf, math.inf)
    muhat = float(xbar.mean())
    var_s2 = float(s2.var(ddof=1))
    cov_s2_x2 = float(np.cov(s2, xbar ** 2, ddof=1)[0, 1])
    cov_s2_x = float(np.cov(s2, xbar, ddof=1)[0, 1])
    k = 1.0 + 1.0 / m
    V = (n - 1.0) / n * W + k * B / n
    var_V = ((n - 1.0) ** 2 * var_s2 / m + k ** 2 * 2.0 * B ** 2 / (m - 1.0)
             + 2.0 * (n - 1.0) * k * (n / m) * (cov_s2_x2 - 2.0 * muhat * cov_s2_x)) / n ** 2
    d_adj = 1.0 if not var_V > 0.0 else ((2.0 * V ** 2 / var_V) + 3.0) / ((2.0 * V ** 2 / var_V) + 1.0)
    r_fixed = (n - 1.0) / n
    r_random = k * (B / W) / n
    q = (1.0 + confidence) / 2.0
    if var_s2 > 0.0:
        fq = float(stats.f.ppf(q, m - 1, 2.0 * W ** 2 * m / var_s2))
    else:  # W known exactly: the F(m - 1, inf) quantile is chi2(m - 1) / (m - 1)
        fq = float(stats.chi2.ppf(q, m - 1) / (m - 1))
    return math.sqrt(d_adj * (r_fixed + r_random)), math.sqrt(d_adj * (r_fixed + fq * r_random))


def gelman_diag(x, confidence=0.9):
    """(R, upper limit) of raw chains x[m, n] of one scalar."""
    x = np.asarray(x, np.float64)
    return gelman_diag_from_moments(x.mean(1), x.var(1, ddof=1), x.shape[1], confidence)
