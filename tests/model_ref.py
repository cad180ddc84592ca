"""Independent restatement of the FSMP model with library routines, used only to pin the
CPU oracle: the SER and phi from scipy's ``exponnorm`` (the ex-Gaussian), the Gaussian
marginal likelihood of Appendix A.1 from ``scipy.stats.multivariate_normal``, and the
grid prior of a PE multiset written out term by term (with the MCP components of
Eq. (mcp-pzmu) when the parameters carry a mixture)."""
from __future__ import annotations

import itertools
import math
from collections import Counter

import numpy as np
from scipy import stats

from paper_2403_03156_gb300 import workloads


def ser_table(params):
    """Peak-normalised SER on the PE grid with the truncation rule: keep grid points up to
    the last one with |V| >= eps (scan over [0, end]), rounded up to whole samples."""
    g, dt = params["grid_ns"], params["dt_sample_ns"]
    R = int(round(dt / g))
    s, tau = params["ser_sigma"], params["ser_tau"]
    end = 8 * s + 50 * tau
    if params.get("ser_kind", 0) == 1:
        end = 2 * end + 8 * params["ser_under_sigma"] + 50 * params["ser_under_tau"]
    m_end = int(math.ceil(end / g)) + 1
    grid = np.arange(m_end + R) * g
    if params.get("ser_kind", 0) == 1:
        v = workloads.pulse_shape(params, grid)
    else:
        v = stats.exponnorm.pdf(grid - 4 * s, tau / s, scale=s)
    v = v / v[:m_end].max()
    last = int(np.nonzero(np.abs(v[:m_end]) >= params["ser_eps"])[0][-1])
    Lt = -(-(last + 1) // R) * R
    return v[:Lt], R


def phi(params, t):
    t = np.asarray(t, np.float64)
    if params.get("phi_kind", 0) == 0:
        v = stats.exponnorm.pdf(t, params["phi_p2"] / params["phi_p1"], scale=params["phi_p1"])
    else:
        t1, t2 = params["phi_p1"], params["phi_p2"]
        tt = np.maximum(t, 0.0)
        v = np.where(t >= 0, (t1 + t2) / t2 ** 2 * (1 - np.exp(-tt / t1)) * np.exp(-tt / t2), 0.0)
    return np.where(np.abs(t) <= params["phi_support_ns"], v, 0.0)


def pe_matrix(V, R, n, js):
    """A[i, w] = V[w R - js[i]] inside the table, else 0 (one row per PE)."""
    w = np.arange(n)
    m = w[None, :] * R - np.asarray(js)[:, None]
    ok = (m >= 0) & (m < len(V))
    return np.where(ok, V[np.clip(m, 0, len(V) - 1)], 0.0)


def charge(params, e):
    """(mu, sigma^2) of a PE of MCP component e (the dynode mu_q, sigma_q without a mixture)."""
    if params.get("n_mix", 0) or params.get("mix_G"):
        return params["mix_mu"][e], params["mix_sigma"][e] ** 2
    return params["mu_q"], params["sigma_q"] ** 2


def loglik(params, V, R, w, js, es=None):
    n = len(w)
    A = pe_matrix(V, R, n, js) if len(js) else np.zeros((0, n))
    es = np.zeros(len(js), int) if es is None else np.asarray(es)
    mus = np.array([charge(params, int(e))[0] for e in es])
    s2s = np.array([charge(params, int(e))[1] for e in es])
    U = (mus[:, None] * A).sum(0) if len(js) else np.zeros(n)
    S = A.T @ (s2s[:, None] * A) + params["sigma_noise"] ** 2 * np.eye(n)
    return stats.multivariate_normal.logpdf(np.asarray(w, np.float64), mean=U, cov=S), U, S


def enumerate_posterior(params, w, T_lo, T_hi, k0_values, lambda0, n_cap, t_origin=0.0):
    """Exact posterior over (t0 on its grid, PE multiset on [T_lo, T_hi)) with at most n_cap
    PEs: mass = p(t0) prod_j (lambda0 phi_j g)^m_j / m_j! p(w | multiset). With an MCP
    mixture the multiset is over (grid point, component) pairs and each PE's factor carries
    G(e) (Eq. (mcp-pzmu)); ``comp`` is then the expected number of PEs per component."""
    V, R = ser_table(params)
    g = params["grid_ns"]
    js = np.arange(T_lo, T_hi)
    nT = len(js)
    G = list(params["mix_G"]) if params.get("mix_G") else [1.0]
    nE = len(G)
    types = [(i, e) for i in range(nT) for e in range(nE)]
    logmass, Ns, occs, comps, t0s = [], [], [], [], []
    for k in range(n_cap + 1):
        for S in itertools.combinations_with_replacement(range(len(types)), k):
            pes = [types[x] for x in S]
            ll, _, _ = loglik(params, V, R, w, js[[i for i, _ in pes]], [e for _, e in pes])
            cnt = Counter(S)
            occ = np.zeros(nT)
            comp = np.zeros(nE)
            for x, m in cnt.items():
                occ[types[x][0]] += m
                comp[types[x][1]] += m
            for k0 in k0_values:
                ph = phi(params, (js - k0) * g)
                lp = 0.0
                for x, m in cnt.items():
                    i, e = types[x]
                    if ph[i] <= 0 or G[e] <= 0:
                        lp = -np.inf
                        break
                    lp += m * math.log(lambda0 * ph[i] * g * G[e]) - math.lgamma(m + 1)
                logmass.append(ll + lp)
                Ns.append(k)
                occs.append(occ)
                comps.append(comp)
                t0s.append(t_origin + k0 * g)
    logmass = np.array(logmass)
    p = np.exp(logmass - logmass.max())
    p /= p.sum()
    Ns = np.array(Ns)
    return dict(pN=np.array([p[Ns == k].sum() for k in range(n_cap + 1)]),
                occ=(p[:, None] * np.array(occs)).sum(0), t0=float((p * np.array(t0s)).sum()),
                EN=float((p * Ns).sum()), comp=(p[:, None] * np.array(comps)).sum(0))
