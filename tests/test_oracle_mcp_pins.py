"""Pins of the oracle's MCP charge model (CPU only): a PE is (t, e) with charge
N(mu_e, sigma_e^2) drawn with probability G(e) (Eq. (mcp-multi-norm), Sec. 2.1), the jumps
of Eq. (mcp) with the prior of Eq. (mcp-pzmu), and U, Sigma, Lambda redefined per PE
(Appendix A.2).

Independent sources: numerical quadrature of the charge integrals (scipy.integrate), which
does not use the Gaussian-marginal algebra at all; the closed form of a first birth; the
Cholesky (definition) mode against the Woodbury (incremental) mode; brute-force enumeration
of the posterior over (grid point, component) multisets; and prior-only limits.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

from paper_2403_03156_gb300 import workloads
from tests import model_ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")
C1 = workloads.CONFIGS["plain_fp64_256x128"]["params"]
MIX2 = dict(n_mix=2, mix_G=[0.3, 0.7], mix_mu=[1.0, 2.2], mix_sigma=[0.25, 0.6])


def _paper_mixture():
    rows = json.load(open(GOLDEN))["mcp_mixture"]["rows"]
    G = np.array([r[1] for r in rows])
    return dict(n_mix=len(rows), mix_G=list(G / G.sum()), mix_mu=[r[2] for r in rows],
                mix_sigma=[r[3] for r in rows])


def _waveform(params, js, qs, n, seed):
    V, R = model_ref.ser_table(params)
    A = model_ref.pe_matrix(V, R, n, js)
    rng = np.random.default_rng(seed)
    return (np.asarray(qs) @ A + rng.normal(0, params["sigma_noise"], n)).astype(np.float32), V, R


def test_single_pe_marginal_by_quadrature(orc):
    """p(w | one PE of component e) = integral over q of N(q; mu_e, sigma_e^2) prod_i
    N(w_i; q a_i, sigma_eps^2): scipy quadrature against the oracle's Gaussian marginal."""
    params = dict(C1, **_paper_mixture(), sigma_noise=0.15)
    w, V, R = _waveform(params, [60], [3.1], 24, seed=4)
    a = model_ref.pe_matrix(V, R, 24, [60])[0]
    se = params["sigma_noise"]
    wd = w.astype(np.float64)
    for e in range(params["n_mix"]):
        mu, sg = params["mix_mu"][e], params["mix_sigma"][e]

        def integrand(q, shift):
            return math.exp(stats.norm.logpdf(q, mu, sg) + stats.norm.logpdf(wd, q * a, se).sum() - shift)

        shift = stats.norm.logpdf(wd, (a @ wd / (a @ a)) * a, se).sum()  # keeps the integrand O(1)
        val, err = integrate.quad(integrand, mu - 12 * sg, mu + 12 * sg, args=(shift,), epsabs=0, epsrel=1e-12,
                                  limit=400)
        ref = math.log(val) + shift
        got, _, _ = orc.logp_definition(params, w, [60], e=[e])
        assert got == pytest.approx(ref, rel=1e-9, abs=1e-8), e


def test_two_pe_marginal_by_quadrature(orc):
    """Two overlapping PEs of different components: a two-dimensional quadrature of the
    charge integral against the oracle's Gaussian marginal."""
    params = dict(C1, **MIX2, sigma_noise=0.2)
    js, es = [40, 46], [0, 1]
    w, V, R = _waveform(params, js, [1.1, 2.0], 20, seed=7)
    A = model_ref.pe_matrix(V, R, 20, js)
    se = params["sigma_noise"]
    wd = w.astype(np.float64)
    mus = [params["mix_mu"][e] for e in es]
    sgs = [params["mix_sigma"][e] for e in es]
    qhat = np.linalg.lstsq(A.T, wd, rcond=None)[0]
    shift = stats.norm.logpdf(wd, qhat @ A, se).sum()

    def integrand(q1, q0):
        r = wd - q0 * A[0] - q1 * A[1]
        return math.exp(stats.norm.logpdf(q0, mus[0], sgs[0]) + stats.norm.logpdf(q1, mus[1], sgs[1])
                        - 0.5 * (r @ r) / se ** 2 - len(wd) * math.log(se * math.sqrt(2 * math.pi)) - shift)

    val, _ = integrate.dblquad(integrand, mus[0] - 9 * sgs[0], mus[0] + 9 * sgs[0],
                               mus[1] - 9 * sgs[1], mus[1] + 9 * sgs[1], epsabs=0, epsrel=1e-10)
    got, _, _ = orc.logp_definition(params, w, js, e=es)
    assert got == pytest.approx(math.log(val) + shift, rel=1e-8, abs=1e-7)


def test_first_birth_closed_form_per_component(orc):
    """Delta nu of a first birth of component e in closed form,
    1/2 [(a.w/se^2 + mu_e/s_e^2)^2 / (1/s_e^2 + |a|^2/se^2) - mu_e^2/s_e^2 - log(1 + s_e^2 |a|^2/se^2)],
    both oracle modes."""
    params = dict(C1, **_paper_mixture(), sigma_noise=0.12)
    w, V, R = _waveform(params, [130], [4.0], 128, seed=2)
    se2 = params["sigma_noise"] ** 2
    wd = w.astype(np.float64)
    for jp in (3, 130, 300):
        a = model_ref.pe_matrix(V, R, 128, [jp])[0]
        for e in range(params["n_mix"]):
            mu, s2 = params["mix_mu"][e], params["mix_sigma"][e] ** 2
            ref = 0.5 * ((a @ wd / se2 + mu / s2) ** 2 / (1 / s2 + a @ a / se2) - mu * mu / s2
                         - math.log1p(s2 * (a @ a) / se2))
            for mode in (orc.MODE_INCREMENTAL, orc.MODE_DEFINITION):
                d = orc.delta_nu(params, w, [], 0, jp=jp, mode=mode, ep=e)
                assert d == pytest.approx(ref, rel=1e-10, abs=1e-9), (jp, e, mode)


def test_delta_nu_modes_with_components(orc):
    """Eqs. (11)-(18) with Lambda = diag(-s_{e-}^2, s_{e+}^2), lambda = (-mu_{e-}, mu_{e+})
    (Appendix A.2) against the Cholesky difference, including an update that keeps the time
    and changes only the component, and birth / death antisymmetry."""
    params = dict(C1, **_paper_mixture(), sigma_noise=0.12)
    w, _, _ = _waveform(params, [150, 170, 240], [2.0, 4.5, 1.0], 128, seed=3)
    rng = np.random.default_rng(13)
    for trial in range(12):
        N = int(rng.integers(1, 7))
        z = [int(x) for x in rng.integers(100, 400, N)]
        e = [int(x) for x in rng.integers(0, 5, N)]
        jp, ep, k = int(rng.integers(0, 512)), int(rng.integers(0, 5)), int(rng.integers(0, N))
        cases = [(0, 0, jp, ep), (1, k, 0, 0), (2, k, jp, ep), (2, k, z[k], (e[k] + 1) % 5)]
        for kind, kk, jj, ee in cases:
            d_inc = orc.delta_nu(params, w, z, kind, kk, jj, orc.MODE_INCREMENTAL, e=e, ep=ee)
            d_def = orc.delta_nu(params, w, z, kind, kk, jj, orc.MODE_DEFINITION, e=e, ep=ee)
            assert d_inc == pytest.approx(d_def, rel=1e-9, abs=1e-8), (trial, kind)
        d_birth = orc.delta_nu(params, w, z, 0, 0, jp, orc.MODE_DEFINITION, e=e, ep=ep)
        d_death = orc.delta_nu(params, w, z + [jp], 1, N, 0, orc.MODE_INCREMENTAL, e=e + [ep])
        assert d_birth == pytest.approx(-d_death, rel=1e-9, abs=1e-8)
        # same time, same component: no change
        assert abs(orc.delta_nu(params, w, z, 2, k, z[k], orc.MODE_INCREMENTAL, e=e, ep=e[k])) < 1e-9


def test_component_uniform_is_a_third_philox_block(orc):
    """The component draw uses the first output of Philox4x64-10 at counter (step, 2, 0, 0)
    under key (seed, waveform index), mapped to ((x >> 11) + 0.5) 2^-53."""
    seed, wf = 0x1234ABCD, 77
    for step in (0, 1, 999):
        x = orc.philox_blocks([seed, wf], np.array([[step, 2, 0, 0]], np.uint64))[0, 0]
        assert orc.step_uniform_e(seed, wf, step) == ((int(x) >> 11) + 0.5) * 2.0 ** -53


def test_mcp_trace_definition_vs_incremental(orc):
    """An MCP chain (the paper's five-component table) in both oracle modes: identical
    decisions, log acceptance ratios to 1e-9 relative (floor 1), charge summaries to 1e-9."""
    params = dict(C1, **_paper_mixture(), sigma_noise=0.15)
    W, n = 4, 128
    rng = np.random.default_rng(5)
    ws = []
    for i in range(W):
        js = rng.integers(140, 300, rng.integers(1, 5))
        es = rng.choice(5, len(js), p=params["mix_G"])
        qs = rng.normal(np.array(params["mix_mu"])[es], np.array(params["mix_sigma"])[es])
        ws.append(_waveform(params, js, qs, n, seed=100 + i)[0])
    b = dict(samples=np.concatenate(ws), offsets=np.arange(W + 1, dtype=np.int32) * n,
             lambda0=np.full(W, 3.0), t_origin_ns=np.zeros(W), seed=11, index_base=0, n_steps=300, burn_in=0)
    s_inc, t_inc = orc.run_batch(params, b, orc.MODE_INCREMENTAL, trace=True)
    s_def, t_def = orc.run_batch(params, b, orc.MODE_DEFINITION, trace=True)
    assert np.array_equal(t_inc["flags"], t_def["flags"])
    assert np.array_equal(t_inc["N"], t_def["N"])
    la_i, la_d = t_inc["la"], t_def["la"]
    fin = np.isfinite(la_d)
    assert np.array_equal(np.isfinite(la_i), fin)
    assert np.all(np.abs(la_i[fin] - la_d[fin]) <= 1e-9 * np.maximum(1.0, np.abs(la_d[fin])))
    assert np.allclose(s_inc["mean_Q"], s_def["mean_Q"], rtol=1e-9)
    assert np.allclose(s_inc["logL"], s_def["logL"], rtol=1e-10)
    assert s_inc["acc"][:, 2].sum() > 0


TINY = dict(C1, ser_sigma=0.5, ser_tau=1.5, phi_p1=1.0, phi_p2=3.0, sigma_noise=0.3,
            n_cap=4, t0_lo=1.0, t0_hi=1.0, sample_t0=0, **MIX2)


def _check(mean_per_chain, exact, k=4.0, floor=2e-3):
    m = mean_per_chain.mean(0)
    se = mean_per_chain.std(0, ddof=1) / math.sqrt(len(mean_per_chain))
    assert np.all(np.abs(m - exact) <= k * se + floor), (m, exact, se)


def _tiny_batch(w, n_chains, n_steps, burn_in, T_lo, T_hi, lambda0):
    n = len(w)
    return dict(samples=np.tile(w, n_chains), offsets=np.arange(n_chains + 1, dtype=np.int32) * n,
                lambda0=np.full(n_chains, lambda0), t_origin_ns=np.zeros(n_chains),
                T_lo=np.full(n_chains, T_lo, np.int32), T_hi=np.full(n_chains, T_hi, np.int32),
                seed=2025, index_base=0, n_steps=n_steps, burn_in=burn_in, occ_width=T_hi - T_lo, occ_e=2)


@pytest.mark.parametrize("mode", [1, 0])
def test_enumeration_with_components(orc, mode):
    """Brute force over (grid point, component) multisets (N <= 4, |T| = 8, two components,
    t0 fixed) with the prior of Eq. (mcp-pzmu): the chains' N distribution, PE-time marginal
    and expected number of PEs per component. Pins the G(e) factors of Eq. (mcp), the
    component draw and the per-PE Lambda, lambda."""
    params = dict(TINY)
    V, R = model_ref.ser_table(params)
    A = model_ref.pe_matrix(V, R, 8, [12, 14])
    w = (0.9 * A[0] + 2.4 * A[1] + np.random.default_rng(0).normal(0, 0.3, 8)).astype(np.float32)
    lam0, T_lo, T_hi = 1.5, 10, 18
    ex = model_ref.enumerate_posterior(params, w, T_lo, T_hi, [4], lam0, 4)
    b = _tiny_batch(w, 64, 12000, 1000, T_lo, T_hi, lam0)
    s, tr, occ, occ_e = orc.run_batch(params, b, mode, n_threads=8, trace=True)
    assert np.all((s["status"] & ~orc.ST_CAPACITY) == 0)
    Ns = tr["N"][:, 1000:]
    pN = np.stack([(Ns == k).mean(1) for k in range(5)], 1)
    _check(pN, ex["pN"])
    _check(occ, ex["occ"])
    _check(occ_e, ex["comp"])


def test_prior_only_component_marginal(orc):
    """Delta nu := 0: the number of PEs of component e is Poisson(lambda0 Phi_T G(e)) (the
    marked Poisson process of Eq. (mcp-pzmu)), truncated jointly at n_cap -- here far above
    the mean, so E[count_e] = lambda0 Phi_T G(e)."""
    params = dict(C1, **_paper_mixture(), prior_only=1, sample_t0=0, t0_lo=30.0, t0_hi=30.0, n_cap=16)
    T_lo, T_hi, lam0 = 100, 180, 2.0
    n = 64
    b = dict(samples=np.zeros(n * 64, np.float32), offsets=np.arange(65, dtype=np.int32) * n,
             lambda0=np.full(64, lam0), t_origin_ns=np.zeros(64), T_lo=np.full(64, T_lo, np.int32),
             T_hi=np.full(64, T_hi, np.int32), seed=5, index_base=0, n_steps=8000, burn_in=500, occ_e=5)
    s, _, _, occ_e = orc.run_batch(params, b, orc.MODE_INCREMENTAL, n_threads=8)
    g = params["grid_ns"]
    Phi = model_ref.phi(params, (np.arange(T_lo, T_hi) - 120) * g).sum() * g
    _check(occ_e, lam0 * Phi * np.array(params["mix_G"]), floor=5e-3)


def test_noiseless_recovery_of_the_charge(orc):
    """sigma_eps = 1e-4, one PE of charge 3.3 at grid index 40 with the paper's mixture. The
    data fix only the total charge there (one PE, or several whose charges add up, depending
    on the components), so every chain's charge summary
    sum_k (mu_{e_k} + s_{e_k}^2 a_k^T Sigma^-1 y) must recover 3.3. Two PEs one grid step
    apart fit the pulse almost as well and split the charge, so the tolerance is 5e-3."""
    params = dict(C1, **_paper_mixture(), sigma_noise=1e-4, sample_t0=0, t0_lo=5.0, t0_hi=5.0)
    V, R = model_ref.ser_table(params)
    w = (3.3 * model_ref.pe_matrix(V, R, 48, [40])[0]).astype(np.float32)
    b = dict(samples=np.tile(w, 8), offsets=np.arange(9, dtype=np.int32) * 48, lambda0=np.full(8, 1.0),
             t_origin_ns=np.zeros(8), T_lo=np.full(8, 20, np.int32), T_hi=np.full(8, 60, np.int32),
             seed=3, index_base=0, n_steps=4000, burn_in=2000)
    s, _ = orc.run_batch(params, b, orc.MODE_INCREMENTAL, n_threads=8)
    assert np.all(s["N_final"] >= 1) and np.all(s["mean_N"] >= 1.0)
    assert np.allclose(s["mean_Q"], 3.3, atol=5e-3)
