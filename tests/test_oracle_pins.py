"""Pins of the FP64 CPU oracle against things other than itself (CPU only).

Each test names the passage of arXiv 2403.03156 it checks and the independent source it
checks it against: numpy's Philox4x64-10, scipy's ex-Gaussian and multivariate normal,
closed forms, brute-force enumeration of the posterior on tiny grids, and prior-only limits.
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


# ---------------------------------------------------------------- RNG (step a2) --
def test_philox_matches_numpy_stream(orc):
    """Philox4x64-10 (Salmon et al. 2011) against numpy's independent implementation.
    numpy increments its 256-bit counter before each block."""
    rng = np.random.default_rng(1)
    for _ in range(4):
        key = [int(x) for x in rng.integers(0, 2**63, 2)]
        c0 = [int(x) for x in rng.integers(1, 2**62, 4)]
        bg = np.random.Philox(key=key, counter=[c0[0] - 1, c0[1], c0[2], c0[3]])
        n = 20000
        ref = bg.random_raw(4 * n).reshape(n, 4)
        ctrs = np.zeros((n, 4), np.uint64)
        ctrs[:, 0] = np.uint64(c0[0]) + np.arange(n, dtype=np.uint64)
        ctrs[:, 1:] = np.array(c0[1:], np.uint64)
        got = orc.philox_blocks(key, ctrs)
        assert np.array_equal(got, ref)


def test_step_uniforms_layout(orc):
    """The 8 uniforms of a step: blocks (step, 0, 0, 0) and (step, 1, 0, 0) under key
    (seed, waveform index), u = ((x >> 11) + 0.5) 2^-53, all inside (0, 1)."""
    seed, wf, step = 12345, 77, 999
    u = orc.step_uniforms(seed, wf, step)
    raw = np.concatenate([orc.philox_blocks([seed, wf], np.array([[step, b, 0, 0]], np.uint64))[0]
                          for b in (0, 1)])
    ref = ((raw >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    assert np.array_equal(u, ref)
    assert np.all((u > 0) & (u < 1))


# ------------------------------------------------------------- tables (step a0) --
@pytest.mark.parametrize("name", ["plain_fp64_256x128", "lowocc_bulk_1m", "highpileup_20k_1024"])
def test_ser_table_matches_scipy(orc, name):
    """SER of Sec. 3 (ex-Gaussian shifted by 4 sigma) on the grid, peak 1, against scipy's
    exponnorm; same support rule on both sides."""
    params = workloads.CONFIGS[name]["params"]
    tab, _ = orc.ser_table(params)
    ref, R = model_ref.ser_table(params)
    assert len(tab) == len(ref) and len(tab) % R == 0
    assert np.max(np.abs(tab - ref)) < 1e-11
    assert abs(tab.max() - 1.0) < 1e-15


def test_ser_support_config1(orc):
    """SER exG(1.5, 6) at g = 0.25: 65 samples of support above 1e-4 of the peak."""
    tab, peak = orc.ser_table(C1)
    assert len(tab) == 65 * 4
    assert abs(tab[-4:]).max() >= 1e-4                      # last kept grid point is in the last sample
    assert all(orc.ser_raw(C1, m * 0.25) / peak < 1e-4 for m in range(260, 300))


def test_ser_raw_is_a_density(orc):
    """The unnormalised SER formula of Sec. 3 is an ex-Gaussian density: integral 1, mean
    4 sigma + tau (paper's SER parameters, golden file)."""
    g = json.load(open(GOLDEN))["ser"]
    prm = dict(C1, ser_sigma=g["sigma_ns"], ser_tau=g["tau_ns"])
    f = lambda t: orc.ser_raw(prm, t)
    area, _ = integrate.quad(f, -60, 400, limit=400, points=[0, 10, 30])
    mean, _ = integrate.quad(lambda t: t * f(t), -60, 400, limit=400, points=[0, 10, 30])
    assert abs(area - 1.0) < 1e-8
    assert abs(mean - (4 * g["sigma_ns"] + g["tau_ns"])) < 1e-6


def test_phi_exgauss_matches_scipy(orc):
    for t in np.linspace(-20, 300, 97):
        assert orc.phi(C1, t) == pytest.approx(float(model_ref.phi(C1, t)), rel=1e-10, abs=1e-300)


def test_phi_ls_normalised_with_closed_form_mean(orc):
    """LS profile of Sec. 3 with the paper's tau1, tau2: integrates to 1 and has mean
    tau1 + tau2 - tau1^2 / (tau1 + tau2)."""
    g = json.load(open(GOLDEN))["phi_ls"]
    t1, t2 = g["tau1_ns"], g["tau2_ns"]
    prm = dict(C1, phi_kind=1, phi_p1=t1, phi_p2=t2)
    area, _ = integrate.quad(lambda t: orc.phi(prm, t), 0, 2000, limit=500)
    mean, _ = integrate.quad(lambda t: t * orc.phi(prm, t), 0, 2000, limit=500)
    assert abs(area - 1.0) < 1e-8
    assert abs(mean - (t1 + t2 - t1 * t1 / (t1 + t2))) < 1e-6
    assert orc.phi(prm, -1.0) == 0.0


def test_golden_mixture_and_J():
    """Table (tbl:mgm) probabilities sum to 1 within the printed rounding; J = 1/4."""
    g = json.load(open(GOLDEN))
    G = [r[1] for r in g["mcp_mixture"]["rows"]]
    assert abs(sum(G) - 1.0) < 1e-3
    assert workloads.CONFIGS["plain_fp64_256x128"]["params"]["jump_J"] == g["jump_J"]["value"]


# ------------------------------------------------- likelihood (Appendix A.1) ------
def _c1_waveform(i=0):
    w = workloads.make_workload("plain_fp64_256x128")
    b = w["batch"]
    return w, b["samples"][b["offsets"][i]:b["offsets"][i + 1]]


def test_logp_definition_matches_scipy(orc):
    """log p(w|z) of Appendix A.1 (Eq. (mgauss) and the log-density below it) against
    scipy's multivariate normal with Sigma(z), U(z) built from scipy's SER."""
    _, w = _c1_waveform(3)
    V, R = model_ref.ser_table(C1)
    rng = np.random.default_rng(5)
    for N in (0, 1, 3, 7):
        js = rng.integers(0, 128 * 4, N)
        lp, ld, q = orc.logp_definition(C1, w, js)
        ref, U, S = model_ref.loglik(C1, V, R, w, js)
        assert lp == pytest.approx(ref, rel=1e-11)
        assert ld == pytest.approx(np.linalg.slogdet(S)[1], rel=1e-11)


def test_birth_from_empty_closed_form(orc):
    """Delta nu of the first birth (Sigma^-1 = I / sigma_eps^2) in closed form:
    1/2 [(a.w/se^2 + mu/sq^2)^2 / (1/sq^2 + |a|^2/se^2) - mu^2/sq^2 - log(1 + sq^2 |a|^2 / se^2)],
    both oracle modes."""
    _, w = _c1_waveform(1)
    V, R = model_ref.ser_table(C1)
    se2, sq2, mu = C1["sigma_noise"] ** 2, C1["sigma_q"] ** 2, C1["mu_q"]
    for jp in (0, 3, 130, 201, 400, 511):
        a = model_ref.pe_matrix(V, R, 128, [jp])[0]
        wd = w.astype(np.float64)
        ref = 0.5 * ((a @ wd / se2 + mu / sq2) ** 2 / (1 / sq2 + a @ a / se2) - mu * mu / sq2
                     - math.log1p(sq2 * (a @ a) / se2))
        for mode in (orc.MODE_INCREMENTAL, orc.MODE_DEFINITION):
            d = orc.delta_nu(C1, w, [], 0, jp=jp, mode=mode)
            assert d == pytest.approx(ref, rel=1e-10, abs=1e-9)


def test_delta_nu_identities_and_modes(orc):
    """Eqs. (11)-(18) (incremental) against Delta nu = log p(w|z') - log p(w|z) by Cholesky
    (definition), birth/death antisymmetry, and a zero update."""
    _, w = _c1_waveform(2)
    rng = np.random.default_rng(11)
    for trial in range(12):
        N = int(rng.integers(1, 8))
        z = [int(x) for x in rng.integers(60, 400, N)]
        jp = int(rng.integers(0, 512))
        k = int(rng.integers(0, N))
        for kind, kk, jj in ((0, 0, jp), (1, k, 0), (2, k, jp)):
            d_inc = orc.delta_nu(C1, w, z, kind, kk, jj, orc.MODE_INCREMENTAL)
            d_def = orc.delta_nu(C1, w, z, kind, kk, jj, orc.MODE_DEFINITION)
            assert d_inc == pytest.approx(d_def, rel=1e-9, abs=1e-8)
        # birth of jp into z, then its death, cancel exactly in exact arithmetic
        d_birth = orc.delta_nu(C1, w, z, 0, 0, jp, orc.MODE_DEFINITION)
        d_death = orc.delta_nu(C1, w, z + [jp], 1, N, 0, orc.MODE_INCREMENTAL)
        assert d_birth == pytest.approx(-d_death, rel=1e-9, abs=1e-8)
        # an update onto its own position leaves the likelihood unchanged
        assert abs(orc.delta_nu(C1, w, z, 2, k, z[k], orc.MODE_INCREMENTAL)) < 1e-9


def test_incremental_state_matches_direct_rebuild(orc):
    """After a 1500-step chain, the Woodbury-updated Sigma^-1 (Eq. (12)), y = w - U(z) and
    log|Sigma| (Eq. (17) accumulated) against a direct rebuild with numpy's inverse and
    slogdet."""
    wl, _ = _c1_waveform()
    b = workloads.subset(wl["batch"], [7])
    b["n_steps"] = 1500
    st = orc.run_chain_state(C1, b, orc.MODE_INCREMENTAL)
    assert st["summary"]["acc"].sum() > 50
    w = b["samples"]
    V, R = model_ref.ser_table(C1)
    _, U, S = model_ref.loglik(C1, V, R, w, st["z"])
    Sinv = np.linalg.inv(S)
    assert np.max(np.abs(st["sinv"] - Sinv)) / np.max(np.abs(Sinv)) < 1e-10
    assert np.max(np.abs(st["y"] - (w.astype(np.float64) - U))) < 1e-10
    assert st["logdet"] == pytest.approx(np.linalg.slogdet(S)[1], rel=1e-10)
    y = w.astype(np.float64) - U
    ref_logL = -0.5 * (128 * math.log(2 * math.pi) + np.linalg.slogdet(S)[1] + y @ np.linalg.solve(S, y))
    assert st["summary"]["logL"] == pytest.approx(ref_logL, rel=1e-10)


def test_trace_definition_vs_incremental(orc):
    """Same Philox streams: the two oracle modes take the same decisions and their log
    acceptance ratios agree to 1e-9 relative (floor 1)."""
    wl = workloads.make_workload("plain_fp64_256x128")
    b = workloads.subset(wl["batch"], range(6))
    b["n_steps"] = 300
    s_inc, t_inc = orc.run_batch(C1, b, orc.MODE_INCREMENTAL, trace=True)
    s_def, t_def = orc.run_batch(C1, b, orc.MODE_DEFINITION, trace=True)
    assert np.array_equal(t_inc["flags"], t_def["flags"])
    assert np.array_equal(t_inc["N"], t_def["N"])
    la_i, la_d = t_inc["la"], t_def["la"]
    fin = np.isfinite(la_d)
    assert np.array_equal(np.isfinite(la_i), fin)
    assert np.all(np.abs(la_i[fin] - la_d[fin]) <= 1e-9 * np.maximum(1.0, np.abs(la_d[fin])))
    assert np.allclose(s_inc["mean_Q"], s_def["mean_Q"], rtol=1e-9)
    assert np.allclose(s_inc["logL"], s_def["logL"], rtol=1e-10)


# ------------------------------------------- stationary distribution (Sec. 2.4) ---
TINY = dict(C1, ser_sigma=0.5, ser_tau=1.5, phi_p1=1.0, phi_p2=3.0, sigma_noise=0.3, sigma_q=0.3,
            n_cap=4, t0_lo=1.0, t0_hi=1.0, sample_t0=0)


def _tiny_waveform(params, seed=0):
    """10 samples with PEs at grid 12 and 14 (t = 3.0, 3.5 ns), charges 1.0 and 0.8."""
    V, R = model_ref.ser_table(params)
    A = model_ref.pe_matrix(V, R, 10, [12, 14])
    rng = np.random.default_rng(seed)
    return (A[0] + 0.8 * A[1] + rng.normal(0, params["sigma_noise"], 10)).astype(np.float32)


def _tiny_batch(w, n_chains, n_steps, burn_in, T_lo, T_hi, lambda0, occ_width):
    n = len(w)
    return dict(samples=np.tile(w, n_chains), offsets=np.arange(n_chains + 1, dtype=np.int32) * n,
                lambda0=np.full(n_chains, lambda0), t_origin_ns=np.zeros(n_chains),
                T_lo=np.full(n_chains, T_lo, np.int32), T_hi=np.full(n_chains, T_hi, np.int32),
                seed=2024, index_base=0, n_steps=n_steps, burn_in=burn_in, occ_width=occ_width)


def _check(mean_per_chain, exact, k=4.0, floor=2e-3):
    m = mean_per_chain.mean(0)
    se = mean_per_chain.std(0, ddof=1) / math.sqrt(len(mean_per_chain))
    assert np.all(np.abs(m - exact) <= k * se + floor), (m, exact, se)


def _chain_pN(trace, burn_in, n_cap):
    Ns = trace["N"][:, burn_in:]
    return np.stack([(Ns == k).mean(1) for k in range(n_cap + 1)], 1)


@pytest.mark.parametrize("mode", [1, 0])
def test_enumeration_fixed_t0(orc, mode):
    """Brute force: the exact posterior over PE multisets (N <= 4, |T| = 12, t0 fixed) against
    64 independent chains. Pins the birth / death / update ratios, the J rules and h."""
    params = dict(TINY)
    w = _tiny_waveform(params)
    lam0, T_lo, T_hi = 1.5, 8, 20
    ex = model_ref.enumerate_posterior(params, w, T_lo, T_hi, [4], lam0, 4)
    b = _tiny_batch(w, 64, 12000, 1000, T_lo, T_hi, lam0, T_hi - T_lo)
    s, tr, occ = orc.run_batch(params, b, mode, n_threads=8, trace=True)
    assert np.all(s["status"] == 0) or np.all((s["status"] & ~orc.ST_CAPACITY) == 0)
    _check(_chain_pN(tr, 1000, 4), ex["pN"])
    _check(occ, ex["occ"])
    _check(s["mean_N"][:, None], np.array([ex["EN"]]))


def test_enumeration_sampled_t0(orc):
    """Brute force with t0 sampled on an 8-point grid (uniform prior, Eq. (t0prior)): N
    distribution, PE-time marginals and E[t0]."""
    params = dict(TINY, sample_t0=1, t0_lo=0.0, t0_hi=1.75)
    w = _tiny_waveform(params, seed=1)
    lam0, T_lo, T_hi = 1.5, 8, 20
    ex = model_ref.enumerate_posterior(params, w, T_lo, T_hi, range(0, 8), lam0, 4)
    b = _tiny_batch(w, 64, 12000, 1000, T_lo, T_hi, lam0, T_hi - T_lo)
    s, tr, occ = orc.run_batch(params, b, orc.MODE_INCREMENTAL, n_threads=8, trace=True)
    _check(_chain_pN(tr, 1000, 4), ex["pN"])
    _check(occ, ex["occ"])
    _check(s["mean_t0"][:, None], np.array([ex["t0"]]), floor=5e-3)


def test_prior_only_poisson_fixed_t0(orc):
    """Delta nu := 0: N ~ Poisson(lambda0 Phi_T) truncated at n_cap and PE positions iid
    proportional to phi on T (Eq. (pzmu) restricted to T)."""
    params = dict(C1, prior_only=1, sample_t0=0, t0_lo=30.0, t0_hi=30.0, n_cap=12)
    T_lo, T_hi, lam0 = 100, 180, 3.0   # t in [25, 45) ns
    w = np.zeros(64, np.float32)
    b = _tiny_batch(w, 64, 8000, 500, T_lo, T_hi, lam0, T_hi - T_lo)
    s, tr, occ = orc.run_batch(params, b, orc.MODE_INCREMENTAL, n_threads=8, trace=True)
    g = params["grid_ns"]
    ph = model_ref.phi(params, (np.arange(T_lo, T_hi) - 120) * g)
    mu = lam0 * ph.sum() * g
    pN = stats.poisson.pmf(np.arange(13), mu)
    pN /= pN.sum()
    _check(_chain_pN(tr, 500, 12), pN)
    EN = (np.arange(13) * pN).sum()
    _check(occ, EN * ph / ph.sum())


def test_prior_only_t0_marginal(orc):
    """Delta nu := 0 with t0 sampled: p(t0) proportional to sum_{k <= n_cap} (lambda0 Phi_T(t0))^k / k!
    (the multiset sum of the grid prior), on a 41-point t0 grid."""
    params = dict(C1, prior_only=1, sample_t0=1, t0_lo=25.0, t0_hi=35.0, n_cap=12)
    T_lo, T_hi, lam0 = 100, 180, 3.0
    w = np.zeros(64, np.float32)
    b = _tiny_batch(w, 64, 8000, 500, T_lo, T_hi, lam0, 0)
    b.pop("occ_width")
    s, _ = orc.run_batch(params, b, orc.MODE_INCREMENTAL, n_threads=8)
    g = params["grid_ns"]
    k0s = np.arange(100, 141)
    Phi = np.array([model_ref.phi(params, (np.arange(T_lo, T_hi) - k0) * g).sum() * g for k0 in k0s])
    logw = np.array([np.log(sum((lam0 * P) ** k / math.factorial(k) for k in range(13))) for P in Phi])
    pt = np.exp(logw - logw.max())
    pt /= pt.sum()
    _check(s["mean_t0"][:, None], np.array([(pt * k0s * g).sum()]), floor=0.02)


def test_noiseless_single_pe_recovery(orc):
    """sigma_eps = 1e-4 (charge spread kept at 0.3), one PE of charge 1 at grid index 40: every
    chain sits at N = 1 on that grid point and the charge summary recovers 1 to 1e-3.
    (With sigma_q -> 0 as well, chains started empty can stall in split-PE modes.)"""
    params = dict(C1, sigma_noise=1e-4, sigma_q=0.3, sample_t0=0, t0_lo=9.0, t0_hi=9.0, n_cap=6)
    V, R = model_ref.ser_table(params)
    w = model_ref.pe_matrix(V, R, 30, [40])[0].astype(np.float32)
    b = _tiny_batch(w, 16, 6000, 3000, 32, 48, 1.0, 16)
    s, tr, occ = orc.run_batch(params, b, orc.MODE_INCREMENTAL, n_threads=8, trace=True)
    assert np.all(s["N_final"] == 1)
    assert np.all((tr["N"][:, 3000:] == 1).mean(1) > 0.99)
    assert np.all(occ[:, 40 - 32] > 0.99)
    assert np.all(np.abs(s["mean_Q"] - 1.0) < 1e-3)


def test_charge_summary_information_form(orc):
    """Charge summary (reading R8) at a fixed state against the Gaussian posterior of the
    charges in information form, (I/sq^2 + A^T A/se^2)^-1 (mu/sq^2 1 + A^T w/se^2), summed."""
    wl = workloads.make_workload("plain_fp64_256x128")
    V, R = model_ref.ser_table(C1)
    for i in (5, 9, 21):
        b = workloads.subset(wl["batch"], [i])
        b.update(n_steps=400, burn_in=399)
        st = orc.run_chain_state(C1, b, orc.MODE_INCREMENTAL)
        z = st["z"]
        A = model_ref.pe_matrix(V, R, 128, z).T if len(z) else np.zeros((128, 0))
        se2, sq2, mu = C1["sigma_noise"] ** 2, C1["sigma_q"] ** 2, C1["mu_q"]
        prec = np.eye(len(z)) / sq2 + A.T @ A / se2
        qpost = np.linalg.solve(prec, mu / sq2 * np.ones(len(z)) + A.T @ b["samples"].astype(np.float64) / se2)
        assert st["summary"]["mean_Q"] == pytest.approx(qpost.sum(), rel=1e-10, abs=1e-10)


# ---------------------------------------------------------------- lambda_FSMP (Eq. (reduce-mu0))
def test_lambda_mle_single_count_is_that_count(orc):
    """All samples at N0: l = -lambda + N0 log lambda + const, maximised at lambda = N0."""
    for n0, lam0 in ((1, 2.0), (7, 3.5), (40, 55.0)):
        h = np.zeros(64)
        h[n0] = 100.0
        assert abs(orc.lambda_mle(h, lam0) - n0) < 1e-9 * max(1, n0)


def test_lambda_mle_two_point_closed_form(orc):
    """h = {0: a, 1: b}: l' = -1 + (b / lam0) / (a + b lam / lam0) = 0 gives
    lambda = 1 - a lam0 / b, or 0 when that is negative."""
    for a, b, lam0 in ((1.0, 3.0, 1.5), (2.0, 5.0, 0.5), (5.0, 1.0, 2.0)):
        h = np.zeros(8)
        h[0], h[1] = a, b
        want = max(0.0, 1.0 - a * lam0 / b)
        assert abs(orc.lambda_mle(h, lam0) - want) < 1e-9


def test_lambda_mle_empty_chain_is_zero(orc):
    h = np.zeros(8)
    h[0] = 10.0
    assert orc.lambda_mle(h, 3.0) == 0.0


def test_chain_summary_lambda_matches_its_own_histogram(orc):
    """The summary's lambda_hat is the MLE of the chain's N samples: recompute it from the
    traced N of the same run (after burn-in)."""
    from paper_2403_03156_gb300 import workloads
    wl = workloads.make_workload("plain_fp64_256x128", n_waveforms=3, n_steps=400, burn_in=100, seed=4)
    s, t = orc.run_batch(wl["params"], wl["batch"], orc.MODE_INCREMENTAL, n_threads=1, trace=True)
    for i in range(3):
        N = t["N"][i, 100:]
        h = np.bincount(N, minlength=wl["params"]["n_cap"] + 1).astype(float)
        assert abs(s["lambda_hat"][i] - orc.lambda_mle(h, wl["batch"]["lambda0"][i])) < 1e-12


def _lambda_loglik_np(h, lambda0, lam):
    """l(lambda) = -lambda + log sum_N h_N (lambda / lambda0)^N (Eq. (reduce-mu0)), by
    scipy's logsumexp; independent of the oracle's C code. lam may be an array (> 0)."""
    from scipy.special import logsumexp
    lam = np.atleast_1d(np.asarray(lam, np.float64))
    k = np.nonzero(h > 0)[0]
    terms = np.log(h[k])[None, :] + k[None, :] * np.log(lam[:, None] / lambda0)
    return -lam + logsumexp(terms, axis=1)


def _lambda_global_max(h, lambda0):
    """Global maximiser of l over [0, inf) found without the oracle: every local maximum of a
    dense evaluation on (0, 2 top + 10], each refined by scipy's bounded Brent search, and the
    boundary lambda = 0 (l(0) = log h_0). Returns (lambda*, l(lambda*), number of interior
    local maxima)."""
    from scipy.optimize import minimize_scalar
    top = int(np.nonzero(h > 0)[0].max())
    grid = np.linspace(0.0, 2.0 * top + 10.0, 60001)[1:]
    ll = _lambda_loglik_np(h, lambda0, grid)
    peaks = [i for i in range(len(grid)) if (i == 0 or ll[i] >= ll[i - 1]) and (i == len(grid) - 1 or ll[i] > ll[i + 1])]
    best = (0.0, math.log(h[0]) if h[0] > 0 else -math.inf)
    for i in peaks:
        lo, hi = grid[max(i - 1, 0)] if i > 0 else 1e-12, grid[min(i + 1, len(grid) - 1)]
        r = minimize_scalar(lambda x: -_lambda_loglik_np(h, lambda0, x)[0], bounds=(lo, hi), method="bounded",
                            options={"xatol": 1e-13 * max(1.0, hi)})
        lv = -float(r.fun)
        if lv > best[1]:
            best = (float(r.x), lv)
    return best[0], best[1], len(peaks)


def test_lambda_mle_multimodal_global_maximum(orc):
    """lambda_FSMP (Eq. (reduce-mu0)) when l has several local maxima: N histograms made of two
    or three well separated clusters (a chain that visits clusters of N far apart), with
    lambda0 chosen so that the clusters' local maxima compete (heights within a few units).
    The oracle must return the GLOBAL maximiser found independently (dense scan + Brent
    refinement of every local maximum, scipy); a method that stopped at a local maximum fails."""
    rng = np.random.default_rng(2024)
    n_multi = n_close = 0
    for case in range(60):
        n_max = int(rng.choice([64, 128, 384]))
        n_cl = int(rng.choice([2, 3]))
        centers = np.sort(rng.choice(np.arange(0, n_max - 4), n_cl, replace=False))
        h = np.zeros(n_max + 1)
        for c in centers:
            width = max(1, int(rng.integers(1, 4)))
            for d in range(-width, width + 1):
                if 0 <= c + d <= n_max:
                    h[c + d] += float(rng.integers(1, 400))
        # lambda0 where the two outermost clusters' single-term heights are equal, moved by a
        # random factor: l_c(lambda) ~ -c + log h_c + c log(c / lambda0) at lambda = c
        a, b = int(centers[0]), int(centers[-1])
        ha, hb = h[a], h[b]
        la = (-a + (a * math.log(a) if a > 0 else 0.0) + math.log(ha))
        lb = (-b + b * math.log(b) + math.log(hb))
        log_l0 = (lb - la) / (b - a) + rng.uniform(-0.08, 0.08)
        lambda0 = math.exp(log_l0)
        want, lwant, npk = _lambda_global_max(h, lambda0)
        got = orc.lambda_mle(h, lambda0)
        lgot = _lambda_loglik_np(h, lambda0, max(got, 1e-300))[0] if got > 0 else (math.log(h[0]) if h[0] > 0 else -math.inf)
        assert lgot >= lwant - 1e-9 * max(1.0, abs(lwant)), (case, got, want, lgot, lwant)
        assert abs(got - want) <= 1e-6 * max(1.0, want), (case, got, want, npk)
        if npk >= 2:
            n_multi += 1
            ll_grid = _lambda_loglik_np(h, lambda0, np.linspace(0.0, 2.0 * n_max + 10.0, 60001)[1:])
            # the runner-up local maximum lies within 3 units of the global one
            second = np.sort(ll_grid[[i for i in range(1, len(ll_grid) - 1)
                                      if ll_grid[i] >= ll_grid[i - 1] and ll_grid[i] > ll_grid[i + 1]]])
            if len(second) >= 2 and second[-1] - second[-2] < 3.0:
                n_close += 1
    assert n_multi >= 30 and n_close >= 15, (n_multi, n_close)
