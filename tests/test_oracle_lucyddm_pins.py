"""Pins of the oracle's LucyDDM step (Sec. 2.3, CPU only): Lucy's iterative deconvolution of a
waveform by the SER at the sample times, the initial PEs {tau : q-hat(tau) > 0.1}, the solution
space [t_min - 4 ns, t_max + 4 ns] and t0 = t_min; and chains started from such a state.

Independent sources: the exact flux identity of Lucy's iteration, the monotone rise of the
Poisson likelihood (Lucy's method is an EM algorithm), the same iteration written with numpy's
convolution and correlation, noiseless spike recovery, and the Cholesky (definition) mode."""
import math

import numpy as np
import pytest

from paper_2403_03156_gb300 import workloads
from tests import model_ref

C1 = workloads.CONFIGS["plain_fp64_256x128"]["params"]


def _kernel(params):
    V, R = model_ref.ser_table(params)
    raw = V[::R]
    return raw / raw.sum(), raw.sum(), R


def _noisy(params, taus, qs, n, seed):
    v, S, _ = _kernel(params)
    w = np.zeros(n)
    for tau, q in zip(taus, qs):
        for m in range(len(v)):
            if 0 <= tau + m < n:
                w[tau + m] += q * S * v[m]
    w += np.random.default_rng(seed).normal(0, params["sigma_noise"], n)
    return w.astype(np.float32)


def _lucy_numpy(params, w, n_iter):
    """Lucy's iteration with numpy's full convolution and valid-mode correlation."""
    v, S, _ = _kernel(params)
    d = np.maximum(w.astype(np.float64), 0.0) / S
    n, LV = len(d), len(v)
    q = np.full(n + LV - 1, d.sum() / (n + LV - 1))
    for _ in range(n_iter):
        wr = np.convolve(q, v, mode="full")[LV - 1:LV - 1 + n]   # w^r(t), t = 0 .. n-1
        ratio = np.where(wr > 0, d / np.where(wr > 0, wr, 1.0), 0.0)
        pad = np.concatenate([np.zeros(LV - 1), ratio, np.zeros(LV - 1)])
        q = q * np.correlate(pad, v, mode="valid")                # sum_m ratio(tau + m) v(m)
    return q


def test_lucy_matches_numpy_convolution(orc):
    """The oracle's loops against numpy's convolve / correlate, 60 iterations, noisy
    waveform with three PEs (q-hat for tau = -L_V+1 .. n-1)."""
    w = _noisy(C1, [30, 34, 70], [1.0, 0.7, 1.4], 128, seed=1)
    got = orc.lucyddm(C1, w, n_iter=60)["q"]
    ref = _lucy_numpy(C1, w, 60)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-14)


def test_lucy_flux_identity(orc):
    """sum_tau q-hat^(r+1) = sum_t d(t) exactly (the tau range covers every t's kernel), with
    d = max(w, 0) / S."""
    w = _noisy(C1, [20, 60, 61, 100], [1.2, 0.8, 1.0, 2.0], 160, seed=2)
    _, S, _ = _kernel(C1)
    dsum = np.maximum(w.astype(np.float64), 0).sum() / S
    for it in (1, 7, 300):
        q = orc.lucyddm(C1, w, n_iter=it)["q"]
        assert q.sum() == pytest.approx(dsum, rel=1e-12)
        assert np.all(q >= 0)


def test_lucy_increases_the_poisson_likelihood(orc):
    """Lucy's iteration is an EM algorithm: the Poisson log-likelihood sum_t d log w^r - w^r
    does not decrease from one iteration count to a larger one."""
    w = _noisy(C1, [25, 31, 80], [1.0, 1.3, 0.6], 128, seed=3)
    v, S, _ = _kernel(C1)
    d = np.maximum(w.astype(np.float64), 0) / S
    LV = len(v)
    prev = -np.inf
    for it in (0, 1, 2, 5, 20, 100, 500):
        q = orc.lucyddm(C1, w, n_iter=it)["q"]
        wr = np.convolve(q, v, mode="full")[LV - 1:LV - 1 + len(d)]
        ll = float(np.sum(np.where(d > 0, d * np.log(wr), 0.0) - wr))
        assert ll >= prev - 1e-12, (it, ll, prev)
        prev = ll


def test_noiseless_spikes_give_the_initial_state(orc):
    """Two noiseless PEs on sample times 40 and 55 (charges 1.0, 1.5): after 2000 iterations
    q-hat concentrates on them (the charge of each sits within one sample of it), the
    initial z is their grid indices, T = [t_min - 4, t_max + 4] on the 0.25 ns grid and
    t0 = t_origin + t_min."""
    v, S, R = _kernel(C1)
    n, LV = 128, len(v)
    w = np.zeros(n)
    for tau, q in ((40, 1.0), (55, 1.5)):
        w[tau:tau + LV] += (q * S * v)[:n - tau]
    r = orc.lucyddm(C1, w.astype(np.float32), n_iter=2000, t_origin=100.0)
    q = r["q"]
    at = lambda tau: q[tau + LV - 1]
    assert at(40) > 0.9 and at(55) > 1.3
    assert sum(at(t) for t in (39, 40, 41)) == pytest.approx(1.0, abs=0.02)
    assert sum(at(t) for t in (54, 55, 56)) == pytest.approx(1.5, abs=0.02)
    assert list(r["z"]) == [40 * R, 55 * R]
    g = C1["grid_ns"]
    assert (r["T_lo"], r["T_hi"]) == (math.floor((40 - 4) / g), math.ceil((55 + 4) / g) + 1)
    assert r["t0"] == pytest.approx(140.0)


def test_empty_waveform_gives_no_initial_pe(orc):
    """Noise below the threshold: no initial PE, T = the whole window, t0 = NaN (the paper
    leaves such a waveform out)."""
    w = np.random.default_rng(9).normal(0, 0.01, 96).astype(np.float32)
    r = orc.lucyddm(C1, w, n_iter=2000)
    assert r["n_z"] == 0 and (r["T_lo"], r["T_hi"]) == (0, 96 * 4) and math.isnan(r["t0"])


def _batch_from(w, z, T_lo, T_hi, t0, n_steps, lam=2.0, seed=5):
    n = len(w)
    zi = np.zeros((1, max(len(z), 1)), np.int32)
    zi[0, :len(z)] = z
    return dict(samples=w, offsets=np.array([0, n], np.int32), lambda0=np.array([lam]),
                t_origin_ns=np.zeros(1), T_lo=np.array([T_lo], np.int32), T_hi=np.array([T_hi], np.int32),
                t0_init=np.array([t0]), seed=seed, index_base=0, n_steps=n_steps, burn_in=0,
                z_init=zi, n_init=np.array([len(z)], np.int32))


def test_chain_from_initial_state(orc):
    """A chain started from the LucyDDM state: with no step its log-likelihood is
    log p(w | z_init) by Cholesky (definition) and by successive births (incremental); with
    steps, the two modes take the same decisions."""
    params = dict(C1, t0_lo=20.0, t0_hi=60.0)
    w = _noisy(C1, [30, 34, 70], [1.0, 0.7, 1.4], 128, seed=4)
    r = orc.lucyddm(C1, w, n_iter=2000)
    assert r["n_z"] >= 2
    ref, _, _ = orc.logp_definition(params, w, r["z"])
    for mode in (orc.MODE_INCREMENTAL, orc.MODE_DEFINITION):
        s, _ = orc.run_batch(params, _batch_from(w, r["z"], r["T_lo"], r["T_hi"], r["t0"], 0), mode)
        assert s["logL"][0] == pytest.approx(ref, rel=1e-10)
        assert s["N_final"][0] == r["n_z"]
    b = _batch_from(w, r["z"], r["T_lo"], r["T_hi"], r["t0"], 400)
    s_i, t_i = orc.run_batch(params, b, orc.MODE_INCREMENTAL, trace=True)
    s_d, t_d = orc.run_batch(params, b, orc.MODE_DEFINITION, trace=True)
    assert np.array_equal(t_i["flags"], t_d["flags"]) and np.array_equal(t_i["N"], t_d["N"])
    assert t_i["N"][0, 0] >= r["n_z"] - 1
