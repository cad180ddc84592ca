"""Seeded synthetic inputs for the FSMP chain: the five workload configurations.

This module only SIMULATES data with the waveform model of Eq. (waveform) (Sec. 1): a
Poisson number of PEs with times t0 + an ex-Gaussian delay, Gaussian charges, the
single-electron response, and white noise. It holds none of the inference arithmetic
(no likelihood, no Woodbury, no acceptance ratios); both the CUDA path and the CPU oracle
consume what it produces. The pulse shape is scipy's ``exponnorm`` (an ex-Gaussian),
shifted by 4 sigma as in the SER formula of Sec. 3 and normalised to peak 1 on the PE grid.

There is no dataset: the paper's simulation (Sec. 3) and the workload list are reproduced
with seeded NumPy PCG64 generators. PE times are snapped to the PE grid so that the
sampler's grid model describes the data exactly.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import stats

# Model parameters shared by the configurations (see each config for its overrides).
_BASE = dict(dt_sample_ns=1.0, grid_ns=0.25, ser_kind=0, ser_sigma=1.5, ser_tau=6.0,
             ser_under_frac=0.0, ser_under_sigma=1.0, ser_under_tau=16.0, ser_eps=1e-4,
             phi_kind=0, phi_p1=1.5, phi_p2=20.0, phi_support_ns=4096.0, mu_q=1.0, sigma_q=0.3,
             sigma_noise=0.06, t0_lo=30.0, t0_hi=40.0, sample_t0=1, jump_J=0.25, n_cap=32)

CONFIGS = {
    # 256 waveforms x 128 samples, lambda = 2, FP64, 1000 steps.
    "plain_fp64_256x128": dict(params=dict(_BASE), n_waveforms=256, window=128,
                               lam=("fixed", 2.0), n_steps=1000, precision="fp64"),
    # 100k waveforms, lambda log-uniform 0.5-50, windows 64-512 trimmed to the PE span.
    "batched_uneven_100k": dict(params=dict(_BASE, n_cap=128), n_waveforms=100_000,
                                window="trimmed", win_min=64, win_max=512,
                                lam=("loguniform", 0.5, 50.0), n_steps=2000,
                                precision="fp32", refresh_every=64),
    # 1M waveforms x 128 samples, lambda uniform 0.05-3, noise 0.08, 0.2 ns grid.
    "lowocc_bulk_1m": dict(params=dict(_BASE, grid_ns=0.2, sigma_noise=0.08, n_cap=24),
                           n_waveforms=1_000_000, window=128, lam=("uniform", 0.05, 3.0),
                           n_steps=1000, precision="fp32", refresh_every=64),
    # Serving: events of 1-64 waveforms of 64-512 samples, per-event lambda 0.5-100.
    "serving_20k_eps": dict(params=dict(_BASE, n_cap=192), n_waveforms=None, window="uniform",
                            win_min=64, win_max=512, lam=("loguniform", 0.5, 100.0),
                            n_steps=1500, precision="fp32", refresh_every=64,
                            rate_hz=20000.0, duration_s=60.0, wf_per_event=(1, 64)),
    # MCP-PMT charge model: 20k waveforms like batched_uneven_100k, charges from the paper's
    # five-component Gaussian mixture (Table tbl:mgm, pC). The waveform unit is the SER peak
    # per pC, and sigma_noise = 0.18 keeps the dynode configurations' single-PE SNR (mean
    # charge 2.95 pC / 0.18 ~ 1 / 0.06).
    "mcp_uneven_20k": dict(params=dict(_BASE, n_cap=128, sigma_noise=0.18, n_mix=5,
                                       mix_G=[0.041, 0.516, 0.187, 0.195, 0.061],
                                       mix_mu=[0.92, 1.98, 3.01, 4.70, 6.79],
                                       mix_sigma=[0.22, 0.48, 0.80, 1.30, 2.04]),
                           n_waveforms=20_000, window="trimmed", win_min=64, win_max=512,
                           lam=("loguniform", 0.5, 50.0), n_steps=2000,
                           precision="fp32", refresh_every=64),
    # 20k waveforms x 1024 samples, lambda 50-200, faster SER with a 3% undershoot.
    "highpileup_20k_1024": dict(params=dict(_BASE, grid_ns=0.2, ser_kind=1, ser_sigma=1.0,
                                            ser_tau=4.0, ser_under_frac=0.03,
                                            ser_under_sigma=1.0, ser_under_tau=16.0,
                                            sigma_q=0.5, sigma_noise=0.05, n_cap=384),
                                n_waveforms=20_000, window=1024, lam=("uniform", 50.0, 200.0),
                                n_steps=4000, precision="fp32", refresh_every=32),
}


def _exgauss_shape(t, sigma, tau):
    """Ex-Gaussian density shifted by 4 sigma (scipy's exponnorm), 0 for t < 0."""
    t = np.asarray(t, np.float64)
    v = stats.exponnorm.pdf(t - 4.0 * sigma, tau / sigma, loc=0.0, scale=sigma)
    return np.where(t >= 0.0, v, 0.0)


def pulse_shape(params, t):
    """Peak-normalised single-electron response used to simulate waveforms."""
    g = params["grid_ns"]
    s, tau = params["ser_sigma"], params["ser_tau"]
    grid = np.arange(0.0, 8 * s + 50 * tau, g)
    main = _exgauss_shape(grid, s, tau)
    if params.get("ser_kind", 0) == 1:
        su, tu = params["ser_under_sigma"], params["ser_under_tau"]
        t_pk = grid[int(np.argmax(main))]
        under_grid = _exgauss_shape(grid, su, tu)

        def shape(x):
            return (_exgauss_shape(x, s, tau) / main.max()
                    - params["ser_under_frac"] * _exgauss_shape(x - t_pk, su, tu) / under_grid.max())

        peak = shape(np.arange(0.0, 2 * (8 * s + 50 * tau) + 8 * su + 50 * tu, g)).max()
        return shape(t) / peak
    return _exgauss_shape(t, s, tau) / main.max()


def pulse_support_samples(params, eps=None):
    """Samples after a PE during which the pulse stays above eps * peak."""
    eps = params.get("ser_eps", 1e-4) if eps is None else eps
    g = params["grid_ns"]
    grid = np.arange(0.0, 16 * params["ser_sigma"] + 100 * params["ser_tau"] + 200.0, g)
    v = np.abs(pulse_shape(params, grid))
    last = int(np.nonzero(v >= eps)[0][-1])
    return int(math.ceil((last + 1) * g / params["dt_sample_ns"]))


def _draw_lambda(rng, spec, size):
    kind = spec[0]
    if kind == "fixed":
        return np.full(size, float(spec[1]))
    if kind == "uniform":
        return rng.uniform(spec[1], spec[2], size)
    if kind == "loguniform":
        return np.exp(rng.uniform(math.log(spec[1]), math.log(spec[2]), size))
    raise ValueError(kind)


def simulate(params, lam, t0, rng, window_rule, win_min=64, win_max=512, fixed_window=128):
    """Simulate len(lam) waveforms. Returns a dict of batch arrays plus the truth.

    window_rule "fixed": every window starts at t = 0 and has ``fixed_window`` samples, and
    the PE solution space is the whole window. "trimmed": the window is
    [floor(t_first) - 4, ceil(t_last) + 4 + L_V] ns clamped to [win_min, win_max] samples and
    the solution space is the true PE span +- 4 ns (the span the paper's deconvolution
    step would supply, Sec. 2.3). "uniform": window length ~ U{win_min..win_max} starting
    4 ns before the first PE; solution space = whole window.
    """
    g, dt = params["grid_ns"], params["dt_sample_ns"]
    R = int(round(dt / g))
    W = len(lam)
    L_V = pulse_support_samples(params)
    Ns = rng.poisson(lam)
    tot = int(Ns.sum())
    delays = rng.normal(0.0, params["phi_p1"], tot) + rng.exponential(params["phi_p2"], tot)
    owner = np.repeat(np.arange(W), Ns)
    t_pe = np.repeat(t0, Ns) + delays
    j_abs = np.rint(t_pe / g).astype(np.int64)           # absolute grid index (t = j g)
    if params.get("mix_G"):  # MCP mixture: component e ~ G, then its Gaussian charge
        comp = rng.choice(len(params["mix_G"]), tot, p=np.asarray(params["mix_G"]) / np.sum(params["mix_G"]))
        q = rng.normal(np.asarray(params["mix_mu"])[comp], np.asarray(params["mix_sigma"])[comp])
    else:
        q = rng.normal(params["mu_q"], params["sigma_q"], tot)
    first = np.full(W, np.inf)
    last = np.full(W, -np.inf)
    np.minimum.at(first, owner, j_abs * g)
    np.maximum.at(last, owner, j_abs * g)
    if window_rule == "fixed":
        start = np.zeros(W, np.int64)
        length = np.full(W, fixed_window, np.int64)
    elif window_rule == "trimmed":
        has = Ns > 0
        start = np.where(has, np.floor(np.where(has, first, 0.0)) - 4, np.floor(t0) - 4).astype(np.int64)
        end = np.where(has, np.ceil(np.where(has, last, 0.0)) + 4 + L_V, start + win_min)
        length = np.clip(end - start, win_min, win_max).astype(np.int64)
    elif window_rule == "uniform":
        has = Ns > 0
        start = np.where(has, np.floor(np.where(has, first, 0.0)) - 4, np.floor(t0) - 4).astype(np.int64)
        length = rng.integers(win_min, win_max + 1, W).astype(np.int64)
    else:
        raise ValueError(window_rule)
    offsets = np.zeros(W + 1, np.int64)
    offsets[1:] = np.cumsum(length)
    samples = rng.normal(0.0, params["sigma_noise"], int(offsets[-1]))
    # add the pulses: PE k covers samples s with (s*R - j_rel) in [0, L_V*R + R)
    t_origin = start.astype(np.float64) * dt
    j_rel = j_abs - np.repeat(start * R, Ns)
    span = L_V + 2
    # pulse values at every grid offset a PE can have from a sample
    shape_tab = pulse_shape(params, np.arange((span + 1) * R) * g)
    s0 = np.maximum(0, -(-j_rel // R))                   # first sample at or after each PE
    phase = s0 * R - j_rel                                # grid offset of that sample
    base_idx = offsets[owner] + s0
    n_left = length[owner] - s0                           # samples left in the window
    for m in range(span):                                 # m-th sample after each PE
        live = n_left > m
        np.add.at(samples, base_idx[live] + m, q[live] * shape_tab[phase[live] + m * R])
    out = dict(samples=samples.astype(np.float32), offsets=offsets.astype(np.int32),
               lambda0=np.asarray(lam, np.float64), t_origin_ns=t_origin)
    if window_rule == "trimmed":
        has = Ns > 0
        T_lo = np.where(has, np.floor((np.where(has, first, 0.0) - 4.0 - t_origin) / g), 0)
        T_hi = np.where(has, np.ceil((np.where(has, last, 0.0) + 4.0 - t_origin) / g) + 1, length * R)
        T_hi = np.minimum(T_hi, length * R)
        out["T_lo"] = T_lo.astype(np.int32)
        out["T_hi"] = np.maximum(T_hi, T_lo + 1).astype(np.int32)
    truth = dict(N=Ns, t0=np.asarray(t0, np.float64), owner=owner, t_pe=j_abs * g, q=q)
    return out, truth


def make_workload(name, n_waveforms=None, seed=0, n_steps=None, burn_in=0):
    """Build the named configuration (optionally with fewer waveforms or steps).

    Returns dict(name, params, batch, truth, meta). ``batch`` carries the arrays of the
    C-ABI batch (samples, offsets, lambda0, t_origin_ns, optional T_lo/T_hi) plus seed,
    n_steps and burn_in.
    """
    cfg = CONFIGS[name]
    params = dict(cfg["params"])
    rng = np.random.Generator(np.random.PCG64(seed))
    W = int(n_waveforms if n_waveforms is not None else cfg["n_waveforms"])
    lam = _draw_lambda(rng, cfg["lam"], W)
    t0 = rng.uniform(params["t0_lo"], params["t0_hi"], W)
    if cfg["window"] == "trimmed":
        batch, truth = simulate(params, lam, t0, rng, "trimmed", cfg["win_min"], cfg["win_max"])
    elif cfg["window"] == "uniform":
        batch, truth = simulate(params, lam, t0, rng, "uniform", cfg["win_min"], cfg["win_max"])
    else:
        batch, truth = simulate(params, lam, t0, rng, "fixed", fixed_window=cfg["window"])
    batch.update(seed=seed, index_base=0, n_steps=int(n_steps or cfg["n_steps"]), burn_in=int(burn_in))
    meta = dict(precision=cfg["precision"], refresh_every=cfg.get("refresh_every", 0))
    return dict(name=name, params=params, batch=batch, truth=truth, meta=meta)


def make_events(name, n_events, seed=0, n_steps=None, burn_in=0):
    """Events of the serving configuration: each event is one physics event seen by U{1..64}
    channels (waveforms) that share the event's lambda (log-uniform, per event) and t0; each
    channel draws its own PEs, charges and noise, and its own window length U{64..512}.
    Returns (params, events) with each event a batch dict whose ``index_base`` gives its
    waveforms distinct RNG indices across the list."""
    cfg = CONFIGS[name]
    params = dict(cfg["params"])
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = cfg["wf_per_event"]
    events, base = [], 0
    for e in range(n_events):
        nw = int(rng.integers(lo, hi + 1))
        lam = float(_draw_lambda(rng, cfg["lam"], 1)[0])
        t0 = float(rng.uniform(params["t0_lo"], params["t0_hi"]))
        batch, _ = simulate(params, np.full(nw, lam), np.full(nw, t0), rng, cfg["window"],
                            cfg["win_min"], cfg["win_max"])
        batch.update(seed=seed, index_base=base, n_steps=int(n_steps or cfg["n_steps"]), burn_in=int(burn_in))
        base += nw
        events.append(batch)
    return params, events


def subset(batch, idx):
    """Batch restricted to the waveforms ``idx`` (keeps each waveform's RNG index)."""
    idx = np.asarray(idx, np.int64)
    off = batch["offsets"].astype(np.int64)
    lens = off[idx + 1] - off[idx]
    new_off = np.zeros(len(idx) + 1, np.int64)
    new_off[1:] = np.cumsum(lens)
    samples = np.concatenate([batch["samples"][off[i]:off[i + 1]] for i in idx]) if len(idx) else np.zeros(0, np.float32)
    out = dict(batch)
    ids = batch.get("wf_ids")
    ids = (np.asarray(ids, np.uint64)[idx] if ids is not None
           else np.uint64(batch.get("index_base", 0)) + idx.astype(np.uint64))
    out.update(samples=samples.astype(np.float32), offsets=new_off.astype(np.int32),
               lambda0=batch["lambda0"][idx], t_origin_ns=batch["t_origin_ns"][idx], wf_ids=ids)
    for k in ("T_lo", "T_hi", "t0_init"):
        if batch.get(k) is not None:
            out[k] = batch[k][idx]
    return out
