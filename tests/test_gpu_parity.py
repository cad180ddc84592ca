"""GPU (C-ABI) against the FP64 CPU oracle, step by step, on identical Philox streams."""
import numpy as np
import pytest

from paper_2403_03156_gb300 import fsmp, workloads
from tests import gpu_util

pytestmark = pytest.mark.gpu

C1 = workloads.CONFIGS["plain_fp64_256x128"]["params"]


@pytest.fixture(scope="module")
def lib():
    from paper_2403_03156_gb300 import build
    build.build()
    return fsmp.load()


def test_tables_match_oracle(lib, orc):
    for name in ("plain_fp64_256x128", "lowocc_bulk_1m", "highpileup_20k_1024"):
        params = workloads.CONFIGS[name]["params"]
        with fsmp.Context(params, n_max=256) as ctx:
            ser, phi, lphi = ctx.tables(-2000, 4001)
            ref, _ = orc.ser_table(params)
            assert len(ser) == len(ref)
            assert np.max(np.abs(ser - ref)) < 1e-13
            g = params["grid_ns"]
            ref_phi = np.array([orc.phi(params, d * g) for d in range(-2000, 2001)])
            # values agree to rounding except where phi underflows (below 1e-300 the two
            # libms may differ by a denormal; log phi < -690 there, a certain reject anyway)
            big = ref_phi > 1e-300
            np.testing.assert_allclose(phi[big], ref_phi[big], rtol=1e-13)
            np.testing.assert_allclose(lphi[big], np.log(ref_phi[big]), rtol=1e-13, atol=1e-13)
            assert np.all(phi[~big] <= 1e-300) and np.all(lphi[~big] < -690)


def test_philox_gpu_matches_cpu_bit_for_bit(lib, orc):
    rng = np.random.default_rng(3)
    n = 1_000_000
    ctrs = np.zeros((n, 4), np.uint64)
    ctrs[:, 0] = np.arange(n, dtype=np.uint64)
    ctrs[:, 1] = rng.integers(0, 2, n).astype(np.uint64)
    ctrs[:, 2] = rng.integers(0, 2**63, n).astype(np.uint64)
    key = [0x243F6A8885A308D3, 77]
    with fsmp.Context(C1, n_max=128) as ctx:
        got = ctx.philox_blocks(key, ctrs)
    assert np.array_equal(got, orc.philox_blocks(key, ctrs))


def _oracle_trace(orc, params, batch, threads=16):
    s, t = orc.run_batch(params, batch, orc.MODE_INCREMENTAL, n_threads=threads, trace=True)
    return s, t


@pytest.mark.parametrize("kernel,lanes", [pytest.param(fsmp.KERNEL_SMEM, 32, id="sigma-smem"),
                                          pytest.param(fsmp.KERNEL_GLOBAL, 32, id="sigma-global"),
                                          pytest.param(fsmp.KERNEL_PE, 32, id="pe"),
                                          pytest.param(fsmp.KERNEL_PE, 16, id="pe16")])
def test_lockstep_fp64_config1(lib, orc, kernel, lanes):
    """Config 1 (256 x 128 samples, lambda 2, 1000 steps): every log acceptance ratio to 1e-9
    relative, identical decisions and summaries (PE kernel: a warp or a half warp per chain)."""
    wl = workloads.make_workload("plain_fp64_256x128")
    b = wl["batch"]
    with fsmp.Context(C1, n_max=128, precision=fsmp.FP64, kernel=kernel, pe_lanes=lanes) as ctx:
        s_gpu, t_gpu = ctx.run(b, record_trace=True)
    s_orc, t_orc = _oracle_trace(orc, C1, b)
    gpu_util.compare_traces(t_gpu, t_orc)
    for f in ("mean_N", "var_N", "mean_t0", "var_t0"):
        np.testing.assert_allclose(s_gpu[f], s_orc[f], rtol=1e-12, atol=1e-12)
    for f in ("mean_Q", "var_Q", "logL", "logdet", "lambda_hat", "mean_wt", "var_wt", "mean_we", "var_we"):
        np.testing.assert_allclose(s_gpu[f], s_orc[f], rtol=1e-9, atol=1e-9)
    for f in ("acc", "prop", "acc_t0", "prop_t0", "N_final", "k0_final", "status"):
        np.testing.assert_array_equal(s_gpu[f], s_orc[f])
    if kernel == fsmp.KERNEL_PE:
        # the roofline's algorithmic bytes: the kernel's own count equals the oracle's count of
        # the same words along the same path (8-byte words)
        np.testing.assert_array_equal(s_gpu["alg_bytes"], 8.0 * s_orc["alg_words"])


def test_gelman_rubin_of_gpu_chains_matches_oracle(lib, orc):
    """Four chains of each of 8 waveforms (distinct RNG streams, t0 started across the prior
    range): R for N and t0 from the GPU summaries equals R from the oracle's (FP64, lockstep)."""
    wl = workloads.make_workload("plain_fp64_256x128", n_waveforms=8, n_steps=1500, burn_in=300, seed=17)
    b = wl["batch"]
    m = 4
    idx = np.repeat(np.arange(8), m)
    rb = workloads.subset(b, idx)
    rb["wf_ids"] = np.arange(len(idx), dtype=np.uint64) + np.uint64(10_000)
    rb["t0_init"] = np.tile(np.linspace(C1["t0_lo"], C1["t0_hi"], m), 8)
    with fsmp.Context(C1, n_max=128, precision=fsmp.FP64) as ctx:
        s_gpu, _ = ctx.run(rb)
    s_orc, _ = orc.run_batch(C1, rb, orc.MODE_INCREMENTAL, n_threads=16)
    for w in range(8):
        g = s_gpu[w * m:(w + 1) * m]
        o = np.zeros(m, fsmp.SUMMARY_DTYPE)
        for f in ("mean_N", "var_N", "mean_t0", "var_t0", "mean_Q", "var_Q", "n_samples"):
            o[f] = s_orc[f][w * m:(w + 1) * m]
        for field in (fsmp.RHAT_N, fsmp.RHAT_T0):
            rg, ro = fsmp.gelman_rubin(g, field), fsmp.gelman_rubin(o, field)
            assert np.isfinite(rg) and abs(rg - ro) <= 1e-9 * max(1.0, ro), (w, field, rg, ro)


def test_lockstep_fp64_pileup_variant(lib, orc):
    """The pile-up variant of the PE-space kernel (n_cap > 192: unrolled gathers, accept pass and
    rebuild) with C^-1 in its global slot from the fifth PE on (pe_tile = 4): 48 uneven-window
    chains, FP64, every log acceptance ratio to 1e-9 against the oracle's definition mode."""
    wl = workloads.make_workload("batched_uneven_100k", n_waveforms=48, n_steps=500, seed=41)
    b = wl["batch"]
    n_max = int(np.diff(b["offsets"]).max())
    params = dict(wl["params"], n_cap=200)
    with fsmp.Context(params, n_max=n_max, precision=fsmp.FP64, kernel=fsmp.KERNEL_PE, pe_tile=4) as ctx:
        s_gpu, t_gpu = ctx.run(b, record_trace=True)
    s_orc, t_orc = orc.run_batch(params, b, orc.MODE_DEFINITION, n_threads=16, trace=True)
    gpu_util.compare_traces(t_gpu, t_orc)
    for f in ("mean_Q", "logL", "logdet", "lambda_hat"):
        np.testing.assert_allclose(s_gpu[f], s_orc[f], rtol=1e-9, atol=1e-9)
    np.testing.assert_array_equal(s_gpu["acc"], s_orc["acc"])
    assert t_gpu["N"].max() >= 20  # the unrolled accept pass ran (4 x 32 entries per pass)


def test_fp32_pileup_variant_statistics(lib, orc):
    """The pile-up variant in FP32 mode (float-float C^-1 in the global slot, the unrolled FP64
    rebuild every 16 accepts): mean paired differences GPU - oracle of the posterior N and
    charge within 3 standard errors over 192 uneven-window waveforms."""
    import math
    wl = workloads.make_workload("batched_uneven_100k", n_waveforms=192, n_steps=1200, seed=43, burn_in=240)
    b = wl["batch"]
    n_max = int(np.diff(b["offsets"]).max())
    params = dict(wl["params"], n_cap=200)
    with fsmp.Context(params, n_max=n_max, precision=fsmp.FP32_REFRESH, refresh_every=16, kernel=fsmp.KERNEL_PE,
                      pe_tile=8) as ctx:
        s_gpu, _ = ctx.run(b)
    s_orc, _ = orc.run_batch(params, b, orc.MODE_INCREMENTAL, n_threads=16)
    for f in ("mean_N", "mean_Q"):
        d = s_gpu[f] - s_orc[f]
        se = d.std(ddof=1) / math.sqrt(len(d))
        assert abs(d.mean()) <= 3 * se + 1e-9, (f, d.mean(), se)
    assert np.all((s_gpu["status"] & (fsmp.ST_DRIFT | fsmp.ST_BADDET | fsmp.ST_NONFINITE | fsmp.ST_INVALID)) == 0)
    assert s_gpu["n_refresh"].sum() > 0


@pytest.mark.parametrize("workload", ["plain_fp64_256x128", "mcp_uneven_20k"])
def test_gelman_diag_of_gpu_chains_matches_oracle(lib, orc, workload):
    """The convergence check as Sec. 3.2 plots it: four chains of each of 8 waveforms (distinct
    RNG streams, t0 started across the prior range, FP64), and for N, t0 and the Wasserstein
    scalars of {t_i} (and, with the MCP mixture, {e_i}) the degrees-of-freedom corrected R with
    its 90 % upper limit from the GPU summaries (fsmp_gelman_diag) equal to the oracle's
    gelman_diag on the oracle's raw per-step samples of the same chains (lockstep)."""
    from oracle import convergence
    burn, steps, m = 300, 1500, 4
    wl = workloads.make_workload(workload, n_waveforms=8, n_steps=steps, burn_in=burn, seed=19)
    params, b = wl["params"], wl["batch"]
    idx = np.repeat(np.arange(8), m)
    rb = workloads.subset(b, idx)
    rb["wf_ids"] = np.arange(len(idx), dtype=np.uint64) + np.uint64(20_000)
    rb["t0_init"] = np.tile(np.linspace(params["t0_lo"], params["t0_hi"], m), 8)
    n_max = max(64, int(np.diff(rb["offsets"]).max()))
    with fsmp.Context(params, n_max=n_max, precision=fsmp.FP64, kernel=fsmp.KERNEL_PE) as ctx:
        s_gpu, _ = ctx.run(rb)
    s_orc, t_orc = orc.run_batch(params, rb, orc.MODE_DEFINITION if params.get("n_mix") else orc.MODE_INCREMENTAL,
                                 n_threads=16, trace=True)
    g = params["grid_ns"]
    raw = {fsmp.RHAT_N: t_orc["N"].astype(float), fsmp.RHAT_T0: rb["t_origin_ns"][:, None] + g * t_orc["k0"],
           fsmp.RHAT_WT: t_orc["wt"]}
    if params.get("n_mix"):
        raw[fsmp.RHAT_WE] = t_orc["we"]
    n_checked = 0
    for w in range(8):
        sl = slice(w * m, (w + 1) * m)
        for field, x in raw.items():
            xs = x[sl, burn:]
            if np.all(xs.var(1) == 0):
                continue
            r, u = fsmp.gelman_diag(s_gpu[sl], field, 0.9)
            r0, u0 = convergence.gelman_diag(xs, 0.9)
            assert np.isfinite(r) and abs(r - r0) <= 1e-7 * r0 and abs(u - u0) <= 1e-7 * u0, (w, field, r, r0, u, u0)
            n_checked += 1
    assert n_checked >= 24
