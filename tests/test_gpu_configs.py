"""The GPU (C ABI) against the FP64 CPU oracle at the model settings of the other workloads,
and the forms and paths the lockstep tests of the default workload do not reach:

- the 0.2 ns PE grid (R = 5) with the low-occupancy workload's noise and capacity;
- the high pile-up workload: the SER with the 3 % undershoot term (ser_kind = 1), 1024-sample
  windows, lambda 50-200, sigma_q 0.5, n_cap 384 (the pile-up kernel variant, C^-1 in the
  chain's global slot), in FP64 lockstep and in FP32 mode against the oracle's statistics;
- the plain one-launch-per-chain FP64 form (the baseline of the throughput comparison);
- a CUDA-graph replay of a device batch against its eager run;
- lambda_FSMP of multimodal N histograms computed by the chains' device function.

Every case follows the chain of Sec. 2.4 scored by Eqs. (12)-(18) (Appendix A), on the
simulation settings of Sec. 3."""
import math

import numpy as np
import pytest

from paper_2403_03156_gb300 import fsmp, workloads
from tests import gpu_util

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2403_03156_gb300 import build
    build.build()
    return fsmp.load()


def _device(torch, b, n_steps=None, trace=False, z=None):
    """Device tensors of a host batch (and an output buffer, a trace buffer, an initial z)."""
    d = torch.device("cuda", 0)
    W = len(b["offsets"]) - 1
    t = {"samples": torch.from_numpy(b["samples"]).to(d),
         "offsets": torch.from_numpy(b["offsets"].astype(np.int32)).to(d),
         "lambda0": torch.from_numpy(np.asarray(b["lambda0"], np.float64)).to(d),
         "t_origin_ns": torch.from_numpy(np.asarray(b["t_origin_ns"], np.float64)).to(d),
         "out": torch.zeros(W * fsmp.SUMMARY_DTYPE.itemsize, dtype=torch.uint8, device=d)}
    if b.get("wf_ids") is not None:
        t["wf_ids"] = torch.from_numpy(np.asarray(b["wf_ids"], np.uint64).astype(np.int64)).to(d)
    for k in ("T_lo", "T_hi"):
        if b.get(k) is not None:
            t[k] = torch.from_numpy(np.asarray(b[k], np.int32)).to(d)
    if b.get("t0_init") is not None:
        t["t0_init"] = torch.from_numpy(np.asarray(b["t0_init"], np.float64)).to(d)
    if z is not None:
        t["z_init"] = torch.from_numpy(z[0]).to(d)
        t["n_init"] = torch.from_numpy(z[1]).to(d)
    if trace:
        t["trace"] = torch.zeros(W * int(n_steps) * fsmp.TRACE_DTYPE.itemsize, dtype=torch.uint8, device=d)
    return t


def _results(t, W, n_steps=None):
    s = fsmp.summaries_from_bytes(t["out"].cpu().numpy())
    tr = fsmp.traces_from_bytes(t["trace"].cpu().numpy(), W) if "trace" in t else None
    return s, tr


def _lucy_state(orc, params, b, cap):
    """The oracle's LucyDDM state (Sec. 2.3) of every waveform: T, t0 and the initial z."""
    W = len(b["offsets"]) - 1
    z = np.zeros((W, cap), np.int32)
    nz = np.zeros(W, np.int32)
    T_lo, T_hi, t0 = np.zeros(W, np.int32), np.zeros(W, np.int32), np.zeros(W)
    for i in range(W):
        w = b["samples"][b["offsets"][i]:b["offsets"][i + 1]]
        o = orc.lucyddm(params, w, n_iter=2000, thresh=0.1, t_origin=b["t_origin_ns"][i], z_cap=cap)
        nz[i] = min(o["n_z"], cap)
        z[i, :nz[i]] = o["z"][:nz[i]]
        T_lo[i], T_hi[i], t0[i] = o["T_lo"], o["T_hi"], o["t0"]
    return dict(T_lo=T_lo, T_hi=T_hi, t0_init=t0, z_init=z, n_init=nz, z_stride=cap)


def _assert_summaries(s_gpu, s_orc, lam=True, words=False):
    for f in ("mean_N", "mean_t0"):
        np.testing.assert_allclose(s_gpu[f], s_orc[f], rtol=1e-12, atol=1e-12, err_msg=f)
    # the variances come from the same exact integer sums as E[x^2] - E[x]^2, which cancels by
    # a factor E[x^2] / var (about 2000 for t0 on a 1024-sample window): the two sides' last-bit
    # roundings there show at 1e-12
    for f in ("var_N", "var_t0", "mean_Q", "var_Q", "logL", "logdet", "mean_wt", "var_wt", "mean_we",
              "var_we") + (("lambda_hat",) if lam else ()):
        np.testing.assert_allclose(s_gpu[f], s_orc[f], rtol=1e-9, atol=1e-9, err_msg=f)
    for f in ("acc", "prop", "acc_t0", "prop_t0", "N_final", "k0_final", "status"):
        np.testing.assert_array_equal(s_gpu[f], s_orc[f], err_msg=f)
    if words:  # the PE-space kernel's algorithmic bytes against the oracle's count of its words
        np.testing.assert_array_equal(s_gpu["alg_bytes"], 8.0 * s_orc["alg_words"])


# ------------------------------------------------------------------ 0.2 ns grid (R = 5)
@pytest.mark.parametrize("kernel,lanes", [pytest.param(fsmp.KERNEL_PE, 32, id="pe"),
                                          pytest.param(fsmp.KERNEL_PE, 16, id="pe16"),
                                          pytest.param(fsmp.KERNEL_SMEM, 32, id="sigma-smem")])
def test_lockstep_fp64_lowocc_grid_0p2ns(lib, orc, kernel, lanes):
    """The low-occupancy workload's model (0.2 ns grid, so R = 5 grid points per sample and five
    SER phases; noise 0.08; n_cap 24; lambda 0.05-3): 64 waveforms x 500 steps, every log
    acceptance ratio to 1e-9 and every decision as the oracle's."""
    wl = workloads.make_workload("lowocc_bulk_1m", n_waveforms=64, n_steps=500, seed=51)
    b, params = wl["batch"], wl["params"]
    assert params["grid_ns"] == 0.2
    with fsmp.Context(params, n_max=128, precision=fsmp.FP64, kernel=kernel, pe_lanes=lanes) as ctx:
        assert ctx.info()["R"] == 5
        s_gpu, t_gpu = ctx.run(b, record_trace=True)
    s_orc, t_orc = orc.run_batch(params, b, orc.MODE_INCREMENTAL, n_threads=16, trace=True)
    gpu_util.compare_traces(t_gpu, t_orc)
    _assert_summaries(s_gpu, s_orc, words=kernel == fsmp.KERNEL_PE)
    assert s_gpu["acc"].sum() > 1000 and t_gpu["N"].max() >= 4


# ------------------------------------------------------------------ high pile-up workload
def _pileup(orc, n_waveforms, n_steps, seed, burn_in=0):
    wl = workloads.make_workload("highpileup_20k_1024", n_waveforms=n_waveforms, n_steps=n_steps, seed=seed,
                                 burn_in=burn_in)
    params = wl["params"]
    assert params["ser_kind"] == 1 and params["n_cap"] == 384 and params["grid_ns"] == 0.2
    b = dict(wl["batch"])
    assert np.all(np.diff(b["offsets"]) == 1024)
    b.update(_lucy_state(orc, params, b, params["n_cap"]))
    return wl, params, b


def test_lockstep_fp64_highpileup(lib, orc):
    """The high pile-up workload's model and windows (undershoot SER, 1024 samples, lambda
    50-200, sigma_q 0.5, sigma_eps 0.05, n_cap 384), each chain started from its LucyDDM state
    so that it carries about a hundred PEs from the first step (C^-1 in the chain's global
    slot, the pile-up kernel variant): 4 waveforms x 150 steps, every log acceptance ratio to
    1e-9 against the oracle's definition mode (log p(w|z) by Cholesky of Sigma(z), Eq.
    (mgauss)), with the same decisions."""
    torch = pytest.importorskip("torch")
    n_steps = 150
    wl, params, b = _pileup(orc, 4, n_steps, seed=61)
    assert b["n_init"].min() >= 40
    W = 4
    t = _device(torch, b, n_steps, trace=True, z=(b["z_init"], b["n_init"]))
    with fsmp.Context(params, n_max=1024, precision=fsmp.FP64, kernel=fsmp.KERNEL_PE) as ctx:
        ctx.run_device(t, n_steps=n_steps, burn_in=0, seed=int(b["seed"]), n_max_hint=1024)
        torch.cuda.synchronize()
    s_gpu, t_gpu = _results(t, W)
    s_orc, t_orc = orc.run_batch(params, b, orc.MODE_DEFINITION, n_threads=16, trace=True)
    gpu_util.compare_traces(t_gpu, t_orc)
    _assert_summaries(s_gpu, s_orc, words=True)
    assert t_gpu["N"].max() >= 60 and s_gpu["acc"].sum() >= 100


def test_fp32_highpileup_statistics(lib, orc):
    """FP32 mode on the high pile-up workload with its FP64 refresh every 32 accepts: 256
    waveforms from their LucyDDM states, 400 steps (burn-in 100). The mean paired differences
    GPU - oracle of the posterior N, charge and t0 lie within 3 standard errors, no chain is
    flagged, and the refreshes ran."""
    torch = pytest.importorskip("torch")
    n_steps, burn = 400, 100
    wl, params, b = _pileup(orc, 256, n_steps, seed=63, burn_in=burn)
    W = 256
    t = _device(torch, b, z=(b["z_init"], b["n_init"]))
    with fsmp.Context(params, n_max=1024, precision=fsmp.FP32_REFRESH, refresh_every=32,
                      kernel=fsmp.KERNEL_PE) as ctx:
        ctx.run_device(t, n_steps=n_steps, burn_in=burn, seed=int(b["seed"]), n_max_hint=1024)
        torch.cuda.synchronize()
    s_gpu, _ = _results(t, W)
    s_orc, _ = orc.run_batch(params, b, orc.MODE_INCREMENTAL, n_threads=16)
    for f in ("mean_N", "mean_Q", "mean_t0"):
        d = s_gpu[f] - s_orc[f]
        se = d.std(ddof=1) / math.sqrt(len(d))
        assert abs(d.mean()) <= 3 * se + 1e-9, (f, d.mean(), se)
    bad = fsmp.ST_DRIFT | fsmp.ST_BADDET | fsmp.ST_NONFINITE | fsmp.ST_INVALID
    assert np.all((s_gpu["status"] & bad) == 0)
    assert s_gpu["n_refresh"].min() >= 1 and s_gpu["mean_N"].mean() > 50


def test_fp32_pileup_refresh_tracks_oracle(lib, orc):
    """FP32 mode in the pile-up variant with an FP64 rebuild after every accepted move (K = 1):
    12 of the high pile-up workload's waveforms from their LucyDDM states, 100 steps. Each
    rebuild recomputes C^-1, v, y, log|Sigma| and log L in FP64 from the PE list (the blocked
    sweep with its register-swept diagonal blocks, the residual summed PE by PE), so the chains
    follow the FP64 oracle step by step with log acceptance ratios equal to FP32 rounding, and a
    chain that stays in lockstep to the end reports the log-likelihood and log|Sigma| of its
    final state (Eq. (mgauss), by Cholesky of Sigma in the oracle) to 1e-8: they come from the
    final rebuild."""
    torch = pytest.importorskip("torch")
    n_steps, W = 100, 12
    wl, params, b = _pileup(orc, W, n_steps, seed=65)
    assert b["n_init"].min() >= 30
    t = _device(torch, b, n_steps, trace=True, z=(b["z_init"], b["n_init"]))
    with fsmp.Context(params, n_max=1024, precision=fsmp.FP32_REFRESH, refresh_every=1,
                      kernel=fsmp.KERNEL_PE) as ctx:
        ctx.run_device(t, n_steps=n_steps, burn_in=0, seed=int(b["seed"]), n_max_hint=1024)
        torch.cuda.synchronize()
    s_gpu, t_gpu = _results(t, W)
    s_orc, t_orc = orc.run_batch(params, b, orc.MODE_INCREMENTAL, n_threads=16, trace=True)
    same = (t_gpu["flags"] == t_orc["flags"]) & (t_gpu["N"] == t_orc["N"]) & (t_gpu["k0"] == t_orc["k0"])
    pref = np.where((~same).any(1), (~same).argmax(1), n_steps)
    bad = fsmp.ST_DRIFT | fsmp.ST_BADDET | fsmp.ST_NONFINITE | fsmp.ST_INVALID
    assert np.all((s_gpu["status"] & bad) == 0)
    assert s_gpu["n_refresh"].min() >= 10 and t_gpu["N"].min() >= 30
    full = pref == n_steps
    assert full.sum() >= W // 2, pref
    errs = []
    for i in range(W):
        a = np.maximum(np.nan_to_num(t_gpu["la"][i, :pref[i]], nan=0.0), gpu_util.LA_FLOOR)
        o = np.maximum(np.nan_to_num(t_orc["la"][i, :pref[i]], nan=0.0), gpu_util.LA_FLOOR)
        near = np.abs(o) < 20
        errs.append(np.abs(a - o)[near])
    err = np.concatenate(errs)
    print("|dla| p50 %.2e p99 %.2e max %.2e; lockstep to the end: %d of %d" % (
        *np.percentile(err, [50, 99, 100]), full.sum(), W))
    assert np.percentile(err, 99) < 2e-2 and err.max() < 1.0
    # the reference for the rebuilt log L and log|Sigma|: Eq. (mgauss) by Cholesky of Sigma(z) on
    # the final state. The rebuild inverts C = diag(r) + A^T A in FP64: r = sigma_eps^2 / sigma_q^2
    # = 0.01 bounds its smallest eigenvalue and N |a|^2 (about 600 here) its largest, so kappa(C)
    # reaches ~6e4 and rounding in h^T C^-1 h (~1e3) enters log L amplified by 1 / (2 sigma_eps^2)
    # = 200: 1e-8 of log L (measured worst 1.1e-9) is within that arithmetic, 1e-9 is not always
    for i in np.nonzero(full)[0]:
        one = {k: b[k][i:i + 1] for k in ("lambda0", "t_origin_ns", "T_lo", "T_hi", "t0_init", "n_init")}
        o0, o1 = int(b["offsets"][i]), int(b["offsets"][i + 1])
        one.update(samples=b["samples"][o0:o1], offsets=np.array([0, o1 - o0], np.int32), z_init=b["z_init"][i:i + 1],
                   seed=b["seed"], n_steps=n_steps, burn_in=0, index_base=int(b.get("index_base", 0)) + int(i))
        st = orc.run_chain_state(params, one)
        assert st["N"] == s_gpu["N_final"][i] and st["k0"] == s_gpu["k0_final"][i]
        logp, logdet, _ = orc.logp_definition(params, b["samples"][o0:o1], st["z"])
        np.testing.assert_allclose(s_gpu["logL"][i], logp, rtol=1e-8, atol=1e-8, err_msg=str(i))
        np.testing.assert_allclose(s_gpu["logdet"][i], logdet, rtol=1e-8, atol=1e-8, err_msg=str(i))


# ------------------------------------------------------------------ the plain FP64 form
def test_lockstep_plain_form(lib, orc):
    """The plain one-launch-per-chain FP64 form (full Sigma^-1 in global memory): 32 waveforms
    of the 256 x 128-sample workload x 1000 steps in lockstep with the oracle."""
    wl = workloads.make_workload("plain_fp64_256x128")
    b = workloads.subset(wl["batch"], np.arange(0, 256, 8))
    params = wl["params"]
    with fsmp.Context(params, n_max=128, precision=fsmp.FP64, kernel=fsmp.KERNEL_PLAIN) as ctx:
        launches0 = ctx.info()["n_launches"]
        s_gpu, t_gpu = ctx.run(b, record_trace=True)
        assert ctx.info()["n_launches"] - launches0 == 32  # one launch per chain
    s_orc, t_orc = orc.run_batch(params, b, orc.MODE_INCREMENTAL, n_threads=16, trace=True)
    gpu_util.compare_traces(t_gpu, t_orc)
    _assert_summaries(s_gpu, s_orc, lam=False)


# ------------------------------------------------------------------ CUDA-graph replay
def test_cuda_graph_replay_equals_eager(lib):
    """A device batch captured into a CUDA graph (the chain-counter reset and the persistent
    launch) and replayed twice gives the eager fsmp_run_device summaries byte for byte."""
    torch = pytest.importorskip("torch")
    wl = workloads.make_workload("batched_uneven_100k", n_waveforms=3000, n_steps=300, seed=71, burn_in=60)
    b = wl["batch"]
    W = len(b["offsets"]) - 1
    n_max = int(np.diff(b["offsets"]).max())
    t = _device(torch, b)
    with fsmp.Context(wl["params"], n_max=n_max, precision=fsmp.FP32_REFRESH, kernel=fsmp.KERNEL_PE) as ctx:
        ctx.run_device(t, n_steps=300, burn_in=60, seed=int(b["seed"]), n_max_hint=n_max)
        torch.cuda.synchronize()
        eager = t["out"].cpu().numpy().tobytes()
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream()
        cs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cs):
            with torch.cuda.graph(g, stream=cs):
                ctx.run_device(t, n_steps=300, burn_in=60, seed=int(b["seed"]), n_max_hint=n_max, stream=cs)
        torch.cuda.current_stream().wait_stream(cs)
        for rep in range(2):
            t["out"].fill_(0xCD)
            g.replay()
            torch.cuda.synchronize()
            assert t["out"].cpu().numpy().tobytes() == eager, "replay %d differs from the eager run" % rep
    s = fsmp.summaries_from_bytes(np.frombuffer(eager, np.uint8))
    assert np.all(s["status"] & fsmp.ST_INVALID == 0) and s["acc"].sum() > 0


# ------------------------------------------------------------------ lambda_FSMP on the device
@pytest.mark.parametrize("lanes", [32, 16])
def test_device_lambda_mle_multimodal(lib, orc, lanes):
    """lambda_FSMP (Eq. (reduce-mu0)) by the device function every chain ends with, on N
    histograms of two or three separated clusters whose local maxima of l compete, and on
    unimodal ones: equal to the oracle's global maximiser (itself pinned against an
    independent scan + Brent search) to 1e-9 relative."""
    rng = np.random.default_rng(99)
    hs, l0s = [], []
    for case in range(400):
        n_max = 384 if lanes == 32 else 192
        h = np.zeros(n_max + 1, np.int64)
        n_cl = int(rng.choice([1, 2, 3]))
        centers = np.sort(rng.choice(np.arange(0, n_max - 4), n_cl, replace=False))
        for c in centers:
            for dlt in range(-int(rng.integers(0, 4)), int(rng.integers(1, 4))):
                if 0 <= c + dlt <= n_max:
                    h[c + dlt] += int(rng.integers(1, 400))
        a, bb = int(centers[0]), int(centers[-1])
        if bb > a:
            la = -a + (a * math.log(a) if a > 0 else 0.0) + math.log(h[a])
            lb = -bb + bb * math.log(bb) + math.log(h[bb])
            lam0 = math.exp((lb - la) / (bb - a) + rng.uniform(-0.08, 0.08))
        else:
            lam0 = float(rng.uniform(0.5, 2.0 * max(1, a)))
        hs.append(h)
        l0s.append(lam0)
    H = np.stack(hs)
    with fsmp.Context(workloads.CONFIGS["plain_fp64_256x128"]["params"], n_max=128) as ctx:
        got = ctx.lambda_mle(H, np.array(l0s), lanes=lanes)
    want = np.array([orc.lambda_mle(h.astype(float), l0) for h, l0 in zip(hs, l0s)])
    err = np.abs(got - want) / np.maximum(1.0, want)
    assert err.max() <= 1e-9, (err.max(), int(err.argmax()), got[err.argmax()], want[err.argmax()])
