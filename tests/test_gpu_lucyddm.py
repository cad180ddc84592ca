"""LucyDDM on the GPU (Sec. 2.3) against the FP64 CPU oracle, and chains started from a
LucyDDM state: the deconvolution q-hat element by element, the initial PEs, solution space and
t0 where the threshold decision is unambiguous, and the chain's first steps in FP64 lockstep."""
import math

import numpy as np
import pytest

from paper_2403_03156_gb300 import fsmp, workloads
from tests import gpu_util

pytestmark = pytest.mark.gpu

THRESH = 0.1
N_ITER = 2000


@pytest.fixture(scope="module")
def lib():
    from paper_2403_03156_gb300 import build
    build.build()
    return fsmp.load()


def _dev(torch, b):
    d = torch.device("cuda", 0)
    out = {"samples": torch.from_numpy(b["samples"]).to(d),
           "offsets": torch.from_numpy(b["offsets"].astype(np.int32)).to(d),
           "lambda0": torch.from_numpy(b["lambda0"]).to(d),
           "t_origin_ns": torch.from_numpy(b["t_origin_ns"]).to(d)}
    return out


def test_lucyddm_matches_oracle(lib, orc):
    """q-hat after 2000 FP32 iterations within 1e-3 of the oracle's FP64 value (relative to the
    waveform's largest q-hat). Every tau where the two sides take different sides of the 0.1
    threshold must have the oracle's q-hat within that tolerance of 0.1 (FP32 decides there);
    on the other waveforms the initial PEs, T and t0 are equal."""
    torch = pytest.importorskip("torch")
    wl = workloads.make_workload("batched_uneven_100k", n_waveforms=160, seed=21)
    b = wl["batch"]
    n_max = int(np.diff(b["offsets"]).max())
    with fsmp.Context(wl["params"], n_max=n_max, kernel=fsmp.KERNEL_PE) as ctx:
        L_V = ctx.info()["L_V"]
        r = ctx.lucyddm(_dev(torch, b), n_iter=N_ITER, thresh=THRESH, z_stride=64, with_q=True)
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in r.items()}
    off = b["offsets"]
    worst, split, n_near = 0.0, 0, 0
    for i in range(len(off) - 1):
        w = b["samples"][off[i]:off[i + 1]]
        o = orc.lucyddm(wl["params"], w, n_iter=N_ITER, thresh=THRESH, t_origin=b["t_origin_ns"][i], z_cap=64)
        assert o["L_V"] == L_V
        qg = g["q"][off[i] + i * (L_V - 1): off[i + 1] + (i + 1) * (L_V - 1)]
        scale = max(o["q"].max(), 1e-6)
        err = np.abs(qg - o["q"]).max() / scale
        worst = max(worst, err)
        assert err < 1e-3, (i, err)
        assert g["status"][i] == 0
        # a waveform can take a threshold decision differently only where the oracle's q-hat lies
        # within the q-hat tolerance of the threshold
        n_near += int(np.any(np.abs(o["q"] - THRESH) <= 1e-3 * scale))
        differ = (qg > THRESH) != (o["q"] > THRESH)
        if differ.any():
            assert np.all(np.abs(o["q"][differ] - THRESH) <= 1e-3 * scale), i
            split += 1
            continue
        assert g["n_init"][i] == o["n_z"]
        assert list(g["z_init"][i, :min(o["n_z"], 64)]) == list(o["z"])
        assert (g["T_lo"][i], g["T_hi"][i]) == (o["T_lo"], o["T_hi"])
        if o["n_z"]:
            assert g["t0_init"][i] == pytest.approx(o["t0"], abs=1e-9)
        else:
            assert math.isnan(g["t0_init"][i])
    # the cap is the number of waveforms that have a tau within the tolerance band of the
    # threshold (taken from the oracle alone), not a fixed count
    assert split <= n_near
    print("LucyDDM: worst relative q-hat error %.2e; %d of %d waveforms with a threshold decision taken "
          "differently in FP32, %d with a tau within the tolerance of the threshold" % (worst, split, len(off) - 1,
                                                                                         n_near))


def _trace_buf(torch, W, n_steps):
    return torch.zeros(W * n_steps * fsmp.TRACE_DTYPE.itemsize, dtype=torch.uint8, device=torch.device("cuda", 0))


@pytest.mark.parametrize("lanes", [32, 16])
def test_chain_from_lucyddm_state_fp64_lockstep(lib, orc, lanes):
    """The oracle's LucyDDM state (z, T, t0) as the initial state of both sides: the GPU's C^-1
    built by successive double-double births and the oracle's Cholesky (definition mode) give
    the same log acceptance ratios to 1e-9 and the same decisions over 500 steps."""
    torch = pytest.importorskip("torch")
    wl = workloads.make_workload("batched_uneven_100k", n_waveforms=48, seed=33, n_steps=500)
    b = dict(wl["batch"])
    W = len(b["offsets"]) - 1
    zs = wl["params"]["n_cap"]
    z = np.zeros((W, zs), np.int32)
    nz = np.zeros(W, np.int32)
    T_lo, T_hi, t0 = np.zeros(W, np.int32), np.zeros(W, np.int32), np.zeros(W)
    for i in range(W):
        w = b["samples"][b["offsets"][i]:b["offsets"][i + 1]]
        o = orc.lucyddm(wl["params"], w, n_iter=N_ITER, thresh=THRESH, t_origin=b["t_origin_ns"][i], z_cap=zs)
        nz[i] = min(o["n_z"], zs)
        z[i, :nz[i]] = o["z"][:nz[i]]
        T_lo[i], T_hi[i], t0[i] = o["T_lo"], o["T_hi"], o["t0"]
    b.update(T_lo=T_lo, T_hi=T_hi, t0_init=t0, z_init=z, n_init=nz, z_stride=zs)
    assert (nz > 0).sum() >= W // 2
    n_max = int(np.diff(b["offsets"]).max())
    dev = _dev(torch, b)
    d = dev["offsets"].device
    for k in ("T_lo", "T_hi", "n_init"):
        dev[k] = torch.from_numpy(b[k]).to(d)
    dev["t0_init"] = torch.from_numpy(t0).to(d)
    dev["z_init"] = torch.from_numpy(z).to(d)
    dev["out"] = torch.zeros(W * fsmp.SUMMARY_DTYPE.itemsize, dtype=torch.uint8, device=d)
    dev["trace"] = _trace_buf(torch, W, 500)
    with fsmp.Context(wl["params"], n_max=n_max, precision=fsmp.FP64, kernel=fsmp.KERNEL_PE, pe_lanes=lanes) as ctx:
        ctx.run_device(dev, n_steps=500, burn_in=0, seed=int(b["seed"]), n_max_hint=n_max)
        torch.cuda.synchronize()
    s_gpu = fsmp.summaries_from_bytes(dev["out"].cpu().numpy())
    t_gpu = np.frombuffer(dev["trace"].cpu().numpy().tobytes(), fsmp.TRACE_DTYPE).reshape(W, 500)
    s_orc, t_orc = orc.run_batch(wl["params"], b, orc.MODE_DEFINITION, n_threads=16, trace=True)
    gpu_util.compare_traces(t_gpu, t_orc)
    for f in ("mean_N", "mean_t0"):
        np.testing.assert_allclose(s_gpu[f], s_orc[f], rtol=1e-12, atol=1e-12)
    for f in ("mean_Q", "logL", "logdet", "mean_wt", "var_wt"):
        np.testing.assert_allclose(s_gpu[f], s_orc[f], rtol=1e-9, atol=1e-9)
    np.testing.assert_array_equal(s_gpu["status"], s_orc["status"])
    # the chains did start from the given PEs
    assert np.all(t_gpu["N"][:, 0] >= nz - 1)


def test_lucyddm_then_fp32_chains(lib):
    """The pipeline on the device: LucyDDM's T, t0 and z feed FP32 chains directly; no chain
    is flagged and each starts from its LucyDDM PEs."""
    torch = pytest.importorskip("torch")
    wl = workloads.make_workload("batched_uneven_100k", n_waveforms=2000, seed=35)
    b = wl["batch"]
    W = len(b["offsets"]) - 1
    n_max = int(np.diff(b["offsets"]).max())
    dev = _dev(torch, b)
    with fsmp.Context(wl["params"], n_max=n_max, precision=fsmp.FP32_REFRESH, kernel=fsmp.KERNEL_PE) as ctx:
        r = ctx.lucyddm(dev, n_iter=N_ITER, thresh=THRESH)
        dev.update(T_lo=r["T_lo"], T_hi=r["T_hi"], t0_init=r["t0_init"], z_init=r["z_init"], n_init=r["n_init"])
        dev["out"] = torch.zeros(W * fsmp.SUMMARY_DTYPE.itemsize, dtype=torch.uint8, device=dev["offsets"].device)
        dev["trace"] = _trace_buf(torch, W, 200)
        ctx.run_device(dev, n_steps=200, burn_in=0, seed=int(b["seed"]), n_max_hint=n_max)
        torch.cuda.synchronize()
        n_init = r["n_init"].cpu().numpy()
    s = fsmp.summaries_from_bytes(dev["out"].cpu().numpy())
    t = np.frombuffer(dev["trace"].cpu().numpy().tobytes(), fsmp.TRACE_DTYPE).reshape(W, 200)
    bad = fsmp.ST_INVALID | fsmp.ST_BADDET | fsmp.ST_NONFINITE | fsmp.ST_DRIFT
    assert not np.any(s["status"] & bad)
    cap = wl["params"]["n_cap"]
    assert np.all(np.abs(t["N"][:, 0] - np.minimum(n_init, cap)) <= 1)
    print("LucyDDM initial N: mean %.2f (truth %.2f)" % (n_init.mean(), wl["truth"]["N"].mean()))


def test_lucyddm_edge_cases(lib, orc):
    """A one-sample window, an all-zero window, a window longer than the launch's bound (flagged
    FSMP_ST_INVALID, nothing else written but T = the whole window) and a noiseless PE: each as
    the oracle gives it (the zero and the long one give no initial PE and t0 = NaN)."""
    torch = pytest.importorskip("torch")
    params = workloads.CONFIGS["plain_fp64_256x128"]["params"]
    V, _ = orc.ser_table(params)
    pulse = np.zeros(96, np.float32)
    pulse[20:20 + 65] = 1.7 * V[::4][:65] / 1.0
    wins = [np.array([0.3], np.float32), np.zeros(64, np.float32), np.zeros(200, np.float32), pulse]
    offs = np.concatenate([[0], np.cumsum([len(w) for w in wins])]).astype(np.int32)
    b = dict(samples=np.concatenate(wins), offsets=offs, lambda0=np.ones(4), t_origin_ns=np.zeros(4))
    with fsmp.Context(params, n_max=256, kernel=fsmp.KERNEL_PE) as ctx:
        r = ctx.lucyddm(_dev(torch, b), n_iter=N_ITER, thresh=THRESH, n_max_hint=128)
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in r.items()}
    assert list(g["status"]) == [0, 0, fsmp.ST_INVALID, 0]
    for i in (0, 1, 3):
        o = orc.lucyddm(params, wins[i], n_iter=N_ITER, thresh=THRESH)
        assert g["n_init"][i] == o["n_z"], i
        assert list(g["z_init"][i, :o["n_z"]]) == list(o["z"]), i
        assert (g["T_lo"][i], g["T_hi"][i]) == (o["T_lo"], o["T_hi"]), i
        assert (math.isnan(g["t0_init"][i]) and math.isnan(o["t0"])) or g["t0_init"][i] == pytest.approx(o["t0"])
    assert g["n_init"][2] == 0 and math.isnan(g["t0_init"][2]) and (g["T_lo"][2], g["T_hi"][2]) == (0, 200 * 4)
    assert g["n_init"][3] >= 1 and g["z_init"][3, 0] in (19 * 4, 20 * 4)
