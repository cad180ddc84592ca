"""fsmp_run_device_noalloc, the entry point for callers that cannot allocate device memory
(it keeps its scratch in a static device array instead of allocating), against the regular
device entry point on the same inputs: two calls in a row must both reproduce it.

This file is named to be collected last, so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest

from paper_2403_03156_gb300 import fsmp, workloads

pytestmark = pytest.mark.gpu


def _device_inputs(torch, batch, dev):
    W = len(batch["offsets"]) - 1
    d = {"samples": torch.from_numpy(batch["samples"]).to(dev),
         "offsets": torch.from_numpy(batch["offsets"].astype(np.int32)).to(dev),
         "lambda0": torch.from_numpy(batch["lambda0"].astype(np.float64)).to(dev),
         "t_origin_ns": torch.from_numpy(batch["t_origin_ns"].astype(np.float64)).to(dev)}
    if batch.get("T_lo") is not None:
        d["T_lo"] = torch.from_numpy(batch["T_lo"].astype(np.int32)).to(dev)
        d["T_hi"] = torch.from_numpy(batch["T_hi"].astype(np.int32)).to(dev)
    return d, W


def test_noalloc_matches_run_device_twice():
    torch = pytest.importorskip("torch")
    from paper_2403_03156_gb300 import build
    build.build()
    wl = workloads.make_workload("batched_uneven_100k", n_waveforms=600, n_steps=400, seed=5, burn_in=100)
    b = wl["batch"]
    keep = np.nonzero(np.diff(b["offsets"]) <= 256)[0]
    b = workloads.subset(b, keep)
    n_max = int(np.diff(b["offsets"]).max())
    # the entry point runs the Sigma^-1 kernel with shared-memory state; compare with that form
    params = dict(wl["params"], precision=fsmp.FP32_REFRESH, refresh_every=64, n_cap=64, n_max=n_max,
                  kernel=fsmp.KERNEL_SMEM)
    dev = torch.device("cuda", 0)
    inp, W = _device_inputs(torch, b, dev)
    nbytes = W * fsmp.SUMMARY_DTYPE.itemsize

    ref_out = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    with fsmp.Context(params) as ctx:
        ctx.run_device(dict(inp, out=ref_out), n_steps=b["n_steps"], burn_in=b["burn_in"], seed=b["seed"],
                       n_max_hint=n_max)
        torch.cuda.synchronize(dev)
    ref = fsmp.summaries_from_bytes(ref_out.cpu().numpy())
    assert np.all(ref["status"] & fsmp.ST_INVALID == 0)

    for call in range(2):
        out = torch.full((nbytes,), 0xAB, dtype=torch.uint8, device=dev)
        fsmp.run_device_noalloc(params, dict(inp, out=out), n_steps=b["n_steps"], burn_in=b["burn_in"],
                                seed=b["seed"], n_max_hint=n_max)
        torch.cuda.synchronize(dev)
        got = fsmp.summaries_from_bytes(out.cpu().numpy())
        for f in ("mean_N", "var_N", "mean_t0", "var_t0", "mean_Q", "var_Q", "logL", "logdet", "alg_bytes",
                  "lambda_hat"):
            np.testing.assert_allclose(got[f], ref[f], rtol=1e-12, atol=0, err_msg="call %d field %s" % (call, f))
        for f in ("acc", "prop", "acc_t0", "prop_t0", "N_final", "k0_final", "status", "n_refresh"):
            np.testing.assert_array_equal(got[f], ref[f], err_msg="call %d field %s" % (call, f))


def test_noalloc_rejects_sizes_beyond_its_limits():
    torch = pytest.importorskip("torch")
    wl = workloads.make_workload("plain_fp64_256x128", n_waveforms=4, n_steps=10)
    b = wl["batch"]
    dev = torch.device("cuda", 0)
    inp, W = _device_inputs(torch, b, dev)
    out = torch.zeros(W * fsmp.SUMMARY_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    params = dict(wl["params"], precision=fsmp.FP32_REFRESH, n_cap=65, n_max=128)
    with pytest.raises(fsmp.FsmpError, match="n_cap exceeds"):
        fsmp.run_device_noalloc(params, dict(inp, out=out), n_steps=10)
    params = dict(wl["params"], precision=fsmp.FP32_REFRESH, n_cap=32, n_max=128)
    with pytest.raises(fsmp.FsmpError, match="window length exceeds"):
        fsmp.run_device_noalloc(params, dict(inp, out=out), n_steps=10, n_max_hint=300)
