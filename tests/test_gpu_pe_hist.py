"""PE-time histograms (the posterior mean PE count per grid point, an estimator beside lambda_FSMP
and t0-hat): the FP64 PE-space kernel's counts equal the oracle's, step for step, on identical
Philox streams (integer counts, compared exactly)."""
import numpy as np
import pytest

from paper_2403_03156_gb300 import fsmp, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2403_03156_gb300 import build
    build.build()
    return fsmp.load()


@pytest.mark.parametrize("name", ["plain_fp64_256x128", "batched_uneven_100k"])
def test_pe_hist_matches_oracle(lib, orc, name):
    torch = pytest.importorskip("torch")
    wl = workloads.make_workload(name, n_waveforms=64, n_steps=800, burn_in=200, seed=3)
    b = wl["batch"]
    W = len(b["offsets"]) - 1
    n_max = max(64, int(np.diff(b["offsets"]).max()))
    width = int(n_max * round(wl["params"]["dt_sample_ns"] / wl["params"]["grid_ns"]))
    d = torch.device("cuda", 0)
    dev = {"samples": torch.from_numpy(b["samples"]).to(d),
           "offsets": torch.from_numpy(b["offsets"].astype(np.int32)).to(d),
           "lambda0": torch.from_numpy(b["lambda0"]).to(d),
           "t_origin_ns": torch.from_numpy(b["t_origin_ns"]).to(d),
           "out": torch.zeros(W * fsmp.SUMMARY_DTYPE.itemsize, dtype=torch.uint8, device=d),
           "pe_hist": torch.zeros((W, width), dtype=torch.int32, device=d)}
    for k in ("T_lo", "T_hi"):
        if b.get(k) is not None:
            dev[k] = torch.from_numpy(b[k]).to(d)
    with fsmp.Context(wl["params"], n_max=n_max, precision=fsmp.FP64, kernel=fsmp.KERNEL_PE) as ctx:
        ctx.run_device(dev, n_steps=800, burn_in=200, seed=int(b["seed"]), n_max_hint=n_max)
        torch.cuda.synchronize()
    hist = dev["pe_hist"].cpu().numpy()
    s_gpu = fsmp.summaries_from_bytes(dev["out"].cpu().numpy())
    bb = dict(b, occ_width=width)
    s_orc, _, occ = orc.run_batch(wl["params"], bb, orc.MODE_INCREMENTAL, n_threads=16)
    ns = s_orc["n_samples"][:, None].astype(np.float64)
    np.testing.assert_array_equal(s_gpu["acc"], s_orc["acc"])
    np.testing.assert_array_equal(hist, np.rint(occ * ns).astype(np.int64))
    # the histogram sums to the N samples
    np.testing.assert_allclose(hist.sum(1) / ns[:, 0], s_gpu["mean_N"], rtol=1e-12)
