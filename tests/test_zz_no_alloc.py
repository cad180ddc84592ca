"""fsmp_run_device_noalloc, the entry point for callers that cannot allocate device memory
(it keeps its scratch in a static device array instead of allocating), against the regular
device entry point on the same inputs: two calls in a row must both reproduce it, and so must
calls that alternate between two models (which rebuild the tables held in the array).

This file is named to be collected last, so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest

from paper_2403_03156_gb300 import fsmp, workloads

pytestmark = pytest.mark.gpu

_INT_FIELDS = ("acc", "prop", "acc_t0", "prop_t0", "N_final", "k0_final", "status", "n_refresh")
_FLOAT_FIELDS = ("mean_N", "var_N", "mean_t0", "var_t0", "mean_Q", "var_Q", "logL", "logdet", "alg_bytes",
                 "lambda_hat")


@pytest.fixture(scope="module")
def lib():
    from paper_2403_03156_gb300 import build
    build.build()
    return fsmp.load()


def _device_inputs(torch, batch, dev, with_T=True):
    W = len(batch["offsets"]) - 1
    d = {"samples": torch.from_numpy(batch["samples"]).to(dev),
         "offsets": torch.from_numpy(batch["offsets"].astype(np.int32)).to(dev),
         "lambda0": torch.from_numpy(batch["lambda0"].astype(np.float64)).to(dev),
         "t_origin_ns": torch.from_numpy(batch["t_origin_ns"].astype(np.float64)).to(dev)}
    if with_T and batch.get("T_lo") is not None:
        d["T_lo"] = torch.from_numpy(batch["T_lo"].astype(np.int32)).to(dev)
        d["T_hi"] = torch.from_numpy(batch["T_hi"].astype(np.int32)).to(dev)
    return d, W


def _reference(torch, params, inp, W, b, n_max, dev):
    """Summaries of fsmp_run_device on a context made with the same parameters."""
    out = torch.zeros(W * fsmp.SUMMARY_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    with fsmp.Context(params) as ctx:
        ctx.run_device(dict(inp, out=out), n_steps=b["n_steps"], burn_in=b["burn_in"], seed=b["seed"],
                       n_max_hint=n_max)
        torch.cuda.synchronize(dev)
    return fsmp.summaries_from_bytes(out.cpu().numpy())


def _noalloc(torch, params, inp, W, b, n_max, dev):
    out = torch.full((W * fsmp.SUMMARY_DTYPE.itemsize,), 0xAB, dtype=torch.uint8, device=dev)
    fsmp.run_device_noalloc(params, dict(inp, out=out), n_steps=b["n_steps"], burn_in=b["burn_in"], seed=b["seed"],
                            n_max_hint=n_max)
    torch.cuda.synchronize(dev)
    return fsmp.summaries_from_bytes(out.cpu().numpy())


def _assert_same(got, ref, what):
    for f in _FLOAT_FIELDS:
        np.testing.assert_allclose(got[f], ref[f], rtol=1e-12, atol=0, err_msg="%s field %s" % (what, f))
    for f in _INT_FIELDS:
        np.testing.assert_array_equal(got[f], ref[f], err_msg="%s field %s" % (what, f))


def _uneven_batch():
    wl = workloads.make_workload("batched_uneven_100k", n_waveforms=600, n_steps=400, seed=5, burn_in=100)
    b = wl["batch"]
    b = workloads.subset(b, np.nonzero(np.diff(b["offsets"]) <= 256)[0])
    return wl, b


def test_noalloc_matches_run_device_twice(lib):
    torch = pytest.importorskip("torch")
    wl, b = _uneven_batch()
    n_max = int(np.diff(b["offsets"]).max())
    # the entry point runs the Sigma^-1 kernel with shared-memory state; compare with that form
    params = dict(wl["params"], precision=fsmp.FP32_REFRESH, refresh_every=64, n_cap=64, n_max=n_max,
                  kernel=fsmp.KERNEL_SMEM)
    dev = torch.device("cuda", 0)
    inp, W = _device_inputs(torch, b, dev)
    ref = _reference(torch, params, inp, W, b, n_max, dev)
    assert np.all(ref["status"] & fsmp.ST_INVALID == 0)
    for call in range(2):
        _assert_same(_noalloc(torch, params, inp, W, b, n_max, dev), ref, "call %d" % call)


def test_noalloc_rebuilds_tables_when_the_model_changes(lib):
    """Calls alternating between model A (0.25 ns grid, SER sigma 1.5 / tau 6 ns) and model B
    (0.2 ns grid, a faster SER and a shorter phi support, so that R, the SER length and the phi
    range all change) rebuild the tables in the static array each time: A, B, A each match
    fsmp_run_device of a context made with their own parameters, and the second A reproduces
    the first bit for bit."""
    torch = pytest.importorskip("torch")
    wl, b = _uneven_batch()
    n_max = int(np.diff(b["offsets"]).max())
    pa = dict(wl["params"], precision=fsmp.FP32_REFRESH, refresh_every=32, n_cap=48, n_max=n_max,
              kernel=fsmp.KERNEL_SMEM)
    pb = dict(pa, grid_ns=0.2, ser_sigma=1.0, ser_tau=4.0, phi_support_ns=1024.0, sigma_q=0.4)
    dev = torch.device("cuda", 0)
    # the whole window as the solution space (the workload's T is in units of A's grid)
    inp, W = _device_inputs(torch, b, dev, with_T=False)
    ref_a = _reference(torch, pa, inp, W, b, n_max, dev)
    ref_b = _reference(torch, pb, inp, W, b, n_max, dev)
    assert not np.array_equal(ref_a["acc"], ref_b["acc"])  # the two models give other chains
    got = []
    for params, ref, name in ((pa, ref_a, "A"), (pb, ref_b, "B"), (pa, ref_a, "A again")):
        s = _noalloc(torch, params, inp, W, b, n_max, dev)
        _assert_same(s, ref, name)
        got.append(s)
    assert got[0].tobytes() == got[2].tobytes()


def test_noalloc_rejects_sizes_beyond_its_limits(lib):
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
    with pytest.raises(fsmp.FsmpError, match="checks of fsmp_create"):
        fsmp.run_device_noalloc(dict(params, threads_per_chain=48), dict(inp, out=out), n_steps=10)
