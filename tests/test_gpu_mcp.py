"""The MCP charge model on the GPU (PE-space kernel) against the FP64 CPU oracle: a PE is
(t, e) with a charge from the paper's five-component Gaussian mixture (Table tbl:mgm),
e+ ~ G is drawn for every birth and update (Eq. (mcp)), and U, Sigma, Lambda carry each PE's
mu_e, sigma_e^2 (Appendix A.2)."""
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


def _wl(n, steps, seed, burn_in=0):
    wl = workloads.make_workload("mcp_uneven_20k", n_waveforms=n, n_steps=steps, seed=seed, burn_in=burn_in)
    n_max = int(np.diff(wl["batch"]["offsets"]).max())
    return wl, max(64, n_max)


@pytest.mark.parametrize("lanes", [32, 16])
def test_mcp_lockstep_fp64(lib, orc, lanes):
    """FP64 mode, identical Philox streams (the component draw included): every log
    acceptance ratio to 1e-9 relative, identical decisions, summaries to 1e-9. The reference
    is the oracle's definition mode (a Cholesky of Sigma(z) per step): on pile-up chains with
    the widest component (r = sigma_eps^2 / sigma_e^2 = 0.008) the oracle's own rank-2 updates
    of Sigma^-1 drift by up to 1e-8 from it, while the kernel's double-double C^-1 stays within
    2e-10."""
    wl, n_max = _wl(96, 600, seed=4)
    b = wl["batch"]
    with fsmp.Context(wl["params"], n_max=n_max, precision=fsmp.FP64, kernel=fsmp.KERNEL_PE, pe_lanes=lanes) as ctx:
        s_gpu, t_gpu = ctx.run(b, record_trace=True)
    s_orc, t_orc = orc.run_batch(wl["params"], b, orc.MODE_DEFINITION, n_threads=16, trace=True)
    gpu_util.compare_traces(t_gpu, t_orc)
    for f in ("mean_N", "var_N", "mean_t0", "var_t0"):
        np.testing.assert_allclose(s_gpu[f], s_orc[f], rtol=1e-12, atol=1e-12)
    for f in ("mean_Q", "var_Q", "logL", "logdet", "lambda_hat", "mean_wt", "var_wt", "mean_we", "var_we"):
        np.testing.assert_allclose(s_gpu[f], s_orc[f], rtol=1e-9, atol=1e-9)
    for f in ("acc", "prop", "acc_t0", "prop_t0", "N_final", "k0_final", "status"):
        np.testing.assert_array_equal(s_gpu[f], s_orc[f])
    # the chains did move PEs between components
    assert s_gpu["acc"][:, 2].sum() > 100


def test_mcp_fp32_matches_oracle(lib, orc):
    """FP32 state with an FP64 refresh every 64 accepts: log acceptance ratios on the lockstep
    prefixes close to the FP64 oracle's, and the mean paired difference GPU - oracle of the
    posterior N, charge, t0 and lambda_FSMP within 3 standard errors over 256 waveforms."""
    wl, n_max = _wl(256, 1200, seed=8, burn_in=240)
    b = wl["batch"]
    with fsmp.Context(wl["params"], n_max=n_max, precision=fsmp.FP32_REFRESH, refresh_every=64,
                      kernel=fsmp.KERNEL_PE) as ctx:
        s_gpu, t_gpu = ctx.run(b, record_trace=True)
    s_orc, t_orc = orc.run_batch(wl["params"], b, orc.MODE_INCREMENTAL, n_threads=16, trace=True)
    bad = fsmp.ST_INVALID | fsmp.ST_BADDET | fsmp.ST_NONFINITE
    assert not np.any(s_gpu["status"] & bad)
    same = (t_gpu["flags"] == t_orc["flags"]) & (t_gpu["N"] == t_orc["N"]) & (t_gpu["k0"] == t_orc["k0"])
    pref = np.where((~same).any(1), (~same).argmax(1), same.shape[1])
    errs = []
    for i, p in enumerate(pref):
        a = np.maximum(np.nan_to_num(t_gpu["la"][i, :p], nan=0.0), gpu_util.LA_FLOOR)
        o = np.maximum(np.nan_to_num(t_orc["la"][i, :p], nan=0.0), gpu_util.LA_FLOOR)
        errs.append(np.abs(a - o) / np.maximum(1.0, np.abs(o)))
    errs = np.concatenate(errs)
    assert np.median(pref) >= 300 and np.quantile(errs, 0.99) < 1e-2, (np.median(pref), np.quantile(errs, 0.99))
    for f in ("mean_N", "mean_Q", "mean_t0", "lambda_hat"):
        d = s_gpu[f] - s_orc[f]
        se = d.std(ddof=1) / math.sqrt(len(d))
        assert abs(d.mean()) <= 3 * se + 1e-9, (f, d.mean(), se)
    assert not np.any(s_gpu["status"] & fsmp.ST_DRIFT)
