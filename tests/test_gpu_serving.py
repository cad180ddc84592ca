"""The serving loop (fsmp_submit / fsmp_poll): requests that are in flight together share the
GPU, and each request's result is the same as when it runs alone."""
import time

import numpy as np
import pytest

from paper_2403_03156_gb300 import fsmp, workloads

pytestmark = pytest.mark.gpu

FLOAT_FIELDS = ("mean_N", "var_N", "mean_t0", "var_t0", "mean_Q", "var_Q", "logL", "logdet", "drift_max",
                "alg_bytes", "lambda_hat")
INT_FIELDS = ("acc", "prop", "acc_t0", "prop_t0", "N_final", "k0_final", "status", "n_samples", "n_refresh")


@pytest.fixture(scope="module")
def lib():
    from paper_2403_03156_gb300 import build
    build.build()
    return fsmp.load()


def _params(params, **kw):
    return dict(params, precision=fsmp.FP32_REFRESH, refresh_every=64, n_max=512, **kw)


def test_result_same_alone_and_in_the_mix(lib):
    """Twelve events of 1-64 uneven waveforms: run one at a time, then submitted all at once
    under a device-memory budget that holds only part of them (so later requests are admitted
    as earlier ones finish). Every summary must be bit-identical: a chain's arithmetic does not
    depend on what else is on the GPU."""
    params, events = workloads.make_events("serving_20k_eps", n_events=12, seed=21, n_steps=300, burn_in=60)
    sizes = [len(e["offsets"]) - 1 for e in events]
    budget = 4 << 20  # a few requests at a time
    with fsmp.Context(_params(params, device_mem_budget=budget)) as ctx:
        alone = []
        t = time.perf_counter()
        for i, ev in enumerate(events):
            s, _ = ctx.run(ev, request_id=i)
            alone.append(s)
        t_alone = time.perf_counter() - t
        t = time.perf_counter()
        for i, ev in enumerate(events):
            assert ctx.submit(ev, request_id=1000 + i) == fsmp.OK
        got = {}
        while len(got) < len(events):
            for r in ctx.poll(64, 2000):
                got[r["request_id"]] = r
            assert time.perf_counter() - t < 120, "serving loop stalled"
        t_mix = time.perf_counter() - t
    for i in range(len(events)):
        r = got[1000 + i]
        assert r["status"] == fsmp.OK
        s_mix, s_alone = r["summaries"], alone[i]
        assert len(s_mix) == sizes[i]
        for f in FLOAT_FIELDS:
            np.testing.assert_array_equal(s_mix[f], s_alone[f], err_msg="event %d field %s" % (i, f))
        for f in INT_FIELDS:
            np.testing.assert_array_equal(s_mix[f], s_alone[f], err_msg="event %d field %s" % (i, f))
    print("alone %.3f s, in the mix %.3f s (%d events, %d waveforms)" % (t_alone, t_mix, len(events), sum(sizes)))


def test_requests_overlap_on_the_device(lib):
    """Many small requests submitted together finish much sooner than the same requests run
    one after another: they are packed and run concurrently, not queued behind each other."""
    params, events = workloads.make_events("serving_20k_eps", n_events=24, seed=5, n_steps=400)
    with fsmp.Context(_params(params)) as ctx:
        ctx.run(events[0], request_id=0)  # warm-up
        t = time.perf_counter()
        for i, ev in enumerate(events):
            ctx.run(ev, request_id=1 + i)
        t_serial = time.perf_counter() - t
        t = time.perf_counter()
        for i, ev in enumerate(events):
            assert ctx.submit(ev, request_id=100 + i) == fsmp.OK
        n = 0
        lat = []
        while n < len(events):
            rs = ctx.poll(64, 2000)
            n += len(rs)
            lat += [r["latency_s"] for r in rs]
        t_mix = time.perf_counter() - t
    assert t_mix < 0.5 * t_serial, (t_mix, t_serial)
    assert all(0 < x < t_mix + 1 for x in lat)
