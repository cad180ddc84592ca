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
    return dict(dict(params, precision=fsmp.FP32_REFRESH, refresh_every=64, n_max=512), **kw)


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


# ---------------------------------------------------------------- error paths of the serving ABI
def _drain(ctx, n, timeout_s=120.0):
    got, t = [], time.perf_counter()
    while len(got) < n:
        got += ctx.poll(64, 1000)
        assert time.perf_counter() - t < timeout_s, "serving loop stalled"
    return got


def test_submit_returns_busy_when_the_queue_is_full(lib):
    """max_queued = 1 and one launch stream: while a long request holds the stream, one more
    request waits in the queue and the next submit returns FSMP_ERR_BUSY (nothing queued).
    Every request that was accepted still completes."""
    params, events = workloads.make_events("serving_20k_eps", n_events=2, seed=7, n_steps=200)
    wl = workloads.make_workload("batched_uneven_100k", n_waveforms=20000, n_steps=6000, seed=8)
    with fsmp.Context(_params(params, n_streams=1, max_queued=1)) as ctx:
        assert ctx.submit(wl["batch"], request_id=0) == fsmp.OK  # several seconds of work
        codes = []
        t = time.perf_counter()
        while fsmp.ERR_BUSY not in codes and time.perf_counter() - t < 1.0:
            codes.append(ctx.submit(events[len(codes) % 2], request_id=1 + len(codes)))
        assert fsmp.ERR_BUSY in codes, codes
        accepted = [c for c in codes if c == fsmp.OK]
        assert len(accepted) <= 2 and set(codes) <= {fsmp.OK, fsmp.ERR_BUSY}
        done = _drain(ctx, 1 + len(accepted))
    assert all(r["status"] == fsmp.OK for r in done)


def test_submit_refuses_a_request_over_the_memory_budget(lib):
    """A request whose device footprint exceeds device_mem_budget is refused at submit with
    FSMP_ERR_NOMEM (it could never be admitted); a smaller one still runs."""
    params, events = workloads.make_events("serving_20k_eps", n_events=8, seed=9, n_steps=100)
    big = max(events, key=lambda e: len(e["samples"]))
    small = min(events, key=lambda e: len(e["samples"]))
    budget = 32 * 1024
    assert len(big["samples"]) * 4 > budget and len(small["samples"]) * 8 + 8192 < budget
    with fsmp.Context(_params(params, device_mem_budget=budget)) as ctx:
        assert ctx.submit(big, request_id=1) == fsmp.ERR_NOMEM
        assert ctx.submit(small, request_id=2) == fsmp.OK
        assert _drain(ctx, 1)[0]["status"] == fsmp.OK


def test_submit_refuses_malformed_batches(lib):
    """Malformed host batches are refused at submit with FSMP_ERR_INVALID and nothing queued:
    offsets not starting at 0, a non-positive lambda0, an empty window, a window longer than
    n_max, T_lo without T_hi, T_hi <= T_lo, negative steps."""
    params, events = workloads.make_events("serving_20k_eps", n_events=1, seed=11, n_steps=50)
    ev = events[0]
    W = len(ev["offsets"]) - 1
    offs = np.asarray(ev["offsets"], np.int32)
    n = np.diff(offs)
    bad = [dict(offsets=offs + 1), dict(lambda0=np.where(np.arange(W) == 0, 0.0, ev["lambda0"])),
           dict(offsets=np.concatenate([[0, 0], offs[1:]]).astype(np.int32)[:W + 1]),
           dict(T_lo=np.zeros(W, np.int32)), dict(T_lo=np.full(W, 5, np.int32), T_hi=np.full(W, 5, np.int32)),
           dict(n_steps=-1)]
    with fsmp.Context(_params(params, n_max=int(n.max()))) as ctx:
        for k, extra in enumerate(bad):
            with pytest.raises(fsmp.FsmpError) as ei:
                ctx.submit(dict(ev, **extra), request_id=k)
            assert ei.value.code == fsmp.ERR_INVALID, extra
        long_ev = dict(ev, samples=np.zeros(int(offs[-1]) + 600, np.float32),
                       offsets=np.concatenate([offs[:-1], [offs[-1] + 600]]).astype(np.int32))
        with pytest.raises(fsmp.FsmpError) as ei:
            ctx.submit(long_ev, request_id=99)
        assert ei.value.code == fsmp.ERR_INVALID
        assert ctx.poll(8, 200) == []  # nothing was queued
        assert ctx.submit(ev, request_id=100) == fsmp.OK
        assert _drain(ctx, 1)[0]["status"] == fsmp.OK


def test_drift_flag_under_a_tiny_tolerance(lib):
    """FP32 mode with drift_tol = 1e-300: an FP64 refresh that finds the incremental FP32 state
    different from its rebuild at all flags the chain FSMP_ST_DRIFT, so nearly every chain that
    refreshed is flagged (a refresh with no PE has nothing to drift) and none without a
    refresh is; with the default tolerance none is."""
    wl = workloads.make_workload("batched_uneven_100k", n_waveforms=256, n_steps=400, seed=13)
    n_max = int(np.diff(wl["batch"]["offsets"]).max())
    res = {}
    for tol in (1e-300, 0.0):
        with fsmp.Context(wl["params"], n_max=n_max, precision=fsmp.FP32_REFRESH, refresh_every=8,
                          drift_tol=tol) as ctx:
            res[tol], _ = ctx.run(wl["batch"])
    s = res[1e-300]
    refreshed = s["n_refresh"] > 0
    assert refreshed.sum() > 100
    assert np.mean((s["status"][refreshed] & fsmp.ST_DRIFT) != 0) > 0.9
    assert np.all((s["status"][~refreshed] & fsmp.ST_DRIFT) == 0)
    assert np.all((res[0.0]["status"] & fsmp.ST_DRIFT) == 0)


def test_request_returns_when_its_own_chains_finish(lib):
    """A light request packed into the same launch as a heavy one returns as soon as its own
    chain is done (each chain raises a flag in host-mapped memory after writing its summary there,
    and the serving loop returns a request once all its chains' flags are up), not when the
    launch ends; the heavy one's result is unaffected."""
    params = workloads.CONFIGS["serving_20k_eps"]["params"]
    wl = workloads.make_workload("batched_uneven_100k", n_waveforms=400, seed=23)
    b = wl["batch"]
    heavy_i, light_i = int(np.argmax(b["lambda0"])), int(np.argmin(b["lambda0"]))
    heavy = dict(workloads.subset(b, [heavy_i]), n_steps=20000, burn_in=0)
    light = dict(workloads.subset(b, [light_i]), n_steps=20000, burn_in=0)
    first = dict(workloads.subset(b, [light_i]), n_steps=3000, burn_in=0)
    with fsmp.Context(_params(params, n_streams=1)) as ctx:
        s_alone, _ = ctx.run(heavy, request_id=9)
        # while `first` holds the only launch stream, the heavy and the light request queue up
        # and are then packed into one launch
        assert ctx.submit(first, request_id=0) == fsmp.OK
        assert ctx.submit(heavy, request_id=1) == fsmp.OK
        assert ctx.submit(light, request_id=2) == fsmp.OK
        got = {r["request_id"]: r for r in _drain(ctx, 3)}
    assert all(r["status"] == fsmp.OK for r in got.values())
    lat_heavy, lat_light = got[1]["latency_s"], got[2]["latency_s"]
    assert lat_light < 0.5 * lat_heavy, (lat_light, lat_heavy)
    for f in FLOAT_FIELDS:
        np.testing.assert_array_equal(got[1]["summaries"][f], s_alone[f], err_msg=f)
