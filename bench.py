#!/usr/bin/env python
"""FSMP MCMC throughput on GB300 (one JSON line on stdout).

Default workload: 100k waveforms of 64-512 samples (lambda log-uniform 0.5-50, windows
trimmed to the PE span plus the SER support), 2000 MCMC steps per chain, FP32 chain state
with FP64 refreshes every 64 accepted moves. One bench "step" runs every chain of the batch
through all its MCMC steps (the whole hot path: tables are built once per context).

  value   MCMC steps/s with inputs resident in HBM (fsmp_run_device, CUDA events on the stream)
  e2e     the same metric through fsmp_submit / fsmp_poll with host buffers (host<->device
          copies inside the timed region)

`--impl reference` times the FP64 CPU oracle on the host cores instead (a bounded sample of
the same workload per step). Under torchrun each rank runs its own shard (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FSMP MCMC steps/s at stated error vs plain FP64 form; p50/p99 event latency"
UNIT = "MCMC steps/s"
BUCKET_EDGES = [64, 96, 128, 160, 192, 224, 256, 320, 384, 512, 768, 1024, 2048, 8192]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched_uneven_100k")
    ap.add_argument("--n-waveforms", type=int, default=0, help="override the workload size (testing)")
    ap.add_argument("--mcmc-steps", type=int, default=0, help="override MCMC steps per chain (testing)")
    ap.add_argument("--precision", default="", help="fp32 | fp64 (default: the workload's)")
    ap.add_argument("--threads", type=int, default=0, help="threads per chain CTA (0: library default)")
    ap.add_argument("--pe-tile", type=int, default=0, help="PE kernel: shared-memory C^-1 tile (0: default)")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="PE kernel: resident CTAs per SM (0: max)")
    ap.add_argument("--pe-lanes", type=int, default=0, choices=[0, 16, 32],
                    help="PE kernel: lanes per chain (0: chosen by the autotuner)")
    ap.add_argument("--kernel", default="auto", choices=["auto", "smem", "global", "plain", "pe"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="PE kernel: keep the default launch shape")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target wall time of the CPU sample")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--window-range", default="", help="lo,hi: keep only windows of lo..hi samples (profiling)")
    ap.add_argument("--graph", default="auto", choices=["auto", "on", "off"],
                    help="capture each step's launches in a CUDA graph (auto: on for lowocc_bulk_1m)")
    ap.add_argument("--rate", type=float, default=0.0, help="serving: offered events/s (0: the workload's)")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="serving: length of the arrival stream")
    ap.add_argument("--serve-pool", type=int, default=1024, help="serving: distinct events replayed by the stream")
    ap.add_argument("--serve-streams", type=int, default=0, help="serving: concurrent launch streams (0: library default)")
    ap.add_argument("--stage", default="chain", choices=["chain", "lucyddm"],
                    help="lucyddm: time the LucyDDM deconvolution (Sec. 2.3) of the workload instead of the chains")
    ap.add_argument("--lucy-iters", type=int, default=2000, help="lucyddm stage: Lucy iterations")
    ap.add_argument("--plain-sample", type=int, default=48,
                    help="waveforms of the workload timed in the plain FP64 form (vs_baseline; 0: skip)")
    ap.add_argument("--error-sample", type=int, default=256,
                    help="waveforms of the workload compared with the FP64 oracle (error; 0: skip)")
    ap.add_argument("--latency-rate", type=float, default=1000.0,
                    help="events/s of the serving leg that gives the p50/p99 latency (0: skip)")
    ap.add_argument("--latency-seconds", type=float, default=8.0, help="length of that serving leg's stream")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def emit(obj):
    print(json.dumps(obj), flush=True)


def serving_workload(name):
    from paper_2403_03156_gb300 import workloads
    return "rate_hz" in workloads.CONFIGS[name]


def shard_workload(args, rank):
    from paper_2403_03156_gb300 import workloads
    if serving_workload(args.workload):  # events of the pool, as one batch
        params, events = workloads.make_events(args.workload, min(args.serve_pool, 256), seed=args.seed + 1000 * rank,
                                               n_steps=args.mcmc_steps or None)
        batch = concat_events(events)
        batch["burn_in"] = int(batch["n_steps"]) // 5
        cfg = workloads.CONFIGS[args.workload]
        return dict(name=args.workload, params=params, batch=batch,
                    meta=dict(precision=cfg["precision"], refresh_every=cfg.get("refresh_every", 0)))
    from paper_2403_03156_gb300 import sharding
    # RNG ids unique across ranks: rank r owns waveforms [r W, (r+1) W) of the job
    wl = sharding.rank_workload(args.workload, rank, n_waveforms=args.n_waveforms or None, seed=args.seed,
                                n_steps=args.mcmc_steps or None)
    # burn-in of one fifth of the chain for the posterior summaries (it costs the same steps)
    wl["batch"]["burn_in"] = int(wl["batch"]["n_steps"]) // 5
    b = wl["batch"]
    if args.window_range:
        lo, hi = (int(x) for x in args.window_range.split(","))
        n = np.diff(b["offsets"])
        keep = np.nonzero((n >= lo) & (n <= hi))[0]
        wl["batch"] = workloads.subset(b, keep)
    return wl


def concat_events(events):
    """The events' waveforms as one batch (each keeps its RNG index)."""
    offs, samples, ids = [0], [], []
    for e in events:
        samples.append(e["samples"])
        offs.extend((offs[-1] + e["offsets"][1:]).tolist())
        ids.append(np.uint64(e["index_base"]) + np.arange(len(e["offsets"]) - 1, dtype=np.uint64))
    out = dict(samples=np.concatenate(samples), offsets=np.asarray(offs, np.int32),
               lambda0=np.concatenate([e["lambda0"] for e in events]),
               t_origin_ns=np.concatenate([e["t_origin_ns"] for e in events]),
               wf_ids=np.concatenate(ids), seed=events[0]["seed"], index_base=0,
               n_steps=events[0]["n_steps"], burn_in=events[0].get("burn_in", 0))
    return out


# ------------------------------------------------------------------------ CPU oracle arm
def oracle_rate(wl, target_s, rng_seed=0, max_wf=None):
    """Time the FP64 CPU oracle (incremental mode, one thread per host core) on a random
    sample of the workload's waveforms, sized to about target_s seconds of wall time."""
    from oracle import oracle
    from paper_2403_03156_gb300 import workloads
    b = wl["batch"]
    W = len(b["offsets"]) - 1
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(rng_seed)
    n_probe = min(W, max(cores, 16))
    idx = rng.choice(W, n_probe, replace=False)
    sub = workloads.subset(b, idx)
    t = time.perf_counter()
    oracle.run_batch(wl["params"], sub, oracle.MODE_INCREMENTAL, n_threads=cores)
    dt = max(time.perf_counter() - t, 1e-3)
    n_full = int(min(W if max_wf is None else max_wf, max(n_probe, n_probe * target_s / dt)))
    idx = rng.choice(W, n_full, replace=False)
    sub = workloads.subset(b, idx)
    t = time.perf_counter()
    oracle.run_batch(wl["params"], sub, oracle.MODE_INCREMENTAL, n_threads=cores)
    dt = time.perf_counter() - t
    steps = n_full * int(b["n_steps"])
    return dict(value=steps / dt, unit=UNIT, cores=cores, kind="oracle",
                sample="%d random waveforms of %s x %d MCMC steps (FP64 incremental oracle, %d threads, %.1f s)"
                       % (n_full, wl["name"], int(b["n_steps"]), cores, dt)), dt, n_full


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = shard_workload(args, 0)
    b = wl["batch"]
    cores = os.cpu_count() or 1
    # each step: a bounded random sample, sized so warmup + steps end within a few minutes
    per_step_target = min(args.cpu_seconds, 20.0, 150.0 / max(1, args.steps + args.warmup))
    base, _, n_wf = oracle_rate(wl, per_step_target)
    from oracle import oracle
    from paper_2403_03156_gb300 import workloads
    rng = np.random.default_rng(7)
    W = len(b["offsets"]) - 1
    times = []
    for it in range(args.warmup + args.steps):
        sub = workloads.subset(b, rng.choice(W, n_wf, replace=False))
        t = time.perf_counter()
        oracle.run_batch(wl["params"], sub, oracle.MODE_INCREMENTAL, n_threads=cores)
        if it >= args.warmup:
            times.append(time.perf_counter() - t)
    steps = n_wf * int(b["n_steps"])
    value = steps / (sum(times) / len(times))
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times),
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
          "data": "synthetic",
          "config": {"workload": wl["name"], "n_waveforms": W, "mcmc_steps_per_chain": int(b["n_steps"]),
                     "sample_per_step": n_wf},
          "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                           "sample": "%d random waveforms x %d MCMC steps per step" % (n_wf, int(b["n_steps"]))},
          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


# ------------------------------------------------------------------------ GPU arm
class Clocks:
    """nvidia-smi samples of SM clocks and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.QUERY,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def buckets_of(lengths):
    """Length buckets (indices into a decreasing-length order) for one launch each."""
    order = np.argsort(-lengths, kind="stable")
    n_sorted = lengths[order]
    out, i, W = [], 0, len(order)
    while i < W:
        nmax = int(n_sorted[i])
        lo = max([e for e in BUCKET_EDGES if e < nmax], default=0)
        j = i
        while j < W and n_sorted[j] > lo:
            j += 1
        out.append((order[i:j], nmax))
        i = j
    return out


def cost_order(lengths, lambda0):
    """Waveforms by decreasing expected chain cost, window length x (1 + lambda0): the
    persistent launch hands chains out in this order, so the heaviest start first and the
    launch's tail is made of light chains."""
    return np.argsort(-(np.asarray(lengths, np.float64) * (1.0 + np.asarray(lambda0, np.float64))), kind="stable")


def device_batches(torch, wl, dev, n_smem_max, one_launch=False):
    """Split the workload into length buckets, each a device-resident sub-batch (or, for the
    PE-space kernel, one batch in decreasing expected chain cost)."""
    from paper_2403_03156_gb300 import fsmp, workloads
    b = wl["batch"]
    lengths = np.diff(b["offsets"]).astype(np.int64)
    subs = []
    if one_launch:
        order = cost_order(lengths, b["lambda0"])
        groups = [(order, int(lengths.max()))]
    else:
        groups = buckets_of(lengths)
    for idx, nmax in groups:
        if not one_launch and nmax > n_smem_max and int(lengths[idx].min()) <= n_smem_max:
            # never mix windows on both sides of the shared-memory limit
            big = idx[lengths[idx] > n_smem_max]
            small = idx[lengths[idx] <= n_smem_max]
            parts = [(big, nmax), (small, int(lengths[small].max()))]
        else:
            parts = [(idx, nmax)]
        for ii, nm in parts:
            sb = workloads.subset(b, ii)
            W = len(ii)
            t = {
                "samples": torch.from_numpy(sb["samples"]).to(dev),
                "offsets": torch.from_numpy(sb["offsets"].astype(np.int32)).to(dev),
                "lambda0": torch.from_numpy(sb["lambda0"].astype(np.float64)).to(dev),
                "t_origin_ns": torch.from_numpy(sb["t_origin_ns"].astype(np.float64)).to(dev),
                "wf_ids": torch.from_numpy(sb["wf_ids"].astype(np.int64)).to(dev),
                "out": torch.zeros(W * fsmp.SUMMARY_DTYPE.itemsize, dtype=torch.uint8, device=dev),
            }
            if sb.get("T_lo") is not None:
                t["T_lo"] = torch.from_numpy(sb["T_lo"].astype(np.int32)).to(dev)
                t["T_hi"] = torch.from_numpy(sb["T_hi"].astype(np.int32)).to(dev)
            subs.append((t, nm, W, np.asarray(ii)))
    return subs


def load_traffic(kernel_src, name, workload):
    """DRAM traffic and instructions per launch of a chain kernel on a workload, from the committed
    ncu summary profiles/<name>_dram_traffic.json, if it was taken on the current kernel source
    and on that workload; else None."""
    path = os.path.join(ROOT, "profiles", name + "_dram_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    if d.get("kernel_sha") != sha:
        return None
    return d.get("workloads", {}).get(workload)


def plain_fp64_baseline(torch, wl, dev, n_sample, sample_seed=3):
    """The plain one-launch-per-chain FP64 form (FSMP_KERNEL_PLAIN: one kernel launch per chain,
    full Sigma^-1 in global memory), the baseline the metric compares with, timed with CUDA
    events on a random sample of the same workload on the same GPU. Returns (stats, summaries,
    the sample's waveform indices)."""
    from paper_2403_03156_gb300 import fsmp, workloads
    b = wl["batch"]
    W = len(b["offsets"]) - 1
    rng = np.random.default_rng(sample_seed)
    idx = np.sort(rng.choice(W, min(n_sample, W), replace=False))
    sb = workloads.subset(b, idx)
    n_max = int(np.diff(sb["offsets"]).max())
    params = dict(wl["params"], precision=fsmp.FP64, kernel=fsmp.KERNEL_PLAIN, n_max=max(n_max, 64),
                  device=dev.index or 0)
    n_steps, burn = int(b["n_steps"]), int(b.get("burn_in", 0))
    t = _device_tensors(torch, sb, dev)
    with fsmp.Context(params) as ctx:
        w = _device_tensors(torch, workloads.subset(sb, np.arange(2)), dev)  # warm-up (code, caches)
        ctx.run_device(w, n_steps=50, burn_in=0, seed=int(b["seed"]), n_max_hint=n_max)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream(dev)
        e0.record(stream)
        ctx.run_device(t, n_steps=n_steps, burn_in=burn, seed=int(b["seed"]), n_max_hint=n_max, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
    summ = fsmp.summaries_from_bytes(t["out"].cpu().numpy())
    rate = len(idx) * n_steps / (ms * 1e-3)
    stats = {"value": rate, "unit": UNIT, "form": "plain FP64: one launch per chain, Sigma^-1 in global memory",
             "sample": "%d random waveforms of %s x %d MCMC steps, %d launches, %.2f s (CUDA events)"
                       % (len(idx), wl["name"], n_steps, len(idx), ms * 1e-3)}
    return stats, summ, idx


def _device_tensors(torch, sb, dev, trace_steps=0):
    from paper_2403_03156_gb300 import fsmp
    W = len(sb["offsets"]) - 1
    t = {"samples": torch.from_numpy(sb["samples"]).to(dev),
         "offsets": torch.from_numpy(sb["offsets"].astype(np.int32)).to(dev),
         "lambda0": torch.from_numpy(np.asarray(sb["lambda0"], np.float64)).to(dev),
         "t_origin_ns": torch.from_numpy(np.asarray(sb["t_origin_ns"], np.float64)).to(dev),
         "wf_ids": torch.from_numpy(np.asarray(sb["wf_ids"], np.uint64).astype(np.int64)).to(dev),
         "out": torch.zeros(W * fsmp.SUMMARY_DTYPE.itemsize, dtype=torch.uint8, device=dev)}
    if sb.get("T_lo") is not None:
        t["T_lo"] = torch.from_numpy(sb["T_lo"].astype(np.int32)).to(dev)
        t["T_hi"] = torch.from_numpy(sb["T_hi"].astype(np.int32)).to(dev)
    if trace_steps:
        t["trace"] = torch.zeros(W * trace_steps * fsmp.TRACE_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    return t


def _paired(d):
    """mean +- standard error of paired differences, and whether |mean| < 3 SE."""
    d = np.asarray(d, np.float64)
    se = float(d.std(ddof=1) / math.sqrt(len(d))) if len(d) > 1 else float("nan")
    m = float(d.mean())
    return {"mean": m, "se": se, "within_3se": bool(abs(m) <= 3 * se + 1e-12)}


def error_vs_fp64(torch, ctx, wl, dev, n_sample, sample_seed=5):
    """The stated error of the measured FP32 path against the FP64 oracle on a random sample of
    the same workload (same chains: same Philox streams): paired differences of the posterior
    summaries (mean +- SE over waveforms), and |Delta log alpha| per step over each chain's
    lockstep prefix (the steps before its first decision that differs from the FP64 chain's)."""
    from oracle import oracle
    from paper_2403_03156_gb300 import fsmp, workloads
    b = wl["batch"]
    W = len(b["offsets"]) - 1
    rng = np.random.default_rng(sample_seed)
    idx = np.sort(rng.choice(W, min(n_sample, W), replace=False))
    sb = workloads.subset(b, idx)
    n_steps, burn = int(b["n_steps"]), int(b.get("burn_in", 0))
    n_max = int(np.diff(sb["offsets"]).max())
    t = _device_tensors(torch, sb, dev, trace_steps=n_steps)
    ctx.run_device(t, n_steps=n_steps, burn_in=burn, seed=int(b["seed"]), n_max_hint=n_max)
    torch.cuda.synchronize(dev)
    sg = fsmp.summaries_from_bytes(t["out"].cpu().numpy())
    tg = fsmp.traces_from_bytes(t["trace"].cpu().numpy(), len(idx))
    so, to = oracle.run_batch(wl["params"], sb, oracle.MODE_INCREMENTAL, n_threads=os.cpu_count() or 1, trace=True)
    out = {"reference": "FP64 CPU oracle (incremental Woodbury), %d random waveforms x %d steps, burn-in %d"
                        % (len(idx), n_steps, burn)}
    for f in ("mean_N", "mean_Q", "mean_t0", "lambda_hat"):
        out[f] = _paired(sg[f] - so[f])
    differ = tg["flags"] != to["flags"]
    first = np.where(differ.any(1), differ.argmax(1), n_steps)
    keep = np.arange(n_steps)[None, :] < first[:, None]
    la_g, la_o = tg["la"][keep], to["la"][keep]
    ok = np.isfinite(la_g) & np.isfinite(la_o) & (la_o > -40.0)
    dla = np.abs(la_g[ok] - la_o[ok])
    out["dlog_alpha"] = {"p50": float(np.percentile(dla, 50)), "p99": float(np.percentile(dla, 99)),
                         "max": float(dla.max()), "steps": int(ok.sum()),
                         "lockstep_fraction": float(keep.sum() / keep.size)}
    return out


def serve_stream(ctx, pool, rate, seconds, seed, warmup=3):
    """The serving loop under a Poisson stream of events (submit / poll through the C ABI, host
    buffers, copies included). Events are replayed from `pool`, each arrival with its own RNG
    seed. Returns steps/s of the served events, p50/p99 event latency (submit to result) and
    whether the offered rate was sustained."""
    import threading
    from paper_2403_03156_gb300 import fsmp
    n_steps = int(pool[0]["n_steps"])
    for i in range(warmup):  # the first requests pay for lazy initialisation
        ctx.run(pool[i % len(pool)], request_id=(1 << 40) + i)
    rng = np.random.default_rng(1234 + seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, int(rate * seconds * 1.2) + 16))
    arrivals = arrivals[arrivals < seconds]
    n_ev = len(arrivals)
    sizes = np.zeros(n_ev, np.int64)
    lat = np.full(n_ev, np.nan)
    t_done_last = [0.0]
    done = [0]
    stop = threading.Event()

    def poller():
        while not stop.is_set() or done[0] < n_ev:
            for r in ctx.poll(4096, 50):
                i = int(r["request_id"])
                lat[i] = r["latency_s"]
                done[0] += 1
                t_done_last[0] = time.perf_counter()
            if stop.is_set() and done[0] >= n_ev:
                break

    launches0 = ctx.info()["n_launches"]
    th = threading.Thread(target=poller, daemon=True)
    th.start()
    t0 = time.perf_counter()
    busy = 0
    for i in range(n_ev):
        ev = dict(pool[i % len(pool)])
        ev["seed"] = int(seed) * 1000003 + i  # each arrival is a new event for the sampler
        sizes[i] = len(ev["offsets"]) - 1
        wait = t0 + arrivals[i] - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        while ctx.submit(ev, request_id=i) == fsmp.ERR_BUSY:
            busy += 1
            time.sleep(0.001)
    t_sub = time.perf_counter() - t0
    stop.set()
    th.join()
    t_all = t_done_last[0] - t0
    steps = float(sizes.sum()) * n_steps
    completed = n_ev / t_all
    bytes_in = sum(int(pool[i % len(pool)]["samples"].nbytes) for i in range(n_ev)) / n_ev
    return {"value": steps / t_all, "steps": steps, "t_all": t_all, "events": n_ev, "waveforms": int(sizes.sum()),
            "offered_rate_hz": rate, "completed_rate_hz": completed, "sustained": bool(completed >= 0.95 * rate),
            "submitted_in_s": t_sub, "stream_s": seconds, "busy_retries": busy,
            "launches": int(ctx.info()["n_launches"] - launches0), "mcmc_steps_per_chain": n_steps,
            "p50_s": float(np.nanpercentile(lat, 50)), "p99_s": float(np.nanpercentile(lat, 99)),
            "mean_s": float(np.nanmean(lat)), "max_s": float(np.nanmax(lat)),
            "h2d_bytes_per_event": int(bytes_in), "d2h_bytes_per_event": int(sizes.mean() * fsmp.SUMMARY_DTYPE.itemsize)}


def serving_latency_leg(local, rate, seconds, seed, pool_n=256):
    """A short serving stream of the serving workload (events of 1-64 waveforms of 64-512
    samples, lambda to 100, 1500 steps) at a rate the loop sustains on one GPU: the p50/p99 event
    latency part of the metric."""
    from paper_2403_03156_gb300 import fsmp, workloads
    cfg = workloads.CONFIGS["serving_20k_eps"]
    params, pool = workloads.make_events("serving_20k_eps", pool_n, seed=seed)
    for e in pool:
        e["burn_in"] = int(e["n_steps"]) // 5
    with fsmp.Context(dict(params, precision=fsmp.FP32_REFRESH, refresh_every=cfg.get("refresh_every", 64),
                           n_max=cfg["win_max"], device=local, max_queued=1 << 20)) as ctx:
        r = serve_stream(ctx, pool, rate, seconds, seed)
    return {"workload": "serving_20k_eps", "p50_s": r["p50_s"], "p99_s": r["p99_s"], "mean_s": r["mean_s"],
            "max_s": r["max_s"], "offered_rate_hz": rate, "completed_rate_hz": r["completed_rate_hz"],
            "sustained": r["sustained"], "events": r["events"], "waveforms": r["waveforms"],
            "stream_s": seconds, "steps_per_s": r["value"],
            "timing": "host clock, submit to result visible in fsmp_poll, host buffers"}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2403_03156_gb300 import build, fsmp, sharding, workloads

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    build.build()
    wl = shard_workload(args, rank)
    cfg = workloads.CONFIGS[args.workload]
    prec = {"fp32": fsmp.FP32_REFRESH, "fp64": fsmp.FP64}[args.precision or cfg["precision"]]
    b = wl["batch"]
    W = len(b["offsets"]) - 1
    lengths = np.diff(b["offsets"])
    params = dict(wl["params"], precision=prec, refresh_every=wl["meta"].get("refresh_every") or 64,
                  n_max=int(max(lengths.max(), 64)), device=local, threads_per_chain=args.threads,
                  pe_tile=args.pe_tile, pe_ctas_per_sm=args.ctas_per_sm, pe_lanes=args.pe_lanes,
                  kernel={"auto": fsmp.KERNEL_AUTO, "smem": fsmp.KERNEL_SMEM, "global": fsmp.KERNEL_GLOBAL,
                          "plain": fsmp.KERNEL_PLAIN, "pe": fsmp.KERNEL_PE}[args.kernel])
    ctx = fsmp.Context(params)
    info = ctx.info()
    peaks = ctx.measure_peaks()
    pe = args.kernel in ("auto", "pe")
    subs = device_batches(torch, wl, dev, info["n_smem_max"], one_launch=pe)
    n_steps = int(b["n_steps"])
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    tuned = None
    if pe and not args.no_autotune:  # launch shape from timed trials on a sample (not timed)
        t0_, nm0, _, _ = subs[0]
        # trials of the full chain length: the cost per step grows with N over a chain, and a
        # short trial would favour shapes that suit the first steps
        # (a sample of at most a quarter of the batch, so that the trials stay short next to it)
        tuned = ctx.autotune(t0_, sample=min(32768, max(2048, W // 4)), trial_steps=n_steps, seed=int(b["seed"]),
                             n_max_hint=nm0)

    def one_step(ev=None):
        for k, (t, nm, _, _) in enumerate(subs):
            if ev is not None:
                ev[k][0].record(stream)
            ctx.run_device(t, n_steps=n_steps, burn_in=int(b.get("burn_in", 0)), seed=int(b["seed"]),
                           n_max_hint=nm, stream=stream)
            if ev is not None:
                ev[k][1].record(stream)

    for _ in range(args.warmup):
        flush.zero_()
        one_step()
    torch.cuda.synchronize(dev)
    use_graph = args.graph == "on" or (args.graph == "auto" and args.workload == "lowocc_bulk_1m")
    graph = None
    if use_graph:
        # one CUDA graph per step: the chain launches (counter reset + kernel) replayed as a unit
        graph = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream(dev)
        cs.wait_stream(stream)
        with torch.cuda.stream(cs):
            with torch.cuda.graph(graph, stream=cs):
                for (t, nm, _, _) in subs:
                    ctx.run_device(t, n_steps=n_steps, burn_in=int(b.get("burn_in", 0)), seed=int(b["seed"]),
                                   n_max_hint=nm, stream=cs)
        stream.wait_stream(cs)
        graph.replay()
        torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    evs = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in subs]
           for _ in range(args.steps)]
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        flush.zero_()                      # L2 flush between timed steps (256 MiB write)
        if graph is not None:
            evs[i][0][0].record(stream)
            graph.replay()
            evs[i][0][1].record(stream)
        else:
            one_step(evs[i])
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    W_total, elapsed_ms = sharding.job_totals(dist if world > 1 else None, W, elapsed_ms, device=dev)
    ms_per_step = elapsed_ms / args.steps
    value = W_total * n_steps / (ms_per_step / 1000.0)

    # per-launch roofline of the dominant kernel (the longest bucket launch)
    summ = [fsmp.summaries_from_bytes(t["out"].cpu().numpy()) for (t, _, _, _) in subs]
    if graph is not None:  # one timed interval per step: the whole graph
        durs = np.array([[evs[i][0][0].elapsed_time(evs[i][0][1])] + [0.0] * (len(subs) - 1)
                         for i in range(args.steps)])
    else:
        durs = np.array([[evs[i][k][0].elapsed_time(evs[i][k][1]) for k in range(len(subs))]
                         for i in range(args.steps)])
    mean_dur = durs.mean(0)
    kdom = int(np.argmax(mean_dur))
    alg_bytes = float(summ[kdom]["alg_bytes"].sum())
    achieved = alg_bytes / (mean_dur[kdom] * 1e-3) / 1e9
    kernel_src = os.path.join(ROOT, "paper_2403_03156_gb300", "csrc", "fsmp_pe_kernel.cuh" if pe else "fsmp_chain.cu")
    tr = load_traffic(kernel_src, "pe_kernel" if pe else "chain_kernel", args.workload)
    allsum = np.concatenate(summ)
    acc = allsum["acc"].sum(0)
    prop = allsum["prop"].sum(0)
    roofline = {"bound": "smem", "achieved": achieved, "peak": peaks["smem_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["smem_gbs"],
                "traffic": None if tr is None else tr["traffic_bytes_per_launch"] * (
                    (summ[kdom]["prop"].sum() / max(1.0, tr["units_per_launch"])) if tr.get("scale_by_units") else 1.0),
                "peak_source": "measured live: fsmp_measure_peaks (16-byte shared loads, 4 CTAs/SM)",
                "kernel": ("pe_kernel<%s>, one launch, n<=%d (%d chains)" if pe else
                           "chain_kernel<%s, smem>, bucket n<=%d (%d chains)") % (
                    "float" if prec == fsmp.FP32_REFRESH else "double", subs[kdom][1], subs[kdom][2]),
                "alg_bytes_per_launch": alg_bytes, "launch_ms": float(mean_dur[kdom]),
                "all_launch_ms": [float(x) for x in mean_dur]}
    if prec == fsmp.FP64:
        fp64 = peaks["fp64_tflops"]
        roofline["note"] = "FP64 mode is FP64-FMA bound on this part (measured %.2f TFLOP/s FP64)" % fp64
    if tr is not None and tr.get("warp_inst_per_step"):
        # the binding roofline of a latency-bound chain: instruction issue. Warp instructions per
        # MCMC step from the committed ncu capture of the same kernel source (smsp__inst_executed
        # / steps), times the launch's steps per second, against 4 issue slots per SM per clock at
        # the SM clock sampled during the timed region
        steps_launch = float(summ[kdom]["prop"].sum())
        mhz = (clk or {}).get("sm_mhz") or 2070.0
        ach = tr["warp_inst_per_step"] * steps_launch / (mean_dur[kdom] * 1e-3)
        pk_issue = info["sm_count"] * 4 * mhz * 1e6
        roofline["issue"] = {"achieved": ach, "peak": pk_issue, "unit": "warp instructions/s", "frac": ach / pk_issue,
                             "warp_inst_per_step": tr["warp_inst_per_step"],
                             "source": "instructions per step: " + tr.get("command", "ncu capture")}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == fsmp.FP32_REFRESH else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "kernel": args.kernel, "n_waveforms": W_total,
                       "mcmc_steps_per_chain": n_steps,
                       "precision": "fp32 state + fp64 refresh" if prec == fsmp.FP32_REFRESH else "fp64",
                       "refresh_every": params["refresh_every"],
                       "window_samples": [int(lengths.min()), int(np.median(lengths)), int(lengths.max())],
                       "launches_per_step": len(subs), "threads_per_chain": info["threads_per_chain"],
                       "cuda_graph": graph is not None, "autotune": tuned,
                       "l2": "flushed between timed steps (256 MiB write)",
                       "accept_rate": float(acc.sum() / max(1, prop.sum())),
                       "accepts_per_type": [int(x) for x in acc], "proposals_per_type": [int(x) for x in prop]},
            "roofline": roofline,
            "gpu_launches": (W if args.kernel == "plain" else len(subs)) * args.steps, "clocks": clk,
            "peaks_measured": peaks}

    # e2e: the public host-buffer API (submit / poll), copies inside the timed region
    if not args.no_e2e:
        host = dict(b)
        e2e_times = []
        lat = []
        for i in range(1 + min(args.steps, 3)):
            t0 = time.perf_counter()
            ctx.run(host, request_id=100 + i)
            dt = time.perf_counter() - t0
            if i > 0:
                e2e_times.append(dt)
        # what the serving loop stages per request: samples, offsets and 11 per-waveform
        # arrays (lambda0, t_origin, T_lo, T_hi, t0_init, wf_id, seed, n_steps, burn_in,
        # trace offset, processing order)
        h2d = b["samples"].nbytes + 4 * (W + 1) + W * (8 + 8 + 4 + 4 + 8 + 8 + 8 + 4 + 4 + 8 + 4)
        d2h = W * fsmp.SUMMARY_DTYPE.itemsize
        e2e_val = W * n_steps / statistics.mean(e2e_times)
        if world > 1:
            te = torch.tensor([statistics.mean(e2e_times)], dtype=torch.float64, device=dev)
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
            e2e_val = W_total * n_steps / float(te.item())
        line["e2e"] = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(d2h), "steps": len(e2e_times)}
    # the metric's other clauses, measured after the timed region on rank 0: the plain FP64 form
    # on a sample of the same workload (vs_baseline), the stated error against FP64, and the
    # p50/p99 event latency of a serving stream
    if rank == 0 and not serving_workload(args.workload):
        full = np.zeros(W, fsmp.SUMMARY_DTYPE)
        for (_, _, _, ii), sm in zip(subs, summ):
            full[ii] = sm
        if args.plain_sample > 0 and args.kernel != "plain":
            plain, s_plain, pidx = plain_fp64_baseline(torch, wl, dev, args.plain_sample)
            line["vs_baseline"] = value / plain["value"]
            plain["ratio"] = line["vs_baseline"]
            # the same chains (same Philox streams) in both forms: the measured path's error
            # against the plain FP64 form itself
            plain["error_vs_plain"] = {f: _paired(full[f][pidx] - s_plain[f]) for f in
                                       ("mean_N", "mean_Q", "mean_t0", "lambda_hat")}
            plain["error_vs_plain"]["waveforms"] = int(len(pidx))
            line["baseline"] = plain
            line["config"]["vs_baseline_of"] = "the plain one-launch-per-chain FP64 form on the same GPU"
        if args.error_sample > 0:
            line["error"] = error_vs_fp64(torch, ctx, wl, dev, args.error_sample)
    ctx.close()
    if rank == 0 and args.latency_rate > 0 and not serving_workload(args.workload):
        line["latency"] = serving_latency_leg(local, args.latency_rate, args.latency_seconds, args.seed)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base, _, _ = oracle_rate(wl, args.cpu_seconds)
        line["cpu_baseline"] = base
    if rank == 0:
        emit(line)
    if world > 1:
        dist.destroy_process_group()


def run_serving(args):
    """The serving loop under a Poisson stream of events (submit / poll through the C ABI, host
    buffers, copies included): steps/s of the served events and p50/p99 event latency (submit
    to result). Events are replayed from a pool of distinct simulated events, each arrival with
    its own RNG seed."""
    import torch
    import torch.distributed as dist
    from paper_2403_03156_gb300 import build, fsmp, workloads

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    build.build()
    cfg = workloads.CONFIGS[args.workload]
    params, pool = workloads.make_events(args.workload, args.serve_pool, seed=args.seed + 1000 * rank,
                                         n_steps=args.mcmc_steps or None)
    n_steps = int(pool[0]["n_steps"])
    for e in pool:
        e["burn_in"] = n_steps // 5
    rate = args.rate or cfg["rate_hz"]
    ctx = fsmp.Context(dict(params, precision=fsmp.FP32_REFRESH, refresh_every=cfg.get("refresh_every", 64),
                            n_max=cfg["win_max"], device=local, max_queued=1 << 20, n_streams=args.serve_streams))
    # launch shape from timed trials on the pool of events (untimed), and the same events as one
    # device batch: the rate the serving loop would reach if every event arrived at once
    pb = concat_events(pool)
    dvc = torch.device("cuda", local)
    tb = _device_tensors(torch, pb, dvc)
    nm = int(np.diff(pb["offsets"]).max())
    tuned = None if args.no_autotune else ctx.autotune(tb, sample=32768, trial_steps=n_steps, seed=int(pb["seed"]),
                                                        n_max_hint=nm)
    Wp = len(pb["offsets"]) - 1
    batch_ms = []
    for rep in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.run_device(tb, n_steps=n_steps, burn_in=n_steps // 5, seed=int(pb["seed"]), n_max_hint=nm)
        e1.record()
        torch.cuda.synchronize()
        batch_ms.append(e0.elapsed_time(e1))
    batch_rate = Wp * n_steps / (batch_ms[-1] * 1e-3)
    del tb
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    r = serve_stream(ctx, pool, rate, args.serve_seconds, args.seed, warmup=args.warmup)
    clk = clocks.stop()
    ctx.close()
    value, t_all = r["value"], r["t_all"]
    if world > 1:
        tv = torch.tensor([r["steps"]], dtype=torch.float64, device="cuda")
        dist.all_reduce(tv, op=dist.ReduceOp.SUM)
        tmax = torch.tensor([t_all], dtype=torch.float64, device="cuda")
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        value = float(tv[0].item()) / float(tmax.item())
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": r["events"],
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_all / r["events"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "offered_rate_hz": rate, "submitted_in_s": r["submitted_in_s"],
                       "stream_s": args.serve_seconds, "events": r["events"], "waveforms": r["waveforms"],
                       "mcmc_steps_per_chain": n_steps, "completed_rate_hz": r["completed_rate_hz"],
                       "sustained": r["sustained"], "busy_retries": r["busy_retries"],
                       "timing": "host wall clock from the first submit to the last result (end to end)",
                       "kernel": "pe_kernel<float> (serving loop)", "autotune": tuned,
                       "pool_as_one_batch_steps_per_s": batch_rate, "pool_waveforms": Wp},
            "latency": {"p50_s": r["p50_s"], "p99_s": r["p99_s"], "mean_s": r["mean_s"], "max_s": r["max_s"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": r["h2d_bytes_per_event"],
                    "d2h_bytes_per_step": r["d2h_bytes_per_event"]},
            "gpu_launches": r["launches"], "clocks": clk}
    if rank == 0:
        emit(line)
    if world > 1:
        dist.destroy_process_group()


def run_lucyddm_stage(args):
    """LucyDDM (Sec. 2.3) of every waveform of the workload: waveforms/s on one GPU, the FP32
    FMA roofline of the deconvolution, the oracle on the host cores, and an end-to-end time with
    the samples copied in and the initial states copied out."""
    import torch
    from paper_2403_03156_gb300 import build, fsmp, workloads
    from oracle import oracle as orc
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    wl = workloads.make_workload(args.workload, n_waveforms=args.n_waveforms or None, seed=args.seed)
    b = wl["batch"]
    W = len(b["offsets"]) - 1
    lengths = np.diff(b["offsets"])
    n_max = int(max(lengths.max(), 64))
    ctx = fsmp.Context(dict(wl["params"], n_max=n_max, kernel=fsmp.KERNEL_PE))
    info, peaks = ctx.info(), ctx.measure_peaks()
    L_V = info["L_V"]
    t = {"samples": torch.from_numpy(b["samples"]).to(dev),
         "offsets": torch.from_numpy(b["offsets"].astype(np.int32)).to(dev),
         "t_origin_ns": torch.from_numpy(b["t_origin_ns"]).to(dev)}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        ctx.lucyddm(t, n_iter=args.lucy_iters)
    torch.cuda.synchronize(dev)
    clocks = Clocks(0)
    clocks.start()
    times = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = ctx.lucyddm(t, n_iter=args.lucy_iters)
        e1.record()
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    ms = statistics.mean(times)
    n_init = r["n_init"].cpu().numpy()
    # algorithmic FLOPs: per iteration and waveform, n outputs of w^r and n + L_V - 1 of the
    # q-hat update, L_V taps each, one FMA (2 FLOPs) per tap
    flops = 2.0 * L_V * float(np.sum(2 * lengths + L_V - 1)) * args.lucy_iters
    achieved = flops / (ms * 1e-3) / 1e12
    line = {"metric": "LucyDDM waveforms/s (%d iterations)" % args.lucy_iters, "value": W / (ms * 1e-3),
            "unit": "waveforms/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "stage": "lucyddm", "n_waveforms": W, "L_V": L_V,
                       "window_samples": [int(lengths.min()), int(np.median(lengths)), int(lengths.max())],
                       "mean_initial_pes": float(n_init.mean()), "mean_true_pes": float(wl["truth"]["N"].mean()),
                       "l2": "flushed between timed steps (256 MiB write)"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peaks["fp32_tflops"], "unit": "TFLOP/s",
                         "frac": achieved / peaks["fp32_tflops"], "traffic": None,
                         "peak_source": "measured live: fsmp_measure_peaks (FP32 FMA)",
                         "kernel": "lucy_kernel, one launch (%d waveforms)" % W},
            "gpu_launches": args.steps, "clocks": clk, "peaks_measured": peaks}
    if not args.no_e2e:
        host = torch.from_numpy(b["samples"]).pin_memory()
        e2e = []
        for i in range(1 + min(args.steps, 3)):
            t1 = time.perf_counter()
            t["samples"] = host.to(dev, non_blocking=True)
            r = ctx.lucyddm(t, n_iter=args.lucy_iters)
            outs = [r[k].cpu() for k in ("T_lo", "T_hi", "t0_init", "z_init", "n_init")]
            if i > 0:
                e2e.append(time.perf_counter() - t1)
        d2h = sum(o.numel() * o.element_size() for o in outs)
        line["e2e"] = {"value": W / statistics.mean(e2e), "unit": "waveforms/s", "h2d_bytes_per_step": int(host.numel() * 4),
                       "d2h_bytes_per_step": int(d2h), "steps": len(e2e)}
    if not args.no_cpu_baseline:
        rng = np.random.default_rng(0)
        idx = rng.permutation(W)
        t1, k = time.perf_counter(), 0
        while k < W and time.perf_counter() - t1 < args.cpu_seconds:
            i = int(idx[k])
            orc.lucyddm(wl["params"], b["samples"][b["offsets"][i]:b["offsets"][i + 1]], n_iter=args.lucy_iters)
            k += 1
        el = time.perf_counter() - t1
        line["cpu_baseline"] = {"value": k / el, "unit": "waveforms/s", "cores": 1, "kind": "oracle",
                                "sample": "%d random waveforms of %s, %d iterations, FP64, one thread, %.1f s"
                                          % (k, args.workload, args.lucy_iters, el)}
    ctx.close()
    emit(line)


def main():
    args = parse()
    if args.stage == "lucyddm":
        run_lucyddm_stage(args)
    elif args.impl == "reference":
        run_reference(args)
    elif serving_workload(args.workload):
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
