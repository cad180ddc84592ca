"""Python binding of libfsmp.so (include/fsmp.h): argument marshalling only.

Every step of the chain runs in the library's CUDA kernels. This module loads the in-tree
library and raises if it is missing; there is no CPU fallback. PyTorch tensors may be passed
to the device-resident entry point (``run_device``); PyTorch is used only for device memory
and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK, ERR_INVALID, ERR_CUDA, ERR_NOMEM, ERR_BUSY, ERR_TIMEOUT, ERR_CLOSED = 0, -1, -2, -3, -4, -5, -6
ST_CAPACITY, ST_BADDET, ST_DRIFT, ST_INVALID, ST_NONFINITE = 1, 2, 4, 8, 16
FP64, FP32_REFRESH = 0, 1
KERNEL_AUTO, KERNEL_SMEM, KERNEL_GLOBAL, KERNEL_PLAIN, KERNEL_PE = 0, 1, 2, 3, 4

SUMMARY_DTYPE = np.dtype([("mean_N", "<f8"), ("var_N", "<f8"), ("mean_t0", "<f8"),
                          ("var_t0", "<f8"), ("mean_Q", "<f8"), ("var_Q", "<f8"),
                          ("logL", "<f8"), ("logdet", "<f8"), ("drift_max", "<f8"),
                          ("alg_bytes", "<f8"), ("lambda_hat", "<f8"), ("mean_wt", "<f8"), ("var_wt", "<f8"),
                          ("mean_we", "<f8"), ("var_we", "<f8"), ("acc", "<i4", (3,)), ("prop", "<i4", (3,)),
                          ("acc_t0", "<i4"), ("prop_t0", "<i4"), ("N_final", "<i4"),
                          ("k0_final", "<i4"), ("status", "<i4"), ("n_samples", "<i4"),
                          ("n_refresh", "<i4"), ("reserved", "<i4")])
TRACE_DTYPE = np.dtype([("la0", "<f8"), ("lu0", "<f8"), ("la", "<f8"), ("lu", "<f8"),
                        ("dnu", "<f8"), ("N", "<i4"), ("k0", "<i4"), ("jump", "<i4"),
                        ("flags", "<i4")])

_c_double, _c_int, _c_u64, _vp = ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p
MAX_MIX = 8  # FSMP_MAX_MIX


class Params(ctypes.Structure):
    _fields_ = [("dt_sample_ns", _c_double), ("grid_ns", _c_double), ("ser_kind", _c_int),
                ("ser_sigma", _c_double), ("ser_tau", _c_double), ("ser_under_frac", _c_double),
                ("ser_under_sigma", _c_double), ("ser_under_tau", _c_double),
                ("ser_eps", _c_double), ("phi_kind", _c_int), ("phi_p1", _c_double),
                ("phi_p2", _c_double), ("phi_support_ns", _c_double), ("mu_q", _c_double),
                ("sigma_q", _c_double), ("sigma_noise", _c_double), ("t0_lo", _c_double),
                ("t0_hi", _c_double), ("sample_t0", _c_int), ("jump_J", _c_double),
                ("n_cap", _c_int), ("n_max", _c_int), ("precision", _c_int),
                ("refresh_every", _c_int), ("drift_tol", _c_double), ("kernel", _c_int),
                ("threads_per_chain", _c_int), ("device_mem_budget", ctypes.c_size_t),
                ("device", _c_int), ("max_queued", _c_int), ("n_streams", _c_int),
                ("pe_tile", _c_int), ("pe_ctas_per_sm", _c_int), ("pe_lanes", _c_int),
                ("n_mix", _c_int), ("mix_G", _c_double * MAX_MIX), ("mix_mu", _c_double * MAX_MIX),
                ("mix_sigma", _c_double * MAX_MIX)]


class Batch(ctypes.Structure):
    _fields_ = [("request_id", _c_u64), ("seed", _c_u64), ("index_base", _c_u64),
                ("n_waveforms", _c_int), ("n_steps", _c_int), ("burn_in", _c_int),
                ("record_trace", _c_int), ("samples", _vp), ("offsets", _vp), ("lambda0", _vp),
                ("t_origin_ns", _vp), ("T_lo", _vp), ("T_hi", _vp), ("t0_init", _vp),
                ("wf_ids", _vp)]


class Result(ctypes.Structure):
    _fields_ = [("request_id", _c_u64), ("n_waveforms", _c_int), ("status", _c_int),
                ("summaries", _vp), ("trace", _vp), ("latency_s", _c_double)]


class DeviceBatch(ctypes.Structure):
    _fields_ = [("n_waveforms", _c_int), ("n_steps", _c_int), ("burn_in", _c_int),
                ("n_max_hint", _c_int), ("seed", _c_u64), ("index_base", _c_u64),
                ("samples", _vp), ("offsets", _vp), ("lambda0", _vp), ("t_origin_ns", _vp),
                ("T_lo", _vp), ("T_hi", _vp), ("t0_init", _vp), ("wf_ids", _vp), ("out", _vp),
                ("trace", _vp), ("z_init", _vp), ("n_init", _vp), ("z_stride", _c_int),
                ("pe_hist", _vp), ("pe_hist_width", _c_int)]


class LucyBatch(ctypes.Structure):
    _fields_ = [("n_waveforms", _c_int), ("n_max_hint", _c_int), ("samples", _vp), ("offsets", _vp),
                ("t_origin_ns", _vp), ("n_iter", _c_int), ("thresh", _c_double), ("q_out", _vp),
                ("T_lo", _vp), ("T_hi", _vp), ("t0_init", _vp), ("z_init", _vp), ("n_init", _vp),
                ("z_stride", _c_int), ("status", _vp)]


class Tune(ctypes.Structure):
    _fields_ = [("pe_tile", _c_int), ("chains_per_cta", _c_int), ("ctas_per_sm", _c_int), ("n_tried", _c_int),
                ("best_steps_per_s", _c_double), ("default_steps_per_s", _c_double),
                ("lanes_per_chain", _c_int)]


class Info(ctypes.Structure):
    _fields_ = [("device", _c_int), ("sm_count", _c_int), ("smem_per_block_optin", _c_int),
                ("ser_len", _c_int), ("R", _c_int), ("L_V", _c_int), ("n_smem_max", _c_int),
                ("threads_per_chain", _c_int), ("ctas_per_sm", _c_int),
                ("scratch_bytes", ctypes.c_size_t), ("name", ctypes.c_char * 64),
                ("n_launches", ctypes.c_longlong)]


EXPORTS = ["fsmp_create", "fsmp_submit", "fsmp_poll", "fsmp_destroy", "fsmp_run_device",
           "fsmp_get_tables", "fsmp_get_info", "fsmp_philox_blocks", "fsmp_strerror",
           "fsmp_last_error", "fsmp_measure_peaks", "fsmp_run_device_noalloc", "fsmp_autotune",
           "fsmp_gelman_rubin", "fsmp_gelman_diag", "fsmp_lucyddm", "fsmp_lambda_mle"]

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libfsmp.so. Raises if it is missing (no fallback of any kind)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libfsmp.so is not built (%s); run paper_2403_03156_gb300.build.build()" % path)
        _build.build()
    L = ctypes.CDLL(path)
    L.fsmp_create.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(_vp)]
    L.fsmp_submit.argtypes = [_vp, ctypes.POINTER(Batch)]
    L.fsmp_poll.argtypes = [_vp, ctypes.POINTER(Result), _c_int, _c_int]
    L.fsmp_destroy.argtypes = [_vp]
    L.fsmp_run_device.argtypes = [_vp, ctypes.POINTER(DeviceBatch), _vp]
    L.fsmp_run_device_noalloc.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(DeviceBatch), _vp]
    L.fsmp_autotune.argtypes = [_vp, ctypes.POINTER(DeviceBatch), _c_int, _c_int, ctypes.POINTER(Tune)]
    L.fsmp_gelman_rubin.argtypes = [_vp, _c_int, _c_int, ctypes.POINTER(_c_double)]
    L.fsmp_gelman_diag.argtypes = [_vp, _c_int, _c_int, _c_double, ctypes.POINTER(_c_double),
                                   ctypes.POINTER(_c_double)]
    L.fsmp_lucyddm.argtypes = [_vp, ctypes.POINTER(LucyBatch), _vp]
    L.fsmp_lambda_mle.argtypes = [_vp, _vp, _c_int, _c_int, _vp, _c_int, _vp]
    L.fsmp_get_tables.argtypes = [_vp, _vp, _c_int, ctypes.POINTER(_c_int), _c_int, _c_int, _vp, _vp]
    L.fsmp_get_info.argtypes = [_vp, ctypes.POINTER(Info)]
    L.fsmp_philox_blocks.argtypes = [_vp, ctypes.POINTER(_c_u64), _vp, _c_int, _vp]
    L.fsmp_measure_peaks.argtypes = [_vp, ctypes.POINTER(_c_double), ctypes.POINTER(_c_double),
                                     ctypes.POINTER(_c_double)]
    L.fsmp_strerror.restype = ctypes.c_char_p
    L.fsmp_strerror.argtypes = [_c_int]
    L.fsmp_last_error.restype = ctypes.c_char_p
    L.fsmp_last_error.argtypes = []
    for name in EXPORTS:
        if name not in ("fsmp_strerror", "fsmp_last_error"):
            getattr(L, name).restype = _c_int
    _lib = L
    return L


def strerror(code: int) -> str:
    return load().fsmp_strerror(int(code)).decode()


class FsmpError(RuntimeError):
    def __init__(self, code, what):
        detail = load().fsmp_last_error().decode()
        super().__init__("%s: %s (%d)%s" % (what, strerror(code), code, " -- " + detail if detail else ""))
        self.code = code


def _check(rc, what):
    if rc != OK:
        raise FsmpError(rc, what)
    return rc


_PARAM_DEFAULTS = dict(dt_sample_ns=1.0, grid_ns=0.25, ser_kind=0, ser_sigma=1.5, ser_tau=6.0,
                       ser_under_frac=0.0, ser_under_sigma=1.0, ser_under_tau=16.0, ser_eps=1e-4,
                       phi_kind=0, phi_p1=1.5, phi_p2=20.0, phi_support_ns=4096.0, mu_q=1.0,
                       sigma_q=0.3, sigma_noise=0.06, t0_lo=30.0, t0_hi=40.0, sample_t0=1,
                       jump_J=0.25, n_cap=32, n_max=1024, precision=FP64, refresh_every=64,
                       drift_tol=0.0, kernel=KERNEL_AUTO, threads_per_chain=0,
                       device_mem_budget=0, device=0, max_queued=0, n_streams=0, pe_tile=0,
                       pe_ctas_per_sm=0, pe_lanes=0, n_mix=0)
_MIX_KEYS = ("mix_G", "mix_mu", "mix_sigma")


def make_params(d: dict | None = None, **kw) -> Params:
    """fsmp_params from a dict (unknown keys are ignored). The MCP charge mixture is given as
    lists ``mix_G``, ``mix_mu``, ``mix_sigma``; n_mix defaults to their length."""
    vals = dict(_PARAM_DEFAULTS)
    mix = {}
    for src in (d or {}, kw):
        for k, v in src.items():
            if k in vals:
                vals[k] = v
            elif k in _MIX_KEYS and v is not None:
                mix[k] = [float(x) for x in v]
    if mix and not vals["n_mix"]:
        vals["n_mix"] = len(mix["mix_G"])
    if len(mix.get("mix_G", ())) > MAX_MIX:
        raise ValueError("at most %d mixture components" % MAX_MIX)
    p = Params()
    for k, v in vals.items():
        setattr(p, k, v)
    for k, v in mix.items():
        arr = getattr(p, k)
        for i, x in enumerate(v):
            arr[i] = x
    return p


def _np(a, dt):
    return None if a is None else np.ascontiguousarray(a, dt)


def _ptr(a):
    return None if a is None else a.ctypes.data


class Context:
    """One fsmp_ctx: tables on the GPU, scratch, and the serving loop."""

    def __init__(self, params: dict | None = None, **kw):
        L = load()
        self.params = make_params(params, **kw)
        h = _vp()
        _check(L.fsmp_create(ctypes.byref(self.params), ctypes.byref(h)), "fsmp_create")
        self.h = h
        self._keep = {}

    def close(self):
        if getattr(self, "h", None):
            _check(load().fsmp_destroy(self.h), "fsmp_destroy")
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- serving API
    def submit(self, batch: dict, request_id: int = 0, record_trace: bool = False) -> int:
        """Queue a host batch (dict of numpy arrays, as produced by workloads). Returns the
        status code (OK, ERR_BUSY, ...); raises on ERR_INVALID / ERR_CUDA."""
        b = Batch()
        arrs = dict(samples=_np(batch["samples"], np.float32), offsets=_np(batch["offsets"], np.int32),
                    lambda0=_np(batch["lambda0"], np.float64),
                    t_origin=_np(batch.get("t_origin_ns"), np.float64),
                    T_lo=_np(batch.get("T_lo"), np.int32), T_hi=_np(batch.get("T_hi"), np.int32),
                    t0_init=_np(batch.get("t0_init"), np.float64),
                    wf_ids=_np(batch.get("wf_ids"), np.uint64))
        b.request_id = int(request_id)
        b.seed = int(batch.get("seed", 0))
        b.index_base = int(batch.get("index_base", 0))
        b.n_waveforms = len(arrs["offsets"]) - 1
        b.n_steps = int(batch["n_steps"])
        b.burn_in = int(batch.get("burn_in", 0))
        b.record_trace = 1 if record_trace else 0
        b.samples, b.offsets, b.lambda0 = _ptr(arrs["samples"]), _ptr(arrs["offsets"]), _ptr(arrs["lambda0"])
        b.t_origin_ns, b.T_lo, b.T_hi = _ptr(arrs["t_origin"]), _ptr(arrs["T_lo"]), _ptr(arrs["T_hi"])
        b.t0_init, b.wf_ids = _ptr(arrs["t0_init"]), _ptr(arrs["wf_ids"])
        rc = load().fsmp_submit(self.h, ctypes.byref(b))
        if rc in (ERR_INVALID, ERR_CUDA):
            raise FsmpError(rc, "fsmp_submit")
        return rc

    def poll(self, max_results: int = 64, timeout_ms: int = 0):
        """Finished requests as a list of dicts (summaries / trace copied to numpy)."""
        res = (Result * max(1, max_results))()
        k = load().fsmp_poll(self.h, res, int(max_results), int(timeout_ms))
        if k < 0:
            raise FsmpError(k, "fsmp_poll")
        out = []
        for i in range(k):
            r = res[i]
            W = r.n_waveforms
            summ = None
            if r.summaries:
                buf = (ctypes.c_char * (W * SUMMARY_DTYPE.itemsize)).from_address(r.summaries)
                summ = np.frombuffer(buf, SUMMARY_DTYPE).copy()
            tr = None
            if r.trace:
                n = W * int(self._keep.get(("nsteps", r.request_id), 0))
                if n:
                    buf = (ctypes.c_char * (n * TRACE_DTYPE.itemsize)).from_address(r.trace)
                    tr = np.frombuffer(buf, TRACE_DTYPE).copy().reshape(W, -1)
            out.append(dict(request_id=r.request_id, status=r.status, summaries=summ, trace=tr,
                            latency_s=r.latency_s))
        return out

    def run(self, batch: dict, record_trace: bool = False, request_id: int = 0, timeout_s: float = 600.0):
        """Submit one host batch and wait for it (convenience for tests)."""
        self._keep[("nsteps", request_id)] = int(batch["n_steps"])
        rc = self.submit(batch, request_id=request_id, record_trace=record_trace)
        _check(rc, "fsmp_submit")
        got = self.poll(1, int(timeout_s * 1000))
        if not got:
            raise FsmpError(ERR_TIMEOUT, "fsmp_poll")
        r = got[0]
        _check(r["status"], "request")
        return r["summaries"], r["trace"]

    # ---------------------------------------------------------------- device-resident API
    def run_device(self, dev: dict, n_steps: int, burn_in: int = 0, seed: int = 0, index_base: int = 0,
                   n_max_hint: int = 0, stream=None):
        """Enqueue chains on device-resident tensors (dict of torch CUDA tensors: samples f32,
        offsets i32, lambda0 f64, optional t_origin_ns f64, T_lo/T_hi i32, t0_init f64,
        wf_ids i64, out (uint8 buffer of n * summary bytes), optional trace buffer)."""
        def p(name):
            t = dev.get(name)
            return None if t is None else t.data_ptr()

        b = DeviceBatch()
        b.n_waveforms = int(dev["offsets"].numel()) - 1
        b.n_steps, b.burn_in, b.n_max_hint = int(n_steps), int(burn_in), int(n_max_hint)
        b.seed, b.index_base = int(seed), int(index_base)
        b.samples, b.offsets, b.lambda0, b.t_origin_ns = p("samples"), p("offsets"), p("lambda0"), p("t_origin_ns")
        b.T_lo, b.T_hi, b.t0_init, b.wf_ids = p("T_lo"), p("T_hi"), p("t0_init"), p("wf_ids")
        b.out, b.trace = p("out"), p("trace")
        _set_z_init(b, dev)
        st = None if stream is None else int(stream.cuda_stream)
        _check(load().fsmp_run_device(self.h, ctypes.byref(b), st), "fsmp_run_device")

    def lucyddm(self, dev: dict, n_iter: int = 2000, thresh: float = 0.1, z_stride: int = 0, with_q: bool = False,
                n_max_hint: int = 0, stream=None) -> dict:
        """fsmp_lucyddm (Sec. 2.3) on device tensors (samples f32, offsets i32, optional
        t_origin_ns f64). Returns torch tensors on the same device: T_lo, T_hi (i32), t0_init
        (f64), z_init (i32, [n, z_stride]; z_stride defaults to n_cap), n_init, status (i32)
        and, with ``with_q``, q (f32, waveform i at offsets[i] + i (L_V - 1)) -- ready to pass
        to run_device as an initial state."""
        import torch
        W = int(dev["offsets"].numel()) - 1
        zs = int(z_stride or self.params.n_cap)
        d = dev["offsets"].device
        out = dict(T_lo=torch.zeros(W, dtype=torch.int32, device=d), T_hi=torch.zeros(W, dtype=torch.int32, device=d),
                   t0_init=torch.zeros(W, dtype=torch.float64, device=d),
                   z_init=torch.zeros((W, zs), dtype=torch.int32, device=d),
                   n_init=torch.zeros(W, dtype=torch.int32, device=d), status=torch.zeros(W, dtype=torch.int32, device=d))
        if with_q:
            L_V = self.info()["L_V"]
            out["q"] = torch.zeros(int(dev["samples"].numel()) + W * (L_V - 1), dtype=torch.float32, device=d)
        b = LucyBatch()
        b.n_waveforms, b.n_max_hint = W, int(n_max_hint)
        b.samples, b.offsets = dev["samples"].data_ptr(), dev["offsets"].data_ptr()
        b.t_origin_ns = dev["t_origin_ns"].data_ptr() if dev.get("t_origin_ns") is not None else None
        b.n_iter, b.thresh = int(n_iter), float(thresh)
        b.q_out = out["q"].data_ptr() if with_q else None
        b.T_lo, b.T_hi, b.t0_init = out["T_lo"].data_ptr(), out["T_hi"].data_ptr(), out["t0_init"].data_ptr()
        b.z_init, b.n_init, b.z_stride = out["z_init"].data_ptr(), out["n_init"].data_ptr(), zs
        b.status = out["status"].data_ptr()
        st = None if stream is None else int(stream.cuda_stream)
        _check(load().fsmp_lucyddm(self.h, ctypes.byref(b), st), "fsmp_lucyddm")
        return out

    def autotune(self, dev: dict, sample: int = 8192, trial_steps: int = 128, n_steps: int = 0, seed: int = 0,
                 n_max_hint: int = 0) -> dict:
        """fsmp_autotune on device tensors laid out as for run_device: times trial runs of
        the first `sample` waveforms in candidate launch shapes and keeps the fastest."""
        b = _device_batch(dev, n_steps, 0, seed, 0, n_max_hint)
        t = Tune()
        _check(load().fsmp_autotune(self.h, ctypes.byref(b), int(sample), int(trial_steps), ctypes.byref(t)),
               "fsmp_autotune")
        return {k: getattr(t, k) for k, _ in Tune._fields_}

    # ---------------------------------------------------------------- testing aids
    def tables(self, d_lo: int = 0, count: int = 0):
        n = _c_int()
        _check(load().fsmp_get_tables(self.h, None, 0, ctypes.byref(n), 0, 0, None, None), "fsmp_get_tables")
        ser = np.zeros(n.value, np.float64)
        phi = np.zeros(count, np.float64)
        lphi = np.zeros(count, np.float64)
        _check(load().fsmp_get_tables(self.h, ser.ctypes.data, n.value, ctypes.byref(n), int(d_lo), int(count),
                                      phi.ctypes.data if count else None,
                                      lphi.ctypes.data if count else None), "fsmp_get_tables")
        return ser, phi, lphi

    def info(self) -> dict:
        i = Info()
        _check(load().fsmp_get_info(self.h, ctypes.byref(i)), "fsmp_get_info")
        d = {k: getattr(i, k) for k, _ in Info._fields_}
        d["name"] = i.name.decode()
        return d

    def measure_peaks(self) -> dict:
        a, b, c = _c_double(), _c_double(), _c_double()
        _check(load().fsmp_measure_peaks(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "fsmp_measure_peaks")
        return dict(smem_gbs=a.value, fp64_tflops=b.value, fp32_tflops=c.value)

    def lambda_mle(self, hist, lambda0, lanes: int = 32) -> np.ndarray:
        """fsmp_lambda_mle: lambda_FSMP of each row of ``hist`` (counts of N = 0 .. n_max) on
        the GPU, by the device function the chains end with."""
        h = np.ascontiguousarray(np.atleast_2d(hist), np.int32)
        lam = np.ascontiguousarray(np.broadcast_to(np.asarray(lambda0, np.float64), (h.shape[0],)))
        out = np.zeros(h.shape[0], np.float64)
        _check(load().fsmp_lambda_mle(self.h, h.ctypes.data, h.shape[0], h.shape[1] - 1, lam.ctypes.data, int(lanes),
                                      out.ctypes.data), "fsmp_lambda_mle")
        return out

    def philox_blocks(self, key, ctrs):
        ctrs = np.ascontiguousarray(ctrs, np.uint64)
        out = np.zeros_like(ctrs)
        k = (_c_u64 * 2)(*[int(x) for x in key])
        _check(load().fsmp_philox_blocks(self.h, k, ctrs.ctypes.data, len(ctrs), out.ctypes.data),
               "fsmp_philox_blocks")
        return out


def _device_batch(dev, n_steps, burn_in, seed, index_base, n_max_hint):
    def p(name):
        t = dev.get(name)
        return None if t is None else t.data_ptr()

    b = DeviceBatch()
    b.n_waveforms = int(dev["offsets"].numel()) - 1
    b.n_steps, b.burn_in, b.n_max_hint = int(n_steps), int(burn_in), int(n_max_hint)
    b.seed, b.index_base = int(seed), int(index_base)
    b.samples, b.offsets, b.lambda0, b.t_origin_ns = p("samples"), p("offsets"), p("lambda0"), p("t_origin_ns")
    b.T_lo, b.T_hi, b.t0_init, b.wf_ids = p("T_lo"), p("T_hi"), p("t0_init"), p("wf_ids")
    b.out, b.trace = p("out"), p("trace")
    _set_z_init(b, dev)
    return b


def _set_z_init(b, dev):
    """Initial-state fields of a DeviceBatch from dev["z_init"] ([n, z_stride] i32) and
    dev["n_init"] (i32), and the PE-time histogram dev["pe_hist"] ([n, width] i32), if given."""
    h = dev.get("pe_hist")
    if h is not None:  # [n, width] int32 / uint32 counts
        b.pe_hist, b.pe_hist_width = h.data_ptr(), int(h.shape[1])
    z = dev.get("z_init")
    if z is None:
        return
    b.z_init, b.n_init = z.data_ptr(), dev["n_init"].data_ptr()
    b.z_stride = int(z.shape[1]) if z.dim() == 2 else int(dev["z_stride"])


def run_device_noalloc(params: dict, dev: dict, n_steps: int, burn_in: int = 0, seed: int = 0,
                       index_base: int = 0, n_max_hint: int = 0, stream=None):
    """Run chains on device tensors (as ``Context.run_device``) without allocating device
    memory, for callers that cannot allocate: code under a framework allocator that owns all
    device memory, or a service that forbids allocation after start-up. Needs no Context; its
    scratch is one static 64 MiB device array shared by all calls: calls on one stream run in
    order, calls on different streams must not overlap on the GPU. FP32 mode only, windows of at most 256 samples, n_cap at most 64. The first
    call on a device, and the first after the model parameters change, synchronise ``stream``
    once; make such a call before any stream capture."""
    prm = make_params(params)
    b = _device_batch(dev, n_steps, burn_in, seed, index_base, n_max_hint)
    st = None if stream is None else int(stream.cuda_stream)
    _check(load().fsmp_run_device_noalloc(ctypes.byref(prm), ctypes.byref(b), st), "fsmp_run_device_noalloc")


RHAT_N, RHAT_T0, RHAT_Q, RHAT_WT, RHAT_WE = 0, 1, 2, 3, 4


def gelman_rubin(summaries: np.ndarray, field: int = RHAT_N) -> float:
    """fsmp_gelman_rubin over the chains of one waveform (a SUMMARY_DTYPE array)."""
    s = np.ascontiguousarray(summaries, SUMMARY_DTYPE)
    r = _c_double()
    _check(load().fsmp_gelman_rubin(s.ctypes.data, len(s), int(field), ctypes.byref(r)), "fsmp_gelman_rubin")
    return r.value


def gelman_diag(summaries: np.ndarray, field: int = RHAT_N, confidence: float = 0.9):
    """fsmp_gelman_diag over the chains of one waveform: (R, its upper confidence limit), the
    degrees-of-freedom corrected potential scale reduction (Sec. 3.2 plots the 90 % limit)."""
    s = np.ascontiguousarray(summaries, SUMMARY_DTYPE)
    r, u = _c_double(), _c_double()
    _check(load().fsmp_gelman_diag(s.ctypes.data, len(s), int(field), float(confidence), ctypes.byref(r),
                                   ctypes.byref(u)), "fsmp_gelman_diag")
    return r.value, u.value


def summaries_from_bytes(buf) -> np.ndarray:
    """View a uint8 buffer (e.g. a CPU copy of the ``out`` tensor) as summaries."""
    return np.frombuffer(np.ascontiguousarray(buf).tobytes(), SUMMARY_DTYPE)


def traces_from_bytes(buf, n_waveforms) -> np.ndarray:
    return np.frombuffer(np.ascontiguousarray(buf).tobytes(), TRACE_DTYPE).reshape(n_waveforms, -1)
