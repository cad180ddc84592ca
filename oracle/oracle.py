"""ctypes wrapper of the plain FP64 CPU oracle (``fsmp_oracle.c``).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs may import this module. The CUDA product path
never imports it, and it imports nothing from the product package.

The oracle computes the FSMP chain of arXiv 2403.03156 step by step (Sec. 2.4 and
Appendix A.1); see the header comment of ``fsmp_oracle.c`` for the readings it takes where
the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fsmp_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libfsmp_oracle.so")
_lock = threading.Lock()
_lib = None

MODE_DEFINITION = 0
MODE_INCREMENTAL = 1

F_T0_PROPOSED, F_T0_ACCEPTED, F_ACCEPTED, F_NOOP, F_T0_DISAGREE, F_DISAGREE = 1, 2, 4, 8, 16, 32
ST_CAPACITY, ST_BADDET, ST_NONFINITE, ST_DISAGREE = 1, 2, 16, 32
MAX_MIX = 8

TRACE_DTYPE = np.dtype([("la0", "<f8"), ("lu0", "<f8"), ("la", "<f8"), ("lu", "<f8"),
                        ("dnu", "<f8"), ("N", "<i4"), ("k0", "<i4"), ("jump", "<i4"),
                        ("flags", "<i4"), ("wt", "<f8"), ("we", "<f8")])
SUMMARY_DTYPE = np.dtype([("mean_N", "<f8"), ("var_N", "<f8"), ("mean_t0", "<f8"),
                          ("var_t0", "<f8"), ("mean_Q", "<f8"), ("var_Q", "<f8"),
                          ("logL", "<f8"), ("logdet", "<f8"), ("acc", "<i4", (3,)),
                          ("prop", "<i4", (3,)), ("acc_t0", "<i4"), ("prop_t0", "<i4"),
                          ("N_final", "<i4"), ("k0_final", "<i4"), ("status", "<i4"),
                          ("n_samples", "<i4"), ("lambda_hat", "<f8"), ("mean_wt", "<f8"),
                          ("var_wt", "<f8"), ("mean_we", "<f8"), ("var_we", "<f8"), ("alg_words", "<f8")])


class OrcParams(ctypes.Structure):
    _fields_ = [("dt_sample_ns", ctypes.c_double), ("grid_ns", ctypes.c_double),
                ("ser_kind", ctypes.c_int), ("ser_sigma", ctypes.c_double),
                ("ser_tau", ctypes.c_double), ("ser_under_frac", ctypes.c_double),
                ("ser_under_sigma", ctypes.c_double), ("ser_under_tau", ctypes.c_double),
                ("ser_eps", ctypes.c_double), ("phi_kind", ctypes.c_int),
                ("phi_p1", ctypes.c_double), ("phi_p2", ctypes.c_double),
                ("phi_support_ns", ctypes.c_double), ("mu_q", ctypes.c_double),
                ("sigma_q", ctypes.c_double), ("sigma_noise", ctypes.c_double),
                ("t0_lo", ctypes.c_double), ("t0_hi", ctypes.c_double),
                ("sample_t0", ctypes.c_int), ("jump_J", ctypes.c_double),
                ("n_cap", ctypes.c_int), ("prior_only", ctypes.c_int),
                ("n_mix", ctypes.c_int), ("mix_G", ctypes.c_double * MAX_MIX),
                ("mix_mu", ctypes.c_double * MAX_MIX), ("mix_sigma", ctypes.c_double * MAX_MIX)]


class OrcBatch(ctypes.Structure):
    _fields_ = [("n_waveforms", ctypes.c_int), ("samples", ctypes.c_void_p),
                ("offsets", ctypes.c_void_p), ("lambda0", ctypes.c_void_p),
                ("t_origin_ns", ctypes.c_void_p), ("T_lo", ctypes.c_void_p),
                ("T_hi", ctypes.c_void_p), ("t0_init", ctypes.c_void_p),
                ("seed", ctypes.c_uint64), ("index_base", ctypes.c_uint64),
                ("wf_ids", ctypes.c_void_p), ("n_steps", ctypes.c_int), ("burn_in", ctypes.c_int),
                ("forced", ctypes.c_void_p), ("occ", ctypes.c_void_p),
                ("occ_width", ctypes.c_int), ("occ_e", ctypes.c_void_p),
                ("z_init", ctypes.c_void_p), ("n_init", ctypes.c_void_p), ("z_stride", ctypes.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no FMA contraction) into ``oracle/_build``."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            os.makedirs(os.path.dirname(_LIB), exist_ok=True)
            tmp = _LIB + ".tmp.%d" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                                   "-o", tmp, _SRC, "-lm", "-lpthread"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        L.orc_philox4x64_10.argtypes = [ctypes.POINTER(ctypes.c_uint64)] * 3
        L.orc_philox_blocks.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_void_p]
        L.orc_step_uniforms.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_double)]
        L.orc_step_uniform_e.restype = ctypes.c_double
        L.orc_step_uniform_e.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        L.orc_ser_raw.restype = ctypes.c_double
        L.orc_ser_raw.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_double]
        L.orc_phi.restype = ctypes.c_double
        L.orc_phi.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_double]
        L.orc_ser_table.restype = ctypes.c_int
        L.orc_ser_table.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_void_p, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_double)]
        L.orc_logp_definition.restype = ctypes.c_double
        L.orc_logp_definition.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
        L.orc_logp_definition_e.restype = ctypes.c_double
        L.orc_logp_definition_e.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double)]
        L.orc_delta_nu_e.restype = ctypes.c_int
        L.orc_delta_nu_e.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_double)]
        L.orc_delta_nu.restype = ctypes.c_int
        L.orc_delta_nu.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_void_p, ctypes.c_int,
                                   ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        L.orc_run_batch.restype = ctypes.c_int
        L.orc_run_batch.argtypes = [ctypes.POINTER(OrcParams), ctypes.POINTER(OrcBatch),
                                    ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_lucyddm.restype = ctypes.c_int
        L.orc_lucyddm.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_wasserstein1.restype = ctypes.c_double
        L.orc_wasserstein1.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
        L.orc_pe_wasserstein.restype = ctypes.c_double
        L.orc_pe_wasserstein.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_lambda_mle.restype = ctypes.c_double
        L.orc_lambda_mle.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
        L.orc_run_chain_state.restype = ctypes.c_int
        L.orc_run_chain_state.argtypes = [ctypes.POINTER(OrcParams), ctypes.POINTER(OrcBatch),
                                          ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p]
        _lib = L
    return _lib


_PARAM_DEFAULTS = dict(dt_sample_ns=1.0, grid_ns=0.25, ser_kind=0, ser_sigma=1.5, ser_tau=6.0,
                       ser_under_frac=0.0, ser_under_sigma=1.0, ser_under_tau=16.0, ser_eps=1e-4,
                       phi_kind=0, phi_p1=1.5, phi_p2=20.0, phi_support_ns=4096.0, mu_q=1.0,
                       sigma_q=0.3, sigma_noise=0.06, t0_lo=30.0, t0_hi=40.0, sample_t0=1,
                       jump_J=0.25, n_cap=32, prior_only=0, n_mix=0)
_MIX_KEYS = ("mix_G", "mix_mu", "mix_sigma")


def make_params(d: dict | None = None, **kw) -> OrcParams:
    """Oracle parameter struct from a dict of model parameters (extra keys are ignored).
    The MCP mixture is given as lists ``mix_G``, ``mix_mu``, ``mix_sigma`` (n_mix = their
    length unless given)."""
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
    p = OrcParams()
    for k, v in vals.items():
        setattr(p, k, v)
    for k, v in mix.items():
        arr = getattr(p, k)
        for i, x in enumerate(v[:MAX_MIX]):
            arr[i] = x
    return p


def _ptr(a):
    return None if a is None else a.ctypes.data


def philox4x64(ctr, key):
    c = (ctypes.c_uint64 * 4)(*[int(x) for x in ctr])
    k = (ctypes.c_uint64 * 2)(*[int(x) for x in key])
    o = (ctypes.c_uint64 * 4)()
    lib().orc_philox4x64_10(c, k, o)
    return [int(x) for x in o]


def philox_blocks(key, ctrs):
    """Philox4x64-10 of each row of ``ctrs`` (shape (n, 4), uint64) under ``key``."""
    ctrs = np.ascontiguousarray(ctrs, np.uint64)
    out = np.zeros_like(ctrs)
    k = (ctypes.c_uint64 * 2)(*[int(x) for x in key])
    lib().orc_philox_blocks(k, ctrs.ctypes.data, len(ctrs), out.ctypes.data)
    return out


def step_uniforms(seed, wf_index, step):
    u = (ctypes.c_double * 8)()
    lib().orc_step_uniforms(int(seed), int(wf_index), int(step), u)
    return np.array(list(u))


def step_uniform_e(seed, wf_index, step):
    """The ninth uniform of a step: it draws the MCP component of a new PE."""
    return lib().orc_step_uniform_e(int(seed), int(wf_index), int(step))


def ser_raw(params, t):
    p = make_params(params)
    return lib().orc_ser_raw(ctypes.byref(p), float(t))


def phi(params, t):
    p = make_params(params)
    return lib().orc_phi(ctypes.byref(p), float(t))


def ser_table(params):
    """(table, peak): the peak-normalised SER on the PE grid, length L_V * R."""
    p = make_params(params)
    n = lib().orc_ser_table(ctypes.byref(p), None, 0, None)
    if n < 0:
        raise ValueError("invalid SER parameters")
    out = np.zeros(n, np.float64)
    peak = ctypes.c_double()
    lib().orc_ser_table(ctypes.byref(p), out.ctypes.data, n, ctypes.byref(peak))
    return out, peak.value


def logp_definition(params, w, j, e=None):
    """log p(w|z), log|Sigma|, quadratic form; e: the PEs' MCP components (None: all 0)."""
    p = make_params(params)
    w = np.ascontiguousarray(w, np.float32)
    j = np.ascontiguousarray(j, np.int32)
    ld, q = ctypes.c_double(), ctypes.c_double()
    if e is None:
        r = lib().orc_logp_definition(ctypes.byref(p), w.ctypes.data, len(w), j.ctypes.data, len(j),
                                      ctypes.byref(ld), ctypes.byref(q))
    else:
        e = np.ascontiguousarray(e, np.int32)
        r = lib().orc_logp_definition_e(ctypes.byref(p), w.ctypes.data, len(w), j.ctypes.data,
                                        e.ctypes.data, len(j), ctypes.byref(ld), ctypes.byref(q))
    return r, ld.value, q.value


def lambda_mle(hist, lambda0):
    """lambda_FSMP of an N histogram (counts h[0..n_max]) by Eq. (reduce-mu0)."""
    h = np.ascontiguousarray(hist, np.float64)
    return lib().orc_lambda_mle(h.ctypes.data, len(h) - 1, float(lambda0))


def wasserstein1(a, b):
    """1-Wasserstein distance between the empirical distributions of a and b (1-D)."""
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    return lib().orc_wasserstein1(a.ctypes.data, len(a), b.ctypes.data, len(b))


def pe_wasserstein(v):
    """The convergence scalar of a PE sequence (Sec. 3.2): W1 from {0} and v to {0}."""
    v = np.ascontiguousarray(v, np.float64)
    return lib().orc_pe_wasserstein(v.ctypes.data if len(v) else None, len(v))


def delta_nu(params, w, j, kind, k=0, jp=0, mode=MODE_INCREMENTAL, e=None, ep=0):
    """Delta nu of one proposal (kind 0 birth of jp, 1 death of slot k, 2 update k -> jp);
    e: the PEs' MCP components (None: all 0), ep: the component of the new PE."""
    p = make_params(params)
    w = np.ascontiguousarray(w, np.float32)
    N = len(j)
    jj = np.zeros(max(N, 1), np.int32)
    jj[:N] = np.asarray(j, np.int32)
    ee = np.zeros(max(N, 1), np.int32)
    if e is not None:
        ee[:N] = np.asarray(e, np.int32)
    out = ctypes.c_double()
    rc = lib().orc_delta_nu_e(ctypes.byref(p), w.ctypes.data, len(w), jj.ctypes.data, ee.ctypes.data, N,
                              int(kind), int(k), int(jp), int(ep), int(mode), ctypes.byref(out))
    if rc != 0:
        raise ValueError("orc_delta_nu failed: %d" % rc)
    return out.value


class _BatchKeep:
    """Holds the numpy arrays referenced by an OrcBatch alive."""

    def __init__(self, batch):
        def f(name, dt):
            v = batch.get(name)
            return None if v is None else np.ascontiguousarray(v, dt)

        self.samples = f("samples", np.float32)
        self.offsets = f("offsets", np.int32)
        self.lambda0 = f("lambda0", np.float64)
        self.t_origin = f("t_origin_ns", np.float64)
        self.T_lo = f("T_lo", np.int32)
        self.T_hi = f("T_hi", np.int32)
        self.t0_init = f("t0_init", np.float64)
        self.forced = f("forced", np.uint8)
        self.wf_ids = f("wf_ids", np.uint64)
        self.z_init = f("z_init", np.int32)
        self.n_init = f("n_init", np.int32)
        b = OrcBatch()
        b.n_waveforms = len(self.offsets) - 1
        b.samples = _ptr(self.samples)
        b.offsets = _ptr(self.offsets)
        b.lambda0 = _ptr(self.lambda0)
        b.t_origin_ns = _ptr(self.t_origin)
        b.T_lo = _ptr(self.T_lo)
        b.T_hi = _ptr(self.T_hi)
        b.t0_init = _ptr(self.t0_init)
        b.seed = int(batch.get("seed", 0))
        b.index_base = int(batch.get("index_base", 0))
        b.wf_ids = _ptr(self.wf_ids)
        b.n_steps = int(batch["n_steps"])
        b.burn_in = int(batch.get("burn_in", 0))
        b.forced = _ptr(self.forced)
        if self.z_init is not None:
            b.z_init = _ptr(self.z_init)
            b.n_init = _ptr(self.n_init)
            b.z_stride = int(self.z_init.shape[1]) if self.z_init.ndim == 2 else int(batch["z_stride"])
        self.occ = None
        if batch.get("occ_width"):
            self.occ = np.zeros((b.n_waveforms, int(batch["occ_width"])), np.float64)
            b.occ = self.occ.ctypes.data
            b.occ_width = int(batch["occ_width"])
        self.occ_e = None
        if batch.get("occ_e"):
            self.occ_e = np.zeros((b.n_waveforms, int(batch["occ_e"])), np.float64)
            b.occ_e = self.occ_e.ctypes.data
        self.b = b


def run_batch(params, batch, mode=MODE_INCREMENTAL, n_threads=1, trace=False):
    """Run every chain of ``batch`` (a dict of arrays, see ``orc_batch``).

    Returns (summaries, trace) with ``trace`` of shape (n_waveforms, n_steps) or None, then
    the PE-time histogram if ``batch["occ_width"]`` is set, then the per-component PE counts
    if ``batch["occ_e"]`` (the number of components) is set.
    """
    p = make_params(params)
    keep = _BatchKeep(batch)
    W = keep.b.n_waveforms
    out = np.zeros(W, SUMMARY_DTYPE)
    tr = np.zeros((W, keep.b.n_steps), TRACE_DTYPE) if trace else None
    rc = lib().orc_run_batch(ctypes.byref(p), ctypes.byref(keep.b), int(mode), int(n_threads),
                             out.ctypes.data, None if tr is None else tr.ctypes.data)
    if rc != 0:
        raise ValueError("orc_run_batch failed: %d" % rc)
    if keep.occ_e is not None:
        return out, tr, keep.occ, keep.occ_e
    if keep.occ is not None:
        return out, tr, keep.occ
    return out, tr


def run_chain_state(params, batch, mode=MODE_INCREMENTAL):
    """Run waveform 0 of ``batch`` and return its summary, trace and final state."""
    p = make_params(params)
    keep = _BatchKeep(batch)
    n = int(keep.offsets[1] - keep.offsets[0])
    out = np.zeros(1, SUMMARY_DTYPE)
    tr = np.zeros(keep.b.n_steps, TRACE_DTYPE)
    lst = np.zeros(int(p.n_cap) + 1, np.int32)
    lst_e = np.zeros(int(p.n_cap) + 1, np.int32)
    N = np.zeros(1, np.int32)
    k0 = np.zeros(1, np.int32)
    sinv = np.zeros((n, n), np.float64)
    y = np.zeros(n, np.float64)
    ld = np.zeros(1, np.float64)
    rc = lib().orc_run_chain_state(ctypes.byref(p), ctypes.byref(keep.b), int(mode),
                                   out.ctypes.data, tr.ctypes.data, lst.ctypes.data, N.ctypes.data,
                                   k0.ctypes.data, sinv.ctypes.data, y.ctypes.data, ld.ctypes.data,
                                   lst_e.ctypes.data)
    if rc != 0:
        raise ValueError("orc_run_chain_state failed: %d" % rc)
    return dict(summary=out[0], trace=tr, z=lst[:N[0]].copy(), e=lst_e[:N[0]].copy(), N=int(N[0]),
                k0=int(k0[0]), sinv=sinv, y=y, logdet=float(ld[0]))


def lucyddm(params, w, n_iter=2000, thresh=0.1, t_origin=0.0, z_cap=None):
    """LucyDDM of one waveform (Sec. 2.3). Returns dict(q, z, n_z, T_lo, T_hi, t0): q-hat for
    tau = -L_V+1 .. n-1, the initial PE grid indices, the solution space and t0."""
    p = make_params(params)
    w = np.ascontiguousarray(w, np.float32)
    n = len(w)
    nq_max = n + 4096
    q = np.zeros(nq_max, np.float64)
    cap = int(z_cap if z_cap is not None else n + 4096)
    z = np.zeros(max(cap, 1), np.int32)
    nz, tlo, thi = np.zeros(1, np.int32), np.zeros(1, np.int32), np.zeros(1, np.int32)
    t0 = np.zeros(1, np.float64)
    LV = lib().orc_lucyddm(ctypes.byref(p), w.ctypes.data, n, float(t_origin), int(n_iter), float(thresh),
                           q.ctypes.data, z.ctypes.data, cap, nz.ctypes.data, tlo.ctypes.data, thi.ctypes.data,
                           t0.ctypes.data)
    if LV < 0:
        raise ValueError("orc_lucyddm failed: %d" % LV)
    return dict(q=q[:n + LV - 1].copy(), L_V=LV, z=z[:min(int(nz[0]), cap)].copy(), n_z=int(nz[0]),
                T_lo=int(tlo[0]), T_hi=int(thi[0]), t0=float(t0[0]))
