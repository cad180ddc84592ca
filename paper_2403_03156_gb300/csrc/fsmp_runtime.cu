// fsmp_runtime.cu -- host runtime behind the C ABI of include/fsmp.h: context creation
// (model tables computed on the GPU), launch shapes, the device-resident entry point, and
// the serving loop (a scheduler thread that admits submitted requests by device memory,
// packs them into persistent-kernel launches on a pool of streams, and hands finished
// requests to fsmp_poll).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "fsmp_internal.h"

using namespace fsmp;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

thread_local char g_last_error[256] = "";

void set_error(const char* what, const char* detail, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s (fsmp_runtime.cu:%d)", what, detail, line);
}

#define CK(call)                                               \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) {                                   \
      set_error(#call, cudaGetErrorString(e_), __LINE__);      \
      return FSMP_ERR_CUDA;                                    \
    }                                                          \
  } while (0)
#define FAIL(code, msg)                   \
  do {                                    \
    set_error("rejected", msg, __LINE__); \
    return code;                          \
  } while (0)

// One submitted request (host copy of its inputs; results once finished).
struct Request {
  uint64_t id = 0, seed = 0, index_base = 0;
  int W = 0, n_steps = 0, burn_in = 0, record_trace = 0, n_max = 0;
  std::vector<float> samples;
  std::vector<int32_t> offsets, T_lo, T_hi;
  std::vector<double> lambda0, t_origin, t0_init;
  std::vector<uint64_t> wf_ids;
  std::vector<fsmp_summary> out;
  std::vector<fsmp_trace> trace;
  size_t dev_bytes = 0;
  double t_submit = 0, t_done = 0;
  int status = FSMP_OK;
};

// A launch: several admitted requests packed into one BatchView.
struct Pack {
  std::vector<Request*> reqs;
  std::vector<int> first;          // first waveform of each request in the pack
  void* dev = nullptr;             // one device block for all arrays
  void* host = nullptr;            // pinned staging (inputs, then outputs)
  size_t dev_bytes = 0, host_bytes = 0, in_bytes = 0, out_off = 0, trace_off_bytes = 0;
  size_t n_trace = 0;
  int stream = 0;
  std::atomic<int> done{0};
  double t_done = 0;
  struct fsmp_ctx* ctx = nullptr;
  // per waveform: the chain is done (host-mapped flags the kernels raise); per request: whether
  // the serving loop has returned it
  volatile unsigned int* wf_done = nullptr;
  std::vector<char> returned;
  // the pinned block's output regions and each request's first trace record, fixed at launch
  // (a returned request may already be freed by fsmp_poll while its pack still runs, so nothing
  // after the launch reads the other requests of the pack)
  size_t out_region = 0, trace_region = 0;
  std::vector<size_t> trace_first;
};

}  // namespace

struct fsmp_ctx {
  fsmp_params p;
  DevModel M;
  cudaDeviceProp prop;
  int n_smem_max = 0;
  // device tables and scratch
  double *V64 = nullptr, *phi = nullptr, *logphi = nullptr, *cphi = nullptr, *scan = nullptr;
  float *V32 = nullptr, *phi32 = nullptr, *logphi32 = nullptr, *cphi32 = nullptr;
  void* rscratch = nullptr;        // FP64 refresh workspace (FP32 mode)
  size_t rscratch_stride = 0;      // doubles per CTA slot
  int rscratch_slots = 0;
  int* Lt_dev = nullptr;
  void* gscratch = nullptr;
  size_t gscratch_bytes = 0;
  int gscratch_ctas = 0;
  LaunchShape shape_smem{256, 0, 0}, shape_gmem{256, 0, 0};
  // PE-space kernel: SER cross-correlation tables and one scratch set per launch stream (the
  // serving streams, then one for fsmp_run_device), each with slots for every resident chain
  double* tc64 = nullptr;
  float* tc32 = nullptr;
  float* tcff = nullptr;
  // LucyDDM: the kernel taps v(m) = V(m dt) / S (padded to groups of four) and S
  float* lucy_v4 = nullptr;
  float* lucy_S_dev = nullptr;
  float lucy_S = 0.0f;
  std::vector<float> lucy_v4_host;
  struct PeSet {
    void* cinv = nullptr;    // C^-1 slots
    double* ws = nullptr;    // FP64 refresh workspace slots
    int* hist = nullptr;     // N histogram slots
    int* counter = nullptr;  // chain counter of the launch
  };
  std::vector<PeSet> pe_sets;
  int pe_slots = 0, pe_warps = 4, pe_tile = 0, pe_lanes = 32;
  bool pe_lanes_free = false;  // pe_lanes left to fsmp_autotune
  size_t pe_c_stride = 0, pe_ws_stride = 0, pe_bytes = 0;
  std::atomic<long long> n_launches{0};  // chain-kernel launches
  std::mutex tune_mu;                    // serialises fsmp_autotune calls
  // serving loop
  std::vector<cudaStream_t> streams;
  cudaStream_t gmem_stream = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queued;
  std::vector<Pack*> inflight;
  std::deque<Request*> done;
  std::vector<Request*> returned;
  size_t mem_in_use = 0;
  bool stopping = false;
  int fatal = FSMP_OK;
  std::thread worker;
  int next_stream = 0;
  // the last fsmp_run_device / fsmp_lucyddm work of each caller stream (fsmp_destroy waits on it)
  std::mutex user_mu;
  std::vector<std::pair<cudaStream_t, cudaEvent_t>> user_events;
};

namespace {

size_t packed_len(int n) { return (size_t)n * (size_t)(n + 1) / 2; }

// Largest window whose packed Sigma^-1 and vectors fit in one CTA's shared memory.
int smem_n_max(const fsmp_ctx* c) {
  int lo = 1, hi = 4096;
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    size_t b = chain_smem_bytes(c->M, mid, true);
    if (b <= (size_t)c->prop.sharedMemPerBlockOptin) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// CTA size for windows up to n_alloc samples: enough threads for the per-row phases, few
// enough that several chains share an SM (the per-step critical path runs on one warp).
int default_threads(const fsmp_ctx* c, int n_alloc) {
  if (c->p.threads_per_chain > 0) return c->p.threads_per_chain;
  if (c->p.precision == FSMP_FP64) return 128;
  return n_alloc <= 128 ? 128 : 256;
}

// Launch shape for windows up to n_alloc: CTAs = resident CTAs per SM x SMs (persistent).
int make_shape(fsmp_ctx* c, int n_alloc, bool smemP, LaunchShape* out) {
  LaunchShape s;
  s.threads = default_threads(c, n_alloc);
  s.smem = chain_smem_bytes(c->M, n_alloc, smemP);
  if (s.smem > (size_t)c->prop.sharedMemPerBlockOptin) return FSMP_ERR_INVALID;
  // resident CTAs per SM as the hardware computes it (registers, shared memory, threads)
  int per_sm = chain_kernel_occupancy(c->p.precision, smemP, s.threads, s.smem);
  if (per_sm < 1) return FSMP_ERR_INVALID;
  s.ctas = per_sm * c->prop.multiProcessorCount;
  *out = s;
  return FSMP_OK;
}

}  // namespace

// Checks of fsmp_params shared by fsmp_create and fsmp_run_device_noalloc.
int fsmp::validate_params(const fsmp_params* p) {
  if (!p) return FSMP_ERR_INVALID;
  if (!(p->dt_sample_ns > 0) || !(p->grid_ns > 0)) return FSMP_ERR_INVALID;
  double r = p->dt_sample_ns / p->grid_ns;
  long R = lround(r);
  if (R < 1 || R > 64 || fabs(r - (double)R) > 1e-9 * r) return FSMP_ERR_INVALID;
  if (!(p->ser_sigma > 0) || !(p->ser_tau > 0) || !(p->ser_eps > 0) || p->ser_eps >= 1) return FSMP_ERR_INVALID;
  if (p->ser_kind != 0 && p->ser_kind != 1) return FSMP_ERR_INVALID;
  if (p->ser_kind == 1 && (!(p->ser_under_sigma > 0) || !(p->ser_under_tau > 0))) return FSMP_ERR_INVALID;
  if (p->phi_kind != 0 && p->phi_kind != 1) return FSMP_ERR_INVALID;
  if (!(p->phi_p1 > 0) || !(p->phi_p2 > 0) || !(p->phi_support_ns > 0)) return FSMP_ERR_INVALID;
  if (!(p->sigma_q > 0) || !(p->sigma_noise > 0) || !isfinite(p->mu_q)) return FSMP_ERR_INVALID;
  if (!(p->t0_hi >= p->t0_lo)) return FSMP_ERR_INVALID;
  if (!(p->jump_J > 0) || !(p->jump_J <= 0.5)) return FSMP_ERR_INVALID;
  if (p->n_cap < 1 || p->n_cap > 4096 || p->n_max < 1 || p->n_max > 8192) return FSMP_ERR_INVALID;
  if (p->precision != FSMP_FP64 && p->precision != FSMP_FP32_REFRESH) return FSMP_ERR_INVALID;
  if (p->kernel < 0 || p->kernel > 4) return FSMP_ERR_INVALID;
  if (p->pe_tile < 0 || p->pe_tile > 128) return FSMP_ERR_INVALID;
  if (p->pe_ctas_per_sm < 0 || p->pe_ctas_per_sm > 64) return FSMP_ERR_INVALID;
  if (p->pe_lanes != 0 && p->pe_lanes != 16 && p->pe_lanes != 32) return FSMP_ERR_INVALID;
  if (p->kernel == FSMP_KERNEL_PE && p->pe_lanes == 16 && !pe_lanes_ok(16, p->n_cap)) return FSMP_ERR_INVALID;
  if (p->threads_per_chain != 0 && (p->threads_per_chain < 32 || p->threads_per_chain > 512 ||
                                    p->threads_per_chain % 32))
    return FSMP_ERR_INVALID;
  if (p->phi_support_ns / p->grid_ns > 4.0e6) return FSMP_ERR_INVALID;
  if (p->n_mix < 0 || p->n_mix > FSMP_MAX_MIX) return FSMP_ERR_INVALID;
  if (p->n_mix > 0) {
    double sum = 0.0;
    for (int e = 0; e < p->n_mix; ++e) {
      if (!(p->mix_G[e] >= 0.0) || !(p->mix_sigma[e] > 0.0) || !isfinite(p->mix_mu[e])) return FSMP_ERR_INVALID;
      sum += p->mix_G[e];
    }
    if (!(fabs(sum - 1.0) <= 1e-9)) return FSMP_ERR_INVALID;  // G is a distribution
    // the Sigma^-1 kernels carry one charge model; the mixture runs in the PE-space kernel
    if (p->kernel != FSMP_KERNEL_AUTO && p->kernel != FSMP_KERNEL_PE) return FSMP_ERR_INVALID;
  }
  return FSMP_OK;
}

namespace {

void free_ctx(fsmp_ctx* c) {
  if (!c) return;
  cudaFree(c->V64); cudaFree(c->V32); cudaFree(c->phi); cudaFree(c->logphi); cudaFree(c->cphi);
  cudaFree(c->scan); cudaFree(c->Lt_dev); cudaFree(c->gscratch);
  cudaFree(c->phi32); cudaFree(c->logphi32); cudaFree(c->cphi32); cudaFree(c->rscratch);
  cudaFree(c->tc64); cudaFree(c->tc32); cudaFree(c->tcff);
  cudaFree(c->lucy_v4); cudaFree(c->lucy_S_dev);
  for (auto& ps : c->pe_sets) { cudaFree(ps.cinv); cudaFree(ps.ws); cudaFree(ps.hist); cudaFree(ps.counter); }
  for (auto s : c->streams) cudaStreamDestroy(s);
  if (c->gmem_stream) cudaStreamDestroy(c->gmem_stream);
  for (auto& se : c->user_events) cudaEventDestroy(se.second);
  delete c;
}

void CUDART_CB pack_done_cb(void* arg) {
  Pack* pk = (Pack*)arg;
  pk->t_done = now_s();
  {
    std::lock_guard<std::mutex> lk(pk->ctx->mu);
    pk->done.store(1);
  }
  pk->ctx->cv_work.notify_all();
}

// ---- device batch from arrays already on the device
// Launch shape of the PE-space kernel for windows up to n_alloc: warps per CTA, lanes per chain,
// the shared tile of C^-1, and resident CTAs per SM from the hardware's occupancy rule.
int pe_chains_per_cta(const fsmp_ctx* c) { return c->pe_warps * (32 / c->pe_lanes); }
int pe_shape(fsmp_ctx* c, int n_alloc, int* ctas, size_t* smem) {
  *smem = pe_smem_bytes(c->M, n_alloc, c->pe_warps, c->pe_lanes, c->pe_tile);
  if (*smem > (size_t)c->prop.sharedMemPerBlockOptin) return FSMP_ERR_INVALID;
  int per_sm = pe_kernel_occupancy(c->p.precision, c->pe_warps * 32, *smem, pe_big(c->p.n_cap), c->pe_lanes,
                                   c->M.n_comp > 1);
  if (per_sm < 1) return FSMP_ERR_INVALID;
  if (c->p.pe_ctas_per_sm > 0) per_sm = std::min(per_sm, c->p.pe_ctas_per_sm);
  *ctas = per_sm * c->prop.multiProcessorCount;
  return FSMP_OK;
}

int run_pe(fsmp_ctx* c, BatchView B, int set, cudaStream_t st) {
  if (c->pe_sets.empty()) FAIL(FSMP_ERR_INVALID, "the PE-space kernel was not set up at fsmp_create");
  if (B.n_max > c->p.n_max) FAIL(FSMP_ERR_INVALID, "window longer than n_max");
  int ctas = 0;
  size_t smem = 0;
  if (pe_shape(c, B.n_max, &ctas, &smem) != FSMP_OK) FAIL(FSMP_ERR_INVALID, "window too long for the PE-space kernel");
  const int cpc = pe_chains_per_cta(c);
  ctas = std::min(ctas, c->pe_slots / cpc);
  ctas = std::min(ctas, (B.n_waveforms + cpc - 1) / cpc);
  const fsmp_ctx::PeSet& ps = c->pe_sets[set];
  cudaError_t e = launch_pe(c->M, B, c->pe_warps, c->pe_lanes, ctas, c->pe_tile, smem, ps.cinv, c->pe_c_stride,
                            ps.ws, c->pe_ws_stride, ps.hist, ps.counter, st);
  c->n_launches++;
  if (e != cudaSuccess) { set_error("launch_pe", cudaGetErrorString(e), __LINE__); return FSMP_ERR_CUDA; }
  return FSMP_OK;
}

int run_view(fsmp_ctx* c, BatchView B, cudaStream_t st, int set) {
  if (B.n_waveforms <= 0) return FSMP_OK;
  int form = c->p.kernel;
  if (form == FSMP_KERNEL_PE) return run_pe(c, B, set, st);
  if (form == FSMP_KERNEL_AUTO) form = B.n_max <= c->n_smem_max ? FSMP_KERNEL_SMEM : FSMP_KERNEL_GLOBAL;
  if (form == FSMP_KERNEL_SMEM && B.n_max > c->n_smem_max) form = FSMP_KERNEL_GLOBAL;
  if (form == FSMP_KERNEL_PLAIN) {
    // the baseline form: one launch per chain, one CTA, Sigma^-1 in global memory, FP64
    if (c->p.precision != FSMP_FP64 || !c->gscratch) FAIL(FSMP_ERR_INVALID, "the plain form needs precision FSMP_FP64");
    LaunchShape s;
    s.threads = default_threads(c, B.n_max);
    s.smem = chain_smem_bytes(c->M, B.n_max, false);
    s.ctas = 1;
    for (int i = 0; i < B.n_waveforms; ++i) {
      BatchView b1 = B;
      b1.n_waveforms = 1;
      b1.offsets = B.offsets + i;
      b1.lambda0 = B.lambda0 + i;
      if (B.t_origin) b1.t_origin = B.t_origin + i;
      if (B.T_lo) b1.T_lo = B.T_lo + i;
      if (B.T_hi) b1.T_hi = B.T_hi + i;
      if (B.t0_init) b1.t0_init = B.t0_init + i;
      if (B.wf_ids) b1.wf_ids = B.wf_ids + i; else b1.index_base = B.index_base + (uint64_t)i;
      if (B.seeds) b1.seeds = B.seeds + i;
      if (B.n_steps_arr) b1.n_steps_arr = B.n_steps_arr + i;
      if (B.burn_in_arr) b1.burn_in_arr = B.burn_in_arr + i;
      b1.out = B.out + i;
      if (B.trace) {
        if (B.trace_off) b1.trace_off = B.trace_off + i;
        else b1.trace = B.trace + (size_t)i * B.n_steps;
      }
      b1.order = nullptr;
      if (B.wf_done) b1.wf_done = B.wf_done + i;
      cudaError_t e = launch_chains(c->M, b1, FSMP_KERNEL_GLOBAL, s, c->gscratch, c->gscratch_bytes, nullptr, 0, 0, st);
      c->n_launches++;
      if (e != cudaSuccess) { set_error("launch_chains", cudaGetErrorString(e), __LINE__); return FSMP_ERR_CUDA; }
    }
    return FSMP_OK;
  }
  LaunchShape s;
  int rc = make_shape(c, B.n_max, form == FSMP_KERNEL_SMEM, &s);
  if (rc) return rc;
  if (form == FSMP_KERNEL_GLOBAL) {
    if (!c->gscratch) FAIL(FSMP_ERR_INVALID, "windows beyond shared memory need n_max above it at fsmp_create");
    size_t per = packed_len(B.n_max) * (c->p.precision == FSMP_FP64 ? 8 : 4);
    int cap = (int)std::min<size_t>((size_t)s.ctas, c->gscratch_bytes / per);
    if (cap < 1) FAIL(FSMP_ERR_NOMEM, "global scratch too small for this window");
    s.ctas = cap;
  }
  if (c->p.precision != FSMP_FP64) {
    if (!c->rscratch || chain_refresh_bytes(c->p.n_cap, B.n_max) > c->rscratch_stride)
      FAIL(FSMP_ERR_INVALID, "refresh workspace missing or too small");
    s.ctas = std::min(s.ctas, c->rscratch_slots);
  }
  s.ctas = std::min(s.ctas, B.n_waveforms);
  cudaError_t e = launch_chains(c->M, B, form, s, c->gscratch, c->gscratch_bytes, c->rscratch,
                                c->rscratch_stride, c->rscratch_slots, st);
  c->n_launches++;
  if (e != cudaSuccess) { set_error("launch_chains", cudaGetErrorString(e), __LINE__); return FSMP_ERR_CUDA; }
  return FSMP_OK;
}

// Launch the chains of B in length buckets. order_dev lists B's waveforms by decreasing
// window length (n_sorted[i] = length of waveform order[i], host copy). Each bucket gets its
// own persistent launch sized for its longest window, so short windows run with a small
// shared-memory footprint and more CTAs per SM.
int run_bucketed(fsmp_ctx* c, BatchView B, const int32_t* order_dev, const std::vector<int>& n_sorted,
                 cudaStream_t st, int set) {
  static const int kEdges[] = {64, 96, 128, 160, 192, 224, 256, 320, 384, 512, 768, 1024, 2048, 8192};
  const int W = (int)n_sorted.size();
  if (c->p.kernel == FSMP_KERNEL_PE) {  // one launch: warps take chains in the given order
    BatchView b = B;
    b.order = order_dev;
    b.n_max = W > 0 ? *std::max_element(n_sorted.begin(), n_sorted.end()) : 1;
    return run_view(c, b, st, set);
  }
  int i = 0;
  while (i < W) {
    const int nmax = n_sorted[i];
    int lo_edge = 0;
    for (int e : kEdges) if (e < nmax) lo_edge = e;
    // a bucket never straddles the shared-memory limit
    if (nmax > c->n_smem_max && lo_edge < c->n_smem_max) lo_edge = c->n_smem_max;
    int j = i;
    while (j < W && n_sorted[j] > lo_edge) ++j;
    BatchView b = B;
    b.order = order_dev + i;
    b.n_waveforms = j - i;
    b.n_max = nmax;
    int rc = run_view(c, b, st, set);
    if (rc) return rc;
    i = j;
  }
  return FSMP_OK;
}

// ---- serving loop
size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct PackLayout {
  size_t samples, offsets, lambda0, t_origin, T_lo, T_hi, t0_init, wf_ids, seeds, nsteps, burnin,
      trace_off, order, in_end, out, trace, done, total;
};

// Inputs (staged in pinned memory and copied to the device), then the outputs and the per-waveform
// done flags, which the kernels write straight into the pinned host block (host-mapped).
PackLayout pack_layout(size_t n_samp, int W, size_t n_trace) {
  PackLayout L;
  size_t o = 0;
  L.samples = o; o = align_up(o + n_samp * 4, 256);
  L.offsets = o; o = align_up(o + (size_t)(W + 1) * 4, 256);
  L.lambda0 = o; o = align_up(o + (size_t)W * 8, 256);
  L.t_origin = o; o = align_up(o + (size_t)W * 8, 256);
  L.T_lo = o; o = align_up(o + (size_t)W * 4, 256);
  L.T_hi = o; o = align_up(o + (size_t)W * 4, 256);
  L.t0_init = o; o = align_up(o + (size_t)W * 8, 256);
  L.wf_ids = o; o = align_up(o + (size_t)W * 8, 256);
  L.seeds = o; o = align_up(o + (size_t)W * 8, 256);
  L.nsteps = o; o = align_up(o + (size_t)W * 4, 256);
  L.burnin = o; o = align_up(o + (size_t)W * 4, 256);
  L.trace_off = o; o = align_up(o + (size_t)W * 8, 256);
  L.order = o; o = align_up(o + (size_t)W * 4, 256);
  L.in_end = o;
  L.out = o; o = align_up(o + (size_t)W * sizeof(fsmp_summary), 256);
  L.trace = o; o = align_up(o + n_trace * sizeof(fsmp_trace), 256);
  L.done = o; o = align_up(o + (size_t)W * sizeof(unsigned int), 256);
  L.total = o;
  return L;
}

// Device memory a request holds while it runs: its inputs (outputs go to pinned host memory).
size_t request_bytes(const Request* r) {
  size_t n_trace = r->record_trace ? (size_t)r->W * r->n_steps : 0;
  return pack_layout(r->samples.size(), r->W, n_trace).in_end;
}

// Stage and launch one pack (called by the worker without the lock held).
int launch_pack(fsmp_ctx* c, Pack* pk) {
  size_t n_samp = 0, n_trace = 0;
  int W = 0, n_max = 1;
  for (Request* r : pk->reqs) {
    pk->first.push_back(W);
    n_samp += r->samples.size();
    W += r->W;
    if (r->record_trace) n_trace += (size_t)r->W * r->n_steps;
    n_max = std::max(n_max, r->n_max);
  }
  const int n_req = (int)pk->reqs.size();
  PackLayout L = pack_layout(n_samp, W, n_trace);
  pk->out_region = L.out;
  pk->trace_region = L.trace;
  {
    size_t tf = 0;
    for (Request* r : pk->reqs) {
      pk->trace_first.push_back(tf);
      if (r->record_trace) tf += (size_t)r->W * r->n_steps;
    }
  }
  pk->dev_bytes = L.in_end;
  pk->host_bytes = L.total;
  pk->in_bytes = L.in_end;
  pk->out_off = L.out;
  pk->n_trace = n_trace;
  { cudaError_t e_ = cudaMallocHost(&pk->host, L.total); if (e_ != cudaSuccess) { set_error("cudaMallocHost", cudaGetErrorString(e_), __LINE__); return FSMP_ERR_NOMEM; } }
  unsigned char* h = (unsigned char*)pk->host;
  float* samples = (float*)(h + L.samples);
  int32_t* offsets = (int32_t*)(h + L.offsets);
  double* lambda0 = (double*)(h + L.lambda0);
  double* t_origin = (double*)(h + L.t_origin);
  int32_t* T_lo = (int32_t*)(h + L.T_lo);
  int32_t* T_hi = (int32_t*)(h + L.T_hi);
  double* t0_init = (double*)(h + L.t0_init);
  uint64_t* wf_ids = (uint64_t*)(h + L.wf_ids);
  uint64_t* seeds = (uint64_t*)(h + L.seeds);
  int32_t* nsteps = (int32_t*)(h + L.nsteps);
  int32_t* burnin = (int32_t*)(h + L.burnin);
  int64_t* toff = (int64_t*)(h + L.trace_off);
  int32_t* order = (int32_t*)(h + L.order);
  unsigned int* wf_done = (unsigned int*)(h + L.done);
  for (int i = 0; i < W; ++i) wf_done[i] = 0;
  pk->wf_done = wf_done;
  pk->returned.assign(n_req, 0);
  size_t so = 0, to = 0;
  int wi = 0;
  offsets[0] = 0;
  for (Request* r : pk->reqs) {
    memcpy(samples + so, r->samples.data(), r->samples.size() * 4);
    for (int i = 0; i < r->W; ++i, ++wi) {
      offsets[wi + 1] = (int32_t)(so + r->offsets[i + 1]);
      lambda0[wi] = r->lambda0[i];
      t_origin[wi] = r->t_origin.empty() ? 0.0 : r->t_origin[i];
      int n = r->offsets[i + 1] - r->offsets[i];
      T_lo[wi] = r->T_lo.empty() ? 0 : r->T_lo[i];
      T_hi[wi] = r->T_hi.empty() ? n * c->M.R : r->T_hi[i];
      t0_init[wi] = r->t0_init.empty() ? NAN : r->t0_init[i];
      wf_ids[wi] = r->wf_ids.empty() ? r->index_base + (uint64_t)i : r->wf_ids[i];
      seeds[wi] = r->seed;
      nsteps[wi] = r->n_steps;
      burnin[wi] = r->burn_in;
      toff[wi] = r->record_trace ? (int64_t)to : -1;
      if (r->record_trace) to += (size_t)r->n_steps;
    }
    so += r->samples.size();
  }
  // processing order: the PE-space kernel takes chains by decreasing expected cost, window
  // length x (1 + lambda0), so that the heaviest start first and the launch's tail is light;
  // the Sigma^-1 kernels by decreasing window length (their length buckets)
  std::vector<int> n_sorted(W);
  for (int i = 0; i < W; ++i) order[i] = i;
  if (c->p.kernel == FSMP_KERNEL_PE) {
    std::stable_sort(order, order + W, [&](int a, int b) {
      return (double)(offsets[a + 1] - offsets[a]) * (1.0 + lambda0[a]) >
             (double)(offsets[b + 1] - offsets[b]) * (1.0 + lambda0[b]);
    });
  } else {
    std::stable_sort(order, order + W, [&](int a, int b) {
      return offsets[a + 1] - offsets[a] > offsets[b + 1] - offsets[b];
    });
  }
  for (int i = 0; i < W; ++i) n_sorted[i] = offsets[order[i] + 1] - offsets[order[i]];
  // packs of the Sigma^-1 kernels that use context scratch (global Sigma^-1, or the FP32-mode
  // refresh workspace) share it, so they run on one stream; the PE-space kernel has a scratch
  // set per stream
  const bool uses_scratch = c->p.kernel != FSMP_KERNEL_PE &&
                            (n_max > c->n_smem_max || c->p.kernel == FSMP_KERNEL_GLOBAL ||
                             c->p.kernel == FSMP_KERNEL_PLAIN || c->p.precision != FSMP_FP64);
  cudaStream_t st = uses_scratch ? c->gmem_stream : c->streams[pk->stream];
  pk->stream = uses_scratch ? -1 : pk->stream;
  { cudaError_t e_ = cudaMallocAsync(&pk->dev, L.in_end, st); if (e_ != cudaSuccess) { set_error("cudaMallocAsync", cudaGetErrorString(e_), __LINE__); return FSMP_ERR_NOMEM; } }
  // the outputs and counters stay in the pinned host block, which the kernels write through
  // its device mapping
  unsigned char* hd = nullptr;
  { cudaError_t e_ = cudaHostGetDevicePointer((void**)&hd, pk->host, 0); if (e_ != cudaSuccess) { set_error("cudaHostGetDevicePointer", cudaGetErrorString(e_), __LINE__); return FSMP_ERR_CUDA; } }
  { cudaError_t e_ = cudaMemcpyAsync(pk->dev, pk->host, L.in_end, cudaMemcpyHostToDevice, st); if (e_ != cudaSuccess) { set_error("cudaMemcpyAsync", cudaGetErrorString(e_), __LINE__); return FSMP_ERR_CUDA; } }
  unsigned char* d = (unsigned char*)pk->dev;
  BatchView B{};
  B.n_waveforms = W;
  B.n_steps = 0;
  B.burn_in = 0;
  B.n_max = n_max;
  B.samples = (const float*)(d + L.samples);
  B.offsets = (const int32_t*)(d + L.offsets);
  B.lambda0 = (const double*)(d + L.lambda0);
  B.t_origin = (const double*)(d + L.t_origin);
  B.T_lo = (const int32_t*)(d + L.T_lo);
  B.T_hi = (const int32_t*)(d + L.T_hi);
  B.t0_init = (const double*)(d + L.t0_init);
  B.wf_ids = (const uint64_t*)(d + L.wf_ids);
  B.seeds = (const uint64_t*)(d + L.seeds);
  B.n_steps_arr = (const int32_t*)(d + L.nsteps);
  B.burn_in_arr = (const int32_t*)(d + L.burnin);
  B.trace_off = n_trace ? (const int64_t*)(d + L.trace_off) : nullptr;
  B.out = (fsmp_summary*)(hd + L.out);
  B.trace = n_trace ? (fsmp_trace*)(hd + L.trace) : nullptr;
  B.wf_done = (unsigned int*)(hd + L.done);
  int rc = run_bucketed(c, B, (const int32_t*)(d + L.order), n_sorted, st,
                        pk->stream < 0 ? (int)c->streams.size() : pk->stream);
  if (rc) return rc;
  { cudaError_t e_ = cudaFreeAsync(pk->dev, st); if (e_ != cudaSuccess) { set_error("cudaFreeAsync", cudaGetErrorString(e_), __LINE__); return FSMP_ERR_CUDA; } }
  { cudaError_t e_ = cudaLaunchHostFunc(st, pack_done_cb, pk); if (e_ != cudaSuccess) { set_error("cudaLaunchHostFunc", cudaGetErrorString(e_), __LINE__); return FSMP_ERR_CUDA; } }
  return FSMP_OK;
}

// Copy request q's outputs out of the pack's pinned block into the request (its chains are done).
void finish_request(Pack* pk, int q) {
  const unsigned char* h = (const unsigned char*)pk->host;
  const fsmp_summary* out = (const fsmp_summary*)(h + pk->out_region);
  const fsmp_trace* tr = (const fsmp_trace*)(h + pk->trace_region);
  const size_t to = pk->trace_first[q];
  Request* r = pk->reqs[q];
  r->out.assign(out + pk->first[q], out + pk->first[q] + r->W);
  if (r->record_trace) r->trace.assign(tr + to, tr + to + (size_t)r->W * r->n_steps);
  r->t_done = now_s();
  r->status = FSMP_OK;
}

// Requests of the in-flight pack whose chains have all finished (the kernels' flags in the
// pinned block), not yet returned.
std::vector<int> ready_requests(Pack* pk) {
  std::vector<int> ready;
  for (int q = 0; q < (int)pk->reqs.size(); ++q) {
    if (pk->returned[q]) continue;
    const int w0 = pk->first[q], w1 = w0 + pk->reqs[q]->W;
    int w = w0;
    while (w < w1 && pk->wf_done[w]) ++w;
    if (w == w1) ready.push_back(q);
  }
  if (!ready.empty()) std::atomic_thread_fence(std::memory_order_acquire);  // then read their outputs
  return ready;
}

void finish_pack(fsmp_ctx* c, Pack* pk, int status) {
  (void)c;
  for (int q = 0; q < (int)pk->reqs.size(); ++q) {
    if (pk->returned[q]) continue;
    if (status == FSMP_OK) {
      finish_request(pk, q);
    } else {
      pk->reqs[q]->status = status;
      pk->reqs[q]->t_done = now_s();
    }
  }
  if (pk->host) cudaFreeHost(pk->host);
}

void worker_main(fsmp_ctx* c) {
  cudaSetDevice(c->p.device);
  std::unique_lock<std::mutex> lk(c->mu);
  while (true) {
    // requests whose own chains are done return at once, before the rest of their pack
    for (Pack* pk : c->inflight) {
      if (pk->returned.empty()) continue;  // not launched yet
      const std::vector<int> ready = ready_requests(pk);
      if (ready.empty()) continue;
      lk.unlock();
      for (int q : ready) finish_request(pk, q);
      lk.lock();
      for (int q : ready) {
        pk->returned[q] = 1;
        c->done.push_back(pk->reqs[q]);
      }
      c->cv_done.notify_all();
    }
    // completed packs: their memory frees
    for (size_t i = 0; i < c->inflight.size();) {
      Pack* pk = c->inflight[i];
      if (pk->done.load()) {
        c->inflight.erase(c->inflight.begin() + i);
        lk.unlock();
        finish_pack(c, pk, FSMP_OK);
        lk.lock();
        c->mem_in_use -= pk->dev_bytes;
        for (size_t q = 0; q < pk->reqs.size(); ++q)
          if (!pk->returned[q]) c->done.push_back(pk->reqs[q]);
        delete pk;
        c->cv_done.notify_all();
      } else {
        ++i;
      }
    }
    if (c->stopping && c->inflight.empty()) break;
    // admission: pack queued requests that fit the memory budget into one launch per stream
    if (!c->stopping && !c->queued.empty() && (int)c->inflight.size() < (int)c->streams.size()) {
      Pack* pk = new Pack();
      pk->ctx = c;
      size_t bytes = 0;
      int traced = -1;
      while (!c->queued.empty()) {
        Request* r = c->queued.front();
        if (traced >= 0 && traced != r->record_trace) break;
        size_t b = r->dev_bytes;
        if (c->mem_in_use + bytes + b > c->p.device_mem_budget) break;  // wait for memory to free
        traced = r->record_trace;
        bytes += b;
        pk->reqs.push_back(r);
        c->queued.pop_front();
        if (pk->reqs.size() >= 4096) break;
      }
      if (!pk->reqs.empty()) {
        pk->stream = c->next_stream;
        c->next_stream = (c->next_stream + 1) % (int)c->streams.size();
        c->mem_in_use += bytes;
        c->inflight.push_back(pk);
        lk.unlock();
        int rc = launch_pack(c, pk);
        lk.lock();
        pk->dev_bytes = bytes;
        if (rc != FSMP_OK) {
          c->inflight.erase(std::find(c->inflight.begin(), c->inflight.end(), pk));
          c->mem_in_use -= bytes;
          lk.unlock();
          cudaStreamSynchronize(pk->stream < 0 ? c->gmem_stream : c->streams[pk->stream]);
          pk->returned.assign(pk->reqs.size(), 0);
          finish_pack(c, pk, rc);
          lk.lock();
          for (Request* r : pk->reqs) c->done.push_back(r);
          delete pk;
          c->cv_done.notify_all();
        }
        continue;
      }
      delete pk;
    }
    c->cv_work.wait_for(lk, std::chrono::microseconds(200));
  }
}

// Mark the end of work the caller enqueued on `st` through the context (fsmp_destroy waits
// for it). Skipped while `st` is being captured into a graph: the graph's launches are the
// caller's to wait for.
int note_user_work(fsmp_ctx* c, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return FSMP_OK;
  std::lock_guard<std::mutex> lk(c->user_mu);
  cudaEvent_t ev = nullptr;
  for (auto& se : c->user_events)
    if (se.first == st) ev = se.second;
  if (!ev) {
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return FSMP_ERR_CUDA;
    c->user_events.emplace_back(st, ev);
  }
  return cudaEventRecord(ev, st) == cudaSuccess ? FSMP_OK : FSMP_ERR_CUDA;
}

int copy_batch(fsmp_ctx* c, const fsmp_batch* b, Request* r) {
  if (!b->samples || !b->offsets || !b->lambda0 || b->n_waveforms < 1 || b->n_steps < 0 || b->burn_in < 0)
    return FSMP_ERR_INVALID;
  if (b->offsets[0] != 0) return FSMP_ERR_INVALID;
  r->id = b->request_id; r->seed = b->seed; r->index_base = b->index_base;
  r->W = b->n_waveforms; r->n_steps = b->n_steps; r->burn_in = b->burn_in;
  r->record_trace = b->record_trace ? 1 : 0;
  r->n_max = 1;
  for (int i = 0; i < r->W; ++i) {
    int n = b->offsets[i + 1] - b->offsets[i];
    if (n < 1 || n > c->p.n_max) return FSMP_ERR_INVALID;
    if (!(b->lambda0[i] > 0)) return FSMP_ERR_INVALID;
    if (b->T_lo && b->T_hi && b->T_hi[i] <= b->T_lo[i]) return FSMP_ERR_INVALID;
    r->n_max = std::max(r->n_max, n);
  }
  size_t ns = (size_t)b->offsets[r->W];
  r->samples.assign(b->samples, b->samples + ns);
  r->offsets.assign(b->offsets, b->offsets + r->W + 1);
  r->lambda0.assign(b->lambda0, b->lambda0 + r->W);
  if (b->t_origin_ns) r->t_origin.assign(b->t_origin_ns, b->t_origin_ns + r->W);
  if (b->T_lo && b->T_hi) {
    r->T_lo.assign(b->T_lo, b->T_lo + r->W);
    r->T_hi.assign(b->T_hi, b->T_hi + r->W);
  } else if (b->T_lo || b->T_hi) {
    return FSMP_ERR_INVALID;
  }
  if (b->t0_init) r->t0_init.assign(b->t0_init, b->t0_init + r->W);
  if (b->wf_ids) r->wf_ids.assign(b->wf_ids, b->wf_ids + r->W);
  r->dev_bytes = request_bytes(r);
  return FSMP_OK;
}

}  // namespace

extern "C" {

const char* fsmp_last_error(void) { return g_last_error; }

}  // extern "C"

void fsmp::record_error(const char* what, const char* detail) {
  if (!what) { g_last_error[0] = 0; return; }
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, detail ? detail : "");
}

extern "C" {

const char* fsmp_strerror(int s) {
  switch (s) {
    case FSMP_OK: return "ok";
    case FSMP_ERR_INVALID: return "invalid argument";
    case FSMP_ERR_CUDA: return "CUDA error";
    case FSMP_ERR_NOMEM: return "out of memory or over the device memory budget";
    case FSMP_ERR_BUSY: return "submit queue full";
    case FSMP_ERR_TIMEOUT: return "timed out";
    case FSMP_ERR_CLOSED: return "context is shutting down";
    default: return "unknown status";
  }
}

int fsmp_create(const fsmp_params* params, fsmp_ctx** out) {
  g_last_error[0] = 0;
  if (!out) return FSMP_ERR_INVALID;
  int rc = validate_params(params);
  if (rc) FAIL(rc, "invalid fsmp_params");
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (params->device < 0 || params->device >= ndev) FAIL(FSMP_ERR_INVALID, "no such device");
  std::unique_ptr<fsmp_ctx, void (*)(fsmp_ctx*)> c(new fsmp_ctx(), free_ctx);
  c->p = *params;
  // the automatic choice is the PE-space kernel (fastest form at every measured window length)
  if (c->p.kernel == FSMP_KERNEL_AUTO) c->p.kernel = FSMP_KERNEL_PE;
  if (c->p.refresh_every <= 0) c->p.refresh_every = 64;
  if (!(c->p.drift_tol > 0)) c->p.drift_tol = 5e-2;
  if (c->p.device_mem_budget == 0) c->p.device_mem_budget = (size_t)4 << 30;
  if (c->p.max_queued <= 0) c->p.max_queued = 1024;
  if (c->p.n_streams <= 0) c->p.n_streams = 4;
  CK(cudaSetDevice(c->p.device));
  CK(cudaGetDeviceProperties(&c->prop, c->p.device));
  // the context's own stream for its set-up work (and later for the work that shares the
  // context's Sigma^-1 scratch): set-up waits on it alone, never on other work of the device
  CK(cudaStreamCreateWithFlags(&c->gmem_stream, cudaStreamNonBlocking));
  cudaStream_t setup = c->gmem_stream;
  const fsmp_params& p = c->p;
  DevModel& M = c->M;
  M.R = (int)lround(p.dt_sample_ns / p.grid_ns);
  M.inv_Rf = 1.0f / (float)M.R;
  M.g = p.grid_ns;
  M.inv_g = 1.0 / p.grid_ns;
  M.dt = p.dt_sample_ns;
  // phi table range: the largest D with D g <= phi_support_ns
  long D = (long)floor(p.phi_support_ns / p.grid_ns);
  while ((double)(D + 1) * p.grid_ns <= p.phi_support_ns) ++D;
  while (D > 0 && (double)D * p.grid_ns > p.phi_support_ns) --D;
  M.D = (int)D;
  M.mu_q = p.mu_q; M.sigma_q = p.sigma_q; M.sq2 = p.sigma_q * p.sigma_q;
  M.se2 = p.sigma_noise * p.sigma_noise; M.inv_se2 = 1.0 / M.se2;
  M.log_se2 = log(M.se2); M.log_r = log(M.se2 / M.sq2);
  split_pair(M.mu_q, &M.mu_hi, &M.mu_lo); split_pair(M.se2 / M.sq2, &M.r_hi, &M.r_lo);
  // charge components (the cumulative G is summed left to right, as the draw compares it)
  M.n_comp = p.n_mix > 0 ? p.n_mix : 1;
  M.cm_last = 0;
  M.cm_mode = 0;
  for (int e = 1; e < p.n_mix; ++e)
    if (p.mix_G[e] > p.mix_G[M.cm_mode]) M.cm_mode = e;
  {
    double cum = 0.0;
    for (int e = 0; e < FSMP_MAX_MIX; ++e) {
      const bool on = e < M.n_comp;
      const double mu = p.n_mix > 0 ? p.mix_mu[e] : p.mu_q, sg = p.n_mix > 0 ? p.mix_sigma[e] : p.sigma_q;
      const double G = p.n_mix > 0 ? p.mix_G[e] : 1.0;
      M.cm_mu[e] = on ? mu : 0.0;
      M.cm_q[e] = on ? sg * sg : 1.0;
      M.cm_iq[e] = 1.0 / M.cm_q[e];
      M.cm_r[e] = M.se2 / M.cm_q[e];
      M.cm_lr[e] = log(M.cm_r[e]);
      if (on) cum += G;
      M.cm_cum[e] = on ? cum : 2.0;
      if (on && G > 0.0) M.cm_last = e;
      split_pair(M.cm_mu[e], &M.cm_mu_hi[e], &M.cm_mu_lo[e]);
      split_pair(M.cm_r[e], &M.cm_r_hi[e], &M.cm_r_lo[e]);
      M.cmf_mu[e] = (float)M.cm_mu[e];
      M.cmf_q[e] = (float)M.cm_q[e];
      M.cmf_iq[e] = (float)M.cm_iq[e];
      M.cmf_r[e] = (float)M.cm_r[e];
    }
  }
  M.t0_lo = p.t0_lo; M.t0_hi = p.t0_hi; M.sample_t0 = p.sample_t0 ? 1 : 0;
  M.J = p.jump_J; M.log_J = log(p.jump_J);
  M.n_cap = p.n_cap;
  M.precision = p.precision; M.refresh_every = p.refresh_every; M.drift_tol = p.drift_tol;
  // SER scan range (must match the tables' own rule)
  double scan_end = 8.0 * p.ser_sigma + 50.0 * p.ser_tau;
  if (p.ser_kind == 1) scan_end += 8.0 * p.ser_under_sigma + 50.0 * p.ser_under_tau + scan_end;
  int m_end = (int)ceil(scan_end / p.grid_ns) + 1;
  if (m_end > (1 << 22)) FAIL(FSMP_ERR_INVALID, "SER scan range too long");
  CK(cudaMalloc(&c->scan, sizeof(double) * (m_end + M.R)));
  CK(cudaMalloc(&c->V64, sizeof(double) * (m_end + M.R)));
  CK(cudaMalloc(&c->V32, sizeof(float) * (m_end + M.R)));
  CK(cudaMalloc(&c->phi, sizeof(double) * (2 * M.D + 1)));
  CK(cudaMalloc(&c->logphi, sizeof(double) * (2 * M.D + 1)));
  CK(cudaMalloc(&c->cphi, sizeof(double) * (2 * M.D + 1)));
  CK(cudaMalloc(&c->phi32, sizeof(float) * (2 * M.D + 1)));
  CK(cudaMalloc(&c->logphi32, sizeof(float) * (2 * M.D + 1)));
  CK(cudaMalloc(&c->cphi32, sizeof(float) * (2 * M.D + 1)));
  CK(cudaMalloc(&c->Lt_dev, sizeof(int)));
  CK(launch_tables(p, M.R, M.D, m_end, c->V64, c->V32, c->phi, c->logphi, c->cphi, c->phi32,
                   c->logphi32, c->cphi32, c->Lt_dev, c->scan, setup));
  int Lt = 0;
  CK(cudaMemcpyAsync(&Lt, c->Lt_dev, sizeof(int), cudaMemcpyDeviceToHost, setup));
  CK(cudaStreamSynchronize(setup));
  if (Lt < M.R) FAIL(FSMP_ERR_INVALID, "SER table shorter than one sample");
  M.Lt = Lt;
  M.L_V = Lt / M.R;
  // the longest |update shift| is below 8.7 ns (the smallest uniform is 2^-54)
  M.LU = M.L_V + (int)ceil(8.7 / p.dt_sample_ns) + 2;
  M.win_extra = (int)ceil((p.t0_hi - p.t0_lo) / p.grid_ns) + 4;
  if (M.LU > 128) FAIL(FSMP_ERR_INVALID, "SER support above 117 samples is not supported");
  M.V64 = c->V64; M.V32 = c->V32; M.phi = c->phi; M.logphi = c->logphi; M.cphi = c->cphi;
  M.phi32 = c->phi32; M.logphi32 = c->logphi32; M.cphi32 = c->cphi32;
  // SER cross-correlation prefix sums for the PE-space kernel
  {
    const size_t ntc = (size_t)M.R * xcorr_rows(M.Lt, M.R) * (2 * M.Lt - 1);
    CK(cudaMalloc(&c->tc64, sizeof(double) * ntc));
    CK(cudaMalloc(&c->tc32, sizeof(float) * ntc));
    CK(cudaMalloc(&c->tcff, 2 * sizeof(float) * ntc));
    CK(launch_xcorr_table(c->V64, M.Lt, M.R, c->tc64, c->tc32, setup));
    CK(launch_split_ff(c->tc64, c->tcff, ntc, setup));
    M.tc64 = c->tc64; M.tc32 = c->tc32; M.tcff = c->tcff; M.tcM = xcorr_rows(M.Lt, M.R);
  }
  // LucyDDM taps
  CK(cudaMalloc((void**)&c->lucy_v4, sizeof(float) * 4 * ((M.L_V + 3) / 4)));
  CK(cudaMalloc((void**)&c->lucy_S_dev, sizeof(float)));
  CK(launch_lucy_taps(c->V32, M.L_V, M.R, c->lucy_v4, c->lucy_S_dev, setup));
  c->lucy_v4_host.assign(4 * ((M.L_V + 3) / 4), 0.0f);
  CK(cudaMemcpyAsync(&c->lucy_S, c->lucy_S_dev, sizeof(float), cudaMemcpyDeviceToHost, setup));
  CK(cudaMemcpyAsync(c->lucy_v4_host.data(), c->lucy_v4, sizeof(float) * c->lucy_v4_host.size(),
                     cudaMemcpyDeviceToHost, setup));
  CK(cudaStreamSynchronize(setup));
  c->n_smem_max = smem_n_max(c.get());
  int max_smem = (int)c->prop.sharedMemPerBlockOptin;
  CK(chain_kernel_attributes(p.precision, true, max_smem));
  CK(chain_kernel_attributes(p.precision, false, max_smem));
  CK(lucy_kernel_attributes(max_smem));
  if (p.precision != FSMP_FP64) {
    CK(chain_kernel_attributes(FSMP_FP64, false, max_smem));
  }
  // global scratch for Sigma^-1 of windows beyond shared memory (and the plain baseline form)
  bool need_g = p.n_max > c->n_smem_max || p.kernel == FSMP_KERNEL_GLOBAL || p.kernel == FSMP_KERNEL_PLAIN;
  if (need_g) {
    LaunchShape s;
    if (make_shape(c.get(), p.n_max, false, &s) != FSMP_OK) FAIL(FSMP_ERR_INVALID, "n_max too large for the global-memory kernel");
    size_t per = packed_len(p.n_max) * (p.precision == FSMP_FP64 ? 8 : 4);
    c->gscratch_ctas = s.ctas;
    c->gscratch_bytes = per * (size_t)s.ctas;
    { cudaError_t e_ = cudaMalloc(&c->gscratch, c->gscratch_bytes); if (e_ != cudaSuccess) { set_error("cudaMalloc", cudaGetErrorString(e_), __LINE__); return FSMP_ERR_NOMEM; } }
  }
  // FP32 mode: per-CTA FP64 refresh workspace, one slot per resident CTA of the widest launch
  if (p.precision != FSMP_FP64) {
    int slots = 0;
    for (int nn : {64, std::min(p.n_max, c->n_smem_max), p.n_max}) {
      LaunchShape s;
      if (make_shape(c.get(), std::max(1, nn), nn <= c->n_smem_max, &s) == FSMP_OK) slots = std::max(slots, s.ctas);
    }
    c->rscratch_slots = slots;
    c->rscratch_stride = (chain_refresh_bytes(p.n_cap, p.n_max) + 255) / 256 * 256;
    if (cudaMalloc(&c->rscratch, c->rscratch_stride * (size_t)slots) != cudaSuccess)
      FAIL(FSMP_ERR_NOMEM, "refresh workspace allocation failed");
  }
  // PE-space kernel: per-chain slots of C^-1 (when the shared tile can overflow), of the FP64
  // refresh workspace (FP32 mode) and of the N histogram, one set per launch stream; enough
  // slots for every shape the context may launch (both lane counts when the tuner picks it)
  if (p.kernel == FSMP_KERNEL_PE) {
    c->pe_warps = p.threads_per_chain > 0 ? std::min(4, p.threads_per_chain / 32) : 4;
    const size_t esz = pe_c_entry_bytes(p.precision);
    c->pe_tile = p.pe_tile > 0 ? std::min(p.pe_tile, p.n_cap) : std::min(p.n_cap, 32);
    c->pe_lanes = p.pe_lanes > 0 ? p.pe_lanes : 32;
    c->pe_lanes_free = p.pe_lanes == 0 && pe_lanes_ok(16, p.n_cap);
    CK(pe_kernel_attributes(p.precision, max_smem));
    int slots = 0;
    const int lanes0 = c->pe_lanes;
    for (int lanes : {32, 16}) {
      if (lanes != lanes0 && !c->pe_lanes_free) continue;
      c->pe_lanes = lanes;
      for (int nn : {std::min(64, p.n_max), p.n_max}) {
        int ctas = 0;
        size_t sm = 0;
        if (pe_shape(c.get(), nn, &ctas, &sm) == FSMP_OK) slots = std::max(slots, ctas * pe_chains_per_cta(c.get()));
      }
    }
    c->pe_lanes = lanes0;
    if (slots < 1) FAIL(FSMP_ERR_INVALID, "n_max too large for the PE-space kernel");
    c->pe_slots = slots;
    c->pe_c_stride = c->pe_tile < p.n_cap ? pe_c_entries(p.n_cap) : 0;
    // the FP64 rebuild runs in FP32 mode every K accepts, and in both modes for a chain that
    // starts from a given z
    c->pe_ws_stride = pe_ws_slot_doubles(p.n_cap);
    for (int i = 0; i <= p.n_streams; ++i) {
      fsmp_ctx::PeSet ps;
      const size_t cb = c->pe_c_stride * esz * (size_t)slots, wb = c->pe_ws_stride * 8 * (size_t)slots;
      const size_t hb = pe_hist_ints(p.n_cap) * sizeof(int) * (size_t)slots;
      if (cb && cudaMalloc(&ps.cinv, cb) != cudaSuccess) FAIL(FSMP_ERR_NOMEM, "PE-space C^-1 slots");
      if (wb && cudaMalloc((void**)&ps.ws, wb) != cudaSuccess) FAIL(FSMP_ERR_NOMEM, "PE-space refresh workspace");
      if (cudaMalloc((void**)&ps.hist, hb) != cudaSuccess) FAIL(FSMP_ERR_NOMEM, "PE-space N histograms");
      CK(cudaMalloc((void**)&ps.counter, sizeof(int)));
      c->pe_bytes += cb + wb + hb + sizeof(int);
      c->pe_sets.push_back(ps);
    }
  }
  for (int i = 0; i < p.n_streams; ++i) {
    cudaStream_t s;
    CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    c->streams.push_back(s);
  }
  fsmp_ctx* raw = c.release();
  raw->worker = std::thread(worker_main, raw);
  *out = raw;
  return FSMP_OK;
}

int fsmp_submit(fsmp_ctx* c, const fsmp_batch* b) {
  g_last_error[0] = 0;
  if (!c || !b) return FSMP_ERR_INVALID;
  std::unique_ptr<Request> r(new Request());
  int rc = copy_batch(c, b, r.get());
  if (rc) FAIL(rc, "malformed fsmp_batch");
  if (r->dev_bytes > c->p.device_mem_budget) return FSMP_ERR_NOMEM;
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->stopping) return FSMP_ERR_CLOSED;
    if ((int)c->queued.size() >= c->p.max_queued) return FSMP_ERR_BUSY;
    c->queued.push_back(r.release());
  }
  c->cv_work.notify_all();
  return FSMP_OK;
}

int fsmp_poll(fsmp_ctx* c, fsmp_result* out, int max, int timeout_ms) {
  if (!c || (!out && max > 0) || max < 0) return FSMP_ERR_INVALID;
  std::unique_lock<std::mutex> lk(c->mu);
  for (Request* r : c->returned) delete r;
  c->returned.clear();
  if (c->done.empty() && timeout_ms != 0) {
    auto pred = [&] { return !c->done.empty(); };
    if (timeout_ms < 0) c->cv_done.wait(lk, pred);
    else c->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred);
  }
  int k = 0;
  while (k < max && !c->done.empty()) {
    Request* r = c->done.front();
    c->done.pop_front();
    fsmp_result& o = out[k++];
    o.request_id = r->id;
    o.n_waveforms = r->W;
    o.status = r->status;
    o.summaries = r->out.empty() ? nullptr : r->out.data();
    o.trace = r->trace.empty() ? nullptr : r->trace.data();
    o.latency_s = r->t_done - r->t_submit;
    c->returned.push_back(r);
  }
  return k;
}

int fsmp_destroy(fsmp_ctx* c) {
  if (!c) return FSMP_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    c->stopping = true;
    for (Request* r : c->queued) delete r;
    c->queued.clear();
  }
  c->cv_work.notify_all();
  if (c->worker.joinable()) c->worker.join();
  cudaSetDevice(c->p.device);
  // wait for the context's own streams and for the last work the caller enqueued through the
  // context on each of its streams (fsmp_run_device, fsmp_lucyddm), not for the whole device
  for (cudaStream_t s : c->streams) cudaStreamSynchronize(s);
  if (c->gmem_stream) cudaStreamSynchronize(c->gmem_stream);
  {
    std::lock_guard<std::mutex> lk(c->user_mu);
    for (auto& se : c->user_events) cudaEventSynchronize(se.second);
  }
  for (Request* r : c->done) delete r;
  for (Request* r : c->returned) delete r;
  free_ctx(c);
  return FSMP_OK;
}

int fsmp_run_device(fsmp_ctx* c, const fsmp_device_batch* b, void* stream) {
  g_last_error[0] = 0;
  if (!c || !b || b->n_waveforms < 0 || !b->samples || !b->offsets || !b->lambda0 || !b->out ||
      b->n_steps < 0 || b->burn_in < 0)
    return FSMP_ERR_INVALID;
  if ((b->T_lo == nullptr) != (b->T_hi == nullptr)) return FSMP_ERR_INVALID;
  BatchView B{};
  B.n_waveforms = b->n_waveforms;
  B.n_steps = b->n_steps;
  B.burn_in = b->burn_in;
  B.n_max = b->n_max_hint > 0 ? b->n_max_hint : c->p.n_max;
  if (B.n_max > c->p.n_max) return FSMP_ERR_INVALID;
  B.seed = b->seed;
  B.index_base = b->index_base;
  B.samples = b->samples; B.offsets = b->offsets; B.lambda0 = b->lambda0; B.t_origin = b->t_origin_ns;
  B.T_lo = b->T_lo; B.T_hi = b->T_hi; B.t0_init = b->t0_init; B.wf_ids = b->wf_ids;
  B.out = b->out; B.trace = b->trace;
  if (b->z_init) {
    if (!b->n_init || b->z_stride < 1) FAIL(FSMP_ERR_INVALID, "z_init needs n_init and z_stride >= 1");
    if (c->p.kernel != FSMP_KERNEL_PE) FAIL(FSMP_ERR_INVALID, "an initial z needs the PE-space kernel");
    B.z_init = b->z_init; B.n_init = b->n_init; B.z_stride = b->z_stride;
  }
  if (b->pe_hist) {
    if (b->pe_hist_width < 1) FAIL(FSMP_ERR_INVALID, "pe_hist needs pe_hist_width >= 1");
    if (c->p.kernel != FSMP_KERNEL_PE) FAIL(FSMP_ERR_INVALID, "a PE-time histogram needs the PE-space kernel");
    B.pe_hist = b->pe_hist; B.pe_hist_width = b->pe_hist_width;
  }
  { cudaError_t e_ = cudaSetDevice(c->p.device); if (e_ != cudaSuccess) { set_error("cudaSetDevice", cudaGetErrorString(e_), __LINE__); return FSMP_ERR_CUDA; } }
  const int rc = run_view(c, B, (cudaStream_t)stream, (int)c->streams.size());
  if (rc != FSMP_OK) return rc;
  return note_user_work(c, (cudaStream_t)stream);
}

int fsmp_lucyddm(fsmp_ctx* c, const fsmp_lucy_batch* b, void* stream) {
  g_last_error[0] = 0;
  if (!c || !b || b->n_waveforms < 0 || !b->samples || !b->offsets || b->n_iter < 0 || !b->T_lo || !b->T_hi ||
      !b->t0_init || !b->n_init || !b->status || b->z_stride < 0 || (b->z_stride > 0 && !b->z_init))
    FAIL(FSMP_ERR_INVALID, "fsmp_lucyddm: bad arguments");
  const int n_alloc = b->n_max_hint > 0 ? b->n_max_hint : c->p.n_max;
  if (n_alloc > c->p.n_max) FAIL(FSMP_ERR_INVALID, "fsmp_lucyddm: window longer than n_max");
  if (lucy_smem_bytes(c->M.L_V, n_alloc) > (size_t)c->prop.sharedMemPerBlockOptin)
    FAIL(FSMP_ERR_INVALID, "fsmp_lucyddm: window too long for shared memory");
  { cudaError_t e_ = cudaSetDevice(c->p.device); if (e_ != cudaSuccess) { set_error("cudaSetDevice", cudaGetErrorString(e_), __LINE__); return FSMP_ERR_CUDA; } }
  cudaError_t e = launch_lucy(c->lucy_v4_host.data(), c->lucy_S, c->M.L_V, c->M.R, c->M.dt, c->M.g, b->n_waveforms, n_alloc,
                              b->samples, b->offsets, b->t_origin_ns, b->n_iter, (float)b->thresh, b->q_out, b->T_lo,
                              b->T_hi, b->t0_init, b->z_init, b->n_init, b->z_stride, b->status,
                              (cudaStream_t)stream);
  c->n_launches++;
  if (e != cudaSuccess) { set_error("launch_lucy", cudaGetErrorString(e), __LINE__); return FSMP_ERR_CUDA; }
  return note_user_work(c, (cudaStream_t)stream);
}

int fsmp_autotune(fsmp_ctx* c, const fsmp_device_batch* b, int sample, int trial_steps, fsmp_tune* out) {
  g_last_error[0] = 0;
  if (!c || !b || b->n_waveforms < 1 || !b->samples || !b->offsets || !b->lambda0 || sample < 1 || trial_steps < 1)
    FAIL(FSMP_ERR_INVALID, "fsmp_autotune: bad arguments");
  if (c->p.kernel != FSMP_KERNEL_PE || c->pe_sets.empty()) FAIL(FSMP_ERR_INVALID, "fsmp_autotune needs a PE-space context");
  { cudaError_t e_ = cudaSetDevice(c->p.device); if (e_ != cudaSuccess) { set_error("cudaSetDevice", cudaGetErrorString(e_), __LINE__); return FSMP_ERR_CUDA; } }
  std::lock_guard<std::mutex> lk(c->tune_mu);
  const int W = std::min(sample, b->n_waveforms);
  BatchView B{};
  B.n_waveforms = W;
  B.n_steps = trial_steps;
  B.burn_in = 0;
  B.n_max = b->n_max_hint > 0 ? b->n_max_hint : c->p.n_max;
  if (B.n_max > c->p.n_max) FAIL(FSMP_ERR_INVALID, "fsmp_autotune: window longer than n_max");
  B.seed = b->seed;
  B.index_base = b->index_base;
  B.samples = b->samples; B.offsets = b->offsets; B.lambda0 = b->lambda0; B.t_origin = b->t_origin_ns;
  B.T_lo = b->T_lo; B.T_hi = b->T_hi; B.t0_init = b->t0_init; B.wf_ids = b->wf_ids;
  fsmp_summary* scratch = nullptr;
  CK(cudaMalloc(&scratch, sizeof(fsmp_summary) * (size_t)W));
  B.out = scratch;
  B.trace = nullptr;
  cudaStream_t st = c->gmem_stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int set = (int)c->streams.size();
  const int tile0 = c->pe_tile, warps0 = c->pe_warps, ctas0 = c->p.pe_ctas_per_sm, lanes0 = c->pe_lanes;
  auto trial = [&](int lanes, int tile, int warps, int ctas, double* rate) -> int {
    c->pe_lanes = lanes; c->pe_tile = tile; c->pe_warps = warps; c->p.pe_ctas_per_sm = ctas;
    int cc = 0;
    size_t sm = 0;
    if (pe_shape(c, B.n_max, &cc, &sm) != FSMP_OK) { *rate = -1.0; return FSMP_OK; }
    float best_ms = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {  // the first run warms the caches and the code
      if (cudaEventRecord(e0, st) != cudaSuccess) return FSMP_ERR_CUDA;
      int rc = run_pe(c, B, set, st);
      if (rc) return rc;
      if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return FSMP_ERR_CUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) best_ms = std::min(best_ms, ms);
    }
    *rate = (double)W * trial_steps / (best_ms * 1e-3);
    return FSMP_OK;
  };
  // candidates: a tile needs the global C^-1 slots unless it covers n_cap
  const bool have_slots = c->pe_c_stride > 0;
  std::vector<int> tiles;
  for (int t : {8, 16, 24, 32, 48, 64})
    if (t < c->p.n_cap ? have_slots : true) tiles.push_back(std::min(t, c->p.n_cap));
  if (!have_slots) tiles = {tile0};
  std::sort(tiles.begin(), tiles.end());
  tiles.erase(std::unique(tiles.begin(), tiles.end()), tiles.end());
  double r0 = 0.0, best = -1.0;
  int bl = lanes0, bt = tile0, bw = warps0, bc = ctas0, n_tried = 0;
  int rc = trial(lanes0, tile0, warps0, ctas0, &r0);
  if (rc == FSMP_OK) {
    best = r0; ++n_tried;
    // coordinate search: lanes per chain (when the context leaves it free), tile, warps per
    // CTA, then resident CTAs per SM
    if (c->pe_lanes_free) {
      for (int l : {32, 16}) {
        double r;
        if (l == lanes0) continue;
        if ((rc = trial(l, bt, bw, bc, &r)) != FSMP_OK) break;
        ++n_tried;
        if (r > best) { best = r; bl = l; }
      }
    }
    for (int t : tiles) {
      double r;
      if (rc != FSMP_OK || (rc = trial(bl, t, bw, bc, &r)) != FSMP_OK) break;
      ++n_tried;
      if (r > best) { best = r; bt = t; }
    }
    for (int w : {1, 2, 4}) {
      double r;
      if (rc != FSMP_OK || (rc = trial(bl, bt, w, bc, &r)) != FSMP_OK) break;
      ++n_tried;
      if (r > best) { best = r; bw = w; }
    }
    for (int k : {1, 2, 3}) {
      double r;
      if (rc != FSMP_OK || (rc = trial(bl, bt, bw, k, &r)) != FSMP_OK) break;
      ++n_tried;
      if (r > best) { best = r; bc = k; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(scratch);
  if (rc != FSMP_OK) {
    c->pe_lanes = lanes0; c->pe_tile = tile0; c->pe_warps = warps0; c->p.pe_ctas_per_sm = ctas0;
    return rc;
  }
  c->pe_lanes = bl; c->pe_tile = bt; c->pe_warps = bw; c->p.pe_ctas_per_sm = bc;
  if (out) {
    out->pe_tile = bt; out->chains_per_cta = bw * (32 / bl); out->ctas_per_sm = bc; out->n_tried = n_tried;
    out->lanes_per_chain = bl;
    out->best_steps_per_s = best; out->default_steps_per_s = r0;
  }
  return FSMP_OK;
}

int fsmp_get_tables(fsmp_ctx* c, double* ser_out, int max_ser, int* ser_len, int d_lo, int count,
                    double* phi_out, double* logphi_out) {
  if (!c) return FSMP_ERR_INVALID;
  CK(cudaSetDevice(c->p.device));
  if (ser_len) *ser_len = c->M.Lt;
  if (ser_out) {
    if (max_ser < c->M.Lt) return FSMP_ERR_INVALID;
    CK(cudaMemcpy(ser_out, c->V64, sizeof(double) * c->M.Lt, cudaMemcpyDeviceToHost));
  }
  if (count > 0) {
    if (d_lo < -c->M.D || d_lo + count - 1 > c->M.D) return FSMP_ERR_INVALID;
    if (phi_out) CK(cudaMemcpy(phi_out, c->phi + (d_lo + c->M.D), sizeof(double) * count, cudaMemcpyDeviceToHost));
    if (logphi_out) CK(cudaMemcpy(logphi_out, c->logphi + (d_lo + c->M.D), sizeof(double) * count, cudaMemcpyDeviceToHost));
  }
  return FSMP_OK;
}

int fsmp_get_info(fsmp_ctx* c, fsmp_info* o) {
  if (!c || !o) return FSMP_ERR_INVALID;
  memset(o, 0, sizeof(*o));
  o->device = c->p.device;
  o->sm_count = c->prop.multiProcessorCount;
  o->smem_per_block_optin = (int)c->prop.sharedMemPerBlockOptin;
  o->ser_len = c->M.Lt;
  o->R = c->M.R;
  o->L_V = c->M.L_V;
  o->n_smem_max = c->n_smem_max;
  if (c->p.kernel == FSMP_KERNEL_PE) {  // pe_lanes lanes per chain, pe_warps warps per CTA
    int ctas = 0;
    size_t sm = 0;
    if (pe_shape(c, c->p.n_max, &ctas, &sm) == FSMP_OK) {
      o->threads_per_chain = c->pe_lanes;
      o->ctas_per_sm = ctas / c->prop.multiProcessorCount;
    }
  } else {
    LaunchShape s;
    if (make_shape(c, std::min(c->p.n_max, c->n_smem_max), true, &s) == FSMP_OK) {
      o->threads_per_chain = s.threads;
      o->ctas_per_sm = s.ctas / c->prop.multiProcessorCount;
    }
  }
  o->scratch_bytes = c->gscratch_bytes + c->rscratch_stride * (size_t)c->rscratch_slots + c->pe_bytes;
  snprintf(o->name, sizeof(o->name), "%.63s", c->prop.name);
  o->n_launches = c->n_launches.load();
  return FSMP_OK;
}

int fsmp_philox_blocks(fsmp_ctx* c, const uint64_t key[2], const uint64_t* ctrs, int n, uint64_t* out) {
  if (!c || !key || !ctrs || !out || n < 0) return FSMP_ERR_INVALID;
  if (n == 0) return FSMP_OK;
  CK(cudaSetDevice(c->p.device));
  uint64_t *dc = nullptr, *dout = nullptr;
  size_t bytes = sizeof(uint64_t) * 4 * (size_t)n;
  { cudaError_t e_ = cudaMalloc(&dc, bytes); if (e_ != cudaSuccess) { set_error("cudaMalloc", cudaGetErrorString(e_), __LINE__); return FSMP_ERR_NOMEM; } }
  if (cudaMalloc(&dout, bytes) != cudaSuccess) { cudaFree(dc); return FSMP_ERR_NOMEM; }
  int rc = FSMP_OK;
  if (cudaMemcpy(dc, ctrs, bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      launch_philox(dc, dout, n, key[0], key[1], 0) != cudaSuccess ||
      cudaMemcpy(out, dout, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = FSMP_ERR_CUDA;
  cudaFree(dc);
  cudaFree(dout);
  return rc;
}

int fsmp_lambda_mle(fsmp_ctx* c, const int32_t* hist, int n_hist, int n_max, const double* lambda0, int lanes,
                    double* out) {
  g_last_error[0] = 0;
  if (!c || !hist || !lambda0 || !out || n_hist < 0 || n_max < 0 || (lanes != 16 && lanes != 32))
    FAIL(FSMP_ERR_INVALID, "fsmp_lambda_mle: bad arguments");
  for (int i = 0; i < n_hist; ++i)
    if (!(lambda0[i] > 0.0)) FAIL(FSMP_ERR_INVALID, "fsmp_lambda_mle: lambda0 must be positive");
  if (n_hist == 0) return FSMP_OK;
  CK(cudaSetDevice(c->p.device));
  const size_t hb = sizeof(int32_t) * (size_t)n_hist * (n_max + 1), lb = sizeof(double) * (size_t)n_hist;
  int* dh = nullptr;
  double *dl = nullptr, *dout = nullptr;
  int rc = FSMP_OK;
  if (cudaMalloc(&dh, hb) != cudaSuccess || cudaMalloc(&dl, lb) != cudaSuccess || cudaMalloc(&dout, lb) != cudaSuccess) {
    rc = FSMP_ERR_NOMEM;
  } else {
    cudaStream_t st = c->gmem_stream;
    if (cudaMemcpyAsync(dh, hist, hb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dl, lambda0, lb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        launch_lambda_mle(dh, n_hist, n_max, dl, dout, lanes, st) != cudaSuccess ||
        cudaMemcpyAsync(out, dout, lb, cudaMemcpyDeviceToHost, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
      rc = FSMP_ERR_CUDA;
  }
  cudaFree(dh);
  cudaFree(dl);
  cudaFree(dout);
  if (rc == FSMP_ERR_CUDA) set_error("fsmp_lambda_mle", "a copy or the launch failed", __LINE__);
  return rc;
}

int fsmp_measure_peaks(fsmp_ctx* c, double* smem_gbs, double* fp64_tflops, double* fp32_tflops) {
  g_last_error[0] = 0;
  if (!c || !smem_gbs || !fp64_tflops || !fp32_tflops) FAIL(FSMP_ERR_INVALID, "null argument");
  CK(cudaSetDevice(c->p.device));
  CK(measure_peaks(c->prop.multiProcessorCount, smem_gbs, fp64_tflops, fp32_tflops));
  return FSMP_OK;
}

}  // extern "C"
