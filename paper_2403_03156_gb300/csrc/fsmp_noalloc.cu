// fsmp_noalloc.cu -- fsmp_run_device_noalloc: the FP32 chain kernel run without any device
// allocation, for callers that cannot call cudaMalloc (for example code running under an
// allocator that owns all device memory, or inside an environment that forbids allocation
// after start-up). All device scratch the run needs -- the model tables and the per-CTA FP64
// refresh workspaces -- lives in one file-scope static __device__ array of
// kNoallocScratchBytes, which every GPU that loads this code holds until the process exits.
//
// Set-up: the first call on a device resolves the array's device address with
// cudaGetSymbolAddress (with that device current) and sets the kernel's shared-memory limit;
// the first call on a device, and the first call after the model parameters change, also
// builds the tables into the array and synchronises the stream once to read the SER length.
// Such a call should therefore come before any stream capture.
//
// Every call shares the array and leaves its contents behind for the next call. Work on one
// stream runs in order, so calls on one stream are safe whatever their parameters (a table
// rebuild follows the previous call's kernel on that stream). Calls on different streams that
// overlap on the GPU race on the array. Nothing in the array has to start at zero: every table
// entry and workspace word is written before it is read.
#include <math.h>
#include <string.h>

#include <mutex>

#include "fsmp_internal.h"

namespace fsmp {
namespace {

constexpr size_t kNoallocScratchBytes = (size_t)64 << 20;  // 64 MiB
constexpr int kNoallocMaxWindow = 256;                      // samples
constexpr int kNoallocMaxCap = 64;                          // PEs per chain
constexpr int kNoallocMaxPhiHalf = 32768;                   // phi table: grid offsets [-D, D]
constexpr int kNoallocMaxSerScan = 16384;                   // SER scan points

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

struct DeviceState {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch on this device
  int sm_count = 0;
  size_t smem_optin = 0;
  bool have_tables = false;
  fsmp_params tparams;            // the parameters the tables in the array were built for
  DevModel M;
};

std::mutex g_mu;
DeviceState g_dev[64];

size_t rup(size_t x) { return (x + 255) / 256 * 256; }

bool same_model(const fsmp_params& a, const fsmp_params& b) {
  return a.dt_sample_ns == b.dt_sample_ns && a.grid_ns == b.grid_ns && a.ser_kind == b.ser_kind &&
         a.ser_sigma == b.ser_sigma && a.ser_tau == b.ser_tau && a.ser_under_frac == b.ser_under_frac &&
         a.ser_under_sigma == b.ser_under_sigma && a.ser_under_tau == b.ser_under_tau && a.ser_eps == b.ser_eps &&
         a.phi_kind == b.phi_kind && a.phi_p1 == b.phi_p1 && a.phi_p2 == b.phi_p2 &&
         a.phi_support_ns == b.phi_support_ns;
}

int fail(int code, const char* msg) {
  record_error("fsmp_run_device_noalloc", msg);
  return code;
}

// Table regions inside the static array (bytes from its start) for a given SER scan length
// m_end and phi half-range D.
struct TableLayout {
  size_t scan, V64, V32, phi, logphi, cphi, phi32, logphi32, cphi32, Lt, end;
};
TableLayout table_layout(int m_end, int R, int D) {
  TableLayout t;
  size_t o = 0, nv = (size_t)m_end + R, nd = 2 * (size_t)D + 1;
  t.scan = o; o = rup(o + nv * 8);
  t.V64 = o; o = rup(o + nv * 8);
  t.V32 = o; o = rup(o + nv * 4);
  t.phi = o; o = rup(o + nd * 8);
  t.logphi = o; o = rup(o + nd * 8);
  t.cphi = o; o = rup(o + nd * 8);
  t.phi32 = o; o = rup(o + nd * 4);
  t.logphi32 = o; o = rup(o + nd * 4);
  t.cphi32 = o; o = rup(o + nd * 4);
  t.Lt = o; o = rup(o + sizeof(int));
  t.end = o;
  return t;
}

int table_region_bytes() {
  return (int)table_layout(kNoallocMaxSerScan, 64, kNoallocMaxPhiHalf).end;
}

}  // namespace
}  // namespace fsmp

using namespace fsmp;

extern "C" int fsmp_run_device_noalloc(const fsmp_params* p, const fsmp_device_batch* b, void* stream) {
  record_error(nullptr, nullptr);
  if (!p || !b) return fail(FSMP_ERR_INVALID, "null argument");
  if (p->precision != FSMP_FP32_REFRESH) return fail(FSMP_ERR_INVALID, "precision must be FSMP_FP32_REFRESH");
  // the checks fsmp_create makes (threads_per_chain a multiple of 32 in 32..512, finite mu_q,
  // an integer dt / grid ratio, ...), then this entry point's own limits
  if (validate_params(p) != FSMP_OK) return fail(FSMP_ERR_INVALID, "invalid fsmp_params (the checks of fsmp_create)");
  const long R = lround(p->dt_sample_ns / p->grid_ns);
  if (p->n_mix != 0) return fail(FSMP_ERR_INVALID, "the MCP charge mixture runs only in the PE-space kernel");
  if (p->n_cap < 1 || p->n_cap > kNoallocMaxCap) return fail(FSMP_ERR_INVALID, "n_cap exceeds the static-scratch limit of 64");
  const int n_max = b->n_max_hint > 0 ? b->n_max_hint : p->n_max;
  if (n_max < 1 || n_max > kNoallocMaxWindow) return fail(FSMP_ERR_INVALID, "window length exceeds the static-scratch limit of 256 samples");
  if (b->n_waveforms < 0 || !b->samples || !b->offsets || !b->lambda0 || !b->out || b->n_steps < 0 || b->burn_in < 0 ||
      (b->T_lo == nullptr) != (b->T_hi == nullptr))
    return fail(FSMP_ERR_INVALID, "malformed fsmp_device_batch");
  if (p->device < 0 || p->device >= 64) return fail(FSMP_ERR_INVALID, "device ordinal out of range");
  // model constants, derived exactly as fsmp_create derives them
  long D = (long)floor(p->phi_support_ns / p->grid_ns);
  while ((double)(D + 1) * p->grid_ns <= p->phi_support_ns) ++D;
  while (D > 0 && (double)D * p->grid_ns > p->phi_support_ns) --D;
  if (D > kNoallocMaxPhiHalf) return fail(FSMP_ERR_INVALID, "phi_support_ns / grid_ns exceeds the static-scratch limit of 32768");
  double scan_end = 8.0 * p->ser_sigma + 50.0 * p->ser_tau;
  if (p->ser_kind == 1) scan_end += 8.0 * p->ser_under_sigma + 50.0 * p->ser_under_tau + scan_end;
  const int m_end = (int)ceil(scan_end / p->grid_ns) + 1;
  if (m_end > kNoallocMaxSerScan) return fail(FSMP_ERR_INVALID, "SER scan exceeds the static-scratch limit of 16384 grid points");

  int prev_dev = 0;
  if (cudaGetDevice(&prev_dev) != cudaSuccess) return fail(FSMP_ERR_CUDA, "cudaGetDevice failed");
  if (cudaSetDevice(p->device) != cudaSuccess) return fail(FSMP_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = FSMP_OK;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState& ds = g_dev[p->device];
    if (!ds.ready) {  // once per device, with the device current
      void* addr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess) { cudaSetDevice(prev_dev); return fail(FSMP_ERR_CUDA, cudaGetErrorString(e)); }
      cudaDeviceProp prop;
      e = cudaGetDeviceProperties(&prop, p->device);
      if (e == cudaSuccess) e = chain_kernel_attributes(FSMP_FP32_REFRESH, true, (int)prop.sharedMemPerBlockOptin);
      if (e != cudaSuccess) { cudaSetDevice(prev_dev); return fail(FSMP_ERR_CUDA, cudaGetErrorString(e)); }
      ds.base = (unsigned char*)addr;
      ds.sm_count = prop.multiProcessorCount;
      ds.smem_optin = prop.sharedMemPerBlockOptin;
      ds.ready = true;
    }
    DevModel& M = ds.M;
    const TableLayout tl = table_layout(m_end, (int)R, (int)D);
    if (!ds.have_tables || !same_model(ds.tparams, *p)) {
      unsigned char* B0 = ds.base;
      cudaError_t e = launch_tables(*p, (int)R, (int)D, m_end, (double*)(B0 + tl.V64), (float*)(B0 + tl.V32),
                                    (double*)(B0 + tl.phi), (double*)(B0 + tl.logphi), (double*)(B0 + tl.cphi),
                                    (float*)(B0 + tl.phi32), (float*)(B0 + tl.logphi32), (float*)(B0 + tl.cphi32),
                                    (int*)(B0 + tl.Lt), (double*)(B0 + tl.scan), st);
      int Lt = 0;
      if (e == cudaSuccess) e = cudaMemcpyAsync(&Lt, B0 + tl.Lt, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) { ds.have_tables = false; cudaSetDevice(prev_dev); return fail(FSMP_ERR_CUDA, cudaGetErrorString(e)); }
      if (Lt < R) { ds.have_tables = false; cudaSetDevice(prev_dev); return fail(FSMP_ERR_INVALID, "SER table shorter than one sample"); }
      M = DevModel{};
      M.R = (int)R; M.inv_Rf = 1.0f / (float)R; M.g = p->grid_ns; M.inv_g = 1.0 / p->grid_ns; M.dt = p->dt_sample_ns; M.D = (int)D;
      M.Lt = Lt; M.L_V = Lt / (int)R;
      M.LU = M.L_V + (int)ceil(8.7 / p->dt_sample_ns) + 2;
      M.V64 = (const double*)(B0 + tl.V64); M.V32 = (const float*)(B0 + tl.V32);
      M.phi = (const double*)(B0 + tl.phi); M.logphi = (const double*)(B0 + tl.logphi); M.cphi = (const double*)(B0 + tl.cphi);
      M.phi32 = (const float*)(B0 + tl.phi32); M.logphi32 = (const float*)(B0 + tl.logphi32);
      M.cphi32 = (const float*)(B0 + tl.cphi32);
      ds.tparams = *p;
      ds.have_tables = true;
    }
    if (M.LU > 128) rc = fail(FSMP_ERR_INVALID, "SER support above 117 samples is not supported");
    // per-call model terms (not part of the tables)
    M.win_extra = (int)ceil((p->t0_hi - p->t0_lo) / p->grid_ns) + 4;
    M.mu_q = p->mu_q; M.sigma_q = p->sigma_q; M.sq2 = p->sigma_q * p->sigma_q;
    M.se2 = p->sigma_noise * p->sigma_noise; M.inv_se2 = 1.0 / M.se2;
    M.log_se2 = log(M.se2); M.log_r = log(M.se2 / M.sq2);
    split_pair(M.mu_q, &M.mu_hi, &M.mu_lo); split_pair(M.se2 / M.sq2, &M.r_hi, &M.r_lo);
    M.t0_lo = p->t0_lo; M.t0_hi = p->t0_hi; M.sample_t0 = p->sample_t0 ? 1 : 0;
    M.J = p->jump_J; M.log_J = log(p->jump_J);
    M.n_cap = p->n_cap;
    M.precision = FSMP_FP32_REFRESH;
    M.refresh_every = p->refresh_every > 0 ? p->refresh_every : 64;
    M.drift_tol = p->drift_tol > 0 ? p->drift_tol : 5e-2;
    if (rc == FSMP_OK && b->n_waveforms > 0) {
      LaunchShape s;
      s.threads = p->threads_per_chain > 0 ? p->threads_per_chain : (n_max <= 128 ? 128 : 256);
      s.smem = chain_smem_bytes(M, n_max, true);
      const int per_sm = s.smem <= ds.smem_optin ? chain_kernel_occupancy(FSMP_FP32_REFRESH, true, s.threads, s.smem) : 0;
      // refresh workspaces fill the array after the table region
      const size_t tbytes = (size_t)table_region_bytes();
      const size_t stride = rup(chain_refresh_bytes(p->n_cap, n_max));
      const int slots = (int)((kNoallocScratchBytes - tbytes) / stride);
      if (per_sm < 1) {
        rc = fail(FSMP_ERR_INVALID, "window does not fit the kernel's shared memory");
      } else if (slots < 1) {
        rc = fail(FSMP_ERR_INVALID, "refresh workspace exceeds the static scratch");
      } else {
        s.ctas = per_sm * ds.sm_count;
        if (s.ctas > slots) s.ctas = slots;
        if (s.ctas > b->n_waveforms) s.ctas = b->n_waveforms;
        BatchView B{};
        B.n_waveforms = b->n_waveforms; B.n_steps = b->n_steps; B.burn_in = b->burn_in; B.n_max = n_max;
        B.seed = b->seed; B.index_base = b->index_base;
        B.samples = b->samples; B.offsets = b->offsets; B.lambda0 = b->lambda0; B.t_origin = b->t_origin_ns;
        B.T_lo = b->T_lo; B.T_hi = b->T_hi; B.t0_init = b->t0_init; B.wf_ids = b->wf_ids;
        B.out = b->out; B.trace = b->trace;
        cudaError_t e = launch_chains(M, B, FSMP_KERNEL_SMEM, s, nullptr, 0, ds.base + tbytes, stride, slots, st);
        if (e != cudaSuccess) rc = fail(FSMP_ERR_CUDA, cudaGetErrorString(e));
      }
    }
  }
  cudaSetDevice(prev_dev);
  return rc;
}
