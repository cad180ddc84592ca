// fsmp_internal.h -- definitions shared by the library's translation units (device model,
// batch view, Philox4x64-10, launch entry points). Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fsmp.h"

#define FSMP_HD __host__ __device__ __forceinline__

namespace fsmp {

constexpr double kTwoPi = 6.283185307179586;
constexpr double kLog2Pi = 1.8378770664093453;
constexpr int kMaxWarps = 16;  // CTAs of at most 512 threads

// Model constants and table pointers, passed by value to every kernel.
struct DevModel {
  double g, inv_g, dt;        // PE grid step, 1 / g (grid steps per ns), sample period
  int R;                      // grid points per sample
  float inv_Rf;               // 1 / R in FP32 (a first estimate of the sample of a grid index)
  int Lt, L_V;                // SER table length (L_V * R) and support in samples
  int D;                      // phi tables cover grid offsets d in [-D, D]
  int LU;                     // longest union support of a two-PE jump (samples)
  int win_extra;              // phi window per chain: n R + win_extra grid offsets (t0 range + 2)
  double mu_q, sigma_q, sq2, se2, inv_se2;
  double log_se2, log_r;       // log sigma_eps^2 and log(sigma_eps^2 / sigma_q^2)
  float mu_hi, mu_lo, r_hi, r_lo;  // mu_q and sigma_eps^2 / sigma_q^2 as float pairs (hi + lo)
  // Charge components of the PE-space kernel: one (mu_q, sigma_q) for the dynode model, else
  // the MCP mixture (Eq. (mcp-multi-norm)). For component e: mean cm_mu, variance cm_q,
  // its inverse cm_iq, cm_r = sigma_eps^2 / cm_q and its log, cumulative probability
  // G(0) + .. + G(e), and the float pairs of cm_mu and cm_r.
  int n_comp, cm_last;        // components; the last one with G > 0
  int cm_mode;                // the most probable component (of an initial PE)
  double cm_mu[FSMP_MAX_MIX], cm_q[FSMP_MAX_MIX], cm_iq[FSMP_MAX_MIX], cm_r[FSMP_MAX_MIX], cm_lr[FSMP_MAX_MIX];
  double cm_cum[FSMP_MAX_MIX];
  float cm_mu_hi[FSMP_MAX_MIX], cm_mu_lo[FSMP_MAX_MIX], cm_r_hi[FSMP_MAX_MIX], cm_r_lo[FSMP_MAX_MIX];
  // FP32 copies of cm_mu, cm_q, cm_iq, cm_r for the FP32 scoring (no FP64 conversion in the step)
  float cmf_mu[FSMP_MAX_MIX], cmf_q[FSMP_MAX_MIX], cmf_iq[FSMP_MAX_MIX], cmf_r[FSMP_MAX_MIX];
  double t0_lo, t0_hi;
  int sample_t0;
  double J, log_J;
  int n_cap;
  int precision, refresh_every;
  double drift_tol;
  const double* V64;          // SER on the PE grid, peak 1          [Lt]
  const float* V32;           // FP32 copy                           [Lt]
  const double* phi;          // phi(d g)                            [2D + 1], index d + D
  const double* logphi;       // log phi(d g), -inf where phi = 0
  const double* cphi;         // running sum of phi over d' <= d (no g factor)
  const float* phi32;         // FP32 copies of the three phi tables (FP32 mode)
  const float* logphi32;
  const float* cphi32;
  // SER cross-correlation prefix sums [R][tcM][2 Lt - 1] (the PE-space kernel; may be null)
  const double* tc64;
  const float* tc32;
  const float* tcff;          // float-float pairs (hi, lo) of tc64
  int tcM;                    // rows per phase: ceil(Lt / R) + 1
};

// x = hi + lo with hi = fl32(x), lo = fl32(x - hi) (host side).
inline void split_pair(double x, float* hi, float* lo) {
  *hi = (float)x;
  *lo = (float)(x - (double)*hi);
}

// Rows per phase of the cross-correlation table: prefix lengths 0 .. ceil(Lt / R).
FSMP_HD int xcorr_rows(int Lt, int R) { return (Lt + R - 1) / R + 1; }

// One launch's chains. Waveform i of the view is samples[offsets[i] .. offsets[i+1]).
// Optional per-waveform arrays override the batch-wide scalars.
struct BatchView {
  int n_waveforms, n_steps, burn_in, n_max;
  uint64_t seed, index_base;
  const float* samples;
  const int32_t* offsets;
  const double* lambda0;
  const double* t_origin;      // may be null
  const int32_t* T_lo;         // may be null
  const int32_t* T_hi;         // may be null
  const double* t0_init;       // may be null
  const uint64_t* wf_ids;      // may be null
  const uint64_t* seeds;       // may be null: per-waveform seed
  const int32_t* n_steps_arr;  // may be null
  const int32_t* burn_in_arr;  // may be null
  const int64_t* trace_off;    // may be null: first trace record of each waveform
  const int32_t* order;        // may be null: processing order (a permutation of waveforms)
  fsmp_summary* out;
  fsmp_trace* trace;           // may be null
  const int32_t* z_init;       // may be null: initial PEs, waveform i at z_init[i * z_stride]
  const int32_t* n_init;
  int z_stride;
  uint32_t* pe_hist;           // may be null: PE counts per grid point after burn-in
  int pe_hist_width;
  // serving packs (may be null): per waveform a flag in host-mapped memory that the serving
  // loop polls, set once the chain's summary (and trace) are written
  unsigned int* wf_done;
};

#ifdef __CUDACC__
// A chain's summary (and trace) are written: make them visible to the host, then raise the
// chain's flag (a plain store, no host atomics needed), so that the serving loop can return a
// request as soon as its own chains are done. The group's or block's writing thread calls it.
__device__ __forceinline__ void note_chain_done(const BatchView& B, int wi) {
  if (B.wf_done != nullptr) {
    __threadfence_system();
    *(volatile unsigned int*)(B.wf_done + wi) = 1u;
  }
}
#endif

// Philox4x64-10 (Salmon et al., SC'11): two 64x64->128 multiplies per round, Weyl key bumps.
FSMP_HD void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
#ifdef __CUDA_ARCH__
    uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
#else
    unsigned __int128 p0 = (unsigned __int128)M0 * c[0], p1 = (unsigned __int128)M1 * c[2];
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
#endif
    uint64_t y0 = hi1 ^ c[1] ^ k0, y2 = hi0 ^ c[3] ^ k1;
    c[0] = y0; c[1] = lo1; c[2] = y2; c[3] = lo0;
  }
}

FSMP_HD double u01_from_bits(uint64_t x) { return ((double)(x >> 11) + 0.5) * 0x1.0p-53; }

#ifdef __CUDACC__
// lambda_FSMP of a chain (Eq. (reduce-mu0)): the maximiser of
//   l(lambda) = -lambda + log sum_N h[N] (lambda / lambda0)^N
// over its N-sample counts h[0 .. n_max]. l can have several local maxima (a chain that visits
// clusters of N far apart), all inside (0, top] with top the largest N sampled, since a
// stationary point satisfies lambda = E_w[N] with w_N ∝ h[N] (lambda / lambda0)^N. So:
// (1) scan l on 2 L to 8 L points of (0, top] in FP32 (lanes over points) and take the best;
// (2) Newton steps on l'(lambda) = -1 + E_w[N] / lambda, l''(lambda) = (Var_w[N] - E_w[N]) /
//     lambda^2, kept within two scan cells of the best point (bisection where a step would
//     leave them, fixed-point steps lambda <- E_w[N] where l'' >= 0): first in FP32 to 1e-6,
//     then at most 12 steps in FP64 to 1e-14 (two or three from there) -- FP64 costs this part
//     64 FP32 operations each, and every chain of a launch ends here; (3) the boundary
//     lambda = 0 when l(0) is not smaller (a maximum that the FP32 steps push below 1e-6 of a
//     scan cell is taken as the boundary). A group of L consecutive lanes (mask gm, sl the lane
//     within it) calls it and every lane gets the result; NAN if h is empty.
template <typename F, int L>
__device__ inline F lmle_newton(const int* h, int bot, int top, F lambda0, F lam, F& lo, F& hi, F tol, int max_it,
                                int sl, unsigned gm, F* ll_out) {
  F ll = -INFINITY;
  for (int it = 0; it < max_it; ++it) {
    if (hi - lo <= tol * hi) break;  // the bracket has closed
    const F s = log(lam / lambda0);
    F mx = -INFINITY;
    for (int k = bot + sl; k <= top; k += L)
      if (h[k] > 0) mx = fmax(mx, log((F)h[k]) + k * s);
    for (int o = L / 2; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(gm, mx, o, L));
    F sw = 0, s1 = 0, s2 = 0;
    for (int k = bot + sl; k <= top; k += L)
      if (h[k] > 0) {
        const F e = exp(log((F)h[k]) + k * s - mx);
        sw += e; s1 += k * e; s2 += (F)k * k * e;
      }
    for (int o = L / 2; o > 0; o >>= 1) {
      sw += __shfl_xor_sync(gm, sw, o, L);
      s1 += __shfl_xor_sync(gm, s1, o, L);
      s2 += __shfl_xor_sync(gm, s2, o, L);
    }
    const F E = s1 / sw, Vr = s2 / sw - E * E;
    ll = -lam + mx + log(sw);
    const F g = -1 + E / lam, H = (Vr - E) / (lam * lam);
    if (g == 0) break;                    // a stationary point
    if (g > 0) lo = lam; else hi = lam;   // the maximum lies on the side l' points to
    F nl = H < 0 ? lam - g / H : E;
    if (!(nl > lo && nl < hi)) nl = (F)0.5 * (lo + hi);
    const bool done = fabs(nl - lam) <= tol * lam;
    lam = nl;
    if (done) break;
  }
  *ll_out = ll;
  return lam;
}

template <int L>
__device__ inline double group_lambda_mle(const int* h, int n_max, double lambda0, int sl, unsigned gm) {
  int top = -1, bot = n_max + 1;
  for (int k = sl; k <= n_max; k += L)
    if (h[k] > 0) { top = k; bot = min(bot, k); }
  for (int o = L / 2; o > 0; o >>= 1) {
    top = max(top, __shfl_xor_sync(gm, top, o, L));
    bot = min(bot, __shfl_xor_sync(gm, bot, o, L));
  }
  if (top < 0) return NAN;
  if (top == 0) return 0.0;
  // (1) coarse scan, log2 units: l / ln 2 = -lambda / ln 2 + log2 sum_N h[N] 2^(N log2(lambda / lambda0)),
  // on G points with a spacing of at most top / (8 L), and of at most 16 / (2 L) below top = 16
  const int G = min(8, 2 * ((top + 15) / 16)) * L;
  const float lr0 = log2f((float)lambda0);
  float best = -INFINITY;
  int bi = 0;
  for (int g = sl; g < G; g += L) {
    const float lam = (float)top * (float)(g + 1) / (float)G;
    const float s2 = log2f(lam) - lr0;
    float mx = -INFINITY;
    for (int k = bot; k <= top; ++k)
      if (h[k] > 0) mx = fmaxf(mx, log2f((float)h[k]) + (float)k * s2);
    float acc = 0.0f;
    for (int k = bot; k <= top; ++k)
      if (h[k] > 0) acc += exp2f(log2f((float)h[k]) + (float)k * s2 - mx);
    const float l = -lam * 1.44269504f + mx + log2f(acc);
    if (l > best) { best = l; bi = g; }
  }
  for (int o = L / 2; o > 0; o >>= 1) {  // argmax, the smaller index on ties
    const float ob = __shfl_xor_sync(gm, best, o, L);
    const int oi = __shfl_xor_sync(gm, bi, o, L);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  // (2) Newton within [lambda_(b-2), lambda_(b+2)] (two scan cells of slack for the FP32
  // rounding of the scan): FP32, then FP64 from its result
  const double cell = (double)top / G;
  const double lo0 = fmax(cell * (bi - 1), 1e-6 * cell), hi0 = cell * (bi + 3);
  float lo32 = (float)lo0, hi32 = (float)hi0, ll32;
  const float lam32 = lmle_newton<float, L>(h, bot, top, (float)lambda0, (float)(cell * (bi + 1)), lo32, hi32,
                                            1e-6f, 60, sl, gm, &ll32);
  const double l0 = h[0] > 0 ? log((double)h[0]) : -INFINITY;  // l(0): only N = 0 contributes
  double lo = lo0, hi = hi0, ll;
  double lam = (double)lam32;
  if (!(lam > lo && lam < hi)) lam = cell * (bi + 1);
  if (h[0] > 0 && hi32 <= 2e-6 * cell) return 0.0;  // the steps ran into the boundary
  lam = lmle_newton<double, L>(h, bot, top, lambda0, lam, lo, hi, 1e-14, 12, sl, gm, &ll);
  return l0 >= ll ? 0.0 : lam;
}
__device__ inline double warp_lambda_mle(const int* h, int n_max, double lambda0, int lane) {
  return group_lambda_mle<32>(h, n_max, lambda0, lane, 0xffffffffu);
}
#endif

// Launchers (fsmp_tables.cu / fsmp_chain.cu). All return cudaError_t of the launch.
cudaError_t launch_tables(const fsmp_params& p, int R, int D, int m_end, double* V64, float* V32,
                          double* phi, double* logphi, double* cphi, float* phi32, float* logphi32,
                          float* cphi32, int* Lt_out_dev, double* scan_buf, cudaStream_t st);
cudaError_t launch_xcorr_table(const double* V64, int Lt, int R, double* tc64, float* tc32, cudaStream_t st);
cudaError_t launch_philox(const uint64_t* ctrs, uint64_t* out, int n, uint64_t k0, uint64_t k1,
                          cudaStream_t st);

struct LaunchShape {
  int threads, ctas;
  size_t smem;
};
// Shared-memory bytes of one chain CTA for windows up to n_alloc samples.
size_t chain_smem_bytes(const DevModel& M, int n_alloc, bool sigma_in_smem);
// Launch the chain kernel. gmem_scratch: packed Sigma^-1 slots for the global-memory form;
// refresh_ws: FP32-mode refresh workspace, refresh_slots slots of refresh_stride bytes.
cudaError_t launch_chains(const DevModel& M, const BatchView& B, int kernel_form, LaunchShape shape,
                          void* gmem_scratch, size_t gmem_scratch_bytes, void* refresh_ws,
                          size_t refresh_stride, int refresh_slots, cudaStream_t st);
// Bytes of one CTA's refresh workspace for windows up to n_alloc samples.
size_t chain_refresh_bytes(int n_cap, int n_alloc);
cudaError_t chain_kernel_attributes(int precision, bool sigma_in_smem, int max_smem);
// Resident CTAs per SM of the chain kernel for this block size and dynamic shared memory.
int chain_kernel_occupancy(int precision, bool sigma_in_smem, int threads, size_t smem);
cudaError_t measure_peaks(int sm_count, double* smem_gbs, double* fp64_tflops, double* fp32_tflops);
// PE-space kernel (fsmp_pe.cu, fsmp_pe_mix.cu, fsmp_pe_kernel.cuh): a chain on `lanes` (32 or 16)
// lanes, warps per CTA. Shared memory
// per CTA with windows up to n_alloc and a shared tile of C^-1 for Ns PEs per chain; FP64
// workspace doubles per chain slot (FP32 mode); entries of a global C^-1 slot; ints of an N
// histogram slot.
size_t pe_smem_bytes(const DevModel& M, int n_alloc, int warps, int lanes, int Ns);
size_t pe_ws_slot_doubles(int n_cap);
size_t pe_c_entries(int n_cap);  // entries of a global C^-1 slot (packed triangle)
size_t pe_c_entry_bytes(int precision);  // bytes of one C^-1 entry (a pair of FP64 or FP32 values)
inline size_t pe_hist_ints(int n_cap) { return (size_t)n_cap + 1; }
cudaError_t pe_kernel_attributes(int precision, int max_smem);
cudaError_t launch_split_ff(const double* a, float* out, size_t n, cudaStream_t st);
int pe_kernel_occupancy(int precision, int threads, size_t smem, bool big, int lanes, bool mix);
// The MCP-mixture instances (fsmp_pe_mix.cu); launch_pe dispatches to them when M.n_comp > 1.
cudaError_t pe_mix_attributes(int precision, int max_smem);
int pe_mix_occupancy(int precision, int threads, size_t smem, int lanes);
cudaError_t pe_mix_launch(const DevModel& M, const BatchView& B, int warps, int lanes, int ctas, int Ns, size_t smem,
                          void* cinv, size_t c_stride, double* ws, size_t ws_stride, int* hist, int* counter,
                          cudaStream_t st);
bool pe_big(int n_cap);
bool pe_lanes_ok(int lanes, int n_cap);
// Slots (C^-1, workspace, histogram) are indexed by resident chain: CTA x warps x (32 / lanes).
// counter: one int of device memory, zeroed on `st` before the launch.
cudaError_t launch_pe(const DevModel& M, const BatchView& B, int warps, int lanes, int ctas, int Ns, size_t smem,
                      void* cinv, size_t c_stride, double* ws, size_t ws_stride, int* hist, int* counter,
                      cudaStream_t st);
// lambda_FSMP of n_hist histograms of n_max + 1 counts on `lanes` (32 or 16) lanes each, by the
// device function the chain kernels end with (testing aid; fsmp_pe.cu).
cudaError_t launch_lambda_mle(const int* h, int n_hist, int n_max, const double* lambda0, double* out, int lanes,
                              cudaStream_t st);
// LucyDDM (fsmp_lucy.cu): shared memory per CTA for windows up to n_alloc; the kernel taps
// v(m) = V(m dt) / S, padded to whole groups of four, and S (on the device); the deconvolution
// launch, given the taps in host memory (they travel in the kernel's parameters).
size_t lucy_smem_bytes(int LV, int n_alloc);
cudaError_t lucy_kernel_attributes(int max_smem);
cudaError_t launch_lucy_taps(const float* V32, int LV, int R, float* v4, float* S_dev, cudaStream_t st);
cudaError_t launch_lucy(const float* v4_host, float S, int LV, int R, double dt, double g, int n_waveforms, int n_alloc,
                        const float* samples, const int32_t* offsets, const double* t_origin, int n_iter, float thresh,
                        float* q_out, int32_t* T_lo, int32_t* T_hi, double* t0, int32_t* z, int32_t* n_z, int z_stride,
                        int* status, cudaStream_t st);
// FSMP_OK if the model and engine parameters are valid, else FSMP_ERR_INVALID (fsmp_runtime.cu).
int validate_params(const fsmp_params* p);
// Set (or, with what == nullptr, clear) the calling thread's fsmp_last_error() message.
void record_error(const char* what, const char* detail);

}  // namespace fsmp
