// fsmp_tables.cu -- model tables on the PE grid, computed on the GPU once per context.
//
//  * SER (Sec. 3 of arXiv 2403.03156): the ex-Gaussian shifted by 4 sigma,
//      V(t) = (1/2tau) exp((s^2 - 2(t-4s)tau) / 2tau^2) (1 + Erf(-(s^2 - (t-4s)tau) / (sqrt2 s tau))),
//    with 1 + Erf(-u) evaluated as erfc(u); optionally minus a peak-normalised undershoot pulse
//    started at the main peak (ser_kind 1). Normalised to its maximum over the grid points
//    m g, m in [0, m_end), and truncated after the last grid point with |V| >= ser_eps,
//    rounded up to whole samples: Lt = L_V * R entries.
//  * phi(d g) for grid offsets d in [-D, D] (the PE time density about t0 of Eq. (pzmu)),
//    log phi (-inf where phi = 0), and the running sum of phi used by the birth proposal
//    h(t) = phi(t - t0) / int_T phi (Sec. 2.4, last equation) and its normaliser Phi_T.
#include <math.h>

#include "fsmp_internal.h"

namespace fsmp {
namespace {

__device__ double exgauss_shifted(double t, double sigma, double tau) {
  double x = t - 4.0 * sigma;
  double expo = (sigma * sigma - 2.0 * x * tau) / (2.0 * tau * tau);
  double c = erfc((sigma * sigma - x * tau) / (sqrt(2.0) * sigma * tau));
  if (!(c > 0.0)) return 0.0;
  return exp(expo + log(c) - log(2.0 * tau));
}

__device__ double exgauss_density(double x, double sigma, double tau) {
  double expo = (sigma * sigma - 2.0 * x * tau) / (2.0 * tau * tau);
  double c = erfc((sigma * sigma - x * tau) / (sqrt(2.0) * sigma * tau));
  if (!(c > 0.0)) return 0.0;
  return exp(expo + log(c) - log(2.0 * tau));
}

struct SerArgs {
  int kind;
  double sigma, tau, under_frac, under_sigma, under_tau, eps, g;
  int m_end, R;
};

// Block-wide argmax (first index of the maximum) over v[0..m).
__device__ void block_argmax(const double* v, int m, double* best_v, int* best_i) {
  __shared__ double sv[32];
  __shared__ int si[32];
  double bv = -1.0;
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    if (v[i] > bv) { bv = v[i]; bi = i; }
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, bv, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (l == 0) { sv[w] = bv; si[w] = bi; }
  __syncthreads();
  if (w == 0) {
    bv = l < nw ? sv[l] : -1.0;
    bi = l < nw ? si[l] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (l == 0) { sv[0] = bv; si[0] = bi; }
  }
  __syncthreads();
  *best_v = sv[0];
  *best_i = si[0];
  __syncthreads();
}

// One CTA: scan the SER on [0, m_end), normalise, truncate, fill the tables.
__global__ void __launch_bounds__(1024) ser_table_kernel(SerArgs a, double* scan, double* V64, float* V32, int* Lt_out) {
  const int m_end = a.m_end;
  // main pulse and its grid peak time
  for (int m = threadIdx.x; m < m_end; m += blockDim.x) scan[m] = exgauss_shifted(m * a.g, a.sigma, a.tau);
  __syncthreads();
  double main_peak, under_peak = 1.0, t_peak;
  int i_peak;
  block_argmax(scan, m_end, &main_peak, &i_peak);
  t_peak = i_peak * a.g;
  if (a.kind == 1) {
    for (int m = threadIdx.x; m < m_end; m += blockDim.x)
      scan[m] = exgauss_shifted(m * a.g, a.under_sigma, a.under_tau);
    __syncthreads();
    int dummy;
    block_argmax(scan, m_end, &under_peak, &dummy);
  }
  // combined shape on [0, m_end + R) (the extra R covers rounding Lt up to whole samples)
  for (int m = threadIdx.x; m < m_end + a.R; m += blockDim.x) {
    double t = m * a.g;
    double v = exgauss_shifted(t, a.sigma, a.tau);
    if (a.kind == 1) {
      double tu = t - t_peak;
      double vu = tu >= 0.0 ? exgauss_shifted(tu, a.under_sigma, a.under_tau) : 0.0;
      v = v / main_peak - a.under_frac * vu / under_peak;
    }
    scan[m] = v;
  }
  __syncthreads();
  double peak;
  int dummy;
  block_argmax(scan, m_end, &peak, &dummy);
  // last grid point with |V| / peak >= eps
  __shared__ int s_last;
  if (threadIdx.x == 0) s_last = 0;
  __syncthreads();
  int last = 0;
  for (int m = threadIdx.x; m < m_end; m += blockDim.x)
    if (fabs(scan[m]) / peak >= a.eps) last = max(last, m);
  atomicMax(&s_last, last);
  __syncthreads();
  int Lt = ((s_last + 1 + a.R - 1) / a.R) * a.R;
  for (int m = threadIdx.x; m < Lt; m += blockDim.x) {
    double v = scan[m] / peak;
    V64[m] = v;
    V32[m] = (float)v;
  }
  if (threadIdx.x == 0) *Lt_out = Lt;
}

__global__ void phi_table_kernel(int kind, double p1, double p2, double support, double g, int D,
                                 double* phi, double* logphi) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > 2 * D) return;
  double t = (double)(i - D) * g;
  double v;
  if (fabs(t) > support) {
    v = 0.0;
  } else if (kind == 0) {
    v = exgauss_density(t, p1, p2);
  } else {
    v = t < 0.0 ? 0.0 : (p1 + p2) / (p2 * p2) * (1.0 - exp(-t / p1)) * exp(-t / p2);
  }
  phi[i] = v;
  logphi[i] = v > 0.0 ? log(v) : -INFINITY;
}

// Running sum of phi over the table (one CTA: per-thread chunks, then a scan of chunk sums).
__global__ void to_float_kernel(const double* a, float* b, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

__global__ void __launch_bounds__(1024) phi_cumsum_kernel(const double* phi, double* cphi, int n) {
  __shared__ double part[1024];
  int T = blockDim.x, t = threadIdx.x;
  int chunk = (n + T - 1) / T;
  int b = t * chunk, e = min(n, b + chunk);
  double s = 0.0;
  for (int i = b; i < e; ++i) s += phi[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    double run = 0.0;
    for (int i = 0; i < T; ++i) { double v = part[i]; part[i] = run; run += v; }
  }
  __syncthreads();
  double run = part[t];
  for (int i = b; i < e; ++i) { run += phi[i]; cphi[i] = run; }
}

__global__ void philox_kernel(const uint64_t* ctrs, uint64_t* out, int n, uint64_t k0, uint64_t k1) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t c[4] = {ctrs[4 * i], ctrs[4 * i + 1], ctrs[4 * i + 2], ctrs[4 * i + 3]};
  philox4x64_10(c, k0, k1);
  for (int k = 0; k < 4; ++k) out[4 * i + k] = c[k];
}

// Prefix sums of SER cross-correlations on the PE grid. For a PE whose first sample sits at
// phase ph (the grid distance from the PE to that sample, 0 <= ph < R) and a second PE o grid
// points earlier:
//   tc[ph][m][o + Lt - 1] = sum_{i < m} V[ph + i R] V[ph + i R + o],  V = 0 outside [0, Lt).
// The inner product of the two PEs' columns over the samples i in [ilo, ihi) of the first one's
// support is then tc[.][ihi][.] - tc[.][ilo][.]; with o = 0 it is the squared norm. One thread per
// (ph, o), FP64 running sums.
__global__ void xcorr_table_kernel(const double* V, int Lt, int R, int M1, double* tc) {
  const int O = 2 * Lt - 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= R * O) return;
  const int ph = t / O, oi = t - ph * O, o = oi - (Lt - 1);
  double acc = 0.0;
  for (int m = 0; m < M1; ++m) {
    tc[((size_t)ph * M1 + m) * O + oi] = acc;
    const int a = ph + m * R, b = a + o;
    if (a < Lt && b >= 0 && b < Lt) acc += V[a] * V[b];
  }
}

}  // namespace

cudaError_t launch_xcorr_table(const double* V64, int Lt, int R, double* tc64, float* tc32, cudaStream_t st) {
  const int M1 = xcorr_rows(Lt, R);
  const int n = R * (2 * Lt - 1);
  xcorr_table_kernel<<<(n + 127) / 128, 128, 0, st>>>(V64, Lt, R, M1, tc64);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int tot = n * M1;
  to_float_kernel<<<(tot + 255) / 256, 256, 0, st>>>(tc64, tc32, tot);
  return cudaGetLastError();
}

cudaError_t launch_tables(const fsmp_params& p, int R, int D, int m_end, double* V64, float* V32,
                          double* phi, double* logphi, double* cphi, float* phi32, float* logphi32,
                          float* cphi32, int* Lt_out_dev, double* scan_buf, cudaStream_t st) {
  SerArgs a{p.ser_kind, p.ser_sigma, p.ser_tau, p.ser_under_frac, p.ser_under_sigma, p.ser_under_tau,
            p.ser_eps, p.grid_ns, m_end, R};
  ser_table_kernel<<<1, 1024, 0, st>>>(a, scan_buf, V64, V32, Lt_out_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int n = 2 * D + 1;
  phi_table_kernel<<<(n + 255) / 256, 256, 0, st>>>(p.phi_kind, p.phi_p1, p.phi_p2, p.phi_support_ns,
                                                    p.grid_ns, D, phi, logphi);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  phi_cumsum_kernel<<<1, 1024, 0, st>>>(phi, cphi, n);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  to_float_kernel<<<(n + 255) / 256, 256, 0, st>>>(phi, phi32, n);
  to_float_kernel<<<(n + 255) / 256, 256, 0, st>>>(logphi, logphi32, n);
  to_float_kernel<<<(n + 255) / 256, 256, 0, st>>>(cphi, cphi32, n);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint64_t* ctrs, uint64_t* out, int n, uint64_t k0, uint64_t k1,
                          cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  philox_kernel<<<(n + 255) / 256, 256, 0, st>>>(ctrs, out, n, k0, k1);
  return cudaGetLastError();
}

}  // namespace fsmp
