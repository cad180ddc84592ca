// fsmp_lucy.cu -- LucyDDM on the GPU (arXiv 2403.03156, Sec. 2.3): Lucy's iterative
// deconvolution of each waveform by the SER at the sample times, then the solution space
// T = [t_min - 4 ns, t_max + 4 ns], the initial PEs {tau : q-hat(tau) > thresh} and t0 = t_min.
//
// With the kernel v(m) = V(m dt) / S (m = 0 .. L_V - 1, unit sum) and the data
// d(t) = max(w(t), 0) / S, one iteration is two correlations over the window:
//   w^r(t) = sum_m q(t - m) v(m)                          t = 0 .. n-1
//   q(tau) <- q(tau) sum_m [d / w^r](tau + m) v(m)         tau = -L_V+1 .. n-1
// (a ratio with w^r = 0 is 0; d / w^r is 0 outside the window). q^0 is uniform with the sum
// of d.
//
// Layout: one warp per waveform, its d, q-hat and ratio in shared memory (FP32), zero-padded so
// that no tap needs a bounds check. Each lane computes four consecutive outputs: per group of
// four taps it loads one aligned float4 of the source and does 16 FMAs, the previous float4
// supplying the other operands (the loads are conflict-free 128-bit accesses). The taps travel
// in the kernel's parameters and are read through the constant cache, which leaves the shared
// memory pipe to the sources. Arithmetic: 2 (n + L_V) L_V FMAs per iteration, FP32.
#include <math.h>

#include "fsmp_internal.h"

namespace fsmp {
namespace {

constexpr int kLucyWarps = 4;  // waveforms per CTA
constexpr int kLucyMaxJV = 32;  // groups of four taps the parameters carry (L_V <= 128)

// Padded per-warp arrays: Q[kq + tau] (tau from -kq), Rr[kr + t] (t from -kr), d[t].
struct LucyLayout {
  int jv;        // groups of four taps: ceil(L_V / 4)
  int kq, kr;    // leading zero pads (multiples of 4)
  int qlen, rlen, dlen;
};
__host__ __device__ inline LucyLayout lucy_layout(int LV, int n_alloc) {
  LucyLayout l;
  l.jv = (LV + 3) / 4;
  l.kq = 4 * (l.jv + 1);
  l.kr = 4 * (l.jv + 1);
  const int tb = (n_alloc + 127) / 128 * 128;                      // t outputs, in blocks of 128
  const int ub = (n_alloc + 4 * l.jv + 127) / 128 * 128;           // tau outputs from -4 jv
  l.qlen = l.kq + tb + 8;
  l.rlen = l.kr + ub + 4 * (l.jv + 1) + 8;
  l.dlen = (n_alloc + 3) / 4 * 4;
  return l;
}
__host__ __device__ inline size_t lucy_warp_bytes(int LV, int n_alloc) {
  const LucyLayout l = lucy_layout(LV, n_alloc);
  return sizeof(float) * (size_t)(l.qlen + l.rlen + l.dlen);
}

struct LucyArgs {
  float4 taps[kLucyMaxJV];  // v(4j .. 4j+3), zero beyond L_V
  const float* samples;
  const int32_t* offsets;
  const double* t_origin;
  int n_waveforms, n_alloc, n_iter, LV, R, z_stride;
  float thresh, inv_S;
  double dt, g;
  float* q_out;
  int32_t* T_lo;
  int32_t* T_hi;
  double* t0;
  int32_t* z;
  int32_t* n_z;
  int* status;  // per waveform: 0, or FSMP_ST_INVALID when the window is empty or longer than n_alloc
};

__global__ void __launch_bounds__(kLucyWarps * 32) lucy_kernel(const __grid_constant__ LucyArgs A) {
  extern __shared__ __align__(16) float lsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wi = blockIdx.x * kLucyWarps + warp;
  if (wi >= A.n_waveforms) return;
  const LucyLayout ly = lucy_layout(A.LV, A.n_alloc);
  float* Q = lsm + (size_t)warp * (ly.qlen + ly.rlen + ly.dlen);
  float* Rr = Q + ly.qlen;
  float* d = Rr + ly.rlen;
  const int o0 = A.offsets[wi], n = A.offsets[wi + 1] - o0;
  const int LV = A.LV, nq = n + LV - 1;
  if (n < 1 || n > A.n_alloc) {
    if (lane == 0) {
      A.status[wi] = FSMP_ST_INVALID;
      A.n_z[wi] = 0; A.T_lo[wi] = 0; A.T_hi[wi] = max(n, 0) * A.R; A.t0[wi] = NAN;
    }
    return;
  }
  // data, zero pads, q^0
  float ds = 0.0f;
  for (int t = lane; t < ly.dlen; t += 32) {
    const float x = t < n ? A.samples[o0 + t] : 0.0f;
    const float dv = x > 0.0f ? x * A.inv_S : 0.0f;
    d[t] = dv;
    ds += dv;
  }
  for (int o = 16; o > 0; o >>= 1) ds += __shfl_xor_sync(0xffffffffu, ds, o);
  const float q0 = ds / (float)nq;
  for (int i = lane; i < ly.qlen; i += 32) {
    const int tau = i - ly.kq;
    Q[i] = (tau >= -(LV - 1) && tau < n) ? q0 : 0.0f;
  }
  for (int i = lane; i < ly.rlen; i += 32) Rr[i] = 0.0f;
  __syncwarp();
  const float4* Q4 = reinterpret_cast<const float4*>(Q);
  const float4* R4 = reinterpret_cast<const float4*>(Rr);
  const int jv = ly.jv;
#pragma unroll 1
  for (int it = 0; it < A.n_iter; ++it) {
    // w^r(t) for t = t0 .. t0+3, t0 = base + 4 lane: taps m = 4j + r read q(t0 + k - 4j - r),
    // i.e. the float4 at t0 - 4j (k >= r) and the one at t0 - 4j - 4 (k < r)
#pragma unroll 1
    for (int base = 0; base < n; base += 128) {
      const int t0 = base + 4 * lane;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
      float4 cur = Q4[(ly.kq + t0) / 4];
#pragma unroll 1
      for (int j = 0; j < jv; ++j) {
        const float4 nxt = Q4[(ly.kq + t0) / 4 - j - 1];
        const float4 vv = A.taps[j];
        // r = 0: q(t0 + k - 4j)
        a0 = fmaf(cur.x, vv.x, a0); a1 = fmaf(cur.y, vv.x, a1); a2 = fmaf(cur.z, vv.x, a2); a3 = fmaf(cur.w, vv.x, a3);
        // r = 1: q(t0 + k - 4j - 1)
        a0 = fmaf(nxt.w, vv.y, a0); a1 = fmaf(cur.x, vv.y, a1); a2 = fmaf(cur.y, vv.y, a2); a3 = fmaf(cur.z, vv.y, a3);
        // r = 2
        a0 = fmaf(nxt.z, vv.z, a0); a1 = fmaf(nxt.w, vv.z, a1); a2 = fmaf(cur.x, vv.z, a2); a3 = fmaf(cur.y, vv.z, a3);
        // r = 3
        a0 = fmaf(nxt.y, vv.w, a0); a1 = fmaf(nxt.z, vv.w, a1); a2 = fmaf(nxt.w, vv.w, a2); a3 = fmaf(cur.x, vv.w, a3);
        cur = nxt;
      }
      const float acc[4] = {a0, a1, a2, a3};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int t = t0 + k;
        if (t < n) Rr[ly.kr + t] = acc[k] > 0.0f ? d[t] / acc[k] : 0.0f;
      }
    }
    __syncwarp();
    // q(tau) *= sum_m ratio(tau + m) v(m) for tau = u0 .. u0+3, u0 = -4 jv + base + 4 lane: taps
    // m = 4j + r read ratio(u0 + k + 4j + r), the float4 at u0 + 4j (k + r < 4) and the next one
#pragma unroll 1
    for (int base = 0; base < n + 4 * jv; base += 128) {
      const int u0 = -4 * jv + base + 4 * lane;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
      float4 cur = R4[(ly.kr + u0) / 4];
#pragma unroll 1
      for (int j = 0; j < jv; ++j) {
        const float4 nxt = R4[(ly.kr + u0) / 4 + j + 1];
        const float4 vv = A.taps[j];
        a0 = fmaf(cur.x, vv.x, a0); a1 = fmaf(cur.y, vv.x, a1); a2 = fmaf(cur.z, vv.x, a2); a3 = fmaf(cur.w, vv.x, a3);
        a0 = fmaf(cur.y, vv.y, a0); a1 = fmaf(cur.z, vv.y, a1); a2 = fmaf(cur.w, vv.y, a2); a3 = fmaf(nxt.x, vv.y, a3);
        a0 = fmaf(cur.z, vv.z, a0); a1 = fmaf(cur.w, vv.z, a1); a2 = fmaf(nxt.x, vv.z, a2); a3 = fmaf(nxt.y, vv.z, a3);
        a0 = fmaf(cur.w, vv.w, a0); a1 = fmaf(nxt.x, vv.w, a1); a2 = fmaf(nxt.y, vv.w, a2); a3 = fmaf(nxt.z, vv.w, a3);
        cur = nxt;
      }
      const float acc[4] = {a0, a1, a2, a3};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int tau = u0 + k;
        if (tau >= -(LV - 1) && tau < n) Q[ly.kq + tau] *= acc[k];
      }
    }
    __syncwarp();
  }
  // q-hat out, initial PEs in tau order, solution space and t0 (Sec. 2.3)
  float* qo = A.q_out ? A.q_out + (size_t)o0 + (size_t)wi * (LV - 1) : nullptr;
  int cnt = 0, tmin = 0, tmax = 0;
  int32_t* zo = A.z + (size_t)wi * A.z_stride;
#pragma unroll 1
  for (int b = 0; b < nq; b += 32) {
    const int i = b + lane;
    const int tau = i - (LV - 1);
    const float qv = i < nq ? Q[ly.kq + tau] : 0.0f;
    if (qo && i < nq) qo[i] = qv;
    const bool on = i < nq && qv > A.thresh;
    const unsigned m = __ballot_sync(0xffffffffu, on);
    if (on) {
      const int pos = cnt + __popc(m & ((1u << lane) - 1u));
      if (pos < A.z_stride) zo[pos] = tau * A.R;
    }
    if (m) {
      if (cnt == 0) tmin = b + __ffs(m) - 1 - (LV - 1);
      tmax = b + 31 - __clz(m) - (LV - 1);
    }
    cnt += __popc(m);
  }
  if (lane == 0) {
    A.status[wi] = 0;
    A.n_z[wi] = cnt;
    if (cnt == 0) {
      A.T_lo[wi] = 0;
      A.T_hi[wi] = n * A.R;
      A.t0[wi] = NAN;
    } else {
      A.T_lo[wi] = (int32_t)floor((tmin * A.dt - 4.0) / A.g + 1e-9);
      A.T_hi[wi] = (int32_t)ceil((tmax * A.dt + 4.0) / A.g - 1e-9) + 1;
      A.t0[wi] = (A.t_origin ? A.t_origin[wi] : 0.0) + tmin * A.dt;
    }
  }
}

// The kernel taps v(m) = V(m dt) / S, zero-padded to whole groups of four.
__global__ void lucy_taps_kernel(const float* V32, int LV, int R, int jv, float* v4, float* S_out) {
  float s = 0.0f;
  for (int m = 0; m < LV; ++m) s += V32[m * R];
  for (int m = threadIdx.x; m < 4 * jv; m += blockDim.x) v4[m] = m < LV ? V32[m * R] / s : 0.0f;
  if (threadIdx.x == 0) *S_out = s;
}

}  // namespace

size_t lucy_smem_bytes(int LV, int n_alloc) { return (size_t)kLucyWarps * lucy_warp_bytes(LV, n_alloc); }

cudaError_t lucy_kernel_attributes(int max_smem) {
  return cudaFuncSetAttribute(lucy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

cudaError_t launch_lucy_taps(const float* V32, int LV, int R, float* v4, float* S_dev, cudaStream_t st) {
  lucy_taps_kernel<<<1, 128, 0, st>>>(V32, LV, R, (LV + 3) / 4, v4, S_dev);
  return cudaGetLastError();
}

cudaError_t launch_lucy(const float* v4_host, float S, int LV, int R, double dt, double g, int n_waveforms, int n_alloc,
                        const float* samples, const int32_t* offsets, const double* t_origin, int n_iter, float thresh,
                        float* q_out, int32_t* T_lo, int32_t* T_hi, double* t0, int32_t* z, int32_t* n_z, int z_stride,
                        int* status, cudaStream_t st) {
  if (n_waveforms <= 0) return cudaSuccess;
  const int jv = (LV + 3) / 4;
  if (jv > kLucyMaxJV) return cudaErrorInvalidValue;
  LucyArgs A;
  for (int j = 0; j < kLucyMaxJV; ++j)
    A.taps[j] = j < jv ? make_float4(v4_host[4 * j], v4_host[4 * j + 1], v4_host[4 * j + 2], v4_host[4 * j + 3])
                       : make_float4(0.f, 0.f, 0.f, 0.f);
  A.samples = samples; A.offsets = offsets; A.t_origin = t_origin;
  A.n_waveforms = n_waveforms; A.n_alloc = n_alloc; A.n_iter = n_iter; A.LV = LV; A.R = R; A.z_stride = z_stride;
  A.thresh = thresh; A.inv_S = 1.0f / S; A.dt = dt; A.g = g;
  A.q_out = q_out; A.T_lo = T_lo; A.T_hi = T_hi; A.t0 = t0; A.z = z; A.n_z = n_z; A.status = status;
  const unsigned blocks = (unsigned)((n_waveforms + kLucyWarps - 1) / kLucyWarps);
  lucy_kernel<<<blocks, kLucyWarps * 32, lucy_smem_bytes(LV, n_alloc), st>>>(A);
  return cudaGetLastError();
}

}  // namespace fsmp
