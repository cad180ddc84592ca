// fsmp_chain.cu -- the FSMP chain kernel (arXiv 2403.03156, Sec. 2.4 and Appendix A.1).
//
// One CTA runs one chain at a time and loops over the chains of its launch (persistent).
// The chain state lives in shared memory: the packed lower triangle of Sigma^-1 (n(n+1)/2
// entries; or a per-CTA slice of global scratch for windows too long for shared memory),
// s = Sigma^-1 y, y = w - U(z) (FP32 mode), u = sum_k a_k, and the PE list.
//
// Every 32 steps the CTA draws the Philox4x64-10 blocks of the next 32 steps in parallel and
// turns them into the step's Box-Muller normals and log uniforms (one thread per step). A step:
//   A  (warp 0)  MH move on t0 (log phi table lookups, warp sum); jump choice and proposal
//                (birth: warp-parallel search of the cumulative phi, h(t) = phi(t - t0) /
//                Phi_T); gather a_- and a_+ on the union U of their supports.
//   B  (all)     M = a^T Sigma^-1 a over the lower triangle of the U x U block and g = a^T s
//                (per-lane sums, Neumaier-compensated in FP32, then warp shuffles).
//   C  (lane 0)  Delta nu = -1/2 (Delta T + Delta R) with Delta T = log det(I + Lambda M)
//                (Eq. (17) by Sylvester's identity) and Delta R = -2 lambda^T g + lambda^T M
//                lambda - r^T B r, r = g - M lambda, B = (I + Lambda M)^-1 Lambda (Eqs. (12),
//                (16)); log acceptance of Eqs. (birth) / (death) / (update); MH decision.
//   On accept:
//   D  (all)     c = Sigma^-1 a (k lanes per row), b = c B.
//   E  (all)     Sigma^-1 -= c B c^T (Eq. (12); warp per row, lanes over columns),
//                s -= c (lambda + B r), y -= a lambda (Eq. (DeltaU)), u += a_+ - a_-,
//                log|Sigma| += Delta T, log-likelihood += Delta nu (both FP64).
//   R  (FP32 mode, every refresh_every accepted moves) FP64 rebuild of Sigma^-1, s, y, u,
//                log|Sigma| and the log-likelihood from z (capacitance form), with the drift
//                of the incremental state recorded.
// The arithmetic of Delta nu is Eqs. (16)-(18) rearranged so that Lambda^-1 never appears
// (equal in exact arithmetic; it avoids 1/sigma_q^2 cancellations). In FP32 mode the per-step
// scalar arithmetic is FP32 too (this part executes FP64 at a small fraction of the FP32
// rate); FP64 holds the log-likelihood, log|Sigma| and the refresh.
#include <math.h>

#include "fsmp_internal.h"

namespace fsmp {
namespace {

constexpr int kRB = 32;  // steps per batch of random draws

__host__ __device__ __forceinline__ size_t rowbase(int x) { return (size_t)x * (size_t)(x + 1) / 2; }

// Tables at the state precision.
template <typename T> struct Tab;
template <> struct Tab<double> {
  __device__ static const double* V(const DevModel& M) { return M.V64; }
  __device__ static const double* phi(const DevModel& M) { return M.phi; }
  __device__ static const double* logphi(const DevModel& M) { return M.logphi; }
  __device__ static const double* cphi(const DevModel& M) { return M.cphi; }
};
template <> struct Tab<float> {
  __device__ static const float* V(const DevModel& M) { return M.V32; }
  __device__ static const float* phi(const DevModel& M) { return M.phi32; }
  __device__ static const float* logphi(const DevModel& M) { return M.logphi32; }
  __device__ static const float* cphi(const DevModel& M) { return M.cphi32; }
};

template <typename T> __device__ __forceinline__ T logphi_at(const DevModel& M, int d) {
  return (d < -M.D || d > M.D) ? (T)-INFINITY : Tab<T>::logphi(M)[d + M.D];
}
template <typename T> __device__ __forceinline__ T phi_at(const DevModel& M, int d) {
  return (d < -M.D || d > M.D) ? (T)0 : Tab<T>::phi(M)[d + M.D];
}
template <typename T> __device__ __forceinline__ T cphi_at(const DevModel& M, int d) {
  if (d < -M.D) return (T)0;
  if (d > M.D) return Tab<T>::cphi(M)[2 * M.D];
  return Tab<T>::cphi(M)[d + M.D];
}

// Per-lane sums: plain in FP64, Neumaier-compensated in FP32.
template <typename T> struct CSum;
template <> struct CSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct CSum<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
  }
  __device__ __forceinline__ float value() const { return s + c; }
};

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_maxf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// sum_{c in [c0, c1)} e_c a_c for both halves of the interleaved a pair, four independent
// partial sums so the loads of consecutive elements overlap.
template <typename T>
__device__ __forceinline__ void dot2_range(const T* __restrict__ row, const typename Vec2<T>::type* __restrict__ a2v,
                                           int c0, int c1, T& rm, T& rp) {
  T m0 = 0, m1 = 0, m2 = 0, m3 = 0, p0 = 0, p1 = 0, p2 = 0, p3 = 0;
  int c = c0;
  for (; c + 3 < c1; c += 4) {
    const T e0 = row[c], e1 = row[c + 1], e2 = row[c + 2], e3 = row[c + 3];
    const auto a0 = a2v[c], a1 = a2v[c + 1], a2 = a2v[c + 2], a3 = a2v[c + 3];
    m0 += e0 * a0.x; p0 += e0 * a0.y;
    m1 += e1 * a1.x; p1 += e1 * a1.y;
    m2 += e2 * a2.x; p2 += e2 * a2.y;
    m3 += e3 * a3.x; p3 += e3 * a3.y;
  }
  for (; c < c1; ++c) {
    const T e = row[c];
    const auto a = a2v[c];
    m0 += e * a.x; p0 += e * a.y;
  }
  rm = (m0 + m1) + (m2 + m3);
  rp = (p0 + p1) + (p2 + p3);
}

// Random quantities of one step, drawn ahead in batches of kRB steps.
template <typename T> struct StepRand {
  T z1, lu0, u3, u4, z2, lu;  // t0 shift normal, log u2, jump type, PE choice, update normal, log u7
};

// Scalars of the chain in flight (shared memory). Per-step scalars are at the state
// precision T; the log-likelihood and log|Sigma| accumulate in FP64.
template <typename T>
struct ChainScalars {
  const float* w;
  fsmp_summary* out;
  fsmp_trace* trace;
  double lambda0, t_origin;
  uint64_t seed, wf_id;
  int n, T_lo, T_hi, k0_lo, k0_hi, n_steps, burn_in, invalid;
  int d0, win_ok;  // grid-offset window of the phi tables held in shared memory
  // state (the step loop keeps N and k0 in warp 0's registers; these copies serve the other
  // warps, the refresh and the bookkeeping)
  int N, k0, status, n_acc_refresh;
  double logdet, logL;
  // proposal of the current step, broadcast to the other warps
  int valid, u_lo, u_len, has_m, has_p, apply;
  // decision, broadcast for the accept phases
  T B11, B12, B22, v0, v1;
  // snapshot of the last decided step for the bookkeeping warp
  int bk_pending, bk_step, bk_N, bk_k0, bk_jump, bk_flags, bk_status, bk_ulen, bk_apply;
  T bk_la0, bk_lu0, bk_la, bk_lu, bk_dnu;
  T dT_pending, dnu_pending;  // Delta T, Delta nu of an applied step (added in FP64 by thread 0)
  // summaries: exact integer sums for N and the t0 grid index; the charge summary is held
  // between state changes and added with its holding time
  long long sN, sN2, sK, sK2;
  double q_cur, sQ, sQ2;
  // the Wasserstein scalar of the PE times (Sec. 3.2), held like the charge summary: St is the
  // sum of |t_k| in grid units over the PEs of the state
  long long St;
  double wt_cur, sWt, sWt2;
  int q_from, q_pending, pending_step;
  unsigned long long alg_words;
  double drift_max;
  double lambda_hat;
  int acc[3], prop[3], acc_t0, prop_t0, n_refresh, refresh_fail;
};

template <typename T> struct Layout {
  ChainScalars<T>* S;
  T* red;                   // [kMaxWarps][8] per-warp partial sums (T view of redd)
  double* redd;             // the same region as [kMaxWarps][8] doubles (block-reduction scratch)
  int* list;                // [n_cap]
  int* hist;                // counts of N after burn-in [n_cap + 1]
  StepRand<T>* rnd;         // [kRB]
  unsigned long long* raw;  // [2 kRB][4] Philox output of a batch
  T* a2;                    // [LU][2]: (a_-, a_+) interleaved
  T* Vs;                    // [Lt] SER table (copied once per CTA)
  T* lgN;                   // [n_cap + 2] log(i)
  T* lPhi;                  // [win_extra] log(Phi_T(t0) g) on the chain's t0 grid
  T* lphw;                  // [win] log phi on the chain's grid-offset window
  T* cphw;                  // [win] cumulative phi on the same window
  T* s;                     // [n]
  T* slo;                   // [n] FP32 mode: low part of s (s = s + slo, compensated updates)
  T* y;                     // [n] (FP32 mode)
  T* u;                     // [n]
  T* c2;                    // [n][2]: (c_-, c_+)
  T* b2;                    // [n][2]: (c B)_-, (c B)_+   (c2 and b2 are contiguous)
  T* P;                     // packed Sigma^-1, when held in shared memory
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline int win_alloc(int n_alloc, int R, int win_extra) { return n_alloc * R + win_extra; }

template <typename T>
__host__ __device__ inline size_t layout_bytes(int n_alloc, int n_cap, int LU, bool with_P, int Lt, int win) {
  size_t b = align16(sizeof(ChainScalars<T>));
  b += align16(sizeof(double) * kMaxWarps * 8);
  b += align16(sizeof(int) * n_cap);
  b += align16(sizeof(int) * (n_cap + 1));
  b += align16(sizeof(StepRand<T>) * kRB);
  b += align16(sizeof(unsigned long long) * 2 * kRB * 4);
  b += align16(sizeof(T) * 2 * LU);
  b += align16(sizeof(T) * Lt) + 2 * align16(sizeof(T) * win);
  b += align16(sizeof(T) * (n_cap + 2)) + align16(sizeof(T) * (win - n_alloc * 0));
  b += (sizeof(T) == 4 ? 4 : 2) * align16(sizeof(T) * n_alloc);
  b += align16(sizeof(T) * 4 * n_alloc);
  if (with_P) b += align16(sizeof(T) * rowbase(n_alloc));
  return b;
}

template <typename T>
__device__ inline Layout<T> carve(unsigned char* base, int n_alloc, int n_cap, int LU, int Lt, int win) {
  Layout<T> L;
  size_t o = 0;
  L.S = reinterpret_cast<ChainScalars<T>*>(base + o); o += align16(sizeof(ChainScalars<T>));
  L.red = reinterpret_cast<T*>(base + o);
  L.redd = reinterpret_cast<double*>(base + o);
  o += align16(sizeof(double) * kMaxWarps * 8);
  L.list = reinterpret_cast<int*>(base + o); o += align16(sizeof(int) * n_cap);
  L.hist = reinterpret_cast<int*>(base + o); o += align16(sizeof(int) * (n_cap + 1));
  L.rnd = reinterpret_cast<StepRand<T>*>(base + o); o += align16(sizeof(StepRand<T>) * kRB);
  L.raw = reinterpret_cast<unsigned long long*>(base + o); o += align16(sizeof(unsigned long long) * 2 * kRB * 4);
  L.a2 = reinterpret_cast<T*>(base + o); o += align16(sizeof(T) * 2 * LU);
  L.Vs = reinterpret_cast<T*>(base + o); o += align16(sizeof(T) * Lt);
  L.lgN = reinterpret_cast<T*>(base + o); o += align16(sizeof(T) * (n_cap + 2));
  L.lPhi = reinterpret_cast<T*>(base + o); o += align16(sizeof(T) * win);
  L.lphw = reinterpret_cast<T*>(base + o); o += align16(sizeof(T) * win);
  L.cphw = reinterpret_cast<T*>(base + o); o += align16(sizeof(T) * win);
  L.s = reinterpret_cast<T*>(base + o); o += align16(sizeof(T) * n_alloc);
  if (sizeof(T) == 4) { L.slo = reinterpret_cast<T*>(base + o); o += align16(sizeof(T) * n_alloc); }
  else L.slo = nullptr;
  if (sizeof(T) == 4) { L.y = reinterpret_cast<T*>(base + o); o += align16(sizeof(T) * n_alloc); }
  else L.y = nullptr;
  L.u = reinterpret_cast<T*>(base + o); o += align16(sizeof(T) * n_alloc);
  L.c2 = reinterpret_cast<T*>(base + o);
  L.b2 = L.c2 + 2 * n_alloc;
  o += align16(sizeof(T) * 4 * n_alloc);
  L.P = reinterpret_cast<T*>(base + o);
  return L;
}

// Support of a PE at grid index j inside a window of n samples: samples s with
// 0 <= s R - j < Lt, i.e. [ceil(j / R), floor((j + Lt - 1) / R)] clipped to [0, n).
// floor(a / R) by an IEEE FP32 division: exact for |a| < 2^22 since a / R is at least 1/R
// away from the next integer when it is not one.
__device__ __forceinline__ int floordiv_small(int a, float Rf) { return (int)floorf((float)a / Rf); }

__device__ __forceinline__ void pe_support(const DevModel& M, int n, int j, int& lo, int& hi) {
  const float Rf = (float)M.R;
  lo = max(0, floordiv_small(j + M.R - 1, Rf));
  hi = min(n, floordiv_small(j + M.Lt - 1, Rf) + 1);
  if (hi < lo) hi = lo;
}

// Smallest j in [T_lo, T_hi) with cphi(j - k0) - base > target (warp-cooperative 32-ary
// search); if rounding leaves none, the last j of T with phi > 0 (the oracle's rule).
template <typename T, typename CF, typename LF>
__device__ int birth_search(CF cph, LF lph, int T_lo, int T_hi, int k0, T base, T target, int lane) {
  int lo = T_lo, hi = T_hi - 1;
  if ((cph(hi - k0) - base) > target) {
    while (lo < hi) {
      const int len = hi - lo + 1;
      const int step = (len + 31) / 32;
      const int p = min(hi, lo + (lane + 1) * step - 1);
      const bool pred = (cph(p - k0) - base) > target;
      const unsigned b = __ballot_sync(0xffffffffu, pred);
      const int f = __ffs(b) - 1;  // b != 0: the top probe (hi) is true
      const int new_lo = lo + f * step;
      hi = min(hi, lo + (f + 1) * step - 1);
      lo = new_lo;
    }
    return lo;
  }
  int last = -1;
  for (int top = T_hi - 1; top >= T_lo; top -= 32) {
    const int j = top - lane;
    const bool ok = j >= T_lo && lph(j - k0) > (T)-INFINITY;  // phi > 0
    const unsigned b = __ballot_sync(0xffffffffu, ok);
    if (b) { last = top - (__ffs(b) - 1); break; }
  }
  return last;
}

// Draws of steps [step0, step0 + kRB): Philox blocks (step, 0|1, 0, 0) under key
// (seed, wf_id), then Box-Muller and logs (one thread per step).
template <typename T>
__device__ void draw_batch(Layout<T>& L, const ChainScalars<T>& S, int step0) {
  const int tid = threadIdx.x;
  for (int b = tid; b < 2 * kRB; b += blockDim.x) {
    uint64_t c[4] = {(uint64_t)(step0 + (b >> 1)), (uint64_t)(b & 1), 0, 0};
    philox4x64_10(c, S.seed, S.wf_id);
    for (int k = 0; k < 4; ++k) L.raw[4 * b + k] = c[k];
  }
  __syncthreads();
  for (int t = tid; t < kRB; t += blockDim.x) {
    double u[8];
    for (int k = 0; k < 4; ++k) {
      u[k] = u01_from_bits(L.raw[8 * t + k]);
      u[4 + k] = u01_from_bits(L.raw[8 * t + 4 + k]);
    }
    StepRand<T> r;
    if (sizeof(T) == 8) {
      r.z1 = (T)(sqrt(-2.0 * log(u[0])) * cos(kTwoPi * u[1]));
      r.lu0 = (T)log(u[2]);
      r.z2 = (T)(sqrt(-2.0 * log(u[5])) * cos(kTwoPi * u[6]));
      r.lu = (T)log(u[7]);
    } else {
      r.z1 = (T)(sqrtf(-2.0f * logf((float)u[0])) * cosf(6.2831853f * (float)u[1]));
      r.lu0 = (T)logf((float)u[2]);
      r.z2 = (T)(sqrtf(-2.0f * logf((float)u[5])) * cosf(6.2831853f * (float)u[6]));
      r.lu = (T)logf((float)u[7]);
    }
    r.u3 = (T)u[3];
    r.u4 = (T)u[4];
    L.rnd[t] = r;
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------------
// FP64 refresh (FP32 mode). Capacitance form of Sigma(z) = sigma_eps^2 I + sigma_q^2 A A^T
// (A = [a_1..a_N]): with C = (sigma_eps^2 / sigma_q^2) I_N + A^T A = L L^T and W = L^-1 A^T,
//   Sigma^-1 = (I - W^T W) / sigma_eps^2,     s = Sigma^-1 y = (y - W^T (W y)) / sigma_eps^2,
//   log|Sigma| = n log sigma_eps^2 + N log(sigma_q^2 / sigma_eps^2) + 2 sum_k log L_kk,
//   y^T Sigma^-1 y = (|y|^2 - |W y|^2) / sigma_eps^2          (Woodbury applied to all of A).
// The PEs are sorted by time so that C, L and W have an envelope structure (a PE only
// overlaps its neighbours; W[k, x] = 0 before the first PE covering sample x).
// Workspace (global, per CTA): C/L packed, W y, y (FP64), W, and integer index arrays.
// ------------------------------------------------------------------------------------
__host__ __device__ inline size_t refresh_doubles(int n_cap, int n_alloc) {
  return rowbase(n_cap) + (size_t)n_cap + (size_t)n_alloc + (size_t)n_cap * n_alloc;
}
__host__ __device__ inline size_t refresh_ws_bytes(int n_cap, int n_alloc) {
  return align16(refresh_doubles(n_cap, n_alloc) * sizeof(double)) +
         align16(sizeof(int) * (4 * (size_t)n_cap + n_alloc));
}

template <typename T>
__device__ void refresh_state(const DevModel& M, Layout<T>& L, T* P, unsigned char* ws, int n, int n_alloc) {
  ChainScalars<T>& S = *L.S;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  const int ncap = M.n_cap, N = S.N, R = M.R;
  double* Cp = reinterpret_cast<double*>(ws);
  double* vv = Cp + rowbase(ncap);
  double* y64 = vv + ncap;
  double* W = y64 + n_alloc;
  int* slist = reinterpret_cast<int*>(ws + align16(refresh_doubles(ncap, n_alloc) * sizeof(double)));
  int* slo = slist + ncap;
  int* shi = slo + ncap;
  int* sfirst = shi + ncap;
  int* xA = sfirst + ncap;
  const double* V64 = M.V64;
  const float* __restrict__ w = S.w;
  // R0: PEs sorted by grid index (rank sort, ties by slot), their supports
  for (int k = tid; k < N; k += nthr) {
    const int jk = L.list[k];
    int r = 0;
    for (int m = 0; m < N; ++m) {
      const int jm = L.list[m];
      r += (jm < jk) || (jm == jk && m < k);
    }
    slist[r] = jk;
  }
  __syncthreads();
  for (int k = tid; k < N; k += nthr) {
    int lo, hi;
    pe_support(M, n, slist[k], lo, hi);
    slo[k] = lo;
    shi[k] = hi;
  }
  __syncthreads();
  // envelope: first PE overlapping each PE; first PE covering each sample (N if none)
  for (int k = tid; k < N; k += nthr) {
    int f = k;
    while (f > 0 && max(slo[f - 1], slo[k]) < min(shi[f - 1], shi[k])) --f;
    sfirst[k] = f;
  }
  for (int x = tid; x < n; x += nthr) {
    int k = 0;
    while (k < N && !(slo[k] <= x && x < shi[k])) ++k;
    xA[x] = k;
  }
  __syncthreads();
  // R1: y = w - mu_q sum_k a_k (FP64), u = sum_k a_k
  for (int x = tid; x < n; x += nthr) {
    double uu = 0.0;
    for (int k = xA[x]; k < N && slo[k] <= x; ++k)
      if (x < shi[k]) uu += V64[x * R - slist[k]];
    const double yy = (double)w[x] - M.mu_q * uu;
    y64[x] = yy;
    L.y[x] = (T)yy;
    L.u[x] = (T)uu;
  }
  // R2: C = (se2 / sq2) I + A^T A inside the envelope (packed lower)
  const size_t npairs = rowbase(N);
  for (size_t p = tid; p < npairs; p += nthr) {
    int k = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
    while (rowbase(k + 1) <= p) ++k;
    while (rowbase(k) > p) --k;
    const int l = (int)(p - rowbase(k));
    double val = (k == l) ? M.se2 / M.sq2 : 0.0;
    if (l >= sfirst[k]) {
      const int s0 = max(slo[k], slo[l]), s1 = min(shi[k], shi[l]);
      const int jk = slist[k], jl = slist[l];
      for (int sidx = s0; sidx < s1; ++sidx) val += V64[sidx * R - jk] * V64[sidx * R - jl];
    }
    Cp[p] = val;
  }
  if (tid == 0) S.refresh_fail = 0;
  __syncthreads();
  // R3: envelope Cholesky C = L L^T in place
  for (int j = 0; j < N; ++j) {
    const size_t rj = rowbase(j);
    if (tid == 0) {
      double d = Cp[rj + j];
      for (int m = sfirst[j]; m < j; ++m) d -= Cp[rj + m] * Cp[rj + m];
      if (!(d > 0.0)) S.refresh_fail = 1;
      Cp[rj + j] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double ljj = Cp[rj + j];
    for (int i = j + 1 + tid; i < N; i += nthr) {
      if (sfirst[i] > j) continue;
      const size_t ri = rowbase(i);
      double d = Cp[ri + j];
      for (int m = max(sfirst[i], sfirst[j]); m < j; ++m) d -= Cp[ri + m] * Cp[rj + m];
      Cp[ri + j] = d / ljj;
    }
    __syncthreads();
  }
  if (S.refresh_fail) {  // keep the incremental state; flag it
    __syncthreads();
    if (tid == 0) { S.status |= FSMP_ST_DRIFT; S.n_acc_refresh = 0; }
    __syncthreads();
    return;
  }
  // R4: W = L^-1 A^T, one column (sample) per thread, forward substitution in the envelope
  for (int x = tid; x < n; x += nthr) {
    const int k0x = xA[x];
    for (int k = k0x; k < N; ++k) {
      const size_t rk = rowbase(k);
      double d = (x >= slo[k] && x < shi[k]) ? V64[x * R - slist[k]] : 0.0;
      for (int m = max(k0x, sfirst[k]); m < k; ++m) d -= Cp[rk + m] * W[(size_t)m * n_alloc + x];
      W[(size_t)k * n_alloc + x] = d / Cp[rk + k];
    }
  }
  __syncthreads();
  // R5: v = W y
  for (int k = tid; k < N; k += nthr) {
    double d = 0.0;
    for (int x = 0; x < n; ++x)
      if (xA[x] <= k) d += W[(size_t)k * n_alloc + x] * y64[x];
    vv[k] = d;
  }
  __syncthreads();
  // R6: new s and diagonal of Sigma^-1 (FP64), drift of the incremental state, |y|^2
  float ds = 0.f, ms = 0.f, dd = 0.f, md = 0.f;
  double ysq = 0.0;
  for (int x = tid; x < n; x += nthr) {
    double t = y64[x], q = 0.0;
    for (int k = xA[x]; k < N; ++k) {
      const double wk = W[(size_t)k * n_alloc + x];
      t -= wk * vv[k];
      q += wk * wk;
    }
    const double s_new = t * M.inv_se2, d_new = (1.0 - q) * M.inv_se2;
    ds = fmaxf(ds, fabsf((float)(s_new - ((double)L.s[x] + (double)L.slo[x]))));
    ms = fmaxf(ms, fabsf((float)s_new));
    dd = fmaxf(dd, fabsf((float)d_new - (float)P[rowbase(x) + x]));
    md = fmaxf(md, fabsf((float)d_new));
    L.s[x] = (T)s_new;
    L.slo[x] = (T)(s_new - (double)(T)s_new);
    ysq += y64[x] * y64[x];
  }
  ds = warp_maxf(ds); ms = warp_maxf(ms); dd = warp_maxf(dd); md = warp_maxf(md);
  ysq = warp_sum<double>(ysq);
  double* redd = L.redd;  // 5 nw doubles
  if (lane == 0) {
    redd[5 * warp + 0] = ds; redd[5 * warp + 1] = ms; redd[5 * warp + 2] = dd; redd[5 * warp + 3] = md;
    redd[5 * warp + 4] = ysq;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0, b = 0, c = 0, d = 0, e = 0;
    for (int i = 0; i < nw; ++i) {
      a = fmax(a, redd[5 * i]); b = fmax(b, redd[5 * i + 1]); c = fmax(c, redd[5 * i + 2]);
      d = fmax(d, redd[5 * i + 3]); e += redd[5 * i + 4];
    }
    const double drift = fmax(b > 0 ? a / b : 0.0, d > 0 ? c / d : 0.0);
    S.drift_max = fmax(S.drift_max, drift);
    if (drift > M.drift_tol) S.status |= FSMP_ST_DRIFT;
    double vsq = 0.0, ld = 0.0;
    for (int k = 0; k < N; ++k) { vsq += vv[k] * vv[k]; ld += log(Cp[rowbase(k) + k]); }
    S.logdet = n * log(M.se2) + N * log(M.sq2 / M.se2) + 2.0 * ld;
    S.logL = -0.5 * (n * kLog2Pi + S.logdet + (e - vsq) * M.inv_se2);
    S.n_refresh++;
    S.n_acc_refresh = 0;
  }
  __syncthreads();
  // R7: Sigma^-1 = (I - W^T W) / sigma_eps^2, four rows of W at a time staged in shared memory
  {
    const size_t np = rowbase(n);
    for (size_t e = tid; e < np; e += nthr) P[e] = (T)0;
    __syncthreads();
    for (int x = tid; x < n; x += nthr) P[rowbase(x) + x] = (T)M.inv_se2;
    __syncthreads();
    T* stage = L.c2;  // [n][4]
    const T nis = (T)(-M.inv_se2);
    for (int kb = 0; kb < N; kb += 4) {
      for (int x = tid; x < n; x += nthr)
        for (int i = 0; i < 4; ++i) {
          const int k = kb + i;
          stage[4 * x + i] = (k < N && k >= xA[x]) ? (T)W[(size_t)k * n_alloc + x] : (T)0;
        }
      __syncthreads();
      for (int x = warp; x < n; x += nw) {
        const T wx0 = stage[4 * x], wx1 = stage[4 * x + 1], wx2 = stage[4 * x + 2], wx3 = stage[4 * x + 3];
        if (wx0 == (T)0 && wx1 == (T)0 && wx2 == (T)0 && wx3 == (T)0) continue;
        T* Prow = P + rowbase(x);
        for (int v = lane; v <= x; v += 32) {
          const T d = wx0 * stage[4 * v] + wx1 * stage[4 * v + 1] + wx2 * stage[4 * v + 2] + wx3 * stage[4 * v + 3];
          Prow[v] += nis * d;
        }
      }
      __syncthreads();
    }
  }
  // charge summary partial u^T s for the pending step
  {
    CSum<T> qs;
    for (int x = tid; x < n; x += nthr) {
      qs.add(L.u[x] * L.s[x]);
      qs.add(L.u[x] * L.slo[x]);
    }
    const T v = warp_sum<T>(qs.value());
    if (lane == 0) L.red[warp * 8 + 5] = v;
  }
  __syncthreads();
}

// Add the charge summary held since the last state change (lane 0 of warp 0).
// The Wasserstein scalar of the PE times is held with it: with a dummy PE at t = 0 added, the
// 1-Wasserstein distance from the sequence to the dummy alone, sum_k |t_k| / (N + 1).
template <typename T>
__device__ __forceinline__ void close_charge_hold(ChainScalars<T>& S, int upto) {
  const int hold = upto - max(S.q_from, S.burn_in);
  if (hold > 0) {
    S.sQ += S.q_cur * hold;
    S.sQ2 += S.q_cur * S.q_cur * hold;
    S.sWt += S.wt_cur * hold;
    S.sWt2 += S.wt_cur * S.wt_cur * hold;
  }
}

// Bookkeeping of one decided step from its snapshot (one thread): counters, status, the
// algorithmic-byte count, summary sums after burn-in, the trace record. It runs on a warp that
// is idle while warp 0 works on the next proposal.
template <typename T>
__device__ void bookkeep(ChainScalars<T>& S, int* hist) {
  const int jump = S.bk_jump, fl = S.bk_flags;
  S.prop[jump]++;
  if (fl & 1) { S.prop_t0++; if (fl & 2) S.acc_t0++; }
  if ((fl & 4) && !(fl & 8)) S.acc[jump]++;
  S.status |= S.bk_status;
  if (S.bk_ulen > 0) {
    const unsigned long long ul = S.bk_ulen, nn = S.n;
    S.alg_words += ul * (ul + 1) / 2 + ul;                             // U block of Sigma^-1, s on U
    if (S.bk_apply) S.alg_words += nn * ul + nn * (nn + 1) + 2 * nn;   // c, packed rank-2 r+w, s r+w
  }
  if (S.bk_step >= S.burn_in) {
    const long long Nn = S.bk_N, kk = S.bk_k0;
    S.sN += Nn; S.sN2 += Nn * Nn; S.sK += kk; S.sK2 += kk * kk;
    hist[S.bk_N] += 1;
  }
  if (S.trace) {
    fsmp_trace tr;
    tr.la0 = (double)S.bk_la0; tr.lu0 = (double)S.bk_lu0; tr.la = (double)S.bk_la; tr.lu = (double)S.bk_lu;
    tr.dnu = (double)S.bk_dnu; tr.N = S.bk_N; tr.k0 = S.bk_k0; tr.jump = jump; tr.flags = fl;
    S.trace[S.bk_step] = tr;
  }
  S.bk_pending = 0;
}

template <typename T, bool SMEM_P>
__global__ void __launch_bounds__(512) chain_kernel(DevModel M, BatchView B, T* gP, size_t gP_stride,
                                                    unsigned char* rws, size_t rws_stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n_alloc = B.n_max;
  const int win = win_alloc(n_alloc, M.R, M.win_extra);
  Layout<T> L = carve<T>(smem_raw, n_alloc, M.n_cap, M.LU, M.Lt, win);
  ChainScalars<T>& S = *L.S;
  T* __restrict__ P = SMEM_P ? L.P : gP + (size_t)blockIdx.x * gP_stride;
  unsigned char* ws = rws ? rws + (size_t)blockIdx.x * rws_stride : nullptr;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int bk_warp = nw > 1 ? 1 : 0;
  constexpr bool fp32 = sizeof(T) == 4;
  using T2 = typename Vec2<T>::type;
  // per-CTA tables: the SER and log(i), i = 1 .. n_cap + 1 (log(0) unused)
  for (int m = tid; m < M.Lt; m += blockDim.x) L.Vs[m] = Tab<T>::V(M)[m];
  for (int i = tid; i < M.n_cap + 2; i += blockDim.x) L.lgN[i] = i > 0 ? (T)log((double)i) : (T)0;
  const T* __restrict__ V = L.Vs;
  const T2* __restrict__ a2v = reinterpret_cast<const T2*>(L.a2);

  for (int ci = blockIdx.x; ci < B.n_waveforms; ci += gridDim.x) {
    const int wi = B.order ? B.order[ci] : ci;
    // ------------------------------------------------------------- chain set-up
    if (tid == 0) {
      int o0 = B.offsets[wi], o1 = B.offsets[wi + 1];
      S.n = o1 - o0;
      S.w = B.samples + o0;
      S.lambda0 = B.lambda0[wi];
      S.t_origin = B.t_origin ? B.t_origin[wi] : 0.0;
      S.T_lo = B.T_lo ? B.T_lo[wi] : 0;
      S.T_hi = B.T_hi ? B.T_hi[wi] : S.n * M.R;
      S.k0_lo = (int)ceil((M.t0_lo - S.t_origin) / M.g - 1e-9);
      S.k0_hi = (int)floor((M.t0_hi - S.t_origin) / M.g + 1e-9);
      double t0i = B.t0_init ? B.t0_init[wi] : NAN;
      if (!isnan(t0i)) {
        double kk = rint((t0i - S.t_origin) / M.g);
        kk = fmin(fmax(kk, (double)S.k0_lo), (double)S.k0_hi);
        S.k0 = (int)kk;
      } else {
        S.k0 = S.k0_lo + (S.k0_hi - S.k0_lo) / 2;
      }
      S.seed = B.seeds ? B.seeds[wi] : B.seed;
      S.wf_id = B.wf_ids ? B.wf_ids[wi] : B.index_base + (uint64_t)wi;
      S.n_steps = B.n_steps_arr ? B.n_steps_arr[wi] : B.n_steps;
      S.burn_in = B.burn_in_arr ? B.burn_in_arr[wi] : B.burn_in;
      S.out = B.out + wi;
      S.trace = B.trace ? B.trace + (B.trace_off ? B.trace_off[wi] : (int64_t)wi * S.n_steps) : nullptr;
      S.invalid = (S.n < 1 || S.n > n_alloc || S.T_hi <= S.T_lo || S.k0_hi < S.k0_lo ||
                   !(S.lambda0 > 0.0) || S.n_steps < 0 || S.burn_in < 0 || (fp32 && ws == nullptr) ||
                   S.k0_hi - S.k0_lo + 1 > M.win_extra);
      // phi offsets d = j - t0 the chain can meet: j in T, t0 in its prior range (and one below
      // T for the cumulative table)
      S.d0 = S.T_lo - S.k0_hi - 1;
      S.win_ok = (long long)(S.T_hi - 1 - S.k0_lo) - S.d0 + 1 <= win;
      S.N = 0; S.status = 0; S.n_acc_refresh = 0;
      S.sN = S.sN2 = S.sK = S.sK2 = 0;
      S.q_cur = 0.0; S.sQ = S.sQ2 = 0.0; S.q_from = 0; S.q_pending = 0; S.bk_pending = 0;
      S.St = 0; S.wt_cur = 0.0; S.sWt = S.sWt2 = 0.0;
      for (int k = 0; k < 3; ++k) { S.acc[k] = 0; S.prop[k] = 0; }
      S.acc_t0 = 0; S.prop_t0 = 0; S.n_refresh = 0;
      S.alg_words = 0; S.drift_max = 0.0;
    }
    for (int k = tid; k <= M.n_cap; k += blockDim.x) L.hist[k] = 0;
    __syncthreads();
    if (S.invalid) {
      if (tid == 0) {
        fsmp_summary o;
        o.mean_N = o.var_N = o.mean_t0 = o.var_t0 = o.mean_Q = o.var_Q = o.logL = o.logdet = NAN;
        o.drift_max = 0.0; o.alg_bytes = 0.0; o.lambda_hat = NAN;
        o.mean_wt = o.var_wt = o.mean_we = o.var_we = NAN;
        for (int k = 0; k < 3; ++k) { o.acc[k] = 0; o.prop[k] = 0; }
        o.acc_t0 = o.prop_t0 = o.N_final = o.k0_final = o.n_samples = o.n_refresh = o.reserved = 0;
        o.status = FSMP_ST_INVALID;
        *S.out = o;
        note_chain_done(B, wi);
      }
      __syncthreads();
      continue;
    }
    const int n = S.n;
    const float* __restrict__ w = S.w;
    const int d0 = S.d0, T_lo = S.T_lo, T_hi = S.T_hi, k0_lo = S.k0_lo, k0_hi = S.k0_hi;
    const bool win_ok = S.win_ok;
    const uint64_t seed = S.seed, wf_id = S.wf_id;
    const int n_steps = S.n_steps;
    if (win_ok) {
      const int dlen = T_hi - 1 - k0_lo - d0 + 1;
      for (int i = tid; i < dlen; i += blockDim.x) {
        L.lphw[i] = logphi_at<T>(M, d0 + i);
        L.cphw[i] = cphi_at<T>(M, d0 + i);
      }
    }
    auto LPH = [&](int d) -> T { return win_ok ? L.lphw[d - d0] : logphi_at<T>(M, d); };
    auto CPH = [&](int d) -> T { return win_ok ? L.cphw[d - d0] : cphi_at<T>(M, d); };
    // log(Phi_T(t0) g) on the t0 grid (-inf where Phi_T = 0), from the FP64 tables
    for (int k = tid; k <= k0_hi - k0_lo; k += blockDim.x) {
      const int k0 = k0_lo + k;
      const double tot = cphi_at<double>(M, T_hi - 1 - k0) - cphi_at<double>(M, T_lo - 1 - k0);
      L.lPhi[k] = tot > 0.0 ? (T)log(tot * M.g) : (T)-INFINITY;
    }
    const T log_lambda0 = (T)log(S.lambda0);
    const T Jt = (T)M.J, logJ = (T)M.log_J, inv_gT = (T)M.inv_g;
    // Sigma^-1 = I / sigma_eps^2, s = w / sigma_eps^2, y = w, u = 0 (empty z)
    {
      const size_t np = rowbase(n);
      for (size_t e = tid; e < np; e += blockDim.x) P[e] = (T)0;
      __syncthreads();
      double wsq = 0.0;
      for (int x = tid; x < n; x += blockDim.x) {
        P[rowbase(x) + x] = (T)M.inv_se2;
        const float wx = w[x];
        const double sx = (double)wx * M.inv_se2;
        L.s[x] = (T)sx;
        if constexpr (fp32) {
          L.slo[x] = (T)(sx - (double)(T)sx);
          L.y[x] = (T)wx;
        }
        L.u[x] = (T)0;
        wsq += (double)wx * (double)wx;
      }
      wsq = warp_sum<double>(wsq);
      if (lane == 0) L.redd[warp] = wsq;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int i = 0; i < nw; ++i) t += L.redd[i];
        S.logdet = n * log(M.se2);
        S.logL = -0.5 * (n * kLog2Pi + S.logdet + t * M.inv_se2);
      }
      __syncthreads();
    }

    // warp 0's view of the chain state (uniform across its lanes)
    int N = 0, k0 = S.k0;
    // values warp 0 carries from phase A to phase C of a step
    int jump = 0, valid = 0, noop = 0, kk = -1, jp = -1, t0f = 0, st_a = 0;
    T la_prior = (T)0, la_fixed = (T)0, la0 = (T)0, lu0 = (T)0, lu = (T)0;

    for (int step = 0; step < n_steps; ++step) {
      if (step % kRB == 0) draw_batch<T>(L, S, step);
      // ========================================================= A: warp 0 (and bookkeeping)
      if (warp == bk_warp) {
        if (S.q_pending) {  // charge summary of the state created by the last accepted step
          T part = lane < nw ? L.red[lane * 8 + 5] : (T)0;
          part = warp_sum<T>(part);
          if (lane == 0) {
            close_charge_hold(S, S.pending_step);
            S.q_cur = S.N * M.mu_q + M.sq2 * (double)part;
            S.wt_cur = M.g * (double)S.St / (double)(S.N + 1);
            S.q_from = S.pending_step;
            S.q_pending = 0;
          }
        }
        if (lane == 0 && S.bk_pending) bookkeep(S, L.hist);
        __syncwarp();
      }
      if (warp == 0) {
        const StepRand<T> rd = L.rnd[step % kRB];
        // ---- Gibbs part 1: MH on t0 (Sec. 2.4), uniform prior on its grid range
        la0 = (T)NAN;
        lu0 = rd.lu0;
        t0f = 0;
        st_a = 0;
        if (M.sample_t0) {
          t0f = 1;
          const int Dm = fp32 ? __float2int_rn((float)(rd.z1 * inv_gT)) : __double2int_rn((double)(rd.z1 * inv_gT));
          const int k0p = k0 + Dm;
          if (Dm == 0) {
            la0 = (T)0;
          } else if (k0p < k0_lo || k0p > k0_hi) {
            la0 = (T)-INFINITY;
          } else {
            T part = (T)0;
            for (int k = lane; k < N; k += 32) {
              const int j = L.list[k];
              part += LPH(j - k0p) - LPH(j - k0);
            }
            la0 = warp_sum<T>(part);
          }
          if (lu0 < la0) { k0 = k0p; t0f |= 2; }
        }
        // ---- Gibbs part 2: one RJMCMC jump (Sec. 2.4)
        jump = (N == 0) ? 0 : (rd.u3 < Jt ? 0 : (rd.u3 < (T)2 * Jt ? 1 : 2));
        valid = 0; noop = 0; kk = -1; jp = -1;
        int jm = -1;
        la_prior = (T)0;
        la_fixed = (T)-INFINITY;
        lu = rd.lu;
        const T lphi_t0 = L.lPhi[k0 - k0_lo];  // log(Phi_T(t0) g)
        if (jump == 0) {
          if (N >= M.n_cap) {
            st_a |= FSMP_ST_CAPACITY;
          } else if (lphi_t0 > (T)-INFINITY) {
            const T base = CPH(T_lo - 1 - k0), tot = CPH(T_hi - 1 - k0) - base;
            jp = birth_search<T>(CPH, LPH, T_lo, T_hi, k0, base, rd.u4 * tot, lane);
            valid = jp >= T_lo;
            la_prior = log_lambda0 + lphi_t0 - L.lgN[N + 1] + (N == 0 ? logJ : (T)0);
          }
        } else {
          kk = fp32 ? __float2int_rd((float)(rd.u4 * (T)N)) : __double2int_rd((double)(rd.u4 * (T)N));
          if (kk >= N) kk = N - 1;
          jm = L.list[kk];
          if (jump == 1) {
            valid = 1;
            la_prior = -log_lambda0 - lphi_t0 + L.lgN[N] - (N == 1 ? logJ : (T)0);
          } else {
            const int Dm = fp32 ? __float2int_rn((float)(rd.z2 * inv_gT)) : __double2int_rn((double)(rd.z2 * inv_gT));
            const int jpl = jm + Dm;
            if (Dm == 0) {
              noop = 1;
              la_fixed = (T)0;
            } else if (jpl < T_lo || jpl >= T_hi || LPH(jpl - k0) == (T)-INFINITY) {
              la_fixed = (T)-INFINITY;
            } else {
              jp = jpl;
              valid = 1;
              la_prior = LPH(jp - k0) - LPH(jm - k0);
            }
          }
        }
        // supports and the union interval U
        int mlo = 0, mhi = 0, plo = 0, phi_ = 0, ulo = 0, ulen = 0, hm = 0, hp = 0;
        if (valid) {
          if (jump != 0) { pe_support(M, n, jm, mlo, mhi); hm = mhi > mlo; }
          if (jump != 1) { pe_support(M, n, jp, plo, phi_); hp = phi_ > plo; }
          if (hm && hp) { ulo = min(mlo, plo); ulen = max(mhi, phi_) - ulo; }
          else if (hm) { ulo = mlo; ulen = mhi - mlo; }
          else if (hp) { ulo = plo; ulen = phi_ - plo; }
          if (ulen > M.LU) { valid = 0; la_fixed = (T)-INFINITY; st_a |= FSMP_ST_NONFINITE; ulen = 0; }
        }
        for (int t = lane; t < ulen; t += 32) {
          const int sidx = ulo + t;
          T2 a;
          a.x = (hm && sidx >= mlo && sidx < mhi) ? V[sidx * M.R - jm] : (T)0;
          a.y = (hp && sidx >= plo && sidx < phi_) ? V[sidx * M.R - jp] : (T)0;
          reinterpret_cast<T2*>(L.a2)[t] = a;
        }
        if (lane == 0) {
          S.valid = valid; S.u_lo = ulo; S.u_len = ulen; S.has_m = hm; S.has_p = hp;
        }
      }
      __syncthreads();

      // ========================================================= B: all threads
      const int ulo = S.u_lo, ulen = S.u_len;
      const bool scored = S.valid && ulen > 0;
      if (scored) {
        const int hm = S.has_m, hp = S.has_p;
        using T2 = typename Vec2<T>::type;
        const T2* __restrict__ a2v = reinterpret_cast<const T2*>(L.a2);
        // The lower triangle of the U x U block as row pairs (r, ulen-1-r) of ulen+1 elements,
        // each pair split evenly over H threads. Row r contributes a_r (2 sum_{c<=r} e_rc a_c -
        // e_rr a_r) to a^T Sigma^-1 a (and the mixed form to the cross term).
        T Smm = 0, Smp = 0, Spp = 0, Gm = 0, Gp = 0;
        const int npair = (ulen + 1) >> 1;
        const int H = max(1, (int)blockDim.x / npair);
        const int pr = tid / H, h = tid - pr * H;
        if (pr < npair) {
          const int r1 = pr, r2 = ulen - 1 - pr;
          const int L1 = r1 + 1;
          const int Lseg = (r1 == r2) ? L1 : ulen + 1;
          const int i0 = (h * Lseg) / H, i1 = ((h + 1) * Lseg) / H;
          const int e1 = min(i1, L1);
          if (i0 < e1) {
            const T* __restrict__ Prow = P + rowbase(ulo + r1) + ulo;
            T rm, rp;
            dot2_range<T>(Prow, a2v, i0, e1, rm, rp);
            const T2 ar = a2v[r1];
            const T ed = (r1 >= i0 && r1 < e1) ? Prow[r1] : (T)0;
            Smm += ar.x * ((T)2 * rm - ed * ar.x);
            Spp += ar.y * ((T)2 * rp - ed * ar.y);
            Smp += ar.x * rp + ar.y * rm - ed * ar.x * ar.y;
          }
          if (r2 != r1 && i1 > L1) {
            const int c0 = max(i0, L1) - L1, c1 = i1 - L1;
            const T* __restrict__ Prow = P + rowbase(ulo + r2) + ulo;
            T rm, rp;
            dot2_range<T>(Prow, a2v, c0, c1, rm, rp);
            const T2 ar = a2v[r2];
            const T ed = (r2 >= c0 && r2 < c1) ? Prow[r2] : (T)0;
            Smm += ar.x * ((T)2 * rm - ed * ar.x);
            Spp += ar.y * ((T)2 * rp - ed * ar.y);
            Smp += ar.x * rp + ar.y * rm - ed * ar.x * ar.y;
          }
        }
        for (int t = tid; t < ulen; t += blockDim.x) {
          T sv = L.s[ulo + t];
          if constexpr (fp32) sv += L.slo[ulo + t];
          const T2 a = a2v[t];
          Gm += a.x * sv;
          Gp += a.y * sv;
        }
        const T v0 = hm ? warp_sum<T>(Smm) : (T)0;
        const T v2 = hp ? warp_sum<T>(Spp) : (T)0;
        const T v1 = (hm && hp) ? warp_sum<T>(Smp) : (T)0;
        const T v3 = hm ? warp_sum<T>(Gm) : (T)0;
        const T v4 = hp ? warp_sum<T>(Gp) : (T)0;
        if (lane == 0) {
          T* r = L.red + warp * 8;
          r[0] = v0; r[1] = v1; r[2] = v2; r[3] = v3; r[4] = v4;
        }
      }
      __syncthreads();

      // ========================================================= C: warp 0
      if (warp == 0) {
        T v = (T)0;
        if (scored && lane < 5)
          for (int i = 0; i < nw; ++i) v += L.red[i * 8 + lane];
        const T mmm = __shfl_sync(0xffffffffu, v, 0), mmp = __shfl_sync(0xffffffffu, v, 1);
        const T mpp = __shfl_sync(0xffffffffu, v, 2), gm = __shfl_sync(0xffffffffu, v, 3);
        const T gp = __shfl_sync(0xffffffffu, v, 4);
        T la = la_fixed, dnu = (T)NAN, dT = (T)0;
        int apply = 0, st_c = 0;
        // FP32: every lane evaluates the 2x2 algebra (identical results, no divergence);
        // FP64: lane 0 only (the FP64 pipe is narrow), decision broadcast by shuffle
        if (fp32 || lane == 0) {
          if (valid) {
            const T q = (T)M.sq2, mu = (T)M.mu_q;
            // det(I + Lambda M), Lambda = sigma_q^2 diag(-1, 1)
            const T Dd = ((T)1 - q * mmm) * ((T)1 + q * mpp) + q * q * mmp * mmp;
            if (!(Dd > (T)0)) {
              la = (T)-INFINITY;
              st_c |= FSMP_ST_BADDET;
            } else {
              const T iD = (T)1 / Dd;
              const T B11 = -q * ((T)1 + q * mpp) * iD, B12 = q * q * mmp * iD, B22 = q * ((T)1 - q * mmm) * iD;
              const T rm = gm - mu * (mmp - mmm), rp = gp - mu * (mpp - mmp);
              const T dR = (T)-2 * mu * (gp - gm) + mu * mu * (mmm - (T)2 * mmp + mpp) -
                           (B11 * rm * rm + (T)2 * B12 * rm * rp + B22 * rp * rp);
              dT = log(Dd);
              dnu = (T)-0.5 * (dT + dR);
              if (!isfinite(dnu)) {
                la = (T)-INFINITY;
                st_c |= FSMP_ST_NONFINITE;
              } else {
                la = dnu + la_prior;
                if (lane == 0) {
                  S.B11 = B11; S.B12 = B12; S.B22 = B22;
                  S.v0 = -mu + B11 * rm + B12 * rp;
                  S.v1 = mu + B12 * rm + B22 * rp;
                }
              }
            }
          }
          const int acc = lu < la;
          apply = acc && valid && isfinite(la);
          if (lane == 0) {
            const int Nafter = N + (apply ? (jump == 0 ? 1 : (jump == 1 ? -1 : 0)) : 0);
            S.apply = apply;
            S.bk_step = step; S.bk_N = Nafter; S.bk_k0 = k0; S.bk_jump = jump;
            S.bk_flags = t0f | (acc ? 4 : 0) | ((acc && noop) ? 8 : 0);
            S.bk_status = st_a | st_c; S.bk_ulen = valid ? S.u_len : 0; S.bk_apply = apply;
            S.bk_la0 = la0; S.bk_lu0 = lu0; S.bk_la = la; S.bk_lu = lu; S.bk_dnu = dnu;
            S.bk_pending = 1;
            if (apply) {  // thread 0 applies the list change and the FP64 running sums in E
              S.dT_pending = dT;
              S.dnu_pending = dnu;
            }
          }
        }
        if (!fp32) apply = __shfl_sync(0xffffffffu, apply, 0);
        if (apply) N += (jump == 0 ? 1 : (jump == 1 ? -1 : 0));
      }
      __syncthreads();
      if (!S.apply) continue;

      // ========================================================= D: c = Sigma^-1 a, b = c B
      {
        const int hm = S.has_m, hp = S.has_p;
        const T B11 = S.B11, B12 = S.B12, B22 = S.B22;
        using T2 = typename Vec2<T>::type;
        const T2* __restrict__ a2v = reinterpret_cast<const T2*>(L.a2);
        const int uhi = ulo + ulen;
        // kg consecutive lanes share a row, each taking every kg-th column of U; columns v <= x
        // are read along row x, columns v > x down column x (row v)
        int kg = 1;
        while (kg < 32 && kg * 2 * n <= (int)blockDim.x) kg *= 2;
        const int sub = lane & (kg - 1);
        const int rows_per_pass = (int)blockDim.x / kg;
        const int npass = (n + rows_per_pass - 1) / rows_per_pass;
        for (int pass = 0; pass < npass; ++pass) {
          const int x = pass * rows_per_pass + tid / kg;
          T cm = 0, cp = 0;
          if (x < n) {
            const T* __restrict__ Prow = P + rowbase(x);
            const int vsplit = min(uhi, x + 1);
            if (kg == 1) {
              dot2_range<T>(Prow + ulo, a2v, 0, vsplit - ulo, cm, cp);
            } else {
              for (int v = ulo + sub; v < vsplit; v += kg) {
                const T e = Prow[v];
                const T2 a = a2v[v - ulo];
                cm += e * a.x;
                cp += e * a.y;
              }
            }
            // column x below the diagonal: element (v, x) of row v, v in (x, uhi)
            T cm1 = 0, cp1 = 0;
            int v = max(ulo, x + 1) + sub;
            for (; v + kg < uhi; v += 2 * kg) {
              const T e0 = P[rowbase(v) + x], e1 = P[rowbase(v + kg) + x];
              const T2 a0 = a2v[v - ulo], a1 = a2v[v + kg - ulo];
              cm += e0 * a0.x; cp += e0 * a0.y;
              cm1 += e1 * a1.x; cp1 += e1 * a1.y;
            }
            if (v < uhi) {
              const T e0 = P[rowbase(v) + x];
              const T2 a0 = a2v[v - ulo];
              cm += e0 * a0.x; cp += e0 * a0.y;
            }
            cm += cm1;
            cp += cp1;
          }
          for (int o = kg >> 1; o > 0; o >>= 1) {
            cm += __shfl_xor_sync(0xffffffffu, cm, o);
            cp += __shfl_xor_sync(0xffffffffu, cp, o);
          }
          if (x < n && sub == 0) {
            if (!hm) cm = 0;
            if (!hp) cp = 0;
            L.c2[2 * x] = cm;
            L.c2[2 * x + 1] = cp;
            L.b2[2 * x] = B11 * cm + B12 * cp;
            L.b2[2 * x + 1] = B12 * cm + B22 * cp;
          }
        }
      }
      __syncthreads();

      // ========================================================= E: rank-2 update
      {
        const int hm = S.has_m, hp = S.has_p;
        // warp per row, lanes over the row's columns. Each lane keeps (c_-, c_+) of its columns
        // (lane + 32 q, one chunk of 4 q at a time) in registers; a row's loads are issued
        // before its stores.
        const T2* __restrict__ c2v = reinterpret_cast<const T2*>(L.c2);
        const T2* __restrict__ b2v = reinterpret_cast<const T2*>(L.b2);
        for (int q0 = 0; q0 * 32 < n; q0 += 4) {
          T2 cv[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int vv = lane + 32 * (q0 + q);
            cv[q] = vv < n ? c2v[vv] : T2{(T)0, (T)0};
            if (!hm) cv[q].x = (T)0;
            if (!hp) cv[q].y = (T)0;
          }
          const int xstart = 32 * q0;  // rows below hold no column of this chunk
          for (int x = xstart + warp; x < n; x += nw) {
            const T2 bx = b2v[x];
            T* Prow = P + rowbase(x);
            T pv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int vv = lane + 32 * (q0 + q);
              pv[q] = vv <= x ? Prow[vv] : (T)0;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int vv = lane + 32 * (q0 + q);
              if (vv <= x) Prow[vv] = pv[q] - (bx.x * cv[q].x + bx.y * cv[q].y);
            }
          }
        }
        // s -= c (lambda + B r); y -= a lambda; u += a_+ - a_-; partial u^T s
        const T v0 = S.v0, v1 = S.v1, mu = (T)M.mu_q;
        CSum<T> qs;
        for (int x = tid; x < n; x += blockDim.x) {
          const T cm = L.c2[2 * x], cp = L.c2[2 * x + 1];
          T sx;
          if constexpr (fp32) {
            // (s + slo) -= cm v0 + cp v1 in float-float: exact products (FMA residuals) and
            // an error-free sum; the low parts carry what FP32 rounding would lose
            const T p1 = cm * v0, e1 = fmaf(cm, v0, -p1);
            const T p2 = cp * v1, e2 = fmaf(cp, v1, -p2);
            const T ps = p1 + p2, bp = ps - p1, ep = (p1 - (ps - bp)) + (p2 - bp);
            const T lo = e1 + e2 + ep;
            const T sh = L.s[x], t = sh - ps, bt = t - sh, et = (sh - (t - bt)) + (-ps - bt);
            const T l2 = L.slo[x] - lo + et;
            sx = t + l2;
            L.slo[x] = l2 - (sx - t);
          } else {
            sx = L.s[x] - (cm * v0 + cp * v1);
          }
          L.s[x] = sx;
          T ux = L.u[x];
          const int t = x - ulo;
          if (t >= 0 && t < ulen) {
            const T2 a = a2v[t];
            ux = ux + a.y - a.x;
            L.u[x] = ux;
            if constexpr (fp32) L.y[x] = L.y[x] + mu * a.x - mu * a.y;
          }
          qs.add(ux * sx);
          if constexpr (fp32) qs.add(ux * L.slo[x]);
        }
        const T qv = warp_sum<T>(qs.value());
        if (lane == 0) L.red[warp * 8 + 5] = qv;
        if (tid == 0) {  // warp 0 lane 0 holds the step's proposal in registers
          const int jrem = jump != 0 ? L.list[kk] : 0;  // the PE a death or update removes
          if (jump == 0) { L.list[N - 1] = jp; }
          else if (jump == 1) { L.list[kk] = L.list[N]; }
          else L.list[kk] = jp;
          S.St += (jump != 1 ? abs(jp) : 0) - (jump != 0 ? abs(jrem) : 0);
          S.N = N;
          S.logdet += (double)S.dT_pending;
          S.logL += (double)S.dnu_pending;
          S.n_acc_refresh++;
          S.q_pending = 1;
          S.pending_step = step;
        }
      }
      __syncthreads();
      if constexpr (fp32) {
        if (M.refresh_every > 0 && S.n_acc_refresh >= M.refresh_every) refresh_state<T>(M, L, P, ws, n, n_alloc);
      }
    }

    // ------------------------------------------------------------- chain end
    if (warp == bk_warp) {
      if (S.q_pending) {
        T part = lane < nw ? L.red[lane * 8 + 5] : (T)0;
        part = warp_sum<T>(part);
        if (lane == 0) {
          close_charge_hold(S, S.pending_step);
          S.q_cur = S.N * M.mu_q + M.sq2 * (double)part;
          S.wt_cur = M.g * (double)S.St / (double)(S.N + 1);
          S.q_from = S.pending_step;
          S.q_pending = 0;
        }
      }
      if (lane == 0 && S.bk_pending) bookkeep(S, L.hist);
    }
    __syncthreads();
    if constexpr (fp32) {
      // the reported log-likelihood and log|Sigma| of the final state come from an FP64
      // rebuild, not from the FP32 increments accumulated since the last refresh
      if (M.refresh_every > 0 && S.n_acc_refresh > 0) refresh_state<T>(M, L, P, ws, n, n_alloc);
    }
    if (warp == 0) {  // lambda_FSMP of the chain's N samples (Eq. (reduce-mu0))
      const double lh = warp_lambda_mle(L.hist, M.n_cap, S.lambda0, lane);
      if (lane == 0) S.lambda_hat = lh;
    }
    __syncthreads();
    if (tid == 0) {
      close_charge_hold(S, n_steps);
      fsmp_summary o;
      int ns = n_steps - S.burn_in;
      if (ns < 0) ns = 0;
      const double inv = ns > 0 ? 1.0 / ns : NAN;
      const double mN = (double)S.sN * inv, mK = (double)S.sK * inv;
      o.mean_N = mN; o.var_N = (double)S.sN2 * inv - mN * mN;
      o.mean_t0 = S.t_origin + M.g * mK; o.var_t0 = M.g * M.g * ((double)S.sK2 * inv - mK * mK);
      o.mean_Q = S.sQ * inv; o.var_Q = S.sQ2 * inv - o.mean_Q * o.mean_Q;
      o.mean_wt = S.sWt * inv; o.var_wt = S.sWt2 * inv - o.mean_wt * o.mean_wt;
      o.mean_we = 0.0; o.var_we = 0.0;  // one charge model: every e is 0
      o.logL = S.logL; o.logdet = S.logdet;
      o.drift_max = S.drift_max; o.alg_bytes = (double)S.alg_words * (double)sizeof(T);
      o.lambda_hat = S.lambda_hat;
      for (int k = 0; k < 3; ++k) { o.acc[k] = S.acc[k]; o.prop[k] = S.prop[k]; }
      o.acc_t0 = S.acc_t0; o.prop_t0 = S.prop_t0; o.N_final = S.N; o.k0_final = k0;
      o.status = S.status; o.n_samples = ns; o.n_refresh = S.n_refresh; o.reserved = 0;
      *S.out = o;
      note_chain_done(B, wi);
    }
    __syncthreads();
  }
}

}  // namespace

size_t chain_smem_bytes(const DevModel& M, int n_alloc, bool sigma_in_smem) {
  const int win = win_alloc(n_alloc, M.R, M.win_extra);
  return M.precision == FSMP_FP64 ? layout_bytes<double>(n_alloc, M.n_cap, M.LU, sigma_in_smem, M.Lt, win)
                                  : layout_bytes<float>(n_alloc, M.n_cap, M.LU, sigma_in_smem, M.Lt, win);
}

size_t chain_refresh_bytes(int n_cap, int n_alloc) { return refresh_ws_bytes(n_cap, n_alloc); }

int chain_kernel_occupancy(int precision, bool sigma_in_smem, int threads, size_t smem) {
  int n = 0;
  cudaError_t e;
  if (precision == FSMP_FP64)
    e = sigma_in_smem ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, chain_kernel<double, true>, threads, smem)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, chain_kernel<double, false>, threads, smem);
  else
    e = sigma_in_smem ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, chain_kernel<float, true>, threads, smem)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, chain_kernel<float, false>, threads, smem);
  return e == cudaSuccess ? n : 0;
}

cudaError_t chain_kernel_attributes(int precision, bool sigma_in_smem, int max_smem) {
  cudaError_t e;
  if (precision == FSMP_FP64) {
    e = sigma_in_smem ? cudaFuncSetAttribute(chain_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem)
                      : cudaFuncSetAttribute(chain_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  } else {
    e = sigma_in_smem ? cudaFuncSetAttribute(chain_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem)
                      : cudaFuncSetAttribute(chain_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  }
  return e;
}

cudaError_t launch_chains(const DevModel& M, const BatchView& B, int kernel_form, LaunchShape shape,
                          void* gmem_scratch, size_t gmem_scratch_bytes, void* refresh_ws,
                          size_t refresh_stride, int refresh_slots, cudaStream_t st) {
  if (B.n_waveforms <= 0) return cudaSuccess;
  const bool smemP = kernel_form != FSMP_KERNEL_GLOBAL;
  const size_t stride = rowbase(B.n_max);
  if (M.precision == FSMP_FP64) {
    if (smemP) {
      chain_kernel<double, true><<<shape.ctas, shape.threads, shape.smem, st>>>(M, B, nullptr, 0, nullptr, 0);
    } else {
      if ((size_t)shape.ctas * stride * sizeof(double) > gmem_scratch_bytes) return cudaErrorInvalidValue;
      chain_kernel<double, false><<<shape.ctas, shape.threads, shape.smem, st>>>(M, B, (double*)gmem_scratch, stride,
                                                                                  nullptr, 0);
    }
  } else {
    if (shape.ctas > refresh_slots || refresh_stride < refresh_ws_bytes(M.n_cap, B.n_max)) return cudaErrorInvalidValue;
    unsigned char* rw = (unsigned char*)refresh_ws;
    if (smemP) {
      chain_kernel<float, true><<<shape.ctas, shape.threads, shape.smem, st>>>(M, B, nullptr, 0, rw, refresh_stride);
    } else {
      if ((size_t)shape.ctas * stride * sizeof(float) > gmem_scratch_bytes) return cudaErrorInvalidValue;
      chain_kernel<float, false><<<shape.ctas, shape.threads, shape.smem, st>>>(M, B, (float*)gmem_scratch, stride, rw,
                                                                                refresh_stride);
    }
  }
  return cudaGetLastError();
}

}  // namespace fsmp
