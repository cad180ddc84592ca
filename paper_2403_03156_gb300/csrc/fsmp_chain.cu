// fsmp_chain.cu -- the FSMP chain kernel (arXiv 2403.03156, Sec. 2.4 and Appendix A.1).
//
// One CTA runs one chain at a time and loops over the chains of its launch (persistent).
// The chain state lives in shared memory: the packed lower triangle of Sigma^-1 (n(n+1)/2
// entries; or a per-CTA slice of global scratch for windows too long for shared memory),
// s = Sigma^-1 y, y = w - U(z), u = sum_k a_k, and the PE list. One step is
//   A  (warp 0)  Philox draws; MH move on t0 (log phi table lookups, warp sum);
//                jump choice and proposal (birth: warp-parallel search of the cumulative
//                phi, h(t) = phi(t - t0) / Phi_T); gather a_- and a_+ on the union U of their
//                supports (|U| <= L_V + a few samples).
//   B  (all)     M = a^T Sigma^-1 a over the lower triangle of the U x U block and g = a^T s
//                (per-thread sums, compensated in FP32, then warp shuffles).
//   C  (warp 0)  Delta nu = -1/2 (Delta T + Delta R) with Delta T = log det(I + Lambda M)
//                (Eq. (17) by Sylvester's identity) and Delta R = -2 lambda^T g + lambda^T M
//                lambda - r^T B r, r = g - M lambda, B = (I + Lambda M)^-1 Lambda (Eqs. (12),
//                (16)); log acceptance of Eqs. (birth) / (death) / (update); MH decision.
//   On accept:
//   D  (all)     c = Sigma^-1 a (thread per row), b = c B.
//   E  (all)     Sigma^-1 -= c B c^T (Eq. (12); thread per column pair, rows streamed),
//                s -= c (lambda + B r), y -= a lambda (Eq. (DeltaU)), u += a_+ - a_-,
//                log|Sigma| += Delta T; partial sums of u^T s for the charge summary.
//   R  (FP32 mode, every refresh_every accepts) FP64 rebuild of Sigma^-1, s, y, log|Sigma|.
// The arithmetic of Delta nu is Eqs. (16)-(18) rearranged so that Lambda^-1 never appears
// (equal in exact arithmetic; it avoids 1/sigma_q^2 cancellations).
#include <math.h>

#include "fsmp_internal.h"

namespace fsmp {
namespace {

__host__ __device__ __forceinline__ size_t rowbase(int x) { return (size_t)x * (size_t)(x + 1) / 2; }

__device__ __forceinline__ int floordiv(int a, int b) {
  int q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

__device__ __forceinline__ double logphi_at(const DevModel& M, int d) {
  return (d < -M.D || d > M.D) ? -INFINITY : M.logphi[d + M.D];
}
__device__ __forceinline__ double phi_at(const DevModel& M, int d) {
  return (d < -M.D || d > M.D) ? 0.0 : M.phi[d + M.D];
}
__device__ __forceinline__ double cphi_at(const DevModel& M, int d) {
  if (d < -M.D) return 0.0;
  if (d > M.D) return M.cphi[2 * M.D];
  return M.cphi[d + M.D];
}

// Per-thread sums: plain in FP64; Neumaier-compensated in FP32 with an error-free (TwoSum)
// warp reduction, so FP32 reductions carry about twice the working precision.
template <typename T> struct CSum;
template <> struct CSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
  __device__ __forceinline__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
};
template <> struct CSum<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
  __device__ __forceinline__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
      float t = s + s2, bp = t - s;
      float err = (s - (t - bp)) + (s2 - bp);
      s = t;
      c = c + c2 + err;
    }
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T> __device__ __forceinline__ const T* ser_table(const DevModel& M);
template <> __device__ __forceinline__ const double* ser_table<double>(const DevModel& M) { return M.V64; }
template <> __device__ __forceinline__ const float* ser_table<float>(const DevModel& M) { return M.V32; }

// Scalars of the chain in flight (shared memory).
struct ChainScalars {
  const float* w;
  fsmp_summary* out;
  fsmp_trace* trace;
  double lambda0, log_lambda0, t_origin;
  uint64_t seed, wf_id;
  int n, T_lo, T_hi, k0_lo, k0_hi, n_steps, burn_in, invalid;
  // state
  int N, k0, status, n_acc_refresh;
  double logdet, logL, q_cur;
  // proposal of the current step
  int jump, valid, noop, kk, jp, jm, u_lo, u_len, has_m, has_p, apply, accepted, t0_flags;
  int q_pending, pending_step;
  double la_prior, la_fixed, lu, la0, lu0;
  // decision
  double B11, B12, B22, v0, v1, dT, dnu, la;
  // summary sums
  double sN, sN2, st0, st02, sQ, sQ2;
  int acc[3], prop[3], acc_t0, prop_t0;
};

template <typename T> struct Layout {
  ChainScalars* S;
  double* red;      // [kMaxWarps][8]
  int* list;        // [n_cap]
  T* a2;            // [LU][2]: (a_-, a_+) interleaved
  T* s;             // [n]
  T* y;             // [n] (FP32 mode only: the FP64 refresh rebuilds from it)
  T* u;             // [n]
  T* c2;            // [n][2]: (c_-, c_+)
  T* b2;            // [n][2]: (c B)_-, (c B)_+
  T* P;             // packed Sigma^-1, when held in shared memory
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename T>
__host__ __device__ inline size_t layout_bytes(int n_alloc, int n_cap, int LU, bool with_P) {
  size_t b = align16(sizeof(ChainScalars));
  b += align16(sizeof(double) * kMaxWarps * 8);
  b += align16(sizeof(int) * n_cap);
  b += align16(sizeof(T) * 2 * LU);
  b += (sizeof(T) == 4 ? 3 : 2) * align16(sizeof(T) * n_alloc);
  b += 2 * align16(sizeof(T) * 2 * n_alloc);
  if (with_P) b += align16(sizeof(T) * rowbase(n_alloc));
  return b;
}

template <typename T>
__device__ inline Layout<T> carve(unsigned char* base, int n_alloc, int n_cap, int LU) {
  Layout<T> L;
  size_t o = 0;
  L.S = reinterpret_cast<ChainScalars*>(base + o); o += align16(sizeof(ChainScalars));
  L.red = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * kMaxWarps * 8);
  L.list = reinterpret_cast<int*>(base + o); o += align16(sizeof(int) * n_cap);
  L.a2 = reinterpret_cast<T*>(base + o); o += align16(sizeof(T) * 2 * LU);
  L.s = reinterpret_cast<T*>(base + o); o += align16(sizeof(T) * n_alloc);
  if (sizeof(T) == 4) { L.y = reinterpret_cast<T*>(base + o); o += align16(sizeof(T) * n_alloc); }
  else L.y = nullptr;
  L.u = reinterpret_cast<T*>(base + o); o += align16(sizeof(T) * n_alloc);
  L.c2 = reinterpret_cast<T*>(base + o); o += align16(sizeof(T) * 2 * n_alloc);
  L.b2 = reinterpret_cast<T*>(base + o); o += align16(sizeof(T) * 2 * n_alloc);
  L.P = reinterpret_cast<T*>(base + o);
  return L;
}

// Support of a PE at grid index j inside a window of n samples: samples s with
// 0 <= s R - j < Lt, i.e. [ceil(j / R), floor((j + Lt - 1) / R)] clipped to [0, n).
__device__ __forceinline__ void pe_support(const DevModel& M, int n, int j, int& lo, int& hi) {
  lo = max(0, floordiv(j + M.R - 1, M.R));
  hi = min(n, floordiv(j + M.Lt - 1, M.R) + 1);
  if (hi < lo) hi = lo;
}

// Smallest j in [T_lo, T_hi) with cphi(j - k0) - base > target (warp-cooperative 32-ary
// search); if rounding leaves none, the last j of T with phi > 0 (the oracle's rule).
__device__ int birth_search(const DevModel& M, int T_lo, int T_hi, int k0, double base, double target,
                            int lane) {
  int lo = T_lo, hi = T_hi - 1;
  bool any = (cphi_at(M, hi - k0) - base) > target;
  if (any) {
    while (lo < hi) {
      int len = hi - lo + 1;
      int step = (len + 31) / 32;
      int p = min(hi, lo + (lane + 1) * step - 1);
      bool pred = (cphi_at(M, p - k0) - base) > target;
      unsigned b = __ballot_sync(0xffffffffu, pred);
      int f = __ffs(b) - 1;  // b != 0: the top probe (hi) is true
      int new_lo = lo + f * step;
      int new_hi = min(hi, lo + (f + 1) * step - 1);
      lo = new_lo;
      hi = new_hi;
    }
    return lo;
  }
  int last = -1;
  for (int top = T_hi - 1; top >= T_lo; top -= 32) {
    const int j = top - lane;
    const bool ok = j >= T_lo && phi_at(M, j - k0) > 0.0;
    const unsigned b = __ballot_sync(0xffffffffu, ok);
    if (b) { last = top - (__ffs(b) - 1); break; }
  }
  return last;
}

template <typename T, bool SMEM_P>
__global__ void __launch_bounds__(512) chain_kernel(DevModel M, BatchView B, T* gP, size_t gP_stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n_alloc = B.n_max;
  Layout<T> L = carve<T>(smem_raw, n_alloc, M.n_cap, M.LU);
  ChainScalars& S = *L.S;
  T* __restrict__ P = SMEM_P ? L.P : gP + (size_t)blockIdx.x * gP_stride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const T* __restrict__ V = ser_table<T>(M);

  for (int ci = blockIdx.x; ci < B.n_waveforms; ci += gridDim.x) {
    const int wi = B.order ? B.order[ci] : ci;
    // ------------------------------------------------------------- chain set-up
    if (tid == 0) {
      int o0 = B.offsets[wi], o1 = B.offsets[wi + 1];
      S.n = o1 - o0;
      S.w = B.samples + o0;
      S.lambda0 = B.lambda0[wi];
      S.log_lambda0 = log(S.lambda0);
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
                   !(S.lambda0 > 0.0) || S.n_steps < 0 || S.burn_in < 0);
      S.N = 0; S.status = 0; S.n_acc_refresh = 0; S.q_cur = 0.0; S.q_pending = 0;
      S.sN = S.sN2 = S.st0 = S.st02 = S.sQ = S.sQ2 = 0.0;
      for (int k = 0; k < 3; ++k) { S.acc[k] = 0; S.prop[k] = 0; }
      S.acc_t0 = 0; S.prop_t0 = 0;
    }
    __syncthreads();
    if (S.invalid) {
      if (tid == 0) {
        fsmp_summary o;
        o.mean_N = o.var_N = o.mean_t0 = o.var_t0 = o.mean_Q = o.var_Q = o.logL = o.logdet = NAN;
        for (int k = 0; k < 3; ++k) { o.acc[k] = 0; o.prop[k] = 0; }
        o.acc_t0 = o.prop_t0 = o.N_final = o.k0_final = o.n_samples = 0;
        o.status = FSMP_ST_INVALID;
        *S.out = o;
      }
      __syncthreads();
      continue;
    }
    const int n = S.n;
    const float* __restrict__ w = S.w;
    // Sigma^-1 = I / sigma_eps^2, s = w / sigma_eps^2, y = w, u = 0 (empty z)
    {
      const size_t np = rowbase(n);
      for (size_t e = tid; e < np; e += blockDim.x) P[e] = (T)0;
      __syncthreads();
      double wsq = 0.0;
      for (int x = tid; x < n; x += blockDim.x) {
        P[rowbase(x) + x] = (T)M.inv_se2;
        double wx = (double)w[x];
        L.s[x] = (T)(wx * M.inv_se2);
        if (L.y) L.y[x] = (T)wx;
        L.u[x] = (T)0;
        wsq += wx * wx;
      }
      wsq = warp_sum(wsq);
      if (lane == 0) L.red[warp * 8] = wsq;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int i = 0; i < nw; ++i) t += L.red[i * 8];
        S.logdet = n * log(M.se2);
        S.logL = -0.5 * (n * kLog2Pi + S.logdet + t * M.inv_se2);
      }
      __syncthreads();
    }

    for (int step = 0; step < S.n_steps; ++step) {
      // ========================================================= A: warp 0
      if (warp == 0) {
        if (S.q_pending) {  // charge summary of the previous (accepted) step
          double part = lane < nw ? L.red[lane * 8 + 5] : 0.0;
          part = warp_sum(part);
          if (lane == 0) {
            S.q_cur = S.N * M.mu_q + M.sq2 * part;
            if (S.pending_step >= S.burn_in) {
              double t0ns = S.t_origin + S.k0 * M.g;
              S.sN += S.N; S.sN2 += (double)S.N * S.N; S.st0 += t0ns; S.st02 += t0ns * t0ns;
              S.sQ += S.q_cur; S.sQ2 += S.q_cur * S.q_cur;
            }
            S.q_pending = 0;
          }
          __syncwarp();
        }
        // Philox: lane 0 block (step, 0, 0, 0), lane 1 block (step, 1, 0, 0)
        uint64_t c[4] = {(uint64_t)step, (uint64_t)(lane & 1), 0, 0};
        philox4x64_10(c, S.seed, S.wf_id);
        double u[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          u[i] = u01_from_bits(__shfl_sync(0xffffffffu, c[i], 0));
          u[4 + i] = u01_from_bits(__shfl_sync(0xffffffffu, c[i], 1));
        }
        const int N = S.N;
        int k0 = S.k0;
        // ---- Gibbs part 1: MH on t0 (Sec. 2.4), uniform prior on its grid range
        double la0 = NAN, lu0 = NAN;
        int t0f = 0;
        if (M.sample_t0) {
          t0f = 1;
          double z1 = sqrt(-2.0 * log(u[0])) * cos(kTwoPi * u[1]);
          long long Dm = llrint(z1 * M.inv_g);
          long long k0p = (long long)k0 + Dm;
          if (Dm == 0) {
            la0 = 0.0;
          } else if (k0p < S.k0_lo || k0p > S.k0_hi) {
            la0 = -INFINITY;
          } else {
            double part = 0.0;
            for (int k = lane; k < N; k += 32) {
              int j = L.list[k];
              part += logphi_at(M, j - (int)k0p) - logphi_at(M, j - k0);
            }
            la0 = warp_sum(part);
          }
          lu0 = log(u[2]);
          if (lu0 < la0) { k0 = (int)k0p; t0f |= 2; }
        }
        // ---- Gibbs part 2: one RJMCMC jump (Sec. 2.4)
        const int jump = (N == 0) ? 0 : (u[3] < M.J ? 0 : (u[3] < 2.0 * M.J ? 1 : 2));
        int valid = 0, noop = 0, kk = -1, jp = -1, jm = -1, st_add = 0;
        double la_prior = 0.0, la_fixed = -INFINITY;
        const int T_lo = S.T_lo, T_hi = S.T_hi;
        if (jump == 0) {
          if (N >= M.n_cap) {
            st_add |= FSMP_ST_CAPACITY;
          } else {
            double base = cphi_at(M, T_lo - 1 - k0), tot = cphi_at(M, T_hi - 1 - k0) - base;
            if (tot > 0.0) {
              jp = birth_search(M, T_lo, T_hi, k0, base, u[4] * tot, lane);
              valid = jp >= T_lo;
              la_prior = S.log_lambda0 + log(tot * M.g) - log((double)(N + 1)) + (N == 0 ? M.log_J : 0.0);
            }
          }
        } else {
          kk = (int)floor(u[4] * N);
          if (kk >= N) kk = N - 1;
          jm = L.list[kk];
          if (jump == 1) {
            double tot = cphi_at(M, T_hi - 1 - k0) - cphi_at(M, T_lo - 1 - k0);
            valid = 1;
            la_prior = -S.log_lambda0 - log(tot * M.g) + log((double)N) - (N == 1 ? M.log_J : 0.0);
          } else {
            double z2 = sqrt(-2.0 * log(u[5])) * cos(kTwoPi * u[6]);
            long long Dm = llrint(z2 * M.inv_g);
            long long jpl = (long long)jm + Dm;
            if (Dm == 0) {
              noop = 1;
              la_fixed = 0.0;
            } else if (jpl < T_lo || jpl >= T_hi || logphi_at(M, (int)jpl - k0) == -INFINITY) {
              la_fixed = -INFINITY;
            } else {
              jp = (int)jpl;
              valid = 1;
              la_prior = logphi_at(M, jp - k0) - logphi_at(M, jm - k0);
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
          if (ulen > M.LU) { valid = 0; la_fixed = -INFINITY; st_add |= FSMP_ST_NONFINITE; ulen = 0; }
        }
        for (int t = lane; t < ulen; t += 32) {
          int sidx = ulo + t;
          T am = (hm && sidx >= mlo && sidx < mhi) ? V[sidx * M.R - jm] : (T)0;
          T ap = (hp && sidx >= plo && sidx < phi_) ? V[sidx * M.R - jp] : (T)0;
          L.a2[2 * t] = am;
          L.a2[2 * t + 1] = ap;
        }
        __syncwarp();
        if (lane == 0) {
          S.k0 = k0;
          if (t0f & 1) { S.prop_t0++; if (t0f & 2) S.acc_t0++; }
          S.t0_flags = t0f; S.la0 = la0; S.lu0 = lu0;
          S.jump = jump; S.valid = valid; S.noop = noop; S.kk = kk; S.jp = jp; S.jm = jm;
          S.u_lo = ulo; S.u_len = ulen; S.has_m = hm; S.has_p = hp;
          S.la_prior = la_prior; S.la_fixed = la_fixed; S.lu = log(u[7]);
          S.status |= st_add;
          S.prop[jump]++;
        }
      }
      __syncthreads();

      // ========================================================= B: all threads
      const int ulo = S.u_lo, ulen = S.u_len;
      const bool scored = S.valid && ulen > 0;
      if (scored) {
        const int hm = S.has_m, hp = S.has_p;
        CSum<T> Smm, Smp, Spp, Gm, Gp;
        T amr[4], apr[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int cidx = lane + 32 * q;
          amr[q] = cidx < ulen ? L.a2[2 * cidx] : (T)0;
          apr[q] = cidx < ulen ? L.a2[2 * cidx + 1] : (T)0;
        }
        for (int r = warp; r < ulen; r += nw) {
          const T* __restrict__ Prow = P + rowbase(ulo + r) + ulo;
          T rm = 0, rp = 0, ed = 0;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            int cidx = lane + 32 * q;
            if (cidx < r) {
              T e = Prow[cidx];
              rm += e * amr[q];
              rp += e * apr[q];
            } else if (cidx == r) {
              ed = Prow[cidx];
            }
          }
          T amw = L.a2[2 * r], apw = L.a2[2 * r + 1];
          if (hm) Smm.add(amw * ((T)2 * rm + ed * amw));
          if (hp) Spp.add(apw * ((T)2 * rp + ed * apw));
          if (hm && hp) Smp.add(amw * rp + apw * rm + ed * amw * apw);
        }
        for (int t = tid; t < ulen; t += blockDim.x) {
          T sv = L.s[ulo + t];
          Gm.add(L.a2[2 * t] * sv);
          Gp.add(L.a2[2 * t + 1] * sv);
        }
        Smm.warp_reduce(); Smp.warp_reduce(); Spp.warp_reduce(); Gm.warp_reduce(); Gp.warp_reduce();
        if (lane == 0) {
          double* r = L.red + warp * 8;
          r[0] = Smm.value(); r[1] = Smp.value(); r[2] = Spp.value(); r[3] = Gm.value(); r[4] = Gp.value();
        }
      }
      __syncthreads();

      // ========================================================= C: warp 0
      if (warp == 0) {
        double v = 0.0;
        if (scored && lane < 5)
          for (int i = 0; i < nw; ++i) v += L.red[i * 8 + lane];
        const double mmm = __shfl_sync(0xffffffffu, v, 0), mmp = __shfl_sync(0xffffffffu, v, 1);
        const double mpp = __shfl_sync(0xffffffffu, v, 2), gm = __shfl_sync(0xffffffffu, v, 3);
        const double gp = __shfl_sync(0xffffffffu, v, 4);
        if (lane == 0) {
          double la = S.la_fixed, dnu = NAN;
          int apply = 0, st_add = 0;
          if (S.valid) {
            const double q = M.sq2, mu = M.mu_q;
            // det(I + Lambda M), Lambda = sigma_q^2 diag(-1, 1)
            double Dd = (1.0 - q * mmm) * (1.0 + q * mpp) + q * q * mmp * mmp;
            if (!(Dd > 0.0)) {
              la = -INFINITY;
              st_add |= FSMP_ST_BADDET;
            } else {
              double B11 = -q * (1.0 + q * mpp) / Dd, B12 = q * q * mmp / Dd, B22 = q * (1.0 - q * mmm) / Dd;
              double rm = gm - mu * (mmp - mmm), rp = gp - mu * (mpp - mmp);
              double dR = -2.0 * mu * (gp - gm) + mu * mu * (mmm - 2.0 * mmp + mpp) -
                          (B11 * rm * rm + 2.0 * B12 * rm * rp + B22 * rp * rp);
              double dT = log(Dd);
              dnu = -0.5 * (dT + dR);
              if (!isfinite(dnu)) {
                la = -INFINITY;
                st_add |= FSMP_ST_NONFINITE;
              } else {
                la = dnu + S.la_prior;
                S.B11 = B11; S.B12 = B12; S.B22 = B22; S.dT = dT; S.dnu = dnu;
                S.v0 = -mu + B11 * rm + B12 * rp;
                S.v1 = mu + B12 * rm + B22 * rp;
              }
            }
          }
          const int acc = S.lu < la;
          if (acc && S.valid && isfinite(la)) apply = 1;
          if (acc && !S.noop) S.acc[S.jump]++;
          S.status |= st_add;
          S.apply = apply;
          S.accepted = acc;
          if (S.trace) {
            fsmp_trace tr;
            tr.la0 = S.la0; tr.lu0 = S.lu0; tr.la = la; tr.lu = S.lu; tr.dnu = dnu;
            tr.N = S.N + (apply ? (S.jump == 0 ? 1 : (S.jump == 1 ? -1 : 0)) : 0);
            tr.k0 = S.k0; tr.jump = S.jump;
            tr.flags = S.t0_flags | (acc ? 4 : 0) | ((acc && S.noop) ? 8 : 0);
            S.trace[step] = tr;
          }
          if (!apply) {
            if (step >= S.burn_in) {
              double t0ns = S.t_origin + S.k0 * M.g;
              S.sN += S.N; S.sN2 += (double)S.N * S.N; S.st0 += t0ns; S.st02 += t0ns * t0ns;
              S.sQ += S.q_cur; S.sQ2 += S.q_cur * S.q_cur;
            }
          } else {
            S.q_pending = 1;
            S.pending_step = step;
          }
        }
      }
      __syncthreads();
      if (!S.apply) continue;

      // ========================================================= D: c = Sigma^-1 a, b = c B
      {
        const int hm = S.has_m, hp = S.has_p;
        const T B11 = (T)S.B11, B12 = (T)S.B12, B22 = (T)S.B22;
        for (int x = tid; x < n; x += blockDim.x) {
          T cm = 0, cp = 0;
          const size_t rbx = rowbase(x);
          for (int t = 0; t < ulen; ++t) {
            const int vv = ulo + t;
            const T e = vv <= x ? P[rbx + vv] : P[rowbase(vv) + x];
            if (hm) cm += e * L.a2[2 * t];
            if (hp) cp += e * L.a2[2 * t + 1];
          }
          L.c2[2 * x] = cm;
          L.c2[2 * x + 1] = cp;
          L.b2[2 * x] = B11 * cm + B12 * cp;
          L.b2[2 * x + 1] = B12 * cm + B22 * cp;
        }
      }
      __syncthreads();

      // ========================================================= E: rank-2 update
      {
        const int hm = S.has_m, hp = S.has_p;
        const int npairs = (n + 1) / 2;
        for (int pidx = tid; pidx < npairs; pidx += blockDim.x) {
#pragma unroll 1
          for (int h = 0; h < 2; ++h) {
            const int v = h == 0 ? pidx : n - 1 - pidx;
            if (h == 1 && v == pidx) break;
            const T cmv = L.c2[2 * v], cpv = L.c2[2 * v + 1];
            size_t rb = rowbase(n - 1);
            for (int x = n - 1; x >= v; --x) {
              T d;
              if (hm && hp) d = L.b2[2 * x] * cmv + L.b2[2 * x + 1] * cpv;
              else if (hm) d = L.b2[2 * x] * cmv;
              else d = L.b2[2 * x + 1] * cpv;
              P[rb + v] -= d;
              rb -= x;
            }
          }
        }
        // s -= c (lambda + B r); y -= a lambda; u += a_+ - a_-; partial u^T s
        const T v0 = (T)S.v0, v1 = (T)S.v1, mu = (T)M.mu_q;
        CSum<T> qs;
        for (int x = tid; x < n; x += blockDim.x) {
          T sx = L.s[x] - (L.c2[2 * x] * v0 + L.c2[2 * x + 1] * v1);
          L.s[x] = sx;
          T ux = L.u[x];
          int t = x - ulo;
          if (t >= 0 && t < ulen) {
            T am = L.a2[2 * t], ap = L.a2[2 * t + 1];
            ux = ux + ap - am;
            L.u[x] = ux;
            if (L.y) L.y[x] = L.y[x] + mu * am - mu * ap;
          }
          qs.add(ux * sx);
        }
        qs.warp_reduce();
        if (lane == 0) L.red[warp * 8 + 5] = qs.value();
        if (tid == 0) {
          if (S.jump == 0) { L.list[S.N] = S.jp; S.N++; }
          else if (S.jump == 1) { L.list[S.kk] = L.list[S.N - 1]; S.N--; }
          else L.list[S.kk] = S.jp;
          S.logdet += S.dT;
          S.logL += S.dnu;
          S.n_acc_refresh++;
        }
      }
      __syncthreads();
    }

    // ------------------------------------------------------------- chain end
    if (warp == 0) {
      if (S.q_pending) {
        double part = lane < nw ? L.red[lane * 8 + 5] : 0.0;
        part = warp_sum(part);
        if (lane == 0) {
          S.q_cur = S.N * M.mu_q + M.sq2 * part;
          if (S.pending_step >= S.burn_in) {
            double t0ns = S.t_origin + S.k0 * M.g;
            S.sN += S.N; S.sN2 += (double)S.N * S.N; S.st0 += t0ns; S.st02 += t0ns * t0ns;
            S.sQ += S.q_cur; S.sQ2 += S.q_cur * S.q_cur;
          }
          S.q_pending = 0;
        }
      }
      if (lane == 0) {
        fsmp_summary o;
        int ns = S.n_steps - S.burn_in;
        if (ns < 0) ns = 0;
        double inv = ns > 0 ? 1.0 / ns : NAN;
        o.mean_N = S.sN * inv; o.var_N = S.sN2 * inv - o.mean_N * o.mean_N;
        o.mean_t0 = S.st0 * inv; o.var_t0 = S.st02 * inv - o.mean_t0 * o.mean_t0;
        o.mean_Q = S.sQ * inv; o.var_Q = S.sQ2 * inv - o.mean_Q * o.mean_Q;
        o.logL = S.logL; o.logdet = S.logdet;
        for (int k = 0; k < 3; ++k) { o.acc[k] = S.acc[k]; o.prop[k] = S.prop[k]; }
        o.acc_t0 = S.acc_t0; o.prop_t0 = S.prop_t0; o.N_final = S.N; o.k0_final = S.k0;
        o.status = S.status; o.n_samples = ns;
        *S.out = o;
      }
    }
    __syncthreads();
  }
}

}  // namespace

size_t chain_smem_bytes(int precision, int n_alloc, int n_cap, int LU, int threads, bool sigma_in_smem) {
  (void)threads;
  return precision == FSMP_FP64 ? layout_bytes<double>(n_alloc, n_cap, LU, sigma_in_smem)
                                : layout_bytes<float>(n_alloc, n_cap, LU, sigma_in_smem);
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
                          void* gmem_scratch, size_t gmem_scratch_bytes, cudaStream_t st) {
  if (B.n_waveforms <= 0) return cudaSuccess;
  const bool smemP = kernel_form != FSMP_KERNEL_GLOBAL;
  size_t stride = rowbase(B.n_max);
  if (M.precision == FSMP_FP64) {
    if (smemP) {
      chain_kernel<double, true><<<shape.ctas, shape.threads, shape.smem, st>>>(M, B, nullptr, 0);
    } else {
      if ((size_t)shape.ctas * stride * sizeof(double) > gmem_scratch_bytes) return cudaErrorInvalidValue;
      chain_kernel<double, false><<<shape.ctas, shape.threads, shape.smem, st>>>(M, B, (double*)gmem_scratch, stride);
    }
  } else {
    if (smemP) {
      chain_kernel<float, true><<<shape.ctas, shape.threads, shape.smem, st>>>(M, B, nullptr, 0);
    } else {
      if ((size_t)shape.ctas * stride * sizeof(float) > gmem_scratch_bytes) return cudaErrorInvalidValue;
      chain_kernel<float, false><<<shape.ctas, shape.threads, shape.smem, st>>>(M, B, (float*)gmem_scratch, stride);
    }
  }
  return cudaGetLastError();
}

}  // namespace fsmp
