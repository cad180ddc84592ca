// fsmp_pe.cu -- the FSMP chain in PE space, one warp per chain (arXiv 2403.03156, Sec. 2.4 and
// Appendix A.1, with the Woodbury identity applied to the whole of A).
//
// Sigma(z) = sigma_eps^2 I + sigma_q^2 A A^T with A = [a_1 .. a_N] (n x N). With
// r = sigma_eps^2 / sigma_q^2 and the N x N capacitance matrix C = r I + A^T A,
//   Sigma^-1 = (I - A C^-1 A^T) / sigma_eps^2,   log|Sigma| = n log sigma_eps^2 + log|C| - N log r.
// A chain keeps C^-1, v = C^-1 A^T y and the residual y = w - mu_q sum_k a_k. For a move with the
// columns a_- = a_k (a PE of z) and a_+ (a new position), and b = A^T a_+,
//   a_+^T Sigma^-1 a_+ = (|a_+|^2 - b^T C^-1 b) / sigma_eps^2,   a_+^T Sigma^-1 y = (a_+^T y - b^T v) / sigma_eps^2,
//   1 - sigma_q^2 a_k^T Sigma^-1 a_k = r C^-1_kk,                a_k^T Sigma^-1 y = v_k / sigma_q^2,
//   a_k^T Sigma^-1 a_+ = (C^-1 b)_k / sigma_q^2,
// the 2x2 quantities of Eqs. (16)-(18). Only the p PEs whose support overlaps a_+ have b != 0, so a
// proposal reads p^2 + O(p) entries of C^-1 and no n-vector beyond a_+'s support. An accepted move
// updates C^-1 by bordering (birth), a Schur-complement downdate (death) or both in one pass
// (update): O(N^2) instead of the O(n^2) of Sigma^-1. The charge summary is
// E[Q | z, w] = N mu_q + sum_k v_k. Inner products a_i^T a_j over the window come from the SER
// cross-correlation prefix table.
//
// Layout: a CTA holds several independent chains, one per warp; a warp takes chains from a
// launch-wide counter. C^-1 sits in a per-warp shared-memory tile of Ns x Ns while N <= Ns and
// moves to the warp's global slot (n_cap x ldc) when a birth would exceed the tile.
//
// Precision: C^-1, v and b are FP64 in both modes. For PEs close in time C is nearly singular
// (eigenvalues down to r) and C^-1 holds entries near 1/r that cancel in b^T C^-1 b; stored in
// FP32 they cost about 1e-2 in log alpha per step. In FP32 mode the residual y, the SER and phi
// tables, the random draws and the 2x2 algebra are FP32, and C^-1, v, y, log|Sigma| and the
// log-likelihood are rebuilt from z in FP64 (Gauss-Jordan inversion of C, which is symmetric
// positive definite) every refresh_every accepted moves and at the end. Per step the random
// draws, proposal rules and acceptance tests are those of the Sigma^-1 kernel.
#include <math.h>

#include "fsmp_internal.h"

namespace fsmp {
namespace {

constexpr int kPeRB = 32;  // steps per batch of random draws
constexpr unsigned kFull = 0xffffffffu;

template <typename T> struct PeTab;
template <> struct PeTab<double> {
  __device__ static const double* V(const DevModel& M) { return M.V64; }
  __device__ static const double* logphi(const DevModel& M) { return M.logphi; }
  __device__ static const double* cphi(const DevModel& M) { return M.cphi; }
  __device__ static const double* tc(const DevModel& M) { return M.tc64; }
};
template <> struct PeTab<float> {
  __device__ static const float* V(const DevModel& M) { return M.V32; }
  __device__ static const float* logphi(const DevModel& M) { return M.logphi32; }
  __device__ static const float* cphi(const DevModel& M) { return M.cphi32; }
  __device__ static const float* tc(const DevModel& M) { return M.tc32; }
};

template <typename T> __device__ __forceinline__ T pe_logphi(const DevModel& M, int d) {
  return (d < -M.D || d > M.D) ? (T)-INFINITY : __ldg(PeTab<T>::logphi(M) + (d + M.D));
}
template <typename T> __device__ __forceinline__ T pe_cphi(const DevModel& M, int d) {
  if (d < -M.D) return (T)0;
  if (d > M.D) return __ldg(PeTab<T>::cphi(M) + 2 * M.D);
  return __ldg(PeTab<T>::cphi(M) + (d + M.D));
}

template <typename T> __device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
// Sum over lanes [0, m) of values that are zero on lanes >= m (1 <= m <= 32); every lane of
// [0, next power of two >= m) gets the sum.
__device__ __forceinline__ double wsum_first(double v, int m) {
  for (int o = 16; o > 0; o >>= 1)
    if (o < m) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
template <typename T> __device__ __forceinline__ T wmax(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// Support of the PE at grid index j in a window of n samples: its first sample w0 = ceil(j / R),
// the phase ph = w0 R - j of that sample, and the range [ilo, ihi) of its support samples
// (sample w0 + i, SER index ph + i R) that lie in the window.
struct Sup {
  int w0, ph, ilo, ihi;
};
__device__ __forceinline__ Sup pe_sup(const DevModel& M, int n, int j) {
  Sup s;
  s.w0 = (int)floorf((float)(j + M.R - 1) / (float)M.R);  // exact for |j| < 2^22
  s.ph = s.w0 * M.R - j;
  const int mph = (M.Lt - s.ph + M.R - 1) / M.R;
  s.ilo = max(0, -s.w0);
  s.ihi = min(mph, n - s.w0);
  if (s.ihi <= s.ilo) s.ilo = s.ihi = 0;  // no sample of the window: an all-zero column
  return s;
}

// a_x^T a_q over the window, for x with support s and q = x - o (|o| < Lt), from the prefix table.
template <typename T> __device__ __forceinline__ T xcorr(const DevModel& M, const T* __restrict__ tc, const Sup& s, int o) {
  const int O = 2 * M.Lt - 1;
  const T* base = tc + (size_t)s.ph * M.tcM * O + (o + M.Lt - 1);
  T v = __ldg(base + (size_t)s.ihi * O);
  if (s.ilo > 0) v -= __ldg(base + (size_t)s.ilo * O);
  return v;
}

// Smallest j in [T_lo, T_hi) with cphi(j - k0) - base > target (32-ary warp search); if rounding
// leaves none, the last j of T with phi > 0.
template <typename T>
__device__ int pe_birth_search(const DevModel& M, int T_lo, int T_hi, int k0, T base, T target, int lane) {
  int lo = T_lo, hi = T_hi - 1;
  if ((pe_cphi<T>(M, hi - k0) - base) > target) {
    while (lo < hi) {
      const int len = hi - lo + 1;
      const int step = (len + 31) / 32;
      const int p = min(hi, lo + (lane + 1) * step - 1);
      const bool pred = (pe_cphi<T>(M, p - k0) - base) > target;
      const unsigned b = __ballot_sync(kFull, pred);
      const int f = __ffs(b) - 1;
      const int new_lo = lo + f * step;
      hi = min(hi, lo + (f + 1) * step - 1);
      lo = new_lo;
    }
    return lo;
  }
  int last = -1;
  for (int top = T_hi - 1; top >= T_lo; top -= 32) {
    const int j = top - lane;
    const bool ok = j >= T_lo && pe_logphi<T>(M, j - k0) > (T)-INFINITY;
    const unsigned b = __ballot_sync(kFull, ok);
    if (b) { last = top - (__ffs(b) - 1); break; }
  }
  return last;
}

template <typename T> struct PeRand {
  T z1, lu0, u3, u4, z2, lu;  // t0 shift normal, log u2, jump type, PE choice, shift normal, log u7
};

// Per-chain statistics (shared memory, written by lane 0).
struct PeStats {
  long long sN, sN2, sK, sK2;
  double sQ, sQ2, q_cur, logdet, logL, drift_max;
  unsigned long long alg_words;
  int acc[3], prop[3], acc_t0, prop_t0, n_refresh, status, q_from, n_acc_refresh, refresh_fail, pad;
};

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

// Per-warp shared memory.
template <typename T> struct PeWarp {
  PeStats* st;
  PeRand<T>* rnd;
  int* list;   // PE grid indices [n_cap]
  int* ovi;    // PEs overlapping the proposed one [n_cap]
  double* ovb; // their inner products with it [n_cap]
  double* v;   // C^-1 A^T y [n_cap]
  T* vT;       // v at the scoring precision [n_cap]
  double* cv;  // row k of C^-1 / C^-1 b [n_cap]
  double* uv;  // second work vector [n_cap]
  T* y;        // residual [n_alloc]
  T* lPhi;     // log(Phi_T(t0) g) on the chain's t0 grid [win_extra]
  double* Cs;  // C^-1 tile [Ns * Ns]
};
template <typename T> __host__ __device__ inline size_t pe_warp_bytes(int n_cap, int n_alloc, int win_extra, int Ns) {
  return a16(sizeof(PeStats)) + a16(sizeof(PeRand<T>) * kPeRB) + 2 * a16(sizeof(int) * n_cap) +
         4 * a16(sizeof(double) * n_cap) + a16(sizeof(T) * n_cap) + a16(sizeof(T) * n_alloc) +
         a16(sizeof(T) * win_extra) +
         a16(sizeof(double) * (size_t)Ns * Ns);
}
template <typename T> __host__ __device__ inline size_t pe_block_bytes(int Lt, int n_cap) {
  return a16(sizeof(T) * Lt) + a16(sizeof(T) * (n_cap + 2));
}
template <typename T> __device__ PeWarp<T> pe_carve(unsigned char* p, int n_cap, int n_alloc, int win_extra, int Ns) {
  PeWarp<T> W;
  size_t o = 0;
  W.st = reinterpret_cast<PeStats*>(p + o); o += a16(sizeof(PeStats));
  W.rnd = reinterpret_cast<PeRand<T>*>(p + o); o += a16(sizeof(PeRand<T>) * kPeRB);
  W.list = reinterpret_cast<int*>(p + o); o += a16(sizeof(int) * n_cap);
  W.ovi = reinterpret_cast<int*>(p + o); o += a16(sizeof(int) * n_cap);
  W.ovb = reinterpret_cast<double*>(p + o); o += a16(sizeof(double) * n_cap);
  W.v = reinterpret_cast<double*>(p + o); o += a16(sizeof(double) * n_cap);
  W.vT = reinterpret_cast<T*>(p + o); o += a16(sizeof(T) * n_cap);
  W.cv = reinterpret_cast<double*>(p + o); o += a16(sizeof(double) * n_cap);
  W.uv = reinterpret_cast<double*>(p + o); o += a16(sizeof(double) * n_cap);
  W.y = reinterpret_cast<T*>(p + o); o += a16(sizeof(T) * n_alloc);
  W.lPhi = reinterpret_cast<T*>(p + o); o += a16(sizeof(T) * win_extra);
  W.Cs = reinterpret_cast<double*>(p + o);
  return W;
}

// Global per-warp slots.
struct PeSlots {
  double* C;           // C^-1 slots: n_cap rows of ldc entries each
  size_t c_stride;     // elements per slot
  int ldc;
  double* ws;          // FP64 refresh workspace slots (FP32 mode)
  size_t ws_stride;    // doubles per slot
  int* counter;        // next chain of the launch (zeroed before the launch)
  int Ns;              // shared-memory tile of C^-1 (0: always global)
};

// FP64 refresh workspace of one warp: C (n_cap x n_cap) and four vectors of max(n_cap, n_alloc).
__host__ __device__ inline int pe_lvec(int n_cap, int n_alloc) { return n_cap > n_alloc ? n_cap : n_alloc; }
__host__ __device__ inline size_t pe_ws_doubles(int n_cap, int n_alloc) {
  return (size_t)n_cap * n_cap + 4 * (size_t)pe_lvec(n_cap, n_alloc);
}

// Charge hold: the state's charge summary q_cur holds from step q_from on; close it at step s.
__device__ __forceinline__ void close_hold(PeStats& S, int s, int burn_in) {
  const int from = max(S.q_from, burn_in);
  if (s > from) {
    const double c = (double)(s - from);
    S.sQ += S.q_cur * c;
    S.sQ2 += S.q_cur * S.q_cur * c;
  }
}

// FP64 rebuild of C^-1, v, y, log|Sigma| and the log-likelihood from the PE list (FP32 mode).
// Returns false (state untouched) if C is not numerically positive definite.
template <typename T>
__device__ __noinline__ bool pe_refresh(const DevModel& M, PeWarp<T>& W, double* Cp, int ld, double* ws, int n_cap, int lvec,
                           const float* w, int n, int N, int lane, double& logdet_out, double& logL_out,
                           double& drift_out) {
  const int ws_ld = n_cap;
  double* A = ws;                               // C, then C^-1 (row-major, stride n_cap)
  double* yres = A + (size_t)n_cap * n_cap;     // residual y (FP64)
  double* h = yres + lvec;                      // A^T y
  double* rowk = h + lvec;                      // staged pivot row
  double* colk = rowk + lvec;                   // staged pivot column
  const double* V = M.V64;
  const double mu = M.mu_q, r = M.se2 / M.sq2;
  // residual y = w - mu sum_k a_k
  for (int x = lane; x < n; x += 32) yres[x] = (double)w[x];
  __syncwarp();
  for (int k = 0; k < N; ++k) {
    const Sup s = pe_sup(M, n, W.list[k]);
    for (int i = s.ilo + lane; i < s.ihi; i += 32) yres[s.w0 + i] -= mu * V[s.ph + i * M.R];
    __syncwarp();
  }
  // C = r I + A^T A (full, row-major)
  for (int i = 0; i < N; ++i) {
    const int ji = W.list[i];
    const Sup si = pe_sup(M, n, ji);
    for (int j = lane; j < N; j += 32) {
      const int o = ji - W.list[j];
      double c = (o > -M.Lt && o < M.Lt) ? xcorr<double>(M, M.tc64, si, o) : 0.0;
      if (j == i) c += r;
      A[(size_t)i * ws_ld + j] = c;
    }
  }
  // h = A^T y
  for (int k = lane; k < N; k += 32) {
    const Sup s = pe_sup(M, n, W.list[k]);
    double a0 = 0.0, a1 = 0.0;
    int i = s.ilo;
    for (; i + 1 < s.ihi; i += 2) {
      a0 += V[s.ph + i * M.R] * yres[s.w0 + i];
      a1 += V[s.ph + (i + 1) * M.R] * yres[s.w0 + i + 1];
    }
    if (i < s.ihi) a0 += V[s.ph + i * M.R] * yres[s.w0 + i];
    h[k] = a0 + a1;
  }
  __syncwarp();
  // Gauss-Jordan inversion in place with diagonal pivots (C is SPD: the pivots are the
  // LDL^T pivots, all positive); log|C| = sum log pivot, kept as mantissa x 2^exponent
  double pm = 1.0;
  int pe = 0;
  for (int k = 0; k < N; ++k) {
    for (int j = lane; j < N; j += 32) {
      rowk[j] = A[(size_t)k * ws_ld + j];
      colk[j] = A[(size_t)j * ws_ld + k];
    }
    __syncwarp();
    const double piv = rowk[k];
    if (!(piv > 0.0) || !isfinite(piv)) return false;
    const double ip = 1.0 / piv;
    int ex;
    pm *= frexp(piv, &ex);
    pe += ex;
    pm = frexp(pm, &ex);
    pe += ex;
    for (int i = 0; i < N; ++i) {
      double* Ai = A + (size_t)i * ws_ld;
      if (i == k) {
        for (int j = lane; j < N; j += 32) Ai[j] = (j == k) ? ip : rowk[j] * ip;
      } else {
        const double f = colk[i] * ip;
        for (int j = lane; j < N; j += 32) Ai[j] = (j == k) ? -f : fma(-f, rowk[j], Ai[j]);
      }
    }
    __syncwarp();
  }
  const double logdetC = log(pm) + (double)pe * 0.6931471805599453;
  // v = C^-1 h (C^-1 symmetric: lanes over columns)
  double dmax = 0.0, amax = 0.0;
  for (int i = lane; i < N; i += 32) {
    double s = 0.0;
    for (int j = 0; j < N; ++j) s = fma(A[(size_t)j * ws_ld + i], h[j], s);
    rowk[i] = s;
  }
  __syncwarp();
  double hv = 0.0;
  for (int i = lane; i < N; i += 32) hv += h[i] * rowk[i];
  hv = wsum(hv);
  double yy = 0.0;
  for (int x = lane; x < n; x += 32) yy += yres[x] * yres[x];
  yy = wsum(yy);
  // drift of the incremental state, then the refreshed state
  for (int i = 0; i < N; ++i) {
    for (int j = lane; j < N; j += 32) {
      const double nv = A[(size_t)i * ws_ld + j];
      dmax = fmax(dmax, fabs(nv - Cp[(size_t)i * ld + j]));
      amax = fmax(amax, fabs(nv));
      Cp[(size_t)i * ld + j] = nv;
    }
  }
  double vd = 0.0, va = 0.0;
  for (int i = lane; i < N; i += 32) {
    vd = fmax(vd, fabs(rowk[i] - W.v[i]));
    va = fmax(va, fabs(rowk[i]));
    W.v[i] = rowk[i];
    W.vT[i] = (T)rowk[i];
  }
  for (int x = lane; x < n; x += 32) W.y[x] = (T)yres[x];
  dmax = wmax(dmax); amax = wmax(amax); vd = wmax(vd); va = wmax(va);
  __syncwarp();
  drift_out = fmax(amax > 0.0 ? dmax / amax : 0.0, va > 0.0 ? vd / fmax(va, 1.0) : 0.0);
  logdet_out = n * log(M.se2) + logdetC - N * log(r);
  logL_out = -0.5 * (n * kLog2Pi + logdet_out + (yy - hv) / M.se2);
  return true;
}

// Scalars of an accepted move, from the proposal and its scoring.
struct PeMove {
  int jump, kk, jp, jm, np;
  double aa, quad, bv, vk, ay;
  Sup sp;
};

// Apply an accepted move to C^-1, v, y and the PE list (out of line: it runs on a minority of
// steps and keeps the per-step code compact). Returns the new N; *Cp / *ld change when C^-1
// moves from the shared tile to the global slot.
template <typename T>
__device__ __noinline__ int pe_accept(const DevModel& M, const PeWarp<T>& W, const T* Vs, double** Cpp, int* ldp,
                                      double* Cg, int ldc, const PeMove mv, int n, int N, int lane,
                                      unsigned long long* words) {
  double* Cp = *Cpp;
  int ld = *ldp;
  const double mu = M.mu_q, rr = M.se2 / M.sq2;
  const T muT = (T)M.mu_q;
  const int R = M.R, np = mv.np, kk = mv.kk;
  const Sup sp = mv.sp;
  if (mv.jump == 0) {
    // bordering: u = C^-1 b, delta = r + |a|^2 - b^T u
    for (int i = lane; i < N; i += 32) {
      double s = 0.0;
      for (int a = 0; a < np; ++a) s = fma(Cp[(size_t)W.ovi[a] * ld + i], W.ovb[a], s);
      W.cv[i] = s;
    }
    __syncwarp();
    const double idl = 1.0 / (rr + mv.aa - mv.quad);
    if (N + 1 > ld && Cp != Cg) {  // the tile is full: move C^-1 to the global slot
      for (int i = 0; i < N; ++i)
        for (int j = lane; j < N; j += 32) Cg[(size_t)i * ldc + j] = Cp[(size_t)i * ld + j];
      Cp = Cg;
      ld = ldc;
      __syncwarp();
    }
    for (int j0 = 0; j0 <= N; j0 += 32) {
      const int j = j0 + lane;
      const double uj = j < N ? W.cv[j] * idl : 0.0;
      for (int i = 0; i < N; ++i) {
        const double ui = W.cv[i];
        double* Ci = Cp + (size_t)i * ld;
        if (j < N) Ci[j] = fma(ui, uj, Ci[j]);
        else if (j == N) Ci[N] = -ui * idl;
      }
      if (j < N) Cp[(size_t)N * ld + j] = -uj;
      else if (j == N) Cp[(size_t)N * ld + N] = idl;
    }
    // v' = [v + (t - mu) u; -t], t = (b^T v - mu b^T u - h_new) / delta, h_new = a^T y'
    const double hnew = mv.ay - mu * mv.aa;
    const double t = (mv.bv - mu * mv.quad - hnew) * idl;
    for (int i = lane; i < N; i += 32) W.v[i] = fma(t - mu, W.cv[i], W.v[i]);
    if (lane == 0) { W.v[N] = -t; W.list[N] = mv.jp; }
    for (int i = sp.ilo + lane; i < sp.ihi; i += 32) W.y[sp.w0 + i] -= muT * Vs[sp.ph + i * R];
    *words += (unsigned long long)N * np + 2ull * (N + 1) * (N + 1) + 2 * N + 2 * (sp.ihi - sp.ilo);
    N += 1;
  } else if (mv.jump == 1) {
    // Schur downdate by row k, then the last PE moves into slot k
    for (int i = lane; i < N; i += 32) W.cv[i] = Cp[(size_t)kk * ld + i];
    __syncwarp();
    const double ig = 1.0 / W.cv[kk];
    const int last = N - 1;
    for (int j0 = 0; j0 < last; j0 += 32) {
      const int j = j0 + lane;
      if (j < last) {
        const int mj = (j == kk) ? last : j;
        const double cj = W.cv[mj] * ig;
        for (int i = 0; i < last; ++i) {
          const int mi = (i == kk) ? last : i;
          Cp[(size_t)i * ld + j] = fma(-W.cv[mi], cj, Cp[(size_t)mi * ld + mj]);
        }
      }
    }
    const double fv = (mv.vk + mu) * ig;
    for (int i = lane; i < last; i += 32) {
      const int mi = (i == kk) ? last : i;
      W.v[i] = fma(-W.cv[mi], fv, W.v[mi]);
    }
    const Sup sm = pe_sup(M, n, mv.jm);
    for (int i = sm.ilo + lane; i < sm.ihi; i += 32) W.y[sm.w0 + i] += muT * Vs[sm.ph + i * R];
    __syncwarp();
    if (lane == 0) W.list[kk] = W.list[last];
    *words += (unsigned long long)N + 2ull * last * last + 2 * N + 2 * (sm.ihi - sm.ilo);
    N -= 1;
  } else {
    // update of PE k: downdate by row k and border with b~ = b without its k entry
    double bk = 0.0;
    for (int a = lane; a < np; a += 32)
      if (W.ovi[a] == kk) bk = W.ovb[a];
    bk = wsum(bk);
    for (int i = lane; i < N; i += 32) {
      double s = 0.0;
      for (int a = 0; a < np; ++a) {
        const int qa = W.ovi[a];
        if (qa != kk) s = fma(Cp[(size_t)qa * ld + i], W.ovb[a], s);
      }
      W.uv[i] = s;                        // w = C^-1 b~
      W.cv[i] = Cp[(size_t)kk * ld + i];  // c = row k
    }
    __syncwarp();
    const double ig = 1.0 / W.cv[kk], wk = W.uv[kk];
    for (int i = lane; i < N; i += 32) W.uv[i] = (i == kk) ? 0.0 : fma(-W.cv[i] * ig, wk, W.uv[i]);  // u'
    __syncwarp();
    double bu = 0.0;
    for (int a = lane; a < np; a += 32) {
      const int qa = W.ovi[a];
      if (qa != kk) bu = fma(W.ovb[a], W.uv[qa], bu);
    }
    bu = wsum(bu);
    const double idl = 1.0 / (rr + mv.aa - bu);
    for (int j0 = 0; j0 < N; j0 += 32) {
      const int j = j0 + lane;
      if (j < N) {
        const double cj = W.cv[j] * ig, uj = W.uv[j] * idl;
        for (int i = 0; i < N; ++i) {
          double* Ci = Cp + (size_t)i * ld;
          if (i == kk) Ci[j] = (j == kk) ? idl : -uj;
          else if (j == kk) Ci[j] = -W.uv[i] * idl;
          else Ci[j] = fma(W.uv[i], uj, fma(-W.cv[i], cj, Ci[j]));
        }
      }
    }
    // v: death of k (v_mid), then the birth at slot k on the reduced system
    const double fv = (mv.vk + mu) * ig;
    const double bvm = (mv.bv - bk * mv.vk) - wk * fv;
    const double hnew = mv.ay + mu * bk - mu * mv.aa;
    const double t = (bvm - mu * bu - hnew) * idl;
    for (int i = lane; i < N; i += 32)
      W.v[i] = (i == kk) ? -t : fma(t - mu, W.uv[i], fma(-W.cv[i], fv, W.v[i]));
    const Sup sm = pe_sup(M, n, mv.jm);
    for (int i = sm.ilo + lane; i < sm.ihi; i += 32) W.y[sm.w0 + i] += muT * Vs[sm.ph + i * R];
    __syncwarp();
    for (int i = sp.ilo + lane; i < sp.ihi; i += 32) W.y[sp.w0 + i] -= muT * Vs[sp.ph + i * R];
    if (lane == 0) W.list[kk] = mv.jp;
    *words += (unsigned long long)N * np + N + 2ull * N * N + 2 * N + 2 * (sm.ihi - sm.ilo) + 2 * (sp.ihi - sp.ilo);
  }
  __syncwarp();
  for (int i = lane; i < N; i += 32) W.vT[i] = (T)W.v[i];
  __syncwarp();
  *Cpp = Cp;
  *ldp = ld;
  return N;
}

template <typename T>
__global__ void __launch_bounds__(256) pe_kernel(DevModel M, BatchView B, PeSlots G) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool fp32 = sizeof(T) == 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int n_alloc = B.n_max, n_cap = M.n_cap, Ns = G.Ns;
  // block tables: the SER and log(i), i = 1 .. n_cap + 1
  T* Vs = reinterpret_cast<T*>(smem_raw);
  T* lgN = reinterpret_cast<T*>(smem_raw + a16(sizeof(T) * M.Lt));
  for (int m = threadIdx.x; m < M.Lt; m += blockDim.x) Vs[m] = PeTab<T>::V(M)[m];
  for (int i = threadIdx.x; i < n_cap + 2; i += blockDim.x) lgN[i] = i > 0 ? (T)log((double)i) : (T)0;
  __syncthreads();
  PeWarp<T> W = pe_carve<T>(smem_raw + pe_block_bytes<T>(M.Lt, n_cap) +
                                (size_t)warp * pe_warp_bytes<T>(n_cap, n_alloc, M.win_extra, Ns),
                            n_cap, n_alloc, M.win_extra, Ns);
  PeStats& S = *W.st;
  const size_t slot = (size_t)blockIdx.x * nwarps + warp;
  double* const Cg = G.C ? G.C + slot * G.c_stride : nullptr;
  double* const ws = G.ws ? G.ws + slot * G.ws_stride : nullptr;
  const double* __restrict__ tc = M.tc64;
  const double iq = 1.0 / M.sq2, rr = M.se2 / M.sq2;
  const T q = (T)M.sq2, mu = (T)M.mu_q;
  const T Jt = (T)M.J, logJ = (T)M.log_J, inv_gT = (T)M.inv_g;
  const int R = M.R;

  for (;;) {
    int ci = 0;
    if (lane == 0) ci = atomicAdd(G.counter, 1);
    ci = __shfl_sync(kFull, ci, 0);
    if (ci >= B.n_waveforms) break;
    const int wi = B.order ? B.order[ci] : ci;
    // ------------------------------------------------------------- chain set-up
    const int o0 = B.offsets[wi], n = B.offsets[wi + 1] - o0;
    const float* __restrict__ w = B.samples + o0;
    const double lambda0 = B.lambda0[wi];
    const double t_origin = B.t_origin ? B.t_origin[wi] : 0.0;
    const int T_lo = B.T_lo ? B.T_lo[wi] : 0;
    const int T_hi = B.T_hi ? B.T_hi[wi] : n * R;
    const int k0_lo = (int)ceil((M.t0_lo - t_origin) / M.g - 1e-9);
    const int k0_hi = (int)floor((M.t0_hi - t_origin) / M.g + 1e-9);
    const uint64_t seed = B.seeds ? B.seeds[wi] : B.seed;
    const uint64_t wf_id = B.wf_ids ? B.wf_ids[wi] : B.index_base + (uint64_t)wi;
    const int n_steps = B.n_steps_arr ? B.n_steps_arr[wi] : B.n_steps;
    const int burn_in = B.burn_in_arr ? B.burn_in_arr[wi] : B.burn_in;
    fsmp_summary* out = B.out + wi;
    fsmp_trace* trace = B.trace ? B.trace + (B.trace_off ? B.trace_off[wi] : (int64_t)wi * n_steps) : nullptr;
    const bool invalid = n < 1 || n > n_alloc || T_hi <= T_lo || k0_hi < k0_lo || !(lambda0 > 0.0) || n_steps < 0 ||
                         burn_in < 0 || (fp32 && ws == nullptr) || k0_hi - k0_lo + 1 > M.win_extra ||
                         (Cg == nullptr && Ns < n_cap);
    if (invalid) {
      if (lane == 0) {
        fsmp_summary o;
        o.mean_N = o.var_N = o.mean_t0 = o.var_t0 = o.mean_Q = o.var_Q = o.logL = o.logdet = NAN;
        o.drift_max = 0.0; o.alg_bytes = 0.0;
        for (int k = 0; k < 3; ++k) { o.acc[k] = 0; o.prop[k] = 0; }
        o.acc_t0 = o.prop_t0 = o.N_final = o.k0_final = o.n_samples = o.n_refresh = o.reserved = 0;
        o.status = FSMP_ST_INVALID;
        *out = o;
      }
      __syncwarp();
      continue;
    }
    int k0;
    {
      const double t0i = B.t0_init ? B.t0_init[wi] : NAN;
      if (!isnan(t0i)) {
        double kq = rint((t0i - t_origin) / M.g);
        kq = fmin(fmax(kq, (double)k0_lo), (double)k0_hi);
        k0 = (int)kq;
      } else {
        k0 = k0_lo + (k0_hi - k0_lo) / 2;
      }
    }
    // log(Phi_T(t0) g) on the t0 grid (-inf where Phi_T = 0), from the FP64 tables
    for (int k = lane; k <= k0_hi - k0_lo; k += 32) {
      const int kq = k0_lo + k;
      const double tot = pe_cphi<double>(M, T_hi - 1 - kq) - pe_cphi<double>(M, T_lo - 1 - kq);
      W.lPhi[k] = tot > 0.0 ? (T)log(tot * M.g) : (T)-INFINITY;
    }
    // empty z: y = w
    double wsq = 0.0;
    for (int x = lane; x < n; x += 32) {
      const float wx = w[x];
      W.y[x] = (T)wx;
      wsq += (double)wx * (double)wx;
    }
    wsq = wsum(wsq);
    if (lane == 0) {
      S.sN = S.sN2 = S.sK = S.sK2 = 0;
      S.sQ = S.sQ2 = 0.0; S.q_cur = 0.0; S.q_from = 0;
      S.logdet = n * log(M.se2);
      S.logL = -0.5 * (n * kLog2Pi + S.logdet + wsq * M.inv_se2);
      S.drift_max = 0.0; S.alg_words = 0;
      for (int k = 0; k < 3; ++k) { S.acc[k] = 0; S.prop[k] = 0; }
      S.acc_t0 = S.prop_t0 = S.n_refresh = S.status = S.n_acc_refresh = S.refresh_fail = 0;
    }
    __syncwarp();
    const T log_lambda0 = (T)log(lambda0);
    double* Cp = Ns > 0 ? W.Cs : Cg;  // C^-1, row stride ld
    int ld = Ns > 0 ? Ns : G.ldc;
    int N = 0;

    for (int step = 0; step < n_steps; ++step) {
      // ---- random draws of the next kPeRB steps: lane l takes step step + l
      if ((step & (kPeRB - 1)) == 0) {
        double u[8];
#pragma unroll 1
        for (int blk = 0; blk < 2; ++blk) {
          uint64_t c[4] = {(uint64_t)(step + lane), (uint64_t)blk, 0, 0};
          philox4x64_10(c, seed, wf_id);
          for (int k = 0; k < 4; ++k) u[4 * blk + k] = u01_from_bits(c[k]);
        }
        PeRand<T> rd;
        if (!fp32) {
          rd.z1 = (T)(sqrt(-2.0 * log(u[0])) * cos(kTwoPi * u[1]));
          rd.lu0 = (T)log(u[2]);
          rd.z2 = (T)(sqrt(-2.0 * log(u[5])) * cos(kTwoPi * u[6]));
          rd.lu = (T)log(u[7]);
        } else {
          rd.z1 = (T)(sqrtf(-2.0f * logf((float)u[0])) * cosf(6.2831853f * (float)u[1]));
          rd.lu0 = (T)logf((float)u[2]);
          rd.z2 = (T)(sqrtf(-2.0f * logf((float)u[5])) * cosf(6.2831853f * (float)u[6]));
          rd.lu = (T)logf((float)u[7]);
        }
        rd.u3 = (T)u[3];
        rd.u4 = (T)u[4];
        W.rnd[lane] = rd;
        __syncwarp();
      }
      const PeRand<T> rd = W.rnd[step & (kPeRB - 1)];
      // ---- Gibbs part 1: MH on t0 (Sec. 2.4), uniform prior on its grid range
      T la0 = (T)NAN;
      const T lu0 = rd.lu0;
      int t0f = 0, st_a = 0;
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
            const int j = W.list[k];
            part += pe_logphi<T>(M, j - k0p) - pe_logphi<T>(M, j - k0);
          }
          la0 = wsum(part);
        }
        if (lu0 < la0) { k0 = k0p; t0f |= 2; }
      }
      // ---- Gibbs part 2: one RJMCMC jump (Sec. 2.4)
      const int jump = (N == 0) ? 0 : (rd.u3 < Jt ? 0 : (rd.u3 < (T)2 * Jt ? 1 : 2));
      int valid = 0, noop = 0, kk = -1, jp = -1, jm = -1;
      T la_prior = (T)0, la_fixed = (T)-INFINITY;
      const T lu = rd.lu;
      const T lphi_t0 = W.lPhi[k0 - k0_lo];
      if (jump == 0) {
        if (N >= n_cap) {
          st_a |= FSMP_ST_CAPACITY;
        } else if (lphi_t0 > (T)-INFINITY) {
          const T base = pe_cphi<T>(M, T_lo - 1 - k0), tot = pe_cphi<T>(M, T_hi - 1 - k0) - base;
          jp = pe_birth_search<T>(M, T_lo, T_hi, k0, base, rd.u4 * tot, lane);
          valid = jp >= T_lo;
          la_prior = log_lambda0 + lphi_t0 - lgN[N + 1] + (N == 0 ? logJ : (T)0);
        }
      } else {
        kk = fp32 ? __float2int_rd((float)(rd.u4 * (T)N)) : __double2int_rd((double)(rd.u4 * (T)N));
        if (kk >= N) kk = N - 1;
        jm = W.list[kk];
        if (jump == 1) {
          valid = 1;
          la_prior = -log_lambda0 - lphi_t0 + lgN[N] - (N == 1 ? logJ : (T)0);
        } else {
          const int Dm = fp32 ? __float2int_rn((float)(rd.z2 * inv_gT)) : __double2int_rn((double)(rd.z2 * inv_gT));
          const int jpl = jm + Dm;
          if (Dm == 0) {
            noop = 1;
            la_fixed = (T)0;
          } else if (jpl < T_lo || jpl >= T_hi || pe_logphi<T>(M, jpl - k0) == (T)-INFINITY) {
            la_fixed = (T)-INFINITY;
          } else {
            jp = jpl;
            valid = 1;
            la_prior = pe_logphi<T>(M, jp - k0) - pe_logphi<T>(M, jm - k0);
          }
        }
      }
      // ---- scoring: the 2x2 quantities in PE space (FP64), then the 2x2 algebra in T
      PeMove mv;
      mv.jump = jump; mv.kk = kk; mv.jp = jp; mv.jm = jm; mv.np = 0;
      mv.aa = mv.quad = mv.bv = mv.vk = mv.ay = 0.0;
      mv.sp = Sup{0, 0, 0, 0};
      double mmm = 0, mmp = 0, mpp = 0, gm = 0, gp = 0, em = 1;
      unsigned long long words = 0;
      if (valid) {
        if (jump != 1) {
          const Sup sp = pe_sup(M, n, jp);
          mv.sp = sp;
          // PEs overlapping a_+, with b_q = a_q^T a_+
          int np = 0;
          for (int base = 0; base < N; base += 32) {
            const int qi = base + lane;
            double bq = 0.0;
            if (qi < N) {
              const int o = jp - W.list[qi];
              if (o > -M.Lt && o < M.Lt) bq = xcorr<double>(M, tc, sp, o);
            }
            const bool ov = bq != 0.0;
            const unsigned m = __ballot_sync(kFull, ov);
            if (ov) {
              const int pos = np + __popc(m & ((1u << lane) - 1u));
              W.ovi[pos] = qi;
              W.ovb[pos] = bq;
            }
            np += __popc(m);
          }
          __syncwarp();
          mv.np = np;
          mv.aa = xcorr<double>(M, tc, sp, 0);
          // rows of C^-1 b on the overlap set: lane a holds (C^-1 b)_{ovi[a]} (FP64), so that
          // b^T C^-1 b reduces over np lanes and (C^-1 b)_k is one of them for an update
          T ayp = (T)0, bvp = (T)0;
          for (int i = sp.ilo + lane; i < sp.ihi; i += 32) ayp += Vs[sp.ph + i * R] * W.y[sp.w0 + i];
          double qp = 0.0, ck = 0.0;
          int kpos = -1;
          for (int a0 = 0; a0 < np; a0 += 32) {
            const int a = a0 + lane;
            if (a < np) {
              const double* Crow = Cp + (size_t)W.ovi[a] * ld;
              double rq = 0.0;
              for (int b = 0; b < np; ++b) rq = fma(Crow[W.ovi[b]], W.ovb[b], rq);
              const double ba = W.ovb[a];
              qp = fma(ba, rq, qp);
              bvp += (T)ba * W.vT[W.ovi[a]];
              if (jump == 2 && W.ovi[a] == kk) { ck = rq; kpos = a; }
            }
          }
          mv.quad = np <= 32 ? __shfl_sync(kFull, wsum_first(qp, np), 0) : wsum(qp);
          const T bvT = wsum(bvp);
          const T ayT = wsum(ayp);
          mv.ay = (double)ayT;
          mv.bv = (double)bvT;
          if (jump == 2) {
            // (C^-1 b)_k: from the lane that holds PE k's row, else (no overlap with the
            // old position) a separate dot product
            const unsigned hk = __ballot_sync(kFull, kpos >= 0);
            if (hk) {
              ck = __shfl_sync(kFull, ck, __ffs(hk) - 1);
            } else {
              double c2 = 0.0;
              for (int a = lane; a < np; a += 32) c2 = fma(Cp[(size_t)kk * ld + W.ovi[a]], W.ovb[a], c2);
              ck = wsum(c2);
            }
          }
          mpp = (mv.aa - mv.quad) * M.inv_se2;
          gp = (double)((ayT - bvT) * (T)M.inv_se2);
          mmp = ck * iq;
          words += (unsigned long long)(N + 2 * np + 2 * (sp.ihi - sp.ilo) + np * np + np);
        }
        if (jump != 0) {
          mv.vk = W.v[kk];
          em = rr * Cp[(size_t)kk * ld + kk];
          mmm = (1.0 - em) * iq;
          gm = (double)(W.vT[kk] * (T)iq);
          words += 2;
        }
      }
      T la = la_fixed, dnu = (T)NAN, dT = (T)0;
      int st_c = 0;
      if (valid) {
        // det(I + Lambda M), Lambda = sigma_q^2 diag(-1, 1), with 1 - q m_-- = em
        const T tmm = (T)mmm, tmp = (T)mmp, tpp = (T)mpp, tgm = (T)gm, tgp = (T)gp, tem = (T)em;
        const T Dd = tem * ((T)1 + q * tpp) + q * q * tmp * tmp;
        if (!(Dd > (T)0)) {
          la = (T)-INFINITY;
          st_c |= FSMP_ST_BADDET;
        } else {
          const T iD = (T)1 / Dd;
          const T B11 = -q * ((T)1 + q * tpp) * iD, B12 = q * q * tmp * iD, B22 = q * tem * iD;
          const T rm = tgm - mu * (tmp - tmm), rp = tgp - mu * (tpp - tmp);
          const T dR = (T)-2 * mu * (tgp - tgm) + mu * mu * (tmm - (T)2 * tmp + tpp) -
                       (B11 * rm * rm + (T)2 * B12 * rm * rp + B22 * rp * rp);
          dT = log(Dd);
          dnu = (T)-0.5 * (dT + dR);
          if (!isfinite(dnu)) {
            la = (T)-INFINITY;
            st_c |= FSMP_ST_NONFINITE;
          } else {
            la = dnu + la_prior;
          }
        }
      }
      const int acc = lu < la;
      const int apply = acc && valid && isfinite(la);

      // ---- accepted move: C^-1, v, y and the PE list
      if (apply) {
        N = pe_accept<T>(M, W, Vs, &Cp, &ld, Cg, G.ldc, mv, n, N, lane, &words);
        double qs = 0.0;
        for (int i = lane; i < N; i += 32) qs += W.v[i];
        qs = wsum(qs);
        if (lane == 0) {
          close_hold(S, step, burn_in);
          S.q_cur = N * M.mu_q + qs;
          S.q_from = step;
          S.logdet += (double)dT;
          S.logL += (double)dnu;
          S.n_acc_refresh++;
        }
        __syncwarp();
        if (fp32 && M.refresh_every > 0 && S.n_acc_refresh >= M.refresh_every) {
          double ldv = 0.0, llv = 0.0, dr = 0.0;
          const bool ok = pe_refresh<T>(M, W, Cp, ld, ws, n_cap, pe_lvec(n_cap, n_alloc), w, n, N, lane, ldv, llv, dr);
          double qr = 0.0;
          for (int i = lane; i < N; i += 32) qr += W.v[i];
          qr = wsum(qr);
          if (lane == 0) {
            S.n_acc_refresh = 0;
            if (ok) {
              S.logdet = ldv; S.logL = llv;
              S.drift_max = fmax(S.drift_max, dr);
              if (dr > M.drift_tol) S.status |= FSMP_ST_DRIFT;
              S.n_refresh++;
              S.q_cur = N * M.mu_q + qr;
            } else {
              S.status |= FSMP_ST_DRIFT;
              S.refresh_fail++;
            }
          }
          __syncwarp();
        }
      }

      // ---- bookkeeping of the decided step (lane 0)
      if (lane == 0) {
        S.prop[jump]++;
        if (t0f & 1) { S.prop_t0++; if (t0f & 2) S.acc_t0++; }
        if (apply) S.acc[jump]++;
        S.status |= st_a | st_c;
        S.alg_words += words;
        if (step >= burn_in) {
          const long long Nn = N, kq = k0;
          S.sN += Nn; S.sN2 += Nn * Nn; S.sK += kq; S.sK2 += kq * kq;
        }
        if (trace) {
          fsmp_trace tr;
          tr.la0 = (double)la0; tr.lu0 = (double)lu0; tr.la = (double)la; tr.lu = (double)lu;
          tr.dnu = (double)dnu; tr.N = N; tr.k0 = k0; tr.jump = jump;
          tr.flags = t0f | (acc ? 4 : 0) | ((acc && noop) ? 8 : 0);
          trace[step] = tr;
        }
      }
      __syncwarp();
    }

    // ------------------------------------------------------------- chain end
    if (fp32 && M.refresh_every > 0 && S.n_acc_refresh > 0) {
      // the reported log-likelihood and log|Sigma| come from an FP64 rebuild
      double ldv = 0.0, llv = 0.0, dr = 0.0;
      const bool ok = pe_refresh<T>(M, W, Cp, ld, ws, n_cap, pe_lvec(n_cap, n_alloc), w, n, N, lane, ldv, llv, dr);
      if (lane == 0) {
        if (ok) {
          S.logdet = ldv; S.logL = llv;
          S.drift_max = fmax(S.drift_max, dr);
          if (dr > M.drift_tol) S.status |= FSMP_ST_DRIFT;
          S.n_refresh++;
        } else {
          S.status |= FSMP_ST_DRIFT;
        }
      }
    }
    if (lane == 0) {
      close_hold(S, n_steps, burn_in);
      fsmp_summary o;
      int ns = n_steps - burn_in;
      if (ns < 0) ns = 0;
      const double inv = ns > 0 ? 1.0 / ns : NAN;
      const double mN = (double)S.sN * inv, mK = (double)S.sK * inv;
      o.mean_N = mN; o.var_N = (double)S.sN2 * inv - mN * mN;
      o.mean_t0 = t_origin + M.g * mK; o.var_t0 = M.g * M.g * ((double)S.sK2 * inv - mK * mK);
      o.mean_Q = S.sQ * inv; o.var_Q = S.sQ2 * inv - o.mean_Q * o.mean_Q;
      o.logL = S.logL; o.logdet = S.logdet;
      o.drift_max = S.drift_max; o.alg_bytes = (double)S.alg_words * 8.0;
      for (int k = 0; k < 3; ++k) { o.acc[k] = S.acc[k]; o.prop[k] = S.prop[k]; }
      o.acc_t0 = S.acc_t0; o.prop_t0 = S.prop_t0; o.N_final = N; o.k0_final = k0;
      o.status = S.status; o.n_samples = ns; o.n_refresh = S.n_refresh; o.reserved = 0;
      *out = o;
    }
    __syncwarp();
  }
}

}  // namespace

size_t pe_smem_bytes(const DevModel& M, int n_alloc, int warps, int Ns) {
  if (M.precision == FSMP_FP64)
    return pe_block_bytes<double>(M.Lt, M.n_cap) + (size_t)warps * pe_warp_bytes<double>(M.n_cap, n_alloc, M.win_extra, Ns);
  return pe_block_bytes<float>(M.Lt, M.n_cap) + (size_t)warps * pe_warp_bytes<float>(M.n_cap, n_alloc, M.win_extra, Ns);
}

size_t pe_ws_slot_doubles(int n_cap, int n_alloc) { return pe_ws_doubles(n_cap, n_alloc); }

int pe_ldc(int n_cap) { return (n_cap + 31) / 32 * 32; }

cudaError_t pe_kernel_attributes(int precision, int max_smem) {
  if (precision == FSMP_FP64)
    return cudaFuncSetAttribute(pe_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  return cudaFuncSetAttribute(pe_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

int pe_kernel_occupancy(int precision, int threads, size_t smem) {
  int n = 0;
  cudaError_t e = precision == FSMP_FP64
                      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pe_kernel<double>, threads, smem)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pe_kernel<float>, threads, smem);
  return e == cudaSuccess ? n : 0;
}

cudaError_t launch_pe(const DevModel& M, const BatchView& B, int warps, int ctas, int Ns, size_t smem, void* cinv,
                      size_t c_stride, double* ws, size_t ws_stride, int* counter, cudaStream_t st) {
  PeSlots G;
  G.C = reinterpret_cast<double*>(cinv);
  G.c_stride = c_stride;
  G.ldc = pe_ldc(M.n_cap);
  G.ws = ws;
  G.ws_stride = ws_stride;
  G.counter = counter;
  G.Ns = Ns;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (M.precision == FSMP_FP64) pe_kernel<double><<<ctas, warps * 32, smem, st>>>(M, B, G);
  else pe_kernel<float><<<ctas, warps * 32, smem, st>>>(M, B, G);
  return cudaGetLastError();
}

}  // namespace fsmp
