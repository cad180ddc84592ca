// fsmp_pe_kernel.cuh -- device code of the PE-space chain kernel, compiled by fsmp_pe.cu (the
// dynode charge model) and fsmp_pe_mix.cu (the MCP charge mixture), each instantiating its own
// kernels so that the two build in parallel.
//
// The FSMP chain in PE space, a warp or half warp per chain (arXiv 2403.03156, Sec. 2.4 and
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
// the 2x2 quantities of Eqs. (16)-(18). With the MCP charge mixture (Appendix A.2) each PE k has
// its own mean mu_k, variance sigma_k^2 and r_k = sigma_eps^2 / sigma_k^2: C = diag(r_k) + A^T A,
// log|Sigma| = n log sigma_eps^2 + log|C| - sum_k log r_k, and sigma_q^2, r above become those of
// the PE concerned (the dynode model is the one-component case). Only the p PEs whose support
// overlaps a_+ have b != 0, so a
// proposal reads p^2 + O(p) entries of C^-1 and no n-vector beyond a_+'s support. An accepted move
// updates C^-1 by bordering (birth), a Schur-complement downdate (death) or both in one pass
// (update): O(N^2) instead of the O(n^2) of Sigma^-1. The charge summary is
// E[Q | z, w] = sum_k (mu_k + v_k). Inner products a_i^T a_j over the window come from the SER
// cross-correlation prefix table.
//
// Layout: a chain runs on a group of L consecutive lanes (L = 32: a warp; L = 16: two chains per
// warp, for chains with few PEs, where most of a step is work that every lane repeats); a CTA
// holds several independent chains and a group takes chains from a launch-wide counter. C^-1 sits
// in a per-chain shared-memory tile (the packed triangle of Ns PEs) while N <= Ns and moves to the
// chain's global slot (n_cap PEs) when a birth would exceed the tile. The counts of N after
// burn-in (for lambda_FSMP) sit in a global slot per chain.
//
// Precision. For PEs close in time C is nearly singular (eigenvalues down to r) and C^-1 holds
// entries near 1/r that cancel in b^T C^-1 b; stored in FP32 they cost about 1e-2 in log alpha per
// step. C^-1, v and b therefore carry twice the working precision: in FP32 mode float-float pairs
// (hi + lo, Dekker's exact product and Knuth's TwoSum) that run on the FP32 pipe -- an FP64
// instruction costs this part as much as 64 FP32 ones -- and in FP64 mode double-double pairs
// built the same way, so that a_+^T Sigma^-1 a_+ = (|a_+|^2 - b^T C^-1 b) / sigma_eps^2 keeps FP64
// accuracy where |a_+|^2 and b^T C^-1 b nearly cancel (chains with many overlapping PEs, and
// small r when a mixture component is wide). In FP32 mode the residual y,
// the SER and phi tables, the random draws and the 2x2 algebra are FP32, and C^-1, v, y, log|Sigma|
// and the log-likelihood are rebuilt from z in FP64 (Gauss-Jordan inversion of C, which is
// symmetric positive definite) every refresh_every accepted moves and at the end. Per step the
// random draws, proposal rules and acceptance tests are those of the Sigma^-1 kernel.
#pragma once
#include <math.h>

#include "fsmp_internal.h"

namespace fsmp {
namespace {

constexpr int kPeMaxThreads = 128;  // warps per CTA: at most 4

// The lanes of one chain: L consecutive lanes of a warp. Exchanges and reductions stay inside the
// group; gm is its lane mask. A step draws the random numbers of the next L steps (one per lane).
template <int L> struct Lanes {
  int sl;       // lane within the group
  int g;        // group within the warp
  unsigned gm;  // lane mask of the group
};
template <int L> __device__ __forceinline__ Lanes<L> pe_lanes() {
  static_assert(L == 32 || L == 16, "a chain runs on 32 or 16 lanes");
  const int lane = threadIdx.x & 31;
  Lanes<L> r;
  r.sl = lane & (L - 1);
  r.g = lane / L;
  r.gm = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << (r.g * L));
  return r;
}
// the group's lanes with p set, as bits 0 .. L-1
template <int L> __device__ __forceinline__ unsigned gballot(bool p, const Lanes<L> ln) {
  const unsigned b = __ballot_sync(ln.gm, p);
  if constexpr (L == 32) return b;
  else return (b >> (ln.g * L)) & ((1u << L) - 1u);
}

// ---------------------------------------------------------------- float-float / double-double arithmetic
// A value hi + lo with |lo| <= ulp(hi) / 2. TwoSum (Knuth) and the FMA-based exact product
// (Dekker) give the rounding error of one FP32 operation exactly; the pair operations below are
// the usual "sloppy" double-float forms (relative error about 2^-44).
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_quick(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff x, ff y) {
  const float s = __fadd_rn(x.hi, y.hi);
  const float bb = __fsub_rn(s, x.hi);
  const float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y.hi, bb));
  return ff_quick(s, __fadd_rn(e, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return ff_quick(p, e);
}
__device__ __forceinline__ ff ff_neg(ff x) { return ff{-x.hi, -x.lo}; }

// The same pair arithmetic in FP64 (double-double, about 2^-100 relative error).
struct dd {
  double hi, lo;
};
__device__ __forceinline__ dd dd_quick(double a, double b) {  // |a| >= |b|
  const double s = __dadd_rn(a, b);
  return dd{s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ __forceinline__ dd dd_add(dd x, dd y) {
  const double s = __dadd_rn(x.hi, y.hi);
  const double bb = __dsub_rn(s, x.hi);
  const double e = __dadd_rn(__dsub_rn(x.hi, __dsub_rn(s, bb)), __dsub_rn(y.hi, bb));
  return dd_quick(s, __dadd_rn(e, __dadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dd dd_mul(dd x, dd y) {
  const double p = __dmul_rn(x.hi, y.hi);
  double e = __fma_rn(x.hi, y.hi, -p);
  e = __fma_rn(x.hi, y.lo, e);
  e = __fma_rn(x.lo, y.hi, e);
  return dd_quick(p, e);
}
__device__ __forceinline__ dd dd_neg(dd x) { return dd{-x.hi, -x.lo}; }

// The state arithmetic: C = dd (FP64 mode) or ff (FP32 mode). The plain FP64 forms serve the
// FP64 refresh.
__device__ __forceinline__ double cadd(double a, double b) { return a + b; }
__device__ __forceinline__ double csub(double a, double b) { return a - b; }
__device__ __forceinline__ double cmul(double a, double b) { return a * b; }
__device__ __forceinline__ double cfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double cneg(double a) { return -a; }
__device__ __forceinline__ double crcp(double a) { return 1.0 / a; }
__device__ __forceinline__ double cnum(double a) { return a; }   // to the scoring precision
__device__ __forceinline__ double c64(double a) { return a; }    // to FP64
__device__ __forceinline__ bool cnz(double a) { return a != 0.0; }
template <int L> __device__ __forceinline__ double cshfl_xor(double a, int o, unsigned gm) {
  return __shfl_xor_sync(gm, a, o, L);
}
template <int L> __device__ __forceinline__ double cshfl(double a, int src, unsigned gm) {
  return __shfl_sync(gm, a, src, L);
}
template <typename C> __device__ __forceinline__ C czero();
template <> __device__ __forceinline__ double czero<double>() { return 0.0; }

__device__ __forceinline__ dd cadd(dd a, dd b) { return dd_add(a, b); }
__device__ __forceinline__ dd csub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ dd cmul(dd a, dd b) { return dd_mul(a, b); }
__device__ __forceinline__ dd cfma(dd a, dd b, dd c) { return dd_add(dd_mul(a, b), c); }
__device__ __forceinline__ dd cneg(dd a) { return dd_neg(a); }
__device__ __forceinline__ dd crcp(dd a) {  // one Newton step on the FP64 reciprocal
  const double r = 1.0 / a.hi;
  const dd e = dd_add(dd{1.0, 0.0}, dd_neg(dd_mul(a, dd{r, 0.0})));
  return dd_add(dd{r, 0.0}, dd_mul(e, dd{r, 0.0}));
}
__device__ __forceinline__ double cnum(dd a) { return __dadd_rn(a.hi, a.lo); }
__device__ __forceinline__ double c64(dd a) { return __dadd_rn(a.hi, a.lo); }
__device__ __forceinline__ bool cnz(dd a) { return a.hi != 0.0; }
template <int L> __device__ __forceinline__ dd cshfl_xor(dd a, int o, unsigned gm) {
  return dd{__shfl_xor_sync(gm, a.hi, o, L), __shfl_xor_sync(gm, a.lo, o, L)};
}
template <int L> __device__ __forceinline__ dd cshfl(dd a, int src, unsigned gm) {
  return dd{__shfl_sync(gm, a.hi, src, L), __shfl_sync(gm, a.lo, src, L)};
}
template <> __device__ __forceinline__ dd czero<dd>() { return dd{0.0, 0.0}; }

__device__ __forceinline__ ff cadd(ff a, ff b) { return ff_add(a, b); }
__device__ __forceinline__ ff csub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff cmul(ff a, ff b) { return ff_mul(a, b); }
__device__ __forceinline__ ff cfma(ff a, ff b, ff c) { return ff_add(ff_mul(a, b), c); }
__device__ __forceinline__ ff cneg(ff a) { return ff_neg(a); }
__device__ __forceinline__ ff crcp(ff a) {  // one Newton step on the FP32 reciprocal
  const float r = __frcp_rn(a.hi);
  const ff e = ff_add(ff{1.0f, 0.0f}, ff_neg(ff_mul(a, ff{r, 0.0f})));
  return ff_add(ff{r, 0.0f}, ff_mul(e, ff{r, 0.0f}));
}
__device__ __forceinline__ float cnum(ff a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ double c64(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ bool cnz(ff a) { return a.hi != 0.0f; }
template <int L> __device__ __forceinline__ ff cshfl_xor(ff a, int o, unsigned gm) {
  return ff{__shfl_xor_sync(gm, a.hi, o, L), __shfl_xor_sync(gm, a.lo, o, L)};
}
template <int L> __device__ __forceinline__ ff cshfl(ff a, int src, unsigned gm) {
  return ff{__shfl_sync(gm, a.hi, src, L), __shfl_sync(gm, a.lo, src, L)};
}
// a scoring-precision value (T) as a state value
__device__ __forceinline__ ff cfromf(float a) { return ff{a, 0.0f}; }
__device__ __forceinline__ dd cfromf(double a) { return dd{a, 0.0}; }
// a table entry as a value of type C: cross-correlation tables are FP64 (refresh, FP64 mode)
// or float-float (FP32 mode)
template <typename C> __device__ __forceinline__ C cload(double a);
template <> __device__ __forceinline__ double cload<double>(double a) { return a; }
template <> __device__ __forceinline__ dd cload<dd>(double a) { return dd{a, 0.0}; }
template <typename C> __device__ __forceinline__ C cload(ff a);
template <> __device__ __forceinline__ ff cload<ff>(ff a) { return a; }
template <> __device__ __forceinline__ ff czero<ff>() { return ff{0.0f, 0.0f}; }
// FP64 -> state value (refresh only)
template <typename C> __device__ __forceinline__ C cfrom64(double a);
template <> __device__ __forceinline__ dd cfrom64<dd>(double a) { return dd{a, 0.0}; }
template <> __device__ __forceinline__ ff cfrom64<ff>(double a) {
  const float h = (float)a;
  return ff{h, (float)(a - (double)h)};
}
// mean and r = sigma_eps^2 / sigma_e^2 of charge component e as state values (split into
// pairs on the host)
template <typename C> __device__ __forceinline__ C c_mu(const DevModel& M, int e);
template <> __device__ __forceinline__ dd c_mu<dd>(const DevModel& M, int e) { return dd{M.cm_mu[e], 0.0}; }
template <> __device__ __forceinline__ ff c_mu<ff>(const DevModel& M, int e) { return ff{M.cm_mu_hi[e], M.cm_mu_lo[e]}; }
template <typename C> __device__ __forceinline__ C c_r(const DevModel& M, int e);
template <> __device__ __forceinline__ dd c_r<dd>(const DevModel& M, int e) { return dd{M.cm_r[e], 0.0}; }
template <> __device__ __forceinline__ ff c_r<ff>(const DevModel& M, int e) { return ff{M.cm_r_hi[e], M.cm_r_lo[e]}; }

// A charge component's constant in the scoring precision T: the FP32 copies in FP32 mode, so
// that the step loop converts nothing from FP64 (an FP64 instruction costs this part as much as
// 64 FP32 ones).
template <typename T> struct CmT;
template <> struct CmT<float> {
  __device__ static float mu(const DevModel& M, int e) { return M.cmf_mu[e]; }
  __device__ static float q(const DevModel& M, int e) { return M.cmf_q[e]; }
  __device__ static float iq(const DevModel& M, int e) { return M.cmf_iq[e]; }
  __device__ static float r(const DevModel& M, int e) { return M.cmf_r[e]; }
};
template <> struct CmT<double> {
  __device__ static double mu(const DevModel& M, int e) { return M.cm_mu[e]; }
  __device__ static double q(const DevModel& M, int e) { return M.cm_q[e]; }
  __device__ static double iq(const DevModel& M, int e) { return M.cm_iq[e]; }
  __device__ static double r(const DevModel& M, int e) { return M.cm_r[e]; }
};

// Component of a born or updated PE, e+ ~ G (Sec. 2.4): the smallest e whose cumulative
// probability exceeds the uniform u, else the last component with G > 0. The comparison is
// in FP64 in both modes, so the draw is the same as the FP64 reference's.
__device__ __forceinline__ int pe_draw_comp(const DevModel& M, double u) {
  for (int e = 0; e < M.n_comp; ++e)
    if (M.cm_cum[e] > u) return e;
  return M.cm_last;
}

// group sums of state values: over all lanes, or over lanes [0, m) (zero beyond m)
template <int L, typename C> __device__ __forceinline__ C csum(C v, const Lanes<L> ln) {
#pragma unroll 1
  for (int o = L / 2; o > 0; o >>= 1) v = cadd(v, cshfl_xor<L>(v, o, ln.gm));
  return v;
}
template <int L, typename C> __device__ __forceinline__ C csum_first(C v, int m, const Lanes<L> ln) {
  for (int o = L / 2; o > 0; o >>= 1)
    if (o < m) v = cadd(v, cshfl_xor<L>(v, o, ln.gm));
  return cshfl<L>(v, 0, ln.gm);
}

// twice a state value (exact)
__device__ __forceinline__ double ctwice(double a) { return 2.0 * a; }
__device__ __forceinline__ dd ctwice(dd a) { return dd{2.0 * a.hi, 2.0 * a.lo}; }
__device__ __forceinline__ ff ctwice(ff a) { return ff{2.0f * a.hi, 2.0f * a.lo}; }

// two group sums of state values in one butterfly
template <int L, typename C> __device__ __forceinline__ void csum2(C& a, C& b, const Lanes<L> ln) {
#pragma unroll 1
  for (int o = L / 2; o > 0; o >>= 1) {
    const C a2 = cshfl_xor<L>(a, o, ln.gm), b2 = cshfl_xor<L>(b, o, ln.gm);
    a = cadd(a, a2);
    b = cadd(b, b2);
  }
}

// four group sums in one butterfly (two state values, two scoring-precision values), so that
// their shuffles and additions overlap
template <int L, typename C, typename T>
__device__ __forceinline__ void gsum4(C& a, C& b, T& x, T& y, const Lanes<L> ln) {
#pragma unroll 1
  for (int o = L / 2; o > 0; o >>= 1) {
    const C a2 = cshfl_xor<L>(a, o, ln.gm), b2 = cshfl_xor<L>(b, o, ln.gm);
    const T x2 = __shfl_xor_sync(ln.gm, x, o, L), y2 = __shfl_xor_sync(ln.gm, y, o, L);
    a = cadd(a, a2);
    b = cadd(b, b2);
    x += x2;
    y += y2;
  }
}

// C^-1 is symmetric and stored as its lower triangle, row by row: entry (i, j), j <= i, at
// tri(i) + j. The storage has no row stride, so a chain's C^-1 moves from the shared tile to
// its global slot by a plain copy.
__host__ __device__ __forceinline__ int tri(int i) { return i * (i + 1) / 2; }
__device__ __forceinline__ int pk(int i, int j) { return i >= j ? tri(i) + j : tri(j) + i; }
// (i, j) of packed position e (j <= i); the FP32 square root is exact enough below 2^22
__device__ __forceinline__ void untri(int e, int& i, int& j) {
  i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  if (tri(i + 1) <= e) ++i;
  if (tri(i) > e) --i;
  j = e - tri(i);
}

// sum_a C^-1[q][idx[a]] b[a] over a < m (skipping idx[a] == skip); BIG (C^-1 in global memory):
// four independent partial sums so that the gathers of consecutive terms overlap
template <typename C, bool BIG>
__device__ __forceinline__ C dot_row(const C* __restrict__ Cp, int q, const int* __restrict__ idx,
                                     const C* __restrict__ b, int m, int skip) {
  C s0 = czero<C>();
  int a = 0;
  if constexpr (BIG) {
    constexpr int G = 4;
    C sp[G];
#pragma unroll
    for (int u = 0; u < G; ++u) sp[u] = czero<C>();
#pragma unroll 1
    for (; a + G - 1 < m; a += G) {
      int ix[G];
      C r[G];
#pragma unroll
      for (int u = 0; u < G; ++u) {
        ix[u] = idx[a + u];
        r[u] = Cp[pk(q, ix[u])];
      }
#pragma unroll
      for (int u = 0; u < G; ++u)
        if (ix[u] != skip) sp[u] = cfma(r[u], b[a + u], sp[u]);
    }
#pragma unroll
    for (int u = 1; u < G; ++u) sp[0] = cadd(sp[0], sp[u]);
    s0 = sp[0];
  }
#pragma unroll 1
  for (; a < m; ++a)
    if (idx[a] != skip) s0 = cfma(Cp[pk(q, idx[a])], b[a], s0);
  return s0;
}

template <int L, typename T> __device__ __forceinline__ T wsum(T v, const Lanes<L> ln) {
#pragma unroll 1
  for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(ln.gm, v, o, L);
  return v;
}
template <int L, typename T> __device__ __forceinline__ T wmax(T v, const Lanes<L> ln) {
#pragma unroll 1
  for (int o = L / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(ln.gm, v, o, L));
  return v;
}

// ---------------------------------------------------------------- model tables
template <typename T> struct PeTab;
template <> struct PeTab<double> {
  using C = dd;
  __device__ static const double* V(const DevModel& M) { return M.V64; }
  __device__ static const double* logphi(const DevModel& M) { return M.logphi; }
  __device__ static const double* cphi(const DevModel& M) { return M.cphi; }
  __device__ static const double* tc(const DevModel& M) { return M.tc64; }
};
template <> struct PeTab<float> {
  using C = ff;
  __device__ static const float* V(const DevModel& M) { return M.V32; }
  __device__ static const float* logphi(const DevModel& M) { return M.logphi32; }
  __device__ static const float* cphi(const DevModel& M) { return M.cphi32; }
  __device__ static const ff* tc(const DevModel& M) { return reinterpret_cast<const ff*>(M.tcff); }
};

template <typename T> __device__ __forceinline__ T pe_logphi(const DevModel& M, int d) {
  return (d < -M.D || d > M.D) ? (T)-INFINITY : __ldg(PeTab<T>::logphi(M) + (d + M.D));
}
template <typename T> __device__ __forceinline__ T pe_cphi(const DevModel& M, int d) {
  if (d < -M.D) return (T)0;
  if (d > M.D) return __ldg(PeTab<T>::cphi(M) + 2 * M.D);
  return __ldg(PeTab<T>::cphi(M) + (d + M.D));
}

// Support of the PE at grid index j in a window of n samples: its first sample w0 = ceil(j / R),
// the phase ph = w0 R - j of that sample, and the range [ilo, ihi) of its support samples
// (sample w0 + i, SER index ph + i R) that lie in the window.
struct Sup {
  int w0, ph, ilo, ihi;
};
__device__ __forceinline__ Sup pe_sup(const DevModel& M, int n, int j) {
  Sup s;
  // w0 = ceil(j / R) = floor((j + R - 1) / R): an FP32 estimate (off by at most one for
  // |j| < 2^22) corrected by one integer step, instead of a division
  const int num = j + M.R - 1;
  int q = __float2int_rd((float)num * M.inv_Rf);
  if (q * M.R > num) --q;
  else if ((q + 1) * M.R <= num) ++q;
  s.w0 = q;
  s.ph = q * M.R - j;
  s.ilo = max(0, -q);
  s.ihi = min(M.L_V, n - q);  // every phase ph < R covers L_V samples (Lt = L_V R)
  if (s.ihi <= s.ilo) s.ilo = s.ihi = 0;  // no sample of the window: an all-zero column
  return s;
}

// a_x^T a_q over the window, for x with support s and q = x - o (|o| < Lt), from the prefix table.
template <typename C, typename TT>
__device__ __forceinline__ C xcorr(const DevModel& M, const TT* __restrict__ tc, const Sup& s, int o) {
  const int O = 2 * M.Lt - 1;
  const TT* base = tc + (size_t)s.ph * M.tcM * O + (o + M.Lt - 1);
  C v = cload<C>(base[(size_t)s.ihi * O]);
  if (s.ilo > 0) v = csub(v, cload<C>(base[(size_t)s.ilo * O]));
  return v;
}

// Smallest j in [T_lo, T_hi) with cphi(j - k0) - base > target (L-ary group search; cphi is
// non-decreasing, so the answer does not depend on L); if rounding leaves none, the last j of T
// with phi > 0.
template <typename T, int L>
__device__ int pe_birth_search(const DevModel& M, int T_lo, int T_hi, int k0, T base, T target, const Lanes<L> ln) {
  int lo = T_lo, hi = T_hi - 1;
  if ((pe_cphi<T>(M, hi - k0) - base) > target) {
    while (lo < hi) {
      const int len = hi - lo + 1;
      const int step = (len + L - 1) / L;
      const int p = min(hi, lo + (ln.sl + 1) * step - 1);
      const bool pred = (pe_cphi<T>(M, p - k0) - base) > target;
      const unsigned b = gballot(pred, ln);
      const int f = __ffs(b) - 1;
      const int new_lo = lo + f * step;
      hi = min(hi, lo + (f + 1) * step - 1);
      lo = new_lo;
    }
    return lo;
  }
  int last = -1;
  for (int top = T_hi - 1; top >= T_lo; top -= L) {
    const int j = top - ln.sl;
    const bool ok = j >= T_lo && pe_logphi<T>(M, j - k0) > (T)-INFINITY;
    const unsigned b = gballot(ok, ln);
    if (b) { last = top - (__ffs(b) - 1); break; }
  }
  return last;
}

template <typename T> struct PeRand {
  T z1, lu0, u3, u4, z2, lu;  // t0 shift normal, log u2, jump type, PE choice, shift normal, log u7
  int ep;                     // charge component of a born or updated PE
};

// FP32 value of the uniform ((x >> 11) + 0.5) 2^-53: the odd 54-bit integer 2 (x >> 11) + 1
// rounded to FP32, times 2^-54 (exact), i.e. the FP64 uniform rounded to FP32 without FP64 work.
__device__ __forceinline__ float u01_float(uint64_t x) {
  return __ull2float_rn(((x >> 11) << 1) | 1ull) * 0x1.0p-54f;
}

// Per-chain statistics (shared memory, written by the group's first lane).
struct PeStats {
  long long sN, sN2, sK, sK2;
  long long St, Se;  // sum of |t_k| (grid units) and of e_k over the PEs of the state
  double sQ, sQ2, q_cur, logdet, logL, drift_max, wsq;
  // the Wasserstein scalars of the state (held like q_cur) and their sums
  double wt_cur, we_cur, sWt, sWt2, sWe, sWe2;
  unsigned long long alg_words;
  int acc[3], prop[3], acc_t0, prop_t0, n_refresh, status, q_from, n_acc_refresh, refresh_fail, pad;
};

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

// Per-chain shared memory. C is the state type (16 bytes in FP64 mode, 8 in FP32 mode).
template <typename T> struct PeChain {
  using C = typename PeTab<T>::C;
  PeStats* st;
  PeRand<T>* rnd;  // draws of the next L steps [L]
  int* list;   // PE grid indices [n_cap]
  unsigned char* le;  // PE charge components [n_cap]
  int* ovi;    // PEs overlapping the proposed one [n_cap]
  C* ovb;      // their inner products with it [n_cap]
  C* v;        // C^-1 A^T y [n_cap]
  C* cv;       // row k of C^-1 / C^-1 b [n_cap]
  C* uv;       // second work vector [n_cap]
  T* y;        // residual [n_alloc]
  T* lPhi;     // log(Phi_T(t0) g) on the chain's t0 grid [win_extra]
  C* Cs;       // C^-1 tile: packed triangle of Ns PEs
};
template <typename T, int L> __host__ __device__ inline size_t pe_chain_bytes(int n_cap, int n_alloc, int win_extra, int Ns) {
  constexpr size_t cs = sizeof(typename PeTab<T>::C);
  return a16(sizeof(PeStats)) + a16(sizeof(PeRand<T>) * L) + 2 * a16(sizeof(int) * n_cap) + a16((size_t)n_cap) +
         4 * a16(cs * (size_t)n_cap) + a16(sizeof(T) * n_alloc) + a16(sizeof(T) * win_extra) +
         a16(cs * (size_t)tri(Ns));
}
// Block tables: the SER, log(i) and 1 / i (i <= n_cap + 1).
template <typename T> __host__ __device__ inline size_t pe_block_bytes(const DevModel& M) {
  return a16(sizeof(T) * M.Lt) + a16(sizeof(T) * (M.n_cap + 2)) + a16(sizeof(double) * (M.n_cap + 2));
}
template <typename T, int L> __device__ PeChain<T> pe_carve(unsigned char* p, int n_cap, int n_alloc, int win_extra, int Ns) {
  using C = typename PeTab<T>::C;
  PeChain<T> W;
  size_t o = 0;
  W.st = reinterpret_cast<PeStats*>(p + o); o += a16(sizeof(PeStats));
  W.rnd = reinterpret_cast<PeRand<T>*>(p + o); o += a16(sizeof(PeRand<T>) * L);
  W.list = reinterpret_cast<int*>(p + o); o += a16(sizeof(int) * n_cap);
  W.le = p + o; o += a16((size_t)n_cap);
  W.ovi = reinterpret_cast<int*>(p + o); o += a16(sizeof(int) * n_cap);
  W.ovb = reinterpret_cast<C*>(p + o); o += a16(sizeof(C) * (size_t)n_cap);
  W.v = reinterpret_cast<C*>(p + o); o += a16(sizeof(C) * (size_t)n_cap);
  W.cv = reinterpret_cast<C*>(p + o); o += a16(sizeof(C) * (size_t)n_cap);
  W.uv = reinterpret_cast<C*>(p + o); o += a16(sizeof(C) * (size_t)n_cap);
  W.y = reinterpret_cast<T*>(p + o); o += a16(sizeof(T) * n_alloc);
  W.lPhi = reinterpret_cast<T*>(p + o); o += a16(sizeof(T) * win_extra);
  W.Cs = reinterpret_cast<C*>(p + o);
  return W;
}

// Global per-chain slots (one per resident chain of the launch).
struct PeSlots {
  void* C;             // C^-1 slots (state entries): the packed triangle of n_cap PEs
  size_t c_stride;     // entries per slot
  double* ws;          // FP64 refresh workspace slots (FP32 mode)
  size_t ws_stride;    // doubles per slot
  int* hist;           // N histogram slots, n_cap + 1 counts each
  int* counter;        // next chain of the launch (zeroed before the launch)
  int Ns;              // shared-memory tile of C^-1 (0: always global)
};

// FP64 refresh workspace of one chain: C (n_cap x n_cap), h and v (n_cap each), a sweep block's
// rows before and after its sweep (n_cap x kSweepBlock each; together they also hold an FP64
// copy of the window while the residual is rebuilt) and the block's pivot factors
// (kSweepBlock x kSweepBlock); every part starts on a 16-byte boundary.
constexpr int kSweepBlock = 8;
__host__ __device__ inline size_t pe_ws_a2(size_t n) { return (n + 1) & ~(size_t)1; }
__host__ __device__ inline size_t pe_ws_doubles(int n_cap) {
  return pe_ws_a2((size_t)n_cap * n_cap) + (2 + 2 * kSweepBlock) * pe_ws_a2(n_cap) + kSweepBlock * kSweepBlock;
}

// Hold of the state's summaries: the charge summary q_cur and the Wasserstein scalars wt_cur,
// we_cur hold from step q_from on (they change only with z); close the hold at step s.
__device__ __forceinline__ void close_hold(PeStats& S, int s, int burn_in) {
  const int from = max(S.q_from, burn_in);
  if (s > from) {
    const double c = (double)(s - from);
    S.sQ += S.q_cur * c;
    S.sQ2 += S.q_cur * S.q_cur * c;
    S.sWt += S.wt_cur * c;
    S.sWt2 += S.wt_cur * S.wt_cur * c;
    S.sWe += S.we_cur * c;
    S.sWe2 += S.we_cur * S.we_cur * c;
  }
}

// The Wasserstein scalars of a state with N PEs (the convergence check of Sec. 3.2): with a
// dummy PE at t = 0, e = 0 added, the 1-Wasserstein distance from the sequence to the dummy
// alone is the mean of |t| (or of e) over the N + 1 points.
// inv1[i] = 1 / i (a block table, so that no FP64 division runs in the step loop).
__device__ __forceinline__ void set_wasserstein(PeStats& S, double g, int N, const double* inv1) {
  const double inv = inv1[N + 1];
  S.wt_cur = g * (double)S.St * inv;
  S.we_cur = (double)S.Se * inv;
}

// lambda_FSMP at the chain end, out of line: the estimator's code stays out of the step loop's
// instruction stream
template <int L>
__device__ __noinline__ double pe_lambda_mle(const int* h, int n_max, double lambda0, int sl, unsigned gm) {
  return group_lambda_mle<L>(h, n_max, lambda0, sl, gm);
}

struct RefreshOut {
  int ok;
  double logdet, logL, drift;
};

// FP64 rebuild of C^-1, v, y, log|Sigma| and the log-likelihood from the PE list (FP32 mode).
// ok = 0 (state untouched) if C is not numerically positive definite. Arguments are passed by
// value (no address of the caller's locals escapes, so they stay in registers).
template <typename T, bool BIG, int L, bool MIX>
__device__ __noinline__ RefreshOut pe_refresh(const DevModel& M, const PeChain<T> W, typename PeTab<T>::C* Cp,
                                              double* ws, int n_cap, const float* w, double wsq, int n,
                                              int N, const Lanes<L> ln) {
  using C = typename PeTab<T>::C;
  RefreshOut out{0, 0.0, 0.0, 0.0};
  const int ws_ld = N > 0 ? N : 1;
  constexpr int SB = BIG ? kSweepBlock : kSweepBlock / 2;  // fewer registers in the compact variant
  const size_t lv = pe_ws_a2(n_cap);
  double* A = ws;                                 // C, then -C^-1 (row-major N x N, lower triangle)
  double* h = A + pe_ws_a2((size_t)n_cap * n_cap);  // A^T y
  double* rowk = h + lv;                          // v
  double* P = rowk + lv;                          // a sweep block's rows before its sweep (N x SB)
  double* Pn = P + (size_t)kSweepBlock * lv;      // the same rows during and after it
  // the block's pivot factors: F[q SB + r] = A_rp / pivot (r != q), F[q SB + q] = 1 / pivot
  double* F = Pn + (size_t)kSweepBlock * lv;
  const double* V = M.V64;
  constexpr bool mix = MIX;
  const double mu = M.cm_mu[0], r = M.cm_r[0];  // the dynode model's (one component)
  // C = diag(r_k) + A^T A (its lower triangle, row-major: entry (i, j) at i N + j for j <= i);
  // lanes over columns, RC rows at a time so that the
  // table loads of the rows overlap. The unrolled forms (BIG: many PEs per chain) cost the
  // caller registers around the call, which the compact variant cannot spare.
  constexpr int RC = BIG ? 4 : 1, RG = BIG ? 4 : 1;
#pragma unroll 1
  for (int j = ln.sl; j < N; j += L) {
    const int jj = W.list[j];
#pragma unroll 1
    for (int i0 = j; i0 < N; i0 += RC) {
      double c[RC];
#pragma unroll
      for (int q = 0; q < RC; ++q) {
        const int i = min(i0 + q, N - 1);
        const int ji = W.list[i];
        const int o = ji - jj;
        c[q] = (o > -M.Lt && o < M.Lt) ? xcorr<double>(M, M.tc64, pe_sup(M, n, ji), o) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < RC; ++q) {
        const int i = i0 + q;
        if (i < N) A[(size_t)i * ws_ld + j] = c[q] + (j == i ? (mix ? M.cm_r[W.le[i]] : r) : 0.0);
      }
    }
  }
  __syncwarp(ln.gm);
  // With y = w - sum_k mu_k a_k: h = A^T y = A^T w - (A^T A) m (m the PEs' means), and
  // y^T y = w^T w - 2 m^T A^T w + m^T A^T A m -- no FP64 copy of y is needed. The dynode
  // model factors its single mean out.
  double awt = 0.0, rst = 0.0;
#pragma unroll 1
  for (int k = ln.sl; k < N; k += L) {
    const Sup s = pe_sup(M, n, W.list[k]);
    // the loops' loads go four at a time ahead of their (unchanged) sums
    double a0 = 0.0, a1 = 0.0;
    int i = s.ilo;
#pragma unroll 1
    for (; i + 3 < s.ihi; i += 4) {
      double vv[4], ww[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        vv[u] = V[s.ph + (i + u) * M.R];
        ww[u] = (double)w[s.w0 + i + u];
      }
      a0 = fma(vv[0], ww[0], a0);
      a1 = fma(vv[1], ww[1], a1);
      a0 = fma(vv[2], ww[2], a0);
      a1 = fma(vv[3], ww[3], a1);
    }
#pragma unroll 1
    for (; i + 1 < s.ihi; i += 2) {
      a0 = fma(V[s.ph + i * M.R], (double)w[s.w0 + i], a0);
      a1 = fma(V[s.ph + (i + 1) * M.R], (double)w[s.w0 + i + 1], a1);
    }
    if (i < s.ihi) a0 = fma(V[s.ph + i * M.R], (double)w[s.w0 + i], a0);
    const double aw = a0 + a1;
    auto c_kj = [&](int j) { return *(j <= k ? A + (size_t)k * ws_ld + j : A + (size_t)j * ws_ld + k); };
    int j = 0;
    if (mix) {
      const int ek = W.le[k];
      const double mk = M.cm_mu[ek];
      double hs = -M.cm_r[ek] * mk;  // (A^T A m)_k = sum_j C_kj m_j - r_k m_k
#pragma unroll 1
      for (; j + 3 < N; j += 4) {
        double cc[4], mm[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          cc[u] = c_kj(j + u);
          mm[u] = M.cm_mu[W.le[j + u]];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) hs = fma(cc[u], mm[u], hs);
      }
#pragma unroll 1
      for (; j < N; ++j) hs = fma(c_kj(j), M.cm_mu[W.le[j]], hs);
      h[k] = aw - hs;
      awt = fma(mk, aw, awt);
      rst = fma(mk, hs, rst);
    } else {
      double rs = -r;
#pragma unroll 1
      for (; j + 3 < N; j += 4) {
        double cc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) cc[u] = c_kj(j + u);
#pragma unroll
        for (int u = 0; u < 4; ++u) rs += cc[u];
      }
#pragma unroll 1
      for (; j < N; ++j) rs += c_kj(j);
      h[k] = aw - mu * rs;
      awt += aw;
      rst += rs;
    }
  }
  awt = wsum(awt, ln);
  rst = wsum(rst, ln);
  const double yy = mix ? wsq - 2.0 * awt + rst : wsq - 2.0 * mu * awt + mu * mu * rst;
  // the FP32 residual, each sample summed in FP64 over the PEs that cover it, in list order: PE
  // by PE with lanes over its support samples, into an FP64 copy of the window held in the
  // sweep's panel buffers (free until the sweep); sample by sample where the window does not fit
  if (n <= 2 * kSweepBlock * (int)lv) {
    double* yd = P;  // P and Pn are contiguous
#pragma unroll 1
    for (int x = ln.sl; x < n; x += L) yd[x] = (double)w[x];
    __syncwarp(ln.gm);
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
      const Sup s = pe_sup(M, n, W.list[k]);
      const double mk = mix ? -M.cm_mu[W.le[k]] : -mu;
#pragma unroll 1
      for (int i = s.ilo + ln.sl; i < s.ihi; i += L) yd[s.w0 + i] = fma(mk, V[s.ph + i * M.R], yd[s.w0 + i]);
      __syncwarp(ln.gm);
    }
#pragma unroll 1
    for (int x = ln.sl; x < n; x += L) W.y[x] = (T)yd[x];
  } else {
#pragma unroll 1
    for (int x = ln.sl; x < n; x += L) {
      double yv = (double)w[x];
#pragma unroll 1
      for (int k = 0; k < N; ++k) {
        const int idx = x * M.R - W.list[k];
        if (idx >= 0 && idx < M.Lt) yv = fma(mix ? -M.cm_mu[W.le[k]] : -mu, V[idx], yv);
      }
      W.y[x] = (T)yv;
    }
  }
  __syncwarp(ln.gm);
  // Inversion by the symmetric sweep operator (Gauss-Jordan with diagonal pivots, kept
  // symmetric): sweeping pivot p maps A_pp -> -1/A_pp, A_pj -> A_pj/A_pp, A_ip -> A_ip/A_pp and
  // A_ij -> A_ij - A_ip A_pj/A_pp. Sweeps commute, sweeping every index leaves -C^-1, and only
  // the lower triangle is kept. The pivots are C's LDL^T pivots (all positive for SPD C):
  // log|C| = sum log pivot, kept as mantissa x 2^exponent. Pivots go SB at a time with one pass
  // over the matrix per block K = [k0, k1): the block's rows A_K. (the panel) are swept first --
  // they change only through their own entries -- then every other entry (i, j), i, j outside K,
  // takes the rank-SB update A_ij -= sum_q P_iq G_qj, with P_i. = A_Ki before the sweep and
  // G_.j = A_Kj after it. Within the panel, the diagonal block A_KK depends on nothing else, so
  // it is swept first and its pivots and factors recorded; each other column A_Kj then takes
  // them in turn (the same operations in the same order as sweeping the panel pivot by pivot).
  double pm = 1.0;
  int pe = 0;
#pragma unroll 1
  for (int k0 = 0; k0 < N; k0 += SB) {
    const int nb = min(SB, N - k0), k1 = k0 + nb;
    // the diagonal block A_KK swept on its own, lane r holding its row r in full; each pivot's
    // row goes to the other lanes by shuffles
    const int rl = ln.sl;
    double kr[SB];
#pragma unroll
    for (int c = 0; c < SB; ++c)
      kr[c] = (rl < nb && c < nb)
                  ? *(c <= rl ? A + (size_t)(k0 + rl) * ws_ld + k0 + c : A + (size_t)(k0 + c) * ws_ld + k0 + rl)
                  : 0.0;
#pragma unroll
    for (int q = 0; q < SB; ++q) {
      if (q < nb) {
        const double piv = __shfl_sync(ln.gm, kr[q], q, L);
        if (!(piv > 0.0) || !isfinite(piv)) return out;
        const double ip = 1.0 / piv;
        int ex;
        pm *= frexp(piv, &ex);
        pe += ex;
        pm = frexp(pm, &ex);
        pe += ex;
        const double fr = kr[q] * ip;  // A_rp / pivot for this lane's row r
        double aq[SB];
#pragma unroll
        for (int c = 0; c < SB; ++c) aq[c] = __shfl_sync(ln.gm, kr[c], q, L);
#pragma unroll
        for (int c = 0; c < SB; ++c)
          kr[c] = (rl == q) ? (c == q ? -ip : aq[c] * ip) : (c == q ? fr : fma(-fr, aq[c], kr[c]));
        if (rl < nb) F[q * SB + rl] = (rl == q) ? ip : fr;
      }
    }
    if (rl < nb) {
#pragma unroll
      for (int c = 0; c < SB; ++c)
        if (c <= rl) A[(size_t)(k0 + rl) * ws_ld + k0 + c] = kr[c];
    }
    __syncwarp(ln.gm);
    // the panel A_Kj of every column j outside the block: P_j. keeps it as it was, then the
    // block's pivots are applied to it in registers and it goes to Pn_j. and back into A
#pragma unroll 1
    for (int j = ln.sl; j < N; j += L) {
      if (j >= k0 && j < k1) continue;
      double b[SB];
#pragma unroll
      for (int q = 0; q < SB; ++q)
        b[q] = q < nb ? *(j > k0 ? A + (size_t)j * ws_ld + k0 + q : A + (size_t)(k0 + q) * ws_ld + j) : 0.0;
#pragma unroll
      for (int q = 0; q < SB; ++q) P[(size_t)j * SB + q] = b[q];
#pragma unroll
      for (int q = 0; q < SB; ++q) {
        if (q < nb) {
          const double apj = b[q];
#pragma unroll
          for (int r = 0; r < SB; ++r)
            if (r < nb) b[r] = (r == q) ? apj * F[q * SB + q] : fma(-F[q * SB + r], apj, b[r]);
        }
      }
#pragma unroll
      for (int q = 0; q < SB; ++q) {
        Pn[(size_t)j * SB + q] = b[q];
        if (q < nb) *(j < k0 ? A + (size_t)(k0 + q) * ws_ld + j : A + (size_t)j * ws_ld + k0 + q) = b[q];
      }
    }
    __syncwarp(ln.gm);
    // every entry (i, j), i >= j, outside the block's rows and columns: lanes over a group of L
    // columns, the rows in step across the lanes (a row's loads coalesce and its P row is one
    // broadcast), RG rows at a time so that their loads overlap
#pragma unroll 1
    for (int j0 = 0; j0 < N; j0 += L) {
      const int j = j0 + ln.sl;
      const bool jv = j < N && (j < k0 || j >= k1);
      double g[SB];
#pragma unroll
      for (int q = 0; q < SB; ++q) g[q] = jv ? Pn[(size_t)j * SB + q] : 0.0;
      // the column group's rows: [j0, k0) above the block, then [max(j0, k1), N) below it; the
      // next RG rows' entries are loaded while the current ones are updated
      const int nA = max(0, k0 - j0), s2 = max(j0, k1), nr = nA + max(0, N - s2);
      auto row = [&](int t) { return t < nA ? j0 + t : s2 + (t - nA); };
      double xn[RG];
#pragma unroll
      for (int t = 0; t < RG; ++t) {
        const int r = row(t);
        xn[t] = (jv && t < nr && r >= j) ? A[(size_t)r * ws_ld + j] : 0.0;
      }
#pragma unroll 1
      for (int t0 = 0; t0 < nr; t0 += RG) {
        double x[RG];
        int rr[RG];
#pragma unroll
        for (int t = 0; t < RG; ++t) {
          x[t] = xn[t];
          rr[t] = row(min(t0 + t, nr - 1));
          const int tt = t0 + RG + t, r = row(tt);
          xn[t] = (jv && tt < nr && r >= j) ? A[(size_t)r * ws_ld + j] : 0.0;
        }
#pragma unroll
        for (int t = 0; t < RG; ++t) {
          const double2* Pi = reinterpret_cast<const double2*>(P + (size_t)rr[t] * SB);
#pragma unroll
          for (int q = 0; q < SB / 2; ++q) {
            const double2 pq = Pi[q];
            x[t] = fma(-pq.x, g[2 * q], x[t]);
            x[t] = fma(-pq.y, g[2 * q + 1], x[t]);
          }
        }
#pragma unroll
        for (int t = 0; t < RG; ++t)
          if (jv && t0 + t < nr && rr[t] >= j) A[(size_t)rr[t] * ws_ld + j] = x[t];
      }
    }
    __syncwarp(ln.gm);
  }
  const double logdetC = log(pm) + (double)pe * 0.6931471805599453;
  // v = C^-1 h = -A h (entry (i, j) of the symmetric A from the lower triangle; lanes over rows;
  // BIG: four partial sums)
#pragma unroll 1
  for (int i = ln.sl; i < N; i += L) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    auto a_ij = [&](int j) { return *(j < i ? A + (size_t)i * ws_ld + j : A + (size_t)j * ws_ld + i); };
    int j = 0;
#pragma unroll 1
    for (; BIG && j + 3 < N; j += 4) {
      s0 = fma(a_ij(j), h[j], s0);
      s1 = fma(a_ij(j + 1), h[j + 1], s1);
      s2 = fma(a_ij(j + 2), h[j + 2], s2);
      s3 = fma(a_ij(j + 3), h[j + 3], s3);
    }
#pragma unroll 1
    for (; j < N; ++j) s0 = fma(a_ij(j), h[j], s0);
    rowk[i] = -((s0 + s1) + (s2 + s3));
  }
  __syncwarp(ln.gm);
  double hv = 0.0;
#pragma unroll 1
  for (int i = ln.sl; i < N; i += L) hv += h[i] * rowk[i];
  hv = wsum(hv, ln);
  // drift of the incremental state, then the refreshed state (packed lower triangle)
  double dmax = 0.0, amax = 0.0;
  constexpr int RD = BIG ? 4 : 1;  // entries per lane at a time, their loads ahead of their stores
  const int nt = tri(N);
#pragma unroll 1
  for (int e0 = ln.sl; e0 < nt; e0 += RD * L) {
    double nv[RD], ov[RD];
#pragma unroll
    for (int u = 0; u < RD; ++u) {
      const int e = e0 + u * L;
      nv[u] = ov[u] = 0.0;
      if (e < nt) {
        int i, j;
        untri(e, i, j);
        nv[u] = -A[(size_t)i * ws_ld + j];
        ov[u] = c64(Cp[e]);
      }
    }
#pragma unroll
    for (int u = 0; u < RD; ++u) {
      const int e = e0 + u * L;
      if (e < nt) {
        dmax = fmax(dmax, fabs(nv[u] - ov[u]));
        amax = fmax(amax, fabs(nv[u]));
        Cp[e] = cfrom64<C>(nv[u]);
      }
    }
  }
  double vd = 0.0, va = 0.0;
#pragma unroll 1
  for (int i = ln.sl; i < N; i += L) {
    vd = fmax(vd, fabs(rowk[i] - c64(W.v[i])));
    va = fmax(va, fabs(rowk[i]));
    W.v[i] = cfrom64<C>(rowk[i]);
  }
  dmax = wmax(dmax, ln); amax = wmax(amax, ln); vd = wmax(vd, ln); va = wmax(va, ln);
  __syncwarp(ln.gm);
  // sum_k log r_k
  double lrs = N * M.cm_lr[0];
  if (mix) {
    lrs = 0.0;
#pragma unroll 1
    for (int k = ln.sl; k < N; k += L) lrs += M.cm_lr[W.le[k]];
    lrs = wsum(lrs, ln);
  }
  out.ok = 1;
  out.drift = fmax(amax > 0.0 ? dmax / amax : 0.0, va > 0.0 ? vd / fmax(va, 1.0) : 0.0);
  out.logdet = n * M.log_se2 + logdetC - lrs;
  out.logL = -0.5 * (n * kLog2Pi + out.logdet + (yy - hv) / M.se2);
  return out;
}

// Scalars of an accepted move, from the proposal and its scoring.
template <typename C> struct PeMove {
  int jump, kk, jp, jm, np;
  int em, ep;  // charge components of the removed and the new PE
  C aa, quad, bv, vk, ay;
  Sup sp;
};

template <typename C> struct AcceptOut {
  C* Cp;
  int cap, N;
  unsigned long long words;
  C idl;  // 1 / delta, delta the Schur complement of the new PE (birth, update)
};

// Apply an accepted move to C^-1, v, y and the PE list (out of line: it runs on a minority of
// steps and keeps the per-step code compact). Returns the new N, and the new C^-1 storage when
// it moves from the shared tile (capacity cap PEs) to the global slot (n_cap PEs).
template <typename T, bool BIG, int L, bool MIX>
__device__ __noinline__ AcceptOut<typename PeTab<T>::C> pe_accept(const DevModel& M, const PeChain<T> W, const T* Vs,
                                                                  typename PeTab<T>::C* Cp, int cap,
                                                                  typename PeTab<T>::C* Cg,
                                                                  const PeMove<typename PeTab<T>::C> mv, int n, int N,
                                                                  const Lanes<L> ln) {
  // One form for the three moves. With c = row k of C^-1 (death, update), gamma = c_k, and
  // u' = C_-^-1 b~ (birth, update: C_- is C without PE k for an update, C itself for a birth;
  // b~ is b without its k entry), delta = r + |a_+|^2 - b~^T u':
  //   C'_ij = C_{m(i) m(j)} - c_m(i) c_m(j) / gamma + u'_i u'_j / delta   (i, j != s),
  //   C'_is = -u'_i / delta,  C'_ss = 1 / delta,
  // where s is the slot of the new PE (N for a birth, k for an update; none for a death) and
  // m moves the last PE into slot k for a death (identity otherwise). v changes the same way.
  // The removed PE has mean mu_- (component em), the new one mean mu_+ and r_+ (component ep).
  using C = typename PeTab<T>::C;
  const int em = MIX ? mv.em : 0, ep = MIX ? mv.ep : 0;
  const C mum = c_mu<C>(M, em), mup = c_mu<C>(M, ep), rrp = c_r<C>(M, ep);
  const T mumT = CmT<T>::mu(M, em), mupT = CmT<T>::mu(M, ep);
  const int R = M.R, np = mv.np, kk = mv.kk, jump = mv.jump;
  const bool has_m = jump != 0, has_p = jump != 1;
  const int skip = jump == 2 ? kk : -1;
  const int Nout = N + (jump == 0 ? 1 : (jump == 1 ? -1 : 0));
  const int s = jump == 0 ? N : (jump == 2 ? kk : -1);
  const int last = N - 1;
  // vectors: c (cv; zero for a birth) and C^-1 b~ (uv; zero for a death). The passes below
  // always apply both terms, so that they have no branches on the move type.
  const int krow = has_m ? kk : 0;
  const int npu = has_p ? np : 0;
  if constexpr (BIG) {
#pragma unroll 1
    for (int i = ln.sl; i < N; i += L) {
      const C ci = Cp[pk(krow, i)];
      W.cv[i] = has_m ? ci : czero<C>();
      W.uv[i] = dot_row<C, BIG>(Cp, i, W.ovi, W.ovb, npu, skip);
    }
  } else {
    // s lanes per row (s N <= L), each summing every s-th term of the row's product with b~,
    // then a butterfly over the s lanes: the dependent chain of a row is npu / s terms long
    int s = 1;
    while (s < 8 && 2 * s * N <= L) s <<= 1;
    const int rq = ln.sl / s, qq = ln.sl - rq * s, rpp = L / s;
#pragma unroll 1
    for (int i0 = 0; i0 < N; i0 += rpp) {
      const int i = i0 + rq;
      C acc = czero<C>();
      if (i < N) {
#pragma unroll 1
        for (int a = qq; a < npu; a += s)
          if (W.ovi[a] != skip) acc = cfma(Cp[pk(i, W.ovi[a])], W.ovb[a], acc);
      }
#pragma unroll 1
      for (int o = 1; o < s; o <<= 1) acc = cadd(acc, cshfl_xor<L>(acc, o, ln.gm));
      if (i < N && qq == 0) {
        W.cv[i] = has_m ? Cp[pk(krow, i)] : czero<C>();
        W.uv[i] = acc;
      }
    }
  }
  if (ln.sl == 0 && jump == 0) { W.cv[N] = czero<C>(); W.uv[N] = czero<C>(); }  // slot N of a birth (N < n_cap)
  __syncwarp(ln.gm);
  C ig = czero<C>(), idl = czero<C>(), t = czero<C>(), fv = czero<C>();
  if (has_m) {
    ig = crcp(W.cv[kk]);
    fv = cmul(cadd(mv.vk, mum), ig);
  }
  if (has_p) {
    // b^T v in full state precision (the scoring used an FP32 sum) and, for an update, the
    // entry of b for PE k, in one butterfly
    C bvf = czero<C>(), bk = czero<C>();
#pragma unroll 1
    for (int a = ln.sl; a < np; a += L) {
      bvf = cfma(W.ovb[a], W.v[W.ovi[a]], bvf);
      if (jump == 2 && W.ovi[a] == kk) bk = W.ovb[a];
    }
    const C wk = jump == 2 ? W.uv[kk] : czero<C>();  // read by every lane before the butterfly
    csum2(bvf, bk, ln);
    if (jump == 2) {
      // u' = w - c w_k / gamma on the system without PE k
      const C wkg = cneg(cmul(wk, ig));
#pragma unroll 1
      for (int i = ln.sl; i < N; i += L) W.uv[i] = (i == kk) ? czero<C>() : cfma(W.cv[i], wkg, W.uv[i]);
      __syncwarp(ln.gm);
    }
    C bu = czero<C>();
#pragma unroll 1
    for (int a = ln.sl; a < np; a += L)
      if (W.ovi[a] != skip) bu = cfma(W.ovb[a], W.uv[W.ovi[a]], bu);
    bu = csum(bu, ln);
    idl = crcp(csub(cadd(rrp, mv.aa), bu));
    // t = (b~^T v_- - mu_+ b~^T u' - h_new) / delta with v_- = v after removing PE k and h_new
    // the new PE's a^T y on the final residual (PE k removed, the new PE added)
    const C bvm = jump == 2 ? csub(csub(bvf, cmul(bk, mv.vk)), cmul(wk, fv)) : bvf;
    const C hnew = csub(cadd(mv.ay, cmul(mum, bk)), cmul(mup, mv.aa));
    t = cmul(csub(csub(bvm, cmul(mup, bu)), hnew), idl);
  }
  if (jump == 0 && N + 1 > cap && Cp != Cg) {  // the tile is full: move C^-1 to the global slot
#pragma unroll 1
    for (int e = ln.sl; e < tri(N); e += L) Cg[e] = Cp[e];
    Cp = Cg;
    cap = M.n_cap;
    __syncwarp(ln.gm);
  }
  // C^-1 in place over the packed triangle, all lanes on consecutive entries. A pass reads an
  // entry only where it writes it, or in the last row for a death (which it does not write).
  const C nig = cneg(ig);
  const int kmap = jump == 1 ? kk : -1;  // the slot the last PE moves into
  const int ne = tri(Nout);               // rows 0 .. Nout-1
  int e0 = 0;
  if constexpr (BIG) {
    // C^-1 in the global slot: four entries per lane and pass, all read before any is written
    // (each read is the entry itself or one in the unwritten last row), so that the loads of a
    // pass overlap
#pragma unroll 1
    for (; e0 + 4 * L <= ne; e0 += 4 * L) {
      int ii[4], jj[4];
      C old[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        untri(e0 + q * L + ln.sl, ii[q], jj[q]);
        const int mi = (ii[q] == kmap) ? last : ii[q], mj = (jj[q] == kmap) ? last : jj[q];
        old[q] = Cp[pk(mi, mj)];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = ii[q], j = jj[q];
        const int mi = (i == kmap) ? last : i, mj = (j == kmap) ? last : j;
        const C val = cfma(W.uv[i], cmul(W.uv[j], idl), cfma(W.cv[mi], cmul(W.cv[mj], nig), old[q]));
        const C sv = (i == s && j == s) ? idl : cneg(cmul(W.uv[i == s ? j : i], idl));
        Cp[e0 + q * L + ln.sl] = (i == s || j == s) ? sv : val;
      }
    }
  }
#pragma unroll 1
  for (int e = e0 + ln.sl; e < ne; e += L) {
    int i, j;
    untri(e, i, j);
    const int mi = (i == kmap) ? last : i, mj = (j == kmap) ? last : j;
    const C old = Cp[pk(mi, mj)];
    const C val = cfma(W.uv[i], cmul(W.uv[j], idl), cfma(W.cv[mi], cmul(W.cv[mj], nig), old));
    const C sv = (i == s && j == s) ? idl : cneg(cmul(W.uv[i == s ? j : i], idl));
    Cp[e] = (i == s || j == s) ? sv : val;
  }
  // v' = v_m - c_m fv + (t - mu_+) u', v'_s = -t
  const C tm = csub(t, mup), nfv = cneg(fv);
#pragma unroll 1
  for (int i = ln.sl; i < Nout; i += L) {
    const int mi = (i == kmap) ? last : i;
    const C val = cfma(tm, W.uv[i], cfma(W.cv[mi], nfv, W.v[mi]));
    W.v[i] = (i == s) ? cneg(t) : val;
  }
  // residual and PE list
  unsigned long long wds = (unsigned long long)N * np + 2ull * tri(Nout) + 2ull * Nout;
  if (has_m) {
    const Sup sm = pe_sup(M, n, mv.jm);
#pragma unroll 1
    for (int i = sm.ilo + ln.sl; i < sm.ihi; i += L) W.y[sm.w0 + i] += mumT * Vs[sm.ph + i * R];
    wds += 2 * (sm.ihi - sm.ilo) + N;
    __syncwarp(ln.gm);
  }
  if (has_p) {
    const Sup sp = mv.sp;
#pragma unroll 1
    for (int i = sp.ilo + ln.sl; i < sp.ihi; i += L) W.y[sp.w0 + i] -= mupT * Vs[sp.ph + i * R];
    wds += 2 * (sp.ihi - sp.ilo);
  }
  if (ln.sl == 0) {
    if (jump == 0) {
      W.list[N] = mv.jp;
      if constexpr (MIX) W.le[N] = (unsigned char)ep;
    } else if (jump == 1) {
      W.list[kk] = W.list[last];
      if constexpr (MIX) W.le[kk] = W.le[last];
    } else {
      W.list[kk] = mv.jp;
      if constexpr (MIX) W.le[kk] = (unsigned char)ep;
    }
  }
  __syncwarp(ln.gm);
  return AcceptOut<C>{Cp, cap, Nout, wds, idl};
}

// Random draws of the L steps from `step` on, lane l taking step + l (Philox4x64-10 keyed by
// (seed, waveform), counter (step, block, 0, 0); Box-Muller for the two shifts). Out of line:
// it runs once per L steps, and keeping it out of the step loop keeps the loop's code compact.
// FP32 mode takes cos(2 pi u) as cospif(2u), whose argument reduction is exact.
template <typename T, int L, bool MIX>
__device__ __noinline__ void pe_draw(const DevModel& M, PeRand<T>* rnd, uint64_t seed, uint64_t wf_id, int step,
                                     const Lanes<L> ln) {
  constexpr bool fp32 = sizeof(T) == 4;
  PeRand<T> rd;
  rd.ep = 0;
#pragma unroll 1
  for (int blk = 0; blk < (MIX ? 3 : 2); ++blk) {
    uint64_t c[4] = {(uint64_t)(step + ln.sl), (uint64_t)blk, 0, 0};
    philox4x64_10(c, seed, wf_id);
    if (blk == 2) {  // MCP component of a born or updated PE
      rd.ep = pe_draw_comp(M, u01_from_bits(c[0]));
    } else if constexpr (fp32) {
      const float a = u01_float(c[0]), b = u01_float(c[1]), d = u01_float(c[2]), e = u01_float(c[3]);
      if (blk == 0) {
        rd.z1 = (T)(sqrtf(-2.0f * logf(a)) * cospif(2.0f * b));
        rd.lu0 = (T)logf(d);
        rd.u3 = (T)e;
      } else {
        rd.u4 = (T)a;
        rd.z2 = (T)(sqrtf(-2.0f * logf(b)) * cospif(2.0f * d));
        rd.lu = (T)logf(e);
      }
    } else {
      const double a = u01_from_bits(c[0]), b = u01_from_bits(c[1]), d = u01_from_bits(c[2]), e = u01_from_bits(c[3]);
      if (blk == 0) {
        rd.z1 = (T)(sqrt(-2.0 * log(a)) * cos(kTwoPi * b));
        rd.lu0 = (T)log(d);
        rd.u3 = (T)e;
      } else {
        rd.u4 = (T)a;
        rd.z2 = (T)(sqrt(-2.0 * log(b)) * cos(kTwoPi * d));
        rd.lu = (T)log(e);
      }
    }
  }
  rnd[ln.sl] = rd;
  __syncwarp(ln.gm);
}

// Out-of-line pieces of the step that run only when the caller asked for them (a trace record,
// the PE-time histogram), so that their code stays out of the step loop's instruction stream.
__device__ __noinline__ void pe_trace_record(fsmp_trace* t, double la0, double lu0, double la, double lu, double dnu,
                                             int N, int k0, int jump, int flags) {
  fsmp_trace tr;
  tr.la0 = la0; tr.lu0 = lu0; tr.la = la; tr.lu = lu; tr.dnu = dnu;
  tr.N = N; tr.k0 = k0; tr.jump = jump; tr.flags = flags;
  *t = tr;
}
template <int L>
__device__ __noinline__ void pe_hist_add(uint32_t* peh, const int* list, int N, int T_lo, int width, const Lanes<L> ln) {
  for (int k = ln.sl; k < N; k += L) {
    const int c = list[k] - T_lo;
    if (c >= 0 && c < width) atomicAdd(peh + c, 1u);
  }
}

template <typename T, bool BIG, int L, bool MIX>
__global__ void __launch_bounds__(kPeMaxThreads, 4)
    pe_kernel(const __grid_constant__ DevModel M, const __grid_constant__ BatchView B, const __grid_constant__ PeSlots G) {
  using C = typename PeTab<T>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool fp32 = sizeof(T) == 4;
  const Lanes<L> ln = pe_lanes<L>();
  constexpr int kGroups = 32 / L;  // chains per warp
  const int cw = (threadIdx.x >> 5) * kGroups + ln.g, nchains = (blockDim.x >> 5) * kGroups;
  const int n_alloc = B.n_max, n_cap = M.n_cap, Ns = G.Ns;
  // block tables: the SER, log(i) and 1 / i, i = 1 .. n_cap + 1
  T* Vs = reinterpret_cast<T*>(smem_raw);
  T* lgN = reinterpret_cast<T*>(smem_raw + a16(sizeof(T) * M.Lt));
  double* inv1 = reinterpret_cast<double*>(smem_raw + a16(sizeof(T) * M.Lt) + a16(sizeof(T) * (n_cap + 2)));
  for (int m = threadIdx.x; m < M.Lt; m += blockDim.x) Vs[m] = PeTab<T>::V(M)[m];
  for (int i = threadIdx.x; i < n_cap + 2; i += blockDim.x) {
    lgN[i] = i > 0 ? (fp32 ? (T)logf((float)i) : (T)log((double)i)) : (T)0;
    inv1[i] = i > 0 ? 1.0 / (double)i : 0.0;
  }
  __syncthreads();
  PeChain<T> W = pe_carve<T, L>(smem_raw + pe_block_bytes<T>(M) +
                                    (size_t)cw * pe_chain_bytes<T, L>(n_cap, n_alloc, M.win_extra, Ns),
                                n_cap, n_alloc, M.win_extra, Ns);
  PeStats& S = *W.st;
  const size_t slot = (size_t)blockIdx.x * nchains + cw;
  int* const hist = G.hist + slot * (size_t)(n_cap + 1);
  C* const Cg = G.C ? reinterpret_cast<C*>(G.C) + slot * G.c_stride : nullptr;
  double* const ws = G.ws ? G.ws + slot * G.ws_stride : nullptr;
  const auto* __restrict__ tc = PeTab<T>::tc(M);
  const T ise2T = (T)M.inv_se2;
  constexpr bool mix = MIX;  // MCP charge mixture: per-PE components (else the one dynode model)
  const T Jt = (T)M.J, logJ = (T)M.log_J, inv_gT = (T)M.inv_g;
  const int R = M.R;

  for (;;) {
    int ci = 0;
    if (ln.sl == 0) ci = atomicAdd(G.counter, 1);
    ci = __shfl_sync(ln.gm, ci, 0, L);
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
    uint32_t* const peh = B.pe_hist ? B.pe_hist + (size_t)wi * B.pe_hist_width : nullptr;
    fsmp_trace* trace = B.trace ? B.trace + (B.trace_off ? B.trace_off[wi] : (int64_t)wi * n_steps) : nullptr;
    const bool invalid = n < 1 || n > n_alloc || T_hi <= T_lo || k0_hi < k0_lo || !(lambda0 > 0.0) || n_steps < 0 ||
                         burn_in < 0 || ((fp32 || B.z_init) && ws == nullptr) || k0_hi - k0_lo + 1 > M.win_extra ||
                         (Cg == nullptr && Ns < n_cap);
    if (invalid) {
      if (ln.sl == 0) {
        fsmp_summary o;
        o.mean_N = o.var_N = o.mean_t0 = o.var_t0 = o.mean_Q = o.var_Q = o.logL = o.logdet = NAN;
        o.drift_max = 0.0; o.alg_bytes = 0.0; o.lambda_hat = NAN;
        o.mean_wt = o.var_wt = o.mean_we = o.var_we = NAN;
        for (int k = 0; k < 3; ++k) { o.acc[k] = 0; o.prop[k] = 0; }
        o.acc_t0 = o.prop_t0 = o.N_final = o.k0_final = o.n_samples = o.n_refresh = o.reserved = 0;
        o.status = FSMP_ST_INVALID;
        *out = o;
        note_chain_done(B, wi);
      }
      __syncwarp(ln.gm);
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
    for (int k = ln.sl; k <= k0_hi - k0_lo; k += L) {
      const int kq = k0_lo + k;
      const double tot = pe_cphi<double>(M, T_hi - 1 - kq) - pe_cphi<double>(M, T_lo - 1 - kq);
      W.lPhi[k] = tot > 0.0 ? (fp32 ? (T)logf((float)(tot * M.g)) : (T)log(tot * M.g)) : (T)-INFINITY;
    }
#pragma unroll 1
    for (int k = ln.sl; k <= n_cap; k += L) hist[k] = 0;
    // empty z: y = w
    double wsq = 0.0;
    for (int x = ln.sl; x < n; x += L) {
      const float wx = w[x];
      W.y[x] = (T)wx;
      wsq += (double)wx * (double)wx;
    }
    wsq = wsum(wsq, ln);
    if (ln.sl == 0) {
      S.sN = S.sN2 = S.sK = S.sK2 = 0;
      S.sQ = S.sQ2 = 0.0; S.q_cur = 0.0; S.q_from = 0;
      S.St = S.Se = 0; S.wt_cur = S.we_cur = 0.0;
      S.sWt = S.sWt2 = S.sWe = S.sWe2 = 0.0;
      S.logdet = n * M.log_se2;
      S.logL = -0.5 * (n * kLog2Pi + S.logdet + wsq * M.inv_se2);
      S.wsq = wsq;
      S.drift_max = 0.0; S.alg_words = 0;
      for (int k = 0; k < 3; ++k) { S.acc[k] = 0; S.prop[k] = 0; }
      S.acc_t0 = S.prop_t0 = S.n_refresh = S.status = S.n_acc_refresh = S.refresh_fail = 0;
    }
    __syncwarp(ln.gm);
    const T log_lambda0 = fp32 ? (T)logf((float)lambda0) : (T)log(lambda0);
    C* Cp = Ns > 0 ? W.Cs : Cg;  // C^-1 (packed), room for cap PEs
    int cap = Ns > 0 ? Ns : n_cap;
    int N = 0;
    if (B.z_init) {
      // a given initial state (LucyDDM, Sec. 2.3): the PE list, each PE of the most probable
      // component, then C^-1, v, y, log|Sigma| and log L from it by the FP64 rebuild
      int ni = min(B.n_init[wi], B.z_stride);
      const bool cut = ni > n_cap;
      if (cut) ni = n_cap;
      for (int k = ln.sl; k < ni; k += L) {
        W.list[k] = B.z_init[(size_t)wi * B.z_stride + k];
        if constexpr (MIX) W.le[k] = (unsigned char)M.cm_mode;
      }
      __syncwarp(ln.gm);
      if (ni > cap) { Cp = Cg; cap = n_cap; }
      if (ni > 0) {
        bool ok = true;
        double ms = 0.0;
        C qs = czero<C>();
        if constexpr (fp32) {
          // FP32 mode: the FP64 rebuild
          const RefreshOut ro = pe_refresh<T, BIG, L, MIX>(M, W, Cp, ws, n_cap, w, S.wsq, n, ni, ln);
          ok = ro.ok != 0;
          if (ok && ln.sl == 0) { S.logdet = ro.logdet; S.logL = ro.logL; }
        } else {
          // FP64 mode: the PEs born one by one through the accepted-move update in double-double
          // (the FP64 rebuild would leave C^-1 only as accurate as FP64 times its condition
          // number); log|C| is the sum of the log Schur complements
          double lC = 0.0;
#pragma unroll 1
          for (int k = 0; k < ni; ++k) {
            PeMove<C> mv;
            mv.jump = 0; mv.kk = -1; mv.jp = W.list[k]; mv.jm = -1;
            mv.em = mv.ep = MIX ? M.cm_mode : 0;
            const Sup sp = pe_sup(M, n, mv.jp);
            mv.sp = sp;
            int np = 0;
#pragma unroll 1
            for (int base = 0; base < N; base += L) {
              const int qi = base + ln.sl;
              C bq = czero<C>();
              if (qi < N) {
                const int o = mv.jp - W.list[qi];
                if (o > -M.Lt && o < M.Lt) bq = xcorr<C>(M, tc, sp, o);
              }
              const bool ov = cnz(bq);
              const unsigned m = gballot(ov, ln);
              if (ov) {
                const int pos = np + __popc(m & ((1u << ln.sl) - 1u));
                W.ovi[pos] = qi;
                W.ovb[pos] = bq;
              }
              np += __popc(m);
            }
            __syncwarp(ln.gm);
            mv.np = np;
            mv.aa = xcorr<C>(M, tc, sp, 0);
            T ayp = (T)0;
            for (int i = sp.ilo + ln.sl; i < sp.ihi; i += L) ayp += Vs[sp.ph + i * R] * W.y[sp.w0 + i];
            mv.ay = cfromf(wsum(ayp, ln));
            mv.quad = mv.bv = mv.vk = czero<C>();
            const AcceptOut<C> ao = pe_accept<T, BIG, L, MIX>(M, W, Vs, Cp, cap, Cg, mv, n, N, ln);
            Cp = ao.Cp;
            cap = ao.cap;
            N = ao.N;
            const double dl = c64(ao.idl);
            if (!(dl > 0.0) || !isfinite(dl)) ok = false;
            lC -= log(dl);
          }
          N = 0;
          // log|Sigma| = n log se2 + log|C| - sum_k log r_k; y^T Sigma^-1 y = (y^T y - h^T v) / se2
          double lr = 0.0, yy = 0.0, hv = 0.0;
          for (int k = ln.sl; k < ni; k += L) {
            lr += M.cm_lr[MIX ? M.cm_mode : 0];
            const Sup s = pe_sup(M, n, W.list[k]);
            double hk = 0.0;
            for (int i = s.ilo; i < s.ihi; ++i) hk = fma((double)Vs[s.ph + i * R], (double)W.y[s.w0 + i], hk);
            hv = fma(hk, c64(W.v[k]), hv);
          }
          for (int x = ln.sl; x < n; x += L) yy = fma((double)W.y[x], (double)W.y[x], yy);
          lr = wsum(lr, ln); yy = wsum(yy, ln); hv = wsum(hv, ln);
          if (ok && ln.sl == 0) {
            S.logdet = n * M.log_se2 + lC - lr;
            S.logL = -0.5 * (n * kLog2Pi + S.logdet + (yy - hv) * M.inv_se2);
          }
        }
        for (int i = ln.sl; i < ni; i += L) {
          qs = cadd(qs, W.v[i]);
          if (mix) ms += M.cm_mu[W.le[i]];
        }
        qs = csum(qs, ln);
        ms = mix ? wsum(ms, ln) : ni * M.cm_mu[0];
        if (ok) {
          N = ni;
        } else {  // C not numerically positive definite: start empty
          for (int x = ln.sl; x < n; x += L) W.y[x] = (T)w[x];
          Cp = Ns > 0 ? W.Cs : Cg;
          cap = Ns > 0 ? Ns : n_cap;
        }
        long long st = 0;
        for (int k = ln.sl; k < ni; k += L) st += abs(W.list[k]);
        st = wsum(st, ln);
        if (ln.sl == 0) {
          if (ok) {
            S.q_cur = ms + c64(qs);
            S.St = st;
            S.Se = MIX ? (long long)ni * M.cm_mode : 0;
            set_wasserstein(S, M.g, ni, inv1);
          } else {
            S.status |= FSMP_ST_BADDET;
          }
        }
      }
      if (ln.sl == 0 && cut) S.status |= FSMP_ST_CAPACITY;
      __syncwarp(ln.gm);
    }

    for (int step = 0; step < n_steps; ++step) {
      // ---- random draws of the next L steps: lane l takes step step + l
      if ((step & (L - 1)) == 0) pe_draw<T, L, MIX>(M, W.rnd, seed, wf_id, step, ln);
      const PeRand<T> rd = W.rnd[step & (L - 1)];
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
#pragma unroll 1
          for (int k = ln.sl; k < N; k += L) {
            const int j = W.list[k];
            part += pe_logphi<T>(M, j - k0p) - pe_logphi<T>(M, j - k0);
          }
          la0 = wsum(part, ln);
        }
        if (lu0 < la0) { k0 = k0p; t0f |= 2; }
      }
      // ---- Gibbs part 2: one RJMCMC jump (Sec. 2.4)
      const int jump = (N == 0) ? 0 : (rd.u3 < Jt ? 0 : (rd.u3 < (T)2 * Jt ? 1 : 2));
      int valid = 0, noop = 0, kk = -1, jp = -1, jm = -1, e_m = MIX ? rd.ep : 0;
      T la_prior = (T)0, la_fixed = (T)-INFINITY;
      const T lu = rd.lu;
      const T lphi_t0 = W.lPhi[k0 - k0_lo];
      if (jump == 0) {
        if (N >= n_cap) {
          st_a |= FSMP_ST_CAPACITY;
        } else if (lphi_t0 > (T)-INFINITY) {
          const T base = pe_cphi<T>(M, T_lo - 1 - k0), tot = pe_cphi<T>(M, T_hi - 1 - k0) - base;
          jp = pe_birth_search<T, L>(M, T_lo, T_hi, k0, base, rd.u4 * tot, ln);
          valid = jp >= T_lo;
          la_prior = log_lambda0 + lphi_t0 - lgN[N + 1] + (N == 0 ? logJ : (T)0);
        }
      } else {
        kk = fp32 ? __float2int_rd((float)(rd.u4 * (T)N)) : __double2int_rd((double)(rd.u4 * (T)N));
        if (kk >= N) kk = N - 1;
        jm = W.list[kk];
        if constexpr (MIX) e_m = W.le[kk];
        if (jump == 1) {
          valid = 1;
          la_prior = -log_lambda0 - lphi_t0 + lgN[N] - (N == 1 ? logJ : (T)0);
        } else {
          const int Dm = fp32 ? __float2int_rn((float)(rd.z2 * inv_gT)) : __double2int_rn((double)(rd.z2 * inv_gT));
          const int jpl = jm + Dm;
          if (Dm == 0 && (!MIX || rd.ep == e_m)) {  // same time and component: an accepted no-op
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
      // ---- scoring: the 2x2 quantities in PE space, then the 2x2 algebra in T
      PeMove<C> mv;
      mv.jump = jump; mv.kk = kk; mv.jp = jp; mv.jm = jm; mv.np = 0;
      // components of a_- and a_+; the absent one of a birth or death takes the other's values
      // (its terms vanish)
      mv.em = e_m;
      mv.ep = MIX ? (jump == 1 ? e_m : rd.ep) : 0;
      mv.aa = mv.quad = mv.bv = mv.vk = mv.ay = czero<C>();
      mv.sp = Sup{0, 0, 0, 0};
      T mmm = 0, mmp = 0, mpp = 0, gm = 0, gp = 0, em = 1;
      unsigned long long words = 0;
      if (valid) {
        if (jump != 1) {
          const Sup sp = pe_sup(M, n, jp);
          mv.sp = sp;
          mv.aa = xcorr<C>(M, tc, sp, 0);  // issued first: its table load overlaps the scan's
          // PEs overlapping a_+, with b_q = a_q^T a_+
          int np = 0;
#pragma unroll 1
          for (int base = 0; base < N; base += L) {
            const int qi = base + ln.sl;
            C bq = czero<C>();
            if (qi < N) {
              const int o = jp - W.list[qi];
              if (o > -M.Lt && o < M.Lt) bq = xcorr<C>(M, tc, sp, o);
            }
            const bool ov = cnz(bq);
            const unsigned m = gballot(ov, ln);
            if (ov) {
              const int pos = np + __popc(m & ((1u << ln.sl) - 1u));
              W.ovi[pos] = qi;
              W.ovb[pos] = bq;
            }
            np += __popc(m);
          }
          __syncwarp(ln.gm);
          mv.np = np;
          // b^T C^-1 b over the lower triangle of the overlap block (lanes over its entries, the
          // off-diagonal ones counted twice), b^T v, (C^-1 b)_k of an update and a_+^T y, then one
          // reduction of the four over the group
          T ayp = (T)0;
#pragma unroll 1
          for (int i = sp.ilo + ln.sl; i < sp.ihi; i += L) ayp += Vs[sp.ph + i * R] * W.y[sp.w0 + i];
          C qp = czero<C>(), ck = czero<C>();
          T bvp = (T)0;
          const int nt = tri(np);
          int e = ln.sl;
          if constexpr (BIG) {  // C^-1 in the global slot: four entries' loads ahead of their sums
#pragma unroll 1
            for (; e + 3 * L < nt; e += 4 * L) {
              C cq[4], bb[4];
              bool dg[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                int a, b2;
                untri(e + u * L, a, b2);
                cq[u] = Cp[pk(W.ovi[a], W.ovi[b2])];
                bb[u] = cmul(W.ovb[a], W.ovb[b2]);
                dg[u] = a == b2;
              }
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const C t = cmul(cq[u], bb[u]);
                qp = cadd(qp, dg[u] ? t : ctwice(t));
              }
            }
          }
#pragma unroll 1
          for (; e < nt; e += L) {
            int a, b2;
            untri(e, a, b2);
            const C t = cmul(Cp[pk(W.ovi[a], W.ovi[b2])], cmul(W.ovb[a], W.ovb[b2]));
            qp = cadd(qp, a == b2 ? t : ctwice(t));
          }
#pragma unroll 1
          for (int a = ln.sl; a < np; a += L) {
            const C ba = W.ovb[a];
            bvp += (T)cnum(ba) * (T)cnum(W.v[W.ovi[a]]);
            if (jump == 2) ck = cfma(Cp[pk(kk, W.ovi[a])], ba, ck);
          }
          gsum4<L>(qp, ck, bvp, ayp, ln);
          mv.quad = qp;
          const T bvT = bvp;  // b^T v at the scoring precision (the accept recomputes it)
          const T ayT = ayp;
          mv.ay = cfromf(ayT);
          mpp = (T)cnum(csub(mv.aa, mv.quad)) * ise2T;
          gp = (ayT - bvT) * ise2T;
          mmp = (T)cnum(ck);  // times 1 / sigma_-^2 below (update only)
          words += (unsigned long long)(N + 2 * np + 2 * (sp.ihi - sp.ilo) + np * np + np);
        }
        if (jump != 0) {
          const T iqm = CmT<T>::iq(M, mv.em);
          mv.vk = W.v[kk];
          em = CmT<T>::r(M, mv.em) * (T)cnum(Cp[tri(kk) + kk]);
          mmm = ((T)1 - em) * iqm;
          gm = (T)cnum(mv.vk) * iqm;
          mmp *= iqm;
          words += 2;
        }
      }
      T la = la_fixed, dnu = (T)NAN, dT = (T)0;
      int st_c = 0;
      if (valid) {
        // det(I + Lambda M), Lambda = diag(-q_-, q_+) (q = sigma_e^2 of the PE concerned), with
        // 1 - q_- m_-- = em; lambda = (-mu_-, mu_+) (Eq. (DeltaU), Appendix A.2)
        const T qm = CmT<T>::q(M, mv.em), qp = CmT<T>::q(M, mv.ep);
        const T mum = CmT<T>::mu(M, mv.em), mup = CmT<T>::mu(M, mv.ep);
        const T Dd = em * ((T)1 + qp * mpp) + qm * qp * mmp * mmp;
        if (!(Dd > (T)0)) {
          la = (T)-INFINITY;
          st_c |= FSMP_ST_BADDET;
        } else {
          const T iD = (T)1 / Dd;
          const T B11 = -qm * ((T)1 + qp * mpp) * iD, B12 = qm * qp * mmp * iD, B22 = qp * em * iD;
          // rho = g - M lambda; dR = -2 lambda^T g + lambda^T M lambda - rho^T B rho
          const T rm = gm + mum * mmm - mup * mmp, rp = gp + mum * mmp - mup * mpp;
          const T dR = (T)-2 * (mup * gp - mum * gm) + (mum * mum * mmm - (T)2 * mum * mup * mmp + mup * mup * mpp) -
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
        {
          const AcceptOut<C> ao = pe_accept<T, BIG, L, MIX>(M, W, Vs, Cp, cap, Cg, mv, n, N, ln);
          Cp = ao.Cp;
          cap = ao.cap;
          N = ao.N;
          words += ao.words;
        }
        C qs = czero<C>();
        double ms = 0.0;  // sum of the PEs' means (the mixture; N mu_q for the dynode model)
        for (int i = ln.sl; i < N; i += L) {
          qs = cadd(qs, W.v[i]);
          if (mix) ms += M.cm_mu[W.le[i]];
        }
        qs = csum(qs, ln);
        ms = mix ? wsum(ms, ln) : N * M.cm_mu[0];
        if (ln.sl == 0) {
          close_hold(S, step, burn_in);
          S.q_cur = ms + c64(qs);
          S.q_from = step;
          // the PE removed (death, update) and the one added (birth, update)
          if (jump != 1) { S.St += abs(mv.jp); S.Se += mv.ep; }
          if (jump != 0) { S.St -= abs(mv.jm); S.Se -= mv.em; }
          set_wasserstein(S, M.g, N, inv1);
          S.logdet += (double)dT;
          S.logL += (double)dnu;
          S.n_acc_refresh++;
        }
        __syncwarp(ln.gm);
        if (fp32 && M.refresh_every > 0 && S.n_acc_refresh >= M.refresh_every) {
          const RefreshOut ro = pe_refresh<T, BIG, L, MIX>(M, W, Cp, ws, n_cap, w, S.wsq, n, N, ln);
          C qr = czero<C>();
          for (int i = ln.sl; i < N; i += L) qr = cadd(qr, W.v[i]);
          qr = csum(qr, ln);
          if (ln.sl == 0) {
            S.n_acc_refresh = 0;
            if (ro.ok) {
              S.logdet = ro.logdet; S.logL = ro.logL;
              S.drift_max = fmax(S.drift_max, ro.drift);
              if (ro.drift > M.drift_tol) S.status |= FSMP_ST_DRIFT;
              S.n_refresh++;
              S.q_cur = ms + c64(qr);
            } else {
              S.status |= FSMP_ST_DRIFT;
              S.refresh_fail++;
            }
          }
          __syncwarp(ln.gm);
        }
      }

      // ---- bookkeeping of the decided step (the group's first lane)
      if (ln.sl == 0) {
        S.prop[jump]++;
        if (t0f & 1) { S.prop_t0++; if (t0f & 2) S.acc_t0++; }
        if (apply) S.acc[jump]++;
        S.status |= st_a | st_c;
        S.alg_words += words;
        if (step >= burn_in) {
          const long long Nn = N, kq = k0;
          S.sN += Nn; S.sN2 += Nn * Nn; S.sK += kq; S.sK2 += kq * kq;
          atomicAdd(hist + N, 1);  // no value returned: the lane does not wait on it
        }
        if (trace) pe_trace_record(trace + step, (double)la0, (double)lu0, (double)la, (double)lu, (double)dnu, N, k0, jump,
                                   t0f | (acc ? 4 : 0) | ((acc && noop) ? 8 : 0));
      }
      if (peh && step >= burn_in) pe_hist_add<L>(peh, W.list, N, T_lo, B.pe_hist_width, ln);
      __syncwarp(ln.gm);
    }

    // ------------------------------------------------------------- chain end
    if (fp32 && M.refresh_every > 0 && S.n_acc_refresh > 0) {
      // the reported log-likelihood and log|Sigma| come from an FP64 rebuild
      const RefreshOut ro = pe_refresh<T, BIG, L, MIX>(M, W, Cp, ws, n_cap, w, S.wsq, n, N, ln);
      if (ln.sl == 0) {
        if (ro.ok) {
          S.logdet = ro.logdet; S.logL = ro.logL;
          S.drift_max = fmax(S.drift_max, ro.drift);
          if (ro.drift > M.drift_tol) S.status |= FSMP_ST_DRIFT;
          S.n_refresh++;
        } else {
          S.status |= FSMP_ST_DRIFT;
        }
      }
    }
    const double lam_hat = pe_lambda_mle<L>(hist, n_cap, lambda0, ln.sl, ln.gm);
    if (ln.sl == 0) {
      close_hold(S, n_steps, burn_in);
      fsmp_summary o;
      o.lambda_hat = lam_hat;
      int ns = n_steps - burn_in;
      if (ns < 0) ns = 0;
      const double inv = ns > 0 ? 1.0 / ns : NAN;
      const double mN = (double)S.sN * inv, mK = (double)S.sK * inv;
      o.mean_N = mN; o.var_N = (double)S.sN2 * inv - mN * mN;
      o.mean_t0 = t_origin + M.g * mK; o.var_t0 = M.g * M.g * ((double)S.sK2 * inv - mK * mK);
      o.mean_Q = S.sQ * inv; o.var_Q = S.sQ2 * inv - o.mean_Q * o.mean_Q;
      o.mean_wt = S.sWt * inv; o.var_wt = S.sWt2 * inv - o.mean_wt * o.mean_wt;
      o.mean_we = S.sWe * inv; o.var_we = S.sWe2 * inv - o.mean_we * o.mean_we;
      o.logL = S.logL; o.logdet = S.logdet;
      o.drift_max = S.drift_max; o.alg_bytes = (double)S.alg_words * 8.0;
      for (int k = 0; k < 3; ++k) { o.acc[k] = S.acc[k]; o.prop[k] = S.prop[k]; }
      o.acc_t0 = S.acc_t0; o.prop_t0 = S.prop_t0; o.N_final = N; o.k0_final = k0;
      o.status = S.status; o.n_samples = ns; o.n_refresh = S.n_refresh; o.reserved = 0;
      *out = o;
      note_chain_done(B, wi);
    }
    __syncwarp(ln.gm);
  }
}

// Float-float copy of an FP64 table: hi = fl(x), lo = fl(x - hi).
__global__ void split_ff_kernel(const double* a, float* out, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float h = (float)a[i];
  out[2 * i] = h;
  out[2 * i + 1] = (float)(a[i] - (double)h);
}


// The kernel instance for (precision, BIG, lanes) of a charge model; f receives its address.
// The mixture has no BIG instance (its chains use the compact loops at any n_cap).
template <bool MIX, typename F> cudaError_t with_pe_kernel(int precision, bool big, int lanes, F f) {
  if constexpr (MIX) {
    if (precision == FSMP_FP64)
      return lanes == 16 ? f(pe_kernel<double, false, 16, true>) : f(pe_kernel<double, false, 32, true>);
    return lanes == 16 ? f(pe_kernel<float, false, 16, true>) : f(pe_kernel<float, false, 32, true>);
  } else {
    if (precision == FSMP_FP64) {
      if (big) return f(pe_kernel<double, true, 32, false>);
      return lanes == 16 ? f(pe_kernel<double, false, 16, false>) : f(pe_kernel<double, false, 32, false>);
    }
    if (big) return f(pe_kernel<float, true, 32, false>);
    return lanes == 16 ? f(pe_kernel<float, false, 16, false>) : f(pe_kernel<float, false, 32, false>);
  }
}

template <bool MIX> cudaError_t pe_set_attributes(int precision, int max_smem) {
  for (int big = 0; big < (MIX ? 1 : 2); ++big)
    for (int lanes : {32, 16}) {
      if (big && lanes == 16) continue;
      const cudaError_t e = with_pe_kernel<MIX>(precision, big != 0, lanes, [&](auto k) {
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
      });
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

template <bool MIX> int pe_occupancy(int precision, int threads, size_t smem, bool big, int lanes) {
  int n = 0;
  const cudaError_t e = with_pe_kernel<MIX>(precision, big, lanes, [&](auto k) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem);
  });
  return e == cudaSuccess ? n : 0;
}

template <bool MIX>
cudaError_t pe_launch(const DevModel& M, const BatchView& B, int warps, int lanes, int ctas, int Ns, size_t smem,
                      void* cinv, size_t c_stride, double* ws, size_t ws_stride, int* hist, int* counter,
                      bool big, cudaStream_t st) {
  PeSlots G;
  G.C = cinv;
  G.c_stride = c_stride;
  G.ws = ws;
  G.ws_stride = ws_stride;
  G.hist = hist;
  G.counter = counter;
  G.Ns = Ns;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  e = with_pe_kernel<MIX>(M.precision, big, lanes, [&](auto k) {
    k<<<ctas, warps * 32, smem, st>>>(M, B, G);
    return cudaSuccess;
  });
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace
}  // namespace fsmp
