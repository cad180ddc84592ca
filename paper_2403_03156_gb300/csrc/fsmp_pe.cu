// fsmp_pe.cu -- host side of the PE-space chain kernel (arXiv 2403.03156, Sec. 2.4 and Appendix
// A.1) and its dynode-model instances; the kernel itself is in fsmp_pe_kernel.cuh.
#include "fsmp_pe_kernel.cuh"

namespace fsmp {

size_t pe_smem_bytes(const DevModel& M, int n_alloc, int warps, int lanes, int Ns) {
  const int chains = warps * (32 / lanes);
  const bool l16 = lanes == 16;
  if (M.precision == FSMP_FP64)
    return pe_block_bytes<double>(M) +
           (size_t)chains * (l16 ? pe_chain_bytes<double, 16>(M.n_cap, n_alloc, M.win_extra, Ns)
                                 : pe_chain_bytes<double, 32>(M.n_cap, n_alloc, M.win_extra, Ns));
  return pe_block_bytes<float>(M) +
         (size_t)chains * (l16 ? pe_chain_bytes<float, 16>(M.n_cap, n_alloc, M.win_extra, Ns)
                               : pe_chain_bytes<float, 32>(M.n_cap, n_alloc, M.win_extra, Ns));
}

size_t pe_ws_slot_doubles(int n_cap) { return pe_ws_doubles(n_cap); }

size_t pe_c_entries(int n_cap) { return (size_t)tri(n_cap); }

size_t pe_c_entry_bytes(int precision) {
  return precision == FSMP_FP64 ? sizeof(PeTab<double>::C) : sizeof(PeTab<float>::C);
}

cudaError_t launch_split_ff(const double* a, float* out, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  split_ff_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, out, n);
  return cudaGetLastError();
}

// The pile-up variant (BIG) unrolls the gathers and row passes over C^-1 four ways so that
// their loads overlap; it pays off when chains carry many PEs (C^-1 in global memory) and costs
// registers otherwise.
bool pe_big(int n_cap) { return n_cap > 192; }

// Lanes per chain the kernel is built for: 32, and 16 where chains are small (not BIG).
bool pe_lanes_ok(int lanes, int n_cap) { return lanes == 32 || (lanes == 16 && !pe_big(n_cap)); }


cudaError_t pe_kernel_attributes(int precision, int max_smem) {
  const cudaError_t e = pe_set_attributes<false>(precision, max_smem);
  return e != cudaSuccess ? e : pe_mix_attributes(precision, max_smem);
}

int pe_kernel_occupancy(int precision, int threads, size_t smem, bool big, int lanes, bool mix) {
  if (mix) return pe_mix_occupancy(precision, threads, smem, lanes);
  return pe_occupancy<false>(precision, threads, smem, big, lanes);
}

// lambda_FSMP of given N histograms (testing aid): the device function every chain ends with,
// one histogram per group of L lanes. Histogram i is h[i * (n_max + 1) .. (i + 1) * (n_max + 1)).
template <int L>
__global__ void lambda_mle_kernel(const int* __restrict__ h, int n_hist, int n_max, const double* __restrict__ lambda0,
                                  double* __restrict__ out) {
  const Lanes<L> ln = pe_lanes<L>();
  const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) / L);
  if (i >= n_hist) return;  // i is the same on every lane of a group
  const double lam = group_lambda_mle<L>(h + (size_t)i * (n_max + 1), n_max, lambda0[i], ln.sl, ln.gm);
  if (ln.sl == 0) out[i] = lam;
}

cudaError_t launch_lambda_mle(const int* h, int n_hist, int n_max, const double* lambda0, double* out, int lanes,
                              cudaStream_t st) {
  if (n_hist <= 0) return cudaSuccess;
  const int threads = 128, per_block = threads / lanes;
  const unsigned blocks = (unsigned)((n_hist + per_block - 1) / per_block);
  if (lanes == 16) lambda_mle_kernel<16><<<blocks, threads, 0, st>>>(h, n_hist, n_max, lambda0, out);
  else lambda_mle_kernel<32><<<blocks, threads, 0, st>>>(h, n_hist, n_max, lambda0, out);
  return cudaGetLastError();
}

cudaError_t launch_pe(const DevModel& M, const BatchView& B, int warps, int lanes, int ctas, int Ns, size_t smem,
                      void* cinv, size_t c_stride, double* ws, size_t ws_stride, int* hist, int* counter,
                      cudaStream_t st) {
  if (hist == nullptr || !pe_lanes_ok(lanes, M.n_cap)) return cudaErrorInvalidValue;
  if (M.n_comp > 1)
    return pe_mix_launch(M, B, warps, lanes, ctas, Ns, smem, cinv, c_stride, ws, ws_stride, hist, counter, st);
  return pe_launch<false>(M, B, warps, lanes, ctas, Ns, smem, cinv, c_stride, ws, ws_stride, hist, counter,
                          pe_big(M.n_cap), st);
}

}  // namespace fsmp
