// fsmp_pe_mix.cu -- the PE-space chain kernel for the MCP charge mixture (Eq. (mcp-multi-norm),
// Eq. (mcp), Appendix A.2): every PE carries its component, e+ ~ G is drawn for every birth and
// update. Its own translation unit, so that these instances compile beside the dynode ones.
#include "fsmp_pe_kernel.cuh"

namespace fsmp {

cudaError_t pe_mix_attributes(int precision, int max_smem) { return pe_set_attributes<true>(precision, max_smem); }

int pe_mix_occupancy(int precision, int threads, size_t smem, int lanes) {
  return pe_occupancy<true>(precision, threads, smem, false, lanes);
}

cudaError_t pe_mix_launch(const DevModel& M, const BatchView& B, int warps, int lanes, int ctas, int Ns, size_t smem,
                          void* cinv, size_t c_stride, double* ws, size_t ws_stride, int* hist, int* counter,
                          cudaStream_t st) {
  return pe_launch<true>(M, B, warps, lanes, ctas, Ns, smem, cinv, c_stride, ws, ws_stride, hist, counter, false, st);
}

}  // namespace fsmp
