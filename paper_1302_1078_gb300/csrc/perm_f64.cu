// ROWS and MERGE_DIRECT launchers for double values read through a permutation
// (the backward pass's A^T product on A's values; see rows_kernel.cuh).
#include "launch_impl.cuh"

namespace gbs {
cudaError_t launch_rows_perm_f64(const CsrView& A, const DenseView& D, int lanes, bool vec16, int threads, int tile,
                                 int row_base, int rows, cudaStream_t s) {
  return launch_rows_t<double, true>(A, D, lanes, vec16, threads, tile, row_base, rows, s);
}
cudaError_t launch_merge_perm_f64(const CsrView& A, const DenseView& D, int g, bool vec16, bool direct, int threads,
                                  int items, const MergeScratch& S, cudaStream_t s) {
  return launch_merge_t<double, true>(A, D, g, vec16, direct, threads, items, S, s);
}
}  // namespace gbs
