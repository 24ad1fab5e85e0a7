// ROWS and ROWS_DIRECT launchers for double values (see rows_kernel.cuh).
#include "launch_impl.cuh"

namespace gbs {
cudaError_t launch_rows_f64(const CsrView& A, const DenseView& D, int lanes, bool vec16, int threads, int tile,
                           int row_base, int rows, cudaStream_t s) {
  return launch_rows_t<double>(A, D, lanes, vec16, threads, tile, row_base, rows, s);
}
cudaError_t launch_rows_direct_f64(const CsrView& A, const DenseView& D, int lanes, bool vec16, int threads,
                                  cudaStream_t s) {
  return launch_rows_direct_t<double>(A, D, lanes, vec16, threads, s);
}
}  // namespace gbs
