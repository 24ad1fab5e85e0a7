// ROWS_TMA-variant launcher for float values (see rows_tma.cuh).
#include "launch_impl.cuh"

namespace gbs {
cudaError_t launch_rows_tma_f32(const CsrView& A, const DenseView& D, int lanes, bool vec16, int threads, int tile,
                               int emul, int* status, cudaStream_t s) {
  return launch_rows_tma_t<float>(A, D, lanes, vec16, threads, tile, emul, status, s);
}
}  // namespace gbs
