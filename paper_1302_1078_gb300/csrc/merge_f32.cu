// MERGE-variant launcher for float values (see merge_kernel.cuh).
#include "launch_impl.cuh"

namespace gbs {
cudaError_t launch_merge_f32(const CsrView& A, const DenseView& D, int g, bool vec16, bool direct, int threads,
                            int items, const MergeScratch& S, cudaStream_t s) {
  return launch_merge_t<float>(A, D, g, vec16, direct, threads, items, S, s);
}
}  // namespace gbs
