// Backward pass of Y = A X with respect to the stored values (the paper has
// no backward pass): the sampled dense-dense product over A's pattern
//   dvals[p] = sum_c dY[row(p), c] * X[col_idx[p], c].
// One thread per nonzero sums its k products in column order, so no FP64
// reduction across lanes is needed (on GB300 every FP64 instruction counts);
// consecutive threads hold consecutive nonzeros, so their dY rows are mostly
// the same row (served by L1) and their col_idx/row reads are coalesced.
// The X rows are gathered with the L2 evict-last policy, like SpMM.
#include <algorithm>
#include <cstdint>

#include "device_common.cuh"
#include "gbspmv.h"
#include "launch.h"

namespace gbs {

template <typename T, int VEC>
__global__ void __launch_bounds__(256) sddmm_kernel(int nnz, int k, const int* __restrict__ rows,
                                                    const int* __restrict__ col_idx, const T* __restrict__ X,
                                                    long long ldx, const T* __restrict__ dY, long long lddy,
                                                    T* __restrict__ dvals) {
  const uint64_t pol_keep = policy_evict_last();
  const uint64_t pol_stream = policy_evict_first();
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (long long)gridDim.x * blockDim.x) {
    const int i = ld_stream(rows + p, pol_stream);
    const int j = ld_stream(col_idx + p, pol_stream);
    const T* __restrict__ xr = X + (long long)j * ldx;
    const T* __restrict__ yr = dY + (long long)i * lddy;
    Acc<T> acc;
    int c = 0;
    if constexpr (VEC > 1) {
      for (; c + VEC <= k; c += VEC) {
        Vec<T, VEC> xv = ld_keep_vec<T, VEC>(xr + c, pol_keep);
        Vec<T, VEC> yv = ld_keep_vec<T, VEC>(yr + c, pol_keep);
#pragma unroll
        for (int q = 0; q < VEC; ++q) acc.add(yv.v[q], xv.v[q]);
      }
    }
    for (; c < k; ++c) acc.add(ld_keep(yr + c, pol_keep), ld_keep(xr + c, pol_keep));
    st_stream(dvals + p, acc.value());
  }
}

template <typename T>
static cudaError_t sddmm_t(int nnz, int k, const int* rows, const int* col_idx, const void* X, long long ldx,
                           const void* dY, long long lddy, void* dvals, cudaStream_t s) {
  if (nnz == 0) return cudaSuccess;
  constexpr int V = 16 / (int)sizeof(T);
  const bool vec = k >= V && (reinterpret_cast<uintptr_t>(X) % 16 == 0) && (reinterpret_cast<uintptr_t>(dY) % 16 == 0) &&
                   (ldx * (long long)sizeof(T)) % 16 == 0 && (lddy * (long long)sizeof(T)) % 16 == 0;
  const int grid = (int)std::min<long long>(152LL * 16, (nnz + 255) / 256);
  if (vec)
    sddmm_kernel<T, V><<<grid, 256, 0, s>>>(nnz, k, rows, col_idx, static_cast<const T*>(X), ldx,
                                            static_cast<const T*>(dY), lddy, static_cast<T*>(dvals));
  else
    sddmm_kernel<T, 1><<<grid, 256, 0, s>>>(nnz, k, rows, col_idx, static_cast<const T*>(X), ldx,
                                            static_cast<const T*>(dY), lddy, static_cast<T*>(dvals));
  return cudaGetLastError();
}

cudaError_t launch_sddmm(int dtype, int nnz, int k, const int* rows, const int* col_idx, const void* X, long long ldx,
                         const void* dY, long long lddy, void* dvals, cudaStream_t s) {
  return dtype == GBS_F64 ? sddmm_t<double>(nnz, k, rows, col_idx, X, ldx, dY, lddy, dvals, s)
                          : sddmm_t<float>(nnz, k, rows, col_idx, X, ldx, dY, lddy, dvals, s);
}

}  // namespace gbs
