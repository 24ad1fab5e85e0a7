// Backward pass of Y = A X with respect to the stored values (the paper has
// no backward pass): the sampled dense-dense product over A's pattern
//   dvals[p] = sum_c dY[row(p), c] * X[col_idx[p], c].
// Each lane of a warp takes U nonzeros 32 apart (the warp covers 32 * U consecutive ones) and
// sums each one's k products in column order, so no FP64 reduction across lanes is needed (on
// GB300 every FP64 instruction counts).  Every id load and dvals store of the warp is 32
// consecutive elements, and a lane's U gathers are independent, so U are in flight per lane;
// neighbouring nonzeros mostly share their dY row (served by L1).  The X rows are gathered with the
// L2 evict-last policy, like SpMM.
#include <algorithm>
#include <cstdint>

#include "device_common.cuh"
#include "gbspmv.h"
#include "launch.h"

namespace gbs {

template <typename T, int VEC, int U, bool K1>
__global__ void __launch_bounds__(256) sddmm_kernel(int nnz, int k, const int* __restrict__ rows,
                                                    const int* __restrict__ col_idx, const T* __restrict__ X,
                                                    long long ldx, const T* __restrict__ dY, long long lddy,
                                                    T* __restrict__ dvals) {
  const uint64_t pol_keep = policy_evict_last();
  const uint64_t pol_stream = policy_evict_first();
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long step = ((long long)gridDim.x * blockDim.x >> 5) * 32 * U;
  for (long long base = warp * 32 * U; base < nnz; base += step) {
    long long p[U];
    bool in[U];
    int iu[U], ju[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      p[u] = base + 32 * u + lane;
      in[u] = p[u] < nnz;
      iu[u] = in[u] ? ld_stream(rows + p[u], pol_stream) : 0;
      ju[u] = in[u] ? ld_stream(col_idx + p[u], pol_stream) : 0;
    }
    Acc<T> acc[U];
    int c = 0;
    if constexpr (K1) {
      T xs[U], ys[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (in[u]) {
          xs[u] = ld_keep(X + ju[u], pol_keep);
          ys[u] = ld_keep(dY + iu[u], pol_keep);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) acc[u].add(ys[u], xs[u]);
      c = k;
    }
    if constexpr (VEC > 1) {
      for (; c + VEC <= k; c += VEC) {
        Vec<T, VEC> xv[U], yv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (in[u]) {
            xv[u] = ld_keep_vec<T, VEC>(X + (long long)ju[u] * ldx + c, pol_keep);
            yv[u] = ld_keep_vec<T, VEC>(dY + (long long)iu[u] * lddy + c, pol_keep);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int q = 0; q < VEC; ++q) acc[u].add(yv[u].v[q], xv[u].v[q]);
      }
    }
    for (; c < k; ++c) {
      T xs[U], ys[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (in[u]) {
          xs[u] = ld_keep(X + (long long)ju[u] * ldx + c, pol_keep);
          ys[u] = ld_keep(dY + (long long)iu[u] * lddy + c, pol_keep);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) acc[u].add(ys[u], xs[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (in[u]) st_stream(dvals + p[u], acc[u].value());
  }
}

template <typename T>
static cudaError_t sddmm_t(int nnz, int k, const int* rows, const int* col_idx, const void* X, long long ldx,
                           const void* dY, long long lddy, void* dvals, cudaStream_t s) {
  if (nnz == 0) return cudaSuccess;
  constexpr int V = 16 / (int)sizeof(T);
  const bool vec = k >= V && (reinterpret_cast<uintptr_t>(X) % 16 == 0) && (reinterpret_cast<uintptr_t>(dY) % 16 == 0) &&
                   (ldx * (long long)sizeof(T)) % 16 == 0 && (lddy * (long long)sizeof(T)) % 16 == 0;
  constexpr int U = 2;  // nonzeros per lane (four measured no faster; the dot products are the same)
  const int grid = (int)std::min<long long>(152LL * 16, ((long long)nnz + U * 256 - 1) / (U * 256));
  const T* x = static_cast<const T*>(X);
  const T* dy = static_cast<const T*>(dY);
  T* dv = static_cast<T*>(dvals);
  if (k == 1)
    sddmm_kernel<T, 1, U, true><<<grid, 256, 0, s>>>(nnz, k, rows, col_idx, x, 1, dy, 1, dv);
  else if (vec)
    sddmm_kernel<T, V, U, false><<<grid, 256, 0, s>>>(nnz, k, rows, col_idx, x, ldx, dy, lddy, dv);
  else
    sddmm_kernel<T, 1, U, false><<<grid, 256, 0, s>>>(nnz, k, rows, col_idx, x, ldx, dy, lddy, dv);
  return cudaGetLastError();
}

cudaError_t launch_sddmm(int dtype, int nnz, int k, const int* rows, const int* col_idx, const void* X, long long ldx,
                         const void* dY, long long lddy, void* dvals, cudaStream_t s) {
  return dtype == GBS_F64 ? sddmm_t<double>(nnz, k, rows, col_idx, X, ldx, dY, lddy, dvals, s)
                          : sddmm_t<float>(nnz, k, rows, col_idx, X, ldx, dY, lddy, dvals, s);
}

}  // namespace gbs
