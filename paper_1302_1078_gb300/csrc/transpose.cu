// Deterministic CSR transpose (the CRS of A^T, i.e. the CCS of A: Sec. 3
// notes that the two formats are dual) and the transpose plan used by the
// backward pass.
//
// The nonzeros are stably sorted by column id with an LSD radix sort (8-bit
// digits) whose values are the original positions; the stable order inside
// each column of A is therefore the order of storage, exactly as a counting
// sort gives it.  Every pass is:
//   1. per tile of 2048 keys, a 256-bin digit histogram (shared memory);
//   2. an exclusive scan of the histograms in digit-major order;
//   3. a scatter in which each key's rank among equal digits of its tile is
//      computed in position order (warp match + popcount, then a per-digit
//      prefix over warps), so no atomic decides any output position.
// row_ptr of A^T comes from the boundaries of the sorted keys, col_idx of
// A^T by gathering the row of each sorted nonzero.  All of it is integer
// work and bit-exact.
#include <algorithm>
#include <cstdint>
#include <string>

#include "gbspmv.h"
#include "launch.h"

namespace gbs {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048 keys per tile

__global__ void iota_kernel(int* __restrict__ out, int n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) out[i] = i;
}

// Row of every nonzero: one warp per row writes the row id over its range.
__global__ void expand_rows_kernel(const int* __restrict__ row_ptr, int m, int* __restrict__ rows) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = warp; i < m; i += nwarps) {
    const int s = row_ptr[i], e = row_ptr[i + 1];
    for (int p = s + lane; p < e; p += 32) rows[p] = (int)i;
  }
}

__global__ void __launch_bounds__(kSortThreads) radix_upsweep(const int* __restrict__ keys, int n, int shift, int ntiles,
                                                              int* __restrict__ hist) {
  __shared__ int h[256];
  const int tile = blockIdx.x;
  h[threadIdx.x] = 0;
  __syncthreads();
  const int base = tile * kSortTile;
  for (int q = threadIdx.x; q < kSortTile; q += kSortThreads) {
    const int idx = base + q;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255], 1);  // counts only: order-free
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * ntiles + tile] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) radix_downsweep(const int* __restrict__ keys_in,
                                                                const int* __restrict__ vals_in,
                                                                int* __restrict__ keys_out, int* __restrict__ vals_out,
                                                                int n, int shift, int ntiles,
                                                                const int* __restrict__ offs) {
  constexpr int W = kSortThreads / 32;
  __shared__ int wcnt[W][256];
  __shared__ int dbase[256];
  const int tile = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = threadIdx.x; q < W * 256; q += kSortThreads) (&wcnt[0][0])[q] = 0;
  dbase[threadIdx.x] = offs[(size_t)threadIdx.x * ntiles + tile];
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  int key[kSortItems], val[kSortItems], dig[kSortItems], wr[kSortItems];
  // warp w owns the contiguous run [w*256, w*256 + 256) of the tile, 32 keys per round
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int idx = tile * kSortTile + w * 256 + r * 32 + lane;
    const bool valid = idx < n;
    const int k = valid ? keys_in[idx] : 0;
    const int d = valid ? ((k >> shift) & 255) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, valid ? d : 256 + lane);
    const int rank = __popc(peers & lt);
    const int leader = __ffs(peers) - 1;
    const int before = valid ? wcnt[w][d] : 0;
    __syncwarp();
    if (valid && lane == leader) wcnt[w][d] = before + __popc(peers);
    __syncwarp();
    key[r] = k;
    val[r] = valid ? vals_in[idx] : 0;
    dig[r] = d;
    wr[r] = before + rank;
  }
  __syncthreads();
  {
    // per-digit exclusive prefix over warps (warp order = position order)
    const int d = threadIdx.x;
    int s = 0;
#pragma unroll
    for (int ww = 0; ww < W; ++ww) {
      const int t = wcnt[ww][d];
      wcnt[ww][d] = s;
      s += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    if (dig[r] >= 0) {
      const int dst = dbase[dig[r]] + wcnt[w][dig[r]] + wr[r];
      keys_out[dst] = key[r];
      vals_out[dst] = val[r];
    }
  }
}

// row_ptr of A^T from the sorted column ids: rptrT[j] = first position whose key >= j.
__global__ void boundaries_kernel(const int* __restrict__ skeys, int nnz, int n, int* __restrict__ rptrT) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q <= nnz; q += (long long)gridDim.x * blockDim.x) {
    const int lo = q == 0 ? 0 : skeys[q - 1] + 1;  // first column starting at q
    const int hi = q == nnz ? n : skeys[q];         // last column starting at q
    for (int j = lo; j <= hi; ++j) rptrT[j] = q;
  }
}

__global__ void gather_int_kernel(const int* __restrict__ src, const int* __restrict__ idx, int n, int* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) out[i] = src[idx[i]];
}

template <typename T>
__global__ void gather_vals_kernel(const T* __restrict__ src, const int* __restrict__ idx, int n, T* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) out[i] = src[idx[i]];
}

static int grid_for(long long work, int threads = 256) {
  return (int)std::min<long long>(152LL * 32, std::max<long long>(1, (work + threads - 1) / threads));
}

// Stable LSD radix sort of n (key, value) pairs by the low `bits` bits of the keys, 8-bit digits
// per pass; keys must be non-negative.  Input in keys_a / vals_a, keys_b / vals_b are the other
// half of the ping-pong; *keys_out / *vals_out point at whichever pair holds the result.  hist and
// scan_ws as for the transpose (transpose_hist_ints(n), transpose_scan_ws_ints(n) ints).
cudaError_t radix_sort_pairs(int n, int bits, int* keys_a, int* keys_b, int* vals_a, int* vals_b, int* hist,
                             int* scan_ws, int** keys_out, int** vals_out, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  int *ki = keys_a, *ko = keys_b, *vi = vals_a, *vo = vals_b;
  if (n > 0) {
    const int ntiles = (n + kSortTile - 1) / kSortTile;
    const long long hcount = 256LL * ntiles;
    for (int shift = 0; shift < bits; shift += 8) {
      radix_upsweep<<<ntiles, kSortThreads, 0, s>>>(ki, n, shift, ntiles, hist);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = exclusive_scan_i32(hist, hist, hcount, scan_ws, s)) != cudaSuccess) return e;
      radix_downsweep<<<ntiles, kSortThreads, 0, s>>>(ki, vi, ko, vo, n, shift, ntiles, hist);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      std::swap(ki, ko);
      std::swap(vi, vo);
    }
  }
  *keys_out = ki;
  *vals_out = vi;
  return e;
}

// Transpose with caller-provided device buffers (see tplan_create for sizes).
// Returns a CUDA error.  tmp must hold 2 * nnz + 2 * nnz ints + hist + scan workspace.
cudaError_t transpose_run(int m, int n, int nnz, const int* row_ptr, const int* col_idx, int* rptrT, int* colT,
                          int* perm, int* rows, int* keys_a, int* keys_b, int* vals_a, int* vals_b, int* hist,
                          int* scan_ws, cudaStream_t s) {
  cudaError_t e;
  if (m > 0 && nnz > 0) {
    expand_rows_kernel<<<grid_for((long long)m * 32), 256, 0, s>>>(row_ptr, m, rows);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (nnz == 0) {
    // every column of A^T is empty
    return cudaMemsetAsync(rptrT, 0, sizeof(int) * ((size_t)n + 1), s);
  }
  iota_kernel<<<grid_for(nnz), 256, 0, s>>>(vals_a, nnz);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(keys_a, col_idx, sizeof(int) * (size_t)nnz, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return e;
  int bits = 0;
  while (bits < 31 && (1LL << bits) < (long long)n) ++bits;
  int *ki = nullptr, *vi = nullptr;
  if ((e = radix_sort_pairs(nnz, bits, keys_a, keys_b, vals_a, vals_b, hist, scan_ws, &ki, &vi, s)) != cudaSuccess)
    return e;
  // ki: sorted column ids, vi: original positions
  boundaries_kernel<<<grid_for((long long)nnz + 1), 256, 0, s>>>(ki, nnz, n, rptrT);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(perm, vi, sizeof(int) * (size_t)nnz, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
  gather_int_kernel<<<grid_for(nnz), 256, 0, s>>>(rows, vi, nnz, colT);
  return cudaGetLastError();
}

cudaError_t gather_values(int dtype, const void* src, const int* perm, int nnz, void* out, cudaStream_t s) {
  if (nnz == 0) return cudaSuccess;
  if (dtype == GBS_F64)
    gather_vals_kernel<double><<<grid_for(nnz), 256, 0, s>>>(static_cast<const double*>(src), perm, nnz,
                                                                 static_cast<double*>(out));
  else
    gather_vals_kernel<float><<<grid_for(nnz), 256, 0, s>>>(static_cast<const float*>(src), perm, nnz,
                                                                static_cast<float*>(out));
  return cudaGetLastError();
}

size_t transpose_scan_ws_ints(int nnz) {
  const int ntiles = (nnz + kSortTile - 1) / kSortTile;
  return scan_workspace_ints(256LL * std::max(ntiles, 1));
}

size_t transpose_hist_ints(int nnz) {
  const int ntiles = (nnz + kSortTile - 1) / kSortTile;
  return 256ULL * std::max(ntiles, 1);
}

}  // namespace gbs
