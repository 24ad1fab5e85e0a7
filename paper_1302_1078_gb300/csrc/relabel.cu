// Column relabelling by in-degree, hottest column first (plans of matrices
// whose column degrees are skewed, such as power-law graphs).
//
// The paper ties SpMV speed to how well the gathers of x reuse cache lines
// (Sec. 4.1, Sec. 4.3) and reorders matrices to improve that reuse
// (Sec. 4.4).  On a power-law matrix a few columns take a large share of
// the nonzeros, but in their original numbering they lie scattered over x,
// one per cache line.  Relabelling the columns by their number of stored
// entries, most first, packs the hot entries of x into a few lines that L1
// keeps.  Only the column ids change: rows, and with them y and the
// order of every row's terms, stay as stored, so the relabelled product is
// bitwise the original one.
//
//   plan time (once):  deg[j] = entries in column j;  the columns ranked by
//                      deg descending, ties by ascending id (a stable radix
//                      sort of the keys maxdeg - deg[j]);  newid[j] = rank;
//                      col'[p] = newid[col_idx[p]].
//   every call:        x'[newid[j]] = x[j]  (SpMM: the row X'[newid[j], :]),
//                      then the product of (row_ptr, col', vals) with x'.
//
// All of it is integer index work and deterministic (the degree counts use
// integer atomics, whose order does not matter).
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "gbspmv.h"
#include "launch.h"

namespace gbs {

namespace {

int grid_for(long long work, int threads = 256) {
  return (int)std::min<long long>(152LL * 32, std::max<long long>(1, (work + threads - 1) / threads));
}

__global__ void col_degree_kernel(const int* __restrict__ col_idx, int nnz, int* __restrict__ deg) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (long long)gridDim.x * blockDim.x)
    atomicAdd(deg + col_idx[p], 1);
}

// sums of the degree statistics: acc[0] = sum deg^2 (64-bit), max degree in *mx
__global__ void degree_moments_kernel(const int* __restrict__ deg, int n, unsigned long long* __restrict__ acc,
                                      int* __restrict__ mx) {
  unsigned long long sq = 0;
  int m = 0;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    const int d = deg[j];
    sq += (unsigned long long)d * (unsigned long long)d;
    m = max(m, d);
  }
  for (int o = 16; o > 0; o >>= 1) {
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
    m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc, sq);
    atomicMax(mx, m);
  }
}

// key[j] = maxdeg - deg[j] (ascending key = descending degree), val[j] = j
__global__ void degree_keys_kernel(const int* __restrict__ deg, int n, int maxdeg, int* __restrict__ key,
                                   int* __restrict__ val) {
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    key[j] = maxdeg - deg[j];
    val[j] = (int)j;
  }
}

__global__ void invert_kernel(const int* __restrict__ order, int n, int* __restrict__ newid) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    newid[order[q]] = (int)q;
}

__global__ void relabel_cols_kernel(const int* __restrict__ col_idx, const int* __restrict__ newid, int nnz,
                                    int* __restrict__ out) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (long long)gridDim.x * blockDim.x)
    out[p] = __ldg(newid + col_idx[p]);
}

// x'[newid[j]] = x[j]: coalesced reads of x and newid, scattered 8- or 4-byte writes
template <typename T>
__global__ void scatter_vec_kernel(const T* __restrict__ x, const int* __restrict__ newid, int n, T* __restrict__ xp) {
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
    xp[newid[j]] = x[j];
}

// X'[newid[j], :] = X[j, :], one 16-byte chunk per thread (rows 16-byte aligned, k * sizeof(T) a
// multiple of 16 within the row's chunks; a ragged last chunk is copied element-wise)
template <typename T>
__global__ void scatter_rows_kernel(const T* __restrict__ X, long long ldx, int k, const int* __restrict__ newid, int n,
                                    T* __restrict__ Xp, long long ldxp, bool vec16) {
  constexpr int V = 16 / (int)sizeof(T);
  const int chunks = vec16 ? (k + V - 1) / V : k;
  const long long total = (long long)n * chunks;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long j = t / chunks;
    const int c = (int)(t - j * chunks);
    const T* src = X + j * ldx;
    T* dst = Xp + (long long)__ldg(newid + j) * ldxp;
    if (vec16 && (c + 1) * V <= k) {
      reinterpret_cast<uint4*>(dst)[c] = reinterpret_cast<const uint4*>(src)[c];
    } else if (vec16) {
      for (int q = c * V; q < k; ++q) dst[q] = src[q];
    } else {
      dst[c] = src[c];
    }
  }
}

}  // namespace

cudaError_t col_degree_stats(int n, int nnz, const int* col_idx, int* max_deg, double* cv_deg, cudaStream_t s) {
  *max_deg = 0;
  *cv_deg = 0.0;
  if (n <= 0 || nnz <= 0) return cudaSuccess;
  void* buf = nullptr;
  const size_t bdeg = ((size_t)n * sizeof(int) + 255) & ~(size_t)255;
  cudaError_t e = cudaMallocAsync(&buf, bdeg + 64, s);
  if (e != cudaSuccess) return e;
  int* deg = static_cast<int*>(buf);
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(static_cast<char*>(buf) + bdeg);
  int* mx = reinterpret_cast<int*>(acc + 1);
  unsigned long long h_sq = 0;
  int h_mx = 0;
  e = cudaMemsetAsync(buf, 0, bdeg + 64, s);
  if (e == cudaSuccess) {
    col_degree_kernel<<<grid_for(nnz), 256, 0, s>>>(col_idx, nnz, deg);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    degree_moments_kernel<<<std::min(1024, grid_for(n)), 256, 0, s>>>(deg, n, acc, mx);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_sq, acc, sizeof(h_sq), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_mx, mx, sizeof(h_mx), cudaMemcpyDeviceToHost, s);
  cudaError_t e2 = cudaFreeAsync(buf, s);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  const double mean = (double)nnz / n;
  const double var = (double)h_sq / n - mean * mean;
  *max_deg = h_mx;
  *cv_deg = mean > 0 ? std::sqrt(std::max(0.0, var)) / mean : 0.0;
  return cudaSuccess;
}

cudaError_t relabel_build(int n, int nnz, const int* col_idx, int* newid, int* col_rl, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t bi = ((size_t)n * sizeof(int) + 255) & ~(size_t)255;
  const size_t bh = (transpose_hist_ints(n) * sizeof(int) + 255) & ~(size_t)255;
  const size_t bw = (transpose_scan_ws_ints(n) * sizeof(int) + 255) & ~(size_t)255;
  void* buf = nullptr;
  cudaError_t e = cudaMallocAsync(&buf, 5 * bi + bh + bw + 256, s);
  if (e != cudaSuccess) return e;
  char* b = static_cast<char*>(buf);
  int* deg = reinterpret_cast<int*>(b);
  int* ka = reinterpret_cast<int*>(b + bi);
  int* kb = reinterpret_cast<int*>(b + 2 * bi);
  int* va = reinterpret_cast<int*>(b + 3 * bi);
  int* vb = reinterpret_cast<int*>(b + 4 * bi);
  int* hist = reinterpret_cast<int*>(b + 5 * bi);
  int* ws = reinterpret_cast<int*>(b + 5 * bi + bh);
  int* mx = reinterpret_cast<int*>(b + 5 * bi + bh + bw);
  unsigned long long* sq = reinterpret_cast<unsigned long long*>(mx + 2);
  int h_mx = 0;
  e = cudaMemsetAsync(deg, 0, (size_t)n * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(mx, 0, 256, s);
  if (e == cudaSuccess && nnz > 0) {
    col_degree_kernel<<<grid_for(nnz), 256, 0, s>>>(col_idx, nnz, deg);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    degree_moments_kernel<<<std::min(1024, grid_for(n)), 256, 0, s>>>(deg, n, sq, mx);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_mx, mx, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) {
    degree_keys_kernel<<<grid_for(n), 256, 0, s>>>(deg, n, h_mx, ka, va);
    e = cudaGetLastError();
  }
  int bits = 0;
  while (bits < 31 && (1LL << bits) <= (long long)h_mx) ++bits;
  int *ko = nullptr, *vo = nullptr;
  if (e == cudaSuccess) e = radix_sort_pairs(n, bits, ka, kb, va, vb, hist, ws, &ko, &vo, s);
  if (e == cudaSuccess) {
    invert_kernel<<<grid_for(n), 256, 0, s>>>(vo, n, newid);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && nnz > 0) {
    relabel_cols_kernel<<<grid_for(nnz), 256, 0, s>>>(col_idx, newid, nnz, col_rl);
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaFreeAsync(buf, s);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

cudaError_t relabel_dense(int dtype, int n, int k, const void* X, long long ldx, const int* newid, void* Xp,
                          long long ldxp, bool vec16, cudaStream_t s) {
  if (n <= 0 || k <= 0) return cudaSuccess;
  if (k == 1 && ldx == 1 && ldxp == 1) {
    if (dtype == GBS_F64)
      scatter_vec_kernel<double><<<grid_for(n), 256, 0, s>>>(static_cast<const double*>(X), newid, n,
                                                              static_cast<double*>(Xp));
    else
      scatter_vec_kernel<float><<<grid_for(n), 256, 0, s>>>(static_cast<const float*>(X), newid, n,
                                                             static_cast<float*>(Xp));
    return cudaGetLastError();
  }
  const int V = dtype == GBS_F64 ? 2 : 4;
  const long long chunks = vec16 ? (k + V - 1) / V : k;
  if (dtype == GBS_F64)
    scatter_rows_kernel<double><<<grid_for((long long)n * chunks), 256, 0, s>>>(
        static_cast<const double*>(X), ldx, k, newid, n, static_cast<double*>(Xp), ldxp, vec16);
  else
    scatter_rows_kernel<float><<<grid_for((long long)n * chunks), 256, 0, s>>>(
        static_cast<const float*>(X), ldx, k, newid, n, static_cast<float*>(Xp), ldxp, vec16);
  return cudaGetLastError();
}

}  // namespace gbs
