// Register-blocked CRS ("BCSR", the paper's register blocking, Sec. 4.5):
// A is cut into aligned a x b regions; every region holding a stored entry
// becomes a dense row-major block (zeros included), and the blocks of each
// block row (rows I*a .. I*a+a-1) are listed by block column, ascending.
//
// Conversion (once per matrix; the paper leaves it out of its timings):
//   * the block columns col/b of each block row are a contiguous slice of
//     col_idx; two stable transposes sort each slice, and a ballot count of
//     value changes gives the distinct block columns (count, scan, write);
//   * one thread per row of A adds its entries into their blocks in storage
//     order (a binary search finds the block), so repeated entries add up in
//     a fixed order and no two threads touch the same value.
//
// SpMV: a group of min(32, a*b) lanes per block row, each lane holding one or
// two elements of every block (element e = lane + e*group, row e / b, column
// e % b).  A block's values are one coalesced load of a*b consecutive
// elements, its x slice x[J*b .. J*b+b-1] a contiguous gather (one broadcast
// element for b == 1), and each block costs a*b fused multiply-adds, zeros
// included: on GB300 the fill ratio of the blocks is paid on the FP64 pipe as
// well as in bytes.  The b lanes of a row then add their partials with
// shuffles and the lane of column 0 writes y.  Sums run in a fixed order.
#include <algorithm>
#include <cstdint>

#include "device_common.cuh"
#include "gbspmv.h"
#include "launch.h"

namespace gbs {

namespace {

constexpr int kThreads = 256;

int grid_for(long long work) {
  return (int)std::min<long long>(152LL * 32, std::max<long long>(1, (work + kThreads - 1) / kThreads));
}

__global__ void slice_rows_k(int mb, int a, int m, const int* __restrict__ rp, int* __restrict__ gp) {
  for (long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x; I <= mb; I += (long long)gridDim.x * blockDim.x)
    gp[I] = rp[min(I * a, (long long)m)];
}
__global__ void block_cols_k(int nnz, int b, const int* __restrict__ ci, int* __restrict__ gc) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (long long)gridDim.x * blockDim.x) gc[p] = ci[p] / b;
}
// distinct sorted values per row: count (FILL == false) or write
template <bool FILL>
__global__ void unique_k(int mb, const int* __restrict__ rp, const int* __restrict__ c, int* __restrict__ cnt,
                         const int* __restrict__ outp, int* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < mb;
       w += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int s = rp[w], e = rp[w + 1];
    int k = 0;
    for (int base = s; base < e; base += 32) {
      const int p = base + lane;
      const bool first = p < e && (p == s || c[p] != c[p - 1]);
      const unsigned m = __ballot_sync(0xffffffffu, first);
      if (FILL && first) out[outp[w] + k + __popc(m & lt)] = c[p];
      k += __popc(m);
    }
    if (!FILL && lane == 0) cnt[w] = k;
  }
}
template <typename T>
__global__ void scatter_vals_k(int m, int a, int b, const int* __restrict__ rp, const int* __restrict__ ci,
                               const T* __restrict__ vals, const int* __restrict__ bptr, const int* __restrict__ bcol,
                               T* __restrict__ bval) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const int I = i / a, r = i - I * a;
    const int lo0 = bptr[I], hi0 = bptr[I + 1];
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      const int j = ci[p], J = j / b;
      int lo = lo0, hi = hi0 - 1;
      while (lo < hi) {  // first block column >= J (it is present)
        const int mid = (lo + hi) >> 1;
        if (bcol[mid] < J)
          lo = mid + 1;
        else
          hi = mid;
      }
      T* slot = bval + (long long)lo * a * b + (long long)r * b + (j - J * b);
      *slot = *slot + vals[p];
    }
  }
}
__global__ void tail_k(const int* __restrict__ off, const int* __restrict__ cnt, int k, int* __restrict__ out) {
  out[0] = off[k - 1] + cnt[k - 1];
}

size_t tx_ints(int cap) {
  return 5 * (size_t)std::max(cap, 1) + transpose_hist_ints(cap) + transpose_scan_ws_ints(cap);
}

// ---- SpMV
template <typename T, int A, int B>
__global__ void __launch_bounds__(kThreads) bcsr_spmv_k(int m, int n, int mb, const int* __restrict__ bptr,
                                                        const int* __restrict__ bcol, const T* __restrict__ bval,
                                                        const T* __restrict__ x, T* __restrict__ y) {
  constexpr int AB = A * B;
  constexpr int G = AB < 32 ? AB : 32;  // lanes per block row
  constexpr int E = AB / G;             // elements per lane
  constexpr int GPW = 32 / G;           // block rows per warp
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_keep = policy_evict_last();
  const int lane = threadIdx.x & 31;
  const int gl = lane % G;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long I0 = warp * GPW; I0 < mb; I0 += nwarps * GPW) {
    const long long I = I0 + lane / G;
    const bool active = I < mb;
    Acc<T> acc[E];
    if (active) {
      const int k0 = bptr[I], k1 = bptr[I + 1];
      for (int k = k0; k < k1; ++k) {
        const int J = bcol[k];
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int idx = gl + e * G;
          const int j = J * B + idx % B;
          const T v = ld_stream(bval + (long long)k * AB + idx, pol_stream);
          const T xv = j < n ? ld_keep(x + j, pol_keep) : T(0);
          acc[e].add(v, xv);
        }
      }
    }
    // the B lanes of a row (consecutive, B-aligned inside the group) add their partials
#pragma unroll
    for (int e = 0; e < E; ++e) {
      T s = acc[e].value();
#pragma unroll
      for (int o = B / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const int idx = gl + e * G;
      const long long row = I * A + idx / B;
      if (active && idx % B == 0 && row < m) st_stream(y + row, s);
    }
  }
}

template <typename T, int A, int B>
cudaError_t go(int m, int n, int mb, const int* bptr, const int* bcol, const void* bval, const void* x, void* y,
               cudaStream_t s) {
  constexpr int G = A * B < 32 ? A * B : 32;
  const long long warps = (mb + (32 / G) - 1) / (32 / G);
  bcsr_spmv_k<T, A, B><<<grid_for(warps * 32), kThreads, 0, s>>>(m, n, mb, bptr, bcol, static_cast<const T*>(bval),
                                                                 static_cast<const T*>(x), static_cast<T*>(y));
  return cudaGetLastError();
}

template <typename T, int A>
cudaError_t go_b(int b, int m, int n, int mb, const int* bptr, const int* bcol, const void* bval, const void* x,
                 void* y, cudaStream_t s) {
  switch (b) {
    case 1: return go<T, A, 1>(m, n, mb, bptr, bcol, bval, x, y, s);
    case 2: return go<T, A, 2>(m, n, mb, bptr, bcol, bval, x, y, s);
    case 4: return go<T, A, 4>(m, n, mb, bptr, bcol, bval, x, y, s);
    case 8: return go<T, A, 8>(m, n, mb, bptr, bcol, bval, x, y, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t go_ab(int a, int b, int m, int n, int mb, const int* bptr, const int* bcol, const void* bval,
                  const void* x, void* y, cudaStream_t s) {
  switch (a) {
    case 1: return go_b<T, 1>(b, m, n, mb, bptr, bcol, bval, x, y, s);
    case 2: return go_b<T, 2>(b, m, n, mb, bptr, bcol, bval, x, y, s);
    case 4: return go_b<T, 4>(b, m, n, mb, bptr, bcol, bval, x, y, s);
    case 8: return go_b<T, 8>(b, m, n, mb, bptr, bcol, bval, x, y, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t bcsr_count(int m, int n, int nnz, const int* row_ptr, const int* col_idx, int a, int b, int* bptr,
                       int** bcol_sorted, int* nblocks, void** scratch, cudaStream_t s) {
  // scratch layout (ints): gp (mb+1), gc (nnz), T1 rp (nbc+1), T1 col, T1 perm, T2 rp (mb+1), T2 col, T2 perm,
  // counts (mb), small, scan workspace, transpose scratch
  const int mb = (m + a - 1) / a, nbc = (n + b - 1) / b;
  const size_t c = (size_t)std::max(nnz, 1);
  const size_t ints = (mb + 1) + c + (nbc + 1) + 2 * c + (mb + 1) + 2 * c + (mb + 1) + 64 +
                      scan_workspace_ints((long long)mb + 1) + tx_ints(nnz);
  int* base = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&base), ints * sizeof(int), s);
  if (e != cudaSuccess) return e;
  *scratch = base;
  int* p = base;
  auto take = [&](size_t k) {
    int* r = p;
    p += k;
    return r;
  };
  int *gp = take(mb + 1), *gc = take(c), *rp1 = take(nbc + 1), *c1 = take(c), *p1 = take(c);
  int *rp2 = take(mb + 1), *c2 = take(c), *p2 = take(c), *cnt = take(mb + 1), *small = take(64);
  int* sws = take(scan_workspace_ints((long long)mb + 1));
  int* txb = take(tx_ints(nnz));
  const size_t cc = (size_t)std::max(nnz, 1);
  int* tx_rows = txb;
  int* tx_ka = txb + cc;
  int* tx_kb = txb + 2 * cc;
  int* tx_va = txb + 3 * cc;
  int* tx_vb = txb + 4 * cc;
  int* tx_hist = txb + 5 * cc;
  int* tx_ws = tx_hist + transpose_hist_ints(nnz);
  slice_rows_k<<<grid_for(mb + 1), kThreads, 0, s>>>(mb, a, m, row_ptr, gp);
  if (nnz > 0) block_cols_k<<<grid_for(nnz), kThreads, 0, s>>>(nnz, b, col_idx, gc);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = transpose_run(mb, nbc, nnz, gp, gc, rp1, c1, p1, tx_rows, tx_ka, tx_kb, tx_va, tx_vb, tx_hist, tx_ws, s)) !=
      cudaSuccess)
    return e;
  if ((e = transpose_run(nbc, mb, nnz, rp1, c1, rp2, c2, p2, tx_rows, tx_ka, tx_kb, tx_va, tx_vb, tx_hist, tx_ws, s)) !=
      cudaSuccess)
    return e;
  unique_k<false><<<grid_for((long long)mb * 32), kThreads, 0, s>>>(mb, rp2, c2, cnt, nullptr, nullptr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = exclusive_scan_i32(cnt, bptr, mb, sws, s)) != cudaSuccess) return e;
  tail_k<<<1, 1, 0, s>>>(bptr, cnt, mb, small);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(bptr + mb, small, sizeof(int), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(nblocks, small, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  *bcol_sorted = c2;  // rows of the sorted block columns (rp2), used by bcsr_fill
  (void)rp2;
  return cudaSuccess;
}

cudaError_t bcsr_fill(int m, int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals, int dtype,
                      int a, int b, const int* bptr, int* bcol, void* bval, long long nblocks, void* scratch,
                      cudaStream_t s) {
  const int mb = (m + a - 1) / a, nbc = (n + b - 1) / b;
  const size_t c = (size_t)std::max(nnz, 1);
  int* base = static_cast<int*>(scratch);
  int* rp2 = base + (mb + 1) + c + (nbc + 1) + 2 * c;
  int* c2 = rp2 + (mb + 1);
  cudaError_t e = cudaSuccess;
  if (mb > 0) unique_k<true><<<grid_for((long long)mb * 32), kThreads, 0, s>>>(mb, rp2, c2, nullptr, bptr, bcol);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t es = dtype == GBS_F64 ? 8 : 4;
  if ((e = cudaMemsetAsync(bval, 0, (size_t)nblocks * a * b * es, s)) != cudaSuccess) return e;
  if (m > 0 && nnz > 0) {
    if (dtype == GBS_F64)
      scatter_vals_k<double><<<grid_for(m), kThreads, 0, s>>>(m, a, b, row_ptr, col_idx,
                                                             static_cast<const double*>(vals), bptr, bcol,
                                                             static_cast<double*>(bval));
    else
      scatter_vals_k<float><<<grid_for(m), kThreads, 0, s>>>(m, a, b, row_ptr, col_idx,
                                                            static_cast<const float*>(vals), bptr, bcol,
                                                            static_cast<float*>(bval));
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t bcsr_spmv(int dtype, int a, int b, int m, int n, const int* bptr, const int* bcol, const void* bval,
                      const void* x, void* y, cudaStream_t s) {
  const int mb = (m + a - 1) / a;
  if (mb == 0) return cudaSuccess;
  return dtype == GBS_F64 ? go_ab<double>(a, b, m, n, mb, bptr, bcol, bval, x, y, s)
                          : go_ab<float>(a, b, m, n, mb, bptr, bcol, bval, x, y, s);
}

}  // namespace gbs
