// Exclusive prefix sum of int32 on the device (reduce, scan of block sums,
// apply), used by the transpose's radix sort.  Integer only, in place allowed.
#include <algorithm>

#include "launch.h"

namespace gbs {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan of v across the CTA (every thread calls it); returns the CTA total in *total.
__device__ __forceinline__ int cta_exclusive_scan(int v, int* total) {
  __shared__ int warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_sums[w] = inc;
  __syncthreads();
  if (w == 0) {
    int s = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = s;  // inclusive over warps
  }
  __syncthreads();
  const int before = w == 0 ? 0 : warp_sums[w - 1];
  *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return before + inc - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const int* __restrict__ in, long long count,
                                                                   int* __restrict__ bsum) {
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  int s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < count) s += in[base + i];
  int total;
  cta_exclusive_scan(s, &total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_bsums_kernel(int* __restrict__ bsum, int nb) {
  int carry = 0;
  for (int c0 = 0; c0 < nb; c0 += kScanThreads) {
    const int i = c0 + threadIdx.x;
    const int v = i < nb ? bsum[i] : 0;
    int total;
    const int ex = cta_exclusive_scan(v, &total);
    if (i < nb) bsum[i] = carry + ex;
    carry += total;
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const int* in, int* out, long long count,
                                                                  const int* __restrict__ bsum) {
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  int v[kScanItems];
  int s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < count ? in[base + i] : 0;
    s += v[i];
  }
  int total;
  int ex = cta_exclusive_scan(s, &total) + bsum[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < count) out[base + i] = ex;
    ex += v[i];
  }
}

size_t scan_workspace_ints(long long count) { return (size_t)std::max<long long>(1, (count + kScanTile - 1) / kScanTile); }

cudaError_t exclusive_scan_i32(const int* in, int* out, long long count, int* ws, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int nb = (int)((count + kScanTile - 1) / kScanTile);
  scan_reduce_kernel<<<nb, kScanThreads, 0, s>>>(in, count, ws);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  scan_bsums_kernel<<<1, kScanThreads, 0, s>>>(ws, nb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  scan_apply_kernel<<<nb, kScanThreads, 0, s>>>(in, out, count, ws);
  return cudaGetLastError();
}

}  // namespace gbs
