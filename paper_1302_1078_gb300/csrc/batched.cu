// Batched mode: many CSR products in one persistent launch.
//
// The paper multiplies one matrix at a time (Sec. 4, Sec. 5).  Serving many
// small and uneven matrices one launch each leaves most of GB300's 152 SMs idle
// for the small ones and pays a launch per matrix.  Here one persistent kernel
// walks a work list of (matrix, row block | merge tile) items.  A CTA takes the
// next unclaimed item from a device counter (reset by the graph before every
// launch), so the SMs stay busy until the list is exhausted whatever the items'
// costs; the matrix comes from a binary search of the descriptors' first items
// (a CTA's items only increase, so the search starts at its previous matrix),
// and each item runs exactly the device function the standalone kernels run
// (rows_block / merge_tile) with the matrix's own tuned configuration, so the
// batched result equals the per-matrix loop bitwise: which CTA runs an item
// does not change what the item computes.
//
// A merge-path matrix needs its per-tile carries added after all its tiles are
// done.  The CTA that finishes a matrix's last tile (a per-matrix counter,
// incremented after a memory fence) performs that fix-up and resets the
// counter for the next launch.  No CTA ever waits for another.
#include <cstdint>

#include "batched.cuh"
#include "gbspmv.h"
#include "launch.h"
#include "merge_kernel.cuh"
#include "rows_kernel.cuh"

namespace gbs {

template <typename T>
__device__ __forceinline__ RowsArgs<T> rows_args(const BatchDesc<T>& d) {
  RowsArgs<T> a;
  a.m = d.m;
  a.k = d.k;
  a.row_ptr = d.row_ptr;
  a.col_idx = d.col_idx;
  a.vals = d.vals;
  a.X = d.X;
  a.Y = d.Y;
  a.ldx = d.ldx;
  a.ldy = d.ldy;
  a.tile = d.tile;
  a.row_base = 0;
  a.aligned_vals = d.aligned_vals;
  a.aligned_cols = d.aligned_cols;
  return a;
}

template <typename T>
__device__ __forceinline__ MergeArgs<T> merge_args(const BatchDesc<T>& d) {
  MergeArgs<T> a;
  a.m = d.m;
  a.k = d.k;
  a.nnz = d.nnz;
  a.row_ptr = d.row_ptr;
  a.col_idx = d.col_idx;
  a.vals = d.vals;
  a.X = d.X;
  a.Y = d.Y;
  a.ldx = d.ldx;
  a.ldy = d.ldy;
  a.items = d.items;
  a.ctas = d.nitems;
  a.coords = d.coords;
  a.carry_row = d.carry_row;
  a.carry_val = d.carry_val;
  a.aligned_vals = d.aligned_vals;
  a.aligned_cols = d.aligned_cols;
  return a;
}

// SPLIT (k == 1): ROWS lanes vary per matrix.  !SPLIT (k > 1): every matrix uses G column lanes.
// (ROWS_DIRECT items are not offered: they lost every whole-batch policy, and their code cost this
// register-bound kernel spills.)
template <typename T, int VEC, bool SPLIT, int G>
__global__ void __launch_bounds__(256, 4) batched_kernel(const BatchDesc<T>* __restrict__ descs, int nmat,
                                                      int total_items, int* __restrict__ next_item) {
  __shared__ int s_last, s_item;
  int lo = 0;  // matrix of this CTA's previous item
  // items are claimed one ahead: the claim of the next item is issued when the current one
  // starts, so the atomic's round trip overlaps the current item's work
  if (threadIdx.x == 0) s_item = atomicAdd(next_item, 1);
  __syncthreads();
  for (;;) {
    const int item = s_item;
    if (item >= total_items) break;
    int claimed = 0;
    if (threadIdx.x == 0) claimed = atomicAdd(next_item, 1);
    int hi = nmat - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(&descs[mid].item_begin) <= item)
        lo = mid;
      else
        hi = mid - 1;
    }
    const BatchDesc<T> d = descs[lo];
    const int local = item - d.item_begin;
    if (d.variant == GBS_VARIANT_ROWS) {
      const RowsArgs<T> a = rows_args(d);
      if constexpr (SPLIT) {
        switch (d.lanes) {
          case 1: rows_block<T, 1, 1, true>(a, local); break;
          case 2: rows_block<T, 1, 2, true>(a, local); break;
          case 4: rows_block<T, 1, 4, true>(a, local); break;
          case 8: rows_block<T, 1, 8, true>(a, local); break;
          case 16: rows_block<T, 1, 16, true>(a, local); break;
          default: rows_block<T, 1, 32, true>(a, local); break;
        }
      } else {
        rows_block<T, VEC, G, false>(a, local);
      }
    } else {
      const MergeArgs<T> a = merge_args(d);
      merge_tile<T, VEC, (SPLIT ? 1 : G), false>(a, local);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();  // this tile's Y rows and carry are visible before it is counted
        s_last = atomicAdd(d.done, 1) == d.nitems - 1;
      }
      __syncthreads();
      if (s_last) {
        __threadfence();  // every other tile of the matrix has been counted: read their carries
        for (int t = threadIdx.x; t < d.nitems; t += blockDim.x)
          merge_fixup_one<T>(t, d.nitems, d.k, d.carry_row, d.carry_val, d.Y, d.ldy);
        if (threadIdx.x == 0) *d.done = 0;
      }
    }
    // every thread read s_item before the item's first internal barrier, and no thread reads
    // shared memory after the item's last barrier (ROWS: the last tile pass ends with one; MERGE:
    // the barrier before the completion count), so the next item's index is published, and the
    // shared memory handed over, with a single barrier
    if (threadIdx.x == 0) s_item = claimed;
    __syncthreads();
  }
}

template <typename T, int VEC, bool SPLIT, int G>
static cudaError_t batched_go(bool launch, const void* descs, int nmat, int total_items, int* next_item, int grid,
                              size_t smem, int* blocks_per_sm, cudaStream_t s) {
  auto kern = batched_kernel<T, VEC, SPLIT, G>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (!launch) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, 256, smem);
  kern<<<grid, 256, smem, s>>>(static_cast<const BatchDesc<T>*>(descs), nmat, total_items, next_item);
  return cudaGetLastError();
}

template <typename T, int VEC>
static cudaError_t batched_g(bool launch, bool split, int G, const void* descs, int nmat, int total_items,
                             int* next_item, int grid, size_t smem, int* bps, cudaStream_t s) {
  if (split) return batched_go<T, 1, true, 1>(launch, descs, nmat, total_items, next_item, grid, smem, bps, s);
  switch (G) {
    case 1: return batched_go<T, VEC, false, 1>(launch, descs, nmat, total_items, next_item, grid, smem, bps, s);
    case 2: return batched_go<T, VEC, false, 2>(launch, descs, nmat, total_items, next_item, grid, smem, bps, s);
    case 4: return batched_go<T, VEC, false, 4>(launch, descs, nmat, total_items, next_item, grid, smem, bps, s);
    case 8: return batched_go<T, VEC, false, 8>(launch, descs, nmat, total_items, next_item, grid, smem, bps, s);
    case 16: return batched_go<T, VEC, false, 16>(launch, descs, nmat, total_items, next_item, grid, smem, bps, s);
    case 32: return batched_go<T, VEC, false, 32>(launch, descs, nmat, total_items, next_item, grid, smem, bps, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t batched_kernel_call(bool launch, int dtype, bool split, int G, bool vec16, const void* descs, int nmat,
                                int total_items, int* next_item, int grid, size_t smem, int* blocks_per_sm,
                                cudaStream_t s) {
  if (dtype == GBS_F64)
    return vec16 ? batched_g<double, 2>(launch, split, G, descs, nmat, total_items, next_item, grid, smem,
                                        blocks_per_sm, s)
                 : batched_g<double, 1>(launch, split, G, descs, nmat, total_items, next_item, grid, smem,
                                        blocks_per_sm, s);
  return vec16 ? batched_g<float, 4>(launch, split, G, descs, nmat, total_items, next_item, grid, smem, blocks_per_sm,
                                     s)
               : batched_g<float, 1>(launch, split, G, descs, nmat, total_items, next_item, grid, smem, blocks_per_sm,
                                     s);
}

}  // namespace gbs
