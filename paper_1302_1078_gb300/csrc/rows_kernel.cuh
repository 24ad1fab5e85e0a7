// Sub-warp-per-row CSR kernel ("ROWS" variant) for SpMV and SpMM.
//
// The paper's kernel (Sec. 3, Sec. 4.1) gives each row to one thread and
// computes y_i as the dot product of row i with x; its SpMM (Sec. 5) keeps a
// k-wide temporary per row and streams one contiguous row X[j, :] per
// nonzero.  On GB300 the same row-wise scheme is kept, with three changes:
//
//   * A CTA owns a block of consecutive rows.  Their nonzeros (vals, col_idx)
//     are one contiguous range, which the CTA stages into shared memory with
//     coalesced 128-bit loads, TILE nonzeros per pass, so the HBM stream is
//     fully coalesced even when a single lane walks a whole row.
//   * A group of LANES consecutive lanes shares one row.  For SpMV (SPLIT)
//     the lanes split the row's nonzeros and add their partial sums with
//     warp shuffles at the end; for SpMM (!SPLIT) each lane owns VEC of the k
//     columns and walks the whole row, so no reduction is needed.
//   * FP64 arithmetic is a scarce pipe on GB300 (about 1/64 of the FP32
//     rate): each nonzero costs exactly one fused multiply-add per output
//     element, and lanes split columns rather than nonzeros whenever k > 1.
//
// Summation order per output element is fixed (each lane in stored order,
// then a fixed shuffle tree), so results are bitwise reproducible.
//
// PERM: the value of stored entry p is vals[perm[p]] (the backward pass runs
// A^T with A's values in place, perm being the transpose permutation).  The
// CTA then stages perm instead of vals and gathers each value once.
#pragma once
#include "device_common.cuh"

namespace gbs {

template <typename T>
struct RowsArgs {
  int m, k;
  const int* __restrict__ row_ptr;
  const int* __restrict__ col_idx;
  const T* __restrict__ vals;
  const T* __restrict__ X;  // n x k (ldx)
  T* __restrict__ Y;        // m x k (ldy)
  long long ldx, ldy;
  int tile;            // nonzeros staged per pass
  int row_base;        // first row of block 0 (for batched / split launches)
  bool aligned_vals;   // vals (perm when PERM) 16-byte aligned
  bool aligned_cols;   // col_idx 16-byte aligned
  const int* __restrict__ perm = nullptr;  // PERM: value of entry p is vals[perm[p]]
};

// Shared-memory layout: s_rp[rows + 1] | s_val[tile + 4] | s_col[tile + 4]
template <typename T>
__host__ __device__ inline size_t rows_smem_bytes(int rows_per_cta, int tile) {
  size_t a = ((size_t)(rows_per_cta + 1) * sizeof(int) + 15) & ~(size_t)15;
  size_t b = ((size_t)(tile + 4) * sizeof(T) + 15) & ~(size_t)15;
  size_t c = ((size_t)(tile + 4) * sizeof(int) + 15) & ~(size_t)15;
  return a + b + c;
}

constexpr int kUnroll = 4;

template <typename T, int VEC, int LANES, bool SPLIT, bool PERM = false>
__device__ __forceinline__ void rows_block(const RowsArgs<T>& a, int block) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rpc = blockDim.x / LANES;
  const int r0 = a.row_base + block * rpc;
  const int nrows = min(rpc, a.m - r0);
  if (nrows <= 0) return;
  const int tile = a.tile;
  int* s_rp = reinterpret_cast<int*>(smem_raw);
  T* s_val = reinterpret_cast<T*>(smem_raw + (((size_t)(rpc + 1) * sizeof(int) + 15) & ~(size_t)15));
  int* s_col = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(s_val) +
                                      (((size_t)(tile + 4) * sizeof(T) + 15) & ~(size_t)15));
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_keep = policy_evict_last();

  // the block's nonzero range straight from global memory (the same two words for every thread),
  // so that the row pointers and the first tile are staged together, before one barrier
  const int bs = __ldg(a.row_ptr + r0), be = __ldg(a.row_ptr + r0 + nrows);
  for (int i = threadIdx.x; i <= nrows; i += blockDim.x) s_rp[i] = ld_stream(a.row_ptr + r0 + i, pol_stream);

  const int g = threadIdx.x / LANES;
  const int lane = threadIdx.x % LANES;
  const bool active = g < nrows;

  // column slice of this lane (SpMM): [c_lo, c_lo + VEC) clipped to k
  const int c_lo = SPLIT ? 0 : lane * VEC;
  const bool col_active = SPLIT ? true : (c_lo < a.k);
  const bool col_full = SPLIT ? true : (c_lo + VEC <= a.k);

  Acc<T> acc[VEC];
  // value of the staged entry at offset i of the tile
  auto val_at = [&](int i) -> T {
    if constexpr (PERM)
      return __ldg(a.vals + reinterpret_cast<const int*>(s_val)[i]);
    else
      return s_val[i];
  };

  // passes over the block's nonzeros [bs, be), tile at a time (c0 + tile is never formed past be,
  // so positions near 2^31 do not overflow); each pass stages its tile, then one barrier, then
  // computes, then one barrier before the next pass overwrites the tile
  auto stage = [&](int c0, int c1) {
    const int a0 = c0 & ~3;
    if constexpr (PERM)
      stage_copy<int>(reinterpret_cast<int*>(s_val), a.perm, a0, c1, a.aligned_vals, pol_stream);
    else
      stage_copy<T>(s_val, a.vals, a0, c1, a.aligned_vals, pol_stream);
    stage_copy<int>(s_col, a.col_idx, a0, c1, a.aligned_cols, pol_stream);
  };
  int c1 = be - bs > tile ? bs + tile : be;
  if (bs < be) stage(bs, c1);
  __syncthreads();  // row pointers and the first tile
  const int rs = active ? s_rp[g] : 0;
  const int re = active ? s_rp[g + 1] : 0;
  for (int c0 = bs; c0 < be;) {
    const int a0 = c0 & ~3;
    if (active && col_active) {
      const int lo = max(rs, c0), hi = min(re, c1);
      constexpr int STEP = SPLIT ? LANES : 1;
      int p = lo;
      if constexpr (SPLIT) {
        // first p >= lo with (p - rs) % LANES == lane
        int off = (lo - rs) % LANES;
        p = lo + ((lane - off + LANES) % LANES);
      }
      const T* __restrict__ Xc = a.X + c_lo;
      if (col_full) {
        for (; p + (kUnroll - 1) * STEP < hi; p += kUnroll * STEP) {
          T v[kUnroll];
          int c[kUnroll];
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            v[u] = val_at(p + u * STEP - a0);
            c[u] = s_col[p + u * STEP - a0];
          }
          Vec<T, VEC> xv[kUnroll];
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) xv[u] = ld_keep_vec<T, VEC>(Xc + (long long)c[u] * a.ldx, pol_keep);
#pragma unroll
          for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int j = 0; j < VEC; ++j) acc[j].add(v[u], xv[u].v[j]);
        }
        for (; p < hi; p += STEP) {
          const T v = val_at(p - a0);
          const int c = s_col[p - a0];
          Vec<T, VEC> xv = ld_keep_vec<T, VEC>(Xc + (long long)c * a.ldx, pol_keep);
#pragma unroll
          for (int j = 0; j < VEC; ++j) acc[j].add(v, xv.v[j]);
        }
      } else {
        // ragged last column slice: scalar gathers of the valid columns
        const int nv = a.k - c_lo;
        for (; p < hi; p += STEP) {
          const T v = val_at(p - a0);
          const T* xr = Xc + (long long)s_col[p - a0] * a.ldx;
#pragma unroll
          for (int j = 0; j < VEC; ++j)
            if (j < nv) acc[j].add(v, ld_keep(xr + j, pol_keep));
        }
      }
    }
    __syncthreads();  // the tile has been read
    c0 = c1;
    if (c0 < be) {
      c1 = be - c0 > tile ? c0 + tile : be;
      stage(c0, c1);
      __syncthreads();
    }
  }

  if constexpr (SPLIT) {
    // fixed shuffle tree over the LANES lanes of the group
    T s = acc[0].value();
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LANES);
    if (active && lane == 0) st_stream(a.Y + (long long)(r0 + g) * a.ldy, s);
  } else {
    if (active && col_active) {
      T out[VEC];
#pragma unroll
      for (int j = 0; j < VEC; ++j) out[j] = acc[j].value();
      T* yr = a.Y + (long long)(r0 + g) * a.ldy + c_lo;
      if (col_full) {
        st_stream_vec<T, VEC>(yr, out);
      } else {
        for (int j = 0; j < a.k - c_lo; ++j) st_stream(yr + j, out[j]);
      }
    }
  }
}

template <typename T, int VEC, int LANES, bool SPLIT, bool PERM = false>
__global__ void __launch_bounds__(1024) rows_kernel(RowsArgs<T> a) {
  rows_block<T, VEC, LANES, SPLIT, PERM>(a, blockIdx.x);
}

// ROWS_DIRECT: the row-wise arithmetic of rows_block without shared memory.  Every lane loads
// its row's values and column ids itself, through L1 (the lanes of a row read the same words, so
// one request serves them all, and the next words of the row then hit L1), and walks the whole
// row, so a block has no barrier at all.  This is for short rows, where staging a tile and its
// barriers cost more than the products (a 64-row block of a 5-point stencil holds 320
// nonzeros), and for the batched kernel, where every block is a work item.  k > 1: LANES lanes
// split the columns, VEC each; k == 1: one lane per row (LANES == 1).  Each lane sums its
// products in stored order, as rows_block does with lanes that split the columns (or with one
// lane per row), so the two variants give the same bits.
template <typename T, int VEC, int LANES, bool PERM = false>
__device__ __forceinline__ void rows_direct_block(const RowsArgs<T>& a, int block) {
  const int rpc = blockDim.x / LANES;
  const int r = a.row_base + block * rpc + (int)threadIdx.x / LANES;
  const int c_lo = ((int)threadIdx.x % LANES) * VEC;
  if (r >= a.m || c_lo >= a.k) return;
  const bool col_full = c_lo + VEC <= a.k;
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_keep = policy_evict_last();
  const int rs = ld_keep(a.row_ptr + r, pol_stream), re = ld_keep(a.row_ptr + r + 1, pol_stream);
  auto val_at = [&](int p) -> T {
    if constexpr (PERM)
      return __ldg(a.vals + ld_keep(a.perm + p, pol_stream));
    else
      return ld_keep(a.vals + p, pol_stream);
  };
  const T* __restrict__ Xc = a.X + c_lo;
  Acc<T> acc[VEC];
  int p = rs;
  if (col_full) {
    for (; p + kUnroll <= re; p += kUnroll) {
      T v[kUnroll];
      int c[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        v[u] = val_at(p + u);
        c[u] = ld_keep(a.col_idx + p + u, pol_stream);
      }
      Vec<T, VEC> xv[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) xv[u] = ld_keep_vec<T, VEC>(Xc + (long long)c[u] * a.ldx, pol_keep);
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int j = 0; j < VEC; ++j) acc[j].add(v[u], xv[u].v[j]);
    }
    for (; p < re; ++p) {
      const T v = val_at(p);
      Vec<T, VEC> xv = ld_keep_vec<T, VEC>(Xc + (long long)ld_keep(a.col_idx + p, pol_stream) * a.ldx, pol_keep);
#pragma unroll
      for (int j = 0; j < VEC; ++j) acc[j].add(v, xv.v[j]);
    }
  } else {
    // ragged last column slice: scalar gathers of the valid columns
    const int nv = a.k - c_lo;
    for (; p < re; ++p) {
      const T v = val_at(p);
      const T* xr = Xc + (long long)ld_keep(a.col_idx + p, pol_stream) * a.ldx;
#pragma unroll
      for (int j = 0; j < VEC; ++j)
        if (j < nv) acc[j].add(v, ld_keep(xr + j, pol_keep));
    }
  }
  T out[VEC];
#pragma unroll
  for (int j = 0; j < VEC; ++j) out[j] = acc[j].value();
  T* yr = a.Y + (long long)r * a.ldy + c_lo;
  if (col_full)
    st_stream_vec<T, VEC>(yr, out);
  else
    for (int j = 0; j < a.k - c_lo; ++j) st_stream(yr + j, out[j]);
}

template <typename T, int VEC, int LANES, bool PERM = false>
__global__ void __launch_bounds__(1024) rows_direct_kernel(RowsArgs<T> a) {
  rows_direct_block<T, VEC, LANES, PERM>(a, blockIdx.x);
}

}  // namespace gbs
