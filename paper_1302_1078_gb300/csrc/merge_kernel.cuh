// Merge-path CSR kernel ("MERGE" variant) for SpMV and SpMM.
//
// Load balance for power-law rows, which the paper's one-row-per-thread
// kernel (Sec. 4.1) cannot give (webbase-1M has a 4700-nonzero row among
// 3-nonzero ones, Sec. 4 Table "tab:matrices").  The work is the merge of two
// sorted lists, the row ends row_ptr[1..m] and the nonzero positions
// 0..nnz-1 (Merrill & Garland, "Merge-based parallel sparse matrix-vector
// multiplication", SC'16): every thread takes the same number of items
// (row ends + nonzeros), whatever the row lengths.
//
// GB300-specific choices:
//   * The inner loop walks the thread's nonzeros and emits the rows that end
//     between them, so each nonzero costs one fused multiply-add per output
//     element and row ends cost no FP64 work (GB300's FP64 pipe is the
//     scarce resource; a masked FP64 instruction costs as much as a full one).
//   * A row split across threads is finished by the thread where it ends.
//     The carries of the threads before it arrive through a segmented
//     inclusive scan keyed by row (Hillis-Steele over the merge threads of a
//     warp, then a carry-in chain over the CTA's warps).  A scan step whose
//     additions no lane needs is skipped for the whole warp, so a tile of
//     short rows pays about one FP64 add per merge thread, and a hub row
//     spanning many threads pays a logarithmic number, not a walk.
//   * A row split across CTAs is finished by a separate fix-up pass over the
//     per-CTA carries, in CTA order.  No atomics: the result is bitwise
//     reproducible.
//   * A group of G lanes shares one merge thread; each lane owns VEC of the
//     k columns (SpMM), so the X row of a nonzero is gathered with G
//     coalesced 128-bit loads.
//   * Two ways to fetch the nonzeros (template DIRECT): the CTA stages the
//     tile's vals / col_idx in shared memory with coalesced loads (MERGE), or
//     each merge thread reads its own contiguous segment straight from
//     global memory in aligned 128-bit groups of four (MERGE_DIRECT).  The
//     direct form stages nothing: it reads the tile's row pointers through L1
//     as well and keeps the next row end in a register, so shared memory holds
//     only the carry scan's few KB and L1 keeps the rest of the SM's 256 KB
//     for the gathered x (on a power-law matrix the hot columns of x are what
//     L1 can hold, and more of them stay there the larger L1 is).
//   * HOT (direct form, one column): the matrix's columns were relabelled
//     hottest first (relabel.cu), so the x entries below `hot_cols` are the
//     ones gathered most often.  Gathers of columns at or above it skip L1,
//     so that the rarely reused lines do not evict the hot head of x.
//   * PERM: the value of stored entry p is vals[perm[p]], so the backward
//     pass can run A^T on A's values without a permuted copy.  The staged
//     form gathers the tile's values into shared memory (perm read with
//     128-bit loads); the direct form gathers them in its walk.
#pragma once
#include "device_common.cuh"

namespace gbs {

// A 32-bit read that may hit L1 (the direct form's row pointers, which its searches re-read),
// with an L2 policy.
__device__ __forceinline__ int ld_l1_i32(const int* ptr, uint64_t pol) {
  int r;
  asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(r) : "l"(ptr), "l"(pol));
  return r;
}

template <typename T>
struct MergeArgs {
  int m, k, nnz;
  const int* __restrict__ row_ptr;
  const int* __restrict__ col_idx;
  const T* __restrict__ vals;
  const T* __restrict__ X;
  T* __restrict__ Y;
  long long ldx, ldy;
  int items;             // merge items per merge thread
  int ctas;              // number of CTA tiles
  const int2* __restrict__ coords;  // [ctas + 1] (row, nonzero) at the start of each tile
  int* __restrict__ carry_row;      // [ctas]
  T* __restrict__ carry_val;        // [ctas * k]
  bool aligned_vals, aligned_cols;  // aligned_vals: perm when PERM
  bool vals32 = false;              // vals 32-byte aligned: a group of four doubles is one 256-bit load
  const int* __restrict__ perm = nullptr;  // PERM: value of entry p is vals[perm[p]]
  int hot_cols = 0x7fffffff;               // HOT: columns below this are gathered through L1
};

// Merge-path search: split diagonal d of the (row ends x nonzeros) grid.
// Returns (i, d - i): i row ends and d - i nonzeros precede the split.
// A row end that equals a nonzero position is taken first (that nonzero
// belongs to a later row).
__device__ __forceinline__ int2 merge_search_global(const int* __restrict__ row_ptr, int m, int nnz, long long d) {
  long long lo = d - nnz > 0 ? d - nnz : 0;
  long long hi = d < m ? d : m;
  while (lo < hi) {
    long long mid = (lo + hi) >> 1;
    if ((long long)__ldg(row_ptr + mid + 1) <= d - 1 - mid)
      lo = mid + 1;
    else
      hi = mid;
  }
  return make_int2((int)lo, (int)(d - lo));
}

template <typename T, int VEC, int G, bool DIRECT = false>
__host__ __device__ inline size_t merge_smem_bytes(int threads, int items) {
  int nt = threads / G;
  size_t ipc = (size_t)nt * items;
  size_t a = DIRECT ? 0 : ((ipc + 2) * sizeof(int) + 15) & ~(size_t)15;  // s_rp
  size_t b = DIRECT ? 0 : ((ipc + 4) * sizeof(T) + 15) & ~(size_t)15;  // s_val
  size_t c = DIRECT ? 0 : ((ipc + 4) * sizeof(int) + 15) & ~(size_t)15;  // s_col
  size_t d = 2 * (size_t)(threads / 32) * sizeof(int);               // s_wkey, s_cinkey (per warp)
  size_t e = 2 * (size_t)(threads / 32) * G * VEC * sizeof(T);       // s_wval, s_cinval (per warp: G lanes x VEC)
  return a + b + c + d + e;
}

// One merge-path tile b of the product (the whole CTA works on it).  Used by the
// standalone kernel below and by the batched persistent kernel.
template <typename T, int VEC, int G, bool DIRECT = false, bool PERM = false, bool HOT = false, bool K1 = false>
__device__ __forceinline__ void merge_tile(const MergeArgs<T>& a, int b) {
  static_assert(!HOT || (DIRECT && VEC == 1), "the hot-column policy is for the direct form's scalar gathers");
  static_assert(!K1 || (VEC == 1 && G == 1), "the SpMV form has one column and one lane per merge thread");
  // K1: SpMV (k == 1) with contiguous x and y, so their strides drop out of every address
  const int kk = K1 ? 1 : a.k;
  const long long ldx = K1 ? 1 : a.ldx, ldy = K1 ? 1 : a.ldy;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nt = blockDim.x / G;
  const int nw = blockDim.x / 32;
  const int ipc = nt * a.items;
  const int2 cs = a.coords[b], ce = a.coords[b + 1];
  const int row0 = cs.x, nz0 = cs.y, row1 = ce.x, nz1 = ce.y;
  const long long d0 = (long long)row0 + nz0;
  const int span = (int)((long long)row1 + nz1 - d0);  // items in this tile

  int* s_rp = reinterpret_cast<int*>(smem_raw);
  size_t off = DIRECT ? 0 : (((size_t)ipc + 2) * sizeof(int) + 15) & ~(size_t)15;
  T* s_val = reinterpret_cast<T*>(smem_raw + off);
  if (!DIRECT) off += (((size_t)ipc + 4) * sizeof(T) + 15) & ~(size_t)15;
  int* s_col = reinterpret_cast<int*>(smem_raw + off);
  if (!DIRECT) off += (((size_t)ipc + 4) * sizeof(int) + 15) & ~(size_t)15;
  int* s_wkey = reinterpret_cast<int*>(smem_raw + off);  // [nw]
  int* s_cinkey = s_wkey + nw;                            // [nw]
  off += 2 * (size_t)nw * sizeof(int);
  T* s_wval = reinterpret_cast<T*>(smem_raw + off);      // [nw][G * VEC]
  T* s_cinval = s_wval + (size_t)nw * G * VEC;           // [nw][G * VEC]

  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_keep = policy_evict_last();

  // row_ptr window rp(q) = row_ptr[row0 + q], q in [0, row1 - row0]: staged in shared memory
  // (rows row0 .. min(row1, m-1) plus the last one's end), or read through L1 (DIRECT)
  const int a0 = nz0 & ~3;
  if constexpr (!DIRECT) {
    const int rlast = min(row1, a.m - 1);
    const int nrp = rlast >= row0 ? rlast - row0 + 2 : 0;
    for (int q = threadIdx.x; q < nrp; q += blockDim.x) s_rp[q] = ld_stream(a.row_ptr + row0 + q, pol_stream);
    if (nz1 > nz0) {
      if constexpr (PERM)
        stage_gather<T>(s_val, a.vals, a.perm, a0, nz1, a.aligned_vals, pol_stream);
      else
        stage_copy<T>(s_val, a.vals, a0, nz1, a.aligned_vals, pol_stream);
      stage_copy<int>(s_col, a.col_idx, a0, nz1, a.aligned_cols, pol_stream);
    }
    __syncthreads();
  }
  auto rp = [&](int q) -> int {
    if constexpr (DIRECT)
      return ld_l1_i32(a.row_ptr + row0 + q, pol_stream);
    else
      return s_rp[q];
  };

  const int t = threadIdx.x / G;            // merge thread
  const int lane = threadIdx.x % G;         // column lane inside the merge thread
  const int wl = threadIdx.x & 31;          // lane in warp
  const int w = threadIdx.x >> 5;           // warp
  constexpr int MT = 32 / G;                // merge threads per warp
  const int mt = wl / G;                    // merge thread inside the warp
  const int c_lo = lane * VEC;
  const bool col_active = c_lo < kk;
  const bool col_full = c_lo + VEC <= kk;

  // this merge thread's share of the tile: diagonals [ds, de) relative to d0, each located by a
  // binary search of the window; the two searches step together so their reads overlap
  const int ds = min(t * a.items, span), de = min(ds + a.items, span);
  const int wrows = row1 - row0, wnz = nz1 - nz0;
  int ri_s = max(0, ds - wnz), hi_s = min(ds, wrows);
  int ri_e = max(0, de - wnz), hi_e = min(de, wrows);
  while (ri_s < hi_s || ri_e < hi_e) {
    const int ms = (ri_s + hi_s) >> 1, me = (ri_e + hi_e) >> 1;
    const int vs = rp(min(ms + 1, wrows)), ve = rp(min(me + 1, wrows));
    if (ri_s < hi_s) {
      if (vs <= nz0 + ds - 1 - ms)
        ri_s = ms + 1;
      else
        hi_s = ms;
    }
    if (ri_e < hi_e) {
      if (ve <= nz0 + de - 1 - me)
        ri_e = me + 1;
      else
        hi_e = me;
    }
  }
  const int row_s = row0 + ri_s, nz_s = nz0 + ds - ri_s;
  const int row_e = row0 + ri_e, nz_e = nz0 + de - ri_e;

  // the thread's first row started before its first nonzero: earlier threads hold its start
  const bool head_partial = (row_s < a.m) && (nz_s > rp(ri_s));

  Acc<T> acc[VEC];
  T head[VEC];
  int head_row = -1;
  bool first = true;
  int row = row_s;
  const T* __restrict__ Xc = a.X + c_lo;

  auto store_row = [&](int r, const T* out) {
    T* yr = a.Y + (long long)r * ldy + c_lo;
    if (col_full)
      st_stream_vec<T, VEC>(yr, out);
    else
      for (int j = 0; j < kk - c_lo; ++j) st_stream(yr + j, out[j]);
  };
  auto emit = [&](int r) {
    T out[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) out[j] = acc[j].value();
    if (first && head_partial) {
#pragma unroll
      for (int j = 0; j < VEC; ++j) head[j] = out[j];
      head_row = r;
    } else if (col_active) {
      store_row(r, out);
    }
    first = false;
#pragma unroll
    for (int j = 0; j < VEC; ++j) acc[j].reset();
  };

  if constexpr (DIRECT) {
    // each merge thread streams its own contiguous segment [nz_s, nz_e) from global memory:
    // scalar up to a multiple of 4, then aligned 128-bit groups of four, then the tail
    auto gather = [&](int c) {
      Vec<T, VEC> xv;
      if constexpr (HOT) {
        xv.v[0] = c < a.hot_cols ? ld_keep(Xc + (long long)c * ldx, pol_keep)
                                 : ld_keep_na(Xc + (long long)c * ldx, pol_keep);
      } else if (col_full) {
        xv = ld_keep_vec<T, VEC>(Xc + (long long)c * ldx, pol_keep);
      } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) xv.v[j] = (c_lo + j < kk) ? ld_keep(Xc + (long long)c * ldx + j, pol_keep) : T(0);
      }
      return xv;
    };
    // end of the current row, row_ptr[row + 1]; past every nonzero once the thread's rows are emitted
    int rnext = row < row_e ? rp(row - row0 + 1) : 0x7fffffff;
    auto close_rows = [&](int q) {
      while (rnext <= q) {
        emit(row);
        ++row;
        rnext = row < row_e ? rp(row - row0 + 1) : 0x7fffffff;
      }
    };
    auto one = [&](int q) {
      T vv;
      if constexpr (PERM)
        vv = __ldg(a.vals + ld_stream(a.perm + q, pol_stream));
      else
        vv = ld_stream(a.vals + q, pol_stream);
      const int cc = ld_stream(a.col_idx + q, pol_stream);
      Vec<T, VEC> xv;
      if (col_active) xv = gather(cc);
      close_rows(q);
      if (col_active) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) acc[j].add(vv, xv.v[j]);
      }
    };
    int nz = nz_s;
    if (a.aligned_vals && a.aligned_cols) {
      // aligned groups of four from the one holding nz_s to the one holding nz_e - 1, each read
      // with vector loads; the entries of a group outside [nz_s, nz_e) belong to the neighbouring
      // threads and are skipped (a scalar read of a segment's ragged ends would cost an L2
      // request per 8-byte value and per 4-byte column id); only a group that runs past the end
      // of the arrays is read element by element
      // groups below vec_end lie wholly inside the arrays; the arrays' last partial group (only
      // the matrix's last merge thread reaches it) is read element by element after the loop
      const int vec_end = a.nnz & ~3;
      int g = nz_s & ~3;
      for (; g < nz_e && g < vec_end; g += 4) {
        T v[4];
        if constexpr (PERM) {
          const uint4 pw = ld_stream_l1_v4(a.perm + g, pol_stream);
          const int pq[4] = {(int)pw.x, (int)pw.y, (int)pw.z, (int)pw.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (g + u >= nz_s && g + u < nz_e) v[u] = __ldg(a.vals + pq[u]);
        } else if constexpr (sizeof(T) == 8) {
          if (a.vals32) {
            ld_stream_4d(reinterpret_cast<const double*>(a.vals + g), pol_stream, reinterpret_cast<double*>(v));
          } else {
            const uint4 w0 = ld_stream_l1_v4(a.vals + g, pol_stream);
            const uint4 w1 = ld_stream_l1_v4(a.vals + g + 2, pol_stream);
            v[0] = __hiloint2double((int)w0.y, (int)w0.x);
            v[1] = __hiloint2double((int)w0.w, (int)w0.z);
            v[2] = __hiloint2double((int)w1.y, (int)w1.x);
            v[3] = __hiloint2double((int)w1.w, (int)w1.z);
          }
        } else {
          const uint4 w = ld_stream_l1_v4(a.vals + g, pol_stream);
          v[0] = __uint_as_float(w.x);
          v[1] = __uint_as_float(w.y);
          v[2] = __uint_as_float(w.z);
          v[3] = __uint_as_float(w.w);
        }
        const uint4 cw = ld_stream_l1_v4(a.col_idx + g, pol_stream);
        const int c4[4] = {(int)cw.x, (int)cw.y, (int)cw.z, (int)cw.w};
        Vec<T, VEC> xv[4];
        if (col_active) {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (g + u >= nz_s && g + u < nz_e) xv[u] = gather(c4[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (g + u >= nz_s && g + u < nz_e) {
            close_rows(g + u);
            if (col_active) {
#pragma unroll
              for (int j = 0; j < VEC; ++j) acc[j].add(v[u], xv[u].v[j]);
            }
          }
        }
      }
      for (nz = max(g, nz_s); nz < nz_e; ++nz) one(nz);
      nz = nz_e;
    }
    for (; nz < nz_e; ++nz) one(nz);
  } else {
  constexpr int U = 4;
  for (int nz = nz_s; nz < nz_e; nz += U) {
    const int cnt = min(U, nz_e - nz);
    T v[U];
    Vec<T, VEC> xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (u < cnt && col_active) {
        v[u] = s_val[nz + u - a0];
        const int c = s_col[nz + u - a0];
        if (col_full) {
          xv[u] = ld_keep_vec<T, VEC>(Xc + (long long)c * ldx, pol_keep);
        } else {
#pragma unroll
          for (int j = 0; j < VEC; ++j) xv[u].v[j] = (c_lo + j < kk) ? ld_keep(Xc + (long long)c * ldx + j, pol_keep) : T(0);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (u < cnt) {
        while (row < row_e && s_rp[row - row0 + 1] <= nz + u) {
          emit(row);
          ++row;
        }
        if (col_active) {
#pragma unroll
          for (int j = 0; j < VEC; ++j) acc[j].add(v[u], xv[u].v[j]);
        }
      }
    }
  }
  }  // staged
  while (row < row_e) {
    emit(row);
    ++row;
  }

  // ---- carries: segmented inclusive scan over merge threads, keyed by the open row
  const int key = row_e;
  T S[VEC];
#pragma unroll
  for (int j = 0; j < VEC; ++j) S[j] = acc[j].value();
#pragma unroll
  for (int dd = 1; dd < MT; dd <<= 1) {
    const int okey = __shfl_up_sync(0xffffffffu, key, dd * G);
    T o[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) o[j] = __shfl_up_sync(0xffffffffu, S[j], dd * G);
    const bool take = mt >= dd && okey == key;
    if (__any_sync(0xffffffffu, take)) {
#pragma unroll
      for (int j = 0; j < VEC; ++j)
        if (take) S[j] += o[j];
    }
  }
  // warp summaries: key and run sum of each warp's last merge thread
  if (mt == MT - 1) {
    if (lane == 0) s_wkey[w] = key;
#pragma unroll
    for (int j = 0; j < VEC; ++j) s_wval[((size_t)w * G + lane) * VEC + j] = S[j];
  }
  __syncthreads();
  // carry into warp ww: the run of the previous warp's last key, chained over whole-warp runs
  if (threadIdx.x < G) {
    const int c = threadIdx.x;
    T cin[VEC];
    int cin_key = -1;
    for (int ww = 1; ww < nw; ++ww) {
      const int k_prev = s_wkey[ww - 1];
      T nv[VEC];
#pragma unroll
      for (int j = 0; j < VEC; ++j) nv[j] = s_wval[((size_t)(ww - 1) * G + c) * VEC + j];
      if (ww >= 2 && cin_key == k_prev) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) nv[j] += cin[j];
      }
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        cin[j] = nv[j];
        s_cinval[((size_t)ww * G + c) * VEC + j] = nv[j];
      }
      cin_key = k_prev;
      if (c == 0) s_cinkey[ww] = k_prev;
    }
    if (c == 0) s_cinkey[0] = -1;
  }
  __syncthreads();
  const int wkey = s_cinkey[w];
  {
    const bool take = w > 0 && key == wkey;
    if (__any_sync(0xffffffffu, take)) {
#pragma unroll
      for (int j = 0; j < VEC; ++j)
        if (take) S[j] += s_cinval[((size_t)w * G + lane) * VEC + j];
    }
  }
  // finish the split head row with the run that ends just before this merge thread
  {
    int pkey = __shfl_up_sync(0xffffffffu, key, G);
    T ps[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) ps[j] = __shfl_up_sync(0xffffffffu, S[j], G);
    if (mt == 0) {
      pkey = w > 0 ? wkey : -1;
#pragma unroll
      for (int j = 0; j < VEC; ++j) ps[j] = w > 0 ? s_cinval[((size_t)w * G + lane) * VEC + j] : T(0);
    }
    const bool take = head_row >= 0 && pkey == head_row;
    if (__any_sync(0xffffffffu, take)) {
#pragma unroll
      for (int j = 0; j < VEC; ++j)
        if (take) head[j] += ps[j];
    }
    if (head_row >= 0 && col_active) store_row(head_row, head);
  }
  if (t == nt - 1) {
    // CTA carry: run sum of the row still open at the tile's end
    if (lane == 0) a.carry_row[b] = key < a.m ? key : -1;
    if (col_active)
      for (int j = 0; j < VEC && c_lo + j < kk; ++j) a.carry_val[(size_t)b * kk + c_lo + j] = S[j];
  }
}

template <typename T, int VEC, int G, bool DIRECT, bool PERM = false, bool HOT = false>
__global__ void __launch_bounds__(256) merge_kernel(MergeArgs<T> a) {
  merge_tile<T, VEC, G, DIRECT, PERM, HOT>(a, blockIdx.x);
}

// The direct SpMV walk held to 40 registers (six resident 256-thread CTAs per SM, or twelve of
// 128 threads): the power-law products it serves wait on their gathers, and more warps in flight
// hide more of it.
template <typename T, bool PERM, bool HOT, bool K1>
__global__ void __launch_bounds__(256, 6) merge_direct6_kernel(MergeArgs<T> a) {
  merge_tile<T, 1, 1, true, PERM, HOT, K1>(a, blockIdx.x);
}

// Adds the CTA carries to the rows they belong to: the first CTA of each run of
// equal carry rows sums the run in CTA order and adds it to Y (row finished by a
// later CTA, which has already written its own part).  A hub row spans tens of
// tiles, so the run's end and its carries are read 8 tiles at a time with
// independent loads; the additions stay in CTA order.
template <typename T>
__device__ __forceinline__ void merge_fixup_one(int b, int ctas, int k, const int* __restrict__ carry_row,
                                                const T* __restrict__ carry_val, T* __restrict__ Y, long long ldy) {
  constexpr int W = 8;
  const int r = __ldcg(carry_row + b);
  if (r < 0) return;
  if (b > 0 && __ldcg(carry_row + b - 1) == r) return;
  int e = b + 1;  // the run is [b, e)
  for (;;) {
    int rr[W];
#pragma unroll
    for (int j = 0; j < W; ++j) rr[j] = e + j < ctas ? __ldcg(carry_row + e + j) : -2;
    int stop = W;
#pragma unroll
    for (int j = W - 1; j >= 0; --j)
      if (rr[j] != r) stop = j;
    e += stop;
    if (stop < W) break;
  }
  for (int c = 0; c < k; ++c) {
    Acc<T> s;
    for (int bb = b; bb < e; bb += W) {
      T v[W];
#pragma unroll
      for (int j = 0; j < W; ++j) v[j] = bb + j < e ? __ldcg(carry_val + (size_t)(bb + j) * k + c) : T(0);
#pragma unroll
      for (int j = 0; j < W; ++j)
        if (bb + j < e) s.add_partial(v[j]);
    }
    T* yp = Y + (long long)r * ldy + c;
    *yp = __ldcg(yp) + s.value();
  }
}

// The standalone fix-up: one thread per tile, as merge_fixup_one, except for runs longer than 8
// tiles (a hub row; on R-MAT 22 one row spans 85 tiles), which the thread's warp takes over: the
// run's end is found 32 tiles per step by a ballot, and its carries are loaded 32 at a time by
// the lanes and added in tile order from shuffles.  The additions are merge_fixup_one's, in the
// same order (so the batched kernel's fix-up gives the same bits); only the chain of dependent
// loads is shortened.
template <typename T>
__global__ void merge_fixup_kernel(int ctas, int k, const int* __restrict__ carry_row, const T* __restrict__ carry_val,
                                   T* __restrict__ Y, long long ldy) {
  constexpr int W = 8;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int r = -1;
  bool start = false;
  if (b < ctas) {
    r = __ldcg(carry_row + b);
    start = r >= 0 && !(b > 0 && __ldcg(carry_row + b - 1) == r);
  }
  // a run of at most W tiles is summed by its own thread
  bool longrun = false;
  if (start) {
    int rr[W];
#pragma unroll
    for (int j = 0; j < W; ++j) rr[j] = b + 1 + j < ctas ? __ldcg(carry_row + b + 1 + j) : -2;
    bool ends = false;
#pragma unroll
    for (int j = 0; j < W; ++j) ends = ends || rr[j] != r;
    if (ends)
      merge_fixup_one<T>(b, ctas, k, carry_row, carry_val, Y, ldy);
    else
      longrun = true;
  }
  unsigned m = __ballot_sync(0xffffffffu, longrun);
  while (m) {
    const int src = __ffs(m) - 1;
    m &= m - 1;
    const int rb = __shfl_sync(0xffffffffu, b, src), rr = __shfl_sync(0xffffffffu, r, src);
    int re = ctas;  // the run is [rb, re)
    for (int base = rb + 1; base < ctas; base += 32) {
      const int t = base + lane;
      const unsigned dm = __ballot_sync(0xffffffffu, t >= ctas || __ldcg(carry_row + t) != rr);
      if (dm) {
        re = base + __ffs(dm) - 1;
        break;
      }
    }
    for (int c = 0; c < k; ++c) {
      Acc<T> acc;
      for (int base = rb; base < re; base += 32) {
        const T v = base + lane < re ? __ldcg(carry_val + (size_t)(base + lane) * k + c) : T(0);
        const int cnt = min(32, re - base);
        for (int j = 0; j < cnt; ++j) acc.add_partial(__shfl_sync(0xffffffffu, v, j));
      }
      if (lane == 0) {
        T* yp = Y + (long long)rr * ldy + c;
        *yp = __ldcg(yp) + acc.value();
      }
    }
  }
}

}  // namespace gbs
