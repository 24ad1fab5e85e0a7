// Template launchers behind launch.h, instantiated once per dtype in
// kernels_f64.cu / kernels_f32.cu so that the two compile in parallel.
#pragma once
#include <algorithm>
#include <atomic>
#include <mutex>

#include "launch.h"
#include "merge_kernel.cuh"
#include "rows_kernel.cuh"
#include "rows_tma.cuh"

namespace gbs {

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// The SM's 256 KB of unified storage is split between shared memory and L1.  Left to itself the
// CUDA driver sizes the shared part for the 32 CTAs an SM can hold at most (64 KB for the direct merge
// walk, which uses a few hundred bytes per CTA), and what it takes is lost to L1, where these
// kernels' gathers of x hit.  The carveout attribute is only a hint, and the CUDA driver maps it to a
// configuration in its own way; measured on GB300 (one probe kernel, ncu's
// launch__shared_mem_config_size): hint 0 gives 8 KB, 1 gives 16 KB, 2 and 3 give 32 KB, 4 to 7
// the default 64 KB, and the CUDA driver keeps the small ones even where they limit occupancy.
// prefer_l1 therefore picks the smallest of 8, 16 and 32 KB that holds every CTA that can be
// resident: an upper bound on that count from the thread, block and register limits (register
// allocation rounded to 256 per warp), times the CTA's dynamic shared memory (rounded up to 256
// bytes) plus the 1 KB the system reserves per CTA; above 32 KB it leaves the CUDA driver's default.
// The bound can only over-count, so the split never limits occupancy.  The device's limits are
// read once per process (the library serves one kind of GPU); each kernel keeps its register
// count and the hint it last set on which device, so a repeated launch makes no extra runtime call.
struct SmLimits {
  int reserved = 0, thr_sm = 0, blk_sm = 0, regs_sm = 0;
};
// The current device's limits, read once per process and kept only once they were read (a
// failed query is returned and retried at the next launch).
static cudaError_t sm_limits(SmLimits* out) {
  static std::atomic<bool> ready{false};
  static SmLimits cached;
  static std::mutex mu;
  if (ready.load(std::memory_order_acquire)) {
    *out = cached;
    return cudaSuccess;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!ready.load(std::memory_order_relaxed)) {
    SmLimits l;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l.reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l.thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l.blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l.regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e != cudaSuccess) return e;
    cached = l;
    ready.store(true, std::memory_order_release);
  }
  *out = cached;
  return cudaSuccess;
}

struct L1Split {
  std::atomic<int> regs{0};
  std::atomic<int> last{-1};  // (device << 8) | (hint & 0xff) last set
};

template <typename K>
static cudaError_t prefer_l1(K kernel, int threads, size_t smem, L1Split& st) {
  SmLimits l;
  cudaError_t e = sm_limits(&l);
  if (e != cudaSuccess) return e;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int r = st.regs.load(std::memory_order_relaxed);
  if (r <= 0) {
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kernel)) != cudaSuccess) return e;
    r = fa.numRegs > 0 ? fa.numRegs : 1;
    st.regs.store(r, std::memory_order_relaxed);
  }
  const int warps = (threads + 31) / 32;
  const long long per_warp = ((long long)r * 32 + 255) / 256 * 256;
  long long ctas = std::min<long long>(l.thr_sm / threads, l.blk_sm);
  ctas = std::min<long long>(ctas, l.regs_sm / (per_warp * warps));
  ctas = std::max<long long>(ctas, 1);
  const long long need = ctas * ((((long long)smem + 255) & ~255LL) + l.reserved);  // 256-byte allocation units
  const int pct = need <= 8 * 1024 ? 0 : need <= 16 * 1024 ? 1 : need <= 32 * 1024 ? 2 : (int)cudaSharedmemCarveoutDefault;
  const int tag = (dev << 8) | (pct & 0xff);
  if (st.last.load(std::memory_order_relaxed) == tag) return cudaSuccess;
  if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct)) != cudaSuccess) return e;
  st.last.store(tag, std::memory_order_relaxed);
  return cudaSuccess;
}

template <typename T, int VEC, int LANES, bool SPLIT, bool PERM>
static cudaError_t rows_go(const RowsArgs<T>& a, int grid, int threads, size_t smem, cudaStream_t s) {
  auto kern = rows_kernel<T, VEC, LANES, SPLIT, PERM>;
  static L1Split split;
  cudaError_t e = set_smem(kern, smem);
  if (e == cudaSuccess) e = prefer_l1(kern, threads, smem, split);
  if (e != cudaSuccess) return e;
  kern<<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int LANES, bool PERM>
static cudaError_t rows_lanes(const RowsArgs<T>& a, bool split, bool vec16, int grid, int threads, size_t smem,
                              cudaStream_t s) {
  constexpr int V = 16 / (int)sizeof(T);
  if (split) return rows_go<T, 1, LANES, true, PERM>(a, grid, threads, smem, s);
  if (vec16) return rows_go<T, V, LANES, false, PERM>(a, grid, threads, smem, s);
  return rows_go<T, 1, LANES, false, PERM>(a, grid, threads, smem, s);
}

// PERM: A.perm is set and the value of entry p is A.vals[A.perm[p]].
template <typename T, bool PERM = false>
cudaError_t launch_rows_t(const CsrView& A, const DenseView& D, int lanes, bool vec16, int threads, int tile,
                          int row_base, int rows, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  RowsArgs<T> a;
  a.m = row_base + rows;
  a.k = D.k;
  a.row_ptr = A.row_ptr;
  a.col_idx = A.col_idx;
  a.vals = static_cast<const T*>(A.vals);
  a.X = static_cast<const T*>(D.X);
  a.Y = static_cast<T*>(D.Y);
  a.ldx = D.ldx;
  a.ldy = D.ldy;
  a.tile = tile;
  a.row_base = row_base;
  a.perm = PERM ? A.perm : nullptr;
  a.aligned_vals = (reinterpret_cast<uintptr_t>(PERM ? static_cast<const void*>(A.perm) : A.vals) & 15) == 0;
  a.aligned_cols = (reinterpret_cast<uintptr_t>(A.col_idx) & 15) == 0;
  const int rpc = threads / lanes;
  const int grid = (rows + rpc - 1) / rpc;
  const size_t smem = rows_smem_bytes<T>(rpc, tile);
  const bool split = D.k == 1;
  switch (lanes) {
    case 1: return rows_lanes<T, 1, PERM>(a, split, vec16, grid, threads, smem, s);
    case 2: return rows_lanes<T, 2, PERM>(a, split, vec16, grid, threads, smem, s);
    case 4: return rows_lanes<T, 4, PERM>(a, split, vec16, grid, threads, smem, s);
    case 8: return rows_lanes<T, 8, PERM>(a, split, vec16, grid, threads, smem, s);
    case 16: return rows_lanes<T, 16, PERM>(a, split, vec16, grid, threads, smem, s);
    case 32: return rows_lanes<T, 32, PERM>(a, split, vec16, grid, threads, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int VEC, int LANES>
static cudaError_t rows_direct_go(const RowsArgs<T>& a, int grid, int threads, cudaStream_t s) {
  static L1Split split;
  const cudaError_t e = prefer_l1(rows_direct_kernel<T, VEC, LANES>, threads, 0, split);
  if (e != cudaSuccess) return e;
  rows_direct_kernel<T, VEC, LANES><<<grid, threads, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int LANES>
static cudaError_t rows_direct_lanes(const RowsArgs<T>& a, bool vec16, int grid, int threads, cudaStream_t s) {
  constexpr int V = 16 / (int)sizeof(T);
  if (vec16) return rows_direct_go<T, V, LANES>(a, grid, threads, s);
  return rows_direct_go<T, 1, LANES>(a, grid, threads, s);
}

// ROWS_DIRECT (rows_direct_block): k == 1 runs one lane per row whatever `lanes` says.
template <typename T>
cudaError_t launch_rows_direct_t(const CsrView& A, const DenseView& D, int lanes, bool vec16, int threads,
                                 cudaStream_t s) {
  if (A.m <= 0) return cudaSuccess;
  RowsArgs<T> a;
  a.m = A.m;
  a.k = D.k;
  a.row_ptr = A.row_ptr;
  a.col_idx = A.col_idx;
  a.vals = static_cast<const T*>(A.vals);
  a.X = static_cast<const T*>(D.X);
  a.Y = static_cast<T*>(D.Y);
  a.ldx = D.ldx;
  a.ldy = D.ldy;
  a.tile = 0;
  a.row_base = 0;
  a.aligned_vals = false;
  a.aligned_cols = false;
  if (D.k == 1) lanes = 1;
  const int rpc = threads / lanes;
  const int grid = (A.m + rpc - 1) / rpc;
  switch (lanes) {
    case 1: return rows_direct_lanes<T, 1>(a, vec16 && D.k > 1, grid, threads, s);
    case 2: return rows_direct_lanes<T, 2>(a, vec16, grid, threads, s);
    case 4: return rows_direct_lanes<T, 4>(a, vec16, grid, threads, s);
    case 8: return rows_direct_lanes<T, 8>(a, vec16, grid, threads, s);
    case 16: return rows_direct_lanes<T, 16>(a, vec16, grid, threads, s);
    case 32: return rows_direct_lanes<T, 32>(a, vec16, grid, threads, s);
    default: return cudaErrorInvalidValue;
  }
}

// The persistent grid (resident CTAs per SM x SMs) and the shared-memory attribute are worked out
// once per kernel, block size and shared-memory size on a device and kept, so that a repeated
// launch makes no runtime query between the caller's events and the kernel.
struct GridCache {
  std::atomic<long long> key{-1};  // (device << 48) | (threads << 32) | smem
  std::atomic<int> grid_cap{0};    // resident CTAs per SM x SMs
};

template <typename K>
static cudaError_t persistent_cap(K kern, int threads, size_t smem, GridCache& gc, int* cap) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const long long key = ((long long)dev << 48) | ((long long)threads << 32) | (long long)smem;
  if (gc.key.load(std::memory_order_acquire) == key) {
    *cap = gc.grid_cap.load(std::memory_order_relaxed);
    return cudaSuccess;
  }
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
  int bps = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, threads, smem)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (bps < 1) return cudaErrorInvalidConfiguration;
  *cap = bps * sms;
  gc.grid_cap.store(*cap, std::memory_order_relaxed);
  gc.key.store(key, std::memory_order_release);
  return cudaSuccess;
}

template <typename T, int VEC, int LANES, bool SPLIT, int EMUL, bool UNIT = false>
static cudaError_t rows_tma_go(const RowsArgs<T>& a, int nblocks, int nnz, int* status, int threads, size_t smem,
                               cudaStream_t s) {
  auto kern = rows_tma_kernel<T, VEC, LANES, SPLIT, EMUL, UNIT>;
  static GridCache gc;
  int cap = 0;
  const cudaError_t e = persistent_cap(kern, threads, smem, gc, &cap);
  if (e != cudaSuccess) return e;
  const int grid = std::min(nblocks, cap);
  kern<<<grid, threads, smem, s>>>(a, nblocks, nnz, status);
  return cudaGetLastError();
}

template <typename T, int VEC, int LANES, bool SPLIT>
static cudaError_t rows_tma_emul(const RowsArgs<T>& a, int emul, int nblocks, int nnz, int* status, int threads,
                                 size_t smem, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    switch (emul) {
      case 1: return rows_tma_go<T, VEC, LANES, SPLIT, 1>(a, nblocks, nnz, status, threads, smem, s);
      case 2: return rows_tma_go<T, VEC, LANES, SPLIT, 2>(a, nblocks, nnz, status, threads, smem, s);
      case 3: return rows_tma_go<T, VEC, LANES, SPLIT, 3>(a, nblocks, nnz, status, threads, smem, s);
      default: break;
    }
  }
  if constexpr (SPLIT && VEC == 1)
    if (a.ldx == 1 && a.ldy == 1) return rows_tma_go<T, 1, LANES, true, 0, true>(a, nblocks, nnz, status, threads, smem, s);
  return rows_tma_go<T, VEC, LANES, SPLIT, 0>(a, nblocks, nnz, status, threads, smem, s);
}

template <typename T, int LANES>
static cudaError_t rows_tma_lanes(const RowsArgs<T>& a, bool split, bool vec16, int emul, int nblocks, int nnz,
                                  int* status, int threads, size_t smem, cudaStream_t s) {
  constexpr int V = 16 / (int)sizeof(T);
  if (split) return rows_tma_emul<T, 1, LANES, true>(a, emul, nblocks, nnz, status, threads, smem, s);
  if (vec16) return rows_tma_emul<T, V, LANES, false>(a, emul, nblocks, nnz, status, threads, smem, s);
  return rows_tma_emul<T, 1, LANES, false>(a, emul, nblocks, nnz, status, threads, smem, s);
}

template <typename T>
cudaError_t launch_rows_tma_t(const CsrView& A, const DenseView& D, int lanes, bool vec16, int threads, int tile,
                              int emul, int* status, cudaStream_t s) {
  if (A.m <= 0) return cudaSuccess;
  RowsArgs<T> a;
  a.m = A.m;
  a.k = D.k;
  a.row_ptr = A.row_ptr;
  a.col_idx = A.col_idx;
  a.vals = static_cast<const T*>(A.vals);
  a.X = static_cast<const T*>(D.X);
  a.Y = static_cast<T*>(D.Y);
  a.ldx = D.ldx;
  a.ldy = D.ldy;
  a.tile = tile;
  a.row_base = 0;
  a.aligned_vals = true;
  a.aligned_cols = true;
  const int rpc = threads / lanes;
  const int nblocks = (A.m + rpc - 1) / rpc;
  const size_t smem = rows_tma_smem_bytes<T>(rpc, tile);
  const bool split = D.k == 1;
  switch (lanes) {
    case 1: return rows_tma_lanes<T, 1>(a, split, vec16, emul, nblocks, A.nnz, status, threads, smem, s);
    case 2: return rows_tma_lanes<T, 2>(a, split, vec16, emul, nblocks, A.nnz, status, threads, smem, s);
    case 4: return rows_tma_lanes<T, 4>(a, split, vec16, emul, nblocks, A.nnz, status, threads, smem, s);
    case 8: return rows_tma_lanes<T, 8>(a, split, vec16, emul, nblocks, A.nnz, status, threads, smem, s);
    case 16: return rows_tma_lanes<T, 16>(a, split, vec16, emul, nblocks, A.nnz, status, threads, smem, s);
    case 32: return rows_tma_lanes<T, 32>(a, split, vec16, emul, nblocks, A.nnz, status, threads, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int VEC, int G, bool DIRECT, bool PERM, bool HOT = false>
static cudaError_t merge_go(const MergeArgs<T>& a, int threads, cudaStream_t s) {
  auto kern = merge_kernel<T, VEC, G, DIRECT, PERM, HOT>;
  static L1Split split, split_k1;
  bool k1 = false;
  if constexpr (DIRECT && VEC == 1 && G == 1) {  // 40 registers; its own form for SpMV with contiguous x, y
    k1 = a.k == 1 && a.ldx == 1 && a.ldy == 1;
    kern = k1 ? merge_direct6_kernel<T, PERM, HOT, true> : merge_direct6_kernel<T, PERM, HOT, false>;
  }
  const size_t smem = merge_smem_bytes<T, VEC, G, DIRECT>(threads, a.items);
  cudaError_t e = set_smem(kern, smem);
  if (e == cudaSuccess) e = prefer_l1(kern, threads, smem, k1 ? split_k1 : split);
  if (e != cudaSuccess) return e;
  kern<<<a.ctas, threads, smem, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  merge_fixup_kernel<T><<<(a.ctas + 255) / 256, 256, 0, s>>>(a.ctas, a.k, a.carry_row, a.carry_val, a.Y, a.ldy);
  return cudaGetLastError();
}

template <typename T, int G, bool PERM>
static cudaError_t merge_g(const MergeArgs<T>& a, bool vec16, bool direct, int threads, cudaStream_t s) {
  constexpr int V = 16 / (int)sizeof(T);
  if (direct) {
    if (vec16 && a.k > 1) return merge_go<T, V, G, true, PERM>(a, threads, s);
    if constexpr (G == 1) {
      if (a.hot_cols < 0x7fffffff) return merge_go<T, 1, 1, true, PERM, true>(a, threads, s);
    }
    return merge_go<T, 1, G, true, PERM>(a, threads, s);
  }
  if (vec16 && a.k > 1) return merge_go<T, V, G, false, PERM>(a, threads, s);
  return merge_go<T, 1, G, false, PERM>(a, threads, s);
}

// PERM: A.perm is set and the value of entry p is A.vals[A.perm[p]].
template <typename T, bool PERM = false>
cudaError_t launch_merge_t(const CsrView& A, const DenseView& D, int g, bool vec16, bool direct, int threads,
                           int items, const MergeScratch& S, cudaStream_t s) {
  if (A.m == 0) return cudaSuccess;
  MergeArgs<T> a;
  a.m = A.m;
  a.k = D.k;
  a.nnz = A.nnz;
  a.row_ptr = A.row_ptr;
  a.col_idx = A.col_idx;
  a.vals = static_cast<const T*>(A.vals);
  a.X = static_cast<const T*>(D.X);
  a.Y = static_cast<T*>(D.Y);
  a.ldx = D.ldx;
  a.ldy = D.ldy;
  a.items = items;
  a.ctas = S.ctas;
  a.coords = S.coords;
  a.carry_row = S.carry_row;
  a.carry_val = static_cast<T*>(S.carry_val);
  a.perm = PERM ? A.perm : nullptr;
  a.aligned_vals = (reinterpret_cast<uintptr_t>(PERM ? static_cast<const void*>(A.perm) : A.vals) & 15) == 0;
  a.aligned_cols = (reinterpret_cast<uintptr_t>(A.col_idx) & 15) == 0;
  a.vals32 = !PERM && (reinterpret_cast<uintptr_t>(A.vals) & 31) == 0;
  a.hot_cols = A.hot_cols > 0 ? A.hot_cols : 0x7fffffff;
  switch (g) {
    case 1: return merge_g<T, 1, PERM>(a, vec16, direct, threads, s);
    case 2: return merge_g<T, 2, PERM>(a, vec16, direct, threads, s);
    case 4: return merge_g<T, 4, PERM>(a, vec16, direct, threads, s);
    case 8: return merge_g<T, 8, PERM>(a, vec16, direct, threads, s);
    case 16: return merge_g<T, 16, PERM>(a, vec16, direct, threads, s);
    case 32: return merge_g<T, 32, PERM>(a, vec16, direct, threads, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
size_t merge_smem_t(int g, bool vec16, bool direct, int threads, int items) {
  constexpr int V = 16 / (int)sizeof(T);
  const int vec = vec16 ? V : 1;
  // same formula for every G: s_cval holds threads * vec elements
  const int nt = threads / g;
  const size_t ipc = (size_t)nt * items;
  size_t a = ((ipc + 2) * sizeof(int) + 15) & ~(size_t)15;
  size_t b = direct ? 0 : ((ipc + 4) * sizeof(T) + 15) & ~(size_t)15;
  size_t c = direct ? 0 : ((ipc + 4) * sizeof(int) + 15) & ~(size_t)15;
  size_t d = 2 * 32 * sizeof(int);
  size_t e = 2 * (size_t)threads * vec * sizeof(T);
  return a + b + c + d + e;
}

}  // namespace gbs
