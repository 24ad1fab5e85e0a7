// C-ABI entry points of gbspmv (declared in include/gbspmv.h): argument
// checks, configuration choice, plans, the autotuner, CSR statistics and
// validation.  Every product runs in the kernels of rows_kernel.cuh and
// merge_kernel.cuh; nothing here computes on the host.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "batched.cuh"
#include "gbspmv.h"
#include "launch.h"
#include "merge_kernel.cuh"
#include "rows_kernel.cuh"
#include "rows_tma.cuh"

using namespace gbs;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return GBS_ECUDA;
}

bool valid_dtype(int d) { return d == GBS_F64 || d == GBS_F32; }
bool is_merge(int v) { return v == GBS_VARIANT_MERGE || v == GBS_VARIANT_MERGE_DIRECT; }
size_t dsize(int d) { return d == GBS_F64 ? 8 : 4; }
int vec_of(int d) { return d == GBS_F64 ? 2 : 4; }
bool pow2_lanes(int l) { return l == 1 || l == 2 || l == 4 || l == 8 || l == 16 || l == 32; }
int pow2ceil(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

constexpr long long kMaxRowsPlusNnz = 0x7fffffffLL - 4096;

int check_csr(int m, int n, int nnz, const int* rp, const int* ci, const void* vals) {
  if (m < 0 || n < 0 || nnz < 0) return fail(GBS_EINVAL, "negative size");
  if (m > 0 && rp == nullptr) return fail(GBS_EINVAL, "row_ptr is NULL");
  if (nnz > 0 && (ci == nullptr || vals == nullptr)) return fail(GBS_EINVAL, "col_idx or vals is NULL");
  // 32-bit positions with headroom: the kernels round nonzero ranges out to 4-element groups
  // and step a few groups past a position before comparing it with the range's end
  if ((long long)m + nnz > kMaxRowsPlusNnz) return fail(GBS_EUNSUPPORTED, "m + nnz must be at most 2^31 - 4097");
  return GBS_OK;
}

bool tune_log() {
  const char* e = std::getenv("GBSPMV_TUNE_LOG");
  return e && e[0] && e[0] != '0';
}

bool checked_mode() {
  const char* e = std::getenv("GBSPMV_CHECKED");
  return e && e[0] && e[0] != '0';
}

// Columns handled by one launch: 32 lanes x VEC (128-bit) or 32 lanes x 1.
int panel_cols(int dtype, bool vec16) { return 32 * (vec16 ? vec_of(dtype) : 1); }

// Lanes that cover kp columns.
int col_lanes(int kp, int dtype, bool vec16) {
  int v = vec16 ? vec_of(dtype) : 1;
  return std::min(32, pow2ceil((kp + v - 1) / v));
}

bool dense_vec16(int dtype, int k, const void* X, long long ldx, const void* Y, long long ldy) {
  if (k <= 1) return false;
  const size_t es = dsize(dtype);
  return aligned16(X) && aligned16(Y) && ((ldx * (long long)es) % 16 == 0) && ((ldy * (long long)es) % 16 == 0);
}

// Items per merge thread: about 3840 items per CTA, an odd count so that the merge threads'
// contiguous segments in shared memory start in different banks.
int default_items(int g, int threads) {
  int it = std::max(5, (3840 * g) / threads);
  if (it % 2 == 0) --it;
  return std::min(it, 255);
}

gbs_config normalize(const gbs_config& c, int dtype) {
  gbs_config r = c;
  if (r.threads <= 0) r.threads = 256;
  if (r.variant == GBS_VARIANT_ROWS_DIRECT && r.lanes <= 0) r.lanes = 1;
  if (r.variant == GBS_VARIANT_ROWS || r.variant == GBS_VARIANT_ROWS_TMA) {
    if (r.lanes <= 0) r.lanes = 1;
    if (r.tile_nnz <= 0) r.tile_nnz = dtype == GBS_F64 ? 2048 : 3072;
  }
  return r;
}

// Merge geometry of one call: lanes per merge thread (columns), items per merge thread, CTAs.
struct MergeGeom {
  int g, items, ctas, kp_max;
};

int check_cfg(const gbs_config& c) {
  if (c.variant != GBS_VARIANT_ROWS && !is_merge(c.variant) && c.variant != GBS_VARIANT_ROWS_TMA &&
      c.variant != GBS_VARIANT_ROWS_DIRECT)
    return fail(GBS_EINVAL, "variant must be ROWS, MERGE, ROWS_TMA, MERGE_DIRECT or ROWS_DIRECT after resolution");
  if (c.variant == GBS_VARIANT_ROWS_TMA && c.threads > 256) return fail(GBS_EINVAL, "ROWS_TMA threads must be <= 256");
  if (c.threads % 32 != 0 || c.threads < 32 || c.threads > 1024) return fail(GBS_EINVAL, "threads must be 32..1024, multiple of 32");
  if (is_merge(c.variant) && c.threads > 256) return fail(GBS_EINVAL, "MERGE threads must be <= 256");
  if (c.lanes != 0 && !pow2_lanes(c.lanes)) return fail(GBS_EINVAL, "lanes must be 1, 2, 4, 8, 16 or 32");
  if ((c.variant == GBS_VARIANT_ROWS || c.variant == GBS_VARIANT_ROWS_TMA) && (c.tile_nnz < 32 || c.tile_nnz > (1 << 14)))
    return fail(GBS_EINVAL, "tile_nnz must be in [32, 16384]");
  if (is_merge(c.variant) && (c.items < 0 || c.items > 256)) return fail(GBS_EINVAL, "items must be in [0, 256]");
  if (c.emul < 0 || c.emul > 3) return fail(GBS_EINVAL, "emul must be in [0, 3]");
  if (c.relabel < 0 || c.relabel > 1024) return fail(GBS_EINVAL, "relabel must be in [0, 1024]");
  return GBS_OK;
}

// ---------------------------------------------------------------- execution

struct MergeBuffers {
  MergeScratch s{};
  void* base = nullptr;
  size_t bytes = 0;
};

size_t merge_scratch_bytes(int ctas, int kp, int dtype) {
  size_t a = ((size_t)(ctas + 1) * sizeof(int2) + 255) & ~(size_t)255;
  size_t b = ((size_t)ctas * sizeof(int) + 255) & ~(size_t)255;
  size_t c = (size_t)ctas * std::max(kp, 1) * dsize(dtype);
  return a + b + c;
}

void merge_carve(MergeBuffers& mb, int ctas, int kp, int dtype) {
  char* p = static_cast<char*>(mb.base);
  mb.s.ctas = ctas;
  mb.s.coords = reinterpret_cast<int2*>(p);
  p += ((size_t)(ctas + 1) * sizeof(int2) + 255) & ~(size_t)255;
  mb.s.carry_row = reinterpret_cast<int*>(p);
  p += ((size_t)ctas * sizeof(int) + 255) & ~(size_t)255;
  mb.s.carry_val = p;
  (void)kp;
  (void)dtype;
}

int merge_ctas(int m, int nnz, int threads, int g, int items) {
  long long ipc = (long long)(threads / g) * items;
  long long total = (long long)m + nnz;
  return (int)std::max<long long>(1, (total + ipc - 1) / ipc);
}

MergeGeom merge_geom(const gbs_config& cfg, int m, int nnz, int dtype, int k, bool vec16) {
  MergeGeom g{};
  g.kp_max = std::min(panel_cols(dtype, vec16), k);
  g.g = k == 1 ? 1 : std::max(cfg.lanes > 0 ? cfg.lanes : 1, col_lanes(g.kp_max, dtype, vec16));
  g.g = std::min(g.g, cfg.threads);
  g.items = cfg.items > 0 ? cfg.items : default_items(g.g, cfg.threads);
  g.ctas = merge_ctas(m, nnz, cfg.threads, g.g, g.items);
  return g;
}

// Run one product Y = A X (k >= 1; k == 1 with ldx = ldy = 1 is SpMV) with a resolved
// configuration.  Merge scratch comes from `mb` if given (plan), else from the stream-ordered
// allocator.  `coords_ready`: the partition in mb is valid for this configuration.
int run_product(const CsrView& A, int dtype, int k, const void* X, long long ldx, void* Y, long long ldy,
                const gbs_config& cfg, MergeBuffers* mb, bool coords_ready, cudaStream_t s, int* status = nullptr,
                int vec16_as = -1) {
  if (A.m == 0 || k == 0) return GBS_OK;
  // 128-bit column access when X, Y and their leading dimensions allow it; vec16_as (0 / 1)
  // imposes the decision made for the caller's own operands (0 is always safe; 1 only for
  // operands that allow it)
  const bool vec16 = vec16_as >= 0 ? vec16_as != 0 : dense_vec16(dtype, k, X, ldx, Y, ldy);
  const int P = panel_cols(dtype, vec16);
  const size_t es = dsize(dtype);
  cudaError_t e = cudaSuccess;
  const bool perm = A.perm != nullptr;
  if (perm && cfg.variant == GBS_VARIANT_ROWS_TMA)
    return fail(GBS_EUNSUPPORTED, "values read through a permutation need the ROWS, MERGE or MERGE_DIRECT variant");
  if (cfg.variant == GBS_VARIANT_ROWS_TMA && status && aligned16(A.vals) && aligned16(A.col_idx)) {
    for (int c0 = 0; c0 < k; c0 += P) {
      const int kp = std::min(P, k - c0);
      int lanes = cfg.lanes;
      if (k > 1) lanes = std::max(lanes, col_lanes(kp, dtype, vec16));
      DenseView D{kp, static_cast<const char*>(X) + c0 * es, ldx, static_cast<char*>(Y) + c0 * es, ldy};
      e = dtype == GBS_F64 ? launch_rows_tma_f64(A, D, lanes, vec16, cfg.threads, cfg.tile_nnz, cfg.emul, status, s)
                           : launch_rows_tma_f32(A, D, lanes, vec16, cfg.threads, cfg.tile_nnz, 0, status, s);
      if (e != cudaSuccess) return cuda_fail(e, "ROWS_TMA launch");
    }
    return GBS_OK;
  }
  if (cfg.variant == GBS_VARIANT_ROWS_DIRECT) {
    if (perm) return fail(GBS_EUNSUPPORTED, "ROWS_DIRECT does not read values through a permutation");
    for (int c0 = 0; c0 < k; c0 += P) {
      const int kp = std::min(P, k - c0);
      int lanes = cfg.lanes;
      if (k > 1) lanes = std::max(lanes, col_lanes(kp, dtype, vec16));
      DenseView D{kp, static_cast<const char*>(X) + c0 * es, ldx, static_cast<char*>(Y) + c0 * es, ldy};
      e = dtype == GBS_F64 ? launch_rows_direct_f64(A, D, lanes, vec16, cfg.threads, s)
                           : launch_rows_direct_f32(A, D, lanes, vec16, cfg.threads, s);
      if (e != cudaSuccess) return cuda_fail(e, "ROWS_DIRECT launch");
    }
    return GBS_OK;
  }
  if (cfg.variant == GBS_VARIANT_ROWS || cfg.variant == GBS_VARIANT_ROWS_TMA) {
    for (int c0 = 0; c0 < k; c0 += P) {
      const int kp = std::min(P, k - c0);
      int lanes = cfg.lanes;
      if (k > 1) lanes = std::max(lanes, col_lanes(kp, dtype, vec16));
      DenseView D{kp, static_cast<const char*>(X) + c0 * es, ldx, static_cast<char*>(Y) + c0 * es, ldy};
      auto launch = dtype == GBS_F64 ? (perm ? launch_rows_perm_f64 : launch_rows_f64)
                                     : (perm ? launch_rows_perm_f32 : launch_rows_f32);
      e = launch(A, D, lanes, vec16, cfg.threads, cfg.tile_nnz, 0, A.m, s);
      if (e != cudaSuccess) return cuda_fail(e, "ROWS launch");
    }
    return GBS_OK;
  }
  // MERGE
  const MergeGeom G = merge_geom(cfg, A.m, A.nnz, dtype, k, vec16);
  const int kp_max = G.kp_max, g = G.g, ctas = G.ctas;
  MergeBuffers local;
  MergeBuffers* use = mb;
  if (use == nullptr) {
    local.bytes = merge_scratch_bytes(ctas, kp_max, dtype);
    e = cudaMallocAsync(&local.base, local.bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (merge scratch)");
    merge_carve(local, ctas, kp_max, dtype);
    use = &local;
    coords_ready = false;
  } else if (use->s.ctas != ctas) {
    return fail(GBS_EINVAL, "plan scratch does not match the configuration");
  }
  int rc = GBS_OK;
  if (!coords_ready) {
    e = launch_merge_partition(A, (long long)(cfg.threads / g) * G.items, use->s, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "merge partition");
  }
  for (int c0 = 0; rc == GBS_OK && c0 < k; c0 += P) {
    const int kp = std::min(P, k - c0);
    DenseView D{kp, static_cast<const char*>(X) + c0 * es, ldx, static_cast<char*>(Y) + c0 * es, ldy};
    const bool direct = cfg.variant == GBS_VARIANT_MERGE_DIRECT;
    auto launch = dtype == GBS_F64 ? (perm ? launch_merge_perm_f64 : launch_merge_f64)
                                   : (perm ? launch_merge_perm_f32 : launch_merge_f32);
    e = launch(A, D, g, vec16, direct, cfg.threads, G.items, use->s, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "MERGE launch");
  }
  if (use == &local) {
    e = cudaFreeAsync(local.base, s);
    if (e != cudaSuccess && rc == GBS_OK) rc = cuda_fail(e, "cudaFreeAsync");
  }
  return rc;
}

// --------------------------------------------------------------- statistics

__global__ void stats_kernel(const int* __restrict__ rp, int m, unsigned long long* __restrict__ acc, int* __restrict__ maxrow) {
  unsigned long long sq = 0, empty = 0, o32 = 0, o256 = 0, o4k = 0;
  int mx = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const int len = rp[i + 1] - rp[i];
    sq += (unsigned long long)len * (unsigned long long)len;
    empty += len == 0;
    o32 += len > 32;
    o256 += len > 256;
    o4k += len > 4096;
    mx = max(mx, len);
  }
  for (int o = 16; o > 0; o >>= 1) {
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
    empty += __shfl_xor_sync(0xffffffffu, empty, o);
    o32 += __shfl_xor_sync(0xffffffffu, o32, o);
    o256 += __shfl_xor_sync(0xffffffffu, o256, o);
    o4k += __shfl_xor_sync(0xffffffffu, o4k, o);
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc + 0, sq);
    atomicAdd(acc + 1, empty);
    atomicAdd(acc + 2, o32);
    atomicAdd(acc + 3, o256);
    atomicAdd(acc + 4, o4k);
    atomicMax(maxrow, mx);
  }
}

__global__ void validate_kernel(const int* __restrict__ rp, const int* __restrict__ ci, int m, int n, int nnz,
                                int* __restrict__ flags) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
  int f = 0;
  if (tid == 0) {
    if (rp[0] != 0) f |= 1;
    if (rp[m] != nnz) f |= 2;
  }
  for (long long i = tid; i < m; i += nt)
    if (rp[i + 1] < rp[i]) f |= 4;
  for (long long p = tid; p < nnz; p += nt) {
    const int c = ci[p];
    if (c < 0 || c >= n) f |= 8;
  }
  if (f) atomicOr(flags, f);
}

int compute_stats(int m, int n, int nnz, const int* rp, gbs_stats* out, cudaStream_t s) {
  std::memset(out, 0, sizeof(*out));
  out->m = m;
  out->n = n;
  out->nnz = nnz;
  if (m == 0) return GBS_OK;
  void* buf = nullptr;
  cudaError_t e = cudaMallocAsync(&buf, 64, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (stats)");
  unsigned long long* acc = static_cast<unsigned long long*>(buf);
  int* mx = reinterpret_cast<int*>(acc + 5);
  unsigned long long h[5];
  int hm = 0;
  e = cudaMemsetAsync(buf, 0, 64, s);
  if (e == cudaSuccess) {
    int blocks = std::min(1024, (m + 255) / 256);
    stats_kernel<<<blocks, 256, 0, s>>>(rp, m, acc, mx);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hm, mx, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e2 = cudaFreeAsync(buf, s);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "CSR statistics");
  out->max_row = hm;
  out->empty_rows = (int)h[1];
  out->mean_row = (double)nnz / m;
  double var = (double)h[0] / m - out->mean_row * out->mean_row;
  out->cv_row = out->mean_row > 0 ? std::sqrt(std::max(0.0, var)) / out->mean_row : 0.0;
  out->rows_over_32 = (long long)h[2];
  out->rows_over_256 = (long long)h[3];
  out->rows_over_4096 = (long long)h[4];
  return GBS_OK;
}

// A wait that runs out on purpose, for testing the timeout path: one CTA arms an mbarrier for a
// 16-byte copy that is never issued and waits on it (bounded by limit_ns); status[0] = 1 when
// the wait gave up, 0 if it completed.
__global__ void wait_probe_kernel(int* __restrict__ status, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16);
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
  if (threadIdx.x == 0) status[0] = ok ? 0 : 1;
}

__global__ void block_max_nnz_kernel(const int* __restrict__ rp, int m, int rpc, int* __restrict__ out) {
  const int nb = (m + rpc - 1) / rpc;
  int mx = 0;
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (long long)gridDim.x * blockDim.x)
    mx = max(mx, rp[min((long long)m, (b + 1) * rpc)] - rp[b * rpc]);
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

// Largest nonzero count of a block of rpc consecutive rows (synchronises s).
int block_max_nnz(const int* rp, int m, int rpc, int* out, cudaStream_t s) {
  int* d = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d), sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (block max)");
  e = cudaMemsetAsync(d, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    const int nb = (m + rpc - 1) / rpc;
    block_max_nnz_kernel<<<std::min(1024, (nb + 255) / 256), 256, 0, s>>>(rp, m, rpc, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e2 = cudaFreeAsync(d, s);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? GBS_OK : cuda_fail(e, "block max nnz");
}

gbs_config heuristic_config(const gbs_stats& st, int dtype, int k) {
  gbs_config c{};
  c.threads = 256;
  const double mean = st.mean_row;
  const bool skewed = st.max_row > 16.0 * mean + 256.0 || st.cv_row > 2.0;
  if (skewed) {
    c.variant = GBS_VARIANT_MERGE;
    c.lanes = 0;
    c.items = 0;
  } else {
    c.variant = GBS_VARIANT_ROWS;
    if (k == 1) {
      // FP64: one lane per row keeps every FMA lane busy and needs no reduction;
      // long rows get more lanes so that a warp's rows finish together.
      const double per = dtype == GBS_F64 ? 64.0 : 16.0;
      int l = 1;
      while (l < 32 && mean > per * l) l <<= 1;
      c.lanes = l;
    } else {
      c.lanes = 0;  // column lanes follow k
    }
    c.tile_nnz = dtype == GBS_F64 ? 2048 : 3072;
  }
  return normalize(c, dtype);
}

// Eight independent FMA chains per thread: the FP64 pipe's throughput, not its latency.
__global__ void fp64_probe_kernel(double* __restrict__ out, int iters) {
  double a0 = threadIdx.x * 1e-3, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
         a7 = a0 + 7;
  const double b = 0.999999, c = 1e-7;
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, b, c);
    a1 = fma(a1, b, c);
    a2 = fma(a2, b, c);
    a3 = fma(a3, b, c);
    a4 = fma(a4, b, c);
    a5 = fma(a5, b, c);
    a6 = fma(a6, b, c);
    a7 = fma(a7, b, c);
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

}  // namespace

namespace gbs {
void set_last_error(const char* msg) { g_err = msg ? msg : ""; }

size_t rows_tma_smem(int dtype, int rpc, int tile) {
  return dtype == GBS_F64 ? rows_tma_smem_bytes<double>(rpc, tile) : rows_tma_smem_bytes<float>(rpc, tile);
}

// Start coordinates of every merge-path tile: one thread per tile boundary.
__global__ void merge_partition_kernel(const int* __restrict__ row_ptr, int m, int nnz, int ctas,
                                       long long items_per_cta, int2* __restrict__ coords) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b > ctas) return;
  long long total = (long long)m + nnz;
  long long d = (long long)b * items_per_cta;
  if (d > total) d = total;
  coords[b] = merge_search_global(row_ptr, m, nnz, d);
}

cudaError_t launch_merge_partition(const CsrView& A, long long items_per_cta, const MergeScratch& S, cudaStream_t s) {
  const int n = S.ctas + 1;
  merge_partition_kernel<<<(n + 255) / 256, 256, 0, s>>>(A.row_ptr, A.m, A.nnz, S.ctas, items_per_cta, S.coords);
  return cudaGetLastError();
}
}  // namespace gbs

// ====================================================================== ABI

extern "C" {

int gbs_version(void) { return 100; }

int gbs_wait_probe(long long limit_ns, void* stream) {
  if (limit_ns < 1 || limit_ns > 2000000000LL) return fail(GBS_EINVAL, "limit_ns must be in [1, 2e9]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* d = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d), sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (wait probe)");
  e = cudaMemsetAsync(d, 0xff, sizeof(int), s);
  if (e == cudaSuccess) {
    wait_probe_kernel<<<1, 32, 0, s>>>(d, (unsigned long long)limit_ns);
    e = cudaGetLastError();
  }
  int h = -1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "wait probe");
  if (h == 1) return fail(GBS_ETIMEOUT, "wait probe: the bounded wait gave up (expected)");
  return h == 0 ? GBS_OK : fail(GBS_ECUDA, "wait probe: no status written");
}

int gbs_fp64_probe(double* out, int blocks, int threads, int iters, void* stream) {
  if (!out || blocks < 1 || threads < 32 || threads > 1024 || threads % 32 || iters < 1)
    return fail(GBS_EINVAL, "fp64 probe arguments");
  fp64_probe_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(out, iters);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GBS_OK : cuda_fail(e, "fp64 probe");
}

const char* gbs_status_string(int status) {
  switch (status) {
    case GBS_OK: return "ok";
    case GBS_EINVAL: return "invalid argument";
    case GBS_EALIGN: return "misaligned pointer or leading dimension";
    case GBS_EDTYPE: return "unknown dtype";
    case GBS_ECUDA: return "CUDA error";
    case GBS_EINDEX: return "invalid CSR structure";
    case GBS_ETIMEOUT: return "device wait timed out";
    case GBS_ENOMEM: return "out of memory";
    case GBS_EUNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

const char* gbs_last_error(void) { return g_err.c_str(); }

int gbs_validate_csr(int m, int n, int nnz, const int* row_ptr, const int* col_idx, void* stream) {
  if (m < 0 || n < 0 || nnz < 0) return fail(GBS_EINVAL, "negative size");
  if (row_ptr == nullptr || (nnz > 0 && col_idx == nullptr)) return fail(GBS_EINVAL, "NULL pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* flags = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&flags), sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (validate)");
  int h = 0;
  e = cudaMemsetAsync(flags, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    long long work = std::max<long long>(m, nnz);
    int blocks = (int)std::min<long long>(2048, std::max<long long>(1, (work + 255) / 256));
    validate_kernel<<<blocks, 256, 0, s>>>(row_ptr, col_idx, m, n, nnz, flags);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flags, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e2 = cudaFreeAsync(flags, s);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "validate");
  if (h) {
    std::string msg = "invalid CSR:";
    if (h & 1) msg += " row_ptr[0] != 0;";
    if (h & 2) msg += " row_ptr[m] != nnz;";
    if (h & 4) msg += " row_ptr decreases;";
    if (h & 8) msg += " col_idx outside [0, n);";
    return fail(GBS_EINDEX, msg);
  }
  return GBS_OK;
}

int gbs_csr_stats(int m, int n, int nnz, const int* row_ptr, gbs_stats* out, void* stream) {
  if (out == nullptr) return fail(GBS_EINVAL, "out is NULL");
  int rc = check_csr(m, n, nnz, row_ptr, reinterpret_cast<const int*>(1), reinterpret_cast<const void*>(1));
  if (rc) return rc;
  return compute_stats(m, n, nnz, row_ptr, out, static_cast<cudaStream_t>(stream));
}

int gbs_ucld(int m, int n, int nnz, const int* row_ptr, const int* col_idx, int line_elems, double* ucld,
             long long* lines, long long* nonempty_rows, void* stream) {
  int rc = check_csr(m, n, nnz, row_ptr, col_idx, reinterpret_cast<const void*>(1));
  if (rc) return rc;
  if (line_elems < 1) return fail(GBS_EINVAL, "line_elems must be >= 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long h[3] = {0, 0, 0};
  if (m > 0 && nnz > 0) {
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d), sizeof(h), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (ucld)");
    e = cudaMemsetAsync(d, 0, sizeof(h), s);
    if (e == cudaSuccess) e = launch_ucld(row_ptr, col_idx, m, line_elems, d, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "ucld");
  }
  if (ucld) *ucld = h[2] ? (double)h[0] / 2147483648.0 / (double)h[2] : 0.0;
  if (lines) *lines = (long long)h[1];
  if (nonempty_rows) *nonempty_rows = (long long)h[2];
  return GBS_OK;
}

int gbs_rcm(int n, int nnz, const int* row_ptr, const int* col_idx, int* perm, void* stream) {
  int rc = check_csr(n, n, nnz, row_ptr, col_idx, reinterpret_cast<const void*>(1));
  if (rc) return rc;
  if (n > 0 && !perm) return fail(GBS_EINVAL, "perm is NULL");
  if (nnz > INT_MAX / 2) return fail(GBS_EUNSUPPORTED, "nnz above 2^30: the symmetric pattern would not fit int32");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (checked_mode()) {
    rc = gbs_validate_csr(n, n, nnz, row_ptr, col_idx, stream);
    if (rc) return rc;
  }
  cudaError_t e = rcm_run(n, nnz, row_ptr, col_idx, perm, s);
  return e == cudaSuccess ? GBS_OK : cuda_fail(e, "rcm");
}

int gbs_permute_csr(int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals, int dtype,
                    const int* perm, int* b_row_ptr, int* b_col_idx, void* b_vals, void* stream) {
  int rc = check_csr(n, n, nnz, row_ptr, col_idx, reinterpret_cast<const void*>(1));
  if (rc) return rc;
  if (vals && !valid_dtype(dtype)) return fail(GBS_EDTYPE, "dtype");
  if (n > 0 && (!perm || !b_row_ptr)) return fail(GBS_EINVAL, "perm or b_row_ptr is NULL");
  if (nnz > 0 && !b_col_idx) return fail(GBS_EINVAL, "b_col_idx is NULL");
  if (nnz > 0 && (vals != nullptr) != (b_vals != nullptr)) return fail(GBS_EINVAL, "vals and b_vals: both or neither");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = permute_run(n, nnz, row_ptr, col_idx, vals, dtype, perm, b_row_ptr, b_col_idx, b_vals, s);
  return e == cudaSuccess ? GBS_OK : cuda_fail(e, "permute");
}

int gbs_default_config(const gbs_stats* stats, int dtype, int k, gbs_config* out) {
  if (stats == nullptr || out == nullptr) return fail(GBS_EINVAL, "NULL pointer");
  if (!valid_dtype(dtype)) return fail(GBS_EDTYPE, "dtype");
  if (k < 1) return fail(GBS_EINVAL, "k must be >= 1");
  *out = heuristic_config(*stats, dtype, k);
  return GBS_OK;
}

static int product_entry(int m, int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals, int dtype,
                         int k, const void* X, long long ldx, void* Y, long long ldy, const gbs_config* cfg,
                         void* stream) {
  if (!valid_dtype(dtype)) return fail(GBS_EDTYPE, "dtype must be GBS_F64 or GBS_F32");
  int rc = check_csr(m, n, nnz, row_ptr, col_idx, vals);
  if (rc) return rc;
  if (k < 1) return fail(GBS_EINVAL, "k must be >= 1");
  if (ldx < k || ldy < k) return fail(GBS_EINVAL, "leading dimension smaller than k");
  if (m > 0 && Y == nullptr) return fail(GBS_EINVAL, "y/Y is NULL");
  if (nnz > 0 && X == nullptr) return fail(GBS_EINVAL, "x/X is NULL");
  const size_t es = dsize(dtype);
  if ((reinterpret_cast<uintptr_t>(vals) % es) || (reinterpret_cast<uintptr_t>(X) % es) ||
      (reinterpret_cast<uintptr_t>(Y) % es) || (reinterpret_cast<uintptr_t>(col_idx) % 4) ||
      (reinterpret_cast<uintptr_t>(row_ptr) % 4))
    return fail(GBS_EALIGN, "arrays must be aligned to their element size");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (checked_mode()) {
    rc = gbs_validate_csr(m, n, nnz, row_ptr, col_idx, stream);
    if (rc) return rc;
  }
  gbs_config c{};
  if (cfg == nullptr || cfg->variant == GBS_VARIANT_AUTO) {
    // merge-path, which needs no row statistics: SpMV with contiguous x and y takes the direct
    // walk's SpMV form (128 threads x 9 items; 1.5-2x the staged form on the 27-point stencil,
    // the banded matrix and R-MAT 22, scratch and partition included), SpMM the staged form
    const bool spmv = k == 1 && ldx == 1 && ldy == 1;
    c.variant = spmv ? GBS_VARIANT_MERGE_DIRECT : GBS_VARIANT_MERGE;
    c.threads = cfg && cfg->threads ? cfg->threads : (spmv ? 128 : 256);
    c.items = cfg && cfg->items ? cfg->items : (spmv ? 9 : 0);
    c.lanes = cfg ? cfg->lanes : 0;
    c.tile_nnz = 0;
  } else {
    c = *cfg;
  }
  if (c.relabel != 0) return fail(GBS_EINVAL, "relabel needs a plan (gbs_plan_create / gbs_plan_set_config)");
  c = normalize(c, dtype);
  rc = check_cfg(c);
  if (rc) return rc;
  CsrView A{m, n, nnz, row_ptr, col_idx, vals};
  return run_product(A, dtype, k, X, ldx, Y, ldy, c, nullptr, false, s);
}

int spmv_csr(int m, int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals, int dtype,
             const void* x, void* y, void* stream) {
  return product_entry(m, n, nnz, row_ptr, col_idx, vals, dtype, 1, x, 1, y, 1, nullptr, stream);
}

int spmv_csr_cfg(int m, int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals, int dtype,
                 const void* x, void* y, const gbs_config* cfg, void* stream) {
  return product_entry(m, n, nnz, row_ptr, col_idx, vals, dtype, 1, x, 1, y, 1, cfg, stream);
}

int spmm_csr(int m, int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals, int dtype, int k,
             const void* X, int ldx, void* Y, int ldy, void* stream) {
  return product_entry(m, n, nnz, row_ptr, col_idx, vals, dtype, k, X, ldx, Y, ldy, nullptr, stream);
}

int spmm_csr_cfg(int m, int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals, int dtype, int k,
                 const void* X, int ldx, void* Y, int ldy, const gbs_config* cfg, void* stream) {
  return product_entry(m, n, nnz, row_ptr, col_idx, vals, dtype, k, X, ldx, Y, ldy, cfg, stream);
}

}  // extern "C"

// ==================================================================== plans

struct gbs_plan {
  int m = 0, n = 0, nnz = 0, k = 1, dtype = GBS_F64, device = 0;
  const int* row_ptr = nullptr;
  const int* col_idx = nullptr;
  gbs_stats stats{};
  gbs_config cfg{};
  MergeBuffers mb{};
  bool coords_ready = false;
  int flags = 0;
  int* status = nullptr;  // device word: bounded-wait status of the pipelined variant
  const int* perm = nullptr;  // values read through this permutation (plans of A^T inside a transpose plan)
  float tuned_ms = 0.0f;      // the tuner's time of the chosen configuration (0: not tuned)
  // column relabelling (cfg.relabel != 0): newid[n], col_rl[nnz] = newid[col_idx], and the
  // relabelled copy of x / X (n rows of ldxp elements)
  int* newid = nullptr;
  int* col_rl = nullptr;
  void* xbuf = nullptr;
  long long ldxp = 1;
  int col_max_deg = -1;  // column-degree statistics, computed on first need
  double col_cv = 0.0;
  bool tuning = false;   // the tuner is trying configurations: keep the relabelling between them
};

namespace {

// Allocate (or free) the plan's merge scratch for its configuration and compute the
// partition.  Scratch is sized for 128-bit column panels, the widest case.
void relabel_release(gbs_plan* p) {
  if (p->newid) cudaFree(p->newid);
  if (p->col_rl) cudaFree(p->col_rl);
  if (p->xbuf) cudaFree(p->xbuf);
  p->newid = p->col_rl = nullptr;
  p->xbuf = nullptr;
}

// The relabelled indices and x buffer of a plan whose configuration relabels (built once).
int relabel_prepare(gbs_plan* p, cudaStream_t s) {
  if (p->cfg.relabel == 0 || p->newid || p->n == 0) return GBS_OK;
  const size_t es = dsize(p->dtype);
  const int v = (int)(16 / es);
  p->ldxp = p->k == 1 ? 1 : (long long)((p->k + v - 1) / v) * v;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p->newid), sizeof(int) * (size_t)p->n);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->col_rl), sizeof(int) * (size_t)std::max(p->nnz, 1));
  if (e == cudaSuccess) e = cudaMalloc(&p->xbuf, es * (size_t)p->n * (size_t)p->ldxp);
  if (e == cudaSuccess) e = relabel_build(p->n, p->nnz, p->col_idx, p->newid, p->col_rl, s);
  if (e != cudaSuccess) {
    relabel_release(p);
    return cuda_fail(e, "column relabelling");
  }
  return GBS_OK;
}

int plan_prepare(gbs_plan* p, cudaStream_t s) {
  if (p->mb.base) {
    cudaFree(p->mb.base);
    p->mb = MergeBuffers{};
  }
  p->coords_ready = false;
  if (p->cfg.relabel == 0) {
    if (!p->tuning) relabel_release(p);
  } else {
    const int rc = relabel_prepare(p, s);
    if (rc) return rc;
  }
  if (p->cfg.variant == GBS_VARIANT_ROWS_TMA && p->m > 0) {
    // the tile must hold the largest row block: measure it on the device
    int lanes = p->cfg.lanes;
    if (p->k > 1) lanes = std::max(lanes, col_lanes(std::min(panel_cols(p->dtype, true), p->k), p->dtype, true));
    const int rpc = p->cfg.threads / lanes;
    int mx = 0;
    int rc = block_max_nnz(p->row_ptr, p->m, rpc, &mx, s);
    if (rc) return rc;
    const int tile = ((mx + 8 + 31) / 32) * 32;
    const size_t smem = rows_tma_smem(p->dtype, rpc, tile);
    // 227 KB per CTA, less the kernel's static shared memory (two blocks of row partials, and
    // of float-float pairs when emulating)
    const size_t stat = 2 * 256 * 8 + (p->cfg.emul ? 2 * 256 * 8 : 0) + 64;
    if (tile > (1 << 14) || smem > 227 * 1024 - stat)
      return fail(GBS_EUNSUPPORTED, "row blocks too large for ROWS_TMA");
    p->cfg.tile_nnz = tile;
    return GBS_OK;
  }
  if (!is_merge(p->cfg.variant) || p->m == 0) return GBS_OK;
  // the partition depends on the lanes per merge thread, which depend on whether a call
  // can use 128-bit column access; the plan is made for that case (k > 1) and calls that
  // cannot use it take the stream-ordered path
  const MergeGeom G = merge_geom(p->cfg, p->m, p->nnz, p->dtype, p->k, p->k > 1);
  p->mb.bytes = merge_scratch_bytes(G.ctas, G.kp_max, p->dtype);
  cudaError_t e = cudaMalloc(&p->mb.base, p->mb.bytes);
  if (e != cudaSuccess) {
    p->mb = MergeBuffers{};
    return cuda_fail(e, "cudaMalloc (plan scratch)");
  }
  merge_carve(p->mb, G.ctas, G.kp_max, p->dtype);
  CsrView A{p->m, p->n, p->nnz, p->row_ptr, p->col_idx, nullptr};
  e = launch_merge_partition(A, (long long)(p->cfg.threads / G.g) * G.items, p->mb.s, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "merge partition");
  p->coords_ready = true;
  return GBS_OK;
}

int plan_run(const gbs_plan* p, const void* vals, const void* X, long long ldx, void* Y, long long ldy, cudaStream_t s) {
  CsrView A{p->m, p->n, p->nnz, p->row_ptr, p->col_idx, vals, p->perm};
  // the caller's operands decide the column access (and with it the merge geometry), also when
  // the product reads the relabelled copy of X, so that relabelling never changes a result
  const bool vec16 = dense_vec16(p->dtype, p->k, X, ldx, Y, ldy);
  if (p->cfg.relabel != 0 && p->newid && p->m > 0 && p->k > 0) {
    // x' = x in the relabelled column order, then the product with the relabelled column ids
    const bool src16 = p->k > 1 && aligned16(X) && (ldx * (long long)dsize(p->dtype)) % 16 == 0;
    cudaError_t e = relabel_dense(p->dtype, p->n, p->k, X, ldx, p->newid, p->xbuf, p->ldxp, src16, s);
    if (e != cudaSuccess) return cuda_fail(e, "relabel of x");
    A.col_idx = p->col_rl;
    if (p->cfg.relabel >= 2) A.hot_cols = (int)std::min<long long>(INT_MAX - 1, (long long)p->cfg.relabel * 1024);
    X = p->xbuf;
    ldx = p->ldxp;
  }
  const int as = vec16 ? 1 : 0;
  if (is_merge(p->cfg.variant)) {
    // the partition was made for 128-bit column access; if this call cannot use it the
    // lane count differs and the stream-ordered path is used instead
    if (p->k > 1 && !vec16) return run_product(A, p->dtype, p->k, X, ldx, Y, ldy, p->cfg, nullptr, false, s, nullptr, as);
    MergeBuffers mb = p->mb;
    return run_product(A, p->dtype, p->k, X, ldx, Y, ldy, p->cfg, &mb, p->coords_ready, s, nullptr, as);
  }
  return run_product(A, p->dtype, p->k, X, ldx, Y, ldy, p->cfg, nullptr, false, s, p->status, as);
}

// Candidate configurations for the tuner.
std::vector<gbs_config> tune_candidates(const gbs_plan* p) {
  std::vector<gbs_config> c;
  auto add = [&](int variant, int lanes, int threads, int tile, int items) {
    gbs_config g{};
    g.variant = variant;
    g.lanes = lanes;
    g.threads = threads;
    g.tile_nnz = tile;
    g.items = items;
    c.push_back(normalize(g, p->dtype));
  };
  const int base_tile = p->dtype == GBS_F64 ? 2048 : 3072;
  // a tile that holds a whole row block in the common case: rows per CTA x mean row length
  auto fit_tile = [&](int threads, int lanes) {
    double want = (double)(threads / lanes) * p->stats.mean_row * 1.1 + 64;
    int t = 1024;
    while (t < want && t < 16384) t <<= 1;
    return t;
  };
  if (p->k == 1) {
    for (int l : {1, 2, 4, 8, 16, 32}) {
      if (l > 1 && p->stats.mean_row < 0.5 * l) continue;
      add(GBS_VARIANT_ROWS, l, 256, base_tile, 0);
      if (fit_tile(256, l) != base_tile) add(GBS_VARIANT_ROWS, l, 256, fit_tile(256, l), 0);
    }
    add(GBS_VARIANT_ROWS, 1, 128, fit_tile(128, 1), 0);
    add(GBS_VARIANT_ROWS, 2, 128, fit_tile(128, 2), 0);
    const int tma_shapes[][2] = {{1, 32}, {1, 64}, {1, 128}, {2, 64}, {2, 128}, {2, 256}, {4, 96}, {4, 128},
                                 {4, 160}, {4, 192}, {4, 224}, {4, 256}, {8, 256}};
    for (const auto& sh : tma_shapes)
      for (int l = sh[0], th = sh[1], once = 1; once; once = 0)
        if (l == 1 || p->stats.mean_row >= 0.5 * l) {
          add(GBS_VARIANT_ROWS_TMA, l, th, 0, 0);
          if (p->dtype == GBS_F64 && (p->flags & GBS_PLAN_EMULATE))
            for (int em : {1, 2}) {
              add(GBS_VARIANT_ROWS_TMA, l, th, 0, 0);
              c.back().emul = em;
            }
        }
    for (int it : {7, 11, 15, 23, 31}) add(GBS_VARIANT_MERGE, 0, 256, 0, it);
    for (int it : {7, 9, 11, 13, 15, 23, 31, 47, 63}) add(GBS_VARIANT_MERGE_DIRECT, 0, 256, 0, it);
    // smaller CTAs: the direct walk is held to 40 registers, so twelve 128-thread (or twenty-four
    // 64-thread) CTAs fill an SM as six of 256 do, with finer tiles at the end of the grid
    for (int it : {7, 8, 9, 10, 11, 13, 15}) add(GBS_VARIANT_MERGE_DIRECT, 0, 128, 0, it);
    for (int it : {8, 9, 10, 11}) add(GBS_VARIANT_MERGE_DIRECT, 0, 64, 0, it);
    for (int th : {128, 256}) add(GBS_VARIANT_ROWS_DIRECT, 1, th, 0, 0);
  } else {
    add(GBS_VARIANT_ROWS, 0, 256, base_tile, 0);
    add(GBS_VARIANT_ROWS, 0, 128, base_tile, 0);
    add(GBS_VARIANT_ROWS, 0, 256, base_tile / 2, 0);
    add(GBS_VARIANT_ROWS_TMA, 0, 64, 0, 0);
    add(GBS_VARIANT_ROWS_TMA, 0, 128, 0, 0);
    add(GBS_VARIANT_ROWS_TMA, 0, 256, 0, 0);
    if (p->dtype == GBS_F64 && (p->flags & GBS_PLAN_EMULATE))
      for (int th : {128, 256})
        for (int em : {1, 2, 3}) {
          add(GBS_VARIANT_ROWS_TMA, 0, th, 0, 0);
          c.back().emul = em;
        }
    add(GBS_VARIANT_MERGE, 0, 256, 0, 0);
    add(GBS_VARIANT_MERGE, 0, 128, 0, 0);
    add(GBS_VARIANT_MERGE_DIRECT, 0, 256, 0, 0);
    for (int th : {128, 256}) add(GBS_VARIANT_ROWS_DIRECT, 0, th, 0, 0);
  }
  // skewed column degrees (a power-law matrix): the merge forms again on columns relabelled
  // hottest first, with every gather through L1 or with the cold ones bypassing it
  const double mean_col = p->n > 0 ? (double)p->nnz / p->n : 0.0;
  if (p->col_max_deg > 16.0 * mean_col + 256.0 || p->col_cv > 2.0) {
    std::vector<gbs_config> rl;
    for (const gbs_config& g : c)
      if (is_merge(g.variant) && g.emul == 0) {
        rl.push_back(g);
        rl.back().relabel = 1;
        if (p->k == 1 && g.variant == GBS_VARIANT_MERGE_DIRECT && g.items <= 15) {
          rl.push_back(g);
          rl.back().relabel = 8;
        }
      }
    c.insert(c.end(), rl.begin(), rl.end());
  }
  if (p->perm) {
    // values through a permutation: the variants that support it
    std::vector<gbs_config> keep;
    for (const gbs_config& g : c)
      if (g.variant != GBS_VARIANT_ROWS_TMA && g.variant != GBS_VARIANT_ROWS_DIRECT && g.emul == 0) keep.push_back(g);
    c.swap(keep);
  }
  return c;
}

int plan_tune(gbs_plan* p, cudaStream_t s) {
  const size_t es = dsize(p->dtype);
  const long long ld = p->k == 1 ? 1 : ((p->k + 1) / 2 * 2);  // even leading dimension keeps 16-byte rows for f64
  const long long ldp = p->dtype == GBS_F64 ? ld : ((p->k + 3) / 4 * 4);
  void *vals = nullptr, *X = nullptr, *Y = nullptr;
  size_t bv = std::max<size_t>(16, (size_t)p->nnz * es);
  size_t bx = std::max<size_t>(16, (size_t)p->n * (p->k == 1 ? 1 : ldp) * es);
  size_t by = std::max<size_t>(16, (size_t)p->m * (p->k == 1 ? 1 : ldp) * es);
  cudaError_t e = cudaMalloc(&vals, bv);
  if (e == cudaSuccess) e = cudaMalloc(&X, bx);
  if (e == cudaSuccess) e = cudaMalloc(&Y, by);
  if (e == cudaSuccess) e = cudaMemsetAsync(vals, 0, bv, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(X, 0, bx, s);
  // Every timed run starts with a cold L2, as a product inside an application usually does: a
  // write of twice the L2's size before it evicts the previous run's matrix and x (without it,
  // candidates that differ only in how they use L1 and L2 rank differently).  Optional: the
  // tuner times warm if the buffer cannot be had.
  void* flush = nullptr;
  size_t bf = 0;
  if (e == cudaSuccess) {
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess &&
        l2 > 0 && cudaMalloc(&flush, 2 * (size_t)l2) == cudaSuccess)
      bf = 2 * (size_t)l2;
    else
      flush = nullptr;
    cudaGetLastError();
  }
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ev1);
  int rc = e == cudaSuccess ? GBS_OK : cuda_fail(e, "tuner allocation");
  const long long ldx = p->k == 1 ? 1 : ldp;
  float best = 1e30f;
  gbs_config best_cfg = p->cfg;
  if (rc == GBS_OK && p->col_max_deg < 0) {
    if (col_degree_stats(p->n, p->nnz, p->col_idx, &p->col_max_deg, &p->col_cv, s) != cudaSuccess) {
      p->col_max_deg = 0;  // statistics unavailable: no relabelled candidates
      p->col_cv = 0.0;
      cudaGetLastError();
    }
  }
  p->tuning = true;
  if (rc == GBS_OK) {
    // median of `reps` timed runs (after one untimed) of the prepared configuration, < 0 on failure
    auto median_ms = [&](int reps) -> float {
      std::vector<float> times((size_t)reps);
      bool ok = true;
      for (int r = 0; r <= reps && ok; ++r) {
        if (flush && cudaMemsetAsync(flush, r, bf, s) != cudaSuccess) ok = false;
        if (ok && cudaEventRecord(ev0, s) != cudaSuccess) ok = false;
        if (ok && plan_run(p, vals, X, ldx, Y, ldx, s) != GBS_OK) ok = false;
        if (ok && cudaEventRecord(ev1, s) != cudaSuccess) ok = false;
        if (ok && cudaEventSynchronize(ev1) != cudaSuccess) ok = false;
        float ms = 0;
        if (ok) cudaEventElapsedTime(&ms, ev0, ev1);
        if (r > 0) times[(size_t)r - 1] = ms;
      }
      if (!ok) return -1.0f;
      std::sort(times.begin(), times.end());
      return times[(size_t)reps / 2];
    };
    std::vector<std::pair<float, gbs_config>> timed;
    for (const gbs_config& c : tune_candidates(p)) {
      if (check_cfg(c) != GBS_OK) continue;
      p->cfg = c;
      if (plan_prepare(p, s) != GBS_OK) continue;
      const float ms = median_ms(7);
      if (ms < 0) continue;
      if (tune_log())
        std::fprintf(stderr, "gbspmv tune m=%d nnz=%d k=%d: variant=%d lanes=%d threads=%d tile=%d items=%d emul=%d "
                     "relabel=%d -> %.4f ms\n", p->m, p->nnz, p->k, c.variant, c.lanes, c.threads, p->cfg.tile_nnz,
                     c.items, c.emul, c.relabel, ms);
      timed.emplace_back(ms, c);
    }
    // the leaders often differ by a few per cent, about the spread of seven runs: the three best
    // are timed again, fifteen runs each, and the best of those medians is kept
    std::stable_sort(timed.begin(), timed.end(),
                     [](const std::pair<float, gbs_config>& x, const std::pair<float, gbs_config>& y) { return x.first < y.first; });
    const size_t lead = std::min<size_t>(3, timed.size());
    for (size_t i = 0; i < lead; ++i) {
      float ms = timed[i].first;
      p->cfg = timed[i].second;
      if (lead > 1 && plan_prepare(p, s) == GBS_OK) {
        const float again = median_ms(15);
        if (again >= 0) ms = again;
      }
      if (tune_log())
        std::fprintf(stderr, "gbspmv tune m=%d nnz=%d k=%d: leader %zu variant=%d threads=%d items=%d relabel=%d -> %.4f ms\n",
                     p->m, p->nnz, p->k, i, timed[i].second.variant, timed[i].second.threads, timed[i].second.items,
                     timed[i].second.relabel, ms);
      if (ms < best) {
        best = ms;
        best_cfg = timed[i].second;
      }
    }
    p->cfg = best_cfg;
    p->tuned_ms = best < 1e30f ? best : 0.0f;
    p->tuning = false;
    rc = plan_prepare(p, s);
  }
  p->tuning = false;
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  cudaFree(vals);
  cudaFree(X);
  cudaFree(Y);
  cudaFree(flush);
  g_err.clear();
  return rc;
}

// gbs_plan_create with an optional permutation through which the values are read
// (perm != nullptr: the plan is restricted to the ROWS and MERGE_DIRECT variants).
int plan_create_impl(gbs_plan** plan, int m, int n, int nnz, const int* row_ptr, const int* col_idx, int dtype, int k,
                     int flags, const int* perm, void* stream) {
  if (plan == nullptr) return fail(GBS_EINVAL, "plan is NULL");
  *plan = nullptr;
  if (!valid_dtype(dtype)) return fail(GBS_EDTYPE, "dtype");
  int rc = check_csr(m, n, nnz, row_ptr, col_idx, reinterpret_cast<const void*>(1));
  if (rc) return rc;
  if (k < 1) return fail(GBS_EINVAL, "k must be >= 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((flags & GBS_PLAN_CHECK) || checked_mode()) {
    rc = gbs_validate_csr(m, n, nnz, row_ptr, col_idx, stream);
    if (rc) return rc;
  }
  gbs_plan* p = new (std::nothrow) gbs_plan();
  if (!p) return fail(GBS_ENOMEM, "host allocation");
  p->m = m;
  p->n = n;
  p->nnz = nnz;
  p->k = k;
  p->dtype = dtype;
  p->row_ptr = row_ptr;
  p->col_idx = col_idx;
  p->flags = flags;
  p->perm = perm;
  cudaGetDevice(&p->device);
  if (cudaMalloc(reinterpret_cast<void**>(&p->status), 256) != cudaSuccess ||
      cudaMemsetAsync(p->status, 0, 256, s) != cudaSuccess) {
    if (p->status) cudaFree(p->status);
    delete p;
    return fail(GBS_ENOMEM, "plan status word");
  }
  rc = compute_stats(m, n, nnz, row_ptr, &p->stats, s);
  if (rc == GBS_OK) {
    p->cfg = heuristic_config(p->stats, dtype, k);
    // values through a permutation: the direct merge form gathers them in its walk, with
    // more of them in flight than the staged form's synchronous gather (the tuner may still
    // pick the staged form)
    if (perm && p->cfg.variant == GBS_VARIANT_MERGE) p->cfg.variant = GBS_VARIANT_MERGE_DIRECT;
    rc = (flags & GBS_PLAN_TUNE) && m > 0 ? plan_tune(p, s) : plan_prepare(p, s);
  }
  if (rc != GBS_OK) {
    relabel_release(p);
    if (p->mb.base) cudaFree(p->mb.base);
    cudaFree(p->status);
    delete p;
    return rc;
  }
  *plan = p;
  return GBS_OK;
}

}  // namespace

extern "C" {

int gbs_plan_create(gbs_plan** plan, int m, int n, int nnz, const int* row_ptr, const int* col_idx, int dtype, int k,
                    int flags, void* stream) {
  return plan_create_impl(plan, m, n, nnz, row_ptr, col_idx, dtype, k, flags, nullptr, stream);
}

int gbs_plan_destroy(gbs_plan* plan) {
  if (!plan) return GBS_OK;
  relabel_release(plan);
  if (plan->mb.base) cudaFree(plan->mb.base);
  if (plan->status) cudaFree(plan->status);
  delete plan;
  return GBS_OK;
}

int gbs_plan_status(gbs_plan* plan, int* status, void* stream) {
  if (!plan || !status) return fail(GBS_EINVAL, "NULL pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(status, plan->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(plan->status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? GBS_OK : cuda_fail(e, "plan status");
}

int gbs_plan_get_config(const gbs_plan* plan, gbs_config* cfg) {
  if (!plan || !cfg) return fail(GBS_EINVAL, "NULL pointer");
  *cfg = plan->cfg;
  return GBS_OK;
}

int gbs_plan_get_stats(const gbs_plan* plan, gbs_stats* out) {
  if (!plan || !out) return fail(GBS_EINVAL, "NULL pointer");
  *out = plan->stats;
  return GBS_OK;
}

int gbs_plan_relabel_ids(const gbs_plan* plan, int* newid, void* stream) {
  if (!plan || (!newid && plan->n > 0)) return fail(GBS_EINVAL, "NULL pointer");
  if (plan->cfg.relabel == 0 || (!plan->newid && plan->n > 0)) return fail(GBS_EINVAL, "the plan does not relabel");
  if (plan->n == 0) return GBS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(newid, plan->newid, sizeof(int) * (size_t)plan->n, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? GBS_OK : cuda_fail(e, "relabel export");
}

int gbs_plan_set_config(gbs_plan* plan, const gbs_config* cfg) {
  if (!plan || !cfg) return fail(GBS_EINVAL, "NULL pointer");
  gbs_config c = cfg->variant == GBS_VARIANT_AUTO ? heuristic_config(plan->stats, plan->dtype, plan->k)
                                                  : normalize(*cfg, plan->dtype);
  int rc = check_cfg(c);
  if (rc) return rc;
  plan->cfg = c;
  return plan_prepare(plan, nullptr);
}

int spmv_csr_plan(const gbs_plan* plan, const void* vals, const void* x, void* y, void* stream) {
  if (!plan) return fail(GBS_EINVAL, "plan is NULL");
  if (plan->k != 1) return fail(GBS_EINVAL, "plan was made for k > 1: use spmm_csr_plan");
  if ((plan->nnz > 0 && (!vals || !x)) || (plan->m > 0 && !y)) return fail(GBS_EINVAL, "NULL pointer");
  return plan_run(plan, vals, x, 1, y, 1, static_cast<cudaStream_t>(stream));
}

int spmm_csr_plan(const gbs_plan* plan, const void* vals, const void* X, int ldx, void* Y, int ldy, void* stream) {
  if (!plan) return fail(GBS_EINVAL, "plan is NULL");
  if (ldx < plan->k || ldy < plan->k) return fail(GBS_EINVAL, "leading dimension smaller than k");
  if ((plan->nnz > 0 && (!vals || !X)) || (plan->m > 0 && !Y)) return fail(GBS_EINVAL, "NULL pointer");
  return plan_run(plan, vals, X, ldx, Y, ldy, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

// ======================================================= transpose + backward

struct gbs_tplan {
  int m = 0, n = 0, nnz = 0, device = 0;
  int* rptrT = nullptr;      // n + 1
  int* colT = nullptr;       // nnz
  int* perm = nullptr;       // nnz
  int* rows = nullptr;       // nnz: row of every nonzero of A (the dvals pass)
  void* base = nullptr;
  void* valsT = nullptr;     // nnz values, only for a prepared plan that permutes the values first
  gbs_stats statsT{};
  struct Prepared {
    int dtype, k;
    gbs_plan* plan;  // plan of A^T: reads A's values through perm, or valsT if `gather`
    bool gather;
  };
  std::vector<Prepared> plans;  // one per (dtype, k), made by gbs_tplan_prepare
  // the dvals pass runs on this plan-owned stream, forked from and joined back into the
  // caller's stream, concurrently with the dX product
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace {
size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Time `fn` (enqueued on s) as the median of 3 runs after one warm-up; returns ms or -1.
template <typename F>
float time_median(F fn, cudaStream_t s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return -1.0f;
  }
  float t[3] = {0, 0, 0};
  bool ok = true;
  for (int r = 0; r < 4 && ok; ++r) {
    ok = cudaEventRecord(e0, s) == cudaSuccess && fn() && cudaEventRecord(e1, s) == cudaSuccess &&
         cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0;
    if (ok) cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0) t[r - 1] = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return -1.0f;
  std::sort(t, t + 3);
  return t[1];
}

// Keep `plan` as the prepared plan of A^T for (dtype, k), replacing an earlier one.
int tplan_install(gbs_tplan* t, int dtype, int k, gbs_plan* plan, bool gather) {
  if (gather && !t->valsT && cudaMalloc(&t->valsT, (size_t)std::max(t->nnz, 1) * 8) != cudaSuccess) {
    t->valsT = nullptr;
    gbs_plan_destroy(plan);
    return fail(GBS_ENOMEM, "cudaMalloc (permuted values)");
  }
  for (auto& pp : t->plans)
    if (pp.dtype == dtype && pp.k == k) {
      gbs_plan_destroy(pp.plan);
      pp.plan = plan;
      pp.gather = gather;
      return GBS_OK;
    }
  t->plans.push_back({dtype, k, plan, gather});
  return GBS_OK;
}
}  // namespace

extern "C" {

int gbs_transpose_plan(gbs_tplan** out, int m, int n, int nnz, const int* row_ptr, const int* col_idx, void* stream) {
  if (!out) return fail(GBS_EINVAL, "plan is NULL");
  *out = nullptr;
  int rc = check_csr(m, n, nnz, row_ptr, col_idx, reinterpret_cast<const void*>(1));
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (checked_mode()) {
    rc = gbs_validate_csr(m, n, nnz, row_ptr, col_idx, stream);
    if (rc) return rc;
  }
  gbs_tplan* t = new (std::nothrow) gbs_tplan();
  if (!t) return fail(GBS_ENOMEM, "host allocation");
  t->m = m;
  t->n = n;
  t->nnz = nnz;
  cudaGetDevice(&t->device);
  const size_t z = (size_t)std::max(nnz, 1);
  size_t b_rptr = align256(sizeof(int) * ((size_t)n + 1)), b_i = align256(sizeof(int) * z);
  size_t keep = b_rptr + 3 * b_i;
  size_t b_hist = align256(sizeof(int) * transpose_hist_ints(nnz));
  size_t b_scan = align256(sizeof(int) * transpose_scan_ws_ints(nnz));
  size_t tmp = 4 * b_i + b_hist + b_scan;
  cudaError_t e = cudaMalloc(&t->base, keep);
  if (e != cudaSuccess) {
    delete t;
    return cuda_fail(e, "cudaMalloc (transpose plan)");
  }
  char* p = static_cast<char*>(t->base);
  t->rptrT = reinterpret_cast<int*>(p);
  p += b_rptr;
  t->colT = reinterpret_cast<int*>(p);
  p += b_i;
  t->perm = reinterpret_cast<int*>(p);
  p += b_i;
  t->rows = reinterpret_cast<int*>(p);
  void* work = nullptr;
  e = cudaMallocAsync(&work, tmp, s);
  if (e == cudaSuccess) {
    char* w = static_cast<char*>(work);
    int* ka = reinterpret_cast<int*>(w);
    int* kb = reinterpret_cast<int*>(w + b_i);
    int* va = reinterpret_cast<int*>(w + 2 * b_i);
    int* vb = reinterpret_cast<int*>(w + 3 * b_i);
    int* hist = reinterpret_cast<int*>(w + 4 * b_i);
    int* ws = reinterpret_cast<int*>(w + 4 * b_i + b_hist);
    e = transpose_run(m, n, nnz, row_ptr, col_idx, t->rptrT, t->colT, t->perm, t->rows, ka, kb, va, vb, hist, ws, s);
    cudaError_t e2 = cudaFreeAsync(work, s);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(t->base);
    delete t;
    return cuda_fail(e, "transpose");
  }
  rc = compute_stats(n, m, nnz, t->rptrT, &t->statsT, s);
  if (rc == GBS_OK) {
    e = cudaStreamCreateWithFlags(&t->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) rc = cuda_fail(e, "backward stream and events");
  }
  if (rc) {
    gbs_tplan_destroy(t);
    return rc;
  }
  *out = t;
  return GBS_OK;
}

int gbs_tplan_arrays(const gbs_tplan* t, const int** rowptrT, const int** colT, const int** perm) {
  if (!t) return fail(GBS_EINVAL, "plan is NULL");
  if (rowptrT) *rowptrT = t->rptrT;
  if (colT) *colT = t->colT;
  if (perm) *perm = t->perm;
  return GBS_OK;
}

int gbs_tplan_export(const gbs_tplan* t, int* rowptrT, int* colT, int* perm, void* stream) {
  if (!t) return fail(GBS_EINVAL, "plan is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (rowptrT) e = cudaMemcpyAsync(rowptrT, t->rptrT, sizeof(int) * ((size_t)t->n + 1), cudaMemcpyDefault, s);
  if (e == cudaSuccess && colT && t->nnz)
    e = cudaMemcpyAsync(colT, t->colT, sizeof(int) * (size_t)t->nnz, cudaMemcpyDefault, s);
  if (e == cudaSuccess && perm && t->nnz)
    e = cudaMemcpyAsync(perm, t->perm, sizeof(int) * (size_t)t->nnz, cudaMemcpyDefault, s);
  return e == cudaSuccess ? GBS_OK : cuda_fail(e, "tplan export");
}

int gbs_tplan_destroy(gbs_tplan* t) {
  if (!t) return GBS_OK;
  if (t->ev_fork) cudaEventDestroy(t->ev_fork);
  if (t->ev_join) cudaEventDestroy(t->ev_join);
  if (t->side) cudaStreamDestroy(t->side);
  for (auto& pp : t->plans) gbs_plan_destroy(pp.plan);
  if (t->valsT) cudaFree(t->valsT);
  if (t->base) cudaFree(t->base);
  delete t;
  return GBS_OK;
}

int gbs_tplan_prepare(gbs_tplan* t, int dtype, int k, int flags, void* stream) {
  if (!t) return fail(GBS_EINVAL, "plan is NULL");
  if (!valid_dtype(dtype)) return fail(GBS_EDTYPE, "dtype");
  if (k < 1) return fail(GBS_EINVAL, "k must be >= 1");
  for (auto& pp : t->plans)
    if (pp.dtype == dtype && pp.k == k) return GBS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  flags &= ~GBS_PLAN_CHECK;
  gbs_plan* pp = nullptr;  // A^T reading A's values through perm
  int rc = plan_create_impl(&pp, t->n, t->m, t->nnz, t->rptrT, t->colT, dtype, k, flags, t->perm, stream);
  if (rc) return rc;
  bool gather = false;
  gbs_plan* pg = nullptr;  // A^T on values permuted by a separate gather
  if ((flags & GBS_PLAN_TUNE) && t->nnz > 0 && pp->tuned_ms > 0) {
    // the alternative route: permute the values once per call, then the best plain plan of A^T
    rc = plan_create_impl(&pg, t->n, t->m, t->nnz, t->rptrT, t->colT, dtype, k, flags, nullptr, stream);
    if (rc == GBS_OK && pg->tuned_ms > 0 && pg->tuned_ms < pp->tuned_ms) {
      void *src = nullptr, *dst = nullptr;
      const size_t bytes = (size_t)t->nnz * dsize(dtype);
      float tg = -1.0f;
      if (cudaMalloc(&src, bytes) == cudaSuccess && cudaMalloc(&dst, bytes) == cudaSuccess &&
          cudaMemsetAsync(src, 0, bytes, s) == cudaSuccess)
        tg = time_median([&] { return gather_values(dtype, src, t->perm, t->nnz, dst, s) == cudaSuccess; }, s);
      if (src) cudaFree(src);
      if (dst) cudaFree(dst);
      gather = tg >= 0 && tg + pg->tuned_ms < pp->tuned_ms;
    }
    if (tune_log())
      std::fprintf(stderr, "gbspmv tplan prepare k=%d: through perm %.4f ms, gather + plain %s\n", k, pp->tuned_ms,
                   gather ? "chosen" : "not chosen");
    g_err.clear();
    rc = GBS_OK;
  }
  if (gather) {
    gbs_plan_destroy(pp);
    return tplan_install(t, dtype, k, pg, true);
  }
  if (pg) gbs_plan_destroy(pg);
  return tplan_install(t, dtype, k, pp, false);
}

int gbs_tplan_set_config(gbs_tplan* t, int dtype, int k, const gbs_config* cfg, void* stream) {
  if (!t || !cfg) return fail(GBS_EINVAL, "NULL pointer");
  if (!valid_dtype(dtype)) return fail(GBS_EDTYPE, "dtype");
  if (k < 1) return fail(GBS_EINVAL, "k must be >= 1");
  if (cfg->variant == GBS_VARIANT_ROWS_DIRECT)
    return fail(GBS_EUNSUPPORTED, "ROWS_DIRECT does not read values through the transpose permutation");
  const bool gather = cfg->variant == GBS_VARIANT_ROWS_TMA;
  gbs_plan* p = nullptr;
  int rc = plan_create_impl(&p, t->n, t->m, t->nnz, t->rptrT, t->colT, dtype, k, 0, gather ? nullptr : t->perm,
                            stream);
  if (rc) return rc;
  if (cfg->variant != GBS_VARIANT_AUTO) {
    rc = gbs_plan_set_config(p, cfg);
    if (rc) {
      gbs_plan_destroy(p);
      return rc;
    }
  }
  return tplan_install(t, dtype, k, p, gather);
}

int gbs_tplan_get_config(const gbs_tplan* t, int dtype, int k, gbs_config* cfg) {
  if (!t || !cfg) return fail(GBS_EINVAL, "NULL pointer");
  for (auto& pp : t->plans)
    if (pp.dtype == dtype && pp.k == k) return gbs_plan_get_config(pp.plan, cfg);
  if (!valid_dtype(dtype) || k < 1) return fail(GBS_EINVAL, "dtype or k");
  gbs_config c = heuristic_config(t->statsT, dtype, k);
  if (c.variant == GBS_VARIANT_MERGE) c.variant = GBS_VARIANT_MERGE_DIRECT;
  *cfg = c;
  return GBS_OK;
}

int spmv_csr_backward(gbs_tplan* t, const int* row_ptr, const int* col_idx, const void* vals, int dtype, int k,
                      const void* X, int ldx, const void* dY, int lddy, void* dX, int lddx, void* dvals,
                      void* stream) {
  if (!t) return fail(GBS_EINVAL, "plan is NULL");
  if (!valid_dtype(dtype)) return fail(GBS_EDTYPE, "dtype");
  if (k < 1 || ldx < k || lddy < k || (dX && lddx < k)) return fail(GBS_EINVAL, "k or leading dimension");
  if (t->nnz > 0 && (!col_idx || !vals)) return fail(GBS_EINVAL, "col_idx or vals is NULL");
  if (dvals && t->nnz > 0 && (!X || !dY)) return fail(GBS_EINVAL, "X or dY is NULL");
  if (dX && t->m > 0 && !dY) return fail(GBS_EINVAL, "dY is NULL");
  (void)row_ptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  // both outputs: the dvals pass runs on the plan's side stream while dX runs on `stream`; the
  // two read the same inputs and write different outputs, and `stream` waits for the side
  // stream before anything after this call
  const bool fork = dX && dvals && t->nnz > 0 && t->side;
  if (fork) {
    e = cudaEventRecord(t->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(t->side, t->ev_fork, 0);
    if (e == cudaSuccess)
      e = launch_sddmm(dtype, t->nnz, k, t->rows, col_idx, X, k == 1 ? 1 : ldx, dY, k == 1 ? 1 : lddy, dvals, t->side);
    if (e == cudaSuccess) e = cudaEventRecord(t->ev_join, t->side);
    if (e != cudaSuccess) return cuda_fail(e, "SDDMM launch (side stream)");
  }
  if (dX) {
    // dX = A^T dY on the precomputed transpose
    const gbs_tplan::Prepared* prepared = nullptr;
    for (auto& pp : t->plans)
      if (pp.dtype == dtype && pp.k == k) prepared = &pp;
    int rc;
    if (prepared && prepared->gather) {
      e = gather_values(dtype, vals, t->perm, t->nnz, t->valsT, s);
      if (e != cudaSuccess) return cuda_fail(e, "gather of A^T values");
      rc = plan_run(prepared->plan, t->valsT, dY, k == 1 ? 1 : lddy, dX, k == 1 ? 1 : lddx, s);
    } else if (prepared) {
      rc = plan_run(prepared->plan, vals, dY, k == 1 ? 1 : lddy, dX, k == 1 ? 1 : lddx, s);
    } else {
      // A's values read in place through perm, configuration from A^T's row statistics
      CsrView AT{t->n, t->m, t->nnz, t->rptrT, t->colT, vals, t->perm};
      gbs_config c = heuristic_config(t->statsT, dtype, k);
      if (c.variant == GBS_VARIANT_MERGE) c.variant = GBS_VARIANT_MERGE_DIRECT;
      rc = run_product(AT, dtype, k, dY, k == 1 ? 1 : lddy, dX, k == 1 ? 1 : lddx, c, nullptr, false, s);
    }
    if (rc) {
      if (fork) cudaStreamWaitEvent(s, t->ev_join, 0);  // never leave the side stream unjoined
      return rc;
    }
  }
  if (fork) {
    e = cudaStreamWaitEvent(s, t->ev_join, 0);
    if (e != cudaSuccess) return cuda_fail(e, "join of the side stream");
  } else if (dvals) {
    e = launch_sddmm(dtype, t->nnz, k, t->rows, col_idx, X, k == 1 ? 1 : ldx, dY, k == 1 ? 1 : lddy, dvals, s);
    if (e != cudaSuccess) return cuda_fail(e, "SDDMM launch");
  }
  return GBS_OK;
}

}  // extern "C"

// ===================================================================== BCSR

struct gbs_bcsr {
  int m = 0, n = 0, a = 1, b = 1, mb = 0, dtype = GBS_F64, device = 0;
  long long nblocks = 0;
  int* bptr = nullptr;
  int* bcol = nullptr;
  void* bval = nullptr;
};

namespace {
bool block_dim_ok(int d) { return d == 1 || d == 2 || d == 4 || d == 8; }
void bcsr_free(gbs_bcsr* h) {
  if (h->bptr) cudaFree(h->bptr);
  if (h->bcol) cudaFree(h->bcol);
  if (h->bval) cudaFree(h->bval);
  delete h;
}
}  // namespace

extern "C" {

int gbs_bcsr_create(gbs_bcsr** out, int m, int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals,
                    int dtype, int a, int b, void* stream) {
  if (!out) return fail(GBS_EINVAL, "plan is NULL");
  *out = nullptr;
  if (!valid_dtype(dtype)) return fail(GBS_EDTYPE, "dtype");
  int rc = check_csr(m, n, nnz, row_ptr, col_idx, vals);
  if (rc) return rc;
  if (!block_dim_ok(a) || !block_dim_ok(b)) return fail(GBS_EUNSUPPORTED, "block dimensions must be 1, 2, 4 or 8");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (checked_mode()) {
    rc = gbs_validate_csr(m, n, nnz, row_ptr, col_idx, stream);
    if (rc) return rc;
  }
  gbs_bcsr* h = new (std::nothrow) gbs_bcsr();
  if (!h) return fail(GBS_ENOMEM, "host allocation");
  h->m = m;
  h->n = n;
  h->a = a;
  h->b = b;
  h->mb = (m + a - 1) / a;
  h->dtype = dtype;
  cudaGetDevice(&h->device);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&h->bptr), sizeof(int) * ((size_t)h->mb + 1));
  if (e != cudaSuccess) {
    bcsr_free(h);
    return cuda_fail(e, "cudaMalloc (block row pointers)");
  }
  int* sorted = nullptr;
  void* scratch = nullptr;
  int nb = 0;
  e = bcsr_count(m, n, nnz, row_ptr, col_idx, a, b, h->bptr, &sorted, &nb, &scratch, s);
  if (e == cudaSuccess) {
    h->nblocks = nb;
    const size_t vbytes = (size_t)nb * a * b * dsize(dtype);
    e = cudaMalloc(reinterpret_cast<void**>(&h->bcol), sizeof(int) * (size_t)std::max(nb, 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->bval, std::max<size_t>(vbytes, 16));
    if (e == cudaSuccess)
      e = bcsr_fill(m, n, nnz, row_ptr, col_idx, vals, dtype, a, b, h->bptr, h->bcol, h->bval, nb, scratch, s);
  }
  if (scratch) {
    cudaError_t e2 = cudaFreeAsync(scratch, s);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    bcsr_free(h);
    return cuda_fail(e, "BCSR conversion");
  }
  *out = h;
  return GBS_OK;
}

int gbs_bcsr_info(const gbs_bcsr* h, int* block_rows, long long* nblocks, int* a, int* b) {
  if (!h) return fail(GBS_EINVAL, "plan is NULL");
  if (block_rows) *block_rows = h->mb;
  if (nblocks) *nblocks = h->nblocks;
  if (a) *a = h->a;
  if (b) *b = h->b;
  return GBS_OK;
}

int gbs_bcsr_arrays(const gbs_bcsr* h, const int** bptr, const int** bcol, const void** bval) {
  if (!h) return fail(GBS_EINVAL, "plan is NULL");
  if (bptr) *bptr = h->bptr;
  if (bcol) *bcol = h->bcol;
  if (bval) *bval = h->bval;
  return GBS_OK;
}

int spmv_bcsr(const gbs_bcsr* h, const void* x, void* y, void* stream) {
  if (!h) return fail(GBS_EINVAL, "plan is NULL");
  if ((h->m > 0 && !y) || (h->nblocks > 0 && !x)) return fail(GBS_EINVAL, "x or y is NULL");
  cudaError_t e = bcsr_spmv(h->dtype, h->a, h->b, h->m, h->n, h->bptr, h->bcol, h->bval, x, y,
                            static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GBS_OK : cuda_fail(e, "BCSR SpMV launch");
}

int gbs_bcsr_destroy(gbs_bcsr* h) {
  if (h) bcsr_free(h);
  return GBS_OK;
}

}  // extern "C"

// ================================================================== batched

struct gbs_batch_plan {
  int nmat = 0, dtype = GBS_F64, k = 1, device = 0;
  bool split = true, vec16 = false;
  int G = 1;
  std::vector<gbs_batch_item> items;
  std::vector<gbs_config> cfgs;
  std::vector<gbs_stats> stats;  // row statistics of each matrix
  std::vector<int> item_begin;  // nmat + 1
  std::vector<MergeBuffers> mbs;
  std::vector<unsigned char> h_desc;
  void* d_desc = nullptr;
  void* scratch = nullptr;
  int* next_item = nullptr;  // device work counter, reset by the graph before every launch
  size_t smem = 0;
  int grid = 0, total_items = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

constexpr int kBatchThreads = 256;
// Shared memory per CTA of the batched kernel: four 256-thread CTAs per SM (the kernel is
// compiled for four) fit in 228 KB with 1 KB reserved per CTA.
constexpr size_t kBatchSmemBudget = 54 * 1024;

size_t rows_smem_host(int dtype, int rpc, int tile) {
  return dtype == GBS_F64 ? rows_smem_bytes<double>(rpc, tile) : rows_smem_bytes<float>(rpc, tile);
}
size_t merge_smem_host(int dtype, int g, bool vec16, int items, bool direct) {
  const int vec = vec16 ? vec_of(dtype) : 1;
  const int nt = kBatchThreads / g;
  const size_t es = dsize(dtype);
  const size_t ipc = (size_t)nt * items;
  size_t a = direct ? 0 : ((ipc + 2) * sizeof(int) + 15) & ~(size_t)15;
  size_t b = direct ? 0 : ((ipc + 4) * es + 15) & ~(size_t)15;
  size_t c = direct ? 0 : ((ipc + 4) * sizeof(int) + 15) & ~(size_t)15;
  return a + b + c + 2 * (size_t)(kBatchThreads / 32) * sizeof(int) + 2 * (size_t)(kBatchThreads / 32) * g * vec * es;
}

template <typename T>
void fill_desc(gbs_batch_plan* p, int b, BatchDesc<T>* d) {
  const gbs_batch_item& it = p->items[b];
  const gbs_config& c = p->cfgs[b];
  std::memset(d, 0, sizeof(*d));
  d->m = it.m;
  d->n = it.n;
  d->nnz = it.nnz;
  d->k = p->k;
  d->row_ptr = it.row_ptr;
  d->col_idx = it.col_idx;
  d->vals = static_cast<const T*>(it.vals);
  d->X = static_cast<const T*>(it.X);
  d->Y = static_cast<T*>(it.Y);
  d->ldx = p->k == 1 ? 1 : it.ldx;
  d->ldy = p->k == 1 ? 1 : it.ldy;
  d->variant = c.variant;
  d->lanes = p->split ? c.lanes : p->G;
  d->tile = c.tile_nnz;
  d->items = c.items;
  d->item_begin = p->item_begin[b];
  d->nitems = p->item_begin[b + 1] - p->item_begin[b];
  if (is_merge(c.variant)) {
    d->coords = p->mbs[b].s.coords;
    d->carry_row = p->mbs[b].s.carry_row;
    d->carry_val = static_cast<T*>(p->mbs[b].s.carry_val);
    d->done = reinterpret_cast<int*>(static_cast<char*>(p->mbs[b].base) + p->mbs[b].bytes - sizeof(int));
  }
  d->aligned_vals = aligned16(it.vals);
  d->aligned_cols = aligned16(it.col_idx);
}

void batch_free(gbs_batch_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->d_desc) cudaFree(p->d_desc);
  if (p->scratch) cudaFree(p->scratch);
  if (p->next_item) cudaFree(p->next_item);
  delete p;
}

// Per-matrix configuration for the batch: 256 threads; k > 1 uses the plan's column lanes.
std::vector<gbs_config> batch_candidates(const gbs_stats& st, int dtype, int k) {
  std::vector<gbs_config> c;
  const int base_tile = dtype == GBS_F64 ? 2048 : 3072;
  auto add = [&](int variant, int lanes, int tile, int items) {
    gbs_config g{};
    g.variant = variant;
    g.lanes = lanes;
    g.threads = kBatchThreads;
    g.tile_nnz = tile;
    g.items = items;
    c.push_back(g);
  };
  if (k == 1) {
    for (int l : {1, 2, 4, 8, 16, 32})
      if (l == 1 || st.mean_row >= 0.5 * l) add(GBS_VARIANT_ROWS, l, base_tile, 0);
    for (int it : {7, 15, 31}) add(GBS_VARIANT_MERGE, 0, 0, it);
  } else {
    add(GBS_VARIANT_ROWS, 0, base_tile, 0);
    add(GBS_VARIANT_ROWS, 0, base_tile / 2, 0);
    add(GBS_VARIANT_ROWS, 0, base_tile * 2, 0);
    add(GBS_VARIANT_MERGE, 0, 0, 0);
    add(GBS_VARIANT_MERGE, 0, 0, 15);
  }
  return c;
}

// Largest odd merge items per thread (at most `items`, at least 3) whose shared memory fits
// the batched kernel's budget.
int batch_cap_items(int dtype, int g, bool vec16, int items) {
  int it = std::max(3, items | 1);
  while (it > 3 && merge_smem_host(dtype, g, vec16, it, false) > kBatchSmemBudget) it -= 2;
  return it;
}

}  // namespace

extern "C" {

int spmv_csr_batched_plan(gbs_batch_plan** out, int nmat, const gbs_batch_item* items, int dtype, int k, int flags,
                          void* stream) {
  int rc = spmv_csr_batched_plan_cfg(out, nmat, items, dtype, k, flags, nullptr, stream);
  if (rc || !(flags & GBS_PLAN_TUNE) || !*out || !(*out)->exec) return rc;
  // Standalone timings of a small matrix measure its launch latency, not what its items cost
  // inside a full batch.  So whole-batch policies are also built and timed on the batched
  // kernel itself, and the fastest plan is kept (the per-matrix choice is one of them).  A
  // policy starts from the per-matrix choice or from the statistics' variant (ROWS with a given
  // tile, MERGE for skewed rows), and sends matrices whose mean row is shorter than a threshold
  // to MERGE; MERGE tiles take a given number of items per thread (then capped to the budget).
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  gbs_batch_plan* best = *out;
  auto time_plan = [&](gbs_batch_plan* q) {
    return time_median([&] { return cudaGraphLaunch(q->exec, s) == cudaSuccess; }, s);
  };
  float best_ms = time_plan(best);
  if (best_ms < 0) best_ms = 1e30f;
  const std::vector<gbs_config> tuned = best->cfgs;
  const std::vector<gbs_stats> stats = best->stats;
  const int base_tile = dtype == GBS_F64 ? 2048 : 3072;
  struct Policy {
    bool from_stats;  // statistics' variant (else the per-matrix choice)
    int rows_tile;    // ROWS tile when from_stats
    double short_row; // mean row below which a matrix takes `short_variant` (0: none)
    int merge_items;  // items per merge thread for the MERGE matrices (0: default)
    int short_variant;  // MERGE, or ROWS_DIRECT (no staging, no barriers)
  };
  std::vector<Policy> policies;
  // (on the 512-matrix k = 8 batch every policy was slower with merge tiles larger or smaller
  // than the default, and with ROWS_DIRECT matrices, whether for the short rows or for all the
  // statistics' ROWS matrices, so neither is tried)
  for (double thr : {0.0, 8.0, 12.0, 20.0}) {
    policies.push_back({false, 0, thr, 0, GBS_VARIANT_MERGE});
    for (int t : {base_tile, 2 * base_tile}) policies.push_back({true, t, thr, 0, GBS_VARIANT_MERGE});
  }
  int pol_id = 0;
  for (const Policy& pol : policies) {
    ++pol_id;
    if (!pol.from_stats && pol.short_row == 0.0 && pol.merge_items == 0) continue;  // the per-matrix choice
    std::vector<gbs_config> cf(nmat);
    for (int b = 0; b < nmat; ++b) {
      const gbs_stats& st = stats[b];
      gbs_config c = tuned[b];
      if (pol.from_stats) {
        c = heuristic_config(st, dtype, k);
        if (c.variant == GBS_VARIANT_ROWS) c.tile_nnz = pol.rows_tile;
      }
      if (pol.short_row > 0.0 && st.mean_row < pol.short_row) {
        c = gbs_config{};
        c.variant = pol.short_variant;
      }
      if (c.variant == GBS_VARIANT_MERGE && (pol.from_stats || pol.short_row > 0.0 || pol.merge_items > 0))
        c.items = pol.merge_items;
      c.threads = kBatchThreads;
      cf[b] = c;
    }
    gbs_batch_plan* q = nullptr;
    if (spmv_csr_batched_plan_cfg(&q, nmat, items, dtype, k, flags & ~GBS_PLAN_TUNE, cf.data(), stream) != GBS_OK ||
        !q || !q->exec) {
      if (q) batch_free(q);
      continue;
    }
    const float ms = time_plan(q);
    if (tune_log())
      std::fprintf(stderr, "gbspmv batch policy %d (stats %d tile %d short<%.0f -> variant %d, items %d): %.4f ms "
                   "(best %.4f ms)\n", pol_id, (int)pol.from_stats, pol.rows_tile, pol.short_row, pol.short_variant,
                   pol.merge_items, ms, best_ms);
    if (ms > 0 && ms < best_ms) {
      batch_free(best);
      best = q;
      best_ms = ms;
    } else {
      batch_free(q);
    }
  }
  *out = best;
  g_err.clear();
  return GBS_OK;
}

int spmv_csr_batched_plan_cfg(gbs_batch_plan** out, int nmat, const gbs_batch_item* items, int dtype, int k,
                              int flags, const gbs_config* cfgs, void* stream) {
  if (!out) return fail(GBS_EINVAL, "plan is NULL");
  *out = nullptr;
  if (nmat < 1 || !items) return fail(GBS_EINVAL, "nmat must be >= 1 and items non-NULL");
  if (!valid_dtype(dtype)) return fail(GBS_EDTYPE, "dtype");
  if (k < 1) return fail(GBS_EINVAL, "k must be >= 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t es = dsize(dtype);
  bool vec16 = k > 1;
  for (int b = 0; b < nmat; ++b) {
    const gbs_batch_item& it = items[b];
    int rc = check_csr(it.m, it.n, it.nnz, it.row_ptr, it.col_idx, it.vals);
    if (rc) return fail(rc, "item " + std::to_string(b) + ": " + g_err);
    if (k > 1 && (it.ldx < k || it.ldy < k)) return fail(GBS_EINVAL, "item " + std::to_string(b) + ": ld < k");
    if ((it.m > 0 && !it.Y) || (it.nnz > 0 && !it.X)) return fail(GBS_EINVAL, "item " + std::to_string(b) + ": NULL X/Y");
    if (k > 1) vec16 = vec16 && dense_vec16(dtype, k, it.X, it.ldx, it.Y, it.ldy);
    if ((reinterpret_cast<uintptr_t>(it.vals) % es) || (reinterpret_cast<uintptr_t>(it.X) % es) ||
        (reinterpret_cast<uintptr_t>(it.Y) % es))
      return fail(GBS_EALIGN, "item " + std::to_string(b) + ": arrays must be aligned to their element size");
    if ((flags & GBS_PLAN_CHECK) || checked_mode()) {
      rc = gbs_validate_csr(it.m, it.n, it.nnz, it.row_ptr, it.col_idx, stream);
      if (rc) return fail(rc, "item " + std::to_string(b) + ": " + g_err);
    }
  }
  if (k > panel_cols(dtype, vec16)) return fail(GBS_EUNSUPPORTED, "batched k wider than one column panel (32 lanes)");
  gbs_batch_plan* p = new (std::nothrow) gbs_batch_plan();
  if (!p) return fail(GBS_ENOMEM, "host allocation");
  p->nmat = nmat;
  p->dtype = dtype;
  p->k = k;
  p->split = k == 1;
  p->vec16 = vec16;
  p->G = k == 1 ? 1 : col_lanes(k, dtype, vec16);
  cudaGetDevice(&p->device);
  p->items.assign(items, items + nmat);
  p->cfgs.resize(nmat);
  p->stats.resize(nmat);
  p->mbs.resize(nmat);

  // ---- the caller's configurations: ROWS or MERGE, run by the batch's 256-thread CTAs
  std::vector<gbs_config> given_cfgs;
  if (cfgs) {
    given_cfgs.assign(cfgs, cfgs + nmat);
    for (int b = 0; b < nmat; ++b) {
      gbs_config& g = given_cfgs[b];
      if (g.variant == GBS_VARIANT_AUTO) continue;
      int rc = GBS_OK;
      if (g.variant != GBS_VARIANT_ROWS && g.variant != GBS_VARIANT_MERGE) {
        rc = fail(GBS_EUNSUPPORTED, "item " + std::to_string(b) + ": batched configurations are ROWS or MERGE");
      } else if (g.relabel != 0) {
        rc = fail(GBS_EUNSUPPORTED, "item " + std::to_string(b) + ": column relabelling is for plans of one matrix");
      } else {
        g.threads = kBatchThreads;
        g.emul = 0;
        if (g.variant == GBS_VARIANT_ROWS && k > 1) g.lanes = p->G;
        g = normalize(g, dtype);
        rc = check_cfg(g);
      }
      if (rc) {
        batch_free(p);
        return rc;
      }
    }
  }

  // ---- per-matrix configuration (given, heuristic, or timed with standalone launches)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  const bool tune = (flags & GBS_PLAN_TUNE) != 0;
  if (tune) {
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
  }
  for (int b = 0; b < nmat; ++b) {
    const gbs_batch_item& it = p->items[b];
    gbs_stats& st = p->stats[b];
    int rc = compute_stats(it.m, it.n, it.nnz, it.row_ptr, &st, s);
    if (rc) {
      batch_free(p);
      return rc;
    }
    gbs_config c = heuristic_config(st, dtype, k);
    c.threads = kBatchThreads;
    if (c.variant == GBS_VARIANT_ROWS && k > 1) c.lanes = p->G;
    const bool given = !given_cfgs.empty() && given_cfgs[b].variant != GBS_VARIANT_AUTO;
    if (given) c = given_cfgs[b];
    if (tune && !given && it.m > 0) {
      float best = 1e30f;
      for (gbs_config cand : batch_candidates(st, dtype, k)) {
        if (k > 1 && cand.variant == GBS_VARIANT_ROWS) cand.lanes = p->G;
        if (is_merge(cand.variant)) {
          // time the tile size the batch will run (capped to the shared-memory budget)
          const MergeGeom G = merge_geom(cand, it.m, it.nnz, dtype, k, vec16);
          cand.items = batch_cap_items(dtype, G.g, vec16, G.items);
        }
        CsrView A{it.m, it.n, it.nnz, it.row_ptr, it.col_idx, it.vals};
        float ms_sum = 0;
        bool ok = true;
        for (int r = 0; r < 3 && ok; ++r) {
          ok = cudaEventRecord(ev0, s) == cudaSuccess &&
               run_product(A, dtype, k, it.X, k == 1 ? 1 : it.ldx, it.Y, k == 1 ? 1 : it.ldy, cand, nullptr, false, s) ==
                   GBS_OK &&
               cudaEventRecord(ev1, s) == cudaSuccess && cudaEventSynchronize(ev1) == cudaSuccess;
          float ms = 0;
          if (ok && r > 0) {
            cudaEventElapsedTime(&ms, ev0, ev1);
            ms_sum += ms;
          }
        }
        if (ok && ms_sum < best) {
          best = ms_sum;
          c = cand;
        }
      }
    }
    p->cfgs[b] = c;
  }
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  g_err.clear();

  // ---- work list, shared memory, merge scratch
  p->item_begin.assign(nmat + 1, 0);
  size_t scratch_total = 0;
  std::vector<size_t> scratch_off(nmat, 0);
  for (int b = 0; b < nmat; ++b) {
    const gbs_batch_item& it = p->items[b];
    const gbs_config& c = p->cfgs[b];
    long long nitems = 0;
    if (c.variant == GBS_VARIANT_ROWS) {
      const int lanes = k == 1 ? c.lanes : p->G;
      const int rpc = kBatchThreads / lanes;
      nitems = (it.m + rpc - 1) / rpc;
      // the staged tile within the batch kernel's shared-memory budget
      while (p->cfgs[b].tile_nnz > 256 && rows_smem_host(dtype, rpc, p->cfgs[b].tile_nnz) > kBatchSmemBudget)
        p->cfgs[b].tile_nnz /= 2;
      p->smem = std::max(p->smem, rows_smem_host(dtype, rpc, p->cfgs[b].tile_nnz));
    } else {
      MergeGeom G = merge_geom(c, it.m, it.nnz, dtype, k, vec16);
      const int capped = batch_cap_items(dtype, G.g, vec16, G.items);
      if (capped != G.items) {
        p->cfgs[b].items = capped;
        G = merge_geom(p->cfgs[b], it.m, it.nnz, dtype, k, vec16);
      }
      p->cfgs[b].items = G.items;
      nitems = it.m > 0 ? G.ctas : 0;
      p->smem = std::max(p->smem, merge_smem_host(dtype, G.g, vec16, G.items, c.variant == GBS_VARIANT_MERGE_DIRECT));
      scratch_off[b] = scratch_total;
      const size_t bytes = align256(merge_scratch_bytes(G.ctas, G.kp_max, dtype) + sizeof(int));
      p->mbs[b].bytes = bytes;
      scratch_total += bytes;
    }
    if ((long long)p->item_begin[b] + nitems > 0x7fffffffLL) {
      batch_free(p);
      return fail(GBS_EUNSUPPORTED, "batch work list exceeds 2^31 items");
    }
    p->item_begin[b + 1] = p->item_begin[b] + (int)nitems;
  }
  p->total_items = p->item_begin[nmat];
  cudaError_t e = cudaSuccess;
  if (scratch_total) {
    e = cudaMalloc(&p->scratch, scratch_total);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->scratch, 0, scratch_total, s);
    for (int b = 0; b < nmat && e == cudaSuccess; ++b) {
      if (!is_merge(p->cfgs[b].variant)) continue;
      const gbs_batch_item& it = p->items[b];
      const MergeGeom G = merge_geom(p->cfgs[b], it.m, it.nnz, dtype, k, vec16);
      p->mbs[b].base = static_cast<char*>(p->scratch) + scratch_off[b];
      merge_carve(p->mbs[b], G.ctas, G.kp_max, dtype);
      if (it.m > 0) {
        CsrView A{it.m, it.n, it.nnz, it.row_ptr, it.col_idx, it.vals};
        e = launch_merge_partition(A, (long long)(kBatchThreads / G.g) * G.items, p->mbs[b].s, s);
      }
    }
  }
  // ---- descriptors
  const size_t dsz = dtype == GBS_F64 ? sizeof(BatchDesc<double>) : sizeof(BatchDesc<float>);
  p->h_desc.assign(dsz * nmat, 0);
  for (int b = 0; b < nmat; ++b) {
    if (dtype == GBS_F64)
      fill_desc<double>(p, b, reinterpret_cast<BatchDesc<double>*>(p->h_desc.data() + dsz * b));
    else
      fill_desc<float>(p, b, reinterpret_cast<BatchDesc<float>*>(p->h_desc.data() + dsz * b));
  }
  if (e == cudaSuccess) e = cudaMalloc(&p->d_desc, p->h_desc.size());
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->next_item), 256);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_desc, p->h_desc.data(), p->h_desc.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  // ---- persistent grid: every resident CTA slot of the GPU
  int bps = 0, sms = 0;
  if (e == cudaSuccess)
    e = batched_kernel_call(false, dtype, p->split, p->G, vec16, nullptr, 0, 0, nullptr, 0, p->smem, &bps, s);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  if (e != cudaSuccess) {
    batch_free(p);
    return cuda_fail(e, "batched plan");
  }
  p->grid = std::max(1, std::min(p->total_items, std::max(1, bps) * sms));
  // ---- capture the launch in a CUDA graph
  if (p->total_items > 0) {
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      // the work counter is zeroed by the graph itself, so every replay starts a fresh list
      cudaError_t el = cudaMemsetAsync(p->next_item, 0, sizeof(int), cs);
      if (el == cudaSuccess)
        el = batched_kernel_call(true, dtype, p->split, p->G, vec16, p->d_desc, nmat, p->total_items, p->next_item,
                                 p->grid, p->smem, nullptr, cs);
      e = cudaStreamEndCapture(cs, &p->graph);
      if (el != cudaSuccess) e = el;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      batch_free(p);
      return cuda_fail(e, "batched graph capture");
    }
  }
  *out = p;
  return GBS_OK;
}

int spmv_csr_batched(gbs_batch_plan* p, const void* const* X, void* const* Y, void* stream) {
  if (!p) return fail(GBS_EINVAL, "plan is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (X || Y) {
    // new dense operands: same shapes and alignment class as at plan time
    const size_t dsz = p->dtype == GBS_F64 ? sizeof(BatchDesc<double>) : sizeof(BatchDesc<float>);
    for (int b = 0; b < p->nmat; ++b) {
      if (X) p->items[b].X = X[b];
      if (Y) p->items[b].Y = Y[b];
      const gbs_batch_item& it = p->items[b];
      if ((it.m > 0 && !it.Y) || (it.nnz > 0 && !it.X)) return fail(GBS_EINVAL, "NULL X/Y");
      if (p->k > 1 && p->vec16 && !dense_vec16(p->dtype, p->k, it.X, it.ldx, it.Y, it.ldy))
        return fail(GBS_EALIGN, "X/Y lost the 16-byte alignment the plan was made for");
      if (p->dtype == GBS_F64)
        fill_desc<double>(p, b, reinterpret_cast<BatchDesc<double>*>(p->h_desc.data() + dsz * b));
      else
        fill_desc<float>(p, b, reinterpret_cast<BatchDesc<float>*>(p->h_desc.data() + dsz * b));
    }
    cudaError_t e = cudaMemcpyAsync(p->d_desc, p->h_desc.data(), p->h_desc.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host table may change again after return
    if (e != cudaSuccess) return cuda_fail(e, "descriptor update");
  }
  if (!p->exec) return GBS_OK;
  cudaError_t e = cudaGraphLaunch(p->exec, s);
  return e == cudaSuccess ? GBS_OK : cuda_fail(e, "cudaGraphLaunch");
}

int spmv_csr_batched_looped(gbs_batch_plan* p, void* stream) {
  if (!p) return fail(GBS_EINVAL, "plan is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int b = 0; b < p->nmat; ++b) {
    const gbs_batch_item& it = p->items[b];
    if (it.m == 0) continue;
    CsrView A{it.m, it.n, it.nnz, it.row_ptr, it.col_idx, it.vals};
    gbs_config c = p->cfgs[b];
    if (c.variant == GBS_VARIANT_ROWS && p->k > 1) c.lanes = p->G;
    MergeBuffers mb = p->mbs[b];
    int rc = run_product(A, p->dtype, p->k, it.X, p->k == 1 ? 1 : it.ldx, it.Y, p->k == 1 ? 1 : it.ldy, c,
                         is_merge(c.variant) ? &mb : nullptr, true, s);
    if (rc) return rc;
  }
  return GBS_OK;
}

int spmv_csr_batched_info(const gbs_batch_plan* p, gbs_config* cfgs, int* item_begin, int* grid, int* total_items) {
  if (!p) return fail(GBS_EINVAL, "plan is NULL");
  if (cfgs) std::copy(p->cfgs.begin(), p->cfgs.end(), cfgs);
  if (item_begin) std::copy(p->item_begin.begin(), p->item_begin.end(), item_begin);
  if (grid) *grid = p->grid;
  if (total_items) *total_items = p->total_items;
  return GBS_OK;
}

int spmv_csr_batched_offsets(const gbs_batch_plan* p, long long* off_rows, long long* off_nnz, long long* off_rptr,
                             long long* off_x, long long* off_y) {
  if (!p) return fail(GBS_EINVAL, "plan is NULL");
  long long r = 0, z = 0, rp = 0, xo = 0, yo = 0;
  for (int b = 0; b <= p->nmat; ++b) {
    if (off_rows) off_rows[b] = r;
    if (off_nnz) off_nnz[b] = z;
    if (off_rptr) off_rptr[b] = rp;
    if (off_x) off_x[b] = xo;
    if (off_y) off_y[b] = yo;
    if (b == p->nmat) break;
    const gbs_batch_item& it = p->items[b];
    r += it.m;
    z += it.nnz;
    rp += (long long)it.m + 1;
    xo += (long long)it.n * p->k;
    yo += (long long)it.m * p->k;
  }
  return GBS_OK;
}

int spmv_csr_batched_destroy(gbs_batch_plan* p) {
  if (p) batch_free(p);
  return GBS_OK;
}

}  // extern "C"
