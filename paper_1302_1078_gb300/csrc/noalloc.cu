// spmv_csr_noalloc: y <- A x without any device allocation by the library.
//
// The merge-path SpMV needs scratch memory beyond its inputs and outputs:
// the start coordinates of every CTA tile and one carry (row, partial sum)
// per tile.  spmv_csr takes that scratch from the stream-ordered allocator;
// this entry point takes it from the file-scope array below instead, so it
// calls no cudaMalloc, cudaFree, cudaMallocAsync or any other allocating
// routine.  It exists for callers that must not allocate device memory.
// Examples: a host application that owns and accounts for every device
// allocation (a memory-capped service or a plug-in host); a latency-critical
// loop where an allocation could block or fail under memory pressure.
//
// The array lives in this module's device memory from the moment the module
// is loaded until the process exits, on every GPU that loads the library:
// kNoAllocScratchBytes bytes per device.
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <string>

#include "gbspmv.h"
#include "launch.h"

namespace {

constexpr size_t kNoAllocScratchBytes = 4u << 20;  // 4 MiB
constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocItems = 15;  // merge items per thread: 3840 per CTA tile
constexpr int kMaxDevices = 64;

// Shared by every call on a device; keeps the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Bytes of scratch one call needs for `ctas` tiles of `elem`-byte values.
size_t scratch_bytes(long long ctas, size_t elem) {
  return align256(sizeof(int2) * (size_t)(ctas + 1)) + align256(sizeof(int) * (size_t)ctas) + elem * (size_t)ctas;
}

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once per
// device, with that device current, and cached.
int scratch_on_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    gbs::set_last_error((std::string("cudaGetDevice: ") + cudaGetErrorString(e)).c_str());
    return GBS_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    gbs::set_last_error("spmv_csr_noalloc: device ordinal out of range");
    return GBS_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      gbs::set_last_error((std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
      return GBS_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return GBS_OK;
}

}  // namespace

extern "C" int spmv_csr_noalloc(int m, int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals,
                                int dtype, const void* x, void* y, void* stream) {
  using namespace gbs;
  if (dtype != GBS_F64 && dtype != GBS_F32) {
    set_last_error("spmv_csr_noalloc: dtype must be GBS_F64 or GBS_F32");
    return GBS_EDTYPE;
  }
  if (m < 0 || n < 0 || nnz < 0) {
    set_last_error("spmv_csr_noalloc: negative size");
    return GBS_EINVAL;
  }
  if ((m > 0 && (row_ptr == nullptr || y == nullptr)) || (nnz > 0 && (col_idx == nullptr || vals == nullptr || x == nullptr))) {
    set_last_error("spmv_csr_noalloc: NULL pointer");
    return GBS_EINVAL;
  }
  // the same alignment rule as spmv_csr: every array aligned to its element size, refused on
  // the host so that a misaligned pointer never reaches a kernel
  const uintptr_t es = dtype == GBS_F64 ? sizeof(double) : sizeof(float);
  if ((reinterpret_cast<uintptr_t>(vals) % es) || (reinterpret_cast<uintptr_t>(x) % es) ||
      (reinterpret_cast<uintptr_t>(y) % es) || (reinterpret_cast<uintptr_t>(col_idx) % 4) ||
      (reinterpret_cast<uintptr_t>(row_ptr) % 4)) {
    set_last_error("spmv_csr_noalloc: arrays must be aligned to their element size");
    return GBS_EALIGN;
  }
  const long long total = (long long)m + nnz;
  const long long ipc = (long long)kNoAllocThreads * kNoAllocItems;
  const long long ctas = std::max<long long>(1, (total + ipc - 1) / ipc);
  const size_t elem = dtype == GBS_F64 ? sizeof(double) : sizeof(float);
  const size_t need = scratch_bytes(ctas, elem);
  if (need > kNoAllocScratchBytes) {
    // checked before any CUDA call: nothing is launched
    std::string msg = "spmv_csr_noalloc: m + nnz = " + std::to_string(total) + " needs " + std::to_string(need) +
                      " bytes of scratch, more than the " + std::to_string(kNoAllocScratchBytes) +
                      "-byte static scratch array holds; use spmv_csr";
    set_last_error(msg.c_str());
    return GBS_EUNSUPPORTED;
  }
  if (m == 0) return GBS_OK;
  void* base = nullptr;
  int rc = scratch_on_current_device(&base);
  if (rc != GBS_OK) return rc;
  // carve the array; every element read later is written earlier in the same call
  // (coordinates by the partition kernel, carries by the tile that owns them), so
  // nothing has to be cleared between calls
  char* p = static_cast<char*>(base);
  MergeScratch S;
  S.ctas = (int)ctas;
  S.coords = reinterpret_cast<int2*>(p);
  p += align256(sizeof(int2) * (size_t)(ctas + 1));
  S.carry_row = reinterpret_cast<int*>(p);
  p += align256(sizeof(int) * (size_t)ctas);
  S.carry_val = p;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CsrView A{m, n, nnz, row_ptr, col_idx, vals};
  DenseView D{1, x, 1, y, 1};
  cudaError_t e = launch_merge_partition(A, ipc, S, s);
  if (e == cudaSuccess)
    e = dtype == GBS_F64 ? launch_merge_f64(A, D, 1, false, false, kNoAllocThreads, kNoAllocItems, S, s)
                         : launch_merge_f32(A, D, 1, false, false, kNoAllocThreads, kNoAllocItems, S, s);
  if (e != cudaSuccess) {
    set_last_error((std::string("spmv_csr_noalloc launch: ") + cudaGetErrorString(e)).c_str());
    return GBS_ECUDA;
  }
  return GBS_OK;
}
