// Useful cacheline density (UCLD) of Sec. 4.1: how many of the x elements in
// the lines a row's gathers touch are used.  x is cut into aligned lines of
// `line` elements; a non-empty row i with nnz_i nonzeros touching lines_i
// distinct lines has density nnz_i / (line * lines_i), and UCLD is the mean
// over the non-empty rows.  On GB300 the natural line sizes are 4 doubles (a
// 32-byte L2 sector, the unit of an x gather) and 16 (a 128-byte line); the
// paper's Xeon Phi used 8 (64-byte lines).
//
// One warp per row.  For a row whose columns are sorted, an entry starts a new
// line when its line differs from the previous entry's, so lines_i is a
// ballot count; a row found unsorted is recounted by comparing every entry
// with all earlier entries of the row (quadratic in the row length, fine for
// a diagnostic).  Sums are integers (the ratio in 2^-31 fixed point), so the
// result does not depend on the order of the atomics.
#include <cstdint>

#include "launch.h"

namespace gbs {

__global__ void __launch_bounds__(256) ucld_kernel(const int* __restrict__ rp, const int* __restrict__ ci, int m,
                                                   int line, unsigned long long* __restrict__ acc) {
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long fsum = 0, lsum = 0, rows = 0;
  for (long long i = warp; i < m; i += nwarps) {
    const int rs = __ldg(rp + i), re = __ldg(rp + i + 1);
    if (re <= rs) continue;  // empty row: no density (warp-uniform)
    int lines = 0;
    bool unsorted = false;
    for (int b = rs; b < re; b += 32) {
      const int p = b + lane;
      bool first = false;
      if (p < re) {
        const int c = __ldg(ci + p);
        if (p == rs) {
          first = true;
        } else {
          const int cp = __ldg(ci + p - 1);
          first = cp / line != c / line;
          unsorted |= cp > c;
        }
      }
      lines += __popc(__ballot_sync(kFull, first));
    }
    if (__any_sync(kFull, unsorted)) {
      lines = 0;
      for (int b = rs; b < re; b += 32) {
        const int p = b + lane;
        bool first = false;
        if (p < re) {
          const int ln = __ldg(ci + p) / line;
          first = true;
          for (int q = rs; q < p && first; ++q) first = __ldg(ci + q) / line != ln;
        }
        lines += __popc(__ballot_sync(kFull, first));
      }
    }
    if (lane == 0) {
      const double r = (double)(re - rs) / ((double)line * (double)lines);
      fsum += __double2ull_rn(r * 2147483648.0);
      lsum += (unsigned long long)lines;
      rows += 1;
    }
  }
  if (lane == 0 && rows) {
    atomicAdd(acc + 0, fsum);
    atomicAdd(acc + 1, lsum);
    atomicAdd(acc + 2, rows);
  }
}

cudaError_t launch_ucld(const int* row_ptr, const int* col_idx, int m, int line, unsigned long long* acc,
                        cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const long long warps = (long long)m;
  const int grid = (int)((warps * 32 + 255) / 256 < 152 * 16 ? (warps * 32 + 255) / 256 : 152 * 16);
  ucld_kernel<<<grid, 256, 0, s>>>(row_ptr, col_idx, m, line, acc);
  return cudaGetLastError();
}

}  // namespace gbs
