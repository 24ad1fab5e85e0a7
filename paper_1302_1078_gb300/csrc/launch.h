// Internal launcher interface between the C-ABI layer (api.cu) and the
// per-dtype kernel translation units.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

namespace gbs {

struct CsrView {
  int m, n, nnz;
  const int* row_ptr;
  const int* col_idx;
  const void* vals;
  const int* perm = nullptr;  // if set, the value of entry p is vals[perm[p]] (ROWS, MERGE, MERGE_DIRECT)
  int hot_cols = 0;           // > 0: columns relabelled hottest first; MERGE_DIRECT SpMV gathers
                              // columns >= hot_cols without L1 allocation
};

struct DenseView {
  int k;
  const void* X;
  long long ldx;
  void* Y;
  long long ldy;
};

struct MergeScratch {
  int ctas;
  int2* coords;     // [ctas + 1]
  int* carry_row;   // [ctas]
  void* carry_val;  // [ctas * k] elements of the dtype
};

// ROWS variant.  lanes: 1..32 (power of two); k == 1 -> lanes split nonzeros,
// k > 1 -> lanes split columns (k <= lanes * VEC is required per launch;
// wider k is done in column panels by the caller).  vec16: use 128-bit
// gathers/stores of X/Y (caller checked the alignment).
cudaError_t launch_rows_f64(const CsrView& A, const DenseView& D, int lanes, bool vec16, int threads, int tile,
                            int row_base, int rows, cudaStream_t s);
cudaError_t launch_rows_f32(const CsrView& A, const DenseView& D, int lanes, bool vec16, int threads, int tile,
                            int row_base, int rows, cudaStream_t s);

// ROWS_DIRECT variant (no shared memory, no barriers): lanes split the columns (k > 1; same
// rules as ROWS), one lane per row for k == 1; values are not read through a permutation.
cudaError_t launch_rows_direct_f64(const CsrView& A, const DenseView& D, int lanes, bool vec16, int threads,
                                   cudaStream_t s);
cudaError_t launch_rows_direct_f32(const CsrView& A, const DenseView& D, int lanes, bool vec16, int threads,
                                   cudaStream_t s);

// ROWS_TMA variant (persistent, bulk-copy pipeline).  tile must hold the largest block's
// nonzeros + 8; vals and col_idx 16-byte aligned; status: device int (bit 0 = wait timeout).
// emul (FP64 only, 0..3): products per group of 4 nonzeros computed on the FP32 pipe (df64.cuh).
cudaError_t launch_rows_tma_f64(const CsrView& A, const DenseView& D, int lanes, bool vec16, int threads, int tile,
                                int emul, int* status, cudaStream_t s);
cudaError_t launch_rows_tma_f32(const CsrView& A, const DenseView& D, int lanes, bool vec16, int threads, int tile,
                                int emul, int* status, cudaStream_t s);
size_t rows_tma_smem(int dtype, int rows_per_cta, int tile);

// MERGE variant: partition (coords) must have been computed for (threads / g) * items
// items per CTA.  g lanes per merge thread (columns), g * VEC >= k.  direct: each merge
// thread loads its nonzeros from global memory (MERGE_DIRECT) instead of shared memory.
cudaError_t launch_merge_f64(const CsrView& A, const DenseView& D, int g, bool vec16, bool direct, int threads,
                             int items, const MergeScratch& S, cudaStream_t s);
cudaError_t launch_merge_f32(const CsrView& A, const DenseView& D, int g, bool vec16, bool direct, int threads,
                             int items, const MergeScratch& S, cudaStream_t s);
// The same launchers for a CsrView whose values are read through A.perm (the backward pass's
// A^T on A's values).
cudaError_t launch_rows_perm_f64(const CsrView& A, const DenseView& D, int lanes, bool vec16, int threads, int tile,
                                 int row_base, int rows, cudaStream_t s);
cudaError_t launch_rows_perm_f32(const CsrView& A, const DenseView& D, int lanes, bool vec16, int threads, int tile,
                                 int row_base, int rows, cudaStream_t s);
cudaError_t launch_merge_perm_f64(const CsrView& A, const DenseView& D, int g, bool vec16, bool direct, int threads,
                                  int items, const MergeScratch& S, cudaStream_t s);
cudaError_t launch_merge_perm_f32(const CsrView& A, const DenseView& D, int g, bool vec16, bool direct, int threads,
                                  int items, const MergeScratch& S, cudaStream_t s);
cudaError_t launch_merge_partition(const CsrView& A, long long items_per_cta, const MergeScratch& S, cudaStream_t s);

// Exclusive prefix sum of int32 (in == out allowed); ws holds scan_workspace_ints(count) ints.
cudaError_t exclusive_scan_i32(const int* in, int* out, long long count, int* ws, cudaStream_t s);
size_t scan_workspace_ints(long long count);

// Transpose (transpose.cu).  Buffer sizes: rptrT n+1, colT/perm/rows/keys_a/keys_b/vals_a/vals_b nnz,
// hist transpose_hist_ints(nnz), scan_ws transpose_scan_ws_ints(nnz).
cudaError_t transpose_run(int m, int n, int nnz, const int* row_ptr, const int* col_idx, int* rptrT, int* colT,
                          int* perm, int* rows, int* keys_a, int* keys_b, int* vals_a, int* vals_b, int* hist,
                          int* scan_ws, cudaStream_t s);
size_t transpose_hist_ints(int nnz);
size_t transpose_scan_ws_ints(int nnz);
// Stable LSD radix sort of n (key >= 0, value) pairs by the keys' low `bits` bits (transpose.cu);
// hist / scan_ws sized as for a transpose of n nonzeros.
cudaError_t radix_sort_pairs(int n, int bits, int* keys_a, int* keys_b, int* vals_a, int* vals_b, int* hist,
                             int* scan_ws, int** keys_out, int** vals_out, cudaStream_t s);

// Column relabelling by in-degree, hottest first (relabel.cu).  col_degree_stats: the largest
// column degree and the coefficient of variation of the degrees (synchronises s).  relabel_build:
// newid[n] (rank of each column) and col_rl[nnz] = newid[col_idx] (synchronises s).
// relabel_dense: X'[newid[j], :] = X[j, :] for the n rows of X (k columns; vec16: X, X' and both
// leading dimensions 16-byte aligned).
cudaError_t col_degree_stats(int n, int nnz, const int* col_idx, int* max_deg, double* cv_deg, cudaStream_t s);
cudaError_t relabel_build(int n, int nnz, const int* col_idx, int* newid, int* col_rl, cudaStream_t s);
cudaError_t relabel_dense(int dtype, int n, int k, const void* X, long long ldx, const int* newid, void* Xp,
                          long long ldxp, bool vec16, cudaStream_t s);

// out[q] = src[perm[q]] for values of `dtype`.
cudaError_t gather_values(int dtype, const void* src, const int* perm, int nnz, void* out, cudaStream_t s);

// dvals[p] = sum_c dY[rows[p], c] * X[col_idx[p], c]  (backward.cu)
cudaError_t launch_sddmm(int dtype, int nnz, int k, const int* rows, const int* col_idx, const void* X, long long ldx,
                         const void* dY, long long lddy, void* dvals, cudaStream_t s);

// Batched persistent kernel (batched.cu).  launch == false: set the shared-memory
// attribute and report the resident CTAs per SM in *blocks_per_sm; launch == true: launch
// `grid` CTAs of 256 threads over `descs` (device BatchDesc<T>[nmat]); CTAs claim items
// from the device counter *next_item, which must be 0 at launch.
cudaError_t batched_kernel_call(bool launch, int dtype, bool split, int G, bool vec16, const void* descs, int nmat,
                                int total_items, int* next_item, int grid, size_t smem, int* blocks_per_sm,
                                cudaStream_t s);

// UCLD sums (ucld.cu): acc[0] += sum of nnz_i / (line * lines_i) over non-empty rows in 2^-31
// fixed point, acc[1] += sum of lines_i, acc[2] += non-empty rows.
cudaError_t launch_ucld(const int* row_ptr, const int* col_idx, int m, int line, unsigned long long* acc,
                        cudaStream_t s);

// Reverse Cuthill-McKee permutation of the symmetric pattern of a square A (rcm.cu;
// allocates its scratch stream-ordered and synchronises s), and B = P A P^T (vals and
// bvals may be NULL for the pattern only).
cudaError_t rcm_run(int n, int nnz, const int* row_ptr, const int* col_idx, int* perm, cudaStream_t s);
cudaError_t permute_run(int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals, int dtype,
                        const int* perm, int* brp, int* bcol, void* bvals, cudaStream_t s);

// Register-blocked CRS (bcsr.cu).  bcsr_count fills bptr[mb+1] and *nblocks (synchronises s)
// and leaves the sorted block columns in *scratch (stream-ordered allocation) for bcsr_fill,
// which writes bcol / bval; the caller frees scratch with cudaFreeAsync.
cudaError_t bcsr_count(int m, int n, int nnz, const int* row_ptr, const int* col_idx, int a, int b, int* bptr,
                       int** bcol_sorted, int* nblocks, void** scratch, cudaStream_t s);
cudaError_t bcsr_fill(int m, int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals, int dtype,
                      int a, int b, const int* bptr, int* bcol, void* bval, long long nblocks, void* scratch,
                      cudaStream_t s);
cudaError_t bcsr_spmv(int dtype, int a, int b, int m, int n, const int* bptr, const int* bcol, const void* bval,
                      const void* x, void* y, cudaStream_t s);

// Message returned by gbs_last_error() on the calling thread (api.cu).
void set_last_error(const char* msg);

// Shared-memory bytes of one CTA (host helpers).
size_t rows_smem(int dtype, int rows_per_cta, int tile);
size_t merge_smem(int dtype, int g, bool vec16, int threads, int items);

}  // namespace gbs
