/*
 * gbspmv — CSR sparse-matrix products on NVIDIA GB300 (sm_103a), C ABI.
 *
 * Operations (Saule, Kaya, Catalyurek, "Performance Evaluation of Sparse
 * Matrix Multiplication Kernels on Intel Xeon Phi", arXiv:1302.1078):
 *
 *   SpMV  y <- A x       (Sec. 1, Sec. 3): A is m x n, x has n entries,
 *                        y has m entries; y_i is the dot product of row i of
 *                        A with x (2 * nnz flops).
 *   SpMM  Y <- A X       (Sec. 3, Sec. 5): X is n x k and Y is m x k, both
 *                        row major, so that each nonzero (i, j) reads the
 *                        contiguous row X[j, :] (2 * nnz * k flops).
 *
 * A is given in the compressed-row storage of Sec. 3: row_ptr[m+1] with
 * row_ptr[0] = 0 and row_ptr[m] = nnz; the nonzeros of row i are stored at
 * positions row_ptr[i] .. row_ptr[i+1]-1 of col_idx[nnz] (column ids) and
 * vals[nnz] (values).  Indices are 32-bit (Sec. 4).  Values are double
 * (the paper's precision, Sec. 4) or float.  Columns inside a row may be
 * unsorted or repeated; repeated entries add up.
 *
 * Beyond the paper: the backward pass of Y = A X (dX = A^T dY and dvals, the
 * gradient of a loss with respect to the stored values), a deterministic CSR
 * transpose, and a batched mode that multiplies many matrices in one
 * persistent launch replayed from a CUDA graph.
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers owned by the caller, unless the
 *     argument says "host".  The library never frees them and keeps no
 *     reference to them after the call returns, except where a plan says so.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream unless stated.
 *   - y / Y / dX / dvals are overwritten, never read (no alpha/beta).  An
 *     empty row yields 0.
 *   - Results are bitwise reproducible from run to run: no floating-point
 *     atomics are used and every summation order is fixed.
 *   - Return value: GBS_OK (0) or a negative status below.  A status other
 *     than GBS_OK means nothing was launched, except GBS_ECUDA, which may
 *     follow a failed launch.  gbs_last_error() gives a message for the
 *     calling thread.
 *   - The library does not check the values of row_ptr or col_idx on the
 *     device unless asked (gbs_validate_csr, or a plan built with
 *     GBS_PLAN_CHECK): malformed indices read out of bounds.
 *   - Sizes: m + nnz <= 2^31 - 4097 for every entry point that takes a CSR
 *     matrix (32-bit positions, with headroom for the kernels' rounding of
 *     nonzero ranges); larger returns GBS_EUNSUPPORTED before any launch.
 *     Dense operands are addressed with 64-bit offsets (column j of X at
 *     j * ldx), so n * ldx may exceed 2^31.
 */
#ifndef GBSPMV_H
#define GBSPMV_H

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- status */
#define GBS_OK 0
#define GBS_EINVAL (-1)       /* a size is negative, a required pointer is NULL, ld < k, ... */
#define GBS_EALIGN (-2)       /* a pointer or leading dimension breaks a stated alignment rule */
#define GBS_EDTYPE (-3)       /* unknown gbs_dtype */
#define GBS_ECUDA (-4)        /* a CUDA runtime call or launch failed */
#define GBS_EINDEX (-5)       /* CSR structure invalid (validation only) */
#define GBS_ETIMEOUT (-6)     /* a bounded device-side wait gave up */
#define GBS_ENOMEM (-7)       /* device or host allocation failed */
#define GBS_EUNSUPPORTED (-8) /* valid request this build does not support */

/* ------------------------------------------------------------------ types */
typedef enum { GBS_F64 = 0, GBS_F32 = 1 } gbs_dtype;

/* Kernel variants. */
typedef enum {
  GBS_VARIANT_AUTO = 0,   /* let the library choose from the row-length statistics */
  GBS_VARIANT_ROWS = 1,   /* sub-warp per row: `lanes` lanes share one row */
  GBS_VARIANT_MERGE = 2,  /* merge-path: equal shares of (rows + nonzeros) per thread */
  GBS_VARIANT_ROWS_TMA = 3, /* ROWS with persistent CTAs and a double-buffered bulk-copy (TMA)
                              pipeline; plans only (the plan sizes the tile to the largest
                              row block); needs 16-byte aligned vals and col_idx, else runs as ROWS */
  GBS_VARIANT_MERGE_DIRECT = 4, /* merge-path whose threads load their own nonzeros from global
                                  memory in 128-bit groups (no shared-memory staging of vals /
                                  col_idx), so more items per thread fit */
  GBS_VARIANT_ROWS_DIRECT = 5 /* ROWS without shared memory or barriers: every lane reads its
                                 row's values and column ids itself through L1 and walks the
                                 whole row; k > 1: `lanes` lanes split the columns, as in ROWS;
                                 k == 1: one lane per row (lanes ignored).  Same results, bit
                                 for bit, as ROWS with lanes that split the columns (k > 1) or
                                 with one lane per row (k == 1); for short rows.  Not a
                                 batched item form, and values are not read through a
                                 permutation (not for the backward pass's A^T) */
} gbs_variant;

/*
 * Launch configuration of one product.  Zero fields mean "library default".
 *   variant      gbs_variant.
 *   lanes        ROWS: lanes per row, one of 1, 2, 4, 8, 16, 32.  For SpMV
 *                the lanes split the row's nonzeros (then add their partial
 *                sums); for SpMM (k > 1) they split the k columns.
 *   threads      threads per CTA (multiple of 32, <= 1024).
 *   tile_nnz     ROWS: nonzeros staged in shared memory per pass.
 *   items        MERGE: merge-path items (rows + nonzeros) per thread.
 *   emul         ROWS_TMA with double values: in every group of 4 nonzeros
 *                a lane handles, the first `emul` (0..3) products run on the
 *                FP32 pipe as float-float arithmetic (double operands split
 *                into two floats by integer operations, TwoSum accumulation),
 *                the others on the FP64 pipe, so both pipes work at once.
 *                Each such product is accurate to about 2^-44 of |a x| and the
 *                sums stay within 3e-13 of sum |a x| per entry; operands
 *                outside [2^-38, 2^39) in magnitude use the FP64 pipe.
 *   relabel      plans only (0 elsewhere): the plan relabels the columns by
 *                their number of stored entries, most first (ties by column
 *                id), once, and every call first scatters x into that order
 *                (x'[newid[j]] = x[j], or the rows of X) and multiplies with
 *                the relabelled column ids.  The paper ties SpMV speed to the
 *                reuse of x's cache lines (Sec. 4.1, Sec. 4.3) and reorders
 *                matrices for it (Sec. 4.4); on a power-law matrix this packs
 *                the most gathered entries of x into the fewest lines.  Rows
 *                and the order of each row's terms are unchanged, so results
 *                are bitwise those of relabel = 0.  1: relabel; h >= 2:
 *                relabel, and the MERGE_DIRECT SpMV gathers columns at or
 *                above h * 1024 without allocating them in L1.  The plan then
 *                owns 4 * nnz + 4 * n bytes of relabelled indices and an
 *                n x k copy of x / X.
 */
typedef struct {
  int variant;
  int lanes;
  int threads;
  int tile_nnz;
  int items;
  int emul;
  int relabel;
} gbs_config;

/* Row-length statistics computed on the device (gbs_csr_stats). */
typedef struct {
  int m, n, nnz;
  int max_row;          /* longest row */
  int empty_rows;       /* rows with no nonzero */
  double mean_row;      /* nnz / m */
  double cv_row;        /* coefficient of variation of row lengths */
  long long rows_over_32, rows_over_256, rows_over_4096; /* counts of long rows */
} gbs_stats;

/* ------------------------------------------------------------- misc API */
int gbs_version(void);                       /* 10000 * major + 100 * minor + patch */
const char* gbs_status_string(int status);   /* static string */
const char* gbs_last_error(void);            /* message of the last failure on this thread */

/*
 * Check a CSR structure on the device: row_ptr[0] == 0, row_ptr
 * non-decreasing, row_ptr[m] == nnz, 0 <= col_idx[p] < n.  Synchronises
 * `stream`.  Returns GBS_OK or GBS_EINDEX.
 */
int gbs_validate_csr(int m, int n, int nnz, const int* row_ptr, const int* col_idx, void* stream);

/*
 * Row-length statistics of A (Sec. 4 Table "tab:matrices" lists the same
 * quantities: rows, nonzeros, nnz/row, max nnz/row).  Synchronises `stream`;
 * `out` is a host pointer.
 */
int gbs_csr_stats(int m, int n, int nnz, const int* row_ptr, gbs_stats* out, void* stream);

/* The configuration the library would pick for these statistics and k (host only). */
int gbs_default_config(const gbs_stats* stats, int dtype, int k, gbs_config* out);

/*
 * Diagnostic: FP64 fused-multiply-add throughput.  Launches `blocks` x
 * `threads` threads that each run `iters` x 8 independent FMAs and write one
 * double to out[blocks * threads] (device).  The caller times it: flops =
 * 2 * 8 * iters * blocks * threads.  On GB300 the FP64 pipe is about 1/64
 * of the FP32 rate, which makes it a second roof of FP64 SpMV beside HBM
 * bandwidth (Sec. 4.1 notes that on the Xeon Phi the FP peak was not the
 * bottleneck; here it can be).  The paper has no counterpart.
 */
int gbs_fp64_probe(double* out, int blocks, int threads, int iters, void* stream);

/*
 * Diagnostic for the failure path of the bounded device waits.  ROWS_TMA's
 * CTAs wait on mbarriers for their bulk copies; every such wait gives up
 * after 1 s of GPU global time (or 2^22 polls should the timer not advance),
 * flags the plan's status word (gbs_plan_status then returns GBS_ETIMEOUT)
 * and returns, so the context stays usable.  This call runs one such wait on
 * a barrier that nothing completes (a 16-byte copy is announced and never
 * issued), bounded by limit_ns (1 .. 2e9), on `stream`, and synchronises it.
 * Returns GBS_ETIMEOUT when the wait gave up, which is the expected result;
 * GBS_EINVAL for a limit out of range.  The paper has no counterpart.
 */
int gbs_wait_probe(long long limit_ns, void* stream);

/*
 * Diagnostic: useful cacheline density (UCLD, Sec. 4.1, the figure that ties
 * the gain of vectorised SpMV to it).  x is cut into aligned lines of
 * `line_elems` elements (line j = x[j*line_elems .. (j+1)*line_elems - 1]); a
 * non-empty row i with nnz_i nonzeros whose columns touch lines_i distinct
 * lines has density nnz_i / (line_elems * lines_i).  Writes to host pointers
 * (each may be NULL): *ucld = the mean density over non-empty rows (0 if
 * none; computed in 2^-31 fixed point, so within 5e-10 of the exact mean),
 * *lines = sum of lines_i over the rows (the line fetches of x if no line were
 * reused between rows), *nonempty_rows.  The paper's example: columns 0, 19,
 * 20 with 8-element lines give 3/16.  line_elems = 4 is GB300's 32-byte L2
 * sector of doubles.  Unsorted or repeated columns are counted correctly (an
 * unsorted row costs time quadratic in its length).  Synchronises `stream`.
 * Errors: GBS_EINVAL (line_elems < 1, bad sizes, NULL arrays).
 */
int gbs_ucld(int m, int n, int nnz, const int* row_ptr, const int* col_idx, int line_elems, double* ucld,
             long long* lines, long long* nonempty_rows, void* stream);

/* ------------------------------------------------------------ reordering */
/*
 * Reverse Cuthill-McKee ordering (Sec. 4.4 studies its effect on SpMV) of
 * the symmetric pattern of A + A^T of a square A (n x n), without self loops
 * or repeated edges.  Nodes are compared by (degree, index): nodes of degree
 * 0 come first in index order; then, while nodes remain, the smallest
 * remaining node s is moved to a pseudo-peripheral node r of its component
 * (George & Liu: from the BFS level structure of r, take the smallest node x
 * of the last level, and move r to x while x's structure has more levels),
 * and the component is numbered breadth first from r, each node appending
 * its unnumbered neighbours smallest first; the order is then reversed.
 * perm (device, n ints) receives the node placed at each position.
 * Runs on the device (level-synchronous, exactly the sequential order);
 * allocates scratch (about 9 ints per row and 7 per nonzero of A) with the
 * stream-ordered allocator and synchronises `stream`.
 * Errors: GBS_EINVAL, GBS_EUNSUPPORTED (nnz > 2^30), GBS_ECUDA.
 */
int gbs_rcm(int n, int nnz, const int* row_ptr, const int* col_idx, int* perm, void* stream);
/*
 * B = P A P^T for a permutation perm of 0..n-1 (perm[i] = the row / column of
 * A placed at i): row i of B is row perm[i] of A, every column j renumbered
 * to i' with perm[i'] = j, columns sorted within the row (stably, so repeated
 * columns keep their order), values (`dtype`) moving with their entries.
 * Caller buffers (device): b_row_ptr[n+1], b_col_idx[nnz], b_vals[nnz] (vals
 * and b_vals both NULL for the pattern only).  perm is not checked to be a
 * permutation.  Asynchronous on `stream` (scratch from the stream-ordered
 * allocator).
 */
int gbs_permute_csr(int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals, int dtype,
                    const int* perm, int* b_row_ptr, int* b_col_idx, void* b_vals, void* stream);

/* ------------------------------------------------- register blocking (BCSR) */
/*
 * Register-blocked CRS (Sec. 4.5): A (m x n) is cut into aligned a x b
 * regions (block row I = rows I*a .. I*a+a-1, block column J = columns
 * J*b .. J*b+b-1, a and b each 1, 2, 4 or 8); every region holding a stored
 * entry becomes a dense row-major block, zeros included, and the blocks of
 * a block row are listed by block column, ascending.  Repeated entries add
 * up in storage order.  The object owns device arrays bptr[ceil(m/a)+1],
 * bcol[nblocks], bval[nblocks*a*b] (dtype of vals); conversion runs on the
 * device and synchronises `stream`.  Each block costs a*b multiply-adds in
 * spmv_bcsr, zeros included, so register blocking pays only where blocks
 * are dense (the paper: where at least about 70 % of their values are
 * nonzeros).  x must be finite: a zero of a block times an infinite x is NaN.
 * Errors: GBS_EINVAL, GBS_EDTYPE, GBS_EUNSUPPORTED (other block sizes),
 * GBS_ECUDA (including out of memory for sparse blocks).
 */
typedef struct gbs_bcsr gbs_bcsr;

int gbs_bcsr_create(gbs_bcsr** plan, int m, int n, int nnz, const int* row_ptr, const int* col_idx,
                    const void* vals, int dtype, int a, int b, void* stream);
/* Host copies (any may be NULL): block rows, blocks, a, b. */
int gbs_bcsr_info(const gbs_bcsr* plan, int* block_rows, long long* nblocks, int* a, int* b);
/* Device pointers owned by the object (any output may be NULL). */
int gbs_bcsr_arrays(const gbs_bcsr* plan, const int** bptr, const int** bcol, const void** bval);
/* y <- A x from the blocks (y: m entries, x: n entries, device, the object's dtype). */
int spmv_bcsr(const gbs_bcsr* plan, const void* x, void* y, void* stream);
int gbs_bcsr_destroy(gbs_bcsr* plan);

/* ------------------------------------------------------------------ SpMV */
/*
 * y <- A x  (Sec. 3).  vals, x and y have type `dtype`; x has n entries and
 * y has m entries.  The variant is chosen without looking at row_ptr
 * (merge-path, which balances any row-length distribution: MERGE_DIRECT with
 * 128 threads and 9 items per thread); its scratch
 * (one carry per CTA) comes from the stream-ordered allocator of the
 * current device (cudaMallocAsync / cudaFreeAsync on `stream`).  This
 * one-shot call never reads the row-length statistics, because reading them
 * back would synchronise `stream` on every call.  A plan (gbs_plan_create)
 * is the path that picks the kernel and the lanes per row from the row
 * lengths, once: row-wise with lanes from the mean row length for regular
 * matrices, merge-path for skewed ones, or the autotuner's choice.
 * m, n >= 0, nnz >= 0; nnz == 0 or m == 0 writes zeros / nothing.
 */
int spmv_csr(int m, int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals,
             int dtype, const void* x, void* y, void* stream);

/* As spmv_csr, with an explicit configuration (NULL = spmv_csr's choice). */
int spmv_csr_cfg(int m, int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals,
                 int dtype, const void* x, void* y, const gbs_config* cfg, void* stream);

/*
 * y <- A x, as spmv_csr, for callers that must not allocate device memory:
 * for example a host application that owns and accounts for every device
 * allocation (a memory-capped service, a plug-in host), or a latency-critical
 * loop where an allocation could block or fail under memory pressure.  The
 * paper has no counterpart.
 *
 * The merge-path scratch (tile coordinates and per-tile carries) comes from a
 * 4 MiB static array in the library's device memory, which every GPU that
 * loads the library holds until the process exits; no cudaMalloc, cudaFree
 * or other allocating routine is called.  Limit: the scratch of one call is
 * about 20 bytes (FP64; 16 for FP32) per 3840 rows + nonzeros, so m + nnz up
 * to about 8.05e8 (FP64) or 1.0e9 (FP32) fits; larger sizes return
 * GBS_EUNSUPPORTED with a message (gbs_last_error) before anything is
 * launched.  Same dtypes, arguments and determinism as spmv_csr; the
 * product is the staged merge-path one (MERGE, 256 threads, 15 items per
 * thread): bit for bit spmv_csr_cfg's result with that configuration, and
 * within rounding of spmv_csr's own choice.  GBSPMV_CHECKED validation is
 * not run.
 *
 * The first call on each device looks up the array's device address (with
 * that device current) and caches it: make that first call before any
 * stream capture.  The cached address belongs to the device's current
 * context: after cudaDeviceReset (or any teardown of the primary context)
 * the module may be loaded at another address, so do not call this entry
 * point again in that process.  Misaligned arrays return GBS_EALIGN, as in
 * spmv_csr, before anything is launched.  Every call shares the one array, whose contents persist
 * from the previous call; each call writes every scratch element before
 * reading it, so nothing needs clearing.  Calls that overlap on the GPU (on
 * different streams, or from different threads without ordering) race on
 * the array and may produce wrong results: order them on one stream.
 */
int spmv_csr_noalloc(int m, int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals,
                     int dtype, const void* x, void* y, void* stream);

/* ------------------------------------------------------------------ SpMM */
/*
 * Y <- A X  (Sec. 5): X is n x k with leading dimension ldx >= k, Y is m x k
 * with leading dimension ldy >= k, both row major, elements of `dtype`.
 * k >= 1.  When X, Y and their leading dimensions are 16-byte aligned the
 * gathers of X rows use 128-bit loads; otherwise narrower loads are used.
 * Y is written with streaming (evict-first) stores.
 */
int spmm_csr(int m, int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals,
             int dtype, int k, const void* X, int ldx, void* Y, int ldy, void* stream);

int spmm_csr_cfg(int m, int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals,
                 int dtype, int k, const void* X, int ldx, void* Y, int ldy, const gbs_config* cfg,
                 void* stream);

/* ------------------------------------------------------------------ plans */
/*
 * A plan fixes the structure (m, n, nnz, row_ptr, col_idx), the dtype and k,
 * computes the row-length statistics, picks a configuration and owns any
 * scratch it needs.  With GBS_PLAN_TUNE it times candidate configurations
 * on the device (on scratch values it allocates itself, each run after a
 * write of twice the L2's size so that it starts cold) and keeps the
 * fastest (with GBS_PLAN_EMULATE also candidates that run part of the FP64
 * products on the FP32 pipe).  With GBS_PLAN_CHECK it validates the structure first.  The plan
 * keeps row_ptr and col_idx as given: they must stay valid and unchanged
 * while the plan is used.  gbs_plan_create synchronises `stream`.
 * Executing a plan allocates nothing and can be captured in a CUDA graph.
 */
#define GBS_PLAN_TUNE 1
#define GBS_PLAN_CHECK 2
#define GBS_PLAN_EMULATE 4 /* let the tuner try FP32-pipe emulation (gbs_config.emul) for double values */

typedef struct gbs_plan gbs_plan;

int gbs_plan_create(gbs_plan** plan, int m, int n, int nnz, const int* row_ptr, const int* col_idx,
                    int dtype, int k, int flags, void* stream);
int gbs_plan_destroy(gbs_plan* plan);
int gbs_plan_get_config(const gbs_plan* plan, gbs_config* cfg);
int gbs_plan_set_config(gbs_plan* plan, const gbs_config* cfg);
int gbs_plan_get_stats(const gbs_plan* plan, gbs_stats* out);
/*
 * The column relabelling of a plan whose configuration has relabel != 0:
 * newid[j] for the n columns (int32, device or host pointer), the rank of
 * column j when the columns are ordered by stored entries, most first, ties
 * by column id.  GBS_EINVAL if the plan does not relabel.  Synchronises
 * `stream`.
 */
int gbs_plan_relabel_ids(const gbs_plan* plan, int* newid, void* stream);
/* y <- A x (plan k must be 1) or Y <- A X (ldx, ldy >= plan k). */
int spmv_csr_plan(const gbs_plan* plan, const void* vals, const void* x, void* y, void* stream);
/*
 * Device status of the plan's bounded waits (host `*status`; bit 0: a pipeline
 * wait of GBS_VARIANT_ROWS_TMA timed out and its CTA returned early, so the
 * result of that call is incomplete).  Reads and clears it; synchronises `stream`.
 */
int gbs_plan_status(gbs_plan* plan, int* status, void* stream);
int spmm_csr_plan(const gbs_plan* plan, const void* vals, const void* X, int ldx, void* Y, int ldy,
                  void* stream);

/* ---------------------------------------------------- transpose + backward */
/*
 * CSR of A^T (n x m), i.e. the CCS of A (Sec. 3: the two formats are dual),
 * built on the device by a stable sort of the nonzeros by column: inside a
 * row of A^T the entries keep their order of storage in A, so the result is
 * unique and bit-exact (no atomics decide any position).  The plan owns
 *   rowptrT[n+1], colT[nnz] (row of A of each entry), perm[nnz] (position in
 *   A of each entry of A^T) and the row of every nonzero of A (the dvals
 *   pass); plus, only if a configuration that permutes the values first is
 *   chosen, nnz doubles of scratch.
 * It does not keep row_ptr / col_idx.  It also creates a non-blocking
 * stream and two events on the current device (spmv_csr_backward).
 * Synchronises `stream`.  The transpose is the one-time set-up of the
 * backward pass.
 */
typedef struct gbs_tplan gbs_tplan;

int gbs_transpose_plan(gbs_tplan** plan, int m, int n, int nnz, const int* row_ptr, const int* col_idx,
                       void* stream);
/* Device pointers owned by the plan (any output may be NULL). */
int gbs_tplan_arrays(const gbs_tplan* plan, const int** rowptrT, const int** colT, const int** perm);
/* Copy the plan's arrays into caller buffers (device or host, cudaMemcpyDefault), async on `stream`. */
int gbs_tplan_export(const gbs_tplan* plan, int* rowptrT, int* colT, int* perm, void* stream);
int gbs_tplan_destroy(gbs_tplan* plan);
/*
 * Make (and keep) a plan of A^T for `dtype` and k, with gbs_plan_create's
 * flags (GBS_PLAN_TUNE to autotune it); spmv_csr_backward then computes dX with
 * that plan's configuration instead of the one picked from A^T's row
 * statistics.  dX reads A's values in place through perm (ROWS, MERGE or
 * MERGE_DIRECT); with GBS_PLAN_TUNE the tuner also times permuting the
 * values into scratch first (one extra pass) followed by the best of all
 * variants, and keeps that route if it is faster.  Synchronises `stream`.
 * Idempotent per (dtype, k).
 */
int gbs_tplan_prepare(gbs_tplan* plan, int dtype, int k, int flags, void* stream);
/*
 * Set the configuration of dX for (dtype, k), replacing a prepared one.
 * GBS_VARIANT_ROWS, GBS_VARIANT_MERGE and GBS_VARIANT_MERGE_DIRECT read A's
 * values in place through perm; GBS_VARIANT_ROWS_TMA permutes them into
 * plan-owned scratch first (allocated here, nnz doubles); GBS_VARIANT_AUTO
 * takes the configuration from A^T's row statistics.  Errors as
 * gbs_plan_set_config.  Synchronises `stream`.
 */
int gbs_tplan_set_config(gbs_tplan* plan, int dtype, int k, const gbs_config* cfg, void* stream);
/* The configuration dX uses for (dtype, k): the prepared one, else the one from A^T's row statistics. */
int gbs_tplan_get_config(const gbs_tplan* plan, int dtype, int k, gbs_config* cfg);

/*
 * Backward of Y = A X (k >= 1 columns; k == 1 is SpMV) for a loss L with
 * upstream gradient dY = dL/dY (m x k, ld lddy):
 *   dX[j, c] = sum_{p : col_idx[p] = j} vals[p] * dY[row(p), c]   i.e. dX = A^T dY
 *   dvals[p] = sum_c dY[row(p), c] * X[col_idx[p], c]             (sampled dense-dense product)
 * dX (n x k, ld lddx) and dvals (nnz) may each be NULL to skip that output.
 * dX runs the forward kernels on A^T, reading A's values through perm (or,
 * for a configuration that permutes them first, through the plan's scratch:
 * calls that share such a plan must be ordered on one stream); dvals sums
 * each nonzero's k products in column order.  `plan` must come from
 * gbs_transpose_plan on the same (row_ptr, col_idx); row_ptr is unused.
 * When both dX and dvals are asked for, the dvals pass runs on a stream the
 * plan owns, concurrently with dX: it waits for the work enqueued on
 * `stream` before the call, and `stream` waits for it before anything
 * enqueued after the call (an event each way, which stream capture
 * follows), so the call is ordered on `stream` like any other.  The plan's
 * events are reused by every call: calls that share a plan must be issued
 * from one host thread at a time.
 */
int spmv_csr_backward(gbs_tplan* plan, const int* row_ptr, const int* col_idx, const void* vals, int dtype,
                      int k, const void* X, int ldx, const void* dY, int lddy, void* dX, int lddx, void* dvals,
                      void* stream);

/* ---------------------------------------------------------------- batched */
/*
 * Many independent products Y_b <- A_b X_b (b < nmat; k columns for all, k
 * == 1 is SpMV), each the product of Sec. 3 / Sec. 5, run by one persistent
 * kernel replayed from a CUDA graph.  The plan
 *   - picks each matrix's configuration (ROWS lanes / tile or MERGE items;
 *     256 threads) from its row statistics, or with GBS_PLAN_TUNE by timing
 *     candidates with standalone launches on the given operands (this
 *     writes Y_b), and then by timing whole-batch policies on the batched
 *     kernel itself (the statistics' variant with a given ROWS tile, MERGE
 *     for matrices of short rows, a given merge tile), keeping the fastest;
 *   - builds the work list: matrix b owns the contiguous items
 *     [item_begin[b], item_begin[b+1]) (row blocks or merge tiles); the
 *     grid is every resident CTA slot (`grid`), and each CTA claims the next
 *     unclaimed item from a device counter that the graph zeroes before the
 *     kernel, so launches of one plan must be ordered on one stream;
 *   - owns a device descriptor table, the merge scratch and the graph.
 * The arrays of every item must stay valid and unchanged while the plan is
 * used (only X and Y may be replaced, below).  Results equal
 * spmv_csr_batched_looped (one standalone launch per matrix with the same
 * configuration) bitwise, whichever CTA runs an item.  Plan creation
 * synchronises `stream`.
 * k must fit one column panel (k <= 64 for FP64 / 128 for FP32 with 16-byte
 * aligned X/Y rows, else k <= 32).
 */
typedef struct {
  int m, n, nnz;
  const int* row_ptr;
  const int* col_idx;
  const void* vals;
  const void* X; /* n x k, row major, leading dimension ldx (ignored for k == 1) */
  int ldx;
  void* Y;       /* m x k, row major, leading dimension ldy (ignored for k == 1) */
  int ldy;
} gbs_batch_item;

typedef struct gbs_batch_plan gbs_batch_plan;

int spmv_csr_batched_plan(gbs_batch_plan** plan, int nmat, const gbs_batch_item* items /* host */, int dtype,
                          int k, int flags, void* stream);
/*
 * The same plan with the caller's per-matrix configurations: cfgs (host,
 * nmat entries) gives each matrix GBS_VARIANT_ROWS or GBS_VARIANT_MERGE with
 * its lanes (k == 1; k > 1 uses the batch's column lanes), tile_nnz or items,
 * or GBS_VARIANT_AUTO for the heuristic / tuner choice of
 * spmv_csr_batched_plan.  threads is always 256; merge items are capped to the
 * batch kernel's shared-memory budget (spmv_csr_batched_info reports the values
 * used).  Errors: GBS_EUNSUPPORTED (another variant), GBS_EINVAL (as
 * gbs_plan_set_config).  cfgs == NULL is spmv_csr_batched_plan.
 */
int spmv_csr_batched_plan_cfg(gbs_batch_plan** plan, int nmat, const gbs_batch_item* items /* host */,
                              int dtype, int k, int flags, const gbs_config* cfgs /* host, may be NULL */,
                              void* stream);
/*
 * Launch the captured graph on `stream`.  X and Y (host arrays of nmat device
 * pointers, or NULL to keep the current ones) replace the dense operands
 * first; they must keep the shapes and the 16-byte alignment class of plan
 * time.  Replacing them synchronises `stream`.
 */
int spmv_csr_batched(gbs_batch_plan* plan, const void* const* X, void* const* Y, void* stream);
/* The same products as a host loop of per-matrix launches (no graph): the baseline. */
int spmv_csr_batched_looped(gbs_batch_plan* plan, void* stream);
/* Host copies: cfgs[nmat], item_begin[nmat+1], grid, total work items (any may be NULL). */
int spmv_csr_batched_info(const gbs_batch_plan* plan, gbs_config* cfgs, int* item_begin, int* grid,
                          int* total_items);
/*
 * Offsets of each matrix in concatenated batch buffers (host arrays of nmat+1,
 * exclusive prefix sums in input order): rows, nonzeros, row_ptr entries (m+1
 * each), X entries (n*k) and Y entries (m*k).  Any may be NULL.
 */
int spmv_csr_batched_offsets(const gbs_batch_plan* plan, long long* off_rows, long long* off_nnz,
                             long long* off_rptr, long long* off_x, long long* off_y);
int spmv_csr_batched_destroy(gbs_batch_plan* plan);

#ifdef __cplusplus
}
#endif
#endif /* GBSPMV_H */
