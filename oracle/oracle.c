/*
 * CPU oracle for CSR sparse-matrix products (TEST INFRASTRUCTURE).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  The GPU library never links, includes or calls it, and
 * this file includes nothing of the GPU library's: the two share no code.
 *
 * Everything here is the plain definition, written so that it can be checked
 * against the paper by eye:
 *
 *   Storage (Sec. 3, CRS): rptrs[m+1] with rptrs[0] = 0 and rptrs[m] = tau;
 *   the column ids of row i are cids[rptrs[i] .. rptrs[i+1]-1]; val[p] is
 *   the value of the nonzero stored at cids[p].  Indices are 32-bit, values
 *   are double precision (Sec. 4).
 *
 *   SpMV (Sec. 1 and Sec. 3): y <- A x with A m x n, x of n entries and y of
 *   m entries.  Each y_i is the dot product of row i with x: one multiply
 *   and one add per nonzero, 2*tau flops in total.
 *
 *   SpMM (Sec. 3 and Sec. 5): Y <- A X with X n x k and Y m x k, both row
 *   major.  For row i a temporary of k entries starts at zero; every nonzero
 *   (i, j) adds val * X[j, :] to it; the temporary is then written to Y[i, :].
 *
 * Arithmetic: sums run left to right in stored order, as plain s = s + a*b
 * in double precision (the file is compiled with -ffp-contract=off, so no
 * fused multiply-add is formed).  Single-precision inputs are widened to
 * double; their products are then exact and only the sum rounds.
 * Alongside each result the oracle returns the sum of absolute products,
 * sum |val * x|, which scales the accuracy bound of a parallel result.
 *
 * Readings where the paper is silent: an empty row yields 0; y (and Y) is
 * overwritten, never read; repeated or unsorted column ids inside a row are
 * allowed and simply add up.  Where the paper's X is called m x k (Sec. 5)
 * the oracle follows Sec. 3's n x k.
 *
 * Beyond the paper (it has no backward pass or transpose), the gradient of
 * L = <A X, W> and the CSR transpose are their plain definitions:
 *   dX[j, c]  = sum over nonzeros p with cids[p] = j of val[p] * dY[row(p), c]
 *               (computed by scattering over A, not through a transpose);
 *   dval[p]   = sum_c dY[row(p), c] * X[cids[p], c];
 *   transpose = stable counting sort of the nonzeros by column (Sec. 3 notes
 *               that CRS and CCS are dual): inside a row of A^T the entries
 *               keep their original order of storage.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ SpMV */

/*
 * y_i = sum_{p = rptrs[i]}^{rptrs[i+1]-1} val[p] * x[cids[p]]   (Sec. 3)
 * r_i = sum |val[p] * x[cids[p]]|                                (may be NULL)
 *
 * `threads` > 1 runs the rows in parallel exactly as the paper's Sec. 4.1
 * kernel does (OpenMP, dynamic schedule, chunks of 64 rows).  Each row is
 * still summed by one thread in stored order, so the result does not depend
 * on the thread count.
 */
void orc_spmv_f64(int m, const int* rptrs, const int* cids, const double* val, const double* x,
                  double* y, double* r, int threads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(threads > 0 ? threads : 1) if (threads > 1)
#endif
  for (int i = 0; i < m; ++i) {
    double s = 0.0, a = 0.0;
    for (int p = rptrs[i]; p < rptrs[i + 1]; ++p) {
      double t = val[p] * x[cids[p]];
      s = s + t;
      a = a + fabs(t);
    }
    y[i] = s;
    if (r) r[i] = a;
  }
}

/* Single-precision inputs, double accumulation, double outputs. */
void orc_spmv_f32(int m, const int* rptrs, const int* cids, const float* val, const float* x,
                  double* y, double* r, int threads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(threads > 0 ? threads : 1) if (threads > 1)
#endif
  for (int i = 0; i < m; ++i) {
    double s = 0.0, a = 0.0;
    for (int p = rptrs[i]; p < rptrs[i + 1]; ++p) {
      double t = (double)val[p] * (double)x[cids[p]];
      s = s + t;
      a = a + fabs(t);
    }
    y[i] = s;
    if (r) r[i] = a;
  }
}

/* ------------------------------------------------------------------ SpMM */

/*
 * Y[i, c] = sum_p val[p] * X[cids[p], c], c < k  (Sec. 5): per row, a
 * k-entry temporary starts at zero, each nonzero streams row X[cids[p], :]
 * into it, and the temporary is written to Y[i, :].  X has leading dimension
 * ldx >= k, Y (and R, if not NULL) leading dimension ldy >= k.
 */
void orc_spmm_f64(int m, int k, const int* rptrs, const int* cids, const double* val,
                  const double* X, long long ldx, double* Y, long long ldy, double* R, int threads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(threads > 0 ? threads : 1) if (threads > 1)
#endif
  for (int i = 0; i < m; ++i) {
    double* tmp = (double*)calloc((size_t)(k > 0 ? k : 1), sizeof(double));
    double* tab = (double*)calloc((size_t)(k > 0 ? k : 1), sizeof(double));
    for (int p = rptrs[i]; p < rptrs[i + 1]; ++p) {
      const double* xr = X + (long long)cids[p] * ldx;
      for (int c = 0; c < k; ++c) {
        double t = val[p] * xr[c];
        tmp[c] = tmp[c] + t;
        tab[c] = tab[c] + fabs(t);
      }
    }
    for (int c = 0; c < k; ++c) {
      Y[(long long)i * ldy + c] = tmp[c];
      if (R) R[(long long)i * ldy + c] = tab[c];
    }
    free(tmp);
    free(tab);
  }
}

void orc_spmm_f32(int m, int k, const int* rptrs, const int* cids, const float* val,
                  const float* X, long long ldx, double* Y, long long ldy, double* R, int threads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(threads > 0 ? threads : 1) if (threads > 1)
#endif
  for (int i = 0; i < m; ++i) {
    double* tmp = (double*)calloc((size_t)(k > 0 ? k : 1), sizeof(double));
    double* tab = (double*)calloc((size_t)(k > 0 ? k : 1), sizeof(double));
    for (int p = rptrs[i]; p < rptrs[i + 1]; ++p) {
      const float* xr = X + (long long)cids[p] * ldx;
      for (int c = 0; c < k; ++c) {
        double t = (double)val[p] * (double)xr[c];
        tmp[c] = tmp[c] + t;
        tab[c] = tab[c] + fabs(t);
      }
    }
    for (int c = 0; c < k; ++c) {
      Y[(long long)i * ldy + c] = tmp[c];
      if (R) R[(long long)i * ldy + c] = tab[c];
    }
    free(tmp);
    free(tab);
  }
}

/* ------------------------------------------------------------- transpose */

/*
 * CSR of A^T (n x m) by a stable counting sort over the column ids:
 *   rptrsT  = exclusive prefix sum of the column counts (n+1 entries);
 *   permT[q] = position in A of the q-th nonzero of A^T, where the nonzeros
 *              of one column keep their order of storage in A;
 *   cidsT[q] = row of A holding nonzero permT[q].
 * Returns 0, or -1 if a column id is outside [0, n).
 */
int orc_transpose(int m, int n, const int* rptrs, const int* cids, int* rptrsT, int* cidsT, int* permT) {
  int nnz = rptrs[m];
  for (int j = 0; j <= n; ++j) rptrsT[j] = 0;
  for (int p = 0; p < nnz; ++p) {
    if (cids[p] < 0 || cids[p] >= n) return -1;
    rptrsT[cids[p] + 1] += 1;
  }
  for (int j = 0; j < n; ++j) rptrsT[j + 1] += rptrsT[j];
  int* next = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  for (int j = 0; j < n; ++j) next[j] = rptrsT[j];
  for (int i = 0; i < m; ++i) {
    for (int p = rptrs[i]; p < rptrs[i + 1]; ++p) {
      int q = next[cids[p]]++;
      cidsT[q] = i;
      permT[q] = p;
    }
  }
  free(next);
  return 0;
}

/* -------------------------------------------------------------- backward */

/*
 * Gradients of L = <Y, W> for Y = A X, given dY = dL/dY (m x k, ld lddy):
 *   dX[j, c] = sum_{p : cids[p] = j} val[p] * dY[row(p), c]   (scatter over A)
 *   dval[p]  = sum_c dY[row(p), c] * X[cids[p], c]
 * dX is n x k with leading dimension lddx and is overwritten.  RdX and Rdval
 * (may be NULL) receive the matching sums of absolute products.
 */
void orc_backward_f64(int m, int n, int k, const int* rptrs, const int* cids, const double* val,
                      const double* X, long long ldx, const double* dY, long long lddy,
                      double* dX, long long lddx, double* dval, double* RdX, double* Rdval) {
  for (int j = 0; j < n; ++j)
    for (int c = 0; c < k; ++c) {
      dX[(long long)j * lddx + c] = 0.0;
      if (RdX) RdX[(long long)j * lddx + c] = 0.0;
    }
  for (int i = 0; i < m; ++i) {
    for (int p = rptrs[i]; p < rptrs[i + 1]; ++p) {
      int j = cids[p];
      double g = 0.0, ga = 0.0;
      for (int c = 0; c < k; ++c) {
        double d = dY[(long long)i * lddy + c];
        double t = val[p] * d;
        dX[(long long)j * lddx + c] = dX[(long long)j * lddx + c] + t;
        if (RdX) RdX[(long long)j * lddx + c] = RdX[(long long)j * lddx + c] + fabs(t);
        double u = d * X[(long long)j * ldx + c];
        g = g + u;
        ga = ga + fabs(u);
      }
      dval[p] = g;
      if (Rdval) Rdval[p] = ga;
    }
  }
}

void orc_backward_f32(int m, int n, int k, const int* rptrs, const int* cids, const float* val,
                      const float* X, long long ldx, const float* dY, long long lddy,
                      double* dX, long long lddx, double* dval, double* RdX, double* Rdval) {
  for (int j = 0; j < n; ++j)
    for (int c = 0; c < k; ++c) {
      dX[(long long)j * lddx + c] = 0.0;
      if (RdX) RdX[(long long)j * lddx + c] = 0.0;
    }
  for (int i = 0; i < m; ++i) {
    for (int p = rptrs[i]; p < rptrs[i + 1]; ++p) {
      int j = cids[p];
      double g = 0.0, ga = 0.0;
      for (int c = 0; c < k; ++c) {
        double d = (double)dY[(long long)i * lddy + c];
        double t = (double)val[p] * d;
        dX[(long long)j * lddx + c] = dX[(long long)j * lddx + c] + t;
        if (RdX) RdX[(long long)j * lddx + c] = RdX[(long long)j * lddx + c] + fabs(t);
        double u = d * (double)X[(long long)j * ldx + c];
        g = g + u;
        ga = ga + fabs(u);
      }
      dval[p] = g;
      if (Rdval) Rdval[p] = ga;
    }
  }
}

/* ------------------------------------------------------------- batching */

/*
 * Offsets of matrix b inside the concatenated batch buffers, exclusive prefix
 * sums in input order: rows (sum of m), nonzeros, row_ptr entries (sum of
 * m+1), X entries (sum of n*k) and Y entries (sum of m*k).
 */
void orc_batch_offsets(int nmat, const int* ms, const int* ns, const long long* nnzs, int k,
                       long long* off_rows, long long* off_nnz, long long* off_rptr,
                       long long* off_x, long long* off_y) {
  long long r = 0, z = 0, rp = 0, xo = 0, yo = 0;
  for (int b = 0; b < nmat; ++b) {
    off_rows[b] = r;
    off_nnz[b] = z;
    off_rptr[b] = rp;
    off_x[b] = xo;
    off_y[b] = yo;
    r += ms[b];
    z += nnzs[b];
    rp += (long long)ms[b] + 1;
    xo += (long long)ns[b] * k;
    yo += (long long)ms[b] * k;
  }
  off_rows[nmat] = r;
  off_nnz[nmat] = z;
  off_rptr[nmat] = rp;
  off_x[nmat] = xo;
  off_y[nmat] = yo;
}

/* ------------------------------------------------------------------ UCLD */

static int cmp_int(const void* a, const void* b) {
  const int x = *(const int*)a, y = *(const int*)b;
  return (x > y) - (x < y);
}

/*
 * Useful cacheline density (Sec. 4.1, the figure relating vectorised SpMV
 * speed to it): x is cut into aligned lines of `line` elements (line j holds
 * x[j*line .. j*line+line-1]).  For a non-empty row i with nnz_i nonzeros
 * whose columns touch lines_i distinct lines, the row's density is
 *     nnz_i / (line * lines_i),
 * and UCLD is the mean of that ratio over the non-empty rows (an empty row
 * has no ratio; the paper is silent on it).  The paper's example: columns 0,
 * 19 and 20 with 8-element lines touch lines 0 and 2, so the row's density
 * is 3 / 16.  Also returned: the sum of lines_i over all rows (the line
 * fetches of one pass over x if no line were reused between rows) and the
 * number of non-empty rows.  Distinct lines are counted by sorting a copy of
 * the row's line ids, so unsorted or repeated columns are handled.
 */
void orc_ucld(int m, const int* rptrs, const int* cids, int line, double* ucld, long long* lines_total,
              long long* nonempty) {
  long long maxlen = 0;
  for (int i = 0; i < m; ++i)
    if (rptrs[i + 1] - rptrs[i] > maxlen) maxlen = rptrs[i + 1] - rptrs[i];
  int* buf = (int*)malloc(sizeof(int) * (size_t)(maxlen > 0 ? maxlen : 1));
  double sum = 0.0;
  long long tot = 0, rows = 0;
  for (int i = 0; i < m; ++i) {
    const int len = rptrs[i + 1] - rptrs[i];
    if (len == 0) continue;
    for (int q = 0; q < len; ++q) buf[q] = cids[rptrs[i] + q] / line;
    qsort(buf, (size_t)len, sizeof(int), cmp_int);
    long long distinct = 1;
    for (int q = 1; q < len; ++q) distinct += buf[q] != buf[q - 1];
    sum += (double)len / ((double)line * (double)distinct);
    tot += distinct;
    rows += 1;
  }
  free(buf);
  *ucld = rows > 0 ? sum / (double)rows : 0.0;
  *lines_total = tot;
  *nonempty = rows;
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
