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

/* ------------------------------------------------------------------ RCM */

/*
 * Reverse Cuthill-McKee ordering (Sec. 4.4 applies it to study SpMV; the
 * paper used MATLAB's implementation, so the tie-breaking rules here are
 * this library's own, stated in full).  The graph is the symmetric pattern
 * of A + A^T of a square A, without self loops or repeated edges; deg(v) is
 * the number of distinct neighbours of v.  Nodes are compared by
 * (degree, index).
 *
 *   1. Nodes of degree 0 come first, in index order.
 *   2. Then, while nodes remain: s = the smallest remaining node.  A
 *      pseudo-peripheral node r is found from s (George & Liu): build the
 *      BFS level structure from r = s; repeatedly take x = the smallest
 *      node of its last level and build the structure from x; if x's has
 *      more levels, r = x and continue, otherwise stop.  Cuthill-McKee then
 *      numbers r's component breadth first from r: the nodes are taken in
 *      the order they were numbered, and each appends its not yet numbered
 *      neighbours, smallest first.
 *   3. The order is reversed: perm[i] is the node placed at position i.
 *
 * Returns 0, or -1 if a scratch allocation fails.
 */
static int cmp_deg_idx(const int* deg, int a, int b) {
  if (deg[a] != deg[b]) return deg[a] < deg[b] ? -1 : 1;
  return (a > b) - (a < b);
}

static const int* g_sort_deg; /* comparison context for qsort */
static int cmp_nodes(const void* a, const void* b) {
  return cmp_deg_idx(g_sort_deg, *(const int*)a, *(const int*)b);
}

/* Symmetric pattern of A + A^T (no self loops, no repeats): srp[n+1], scol (malloc'd). */
static int sym_pattern(int n, const int* rptrs, const int* cids, int** srp_out, int** scol_out) {
  long long nnz = rptrs[n];
  int* cnt = (int*)calloc((size_t)n + 1, sizeof(int));
  int* src = (int*)malloc(sizeof(int) * (size_t)(2 * nnz + 1));
  int* dst = (int*)malloc(sizeof(int) * (size_t)(2 * nnz + 1));
  if (!cnt || !src || !dst) { free(cnt); free(src); free(dst); return -1; }
  long long e = 0;
  for (int i = 0; i < n; ++i)
    for (int p = rptrs[i]; p < rptrs[i + 1]; ++p) {
      const int j = cids[p];
      if (j == i) continue;
      src[e] = i; dst[e] = j; ++e;
      src[e] = j; dst[e] = i; ++e;
    }
  /* bucket the directed edges by source, then sort each bucket and drop repeats */
  for (long long q = 0; q < e; ++q) cnt[src[q] + 1]++;
  for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  int* fill = (int*)malloc(sizeof(int) * (size_t)n);
  int* adj = (int*)malloc(sizeof(int) * (size_t)(e + 1));
  if (!fill || !adj) { free(cnt); free(src); free(dst); free(fill); free(adj); return -1; }
  memcpy(fill, cnt, sizeof(int) * (size_t)n);
  for (long long q = 0; q < e; ++q) adj[fill[src[q]]++] = dst[q];
  free(src); free(dst); free(fill);
  int* srp = (int*)malloc(sizeof(int) * ((size_t)n + 1));
  if (!srp) { free(cnt); free(adj); return -1; }
  int out = 0;
  srp[0] = 0;
  for (int i = 0; i < n; ++i) {
    const int b = cnt[i], len = cnt[i + 1] - cnt[i];
    qsort(adj + b, (size_t)len, sizeof(int), cmp_int);
    for (int q = 0; q < len; ++q)
      if (q == 0 || adj[b + q] != adj[b + q - 1]) adj[out++] = adj[b + q];
    srp[i + 1] = out;
  }
  free(cnt);
  *srp_out = srp;
  *scol_out = adj;
  return 0;
}

/* BFS level structure from r over unnumbered nodes; returns the number of levels and
   the smallest node of the last level in *last_min.  mark/stamp: visited iff mark[v] == stamp. */
static int bfs_levels(int r, const int* srp, const int* scol, const int* deg, const int* numbered, int* mark,
                      int stamp, int* queue, int* last_min) {
  int head = 0, tail = 0, levels = 0;
  queue[tail++] = r;
  mark[r] = stamp;
  while (head < tail) {
    const int level_end = tail;
    int best = -1;
    for (int q = head; q < level_end; ++q)
      if (best < 0 || cmp_deg_idx(deg, queue[q], best) < 0) best = queue[q];
    *last_min = best;
    levels++;
    for (; head < level_end; ++head) {
      const int u = queue[head];
      for (int p = srp[u]; p < srp[u + 1]; ++p) {
        const int v = scol[p];
        if (!numbered[v] && mark[v] != stamp) {
          mark[v] = stamp;
          queue[tail++] = v;
        }
      }
    }
  }
  return levels;
}

int orc_rcm(int n, const int* rptrs, const int* cids, int* perm) {
  int *srp = NULL, *scol = NULL;
  if (n <= 0) return 0;
  if (sym_pattern(n, rptrs, cids, &srp, &scol)) return -1;
  int* deg = (int*)malloc(sizeof(int) * (size_t)n);
  int* byrank = (int*)malloc(sizeof(int) * (size_t)n);
  int* numbered = (int*)calloc((size_t)n, sizeof(int));
  int* mark = (int*)calloc((size_t)n, sizeof(int));
  int* queue = (int*)malloc(sizeof(int) * (size_t)n);
  int* order = (int*)malloc(sizeof(int) * (size_t)n);
  int* nb = (int*)malloc(sizeof(int) * (size_t)n);
  if (!deg || !byrank || !numbered || !mark || !queue || !order || !nb) {
    free(srp); free(scol); free(deg); free(byrank); free(numbered); free(mark); free(queue); free(order); free(nb);
    return -1;
  }
  for (int v = 0; v < n; ++v) {
    deg[v] = srp[v + 1] - srp[v];
    byrank[v] = v;
  }
  g_sort_deg = deg;
  qsort(byrank, (size_t)n, sizeof(int), cmp_nodes); /* nodes by (degree, index) */
  int placed = 0, cursor = 0, stamp = 0;
  while (placed < n) {
    while (numbered[byrank[cursor]]) ++cursor;
    const int s = byrank[cursor];
    if (deg[s] == 0) { /* an isolated node: its own component */
      numbered[s] = 1;
      order[placed++] = s;
      continue;
    }
    /* pseudo-peripheral node of s's component */
    int r = s, last = s;
    int levels = bfs_levels(r, srp, scol, deg, numbered, mark, ++stamp, queue, &last);
    for (;;) {
      int last_x = last;
      const int x = last;
      const int lx = bfs_levels(x, srp, scol, deg, numbered, mark, ++stamp, queue, &last_x);
      if (lx > levels) {
        r = x;
        levels = lx;
        last = last_x;
      } else {
        break;
      }
    }
    /* Cuthill-McKee from r: each numbered node appends its unnumbered neighbours, smallest first */
    int head = placed;
    numbered[r] = 1;
    order[placed++] = r;
    while (head < placed) {
      const int u = order[head++];
      int k = 0;
      for (int p = srp[u]; p < srp[u + 1]; ++p)
        if (!numbered[scol[p]]) nb[k++] = scol[p];
      qsort(nb, (size_t)k, sizeof(int), cmp_nodes);
      for (int q = 0; q < k; ++q) {
        numbered[nb[q]] = 1;
        order[placed++] = nb[q];
      }
    }
  }
  for (int i = 0; i < n; ++i) perm[i] = order[n - 1 - i];
  free(srp); free(scol); free(deg); free(byrank); free(numbered); free(mark); free(queue); free(order); free(nb);
  return 0;
}

/*
 * B = P A P^T for perm (perm[i] = the row / column of A placed at i): row i of B is row
 * perm[i] of A with every column j renumbered to iperm[j], columns sorted ascending
 * (a stable sort, so repeated columns keep their order).  Values move with their entries.
 */
static const int* g_sort_key;
static int cmp_by_key(const void* a, const void* b) {
  const int x = g_sort_key[*(const int*)a], y = g_sort_key[*(const int*)b];
  if (x != y) return (x > y) - (x < y);
  return (*(const int*)a > *(const int*)b) - (*(const int*)a < *(const int*)b);
}

int orc_permute(int n, const int* rptrs, const int* cids, const double* val, const int* perm, int* brp, int* bcol,
                double* bval) {
  int* iperm = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  if (!iperm) return -1;
  for (int i = 0; i < n; ++i) iperm[perm[i]] = i;
  brp[0] = 0;
  for (int i = 0; i < n; ++i) brp[i + 1] = brp[i] + (rptrs[perm[i] + 1] - rptrs[perm[i]]);
  int maxlen = 0;
  for (int i = 0; i < n; ++i)
    if (rptrs[i + 1] - rptrs[i] > maxlen) maxlen = rptrs[i + 1] - rptrs[i];
  int* idx = (int*)malloc(sizeof(int) * (size_t)(maxlen > 0 ? maxlen : 1));
  int* key = (int*)malloc(sizeof(int) * (size_t)(maxlen > 0 ? maxlen : 1));
  if (!idx || !key) { free(iperm); free(idx); free(key); return -1; }
  for (int i = 0; i < n; ++i) {
    const int a = rptrs[perm[i]], len = rptrs[perm[i] + 1] - a;
    for (int q = 0; q < len; ++q) {
      idx[q] = q;
      key[q] = iperm[cids[a + q]];
    }
    g_sort_key = key;
    qsort(idx, (size_t)len, sizeof(int), cmp_by_key);
    for (int q = 0; q < len; ++q) {
      bcol[brp[i] + q] = key[idx[q]];
      if (val && bval) bval[brp[i] + q] = val[a + idx[q]];
    }
  }
  free(iperm); free(idx); free(key);
  return 0;
}

/* ------------------------------------------------- degree relabelling */

/*
 * Column relabelling by in-degree, hottest column first.  Sec. 4.1 and
 * Sec. 4.3 tie SpMV speed to how well the x accesses reuse cache lines, and
 * Sec. 4.4 reorders the matrix to improve that reuse; this is the column-only
 * reordering whose target is the reuse of the most frequently gathered x
 * entries (it leaves the rows, and so y, in place):
 *   deg[j]   = number of stored entries in column j;
 *   the columns are ranked by deg descending, ties by ascending column id;
 *   newid[j] = the rank of column j, 0 for the hottest.
 * The relabelled matrix keeps every row's entries in storage order with
 * cids'[p] = newid[cids[p]], and x'[newid[j]] = x[j], so that A' x' = A x
 * term by term.  Returns 0, -1 if a column id is outside [0, n), or -2 if a
 * scratch allocation fails.
 */
static const int* g_rl_deg; /* comparison context for qsort */
static int cmp_hot_first(const void* a, const void* b) {
  const int ja = *(const int*)a, jb = *(const int*)b;
  if (g_rl_deg[ja] != g_rl_deg[jb]) return g_rl_deg[ja] > g_rl_deg[jb] ? -1 : 1; /* more entries first */
  return (ja > jb) - (ja < jb);                                                   /* then by column id */
}

int orc_degree_relabel(int n, int nnz, const int* cids, int* newid) {
  int* deg = (int*)calloc((size_t)(n > 0 ? n : 1), sizeof(int));
  int* order = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  if (!deg || !order) { free(deg); free(order); return -2; }
  for (int p = 0; p < nnz; ++p) {
    if (cids[p] < 0 || cids[p] >= n) { free(deg); free(order); return -1; }
    deg[cids[p]] += 1;
  }
  for (int j = 0; j < n; ++j) order[j] = j;
  g_rl_deg = deg;
  qsort(order, (size_t)n, sizeof(int), cmp_hot_first);
  for (int q = 0; q < n; ++q) newid[order[q]] = q;
  free(deg);
  free(order);
  return 0;
}

/* ----------------------------------------------------------------- BCSR */

/*
 * Register blocking (Sec. 4.5): A is cut into aligned a x b regions (block
 * row I = rows I*a .. I*a+a-1, block column J = columns J*b .. J*b+b-1); every
 * region holding at least one stored entry becomes a dense block, zeros
 * included, and the list of blocks is stored as CRS over the ceil(m/a) block
 * rows: bptr[mb+1], bcol[nblocks] (block columns ascending within a block
 * row), bval[nblocks * a * b] with each block's values row major.  Repeated
 * entries add up, in storage order.  The first call with bcol == NULL only
 * returns the block count.
 */
long long orc_bcsr(int m, int n, const int* rptrs, const int* cids, const double* val, int a, int b, int* bptr,
                   int* bcol, double* bval) {
  const int mb = (m + a - 1) / a;
  int maxlen = 0;
  for (int I = 0; I < mb; ++I) {
    const int r1 = (I + 1) * a < m ? (I + 1) * a : m;
    const int len = rptrs[r1] - rptrs[I * a];
    if (len > maxlen) maxlen = len;
  }
  int* buf = (int*)malloc(sizeof(int) * (size_t)(maxlen > 0 ? maxlen : 1));
  if (!buf) return -1;
  long long nblocks = 0;
  if (bptr) bptr[0] = 0;
  for (int I = 0; I < mb; ++I) {
    const int r0 = I * a, r1 = (I + 1) * a < m ? (I + 1) * a : m;
    const int p0 = rptrs[r0], len = rptrs[r1] - p0;
    for (int q = 0; q < len; ++q) buf[q] = cids[p0 + q] / b;
    qsort(buf, (size_t)len, sizeof(int), cmp_int);
    const long long first = nblocks;
    for (int q = 0; q < len; ++q)
      if (q == 0 || buf[q] != buf[q - 1]) {
        if (bcol) bcol[nblocks] = buf[q];
        ++nblocks;
      }
    if (bptr) bptr[I + 1] = (int)nblocks;
    if (bcol && bval) {
      const long long nbI = nblocks - first;
      for (long long k = first * a * b; k < nblocks * a * b; ++k) bval[k] = 0.0;
      for (int i = r0; i < r1; ++i)
        for (int p = rptrs[i]; p < rptrs[i + 1]; ++p) {
          const int J = cids[p] / b;
          long long k = first;
          while (k < first + nbI && bcol[k] != J) ++k; /* the block of (i, J) */
          bval[k * a * b + (long long)(i - r0) * b + (cids[p] - J * b)] += val[p];
        }
    }
  }
  free(buf);
  (void)n;
  return nblocks;
}

/* y <- A x from the blocks: y_i = sum over the blocks of block row i/a of sum_c block[i%a][c] * x[J*b+c]
   (columns past n do not exist and are skipped), left to right; r = the same sum of |products|. */
void orc_bcsr_spmv(int m, int n, int a, int b, const int* bptr, const int* bcol, const double* bval,
                   const double* x, double* y, double* r) {
  const int mb = (m + a - 1) / a;
  for (int I = 0; I < mb; ++I)
    for (int rr = 0; rr < a && I * a + rr < m; ++rr) {
      double s = 0.0, t = 0.0;
      for (int k = bptr[I]; k < bptr[I + 1]; ++k)
        for (int c = 0; c < b; ++c) {
          const int j = bcol[k] * b + c;
          if (j >= n) continue;
          const double pr = bval[(long long)k * a * b + (long long)rr * b + c] * x[j];
          s = s + pr;
          t = t + fabs(pr);
        }
      y[I * a + rr] = s;
      if (r) r[I * a + rr] = t;
    }
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
