/*
 * Seeded synthetic CSR matrices and dense operands.
 *
 * This module only builds inputs.  It holds none of the multiplication
 * arithmetic: it is shared by the CPU oracle tests and by the GPU library's
 * tests and benchmark, and neither side imports the other.
 *
 * Storage follows the compressed-row layout of the paper's Sec. 3 ("rptrs",
 * "cids", "val"): row_ptr[m+1] with row_ptr[0] = 0 and row_ptr[m] = nnz,
 * col_idx[nnz] in row-major order with ascending columns inside each row,
 * 32-bit indices (Sec. 4).
 *
 * Families (stand-ins for the paper's UFL test set, Table "tab:matrices"):
 *   - 2D 5-point Laplacian on an N x N grid (the paper's mesh_2048 is N=2048),
 *     diagonal 4, off-diagonals -1, Dirichlet boundary (missing neighbours
 *     are dropped), rows numbered i*N + j;
 *   - 3D 27-point stencil on N^3, diagonal 26, off-diagonals -1;
 *   - random banded "FEM-like": each row holds its diagonal plus distinct
 *     off-diagonal columns drawn uniformly from |i-j| <= hbw, N(0,1) values,
 *     diagonal = sum |off-diagonal| + 1;
 *   - R-MAT graph (Chakrabarti et al.), per-level quadrant choice with
 *     probabilities a, b, c, d = 1-a-b-c, duplicate edges removed, self
 *     loops kept, not symmetrised.
 *
 * Random numbers: splitmix64 seeds xoshiro256** streams (Blackman & Vigna).
 * Every stream is a pure function of (seed, stream id), so the output is the
 * same whatever the machine.  Uniform doubles take the top 53 bits.  Normal
 * deviates use Box-Muller through libm (last-bit differences across libm
 * builds are possible; nothing stored depends on them).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s[4]; } xo_t;

static uint64_t splitmix64(uint64_t* x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static void xo_seed(xo_t* r, uint64_t seed, uint64_t stream) {
  uint64_t x = seed * 0xD1B54A32D192ED03ULL + stream * 0x9E3779B97F4A7C15ULL + 0x632BE59BD9B4E019ULL;
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t xo_next(xo_t* r) {
  uint64_t* s = r->s;
  uint64_t result = rotl(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
  s[2] ^= t; s[3] = rotl(s[3], 45);
  return result;
}

/* uniform double in [0, 1) with 53 random bits */
static inline double xo_unit(xo_t* r) { return (double)(xo_next(r) >> 11) * 0x1.0p-53; }

/* uniform integer in [0, bound) (bound >= 1), Lemire's multiply-shift with rejection */
static inline uint32_t xo_below(xo_t* r, uint32_t bound) {
  uint64_t m = (uint64_t)(uint32_t)(xo_next(r) >> 32) * bound;
  uint32_t lo = (uint32_t)m;
  if (lo < bound) {
    uint32_t t = (uint32_t)(-bound) % bound;
    while (lo < t) {
      m = (uint64_t)(uint32_t)(xo_next(r) >> 32) * bound;
      lo = (uint32_t)m;
    }
  }
  return (uint32_t)(m >> 32);
}

/* ---------------------------------------------------------------- dense */

/* out[i] = lo + (hi - lo) * U[0,1), stream `stream` of `seed` */
void syn_uniform_f64(long long count, double lo, double hi, uint64_t seed, uint64_t stream, double* out) {
  xo_t r;
  xo_seed(&r, seed, stream);
  double w = hi - lo;
  for (long long i = 0; i < count; ++i) out[i] = lo + w * xo_unit(&r);
}

/* standard normal deviates (Box-Muller, both outputs used) */
void syn_normal_f64(long long count, uint64_t seed, uint64_t stream, double* out) {
  xo_t r;
  xo_seed(&r, seed, stream);
  const double two_pi = 6.283185307179586476925286766559;
  long long i = 0;
  while (i < count) {
    double u1 = xo_unit(&r), u2 = xo_unit(&r);
    if (u1 <= 0.0) continue;
    double rad = sqrt(-2.0 * log(u1));
    out[i++] = rad * cos(two_pi * u2);
    if (i < count) out[i++] = rad * sin(two_pi * u2);
  }
}

/* ------------------------------------------------------------- stencils */

/* 2D 5-point: m = N*N, nnz = 5N^2 - 4N.  Arrays sized by the caller. */
long long syn_stencil2d(int N, int* row_ptr, int* col_idx, double* vals) {
  long long p = 0;
  long long m = (long long)N * N;
  for (long long r = 0; r < m; ++r) {
    int i = (int)(r / N), j = (int)(r % N);
    row_ptr[r] = (int)p;
    /* ascending column order: (i-1,j) (i,j-1) (i,j) (i,j+1) (i+1,j) */
    if (i > 0) { col_idx[p] = (int)(r - N); vals[p] = -1.0; ++p; }
    if (j > 0) { col_idx[p] = (int)(r - 1); vals[p] = -1.0; ++p; }
    col_idx[p] = (int)r; vals[p] = 4.0; ++p;
    if (j < N - 1) { col_idx[p] = (int)(r + 1); vals[p] = -1.0; ++p; }
    if (i < N - 1) { col_idx[p] = (int)(r + N); vals[p] = -1.0; ++p; }
  }
  row_ptr[m] = (int)p;
  return p;
}

/* 3D 27-point: m = N^3, nnz = (3N-2)^3, rows numbered (i*N + j)*N + k. */
long long syn_stencil3d(int N, int* row_ptr, int* col_idx, double* vals) {
  long long p = 0;
  long long NN = (long long)N * N, m = NN * N;
  for (long long r = 0; r < m; ++r) {
    int i = (int)(r / NN), j = (int)((r / N) % N), k = (int)(r % N);
    row_ptr[r] = (int)p;
    for (int di = -1; di <= 1; ++di) {
      int ii = i + di;
      if (ii < 0 || ii >= N) continue;
      for (int dj = -1; dj <= 1; ++dj) {
        int jj = j + dj;
        if (jj < 0 || jj >= N) continue;
        for (int dk = -1; dk <= 1; ++dk) {
          int kk = k + dk;
          if (kk < 0 || kk >= N) continue;
          long long c = ((long long)ii * N + jj) * N + kk;
          col_idx[p] = (int)c;
          vals[p] = (c == r) ? 26.0 : -1.0;
          ++p;
        }
      }
    }
  }
  row_ptr[m] = (int)p;
  return p;
}

/* ---------------------------------------------------------------- banded */

static int cmp_int(const void* a, const void* b) {
  int x = *(const int*)a, y = *(const int*)b;
  return (x > y) - (x < y);
}

/* Row counts of the banded family: min(per_row, window size incl. diagonal). */
long long syn_banded_rowptr(int m, int hbw, int per_row, int* row_ptr) {
  long long p = 0;
  for (int i = 0; i < m; ++i) {
    row_ptr[i] = (int)p;
    long long lo = (long long)i - hbw < 0 ? 0 : (long long)i - hbw;
    long long hi = (long long)i + hbw > m - 1 ? m - 1 : (long long)i + hbw;
    long long w = hi - lo + 1;
    p += (w < per_row) ? w : per_row;
  }
  row_ptr[m] = (int)p;
  return p;
}

/*
 * Fill a banded matrix whose row_ptr came from syn_banded_rowptr.  Row i uses
 * its own random stream (seed, i), so the rows are independent of each other.
 */
void syn_banded_fill(int m, int hbw, uint64_t seed, const int* row_ptr, int* col_idx, double* vals) {
  int* stamp = (int*)malloc(sizeof(int) * (size_t)m);
  for (int i = 0; i < m; ++i) stamp[i] = -1;
  for (int i = 0; i < m; ++i) {
    xo_t r;
    xo_seed(&r, seed, (uint64_t)i);
    int lo = i - hbw < 0 ? 0 : i - hbw;
    int hi = i + hbw > m - 1 ? m - 1 : i + hbw;
    uint32_t w = (uint32_t)(hi - lo + 1);
    int cnt = row_ptr[i + 1] - row_ptr[i];
    int* c = col_idx + row_ptr[i];
    int got = 0;
    stamp[i] = i; /* the diagonal is always present */
    c[got++] = i;
    if ((uint32_t)cnt == w) {
      for (int j = lo; j <= hi; ++j)
        if (j != i) c[got++] = j;
    } else {
      while (got < cnt) {
        int j = lo + (int)xo_below(&r, w);
        if (stamp[j] == i) continue;
        stamp[j] = i;
        c[got++] = j;
      }
    }
    qsort(c, (size_t)cnt, sizeof(int), cmp_int);
    /* values: N(0,1) off-diagonal in column order, diagonal dominant */
    double* v = vals + row_ptr[i];
    const double two_pi = 6.283185307179586476925286766559;
    double abs_sum = 0.0, spare = 0.0;
    int have_spare = 0, diag_pos = -1;
    for (int q = 0; q < cnt; ++q) {
      if (c[q] == i) { diag_pos = q; continue; }
      double g;
      if (have_spare) { g = spare; have_spare = 0; }
      else {
        double u1, u2;
        do { u1 = xo_unit(&r); } while (u1 <= 0.0);
        u2 = xo_unit(&r);
        double rad = sqrt(-2.0 * log(u1));
        g = rad * cos(two_pi * u2);
        spare = rad * sin(two_pi * u2);
        have_spare = 1;
      }
      v[q] = g;
      abs_sum += fabs(g);
    }
    v[diag_pos] = abs_sum + 1.0;
  }
  free(stamp);
}

/* ----------------------------------------------------------------- R-MAT */

/*
 * Directed R-MAT edges, then a CSR with duplicates removed.  Edge block b
 * (2^16 edges) draws from stream b.  Each level consumes 21 random bits
 * (three levels per 64-bit draw), so the quadrant probabilities are resolved
 * to 2^-21.
 *
 * row_ptr has 2^scale + 1 entries; col_idx must hold ef * 2^scale entries.
 * Returns the number of nonzeros after deduplication.
 */
long long syn_rmat(int scale, int ef, double a, double b, double c, uint64_t seed, int* row_ptr, int* col_idx) {
  long long m = 1LL << scale;
  long long E = (long long)ef * m;
  uint32_t ta = (uint32_t)(a * 2097152.0);
  uint32_t tb = (uint32_t)((a + b) * 2097152.0);
  uint32_t tc = (uint32_t)((a + b + c) * 2097152.0);
  int* src = (int*)malloc(sizeof(int) * (size_t)E);
  int* dst = (int*)malloc(sizeof(int) * (size_t)E);
  const long long BLK = 1LL << 16;
  for (long long b0 = 0; b0 < E; b0 += BLK) {
    xo_t r;
    xo_seed(&r, seed, (uint64_t)(b0 / BLK));
    long long b1 = b0 + BLK < E ? b0 + BLK : E;
    for (long long e = b0; e < b1; ++e) {
      uint32_t row = 0, col = 0;
      uint64_t bits = 0;
      int avail = 0;
      for (int lvl = 0; lvl < scale; ++lvl) {
        if (avail == 0) { bits = xo_next(&r); avail = 3; }
        uint32_t u = (uint32_t)(bits & 0x1FFFFF);
        bits >>= 21;
        --avail;
        uint32_t rb = 0, cb = 0;
        if (u < ta) { rb = 0; cb = 0; }
        else if (u < tb) { rb = 0; cb = 1; }
        else if (u < tc) { rb = 1; cb = 0; }
        else { rb = 1; cb = 1; }
        row = (row << 1) | rb;
        col = (col << 1) | cb;
      }
      src[e] = (int)row;
      dst[e] = (int)col;
    }
  }
  /* counting sort by row */
  long long* cnt = (long long*)calloc((size_t)m + 1, sizeof(long long));
  for (long long e = 0; e < E; ++e) cnt[src[e] + 1]++;
  for (long long i = 0; i < m; ++i) cnt[i + 1] += cnt[i];
  long long* cur = (long long*)malloc(sizeof(long long) * (size_t)m);
  for (long long i = 0; i < m; ++i) cur[i] = cnt[i];
  for (long long e = 0; e < E; ++e) col_idx[cur[src[e]]++] = dst[e];
  free(cur);
  free(src);
  free(dst);
  /* per-row sort and dedup, compacting in place */
  long long p = 0;
  for (long long i = 0; i < m; ++i) {
    long long s = cnt[i], t = cnt[i + 1];
    row_ptr[i] = (int)p;
    if (t > s) qsort(col_idx + s, (size_t)(t - s), sizeof(int), cmp_int);
    for (long long q = s; q < t; ++q) {
      if (q > s && col_idx[q] == col_idx[q - 1]) continue;
      col_idx[p++] = col_idx[q];
    }
  }
  row_ptr[m] = (int)p;
  free(cnt);
  return p;
}
