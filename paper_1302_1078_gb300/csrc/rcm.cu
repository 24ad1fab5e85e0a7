// Reverse Cuthill-McKee ordering and symmetric permutation on the device (the
// paper studies RCM's effect on SpMV in Sec. 4.4, using MATLAB's RCM; the
// tie-breaking rules below are this library's own, and the CPU oracle follows
// the same rules, so the two orders are equal element by element).
//
// Graph: the symmetric pattern of A + A^T of a square A, without self loops or
// repeated edges.  Nodes are compared by (degree, index).
//   1. Nodes of degree 0 come first, in index order.
//   2. While nodes remain, s = the smallest remaining node; a pseudo-
//      peripheral node r is found from s (George & Liu: BFS level structure
//      from r; x = the smallest node of its last level; if the structure
//      from x has more levels, r = x and repeat); Cuthill-McKee then numbers
//      r's component breadth first, each node appending its unnumbered
//      neighbours smallest first.
//   3. The order is reversed.
//
// Everything is built from the library's stable radix-sort transpose:
//   * A's rows sorted by column = (A^T)^T; S row i = merge of that row and
//     row i of A^T, without i and repeats;
//   * the nodes in (degree, index) order = a stable sort of the degrees;
//   * S's rows ordered by (degree, index) = the transpose of S with its rows
//     permuted into that order (the transpose lists each column's rows in
//     increasing row order).
// The Cuthill-McKee numbering is level synchronous and reproduces the
// sequential order exactly: a node of the next level is appended by its
// earliest numbered neighbour in the current level (an atomic minimum of
// positions, which does not depend on timing), and the children of one node
// come in its adjacency order, which is (degree, index).  So a level is: the
// parent minimum, a count per parent, an exclusive scan, and an ordered write.
// The host reads one count per level.
//
// The permutation B = P A P^T gathers rows, renumbers columns and sorts each
// row's columns with two stable transposes, so repeated columns keep their
// order; values follow their entries.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <vector>

#include "gbspmv.h"
#include "launch.h"

namespace gbs {

namespace {

constexpr int kThreads = 256;

int grid_for(long long work) {
  return (int)std::min<long long>(152LL * 32, std::max<long long>(1, (work + kThreads - 1) / kThreads));
}
int grid_warps(long long warps) { return grid_for(warps * 32); }

__global__ void iota_k(int* __restrict__ out, int n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) out[i] = i;
}

// Merge of two sorted lists per row without `i` and repeats: count (fill == false) or write.
template <bool FILL>
__global__ void sym_merge_k(int n, const int* __restrict__ rpa, const int* __restrict__ ca, const int* __restrict__ rpb,
                            const int* __restrict__ cb, int* __restrict__ cnt, const int* __restrict__ rps,
                            int* __restrict__ cs) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int p = rpa[i], pe = rpa[i + 1], q = rpb[i], qe = rpb[i + 1];
    int out = FILL ? rps[i] : 0, k = 0, last = -1;
    while (p < pe || q < qe) {
      int v;
      if (q >= qe || (p < pe && ca[p] <= cb[q]))
        v = ca[p++];
      else
        v = cb[q++];
      if (v == i || v == last) continue;
      last = v;
      if (FILL) cs[out + k] = v;
      ++k;
    }
    if (!FILL) cnt[i] = k;
  }
}

__global__ void degrees_k(int n, const int* __restrict__ rp, int* __restrict__ deg) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) deg[i] = rp[i + 1] - rp[i];
}

__global__ void rank_of_k(int n, const int* __restrict__ byrank, int* __restrict__ rank) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) rank[byrank[r]] = r;
}

// rows of S in rank order: length and copy
__global__ void qlen_k(int n, const int* __restrict__ byrank, const int* __restrict__ deg, int* __restrict__ qlen) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) qlen[r] = deg[byrank[r]];
}
__global__ void qfill_k(int n, const int* __restrict__ byrank, const int* __restrict__ rps, const int* __restrict__ cs,
                        const int* __restrict__ rpq, int* __restrict__ cq) {
  const int lane = threadIdx.x & 31;
  for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n;
       w += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int u = byrank[w];
    const int s = rps[u], len = rps[u + 1] - s, d = rpq[w];
    for (int k = lane; k < len; k += 32) cq[d + k] = cs[s + k];
  }
}
__global__ void map_k(long long cnt, const int* __restrict__ idx, const int* __restrict__ table, int* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (long long)gridDim.x * blockDim.x)
    out[i] = table[idx[i]];
}

__global__ void fill_k(int* __restrict__ a, int n, int v) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) a[i] = v;
}

// isolated nodes: the first `iso` nodes in rank order
__global__ void place_prefix_k(int iso, const int* __restrict__ byrank, int* __restrict__ order, int* __restrict__ pos) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < iso; r += (long long)gridDim.x * blockDim.x) {
    order[r] = byrank[r];
    pos[byrank[r]] = r;
  }
}
__global__ void count_zero_deg_k(int n, const int* __restrict__ deg, int* __restrict__ out) {
  int c = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) c += deg[i] == 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// smallest k in [b, e) whose node byrank[k] is not numbered
__global__ void find_unnumbered_k(int b, int e, const int* __restrict__ byrank, const int* __restrict__ pos,
                                  int* __restrict__ out) {
  for (long long k = b + (long long)blockIdx.x * blockDim.x + threadIdx.x; k < e; k += (long long)gridDim.x * blockDim.x)
    if (pos[byrank[k]] < 0) atomicMin(out, (int)k);
}

// one BFS level over unnumbered nodes, order-free (pseudo-peripheral search); warp per node
__global__ void bfs_level_k(const int* __restrict__ front, int fcount, const int* __restrict__ rp,
                            const int* __restrict__ adj, const int* __restrict__ pos, int* __restrict__ mark, int stamp,
                            const int* __restrict__ rank, int* __restrict__ next, int* __restrict__ info) {
  const int lane = threadIdx.x & 31;
  for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < fcount;
       w += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int u = front[w];
    for (int p = rp[u] + lane; p < rp[u + 1]; p += 32) {
      const int v = adj[p];
      if (pos[v] >= 0 || mark[v] == stamp) continue;
      if (atomicExch(&mark[v], stamp) != stamp) {
        next[atomicAdd(&info[0], 1)] = v;  // the level's order does not matter here
        atomicMin(&info[1], rank[v]);
      }
    }
  }
}

// Cuthill-McKee level: positions [f0, f1) are the current level (in order)
__global__ void cm_parent_k(const int* __restrict__ order, int f0, int f1, const int* __restrict__ rp,
                            const int* __restrict__ adj, const int* __restrict__ pos, int* __restrict__ parent) {
  const int lane = threadIdx.x & 31;
  for (long long q = f0 + (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5); q < f1;
       q += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int u = order[q];
    for (int p = rp[u] + lane; p < rp[u + 1]; p += 32) {
      const int v = adj[p];
      if (pos[v] < 0) atomicMin(&parent[v], (int)q);
    }
  }
}
__global__ void cm_count_k(const int* __restrict__ order, int f0, int f1, const int* __restrict__ rp,
                           const int* __restrict__ adj, const int* __restrict__ parent, int* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  for (long long q = f0 + (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5); q < f1;
       q += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int u = order[q];
    int c = 0;
    for (int b = rp[u]; b < rp[u + 1]; b += 32) {
      const int p = b + lane;
      const bool child = p < rp[u + 1] && parent[adj[p]] == (int)q;
      c += __popc(__ballot_sync(0xffffffffu, child));
    }
    if (lane == 0) cnt[q - f0] = c;
  }
}
// reads order[f0, f1) and writes order[f1, ...): the same array, disjoint ranges
__global__ void cm_write_k(const int* order_in, int f0, int f1, const int* __restrict__ rp,
                           const int* __restrict__ adj, const int* __restrict__ parent, const int* __restrict__ off,
                           int* order, int* __restrict__ pos) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (long long q = f0 + (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5); q < f1;
       q += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int u = order_in[q];
    int base = f1 + off[q - f0];
    for (int b = rp[u]; b < rp[u + 1]; b += 32) {
      const int p = b + lane;
      const int v = p < rp[u + 1] ? adj[p] : -1;
      const bool child = v >= 0 && parent[v] == (int)q;
      const unsigned m = __ballot_sync(0xffffffffu, child);
      if (child) {
        const int at = base + __popc(m & lt);
        order[at] = v;
        pos[v] = at;
      }
      base += __popc(m);
    }
  }
}
__global__ void last_sum_k(const int* __restrict__ off, const int* __restrict__ cnt, int k, int* __restrict__ out) {
  out[0] = off[k - 1] + cnt[k - 1];
}
__global__ void reverse_k(int n, const int* __restrict__ order, int* __restrict__ perm) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) perm[i] = order[n - 1 - i];
}
__global__ void set_one_k(int* __restrict__ order, int* __restrict__ pos, int at, int v) {
  order[at] = v;
  pos[v] = at;
}
__global__ void bfs_seed_k(int* __restrict__ front, int* __restrict__ mark, int root, int stamp) {
  front[0] = root;
  mark[root] = stamp;
}

// ---- permutation
__global__ void iperm_k(int n, const int* __restrict__ perm, int* __restrict__ iperm) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) iperm[perm[i]] = i;
}
__global__ void ulen_k(int n, const int* __restrict__ perm, const int* __restrict__ rp, int* __restrict__ len) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    len[i] = rp[perm[i] + 1] - rp[perm[i]];
}
__global__ void ufill_k(int n, const int* __restrict__ perm, const int* __restrict__ iperm, const int* __restrict__ rp,
                        const int* __restrict__ ci, const int* __restrict__ urp, int* __restrict__ ucol,
                        int* __restrict__ usrc) {
  const int lane = threadIdx.x & 31;
  for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n;
       w += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int a = rp[perm[w]], len = rp[perm[w] + 1] - a, d = urp[w];
    for (int k = lane; k < len; k += 32) {
      ucol[d + k] = iperm[ci[a + k]];
      usrc[d + k] = a + k;
    }
  }
}
template <typename T>
__global__ void gather_src_k(int nnz, const int* __restrict__ p2, const int* __restrict__ p1,
                             const int* __restrict__ usrc, const T* __restrict__ vals, T* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (long long)gridDim.x * blockDim.x)
    out[i] = vals[usrc[p1[p2[i]]]];
}

// Device scratch for transpose_run at up to `cap` nonzeros.
struct Tx {
  int *rows, *ka, *kb, *va, *vb, *hist, *ws;
};

size_t tx_ints(long long cap) {
  return 5 * (size_t)std::max<long long>(cap, 1) + transpose_hist_ints((int)cap) + transpose_scan_ws_ints((int)cap);
}
Tx tx_carve(int* base, long long cap) {
  Tx t;
  const size_t c = (size_t)std::max<long long>(cap, 1);
  t.rows = base;
  t.ka = base + c;
  t.kb = base + 2 * c;
  t.va = base + 3 * c;
  t.vb = base + 4 * c;
  t.hist = base + 5 * c;
  t.ws = t.hist + transpose_hist_ints((int)cap);
  return t;
}
cudaError_t tx_run(int m, int n, int nnz, const int* rp, const int* ci, int* rpT, int* colT, int* permT, Tx& t,
                   cudaStream_t s) {
  return transpose_run(m, n, nnz, rp, ci, rpT, colT, permT, t.rows, t.ka, t.kb, t.va, t.vb, t.hist, t.ws, s);
}

// Exclusive scan of n counts into out[0..n] (out[n] = total).
cudaError_t scan_counts(const int* cnt, int n, int* out, int* ws, int* tail, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (n > 0) e = exclusive_scan_i32(cnt, out, n, ws, s);
  if (e == cudaSuccess && n > 0) {
    last_sum_k<<<1, 1, 0, s>>>(out, cnt, n, tail);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out + n, tail, sizeof(int), cudaMemcpyDeviceToDevice, s);
  } else if (e == cudaSuccess) {
    e = cudaMemsetAsync(out, 0, sizeof(int), s);
  }
  return e;
}

cudaError_t read_int(const int* d, int* h, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace

cudaError_t rcm_run(int n, int nnz, const int* row_ptr, const int* col_idx, int* perm, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long cap = std::max<long long>(2LL * nnz, n);  // the largest array any transpose sees
  const size_t c = (size_t)std::max<long long>(cap, 1), nn = (size_t)n + 1;
  // layout (ints): A^T (nn + 2c), A sorted (nn + 2c), S (nn + c), deg/rank/byrank/order/pos/parent/mark
  // (7 nn), two frontiers (2 nn), counts / offsets (2 nn), Q (nn + c), Q^T (nn + 2c), adj (c),
  // small (64), transpose scratch
  const size_t ints = (nn + 2 * c) * 2 + (nn + c) + 7 * nn + 2 * nn + 2 * nn + (nn + c) + (nn + 2 * c) + c + 64 +
                      scan_workspace_ints((long long)nn) + tx_ints(cap);
  int* base = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&base), ints * sizeof(int), s);
  if (e != cudaSuccess) return e;
  int* p = base;
  auto take = [&](size_t k) {
    int* r = p;
    p += k;
    return r;
  };
  int *rpT = take(nn), *colT = take(c), *permT = take(c);
  int *rpA = take(nn), *colA = take(c), *permA = take(c);
  int *rpS = take(nn), *colS = take(c);
  int *deg = take(nn), *rank = take(nn), *byrank = take(nn), *order = take(nn), *pos = take(nn), *parent = take(nn),
      *mark = take(nn);
  int *fa = take(nn), *fb = take(nn);
  int *cnt = take(nn), *off = take(nn);
  int *rpQ = take(nn), *colQ = take(c);
  int *rpQT = take(nn), *colQT = take(c), *permQT = take(c);
  int* adj = take(c);
  int* small = take(64);
  int* sws = take(scan_workspace_ints((long long)nn));  // scans of up to n + 1 counts
  Tx tx = tx_carve(take(tx_ints(cap)), cap);

  do {
    // ---- symmetric pattern S of A + A^T
    if ((e = tx_run(n, n, nnz, row_ptr, col_idx, rpT, colT, permT, tx, s)) != cudaSuccess) break;
    if ((e = tx_run(n, n, nnz, rpT, colT, rpA, colA, permA, tx, s)) != cudaSuccess) break;  // A, rows sorted
    sym_merge_k<false><<<grid_for(n), kThreads, 0, s>>>(n, rpA, colA, rpT, colT, cnt, nullptr, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = scan_counts(cnt, n, rpS, sws, small, s)) != cudaSuccess) break;
    sym_merge_k<true><<<grid_for(n), kThreads, 0, s>>>(n, rpA, colA, rpT, colT, nullptr, rpS, colS);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    int nnzS = 0;
    if ((e = read_int(rpS + n, &nnzS, s)) != cudaSuccess) break;
    // ---- nodes in (degree, index) order: a stable sort of the degrees (one entry per row)
    degrees_k<<<grid_for(n), kThreads, 0, s>>>(n, rpS, deg);
    iota_k<<<grid_for(nn), kThreads, 0, s>>>(rpQ, n + 1);  // rpQ as the one-entry-per-row row_ptr
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = tx_run(n, n, n, rpQ, deg, rpQT, byrank, permQT, tx, s)) != cudaSuccess) break;
    rank_of_k<<<grid_for(n), kThreads, 0, s>>>(n, byrank, rank);
    // ---- S's rows in rank order, transposed: each node's neighbours in (degree, index) order
    qlen_k<<<grid_for(n), kThreads, 0, s>>>(n, byrank, deg, cnt);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = scan_counts(cnt, n, rpQ, sws, small, s)) != cudaSuccess) break;
    qfill_k<<<grid_warps(n), kThreads, 0, s>>>(n, byrank, rpS, colS, rpQ, colQ);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = tx_run(n, n, nnzS, rpQ, colQ, rpQT, colQT, permQT, tx, s)) != cudaSuccess) break;
    map_k<<<grid_for(nnzS), kThreads, 0, s>>>(nnzS, colQT, byrank, adj);  // rank -> node
    const int* rpAdj = rpQT;
    // ---- numbering
    fill_k<<<grid_for(n), kThreads, 0, s>>>(pos, n, -1);
    fill_k<<<grid_for(n), kThreads, 0, s>>>(parent, n, INT_MAX);
    fill_k<<<grid_for(n), kThreads, 0, s>>>(mark, n, 0);
    if ((e = cudaMemsetAsync(small, 0, sizeof(int), s)) != cudaSuccess) break;
    count_zero_deg_k<<<grid_for(n), kThreads, 0, s>>>(n, deg, small);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    int iso = 0;
    if ((e = read_int(small, &iso, s)) != cudaSuccess) break;
    if (iso > 0) place_prefix_k<<<grid_for(iso), kThreads, 0, s>>>(iso, byrank, order, pos);
    int placed = iso, cursor = iso, stamp = 0;
    // BFS level structure from root over unnumbered nodes: levels and the smallest rank of the last level
    auto bfs = [&](int root, int root_rank, int& levels, int& last_rank) -> cudaError_t {
      ++stamp;
      bfs_seed_k<<<1, 1, 0, s>>>(fa, mark, root, stamp);
      cudaError_t ee = cudaGetLastError();
      if (ee != cudaSuccess) return ee;
      int fcount = 1, cur_min = root_rank;
      int* f = fa;
      int* g = fb;
      levels = 0;
      for (;;) {
        levels++;
        int init[2] = {0, INT_MAX};
        if ((ee = cudaMemcpyAsync(small + 8, init, sizeof(init), cudaMemcpyHostToDevice, s)) != cudaSuccess) return ee;
        bfs_level_k<<<grid_warps(fcount), kThreads, 0, s>>>(f, fcount, rpAdj, adj, pos, mark, stamp, rank, g,
                                                             small + 8);
        if ((ee = cudaGetLastError()) != cudaSuccess) return ee;
        int got[2];
        if ((ee = cudaMemcpyAsync(got, small + 8, sizeof(got), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return ee;
        if ((ee = cudaStreamSynchronize(s)) != cudaSuccess) return ee;
        if (got[0] == 0) break;
        fcount = got[0];
        cur_min = got[1];
        std::swap(f, g);
      }
      last_rank = cur_min;
      return cudaSuccess;
    };
    while (placed < n && e == cudaSuccess) {
      // next start: the smallest unnumbered node in rank order at or after the cursor
      int found = INT_MAX;
      for (int w = 4096; cursor < n; w *= 2) {
        const int end = (int)std::min<long long>(n, (long long)cursor + w);
        int init = INT_MAX;
        if ((e = cudaMemcpyAsync(small + 16, &init, sizeof(int), cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
        find_unnumbered_k<<<grid_for(end - cursor), kThreads, 0, s>>>(cursor, end, byrank, pos, small + 16);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = read_int(small + 16, &found, s)) != cudaSuccess) break;
        if (found != INT_MAX) break;
        cursor = end;
      }
      if (e != cudaSuccess) break;
      if (found == INT_MAX) {
        e = cudaErrorUnknown;  // unreachable: placed < n means a node is unnumbered
        break;
      }
      cursor = found;
      int srank = found, s_node = 0;
      if ((e = cudaMemcpyAsync(&s_node, byrank + srank, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
      // pseudo-peripheral node (George & Liu)
      int r = s_node, levels = 0, last_rank = srank;
      if ((e = bfs(r, srank, levels, last_rank)) != cudaSuccess) break;
      for (;;) {
        int x = 0;
        if ((e = cudaMemcpyAsync(&x, byrank + last_rank, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
        int lx = 0, last_x = last_rank;
        if ((e = bfs(x, last_rank, lx, last_x)) != cudaSuccess) break;
        if (lx > levels) {
          r = x;
          levels = lx;
          last_rank = last_x;
        } else {
          break;
        }
      }
      if (e != cudaSuccess) break;
      // Cuthill-McKee from r
      set_one_k<<<1, 1, 0, s>>>(order, pos, placed, r);
      if ((e = cudaGetLastError()) != cudaSuccess) break;
      int f0 = placed, f1 = placed + 1;
      while (f1 > f0) {
        const int k = f1 - f0;
        cm_parent_k<<<grid_warps(k), kThreads, 0, s>>>(order, f0, f1, rpAdj, adj, pos, parent);
        cm_count_k<<<grid_warps(k), kThreads, 0, s>>>(order, f0, f1, rpAdj, adj, parent, cnt);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = scan_counts(cnt, k, off, sws, small + 24, s)) != cudaSuccess) break;
        cm_write_k<<<grid_warps(k), kThreads, 0, s>>>(order, f0, f1, rpAdj, adj, parent, off, order, pos);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        int total = 0;
        if ((e = read_int(off + k, &total, s)) != cudaSuccess) break;
        f0 = f1;
        f1 += total;
      }
      placed = f1;
    }
    if (e != cudaSuccess) break;
    reverse_k<<<grid_for(n), kThreads, 0, s>>>(n, order, perm);
    e = cudaGetLastError();
  } while (false);
  cudaError_t e2 = cudaFreeAsync(base, s);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

cudaError_t permute_run(int n, int nnz, const int* row_ptr, const int* col_idx, const void* vals, int dtype,
                        const int* perm, int* brp, int* bcol, void* bvals, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t c = (size_t)std::max(nnz, 1), nn = (size_t)n + 1;
  // iperm, lengths, U (ucol, usrc), T1 (rp, col, perm), T2 (perm), small, transpose scratch
  const size_t ints = nn + nn + 2 * c + (nn + 2 * c) + c + 64 + scan_workspace_ints((long long)nn) + tx_ints(nnz);
  int* base = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&base), ints * sizeof(int), s);
  if (e != cudaSuccess) return e;
  int* p = base;
  auto take = [&](size_t k) {
    int* r = p;
    p += k;
    return r;
  };
  int *iperm = take(nn), *len = take(nn), *ucol = take(c), *usrc = take(c);
  int *rp1 = take(nn), *col1 = take(c), *perm1 = take(c), *perm2 = take(c), *small = take(64);
  int* sws = take(scan_workspace_ints((long long)nn));
  Tx tx = tx_carve(take(tx_ints(nnz)), nnz);
  do {
    iperm_k<<<grid_for(n), kThreads, 0, s>>>(n, perm, iperm);
    ulen_k<<<grid_for(n), kThreads, 0, s>>>(n, perm, row_ptr, len);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = scan_counts(len, n, brp, sws, small, s)) != cudaSuccess) break;  // B's row_ptr
    ufill_k<<<grid_warps(n), kThreads, 0, s>>>(n, perm, iperm, row_ptr, col_idx, brp, ucol, usrc);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    // two stable transposes sort each row's columns; the second writes B's columns
    if ((e = tx_run(n, n, nnz, brp, ucol, rp1, col1, perm1, tx, s)) != cudaSuccess) break;
    if ((e = tx_run(n, n, nnz, rp1, col1, len, bcol, perm2, tx, s)) != cudaSuccess) break;  // len: scratch row_ptr
    if (vals && bvals && nnz > 0) {
      if (dtype == GBS_F64)
        gather_src_k<double><<<grid_for(nnz), kThreads, 0, s>>>(nnz, perm2, perm1, usrc,
                                                                static_cast<const double*>(vals),
                                                                static_cast<double*>(bvals));
      else
        gather_src_k<float><<<grid_for(nnz), kThreads, 0, s>>>(nnz, perm2, perm1, usrc,
                                                               static_cast<const float*>(vals),
                                                               static_cast<float*>(bvals));
      e = cudaGetLastError();
    }
  } while (false);
  cudaError_t e2 = cudaFreeAsync(base, s);
  if (e == cudaSuccess) e = e2;
  return e;
}

}  // namespace gbs
