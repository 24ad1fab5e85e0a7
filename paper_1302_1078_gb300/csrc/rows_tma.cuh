// ROWS variant with persistent CTAs and a double-buffered bulk-copy pipeline
// ("ROWS_TMA").
//
// Same per-row arithmetic as rows_kernel.cuh (the paper's row-wise kernel,
// Sec. 4.1 / Sec. 5, with LANES lanes per row), but the nonzero stream of
// the next row block is copied into shared memory by the bulk-copy (TMA)
// engine while the CTA computes the current block:
//   * one thread issues cp.async.bulk copies of the block's vals and col_idx
//     ranges and arms an mbarrier with the expected byte count;
//   * every thread waits on that mbarrier (bounded) before computing;
//   * row_ptr of the block after next is prefetched into registers during
//     the compute and parked in a third row-pointer slot.
// CTAs are persistent (grid = resident CTA slots); CTA c takes row blocks
// c, c + grid, c + 2 grid, ...  The tile must hold the largest row block's
// nonzeros (+ 8); the plan checks this.  vals and col_idx must be 16-byte
// aligned.  The copies round the range out to 4-element boundaries; the
// last <= 3 nonzeros of the arrays, which cannot be rounded up without
// reading past the end, are loaded with plain loads.
//
// Every wait is bounded (1 s of GPU global time, with a poll count as a backstop): on timeout
// the kernel sets the device error flag, waits (again bounded) for the copies it issued, and
// returns.
//
// EMUL (FP64 only): in every unrolled group of 4 nonzeros, the first EMUL
// products run on the FP32 pipe (df64.cuh) and the rest on the FP64 pipe.
// The choice depends only on the loop position, so it is warp-uniform and
// never masks an FP64 instruction.  The float-float partial sums are flushed
// into the double accumulator every 16 groups (at most 48 terms).
#pragma once
#include "df64.cuh"
#include "device_common.cuh"
#include "rows_kernel.cuh"

namespace gbs {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait; returns false on timeout.  The limit is global time (1 s by default), with 2^22
// polls as a backstop should the timer not advance.  The timer is read only once the first
// poll has failed.
constexpr uint64_t kWaitLimitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (int i = 0; i < (1 << 22); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
  return false;
}


// Bulk copy global -> shared, completing on `bar`, with an L2 eviction policy (the matrix
// streams are read once: evict-first keeps the gathered vector resident in L2).
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <typename T>
__host__ __device__ inline size_t rows_tma_smem_bytes(int rpc, int tile) {
  size_t bars = 16;
  size_t rp = 3 * (((size_t)(rpc + 1) * sizeof(int) + 15) & ~(size_t)15);
  size_t val = (((size_t)tile + 8) * sizeof(T) + 15) & ~(size_t)15;
  size_t col = (((size_t)tile + 8) * sizeof(int) + 15) & ~(size_t)15;
  return bars + rp + 2 * (val + col);
}

// UNIT (SpMV with contiguous x and y): the strides are 1 and drop out of every address.
template <typename T, int VEC, int LANES, bool SPLIT, int EMUL, bool UNIT = false>
__global__ void __launch_bounds__(256) rows_tma_kernel(RowsArgs<T> a, int nblocks, int nnz, int* __restrict__ status) {
  static_assert(!UNIT || (SPLIT && VEC == 1), "unit strides are the SpMV form's");
  const long long ldx = UNIT ? 1 : a.ldx, ldy = UNIT ? 1 : a.ldy;
  static_assert(EMUL == 0 || sizeof(T) == 8, "FP32-pipe emulation is for double values");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int rpc = blockDim.x / LANES;
  const int tile = a.tile;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  const size_t rp_stride = ((size_t)(rpc + 1) * sizeof(int) + 15) & ~(size_t)15;
  int* s_rp_base = reinterpret_cast<int*>(smem_raw + 16);
  unsigned char* stage_base = smem_raw + 16 + 3 * rp_stride;
  const size_t val_bytes = (((size_t)tile + 8) * sizeof(T) + 15) & ~(size_t)15;
  const size_t col_bytes = (((size_t)tile + 8) * sizeof(int) + 15) & ~(size_t)15;
  auto s_rp = [&](int slot) { return reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(s_rp_base) + slot * rp_stride); };
  auto s_val = [&](int st) { return reinterpret_cast<T*>(stage_base + st * (val_bytes + col_bytes)); };
  auto s_col = [&](int st) { return reinterpret_cast<int*>(stage_base + st * (val_bytes + col_bytes) + val_bytes); };

  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_keep = policy_evict_last();
  const int tid = threadIdx.x;

  auto blk_of = [&](int i) { return blockIdx.x + i * gridDim.x; };
  auto rows_of = [&](int blk) { return min(rpc, a.m - blk * rpc); };

  // row_ptr entries of block blk into registers (thread t holds entry t; thread 0 also the last)
  auto load_rp = [&](int blk, int& v0, int& v1) {
    v0 = 0;
    v1 = 0;
    if (blk < nblocks) {
      const int nr = rows_of(blk);
      if (tid <= nr) v0 = ld_stream(a.row_ptr + blk * rpc + tid, pol_stream);
      if (tid == 0 && nr >= (int)blockDim.x) v1 = ld_stream(a.row_ptr + blk * rpc + nr, pol_stream);
    }
  };
  auto park_rp = [&](int blk, int slot, int v0, int v1) {
    if (blk < nblocks) {
      const int nr = rows_of(blk);
      int* d = s_rp(slot);
      if (tid <= nr) d[tid] = v0;
      if (tid == 0 && nr >= (int)blockDim.x) d[nr] = v1;
    }
  };
  // the copy of block blk into stage st (thread 0); rounds [s, e) out to 4-element boundaries
  auto issue = [&](int blk, int slot, int st) {
    const int nr = rows_of(blk);
    const int s = s_rp(slot)[0], e = s_rp(slot)[nr];
    const int a0 = s & ~3;
    int e_cp = (e + 3) & ~3;
    if (e_cp > nnz) e_cp = e & ~3;
    const uint32_t nv = e_cp > a0 ? (uint32_t)(e_cp - a0) : 0u;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bars[st], nv * (uint32_t)(sizeof(T) + sizeof(int)));
    if (nv) {
      bulk_copy_g2s(s_val(st), a.vals + a0, nv * (uint32_t)sizeof(T), &bars[st], pol_stream);
      bulk_copy_g2s(s_col(st), a.col_idx + a0, nv * (uint32_t)sizeof(int), &bars[st], pol_stream);
    }
  };

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    int v0, v1;
    load_rp(blk_of(0), v0, v1);
    park_rp(blk_of(0), 0, v0, v1);
    load_rp(blk_of(1), v0, v1);
    park_rp(blk_of(1), 1, v0, v1);
  }
  __syncthreads();
  if (tid == 0 && blk_of(0) < nblocks) issue(blk_of(0), 0, 0);

  const int g = tid / LANES;
  const int lane = tid % LANES;
  const int c_lo = SPLIT ? 0 : lane * VEC;
  const bool col_active = SPLIT ? true : (c_lo < a.k);
  const bool col_full = SPLIT ? true : (c_lo + VEC <= a.k);
  const T* __restrict__ Xc = a.X + c_lo;
  // row partials of the last two blocks (SpMV with LANES > 1), summed one iteration later
  __shared__ T s_red[SPLIT && LANES > 1 ? 2 * 256 : 1];
  __shared__ float2 s_redf[SPLIT && LANES > 1 && EMUL > 0 ? 2 * 256 : 1];  // the lanes' float-float pairs

  // Wait (bounded) for block j's copy in stage j & 1 and add the arrays' last <= 3 nonzeros
  // with plain loads; returns false on timeout.  The caller's barrier publishes the stage.
  auto arrive_block = [&](int j) {
    const int bj = blk_of(j);
    if (bj >= nblocks) return true;
    const int st = j & 1;
    const bool ok = mbar_wait_bounded(&bars[st], (uint32_t)((j >> 1) & 1));
    const int nr = rows_of(bj);
    const int* rp = s_rp(j % 3);
    const int s = rp[0], e = rp[nr];
    const int a0 = s & ~3;
    int e_cp = (e + 3) & ~3;
    if (e_cp > nnz) e_cp = e & ~3;
    if (e_cp < e && tid < e - e_cp) {
      s_val(st)[e_cp - a0 + tid] = a.vals[e_cp + tid];
      s_col(st)[e_cp - a0 + tid] = a.col_idx[e_cp + tid];
    }
    return ok;
  };
  // Row sums of block j from s_red (SpMV with LANES > 1): one thread per row adds the LANES
  // partials in lane order, so a warp of rows shares each FP64 add.
  auto finish_rows = [&](int j) {
    if constexpr (SPLIT && LANES > 1) {
      const int bj = blk_of(j);
      const int nr = rows_of(bj);
      const T* red = s_red + (j & 1) * 256;
      if (tid < nr) {
        T sum = red[tid * LANES];
#pragma unroll
        for (int l = 1; l < LANES; ++l) sum += red[tid * LANES + l];
        if constexpr (EMUL > 0) {
          const float2* rf = s_redf + (j & 1) * 256;
          DFAcc e;
          e.s = rf[tid * LANES].x;
          e.c = rf[tid * LANES].y;
#pragma unroll
          for (int l = 1; l < LANES; ++l) {
            DFAcc o;
            o.s = rf[tid * LANES + l].x;
            o.c = rf[tid * LANES + l].y;
            e.merge(o);
          }
          sum += (T)e.value();
        }
        st_stream(a.Y + (long long)(bj * rpc + tid) * ldy, sum);
      }
    }
  };

  bool abort = __syncthreads_or(!arrive_block(0)) != 0;
  int i = 0;
  for (; !abort && blk_of(i) < nblocks; ++i) {
    // One barrier per block.  At the top of iteration i, stage i & 1 holds block i (waited
    // for at the end of the previous iteration) and stage (i + 1) & 1 is free.
    const int blk = blk_of(i), st = i & 1, slot = i % 3;
    if (tid == 0 && blk_of(i + 1) < nblocks) issue(blk_of(i + 1), (i + 1) % 3, st ^ 1);
    int pv0, pv1;
    load_rp(blk_of(i + 2), pv0, pv1);  // parked at the end of this iteration
    if (i > 0) finish_rows(i - 1);
    const int nr = rows_of(blk);
    const int* rp = s_rp(slot);
    const int a0 = rp[0] & ~3;
    const T* sv = s_val(st);
    const int* sc = s_col(st);

    // ---- compute the rows of block blk from stage st
    const bool active = g < nr;
    Acc<T> acc[VEC];
    DFAcc eacc[EMUL > 0 ? VEC : 1];
    if constexpr (SPLIT) {
      {
        // SpMV: software-pipelined walk of this lane's nonzeros p, p + STEP, ... < re.  The
        // gathers of group q + 1 are issued before the FMAs of group q wait for theirs, and
        // the last 0..3 nonzeros are gathered together, so a row costs about one round trip
        // to L2 per two groups instead of one per group and one per leftover nonzero.  The
        // products are added in the same order as a plain walk (with EMUL > 0 the first
        // EMUL products of every full group go to the float-float accumulator, flushed
        // into the double one every 16 groups).  Every lane of the warp runs the walk (a lane
        // without a row has no nonzeros), so that the tail can skip warp-wide a product no
        // lane needs: a warp FP64 instruction costs its full pipe slot whatever its mask.
        const int rs = active ? rp[g] : 0, re = active ? rp[g + 1] : 0;
        constexpr int STEP = LANES;
        const int p = rs + lane;
        const int cnt = p < re ? (re - p + STEP - 1) / STEP : 0;
        const int full = cnt / kUnroll;
        T va[kUnroll], vb[kUnroll];
        T xa[kUnroll], xb[kUnroll];
        auto fetch = [&](int q0, T* v, T* x) {
          int c[kUnroll];
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            v[u] = sv[p + (q0 + u) * STEP - a0];
            c[u] = sc[p + (q0 + u) * STEP - a0];
          }
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) x[u] = ld_keep(Xc + (long long)c[u] * ldx, pol_keep);
        };
        int egroups = 0;
        auto fma4 = [&](const T* v, const T* x) {
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            if constexpr (EMUL > 0) {
              if (u < EMUL) {
                float ah, al, xh, xl;
                const bool oka = split_f64((double)v[u], ah, al);
                const bool okx = split_f64((double)x[u], xh, xl);
                if (oka && okx)
                  eacc[0].add(ah, al, xh, xl);
                else
                  acc[0].add(v[u], x[u]);  // out of the FP32 range: native pipe
                continue;
              }
            }
            acc[0].add(v[u], x[u]);
          }
          if constexpr (EMUL > 0) {
            if (++egroups == 16) {
              egroups = 0;
              acc[0].add_partial((T)eacc[0].value());
              eacc[0].reset();
            }
          }
        };
        if (full > 0) {
          fetch(0, va, xa);
          int gi = 1;
          for (; gi + 1 < full; gi += 2) {
            fetch(gi * kUnroll, vb, xb);
            fma4(va, xa);
            fetch((gi + 1) * kUnroll, va, xa);
            fma4(vb, xb);
          }
          if (gi < full) {
            fetch(gi * kUnroll, vb, xb);
            fma4(va, xa);
            fma4(vb, xb);
          } else {
            fma4(va, xa);
          }
        }
        const int rem = cnt - full * kUnroll;
        const int q0 = full * kUnroll;
#pragma unroll
        for (int u = 0; u < kUnroll - 1; ++u)
          if (u < rem) {
            vb[u] = sv[p + (q0 + u) * STEP - a0];
            xb[u] = ld_keep(Xc + (long long)sc[p + (q0 + u) * STEP - a0] * ldx, pol_keep);
          }
        // A guarded product would be computed on every lane and kept by a select (a multiply-add
        // has no side effects, so the compiler may lift it out of its branch).  For double values
        // the product is a volatile instruction, which runs only on the lanes that need it, and a
        // warp-wide test skips a product no lane needs.  (Counting the tail's products by a warp
        // vote in a loop issues fewer FP64 instructions but was slower: the vote serialises.)
#pragma unroll
        for (int u = 0; u < kUnroll - 1; ++u)
          if (__any_sync(0xffffffffu, u < rem)) {
            if (u < rem) {
              if constexpr (sizeof(T) == 8)
                asm volatile("fma.rn.f64 %0, %1, %2, %0;" : "+d"(acc[0].s) : "d"(vb[u]), "d"(xb[u]));
              else
                acc[0].add(vb[u], xb[u]);
            }
          }
        // one lane per row: fold the float-float partial in now; several lanes: the row's
        // reduction merges the lanes' pairs in FP32 and converts once per row
        if constexpr (EMUL > 0 && LANES == 1) acc[0].add_partial((T)eacc[0].value());
      }
    } else if (active && col_active) {
      const int rs = rp[g], re = rp[g + 1];
      constexpr int STEP = 1;
      int p = rs;
      if (EMUL == 0 && col_full) {
        // SpMM (the lane owns VEC columns and walks the whole row): the same software
        // pipeline as the SpMV walk, each gather a VEC-wide slice of an X row
        const int cnt = re - p;
        const int full = cnt / kUnroll;
        T va[kUnroll], vb[kUnroll];
        Vec<T, VEC> xa[kUnroll], xb[kUnroll];
        auto fetch = [&](int q0, T* v, Vec<T, VEC>* x) {
          int c[kUnroll];
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            v[u] = sv[p + q0 + u - a0];
            c[u] = sc[p + q0 + u - a0];
          }
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) x[u] = ld_keep_vec<T, VEC>(Xc + (long long)c[u] * ldx, pol_keep);
        };
        auto fma4 = [&](const T* v, const Vec<T, VEC>* x) {
#pragma unroll
          for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int j = 0; j < VEC; ++j) acc[j].add(v[u], x[u].v[j]);
        };
        if (full > 0) {
          fetch(0, va, xa);
          int gi = 1;
          for (; gi + 1 < full; gi += 2) {
            fetch(gi * kUnroll, vb, xb);
            fma4(va, xa);
            fetch((gi + 1) * kUnroll, va, xa);
            fma4(vb, xb);
          }
          if (gi < full) {
            fetch(gi * kUnroll, vb, xb);
            fma4(va, xa);
            fma4(vb, xb);
          } else {
            fma4(va, xa);
          }
        }
        for (int q = full * kUnroll; q < cnt; ++q) {
          Vec<T, VEC> xv = ld_keep_vec<T, VEC>(Xc + (long long)sc[p + q - a0] * ldx, pol_keep);
#pragma unroll
          for (int j = 0; j < VEC; ++j) acc[j].add(sv[p + q - a0], xv.v[j]);
        }
      } else if (col_full) {
        int groups = 0;
        for (; p + (kUnroll - 1) * STEP < re; p += kUnroll * STEP) {
          T v[kUnroll];
          int c[kUnroll];
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            v[u] = sv[p + u * STEP - a0];
            c[u] = sc[p + u * STEP - a0];
          }
          Vec<T, VEC> xv[kUnroll];
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) xv[u] = ld_keep_vec<T, VEC>(Xc + (long long)c[u] * ldx, pol_keep);
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            if constexpr (EMUL > 0) {
              if (u < EMUL) {
                float ah, al;
                const bool oka = split_f64((double)v[u], ah, al);
#pragma unroll
                for (int j = 0; j < VEC; ++j) {
                  float xh, xl;
                  const bool okx = split_f64((double)xv[u].v[j], xh, xl);
                  if (oka && okx)
                    eacc[j].add(ah, al, xh, xl);
                  else
                    acc[j].add(v[u], xv[u].v[j]);  // out of the FP32 range: native pipe
                }
                continue;
              }
            }
#pragma unroll
            for (int j = 0; j < VEC; ++j) acc[j].add(v[u], xv[u].v[j]);
          }
          if constexpr (EMUL > 0) {
            if (++groups == 16) {
              groups = 0;
#pragma unroll
              for (int j = 0; j < VEC; ++j) {
                acc[j].add_partial((T)eacc[j].value());
                eacc[j].reset();
              }
            }
          }
        }
        if constexpr (EMUL > 0) {
#pragma unroll
          for (int j = 0; j < VEC; ++j) acc[j].add_partial((T)eacc[j].value());
        }
        for (; p < re; p += STEP) {
          Vec<T, VEC> xv = ld_keep_vec<T, VEC>(Xc + (long long)sc[p - a0] * ldx, pol_keep);
#pragma unroll
          for (int j = 0; j < VEC; ++j) acc[j].add(sv[p - a0], xv.v[j]);
        }
      } else {
        const int nv = a.k - c_lo;
        for (; p < re; p += STEP) {
          const T* xr = Xc + (long long)sc[p - a0] * ldx;
#pragma unroll
          for (int j = 0; j < VEC; ++j)
            if (j < nv) acc[j].add(sv[p - a0], ld_keep(xr + j, pol_keep));
        }
      }
    }
    const int r0 = blk * rpc;
    if constexpr (SPLIT && LANES > 1) {
      s_red[st * 256 + tid] = acc[0].value();
      if constexpr (EMUL > 0) s_redf[st * 256 + tid] = make_float2(eacc[0].s, eacc[0].c);
    } else if constexpr (SPLIT) {
      if (active) st_stream(a.Y + (long long)(r0 + g) * ldy, acc[0].value());
    } else {
      if (active && col_active) {
        T out[VEC];
#pragma unroll
        for (int j = 0; j < VEC; ++j) out[j] = acc[j].value();
        T* yr = a.Y + (long long)(r0 + g) * ldy + c_lo;
        if (col_full)
          st_stream_vec<T, VEC>(yr, out);
        else
          for (int j = 0; j < a.k - c_lo; ++j) st_stream(yr + j, out[j]);
      }
    }
    park_rp(blk_of(i + 2), (i + 2) % 3, pv0, pv1);
    const bool ok = arrive_block(i + 1);
    fence_proxy_async_smem();  // generic accesses to stage st before the bulk engine reuses it
    // stage st, row slot i % 3 and s_red half st ^ 1 are free again; block i + 1 is published
    abort = __syncthreads_or(!ok) != 0;
  }
  if (abort) {
    // a wait gave up for block i (i is the block the loop stopped at, waited for after
    // iteration i - 1 or in the prologue): the only copy this CTA may still have in flight is
    // block i's, so wait (bounded) for it before the CTA leaves
    if (tid == 0) atomicOr(status, 1);
    mbar_wait_bounded(&bars[i & 1], (uint32_t)((i >> 1) & 1));
    return;
  }
  if (i > 0) finish_rows(i - 1);
}

}  // namespace gbs
