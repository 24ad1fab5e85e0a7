// Device helpers shared by the gbspmv kernels: cache-steered loads, the
// shared-memory staging copy, and small vector types.
//
// Cache steering (GB300 has a 126 MB L2): the matrix streams (vals, col_idx,
// row_ptr) are read exactly once, so they are loaded with an L2 evict-first
// policy and without L1 allocation; the dense operand x / X is gathered many
// times at random and is loaded with an L2 evict-last policy, so that it
// stays in L2 while the streams pass through.  This is the GPU counterpart of
// the paper's observation (Sec. 4.1, Sec. 4.3) that SpMV speed follows how
// well the x accesses reuse cache lines.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gbs {

__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// ---- streaming loads (read once): no L1 allocation, L2 evict-first
__device__ __forceinline__ uint4 ld_stream_v4(const void* ptr, uint64_t pol) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(ptr), "l"(pol));
  return r;
}
__device__ __forceinline__ int ld_stream_i32(const int* ptr, uint64_t pol) {
  int r;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(r) : "l"(ptr), "l"(pol));
  return r;
}
__device__ __forceinline__ double ld_stream(const double* ptr, uint64_t pol) {
  double r;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(ptr), "l"(pol));
  return r;
}
__device__ __forceinline__ float ld_stream(const float* ptr, uint64_t pol) {
  float r;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r) : "l"(ptr), "l"(pol));
  return r;
}
__device__ __forceinline__ int ld_stream(const int* ptr, uint64_t pol) { return ld_stream_i32(ptr, pol); }

// Four doubles (one whole 32-byte sector) in one 256-bit load that skips L1, leaving L1 to the
// gathered x and the column sectors; ptr 32-byte aligned.
__device__ __forceinline__ void ld_stream_4d(const double* ptr, uint64_t pol, double* v) {
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f64 {%0,%1,%2,%3}, [%4], %5;"
               : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
               : "l"(ptr), "l"(pol));
}

// ---- streaming loads that do allocate in L1 (for per-thread contiguous segments whose
//      16-byte loads each use half of a 32-byte sector: the other half then hits L1)
__device__ __forceinline__ uint4 ld_stream_l1_v4(const void* ptr, uint64_t pol) {
  uint4 r;
  asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(ptr), "l"(pol));
  return r;
}

// ---- gathers of the dense operand (reused): L2 evict-last
__device__ __forceinline__ double ld_keep(const double* ptr, uint64_t pol) {
  double r;
  asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(ptr), "l"(pol));
  return r;
}
__device__ __forceinline__ float ld_keep(const float* ptr, uint64_t pol) {
  float r;
  asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r) : "l"(ptr), "l"(pol));
  return r;
}
__device__ __forceinline__ int ld_keep(const int* ptr, uint64_t pol) {
  int r;
  asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(r) : "l"(ptr), "l"(pol));
  return r;
}

// The same gathers without L1 allocation: for the entries of x that are rarely reused (the cold
// columns of a relabelled matrix), so that they do not evict the hot ones from L1.
__device__ __forceinline__ double ld_keep_na(const double* ptr, uint64_t pol) {
  double r;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(ptr), "l"(pol));
  return r;
}
__device__ __forceinline__ float ld_keep_na(const float* ptr, uint64_t pol) {
  float r;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r) : "l"(ptr), "l"(pol));
  return r;
}
__device__ __forceinline__ double2 ld_keep_v2(const double* ptr, uint64_t pol) {
  double2 r;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;" : "=d"(r.x), "=d"(r.y) : "l"(ptr), "l"(pol));
  return r;
}
__device__ __forceinline__ float4 ld_keep_v4(const float* ptr, uint64_t pol) {
  float4 r;
  asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
               : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
               : "l"(ptr), "l"(pol));
  return r;
}

// ---- streaming stores of the output (written once, not re-read): st.global.cs
__device__ __forceinline__ void st_stream(double* p, double v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(float* p, float v) { __stcs(p, v); }

// A VEC-wide slice of one row of the dense operand.
template <typename T, int VEC>
struct Vec {
  T v[VEC];
};

// Load VEC consecutive elements starting at p (16-byte aligned when VEC > 1).
template <typename T, int VEC>
__device__ __forceinline__ Vec<T, VEC> ld_keep_vec(const T* p, uint64_t pol) {
  Vec<T, VEC> r;
  if constexpr (VEC == 1) {
    r.v[0] = ld_keep(p, pol);
  } else if constexpr (VEC == 2) {
    static_assert(sizeof(T) == 8, "VEC 2 is for double");
    double2 t = ld_keep_v2(reinterpret_cast<const double*>(p), pol);
    r.v[0] = t.x;
    r.v[1] = t.y;
  } else {
    static_assert(VEC == 4 && sizeof(T) == 4, "VEC 4 is for float");
    float4 t = ld_keep_v4(reinterpret_cast<const float*>(p), pol);
    r.v[0] = t.x;
    r.v[1] = t.y;
    r.v[2] = t.z;
    r.v[3] = t.w;
  }
  return r;
}

// Store VEC consecutive elements with streaming stores (16-byte aligned when VEC > 1).
template <typename T, int VEC>
__device__ __forceinline__ void st_stream_vec(T* p, const T* v) {
  if constexpr (VEC == 1) {
    st_stream(p, v[0]);
  } else if constexpr (VEC == 2) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(v[0], v[1]));
  } else {
    __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
  }
}

// Copy g[a0 .. c1) into s[0 .. c1 - a0) with the whole CTA.  a0 is a multiple
// of 4 elements, so g + a0 is 16-byte aligned whenever g is (`aligned`); the
// body then moves in 128-bit streaming loads, and the ragged tail (and every
// element when g is not aligned) in scalar loads.  Nothing outside
// [a0, c1) is read.  s must be 16-byte aligned.
template <typename E>
__device__ __forceinline__ void stage_copy(E* __restrict__ s, const E* __restrict__ g, int a0, int c1, bool aligned,
                                           uint64_t pol) {
  const int cnt = c1 - a0;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (aligned) {
    constexpr int P = 16 / (int)sizeof(E);
    const int nvec = cnt / P;
    const char* src = reinterpret_cast<const char*>(g + a0);
    uint4* dst = reinterpret_cast<uint4*>(s);
    for (int q = tid; q < nvec; q += nt) dst[q] = ld_stream_v4(src + (size_t)q * 16, pol);
    for (int q = nvec * P + tid; q < cnt; q += nt) s[q] = ld_stream(g + a0 + q, pol);
  } else {
    for (int q = tid; q < cnt; q += nt) s[q] = ld_stream(g + a0 + q, pol);
  }
}

// s[0 .. c1 - a0) = vals[perm[a0 .. c1)] with the whole CTA: the permutation is read with
// 128-bit streaming loads when `aligned` (perm 16-byte aligned; a0 is a multiple of 4), and
// each thread then has four independent value gathers in flight.
template <typename T>
__device__ __forceinline__ void stage_gather(T* __restrict__ s, const T* __restrict__ vals,
                                             const int* __restrict__ perm, int a0, int c1, bool aligned,
                                             uint64_t pol) {
  const int cnt = c1 - a0;
  const int tid = threadIdx.x, nt = blockDim.x;
  int done = 0;
  if (aligned) {
    const int nvec = cnt / 4;
    for (int q = tid; q < nvec; q += nt) {
      const uint4 w = ld_stream_v4(perm + a0 + 4 * q, pol);
      const T v0 = __ldg(vals + (int)w.x), v1 = __ldg(vals + (int)w.y);
      const T v2 = __ldg(vals + (int)w.z), v3 = __ldg(vals + (int)w.w);
      s[4 * q] = v0;
      s[4 * q + 1] = v1;
      s[4 * q + 2] = v2;
      s[4 * q + 3] = v3;
    }
    done = nvec * 4;
  }
  for (int q = done + tid; q < cnt; q += nt) s[q] = __ldg(vals + ld_stream(perm + a0 + q, pol));
}

// Accumulator for one output element.  double: plain fused multiply-add in
// double.  float: the product is rounded once and added with Knuth's TwoSum,
// the rounding errors collected in a second float (compensated summation), so
// that long rows keep their accuracy; the FP32 pipe has ample headroom for it.
template <typename T>
struct Acc;

template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double x) { s = fma(a, x, s); }
  __device__ __forceinline__ void add_partial(double o) { s += o; }
  __device__ __forceinline__ double value() const { return s; }
  __device__ __forceinline__ void reset() { s = 0.0; }
};

template <>
struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float x) {
    float p = __fmul_rn(a, x);
    float t = __fadd_rn(s, p);
    float bp = __fsub_rn(t, s);
    float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s = t;
    c = __fadd_rn(c, e);
  }
  __device__ __forceinline__ void add_partial(float o) { add(o, 1.0f); }
  __device__ __forceinline__ float value() const { return __fadd_rn(s, c); }
  __device__ __forceinline__ void reset() { s = 0.f; c = 0.f; }
};

}  // namespace gbs
