// Device helpers shared by the fused COCG kernels.
#pragma once
#include <cuda_runtime.h>

#include "rpa_internal.cuh"

#include <type_traits>

#ifndef RPA_DOT_F64
#define RPA_DOT_F64 0
#endif

namespace rpa {

// Accumulator type of the COCG dot products (p^T w, r^T r, ||r||^2) inside the FP32 kernels:
// the working precision by default; FP64 (exact products of the FP32 values, FP64 sums) when
// built with RPA_DOT_F64=1.
template <typename T>
using dacc_t = typename std::conditional<RPA_DOT_F64 != 0, double, T>::type;

// periodic wrap (bc 0) of a grid index, or -1 outside a Dirichlet axis
static __device__ __forceinline__ int wrap_or_neg(int j, int n, int bc) {
  if (bc == 0) {
    while (j < 0) j += n;
    while (j >= n) j -= n;
    return j;
  }
  return (j < 0 || j >= n) ? -1 : j;
}

// Block reduction in the working precision (the partial sums of one block are short, so
// FP32 keeps ~1e-6 relative accuracy); thread 0 returns the totals.  FP64 arithmetic is
// avoided here because it runs at 1/58 of the FP32 rate on this GPU.
template <typename T, int NQ>
static __device__ __forceinline__ void block_sum_t(T (&v)[NQ], T* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) sh[wid * NQ + q] = v[q];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < nw; ++w)
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[q] += sh[w * NQ + q];
}

// ---- double-float arithmetic (each value an unevaluated sum hi + lo of two floats) ------
struct df {
  float hi, lo;
};
static __device__ __forceinline__ df df_of(double x) {
  const float h = __double2float_rn(x);
  return df{h, __double2float_rn(x - (double)h)};
}
static __device__ __forceinline__ double df_val(df a) { return (double)a.hi + (double)a.lo; }
// The error-free transformations below use the _rn intrinsics: they are never contracted
// into a fused multiply-add, which would round the product and void the exact error terms.
// s + e = a + b exactly (Knuth's two-sum)
static __device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return df{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// s + e = a + b exactly, |a| >= |b|
static __device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}
static __device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
static __device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
// acc + c * x with the product formed exactly in hi (Dekker's product through FMA)
static __device__ __forceinline__ df df_fma(df acc, df c, df x) {
  const float p = __fmul_rn(c.hi, x.hi);
  float e = __fmaf_rn(c.hi, x.hi, -p);
  e = __fmaf_rn(c.hi, x.lo, __fmaf_rn(c.lo, x.hi, e));
  const df s = two_sum(acc.hi, p);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(acc.lo, e)));
}
static __device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}
struct cdf {
  df re, im;
};
static __device__ __forceinline__ cdf cdf_of(const cpx<double>& v) { return cdf{df_of(v.re), df_of(v.im)}; }
// a complex value stored as (re.hi, re.lo, im.hi, im.lo)
static __device__ __forceinline__ cdf cdf_ld(const float4& v) { return cdf{df{v.x, v.y}, df{v.z, v.w}}; }

// four projector values of one entry (16-byte / 32-byte aligned vector loads)
static __device__ __forceinline__ void load_chi4(const float* p, float (&c)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  c[0] = v.x;
  c[1] = v.y;
  c[2] = v.z;
  c[3] = v.w;
}
static __device__ __forceinline__ void load_chi4(const double* p, double (&c)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  c[0] = a.x;
  c[1] = a.y;
  c[2] = b.x;
  c[3] = b.y;
}


}  // namespace rpa
