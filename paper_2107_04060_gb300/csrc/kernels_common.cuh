// Device helpers shared by the kernels: DoF existence / freedom masks of the structured
// layout (Dirichlet displacement on the boundary, natural pressure condition), and
// FP64 <-> FP32 conversions in integer arithmetic (on this GPU the hardware conversions
// issue to the FP64 pipe, at a quarter of its fused multiply-add rate).
#pragma once

#include <cmath>
#include <cstring>
#include <type_traits>
#include <utility>

#include "bmg_internal.h"

namespace bmg {

// P1 displacement at vertex (i, j) is free iff the vertex is interior.
__device__ __forceinline__ bool vfree(int i, int j, int n) {
  return i > 0 && i < n && j > 0 && j < n;
}

// Which slots at grid position (i, j) (0 <= i, j <= n) hold free DoFs, per block.
__device__ __forceinline__ void dof_masks(int i, int j, int n, bool m[NBLK]) {
  const bool in_i = i < n, in_j = j < n;
  m[UX] = m[UY] = vfree(i, j, n);
  m[BH] = in_i && j > 0 && j < n;
  m[BV] = in_j && i > 0 && i < n;
  m[BD] = in_i && in_j;
  m[WH] = in_i;
  m[WV] = in_j;
  m[WD] = m[PL] = m[PU] = in_i && in_j;
}

// Compile-time loop: f(std::integral_constant<int, I>) for I = 0 .. N-1, so that the body
// can branch on the index with `if constexpr` and index arrays with constants.
template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F &f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F &&f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// Bit casts and correctly rounded FP32 steps for the conversion and double-float helpers
// below: device intrinsics on the GPU (the _rn forms are never contracted or reassociated),
// plain IEEE operations on the host, where the helpers are compiled only for checking.
namespace fbits {
__host__ __device__ __forceinline__ unsigned hi32(double v) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2hiint(v);
#else
  unsigned long long u;
  std::memcpy(&u, &v, sizeof u);
  return (unsigned)(u >> 32);
#endif
}
__host__ __device__ __forceinline__ unsigned lo32(double v) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2loint(v);
#else
  unsigned long long u;
  std::memcpy(&u, &v, sizeof u);
  return (unsigned)u;
#endif
}
__host__ __device__ __forceinline__ double make_f64(unsigned hi, unsigned lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const unsigned long long u = ((unsigned long long)hi << 32) | lo;
  double v;
  std::memcpy(&v, &u, sizeof v);
  return v;
#endif
}
__host__ __device__ __forceinline__ float as_f32(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, sizeof f);
  return f;
#endif
}
__host__ __device__ __forceinline__ unsigned as_u32(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  std::memcpy(&u, &f, sizeof u);
  return u;
#endif
}
#ifdef __CUDA_ARCH__
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
inline float add(float a, float b) { return a + b; }
inline float sub(float a, float b) { return a - b; }
inline float mul(float a, float b) { return a * b; }
inline float fma(float a, float b, float c) { return std::fma(a, b, c); }
#endif
}  // namespace fbits

// binary64 -> binary32 by truncation of the significand (rounding toward zero), from the two
// formats' bit layouts: the exponent is rebiased (1023 -> 127) and the top 23 of the 52
// fraction bits are kept.  Magnitudes below the binary32 normal range give a signed zero;
// magnitudes of 2^128 and above, infinities and NaNs give a NaN.  Integer instructions only,
// so the conversion does not occupy the FP64 pipe.
__host__ __device__ __forceinline__ float f64_to_f32_trunc(double v) {
  const unsigned hi = fbits::hi32(v), lo = fbits::lo32(v);
  const unsigned e = (hi >> 20) & 0x7ffu;
  unsigned mag = (((hi << 3) | (lo >> 29)) - ((1023u - 127u) << 23)) & 0x7fffffffu;
  if (e < 1023u - 126u) mag = 0u;
  if (e > 1023u + 127u) mag = 0x7fc00000u;
  return fbits::as_f32((hi & 0x80000000u) | mag);
}

// binary32 -> binary64, exact for normal numbers, infinities and NaNs (the exponent is rebiased
// 127 -> 1023 and the 23 fraction bits become the top of the 52); subnormal inputs give a
// signed zero.  Integer instructions only.
__host__ __device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned u = fbits::as_u32(f);
  const unsigned e = (u >> 23) & 0xffu;
  unsigned hi = u & 0x80000000u, lo = 0u;
  if (e != 0u) {
    const unsigned ed = e == 0xffu ? 0x7ffu : e + (1023u - 127u);
    hi |= (ed << 20) | ((u & 0x7fffffu) >> 3);
    lo = u << 29;
  }
  return fbits::make_f64(hi, lo);
}

// v = head + tail with head = f64_to_f32_trunc(v) and tail the 29 fraction bits that head
// drops, of which the top 23 are kept (relative error 2^-23 of the tail, 2^-46 of v): those
// 23 bits become an exact float by the magic-number construction (2^23 + m has m as its
// fraction field, and subtracting 2^23 is exact), scaled by 2^(e - 1069) (e the biased
// binary64 exponent) and given v's sign.  Integer and FP32 instructions only (no conversion
// instruction).  Tails below the FP32 normal range (|v| below about 2^-80) are dropped.
__host__ __device__ __forceinline__ void split_f64(double v, float &head, float &tail) {
  const unsigned hi = fbits::hi32(v), lo = fbits::lo32(v);
  const unsigned e = (hi >> 20) & 0x7ffu;
  head = f64_to_f32_trunc(v);
  const float m = fbits::sub(fbits::as_f32(0x4b000000u | ((lo >> 6) & 0x7fffffu)), 8388608.0f);
  const float r = fbits::mul(m, fbits::as_f32((e - 942u) << 23));
  tail = (e > 942u && e < 1151u) ? fbits::as_f32(fbits::as_u32(r) ^ (hi & 0x80000000u)) : 0.f;
}

// One step of a double-float dot product: (sh, sl) += (ah + al) (bh + bl), dropping al bl.
// ah bh is split exactly into its rounded value and error (fused multiply-add), the running
// head sum takes it through the error-free two-sum (Knuth), and the tail collects both
// errors and the cross terms.
__host__ __device__ __forceinline__ void df_dot_step(float ah, float al, float bh, float bl, float &sh, float &sl) {
  const float p = fbits::mul(ah, bh);
  const float pe = fbits::fma(ah, bh, -p);
  const float c = fbits::fma(ah, bl, fbits::mul(al, bh));
  const float t = fbits::add(sh, p);
  const float bb = fbits::sub(t, sh);
  const float err = fbits::add(fbits::sub(sh, fbits::sub(t, bb)), fbits::sub(p, bb));
  sh = t;
  sl = fbits::add(sl, fbits::add(fbits::add(pe, c), err));
}

}  // namespace bmg
