// Device helpers shared by the kernels: DoF existence / freedom masks of the structured
// layout (Dirichlet displacement on the boundary, natural pressure condition), and
// FP64 <-> FP32 conversions in integer arithmetic (on this GPU the hardware conversions
// issue to the FP64 pipe, at a quarter of its fused multiply-add rate).
#pragma once

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

// binary64 -> binary32 by truncation of the significand (rounding toward zero), from the two
// formats' bit layouts: the exponent is rebiased (1023 -> 127) and the top 23 of the 52
// fraction bits are kept.  Magnitudes below the binary32 normal range give a signed zero;
// magnitudes of 2^128 and above, infinities and NaNs give a NaN.  Integer instructions only,
// so the conversion does not occupy the FP64 pipe.
__device__ __forceinline__ float f64_to_f32_trunc(double v) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const unsigned e = (hi >> 20) & 0x7ffu;
  unsigned mag = (((hi << 3) | (lo >> 29)) - ((1023u - 127u) << 23)) & 0x7fffffffu;
  if (e < 1023u - 126u) mag = 0u;
  if (e > 1023u + 127u) mag = 0x7fc00000u;
  return __uint_as_float((hi & 0x80000000u) | mag);
}

// binary32 -> binary64, exact for normal numbers, infinities and NaNs (the exponent is rebiased
// 127 -> 1023 and the 23 fraction bits become the top of the 52); subnormal inputs give a
// signed zero.  Integer instructions only.
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  unsigned hi = u & 0x80000000u, lo = 0u;
  if (e != 0u) {
    const unsigned ed = e == 0xffu ? 0x7ffu : e + (1023u - 127u);
    hi |= (ed << 20) | ((u & 0x7fffffu) >> 3);
    lo = u << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// v = head + tail with head = f64_to_f32_trunc(v) and tail the 29 fraction bits that head
// drops, of which the top 23 are kept (relative error 2^-23 of the tail, 2^-46 of v): those
// 23 bits become an exact float by the magic-number construction (2^23 + m has m as its
// fraction field, and subtracting 2^23 is exact), scaled by 2^(e - 1069) (e the biased
// binary64 exponent) and given v's sign.  Integer and FP32 instructions only (no conversion
// instruction).  Tails below the FP32 normal range (|v| below about 2^-80) are dropped.
__device__ __forceinline__ void split_f64(double v, float &head, float &tail) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const unsigned e = (hi >> 20) & 0x7ffu;
  head = f64_to_f32_trunc(v);
  const float m = __fsub_rn(__uint_as_float(0x4b000000u | ((lo >> 6) & 0x7fffffu)), 8388608.0f);
  const float r = __fmul_rn(m, __uint_as_float((e - 942u) << 23));
  tail = (e > 942u && e < 1151u) ? __uint_as_float(__float_as_uint(r) ^ (hi & 0x80000000u)) : 0.f;
}

// One step of a double-float dot product: (sh, sl) += (ah + al) (bh + bl), dropping al bl.
// ah bh is split exactly into its rounded value and error (fused multiply-add), the running
// head sum takes it through the error-free two-sum (Knuth), and the tail collects both
// errors and the cross terms.  The _rn intrinsics keep the compiler from contracting or
// reassociating the steps.
__device__ __forceinline__ void df_dot_step(float ah, float al, float bh, float bl, float &sh, float &sl) {
  const float p = __fmul_rn(ah, bh);
  const float pe = __fmaf_rn(ah, bh, -p);
  const float c = __fmaf_rn(ah, bl, __fmul_rn(al, bh));
  const float t = __fadd_rn(sh, p);
  const float bb = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(__fadd_rn(pe, c), err));
}

}  // namespace bmg
