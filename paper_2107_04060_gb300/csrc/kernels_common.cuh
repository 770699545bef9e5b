// Device helpers shared by the kernels: DoF existence / freedom masks of the structured
// layout (Dirichlet displacement on the boundary, natural pressure condition).
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

}  // namespace bmg
