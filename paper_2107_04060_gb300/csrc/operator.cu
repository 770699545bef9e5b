// Matrix-free application of the reduced-quadrature Biot operator (Sec. 2.3,
// Eq. block_form_rq) on the structured triangulation: y = A x or r = b - A x.
//
// Element-gather design: a CTA owns a tile of output positions.  Phase 1 computes, one task
// per cell, the local products of the cell's two triangles into 20 shared-memory slots (the
// rows of the six DoFs the two triangles share continue one sum), for the tile's cells and
// for a one-cell halo on the low side, where only the rows the tile's DoFs need are formed;
// phase 2 gathers, for every DoF of the tile, the slots of the cells around it (4 for a
// vertex, 2 for an edge off the diagonal, 1 otherwise).  No atomics: the result is
// deterministic.
// Constrained displacement slots are ignored on input and written as 0.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <utility>

#include "bmg_internal.h"
#include "kernels_common.cuh"

namespace bmg {

template <typename T>
struct ApplyArgs {
  Grid g;
  const T *x;
  const T *b;        // residual mode only
  T *y;
  const T *kinv;     // [2][blk]          (WM == 0)
  const T *wm;       // [2][6][blk]       (WM == 1)
  size_t bstride;    // batch stride (elements) for batched application
  int residual;
  int wm_full;       // batched form only: per-instance choice between kinv and wm
  const int *gate;
  OpCoefs<T> c;
};


// Local product of one triangle, accumulated: yl[a] += (E_T xl)_a for the rows a in ROWS
// (bit a; 13 rows), xl = (u[9], w[3], p).  Products with the structural zeros of the
// element matrices are not formed (Aeps 30 of 81, g 2 of 9, the unit RT0 mass 4 of 9; see
// kElemNonzeros), and neither are the rows outside ROWS nor the shared terms only they use.
// Every row is one chain of fused multiply-adds starting from yl[a], so a row that continues
// another triangle's sum for the same DoF costs no separate addition.
constexpr unsigned kAllRows = 0x1fffu;

template <unsigned ROWS>
__host__ __device__ constexpr bool rows_need_gu() {
  bool need = (ROWS >> 12) & 1u;                   // the pressure row
  for (int a = 0; a < 9; ++a) need = need || (((ROWS >> a) & 1u) && g_nonzero(a));
  return need;
}
template <unsigned ROWS>
__host__ __device__ constexpr bool rows_need_s() {
  bool need = false;
  for (int a = 0; a < 9; ++a) need = need || (((ROWS >> a) & 1u) && g_nonzero(a));
  return need;
}

template <typename T, int WM, unsigned ROWS, bool DENSE = false>
__device__ __forceinline__ void tri_product(const OpCoefs<T> &c, int o, const T u[9],
                                            const T w[3], T p, T kinv, const T *wmT,
                                            T *yl) {
  T gu = 0, s = 0;
  if constexpr (rows_need_gu<ROWS>()) {
    static_for<9>([&](auto k_) {
      constexpr int k = decltype(k_)::value;
      if constexpr (g_nonzero(k)) gu = fma(c.g[o][k], u[k], gu);
    });
  }
  if constexpr (rows_need_s<ROWS>()) s = fma(c.lam_area, gu, -c.alpha * p);
  static_for<9>([&](auto a_) {
    constexpr int a = decltype(a_)::value;
    if constexpr (((ROWS >> a) & 1u) != 0) {
      T acc = yl[a];
      if constexpr (g_nonzero(a)) acc = fma(c.g[o][a], s, acc);
      static_for<9>([&](auto b_) {
        constexpr int b = decltype(b_)::value;
        if constexpr (DENSE || aeps_nonzero(a, b)) acc = fma(c.A[o][a * 9 + b], u[b], acc);
      });
      yl[a] = acc;
    }
  });
  static_for<3>([&](auto a_) {
    constexpr int a = decltype(a_)::value;
    if constexpr (((ROWS >> (9 + a)) & 1u) != 0) {
      T m = 0;
      if constexpr (WM == 0) {
        static_for<3>([&](auto b_) {
          constexpr int b = decltype(b_)::value;
          if constexpr (mw_nonzero(a, b)) m = fma(c.M1[o][a * 3 + b], w[b], m);
        });
        yl[9 + a] = fma(kinv, m, fma(-c.dw[o][a], p, yl[9 + a]));
      } else {
        // symmetric 3x3: (00, 01, 02, 11, 12, 22)
        constexpr int r0 = a == 0 ? 0 : a == 1 ? 1 : 2;
        constexpr int r1 = a == 0 ? 1 : a == 1 ? 3 : 4;
        constexpr int r2 = a == 0 ? 2 : a == 1 ? 4 : 5;
        m = fma(wmT[r0], w[0], fma(wmT[r1], w[1], fma(wmT[r2], w[2], fma(-c.dw[o][a], p, yl[9 + a]))));
        yl[9 + a] = m;
      }
    }
  });
  if constexpr (((ROWS >> 12) & 1u) != 0) {
    T r = fma(-c.pp, p, yl[12]);
    r = fma(-c.alpha, gu, r);
#pragma unroll
    for (int k = 0; k < 3; ++k) r = fma(-c.dw[o][k], w[k], r);
    yl[12] = r;
  }
}

// Where phase 1 reads the input vector and the coefficients: global memory, or a slab of
// them staged in shared memory by the tensor-memory-accelerator (TMA) loads of
// apply_tma_kernel.  xv(k, i, j): block k at position (i, j); kv(o, ci, cj): K^{-1} of
// triangle o of cell (ci, cj); wv(o, k, ci, cj): entry k of its 3 x 3 RT0 mass.
template <typename T>
struct GlobalSrc {
  const T *x, *kinv, *wm;
  size_t blk;
  int P;
  __device__ __forceinline__ T xv(int k, int i, int j) const { return x[k * blk + (size_t)j * P + i]; }
  __device__ __forceinline__ T kv(int o, int ci, int cj) const {
    return kinv[(size_t)o * blk + (size_t)cj * P + ci];
  }
  __device__ __forceinline__ T wv(int o, int k, int ci, int cj) const {
    return wm[(size_t)(6 * o + k) * blk + (size_t)cj * P + ci];
  }
};

template <int BX, int BY>
struct SmemSrc {                 // slab: x [10][BY][BX], coefficients [NC][BY - 1][BX]
  const float *xs, *cs;
  int x0, y0;                    // grid position of slab element (0, 0)
  __device__ __forceinline__ float xv(int k, int i, int j) const {
    return xs[(k * BY + (j - y0)) * BX + (i - x0)];
  }
  __device__ __forceinline__ float kv(int o, int ci, int cj) const {
    return cs[(o * (BY - 1) + (cj - y0)) * BX + (ci - x0)];
  }
  __device__ __forceinline__ float wv(int o, int k, int ci, int cj) const {
    return cs[((6 * o + k) * (BY - 1) + (cj - y0)) * BX + (ci - x0)];
  }
};

// Both triangles of cell (ci, cj), accumulated into the cell's kCellSlots shared-memory
// slots.  L: v0 = (ci,cj), v1 = (ci+1,cj), v2 = (ci,cj+1); e0 = d, e1 = v(ci,cj), e2 = h(ci,cj).
// U: v0 = (ci+1,cj+1), v1 = (ci,cj+1), v2 = (ci+1,cj); e0 = d, e1 = v(ci+1,cj), e2 = h(ci,cj+1).
// The two triangles share the vertices (ci+1,cj) and (ci,cj+1) and the diagonal edge: U's
// rows for those six DoFs continue L's sums, so each cell leaves 20 values:
//   0 ux(ci,cj)  1 uy(ci,cj)  2 bv(ci,cj)  3 bh(ci,cj)  4 wv(ci,cj)  5 wh(ci,cj)  6 pL
//   7 ux(ci+1,cj)  8 uy(ci+1,cj)  9 ux(ci,cj+1)  10 uy(ci,cj+1)  11 bd  12 wd
//   13 ux(ci+1,cj+1)  14 uy(ci+1,cj+1)  15 bv(ci+1,cj)  16 bh(ci,cj+1)  17 wv(ci+1,cj)
//   18 wh(ci,cj+1)  19 pU
// LROWS / UROWS select the rows of each triangle that are formed (halo cells need a few).
constexpr int kCellSlots = 20;

template <typename T, int WM, unsigned LROWS, unsigned UROWS, bool DENSE, typename Src>
__device__ __forceinline__ void cell_product(const OpCoefs<T> &c, const Src &src, int ci, int cj, int n,
                                             T *slot) {
  if (ci < 0 || cj < 0 || ci >= n || cj >= n) {
#pragma unroll
    for (int k = 0; k < kCellSlots; ++k) slot[k] = 0;
    return;
  }
  const bool f00 = vfree(ci, cj, n), f10 = vfree(ci + 1, cj, n), f01 = vfree(ci, cj + 1, n),
             f11 = vfree(ci + 1, cj + 1, n);
  const T ux00 = f00 ? src.xv(UX, ci, cj) : T(0), uy00 = f00 ? src.xv(UY, ci, cj) : T(0);
  const T ux10 = f10 ? src.xv(UX, ci + 1, cj) : T(0), uy10 = f10 ? src.xv(UY, ci + 1, cj) : T(0);
  const T ux01 = f01 ? src.xv(UX, ci, cj + 1) : T(0), uy01 = f01 ? src.xv(UY, ci, cj + 1) : T(0);
  const T ux11 = f11 ? src.xv(UX, ci + 1, cj + 1) : T(0), uy11 = f11 ? src.xv(UY, ci + 1, cj + 1) : T(0);
  const T bd = src.xv(BD, ci, cj);
  const T bvL = ci > 0 ? src.xv(BV, ci, cj) : T(0), bvU = ci + 1 < n ? src.xv(BV, ci + 1, cj) : T(0);
  const T bhL = cj > 0 ? src.xv(BH, ci, cj) : T(0), bhU = cj + 1 < n ? src.xv(BH, ci, cj + 1) : T(0);
  const T wd = src.xv(WD, ci, cj);
  const T wvL = src.xv(WV, ci, cj), wvU = src.xv(WV, ci + 1, cj);
  const T whL = src.xv(WH, ci, cj), whU = src.xv(WH, ci, cj + 1);
  T kin[2] = {0, 0};
  T wm[2][6];
  if (WM == 0) {
    kin[0] = src.kv(0, ci, cj);
    kin[1] = src.kv(1, ci, cj);
  } else {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      wm[0][k] = src.wv(0, k, ci, cj);
      wm[1][k] = src.wv(1, k, ci, cj);
    }
  }
  T yl[13];
#pragma unroll
  for (int k = 0; k < 13; ++k) yl[k] = 0;
  {
    const T u[9] = {ux00, ux10, ux01, uy00, uy10, uy01, bd, bvL, bhL};
    const T w[3] = {wd, wvL, whL};
    tri_product<T, WM, LROWS, DENSE>(c, 0, u, w, src.xv(PL, ci, cj), kin[0], wm[0], yl);
  }
  slot[0] = yl[0]; slot[1] = yl[3]; slot[2] = yl[7]; slot[3] = yl[8];
  slot[4] = yl[10]; slot[5] = yl[11]; slot[6] = yl[12];
  T yu[13];
#pragma unroll
  for (int k = 0; k < 13; ++k) yu[k] = 0;
  yu[2] = yl[1]; yu[5] = yl[4]; yu[1] = yl[2]; yu[4] = yl[5]; yu[6] = yl[6]; yu[9] = yl[9];
  {
    const T u[9] = {ux11, ux01, ux10, uy11, uy01, uy10, bd, bvU, bhU};
    const T w[3] = {wd, wvU, whU};
    tri_product<T, WM, UROWS, DENSE>(c, 1, u, w, src.xv(PU, ci, cj), kin[1], wm[1], yu);
  }
  slot[7] = yu[2]; slot[8] = yu[5]; slot[9] = yu[1]; slot[10] = yu[4]; slot[11] = yu[6];
  slot[12] = yu[9]; slot[13] = yu[0]; slot[14] = yu[3]; slot[15] = yu[7]; slot[16] = yu[8];
  slot[17] = yu[10]; slot[18] = yu[11]; slot[19] = yu[12];
}

__host__ __device__ constexpr unsigned rowbits(int a) { return 1u << a; }
// rows the tile's DoFs gather from its halo cells (see the gather in apply_tile):
// left column (ci = i0 - 1): slots 7, 8 (L rows 1, 4 + U rows 2, 5), 13, 14 (U 0, 3), 15 (U 7),
// 17 (U 10); bottom row (cj = j0 - 1): slots 9, 10 (L 2, 5 + U 1, 4), 13, 14, 16 (U 8),
// 18 (U 11); corner: slots 13, 14
constexpr unsigned kLeftL = rowbits(1) | rowbits(4);
constexpr unsigned kLeftU = rowbits(0) | rowbits(2) | rowbits(3) | rowbits(5) | rowbits(7) | rowbits(10);
constexpr unsigned kBottomL = rowbits(2) | rowbits(5);
constexpr unsigned kBottomU = rowbits(0) | rowbits(1) | rowbits(3) | rowbits(4) | rowbits(8) | rowbits(11);
constexpr unsigned kCornerU = rowbits(0) | rowbits(3);

__host__ __device__ constexpr int round32(int v) { return (v + 31) / 32 * 32; }

// Tile of kTX x kTY output positions per CTA (template: large tiles on large grids, small
// tiles on the coarse levels so that their work spreads over many SMs).  sy: shared scratch
// of kCellSlots values per cell of the tile and of its one-cell halo on the low side.
// PF: the residual form loads the thread's b values before the element products, so their
// latency overlaps phase 1 instead of following the barrier (always in FP32; an FP64 tuning
// candidate, since it holds 20 more registers through phase 1).
template <typename T, int WM, int kTX, int kTY, int NT, bool DENSE, typename Src, bool PF = (sizeof(T) == 4)>
__device__ __forceinline__ void apply_tile(const ApplyArgs<T> &a, const Src &src, T (*sy)[kCellSlots], int bx,
                                           int by, size_t boff) {
  constexpr int kEX = kTX + 1;
  constexpr int kOwn = kTX * kTY;
  static_assert(NT >= kOwn, "one thread per output position in phase 2");
  // halo tasks: bottom row (kTX cells), left column (kTY cells), corner; each kind starts on
  // a warp boundary where the CTA has the threads, after the own cells if they leave room
  constexpr int kH0 = round32(kOwn) + round32(kTX) + kTY + 1 <= NT ? round32(kOwn) : 0;
  constexpr int kHL = kH0 + round32(kTX) + kTY <= NT ? kH0 + round32(kTX) : kH0 + kTX;
  constexpr int kHC = kHL + round32(kTY) < NT ? kHL + round32(kTY) : kHL + kTY;
  static_assert(kHC < NT && kH0 + kTX <= kHL && kHL + kTY <= kHC, "halo task layout");
  const Grid g = a.g;
  const int n = g.n, P = g.pitch;
  const size_t blk = g.blk;
  T *y = a.y + boff;
  const int i0 = bx * kTX, j0 = by * kTY;
  const int tid = threadIdx.x;
  auto S = [&](int ci, int cj) -> T * { return sy[(cj - j0 + 1) * kEX + (ci - i0 + 1)]; };
  constexpr bool kPrefetchB = PF;
  T bpre[NBLK];
  if constexpr (kPrefetchB) {
    const int ip = i0 + tid % kTX, jp = j0 + tid / kTX;
    const bool ok = a.residual && tid < kOwn && jp <= n && ip <= n;
    const T *bb = a.b + boff;
    const size_t op = (size_t)jp * P + ip;
#pragma unroll
    for (int k = 0; k < NBLK; ++k) bpre[k] = ok ? bb[k * blk + op] : T(0);
  }

  // phase 1: one task per cell of the tile (both triangles), then the halo cells with only
  // the rows the tile gathers
  if (tid < kOwn) {
    const int ci = i0 + tid % kTX, cj = j0 + tid / kTX;
    cell_product<T, WM, kAllRows, kAllRows, DENSE>(a.c, src, ci, cj, n, S(ci, cj));
  }
  if (tid >= kH0 && tid < kH0 + kTX) {
    const int ci = i0 + (tid - kH0), cj = j0 - 1;
    cell_product<T, WM, kBottomL, kBottomU, DENSE>(a.c, src, ci, cj, n, S(ci, cj));
  } else if (tid >= kHL && tid < kHL + kTY) {
    const int ci = i0 - 1, cj = j0 + (tid - kHL);
    cell_product<T, WM, kLeftL, kLeftU, DENSE>(a.c, src, ci, cj, n, S(ci, cj));
  } else if (tid == kHC) {
    cell_product<T, WM, 0u, kCornerU, DENSE>(a.c, src, i0 - 1, j0 - 1, n, S(i0 - 1, j0 - 1));
  }
  __syncthreads();

  if (tid >= kOwn) return;
  const int i = i0 + tid % kTX, j = j0 + tid / kTX;
  if (j > n || i >= P) return;
  const size_t o = (size_t)j * P + i;
  if (i > n) {                                       // padding columns
#pragma unroll
    for (int k = 0; k < NBLK; ++k) y[k * blk + o] = 0;
    return;
  }
  const T *c00 = S(i, j), *c10 = S(i - 1, j), *c01 = S(i, j - 1), *c11 = S(i - 1, j - 1);
  T v[NBLK];
  v[UX] = c00[0] + c10[7] + c01[9] + c11[13];
  v[UY] = c00[1] + c10[8] + c01[10] + c11[14];
  v[BH] = c00[3] + c01[16];
  v[BV] = c00[2] + c10[15];
  v[BD] = c00[11];
  v[WH] = c00[5] + c01[18];
  v[WV] = c00[4] + c10[17];
  v[WD] = c00[12];
  v[PL] = c00[6];
  v[PU] = c00[19];
  bool m[NBLK];
  dof_masks(i, j, n, m);
  const T *b = a.residual ? a.b + boff : nullptr;
#pragma unroll
  for (int k = 0; k < NBLK; ++k) {
    T out = 0;
    if constexpr (kPrefetchB) {
      if (m[k]) out = a.residual ? bpre[k] - v[k] : v[k];
    } else {
      if (m[k]) out = a.residual ? b[k * blk + o] - v[k] : v[k];
    }
    y[k * blk + o] = out;
  }
}

template <typename T, int WM, int kTX, int kTY, int NT, bool DENSE, bool PF>
__device__ __forceinline__ void apply_global(const ApplyArgs<T> &a) {
  pdl_enter();
  BMG_GATE(a.gate);
  extern __shared__ unsigned char smem_raw[];
  const size_t boff = (size_t)blockIdx.z * a.bstride;
  const GlobalSrc<T> src{a.x + boff, a.kinv, a.wm, a.g.blk, a.g.pitch};
  apply_tile<T, WM, kTX, kTY, NT, DENSE, GlobalSrc<T>, PF>(a, src, reinterpret_cast<T(*)[kCellSlots]>(smem_raw),
                                                           blockIdx.x, blockIdx.y, boff);
}

// MINB > 1 caps the registers so that MINB CTAs fit on an SM (more warps to hide the loads
// and the barrier, at the price of a few spilled values): tuning candidates.  MINB = 1 keeps
// the plain bound (an explicit minimum of one CTA lets the compiler take more registers).
template <typename T, int WM, int kTX, int kTY, int NT, bool DENSE, bool PF>
__global__ void __launch_bounds__(NT) apply_kernel(const __grid_constant__ ApplyArgs<T> a) {
  apply_global<T, WM, kTX, kTY, NT, DENSE, PF>(a);
}

template <typename T, int WM, int kTX, int kTY, int NT, bool DENSE, int MINB, bool PF>
__global__ void __launch_bounds__(NT, MINB) apply_kernel_capped(const __grid_constant__ ApplyArgs<T> a) {
  apply_global<T, WM, kTX, kTY, NT, DENSE, PF>(a);
}

template <typename T, int WM, int kTX, int kTY, int NT, bool DENSE, int MINB, bool PF>
constexpr auto apply_kernel_ptr() {
  if constexpr (MINB > 1) return &apply_kernel_capped<T, WM, kTX, kTY, NT, DENSE, MINB, PF>;
  else return &apply_kernel<T, WM, kTX, kTY, NT, DENSE, PF>;
}

// Batched form: several instances of one grid size in one launch, blockIdx.z selecting the
// instance whose arguments (coefficients, vectors, gate) are read from a device array.  The
// FP64 pipe bounds this kernel, so the coefficients' loads from global memory (broadcast,
// L1-resident) cost little next to the constant-bank operands of the single form.
template <int kTX, int kTY, int NT>
__global__ void __launch_bounds__(NT) apply_batch_kernel(const ApplyArgs<double> *__restrict__ args) {
  const ApplyArgs<double> &a = args[blockIdx.z];
  BMG_GATE(a.gate);
  extern __shared__ unsigned char smem_raw[];
  double(*sy)[kCellSlots] = reinterpret_cast<double(*)[kCellSlots]>(smem_raw);
  const GlobalSrc<double> src{a.x, a.kinv, a.wm, a.g.blk, a.g.pitch};
  if (a.wm_full) apply_tile<double, 1, kTX, kTY, NT, false>(a, src, sy, blockIdx.x, blockIdx.y, 0);
  else apply_tile<double, 0, kTX, kTY, NT, false>(a, src, sy, blockIdx.x, blockIdx.y, 0);
}

// ---- FP32 operator with TMA-staged input --------------------------------------------------
// One CTA per 32 x 8 tile.  Thread 0 issues two bulk tensor copies into shared memory: the
// 10 blocks of x over the tile and its halo (rows j0-1 .. j0+8, columns i0-4 .. i0+35: the
// start column is rounded down so that it is 16-byte aligned; positions outside the grid
// arrive as zeros) and the coefficient planes of cells (i0-4 .., j0-1 .. j0+7).  An mbarrier
// counts the bytes; every thread waits on it (bounded: after the limit the CTA sets the
// level's error flag, waits once more for its copies and leaves).  Phases 1 and 2 are
// apply_tile's, reading the slab instead of global memory.
constexpr int kTmaTX = 32, kTmaTY = 8, kTmaNT = 256, kTmaBX = 40, kTmaBY = kTmaTY + 2;
constexpr long long kTmaWaitLimit = 1ll << 22;

struct TmaMaps {
  const void *xptr[2] = {nullptr, nullptr};
  CUtensorMap x[2];
  CUtensorMap coef;
  // iteration limit of the first wait on the copies (the environment variable
  // BMG_DEBUG_TMA_WAIT_LIMIT lowers it at setup, so that a test can make the wait run out;
  // the second wait, for the copies still in flight, keeps the full limit)
  long long wait_limit = kTmaWaitLimit;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long limit) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];"
      :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

template <int WM>
constexpr size_t tma_smem_bytes() {
  return 128 + sizeof(float) * (10 * kTmaBY * kTmaBX + (WM ? 12 : 2) * (kTmaBY - 1) * kTmaBX +
                                kCellSlots * (kTmaTX + 1) * (kTmaTY + 1));
}

template <int WM>
__global__ void __launch_bounds__(kTmaNT) apply_tma_kernel(const __grid_constant__ ApplyArgs<float> a,
                                                           const __grid_constant__ CUtensorMap tx,
                                                           const __grid_constant__ CUtensorMap tc,
                                                           int *err, long long wait_limit) {
  constexpr int NC = WM ? 12 : 2;
  constexpr uint32_t kBytes = sizeof(float) * (10 * kTmaBY * kTmaBX + NC * (kTmaBY - 1) * kTmaBX);
  pdl_enter();
  BMG_GATE(a.gate);
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  float *xs = reinterpret_cast<float *>(base);
  float *cs = xs + 10 * kTmaBY * kTmaBX;
  float(*sy)[kCellSlots] = reinterpret_cast<float(*)[kCellSlots]>(cs + NC * (kTmaBY - 1) * kTmaBX);
  __shared__ alignas(8) unsigned long long bar;
  const int x0 = blockIdx.x * kTmaTX - 4, y0 = blockIdx.y * kTmaTY - 1;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // the input was written by earlier kernels through ordinary stores: order those writes
    // before the bulk copies' reads (a different memory proxy)
    asm volatile("fence.proxy.async.global;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(b), "r"(kBytes) : "memory");
    tma_load_3d(smem_u32(xs), &tx, x0, y0, 0, b);
    tma_load_3d(smem_u32(cs), &tc, x0, y0, 0, b);
  }
  const bool ok = mbar_wait_bounded(b, 0, wait_limit);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicOr(err, kErrTmaTimeout);
    mbar_wait_bounded(b, 0, kTmaWaitLimit);          // let the copies in flight land
    return;
  }
  const SmemSrc<kTmaBX, kTmaBY> src{xs, cs, x0, y0};
  apply_tile<float, WM, kTmaTX, kTmaTY, kTmaNT, false>(a, src, sy, blockIdx.x, blockIdx.y, 0);
}

template <int WM>
static int launch_apply_tma(const ApplyArgs<float> &a, const Level &L, const CUtensorMap &tx,
                            cudaStream_t st) {
  static bool attr = false;
  const size_t smem = tma_smem_bytes<WM>();
  if (!attr) {
    BMG_CUDA(cudaFuncSetAttribute(apply_tma_kernel<WM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  dim3 grid((L.g.pitch + kTmaTX - 1) / kTmaTX, (L.n + 1 + kTmaTY - 1) / kTmaTY);
  BMG_CUDA(launch_pdl(apply_tma_kernel<WM>, grid, dim3(kTmaNT), smem, st, a, tx, L.tma->coef, L.err,
                      L.tma->wait_limit));
  return BMG_OK;
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 3-D FP32 map (pitch, rows, planes) with plane stride plane_elems, box (40, box_rows, planes)
static bool encode_planes(CUtensorMap *m, const void *base, int pitch, int rows, int planes,
                          size_t plane_elems, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || !base) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)rows, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {(cuuint64_t)pitch * sizeof(float), (cuuint64_t)plane_elems * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)kTmaBX, (cuuint32_t)box_rows, (cuuint32_t)planes};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int setup_apply_tma(Level &L, const float *xa, const float *xb) {
  free_apply_tma(L);
  const float *coef = L.wm_full ? L.wm32 : L.kinv32;
  if (!coef || L.n < kTmaTX) return BMG_OK;
  TmaMaps *t = new TmaMaps();
  if (const char *lim = std::getenv("BMG_DEBUG_TMA_WAIT_LIMIT")) {
    const long long v = std::atoll(lim);
    if (*lim && v >= 0 && v < kTmaWaitLimit) t->wait_limit = v;
  }
  bool ok = encode_planes(&t->coef, coef, L.g.pitch, L.n + 1, L.wm_full ? 12 : 2, L.g.blk, kTmaBY - 1);
  const float *xs[2] = {xa, xb};
  for (int k = 0; k < 2 && ok; ++k) {
    if (!xs[k]) continue;
    ok = encode_planes(&t->x[k], xs[k], L.g.pitch, L.n + 1, NBLK, L.g.blk, kTmaBY);
    t->xptr[k] = xs[k];
  }
  if (ok) L.tma = t;
  else delete t;
  return BMG_OK;
}

void free_apply_tma(Level &L) {
  delete L.tma;
  L.tma = nullptr;
}

template <typename T, int WM, int TX, int TY, int NT, bool DENSE, int MINB = 1, bool PF = (sizeof(T) == 4)>
static int launch_apply_tile(const ApplyArgs<T> &a, const Level &L, int batch, cudaStream_t st) {
  dim3 block(NT);
  dim3 grid((L.g.pitch + TX - 1) / TX, (L.n + 1 + TY - 1) / TY, batch);
  const size_t smem = sizeof(T) * kCellSlots * (TX + 1) * (TY + 1);
  if (smem > 48 * 1024) {
    static bool attr = false;
    if (!attr) {
      BMG_CUDA(cudaFuncSetAttribute(apply_kernel_ptr<T, WM, TX, TY, NT, DENSE, MINB, PF>(),
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      attr = true;
    }
  }
  BMG_CUDA(launch_pdl(apply_kernel_ptr<T, WM, TX, TY, NT, DENSE, MINB, PF>(), dim3(grid), dim3(block), smem, st, a));
  return BMG_OK;
}

// CTAs a tile shape would launch on this level.
static long long ctas_for(const Level &L, int tx, int ty, int batch) {
  return (long long)((L.g.pitch + tx - 1) / tx) * ((L.n + 1 + ty - 1) / ty) * batch;
}

template <typename T, int WM, bool D>
static int launch_apply_wm(const ApplyArgs<T> &a, const Level &L, int batch, cudaStream_t st) {
  switch (L.tile_apply) {            // tuned at setup (same candidates as the batched form)
    case 0: return launch_apply_tile<T, WM, 32, 8, 256, D>(a, L, batch, st);
    case 1: return launch_apply_tile<T, WM, 16, 8, 128, D>(a, L, batch, st);
    case 2: return launch_apply_tile<T, WM, 8, 8, 128, D>(a, L, batch, st);
    case 3: return launch_apply_tile<T, WM, 8, 4, 96, D>(a, L, batch, st);
    case 4: return launch_apply_tile<T, WM, 4, 4, 64, D>(a, L, batch, st);
    case 5:                         // FP32, input staged by TMA (else the same 32 x 8 tile)
      if constexpr (sizeof(T) == 4 && !D) {
        if (L.tma && L.err && batch == 1)
          for (int k = 0; k < 2; ++k)
            if (L.tma->xptr[k] == (const void *)a.x) return launch_apply_tma<WM>(a, L, L.tma->x[k], st);
      }
      return launch_apply_tile<T, WM, 32, 8, 256, D>(a, L, batch, st);
    case 6: return launch_apply_tile<T, WM, 32, 8, 256, D, 4>(a, L, batch, st);   // 4 CTAs / SM
    case 7: return launch_apply_tile<T, WM, 16, 8, 128, D, 8>(a, L, batch, st);   // 8 CTAs / SM
    case 8:                         // FP64 with b prefetched (FP32 prefetches in every tile)
      if constexpr (sizeof(T) == 8) return launch_apply_tile<T, WM, 32, 8, 256, D, 1, true>(a, L, batch, st);
      return launch_apply_tile<T, WM, 32, 8, 256, D>(a, L, batch, st);
    case 9:
      if constexpr (sizeof(T) == 8) return launch_apply_tile<T, WM, 16, 8, 128, D, 1, true>(a, L, batch, st);
      return launch_apply_tile<T, WM, 16, 8, 128, D>(a, L, batch, st);
    default: break;
  }
  // the largest tile that still gives every SM about two CTAs
  const long long want = 2 * 152;
  // small tiles get more threads than positions so that the triangle products (phase 1)
  // of a tile are spread over more warps
  if (ctas_for(L, 32, 8, batch) >= want) return launch_apply_tile<T, WM, 32, 8, 256, D>(a, L, batch, st);
  if (ctas_for(L, 16, 8, batch) >= want) return launch_apply_tile<T, WM, 16, 8, 128, D>(a, L, batch, st);
  if (ctas_for(L, 8, 8, batch) >= want) return launch_apply_tile<T, WM, 8, 8, 128, D>(a, L, batch, st);
  if (ctas_for(L, 8, 4, batch) >= want) return launch_apply_tile<T, WM, 8, 4, 96, D>(a, L, batch, st);
  return launch_apply_tile<T, WM, 4, 4, 64, D>(a, L, batch, st);
}

template <typename T>
int launch_apply(const Level &L, const T *x, const T *b, T *y, bool residual, int batch,
                 size_t bstride, cudaStream_t st) {
  ApplyArgs<T> a;
  a.g = L.g;
  a.x = x;
  a.b = b;
  a.y = y;
  a.bstride = bstride;
  a.residual = residual ? 1 : 0;
  a.gate = L.gate;
  const bool f64 = sizeof(T) == 8;
  a.kinv = (const T *)(f64 ? (const void *)L.kinv64 : (const void *)L.kinv32);
  a.wm = (const T *)(f64 ? (const void *)L.wm64 : (const void *)L.wm32);
  a.c = *reinterpret_cast<const OpCoefs<T> *>(f64 ? (const void *)&L.c64 : (const void *)&L.c32);
  BMG_PROF_BEGIN(BMG_PROF_APPLY, L.n, st);
  // Galerkin coarse levels: dense elasticity element matrices
  int rc = L.dense_a ? (L.wm_full ? launch_apply_wm<T, 1, true>(a, L, batch, st) : launch_apply_wm<T, 0, true>(a, L, batch, st))
                     : (L.wm_full ? launch_apply_wm<T, 1, false>(a, L, batch, st) : launch_apply_wm<T, 0, false>(a, L, batch, st));
  BMG_PROF_END(st, (double)L.n * L.n * batch);
  if (rc) return rc;
  BMG_CHECK_LAUNCH("apply_kernel");
  return BMG_OK;
}

template int launch_apply<double>(const Level &, const double *, const double *, double *, bool,
                                  int, size_t, cudaStream_t);
template int launch_apply<float>(const Level &, const float *, const float *, float *, bool, int,
                                 size_t, cudaStream_t);

// ---- batched application ---------------------------------------------------------------
size_t apply_args_bytes() { return sizeof(ApplyArgs<double>); }

void make_apply_args(const Level &L, const double *x, const double *b, double *y, bool residual,
                     const int *gate, void *dst) {
  ApplyArgs<double> a;
  a.g = L.g;
  a.x = x;
  a.b = b;
  a.y = y;
  a.bstride = 0;
  a.residual = residual ? 1 : 0;
  a.wm_full = L.wm_full ? 1 : 0;
  a.gate = gate;
  a.kinv = L.kinv64;
  a.wm = L.wm64;
  a.c = L.c64;
  std::memcpy(dst, &a, sizeof(a));
}

template <int TX, int TY, int NT>
static int launch_apply_batch_tile(const void *d_args, int count, int n, cudaStream_t st) {
  const Grid g = grid_of(n);
  dim3 grid((g.pitch + TX - 1) / TX, (n + 1 + TY - 1) / TY, count);
  const size_t smem = sizeof(double) * kCellSlots * (TX + 1) * (TY + 1);
  if (smem > 48 * 1024) {
    const int rc = prepare_apply_batch();
    if (rc) return rc;
  }
  apply_batch_kernel<TX, TY, NT><<<grid, NT, smem, st>>>((const ApplyArgs<double> *)d_args);
  BMG_CHECK_LAUNCH("apply_batch_kernel");
  return BMG_OK;
}

// Opt-in to the shared memory of the large tiles once, outside any stream capture.
int prepare_apply_batch() {
  static bool done = false;
  if (done) return BMG_OK;
  BMG_CUDA(cudaFuncSetAttribute(apply_batch_kernel<32, 8, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(double) * kCellSlots * 33 * 9)));
  done = true;
  return BMG_OK;
}

// tile t: 0 = 32 x 8, 1 = 16 x 8, 2 = 8 x 8, 3 = 8 x 4, 4 = 4 x 4 output positions
int launch_apply_batch(const void *d_args, int count, int n, int tile, cudaStream_t st) {
  if (count <= 0) return BMG_OK;
  switch (tile) {
    case 0: return launch_apply_batch_tile<32, 8, 256>(d_args, count, n, st);
    case 1: return launch_apply_batch_tile<16, 8, 128>(d_args, count, n, st);
    case 2: return launch_apply_batch_tile<8, 8, 128>(d_args, count, n, st);
    case 3: return launch_apply_batch_tile<8, 4, 96>(d_args, count, n, st);
    default: return launch_apply_batch_tile<4, 4, 64>(d_args, count, n, st);
  }
}

// the single-instance rule: the largest tile that gives every SM about two CTAs
int default_apply_tile(int n, int count) {
  static const int tx[kApplyTiles] = {32, 16, 8, 8, 4}, ty[kApplyTiles] = {8, 8, 8, 4, 4};
  const Grid g = grid_of(n);
  for (int t = 0; t + 1 < kApplyTiles; ++t) {
    const long long c = (long long)((g.pitch + tx[t] - 1) / tx[t]) * ((n + 1 + ty[t] - 1) / ty[t]) * count;
    if (c >= 2 * 152) return t;
  }
  return kApplyTiles - 1;
}

// --------------------------------------------------------------------------------------
// Galerkin coarsening of the RT0 mass (the coarse-level reading for a per-triangle K):
// Wm_T = sum over the 4 children c of Q_c^T Wm_c Q_c.
struct CoarsenArgs {
  Grid gf, gc;
  const double *kinv_f;   // fine per-triangle K^{-1} (fine_full == 0)
  const double *wm_f;     // fine 3x3 masses (fine_full == 1)
  int fine_full;
  double M1[2][9];        // tau * unit RT0 mass of the fine level
  double *wm_c64;
  float *wm_c32;
  int child_o[2][4], child_di[2][4], child_dj[2][4];
  double Q[2][4][3][3];
};

__global__ void coarsen_wmass_kernel(const __grid_constant__ CoarsenArgs a) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int nc = a.gc.n;
  if (I >= nc || J >= nc) return;
  for (int o = 0; o < 2; ++o) {
    double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int c = 0; c < 4; ++c) {
      const int co = a.child_o[o][c];
      const size_t fo = (size_t)(2 * J + a.child_dj[o][c]) * a.gf.pitch + (2 * I + a.child_di[o][c]);
      double Mc[3][3];
      if (a.fine_full) {
        const double *w = a.wm_f + (size_t)co * 6 * a.gf.blk + fo;
        const size_t s = a.gf.blk;
        Mc[0][0] = w[0]; Mc[0][1] = Mc[1][0] = w[s]; Mc[0][2] = Mc[2][0] = w[2 * s];
        Mc[1][1] = w[3 * s]; Mc[1][2] = Mc[2][1] = w[4 * s]; Mc[2][2] = w[5 * s];
      } else {
        const double k = a.kinv_f[(size_t)co * a.gf.blk + fo];
        for (int r = 0; r < 3; ++r)
          for (int s = 0; s < 3; ++s) Mc[r][s] = k * a.M1[co][r * 3 + s];
      }
      for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) {
          double acc = 0;
          for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) acc += a.Q[o][c][p][r] * Mc[p][q] * a.Q[o][c][q][s];
          M[r][s] += acc;
        }
    }
    const size_t co = (size_t)J * a.gc.pitch + I;
    const double vals[6] = {M[0][0], 0.5 * (M[0][1] + M[1][0]), 0.5 * (M[0][2] + M[2][0]),
                            M[1][1], 0.5 * (M[1][2] + M[2][1]), M[2][2]};
    for (int k = 0; k < 6; ++k) {
      a.wm_c64[(size_t)(o * 6 + k) * a.gc.blk + co] = vals[k];
      a.wm_c32[(size_t)(o * 6 + k) * a.gc.blk + co] = (float)vals[k];
    }
  }
}

extern TransferTables g_tables_host;

int launch_coarsen_wmass(const Level &fine, Level &coarse, cudaStream_t st) {
  CoarsenArgs a;
  a.gf = fine.g;
  a.gc = coarse.g;
  a.kinv_f = fine.kinv64;
  a.wm_f = fine.wm64;
  a.fine_full = fine.wm_full ? 1 : 0;
  for (int o = 0; o < 2; ++o)
    for (int k = 0; k < 9; ++k) a.M1[o][k] = fine.c64.M1[o][k];
  a.wm_c64 = coarse.wm64;
  a.wm_c32 = coarse.wm32;
  const TransferTables &t = g_tables_host;
  for (int o = 0; o < 2; ++o)
    for (int c = 0; c < 4; ++c) {
      a.child_o[o][c] = t.child_o[o][c];
      a.child_di[o][c] = t.child_di[o][c];
      a.child_dj[o][c] = t.child_dj[o][c];
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) a.Q[o][c][p][q] = t.Q[o][c][p][q];
    }
  dim3 block(16, 16);
  dim3 grid((coarse.n + 15) / 16, (coarse.n + 15) / 16);
  coarsen_wmass_kernel<<<grid, block, 0, st>>>(a);
  BMG_CHECK_LAUNCH("coarsen_wmass_kernel");
  return BMG_OK;
}

}  // namespace bmg
