// Matrix-free application of the reduced-quadrature Biot operator (Sec. 2.3,
// Eq. block_form_rq) on the structured triangulation: y = A x or r = b - A x.
//
// Element-gather design: a CTA owns a 32 x 8 tile of output positions.  Phase 1 computes
// the 13-entry local products of both triangles of every cell of the tile plus a one-cell
// halo on the low side (the triangles that touch the tile's DoFs) into shared memory;
// phase 2 gathers, for every DoF of the tile, the contributions of its triangles (6 for a
// vertex, 2 for an edge, 1 for a triangle).  No atomics: the result is deterministic.
// Constrained displacement slots are ignored on input and written as 0.
#include <cuda.h>
#include <cudaTypedefs.h>

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


// Local product of one triangle: yl[13] = E_T xl, xl = (u[9], w[3], p).  Products with the
// structural zeros of the element matrices are not formed (Aeps 30 of 81, g 2 of 9, the
// unit RT0 mass 4 of 9; see kElemNonzeros).
template <typename T, int WM>
__device__ __forceinline__ void tri_product(const OpCoefs<T> &c, int o, const T u[9],
                                            const T w[3], T p, T kinv, const T *wmT,
                                            T *yl) {
  T gu = 0;
  static_for<9>([&](auto k_) {
    constexpr int k = decltype(k_)::value;
    if constexpr (g_nonzero(k)) gu = fma(c.g[o][k], u[k], gu);
  });
  const T s = c.lam_area * gu - c.alpha * p;
  static_for<9>([&](auto a_) {
    constexpr int a = decltype(a_)::value;
    T acc = 0;
    if constexpr (g_nonzero(a)) acc = c.g[o][a] * s;
    static_for<9>([&](auto b_) {
      constexpr int b = decltype(b_)::value;
      if constexpr (aeps_nonzero(a, b)) acc = fma(c.A[o][a * 9 + b], u[b], acc);
    });
    yl[a] = acc;
  });
  T dww = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) dww = fma(c.dw[o][k], w[k], dww);
  if (WM == 0) {
    static_for<3>([&](auto a_) {
      constexpr int a = decltype(a_)::value;
      T acc = 0;
      static_for<3>([&](auto b_) {
        constexpr int b = decltype(b_)::value;
        if constexpr (mw_nonzero(a, b)) acc = fma(c.M1[o][a * 3 + b], w[b], acc);
      });
      yl[9 + a] = kinv * acc - c.dw[o][a] * p;
    });
  } else {
    // symmetric 3x3: (00, 01, 02, 11, 12, 22)
    yl[9] = wmT[0] * w[0] + wmT[1] * w[1] + wmT[2] * w[2] - c.dw[o][0] * p;
    yl[10] = wmT[1] * w[0] + wmT[3] * w[1] + wmT[4] * w[2] - c.dw[o][1] * p;
    yl[11] = wmT[2] * w[0] + wmT[4] * w[1] + wmT[5] * w[2] - c.dw[o][2] * p;
  }
  yl[12] = -c.alpha * gu - dww - c.pp * p;
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

// Tile of kTX x kTY output positions per CTA (template: large tiles on large grids, small
// tiles on the coarse levels so that their work spreads over many SMs).  sy: shared scratch
// of 26 values per cell of the tile and its halo.
template <typename T, int WM, int kTX, int kTY, int NT, typename Src>
__device__ __forceinline__ void apply_tile(const ApplyArgs<T> &a, const Src &src, T (*sy)[26], int bx,
                                           int by, size_t boff) {
  constexpr int kEX = kTX + 1, kEY = kTY + 1;
  static_assert(NT >= kTX * kTY, "one thread per output position in phase 2");
  const Grid g = a.g;
  const int n = g.n, P = g.pitch;
  const size_t blk = g.blk;
  T *y = a.y + boff;
  const int i0 = bx * kTX, j0 = by * kTY;
  const int tid = threadIdx.x;

  // phase 1: one task per triangle of the tile plus its low-side halo; all lower-left
  // triangles come first so that a warp works on one orientation (no divergence between
  // the two inlined element products)
  constexpr int NE = kEX * kEY;
  for (int e = tid; e < 2 * NE; e += NT) {
    const int o = e >= NE ? 1 : 0, cell = e - o * NE;
    const int ci = i0 - 1 + cell % kEX, cj = j0 - 1 + cell / kEX;
    T *yl = sy[cell] + 13 * o;
    if (ci < 0 || cj < 0 || ci >= n || cj >= n) {
#pragma unroll
      for (int k = 0; k < 13; ++k) yl[k] = 0;
      continue;
    }
    // L: v0 = (ci,cj), v1 = (ci+1,cj), v2 = (ci,cj+1); e0 = d, e1 = v(ci,cj), e2 = h(ci,cj)
    // U: v0 = (ci+1,cj+1), v1 = (ci,cj+1), v2 = (ci+1,cj); e0 = d, e1 = v(ci+1,cj), e2 = h(ci,cj+1)
    const int v0i = ci + o, v0j = cj + o;
    const int v1i = o ? ci : ci + 1, v1j = o ? cj + 1 : cj;
    const int v2i = o ? ci + 1 : ci, v2j = o ? cj : cj + 1;
    const bool f0 = vfree(v0i, v0j, n), f1 = vfree(v1i, v1j, n), f2 = vfree(v2i, v2j, n);
    const int evi = ci + o;                          // v(ci + o, cj)
    const int ehj = cj + o;                          // h(ci, cj + o)
    const bool bvf = o ? (ci + 1 < n) : (ci > 0);
    const bool bhf = o ? (cj + 1 < n) : (cj > 0);
    const T u[9] = {f0 ? src.xv(UX, v0i, v0j) : T(0), f1 ? src.xv(UX, v1i, v1j) : T(0), f2 ? src.xv(UX, v2i, v2j) : T(0),
                    f0 ? src.xv(UY, v0i, v0j) : T(0), f1 ? src.xv(UY, v1i, v1j) : T(0), f2 ? src.xv(UY, v2i, v2j) : T(0),
                    src.xv(BD, ci, cj), bvf ? src.xv(BV, evi, cj) : T(0), bhf ? src.xv(BH, ci, ehj) : T(0)};
    const T w[3] = {src.xv(WD, ci, cj), src.xv(WV, evi, cj), src.xv(WH, ci, ehj)};
    const T p = src.xv(o ? PU : PL, ci, cj);
    T kin = 0;
    T wm[6];
    if (WM == 0) {
      kin = src.kv(o, ci, cj);
    } else {
#pragma unroll
      for (int k = 0; k < 6; ++k) wm[k] = src.wv(o, k, ci, cj);
    }
    // FP32: orientation as a compile-time constant, so the element coefficients become
    // immediate constant-bank operands (the FP32 pipe would otherwise wait on indexed
    // constant loads).  FP64: one shared body with the orientation as an index (fewer
    // registers, more warps; the FP64 pipe is the limit either way).
    if constexpr (sizeof(T) == 4) {
      if (o == 0) tri_product<T, WM>(a.c, 0, u, w, p, kin, wm, yl);
      else tri_product<T, WM>(a.c, 1, u, w, p, kin, wm, yl);
    } else {
      tri_product<T, WM>(a.c, o, u, w, p, kin, wm, yl);
    }
  }
  __syncthreads();

  if (tid >= kTX * kTY) return;
  const int i = i0 + tid % kTX, j = j0 + tid / kTX;
  if (j > n || i >= P) return;
  const size_t o = (size_t)j * P + i;
  if (i > n) {                                       // padding columns
#pragma unroll
    for (int k = 0; k < NBLK; ++k) y[k * blk + o] = 0;
    return;
  }
  auto Y = [&](int ci, int cj, int k) -> T {
    return sy[(cj - j0 + 1) * kEX + (ci - i0 + 1)][k];
  };
  T v[NBLK];
  v[UX] = Y(i, j, 0) + Y(i - 1, j, 1) + Y(i, j - 1, 2) + Y(i - 1, j - 1, 13) +
          Y(i, j - 1, 14) + Y(i - 1, j, 15);
  v[UY] = Y(i, j, 3) + Y(i - 1, j, 4) + Y(i, j - 1, 5) + Y(i - 1, j - 1, 16) +
          Y(i, j - 1, 17) + Y(i - 1, j, 18);
  v[BH] = Y(i, j, 8) + Y(i, j - 1, 21);
  v[BV] = Y(i, j, 7) + Y(i - 1, j, 20);
  v[BD] = Y(i, j, 6) + Y(i, j, 19);
  v[WH] = Y(i, j, 11) + Y(i, j - 1, 24);
  v[WV] = Y(i, j, 10) + Y(i - 1, j, 23);
  v[WD] = Y(i, j, 9) + Y(i, j, 22);
  v[PL] = Y(i, j, 12);
  v[PU] = Y(i, j, 25);
  bool m[NBLK];
  dof_masks(i, j, n, m);
  const T *b = a.residual ? a.b + boff : nullptr;
#pragma unroll
  for (int k = 0; k < NBLK; ++k) {
    T out = 0;
    if (m[k]) out = a.residual ? b[k * blk + o] - v[k] : v[k];
    y[k * blk + o] = out;
  }
}

template <typename T, int WM, int kTX, int kTY, int NT>
__global__ void __launch_bounds__(NT) apply_kernel(const __grid_constant__ ApplyArgs<T> a) {
  pdl_enter();
  BMG_GATE(a.gate);
  extern __shared__ unsigned char smem_raw[];
  const size_t boff = (size_t)blockIdx.z * a.bstride;
  const GlobalSrc<T> src{a.x + boff, a.kinv, a.wm, a.g.blk, a.g.pitch};
  apply_tile<T, WM, kTX, kTY, NT>(a, src, reinterpret_cast<T(*)[26]>(smem_raw), blockIdx.x, blockIdx.y, boff);
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
  double(*sy)[26] = reinterpret_cast<double(*)[26]>(smem_raw);
  const GlobalSrc<double> src{a.x, a.kinv, a.wm, a.g.blk, a.g.pitch};
  if (a.wm_full) apply_tile<double, 1, kTX, kTY, NT>(a, src, sy, blockIdx.x, blockIdx.y, 0);
  else apply_tile<double, 0, kTX, kTY, NT>(a, src, sy, blockIdx.x, blockIdx.y, 0);
}

// ---- FP32 operator with TMA-staged input --------------------------------------------------
// One CTA per 32 x 8 tile.  Thread 0 issues two bulk tensor copies into shared memory: the
// 10 blocks of x over the tile and its halo (rows j0-1 .. j0+8, columns i0-4 .. i0+35: the
// start column is rounded down so that it is 16-byte aligned; positions outside the grid
// arrive as zeros) and the coefficient planes of cells (i0-4 .., j0-1 .. j0+7).  An mbarrier
// counts the bytes; every thread waits on it (bounded: after the limit the CTA sets the
// level's error flag, waits once more for its copies and leaves).  Phases 1 and 2 are
// apply_tile's, reading the slab instead of global memory.
struct TmaMaps {
  const void *xptr[2] = {nullptr, nullptr};
  CUtensorMap x[2];
  CUtensorMap coef;
};

constexpr int kTmaTX = 32, kTmaTY = 8, kTmaNT = 256, kTmaBX = 40, kTmaBY = kTmaTY + 2;
constexpr long long kTmaWaitLimit = 1ll << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kTmaWaitLimit; ++it) {
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
                                26 * (kTmaTX + 1) * (kTmaTY + 1));
}

template <int WM>
__global__ void __launch_bounds__(kTmaNT) apply_tma_kernel(const __grid_constant__ ApplyArgs<float> a,
                                                           const __grid_constant__ CUtensorMap tx,
                                                           const __grid_constant__ CUtensorMap tc,
                                                           int *err) {
  constexpr int NC = WM ? 12 : 2;
  constexpr uint32_t kBytes = sizeof(float) * (10 * kTmaBY * kTmaBX + NC * (kTmaBY - 1) * kTmaBX);
  pdl_enter();
  BMG_GATE(a.gate);
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  float *xs = reinterpret_cast<float *>(base);
  float *cs = xs + 10 * kTmaBY * kTmaBX;
  float(*sy)[26] = reinterpret_cast<float(*)[26]>(cs + NC * (kTmaBY - 1) * kTmaBX);
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
  const bool ok = mbar_wait_bounded(b, 0);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicOr(err, kErrTmaTimeout);
    mbar_wait_bounded(b, 0);
    return;
  }
  const SmemSrc<kTmaBX, kTmaBY> src{xs, cs, x0, y0};
  apply_tile<float, WM, kTmaTX, kTmaTY, kTmaNT>(a, src, sy, blockIdx.x, blockIdx.y, 0);
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
  BMG_CUDA(launch_pdl(apply_tma_kernel<WM>, grid, dim3(kTmaNT), smem, st, a, tx, L.tma->coef, L.err));
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

template <typename T, int WM, int TX, int TY, int NT>
static int launch_apply_tile(const ApplyArgs<T> &a, const Level &L, int batch, cudaStream_t st) {
  dim3 block(NT);
  dim3 grid((L.g.pitch + TX - 1) / TX, (L.n + 1 + TY - 1) / TY, batch);
  const size_t smem = sizeof(T) * 26 * (TX + 1) * (TY + 1);
  if (smem > 48 * 1024) {
    static bool attr = false;
    if (!attr) {
      BMG_CUDA(cudaFuncSetAttribute(apply_kernel<T, WM, TX, TY, NT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      attr = true;
    }
  }
  BMG_CUDA(launch_pdl(apply_kernel<T, WM, TX, TY, NT>, dim3(grid), dim3(block), smem, st, a));
  return BMG_OK;
}

// CTAs a tile shape would launch on this level.
static long long ctas_for(const Level &L, int tx, int ty, int batch) {
  return (long long)((L.g.pitch + tx - 1) / tx) * ((L.n + 1 + ty - 1) / ty) * batch;
}

template <typename T, int WM>
static int launch_apply_wm(const ApplyArgs<T> &a, const Level &L, int batch, cudaStream_t st) {
  switch (L.tile_apply) {            // tuned at setup (same candidates as the batched form)
    case 0: return launch_apply_tile<T, WM, 32, 8, 256>(a, L, batch, st);
    case 1: return launch_apply_tile<T, WM, 16, 8, 128>(a, L, batch, st);
    case 2: return launch_apply_tile<T, WM, 8, 8, 128>(a, L, batch, st);
    case 3: return launch_apply_tile<T, WM, 8, 4, 96>(a, L, batch, st);
    case 4: return launch_apply_tile<T, WM, 4, 4, 64>(a, L, batch, st);
    case 5:                         // FP32, input staged by TMA (else the same 32 x 8 tile)
      if constexpr (sizeof(T) == 4) {
        if (L.tma && L.err && batch == 1)
          for (int k = 0; k < 2; ++k)
            if (L.tma->xptr[k] == (const void *)a.x) return launch_apply_tma<WM>(a, L, L.tma->x[k], st);
      }
      return launch_apply_tile<T, WM, 32, 8, 256>(a, L, batch, st);
    default: break;
  }
  // the largest tile that still gives every SM about two CTAs
  const long long want = 2 * 152;
  // small tiles get more threads than positions so that the triangle products (phase 1)
  // of a tile are spread over more warps
  if (ctas_for(L, 32, 8, batch) >= want) return launch_apply_tile<T, WM, 32, 8, 256>(a, L, batch, st);
  if (ctas_for(L, 16, 8, batch) >= want) return launch_apply_tile<T, WM, 16, 8, 128>(a, L, batch, st);
  if (ctas_for(L, 8, 8, batch) >= want) return launch_apply_tile<T, WM, 8, 8, 128>(a, L, batch, st);
  if (ctas_for(L, 8, 4, batch) >= want) return launch_apply_tile<T, WM, 8, 4, 96>(a, L, batch, st);
  return launch_apply_tile<T, WM, 4, 4, 64>(a, L, batch, st);
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
  int rc = L.wm_full ? launch_apply_wm<T, 1>(a, L, batch, st) : launch_apply_wm<T, 0>(a, L, batch, st);
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
  const size_t smem = sizeof(double) * 26 * (TX + 1) * (TY + 1);
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
                                (int)(sizeof(double) * 26 * 33 * 9)));
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
