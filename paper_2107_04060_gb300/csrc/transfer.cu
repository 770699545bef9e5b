// Grid transfers (Sec. 3, Eq. block_interp; Sec. 3.1): prolongation-and-correct
// x_f += P x_c and restriction r_c = P^T r_f, as constant stencils per DoF type (and per
// parity class of the fine position for P).  The tables are built once on the host from
// the definitions of P_u (divergence-preserving), P_w (canonical RT0) and P_p (injection);
// see element.cpp.  Couplings to positions outside the grid are skipped and slots beyond
// the valid ranges hold zeros, so the interior stencil is exact up to the boundary.
#include <type_traits>

#include "bmg_internal.h"
#include "kernels_common.cuh"

namespace bmg {

TransferTables g_tables_host;
// |di|, |dj| bounds of the restriction and prolongation stencil tables: the tiled kernels
// stage slabs of that reach (checked when the tables are built)
constexpr int kResReach = 2, kProReach = 1;
__constant__ StencilEntry c_pro[NBLK][4][kMaxPro];
__constant__ int c_npro[NBLK][4];
__constant__ StencilEntry c_res[NBLK][kMaxRes];
__constant__ int c_nres[NBLK];

int upload_transfer_tables() {
  static bool done = false;
  if (done) return BMG_OK;
  build_transfer_tables(&g_tables_host);
  // the tiled transfer kernels stage slabs that reach kResReach / kProReach positions
  for (int t = 0; t < NBLK; ++t) {
    for (int e = 0; e < g_tables_host.nres[t]; ++e) {
      const StencilEntry &se = g_tables_host.res[t][e];
      if (se.di < -kResReach || se.di > kResReach || se.dj < -kResReach || se.dj > kResReach) {
        set_error("transfer tables: restriction stencil wider than the staged slab");
        return BMG_ERR_ARG;
      }
    }
    for (int p = 0; p < 4; ++p)
      for (int e = 0; e < g_tables_host.npro[t][p]; ++e) {
        const StencilEntry &se = g_tables_host.pro[t][p][e];
        if (se.di < -kProReach || se.di > kProReach || se.dj < -kProReach || se.dj > kProReach) {
          set_error("transfer tables: prolongation stencil wider than the staged slab");
          return BMG_ERR_ARG;
        }
      }
  }
  BMG_CUDA(cudaMemcpyToSymbol(c_pro, g_tables_host.pro, sizeof(g_tables_host.pro)));
  BMG_CUDA(cudaMemcpyToSymbol(c_npro, g_tables_host.npro, sizeof(g_tables_host.npro)));
  BMG_CUDA(cudaMemcpyToSymbol(c_res, g_tables_host.res, sizeof(g_tables_host.res)));
  BMG_CUDA(cudaMemcpyToSymbol(c_nres, g_tables_host.nres, sizeof(g_tables_host.nres)));
  done = true;
  return BMG_OK;
}

// One thread per (coarse position, DoF type): blockIdx.z is the type.
template <typename T>
__global__ void restrict_kernel(Grid gf, Grid gc, const T *__restrict__ rf, T *__restrict__ rc,
                                const int *gate) {
  pdl_enter();
  BMG_GATE(gate);
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int ct = blockIdx.z;
  const int nc = gc.n, nf = gf.n;
  if (I >= gc.pitch || J > nc) return;
  const size_t o = (size_t)J * gc.pitch + I;
  T acc = 0;
  if (I <= nc) {
    bool m[NBLK];
    dof_masks(I, J, nc, m);
    if (m[ct]) {
      const int ne = c_nres[ct];
      for (int e = 0; e < ne; ++e) {
        const StencilEntry se = c_res[ct][e];
        const int fi = 2 * I + se.di, fj = 2 * J + se.dj;
        if (fi < 0 || fj < 0 || fi > nf || fj > nf) continue;
        acc += (T)se.coef * __ldg(rf + se.type * gf.blk + (size_t)fj * gf.pitch + fi);
      }
    }
  }
  rc[ct * gc.blk + o] = acc;
}

// One thread per (fine position, DoF type): blockIdx.z is the type.  threadIdx.y is the parity
// class (i & 1) + 2 (j & 1) of the position, so every warp reads one stencil table and runs one
// loop length (block 32 x 4 covers 64 fine columns of two fine rows).
template <typename T>
__global__ void prolong_kernel(Grid gf, Grid gc, const T *__restrict__ xc, T *__restrict__ xf,
                               const int *gate) {
  pdl_enter();
  BMG_GATE(gate);
  const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + (threadIdx.y & 1);
  const int j = 2 * blockIdx.y + (threadIdx.y >> 1);
  const int t = blockIdx.z;
  const int nf = gf.n, nc = gc.n;
  if (i > nf || j > nf) return;
  bool m[NBLK];
  dof_masks(i, j, nf, m);
  if (!m[t]) return;
  const int par = (i & 1) + 2 * (j & 1);
  const int I0 = i >> 1, J0 = j >> 1;
  const size_t o = (size_t)j * gf.pitch + i;
  T acc = 0;
  const int ne = c_npro[t][par];
  for (int e = 0; e < ne; ++e) {
    const StencilEntry se = c_pro[t][par][e];
    const int I = I0 + se.di, J = J0 + se.dj;
    if (I < 0 || J < 0 || I > nc || J > nc) continue;
    acc += (T)se.coef * __ldg(xc + se.type * gc.blk + (size_t)J * gc.pitch + I);
  }
  xf[t * gf.blk + o] += acc;
}

// ---- tiled transfers ----------------------------------------------------------------
// Restriction: a CTA of TX x TY threads forms the 10 outputs of TX x TY coarse positions.
// Every coupling of coarse position (I, J) reads a fine position (2I + di, 2J + dj) with
// di, dj in [-kResReach, kResReach], so the CTA first stages the fine slab of all 10 blocks,
// columns 2 I0 - 2 .. 2 (I0 + TX) + 1 and rows 2 J0 - 2 .. 2 (J0 + TY), in shared memory with
// coalesced two-element loads (the first column is even, every row starts 8- or 16-byte
// aligned); positions outside the fine grid read as zero, which is what skipping them means.
// Each value is then loaded from global memory once instead of once per coupling.
// slab of a restriction tile: columns 2 I0 - kResReach .. 2 (I0 + TX - 1) + kResReach (one
// spare column keeps the width even), rows 2 J0 - kResReach .. 2 (J0 + TY - 1) + kResReach
template <int TX>
__host__ __device__ constexpr int restrict_slab_w() { return 2 * TX + 2 * kResReach; }
template <int TY>
__host__ __device__ constexpr int restrict_slab_h() { return 2 * TY + 2 * kResReach - 1; }

template <typename T, int TX, int TY>
constexpr size_t restrict_smem_bytes() {
  return sizeof(T) * (size_t)NBLK * restrict_slab_h<TY>() * restrict_slab_w<TX>();
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) restrict_tiled_kernel(Grid gf, Grid gc, const T *__restrict__ rf,
                                                                T *__restrict__ rc, const int *gate) {
  pdl_enter();
  BMG_GATE(gate);
  constexpr int SW = restrict_slab_w<TX>(), SH = restrict_slab_h<TY>();   // SW even: pairs
  extern __shared__ __align__(16) unsigned char tr_smem[];
  T *slab = reinterpret_cast<T *>(tr_smem);             // [NBLK][SH][SW]
  const int I0 = blockIdx.x * TX, J0 = blockIdx.y * TY;
  const int fi0 = 2 * I0 - kResReach, fj0 = 2 * J0 - kResReach;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int nf = gf.n;
  using T2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
  for (int q = tid; q < NBLK * SH * (SW / 2); q += TX * TY) {
    const int k = q / (SH * (SW / 2)), rem = q % (SH * (SW / 2));
    const int r = rem / (SW / 2), c2 = rem % (SW / 2);
    const int fi = fi0 + 2 * c2, fj = fj0 + r;           // fi is even
    T2 v;
    v.x = T(0);
    v.y = T(0);
    if (fj >= 0 && fj <= nf && fi >= 0 && fi + 1 < gf.pitch) {
      v = *reinterpret_cast<const T2 *>(rf + (size_t)k * gf.blk + (size_t)fj * gf.pitch + fi);
      if (fi > nf) v.x = T(0);
      if (fi + 1 > nf) v.y = T(0);
    }
    T *d = slab + ((size_t)k * SH + r) * SW + 2 * c2;
    d[0] = v.x;
    d[1] = v.y;
  }
  __syncthreads();
  const int I = I0 + threadIdx.x, J = J0 + threadIdx.y;
  const int nc = gc.n;
  if (I >= gc.pitch || J > nc) return;
  const size_t o = (size_t)J * gc.pitch + I;
  bool m[NBLK];
  dof_masks(I, J, nc, m);
  const int li = 2 * threadIdx.x + kResReach, lj = 2 * threadIdx.y + kResReach;   // (2I, 2J)
#pragma unroll 1
  for (int ct = 0; ct < NBLK; ++ct) {
    T acc = 0;
    if (I <= nc && m[ct]) {
      const int ne = c_nres[ct];
      for (int e = 0; e < ne; ++e) {
        const StencilEntry se = c_res[ct][e];
        acc += (T)se.coef * slab[((size_t)se.type * SH + lj + se.dj) * SW + li + se.di];
      }
    }
    rc[ct * gc.blk + o] = acc;
  }
}

// Prolongation and correction: a CTA of TX x TY threads updates the fine positions of the
// TX x TY/2 coarse cells (I0 .., J0 ..): thread (x, y) takes the even/odd pair of columns
// 2 (I0 + x), 2 (I0 + x) + 1 of fine row 2 J0 + y.  Its couplings read coarse positions
// (i/2 + di, j/2 + dj) with di, dj in [-kProReach, kProReach], staged beforehand as the coarse
// slab of columns I0 - 1 .. I0 + TX + 1 and rows J0 - 1 .. J0 + TY/2 + 1; the pair is read
// and written with one two-element access.
template <typename T, int TX, int TY>
constexpr size_t prolong_smem_bytes() {
  return sizeof(T) * (size_t)NBLK * (TY / 2 + 2 * kProReach + 1) * (TX + 2 * kProReach + 1);
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) prolong_tiled_kernel(Grid gf, Grid gc, const T *__restrict__ xc,
                                                               T *__restrict__ xf, const int *gate) {
  pdl_enter();
  BMG_GATE(gate);
  constexpr int CW = TX + 2 * kProReach + 1, CH = TY / 2 + 2 * kProReach + 1;   // from (I0 - 1, J0 - 1)
  extern __shared__ __align__(16) unsigned char tr_smem[];
  T *slab = reinterpret_cast<T *>(tr_smem);             // [NBLK][CH][CW]
  const int I0 = blockIdx.x * TX, J0 = blockIdx.y * (TY / 2);
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int nc = gc.n, nf = gf.n;
  for (int q = tid; q < NBLK * CH * CW; q += TX * TY) {
    const int k = q / (CH * CW), rem = q % (CH * CW);
    const int r = rem / CW, c = rem % CW;
    const int I = I0 - kProReach + c, J = J0 - kProReach + r;
    T v = T(0);
    if (I >= 0 && I <= nc && J >= 0 && J <= nc) v = xc[(size_t)k * gc.blk + (size_t)J * gc.pitch + I];
    slab[((size_t)k * CH + r) * CW + c] = v;
  }
  __syncthreads();
  const int i = 2 * (I0 + threadIdx.x), j = 2 * J0 + threadIdx.y;   // fine row j, columns i, i + 1
  if (j > nf || i > nf) return;
  const int ci = threadIdx.x + kProReach, cj = (j >> 1) - J0 + kProReach;   // (i/2, j/2) in the slab
  const size_t o = (size_t)j * gf.pitch + i;
  using T2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
  bool m0[NBLK], m1[NBLK];
  dof_masks(i, j, nf, m0);
  dof_masks(i + 1, j, nf, m1);
  const bool second = i + 1 <= nf;
#pragma unroll 1
  for (int t = 0; t < NBLK; ++t) {
    T a0 = 0, a1 = 0;
    const int p0 = 2 * (j & 1), p1 = 1 + 2 * (j & 1);
    if (m0[t]) {
      const int ne = c_npro[t][p0];
      for (int e = 0; e < ne; ++e) {
        const StencilEntry se = c_pro[t][p0][e];
        a0 += (T)se.coef * slab[((size_t)se.type * CH + cj + se.dj) * CW + ci + se.di];
      }
    }
    if (second && m1[t]) {
      const int ne = c_npro[t][p1];
      for (int e = 0; e < ne; ++e) {
        const StencilEntry se = c_pro[t][p1][e];
        a1 += (T)se.coef * slab[((size_t)se.type * CH + cj + se.dj) * CW + ci + se.di];
      }
    }
    T2 *px = reinterpret_cast<T2 *>(xf + (size_t)t * gf.blk + o);
    T2 v = *px;
    v.x += a0;
    v.y += a1;
    *px = v;
  }
}

template <typename T, int TX, int TY>
static cudaError_t opt_in_transfer_smem() {
  static cudaError_t e = [] {
    cudaError_t r = cudaSuccess;
    constexpr size_t rs = restrict_smem_bytes<T, TX, TY>(), ps = prolong_smem_bytes<T, TX, TY>();
    if (rs > 48 * 1024)
      r = cudaFuncSetAttribute(restrict_tiled_kernel<T, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs);
    if (r == cudaSuccess && ps > 48 * 1024)
      r = cudaFuncSetAttribute(prolong_tiled_kernel<T, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps);
    return r;
  }();
  return e;
}

// tile of the tiled transfers: 32 x 8 (FP32) / 16 x 8 (FP64) coarse positions for the
// restriction, 32 x 8 threads (FP32) / 16 x 8 (FP64) for the prolongation
template <typename T>
struct TransferTile {
  static constexpr int TX = sizeof(T) == 8 ? 16 : 32, TY = 8;
};

template <typename T>
int launch_restrict(const Level &fine, const Level &coarse, const T *rf, T *rc, cudaStream_t st) {
  constexpr int TX = TransferTile<T>::TX, TY = TransferTile<T>::TY;
  BMG_CUDA((opt_in_transfer_smem<T, TX, TY>()));
  dim3 block(TX, TY);
  dim3 grid((coarse.g.pitch + TX - 1) / TX, (coarse.n + 1 + TY - 1) / TY);
  { BMG_PROF_BEGIN(BMG_PROF_RESTRICT, fine.n, st);
  BMG_CUDA(launch_pdl(restrict_tiled_kernel<T, TX, TY>, dim3(grid), dim3(block), restrict_smem_bytes<T, TX, TY>(),
                      st, fine.g, coarse.g, rf, rc, fine.gate));
    BMG_PROF_END(st, (double)fine.n * fine.n); }
  BMG_CHECK_LAUNCH("restrict_tiled_kernel");
  return BMG_OK;
}

template <typename T>
int launch_prolong_add(const Level &fine, const Level &coarse, const T *xc, T *xf,
                       cudaStream_t st) {
  constexpr int TX = TransferTile<T>::TX, TY = TransferTile<T>::TY;
  BMG_CUDA((opt_in_transfer_smem<T, TX, TY>()));
  dim3 block(TX, TY);
  dim3 grid((fine.n / 2 + 1 + TX - 1) / TX, (fine.n + 1 + TY - 1) / TY);
  { BMG_PROF_BEGIN(BMG_PROF_PROLONG, fine.n, st);
  BMG_CUDA(launch_pdl(prolong_tiled_kernel<T, TX, TY>, dim3(grid), dim3(block), prolong_smem_bytes<T, TX, TY>(),
                      st, fine.g, coarse.g, xc, xf, fine.gate));
    BMG_PROF_END(st, (double)fine.n * fine.n); }
  BMG_CHECK_LAUNCH("prolong_tiled_kernel");
  return BMG_OK;
}

// ---- batched transfers: blockIdx.z = instance * NBLK + type -----------------------------
__global__ void restrict_batch_kernel(const TransferArgs *__restrict__ args) {
  const TransferArgs &a = args[blockIdx.z / NBLK];
  BMG_GATE(a.gate);
  const Grid gf = a.gf, gc = a.gc;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int ct = blockIdx.z % NBLK;
  const int nc = gc.n, nf = gf.n;
  if (I >= gc.pitch || J > nc) return;
  const size_t o = (size_t)J * gc.pitch + I;
  double acc = 0;
  if (I <= nc) {
    bool m[NBLK];
    dof_masks(I, J, nc, m);
    if (m[ct]) {
      const int ne = c_nres[ct];
      for (int e = 0; e < ne; ++e) {
        const StencilEntry se = c_res[ct][e];
        const int fi = 2 * I + se.di, fj = 2 * J + se.dj;
        if (fi < 0 || fj < 0 || fi > nf || fj > nf) continue;
        acc += se.coef * __ldg(a.src + se.type * gf.blk + (size_t)fj * gf.pitch + fi);
      }
    }
  }
  a.dst[ct * gc.blk + o] = acc;
}

__global__ void prolong_batch_kernel(const TransferArgs *__restrict__ args) {
  const TransferArgs &a = args[blockIdx.z / NBLK];
  BMG_GATE(a.gate);
  const Grid gf = a.gf, gc = a.gc;
  const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + (threadIdx.y & 1);   // parity per warp
  const int j = 2 * blockIdx.y + (threadIdx.y >> 1);
  const int t = blockIdx.z % NBLK;
  const int nf = gf.n, nc = gc.n;
  if (i > nf || j > nf) return;
  bool m[NBLK];
  dof_masks(i, j, nf, m);
  if (!m[t]) return;
  const int par = (i & 1) + 2 * (j & 1);
  const int I0 = i >> 1, J0 = j >> 1;
  const size_t o = (size_t)j * gf.pitch + i;
  double acc = 0;
  const int ne = c_npro[t][par];
  for (int e = 0; e < ne; ++e) {
    const StencilEntry se = c_pro[t][par][e];
    const int I = I0 + se.di, J = J0 + se.dj;
    if (I < 0 || J < 0 || I > nc || J > nc) continue;
    acc += se.coef * __ldg(a.src + se.type * gc.blk + (size_t)J * gc.pitch + I);
  }
  a.dst[t * gf.blk + o] += acc;
}

int launch_restrict_batch(const TransferArgs *d_args, int count, int nf, cudaStream_t st) {
  if (count <= 0) return BMG_OK;
  const Grid gc = grid_of(nf / 2);
  dim3 block(32, 4);
  dim3 grid((gc.pitch + 31) / 32, (gc.n + 1 + 3) / 4, NBLK * count);
  restrict_batch_kernel<<<grid, block, 0, st>>>(d_args);
  BMG_CHECK_LAUNCH("restrict_batch_kernel");
  return BMG_OK;
}

int launch_prolong_batch(const TransferArgs *d_args, int count, int nf, cudaStream_t st) {
  if (count <= 0) return BMG_OK;
  dim3 block(32, 4);
  dim3 grid((nf + 1 + 63) / 64, (nf + 1 + 1) / 2, NBLK * count);
  prolong_batch_kernel<<<grid, block, 0, st>>>(d_args);
  BMG_CHECK_LAUNCH("prolong_batch_kernel");
  return BMG_OK;
}

template int launch_restrict<double>(const Level &, const Level &, const double *, double *, cudaStream_t);
template int launch_restrict<float>(const Level &, const Level &, const float *, float *, cudaStream_t);
template int launch_prolong_add<double>(const Level &, const Level &, const double *, double *, cudaStream_t);
template int launch_prolong_add<float>(const Level &, const Level &, const float *, float *, cudaStream_t);

}  // namespace bmg
