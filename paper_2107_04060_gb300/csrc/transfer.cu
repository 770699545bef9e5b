// Grid transfers (Sec. 3, Eq. block_interp; Sec. 3.1): prolongation-and-correct
// x_f += P x_c and restriction r_c = P^T r_f, as constant stencils per DoF type (and per
// parity class of the fine position for P).  The tables are built once on the host from
// the definitions of P_u (divergence-preserving), P_w (canonical RT0) and P_p (injection);
// see element.cpp.  Couplings to positions outside the grid are skipped and slots beyond
// the valid ranges hold zeros, so the interior stencil is exact up to the boundary.
#include "bmg_internal.h"
#include "kernels_common.cuh"

namespace bmg {

TransferTables g_tables_host;
__constant__ StencilEntry c_pro[NBLK][4][kMaxPro];
__constant__ int c_npro[NBLK][4];
__constant__ StencilEntry c_res[NBLK][kMaxRes];
__constant__ int c_nres[NBLK];

int upload_transfer_tables() {
  static bool done = false;
  if (done) return BMG_OK;
  build_transfer_tables(&g_tables_host);
  BMG_CUDA(cudaMemcpyToSymbol(c_pro, g_tables_host.pro, sizeof(g_tables_host.pro)));
  BMG_CUDA(cudaMemcpyToSymbol(c_npro, g_tables_host.npro, sizeof(g_tables_host.npro)));
  BMG_CUDA(cudaMemcpyToSymbol(c_res, g_tables_host.res, sizeof(g_tables_host.res)));
  BMG_CUDA(cudaMemcpyToSymbol(c_nres, g_tables_host.nres, sizeof(g_tables_host.nres)));
  done = true;
  return BMG_OK;
}

// FP32 stencil tables staged in shared memory by each CTA: the flat offset of every entry
// (type plane, row and column folded for this level's layout) and its FP32 coefficient, with
// the largest row/column reach of the table.  Positions whose whole stencil lies inside the
// grid then cost one shared read, one load and one multiply-add per entry, with no bounds
// test; the others take the checked path.  The sums keep the table's order.  (The FP32
// transfers are bound by instruction issue; the FP64 ones keep the plain per-entry loop.)
template <int N>
struct StagedStencil {
  long long off[N];
  float coef[N];
  int n, reach;
};

__device__ __forceinline__ void stage_stencil_entry(const StencilEntry &se, size_t blk, int pitch,
                                                    long long &off, float &coef) {
  off = (long long)se.type * (long long)blk + (long long)se.dj * pitch + se.di;
  coef = se.coef32;
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
  if constexpr (sizeof(T) == 4) {
    __shared__ StagedStencil<kMaxRes> st;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    const int ne = c_nres[ct];
    for (int e = tid; e < ne; e += nt) stage_stencil_entry(c_res[ct][e], gf.blk, gf.pitch, st.off[e], st.coef[e]);
    if (tid == 0) {
      int r = 0;
      for (int e = 0; e < ne; ++e) r = max(r, max(abs((int)c_res[ct][e].di), abs((int)c_res[ct][e].dj)));
      st.n = ne;
      st.reach = r;
    }
    __syncthreads();
    if (I >= gc.pitch || J > nc) return;
    const size_t o = (size_t)J * gc.pitch + I;
    float acc = 0.f;
    if (I <= nc) {
      bool m[NBLK];
      dof_masks(I, J, nc, m);
      if (m[ct]) {
        const int rch = st.reach, fi0 = 2 * I, fj0 = 2 * J;
        if (fi0 - rch >= 0 && fj0 - rch >= 0 && fi0 + rch <= nf && fj0 + rch <= nf) {
          const float *base = rf + (size_t)fj0 * gf.pitch + fi0;
#pragma unroll 4
          for (int e = 0; e < ne; ++e) acc += st.coef[e] * __ldg(base + st.off[e]);
        } else {
          for (int e = 0; e < ne; ++e) {
            const StencilEntry se = c_res[ct][e];
            const int fi = fi0 + se.di, fj = fj0 + se.dj;
            if (fi < 0 || fj < 0 || fi > nf || fj > nf) continue;
            acc += se.coef32 * __ldg(rf + se.type * gf.blk + (size_t)fj * gf.pitch + fi);
          }
        }
      }
    }
    rc[ct * gc.blk + o] = acc;
    return;
  }
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
  if constexpr (sizeof(T) == 4) {
    // the four parity classes' tables (threadIdx.y is the class), staged as in restrict_kernel
    __shared__ StagedStencil<kMaxPro> st[4];
    const int cls = threadIdx.y, ne = c_npro[t][cls];
    for (int e = threadIdx.x; e < ne; e += blockDim.x)
      stage_stencil_entry(c_pro[t][cls][e], gc.blk, gc.pitch, st[cls].off[e], st[cls].coef[e]);
    if (threadIdx.x == 0) {
      int r = 0;
      for (int e = 0; e < ne; ++e) r = max(r, max(abs((int)c_pro[t][cls][e].di), abs((int)c_pro[t][cls][e].dj)));
      st[cls].n = ne;
      st[cls].reach = r;
    }
    __syncthreads();
    if (i > nf || j > nf) return;
    bool mk[NBLK];
    dof_masks(i, j, nf, mk);
    if (!mk[t]) return;
    const int I0 = i >> 1, J0 = j >> 1, rch = st[cls].reach;
    const size_t o = (size_t)j * gf.pitch + i;
    float acc = 0.f;
    if (I0 - rch >= 0 && J0 - rch >= 0 && I0 + rch <= nc && J0 + rch <= nc) {
      const float *base = xc + (size_t)J0 * gc.pitch + I0;
#pragma unroll 4
      for (int e = 0; e < ne; ++e) acc += st[cls].coef[e] * __ldg(base + st[cls].off[e]);
    } else {
      for (int e = 0; e < ne; ++e) {
        const StencilEntry se = c_pro[t][cls][e];
        const int I = I0 + se.di, J = J0 + se.dj;
        if (I < 0 || J < 0 || I > nc || J > nc) continue;
        acc += se.coef32 * __ldg(xc + se.type * gc.blk + (size_t)J * gc.pitch + I);
      }
    }
    xf[t * gf.blk + o] += acc;
    return;
  }
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

template <typename T>
int launch_restrict(const Level &fine, const Level &coarse, const T *rf, T *rc, cudaStream_t st) {
  dim3 block(32, 4);
  dim3 grid((coarse.g.pitch + 31) / 32, (coarse.n + 1 + 3) / 4, NBLK);
  { BMG_PROF_BEGIN(BMG_PROF_RESTRICT, fine.n, st);
  BMG_CUDA(launch_pdl(restrict_kernel<T>, dim3(grid), dim3(block), 0, st, fine.g, coarse.g, rf, rc, fine.gate));
    BMG_PROF_END(st, (double)fine.n * fine.n); }
  BMG_CHECK_LAUNCH("restrict_kernel");
  return BMG_OK;
}

template <typename T>
int launch_prolong_add(const Level &fine, const Level &coarse, const T *xc, T *xf,
                       cudaStream_t st) {
  dim3 block(32, 4);
  dim3 grid((fine.n + 1 + 63) / 64, (fine.n + 1 + 1) / 2, NBLK);
  { BMG_PROF_BEGIN(BMG_PROF_PROLONG, fine.n, st);
  BMG_CUDA(launch_pdl(prolong_kernel<T>, dim3(grid), dim3(block), 0, st, fine.g, coarse.g, xc, xf, fine.gate));
    BMG_PROF_END(st, (double)fine.n * fine.n); }
  BMG_CHECK_LAUNCH("prolong_kernel");
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
