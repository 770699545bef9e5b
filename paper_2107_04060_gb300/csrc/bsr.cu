// Inexact Braess-Sarazin relaxation (Sec. 3.2.2, App. D) on the saddle-point form
// [[A, B^T], [B, -C]], y = (u, w):
//   F   = blockdiag(additive Vanka on A_u^RQ with the 8-DoF displacement patches of Fig. 3
//         left (undamped, natural weights), tau D_w),  D_w = diag(M_w)
//   S  ~= (1/M + alpha^2 / (lambda + 2 mu / d)) M_p + tau B_w D_w^{-1} B_w^T   (d = 2)
//   z   = F^{-1} r_y;   dp = omega_J diag(S)^{-1} (B z - r_p);   dy = F^{-1}(r_y - B^T dp)
//   x  <- x + omega (dy, dp)
// Kernels: (1) z = F^{-1} r_y; (2) dp per triangle; (3) dy = F^{-1}(r_y - B^T dp) fused with
// the update, r_y - B^T dp formed from the coupling terms of the element products alone
// (alpha g_T dp_T, tau dw_T dp_T) while the residual is gathered.
#include <algorithm>

#include "bmg_internal.h"
#include "kernels_common.cuh"

namespace bmg {

// 1 / (tau D_w) on every edge and omega_J / diag(S) on every triangle.
struct BsrSetupArgs {
  Grid g;
  const double *kinv;
  const double *wm;
  int wm_full;
  OpCoefs<double> c;
  double c_fs_area;   // (1/M + alpha^2/(lambda + mu)) |T|
  double omega_J;
  double *dinv64;
  float *dinv32;
  double *sinv64;
  float *sinv32;
};

__device__ __forceinline__ double wdiag(const BsrSetupArgs &a, int o, int ci, int cj, int k) {
  const size_t co = (size_t)o * (a.wm_full ? 6 : 1) * a.g.blk + (size_t)cj * a.g.pitch + ci;
  if (a.wm_full) {
    const int d[3] = {0, 3, 5};
    return a.wm[co + (size_t)d[k] * a.g.blk];
  }
  return a.kinv[co] * a.c.M1[o][k * 3 + k];
}

__global__ void bsr_setup_kernel(const __grid_constant__ BsrSetupArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = a.g.n;
  if (i > n || j > n) return;
  const size_t o = (size_t)j * a.g.pitch + i;
  const size_t blk = a.g.blk;
  // tau D_w of h(i,j): L(i,j) e2 + U(i,j-1) e2;  v(i,j): L(i,j) e1 + U(i-1,j) e1;
  // d(i,j): L(i,j) e0 + U(i,j) e0
  double dh = 0, dv = 0, dd = 0;
  if (i < n) {
    if (j < n) dh += wdiag(a, 0, i, j, 2);
    if (j > 0) dh += wdiag(a, 1, i, j - 1, 2);
  }
  if (j < n) {
    if (i < n) dv += wdiag(a, 0, i, j, 1);
    if (i > 0) dv += wdiag(a, 1, i - 1, j, 1);
  }
  if (i < n && j < n) dd = wdiag(a, 0, i, j, 0) + wdiag(a, 1, i, j, 0);
  const double ih = dh > 0 ? 1.0 / dh : 0.0, iv = dv > 0 ? 1.0 / dv : 0.0, id = dd > 0 ? 1.0 / dd : 0.0;
  a.dinv64[0 * blk + o] = ih; a.dinv32[0 * blk + o] = (float)ih;
  a.dinv64[1 * blk + o] = iv; a.dinv32[1 * blk + o] = (float)iv;
  a.dinv64[2 * blk + o] = id; a.dinv32[2 * blk + o] = (float)id;
  if (i < n && j < n) {
    // diag(S)_T = c_fs |T| + sum_e (tau B_w)_{T,e}^2 / (tau D_w)_e
    const double dL[3] = {dd, dv, dh};
    double dvU = 0, dhU = 0;
    dvU = wdiag(a, 1, i, j, 1) + (i + 1 < n ? wdiag(a, 0, i + 1, j, 1) : 0.0);
    dhU = wdiag(a, 1, i, j, 2) + (j + 1 < n ? wdiag(a, 0, i, j + 1, 2) : 0.0);
    const double dU[3] = {dd, dvU, dhU};
    double sL = a.c_fs_area, sU = a.c_fs_area;
    for (int k = 0; k < 3; ++k) {
      sL += a.c.dw[0][k] * a.c.dw[0][k] / dL[k];
      sU += a.c.dw[1][k] * a.c.dw[1][k] / dU[k];
    }
    a.sinv64[0 * blk + o] = a.omega_J / sL; a.sinv32[0 * blk + o] = (float)(a.omega_J / sL);
    a.sinv64[1 * blk + o] = a.omega_J / sU; a.sinv32[1 * blk + o] = (float)(a.omega_J / sU);
  } else {
    a.sinv64[o] = 0; a.sinv32[o] = 0; a.sinv64[blk + o] = 0; a.sinv32[blk + o] = 0;
  }
}

int launch_bsr_setup(Level &L, double omega_J, double c_fs_area, cudaStream_t st) {
  const size_t blk = L.g.blk;
  BMG_CUDA(cudaMalloc(&L.dinv64, sizeof(double) * 3 * blk));
  BMG_CUDA(cudaMalloc(&L.dinv32, sizeof(float) * 3 * blk));
  BMG_CUDA(cudaMalloc(&L.sinv64, sizeof(double) * 2 * blk));
  BMG_CUDA(cudaMalloc(&L.sinv32, sizeof(float) * 2 * blk));
  BMG_CUDA(cudaMemsetAsync(L.dinv64, 0, sizeof(double) * 3 * blk, st));
  BMG_CUDA(cudaMemsetAsync(L.dinv32, 0, sizeof(float) * 3 * blk, st));
  BMG_CUDA(cudaMemsetAsync(L.sinv64, 0, sizeof(double) * 2 * blk, st));
  BMG_CUDA(cudaMemsetAsync(L.sinv32, 0, sizeof(float) * 2 * blk, st));
  BsrSetupArgs a;
  a.g = L.g;
  a.kinv = L.kinv64;
  a.wm = L.wm64;
  a.wm_full = L.wm_full ? 1 : 0;
  a.c = L.c64;
  a.c_fs_area = c_fs_area;
  a.omega_J = omega_J;
  a.dinv64 = L.dinv64;
  a.dinv32 = L.dinv32;
  a.sinv64 = L.sinv64;
  a.sinv32 = L.sinv32;
  dim3 b(32, 8), gr((L.n + 1 + 31) / 32, (L.n + 1 + 7) / 8);
  bsr_setup_kernel<<<gr, b, 0, st>>>(a);
  BMG_CHECK_LAUNCH("bsr_setup_kernel");
  return BMG_OK;
}

// --------------------------------------------------------------------------------------
// Displacement Vanka (8-DoF patches) applied to the u part of `r` plus the Jacobi step on
// the w part.  mode 0: z_y = F^{-1} r_y written into `z` (u, w blocks);
// mode 1: x_y += omega F^{-1} r_y and x_p += omega dp (dp from the p blocks of `d`).
template <typename T>
struct VankaUArgs {
  Grid g;
  const T *r;
  T *z;          // mode 0 output
  T *x;          // mode 1 update
  const T *d;    // mode 1: dp in the p blocks
  const int *slot;
  const T *inv;
  int nslots;
  const T *dinv;
  T omega;
  int mode;
  int assign;    // mode 1 only: x was zero, write instead of add
  const int *gate;
  // mode 1: r is the original residual and r_y - B^T dp is formed on the fly from dp:
  // + alpha g_T dp_T on the displacement DoFs, + tau dw_T dp_T on the flux DoFs
  T ag[2][9];    // alpha * g
  T dwc[2][3];   // tau * dw
};

// dp of triangle b (PL or PU) of cell (ci, cj); 0 outside the grid
template <typename T>
__device__ __forceinline__ T dp_at(const VankaUArgs<T> &a, int b, int ci, int cj) {
  const int n = a.g.n;
  return (ci >= 0 && cj >= 0 && ci < n && cj < n) ? a.d[b * a.g.blk + (size_t)cj * a.g.pitch + ci] : T(0);
}

// kQX x kQY patches per CTA, NT threads; outputs (kQX - 1) x (kQY - 1).  Same three phases
// as the 20-DoF sweep: residual gather, (patch, row) solve tasks, weighted gather.
// kPT: the thread that gathers a patch's residual also solves it (64 FMAs, each inverse
// entry loaded once per patch, in the order of the row tasks' sums), and the task phase is
// skipped.
template <typename T, int kQX, int kQY, int NT, bool kPT = false>
__global__ void __launch_bounds__(NT) vanka_u_kernel(const __grid_constant__ VankaUArgs<T> a) {
  pdl_enter();
  BMG_GATE(a.gate);
  constexpr int NP = kQX * kQY, LD = 9;
  __shared__ T sr[NP * LD];
  __shared__ T sx[NP * LD];
  __shared__ int ss[NP];
  const int n = a.g.n, P = a.g.pitch;
  const size_t blk = a.g.blk;
  const int i0 = blockIdx.x * (kQX - 1), j0 = blockIdx.y * (kQY - 1);
  const int tid = threadIdx.x;
  for (int p = tid; p < NP; p += NT) {
    const int pi = i0 + p % kQX, pj = j0 + p / kQX;
    T *rl = sr + p * LD;
    if (pi <= n && pj <= n) {
      const T *r = a.r;
      const size_t o = (size_t)pj * P + pi;
      const bool li = pi >= 1, lj = pj >= 1;
      rl[0] = r[UX * blk + o];
      rl[1] = r[UY * blk + o];
      rl[2] = r[BH * blk + o];
      rl[3] = r[BV * blk + o];
      rl[4] = li ? r[BH * blk + o - 1] : T(0);
      rl[5] = lj ? r[BV * blk + o - P] : T(0);
      rl[6] = li ? r[BD * blk + o - 1] : T(0);
      rl[7] = lj ? r[BD * blk + o - P] : T(0);
      if (a.mode == 1) {
        // r_y - B^T dp: the couplings of the six triangles around the vertex (local vertex 0
        // of L(pi,pj), U(pi-1,pj-1); 1 of L(pi-1,pj), U(pi,pj-1); 2 of L(pi,pj-1), U(pi-1,pj))
        // onto its displacement and the bubbles of its six edges; constrained slots stay 0
        const T dL = dp_at(a, PL, pi, pj), dLw = dp_at(a, PL, pi - 1, pj), dLs = dp_at(a, PL, pi, pj - 1);
        const T dUw = dp_at(a, PU, pi - 1, pj), dUsw = dp_at(a, PU, pi - 1, pj - 1), dUs = dp_at(a, PU, pi, pj - 1);
        const bool vf = pi > 0 && pi < n && pj > 0 && pj < n;
        const bool hf = pj > 0 && pj < n, vvf = pi > 0 && pi < n;
        if (vf) {
          rl[0] += a.ag[0][0] * dL + a.ag[0][1] * dLw + a.ag[0][2] * dLs + a.ag[1][2] * dUw +
                   a.ag[1][0] * dUsw + a.ag[1][1] * dUs;
          rl[1] += a.ag[0][3] * dL + a.ag[0][4] * dLw + a.ag[0][5] * dLs + a.ag[1][5] * dUw +
                   a.ag[1][3] * dUsw + a.ag[1][4] * dUs;
        }
        if (pi < n && hf) rl[2] += a.ag[0][8] * dL + a.ag[1][8] * dUs;          // h(pi, pj)
        if (pj < n && vvf) rl[3] += a.ag[0][7] * dL + a.ag[1][7] * dUw;         // v(pi, pj)
        if (li && hf) rl[4] += a.ag[0][8] * dLw + a.ag[1][8] * dUsw;            // h(pi-1, pj)
        if (lj && vvf) rl[5] += a.ag[0][7] * dLs + a.ag[1][7] * dUsw;           // v(pi, pj-1)
        if (li && pj < n) rl[6] += a.ag[0][6] * dLw + a.ag[1][6] * dUw;         // d(pi-1, pj)
        if (lj && pi < n) rl[7] += a.ag[0][6] * dLs + a.ag[1][6] * dUs;         // d(pi, pj-1)
      }
      ss[p] = a.slot[(size_t)pj * (n + 1) + pi];
    } else {
#pragma unroll
      for (int c = 0; c < 8; ++c) rl[c] = T(0);
      ss[p] = 0;
    }
    if constexpr (kPT) {
      T r[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) r[c] = rl[c];
      const T *inv = a.inv + ss[p];
      const size_t ld = (size_t)a.nslots;
#pragma unroll
      for (int row = 0; row < 8; ++row) {
        T acc = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) acc = fma(__ldg(inv + (size_t)(row * 8 + c) * ld), r[c], acc);
        sx[p * LD + row] = acc;
      }
    }
  }
  __syncthreads();
  const size_t ld = (size_t)a.nslots;
  for (int t = tid; t < (kPT ? 0 : NP * 8); t += NT) {
    const int row = t / NP, p = t % NP;
    const T *inv = a.inv + ss[p] + (size_t)(row * 8) * ld;
    const T *rl = sr + p * LD;
    T acc = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) acc = fma(inv[(size_t)c * ld], rl[c], acc);
    sx[p * LD + row] = acc;
  }
  if constexpr (!kPT) __syncthreads();
  for (int q = tid; q < (kQX - 1) * (kQY - 1); q += NT) {
    const int i = i0 + q % (kQX - 1), j = j0 + q / (kQX - 1);
    if (j > n) continue;
    if (i > n) {                  // padding columns: written only when assigning
      if ((a.mode == 1 && a.assign) && i < P) {
#pragma unroll
        for (int k = 0; k < NBLK; ++k) a.x[k * blk + (size_t)j * P + i] = T(0);
      }
      continue;
    }
    auto X = [&](int pi, int pj, int k) -> T { return sx[((pj - j0) * kQX + (pi - i0)) * LD + k]; };
    bool m[NBLK];
    dof_masks(i, j, n, m);
    const size_t o = (size_t)j * P + i;
    const T h = T(0.5);
    T v[8];
    v[UX] = m[UX] ? X(i, j, 0) : T(0);
    v[UY] = m[UY] ? X(i, j, 1) : T(0);
    v[BH] = m[BH] ? h * (X(i, j, 2) + X(i + 1, j, 4)) : T(0);
    v[BV] = m[BV] ? h * (X(i, j, 3) + X(i, j + 1, 5)) : T(0);
    v[BD] = m[BD] ? h * (X(i, j + 1, 7) + X(i + 1, j, 6)) : T(0);
    T rwh = a.r[WH * blk + o], rwv = a.r[WV * blk + o], rwd = a.r[WD * blk + o];
    if (a.mode == 1) {            // + tau dw_T dp_T of the two triangles of each edge
      const T dL = dp_at(a, PL, i, j), dU = dp_at(a, PU, i, j);
      rwh += a.dwc[0][2] * dL + a.dwc[1][2] * dp_at(a, PU, i, j - 1);
      rwv += a.dwc[0][1] * dL + a.dwc[1][1] * dp_at(a, PU, i - 1, j);
      rwd += a.dwc[0][0] * dL + a.dwc[1][0] * dU;
    }
    v[WH] = m[WH] ? a.dinv[0 * blk + o] * rwh : T(0);
    v[WV] = m[WV] ? a.dinv[1 * blk + o] * rwv : T(0);
    v[WD] = m[WD] ? a.dinv[2 * blk + o] * rwd : T(0);
    if (a.mode == 0) {
#pragma unroll
      for (int k = 0; k < 8; ++k) a.z[k * blk + o] = v[k];
    } else if (a.assign) {
      T *x = a.x;
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k * blk + o] = m[k] ? a.omega * v[k] : T(0);
      x[PL * blk + o] = m[PL] ? a.omega * a.d[PL * blk + o] : T(0);
      x[PU * blk + o] = m[PU] ? a.omega * a.d[PU * blk + o] : T(0);
    } else {
      T *x = a.x;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (m[k]) x[k * blk + o] += a.omega * v[k];
      if (m[PL]) x[PL * blk + o] += a.omega * a.d[PL * blk + o];
      if (m[PU]) x[PU * blk + o] += a.omega * a.d[PU * blk + o];
    }
  }
}

// dp_T = omega_J / diag(S)_T * ((B z)_T - r_p,T),  (B z)_T = -alpha g_T . z_u - tau dw_T . z_w
template <typename T>
struct DpArgs {
  Grid g;
  const T *z;
  const T *r;
  T *d;
  const T *sinv;
  const int *gate;
  OpCoefs<T> c;
  int raw;       // 1: write B z - r_p itself (exact BSR's right-hand side) into d[0 .. 2 blk)
};

template <typename T>
__global__ void bsr_dp_kernel(const __grid_constant__ DpArgs<T> a) {
  pdl_enter();
  BMG_GATE(a.gate);
  const int ci = blockIdx.x * blockDim.x + threadIdx.x;
  const int cj = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = a.g.n, P = a.g.pitch;
  const size_t blk = a.g.blk;
  if (ci >= n || cj >= n) return;
  const T *z = a.z;
  const size_t c00 = (size_t)cj * P + ci, c10 = c00 + 1, c01 = c00 + P, c11 = c00 + P + 1;
  const T bd = z[BD * blk + c00], wd = z[WD * blk + c00];
  {
    const T u[9] = {z[UX * blk + c00], z[UX * blk + c10], z[UX * blk + c01],
                    z[UY * blk + c00], z[UY * blk + c10], z[UY * blk + c01],
                    bd, z[BV * blk + c00], z[BH * blk + c00]};
    const T w[3] = {wd, z[WV * blk + c00], z[WH * blk + c00]};
    T gu = 0, dz = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) gu = fma(a.c.g[0][k], u[k], gu);
#pragma unroll
    for (int k = 0; k < 3; ++k) dz = fma(a.c.dw[0][k], w[k], dz);
    const T Bz = -a.c.alpha * gu - dz;
    const T v = Bz - a.r[PL * blk + c00];
    if (a.raw) a.d[c00] = v;
    else a.d[PL * blk + c00] = a.sinv[c00] * v;
  }
  {
    const T u[9] = {z[UX * blk + c11], z[UX * blk + c01], z[UX * blk + c10],
                    z[UY * blk + c11], z[UY * blk + c01], z[UY * blk + c10],
                    bd, z[BV * blk + c10], z[BH * blk + c01]};
    const T w[3] = {wd, z[WV * blk + c10], z[WH * blk + c01]};
    T gu = 0, dz = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) gu = fma(a.c.g[1][k], u[k], gu);
#pragma unroll
    for (int k = 0; k < 3; ++k) dz = fma(a.c.dw[1][k], w[k], dz);
    const T Bz = -a.c.alpha * gu - dz;
    const T v = Bz - a.r[PU * blk + c00];
    if (a.raw) a.d[blk + c00] = v;
    else a.d[PU * blk + c00] = a.sinv[blk + c00] * v;
  }
}

template <typename T, int QX, int QY, int NT, bool PT = false>
static void launch_vanka_u_tile(const VankaUArgs<T> &a, const Level &L, cudaStream_t st) {
  dim3 grid((L.g.pitch + QX - 2) / (QX - 1), (L.n + 1 + QY - 2) / (QY - 1));
  (void)launch_pdl(vanka_u_kernel<T, QX, QY, NT, PT>, dim3(grid), dim3(NT), 0, st, a);
}

template <typename T>
static int launch_vanka_u(const Level &L, const T *r, T *z, T *x, const T *d, T omega, int mode,
                          bool assign, cudaStream_t st) {
  const bool f64 = sizeof(T) == 8;
  VankaUArgs<T> a;
  a.g = L.g;
  a.r = r;
  a.z = z;
  a.x = x;
  a.d = d;
  a.slot = L.slot;
  a.inv = (const T *)(f64 ? (const void *)L.pinv64 : (const void *)L.pinv32);
  a.nslots = L.nslots;
  a.dinv = (const T *)(f64 ? (const void *)L.dinv64 : (const void *)L.dinv32);
  a.omega = omega;
  a.mode = mode;
  a.assign = assign ? 1 : 0;
  a.gate = L.gate;
  {
    const OpCoefs<T> &c = *reinterpret_cast<const OpCoefs<T> *>(f64 ? (const void *)&L.c64 : (const void *)&L.c32);
    for (int o = 0; o < 2; ++o) {
      for (int k = 0; k < 9; ++k) a.ag[o][k] = c.alpha * c.g[o][k];
      for (int k = 0; k < 3; ++k) a.dwc[o][k] = c.dw[o][k];
    }
  }
  auto ctas = [&](int px, int py) {
    return (long long)((L.g.pitch + px - 2) / (px - 1)) * ((L.n + 1 + py - 2) / (py - 1));
  };
  BMG_PROF_BEGIN(BMG_PROF_VANKA_U, L.n, st);
  const long long want = 2 * 152;
  switch (L.tile_vanka_u) {          // tuned at setup
    case 0: launch_vanka_u_tile<T, 32, 8, 256>(a, L, st); break;
    case 1: launch_vanka_u_tile<T, 16, 8, 256>(a, L, st); break;
    case 2: launch_vanka_u_tile<T, 8, 8, 128>(a, L, st); break;
    case 3: launch_vanka_u_tile<T, 8, 4, 128>(a, L, st); break;
    case 4: launch_vanka_u_tile<T, 4, 4, 64>(a, L, st); break;
    case 5: launch_vanka_u_tile<T, 32, 8, 256, true>(a, L, st); break;   // one thread per patch solve
    case 6: launch_vanka_u_tile<T, 16, 8, 128, true>(a, L, st); break;
    case 7: launch_vanka_u_tile<T, 8, 8, 64, true>(a, L, st); break;
    default:
      if (ctas(32, 8) >= want) launch_vanka_u_tile<T, 32, 8, 256>(a, L, st);
      else if (ctas(16, 8) >= want) launch_vanka_u_tile<T, 16, 8, 256>(a, L, st);
      else if (ctas(8, 8) >= want) launch_vanka_u_tile<T, 8, 8, 128>(a, L, st);
      else if (ctas(8, 4) >= want) launch_vanka_u_tile<T, 8, 4, 128>(a, L, st);
      else launch_vanka_u_tile<T, 4, 4, 64>(a, L, st);
  }
  BMG_PROF_END(st, (double)L.n * L.n);
  BMG_CHECK_LAUNCH("vanka_u_kernel");
  return BMG_OK;
}

// One BSR relaxation x <- x + omega M^{-1} r.  Work vectors of the level: bz (z = F^{-1} r_y),
// bd (dp in the p blocks; its u and w blocks stay zero).
template <typename T>
int launch_bsr_sweep(const Level &L, const T *r, T *x, T omega, cudaStream_t st, bool assign) {
  const bool f64 = sizeof(T) == 8;
  T *z = (T *)L.bz;
  T *d = (T *)L.bd;
  int rc = launch_vanka_u<T>(L, r, z, nullptr, nullptr, omega, 0, false, st);
  if (rc) return rc;
  DpArgs<T> a;
  a.g = L.g;
  a.z = z;
  a.r = r;
  a.d = d;
  a.sinv = (const T *)(f64 ? (const void *)L.sinv64 : (const void *)L.sinv32);
  a.gate = L.gate;
  a.c = *reinterpret_cast<const OpCoefs<T> *>(f64 ? (const void *)&L.c64 : (const void *)&L.c32);
  a.raw = 0;
  dim3 b(32, 8), gr((L.n + 31) / 32, (L.n + 7) / 8);
  { BMG_PROF_BEGIN(BMG_PROF_VANKA_U, L.n, st);
  BMG_CUDA(launch_pdl(bsr_dp_kernel<T>, dim3(gr), dim3(b), 0, st, a));
    BMG_PROF_END(st, 0.0); }
  BMG_CHECK_LAUNCH("bsr_dp_kernel");
  // dy = F^{-1}(r_y - B^T dp) with r_y - B^T dp formed inside the displacement sweep
  return launch_vanka_u<T>(L, r, nullptr, x, d, omega, 1, assign, st);
}

template int launch_bsr_sweep<double>(const Level &, const double *, double *, double, cudaStream_t, bool);
template int launch_bsr_sweep<float>(const Level &, const float *, float *, float, cudaStream_t, bool);

// ---- exact BSR (Sec. 3.2.2: Eq. bsr_p with the fixed-stress S solved, not relaxed) -------
// S = c I + (tau B_w) (tau D_w)^{-1} (tau B_w)^T on the P0 space, c = (1/M + alpha^2/(lambda +
// mu)) |T|, is symmetric positive definite; the pressure step runs preconditioned conjugate
// gradients on it to a relative residual of kCgRtol: with a multigrid V-cycle on the S of the
// coarser levels (smg_vcycle below) where the hierarchy has them, with Jacobi on its last
// smoothing level.  The P0 space is the two
// triangle blocks (L, U) of blk slots each; cell (i, j) sits at j * pitch + i in both, and the
// slots outside the n x n cells stay zero in every CG vector.  Per triangle the product is
//   (S y)_T = c y_T + sum_{edges e of T} (tau B_w)_{T,e} (tau D_w)_e^{-1} sum_{T' on e} (tau B_w)_{T',e} y_T'
// with the edges d(i,j) (L(i,j), U(i,j)), v(i,j) (L(i,j), U(i-1,j)), h(i,j) (L(i,j), U(i,j-1));
// boundary edges carry one triangle.  The sign of (tau B_w) cancels in every product.
//
// One CG iteration is two kernels over a fixed grid of CTAs (grid-stride over cells):
//   dir_apply(k): rz_k, rr_k from the previous kernel's per-CTA partials (every CTA sums them
//                 in the same order, so all see the same scalars); stop test; beta; the new
//                 direction p_k = z + beta p_{k-1} on the cell and its four neighbours (so no
//                 CTA waits for another); q = S p_k; partials of p_k . q
//   update(k):    alpha = rz_k / (p_k . q); x += alpha p_k; r -= alpha q; with Jacobi:
//                 z = D^{-1} r and the partials of r . z and r . r; with the multigrid
//                 preconditioner the V-cycle's kernels form z and cg_dots_kernel the partials
// Partials, rz and the direction alternate between two slots by iteration parity, so a kernel
// never overwrites what a CTA of the same launch still reads.  A device flag ends the
// iteration: the kernels after the stop return at once, and the host reads the flag every
// kCgCheck iterations (every 4 with the multigrid preconditioner).
constexpr int kCgThreads = 256;
constexpr double kCgRtol = 1e-11;
constexpr int kCgMaxIt = 20000;
constexpr int kCgCheck = 16;
constexpr int kCgVecs = 5;       // r, z, q, p (two slots)

struct CgArgs {
  Grid g;
  double c;
  double dw[2][3];          // (tau B_w) up to sign, L and U orientation, edges d, v, h
  const double *dinv;       // [3][blk] 1 / (tau D_w): h, v, d
  const double *minv;       // [2][blk] 1 / diag(S)
  double *r, *z, *q, *p[2]; // 2 blk each
  double *x;                // the p blocks of the BSR work vector (2 blk)
  double *part;             // [5][grid]: rz (2 parity slots), rr (2), pq
  double *scal;             // [3]: rz by parity, rr_0
  int *flag;                // [0] 0 running, 1 converged, 2 non-finite; [1] iterations
  int k;
  double tol2;
  int mg;                   // 1: z = M r by the multigrid preconditioner (separate kernels)
};

// (S y) at the two triangles of cell (i, j) of an n x n level; val(e) gives y at slot e of the
// two-block P0 vector (e in [0, 2 blk)).
template <typename F>
__device__ __forceinline__ void s_product(const Grid &g, double c, const double (&dw)[2][3], const double *dinv,
                                          int i, int j, F &&val, double &yL, double &yU, double &qL,
                                          double &qU) {
  const int n = g.n, P = g.pitch;
  const size_t blk = g.blk, o = (size_t)j * P + i;
  yL = val(o);
  yU = val(blk + o);
  const double yUw = i > 0 ? val(blk + o - 1) : 0.0;        // U(i-1, j)
  const double yUs = j > 0 ? val(blk + o - P) : 0.0;        // U(i, j-1)
  const double yLe = i + 1 < n ? val(o + 1) : 0.0;          // L(i+1, j)
  const double yLn = j + 1 < n ? val(o + P) : 0.0;          // L(i, j+1)
  const double L0 = dw[0][0], L1 = dw[0][1], L2 = dw[0][2];
  const double U0 = dw[1][0], U1 = dw[1][1], U2 = dw[1][2];
  const double id = dinv[2 * blk + o];                      // d(i, j)
  const double ivL = dinv[1 * blk + o], ivU = dinv[1 * blk + o + 1];   // v(i, j), v(i+1, j)
  const double ihL = dinv[0 * blk + o], ihU = dinv[0 * blk + o + P];   // h(i, j), h(i, j+1)
  const double fd = id * fma(L0, yL, U0 * yU);
  qL = c * yL + L0 * fd + L1 * ivL * fma(L1, yL, U1 * yUw) + L2 * ihL * fma(L2, yL, U2 * yUs);
  qU = c * yU + U0 * fd + U1 * ivU * fma(U1, yU, L1 * yLe) + U2 * ihU * fma(U2, yU, L2 * yLn);
}

__device__ __forceinline__ double cg_block_sum(double v, double *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();                     // sh may still be read by a previous call
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < kCgThreads / 32; ++i) t += sh[i];
  return t;
}

// The stop flag as one value for the whole CTA (a later CTA of the same launch may see it
// set by CTA 0; the threads of one CTA must agree before the barriers that follow).
__device__ __forceinline__ bool cg_stopped(const int *flag) {
  __shared__ int s;
  if (threadIdx.x == 0) s = *(volatile const int *)flag;
  __syncthreads();
  return s != 0;
}

// sum of the `grid` partials at p, the same value in every CTA
__device__ __forceinline__ double cg_reduce(const double *p, int grid, double *sh) {
  double v = 0.0;
  for (int i = threadIdx.x; i < grid; i += kCgThreads) v += p[i];
  return cg_block_sum(v, sh);
}

__global__ void __launch_bounds__(kCgThreads) cg_init_kernel(const __grid_constant__ CgArgs a) {
  __shared__ double sh[kCgThreads / 32];
  const int n = a.g.n, P = a.g.pitch;
  const size_t blk = a.g.blk;
  double rz = 0.0, rr = 0.0;
  for (int c = blockIdx.x * kCgThreads + threadIdx.x; c < n * n; c += gridDim.x * kCgThreads) {
    const size_t o = (size_t)(c / n) * P + c % n;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const size_t e = t * blk + o;
      a.x[e] = 0.0;
      if (a.mg) continue;
      const double r = a.r[e], z = a.minv[e] * r;
      a.z[e] = z;
      rz = fma(r, z, rz);
      rr = fma(r, r, rr);
    }
  }
  const int G = gridDim.x;
  rz = cg_block_sum(rz, sh);
  rr = cg_block_sum(rr, sh);
  if (threadIdx.x == 0) {
    a.part[0 * G + blockIdx.x] = rz;
    a.part[2 * G + blockIdx.x] = rr;
    if (blockIdx.x == 0) a.flag[0] = a.flag[1] = 0;
  }
}

__global__ void __launch_bounds__(kCgThreads) cg_dir_apply_kernel(const __grid_constant__ CgArgs a) {
  __shared__ double sh[kCgThreads / 32];
  if (cg_stopped(a.flag)) return;
  const int G = gridDim.x, k = a.k, par = k & 1;
  const double rz = cg_reduce(a.part + (0 + par) * G, G, sh);
  const double rr = cg_reduce(a.part + (2 + par) * G, G, sh);
  const double rr0 = k == 0 ? rr : a.scal[2];
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  if (!isfinite(rr) || !isfinite(rz) || rr <= a.tol2 * rr0) {
    if (lead) {
      a.flag[0] = isfinite(rr) && isfinite(rz) ? 1 : 2;
      a.flag[1] = k;
    }
    return;
  }
  const double beta = k == 0 ? 0.0 : rz / a.scal[par ^ 1];
  if (lead) {
    a.scal[par] = rz;
    if (k == 0) a.scal[2] = rr;
  }
  const int n = a.g.n, P = a.g.pitch;
  const size_t blk = a.g.blk;
  const double *z = a.z, *po = a.p[par ^ 1];
  double *pn = a.p[par];
  // p_k at slot e (k = 0: z alone, the other slot is not read)
  auto pk = [&](size_t e) { return k == 0 ? z[e] : fma(beta, po[e], z[e]); };
  double pq = 0.0;
  for (int cc = blockIdx.x * kCgThreads + threadIdx.x; cc < n * n; cc += G * kCgThreads) {
    const int i = cc % n, j = cc / n;
    const size_t o = (size_t)j * P + i;
    double pL, pU, qL, qU;
    s_product(a.g, a.c, a.dw, a.dinv, i, j, pk, pL, pU, qL, qU);
    pn[o] = pL;
    pn[blk + o] = pU;
    a.q[o] = qL;
    a.q[blk + o] = qU;
    pq = fma(pL, qL, pq);
    pq = fma(pU, qU, pq);
  }
  pq = cg_block_sum(pq, sh);
  if (threadIdx.x == 0) a.part[4 * G + blockIdx.x] = pq;
}

__global__ void __launch_bounds__(kCgThreads) cg_update_kernel(const __grid_constant__ CgArgs a) {
  __shared__ double sh[kCgThreads / 32];
  if (cg_stopped(a.flag)) return;
  const int G = gridDim.x, k = a.k, par = k & 1;
  const double pq = cg_reduce(a.part + 4 * G, G, sh);
  const double alpha = a.scal[par] / pq;
  const int n = a.g.n, P = a.g.pitch;
  const size_t blk = a.g.blk;
  const double *p = a.p[par];
  double rz = 0.0, rr = 0.0;
  for (int cc = blockIdx.x * kCgThreads + threadIdx.x; cc < n * n; cc += G * kCgThreads) {
    const size_t o = (size_t)(cc / n) * P + cc % n;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const size_t e = t * blk + o;
      a.x[e] = fma(alpha, p[e], a.x[e]);
      const double r = fma(-alpha, a.q[e], a.r[e]);
      a.r[e] = r;
      if (a.mg) continue;
      const double z = a.minv[e] * r;
      a.z[e] = z;
      rz = fma(r, z, rz);
      rr = fma(r, r, rr);
    }
  }
  if (a.mg) return;                          // the partials come from cg_dots_kernel
  rz = cg_block_sum(rz, sh);
  rr = cg_block_sum(rr, sh);
  if (threadIdx.x == 0) {
    a.part[(0 + (par ^ 1)) * G + blockIdx.x] = rz;
    a.part[(2 + (par ^ 1)) * G + blockIdx.x] = rr;
  }
}

// Multigrid preconditioner: the partials of r . z and r . r for the next iteration (slot
// (k + 1) & 1; k = -1 before the first one).
__global__ void __launch_bounds__(kCgThreads) cg_dots_kernel(const __grid_constant__ CgArgs a) {
  __shared__ double sh[kCgThreads / 32];
  if (cg_stopped(a.flag)) return;
  const int n = a.g.n, P = a.g.pitch, G = gridDim.x, slot = (a.k + 1) & 1;
  const size_t blk = a.g.blk;
  double rz = 0.0, rr = 0.0;
  for (int cc = blockIdx.x * kCgThreads + threadIdx.x; cc < n * n; cc += G * kCgThreads) {
    const size_t o = (size_t)(cc / n) * P + cc % n;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const double r = a.r[t * blk + o];
      rz = fma(r, a.z[t * blk + o], rz);
      rr = fma(r, r, rr);
    }
  }
  rz = cg_block_sum(rz, sh);
  rr = cg_block_sum(rr, sh);
  if (threadIdx.x == 0) {
    a.part[(0 + slot) * G + blockIdx.x] = rz;
    a.part[(2 + slot) * G + blockIdx.x] = rr;
  }
}

// ---- multigrid V-cycle for S (the CG's preconditioner) ----------------------------------
// Levels of the hierarchy below the one being relaxed, each with its own rediscretised S
// (its c, (tau B_w) and (tau D_w)^{-1}).  For uniform K the Galerkin product P^T S P keeps
// c |T| and sums the two fine edges of every coarse edge (twice the rediscretised flux
// part); the rediscretised operator's smaller coarse flux over-corrects, which the
// piecewise-constant prolongation needs (measured at 512^2, K = 1: 115 CG iterations per
// pressure step against 153 with the Galerkin-scaled operators).  Weighted Jacobi smoothing (kSmgOmega D^{-1}, two
// steps before and after the coarse correction, eight from zero on the last level), P0
// restriction by summing the four child triangles and prolongation by injection (R = P^T).
// With the same smoothing before and after and R = P^T the cycle is a symmetric positive
// definite operator, as conjugate gradients needs.  Children of coarse cell (I, J): coarse L
// holds L and U of fine (2I, 2J) and L of (2I+1, 2J), (2I, 2J+1); coarse U holds L and U of
// (2I+1, 2J+1) and U of (2I+1, 2J), (2I, 2J+1).  The kernels return at once once the CG has
// stopped.
constexpr double kSmgOmega = 2.0 / 3.0;
constexpr int kSmgBottom = 8;
constexpr int kSmgVecs = 5;                  // b, xa, xb, r, e (2 blk each)

struct SOp {
  Grid g;
  double c;
  double dw[2][3];
  const double *dinv, *minv;  // minv: 1 / diag(S)
  const int *stop;
};

// xout = xin + w D^{-1} (b - S xin)   (xin == nullptr: from zero, xout = w D^{-1} b)
__global__ void __launch_bounds__(kCgThreads) s_jacobi_kernel(const __grid_constant__ SOp o, const double *b,
                                                              const double *xin, double *xout, double w) {
  if (*(volatile const int *)o.stop) return;
  const int n = o.g.n, P = o.g.pitch;
  const size_t blk = o.g.blk;
  for (int cc = blockIdx.x * kCgThreads + threadIdx.x; cc < n * n; cc += gridDim.x * kCgThreads) {
    const int i = cc % n, j = cc / n;
    const size_t e = (size_t)j * P + i;
    if (!xin) {
      xout[e] = w * o.minv[e] * b[e];
      xout[blk + e] = w * o.minv[blk + e] * b[blk + e];
      continue;
    }
    double yL, yU, qL, qU;
    s_product(o.g, o.c, o.dw, o.dinv, i, j, [&](size_t k) { return xin[k]; }, yL, yU, qL, qU);
    xout[e] = fma(w * o.minv[e], b[e] - qL, yL);
    xout[blk + e] = fma(w * o.minv[blk + e], b[blk + e] - qU, yU);
  }
}

__global__ void __launch_bounds__(kCgThreads) s_residual_kernel(const __grid_constant__ SOp o, const double *b,
                                                                const double *x, double *r) {
  if (*(volatile const int *)o.stop) return;
  const int n = o.g.n, P = o.g.pitch;
  const size_t blk = o.g.blk;
  for (int cc = blockIdx.x * kCgThreads + threadIdx.x; cc < n * n; cc += gridDim.x * kCgThreads) {
    const int i = cc % n, j = cc / n;
    const size_t e = (size_t)j * P + i;
    double yL, yU, qL, qU;
    s_product(o.g, o.c, o.dw, o.dinv, i, j, [&](size_t k) { return x[k]; }, yL, yU, qL, qU);
    r[e] = b[e] - qL;
    r[blk + e] = b[blk + e] - qU;
  }
}

// b_c = P^T r_f (one thread per coarse cell)
__global__ void __launch_bounds__(kCgThreads) s_restrict_kernel(Grid gf, Grid gc, const double *rf, double *bc,
                                                                const int *stop) {
  if (*(volatile const int *)stop) return;
  const int nc = gc.n;
  const size_t bf = gf.blk, bcb = gc.blk;
  for (int cc = blockIdx.x * kCgThreads + threadIdx.x; cc < nc * nc; cc += gridDim.x * kCgThreads) {
    const int I = cc % nc, J = cc / nc;
    const size_t f00 = (size_t)(2 * J) * gf.pitch + 2 * I, f10 = f00 + 1, f01 = f00 + gf.pitch, f11 = f01 + 1;
    const size_t c = (size_t)J * gc.pitch + I;
    bc[c] = (rf[f00] + rf[bf + f00]) + (rf[f10] + rf[f01]);
    bc[bcb + c] = (rf[f11] + rf[bf + f11]) + (rf[bf + f10] + rf[bf + f01]);
  }
}

// xout = xin + P e_c (one thread per fine cell)
__global__ void __launch_bounds__(kCgThreads) s_prolong_kernel(Grid gf, Grid gc, const double *xin,
                                                               const double *ec, double *xout, const int *stop) {
  if (*(volatile const int *)stop) return;
  const int n = gf.n;
  const size_t bf = gf.blk, bcb = gc.blk;
  for (int cc = blockIdx.x * kCgThreads + threadIdx.x; cc < n * n; cc += gridDim.x * kCgThreads) {
    const int i = cc % n, j = cc / n;
    const size_t f = (size_t)j * gf.pitch + i, c = (size_t)(j / 2) * gc.pitch + i / 2;
    const int a = i & 1, b = j & 1;
    const double eL = ec[c], eU = ec[bcb + c];
    xout[f] = xin[f] + ((a & b) ? eU : eL);              // fine L: coarse U only in the (1, 1) child
    xout[bf + f] = xin[bf + f] + ((a | b) ? eU : eL);    // fine U: coarse L only in the (0, 0) child
  }
}

// P0 index r in [0, 2 n^2) (L cells first, then U, row-major) -> slot of the two-block vector
__device__ __forceinline__ size_t s_slot(const Grid &g, int r) {
  const int nn = g.n * g.n, t = r / nn, c = r % nn;
  return (size_t)t * g.blk + (size_t)(c / g.n) * g.pitch + c % g.n;
}

// Aug = [S | I] for the dense inversion: column c of S is S applied to the unit vector e_c
// (one thread per (cell, column)).
__global__ void s_dense_kernel(const __grid_constant__ SOp o, double *Aug) {
  const int n = o.g.n, N = 2 * n * n;
  const int col = blockIdx.y;
  const size_t sc = s_slot(o.g, col), ld = 2 * (size_t)N;
  for (int cc = blockIdx.x * blockDim.x + threadIdx.x; cc < n * n; cc += gridDim.x * blockDim.x) {
    const int i = cc % n, j = cc / n;
    double yL, yU, qL, qU;
    s_product(o.g, o.c, o.dw, o.dinv, i, j, [&](size_t k) { return k == sc ? 1.0 : 0.0; }, yL, yU, qL, qU);
    Aug[(size_t)cc * ld + col] = qL;
    Aug[(size_t)(n * n + cc) * ld + col] = qU;
    Aug[(size_t)cc * ld + N + cc] = 1.0;
    Aug[(size_t)(n * n + cc) * ld + N + n * n + cc] = 1.0;
  }
}

// out = S^{-1} b from the dense inverse, one warp per row
__global__ void s_dense_solve_kernel(Grid g, const double *__restrict__ inv, const double *b, double *out,
                                     const int *stop) {
  if (*(volatile const int *)stop) return;
  const int N = 2 * g.n * g.n;
  const int lane = threadIdx.x & 31;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < N; r += (gridDim.x * blockDim.x) >> 5) {
    double acc = 0.0;
    for (int c = lane; c < N; c += 32) acc = fma(inv[(size_t)r * N + c], b[s_slot(g, c)], acc);
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, s);
    if (lane == 0) out[s_slot(g, r)] = acc;
  }
}

static SOp sop_of(const Level &L, const int *stop) {
  SOp o;
  o.g = L.g;
  o.c = L.s_c;
  for (int t = 0; t < 2; ++t)
    for (int k = 0; k < 3; ++k) o.dw[t][k] = L.c64.dw[t][k];
  o.dinv = L.dinv64;
  o.minv = L.sinv64;
  o.stop = stop;
  return o;
}

static int smg_grid(const Level &L) {
  const long long cells = (long long)L.n * L.n;
  return (int)std::min<long long>((cells + kCgThreads - 1) / kCgThreads, 4 * 152);
}

// out = M_l b on level l of `levels` (levels l .. nsmooth - 1 carry S); b and out are 2-blk
// vectors of level l, out distinct from the level's work vectors.
static int smg_vcycle(const Level *levels, int nsmooth, int l, const double *b, double *out, const int *stop,
                      cudaStream_t st) {
  const Level &L = levels[l];
  const size_t v = 2 * L.g.blk;
  double *xa = L.smg + 1 * v, *xb = L.smg + 2 * v, *r = L.smg + 3 * v;
  const SOp o = sop_of(L, stop);
  const dim3 grid(smg_grid(L)), block(kCgThreads);
  if (l + 1 >= nsmooth && L.sdense) {       // last level: its factored S
    s_dense_solve_kernel<<<dim3((2 * L.n * L.n * 32 + kCgThreads - 1) / kCgThreads), block, 0, st>>>(
        L.g, L.sdense, b, out, stop);
    BMG_CHECK_LAUNCH("s_dense_solve_kernel");
    return BMG_OK;
  }
  if (l + 1 >= nsmooth) {                   // last level: Jacobi steps from zero
    const double *xin = nullptr;
    for (int s = 0; s < kSmgBottom; ++s) {
      double *xo = s + 1 == kSmgBottom ? out : (s & 1 ? xb : xa);
      s_jacobi_kernel<<<grid, block, 0, st>>>(o, b, xin, xo, kSmgOmega);
      BMG_CHECK_LAUNCH("s_jacobi_kernel");
      xin = xo;
    }
    return BMG_OK;
  }
  const Level &C = levels[l + 1];
  const size_t vc = 2 * C.g.blk;
  double *bc = C.smg, *ec = C.smg + 4 * vc;
  s_jacobi_kernel<<<grid, block, 0, st>>>(o, b, nullptr, xa, kSmgOmega);
  BMG_CHECK_LAUNCH("s_jacobi_kernel");
  s_jacobi_kernel<<<grid, block, 0, st>>>(o, b, xa, xb, kSmgOmega);
  BMG_CHECK_LAUNCH("s_jacobi_kernel");
  s_residual_kernel<<<grid, block, 0, st>>>(o, b, xb, r);
  BMG_CHECK_LAUNCH("s_residual_kernel");
  s_restrict_kernel<<<dim3(smg_grid(C)), block, 0, st>>>(L.g, C.g, r, bc, stop);
  BMG_CHECK_LAUNCH("s_restrict_kernel");
  int rc = smg_vcycle(levels, nsmooth, l + 1, bc, ec, stop, st);
  if (rc) return rc;
  s_prolong_kernel<<<grid, block, 0, st>>>(L.g, C.g, xb, ec, xa, stop);
  BMG_CHECK_LAUNCH("s_prolong_kernel");
  s_jacobi_kernel<<<grid, block, 0, st>>>(o, b, xa, xb, kSmgOmega);
  BMG_CHECK_LAUNCH("s_jacobi_kernel");
  s_jacobi_kernel<<<grid, block, 0, st>>>(o, b, xb, out, kSmgOmega);
  BMG_CHECK_LAUNCH("s_jacobi_kernel");
  return BMG_OK;
}

// The dense inverse of S on the last smoothing level (at most kSmgDenseMax unknowns; larger
// levels keep the Jacobi bottom): S assembled column by column from the stencil and inverted
// by Gauss-Jordan with partial pivoting (the coarsest-grid kernels).
constexpr int kSmgDenseMax = 2048;

int bsr_exact_bottom_setup(Level &L, int *d_flag, cudaStream_t st) {
  const int N = 2 * L.n * L.n;
  if (N > kSmgDenseMax) return BMG_OK;
  int zero = 0;
  int *nostop = nullptr;
  double *Aug = nullptr, *fac = nullptr;
  float *inv32 = nullptr;
  BMG_CUDA(cudaMalloc(&nostop, sizeof(int)));
  BMG_CUDA(cudaMemcpyAsync(nostop, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
  BMG_CUDA(cudaMalloc(&Aug, sizeof(double) * 2 * (size_t)N * N));
  BMG_CUDA(cudaMemsetAsync(Aug, 0, sizeof(double) * 2 * (size_t)N * N, st));
  BMG_CUDA(cudaMalloc(&fac, sizeof(double) * N));
  BMG_CUDA(cudaMalloc(&inv32, sizeof(float) * (size_t)N * N));
  BMG_CUDA(cudaMalloc(&L.sdense, sizeof(double) * (size_t)N * N));
  const SOp o = sop_of(L, nostop);
  s_dense_kernel<<<dim3((L.n * L.n + 127) / 128, N), 128, 0, st>>>(o, Aug);
  BMG_CHECK_LAUNCH("s_dense_kernel");
  for (int k = 0; k < N; ++k) {
    gj_pivot_kernel<<<1, 1024, 0, st>>>(Aug, N, k, fac, 1e-300, d_flag);
    gj_eliminate_kernel<<<dim3((2 * N + 255) / 256, N), 256, 0, st>>>(Aug, N, k, fac);
  }
  g_launches += 2 * (long long)N - 1;
  BMG_CHECK_LAUNCH("gauss_jordan");
  extract_inverse_kernel<<<dim3((N + 255) / 256, N), 256, 0, st>>>(Aug, N, L.sdense, inv32);
  BMG_CHECK_LAUNCH("extract_inverse_kernel");
  BMG_CUDA(cudaStreamSynchronize(st));
  cudaFree(Aug);
  cudaFree(fac);
  cudaFree(inv32);
  cudaFree(nostop);
  return BMG_OK;
}

// Work space of the exact pressure step and 1 / diag(S) (sinv with omega_J = 1).
int bsr_exact_setup(Level &L, cudaStream_t st) {
  const size_t blk = L.g.blk;
  const long long cells = (long long)L.n * L.n;
  L.cg_grid = (int)std::min<long long>((cells + kCgThreads - 1) / kCgThreads, 4 * 152);
  const size_t len = kCgVecs * 2 * blk + 5 * (size_t)L.cg_grid + 3;
  BMG_CUDA(cudaMalloc(&L.cg, sizeof(double) * len));
  BMG_CUDA(cudaMemsetAsync(L.cg, 0, sizeof(double) * len, st));
  BMG_CUDA(cudaMalloc(&L.cg_flag, sizeof(int) * 2));
  BMG_CUDA(cudaMemsetAsync(L.cg_flag, 0, sizeof(int) * 2, st));
  BMG_CUDA(cudaMalloc(&L.smg, sizeof(double) * kSmgVecs * 2 * blk));
  BMG_CUDA(cudaMemsetAsync(L.smg, 0, sizeof(double) * kSmgVecs * 2 * blk, st));
  return BMG_OK;
}

// x <- x + omega (dy, dp) with dp = S^{-1}(B z - r_p) from conjugate gradients.  Runs kernel by
// kernel with host reads of the stop flag (not capturable into a graph).
int launch_bsr_exact_sweep(const Level *levels, int nsmooth, int l, const double *r, double *x, double omega,
                           cudaStream_t st, bool assign, int *iters_max) {
  const Level &L = levels[l];
  const bool mg = l + 1 < nsmooth;         // a coarser level with S below: multigrid preconditioner
  if (capturing(st)) {
    set_error("exact BSR reads its stop flag on the host and cannot be captured into a graph");
    return BMG_ERR_ARG;
  }
  const size_t blk = L.g.blk;
  double *z = (double *)L.bz;
  double *d = (double *)L.bd;
  int rc = launch_vanka_u<double>(L, r, z, nullptr, nullptr, omega, 0, false, st);
  if (rc) return rc;
  CgArgs c;
  c.g = L.g;
  c.c = L.s_c;
  for (int o = 0; o < 2; ++o)
    for (int k = 0; k < 3; ++k) c.dw[o][k] = L.c64.dw[o][k];
  c.dinv = L.dinv64;
  c.minv = L.sinv64;
  c.r = L.cg;
  c.z = L.cg + 2 * blk;
  c.q = L.cg + 4 * blk;
  c.p[0] = L.cg + 6 * blk;
  c.p[1] = L.cg + 8 * blk;
  c.x = d + (size_t)PL * blk;
  c.part = L.cg + kCgVecs * 2 * blk;
  c.scal = c.part + 5 * (size_t)L.cg_grid;
  c.flag = L.cg_flag;
  c.k = 0;
  c.tol2 = kCgRtol * kCgRtol;
  c.mg = mg ? 1 : 0;
  BMG_PROF_BEGIN(BMG_PROF_SCHUR, L.n, st);
  {
    DpArgs<double> a;
    a.g = L.g;
    a.z = z;
    a.r = r;
    a.d = c.r;
    a.sinv = L.sinv64;
    a.gate = L.gate;
    a.c = L.c64;
    a.raw = 1;
    dim3 b(32, 8), gr((L.n + 31) / 32, (L.n + 7) / 8);
    BMG_CUDA(launch_pdl(bsr_dp_kernel<double>, dim3(gr), dim3(b), 0, st, a));
    BMG_CHECK_LAUNCH("bsr_dp_kernel");
  }
  const dim3 grid(L.cg_grid), block(kCgThreads);
  cg_init_kernel<<<grid, block, 0, st>>>(c);
  BMG_CHECK_LAUNCH("cg_init_kernel");
  // z = M r and the partials of r . z, r . r for iteration k + 1
  auto precondition = [&](int k) -> int {
    int rc2 = smg_vcycle(levels, nsmooth, l, c.r, c.z, L.cg_flag, st);
    if (rc2) return rc2;
    c.k = k;
    cg_dots_kernel<<<grid, block, 0, st>>>(c);
    BMG_CHECK_LAUNCH("cg_dots_kernel");
    return BMG_OK;
  };
  if (mg && (rc = precondition(-1))) return rc;
  const int check = mg ? 4 : kCgCheck;
  int hflag[2] = {0, 0};
  for (int k = 0; k < kCgMaxIt; ++k) {
    c.k = k;
    cg_dir_apply_kernel<<<grid, block, 0, st>>>(c);
    BMG_CHECK_LAUNCH("cg_dir_apply_kernel");
    cg_update_kernel<<<grid, block, 0, st>>>(c);
    BMG_CHECK_LAUNCH("cg_update_kernel");
    if (mg && (rc = precondition(k))) return rc;
    if ((k + 1) % check == 0 || k + 1 == kCgMaxIt) {
      BMG_CUDA(cudaMemcpyAsync(hflag, L.cg_flag, sizeof(hflag), cudaMemcpyDeviceToHost, st));
      BMG_CUDA(cudaStreamSynchronize(st));
      if (hflag[0]) break;
    }
  }
  BMG_PROF_END(st, (double)L.n * L.n);
  if (hflag[0] == 0) {
    set_error("exact BSR: conjugate gradients on the Schur complement did not reach the tolerance");
    return BMG_ERR_NOCONV;
  }
  if (hflag[0] == 2) {
    set_error("exact BSR: non-finite residual in the Schur-complement solve");
    return BMG_ERR_NONFINITE;
  }
  if (iters_max && hflag[1] > *iters_max) *iters_max = hflag[1];
  return launch_vanka_u<double>(L, r, nullptr, x, d, omega, 1, assign, st);
}

}  // namespace bmg
