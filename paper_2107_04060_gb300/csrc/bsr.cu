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
template <typename T, int kQX, int kQY, int NT>
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
  }
  __syncthreads();
  const size_t ld = (size_t)a.nslots;
  for (int t = tid; t < NP * 8; t += NT) {
    const int row = t / NP, p = t % NP;
    const T *inv = a.inv + ss[p] + (size_t)(row * 8) * ld;
    const T *rl = sr + p * LD;
    T acc = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) acc = fma(inv[(size_t)c * ld], rl[c], acc);
    sx[p * LD + row] = acc;
  }
  __syncthreads();
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
    a.d[PL * blk + c00] = a.sinv[c00] * (Bz - a.r[PL * blk + c00]);
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
    a.d[PU * blk + c00] = a.sinv[blk + c00] * (Bz - a.r[PU * blk + c00]);
  }
}

template <typename T, int QX, int QY, int NT>
static void launch_vanka_u_tile(const VankaUArgs<T> &a, const Level &L, cudaStream_t st) {
  dim3 grid((L.g.pitch + QX - 2) / (QX - 1), (L.n + 1 + QY - 2) / (QY - 1));
  (void)launch_pdl(vanka_u_kernel<T, QX, QY, NT>, dim3(grid), dim3(NT), 0, st, a);
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

}  // namespace bmg
