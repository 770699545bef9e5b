// Adjoint parameter gradients of a loss on the solution of A(theta, lambda, mu) x = b.
//
// With the adjoint solution xi of A xi = dL/dx (A is symmetric, Sec. 2.1), dL/dq =
// -xi^T (dA/dq) x for every parameter q.  Element-wise (Sec. 2.3 element matrices):
//   dL/dtheta_T = e^{-theta_T} xi_w,T^T (tau M_T) w_T        (theta_T = log K_T)
//   dL/dlambda  = -sum_T (g_T . xi_u,T)(g_T . u_T) / |T|
//   dL/dmu      = -sum_T xi_u,T^T (2 A_eps,T) u_T
// One thread per cell (both triangles); dL/dtheta is written per triangle, the two Lame
// sums are reduced per CTA and then across CTAs in a fixed order (deterministic).
#include <cmath>

#include "bmg_internal.h"
#include "kernels_common.cuh"

namespace bmg {

struct AdjArgs {
  Grid g;
  const double *x, *xi, *kinv;
  double M1[2][9];       // tau * unit RT0 mass
  double A2[2][81];      // 2 * A_eps
  double gd[2][9];       // int div phi
  double inv_area;
  double *dtheta;        // [2][blk]
  double *partial;       // [2][gridDim.x]
};

__device__ __forceinline__ void load_tri(const double *v, const Grid &g, int o, int ci, int cj,
                                         double u[9], double w[3]) {
  const int n = g.n, P = g.pitch;
  const size_t blk = g.blk, c00 = (size_t)cj * P + ci;
  const int v0i = ci + o, v0j = cj + o;
  const int v1i = o ? ci : ci + 1, v1j = o ? cj + 1 : cj;
  const int v2i = o ? ci + 1 : ci, v2j = o ? cj : cj + 1;
  const size_t a0 = (size_t)v0j * P + v0i, a1 = (size_t)v1j * P + v1i, a2 = (size_t)v2j * P + v2i;
  const bool f0 = vfree(v0i, v0j, n), f1 = vfree(v1i, v1j, n), f2 = vfree(v2i, v2j, n);
  const size_t ev = o ? c00 + 1 : c00, eh = o ? c00 + P : c00;
  const bool bvf = o ? (ci + 1 < n) : (ci > 0), bhf = o ? (cj + 1 < n) : (cj > 0);
  u[0] = f0 ? v[UX * blk + a0] : 0.0; u[1] = f1 ? v[UX * blk + a1] : 0.0; u[2] = f2 ? v[UX * blk + a2] : 0.0;
  u[3] = f0 ? v[UY * blk + a0] : 0.0; u[4] = f1 ? v[UY * blk + a1] : 0.0; u[5] = f2 ? v[UY * blk + a2] : 0.0;
  u[6] = v[BD * blk + c00];
  u[7] = bvf ? v[BV * blk + ev] : 0.0;
  u[8] = bhf ? v[BH * blk + eh] : 0.0;
  w[0] = v[WD * blk + c00];
  w[1] = v[WV * blk + ev];
  w[2] = v[WH * blk + eh];
}

__global__ void __launch_bounds__(256) adjoint_gradient_kernel(const __grid_constant__ AdjArgs a) {
  __shared__ double red[2][8];
  const int n = a.g.n, P = a.g.pitch;
  const size_t blk = a.g.blk;
  double sl = 0.0, sm = 0.0;
  const size_t ncell = (size_t)n * n;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < ncell; c += (size_t)gridDim.x * blockDim.x) {
    const int ci = (int)(c % n), cj = (int)(c / n);
    const size_t c00 = (size_t)cj * P + ci;
    for (int o = 0; o < 2; ++o) {
      double u[9], w[3], z[9], q[3];
      load_tri(a.x, a.g, o, ci, cj, u, w);
      load_tri(a.xi, a.g, o, ci, cj, z, q);
      double mw = 0.0;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        double t = 0.0;
#pragma unroll
        for (int s = 0; s < 3; ++s) t = fma(a.M1[o][r * 3 + s], w[s], t);
        mw = fma(q[r], t, mw);
      }
      a.dtheta[(size_t)o * blk + c00] = a.kinv[(size_t)o * blk + c00] * mw;
      double gu = 0.0, gz = 0.0;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        gu = fma(a.gd[o][k], u[k], gu);
        gz = fma(a.gd[o][k], z[k], gz);
      }
      sl -= gz * gu * a.inv_area;
      double e = 0.0;
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        double t = 0.0;
#pragma unroll
        for (int s = 0; s < 9; ++s) t = fma(a.A2[o][r * 9 + s], u[s], t);
        e = fma(z[r], t, e);
      }
      sm -= e;
    }
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    sl += __shfl_xor_sync(0xffffffffu, sl, s);
    sm += __shfl_xor_sync(0xffffffffu, sm, s);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { red[0][wid] = sl; red[1][wid] = sm; }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[threadIdx.x][k];
    a.partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void zero_theta_padding_kernel(Grid g, double *dtheta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.pitch || j > g.n) return;
  if (i < g.n && j < g.n) return;
  dtheta[(size_t)j * g.pitch + i] = 0.0;
  dtheta[g.blk + (size_t)j * g.pitch + i] = 0.0;
}

// out[q] = sum_b partial[q * nb + b], q = 0, 1 (one warp per sum, fixed order)
__global__ void adjoint_reduce_kernel(const double *partial, int nb, double *out) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double t = 0.0;
  for (int b = lane; b < nb; b += 32) t += partial[(size_t)q * nb + b];
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) t += __shfl_xor_sync(0xffffffffu, t, s);
  if (lane == 0) out[q] = t;
}

}  // namespace bmg

using namespace bmg;

extern "C" int bmg_adjoint_gradient(const bmg_system *s, const double *x, const double *xi,
                                    double *dtheta, double *dlame, void *stream) {
  if (!s || !x || !xi || !dtheta || !dlame) {
    set_error("bmg_adjoint_gradient: NULL argument");
    return BMG_ERR_ARG;
  }
  if (s->prm.exact_divdiv) {
    set_error("bmg_adjoint_gradient: the gradients are those of the reduced-quadrature system");
    return BMG_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const Level &L = s->fine;
  AdjArgs a;
  a.g = L.g;
  a.x = x;
  a.xi = xi;
  a.kinv = L.kinv64;
  ElemIntegrals e;
  element_integrals(1.0 / s->n, &e);
  for (int o = 0; o < 2; ++o) {
    for (int k = 0; k < 9; ++k) {
      a.M1[o][k] = s->prm.tau * e.Mw[o][k / 3][k % 3];
      a.gd[o][k] = e.g[o][k];
    }
    for (int k = 0; k < 81; ++k) a.A2[o][k] = 2.0 * e.Aeps[o][k / 9][k % 9];
  }
  a.inv_area = 1.0 / e.area;
  a.dtheta = dtheta;
  a.partial = s->adj_partial;
  const int nb = kAdjBlocks;
  adjoint_gradient_kernel<<<nb, 256, 0, st>>>(a);
  BMG_CHECK_LAUNCH("adjoint_gradient_kernel");
  dim3 b2(32, 8), g2((L.g.pitch + 31) / 32, (s->n + 1 + 7) / 8);
  zero_theta_padding_kernel<<<g2, b2, 0, st>>>(L.g, dtheta);
  BMG_CHECK_LAUNCH("zero_theta_padding_kernel");
  adjoint_reduce_kernel<<<1, 64, 0, st>>>(s->adj_partial, nb, dlame);
  BMG_CHECK_LAUNCH("adjoint_reduce_kernel");
  return BMG_OK;
}
