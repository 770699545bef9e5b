// Right-hand side of one backward-Euler step (Sec. 2.1, Eqs. discrete1-3).
//
// With eq. discrete3 scaled by -1, the pressure rows of step m read
//   alpha B_u u^m + tau B_w w^m - (1/M) M_p p^m = -tau (f, q) + alpha B_u u^{m-1} - (1/M) M_p p^{m-1},
// i.e. the history term is the pressure rows of A applied to (u^{m-1}, 0, p^{m-1}); the
// displacement and flux rows carry only the step's loads.  One thread per grid position
// forms the 10 entries of b there: the loads of the displacement and flux blocks, and for
// the two triangles of the cell the load plus -alpha g_T . u_T - (1/M) |T| p_T, the element
// coefficients of the system's fine level (the operator's own, so the history term is the
// same discrete B_u and M_p).  Constrained and unused slots of b are written as zero.
#include "bmg_internal.h"
#include "kernels_common.cuh"

namespace bmg {

struct HistoryArgs {
  Grid g;
  const double *x;      // previous step (u, w, p); w is not read
  const double *load;   // this step's loads
  double *b;
  double ag[2][9];      // -alpha g_T (local order of each triangle orientation)
  double pp;            // (1/M) |T|
};

__global__ void __launch_bounds__(256) backward_euler_rhs_kernel(const __grid_constant__ HistoryArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = a.g.n, P = a.g.pitch;
  const size_t blk = a.g.blk;
  if (i >= P || j > n) return;
  const size_t o = (size_t)j * P + i;
  bool m[NBLK];
  if (i <= n) {
    dof_masks(i, j, n, m);
  } else {
#pragma unroll
    for (int k = 0; k < NBLK; ++k) m[k] = false;
  }
#pragma unroll
  for (int k = 0; k < PL; ++k) a.b[k * blk + o] = m[k] ? a.load[k * blk + o] : 0.0;
  const double *x = a.x;
  for (int t = 0; t < 2; ++t) {
    double v = 0.0;
    if (m[PL + t]) {
      // local DoFs: L = v0 (i,j), v1 (i+1,j), v2 (i,j+1), edges d(i,j), v(i,j), h(i,j);
      //             U = v0 (i+1,j+1), v1 (i,j+1), v2 (i+1,j), edges d(i,j), v(i+1,j), h(i,j+1)
      const int v0i = i + t, v0j = j + t;
      const int v1i = t ? i : i + 1, v1j = t ? j + 1 : j;
      const int v2i = t ? i + 1 : i, v2j = t ? j : j + 1;
      const size_t a0 = (size_t)v0j * P + v0i, a1 = (size_t)v1j * P + v1i, a2 = (size_t)v2j * P + v2i;
      const bool f0 = vfree(v0i, v0j, n), f1 = vfree(v1i, v1j, n), f2 = vfree(v2i, v2j, n);
      const size_t ev = t ? o + 1 : o, eh = t ? o + P : o;
      const bool bvf = t ? (i + 1 < n) : (i > 0), bhf = t ? (j + 1 < n) : (j > 0);
      const double u[9] = {f0 ? x[UX * blk + a0] : 0.0, f1 ? x[UX * blk + a1] : 0.0,
                           f2 ? x[UX * blk + a2] : 0.0, f0 ? x[UY * blk + a0] : 0.0,
                           f1 ? x[UY * blk + a1] : 0.0, f2 ? x[UY * blk + a2] : 0.0,
                           x[BD * blk + o], bvf ? x[BV * blk + ev] : 0.0,
                           bhf ? x[BH * blk + eh] : 0.0};
      double s = a.load[(PL + t) * blk + o];
#pragma unroll
      for (int k = 0; k < 9; ++k) s = fma(a.ag[t][k], u[k], s);
      v = fma(-a.pp, x[(PL + t) * blk + o], s);
    }
    a.b[(PL + t) * blk + o] = v;
  }
}

}  // namespace bmg

using namespace bmg;

extern "C" int bmg_backward_euler_rhs(const bmg_system *s, const double *x_prev, const double *load,
                                      double *b, void *stream) {
  if (!s || !x_prev || !load || !b) {
    set_error("bmg_backward_euler_rhs: NULL argument");
    return BMG_ERR_ARG;
  }
  if (b == x_prev || b == load) {
    set_error("bmg_backward_euler_rhs: b may not alias x_prev or load");
    return BMG_ERR_ARG;
  }
  const Level &L = s->fine;
  HistoryArgs a;
  a.g = L.g;
  a.x = x_prev;
  a.load = load;
  a.b = b;
  for (int o = 0; o < 2; ++o)
    for (int k = 0; k < 9; ++k) a.ag[o][k] = -L.c64.alpha * L.c64.g[o][k];
  a.pp = L.c64.pp;
  dim3 block(32, 8), grid((L.g.pitch + 31) / 32, (L.n + 1 + 7) / 8);
  backward_euler_rhs_kernel<<<grid, block, 0, (cudaStream_t)stream>>>(a);
  BMG_CHECK_LAUNCH("backward_euler_rhs_kernel");
  return BMG_OK;
}
