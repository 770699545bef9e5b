// FGMRES solve whose Krylov workspace lives in a fixed device array reserved when the
// library is loaded, for callers that cannot allocate device memory while they run (see
// bmg_fgmres_solve_noalloc in include/biotmg.h).
//
// The algorithm is that of bmg_fgmres_solve with the FP64 Arnoldi: right-preconditioned
// FGMRES(m), one V-cycle of the hierarchy per iteration, classical Gram-Schmidt with one
// re-orthogonalisation pass in FP64 (here as separate product and update kernels).  The
// storage differs: the basis V, the preconditioned vectors Z, the work vectors and the
// reduction buffers are carved out of g_noalloc_scratch instead of buffers the hierarchy
// allocates on first use.
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>

#include "bmg_internal.h"

namespace bmg {
namespace {

// 8 MiB of FP64 workspace on every device that loads the library, held until exit.
constexpr size_t kNoAllocDoubles = (size_t)1 << 20;
constexpr int kNoAllocMaxRestart = 64;
constexpr int kNoAllocDotBlocks = 152 * 4;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// Device address of g_noalloc_scratch, looked up once per device.  In host code the
// symbol's name is only a host-side stand-in, never a device address.
double *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

int scratch_for_current_device(double **out) {
  int dev = 0;
  BMG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("bmg_fgmres_solve_noalloc: device ordinal out of range");
    return BMG_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    double *p = nullptr;
    BMG_CUDA(cudaGetSymbolAddress((void **)&p, g_noalloc_scratch));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return BMG_OK;
}

}  // namespace
}  // namespace bmg

using namespace bmg;

extern "C" size_t bmg_noalloc_capacity(void) { return kNoAllocDoubles; }

extern "C" int bmg_fgmres_solve_noalloc(bmg_hierarchy *h, const double *b, double *x,
                                        const bmg_krylov_opts *o, bmg_solve_info *info,
                                        void *stream) {
  auto t0 = std::chrono::steady_clock::now();
  if (!h || !b || !x || !o) {
    set_error("bmg_fgmres_solve_noalloc: NULL argument");
    return BMG_ERR_ARG;
  }
  if (b == x) {
    set_error("bmg_fgmres_solve_noalloc: x may not alias b");
    return BMG_ERR_ARG;
  }
  if (!(o->rtol > 0.0 && o->rtol < 1.0) || o->restart < 1 || o->restart > kNoAllocMaxRestart ||
      o->maxit < 0) {
    set_error("bmg_fgmres_solve_noalloc: need 0 < rtol < 1, 1 <= restart <= 64, maxit >= 0");
    return BMG_ERR_ARG;
  }
  const int m = o->restart;
  const size_t vl = vec_len_of(h->sys->n);
  const size_t need = (size_t)(2 * m + 3) * vl + (size_t)kNoAllocDotBlocks * (m + 2) + 4 * (size_t)(m + 2);
  if (need > kNoAllocDoubles) {
    set_error("bmg_fgmres_solve_noalloc: (2*restart + 3) * bmg_vector_len(n) + 612 * (restart + 2) "
              "doubles exceed the fixed workspace of " + std::to_string(kNoAllocDoubles) +
              " doubles; use a smaller restart or grid, or bmg_fgmres_solve");
    return BMG_ERR_ARG;
  }
  double *base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  double *V = base;                                  // (m + 1) vectors
  double *Z = V + (size_t)(m + 1) * vl;              // m vectors
  double *w = Z + (size_t)m * vl;
  double *r = w + vl;
  double *partial = r + vl;                          // kNoAllocDotBlocks * (m + 2)
  double *dres = partial + (size_t)kNoAllocDotBlocks * (m + 2);   // 4 (m + 2)
  double hr[3 * (kNoAllocMaxRestart + 2)];
  double H[(kNoAllocMaxRestart + 1) * kNoAllocMaxRestart];
  double cs[kNoAllocMaxRestart], sn[kNoAllocMaxRestart], g[kNoAllocMaxRestart + 1],
      y[kNoAllocMaxRestart];
  auto Hij = [&](int i, int j) -> double & { return H[(size_t)i * m + j]; };

  if (o->x0_is_zero && (rc = launch_fill<double>(x, 0.0, vl, st))) return rc;
  if ((rc = launch_dots(nullptr, vl, 0, b, vl, partial, kNoAllocDotBlocks, dres, st))) return rc;
  BMG_CUDA(cudaMemcpyAsync(hr, dres, sizeof(double), cudaMemcpyDeviceToHost, st));
  BMG_CUDA(cudaStreamSynchronize(st));
  const double bnorm = std::sqrt(hr[0]);
  bmg_solve_info inf;
  std::memset(&inf, 0, sizeof(inf));
  inf.status = BMG_MAXIT;
  if (!std::isfinite(bnorm)) {
    set_error("bmg_fgmres_solve_noalloc: right-hand side is not finite");
    return BMG_ERR_NONFINITE;
  }
  if (bnorm == 0.0) {
    if ((rc = launch_fill<double>(x, 0.0, vl, st))) return rc;
    BMG_CUDA(cudaStreamSynchronize(st));
    inf.status = BMG_CONVERGED;
    if (info) *info = inf;
    return BMG_OK;
  }
  double est = 1.0;
  double *scal = dres + 3 * (m + 2);
  for (;;) {
    if ((rc = bmg_residual(h->sys, b, x, r, stream))) return rc;
    if ((rc = launch_dots(nullptr, vl, 0, r, vl, partial, kNoAllocDotBlocks, dres, st))) return rc;
    BMG_CUDA(cudaMemcpyAsync(hr, dres, sizeof(double), cudaMemcpyDeviceToHost, st));
    BMG_CUDA(cudaStreamSynchronize(st));
    const double beta = std::sqrt(hr[0]);
    inf.relres = beta / bnorm;
    if (!std::isfinite(beta)) { inf.status = BMG_DIVERGED; break; }
    if (beta <= o->rtol * bnorm) { inf.status = BMG_CONVERGED; break; }
    if (inf.iters >= o->maxit) { inf.status = BMG_MAXIT; break; }
    if (inf.status == BMG_BREAKDOWN) break;
    inf.restarts++;
    for (int k = 0; k < (m + 1) * m; ++k) H[k] = 0.0;
    for (int k = 0; k <= m; ++k) g[k] = 0.0;
    g[0] = beta;
    BMG_CUDA(cudaMemcpyAsync(scal, &beta, sizeof(double), cudaMemcpyHostToDevice, st));
    if ((rc = launch_scale(r, V, scal, vl, st))) return rc;
    int k = 0;
    bool stop = false;
    for (int j = 0; j < m && !stop; ++j) {
      double *vj = V + (size_t)j * vl;
      double *zj = Z + (size_t)j * vl;
      if ((rc = bmg_vcycle(h, vj, zj, stream))) return rc;
      if ((rc = bmg_apply(h->sys, zj, w, stream))) return rc;
      double *d1 = dres, *d2 = dres + (m + 2), *d3 = dres + 2 * (m + 2);
      if ((rc = launch_dots(V, vl, j + 1, w, vl, partial, kNoAllocDotBlocks, d1, st))) return rc;
      if ((rc = launch_update(w, V, vl, j + 1, d1, vl, st))) return rc;
      if ((rc = launch_dots(V, vl, j + 1, w, vl, partial, kNoAllocDotBlocks, d2, st))) return rc;
      if ((rc = launch_update(w, V, vl, j + 1, d2, vl, st))) return rc;
      if ((rc = launch_dots(nullptr, vl, 0, w, vl, partial, kNoAllocDotBlocks, d3, st))) return rc;
      BMG_CUDA(cudaMemcpyAsync(hr, dres, sizeof(double) * 3 * (m + 2), cudaMemcpyDeviceToHost, st));
      BMG_CUDA(cudaStreamSynchronize(st));
      const double hn = std::sqrt(hr[2 * (m + 2)]);
      bool finite = std::isfinite(hn);
      for (int i = 0; i <= j; ++i) {
        Hij(i, j) = hr[i] + hr[(m + 2) + i];
        finite = finite && std::isfinite(Hij(i, j));
      }
      Hij(j + 1, j) = hn;
      inf.iters++;
      if (!finite) { inf.status = BMG_DIVERGED; stop = true; k = j; break; }
      if (hn > 0.0) {
        BMG_CUDA(cudaMemcpyAsync(scal, &Hij(j + 1, j), sizeof(double), cudaMemcpyHostToDevice, st));
        if ((rc = launch_scale(w, V + (size_t)(j + 1) * vl, scal, vl, st))) return rc;
      }
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
        Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
        Hij(i, j) = t;
      }
      const double den = std::hypot(Hij(j, j), Hij(j + 1, j));
      cs[j] = den > 0 ? Hij(j, j) / den : 1.0;
      sn[j] = den > 0 ? Hij(j + 1, j) / den : 0.0;
      Hij(j, j) = den;
      Hij(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      k = j + 1;
      est = std::fabs(g[j + 1]) / bnorm;
      if (std::fabs(g[j + 1]) <= o->rtol * bnorm) stop = true;
      else if (hn == 0.0) { stop = true; inf.status = BMG_BREAKDOWN; }
      if (inf.iters >= o->maxit) stop = true;
    }
    if (inf.status == BMG_DIVERGED) break;
    for (int i = k - 1; i >= 0; --i) {
      double acc = g[i];
      for (int c = i + 1; c < k; ++c) acc -= Hij(i, c) * y[c];
      y[i] = Hij(i, i) != 0.0 ? acc / Hij(i, i) : 0.0;
    }
    BMG_CUDA(cudaMemcpyAsync(dres, y, sizeof(double) * k, cudaMemcpyHostToDevice, st));
    if ((rc = launch_axpy_multi(x, Z, vl, k, dres, vl, st))) return rc;
    // the copy of y above reads host memory of this frame: wait before the next reuse
    BMG_CUDA(cudaStreamSynchronize(st));
  }
  BMG_CUDA(cudaStreamSynchronize(st));
  if (h->opts.precision == BMG_FP32) {         // a timed-out TMA wait leaves its CTA's output unset
    int flag = 0;
    BMG_CUDA(cudaMemcpy(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag & kErrTmaTimeout) {
      set_error("bmg_fgmres_solve_noalloc: a bulk-copy wait in the FP32 operator timed out");
      return BMG_ERR_CUDA;
    }
  }
  inf.relres_est = est;
  inf.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  return BMG_OK;
}
