// Vector kernels of the FGMRES solver (Sec. 5.1): block-partial dot products against a
// set of basis vectors with a deterministic second-stage reduction, the Gram-Schmidt
// update, scaling, the solution update x += Z y, and precision conversion.
#include "bmg_internal.h"

namespace bmg {

template <typename T>
__global__ void fill_kernel(T *x, T v, size_t n, const int *gate) {
  pdl_enter();
  BMG_GATE(gate);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] = v;
}

template <typename T>
int launch_fill(T *x, T v, size_t n, cudaStream_t st, const int *gate) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  BMG_CUDA(launch_pdl(fill_kernel<T>, dim3(blocks), dim3(256), 0, st, x, v, n, gate));
  BMG_CHECK_LAUNCH("fill_kernel");
  return BMG_OK;
}
template int launch_fill<double>(double *, double, size_t, cudaStream_t, const int *);
template int launch_fill<float>(float *, float, size_t, cudaStream_t, const int *);

__global__ void d2f_kernel(const double *x, float *y, size_t n) {
  pdl_enter();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void f2d_kernel(const float *x, double *y, size_t n) {
  pdl_enter();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}
int launch_convert_d2f(const double *x, float *y, size_t n, cudaStream_t st) {
  BMG_CUDA(launch_pdl(d2f_kernel, dim3(152 * 8), dim3(256), 0, st, x, y, n));
  BMG_CHECK_LAUNCH("d2f_kernel");
  return BMG_OK;
}
int launch_convert_f2d(const float *x, double *y, size_t n, cudaStream_t st) {
  BMG_CUDA(launch_pdl(f2d_kernel, dim3(152 * 8), dim3(256), 0, st, x, y, n));
  BMG_CHECK_LAUNCH("f2d_kernel");
  return BMG_OK;
}

// partial[q * nblocks + b] = sum over block b's chunk of V_q . w   (q < k)
// partial[k * nblocks + b] = sum over the chunk of w . w
// Basis vectors are taken in groups of 8: each element of w is read once per group and the
// 8 products accumulate in registers, so 8 independent loads are in flight per element.
__global__ void __launch_bounds__(256) dots_kernel(const double *__restrict__ V, size_t ldv, int k,
                                                   const double *__restrict__ w, size_t n,
                                                   double *__restrict__ partial) {
  pdl_enter();
  constexpr int G = 8;
  __shared__ double red[G][8];
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const size_t c0 = blockIdx.x * chunk;
  const size_t c1 = c0 + chunk < n ? c0 + chunk : n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q0 = 0; q0 <= k; q0 += G) {
    const int cnt = (k + 1 - q0) < G ? (k + 1 - q0) : G;
    double acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = 0.0;
    for (size_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
      const double wi = w[i];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        if (g < cnt) {
          const int q = q0 + g;
          const double v = (q < k) ? V[(size_t)q * ldv + i] : wi;
          acc[g] = fma(v, wi, acc[g]);
        }
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      double a = acc[g];
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) a += __shfl_xor_sync(0xffffffffu, a, s);
      if (lane == 0) red[g][wid] = a;
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
      double t = 0.0;
      for (int u = 0; u < 8; ++u) t += red[threadIdx.x][u];
      partial[(size_t)(q0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

__global__ void reduce_partials_kernel(const double *__restrict__ partial, int nblocks, int cnt,
                                       double *__restrict__ out) {
  pdl_enter();
  const int q = blockIdx.x;
  if (q >= cnt) return;
  __shared__ double red[256];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) acc += partial[(size_t)q * nblocks + b];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[q] = red[0];
}

// out[0..k-1] = V_q . w, out[k] = w . w  (deterministic two-stage reduction)
int launch_dots(const double *V, size_t ldv, int k, const double *w, size_t n, double *partial,
                int nblocks, double *out, cudaStream_t st) {
  BMG_PROF_BEGIN(BMG_PROF_KRYLOV, 0, st);
  BMG_CUDA(launch_pdl(dots_kernel, dim3(nblocks), dim3(256), 0, st, V, ldv, k, w, n, partial));
  BMG_CHECK_LAUNCH("dots_kernel");
  BMG_CUDA(launch_pdl(reduce_partials_kernel, dim3(k + 1), dim3(256), 0, st, partial, nblocks, k + 1, out));
  BMG_PROF_END(st, 0.0);
  BMG_CHECK_LAUNCH("reduce_partials_kernel");
  return BMG_OK;
}

// First Gram-Schmidt pass from an FP32 copy of the basis: partial[q * nblocks + b] = sum
// over block b's chunk of V32_q . w (q < k), products and the per-thread sums in FP32 (a
// thread covers a few dozen elements), the CTA and grid sums in FP64.  The pass only has to
// remove most of w's component along the basis: the FP64 second pass that follows measures
// and removes what it left (to FP64 accuracy), and the Hessenberg column is the sum of the
// two passes' coefficients.
__global__ void __launch_bounds__(256) dots32_kernel(const float *__restrict__ V, size_t ldv, int k,
                                                     const double *__restrict__ w, size_t n,
                                                     double *__restrict__ partial) {
  pdl_enter();
  constexpr int G = 8;
  __shared__ double red[G][8];
  // groups of 4 elements per thread (16-byte loads); n and ldv are multiples of 4
  const size_t n4 = n / 4, chunk = (n4 + gridDim.x - 1) / gridDim.x;
  const size_t c0 = blockIdx.x * chunk;
  const size_t c1 = c0 + chunk < n4 ? c0 + chunk : n4;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double2 *w2 = reinterpret_cast<const double2 *>(w);
  for (int q0 = 0; q0 < k; q0 += G) {
    const int cnt = (k - q0) < G ? (k - q0) : G;
    float acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = 0.f;
    for (size_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
      const double2 wa = w2[2 * i], wb = w2[2 * i + 1];
      const float x0 = (float)wa.x, x1 = (float)wa.y, x2 = (float)wb.x, x3 = (float)wb.y;
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (g < cnt) {
          const float4 v = reinterpret_cast<const float4 *>(V + (size_t)(q0 + g) * ldv)[i];
          acc[g] = fmaf(v.x, x0, fmaf(v.y, x1, fmaf(v.z, x2, fmaf(v.w, x3, acc[g]))));
        }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      double a = (double)acc[g];
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) a += __shfl_xor_sync(0xffffffffu, a, s);
      if (lane == 0) red[g][wid] = a;
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
      double t = 0.0;
      for (int u = 0; u < 8; ++u) t += red[threadIdx.x][u];
      partial[(size_t)(q0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// out[0..k-1] = V32_q . w (first Gram-Schmidt pass, see dots32_kernel)
int launch_dots32(const float *V, size_t ldv, int k, const double *w, size_t n, double *partial,
                  int nblocks, double *out, cudaStream_t st) {
  BMG_PROF_BEGIN(BMG_PROF_KRYLOV, 0, st);
  BMG_CUDA(launch_pdl(dots32_kernel, dim3(nblocks), dim3(256), 0, st, V, ldv, k, w, n, partial));
  BMG_CHECK_LAUNCH("dots32_kernel");
  BMG_CUDA(launch_pdl(reduce_partials_kernel, dim3(k), dim3(256), 0, st, partial, nblocks, k, out));
  BMG_PROF_END(st, 0.0);
  BMG_CHECK_LAUNCH("reduce_partials_kernel");
  return BMG_OK;
}

// w -= sum_q h[q] V_q
__global__ void update_kernel(double *__restrict__ w, const double *__restrict__ V, size_t ldv,
                              int k, const double *__restrict__ h, size_t n) {
  pdl_enter();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double acc = w[i];
    for (int q = 0; q < k; ++q) acc = fma(-h[q], V[(size_t)q * ldv + i], acc);
    w[i] = acc;
  }
}
int launch_update(double *w, const double *V, size_t ldv, int k, const double *h, size_t n,
                  cudaStream_t st) {
  BMG_PROF_BEGIN(BMG_PROF_KRYLOV, 0, st);
  BMG_CUDA(launch_pdl(update_kernel, dim3(152 * 8), dim3(256), 0, st, w, V, ldv, k, h, n));
  BMG_PROF_END(st, 0.0);
  BMG_CHECK_LAUNCH("update_kernel");
  return BMG_OK;
}

// w <- w - sum_q h[q] V_q, fused with the block-partial products of the new w against the
// same basis vectors (q < k, when dots != 0) and with itself (always): one pass over V
// instead of an update pass and a reduction pass.  Each thread owns a contiguous run of
// elements; the second loop over the basis re-reads values this thread has just loaded
// (L1-resident), so V is streamed from HBM once.
__global__ void __launch_bounds__(256) update_dots_kernel(double *__restrict__ w, const double *__restrict__ V,
                                                          size_t ldv, int k, const double *__restrict__ h,
                                                          size_t n, int dots, double *__restrict__ partial) {
  pdl_enter();
  constexpr int G = 8;
  __shared__ double red[G][8];
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const size_t c0 = blockIdx.x * chunk;
  const size_t c1 = c0 + chunk < n ? c0 + chunk : n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nd = dots ? k + 1 : 1;               // products to form: V_q.w (q < k) and w.w
  for (int q0 = 0; q0 < nd; q0 += G) {
    const int cnt = (nd - q0) < G ? (nd - q0) : G;
    double acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = 0.0;
    for (size_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
      double wi;
      if (q0 == 0) {                              // first group: form and store the new w
        wi = w[i];
        for (int q = 0; q < k; ++q) wi = fma(-h[q], V[(size_t)q * ldv + i], wi);
        w[i] = wi;
      } else {
        wi = w[i];
      }
#pragma unroll
      for (int g = 0; g < G; ++g) {
        if (g < cnt) {
          const int q = dots ? q0 + g : k;
          const double v = (q < k) ? V[(size_t)q * ldv + i] : wi;
          acc[g] = fma(v, wi, acc[g]);
        }
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      double a = acc[g];
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) a += __shfl_xor_sync(0xffffffffu, a, s);
      if (lane == 0) red[g][wid] = a;
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
      double t = 0.0;
      for (int u = 0; u < 8; ++u) t += red[threadIdx.x][u];
      partial[(size_t)(q0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// out[0..k-1] = V_q . w_new, out[k] = w_new . w_new after w_new = w - V h (dots != 0);
// out[0] = w_new . w_new when dots == 0.
int launch_update_dots(double *w, const double *V, size_t ldv, int k, const double *h, size_t n,
                       int dots, double *partial, int nblocks, double *out, cudaStream_t st) {
  BMG_PROF_BEGIN(BMG_PROF_KRYLOV, 0, st);
  BMG_CUDA(launch_pdl(update_dots_kernel, dim3(nblocks), dim3(256), 0, st, w, V, ldv, k, h, n, dots, partial));
  BMG_CHECK_LAUNCH("update_dots_kernel");
  const int cnt = dots ? k + 1 : 1;
  BMG_CUDA(launch_pdl(reduce_partials_kernel, dim3(cnt), dim3(256), 0, st, partial, nblocks, cnt, out));
  BMG_PROF_END(st, 0.0);
  BMG_CHECK_LAUNCH("reduce_partials_kernel");
  return BMG_OK;
}

// v = w / s[0]   (s on the device; s[0] == 0 leaves v = 0)
__global__ void scale_kernel(const double *__restrict__ w, double *__restrict__ v,
                             const double *__restrict__ s, size_t n) {
  pdl_enter();
  const double d = s[0] != 0.0 ? 1.0 / s[0] : 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    v[i] = w[i] * d;
}
// Last Gram-Schmidt correction: w <- w - V h with the product V h formed in FP32 from the
// FP32 copy of the basis (h is the second pass's coefficient vector, of the order of the
// first pass's FP32 error, so the FP32 rounding of V h is far below FP64 rounding of w),
// fused with the block-partial sums of w.w (FP64).
__global__ void __launch_bounds__(256) correct32_norm_kernel(double *__restrict__ w, const float *__restrict__ V32,
                                                             size_t ldv, int k, const double *__restrict__ h,
                                                             size_t n, double *__restrict__ partial) {
  pdl_enter();
  __shared__ float hs[256];
  __shared__ double red[8];
  for (int q = threadIdx.x; q < k; q += blockDim.x) hs[q] = (float)h[q];
  __syncthreads();
  // groups of 4 elements per thread (16-byte loads); n and ldv are multiples of 4
  const size_t n4 = n / 4, chunk = (n4 + gridDim.x - 1) / gridDim.x;
  const size_t c0 = blockIdx.x * chunk;
  const size_t c1 = c0 + chunk < n4 ? c0 + chunk : n4;
  double2 *w2 = reinterpret_cast<double2 *>(w);
  double acc = 0.0;
  for (size_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
    float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int q = 0; q < k; ++q) {
      const float4 v = reinterpret_cast<const float4 *>(V32 + (size_t)q * ldv)[i];
      const float hq = hs[q];
      c.x = fmaf(hq, v.x, c.x); c.y = fmaf(hq, v.y, c.y);
      c.z = fmaf(hq, v.z, c.z); c.w = fmaf(hq, v.w, c.w);
    }
    double2 wa = w2[2 * i], wb = w2[2 * i + 1];
    wa.x -= (double)c.x; wa.y -= (double)c.y; wb.x -= (double)c.z; wb.y -= (double)c.w;
    w2[2 * i] = wa;
    w2[2 * i + 1] = wb;
    acc = fma(wa.x, wa.x, fma(wa.y, wa.y, fma(wb.x, wb.x, fma(wb.y, wb.y, acc))));
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int u = 0; u < 8; ++u) t += red[u];
    partial[blockIdx.x] = t;
  }
}

// out[0] = ||w_new||^2 after w_new = w - V32 h (see correct32_norm_kernel); k <= 256
int launch_correct32_norm(double *w, const float *V32, size_t ldv, int k, const double *h, size_t n,
                          double *partial, int nblocks, double *out, cudaStream_t st) {
  BMG_PROF_BEGIN(BMG_PROF_KRYLOV, 0, st);
  BMG_CUDA(launch_pdl(correct32_norm_kernel, dim3(nblocks), dim3(256), 0, st, w, V32, ldv, k, h, n, partial));
  BMG_CHECK_LAUNCH("correct32_norm_kernel");
  BMG_CUDA(launch_pdl(reduce_partials_kernel, dim3(1), dim3(256), 0, st, (const double *)partial, nblocks, 1, out));
  BMG_PROF_END(st, 0.0);
  BMG_CHECK_LAUNCH("reduce_partials_kernel");
  return BMG_OK;
}

// v = w / s[0] and its FP32 copy v32
__global__ void scale2_kernel(const double *__restrict__ w, double *__restrict__ v, float *__restrict__ v32,
                              const double *__restrict__ s, size_t n) {
  pdl_enter();
  const double d = s[0] != 0.0 ? 1.0 / s[0] : 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double x = w[i] * d;
    v[i] = x;
    v32[i] = (float)x;
  }
}
int launch_scale2(const double *w, double *v, float *v32, const double *s, size_t n, cudaStream_t st) {
  BMG_PROF_BEGIN(BMG_PROF_KRYLOV, 0, st);
  BMG_CUDA(launch_pdl(scale2_kernel, dim3(152 * 8), dim3(256), 0, st, w, v, v32, s, n));
  BMG_PROF_END(st, 0.0);
  BMG_CHECK_LAUNCH("scale2_kernel");
  return BMG_OK;
}

int launch_scale(const double *w, double *v, const double *s, size_t n, cudaStream_t st) {
  BMG_PROF_BEGIN(BMG_PROF_KRYLOV, 0, st);
  BMG_CUDA(launch_pdl(scale_kernel, dim3(152 * 8), dim3(256), 0, st, w, v, s, n));
  BMG_PROF_END(st, 0.0);
  BMG_CHECK_LAUNCH("scale_kernel");
  return BMG_OK;
}

// x += sum_q y[q] Z_q
__global__ void axpy_multi_kernel(double *__restrict__ x, const double *__restrict__ Z, size_t ldz,
                                  int k, const double *__restrict__ y, size_t n) {
  pdl_enter();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double acc = x[i];
    for (int q = 0; q < k; ++q) acc = fma(y[q], Z[(size_t)q * ldz + i], acc);
    x[i] = acc;
  }
}
int launch_axpy_multi(double *x, const double *Z, size_t ldz, int k, const double *y, size_t n,
                      cudaStream_t st) {
  BMG_PROF_BEGIN(BMG_PROF_KRYLOV, 0, st);
  BMG_CUDA(launch_pdl(axpy_multi_kernel, dim3(152 * 8), dim3(256), 0, st, x, Z, ldz, k, y, n));
  BMG_PROF_END(st, 0.0);
  BMG_CHECK_LAUNCH("axpy_multi_kernel");
  return BMG_OK;
}

}  // namespace bmg
