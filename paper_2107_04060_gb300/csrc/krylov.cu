// Vector kernels of the FGMRES solver (Sec. 5.1): block-partial dot products against a
// set of basis vectors with a deterministic second-stage reduction, the Gram-Schmidt
// update, scaling, the solution update x += Z y, and precision conversion.
#include "bmg_internal.h"

namespace bmg {

template <typename T>
__global__ void fill_kernel(T *x, T v, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] = v;
}

template <typename T>
int launch_fill(T *x, T v, size_t n, cudaStream_t st) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  fill_kernel<T><<<blocks, 256, 0, st>>>(x, v, n);
  BMG_CHECK_LAUNCH("fill_kernel");
  return BMG_OK;
}
template int launch_fill<double>(double *, double, size_t, cudaStream_t);
template int launch_fill<float>(float *, float, size_t, cudaStream_t);

__global__ void d2f_kernel(const double *x, float *y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void f2d_kernel(const float *x, double *y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}
int launch_convert_d2f(const double *x, float *y, size_t n, cudaStream_t st) {
  d2f_kernel<<<152 * 8, 256, 0, st>>>(x, y, n);
  BMG_CHECK_LAUNCH("d2f_kernel");
  return BMG_OK;
}
int launch_convert_f2d(const float *x, double *y, size_t n, cudaStream_t st) {
  f2d_kernel<<<152 * 8, 256, 0, st>>>(x, y, n);
  BMG_CHECK_LAUNCH("f2d_kernel");
  return BMG_OK;
}

// partial[q * nblocks + b] = sum over block b's chunk of V_q . w   (q < k)
// partial[k * nblocks + b] = sum over the chunk of w . w
__global__ void __launch_bounds__(256) dots_kernel(const double *__restrict__ V, size_t ldv, int k,
                                                   const double *__restrict__ w, size_t n,
                                                   double *__restrict__ partial) {
  __shared__ double red[8];
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const size_t c0 = blockIdx.x * chunk;
  const size_t c1 = c0 + chunk < n ? c0 + chunk : n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q <= k; ++q) {
    const double *v = (q < k) ? V + (size_t)q * ldv : w;
    double acc = 0.0;
    for (size_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) acc = fma(v[i], w[i], acc);
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int u = 0; u < 8; ++u) t += red[u];
      partial[(size_t)q * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

__global__ void reduce_partials_kernel(const double *__restrict__ partial, int nblocks, int cnt,
                                       double *__restrict__ out) {
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
  dots_kernel<<<nblocks, 256, 0, st>>>(V, ldv, k, w, n, partial);
  BMG_CHECK_LAUNCH("dots_kernel");
  reduce_partials_kernel<<<k + 1, 256, 0, st>>>(partial, nblocks, k + 1, out);
  BMG_CHECK_LAUNCH("reduce_partials_kernel");
  return BMG_OK;
}

// w -= sum_q h[q] V_q
__global__ void update_kernel(double *__restrict__ w, const double *__restrict__ V, size_t ldv,
                              int k, const double *__restrict__ h, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double acc = w[i];
    for (int q = 0; q < k; ++q) acc = fma(-h[q], V[(size_t)q * ldv + i], acc);
    w[i] = acc;
  }
}
int launch_update(double *w, const double *V, size_t ldv, int k, const double *h, size_t n,
                  cudaStream_t st) {
  update_kernel<<<152 * 8, 256, 0, st>>>(w, V, ldv, k, h, n);
  BMG_CHECK_LAUNCH("update_kernel");
  return BMG_OK;
}

// v = w / s[0]   (s on the device; s[0] == 0 leaves v = 0)
__global__ void scale_kernel(const double *__restrict__ w, double *__restrict__ v,
                             const double *__restrict__ s, size_t n) {
  const double d = s[0] != 0.0 ? 1.0 / s[0] : 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    v[i] = w[i] * d;
}
int launch_scale(const double *w, double *v, const double *s, size_t n, cudaStream_t st) {
  scale_kernel<<<152 * 8, 256, 0, st>>>(w, v, s, n);
  BMG_CHECK_LAUNCH("scale_kernel");
  return BMG_OK;
}

// x += sum_q y[q] Z_q
__global__ void axpy_multi_kernel(double *__restrict__ x, const double *__restrict__ Z, size_t ldz,
                                  int k, const double *__restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double acc = x[i];
    for (int q = 0; q < k; ++q) acc = fma(y[q], Z[(size_t)q * ldz + i], acc);
    x[i] = acc;
  }
}
int launch_axpy_multi(double *x, const double *Z, size_t ldz, int k, const double *y, size_t n,
                      cudaStream_t st) {
  axpy_multi_kernel<<<152 * 8, 256, 0, st>>>(x, Z, ldz, k, y, n);
  BMG_CHECK_LAUNCH("axpy_multi_kernel");
  return BMG_OK;
}

}  // namespace bmg
