// Vector kernels of the FGMRES solver (Sec. 5.1): block-partial dot products against a
// set of basis vectors with a deterministic second-stage reduction, the Gram-Schmidt
// update, scaling, the solution update x += Z y, and precision conversion.
#include <atomic>
#include <string>

#include "bmg_internal.h"
#include "kernels_common.cuh"

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

template <typename T>
__global__ void add_kernel(T *__restrict__ y, const T *__restrict__ x, size_t n) {
  pdl_enter();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}

template <typename T>
int launch_add(T *y, const T *x, size_t n, cudaStream_t st) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  BMG_CUDA(launch_pdl(add_kernel<T>, dim3(blocks), dim3(256), 0, st, y, x, n));
  BMG_CHECK_LAUNCH("add_kernel");
  return BMG_OK;
}
template int launch_add<double>(double *, const double *, size_t, cudaStream_t);
template int launch_add<float>(float *, const float *, size_t, cudaStream_t);

__global__ void d2f_kernel(const double *x, float *y, size_t n) {
  pdl_enter();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = f64_to_f32_trunc(x[i]);
}
__global__ void f2d_kernel(const float *x, double *y, size_t n) {
  pdl_enter();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = f32_to_f64_bits(x[i]);
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

// Grid of a Gram-Schmidt kernel with blockDim (32, ty): the CTAs resident on the whole GPU
// (one wave), cached per (kernel, ty).
template <typename Kern>
static int resident_blocks(Kern kern, int ty, size_t smem, std::atomic<int> *cache) {
  int b = cache[ty].load(std::memory_order_relaxed);
  if (b > 0) return b;
  int dev = 0, nsm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * ty, smem) != cudaSuccess)
    return 0;
  b = nsm * (per_sm > 0 ? per_sm : 1);
  cache[ty].store(b, std::memory_order_relaxed);
  return b;
}

// First Gram-Schmidt pass from an FP32 copy of the basis: partial[q * gridDim.x + b] = CTA b's
// share of V32_q . w (q < k), products and per-thread sums in FP32 (a thread covers a few
// dozen elements), the warp and grid sums in FP64.  The pass only has to remove most of w's
// component along the basis: the second pass measures and removes what it left, and the
// Hessenberg column is the sum of the two passes' coefficients.
//
// Layout as gs_pass_kernel's: blockDim = (32, TY), lane x of warp y owns elements
// base + 2x, base + 2x + 1 (8-byte loads of V32, 16-byte loads of w) and the vectors
// q = y * KQ .. y * KQ + KQ - 1.  w is converted to FP32 once per element (integer
// truncation, no FP64 pipe work), and the next batch's loads are issued before the current
// batch's products so that memory latency overlaps the arithmetic.
template <int KQ>
__global__ void __launch_bounds__(32 * kDotsMaxTY) dots32_kernel(const float *__restrict__ V, size_t ldv, int k,
                                                      const double *__restrict__ w, size_t n,
                                                      double *__restrict__ partial) {
  pdl_enter();
  const int x = threadIdx.x, q0 = threadIdx.y * KQ;
  const size_t stride = (size_t)gridDim.x * 64;
  float acc[KQ];
#pragma unroll
  for (int j = 0; j < KQ; ++j) acc[j] = 0.f;
  float2 vn[KQ];
  double2 wn = make_double2(0.0, 0.0);
  auto load = [&](size_t base) {
    const size_t i = base + 2 * x;                 // n is even: i < n covers both elements
    const bool valid = i < n;
    if (valid) wn = *reinterpret_cast<const double2 *>(w + i);
#pragma unroll
    for (int j = 0; j < KQ; ++j)
      if (q0 + j < k && valid) vn[j] = *reinterpret_cast<const float2 *>(V + (size_t)(q0 + j) * ldv + i);
      else vn[j] = make_float2(0.f, 0.f);
  };
  size_t base = (size_t)blockIdx.x * 64;
  if (base < n) load(base);
  for (; base < n; base += stride) {
    float2 vc[KQ];
#pragma unroll
    for (int j = 0; j < KQ; ++j) vc[j] = vn[j];
    const bool valid = base + 2 * x < n;
    const float w0 = valid ? f64_to_f32_trunc(wn.x) : 0.f, w1 = valid ? f64_to_f32_trunc(wn.y) : 0.f;
    if (base + stride < n) load(base + stride);
#pragma unroll
    for (int j = 0; j < KQ; ++j) acc[j] = fmaf(vc[j].x, w0, fmaf(vc[j].y, w1, acc[j]));
  }
#pragma unroll
  for (int j = 0; j < KQ; ++j) {
    if (q0 + j < k) {                              // warp-uniform
      double a = (double)acc[j];
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) a += __shfl_xor_sync(0xffffffffu, a, s);
      if (x == 0) partial[(size_t)(q0 + j) * gridDim.x + blockIdx.x] = a;
    }
  }
}

// out[0..k-1] = V32_q . w (first Gram-Schmidt pass, see dots32_kernel); 1 <= k <= kDotsKQ *
// kDotsMaxTY, n even, partial holds max_blocks * k entries
int launch_dots32(const float *V, size_t ldv, int k, const double *w, size_t n, double *partial,
                  int max_blocks, double *out, cudaStream_t st) {
  if (k <= 0 || k > kDotsKQ * kDotsMaxTY || (n & 1) || (ldv & 1)) return BMG_ERR_ARG;
  static std::atomic<int> cache[kDotsMaxTY + 1];
  const int ty = (k + kDotsKQ - 1) / kDotsKQ;
  int nb = resident_blocks(dots32_kernel<kDotsKQ>, ty, 0, cache);
  if (nb <= 0) {
    set_error("dots32: occupancy query failed");
    return BMG_ERR_CUDA;
  }
  const size_t nbatch = (n + 63) / 64;
  if ((size_t)nb > nbatch) nb = (int)nbatch;
  if (nb > max_blocks) nb = max_blocks;
  BMG_PROF_BEGIN(BMG_PROF_KRYLOV, 0, st);
  BMG_CUDA(launch_pdl(dots32_kernel<kDotsKQ>, dim3(nb), dim3(32, ty), 0, st, V, ldv, k, w, n, partial));
  BMG_CHECK_LAUNCH("dots32_kernel");
  BMG_CUDA(launch_pdl(reduce_partials_kernel, dim3(k), dim3(256), 0, st, (const double *)partial, nb, k, out));
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

// One pass of classical Gram-Schmidt over the basis V_0 .. V_{k-1}, optionally preceded by the
// update of the previous pass:
//   UPD:  w <- w - sum_q h[q] V_q (FP64 basis, FP64 products: the Hessenberg coefficients must
//         describe exactly what is subtracted), written back to w;
//   then  block-partial products V_q . w (q < k) of the (updated) w.
// The products are formed either in FP64 (DF = false: plain FP64 Arnoldi, one FP64 fused
// multiply-add per element and vector) or on the FP32 pipe in double-float arithmetic (DF =
// true: each FP64 value split into a truncated FP32 head and an FP32 tail carrying the next 23
// bits, head products made exact with a fused multiply-add, running sums kept as an unevaluated
// FP32 pair by the error-free two-sum), accurate to about 2^-46 relative to the sum of the
// products' magnitudes; then the FP64 pipe does only the update's k fused multiply-adds per
// element.  V is streamed from HBM once per pass.
//
// Layout: blockDim = (32, TY).  Lane x of warp y owns element base + x and the basis vectors
// q = y * KQ .. y * KQ + KQ - 1: a warp's loads of one vector are one coalesced 256-byte
// row, each thread holds at most KQ values, and (UPD) the TY partial updates of an element
// meet in shared memory.  A warp owns its vectors' products, so no cross-warp reduction is
// needed.  The next batch's loads are issued before the current batch's arithmetic.
template <int KQ, bool DF, bool UPD>
__global__ void __launch_bounds__(32 * kUpdMaxTY) gs_pass_kernel(double *__restrict__ w, const double *__restrict__ V,
                                                                 size_t ldv, int k, const double *__restrict__ h,
                                                                 size_t n, double *__restrict__ partial) {
  pdl_enter();
  extern __shared__ double upd_smem[];
  const int TY = blockDim.y, x = threadIdx.x, y = threadIdx.y;
  double *hs = upd_smem;                       // [k]      (UPD)
  double *part = hs + k;                       // [TY][32] (UPD)
  double *wsd = part + 32 * TY;                // [32] updated w (UPD, FP64 products)
  float2 *wsh = reinterpret_cast<float2 *>(wsd);   // [32] its head and tail (UPD, DF)
  if (UPD) {
    for (int q = y * 32 + x; q < k; q += 32 * TY) hs[q] = h[q];
    __syncthreads();
  }
  const int q0 = y * KQ;
  const size_t stride = (size_t)gridDim.x * 32;
  float sh[KQ], sl[KQ];                          // DF: double-float running sums of V_q . w
  double acc[KQ];                                // FP64 running sums
#pragma unroll
  for (int j = 0; j < KQ; ++j) {
    sh[j] = sl[j] = 0.f;
    acc[j] = 0.0;
  }
  double vn[KQ];
  double wn = 0.0;
  auto load = [&](size_t base) {
    const size_t i = base + x;
    const bool valid = i < n;
    wn = ((!UPD || y == 0) && valid) ? w[i] : 0.0;
#pragma unroll
    for (int j = 0; j < KQ; ++j)
      vn[j] = (q0 + j < k && valid) ? V[(size_t)(q0 + j) * ldv + i] : 0.0;
  };
  size_t base = (size_t)blockIdx.x * 32;
  if (base < n) load(base);
  for (; base < n; base += stride) {
    double vc[KQ];
#pragma unroll
    for (int j = 0; j < KQ; ++j) vc[j] = vn[j];
    double p = wn;
    if (base + stride < n) load(base + stride);
    const size_t i = base + x;
    const bool valid = i < n;
    double wv = p;                               // the w the products are taken with
    float2 ws = make_float2(0.f, 0.f);
    if (UPD) {
#pragma unroll
      for (int j = 0; j < KQ; ++j)
        if (q0 + j < k) p = fma(-hs[q0 + j], vc[j], p);      // warp-uniform
      if (TY == 1) {
        if (valid) w[i] = p;
        wv = p;
        if (DF) split_f64(p, ws.x, ws.y);
      } else {
        part[y * 32 + x] = p;
        __syncthreads();
        if (y == 0) {
          double s = part[x];
          for (int u = 1; u < TY; ++u) s += part[u * 32 + x];
          if (valid) w[i] = s;
          if (DF) {
            float2 t;
            split_f64(s, t.x, t.y);
            wsh[x] = t;
          } else {
            wsd[x] = s;
          }
        }
        __syncthreads();
        if (DF) ws = wsh[x];
        else wv = wsd[x];
      }
    } else if (DF) {
      split_f64(p, ws.x, ws.y);
    }
#pragma unroll
    for (int j = 0; j < KQ; ++j) {
      if (q0 + j < k) {
        if (DF) {
          float vh, vl;
          split_f64(vc[j], vh, vl);
          df_dot_step(vh, vl, ws.x, ws.y, sh[j], sl[j]);
        } else {
          acc[j] = fma(vc[j], wv, acc[j]);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < KQ; ++j) {
    const int q = q0 + j;
    if (q < k) {                                 // warp-uniform
      double a = DF ? f32_to_f64_bits(sh[j]) + f32_to_f64_bits(sl[j]) : acc[j];
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) a += __shfl_xor_sync(0xffffffffu, a, s);
      if (x == 0) partial[(size_t)q * gridDim.x + blockIdx.x] = a;
    }
  }
}

static size_t gs_pass_smem(int k, int ty, bool upd) {
  return upd ? sizeof(double) * ((size_t)k + 32 * (size_t)ty + 32) : 0;
}

template <bool DF, bool UPD>
static int launch_gs_pass(double *w, const double *V, size_t ldv, int k, const double *h, size_t n,
                          double *partial, int max_blocks, double *out, cudaStream_t st, const char *what) {
  if (k <= 0 || k > kUpdKQ * kUpdMaxTY) return BMG_ERR_ARG;
  static std::atomic<int> cache[kUpdMaxTY + 1];
  const int ty = (k + kUpdKQ - 1) / kUpdKQ;
  auto kern = gs_pass_kernel<kUpdKQ, DF, UPD>;
  int nb = resident_blocks(kern, ty, gs_pass_smem(kUpdKQ * ty, ty, UPD), cache);
  if (nb <= 0) {
    set_error(std::string(what) + ": occupancy query failed");
    return BMG_ERR_CUDA;
  }
  const size_t nbatch = (n + 31) / 32;
  if ((size_t)nb > nbatch) nb = (int)nbatch;
  if (nb > max_blocks) nb = max_blocks;
  BMG_PROF_BEGIN(BMG_PROF_KRYLOV, 0, st);
  BMG_CUDA(launch_pdl(kern, dim3(nb), dim3(32, ty), gs_pass_smem(k, ty, UPD), st, w, V, ldv, k, h, n, partial));
  BMG_CHECK_LAUNCH(what);
  BMG_CUDA(launch_pdl(reduce_partials_kernel, dim3(k), dim3(256), 0, st, (const double *)partial, nb, k, out));
  BMG_PROF_END(st, 0.0);
  BMG_CHECK_LAUNCH("reduce_partials_kernel");
  return BMG_OK;
}

// out[0..k-1] = V_q . w_new (double-float products) after w_new = w - V h (FP64);
// 1 <= k <= kUpdKQ * kUpdMaxTY.  partial holds max_blocks * k entries.
int launch_update_dots_df(double *w, const double *V, size_t ldv, int k, const double *h, size_t n,
                          double *partial, int max_blocks, double *out, cudaStream_t st) {
  return launch_gs_pass<true, true>(w, V, ldv, k, h, n, partial, max_blocks, out, st, "update_dots_df");
}

// out[0..k-1] = V_q . w_new (FP64 products) after w_new = w - V h (FP64)
int launch_update_dots_f64(double *w, const double *V, size_t ldv, int k, const double *h, size_t n,
                           double *partial, int max_blocks, double *out, cudaStream_t st) {
  return launch_gs_pass<false, true>(w, V, ldv, k, h, n, partial, max_blocks, out, st, "update_dots_f64");
}

// out[0..k-1] = V_q . w (FP64 products; w is only read): the first pass of the FP64 Arnoldi
int launch_dots_f64(const double *w, const double *V, size_t ldv, int k, size_t n, double *partial,
                    int max_blocks, double *out, cudaStream_t st) {
  return launch_gs_pass<false, false>(const_cast<double *>(w), V, ldv, k, nullptr, n, partial, max_blocks,
                                      out, st, "dots_f64");
}

// v = w / s[0]   (s on the device; s[0] == 0 leaves v = 0)
__global__ void scale_kernel(const double *__restrict__ w, double *__restrict__ v,
                             const double *__restrict__ s, size_t n) {
  pdl_enter();
  const double d = s[0] != 0.0 ? 1.0 / s[0] : 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    v[i] = w[i] * d;
}
// Last Gram-Schmidt correction: w <- w - V h (h the second pass's coefficients), with the
// product V h formed in double-float arithmetic on the FP32 pipe from the FP64 basis (each
// value split into head and tail to about 2^-47 relative, the six lowest mantissa bits
// dropped; see split_f64 / df_dot_step), fused with the
// block-partial sums of w.w (FP64).  The product is accurate to about 2^-46 of
// sum_q |h_q V_q|, so what is subtracted is V h to well below FP64 rounding of w: the
// Hessenberg column h1 + h2 describes the update exactly, whatever the accuracy of the
// FP32 first pass that h2 corrects.  Two elements per thread (16-byte loads of V and w).
__global__ void __launch_bounds__(256) correct_df_norm_kernel(double *__restrict__ w, const double *__restrict__ V,
                                                              size_t ldv, int k, const double *__restrict__ h,
                                                              size_t n, double *__restrict__ partial) {
  pdl_enter();
  __shared__ float2 hs[kMaxBasisVecs];
  __shared__ double red[8];
  for (int q = threadIdx.x; q < k; q += blockDim.x) {
    float2 t;
    split_f64(h[q], t.x, t.y);
    hs[q] = t;
  }
  __syncthreads();
  const size_t n2 = n / 2;                         // n and ldv are even
  double2 *w2 = reinterpret_cast<double2 *>(w);
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    float ch0 = 0.f, cl0 = 0.f, ch1 = 0.f, cl1 = 0.f;
#pragma unroll 4
    for (int q = 0; q < k; ++q) {
      const double2 v = reinterpret_cast<const double2 *>(V + (size_t)q * ldv)[i];
      const float2 hq = hs[q];
      float vh, vl;
      split_f64(v.x, vh, vl);
      df_dot_step(hq.x, hq.y, vh, vl, ch0, cl0);
      split_f64(v.y, vh, vl);
      df_dot_step(hq.x, hq.y, vh, vl, ch1, cl1);
    }
    double2 wi = w2[i];
    wi.x -= f32_to_f64_bits(ch0) + f32_to_f64_bits(cl0);
    wi.y -= f32_to_f64_bits(ch1) + f32_to_f64_bits(cl1);
    w2[i] = wi;
    acc = fma(wi.x, wi.x, fma(wi.y, wi.y, acc));
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

// out[0] = ||w_new||^2 after w_new = w - V h (see correct_df_norm_kernel); 1 <= k <=
// kMaxBasisVecs, n and ldv even
int launch_correct_df_norm(double *w, const double *V, size_t ldv, int k, const double *h, size_t n,
                           double *partial, int nblocks, double *out, cudaStream_t st) {
  if (k <= 0 || k > kMaxBasisVecs || (n & 1) || (ldv & 1)) return BMG_ERR_ARG;
  BMG_PROF_BEGIN(BMG_PROF_KRYLOV, 0, st);
  BMG_CUDA(launch_pdl(correct_df_norm_kernel, dim3(nblocks), dim3(256), 0, st, w, V, ldv, k, h, n, partial));
  BMG_CHECK_LAUNCH("correct_df_norm_kernel");
  BMG_CUDA(launch_pdl(reduce_partials_kernel, dim3(1), dim3(256), 0, st, (const double *)partial, nblocks, 1, out));
  BMG_PROF_END(st, 0.0);
  BMG_CHECK_LAUNCH("reduce_partials_kernel");
  return BMG_OK;
}

// Last Gram-Schmidt correction of the FP64 Arnoldi: w <- w - V h (FP64 products), fused with
// the block-partial sums of w.w.  Two elements per thread (16-byte loads of V and w).
__global__ void __launch_bounds__(256) correct_f64_norm_kernel(double *__restrict__ w, const double *__restrict__ V,
                                                               size_t ldv, int k, const double *__restrict__ h,
                                                               size_t n, double *__restrict__ partial) {
  pdl_enter();
  __shared__ double hs[kMaxBasisVecs];
  __shared__ double red[8];
  for (int q = threadIdx.x; q < k; q += blockDim.x) hs[q] = h[q];
  __syncthreads();
  const size_t n2 = n / 2;                         // n and ldv are even
  double2 *w2 = reinterpret_cast<double2 *>(w);
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    double2 wi = w2[i];
#pragma unroll 4
    for (int q = 0; q < k; ++q) {
      const double2 v = reinterpret_cast<const double2 *>(V + (size_t)q * ldv)[i];
      wi.x = fma(-hs[q], v.x, wi.x);
      wi.y = fma(-hs[q], v.y, wi.y);
    }
    w2[i] = wi;
    acc = fma(wi.x, wi.x, fma(wi.y, wi.y, acc));
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

// out[0] = ||w_new||^2 after w_new = w - V h (FP64); 1 <= k <= kMaxBasisVecs, n and ldv even
int launch_correct_f64_norm(double *w, const double *V, size_t ldv, int k, const double *h, size_t n,
                            double *partial, int nblocks, double *out, cudaStream_t st) {
  if (k <= 0 || k > kMaxBasisVecs || (n & 1) || (ldv & 1)) return BMG_ERR_ARG;
  BMG_PROF_BEGIN(BMG_PROF_KRYLOV, 0, st);
  BMG_CUDA(launch_pdl(correct_f64_norm_kernel, dim3(nblocks), dim3(256), 0, st, w, V, ldv, k, h, n, partial));
  BMG_CHECK_LAUNCH("correct_f64_norm_kernel");
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
    v32[i] = f64_to_f32_trunc(x);
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
