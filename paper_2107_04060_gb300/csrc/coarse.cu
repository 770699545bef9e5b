// Direct solve on the coarsest grid (Sec. 5.1: "a direct solve on the coarse mesh").
//
// Setup: the coarse operator is applied to the unit vectors of its free DoFs in one batched
// launch of the matrix-free kernel, the columns are gathered into a dense FP64 matrix, and
// the matrix is inverted by Gauss-Jordan elimination with partial pivoting (one
// single-CTA pivot kernel and one elimination kernel per column).  Solve: z = A_c^{-1} r on
// the free DoFs, one warp per row of the explicit inverse.
#include <vector>

#include "bmg_internal.h"
#include "kernels_common.cuh"

namespace bmg {

__global__ void unit_batch_kernel(double *X, const int *free_idx, int nfree, size_t vlen) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nfree) X[(size_t)k * vlen + free_idx[k]] = 1.0;
}

__global__ void gather_dense_kernel(const double *Y, const int *free_idx, int nfree, size_t vlen,
                                    double *Aug) {
  // Aug is nfree x (2 nfree): [A | I], A[r][c] = (A e_c)[free_idx[r]]
  const int r = blockIdx.y;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < 2 * nfree; c += gridDim.x * blockDim.x) {
    double v;
    if (c < nfree) v = Y[(size_t)c * vlen + free_idx[r]];
    else v = (c - nfree == r) ? 1.0 : 0.0;
    Aug[(size_t)r * 2 * nfree + c] = v;
  }
}

// Pivot search on column k, row swap, scaling of the pivot row, elimination factors.
__global__ void __launch_bounds__(1024) gj_pivot_kernel(double *Aug, int N, int k, double *fac,
                                                        double tol, int *flag) {
  __shared__ double sval[1024];
  __shared__ int sidx[1024];
  const int tid = threadIdx.x;
  const size_t ld = 2 * (size_t)N;
  double best = -1.0;
  int bi = k;
  for (int r = k + tid; r < N; r += blockDim.x) {
    const double v = fabs(Aug[r * ld + k]);
    if (v > best) { best = v; bi = r; }
  }
  sval[tid] = best;
  sidx[tid] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) {
      if (sval[tid + s] > sval[tid] || (sval[tid + s] == sval[tid] && sidx[tid + s] < sidx[tid])) {
        sval[tid] = sval[tid + s];
        sidx[tid] = sidx[tid + s];
      }
    }
    __syncthreads();
  }
  const int piv = sidx[0];
  const double pv = sval[0];
  if (!(pv > tol)) {
    if (tid == 0) atomicOr(flag, 2);
  }
  if (piv != k) {
    for (size_t c = tid; c < ld; c += blockDim.x) {
      const double t = Aug[k * ld + c];
      Aug[k * ld + c] = Aug[piv * ld + c];
      Aug[piv * ld + c] = t;
    }
  }
  __syncthreads();
  const double d = (pv > tol) ? 1.0 / Aug[k * ld + k] : 0.0;
  __syncthreads();
  for (size_t c = tid; c < ld; c += blockDim.x) Aug[k * ld + c] *= d;
  for (int r = tid; r < N; r += blockDim.x) fac[r] = (r == k) ? 0.0 : Aug[r * ld + k];
}

__global__ void gj_eliminate_kernel(double *Aug, int N, int k, const double *fac) {
  const size_t ld = 2 * (size_t)N;
  const int r = blockIdx.y;
  const double f = fac[r];
  if (f == 0.0) return;
  for (size_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ld; c += gridDim.x * blockDim.x)
    Aug[r * ld + c] -= f * Aug[k * ld + c];
}

__global__ void extract_inverse_kernel(const double *Aug, int N, double *inv64, float *inv32) {
  const int r = blockIdx.y;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    const double v = Aug[(size_t)r * 2 * N + N + c];
    inv64[(size_t)r * N + c] = v;
    inv32[(size_t)r * N + c] = (float)v;
  }
}

int coarse_setup(Level &L, int *d_flag, cudaStream_t st) {
  const int n = L.n;
  std::vector<int> idx;
  const int P = L.g.pitch;
  const size_t blk = L.g.blk;
  for (int k = 0; k < NBLK; ++k)
    for (int j = 0; j <= n; ++j)
      for (int i = 0; i <= n; ++i) {
        const bool in_i = i < n, in_j = j < n;
        const bool vf = i > 0 && i < n && j > 0 && j < n;
        bool f = false;
        switch (k) {
          case UX: case UY: f = vf; break;
          case BH: f = in_i && j > 0 && j < n; break;
          case BV: f = in_j && i > 0 && i < n; break;
          case WH: f = in_i; break;
          case WV: f = in_j; break;
          default: f = in_i && in_j; break;
        }
        if (f) idx.push_back((int)(k * blk + (size_t)j * P + i));
      }
  const int N = (int)idx.size();
  L.nfree = N;
  const size_t vlen = vec_len_of(n);
  BMG_CUDA(cudaMalloc(&L.free_idx, sizeof(int) * N));
  BMG_CUDA(cudaMemcpyAsync(L.free_idx, idx.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  double *X = nullptr, *Y = nullptr, *Aug = nullptr, *fac = nullptr;
  BMG_CUDA(cudaMalloc(&X, sizeof(double) * vlen * N));
  BMG_CUDA(cudaMalloc(&Y, sizeof(double) * vlen * N));
  BMG_CUDA(cudaMalloc(&Aug, sizeof(double) * 2 * (size_t)N * N));
  BMG_CUDA(cudaMalloc(&fac, sizeof(double) * N));
  BMG_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * vlen * N, st));
  unit_batch_kernel<<<(N + 255) / 256, 256, 0, st>>>(X, L.free_idx, N, vlen);
  BMG_CHECK_LAUNCH("unit_batch_kernel");
  int rc = launch_apply<double>(L, X, nullptr, Y, false, N, vlen, st);
  if (rc) return rc;
  gather_dense_kernel<<<dim3((2 * N + 255) / 256, N), 256, 0, st>>>(Y, L.free_idx, N, vlen, Aug);
  BMG_CHECK_LAUNCH("gather_dense_kernel");
  for (int k = 0; k < N; ++k) {
    gj_pivot_kernel<<<1, 1024, 0, st>>>(Aug, N, k, fac, 1e-300, d_flag);
    gj_eliminate_kernel<<<dim3((2 * N + 255) / 256, N), 256, 0, st>>>(Aug, N, k, fac);
  }
  g_launches += 2 * (long long)N - 1;
  BMG_CHECK_LAUNCH("gauss_jordan");
  BMG_CUDA(cudaMalloc(&L.cinv64, sizeof(double) * (size_t)N * N));
  BMG_CUDA(cudaMalloc(&L.cinv32, sizeof(float) * (size_t)N * N));
  extract_inverse_kernel<<<dim3((N + 255) / 256, N), 256, 0, st>>>(Aug, N, L.cinv64, L.cinv32);
  BMG_CHECK_LAUNCH("extract_inverse_kernel");
  BMG_CUDA(cudaStreamSynchronize(st));
  cudaFree(X);
  cudaFree(Y);
  cudaFree(Aug);
  cudaFree(fac);
  return BMG_OK;
}

// z = A_c^{-1} r on the free DoFs (z's other slots are zeroed first by the caller).
template <typename T>
__global__ void coarse_solve_kernel(const T *__restrict__ inv, const int *__restrict__ free_idx,
                                    int N, const T *__restrict__ r, T *__restrict__ z,
                                    const int *gate) {
  pdl_enter();
  BMG_GATE(gate);
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= N) return;
  const T *row = inv + (size_t)warp * N;
  T acc = 0;
  for (int c = lane; c < N; c += 32) acc = fma(row[c], r[free_idx[c]], acc);
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  if (lane == 0) z[free_idx[warp]] = acc;
}

template <typename T>
int launch_coarse_solve(const Level &L, const T *r, T *z, cudaStream_t st) {
  int rc = launch_fill<T>(z, T(0), vec_len_of(L.n), st, L.gate);
  if (rc) return rc;
  const T *inv = (const T *)(sizeof(T) == 8 ? (const void *)L.cinv64 : (const void *)L.cinv32);
  const int threads = 256;
  const int blocks = (L.nfree * 32 + threads - 1) / threads;
  { BMG_PROF_BEGIN(BMG_PROF_COARSE, 0, st);
  BMG_CUDA(launch_pdl(coarse_solve_kernel<T>, dim3(blocks), dim3(threads), 0, st, inv, L.free_idx, L.nfree, r, z, L.gate));
    BMG_PROF_END(st, (double)L.n * L.n); }
  BMG_CHECK_LAUNCH("coarse_solve_kernel");
  return BMG_OK;
}

// Batched coarsest solve: blockIdx.y selects the instance; the CTAs of an instance first
// zero its z outside the free DoFs' rows (blockIdx.x == 0) and then form one row each per
// warp.  The free DoFs' values never come from the zeroing pass, so the two are independent.
__global__ void coarse_batch_kernel(const CoarseArgs *__restrict__ args) {
  const CoarseArgs &a = args[blockIdx.y];
  BMG_GATE(a.gate);
  if (blockIdx.x == 0) {
    for (size_t i = threadIdx.x; i < a.vl; i += blockDim.x)
      if (!a.free_mask[i]) a.z[i] = 0.0;
  }
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= a.N) return;
  const double *row = a.inv + (size_t)warp * a.N;
  double acc = 0;
  for (int c = lane; c < a.N; c += 32) acc = fma(row[c], a.r[a.free_idx[c]], acc);
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  if (lane == 0) a.z[a.free_idx[warp]] = acc;
}

int launch_coarse_batch(const CoarseArgs *d_args, int count, int max_free, cudaStream_t st) {
  if (count <= 0) return BMG_OK;
  const int threads = 256;
  dim3 grid((max_free * 32 + threads - 1) / threads, count);
  coarse_batch_kernel<<<grid, threads, 0, st>>>(d_args);
  BMG_CHECK_LAUNCH("coarse_batch_kernel");
  return BMG_OK;
}

template int launch_coarse_solve<double>(const Level &, const double *, double *, cudaStream_t);
template int launch_coarse_solve<float>(const Level &, const float *, float *, cudaStream_t);

}  // namespace bmg
