// Batched FGMRES: many independent systems (each with its own grid size, coefficients and
// multigrid hierarchy) solved together, the whole solve being one CUDA-graph launch.
//
// Method per instance: the right-preconditioned FGMRES(m) of Sec. 5.1 with the V-cycle of
// Sec. 3 as preconditioner, CGS2 Arnoldi and a true-residual check at every restart, the
// same iteration as bmg_fgmres_solve.  Arrangement for many instances:
//  * All FGMRES state (Hessenberg matrix, Givens rotations, counters, status) lives in
//    device memory; small kernels with one thread per instance do the Givens rotations, the
//    triangular solve and the restart decisions, so no host round trip happens inside the
//    solve.  Each instance's state carries two gates: gate_iter (take an Arnoldi step this
//    trip) and gate_end (close the cycle: x += Z y, true residual, restart or stop); every
//    kernel of a trip returns at once for an instance whose gate is closed.
//  * The V-cycles of all instances are scheduled by grid size: one launch covers every
//    instance that has a level of that size (blockIdx.z selects the instance), from the
//    largest size down to the coarsest and back up.  Work items are (instance, tile) pairs
//    of one level size; vector kernels take (instance, chunk) items.
//  * The trip (cycle end + one Arnoldi step for every open instance) is captured once into
//    the body of a graph while-node; a last kernel of the body clears the loop condition
//    when no instance is active, or after a bounded number of trips.
//  * Tile shapes of the batched operator and Vanka launches are chosen per level size by
//    timing the candidates on the batch itself (autotune), else by the single-instance rule.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <vector>

#include "bmg_internal.h"
#include "kernels_common.cuh"

namespace bmg {

constexpr int kChunk = 4096;          // elements of a vector item (256 threads x 16)
constexpr int kVecThreads = 256;
constexpr int kMaxBasis = 201;        // basis vectors of one Arnoldi cycle (restart <= 200)

struct BState {
  int gate_iter;      // 1: take an Arnoldi step this trip
  int gate_end;       // 1: close the current cycle this trip
  int j;              // Arnoldi index of the step to take
  int k;              // columns of the closed cycle (x += Z[:, :k] y)
  int fresh;          // 1: V_0 = r / beta is still to be formed
  int iters, restarts, status, active, zero_x, nonfinite_b;
  double bnorm, beta, hnext, relres, est;
};

struct BInst {
  size_t vl;
  int nb, item0;      // vector items of this instance: item0 .. item0 + nb - 1
  double *B, *X, *R, *W, *V, *Z, *Q, *Zc;
  float *V32;         // FP32 copy of the basis (first Gram-Schmidt pass)
  double *partial;    // [(m + 2)][nb]
  double *d;          // [3][m + 2]: reduced products of the three Arnoldi passes
  double *H;          // [(m + 1)][m]
  double *cs, *sn, *g, *y;
  BState *s;
};

enum VecOp { OP_NORM_B = 0, OP_NORM_R, OP_CGS1, OP_CGS2, OP_CGS3 };

// ---- vector kernels over (instance, chunk) items ---------------------------------------
__global__ void __launch_bounds__(kVecThreads) batch_copyin_kernel(const BInst *__restrict__ I,
                                                                   const int *__restrict__ item_inst,
                                                                   const double *const *__restrict__ user,
                                                                   int x0_zero, int count) {
  const int q = item_inst[blockIdx.x];
  const BInst &a = I[q];
  const size_t c0 = (size_t)(blockIdx.x - a.item0) * kChunk;
  const size_t c1 = min(a.vl, c0 + kChunk);
  const double *bu = user[q], *xu = user[count + q];
  for (size_t i = c0 + threadIdx.x; i < c1; i += kVecThreads) {
    a.B[i] = bu[i];
    a.X[i] = x0_zero ? 0.0 : xu[i];
  }
}

__global__ void __launch_bounds__(kVecThreads) batch_copyout_kernel(const BInst *__restrict__ I,
                                                                    const int *__restrict__ item_inst,
                                                                    const double *const *__restrict__ user,
                                                                    int count) {
  const int q = item_inst[blockIdx.x];
  const BInst &a = I[q];
  const size_t c0 = (size_t)(blockIdx.x - a.item0) * kChunk;
  const size_t c1 = min(a.vl, c0 + kChunk);
  double *xu = const_cast<double *>(user[count + q]);
  const bool zero = a.s->zero_x != 0;
  for (size_t i = c0 + threadIdx.x; i < c1; i += kVecThreads) xu[i] = zero ? 0.0 : a.X[i];
}

// Block-partial products of one Arnoldi pass (or a norm), with the preceding update:
//   OP_NORM_B: b.b                       OP_NORM_R: r.r (gate_end)
//   OP_CGS1:   V_q.w (q <= j); also Z_j = z (gate_iter)
//   OP_CGS2:   w -= V d1 (FP64); V_q.w (q <= j), w.w
//   OP_CGS3:   w -= V d2; w.w
// With df = 0 (BMG_ARNOLDI_FP64) every product is FP64.  With df = 1 (BMG_ARNOLDI_MIXED) the
// OP_CGS1 products come from the FP32 copy of V (FP32 products and per-thread sums, FP64
// beyond), and the OP_CGS2 products and the OP_CGS3 product V d2 are formed in double-float
// arithmetic from the FP64 basis.
// Products are stored at partial[slot][chunk] (slot q for V_q.w, slot j + 1 for w.w; slot 0
// for a norm), then summed over the chunks in a fixed order by batch_reduce_kernel.
__global__ void __launch_bounds__(kVecThreads) batch_vec_kernel(const BInst *__restrict__ I,
                                                                const int *__restrict__ item_inst,
                                                                int op, int m, int df) {
  constexpr int G = 8;
  __shared__ double red[G][kVecThreads / 32];
  const int q = item_inst[blockIdx.x];
  const BInst &a = I[q];
  const BState &s = *a.s;
  if (op == OP_NORM_R ? !s.gate_end : (op >= OP_CGS1 && !s.gate_iter)) return;
  const int chunk = blockIdx.x - a.item0;
  const size_t c0 = (size_t)chunk * kChunk;
  const size_t c1 = min(a.vl, c0 + kChunk);
  const size_t vl = a.vl;
  const int k = s.j + 1;                           // basis vectors V_0 .. V_j
  const bool vdots = op == OP_CGS1 || op == OP_CGS2;
  const bool update = op == OP_CGS2 || op == OP_CGS3;
  const double *h = op == OP_CGS2 ? a.d : a.d + (m + 2);
  double *w = op == OP_NORM_B ? a.B : op == OP_NORM_R ? a.R : a.W;
  double *zj = a.Z + (size_t)s.j * vl;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (op == OP_CGS1 && !df) {
    for (int q0 = 0; q0 < k; q0 += G) {
      const int cnt = min(G, k - q0);
      double acc[G];
#pragma unroll
      for (int gi = 0; gi < G; ++gi) acc[gi] = 0.0;
      for (size_t i = c0 + threadIdx.x; i < c1; i += kVecThreads) {
        const double wi = w[i];
        if (q0 == 0) zj[i] = a.Zc[i];
#pragma unroll
        for (int gi = 0; gi < G; ++gi)
          if (gi < cnt) acc[gi] = fma(a.V[(size_t)(q0 + gi) * vl + i], wi, acc[gi]);
      }
#pragma unroll
      for (int gi = 0; gi < G; ++gi) {
        double t = acc[gi];
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) t += __shfl_xor_sync(0xffffffffu, t, sh);
        if (lane == 0) red[gi][wid] = t;
      }
      __syncthreads();
      if (threadIdx.x < cnt) {
        double t = 0.0;
        for (int u = 0; u < kVecThreads / 32; ++u) t += red[threadIdx.x][u];
        a.partial[(size_t)(q0 + threadIdx.x) * a.nb + chunk] = t;
      }
      __syncthreads();
    }
    return;
  }
  if (op == OP_CGS1) {
    const float *V32 = a.V32;
    for (int q0 = 0; q0 < k; q0 += G) {
      const int cnt = min(G, k - q0);
      float acc[G];
#pragma unroll
      for (int gi = 0; gi < G; ++gi) acc[gi] = 0.f;
      for (size_t i = c0 + threadIdx.x; i < c1; i += kVecThreads) {
        const float wi = f64_to_f32_trunc(w[i]);
        if (q0 == 0) zj[i] = a.Zc[i];
#pragma unroll
        for (int gi = 0; gi < G; ++gi)
          if (gi < cnt) acc[gi] = fmaf(V32[(size_t)(q0 + gi) * vl + i], wi, acc[gi]);
      }
#pragma unroll
      for (int gi = 0; gi < G; ++gi) {
        double t = (double)acc[gi];
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) t += __shfl_xor_sync(0xffffffffu, t, sh);
        if (lane == 0) red[gi][wid] = t;
      }
      __syncthreads();
      if (threadIdx.x < cnt) {
        double t = 0.0;
        for (int u = 0; u < kVecThreads / 32; ++u) t += red[threadIdx.x][u];
        a.partial[(size_t)(q0 + threadIdx.x) * a.nb + chunk] = t;
      }
      __syncthreads();
    }
    return;
  }
  __shared__ float2 hf[kMaxBasis];                 // OP_CGS3: the coefficients, head and tail
  if (op == OP_CGS3 && df) {
    for (int p = threadIdx.x; p < k; p += kVecThreads) {
      float2 t;
      split_f64(h[p], t.x, t.y);
      hf[p] = t;
    }
    __syncthreads();
  }
  const int nd = vdots ? k + 1 : 1;
  for (int q0 = 0; q0 < nd; q0 += G) {
    const int cnt = min(G, nd - q0);
    float sh[G], sl[G];                            // V_q.w: double-float sums (df)
    double acc[G];                                 // V_q.w: FP64 sums (!df)
    double accw = 0.0;                             // w.w in FP64
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
      sh[gi] = sl[gi] = 0.f;
      acc[gi] = 0.0;
    }
    for (size_t i = c0 + threadIdx.x; i < c1; i += kVecThreads) {
      double wi = w[i];
      if (q0 == 0) {
        if (op == OP_CGS3 && df) {
          float ch = 0.f, cl = 0.f;
          for (int p = 0; p < k; ++p) {
            float vh, vt;
            split_f64(a.V[(size_t)p * vl + i], vh, vt);
            df_dot_step(hf[p].x, hf[p].y, vh, vt, ch, cl);
          }
          wi -= f32_to_f64_bits(ch) + f32_to_f64_bits(cl);
          w[i] = wi;
        } else if (update) {
          for (int p = 0; p < k; ++p) wi = fma(-h[p], a.V[(size_t)p * vl + i], wi);
          w[i] = wi;
        }
      }
      float wh = 0.f, wl = 0.f;
      if (vdots && df) split_f64(wi, wh, wl);
#pragma unroll
      for (int gi = 0; gi < G; ++gi) {
        if (gi < cnt) {
          const int p = vdots ? q0 + gi : k;
          if (p < k) {
            if (df) {
              float vh, vt;
              split_f64(a.V[(size_t)p * vl + i], vh, vt);
              df_dot_step(vh, vt, wh, wl, sh[gi], sl[gi]);
            } else {
              acc[gi] = fma(a.V[(size_t)p * vl + i], wi, acc[gi]);
            }
          } else {
            accw = fma(wi, wi, accw);
          }
        }
      }
    }
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
      const int p = vdots ? q0 + gi : k;
      double t = p < k ? (df ? f32_to_f64_bits(sh[gi]) + f32_to_f64_bits(sl[gi]) : acc[gi]) : accw;
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) t += __shfl_xor_sync(0xffffffffu, t, sh);
      if (lane == 0) red[gi][wid] = t;
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
      double t = 0.0;
      for (int u = 0; u < kVecThreads / 32; ++u) t += red[threadIdx.x][u];
      a.partial[(size_t)(q0 + threadIdx.x) * a.nb + chunk] = t;
    }
    __syncthreads();
  }
}

// d[set][slot] = sum over the instance's chunks (fixed order); blockIdx = (slot, instance)
__global__ void __launch_bounds__(128) batch_reduce_kernel(const BInst *__restrict__ I, int op, int m) {
  const BInst &a = I[blockIdx.y];
  const BState &s = *a.s;
  if (op == OP_NORM_R ? !s.gate_end : (op >= OP_CGS1 && !s.gate_iter)) return;
  const int nd = op == OP_CGS1 ? s.j + 1 : op == OP_CGS2 ? s.j + 2 : 1;
  const int slot = blockIdx.x;
  if (slot >= nd) return;
  __shared__ double red[128];
  double t = 0.0;
  for (int b = threadIdx.x; b < a.nb; b += 128) t += a.partial[(size_t)slot * a.nb + b];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int sh = 64; sh > 0; sh >>= 1) {
    if (threadIdx.x < sh) red[threadIdx.x] += red[threadIdx.x + sh];
    __syncthreads();
  }
  const int set = op == OP_CGS2 ? 1 : op == OP_CGS3 ? 2 : 0;
  if (threadIdx.x == 0) a.d[(size_t)set * (m + 2) + slot] = red[0];
}

// x += Z[:, :k] y (gate_end)
__global__ void __launch_bounds__(kVecThreads) batch_axpy_kernel(const BInst *__restrict__ I,
                                                                 const int *__restrict__ item_inst) {
  const int q = item_inst[blockIdx.x];
  const BInst &a = I[q];
  const BState &s = *a.s;
  if (!s.gate_end) return;
  const int k = s.k;
  const size_t c0 = (size_t)(blockIdx.x - a.item0) * kChunk;
  const size_t c1 = min(a.vl, c0 + kChunk);
  for (size_t i = c0 + threadIdx.x; i < c1; i += kVecThreads) {
    double acc = a.X[i];
    for (int p = 0; p < k; ++p) acc = fma(a.y[p], a.Z[(size_t)p * a.vl + i], acc);
    a.X[i] = acc;
  }
}

// New basis vector and V-cycle input (gate_iter): V_j = (fresh ? r / beta : w / h_{j,j-1}),
// Q = V_j.
__global__ void __launch_bounds__(kVecThreads) batch_basis_kernel(const BInst *__restrict__ I,
                                                                  const int *__restrict__ item_inst) {
  const int q = item_inst[blockIdx.x];
  const BInst &a = I[q];
  const BState &s = *a.s;
  if (!s.gate_iter) return;
  const double *src = s.fresh ? a.R : a.W;
  const double den = s.fresh ? s.beta : s.hnext;
  const double dinv = den != 0.0 ? 1.0 / den : 0.0;
  double *vj = a.V + (size_t)s.j * a.vl;
  float *vj32 = a.V32 ? a.V32 + (size_t)s.j * a.vl : nullptr;
  const size_t c0 = (size_t)(blockIdx.x - a.item0) * kChunk;
  const size_t c1 = min(a.vl, c0 + kChunk);
  for (size_t i = c0 + threadIdx.x; i < c1; i += kVecThreads) {
    const double v = src[i] * dinv;
    vj[i] = v;
    if (vj32) vj32[i] = f64_to_f32_trunc(v);
    a.Q[i] = v;
  }
}

// ---- per-instance control (one thread per instance) ------------------------------------
__global__ void batch_init_kernel(const BInst *__restrict__ I, int count, int *trips) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q == 0) *trips = 0;
  if (q >= count) return;
  BState &s = *I[q].s;
  const double bn = sqrt(I[q].d[0]);
  s.bnorm = bn;
  s.gate_iter = 0;
  s.gate_end = 0;
  s.j = s.k = s.fresh = 0;
  s.iters = s.restarts = 0;
  s.status = BMG_MAXIT;
  s.active = 0;
  s.zero_x = 0;
  s.nonfinite_b = 0;
  s.beta = s.hnext = 0.0;
  s.relres = 0.0;
  s.est = 1.0;
  if (!isfinite(bn)) {
    s.nonfinite_b = 1;
    s.status = BMG_DIVERGED;
    s.relres = bn;
  } else if (bn == 0.0) {
    s.zero_x = 1;
    s.status = BMG_CONVERGED;
  } else {
    s.active = 1;
    s.gate_end = 1;                 // first trip: r = b - A x0, then the first cycle
  }
}

// y = H[:k, :k]^{-1} g (gate_end)
__global__ void batch_solve_y_kernel(const BInst *__restrict__ I, int count, int m) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const BInst &a = I[q];
  const BState &s = *a.s;
  if (!s.gate_end) return;
  const int k = s.k;
  for (int i = k - 1; i >= 0; --i) {
    double acc = a.g[i];
    for (int c = i + 1; c < k; ++c) acc -= a.H[(size_t)i * m + c] * a.y[c];
    const double hii = a.H[(size_t)i * m + i];
    a.y[i] = hii != 0.0 ? acc / hii : 0.0;
  }
}

// Cycle end after the true residual (gate_end): stop or restart with V_0 = r / beta.
__global__ void batch_restart_kernel(const BInst *__restrict__ I, int count, double rtol, int maxit) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const BInst &a = I[q];
  BState &s = *a.s;
  if (!s.gate_end) return;
  s.gate_end = 0;
  const double beta = sqrt(a.d[0]);
  s.relres = beta / s.bnorm;
  bool stop = true;
  if (!isfinite(beta)) s.status = BMG_DIVERGED;
  else if (beta <= rtol * s.bnorm) s.status = BMG_CONVERGED;
  else if (s.iters >= maxit) s.status = BMG_MAXIT;
  else if (s.status == BMG_BREAKDOWN) {
  } else stop = false;
  if (stop) {
    s.active = 0;
    return;
  }
  s.restarts++;
  s.beta = beta;
  a.g[0] = beta;
  s.j = 0;
  s.fresh = 1;
  s.gate_iter = 1;
}

// Arnoldi column j after the three CGS2 passes (gate_iter): Hessenberg entries, Givens
// rotations, residual estimate and the decision to continue or close the cycle.
__global__ void batch_givens_kernel(const BInst *__restrict__ I, int count, double rtol, int maxit,
                                    int m) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const BInst &a = I[q];
  BState &s = *a.s;
  if (!s.gate_iter) return;
  const int j = s.j;
  const double *d1 = a.d, *d2 = a.d + (m + 2), *d3 = a.d + 2 * (m + 2);
  double *H = a.H;
  auto h = [&](int r, int c) -> double & { return H[(size_t)r * m + c]; };
  const double hn = sqrt(d3[0]);
  bool finite = isfinite(hn);
  for (int i = 0; i <= j; ++i) {
    h(i, j) = d1[i] + d2[i];
    finite = finite && isfinite(h(i, j));
  }
  h(j + 1, j) = hn;
  s.iters++;
  s.fresh = 0;
  if (!finite) {
    s.status = BMG_DIVERGED;
    s.gate_iter = 0;
    s.active = 0;
    return;
  }
  for (int i = 0; i < j; ++i) {
    const double t = a.cs[i] * h(i, j) + a.sn[i] * h(i + 1, j);
    h(i + 1, j) = -a.sn[i] * h(i, j) + a.cs[i] * h(i + 1, j);
    h(i, j) = t;
  }
  const double den = hypot(h(j, j), h(j + 1, j));
  a.cs[j] = den > 0 ? h(j, j) / den : 1.0;
  a.sn[j] = den > 0 ? h(j + 1, j) / den : 0.0;
  h(j, j) = den;
  h(j + 1, j) = 0.0;
  a.g[j + 1] = -a.sn[j] * a.g[j];
  a.g[j] = a.cs[j] * a.g[j];
  s.k = j + 1;
  s.est = fabs(a.g[j + 1]) / s.bnorm;
  bool stop = false;
  if (fabs(a.g[j + 1]) <= rtol * s.bnorm) stop = true;
  else if (hn == 0.0) {
    stop = true;
    s.status = BMG_BREAKDOWN;
  }
  if (s.iters >= maxit) stop = true;
  if (j + 1 == m) stop = true;
  if (stop) {
    s.gate_iter = 0;
    s.gate_end = 1;
  } else {
    s.j = j + 1;
    s.hnext = hn;
  }
}

// Loop control: clear the while-node condition when no instance is active or after
// max_trips trips (every trip of an active instance takes an Arnoldi step or ends it, so
// max_trips = maxit + 2 is never the binding limit of a correct solve).
__global__ void __launch_bounds__(256) batch_check_kernel(const BInst *__restrict__ I, int count,
                                                          int *trips, int max_trips,
                                                          cudaGraphConditionalHandle handle) {
  int any = 0;
  for (int q = threadIdx.x; q < count; q += blockDim.x) any |= I[q].s->active;
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    const int t = *trips + 1;
    *trips = t;
    if (!any || t >= max_trips) cudaGraphSetConditional(handle, 0);
  }
}

}  // namespace bmg

using namespace bmg;

// ---- batch object -----------------------------------------------------------------------
struct bmg_batch {
  int count = 0, m = 0, maxit = 0, x0_zero = 1;
  int df = 0;                           // 1: mixed Arnoldi (BMG_ARNOLDI_MIXED)
  double rtol = 0.0;
  std::vector<bmg_hierarchy *> hs;
  std::vector<size_t> vl;
  int total_items = 0;
  // device memory
  BInst *d_inst = nullptr;
  BState *d_state = nullptr;
  int *d_item_inst = nullptr;
  int *d_trips = nullptr;
  double **d_user = nullptr;            // [2][count]: b pointers, then x pointers
  unsigned char *d_args = nullptr;      // arguments of the batched level launches
  std::vector<double *> bufs;           // per-instance allocations
  std::vector<float *> fbufs;
  std::vector<unsigned char *> masks;   // coarsest-level free masks
  // host staging (pinned)
  double **h_user = nullptr;
  BState *h_state = nullptr;
  int *h_trips = nullptr;
  // schedule
  struct Launch {
    int kind;            // 0 apply, 1 vanka, 2 restrict, 3 prolong, 4 coarse
    int n, count, tile;
    size_t off;          // byte offset of the argument array in d_args
    int max_free;
  };
  std::vector<Launch> vcycle, resid, wapply;
  std::map<std::pair<int, int>, int> tiles;   // (kind, n) -> tile
  // graph
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long kernels_pro = 0, kernels_body = 0, kernels_epi = 0;
  int last_trips = 0;
};

static int batch_error(const std::string &msg) {
  set_error(msg);
  return BMG_ERR_ARG;
}

static int run_launch(bmg_batch *bt, const bmg_batch::Launch &L, cudaStream_t st) {
  const void *args = bt->d_args + L.off;
  switch (L.kind) {
    case 0: return launch_apply_batch(args, L.count, L.n, bt->tiles[{0, L.n}], st);
    case 1: return launch_vanka_batch(args, L.count, L.n, bt->tiles[{1, L.n}], st);
    case 2: return launch_restrict_batch((const TransferArgs *)args, L.count, L.n, st);
    case 3: return launch_prolong_batch((const TransferArgs *)args, L.count, L.n, st);
    default: return launch_coarse_batch((const CoarseArgs *)args, L.count, L.max_free, st);
  }
}

// Kernels of one trip (captured into the while-node body).
static int record_trip(bmg_batch *bt, cudaStream_t st, cudaGraphConditionalHandle handle) {
  const int C = bt->count, m = bt->m, items = bt->total_items;
  const int tb = 128, cb = (C + tb - 1) / tb;
  int rc;
  // cycle end: x += Z y, r = b - A x, ||r||, restart decision
  batch_solve_y_kernel<<<cb, tb, 0, st>>>(bt->d_inst, C, m);
  BMG_CHECK_LAUNCH("batch_solve_y_kernel");
  batch_axpy_kernel<<<items, kVecThreads, 0, st>>>(bt->d_inst, bt->d_item_inst);
  BMG_CHECK_LAUNCH("batch_axpy_kernel");
  for (const auto &L : bt->resid)
    if ((rc = run_launch(bt, L, st))) return rc;
  batch_vec_kernel<<<items, kVecThreads, 0, st>>>(bt->d_inst, bt->d_item_inst, OP_NORM_R, m, bt->df);
  BMG_CHECK_LAUNCH("batch_vec_kernel");
  batch_reduce_kernel<<<dim3(1, C), 128, 0, st>>>(bt->d_inst, OP_NORM_R, m);
  BMG_CHECK_LAUNCH("batch_reduce_kernel");
  batch_restart_kernel<<<cb, tb, 0, st>>>(bt->d_inst, C, bt->rtol, bt->maxit);
  BMG_CHECK_LAUNCH("batch_restart_kernel");
  // Arnoldi step: V_j, z = M^{-1} V_j, w = A z, CGS2, Givens
  batch_basis_kernel<<<items, kVecThreads, 0, st>>>(bt->d_inst, bt->d_item_inst);
  BMG_CHECK_LAUNCH("batch_basis_kernel");
  for (const auto &L : bt->vcycle)
    if ((rc = run_launch(bt, L, st))) return rc;
  for (const auto &L : bt->wapply)
    if ((rc = run_launch(bt, L, st))) return rc;
  for (int op = OP_CGS1; op <= OP_CGS3; ++op) {
    batch_vec_kernel<<<items, kVecThreads, 0, st>>>(bt->d_inst, bt->d_item_inst, op, m, bt->df);
    BMG_CHECK_LAUNCH("batch_vec_kernel");
    batch_reduce_kernel<<<dim3(op == OP_CGS3 ? 1 : m + 1, C), 128, 0, st>>>(bt->d_inst, op, m);
    BMG_CHECK_LAUNCH("batch_reduce_kernel");
  }
  batch_givens_kernel<<<cb, tb, 0, st>>>(bt->d_inst, C, bt->rtol, bt->maxit, m);
  BMG_CHECK_LAUNCH("batch_givens_kernel");
  batch_check_kernel<<<1, 256, 0, st>>>(bt->d_inst, C, bt->d_trips, std::min(bt->maxit, 1 << 30) + 2, handle);
  BMG_CHECK_LAUNCH("batch_check_kernel");
  return BMG_OK;
}

static int record_prologue(bmg_batch *bt, cudaStream_t st) {
  const int C = bt->count, items = bt->total_items;
  batch_copyin_kernel<<<items, kVecThreads, 0, st>>>(bt->d_inst, bt->d_item_inst,
                                                     (const double *const *)bt->d_user, bt->x0_zero, C);
  BMG_CHECK_LAUNCH("batch_copyin_kernel");
  batch_vec_kernel<<<items, kVecThreads, 0, st>>>(bt->d_inst, bt->d_item_inst, OP_NORM_B, bt->m, bt->df);
  BMG_CHECK_LAUNCH("batch_vec_kernel");
  batch_reduce_kernel<<<dim3(1, C), 128, 0, st>>>(bt->d_inst, OP_NORM_B, bt->m);
  BMG_CHECK_LAUNCH("batch_reduce_kernel");
  batch_init_kernel<<<(C + 127) / 128, 128, 0, st>>>(bt->d_inst, C, bt->d_trips);
  BMG_CHECK_LAUNCH("batch_init_kernel");
  return BMG_OK;
}

static int record_epilogue(bmg_batch *bt, cudaStream_t st) {
  batch_copyout_kernel<<<bt->total_items, kVecThreads, 0, st>>>(bt->d_inst, bt->d_item_inst,
                                                                (const double *const *)bt->d_user, bt->count);
  BMG_CHECK_LAUNCH("batch_copyout_kernel");
  return BMG_OK;
}

// Capture one recording into a fresh graph; counts the kernels it launches.
template <typename F>
static int capture(bmg_batch *bt, cudaGraph_t *out, long long *kernels, F &&rec) {
  BMG_CUDA(cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeThreadLocal));
  const long long k0 = g_launches;
  int rc = rec(bt->cap);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(bt->cap, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  *kernels = g_launches - k0;
  *out = g;
  return BMG_OK;
}

static int build_graph(bmg_batch *bt) {
  cudaGraph_t gpro = nullptr, gepi = nullptr;
  int rc = capture(bt, &gpro, &bt->kernels_pro, [&](cudaStream_t s) { return record_prologue(bt, s); });
  if (rc) return rc;
  rc = capture(bt, &gepi, &bt->kernels_epi, [&](cudaStream_t s) { return record_epilogue(bt, s); });
  if (rc) {
    cudaGraphDestroy(gpro);
    return rc;
  }
  cudaGraph_t top = nullptr;
  auto done = [&](int r) {
    cudaGraphDestroy(gpro);
    cudaGraphDestroy(gepi);
    if (r && top) cudaGraphDestroy(top);
    return r;
  };
  cudaError_t e = cudaGraphCreate(&top, 0);
  if (e != cudaSuccess) return done(cuda_fail(e, "cudaGraphCreate"));
  cudaGraphNode_t npro, nloop, nepi;
  if ((e = cudaGraphAddChildGraphNode(&npro, top, nullptr, 0, gpro)) != cudaSuccess)
    return done(cuda_fail(e, "cudaGraphAddChildGraphNode"));
  cudaGraphConditionalHandle handle;
  if ((e = cudaGraphConditionalHandleCreate(&handle, top, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
    return done(cuda_fail(e, "cudaGraphConditionalHandleCreate"));
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if ((e = cudaGraphAddNode(&nloop, top, &npro, nullptr, 1, &cp)) != cudaSuccess)
    return done(cuda_fail(e, "cudaGraphAddNode (while)"));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(bt->cap, body, nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return done(cuda_fail(e, "cudaStreamBeginCaptureToGraph"));
  const long long k0 = g_launches;
  rc = record_trip(bt, bt->cap, handle);
  cudaGraph_t body_out = nullptr;
  e = cudaStreamEndCapture(bt->cap, &body_out);
  if (rc) return done(rc);
  if (e != cudaSuccess) return done(cuda_fail(e, "cudaStreamEndCapture (body)"));
  bt->kernels_body = g_launches - k0;
  if ((e = cudaGraphAddChildGraphNode(&nepi, top, &nloop, 1, gepi)) != cudaSuccess)
    return done(cuda_fail(e, "cudaGraphAddChildGraphNode"));
  if ((e = cudaGraphInstantiate(&bt->exec, top, 0)) != cudaSuccess)
    return done(cuda_fail(e, "cudaGraphInstantiate"));
  bt->graph = top;
  g_launches -= bt->kernels_pro + bt->kernels_body + bt->kernels_epi;   // recorded, not run
  return done(BMG_OK);
}

// Time the candidate tiles of every (kernel, size) on the batch's own launches.
static int autotune(bmg_batch *bt, cudaStream_t st) {
  // open every gate so that the timed launches do their work
  std::vector<BState> open(bt->count);
  std::memset(open.data(), 0, sizeof(BState) * open.size());
  for (auto &s : open) s.gate_iter = s.gate_end = 1;
  BMG_CUDA(cudaMemcpyAsync(bt->d_state, open.data(), sizeof(BState) * open.size(), cudaMemcpyHostToDevice, st));
  cudaEvent_t e0, e1;
  BMG_CUDA(cudaEventCreate(&e0));
  BMG_CUDA(cudaEventCreate(&e1));
  int rc = BMG_OK;
  std::set<std::pair<int, int>> seen;
  for (const auto &L : bt->vcycle) {
    if (L.kind > 1 || !seen.insert({L.kind, L.n}).second) continue;
    const int ntile = L.kind == 0 ? kApplyTiles : kVankaTiles;
    float best = 1e30f;
    int best_t = bt->tiles[{L.kind, L.n}];
    for (int t = 0; t < ntile && !rc; ++t) {
      bt->tiles[{L.kind, L.n}] = t;
      float tmin = 1e30f;
      for (int rep = 0; rep < 4 && !rc; ++rep) {
        cudaEventRecord(e0, st);
        rc = run_launch(bt, L, st);
        cudaEventRecord(e1, st);
        if (rc) break;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { rc = cuda_fail(e, "autotune"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tmin = std::min(tmin, ms);      // first run warms up
      }
      if (tmin < best) {
        best = tmin;
        best_t = t;
      }
    }
    bt->tiles[{L.kind, L.n}] = best_t;
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

extern "C" void bmg_batch_destroy(bmg_batch *bt) {
  if (!bt) return;
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  if (bt->cap) cudaStreamDestroy(bt->cap);
  for (double *p : bt->bufs) cudaFree(p);
  for (float *p : bt->fbufs) cudaFree(p);
  for (unsigned char *p : bt->masks) cudaFree(p);
  cudaFree(bt->d_inst);
  cudaFree(bt->d_state);
  cudaFree(bt->d_item_inst);
  cudaFree(bt->d_trips);
  cudaFree(bt->d_user);
  cudaFree(bt->d_args);
  cudaFreeHost(bt->h_user);
  cudaFreeHost(bt->h_state);
  cudaFreeHost(bt->h_trips);
  delete bt;
}

extern "C" int bmg_batch_create(bmg_hierarchy *const *hs, int count, const bmg_krylov_opts *o,
                                int autotune_tiles, void *stream, bmg_batch **out) {
  if (!out) return batch_error("bmg_batch_create: out is NULL");
  *out = nullptr;
  if (!hs || !o) return batch_error("bmg_batch_create: NULL argument");
  if (count < 1 || count > 4096) return batch_error("bmg_batch_create: need 1 <= count <= 4096");
  if (!(o->rtol > 0.0 && o->rtol < 1.0) || o->restart < 1 || o->restart > 200 || o->maxit < 0)
    return batch_error("bmg_batch_create: need 0 < rtol < 1, 1 <= restart <= 200, maxit >= 0");
  if (o->arnoldi != BMG_ARNOLDI_FP64 && o->arnoldi != BMG_ARNOLDI_MIXED)
    return batch_error("bmg_batch_create: arnoldi must be BMG_ARNOLDI_FP64 or BMG_ARNOLDI_MIXED");
  std::set<const bmg_hierarchy *> uniq;
  for (int q = 0; q < count; ++q) {
    const bmg_hierarchy *h = hs[q];
    if (!h) return batch_error("bmg_batch_create: NULL hierarchy");
    if (!uniq.insert(h).second) return batch_error("bmg_batch_create: a hierarchy appears twice");
    const bmg_mg_opts &mo = h->opts;
    if (mo.smoother != BMG_VANKA || mo.precision != BMG_FP64)
      return batch_error("bmg_batch_create: hierarchies must use the Vanka smoother in FP64");
    if (mo.gamma == 2)
      return batch_error("bmg_batch_create: hierarchies must use V-cycles (gamma 0 or 1)");
    if (mo.coarse_op != BMG_REDISC)
      return batch_error("bmg_batch_create: hierarchies must use rediscretised coarse operators");
    if (h->sys->prm.exact_divdiv)
      return batch_error("bmg_batch_create: systems must use the reduced-quadrature grad-div term");
    const bmg_mg_opts &o0 = hs[0]->opts;
    if (mo.nu1 < 1 || mo.nu1 != o0.nu1 || mo.nu2 != o0.nu2 || mo.n_coarse != o0.n_coarse)
      return batch_error("bmg_batch_create: hierarchies must share nu1 >= 1, nu2 and n_coarse");
  }
  cudaStream_t st = (cudaStream_t)stream;
  bmg_batch *bt = new bmg_batch();
  auto fail = [&](int rc) {
    bmg_batch_destroy(bt);
    return rc;
  };
#define BT_CUDA(call)                                             \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return fail(cuda_fail(e_, #call));     \
  } while (0)
  bt->count = count;
  bt->m = o->restart;
  bt->maxit = o->maxit;
  bt->rtol = o->rtol;
  bt->x0_zero = o->x0_is_zero ? 1 : 0;
  bt->df = o->arnoldi == BMG_ARNOLDI_MIXED ? 1 : 0;
  bt->hs.assign(hs, hs + count);
  const int m = bt->m;
  // per-instance vectors and FGMRES arrays
  std::vector<BInst> inst(count);
  std::vector<int> item_inst;
  auto dalloc = [&](double **p, size_t n) -> int {
    if (cudaMalloc(p, sizeof(double) * n) != cudaSuccess) return cuda_fail(cudaErrorMemoryAllocation, "batch buffers");
    bt->bufs.push_back(*p);
    if (cudaMemsetAsync(*p, 0, sizeof(double) * n, st) != cudaSuccess) return cuda_fail(cudaErrorUnknown, "memset");
    return BMG_OK;
  };
  if (cudaMalloc(&bt->d_state, sizeof(BState) * count) != cudaSuccess ||
      cudaMalloc(&bt->d_inst, sizeof(BInst) * count) != cudaSuccess ||
      cudaMalloc(&bt->d_trips, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&bt->d_user, sizeof(double *) * 2 * count) != cudaSuccess ||
      cudaMallocHost(&bt->h_user, sizeof(double *) * 2 * count) != cudaSuccess ||
      cudaMallocHost(&bt->h_state, sizeof(BState) * count) != cudaSuccess ||
      cudaMallocHost(&bt->h_trips, sizeof(int)) != cudaSuccess)
    return fail(cuda_fail(cudaErrorMemoryAllocation, "batch state"));
  cudaMemsetAsync(bt->d_state, 0, sizeof(BState) * count, st);
  cudaMemsetAsync(bt->d_trips, 0, sizeof(int), st);
  for (int q = 0; q < count; ++q) {
    const bmg_hierarchy *h = hs[q];
    const Level &L0 = h->levels[0];
    BInst &a = inst[q];
    a.vl = vec_len_of(L0.n);
    a.nb = (int)((a.vl + kChunk - 1) / kChunk);
    a.item0 = (int)item_inst.size();
    for (int b = 0; b < a.nb; ++b) item_inst.push_back(q);
    int rc;
    if ((rc = dalloc(&a.B, a.vl)) || (rc = dalloc(&a.X, a.vl)) || (rc = dalloc(&a.R, a.vl)) ||
        (rc = dalloc(&a.W, a.vl)) || (rc = dalloc(&a.V, a.vl * (m + 1))) ||
        (rc = dalloc(&a.Z, a.vl * m)) || (rc = dalloc(&a.partial, (size_t)(m + 2) * a.nb)) ||
        (rc = dalloc(&a.d, 3 * (size_t)(m + 2))) || (rc = dalloc(&a.H, (size_t)(m + 1) * m)) ||
        (rc = dalloc(&a.cs, m + 1)) || (rc = dalloc(&a.sn, m + 1)) || (rc = dalloc(&a.g, m + 1)) ||
        (rc = dalloc(&a.y, m + 1)))
      return fail(rc);
    a.V32 = nullptr;
    if (bt->df) {
      if (cudaMalloc(&a.V32, sizeof(float) * a.vl * (m + 1)) != cudaSuccess)
        return fail(cuda_fail(cudaErrorMemoryAllocation, "batch buffers"));
      bt->fbufs.push_back(a.V32);
    }
    a.Q = (double *)L0.rhs;
    a.Zc = (double *)L0.z;
    a.s = bt->d_state + q;
    bt->vl.push_back(a.vl);
  }
  bt->total_items = (int)item_inst.size();
  if (cudaMalloc(&bt->d_item_inst, sizeof(int) * item_inst.size()) != cudaSuccess)
    return fail(cuda_fail(cudaErrorMemoryAllocation, "batch items"));
  BT_CUDA(cudaMemcpyAsync(bt->d_inst, inst.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice, st));
  BT_CUDA(cudaMemcpyAsync(bt->d_item_inst, item_inst.data(), sizeof(int) * item_inst.size(),
                           cudaMemcpyHostToDevice, st));

  // ---- schedule of the batched level launches ------------------------------------------
  std::vector<unsigned char> args;
  auto put = [&](size_t bytes) {
    const size_t off = (args.size() + 255) & ~(size_t)255;
    args.resize(off + bytes);
    return off;
  };
  const size_t ab = apply_args_bytes(), vb = vanka_args_bytes();
  std::set<int, std::greater<int>> sizes;
  for (const bmg_hierarchy *h : bt->hs)
    for (const auto &L : h->levels) sizes.insert(L.n);
  const int nu1 = hs[0]->opts.nu1, nu2 = hs[0]->opts.nu2;
  struct Member { int q; size_t l; };
  auto members = [&](int n) {          // instances with a smoothing level of size n
    std::vector<Member> v;
    for (int q = 0; q < count; ++q)
      for (size_t l = 0; l + 1 < hs[q]->levels.size(); ++l)
        if (hs[q]->levels[l].n == n) v.push_back({q, l});
    return v;
  };
  auto gate_iter = [&](int q) { return (const int *)&bt->d_state[q].gate_iter; };
  auto add_apply = [&](std::vector<bmg_batch::Launch> &dst, const std::vector<Member> &G, int n,
                       auto &&xyb) {
    const size_t off = put(ab * G.size());
    for (size_t k = 0; k < G.size(); ++k) {
      const Level &L = hs[G[k].q]->levels[G[k].l];
      const double *x, *b;
      double *y;
      bool residual;
      const int *gate;
      xyb(G[k], L, x, b, y, residual, gate);
      make_apply_args(L, x, b, y, residual, gate, args.data() + off + k * ab);
    }
    dst.push_back({0, n, (int)G.size(), 0, off, 0});
  };
  auto add_vanka = [&](const std::vector<Member> &G, int n, bool assign, bool from_rhs) {
    const size_t off = put(vb * G.size());
    for (size_t k = 0; k < G.size(); ++k) {
      const bmg_hierarchy *h = hs[G[k].q];
      const Level &L = h->levels[G[k].l];
      make_vanka_args(L, (const double *)(from_rhs ? L.rhs : L.t), (double *)L.z, h->opts.omega, assign,
                      gate_iter(G[k].q), args.data() + off + k * vb);
    }
    bt->vcycle.push_back({1, n, (int)G.size(), 0, off, 0});
  };
  auto resid_apply = [&](const std::vector<Member> &G, int n) {   // t = rhs - A z
    add_apply(bt->vcycle, G, n, [&](const Member &mb, const Level &L, const double *&x, const double *&b,
                                    double *&y, bool &res, const int *&gate) {
      x = (const double *)L.z;
      b = (const double *)L.rhs;
      y = (double *)L.t;
      res = true;
      gate = gate_iter(mb.q);
    });
  };
  auto add_transfer = [&](const std::vector<Member> &G, int n, bool restr) {
    const size_t off = put(sizeof(TransferArgs) * G.size());
    for (size_t k = 0; k < G.size(); ++k) {
      const bmg_hierarchy *h = hs[G[k].q];
      const Level &F = h->levels[G[k].l], &Cl = h->levels[G[k].l + 1];
      TransferArgs t;
      t.gf = F.g;
      t.gc = Cl.g;
      t.src = (const double *)(restr ? F.t : Cl.z);
      t.dst = (double *)(restr ? Cl.rhs : F.z);
      t.gate = gate_iter(G[k].q);
      std::memcpy(args.data() + off + k * sizeof(TransferArgs), &t, sizeof(t));
    }
    bt->vcycle.push_back({restr ? 2 : 3, n, (int)G.size(), 0, off, 0});
  };
  // descending half: pre-smoothing, residual, restriction
  for (int n : sizes) {
    auto G = members(n);
    if (G.empty()) continue;
    bt->tiles[{0, n}] = default_apply_tile(n, (int)G.size());
    bt->tiles[{1, n}] = default_vanka_tile(n, (int)G.size());
    for (int sweep = 0; sweep < nu1; ++sweep) {
      if (sweep == 0) {
        add_vanka(G, n, true, true);
      } else {
        resid_apply(G, n);
        add_vanka(G, n, false, false);
      }
    }
    resid_apply(G, n);
    add_transfer(G, n, true);
  }
  // coarsest level of every instance
  {
    const size_t off = put(sizeof(CoarseArgs) * count);
    int max_free = 0;
    std::map<int, unsigned char *> mask_of;
    for (int q = 0; q < count; ++q) {
      const Level &L = hs[q]->levels.back();
      if (!mask_of.count(L.n)) {
        std::vector<int> idx(L.nfree);
        BT_CUDA(cudaMemcpy(idx.data(), L.free_idx, sizeof(int) * L.nfree, cudaMemcpyDeviceToHost));
        std::vector<unsigned char> mk(vec_len_of(L.n), 0);
        for (int f : idx) mk[f] = 1;
        unsigned char *dm = nullptr;
        if (cudaMalloc(&dm, mk.size()) != cudaSuccess) return fail(cuda_fail(cudaErrorMemoryAllocation, "mask"));
        bt->masks.push_back(dm);
        BT_CUDA(cudaMemcpy(dm, mk.data(), mk.size(), cudaMemcpyHostToDevice));
        mask_of[L.n] = dm;
      }
      CoarseArgs c;
      c.inv = L.cinv64;
      c.free_idx = L.free_idx;
      c.free_mask = mask_of[L.n];
      c.N = L.nfree;
      c.vl = vec_len_of(L.n);
      c.r = (const double *)L.rhs;
      c.z = (double *)L.z;
      c.gate = gate_iter(q);
      max_free = std::max(max_free, L.nfree);
      std::memcpy(args.data() + off + q * sizeof(CoarseArgs), &c, sizeof(c));
    }
    bt->vcycle.push_back({4, hs[0]->levels.back().n, count, 0, off, max_free});
  }
  // ascending half: prolongation and post-smoothing
  for (auto it = sizes.rbegin(); it != sizes.rend(); ++it) {
    const int n = *it;
    auto G = members(n);
    if (G.empty()) continue;
    add_transfer(G, n, false);
    for (int sweep = 0; sweep < nu2; ++sweep) {
      resid_apply(G, n);
      add_vanka(G, n, false, false);
    }
  }
  // finest-level operator applications of FGMRES, grouped by instance size
  std::set<int, std::greater<int>> fine_sizes;
  for (const bmg_hierarchy *h : bt->hs) fine_sizes.insert(h->levels[0].n);
  for (int n : fine_sizes) {
    std::vector<Member> G;
    for (int q = 0; q < count; ++q)
      if (hs[q]->levels[0].n == n) G.push_back({q, 0});
    if (!bt->tiles.count({0, n})) bt->tiles[{0, n}] = default_apply_tile(n, (int)G.size());
    add_apply(bt->resid, G, n, [&](const Member &mb, const Level &, const double *&x, const double *&b,
                                   double *&y, bool &res, const int *&gate) {
      x = inst[mb.q].X;
      b = inst[mb.q].B;
      y = inst[mb.q].R;
      res = true;
      gate = (const int *)&bt->d_state[mb.q].gate_end;
    });
    add_apply(bt->wapply, G, n, [&](const Member &mb, const Level &, const double *&x, const double *&b,
                                    double *&y, bool &res, const int *&gate) {
      x = inst[mb.q].Zc;
      b = nullptr;
      y = inst[mb.q].W;
      res = false;
      gate = gate_iter(mb.q);
    });
  }
  if (cudaMalloc(&bt->d_args, std::max<size_t>(args.size(), 256)) != cudaSuccess)
    return fail(cuda_fail(cudaErrorMemoryAllocation, "batch arguments"));
  BT_CUDA(cudaMemcpyAsync(bt->d_args, args.data(), args.size(), cudaMemcpyHostToDevice, st));
  BT_CUDA(cudaStreamSynchronize(st));
  if (autotune_tiles) {
    int rc = autotune(bt, st);
    if (rc) return fail(rc);
  }
  if (cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking) != cudaSuccess)
    return fail(cuda_fail(cudaErrorUnknown, "capture stream"));
  int rc = prepare_apply_batch();
  if (!rc) rc = build_graph(bt);
  if (rc) return fail(rc);
  *out = bt;
  return BMG_OK;
#undef BT_CUDA
}

extern "C" int bmg_batch_solve(bmg_batch *bt, const double *const *b, double *const *x,
                               bmg_solve_info *infos, void *stream) {
  auto t0 = std::chrono::steady_clock::now();
  if (!bt || !b || !x) return batch_error("bmg_batch_solve: NULL argument");
  const int C = bt->count;
  for (int q = 0; q < C; ++q) {
    if (!b[q] || !x[q]) return batch_error("bmg_batch_solve: NULL vector");
    if (b[q] == x[q]) return batch_error("bmg_batch_solve: x may not alias b");
    bt->h_user[q] = const_cast<double *>(b[q]);
    bt->h_user[C + q] = x[q];
  }
  cudaStream_t st = (cudaStream_t)stream;
  BMG_CUDA(cudaMemcpyAsync(bt->d_user, bt->h_user, sizeof(double *) * 2 * C, cudaMemcpyHostToDevice, st));
  BMG_CUDA(cudaGraphLaunch(bt->exec, st));
  BMG_CUDA(cudaMemcpyAsync(bt->h_state, bt->d_state, sizeof(BState) * C, cudaMemcpyDeviceToHost, st));
  BMG_CUDA(cudaMemcpyAsync(bt->h_trips, bt->d_trips, sizeof(int), cudaMemcpyDeviceToHost, st));
  BMG_CUDA(cudaStreamSynchronize(st));
  bt->last_trips = *bt->h_trips;
  g_launches += bt->kernels_pro + (long long)bt->last_trips * bt->kernels_body + bt->kernels_epi;
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  bool nonfinite = false;
  for (int q = 0; q < C; ++q) {
    const BState &s = bt->h_state[q];
    nonfinite = nonfinite || s.nonfinite_b;
    if (infos) {
      bmg_solve_info &inf = infos[q];
      inf.iters = s.iters;
      inf.restarts = s.restarts;
      inf.status = s.status;
      inf.relres = s.relres;
      inf.relres_est = s.est;
      inf.solve_ms = ms;
    }
  }
  if (nonfinite) {
    set_error("bmg_batch_solve: a right-hand side is not finite");
    return BMG_ERR_NONFINITE;
  }
  return BMG_OK;
}

extern "C" int bmg_batch_tile(const bmg_batch *bt, int kernel, int n) {
  if (!bt) return -1;
  const int kind = kernel == BMG_PROF_APPLY ? 0 : kernel == BMG_PROF_VANKA ? 1 : -1;
  auto it = bt->tiles.find({kind, n});
  return it == bt->tiles.end() ? -1 : it->second;
}

extern "C" int bmg_batch_trips(const bmg_batch *bt) { return bt ? bt->last_trips : 0; }

extern "C" long long bmg_batch_kernels_per_trip(const bmg_batch *bt) { return bt ? bt->kernels_body : 0; }
