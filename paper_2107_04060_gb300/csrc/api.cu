// C ABI of the library (include/biotmg.h): systems, hierarchies, the V-cycle and FGMRES.
// Host code only orchestrates: every arithmetic step of assembly, relaxation, transfer,
// coarse solve and Krylov iteration runs in this library's kernels.
#include <algorithm>
#include <type_traits>
#include <cstdlib>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "bmg_internal.h"

namespace bmg {

static thread_local std::string g_last_error;
std::atomic<long long> g_launches{0};

void set_error(const std::string &msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char *what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return BMG_ERR_CUDA;
}

static int arg_error(const std::string &msg) {
  g_last_error = msg;
  return BMG_ERR_ARG;
}

// ---- coefficient kernels ---------------------------------------------------------------
__global__ void kinv_from_k_kernel(Grid g, const double *K, double *kinv64, float *kinv32,
                                   int *flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.pitch || j > g.n) return;
  for (int o = 0; o < 2; ++o) {
    const size_t idx = (size_t)o * g.blk + (size_t)j * g.pitch + i;
    double v = 0.0;
    if (i < g.n && j < g.n) {
      const double k = K[idx];
      if (!(k > 0.0) || !isfinite(k)) atomicOr(flag, 4);
      else v = 1.0 / k;
    }
    kinv64[idx] = v;
    kinv32[idx] = (float)v;
  }
}

// K^{-1} = exp(-theta) from a per-triangle log-permeability (FP32, same layout as K).
__global__ void kinv_from_logk_kernel(Grid g, const float *theta, double *kinv64, float *kinv32,
                                      int *flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.pitch || j > g.n) return;
  for (int o = 0; o < 2; ++o) {
    const size_t idx = (size_t)o * g.blk + (size_t)j * g.pitch + i;
    double v = 0.0;
    if (i < g.n && j < g.n) {
      const double t = (double)theta[idx];
      v = exp(-t);
      if (!isfinite(t) || !(v > 0.0) || !isfinite(v)) atomicOr(flag, 4);
    }
    kinv64[idx] = v;
    kinv32[idx] = (float)v;
  }
}

static int alloc_coefs(Level &L, bool full) {
  const size_t blk = L.g.blk;
  if (!full) {
    BMG_CUDA(cudaMalloc(&L.kinv64, sizeof(double) * 2 * blk));
    BMG_CUDA(cudaMalloc(&L.kinv32, sizeof(float) * 2 * blk));
  } else {
    BMG_CUDA(cudaMalloc(&L.wm64, sizeof(double) * 12 * blk));
    BMG_CUDA(cudaMalloc(&L.wm32, sizeof(float) * 12 * blk));
    BMG_CUDA(cudaMemset(L.wm64, 0, sizeof(double) * 12 * blk));
    BMG_CUDA(cudaMemset(L.wm32, 0, sizeof(float) * 12 * blk));
  }
  return BMG_OK;
}

static void free_level(Level &L) {
  free_apply_tma(L);
  if (L.owns_coefs) {
    cudaFree(L.kinv64); cudaFree(L.kinv32); cudaFree(L.wm64); cudaFree(L.wm32);
  }
  cudaFree(L.slot); cudaFree(L.pinv64); cudaFree(L.pinv32);
  cudaFree(L.dinv64); cudaFree(L.dinv32); cudaFree(L.sinv64); cudaFree(L.sinv32);
  cudaFree(L.free_idx); cudaFree(L.cinv64); cudaFree(L.cinv32);
  cudaFree(L.rhs); cudaFree(L.z); cudaFree(L.t); cudaFree(L.t2); cudaFree(L.wz);
  cudaFree(L.bz); cudaFree(L.bd); cudaFree(L.cg); cudaFree(L.cg_flag); cudaFree(L.smg); cudaFree(L.sdense);
  L = Level();
}

// ---- kernel timing ---------------------------------------------------------------------
// Launches may come from several host threads (solves on distinct handles): each launch keeps
// its own begin event and appends the (begin, end) pair under a lock.
struct ProfState {
  int kernel = 0, n = 0;
  std::vector<cudaEvent_t> ev;     // pairs (begin, end)
  double cells = 0.0;
};
static ProfState g_prof;
static std::mutex g_prof_mutex;

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// V-cycles replayed from CUDA graphs (bmg_use_graphs); on unless BMG_NO_GRAPHS is set
static std::atomic<int> g_use_graphs{[] {
  const char *e = std::getenv("BMG_NO_GRAPHS");
  return (e && *e && *e != '0') ? 0 : 1;
}()};

bool prof_on(int kernel, int n) {
  std::lock_guard<std::mutex> lk(g_prof_mutex);
  return g_prof.kernel != 0 && g_prof.kernel == kernel && (g_prof.n == 0 || g_prof.n == n);
}
cudaEvent_t prof_begin(cudaStream_t st) {
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  cudaEventRecord(e, st);
  return e;
}
void prof_end(cudaStream_t st, cudaEvent_t e0, double cells) {
  cudaEvent_t e = nullptr;
  if (!e0 || cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, st);
  std::lock_guard<std::mutex> lk(g_prof_mutex);
  g_prof.ev.push_back(e0);
  g_prof.ev.push_back(e);
  g_prof.cells += cells;
}

}  // namespace bmg

using namespace bmg;

extern "C" long long bmg_launch_count(void) { return g_launches.load(); }

extern "C" int bmg_use_graphs(int enable) { return g_use_graphs.exchange(enable ? 1 : 0); }

extern "C" int bmg_profile_start(int kernel, int n) {
  if (kernel < 1 || kernel > 8 || n < 0) return arg_error("bmg_profile_start: bad kernel id or n");
  std::lock_guard<std::mutex> lk(g_prof_mutex);
  for (auto e : g_prof.ev) cudaEventDestroy(e);
  g_prof = ProfState();
  g_prof.kernel = kernel;
  g_prof.n = n;
  return BMG_OK;
}

extern "C" int bmg_profile_stop(double *total_ms, long long *launches, double *cells) {
  std::lock_guard<std::mutex> lk(g_prof_mutex);
  double tot = 0.0;
  long long cnt = 0;
  cudaError_t err = cudaSuccess;
  for (size_t k = 0; k + 1 < g_prof.ev.size(); k += 2) {
    cudaError_t e = cudaEventSynchronize(g_prof.ev[k + 1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, g_prof.ev[k], g_prof.ev[k + 1]);
    if (e != cudaSuccess) err = e;
    tot += ms;
    ++cnt;
  }
  if (total_ms) *total_ms = tot;
  if (launches) *launches = cnt;
  if (cells) *cells = g_prof.cells;
  for (auto e : g_prof.ev) cudaEventDestroy(e);
  g_prof = ProfState();
  if (err != cudaSuccess) return cuda_fail(err, "bmg_profile_stop");
  return BMG_OK;
}

// ---- layout ----------------------------------------------------------------------------
extern "C" int bmg_pitch(int n) { return n >= 1 ? pitch_of(n) : 0; }
extern "C" size_t bmg_block_len(int n) { return n >= 1 ? block_len_of(n) : 0; }
extern "C" size_t bmg_vector_len(int n) { return n >= 1 ? vec_len_of(n) : 0; }
extern "C" size_t bmg_free_dofs(int n) {
  if (n < 1) return 0;
  const size_t N = (size_t)n;
  return 2 * (N - 1) * (N - 1) + (3 * N * N - 2 * N) + (3 * N * N + 2 * N) + 2 * N * N;
}

extern "C" const char *bmg_status_string(int code) {
  switch (code) {
    case BMG_OK: return "ok";
    case BMG_ERR_ARG: return "invalid argument";
    case BMG_ERR_CUDA: return "CUDA error";
    case BMG_ERR_ALLOC: return "allocation failed";
    case BMG_ERR_SINGULAR: return "singular factorisation";
    case BMG_ERR_NONFINITE: return "non-finite or non-positive input";
    case BMG_ERR_NOCONV: return "inner iterative solve did not converge";
    default: return "unknown status";
  }
}
extern "C" const char *bmg_last_error(void) { return g_last_error.c_str(); }

// ---- system ----------------------------------------------------------------------------
static int assemble_impl(int n, double lambda, double mu, const double *K, const float *logK,
                         double K_const, double tau, double alpha, double inv_M, bool exact_divdiv,
                         void *stream, bmg_system **out) {
  if (!out) return arg_error("bmg_assemble: out is NULL");
  *out = nullptr;
  if (n < 1 || n > 16384) return arg_error("bmg_assemble: n out of range [1, 16384]");
  if (!(std::isfinite(lambda) && lambda > 0.0) || !(std::isfinite(mu) && mu >= 0.0) ||
      !(std::isfinite(tau) && tau > 0.0) || !std::isfinite(alpha) ||
      !(std::isfinite(inv_M) && inv_M >= 0.0))
    return arg_error("bmg_assemble: physical parameters must be finite with lambda > 0, "
                     "mu >= 0, tau > 0, inv_M >= 0");
  if (!K && !logK && !(std::isfinite(K_const) && K_const > 0.0))
    return arg_error("bmg_assemble: K_const must be finite and > 0 when K is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = upload_transfer_tables();
  if (rc) return rc;
  static const bool pattern_ok = [] {
    std::string why;
    const bool ok = verify_elem_nonzeros(&why);
    if (!ok) set_error("element integrals do not have the compiled sparsity: " + why);
    return ok;
  }();
  if (!pattern_ok) return BMG_ERR_ARG;
  bmg_system *s = new bmg_system();
  s->n = n;
  s->prm = PhysParams{lambda, mu, tau, alpha, inv_M};
  s->prm.exact_divdiv = exact_divdiv;
  s->uniform = (K == nullptr && logK == nullptr);
  s->K_const = K_const;
  Level &L = s->fine;
  L.n = n;
  L.g = grid_of(n);
  L.uniform = s->uniform;
  L.dense_a = exact_divdiv;
  rc = alloc_coefs(L, false);
  if (!rc && cudaMalloc(&s->adj_partial, sizeof(double) * 2 * kAdjBlocks) != cudaSuccess)
    rc = cuda_fail(cudaErrorMemoryAllocation, "bmg_assemble");
  if (rc) { free_level(L); cudaFree(s->adj_partial); delete s; return rc; }
  make_coefs(s->prm, n, &L.c64, &L.c32);
  if (s->uniform) {
    if ((rc = launch_fill<double>(L.kinv64, 1.0 / K_const, 2 * L.g.blk, st)) ||
        (rc = launch_fill<float>(L.kinv32, (float)(1.0 / K_const), 2 * L.g.blk, st))) {
      free_level(L); delete s; return rc;
    }
  } else {
    int *flag = nullptr;
    cudaError_t e = cudaMalloc(&flag, sizeof(int));
    if (e != cudaSuccess) { free_level(L); delete s; return cuda_fail(e, "cudaMalloc(flag)"); }
    cudaMemsetAsync(flag, 0, sizeof(int), st);
    dim3 b(32, 8), gr((L.g.pitch + 31) / 32, (n + 1 + 7) / 8);
    if (K) kinv_from_k_kernel<<<gr, b, 0, st>>>(L.g, K, L.kinv64, L.kinv32, flag);
    else kinv_from_logk_kernel<<<gr, b, 0, st>>>(L.g, logK, L.kinv64, L.kinv32, flag);
    ++g_launches;
    int hflag = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(flag);
    if (e != cudaSuccess) { free_level(L); cudaFree(s->adj_partial); delete s; return cuda_fail(e, "kinv_from_k"); }
    if (hflag) {
      free_level(L); cudaFree(s->adj_partial); delete s;
      set_error("bmg_assemble: permeability must be finite and > 0 on every triangle");
      return BMG_ERR_NONFINITE;
    }
  }
  *out = s;
  return BMG_OK;
}

extern "C" int bmg_assemble(int n, double lambda, double mu, const double *K, double K_const,
                            double tau, double alpha, double inv_M, void *stream,
                            bmg_system **out) {
  return assemble_impl(n, lambda, mu, K, nullptr, K_const, tau, alpha, inv_M, false, stream, out);
}

extern "C" int bmg_assemble_divdiv(int n, double lambda, double mu, const double *K, double K_const,
                                   double tau, double alpha, double inv_M, int divdiv, void *stream,
                                   bmg_system **out) {
  if (divdiv != BMG_DIVDIV_REDUCED && divdiv != BMG_DIVDIV_EXACT) {
    if (out) *out = nullptr;
    return arg_error("bmg_assemble_divdiv: divdiv must be BMG_DIVDIV_REDUCED or BMG_DIVDIV_EXACT");
  }
  return assemble_impl(n, lambda, mu, K, nullptr, K_const, tau, alpha, inv_M, divdiv == BMG_DIVDIV_EXACT,
                       stream, out);
}

extern "C" int bmg_assemble_logk(int n, double lambda, double mu, const float *logK, double tau,
                                 double alpha, double inv_M, void *stream, bmg_system **out) {
  if (!logK) return arg_error("bmg_assemble_logk: logK is NULL");
  return assemble_impl(n, lambda, mu, nullptr, logK, 0.0, tau, alpha, inv_M, false, stream, out);
}

extern "C" int bmg_system_n(const bmg_system *s) { return s ? s->n : 0; }

extern "C" void bmg_destroy_system(bmg_system *s) {
  if (!s) return;
  free_level(s->fine);
  cudaFree(s->adj_partial);
  delete s;
}

extern "C" int bmg_apply(const bmg_system *s, const double *x, double *y, void *stream) {
  if (!s || !x || !y) return arg_error("bmg_apply: NULL argument");
  if (x == y) return arg_error("bmg_apply: y may not alias x");
  return launch_apply<double>(s->fine, x, nullptr, y, false, 1, 0, (cudaStream_t)stream);
}

extern "C" int bmg_residual(const bmg_system *s, const double *b, const double *x, double *r,
                            void *stream) {
  if (!s || !b || !x || !r) return arg_error("bmg_residual: NULL argument");
  if (x == r) return arg_error("bmg_residual: r may not alias x");
  return launch_apply<double>(s->fine, x, b, r, true, 1, 0, (cudaStream_t)stream);
}

// ---- hierarchy -------------------------------------------------------------------------
static int setup_patches(bmg_hierarchy *h, Level &L, int psize, double p_shift,
                         cudaStream_t st) {
  const int n = L.n;
  std::vector<int> slot((size_t)(n + 1) * (n + 1));
  std::vector<int> ri, rj;
  if (L.uniform && n >= 2) {
    ri.push_back(1);
    rj.push_back(1);
    for (int j = 0; j <= n; ++j)
      for (int i = 0; i <= n; ++i) {
        const bool interior = i > 0 && i < n && j > 0 && j < n;
        if (interior) {
          slot[(size_t)j * (n + 1) + i] = 0;
        } else {
          slot[(size_t)j * (n + 1) + i] = (int)ri.size();
          ri.push_back(i);
          rj.push_back(j);
        }
      }
  } else {
    for (int j = 0; j <= n; ++j)
      for (int i = 0; i <= n; ++i) {
        slot[(size_t)j * (n + 1) + i] = (int)ri.size();
        ri.push_back(i);
        rj.push_back(j);
      }
  }
  const int nrep = (int)ri.size();
  L.nslots = nrep;
  L.psize = psize;
  int *d_ri = nullptr, *d_rj = nullptr;
  BMG_CUDA(cudaMalloc(&L.slot, sizeof(int) * slot.size()));
  BMG_CUDA(cudaMalloc(&d_ri, sizeof(int) * nrep));
  BMG_CUDA(cudaMalloc(&d_rj, sizeof(int) * nrep));
  BMG_CUDA(cudaMalloc(&L.pinv64, sizeof(double) * (size_t)patch_entries(psize) * nrep));
  BMG_CUDA(cudaMalloc(&L.pinv32, sizeof(float) * (size_t)patch_entries(psize) * nrep));
  BMG_CUDA(cudaMemcpyAsync(L.slot, slot.data(), sizeof(int) * slot.size(), cudaMemcpyHostToDevice, st));
  BMG_CUDA(cudaMemcpyAsync(d_ri, ri.data(), sizeof(int) * nrep, cudaMemcpyHostToDevice, st));
  BMG_CUDA(cudaMemcpyAsync(d_rj, rj.data(), sizeof(int) * nrep, cudaMemcpyHostToDevice, st));
  int rc = launch_vanka_setup(L, d_ri, d_rj, nrep, p_shift * 0.5 / ((double)n * n), psize,
                              h->d_flag, st);
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(d_ri);
  cudaFree(d_rj);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "vanka setup");
  return psize == 20 ? vanka_klein_setup(L, st) : BMG_OK;
}

// ---- tile tuning ---------------------------------------------------------------------
// Times every candidate tile of a level's operator and smoother launches (on the level's own
// work vectors) and keeps the fastest.  The results do not depend on the tile: every output
// value is formed by the same arithmetic whichever tile holds it.
template <typename F>
static int time_min(F &&launch, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st, float *ms) {
  // the best of three timings of three back-to-back launches (single launches of ~100 us
  // differ by less than their timing noise)
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    BMG_CUDA(cudaEventRecord(e0, st));
    for (int k = 0; k < 3; ++k) {
      int rc = launch();
      if (rc) return rc;
    }
    BMG_CUDA(cudaEventRecord(e1, st));
    BMG_CUDA(cudaEventSynchronize(e1));
    float t = 0.f;
    BMG_CUDA(cudaEventElapsedTime(&t, e0, e1));
    if (rep > 0) best = std::min(best, t);        // the first launch warms up
  }
  *ms = best;
  return BMG_OK;
}

template <typename F>
static int pick_tile(int *slot, int first, int last, F &&launch, cudaEvent_t e0, cudaEvent_t e1,
                     cudaStream_t st) {
  float best = 1e30f;
  int best_t = -1;
  for (int t = first; t <= last; ++t) {
    *slot = t;
    float ms;
    int rc = time_min(launch, e0, e1, st, &ms);
    if (rc) {
      *slot = -1;
      return rc;
    }
    if (ms < best) {
      best = ms;
      best_t = t;
    }
  }
  *slot = best_t;
  return BMG_OK;
}

// Tiles chosen by timing are kept per device and level shape for the rest of the process: a
// later hierarchy with a level of the same shape (grid size, precision, smoother family,
// coefficient storage, patch-solve precision, whether the TMA operator variant exists) takes
// the earlier choice without timing again.  Setups that rebuild the same hierarchy many
// times (one per gradient of a parameter study) then pay for the timing once.
struct TileKey {
  int dev, n, kind;            // kind: 0 = V-cycle level, 1 = the FP64 FGMRES operator
  int fp32, smoother, uniform, klein, wm_full, dense, solve64, tma;
  bool operator<(const TileKey &o) const {
    const int a[11] = {dev, n, kind, fp32, smoother, uniform, klein, wm_full, dense, solve64, tma};
    const int b[11] = {o.dev, o.n, o.kind, o.fp32, o.smoother, o.uniform, o.klein, o.wm_full, o.dense, o.solve64, o.tma};
    return std::lexicographical_compare(a, a + 11, b, b + 11);
  }
};
struct TileChoice { int apply, vanka, vanka_u; };
static std::mutex g_tile_mutex;
static std::map<TileKey, TileChoice> g_tile_cache;

static TileKey tile_key(const bmg_hierarchy *h, const Level &L, int kind) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int fam = h->opts.smoother == BMG_VANKA ? 0 : 1;
  return TileKey{dev, L.n, kind, kind == 0 && h->opts.precision == BMG_FP32, kind == 0 ? fam : 0,
                 L.uniform, L.klein, L.wm_full, L.dense_a, L.solve64, kind == 0 && L.tma != nullptr};
}

static bool tile_cached(const TileKey &k, TileChoice *c) {
  std::lock_guard<std::mutex> lk(g_tile_mutex);
  auto it = g_tile_cache.find(k);
  if (it == g_tile_cache.end()) return false;
  *c = it->second;
  return true;
}

static void tile_store(const TileKey &k, const TileChoice &c) {
  std::lock_guard<std::mutex> lk(g_tile_mutex);
  g_tile_cache[k] = c;
}

template <typename T>
static int tune_level_timed(bmg_hierarchy *h, Level &L, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st);

template <typename T>
static int tune_level(bmg_hierarchy *h, Level &L, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st) {
  const char *fa = std::getenv("BMG_FORCE_APPLY_TILE"), *fs = std::getenv("BMG_FORCE_SMOOTHER_TILE");
  const bool forced = (fa && *fa) || (fs && *fs);
  const TileKey key = tile_key(h, L, 0);
  TileChoice c;
  if (!forced && tile_cached(key, &c)) {
    L.tile_apply = c.apply;
    L.tile_vanka = c.vanka;
    L.tile_vanka_u = c.vanka_u;
    return BMG_OK;
  }
  int rc = tune_level_timed<T>(h, L, e0, e1, st);
  if (!rc && !forced) tile_store(key, TileChoice{L.tile_apply, L.tile_vanka, L.tile_vanka_u});
  return rc;
}

template <typename T>
static int tune_level_timed(bmg_hierarchy *h, Level &L, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st) {
  T *z = (T *)L.z, *t = (T *)L.t;
  const T *r = (const T *)L.rhs;
  // candidates 0-4: tile shapes; 5 (FP32): 32 x 8 with the input staged by TMA.  The
  // environment variable BMG_FORCE_APPLY_TILE fixes the choice (testing the variants).
  int rc;
  const char *force = std::getenv("BMG_FORCE_APPLY_TILE");
  if (force && *force) {
    L.tile_apply = std::atoi(force);
  } else {
    rc = pick_tile(&L.tile_apply, 0, sizeof(T) == 8 ? 9 : 7,
                   [&] { return launch_apply<T>(L, z, r, t, true, 1, 0, st); }, e0, e1, st);
    if (rc) return rc;
  }
  // BMG_FORCE_SMOOTHER_TILE fixes the Vanka (or, for BSR, the displacement-Vanka) tile
  const char *force_s = std::getenv("BMG_FORCE_SMOOTHER_TILE");
  const bool forced = force_s && *force_s;
  if (h->opts.smoother == BMG_VANKA) {
    if (forced) { L.tile_vanka = std::atoi(force_s); return BMG_OK; }
    return pick_tile(&L.tile_vanka, 0, 7,
                     [&] { return launch_vanka_sweep<T>(L, r, z, (T)h->opts.omega, st, false); }, e0, e1, st);
  }
  if (forced) { L.tile_vanka_u = std::atoi(force_s); return BMG_OK; }
  return pick_tile(&L.tile_vanka_u, 0, 7,
                   [&] { return launch_bsr_sweep<T>(L, r, z, (T)h->opts.omega, st, false); }, e0, e1, st);
}

static int tune_hierarchy(bmg_hierarchy *h, cudaStream_t st) {
  cudaEvent_t e0, e1;
  BMG_CUDA(cudaEventCreate(&e0));
  BMG_CUDA(cudaEventCreate(&e1));
  int rc = BMG_OK;
  const bool fp32 = h->opts.precision == BMG_FP32;
  for (size_t l = 0; l + 1 < h->levels.size() && !rc; ++l)
    rc = fp32 ? tune_level<float>(h, h->levels[l], e0, e1, st) : tune_level<double>(h, h->levels[l], e0, e1, st);
  // the FP64 fine-level operator of FGMRES (its own FP64 scratch vectors)
  TileChoice fc;
  const TileKey fkey = tile_key(h, h->fine_op, 1);
  if (!rc && tile_cached(fkey, &fc)) {
    h->fine_op.tile_apply = fc.apply;
  } else if (!rc) {
    Level &F = h->fine_op;
    const size_t vl = vec_len_of(F.n);
    double *a = nullptr, *b = nullptr;
    if (cudaMalloc(&a, sizeof(double) * vl) != cudaSuccess || cudaMalloc(&b, sizeof(double) * vl) != cudaSuccess) {
      rc = cuda_fail(cudaErrorMemoryAllocation, "tuning vectors");
    } else {
      cudaMemsetAsync(a, 0, sizeof(double) * vl, st);
      rc = pick_tile(&F.tile_apply, 0, 9, [&] { return launch_apply<double>(F, a, a, b, true, 1, 0, st); },
                     e0, e1, st);
      if (!rc) tile_store(fkey, TileChoice{F.tile_apply, -1, -1});
    }
    cudaStreamSynchronize(st);
    cudaFree(a);
    cudaFree(b);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

extern "C" int bmg_setup_hierarchy(const bmg_system *s, const bmg_mg_opts *o, void *stream,
                                   bmg_hierarchy **out) {
  if (!out) return arg_error("bmg_setup_hierarchy: out is NULL");
  *out = nullptr;
  if (!s || !o) return arg_error("bmg_setup_hierarchy: NULL argument");
  if (o->smoother != BMG_VANKA && o->smoother != BMG_BSR && o->smoother != BMG_BSR_EXACT)
    return arg_error("bmg_setup_hierarchy: unknown smoother");
  if (o->smoother == BMG_BSR_EXACT && o->precision != BMG_FP64)
    return arg_error("bmg_setup_hierarchy: exact BSR runs in FP64 only");
  if (o->precision != BMG_FP64 && o->precision != BMG_FP32)
    return arg_error("bmg_setup_hierarchy: unknown precision");
  if (o->nu1 < 0 || o->nu2 < 0 || o->nu1 + o->nu2 < 1 || o->nu1 > 16 || o->nu2 > 16)
    return arg_error("bmg_setup_hierarchy: need 0 <= nu1, nu2 <= 16 and nu1 + nu2 >= 1");
  if (!(std::isfinite(o->omega) && o->omega > 0.0) || !std::isfinite(o->omega_J) ||
      !(std::isfinite(o->p_shift) && o->p_shift >= 0.0))
    return arg_error("bmg_setup_hierarchy: omega > 0, finite omega_J, p_shift >= 0 required");
  if (o->gamma < 0 || o->gamma > 2)
    return arg_error("bmg_setup_hierarchy: gamma must be 0 or 1 (V-cycle) or 2 (W-cycle)");
  if (o->coarse_op != BMG_REDISC && o->coarse_op != BMG_GALERKIN)
    return arg_error("bmg_setup_hierarchy: coarse_op must be BMG_REDISC or BMG_GALERKIN");
  if (o->patch_solve != BMG_PATCH_CYCLE && o->patch_solve != BMG_PATCH_FP64)
    return arg_error("bmg_setup_hierarchy: patch_solve must be BMG_PATCH_CYCLE or BMG_PATCH_FP64");
  const int n = s->n;
  if (o->n_coarse < 2 || o->n_coarse > 64 || n < o->n_coarse || n % o->n_coarse)
    return arg_error("bmg_setup_hierarchy: need 2 <= n_coarse <= 64 dividing n");
  int ratio = n / o->n_coarse;
  if (ratio & (ratio - 1)) return arg_error("bmg_setup_hierarchy: n / n_coarse must be a power of 2");
  cudaStream_t st = (cudaStream_t)stream;
  bmg_hierarchy *h = new bmg_hierarchy();
  h->sys = s;
  h->opts = *o;
  auto fail = [&](int rc) {
    bmg_destroy_hierarchy(h);
    return rc;
  };
  if (cudaMalloc(&h->d_flag, sizeof(int)) != cudaSuccess) return fail(cuda_fail(cudaErrorMemoryAllocation, "flag"));
  cudaMemsetAsync(h->d_flag, 0, sizeof(int), st);
  const bool fp32 = o->precision == BMG_FP32;
  const size_t es = fp32 ? sizeof(float) : sizeof(double);
  for (int m = n;; m /= 2) {
    h->levels.emplace_back();
    Level &L = h->levels.back();
    L.n = m;
    L.g = grid_of(m);
    if (m == n) {
      L.owns_coefs = false;
      L.kinv64 = s->fine.kinv64;
      L.kinv32 = s->fine.kinv32;
      L.c64 = s->fine.c64;
      L.c32 = s->fine.c32;
      L.uniform = s->uniform;
      L.wm_full = false;
      L.dense_a = s->fine.dense_a;
    } else {
      L.uniform = s->uniform;
      L.wm_full = !s->uniform;
      int rc = alloc_coefs(L, L.wm_full);
      if (rc) return fail(rc);
      make_coefs(s->prm, m, &L.c64, &L.c32);
      L.dense_a = s->prm.exact_divdiv;
      if (o->coarse_op == BMG_GALERKIN) {
        galerkin_coarsen_coefs(h->levels[h->levels.size() - 2].c64, &L.c64, &L.c32);
        L.dense_a = true;
      }
      if (s->uniform) {
        if ((rc = launch_fill<double>(L.kinv64, 1.0 / s->K_const, 2 * L.g.blk, st)) ||
            (rc = launch_fill<float>(L.kinv32, (float)(1.0 / s->K_const), 2 * L.g.blk, st)))
          return fail(rc);
      } else {
        rc = launch_coarsen_wmass(h->levels[h->levels.size() - 2], L, st);
        if (rc) return fail(rc);
      }
    }
    const size_t vl = vec_len_of(m);
    if (cudaMalloc(&L.rhs, es * vl) != cudaSuccess || cudaMalloc(&L.z, es * vl) != cudaSuccess ||
        cudaMalloc(&L.t, es * vl) != cudaSuccess || cudaMalloc(&L.t2, es * vl) != cudaSuccess)
      return fail(cuda_fail(cudaErrorMemoryAllocation, "level work vectors"));
    cudaMemsetAsync(L.rhs, 0, es * vl, st);
    cudaMemsetAsync(L.z, 0, es * vl, st);
    cudaMemsetAsync(L.t, 0, es * vl, st);
    cudaMemsetAsync(L.t2, 0, es * vl, st);
    if (o->gamma == 2 && m != n && m != o->n_coarse) {       // levels that take a second cycle
      if (cudaMalloc(&L.wz, es * vl) != cudaSuccess)
        return fail(cuda_fail(cudaErrorMemoryAllocation, "W-cycle work vector"));
      cudaMemsetAsync(L.wz, 0, es * vl, st);
    }
    L.err = h->d_flag;
    L.solve64 = fp32 && o->smoother == BMG_VANKA && o->patch_solve == BMG_PATCH_FP64;
    // FP32 operator input staged by TMA: the V-cycle applies the operator to z (to t2 on the
    // finest level); tuning decides whether that variant runs
    if (fp32 && m != o->n_coarse) {
      int rc = setup_apply_tma(L, (const float *)L.z, m == n ? (const float *)L.t2 : nullptr);
      if (rc) return fail(rc);
    }
    if (m == o->n_coarse) break;
  }
  for (size_t l = 0; l + 1 < h->levels.size(); ++l) {
    Level &L = h->levels[l];
    int rc;
    if (o->smoother == BMG_VANKA) {
      rc = setup_patches(h, L, 20, o->p_shift, st);
    } else {
      rc = setup_patches(h, L, 8, 0.0, st);
      const PhysParams &p = s->prm;
      const double area = 0.5 / ((double)L.n * L.n);
      const double c_fs = p.inv_M + p.alpha * p.alpha / (p.lambda + p.mu);   // 2 mu / d, d = 2
      const bool exact = o->smoother == BMG_BSR_EXACT;     // S solved: 1 / diag(S) unweighted
      if (!rc) rc = launch_bsr_setup(L, exact ? 1.0 : o->omega_J, c_fs * area, st);
      L.s_c = c_fs * area;
      if (!rc && exact) rc = bsr_exact_setup(L, st);
      const size_t vl = vec_len_of(L.n);
      if (!rc && (cudaMalloc(&L.bz, es * vl) != cudaSuccess || cudaMalloc(&L.bd, es * vl) != cudaSuccess))
        rc = cuda_fail(cudaErrorMemoryAllocation, "BSR work vectors");
      if (!rc) {
        cudaMemsetAsync(L.bz, 0, es * vl, st);
        cudaMemsetAsync(L.bd, 0, es * vl, st);
      }
    }
    if (rc) return fail(rc);
  }
  int rc = coarse_setup(h->levels.back(), h->d_flag, st);
  if (rc) return fail(rc);
  // exact BSR: the last smoothing level's S factored once (the bottom of the multigrid
  // preconditioner of the finer levels' Schur-complement solves)
  if (o->smoother == BMG_BSR_EXACT && h->levels.size() >= 3 &&
      (rc = bsr_exact_bottom_setup(h->levels[h->levels.size() - 2], h->d_flag, st)))
    return fail(rc);
  h->fine_op = s->fine;
  h->fine_op.owns_coefs = false;
  if ((rc = tune_hierarchy(h, st))) return fail(rc);
  int hflag = 0;
  cudaError_t e = cudaMemcpyAsync(&hflag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(cuda_fail(e, "bmg_setup_hierarchy"));
  if (hflag) {
    set_error(hflag & kErrTmaTimeout ? "a bulk-copy wait timed out during tile tuning"
              : hflag & 1 ? "a Vanka patch matrix is singular" : "the coarsest operator is singular");
    return fail(BMG_ERR_SINGULAR);
  }
  *out = h;
  return BMG_OK;
}

extern "C" int bmg_hierarchy_levels(const bmg_hierarchy *h) { return h ? (int)h->levels.size() : 0; }

extern "C" int bmg_hierarchy_schur_iters(const bmg_hierarchy *h) {
  return h && h->opts.smoother == BMG_BSR_EXACT ? h->schur_iters_max : -1;
}

extern "C" int bmg_hierarchy_tile(const bmg_hierarchy *h, int level, int kernel) {
  if (!h || level < 0 || level >= (int)h->levels.size()) return -1;
  const Level &L = h->levels[level];
  switch (kernel) {
    case BMG_PROF_APPLY: return L.tile_apply == 5 && !L.tma ? 0 : L.tile_apply;
    case BMG_PROF_VANKA: return L.tile_vanka;
    case BMG_PROF_VANKA_U: return L.tile_vanka_u;
    default: return -1;
  }
}

static void drop_graphs(bmg_hierarchy *h);

extern "C" void bmg_destroy_hierarchy(bmg_hierarchy *h) {
  if (!h) return;
  drop_graphs(h);
  for (auto &L : h->levels) free_level(L);
  cudaFree(h->d_flag);
  cudaFree(h->V); cudaFree(h->Z); cudaFree(h->w); cudaFree(h->r); cudaFree(h->xb);
  cudaFree(h->V32);
  cudaFree(h->partial); cudaFree(h->dres);
  cudaFreeHost(h->hres);
  cudaFree(h->hostbuf_b); cudaFree(h->hostbuf_x);
  delete h;
}

// ---- V-cycle ---------------------------------------------------------------------------
// One relaxation x <- x + omega M^{-1} r; assign: x is zero on entry (first pre-smoothing
// step from the zero initial guess), so the kernel writes x instead of updating it.
template <typename T>
static int smooth(bmg_hierarchy *h, const Level &L, const T *r, T *x, cudaStream_t st,
                  bool assign = false) {
  if (h->opts.smoother == BMG_VANKA) return launch_vanka_sweep<T>(L, r, x, (T)h->opts.omega, st, assign);
  if (h->opts.smoother == BMG_BSR_EXACT) {
    if constexpr (std::is_same<T, double>::value)
      return launch_bsr_exact_sweep(h->levels.data(), (int)h->levels.size() - 1, (int)(&L - h->levels.data()), r,
                                    x, h->opts.omega, st, assign, &h->schur_iters_max);
    return arg_error("exact BSR runs in FP64 only");
  }
  return launch_bsr_sweep<T>(L, r, x, (T)h->opts.omega, st, assign);
}

template <typename T>
static int vcycle_level(bmg_hierarchy *h, size_t l, const T *rhs, T *z, cudaStream_t st) {
  const Level &L = h->levels[l];
  if (l + 1 == h->levels.size()) return launch_coarse_solve<T>(L, rhs, z, st);
  int rc;
  const size_t vl = vec_len_of(L.n);
  T *t = (T *)L.t;
  if (h->opts.nu1 == 0 && (rc = launch_fill<T>(z, T(0), vl, st))) return rc;
  for (int s = 0; s < h->opts.nu1; ++s) {
    if (s == 0) {
      rc = smooth<T>(h, L, rhs, z, st, true);    // zero initial guess: residual = rhs
    } else {
      if ((rc = launch_apply<T>(L, z, rhs, t, true, 1, 0, st))) return rc;
      rc = smooth<T>(h, L, t, z, st);
    }
    if (rc) return rc;
  }
  const T *res = rhs;
  if (h->opts.nu1 > 0) {
    if ((rc = launch_apply<T>(L, z, rhs, t, true, 1, 0, st))) return rc;
    res = t;
  }
  const Level &C = h->levels[l + 1];
  if ((rc = launch_restrict<T>(L, C, res, (T *)C.rhs, st))) return rc;
  if ((rc = vcycle_level<T>(h, l + 1, (const T *)C.rhs, (T *)C.z, st))) return rc;
  if (h->opts.gamma == 2 && l + 2 < h->levels.size()) {
    // W-cycle: a second coarse cycle on the residual left by the first, added to its result
    // (the coarsest level's direct solve needs none)
    if ((rc = launch_apply<T>(C, (const T *)C.z, (const T *)C.rhs, (T *)C.t2, true, 1, 0, st))) return rc;
    if ((rc = vcycle_level<T>(h, l + 1, (const T *)C.t2, (T *)C.wz, st))) return rc;
    if ((rc = launch_add<T>((T *)C.z, (const T *)C.wz, vec_len_of(C.n), st))) return rc;
  }
  if ((rc = launch_prolong_add<T>(L, C, (const T *)C.z, z, st))) return rc;
  for (int s = 0; s < h->opts.nu2; ++s) {
    if ((rc = launch_apply<T>(L, z, rhs, t, true, 1, 0, st))) return rc;
    if ((rc = smooth<T>(h, L, t, z, st))) return rc;
  }
  return BMG_OK;
}

static int vcycle_direct(bmg_hierarchy *h, const double *r, double *z, cudaStream_t st) {
  if (h->opts.precision == BMG_FP64) return vcycle_level<double>(h, 0, r, z, st);
  Level &L = h->levels[0];
  const size_t vl = vec_len_of(L.n);
  int rc = launch_convert_d2f(r, (float *)L.rhs, vl, st);
  if (rc) return rc;
  if ((rc = vcycle_level<float>(h, 0, (const float *)L.rhs, (float *)L.t2, st))) return rc;
  return launch_convert_f2d((const float *)L.t2, z, vl, st);
}

static void drop_graphs(bmg_hierarchy *h) {
  for (auto &g : h->vgraphs) cudaGraphExecDestroy(g.exec);
  h->vgraphs.clear();
}

// One V-cycle.  A cycle is a fixed sequence of some tens of small launches, most of them on the
// coarse levels where each costs more to launch than to run, so after a first cycle launched
// kernel by kernel (which also runs every one-time initialisation of the kernels it uses) the
// sequence is captured once per (r, z) pair as a CUDA graph and replayed with one launch.
// Graphs are not used on the legacy default stream (it cannot be captured), inside a capture
// of the caller's (the launches then join that capture), or while bmg_use_graphs(0) is in
// effect.  Kernel timing (bmg_profile_start) sees only launches made kernel by kernel.
constexpr size_t kMaxVcGraphs = 160;

static int vcycle_any(bmg_hierarchy *h, const double *r, double *z, cudaStream_t st) {
  if (!g_use_graphs.load() || st == nullptr || h->vcycles_direct == 0 || h->graphs_failed ||
      capturing(st) || h->opts.smoother == BMG_BSR_EXACT) {
    ++h->vcycles_direct;
    return vcycle_direct(h, r, z, st);
  }
  for (const auto &g : h->vgraphs)
    if (g.r == r && g.z == z) {
      BMG_CUDA(cudaGraphLaunch(g.exec, st));
      g_launches += g.kernels;
      return BMG_OK;
    }
  if (h->vgraphs.size() >= kMaxVcGraphs) drop_graphs(h);
  const long long before = g_launches.load();
  BMG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  int rc = vcycle_direct(h, r, z, st);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  g_launches = before;                      // the captured launches have not run
  if (rc || e != cudaSuccess) {              // launch kernel by kernel from now on
    if (graph) cudaGraphDestroy(graph);
    (void)cudaGetLastError();
    h->graphs_failed = true;
    ++h->vcycles_direct;
    return vcycle_direct(h, r, z, st);
  }
  VcGraph g;
  g.r = r;
  g.z = z;
  size_t nodes = 0;
  e = cudaGraphGetNodes(graph, nullptr, &nodes);
  if (e == cudaSuccess) e = cudaGraphInstantiateWithFlags(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    h->graphs_failed = true;
    ++h->vcycles_direct;
    return vcycle_direct(h, r, z, st);
  }
  g.kernels = (long long)nodes;
  h->vgraphs.push_back(g);
  BMG_CUDA(cudaGraphLaunch(g.exec, st));
  g_launches += g.kernels;
  return BMG_OK;
}

extern "C" int bmg_vcycle(bmg_hierarchy *h, const double *r, double *z, void *stream) {
  if (!h || !r || !z) return arg_error("bmg_vcycle: NULL argument");
  if (r == z) return arg_error("bmg_vcycle: z may not alias r");
  return vcycle_any(h, r, z, (cudaStream_t)stream);
}

// ---- FGMRES ----------------------------------------------------------------------------
static const int kDotBlocks = 152 * 4;

static int ensure_krylov(bmg_hierarchy *h, int m, bool need32) {
  if (h->m_alloc >= m) {
    if (need32 && !h->V32) BMG_CUDA(cudaMalloc(&h->V32, sizeof(float) * vec_len_of(h->sys->n) * (h->m_alloc + 1)));
    return BMG_OK;
  }
  cudaFree(h->V); cudaFree(h->Z); cudaFree(h->w); cudaFree(h->r); cudaFree(h->V32);
  cudaFree(h->partial); cudaFree(h->dres); cudaFreeHost(h->hres);
  h->V = h->Z = h->w = h->r = h->partial = h->dres = h->hres = nullptr;
  h->V32 = nullptr;
  h->m_alloc = 0;
  const size_t vl = vec_len_of(h->sys->n);
  BMG_CUDA(cudaMalloc(&h->V, sizeof(double) * vl * (m + 1)));
  if (need32) BMG_CUDA(cudaMalloc(&h->V32, sizeof(float) * vl * (m + 1)));
  BMG_CUDA(cudaMalloc(&h->Z, sizeof(double) * vl * m));
  BMG_CUDA(cudaMalloc(&h->w, sizeof(double) * vl));
  BMG_CUDA(cudaMalloc(&h->r, sizeof(double) * vl));
  BMG_CUDA(cudaMalloc(&h->partial, sizeof(double) * std::max(kDotBlocks, kGsMaxBlocks) * (m + 2)));
  BMG_CUDA(cudaMalloc(&h->dres, sizeof(double) * 4 * (m + 2)));
  BMG_CUDA(cudaMallocHost(&h->hres, sizeof(double) * 4 * (m + 2)));
  h->m_alloc = m;
  return BMG_OK;
}

extern "C" int bmg_fgmres_solve(bmg_hierarchy *h, const double *b, double *x,
                                const bmg_krylov_opts *o, bmg_solve_info *info, void *stream) {
  auto t0 = std::chrono::steady_clock::now();
  if (!h || !b || !x || !o) return arg_error("bmg_fgmres_solve: NULL argument");
  if (b == x) return arg_error("bmg_fgmres_solve: x may not alias b");
  if (!(o->rtol > 0.0 && o->rtol < 1.0) || o->restart < 1 || o->restart > 200 || o->maxit < 0)
    return arg_error("bmg_fgmres_solve: need 0 < rtol < 1, 1 <= restart <= 200, maxit >= 0");
  if (o->arnoldi != BMG_ARNOLDI_FP64 && o->arnoldi != BMG_ARNOLDI_MIXED)
    return arg_error("bmg_fgmres_solve: arnoldi must be BMG_ARNOLDI_FP64 or BMG_ARNOLDI_MIXED");
  const bool mixed = o->arnoldi == BMG_ARNOLDI_MIXED;
  cudaStream_t st = (cudaStream_t)stream;
  const int m = o->restart;
  int rc = ensure_krylov(h, m, mixed);
  if (rc) return rc;
  const bmg_system *s = h->sys;
  const size_t vl = vec_len_of(s->n);
  double *hr = h->hres;
  if (o->x0_is_zero && (rc = launch_fill<double>(x, 0.0, vl, st))) return rc;
  // ||b||
  if ((rc = launch_dots(nullptr, vl, 0, b, vl, h->partial, kDotBlocks, h->dres, st))) return rc;
  BMG_CUDA(cudaMemcpyAsync(hr, h->dres, sizeof(double), cudaMemcpyDeviceToHost, st));
  BMG_CUDA(cudaStreamSynchronize(st));
  const double bnorm = std::sqrt(hr[0]);
  bmg_solve_info inf;
  std::memset(&inf, 0, sizeof(inf));
  inf.status = BMG_MAXIT;
  if (!std::isfinite(bnorm)) {
    set_error("bmg_fgmres_solve: right-hand side is not finite");
    return BMG_ERR_NONFINITE;
  }
  if (bnorm == 0.0) {
    if ((rc = launch_fill<double>(x, 0.0, vl, st))) return rc;
    BMG_CUDA(cudaStreamSynchronize(st));
    inf.status = BMG_CONVERGED;
    if (info) *info = inf;
    return BMG_OK;
  }
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  auto Hij = [&](int i, int j) -> double & { return H[(size_t)i * m + j]; };
  const size_t ldv = vl;
  double est = 1.0;
  for (;;) {
    // true residual
    if ((rc = launch_apply<double>(h->fine_op, x, b, h->r, true, 1, 0, st))) return rc;
    if ((rc = launch_dots(nullptr, vl, 0, h->r, vl, h->partial, kDotBlocks, h->dres, st))) return rc;
    BMG_CUDA(cudaMemcpyAsync(hr, h->dres, sizeof(double), cudaMemcpyDeviceToHost, st));
    BMG_CUDA(cudaStreamSynchronize(st));
    const double beta = std::sqrt(hr[0]);
    inf.relres = beta / bnorm;
    if (!std::isfinite(beta)) { inf.status = BMG_DIVERGED; break; }
    if (beta <= o->rtol * bnorm) { inf.status = BMG_CONVERGED; break; }
    if (inf.iters >= o->maxit) { inf.status = BMG_MAXIT; break; }
    if (inf.status == BMG_BREAKDOWN) break;
    inf.restarts++;
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    BMG_CUDA(cudaMemcpyAsync(h->dres + 3 * (m + 2), &beta, sizeof(double), cudaMemcpyHostToDevice, st));
    if ((rc = mixed ? launch_scale2(h->r, h->V, h->V32, h->dres + 3 * (m + 2), vl, st)
                    : launch_scale(h->r, h->V, h->dres + 3 * (m + 2), vl, st))) return rc;
    int k = 0;
    bool stop = false;
    for (int j = 0; j < m && !stop; ++j) {
      double *vj = h->V + (size_t)j * ldv;
      double *zj = h->Z + (size_t)j * ldv;
      if ((rc = vcycle_any(h, vj, zj, st))) return rc;
      if ((rc = launch_apply<double>(h->fine_op, zj, nullptr, h->w, false, 1, 0, st))) return rc;
      double *d1 = h->dres, *d2 = h->dres + (m + 2), *d3 = h->dres + 2 * (m + 2);
      if (mixed) {
        // CGS2: h1 = V^T w (from the FP32 copy of V); w -= V h1 (FP64) fused with h2 = V^T w;
        // w -= V h2 fused with ||w||^2 (both double-float products on the FP32 pipe)
        if ((rc = launch_dots32(h->V32, ldv, j + 1, h->w, vl, h->partial, kGsMaxBlocks, d1, st))) return rc;
        if ((rc = launch_update_dots_df(h->w, h->V, ldv, j + 1, d1, vl, h->partial, kGsMaxBlocks, d2, st)))
          return rc;
        if ((rc = launch_correct_df_norm(h->w, h->V, ldv, j + 1, d2, vl, h->partial, kDotBlocks, d3, st)))
          return rc;
      } else {
        // CGS2 in FP64: h1 = V^T w; w -= V h1 fused with h2 = V^T w; w -= V h2 fused with ||w||^2
        if ((rc = launch_dots_f64(h->w, h->V, ldv, j + 1, vl, h->partial, kGsMaxBlocks, d1, st))) return rc;
        if ((rc = launch_update_dots_f64(h->w, h->V, ldv, j + 1, d1, vl, h->partial, kGsMaxBlocks, d2, st)))
          return rc;
        if ((rc = launch_correct_f64_norm(h->w, h->V, ldv, j + 1, d2, vl, h->partial, kDotBlocks, d3, st)))
          return rc;
      }
      BMG_CUDA(cudaMemcpyAsync(hr, h->dres, sizeof(double) * 3 * (m + 2), cudaMemcpyDeviceToHost, st));
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
        BMG_CUDA(cudaMemcpyAsync(h->dres + 3 * (m + 2), &Hij(j + 1, j), sizeof(double), cudaMemcpyHostToDevice, st));
        if ((rc = mixed ? launch_scale2(h->w, h->V + (size_t)(j + 1) * ldv, h->V32 + (size_t)(j + 1) * ldv,
                                        h->dres + 3 * (m + 2), vl, st)
                        : launch_scale(h->w, h->V + (size_t)(j + 1) * ldv, h->dres + 3 * (m + 2), vl, st)))
          return rc;
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
    // y = H^{-1} g, x += Z y
    for (int i = k - 1; i >= 0; --i) {
      double acc = g[i];
      for (int c = i + 1; c < k; ++c) acc -= Hij(i, c) * y[c];
      y[i] = Hij(i, i) != 0.0 ? acc / Hij(i, i) : 0.0;
    }
    BMG_CUDA(cudaMemcpyAsync(h->dres, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
    if ((rc = launch_axpy_multi(x, h->Z, ldv, k, h->dres, vl, st))) return rc;
  }
  BMG_CUDA(cudaStreamSynchronize(st));
  if (h->opts.precision == BMG_FP32) {         // a timed-out TMA wait leaves its CTA's output unset
    int flag = 0;
    BMG_CUDA(cudaMemcpy(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag & kErrTmaTimeout) {
      set_error("bmg_fgmres_solve: a bulk-copy wait in the FP32 operator timed out");
      return BMG_ERR_CUDA;
    }
  }
  inf.relres_est = est;
  inf.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  return BMG_OK;
}

extern "C" int bmg_fgmres_solve_host(bmg_hierarchy *h, const double *b_host, double *x_host,
                                     const bmg_krylov_opts *o, bmg_solve_info *info,
                                     void *stream) {
  if (!h || !b_host || !x_host || !o) return arg_error("bmg_fgmres_solve_host: NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t vl = vec_len_of(h->sys->n);
  if (!h->hostbuf_b) BMG_CUDA(cudaMalloc(&h->hostbuf_b, sizeof(double) * vl));
  if (!h->hostbuf_x) BMG_CUDA(cudaMalloc(&h->hostbuf_x, sizeof(double) * vl));
  BMG_CUDA(cudaMemcpyAsync(h->hostbuf_b, b_host, sizeof(double) * vl, cudaMemcpyHostToDevice, st));
  if (!o->x0_is_zero)
    BMG_CUDA(cudaMemcpyAsync(h->hostbuf_x, x_host, sizeof(double) * vl, cudaMemcpyHostToDevice, st));
  int rc = bmg_fgmres_solve(h, h->hostbuf_b, h->hostbuf_x, o, info, stream);
  if (rc) return rc;
  BMG_CUDA(cudaMemcpyAsync(x_host, h->hostbuf_x, sizeof(double) * vl, cudaMemcpyDeviceToHost, st));
  BMG_CUDA(cudaStreamSynchronize(st));
  return BMG_OK;
}
