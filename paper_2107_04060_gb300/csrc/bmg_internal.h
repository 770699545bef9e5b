// Internal declarations of the biotmg library (not part of the C ABI).
//
// Structured-grid layout: every DoF type of an n-cell grid lives in an (n+1) x pitch block
// indexed [j][i]; see include/biotmg.h for the block order and the valid ranges.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/biotmg.h"

namespace bmg {

// DoF block order inside a vector.
enum Block { UX = 0, UY, BH, BV, BD, WH, WV, WD, PL, PU, NBLK };

inline int pitch_of(int n) { return ((n + 1) + 7) & ~7; }
inline size_t block_len_of(int n) { return (size_t)(n + 1) * (size_t)pitch_of(n); }
inline size_t vec_len_of(int n) { return (size_t)NBLK * block_len_of(n); }

// Grid shape passed to every kernel.
struct Grid {
  int n;        // cells per side
  int pitch;    // row pitch (elements)
  size_t blk;   // elements per block
};

inline Grid grid_of(int n) { return Grid{n, pitch_of(n), block_len_of(n)}; }

// --------------------------------------------------------------------------------------
// Element integrals of one triangle shape (o = 0: lower-left L, o = 1: upper-right U),
// local DoF order (ux v0..v2, uy v0..v2, bubble e0..e2 | RT0 e0..e2 | P0); local edge k is
// opposite local vertex k.  L(i,j) = {(i,j), (i+1,j), (i,j+1)}, edges (d(i,j), v(i,j),
// h(i,j)); U(i,j) = {(i+1,j+1), (i,j+1), (i+1,j)}, edges (d(i,j), v(i+1,j), h(i,j+1)).
struct ElemIntegrals {
  double Aeps[2][9][9];   // int eps(phi_a) : eps(phi_b)
  double Ddiv[2][9][9];   // int div phi_a div phi_b (exact; the divergence of a bubble is linear)
  double g[2][9];         // int div phi_a
  double Mw[2][3][3];     // int psi_a . psi_b
  double dw[2][3];        // int div psi_a
  double area;            // |T| = h^2 / 2
};
void element_integrals(double h, ElemIntegrals *out);

// Operator coefficients of one level in arithmetic type T (kernel parameter).
//   y_u = A u + g s,  s = lam_area (g.u) - alpha p
//   y_w = kinv_T (M1 w) - dw p        (or Wm_T w with a per-triangle 3x3 RT0 mass)
//   y_p = -alpha (g.u) - dw.w - pp p
template <typename T>
struct OpCoefs {
  T A[2][81];   // 2 mu Aeps
  T g[2][9];
  T M1[2][9];   // tau * Mw (unit permeability)
  T dw[2][3];   // tau * dw
  T lam_area;   // lambda / |T|
  T alpha;
  T pp;         // (1/M) |T|
};

// Structural nonzeros of the element integrals on the two reference right triangles (the
// same pattern for L and U; stiffness-type integrals are scale-free in 2D, so the pattern
// holds for every h): bit b of row a set <=> Aeps[a][b] != 0; the g and unit-mass patterns.
// verify_elem_nonzeros() checks them against element_integrals() before the first assembly.
constexpr unsigned short kAepsRows[9] = {0x0DF, 0x0C3, 0x05D, 0x17D, 0x05D, 0x168, 0x1FF, 0x1C3, 0x1E8};
constexpr unsigned short kGNonzero = 0x1EB;          // g[2] = g[4] = 0
constexpr unsigned short kMwRows[3] = {0x1, 0x6, 0x6};
__host__ __device__ constexpr bool aeps_nonzero(int a, int b) { return (kAepsRows[a] >> b) & 1; }
__host__ __device__ constexpr bool g_nonzero(int k) { return (kGNonzero >> k) & 1; }
__host__ __device__ constexpr bool mw_nonzero(int a, int b) { return (kMwRows[a] >> b) & 1; }
bool verify_elem_nonzeros(std::string *why);

struct PhysParams {
  double lambda, mu, tau, alpha, inv_M;
  bool exact_divdiv = false;   // lambda (div u, div v) integrated exactly (Sec. 2.1) instead of
                               // the reduced quadrature (Sec. 2.3): dense displacement element
                               // matrices 2 mu A_eps + lambda D, lam_area = 0
};

void make_coefs(const PhysParams &p, int n, OpCoefs<double> *c64, OpCoefs<float> *c32);
// Galerkin coarse coefficients: c64 / c32 hold the rediscretised coefficients of the coarse
// level on entry; the displacement block is replaced by the Galerkin product of the fine
// level's (dense elasticity element matrices, fine lambda / |T|).
void galerkin_coarsen_coefs(const OpCoefs<double> &fine, OpCoefs<double> *c64, OpCoefs<float> *c32);

// --------------------------------------------------------------------------------------
// Transfer stencil tables (pure geometry; identical on every level).
//   prolongation: fine value (type t, parity class c = (i&1) + 2 (j&1)) at (i, j) =
//       sum_k coef_k * coarse[ctype_k][(j>>1) + dJ_k][(i>>1) + dI_k]
//   restriction:  coarse value (type t) at (I, J) = sum_k coef_k * fine[ftype_k][2J + dj_k][2I + di_k]
struct StencilEntry {
  int8_t type, di, dj, pad;
  float coef32;                // coef rounded to FP32 (the FP32 transfers' operand)
  double coef;
};
constexpr int kMaxPro = 24;   // entries per (fine type, parity)
constexpr int kMaxRes = 48;   // entries per coarse type
struct TransferTables {
  StencilEntry pro[NBLK][4][kMaxPro];
  int npro[NBLK][4];
  StencilEntry res[NBLK][kMaxRes];
  int nres[NBLK];
  // Galerkin coarsening of a per-triangle RT0 mass: coarse triangle (o) has children
  // c = 0..3 of orientation child_o at fine cell (2I + cdi, 2J + cdj); Q maps the coarse
  // triangle's 3 local RT0 DoFs to the child's 3 local RT0 DoFs.
  int child_o[2][4], child_di[2][4], child_dj[2][4];
  double Q[2][4][3][3];
};
void build_transfer_tables(TransferTables *t);

// --------------------------------------------------------------------------------------
struct TmaMaps;                // tensor maps of a level's FP32 operator input (operator.cu)
constexpr int kErrTmaTimeout = 1 << 16;   // device error flag: a TMA wait ran out

struct Level {
  int n = 0;
  bool owns_coefs = true;      // false for a hierarchy's view of its system's fine level
  Grid g{};
  bool wm_full = false;        // per-triangle 3x3 RT0 mass (coarse levels, varying K)
  bool uniform = false;        // every triangle has the same coefficients
  bool dense_a = false;        // Galerkin coarse level: dense elasticity element matrices
  bool solve64 = false;        // FP32 V-cycle: Vanka patch solves in FP64 (BMG_PATCH_FP64)
  double *kinv64 = nullptr;    // [2][blk] per-triangle K^{-1} (wm_full == false)
  float *kinv32 = nullptr;
  double *wm64 = nullptr;      // [2][6][blk] symmetric 3x3 RT0 mass incl. tau (wm_full)
  float *wm32 = nullptr;
  OpCoefs<double> c64{};
  OpCoefs<float> c32{};
  // additive Vanka (20-DoF patches) or the displacement Vanka inside BSR (8-DoF)
  int nslots = 0;
  int *slot = nullptr;         // [(n+1) * (n+1)] patch -> inverse slot
  int psize = 0;               // 20 (Vanka) or 8 (BSR displacement patches)
  // uniform coefficients: the shared interior inverse in the symmetry-adapted basis (blocks
  // of 4, 5, 7, 4; row k holds block entries 0..size-1), verified against the dense inverse
  bool klein = false;
  double kb64[20][7] = {};
  float kb32[20][7] = {};
  double *pinv64 = nullptr;    // [patch_entries(psize)][nslots]: psize 20 packed symmetric
                               // (upper triangle, row-major), psize 8 full row-major
  float *pinv32 = nullptr;
  // BSR data
  double *dinv64 = nullptr;    // [3][blk] 1 / (tau D_w) per edge family
  float *dinv32 = nullptr;
  double *sinv64 = nullptr;    // [2][blk] omega_J / diag(S) per triangle
  float *sinv32 = nullptr;
  void *bz = nullptr, *bd = nullptr;   // BSR work vectors
  // exact BSR: conjugate gradients on S dp = B z - r_p over the two P0 blocks (length 2 blk)
  double s_c = 0.0;                    // (1/M + alpha^2/(lambda + mu)) |T|
  double *cg = nullptr;                // r, z, q, p[2] (5 x 2 blk), then the block partials
  int cg_grid = 0;                     // CTAs of the CG kernels (partials per reduction)
  int *cg_flag = nullptr;              // device [done, iterations]
  double *smg = nullptr;               // multigrid preconditioner of S: b, xa, xb, r, e (5 x 2 blk)
  double *sdense = nullptr;            // exact BSR, last smoothing level: dense S^{-1} (2 n^2 squared)
  // coarsest level: dense inverse on the free DoFs
  int nfree = 0;
  int *free_idx = nullptr;     // [nfree] vector positions of the free DoFs
  double *cinv64 = nullptr;    // [nfree][nfree]
  float *cinv32 = nullptr;
  // work vectors in the V-cycle precision
  void *rhs = nullptr, *z = nullptr, *t = nullptr, *t2 = nullptr;
  void *wz = nullptr;                  // W-cycle: result of the second coarse cycle
  // Tile shape of the operator / Vanka / displacement-Vanka launches on this level, chosen by
  // timing at setup (index into each kernel's candidate list; -1: the CTA-count rule).
  int tile_apply = -1, tile_vanka = -1, tile_vanka_u = -1;
  // FP32 operator with its input staged by TMA (tile index 5): tensor maps of the level's
  // work vectors and coefficients, and the device flag a timed-out wait sets
  TmaMaps *tma = nullptr;
  int *err = nullptr;
  // Device flag read by every kernel launched for this level (nullptr: always run).  Used by
  // graph-replayed solves: a kernel whose gate holds 0 returns at once.
  const int *gate = nullptr;
};

// Stored entries of one patch inverse: the 20 x 20 Vanka inverse is symmetric (the patch
// matrix V A V^T of the symmetric A) and kept as its upper triangle; the 8 x 8 one is full.
inline int patch_entries(int psize) { return psize == 20 ? 210 : psize * psize; }

// ---- programmatic dependent launch ------------------------------------------------------
// The kernels of the solve path are launched with programmatic stream serialisation and
// start with pdl_enter(): it waits until the grids they depend on have completed and their
// writes are visible (a no-op for a launch without a programmatic dependency), then lets the
// next kernel of the stream start launching, so its launch overlaps this kernel's last wave.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Kernel prologue: leave when a gate is present and closed.
#define BMG_GATE(g) if ((g) != nullptr && *(g) == 0) return

}  // namespace bmg

namespace bmg {
constexpr int kAdjBlocks = 152 * 8;   // CTAs of the adjoint-gradient reduction

// ---- batched launches: one kernel over several instances of one grid size -------------
// The per-instance arguments (vectors, coefficients, inverse tables, gate) sit in a device
// array; blockIdx.z (blockIdx.y for the coarse solve) selects the instance.  FP64 only.
constexpr int kApplyTiles = 5, kVankaTiles = 6;
size_t apply_args_bytes();
void make_apply_args(const Level &L, const double *x, const double *b, double *y, bool residual,
                     const int *gate, void *dst);
int launch_apply_batch(const void *d_args, int count, int n, int tile, cudaStream_t st);
int prepare_apply_batch();
// Tensor maps for the TMA-staged FP32 operator on inputs xa and xb (either may be NULL);
// leaves L.tma NULL (and the kernel unused) when they cannot be encoded.
int setup_apply_tma(Level &L, const float *xa, const float *xb);
void free_apply_tma(Level &L);
int default_apply_tile(int n, int count);
size_t vanka_args_bytes();
void make_vanka_args(const Level &L, const double *r, double *x, double omega, bool assign,
                     const int *gate, void *dst);
int launch_vanka_batch(const void *d_args, int count, int n, int tile, cudaStream_t st);
int default_vanka_tile(int n, int count);
struct TransferArgs {          // restriction: fine src -> coarse dst; prolongation: coarse src, fine dst (+=)
  Grid gf, gc;
  const double *src;
  double *dst;
  const int *gate;
};
int launch_restrict_batch(const TransferArgs *d_args, int count, int nf, cudaStream_t st);
int launch_prolong_batch(const TransferArgs *d_args, int count, int nf, cudaStream_t st);
struct CoarseArgs {
  const double *inv;           // [N][N]
  const int *free_idx;         // [N]
  const unsigned char *free_mask;   // [vl] 1 on the free DoFs
  int N;
  size_t vl;
  const double *r;
  double *z;
  const int *gate;
};
int launch_coarse_batch(const CoarseArgs *d_args, int count, int max_free, cudaStream_t st);
}

struct bmg_system {
  int n;
  bmg::PhysParams prm;
  bool uniform;                // K given as a constant
  double K_const;
  bmg::Level fine;             // coefficients of the fine level (kinv64/kinv32, coefs)
  double *adj_partial = nullptr;   // [2][kAdjBlocks] partial sums of the Lame gradients
};

namespace bmg {
// One V-cycle captured as a CUDA graph for a given (input, output) pair of device vectors.
struct VcGraph {
  const void *r = nullptr, *z = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;       // kernel nodes (added to the launch count per replay)
};
}  // namespace bmg

struct bmg_hierarchy {
  const bmg_system *sys;
  bmg_mg_opts opts;
  std::vector<bmg::Level> levels;
  std::vector<bmg::VcGraph> vgraphs;   // captured V-cycles (see vcycle_any)
  long long vcycles_direct = 0;        // cycles launched kernel by kernel
  bool graphs_failed = false;          // a capture failed: launch kernel by kernel from now on
  int *d_flag = nullptr;       // device error flag (singular pivots)
  int schur_iters_max = 0;     // exact BSR: most CG iterations one pressure step took
  bmg::Level fine_op;          // the system's fine level with the FP64 operator tile tuned
                               // for this device (FGMRES matvec and true residual)
  // FGMRES workspace (FP64)
  int m_alloc = 0;
  double *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr, *xb = nullptr;
  float *V32 = nullptr;        // FP32 copy of the basis (first Gram-Schmidt pass)
  double *partial = nullptr;   // [kMaxDot][nblocks]
  double *dres = nullptr;      // device results of reductions
  double *hres = nullptr;      // pinned host mirror
  double *hostbuf_b = nullptr, *hostbuf_x = nullptr;   // device copies for the host API
};

// ---- error reporting ------------------------------------------------------------------
namespace bmg {
void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
}  // namespace bmg

#define BMG_CUDA(call)                                               \
  do {                                                               \
    cudaError_t e_ = (call);                                         \
    if (e_ != cudaSuccess) return bmg::cuda_fail(e_, #call);         \
  } while (0)

namespace bmg {
// kernels launched by this library (host-side count; solves on distinct handles may run on
// several host threads at once)
extern std::atomic<long long> g_launches;
}
#define BMG_CHECK_LAUNCH(what)                                       \
  do {                                                               \
    ++bmg::g_launches;                                               \
    cudaError_t e_ = cudaGetLastError();                             \
    if (e_ != cudaSuccess) return bmg::cuda_fail(e_, what);          \
  } while (0)

// ---- kernel timing (bmg_profile_start / bmg_profile_stop) ------------------------------
namespace bmg {
bool prof_on(int kernel, int n);
bool capturing(cudaStream_t st);     // st is being captured into a graph
cudaEvent_t prof_begin(cudaStream_t st);
void prof_end(cudaStream_t st, cudaEvent_t e0, double cells);
}  // namespace bmg

#define BMG_PROF_BEGIN(kid, n, st) \
  const bool prof_ = bmg::prof_on(kid, n) && !bmg::capturing(st); \
  cudaEvent_t prof_e0_ = prof_ ? bmg::prof_begin(st) : nullptr
#define BMG_PROF_END(st, cells) if (prof_) bmg::prof_end(st, prof_e0_, cells)

// ---- kernel launchers (implemented in the .cu files) -----------------------------------
namespace bmg {
template <typename T>
int launch_apply(const Level &L, const T *x, const T *b, T *y, bool residual, int batch,
                 size_t bstride, cudaStream_t st);
int vanka_klein_setup(Level &L, cudaStream_t st);
int launch_vanka_setup(const Level &L, const int *rep_i, const int *rep_j, int nrep,
                       double p_shift_area, int psize, int *d_flag, cudaStream_t st);
template <typename T>
int launch_vanka_sweep(const Level &L, const T *r, T *x, T omega, cudaStream_t st, bool assign);
template <typename T>
int launch_restrict(const Level &fine, const Level &coarse, const T *rf, T *rc, cudaStream_t st);
template <typename T>
int launch_prolong_add(const Level &fine, const Level &coarse, const T *xc, T *xf,
                       cudaStream_t st);
int launch_coarsen_wmass(const Level &fine, Level &coarse, cudaStream_t st);
int upload_transfer_tables();
int coarse_setup(Level &L, int *d_flag, cudaStream_t st);
template <typename T>
int launch_coarse_solve(const Level &L, const T *r, T *z, cudaStream_t st);
int launch_bsr_setup(Level &L, double omega_J, double c_fs_area, cudaStream_t st);
int bsr_exact_setup(Level &L, cudaStream_t st);
int bsr_exact_bottom_setup(Level &L, int *d_flag, cudaStream_t st);
// dense Gauss-Jordan inversion kernels (coarse.cu), also used for exact BSR's bottom level
__global__ void gj_pivot_kernel(double *Aug, int N, int k, double *fac, double tol, int *flag);
__global__ void gj_eliminate_kernel(double *Aug, int N, int k, const double *fac);
__global__ void extract_inverse_kernel(const double *Aug, int N, double *inv64, float *inv32);
int launch_bsr_exact_sweep(const Level *levels, int nsmooth, int l, const double *r, double *x, double omega,
                           cudaStream_t st, bool assign, int *iters_max);
template <typename T>
int launch_bsr_sweep(const Level &L, const T *r, T *x, T omega, cudaStream_t st, bool assign);
// vector kernels
template <typename T>
int launch_fill(T *x, T v, size_t n, cudaStream_t st, const int *gate = nullptr);
template <typename T>
int launch_add(T *y, const T *x, size_t n, cudaStream_t st);      // y += x
int launch_convert_d2f(const double *x, float *y, size_t n, cudaStream_t st);
int launch_convert_f2d(const float *x, double *y, size_t n, cudaStream_t st);
int launch_dots(const double *V, size_t ldv, int k, const double *w, size_t n,
                double *partial, int nblocks, double *out, cudaStream_t st);
int launch_update(double *w, const double *V, size_t ldv, int k, const double *h, size_t n,
                  cudaStream_t st);
// Gram-Schmidt kernels with blockDim (32, TY): one warp per KQ basis vectors, so
// k <= KQ * MaxTY (covers the largest restart length, kMaxBasisVecs).  kGsMaxBlocks bounds
// their grids (the partial-sum buffer holds kGsMaxBlocks * k entries).
constexpr int kMaxBasisVecs = 200;
constexpr int kDotsKQ = 16, kDotsMaxTY = 13;      // dots32
constexpr int kUpdKQ = 12, kUpdMaxTY = 17;        // gs_pass (update_dots_df/_f64, dots_f64)
constexpr int kGsMaxBlocks = 152 * 32;
static_assert(kDotsKQ * kDotsMaxTY >= kMaxBasisVecs && kUpdKQ * kUpdMaxTY >= kMaxBasisVecs,
              "Gram-Schmidt kernels must cover every restart length");
int launch_update_dots_df(double *w, const double *V, size_t ldv, int k, const double *h, size_t n,
                         double *partial, int max_blocks, double *out, cudaStream_t st);
int launch_update_dots_f64(double *w, const double *V, size_t ldv, int k, const double *h, size_t n,
                           double *partial, int max_blocks, double *out, cudaStream_t st);
int launch_dots_f64(const double *w, const double *V, size_t ldv, int k, size_t n, double *partial,
                    int max_blocks, double *out, cudaStream_t st);
int launch_correct_f64_norm(double *w, const double *V, size_t ldv, int k, const double *h, size_t n,
                            double *partial, int nblocks, double *out, cudaStream_t st);
int launch_scale(const double *w, double *v, const double *s, size_t n, cudaStream_t st);
int launch_scale2(const double *w, double *v, float *v32, const double *s, size_t n, cudaStream_t st);
int launch_dots32(const float *V, size_t ldv, int k, const double *w, size_t n, double *partial,
                  int max_blocks, double *out, cudaStream_t st);
int launch_correct_df_norm(double *w, const double *V, size_t ldv, int k, const double *h, size_t n,
                           double *partial, int nblocks, double *out, cudaStream_t st);
int launch_axpy_multi(double *x, const double *Z, size_t ldz, int k, const double *y,
                      size_t n, cudaStream_t st);
}  // namespace bmg
