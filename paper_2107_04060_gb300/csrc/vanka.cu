// Additive Vanka relaxation on vertex patches (Sec. 3.2.1, Fig. 3).
//
// Patch of vertex v = (i, j), fixed slot order (20 slots):
//   0, 1      ux, uy at v
//   2 + e     bubble on incident edge e,  8 + e  RT0 on edge e, e = 0..5:
//             E0 = h(i,j), E1 = v(i,j), E2 = h(i-1,j), E3 = v(i,j-1), E4 = d(i-1,j), E5 = d(i,j-1)
//   14 + t    P0 on incident triangle t = 0..5:
//             L(i,j), L(i-1,j), L(i,j-1), U(i-1,j), U(i-1,j-1), U(i,j-1)
// The 8-DoF displacement patch (Fig. 3 left, used inside Braess-Sarazin) is slots 0..7 of
// A_u^RQ.  Slots of DoFs that do not exist or are constrained carry an identity row and
// column, so every patch is a fixed-size system; their residual entries are zero.
//
// Setup: the patch matrix V_l A V_l^T is the sum of the element matrices of the six
// incident triangles restricted to the patch, inverted in FP64 by Gauss-Jordan with
// partial pivoting (one thread per distinct patch).  Patches with identical matrices share
// one inverse ("slot"): with uniform coefficients every interior patch uses slot 0.
//
// Sweep: x <- x + omega * sum_l V_l^T D_l (V_l A V_l^T)^{-1} V_l r with the natural weights
// D_l (1 for a vertex DoF, 1/2 for an edge DoF, 1/3 for a triangle DoF: every edge lies in
// the patches of its two end points, every triangle in those of its three vertices).
// One CTA computes the local solves of a 32 x 8 block of patches into shared memory and
// then gathers the weighted corrections of the 31 x 7 positions whose patches it holds:
// deterministic, no atomics.
#include <cmath>
#include <cstring>

#include "bmg_internal.h"
#include "kernels_common.cuh"

namespace bmg {

// incident triangle t: cell offset, orientation, local index of v, local edge -> patch edge
__constant__ int c_tdi[6] = {0, -1, 0, -1, -1, 0};
__constant__ int c_tdj[6] = {0, 0, -1, 0, -1, -1};
__constant__ int c_to[6] = {0, 0, 0, 1, 1, 1};
__constant__ int c_tlv[6] = {0, 1, 2, 2, 0, 1};
__constant__ int c_temap[6][3] = {{-1, 1, 0}, {4, -1, 2}, {5, 3, -1},
                                  {4, 1, -1}, {-1, 3, 2}, {5, -1, 0}};

// Existence / freedom of the 20 patch slots of vertex (vi, vj).
__device__ __forceinline__ void patch_active(int vi, int vj, int n, bool act[20]) {
  const bool vf = vfree(vi, vj, n);
  act[0] = act[1] = vf;
  const bool ex[6] = {vi < n, vj < n, vi >= 1, vj >= 1, vi >= 1 && vj < n, vi < n && vj >= 1};
  const bool hfree = vj > 0 && vj < n, vfr = vi > 0 && vi < n;
  const bool bfree[6] = {hfree, vfr, hfree, vfr, true, true};
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    act[2 + e] = ex[e] && bfree[e];
    act[8 + e] = ex[e];
  }
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const int ci = vi + c_tdi[t], cj = vj + c_tdj[t];
    act[14 + t] = ci >= 0 && cj >= 0 && ci < n && cj < n;
  }
}

// ---- symmetry-adapted interior patch ---------------------------------------------------
// With uniform coefficients the matrix of an interior patch commutes with the signed slot
// permutations of the three symmetries of the triangulation around the vertex: the point
// reflection (ux, uy, bubble and flux DoFs change sign, E0<->E2, E1<->E3, E4<->E5, L(i,j) <->
// U(i-1,j-1), L(i-1,j) <-> U(i,j-1), L(i,j-1) <-> U(i-1,j)) and the reflections in the two
// diagonals through the vertex (the x <-> y one maps ux <-> uy, E0<->E1, E2<->E3, E4<->E5,
// L(i-1,j) <-> L(i,j-1), U(i-1,j) <-> U(i,j-1), with no sign change: the global normals
// (0,1), (1,0), (1,1)/sqrt2 map onto each other).  The four characters of this group split
// the 20 slots into blocks of 4, 5, 7 and 4: in the basis U (columns of +-1 entries, one per
// character and orbit) the inverse is block diagonal, x = U B U^T r with
// B = diag(1/d) U^T A^{-1} U diag(1/d), d_k = |U_k|^2.  klein_fwd forms U^T r and klein_inv
// forms U x' with butterflies of additions (32 each), so a patch solve costs 106 FMAs plus 64
// additions instead of 400 FMAs.  Transformed index k: block 0 = k 0..3, 1 = 4..8,
// 2 = 9..15, 3 = 16..19.
template <typename T>
__host__ __device__ __forceinline__ void klein_fwd(const T *r, T *q) {
  // bubbles E0..E3 (slots 2..5) and fluxes E0..E3 (slots 8..11): orbits of 4
  {
    const T s01 = r[2] + r[3], d01 = r[2] - r[3], s23 = r[4] + r[5], d23 = r[4] - r[5];
    q[10] = s01 + s23; q[0] = s01 - s23; q[17] = d01 + d23; q[4] = d01 - d23;
  }
  {
    const T s01 = r[8] + r[9], d01 = r[8] - r[9], s23 = r[10] + r[11], d23 = r[10] - r[11];
    q[12] = s01 + s23; q[1] = s01 - s23; q[18] = d01 + d23; q[6] = d01 - d23;
  }
  // pressures L(i-1,j), L(i,j-1), U(i-1,j), U(i,j-1) (slots 15, 16, 17, 19)
  {
    const T s = r[15] + r[16], d = r[15] - r[16], s2 = r[17] + r[19], d2 = r[17] - r[19];
    q[3] = s + s2; q[15] = s - s2; q[19] = d + d2; q[8] = d - d2;
  }
  // orbits of 2: (ux, uy), bubbles and fluxes on E4, E5, pressures L(i,j), U(i-1,j-1)
  q[9] = r[0] + r[1]; q[16] = r[0] - r[1];
  q[11] = r[6] + r[7]; q[5] = r[6] - r[7];
  q[13] = r[12] + r[13]; q[7] = r[12] - r[13];
  q[2] = r[14] + r[18]; q[14] = r[14] - r[18];
}

template <typename T>
__host__ __device__ __forceinline__ void klein_inv(const T *q, T *x) {
  {
    const T a = q[10] + q[0], b = q[10] - q[0], c = q[17] + q[4], d = q[17] - q[4];
    x[2] = a + c; x[3] = a - c; x[4] = b + d; x[5] = b - d;
  }
  {
    const T a = q[12] + q[1], b = q[12] - q[1], c = q[18] + q[6], d = q[18] - q[6];
    x[8] = a + c; x[9] = a - c; x[10] = b + d; x[11] = b - d;
  }
  {
    const T a = q[3] + q[15], b = q[3] - q[15], c = q[8] + q[19], d = q[8] - q[19];
    x[15] = a + c; x[16] = a - c; x[17] = b - d; x[19] = b + d;
  }
  x[0] = q[9] + q[16]; x[1] = q[9] - q[16];
  x[6] = q[11] + q[5]; x[7] = q[11] - q[5];
  x[12] = q[13] + q[7]; x[13] = q[13] - q[7];
  x[14] = q[2] + q[14]; x[18] = q[2] - q[14];
}

__host__ __device__ constexpr int klein_block_start(int k) {
  return k < 4 ? 0 : k < 9 ? 4 : k < 16 ? 9 : 16;
}
__host__ __device__ constexpr int klein_block_size(int k) {
  return k < 4 ? 4 : k < 9 ? 5 : k < 16 ? 7 : 4;
}

// Packed position of entry (r, c) of a symmetric 20 x 20 matrix (upper triangle, row-major).
__host__ __device__ __forceinline__ int sym20(int r, int c) {
  const int a = r < c ? r : c, b = r < c ? c : r;
  return a * 20 - (a * (a - 1)) / 2 + (b - a);
}

// Entry c of row r: for c >= r it is (r, c), at base(r) + c; for c < r it is (c, r), at
// base(c) + r, with base(a) = sym20(a, 0) - a = 19 a - a (a - 1) / 2 (a compile-time
// constant when c is an unrolled loop index).
__device__ __forceinline__ int sym20_row_base(int r) { return r * 19 - (r * (r - 1)) / 2; }

struct VankaSetupArgs {
  Grid g;
  const double *kinv;
  const double *wm;
  int wm_full;
  OpCoefs<double> c;
  double pshift_area;
  const int *rep_i, *rep_j;
  int nrep;
  int psize;
  double *inv64;
  float *inv32;
  int *flag;
};

__global__ void __launch_bounds__(64) vanka_setup_kernel(const __grid_constant__ VankaSetupArgs a) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.nrep) return;
  const int vi = a.rep_i[s], vj = a.rep_j[s];
  const int n = a.g.n, P = a.g.pitch;
  const int ps = a.psize;
  double M[20][20];
  for (int r = 0; r < 20; ++r)
    for (int c = 0; c < 20; ++c) M[r][c] = 0.0;
  bool act[20];
  patch_active(vi, vj, n, act);
  for (int t = 0; t < 6; ++t) {
    if (!act[14 + t]) continue;
    const int ci = vi + c_tdi[t], cj = vj + c_tdj[t], o = c_to[t], lv = c_tlv[t];
    const size_t co = (size_t)cj * P + ci;
    // local DoFs of the triangle that belong to the patch, with their slots
    int la[7], sl[7], nl = 0;
    la[nl] = lv; sl[nl++] = 0;
    la[nl] = 3 + lv; sl[nl++] = 1;
    for (int e = 0; e < 3; ++e)
      if (c_temap[t][e] >= 0) { la[nl] = 6 + e; sl[nl++] = 2 + c_temap[t][e]; }
    const int nu = nl;
    if (ps == 20) {
      for (int e = 0; e < 3; ++e)
        if (c_temap[t][e] >= 0) { la[nl] = 9 + e; sl[nl++] = 8 + c_temap[t][e]; }
      la[nl] = 12; sl[nl++] = 14 + t;
    }
    double W[3][3];
    if (a.wm_full) {
      const double *w = a.wm + (size_t)o * 6 * a.g.blk + co;
      const size_t b = a.g.blk;
      W[0][0] = w[0]; W[0][1] = W[1][0] = w[b]; W[0][2] = W[2][0] = w[2 * b];
      W[1][1] = w[3 * b]; W[1][2] = W[2][1] = w[4 * b]; W[2][2] = w[5 * b];
    } else {
      const double k = a.kinv[(size_t)o * a.g.blk + co];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) W[r][c] = k * a.c.M1[o][r * 3 + c];
    }
    for (int p = 0; p < nl; ++p)
      for (int q = 0; q < nl; ++q) {
        const int A = la[p], B = la[q];
        double v = 0.0;
        if (A < 9 && B < 9) v = a.c.A[o][A * 9 + B] + a.c.lam_area * a.c.g[o][A] * a.c.g[o][B];
        else if (A < 9 && B == 12) v = -a.c.alpha * a.c.g[o][A];
        else if (A == 12 && B < 9) v = -a.c.alpha * a.c.g[o][B];
        else if (A >= 9 && A < 12 && B >= 9 && B < 12) v = W[A - 9][B - 9];
        else if (A >= 9 && A < 12 && B == 12) v = -a.c.dw[o][A - 9];
        else if (A == 12 && B >= 9 && B < 12) v = -a.c.dw[o][B - 9];
        else if (A == 12 && B == 12) v = -a.c.pp - a.pshift_area;
        M[sl[p]][sl[q]] += v;
      }
    (void)nu;
  }
  double mmax = 0.0;
  for (int r = 0; r < ps; ++r) {
    if (!act[r]) {
      for (int c = 0; c < ps; ++c) M[r][c] = M[c][r] = 0.0;
      M[r][r] = 1.0;
    }
  }
  for (int r = 0; r < ps; ++r)
    for (int c = 0; c < ps; ++c) mmax = fmax(mmax, fabs(M[r][c]));
  // Gauss-Jordan with partial pivoting on [M | I]
  double Inv[20][20];
  for (int r = 0; r < ps; ++r)
    for (int c = 0; c < ps; ++c) Inv[r][c] = (r == c) ? 1.0 : 0.0;
  bool ok = true;
  for (int k = 0; k < ps; ++k) {
    int piv = k;
    double best = fabs(M[k][k]);
    for (int r = k + 1; r < ps; ++r)
      if (fabs(M[r][k]) > best) { best = fabs(M[r][k]); piv = r; }
    if (!(best > 1e-15 * mmax)) { ok = false; break; }
    if (piv != k)
      for (int c = 0; c < ps; ++c) {
        double t = M[k][c]; M[k][c] = M[piv][c]; M[piv][c] = t;
        t = Inv[k][c]; Inv[k][c] = Inv[piv][c]; Inv[piv][c] = t;
      }
    const double d = 1.0 / M[k][k];
    for (int c = 0; c < ps; ++c) { M[k][c] *= d; Inv[k][c] *= d; }
    for (int r = 0; r < ps; ++r) {
      if (r == k) continue;
      const double f = M[r][k];
      if (f == 0.0) continue;
      for (int c = 0; c < ps; ++c) { M[r][c] -= f * M[k][c]; Inv[r][c] -= f * Inv[k][c]; }
    }
  }
  if (!ok) atomicOr(a.flag, 1);
  if (ps == 20) {
    // symmetric: the upper triangle of (Inv + Inv^T) / 2, row-major
    for (int r = 0; r < 20; ++r)
      for (int c = r; c < 20; ++c) {
        const double v = ok ? 0.5 * (Inv[r][c] + Inv[c][r]) : 0.0;
        const size_t e = (size_t)sym20(r, c);
        a.inv64[e * a.nrep + s] = v;
        a.inv32[e * a.nrep + s] = (float)v;
      }
  } else {
    for (int r = 0; r < ps; ++r)
      for (int c = 0; c < ps; ++c) {
        const double v = ok ? Inv[r][c] : 0.0;
        a.inv64[(size_t)(r * ps + c) * a.nrep + s] = v;
        a.inv32[(size_t)(r * ps + c) * a.nrep + s] = (float)v;
      }
  }
}

// The shared interior inverse (slot 0) in the symmetry-adapted basis: B = diag(1/d) U^T
// A^{-1} U diag(1/d), kept only if it is block diagonal and reproduces A^{-1} (relative
// 1e-9); otherwise the dense slot-0 path stays in use.
int vanka_klein_setup(Level &L, cudaStream_t st) {
  L.klein = false;
  if (!L.uniform || L.psize != 20 || L.n < 2 || L.nslots < 1) return BMG_OK;
  double packed[210];
  BMG_CUDA(cudaMemcpy2DAsync(packed, sizeof(double), L.pinv64, sizeof(double) * (size_t)L.nslots,
                             sizeof(double), 210, cudaMemcpyDeviceToHost, st));
  BMG_CUDA(cudaStreamSynchronize(st));
  double Ai[20][20], U[20][20];
  for (int r = 0; r < 20; ++r)
    for (int c = 0; c < 20; ++c) Ai[r][c] = packed[sym20(r, c)];
  for (int s = 0; s < 20; ++s) {          // row s of U = U^T e_s
    double e[20] = {}, q[20];
    e[s] = 1.0;
    klein_fwd(e, q);
    for (int k = 0; k < 20; ++k) U[s][k] = q[k];
  }
  double d[20], B[20][20], amax = 0.0;
  for (int k = 0; k < 20; ++k) {
    d[k] = 0.0;
    for (int s = 0; s < 20; ++s) d[k] += U[s][k] * U[s][k];
  }
  for (int r = 0; r < 20; ++r)
    for (int c = 0; c < 20; ++c) amax = std::fmax(amax, std::fabs(Ai[r][c]));
  double bmax = 0.0, off = 0.0;
  for (int k = 0; k < 20; ++k)
    for (int l = 0; l < 20; ++l) {
      double acc = 0.0;
      for (int s = 0; s < 20; ++s)
        for (int t = 0; t < 20; ++t) acc += U[s][k] * Ai[s][t] * U[t][l];
      B[k][l] = acc / (d[k] * d[l]);
      const bool in = klein_block_start(k) == klein_block_start(l);
      if (in) bmax = std::fmax(bmax, std::fabs(B[k][l]));
      else off = std::fmax(off, std::fabs(B[k][l]));
    }
  if (!(bmax > 0.0) || off > 1e-9 * bmax) return BMG_OK;
  double err = 0.0;                        // U B U^T against A^{-1}
  for (int r = 0; r < 20; ++r)
    for (int c = 0; c < 20; ++c) {
      double acc = 0.0;
      for (int k = 0; k < 20; ++k)
        for (int l = klein_block_start(k); l < klein_block_start(k) + klein_block_size(k); ++l)
          acc += U[r][k] * B[k][l] * U[c][l];
      err = std::fmax(err, std::fabs(acc - Ai[r][c]));
    }
  if (!(err <= 1e-9 * amax)) return BMG_OK;
  for (int k = 0; k < 20; ++k)
    for (int l = 0; l < 7; ++l) {
      const double v = l < klein_block_size(k) ? B[k][klein_block_start(k) + l] : 0.0;
      L.kb64[k][l] = v;
      L.kb32[k][l] = (float)v;
    }
  L.klein = true;
  return BMG_OK;
}

int launch_vanka_setup(const Level &L, const int *rep_i, const int *rep_j, int nrep,
                       double p_shift_area, int psize, int *d_flag, cudaStream_t st) {
  VankaSetupArgs a;
  a.g = L.g;
  a.kinv = L.kinv64;
  a.wm = L.wm64;
  a.wm_full = L.wm_full ? 1 : 0;
  a.c = L.c64;
  a.pshift_area = p_shift_area;
  a.rep_i = rep_i;
  a.rep_j = rep_j;
  a.nrep = nrep;
  a.psize = psize;
  a.inv64 = L.pinv64;
  a.inv32 = L.pinv32;
  a.flag = d_flag;
  vanka_setup_kernel<<<(nrep + 63) / 64, 64, 0, st>>>(a);
  BMG_CHECK_LAUNCH("vanka_setup_kernel");
  return BMG_OK;
}

// --------------------------------------------------------------------------------------
// A CTA of NT threads holds kPX x kPY patches and updates the (kPX - 1) x (kPY - 1) positions
// whose patches it holds.  Phase 1 gathers the patches' residuals into shared memory; phase
// 2 splits the 20 x 20 local solves into (patch, row) tasks, so on small grids each thread
// issues 20 * (rows per thread) FP64 FMAs instead of 400 (the FP64 pipe of a GB300 SM
// retires about two FMAs per clock, so the per-warp instruction count sets the time);
// phase 3 gathers the weighted corrections.  Deterministic, no atomics.
// T: vectors and weighted gather; S: the patch solves (the inverses and their products).
// S = double with T = float is the FP32 sweep with FP64 patch solves (BMG_PATCH_FP64).
template <typename T, typename S = T>
struct VankaSweepArgs {
  Grid g;
  const T *r;
  T *x;
  const int *slot;
  const S *inv;
  int nslots;
  T omega;
  int assign;   // 1: x <- omega M^{-1} r on the free DoFs (x was zero); 0: x += omega M^{-1} r
  const int *gate;
  int klein;    // slot 0 also given in the symmetry-adapted basis (kb)
  S kb[20][7];
};

// Dense patch solve x = A_slot^{-1} r by one thread from the packed symmetric inverse in
// global memory: every entry (row, c), c >= row, is loaded once and used for both x[row] and
// x[c] (210 loads, 400 FMAs, entry-major layout: consecutive patches' loads coalesce).
template <typename S>
__device__ __forceinline__ void patch_solve_packed(const S *__restrict__ inv, size_t ld, const S (&r)[20],
                                                   S (&x)[20]) {
#pragma unroll
  for (int c = 0; c < 20; ++c) x[c] = S(0);
  static_for<20>([&](auto row_) {
    constexpr int row = decltype(row_)::value;
    static_for<20 - row>([&](auto d_) {
      constexpr int c = row + decltype(d_)::value;
      constexpr int e = row * 20 - (row * (row - 1)) / 2 + (c - row);
      const S f = __ldg(inv + (size_t)e * ld);
      x[row] = fma(f, r[c], x[row]);
      if constexpr (c != row) x[c] = fma(f, r[row], x[c]);
    });
  });
}

// kKlein = false compiles the symmetry-adapted path out (slot-0 patches then use the dense
// inverse, which is always stored): fewer registers where that path is not used.
// kPatchThread: every patch is solved by the thread that gathered its residual, in registers
// (symmetry-adapted for slot 0 when available, else patch_solve_packed), so the (row, patch)
// tasks of phase 2 are skipped: the per-patch factors stream through once per patch.
template <typename T, int kPX, int kPY, int NT, bool kKlein = true, typename S = T, bool kPatchThread = false>
__device__ __forceinline__ void vanka_tile(const VankaSweepArgs<T, S> &a, int bx, int by) {
  constexpr int NP = kPX * kPY, LD = 21;          // LD: padded row of the shared arrays
  // dynamic shared memory (vanka_smem_bytes): residuals sr[NP][LD], corrections sx[NP][LD],
  // inverse slots ss[NP]
  extern __shared__ __align__(16) unsigned char vanka_smem[];
  T *sr = reinterpret_cast<T *>(vanka_smem);
  T *sx = sr + NP * LD;
  int *ss = reinterpret_cast<int *>(sx + NP * LD);
  __shared__ int s_mixed;                          // some patch of the tile has its own inverse
  if (threadIdx.x == 0) s_mixed = 0;
  __syncthreads();
  const int n = a.g.n, P = a.g.pitch;
  const size_t blk = a.g.blk;
  const int i0 = bx * (kPX - 1), j0 = by * (kPY - 1);
  const int tid = threadIdx.x;
  const bool kl = kKlein && a.klein != 0;
  // phase 1: residual gather, one patch per thread.  A slot-0 patch with the
  // symmetry-adapted inverse (uniform coefficients) is solved right here in registers:
  // q = U^T r, x' = B q (block entries as compile-time parameter operands), x = U x' into sx.
  // Other patches leave their residual in sr for the (row, patch) tasks below.
  for (int p = tid; p < NP; p += NT) {
    const int pi = i0 + p % kPX, pj = j0 + p / kPX;
    T r[20];
    int sl = 0;
    if (pi <= n && pj <= n) {
      const T *rv = a.r;
      const size_t o = (size_t)pj * P + pi;
      const bool li = pi >= 1, lj = pj >= 1;
      r[0] = rv[UX * blk + o];
      r[1] = rv[UY * blk + o];
      r[2] = rv[BH * blk + o];                          // E0 = h(pi,pj)
      r[8] = rv[WH * blk + o];
      r[3] = rv[BV * blk + o];                          // E1 = v(pi,pj)
      r[9] = rv[WV * blk + o];
      r[4] = li ? rv[BH * blk + o - 1] : T(0);          // E2 = h(pi-1,pj)
      r[10] = li ? rv[WH * blk + o - 1] : T(0);
      r[5] = lj ? rv[BV * blk + o - P] : T(0);          // E3 = v(pi,pj-1)
      r[11] = lj ? rv[WV * blk + o - P] : T(0);
      r[6] = li ? rv[BD * blk + o - 1] : T(0);          // E4 = d(pi-1,pj)
      r[12] = li ? rv[WD * blk + o - 1] : T(0);
      r[7] = lj ? rv[BD * blk + o - P] : T(0);          // E5 = d(pi,pj-1)
      r[13] = lj ? rv[WD * blk + o - P] : T(0);
      r[14] = rv[PL * blk + o];                         // L(pi,pj)
      r[15] = li ? rv[PL * blk + o - 1] : T(0);         // L(pi-1,pj)
      r[16] = lj ? rv[PL * blk + o - P] : T(0);         // L(pi,pj-1)
      r[17] = li ? rv[PU * blk + o - 1] : T(0);         // U(pi-1,pj)
      r[18] = (li && lj) ? rv[PU * blk + o - P - 1] : T(0);   // U(pi-1,pj-1)
      r[19] = lj ? rv[PU * blk + o - P] : T(0);         // U(pi,pj-1)
      sl = a.slot[(size_t)pj * (n + 1) + pi];
    } else {
#pragma unroll
      for (int c = 0; c < 20; ++c) r[c] = T(0);
    }
    ss[p] = sl;
    if constexpr (kPatchThread) {
      S rs[20], x[20];
#pragma unroll
      for (int c = 0; c < 20; ++c) rs[c] = (S)r[c];
      if (pi > n || pj > n) {
#pragma unroll
        for (int c = 0; c < 20; ++c) x[c] = S(0);
      } else if (kKlein && kl && sl == 0) {
        S q[20], xq[20];
        klein_fwd(rs, q);
        static_for<20>([&](auto k_) {
          constexpr int k = decltype(k_)::value, b0 = klein_block_start(k);
          S acc = 0;
          static_for<klein_block_size(k)>([&](auto l_) {
            constexpr int l = decltype(l_)::value;
            acc = fma(a.kb[k][l], q[b0 + l], acc);
          });
          xq[k] = acc;
        });
        klein_inv(xq, x);
      } else {
        patch_solve_packed<S>(a.inv + sl, (size_t)a.nslots, rs, x);
      }
#pragma unroll
      for (int c = 0; c < 20; ++c) sx[p * LD + c] = (T)x[c];
    } else if constexpr (!kKlein) {
#pragma unroll
      for (int c = 0; c < 20; ++c) sr[p * LD + c] = r[c];
      if (sl != 0) s_mixed = 1;
    } else if (kl && sl == 0) {
      S rs[20], q[20], xq[20], x[20];
#pragma unroll
      for (int c = 0; c < 20; ++c) rs[c] = (S)r[c];
      klein_fwd(rs, q);
      static_for<20>([&](auto k_) {
        constexpr int k = decltype(k_)::value, b0 = klein_block_start(k);
        S acc = 0;
        static_for<klein_block_size(k)>([&](auto l_) {
          constexpr int l = decltype(l_)::value;
          acc = fma(a.kb[k][l], q[b0 + l], acc);
        });
        xq[k] = acc;
      });
      klein_inv(xq, x);
#pragma unroll
      for (int c = 0; c < 20; ++c) sx[p * LD + c] = (T)x[c];
    } else {
#pragma unroll
      for (int c = 0; c < 20; ++c) sr[p * LD + c] = r[c];
      if (sl != 0) s_mixed = 1;
    }
  }
  __syncthreads();
  const size_t ld = (size_t)a.nslots;
  if constexpr (kPatchThread) {
    // every patch was solved in phase 1
  } else if (kl) {
    // the tile's other patches (boundary patches with their own inverses)
    if (s_mixed) {
#pragma unroll 2
      for (int t = tid; t < NP * 20; t += NT) {
        const int row = t / NP, p = t % NP;
        if (ss[p] == 0) continue;
        const S *inv = a.inv + ss[p];
        const int rb = sym20_row_base(row);
        const T *rl = sr + p * LD;
        S acc = 0;
#pragma unroll
        for (int c = 0; c < 20; ++c) {
          const int e = c < row ? c * 19 - (c * (c - 1)) / 2 + row : rb + c;
          acc = fma(inv[(size_t)e * ld], (S)rl[c], acc);
        }
        sx[p * LD + row] = (T)acc;
      }
    }
  } else if (!s_mixed) {
    // every patch of the tile uses the shared interior inverse (slot 0): thread
    // (row = tid % 20, group = tid / 20) keeps its inverse row in registers and sweeps the
    // group's patches, so the solve issues a few shared loads per patch instead of 400
    // global loads.
    constexpr int NG = NT / 20;
    if (tid < NG * 20) {
      const int row = tid % 20, grp = tid / 20;
      S irow[20];
      const int rb = sym20_row_base(row);
#pragma unroll
      for (int c = 0; c < 20; ++c) {
        const int e = c < row ? c * 19 - (c * (c - 1)) / 2 + row : rb + c;
        irow[c] = a.inv[(size_t)e * ld];
      }
      for (int p = grp; p < NP; p += NG) {
        const T *rl = sr + p * LD;
        S acc = 0;
#pragma unroll
        for (int c = 0; c < 20; ++c) acc = fma(irow[c], (S)rl[c], acc);
        sx[p * LD + row] = (T)acc;
      }
    }
  } else {
    // phase 2 (general): xhat[p][row] = sum_c inv_slot[row][c] r_p[c]; consecutive threads
    // take consecutive patches of one row, so their inverse loads coalesce (or broadcast);
    // in FP32 four tasks per step keep 80 independent factor loads in flight per thread (the
    // FP64 sweep is bound by the FP64 pipe instead and keeps its registers)
    constexpr int kUnroll = sizeof(S) == 4 ? 4 : 1;
#pragma unroll kUnroll
    for (int t = tid; t < NP * 20; t += NT) {
      const int row = t / NP, p = t % NP;
      const S *inv = a.inv + ss[p];
      const int rb = sym20_row_base(row);
      const T *rl = sr + p * LD;
      S acc = 0;
#pragma unroll
      for (int c = 0; c < 20; ++c) {
        const int e = c < row ? c * 19 - (c * (c - 1)) / 2 + row : rb + c;
        acc = fma(inv[(size_t)e * ld], (S)rl[c], acc);
      }
      sx[p * LD + row] = (T)acc;
    }
  }
  __syncthreads();
  // phase 3: weighted gather of the corrections, one position per thread
  for (int q = tid; q < (kPX - 1) * (kPY - 1); q += NT) {
    const int i = i0 + q % (kPX - 1), j = j0 + q / (kPX - 1);
    if (j > n) continue;
    if (i > n) {                  // padding columns: written only when assigning
      if (a.assign && i < P) {
#pragma unroll
        for (int k = 0; k < NBLK; ++k) a.x[k * blk + (size_t)j * P + i] = T(0);
      }
      continue;
    }
    auto X = [&](int pi, int pj, int k) -> T { return sx[((pj - j0) * kPX + (pi - i0)) * LD + k]; };
    bool m[NBLK];
    dof_masks(i, j, n, m);
    T *x = a.x;
    const size_t o = (size_t)j * P + i;
    const T w = a.omega, half = T(0.5) * a.omega, third = a.omega / T(3);
    T v[NBLK];
    v[UX] = w * X(i, j, 0);
    v[UY] = w * X(i, j, 1);
    v[BH] = half * (X(i, j, 2) + X(i + 1, j, 4));
    v[BV] = half * (X(i, j, 3) + X(i, j + 1, 5));
    v[BD] = half * (X(i, j + 1, 7) + X(i + 1, j, 6));
    v[WH] = half * (X(i, j, 8) + X(i + 1, j, 10));
    v[WV] = half * (X(i, j, 9) + X(i, j + 1, 11));
    v[WD] = half * (X(i, j + 1, 13) + X(i + 1, j, 12));
    v[PL] = third * (X(i, j, 14) + X(i + 1, j, 15) + X(i, j + 1, 16));
    v[PU] = third * (X(i + 1, j + 1, 18) + X(i, j + 1, 19) + X(i + 1, j, 17));
    if (a.assign) {
#pragma unroll
      for (int k = 0; k < NBLK; ++k) x[k * blk + o] = m[k] ? v[k] : T(0);
    } else {
#pragma unroll
      for (int k = 0; k < NBLK; ++k)
        if (m[k]) x[k * blk + o] += v[k];
    }
  }
}

template <typename T, int kPX, int kPY, int NT, typename S, bool kPatchThread = false>
__global__ void __launch_bounds__(NT) vanka_sweep_kernel(const __grid_constant__ VankaSweepArgs<T, S> a) {
  pdl_enter();
  BMG_GATE(a.gate);
  vanka_tile<T, kPX, kPY, NT, true, S, kPatchThread>(a, blockIdx.x, blockIdx.y);
}

// Batched form: blockIdx.z selects one of several instances of one grid size; their
// arguments (vectors, inverse tables, damping, gate) are read from a device array.
template <int kPX, int kPY, int NT, bool kPatchThread = false>
__global__ void __launch_bounds__(NT) vanka_batch_kernel(const VankaSweepArgs<double> *__restrict__ args) {
  const VankaSweepArgs<double> &a = args[blockIdx.z];
  BMG_GATE(a.gate);
  vanka_tile<double, kPX, kPY, NT, false, double, kPatchThread>(a, blockIdx.x, blockIdx.y);
}

template <typename T, int PX, int PY>
constexpr size_t vanka_smem_bytes() {
  return 2 * (size_t)PX * PY * 21 * sizeof(T) + (size_t)PX * PY * sizeof(int);
}

template <typename T, int PX, int PY, int NT, typename S, bool PT = false>
static void launch_vanka_tile(const VankaSweepArgs<T, S> &a, const Level &L, cudaStream_t st) {
  constexpr size_t smem = vanka_smem_bytes<T, PX, PY>();
  static_assert(smem <= 200 * 1024, "shared memory of a Vanka tile");
  if constexpr (smem > 48 * 1024) {
    static const bool opted_in = [] {          // once per instantiation, thread-safe
      return cudaFuncSetAttribute(vanka_sweep_kernel<T, PX, PY, NT, S, PT>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess;
    }();
    (void)opted_in;
  }
  dim3 grid((L.g.pitch + PX - 2) / (PX - 1), (L.n + 1 + PY - 2) / (PY - 1));
  (void)launch_pdl(vanka_sweep_kernel<T, PX, PY, NT, S, PT>, dim3(grid), dim3(NT), smem, st, a);
}

static long long vanka_ctas(const Level &L, int px, int py) {
  return (long long)((L.g.pitch + px - 2) / (px - 1)) * ((L.n + 1 + py - 2) / (py - 1));
}

template <typename T, typename S>
static void launch_vanka_sweep_s(const Level &L, const T *r, T *x, T omega, cudaStream_t st, bool assign) {
  VankaSweepArgs<T, S> a;
  a.g = L.g;
  a.r = r;
  a.x = x;
  a.slot = L.slot;
  a.inv = (const S *)(sizeof(S) == 8 ? (const void *)L.pinv64 : (const void *)L.pinv32);
  a.nslots = L.nslots;
  a.omega = omega;
  a.assign = assign ? 1 : 0;
  a.gate = L.gate;
  a.klein = L.klein ? 1 : 0;
  for (int k = 0; k < 20; ++k)
    for (int l = 0; l < 7; ++l) a.kb[k][l] = sizeof(S) == 8 ? (S)L.kb64[k][l] : (S)L.kb32[k][l];
  // the largest patch tile that still gives every SM about two CTAs; smaller tiles also
  // spread each patch's rows over more threads
  // (two 21-wide shared arrays per patch: 32 x 8 patches take 43 KB in FP32, 87 KB in FP64)
  const long long want = 2 * 152;
  bool done = true;
  // tuned at setup: 0 = 32 x 8, 1 = 16 x 8, 2 = 8 x 8, 3 = 8 x 4, 4 = 4 x 4 patches with
  // (row, patch) solve tasks; 5 = 32 x 8, 6 = 16 x 8, 7 = 8 x 8 patches with one thread per
  // patch solve
  switch (L.tile_vanka) {
    case 0: launch_vanka_tile<T, 32, 8, 256>(a, L, st); break;
    case 1: launch_vanka_tile<T, 16, 8, 256>(a, L, st); break;
    case 2: launch_vanka_tile<T, 8, 8, 256>(a, L, st); break;
    case 3: launch_vanka_tile<T, 8, 4, 160>(a, L, st); break;
    case 4: launch_vanka_tile<T, 4, 4, 160>(a, L, st); break;
    case 5: launch_vanka_tile<T, 32, 8, 256, S, true>(a, L, st); break;
    case 6: launch_vanka_tile<T, 16, 8, 128, S, true>(a, L, st); break;
    case 7: launch_vanka_tile<T, 8, 8, 64, S, true>(a, L, st); break;
    default: done = false;
  }
  if constexpr (sizeof(T) == 4) {
    if (!done && vanka_ctas(L, 32, 8) >= want) { launch_vanka_tile<T, 32, 8, 256>(a, L, st); done = true; }
  }
  if (done) {
  } else if (vanka_ctas(L, 16, 8) >= want) launch_vanka_tile<T, 16, 8, 256>(a, L, st);
  else if (vanka_ctas(L, 8, 8) >= want) launch_vanka_tile<T, 8, 8, 256>(a, L, st);
  else if (vanka_ctas(L, 8, 4) >= want) launch_vanka_tile<T, 8, 4, 160>(a, L, st);
  else launch_vanka_tile<T, 4, 4, 160>(a, L, st);
}

template <typename T>
int launch_vanka_sweep(const Level &L, const T *r, T *x, T omega, cudaStream_t st, bool assign) {
  BMG_PROF_BEGIN(BMG_PROF_VANKA, L.n, st);
  // FP32 sweep with FP64 patch solves (FP64 inverses, FP64 products) when the level asks
  if constexpr (sizeof(T) == 4) {
    if (L.solve64) launch_vanka_sweep_s<T, double>(L, r, x, omega, st, assign);
    else launch_vanka_sweep_s<T, T>(L, r, x, omega, st, assign);
  } else {
    launch_vanka_sweep_s<T, T>(L, r, x, omega, st, assign);
  }
  BMG_PROF_END(st, (double)L.n * L.n);
  BMG_CHECK_LAUNCH("vanka_sweep_kernel");
  return BMG_OK;
}

template int launch_vanka_sweep<double>(const Level &, const double *, double *, double, cudaStream_t, bool);
template int launch_vanka_sweep<float>(const Level &, const float *, float *, float, cudaStream_t, bool);

// ---- batched sweep ---------------------------------------------------------------------
size_t vanka_args_bytes() { return sizeof(VankaSweepArgs<double>); }

void make_vanka_args(const Level &L, const double *r, double *x, double omega, bool assign,
                     const int *gate, void *dst) {
  VankaSweepArgs<double> a;
  a.g = L.g;
  a.r = r;
  a.x = x;
  a.slot = L.slot;
  a.inv = L.pinv64;
  a.nslots = L.nslots;
  a.omega = omega;
  a.assign = assign ? 1 : 0;
  a.gate = gate;
  a.klein = L.klein ? 1 : 0;
  std::memcpy(a.kb, L.kb64, sizeof(a.kb));
  std::memcpy(dst, &a, sizeof(a));
}

template <int PX, int PY, int NT, bool PT = false>
static int launch_vanka_batch_tile(const void *d_args, int count, int n, cudaStream_t st) {
  constexpr size_t smem = vanka_smem_bytes<double, PX, PY>();
  static_assert(smem <= 48 * 1024, "batched tiles stay within the default shared memory");
  const Grid g = grid_of(n);
  dim3 grid((g.pitch + PX - 2) / (PX - 1), (n + 1 + PY - 2) / (PY - 1), count);
  vanka_batch_kernel<PX, PY, NT, PT><<<grid, NT, smem, st>>>((const VankaSweepArgs<double> *)d_args);
  BMG_CHECK_LAUNCH("vanka_batch_kernel");
  return BMG_OK;
}

// tile t: 0 = 16 x 8, 1 = 8 x 8, 2 = 8 x 4, 3 = 4 x 4 patches with (row, patch) solve tasks;
// 4 = 16 x 8, 5 = 8 x 8 patches with one thread per patch solve (autotuning candidates)
int launch_vanka_batch(const void *d_args, int count, int n, int tile, cudaStream_t st) {
  if (count <= 0) return BMG_OK;
  switch (tile) {
    case 0: return launch_vanka_batch_tile<16, 8, 256>(d_args, count, n, st);
    case 1: return launch_vanka_batch_tile<8, 8, 256>(d_args, count, n, st);
    case 2: return launch_vanka_batch_tile<8, 4, 160>(d_args, count, n, st);
    case 4: return launch_vanka_batch_tile<16, 8, 128, true>(d_args, count, n, st);
    case 5: return launch_vanka_batch_tile<8, 8, 64, true>(d_args, count, n, st);
    default: return launch_vanka_batch_tile<4, 4, 160>(d_args, count, n, st);
  }
}

int default_vanka_tile(int n, int count) {
  constexpr int kRule = 4;                 // the rule picks among the (row, patch) task tiles
  static const int px[kRule] = {16, 8, 8, 4}, py[kRule] = {8, 8, 4, 4};
  const Grid g = grid_of(n);
  for (int t = 0; t + 1 < kRule; ++t) {
    const long long c = (long long)((g.pitch + px[t] - 2) / (px[t] - 1)) * ((n + 1 + py[t] - 2) / (py[t] - 1)) * count;
    if (c >= 2 * 152) return t;
  }
  return kRule - 1;
}

}  // namespace bmg
