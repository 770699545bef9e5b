// Host-side geometry of the structured triangulation: element integrals of the two
// triangle shapes and the stencil tables of the block interpolation.
//
// Bases (Sec. 2.1 and the conventions under which App. A's stencils hold): P1 hats per
// displacement component; face bubble 4 l_a l_b n_e with global normals n_h = (0,1),
// n_v = (1,0), n_d = (1,1)/sqrt2; RT0 psi_e with psi_e . n_e = 1 on e; P0 indicators.
// Every integrand is a polynomial of degree <= 2, integrated exactly by the three-point
// edge-midpoint rule.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "bmg_internal.h"

namespace bmg {
namespace {

const double kSqrt2 = 1.41421356237309504880;

enum Fam { FH = 0, FV = 1, FD = 2 };

void fam_normal(int f, double n[2]) {
  if (f == FH) { n[0] = 0.0; n[1] = 1.0; }
  else if (f == FV) { n[0] = 1.0; n[1] = 0.0; }
  else { n[0] = 1.0 / kSqrt2; n[1] = 1.0 / kSqrt2; }
}

// Structured edge through two adjacent vertices (grid units): family and index.
void edge_of(int i0, int j0, int i1, int j1, int *fam, int *ei, int *ej) {
  if (j0 == j1) { *fam = FH; *ei = i0 < i1 ? i0 : i1; *ej = j0; return; }
  if (i0 == i1) { *fam = FV; *ei = i0; *ej = j0 < j1 ? j0 : j1; return; }
  *fam = FD; *ei = i0 < i1 ? i0 : i1; *ej = j0 < j1 ? j0 : j1;
}

// Triangle (o, i, j) of the structured mesh: vertices with local vertex k opposite local
// edge k.
void tri_vertices(int o, int i, int j, int v[3][2]) {
  if (o == 0) { v[0][0] = i; v[0][1] = j; v[1][0] = i + 1; v[1][1] = j; v[2][0] = i; v[2][1] = j + 1; }
  else { v[0][0] = i + 1; v[0][1] = j + 1; v[1][0] = i; v[1][1] = j + 1; v[2][0] = i + 1; v[2][1] = j; }
}

struct Tri {
  double X[3][2];
  double grad[3][2];   // grad lambda_k
  double area;
  double cen[2];
  int fam[3];
  double nrm[3][2], nout[3][2], sgn[3], len[3], mid[3][2];

  // vertices in physical coordinates (grid units * scale), families of local edges
  void init(const int v[3][2], double scale) {
    for (int k = 0; k < 3; ++k) { X[k][0] = v[k][0] * scale; X[k][1] = v[k][1] * scale; }
    double sa = 0.5 * ((X[1][0] - X[0][0]) * (X[2][1] - X[0][1]) -
                       (X[2][0] - X[0][0]) * (X[1][1] - X[0][1]));
    area = std::fabs(sa);
    cen[0] = (X[0][0] + X[1][0] + X[2][0]) / 3.0;
    cen[1] = (X[0][1] + X[1][1] + X[2][1]) / 3.0;
    for (int k = 0; k < 3; ++k) {
      int a = (k + 1) % 3, b = (k + 2) % 3;
      grad[k][0] = (X[a][1] - X[b][1]) / (2.0 * sa);
      grad[k][1] = (X[b][0] - X[a][0]) / (2.0 * sa);
      int f, ei, ej;
      edge_of(v[a][0], v[a][1], v[b][0], v[b][1], &f, &ei, &ej);
      fam[k] = f;
      fam_normal(f, nrm[k]);
      double tx = X[b][0] - X[a][0], ty = X[b][1] - X[a][1];
      len[k] = std::sqrt(tx * tx + ty * ty);
      double nx = ty / len[k], ny = -tx / len[k];
      if (nx * (X[a][0] - X[k][0]) + ny * (X[a][1] - X[k][1]) < 0) { nx = -nx; ny = -ny; }
      nout[k][0] = nx; nout[k][1] = ny;
      sgn[k] = (nrm[k][0] * nx + nrm[k][1] * ny) > 0 ? 1.0 : -1.0;
      mid[k][0] = 0.5 * (X[a][0] + X[b][0]);
      mid[k][1] = 0.5 * (X[a][1] + X[b][1]);
    }
  }
  void bary(const double x[2], double l[3]) const {
    for (int k = 0; k < 3; ++k)
      l[k] = 1.0 / 3.0 + grad[k][0] * (x[0] - cen[0]) + grad[k][1] * (x[1] - cen[1]);
  }
  // displacement basis a (0..8): value val[2], gradient G[c][s] = d val_c / d x_s
  void u_basis(int a, const double x[2], double val[2], double G[2][2]) const {
    double l[3];
    bary(x, l);
    val[0] = val[1] = 0.0;
    G[0][0] = G[0][1] = G[1][0] = G[1][1] = 0.0;
    if (a < 6) {
      int k = a % 3, c = a / 3;
      val[c] = l[k];
      G[c][0] = grad[k][0];
      G[c][1] = grad[k][1];
      return;
    }
    int k = a - 6, p = (k + 1) % 3, q = (k + 2) % 3;
    double s = 4.0 * l[p] * l[q];
    double gs[2] = {4.0 * (l[p] * grad[q][0] + l[q] * grad[p][0]),
                    4.0 * (l[p] * grad[q][1] + l[q] * grad[p][1])};
    for (int c = 0; c < 2; ++c) {
      val[c] = s * nrm[k][c];
      G[c][0] = nrm[k][c] * gs[0];
      G[c][1] = nrm[k][c] * gs[1];
    }
  }
  // RT0 basis k: value and divergence
  void w_basis(int k, const double x[2], double val[2], double *div) const {
    double c = sgn[k] * len[k] / (2.0 * area);
    val[0] = c * (x[0] - X[k][0]);
    val[1] = c * (x[1] - X[k][1]);
    *div = 2.0 * c;
  }
};

}  // namespace

void element_integrals(double h, ElemIntegrals *out) {
  std::memset(out, 0, sizeof(*out));
  for (int o = 0; o < 2; ++o) {
    int v[3][2];
    tri_vertices(o, 0, 0, v);
    Tri t;
    t.init(v, h);
    out->area = t.area;
    for (int q = 0; q < 3; ++q) {
      const double *x = t.mid[q];
      double wq = t.area / 3.0;
      double eps[9][2][2], div[9];
      for (int a = 0; a < 9; ++a) {
        double val[2], G[2][2];
        t.u_basis(a, x, val, G);
        for (int r = 0; r < 2; ++r)
          for (int s = 0; s < 2; ++s) eps[a][r][s] = 0.5 * (G[r][s] + G[s][r]);
        div[a] = G[0][0] + G[1][1];
      }
      for (int a = 0; a < 9; ++a) {
        out->g[o][a] += wq * div[a];
        for (int b = 0; b < 9; ++b) {
          double s = 0.0;
          for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) s += eps[a][r][c] * eps[b][r][c];
          out->Aeps[o][a][b] += wq * s;
          out->Ddiv[o][a][b] += wq * div[a] * div[b];
        }
      }
      double psi[3][2], dv[3];
      for (int k = 0; k < 3; ++k) t.w_basis(k, x, psi[k], &dv[k]);
      for (int a = 0; a < 3; ++a) {
        out->dw[o][a] += wq * dv[a];
        for (int b = 0; b < 3; ++b)
          out->Mw[o][a][b] += wq * (psi[a][0] * psi[b][0] + psi[a][1] * psi[b][1]);
      }
    }
  }
}

bool verify_elem_nonzeros(std::string *why) {
  ElemIntegrals e;
  element_integrals(1.0, &e);
  for (int o = 0; o < 2; ++o) {
    double amax = 0.0, gmax = 0.0, mmax = 0.0;
    for (int a = 0; a < 9; ++a) {
      gmax = std::max(gmax, std::fabs(e.g[o][a]));
      for (int b = 0; b < 9; ++b) amax = std::max(amax, std::fabs(e.Aeps[o][a][b]));
    }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) mmax = std::max(mmax, std::fabs(e.Mw[o][a][b]));
    for (int a = 0; a < 9; ++a) {
      if (!g_nonzero(a) && std::fabs(e.g[o][a]) > 1e-13 * gmax) {
        *why = "div-integral pattern";
        return false;
      }
      for (int b = 0; b < 9; ++b)
        if (!aeps_nonzero(a, b) && std::fabs(e.Aeps[o][a][b]) > 1e-13 * amax) {
          *why = "strain-matrix pattern";
          return false;
        }
    }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        if (!mw_nonzero(a, b) && std::fabs(e.Mw[o][a][b]) > 1e-13 * mmax) {
          *why = "RT0 mass pattern";
          return false;
        }
  }
  return true;
}

void make_coefs(const PhysParams &p, int n, OpCoefs<double> *c64, OpCoefs<float> *c32) {
  ElemIntegrals e;
  element_integrals(1.0 / n, &e);
  OpCoefs<double> &c = *c64;
  for (int o = 0; o < 2; ++o) {
    for (int a = 0; a < 9; ++a) {
      c.g[o][a] = e.g[o][a];
      for (int b = 0; b < 9; ++b)
        c.A[o][a * 9 + b] = 2.0 * p.mu * e.Aeps[o][a][b] + (p.exact_divdiv ? p.lambda * e.Ddiv[o][a][b] : 0.0);
    }
    for (int a = 0; a < 3; ++a) {
      c.dw[o][a] = p.tau * e.dw[o][a];
      for (int b = 0; b < 3; ++b) c.M1[o][a * 3 + b] = p.tau * e.Mw[o][a][b];
    }
  }
  c.lam_area = p.exact_divdiv ? 0.0 : p.lambda / e.area;
  c.alpha = p.alpha;
  c.pp = p.inv_M * e.area;
  if (c32) {
    OpCoefs<float> &f = *c32;
    for (int o = 0; o < 2; ++o) {
      for (int k = 0; k < 81; ++k) f.A[o][k] = (float)c.A[o][k];
      for (int k = 0; k < 9; ++k) { f.g[o][k] = (float)c.g[o][k]; f.M1[o][k] = (float)c.M1[o][k]; }
      for (int k = 0; k < 3; ++k) f.dw[o][k] = (float)c.dw[o][k];
    }
    f.lam_area = (float)c.lam_area;
    f.alpha = (float)c.alpha;
    f.pp = (float)c.pp;
  }
}

// --------------------------------------------------------------------------------------
// Block interpolation stencils (Sec. 3, Eq. block_interp; Sec. 3.1).  Built by applying
// the definitions on a small coarse grid with no constrained DoFs and reading the
// couplings off an interior position; the coefficients do not depend on h.
namespace {

struct DofKey {
  int type, i, j;
  bool operator<(const DofKey &o) const {
    return std::tie(type, i, j) < std::tie(o.type, o.i, o.j);
  }
};

// local DoF a (0..12) of structured triangle (o, i, j) -> (block type, i, j)
DofKey tri_dof(int o, int i, int j, int a) {
  int v[3][2];
  tri_vertices(o, i, j, v);
  if (a < 6) return DofKey{a < 3 ? UX : UY, v[a % 3][0], v[a % 3][1]};
  if (a < 12) {
    int k = (a - 6) % 3;
    int p = (k + 1) % 3, q = (k + 2) % 3;
    int f, ei, ej;
    edge_of(v[p][0], v[p][1], v[q][0], v[q][1], &f, &ei, &ej);
    int base = a < 9 ? BH : WH;
    return DofKey{base + f, ei, ej};
  }
  return DofKey{o == 0 ? PL : PU, i, j};
}

// identify a structured triangle from its vertex set
void tri_of(const int v[3][2], int *o, int *i, int *j) {
  int imin = v[0][0], jmin = v[0][1];
  for (int k = 1; k < 3; ++k) { if (v[k][0] < imin) imin = v[k][0]; if (v[k][1] < jmin) jmin = v[k][1]; }
  bool has = false;
  for (int k = 0; k < 3; ++k) if (v[k][0] == imin && v[k][1] == jmin) has = true;
  *o = has ? 0 : 1; *i = imin; *j = jmin;
}

typedef std::map<DofKey, std::map<DofKey, double>> SparseP;

void local_prolongation(int o, int I, int J, SparseP &P) {
  int cv[3][2];
  tri_vertices(o, I, J, cv);
  Tri tc;
  tc.init(cv, 2.0);                       // coarse triangle in fine units (h = 1)
  int A[3][2], M[3][2];
  for (int k = 0; k < 3; ++k) { A[k][0] = 2 * cv[k][0]; A[k][1] = 2 * cv[k][1]; }
  for (int k = 0; k < 3; ++k) {
    int a = (k + 1) % 3, b = (k + 2) % 3;
    M[k][0] = (A[a][0] + A[b][0]) / 2;
    M[k][1] = (A[a][1] + A[b][1]) / 2;
  }
  // fine vertices, half edges, interior edges, children (corner at A_k first)
  int fv[6][2] = {{A[0][0], A[0][1]}, {A[1][0], A[1][1]}, {A[2][0], A[2][1]},
                  {M[0][0], M[0][1]}, {M[1][0], M[1][1]}, {M[2][0], M[2][1]}};
  int half[6][2][2];
  for (int k = 0; k < 3; ++k) {
    int a = (k + 1) % 3, b = (k + 2) % 3;
    half[2 * k][0][0] = A[a][0]; half[2 * k][0][1] = A[a][1];
    half[2 * k][1][0] = M[k][0]; half[2 * k][1][1] = M[k][1];
    half[2 * k + 1][0][0] = M[k][0]; half[2 * k + 1][0][1] = M[k][1];
    half[2 * k + 1][1][0] = A[b][0]; half[2 * k + 1][1][1] = A[b][1];
  }
  int inner[3][2][2] = {{{M[1][0], M[1][1]}, {M[2][0], M[2][1]}},
                        {{M[2][0], M[2][1]}, {M[0][0], M[0][1]}},
                        {{M[0][0], M[0][1]}, {M[1][0], M[1][1]}}};
  int child[4][3][2] = {{{A[0][0], A[0][1]}, {M[2][0], M[2][1]}, {M[1][0], M[1][1]}},
                        {{A[1][0], A[1][1]}, {M[0][0], M[0][1]}, {M[2][0], M[2][1]}},
                        {{A[2][0], A[2][1]}, {M[1][0], M[1][1]}, {M[0][0], M[0][1]}},
                        {{M[0][0], M[0][1]}, {M[1][0], M[1][1]}, {M[2][0], M[2][1]}}};

  auto put = [&](DofKey f, DofKey c, double v) {
    if (v != 0.0) P[f][c] = v;             // values are set, not summed
  };
  // displacement
  for (int a = 0; a < 9; ++a) {
    DofKey col = tri_dof(o, I, J, a);
    double val[6][2];
    for (int p = 0; p < 6; ++p) {
      double x[2] = {(double)fv[p][0], (double)fv[p][1]}, G[2][2];
      tc.u_basis(a, x, val[p], G);
      put(DofKey{UX, fv[p][0], fv[p][1]}, col, val[p][0]);
      put(DofKey{UY, fv[p][0], fv[p][1]}, col, val[p][1]);
    }
    auto vidx = [&](int vi, int vj) {
      for (int p = 0; p < 6; ++p) if (fv[p][0] == vi && fv[p][1] == vj) return p;
      return -1;
    };
    std::map<std::pair<int, int>, double> bub;   // keyed by the two vertex indices
    for (int e = 0; e < 6; ++e) {
      int p = vidx(half[e][0][0], half[e][0][1]), q = vidx(half[e][1][0], half[e][1][1]);
      int f, ei, ej;
      edge_of(half[e][0][0], half[e][0][1], half[e][1][0], half[e][1][1], &f, &ei, &ej);
      double nrm[2];
      fam_normal(f, nrm);
      double x[2] = {0.5 * (half[e][0][0] + half[e][1][0]), 0.5 * (half[e][0][1] + half[e][1][1])};
      double vm[2], G[2][2];
      tc.u_basis(a, x, vm, G);
      double c = nrm[0] * (vm[0] - 0.5 * (val[p][0] + val[q][0])) +
                 nrm[1] * (vm[1] - 0.5 * (val[p][1] + val[q][1]));
      bub[{p < q ? p : q, p < q ? q : p}] = c;
      put(DofKey{BH + f, ei, ej}, col, c);
    }
    // zero net flux through each corner child (Eq. divfreefine)
    for (int c = 0; c < 3; ++c) {
      Tri t;
      t.init(child[c], 1.0);
      double flux = 0.0;
      int kint = -1;
      for (int k = 0; k < 3; ++k) {
        int pa = vidx(child[c][(k + 1) % 3][0], child[c][(k + 1) % 3][1]);
        int pb = vidx(child[c][(k + 2) % 3][0], child[c][(k + 2) % 3][1]);
        flux += t.len[k] * 0.5 * ((val[pa][0] + val[pb][0]) * t.nout[k][0] +
                                  (val[pa][1] + val[pb][1]) * t.nout[k][1]);
        auto it = bub.find({pa < pb ? pa : pb, pa < pb ? pb : pa});
        if (it != bub.end()) flux += (2.0 / 3.0) * t.len[k] * it->second * t.sgn[k];
        else kint = k;
      }
      const int *pa = child[c][(kint + 1) % 3], *pb = child[c][(kint + 2) % 3];
      int f, ei, ej;
      edge_of(pa[0], pa[1], pb[0], pb[1], &f, &ei, &ej);
      double cint = -flux / ((2.0 / 3.0) * t.len[kint] * t.sgn[kint]);
      put(DofKey{BH + f, ei, ej}, col, cint);
    }
  }
  // RT0
  for (int a = 0; a < 3; ++a) {
    DofKey col = tri_dof(o, I, J, 9 + a);
    for (int e = 0; e < 9; ++e) {
      const int(*ed)[2] = e < 6 ? half[e] : inner[e - 6];
      int f, ei, ej;
      edge_of(ed[0][0], ed[0][1], ed[1][0], ed[1][1], &f, &ei, &ej);
      double nrm[2];
      fam_normal(f, nrm);
      double x[2] = {0.5 * (ed[0][0] + ed[1][0]), 0.5 * (ed[0][1] + ed[1][1])};
      double psi[2], dv;
      tc.w_basis(a, x, psi, &dv);
      put(DofKey{WH + f, ei, ej}, col, psi[0] * nrm[0] + psi[1] * nrm[1]);
    }
  }
  // P0 injection
  DofKey col = tri_dof(o, I, J, 12);
  for (int c = 0; c < 4; ++c) {
    int co, ci, cj;
    tri_of(child[c], &co, &ci, &cj);
    put(DofKey{co == 0 ? PL : PU, ci, cj}, col, 1.0);
  }
}

// The four children of coarse triangle (o, I, J) in fine grid units, corner at A_k first,
// the interior child last (the order of local_prolongation).
void coarse_children(int o, int I, int J, int child[4][3][2]) {
  int cv[3][2];
  tri_vertices(o, I, J, cv);
  int A[3][2], M[3][2];
  for (int k = 0; k < 3; ++k) { A[k][0] = 2 * cv[k][0]; A[k][1] = 2 * cv[k][1]; }
  for (int k = 0; k < 3; ++k) {
    int a = (k + 1) % 3, b = (k + 2) % 3;
    M[k][0] = (A[a][0] + A[b][0]) / 2;
    M[k][1] = (A[a][1] + A[b][1]) / 2;
  }
  const int *pts[4][3] = {{A[0], M[2], M[1]}, {A[1], M[0], M[2]}, {A[2], M[1], M[0]}, {M[0], M[1], M[2]}};
  for (int c = 0; c < 4; ++c)
    for (int k = 0; k < 3; ++k) { child[c][k][0] = pts[c][k][0]; child[c][k][1] = pts[c][k][1]; }
}

}  // namespace

// Galerkin displacement block of the next coarser level (Sec. 3, R = P^T: the coarse
// operator P^T A P in place of the rediscretisation).  P_u is local to each coarse triangle
// T: every fine displacement DoF inside T or on its edges is a combination of T's nine
// coarse displacement DoFs (point values, half-edge bubbles and the zero-flux corner
// bubbles of Sec. 3.1 all use T's data only).  Hence P_u^T A_u P_u is again an element
// assembly, with element matrices E_T = sum over the four children t of Q_t^T E_t Q_t,
// Q_t the 9 x 9 map from T's local DoFs to t's.  For the elasticity part this gives a dense
// 9 x 9 matrix (Af -> Ac below).  The grad-div part needs no product: B_u,h P_u puts the
// whole divergence of T into its interior child, so P_u^T (lambda B_u^T M_p^{-1} B_u)_h P_u is
// 4 lambda (B_u^T M_p^{-1} B_u)_H exactly, i.e. lambda / |T| keeps its fine-level value.  The
// other blocks of P^T A P equal the rediscretised ones (nested RT0 and P0 spaces).
void galerkin_elasticity(const double Af[2][81], double Ac[2][81]) {
  for (int o = 0; o < 2; ++o) {
    const int I = 1, J = 1;
    SparseP P;
    local_prolongation(o, I, J, P);
    int child[4][3][2];
    coarse_children(o, I, J, child);
    double E[9][9] = {};
    for (int c = 0; c < 4; ++c) {
      int co, ci, cj;
      tri_of(child[c], &co, &ci, &cj);
      double Q[9][9];
      for (int b = 0; b < 9; ++b) {
        auto row = P.find(tri_dof(co, ci, cj, b));
        for (int a = 0; a < 9; ++a) {
          Q[b][a] = 0.0;
          if (row == P.end()) continue;
          auto it = row->second.find(tri_dof(o, I, J, a));
          if (it != row->second.end()) Q[b][a] = it->second;
        }
      }
      for (int a = 0; a < 9; ++a)
        for (int b = 0; b < 9; ++b) {
          double acc = 0.0;
          for (int r = 0; r < 9; ++r)
            for (int q = 0; q < 9; ++q) acc += Q[r][a] * Af[co][r * 9 + q] * Q[q][b];
          E[a][b] += acc;
        }
    }
    for (int a = 0; a < 9; ++a)
      for (int b = 0; b < 9; ++b) Ac[o][a * 9 + b] = 0.5 * (E[a][b] + E[b][a]);
  }
}

void galerkin_coarsen_coefs(const OpCoefs<double> &fine, OpCoefs<double> *c64, OpCoefs<float> *c32) {
  galerkin_elasticity(fine.A, c64->A);
  c64->lam_area = fine.lam_area;
  for (int o = 0; o < 2; ++o)
    for (int k = 0; k < 81; ++k) c32->A[o][k] = (float)c64->A[o][k];
  c32->lam_area = (float)c64->lam_area;
}

void build_transfer_tables(TransferTables *t) {
  std::memset(t, 0, sizeof(*t));
  const int NC = 6;
  SparseP P;
  for (int J = 0; J < NC; ++J)
    for (int I = 0; I < NC; ++I)
      for (int o = 0; o < 2; ++o) local_prolongation(o, I, J, P);
  const int C0 = 3;                     // interior coarse position
  for (int ty = 0; ty < NBLK; ++ty)
    for (int par = 0; par < 4; ++par) {
      int fi = 2 * C0 + (par & 1), fj = 2 * C0 + (par >> 1);
      auto it = P.find(DofKey{ty, fi, fj});
      int k = 0;
      if (it != P.end())
        for (auto &kv : it->second) {
          if (k >= kMaxPro) break;
          StencilEntry &e = t->pro[ty][par][k++];
          e.type = (int8_t)kv.first.type;
          e.di = (int8_t)(kv.first.i - C0);
          e.dj = (int8_t)(kv.first.j - C0);
          e.coef = kv.second;
          e.coef32 = (float)kv.second;
        }
      t->npro[ty][par] = k;
    }
  for (int ct = 0; ct < NBLK; ++ct) {
    DofKey c{ct, C0, C0};
    int k = 0;
    for (auto &row : P) {
      auto it = row.second.find(c);
      if (it == row.second.end()) continue;
      if (k >= kMaxRes) break;
      StencilEntry &e = t->res[ct][k++];
      e.type = (int8_t)row.first.type;
      e.di = (int8_t)(row.first.i - 2 * C0);
      e.dj = (int8_t)(row.first.j - 2 * C0);
      e.coef = it->second;
      e.coef32 = (float)it->second;
    }
    t->nres[ct] = k;
  }
  // children of a coarse triangle and the local RT0 interpolation onto each child
  for (int o = 0; o < 2; ++o) {
    int cv[3][2];
    tri_vertices(o, 0, 0, cv);
    Tri tc;
    tc.init(cv, 2.0);
    int A[3][2], M[3][2];
    for (int k = 0; k < 3; ++k) { A[k][0] = 2 * cv[k][0]; A[k][1] = 2 * cv[k][1]; }
    for (int k = 0; k < 3; ++k) {
      int a = (k + 1) % 3, b = (k + 2) % 3;
      M[k][0] = (A[a][0] + A[b][0]) / 2;
      M[k][1] = (A[a][1] + A[b][1]) / 2;
    }
    int child[4][3][2] = {{{A[0][0], A[0][1]}, {M[2][0], M[2][1]}, {M[1][0], M[1][1]}},
                          {{A[1][0], A[1][1]}, {M[0][0], M[0][1]}, {M[2][0], M[2][1]}},
                          {{A[2][0], A[2][1]}, {M[1][0], M[1][1]}, {M[0][0], M[0][1]}},
                          {{M[0][0], M[0][1]}, {M[1][0], M[1][1]}, {M[2][0], M[2][1]}}};
    for (int c = 0; c < 4; ++c) {
      int co, ci, cj;
      tri_of(child[c], &co, &ci, &cj);
      t->child_o[o][c] = co;
      t->child_di[o][c] = ci;
      t->child_dj[o][c] = cj;
      int sv[3][2];
      tri_vertices(co, ci, cj, sv);     // the child in its structured local order
      Tri ts;
      ts.init(sv, 1.0);
      for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
          double psi[2], dv;
          tc.w_basis(a, ts.mid[b], psi, &dv);
          t->Q[o][c][b][a] = psi[0] * ts.nrm[b][0] + psi[1] * ts.nrm[b][1];
        }
    }
  }
}

}  // namespace bmg
