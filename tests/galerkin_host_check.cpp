// Host-side check of the Galerkin coarse coefficients (galerkin_coarsen_coefs in
// element.cpp), compiled for the CPU: no device code runs here.
//
// usage: galerkin_host_check <n> <levels> <lambda> <mu> <out.bin>
//   out: for each coarse level l = 1..levels (grid n / 2^l): A[2][81], g[2][9], lam_area as
//        float64 (the displacement-block coefficients the operator kernel uses)
#include <cstdio>
#include <cstdlib>

#include "bmg_internal.h"

int main(int argc, char **argv) {
  if (argc != 6) return 2;
  const int n = std::atoi(argv[1]), levels = std::atoi(argv[2]);
  bmg::PhysParams p{std::atof(argv[3]), std::atof(argv[4]), 1.0, 1.0, 1.0};
  FILE *o = std::fopen(argv[5], "wb");
  if (!o) return 3;
  bmg::OpCoefs<double> fine, coarse;
  bmg::OpCoefs<float> f32;
  bmg::make_coefs(p, n, &fine, &f32);
  int m = n;
  for (int l = 1; l <= levels; ++l) {
    m /= 2;
    bmg::make_coefs(p, m, &coarse, &f32);
    bmg::galerkin_coarsen_coefs(fine, &coarse, &f32);
    std::fwrite(coarse.A, sizeof(double), 2 * 81, o);
    std::fwrite(coarse.g, sizeof(double), 2 * 9, o);
    std::fwrite(&coarse.lam_area, sizeof(double), 1, o);
    fine = coarse;
  }
  std::fclose(o);
  return 0;
}
