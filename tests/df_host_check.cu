// Host-side check of the FP64 <-> FP32 conversions and the double-float dot step used by the
// Arnoldi kernels (kernels_common.cuh), compiled for the CPU: no device code runs here.
//
// usage: df_host_check <in.f64> <out.bin>
//   in:  n (as a double), then n float64 values v[i], then 2m float64 values a[j], b[j]
//        (m = the rest of the file / 2)
//   out: per v[i]: trunc(v) as float32, head, tail (float32), f32_to_f64_bits(trunc(v));
//        then the double-float dot sum_j a[j] b[j] as (sh, sl) float32
#include <cstdio>
#include <vector>

#include "kernels_common.cuh"

int main(int argc, char **argv) {
  if (argc != 3) return 2;
  FILE *f = std::fopen(argv[1], "rb");
  if (!f) return 3;
  std::vector<double> in;
  double x;
  while (std::fread(&x, sizeof x, 1, f) == 1) in.push_back(x);
  std::fclose(f);
  if (in.empty()) return 4;
  const size_t n = (size_t)in[0];
  if (1 + n > in.size() || (in.size() - 1 - n) % 2) return 5;
  const size_t m = (in.size() - 1 - n) / 2;
  FILE *o = std::fopen(argv[2], "wb");
  if (!o) return 6;
  for (size_t i = 0; i < n; ++i) {
    const double v = in[1 + i];
    float head, tail;
    bmg::split_f64(v, head, tail);
    const float t = bmg::f64_to_f32_trunc(v);
    const double back = bmg::f32_to_f64_bits(t);
    std::fwrite(&t, sizeof t, 1, o);
    std::fwrite(&head, sizeof head, 1, o);
    std::fwrite(&tail, sizeof tail, 1, o);
    std::fwrite(&back, sizeof back, 1, o);
  }
  float sh = 0.f, sl = 0.f;
  for (size_t j = 0; j < m; ++j) {
    float ah, al, bh, bl;
    bmg::split_f64(in[1 + n + j], ah, al);
    bmg::split_f64(in[1 + n + m + j], bh, bl);
    bmg::df_dot_step(ah, al, bh, bl, sh, sl);
  }
  std::fwrite(&sh, sizeof sh, 1, o);
  std::fwrite(&sl, sizeof sl, 1, o);
  std::fclose(o);
  return 0;
}
