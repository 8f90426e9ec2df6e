// Host driver of the compile-time register FFT (csrc/fftreg.cuh): reads
// "M keep" then M complex values; prints the forward transform, then the
// inverse transform, then (keep > 0) the inverse / keep-first-`keep` /
// forward sequence of the mask pass -- the three operations of the
// register-resident lattice passes, in the same order of arithmetic.
#include <cmath>
#include <cstdio>
#include <vector>

#include "fftreg.cuh"

using namespace moma;

template <int M>
static void run(const std::vector<float2> &x, int keep) {
  std::vector<float2> tw(M);
  for (int t = 0; t < M; ++t) {
    const double a = -2.0 * M_PI * t / M;
    tw[t] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  float2 v[M];
  for (int m = 0; m < M; ++m) v[m] = x[m];
  rg_fft<M>(v, tw.data());
  for (int m = 0; m < M; ++m) std::printf("%.9g %.9g\n", v[m].x, v[m].y);
  for (int m = 0; m < M; ++m) v[m] = make_float2(x[m].x, -x[m].y);
  rg_fft<M>(v, tw.data());
  const float inv = 1.0f / (float)M;
  for (int m = 0; m < M; ++m) v[m] = make_float2(v[m].x * inv, -v[m].y * inv);
  for (int m = 0; m < M; ++m) std::printf("%.9g %.9g\n", v[m].x, v[m].y);
  for (int m = keep; m < M; ++m) v[m] = make_float2(0.f, 0.f);
  rg_fft<M>(v, tw.data());
  for (int m = 0; m < M; ++m) std::printf("%.9g %.9g\n", v[m].x, v[m].y);
}

int main() {
  int M, keep;
  while (std::scanf("%d %d", &M, &keep) == 2) {
    std::vector<float2> x(M);
    for (int m = 0; m < M; ++m) std::scanf("%f %f", &x[m].x, &x[m].y);
    switch (M) {
#define CASE(n) case n: run<n>(x, keep); break;
      CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(8) CASE(9) CASE(10) CASE(12) CASE(15) CASE(16)
      CASE(18) CASE(20) CASE(24) CASE(25) CASE(27) CASE(30) CASE(32) CASE(36) CASE(40) CASE(45) CASE(48)
      CASE(50) CASE(54) CASE(60) CASE(64)
#undef CASE
      default: return 1;
    }
  }
  return 0;
}
