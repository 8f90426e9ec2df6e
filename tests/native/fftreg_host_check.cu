// Host driver of the compile-time register FFT (csrc/fftreg.cuh): reads
// "M keep P" then M complex values; prints the forward transform, then the
// inverse transform, then (keep > 0) the inverse / keep-first-`keep` /
// forward sequence of the mask pass -- the three operations of the
// register-resident lattice passes, in the same order of arithmetic.
// P > 1: the same through the split transform of P lanes per line, with a
// whole warp emulated (L = 32 / P lines, line l holding the input shifted
// cyclically by l, all lines sharing the exchange buffer as on the device);
// every line's three results are printed, line after line.
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

// One split transform of the emulated warp: y[lane] in the lanes' input
// distribution, in place (the device's lane_stage1, exchange, lane_stage2).
template <int M, int P>
static void lane_transform(std::vector<std::vector<float2>> &y, const float2 *tw) {
  constexpr int Q = M / P, L = 32 / P, U = Q / P;
  std::vector<float2> buf((size_t)Q * kLaneLd, make_float2(NAN, NAN));
  for (int lane = 0; lane < 32; ++lane) {
    float2 v[Q];
    for (int q = 0; q < Q; ++q) v[q] = y[lane][q];
    lane_stage1<M, P>(v, tw);
    lane_put<M, P>(buf.data(), v, lane);
  }
  for (int lane = 0; lane < 32; ++lane) {
    const int s = lane % P, l = lane / P;
    float2 w[U][P];
    lane_twiddles<M, P>(w, tw, s);
    float2 v[Q];
    lane_stage2<M, P>(v, buf.data(), s, l, w, tw);
    for (int q = 0; q < Q; ++q) y[lane][q] = v[q];
  }
  (void)L;
}

template <int M, int P>
static void run_lanes(const std::vector<float2> &x, int keep) {
  constexpr int Q = M / P, L = 32 / P;
  std::vector<float2> tw(M);
  for (int t = 0; t < M; ++t) {
    const double a = -2.0 * M_PI * t / M;
    tw[t] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  auto load = [&](bool conj) {
    std::vector<std::vector<float2>> y(32, std::vector<float2>(Q));
    for (int lane = 0; lane < 32; ++lane) {
      const int s = lane % P, l = lane / P;
      for (int q = 0; q < Q; ++q) {
        float2 v = x[(s + P * q + l) % M];
        if (conj) v.y = -v.y;
        y[lane][q] = v;
      }
    }
    return y;
  };
  std::vector<std::vector<float2>> out[3];
  out[0] = load(false);
  lane_transform<M, P>(out[0], tw.data());
  out[1] = load(true);
  lane_transform<M, P>(out[1], tw.data());
  const float inv = 1.0f / (float)M;
  for (auto &v : out[1])
    for (auto &e : v) e = make_float2(e.x * inv, -e.y * inv);
  out[2] = out[1];
  for (int lane = 0; lane < 32; ++lane)
    for (int q = 0; q < Q; ++q)
      if (lane % P + P * q >= keep) out[2][lane][q] = make_float2(0.f, 0.f);
  lane_transform<M, P>(out[2], tw.data());
  for (int l = 0; l < L; ++l)
    for (int o = 0; o < 3; ++o)
      for (int k = 0; k < M; ++k) {
        const float2 v = out[o][l * P + k % P][k / P];
        std::printf("%.9g %.9g\n", v.x, v.y);
      }
}

int main() {
  int M, keep, P;
  while (std::scanf("%d %d %d", &M, &keep, &P) == 3) {
    std::vector<float2> x(M);
    for (int m = 0; m < M; ++m) std::scanf("%f %f", &x[m].x, &x[m].y);
    if (P == 1) {
      switch (M) {
#define CASE(n) case n: run<n>(x, keep); break;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(8) CASE(9) CASE(10) CASE(12) CASE(15) CASE(16)
        CASE(18) CASE(20) CASE(24) CASE(25) CASE(27) CASE(30) CASE(32) CASE(36) CASE(40) CASE(45) CASE(48)
        CASE(50) CASE(54) CASE(60) CASE(64)
#undef CASE
        default: return 1;
      }
    } else {
      const int key = M * 16 + P;
      switch (key) {
#define LCASE(n, p) case n * 16 + p: run_lanes<n, p>(x, keep); break;
        LCASE(4, 2) LCASE(8, 2) LCASE(12, 2) LCASE(16, 2) LCASE(20, 2) LCASE(24, 2) LCASE(32, 2) LCASE(36, 2)
        LCASE(40, 2) LCASE(48, 2) LCASE(60, 2) LCASE(64, 2) LCASE(16, 4) LCASE(32, 4) LCASE(48, 4) LCASE(64, 4)
        LCASE(64, 8)
#undef LCASE
        default: return 1;
      }
    }
  }
  return 0;
}
