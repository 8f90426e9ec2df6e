// Compile-time register-resident FFT of length M (2, 3, 5-smooth), the
// transform core of fftreg.cu, usable from host code for checks.  The
// radices, spans and digit reversal are those of make_plan / digit_reversal
// in fft.cu, computed as constant expressions so that every register index
// is known at compile time.
#pragma once
#include <utility>

#include "fft.cuh"

namespace moma {

constexpr int kRegMaxM = 64;

// Radix sequence of make_plan (fft.cu): fours, then a two, threes, fives.
constexpr int rg_nst(int M) {
  int n = 0, m = M;
  while (m % 4 == 0) { m /= 4; ++n; }
  while (m % 2 == 0) { m /= 2; ++n; }
  while (m % 3 == 0) { m /= 3; ++n; }
  while (m % 5 == 0) { m /= 5; ++n; }
  return n;
}
constexpr int rg_radix(int M, int s) {
  int n = 0, m = M;
  while (m % 4 == 0) { if (n == s) return 4; m /= 4; ++n; }
  while (m % 2 == 0) { if (n == s) return 2; m /= 2; ++n; }
  while (m % 3 == 0) { if (n == s) return 3; m /= 3; ++n; }
  while (m % 5 == 0) { if (n == s) return 5; m /= 5; ++n; }
  return 1;
}
constexpr int rg_span(int M, int s) {  // span[s] = r_s r_{s+1} ... (span[0] = M)
  int sp = M;
  for (int t = 0; t < s; ++t) sp /= rg_radix(M, t);
  return sp;
}
// Digit reversal of fft.cu: n = r_0 n' + n_0 -> n_0 (M / r_0) + pos'(n').
constexpr int rg_pos(int M, int n, int s = 0, int Mcur = -1) {
  if (Mcur < 0) Mcur = M;
  if (s == rg_nst(M)) return 0;
  const int r = rg_radix(M, s), Mp = Mcur / r;
  return (n % r) * Mp + rg_pos(M, n / r, s + 1, Mp);
}

// One DIT stage on the register line v (compile-time indices throughout).
template <int M, int S>
MOMA_HD void rg_dit_stage(float2 (&v)[M], const float2 *tw) {
  constexpr int R = rg_radix(M, S), Ms = rg_span(M, S), Mp = Ms / R, G = M / Ms;
#pragma unroll
  for (int bt = 0; bt < M / R; ++bt) {
    const int seg = bt / Mp, k = bt % Mp;
    float2 a[R];
#pragma unroll
    for (int n = 0; n < R; ++n) {
      a[n] = v[seg * Ms + n * Mp + k];
      if (n > 0 && k > 0) a[n] = cmul(a[n], tw[k * n * G]);
    }
    butterfly<R>(a, tw, M);
#pragma unroll
    for (int n = 0; n < R; ++n) v[seg * Ms + n * Mp + k] = a[n];
  }
}

template <int M, int S>
MOMA_HD void rg_dit(float2 (&v)[M], const float2 *tw) {
  if constexpr (S >= 0) {
    rg_dit_stage<M, S>(v, tw);
    rg_dit<M, S - 1>(v, tw);
  }
}

// Digit-reversed position of point N as a template constant, so that the
// scatter below indexes registers with true compile-time constants.
template <int M, int N>
struct RgPos {
  static constexpr int value = rg_pos(M, N);
};
template <int M, int... N>
MOMA_HD void rg_scatter(float2 (&u)[M], const float2 (&v)[M], std::integer_sequence<int, N...>) {
  ((u[RgPos<M, N>::value] = v[N]), ...);
}

// v (natural order) -> DFT of v in natural order.  The input is first moved
// to its digit-reversed positions (a register renaming).
template <int M>
MOMA_HD void rg_fft(float2 (&v)[M], const float2 *tw) {
  float2 u[M];
  rg_scatter<M>(u, v, std::make_integer_sequence<int, M>{});
  rg_dit<M, rg_nst(M) - 1>(u, tw);
#pragma unroll
  for (int n = 0; n < M; ++n) v[n] = u[n];
}

}  // namespace moma
