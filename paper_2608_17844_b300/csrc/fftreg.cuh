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
// tw is a table of exp(-2 pi i t / (M TS)): a length-M transform reads every
// TS-th entry, so one table of the longest length serves its divisors.
template <int M, int S, int TS = 1>
MOMA_HD void rg_dit_stage(float2 (&v)[M], const float2 *tw) {
  constexpr int R = rg_radix(M, S), Ms = rg_span(M, S), Mp = Ms / R, G = M / Ms;
#pragma unroll
  for (int bt = 0; bt < M / R; ++bt) {
    const int seg = bt / Mp, k = bt % Mp;
    float2 a[R];
#pragma unroll
    for (int n = 0; n < R; ++n) {
      a[n] = v[seg * Ms + n * Mp + k];
      if (n > 0 && k > 0) a[n] = cmul(a[n], tw[k * n * G * TS]);
    }
    butterfly<R>(a, tw, M * TS);
#pragma unroll
    for (int n = 0; n < R; ++n) v[seg * Ms + n * Mp + k] = a[n];
  }
}

template <int M, int S, int TS = 1>
MOMA_HD void rg_dit(float2 (&v)[M], const float2 *tw) {
  if constexpr (S >= 0) {
    rg_dit_stage<M, S, TS>(v, tw);
    rg_dit<M, S - 1, TS>(v, tw);
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
// to its digit-reversed positions (a register renaming).  tw: see
// rg_dit_stage (TS = 1: a table of length M itself).
template <int M, int TS = 1>
MOMA_HD void rg_fft(float2 (&v)[M], const float2 *tw) {
  float2 u[M];
  rg_scatter<M>(u, v, std::make_integer_sequence<int, M>{});
  rg_dit<M, rg_nst(M) - 1, TS>(u, tw);
#pragma unroll
  for (int n = 0; n < M; ++n) v[n] = u[n];
}

// ------------------------------------------------ several lanes per line --
// A length-M line split over P lanes (M = P Q, P^2 | M): lane s holds the
// points n = s + P q, q = 0 .. Q-1, in y[q].  With n = s + P q and
// k = k2 + Q k1 (Cooley-Tukey, M = P x Q):
//   X[k2 + Q k1] = sum_s W_P^{s k1} W_M^{s k2} sum_q y_s[q] W_Q^{q k2}.
// (1) each lane transforms its own Q points (Y_s[k2]); (2) the lanes of a
// line exchange through shared memory so that lane s gathers Y_t[k2] of
// every lane t for its Q/P frequencies k2 = s + P u; (3) it scales them by
// W_M^{t k2} and transforms across t.  The result X[k2 + Q k1] goes back to
// y[u + (Q/P) k1], whose point index s + P (u + (Q/P) k1) = k2 + Q k1 is
// the lane's own input distribution: the transform maps the distributed
// natural order to itself, so a second transform needs no extra exchange.
//
// Exchange buffer of a warp: [Q][kLaneLd] complex, lane l P + s writing
// row k2 at column l P + s.  The row stride 33 = 1 (mod 16) spreads the
// gather of step (2) -- lanes (l, s) reading row s + P u, column l P + t --
// over all 16 eight-byte bank pairs, two lanes each.
constexpr int kLaneLd = 33;

template <int M, int P>
struct LaneShape {
  static constexpr int Q = M / P, U = Q / P, L = 32 / P;
  static_assert(P >= 1 && 32 % P == 0 && M % (P * P) == 0, "P lanes per line need P^2 | M and P | 32");
};

// Step (1): the lane's own Q-point transform (twiddles: every P-th entry of
// the length-M table).
template <int M, int P>
MOMA_HD void lane_stage1(float2 (&y)[M / P], const float2 *tw) {
  rg_fft<M / P, P>(y, tw);
}
// Write the lane's Y_s[k2] into the warp's exchange buffer.
template <int M, int P>
MOMA_HD void lane_put(float2 *buf, const float2 (&y)[M / P], int lane) {
#pragma unroll
  for (int k2 = 0; k2 < M / P; ++k2) buf[k2 * kLaneLd + lane] = y[k2];
}
// The runtime twiddles W_M^{t k2}, k2 = s + P u, t = 1 .. P-1, of lane s
// (tw_full: the length-M table; t k2 <= (P - 1)(Q - 1) < M).
template <int M, int P>
MOMA_HD void lane_twiddles(float2 (&w)[LaneShape<M, P>::U][P], const float2 *tw_full, int s) {
#pragma unroll
  for (int u = 0; u < LaneShape<M, P>::U; ++u)
#pragma unroll
    for (int t = 0; t < P; ++t) w[u][t] = t == 0 ? make_float2(1.f, 0.f) : tw_full[t * (s + P * u)];
}
// Steps (2), (3): gather, twiddle, transform across the lanes, and leave
// X[s + P q] in y[q].  The buffer must hold every lane's lane_put.
template <int M, int P>
MOMA_HD void lane_stage2(float2 (&y)[M / P], const float2 *buf, int s, int l,
                         const float2 (&w)[LaneShape<M, P>::U][P], const float2 *tw) {
  constexpr int Q = M / P, U = Q / P;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    float2 z[P];
#pragma unroll
    for (int t = 0; t < P; ++t) {
      const float2 v = buf[(s + P * u) * kLaneLd + l * P + t];
      z[t] = t == 0 ? v : cmul(v, w[u][t]);
    }
    rg_fft<P, Q>(z, tw);
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) y[u + U * k1] = z[k1];
  }
}

}  // namespace moma
