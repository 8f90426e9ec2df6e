// Column FFT engine for the lattice transforms of the MLFFT (Eq. 2:
// F^[2] = F_{Ny} (x) (F_{Nx} (x) I_b), i.e. independent 1D DFTs along the
// x and y lattice axes with the basis index untouched).
//
// One thread owns one 1D line of length M held in shared memory with a
// stride of `ld` elements (column m of thread t at col[m * ld + t]), so no
// synchronisation is needed between stages and consecutive threads touch
// consecutive words (conflict-free).  M = r_0 r_1 ... r_{k-1} with radices
// in {2, 3, 4, 5}.
//
//  * dif(): natural-order input -> output X[k] at position pos[k]
//    (decimation in frequency; stage s splits the current sub-problem of
//    length Ms into r_s sub-problems, twiddle after the butterfly).
//  * dit(): input x[n] at position pos[n] -> natural-order output
//    (decimation in time; the mirror image, twiddle before the butterfly).
// pos[] is the mixed-radix digit reversal: with n = r_0 n' + n_0,
// pos(n) = n_0 (M / r_0) + pos'(n') on the remaining radices.
//
// Forward kernel is exp(-2 pi i k n / M) (the sign of Eq. 11); the inverse
// is taken as conj(DFT(conj(.))) / M.
#pragma once
#include "common.cuh"

#define MOMA_FFT_MAXST 16

struct FftPlan {
  int M;
  int nst;
  int radix[MOMA_FFT_MAXST];
  int span[MOMA_FFT_MAXST];  // span[s] = radix[s] * radix[s+1] * ... (span[0] = M)
};

// Radix-R forward DFT in registers: b[k] = sum_n a[n] w_R^{nk}.
// tw[t] = exp(-2 pi i t / M); w_R = tw[M / R].  R is a compile-time
// constant so that a[] stays in registers.
template <int R, typename C>
MOMA_HD void butterfly(C *a, const C *tw, int M) {
  using Rl = decltype(a[0].x);
  if constexpr (R == 2) {
    C t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  } else if constexpr (R == 4) {
    C s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
    C s13 = cadd(a[1], a[3]), d13 = csub(a[1], a[3]);
    a[0] = cadd(s02, s13);
    a[2] = csub(s02, s13);
    a[1] = cadd(d02, cmul_mi(d13));
    a[3] = csub(d02, cmul_mi(d13));
  } else if constexpr (R == 3) {
    const Rl s = -tw[M / 3].y;  // sin(2 pi / 3)
    C t1 = cadd(a[1], a[2]);
    C t2 = csub(a[0], cscale(t1, (Rl)0.5));
    C d = csub(a[1], a[2]);
    C t3 = cscale(cmul_mi(d), s);
    a[0] = cadd(a[0], t1);
    a[1] = cadd(t2, t3);
    a[2] = csub(t2, t3);
  } else {  // R == 5
    const C w1 = tw[M / 5], w2 = tw[(2 * M) / 5];
    const Rl c1 = w1.x, s1 = -w1.y, c2 = w2.x, s2 = -w2.y;
    C t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
    C t3 = csub(a[1], a[4]), t4 = csub(a[2], a[3]);
    C a0 = a[0];
    C p1 = cadd(a0, cadd(cscale(t1, c1), cscale(t2, c2)));
    C p2 = cadd(a0, cadd(cscale(t1, c2), cscale(t2, c1)));
    C q1 = cadd(cscale(t3, s1), cscale(t4, s2));
    C q2 = csub(cscale(t3, s2), cscale(t4, s1));
    a[0] = cadd(a0, cadd(t1, t2));
    a[1] = cadd(p1, cmul_mi(q1));
    a[4] = csub(p1, cmul_mi(q1));
    a[2] = cadd(p2, cmul_mi(q2));
    a[3] = csub(p2, cmul_mi(q2));
  }
}

// One stage of the transform, restricted to the butterflies bt = g, g + ng,
// ... of that stage (ng cooperating threads share a line; the stages must
// be separated by a barrier).  Stage s works on sub-problems of length
// span[s] = r_s r_{s+1} ... r_{k-1}; there are M / span[s] of them.
template <int R, typename C>
MOMA_HD void dif_stage_r(C *col, int ld, const FftPlan &pl, const C *tw, int s, int g, int ng) {
  const int M = pl.M, Ms = pl.span[s], Mp = Ms / R, G = M / Ms;
  const int nbt = M / R;
  for (int bt = g; bt < nbt; bt += ng) {
    const int seg = bt / Mp, k = bt - seg * Mp;
    C *base = col + (size_t)seg * Ms * ld;
    C a[R];
#pragma unroll
    for (int n = 0; n < R; ++n) a[n] = base[(n * Mp + k) * ld];
    butterfly<R>(a, tw, M);
    base[k * ld] = a[0];
    if (k == 0) {  // unit twiddles
#pragma unroll
      for (int n = 1; n < R; ++n) base[n * Mp * ld] = a[n];
    } else {
#pragma unroll
      for (int n = 1; n < R; ++n) base[(n * Mp + k) * ld] = cmul(a[n], tw[k * n * G]);
    }
  }
}

template <int R, typename C>
MOMA_HD void dit_stage_r(C *col, int ld, const FftPlan &pl, const C *tw, int s, int g, int ng) {
  const int M = pl.M, Ms = pl.span[s], Mp = Ms / R, G = M / Ms;
  const int nbt = M / R;
  for (int bt = g; bt < nbt; bt += ng) {
    const int seg = bt / Mp, k = bt - seg * Mp;
    C *base = col + (size_t)seg * Ms * ld;
    C a[R];
    a[0] = base[k * ld];
    if (k == 0) {  // unit twiddles
#pragma unroll
      for (int n = 1; n < R; ++n) a[n] = base[n * Mp * ld];
    } else {
#pragma unroll
      for (int n = 1; n < R; ++n) a[n] = cmul(base[(n * Mp + k) * ld], tw[k * n * G]);
    }
    butterfly<R>(a, tw, M);
#pragma unroll
    for (int n = 0; n < R; ++n) base[(n * Mp + k) * ld] = a[n];
  }
}

template <typename C>
MOMA_HD void dif_stage(C *col, int ld, const FftPlan &pl, const C *tw, int s, int g, int ng) {
  switch (pl.radix[s]) {
    case 2: dif_stage_r<2>(col, ld, pl, tw, s, g, ng); break;
    case 3: dif_stage_r<3>(col, ld, pl, tw, s, g, ng); break;
    case 4: dif_stage_r<4>(col, ld, pl, tw, s, g, ng); break;
    default: dif_stage_r<5>(col, ld, pl, tw, s, g, ng); break;
  }
}

template <typename C>
MOMA_HD void dit_stage(C *col, int ld, const FftPlan &pl, const C *tw, int s, int g, int ng) {
  switch (pl.radix[s]) {
    case 2: dit_stage_r<2>(col, ld, pl, tw, s, g, ng); break;
    case 3: dit_stage_r<3>(col, ld, pl, tw, s, g, ng); break;
    case 4: dit_stage_r<4>(col, ld, pl, tw, s, g, ng); break;
    default: dit_stage_r<5>(col, ld, pl, tw, s, g, ng); break;
  }
}

// Single-thread transforms (one thread owns the whole line).
template <typename C>
MOMA_HD void fft_dif(C *col, int ld, const FftPlan &pl, const C *tw) {
  for (int s = 0; s < pl.nst; ++s) dif_stage(col, ld, pl, tw, s, 0, 1);
}
template <typename C>
MOMA_HD void fft_dit(C *col, int ld, const FftPlan &pl, const C *tw) {
  for (int s = pl.nst - 1; s >= 0; --s) dit_stage(col, ld, pl, tw, s, 0, 1);
}
