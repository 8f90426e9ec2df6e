// Host-side check of the column FFT engine (fft.cuh) and its plans: reads
// M, a mode (dif|dit|inv_mask_fwd keep) and M complex values from stdin;
// prints the transform.  Built with nvcc as host code by the test suite.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"

int main(int argc, char **argv) {
  int M;
  char mode[32];
  int keep = 0;
  if (scanf("%d %31s %d", &M, mode, &keep) != 3) return 2;
  std::vector<double2> x(M);
  for (int i = 0; i < M; ++i)
    if (scanf("%lf %lf", &x[i].x, &x[i].y) != 2) return 2;
  FftPlan pl = moma::make_plan(M);
  std::vector<int> pos = moma::digit_reversal(pl);
  std::vector<double2> tw(M);
  for (int t = 0; t < M; ++t) {
    const double a = -2.0 * M_PI * t / M;
    tw[t] = make_double2(cos(a), sin(a));
  }
  std::vector<double2> col(M), out(M);
  if (!strcmp(mode, "dif")) {  // natural in, X[k] at pos[k]
    col = x;
    fft_dif(col.data(), 1, pl, tw.data());
    for (int k = 0; k < M; ++k) out[k] = col[pos[k]];
  } else if (!strcmp(mode, "difcoop")) {  // stages split over `keep` cooperating threads
    col = x;
    for (int s = 0; s < pl.nst; ++s)
      for (int g = 0; g < keep; ++g) dif_stage(col.data(), 1, pl, tw.data(), s, g, keep);
    for (int k = 0; k < M; ++k) out[k] = col[pos[k]];
  } else if (!strcmp(mode, "ditcoop")) {
    for (int n = 0; n < M; ++n) col[pos[n]] = x[n];
    for (int s = pl.nst - 1; s >= 0; --s)
      for (int g = 0; g < keep; ++g) dit_stage(col.data(), 1, pl, tw.data(), s, g, keep);
    out = col;
  } else if (!strcmp(mode, "dit")) {  // x[n] at pos[n], natural out
    for (int n = 0; n < M; ++n) col[pos[n]] = x[n];
    fft_dit(col.data(), 1, pl, tw.data());
    out = col;
  } else {  // inverse, keep first `keep`, forward again (the masked pass)
    for (int n = 0; n < M; ++n) col[n] = cconj(x[n]);
    fft_dif(col.data(), 1, pl, tw.data());
    for (int m = 0; m < M; ++m) {
      double2 &c = col[pos[m]];
      c = m < keep ? cscale(cconj(c), 1.0 / M) : make_double2(0, 0);
    }
    fft_dit(col.data(), 1, pl, tw.data());
    out = col;
  }
  printf("%d\n", pl.nst);
  for (int k = 0; k < M; ++k) printf("%.17g %.17g\n", out[k].x, out[k].y);
  return 0;
}
