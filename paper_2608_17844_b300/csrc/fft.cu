// Lattice-axis FFT passes: the building block of the MLFFT (Eq. 2) used
// both for the one-time transform of the offset blocks into circulant bins
// (Eqs. 3 and 11) and for the per-iteration transforms of the vectors.
#include <cmath>
#include <stdexcept>

#include "internal.h"

namespace moma {

bool smooth_235(int m) {
  if (m < 1) return false;
  for (int r : {2, 3, 5})
    while (m % r == 0) m /= r;
  return m == 1;
}

int next_smooth(int n) {
  int m = n < 1 ? 1 : n;
  while (!smooth_235(m)) ++m;
  return m;
}

FftPlan make_plan(int M) {
  FftPlan p{};
  p.M = M;
  p.nst = 0;
  int m = M;
  while (m % 4 == 0) { p.radix[p.nst++] = 4; m /= 4; }
  while (m % 2 == 0) { p.radix[p.nst++] = 2; m /= 2; }
  while (m % 3 == 0) { p.radix[p.nst++] = 3; m /= 3; }
  while (m % 5 == 0) { p.radix[p.nst++] = 5; m /= 5; }
  if (m != 1 || p.nst > MOMA_FFT_MAXST) throw std::runtime_error("FFT length is not 2^a 3^b 5^c");
  return p;
}

static int pos_rec(const FftPlan &pl, int n, int M, int s) {
  if (s == pl.nst) return 0;
  const int r = pl.radix[s], Mp = M / r;
  return (n % r) * Mp + pos_rec(pl, n / r, Mp, s + 1);
}

std::vector<int> digit_reversal(const FftPlan &pl) {
  std::vector<int> pos(pl.M);
  for (int n = 0; n < pl.M; ++n) pos[n] = pos_rec(pl, n, pl.M, 0);
  return pos;
}

struct AxisKernelArgs {
  AxisPass p;
  FftPlan pl;
};

template <typename R, typename Cin, typename Cout>
__global__ void axis_kernel(AxisKernelArgs A, const typename Cplx<R>::T *__restrict__ tw_g,
                            const int *__restrict__ pos_g) {
  using C = typename Cplx<R>::T;
  extern __shared__ __align__(16) unsigned char smraw[];
  const AxisPass &p = A.p;
  const int M = A.pl.M;
  const int ld = blockDim.x;
  C *tw = reinterpret_cast<C *>(smraw);
  int *pos = reinterpret_cast<int *>(tw + M);
  C *col = reinterpret_cast<C *>(smraw + ((M * sizeof(C) + M * sizeof(int) + 15) & ~size_t(15)));
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    tw[i] = tw_g[i];
    pos[i] = pos_g[i];
  }
  __syncthreads();

  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p.ninner) return;  // lines are private: no block-wide sync below
  const int o1 = blockIdx.y % p.n1, o2 = blockIdx.y / p.n1;
  C *c = col + threadIdx.x;
  const Cin *src = reinterpret_cast<const Cin *>(p.in) + (long long)o1 * p.in_s1 + (long long)o2 * p.in_s2 + j;

  // Gather the line (zero padded).  in_mode 1 places the 2N-1 offsets of a
  // block-Toeplitz first column at circulant positions D mod M.
  const int Nc = (p.nin + 1) / 2;
#pragma unroll 4
  for (int m = 0; m < M; ++m) {
    int idx = -1;
    if (p.in_mode == 0) {
      if (m < p.nin) idx = m;
    } else {
      if (m < Nc) idx = m + Nc - 1;
      else if (m >= M - Nc + 1) idx = m - M + Nc - 1;
    }
    C v = czero<C>();
    if (idx >= 0) v = cvt<C>(src[(long long)idx * p.in_sm]);
    if (p.inverse) v = cconj(v);
    c[m * ld] = v;
  }

  fft_dif(c, ld, A.pl, tw);
  const R inv_m = (R)1 / (R)M;
  bool natural = false;
  if (p.refft_keep > 0) {
    for (int m = 0; m < M; ++m) {
      const int q = pos[m] * ld;
      c[q] = (m < p.refft_keep) ? cscale(cconj(c[q]), inv_m) : czero<C>();
    }
    fft_dit(c, ld, A.pl, tw);
    natural = true;
  }

  Cout *dst = reinterpret_cast<Cout *>(p.out);
  float2 *dst2 = reinterpret_cast<float2 *>(p.out2);
  for (int k = 0; k < p.nout; ++k) {
    C v = natural ? c[k * ld] : c[pos[k] * ld];
    if (p.inverse && !natural) v = cscale(cconj(v), inv_m);
    long long off;
    if (p.out_mode == 0) {
      off = (long long)o1 * p.out_s1 + (long long)o2 * p.out_s2 + (long long)k * p.out_sm + j;
    } else {
      const int slot = p.slot_of[k * p.slot_mul + o1];
      if (slot < 0) continue;
      const long long jj = p.remap_b > 0 ? (long long)(j / p.remap_b) * p.remap_ld + (j % p.remap_b) : j;
      off = (long long)slot * p.out_sm + jj;
    }
    dst[off] = cvt<Cout>(v);
    if (dst2) dst2[off] = cvt<float2>(v);
  }
}

template <typename R, typename Cin, typename Cout>
static void launch_typed(const AxisPass &p, const FftTables &t, cudaStream_t st) {
  using C = typename Cplx<R>::T;
  const int M = t.plan.M;
  int tj = 128;
  while (tj > 32 && (size_t)M * tj * sizeof(C) > 96 * 1024) tj /= 2;
  while (tj > 32 && tj / 2 >= p.ninner) tj /= 2;
  const size_t head = ((size_t)M * sizeof(C) + (size_t)M * sizeof(int) + 15) & ~size_t(15);
  const size_t smem = head + (size_t)M * tj * sizeof(C);
  static int configured = 0;
  if (!configured) {
    cudaFuncSetAttribute(axis_kernel<R, Cin, Cout>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    configured = 1;
  }
  dim3 grid((p.ninner + tj - 1) / tj, p.n1 * p.n2);
  AxisKernelArgs a{p, t.plan};
  const C *tw = nullptr;
  if constexpr (sizeof(R) == 8) tw = t.tw64; else tw = t.tw32;
  axis_kernel<R, Cin, Cout><<<grid, tj, smem, st>>>(a, tw, t.pos);
}

template <typename R>
void launch_axis_pass(const AxisPass &p, const FftTables &t, cudaStream_t st) {
  if (p.ninner <= 0 || p.n1 * p.n2 <= 0) return;
  if (p.in_c128 && p.out_c128) launch_typed<R, double2, double2>(p, t, st);
  else if (p.in_c128) launch_typed<R, double2, float2>(p, t, st);
  else if (p.out_c128) launch_typed<R, float2, double2>(p, t, st);
  else launch_typed<R, float2, float2>(p, t, st);
}

template void launch_axis_pass<float>(const AxisPass &, const FftTables &, cudaStream_t);
template void launch_axis_pass<double>(const AxisPass &, const FftTables &, cudaStream_t);

}  // namespace moma
