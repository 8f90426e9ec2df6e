// Lattice-axis FFT passes: the building block of the MLFFT (Eq. 2) used
// both for the one-time transform of the offset blocks into circulant bins
// (Eqs. 3 and 11) and for the per-iteration transforms of the vectors.
#include <algorithm>
#include <cmath>
#include <stdexcept>
#include <type_traits>

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
  int span = M;
  for (int s = 0; s < p.nst; ++s) {
    p.span[s] = span;
    span /= p.radix[s];
  }
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

// One CTA transforms 32 consecutive lines (inner indices j0 .. j0+31) of
// one (o1, o2) slice; G = blockDim.x / 32 threads cooperate on each line,
// splitting its loads, butterflies and stores, with a barrier between
// stages.  Line jj lives in shared memory at col[m * 32 + jj], so a warp
// (32 lines, same sub-thread) touches 32 consecutive words.
template <typename R, typename Cin, typename Cout>
__global__ void axis_kernel(AxisKernelArgs A, const typename Cplx<R>::T *__restrict__ tw_g,
                            const int *__restrict__ pos_g) {
  using C = typename Cplx<R>::T;
  extern __shared__ __align__(16) unsigned char smraw[];
  const AxisPass &p = A.p;
  if (p.live && *p.live == 0) return;
  const int M = A.pl.M;
  constexpr int ld = 32;
  C *tw = reinterpret_cast<C *>(smraw);
  int *pos = reinterpret_cast<int *>(tw + M);
  C *col = reinterpret_cast<C *>(smraw + ((M * sizeof(C) + M * sizeof(int) + 15) & ~size_t(15)));
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    tw[i] = tw_g[i];
    pos[i] = pos_g[i];
  }
  const int jj = threadIdx.x & 31, g = threadIdx.x >> 5, G = blockDim.x >> 5;
  const int j = blockIdx.x * 32 + jj;
  const bool act = j < p.ninner;
  const int o1 = blockIdx.y % p.n1, o2 = blockIdx.y / p.n1;
  C *c = col + jj;
  const Cin *src = reinterpret_cast<const Cin *>(p.in) + (long long)o1 * p.in_s1 + (long long)o2 * p.in_s2 + j;

  // Gather this thread's points m = g, g + G, ... (zero padded), UL loads
  // in flight at a time.  in_mode 1 places the 2N-1 offsets of a
  // block-Toeplitz first column at circulant positions D mod M.
  const int Nc = (p.nin + 1) / 2;
  const long long jin = (act && p.inner_in_map) ? (long long)p.inner_in_map[j] - j : 0;
  constexpr int UL = sizeof(R) == 4 ? 16 : 8;
  for (int m0 = g; m0 < M; m0 += G * UL) {
    C v[UL];
#pragma unroll
    for (int u = 0; u < UL; ++u) {
      const int m = m0 + u * G;
      int idx = -1;
      if (act && m < M) {
        if (p.in_mode == 0) {
          if (m < p.nin) idx = m;
        } else {
          if (m < Nc) idx = m + Nc - 1;
          else if (m >= M - Nc + 1) idx = m - M + Nc - 1;
        }
      }
      v[u] = idx >= 0 ? cvt<C>(src[(long long)idx * p.in_sm + jin]) : czero<C>();
    }
#pragma unroll
    for (int u = 0; u < UL; ++u) {
      const int m = m0 + u * G;
      if (m < M) c[m * ld] = p.inverse ? cconj(v[u]) : v[u];
    }
  }
  __syncthreads();
  for (int s = 0; s < A.pl.nst; ++s) {
    dif_stage(c, ld, A.pl, tw, s, g, G);
    __syncthreads();
  }
  const R inv_m = (R)1 / (R)M;
  bool natural = false;
  if (p.refft_keep > 0) {
    for (int m = g; m < M; m += G) {
      const int q = pos[m] * ld;
      c[q] = (m < p.refft_keep) ? cscale(cconj(c[q]), inv_m) : czero<C>();
    }
    __syncthreads();
    for (int s = A.pl.nst - 1; s >= 0; --s) {
      dit_stage(c, ld, A.pl, tw, s, g, G);
      __syncthreads();
    }
    natural = true;
  }
  if (!act) return;

  Cout *dst = reinterpret_cast<Cout *>(p.out);
  float2 *dst2 = reinterpret_cast<float2 *>(p.out2);
  int ti = 0, tj = 0;
  if (p.out_mode == 2) {
    const int2 t = p.tri[j];
    ti = t.x;
    tj = t.y;
  }
  for (int k = g; k < p.nout; k += G) {
    C v = natural ? c[k * ld] : c[pos[k] * ld];
    if (p.inverse && !natural) v = cscale(cconj(v), inv_m);
    long long off, off2 = -1;
    if (p.out_mode == 0) {
      off = (long long)o1 * p.out_s1 + (long long)o2 * p.out_s2 + (long long)k * p.out_sm + j;
    } else if (p.out_mode == 1) {
      const int slot = p.slot_of[k * p.slot_mul + o1];
      if (slot < 0) continue;
      const long long jx = p.remap_b > 0 ? (long long)(j / p.remap_b) * p.remap_ld + (j % p.remap_b) : j;
      off = (long long)slot * p.out_sm + jx;
    } else {
      // Symmetric scatter: line j carries entry (ti, tj), ti <= tj, of every
      // bin.  A stored (canonical) bin takes it at (ti, tj); the partner bin
      // -k is the transpose, so its value lands at (tj, ti) of the stored
      // block; a self-paired bin takes both.
      const int2 bs = p.bin_slot[k * p.slot_mul + o1];
      const long long base = (long long)bs.x * p.out_sm;
      if (bs.y == 1) {
        // The diagonal of the partner is the stored bin's own diagonal:
        // written once, by the stored bin, so the result is deterministic.
        if (ti == tj) continue;
        off = base + (long long)tj * p.remap_ld + ti;
      } else {
        off = base + (long long)ti * p.remap_ld + tj;
        if (bs.y == 2 && ti != tj) off2 = base + (long long)tj * p.remap_ld + ti;
      }
    }
    const Cout o = cvt<Cout>(v);
    dst[off] = o;
    if (dst2) dst2[off] = cvt<float2>(v);
    if (off2 >= 0) {
      dst[off2] = o;
      if (dst2) dst2[off2] = cvt<float2>(v);
    }
  }
}

template <typename R, typename Cin, typename Cout>
static void launch_typed(const AxisPass &p, const FftTables &t, cudaStream_t st) {
  using C = typename Cplx<R>::T;
  const int M = t.plan.M;
  // G threads per line: about 16 points each; when the batch has few lines
  // (vector passes at small nrhs) G grows -- up to one butterfly per thread
  // per stage -- until there are ~24 warps per SM to hide latency.
  int gmax = 1;
  for (int s = 0; s < t.plan.nst; ++s) gmax = std::max(gmax, M / t.plan.radix[s]);
  if (gmax > 32) gmax = 32;
  int G = std::max(1, std::min(8, M / 16));
  const long long ctas = (long long)((p.ninner + 31) / 32) * p.n1 * p.n2;
  while (G * 2 <= gmax && ctas * G < 24LL * 148) G *= 2;
  if (p.G > 0) G = std::min(p.G, 32);
  // Never more threads than the compiled kernel's registers allow.
  static int max_threads = 0;
  if (!max_threads) {
    cudaFuncAttributes attr{};
    max_threads = cudaFuncGetAttributes(&attr, axis_kernel<R, Cin, Cout>) == cudaSuccess ? attr.maxThreadsPerBlock : 256;
  }
  while (G > 1 && 32 * G > max_threads) G >>= 1;
  const size_t head = ((size_t)M * sizeof(C) + (size_t)M * sizeof(int) + 15) & ~size_t(15);
  const size_t smem = head + (size_t)M * 32 * sizeof(C);
  static int configured = 0;
  if (!configured) {
    cudaFuncSetAttribute(axis_kernel<R, Cin, Cout>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    configured = 1;
  }
  dim3 grid((p.ninner + 31) / 32, p.n1 * p.n2);
  AxisKernelArgs a{p, t.plan};
  const C *tw = nullptr;
  if constexpr (std::is_same<R, double>::value) tw = t.tw64;
  else if constexpr (std::is_same<R, dfl>::value) tw = t.twdf;
  else tw = t.tw32;
  axis_kernel<R, Cin, Cout><<<grid, 32 * G, smem, st>>>(a, tw, t.pos);
}

// Element types of the pass's input / output: 0 = c64, 1 = c128, 2 = dfl2.
template <typename R>
void launch_axis_pass(const AxisPass &p, const FftTables &t, cudaStream_t st) {
  if (p.ninner <= 0 || p.n1 * p.n2 <= 0) return;
  if constexpr (std::is_same<R, float>::value) {
    if (axis_reg_supported(p, t.plan.M) && (int)t.tw32_host.size() == t.plan.M) {
      launch_axis_reg(p, t, st);
      return;
    }
  }
  const int io = p.in_c128 * 3 + p.out_c128;
  if constexpr (std::is_same<R, dfl>::value) {
    switch (io) {
      case 0 * 3 + 2: launch_typed<R, float2, dfl2>(p, t, st); break;
      case 1 * 3 + 2: launch_typed<R, double2, dfl2>(p, t, st); break;
      case 2 * 3 + 2: launch_typed<R, dfl2, dfl2>(p, t, st); break;
      case 2 * 3 + 1: launch_typed<R, dfl2, double2>(p, t, st); break;
      default: throw std::runtime_error("axis pass: unsupported element types for dfl");
    }
  } else {
    if (p.in_c128 > 1 || p.out_c128 > 1) throw std::runtime_error("axis pass: dfl2 storage needs dfl arithmetic");
    if (p.in_c128 && p.out_c128) launch_typed<R, double2, double2>(p, t, st);
    else if (p.in_c128) launch_typed<R, double2, float2>(p, t, st);
    else if (p.out_c128) launch_typed<R, float2, double2>(p, t, st);
    else launch_typed<R, float2, float2>(p, t, st);
  }
}

template void launch_axis_pass<float>(const AxisPass &, const FftTables &, cudaStream_t);
template void launch_axis_pass<double>(const AxisPass &, const FftTables &, cudaStream_t);
template void launch_axis_pass<dfl>(const AxisPass &, const FftTables &, cudaStream_t);

}  // namespace moma
