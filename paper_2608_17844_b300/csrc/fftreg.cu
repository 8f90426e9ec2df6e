// Register-resident lattice-axis transforms for circulant lengths M <= 64
// (the 1D building block of the MLFFT product, Eq. 2), for the c64 passes
// of the solve.  One thread owns one whole line of M points in registers;
// consecutive threads own consecutive basis indices j, so every load and
// store of a warp is one contiguous 256-byte row of the strided array (the
// basis index is the innermost dimension of every layout).  There is no
// shared memory, no barrier, and every point of a line is an independent
// load, so latency is hidden by instruction-level parallelism.
//
// The transform is the mixed-radix decimation in time of fft.cuh with M a
// compile-time constant: points enter at their digit-reversed positions
// (compile-time indices), the stages run fully unrolled, the output is in
// natural order.  Twiddles exp(-2 pi i t / M) travel in the kernel's
// parameter block (constant bank), indexed by compile-time offsets.
// Inverse: conj(DFT(conj x)) / M.  The mask pass between the Z and Z^H legs
// inverts, keeps the first refft_keep points, and transforms forward again.
//
// When the batch has few lines (the vector passes hold b x RHS x lattice-row
// lines: 8 K at a 32 x 32 lattice with b = 128 and 2 RHS, under two warps per
// SM sub-partition), P = 2, 4 or 8 lanes share a line instead
// (axis_lane_kernel, the split transform of fftreg.cuh): P times the warps,
// each with a P-th of the loads and about a third of the arithmetic chain.
#include <cstdlib>
#include <stdexcept>

#include "internal.h"
#include "fftreg.cuh"

namespace moma {

namespace {

struct Tw {
  float2 w[kRegMaxM];
};

struct RegArgs {
  AxisPass p;
  Tw tw;
};

template <int M>
__global__ void __launch_bounds__(128) axis_reg_kernel(const __grid_constant__ RegArgs A) {
  const AxisPass &p = A.p;
  if (p.live && *p.live == 0) return;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nlines = (long long)p.n1 * p.n2 * p.ninner;
  if (gid >= nlines) return;
  const int j = (int)(gid % p.ninner);
  const long long l12 = gid / p.ninner;
  const int o1 = (int)(l12 % p.n1), o2 = (int)(l12 / p.n1);
  const float2 *src = reinterpret_cast<const float2 *>(p.in) + (long long)o1 * p.in_s1 + (long long)o2 * p.in_s2 + j;
  float2 *dst = reinterpret_cast<float2 *>(p.out) + (long long)o1 * p.out_s1 + (long long)o2 * p.out_s2 + j;
  const float2 *tw = A.tw.w;
  float2 v[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    float2 x = m < p.nin ? src[(long long)m * p.in_sm] : make_float2(0.f, 0.f);
    if (p.inverse) x.y = -x.y;
    v[m] = x;
  }
  rg_fft<M>(v, tw);
  const float inv_m = 1.0f / (float)M;
  if (p.inverse) {
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = make_float2(v[m].x * inv_m, -v[m].y * inv_m);
    if (p.refft_keep > 0) {
#pragma unroll
      for (int m = 0; m < M; ++m)
        if (m >= p.refft_keep) v[m] = make_float2(0.f, 0.f);
      rg_fft<M>(v, tw);
    }
  }
#pragma unroll
  for (int k = 0; k < M; ++k)
    if (k < p.nout) dst[(long long)k * p.out_sm] = v[k];
}

// P lanes per line: warp w of the grid owns lines w L .. w L + L - 1
// (L = 32 / P), lane l P + s holding points s + P q of line w L + l.  Lanes
// past the last line load zeros and store nothing but still take part in
// the warp's exchange.
constexpr int kLaneThreads = 128;

template <int M, int P>
__global__ void __launch_bounds__(kLaneThreads) axis_lane_kernel(const __grid_constant__ RegArgs A,
                                                                 const float2 *__restrict__ tw_full) {
  using S = LaneShape<M, P>;
  constexpr int Q = S::Q, L = S::L;
  __shared__ float2 xbuf[kLaneThreads / 32][Q * kLaneLd];
  const AxisPass &p = A.p;
  if (p.live && *p.live == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int s = lane % P, l = lane / P;
  const long long nlines = (long long)p.n1 * p.n2 * p.ninner;
  const long long line0 = ((long long)blockIdx.x * (kLaneThreads / 32) + warp) * L;
  if (line0 >= nlines) return;  // the whole warp is past the end
  const long long line = line0 + l;
  const bool act = line < nlines;
  const long long lc = act ? line : line0;  // a valid line for the index arithmetic
  const int j = (int)(lc % p.ninner);
  const long long l12 = lc / p.ninner;
  const int o1 = (int)(l12 % p.n1), o2 = (int)(l12 / p.n1);
  const float2 *src = reinterpret_cast<const float2 *>(p.in) + (long long)o1 * p.in_s1 + (long long)o2 * p.in_s2 + j;
  float2 *dst = reinterpret_cast<float2 *>(p.out) + (long long)o1 * p.out_s1 + (long long)o2 * p.out_s2 + j;
  const float2 *tw = A.tw.w;
  float2 w[S::U][P];
  lane_twiddles<M, P>(w, tw_full, s);
  float2 y[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int m = s + P * q;
    float2 x = (act && m < p.nin) ? src[(long long)m * p.in_sm] : make_float2(0.f, 0.f);
    if (p.inverse) x.y = -x.y;
    y[q] = x;
  }
  float2 *buf = xbuf[warp];
  lane_stage1<M, P>(y, tw);
  lane_put<M, P>(buf, y, lane);
  __syncwarp();
  lane_stage2<M, P>(y, buf, s, l, w, tw);
  const float inv_m = 1.0f / (float)M;
  if (p.inverse) {
#pragma unroll
    for (int q = 0; q < Q; ++q) y[q] = make_float2(y[q].x * inv_m, -y[q].y * inv_m);
    if (p.refft_keep > 0) {
#pragma unroll
      for (int q = 0; q < Q; ++q)
        if (s + P * q >= p.refft_keep) y[q] = make_float2(0.f, 0.f);
      __syncwarp();  // every lane has read the buffer before it is rewritten
      lane_stage1<M, P>(y, tw);
      lane_put<M, P>(buf, y, lane);
      __syncwarp();
      lane_stage2<M, P>(y, buf, s, l, w, tw);
    }
  }
  if (!act) return;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int k = s + P * q;
    if (k < p.nout) dst[(long long)k * p.out_sm] = y[q];
  }
}

RegArgs reg_args(const AxisPass &p, const FftTables &t, int M) {
  RegArgs a;
  a.p = p;
  for (int i = 0; i < kRegMaxM; ++i) a.tw.w[i] = make_float2(0.f, 0.f);
  // twiddles in host memory: copied from the host mirror kept with the plan
  for (int i = 0; i < M; ++i) a.tw.w[i] = t.tw32_host[i];
  return a;
}

template <int M, int P>
void launch_lanes(const AxisPass &p, const FftTables &t, cudaStream_t st) {
  const RegArgs a = reg_args(p, t, M);
  const long long nlines = (long long)p.n1 * p.n2 * p.ninner;
  const long long warps = (nlines + LaneShape<M, P>::L - 1) / LaneShape<M, P>::L;
  const long long blocks = (warps + kLaneThreads / 32 - 1) / (kLaneThreads / 32);
  axis_lane_kernel<M, P><<<(unsigned)blocks, kLaneThreads, 0, st>>>(a, t.tw32);
}

template <int M>
void launch_m(const AxisPass &p, const FftTables &t, cudaStream_t st) {
  const int P = lanes_per_line(p, M);
  if constexpr (M % 4 == 0) {
    if (P == 2) return launch_lanes<M, 2>(p, t, st);
  }
  if constexpr (M % 16 == 0) {
    if (P == 4) return launch_lanes<M, 4>(p, t, st);
  }
  if constexpr (M % 64 == 0) {
    if (P == 8) return launch_lanes<M, 8>(p, t, st);
  }
  const RegArgs a = reg_args(p, t, M);
  const long long nlines = (long long)p.n1 * p.n2 * p.ninner;
  const int threads = 128;
  const long long blocks = (nlines + threads - 1) / threads;
  axis_reg_kernel<M><<<(unsigned)blocks, threads, 0, st>>>(a);
}

}  // namespace

bool axis_lanes_valid(int M, int P) {
  if (P == 1) return true;
  if (P != 2 && P != 4 && P != 8) return false;
  if (M % (P * P) != 0) return false;
  switch (M / P) {  // the lane's own transform length
    case 1: case 2: case 3: case 4: case 5: case 6: case 8: case 9: case 10: case 12: case 15: case 16:
    case 18: case 20: case 24: case 25: case 27: case 30: case 32:
      return true;
    default:
      return false;
  }
}

// Lanes per line, a fixed function of the pass geometry so that a result
// never depends on timing: lanes are added (2, then 4, where valid) while
// the pass has fewer than 64 K lanes (2 K warps, about four per SM
// sub-partition on 148 SMs).  Measured on the 32 x 32, b = 128, 2-RHS
// operator (8 K and 16 K lines per pass): Z x took 86.0 / 79.2 / 76.9 /
// 82.7 us with 1 / 2 / 4 / 8 lanes everywhere, so 8 lanes are never
// chosen.  MOMA_FFT_LANES=P in the environment (read once) imposes P where
// valid: for timing comparisons, it changes rounding.
int lanes_per_line(const AxisPass &p, int M) {
  static const int forced = [] {
    const char *e = std::getenv("MOMA_FFT_LANES");
    return e ? std::atoi(e) : 0;
  }();
  if (forced > 0) return axis_lanes_valid(M, forced) ? forced : 1;
  const long long nlines = (long long)p.n1 * p.n2 * p.ninner;
  int P = 1;
  for (int c : {2, 4})
    if (nlines * P < 64 * 1024 && axis_lanes_valid(M, c)) P = c;
  return P;
}

bool axis_reg_supported(const AxisPass &p, int M) {
  if (M > kRegMaxM || M < 1) return false;
  if (p.in_mode != 0 || p.out_mode != 0 || p.in_c128 != 0 || p.out_c128 != 0 || p.out2 != nullptr) return false;
  if (p.inner_in_map || p.slot_of || p.bin_slot) return false;
  if (p.refft_keep > 0 && !p.inverse) return false;
  switch (M) {
    case 1: case 2: case 3: case 4: case 5: case 6: case 8: case 9: case 10: case 12: case 15: case 16:
    case 18: case 20: case 24: case 25: case 27: case 30: case 32: case 36: case 40: case 45: case 48:
    case 50: case 54: case 60: case 64:
      return true;
    default:
      return false;
  }
}

void launch_axis_reg(const AxisPass &p, const FftTables &t, cudaStream_t st) {
  if (p.ninner <= 0 || p.n1 * p.n2 <= 0) return;
  switch (t.plan.M) {
    case 1: launch_m<1>(p, t, st); break;
    case 2: launch_m<2>(p, t, st); break;
    case 3: launch_m<3>(p, t, st); break;
    case 4: launch_m<4>(p, t, st); break;
    case 5: launch_m<5>(p, t, st); break;
    case 6: launch_m<6>(p, t, st); break;
    case 8: launch_m<8>(p, t, st); break;
    case 9: launch_m<9>(p, t, st); break;
    case 10: launch_m<10>(p, t, st); break;
    case 12: launch_m<12>(p, t, st); break;
    case 15: launch_m<15>(p, t, st); break;
    case 16: launch_m<16>(p, t, st); break;
    case 18: launch_m<18>(p, t, st); break;
    case 20: launch_m<20>(p, t, st); break;
    case 24: launch_m<24>(p, t, st); break;
    case 25: launch_m<25>(p, t, st); break;
    case 27: launch_m<27>(p, t, st); break;
    case 30: launch_m<30>(p, t, st); break;
    case 32: launch_m<32>(p, t, st); break;
    case 36: launch_m<36>(p, t, st); break;
    case 40: launch_m<40>(p, t, st); break;
    case 45: launch_m<45>(p, t, st); break;
    case 48: launch_m<48>(p, t, st); break;
    case 50: launch_m<50>(p, t, st); break;
    case 54: launch_m<54>(p, t, st); break;
    case 60: launch_m<60>(p, t, st); break;
    case 64: launch_m<64>(p, t, st); break;
    default: throw std::runtime_error("register FFT: unsupported length");
  }
}

}  // namespace moma
