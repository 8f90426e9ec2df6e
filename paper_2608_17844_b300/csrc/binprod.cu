// Per-bin product of the MLFFT matvec, Eq. 3: after the lattice FFT the
// circulant embedding of Z is block diagonal, so y_k = Zhat_k x_k for every
// circulant frequency k.
//
// Storage keeps one b x b block per pair {k, -k}: reciprocity (Z = Z^T,
// Sec. II-D) gives Zhat_{-k} = Zhat_k^T, so one stream of the stored block
// serves both members of the pair:
//   normal  (Z):   y_ka = Zhat x_ka,             y_kb = Zhat^T x_kb
//   adjoint (Z^H): y_kb = conj(Zhat) x_kb,       y_ka = conj(Zhat)^T x_ka
// The adjoint uses the same stored bins, conjugated at multiplication time
// (Eq. 6, Hermitian commutation).  Self-paired bins (k = -k) are symmetric
// and need only the row product.
//
// At small nrhs this is a streaming GEMV, bound by HBM: every stored block
// is read once per product.  The kernel is persistent and warp-specialised:
//  * a producer warp streams row tiles of the stored blocks into an
//    NS-deep ring of shared-memory stages with 1D bulk copies
//    (cp.async.bulk), each completing on the stage's "full" mbarrier, and
//    refills a stage once the eight consumer warps have arrived on its
//    "empty" mbarrier;
//  * eight consumer warps own groups of four rows of a tile, lanes own pairs of
//    adjacent columns (eight, so that the 32 groups of a b = 128 block, or
//    the 64 of b = 256, split evenly and no warp idles at the end of a pair).  Row products of a row group are reduced across the
//    warp by recursive halving (one shuffle tree for all 4 rows x nrhs
//    values); column products accumulate in registers over the whole block
//    and are reduced across warps once per pair;
//  * the input vectors of the next pair are prefetched into a second
//    buffer with asynchronous copies (cp.async) while the current pair
//    streams.
// All waits are bounded; a timeout sets DEVERR_TIMEOUT and the CTA drains
// its copies and exits.
#include <algorithm>
#include <type_traits>

#include "internal.h"

namespace moma {

constexpr int BP_CONSUMERS = 8;
constexpr int BP_THREADS = (BP_CONSUMERS + 1) * 32;
constexpr int BP_ROWS = 4;  // rows per warp group
constexpr uint64_t BP_WAIT_NS = 2000000000ull;

struct BinKernelArgs {
  BinProduct P;
  int TR, ntile, NS, q0;
};

MOMA_DEV void consumer_bar() { asm volatile("bar.sync 1, %0;" ::"n"(BP_CONSUMERS * 32) : "memory"); }
template <int BYTES>
MOMA_DEV void cp_async(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES) : "memory");
}
MOMA_DEV void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
MOMA_DEV void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Sum of v[0..NV) over the 32 lanes by recursive halving.  On return v[0]
// of lane l holds the total of value halving_index<NV>(l); lanes with
// (l % (32 / NV)) == 0 are the unique owners.
template <typename T, int NV>
MOMA_DEV void halving_reduce(T (&v)[NV], int lane) {
  int n = NV;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    if (n > 1) {
      const int h = n >> 1;
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < NV / 2; ++i) {
        if (i < h) {
          const T send = up ? v[i] : v[i + h];
          const T keep = up ? v[i + h] : v[i];
          v[i] = keep + shfl_xor(send, o);
        }
      }
      n = h;
    } else {
      v[0] += shfl_xor(v[0], o);
    }
  }
}
template <int NV>
MOMA_DEV int halving_index(int lane) {
  int idx = 0, n = NV;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    if (n > 1) {
      n >>= 1;
      if (lane & o) idx += n;
    }
  }
  return idx;
}

// Two adjacent complex entries (16-byte aligned in c64: c and ldb are even).
MOMA_DEV void load_pair(const float2 *p, float2 (&z)[2]) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  z[0] = make_float2(v.x, v.y);
  z[1] = make_float2(v.z, v.w);
}
MOMA_DEV void load_pair(const dfl2 *p, dfl2 (&z)[2]) {
  z[0] = p[0];
  z[1] = p[1];
}
MOMA_DEV void load_pair(const double2 *p, double2 (&z)[2]) {
  z[0] = p[0];
  z[1] = p[1];
}

// MINB = CTAs per SM the register budget is sized for (1: 168 registers a
// thread, 2: 102, 3: 72; more CTAs keep more warps in flight to hide
// shared-memory and FMA latency, with smaller tiles).
template <typename R, int NR, int U2, bool HERM, int MINB>
__global__ void __launch_bounds__(BP_THREADS, MINB) bin_pair_kernel(BinKernelArgs A) {
  using C = typename Cplx<R>::T;
  extern __shared__ __align__(128) unsigned char sm[];
  const BinProduct &P = A.P;
  if (P.live && *P.live == 0) return;
  const int b = P.b, ldb = P.ldb, nr = P.nr, q0 = A.q0;
  const int TR = A.TR, ntile = A.ntile, NS = A.NS;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;

  uint64_t *full = reinterpret_cast<uint64_t *>(sm);
  uint64_t *empty = full + NS;
  volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + NS);
  C *stage0 = reinterpret_cast<C *>(sm + 256);
  const size_t stage_elems = (size_t)TR * ldb;
  C *xbuf = stage0 + NS * stage_elems;  // [2 buffers][R|C][NR][b]
  C *red = xbuf + (size_t)4 * NR * b;   // [BP_CONSUMERS][b][NR]

  const C *Z = reinterpret_cast<const C *>(P.Z);
  const C *X = reinterpret_cast<const C *>(P.x);
  C *Y = reinterpret_cast<C *>(P.y);

  const int npair = (P.Bp - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int total = npair * ntile;
  if (total <= 0) return;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], BP_CONSUMERS);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (w == BP_CONSUMERS) {
    // ---------------------------------------------------------- producer --
    if (lane != 0) return;
    int issued = 0;
    for (int i = 0; i < total; ++i) {
      const int s = i % NS;
      const uint32_t par = (uint32_t)(((i / NS) & 1) ^ 1);
      bool ok = mbar_try_wait(&empty[s], par);
      if (!ok) {
        const uint64_t t0 = global_ns();
        for (uint32_t it = 0; !ok; ++it) {
          ok = mbar_try_wait(&empty[s], par);
          if (!ok && (it & 255u) == 255u && (*abort_flag || global_ns() - t0 > BP_WAIT_NS)) break;
        }
      }
      if (!ok) {
        if (!*abort_flag) atomicOr(P.err, DEVERR_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      const int pk = i / ntile, t = i % ntile;
      const long long p = (long long)blockIdx.x + (long long)pk * gridDim.x;
      const int r0 = t * TR;
      const int rows = min(TR, b - r0);
      const uint32_t bytes = (uint32_t)(rows * ldb * sizeof(C));
      fence_proxy_async();
      mbar_expect_tx(&full[s], bytes);
      bulk_g2s(stage0 + (size_t)s * stage_elems, Z + ((size_t)p * b + r0) * ldb, bytes, &full[s]);
      issued = i + 1;
    }
    // Drain: every issued copy must land before the CTA can retire.
    for (int i = max(0, issued - NS); i < issued; ++i)
      mbar_wait_bounded(&full[i % NS], (uint32_t)((i / NS) & 1), BP_WAIT_NS);
    return;
  }

  // ------------------------------------------------------------ consumers --
  auto load_x = [&](int pk, int buf) {
    const int p = (int)blockIdx.x + pk * (int)gridDim.x;
    const int2 pr = P.pairs[p];
    const int kR = HERM ? pr.y : pr.x, kC = HERM ? pr.x : pr.y;
    C *xr_s = xbuf + (size_t)buf * 2 * NR * b;
    C *xc_s = xr_s + (size_t)NR * b;
    for (int idx = tid; idx < NR * b; idx += BP_CONSUMERS * 32) {
      const int qq = idx / b, c = idx % b, q = q0 + qq;
      if (q < nr) cp_async<sizeof(C)>(&xr_s[idx], &X[((size_t)kR * nr + q) * b + c]);
      else xr_s[idx] = czero<C>();
      if (q < nr && pr.x != pr.y) cp_async<sizeof(C)>(&xc_s[idx], &X[((size_t)kC * nr + q) * b + c]);
      else xc_s[idx] = czero<C>();
    }
  };
  load_x(0, 0);
  cp_async_wait_all();
  consumer_bar();

  C xr[U2][2][NR];
  C accC[U2][2][NR];
  int kR = 0, kC = 0;
  bool selfp = false;
  const C *xc_s = xbuf;

  for (int i = 0; i < total; ++i) {
    const int pk = i / ntile, t = i % ntile, buf = pk & 1;
    if (t == 0) {
      const int p = (int)blockIdx.x + pk * (int)gridDim.x;
      const int2 pr = P.pairs[p];
      selfp = pr.x == pr.y;
      kR = HERM ? pr.y : pr.x;
      kC = HERM ? pr.x : pr.y;
      const C *xr_s = xbuf + (size_t)buf * 2 * NR * b;
      xc_s = xr_s + (size_t)NR * b;
#pragma unroll
      for (int u = 0; u < U2; ++u)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = 2 * lane + 64 * u + h;
#pragma unroll
          for (int qq = 0; qq < NR; ++qq) {
            xr[u][h][qq] = c < b ? xr_s[qq * b + c] : czero<C>();
            accC[u][h][qq] = czero<C>();
          }
        }
      if (pk + 1 < npair) load_x(pk + 1, buf ^ 1);  // overlaps this pair's tiles
    }

    // Wait for the tile.  After a timeout (here or in the producer) the
    // consumers keep walking the loop without touching data, so that every
    // named barrier below is still reached by all of them.
    const int s = i % NS;
    bool ok = false;
    if (!*abort_flag) {
      const uint32_t par = (uint32_t)((i / NS) & 1);
      ok = mbar_try_wait(&full[s], par);
      if (!ok) {
        const uint64_t t0 = global_ns();
        for (uint32_t it = 0; !ok; ++it) {
          ok = mbar_try_wait(&full[s], par);
          if (!ok && (it & 255u) == 255u && (*abort_flag || global_ns() - t0 > BP_WAIT_NS)) break;
        }
        if (!ok && !*abort_flag) {
          atomicOr(P.err, DEVERR_TIMEOUT);
          *abort_flag = 1;
        }
      }
    }
    const C *tile = stage0 + (size_t)s * stage_elems;
    const int r0 = t * TR, rows = ok ? min(TR, b - r0) : 0;
    constexpr int NV = BP_ROWS * NR * 2;
    // Row group j (rows 4j .. 4j+3 of the block) belongs to warp j mod 8
    // whatever the tile height, so every warp accumulates the same rows in
    // the same order for any tuned shape: results are bitwise independent
    // of TR, NS and CTAs per SM (tiles start on multiples of 4 rows).
    const int gfirst = ((w - r0 / BP_ROWS) % BP_CONSUMERS + BP_CONSUMERS) % BP_CONSUMERS;
    for (int g = gfirst * BP_ROWS; g < rows; g += BP_CONSUMERS * BP_ROWS) {
      R part[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) part[v] = (R)0;
#pragma unroll
      for (int rr = 0; rr < BP_ROWS; ++rr) {
        const int rl = g + rr;
        if (rl < rows) {
          const int r = r0 + rl;
          const C *zrow = tile + (size_t)rl * ldb;
          C xc[NR];
#pragma unroll
          for (int qq = 0; qq < NR; ++qq) xc[qq] = xc_s[qq * b + r];
#pragma unroll
          for (int u = 0; u < U2; ++u) {
            const int c = 2 * lane + 64 * u;
            if (c < b) {
              C z[2];
              load_pair(zrow + c, z);  // c + 1 < ldb; a padding column is zero
              if (HERM) {
                z[0] = cconj(z[0]);
                z[1] = cconj(z[1]);
              }
#pragma unroll
              for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int qq = 0; qq < NR; ++qq) {
                  C pr = mk(part[(rr * NR + qq) * 2], part[(rr * NR + qq) * 2 + 1]);
                  pr = cfma(z[h], xr[u][h][qq], pr);
                  part[(rr * NR + qq) * 2] = pr.x;
                  part[(rr * NR + qq) * 2 + 1] = pr.y;
                  accC[u][h][qq] = cfma(z[h], xc[qq], accC[u][h][qq]);
                }
            }
          }
        }
      }
      halving_reduce<R, NV>(part, lane);
      if ((lane % (32 / NV)) == 0) {
        const int idx = halving_index<NV>(lane);
        const int rr = idx / (NR * 2), qq = (idx / 2) % NR, comp = idx & 1;
        const int rl = g + rr;
        if (rl < rows && q0 + qq < nr) {
          R *dst = reinterpret_cast<R *>(&Y[((size_t)kR * nr + q0 + qq) * b + r0 + rl]);
          dst[comp] = part[0];
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);

    if (t == ntile - 1) {
      if (!selfp) {
#pragma unroll
        for (int u = 0; u < U2; ++u)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c = 2 * lane + 64 * u + h;
            if (c < b)
#pragma unroll
              for (int qq = 0; qq < NR; ++qq) red[((size_t)w * b + c) * NR + qq] = accC[u][h][qq];
          }
      }
      cp_async_wait_all();  // this thread's prefetch of the next pair's x has landed
      consumer_bar();  // red complete; also orders the x prefetch before its use
      if (!selfp) {
        for (int idx = tid; idx < b * NR; idx += BP_CONSUMERS * 32) {
          C v = czero<C>();
#pragma unroll
          for (int ww = 0; ww < BP_CONSUMERS; ++ww) v = cadd(v, red[(size_t)ww * b * NR + idx]);
          const int c = idx / NR, qq = idx % NR;
          if (q0 + qq < nr) Y[((size_t)kC * nr + q0 + qq) * b + c] = v;
        }
      }
      consumer_bar();  // red may be rewritten by the next pair
    }
  }
}

template <typename R, int NR, int U2, bool HERM>
static void launch_one(const BinProduct &P, int num_sms, cudaStream_t st, int q0) {
  using C = typename Cplx<R>::T;
  const int row_bytes = P.ldb * (int)sizeof(C);
  auto smem_for = [&](int ns, int tr) {
    return 256 + (size_t)ns * tr * row_bytes + (size_t)4 * NR * P.b * sizeof(C) +
           (size_t)BP_CONSUMERS * P.b * NR * sizeof(C);
  };
  // Two or three CTAs per SM (smaller tiles, 102- or 72-register budget)
  // only where the per-lane state is small: at most two RHS per chunk and
  // b <= 128; three only for c64.
  constexpr bool occ2_ok = NR <= 2 && U2 <= 2;
  constexpr bool occ3_ok = sizeof(R) == 4 && NR <= 2 && U2 <= 2;
  const int occ = (P.occ == 3 && occ3_ok) ? 3 : (P.occ == 2 && occ2_ok) ? 2 : 1;
  const size_t cap = occ == 3 ? 74 * 1024 : occ == 2 ? 110 * 1024 : 220 * 1024;
  // Tiles of whole rows, at most 48 KB and at most one 4-row group per
  // consumer warp; 3 stages (fewer if shared memory runs out).
  int TR = 49152 / row_bytes;
  if (TR > 4 * BP_CONSUMERS) TR = 4 * BP_CONSUMERS;
  if (TR >= 4) TR &= ~3;
  if (TR < 1) TR = 1;
  if (TR > P.b) TR = P.b;
  int NS = 3;
  // Autotuned shape, if it is valid for this launch.
  if (P.TR > 0 && P.TR <= 4 * BP_CONSUMERS && P.TR % 4 == 0 && P.NS >= 2 && P.NS <= 6) {
    const int tr = std::min(P.TR, P.b);
    if (smem_for(P.NS, tr) <= cap) {
      TR = tr;
      NS = P.NS;
    }
  }
  while (NS > 2 && smem_for(NS, TR) > cap) --NS;
  while (TR > 4 && smem_for(NS, TR) > cap) TR -= 4;  // wide blocks (b > 160) or several CTAs per SM
  const int ntile = (P.b + TR - 1) / TR;
  const size_t smem = smem_for(NS, TR);
  int grid = num_sms * occ;
  if (grid > P.Bp) grid = P.Bp;
  BinKernelArgs a{P, TR, ntile, NS, q0};
  if constexpr (occ3_ok) {
    if (occ == 3) {
      auto kern = bin_pair_kernel<R, NR, U2, HERM, 3>;
      static int configured3 = 0;
      if (!configured3) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 74 * 1024);
        configured3 = 1;
      }
      kern<<<grid, BP_THREADS, smem, st>>>(a);
      return;
    }
  }
  if constexpr (occ2_ok) {
    if (occ == 2) {
      auto kern = bin_pair_kernel<R, NR, U2, HERM, 2>;
      static int configured2 = 0;
      if (!configured2) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024);
        configured2 = 1;
      }
      kern<<<grid, BP_THREADS, smem, st>>>(a);
      return;
    }
  }
  auto kern = bin_pair_kernel<R, NR, U2, HERM, 1>;
  static int configured = 0;
  if (!configured) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    configured = 1;
  }
  kern<<<grid, BP_THREADS, smem, st>>>(a);
}

template <typename R, int NR, bool HERM>
static void launch_u(const BinProduct &P, int num_sms, cudaStream_t st, int q0) {
  const int U2 = (P.b + 63) / 64;
  if (U2 <= 1) launch_one<R, NR, 1, HERM>(P, num_sms, st, q0);
  else if (U2 <= 2) launch_one<R, NR, 2, HERM>(P, num_sms, st, q0);
  else launch_one<R, NR, 4, HERM>(P, num_sms, st, q0);
}

template <typename R, int NR>
static void launch_nr(const BinProduct &P, int num_sms, cudaStream_t st, int q0) {
  if (P.herm) launch_u<R, NR, true>(P, num_sms, st, q0);
  else launch_u<R, NR, false>(P, num_sms, st, q0);
}

template <typename R>
void launch_bin_product(const BinProduct &P, int num_sms, cudaStream_t st) {
  if constexpr (std::is_same<R, float>::value) {
    if (bin_rc_supported(P.b) && P.ldb == P.b) {
      launch_bin_rc(P, num_sms, st);
      return;
    }
  }
  if constexpr (std::is_same<R, dfl>::value) {
    if (bin_rc_dfl_supported(P.b) && P.ldb == P.b) {
      launch_bin_rc_dfl(P, num_sms, st);
      return;
    }
  }
  // RHS are processed in chunks of up to NRMAX columns (the kernel masks
  // columns past nr); each chunk streams the bins once.
  constexpr int NRMAX = sizeof(R) == 4 ? 4 : 2;
  // Double-FP32 accumulators of wide blocks (b > 128) take one RHS per
  // chunk so that they stay in registers.
  const int nrmax = (std::is_same<R, dfl>::value && P.b > 128) ? 1 : NRMAX;
  for (int q0 = 0; q0 < P.nr; q0 += nrmax) {
    const int left = P.nr - q0;
    if (left == 1 || nrmax == 1) launch_nr<R, 1>(P, num_sms, st, q0);
    else if (left == 2) launch_nr<R, 2>(P, num_sms, st, q0);
    else launch_nr<R, NRMAX>(P, num_sms, st, q0);
  }
}

template void launch_bin_product<float>(const BinProduct &, int, cudaStream_t);
template void launch_bin_product<double>(const BinProduct &, int, cudaStream_t);
template void launch_bin_product<dfl>(const BinProduct &, int, cudaStream_t);

}  // namespace moma
