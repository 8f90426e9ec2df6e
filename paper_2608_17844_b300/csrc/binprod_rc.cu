// The per-bin product of Eq. 3 for b a multiple of 32 (64 <= b <= 256), in
// c64 for the inner solve and in double-FP32 (two RHS per launch; 16-row
// tiles above b = 160) for the refinement residual:
// y_ka = Zhat x_ka and y_kb = Zhat^T x_kb from one stored block per pair
// {k, -k} (reciprocity, Sec. II-D), or conj(Zhat) and conj(Zhat)^T for Z^H
// (Eq. 6), as in binprod.cu, with a different split of the work that needs
// no cross-lane reduction trees.
//
// A tile is 32 rows of the stored block.  The producer copies each row with
// its own bulk copy into a stage whose rows are b + 2 complex values apart,
// so that 16-byte loads are free of bank conflicts both along a row and down
// a column.  The eight consumer warps read every tile twice, once per leg:
//  * row warps 0..3 own rows 8w .. 8w+7 of the tile; lane (r, c) = (lane % 8,
//    lane / 8) takes the column pairs 8i + 2c, i = 0 .. b/8 - 1, of row r, so
//    the row leg sum_j Zhat_rj x_R,j is finished by adding the four lanes of
//    the row (two shuffles) and stored once per tile;
//  * column warps 4..7 own column pairs (lane = pair) and a slice of the
//    tile's rows, and accumulate the column leg sum_i Zhat_ij x_C,i in
//    registers over the whole block; the slices are added in a fixed order
//    once per pair.
// Every sum has a fixed order (tile height fixed at 32 rows), so results do
// not depend on the pipeline depth or CTAs per SM that the autotuner picks.
// Waits are bounded like those of binprod.cu; a timeout sets DEVERR_TIMEOUT,
// the CTA drains its copies and exits.
#include <algorithm>

#include "internal.h"

namespace moma {

namespace {

constexpr int RC_TR = 32;
constexpr int RC_CONS = 8;
constexpr int RC_THREADS = (RC_CONS + 1) * 32;
constexpr uint64_t RC_WAIT_NS = 2000000000ull;

struct RcArgs {
  BinProduct P;
  int NS, q0, lds;
};

MOMA_DEV void rc_consumer_bar() { asm volatile("bar.sync 1, %0;" ::"n"(RC_CONS * 32) : "memory"); }
MOMA_DEV void rc_cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
MOMA_DEV void rc_cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
MOMA_DEV void rc_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
MOMA_DEV float2 rc_sum4(float2 v) {  // the four lanes of a row (lane bits 3 and 4)
  v.x += __shfl_xor_sync(0xffffffffu, v.x, 8);
  v.y += __shfl_xor_sync(0xffffffffu, v.y, 8);
  v.x += __shfl_xor_sync(0xffffffffu, v.x, 16);
  v.y += __shfl_xor_sync(0xffffffffu, v.y, 16);
  return v;
}
MOMA_DEV void rc_cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// Arithmetic of the kernel: c64 (E = float2, FP32 accumulators) for the
// inner solve, and double-FP32 (E = dfl2, unnormalised two-float
// accumulators whose additions are exact two-sums) for the refinement
// residual of the mixed path.
struct RcF32 {
  using E = float2;
  struct Acc {
    float2 v;
  };
  MOMA_DEV static Acc zero() { return Acc{make_float2(0.f, 0.f)}; }
  MOMA_DEV static E ezero() { return make_float2(0.f, 0.f); }
  MOMA_DEV static void load2(const E *row, int c, E &z0, E &z1) {  // entries c, c + 1 (one 16-byte load)
    const float4 z4 = *reinterpret_cast<const float4 *>(row + c);
    z0 = make_float2(z4.x, z4.y);
    z1 = make_float2(z4.z, z4.w);
  }
  MOMA_DEV static E conj(E z) { return make_float2(z.x, -z.y); }
  MOMA_DEV static void fma(Acc &a, E z, E x) { a.v = cfma(z, x, a.v); }
  template <int RPW>
  MOMA_DEV static Acc sum_row(Acc a) {  // the lanes of a row: lane bits log2(RPW) .. 4
    static_assert(RPW == 8, "c64 tiles have 32 rows");
    return Acc{rc_sum4(a.v)};
  }
  MOMA_DEV static E value(const Acc &a) { return a.v; }
  MOMA_DEV static void add(Acc &a, const E &u) {
    a.v.x += u.x;
    a.v.y += u.y;
  }
  MOMA_DEV static void copy_async(E *dst, const E *src) { rc_cp_async8(dst, src); }
};
struct RcDfl {
  using E = dfl2;
  struct Acc {
    DfAcc re, im;
  };
  MOMA_DEV static Acc zero() { return Acc{DfAcc{0.f, 0.f}, DfAcc{0.f, 0.f}}; }
  MOMA_DEV static E ezero() { return dfl2{dfl(0.f), dfl(0.f)}; }
  MOMA_DEV static void load2(const E *row, int c, E &z0, E &z1) {
    z0 = row[c];
    z1 = row[c + 1];
  }
  MOMA_DEV static E conj(E z) { return dfl2{z.x, -z.y}; }
  MOMA_DEV static void fma(Acc &a, E z, E x) {  // a += z x
    dfacc_fma(a.re, z.x, x.x);
    dfacc_fma(a.re, -z.y, x.y);
    dfacc_fma(a.im, z.x, x.y);
    dfacc_fma(a.im, z.y, x.x);
  }
  MOMA_DEV static DfAcc shfl_add(DfAcc a, int m) {
    DfAcc o{__shfl_xor_sync(0xffffffffu, a.s, m), __shfl_xor_sync(0xffffffffu, a.t, m)};
    dfacc_add(a, o);
    return a;
  }
  template <int RPW>
  MOMA_DEV static Acc sum_row(Acc a) {  // the lanes of a row: lane bits log2(RPW) .. 4
#pragma unroll
    for (int m = RPW; m < 32; m <<= 1) {
      a.re = shfl_add(a.re, m);
      a.im = shfl_add(a.im, m);
    }
    return a;
  }
  MOMA_DEV static E value(const Acc &a) { return dfl2{dfacc_value(a.re), dfacc_value(a.im)}; }
  MOMA_DEV static void add(Acc &a, const E &u) {
    dfacc_add(a.re, DfAcc{u.x.hi, u.x.lo});
    dfacc_add(a.im, DfAcc{u.y.hi, u.y.lo});
  }
  MOMA_DEV static void copy_async(E *dst, const E *src) { rc_cp_async16(dst, src); }
};

template <typename AR, int NR, bool HERM, int MINB, int TR, int BB>
__global__ void __launch_bounds__(RC_THREADS, MINB) bin_rc_kernel(RcArgs A) {
  using E = typename AR::E;
  using Acc = typename AR::Acc;
  // TR rows per tile: 32, or 16 for double-FP32 blocks wider than 160 (whose
  // 32-row stages would not fit twice).  A row warp owns RPW = TR / 4 rows
  // with 32 / RPW lanes on each.
  constexpr int RPW = TR / 4, LPR = 32 / RPW;
  extern __shared__ __align__(128) unsigned char sm[];
  const BinProduct &P = A.P;
  if (P.live && *P.live == 0) return;
  // BB > 0: the block order as a compile-time constant (loops unrolled,
  // strides folded); the row/column kernels run with ldb = b.
  const int b = BB > 0 ? BB : P.b, ldb = BB > 0 ? BB : P.ldb, lds = BB > 0 ? BB + 2 : A.lds;
  const int nr = P.nr, q0 = A.q0, NS = A.NS;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  uint64_t *full = reinterpret_cast<uint64_t *>(sm);
  uint64_t *empty = full + NS;
  volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + NS);
  uint64_t *red_free = empty + NS + 1;  // redC read out by the slice-0 column warps
  E *stage0 = reinterpret_cast<E *>(sm + 256);
  const size_t stage_elems = (size_t)TR * lds;
  E *xbuf = stage0 + NS * stage_elems;      // [2 buffers][R | C][NR][b]
  E *redC = xbuf + (size_t)4 * NR * b;      // [4 column warps][32 lanes][2][NR]
  const E *Z = reinterpret_cast<const E *>(P.Z);
  const E *X = reinterpret_cast<const E *>(P.x);
  E *Y = reinterpret_cast<E *>(P.y);
  const int ntile = b / TR;
  const int npair = (P.Bp - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int total = npair * ntile;
  if (total <= 0) return;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], RC_CONS);
    }
    mbar_init(red_free, (b / 2 + 31) / 32);  // one arrival per slice-0 column warp
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (w == RC_CONS) {
    // ------------------------------------------------------------ producer --
    if (lane != 0) return;
    int issued = 0;
    const uint32_t row_bytes = (uint32_t)(ldb * sizeof(E));
    int s = 0, t = 0;  // stage, tile of the pair (counters: no division per tile)
    uint32_t ph = 0;   // ring pass parity
    long long p = blockIdx.x;
    for (int i = 0; i < total; ++i) {
      const uint32_t par = ph ^ 1u;
      bool ok = mbar_try_wait(&empty[s], par);
      if (!ok) {
        const uint64_t t0 = global_ns();
        for (uint32_t it = 0; !ok; ++it) {
          ok = mbar_try_wait(&empty[s], par);
          if (!ok && (it & 255u) == 255u && (*abort_flag || global_ns() - t0 > RC_WAIT_NS)) break;
        }
      }
      if (!ok) {
        if (!*abort_flag) atomicOr(P.err, DEVERR_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      const E *src = Z + ((size_t)p * b + (size_t)t * TR) * ldb;
      E *dst = stage0 + (size_t)s * stage_elems;
      fence_proxy_async();
      mbar_expect_tx(&full[s], row_bytes * TR);
      for (int rr = 0; rr < TR; ++rr) bulk_g2s(dst + (size_t)rr * lds, src + (size_t)rr * ldb, row_bytes, &full[s]);
      issued = i + 1;
      if (++t == ntile) {
        t = 0;
        p += gridDim.x;
      }
      if (++s == NS) {
        s = 0;
        ph ^= 1u;
      }
    }
    for (int i = max(0, issued - NS); i < issued; ++i)
      mbar_wait_bounded(&full[i % NS], (uint32_t)((i / NS) & 1), RC_WAIT_NS);
    return;
  }

  // ------------------------------------------------------------ consumers --
  auto load_x = [&](int pk, int buf) {
    const int p = (int)blockIdx.x + pk * (int)gridDim.x;
    const int2 pr = P.pairs[p];
    const int kR = HERM ? pr.y : pr.x, kC = HERM ? pr.x : pr.y;
    E *xr_s = xbuf + (size_t)buf * 2 * NR * b;
    E *xc_s = xr_s + (size_t)NR * b;
    for (int idx = tid; idx < NR * b; idx += RC_CONS * 32) {
      const int qq = idx / b, c = idx % b, q = q0 + qq;
      if (q < nr) AR::copy_async(&xr_s[idx], &X[((size_t)kR * nr + q) * b + c]);
      else xr_s[idx] = AR::ezero();
      if (q < nr && pr.x != pr.y) AR::copy_async(&xc_s[idx], &X[((size_t)kC * nr + q) * b + c]);
      else xc_s[idx] = AR::ezero();
    }
  };
  // Launched as a programmatic dependent of the kernel that writes the bin
  // vectors: the producer streams the pair store from the start, the
  // consumers read x only once that kernel has completed.  (A plain launch
  // passes this wait at once.)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  load_x(0, 0);
  rc_cp_async_wait_all();
  rc_consumer_bar();

  // Column warps: G groups of 32 column pairs, 4 / G row slices per tile.
  const int G = (b / 2 + 31) / 32, nslice = 4 / G, rps = TR / nslice;
  const int kw = w - 4, cgrp = kw % G, slice = kw / G;
  const bool col_active = w >= 4 && kw < G * nslice;
  const int cpair = 32 * cgrp + lane, cc = 2 * cpair;
  const int r8 = lane % RPW, c4 = lane / RPW;  // row in the warp's rows, lane of the row

  Acc accC[2][NR];
  int kR = 0, kC = 0;
  bool selfp = false;
  const E *xr_s = xbuf, *xc_s = xbuf + (size_t)NR * b;

  int s = 0, t = 0, pk = 0;  // stage, tile of the pair, pair (counters: no division per tile)
  uint32_t ph = 0;           // ring pass parity
  for (int i = 0; i < total; ++i) {
    const int buf = pk & 1;
    if (t == 0) {
      const int p = (int)blockIdx.x + pk * (int)gridDim.x;
      const int2 pr = P.pairs[p];
      selfp = pr.x == pr.y;
      kR = HERM ? pr.y : pr.x;
      kC = HERM ? pr.x : pr.y;
      xr_s = xbuf + (size_t)buf * 2 * NR * b;
      xc_s = xr_s + (size_t)NR * b;
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int qq = 0; qq < NR; ++qq) accC[h][qq] = AR::zero();
      if (pk + 1 < npair) load_x(pk + 1, buf ^ 1);  // overlaps this pair's tiles
    }
    bool ok = false;
    if (!*abort_flag) {
      const uint32_t par = ph;
      ok = mbar_try_wait(&full[s], par);
      if (!ok) {
        const uint64_t t0 = global_ns();
        for (uint32_t it = 0; !ok; ++it) {
          ok = mbar_try_wait(&full[s], par);
          if (!ok && (it & 255u) == 255u && (*abort_flag || global_ns() - t0 > RC_WAIT_NS)) break;
        }
        if (!ok && !*abort_flag) {
          atomicOr(P.err, DEVERR_TIMEOUT);
          *abort_flag = 1;
        }
      }
    }
    const E *tile = stage0 + (size_t)s * stage_elems;
    const int r0 = t * TR;
    if (ok) {
      if (w < 4) {
        // Row leg: row rl of the tile, columns 2 LPR i + 2 c4 (+1).
        const int rl = RPW * w + r8;
        const E *zrow = tile + (size_t)rl * lds;
        Acc acc[NR];
#pragma unroll
        for (int qq = 0; qq < NR; ++qq) acc[qq] = AR::zero();
        for (int c = 2 * c4; c < b; c += 2 * LPR) {
          E z0, z1;
          AR::load2(zrow, c, z0, z1);
          if (HERM) {
            z0 = AR::conj(z0);
            z1 = AR::conj(z1);
          }
#pragma unroll
          for (int qq = 0; qq < NR; ++qq) {
            AR::fma(acc[qq], z0, xr_s[qq * b + c]);
            AR::fma(acc[qq], z1, xr_s[qq * b + c + 1]);
          }
        }
#pragma unroll
        for (int qq = 0; qq < NR; ++qq) acc[qq] = AR::template sum_row<RPW>(acc[qq]);
        if (c4 == 0)
#pragma unroll
          for (int qq = 0; qq < NR; ++qq)
            if (q0 + qq < nr) Y[((size_t)kR * nr + q0 + qq) * b + r0 + rl] = AR::value(acc[qq]);
      } else if (col_active && !selfp && cc < b) {
        // Column leg: column pair cc, rows of this warp's slice.
        for (int rl = slice * rps; rl < (slice + 1) * rps; ++rl) {
          E z0, z1;
          AR::load2(tile + (size_t)rl * lds, cc, z0, z1);
          if (HERM) {
            z0 = AR::conj(z0);
            z1 = AR::conj(z1);
          }
#pragma unroll
          for (int qq = 0; qq < NR; ++qq) {
            const E xc = xc_s[qq * b + r0 + rl];
            AR::fma(accC[0][qq], z0, xc);
            AR::fma(accC[1][qq], z1, xc);
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) rc_arrive(&empty[s]);

    if (t == ntile - 1) {
      // The other slices' warps overwrite redC only once the slice-0 warps
      // have read the previous pair's sums (a lazy wait instead of a second
      // barrier of all consumers).
      if (col_active && slice > 0 && pk > 0) {
        int okw = 1;
        if (lane == 0 && !mbar_wait_bounded(red_free, (uint32_t)((pk - 1) & 1), RC_WAIT_NS)) {
          if (!*abort_flag) atomicOr(P.err, DEVERR_TIMEOUT);
          *abort_flag = 1;
          okw = 0;
        }
        okw = __shfl_sync(0xffffffffu, okw, 0);
        (void)okw;
      }
      if (col_active && !selfp && cc < b)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int qq = 0; qq < NR; ++qq) redC[(((size_t)kw * 32 + lane) * 2 + h) * NR + qq] = AR::value(accC[h][qq]);
      rc_cp_async_wait_all();  // this thread's prefetch of the next pair's x has landed
      rc_consumer_bar();       // redC complete; orders the prefetch before its use
      if (col_active && slice == 0) {
        if (!selfp && cc < b && !*abort_flag) {
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int qq = 0; qq < NR; ++qq) {
              Acc v = AR::zero();
              for (int sl = 0; sl < nslice; ++sl) AR::add(v, redC[((((size_t)(sl * G + cgrp)) * 32 + lane) * 2 + h) * NR + qq]);
              if (q0 + qq < nr) Y[((size_t)kC * nr + q0 + qq) * b + cc + h] = AR::value(v);
            }
        }
        __syncwarp();
        if (lane == 0) rc_arrive(red_free);
      }
    }
    if (++t == ntile) {
      t = 0;
      ++pk;
    }
    if (++s == NS) {
      s = 0;
      ph ^= 1u;
    }
  }
}

// Launch with programmatic stream serialisation: the kernel may begin
// while the previous kernel in the stream is finishing (see the consumers'
// griddepcontrol.wait).
template <typename K>
void rc_launch_pdl(K kern, int grid, size_t smem, cudaStream_t st, const RcArgs &a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(RC_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, a);
}

size_t rc_smem(int b, int NR, int NS, size_t esz, int TR = RC_TR) {
  return 256 + (size_t)NS * TR * (b + 2) * esz + (size_t)4 * NR * b * esz + (size_t)4 * 32 * 2 * NR * esz;
}

template <typename AR, int NR, bool HERM, int TR, int BB>
void rc_launch(const BinProduct &P, int num_sms, cudaStream_t st, int q0) {
  constexpr size_t esz = sizeof(typename AR::E);
  // Two CTAs per SM only for c64 (double-FP32 stages are twice as large).
  int occ = (P.occ == 2 && esz == 8) ? 2 : 1;
  const size_t cap = occ == 2 ? 110 * 1024 : 225 * 1024;
  int NS = (P.NS >= 2 && P.NS <= 6) ? P.NS : 4;
  while (NS > 2 && rc_smem(P.b, NR, NS, esz, TR) > cap) --NS;
  if (rc_smem(P.b, NR, NS, esz, TR) > cap) {  // two CTAs do not fit: one CTA per SM
    occ = 1;
    NS = std::min(NS, 3);
    while (NS > 2 && rc_smem(P.b, NR, NS, esz, TR) > 225 * 1024) --NS;
  }
  const size_t smem = rc_smem(P.b, NR, NS, esz, TR);
  int grid = num_sms * occ;
  if (grid > P.Bp) grid = P.Bp;
  RcArgs a{P, NS, q0, P.b + 2};
  if (occ == 2) {
    auto kern = bin_rc_kernel<AR, NR, HERM, 2, TR, BB>;
    static int configured = 0;
    if (!configured) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024);
      configured = 1;
    }
    rc_launch_pdl(kern, grid, smem, st, a);
  } else {
    auto kern = bin_rc_kernel<AR, NR, HERM, 1, TR, BB>;
    static int configured = 0;
    if (!configured) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      configured = 1;
    }
    rc_launch_pdl(kern, grid, smem, st, a);
  }
}

template <typename AR, int NR, int TR, int BB>
void rc_launch_hb(const BinProduct &P, int num_sms, cudaStream_t st, int q0) {
  if (P.herm) rc_launch<AR, NR, true, TR, BB>(P, num_sms, st, q0);
  else rc_launch<AR, NR, false, TR, BB>(P, num_sms, st, q0);
}

// The block orders of the benchmark workloads (b = 96, 128, 256) as
// compile-time constants, any other multiple of 32 at run time.  (A
// double-FP32 launch takes 16-row tiles exactly when b > 160.)
template <typename AR, int NR, int TR = RC_TR>
void rc_launch_h(const BinProduct &P, int num_sms, cudaStream_t st, int q0) {
  constexpr bool dfl_tiles = std::is_same<AR, RcDfl>::value;
  if constexpr (!dfl_tiles || TR == 32) {
    if (P.b == 128) return rc_launch_hb<AR, NR, TR, 128>(P, num_sms, st, q0);
    if (P.b == 96) return rc_launch_hb<AR, NR, TR, 96>(P, num_sms, st, q0);
  }
  if constexpr (!dfl_tiles || TR == 16) {
    if (P.b == 256) return rc_launch_hb<AR, NR, TR, 256>(P, num_sms, st, q0);
  }
  rc_launch_hb<AR, NR, TR, 0>(P, num_sms, st, q0);
}

// Double-FP32 RHS per launch: two (their accumulators are twice the c64
// ones').
constexpr int RC_DFL_NR = 2;

}  // namespace

bool bin_rc_supported(int b) { return b % 32 == 0 && b >= 64 && b <= 256; }

// Tile height of the double-FP32 kernel: 32 rows where two such stages fit,
// else 16.
int rc_dfl_tr(int b) { return rc_smem(b, RC_DFL_NR, 2, sizeof(dfl2), 32) <= 225 * 1024 ? 32 : 16; }

bool bin_rc_dfl_supported(int b) {
  return bin_rc_supported(b) && rc_smem(b, RC_DFL_NR, 2, sizeof(dfl2), rc_dfl_tr(b)) <= 225 * 1024;
}

void launch_bin_rc(const BinProduct &P, int num_sms, cudaStream_t st) {
  for (int q0 = 0; q0 < P.nr; q0 += 4) {
    const int left = P.nr - q0;
    if (left == 1) rc_launch_h<RcF32, 1>(P, num_sms, st, q0);
    else if (left == 2) rc_launch_h<RcF32, 2>(P, num_sms, st, q0);
    else rc_launch_h<RcF32, 4>(P, num_sms, st, q0);
  }
}

void launch_bin_rc_dfl(const BinProduct &P, int num_sms, cudaStream_t st) {
  const bool tall = rc_dfl_tr(P.b) == 32;
  for (int q0 = 0; q0 < P.nr; q0 += RC_DFL_NR) {
    if (P.nr - q0 == 1) {
      if (tall) rc_launch_h<RcDfl, 1, 32>(P, num_sms, st, q0);
      else rc_launch_h<RcDfl, 1, 16>(P, num_sms, st, q0);
    } else {
      if (tall) rc_launch_h<RcDfl, RC_DFL_NR, 32>(P, num_sms, st, q0);
      else rc_launch_h<RcDfl, RC_DFL_NR, 16>(P, num_sms, st, q0);
    }
  }
}

}  // namespace moma
