// Per-bin product of the MLFFT matvec (Eq. 3) on the fifth-generation
// tensor cores, for many right-hand sides: y_k = op(A_k) x_k for every
// circulant frequency k, where A_k = Zhat_k (operator Z) or
// conj(Zhat_{-k}) = Zhat_k^H (operator Z^H, Eq. 6 with reciprocity).
//
// Complex GEMM as one real GEMM.  Row i of a complex b x b matrix stored
// interleaved (re, im, re, im, ...) is a real row of length K' = 2b, so A_k
// is read as the real b x 2b matrix A'.  The RHS block x_k (nr x b,
// RHS-major) becomes the real K' x N' operand B' (N' = 2 nrt, K-major):
//   column j        (real part of y):  ( Re x_kj, -Im x_kj )  per k
//   column nrt + j  (imag part of y):  ( Im x_kj,  Re x_kj )  per k
// (for conj(A) the signs of the Im A terms flip), so A' B' holds Re y in
// its first nrt columns and Im y in the next nrt.
//
// Precision: 3xTF32.  Both operands are split v = hi + lo with hi, lo
// exact TF32 values; the accumulator receives hi*hi + hi*lo + lo*hi in FP32
// (tcgen05.mma kind::tf32, FP32 accumulate), which keeps the product close
// to FP32 accuracy (relative error ~1e-6 instead of TF32's ~1e-3).  B' is
// built and split in shared memory per K chunk.  A is either pre-split
// (the preconditioner factors, tc_split_factor) or read unsplit ("raw": the
// c64 pair store of the bins and its transpose, or the offset blocks of the
// Gram products) and split in shared memory by the same warps that build
// B', in place for hi and into the tile's second slot for lo -- the TMA
// then moves the c64 bytes once, not the two split copies.
//
// The same kernel applies the block preconditioner for many RHS: the
// items are then the lattice elements, A = X_e = L_e^{-1} and A = X_e^H
// (each kept whole, zeros included), and the two products run back to
// back (y = X^H (X x)).
//
// Kernel layout (persistent, one CTA per SM):
//   warp 0     TMA producer: A_hi / A_lo K-chunks (128 rows x 128 B, 128B
//              swizzle) of each 128-row M tile into an NS-deep stage ring;
//   warp 1     allocates tensor memory and (one lane) issues tcgen05.mma;
//   warps 2-5  build B'_hi / B'_lo of each K chunk in the swizzled K-major
//              layout the MMA descriptors describe;
//   warps 6-9  epilogue: tcgen05.ld of the accumulator (two buffers, so the
//              next work unit's MMAs overlap this one's stores) and
//              coalesced stores of y.
// Every mbarrier wait is bounded; on a timeout the CTA sets DEVERR_TIMEOUT,
// waits (bounded) for its own copies and MMAs, frees its tensor memory and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <stdexcept>
#include <string>

#include "internal.h"

namespace moma {

namespace {

constexpr int TC_M = 128;          // rows per M tile (MMA M)
constexpr int TC_KC = 32;          // floats per K chunk (one 128-byte swizzle row)
constexpr int TC_THREADS = 320;    // 10 warps
constexpr int TC_ATILE = TC_M * 128;  // bytes of one A tile (128 rows x 128 B)
constexpr uint64_t TC_WAIT_NS = 2000000000ull;

struct MmaArgs {
  const float2 *x;
  float2 *y;
  long long x_ts, x_rs, y_ts, y_rs;
  const int *amap;
  int T, b, nr, conj;
  int nmt, nkc, nrtiles, NS, acc_bufs, tmem_cols;
  int nmu;  // M-tile groups per item: a unit is (item, RHS tile, group of nmt M tiles)
  unsigned *err;
  const int *live;
  int rawA, check;  // A tiles arrive unsplit (hi slots) and are split by warps 2-5; check their finiteness
  int Tmap;         // raw A: matrices per map (items >= Tmap come from the second map)
};

MOMA_DEV float tf32_hi(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r & 0xFFFFE000u);
}
MOMA_DEV float tf32_trunc(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }

MOMA_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
MOMA_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart.  addr is the byte address of the (1024-aligned) tile
// plus the K offset inside the 128-byte row.
MOMA_DEV uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);         // start address
  d |= (uint64_t)1 << 16;                            // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;                  // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                            // descriptor version
  d |= (uint64_t)2 << 61;                            // 128-byte swizzle
  return d;
}

MOMA_DEV void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
MOMA_DEV void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
MOMA_DEV void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
MOMA_DEV void arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes.
MOMA_DEV void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
MOMA_DEV void tmem_ld16(uint32_t taddr, float (&v)[32]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
MOMA_DEV void tmem_ld8(uint32_t taddr, float (&v)[32]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
template <int W>
MOMA_DEV void tmem_ld(uint32_t taddr, float (&v)[32]) {
  if constexpr (W == 32) tmem_ld32(taddr, v);
  else if constexpr (W == 16) tmem_ld16(taddr, v);
  else tmem_ld8(taddr, v);
}

// Byte offset of 16-byte chunk c of row n in a K-major, 128B-swizzled tile.
MOMA_DEV uint32_t sw128_off(int n, int c) { return (uint32_t)((n >> 3) * 1024 + (n & 7) * 128 + ((c ^ (n & 7)) << 4)); }

// One wait with the CTA-wide abort flag: false (and abort set) on timeout.
MOMA_DEV bool wait_or_abort(uint64_t *bar, uint32_t parity, volatile int *abort_flag, unsigned *err) {
  if (*abort_flag) return false;
  if (mbar_wait_bounded(bar, parity, TC_WAIT_NS)) return true;
  *abort_flag = 1;
  atomicOr(err, DEVERR_TIMEOUT);
  return false;
}

// Warp-uniform variants: lane 0 waits / reads, the warp follows its answer
// (the tcgen05.ld instructions below need a converged warp).
MOMA_DEV bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, unsigned *err) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = wait_or_abort(bar, parity, abort_flag, err) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}
MOMA_DEV bool warp_aborted(volatile int *abort_flag) {
  int a = 0;
  if ((threadIdx.x & 31) == 0) a = *abort_flag;
  return __shfl_sync(0xffffffffu, a, 0) != 0;
}

template <int NRT>
__global__ void __launch_bounds__(TC_THREADS, 1)
    bin_mma_kernel(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
                   const __grid_constant__ CUtensorMap map_x, MmaArgs P) {
  if (P.live && *P.live == 0) return;
  constexpr int NP = 2 * NRT;           // MMA N
  constexpr int BTILE = NP * 128;       // bytes of one B' tile
  constexpr int XTILE = NRT * 128;      // bytes of one raw RHS chunk (NRT rows x 32 floats)
  constexpr int LW = NRT < 32 ? NRT : 32;  // accumulator columns per tcgen05.ld
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int NS = P.NS, nmt = P.nmt, nkc = P.nkc;
  const int stage_bytes = nmt * 2 * TC_ATILE + 2 * BTILE + XTILE;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)NS * stage_bytes);
  uint64_t *fullA = bars, *fullB = bars + NS, *empty = bars + 2 * NS;
  uint64_t *accf = bars + 3 * NS, *acce = accf + 2, *drain = acce + 2;
  uint64_t *fullS = drain + 1;  // [NS] raw A: the lo slots are written
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fullS + NS);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&fullA[s], 1);
      mbar_init(&fullB[s], 4);
      mbar_init(&fullS[s], 4);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], 4);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(P.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int units = P.T * P.nrtiles * P.nmu;
  const int acc_cols = nmt * NP;
  // Unit u: item u / (nrtiles nmu), RHS tile (u / nmu) % nrtiles, M tiles
  // from (u % nmu) nmt on.

  if (warp == 0) {
    // ---------------------------------------------------------- TMA --
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_hi)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_lo)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_x)) : "memory");
      int g = 0;
      int issued_in[8];
      for (int s = 0; s < 8; ++s) issued_in[s] = -1;
      for (int u = blockIdx.x; u < units && !*abort_flag; u += gridDim.x) {
        const int t = u / (P.nrtiles * P.nmu), j0 = ((u / P.nmu) % P.nrtiles) * NRT, m0 = (u % P.nmu) * nmt;
        const int ai = P.amap ? P.amap[t] : t;
        // Raw A: one unsplit tile per M tile, from hi (items < T) or lo.
        const CUtensorMap *rmap = ai < P.Tmap ? &map_hi : &map_lo;
        const int ri = ai < P.Tmap ? ai : ai - P.Tmap;
        for (int kc = 0; kc < nkc; ++kc, ++g) {
          const int s = g % NS;
          const uint32_t ph = (uint32_t)(g / NS) & 1u;
          if (!wait_or_abort(&empty[s], ph ^ 1u, abort_flag, P.err)) break;
          unsigned char *st = smem + (size_t)s * stage_bytes;
          mbar_expect_tx(&fullA[s], (uint32_t)(nmt * (P.rawA ? 1 : 2) * TC_ATILE + XTILE));
          for (int mt = 0; mt < nmt; ++mt) {
            if (P.rawA) {
              tma_load_3d(st + (size_t)(2 * mt) * TC_ATILE, rmap, kc * TC_KC, (m0 + mt) * TC_M, ri, &fullA[s]);
            } else {
              tma_load_3d(st + (size_t)(2 * mt) * TC_ATILE, &map_hi, kc * TC_KC, (m0 + mt) * TC_M, ai, &fullA[s]);
              tma_load_3d(st + (size_t)(2 * mt + 1) * TC_ATILE, &map_lo, kc * TC_KC, (m0 + mt) * TC_M, ai,
                          &fullA[s]);
            }
          }
          // Raw RHS chunk: rows j0 .. j0+NRT-1 (past nr read as zeros).
          tma_load_3d(st + (size_t)nmt * 2 * TC_ATILE + 2 * BTILE, &map_x, kc * TC_KC, t, j0, &fullA[s]);
          issued_in[s] = g;
        }
      }
      // Wait (bounded) until every copy this thread issued has landed.
      for (int s = 0; s < NS; ++s)
        if (issued_in[s] >= 0) mbar_wait_bounded(&fullA[s], (uint32_t)(issued_in[s] / NS) & 1u, TC_WAIT_NS);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA --
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NP >> 3) << 17) |
                             ((uint32_t)(TC_M >> 4) << 24);
      int g = 0, lu = 0;
      for (int u = blockIdx.x; u < units && !*abort_flag; u += gridDim.x, ++lu) {
        const int ab = lu % P.acc_bufs;
        const uint32_t aph = (uint32_t)(lu / P.acc_bufs) & 1u;
        if (!wait_or_abort(&acce[ab], aph ^ 1u, abort_flag, P.err)) break;
        tc_fence_after();
        bool ok = true;
        for (int kc = 0; kc < nkc; ++kc, ++g) {
          const int s = g % NS;
          const uint32_t ph = (uint32_t)(g / NS) & 1u;
          if (!wait_or_abort(&fullA[s], ph, abort_flag, P.err) || !wait_or_abort(&fullB[s], ph, abort_flag, P.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + (size_t)s * stage_bytes);
          const uint32_t bhi = st + (uint32_t)(nmt * 2 * TC_ATILE), blo = bhi + BTILE;
          if (!P.rawA) {
            for (int mt = 0; mt < nmt; ++mt) {
              const uint32_t d = tmem + (uint32_t)(ab * acc_cols + mt * NP);
              const uint32_t ahi = st + (uint32_t)(2 * mt) * TC_ATILE, alo = ahi + TC_ATILE;
#pragma unroll
              for (int k = 0; k < TC_KC / 8; ++k) {
                const uint32_t ko = (uint32_t)k * 32u;  // 8 TF32 values
                mma_tf32(d, sw128_desc(ahi + ko), sw128_desc(bhi + ko), idesc, (kc | k) ? 1u : 0u);
                mma_tf32(d, sw128_desc(ahi + ko), sw128_desc(blo + ko), idesc, 1u);
                mma_tf32(d, sw128_desc(alo + ko), sw128_desc(bhi + ko), idesc, 1u);
              }
            }
          } else {
            // Raw A: its FP32 values serve as A_hi as they landed (the MMA
            // reads the TF32 bits of each FP32 value, dropping the low 13),
            // so hi*hi and hi*lo start at once; lo*hi waits for the split.
            for (int mt = 0; mt < nmt; ++mt) {
              const uint32_t d = tmem + (uint32_t)(ab * acc_cols + mt * NP);
              const uint32_t ahi = st + (uint32_t)(2 * mt) * TC_ATILE;
#pragma unroll
              for (int k = 0; k < TC_KC / 8; ++k) {
                const uint32_t ko = (uint32_t)k * 32u;
                mma_tf32(d, sw128_desc(ahi + ko), sw128_desc(bhi + ko), idesc, (kc | k) ? 1u : 0u);
                mma_tf32(d, sw128_desc(ahi + ko), sw128_desc(blo + ko), idesc, 1u);
              }
            }
            if (!wait_or_abort(&fullS[s], ph, abort_flag, P.err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            for (int mt = 0; mt < nmt; ++mt) {
              const uint32_t d = tmem + (uint32_t)(ab * acc_cols + mt * NP);
              const uint32_t alo = st + (uint32_t)(2 * mt + 1) * TC_ATILE;
#pragma unroll
              for (int k = 0; k < TC_KC / 8; ++k) {
                const uint32_t ko = (uint32_t)k * 32u;
                mma_tf32(d, sw128_desc(alo + ko), sw128_desc(bhi + ko), idesc, 1u);
              }
            }
          }
          mma_commit(&empty[s]);  // stage s free once these MMAs have read it
        }
        if (!ok) break;
        mma_commit(&accf[ab]);
      }
      // Drain: wait (bounded) for every MMA this thread issued.
      mma_commit(drain);
      mbar_wait_bounded(drain, 0, TC_WAIT_NS);
    }
  } else if (warp < 6) {
    // ------------------------------------------------ B' construction --
    const int bt = threadIdx.x - 64;
    const float sgn = P.conj ? 1.0f : -1.0f;  // sign of the Im x term in the real rows
    int g = 0;
    for (int u = blockIdx.x; u < units && !warp_aborted(abort_flag); u += gridDim.x) {
      bool ok = true;
      for (int kc = 0; kc < nkc; ++kc, ++g) {
        const int s = g % NS;
        const uint32_t ph = (uint32_t)(g / NS) & 1u;
        // The stage's copies (issued after the stage was freed) have landed.
        if (!warp_wait(&fullA[s], ph, abort_flag, P.err)) {
          ok = false;
          break;
        }
        unsigned char *bhi = smem + (size_t)s * stage_bytes + (size_t)nmt * 2 * TC_ATILE;
        unsigned char *blo = bhi + BTILE;
        const float4 *xr = reinterpret_cast<const float4 *>(blo + BTILE);  // [NRT][8] float4
#pragma unroll
        for (int it = 0; it < NRT * 8 / 128 + (NRT * 8 % 128 ? 1 : 0); ++it) {
          const int idx = bt + it * 128;
          if (idx >= NRT * 8) break;
          const int j = idx >> 3, c = idx & 7;
          const float4 v = xr[idx];  // x[j][k0], x[j][k0 + 1] with k0 = 16 kc + 2 c
          // Real-part row j and imaginary-part row NRT + j (see header).
          const float re[4] = {v.x, sgn * v.y, v.z, sgn * v.w};
          const float im[4] = {v.y, -sgn * v.x, v.w, -sgn * v.z};
          float4 rh, rl, ih, il;
          float *prh = &rh.x, *prl = &rl.x, *pih = &ih.x, *pil = &il.x;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            prh[e] = tf32_hi(re[e]);
            prl[e] = tf32_trunc(re[e] - prh[e]);
            pih[e] = tf32_hi(im[e]);
            pil[e] = tf32_trunc(im[e] - pih[e]);
          }
          *reinterpret_cast<float4 *>(bhi + sw128_off(j, c)) = rh;
          *reinterpret_cast<float4 *>(blo + sw128_off(j, c)) = rl;
          *reinterpret_cast<float4 *>(bhi + sw128_off(NRT + j, c)) = ih;
          *reinterpret_cast<float4 *>(blo + sw128_off(NRT + j, c)) = il;
        }
        fence_proxy_async();  // generic-proxy writes -> visible to the tensor cores
        __syncwarp();
        if (lane == 0) arrive(&fullB[s]);
        if (P.rawA) {
          // lo = v - trunc(v) of the unsplit A tiles into each tile's second
          // slot (an elementwise map: the swizzled positions carry over); the
          // raw tile itself stands for hi = trunc(v).
          bool bad = false;
          for (int mt = 0; mt < nmt; ++mt) {
            const float4 *ah =
                reinterpret_cast<const float4 *>(smem + (size_t)s * stage_bytes + (size_t)(2 * mt) * TC_ATILE);
            float4 *al = const_cast<float4 *>(ah) + TC_ATILE / 16;
            for (int idx = bt; idx < TC_ATILE / 16; idx += 128) {
              const float4 v = ah[idx];
              bad |= !isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z) || !isfinite(v.w);
              float4 l;
              l.x = tf32_trunc(v.x - tf32_trunc(v.x));
              l.y = tf32_trunc(v.y - tf32_trunc(v.y));
              l.z = tf32_trunc(v.z - tf32_trunc(v.z));
              l.w = tf32_trunc(v.w - tf32_trunc(v.w));
              al[idx] = l;
            }
          }
          if (P.check && __any_sync(0xffffffffu, bad) && lane == 0) atomicOr(P.err, DEVERR_NONFINITE);
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) arrive(&fullS[s]);
        }
      }
      if (!ok) break;
    }
  } else {
    // ----------------------------------------------------- epilogue --
    const int q = warp & 3;  // tensor-memory lane quarter this warp may access
    int lu = 0;
    for (int u = blockIdx.x; u < units && !warp_aborted(abort_flag); u += gridDim.x, ++lu) {
      const int t = u / (P.nrtiles * P.nmu), j0 = ((u / P.nmu) % P.nrtiles) * NRT, m0 = (u % P.nmu) * nmt;
      const int ab = lu % P.acc_bufs;
      const uint32_t aph = (uint32_t)(lu / P.acc_bufs) & 1u;
      if (!warp_wait(&accf[ab], aph, abort_flag, P.err)) break;
      tc_fence_after();
      float2 *yt = P.y + (size_t)t * P.y_ts;
      for (int mt = 0; mt < nmt; ++mt) {
        const int i = (m0 + mt) * TC_M + q * 32 + lane;
        const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * acc_cols + mt * NP);
#pragma unroll
        for (int jc = 0; jc < NRT; jc += LW) {
          float re[32], im[32];
          tmem_ld<LW>(base + (uint32_t)jc, re);
          tmem_ld<LW>(base + (uint32_t)(NRT + jc), im);
          if (i < P.b) {
#pragma unroll
            for (int jj = 0; jj < LW; ++jj)
              if (j0 + jc + jj < P.nr) yt[(size_t)(j0 + jc + jj) * P.y_rs + i] = make_float2(re[jj], im[jj]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) arrive(&acce[ab]);
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P.tmem_cols) : "memory");
}

// One complex value split into TF32 pairs at position o of hi and lo.
MOMA_DEV void put_split(float *hi, float *lo, size_t o, float2 v) {
  float2 h, l;
  h.x = tf32_hi(v.x);
  h.y = tf32_hi(v.y);
  l.x = tf32_trunc(v.x - h.x);
  l.y = tf32_trunc(v.y - h.y);
  reinterpret_cast<float2 *>(hi)[o] = h;
  reinterpret_cast<float2 *>(lo)[o] = l;
}

// Full X_e = L_e^{-1} (zero above the diagonal) from the packed column-major
// inverse factor: X(i, k) sits at colbase(k) - k + i for i >= k.  Tiles of
// 32 x 32 are staged so that the packed columns are read contiguously.
__global__ void tc_split_x_kernel(const float2 *X, size_t x_stride, int b, float *hi, float *lo) {
  __shared__ float2 tile[32][33];
  const int e = blockIdx.z;
  const float2 *Xe = X + (size_t)e * x_stride;
  const int i0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, i = i0 + tx;  // tile[r][tx] = X(i, k)
    float2 v = make_float2(0.f, 0.f);
    if (i < b && k < b && i >= k) v = Xe[(size_t)k * b - (size_t)k * (k - 1) / 2 + (i - k)];
    tile[r][tx] = v;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, k = k0 + tx;
    if (i < b && k < b) put_split(hi, lo, ((size_t)e * b + i) * b + k, tile[tx][r]);
  }
}
// Full X_e^H: X^H(i, k) = conj(X(k, i)), nonzero for k >= i; row i of X^H
// is column i of X, contiguous in the packed layout.
__global__ void tc_split_xh_kernel(const float2 *X, size_t x_stride, int b, float *hi, float *lo) {
  const int e = blockIdx.y, i = blockIdx.x;
  const float2 *col = X + (size_t)e * x_stride + (size_t)i * b - (size_t)i * (i - 1) / 2 - i;  // col[k] = X(k, i)
  for (int k = threadIdx.x; k < b; k += blockDim.x) {
    float2 v = make_float2(0.f, 0.f);
    if (k >= i) v = make_float2(col[k].x, -col[k].y);
    put_split(hi, lo, ((size_t)e * b + i) * b + k, v);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return nullptr;
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Tensor maps over hi / lo viewed as [T][b][2b] floats; boxes of 128 rows x
// 32 floats (128 B, 128-byte swizzle).  Rows past b read as zeros.
void encode_maps(TcMats &m) {
  auto fn = encode_fn();
  if (!fn) throw std::runtime_error("cuTensorMapEncodeTiled is not available");
  const int b = m.b;
  const cuuint64_t dims[3] = {(cuuint64_t)(2 * b), (cuuint64_t)b, (cuuint64_t)m.T};
  const cuuint64_t strides[2] = {(cuuint64_t)(2 * b) * sizeof(float), (cuuint64_t)(2 * b) * b * sizeof(float)};
  const cuuint32_t box[3] = {TC_KC, TC_M, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  float *bases[2] = {m.hi, m.lo};
  CUtensorMap *maps[2] = {&m.map_hi, &m.map_lo};
  for (int h = 0; h < 2; ++h) {
    const CUresult r = fn(maps[h], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, bases[h], dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw std::runtime_error("cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  }
}

template <int NRT>
size_t smem_bytes(int nmt, int NS) {
  const size_t stage = (size_t)nmt * 2 * TC_ATILE + 2 * (size_t)(2 * NRT) * 128 + (size_t)NRT * 128;
  return 1024 + NS * stage + (4 * NS + 5) * sizeof(uint64_t) + 16;
}

template <int NRT>
void launch_nrt(const TcMats &m, const TcProduct &P, int num_sms, cudaStream_t st) {
  const int b = m.b;
  MmaArgs a{};
  a.x = static_cast<const float2 *>(P.x);
  a.y = static_cast<float2 *>(P.y);
  a.x_ts = P.x_ts; a.x_rs = P.x_rs; a.y_ts = P.y_ts; a.y_rs = P.y_rs;
  a.amap = P.amap;
  const int items = P.items > 0 ? P.items : m.T;
  a.T = items; a.b = b; a.nr = P.nr; a.conj = P.conj;
  a.Tmap = m.T;
  // All M tiles of an item in one unit (units of one M tile each, which fit
  // three stages with raw A at b = 256, measured slower: 578 vs 551 us at
  // 24 x 24, b = 256, 64 RHS, from building B' and loading x twice).
  a.nmt = (b + TC_M - 1) / TC_M;
  a.nmu = 1;
  a.nkc = (2 * b + TC_KC - 1) / TC_KC;
  a.nrtiles = (P.nr + NRT - 1) / NRT;
  const int per_buf = a.nmt * 2 * NRT;
  a.acc_bufs = 2 * per_buf <= 512 ? 2 : 1;
  int cols = 32;
  while (cols < a.acc_bufs * per_buf) cols <<= 1;
  a.tmem_cols = cols;
  a.err = P.err;
  a.live = P.live;
  a.rawA = m.raw ? 1 : 0;
  a.check = m.raw && P.check_finite ? 1 : 0;
  int NS = 4;
  while (NS > 2 && smem_bytes<NRT>(a.nmt, NS) > 220 * 1024) --NS;
  a.NS = NS;
  // At least 120 KB so that no two CTAs of this kernel share an SM (and its
  // tensor memory).
  const size_t smem = std::max<size_t>(smem_bytes<NRT>(a.nmt, NS), 120 * 1024);
  auto kern = bin_mma_kernel<NRT>;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    configured = true;
  }
  // RHS chunks by TMA: x viewed as floats [nr][T][2b] with the given item
  // and row strides; boxes of 32 floats x 1 item x NRT rows, no swizzle.
  CUtensorMap map_x;
  {
    auto fn = encode_fn();
    if (!fn) throw std::runtime_error("cuTensorMapEncodeTiled is not available");
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * b), (cuuint64_t)items, (cuuint64_t)P.nr};
    const cuuint64_t strides[2] = {(cuuint64_t)P.x_ts * 8, (cuuint64_t)P.x_rs * 8};
    const cuuint32_t box[3] = {TC_KC, 1, (cuuint32_t)NRT};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(&map_x, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(P.x), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw std::runtime_error("cuTensorMapEncodeTiled (x) failed: " + std::to_string((int)r));
  }
  const int units = a.T * a.nrtiles * a.nmu;
  const int grid = std::min(units, num_sms);
  kern<<<grid, TC_THREADS, smem, st>>>(m.map_hi, (m.raw && !m.lo) ? m.map_hi : m.map_lo, map_x, a);
}

}  // namespace

bool tc_supported(int b) { return b >= 128 && b <= 256 && b % 2 == 0; }

size_t tc_bytes(int T, int b) { return 2 * (size_t)T * b * 2 * b * sizeof(float); }

// Raw maps over [T][b][ld] c64 viewed as floats: the same boxes as
// encode_maps (rows past b and floats past 2b read as zeros).
void tc_raw(TcMats &m, const void *Z64, const void *Z64T, int ld) {
  auto fn = encode_fn();
  if (!fn) throw std::runtime_error("cuTensorMapEncodeTiled is not available");
  m.raw = true;
  m.ld = ld;
  m.hi = reinterpret_cast<float *>(const_cast<void *>(Z64));
  m.lo = reinterpret_cast<float *>(const_cast<void *>(Z64T));
  const int b = m.b;
  const cuuint64_t dims[3] = {(cuuint64_t)(2 * b), (cuuint64_t)b, (cuuint64_t)m.T};
  const cuuint64_t strides[2] = {(cuuint64_t)(2 * ld) * sizeof(float), (cuuint64_t)(2 * ld) * b * sizeof(float)};
  const cuuint32_t box[3] = {TC_KC, TC_M, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  float *bases[2] = {m.hi, m.lo};
  CUtensorMap *maps[2] = {&m.map_hi, &m.map_lo};
  for (int h = 0; h < 2; ++h) {
    if (!bases[h]) continue;
    const CUresult r = fn(maps[h], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, bases[h], dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw std::runtime_error("cuTensorMapEncodeTiled (raw) failed: " + std::to_string((int)r));
  }
}

// Z64T[s][i][j] = Z64[s][j][i], 32 x 32 tiles through shared memory.
__global__ void transpose_pairs_kernel(const float2 *__restrict__ Z, float2 *__restrict__ ZT, int b, int ld) {
  __shared__ float2 tile[32][33];
  const size_t base = (size_t)blockIdx.z * b * ld;
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32, tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, j = j0 + tx;
    tile[r][tx] = (i < b && j < b) ? Z[base + (size_t)i * ld + j] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r, i = i0 + tx;
    if (i < b && j < b) ZT[base + (size_t)j * ld + i] = tile[tx][r];
  }
}

void tc_transpose_pairs(const void *Z64, void *Z64T, int Bp, int b, int ld, cudaStream_t st) {
  dim3 grid((b + 31) / 32, (b + 31) / 32, Bp), block(32, 8);
  transpose_pairs_kernel<<<grid, block, 0, st>>>(static_cast<const float2 *>(Z64), static_cast<float2 *>(Z64T), b,
                                                 ld);
}

void tc_split_factor(TcMats &X, TcMats &XH, const void *Xpk, size_t x_stride, cudaStream_t st) {
  const int b = X.b;
  dim3 grid((b + 31) / 32, (b + 31) / 32, X.T), block(32, 8);
  tc_split_x_kernel<<<grid, block, 0, st>>>(static_cast<const float2 *>(Xpk), x_stride, b, X.hi, X.lo);
  tc_split_xh_kernel<<<dim3(b, XH.T), 128, 0, st>>>(static_cast<const float2 *>(Xpk), x_stride, b, XH.hi, XH.lo);
  encode_maps(X);
  encode_maps(XH);
}

void launch_tc_product(const TcMats &m, const TcProduct &P, int num_sms, cudaStream_t st) {
  if (P.nr > 32) launch_nrt<64>(m, P, num_sms, st);
  else if (P.nr > 16) launch_nrt<32>(m, P, num_sms, st);
  else if (P.nr > 8) launch_nrt<16>(m, P, num_sms, st);
  else launch_nrt<8>(m, P, num_sms, st);
}

}  // namespace moma
