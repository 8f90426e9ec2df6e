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
// The kernel is a persistent streaming GEMV: at small nrhs the bins are
// read once per product and the work is HBM bound.  Each CTA walks its bin
// pairs tile by tile (TR rows of the stored block), staging tiles in shared
// memory with 1D bulk copies (cp.async.bulk) completed on mbarriers, NS
// stages deep, so one elected thread keeps ~NS tiles in flight while eight
// warps compute from shared memory.  Warps own rows; lanes own columns
// c = lane + 32u.  Row products are warp-reduced per row; column products
// accumulate in registers across the whole block and are reduced across
// warps once per pair.
#include "internal.h"

namespace moma {

constexpr int BP_THREADS = 256;
constexpr int BP_WARPS = BP_THREADS / 32;
constexpr uint64_t BP_WAIT_NS = 2000000000ull;  // 2 s bound on any tile wait

struct BinKernelArgs {
  BinProduct P;
  int TR, ntile, NS, q0;
};

template <typename R, int NR, int U>
__global__ void __launch_bounds__(BP_THREADS) bin_pair_kernel(BinKernelArgs A) {
  using C = typename Cplx<R>::T;
  extern __shared__ __align__(128) unsigned char sm[];
  const BinProduct &P = A.P;
  const int b = P.b, ldb = P.ldb, nr = P.nr, q0 = A.q0;
  const int TR = A.TR, ntile = A.ntile, NS = A.NS;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;

  uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
  C *stage0 = reinterpret_cast<C *>(sm + 128);
  const size_t stage_elems = (size_t)TR * ldb;
  C *xR = stage0 + NS * stage_elems;
  C *xC = xR + (size_t)b * NR;
  C *red = xC + (size_t)b * NR;

  const C *Z = reinterpret_cast<const C *>(P.Z);
  const C *X = reinterpret_cast<const C *>(P.x);
  C *Y = reinterpret_cast<C *>(P.y);

  const int npair = (P.Bp - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int total = npair * ntile;
  if (total <= 0) return;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  auto issue = [&](int i) {
    const int pk = i / ntile, t = i % ntile;
    const long long p = (long long)blockIdx.x + (long long)pk * gridDim.x;
    const int r0 = t * TR;
    const int rows = min(TR, b - r0);
    const uint32_t bytes = (uint32_t)(rows * ldb * sizeof(C));
    C *dst = stage0 + (size_t)(i % NS) * stage_elems;
    const C *src = Z + ((size_t)p * b + r0) * ldb;
    fence_proxy_async();
    mbar_expect_tx(&bar[i % NS], bytes);
    bulk_g2s(dst, src, bytes, &bar[i % NS]);
  };
  if (tid == 0)
    for (int i = 0; i < NS && i < total; ++i) issue(i);

  C xr[U][NR];
  C accC[U][NR];
  int kR = 0, kC = 0;
  bool selfp = false;

  for (int i = 0; i < total; ++i) {
    const int pk = i / ntile, t = i % ntile;
    const int p = (int)blockIdx.x + pk * (int)gridDim.x;
    if (t == 0) {
      const int2 pr = P.pairs[p];
      selfp = pr.x == pr.y;
      kR = P.herm ? pr.y : pr.x;
      kC = P.herm ? pr.x : pr.y;
      for (int idx = tid; idx < b * NR; idx += BP_THREADS) {
        const int c = idx / NR, qq = idx % NR, q = q0 + qq;
        xR[idx] = q < nr ? X[((size_t)kR * nr + q) * b + c] : czero<C>();
        xC[idx] = (q < nr && !selfp) ? X[((size_t)kC * nr + q) * b + c] : czero<C>();
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = lane + 32 * u;
#pragma unroll
        for (int qq = 0; qq < NR; ++qq) {
          xr[u][qq] = c < b ? xR[c * NR + qq] : czero<C>();
          accC[u][qq] = czero<C>();
        }
      }
    }

    const int s = i % NS;
    const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)((i / NS) & 1), BP_WAIT_NS);
    if (ok) {
      const C *tile = stage0 + (size_t)s * stage_elems;
      const int r0 = t * TR, rows = min(TR, b - r0);
      for (int rr = w; rr < rows; rr += BP_WARPS) {
        const int r = r0 + rr;
        const C *zrow = tile + (size_t)rr * ldb;
        C pr[NR], xc[NR];
#pragma unroll
        for (int qq = 0; qq < NR; ++qq) {
          pr[qq] = czero<C>();
          xc[qq] = xC[r * NR + qq];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int c = lane + 32 * u;
          if (c < b) {
            C z = zrow[c];
            if (P.herm) z = cconj(z);
#pragma unroll
            for (int qq = 0; qq < NR; ++qq) {
              pr[qq] = cfma(z, xr[u][qq], pr[qq]);
              accC[u][qq] = cfma(z, xc[qq], accC[u][qq]);
            }
          }
        }
#pragma unroll
        for (int qq = 0; qq < NR; ++qq) {
          const C v = warp_sum(pr[qq]);
          if (lane == 0 && q0 + qq < nr) Y[((size_t)kR * nr + q0 + qq) * b + r] = v;
        }
      }
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(P.err, DEVERR_TIMEOUT);
        for (int j = i; j < total && j < i + NS; ++j)
          mbar_wait_bounded(&bar[j % NS], (uint32_t)((j / NS) & 1), BP_WAIT_NS);
      }
      return;
    }
    if (tid == 0 && i + NS < total) issue(i + NS);

    if (t == ntile - 1 && !selfp) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = lane + 32 * u;
        if (c < b) {
#pragma unroll
          for (int qq = 0; qq < NR; ++qq) red[((size_t)w * b + c) * NR + qq] = accC[u][qq];
        }
      }
      __syncthreads();
      for (int idx = tid; idx < b * NR; idx += BP_THREADS) {
        C v = czero<C>();
        for (int ww = 0; ww < BP_WARPS; ++ww) v = cadd(v, red[(size_t)ww * b * NR + idx]);
        const int c = idx / NR, qq = idx % NR;
        if (q0 + qq < nr) Y[((size_t)kC * nr + q0 + qq) * b + c] = v;
      }
    }
  }
}

template <typename R, int NR, int U>
static void launch_one(const BinProduct &P, int num_sms, cudaStream_t st, int q0) {
  using C = typename Cplx<R>::T;
  const int row_bytes = P.ldb * (int)sizeof(C);
  int TR = 16384 / row_bytes;
  if (TR < 1) TR = 1;
  if (TR > P.b) TR = P.b;
  const int ntile = (P.b + TR - 1) / TR;
  const int NS = 4;
  const size_t smem = 128 + (size_t)NS * TR * row_bytes + (size_t)2 * P.b * NR * sizeof(C) +
                      (size_t)BP_WARPS * P.b * NR * sizeof(C);
  auto kern = bin_pair_kernel<R, NR, U>;
  static int configured = 0;
  if (!configured) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    configured = 1;
  }
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BP_THREADS, smem);
  if (per_sm < 1) per_sm = 1;
  int grid = num_sms * per_sm;
  if (grid > P.Bp) grid = P.Bp;
  BinKernelArgs a{P, TR, ntile, NS, q0};
  kern<<<grid, BP_THREADS, smem, st>>>(a);
}

template <typename R, int NR>
static void launch_nr(const BinProduct &P, int num_sms, cudaStream_t st, int q0) {
  const int U = (P.b + 31) / 32;
  if (U <= 1) launch_one<R, NR, 1>(P, num_sms, st, q0);
  else if (U <= 2) launch_one<R, NR, 2>(P, num_sms, st, q0);
  else if (U <= 4) launch_one<R, NR, 4>(P, num_sms, st, q0);
  else launch_one<R, NR, 8>(P, num_sms, st, q0);
}

template <typename R>
void launch_bin_product(const BinProduct &P, int num_sms, cudaStream_t st) {
  // RHS are processed in chunks of up to NRMAX columns (the kernel masks
  // columns past nr); each chunk streams the bins once.
  constexpr int NRMAX = sizeof(R) == 4 ? 4 : 2;
  for (int q0 = 0; q0 < P.nr; q0 += NRMAX) {
    const int left = P.nr - q0;
    if (left == 1) launch_nr<R, 1>(P, num_sms, st, q0);
    else if (left == 2) launch_nr<R, 2>(P, num_sms, st, q0);
    else launch_nr<R, NRMAX>(P, num_sms, st, q0);
  }
}

template void launch_bin_product<float>(const BinProduct &, int, cudaStream_t);
template void launch_bin_product<double>(const BinProduct &, int, cudaStream_t);

}  // namespace moma
