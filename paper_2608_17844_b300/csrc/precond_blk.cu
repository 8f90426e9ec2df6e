// Streaming application of the block preconditioner P^{-1} (Eq. 38; P_e
// factored as in Sec. III-A, P_e^{-1} = X_e^H X_e with X_e = L_e^{-1}) for
// the c64 inner solve: one persistent CTA per SM walks its elements with an
// NS-deep ring of bulk copies, so the next elements' blocks are in flight
// while the current one is applied.
//
// Stored per element (built once per set-up from the packed inverse
// factor): the Hermitian Q_e = P_e^{-1} = X_e^H X_e, its lower triangle
// padded to bp = 8 ceil(b / 8) and cut into 8 x 8 blocks, diagonal blocks
// whole; block (p, q), q <= p, is block number p (p + 1) / 2 + q, and entry
// (i, k) of a block (row i, column k inside it) sits at k * 8 + (i ^ k).
// y = Q x is one pass with no intermediate vector: warp w owns the 8 rows
// of panel w, y_w = sum_{q <= w} Q(w, q) x_q + sum_{p > w} Q(p, w)^H x_p,
//  * row part: lane (r = lane % 8, c = lane / 8) reads entries (r, c) and
//    (r, c + 4) of blocks (w, 0..w);
//  * column part: lane (k = lane % 8, c) reads entries (c, k) and (c + 4, k)
//    of blocks (w+1..P-1, w);
// both free of shared-memory bank conflicts by the XOR swizzle.  Every
// warp touches P blocks per element, and no partial sums cross warps (only
// the four lanes of a row are added, by shuffles).  Q_e holds as many
// bytes as the blocked X_e, so the stream is the same, but the apply is
// one product instead of two dependent ones (the second waited at a
// barrier for the whole first).
#include <stdexcept>

#include "internal.h"

namespace moma {

namespace {

constexpr int PB_MAX_NS = 4;
constexpr size_t PB_SMEM = 227 * 1024;

struct PbArgs {
  const float2 *Xb;
  size_t xbs;  // complex entries per element (P (P + 1) / 2 blocks of 64)
  int nel, b, P, nr, ns;
  size_t stage_bytes;
  const float2 *x;
  float2 *y;
  long long vstride, voff;
  unsigned *err;
  const int *live;
};

MOMA_DEV float2 cfma2(float2 a, float2 b, float2 acc) { return cfma(a, b, acc); }
MOMA_DEV float2 sum4(float2 v) {  // add the four lanes c = 0..3 of a row / column (lane bits 3 and 4)
  v.x += __shfl_xor_sync(0xffffffffu, v.x, 8);
  v.y += __shfl_xor_sync(0xffffffffu, v.y, 8);
  v.x += __shfl_xor_sync(0xffffffffu, v.x, 16);
  v.y += __shfl_xor_sync(0xffffffffu, v.y, 16);
  return v;
}

// Q_e = X_e^H X_e from the packed inverse factor (column-major lower: X(m, j)
// at j b - j (j - 1) / 2 + m - j), staged in shared memory transposed to
// row-major lower (X(m, j) at m (m + 1) / 2 + j) so that a row m serves all
// of a tile's columns; Q(I, K) = sum over m >= max(I, K) of
// conj(X(m, I)) X(m, K).  A thread computes a 2 x 2 tile
// (rows I0, I0 + 1; columns K0, K0 + 1) of one 8 x 8 block, so each value
// it loads serves two multiply-adds; FP32 accumulation (the apply is c64).
// Padding rows and columns (>= b) are zero.
constexpr int PACK_THREADS = 512;

__global__ void __launch_bounds__(PACK_THREADS) pinv_pack_kernel(const float2 *__restrict__ Xpk, size_t x_stride,
                                                                 int b, int P, float2 *Qb, size_t qbs) {
  extern __shared__ __align__(16) unsigned char smx[];
  float2 *Xs = reinterpret_cast<float2 *>(smx);
  const int e = blockIdx.x, npk = b * (b + 1) / 2;
  for (int t = threadIdx.x; t < npk; t += blockDim.x) {
    int m = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while (m * (m + 1) / 2 > t) --m;
    while ((m + 1) * (m + 2) / 2 <= t) ++m;
    const int j = t - m * (m + 1) / 2;
    Xs[t] = Xpk[(size_t)e * x_stride + (size_t)j * b - (size_t)j * (j - 1) / 2 + (m - j)];
  }
  __syncthreads();
  const int ntiles = P * (P + 1) / 2 * 16;
  for (int tt = threadIdx.x; tt < ntiles; tt += blockDim.x) {
    const int blk = tt >> 4, i0 = ((tt >> 2) & 3) * 2, k0 = (tt & 3) * 2;
    int p = 0;
    while ((p + 1) * (p + 2) / 2 <= blk) ++p;
    const int q = blk - p * (p + 1) / 2;
    const int I0 = 8 * p + i0, K0 = 8 * q + k0;
    float2 a00 = make_float2(0.f, 0.f), a01 = a00, a10 = a00, a11 = a00;
    for (int m = max(I0, K0); m < b; ++m) {
      const float2 *row = Xs + m * (m + 1) / 2;
      const float2 xi0 = row[I0], xk0 = row[K0];  // I0, K0 <= m
      const float2 xi1 = I0 + 1 <= m ? row[I0 + 1] : make_float2(0.f, 0.f);
      const float2 xk1 = K0 + 1 <= m ? row[K0 + 1] : make_float2(0.f, 0.f);
      a00 = cfmac(xi0, xk0, a00);
      a01 = cfmac(xi0, xk1, a01);
      a10 = cfmac(xi1, xk0, a10);
      a11 = cfmac(xi1, xk1, a11);
    }
    float2 *out = Qb + (size_t)e * qbs + (size_t)blk * 64;
    out[k0 * 8 + (i0 ^ k0)] = a00;
    out[(k0 + 1) * 8 + (i0 ^ (k0 + 1))] = a01;
    out[k0 * 8 + ((i0 + 1) ^ k0)] = a10;
    out[(k0 + 1) * 8 + ((i0 + 1) ^ (k0 + 1))] = a11;
  }
}

__global__ void __launch_bounds__(1024, 1) precond_blk_kernel(PbArgs A) {
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm);  // [PB_MAX_NS]
  const int P = A.P, bp = 8 * P, b = A.b, nr = A.nr, ns = A.ns;
  unsigned char *stages = sm + 128;
  if (A.live && *A.live == 0) return;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int r8 = lane & 7, c4 = lane >> 3;
  const uint32_t xbytes = (uint32_t)(A.xbs * sizeof(float2)), vbytes = (uint32_t)(b * sizeof(float2));
  if (tid == 0) {
    for (int s = 0; s < ns; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  // The x slots' padding entries b .. bp-1 are never written by the copies.
  for (int s = 0; s < ns; ++s) {
    float2 *xs = reinterpret_cast<float2 *>(stages + (size_t)s * A.stage_bytes + xbytes);
    for (int idx = tid; idx < nr * (bp - b); idx += blockDim.x)
      xs[(idx / (bp - b)) * bp + b + idx % (bp - b)] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  // Thread 0: bulk copies of element blockIdx.x + it * gridDim.x (factor and
  // its RHS slices) into stage it % ns.
  auto issue = [&](int it) {
    const long long e = (long long)blockIdx.x + (long long)it * gridDim.x;
    if (e >= A.nel) return;
    const int s = it % ns;
    unsigned char *st = stages + (size_t)s * A.stage_bytes;
    fence_proxy_async();
    mbar_expect_tx(&bar[s], xbytes + (uint32_t)nr * vbytes);
    bulk_g2s(st, A.Xb + (size_t)e * A.xbs, xbytes, &bar[s]);
    for (int q = 0; q < nr; ++q)
      bulk_g2s(st + xbytes + (size_t)q * bp * sizeof(float2), A.x + q * A.vstride + A.voff + e * b, vbytes, &bar[s]);
  };
  if (tid == 0)
    for (int it = 0; it < ns; ++it) issue(it);

  for (int it = 0;; ++it) {
    const long long e = (long long)blockIdx.x + (long long)it * gridDim.x;
    if (e >= A.nel) break;
    const int s = it % ns;
    const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)((it / ns) & 1), 2000000000ull);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(A.err, DEVERR_TIMEOUT);
        // Drain the copies still in flight (stages it .. it + ns - 1), bounded.
        for (int j = it; j < it + ns; ++j)
          if ((long long)blockIdx.x + (long long)j * gridDim.x < A.nel)
            mbar_wait_bounded(&bar[j % ns], (uint32_t)((j / ns) & 1), 2000000000ull);
      }
      return;
    }
    const float2 *Xs = reinterpret_cast<const float2 *>(stages + (size_t)s * A.stage_bytes);
    const float2 *xs = reinterpret_cast<const float2 *>(stages + (size_t)s * A.stage_bytes + xbytes);
    for (int q0 = 0; q0 < nr; q0 += 2) {
      const bool two = q0 + 1 < nr;
      const float2 *x0 = xs + (size_t)q0 * bp, *x1 = xs + (size_t)(two ? q0 + 1 : q0) * bp;
      if (w < P) {
        float2 a0 = make_float2(0.f, 0.f), a1 = a0;
        // Row part: blocks (w, 0..w), the diagonal block whole.
        const float2 *row = Xs + (size_t)(w * (w + 1) / 2) * 64;
        for (int q = 0; q <= w; ++q) {
          const float2 *blk = row + q * 64;
#pragma unroll
          for (int m = 0; m < 2; ++m) {
            const int k = c4 + 4 * m;
            const float2 qv = blk[k * 8 + (r8 ^ k)];
            a0 = cfma2(qv, x0[8 * q + k], a0);
            a1 = cfma2(qv, x1[8 * q + k], a1);
          }
        }
        // Column part: blocks (w+1..P-1, w), conjugate-transposed.
        for (int p = w + 1; p < P; ++p) {
          const float2 *blk = Xs + (size_t)(p * (p + 1) / 2 + w) * 64;
#pragma unroll
          for (int m = 0; m < 2; ++m) {
            const int i = c4 + 4 * m;
            const float2 qv = blk[r8 * 8 + (i ^ r8)];
            a0 = cfmac(qv, x0[8 * p + i], a0);
            a1 = cfmac(qv, x1[8 * p + i], a1);
          }
        }
        a0 = sum4(a0);
        a1 = sum4(a1);
        const int k = 8 * w + r8;
        if (c4 == 0 && k < b) {
          A.y[q0 * A.vstride + A.voff + e * b + k] = a0;
          if (two) A.y[(q0 + 1) * A.vstride + A.voff + e * b + k] = a1;
        }
      }
    }
    __syncthreads();  // every warp is done with stage s before it is refilled
    if (tid == 0) issue(it + ns);
  }
}

size_t stage_bytes(int b, int nr) {
  const int P = (b + 7) / 8;
  const size_t xbs = (size_t)P * (P + 1) / 2 * 64;
  return ((xbs + (size_t)nr * 8 * P) * sizeof(float2) + 127) / 128 * 128;
}

int stages_for(int b, int nr) {
  const int P = (b + 7) / 8;
  const size_t head = 128;
  const size_t sb = stage_bytes(b, nr);
  if (head + sb > PB_SMEM) return 0;
  return (int)std::min<size_t>(PB_MAX_NS, (PB_SMEM - head) / sb);
}

}  // namespace

size_t xblk_entries(int b) {
  const int P = (b + 7) / 8;
  return (size_t)P * (P + 1) / 2 * 64;
}

bool precond_blk_supported(int b, int nr, long long vstride, long long voff) {
  return b >= 16 && b % 2 == 0 && (b + 7) / 8 <= 32 && nr >= 1 && vstride % 2 == 0 && voff % 2 == 0 &&
         stages_for(b, nr) >= 2;
}

void launch_pinv_pack(const void *Xpk, size_t x_stride, int nel, int b, void *Qb, cudaStream_t st) {
  const int P = (b + 7) / 8;
  const size_t smem = (size_t)b * (b + 1) / 2 * sizeof(float2);
  if (smem > PB_SMEM) throw std::runtime_error("pinv_pack: block too large");
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(pinv_pack_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PB_SMEM);
    configured = true;
  }
  pinv_pack_kernel<<<nel, PACK_THREADS, smem, st>>>(reinterpret_cast<const float2 *>(Xpk), x_stride, b, P,
                                                    reinterpret_cast<float2 *>(Qb), xblk_entries(b));
}

void launch_precond_blk(const void *Qb, int nel, int b, int nr, const void *x, void *y, unsigned *err,
                        const int *live, long long vstride, long long voff, int num_sms, cudaStream_t st) {
  if (!precond_blk_supported(b, nr, vstride, voff)) throw std::runtime_error("precond_blk: unsupported shape");
  PbArgs a;
  a.Xb = reinterpret_cast<const float2 *>(Qb);
  a.xbs = xblk_entries(b);
  a.nel = nel;
  a.b = b;
  a.P = (b + 7) / 8;
  a.nr = nr;
  a.ns = stages_for(b, nr);
  a.stage_bytes = stage_bytes(b, nr);
  a.x = reinterpret_cast<const float2 *>(x);
  a.y = reinterpret_cast<float2 *>(y);
  a.vstride = vstride;
  a.voff = voff;
  a.err = err;
  a.live = live;
  const size_t smem = 128 + (size_t)a.ns * a.stage_bytes;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(precond_blk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PB_SMEM);
    configured = true;
  }
  const int grid = std::min(nel, num_sms);
  precond_blk_kernel<<<grid, 32 * a.P, smem, st>>>(a);
}

}  // namespace moma
