// Restarted GMRES on the preconditioned normal equations (Sec. III-A:
// P^{-1} Z^H Z I = P^{-1} Z^H V) inside an FP64 iterative-refinement loop.
//
// All nr right-hand sides run side by side, each with its own Krylov basis,
// Hessenberg matrix and convergence state (column q freezes when its
// residual estimate reaches its tolerance).  Orthogonalisation is classical
// Gram-Schmidt with one re-orthogonalisation pass (CGS2), fused so that the
// basis is swept three times per step:
//   pass 1: h1 = V^H w
//   pass 2: w -= V h1, then h2 = V^H w       (same sweep)
//   pass 3: w -= V h2, then ||w||^2, Givens  (same sweep)
// Each pass ends with a "last block done" reduction: every CTA writes its
// partial sums, the last CTA to arrive (atomic ticket) adds them in a fixed
// order, so results are deterministic and no CTA ever waits on another.
// Dot products and norms accumulate in FP64; the Hessenberg matrix, the
// Givens rotations and the small least-squares solve are FP64.
#include "krylov.h"

namespace moma {

constexpr int KT = 256;   // threads per CTA
constexpr int KEPT = 4;   // elements per thread
constexpr int KG = 8;     // dot products reduced together

// Block-wide sum of NV complex values held by every thread, in the
// precision of C; result valid in thread 0 (red must hold 8 * NV values).
template <typename C, int NV>
MOMA_DEV void block_sum(C (&v)[NV], C *red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[w * NV + i] = v[i];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      C s = red[i];
      for (int ww = 1; ww < KT / 32; ++ww) s = cadd(s, red[ww * NV + i]);
      v[i] = s;
    }
  }
  __syncthreads();
}

// Sum over the nch chunk partials of value i (stride `stride`), in FP64 and
// a fixed order: lanes take chunks lane, lane+32, ..., then a warp tree.
MOMA_DEV double2 chunk_sum(const double2 *pq, int nch, int stride, int i) {
  const int lane = threadIdx.x & 31;
  double2 s = make_double2(0, 0);
  for (int ch = lane; ch < nch; ch += 32) s = cadd(s, pq[(size_t)ch * stride + i]);
  return warp_sum(s);
}

// Givens step for column j of RHS q (thread-serial, FP64).
MOMA_DEV void givens_step(const KrylovCtl &c, int q, int j, double wnorm) {
  const int m = c.m;
  double2 *h = c.hacc + (size_t)q * (m + 1);
  double *cs = c.cs + (size_t)q * m;
  double2 *sn = c.sn + (size_t)q * m;
  double2 *g = c.g + (size_t)q * (m + 1);
  h[j + 1] = make_double2(wnorm, 0.0);
  for (int i = 0; i < j; ++i) {
    const double2 a = h[i], bb = h[i + 1];
    h[i] = cadd(cscale(a, cs[i]), cmul(sn[i], bb));
    h[i + 1] = csub(cscale(bb, cs[i]), cmul(cconj(sn[i]), a));
  }
  const double2 f = h[j];
  const double af = hypot(f.x, f.y);
  const double t = hypot(af, wnorm);
  if (af == 0.0) {
    cs[j] = 0.0;
    sn[j] = make_double2(1.0, 0.0);
    h[j] = make_double2(wnorm, 0.0);
  } else {
    cs[j] = af / t;
    const double2 ph = cscale(f, 1.0 / af);
    sn[j] = cscale(ph, wnorm / t);  // (f/|f|) conj(g) / t with g = wnorm real
    h[j] = cscale(ph, t);
  }
  h[j + 1] = make_double2(0.0, 0.0);
  const double2 gj = g[j];
  g[j + 1] = cscale(cmul(cconj(sn[j]), gj), -1.0);
  g[j] = cscale(gj, cs[j]);
  double2 *rc = c.Rm + ((size_t)q * m + j) * (m + 1);
  for (int i = 0; i <= j; ++i) rc[i] = h[i];
  const double res = hypot(g[j + 1].x, g[j + 1].y);
  c.res[q] = res;
  const bool conv = res <= c.tol[q];
  // Lucky breakdown: the new direction vanished, the current space is invariant.
  const bool breakdown = !(wnorm > 1e-300) || wnorm <= 1e-14 * c.beta[q];
  if (conv || breakdown || j + 1 >= m || !isfinite(res)) {
    c.kq[q] = j + 1;
    c.active[q] = 0;
    atomicSub(c.nact, 1);
    c.inv_norm[q] = 0.0;
    if (!isfinite(res)) atomicOr(c.err, DEVERR_NONFINITE);
  } else {
    c.inv_norm[q] = 1.0 / wnorm;
  }
}

template <typename R>
__global__ void __launch_bounds__(KT) cgs_kernel(KrylovCtl c, typename Cplx<R>::T *V, size_t vstride, int N, int j,
                                                  int flags) {
  using C = typename Cplx<R>::T;
  __shared__ C red[8 * KG];
  __shared__ C hs[MOMA_MAX_RESTART + 1];
  __shared__ int last;
  const int q = blockIdx.y, chunk = blockIdx.x, tid = threadIdx.x;
  if (!c.active[q]) return;
  const int m = c.m;
  const size_t qoff = (size_t)q * N;
  C *w = V + (size_t)(j + 1) * vstride + qoff;
  const int n0 = chunk * KT * KEPT;

  C wv[KEPT];
#pragma unroll
  for (int t = 0; t < KEPT; ++t) {
    const int n = n0 + tid + KT * t;
    wv[t] = n < N ? w[n] : czero<C>();
  }
  if (flags & KF_UPDATE) {
    for (int i = tid; i <= j; i += KT) hs[i] = cvt<C>(c.hcur[(size_t)q * (m + 1) + i]);
    __syncthreads();
    for (int i = 0; i <= j; ++i) {
      const C hi = hs[i];
      const C *vi = V + (size_t)i * vstride + qoff;
#pragma unroll
      for (int t = 0; t < KEPT; ++t) {
        const int n = n0 + tid + KT * t;
        if (n < N) wv[t] = csub(wv[t], cmul(vi[n], hi));
      }
    }
#pragma unroll
    for (int t = 0; t < KEPT; ++t) {
      const int n = n0 + tid + KT * t;
      if (n < N) w[n] = wv[t];
    }
  }
  double2 *part = c.partial + ((size_t)q * gridDim.x + chunk) * (m + 1);
  // Each thread sums its KEPT products in the vector precision; the partials
  // are reduced across threads, CTAs and chunks in FP64.
  if (flags & KF_DOTS) {
    for (int i0 = 0; i0 <= j; i0 += KG) {
      C accr[KG];
#pragma unroll
      for (int ii = 0; ii < KG; ++ii) accr[ii] = czero<C>();
#pragma unroll
      for (int ii = 0; ii < KG; ++ii) {
        const int i = i0 + ii;
        if (i <= j) {
          const C *vi = V + (size_t)i * vstride + qoff;
#pragma unroll
          for (int t = 0; t < KEPT; ++t) {
            const int n = n0 + tid + KT * t;
            if (n < N) accr[ii] = cfmac(vi[n], wv[t], accr[ii]);
          }
        }
      }
      block_sum<C, KG>(accr, red);
      if (tid == 0)
        for (int ii = 0; ii < KG && i0 + ii <= j; ++ii) part[i0 + ii] = cvt<double2>(accr[ii]);
    }
  }
  if (flags & KF_NORM) {
    C acc[1] = {czero<C>()};
#pragma unroll
    for (int t = 0; t < KEPT; ++t) acc[0].x += wv[t].x * wv[t].x + wv[t].y * wv[t].y;
    block_sum<C, 1>(acc, red);
    if (tid == 0) part[0] = cvt<double2>(acc[0]);
  }

  // Last-block reduction over the chunks of this RHS, in chunk order.
  __threadfence();
  if (tid == 0) last = (atomicAdd(&c.counters[q], 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  const double2 *pq = c.partial + (size_t)q * gridDim.x * (m + 1);
  const int wid = tid >> 5, lane = tid & 31;
  if (flags & KF_DOTS) {
    for (int i = wid; i <= j; i += KT / 32) {
      const double2 sm = chunk_sum(pq, gridDim.x, m + 1, i);
      if (lane == 0) {
        double2 *ha = c.hacc + (size_t)q * (m + 1) + i;
        *ha = (flags & KF_ACCUM) ? cadd(*ha, sm) : sm;
        c.hcur[(size_t)q * (m + 1) + i] = sm;
      }
    }
  }
  if ((flags & KF_NORM) && wid == 0) {
    const double nrm = sqrt(chunk_sum(pq, gridDim.x, m + 1, 0).x);
    if (lane == 0) {
      if (flags & KF_INIT) {
        c.beta[q] = nrm;
        c.g[(size_t)q * (m + 1)] = make_double2(nrm, 0.0);
        c.tol[q] = c.inner_tol * nrm;
        c.res[q] = nrm;
        if (nrm > 0.0 && isfinite(nrm)) {
          c.inv_norm[q] = 1.0 / nrm;
        } else {
          if (!isfinite(nrm)) atomicOr(c.err, DEVERR_NONFINITE);
          c.inv_norm[q] = 0.0;
          c.active[q] = 0;
          c.kq[q] = 0;
          atomicSub(c.nact, 1);
        }
      } else {
        givens_step(c, q, j, nrm);
      }
    }
  }
  if (tid == 0) c.counters[q] = 0;
}

// Grid-wide barrier of the fused Arnoldi step (all CTAs co-resident: the
// kernel is launched cooperatively).  A monotonically increasing counter,
// zeroed once per GMRES cycle; a CTA waits until every CTA has arrived at
// this generation.  The wait is bounded (2 s): on timeout the CTA records
// DEVERR_TIMEOUT and reports failure, and the kernel returns.
MOMA_DEV bool grid_barrier(unsigned *count, unsigned nblocks, unsigned *err) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned old = atomicAdd(count, 1u);
    const unsigned target = (old / nblocks + 1u) * nblocks;
    int ok = 1;
    const uint64_t t0 = global_ns();
    for (unsigned it = 1;; ++it) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
      if ((int)(v - target) >= 0) break;
      if ((it & 255u) == 0 && global_ns() - t0 > 2000000000ull) {
        atomicOr(err, DEVERR_TIMEOUT);
        ok = 0;
        break;
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// The fused Arnoldi step: CTA (chunk, q) keeps its chunk of w = V[j + 1] in
// registers through the three sweeps; the per-chunk partial sums of each
// sweep go to their own buffer and, after a grid barrier, every CTA of RHS q
// adds them in the same fixed order as the last-block reduction of
// cgs_kernel, so the step is bitwise the three-launch version.
template <typename R>
__global__ void __launch_bounds__(KT) arnoldi_fused_kernel(KrylovCtl c, typename Cplx<R>::T *V, size_t vstride,
                                                            int N, int j) {
  using C = typename Cplx<R>::T;
  __shared__ C red[8 * KG];
  __shared__ C hs[MOMA_MAX_RESTART + 1];
  __shared__ double2 hd[MOMA_MAX_RESTART + 1];
  const int q = blockIdx.y, chunk = blockIdx.x, tid = threadIdx.x, nch = gridDim.x;
  const unsigned nblocks = gridDim.x * gridDim.y;
  if (*c.nact == 0) return;  // uniform: nact changes only after the last barrier
  const bool act = c.active[q] != 0;
  const int m = c.m, wid = tid >> 5, lane = tid & 31;
  const size_t qoff = (size_t)q * N;
  C *w = V + (size_t)(j + 1) * vstride + qoff;
  const int n0 = chunk * KT * KEPT;
  C wv[KEPT];
#pragma unroll
  for (int t = 0; t < KEPT; ++t) {
    const int n = n0 + tid + KT * t;
    wv[t] = (act && n < N) ? w[n] : czero<C>();
  }
  // Sweep partial dot products V_i^H w (i <= j) into buf.
  auto dots = [&](double2 *buf) {
    for (int i0 = 0; i0 <= j; i0 += KG) {
      C accr[KG];
#pragma unroll
      for (int ii = 0; ii < KG; ++ii) accr[ii] = czero<C>();
#pragma unroll
      for (int ii = 0; ii < KG; ++ii) {
        const int i = i0 + ii;
        if (i <= j) {
          const C *vi = V + (size_t)i * vstride + qoff;
#pragma unroll
          for (int t = 0; t < KEPT; ++t) {
            const int n = n0 + tid + KT * t;
            if (n < N) accr[ii] = cfmac(vi[n], wv[t], accr[ii]);
          }
        }
      }
      block_sum<C, KG>(accr, red);
      if (tid == 0)
        for (int ii = 0; ii < KG && i0 + ii <= j; ++ii)
          buf[((size_t)q * nch + chunk) * (m + 1) + i0 + ii] = cvt<double2>(accr[ii]);
    }
  };
  // h_i = sum over chunks (fixed order) into hd (FP64) and hs (precision C).
  auto gather = [&](const double2 *buf) {
    const double2 *pq = buf + (size_t)q * nch * (m + 1);
    for (int i = wid; i <= j; i += KT / 32) {
      const double2 sm = chunk_sum(pq, nch, m + 1, i);
      if (lane == 0) {
        hd[i] = sm;
        hs[i] = cvt<C>(sm);
      }
    }
    __syncthreads();
  };
  auto update = [&]() {  // w -= V h
    for (int i = 0; i <= j; ++i) {
      const C hi = hs[i];
      const C *vi = V + (size_t)i * vstride + qoff;
#pragma unroll
      for (int t = 0; t < KEPT; ++t) {
        const int n = n0 + tid + KT * t;
        if (n < N) wv[t] = csub(wv[t], cmul(vi[n], hi));
      }
    }
  };

  if (act) dots(c.partial);
  if (!grid_barrier(c.gbar, nblocks, c.err)) return;
  if (act) {
    gather(c.partial);
    if (chunk == 0)
      for (int i = tid; i <= j; i += KT) c.hacc[(size_t)q * (m + 1) + i] = hd[i];
    update();
    dots(c.partial2);
  }
  if (!grid_barrier(c.gbar, nblocks, c.err)) return;
  double nrm = 0.0;
  if (act) {
    gather(c.partial2);
    if (chunk == 0)
      for (int i = tid; i <= j; i += KT) {
        double2 *ha = c.hacc + (size_t)q * (m + 1) + i;
        *ha = cadd(*ha, hd[i]);
      }
    update();
    C acc[1] = {czero<C>()};
#pragma unroll
    for (int t = 0; t < KEPT; ++t) acc[0].x += wv[t].x * wv[t].x + wv[t].y * wv[t].y;
    block_sum<C, 1>(acc, red);
    if (tid == 0) c.partial3[(size_t)q * nch + chunk] = cvt<double2>(acc[0]);
  }
  if (!grid_barrier(c.gbar, nblocks, c.err)) return;
  if (!act) return;
  {
    __shared__ double nrm_s;
    if (wid == 0) {
      double2 s = make_double2(0, 0);
      for (int ch = lane; ch < nch; ch += 32) s = cadd(s, c.partial3[(size_t)q * nch + ch]);
      s = warp_sum(s);
      if (lane == 0) nrm_s = sqrt(s.x);
    }
    __syncthreads();
    nrm = nrm_s;
  }
  // Givens update (one thread per RHS); every CTA scales its chunk by
  // 1 / ||w|| (a frozen column's new vector is never read again).
  if (chunk == 0 && tid == 0) givens_step(c, q, j, nrm);
  const R sc = (nrm > 0.0 && isfinite(nrm)) ? (R)(1.0 / nrm) : (R)0;
#pragma unroll
  for (int t = 0; t < KEPT; ++t) {
    const int n = n0 + tid + KT * t;
    if (n < N) w[n] = cscale(wv[t], sc);
  }
}

// V[slot] *= inv_norm[q] (zero for frozen columns).
template <typename R>
__global__ void scale_kernel(KrylovCtl c, typename Cplx<R>::T *v, size_t vstride, int N, int nr) {
  const size_t total = (size_t)nr * N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx / N);
    v[idx] = cscale(v[idx], (decltype(v[0].x))c.inv_norm[q]);
  }
}

// y = R^{-1} g per RHS (FP64 back substitution on the rotated Hessenberg).
__global__ void backsolve_kernel(KrylovCtl c, int nr) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nr) return;
  const int m = c.m, k = c.kq[q];
  double2 *y = c.y + (size_t)q * m;
  const double2 *g = c.g + (size_t)q * (m + 1);
  for (int i = k - 1; i >= 0; --i) {
    double2 s = g[i];
    for (int jj = i + 1; jj < k; ++jj) s = csub(s, cmul(c.Rm[((size_t)q * m + jj) * (m + 1) + i], y[jj]));
    const double2 d = c.Rm[((size_t)q * m + i) * (m + 1) + i];
    const double den = d.x * d.x + d.y * d.y;
    y[i] = cscale(cmul(s, cconj(d)), 1.0 / den);
  }
}

// I[q] += scale[q] * sum_{i<kq} V[i][q] y[q][i]   (FP64 accumulation).
template <typename R>
__global__ void lincomb_kernel(KrylovCtl c, const typename Cplx<R>::T *V, size_t vstride, int N, int nr,
                               double2 *I, const double *scale) {
  const size_t total = (size_t)nr * N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx / N);
    const int k = c.kq[q];
    if (k == 0) continue;
    const double2 *y = c.y + (size_t)q * c.m;
    double2 s = make_double2(0, 0);
    for (int i = 0; i < k; ++i) s = cfma(cvt<double2>(V[(size_t)i * vstride + idx]), y[i], s);
    I[idx] = cadd(I[idx], cscale(s, scale[q]));
  }
}

// ---------------------------------------------------------------- FP64 ----
// r = V - y (y may be null: r = V); per-RHS ||r|| into out_norm; optional
// copy of r scaled by 1/||r|| happens in a second kernel.  Last-block
// reduction as above.
__global__ void __launch_bounds__(KT) resid_kernel(const double2 *V, const double2 *y, double2 *r, int N,
                                                   double *partial, unsigned *counters, double *out_norm) {
  __shared__ double2 red[8];
  __shared__ int last;
  const int q = blockIdx.y, chunk = blockIdx.x, tid = threadIdx.x;
  const size_t qoff = (size_t)q * N;
  const int n0 = chunk * KT * KEPT;
  double2 acc[1] = {make_double2(0, 0)};
#pragma unroll
  for (int t = 0; t < KEPT; ++t) {
    const int n = n0 + tid + KT * t;
    if (n < N) {
      double2 v = V[qoff + n];
      if (y) v = csub(v, y[qoff + n]);
      if (r) r[qoff + n] = v;
      acc[0].x += v.x * v.x + v.y * v.y;
    }
  }
  block_sum<double2, 1>(acc, red);
  if (tid == 0) partial[(size_t)q * gridDim.x + chunk] = acc[0].x;
  __threadfence();
  if (tid == 0) last = (atomicAdd(&counters[q], 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (tid < 32) {
    double s = 0;
    for (int ch = tid; ch < (int)gridDim.x; ch += 32) s += partial[(size_t)q * gridDim.x + ch];
    s = warp_sum(s);
    if (tid == 0) {
      out_norm[q] = sqrt(s);
      counters[q] = 0;
    }
  }
}

// dst[q] = src[q] / rnorm[q] in precision R, zero for columns with mask[q] == 0.
template <typename R>
__global__ void to_inner_kernel(const double2 *src, typename Cplx<R>::T *dst, int N, int nr, const double *rnorm,
                                const int *mask) {
  using C = typename Cplx<R>::T;
  const size_t total = (size_t)nr * N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx / N);
    dst[idx] = mask[q] ? cvt<C>(cscale(src[idx], 1.0 / rnorm[q])) : czero<C>();
  }
}

// Port quantities (Eqs. 16-19).
__global__ void ports_kernel(const double2 *I, const double2 *V, int nel, int b, int nr, int pb, double z0,
                             double2 *Za, double2 *Gam, unsigned *err, long long ldv) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nel * nr) return;
  const size_t at = (size_t)(idx / nel) * ldv + (size_t)(idx % nel) * b + pb;  // RHS q, element e
  const double2 ip = I[at];
  const double2 vp = V[at];
  const double den = ip.x * ip.x + ip.y * ip.y;
  double2 za;
  if (den == 0.0 || !isfinite(den)) {
    za = make_double2(nan(""), nan(""));
    atomicOr(err, DEVERR_NONFINITE);
  } else {
    za = cscale(cmul(vp, cconj(ip)), 1.0 / den);
  }
  Za[idx] = za;
  if (Gam) {
    const double2 num = make_double2(za.x - z0, za.y), dd = make_double2(za.x + z0, za.y);
    const double d2 = dd.x * dd.x + dd.y * dd.y;
    Gam[idx] = cscale(cmul(num, cconj(dd)), 1.0 / d2);
  }
}

static int grid_for(size_t total) {
  size_t g = (total + 255) / 256;
  if (g > 4096) g = 4096;
  return (int)(g < 1 ? 1 : g);
}

int krylov_chunks(int N) { return (N + KT * KEPT - 1) / (KT * KEPT); }

template <typename R>
void launch_cgs(const KrylovCtl &c, void *V, size_t vstride, int N, int nr, int j, int flags, cudaStream_t st) {
  dim3 grid(krylov_chunks(N), nr);
  cgs_kernel<R><<<grid, KT, 0, st>>>(c, reinterpret_cast<typename Cplx<R>::T *>(V), vstride, N, j, flags);
}
template <typename R>
void launch_scale(const KrylovCtl &c, void *v, size_t vstride, int N, int nr, cudaStream_t st) {
  scale_kernel<R><<<grid_for((size_t)nr * N), 256, 0, st>>>(c, reinterpret_cast<typename Cplx<R>::T *>(v), vstride,
                                                              N, nr);
}
void launch_backsolve(const KrylovCtl &c, int nr, cudaStream_t st) {
  backsolve_kernel<<<(nr + 63) / 64, 64, 0, st>>>(c, nr);
}
template <typename R>
void launch_lincomb(const KrylovCtl &c, const void *V, size_t vstride, int N, int nr, double2 *I,
                    const double *scale, cudaStream_t st) {
  lincomb_kernel<R><<<grid_for((size_t)nr * N), 256, 0, st>>>(
      c, reinterpret_cast<const typename Cplx<R>::T *>(V), vstride, N, nr, I, scale);
}
void launch_resid(const double2 *V, const double2 *y, double2 *r, int N, int nr, double *partial, unsigned *counters,
                  double *out_norm, cudaStream_t st) {
  dim3 grid(krylov_chunks(N), nr);
  resid_kernel<<<grid, KT, 0, st>>>(V, y, r, N, partial, counters, out_norm);
}
template <typename R>
void launch_to_inner(const double2 *src, void *dst, int N, int nr, const double *rnorm, const int *mask,
                     cudaStream_t st) {
  to_inner_kernel<R><<<grid_for((size_t)nr * N), 256, 0, st>>>(src, reinterpret_cast<typename Cplx<R>::T *>(dst), N,
                                                                 nr, rnorm, mask);
}
void launch_ports(const double2 *I, const double2 *V, int nel, int b, int nr, int pb, double z0, double2 *Za,
                  double2 *Gam, unsigned *err, long long ldv, cudaStream_t st) {
  ports_kernel<<<(nel * nr + 255) / 256, 256, 0, st>>>(I, V, nel, b, nr, pb, z0, Za, Gam, err, ldv);
}

template <typename R>
bool arnoldi_fused_fits(int N, int nr, int num_sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, arnoldi_fused_kernel<R>, KT, 0) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (long long)krylov_chunks(N) * nr <= (long long)per_sm * num_sms;
}
template <typename R>
void launch_arnoldi_fused(const KrylovCtl &c, void *V, size_t vstride, int N, int nr, int j, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(krylov_chunks(N), nr);
  cfg.blockDim = dim3(KT);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, arnoldi_fused_kernel<R>, c, reinterpret_cast<typename Cplx<R>::T *>(V), vstride, N, j);
}
template bool arnoldi_fused_fits<float>(int, int, int);
template bool arnoldi_fused_fits<double>(int, int, int);
template void launch_arnoldi_fused<float>(const KrylovCtl &, void *, size_t, int, int, int, cudaStream_t);
template void launch_arnoldi_fused<double>(const KrylovCtl &, void *, size_t, int, int, int, cudaStream_t);

template void launch_cgs<float>(const KrylovCtl &, void *, size_t, int, int, int, int, cudaStream_t);
template void launch_cgs<double>(const KrylovCtl &, void *, size_t, int, int, int, int, cudaStream_t);
template void launch_scale<float>(const KrylovCtl &, void *, size_t, int, int, cudaStream_t);
template void launch_scale<double>(const KrylovCtl &, void *, size_t, int, int, cudaStream_t);
template void launch_lincomb<float>(const KrylovCtl &, const void *, size_t, int, int, double2 *, const double *,
                                    cudaStream_t);
template void launch_lincomb<double>(const KrylovCtl &, const void *, size_t, int, int, double2 *, const double *,
                                     cudaStream_t);
template void launch_to_inner<float>(const double2 *, void *, int, int, const double *, const int *, cudaStream_t);
template void launch_to_inner<double>(const double2 *, void *, int, int, const double *, const int *, cudaStream_t);

}  // namespace moma

// ================================================================ PCG =====
// Preconditioned conjugate gradients on the normal equations
// Z^H Z d = Z^H r (Sec. II-C): Z^H Z is Hermitian positive definite and P
// (Eq. 38) is applied as the preconditioner M = P = L L^H, which is the
// split form P^{-1/2} Z^H Z P^{-H/2} of Sec. III-A in exact arithmetic.
// Only O(1) vectors per RHS are kept.  Inner products of c64 vectors are
// accumulated per thread in FP32 and across threads / CTAs in FP64, in a
// fixed order; the step lengths alpha, beta are FP64 device scalars.
namespace moma {

// cg_reduce computes out = Re(sum conj(a) b) per RHS; then, by mode:
//   CG_PQ : alpha = rz / pq       (frozen columns: alpha = 0)
//   CG_RZ : beta = rz_new / rz, rz = rz_new     (CG_RZ0: rz = rz_new, no beta)

template <typename R>
__global__ void __launch_bounds__(KT) cg_reduce_kernel(CgCtl c, const typename Cplx<R>::T *a,
                                                       const typename Cplx<R>::T *b, int N, int mode) {
  using C = typename Cplx<R>::T;
  __shared__ C red[8];
  __shared__ int last;
  const int q = blockIdx.y, chunk = blockIdx.x, tid = threadIdx.x;
  if (!c.active[q]) return;
  const size_t qoff = (size_t)q * N;
  const int n0 = chunk * KT * KEPT;
  C acc[1] = {czero<C>()};
#pragma unroll
  for (int t = 0; t < KEPT; ++t) {
    const int n = n0 + tid + KT * t;
    if (n < N) acc[0] = cfmac(a[qoff + n], b[qoff + n], acc[0]);
  }
  block_sum<C, 1>(acc, red);
  if (tid == 0) c.partial[(size_t)q * gridDim.x + chunk] = (double)acc[0].x;
  __threadfence();
  if (tid == 0) last = (atomicAdd(&c.counters[q], 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (tid < 32) {
    double s = 0;
    for (int ch = tid; ch < (int)gridDim.x; ch += 32) s += c.partial[(size_t)q * gridDim.x + ch];
    s = warp_sum(s);
    if (tid == 0) {
      if (mode == CG_PQ) {
        c.alpha[q] = (s > 0.0 && isfinite(s)) ? c.rz[q] / s : 0.0;
        if (!isfinite(s)) atomicOr(c.err, DEVERR_NONFINITE);
      } else {
        if (mode == CG_RZ) c.beta[q] = c.rz[q] != 0.0 ? s / c.rz[q] : 0.0;
        c.rz[q] = s;
      }
      c.counters[q] = 0;
    }
  }
}

// d += alpha p; r -= alpha q; then ||r||^2 -> stop test against tol^2 ||r0||^2
// (mode 0), or just ||r||^2 into rr0 (mode 1, initialisation).
template <typename R>
__global__ void __launch_bounds__(KT) cg_axpy_kernel(CgCtl c, typename Cplx<R>::T *d, const typename Cplx<R>::T *p,
                                                     typename Cplx<R>::T *r, const typename Cplx<R>::T *qv, int N,
                                                     int init) {
  using C = typename Cplx<R>::T;
  using RT = decltype(C{}.x);
  __shared__ C red[8];
  __shared__ int last;
  const int q = blockIdx.y, chunk = blockIdx.x, tid = threadIdx.x;
  if (!c.active[q]) return;
  const size_t qoff = (size_t)q * N;
  const int n0 = chunk * KT * KEPT;
  const RT al = init ? (RT)0 : (RT)c.alpha[q];
  C acc[1] = {czero<C>()};
#pragma unroll
  for (int t = 0; t < KEPT; ++t) {
    const int n = n0 + tid + KT * t;
    if (n < N) {
      C rv = r[qoff + n];
      if (!init) {
        d[qoff + n] = cadd(d[qoff + n], cscale(p[qoff + n], al));
        rv = csub(rv, cscale(qv[qoff + n], al));
        r[qoff + n] = rv;
      }
      acc[0].x += rv.x * rv.x + rv.y * rv.y;
    }
  }
  block_sum<C, 1>(acc, red);
  if (tid == 0) c.partial[(size_t)q * gridDim.x + chunk] = (double)acc[0].x;
  __threadfence();
  if (tid == 0) last = (atomicAdd(&c.counters[q], 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (tid < 32) {
    double s = 0;
    for (int ch = tid; ch < (int)gridDim.x; ch += 32) s += c.partial[(size_t)q * gridDim.x + ch];
    s = warp_sum(s);
    if (tid == 0) {
      if (init) {
        c.rr0[q] = s;
        if (!(s > 0.0) || !isfinite(s)) {  // nothing to solve (or bad input)
          if (!isfinite(s)) atomicOr(c.err, DEVERR_NONFINITE);
          c.active[q] = 0;
          atomicSub(c.nact, 1);
        }
      } else {
        c.rr[q] = s;
        c.iters[q] += 1;
        if (!isfinite(s)) {
          atomicOr(c.err, DEVERR_NONFINITE);
          c.active[q] = 0;
          atomicSub(c.nact, 1);
        } else if (s <= c.tol2 * c.rr0[q]) {
          c.active[q] = 0;
          atomicSub(c.nact, 1);
        }
      }
      c.counters[q] = 0;
    }
  }
}

// p = z + beta p (or p = z when init).
template <typename R>
__global__ void cg_dir_kernel(CgCtl c, typename Cplx<R>::T *p, const typename Cplx<R>::T *z, int N, int nr,
                              int init) {
  using C = typename Cplx<R>::T;
  using RT = decltype(C{}.x);
  const size_t total = (size_t)nr * N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx / N);
    if (!c.active[q]) continue;
    p[idx] = init ? z[idx] : cadd(z[idx], cscale(p[idx], (RT)c.beta[q]));
  }
}

// I += scale[q] * d (FP64 accumulation of the c64 correction).
template <typename R>
__global__ void cg_accum_kernel(const typename Cplx<R>::T *d, int N, int nr, double2 *I, const double *scale) {
  const size_t total = (size_t)nr * N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx / N);
    I[idx] = cadd(I[idx], cscale(cvt<double2>(d[idx]), scale[q]));
  }
}

template <typename R>
void launch_cg_reduce(const CgCtl &c, const void *a, const void *b, int N, int nr, int mode, cudaStream_t st) {
  using C = typename Cplx<R>::T;
  dim3 grid(krylov_chunks(N), nr);
  cg_reduce_kernel<R><<<grid, KT, 0, st>>>(c, reinterpret_cast<const C *>(a), reinterpret_cast<const C *>(b), N,
                                           mode);
}
template <typename R>
void launch_cg_axpy(const CgCtl &c, void *d, const void *p, void *r, const void *q, int N, int nr, int init,
                    cudaStream_t st) {
  using C = typename Cplx<R>::T;
  dim3 grid(krylov_chunks(N), nr);
  cg_axpy_kernel<R><<<grid, KT, 0, st>>>(c, reinterpret_cast<C *>(d), reinterpret_cast<const C *>(p),
                                         reinterpret_cast<C *>(r), reinterpret_cast<const C *>(q), N, init);
}
template <typename R>
void launch_cg_dir(const CgCtl &c, void *p, const void *z, int N, int nr, int init, cudaStream_t st) {
  using C = typename Cplx<R>::T;
  cg_dir_kernel<R><<<grid_for((size_t)nr * N), 256, 0, st>>>(c, reinterpret_cast<C *>(p),
                                                              reinterpret_cast<const C *>(z), N, nr, init);
}
template <typename R>
void launch_cg_accum(const void *d, int N, int nr, double2 *I, const double *scale, cudaStream_t st) {
  using C = typename Cplx<R>::T;
  cg_accum_kernel<R><<<grid_for((size_t)nr * N), 256, 0, st>>>(reinterpret_cast<const C *>(d), N, nr, I, scale);
}

template void launch_cg_reduce<float>(const CgCtl &, const void *, const void *, int, int, int, cudaStream_t);
template void launch_cg_reduce<double>(const CgCtl &, const void *, const void *, int, int, int, cudaStream_t);
template void launch_cg_axpy<float>(const CgCtl &, void *, const void *, void *, const void *, int, int, int,
                                    cudaStream_t);
template void launch_cg_axpy<double>(const CgCtl &, void *, const void *, void *, const void *, int, int, int,
                                     cudaStream_t);
template void launch_cg_dir<float>(const CgCtl &, void *, const void *, int, int, int, cudaStream_t);
template void launch_cg_dir<double>(const CgCtl &, void *, const void *, int, int, int, cudaStream_t);
template void launch_cg_accum<float>(const void *, int, int, double2 *, const double *, cudaStream_t);
template void launch_cg_accum<double>(const void *, int, int, double2 *, const double *, cudaStream_t);

}  // namespace moma
