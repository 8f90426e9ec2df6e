// Block-diagonal preconditioner of the normal equations (Sec. III-A).
//
// Eq. 37: the diagonal block of element e is
//     P_e = sum_j (Z_{j,e})^H Z_{j,e} = sum_{D in W(e)} G_D,   G_D = Z_D^H Z_D,
// where D = j - e runs over the offsets that keep j inside the lattice:
// W(e) = [-ex, Nx-1-ex] x [-ey, Ny-1-ey].  Following the paper's recipe
// (precompute all block products, then sum subsets), G is formed once per
// offset and the box sums P_e are two passes of sliding windows over the
// offset grid (rows, then columns), so the cost is O((2Nx-1)(2Ny-1) b^3)
// for the products and O(Nx Ny b^2) per pass instead of O(Nel^2 b^3).
// P_e = L_e L_e^H by Cholesky in FP64 (Sec. III-A), and P^{-1} is applied
// as X_e^H X_e with X_e = L_e^{-1} stored packed.
#include <algorithm>
#include <type_traits>

#include "internal.h"

namespace moma {

// ------------------------------------------------------------- Gram ------
// G_D[i][j] = sum_k conj(Z_D[k][i]) Z_D[k][j]; 64 x 64 output tile per CTA,
// 16 x 16 threads with 4 x 4 micro-tiles, k staged in chunks of 16.
constexpr int GT = 64, GK = 16;

template <typename R, typename Cin>
__global__ void __launch_bounds__(256) gram_kernel(const Cin *__restrict__ blocks, int b, double2 *__restrict__ G) {
  using C = typename Cplx<R>::T;
  __shared__ C As[GK][GT];
  __shared__ C Bs[GK][GT];
  const int D = blockIdx.z;
  const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
  const Cin *Zd = blocks + (size_t)D * b * b;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  C acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = czero<C>();

  for (int k0 = 0; k0 < b; k0 += GK) {
    for (int idx = threadIdx.x; idx < GK * GT; idx += 256) {
      const int kk = idx / GT, cc = idx % GT;
      const int k = k0 + kk;
      As[kk][cc] = (k < b && i0 + cc < b) ? cvt<C>(Zd[(size_t)k * b + i0 + cc]) : czero<C>();
      Bs[kk][cc] = (k < b && j0 + cc < b) ? cvt<C>(Zd[(size_t)k * b + j0 + cc]) : czero<C>();
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      C av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = cfmac(av[a], bv[c], acc[a][c]);
    }
    __syncthreads();
  }
  double2 *Gd = G + (size_t)D * b * b;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * c;
      if (i < b && j < b) Gd[(size_t)i * b + j] = cvt<double2>(acc[a][c]);
    }
}

template <typename R>
void launch_gram(const void *blocks, int blocks_c128, int nD, int b, double2 *G, cudaStream_t st) {
  dim3 grid((b + GT - 1) / GT, (b + GT - 1) / GT, nD);
  if (blocks_c128)
    gram_kernel<R, double2><<<grid, 256, 0, st>>>(reinterpret_cast<const double2 *>(blocks), b, G);
  else
    gram_kernel<R, float2><<<grid, 256, 0, st>>>(reinterpret_cast<const float2 *>(blocks), b, G);
}
template void launch_gram<float>(const void *, int, int, int, double2 *, cudaStream_t);
template void launch_gram<double>(const void *, int, int, int, double2 *, cudaStream_t);

// ------------------------------------------------------- box + Cholesky ---
// One CTA per element.  The lower triangle of P_e is loaded from the box
// sums (row by row, contiguous) into the packed column-major layout and
// factored by a blocked right-looking Cholesky over panels of CH_NB
// columns, three CTA barriers per panel: (1) one warp factors the panel's
// CH_NB x CH_NB diagonal block column by column (warp synchronisation
// only); (2) every row below it is solved against that block by its own
// thread (L21 = A21 L11^{-H}); (3) the trailing triangle receives the
// rank-CH_NB update A(i,k) -= sum_p L(i,p) conj(L(k,p)) in one sweep.
// The sweep is register-tiled: a thread owns a 2 x 2 tile of (i, k) entries
// (rows i0, i0 + 1; columns k0, k0 + 1), so each of the panel's values it
// loads serves two multiply-adds; tile t of the trailing triangle (row-major
// enumeration of tile rows ti >= tile columns tk) is found from t by a
// square root, so no index table is kept.  A diagonal tile skips its entry
// above the diagonal; the last tile row of an odd trailing size has one row.
// L_e (packed column-major) is written to Lpk.
constexpr int CH_NB = 8;

MOMA_HD int colbase(int k, int b) { return k * b - k * (k - 1) / 2; }  // start of column k (packed)
// Column k of packed column-major entry t: colbase(k) <= t < colbase(k + 1).
MOMA_DEV int packed_col(int t, int b) {
  const float c = (float)(2 * b + 1);
  int k = (int)((c - sqrtf(c * c - 8.0f * (float)t)) * 0.5f);
  k = max(0, min(k, b - 1));
  while (k > 0 && colbase(k, b) > t) --k;
  while (k + 1 < b && colbase(k + 1, b) <= t) ++k;
  return k;
}

// Arithmetic R: double (plain path) or dfl, double-FP32 pairs of ~48 bits
// (mixed path, where B300's FP64 rate would bound the factorisation; the
// factor only has to be an accurate preconditioner, and it is stored FP64).
MOMA_DEV double real_part(double2 v) { return v.x; }
MOMA_DEV double real_part(dfl2 v) { return (double)v.x; }
MOMA_DEV double rsqrt_root(double d, double *l) { *l = sqrt(d); return 1.0 / *l; }
MOMA_DEV dfl rsqrt_root(dfl d, dfl *l) { *l = dsqrt(d); return dfl(1.0f) / *l; }

// acc -= a conj(b) (the Cholesky update term), on the real and imaginary parts.
MOMA_DEV void dfacc_fms_conj(DfAcc &re, DfAcc &im, const dfl2 &a, const dfl2 &b) {
  dfacc_fma(re, -a.x, b.x);
  dfacc_fma(re, -a.y, b.y);
  dfacc_fma(im, -a.y, b.x);
  dfacc_fma(im, a.x, b.y);
}

// ---------------------------------------------------------------- box sums --
// P_e = sum of G_D over the offsets of the element's box (Eq. 37): offset
// indices x' in [Nx-1-ex, 2Nx-2-ex], y' in [Ny-1-ey, 2Ny-2-ey] of the
// (2Ny-1) x (2Nx-1) grid.  Separable sliding windows: first the row windows
// R[y'][ex] = sum over the x' window (one pass over each row of G, each
// step adding the offset entering the window and subtracting the one
// leaving it), then P[ey][ex] = the same over y' of R.  Only the lower
// triangle is formed (P_e is Hermitian): entry t = i (i + 1) / 2 + k,
// i >= k, row-major, taken from position i b + k of the b x b blocks, so
// consecutive threads read consecutive entries of a block row.
// G_D comes either from S (FP64, [D][b][b]) or, for the tensor-core Gram
// products of the reflected offsets, as conj(Y_{-D}) (c64).  The sums run
// in FP64 (ACC = double) or, for the c64 products, in double-FP32 (ACC =
// dfl: B300's FP64 rate would bound the pass), stored as pairs; P_e is
// written in the precision of the factorisation that reads it (OUT =
// double2 or dfl2).
MOMA_DEV int tri_row(int t) {  // row i of row-major lower-triangle entry t
  int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while (i * (i + 1) / 2 > t) --i;
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  return i;
}

// Running sums of complex terms: FP64, or double-FP32 accumulators whose
// additions are exact two-sums (errors gathered in the low part) and which
// are renormalised at every output.
struct WinD {
  double2 v = make_double2(0, 0);
  MOMA_DEV void add(double2 a) { v = cadd(v, a); }
  MOMA_DEV void sub(double2 a) { v = csub(v, a); }
  MOMA_DEV void add(float2 a) { v = cadd(v, make_double2(a.x, a.y)); }
  MOMA_DEV void sub(float2 a) { v = csub(v, make_double2(a.x, a.y)); }
  MOMA_DEV double2 out() const { return v; }
};
struct WinF {
  DfAcc re{0.f, 0.f}, im{0.f, 0.f};
  MOMA_DEV static void acc(DfAcc &a, float x) {
    const dfl q = df_two_sum(a.s, x);
    a.s = q.hi;
    a.t = __fadd_rn(a.t, q.lo);
  }
  MOMA_DEV void add(float2 a) { acc(re, a.x); acc(im, a.y); }
  MOMA_DEV void sub(float2 a) { acc(re, -a.x); acc(im, -a.y); }
  MOMA_DEV void add(const dfl2 &a) {
    acc(re, a.x.hi); re.t = __fadd_rn(re.t, a.x.lo);
    acc(im, a.y.hi); im.t = __fadd_rn(im.t, a.y.lo);
  }
  MOMA_DEV void sub(const dfl2 &a) {
    acc(re, -a.x.hi); re.t = __fsub_rn(re.t, a.x.lo);
    acc(im, -a.y.hi); im.t = __fsub_rn(im.t, a.y.lo);
  }
  MOMA_DEV dfl2 out() {
    const dfl r = df_fast_two_sum(re.s, re.t), i = df_fast_two_sum(im.s, im.t);
    re = DfAcc{r.hi, r.lo};
    im = DfAcc{i.hi, i.lo};
    return dfl2{r, i};
  }
};
template <typename ACC> struct WinOf;
template <> struct WinOf<double> { using W = WinD; using T = double2; };
template <> struct WinOf<dfl> { using W = WinF; using T = dfl2; };

template <bool REFL, typename ACC>
__global__ void box_rows_kernel(const double2 *__restrict__ S, const float2 *__restrict__ Y,
                                typename WinOf<ACC>::T *__restrict__ R, int nx, int ndy, int b) {
  const int npk = b * (b + 1) / 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npk) return;
  const int y = blockIdx.y, ndx = 2 * nx - 1, i = tri_row(t), k = t - i * (i + 1) / 2;
  const size_t bb = (size_t)b * b, ent = (size_t)i * b + k;
  auto G = [&](int x) {
    if constexpr (REFL) {
      const float2 g = Y[((size_t)(ndy - 1 - y) * ndx + (ndx - 1 - x)) * bb + ent];
      return make_float2(g.x, -g.y);
    } else {
      return S[((size_t)y * ndx + x) * bb + ent];
    }
  };
  typename WinOf<ACC>::W run;
  // Unrolled so that several independent loads are in flight ahead of the
  // dependent additions.
#pragma unroll 8
  for (int x = nx - 1; x <= 2 * nx - 2; ++x) run.add(G(x));
  auto *out = R + (size_t)y * nx * npk + t;
  out[0] = run.out();
#pragma unroll 8
  for (int ex = 1; ex < nx; ++ex) {  // window [nx-1-ex, 2nx-2-ex]
    run.add(G(nx - 1 - ex));
    run.sub(G(2 * nx - 1 - ex));
    out[(size_t)ex * npk] = run.out();
  }
}

template <typename ACC, typename OUT>
__global__ void box_cols_kernel(const typename WinOf<ACC>::T *__restrict__ R, OUT *__restrict__ Pbox, int nx, int ny,
                                int b) {
  const int npk = b * (b + 1) / 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npk) return;
  const int ex = blockIdx.y;
  auto Rv = [&](int y) { return R[((size_t)y * nx + ex) * npk + t]; };
  typename WinOf<ACC>::W run;
#pragma unroll 8
  for (int y = ny - 1; y <= 2 * ny - 2; ++y) run.add(Rv(y));
  Pbox[(size_t)ex * npk + t] = cvt<OUT>(run.out());
#pragma unroll 8
  for (int ey = 1; ey < ny; ++ey) {  // window [ny-1-ey, 2ny-2-ey]
    run.add(Rv(ny - 1 - ey));
    run.sub(Rv(2 * ny - 1 - ey));
    Pbox[((size_t)ey * nx + ex) * npk + t] = cvt<OUT>(run.out());
  }
}

size_t box_window_entries(int nx, int ny, int b) {
  return ((size_t)(2 * ny - 1) * nx + (size_t)nx * ny) * ((size_t)b * (b + 1) / 2);
}

template <bool REFL, typename ACC>
static void box_sums_typed(const double2 *S, const float2 *Y, int nx, int ny, int b, double2 *W, bool df,
                           cudaStream_t st) {
  using T = typename WinOf<ACC>::T;
  static_assert(sizeof(T) == sizeof(double2), "window sums are 16-byte complex values");
  const int npk = b * (b + 1) / 2, ndy = 2 * ny - 1;
  T *R = reinterpret_cast<T *>(W);
  double2 *P = W + (size_t)ndy * nx * npk;
  const dim3 g1((npk + 255) / 256, ndy), g2((npk + 255) / 256, nx);
  box_rows_kernel<REFL, ACC><<<g1, 256, 0, st>>>(S, Y, R, nx, ndy, b);
  if (df) box_cols_kernel<ACC, dfl2><<<g2, 256, 0, st>>>(R, reinterpret_cast<dfl2 *>(P), nx, ny, b);
  else box_cols_kernel<ACC, double2><<<g2, 256, 0, st>>>(R, P, nx, ny, b);
}

void launch_box_sums(const double2 *S, const float2 *Y, int nx, int ny, int b, double2 *W, bool df, cudaStream_t st) {
  if (Y) box_sums_typed<true, dfl>(S, Y, nx, ny, b, W, df, st);
  else box_sums_typed<false, double>(S, Y, nx, ny, b, W, df, st);
}

const double2 *box_sums_of(const double2 *W, int nx, int ny, int b) {
  return W + (size_t)(2 * ny - 1) * nx * ((size_t)b * (b + 1) / 2);
}

// The packed lower triangle of columns j0 .. b-1 of a b x b matrix,
// column-major: entry (i, k), k >= j0, at col(k)[i].  j0 = 0 is the whole
// matrix; the trailing triangle of a hybrid factorisation lives in shared
// memory with its own, smaller column bases.
template <typename C>
struct Tri {
  C *base;
  int j0, n;  // first column, order n = b - j0
  MOMA_DEV int off(int k) const { return colbase(k - j0, n) - k; }
  MOMA_DEV C *col(int k) const { return base + off(k); }
};

// Panels jb = jfirst, jfirst + CH_NB, ... < jlast of the blocked
// right-looking factorisation on T (every column from jfirst on lives in
// T).  Returns false (after setting DEVERR_NOT_PD) if a pivot is not
// positive.
template <typename R, typename C>
MOMA_DEV bool chol_panels(const Tri<C> T, int b, int jfirst, int jlast, R *inv_diag, int *not_pd, unsigned *err) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int jb = jfirst; jb < jlast; jb += CH_NB) {
    const int je = min(jb + CH_NB, b);
    // (1) Diagonal block A(jb:je, jb:je), unblocked, by warp 0 alone (warp
    // synchronisation only): column j is scaled by 1 / L(j, j) and the
    // block's remaining lower entries (i, k), j < k <= i < je -- at most 28,
    // one per lane -- receive -L(i, j) conj(L(k, j)).
    if (w == 0) {
      for (int j = jb; j < je; ++j) {
        C *cj = T.col(j);  // cj[i] = A(i, j), i >= j
        const double d = real_part(cj[j]);
        if (!(d > 0.0) || !isfinite(d)) {  // uniform over the warp: every lane reads the same value
          if (lane == 0) *not_pd = 1;
          break;
        }
        R l;
        const R inv_l = rsqrt_root(cj[j].x, &l);
        __syncwarp();  // every lane has read A(j, j) before it is overwritten
        if (lane == 0) {
          cj[j] = mk(l, (R)0);
          inv_diag[j - jb] = inv_l;
        }
        if (lane < je - j - 1) cj[j + 1 + lane] = cscale(cj[j + 1 + lane], inv_l);
        __syncwarp();
        const int m = je - j - 1;
        if (lane < m * (m + 1) / 2) {
          int kk = 0, r = lane;
          while (r >= m - kk) {
            r -= m - kk;
            ++kk;
          }
          const int k = j + 1 + kk, i = k + r;
          C *ck = T.col(k);
          ck[i] = cfms_conj(cj[i], cj[k], ck[i]);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (*not_pd) {
      if (tid == 0) atomicOr(err, DEVERR_NOT_PD);
      return false;
    }
    // (2) Rows below the block, one thread each: row i of L21 solves
    // x L11^H = A(i, jb:je), x_k = (A(i, jb+k) - sum_{p<k} x_p conj(L(jb+k, jb+p))) / L(jb+k, jb+k).
    const int np = je - jb;
    for (int i = je + tid; i < b; i += blockDim.x) {
      // x_p (p < k) are read back from the row, where this thread stored them.
#pragma unroll 1
      for (int k = 0; k < np; ++k) {
        C *ck = T.col(jb + k);
        C v = ck[i];
        if constexpr (std::is_same<R, dfl>::value) {
          DfAcc re = dfacc(v.x), im = dfacc(v.y);
          for (int p = 0; p < k; ++p) dfacc_fms_conj(re, im, T.col(jb + p)[i], T.col(jb + p)[jb + k]);
          v = mk(dfacc_value(re), dfacc_value(im));
        } else {
          for (int p = 0; p < k; ++p) v = cfms_conj(T.col(jb + p)[i], T.col(jb + p)[jb + k], v);
        }
        ck[i] = cscale(v, inv_diag[k]);
      }
    }
    __syncthreads();
    // (3) Trailing rank-(je - jb) update in 2 x 2 register tiles.
    int pb[CH_NB];
#pragma unroll
    for (int p = 0; p < CH_NB; ++p) pb[p] = p < np ? T.off(jb + p) : 0;
    const int nt = (b - je + 1) / 2, ntiles = nt * (nt + 1) / 2;
    for (int t = tid; t < ntiles; t += blockDim.x) {
      int ti = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
      while (ti * (ti + 1) / 2 > t) --ti;
      while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
      const int tk = t - ti * (ti + 1) / 2;
      const int i0 = je + 2 * ti, k0 = je + 2 * tk;
      const bool r1 = i0 + 1 < b;    // second row present
      const bool up = ti != tk;      // (i0, k0 + 1) lies on or below the diagonal
      C *c0 = T.col(k0);
      C *c1 = T.col(k0 + 1);  // dereferenced only where k0 + 1 <= i < b
      C a00 = c0[i0];
      C a10 = r1 ? c0[i0 + 1] : czero<C>();
      C a01 = up ? c1[i0] : czero<C>();
      C a11 = r1 ? c1[i0 + 1] : czero<C>();
      if constexpr (std::is_same<R, dfl>::value) {
        DfAcc r00 = dfacc(a00.x), j00 = dfacc(a00.y), r10 = dfacc(a10.x), j10 = dfacc(a10.y);
        DfAcc r01 = dfacc(a01.x), j01 = dfacc(a01.y), r11 = dfacc(a11.x), j11 = dfacc(a11.y);
#pragma unroll
        for (int p = 0; p < CH_NB; ++p) {
          if (p < np) {
            const C *lp = T.base + pb[p];
            const C li0 = lp[i0], lk0 = lp[k0];
            const C li1 = r1 ? lp[i0 + 1] : czero<C>();
            const C lk1 = (up || r1) ? lp[k0 + 1] : czero<C>();
            dfacc_fms_conj(r00, j00, li0, lk0);
            dfacc_fms_conj(r10, j10, li1, lk0);
            dfacc_fms_conj(r01, j01, li0, lk1);
            dfacc_fms_conj(r11, j11, li1, lk1);
          }
        }
        a00 = mk(dfacc_value(r00), dfacc_value(j00));
        a10 = mk(dfacc_value(r10), dfacc_value(j10));
        a01 = mk(dfacc_value(r01), dfacc_value(j01));
        a11 = mk(dfacc_value(r11), dfacc_value(j11));
      } else {
#pragma unroll
        for (int p = 0; p < CH_NB; ++p) {
          if (p < np) {
            const C *lp = T.base + pb[p];
            const C li0 = lp[i0], lk0 = lp[k0];
            const C li1 = r1 ? lp[i0 + 1] : czero<C>();
            const C lk1 = (up || r1) ? lp[k0 + 1] : czero<C>();
            a00 = cfms_conj(li0, lk0, a00);
            a10 = cfms_conj(li1, lk0, a10);
            a01 = cfms_conj(li0, lk1, a01);
            a11 = cfms_conj(li1, lk1, a11);
          }
        }
      }
      c0[i0] = a00;
      if (r1) {
        c0[i0 + 1] = a10;
        c1[i0 + 1] = a11;
      }
      if (up) c1[i0] = a01;
    }
    __syncthreads();
  }
  return true;
}

// One CTA per element.  Columns 0 .. j0-1 are factored with the matrix in
// global memory (the element's Lpk slot, in the working precision), the
// rest with the trailing triangle of order b - j0 in shared memory: j0 is
// the smallest panel boundary at which that triangle fits the launch's
// shared-memory budget, chosen so that MINB CTAs share an SM (j0 = 0: the
// whole factorisation in shared memory; j0 = b: none of it).
template <typename R, int MINB>
__global__ void __launch_bounds__(MINB == 4 ? 256 : 512, MINB) box_cholesky_kernel(const double2 *__restrict__ Pbox, int b, int j0,
                                                                 double2 *__restrict__ Lpk, unsigned *err) {
  using C = typename Cplx<R>::T;
  static_assert(sizeof(C) == sizeof(double2), "the factor is stored in place of its FP64 output");
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ R inv_diag[CH_NB];  // 1 / L(j, j) of the current panel
  __shared__ int not_pd;
  const int e = blockIdx.x, tid = threadIdx.x;
  const int npk = b * (b + 1) / 2, n0 = b - j0;
  C *Ag = reinterpret_cast<C *>(Lpk + (size_t)e * npk);
  C *As = reinterpret_cast<C *>(smraw);
  const Tri<C> Tg{Ag, 0, b}, Ts{As, j0, n0};
  if (tid == 0) not_pd = 0;

  // Load P_e (row-major lower triangle): columns < j0 into global memory,
  // the rest into shared memory (into global memory as well while the
  // first panels still update them).
  const C *src = reinterpret_cast<const C *>(Pbox) + (size_t)e * npk;  // stored in the working precision
  for (int t0 = tid; t0 < npk; t0 += 8 * blockDim.x) {  // batches of 8 loads in flight per thread
    C v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t0 + u * blockDim.x;
      v[u] = t < npk ? src[t] : czero<C>();
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t0 + u * blockDim.x;
      if (t < npk) {
        const int i = tri_row(t), k = t - i * (i + 1) / 2;
        if (j0 > 0) Tg.col(k)[i] = v[u];
        else Ts.col(k)[i] = v[u];
      }
    }
  }
  __syncthreads();
  if (j0 > 0) {
    if (!chol_panels<R>(Tg, b, 0, j0, inv_diag, &not_pd, err)) return;
    if (j0 < b) {  // move the trailing triangle into shared memory
      for (int q = tid; q < n0 * (n0 + 1) / 2; q += blockDim.x) {
        int kk = 0;  // column of packed entry q of the order-n0 triangle
        while (colbase(kk + 1, n0) <= q) ++kk;
        const int k = j0 + kk, i = k + (q - colbase(kk, n0));
        Ts.col(k)[i] = Tg.col(k)[i];
      }
      __syncthreads();
    }
  }
  if (j0 < b && !chol_panels<R>(Ts, b, j0, b, inv_diag, &not_pd, err)) return;
  // FP64 output: the global-memory columns in place (each thread converts
  // the entries it reads), the shared-memory triangle copied out.
  double2 *dst = Lpk + (size_t)e * npk;
  for (int t = tid; t < npk; t += blockDim.x) {  // packed column-major, coalesced
    const int k = packed_col(t, b), i = k + t - colbase(k, b);
    dst[t] = cvt<double2>(k < j0 ? Tg.col(k)[i] : Ts.col(k)[i]);
  }
}

template <typename R>
static void launch_chol_typed(const double2 *Pbox, int nel, int b, double2 *Lpk, unsigned *err, cudaStream_t st) {
  // Four CTAs of 256 threads per SM where the trailing triangle fits 54 KB
  // of shared memory with at most half the columns factored in global
  // memory (b <= 128: one element's serial panel work overlaps three
  // others' trailing updates); else two CTAs of 512 threads where it fits
  // 110 KB; else one CTA with up to 210 KB.
  constexpr size_t kQuarter = 54 * 1024, kHalf = 110 * 1024, kWhole = 210 * 1024;
  auto tri_bytes = [](int n) { return (size_t)n * (n + 1) / 2 * sizeof(double2); };
  static int configured = 0;
  if (!configured) {
    cudaFuncSetAttribute(box_cholesky_kernel<R, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQuarter);
    cudaFuncSetAttribute(box_cholesky_kernel<R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHalf);
    cudaFuncSetAttribute(box_cholesky_kernel<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWhole);
    configured = 1;
  }
  int jq = 0;
  while (jq < b && tri_bytes(b - jq) > kQuarter) jq += CH_NB;
  if (jq < b && 2 * jq <= b) {
    box_cholesky_kernel<R, 4><<<nel, 256, tri_bytes(b - jq), st>>>(Pbox, b, jq, Lpk, err);
    return;
  }
  int j0 = 0;
  while (j0 < b && tri_bytes(b - j0) > kHalf) j0 += CH_NB;
  if (j0 < b && j0 <= 2 * CH_NB) {
    box_cholesky_kernel<R, 2><<<nel, 512, tri_bytes(b - j0), st>>>(Pbox, b, j0, Lpk, err);
    return;
  }
  j0 = 0;
  while (j0 < b && tri_bytes(b - j0) > kWhole) j0 += CH_NB;
  box_cholesky_kernel<R, 1><<<nel, 512, j0 < b ? tri_bytes(b - j0) : 0, st>>>(Pbox, b, j0, Lpk, err);
}

void launch_box_cholesky(const double2 *Pbox, int nel, int b, double2 *Lpk, unsigned *err, bool df, cudaStream_t st) {
  if (df) launch_chol_typed<dfl>(Pbox, nel, b, Lpk, err, st);
  else launch_chol_typed<double>(Pbox, nel, b, Lpk, err, st);
}

// Full P_e (b x b, FP64) of one element from its lower triangle (debug /
// inspection): the upper entries are the conjugates of their mirrors.
template <typename T>
__global__ void box_one_kernel(const T *Pe, int b, double2 *out) {
  for (int ent = blockIdx.x * blockDim.x + threadIdx.x; ent < b * b; ent += gridDim.x * blockDim.x) {
    const int i = ent / b, k = ent % b;
    const double2 v = cvt<double2>(Pe[i >= k ? i * (i + 1) / 2 + k : k * (k + 1) / 2 + i]);
    out[ent] = i >= k ? v : cconj(v);
  }
}
void launch_box_one(const double2 *Pbox, int nx, int b, int ex, int ey, bool df, double2 *out, cudaStream_t st) {
  const size_t off = ((size_t)ey * nx + ex) * ((size_t)b * (b + 1) / 2);
  const int grid = (b * b + 255) / 256;
  if (df) box_one_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const dfl2 *>(Pbox) + off, b, out);
  else box_one_kernel<<<grid, 256, 0, st>>>(Pbox + off, b, out);
}

// ---------------------------------------------------- inverse factor -----
// X = L^{-1}, one column per warp: column k solves L x = e_k by forward
// substitution in axpy form -- at step m the lane holding row m finishes
// x_m = x_m / L_mm, broadcasts it, and every lane updates its rows i > m
// with column m of L (contiguous in the packed column-major layout).  L is
// staged in shared memory in precision R when it fits (b <= 160 in c64,
// b <= 128 in c128); larger blocks read their columns from global memory
// (FP64, L2-resident while the CTA works on them).  x lives in registers
// (lane owns rows lane + 32u).  X is written packed column-major, so the
// column store is coalesced.
template <typename R, int U, bool L_IN_SMEM>
__global__ void __launch_bounds__(256) tri_inverse_kernel(const double2 *__restrict__ Lpk, int b,
                                                          typename Cplx<R>::T *X, size_t x_stride) {
  using C = typename Cplx<R>::T;
  extern __shared__ __align__(16) unsigned char smraw[];
  R *inv_d = reinterpret_cast<R *>(smraw);  // [b] 1 / L(m, m)
  C *Ls = reinterpret_cast<C *>(smraw + (((size_t)b * sizeof(R) + 15) & ~size_t(15)));
  const int e = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const size_t npk = (size_t)b * (b + 1) / 2;
  const double2 *Le = Lpk + (size_t)e * npk;
  C *Xe = X + (size_t)e * x_stride;
  if (L_IN_SMEM)
    for (size_t q = threadIdx.x; q < npk; q += blockDim.x) Ls[q] = cvt<C>(Le[q]);
  for (int m = threadIdx.x; m < b; m += blockDim.x) inv_d[m] = (R)(1.0 / Le[(size_t)colbase(m, b)].x);
  for (size_t q = npk + threadIdx.x; q < x_stride; q += blockDim.x) Xe[q] = czero<C>();  // pad
  __syncthreads();
  auto Lat = [&](size_t q) -> C { return L_IN_SMEM ? Ls[q] : cvt<C>(__ldg(Le + q)); };
  // Two columns per warp at a time (k and k + nw), interleaved so that
  // their independent substitution chains overlap.
  for (int k1 = w; k1 < b; k1 += 2 * nw) {
    const int k2 = k1 + nw;
    const bool has2 = k2 < b;
    C x1[U], x2[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      x1[u] = (lane + 32 * u == k1) ? mk((R)1, (R)0) : czero<C>();
      x2[u] = (has2 && lane + 32 * u == k2) ? mk((R)1, (R)0) : czero<C>();
    }
#pragma unroll
    for (int u0 = 0; u0 < U; ++u0) {
      for (int lm = 0; lm < 32; ++lm) {
        const int m = 32 * u0 + lm;
        if (m >= b) break;
        if (m < k1) continue;
        const size_t cb = (size_t)colbase(m, b) - m;  // L(i, m) at cb + i
        const R idm = inv_d[m];
        if (lane == lm) {
          x1[u0] = cscale(x1[u0], idm);
          x2[u0] = cscale(x2[u0], idm);
        }
        C xm1, xm2;
        xm1.x = __shfl_sync(0xffffffffu, x1[u0].x, lm);
        xm1.y = __shfl_sync(0xffffffffu, x1[u0].y, lm);
        xm2.x = __shfl_sync(0xffffffffu, x2[u0].x, lm);
        xm2.y = __shfl_sync(0xffffffffu, x2[u0].y, lm);
        const bool use2 = has2 && m >= k2;
#pragma unroll
        for (int u = u0; u < U; ++u) {
          const int i = lane + 32 * u;
          if (i > m && i < b) {
            const C l = Lat(cb + i);
            x1[u] = csub(x1[u], cmul(l, xm1));
            if (use2) x2[u] = csub(x2[u], cmul(l, xm2));
          }
        }
      }
    }
    C *Xc1 = Xe + colbase(k1, b) - k1;  // Xc[i] = X(i, k)
    C *Xc2 = Xe + (has2 ? colbase(k2, b) - k2 : 0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = lane + 32 * u;
      if (i >= k1 && i < b) Xc1[i] = x1[u];
      if (has2 && i >= k2 && i < b) Xc2[i] = x2[u];
    }
  }
}

// Blocked c64 inverse factor for b a multiple of 8 (b <= 160): L (FP32)
// and X in shared memory as 8 x 8 blocks of the lower triangle (block
// (p, q), q <= p, at p (p + 1) / 2 + q, row-major inside).  (1) every
// diagonal block is inverted (one lane per column, forward substitution);
// (2) block column j of X follows from X_jj = L_jj^{-1} and, down the
// column, X_ij = -L_ii^{-1} sum_{k=j}^{i-1} L_ik X_kj -- the sum as 8 x 8 x 8
// block products, lane (r, c) holding entries (r, c) and (r + 4, c).  Warp w
// owns block columns w and P - 1 - w, whose block products add up to the
// same count for every warp.  X is written packed column-major and, if Qb is
// set, (3) Q = X^H X as well, in the blocked layout of the streaming apply
// (precond_blk.cu): Q_pq = sum_{k >= p} X_kp^H X_kq, blocks dealt to the
// warps round-robin.
constexpr int TIB_MAXP = 20;

template <int NB>
__global__ void __launch_bounds__(32 * (TIB_MAXP / 2)) tri_inverse_blocked_kernel(const double2 *__restrict__ Lpk,
                                                                                    int b, float2 *X,
                                                                                    size_t x_stride, float2 *Qb,
                                                                                    size_t qbs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int P = b / NB, nblk = P * (P + 1) / 2;
  float2 *Lb = reinterpret_cast<float2 *>(smraw);  // [nblk][64]
  float2 *Xb = Lb + (size_t)nblk * 64;              // [nblk][64]
  float2 *Db = Xb + (size_t)nblk * 64;              // [P][64] diagonal-block inverses
  float2 *Sw = Db + (size_t)P * 64;                 // [warps][64] scratch
  const int e = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  const size_t npk = (size_t)b * (b + 1) / 2;
  const double2 *Le = Lpk + (size_t)e * npk;
  float2 *Xe = X + (size_t)e * x_stride;
  auto blk = [&](int p, int q) { return (p * (p + 1) / 2 + q) * 64; };
  // Load L (columns by warps, coalesced); zero the diagonal blocks' upper parts.
  for (int p = w; p < P; p += nw)
    for (int t = lane; t < 64; t += 32)
      if ((t & 7) > (t >> 3)) Lb[blk(p, p) + t] = make_float2(0.f, 0.f);
  // One flat pass over the packed entries in batches of 16 per thread: the
  // batch's loads are all issued before any index arithmetic, so they are
  // in flight together.
  for (int t0 = tid; t0 < (int)npk; t0 += 16 * blockDim.x) {
    double2 v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int t = t0 + u * blockDim.x;
      v[u] = t < (int)npk ? Le[t] : make_double2(0, 0);
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int t = t0 + u * blockDim.x;
      if (t < (int)npk) {
        const int k = packed_col(t, b), i = k + t - colbase(k, b);
        Lb[blk(i / NB, k / NB) + (i % NB) * NB + k % NB] = cvt<float2>(v[u]);
      }
    }
  }
  for (size_t q = npk + tid; q < x_stride; q += blockDim.x) Xe[q] = make_float2(0.f, 0.f);  // pad
  __syncthreads();
  // (1) Diagonal-block inverses: lane c < 8 of a warp solves column c.
  for (int p = w; p < P; p += nw) {
    const float2 *L = Lb + blk(p, p);
    float2 *D = Db + p * 64;
    if (lane < NB) {
      const int c = lane;
      float2 x[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) {
        float2 v = make_float2(r == c ? 1.f : 0.f, 0.f);
#pragma unroll
        for (int t = 0; t < NB; ++t)
          if (t < r) v = csub(v, cmul(L[r * NB + t], x[t]));
        x[r] = r < c ? make_float2(0.f, 0.f) : cscale(v, 1.0f / L[r * NB + r].x);
      }
#pragma unroll
      for (int r = 0; r < NB; ++r) D[r * NB + c] = x[r];
    }
  }
  __syncthreads();
  // (2) Block columns.
  const int r0 = lane >> 3, c = lane & 7;
  float2 *S = Sw + w * 64;
  for (int pass = 0; pass < 2; ++pass) {
    const int j = pass == 0 ? w : P - 1 - w;
    if (j >= P || (pass == 1 && j <= w)) continue;
    for (int rr = r0; rr < NB; rr += 4) Xb[blk(j, j) + rr * NB + c] = Db[j * 64 + rr * NB + c];
    __syncwarp();
    for (int i = j + 1; i < P; ++i) {
      float2 a0 = make_float2(0.f, 0.f), a1 = a0;
      for (int k = j; k < i; ++k) {
        const float2 *Lik = Lb + blk(i, k), *Xkj = Xb + blk(k, j);
#pragma unroll
        for (int t = 0; t < NB; ++t) {
          const float2 xv = Xkj[t * NB + c];
          a0 = cfma(Lik[r0 * NB + t], xv, a0);
          a1 = cfma(Lik[(r0 + 4) * NB + t], xv, a1);
        }
      }
      S[r0 * NB + c] = a0;
      S[(r0 + 4) * NB + c] = a1;
      __syncwarp();
      const float2 *D = Db + i * 64;
      float2 y0 = make_float2(0.f, 0.f), y1 = y0;
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        const float2 sv = S[t * NB + c];
        y0 = cfma(D[r0 * NB + t], sv, y0);  // D is lower triangular: zeros above its diagonal
        y1 = cfma(D[(r0 + 4) * NB + t], sv, y1);
      }
      Xb[blk(i, j) + r0 * NB + c] = make_float2(-y0.x, -y0.y);
      Xb[blk(i, j) + (r0 + 4) * NB + c] = make_float2(-y1.x, -y1.y);
      __syncwarp();  // S reused, X_ij read by the next block row
    }
  }
  __syncthreads();
  // X packed column-major (coalesced).
  for (int t = tid; t < (int)npk; t += blockDim.x) {
    const int k = packed_col(t, b), i = k + t - colbase(k, b);
    Xe[t] = Xb[blk(i / NB, k / NB) + (i % NB) * NB + k % NB];
  }
  if (!Qb) return;
  // (3) Q = X^H X, entry (r, c) of block (p, q) at c * 8 + (r ^ c).
  float2 *Qe = Qb + (size_t)e * qbs;
  for (int bq = w; bq < nblk; bq += nw) {
    int p = 0;
    while ((p + 1) * (p + 2) / 2 <= bq) ++p;
    const int q = bq - p * (p + 1) / 2;
    float2 a0 = make_float2(0.f, 0.f), a1 = a0;
    for (int k = p; k < P; ++k) {
      const float2 *Xkp = Xb + blk(k, p), *Xkq = Xb + blk(k, q);
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        const float2 xq = Xkq[t * NB + c];
        a0 = cfmac(Xkp[t * NB + r0], xq, a0);
        a1 = cfmac(Xkp[t * NB + r0 + 4], xq, a1);
      }
    }
    Qe[(size_t)bq * 64 + c * 8 + (r0 ^ c)] = a0;
    Qe[(size_t)bq * 64 + c * 8 + ((r0 + 4) ^ c)] = a1;
  }
}

size_t tri_inverse_blocked_smem(int b) {
  const int P = b / 8;
  return ((size_t)2 * P * (P + 1) / 2 * 64 + (size_t)P * 64 + (size_t)((P + 1) / 2) * 64) * sizeof(float2);
}

template <typename R>
bool launch_tri_inverse(const double2 *Lpk, int nel, int b, void *X, size_t x_stride, cudaStream_t st, void *Qb) {
  using C = typename Cplx<R>::T;
  if constexpr (std::is_same<R, float>::value) {
    if (b % 8 == 0 && b / 8 <= TIB_MAXP && tri_inverse_blocked_smem(b) <= 220 * 1024) {
      const int P = b / 8;
      static bool configured = false;
      if (!configured) {
        cudaFuncSetAttribute(tri_inverse_blocked_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        configured = true;
      }
      tri_inverse_blocked_kernel<8><<<nel, 32 * ((P + 1) / 2), tri_inverse_blocked_smem(b), st>>>(
          Lpk, b, reinterpret_cast<float2 *>(X), x_stride, reinterpret_cast<float2 *>(Qb), (size_t)P * (P + 1) / 2 * 64);
      return true;
    }
  }
  const size_t head = ((size_t)b * sizeof(R) + 15) & ~size_t(15);
  const size_t bytes = (size_t)b * (b + 1) / 2 * sizeof(C);
  const bool in_smem = head + bytes <= 200 * 1024;
  const int U = (b + 31) / 32;
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    kern<<<nel, 256, head + (in_smem ? bytes : 0), st>>>(Lpk, b, reinterpret_cast<C *>(X), x_stride);
  };
  if (in_smem) {
    if (U <= 1) go(tri_inverse_kernel<R, 1, true>);
    else if (U <= 2) go(tri_inverse_kernel<R, 2, true>);
    else if (U <= 4) go(tri_inverse_kernel<R, 4, true>);
    else go(tri_inverse_kernel<R, 8, true>);
  } else {
    go(tri_inverse_kernel<R, 8, false>);
  }
  return false;
}
template bool launch_tri_inverse<float>(const double2 *, int, int, void *, size_t, cudaStream_t, void *);
template bool launch_tri_inverse<double>(const double2 *, int, int, void *, size_t, cudaStream_t, void *);

// ------------------------------------------------------------ apply ------
// y_e = X_e^H (X_e x_e), X_e = L_e^{-1} packed column-major.  One CTA per
// element; X_e arrives in shared memory with one bulk copy when it fits
// (otherwise its columns are read from global memory).
//  Phase 1, t = X x: warps own columns k, lanes own rows i >= k and
//    accumulate X(i,k) x_k in registers; partial t is reduced across warps.
//  Phase 2, z = X^H t: warps own columns k, lanes own rows i >= k, and
//    z_k = sum_i conj(X(i,k)) t_i is a warp reduction.
// Sixteen warps per element: each warp's serial chain over its columns
// (phase 1) or rows (phase 2) is b / 16 long.
constexpr int PA_THREADS = 512, PA_WARPS = 16;

// x_e of RHS q0 .. q0+NR-1 into shared memory, [b][NR].
template <typename R, int NR>
MOMA_DEV void load_x_chunk(const typename Cplx<R>::T *__restrict__ x, typename Cplx<R>::T *xs, int e, int b, int nr,
                           int q0, long long vstride, long long voff) {
  using C = typename Cplx<R>::T;
  for (int idx = threadIdx.x; idx < b * NR; idx += PA_THREADS) {
    const int k = idx / NR, q = q0 + idx % NR;
    xs[idx] = q < nr ? x[(size_t)q * vstride + voff + (size_t)e * b + k] : czero<C>();
  }
}

// The two triangular products of one element (phases 1 and 2 below), X_e
// already in shared memory (or global memory) at Xs; the first RHS chunk
// of x_e is already in xs when first_loaded is set.
template <typename R, int NR, int U>
MOMA_DEV void apply_element(const typename Cplx<R>::T *Xs, int e, int nel, int b, int nr,
                            const typename Cplx<R>::T *__restrict__ x, typename Cplx<R>::T *__restrict__ y,
                            typename Cplx<R>::T *xs, typename Cplx<R>::T *ts, typename Cplx<R>::T *tp,
                            long long vstride, long long voff, bool first_loaded) {
  using C = typename Cplx<R>::T;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int q0 = 0; q0 < nr; q0 += NR) {
    if (q0 > 0 || !first_loaded) load_x_chunk<R, NR>(x, xs, e, b, nr, q0, vstride, voff);
    __syncthreads();
    C acc[U][NR];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int qq = 0; qq < NR; ++qq) acc[u][qq] = czero<C>();
    for (int k = w; k < b; k += PA_WARPS) {
      const C *col = Xs + colbase(k, b) - k;
      C xk[NR];
#pragma unroll
      for (int qq = 0; qq < NR; ++qq) xk[qq] = xs[k * NR + qq];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = lane + 32 * u;
        if (i >= k && i < b) {
          const C xv = col[i];
#pragma unroll
          for (int qq = 0; qq < NR; ++qq) acc[u][qq] = cfma(xv, xk[qq], acc[u][qq]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = lane + 32 * u;
      if (i < b)
#pragma unroll
        for (int qq = 0; qq < NR; ++qq) tp[((size_t)w * b + i) * NR + qq] = acc[u][qq];
    }
    __syncthreads();
    for (int idx = tid; idx < b * NR; idx += PA_THREADS) {
      C v = czero<C>();
      for (int ww = 0; ww < PA_WARPS; ++ww) v = cadd(v, tp[(size_t)ww * b * NR + idx]);
      ts[idx] = v;
    }
    __syncthreads();
    // Phase 2, z = X^H t: lanes own outputs k, warps own rows i (strided
    // so that the triangle is shared evenly); z_k = sum_{i >= k}
    // conj(X(i,k)) t_i accumulates in registers, partial sums of the warps
    // are added through shared memory (no per-column warp reductions).
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int qq = 0; qq < NR; ++qq) acc[u][qq] = czero<C>();
    for (int i = w; i < b; i += PA_WARPS) {
      C ti[NR];
#pragma unroll
      for (int qq = 0; qq < NR; ++qq) ti[qq] = ts[i * NR + qq];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = lane + 32 * u;
        if (k <= i) {
          const C xv = Xs[colbase(k, b) - k + i];  // X(i, k)
#pragma unroll
          for (int qq = 0; qq < NR; ++qq) acc[u][qq] = cfmac(xv, ti[qq], acc[u][qq]);
        }
      }
    }
    __syncthreads();  // every warp has finished reading ts / tp of phase 1
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = lane + 32 * u;
      if (k < b)
#pragma unroll
        for (int qq = 0; qq < NR; ++qq) tp[((size_t)w * b + k) * NR + qq] = acc[u][qq];
    }
    __syncthreads();
    for (int idx = tid; idx < b * NR; idx += PA_THREADS) {
      C v = czero<C>();
      for (int ww = 0; ww < PA_WARPS; ++ww) v = cadd(v, tp[(size_t)ww * b * NR + idx]);
      const int k = idx / NR, qq = idx % NR;
      if (q0 + qq < nr) y[(size_t)(q0 + qq) * vstride + voff + (size_t)e * b + k] = v;
    }
    __syncthreads();
  }
}

template <typename R, int NR, int U, bool X_IN_SMEM>
__global__ void __launch_bounds__(PA_THREADS, U <= 4 ? 2 : 1) precond_apply_kernel(const typename Cplx<R>::T *__restrict__ X,
                                                                   size_t x_stride, int nel, int b, int nr,
                                                                   const typename Cplx<R>::T *__restrict__ x,
                                                                   typename Cplx<R>::T *__restrict__ y,
                                                                   unsigned *err, const int *live,
                                                                   long long vstride, long long voff) {
  using C = typename Cplx<R>::T;
  extern __shared__ __align__(128) unsigned char smraw[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smraw);
  C *xs = reinterpret_cast<C *>(smraw + 128) + (X_IN_SMEM ? x_stride : 0);  // [b][NR]
  const C *Xs = X_IN_SMEM ? reinterpret_cast<const C *>(smraw + 128) : X + (size_t)blockIdx.x * x_stride;
  C *ts = xs + (size_t)b * NR;        // [b][NR]
  C *tp = ts + (size_t)b * NR;        // [PA_WARPS][b][NR]
  const int e = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (live && *live == 0) return;
  if (X_IN_SMEM) {
    if (tid == 0) {
      mbar_init(bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
      const uint32_t bytes = (uint32_t)(x_stride * sizeof(C));
      fence_proxy_async();
      mbar_expect_tx(bar, bytes);
      bulk_g2s(const_cast<C *>(Xs), X + (size_t)e * x_stride, bytes, bar);
    }
    // The first RHS chunk of x_e is read while X_e is in flight.
    load_x_chunk<R, NR>(x, xs, e, b, nr, 0, vstride, voff);
    const bool ok = mbar_wait_bounded(bar, 0, 2000000000ull);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(err, DEVERR_TIMEOUT);
        mbar_wait_bounded(bar, 0, 2000000000ull);
      }
      return;
    }
  }

  apply_element<R, NR, U>(Xs, e, nel, b, nr, x, y, xs, ts, tp, vstride, voff, X_IN_SMEM);
}

template <typename R, int NR, int U>
static void apply_launch(const void *X, size_t x_stride, int nel, int b, int nr, const void *x, void *y,
                         unsigned *err, const int *live, long long vstride, long long voff, cudaStream_t st) {
  using C = typename Cplx<R>::T;
  const size_t vec = (size_t)(2 + PA_WARPS) * b * NR * sizeof(C);
  const bool in_smem = 128 + x_stride * sizeof(C) + vec <= 220 * 1024;
  const size_t smem = 128 + (in_smem ? x_stride * sizeof(C) : 0) + vec;
  static int configured = 0;
  if (!configured) {
    cudaFuncSetAttribute(precond_apply_kernel<R, NR, U, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    cudaFuncSetAttribute(precond_apply_kernel<R, NR, U, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         220 * 1024);
    configured = 1;
  }
  auto kern = in_smem ? precond_apply_kernel<R, NR, U, true> : precond_apply_kernel<R, NR, U, false>;
  kern<<<nel, PA_THREADS, smem, st>>>(
      reinterpret_cast<const C *>(X), x_stride, nel, b, nr, reinterpret_cast<const C *>(x),
      reinterpret_cast<C *>(y), err, live, vstride, voff);
}

template <typename R, int NR>
static void apply_u(const void *X, size_t xs, int nel, int b, int nr, const void *x, void *y, unsigned *err,
                    const int *live, long long vs, long long vo, cudaStream_t st) {
  const int U = (b + 31) / 32;
  if (U <= 1) apply_launch<R, NR, 1>(X, xs, nel, b, nr, x, y, err, live, vs, vo, st);
  else if (U <= 2) apply_launch<R, NR, 2>(X, xs, nel, b, nr, x, y, err, live, vs, vo, st);
  else if (U <= 4) apply_launch<R, NR, 4>(X, xs, nel, b, nr, x, y, err, live, vs, vo, st);
  else apply_launch<R, NR, 8>(X, xs, nel, b, nr, x, y, err, live, vs, vo, st);
}

template <typename R>
void launch_precond_apply(const void *X, size_t x_stride, int nel, int b, int nr, const void *x, void *y,
                          unsigned *err, const int *live, long long vstride, long long voff, cudaStream_t st) {
  if (vstride <= 0) vstride = (long long)nel * b;
  if (nr == 1) apply_u<R, 1>(X, x_stride, nel, b, nr, x, y, err, live, vstride, voff, st);
  else apply_u<R, 2>(X, x_stride, nel, b, nr, x, y, err, live, vstride, voff, st);
}
template void launch_precond_apply<float>(const void *, size_t, int, int, int, const void *, void *, unsigned *,
                                          const int *, long long, long long, cudaStream_t);
template void launch_precond_apply<double>(const void *, size_t, int, int, int, const void *, void *, unsigned *,
                                           const int *, long long, long long, cudaStream_t);

}  // namespace moma
