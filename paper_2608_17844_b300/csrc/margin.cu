// Array margin (Eq. 1's non-MBT border): the MoM matrix of a finite array
// on a ground plane is Z = [Z_A, Z_B^T; Z_B, Z_C] (reciprocal), Z_A the MBT
// element part, Z_B (nm x N) the margin-element coupling, Z_C (nm x nm)
// the margin part.  Vectors are [lattice N | margin nm] per RHS (stride ldv).
//
//   Z   [x_A; x_M] = [Z_A x_A + Z_B^T x_M;   Z_B x_A + Z_C x_M]
//   Z^H [x_A; x_M] = [Z_A^H x_A + Z_B^H x_M; conj(Z_B) x_A + Z_C^H x_M]
//
// (Eq. 5 shows Z^H in this block form.)  The lattice products Z_A x_A run
// through the MLFFT path; the kernels here add the dense margin terms.
// The margin block of the preconditioner (Eq. 38) is
//   P_C = conj(Z_B) Z_B^T + Z_C^H Z_C,
// factored P_C = L_C L_C^H in FP64 on the device and applied, like the
// element blocks, as X_C^H X_C with X_C = L_C^{-1}.
#include "internal.h"

namespace moma {

// y_A[n] += sum_m op(Z_B)[m][n] x_M[m]; op = identity (Z) or conj (Z^H).
template <typename R>
__global__ void margin_to_lattice_kernel(const typename Cplx<R>::T *__restrict__ ZB, int nm, int N, long long ldv,
                                         int herm, const typename Cplx<R>::T *__restrict__ x,
                                         typename Cplx<R>::T *__restrict__ y) {
  using C = typename Cplx<R>::T;
  const int n = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
  if (n >= N) return;
  const C *xm = x + (size_t)q * ldv + N;
  C acc = y[(size_t)q * ldv + n];
  for (int m = 0; m < nm; ++m) {
    const C z = ZB[(size_t)m * N + n];
    acc = herm ? cfmac(z, xm[m], acc) : cfma(z, xm[m], acc);
  }
  y[(size_t)q * ldv + n] = acc;
}

// y_M[m] = sum_n op(Z_B)[m][n] x_A[n] + sum_j op_C(m, j) x_M[j], with
// op_C(m, j) = Z_C[m][j] (Z) or conj(Z_C[j][m]) (Z^H).  One CTA per (m, q).
template <typename R>
__global__ void lattice_to_margin_kernel(const typename Cplx<R>::T *__restrict__ ZB,
                                         const typename Cplx<R>::T *__restrict__ ZC, int nm, int N, long long ldv,
                                         int herm, const typename Cplx<R>::T *__restrict__ x,
                                         typename Cplx<R>::T *__restrict__ y) {
  using C = typename Cplx<R>::T;
  __shared__ C part[32];
  const int m = blockIdx.x, q = blockIdx.y, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const C *xq = x + (size_t)q * ldv;
  const C *zb = ZB + (size_t)m * N;
  C acc = czero<C>();
  for (int n = tid; n < N; n += blockDim.x) acc = herm ? cfmac(zb[n], xq[n], acc) : cfma(zb[n], xq[n], acc);
  for (int j = tid; j < nm; j += blockDim.x) {
    if (herm) acc = cfmac(ZC[(size_t)j * nm + m], xq[N + j], acc);
    else acc = cfma(ZC[(size_t)m * nm + j], xq[N + j], acc);
  }
  acc = warp_sum(acc);
  if (lane == 0) part[w] = acc;
  __syncthreads();
  if (w == 0) {
    C v = lane < (int)(blockDim.x >> 5) ? part[lane] : czero<C>();
    v = warp_sum(v);
    if (lane == 0) y[(size_t)q * ldv + N + m] = v;
  }
}

// P_C[i][j] = sum_n conj(Z_B[i][n]) Z_B[j][n] + sum_k conj(Z_C[k][i]) Z_C[k][j]
// (FP64), one CTA per (i, j) with j <= i; written to both triangles.
__global__ void margin_gram_kernel(const double2 *__restrict__ ZB, const double2 *__restrict__ ZC, int nm, int N,
                                   double2 *__restrict__ P) {
  __shared__ double2 part[32];
  const int i = blockIdx.x, j = blockIdx.y, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (j > i) return;
  double2 acc = make_double2(0.0, 0.0);
  const double2 *bi = ZB + (size_t)i * N, *bj = ZB + (size_t)j * N;
  for (int n = tid; n < N; n += blockDim.x) acc = cfmac(bi[n], bj[n], acc);
  for (int k = tid; k < nm; k += blockDim.x) acc = cfmac(ZC[(size_t)k * nm + i], ZC[(size_t)k * nm + j], acc);
  acc = warp_sum(acc);
  if (lane == 0) part[w] = acc;
  __syncthreads();
  if (w == 0) {
    double2 v = lane < (int)(blockDim.x >> 5) ? part[lane] : make_double2(0.0, 0.0);
    v = warp_sum(v);
    if (lane == 0) {
      P[(size_t)i * nm + j] = v;
      P[(size_t)j * nm + i] = cconj(v);
    }
  }
}

// Cholesky of one n x n Hermitian matrix (row-major full P) into packed
// lower column-major Lpk (FP64); one CTA, column by column.
__global__ void dense_cholesky_kernel(const double2 *__restrict__ P, int n, double2 *__restrict__ L, unsigned *err) {
  const int tid = threadIdx.x;
  auto cb = [&](int k) { return (size_t)k * n - (size_t)k * (k - 1) / 2 - k; };  // L(i, k) at cb(k) + i
  for (int k = 0; k < n; ++k)
    for (int i = k + tid; i < n; i += blockDim.x) L[cb(k) + i] = P[(size_t)i * n + k];
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    double2 *cj = L + cb(j);
    const double d = cj[j].x;
    if (!(d > 0.0) || !isfinite(d)) {
      if (tid == 0) atomicOr(err, DEVERR_NOT_PD);
      return;
    }
    const double l = sqrt(d), inv = 1.0 / l;
    __syncthreads();
    for (int i = j + tid; i < n; i += blockDim.x) cj[i] = (i == j) ? make_double2(l, 0.0) : cscale(cj[i], inv);
    __syncthreads();
    // Trailing update A(i, k) -= L(i, j) conj(L(k, j)), j < k <= i: warps
    // take columns, lanes rows.
    const int lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    for (int k = j + 1 + w; k < n; k += nw) {
      double2 *ck = L + cb(k);
      const double2 lkj = cj[k];
      for (int i = k + lane; i < n; i += 32) ck[i] = cfms_conj(cj[i], lkj, ck[i]);
    }
    __syncthreads();
  }
}

template <typename R>
void launch_margin_apply(const void *ZB, const void *ZC, int nm, int N, long long ldv, int nr, int herm,
                         const void *x, void *y, cudaStream_t st) {
  using C = typename Cplx<R>::T;
  if (nm <= 0 || nr <= 0) return;
  // Margin rows first (they read the lattice part of x only), then the
  // lattice update (reads the margin part of x only): y may not alias x.
  lattice_to_margin_kernel<R><<<dim3(nm, nr), 256, 0, st>>>(static_cast<const C *>(ZB), static_cast<const C *>(ZC), nm,
                                                             N, ldv, herm, static_cast<const C *>(x), static_cast<C *>(y));
  margin_to_lattice_kernel<R><<<dim3((N + 255) / 256, nr), 256, 0, st>>>(static_cast<const C *>(ZB), nm, N, ldv, herm,
                                                                         static_cast<const C *>(x), static_cast<C *>(y));
}
template void launch_margin_apply<float>(const void *, const void *, int, int, long long, int, int, const void *, void *,
                                         cudaStream_t);
template void launch_margin_apply<double>(const void *, const void *, int, int, long long, int, int, const void *,
                                          void *, cudaStream_t);

void launch_margin_precond_build(const double2 *ZB, const double2 *ZC, int nm, int N, double2 *P, double2 *Lpk,
                                 unsigned *err, cudaStream_t st) {
  margin_gram_kernel<<<dim3(nm, nm), 256, 0, st>>>(ZB, ZC, nm, N, P);
  dense_cholesky_kernel<<<1, 1024, 0, st>>>(P, nm, Lpk, err);
}

}  // namespace moma
