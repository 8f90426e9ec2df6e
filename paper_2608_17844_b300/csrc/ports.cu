// Passive port impedance matrix (Eq. 18): with unit voltage on port j and
// zero elsewhere, the solved port currents are column j of the port
// admittance matrix Y_p; Z_p = Y_p^{-1}.  The port solves reuse the
// array's solver (GMRES or PCG inside FP64 refinement) in chunks of RHS;
// the inversion is an FP64 Gauss-Jordan elimination with partial pivoting
// on the device.
#include "internal.h"

namespace moma {

// V[q][e*b + pb] = (e == j0 + q), zero elsewhere (margin entries too); q < nq,
// per-RHS stride ldv.
__global__ void unit_ports_kernel(double2 *V, int nel, int b, int pb, int j0, int nq, long long ldv) {
  const size_t N = (size_t)ldv, total = (size_t)nq * N, NA = (size_t)nel * b;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx / N);
    const size_t n = idx % N;
    const bool on = n < NA && (n % b) == (size_t)pb && (int)(n / b) == j0 + q;
    V[idx] = make_double2(on ? 1.0 : 0.0, 0.0);
  }
}

// Y[i][j0 + q] = I[q][i*b + pb]  (Y row-major n x n).
__global__ void gather_ports_kernel(const double2 *I, int nel, int b, int pb, int j0, int nq, double2 *Y,
                                    long long ldv) {
  const int total = nel * nq;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int q = idx / nel, i = idx % nel;
    Y[(size_t)i * nel + j0 + q] = I[(size_t)q * ldv + (size_t)i * b + pb];
  }
}

// Gauss-Jordan step k, part 1 (one CTA): pivot row = argmax_{i >= k} |A[i][k]|
// (first index on ties), swap rows k and piv, record piv, scale row k by
// 1 / pivot with A[k][k] replaced by 1 (in-place inversion).
__global__ void gj_pivot_kernel(double2 *A, int n, int k, int *perm, double2 *colk, unsigned *err) {
  __shared__ double bv[1024];
  __shared__ int bi[1024];
  __shared__ double2 pv;
  const int t = threadIdx.x;
  double best = -1.0;
  int bidx = k;
  for (int i = k + t; i < n; i += blockDim.x) {
    const double2 v = A[(size_t)i * n + k];
    const double m = v.x * v.x + v.y * v.y;
    if (m > best) { best = m; bidx = i; }
  }
  bv[t] = best;
  bi[t] = bidx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) {
      if (bv[t + s] > bv[t] || (bv[t + s] == bv[t] && bi[t + s] < bi[t])) {
        bv[t] = bv[t + s];
        bi[t] = bi[t + s];
      }
    }
    __syncthreads();
  }
  const int piv = bi[0];
  if (t == 0) {
    perm[k] = piv;
    if (!(bv[0] > 0.0) || !isfinite(bv[0])) atomicOr(err, DEVERR_NONFINITE);
  }
  if (piv != k)
    for (int j = t; j < n; j += blockDim.x) {
      const double2 a = A[(size_t)k * n + j];
      A[(size_t)k * n + j] = A[(size_t)piv * n + j];
      A[(size_t)piv * n + j] = a;
    }
  __syncthreads();
  if (t == 0) pv = A[(size_t)k * n + k];
  // Snapshot of column k (after the swap) for the elimination step.
  for (int i = t; i < n; i += blockDim.x) colk[i] = A[(size_t)i * n + k];
  __syncthreads();
  const double den = pv.x * pv.x + pv.y * pv.y;
  const double2 inv = make_double2(pv.x / den, -pv.y / den);
  for (int j = t; j < n; j += blockDim.x) {
    const double2 a = (j == k) ? make_double2(1.0, 0.0) : A[(size_t)k * n + j];
    A[(size_t)k * n + j] = cmul(a, inv);
  }
}

// Part 2: every row i != k: f = A[i][k] (from the snapshot); A[i][k] = 0;
// A[i][:] -= f * A[k][:].
__global__ void gj_eliminate_kernel(double2 *A, int n, int k, const double2 *colk) {
  const int i = blockIdx.y;
  if (i == k) return;
  const double2 f = colk[i];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const double2 rk = A[(size_t)k * n + j];
    const double2 a = (j == k) ? make_double2(0.0, 0.0) : A[(size_t)i * n + j];
    A[(size_t)i * n + j] = cfms(f, rk, a);
  }
}

// Undo the row interchanges as column interchanges, last step first.
__global__ void gj_unpermute_kernel(double2 *A, int n, const int *perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = n - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k) {
      const double2 a = A[(size_t)i * n + k];
      A[(size_t)i * n + k] = A[(size_t)i * n + p];
      A[(size_t)i * n + p] = a;
    }
  }
}

void launch_unit_ports(double2 *V, int nel, int b, int pb, int j0, int nq, long long ldv, cudaStream_t st) {
  size_t total = (size_t)nq * ldv, g = (total + 255) / 256;
  if (g > 4096) g = 4096;
  unit_ports_kernel<<<(int)g, 256, 0, st>>>(V, nel, b, pb, j0, nq, ldv);
}
void launch_gather_ports(const double2 *I, int nel, int b, int pb, int j0, int nq, double2 *Y, long long ldv,
                         cudaStream_t st) {
  int total = nel * nq, g = (total + 255) / 256;
  if (g > 4096) g = 4096;
  gather_ports_kernel<<<g, 256, 0, st>>>(I, nel, b, pb, j0, nq, Y, ldv);
}
void launch_invert(double2 *A, int n, int *perm, double2 *colk, unsigned *err, cudaStream_t st) {
  for (int k = 0; k < n; ++k) {
    gj_pivot_kernel<<<1, 1024, 0, st>>>(A, n, k, perm, colk, err);
    dim3 grid((n + 255) / 256, n);
    gj_eliminate_kernel<<<grid, 256, 0, st>>>(A, n, k, colk);
  }
  gj_unpermute_kernel<<<(n + 127) / 128, 128, 0, st>>>(A, n, perm);
}

}  // namespace moma
