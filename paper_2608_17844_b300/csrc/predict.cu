// Error predictors for approximating the centre element's active
// impedance (Sec. II-E, after Eq. 19): the column coupling C_n (Eqs. 28-30)
// from a sweep of the inter-element phase, the S -> Z conversion (Eq. 31),
// the idealised scattering matrix behind xi_S (Eq. 36), and the xi_Z
// family (Eqs. 23-25) read off Z_p.
//
//  * C_n: the row-phase excitations V_q = exp(j m_x psi_q) on every port
//    (Eq. 29, psi_q = -pi + 2 pi q / Q) are solved in RHS chunks with the
//    array's solver; the centre element's active reflection coefficient is
//    gathered per sample and C_n = (1/Q) sum_q Gamma_q exp(-j n psi_q) (the
//    trapezoidal rule of the 2 pi periodic integral of Eq. 28, exact for
//    trigonometric polynomials of degree < Q).
//  * Z_p = Z0 (I + S)(I - S)^{-1}: M = I - S inverted in FP64 on the device
//    (Gauss-Jordan, partial pivoting), then Z_p = Z0 (M^{-1} + S M^{-1}).
//  * S_ideal: S_cc on the diagonal, s1 dist^-2 exp(-j k d (dist - 1)) off
//    it (dist = Euclidean element distance in units of d).
#include <cmath>
#include <vector>

#include "internal.h"

namespace moma {

// V[q][e*b + pb] = exp(j mx psi_{q0+q}), zero on the other bases.
__global__ void row_phase_kernel(double2 *V, int nx, int nel, int b, int pb, int q0, int nq, int Q, long long ldv) {
  const size_t N = (size_t)ldv, total = (size_t)nq * N, NA = (size_t)nel * b;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx / N);
    const size_t n = idx % N;
    double2 v = make_double2(0.0, 0.0);
    if (n < NA && (int)(n % b) == pb) {
      const int mx = (int)(n / b) % nx;
      // psi = -pi + 2 pi k / Q, k = q0 + q; mx psi = pi (2 mx k / Q - mx).
      const long long k = q0 + q;
      const long long num = (2 * (long long)mx * k) % (2LL * Q);  // angle / pi = num / Q - mx (mod 2)
      double s, c;
      sincospi((double)num / (double)Q - (double)(mx & 1), &s, &c);
      v = make_double2(c, s);
    }
    V[idx] = v;
  }
}

// C[n + nmax] = (1/Q) sum_q gamma[q] exp(-j n psi_q), n = -nmax .. nmax.
__global__ void column_coupling_kernel(const double2 *gamma, int Q, int nmax, double2 *C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > 2 * nmax) return;
  const long long n = i - nmax;
  double2 acc = make_double2(0.0, 0.0);
  for (int q = 0; q < Q; ++q) {
    // -n psi_q = n pi - 2 pi n q / Q.
    long long r = (n * q) % Q;
    if (r < 0) r += Q;
    double s, c;
    sincospi((double)(n & 1) - 2.0 * (double)r / (double)Q, &s, &c);
    acc = cfma(gamma[q], make_double2(c, s), acc);
  }
  C[i] = make_double2(acc.x / Q, acc.y / Q);
}

// S_ideal (n = nx*ny, row-major).
__global__ void s_ideal_kernel(double2 *S, int nx, int n, double2 s_cc, double2 s1, double kd) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)n * n;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    if (i == j) {
      S[idx] = s_cc;
      continue;
    }
    const double dx = (double)(i % nx - j % nx), dy = (double)(i / nx - j / nx);
    const double dist = sqrt(dx * dx + dy * dy);
    double s, c;
    sincos(-kd * (dist - 1.0), &s, &c);
    const double inv2 = 1.0 / (dist * dist);
    S[idx] = cscale(cmul(s1, make_double2(c, s)), inv2);
  }
}

// A = I - S (or I + S with sign = +1).
__global__ void eye_pm_kernel(const double2 *S, double2 *A, int n, double sign) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)n * n;
       idx += (size_t)gridDim.x * blockDim.x) {
    const bool d = (idx / n) == (idx % n);
    A[idx] = make_double2((d ? 1.0 : 0.0) + sign * S[idx].x, sign * S[idx].y);
  }
}

// C = z0 (B + S B), all n x n row-major FP64 complex; 16 x 16 tiles.
__global__ void z_from_s_gemm_kernel(const double2 *S, const double2 *B, double2 *C, int n, double z0) {
  __shared__ double2 Ss[16][17], Bs[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
  double2 acc = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < n; k0 += 16) {
    Ss[ty][tx] = (i < n && k0 + tx < n) ? S[(size_t)i * n + k0 + tx] : make_double2(0.0, 0.0);
    Bs[ty][tx] = (k0 + ty < n && j < n) ? B[(size_t)(k0 + ty) * n + j] : make_double2(0.0, 0.0);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = cfma(Ss[ty][k], Bs[k][tx], acc);
    __syncthreads();
  }
  if (i < n && j < n) {
    const double2 bij = B[(size_t)i * n + j];
    C[(size_t)i * n + j] = make_double2(z0 * (bij.x + acc.x), z0 * (bij.y + acc.y));
  }
}

static int grid_for(size_t total) {
  size_t g = (total + 255) / 256;
  return (int)(g > 8192 ? 8192 : (g < 1 ? 1 : g));
}

void launch_row_phase(double2 *V, int nx, int nel, int b, int pb, int q0, int nq, int Q, long long ldv,
                      cudaStream_t st) {
  row_phase_kernel<<<grid_for((size_t)nq * ldv), 256, 0, st>>>(V, nx, nel, b, pb, q0, nq, Q, ldv);
}
void launch_column_coupling(const double2 *gamma, int Q, int nmax, double2 *C, cudaStream_t st) {
  column_coupling_kernel<<<(2 * nmax + 1 + 127) / 128, 128, 0, st>>>(gamma, Q, nmax, C);
}
void launch_s_ideal(double2 *S, int nx, int ny, double2 s_cc, double2 s1, double kd, cudaStream_t st) {
  const int n = nx * ny;
  s_ideal_kernel<<<grid_for((size_t)n * n), 256, 0, st>>>(S, nx, n, s_cc, s1, kd);
}
// Z = z0 (I + S)(I - S)^{-1}; work: n*n*2 double2 + n*(double2 + int) bytes.
void launch_z_from_s(const double2 *S, int n, double z0, double2 *Z, double2 *work, unsigned *err, cudaStream_t st) {
  double2 *M = work, *colk = work + (size_t)n * n;
  int *perm = reinterpret_cast<int *>(colk + n);
  eye_pm_kernel<<<grid_for((size_t)n * n), 256, 0, st>>>(S, M, n, -1.0);
  launch_invert(M, n, perm, colk, err, st);
  dim3 grid((n + 15) / 16, (n + 15) / 16), block(16, 16);
  z_from_s_gemm_kernel<<<grid, block, 0, st>>>(S, M, Z, n, z0);
}

}  // namespace moma
