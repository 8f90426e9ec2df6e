// Device control block and launchers of the Krylov / refinement kernels.
#pragma once
#include "internal.h"

#define MOMA_MAX_RESTART 128

namespace moma {

enum : int { KF_UPDATE = 1, KF_DOTS = 2, KF_NORM = 4, KF_ACCUM = 8, KF_INIT = 16 };

// Per-RHS GMRES state (arrays of length nr unless noted), all device memory.
struct KrylovCtl {
  int m;                 // restart length
  double inner_tol;      // relative tolerance of one GMRES cycle
  int *active;           // 1 while column q still iterates
  int *kq;               // Arnoldi steps taken by column q this cycle
  int *nact;             // [1] number of active columns
  double *beta;          // initial residual norm
  double *tol;           // inner_tol * beta
  double *res;           // current residual estimate |g_{j+1}|
  double *inv_norm;      // 1 / h_{j+1,j} (0 when frozen)
  unsigned *counters;    // [nr] last-block tickets
  unsigned *err;         // device error bits
  double2 *partial;      // [nr][nchunk][m+1]
  double2 *hacc;         // [nr][m+1] column j of H (h1 + h2)
  double2 *hcur;         // [nr][m+1] coefficients of the pending update
  double2 *Rm;           // [nr][m][m+1] rotated Hessenberg columns
  double *cs;            // [nr][m]
  double2 *sn;           // [nr][m]
  double2 *g;            // [nr][m+1]
  double2 *y;            // [nr][m]
  double2 *partial2;     // [nr][nchunk][m+1]  (fused step: second and third sweeps)
  double2 *partial3;     // [nr][nchunk]
  unsigned *gbar;        // [1] grid-barrier counter of the fused step (zeroed per cycle)
};

enum : int { CG_PQ = 0, CG_RZ = 1, CG_RZ0 = 2 };  // modes of launch_cg_reduce

// Per-RHS state of the conjugate-gradient inner solver (device memory).
struct CgCtl {
  int *active;        // [nr]
  int *nact;          // [1]
  int *iters;         // [nr] iterations taken
  double *rz, *rr, *rr0, *alpha, *beta;  // [nr]
  double tol2;        // (relative tolerance)^2 on ||r||^2 / ||r0||^2
  unsigned *counters; // [nr]
  double *partial;    // [nr][nchunk]
  unsigned *err;
};
template <typename R>
void launch_cg_reduce(const CgCtl &c, const void *a, const void *b, int N, int nr, int mode, cudaStream_t st);
template <typename R>
void launch_cg_axpy(const CgCtl &c, void *d, const void *p, void *r, const void *q, int N, int nr, int init,
                    cudaStream_t st);
template <typename R>
void launch_cg_dir(const CgCtl &c, void *p, const void *z, int N, int nr, int init, cudaStream_t st);
template <typename R>
void launch_cg_accum(const void *d, int N, int nr, double2 *I, const double *scale, cudaStream_t st);

int krylov_chunks(int N);
template <typename R>
void launch_cgs(const KrylovCtl &c, void *V, size_t vstride, int N, int nr, int j, int flags, cudaStream_t st);
template <typename R>
void launch_scale(const KrylovCtl &c, void *v, size_t vstride, int N, int nr, cudaStream_t st);
// One whole Arnoldi orthogonalisation step j (the three CGS2 sweeps, the
// Givens update and the scaling of the new basis vector) as one cooperative
// launch with grid barriers; false if the grid cannot be co-resident (the
// caller then issues the separate sweeps).
template <typename R>
bool arnoldi_fused_fits(int N, int nr, int num_sms);
template <typename R>
void launch_arnoldi_fused(const KrylovCtl &c, void *V, size_t vstride, int N, int nr, int j, cudaStream_t st);
void launch_backsolve(const KrylovCtl &c, int nr, cudaStream_t st);
template <typename R>
void launch_lincomb(const KrylovCtl &c, const void *V, size_t vstride, int N, int nr, double2 *I,
                    const double *scale, cudaStream_t st);
void launch_resid(const double2 *V, const double2 *y, double2 *r, int N, int nr, double *partial, unsigned *counters,
                  double *out_norm, cudaStream_t st);
template <typename R>
void launch_to_inner(const double2 *src, void *dst, int N, int nr, const double *rnorm, const int *mask,
                     cudaStream_t st);
// ldv: per-RHS vector stride (lattice unknowns first, then any margin).
void launch_ports(const double2 *I, const double2 *V, int nel, int b, int nr, int pb, double z0, double2 *Za,
                  double2 *Gam, unsigned *err, long long ldv, cudaStream_t st);

}  // namespace moma
