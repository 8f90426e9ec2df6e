// Host-side declarations shared by the translation units of libmoma.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fft.cuh"

namespace moma {

// ---------------------------------------------------------------- FFT ----
// Device tables of one transform length: twiddles (both precisions) and
// the digit-reversal permutation.
struct FftTables {
  FftPlan plan;
  double2 *tw64 = nullptr;  // [M]
  float2 *tw32 = nullptr;   // [M]
  dfl2 *twdf = nullptr;     // [M] twiddles as double-FP32 pairs
  int *pos = nullptr;       // [M]
  std::vector<float2> tw32_host;  // host copy of tw32 (kernel-parameter twiddles of fftreg.cu)
};

FftPlan make_plan(int M);
std::vector<int> digit_reversal(const FftPlan &pl);
bool smooth_235(int m);
int next_smooth(int n);

// A batch of 1D transforms along one axis of a strided array.  Line
// (o1, o2), inner index j, axis position m sits at
//   base + o1*s1 + o2*s2 + m*sm + j        (element units).
struct AxisPass {
  const void *in = nullptr;
  void *out = nullptr;
  void *out2 = nullptr;    // optional second output (always c64)
  long long in_s1 = 0, in_s2 = 0, in_sm = 0;
  long long out_s1 = 0, out_s2 = 0, out_sm = 0;
  int n1 = 1, n2 = 1, ninner = 0;
  int nin = 0;             // loaded points (the rest of the M-line is zero)
  int nout = 0;            // stored points
  int in_mode = 0;         // 0: point m <- axis index m; 1: circulant gather of 2N-1 offsets
  int out_mode = 0;        // 0: point k -> axis index k; 1: k -> slot_of[k*slot_mul + o1]; 2: symmetric scatter
  const int *slot_of = nullptr;
  int slot_mul = 0;
  int remap_b = 0, remap_ld = 0;  // out_mode 1: inner j -> (j / remap_b) * remap_ld + j % remap_b
  const int *inner_in_map = nullptr;  // if set: input inner offset of line j is inner_in_map[j]
  const int2 *bin_slot = nullptr;     // out_mode 2: per bin (stored slot, 0 direct | 1 transposed | 2 both)
  const int2 *tri = nullptr;          // out_mode 2: inner j -> block entry (i, j), i <= j
  int inverse = 0;         // conj(DFT(conj x)) / M
  int refft_keep = 0;      // >0: inverse, keep points < refft_keep, zero the rest, forward again
  int in_c128 = 1, out_c128 = 1;  // element types of in / out: 0 c64, 1 c128, 2 dfl2
  const int *live = nullptr;       // if set and *live == 0 the pass does nothing
  int G = 0;                       // threads per line (0 = heuristic; set by the autotuner)
};

// Launch one axis pass computing in precision R (float or double).  Plain
// c64 passes of length M <= 64 run on the register-resident kernels of
// fftreg.cu (one thread, or 2, 4, 8 lanes, per line).
template <typename R>
void launch_axis_pass(const AxisPass &p, const FftTables &t, cudaStream_t st);
bool axis_reg_supported(const AxisPass &p, int M);
// Lanes sharing one line in the register passes: P in {1, 2, 4, 8} with
// P^2 | M (valid), and the choice for a pass (a fixed rule of its geometry).
bool axis_lanes_valid(int M, int P);
int lanes_per_line(const AxisPass &p, int M);
void launch_axis_reg(const AxisPass &p, const FftTables &t, cudaStream_t st);

// Two-dimensional lattice transforms in one launch (lattice2d.cu): mode 0
// F2 lattice -> bins, 1 I2 bins -> lattice, 2 I2MF2 bins -> bins (inverse,
// lattice mask, forward).  Lattice vectors [nr][ldv] with element (y, x) at
// (y Nx + x) b; bins [My][Mx][nr][b].  R = float (c64) or double (c128).
struct Lattice2D {
  int mode = 0;
  const void *in = nullptr;
  void *out = nullptr;
  int nx = 0, ny = 0, b = 0, nr = 0;
  long long ldv = 0;
  const int *live = nullptr;  // if set and *live == 0 the transform does nothing
  int J = 0;                  // basis indices per CTA (1, 2, 4; 0 = heuristic)
  int threads = 0;            // threads per CTA (0 = 256)
};
template <typename R>
bool lattice2d_fits(int Mx, int My, int J);

// The same three c64 transforms on thread-block clusters (lattice_cluster.cu):
// square M x M grids (M = 32, 48, 64), eight CTAs per group of eight basis
// indices exchanging the half-transformed grid in distributed shared memory.
// PX, PY: lanes per x / y line, those of the per-axis register passes for
// the same geometry (lanes_per_line), which makes the results bitwise equal
// to theirs.
struct LatticeCluster {
  int mode = 0;  // 0 F2, 1 I2, 2 I2MF2 (as Lattice2D)
  const void *in = nullptr;
  void *out = nullptr;
  int nx = 0, ny = 0, b = 0, nr = 0;
  long long ldv = 0;
  const int *live = nullptr;  // if set and *live == 0 the transform does nothing
  int PX = 0, PY = 0;
};
bool lattice_cluster_supported(int Mx, int My, int nx, int ny, int PX, int PY);
void launch_lattice_cluster(const LatticeCluster &p, const FftTables &fx, const FftTables &fy, cudaStream_t st);
template <typename R>
void launch_lattice2d(const Lattice2D &p, const FftTables &fx, const FftTables &fy, cudaStream_t st);

// --------------------------------------------------------- bin product ----
struct BinProduct {
  const void *Z = nullptr;    // pair storage [Bp][b][ldb]
  const int2 *pairs = nullptr;  // [Bp] (ka, kb), ka <= kb
  const void *x = nullptr;    // bins [B][nr][b]
  void *y = nullptr;          // bins [B][nr][b]
  int Bp = 0, b = 0, ldb = 0, nr = 0;
  int herm = 0;
  unsigned *err = nullptr;
  const int *live = nullptr;  // if set and *live == 0 the product does nothing
  int TR = 0, NS = 0;         // rows per tile / pipeline stages (0 = heuristic; autotuner)
  int occ = 1;                // CTAs per SM (2, 3: small-tile variants, <= 2 RHS per chunk, b <= 128; 3 for c64 only)
};
template <typename R>
void launch_bin_product(const BinProduct &p, int num_sms, cudaStream_t st);
// The c64 product for b = 64, 96, ..., 256 with row and column warps
// (binprod_rc.cu); launch_bin_product<float> takes it for those sizes.
bool bin_rc_supported(int b);
void launch_bin_rc(const BinProduct &p, int num_sms, cudaStream_t st);
// The same in double-FP32 (stored bins and vectors dfl2) where its stages
// fit shared memory (b <= 160); launch_bin_product<dfl> takes it there.
bool bin_rc_dfl_supported(int b);
void launch_bin_rc_dfl(const BinProduct &p, int num_sms, cudaStream_t st);

// Tensor-core products (tcgen05, 3xTF32) for many right-hand sides.  A
// TcMats holds T complex b x b matrices, each split into exact TF32 pairs
// (hi, lo: [T][b][2b] floats, interleaved complex rows), with TMA maps.
// raw: hi (and lo, if set) are instead plain c64 matrices [T][b][ld] that the
// kernel splits in shared memory; an item t >= T of the product's amap
// selects matrix t - T of lo (the pair store and its transpose).
struct TcMats {
  int b = 0, T = 0;
  float *hi = nullptr, *lo = nullptr;
  CUtensorMap map_hi{}, map_lo{};
  bool raw = false;
  int ld = 0;
};
// y_t[j] = op(A_{amap(t)}) x_t[j] for items t < T, RHS j < nr; op = conj
// if conj.  x_t[j][k] at x + t*x_ts + j*x_rs + k (complex64), same for y.
struct TcProduct {
  const void *x = nullptr;
  void *y = nullptr;
  long long x_ts = 0, x_rs = 0, y_ts = 0, y_rs = 0;
  int nr = 0, conj = 0;
  const int *amap = nullptr;  // nullptr = identity
  unsigned *err = nullptr;
  const int *live = nullptr;
  int check_finite = 0;       // raw A: DEVERR_NONFINITE into err for a non-finite entry of A
  int items = 0;              // items t of x and y (0: the TcMats' T; amap indexes the matrices)
};
bool tc_supported(int b);
// Raw c64 matrices (rows of ld complex values) as the A operand, split in
// shared memory: hi = Z64 (items < T), lo = Z64T (items T .. 2T-1) or null.
void tc_raw(TcMats &m, const void *Z64, const void *Z64T, int ld);
// Z64T[s] = Z64[s]^T for the Bp stored b x b blocks (row stride ld).
void tc_transpose_pairs(const void *Z64, void *Z64T, int Bp, int b, int ld, cudaStream_t st);
size_t tc_bytes(int T, int b);  // hi + lo
// X_e and X_e^H from the packed inverse factors (c64).
void tc_split_factor(TcMats &X, TcMats &XH, const void *Xpk, size_t x_stride, cudaStream_t st);
void launch_tc_product(const TcMats &m, const TcProduct &P, int num_sms, cudaStream_t st);

// ------------------------------------------------------ preconditioner ----
// G_D = Z_D^H Z_D for every offset, output FP64 [nD][b][b].
template <typename R>
void launch_gram(const void *blocks, int blocks_c128, int nD, int b, double2 *G, cudaStream_t st);
// Box sums P_e (Eq. 37) by separable sliding windows, lower triangles only
// (row-major, b(b+1)/2 entries per element): G_D from S (FP64 [nD][b][b],
// summed in FP64) or, if Y is set, conj(Y_{-D}) (the tensor-core Gram
// products of the reflected offsets, c64, summed in double-FP32).  W holds
// box_window_entries() 16-byte complex entries: the row windows, then the
// P_e ([Ny][Nx][b(b+1)/2], at box_sums_of(W)), stored as dfl2 if df (the
// double-FP32 factorisation reads them) else as double2.
size_t box_window_entries(int nx, int ny, int b);
void launch_box_sums(const double2 *S, const float2 *Y, int nx, int ny, int b, double2 *W, bool df, cudaStream_t st);
const double2 *box_sums_of(const double2 *W, int nx, int ny, int b);
// Cholesky of every P_e (box sums in the precision df selects): L_e (packed
// lower, column-major, FP64) into Lpk.  df: double-FP32 arithmetic.
void launch_box_cholesky(const double2 *Pbox, int nel, int b, double2 *Lpk, unsigned *err, bool df, cudaStream_t st);
// Full P_e (b x b, FP64) of one element from the box sums.
void launch_box_one(const double2 *Pbox, int nx, int b, int ex, int ey, bool df, double2 *out, cudaStream_t st);
// Inverse factor X_e = L_e^{-1}, packed column-major lower (as L_e), in precision R.
// Qb (c64 only, may be null): also P_e^{-1} = X_e^H X_e in the blocked layout
// of launch_precond_blk; returns whether it was written (the blocked c64
// kernel, b a multiple of 8 up to 160), else launch_pinv_pack must form it.
template <typename R>
bool launch_tri_inverse(const double2 *Lpk, int nel, int b, void *X, size_t x_stride, cudaStream_t st,
                        void *Qb = nullptr);
// y_e = X_e^H X_e x_e for each element; vectors: RHS q, element e, basis k at
// q * vstride + voff + e * b + k (vstride <= 0: nel * b).
template <typename R>
void launch_precond_apply(const void *X, size_t x_stride, int nel, int b, int nr, const void *x, void *y,
                          unsigned *err, const int *live, long long vstride, long long voff, cudaStream_t st);

// Streaming c64 application of P_e^{-1} = X_e^H X_e, stored Hermitian in
// 8 x 8 blocks (precond_blk.cu): one persistent CTA per SM, a ring of bulk
// copies, one pass per element.  launch_pinv_pack forms the blocks from the
// packed inverse factors (c64, column-major lower, x_stride entries apart).
size_t xblk_entries(int b);  // complex entries per element of the blocked P_e^{-1}
bool precond_blk_supported(int b, int nr, long long vstride, long long voff);
void launch_pinv_pack(const void *Xpk, size_t x_stride, int nel, int b, void *Qb, cudaStream_t st);
void launch_precond_blk(const void *Qb, int nel, int b, int nr, const void *x, void *y, unsigned *err,
                        const int *live, long long vstride, long long voff, int num_sms, cudaStream_t st);

// -------------------------------------------------------------- margin ----
// y += margin terms of Z (herm = 0) or Z^H (herm = 1) for vectors
// [lattice N | margin nm] with per-RHS stride ldv; Z_B [nm][N], Z_C [nm][nm].
template <typename R>
void launch_margin_apply(const void *ZB, const void *ZC, int nm, int N, long long ldv, int nr, int herm,
                         const void *x, void *y, cudaStream_t st);
// P_C = conj(Z_B) Z_B^T + Z_C^H Z_C (FP64, full nm x nm in P) and its
// Cholesky factor (packed lower column-major in Lpk); nm <= 1024.
void launch_margin_precond_build(const double2 *ZB, const double2 *ZC, int nm, int N, double2 *P, double2 *Lpk,
                                 unsigned *err, cudaStream_t st);

// ------------------------------------------------------- port matrix ----
// ldv: per-RHS vector stride (lattice unknowns first, then any margin).
void launch_unit_ports(double2 *V, int nel, int b, int pb, int j0, int nq, long long ldv, cudaStream_t st);
void launch_gather_ports(const double2 *I, int nel, int b, int pb, int j0, int nq, double2 *Y, long long ldv,
                         cudaStream_t st);
// In-place inverse of the n x n row-major complex matrix A (FP64
// Gauss-Jordan, partial pivoting); perm [n], colk [n] scratch.
void launch_invert(double2 *A, int n, int *perm, double2 *colk, unsigned *err, cudaStream_t st);

// ---------------------------------------------------------- predictors ----
void launch_row_phase(double2 *V, int nx, int nel, int b, int pb, int q0, int nq, int Q, long long ldv,
                      cudaStream_t st);
void launch_column_coupling(const double2 *gamma, int Q, int nmax, double2 *C, cudaStream_t st);
void launch_s_ideal(double2 *S, int nx, int ny, double2 s_cc, double2 s1, double kd, cudaStream_t st);
// Z = z0 (I + S)(I - S)^{-1}; work holds n*n + n double2 and n ints.
void launch_z_from_s(const double2 *S, int n, double z0, double2 *Z, double2 *work, unsigned *err, cudaStream_t st);

// ------------------------------------------------------------- Krylov ----
struct ArnoldiCtl;  // device-side control block (krylov.cu)
}  // namespace moma
