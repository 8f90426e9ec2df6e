/*
 * moma.h -- C ABI of the B300 solver for regular finite arrays whose Method
 * of Moments matrix is multilevel block-Toeplitz (MBT).
 *
 * Problem (Sec. II-A and Eq. 15 of arXiv 2608.17844): an Nx x Ny lattice of
 * identical elements, b basis functions per element.  The impedance matrix Z
 * couples observation element m and source element n through a b x b block
 * that depends only on the lattice offset m - n, so Z is fully described by
 * its (2Nx-1)(2Ny-1) unique offset blocks (Eq. 1, Fig. 1).  The library
 * solves Z I = V and forms the port quantities (Eqs. 16-19).
 *
 * Method: Z is applied as a 2D lattice FFT convolution of its circulant
 * embedding (Eq. 3), with Z^H served from the same stored bins through the
 * Hermitian commutation property (Eq. 6).  The system is solved through the
 * preconditioned normal equations P^{-1} Z^H Z I = P^{-1} Z^H V (Sec. III-A)
 * with P the block diagonal of Z^H Z (Eq. 37), Cholesky-factored once, using
 * restarted GMRES inside an FP64 iterative-refinement loop on V - Z I.
 *
 * Conventions shared by every entry point
 *  - Complex numbers are interleaved (re, im): "c128" = two doubles,
 *    "c64" = two floats.
 *  - Offset blocks: [2Ny-1][2Nx-1][b][b] row-major; offset (dx, dy) sits at
 *    index (dy + Ny - 1, dx + Nx - 1); row = observation basis.
 *  - Vectors: [nrhs][Ny][Nx][b] row-major; element e = mx + Nx*my, unknown
 *    e*b + i (the two-level ordering of Eq. 2).
 *  - Every buffer argument may be host or device memory of the current CUDA
 *    device; the library inspects the pointer.  The caller owns all buffers
 *    it passes; the library never keeps a caller pointer past the call.
 *  - All GPU work runs on the stream given at creation.  Calls return after
 *    their results are visible to the caller (host results copied, device
 *    results complete on that stream).
 *  - Status codes are returned; moma_last_error() gives a thread-local
 *    message for the last failing call on that thread.  No C++ exception
 *    crosses the ABI.  Calls on one handle are not thread-safe; distinct
 *    handles are independent.
 */
#ifndef MOMA_H
#define MOMA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MOMA_OK = 0,
    MOMA_ERR_ARG = 1,           /* invalid argument (sizes, null pointers, enum values) */
    MOMA_ERR_STATE = 2,         /* call order violated, e.g. solve before set_blocks */
    MOMA_ERR_OOM = 3,           /* device allocation failed */
    MOMA_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    MOMA_ERR_NOT_PD = 5,        /* a preconditioner block lost positive definiteness */
    MOMA_ERR_NOT_CONVERGED = 6, /* iteration limits reached before the tolerance */
    MOMA_ERR_BREAKDOWN = 7,     /* Krylov breakdown with the residual above tolerance */
    MOMA_ERR_NONFINITE = 8,     /* NaN/Inf in an input or a result */
    MOMA_ERR_TIMEOUT = 9        /* a bounded device wait gave up */
} moma_status;

typedef enum { MOMA_C128 = 0, MOMA_C64 = 1 } moma_dtype;

typedef enum {
    MOMA_PREC_FP64 = 0,  /* plain: every stage in FP64 / complex128 */
    MOMA_PREC_MIXED = 1  /* inner GMRES, FFTs and bin products in FP32/c64;
                            FP64 for the Hessenberg least squares, the
                            storage of the Cholesky factor and the final
                            subtraction of the refinement residual V - Z I.
                            The FP64-class stages -- the transform into the
                            c128-class bins, the residual's product Z I and
                            the block Cholesky factorisation -- run in
                            double-FP32 arithmetic (two floats, ~48
                            significant bits) by default, or in FP64 with
                            MOMA_FLAG_FP64_RESIDUAL. */
} moma_precision;

typedef enum {
    MOMA_OP_Z = 0,      /* y = Z x                         (Eq. 3)            */
    MOMA_OP_ZH = 1,     /* y = Z^H x, bins conjugate-transposed on the fly (Eq. 6) */
    MOMA_OP_NORMAL = 2  /* y = P^{-1} Z^H Z x              (Sec. III-A)      */
} moma_op;

typedef struct moma_array moma_array; /* opaque; owns all device state */

enum {
    MOMA_FLAG_NO_GRAPHS = 1,     /* launch the inner steps directly instead of replaying CUDA graphs */
    MOMA_FLAG_NO_AUTOTUNE = 2,   /* no launch-shape timing trials: shapes tuned earlier in this
                                    process for the same device, lattice, b, precision and RHS
                                    count, else the built-in heuristics (arrays of the serving
                                    loop are created this way); shapes never change results */
    MOMA_FLAG_NO_TENSOR = 4,     /* no tensor-core path: c64 bin products, preconditioner apply
                                    and (set-up) Gram products on the CUDA cores */
    MOMA_FLAG_TENSOR_ALWAYS = 8, /* c64 bin products on the tensor cores from one RHS up
                                    (default: from 16 RHS; MIXED arrays, 128 <= b <= 256, b even) */
    MOMA_FLAG_FP64_RESIDUAL = 16, /* MIXED arrays: compute the block-bin transform, the refinement
                                    residual's Z I (bin product and FFTs) and the block Cholesky in
                                    FP64 instead of double-FP32 (slower on B300, whose FP64 rate is
                                    ~1/58 of FP32; results agree to ~1e-13) */
    MOMA_FLAG_AXIS_FFT = 32,     /* lattice transforms of the c64 / FP64 products as one launch per
                                    lattice axis instead of one 2D launch per transform (the 2D
                                    launches are the default: on thread-block clusters for square
                                    c64 grids of 32, 48 or 64 per axis, whose results are bitwise
                                    those of the per-axis passes; in shared memory where a larger
                                    grid fits it) */
    MOMA_FLAG_PRECOND_PER_ELEMENT = 64, /* c64 preconditioner apply with one CTA per element instead of
                                    the streaming kernel (default for even b <= 160 and fewer
                                    than 16 RHS) */
    MOMA_FLAG_SPLIT_ARNOLDI = 128 /* GMRES orthogonalisation as three sweep launches and a scaling
                                    launch per Arnoldi step instead of one cooperative launch
                                    (the default where its grid fits on the device at once);
                                    results are bitwise the same */
};
/* The tensor-core products (MIXED arrays): every circulant bin's block
 * Zhat_k (Eq. 3) is kept whole as a pair of TF32 values (hi + lo) and
 * multiplied with the RHS block by tcgen05 MMAs (3xTF32: hi*hi + hi*lo +
 * lo*hi, FP32 accumulation), y_k = Zhat_k x_k, or conj(Zhat_{-k}) x_k for
 * Z^H; the block preconditioner is applied the same way as X_e^H (X_e x_e)
 * with X_e = L_e^{-1} kept whole.  The split matrices (16 b^2 (B + 2 Nel)
 * bytes) are built on the first call with enough RHS after moma_set_blocks
 * and kept until the next one. */

typedef struct {
    int precision; /* moma_precision */
    int mx, my;    /* circulant sizes; 0 = smallest 2^a 3^b 5^c >= 2N-1.
                      Any M >= 2N-1 embeds Z exactly (Sec. II-A uses 2N-1). */
    int restart;   /* GMRES restart length m; 0 = 50 */
    int flags;     /* MOMA_FLAG_* */
} moma_options;

typedef enum {
    MOMA_SOLVER_GMRES = 0, /* restarted GMRES on P^{-1} Z^H Z I = P^{-1} Z^H V (Sec. III-A, "new M1") */
    MOMA_SOLVER_PCG = 1    /* preconditioned CG on Z^H Z I = Z^H V with preconditioner P (Sec. II-C);
                              O(1) vectors per RHS */
} moma_solver;

typedef struct {
    double tol;       /* per-RHS relative true residual ||V - Z I|| / ||V||; 0 = 1e-10 */
    double inner_tol; /* relative reduction of the inner residual per refinement step
                         (GMRES: preconditioned; PCG: ||Z^H (r - Z d)||); 0 = 1e-5 (mixed)
                         or tol/10 (FP64) */
    int max_outer;    /* refinement steps (each one inner solve); 0 = 30 */
    int warm_start;   /* nonzero: I holds an initial guess on entry */
    int solver;       /* moma_solver */
    int max_inner;    /* PCG iterations per refinement step; 0 = 500 (GMRES: the restart) */
} moma_solve_opts;

typedef struct {
    int outer_iters;         /* refinement steps taken (true-residual evaluations - 1) */
    int inner_iters;         /* total Arnoldi steps over all refinement steps */
    int converged;           /* 1 if every column met tol */
    double max_rel_residual; /* max over columns of the final FP64 ||V - Z I|| / ||V|| */
    double first_inner_reduction; /* max over columns of the inner residual estimate after
                                     the first inner cycle, relative to its start */
} moma_solve_info;

/* Create a solver for an nx x ny lattice with b bases per element.
 * The circulant embedding sizes Mx, My default to the smallest 2^a 3^b 5^c
 * >= 2N - 1 along each axis (Sec. II-A: any size >= 2N - 1 embeds the MBT
 * product exactly); opt->mx, opt->my override them (each >= 2N - 1).
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Allocates the device store for the transformed bins (c128, plus c64 in
 * MIXED mode), the factored preconditioner and the workspaces.
 * Errors: MOMA_ERR_ARG (nx, ny, b < 1, b > 256, bad options), MOMA_ERR_OOM. */
moma_status moma_create_array(int nx, int ny, int b, const moma_options *opt,
                              void *cuda_stream, moma_array **out);

/* Load the offset blocks (Eq. 1) and build everything derived from them:
 * the transformed first column of the circulant embedding, one block per
 * (k, -k) bin pair since Zhat_{-k} = Zhat_k^T (Eqs. 3, 6, 11); the blocks
 * of P = blockdiag(Z^H Z) as box sums (sliding windows over the offset
 * grid) of the offset Gram products Z_D^H Z_D (Eq. 37); their Cholesky factors P_e = L_e L_e^H
 * (Sec. III-A) and the inverse factors used to apply P^{-1}.
 * blocks: [2Ny-1][2Nx-1][b][b] of dtype (moma_dtype), offset (dx, dy) at
 * index (dy + Ny - 1, dx + Nx - 1), host or device.  The library assumes
 * reciprocity, Z_{-D} = Z_D^T (Sec. II-D: the MoM matrix is symmetric).
 * From host memory only the offsets with dy >= 0 are read (Ny (2Nx - 1)
 * blocks, copied in chunks that overlap the transform and the Gram
 * products); the rows dy < 0 are completed on the device as transposes.
 * A device buffer is read whole and must stay valid for the call only.
 * In MIXED arrays the c128-class bins used by the refinement residual are
 * computed and stored as double-FP32 pairs (~48 significant bits), the
 * Cholesky factorisation runs in the same arithmetic (FP64 output), and for
 * c64 blocks with 128 <= b <= 256 the Gram products run on the tensor cores
 * (3xTF32); the plain FP64 path is FP64 throughout.
 * Errors: MOMA_ERR_NONFINITE (NaN/Inf in the blocks read), MOMA_ERR_NOT_PD. */
moma_status moma_set_blocks(moma_array *a, const void *blocks, int dtype);

/* Apply an operator to nrhs vectors x -> y (layout [nrhs][Ny][Nx][b]):
 * MOMA_OP_Z, y = Z x through the FFT product of the circulant embedding
 * (Eqs. 2-3); MOMA_OP_ZH, y = Z^H x from the same stored bins, conjugated at
 * multiplication time (Eq. 6); MOMA_OP_NORMAL, y = P^{-1} Z^H Z x, the
 * operator of the preconditioned normal equations (Sec. III-A).
 * dtype MOMA_C128 computes in FP64-class arithmetic from the c128 bins;
 * MOMA_C64 in FP32 from the c64 bins (MIXED arrays only).  MOMA_OP_NORMAL
 * runs in the array's inner precision (MOMA_C64 for MIXED arrays,
 * MOMA_C128 for FP64 arrays; MOMA_ERR_ARG otherwise).  All three need
 * set_blocks (MOMA_ERR_STATE otherwise). */
moma_status moma_matvec(moma_array *a, int op, int nrhs, const void *x, void *y, int dtype);

/* Allocation-free variant of moma_matvec for MOMA_OP_Z and MOMA_OP_ZH (no
 * counterpart in the paper; it exists for callers of this library).  Some
 * callers cannot let a library call allocate device memory once they are
 * running: another framework's caching allocator may already hold the free
 * memory, or a latency-bound loop cannot afford the implicit device
 * synchronisation of an allocation.  moma_matvec grows the handle's
 * workspace on demand; this entry point allocates nothing.  Its scratch (the
 * lattice and bin-vector buffers of the FFT product) is one fixed 32 MiB
 * device array compiled into the library, which every GPU that loads the
 * library holds until the process exits.
 *  - x, y: device memory only, layout [nrhs][Ny][Nx][b], dtype as in
 *    moma_matvec; host pointers are rejected with MOMA_ERR_ARG.
 *  - x and y must be on the device the array was created on (the one whose
 *    copy of the scratch array, stream and stored bins the product uses);
 *    buffers on another device are rejected with MOMA_ERR_ARG.
 *  - Scratch needed: align256(nrhs*Ny*Mx*b*s) + 2*align256(Mx*My*nrhs*b*s)
 *    bytes, s = 16 (MOMA_C128) or 8 (MOMA_C64), Mx, My the circulant sizes,
 *    align256 rounding up to a multiple of 256.  Requests above 32 MiB are
 *    rejected with MOMA_ERR_ARG and a message stating the bytes needed (call
 *    again with fewer RHS).
 *  - The first call on a device looks up the device address of the array
 *    (cudaGetSymbolAddress, with the array's device made current for that
 *    call and the caller's current device restored).  The address is cached
 *    for the life of the device's primary context: after a
 *    cudaDeviceReset, destroy and recreate the handles before calling again.
 *  - The call is synchronous (it waits for its stream before returning, to
 *    report device-side errors) and must not be called while the stream is
 *    being captured into a CUDA graph.
 *  - All calls in the process share the one array: calls whose GPU work
 *    overlaps (other streams, other handles, other threads) race on it.  The
 *    scratch is fully rewritten before it is read, so no state leaks from one
 *    call into the next.
 *  - The product always runs on the CUDA cores with the built-in launch
 *    shapes: its bin product is the streaming kernel moma_matvec uses below
 *    16 RHS.  From 16 RHS on a MIXED array with 128 <= b <= 256, moma_matvec
 *    switches its c64 product to the tensor cores (3xTF32), so the two
 *    results then differ by that path's rounding, ~2e-6 relative; below 16
 *    RHS, and for MOMA_C128, they agree to FP32 (c64) or ~1e-13 (c128)
 *    rounding.
 * Errors: as moma_matvec, plus MOMA_ERR_ARG for host pointers, buffers on
 * another device, MOMA_OP_NORMAL or oversized requests. */
moma_status moma_matvec_noalloc(moma_array *a, int op, int nrhs, const void *x, void *y, int dtype);

/* y = P^{-1} x with the factored block-diagonal preconditioner (Eq. 38
 * without margin, applied through L_e^{-H} L_e^{-1}). */
moma_status moma_apply_precond(moma_array *a, int nrhs, const void *x, void *y, int dtype);

/* Copy one transformed bin Zhat_k (b x b, c128 or c64) for circulant
 * frequency (kx, ky): the 2D DFT of the first block column of the circulant
 * embedding (Eqs. 3, 11), resolving the pair storage (transposed if k is
 * the stored partner, Zhat_{-k} = Zhat_k^T).  Inspection aid for tests. */
moma_status moma_get_bin(moma_array *a, int kx, int ky, int dtype, void *out);

/* Copy the preconditioner block P_e (b x b c128, full Hermitian) of element
 * (ex, ey) as built from Eq. 37.  Inspection aid for tests. */
moma_status moma_get_precond_block(moma_array *a, int ex, int ey, void *out);

/* Solve Z I = V (Eq. 15) for nrhs right-hand sides.
 * V, I: c128 [nrhs][Ny][Nx][b], host or device.  I is output (and the
 * initial guess if opts->warm_start).  opts, info may be NULL.
 * rel_residual: optional [nrhs] doubles receiving each column's final
 * FP64 relative residual.
 * Errors: MOMA_ERR_STATE (no blocks), MOMA_ERR_NONFINITE (V or iterate),
 * MOMA_ERR_NOT_CONVERGED (limits reached; I holds the best iterate). */
moma_status moma_solve(moma_array *a, int nrhs, const void *V, void *I,
                       const moma_solve_opts *opts, moma_solve_info *info,
                       double *rel_residual);

/* Port quantities (Eqs. 16-19): with delta-gap ports on basis port_basis,
 * I_p,e = I[q][e][port_basis], V_p,e likewise from V, and
 *   Z_a,e = V_p,e / I_p,e      (Eq. 17 with Z_p I_p = V_p, Eq. 18)
 *   Gamma_e = (Z_a,e - z0) / (Z_a,e + z0), z0 real (Eq. 19).
 * I, V: c128 [nrhs][Ny][Nx][b]; Za, Gamma: c128 [nrhs][Ny][Nx]; Gamma may
 * be NULL.  Errors: MOMA_ERR_NONFINITE if some I_p = 0 (that Z_a is NaN). */
moma_status moma_active_impedance(moma_array *a, int nrhs, const void *I, const void *V,
                                  int port_basis, double z0, void *Za, void *Gamma);

/* Passive port impedance matrix Z_p (Eq. 18): for every element port j
 * (basis port_basis), solve Z I = e_j (unit voltage on port j, zero on the
 * others) with the array's solver, in chunks of `chunk` RHS (0 = 64), and
 * gather column j of the port admittance Y_p (the port currents); then
 * Z_p = Y_p^{-1} by FP64 Gauss-Jordan elimination with partial pivoting.
 * Zp, Yp: c128 [Nel][Nel] row-major (element index e = mx + Nx*my), host or
 * device; either may be NULL.  Z_p is symmetric for a reciprocal Z.  With
 * Z_p, Eq. 17 gives Z_a for any port-current excitation. */
moma_status moma_port_impedance(moma_array *a, int port_basis, int chunk, const moma_solve_opts *opts, void *Zp,
                                void *Yp);

/* Array margin (Eq. 1): Z = [Z_A, Z_B^T; Z_B, Z_C] with Z_A the MBT element
 * part (moma_set_blocks), Z_B [nm][N] the margin-element coupling and Z_C
 * [nm][nm] the margin part (row-major, dtype moma_dtype, host or device;
 * copied).  Afterwards every vector of this array (V, I of moma_solve,
 * moma_matvec, moma_apply_precond, the port calls) is [nrhs][N + nm]: the
 * lattice unknowns in the usual order, then the nm margin unknowns.  The
 * preconditioner gains the margin block P_C = conj(Z_B) Z_B^T + Z_C^H Z_C
 * (Eq. 38; P_A stays the block diagonal of Z_A^H Z_A), factored in FP64.
 * nm = 0 removes the margin.  0 <= nm <= 1024.  Not supported by
 * moma_matvec_noalloc.  Errors: MOMA_ERR_ARG, MOMA_ERR_NONFINITE,
 * MOMA_ERR_NOT_PD (P_C). */
moma_status moma_set_margin(moma_array *a, int nm, const void *ZB, const void *ZC, int dtype);

/* ---- Error predictors (Sec. II-E, after Eq. 19) -------------------------
 * Element index e = mx + Nx*my; the centre c = (Nx/2, Ny/2) (integer
 * division); the border set E_B = the outermost ring of the lattice; "the
 * border element closest to c" = smallest Euclidean lattice distance, ties
 * to the element on the centre's row, then the smallest index. */

/* Column coupling C_n (Eq. 28; Eq. 30 is the same integral over scan angle
 * with psi = k d sin(theta)): solves the row-phase excitations
 * V_q[my][mx][port_basis] = exp(j mx psi_q) (Eq. 29), psi_q = -pi + 2 pi q / nq,
 * q < nq, with the array's solver (opts as moma_solve), takes the centre
 * element's active reflection coefficient Gamma_q (Eq. 19, reference z0) and
 * returns C[n + nmax] = (1/nq) sum_q Gamma_q exp(-j n psi_q) for
 * n = -nmax..nmax (trapezoidal rule; exact for trigonometric polynomials of
 * degree < nq).  C: c128 [2 nmax + 1]; gamma (nullable): c128 [nq]; host or
 * device.  Errors: MOMA_ERR_STATE before set_blocks, MOMA_ERR_ARG, solver
 * errors. */
moma_status moma_column_coupling(moma_array *a, int port_basis, int nq, int nmax, double z0,
                                 const moma_solve_opts *opts, void *C, void *gamma);

/* Eq. 31: Zp = z0 (I + S)(I - S)^{-1} for an n x n c128 row-major S (host or
 * device; Zp likewise), FP64 on the device (Gauss-Jordan inverse of I - S).
 * Allocates and frees its own scratch.  MOMA_ERR_NONFINITE if I - S is
 * singular. */
moma_status moma_s_to_z(const void *S, int n, double z0, void *Zp, void *cuda_stream);

/* The idealised scattering matrix behind xi_S (Eq. 36): S[i][i] = s_cc;
 * S[i][j] = s1 dist^-2 exp(-j kd (dist - 1)) with dist the Euclidean
 * distance of elements i, j in units of the spacing d and kd = k d.  S: c128
 * [Nel][Nel], host or device. */
moma_status moma_s_ideal(int nx, int ny, double s_cc_re, double s_cc_im, double s1_re, double s1_im, double kd,
                         void *S, void *cuda_stream);

/* From Zp (c128 [Nel][Nel], host or device): out[0] = xi_Z predictor
 * |Zp[c][j]| / |Zp[c][c]| with j the border element closest to c (Eq. 25);
 * out[1] = max over j in E_B of |Zp[c][j]| / |Zp[c][c]| (Eq. 24);
 * out[2] = sum over n in E_B of |Zp[c][n]| (the border bound, Eq. 23). */
moma_status moma_xi_z(const void *Zp, int nx, int ny, double *out);

/* Eq. 36: xi_S = |Z[c][j]| / |Z[c][c]| for Z = z0 (I + S_ideal)(I - S_ideal)^{-1}
 * (moma_s_ideal, moma_s_to_z), j the border element closest to c. */
moma_status moma_xi_s(int nx, int ny, double s_cc_re, double s_cc_im, double s1_re, double s1_im, double kd,
                      double z0, double *xi_s);

/* Runtime instrumentation (no counterpart in the paper).
 * Per-kernel timing over the calls made since moma_profile(a, 1), measured
 * with CUDA events recorded on the array's stream around each launch of a
 * kernel family.  kernel: 0 = c64 bin product, 1 = c128 bin product,
 * 2 = preconditioner apply, 3 = c64 lattice FFT passes, 4 = block-bin
 * transform (set-up), 5 = c128 lattice FFT passes, 6 = offset Gram
 * products, 7 = box sums, 8 = Cholesky, 9 = inverse
 * factors, 10 = Arnoldi/Givens/update kernels, 11 = residual and
 * conversion kernels, 12 = tensor-core c64 bin product, 13 = tensor-core
 * preconditioner apply.  Writes the number of
 * timed launches and their total milliseconds.  moma_profile(a, 0) stops
 * timing; either call resets the counters. */
moma_status moma_profile(moma_array *a, int enable);
moma_status moma_kernel_stats(moma_array *a, int kernel, long long *launches, double *total_ms);

/* Device time of one operator application, measured back to back (runtime
 * instrumentation, no counterpart in the paper).  After one untimed
 * application, `reps` applications are captured as one CUDA graph on the
 * solver's internal stream (as the solve replays its inner steps), replayed
 * once untimed and once between two CUDA events, on the solver's own
 * workspace (contents irrelevant: no kernel's run time depends on the
 * values), so the figure is device execution time without host launch gaps
 * or per-launch event overhead.  Arrays created with MOMA_FLAG_NO_GRAPHS
 * time `reps` direct launches on the array's stream instead.  what:
 *   MOMA_TIME_Z       one c64 Z application: lattice FFT passes + bin product (Eq. 3)
 *   MOMA_TIME_BIN     the c64 per-bin product alone
 *   MOMA_TIME_PRECOND the c64 preconditioner apply P^{-1} (Eq. 38)
 *   MOMA_TIME_NORMAL  the c64 normal operator P^{-1} Z^H Z (Sec. III-A)
 * MIXED arrays after set_blocks; nrhs RHS (the kernels the solve would
 * take for that many RHS).  Writes microseconds per application. */
enum { MOMA_TIME_Z = 0, MOMA_TIME_BIN = 1, MOMA_TIME_PRECOND = 2, MOMA_TIME_NORMAL = 3 };
moma_status moma_time_operator(moma_array *a, int what, int nrhs, int reps, double *us_per_application);

/* Rebind the array to another CUDA stream (the old stream is synchronised
 * first).  Lets a pool of workers reuse resident arrays on their streams.
 * Runtime plumbing, no counterpart in the paper. */
moma_status moma_set_stream(moma_array *a, void *cuda_stream);

/* Text summary of the launch shapes the autotuner picked for this array
 * (empty before the first solve).  Each solve first times candidate shapes
 * of the bin product (rows per staged tile, pipeline stages, CTAs per SM)
 * and of every lattice-FFT pass (threads per line) on its own workspace,
 * once per RHS count, and keeps the fastest.  No counterpart in the paper. */
moma_status moma_tuning_report(const moma_array *a, char *buf, size_t len);

/* The CUDA stream the array currently runs on (runtime plumbing). */
void *moma_array_stream(const moma_array *a);

/* Ragged batches (no counterpart in the paper): n independent arrays of
 * uneven sizes processed concurrently.  `workers` host threads (0 = 8),
 * each with its own CUDA stream, take the next array; each array is bound
 * to the worker's stream for the call and returned to its own stream after,
 * so small problems fill the GPU together.  statuses (optional, [n])
 * receives each array's status; the return value is the first failure.
 * moma_set_blocks_batch: blocks[i] / dtypes[i] for arrays[i]; with
 * release_setup the set-up scratch is freed after each build.
 * moma_solve_batch: nrhs[i], V[i], I[i] as in moma_solve; infos optional [n]. */
moma_status moma_set_blocks_batch(int n, moma_array *const *arrays, const void *const *blocks, const int *dtypes,
                                  int release_setup, int workers, moma_status *statuses);
moma_status moma_solve_batch(int n, moma_array *const *arrays, const int *nrhs, const void *const *V,
                             void *const *I, const moma_solve_opts *opts, moma_solve_info *infos, int workers,
                             moma_status *statuses);

/* Memory management, no counterpart in the paper.
 * Free the set-up scratch kept after moma_set_blocks (device copy of the
 * blocks, block-transform intermediate, Gram products, box sums, FP64
 * Cholesky factors).  The bins and the inverse factors stay; solves and
 * products are unaffected; moma_get_precond_block then reports
 * MOMA_ERR_STATE.  For keeping many arrays resident. */
moma_status moma_release_setup(moma_array *a);

/* Memory management, no counterpart in the paper.
 * Upper estimate of the device bytes an array needs: stored bins, factors,
 * workspaces for nrhs right-hand sides and, if with_setup, the set-up
 * scratch.  0 on invalid sizes.  Used for admission by HBM footprint. */
size_t moma_estimate_bytes(int nx, int ny, int b, const moma_options *opt, int nrhs, int with_setup);

/* Runtime instrumentation (no counterpart in the paper).
 * Number of kernel launches issued on the array's stream since creation. */
long long moma_launch_count(moma_array *a);

/* Device bytes held by the array (bins, preconditioner, workspaces). */
size_t moma_device_bytes(const moma_array *a);

/* Release every device buffer, stream and event of the array (after its
 * stream has finished).  NULL is ignored.  No counterpart in the paper. */
void moma_destroy(moma_array *a);
/* Message of the last failing call on this thread (empty if none); the
 * string stays valid until the thread's next failing call.  No counterpart
 * in the paper. */
const char *moma_last_error(void);

/* ------------------------------------------------------------------ serving
 * Continuous batching of independent solve requests on the current device
 * (no counterpart in the paper; it serves many array/excitation problems).
 * A pool of `slots` worker threads, each on its own CUDA stream, takes the
 * next admissible request whenever it is free, so requests arriving while
 * others run start as soon as a slot and memory are available and their
 * GPU work overlaps.  Arrays (stored bins + factored preconditioner) stay
 * resident between requests under the caller's key; a request is admitted
 * when moma_estimate_bytes of its array fits the budget, evicting idle
 * resident arrays least recently used first.  Results equal those of a
 * stand-alone moma_solve (fixed reduction orders). */
typedef struct moma_server moma_server;

typedef struct {
    size_t max_device_bytes; /* budget for resident arrays and workspaces; 0 = 70% of free memory */
    int slots;               /* concurrent requests (worker threads / streams); 0 = 4 */
    int precision;           /* moma_precision of the arrays */
    int restart;             /* GMRES restart; 0 = 50 */
} moma_server_opts;

typedef struct {
    unsigned long long key; /* identity of (lattice, blocks): equal keys share a resident array */
    int nx, ny, b;
    const void *blocks;     /* [2ny-1][2nx-1][b][b]; read only when the key is not resident */
    int blocks_dtype;       /* moma_dtype */
    int nrhs;
    const void *V;          /* c128 [nrhs][ny][nx][b] */
    void *I;                /* c128 output, same layout */
    void *Za, *Gamma;       /* optional c128 [nrhs][ny][nx] port outputs (NULL to skip) */
    int port_basis;
    double z0;              /* 0 = 50 ohm */
    double tol;             /* 0 = 1e-10 */
} moma_request;             /* all buffers must stay valid until moma_server_wait returns the result */

typedef struct {
    int status;             /* moma_status of this request */
    int resident_hit;       /* 1 if the array was resident (no set-up) */
    double queue_ms, run_ms, total_ms;  /* submit->start, start->done, submit->done (host clock) */
    moma_solve_info info;
    char message[256];      /* error text if status != MOMA_OK */
} moma_result;

typedef struct {
    unsigned long long submitted, completed, hits, misses, evictions;
    int resident_arrays, queued;
    size_t resident_bytes, budget_bytes;
} moma_server_stats;

moma_status moma_server_create(const moma_server_opts *opt, moma_server **out);
/* Queue a request; returns immediately with a ticket. */
moma_status moma_server_submit(moma_server *s, const moma_request *r, unsigned long long *ticket);
/* Wait for a ticket's result (timeout_s < 0: forever); MOMA_ERR_TIMEOUT if
 * still running.  Each ticket's result is returned once. */
moma_status moma_server_wait(moma_server *s, unsigned long long ticket, double timeout_s, moma_result *out);
moma_status moma_server_get_stats(moma_server *s, moma_server_stats *out);
/* Drops queued requests, finishes running ones, frees everything. */
void moma_server_destroy(moma_server *s);

#ifdef __cplusplus
}
#endif
#endif /* MOMA_H */
