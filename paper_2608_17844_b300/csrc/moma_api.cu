// C ABI of libmoma: handle management, device memory, and the host-side
// orchestration of the set-up and solve pipelines (see include/moma.h).
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <memory>
#include <type_traits>
#include <thread>
#include <tuple>
#include <cstring>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "moma.h"
#include "krylov.h"
#include "noalloc_check.h"

using namespace moma;

namespace {

thread_local std::string g_last_error;

struct MomaError : std::runtime_error {
  moma_status st;
  MomaError(moma_status s, const std::string &m) : std::runtime_error(m), st(s) {}
};

#define CK(call)                                                                                      \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) {                                                                          \
      cudaGetLastError();                                                                             \
      throw MomaError(e_ == cudaErrorMemoryAllocation ? MOMA_ERR_OOM : MOMA_ERR_CUDA,                \
                      std::string(#call) + ": " + cudaGetErrorString(e_));                            \
    }                                                                                                 \
  } while (0)

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Grow-only device buffer.
struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
  void ensure(size_t bytes, size_t &total) {
    if (bytes <= cap) return;
    if (p) {
      cudaFree(p);
      total -= cap;
      p = nullptr;
      cap = 0;
    }
    void *q = nullptr;
    CK(cudaMalloc(&q, bytes));
    p = q;
    cap = bytes;
    total += bytes;
  }
  void release(size_t &total) {
    if (p) cudaFree(p);
    total -= cap;
    p = nullptr;
    cap = 0;
  }
  template <typename T> T *as() const { return reinterpret_cast<T *>(p); }
};

__global__ void nonfinite_kernel(const void *p, size_t n_real, int is_double, unsigned *err) {
  bool bad = false;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n_real; i += (size_t)gridDim.x * blockDim.x) {
    if (is_double ? !isfinite(reinterpret_cast<const double *>(p)[i]) : !isfinite(reinterpret_cast<const float *>(p)[i]))
      bad = true;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, DEVERR_NONFINITE);
}

// Element-type conversion c64 / c128 (n complex values).
__global__ void convert_kernel(const void *src, int src128, void *dst, int dst128, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double2 v = src128 ? reinterpret_cast<const double2 *>(src)[i]
                       : cvt<double2>(reinterpret_cast<const float2 *>(src)[i]);
    if (dst128) reinterpret_cast<double2 *>(dst)[i] = v;
    else reinterpret_cast<float2 *>(dst)[i] = cvt<float2>(v);
  }
}
void launch_convert(const void *src, int src128, void *dst, int dst128, size_t n, cudaStream_t st) {
  size_t g = (n + 255) / 256;
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  convert_kernel<<<(int)g, 256, 0, st>>>(src, src128, dst, dst128, n);
}

// Reciprocity completion of the staged blocks (Sec. II-D: Z_{-D} = Z_D^T):
// rows (dy index) m in [m0, m1) receive Z[m][ix] = Z[2Ny-2-m][2Nx-2-ix]^T.
template <typename C>
__global__ void reciprocal_fill_kernel(C *Z, int ndy, int ndx, int b, int m0) {
  __shared__ C tile[32][33];
  const int blk = blockIdx.z, m = m0 + blk / ndx, ix = blk % ndx;
  const size_t bb = (size_t)b * b;
  const C *src = Z + ((size_t)(ndy - 1 - m) * ndx + (ndx - 1 - ix)) * bb;
  C *dst = Z + ((size_t)m * ndx + ix) * bb;
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32, tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8)  // tile[r][tx] = src[j0 + r][i0 + tx]
    if (j0 + r < b && i0 + tx < b) tile[r][tx] = src[(size_t)(j0 + r) * b + i0 + tx];
  __syncthreads();
  for (int r = ty; r < 32; r += 8)  // dst[i0 + r][j0 + tx] = src[j0 + tx][i0 + r]
    if (i0 + r < b && j0 + tx < b) dst[(size_t)(i0 + r) * b + j0 + tx] = tile[tx][r];
}

enum {
  PK_BIN64 = 0, PK_BIN128 = 1, PK_PREC = 2, PK_FFT64 = 3, PK_BLOCKFFT = 4, PK_FFT128 = 5,
  PK_GRAM = 6, PK_BOX = 7, PK_CHOL = 8, PK_TRINV = 9, PK_KRYLOV = 10, PK_MISC = 11, PK_BINTC = 12, PK_PRECTC = 13, PK_N = 14
};

}  // namespace

struct moma_array {
  int nx = 0, ny = 0, b = 0, nel = 0, N = 0;
  // Array margin (Z = [Z_A, Z_B^T; Z_B, Z_C]): nm margin unknowns after the
  // N lattice unknowns of every vector; ldv = N + nm is the per-RHS stride.
  int nm = 0;
  long long ldv = 0;
  DevBuf mZB128, mZC128, mZB64, mZC64;  // Z_B [nm][N], Z_C [nm][nm] (FP64; c64 in MIXED)
  DevBuf mP, mL, mX;                    // P_C, its packed Cholesky factor, X_C = L_C^{-1} (inner precision)
  size_t mx_stride = 0;
  int Mx = 0, My = 0, B = 0, Bp = 0, ldb = 0;
  int prec = MOMA_PREC_MIXED, m = 50;
  // Arithmetic of the FP64-class stages of a MIXED array (the block-bin
  // transform into the c128-class bins, the refinement residual's Z I and the
  // block Cholesky): double-FP32 pairs (df = true, the default) or FP64
  // (MOMA_FLAG_FP64_RESIDUAL).  Always false for FP64 arrays.
  bool df = false;
  cudaStream_t st = nullptr;
  int dev = 0, num_sms = 148;
  size_t dev_bytes = 0;
  long long launches = 0;

  FftTables fx, fy;
  DevBuf tabs;      // twiddles / permutations of both plans
  DevBuf pairs, slot_of;
  DevBuf bin_slot, tri, tri_in;  // symmetric block-transform tables
  DevBuf Z128, Z64;  // pair storage [Bp][b][ldb]
  DevBuf Xinv;       // inverse factors, packed column-major, inner precision
  DevBuf Xblk;       // c64 P_e^{-1} = X_e^H X_e in 8 x 8 blocks for the streaming apply (precond_blk.cu)
  bool xblk_ready = false;
  // Tensor-core products (inner precision c64, many RHS): split full bins,
  // the partner table, split X_e and X_e^H; built on first use after
  // set_blocks.
  DevBuf tcA, tcP, partner;
  DevBuf tamap;  // tensor-core A item of every bin: [B] for Z, [B] for Z^H (pair store, or its transpose at + Bp)
  TcMats tcZ, tcX, tcXH;
  bool tc_ready = false;
  bool no_tensor = false;
  int tc_min_nr = 16;
  size_t x_stride = 0;
  bool have_blocks = false;

  // set-up workspace
  DevBuf blk, T, S, Lpk;
  DevBuf Wb;                     // box-sum windows when S cannot hold them
  const double2 *pbox = nullptr;  // the box sums P_e (lower triangles), in S or Wb
  bool pbox_df = false;           // ... stored as double-FP32 pairs
  cudaStream_t cs = nullptr;  // host-to-device copies of the blocks
  DevBuf gramY;               // tensor-core Gram products of the reflected offsets
  bool tgram = false;         // this set-up's Gram products ran on the tensor cores
  cudaEvent_t ev_cs0 = nullptr, ev_chunk[8] = {};
  // solve workspace
  int ws_nr = 0;
  DevBuf lat_in, lat_tmp, lat_u, t1, bx, by, Vk;
  DevBuf Iw, Vw, rw, yw;
  DevBuf kbuf;  // Krylov control arrays
  KrylovCtl ctl{};
  CgCtl cg{};
  std::vector<cudaGraphExec_t> cg_gexec;  // PCG iteration graphs (ring of poll slots)
  int cg_g_nr = -1;
  long long cg_step_launches = 0;
  double *rnorm = nullptr, *vnorm = nullptr, *rpart = nullptr;
  unsigned *rcount = nullptr;
  int *mask = nullptr;
  DevBuf errbuf;
  unsigned *err = nullptr;
  DevBuf one_blk;
  DevBuf portsb;  // Z_a and Gamma results [2][nr][nel]
  DevBuf zp_V, zp_I, zp_Y, zp_tmp;  // port-matrix solves
  // CUDA graphs of the inner Arnoldi steps (one per step index j, for the
  // RHS count g_nr), replayed on an internal capturable stream.
  bool use_graphs = true;
  cudaStream_t gs = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<cudaGraphExec_t> gexec;
  int g_nr = -1;
  // Captured step graphs kept per RHS count, so that calls alternating
  // between RHS counts (serving, batches) replay instead of re-capturing.
  struct GraphSet {
    std::vector<cudaGraphExec_t> g;
    long long step_launches = 0;
  };
  std::map<int, GraphSet> gmres_graphs, pcg_graphs;
  // Autotuned bin-product shapes per RHS count.
  struct TuneBin {
    int tr[2], ns[2], occ[2];
  };
  std::map<int, TuneBin> tune_by_nr;
  long long g_step_launches = 0;
  // Autotuned launch shapes (0 = built-in heuristic), per RHS count.
  int tuned_nr = -1;
  bool no_autotune = false;
  int tune_bin_tr[2] = {0, 0}, tune_bin_ns[2] = {0, 0}, tune_bin_occ[2] = {1, 1};  // [c64, c128]
  std::vector<std::pair<long long, int>> tune_axis;       // pass signature -> threads per line
  std::vector<std::pair<long long, int2>> tune_l2d;       // 2D transform signature -> (J, threads)
  bool axis_fft = false;  // lattice transforms one launch per axis instead of the 2D kernels
  bool no_blk_precond = false;  // c64 preconditioner through the per-element kernel only
  bool no_fused_arnoldi = false;  // CGS2 sweeps as separate launches
  std::string tune_log;
  const int *live = nullptr;  // operator kernels skip their work while *live == 0

  // pinned host mirrors
  int *h_nact = nullptr;  // ring of polled nact values
  double *h_norms = nullptr;
  unsigned *h_err = nullptr;
  std::vector<cudaEvent_t> poll_ev;

  // profiling
  bool prof = false;
  struct EvPair { cudaEvent_t a, b; int kind; };
  std::vector<EvPair> ev_pending;
  std::vector<cudaEvent_t> ev_free;
  long long st_launch[PK_N] = {0};
  double st_ms[PK_N] = {0};

  cudaEvent_t ev_get() {
    if (!ev_free.empty()) {
      cudaEvent_t e = ev_free.back();
      ev_free.pop_back();
      return e;
    }
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    return e;
  }
  void flush_events() {
    for (auto &p : ev_pending) {
      float ms = 0;
      if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
        st_ms[p.kind] += ms;
        st_launch[p.kind] += 1;
      } else {
        cudaGetLastError();
      }
      ev_free.push_back(p.a);
      ev_free.push_back(p.b);
    }
    ev_pending.clear();
  }
  template <typename F> void timed(int kind, F &&f) {
    if (!prof) {
      f();
      return;
    }
    cudaEvent_t a = ev_get(), b2 = ev_get();
    CK(cudaEventRecord(a, st));
    f();
    CK(cudaEventRecord(b2, st));
    ev_pending.push_back({a, b2, kind});
    if (ev_pending.size() > 8192) flush_events();
  }
};

namespace {

void check_launch(moma_array *a) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw MomaError(MOMA_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  a->launches += 1;
}

void build_tables(moma_array *a) {
  a->fx.plan = make_plan(a->Mx);
  a->fy.plan = make_plan(a->My);
  auto px = digit_reversal(a->fx.plan), py = digit_reversal(a->fy.plan);
  const int Ms[2] = {a->Mx, a->My};
  size_t bytes = 0;
  for (int M : Ms) bytes += (size_t)M * (sizeof(double2) + sizeof(float2) + sizeof(dfl2) + sizeof(int)) + 256;
  a->tabs.ensure(bytes, a->dev_bytes);
  std::vector<unsigned char> host(bytes, 0);
  size_t off = 0;
  FftTables *tt[2] = {&a->fx, &a->fy};
  const std::vector<int> *pp[2] = {&px, &py};
  for (int d = 0; d < 2; ++d) {
    const int M = Ms[d];
    double2 *t64 = reinterpret_cast<double2 *>(host.data() + off);
    tt[d]->tw64 = reinterpret_cast<double2 *>(a->tabs.as<unsigned char>() + off);
    off += (size_t)M * sizeof(double2);
    float2 *t32 = reinterpret_cast<float2 *>(host.data() + off);
    tt[d]->tw32 = reinterpret_cast<float2 *>(a->tabs.as<unsigned char>() + off);
    off += (size_t)M * sizeof(float2);
    off = (off + 15) & ~size_t(15);
    dfl2 *tdf = reinterpret_cast<dfl2 *>(host.data() + off);
    tt[d]->twdf = reinterpret_cast<dfl2 *>(a->tabs.as<unsigned char>() + off);
    off += (size_t)M * sizeof(dfl2);
    int *ps = reinterpret_cast<int *>(host.data() + off);
    tt[d]->pos = reinterpret_cast<int *>(a->tabs.as<unsigned char>() + off);
    off += (size_t)M * sizeof(int);
    off = (off + 255) & ~size_t(255);
    for (int t = 0; t < M; ++t) {
      const double ang = -2.0 * M_PI * (double)t / (double)M;
      t64[t] = make_double2(std::cos(ang), std::sin(ang));
      t32[t] = make_float2((float)t64[t].x, (float)t64[t].y);
      tdf[t].x = dfl(t64[t].x);
      tdf[t].y = dfl(t64[t].y);
      ps[t] = (*pp[d])[t];
    }
    tt[d]->tw32_host.assign(t32, t32 + M);
  }
  CK(cudaMemcpy(a->tabs.p, host.data(), bytes, cudaMemcpyHostToDevice));

  // Bin pairs {k, -k}; the smaller index is stored.
  std::vector<int> slot(a->B, -1);
  std::vector<int2> pr;
  for (int ky = 0; ky < a->My; ++ky)
    for (int kx = 0; kx < a->Mx; ++kx) {
      const int k = ky * a->Mx + kx;
      const int nk = ((a->My - ky) % a->My) * a->Mx + ((a->Mx - kx) % a->Mx);
      if (k <= nk) {
        slot[k] = (int)pr.size();
        pr.push_back(make_int2(k, nk));
      }
    }
  a->Bp = (int)pr.size();
  std::vector<int> part(a->B);
  for (int ky = 0; ky < a->My; ++ky)
    for (int kx = 0; kx < a->Mx; ++kx)
      part[ky * a->Mx + kx] = ((a->My - ky) % a->My) * a->Mx + ((a->Mx - kx) % a->Mx);
  a->partner.ensure(part.size() * sizeof(int), a->dev_bytes);
  CK(cudaMemcpy(a->partner.p, part.data(), part.size() * sizeof(int), cudaMemcpyHostToDevice));
  // Tensor-core A operand of bin k: its stored block (the lower member of a
  // pair) or the transpose of its partner's (item Bp + slot); Z^H reads the
  // partner's operand, conjugated (Eq. 6 with reciprocity).
  std::vector<int> am(2 * a->B);
  for (int k = 0; k < a->B; ++k) am[k] = slot[k] >= 0 ? slot[k] : a->Bp + slot[part[k]];
  for (int k = 0; k < a->B; ++k) am[a->B + k] = am[part[k]];
  a->tamap.ensure(am.size() * sizeof(int), a->dev_bytes);
  CK(cudaMemcpy(a->tamap.p, am.data(), am.size() * sizeof(int), cudaMemcpyHostToDevice));
  a->pairs.ensure(pr.size() * sizeof(int2), a->dev_bytes);
  a->slot_of.ensure(slot.size() * sizeof(int), a->dev_bytes);
  CK(cudaMemcpy(a->pairs.p, pr.data(), pr.size() * sizeof(int2), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(a->slot_of.p, slot.data(), slot.size() * sizeof(int), cudaMemcpyHostToDevice));

  // Block-transform tables: only entries (i <= j) are transformed; bin k
  // stores them directly if it is the stored member of its pair, the
  // partner -k scatters them transposed, a self-paired bin writes both.
  std::vector<int2> bs(a->B);
  for (int ky = 0; ky < a->My; ++ky)
    for (int kx = 0; kx < a->Mx; ++kx) {
      const int k = ky * a->Mx + kx;
      const int nk = ((a->My - ky) % a->My) * a->Mx + ((a->Mx - kx) % a->Mx);
      if (k == nk) bs[k] = make_int2(slot[k], 2);
      else if (k < nk) bs[k] = make_int2(slot[k], 0);
      else bs[k] = make_int2(slot[nk], 1);
    }
  const int b = a->b, nt = b * (b + 1) / 2;
  std::vector<int2> tri(nt);
  std::vector<int> tri_in(nt);
  int t = 0;
  for (int i = 0; i < b; ++i)
    for (int j = i; j < b; ++j, ++t) {
      tri[t] = make_int2(i, j);
      tri_in[t] = i * b + j;
    }
  a->bin_slot.ensure(bs.size() * sizeof(int2), a->dev_bytes);
  a->tri.ensure(tri.size() * sizeof(int2), a->dev_bytes);
  a->tri_in.ensure(tri_in.size() * sizeof(int), a->dev_bytes);
  CK(cudaMemcpy(a->bin_slot.p, bs.data(), bs.size() * sizeof(int2), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(a->tri.p, tri.data(), tri.size() * sizeof(int2), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(a->tri_in.p, tri_in.data(), tri_in.size() * sizeof(int), cudaMemcpyHostToDevice));
}

// ----------------------------------------------------- axis pass builders --
AxisPass pass_fx(moma_array *a, int nr, const void *in, void *out, int in128, int out128) {
  AxisPass p;
  p.in = in; p.out = out; p.n1 = nr; p.n2 = a->ny; p.ninner = a->b;
  p.in_s1 = a->ldv; p.in_s2 = (long long)a->nx * a->b; p.in_sm = a->b; p.nin = a->nx;
  p.out_s1 = (long long)a->ny * a->Mx * a->b; p.out_s2 = (long long)a->Mx * a->b; p.out_sm = a->b; p.nout = a->Mx;
  p.in_c128 = in128; p.out_c128 = out128;
  return p;
}
AxisPass pass_fy(moma_array *a, int nr, const void *in, void *out, int c128) {
  AxisPass p;
  p.in = in; p.out = out; p.n1 = nr; p.n2 = a->Mx; p.ninner = a->b;
  p.in_s1 = (long long)a->ny * a->Mx * a->b; p.in_s2 = a->b; p.in_sm = (long long)a->Mx * a->b; p.nin = a->ny;
  p.out_s1 = a->b; p.out_s2 = (long long)nr * a->b; p.out_sm = (long long)a->Mx * nr * a->b; p.nout = a->My;
  p.in_c128 = p.out_c128 = c128;
  return p;
}
AxisPass pass_iy(moma_array *a, int nr, const void *in, void *out, int c128) {
  AxisPass p;
  p.in = in; p.out = out; p.n1 = nr; p.n2 = a->Mx; p.ninner = a->b; p.inverse = 1;
  p.in_s1 = a->b; p.in_s2 = (long long)nr * a->b; p.in_sm = (long long)a->Mx * nr * a->b; p.nin = a->My;
  p.out_s1 = (long long)a->ny * a->Mx * a->b; p.out_s2 = a->b; p.out_sm = (long long)a->Mx * a->b; p.nout = a->ny;
  p.in_c128 = p.out_c128 = c128;
  return p;
}
AxisPass pass_ix(moma_array *a, int nr, const void *in, void *out, int c128, bool mask_refft, int out_code = -1) {
  AxisPass p;
  p.in = in; p.out = out; p.n1 = nr; p.n2 = a->ny; p.ninner = a->b; p.inverse = 1;
  p.in_s1 = (long long)a->ny * a->Mx * a->b; p.in_s2 = (long long)a->Mx * a->b; p.in_sm = a->b; p.nin = a->Mx;
  if (mask_refft) {
    p.refft_keep = a->nx;
    p.out_s1 = p.in_s1; p.out_s2 = p.in_s2; p.out_sm = p.in_sm; p.nout = a->Mx;
  } else {
    p.out_s1 = a->ldv; p.out_s2 = (long long)a->nx * a->b; p.out_sm = a->b; p.nout = a->nx;
  }
  p.in_c128 = c128;
  p.out_c128 = out_code < 0 ? c128 : out_code;
  return p;
}

template <typename R> constexpr int is64() { return sizeof(R) == 8 ? 1 : 0; }
// Storage code of the element type an R computation keeps between passes
// (0 = c64, 1 = c128, 2 = double-FP32 pairs) and of its lattice vectors
// (the double-FP32 path reads and writes c128 lattice vectors).
template <typename R> constexpr int st_code() {
  return std::is_same<R, float>::value ? 0 : (std::is_same<R, double>::value ? 1 : 2);
}
template <typename R> constexpr int lat_code() { return std::is_same<R, float>::value ? 0 : 1; }

long long axis_sig(const AxisPass &p, int M, int is64v) {
  long long h = is64v;
  for (long long v : {(long long)M, (long long)p.ninner, (long long)p.n1 * p.n2, (long long)p.nin,
                      (long long)p.nout, (long long)p.refft_keep, (long long)p.in_mode, (long long)p.out_mode,
                      (long long)p.inverse})
    h = h * 1000003LL + v;
  return h;
}

int tuned_G(const moma_array *a, long long sig) {
  for (auto &kv : a->tune_axis)
    if (kv.first == sig) return kv.second;
  return 0;
}

template <typename R>
void axis(moma_array *a, AxisPass p, const FftTables &t) {
  p.live = a->live;
  if (p.G == 0) p.G = tuned_G(a, axis_sig(p, t.plan.M, st_code<R>()));
  a->timed(is64<R>() ? PK_FFT128 : PK_FFT64, [&] { launch_axis_pass<R>(p, t, a->st); });
  check_launch(a);
}

template <typename R>
void binprod(moma_array *a, int nr, const void *x, void *y, int herm) {
  if (!is64<R>() && a->tc_ready && nr >= a->tc_min_nr) {
    // Bins [B][nr][b]; Z^H reads the partner bin, conjugated (Eq. 6).
    TcProduct T;
    T.x = x; T.y = y; T.nr = nr; T.conj = herm; T.amap = a->tamap.as<int>() + (herm ? a->B : 0);
    T.items = a->B;
    T.x_ts = T.y_ts = (long long)nr * a->b; T.x_rs = T.y_rs = a->b;
    T.err = a->err; T.live = a->live;
    a->timed(PK_BINTC, [&] { launch_tc_product(a->tcZ, T, a->num_sms, a->st); });
    check_launch(a);
    return;
  }
  BinProduct P;
  P.Z = is64<R>() ? a->Z128.p : a->Z64.p;
  P.pairs = a->pairs.as<int2>();
  P.x = x; P.y = y; P.Bp = a->Bp; P.b = a->b; P.ldb = a->ldb; P.nr = nr; P.herm = herm; P.err = a->err;
  P.live = a->live;
  P.TR = a->tune_bin_tr[is64<R>()];
  P.NS = a->tune_bin_ns[is64<R>()];
  P.occ = a->tune_bin_occ[is64<R>()];
  a->timed(is64<R>() ? PK_BIN128 : PK_BIN64, [&] { launch_bin_product<R>(P, a->num_sms, a->st); });
  check_launch(a);
}

// Margin part of P^{-1} (Eq. 38): X_C^H X_C on the margin entries.
template <typename R>
void precond_margin(moma_array *a, int nr, const void *x, void *y) {
  if (a->nm <= 0) return;
  a->timed(PK_PREC, [&] {
    launch_precond_apply<R>(a->mX.p, a->mx_stride, 1, a->nm, nr, x, y, a->err, a->live, a->ldv, a->N, a->st);
  });
  check_launch(a);
}
// Margin terms of Z or Z^H added to y (whose lattice part holds Z_A x or
// Z_A^H x); margin arithmetic follows the lattice vectors' storage.
template <typename R>
void margin_terms(moma_array *a, int nr, const void *x, void *y, int herm) {
  if (a->nm <= 0) return;
  a->timed(PK_MISC, [&] {
    if (std::is_same<R, float>::value)
      launch_margin_apply<float>(a->mZB64.p, a->mZC64.p, a->nm, a->N, a->ldv, nr, herm, x, y, a->st);
    else
      launch_margin_apply<double>(a->mZB128.p, a->mZC128.p, a->nm, a->N, a->ldv, nr, herm, x, y, a->st);
  });
  check_launch(a);
}

template <typename R>
void precond(moma_array *a, int nr, const void *x, void *y) {
  if (!is64<R>() && a->tc_ready && nr >= a->tc_min_nr) {
    // Lattice vectors [nr][nel][b]: item e, RHS j at (j*nel + e)*b.  t = X x
    // goes to the FFT scratch (free here), then y = X^H t.
    TcProduct T;
    T.nr = nr; T.err = a->err; T.live = a->live;
    T.x_ts = T.y_ts = a->b; T.x_rs = T.y_rs = a->ldv;
    T.x = x; T.y = a->t1.p;
    a->timed(PK_PRECTC, [&] { launch_tc_product(a->tcX, T, a->num_sms, a->st); });
    check_launch(a);
    T.x = a->t1.p; T.y = y;
    a->timed(PK_PRECTC, [&] { launch_tc_product(a->tcXH, T, a->num_sms, a->st); });
    check_launch(a);
    precond_margin<R>(a, nr, x, y);
    return;
  }
  if (std::is_same<R, float>::value && a->xblk_ready && precond_blk_supported(a->b, nr, a->ldv, 0)) {
    a->timed(PK_PREC, [&] {
      launch_precond_blk(a->Xblk.p, a->nel, a->b, nr, x, y, a->err, a->live, a->ldv, 0, a->num_sms, a->st);
    });
  } else {
    a->timed(PK_PREC, [&] {
      launch_precond_apply<R>(a->Xinv.p, a->x_stride, a->nel, a->b, nr, x, y, a->err, a->live, a->ldv, 0, a->st);
    });
  }
  check_launch(a);
  precond_margin<R>(a, nr, x, y);
}

// The shared-memory 2D lattice transforms (one launch per transform) serve
// the c64 and FP64 products on grids the register passes do not take; c64
// grids up to 64 per axis use the cluster transforms (square grids) or the
// register per-axis passes, and the double-FP32 residual path keeps the
// per-axis passes.
template <typename R> bool use_l2d(const moma_array *a) {
  if constexpr (std::is_same<R, dfl>::value) return false;
  else {
    // c64 grids whose axes both fit the register-resident line kernels run
    // as per-axis passes on those; the 2D kernels serve the rest.
    if (std::is_same<R, float>::value && a->Mx <= 64 && a->My <= 64) {
      AxisPass probe;
      probe.in_c128 = probe.out_c128 = 0;
      if (axis_reg_supported(probe, a->Mx) && axis_reg_supported(probe, a->My)) return false;
    }
    return !a->axis_fft && lattice2d_fits<R>(a->Mx, a->My, 1);
  }
}

long long l2d_sig(int mode, int nr, int is64v) { return ((long long)mode * 1000003LL + nr) * 4 + is64v; }

template <typename R>
void l2d(moma_array *a, int mode, int nr, const void *in, void *out) {
  Lattice2D p;
  p.mode = mode; p.in = in; p.out = out; p.nx = a->nx; p.ny = a->ny; p.b = a->b; p.nr = nr; p.ldv = a->ldv;
  p.live = a->live;
  const long long sig = l2d_sig(mode, nr, is64<R>());
  for (auto &kv : a->tune_l2d)
    if (kv.first == sig) { p.J = kv.second.x; p.threads = kv.second.y; }
  a->timed(is64<R>() ? PK_FFT128 : PK_FFT64, [&] { launch_lattice2d<R>(p, a->fx, a->fy, a->st); });
  check_launch(a);
}

// c64 transforms on thread-block clusters (one launch per 2D transform)
// where the grid is square and the lane splits that the per-axis passes
// would take for this RHS count are ones the cluster kernels implement.
template <typename R>
bool use_cluster(moma_array *a, int nr, int &PX, int &PY) {
  if constexpr (!std::is_same<R, float>::value) return false;
  else {
    if (a->axis_fft || a->Mx != a->My) return false;
    AxisPass probe;
    probe.in_c128 = probe.out_c128 = 0;
    if (!axis_reg_supported(probe, a->Mx)) return false;
    PX = lanes_per_line(pass_fx(a, nr, nullptr, nullptr, 0, 0), a->Mx);
    PY = lanes_per_line(pass_fy(a, nr, nullptr, nullptr, 0), a->My);
    return lattice_cluster_supported(a->Mx, a->My, a->nx, a->ny, PX, PY);
  }
}
template <typename R>
bool cluster_transform(moma_array *a, int mode, int nr, const void *in, void *out) {
  LatticeCluster p;
  if (!use_cluster<R>(a, nr, p.PX, p.PY)) return false;
  p.mode = mode; p.in = in; p.out = out; p.nx = a->nx; p.ny = a->ny; p.b = a->b; p.nr = nr; p.ldv = a->ldv;
  p.live = a->live;
  a->timed(PK_FFT64, [&] { launch_lattice_cluster(p, a->fx, a->fy, a->st); });
  check_launch(a);
  return true;
}

// lattice -> bins (Fx then Fy); in may be c128 when R is double.
template <typename R>
void lattice_to_bins(moma_array *a, int nr, const void *in, int in128) {
  if (use_l2d<R>(a)) {
    l2d<R>(a, 0, nr, in, a->bx.p);
    return;
  }
  if (!in128 && cluster_transform<R>(a, 0, nr, in, a->bx.p)) return;
  axis<R>(a, pass_fx(a, nr, in, a->t1.p, in128, st_code<R>()), a->fx);
  axis<R>(a, pass_fy(a, nr, a->t1.p, a->bx.p, st_code<R>()), a->fy);
}
template <typename R>
void bins_to_lattice(moma_array *a, int nr, const void *bins, void *out) {
  if (use_l2d<R>(a)) {
    l2d<R>(a, 1, nr, bins, out);
    return;
  }
  if (cluster_transform<R>(a, 1, nr, bins, out)) return;
  axis<R>(a, pass_iy(a, nr, bins, a->t1.p, st_code<R>()), a->fy);
  axis<R>(a, pass_ix(a, nr, a->t1.p, out, st_code<R>(), false, lat_code<R>()), a->fx);
}
// Between the Z and Z^H legs: inverse, lattice mask, forward (by -> bx).
template <typename R>
void mask_between_legs(moma_array *a, int nr) {
  if (use_l2d<R>(a)) {
    l2d<R>(a, 2, nr, a->by.p, a->bx.p);
    return;
  }
  if (cluster_transform<R>(a, 2, nr, a->by.p, a->bx.p)) return;
  axis<R>(a, pass_iy(a, nr, a->by.p, a->t1.p, is64<R>()), a->fy);
  axis<R>(a, pass_ix(a, nr, a->t1.p, a->t1.p, is64<R>(), true), a->fx);
  axis<R>(a, pass_fy(a, nr, a->t1.p, a->bx.p, is64<R>()), a->fy);
}

// y = Z x (herm = 0) or Z^H x (herm = 1), lattice in/out in precision R.
template <typename R>
void apply_z(moma_array *a, int nr, const void *x, void *y, int herm) {
  lattice_to_bins<R>(a, nr, x, lat_code<R>());
  binprod<R>(a, nr, a->bx.p, a->by.p, herm);
  bins_to_lattice<R>(a, nr, a->by.p, y);
  margin_terms<R>(a, nr, x, y, herm);
}

// y = P^{-1} Z^H M Z x, M the restriction to the lattice (mask between legs).
template <typename R>
void apply_normal(moma_array *a, int nr, const void *x, void *y) {
  if (a->nm > 0) {  // with a margin the mask pass cannot stay in the bins
    apply_z<R>(a, nr, x, a->lat_u.p, 0);
    apply_z<R>(a, nr, a->lat_u.p, a->lat_tmp.p, 1);
    precond<R>(a, nr, a->lat_tmp.p, y);
    return;
  }
  lattice_to_bins<R>(a, nr, x, is64<R>());
  binprod<R>(a, nr, a->bx.p, a->by.p, 0);
  mask_between_legs<R>(a, nr);
  binprod<R>(a, nr, a->bx.p, a->by.p, 1);
  bins_to_lattice<R>(a, nr, a->by.p, a->lat_tmp.p);
  precond<R>(a, nr, a->lat_tmp.p, y);
}

// y = Z^H M Z x (the normal matrix, no preconditioner).
template <typename R>
void apply_zhz(moma_array *a, int nr, const void *x, void *y) {
  if (a->nm > 0) {
    apply_z<R>(a, nr, x, a->lat_u.p, 0);
    apply_z<R>(a, nr, a->lat_u.p, y, 1);
    return;
  }
  lattice_to_bins<R>(a, nr, x, is64<R>());
  binprod<R>(a, nr, a->bx.p, a->by.p, 0);
  mask_between_legs<R>(a, nr);
  binprod<R>(a, nr, a->bx.p, a->by.p, 1);
  bins_to_lattice<R>(a, nr, a->by.p, y);
}

// y = P^{-1} Z^H x.
template <typename R>
void apply_zh_p(moma_array *a, int nr, const void *x, void *y) {
  apply_z<R>(a, nr, x, a->lat_tmp.p, 1);
  precond<R>(a, nr, a->lat_tmp.p, y);
}

void sync_and_check(moma_array *a) {
  CK(cudaMemcpyAsync(a->h_err, a->err, sizeof(unsigned), cudaMemcpyDeviceToHost, a->st));
  CK(cudaStreamSynchronize(a->st));
  const unsigned e = *a->h_err;
  if (e) {
    CK(cudaMemsetAsync(a->err, 0, sizeof(unsigned), a->st));
    CK(cudaStreamSynchronize(a->st));
    if (e & DEVERR_TIMEOUT) throw MomaError(MOMA_ERR_TIMEOUT, "a bounded device wait gave up");
    if (e & DEVERR_NOT_PD) throw MomaError(MOMA_ERR_NOT_PD, "a preconditioner block is not positive definite");
    if (e & DEVERR_NONFINITE) throw MomaError(MOMA_ERR_NONFINITE, "non-finite value in input or result");
  }
}

void check_finite(moma_array *a, const void *p, size_t n_real, int is_double) {
  if (n_real == 0) return;
  size_t g = (n_real + 255) / 256;
  if (g > 2048) g = 2048;
  nonfinite_kernel<<<(int)g, 256, 0, a->st>>>(p, n_real, is_double, a->err);
  check_launch(a);
}

void drop_graphs(moma_array *a) {
  for (auto g : a->gexec)
    if (g) cudaGraphExecDestroy(g);
  a->gexec.clear();
  a->g_nr = -1;
  for (auto g : a->cg_gexec)
    if (g) cudaGraphExecDestroy(g);
  a->cg_gexec.clear();
  a->cg_g_nr = -1;
  for (auto *m : {&a->gmres_graphs, &a->pcg_graphs}) {
    for (auto &kv : *m)
      for (auto g : kv.second.g)
        if (g) cudaGraphExecDestroy(g);
    m->clear();
  }
}

void ensure_ws(moma_array *a, int nr) {
  if (nr <= a->ws_nr) return;
  drop_graphs(a);
  a->tuned_nr = -1;
  const size_t c = sizeof(double2);
  const size_t lat = (size_t)nr * a->ldv;
  const size_t tsz = (size_t)nr * a->ny * a->Mx * a->b;
  const size_t bsz = (size_t)a->B * nr * a->b;
  a->lat_in.ensure(lat * c, a->dev_bytes);
  a->lat_tmp.ensure(lat * c, a->dev_bytes);
  if (a->nm > 0) a->lat_u.ensure(lat * c, a->dev_bytes);
  a->t1.ensure(tsz * c, a->dev_bytes);
  a->bx.ensure(bsz * c, a->dev_bytes);
  a->by.ensure(bsz * c, a->dev_bytes);
  const size_t esz = a->prec == MOMA_PREC_FP64 ? sizeof(double2) : sizeof(float2);
  a->Vk.ensure((size_t)std::max(a->m + 1, 5) * lat * esz, a->dev_bytes);
  a->Iw.ensure(lat * c, a->dev_bytes);
  a->Vw.ensure(lat * c, a->dev_bytes);
  a->rw.ensure(lat * c, a->dev_bytes);
  a->yw.ensure(lat * c, a->dev_bytes);
  // Krylov control arrays
  const int m = a->m, nch = krylov_chunks((int)a->ldv);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = (off + bytes + 255) & ~size_t(255); return o; };
  const size_t o_active = take(nr * sizeof(int)), o_kq = take(nr * sizeof(int)), o_nact = take(sizeof(int));
  const size_t o_beta = take(nr * sizeof(double)), o_tol = take(nr * sizeof(double)), o_res = take(nr * sizeof(double));
  const size_t o_inv = take(nr * sizeof(double)), o_cnt = take(nr * sizeof(unsigned) * 2);
  const size_t o_part = take((size_t)nr * nch * (m + 1) * c), o_hacc = take((size_t)nr * (m + 1) * c);
  const size_t o_hcur = take((size_t)nr * (m + 1) * c), o_R = take((size_t)nr * m * (m + 1) * c);
  const size_t o_cs = take((size_t)nr * m * sizeof(double)), o_sn = take((size_t)nr * m * c);
  const size_t o_g = take((size_t)nr * (m + 1) * c), o_y = take((size_t)nr * m * c);
  const size_t o_rn = take(nr * sizeof(double)), o_vn = take(nr * sizeof(double));
  const size_t o_rp = take((size_t)nr * nch * sizeof(double)), o_mask = take(nr * sizeof(int));
  const size_t o_cg_act = take(nr * sizeof(int)), o_cg_nact = take(sizeof(int)), o_cg_it = take(nr * sizeof(int));
  const size_t o_cg_s = take((size_t)5 * nr * sizeof(double)), o_cg_cnt = take(nr * sizeof(unsigned));
  const size_t o_cg_part = take((size_t)nr * nch * sizeof(double));
  const size_t o_part2 = take((size_t)nr * nch * (m + 1) * c), o_part3 = take((size_t)nr * nch * c);
  const size_t o_gbar = take(sizeof(unsigned));
  a->kbuf.ensure(off, a->dev_bytes);
  unsigned char *base = a->kbuf.as<unsigned char>();
  // Ordered on the array's stream: a plain cudaMemset would run on the legacy
  // default stream, which non-blocking streams (batch workers, servers) do
  // not wait for, and could land after the solve has started writing here.
  CK(cudaMemsetAsync(base, 0, off, a->st));
  KrylovCtl &k = a->ctl;
  k.m = m;
  k.active = reinterpret_cast<int *>(base + o_active);
  k.kq = reinterpret_cast<int *>(base + o_kq);
  k.nact = reinterpret_cast<int *>(base + o_nact);
  k.beta = reinterpret_cast<double *>(base + o_beta);
  k.tol = reinterpret_cast<double *>(base + o_tol);
  k.res = reinterpret_cast<double *>(base + o_res);
  k.inv_norm = reinterpret_cast<double *>(base + o_inv);
  k.counters = reinterpret_cast<unsigned *>(base + o_cnt);
  k.partial = reinterpret_cast<double2 *>(base + o_part);
  k.hacc = reinterpret_cast<double2 *>(base + o_hacc);
  k.hcur = reinterpret_cast<double2 *>(base + o_hcur);
  k.Rm = reinterpret_cast<double2 *>(base + o_R);
  k.cs = reinterpret_cast<double *>(base + o_cs);
  k.sn = reinterpret_cast<double2 *>(base + o_sn);
  k.g = reinterpret_cast<double2 *>(base + o_g);
  k.y = reinterpret_cast<double2 *>(base + o_y);
  k.partial2 = reinterpret_cast<double2 *>(base + o_part2);
  k.partial3 = reinterpret_cast<double2 *>(base + o_part3);
  k.gbar = reinterpret_cast<unsigned *>(base + o_gbar);
  k.err = a->err;
  a->rnorm = reinterpret_cast<double *>(base + o_rn);
  a->vnorm = reinterpret_cast<double *>(base + o_vn);
  a->rpart = reinterpret_cast<double *>(base + o_rp);
  a->rcount = k.counters + nr;
  a->mask = reinterpret_cast<int *>(base + o_mask);
  CgCtl &g = a->cg;
  g.active = reinterpret_cast<int *>(base + o_cg_act);
  g.nact = reinterpret_cast<int *>(base + o_cg_nact);
  g.iters = reinterpret_cast<int *>(base + o_cg_it);
  double *cs5 = reinterpret_cast<double *>(base + o_cg_s);
  g.rz = cs5; g.rr = cs5 + nr; g.rr0 = cs5 + 2 * nr; g.alpha = cs5 + 3 * nr; g.beta = cs5 + 4 * nr;
  g.counters = reinterpret_cast<unsigned *>(base + o_cg_cnt);
  g.partial = reinterpret_cast<double *>(base + o_cg_part);
  g.err = a->err;
  if (a->h_norms) cudaFreeHost(a->h_norms);
  CK(cudaMallocHost(&a->h_norms, (size_t)3 * nr * sizeof(double) + 64));
  a->ws_nr = nr;
}

// Stage a caller buffer on the device: returns a device pointer (the
// caller's own if it is device memory, else `tmp` after a copy).
// Split full bins and inverse factors for the tensor-core products, once
// per set_blocks, when a call brings enough right-hand sides to use them.
void ensure_tc(moma_array *a, int nr) {
  if (a->tc_ready || a->no_tensor || a->prec != MOMA_PREC_MIXED || nr < a->tc_min_nr || !tc_supported(a->b)) return;
  drop_graphs(a);
  const int b = a->b;
  // Bins: the c64 pair store and its transpose, split into TF32 pairs by
  // the kernel as it reads them.  Factors: X_e and X_e^H whole, pre-split.
  const size_t zt = (size_t)a->Bp * b * a->ldb * sizeof(float2), xb = tc_bytes(a->nel, b);
  a->tcA.ensure(zt, a->dev_bytes);
  a->tcP.ensure(2 * xb, a->dev_bytes);
  unsigned char *px = a->tcP.as<unsigned char>();
  a->tcZ = TcMats{};
  a->tcZ.b = b; a->tcZ.T = a->Bp;
  a->tcX = TcMats{};
  a->tcX.b = b; a->tcX.T = a->nel;
  a->tcX.hi = reinterpret_cast<float *>(px); a->tcX.lo = reinterpret_cast<float *>(px + xb / 2);
  a->tcXH = a->tcX;
  a->tcXH.hi = reinterpret_cast<float *>(px + xb); a->tcXH.lo = reinterpret_cast<float *>(px + xb + xb / 2);
  try {
    a->timed(PK_BLOCKFFT, [&] { tc_transpose_pairs(a->Z64.p, a->tcA.p, a->Bp, b, a->ldb, a->st); });
    check_launch(a);
    tc_raw(a->tcZ, a->Z64.p, a->tcA.p, a->ldb);
    a->timed(PK_TRINV, [&] { tc_split_factor(a->tcX, a->tcXH, a->Xinv.p, a->x_stride, a->st); });
    check_launch(a);
  } catch (const std::runtime_error &e) {
    throw MomaError(MOMA_ERR_CUDA, e.what());
  }
  a->tc_ready = true;
}

const void *stage_in(moma_array *a, const void *src, size_t bytes, DevBuf &tmp) {
  if (is_device_ptr(src)) return src;
  tmp.ensure(bytes, a->dev_bytes);
  CK(cudaMemcpyAsync(tmp.p, src, bytes, cudaMemcpyHostToDevice, a->st));
  return tmp.p;
}

void copy_out(moma_array *a, void *dst, const void *src, size_t bytes) {
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, a->st));
}

// Gram products G_D = Z_D^H Z_D of offsets [d0, d0 + nd) into S.
template <typename R>
void gram_chunk(moma_array *a, const void *blk, int blk128, int d0, int nd) {
  const size_t bb = (size_t)a->b * a->b, esz = blk128 ? sizeof(double2) : sizeof(float2);
  const void *src = static_cast<const unsigned char *>(blk) + (size_t)d0 * bb * esz;
  a->timed(PK_GRAM, [&] { launch_gram<R>(src, blk128, nd, a->b, a->S.as<double2>() + (size_t)d0 * bb, a->st); });
  check_launch(a);
}

// Box sums, Cholesky, inverse factors (after every offset's Gram product is
// in S, or in gramY for the tensor-core Gram products).
template <typename R>
void finish_preconditioner(moma_array *a) {
  // The sliding-window sums go to S where the Gram products are not in it
  // and it is large enough, else to their own buffer.
  const size_t wents = box_window_entries(a->nx, a->ny, a->b);
  double2 *W;
  if (a->tgram && wents * sizeof(double2) <= a->S.cap) {
    W = a->S.as<double2>();
  } else {
    a->Wb.ensure(wents * sizeof(double2), a->dev_bytes);
    W = a->Wb.as<double2>();
  }
  a->timed(PK_BOX, [&] {
    launch_box_sums(a->tgram ? nullptr : a->S.as<double2>(), a->tgram ? a->gramY.as<float2>() : nullptr, a->nx,
                    a->ny, a->b, W, a->df, a->st);
  });
  check_launch(a);
  a->pbox = box_sums_of(W, a->nx, a->ny, a->b);
  a->pbox_df = a->df;
  const size_t npk = (size_t)a->b * (a->b + 1) / 2;
  a->Lpk.ensure((size_t)a->nel * npk * sizeof(double2), a->dev_bytes);
  a->timed(PK_CHOL, [&] { launch_box_cholesky(a->pbox, a->nel, a->b, a->Lpk.as<double2>(), a->err, a->df, a->st); });
  check_launch(a);
  using C = typename Cplx<R>::T;
  size_t xs = npk;
  while ((xs * sizeof(C)) % 16) ++xs;
  a->x_stride = xs;
  a->Xinv.ensure((size_t)a->nel * xs * sizeof(C), a->dev_bytes);
  // c64: also P_e^{-1} = X_e^H X_e in the blocked layout of the streaming apply.
  a->xblk_ready = false;
  const bool blk = std::is_same<R, float>::value && !a->no_blk_precond && precond_blk_supported(a->b, 1, 2, 0);
  if (blk) a->Xblk.ensure((size_t)a->nel * xblk_entries(a->b) * sizeof(float2), a->dev_bytes);
  bool q_done = false;
  a->timed(PK_TRINV, [&] {
    q_done = launch_tri_inverse<R>(a->Lpk.as<double2>(), a->nel, a->b, a->Xinv.p, xs, a->st, blk ? a->Xblk.p : nullptr);
  });
  check_launch(a);
  if (blk) {
    if (!q_done) {
      a->timed(PK_TRINV, [&] { launch_pinv_pack(a->Xinv.p, a->x_stride, a->nel, a->b, a->Xblk.p, a->st); });
      check_launch(a);
    }
    a->xblk_ready = true;
  }
}

void set_blocks_impl(moma_array *a, const void *blocks, int dtype) {
  if (dtype != MOMA_C128 && dtype != MOMA_C64) throw MomaError(MOMA_ERR_ARG, "blocks dtype must be MOMA_C128 or MOMA_C64");
  if (!blocks) throw MomaError(MOMA_ERR_ARG, "blocks is NULL");
  const int ndy = 2 * a->ny - 1, ndx = 2 * a->nx - 1, nD = ndx * ndy, bb = a->b * a->b;
  const size_t esz = dtype == MOMA_C128 ? sizeof(double2) : sizeof(float2);
  const size_t row_bytes = (size_t)ndx * bb * esz;  // one dy row of offsets
  a->have_blocks = false;
  a->tc_ready = false;

  // Transformed first column of the circulant embedding (Eqs. 3, 11).
  // Reciprocity (Z_{-D} = Z_D^T) makes Zhat_{-k} = Zhat_k^T, so only the
  // b(b+1)/2 entries i <= j are transformed; the y pass scatters each bin's
  // values into the stored block of its pair (transposed for the partner).
  // FP64 in the plain path; double-FP32 pairs (c128-class bins stored as
  // dfl2) in the mixed path, where B300's FP64 rate would bound it, unless
  // the array asked for FP64 there (MOMA_FLAG_FP64_RESIDUAL).
  const bool df = a->df;
  const int nt = a->b * (a->b + 1) / 2;
  a->T.ensure((size_t)ndy * a->Mx * nt * sizeof(double2), a->dev_bytes);
  a->S.ensure((size_t)nD * bb * sizeof(double2), a->dev_bytes);

  // Blocks in host memory: only the rows dy >= 0 cross the bus (the rows
  // dy < 0 are their transposes by reciprocity and are completed on the
  // device), in chunks of rows on a copy stream; each chunk's finiteness
  // check, completion, x-pass of the block transform and Gram products start
  // as soon as it has landed, overlapping the next copy.  Blocks already on
  // the device are read whole.
  const bool host = !is_device_ptr(blocks);
  const unsigned char *blk = static_cast<const unsigned char *>(blocks);
  const int yh = a->ny - 1;  // row index of dy = 0
  int nchunk = 1, r0 = 0;
  if (host) {
    a->blk.ensure((size_t)ndy * row_bytes, a->dev_bytes);
    blk = a->blk.as<unsigned char>();
    r0 = yh;
    nchunk = std::min(ndy - yh, 8);
    if (!a->cs) {
      CK(cudaStreamCreateWithFlags(&a->cs, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&a->ev_cs0, cudaEventDisableTiming));
      for (auto &e : a->ev_chunk) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    CK(cudaEventRecord(a->ev_cs0, a->st));  // earlier work on the staging buffer is done
    CK(cudaStreamWaitEvent(a->cs, a->ev_cs0, 0));
  }
  AxisPass px;
  px.n2 = 1; px.ninner = nt;
  px.in_s1 = (long long)ndx * bb; px.in_sm = bb; px.nin = ndx; px.in_mode = 1;
  px.inner_in_map = a->tri_in.as<int>();
  px.out_s1 = (long long)a->Mx * nt; px.out_sm = nt; px.nout = a->Mx;
  px.in_c128 = dtype == MOMA_C128; px.out_c128 = df ? 2 : 1;
  auto rows_work = [&](int y0, int y1) {  // transform x-pass + Gram of rows [y0, y1)
    if (y1 <= y0) return;
    px.in = blk + (size_t)y0 * row_bytes; px.n1 = y1 - y0;
    px.out = a->T.as<double2>() + (size_t)y0 * a->Mx * nt;
    a->timed(PK_BLOCKFFT, [&] {
      if (df) launch_axis_pass<dfl>(px, a->fx, a->st);
      else launch_axis_pass<double>(px, a->fx, a->st);
    });
    check_launch(a);
    // Gram products of these offsets (Eq. 37 precomputation).
    const int d0 = y0 * ndx, nd = (y1 - y0) * ndx;
    if (a->tgram) {
      // Tensor cores: item D with A = Z_D (conjugated) and RHS rows Z_D[j]
      // gives y_D[j][i] = sum_k conj(Z_D[i][k]) Z_D[j][k], which by
      // reciprocity is G_{-D}[i][j]; the box-sum pass reads it back
      // reflected and conjugated.
      // The blocks are read unsplit (split into TF32 pairs in shared memory,
      // where their finiteness is checked too).
      TcMats mA;
      mA.b = a->b; mA.T = nd;
      const float2 *zb = reinterpret_cast<const float2 *>(blk) + (size_t)d0 * bb;
      TcProduct P;
      P.x = zb; P.y = a->gramY.as<float2>() + (size_t)d0 * bb;
      P.x_ts = P.y_ts = bb; P.x_rs = P.y_rs = a->b; P.nr = a->b; P.conj = 1; P.err = a->err;
      P.check_finite = 1;
      a->timed(PK_GRAM, [&] {
        try {
          tc_raw(mA, zb, nullptr, a->b);
          launch_tc_product(mA, P, a->num_sms, a->st);
        } catch (const std::runtime_error &e) {
          throw MomaError(MOMA_ERR_CUDA, e.what());
        }
      });
      check_launch(a);
    } else if (a->prec == MOMA_PREC_FP64) {
      gram_chunk<double>(a, blk, dtype == MOMA_C128, d0, nd);
    } else {
      gram_chunk<float>(a, blk, dtype == MOMA_C128, d0, nd);
    }
  };
  const int nrows = ndy - r0;
  // Gram products on the tensor cores (3xTF32) for c64 blocks in the mixed
  // path when the block size suits the MMA kernel.
  // The kernel reads the blocks with TMA, which needs a 16-byte aligned base.
  a->tgram = a->prec == MOMA_PREC_MIXED && dtype == MOMA_C64 && !a->no_tensor && tc_supported(a->b) &&
             reinterpret_cast<uintptr_t>(blk) % 16 == 0;
  if (a->tgram) a->gramY.ensure((size_t)nD * bb * sizeof(float2), a->dev_bytes);
  for (int c = 0; c < nchunk; ++c) {
    const int y0 = r0 + (int)((long long)nrows * c / nchunk), y1 = r0 + (int)((long long)nrows * (c + 1) / nchunk);
    if (y1 <= y0) continue;
    unsigned char *dst = const_cast<unsigned char *>(blk) + (size_t)y0 * row_bytes;
    if (host) {
      CK(cudaMemcpyAsync(dst, static_cast<const unsigned char *>(blocks) + (size_t)y0 * row_bytes,
                         (size_t)(y1 - y0) * row_bytes, cudaMemcpyHostToDevice, a->cs));
      CK(cudaEventRecord(a->ev_chunk[c], a->cs));
      CK(cudaStreamWaitEvent(a->st, a->ev_chunk[c], 0));
    }
    // The tensor-core Gram split reads every block of these rows and checks
    // them itself; otherwise a separate pass does.
    if (!a->tgram) check_finite(a, dst, (size_t)(y1 - y0) * ndx * bb * 2, dtype == MOMA_C128);
    rows_work(y0, y1);
    if (host) {
      // Mirror rows of [y0, y1) below dy = 0: [2Ny-1-y1, 2Ny-1-y0) within [0, yh).
      const int m0 = std::max(0, ndy - y1), m1 = std::min(yh, ndy - y0);
      if (m1 > m0) {
        dim3 grid((a->b + 31) / 32, (a->b + 31) / 32, (m1 - m0) * ndx), block(32, 8);
        if (dtype == MOMA_C128)
          reciprocal_fill_kernel<double2><<<grid, block, 0, a->st>>>(a->blk.as<double2>(), ndy, ndx, a->b, m0);
        else
          reciprocal_fill_kernel<float2><<<grid, block, 0, a->st>>>(a->blk.as<float2>(), ndy, ndx, a->b, m0);
        check_launch(a);
        rows_work(m0, m1);
      }
    }
  }
  // Non-finite input: report before anything is marked usable.
  sync_and_check(a);
  AxisPass py;
  py.in = a->T.p; py.out = a->Z128.p; py.out2 = a->prec == MOMA_PREC_MIXED ? a->Z64.p : nullptr;
  py.n1 = a->Mx; py.n2 = 1; py.ninner = nt;
  py.in_s1 = nt; py.in_sm = (long long)a->Mx * nt; py.nin = 2 * a->ny - 1; py.in_mode = 1;
  py.out_mode = 2; py.bin_slot = a->bin_slot.as<int2>(); py.tri = a->tri.as<int2>(); py.slot_mul = a->Mx;
  py.out_sm = (long long)a->b * a->ldb; py.remap_ld = a->ldb; py.nout = a->My;
  py.in_c128 = df ? 2 : 1; py.out_c128 = df ? 2 : 1;
  a->timed(PK_BLOCKFFT, [&] {
    if (df) launch_axis_pass<dfl>(py, a->fy, a->st);
    else launch_axis_pass<double>(py, a->fy, a->st);
  });
  check_launch(a);

  // Preconditioner (Eq. 37) and its factorisation (Sec. III-A).
  if (a->prec == MOMA_PREC_FP64) finish_preconditioner<double>(a);
  else finish_preconditioner<float>(a);
  sync_and_check(a);
  a->have_blocks = true;
}

// ----------------------------------------------------------- autotuner --
// Launch shapes are picked by timing: for the bin product the rows per
// staged tile and the pipeline depth, for every lattice-FFT pass of the
// solve the number of threads cooperating on a line.  Candidates run on the
// solve's own workspace (contents irrelevant, only the timing is used), a
// warm-up launch and two timed launches each, CUDA events on the array's
// stream; the fastest wins.  Done once per (array, RHS count) before any
// graph capture.
template <typename F>
float time_launch(moma_array *a, F &&f) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  f();
  CK(cudaEventRecord(e0, a->st));
  f();
  f();
  CK(cudaEventRecord(e1, a->st));
  CK(cudaEventSynchronize(e1));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  return ms;
}

template <typename R>
void autotune_precision(moma_array *a, int nr, int in128) {
  char buf[256];
  // Bin product: tile rows x stages.
  {
    float best = 1e30f;
    int btr = 0, bns = 0, bocc = 1;
    // The c64 row/column-warp kernel (b = 64 .. 256, multiple of 32) has a
    // fixed 32-row tile: only its pipeline depth and CTAs per SM are tuned.
    const bool rc = std::is_same<R, float>::value && bin_rc_supported(a->b) && a->ldb == a->b;
    for (int occ : {1, 2, 3}) {
      // The multi-CTA variants' domain: at most two RHS, b <= 128; three CTAs for c64 only.
      if (occ > 1 && (nr > 2 || a->b > 128)) continue;
      if (occ == 3 && (is64<R>() || rc)) continue;
      for (int tr : {8, 16, 24, 32}) {
        if (tr > ((a->b + 3) & ~3) && tr != 16) continue;
        if (occ == 1 && tr < 16) continue;
        if (rc && tr != 32) continue;
        for (int ns : {2, 3, 4, 6}) {
          if (!rc && ns == 6) continue;
          BinProduct P;
          P.Z = is64<R>() ? a->Z128.p : a->Z64.p;
          P.pairs = a->pairs.as<int2>();
          P.x = a->bx.p; P.y = a->by.p; P.Bp = a->Bp; P.b = a->b; P.ldb = a->ldb; P.nr = nr; P.err = a->err;
          P.TR = tr; P.NS = ns; P.occ = occ;
          const float ms = time_launch(a, [&] { launch_bin_product<R>(P, a->num_sms, a->st); });
          if (ms < best) { best = ms; btr = tr; bns = ns; bocc = occ; }
        }
      }
    }
    a->tune_bin_tr[is64<R>()] = btr;
    a->tune_bin_ns[is64<R>()] = bns;
    a->tune_bin_occ[is64<R>()] = bocc;
    snprintf(buf, sizeof(buf), "bin_product<%s> nr=%d: TR=%d NS=%d CTAs/SM=%d (%.1f us)\n",
             st_code<R>() == 2 ? "dfl" : (is64<R>() ? "c128" : "c64"), nr, btr, bns, bocc, 1000.0f * best / 2);
    a->tune_log += buf;
  }
  // 2D lattice transforms: basis indices per CTA x threads per CTA.
  if (use_l2d<R>(a)) {
    static const char *names[3] = {"F2", "I2", "I2MF2"};
    for (int mode = 0; mode < 3; ++mode) {
      float best = 1e30f;
      int bj = 0, bt = 0;
      for (int J : {1, 2, 4}) {
        if (!lattice2d_fits<R>(a->Mx, a->My, J)) continue;
        for (int th : {128, 256, 512}) {
          Lattice2D p;
          p.mode = mode; p.nx = a->nx; p.ny = a->ny; p.b = a->b; p.nr = nr; p.ldv = a->ldv; p.J = J; p.threads = th;
          p.in = mode == 0 ? a->lat_in.p : a->by.p;
          p.out = mode == 1 ? a->lat_tmp.p : a->bx.p;
          const float ms = time_launch(a, [&] { launch_lattice2d<R>(p, a->fx, a->fy, a->st); });
          if (ms < best) { best = ms; bj = J; bt = th; }
        }
      }
      a->tune_l2d.push_back({l2d_sig(mode, nr, is64<R>()), make_int2(bj, bt)});
      snprintf(buf, sizeof(buf), "%s<%s> nr=%d: J=%d threads=%d (%.1f us)\n", names[mode], is64<R>() ? "c128" : "c64",
               nr, bj, bt, 1000.0f * best / 2);
      a->tune_log += buf;
    }
    return;
  }
  // Lattice FFT passes of the products and the normal operator.
  const int c = st_code<R>();
  struct Cand { AxisPass p; const FftTables *t; const char *name; };
  const Cand cands[] = {
      {pass_fx(a, nr, a->lat_in.p, a->t1.p, in128, c), &a->fx, "Fx"},
      {pass_fy(a, nr, a->t1.p, a->bx.p, c), &a->fy, "Fy"},
      {pass_iy(a, nr, a->by.p, a->t1.p, c), &a->fy, "Iy"},
      {pass_ix(a, nr, a->t1.p, a->t1.p, c, true), &a->fx, "IxMaskFx"},
      {pass_ix(a, nr, a->t1.p, a->lat_tmp.p, c, false, lat_code<R>()), &a->fx, "Ix"},
  };
  for (const Cand &cd : cands) {
    // Register passes take a fixed lanes-per-line rule (the split changes
    // the rounding, and tuned shapes never change results).
    if (std::is_same<R, float>::value && axis_reg_supported(cd.p, cd.t->plan.M)) continue;
    float best = 1e30f;
    int bg = 0;
    for (int G : {1, 2, 4, 8, 16, 32}) {
      if (G > cd.t->plan.M) continue;
      AxisPass p = cd.p;
      p.G = G;
      const float ms = time_launch(a, [&] { launch_axis_pass<R>(p, *cd.t, a->st); });
      if (ms < best) { best = ms; bg = G; }
    }
    a->tune_axis.push_back({axis_sig(cd.p, cd.t->plan.M, c), bg});
    snprintf(buf, sizeof(buf), "%s<%s> nr=%d: G=%d (%.1f us)\n", cd.name, c == 2 ? "dfl" : (c ? "c128" : "c64"), nr, bg,
             1000.0f * best / 2);
    a->tune_log += buf;
  }
}

// Process-wide cache of tuned launch shapes.  The shapes depend only on the
// device, the lattice and circulant sizes, b, the precision and the RHS
// count (never on the blocks' values, and they never change a result), so
// an array of a shape tuned before in this process takes them without
// timing trials -- the serving loop's arrays, which skip the trials, and
// ragged batches of repeated shapes.
struct TuneKey {
  int dev, nx, ny, b, Mx, My, nr, prec, df, axis_fft;
  long long ldv;
  bool operator<(const TuneKey &o) const {
    return std::tie(dev, nx, ny, b, Mx, My, nr, prec, df, axis_fft, ldv) <
           std::tie(o.dev, o.nx, o.ny, o.b, o.Mx, o.My, o.nr, o.prec, o.df, o.axis_fft, o.ldv);
  }
};
struct TuneEntry {
  moma_array::TuneBin bin;
  std::vector<std::pair<long long, int>> axis;
  std::vector<std::pair<long long, int2>> l2d;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneEntry> g_tune_cache;

void autotune(moma_array *a, int nr) {
  if (a->tuned_nr == nr) return;
  auto it = a->tune_by_nr.find(nr);
  if (it != a->tune_by_nr.end()) {  // tuned before for this RHS count
    for (int k = 0; k < 2; ++k) {
      a->tune_bin_tr[k] = it->second.tr[k];
      a->tune_bin_ns[k] = it->second.ns[k];
      a->tune_bin_occ[k] = it->second.occ[k];
    }
    a->tuned_nr = nr;
    return;
  }
  const TuneKey key{a->dev, a->nx, a->ny, a->b, a->Mx, a->My, nr, a->prec, a->df ? 1 : 0, a->axis_fft ? 1 : 0,
                    a->ldv};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto f = g_tune_cache.find(key);
    if (f != g_tune_cache.end()) {  // tuned before in this process for this shape
      for (int k = 0; k < 2; ++k) {
        a->tune_bin_tr[k] = f->second.bin.tr[k];
        a->tune_bin_ns[k] = f->second.bin.ns[k];
        a->tune_bin_occ[k] = f->second.bin.occ[k];
      }
      a->tune_axis.insert(a->tune_axis.end(), f->second.axis.begin(), f->second.axis.end());
      a->tune_l2d.insert(a->tune_l2d.end(), f->second.l2d.begin(), f->second.l2d.end());
      a->tune_by_nr[nr] = f->second.bin;
      a->tuned_nr = nr;
      a->tune_log += "nr=" + std::to_string(nr) + ": shapes from the process-wide cache\n";
      return;
    }
  }
  if (a->no_autotune || std::getenv("MOMA_NO_AUTOTUNE")) return;
  // FFT pass shapes accumulate in tune_axis (their signatures include the
  // RHS count); the bin-product shapes are kept per RHS count.
  a->tune_bin_tr[0] = a->tune_bin_tr[1] = a->tune_bin_ns[0] = a->tune_bin_ns[1] = 0;
  a->tune_bin_occ[0] = a->tune_bin_occ[1] = 1;
  const size_t n_axis0 = a->tune_axis.size(), n_l2d0 = a->tune_l2d.size();
  if (a->prec == MOMA_PREC_MIXED) autotune_precision<float>(a, nr, 0);
  // The FP64-class residual runs in double-FP32 pairs in the default mixed
  // path, in FP64 otherwise.
  if (a->df) autotune_precision<dfl>(a, nr, 1);
  else autotune_precision<double>(a, nr, 1);
  moma_array::TuneBin t;
  for (int k = 0; k < 2; ++k) {
    t.tr[k] = a->tune_bin_tr[k];
    t.ns[k] = a->tune_bin_ns[k];
    t.occ[k] = a->tune_bin_occ[k];
  }
  a->tune_by_nr[nr] = t;
  a->tuned_nr = nr;
  TuneEntry e;
  e.bin = t;
  e.axis.assign(a->tune_axis.begin() + n_axis0, a->tune_axis.end());
  e.l2d.assign(a->tune_l2d.begin() + n_l2d0, a->tune_l2d.end());
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache.emplace(key, std::move(e));
}

template <typename R>
void gmres_cycle(moma_array *a, int nr, const std::vector<int> &act, int *inner_iters, double *first_red) {
  using C = typename Cplx<R>::T;
  const size_t vstride = (size_t)nr * a->ldv;
  C *V = a->Vk.as<C>();
  KrylovCtl c = a->ctl;
  // Inner right-hand side P^{-1} Z^H r~ into slot 0; its norm starts the cycle.
  apply_zh_p<R>(a, nr, a->lat_in.p, V);
  int nact = 0;
  for (int q = 0; q < nr; ++q) nact += act[q] ? 1 : 0;
  a->h_nact[MOMA_MAX_RESTART + 4] = nact;  // pinned staging slot
  CK(cudaMemcpyAsync(c.active, a->mask, nr * sizeof(int), cudaMemcpyDeviceToDevice, a->st));
  CK(cudaMemsetAsync(c.kq, 0, nr * sizeof(int), a->st));
  CK(cudaMemcpyAsync(c.nact, a->h_nact + MOMA_MAX_RESTART + 4, sizeof(int), cudaMemcpyHostToDevice, a->st));
  a->timed(PK_KRYLOV, [&] { launch_cgs<R>(c, V, vstride, (int)a->ldv, nr, -1, KF_NORM | KF_INIT, a->st); });
  check_launch(a);
  a->timed(PK_KRYLOV, [&] { launch_scale<R>(c, V, vstride, (int)a->ldv, nr, a->st); });
  check_launch(a);

  const int lag = 2;
  if ((int)a->poll_ev.size() < a->m + 1) {
    while ((int)a->poll_ev.size() < a->m + 1) {
      cudaEvent_t e;
      CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      a->poll_ev.push_back(e);
    }
  }
  // One Arnoldi step: the normal operator, the three CGS2 sweeps (the last
  // one applies the Givens rotation), the scaling of the new basis vector,
  // and the copy of the active-column count for the host's lagged poll.
  // The sweeps and the scaling run as one cooperative launch when the grid
  // can be co-resident (its barrier counter restarts with every cycle).
  const bool fused = !a->no_fused_arnoldi && arnoldi_fused_fits<R>((int)a->ldv, nr, a->num_sms);
  if (fused) CK(cudaMemsetAsync(c.gbar, 0, sizeof(unsigned), a->st));
  auto enqueue_step = [&](int j) {
    a->live = c.nact;  // steps queued after convergence cost only their launches
    apply_normal<R>(a, nr, V + (size_t)j * vstride, V + (size_t)(j + 1) * vstride);
    a->live = nullptr;
    if (fused) {
      a->timed(PK_KRYLOV, [&] { launch_arnoldi_fused<R>(c, V, vstride, (int)a->ldv, nr, j, a->st); });
      check_launch(a);
      CK(cudaMemcpyAsync(a->h_nact + j, c.nact, sizeof(int), cudaMemcpyDeviceToHost, a->st));
      CK(cudaEventRecord(a->poll_ev[j], a->st));
      return;
    }
    a->timed(PK_KRYLOV, [&] { launch_cgs<R>(c, V, vstride, (int)a->ldv, nr, j, KF_DOTS, a->st); });
    check_launch(a);
    a->timed(PK_KRYLOV, [&] { launch_cgs<R>(c, V, vstride, (int)a->ldv, nr, j, KF_UPDATE | KF_DOTS | KF_ACCUM, a->st); });
    check_launch(a);
    a->timed(PK_KRYLOV, [&] { launch_cgs<R>(c, V, vstride, (int)a->ldv, nr, j, KF_UPDATE | KF_NORM, a->st); });
    check_launch(a);
    a->timed(PK_KRYLOV, [&] { launch_scale<R>(c, V + (size_t)(j + 1) * vstride, vstride, (int)a->ldv, nr, a->st); });
    check_launch(a);
    CK(cudaMemcpyAsync(a->h_nact + j, c.nact, sizeof(int), cudaMemcpyDeviceToHost, a->st));
    CK(cudaEventRecord(a->poll_ev[j], a->st));
  };
  // With graphs on, step j is captured once (per RHS count) and replayed.
  const bool graphs = a->use_graphs && !a->prof && a->st == a->gs && a->gs != nullptr;
  if (graphs && a->g_nr != nr) {
    // Park the current RHS count's graphs and take (or start) this one's.
    if (a->g_nr >= 0) {
      auto &park = a->gmres_graphs[a->g_nr];
      park.g.swap(a->gexec);
      park.step_launches = a->g_step_launches;
    }
    a->gexec.clear();
    auto it = a->gmres_graphs.find(nr);
    if (it != a->gmres_graphs.end()) {
      a->gexec.swap(it->second.g);
      a->g_step_launches = it->second.step_launches;
      a->gmres_graphs.erase(it);
    }
    if (a->gexec.size() != (size_t)a->m) {
      for (auto g : a->gexec)
        if (g) cudaGraphExecDestroy(g);
      a->gexec.assign(a->m, nullptr);
    }
    a->g_nr = nr;
  }
  int steps = 0;
  for (int j = 0; j < a->m; ++j) {
    if (graphs) {
      if (!a->gexec[j]) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(a->st, cudaStreamCaptureModeThreadLocal));
        const long long l0 = a->launches;
        try {
          enqueue_step(j);
        } catch (...) {
          cudaStreamEndCapture(a->st, &g);
          if (g) cudaGraphDestroy(g);
          throw;
        }
        a->g_step_launches = a->launches - l0;
        a->launches = l0;
        CK(cudaStreamEndCapture(a->st, &g));
        cudaGraphExec_t ge = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        CK(ie);
        a->gexec[j] = ge;
      }
      a->h_nact[j] = -1;  // sentinel, overwritten by the step's copy
      CK(cudaGraphLaunch(a->gexec[j], a->st));
      a->launches += a->g_step_launches;
    } else {
      a->h_nact[j] = -1;
      enqueue_step(j);
    }
    steps = j + 1;
    if (j >= lag) {
      // Lagged poll of the pinned copy written by step j - lag (bounded).
      volatile int *hn = a->h_nact;
      const auto t0 = std::chrono::steady_clock::now();
      while (hn[j - lag] == -1) {
        const cudaError_t q = cudaStreamQuery(a->st);
        if (q != cudaSuccess && q != cudaErrorNotReady) CK(q);  // a device fault: report it now
        if (q == cudaSuccess && hn[j - lag] == -1) throw MomaError(MOMA_ERR_CUDA, "poll copy did not arrive");
        if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60))
          throw MomaError(MOMA_ERR_TIMEOUT, "inner iteration poll timed out");
        std::this_thread::yield();
      }
      if (hn[j - lag] == 0) break;
    }
  }
  CK(cudaStreamSynchronize(a->st));
  int done_at = steps;
  for (int j = 0; j < steps; ++j)
    if (a->h_nact[j] == 0) { done_at = j + 1; break; }
  *inner_iters += done_at;
  if (first_red) {
    std::vector<double> res(nr), beta(nr);
    CK(cudaMemcpy(res.data(), c.res, nr * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(beta.data(), c.beta, nr * sizeof(double), cudaMemcpyDeviceToHost));
    double mx = 0;
    for (int q = 0; q < nr; ++q)
      if (act[q] && beta[q] > 0) mx = std::max(mx, res[q] / beta[q]);
    *first_red = mx;
  }
  a->timed(PK_KRYLOV, [&] { launch_backsolve(c, nr, a->st); });
  check_launch(a);
  a->timed(PK_KRYLOV, [&] { launch_lincomb<R>(c, V, vstride, (int)a->ldv, nr, a->Iw.as<double2>(), a->rnorm, a->st); });
  check_launch(a);
}

// Inner PCG solve of Z^H Z d = Z^H r~ with preconditioner P (Sec. II-C,
// Sec. III-A), then I += ||r|| d.  Vectors (c64 in MIXED): d, r, p, q, z in
// the first five Krylov slots.  Iterations are graph-captured per slot of a
// 16-entry ring of poll copies and replayed.
template <typename R>
void pcg_cycle(moma_array *a, int nr, const std::vector<int> &act, int max_inner, int *inner_iters,
               double *first_red) {
  using C = typename Cplx<R>::T;
  const size_t vs = (size_t)nr * a->ldv;
  C *base = a->Vk.as<C>();
  C *d = base, *r = base + vs, *p = base + 2 * vs, *q = base + 3 * vs, *z = base + 4 * vs;
  CgCtl c = a->cg;
  c.tol2 = a->ctl.inner_tol * a->ctl.inner_tol;
  int nact = 0;
  for (int k = 0; k < nr; ++k) nact += act[k] ? 1 : 0;
  a->h_nact[MOMA_MAX_RESTART + 4] = nact;
  CK(cudaMemcpyAsync(c.active, a->mask, nr * sizeof(int), cudaMemcpyDeviceToDevice, a->st));
  CK(cudaMemcpyAsync(c.nact, a->h_nact + MOMA_MAX_RESTART + 4, sizeof(int), cudaMemcpyHostToDevice, a->st));
  CK(cudaMemsetAsync(c.iters, 0, nr * sizeof(int), a->st));
  CK(cudaMemsetAsync(d, 0, vs * sizeof(C), a->st));
  // r = Z^H r~ (right-hand side of the normal equations), ||r0||, z = P^{-1} r, p = z.
  apply_z<R>(a, nr, a->lat_in.p, r, 1);
  a->timed(PK_KRYLOV, [&] { launch_cg_axpy<R>(c, d, p, r, q, (int)a->ldv, nr, 1, a->st); });
  check_launch(a);
  precond<R>(a, nr, r, z);
  a->timed(PK_KRYLOV, [&] { launch_cg_reduce<R>(c, r, z, (int)a->ldv, nr, CG_RZ0, a->st); });
  check_launch(a);
  a->timed(PK_KRYLOV, [&] { launch_cg_dir<R>(c, p, z, (int)a->ldv, nr, 1, a->st); });
  check_launch(a);

  constexpr int RING = 16;
  auto enqueue_iter = [&](int slot) {
    a->live = c.nact;
    apply_zhz<R>(a, nr, p, q);
    a->timed(PK_KRYLOV, [&] { launch_cg_reduce<R>(c, p, q, (int)a->ldv, nr, CG_PQ, a->st); });
    check_launch(a);
    a->timed(PK_KRYLOV, [&] { launch_cg_axpy<R>(c, d, p, r, q, (int)a->ldv, nr, 0, a->st); });
    check_launch(a);
    precond<R>(a, nr, r, z);
    a->live = nullptr;
    a->timed(PK_KRYLOV, [&] { launch_cg_reduce<R>(c, r, z, (int)a->ldv, nr, CG_RZ, a->st); });
    check_launch(a);
    a->timed(PK_KRYLOV, [&] { launch_cg_dir<R>(c, p, z, (int)a->ldv, nr, 0, a->st); });
    check_launch(a);
    CK(cudaMemcpyAsync(a->h_nact + slot, c.nact, sizeof(int), cudaMemcpyDeviceToHost, a->st));
  };
  const bool graphs = a->use_graphs && !a->prof && a->st == a->gs && a->gs != nullptr;
  if (graphs && a->cg_g_nr != nr) {
    if (a->cg_g_nr >= 0) {
      auto &park = a->pcg_graphs[a->cg_g_nr];
      park.g.swap(a->cg_gexec);
      park.step_launches = a->cg_step_launches;
    }
    a->cg_gexec.clear();
    auto it = a->pcg_graphs.find(nr);
    if (it != a->pcg_graphs.end()) {
      a->cg_gexec.swap(it->second.g);
      a->cg_step_launches = it->second.step_launches;
      a->pcg_graphs.erase(it);
    }
    if (a->cg_gexec.size() != (size_t)RING) {
      for (auto g : a->cg_gexec)
        if (g) cudaGraphExecDestroy(g);
      a->cg_gexec.assign(RING, nullptr);
    }
    a->cg_g_nr = nr;
  }
  const int lag = 2;
  int it = 0;
  for (; it < max_inner; ++it) {
    const int slot = it % RING;
    a->h_nact[slot] = -1;
    if (graphs) {
      if (!a->cg_gexec[slot]) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(a->st, cudaStreamCaptureModeThreadLocal));
        const long long l0 = a->launches;
        try {
          enqueue_iter(slot);
        } catch (...) {
          cudaStreamEndCapture(a->st, &g);
          if (g) cudaGraphDestroy(g);
          throw;
        }
        a->cg_step_launches = a->launches - l0;
        a->launches = l0;
        CK(cudaStreamEndCapture(a->st, &g));
        cudaGraphExec_t ge = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        CK(ie);
        a->cg_gexec[slot] = ge;
      }
      CK(cudaGraphLaunch(a->cg_gexec[slot], a->st));
      a->launches += a->cg_step_launches;
    } else {
      enqueue_iter(slot);
    }
    if (it >= lag) {
      volatile int *hn = a->h_nact;
      const int ps = (it - lag) % RING;
      const auto t0 = std::chrono::steady_clock::now();
      while (hn[ps] == -1) {
        const cudaError_t q = cudaStreamQuery(a->st);
        if (q != cudaSuccess && q != cudaErrorNotReady) CK(q);  // a device fault: report it now
        if (q == cudaSuccess && hn[ps] == -1) throw MomaError(MOMA_ERR_CUDA, "poll copy did not arrive");
        if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60))
          throw MomaError(MOMA_ERR_TIMEOUT, "inner iteration poll timed out");
        std::this_thread::yield();
      }
      if (hn[ps] == 0) break;
    }
  }
  CK(cudaStreamSynchronize(a->st));
  std::vector<int> its(nr);
  CK(cudaMemcpy(its.data(), c.iters, nr * sizeof(int), cudaMemcpyDeviceToHost));
  int mx = 0;
  for (int k = 0; k < nr; ++k) mx = std::max(mx, its[k]);
  *inner_iters += mx;
  if (first_red) {
    std::vector<double> rr(nr), rr0(nr);
    CK(cudaMemcpy(rr.data(), c.rr, nr * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(rr0.data(), c.rr0, nr * sizeof(double), cudaMemcpyDeviceToHost));
    double m2 = 0;
    for (int k = 0; k < nr; ++k)
      if (act[k] && rr0[k] > 0) m2 = std::max(m2, std::sqrt(rr[k] / rr0[k]));
    *first_red = m2;
  }
  a->timed(PK_KRYLOV, [&] { launch_cg_accum<R>(d, (int)a->ldv, nr, a->Iw.as<double2>(), a->rnorm, a->st); });
  check_launch(a);
}

// R: inner (Krylov) arithmetic; H: arithmetic of the refinement residual
// V - Z I (FP64, or double-FP32 pairs of ~48 bits in the default mixed path).
// Inside a solve (and the operator timing) the array works on an internal
// non-blocking stream, capturable into CUDA graphs, ordered after the
// array's own stream on entry and before it on exit.  Without graphs (or
// while profiling) the array's stream is used directly.
struct StreamSwitch {
  moma_array *a;
  cudaStream_t user;
  bool on = false;
  StreamSwitch(moma_array *a_) : a(a_), user(a_->st) {
    if (!a->use_graphs || a->prof) return;
    if (!a->gs) {
      CK(cudaStreamCreateWithFlags(&a->gs, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&a->ev_in, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&a->ev_out, cudaEventDisableTiming));
    }
    CK(cudaEventRecord(a->ev_in, user));
    CK(cudaStreamWaitEvent(a->gs, a->ev_in, 0));
    a->st = a->gs;
    on = true;
  }
  ~StreamSwitch() {
    if (!on) return;
    cudaEventRecord(a->ev_out, a->gs);
    cudaStreamWaitEvent(user, a->ev_out, 0);
    a->st = user;
  }
};

template <typename R, typename H>
void solve_impl(moma_array *a, int nr, const void *Vin, void *Iout, const moma_solve_opts *o, moma_solve_info *info,
                double *relres) {
  const double tol = (o && o->tol > 0) ? o->tol : 1e-10;
  const double itol = (o && o->inner_tol > 0) ? o->inner_tol : (is64<R>() ? tol * 0.1 : 1e-5);
  const int max_outer = (o && o->max_outer > 0) ? o->max_outer : 30;
  const bool warm = o && o->warm_start;
  const size_t bytes = (size_t)nr * a->ldv * sizeof(double2);
  a->ctl.inner_tol = itol;

  // The solve runs on an internal non-blocking stream (capturable into
  // graphs), ordered after the array's stream on entry and before it on exit.
  StreamSwitch sw(a);
  autotune(a, nr);

  // Inputs into the solver's own buffers.
  CK(cudaMemcpyAsync(a->Vw.p, Vin, bytes, cudaMemcpyDefault, a->st));
  if (warm) CK(cudaMemcpyAsync(a->Iw.p, Iout, bytes, cudaMemcpyDefault, a->st));
  else CK(cudaMemsetAsync(a->Iw.p, 0, bytes, a->st));
  check_finite(a, a->Vw.p, (size_t)nr * a->ldv * 2, 1);
  a->timed(PK_MISC, [&] { launch_resid(a->Vw.as<double2>(), nullptr, nullptr, (int)a->ldv, nr, a->rpart, a->rcount, a->vnorm, a->st); });
  check_launch(a);
  sync_and_check(a);

  std::vector<double> vn(nr), rn(nr), rel(nr);
  std::vector<int> mask(nr);
  CK(cudaMemcpy(vn.data(), a->vnorm, nr * sizeof(double), cudaMemcpyDeviceToHost));
  int outer = 0, inner = 0;
  double first_red = -1;
  bool converged = false;
  for (;;) {
    // True residual r = V - Z I in FP64 (c128 bins); I = 0 needs no product.
    if (outer == 0 && !warm) {
      a->timed(PK_MISC, [&] { launch_resid(a->Vw.as<double2>(), nullptr, a->rw.as<double2>(), (int)a->ldv, nr, a->rpart, a->rcount, a->rnorm, a->st); });
    } else {
      apply_z<H>(a, nr, a->Iw.p, a->yw.p, 0);
      a->timed(PK_MISC, [&] { launch_resid(a->Vw.as<double2>(), a->yw.as<double2>(), a->rw.as<double2>(), (int)a->ldv, nr, a->rpart, a->rcount,
                   a->rnorm, a->st); });
    }
    check_launch(a);
    CK(cudaMemcpyAsync(a->h_norms, a->rnorm, nr * sizeof(double), cudaMemcpyDeviceToHost, a->st));
    sync_and_check(a);
    std::memcpy(rn.data(), a->h_norms, nr * sizeof(double));
    int nact = 0;
    for (int q = 0; q < nr; ++q) {
      if (!std::isfinite(rn[q])) throw MomaError(MOMA_ERR_NONFINITE, "non-finite residual");
      rel[q] = vn[q] > 0 ? rn[q] / vn[q] : 0.0;
      mask[q] = rel[q] > tol ? 1 : 0;
      nact += mask[q];
    }
    if (nact == 0) { converged = true; break; }
    if (outer >= max_outer) break;
    CK(cudaMemcpyAsync(a->mask, mask.data(), nr * sizeof(int), cudaMemcpyHostToDevice, a->st));
    a->timed(PK_MISC, [&] { launch_to_inner<R>(a->rw.as<double2>(), a->lat_in.p, (int)a->ldv, nr, a->rnorm, a->mask, a->st); });
    check_launch(a);
    if (o && o->solver == MOMA_SOLVER_PCG)
      pcg_cycle<R>(a, nr, mask, (o->max_inner > 0) ? o->max_inner : 500, &inner, outer == 0 ? &first_red : nullptr);
    else
      gmres_cycle<R>(a, nr, mask, &inner, outer == 0 ? &first_red : nullptr);
    sync_and_check(a);
    ++outer;
  }
  copy_out(a, Iout, a->Iw.p, bytes);
  CK(cudaStreamSynchronize(a->st));
  double mx = 0;
  for (int q = 0; q < nr; ++q) mx = std::max(mx, rel[q]);
  if (relres) std::memcpy(relres, rel.data(), nr * sizeof(double));
  if (info) {
    info->outer_iters = outer;
    info->inner_iters = inner;
    info->converged = converged ? 1 : 0;
    info->max_rel_residual = mx;
    info->first_inner_reduction = first_red;
  }
  if (!converged) throw MomaError(MOMA_ERR_NOT_CONVERGED, "solve reached max_outer before tol");
}

template <typename F> moma_status guarded(F &&f) {
  try {
    f();
    return MOMA_OK;
  } catch (const MomaError &e) {
    g_last_error = e.what();
    return e.st;
  } catch (const std::bad_alloc &) {
    g_last_error = "host allocation failed";
    return MOMA_ERR_OOM;
  } catch (const std::exception &e) {
    g_last_error = e.what();
    return MOMA_ERR_ARG;
  }
}

void destroy_impl(moma_array *a) {
  DevBuf *bufs[] = {&a->tabs, &a->pairs, &a->slot_of, &a->bin_slot, &a->tri, &a->tri_in, &a->Z128, &a->Z64, &a->Xinv, &a->blk, &a->T, &a->S,
                    &a->Lpk, &a->lat_in, &a->lat_tmp, &a->t1, &a->bx, &a->by, &a->Vk, &a->Iw, &a->Vw,
                    &a->rw, &a->yw, &a->kbuf, &a->errbuf, &a->one_blk, &a->portsb, &a->zp_V, &a->zp_I, &a->zp_Y, &a->zp_tmp,
                    &a->tcA, &a->tcP, &a->partner, &a->Xblk, &a->gramY, &a->tamap, &a->lat_u, &a->mZB128,
                    &a->mZC128, &a->mZB64, &a->mZC64, &a->mP, &a->mL, &a->mX, &a->Wb};
  for (DevBuf *b : bufs) b->release(a->dev_bytes);
  if (a->cs) {
    cudaStreamSynchronize(a->cs);
    cudaStreamDestroy(a->cs);
    cudaEventDestroy(a->ev_cs0);
    for (auto e : a->ev_chunk) cudaEventDestroy(e);
  }
  if (a->h_nact) cudaFreeHost(a->h_nact);
  if (a->h_norms) cudaFreeHost(a->h_norms);
  if (a->h_err) cudaFreeHost(a->h_err);
  for (auto e : a->poll_ev) cudaEventDestroy(e);
  drop_graphs(a);
  if (a->gs) {
    cudaStreamSynchronize(a->gs);
    cudaStreamDestroy(a->gs);
    cudaEventDestroy(a->ev_in);
    cudaEventDestroy(a->ev_out);
  }
  for (auto &p : a->ev_pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (auto e : a->ev_free) cudaEventDestroy(e);
  delete a;
}

}  // namespace

// ===================================================================== ABI ==
extern "C" {

const char *moma_last_error(void) { return g_last_error.c_str(); }

moma_status moma_create_array(int nx, int ny, int b, const moma_options *opt, void *cuda_stream, moma_array **out) {
  if (out) *out = nullptr;
  moma_array *a = nullptr;
  moma_status s = guarded([&] {
    if (!out) throw MomaError(MOMA_ERR_ARG, "out is NULL");
    if (nx < 1 || ny < 1 || b < 1) throw MomaError(MOMA_ERR_ARG, "nx, ny, b must be >= 1");
    if ((long long)nx * ny * b > (1ll << 31) / 4) throw MomaError(MOMA_ERR_ARG, "lattice too large");
    a = new moma_array();
    a->nx = nx; a->ny = ny; a->b = b; a->nel = nx * ny; a->N = nx * ny * b;
    a->ldv = a->N;
    a->st = reinterpret_cast<cudaStream_t>(cuda_stream);
    const int prec = opt ? opt->precision : MOMA_PREC_MIXED;
    if (prec != MOMA_PREC_FP64 && prec != MOMA_PREC_MIXED) throw MomaError(MOMA_ERR_ARG, "bad precision");
    // Preconditioner blocks up to 256 x 256 (the box Cholesky's (i, k) table
    // and the bin product's per-warp column sums must fit in shared memory).
    if (b > 256) throw MomaError(MOMA_ERR_ARG, "b too large for this build (b <= 256)");
    a->prec = prec;
    a->df = prec == MOMA_PREC_MIXED && !(opt && (opt->flags & MOMA_FLAG_FP64_RESIDUAL));
    a->m = (opt && opt->restart > 0) ? opt->restart : 50;
    a->use_graphs = !(opt && (opt->flags & MOMA_FLAG_NO_GRAPHS));
    a->no_autotune = opt && (opt->flags & MOMA_FLAG_NO_AUTOTUNE);
    a->no_tensor = opt && (opt->flags & MOMA_FLAG_NO_TENSOR);
    a->axis_fft = opt && (opt->flags & MOMA_FLAG_AXIS_FFT);
    a->no_blk_precond = opt && (opt->flags & MOMA_FLAG_PRECOND_PER_ELEMENT);
    a->no_fused_arnoldi = opt && (opt->flags & MOMA_FLAG_SPLIT_ARNOLDI);
    if (opt && (opt->flags & MOMA_FLAG_TENSOR_ALWAYS)) a->tc_min_nr = 1;
    if (a->m > MOMA_MAX_RESTART) throw MomaError(MOMA_ERR_ARG, "restart too large");
    const int mx = (opt && opt->mx > 0) ? opt->mx : next_smooth(2 * nx - 1);
    const int my = (opt && opt->my > 0) ? opt->my : next_smooth(2 * ny - 1);
    if (mx < 2 * nx - 1 || my < 2 * ny - 1) throw MomaError(MOMA_ERR_ARG, "circulant size must be >= 2N-1");
    if (!smooth_235(mx) || !smooth_235(my)) throw MomaError(MOMA_ERR_ARG, "circulant sizes must be 2^a 3^b 5^c");
    if ((size_t)std::max(mx, my) * 16 * 32 > 190 * 1024) throw MomaError(MOMA_ERR_ARG, "circulant size too large");
    a->Mx = mx; a->My = my; a->B = mx * my;
    a->ldb = (b % 2) ? b + 1 : b;  // rows of the pair storage are 16-byte multiples in c64
    CK(cudaGetDevice(&a->dev));
    CK(cudaDeviceGetAttribute(&a->num_sms, cudaDevAttrMultiProcessorCount, a->dev));
    build_tables(a);
    // The cluster transforms' fit on this device is queried once per kernel
    // shape; do it here, outside any graph capture.
    for (int py : {2, 4}) lattice_cluster_supported(mx, my, nx, ny, 4, py);
    a->Z128.ensure((size_t)a->Bp * b * a->ldb * sizeof(double2), a->dev_bytes);
    CK(cudaMemsetAsync(a->Z128.p, 0, a->Z128.cap, a->st));  // stream-ordered (see ensure_ws)
    if (prec == MOMA_PREC_MIXED) {
      a->Z64.ensure((size_t)a->Bp * b * a->ldb * sizeof(float2), a->dev_bytes);
      CK(cudaMemsetAsync(a->Z64.p, 0, a->Z64.cap, a->st));
    }
    a->errbuf.ensure(256, a->dev_bytes);
    CK(cudaMemsetAsync(a->errbuf.p, 0, 256, a->st));
    CK(cudaStreamSynchronize(a->st));
    a->err = a->errbuf.as<unsigned>();
    CK(cudaMallocHost(&a->h_nact, (MOMA_MAX_RESTART + 8) * sizeof(int)));
    CK(cudaMallocHost(&a->h_err, 64));
    *out = a;
  });
  if (s != MOMA_OK && a) destroy_impl(a);
  return s;
}

moma_status moma_set_blocks(moma_array *a, const void *blocks, int dtype) {
  if (!a) { g_last_error = "array is NULL"; return MOMA_ERR_ARG; }
  return guarded([&] { set_blocks_impl(a, blocks, dtype); });
}

moma_status moma_matvec(moma_array *a, int op, int nrhs, const void *x, void *y, int dtype) {
  if (!a) { g_last_error = "array is NULL"; return MOMA_ERR_ARG; }
  return guarded([&] {
    if (!a->have_blocks) throw MomaError(MOMA_ERR_STATE, "set_blocks must precede matvec");
    if (op < MOMA_OP_Z || op > MOMA_OP_NORMAL) throw MomaError(MOMA_ERR_ARG, "bad op");
    if (nrhs < 0 || (nrhs > 0 && (!x || !y))) throw MomaError(MOMA_ERR_ARG, "bad nrhs or NULL buffer");
    if (dtype != MOMA_C128 && dtype != MOMA_C64) throw MomaError(MOMA_ERR_ARG, "bad dtype");
    const bool d64 = dtype == MOMA_C128;
    if (!d64 && a->prec != MOMA_PREC_MIXED) throw MomaError(MOMA_ERR_ARG, "c64 operators need a MIXED array");
    if (op == MOMA_OP_NORMAL && d64 != (a->prec == MOMA_PREC_FP64))
      throw MomaError(MOMA_ERR_ARG, "the normal operator runs in the array's inner precision");
    if (nrhs == 0) return;
    ensure_ws(a, nrhs);
    ensure_tc(a, nrhs);
    const size_t bytes = (size_t)nrhs * a->ldv * (d64 ? sizeof(double2) : sizeof(float2));
    CK(cudaMemcpyAsync(a->Vw.p, x, bytes, cudaMemcpyDefault, a->st));
    if (d64) {
      if (op == MOMA_OP_NORMAL) apply_normal<double>(a, nrhs, a->Vw.p, a->yw.p);
      else if (a->df) apply_z<dfl>(a, nrhs, a->Vw.p, a->yw.p, op == MOMA_OP_ZH);
      else apply_z<double>(a, nrhs, a->Vw.p, a->yw.p, op == MOMA_OP_ZH);
    } else {
      if (op == MOMA_OP_NORMAL) apply_normal<float>(a, nrhs, a->Vw.p, a->yw.p);
      else apply_z<float>(a, nrhs, a->Vw.p, a->yw.p, op == MOMA_OP_ZH);
    }
    copy_out(a, y, a->yw.p, bytes);
    sync_and_check(a);
  });
}

moma_status moma_apply_precond(moma_array *a, int nrhs, const void *x, void *y, int dtype) {
  if (!a) { g_last_error = "array is NULL"; return MOMA_ERR_ARG; }
  return guarded([&] {
    if (!a->have_blocks) throw MomaError(MOMA_ERR_STATE, "set_blocks must precede apply_precond");
    const bool d64 = dtype == MOMA_C128;
    if ((dtype != MOMA_C128 && dtype != MOMA_C64) || d64 != (a->prec == MOMA_PREC_FP64))
      throw MomaError(MOMA_ERR_ARG, "the preconditioner is stored in the array's inner precision");
    if (nrhs < 0 || (nrhs > 0 && (!x || !y))) throw MomaError(MOMA_ERR_ARG, "bad nrhs or NULL buffer");
    if (nrhs == 0) return;
    ensure_ws(a, nrhs);
    ensure_tc(a, nrhs);
    const size_t bytes = (size_t)nrhs * a->ldv * (d64 ? sizeof(double2) : sizeof(float2));
    CK(cudaMemcpyAsync(a->Vw.p, x, bytes, cudaMemcpyDefault, a->st));
    if (d64) precond<double>(a, nrhs, a->Vw.p, a->yw.p);
    else precond<float>(a, nrhs, a->Vw.p, a->yw.p);
    copy_out(a, y, a->yw.p, bytes);
    sync_and_check(a);
  });
}

moma_status moma_get_bin(moma_array *a, int kx, int ky, int dtype, void *out) {
  if (!a) { g_last_error = "array is NULL"; return MOMA_ERR_ARG; }
  return guarded([&] {
    if (!a->have_blocks) throw MomaError(MOMA_ERR_STATE, "no blocks");
    if (kx < 0 || kx >= a->Mx || ky < 0 || ky >= a->My || !out) throw MomaError(MOMA_ERR_ARG, "bad bin");
    if (dtype != MOMA_C128 && !(dtype == MOMA_C64 && a->prec == MOMA_PREC_MIXED))
      throw MomaError(MOMA_ERR_ARG, "bad dtype");
    const int k = ky * a->Mx + kx;
    const int nk = ((a->My - ky) % a->My) * a->Mx + ((a->Mx - kx) % a->Mx);
    const int canon = std::min(k, nk);
    std::vector<int> slot(a->B);
    CK(cudaMemcpy(slot.data(), a->slot_of.p, a->B * sizeof(int), cudaMemcpyDeviceToHost));
    const int s = slot[canon];
    const size_t esz = dtype == MOMA_C128 ? 16 : 8;
    const int b = a->b, ldb = a->ldb;
    std::vector<unsigned char> blk((size_t)b * ldb * esz), res((size_t)b * b * esz);
    const void *src = dtype == MOMA_C128 ? a->Z128.p : a->Z64.p;
    CK(cudaMemcpy(blk.data(), (const unsigned char *)src + (size_t)s * b * ldb * esz, blk.size(),
                  cudaMemcpyDeviceToHost));
    const bool transpose = k != canon;
    // In the default mixed path the c128-class bins are stored as double-FP32 pairs.
    const bool from_df = dtype == MOMA_C128 && a->df;
    for (int i = 0; i < b; ++i)
      for (int j = 0; j < b; ++j) {
        const int si = transpose ? j : i, sj = transpose ? i : j;
        const unsigned char *e = &blk[((size_t)si * ldb + sj) * esz];
        if (from_df) {
          dfl2 v;
          std::memcpy(&v, e, sizeof(v));
          const double2 d = make_double2((double)v.x, (double)v.y);
          std::memcpy(&res[((size_t)i * b + j) * esz], &d, esz);
        } else {
          std::memcpy(&res[((size_t)i * b + j) * esz], e, esz);
        }
      }
    if (is_device_ptr(out)) CK(cudaMemcpy(out, res.data(), res.size(), cudaMemcpyHostToDevice));
    else std::memcpy(out, res.data(), res.size());
  });
}

moma_status moma_get_precond_block(moma_array *a, int ex, int ey, void *out) {
  if (!a) { g_last_error = "array is NULL"; return MOMA_ERR_ARG; }
  return guarded([&] {
    if (!a->have_blocks) throw MomaError(MOMA_ERR_STATE, "no blocks");
    if (!a->pbox) throw MomaError(MOMA_ERR_STATE, "set-up scratch was released");
    if (ex < 0 || ex >= a->nx || ey < 0 || ey >= a->ny || !out) throw MomaError(MOMA_ERR_ARG, "bad element");
    const size_t bytes = (size_t)a->b * a->b * sizeof(double2);
    a->one_blk.ensure(bytes, a->dev_bytes);
    launch_box_one(a->pbox, a->nx, a->b, ex, ey, a->pbox_df, a->one_blk.as<double2>(), a->st);
    check_launch(a);
    copy_out(a, out, a->one_blk.p, bytes);
    sync_and_check(a);
  });
}

moma_status moma_solve(moma_array *a, int nrhs, const void *V, void *I, const moma_solve_opts *opts,
                       moma_solve_info *info, double *rel_residual) {
  if (!a) { g_last_error = "array is NULL"; return MOMA_ERR_ARG; }
  if (info) std::memset(info, 0, sizeof(*info));
  return guarded([&] {
    if (!a->have_blocks) throw MomaError(MOMA_ERR_STATE, "set_blocks must precede solve");
    if (nrhs < 0 || (nrhs > 0 && (!V || !I))) throw MomaError(MOMA_ERR_ARG, "bad nrhs or NULL buffer");
    if (nrhs == 0) {
      if (info) info->converged = 1;
      return;
    }
    ensure_ws(a, nrhs);
    ensure_tc(a, nrhs);
    if (a->prec == MOMA_PREC_FP64) solve_impl<double, double>(a, nrhs, V, I, opts, info, rel_residual);
    else if (a->df) solve_impl<float, dfl>(a, nrhs, V, I, opts, info, rel_residual);
    else solve_impl<float, double>(a, nrhs, V, I, opts, info, rel_residual);
  });
}

moma_status moma_active_impedance(moma_array *a, int nrhs, const void *I, const void *V, int port_basis, double z0,
                                  void *Za, void *Gamma) {
  if (!a) { g_last_error = "array is NULL"; return MOMA_ERR_ARG; }
  return guarded([&] {
    if (nrhs < 0 || (nrhs > 0 && (!I || !V || !Za))) throw MomaError(MOMA_ERR_ARG, "bad nrhs or NULL buffer");
    if (port_basis < 0 || port_basis >= a->b) throw MomaError(MOMA_ERR_ARG, "port_basis out of range");
    if (nrhs == 0) return;
    ensure_ws(a, nrhs);
    const size_t bytes = (size_t)nrhs * a->ldv * sizeof(double2);
    CK(cudaMemcpyAsync(a->rw.p, I, bytes, cudaMemcpyDefault, a->st));
    CK(cudaMemcpyAsync(a->Vw.p, V, bytes, cudaMemcpyDefault, a->st));
    a->portsb.ensure((size_t)2 * nrhs * a->nel * sizeof(double2), a->dev_bytes);
    double2 *za = a->portsb.as<double2>();
    double2 *ga = Gamma ? za + (size_t)nrhs * a->nel : nullptr;
    launch_ports(a->rw.as<double2>(), a->Vw.as<double2>(), a->nel, a->b, nrhs, port_basis, z0, za, ga, a->err, a->ldv,
                 a->st);
    check_launch(a);
    copy_out(a, Za, za, (size_t)nrhs * a->nel * sizeof(double2));
    if (Gamma) copy_out(a, Gamma, ga, (size_t)nrhs * a->nel * sizeof(double2));
    sync_and_check(a);
  });
}

moma_status moma_port_impedance(moma_array *a, int port_basis, int chunk, const moma_solve_opts *opts, void *Zp,
                                void *Yp) {
  if (!a) { g_last_error = "array is NULL"; return MOMA_ERR_ARG; }
  return guarded([&] {
    if (!a->have_blocks) throw MomaError(MOMA_ERR_STATE, "set_blocks must precede moma_port_impedance");
    if (port_basis < 0 || port_basis >= a->b) throw MomaError(MOMA_ERR_ARG, "port_basis out of range");
    if (!Zp && !Yp) throw MomaError(MOMA_ERR_ARG, "Zp and Yp are both NULL");
    const int n = a->nel;
    if (chunk <= 0) chunk = 64;
    if (chunk > n) chunk = n;
    const size_t vbytes = (size_t)chunk * a->ldv * sizeof(double2);
    a->zp_V.ensure(vbytes, a->dev_bytes);
    a->zp_I.ensure(vbytes, a->dev_bytes);
    a->zp_Y.ensure((size_t)n * n * sizeof(double2), a->dev_bytes);
    a->zp_tmp.ensure((size_t)n * (sizeof(double2) + sizeof(int)) + 256, a->dev_bytes);
    double2 *Y = a->zp_Y.as<double2>();
    for (int j0 = 0; j0 < n; j0 += chunk) {
      const int nq = std::min(chunk, n - j0);
      launch_unit_ports(a->zp_V.as<double2>(), n, a->b, port_basis, j0, nq, a->ldv, a->st);
      check_launch(a);
      CK(cudaMemsetAsync(a->zp_I.p, 0, (size_t)nq * a->ldv * sizeof(double2), a->st));
      moma_solve_info info{};
      const moma_status s = moma_solve(a, nq, a->zp_V.p, a->zp_I.p, opts, &info, nullptr);
      if (s != MOMA_OK) throw MomaError(s, std::string("port solve: ") + moma_last_error());
      launch_gather_ports(a->zp_I.as<double2>(), n, a->b, port_basis, j0, nq, Y, a->ldv, a->st);
      check_launch(a);
    }
    if (Yp) copy_out(a, Yp, Y, (size_t)n * n * sizeof(double2));
    if (Zp) {
      double2 *colk = a->zp_tmp.as<double2>();
      int *perm = reinterpret_cast<int *>(a->zp_tmp.as<unsigned char>() + (size_t)n * sizeof(double2));
      launch_invert(Y, n, perm, colk, a->err, a->st);
      check_launch(a);
      copy_out(a, Zp, Y, (size_t)n * n * sizeof(double2));
    }
    sync_and_check(a);
  });
}

// ------------------------------------------------------------ predictors --
namespace {
int centre_of(int nx, int ny) { return nx / 2 + nx * (ny / 2); }
// Border element (outermost ring) closest to the centre; ties: on the
// centre's row first, then the smallest index.
int closest_border(int nx, int ny) {
  const int cx = nx / 2, cy = ny / 2;
  long best_d = -1;
  int best_row = 2, best_e = -1;
  for (int my = 0; my < ny; ++my)
    for (int mx = 0; mx < nx; ++mx) {
      if (!(mx == 0 || mx == nx - 1 || my == 0 || my == ny - 1)) continue;
      const long d = (long)(mx - cx) * (mx - cx) + (long)(my - cy) * (my - cy);
      const int row = my == cy ? 0 : 1, e = mx + nx * my;
      if (best_e < 0 || d < best_d || (d == best_d && (row < best_row || (row == best_row && e < best_e)))) {
        best_d = d;
        best_row = row;
        best_e = e;
      }
    }
  return best_e;
}
double cabs2(double2 v) { return std::sqrt(v.x * v.x + v.y * v.y); }
// Row c of an n x n c128 matrix (host or device) into host memory.
std::vector<double2> matrix_row(const void *M, int n, int c) {
  std::vector<double2> row(n);
  const double2 *src = static_cast<const double2 *>(M) + (size_t)c * n;
  CK(cudaMemcpy(row.data(), src, (size_t)n * sizeof(double2), cudaMemcpyDefault));
  return row;
}
struct ScratchDev {
  void *p = nullptr;
  explicit ScratchDev(size_t bytes) {
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      throw MomaError(MOMA_ERR_OOM, "device allocation failed");
    }
  }
  ~ScratchDev() {
    if (p) cudaFree(p);
  }
};
// Z = z0 (I + S)(I - S)^{-1} on the device for S host or device.
void z_from_s_impl(const void *S, int n, double z0, void *Zp, cudaStream_t st) {
  const size_t mat = (size_t)n * n * sizeof(double2);
  ScratchDev buf(3 * mat + (size_t)n * (sizeof(double2) + sizeof(int)) + 256);
  double2 *Sd = static_cast<double2 *>(buf.p), *Zd = Sd + (size_t)n * n, *work = Zd + (size_t)n * n;
  unsigned *err = reinterpret_cast<unsigned *>(reinterpret_cast<unsigned char *>(buf.p) + 3 * mat +
                                               (size_t)n * (sizeof(double2) + sizeof(int)));
  CK(cudaMemsetAsync(err, 0, sizeof(unsigned), st));
  CK(cudaMemcpyAsync(Sd, S, mat, cudaMemcpyDefault, st));
  launch_z_from_s(Sd, n, z0, Zd, work, err, st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(Zp, Zd, mat, cudaMemcpyDefault, st));
  unsigned h = 0;
  CK(cudaMemcpyAsync(&h, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h) throw MomaError(MOMA_ERR_NONFINITE, "I - S is singular (zero pivot)");
}
}  // namespace

moma_status moma_column_coupling(moma_array *a, int port_basis, int nq, int nmax, double z0,
                                 const moma_solve_opts *opts, void *C, void *gamma) {
  if (!a) { g_last_error = "array is NULL"; return MOMA_ERR_ARG; }
  return guarded([&] {
    if (!a->have_blocks) throw MomaError(MOMA_ERR_STATE, "set_blocks must precede moma_column_coupling");
    if (port_basis < 0 || port_basis >= a->b) throw MomaError(MOMA_ERR_ARG, "port_basis out of range");
    if (nq < 1 || nmax < 0 || !C) throw MomaError(MOMA_ERR_ARG, "need nq >= 1, nmax >= 0 and C");
    const int chunk = std::min(nq, 64), nel = a->nel, c = centre_of(a->nx, a->ny);
    const size_t vbytes = (size_t)chunk * a->ldv * sizeof(double2);
    a->zp_V.ensure(vbytes, a->dev_bytes);
    a->zp_I.ensure(vbytes, a->dev_bytes);
    a->portsb.ensure((size_t)2 * chunk * nel * sizeof(double2), a->dev_bytes);
    a->zp_tmp.ensure((size_t)(nq + 2 * nmax + 1) * sizeof(double2) + 256, a->dev_bytes);
    double2 *gam_d = a->zp_tmp.as<double2>(), *C_d = gam_d + nq;
    double2 *za = a->portsb.as<double2>(), *ga = za + (size_t)chunk * nel;
    for (int q0 = 0; q0 < nq; q0 += chunk) {
      const int nqc = std::min(chunk, nq - q0);
      launch_row_phase(a->zp_V.as<double2>(), a->nx, nel, a->b, port_basis, q0, nqc, nq, a->ldv, a->st);
      check_launch(a);
      moma_solve_info info{};
      const moma_status s = moma_solve(a, nqc, a->zp_V.p, a->zp_I.p, opts, &info, nullptr);
      if (s != MOMA_OK) throw MomaError(s, std::string("phase-sweep solve: ") + moma_last_error());
      launch_ports(a->zp_I.as<double2>(), a->zp_V.as<double2>(), nel, a->b, nqc, port_basis, z0, za, ga, a->err,
                   a->ldv, a->st);
      check_launch(a);
      CK(cudaMemcpy2DAsync(gam_d + q0, sizeof(double2), ga + c, (size_t)nel * sizeof(double2), sizeof(double2), nqc,
                           cudaMemcpyDeviceToDevice, a->st));
    }
    launch_column_coupling(gam_d, nq, nmax, C_d, a->st);
    check_launch(a);
    copy_out(a, C, C_d, (size_t)(2 * nmax + 1) * sizeof(double2));
    if (gamma) copy_out(a, gamma, gam_d, (size_t)nq * sizeof(double2));
    sync_and_check(a);
  });
}

moma_status moma_s_to_z(const void *S, int n, double z0, void *Zp, void *cuda_stream) {
  return guarded([&] {
    if (!S || !Zp || n < 1) throw MomaError(MOMA_ERR_ARG, "need S, Zp and n >= 1");
    z_from_s_impl(S, n, z0, Zp, reinterpret_cast<cudaStream_t>(cuda_stream));
  });
}

moma_status moma_s_ideal(int nx, int ny, double s_cc_re, double s_cc_im, double s1_re, double s1_im, double kd,
                         void *S, void *cuda_stream) {
  return guarded([&] {
    if (nx < 1 || ny < 1 || !S) throw MomaError(MOMA_ERR_ARG, "need nx, ny >= 1 and S");
    const int n = nx * ny;
    const size_t mat = (size_t)n * n * sizeof(double2);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    double2 *dst = static_cast<double2 *>(S);
    std::unique_ptr<ScratchDev> tmp;
    if (!is_device_ptr(S)) {
      tmp.reset(new ScratchDev(mat));
      dst = static_cast<double2 *>(tmp->p);
    }
    launch_s_ideal(dst, nx, ny, make_double2(s_cc_re, s_cc_im), make_double2(s1_re, s1_im), kd, st);
    CK(cudaGetLastError());
    if (tmp) CK(cudaMemcpyAsync(S, dst, mat, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  });
}

moma_status moma_xi_z(const void *Zp, int nx, int ny, double *out) {
  return guarded([&] {
    if (!Zp || !out || nx < 1 || ny < 1) throw MomaError(MOMA_ERR_ARG, "need Zp, out and nx, ny >= 1");
    const int n = nx * ny, c = centre_of(nx, ny);
    const std::vector<double2> row = matrix_row(Zp, n, c);
    const double zcc = cabs2(row[c]);
    double bound = 0, mx = 0;
    for (int my = 0; my < ny; ++my)
      for (int mxi = 0; mxi < nx; ++mxi) {
        if (!(mxi == 0 || mxi == nx - 1 || my == 0 || my == ny - 1)) continue;
        const double v = cabs2(row[mxi + nx * my]);
        bound += v;
        mx = std::max(mx, v);
      }
    out[0] = cabs2(row[closest_border(nx, ny)]) / zcc;  // Eq. 25
    out[1] = mx / zcc;                                   // Eq. 24
    out[2] = bound;                                      // Eq. 23
  });
}

moma_status moma_xi_s(int nx, int ny, double s_cc_re, double s_cc_im, double s1_re, double s1_im, double kd,
                      double z0, double *xi_s) {
  return guarded([&] {
    if (nx < 1 || ny < 1 || !xi_s) throw MomaError(MOMA_ERR_ARG, "need nx, ny >= 1 and xi_s");
    const int n = nx * ny, c = centre_of(nx, ny);
    const size_t mat = (size_t)n * n * sizeof(double2);
    ScratchDev buf(2 * mat);
    double2 *S = static_cast<double2 *>(buf.p), *Z = S + (size_t)n * n;
    launch_s_ideal(S, nx, ny, make_double2(s_cc_re, s_cc_im), make_double2(s1_re, s1_im), kd, nullptr);
    CK(cudaGetLastError());
    z_from_s_impl(S, n, z0, Z, nullptr);
    const std::vector<double2> row = matrix_row(Z, n, c);
    *xi_s = cabs2(row[closest_border(nx, ny)]) / cabs2(row[c]);  // Eq. 36
  });
}

moma_status moma_set_margin(moma_array *a, int nm, const void *ZB, const void *ZC, int dtype) {
  if (!a) { g_last_error = "array is NULL"; return MOMA_ERR_ARG; }
  return guarded([&] {
    if (nm < 0 || nm > 1024) throw MomaError(MOMA_ERR_ARG, "nm must be in 0..1024");
    if (nm > 0 && (!ZB || !ZC)) throw MomaError(MOMA_ERR_ARG, "ZB and ZC are required");
    if (dtype != MOMA_C128 && dtype != MOMA_C64) throw MomaError(MOMA_ERR_ARG, "bad dtype");
    CK(cudaStreamSynchronize(a->st));
    drop_graphs(a);
    a->ws_nr = 0;  // vector length changes: workspaces are re-sized on the next call
    a->tuned_nr = -1;
    a->nm = nm;
    a->ldv = (long long)a->N + nm;
    if (nm == 0) return;
    const size_t nb = (size_t)nm * a->N, nc = (size_t)nm * nm;
    const size_t esz = dtype == MOMA_C128 ? sizeof(double2) : sizeof(float2);
    DevBuf tmpB, tmpC;
    size_t scratch = 0;
    const void *zb = stage_in(a, ZB, nb * esz, tmpB), *zc = stage_in(a, ZC, nc * esz, tmpC);
    (void)scratch;
    check_finite(a, zb, nb * 2, dtype == MOMA_C128);
    check_finite(a, zc, nc * 2, dtype == MOMA_C128);
    sync_and_check(a);
    a->mZB128.ensure(nb * sizeof(double2), a->dev_bytes);
    a->mZC128.ensure(nc * sizeof(double2), a->dev_bytes);
    launch_convert(zb, dtype == MOMA_C128, a->mZB128.p, 1, nb, a->st);
    launch_convert(zc, dtype == MOMA_C128, a->mZC128.p, 1, nc, a->st);
    if (a->prec == MOMA_PREC_MIXED) {
      a->mZB64.ensure(nb * sizeof(float2), a->dev_bytes);
      a->mZC64.ensure(nc * sizeof(float2), a->dev_bytes);
      launch_convert(zb, dtype == MOMA_C128, a->mZB64.p, 0, nb, a->st);
      launch_convert(zc, dtype == MOMA_C128, a->mZC64.p, 0, nc, a->st);
    }
    // Margin block of the preconditioner (Eq. 38), factored in FP64.
    a->mP.ensure(nc * sizeof(double2), a->dev_bytes);
    const size_t npk = (size_t)nm * (nm + 1) / 2;
    a->mL.ensure(npk * sizeof(double2), a->dev_bytes);
    launch_margin_precond_build(a->mZB128.as<double2>(), a->mZC128.as<double2>(), nm, a->N, a->mP.as<double2>(),
                                a->mL.as<double2>(), a->err, a->st);
    check_launch(a);
    const size_t csz = a->prec == MOMA_PREC_FP64 ? sizeof(double2) : sizeof(float2);
    size_t xs = npk;
    while ((xs * csz) % 16) ++xs;
    a->mx_stride = xs;
    a->mX.ensure(xs * csz, a->dev_bytes);
    if (a->prec == MOMA_PREC_FP64) launch_tri_inverse<double>(a->mL.as<double2>(), 1, nm, a->mX.p, xs, a->st);
    else launch_tri_inverse<float>(a->mL.as<double2>(), 1, nm, a->mX.p, xs, a->st);
    check_launch(a);
    sync_and_check(a);
    tmpB.release(a->dev_bytes);
    tmpC.release(a->dev_bytes);
  });
}

moma_status moma_profile(moma_array *a, int enable) {
  if (!a) { g_last_error = "array is NULL"; return MOMA_ERR_ARG; }
  return guarded([&] {
    CK(cudaStreamSynchronize(a->st));
    a->flush_events();
    for (int k = 0; k < PK_N; ++k) { a->st_launch[k] = 0; a->st_ms[k] = 0; }
    a->prof = enable != 0;
  });
}

moma_status moma_kernel_stats(moma_array *a, int kernel, long long *launches, double *total_ms) {
  if (!a) { g_last_error = "array is NULL"; return MOMA_ERR_ARG; }
  return guarded([&] {
    if (kernel < 0 || kernel >= PK_N) throw MomaError(MOMA_ERR_ARG, "bad kernel id");
    a->flush_events();
    if (launches) *launches = a->st_launch[kernel];
    if (total_ms) *total_ms = a->st_ms[kernel];
  });
}

moma_status moma_time_operator(moma_array *a, int what, int nrhs, int reps, double *us) {
  if (!a) { g_last_error = "array is NULL"; return MOMA_ERR_ARG; }
  return guarded([&] {
    if (!a->have_blocks) throw MomaError(MOMA_ERR_STATE, "set_blocks must precede moma_time_operator");
    if (a->prec != MOMA_PREC_MIXED) throw MomaError(MOMA_ERR_ARG, "c64 operators need a MIXED array");
    if (what < MOMA_TIME_Z || what > MOMA_TIME_NORMAL || nrhs < 1 || reps < 1 || !us)
      throw MomaError(MOMA_ERR_ARG, "bad what, nrhs, reps or output");
    ensure_ws(a, nrhs);
    ensure_tc(a, nrhs);
    autotune(a, nrhs);
    CK(cudaMemsetAsync(a->Vw.p, 0, (size_t)nrhs * a->ldv * sizeof(float2), a->st));
    auto once = [&] {
      switch (what) {
        case MOMA_TIME_Z: apply_z<float>(a, nrhs, a->Vw.p, a->yw.p, 0); break;
        case MOMA_TIME_BIN: binprod<float>(a, nrhs, a->bx.p, a->by.p, 0); break;
        case MOMA_TIME_PRECOND: precond<float>(a, nrhs, a->Vw.p, a->yw.p); break;
        default: apply_normal<float>(a, nrhs, a->Vw.p, a->yw.p); break;
      }
    };
    struct ProfOff {
      moma_array *a;
      bool was;
      ~ProfOff() { a->prof = was; }
    } prof_off{a, a->prof};
    a->prof = false;
    StreamSwitch sw(a);
    once();
    // With graphs (the default) the applications are captured as one CUDA
    // graph and replayed, as the solve replays its inner steps: launches
    // follow each other on the device without host launch gaps.
    cudaGraphExec_t ge = nullptr;
    if (sw.on) {
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(a->st, cudaStreamCaptureModeThreadLocal));
      try {
        for (int r = 0; r < reps; ++r) once();
      } catch (...) {
        cudaStreamEndCapture(a->st, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      CK(cudaStreamEndCapture(a->st, &g));
      const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      CK(ie);
      CK(cudaGraphLaunch(ge, a->st));  // warm-up replay
    }
    struct ExecGuard {
      cudaGraphExec_t e;
      ~ExecGuard() { if (e) cudaGraphExecDestroy(e); }
    } guard{ge};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, a->st));
    if (ge) CK(cudaGraphLaunch(ge, a->st));
    else
      for (int r = 0; r < reps; ++r) once();
    CK(cudaEventRecord(e1, a->st));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    sync_and_check(a);
    *us = 1000.0 * ms / reps;
  });
}

moma_status moma_set_stream(moma_array *a, void *cuda_stream) {
  if (!a) { g_last_error = "array is NULL"; return MOMA_ERR_ARG; }
  return guarded([&] {
    CK(cudaStreamSynchronize(a->st));
    a->st = reinterpret_cast<cudaStream_t>(cuda_stream);
  });
}

void *moma_array_stream(const moma_array *a) { return a ? reinterpret_cast<void *>(a->st) : nullptr; }

moma_status moma_tuning_report(const moma_array *a, char *buf, size_t len) {
  if (!a || !buf || len == 0) { g_last_error = "bad arguments"; return MOMA_ERR_ARG; }
  std::snprintf(buf, len, "%s", a->tune_log.c_str());
  return MOMA_OK;
}

moma_status moma_release_setup(moma_array *a) {
  if (!a) { g_last_error = "array is NULL"; return MOMA_ERR_ARG; }
  return guarded([&] {
    CK(cudaStreamSynchronize(a->st));
    a->blk.release(a->dev_bytes);
    a->gramY.release(a->dev_bytes);
    a->T.release(a->dev_bytes);
    a->S.release(a->dev_bytes);
    a->Wb.release(a->dev_bytes);
    a->pbox = nullptr;
    a->Lpk.release(a->dev_bytes);
  });
}

size_t moma_estimate_bytes(int nx, int ny, int b, const moma_options *opt, int nrhs, int with_setup) {
  if (nx < 1 || ny < 1 || b < 1 || nrhs < 0) return 0;
  const int prec = opt ? opt->precision : MOMA_PREC_MIXED;
  const int m = (opt && opt->restart > 0) ? opt->restart : 50;
  const size_t Mx = (opt && opt->mx > 0) ? opt->mx : next_smooth(2 * nx - 1);
  const size_t My = (opt && opt->my > 0) ? opt->my : next_smooth(2 * ny - 1);
  const size_t B = Mx * My, Bp = B / 2 + 2, ldb = (b % 2) ? b + 1 : b;
  const size_t nel = (size_t)nx * ny, N = nel * b, nt = (size_t)b * (b + 1) / 2;
  const size_t nD = (size_t)(2 * nx - 1) * (2 * ny - 1);
  const size_t c = 16, esz = prec == MOMA_PREC_FP64 ? 16 : 8;
  size_t bytes = Bp * b * ldb * c + (prec == MOMA_PREC_MIXED ? Bp * b * ldb * 8 : 0);  // stored bins
  bytes += nel * (nt + 2) * esz;                                                        // inverse factors
  if (prec == MOMA_PREC_MIXED) bytes += nel * xblk_entries(b) * 8;                    // blocked c64 P_e^{-1}
  bytes += B * 24 + nt * 12 + 4096;                                                     // tables
  const size_t nr = (size_t)nrhs, nch = (N + 1023) / 1024;
  bytes += nr * N * c * 6 + nr * ny * Mx * b * c + 2 * B * nr * b * c;                 // solve vectors
  bytes += (size_t)(m + 1) * nr * N * esz + nr * nch * (m + 1) * c + nr * m * (m + 1) * c;  // Krylov
  bytes += 2 * nr * nel * c;                                                            // ports
  if (with_setup) bytes += nD * b * b * (c + 8) + (size_t)(2 * ny - 1) * Mx * nt * c + nel * nt * c;
  if (with_setup) bytes += box_window_entries(nx, ny, b) * c;                           // box-sum windows
  const bool tens_setup = prec == MOMA_PREC_MIXED && !(opt && (opt->flags & MOMA_FLAG_NO_TENSOR)) && tc_supported(b);
  if (with_setup && tens_setup) bytes += nD * b * b * 8;  // tensor-core Gram products
  const bool tensor = !(opt && (opt->flags & MOMA_FLAG_NO_TENSOR));
  const int tmin = (opt && (opt->flags & MOMA_FLAG_TENSOR_ALWAYS)) ? 1 : 16;
  if (prec == MOMA_PREC_MIXED && tensor && nrhs >= tmin && tc_supported(b))
    bytes += Bp * b * ldb * 8 + 2 * tc_bytes((int)nel, b);  // transposed pair store, split factors
  return bytes;
}

long long moma_launch_count(moma_array *a) { return a ? a->launches : 0; }
size_t moma_device_bytes(const moma_array *a) { return a ? a->dev_bytes : 0; }

void moma_destroy(moma_array *a) {
  if (!a) return;
  cudaStreamSynchronize(a->st);
  destroy_impl(a);
}

}  // extern "C"

// ============================================ allocation-free product ====
// moma_matvec_noalloc: the Z / Z^H product of moma_matvec, for callers that
// must not let a library call allocate device memory at call time.  Its
// scratch (the x-pass lattice buffer and the two bin-vector buffers) lives
// in a file-scope device array of fixed size instead of the handle's
// grow-on-demand workspace.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on device `dev` (the array's device).
// The first call per device resolves it with cudaGetSymbolAddress while
// that device is current, then restores the caller's current device.  The
// cached address stays valid while the device's primary context lives,
// i.e. for the whole process unless the caller resets the device.
void *noalloc_scratch(int dev) {
  if (dev < 0 || dev >= kMaxDevices) throw MomaError(MOMA_ERR_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    int prev = 0;
    CK(cudaGetDevice(&prev));
    if (prev != dev) CK(cudaSetDevice(dev));
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (prev != dev) cudaSetDevice(prev);
    CK(e);
    g_noalloc_ptr[dev] = p;
  }
  return g_noalloc_ptr[dev];
}

// Host-side classification of a caller pointer (no allocation).
PtrWhere where_is(const void *p) {
  PtrWhere w;
  if (!p) return w;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return w;
  }
  w.is_device = (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? 1 : 0;
  w.device = at.device;
  return w;
}

template <typename R>
void noalloc_product(moma_array *a, int nr, const void *x, void *y, int herm, unsigned char *scratch) {
  const size_t esz = sizeof(typename Cplx<R>::T);
  auto a256 = [](size_t n) { return (n + 255) & ~size_t(255); };
  // Layout of noalloc_scratch_need: t1 [nr][Ny][Mx][b], then bx, by [B][nr][b].
  unsigned char *t1 = scratch;
  unsigned char *bx = t1 + a256((size_t)nr * a->ny * a->Mx * a->b * esz);
  unsigned char *by = bx + a256((size_t)a->B * nr * a->b * esz);
  const int c = st_code<R>(), lc = lat_code<R>();
  launch_axis_pass<R>(pass_fx(a, nr, x, t1, lc, c), a->fx, a->st);
  check_launch(a);
  launch_axis_pass<R>(pass_fy(a, nr, t1, bx, c), a->fy, a->st);
  check_launch(a);
  BinProduct P;
  P.Z = is64<R>() ? a->Z128.p : a->Z64.p;
  P.pairs = a->pairs.as<int2>();
  P.x = bx; P.y = by; P.Bp = a->Bp; P.b = a->b; P.ldb = a->ldb; P.nr = nr; P.herm = herm; P.err = a->err;
  launch_bin_product<R>(P, a->num_sms, a->st);
  check_launch(a);
  launch_axis_pass<R>(pass_iy(a, nr, by, t1, c), a->fy, a->st);
  check_launch(a);
  launch_axis_pass<R>(pass_ix(a, nr, t1, y, c, false, lc), a->fx, a->st);
  check_launch(a);
}

}  // namespace

extern "C" moma_status moma_matvec_noalloc(moma_array *a, int op, int nrhs, const void *x, void *y, int dtype) {
  if (!a) { g_last_error = "array is NULL"; return MOMA_ERR_ARG; }
  return guarded([&] {
    if (!a->have_blocks) throw MomaError(MOMA_ERR_STATE, "set_blocks must precede matvec");
    if (op != MOMA_OP_Z && op != MOMA_OP_ZH) throw MomaError(MOMA_ERR_ARG, "op must be MOMA_OP_Z or MOMA_OP_ZH");
    if (dtype != MOMA_C128 && dtype != MOMA_C64) throw MomaError(MOMA_ERR_ARG, "bad dtype");
    if (a->nm > 0) throw MomaError(MOMA_ERR_ARG, "the allocation-free product has no margin terms");
    const bool d64 = dtype == MOMA_C128;
    if (!d64 && a->prec != MOMA_PREC_MIXED) throw MomaError(MOMA_ERR_ARG, "c64 operators need a MIXED array");
    if (nrhs < 0) throw MomaError(MOMA_ERR_ARG, "nrhs < 0");
    if (nrhs == 0) return;
    const size_t esz = d64 ? sizeof(double2) : sizeof(float2);
    const size_t need = noalloc_scratch_need(nrhs, a->ny, a->Mx, a->B, a->b, esz);
    const std::string why = noalloc_check(a->dev, where_is(x), where_is(y), need, kNoAllocScratchBytes);
    if (!why.empty()) throw MomaError(MOMA_ERR_ARG, why);
    unsigned char *scratch = static_cast<unsigned char *>(noalloc_scratch(a->dev));
    if (d64 && a->df) noalloc_product<dfl>(a, nrhs, x, y, op == MOMA_OP_ZH, scratch);
    else if (d64) noalloc_product<double>(a, nrhs, x, y, op == MOMA_OP_ZH, scratch);
    else noalloc_product<float>(a, nrhs, x, y, op == MOMA_OP_ZH, scratch);
    sync_and_check(a);
  });
}
