// Two-dimensional c64 lattice transforms of the MLFFT product (Eq. 2:
// F^[2] = F_{Ny} (x) (F_{Nx} (x) I_b)) in one launch each, on thread-block
// clusters: the x and y passes of one group of basis indices meet in
// distributed shared memory instead of going through L2 between two
// launches.
//
// A cluster of kCl = 8 CTAs owns kClJ = 8 consecutive basis indices j0 ..
// j0+7 of one right-hand side r on the square M x M circulant grid (Eq. 3).
// CTA c of the cluster owns the lattice rows y = c, c + 8, ... (its x lines,
// one per row and basis index) and the grid columns kx = c, c + 8, ... (its y
// lines).  Every line is the split register transform of fftreg.cuh (PX or
// PY lanes per line, one warp-local exchange), with the lane counts the
// per-axis passes of fftreg.cu would take for the same geometry, so each
// line's arithmetic -- and hence the result -- is bit for bit that of those
// passes; only the hand-over between the axes moves:
//   F2     lattice [nr][Ny][Nx][b] -> bins [M][M][nr][b]: x lines of the
//          Ny rows (zero padded to M), each value kx sent to the CTA owning
//          column kx, one cluster barrier, y lines of the owned columns
//          (Ny rows, zero padded), bins stored.
//   I2     bins -> lattice, each axis inverted as conj . DFT . conj / M: y
//          lines of the owned columns, the Ny rows that survive sent to
//          their owners, one cluster barrier, x lines of the owned rows, the
//          Nx points that survive stored.
//   I2MF2  bins -> bins: I2 up to the x lines, whose inverse is masked to
//          the lattice (Sec. III-A: Z^H acts on M Z x) and transformed
//          forward in registers, then sent on as in F2 (a second cluster
//          barrier) and finished by F2's y lines.
// Layouts in shared memory (complex values): Bcol[col][y][jj] with the row
// stride kColJ = 12 (the y lines' loads of four rows by eight basis indices
// cover 32 distinct banks pairs), Brow[row][kx][jj] with the column stride
// kRowJ = 9 (the x lines' loads of eight columns by four basis indices are
// nearly conflict-free); the work split and the offsets are those of
// lattice_cluster.cuh.  Every CTA of a cluster passes every cluster barrier
// (no thread leaves early), so the barriers always complete.  F2 and I2MF2
// let the next kernel launch at their start: the bin product that follows
// is launched as a programmatic dependent and streams its pair store while
// the transform finishes.
#include <stdexcept>

#include "internal.h"
#include "lattice_cluster.cuh"

namespace moma {

namespace {

struct ClTw {
  float2 w[kRegMaxM];
};
struct ClArgs {
  LatticeCluster p;
  ClTw tw;
};

MOMA_DEV uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// The address of the same shared-memory location in CTA `rank` of the cluster.
MOMA_DEV uint32_t cl_map(const void *p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
MOMA_DEV void cl_store(uint32_t addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
MOMA_DEV void cl_arrive_relaxed() { asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory"); }
MOMA_DEV void cl_wait() { asm volatile("barrier.cluster.wait.aligned;" ::: "memory"); }
MOMA_DEV void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// One split transform of the warp's lines, in place (fftreg.cuh steps 1-3).
template <int M, int P>
MOMA_DEV void cl_line_fft(float2 (&v)[M / P], float2 *xb, int lane, int s, int l,
                          const float2 (&w)[LaneShape<M, P>::U][P], const float2 *tw) {
  lane_stage1<M, P>(v, tw);
  lane_put<M, P>(xb, v, lane);
  __syncwarp();
  lane_stage2<M, P>(v, xb, s, l, w, tw);
}
template <int Q>
MOMA_DEV void cl_inverse_finish(float2 (&v)[Q], float inv_m) {
#pragma unroll
  for (int q = 0; q < Q; ++q) v[q] = make_float2(v[q].x * inv_m, -v[q].y * inv_m);
}

template <int M, int PX, int PY, int MODE>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(ClShape<M, PX, PY>::NT)
    lattice_cluster_kernel(const __grid_constant__ ClArgs A, const float2 *__restrict__ tw_full) {
  using S = ClShape<M, PX, PY>;
  extern __shared__ __align__(16) float2 smc[];
  const LatticeCluster &p = A.p;
  if (p.live && *p.live == 0) return;  // the same for every CTA of the grid
  float2 *bcol = smc + S::XBUF;
  float2 *brow = bcol + (MODE != 1 ? S::BCOL : 0);
  const int c = (int)cl_rank();
  const int j0 = (int)(blockIdx.x / kCl) * kClJ, r = blockIdx.y;
  const int nx = p.nx, ny = p.ny, b = p.b;
  const long long bins_row = (long long)p.nr * b;  // elements between consecutive bins
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float2 *xb = smc + warp * S::QMAX * kLaneLd;
  const float2 *tw = A.tw.w;
  const float inv_m = 1.0f / (float)M;
  const float2 zero = make_float2(0.f, 0.f);
  // A bin product launched as a programmatic dependent may start now (it
  // streams the pair store and waits for this grid before reading bins).
  if (MODE != 1) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  cl_arrive_relaxed();  // every CTA of the cluster has started once the matching wait returns

  // ---- y lines: (column colL, basis jj), kx = c + 8 colL ----
  const ClLine ty = cl_line<PY>(c, tid);
  const int sy = ty.s, ly = ty.l, colL = ty.loc, jjy = ty.jj, kx = ty.g;
  const bool acty = colL < S::CPC && j0 + jjy < b;
  // ---- x lines: (row rowL, basis jj), y = c + 8 rowL ----
  const ClLine tx = cl_line<PX>(c, tid);
  const int sx = tx.s, lx = tx.l, rowL = tx.loc, jjx = tx.jj, yx = tx.g;
  const bool rowx = rowL < S::RPC && yx < ny;
  const bool actx = rowx && j0 + jjx < b;

  if constexpr (MODE == 0) {
    // F2 x lines from the lattice.
    float2 w[LaneShape<M, PX>::U][PX];
    lane_twiddles<M, PX>(w, tw_full, sx);
    float2 v[S::QX];
    const float2 *src = static_cast<const float2 *>(p.in) + (long long)r * p.ldv + (long long)yx * nx * b + j0 + jjx;
#pragma unroll
    for (int q = 0; q < S::QX; ++q) {
      const int x = sx + PX * q;
      v[q] = (actx && x < nx) ? src[(long long)x * b] : zero;
    }
    cl_line_fft<M, PX>(v, xb, lane, sx, lx, w, tw);
    cl_wait();
    if (rowx)
#pragma unroll
      for (int q = 0; q < S::QX; ++q) {
        const int k = sx + PX * q;
        cl_store(cl_map(bcol + cl_bcol_off<M, PX, PY>(k, yx, jjx), cl_owner(k)), v[q]);
      }
    cl_sync();
  } else {
    // I2 / I2MF2 y lines from the bins, inverted; rows y < Ny to their owners.
    float2 w[LaneShape<M, PY>::U][PY];
    lane_twiddles<M, PY>(w, tw_full, sy);
    float2 v[S::QY];
    const float2 *src = static_cast<const float2 *>(p.in) + (long long)kx * bins_row + (long long)r * b + j0 + jjy;
#pragma unroll
    for (int q = 0; q < S::QY; ++q) {
      const int ky = sy + PY * q;
      float2 t = acty ? src[(long long)ky * M * bins_row] : zero;
      t.y = -t.y;
      v[q] = t;
    }
    cl_line_fft<M, PY>(v, xb, lane, sy, ly, w, tw);
    cl_inverse_finish<S::QY>(v, inv_m);
    cl_wait();
    if (colL < S::CPC)
#pragma unroll
      for (int q = 0; q < S::QY; ++q) {
        const int y = sy + PY * q;
        if (y < ny) cl_store(cl_map(brow + cl_brow_off<M>(y, kx, jjy), cl_owner(y)), v[q]);
      }
    cl_sync();

    // x lines of the owned rows, inverted.
    float2 wx[LaneShape<M, PX>::U][PX];
    lane_twiddles<M, PX>(wx, tw_full, sx);
    float2 u[S::QX];
#pragma unroll
    for (int q = 0; q < S::QX; ++q) {
      float2 t = rowx ? brow[cl_brow_off<M>(yx, sx + PX * q, jjx)] : zero;
      t.y = -t.y;
      u[q] = t;
    }
    cl_line_fft<M, PX>(u, xb, lane, sx, lx, wx, tw);
    cl_inverse_finish<S::QX>(u, inv_m);
    if constexpr (MODE == 1) {
      if (actx) {
        float2 *dst = static_cast<float2 *>(p.out) + (long long)r * p.ldv + (long long)yx * nx * b + j0 + jjx;
#pragma unroll
        for (int q = 0; q < S::QX; ++q) {
          const int x = sx + PX * q;
          if (x < nx) dst[(long long)x * b] = u[q];
        }
      }
      return;
    } else {
      // Lattice mask, forward x transform, values kx to their owners.
#pragma unroll
      for (int q = 0; q < S::QX; ++q)
        if (sx + PX * q >= nx) u[q] = zero;
      __syncwarp();  // every lane has read the exchange buffer before it is rewritten
      cl_line_fft<M, PX>(u, xb, lane, sx, lx, wx, tw);
      if (rowx)
#pragma unroll
        for (int q = 0; q < S::QX; ++q) {
          const int k = sx + PX * q;
          cl_store(cl_map(bcol + cl_bcol_off<M, PX, PY>(k, yx, jjx), cl_owner(k)), u[q]);
        }
      cl_sync();
    }
  }

  // F2 / I2MF2 y lines from Bcol (rows y < Ny, zero padded), bins stored.
  {
    float2 w[LaneShape<M, PY>::U][PY];
    lane_twiddles<M, PY>(w, tw_full, sy);
    float2 v[S::QY];
#pragma unroll
    for (int q = 0; q < S::QY; ++q) {
      const int y = sy + PY * q;
      v[q] = (colL < S::CPC && y < ny) ? bcol[cl_bcol_off<M, PX, PY>(kx, y, jjy)] : zero;
    }
    cl_line_fft<M, PY>(v, xb, lane, sy, ly, w, tw);
    if (acty) {
      float2 *dst = static_cast<float2 *>(p.out) + (long long)kx * bins_row + (long long)r * b + j0 + jjy;
#pragma unroll
      for (int q = 0; q < S::QY; ++q) dst[(long long)(sy + PY * q) * M * bins_row] = v[q];
    }
  }
}

template <int M, int PX, int PY, int MODE>
size_t cl_smem() {
  using S = ClShape<M, PX, PY>;
  return (size_t)(S::XBUF + (MODE != 1 ? S::BCOL : 0) + (MODE != 0 ? S::BROW : 0)) * sizeof(float2);
}

// Whether a cluster of this kernel fits the device (queried once).
template <int M, int PX, int PY, int MODE>
bool cl_fits() {
  static const int ok = [] {
    auto k = lattice_cluster_kernel<M, PX, PY, MODE>;
    const size_t smem = cl_smem<M, PX, PY, MODE>();
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCl, 1, 1);
    cfg.blockDim = dim3(ClShape<M, PX, PY>::NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = kCl;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return n > 0 ? 1 : 0;
  }();
  return ok != 0;
}

template <int M, int PX, int PY, int MODE>
void cl_launch(const LatticeCluster &p, const FftTables &t, cudaStream_t st) {
  if (!cl_fits<M, PX, PY, MODE>()) throw std::runtime_error("lattice cluster transform does not fit the device");
  ClArgs a;
  a.p = p;
  for (int i = 0; i < kRegMaxM; ++i) a.tw.w[i] = i < M ? t.tw32_host[i] : make_float2(0.f, 0.f);
  dim3 grid((unsigned)(((p.b + kClJ - 1) / kClJ) * kCl), (unsigned)p.nr);
  lattice_cluster_kernel<M, PX, PY, MODE>
      <<<grid, ClShape<M, PX, PY>::NT, cl_smem<M, PX, PY, MODE>(), st>>>(a, t.tw32);
}

template <int M, int PX, int PY>
void cl_mode(const LatticeCluster &p, const FftTables &t, cudaStream_t st) {
  switch (p.mode) {
    case 0: cl_launch<M, PX, PY, 0>(p, t, st); break;
    case 1: cl_launch<M, PX, PY, 1>(p, t, st); break;
    default: cl_launch<M, PX, PY, 2>(p, t, st); break;
  }
}

template <int M, int PX, int PY>
bool cl_fits_all() {
  return cl_fits<M, PX, PY, 0>() && cl_fits<M, PX, PY, 1>() && cl_fits<M, PX, PY, 2>();
}

template <int M>
bool cl_dispatch(const LatticeCluster *p, const FftTables *t, cudaStream_t st, int PX, int PY) {
  if (PX == 4 && PY == 4) return p ? (cl_mode<M, 4, 4>(*p, *t, st), true) : cl_fits_all<M, 4, 4>();
  if (PX == 4 && PY == 2) return p ? (cl_mode<M, 4, 2>(*p, *t, st), true) : cl_fits_all<M, 4, 2>();
  // (The lane rule never gives PX = PY = 2: y lines number at least twice
  // the x lines, so two lanes on x come with one on y.)
  return false;
}

}  // namespace

bool lattice_cluster_supported(int Mx, int My, int nx, int ny, int PX, int PY) {
  if (Mx != My || nx < 1 || ny < 1 || nx > Mx || 2 * ny - 1 > My) return false;
  switch (Mx) {
    case 32: return cl_dispatch<32>(nullptr, nullptr, 0, PX, PY);
    case 48: return cl_dispatch<48>(nullptr, nullptr, 0, PX, PY);
    case 64: return cl_dispatch<64>(nullptr, nullptr, 0, PX, PY);
    default: return false;
  }
}

void launch_lattice_cluster(const LatticeCluster &p, const FftTables &fx, const FftTables &fy, cudaStream_t st) {
  if (p.nr <= 0 || p.b <= 0) return;
  if (fx.plan.M != fy.plan.M) throw std::runtime_error("lattice cluster transform: square grids only");
  bool ok = false;
  switch (fx.plan.M) {
    case 32: ok = cl_dispatch<32>(&p, &fx, st, p.PX, p.PY); break;
    case 48: ok = cl_dispatch<48>(&p, &fx, st, p.PX, p.PY); break;
    case 64: ok = cl_dispatch<64>(&p, &fx, st, p.PX, p.PY); break;
    default: break;
  }
  if (!ok) throw std::runtime_error("lattice cluster transform: unsupported grid or lane split");
}

}  // namespace moma
