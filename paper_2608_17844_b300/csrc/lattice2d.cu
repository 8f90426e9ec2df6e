// Two-dimensional lattice transforms of the MLFFT product (Eq. 2:
// F^[2] = F_{Ny} (x) (F_{Nx} (x) I_b)) in one launch each, instead of one
// launch per lattice axis.
//
// One CTA owns J consecutive basis indices j0 .. j0+J-1 of one right-hand
// side r and holds their whole My x Mx circulant grid in shared memory,
// element (row p, column q, basis jj) at A[p * RS + q * J + jj].  The row
// stride RS = roundup(Mx J, 16) + J makes both passes conflict-free: in the
// x pass consecutive threads own consecutive lines (row, jj), which land in
// distinct banks because RS = J (mod 16); in the y pass consecutive lines
// (column, jj) are consecutive words.  The 1D stages are those of fft.cuh
// (G threads per line, lines fastest, a barrier between stages).
//
// Three transforms (all with zero padding from the Ny x Nx lattice to the
// My x Mx circulant grid, Eq. 3).  Every x pass runs on rows held in natural
// order (the conflict-free case above); the digit reversals of the 1D
// stages are absorbed by row-level scatters / gathers, plus one scatter or
// gather of the Ny x Nx lattice points along x:
//   F2     lattice [nr][Ny][Nx][b] (per-RHS stride ldv) -> bins [My][Mx][nr][b]:
//          points scattered to digit-reversed columns, DIT along x on the Ny
//          occupied rows (natural output), DIF along y on every column, rows
//          gathered from their digit-reversed positions on the way out.
//   I2     bins -> lattice, the inverse as conj . DFT . conj / (Mx My): rows
//          scattered to digit-reversed positions on the way in, DIT along y,
//          DIF along x on the Ny rows that survive the truncation, the
//          Ny x Nx outputs gathered from digit-reversed columns.
//   I2MF2  bins -> bins: that inverse, the lattice mask (Sec. III-A: Z^H
//          acts on M Z x, M the restriction to the lattice) and the forward
//          transform of the masked grid (DIT along x, DIF along y), between
//          the Z and Z^H legs of the normal operator.
#include <algorithm>
#include <stdexcept>
#include <type_traits>

#include "internal.h"

namespace moma {

namespace {

struct L2Args {
  FftPlan px, py;
  const void *in;
  void *out;
  int nx, ny, b, nr, rs;
  long long ldv;
  const int *live;
};

template <typename C>
MOMA_DEV C cconj_(C v) {
  v.y = -v.y;
  return v;
}

// One 1D pass over `nl` lines: line L's points at base(L) + m * ld.  G
// threads per line, lines fastest (thread t: line t % nl, sub-thread t / nl).
template <bool DIT, typename C, typename Base>
MOMA_DEV void lines_pass(int nl, int ld, const FftPlan &pl, const C *tw, Base base, int t, int nt) {
  if (pl.nst == 0 || nl <= 0) return;
  int gmax = pl.M / 2;
  if (gmax < 1) gmax = 1;
  int G = 1;
  while (G * 2 <= gmax && nl * G * 2 <= nt) G *= 2;
  for (int si = 0; si < pl.nst; ++si) {
    const int s = DIT ? pl.nst - 1 - si : si;
    if (G > 1) {
      if (t < nl * G) {
        const int L = t % nl, g = t / nl;
        if (DIT) dit_stage(base(L), ld, pl, tw, s, g, G);
        else dif_stage(base(L), ld, pl, tw, s, g, G);
      }
    } else {
      for (int L = t; L < nl; L += nt) {
        if (DIT) dit_stage(base(L), ld, pl, tw, s, 0, 1);
        else dif_stage(base(L), ld, pl, tw, s, 0, 1);
      }
    }
    __syncthreads();
  }
}

template <typename R, int J, int MODE>
__global__ void __launch_bounds__(512) lattice2d_kernel(L2Args A, const typename Cplx<R>::T *__restrict__ twx_g,
                                                        const typename Cplx<R>::T *__restrict__ twy_g,
                                                        const int *__restrict__ posx_g,
                                                        const int *__restrict__ posy_g) {
  using C = typename Cplx<R>::T;
  extern __shared__ __align__(16) unsigned char sm[];
  if (A.live && *A.live == 0) return;
  const int Mx = A.px.M, My = A.py.M, RS = A.rs, nx = A.nx, ny = A.ny, b = A.b;
  C *twx = reinterpret_cast<C *>(sm);
  C *twy = twx + Mx;
  int *posx = reinterpret_cast<int *>(twy + My);
  int *posy = posx + Mx;
  const size_t head = (((size_t)(Mx + My) * sizeof(C) + (size_t)(Mx + My) * sizeof(int)) + 15) & ~size_t(15);
  C *S = reinterpret_cast<C *>(sm + head);
  const int t = threadIdx.x, nt = blockDim.x;
  const int r = blockIdx.y, j0 = blockIdx.x * J;
  for (int i = t; i < Mx; i += nt) {
    twx[i] = twx_g[i];
    posx[i] = posx_g[i];
  }
  for (int i = t; i < My; i += nt) {
    twy[i] = twy_g[i];
    posy[i] = posy_g[i];
  }
  __syncthreads();  // the tables are read by every thread from here on
  const C zero = mk(R(0), R(0));
  const long long bins_row = (long long)A.nr * b;  // elements between consecutive bins
  const C *in = reinterpret_cast<const C *>(A.in);
  C *out = reinterpret_cast<C *>(A.out);
  const R inv_m = R(1) / R(Mx * My);

  if (MODE == 0) {
    // F2: zero the grid, scatter the lattice points to digit-reversed columns.
    for (int i = t; i < My * RS; i += nt) S[i] = zero;
    __syncthreads();
    const C *src = in + (long long)r * A.ldv;
    for (int i = t; i < ny * nx; i += nt) {
      const int y = i / nx, x = i - y * nx;
      const long long g = (long long)i * b + j0;
      C *d = S + y * RS + posx[x] * J;
#pragma unroll
      for (int jj = 0; jj < J; ++jj)
        if (j0 + jj < b) d[jj] = src[g + jj];
    }
  } else {
    // Inverse transforms: bins conjugated, rows scattered to digit-reversed
    // positions (row ky lands at row posy[ky]).
    for (int i = t; i < My * Mx; i += nt) {
      const int ky = i / Mx, kx = i - ky * Mx;
      const long long g = (long long)i * bins_row + (long long)r * b + j0;
      C *d = S + posy[ky] * RS + kx * J;
#pragma unroll
      for (int jj = 0; jj < J; ++jj) d[jj] = (j0 + jj < b) ? cconj_(in[g + jj]) : zero;
    }
  }
  __syncthreads();
  auto row_line = [&](int L) { return S + (L / J) * RS + (L % J); };  // x-pass line (row L / J, basis L % J)
  auto col_line = [&](int L) { return S + L; };                      // y-pass line (column L / J, basis L % J)

  if (MODE == 0) {
    lines_pass<true>(ny * J, J, A.px, twx, row_line, t, nt);     // natural x out
    lines_pass<false>(Mx * J, RS, A.py, twy, col_line, t, nt);   // bin ky at row posy[ky]
    for (int i = t; i < My * Mx; i += nt) {
      const int ky = i / Mx, kx = i - ky * Mx;
      const long long g = (long long)i * bins_row + (long long)r * b + j0;
      const C *s = S + posy[ky] * RS + kx * J;
#pragma unroll
      for (int jj = 0; jj < J; ++jj)
        if (j0 + jj < b) out[g + jj] = s[jj];
    }
    return;
  }

  // Inverse: y pass (DIT: natural rows out) on every column, x pass (DIF) on
  // the rows y < Ny; value (y, x) then sits at row y, column posx[x].
  lines_pass<true>(Mx * J, RS, A.py, twy, col_line, t, nt);
  lines_pass<false>(ny * J, J, A.px, twx, row_line, t, nt);

  if (MODE == 1) {
    C *dst = out + (long long)r * A.ldv;
    for (int i = t; i < ny * nx; i += nt) {
      const int y = i / nx, x = i - y * nx;
      const long long g = (long long)i * b + j0;
      const C *s = S + y * RS + posx[x] * J;
#pragma unroll
      for (int jj = 0; jj < J; ++jj)
        if (j0 + jj < b) dst[g + jj] = cscale(cconj_(s[jj]), inv_m);
    }
    return;
  }

  // I2MF2: finish the inverse and apply the mask in place (keep x < Nx on the
  // rows y < Ny, zero the other rows), then transform forward again: DIT
  // along x (digit-reversed columns in, natural out) on the Ny rows, DIF
  // along y on every column; rows gathered from digit-reversed positions.
  for (int i = t; i < My * Mx; i += nt) {
    const int y = i / Mx, x = i - y * Mx;
    C *s = S + y * RS + posx[x] * J;
    const bool keep = y < ny && x < nx;
#pragma unroll
    for (int jj = 0; jj < J; ++jj) s[jj] = keep ? cscale(cconj_(s[jj]), inv_m) : zero;
  }
  __syncthreads();
  lines_pass<true>(ny * J, J, A.px, twx, row_line, t, nt);
  lines_pass<false>(Mx * J, RS, A.py, twy, col_line, t, nt);
  for (int i = t; i < My * Mx; i += nt) {
    const long long g = (long long)i * bins_row + (long long)r * b + j0;
    const int ky = i / Mx, kx = i - ky * Mx;
    const C *s = S + posy[ky] * RS + kx * J;
#pragma unroll
    for (int jj = 0; jj < J; ++jj)
      if (j0 + jj < b) out[g + jj] = s[jj];
  }
}

int row_stride(int Mx, int J) { return (Mx * J + 15) / 16 * 16 + J; }

size_t smem_bytes(int Mx, int My, int J, size_t csz) {
  const size_t head = (((size_t)(Mx + My) * csz + (size_t)(Mx + My) * sizeof(int)) + 15) & ~size_t(15);
  return head + (size_t)My * row_stride(Mx, J) * csz;
}

constexpr size_t kMaxSmem = 227 * 1024;

template <typename R, int J, int MODE>
void launch_typed(const Lattice2D &p, const FftTables &fx, const FftTables &fy, int threads, cudaStream_t st) {
  using C = typename Cplx<R>::T;
  const size_t smem = smem_bytes(fx.plan.M, fy.plan.M, J, sizeof(C));
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(lattice2d_kernel<R, J, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    configured = true;
  }
  L2Args a;
  a.px = fx.plan;
  a.py = fy.plan;
  a.in = p.in;
  a.out = p.out;
  a.nx = p.nx;
  a.ny = p.ny;
  a.b = p.b;
  a.nr = p.nr;
  a.rs = row_stride(fx.plan.M, J);
  a.ldv = p.ldv;
  a.live = p.live;
  const C *twx, *twy;
  if constexpr (std::is_same<R, double>::value) {
    twx = fx.tw64;
    twy = fy.tw64;
  } else {
    twx = fx.tw32;
    twy = fy.tw32;
  }
  dim3 grid((p.b + J - 1) / J, p.nr);
  lattice2d_kernel<R, J, MODE><<<grid, threads, smem, st>>>(a, twx, twy, fx.pos, fy.pos);
}

template <typename R, int J>
void launch_mode(const Lattice2D &p, const FftTables &fx, const FftTables &fy, int threads, cudaStream_t st) {
  switch (p.mode) {
    case 0: launch_typed<R, J, 0>(p, fx, fy, threads, st); break;
    case 1: launch_typed<R, J, 1>(p, fx, fy, threads, st); break;
    default: launch_typed<R, J, 2>(p, fx, fy, threads, st); break;
  }
}

}  // namespace

template <typename R>
bool lattice2d_fits(int Mx, int My, int J) {
  return smem_bytes(Mx, My, J, sizeof(typename Cplx<R>::T)) <= kMaxSmem;
}

template <typename R>
void launch_lattice2d(const Lattice2D &p, const FftTables &fx, const FftTables &fy, cudaStream_t st) {
  if (p.nr <= 0 || p.b <= 0) return;
  int J = p.J;
  if (J <= 0) {
    // Heuristic: enough CTAs to cover the SMs, the widest basis group that
    // still gives them.
    J = 1;
    for (int j : {2, 4})
      if ((long long)((p.b + j - 1) / j) * p.nr >= 148 && lattice2d_fits<R>(fx.plan.M, fy.plan.M, j)) J = j;
  }
  if (!lattice2d_fits<R>(fx.plan.M, fy.plan.M, J)) throw std::runtime_error("lattice2d: grid too large for shared memory");
  const int threads = p.threads > 0 ? p.threads : 256;
  switch (J) {
    case 1: launch_mode<R, 1>(p, fx, fy, threads, st); break;
    case 2: launch_mode<R, 2>(p, fx, fy, threads, st); break;
    case 4: launch_mode<R, 4>(p, fx, fy, threads, st); break;
    default: throw std::runtime_error("lattice2d: J must be 1, 2 or 4");
  }
}

template bool lattice2d_fits<float>(int, int, int);
template bool lattice2d_fits<double>(int, int, int);
template void launch_lattice2d<float>(const Lattice2D &, const FftTables &, const FftTables &, cudaStream_t);
template void launch_lattice2d<double>(const Lattice2D &, const FftTables &, const FftTables &, cudaStream_t);

}  // namespace moma
