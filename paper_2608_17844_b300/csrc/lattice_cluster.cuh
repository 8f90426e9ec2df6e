// Work split and hand-over layout of the cluster lattice transforms
// (lattice_cluster.cu), as host/device functions so that a host program can
// check them: which thread owns which x line (lattice row, basis index) and
// y line (grid column, basis index) in CTA c of a cluster, which CTA owns a
// column or a row, and where a hand-over value lands in the owner's shared
// memory.
//   columns kx of the M x M grid: CTA kx % kCl, local column kx / kCl;
//   lattice rows y < Ny:           CTA y % kCl,  local row y / kCl;
//   Bcol[col][y][jj]  (row stride kColJ) receives the x lines' outputs,
//   Brow[row][kx][jj] (column stride kRowJ) the y lines' outputs.
#pragma once

#include "fftreg.cuh"

namespace moma {

constexpr int kCl = 8;           // CTAs per cluster
constexpr int kClJ = 8;          // basis indices per cluster
constexpr int kColJ = kClJ + 4;  // Bcol: stride of consecutive rows of a column
constexpr int kRowJ = kClJ + 1;  // Brow: stride of consecutive columns of a row

template <int M, int PX, int PY>
struct ClShape {
  static constexpr int YMAX = (M + 1) / 2;            // lattice rows at most (M >= 2 Ny - 1)
  static constexpr int RPC = (YMAX + kCl - 1) / kCl;  // rows per CTA at most
  static constexpr int CPC = M / kCl;                 // columns per CTA
  static constexpr int NXT = RPC * kClJ * PX, NYT = CPC * kClJ * PY;
  static constexpr int NT = ((NXT > NYT ? NXT : NYT) + 31) / 32 * 32;
  static constexpr int QX = M / PX, QY = M / PY, QMAX = QX > QY ? QX : QY;
  static constexpr int XBUF = (NT / 32) * QMAX * kLaneLd;  // per-warp exchange buffers
  static constexpr int BCOL = CPC * YMAX * kColJ;
  static constexpr int BROW = RPC * M * kRowJ;
  static_assert(M % kCl == 0, "grid columns are dealt to the cluster's CTAs in turn");
};

// A thread's line: lane s of the line's P lanes, line l of its warp, the
// CTA-local line index (loc: local row or column), basis index jj, and the
// global row y or column kx it stands for.
struct ClLine {
  int s, l, loc, jj, g;
};
template <int P>
MOMA_HD ClLine cl_line(int c, int tid) {
  const int lane = tid & 31, warp = tid >> 5;
  ClLine t;
  t.s = lane % P;
  t.l = lane / P;
  const int ln = warp * (32 / P) + t.l;
  t.loc = ln / kClJ;
  t.jj = ln % kClJ;
  t.g = c + kCl * t.loc;
  return t;
}

// Owner CTA and shared-memory offsets of the hand-overs.
MOMA_HD int cl_owner(int idx) { return idx % kCl; }
template <int M, int PX, int PY>
MOMA_HD int cl_bcol_off(int kx, int y, int jj) {
  return (kx / kCl) * (ClShape<M, PX, PY>::YMAX * kColJ) + y * kColJ + jj;
}
template <int M>
MOMA_HD int cl_brow_off(int y, int kx, int jj) {
  return (y / kCl) * (M * kRowJ) + kx * kRowJ + jj;
}

}  // namespace moma
