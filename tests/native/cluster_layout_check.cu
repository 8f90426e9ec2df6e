// Host check of the cluster lattice transforms' work split and hand-over
// layout (csrc/lattice_cluster.cuh), driven the way lattice_cluster.cu
// drives it: every thread of the eight CTAs of a cluster takes its x line
// and y line from cl_line, sends its values to cl_owner at cl_bcol_off /
// cl_brow_off, and reads back the same layout.  For every instantiated
// (M, PX, PY), every lattice height Ny <= (M + 1) / 2 and each transform
// (F2, I2, I2MF2) it checks that every store stays inside the owner's
// buffer, no location is written twice, and every location a line reads
// was written.  Prints "ok <cases>" or the first failure.
#include <cstdio>
#include <set>
#include <utility>

#include "lattice_cluster.cuh"

using namespace moma;

template <int M, int PX, int PY>
static bool check(int ny, int mode) {
  using S = ClShape<M, PX, PY>;
  std::set<std::pair<int, int>> bcol, brow;  // (owner CTA, offset) written
  auto fail = [&](const char *what, int c, int tid, int off) {
    std::printf("FAIL M=%d PX=%d PY=%d ny=%d mode=%d: %s (cta %d, thread %d, offset %d)\n", M, PX, PY, ny, mode,
                what, c, tid, off);
    return false;
  };
  for (int c = 0; c < kCl; ++c)
    for (int tid = 0; tid < S::NT; ++tid) {
      const ClLine tx = cl_line<PX>(c, tid), ty = cl_line<PY>(c, tid);
      const bool rowx = tx.loc < S::RPC && tx.g < ny;
      // y lines of I2 / I2MF2: rows y < Ny to their owners' Brow.
      if (mode != 0 && ty.loc < S::CPC)
        for (int q = 0; q < S::QY; ++q) {
          const int y = ty.s + PY * q;
          if (y >= ny) continue;
          const int off = cl_brow_off<M>(y, ty.g, ty.jj);
          if (off < 0 || off >= S::BROW) return fail("Brow store out of bounds", c, tid, off);
          if (!brow.insert({cl_owner(y), off}).second) return fail("Brow location written twice", c, tid, off);
        }
      // x lines of F2 / I2MF2: every column kx to its owner's Bcol.
      if (mode != 1 && rowx)
        for (int q = 0; q < S::QX; ++q) {
          const int k = tx.s + PX * q;
          const int off = cl_bcol_off<M, PX, PY>(k, tx.g, tx.jj);
          if (off < 0 || off >= S::BCOL) return fail("Bcol store out of bounds", c, tid, off);
          if (!bcol.insert({cl_owner(k), off}).second) return fail("Bcol location written twice", c, tid, off);
        }
    }
  for (int c = 0; c < kCl; ++c)
    for (int tid = 0; tid < S::NT; ++tid) {
      const ClLine tx = cl_line<PX>(c, tid), ty = cl_line<PY>(c, tid);
      const bool rowx = tx.loc < S::RPC && tx.g < ny;
      if (rowx && tx.g % kCl != c) return fail("x line outside its owner's rows", c, tid, tx.g);
      if (ty.loc < S::CPC && ty.g % kCl != c) return fail("y line outside its owner's columns", c, tid, ty.g);
      // x lines of I2 / I2MF2 read their row's M columns from Brow.
      if (mode != 0 && rowx)
        for (int q = 0; q < S::QX; ++q) {
          const int off = cl_brow_off<M>(tx.g, tx.s + PX * q, tx.jj);
          if (!brow.count({c, off})) return fail("Brow read of an unwritten location", c, tid, off);
        }
      // y lines of F2 / I2MF2 read their column's rows y < Ny from Bcol.
      if (mode != 1 && ty.loc < S::CPC)
        for (int q = 0; q < S::QY; ++q) {
          const int y = ty.s + PY * q;
          if (y >= ny) continue;
          const int off = cl_bcol_off<M, PX, PY>(ty.g, y, ty.jj);
          if (!bcol.count({c, off})) return fail("Bcol read of an unwritten location", c, tid, off);
        }
    }
  // Every line of the grid exists: Ny x 8 x lines, M x 8 y lines per cluster.
  if (mode != 1 && (int)bcol.size() != ny * kClJ * M) return fail("Bcol entries missing", -1, -1, (int)bcol.size());
  if (mode != 0 && (int)brow.size() != ny * kClJ * M) return fail("Brow entries missing", -1, -1, (int)brow.size());
  return true;
}

template <int M, int PX, int PY>
static int check_all() {
  int n = 0;
  for (int ny = 1; ny <= ClShape<M, PX, PY>::YMAX; ++ny)
    for (int mode = 0; mode < 3; ++mode) {
      if (!check<M, PX, PY>(ny, mode)) return -1;
      ++n;
    }
  return n;
}

int main() {
  int total = 0;
  for (int n : {check_all<32, 4, 4>(), check_all<32, 4, 2>(), check_all<48, 4, 4>(), check_all<48, 4, 2>(),
                check_all<64, 4, 4>(), check_all<64, 4, 2>()}) {
    if (n < 0) return 1;
    total += n;
  }
  std::printf("ok %d\n", total);
  return 0;
}
