// Argument checks of moma_matvec_noalloc that need no CUDA call: the
// caller's pointers are classified on the host (device memory or not, and
// which device) and handed in as plain integers, so that these rules compile
// and run without a GPU (tests/native/noalloc_check.cpp).
#pragma once
#include <stddef.h>

#include <string>

namespace moma {

// Where one buffer lives: is_device = 1 for device (or managed) memory,
// device = the CUDA device index that owns it (ignored for host memory).
struct PtrWhere {
  int is_device = 0;
  int device = -1;
};

// Bytes of fixed scratch one product needs: the x-pass lattice buffer
// [nrhs][Ny][Mx][b] and the two bin-vector buffers [B][nrhs][b], each
// rounded up to 256 bytes.  esz = bytes per complex value (8 or 16).
inline size_t noalloc_scratch_need(long long nrhs, long long ny, long long mx, long long B, long long b,
                                   size_t esz) {
  auto a256 = [](size_t n) { return (n + 255) & ~size_t(255); };
  return a256((size_t)nrhs * ny * mx * b * esz) + 2 * a256((size_t)B * nrhs * b * esz);
}

// Returns an empty string when the call may proceed, else the reason
// (reported as MOMA_ERR_ARG).  array_device = the device the handle was
// created on; its stream, stored bins and tables live there, so x, y and
// the scratch must be on that device too.
inline std::string noalloc_check(int array_device, PtrWhere x, PtrWhere y, size_t need, size_t cap) {
  if (!x.is_device || !y.is_device) return "x and y must be device memory";
  if (x.device != array_device || y.device != array_device)
    return "x and y must be on the array's device " + std::to_string(array_device) + " (x on " +
           std::to_string(x.device) + ", y on " + std::to_string(y.device) + ")";
  if (need > cap)
    return "moma_matvec_noalloc needs " + std::to_string(need) + " bytes of scratch; the fixed maximum is " +
           std::to_string(cap) + " (use fewer RHS per call)";
  return std::string();
}

}  // namespace moma
