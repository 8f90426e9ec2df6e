// Host-only driver of the argument rules of moma_matvec_noalloc
// (csrc/noalloc_check.h): reads one case per line,
//   array_device x_is_device x_device y_is_device y_device nrhs ny mx B b esz cap
// and prints "OK" or the rejection message, plus the scratch bytes needed.
#include <cstdio>
#include <iostream>
#include <string>

#include "noalloc_check.h"

int main() {
  int adev;
  moma::PtrWhere x, y;
  long long nrhs, ny, mx, B, b;
  size_t esz, cap;
  while (std::cin >> adev >> x.is_device >> x.device >> y.is_device >> y.device >> nrhs >> ny >> mx >> B >> b >> esz >>
         cap) {
    const size_t need = moma::noalloc_scratch_need(nrhs, ny, mx, B, b, esz);
    const std::string why = moma::noalloc_check(adev, x, y, need, cap);
    std::printf("%zu %s\n", need, why.empty() ? "OK" : why.c_str());
  }
  return 0;
}
