// chunks.h -- how the fused step kernels split each 32 x 8 column of a
// three-dimensional lattice along z among thread blocks.  Host-only C++,
// header-only so tests can build it with a plain C++ compiler.
#pragma once
#include <vector>

namespace nlc {

// z-chunk boundaries b[0] = 0 < b[1] < ... = nz of every column of a
// lattice: chunks of tz planes; with taper, chunks of tz planes until at
// most 2 tz remain, then chunks that halve down to about 8 planes.  Blocks
// run in tile-list order, so a tapered list ends with short blocks and the
// last wave over the SMs leaves less of the GPU idle.
inline std::vector<int> chunk_bounds(int nz, int tz, bool taper) {
  if (tz < 1) tz = 1;
  std::vector<int> b = {0};
  int z = 0;
  if (!taper) {
    while (z < nz) {
      z = z + tz < nz ? z + tz : nz;
      b.push_back(z);
    }
    return b;
  }
  while (nz - z > 2 * tz) {
    z += tz;
    b.push_back(z);
  }
  int r = nz - z;
  while (r > 0) {
    int c = r > 8 ? (r + 1) / 2 : r;
    if (r - c > 0 && r - c < 4) c = r;
    z += c;
    r -= c;
    b.push_back(z);
  }
  return b;
}

}  // namespace nlc
