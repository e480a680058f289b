// common.cuh -- lattice extent, field layout, indexing and small helpers.
#pragma once
#include <cstdint>

namespace nlc {

struct Dims {
  int nx, ny, nz;
  int64_t n;  // nx * ny * nz
};

// Ghost layers of the stencil fields (Q and u).  These fields are stored
// padded, with periodic images of the interior in a 2-cell ring around it in
// each lattice direction, so that every halo tile the kernels need is one
// plain rectangular box (loaded by TMA) and no wrap-around arithmetic is
// needed when reading them.  The interior x = 0 sits at padded column XOFF;
// XOFF = 4 keeps every tile's box start (x0 - 4) 16-byte aligned.
constexpr int GHOST = 2;
constexpr int XOFF = 4;

struct Layout {
  int nxp, nyp, nzp;  // padded extents
  int zoff;           // GHOST on 3D lattices, 0 on a single plane (D2Q9)
  int64_t plane;      // nxp * nyp
  int64_t comp;       // nxp * nyp * nzp
};

inline Layout make_layout(const Dims& d, bool three_d) {
  Layout L;
  L.nxp = ((d.nx + XOFF + GHOST) + 3) / 4 * 4;
  L.nyp = d.ny + 2 * GHOST;
  L.nzp = three_d ? d.nz + 2 * GHOST : 1;
  L.zoff = three_d ? GHOST : 0;
  L.plane = (int64_t)L.nxp * L.nyp;
  L.comp = L.plane * L.nzp;
  return L;
}

// A padded multi-component field; at(k, x, y, z) with x, y, z in interior
// coordinates, valid for -GHOST <= x < nx + GHOST (and likewise y, z).
template <class T>
struct Field {
  T* base;  // start of the allocation
  Layout L;
  __host__ __device__ int64_t off(int k, int x, int y, int z) const {
    return (int64_t)k * L.comp + (int64_t)(z + L.zoff) * L.plane +
           (int64_t)(y + GHOST) * L.nxp + (x + XOFF);
  }
  __device__ T& at(int k, int x, int y, int z) const { return base[off(k, x, y, z)]; }
};

__device__ __forceinline__ int wrap_inc(int v, int n) { return v + 1 == n ? 0 : v + 1; }
__device__ __forceinline__ int wrap_dec(int v, int n) { return v == 0 ? n - 1 : v - 1; }
// v + d for |d| <= n, periodic
__device__ __forceinline__ int wrap_add(int v, int d, int n) {
  int r = v + d;
  r = r >= n ? r - n : r;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ int64_t cell_of(const Dims& d, int x, int y, int z) {
  return (int64_t)x + (int64_t)d.nx * ((int64_t)y + (int64_t)d.ny * z);
}

// Images of coordinate v (0 <= v < n) in the ghost ring: bit (k + GHOST) of
// the result is set when v + k n lies in [-GHOST, n + GHOST), k != 0.
__device__ __forceinline__ unsigned image_mask(int v, int n) {
  unsigned m = 0;
  if (n > 2 * GHOST) {  // at most one image on each side
    if (v < GHOST) m |= 1u << (GHOST + 1);
    if (v >= n - GHOST) m |= 1u << (GHOST - 1);
    return m;
  }
  for (int k = -GHOST; k <= GHOST; k++) {
    const int vi = v + k * n;
    if (k != 0 && vi >= -GHOST && vi < n + GHOST) m |= 1u << (k + GHOST);
  }
  return m;
}

// Stores NC component values of cell (x, y, z) of a padded field, and every
// periodic image of the cell that falls in the ghost ring.  Only cells within
// GHOST of a face have images; lattices thinner than the ring get several.
template <class T, int NC, int DIM>
__device__ __forceinline__ void store_with_images(const Field<T>& F, const Dims& d,
                                                  int x, int y, int z,
                                                  const T v[NC]) {
  const int64_t o = F.off(0, x, y, z);
#pragma unroll
  for (int k = 0; k < NC; k++) F.base[o + k * F.L.comp] = v[k];
  const bool inner = x >= GHOST && x < d.nx - GHOST && y >= GHOST &&
                     y < d.ny - GHOST &&
                     (DIM == 2 || (z >= GHOST && z < d.nz - GHOST));
  if (inner) return;
  const unsigned mx = image_mask(x, d.nx), my = image_mask(y, d.ny);
  const unsigned mz = DIM == 3 ? image_mask(z, d.nz) : 0u;
  if ((mx | my | mz) == 0) return;
  // offsets per axis: 0 plus every image offset
  const unsigned ax = mx | (1u << GHOST), ay = my | (1u << GHOST);
  const unsigned az = mz | (1u << GHOST);
  for (int kz = -GHOST; kz <= GHOST; kz++) {
    if (!(az >> (kz + GHOST) & 1u)) continue;
    for (int ky = -GHOST; ky <= GHOST; ky++) {
      if (!(ay >> (ky + GHOST) & 1u)) continue;
      for (int kx = -GHOST; kx <= GHOST; kx++) {
        if (!(ax >> (kx + GHOST) & 1u)) continue;
        if (kx == 0 && ky == 0 && kz == 0) continue;
        const int xi = x + kx * d.nx, yi = y + ky * d.ny, zi = z + kz * d.nz;
#pragma unroll
        for (int k = 0; k < NC; k++) F.at(k, xi, yi, zi) = v[k];
      }
    }
  }
}

// Stores NC component values of cell (x, y, z) of a padded field whose
// periodic images the caller knows to lie outside the ghost ring (a cell at
// least GHOST away from every face).
template <class T, int NC>
__device__ __forceinline__ void store_interior(const Field<T>& F, int x, int y, int z,
                                               const T v[NC]) {
  T* p = F.base + F.off(0, x, y, z);
#pragma unroll
  for (int k = 0; k < NC; k++) p[k * F.L.comp] = v[k];
}

// fixed-order FP64 block sum (blockDim.x a multiple of 32, <= 1024);
// every thread returns the total
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  const int nw = (int)(blockDim.x >> 5);
  for (int k = 0; k < nw; k++) t += sh[k];
  return t;
}

__device__ __forceinline__ double block_max(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  const int nw = (int)(blockDim.x >> 5);
  for (int k = 0; k < nw; k++) t = fmax(t, sh[k]);
  return t;
}

}  // namespace nlc
