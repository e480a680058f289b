// common.cuh -- lattice extent, indexing and small device helpers.
#pragma once
#include <cstdint>

namespace nlc {

struct Dims {
  int nx, ny, nz;
  int64_t n;  // nx * ny * nz
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
