// step_unfused.cuh -- one time step as four one-cell-per-thread kernels.
//
//   1. stress   : Q^n -> Pi (Eq. 3 for H, Eq. 5 without P0)
//   2. lb       : F = div Pi, pull-stream, rho/u (Eq. 6), BGK + source,
//                 store post-collision deviations g* and u^n
//   3. predict  : R1 = R(Q^n; u^n), Q^P = Q^n + R1          (Sec. 1.2.2, 1-2)
//   4. correct  : R2 = R(Q^P; u^n), Q^{n+1} = Q^n + (R1+R2)/2 (steps 3-5)
//
// Populations are stored as deviations g_i = f_i - w_i rho0 in a pull
// layout: the buffer holds the post-collision values at the cell where the
// collision happened, and the pre-collision f_i(x, t) is
// w_i rho0 + g_i(x - c_i).  Every intermediate goes through global memory;
// the fused schedule (step_fused.cuh) computes the same step with two tiled
// kernels.
#pragma once
#include "common.cuh"
#include "lattice.cuh"
#include "physics.cuh"

namespace nlc {

template <class T, int DIM>
__device__ __forceinline__ void load_q(const T* __restrict__ Q, int64_t n,
                                       int64_t c, T q[5]) {
#pragma unroll
  for (int k = 0; k < 5; k++) q[k] = Q[k * n + c];
}

// central first derivatives and the 2d+1-point Laplacian of the five
// components at (x, y, z), from global memory
template <class T, int DIM>
__device__ __forceinline__ void q_stencil(const T* __restrict__ Q,
                                          const Dims& d, int x, int y, int z,
                                          T q[5], T dq[3][5], T lap[5]) {
  const int64_t c = cell_of(d, x, y, z);
  const int64_t cxp = cell_of(d, wrap_inc(x, d.nx), y, z);
  const int64_t cxm = cell_of(d, wrap_dec(x, d.nx), y, z);
  const int64_t cyp = cell_of(d, x, wrap_inc(y, d.ny), z);
  const int64_t cym = cell_of(d, x, wrap_dec(y, d.ny), z);
  int64_t czp = c, czm = c;
  if (DIM == 3) {
    czp = cell_of(d, x, y, wrap_inc(z, d.nz));
    czm = cell_of(d, x, y, wrap_dec(z, d.nz));
  }
#pragma unroll
  for (int k = 0; k < 5; k++) {
    const T v = Q[k * d.n + c];
    const T xp = Q[k * d.n + cxp], xm = Q[k * d.n + cxm];
    const T yp = Q[k * d.n + cyp], ym = Q[k * d.n + cym];
    q[k] = v;
    dq[0][k] = (xp - xm) / T(2);
    dq[1][k] = (yp - ym) / T(2);
    T l = (xp + xm - T(2) * v) + (yp + ym - T(2) * v);
    if (DIM == 3) {
      const T zp = Q[k * d.n + czp], zm = Q[k * d.n + czm];
      dq[2][k] = (zp - zm) / T(2);
      l += zp + zm - T(2) * v;
    } else {
      dq[2][k] = T(0);
    }
    lap[k] = l;
  }
}

// velocity gradient G[a][b] = d_b u_a by central differences of the stored
// u^n (DIM planes)
template <class T, int DIM>
__device__ __forceinline__ void u_stencil(const T* __restrict__ U,
                                          const Dims& d, int x, int y, int z,
                                          T u[3], T G[3][3]) {
  const int64_t c = cell_of(d, x, y, z);
  const int64_t nb[3][2] = {
      {cell_of(d, wrap_inc(x, d.nx), y, z), cell_of(d, wrap_dec(x, d.nx), y, z)},
      {cell_of(d, x, wrap_inc(y, d.ny), z), cell_of(d, x, wrap_dec(y, d.ny), z)},
      {DIM == 3 ? cell_of(d, x, y, wrap_inc(z, d.nz)) : c,
       DIM == 3 ? cell_of(d, x, y, wrap_dec(z, d.nz)) : c}};
#pragma unroll
  for (int a = 0; a < 3; a++) {
    u[a] = a < DIM ? U[a * d.n + c] : T(0);
#pragma unroll
    for (int b = 0; b < 3; b++)
      G[a][b] = (a < DIM && b < DIM)
                    ? (U[a * d.n + nb[b][0]] - U[a * d.n + nb[b][1]]) / T(2)
                    : T(0);
  }
}

__device__ __forceinline__ bool decode(const Dims& d, int64_t idx, int& x,
                                       int& y, int& z) {
  if (idx >= d.n) return false;
  x = (int)(idx % d.nx);
  const int64_t r = idx / d.nx;
  y = (int)(r % d.ny);
  z = (int)(r / d.ny);
  return true;
}

template <class Lat, class T>
__global__ void __launch_bounds__(256) k_stress(const T* __restrict__ Q,
                                                T* __restrict__ Pi, Dims d,
                                                Par<T> p) {
  constexpr int DIM = Lat::DIM;
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!decode(d, idx, x, y, z)) return;
  T q[5], dq[3][5], lap[5], h[5], P[3][3];
  q_stencil<T, DIM>(Q, d, x, y, z, q, dq, lap);
  molecular_field(q, lap, p, h);
  stress<T, DIM>(q, h, dq, p, P);
#pragma unroll
  for (int a = 0; a < DIM; a++)
#pragma unroll
    for (int b = 0; b < DIM; b++) Pi[(a * DIM + b) * d.n + idx] = P[a][b];
}

// F_a = sum_b [Pi_ab(x + e_b) - Pi_ab(x - e_b)] / 2
template <class T, int DIM>
__device__ __forceinline__ void force_at(const T* __restrict__ Pi,
                                         const Dims& d, int x, int y, int z,
                                         T F[3]) {
  const int64_t nb[3][2] = {
      {cell_of(d, wrap_inc(x, d.nx), y, z), cell_of(d, wrap_dec(x, d.nx), y, z)},
      {cell_of(d, x, wrap_inc(y, d.ny), z), cell_of(d, x, wrap_dec(y, d.ny), z)},
      {DIM == 3 ? cell_of(d, x, y, wrap_inc(z, d.nz)) : 0,
       DIM == 3 ? cell_of(d, x, y, wrap_dec(z, d.nz)) : 0}};
#pragma unroll
  for (int a = 0; a < 3; a++) {
    T s = T(0);
    if (a < DIM) {
#pragma unroll
      for (int b = 0; b < DIM; b++)
        s += (Pi[(a * DIM + b) * d.n + nb[b][0]] -
              Pi[(a * DIM + b) * d.n + nb[b][1]]) / T(2);
    }
    F[a] = s;
  }
}

// pre-collision deviations g_i(x, t) = g*_i(x - c_i) (pull, periodic)
template <class Lat, class T>
__device__ __forceinline__ void pull(const T* __restrict__ gin, const Dims& d,
                                     int x, int y, int z, T g[Lat::Q]) {
#pragma unroll
  for (int i = 0; i < Lat::Q; i++) {
    const int xs = wrap_add(x, -Lat::c(i, 0), d.nx);
    const int ys = wrap_add(y, -Lat::c(i, 1), d.ny);
    const int zs = Lat::DIM == 3 ? wrap_add(z, -Lat::c(i, 2), d.nz) : z;
    g[i] = gin[(int64_t)i * d.n + cell_of(d, xs, ys, zs)];
  }
}

// rho = rho0 + sum g, u = (sum c g + F/2) / rho  (Eq. 6; sum c w rho0 = 0)
template <class Lat, class T>
__device__ __forceinline__ void moments(const T g[Lat::Q], const T F[3],
                                        const Par<T>& p, T& rho, T u[3]) {
  T s = T(0), m[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int i = 0; i < Lat::Q; i++) {
    s += g[i];
#pragma unroll
    for (int a = 0; a < Lat::DIM; a++)
      if (Lat::c(i, a) != 0) m[a] += T(Lat::c(i, a)) * g[i];
  }
  rho = p.rho0 + s;
  const T inv = T(1) / rho;
#pragma unroll
  for (int a = 0; a < 3; a++)
    u[a] = a < Lat::DIM ? (m[a] + F[a] / T(2)) * inv : T(0);
}

template <class Lat, class T>
__global__ void __launch_bounds__(256) k_lb(const T* __restrict__ gin,
                                            T* __restrict__ gout,
                                            const T* __restrict__ Pi,
                                            T* __restrict__ U, Dims d,
                                            Par<T> p) {
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!decode(d, idx, x, y, z)) return;
  T F[3], g[Lat::Q], rho, u[3];
  force_at<T, Lat::DIM>(Pi, d, x, y, z, F);
  pull<Lat, T>(gin, d, x, y, z, g);
  moments<Lat, T>(g, F, p, rho, u);
  collide_bgk<Lat, T>(g, rho, u, F, p);
#pragma unroll
  for (int i = 0; i < Lat::Q; i++) gout[(int64_t)i * d.n + idx] = g[i];
#pragma unroll
  for (int a = 0; a < Lat::DIM; a++) U[a * d.n + idx] = u[a];
}

template <class Lat, class T>
__global__ void __launch_bounds__(256) k_predict(const T* __restrict__ Q,
                                                 const T* __restrict__ U,
                                                 T* __restrict__ QP,
                                                 T* __restrict__ R1, Dims d,
                                                 Par<T> p) {
  constexpr int DIM = Lat::DIM;
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!decode(d, idx, x, y, z)) return;
  T q[5], dq[3][5], lap[5], u[3], G[3][3], r[5];
  q_stencil<T, DIM>(Q, d, x, y, z, q, dq, lap);
  u_stencil<T, DIM>(U, d, x, y, z, u, G);
  be_rhs<T, DIM>(q, dq, lap, u, G, p, r);
#pragma unroll
  for (int k = 0; k < 5; k++) {
    R1[k * d.n + idx] = r[k];
    QP[k * d.n + idx] = q[k] + r[k];
  }
}

template <class Lat, class T>
__global__ void __launch_bounds__(256) k_correct(const T* __restrict__ Q,
                                                 const T* __restrict__ QP,
                                                 const T* __restrict__ R1,
                                                 const T* __restrict__ U,
                                                 T* __restrict__ Qout, Dims d,
                                                 Par<T> p) {
  constexpr int DIM = Lat::DIM;
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!decode(d, idx, x, y, z)) return;
  T qp[5], dq[3][5], lap[5], u[3], G[3][3], r2[5];
  q_stencil<T, DIM>(QP, d, x, y, z, qp, dq, lap);
  u_stencil<T, DIM>(U, d, x, y, z, u, G);
  be_rhs<T, DIM>(qp, dq, lap, u, G, p, r2);
#pragma unroll
  for (int k = 0; k < 5; k++)
    Qout[k * d.n + idx] = Q[k * d.n + idx] + (R1[k * d.n + idx] + r2[k]) / T(2);
}

}  // namespace nlc
