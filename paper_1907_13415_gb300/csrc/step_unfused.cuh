// step_unfused.cuh -- one time step as four one-cell-per-thread kernels.
//
//   1. stress   : Q^n -> Pi (Eq. 3 for H, Eq. 5 without P0)
//   2. lb       : F = div Pi, pull-stream, rho/u (Eq. 6), BGK + source,
//                 store post-collision deviations g* and u^n
//   3. predict  : R1 = R(Q^n; u^n), Q^P = Q^n + R1          (Sec. 1.2.2, 1-2)
//   4. correct  : R2 = R(Q^P; u^n), Q^{n+1} = Q^n + (R1+R2)/2 (steps 3-5)
//
// Populations are stored unpadded as deviations g_i = f_i - w_i rho0 in a
// pull layout: the buffer holds the post-collision values at the cell where
// the collision happened, and the pre-collision f_i(x, t) is
// w_i rho0 + g_i(x - c_i) (periodic).  Q, Q^P and u are padded fields whose
// ghost rings hold periodic images (common.cuh), so their neighbours are read
// without wrap-around.  Every intermediate goes through global memory; the
// fused schedule (step_fused.cuh) computes the same step with two tiled
// kernels.
#pragma once
#include "common.cuh"
#include "lattice.cuh"
#include "physics.cuh"

namespace nlc {

// five components at (x, y, z), their central first derivatives and the
// 2d+1-point Laplacian
template <class T, int DIM>
__device__ __forceinline__ void q_stencil(const Field<T>& Q, int x, int y,
                                          int z, T q[5], T dq[3][5], T lap[5]) {
#pragma unroll
  for (int k = 0; k < 5; k++) {
    const T v = Q.at(k, x, y, z);
    const T xp = Q.at(k, x + 1, y, z), xm = Q.at(k, x - 1, y, z);
    const T yp = Q.at(k, x, y + 1, z), ym = Q.at(k, x, y - 1, z);
    q[k] = v;
    dq[0][k] = (xp - xm) / T(2);
    dq[1][k] = (yp - ym) / T(2);
    T l = (xp + xm - T(2) * v) + (yp + ym - T(2) * v);
    if (DIM == 3) {
      const T zp = Q.at(k, x, y, z + 1), zm = Q.at(k, x, y, z - 1);
      dq[2][k] = (zp - zm) / T(2);
      l += zp + zm - T(2) * v;
    } else {
      dq[2][k] = T(0);
    }
    lap[k] = l;
  }
}

// u and the velocity gradient G[a][b] = d_b u_a by central differences
template <class T, int DIM>
__device__ __forceinline__ void u_stencil(const Field<T>& U, int x, int y,
                                          int z, T u[3], T G[3][3]) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    if (a < DIM) {
      u[a] = U.at(a, x, y, z);
      G[a][0] = (U.at(a, x + 1, y, z) - U.at(a, x - 1, y, z)) / T(2);
      G[a][1] = (U.at(a, x, y + 1, z) - U.at(a, x, y - 1, z)) / T(2);
      G[a][2] = DIM == 3 ? (U.at(a, x, y, z + 1) - U.at(a, x, y, z - 1)) / T(2) : T(0);
    } else {
      u[a] = T(0);
      G[a][0] = G[a][1] = G[a][2] = T(0);
    }
  }
}

// The same three from the isotropic stencils of the lattice's neighbour set:
// d_a v = (1/cs^2) sum_i w_i c_ia v(x + c_i),
// lap v = (2/cs^2) sum_i w_i [v(x + c_i) - v(x)].
template <class Lat, class T>
__device__ __forceinline__ void q_stencil_iso(const Field<T>& Q, int x, int y, int z, T q[5],
                                              T dq[3][5], T lap[5]) {
#pragma unroll
  for (int k = 0; k < 5; k++) {
    const T v = Q.at(k, x, y, z);
    T s = T(0), d[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int i = 1; i < Lat::Q; i++) {
      const T vi = Q.at(k, x + Lat::c(i, 0), y + Lat::c(i, 1), z + Lat::c(i, 2));
      const T w = T(Lat::w(i));
      s += w * (vi - v);
#pragma unroll
      for (int a = 0; a < 3; a++) d[a] += w * T(Lat::c(i, a)) * vi;
    }
    q[k] = v;
    lap[k] = T(6) * s;
#pragma unroll
    for (int a = 0; a < 3; a++) dq[a][k] = T(3) * d[a];
  }
}

template <class Lat, class T>
__device__ __forceinline__ void u_stencil_iso(const Field<T>& U, int x, int y, int z, T u[3],
                                              T G[3][3]) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    u[a] = a < Lat::DIM ? U.at(a, x, y, z) : T(0);
    G[a][0] = G[a][1] = G[a][2] = T(0);
    if (a >= Lat::DIM) continue;
#pragma unroll
    for (int i = 1; i < Lat::Q; i++) {
      const T vi = U.at(a, x + Lat::c(i, 0), y + Lat::c(i, 1), z + Lat::c(i, 2));
#pragma unroll
      for (int b = 0; b < 3; b++) G[a][b] += T(3.0 * Lat::w(i) * Lat::c(i, b)) * vi;
    }
  }
}

// A lattice holds fewer than 2^32 cells (nlc_create refuses more), so the
// cell index splits in unsigned 32-bit arithmetic.
__device__ __forceinline__ bool decode(const Dims& d, int64_t idx, int& x,
                                       int& y, int& z) {
  if (idx >= d.n) return false;
  const unsigned i = (unsigned)idx, nx = (unsigned)d.nx, ny = (unsigned)d.ny;
  const unsigned r = i / nx;
  x = (int)(i - r * nx);
  y = (int)(r % ny);
  z = (int)(r / ny);
  return true;
}

// The four stages at one cell (x, y, z) = decode(idx); the kernels below run
// one cell per thread, the adjoint's segment kernels (adjoint_segment.cuh)
// loop over cells with the same functions.
// iso: isotropic stencils (q_stencil_iso, u_stencil_iso, force_at_iso)
template <class Lat, class T>
__device__ __forceinline__ void stress_at(const Field<T>& Q, T* __restrict__ Pi, const Dims& d,
                                          const Par<T>& p, bool iso, int64_t idx, int x,
                                          int y, int z) {
  constexpr int DIM = Lat::DIM;
  T q[5], dq[3][5], lap[5], h[5], P[3][3];
  if (iso)
    q_stencil_iso<Lat, T>(Q, x, y, z, q, dq, lap);
  else
    q_stencil<T, DIM>(Q, x, y, z, q, dq, lap);
  molecular_field(q, lap, p, h);
  stress<T, DIM>(q, h, dq, p, P);
#pragma unroll
  for (int a = 0; a < DIM; a++)
#pragma unroll
    for (int b = 0; b < DIM; b++) Pi[(a * DIM + b) * d.n + idx] = P[a][b];
}

template <class Lat, class T>
__global__ void __launch_bounds__(256) k_stress(Field<T> Q, T* __restrict__ Pi,
                                                Dims d, Par<T> p, bool iso) {
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (decode(d, idx, x, y, z)) stress_at<Lat, T>(Q, Pi, d, p, iso, idx, x, y, z);
}

// F_a = sum_b [Pi_ab(x + e_b) - Pi_ab(x - e_b)] / 2  (Pi unpadded: wrap)
template <class T, int DIM>
__device__ __forceinline__ void force_at(const T* __restrict__ Pi,
                                         const Dims& d, int x, int y, int z,
                                         T F[3]) {
  // neighbour cells in unsigned 32-bit arithmetic (a lattice holds fewer
  // than 2^32 cells)
  const unsigned nx = (unsigned)d.nx, nxy = nx * (unsigned)d.ny;
  const unsigned pz = (unsigned)z * nxy, ry = (unsigned)y * nx;
  const unsigned nb[3][2] = {
      {pz + ry + (unsigned)wrap_inc(x, d.nx), pz + ry + (unsigned)wrap_dec(x, d.nx)},
      {pz + (unsigned)wrap_inc(y, d.ny) * nx + x, pz + (unsigned)wrap_dec(y, d.ny) * nx + x},
      {DIM == 3 ? (unsigned)wrap_inc(z, d.nz) * nxy + ry + x : 0u,
       DIM == 3 ? (unsigned)wrap_dec(z, d.nz) * nxy + ry + x : 0u}};
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

// F_a = (1/cs^2) sum_i w_i sum_b c_ib Pi_ab(x + c_i)  (isotropic; wrap)
template <class Lat, class T>
__device__ __forceinline__ void force_at_iso(const T* __restrict__ Pi, const Dims& d, int x,
                                             int y, int z, T F[3]) {
  constexpr int DIM = Lat::DIM;
  F[0] = F[1] = F[2] = T(0);
#pragma unroll
  for (int i = 1; i < Lat::Q; i++) {
    const int64_t ci = cell_of(d, wrap_add(x, Lat::c(i, 0), d.nx),
                               wrap_add(y, Lat::c(i, 1), d.ny),
                               DIM == 3 ? wrap_add(z, Lat::c(i, 2), d.nz) : z);
#pragma unroll
    for (int a = 0; a < DIM; a++)
#pragma unroll
      for (int b = 0; b < DIM; b++)
        if (Lat::c(i, b) != 0)
          F[a] += T(3.0 * Lat::w(i) * Lat::c(i, b)) * Pi[(a * DIM + b) * d.n + ci];
  }
}

// pre-collision deviations g_i(x, t) = g*_i(x - c_i) (pull, periodic)
template <class Lat, class T, class G>
__device__ __forceinline__ void pull(const G* __restrict__ gin, const Dims& d,
                                     int x, int y, int z, T g[Lat::Q]) {
  // source offsets along each axis for c = +1, 0, -1 (index 1 - c), in
  // unsigned 32-bit arithmetic (a lattice holds fewer than 2^32 cells)
  const unsigned nx = (unsigned)d.nx, nxy = nx * (unsigned)d.ny;
  const unsigned col[3] = {(unsigned)wrap_dec(x, d.nx), (unsigned)x, (unsigned)wrap_inc(x, d.nx)};
  const unsigned row[3] = {(unsigned)wrap_dec(y, d.ny) * nx, (unsigned)y * nx,
                           (unsigned)wrap_inc(y, d.ny) * nx};
  const unsigned pz = (unsigned)z * nxy;
  const unsigned pla[3] = {Lat::DIM == 3 ? (unsigned)wrap_dec(z, d.nz) * nxy : pz, pz,
                           Lat::DIM == 3 ? (unsigned)wrap_inc(z, d.nz) * nxy : pz};
#pragma unroll
  for (int i = 0; i < Lat::Q; i++) {
    const unsigned off = pla[1 - Lat::c(i, 2)] + row[1 - Lat::c(i, 1)] + col[1 - Lat::c(i, 0)];
    g[i] = T(gin[(int64_t)i * d.n + off]);
  }
}

// mrt: the Q coefficients s_k / |v_k|^2 of the MRT collision, or nullptr
// for BGK
template <class Lat, class T, class G>
__device__ __forceinline__ void lb_at(const G* __restrict__ gin, G* __restrict__ gout,
                                      const T* __restrict__ Pi, const Field<T>& U,
                                      const Dims& d, const Par<T>& p, const T* mrt, bool iso,
                                      int64_t idx, int x, int y, int z) {
  T F[3], g[Lat::Q], rho, u[3];
  if (iso)
    force_at_iso<Lat, T>(Pi, d, x, y, z, F);
  else
    force_at<T, Lat::DIM>(Pi, d, x, y, z, F);
  pull<Lat, T>(gin, d, x, y, z, g);
  moments<Lat, T>(g, F, p, rho, u);
  if (mrt)
    collide_mrt<Lat, T>(g, rho, u, F, p, mrt);
  else
    collide_bgk<Lat, T>(g, rho, u, F, p);
#pragma unroll
  for (int i = 0; i < Lat::Q; i++) gout[(int64_t)i * d.n + idx] = G(g[i]);
  store_with_images<T, Lat::DIM, Lat::DIM>(U, d, x, y, z, u);
}

template <class Lat, class T, class G>
__global__ void __launch_bounds__(256) k_lb(const G* __restrict__ gin,
                                            G* __restrict__ gout,
                                            const T* __restrict__ Pi,
                                            Field<T> U, Dims d, Par<T> p,
                                            const T* __restrict__ mrt, bool iso) {
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (decode(d, idx, x, y, z))
    lb_at<Lat, T>(gin, gout, Pi, U, d, p, mrt, iso, idx, x, y, z);
}

template <class Lat, class T>
__device__ __forceinline__ void predict_at(const Field<T>& Q, const Field<T>& U,
                                           const Field<T>& QP, T* __restrict__ R1,
                                           const Dims& d, const Par<T>& p, bool iso,
                                           int64_t idx, int x, int y, int z) {
  constexpr int DIM = Lat::DIM;
  T q[5], dq[3][5], lap[5], u[3], G[3][3], r[5], qp[5];
  if (iso) {
    q_stencil_iso<Lat, T>(Q, x, y, z, q, dq, lap);
    u_stencil_iso<Lat, T>(U, x, y, z, u, G);
  } else {
    q_stencil<T, DIM>(Q, x, y, z, q, dq, lap);
    u_stencil<T, DIM>(U, x, y, z, u, G);
  }
  be_rhs<T, DIM>(q, dq, lap, u, G, p, r);
#pragma unroll
  for (int k = 0; k < 5; k++) {
    R1[k * d.n + idx] = r[k];
    qp[k] = q[k] + r[k];
  }
  store_with_images<T, 5, DIM>(QP, d, x, y, z, qp);
}

template <class Lat, class T>
__global__ void __launch_bounds__(256) k_predict(Field<T> Q, Field<T> U,
                                                 Field<T> QP,
                                                 T* __restrict__ R1, Dims d,
                                                 Par<T> p, bool iso) {
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (decode(d, idx, x, y, z)) predict_at<Lat, T>(Q, U, QP, R1, d, p, iso, idx, x, y, z);
}

template <class Lat, class T>
__device__ __forceinline__ void correct_at(const Field<T>& Q, const Field<T>& QP,
                                           const T* __restrict__ R1, const Field<T>& U,
                                           const Field<T>& Qout, const Dims& d,
                                           const Par<T>& p, bool iso, int64_t idx, int x,
                                           int y, int z) {
  constexpr int DIM = Lat::DIM;
  T qp[5], dq[3][5], lap[5], u[3], G[3][3], r2[5], out[5];
  if (iso) {
    q_stencil_iso<Lat, T>(QP, x, y, z, qp, dq, lap);
    u_stencil_iso<Lat, T>(U, x, y, z, u, G);
  } else {
    q_stencil<T, DIM>(QP, x, y, z, qp, dq, lap);
    u_stencil<T, DIM>(U, x, y, z, u, G);
  }
  be_rhs<T, DIM>(qp, dq, lap, u, G, p, r2);
#pragma unroll
  for (int k = 0; k < 5; k++)
    out[k] = Q.at(k, x, y, z) + (R1[k * d.n + idx] + r2[k]) / T(2);
  store_with_images<T, 5, DIM>(Qout, d, x, y, z, out);
}

template <class Lat, class T>
__global__ void __launch_bounds__(256) k_correct(Field<T> Q, Field<T> QP,
                                                 const T* __restrict__ R1,
                                                 Field<T> U, Field<T> Qout,
                                                 Dims d, Par<T> p, bool iso) {
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (decode(d, idx, x, y, z))
    correct_at<Lat, T>(Q, QP, R1, U, Qout, d, p, iso, idx, x, y, z);
}

}  // namespace nlc
