// adjoint.cuh -- the stages of one reverse time step of the hybrid scheme
// (hand-written adjoint) as per-cell functions, run by the segment kernels of
// adjoint_segment.cuh, and the kernels of the droplet loss's seed.
//
// Notation: the state at step n is (Q^n, g^n) with g the post-collision
// deviations in pull layout (step_unfused.cuh).  Adjoints are dense [comp][n]
// arrays (neighbours by periodic wrap).  Given the adjoints of the state at
// n+1 (lQn, lGn) the stages produce the adjoints at n (lQ, lG), reading the
// forward intermediates of step n (Pi, u^n, Q^P) recorded for the segment.
//
// The transposes of the stencils are written in gather form:
//   central difference  d_g v(x) = [v(x+e_g) - v(x-e_g)]/2
//        -> vbar(y) += [dbar_g(y-e_g) - dbar_g(y+e_g)]/2
//   Laplacian           lap v(x) = sum_g v(x+e_g) + v(x-e_g) - 2 v(x)
//        -> vbar(y) += sum_g lbar(y+e_g) + lbar(y-e_g) - 2 lbar(y)
//   pull streaming      f_i(x) = g_i(x - c_i)
//        -> gbar_i(x - c_i) = fbar_i(x)        (a permutation: plain stores)
// and, because R (Eq. 1) depends on the derivatives of Q only through
// -u.grad Q and Gamma K lap Q, its stencil adjoints are closed forms:
//   dbar_g = -u_g rbar,  lbar = Gamma K rbar.
#pragma once
#include "adjoint_point.cuh"
#include "common.cuh"
#include "step_unfused.cuh"

namespace nlc {

// neighbour of cell (x, y, z) in direction g (0..2), sign s (+1, -1), periodic
__device__ __forceinline__ int64_t nbr(const Dims& d, int x, int y, int z, int g, int s) {
  if (g == 0) return cell_of(d, s > 0 ? wrap_inc(x, d.nx) : wrap_dec(x, d.nx), y, z);
  if (g == 1) return cell_of(d, x, s > 0 ? wrap_inc(y, d.ny) : wrap_dec(y, d.ny), z);
  return cell_of(d, x, y, s > 0 ? wrap_inc(z, d.nz) : wrap_dec(z, d.nz));
}

// block sum of the three parameter adjoints into this block's accumulator
// slot (acc[block][3]; each block owns its slot, so the order is fixed)
template <class T>
__device__ __forceinline__ void add_param_bar(const ParBar<T>& pb, double* acc) {
  __shared__ double sh[32];
  const double g = block_sum((double)pb.gamma, sh);
  const double k = block_sum((double)pb.K, sh);
  const double G = block_sum((double)pb.Gamma, sh);
  if (threadIdx.x == 0) {
    acc[3 * blockIdx.x + 0] += g;
    acc[3 * blockIdx.x + 1] += k;
    acc[3 * blockIdx.x + 2] += G;
  }
}

// gather of the R-stencil adjoints for rbar = a * A(x) + b * B(x):
//   sum_g [u_g(y+e_g) rbar(y+e_g) - u_g(y-e_g) rbar(y-e_g)] / 2
//   + Gamma K (sum_g rbar(y+e_g) + rbar(y-e_g) - 2 rbar(y))
template <class T, int DIM>
__device__ __forceinline__ void rhs_stencil_gather(const Field<T>& U, const T* __restrict__ A,
                                                   T a, const T* __restrict__ B, T b,
                                                   const Dims& d, int x, int y, int z,
                                                   const Par<T>& p, T out[5]) {
  const int64_t c = cell_of(d, x, y, z);
  const T gk = p.Gamma * p.K;
#pragma unroll
  for (int k = 0; k < 5; k++) {
    const T r0 = a * A[k * d.n + c] + (B ? b * B[k * d.n + c] : T(0));
    out[k] += -T(2) * DIM * gk * r0;
  }
#pragma unroll
  for (int g = 0; g < DIM; g++) {
    const int64_t cp = nbr(d, x, y, z, g, +1), cm = nbr(d, x, y, z, g, -1);
    const int xp = g == 0 ? x + 1 : x, yp = g == 1 ? y + 1 : y, zp = g == 2 ? z + 1 : z;
    const int xm = g == 0 ? x - 1 : x, ym = g == 1 ? y - 1 : y, zm = g == 2 ? z - 1 : z;
    const T up = U.at(g, xp, yp, zp), um = U.at(g, xm, ym, zm);
#pragma unroll
    for (int k = 0; k < 5; k++) {
      const T rp = a * A[k * d.n + cp] + (B ? b * B[k * d.n + cp] : T(0));
      const T rm = a * A[k * d.n + cm] + (B ? b * B[k * d.n + cm] : T(0));
      out[k] += (up * rp - um * rm) / T(2) + gk * (rp + rm);
    }
  }
}

// 1. adjoint of the corrector evaluation R2 = R(Q^P; u): rbar = lQn / 2.
//    lQP = J^T rbar (pointwise at Q^P plus stencil gathers); the adjoints of
//    u (advection) and of G = grad u are stored for the lb adjoint.
template <class Lat, class T>
__device__ __forceinline__ void adj_be2_at(const Field<T>& QP, const Field<T>& U,
                                           const T* __restrict__ lQn, T* __restrict__ lQP,
                                           T* __restrict__ lUa, T* __restrict__ lGv,
                                           const Dims& d, const Par<T>& p, ParBar<T>& pb,
                                           int64_t idx, int x, int y, int z) {
  constexpr int DIM = Lat::DIM;
  {
    T q[5], dq[3][5], lap[5], u[3], G[3][3], rb[5];
    q_stencil<T, DIM>(QP, x, y, z, q, dq, lap);
    u_stencil<T, DIM>(U, x, y, z, u, G);
#pragma unroll
    for (int k = 0; k < 5; k++) rb[k] = lQn[k * d.n + idx] / T(2);
    T qb[5] = {}, dqb[3][5] = {}, lapb[5] = {}, ub[3] = {}, Gb[3][3] = {};
    be_rhs_vjp<T, DIM>(q, dq, lap, u, G, p, rb, qb, dqb, lapb, ub, Gb, pb);
    rhs_stencil_gather<T, DIM>(U, lQn, T(0.5), nullptr, T(0), d, x, y, z, p, qb);
#pragma unroll
    for (int k = 0; k < 5; k++) lQP[k * d.n + idx] = qb[k];
#pragma unroll
    for (int a = 0; a < DIM; a++) {
      lUa[a * d.n + idx] = ub[a];
#pragma unroll
      for (int b = 0; b < DIM; b++) lGv[(a * DIM + b) * d.n + idx] = Gb[a][b];
    }
  }
}

// 2. adjoint of the predictor evaluation R1 = R(Q^n; u), with
//    rbar = lQn / 2 + lQP (R1 enters Q^{n+1} with 1/2 and Q^P with 1), and
//    of Q^{n+1} = Q^n + ..., Q^P = Q^n + R1:  lQ = lQn + lQP + J^T rbar.
template <class Lat, class T>
__device__ __forceinline__ void adj_be1_at(const Field<T>& Q, const Field<T>& U,
                                           const T* __restrict__ lQn,
                                           const T* __restrict__ lQP, T* __restrict__ lQ,
                                           T* __restrict__ lUa, T* __restrict__ lGv,
                                           const Dims& d, const Par<T>& p, ParBar<T>& pb,
                                           int64_t idx, int x, int y, int z) {
  constexpr int DIM = Lat::DIM;
  {
    T q[5], dq[3][5], lap[5], u[3], G[3][3], rb[5];
    q_stencil<T, DIM>(Q, x, y, z, q, dq, lap);
    u_stencil<T, DIM>(U, x, y, z, u, G);
#pragma unroll
    for (int k = 0; k < 5; k++) rb[k] = lQn[k * d.n + idx] / T(2) + lQP[k * d.n + idx];
    T qb[5] = {}, dqb[3][5] = {}, lapb[5] = {}, ub[3] = {}, Gb[3][3] = {};
    be_rhs_vjp<T, DIM>(q, dq, lap, u, G, p, rb, qb, dqb, lapb, ub, Gb, pb);
    rhs_stencil_gather<T, DIM>(U, lQn, T(0.5), lQP, T(1), d, x, y, z, p, qb);
#pragma unroll
    for (int k = 0; k < 5; k++)
      lQ[k * d.n + idx] = lQn[k * d.n + idx] + lQP[k * d.n + idx] + qb[k];
#pragma unroll
    for (int a = 0; a < DIM; a++) {
      lUa[a * d.n + idx] += ub[a];
#pragma unroll
      for (int b = 0; b < DIM; b++) lGv[(a * DIM + b) * d.n + idx] += Gb[a][b];
    }
  }
}

// 3. adjoint of the LB update at cell x: u-bar from the Beris-Edwards side
//    (advection + gather of the grad-u adjoint), then collision and moments;
//    the pre-collision adjoint is stored pulled back: lG_i(x - c_i).
//    Writes the force adjoint lF for the stress adjoint.
//    lGn == nullptr: seed mode (no collision; only u of the final state).
template <class Lat, class T, class G>
__device__ __forceinline__ void adj_lb_at(const G* __restrict__ gin, const T* __restrict__ Pi,
                                          const T* __restrict__ lGn,
                                          const T* __restrict__ lUa,
                                          const T* __restrict__ lGv, T* __restrict__ lG,
                                          T* __restrict__ lF, const Dims& d, const Par<T>& p,
                                          T seed_u, int64_t idx, int x, int y, int z) {
  constexpr int DIM = Lat::DIM;
  T F[3], g[Lat::Q], rho, u[3];
  force_at<T, DIM>(Pi, d, x, y, z, F);
  pull<Lat, T>(gin, d, x, y, z, g);
  moments<Lat, T>(g, F, p, rho, u);
  T ub[3] = {T(0), T(0), T(0)}, Fb[3] = {T(0), T(0), T(0)}, rhob = T(0), gb[Lat::Q];
  if (lGn) {
#pragma unroll
    for (int a = 0; a < DIM; a++) {
      T s = lUa[a * d.n + idx];
#pragma unroll
      for (int b = 0; b < DIM; b++)
        s += (lGv[(a * DIM + b) * d.n + nbr(d, x, y, z, b, -1)] -
              lGv[(a * DIM + b) * d.n + nbr(d, x, y, z, b, +1)]) / T(2);
      ub[a] = s;
    }
#pragma unroll
    for (int i = 0; i < Lat::Q; i++) gb[i] = lGn[(int64_t)i * d.n + idx];
    collide_bgk_vjp<Lat, T>(gb, rho, u, F, p, rhob, ub, Fb);
  } else {
    // loss seed: d/du of seed_u * |u|-norm term handled by the caller's
    // scaling: ubar = seed_u * u
#pragma unroll
    for (int a = 0; a < DIM; a++) ub[a] = seed_u * u[a];
#pragma unroll
    for (int i = 0; i < Lat::Q; i++) gb[i] = T(0);
  }
  moments_vjp<Lat, T>(rho, u, rhob, ub, gb, Fb);
#pragma unroll
  for (int i = 0; i < Lat::Q; i++) {
    const int xs = wrap_add(x, -Lat::c(i, 0), d.nx);
    const int ys = wrap_add(y, -Lat::c(i, 1), d.ny);
    const int zs = DIM == 3 ? wrap_add(z, -Lat::c(i, 2), d.nz) : z;
    lG[(int64_t)i * d.n + cell_of(d, xs, ys, zs)] = gb[i];
  }
#pragma unroll
  for (int a = 0; a < DIM; a++) lF[a * d.n + idx] = Fb[a];
}

template <class Lat, class T, class G>
__global__ void __launch_bounds__(256) k_adj_lb(const G* __restrict__ gin,
                                                const T* __restrict__ Pi,
                                                const T* __restrict__ lGn,
                                                const T* __restrict__ lUa,
                                                const T* __restrict__ lGv,
                                                T* __restrict__ lG, T* __restrict__ lF,
                                                Dims d, Par<T> p, T seed_u) {
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (decode(d, idx, x, y, z))
    adj_lb_at<Lat, T>(gin, Pi, lGn, lUa, lGv, lG, lF, d, p, seed_u, idx, x, y, z);
}

// 4. adjoint of the stress at cell y: Pibar from the divergence transpose of
//    lF, then stress and molecular-field adjoints; adds the pointwise Q
//    adjoint to lQ and stores the derivative/Laplacian adjoints for step 5.
template <class Lat, class T>
__device__ __forceinline__ void adj_stress_at(const Field<T>& Q, const T* __restrict__ lF,
                                              T* __restrict__ lQ, T* __restrict__ lDq,
                                              T* __restrict__ lLap, const Dims& d,
                                              const Par<T>& p, ParBar<T>& pb, int64_t idx,
                                              int x, int y, int z) {
  constexpr int DIM = Lat::DIM;
  {
    T Pib[3][3] = {};
#pragma unroll
    for (int a = 0; a < DIM; a++)
#pragma unroll
      for (int b = 0; b < DIM; b++)
        Pib[a][b] = (lF[a * d.n + nbr(d, x, y, z, b, -1)] -
                     lF[a * d.n + nbr(d, x, y, z, b, +1)]) / T(2);
    T q[5], dq[3][5], lap[5], h[5];
    q_stencil<T, DIM>(Q, x, y, z, q, dq, lap);
    molecular_field(q, lap, p, h);
    T qb[5] = {}, hb[5] = {}, dqb[3][5] = {}, lapb[5] = {};
    stress_vjp<T, DIM>(q, h, dq, p, Pib, qb, hb, dqb, pb);
    molecular_field_vjp(q, lap, p, hb, qb, lapb, pb);
#pragma unroll
    for (int k = 0; k < 5; k++) {
      lQ[k * d.n + idx] += qb[k];
      lLap[k * d.n + idx] = lapb[k];
#pragma unroll
      for (int g = 0; g < DIM; g++) lDq[(g * 5 + k) * d.n + idx] = dqb[g][k];
    }
  }
}

template <class Lat, class T>
__global__ void __launch_bounds__(256) k_adj_stress(Field<T> Q, const T* __restrict__ lF,
                                                    T* __restrict__ lQ, T* __restrict__ lDq,
                                                    T* __restrict__ lLap, Dims d, Par<T> p,
                                                    double* __restrict__ acc) {
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  ParBar<T> pb{T(0), T(0), T(0)};
  if (decode(d, idx, x, y, z))
    adj_stress_at<Lat, T>(Q, lF, lQ, lDq, lLap, d, p, pb, idx, x, y, z);
  add_param_bar(pb, acc);
}

// 5. stencil transposes of the stress adjoint: lQ += div-transpose(lDq) +
//    Laplacian-transpose(lLap)
template <class Lat, class T>
__device__ __forceinline__ void adj_stencil_at(const T* __restrict__ lDq,
                                               const T* __restrict__ lLap, T* __restrict__ lQ,
                                               const Dims& d, int64_t idx, int x, int y,
                                               int z) {
  constexpr int DIM = Lat::DIM;
#pragma unroll
  for (int k = 0; k < 5; k++) {
    T s = -T(2) * DIM * lLap[k * d.n + idx];
#pragma unroll
    for (int g = 0; g < DIM; g++) {
      const int64_t cp = nbr(d, x, y, z, g, +1), cm = nbr(d, x, y, z, g, -1);
      s += (lDq[(g * 5 + k) * d.n + cm] - lDq[(g * 5 + k) * d.n + cp]) / T(2);
      s += lLap[k * d.n + cp] + lLap[k * d.n + cm];
    }
    lQ[k * d.n + idx] += s;
  }
}

template <class Lat, class T>
__global__ void __launch_bounds__(256) k_adj_stencil(const T* __restrict__ lDq,
                                                     const T* __restrict__ lLap,
                                                     T* __restrict__ lQ, Dims d) {
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (decode(d, idx, x, y, z)) adj_stencil_at<Lat, T>(lDq, lLap, lQ, d, idx, x, y, z);
}

// loss seed on Q: lQ = c_R dS/dq with S = sqrt(3/2 Tr Q^2) (0 where S = 0)
template <class T>
__global__ void __launch_bounds__(256) k_adj_seed_q(Field<T> Q, T cR, T* __restrict__ lQ,
                                                    Dims d) {
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!decode(d, idx, x, y, z)) return;
  T q[5];
#pragma unroll
  for (int k = 0; k < 5; k++) q[k] = Q.at(k, x, y, z);
  const T a = q[0], dd = q[3];
  const T tr2 = T(2) * (a * a + dd * dd + a * dd + q[1] * q[1] + q[2] * q[2] + q[4] * q[4]);
  const T S = sqrt(T(1.5) * tr2);
  const T s = S > T(0) ? cR * T(1.5) / (T(2) * S) : T(0);
  lQ[0 * d.n + idx] = s * (T(4) * a + T(2) * dd);
  lQ[1 * d.n + idx] = s * T(4) * q[1];
  lQ[2 * d.n + idx] = s * T(4) * q[2];
  lQ[3 * d.n + idx] = s * (T(4) * dd + T(2) * a);
  lQ[4 * d.n + idx] = s * T(4) * q[4];
}

// dense [5][n] adjoint of Q to float64 (host read-back)
template <class T>
__global__ void __launch_bounds__(256) k_dense_to_double(const T* __restrict__ in,
                                                         double* __restrict__ out,
                                                         int64_t count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = (double)in[i];
}

}  // namespace nlc
