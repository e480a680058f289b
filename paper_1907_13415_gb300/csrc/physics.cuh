// physics.cuh -- pointwise pieces of the hybrid step, templated on the
// arithmetic type T (float or double) and the dimension.
//
// Notation follows Sec. 1.1: Q the order tensor (symmetric, traceless, five
// stored components xx, xy, xz, yy, yz with Qzz = -Qxx - Qyy), H the
// molecular field (Eq. 3), Pi the stress of Eq. 5 without P0, S the
// co-rotational term of Eq. 1, G[a][b] = d_b u_a the velocity gradient.
#pragma once
#ifdef __CUDACC__
#include "packed.cuh"
#endif

namespace nlc {

// fused multiply-add, written out where the pointwise physics wants one
// rounding per product-and-sum (other scalar types, such as the complex
// type of the derivative checks, add their own overload)
__host__ __device__ __forceinline__ double fma_(double a, double b, double c) {
  return fma(a, b, c);
}
__host__ __device__ __forceinline__ float fma_(float a, float b, float c) {
  return fmaf(a, b, c);
}

template <class T>
struct Par {
  T A0, K, gamma, Gamma, xi, tau, rho0;
  T inv_tau;  // 1/tau
  T guo;      // 1 - 1/(2 tau), the prefactor of the source term
  // parameter factors of Eq. 3, Eq. 5 and Eq. 1, formed once by derive() so
  // that no cell divides or recombines parameters
  T Ag;       // A0 gamma
  T A1;       // -A0 (1 - gamma/3)
  T Ag3;      // -A0 gamma/3
  T xm1, xp1; // xi - 1, xi + 1
  T x23;      // 2 xi/3
  T x2;       // 2 xi
  T hp, hm;   // (xi + 1)/2, (xi - 1)/2
  T x29;      // 2 xi/9
};

// inv_tau, guo and the factors above from A0, K, gamma, Gamma, xi, tau
template <class T>
__host__ __device__ inline void derive(Par<T>& p) {
  p.inv_tau = T(1) / p.tau;
  p.guo = T(1) - T(1) / (T(2) * p.tau);
  p.Ag = p.A0 * p.gamma;
  p.A1 = -p.A0 * (T(1) - p.gamma / T(3));
  p.Ag3 = -p.Ag / T(3);
  p.xm1 = p.xi - T(1);
  p.xp1 = p.xi + T(1);
  p.x23 = T(2) * p.xi / T(3);
  p.x2 = T(2) * p.xi;
  p.hp = (p.xi + T(1)) * T(0.5);
  p.hm = (p.xi - T(1)) * T(0.5);
  p.x29 = T(2) * p.xi / T(9);
}

// five stored components -> full symmetric traceless 3x3
template <class T>
__host__ __device__ __forceinline__ void q_full(const T q[5], T Q[3][3]) {
  Q[0][0] = q[0];
  Q[0][1] = q[1];
  Q[0][2] = q[2];
  Q[1][0] = q[1];
  Q[1][1] = q[3];
  Q[1][2] = q[4];
  Q[2][0] = q[2];
  Q[2][1] = q[4];
  Q[2][2] = -q[0] - q[3];
}

// Products of symmetric traceless tensors are written out in the five stored
// components (a, b, c, d, e) = (xx, xy, xz, yy, yz), f = zz = -a - d.

// Eq. 3: H = -A0(1-g/3) Q - A0 g (Tr(Q^2) I/3 - Q Q) - A0 g Q Tr(Q^2) + K lapQ
// (returned as the five independent components; H is symmetric traceless)
template <class T>
__host__ __device__ __forceinline__ void molecular_field(const T q[5], const T lap[5],
                                                const Par<T>& p, T h[5]) {
  const T a = q[0], b = q[1], c = q[2], d = q[3], e = q[4], f = -q[0] - q[3];
  // (Q Q)_xx, _xy, _xz, _yy, _yz
  const T qq0 = a * a + b * b + c * c;
  const T qq1 = a * b + b * d + c * e;
  const T qq2 = a * c + b * e + c * f;
  const T qq3 = b * b + d * d + e * e;
  const T qq4 = b * c + d * e + e * f;
  const T tr2 = a * a + d * d + f * f + T(2) * (b * b + c * c + e * e);
  const T Ag = p.Ag;
  const T c1 = p.A1 - Ag * tr2;
  const T c3 = p.Ag3 * tr2;
  h[0] = c1 * a + Ag * qq0 + c3 + p.K * lap[0];
  h[1] = c1 * b + Ag * qq1 + p.K * lap[1];
  h[2] = c1 * c + Ag * qq2 + p.K * lap[2];
  h[3] = c1 * d + Ag * qq3 + c3 + p.K * lap[3];
  h[4] = c1 * e + Ag * qq4 + p.K * lap[4];
}

// d_a Q : d_b Q over all nine entries of the full tensors, from the
// derivatives A = d_a q, B = d_b q of the five stored components
// (Qzz = -Qxx - Qyy makes the zz entry add A_0 B_0 + A_3 B_3 + A_0 B_3 + A_3 B_0,
// and the off-diagonals count twice):  2 sum_k A_k B_k + A_0 B_3 + A_3 B_0.
template <class T>
__host__ __device__ __forceinline__ T grad_dot(const T A[5], const T B[5]) {
  const T s = fma_(A[0], B[0], fma_(A[1], B[1], fma_(A[2], B[2], fma_(A[3], B[3], A[4] * B[4]))));
  return fma_(T(2), s, fma_(A[0], B[3], A[3] * B[0]));
}

#ifdef __CUDACC__
// FP32: the first four products on packed pairs of components (packed.cuh;
// plain C++ builds of this file take the template above)
__host__ __device__ __forceinline__ float grad_dot(const float A[5], const float B[5]) {
  float2 s2 = pmul(pk(A[0], A[1]), pk(B[0], B[1]));
  s2 = pfma(pk(A[2], A[3]), pk(B[2], B[3]), s2);
  const float s = fma_(A[4], B[4], s2.x + s2.y);
  return fma_(2.0f, s, fma_(A[0], B[3], A[3] * B[0]));
}
#endif

// Eq. 5 without P0, with dF/d(d_b Q) = K d_b Q:
//   Pi_ab = 2 xi Qt_ab (Q:H) - xi (H Qt)_ab - xi (Qt H)_ab
//           - K d_a Q : d_b Q + (Q H)_ab - (H Q)_ab,      Qt = Q + I/3.
// With X = Q H (so H Q = X^T, H Qt = X^T + H/3, Qt H = X + H/3):
//   Pi_ab = 2 xi Qt_ab (Q:H) - (xi - 1) X_ab - (xi + 1) X_ba
//           - (2 xi/3) H_ab - K d_a Q : d_b Q.
// Q:H is the trace of X (Q, H symmetric), and on the diagonal the two X
// terms combine to -2 xi X_aa.
// dq[g][k]: d_g of stored component k.  Only a, b < DIM are produced.
template <class T, int DIM>
__host__ __device__ __forceinline__ void stress(const T q[5], const T h[5],
                                       const T dq[3][5], const Par<T>& p,
                                       T Pi[3][3]) {
  const T Q[3][3] = {{q[0], q[1], q[2]}, {q[1], q[3], q[4]}, {q[2], q[4], -q[0] - q[3]}};
  const T H[3][3] = {{h[0], h[1], h[2]}, {h[1], h[3], h[4]}, {h[2], h[4], -h[0] - h[3]}};
  const T xm1 = p.xm1, xp1 = p.xp1, x23 = p.x23;
  T X[3][3];  // X = Q H
#pragma unroll
  for (int a = 0; a < DIM; a++)
#pragma unroll
    for (int b = 0; b < DIM; b++)
      X[a][b] = fma_(Q[a][0], H[0][b], fma_(Q[a][1], H[1][b], Q[a][2] * H[2][b]));
  const T x22 = DIM == 3 ? X[2][2]
                         : fma_(Q[2][0], H[0][2], fma_(Q[2][1], H[1][2], Q[2][2] * H[2][2]));
  const T xqh = p.x2 * (X[0][0] + X[1][1] + x22);  // 2 xi Q:H
#pragma unroll
  for (int a = 0; a < DIM; a++)
#pragma unroll
    for (int b = a; b < DIM; b++) {
      const T el = grad_dot(dq[a], dq[b]);
      const T qt = Q[a][b] + (a == b ? T(1) / T(3) : T(0));
      const T sym = fma_(xqh, qt, fma_(-x23, H[a][b], -p.K * el));
      if (b == a) {
        Pi[a][a] = fma_(-p.x2, X[a][a], sym);
      } else {
        Pi[a][b] = fma_(-xm1, X[a][b], fma_(-xp1, X[b][a], sym));
        Pi[b][a] = fma_(-xm1, X[b][a], fma_(-xp1, X[a][b], sym));
      }
    }
}

// Co-rotational term of Eq. 1:
//   S = (xi D + W) Qt + Qt (xi D - W) - 2 xi Qt (Q_ge d_g u_e)
//   W_ab = (d_b u_a - d_a u_b)/2, D_ab = (d_b u_a + d_a u_b)/2.
// G[a][b] = d_b u_a.  With M = xi D + W = ((xi+1) G + (xi-1) G^T)/2 one has
// xi D - W = M^T, so S = P + P^T - 2 xi Qt (Q:G^T) with P = M Qt.
// Writes the five stored components of S.
// hp = (xi + 1)/2, hm = (xi - 1)/2, x2 = 2 xi.
template <class T>
__host__ __device__ __forceinline__ void corotation(const T G[3][3], const T q[5],
                                                    T hp, T hm, T x2, T s[5]) {
  const T third = T(1) / T(3);
  const T Qt[3][3] = {{q[0] + third, q[1], q[2]},
                      {q[1], q[3] + third, q[4]},
                      {q[2], q[4], third - q[0] - q[3]}};
  T M[3][3];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) M[a][b] = fma_(hp, G[a][b], hm * G[b][a]);
  // Q_ge d_g u_e = sum Q_ge G_eg
  const T qg = fma_(q[0], G[0][0] - G[2][2], fma_(q[3], G[1][1] - G[2][2],
               fma_(q[1], G[0][1] + G[1][0], fma_(q[2], G[0][2] + G[2][0],
                                                  q[4] * (G[1][2] + G[2][1])))));
  auto P = [&](int a, int b) {
    return fma_(M[a][0], Qt[0][b], fma_(M[a][1], Qt[1][b], M[a][2] * Qt[2][b]));
  };
  const T t = x2 * qg;
  s[0] = fma_(-t, Qt[0][0], T(2) * P(0, 0));
  s[1] = fma_(-t, Qt[0][1], P(0, 1) + P(1, 0));
  s[2] = fma_(-t, Qt[0][2], P(0, 2) + P(2, 0));
  s[3] = fma_(-t, Qt[1][1], T(2) * P(1, 1));
  s[4] = fma_(-t, Qt[1][2], P(1, 2) + P(2, 1));
}

template <class T>
__host__ __device__ __forceinline__ void corotation(const T G[3][3], const T q[5], T xi,
                                                    T s[5]) {
  corotation(G, q, (xi + T(1)) * T(0.5), (xi - T(1)) * T(0.5), T(2) * xi, s);
}

// Right-hand side of Eq. 1 at one cell,
//   R = -u_g d_g Q + S(W, D, Q) + Gamma H,
// made traceless by the orthogonal projection R <- R - Tr(R)/3 I.  The
// advection and H terms are traceless, and for traceless Q the trace of S is
// 2 xi div(u)/3 identically, so Tr(R) = 2 xi (G_xx + G_yy + G_zz)/3.
// Inputs: q (5), its central first derivatives dq[g][k], its Laplacian
// lap[k], u (3), G.
// The same from the advection term already formed, adv[k] = u_g d_g Q_k
// times -1/am (am = -1: adv itself; the fused kernel passes twice the term
// with am = -1/2).
template <class T>
__host__ __device__ __forceinline__ void be_rhs_adv(const T q[5], const T adv[5],
                                           const T lap[5], const T G[3][3],
                                           const Par<T>& p, T r[5], T am = T(-1)) {
  T h[5], s[5];
  molecular_field(q, lap, p, h);
  corotation(G, q, p.hp, p.hm, p.x2, s);
  const T tr3 = p.x29 * (G[0][0] + G[1][1] + G[2][2]);
  r[0] = fma_(p.Gamma, h[0], fma_(am, adv[0], s[0])) - tr3;
  r[1] = fma_(p.Gamma, h[1], fma_(am, adv[1], s[1]));
  r[2] = fma_(p.Gamma, h[2], fma_(am, adv[2], s[2]));
  r[3] = fma_(p.Gamma, h[3], fma_(am, adv[3], s[3])) - tr3;
  r[4] = fma_(p.Gamma, h[4], fma_(am, adv[4], s[4]));
}

template <class T, int DIM>
__host__ __device__ __forceinline__ void be_rhs(const T q[5], const T dq[3][5],
                                       const T lap[5], const T u[3],
                                       const T G[3][3], const Par<T>& p,
                                       T r[5]) {
  T adv[5];
#pragma unroll
  for (int k = 0; k < 5; k++) {
    T a = fma_(u[0], dq[0][k], u[1] * dq[1][k]);
    if (DIM == 3) a = fma_(u[2], dq[2][k], a);
    adv[k] = a;
  }
  be_rhs_adv(q, adv, lap, G, p, r);
}

// Equilibrium deviation g^eq_i = f^eq_i - w_i rho0, with
// f^eq_i = rho w_i [1 + c.u/cs2 + (c.u)^2/(2 cs2^2) - u^2/(2 cs2)] (Sec. 1.2.1)
// and the BGK source term
// S_i = w_i (1 - 1/2tau) [c_i/cs2 (1 + c_i.u/cs2) - u/cs2] . F,
// cs2 = 1/3.  Opposite velocities c_j = -c_i share the even parts
//   g^eq: w (drho + rho (9/2 (c.u)^2 - 3/2 u.u)),  S: w k (9 (c.F)(c.u) - 3 u.F)
// and carry the odd parts with opposite signs
//   g^eq: w rho 3 c.u,                             S: w k 3 c.F.
template <class Lat, class T>
__host__ __device__ __forceinline__ void collide_bgk(T g[Lat::Q], T rho, const T u[3],
                                                     const T F[3], const Par<T>& p) {
  const T uu = u[0] * u[0] + u[1] * u[1] + (Lat::DIM == 3 ? u[2] * u[2] : T(0));
  const T uF = u[0] * F[0] + u[1] * F[1] + (Lat::DIM == 3 ? u[2] * F[2] : T(0));
  const T drho = rho - p.rho0;
  const T keep = T(1) - p.inv_tau;  // g - (g - geq)/tau = keep g + geq/tau
  const T ev_eq = drho - T(1.5) * rho * uu;  // even part shared by every i
  const T ev_src = -T(3) * p.guo * uF;
#pragma unroll
  for (int i = 0; i < Lat::Q; i++) {
    const int j = Lat::opp(i);
    if (j < i) continue;  // handled with its partner
    const T w = T(Lat::w(i));
    T cu = T(Lat::c(i, 0)) * u[0] + T(Lat::c(i, 1)) * u[1];
    T cF = T(Lat::c(i, 0)) * F[0] + T(Lat::c(i, 1)) * F[1];
    if (Lat::DIM == 3) {
      cu += T(Lat::c(i, 2)) * u[2];
      cF += T(Lat::c(i, 2)) * F[2];
    }
    const T e_eq = w * (ev_eq + T(4.5) * rho * cu * cu);
    const T o_eq = w * T(3) * rho * cu;
    const T e_src = w * (ev_src + T(9) * p.guo * cF * cu);
    const T o_src = w * T(3) * p.guo * cF;
    const T gi = g[i];
    g[i] = keep * gi + (e_eq + o_eq) * p.inv_tau + (e_src + o_src);
    if (j != i) {
      const T gj = g[j];
      g[j] = keep * gj + (e_eq - o_eq) * p.inv_tau + (e_src - o_src);
    }
  }
}

// Multiple-relaxation-time collision with the source term in moment space
// (Sec. 1.2.1 names MRT; its rates are the caller's), on deviations:
//   y = g - g^eq + Ft/2,  g* = g + Ft - sum_k v_k a_k (v_k . y),
// with the moment rows v_k of lattice.cuh, a_k = s_k / |v_k|^2 (a[k]), and
// Ft_i = w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F the source term without its
// BGK prefactor.  Equal rates s_k = 1/tau give collide_bgk.  The conserved
// rows (mass, momentum) have v_k . y = 0 and are skipped.
template <class Lat, class T>
__host__ __device__ __forceinline__ void collide_mrt(T g[Lat::Q], T rho, const T u[3],
                                                     const T F[3], const Par<T>& p,
                                                     const T* a) {
  constexpr MomentBasis<Lat> B = make_moment_basis<Lat>();
  const T uu = u[0] * u[0] + u[1] * u[1] + (Lat::DIM == 3 ? u[2] * u[2] : T(0));
  const T uF = u[0] * F[0] + u[1] * F[1] + (Lat::DIM == 3 ? u[2] * F[2] : T(0));
  const T drho = rho - p.rho0;
  T y[Lat::Q], ft[Lat::Q];
#pragma unroll
  for (int i = 0; i < Lat::Q; i++) {
    T cu = T(Lat::c(i, 0)) * u[0] + T(Lat::c(i, 1)) * u[1];
    T cF = T(Lat::c(i, 0)) * F[0] + T(Lat::c(i, 1)) * F[1];
    if (Lat::DIM == 3) {
      cu += T(Lat::c(i, 2)) * u[2];
      cF += T(Lat::c(i, 2)) * F[2];
    }
    const T w = T(Lat::w(i));
    const T geq = w * (drho + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu));
    ft[i] = w * (T(3) * (cF - uF) + T(9) * cu * cF);
    y[i] = g[i] - geq + T(0.5) * ft[i];
  }
#pragma unroll
  for (int i = 0; i < Lat::Q; i++) g[i] += ft[i];
#pragma unroll
  for (int k = 0; k < Lat::Q; k++) {
    if (moment_conserved<Lat>(k)) continue;
    T m = T(0);
#pragma unroll
    for (int i = 0; i < Lat::Q; i++)
      if (B.v[k][i] != 0.0) m += T(B.v[k][i]) * y[i];
    m *= a[k];
#pragma unroll
    for (int i = 0; i < Lat::Q; i++)
      if (B.v[k][i] != 0.0) g[i] -= T(B.v[k][i]) * m;
  }
}

// rho = rho0 + sum g, u = (sum c g + F/2) / rho  (Eq. 6; sum c w rho0 = 0)
template <class Lat, class T>
__host__ __device__ __forceinline__ void moments(const T g[Lat::Q], const T F[3],
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

}  // namespace nlc
