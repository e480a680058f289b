// physics.cuh -- pointwise pieces of the hybrid step, templated on the
// arithmetic type T (float or double) and the dimension.
//
// Notation follows Sec. 1.1: Q the order tensor (symmetric, traceless, five
// stored components xx, xy, xz, yy, yz with Qzz = -Qxx - Qyy), H the
// molecular field (Eq. 3), Pi the stress of Eq. 5 without P0, S the
// co-rotational term of Eq. 1, G[a][b] = d_b u_a the velocity gradient.
#pragma once

namespace nlc {

template <class T>
struct Par {
  T A0, K, gamma, Gamma, xi, tau, rho0;
  T inv_tau;  // 1/tau
  T guo;      // 1 - 1/(2 tau), the prefactor of the source term
};

// five stored components -> full symmetric traceless 3x3
template <class T>
__device__ __forceinline__ void q_full(const T q[5], T Q[3][3]) {
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

// Eq. 3: H = -A0(1-g/3) Q - A0 g (Tr(Q^2) I/3 - Q Q) - A0 g Q Tr(Q^2) + K lapQ
// (returned as the five independent components; H is symmetric traceless)
template <class T>
__device__ __forceinline__ void molecular_field(const T q[5], const T lap[5],
                                                const Par<T>& p, T h[5]) {
  T Q[3][3];
  q_full(q, Q);
  T QQ[3][3];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++)
      QQ[a][b] = Q[a][0] * Q[0][b] + Q[a][1] * Q[1][b] + Q[a][2] * Q[2][b];
  const T tr2 = QQ[0][0] + QQ[1][1] + QQ[2][2];
  const T c1 = -p.A0 * (T(1) - p.gamma / T(3)) - p.A0 * p.gamma * tr2;
  const T c2 = p.A0 * p.gamma;
  const T c3 = -p.A0 * p.gamma * tr2 / T(3);
  h[0] = c1 * Q[0][0] + c2 * QQ[0][0] + c3 + p.K * lap[0];
  h[1] = c1 * Q[0][1] + c2 * QQ[0][1] + p.K * lap[1];
  h[2] = c1 * Q[0][2] + c2 * QQ[0][2] + p.K * lap[2];
  h[3] = c1 * Q[1][1] + c2 * QQ[1][1] + c3 + p.K * lap[3];
  h[4] = c1 * Q[1][2] + c2 * QQ[1][2] + p.K * lap[4];
}

// Eq. 5 without P0, with dF/d(d_b Q) = K d_b Q:
//   Pi_ab = 2 xi Qt_ab (Q:H) - xi (H Qt)_ab - xi (Qt H)_ab
//           - K d_a Q : d_b Q + (Q H)_ab - (H Q)_ab,      Qt = Q + I/3.
// dq[g][k]: d_g of stored component k.  Only a, b < DIM are produced.
template <class T, int DIM>
__device__ __forceinline__ void stress(const T q[5], const T h[5],
                                       const T dq[3][5], const Par<T>& p,
                                       T Pi[3][3]) {
  T Q[3][3], H[3][3];
  q_full(q, Q);
  q_full(h, H);
  T QH[3][3];  // (Q H); since Q, H are symmetric, H Q = (Q H)^T
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++)
      QH[a][b] = Q[a][0] * H[0][b] + Q[a][1] * H[1][b] + Q[a][2] * H[2][b];
  const T qh = QH[0][0] + QH[1][1] + QH[2][2];  // Q:H
  // d_a Q : d_b Q over all nine entries (off-diagonals twice, Qzz included)
  T el[3][3];
#pragma unroll
  for (int a = 0; a < DIM; a++)
#pragma unroll
    for (int b = 0; b < DIM; b++) {
      if (b < a) {
        el[a][b] = el[b][a];
        continue;
      }
      const T zza = -dq[a][0] - dq[a][3], zzb = -dq[b][0] - dq[b][3];
      el[a][b] = dq[a][0] * dq[b][0] + dq[a][3] * dq[b][3] + zza * zzb +
                 T(2) * (dq[a][1] * dq[b][1] + dq[a][2] * dq[b][2] +
                         dq[a][4] * dq[b][4]);
    }
#pragma unroll
  for (int a = 0; a < DIM; a++)
#pragma unroll
    for (int b = 0; b < DIM; b++) {
      const T qt = Q[a][b] + (a == b ? T(1) / T(3) : T(0));
      // H Qt = H Q + H/3 = (QH)^T + H/3 ; Qt H = QH + H/3
      const T HQt = QH[b][a] + H[a][b] * (T(1) / T(3));
      const T QtH = QH[a][b] + H[a][b] * (T(1) / T(3));
      Pi[a][b] = T(2) * p.xi * qt * qh - p.xi * HQt - p.xi * QtH -
                 p.K * el[a][b] + QH[a][b] - QH[b][a];
    }
}

// Co-rotational term of Eq. 1:
//   S = (xi D + W) Qt + Qt (xi D - W) - 2 xi Qt (Q_ge d_g u_e)
//   W_ab = (d_b u_a - d_a u_b)/2, D_ab = (d_b u_a + d_a u_b)/2.
// G[a][b] = d_b u_a.  Writes the five stored components of S.
template <class T>
__device__ __forceinline__ void corotation(const T G[3][3], const T q[5],
                                           T xi, T s[5]) {
  T Q[3][3];
  q_full(q, Q);
  T L[3][3], R[3][3], Qt[3][3];
  T qgu = T(0);
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const T W = (G[a][b] - G[b][a]) * T(0.5);
      const T D = (G[a][b] + G[b][a]) * T(0.5);
      L[a][b] = xi * D + W;
      R[a][b] = xi * D - W;
      Qt[a][b] = Q[a][b] + (a == b ? T(1) / T(3) : T(0));
      qgu += Q[a][b] * G[b][a];
    }
  constexpr int ia[5] = {0, 0, 0, 1, 1};
  constexpr int ib[5] = {0, 1, 2, 1, 2};
#pragma unroll
  for (int k = 0; k < 5; k++) {
    const int a = ia[k], b = ib[k];
    T v = T(0);
#pragma unroll
    for (int g = 0; g < 3; g++) v += L[a][g] * Qt[g][b] + Qt[a][g] * R[g][b];
    s[k] = v - T(2) * xi * Qt[a][b] * qgu;
  }
}

// Right-hand side of Eq. 1 at one cell,
//   R = -u_g d_g Q + S(W, D, Q) + Gamma H,
// made traceless by the orthogonal projection R <- R - Tr(R)/3 I.  The
// advection and H terms are traceless, and for traceless Q the trace of S is
// 2 xi div(u)/3 identically, so Tr(R) = 2 xi (G_xx + G_yy + G_zz)/3.
// Inputs: q (5), its central first derivatives dq[g][k], its Laplacian
// lap[k], u (3), G.
template <class T, int DIM>
__device__ __forceinline__ void be_rhs(const T q[5], const T dq[3][5],
                                       const T lap[5], const T u[3],
                                       const T G[3][3], const Par<T>& p,
                                       T r[5]) {
  T h[5], s[5];
  molecular_field(q, lap, p, h);
  corotation(G, q, p.xi, s);
  T adv[5];
#pragma unroll
  for (int k = 0; k < 5; k++) {
    T a = u[0] * dq[0][k] + u[1] * dq[1][k];
    if (DIM == 3) a += u[2] * dq[2][k];
    adv[k] = a;
  }
  const T tr3 = T(2) * p.xi * (G[0][0] + G[1][1] + G[2][2]) / T(9);
  const T rxx = -adv[0] + s[0] + p.Gamma * h[0];
  const T ryy = -adv[3] + s[3] + p.Gamma * h[3];
  r[0] = rxx - tr3;
  r[1] = -adv[1] + s[1] + p.Gamma * h[1];
  r[2] = -adv[2] + s[2] + p.Gamma * h[2];
  r[3] = ryy - tr3;
  r[4] = -adv[4] + s[4] + p.Gamma * h[4];
}

// Equilibrium deviation g^eq_i = f^eq_i - w_i rho0, with
// f^eq_i = rho w_i [1 + c.u/cs2 + (c.u)^2/(2 cs2^2) - u^2/(2 cs2)] (Sec. 1.2.1)
// and the BGK source term
// S_i = w_i (1 - 1/2tau) [c_i/cs2 (1 + c_i.u/cs2) - u/cs2] . F.
template <class Lat, class T>
__device__ __forceinline__ void collide_bgk(T g[Lat::Q], T rho, const T u[3],
                                            const T F[3], const Par<T>& p) {
  const T uu = u[0] * u[0] + u[1] * u[1] + (Lat::DIM == 3 ? u[2] * u[2] : T(0));
  const T uF = u[0] * F[0] + u[1] * F[1] + (Lat::DIM == 3 ? u[2] * F[2] : T(0));
  const T drho = rho - p.rho0;
#pragma unroll
  for (int i = 0; i < Lat::Q; i++) {
    const T w = T(Lat::w(i));
    T cu = T(Lat::c(i, 0)) * u[0] + T(Lat::c(i, 1)) * u[1];
    T cF = T(Lat::c(i, 0)) * F[0] + T(Lat::c(i, 1)) * F[1];
    if (Lat::DIM == 3) {
      cu += T(Lat::c(i, 2)) * u[2];
      cF += T(Lat::c(i, 2)) * F[2];
    }
    const T geq = w * (drho + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu));
    const T src = w * p.guo * (T(3) * cF * (T(1) + T(3) * cu) - T(3) * uF);
    g[i] = g[i] - (g[i] - geq) * p.inv_tau + src;
  }
}

}  // namespace nlc
