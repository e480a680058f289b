// adjoint_point.cuh -- reverse-mode (vector-Jacobian) products of the
// pointwise pieces in physics.cuh, written by hand.  Each *_vjp function
// takes the inputs of its forward function and the adjoint of its outputs,
// and ADDS the adjoints of its inputs to the given accumulators.
//
// Symmetric traceless tensors enter through their five stored components
// q = (xx, xy, xz, yy, yz), Q = [[q0, q1, q2], [q1, q3, q4], [q2, q4, -q0-q3]].
// The adjoint of a full 3x3 matrix Qbar maps back to the components as
//   qbar = (Qbar_xx - Qbar_zz, Qbar_xy + Qbar_yx, Qbar_xz + Qbar_zx,
//           Qbar_yy - Qbar_zz, Qbar_yz + Qbar_zy).
#pragma once
#include "lattice.cuh"
#include "physics.cuh"

namespace nlc {

// parameter adjoints accumulated by the VJPs (the gradient targets)
template <class T>
struct ParBar {
  T gamma, K, Gamma;
};

template <class T>
__host__ __device__ __forceinline__ void full_to_q5_add(const T M[3][3], T qb[5]) {
  qb[0] += M[0][0] - M[2][2];
  qb[1] += M[0][1] + M[1][0];
  qb[2] += M[0][2] + M[2][0];
  qb[3] += M[1][1] - M[2][2];
  qb[4] += M[1][2] + M[2][1];
}

// molecular_field: h = H(q, lap).  hb -> qb, lapb, (gamma, K)
template <class T>
__host__ __device__ __forceinline__ void molecular_field_vjp(const T q[5], const T lap[5],
                                                             const Par<T>& p, const T hb[5],
                                                             T qb[5], T lapb[5],
                                                             ParBar<T>& pb) {
  const T a = q[0], b = q[1], c = q[2], d = q[3], e = q[4], f = -q[0] - q[3];
  const T qq0 = a * a + b * b + c * c;
  const T qq1 = a * b + b * d + c * e;
  const T qq2 = a * c + b * e + c * f;
  const T qq3 = b * b + d * d + e * e;
  const T qq4 = b * c + d * e + e * f;
  const T tr2 = a * a + d * d + f * f + T(2) * (b * b + c * c + e * e);
  const T Ag = p.A0 * p.gamma;
  const T c1 = -p.A0 * (T(1) - p.gamma / T(3)) - Ag * tr2;
  // h_k = c1 q_k + Ag qq_k + c3 [k = xx, yy] + K lap_k, c3 = -Ag tr2 / 3
  const T c1b = hb[0] * a + hb[1] * b + hb[2] * c + hb[3] * d + hb[4] * e;
  const T c3b = hb[0] + hb[3];
  T Agb = hb[0] * qq0 + hb[1] * qq1 + hb[2] * qq2 + hb[3] * qq3 + hb[4] * qq4;
  Agb += -tr2 * c1b - tr2 / T(3) * c3b;
  const T tr2b = -Ag * c1b - Ag / T(3) * c3b;
  pb.gamma += p.A0 * Agb + p.A0 / T(3) * c1b;
  T Kb = T(0);
#pragma unroll
  for (int k = 0; k < 5; k++) {
    lapb[k] += p.K * hb[k];
    Kb += lap[k] * hb[k];
  }
  pb.K += Kb;
  const T g0 = Ag * hb[0], g1 = Ag * hb[1], g2 = Ag * hb[2], g3 = Ag * hb[3], g4 = Ag * hb[4];
  // qq2 = b e - c d and qq4 = b c - a e once f = -a - d is substituted
  qb[0] += c1 * hb[0] + g0 * T(2) * a + g1 * b - g4 * e + tr2b * (T(4) * a + T(2) * d);
  qb[1] += c1 * hb[1] + g0 * T(2) * b + g1 * (a + d) + g2 * e + g3 * T(2) * b + g4 * c +
           tr2b * T(4) * b;
  qb[2] += c1 * hb[2] + g0 * T(2) * c + g1 * e - g2 * d + g4 * b + tr2b * T(4) * c;
  qb[3] += c1 * hb[3] + g1 * b - g2 * c + g3 * T(2) * d + tr2b * (T(4) * d + T(2) * a);
  qb[4] += c1 * hb[4] + g1 * c + g2 * b + g3 * T(2) * e - g4 * a + tr2b * T(4) * e;
}

// stress (Eq. 5 without P0): Pi = Pi(q, h, dq).  Pib (a, b < DIM) ->
// qb, hb, dqb, (K)
template <class T, int DIM>
__host__ __device__ __forceinline__ void stress_vjp(const T q[5], const T h[5],
                                                    const T dq[3][5], const Par<T>& p,
                                                    const T Pib[3][3], T qb[5], T hb[5],
                                                    T dqb[3][5], ParBar<T>& pb) {
  const T Q[3][3] = {{q[0], q[1], q[2]}, {q[1], q[3], q[4]}, {q[2], q[4], -q[0] - q[3]}};
  const T H[3][3] = {{h[0], h[1], h[2]}, {h[1], h[3], h[4]}, {h[2], h[4], -h[0] - h[3]}};
  const T qh = Q[0][0] * H[0][0] + Q[1][1] * H[1][1] + Q[2][2] * H[2][2] +
               T(2) * (q[1] * h[1] + q[2] * h[2] + q[4] * h[4]);
  const T xm1 = p.xi - T(1), xp1 = p.xi + T(1), x23 = T(2) * p.xi / T(3);
  T Qb[3][3] = {}, Hb[3][3] = {}, Xb[3][3] = {};
  T qhb = T(0);
  T dQb[3][3][3] = {};  // [g][i][j]
#pragma unroll
  for (int a = 0; a < DIM; a++)
#pragma unroll
    for (int b = 0; b < DIM; b++) {
      const T w = Pib[a][b];
      const T qt = Q[a][b] + (a == b ? T(1) / T(3) : T(0));
      Qb[a][b] += T(2) * p.xi * qh * w;
      qhb += T(2) * p.xi * qt * w;
      Xb[a][b] += -xm1 * w;
      Xb[b][a] += -xp1 * w;
      Hb[a][b] += -x23 * w;
    }
  // qh = Q:H over nine entries
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      Qb[i][j] += qhb * H[i][j];
      Hb[i][j] += qhb * Q[i][j];
    }
  // X = Q H: Qb += Xb H^T, Hb += Q^T Xb
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      T s1 = T(0), s2 = T(0);
#pragma unroll
      for (int k = 0; k < 3; k++) {
        s1 += Xb[i][k] * H[j][k];
        s2 += Q[k][i] * Xb[k][j];
      }
      Qb[i][j] += s1;
      Hb[i][j] += s2;
    }
  // -K el_ab with el_ab = dQ_a : dQ_b (nine entries of each)
  T dQ[3][3][3];
#pragma unroll
  for (int g = 0; g < 3; g++) {
    dQ[g][0][0] = dq[g][0];
    dQ[g][0][1] = dQ[g][1][0] = dq[g][1];
    dQ[g][0][2] = dQ[g][2][0] = dq[g][2];
    dQ[g][1][1] = dq[g][3];
    dQ[g][1][2] = dQ[g][2][1] = dq[g][4];
    dQ[g][2][2] = -dq[g][0] - dq[g][3];
  }
  T Kb = T(0);
#pragma unroll
  for (int a = 0; a < DIM; a++)
#pragma unroll
    for (int b = 0; b < DIM; b++) {
      const T w = Pib[a][b];
      T el = T(0);
#pragma unroll
      for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
          el += dQ[a][i][j] * dQ[b][i][j];
          dQb[a][i][j] += -p.K * w * dQ[b][i][j];
          dQb[b][i][j] += -p.K * w * dQ[a][i][j];
        }
      Kb += -el * w;
    }
  pb.K += Kb;
  full_to_q5_add(Qb, qb);
  full_to_q5_add(Hb, hb);
#pragma unroll
  for (int g = 0; g < DIM; g++) full_to_q5_add(dQb[g], dqb[g]);
}

// co-rotational term: s = S(G, q).  sb -> Gb, qb
template <class T>
__host__ __device__ __forceinline__ void corotation_vjp(const T G[3][3], const T q[5], T xi,
                                                        const T sb[5], T Gb[3][3], T qb[5]) {
  const T Qt[3][3] = {{q[0] + T(1) / T(3), q[1], q[2]},
                      {q[1], q[3] + T(1) / T(3), q[4]},
                      {q[2], q[4], -q[0] - q[3] + T(1) / T(3)}};
  const T Q[3][3] = {{q[0], q[1], q[2]}, {q[1], q[3], q[4]}, {q[2], q[4], -q[0] - q[3]}};
  const T hp = (xi + T(1)) * T(0.5), hm = (xi - T(1)) * T(0.5);
  T M[3][3];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) M[a][b] = hp * G[a][b] + hm * G[b][a];
  T qg = T(0);
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) qg += Q[a][b] * G[a][b];
  // adjoint of the five outputs as a matrix (other entries are not outputs)
  T Sb[3][3] = {};
  Sb[0][0] = sb[0];
  Sb[0][1] = sb[1];
  Sb[0][2] = sb[2];
  Sb[1][1] = sb[3];
  Sb[1][2] = sb[4];
  // S = P + P^T - 2 xi Qt qg
  T Pb[3][3], Qtb[3][3];
  T qgb = T(0);
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) {
      Pb[a][b] = Sb[a][b] + Sb[b][a];
      Qtb[a][b] = -T(2) * xi * qg * Sb[a][b];
      qgb += -T(2) * xi * Qt[a][b] * Sb[a][b];
    }
  // P = M Qt: Mb = Pb Qt^T, Qtb += M^T Pb
  T Mb[3][3];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) {
      T s1 = T(0), s2 = T(0);
#pragma unroll
      for (int k = 0; k < 3; k++) {
        s1 += Pb[a][k] * Qt[b][k];
        s2 += M[k][a] * Pb[k][b];
      }
      Mb[a][b] = s1;
      Qtb[a][b] += s2;
    }
  // M = hp G + hm G^T; qg = Q:G
  T Qb[3][3];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) {
      Gb[a][b] += hp * Mb[a][b] + hm * Mb[b][a] + qgb * Q[a][b];
      Qb[a][b] = Qtb[a][b] + qgb * G[a][b];
    }
  full_to_q5_add(Qb, qb);
}

// right-hand side of Eq. 1: r = R(q, dq, lap, u, G).  rb -> qb, dqb, lapb,
// ub, Gb, (gamma, K, Gamma)
template <class T, int DIM>
__host__ __device__ __forceinline__ void be_rhs_vjp(const T q[5], const T dq[3][5],
                                                    const T lap[5], const T u[3],
                                                    const T G[3][3], const Par<T>& p,
                                                    const T rb[5], T qb[5], T dqb[3][5],
                                                    T lapb[5], T ub[3], T Gb[3][3],
                                                    ParBar<T>& pb) {
  // r_k = -u_g dq_g,k + s_k + Gamma h_k - [k in {xx, yy}] 2 xi tr(G) / 9
  T h[5];
  molecular_field(q, lap, p, h);
  T hb[5], Gam = T(0);
#pragma unroll
  for (int k = 0; k < 5; k++) {
    hb[k] = p.Gamma * rb[k];
    Gam += h[k] * rb[k];
  }
  pb.Gamma += Gam;
#pragma unroll
  for (int g = 0; g < DIM; g++) {
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 5; k++) {
      s += dq[g][k] * rb[k];
      dqb[g][k] += -u[g] * rb[k];
    }
    ub[g] += -s;
  }
  const T tb = -T(2) * p.xi / T(9) * (rb[0] + rb[3]);
  Gb[0][0] += tb;
  Gb[1][1] += tb;
  Gb[2][2] += tb;
  corotation_vjp(G, q, p.xi, rb, Gb, qb);
  molecular_field_vjp(q, lap, p, hb, qb, lapb, pb);
}

// BGK collision with the source term (collide_bgk): g' = C(g, rho, u, F).
// gb (adjoint of the post-collision g', overwritten with the adjoint of the
// pre-collision g) -> rhob, ub, Fb
template <class Lat, class T>
__host__ __device__ __forceinline__ void collide_bgk_vjp(T gb[Lat::Q], T rho, const T u[3],
                                                         const T F[3], const Par<T>& p,
                                                         T& rhob, T ub[3], T Fb[3]) {
  const T uu = u[0] * u[0] + u[1] * u[1] + (Lat::DIM == 3 ? u[2] * u[2] : T(0));
  const T keep = T(1) - p.inv_tau;
  T ev_eqb = T(0), ev_srcb = T(0);
#pragma unroll
  for (int i = 0; i < Lat::Q; i++) {
    const int j = Lat::opp(i);
    if (j < i) continue;
    const T w = T(Lat::w(i));
    T cu = T(Lat::c(i, 0)) * u[0] + T(Lat::c(i, 1)) * u[1];
    T cF = T(Lat::c(i, 0)) * F[0] + T(Lat::c(i, 1)) * F[1];
    if (Lat::DIM == 3) {
      cu += T(Lat::c(i, 2)) * u[2];
      cF += T(Lat::c(i, 2)) * F[2];
    }
    const T bi = gb[i];
    const T bj = j != i ? gb[j] : T(0);
    // g_i' = keep g_i + (e_eq + o_eq)/tau + e_src + o_src; g_j' with odd parts negated
    const T e_eqb = (bi + bj) * p.inv_tau, o_eqb = (bi - bj) * p.inv_tau;
    const T e_srcb = bi + bj, o_srcb = bi - bj;
    gb[i] = keep * bi;
    if (j != i) gb[j] = keep * bj;
    // e_eq = w (ev_eq + 4.5 rho cu^2); o_eq = 3 w rho cu
    ev_eqb += w * e_eqb;
    rhob += T(4.5) * w * cu * cu * e_eqb + T(3) * w * cu * o_eqb;
    T cub = T(9) * w * rho * cu * e_eqb + T(3) * w * rho * o_eqb;
    // e_src = w (ev_src + 9 guo cF cu); o_src = 3 w guo cF
    ev_srcb += w * e_srcb;
    const T cFb = T(9) * w * p.guo * cu * e_srcb + T(3) * w * p.guo * o_srcb;
    cub += T(9) * w * p.guo * cF * e_srcb;
#pragma unroll
    for (int a = 0; a < Lat::DIM; a++) {
      ub[a] += T(Lat::c(i, a)) * cub;
      Fb[a] += T(Lat::c(i, a)) * cFb;
    }
  }
  // ev_eq = (rho - rho0) - 1.5 rho uu; ev_src = -3 guo u.F
  rhob += ev_eqb * (T(1) - T(1.5) * uu);
#pragma unroll
  for (int a = 0; a < Lat::DIM; a++) {
    ub[a] += -T(3) * rho * u[a] * ev_eqb - T(3) * p.guo * F[a] * ev_srcb;
    Fb[a] += -T(3) * p.guo * u[a] * ev_srcb;
  }
}

// moments (Eq. 6): rho = rho0 + sum g, u = (sum c g + F/2)/rho.
// rhob, ub -> gb (added), Fb (added)
template <class Lat, class T>
__host__ __device__ __forceinline__ void moments_vjp(T rho, const T u[3], T rhob,
                                                     const T ub[3], T gb[Lat::Q], T Fb[3]) {
  T mb[3] = {T(0), T(0), T(0)};
  T rb = rhob;
#pragma unroll
  for (int a = 0; a < Lat::DIM; a++) {
    mb[a] = ub[a] / rho;
    Fb[a] += ub[a] / (T(2) * rho);
    rb += -u[a] * ub[a] / rho;
  }
#pragma unroll
  for (int i = 0; i < Lat::Q; i++) {
    T s = rb;
#pragma unroll
    for (int a = 0; a < Lat::DIM; a++) s += T(Lat::c(i, a)) * mb[a];
    gb[i] += s;
  }
}

}  // namespace nlc
