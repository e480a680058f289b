// Host build of the library's pointwise physics (csrc/physics.cuh) for CPU
// tests against the oracle.  Test infrastructure only: exposes plain C
// wrappers around the same templates the CUDA kernels instantiate.
#include <complex>

namespace nlc {
// complex-step twin of the fused multiply-add the physics templates use
inline std::complex<double> fma_(std::complex<double> a, std::complex<double> b,
                                 std::complex<double> c) {
  return a * b + c;
}
}  // namespace nlc

#include "../paper_1907_13415_gb300/csrc/lattice.cuh"
#include "../paper_1907_13415_gb300/csrc/physics.cuh"
#include "../paper_1907_13415_gb300/csrc/aux_kernels.cuh"

using namespace nlc;

static Par<double> par(const double* p) {
  Par<double> r;
  r.A0 = p[0]; r.K = p[1]; r.gamma = p[2]; r.Gamma = p[3]; r.xi = p[4]; r.tau = p[5];
  r.rho0 = 1.0;
  derive(r);
  return r;
}

extern "C" {
// the float-float running sum of the observables over v[0..n) (and of the
// products a_i b_i with add_prod), read out in float64
double hp_accff_sum(const float* v, int n) {
  AccFF a;
  for (int i = 0; i < n; i++) a.add(v[i]);
  return a.value();
}
double hp_accff_dot(const float* x, const float* y, int n) {
  AccFF a;
  for (int i = 0; i < n; i++) a.add_prod(x[i], y[i]);
  return a.value();
}
// the FP32 gradient contraction of the stress (packed pairs)
float hp_grad_dot_f32(const float* A5, const float* B5) { return grad_dot(A5, B5); }
void hp_molecular_field(const double* q5, const double* lap5, const double* p, double* h5) {
  molecular_field<double>(q5, lap5, par(p), h5);
}
void hp_stress3(const double* q5, const double* h5, const double* dq15, const double* p,
                double* pi9) {
  double dq[3][5], P[3][3];
  for (int g = 0; g < 3; g++)
    for (int k = 0; k < 5; k++) dq[g][k] = dq15[5 * g + k];
  stress<double, 3>(q5, h5, dq, par(p), P);
  for (int k = 0; k < 9; k++) pi9[k] = P[k / 3][k % 3];
}
void hp_corotation(const double* G9, const double* q5, double xi, double* s5) {
  double G[3][3];
  for (int k = 0; k < 9; k++) G[k / 3][k % 3] = G9[k];
  corotation<double>(G, q5, xi, s5);
}
// BGK collision with the source term on deviations g (rho0 = 1)
int hp_collide(int lattice, double* g, double rho, const double* u, const double* F,
               const double* p) {
  Par<double> pp = par(p);
  double uu[3] = {u[0], u[1], u[2]}, FF[3] = {F[0], F[1], F[2]};
  if (lattice == 0) {
    collide_bgk<LatD2Q9, double>(g, rho, uu, FF, pp);
    return 9;
  }
  collide_bgk<LatD3Q19, double>(g, rho, uu, FF, pp);
  return 19;
}
}  // extern "C"

// the FP32 kernels' moments and BGK + source collision on packed opposite
// pairs (packed.cuh) for deviations g in the library's velocity order
// (rho0 = 1): g is replaced by the post-collision deviations, rho and u
// (Eq. 6, with F/2) are returned in ru[0..3]
template <class Lat>
static void lb_pairs_f32(float* g, const float* F, const double* p, float* ru) {
  constexpr int NP = (Lat::Q - 1) / 2;
  Par<float> pf;
  pf.A0 = float(p[0]); pf.K = float(p[1]); pf.gamma = float(p[2]); pf.Gamma = float(p[3]);
  pf.xi = float(p[4]); pf.tau = float(p[5]); pf.rho0 = 1.0f;
  derive(pf);
  float g0 = g[0];
  float2 gp[NP];
  for (int q = 0; q < NP; q++) {
    const int i = pair_first<Lat>(q);
    gp[q] = make_float2(g[i], g[Lat::opp(i)]);
  }
  float rho, drho, u[3];
  moments_pairs<Lat>(g0, gp, F, pf.rho0, rho, drho, u);
  collide_bgk_pairs<Lat>(g0, gp, rho, drho, u, F, pf.inv_tau, pf.guo);
  g[0] = g0;
  for (int q = 0; q < NP; q++) {
    const int i = pair_first<Lat>(q);
    g[i] = gp[q].x;
    g[Lat::opp(i)] = gp[q].y;
  }
  ru[0] = rho;
  for (int a = 0; a < 3; a++) ru[1 + a] = u[a];
}
extern "C" {
int hp_lb_pairs_f32(int lattice, float* g, const float* F, const double* p, float* ru) {
  if (lattice == 0) {
    lb_pairs_f32<LatD2Q9>(g, F, p, ru);
    return 9;
  }
  lb_pairs_f32<LatD3Q19>(g, F, p, ru);
  return 19;
}
// MRT collision with the source term on deviations g (rho0 = 1); a[k] are
// the per-moment coefficients s_k / |v_k|^2 (filled here from rates s_k)
int hp_collide_mrt(int lattice, double* g, double rho, const double* u, const double* F,
                   const double* p, const double* rates) {
  Par<double> pp = par(p);
  double uu[3] = {u[0], u[1], u[2]}, FF[3] = {F[0], F[1], F[2]}, a[19];
  if (lattice == 0) {
    constexpr MomentBasis<LatD2Q9> B = make_moment_basis<LatD2Q9>();
    for (int k = 0; k < 9; k++) a[k] = rates[k] / B.n2[k];
    collide_mrt<LatD2Q9, double>(g, rho, uu, FF, pp, a);
    return 9;
  }
  constexpr MomentBasis<LatD3Q19> B = make_moment_basis<LatD3Q19>();
  for (int k = 0; k < 19; k++) a[k] = rates[k] / B.n2[k];
  collide_mrt<LatD3Q19, double>(g, rho, uu, FF, pp, a);
  return 19;
}
// the library's moment rows v[k * q + i] in its own velocity order
int hp_moment_basis(int lattice, double* v) {
  if (lattice == 0) {
    constexpr MomentBasis<LatD2Q9> B = make_moment_basis<LatD2Q9>();
    for (int k = 0; k < 9; k++)
      for (int i = 0; i < 9; i++) v[k * 9 + i] = B.v[k][i];
    return 9;
  }
  constexpr MomentBasis<LatD3Q19> B = make_moment_basis<LatD3Q19>();
  for (int k = 0; k < 19; k++)
    for (int i = 0; i < 19; i++) v[k * 19 + i] = B.v[k][i];
  return 19;
}
void hp_lattice(int lattice, int* c, double* w) {
  const int q = lattice == 0 ? 9 : 19;
  for (int i = 0; i < q; i++) {
    for (int a = 0; a < 3; a++) c[3 * i + a] = lattice == 0 ? LatD2Q9::c(i, a) : LatD3Q19::c(i, a);
    w[i] = lattice == 0 ? LatD2Q9::w(i) : LatD3Q19::w(i);
  }
}
void hp_be_rhs3(const double* q5, const double* dq15, const double* lap5, const double* u3,
                const double* G9, const double* p, double* r5) {
  double dq[3][5], G[3][3];
  for (int g = 0; g < 3; g++)
    for (int k = 0; k < 5; k++) dq[g][k] = dq15[5 * g + k];
  for (int k = 0; k < 9; k++) G[k / 3][k % 3] = G9[k];
  be_rhs<double, 3>(q5, dq, lap5, u3, G, par(p), r5);
}
}

// ---------------------------------------------------------------------------
// Adjoint checks: flat-array forms of each pointwise piece, evaluated in
// complex arithmetic for complex-step directional derivatives, and the
// hand-written vector-Jacobian products of csrc/adjoint_point.cuh.
// ---------------------------------------------------------------------------
#include <complex>

#include "../paper_1907_13415_gb300/csrc/adjoint_point.cuh"

using cplx = std::complex<double>;

template <class T>
static Par<T> parT(const T* p) {
  Par<T> r;
  r.A0 = p[0]; r.K = p[1]; r.gamma = p[2]; r.Gamma = p[3]; r.xi = p[4]; r.tau = p[5];
  r.rho0 = T(1.0);
  derive(r);
  return r;
}

// piece 0: molecular field.  in: q5 lap5 | out: h5
// piece 1: stress (3D).       in: q5 h5 dq15 | out: Pi9
// piece 2: corotation.        in: G9 q5 | out: s5
// piece 3: be_rhs (3D).       in: q5 dq15 lap5 u3 G9 | out: r5
// piece 4: lb cell D2Q9.      in: g9 F3 | out: g'9 u3   (moments + collision)
// piece 5: lb cell D3Q19.     in: g19 F3 | out: g'19 u3
template <class T>
static void piece(int k, const T* in, const T* p, T* out) {
  Par<T> pp = parT(p);
  if (k == 0) {
    molecular_field<T>(in, in + 5, pp, out);
  } else if (k == 1) {
    T dq[3][5], P[3][3];
    for (int g = 0; g < 3; g++)
      for (int c = 0; c < 5; c++) dq[g][c] = in[10 + 5 * g + c];
    stress<T, 3>(in, in + 5, dq, pp, P);
    for (int c = 0; c < 9; c++) out[c] = P[c / 3][c % 3];
  } else if (k == 2) {
    T G[3][3];
    for (int c = 0; c < 9; c++) G[c / 3][c % 3] = in[c];
    corotation<T>(G, in + 9, pp.xi, out);
  } else if (k == 3) {
    T dq[3][5], G[3][3];
    for (int g = 0; g < 3; g++)
      for (int c = 0; c < 5; c++) dq[g][c] = in[5 + 5 * g + c];
    for (int c = 0; c < 9; c++) G[c / 3][c % 3] = in[28 + c];
    be_rhs<T, 3>(in, dq, in + 20, in + 25, G, pp, out);
  } else if (k == 4 || k == 5) {
    const int q = k == 4 ? 9 : 19;
    T g[19], F[3] = {in[q], in[q + 1], k == 4 ? T(0) : in[q + 2]}, rho, u[3];
    for (int i = 0; i < q; i++) g[i] = in[i];
    if (k == 4) {
      moments<LatD2Q9, T>(g, F, pp, rho, u);
      collide_bgk<LatD2Q9, T>(g, rho, u, F, pp);
    } else {
      moments<LatD3Q19, T>(g, F, pp, rho, u);
      collide_bgk<LatD3Q19, T>(g, rho, u, F, pp);
    }
    for (int i = 0; i < q; i++) out[i] = g[i];
    for (int a = 0; a < 3; a++) out[q + a] = u[a];
  }
}

extern "C" {
// complex-step directional derivative: out_dir = J(in, p) [v_in, v_p]
void hp_piece_jvp(int k, const double* in, int nin, const double* p, const double* vin,
                  const double* vp, int nout, double* out_dir) {
  const double h = 1e-30;
  cplx ci[64], cp[6], co[64];
  for (int i = 0; i < nin; i++) ci[i] = cplx(in[i], h * vin[i]);
  for (int i = 0; i < 6; i++) cp[i] = cplx(p[i], h * vp[i]);
  piece<cplx>(k, ci, cp, co);
  for (int i = 0; i < nout; i++) out_dir[i] = co[i].imag() / h;
}

// hand-written adjoint: given the output adjoint ob, returns the input
// adjoint ib and the adjoints of (gamma, K, Gamma) in pb
void hp_piece_vjp(int k, const double* in, const double* p, const double* ob, double* ib,
                  double* pbo) {
  Par<double> pp = parT(p);
  ParBar<double> pb{0, 0, 0};
  if (k == 0) {
    for (int i = 0; i < 10; i++) ib[i] = 0;
    molecular_field_vjp<double>(in, in + 5, pp, ob, ib, ib + 5, pb);
  } else if (k == 1) {
    double dq[3][5], Pb[3][3], dqb[3][5] = {}, hb[5] = {}, qb[5] = {};
    for (int g = 0; g < 3; g++)
      for (int c = 0; c < 5; c++) dq[g][c] = in[10 + 5 * g + c];
    for (int c = 0; c < 9; c++) Pb[c / 3][c % 3] = ob[c];
    stress_vjp<double, 3>(in, in + 5, dq, pp, Pb, qb, hb, dqb, pb);
    for (int c = 0; c < 5; c++) {
      ib[c] = qb[c];
      ib[5 + c] = hb[c];
    }
    for (int g = 0; g < 3; g++)
      for (int c = 0; c < 5; c++) ib[10 + 5 * g + c] = dqb[g][c];
  } else if (k == 2) {
    double G[3][3], Gb[3][3] = {}, qb[5] = {};
    for (int c = 0; c < 9; c++) G[c / 3][c % 3] = in[c];
    corotation_vjp<double>(G, in + 9, pp.xi, ob, Gb, qb);
    for (int c = 0; c < 9; c++) ib[c] = Gb[c / 3][c % 3];
    for (int c = 0; c < 5; c++) ib[9 + c] = qb[c];
  } else if (k == 3) {
    double dq[3][5], G[3][3], qb[5] = {}, dqb[3][5] = {}, lapb[5] = {}, ub[3] = {},
                              Gb[3][3] = {};
    for (int g = 0; g < 3; g++)
      for (int c = 0; c < 5; c++) dq[g][c] = in[5 + 5 * g + c];
    for (int c = 0; c < 9; c++) G[c / 3][c % 3] = in[28 + c];
    be_rhs_vjp<double, 3>(in, dq, in + 20, in + 25, G, pp, ob, qb, dqb, lapb, ub, Gb, pb);
    for (int c = 0; c < 5; c++) ib[c] = qb[c];
    for (int g = 0; g < 3; g++)
      for (int c = 0; c < 5; c++) ib[5 + 5 * g + c] = dqb[g][c];
    for (int c = 0; c < 5; c++) ib[20 + c] = lapb[c];
    for (int a = 0; a < 3; a++) ib[25 + a] = ub[a];
    for (int c = 0; c < 9; c++) ib[28 + c] = Gb[c / 3][c % 3];
  } else if (k == 4 || k == 5) {
    const int q = k == 4 ? 9 : 19;
    double g[19], F[3] = {in[q], in[q + 1], k == 4 ? 0.0 : in[q + 2]}, rho, u[3];
    for (int i = 0; i < q; i++) g[i] = in[i];
    double gb[19], rhob = 0, ub[3] = {ob[q], ob[q + 1], k == 4 ? 0.0 : ob[q + 2]},
                   Fb[3] = {0, 0, 0};
    for (int i = 0; i < q; i++) gb[i] = ob[i];
    if (k == 4) {
      moments<LatD2Q9, double>(g, F, pp, rho, u);
      collide_bgk_vjp<LatD2Q9, double>(gb, rho, u, F, pp, rhob, ub, Fb);
      moments_vjp<LatD2Q9, double>(rho, u, rhob, ub, gb, Fb);
    } else {
      moments<LatD3Q19, double>(g, F, pp, rho, u);
      collide_bgk_vjp<LatD3Q19, double>(gb, rho, u, F, pp, rhob, ub, Fb);
      moments_vjp<LatD3Q19, double>(rho, u, rhob, ub, gb, Fb);
    }
    for (int i = 0; i < q; i++) ib[i] = gb[i];
    for (int a = 0; a < (k == 4 ? 2 : 3); a++) ib[q + a] = Fb[a];
  }
  pbo[0] = pb.gamma;
  pbo[1] = pb.K;
  pbo[2] = pb.Gamma;
}
}
