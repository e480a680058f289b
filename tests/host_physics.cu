// Host build of the library's pointwise physics (csrc/physics.cuh) for CPU
// tests against the oracle.  Test infrastructure only: exposes plain C
// wrappers around the same templates the CUDA kernels instantiate.
#include "../paper_1907_13415_gb300/csrc/lattice.cuh"
#include "../paper_1907_13415_gb300/csrc/physics.cuh"

using namespace nlc;

static Par<double> par(const double* p) {
  Par<double> r;
  r.A0 = p[0]; r.K = p[1]; r.gamma = p[2]; r.Gamma = p[3]; r.xi = p[4]; r.tau = p[5];
  r.rho0 = 1.0; r.inv_tau = 1.0 / p[5]; r.guo = 1.0 - 0.5 / p[5];
  return r;
}

extern "C" {
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
void hp_be_rhs3(const double* q5, const double* dq15, const double* lap5, const double* u3,
                const double* G9, const double* p, double* r5) {
  double dq[3][5], G[3][3];
  for (int g = 0; g < 3; g++)
    for (int k = 0; k < 5; k++) dq[g][k] = dq15[5 * g + k];
  for (int k = 0; k < 9; k++) G[k / 3][k % 3] = G9[k];
  be_rhs<double, 3>(q5, dq, lap5, u3, G, par(p), r5);
}
}
