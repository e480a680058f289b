// Exact floating-point operation counts of the library's pointwise physics
// (csrc/physics.cuh), by running the same templates on an op-counting scalar
// on the host.  Test and measurement infrastructure: prints one JSON object.
// An FMA counts as two operations; comparisons and moves count nothing.
// Built as plain C++ (g++ -x c++) with the CUDA qualifiers defined away.
#include <cmath>
#include <cstdio>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

struct OC;
static long g_ops = 0;
struct OC {
  double v;
  OC() : v(0) {}
  OC(double x) : v(x) {}
};
inline OC operator+(OC a, OC b) { g_ops++; return OC(a.v + b.v); }
inline OC operator-(OC a, OC b) { g_ops++; return OC(a.v - b.v); }
inline OC operator*(OC a, OC b) { g_ops++; return OC(a.v * b.v); }
inline OC operator/(OC a, OC b) { g_ops++; return OC(a.v / b.v); }
inline OC operator-(OC a) { return OC(-a.v); }
inline OC& operator+=(OC& a, OC b) { return a = a + b; }
inline OC& operator-=(OC& a, OC b) { return a = a - b; }
inline OC& operator*=(OC& a, OC b) { return a = a * b; }
inline bool operator!=(OC a, double b) { return a.v != b; }

namespace nlc {
inline OC fma_(OC a, OC b, OC c) { g_ops += 2; return OC(a.v * b.v + c.v); }
}  // namespace nlc

#include "../paper_1907_13415_gb300/csrc/lattice.cuh"
#include "../paper_1907_13415_gb300/csrc/physics.cuh"

using namespace nlc;

int main() {
  Par<OC> p;
  p.A0 = 0.1; p.K = 0.02; p.gamma = 2.7; p.Gamma = 0.3; p.xi = 0.7; p.tau = 1.0;
  p.rho0 = 1.0;
  derive(p);
  OC q[5] = {0.1, 0.02, 0.01, -0.05, 0.03}, lap[5] = {1e-3, 2e-3, 3e-3, 4e-3, 5e-3};
  OC dq[3][5], G[3][3], u[3] = {1e-3, 2e-3, 3e-3}, F[3] = {1e-5, 2e-5, 3e-5}, h[5], s[5],
     r[5], P[3][3], adv[5];
  for (int a = 0; a < 3; a++) {
    for (int k = 0; k < 5; k++) dq[a][k] = 1e-3 * (a + k + 1);
    for (int b = 0; b < 3; b++) G[a][b] = 1e-4 * (a - b + 0.5);
  }
  long c;
  printf("{");
  g_ops = 0; molecular_field(q, lap, p, h); printf("\"H\": %ld", g_ops);
  g_ops = 0; stress<OC, 3>(q, h, dq, p, P); printf(", \"Pi_3d\": %ld", g_ops);
  g_ops = 0; stress<OC, 2>(q, h, dq, p, P); printf(", \"Pi_2d\": %ld", g_ops);
  g_ops = 0; corotation(G, q, p.hp, p.hm, p.x2, s); printf(", \"S\": %ld", g_ops);
  g_ops = 0; be_rhs_adv(q, adv, lap, G, p, r); printf(", \"R_from_adv\": %ld", g_ops);
  OC g19[19], g9[9], rho;
  for (int i = 0; i < 19; i++) g19[i] = 1e-3 * i;
  for (int i = 0; i < 9; i++) g9[i] = 1e-3 * i;
  g_ops = 0; moments<LatD3Q19, OC>(g19, F, p, rho, u); printf(", \"moments_d3q19\": %ld", g_ops);
  g_ops = 0; collide_bgk<LatD3Q19, OC>(g19, rho, u, F, p); printf(", \"bgk_d3q19\": %ld", g_ops);
  g_ops = 0; moments<LatD2Q9, OC>(g9, F, p, rho, u); printf(", \"moments_d2q9\": %ld", g_ops);
  g_ops = 0; collide_bgk<LatD2Q9, OC>(g9, rho, u, F, p); printf(", \"bgk_d2q9\": %ld", g_ops);
  OC a19[19], a9[9];
  for (int k = 0; k < 19; k++) a19[k] = 0.1;
  for (int k = 0; k < 9; k++) a9[k] = 0.1;
  g_ops = 0; collide_mrt<LatD3Q19, OC>(g19, rho, u, F, p, a19); printf(", \"mrt_d3q19\": %ld", g_ops);
  g_ops = 0; collide_mrt<LatD2Q9, OC>(g9, rho, u, F, p, a9); printf(", \"mrt_d2q9\": %ld", g_ops);
  (void)c;
  printf("}\n");
  return 0;
}
