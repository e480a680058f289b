/*
 * nlc_oracle.c -- plain FP64 CPU oracle of the hybrid lattice-Boltzmann /
 * finite-difference Beris-Edwards time step of Coelho, Araujo & Telo da Gama,
 * "Lattice-Boltzmann simulation of free nematic-isotropic interfaces"
 * (arxiv 1907.13415), Sec. 1.1 (Eqs. 1-5) and Sec. 1.2 (LB update, Eq. 6,
 * BGK source term, predictor-corrector finite differences).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the
 * CUDA library and the timed CPU baseline.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it; the product path never
 * does.  It shares no code, table or header with the CUDA path.
 *
 * Everything is written per cell in the order of the paper's equations, with
 * no blocking, fusion or reordering.  The same source is compiled twice:
 *   - as real FP64 (functions orc_*), and
 *   - with ORC_COMPLEX defined, as complex FP64 (functions orc_*_cs), so that
 *     the complex-step method (Squire & Trapp, SIAM Rev. 40, 1998) gives
 *     derivatives of any output with respect to any input exact to rounding:
 *     d/dp L(p) = Im L(p + i h) / h with h = 1e-30.  Every operation used in
 *     the step is analytic (+, -, *, /, sqrt of a value with positive real
 *     part), so this holds for the whole time integration.
 *
 * Readings of points the paper leaves open (each one is also listed in the
 * design notes of the repository):
 *   R1  Within one step, the force F^n and the velocity u^n come from the
 *       state (f^n, Q^n); the LB update and both Beris-Edwards evaluations of
 *       the predictor-corrector use that same u^n (and its gradient).
 *   R2  Collision is BGK with the single relaxation time tau (Sec. 1.2.1 gives
 *       the source term in its BGK form; the MRT matrices are not given).
 *       orc_set_mrt switches to a multiple-relaxation-time collision on an
 *       orthogonal moment basis with caller-given rates (see collide_mrt);
 *       with all rates 1/tau it is the BGK step.
 *   R3  The Laplacian is the standard 2d+1-point second-order stencil; first
 *       derivatives (including the advection term and grad u) are central.
 *       orc_set_stencil(1) switches every finite difference to the
 *       isotropic stencils of the lattice's neighbour set (q_grad_lap).
 *   R4  The right-hand side of Eq. 1 is made traceless by the orthogonal
 *       projection R <- R - (Tr R / 3) I before the five independent
 *       components (xx, xy, xz, yy, yz) are stored; Qzz = -Qxx - Qyy.
 *   R5  On the 2D lattice (D2Q9, nz = 1) the out-of-plane force F_z is dropped
 *       and u_z = 0; all five Q components still evolve.
 *   R6  The scalar order parameter is S = sqrt(3/2 Tr Q^2) (exact for a
 *       uniaxial Q = S(nn - I/3), Sec. 1.1).
 *   R7  The velocity used in Eq. 1 is the "actual" one, rho u = sum c f + F/2
 *       (Eq. 6), held fixed over the predictor and the corrector.
 *
 * Storage: structure of arrays, cell index c = x + nx*(y + ny*z), x fastest.
 *   f  [q][N]  pre-collision populations f_i(x, t) at time n
 *   Q5 [5][N]  independent components (xx, xy, xz, yy, yz)
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORC_COMPLEX
typedef double _Complex rt;
#define RSQRT(v) csqrt(v)
#define RPOW(v, e) cpow(v, e)
#define RE(v) creal(v)
#define API(name) name##_cs
#else
typedef double rt;
#define RSQRT(v) sqrt(v)
#define RPOW(v, e) pow(v, e)
#define RE(v) (v)
#define API(name) name
#endif

/* ------------------------------------------------------------------ */
/* Lattices (Sec. 1.2.1).  D2Q9 for the 2D runs, D3Q19 as in the paper.   */
/* c_s^2 = 1/3 for both.                                                */
/* ------------------------------------------------------------------ */
#define ORC_D2Q9 0
#define ORC_D3Q19 1

static const int VEL2[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const double WGT2[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                               1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                               1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static const int VEL3[19][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
    {0, 0, 1},   {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
    {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};
static const double WGT3[19] = {
    1.0 / 3.0,  1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static const double CS2 = 1.0 / 3.0;

static int nvel(int lattice) { return lattice == ORC_D2Q9 ? 9 : 19; }
static const int (*vel(int lattice))[3] {
  return lattice == ORC_D2Q9 ? VEL2 : VEL3;
}
static const double *wgt(int lattice) {
  return lattice == ORC_D2Q9 ? WGT2 : WGT3;
}

/* Parameter vector: A0, K, gamma, Gamma, xi, tau (Sec. 2 lists the set). */
enum { P_A0 = 0, P_K, P_GAMMA, P_GAMMA_ROT, P_XI, P_TAU, NPARAM };

typedef struct {
  int lattice, nx, ny, nz;
  long n;
} grid_t;

static int grid_ok(int lattice, int nx, int ny, int nz, grid_t *g) {
  if (lattice != ORC_D2Q9 && lattice != ORC_D3Q19) return 0;
  if (nx < 1 || ny < 1 || nz < 1) return 0;
  if (lattice == ORC_D2Q9 && nz != 1) return 0;
  g->lattice = lattice;
  g->nx = nx;
  g->ny = ny;
  g->nz = nz;
  g->n = (long)nx * ny * nz;
  return 1;
}

/* periodic wrap (Sec. 2: periodic boundaries in every direction) */
static int wrap(int v, int n) { return ((v % n) + n) % n; }

static long cell_at(const grid_t *g, int x, int y, int z) {
  return (long)wrap(x, g->nx) +
         (long)g->nx * ((long)wrap(y, g->ny) + (long)g->ny * wrap(z, g->nz));
}

static void coords(const grid_t *g, long c, int *x, int *y, int *z) {
  *x = (int)(c % g->nx);
  *y = (int)((c / g->nx) % g->ny);
  *z = (int)(c / ((long)g->nx * g->ny));
}

static long neighbour(const grid_t *g, long c, int dx, int dy, int dz) {
  int x, y, z;
  coords(g, c, &x, &y, &z);
  return cell_at(g, x + dx, y + dy, z + dz);
}

static const int UNIT[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

/* The full 3x3 Q from its five stored components; Qzz = -Qxx - Qyy. */
static void q_full(const rt *Q5, long N, long c, rt Q[3][3]) {
  rt xx = Q5[0 * N + c], xy = Q5[1 * N + c], xz = Q5[2 * N + c];
  rt yy = Q5[3 * N + c], yz = Q5[4 * N + c];
  Q[0][0] = xx;
  Q[0][1] = xy;
  Q[0][2] = xz;
  Q[1][0] = xy;
  Q[1][1] = yy;
  Q[1][2] = yz;
  Q[2][0] = xz;
  Q[2][1] = yz;
  Q[2][2] = -xx - yy;
}

static void q_store(rt *Q5, long N, long c, rt Q[3][3]) {
  Q5[0 * N + c] = Q[0][0];
  Q5[1 * N + c] = Q[0][1];
  Q5[2 * N + c] = Q[0][2];
  Q5[3 * N + c] = Q[1][1];
  Q5[4 * N + c] = Q[1][2];
}

static void matmul(rt A[3][3], rt B[3][3], rt C[3][3]) {
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      rt s = 0;
      for (int k = 0; k < 3; k++) s += A[a][k] * B[k][b];
      C[a][b] = s;
    }
}

static rt ddot(rt A[3][3], rt B[3][3]) {
  rt s = 0;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) s += A[a][b] * B[a][b];
  return s;
}

/* ------------------------------------------------------------------ */
/* Finite differences (Sec. 1.2.2): central first derivative, and the     */
/* 2d+1-point Laplacian (reading R3).                                    */
/* dQ[g][a][b] = d_g Q_ab.                                               */
/* ------------------------------------------------------------------ */
/* Finite-difference stencils.  Standard (reading R3): central first
 * derivatives and the 2d+1-point Laplacian.  Isotropic (orc_set_stencil(1)):
 * the lattice's own neighbour set and weights (9 points on D2Q9, 19 on
 * D3Q19), d_a phi = (1/cs^2) sum_i w_i c_ia phi(x + c_i) and
 * lap phi = (2/cs^2) sum_i w_i [phi(x + c_i) - phi(x)], both second order
 * with a leading error that does not depend on direction. */
static int iso_stencil = 0;

int API(orc_set_stencil)(int kind) {
  if (kind != 0 && kind != 1) return -1;
  iso_stencil = kind;
  return 0;
}

static void q_grad_lap(const grid_t *g, const rt *Q5, long c, rt dQ[3][3][3],
                       rt lap[3][3]) {
  rt Q0[3][3];
  q_full(Q5, g->n, c, Q0);
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) lap[a][b] = 0;
  if (iso_stencil) {
    int q = nvel(g->lattice);
    const int(*cv)[3] = vel(g->lattice);
    const double *w = wgt(g->lattice);
    for (int gdir = 0; gdir < 3; gdir++)
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) dQ[gdir][a][b] = 0;
    for (int i = 1; i < q; i++) {
      rt Qi[3][3];
      q_full(Q5, g->n, neighbour(g, c, cv[i][0], cv[i][1], cv[i][2]), Qi);
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
          for (int gdir = 0; gdir < 3; gdir++)
            dQ[gdir][a][b] += w[i] * cv[i][gdir] * Qi[a][b] / CS2;
          lap[a][b] += 2.0 * w[i] * (Qi[a][b] - Q0[a][b]) / CS2;
        }
    }
    return;
  }
  for (int gdir = 0; gdir < 3; gdir++) {
    rt Qp[3][3], Qm[3][3];
    long cp = neighbour(g, c, UNIT[gdir][0], UNIT[gdir][1], UNIT[gdir][2]);
    long cm = neighbour(g, c, -UNIT[gdir][0], -UNIT[gdir][1], -UNIT[gdir][2]);
    q_full(Q5, g->n, cp, Qp);
    q_full(Q5, g->n, cm, Qm);
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        dQ[gdir][a][b] = (Qp[a][b] - Qm[a][b]) / 2.0;
        lap[a][b] += Qp[a][b] + Qm[a][b] - 2.0 * Q0[a][b];
      }
  }
}

/* ------------------------------------------------------------------ */
/* Molecular field, Eq. 3:                                               */
/*  H = -A0(1-gamma/3) Q - A0 gamma (Tr(Q^2) I/3 - Q Q^T)                 */
/*      - A0 gamma Q Tr(Q^2) + K lap Q                                   */
/* ------------------------------------------------------------------ */
static void molecular_field(rt Q[3][3], rt lap[3][3], const rt *p,
                            rt H[3][3]) {
  rt A0 = p[P_A0], gam = p[P_GAMMA], K = p[P_K];
  rt QQ[3][3];
  matmul(Q, Q, QQ); /* Q symmetric: Q_ag Q_bg = (Q Q)_ab */
  rt trq2 = ddot(Q, Q);
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      rt delta = (a == b) ? 1.0 : 0.0;
      H[a][b] = -A0 * (1.0 - gam / 3.0) * Q[a][b] -
                A0 * gam * (trq2 * delta / 3.0 - QQ[a][b]) -
                A0 * gam * Q[a][b] * trq2 + K * lap[a][b];
    }
}

/* ------------------------------------------------------------------ */
/* Stress without the hydrostatic part, Eq. 5 with P0 removed (the force  */
/* of Sec. 1.2.1 is the divergence of Pi + P0 delta), and with            */
/* dF/d(d_b Q_gn) = K d_b Q_gn substituted:                               */
/*  Pi'_ab = 2 xi (Q_ab + d_ab/3) Q_ge H_ge - xi H_ag (Q_gb + d_gb/3)       */
/*         - xi (Q_ag + d_ag/3) H_gb - K d_a Q_gn d_b Q_gn                 */
/*         + Q_ag H_gb - H_ag Q_gb                                        */
/* ------------------------------------------------------------------ */
static void stress(rt Q[3][3], rt H[3][3], rt dQ[3][3][3], rt K, rt xi,
                   rt Pi[3][3]) {
  rt Qt[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) Qt[a][b] = Q[a][b] + ((a == b) ? 1.0 / 3.0 : 0.0);
  rt QH = ddot(Q, H);
  rt HQt[3][3], QtH[3][3], QHm[3][3], HQm[3][3];
  matmul(H, Qt, HQt);
  matmul(Qt, H, QtH);
  matmul(Q, H, QHm);
  matmul(H, Q, HQm);
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      rt elastic = 0;
      for (int gg = 0; gg < 3; gg++)
        for (int nn = 0; nn < 3; nn++) elastic += dQ[a][gg][nn] * dQ[b][gg][nn];
      Pi[a][b] = 2.0 * xi * Qt[a][b] * QH - xi * HQt[a][b] - xi * QtH[a][b] -
                 K * elastic + QHm[a][b] - HQm[a][b];
    }
}

/* ------------------------------------------------------------------ */
/* Co-rotational term of Eq. 1 (Eq. 2 of Sec. 1.1).  Gu[a][b] = d_b u_a.  */
/*  W_ab = (d_b u_a - d_a u_b)/2,  D_ab = (d_b u_a + d_a u_b)/2            */
/*  S = (xi D + W)(Q + I/3) + (Q + I/3)(xi D - W)                          */
/*      - 2 xi (Q + I/3) (Q_ge d_g u_e)                                    */
/* ------------------------------------------------------------------ */
static void corotation(rt Gu[3][3], rt Q[3][3], rt xi, rt S[3][3]) {
  rt Wm[3][3], Dm[3][3], Qt[3][3], Lm[3][3], Rm[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      Wm[a][b] = (Gu[a][b] - Gu[b][a]) / 2.0;
      Dm[a][b] = (Gu[a][b] + Gu[b][a]) / 2.0;
      Qt[a][b] = Q[a][b] + ((a == b) ? 1.0 / 3.0 : 0.0);
    }
  rt qgu = 0; /* Q_ge d_g u_e */
  for (int gg = 0; gg < 3; gg++)
    for (int e = 0; e < 3; e++) qgu += Q[gg][e] * Gu[e][gg];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      Lm[a][b] = xi * Dm[a][b] + Wm[a][b];
      Rm[a][b] = xi * Dm[a][b] - Wm[a][b];
    }
  rt A[3][3], B[3][3];
  matmul(Lm, Qt, A);
  matmul(Qt, Rm, B);
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++)
      S[a][b] = A[a][b] + B[a][b] - 2.0 * xi * Qt[a][b] * qgu;
}

/* ------------------------------------------------------------------ */
/* Equilibrium (second-order Hermite, Sec. 1.2.1) and BGK source term.    */
/* ------------------------------------------------------------------ */
static void equilibrium(int lattice, rt rho, const rt u[3], rt *feq) {
  int q = nvel(lattice);
  const int(*cv)[3] = vel(lattice);
  const double *w = wgt(lattice);
  rt uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < q; i++) {
    rt cu = cv[i][0] * u[0] + cv[i][1] * u[1] + cv[i][2] * u[2];
    feq[i] = rho * w[i] *
             (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
  }
}

/* S_i = w_i (1 - 1/(2 tau)) [ c_i/cs^2 (1 + c_i.u/cs^2) - u/cs^2 ] . F */
static void guo_source(int lattice, rt tau, const rt u[3], const rt F[3],
                       rt *src) {
  int q = nvel(lattice);
  const int(*cv)[3] = vel(lattice);
  const double *w = wgt(lattice);
  for (int i = 0; i < q; i++) {
    rt cu = cv[i][0] * u[0] + cv[i][1] * u[1] + cv[i][2] * u[2];
    rt s = 0;
    for (int a = 0; a < 3; a++)
      s += (cv[i][a] / CS2 * (1.0 + cu / CS2) - u[a] / CS2) * F[a];
    src[i] = w[i] * (1.0 - 1.0 / (2.0 * tau)) * s;
  }
}

/* ------------------------------------------------------------------ */
/* Multiple-relaxation-time collision (Sec. 1.2.1 names MRT as the       */
/* operator used; its matrices and rates are not given, so the rates are */
/* the caller's).  Moment space: the polynomials below, evaluated on the */
/* lattice velocities and made orthogonal by Gram-Schmidt with unit      */
/* weights in the listed order, rows v_k.  With S = diag(s_k) and the    */
/* force term without its BGK prefactor,                                 */
/*   Ft_i = w_i [c_i/cs^2 (1 + c_i.u/cs^2) - u/cs^2] . F,                 */
/* the post-collision populations are                                   */
/*   f* = f - M^-1 S M (f - feq + Ft/2) + Ft,                            */
/* i.e. f - sum_k v_k s_k (v_k . y)/(v_k . v_k) + Ft with y = f - feq +   */
/* Ft/2.  With every s_k = 1/tau this is the BGK step with its source    */
/* term.  Moments, D2Q9: 1, c^2, c^4, cx, c^2 cx, cy, c^2 cy,            */
/* cx^2 - cy^2, cx cy.  D3Q19: 1, c^2, c^4, cx, c^2 cx, cy, c^2 cy, cz,    */
/* c^2 cz, 3cx^2 - c^2, (3cx^2 - c^2) c^2, cy^2 - cz^2,                   */
/* (cy^2 - cz^2) c^2, cx cy, cy cz, cx cz, cx (cy^2 - cz^2),              */
/* cy (cz^2 - cx^2), cz (cx^2 - cy^2).                                    */
/* ------------------------------------------------------------------ */
static double moment_poly(int lattice, int k, const int cv[3]) {
  double x = cv[0], y = cv[1], z = cv[2], c2 = x * x + y * y + z * z;
  if (lattice == ORC_D2Q9) {
    switch (k) {
      case 0: return 1.0;
      case 1: return c2;
      case 2: return c2 * c2;
      case 3: return x;
      case 4: return c2 * x;
      case 5: return y;
      case 6: return c2 * y;
      case 7: return x * x - y * y;
      default: return x * y;
    }
  }
  switch (k) {
    case 0: return 1.0;
    case 1: return c2;
    case 2: return c2 * c2;
    case 3: return x;
    case 4: return c2 * x;
    case 5: return y;
    case 6: return c2 * y;
    case 7: return z;
    case 8: return c2 * z;
    case 9: return 3.0 * x * x - c2;
    case 10: return (3.0 * x * x - c2) * c2;
    case 11: return y * y - z * z;
    case 12: return (y * y - z * z) * c2;
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return x * (y * y - z * z);
    case 17: return y * (z * z - x * x);
    default: return z * (x * x - y * y);
  }
}

static int mrt_on = 0;
static double mrt_rate[19];
static double mrt_v[19][19];   /* orthogonal rows v_k[i] */
static double mrt_n2[19];      /* v_k . v_k */

static void mrt_basis(int lattice) {
  int q = nvel(lattice);
  const int(*cv)[3] = vel(lattice);
  for (int k = 0; k < q; k++) {
    for (int i = 0; i < q; i++) mrt_v[k][i] = moment_poly(lattice, k, cv[i]);
    for (int j = 0; j < k; j++) {
      double d = 0.0;
      for (int i = 0; i < q; i++) d += mrt_v[k][i] * mrt_v[j][i];
      for (int i = 0; i < q; i++) mrt_v[k][i] -= d / mrt_n2[j] * mrt_v[j][i];
    }
    mrt_n2[k] = 0.0;
    for (int i = 0; i < q; i++) mrt_n2[k] += mrt_v[k][i] * mrt_v[k][i];
  }
}

/* rates: q relaxation rates in the moment order above (those of the
 * conserved moments, 1 and c, have no effect), or NULL for BGK. */
int API(orc_set_mrt)(int lattice, const double *rates) {
  if (!rates) {
    mrt_on = 0;
    return 0;
  }
  if (lattice != ORC_D2Q9 && lattice != ORC_D3Q19) return -1;
  mrt_basis(lattice);
  for (int k = 0; k < nvel(lattice); k++) mrt_rate[k] = rates[k];
  mrt_on = lattice + 1;
  return 0;
}

/* Ft_i: the force term of Sec. 1.2.1 without the factor (1 - 1/(2 tau)) */
static void force_term(int lattice, const rt u[3], const rt F[3], rt *ft) {
  int q = nvel(lattice);
  const int(*cv)[3] = vel(lattice);
  const double *w = wgt(lattice);
  for (int i = 0; i < q; i++) {
    rt cu = cv[i][0] * u[0] + cv[i][1] * u[1] + cv[i][2] * u[2];
    rt s = 0;
    for (int a = 0; a < 3; a++)
      s += (cv[i][a] / CS2 * (1.0 + cu / CS2) - u[a] / CS2) * F[a];
    ft[i] = w[i] * s;
  }
}

static void collide_mrt(int lattice, const rt *f, const rt *feq, const rt *ft,
                        rt *post) {
  int q = nvel(lattice);
  rt y[19];
  for (int i = 0; i < q; i++) y[i] = f[i] - feq[i] + ft[i] / 2.0;
  for (int i = 0; i < q; i++) post[i] = f[i] + ft[i];
  for (int k = 0; k < q; k++) {
    rt m = 0;
    for (int i = 0; i < q; i++) m += mrt_v[k][i] * y[i];
    rt a = mrt_rate[k] * m / mrt_n2[k];
    for (int i = 0; i < q; i++) post[i] -= mrt_v[k][i] * a;
  }
}

/* ------------------------------------------------------------------ */
/* Whole-lattice stages.                                                  */
/* ------------------------------------------------------------------ */

/* H (5 comps) and Pi' (9 comps) at every cell from Q. */
static void stage_fields(const grid_t *g, const rt *p, const rt *Q5, rt *H5,
                         rt *Pi9) {
  long N = g->n;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < N; c++) {
    rt Q[3][3], dQ[3][3][3], lap[3][3], H[3][3];
    q_full(Q5, N, c, Q);
    q_grad_lap(g, Q5, c, dQ, lap);
    molecular_field(Q, lap, p, H);
    if (H5) q_store(H5, N, c, H);
    if (Pi9) {
      rt Pi[3][3];
      stress(Q, H, dQ, p[P_K], p[P_XI], Pi);
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) Pi9[(3 * a + b) * N + c] = Pi[a][b];
    }
  }
}

/* F_a = d_b Pi'_ab by central differences (Sec. 1.2.1, Sec. 1.2.2);
 * reading R5 drops F_z on the 2D lattice. */
static void stage_force(const grid_t *g, const rt *Pi9, rt *F3) {
  long N = g->n;
  int q = nvel(g->lattice);
  const int(*cv)[3] = vel(g->lattice);
  const double *w = wgt(g->lattice);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < N; c++) {
    for (int a = 0; a < 3; a++) {
      rt s = 0;
      if (iso_stencil) {
        for (int i = 1; i < q; i++) {
          long ci = neighbour(g, c, cv[i][0], cv[i][1], cv[i][2]);
          for (int b = 0; b < 3; b++)
            s += w[i] * cv[i][b] * Pi9[(3 * a + b) * N + ci] / CS2;
        }
      } else {
        for (int b = 0; b < 3; b++) {
          long cp = neighbour(g, c, UNIT[b][0], UNIT[b][1], UNIT[b][2]);
          long cm = neighbour(g, c, -UNIT[b][0], -UNIT[b][1], -UNIT[b][2]);
          s += (Pi9[(3 * a + b) * N + cp] - Pi9[(3 * a + b) * N + cm]) / 2.0;
        }
      }
      F3[a * N + c] = s;
    }
    if (g->lattice == ORC_D2Q9) F3[2 * N + c] = 0;
  }
}

/* rho = sum f_i, rho u = sum c_i f_i + F/2  (Eq. 6). */
static void stage_moments(const grid_t *g, const rt *f, const rt *F3, rt *rho,
                          rt *u3) {
  long N = g->n;
  int q = nvel(g->lattice);
  const int(*cv)[3] = vel(g->lattice);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < N; c++) {
    rt r = 0, m[3] = {0, 0, 0};
    for (int i = 0; i < q; i++) {
      r += f[i * N + c];
      for (int a = 0; a < 3; a++) m[a] += cv[i][a] * f[i * N + c];
    }
    rho[c] = r;
    for (int a = 0; a < 3; a++) u3[a * N + c] = (m[a] + F3[a * N + c] / 2.0) / r;
  }
}

/* BGK (or, after orc_set_mrt for this lattice, MRT) collision with the   */
/* source term, then streaming f_i(x + c_i, t + 1) = f*_i(x).             */
static void stage_collide_stream(const grid_t *g, const rt *p, const rt *f,
                                 const rt *rho, const rt *u3, const rt *F3,
                                 rt *fnew) {
  long N = g->n;
  int q = nvel(g->lattice);
  const int(*cv)[3] = vel(g->lattice);
  rt tau = p[P_TAU];
#pragma omp parallel for schedule(static)
  for (long c = 0; c < N; c++) {
    rt u[3] = {u3[0 * N + c], u3[1 * N + c], u3[2 * N + c]};
    rt F[3] = {F3[0 * N + c], F3[1 * N + c], F3[2 * N + c]};
    rt feq[19], src[19], fc[19], post[19];
    equilibrium(g->lattice, rho[c], u, feq);
    if (mrt_on == g->lattice + 1) {
      force_term(g->lattice, u, F, src);
      for (int i = 0; i < q; i++) fc[i] = f[i * N + c];
      collide_mrt(g->lattice, fc, feq, src, post);
    } else {
      guo_source(g->lattice, tau, u, F, src);
      for (int i = 0; i < q; i++) {
        rt fi = f[i * N + c];
        post[i] = fi - (fi - feq[i]) / tau + src[i];
      }
    }
    for (int i = 0; i < q; i++)
      fnew[i * N + neighbour(g, c, cv[i][0], cv[i][1], cv[i][2])] = post[i];
  }
}

/* Velocity gradient Gu[a][b] = d_b u_a by central differences. */
static void vel_grad(const grid_t *g, const rt *u3, long c, rt Gu[3][3]) {
  long N = g->n;
  if (iso_stencil) {
    int q = nvel(g->lattice);
    const int(*cv)[3] = vel(g->lattice);
    const double *w = wgt(g->lattice);
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) Gu[a][b] = 0;
    for (int i = 1; i < q; i++) {
      long ci = neighbour(g, c, cv[i][0], cv[i][1], cv[i][2]);
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) Gu[a][b] += w[i] * cv[i][b] * u3[a * N + ci] / CS2;
    }
    return;
  }
  for (int b = 0; b < 3; b++) {
    long cp = neighbour(g, c, UNIT[b][0], UNIT[b][1], UNIT[b][2]);
    long cm = neighbour(g, c, -UNIT[b][0], -UNIT[b][1], -UNIT[b][2]);
    for (int a = 0; a < 3; a++)
      Gu[a][b] = (u3[a * N + cp] - u3[a * N + cm]) / 2.0;
  }
}

/* Right-hand side of Eq. 1, R = -u.grad Q + S(W, D, Q) + Gamma H, made
 * traceless by the orthogonal projection (reading R4). */
static void stage_rhs(const grid_t *g, const rt *p, const rt *Q5,
                      const rt *u3, rt *R5) {
  long N = g->n;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < N; c++) {
    rt Q[3][3], dQ[3][3][3], lap[3][3], H[3][3], Gu[3][3], S[3][3], R[3][3];
    q_full(Q5, N, c, Q);
    q_grad_lap(g, Q5, c, dQ, lap);
    molecular_field(Q, lap, p, H);
    vel_grad(g, u3, c, Gu);
    corotation(Gu, Q, p[P_XI], S);
    rt u[3] = {u3[0 * N + c], u3[1 * N + c], u3[2 * N + c]};
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        rt adv = 0;
        for (int gg = 0; gg < 3; gg++) adv += u[gg] * dQ[gg][a][b];
        R[a][b] = -adv + S[a][b] + p[P_GAMMA_ROT] * H[a][b];
      }
    rt tr = R[0][0] + R[1][1] + R[2][2];
    for (int a = 0; a < 3; a++) R[a][a] -= tr / 3.0;
    q_store(R5, N, c, R);
  }
}

/* ------------------------------------------------------------------ */
/* Exported API                                                           */
/* ------------------------------------------------------------------ */

int API(orc_lattice)(int lattice, int *c_out, double *w_out) {
  if (lattice != ORC_D2Q9 && lattice != ORC_D3Q19) return -1;
  int q = nvel(lattice);
  const int(*cv)[3] = vel(lattice);
  const double *w = wgt(lattice);
  for (int i = 0; i < q; i++) {
    for (int a = 0; a < 3; a++) c_out[3 * i + a] = cv[i][a];
    w_out[i] = w[i];
  }
  return q;
}

/* Pointwise pieces, exported for the pin tests.  All 3x3 arrays row-major. */
void API(orc_molecular_field_point)(const rt *Q9, const rt *lap9, const rt *p,
                                    rt *H9) {
  rt Q[3][3], L[3][3], H[3][3];
  for (int k = 0; k < 9; k++) {
    Q[k / 3][k % 3] = Q9[k];
    L[k / 3][k % 3] = lap9[k];
  }
  molecular_field(Q, L, p, H);
  for (int k = 0; k < 9; k++) H9[k] = H[k / 3][k % 3];
}

void API(orc_stress_point)(const rt *Q9, const rt *H9, const rt *dQ27, rt K,
                           rt xi, rt *Pi9) {
  rt Q[3][3], H[3][3], dQ[3][3][3], Pi[3][3];
  for (int k = 0; k < 9; k++) {
    Q[k / 3][k % 3] = Q9[k];
    H[k / 3][k % 3] = H9[k];
  }
  for (int k = 0; k < 27; k++) dQ[k / 9][(k / 3) % 3][k % 3] = dQ27[k];
  stress(Q, H, dQ, K, xi, Pi);
  for (int k = 0; k < 9; k++) Pi9[k] = Pi[k / 3][k % 3];
}

void API(orc_corotation_point)(const rt *Gu9, const rt *Q9, rt xi, rt *S9) {
  rt G[3][3], Q[3][3], S[3][3];
  for (int k = 0; k < 9; k++) {
    G[k / 3][k % 3] = Gu9[k];
    Q[k / 3][k % 3] = Q9[k];
  }
  corotation(G, Q, xi, S);
  for (int k = 0; k < 9; k++) S9[k] = S[k / 3][k % 3];
}

void API(orc_equilibrium_point)(int lattice, rt rho, const rt *u, rt *feq) {
  equilibrium(lattice, rho, u, feq);
}

/* one MRT collision at a point (after orc_set_mrt): post from f, rho, u, F */
int API(orc_mrt_point)(int lattice, const rt *f, rt rho, const rt *u, const rt *F,
                       rt *post) {
  if (mrt_on != lattice + 1) return -1;
  rt feq[19], ft[19];
  equilibrium(lattice, rho, u, feq);
  force_term(lattice, u, F, ft);
  collide_mrt(lattice, f, feq, ft, post);
  return 0;
}

/* the orthogonal moment rows after orc_set_mrt: v[k * q + i] */
int API(orc_mrt_basis)(int lattice, double *v) {
  if (mrt_on != lattice + 1) return -1;
  int q = nvel(lattice);
  for (int k = 0; k < q; k++)
    for (int i = 0; i < q; i++) v[k * q + i] = mrt_v[k][i];
  return q;
}

void API(orc_guo_point)(int lattice, rt tau, const rt *u, const rt *F,
                        rt *src) {
  guo_source(lattice, tau, u, F, src);
}

/* f_i = f^eq_i(rho, u) at every cell (rho, u may be NULL: 1 and 0). */
int API(orc_init_equilibrium)(int lattice, int nx, int ny, int nz,
                              const rt *rho, const rt *u3, rt *f) {
  grid_t g;
  if (!grid_ok(lattice, nx, ny, nz, &g)) return -1;
  long N = g.n;
  int q = nvel(lattice);
  for (long c = 0; c < N; c++) {
    rt u[3] = {0, 0, 0}, feq[19];
    if (u3)
      for (int a = 0; a < 3; a++) u[a] = u3[a * N + c];
    if (lattice == ORC_D2Q9) u[2] = 0;
    equilibrium(lattice, rho ? rho[c] : 1.0, u, feq);
    for (int i = 0; i < q; i++) f[i * N + c] = feq[i];
  }
  return 0;
}

/* Intermediates at the current state: H (5N), Pi' (9N, [a][b] row-major
 * planes), F (3N), rho (N), u (3N).  Any output may be NULL. */
int API(orc_fields)(int lattice, int nx, int ny, int nz, const rt *p,
                    const rt *f, const rt *Q5, rt *H5, rt *Pi9, rt *F3,
                    rt *rho, rt *u3) {
  grid_t g;
  if (!grid_ok(lattice, nx, ny, nz, &g)) return -1;
  long N = g.n;
  rt *pi = (rt *)malloc(sizeof(rt) * 9 * N);
  rt *ff = (rt *)malloc(sizeof(rt) * 3 * N);
  rt *rr = (rt *)malloc(sizeof(rt) * N);
  rt *uu = (rt *)malloc(sizeof(rt) * 3 * N);
  if (!pi || !ff || !rr || !uu) {
    free(pi);
    free(ff);
    free(rr);
    free(uu);
    return -2;
  }
  stage_fields(&g, p, Q5, H5, pi);
  stage_force(&g, pi, ff);
  stage_moments(&g, f, ff, rr, uu);
  if (Pi9) memcpy(Pi9, pi, sizeof(rt) * 9 * N);
  if (F3) memcpy(F3, ff, sizeof(rt) * 3 * N);
  if (rho) memcpy(rho, rr, sizeof(rt) * N);
  if (u3) memcpy(u3, uu, sizeof(rt) * 3 * N);
  free(pi);
  free(ff);
  free(rr);
  free(uu);
  return 0;
}

/* Right-hand side R(Q) of Eq. 1 for a given Q and velocity field u. */
int API(orc_rhs)(int lattice, int nx, int ny, int nz, const rt *p,
                 const rt *Q5, const rt *u3, rt *R5) {
  grid_t g;
  if (!grid_ok(lattice, nx, ny, nz, &g)) return -1;
  stage_rhs(&g, p, Q5, u3, R5);
  return 0;
}

/* Advance (f, Q) by nsteps time steps, in place. */
int API(orc_step)(int lattice, int nx, int ny, int nz, const rt *p, rt *f,
                  rt *Q5, long nsteps) {
  grid_t g;
  if (!grid_ok(lattice, nx, ny, nz, &g)) return -1;
  long N = g.n;
  int q = nvel(lattice);
  rt *pi = (rt *)malloc(sizeof(rt) * 9 * N);
  rt *F3 = (rt *)malloc(sizeof(rt) * 3 * N);
  rt *rho = (rt *)malloc(sizeof(rt) * N);
  rt *u3 = (rt *)malloc(sizeof(rt) * 3 * N);
  rt *fnew = (rt *)malloc(sizeof(rt) * q * N);
  rt *R1 = (rt *)malloc(sizeof(rt) * 5 * N);
  rt *R2 = (rt *)malloc(sizeof(rt) * 5 * N);
  rt *QP = (rt *)malloc(sizeof(rt) * 5 * N);
  int rc = 0;
  if (!pi || !F3 || !rho || !u3 || !fnew || !R1 || !R2 || !QP) {
    rc = -2;
    goto done;
  }
  for (long s = 0; s < nsteps; s++) {
    /* force and velocity at time n from (f^n, Q^n)  (reading R1) */
    stage_fields(&g, p, Q5, NULL, pi);
    stage_force(&g, pi, F3);
    stage_moments(&g, f, F3, rho, u3);
    /* lattice Boltzmann: collide and stream */
    stage_collide_stream(&g, p, f, rho, u3, F3, fnew);
    /* Beris-Edwards, predictor-corrector (Sec. 1.2.2 steps 1-5) */
    stage_rhs(&g, p, Q5, u3, R1);                          /* step 1 */
    for (long k = 0; k < 5 * N; k++) QP[k] = Q5[k] + R1[k]; /* step 2 */
    stage_rhs(&g, p, QP, u3, R2);                          /* step 3 */
    for (long k = 0; k < 5 * N; k++)
      Q5[k] = Q5[k] + (R1[k] + R2[k]) / 2.0;               /* steps 4-5 */
    memcpy(f, fnew, sizeof(rt) * q * N);
  }
done:
  free(pi);
  free(F3);
  free(rho);
  free(u3);
  free(fnew);
  free(R1);
  free(R2);
  free(QP);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Observables.  out[] layout (10 values):                               */
/*  0 mass = sum rho          1-3 momentum sum rho u (with F/2, Eq. 6)    */
/*  4 s_area = sum S / s_ref  5 radius (2D: sqrt(A/pi); 3D: (3A/4pi)^1/3) */
/*  6 x_iface (first descending crossing of the y,z-mean of S through    */
/*    s_ref/2, linear interpolation)                                     */
/*  7 max |u|                 8 free energy (Eq. 2, forward-difference   */
/*    gradient term)          9 number of non-finite values in f and Q   */
/* s_profile (nx values, may be NULL): mean of S over y and z.           */
/* ------------------------------------------------------------------ */
static rt bulk_energy(rt Q[3][3], const rt *p) {
  rt A0 = p[P_A0], gam = p[P_GAMMA];
  rt QQ[3][3];
  matmul(Q, Q, QQ);
  rt tr2 = ddot(Q, Q);
  rt tr3 = ddot(QQ, Q); /* Q_ab Q_bg Q_ga for symmetric Q */
  return A0 / 2.0 * (1.0 - gam / 3.0) * tr2 - A0 * gam / 3.0 * tr3 +
         A0 * gam / 4.0 * tr2 * tr2;
}

int API(orc_observables)(int lattice, int nx, int ny, int nz, const rt *p,
                         const rt *f, const rt *Q5, double s_ref, rt *out,
                         rt *s_profile) {
  grid_t g;
  if (!grid_ok(lattice, nx, ny, nz, &g)) return -1;
  long N = g.n;
  int q = nvel(lattice);
  rt *rho = (rt *)malloc(sizeof(rt) * N);
  rt *u3 = (rt *)malloc(sizeof(rt) * 3 * N);
  rt *prof = (rt *)calloc((size_t)nx, sizeof(rt));
  if (!rho || !u3 || !prof) {
    free(rho);
    free(u3);
    free(prof);
    return -2;
  }
  API(orc_fields)(lattice, nx, ny, nz, p, f, Q5, NULL, NULL, NULL, rho, u3);
  rt mass = 0, mom[3] = {0, 0, 0}, area = 0, energy = 0;
  double umax = 0, nonfinite = 0;
  for (long c = 0; c < N; c++) {
    int x, y, z;
    coords(&g, c, &x, &y, &z);
    mass += rho[c];
    rt uu = 0;
    for (int a = 0; a < 3; a++) {
      mom[a] += rho[c] * u3[a * N + c];
      uu += u3[a * N + c] * u3[a * N + c];
    }
    double un = sqrt(fabs(RE(uu)));
    if (un > umax) umax = un;
    rt Q[3][3];
    q_full(Q5, N, c, Q);
    rt S = RSQRT(1.5 * ddot(Q, Q)); /* reading R6 */
    area += S / s_ref;
    prof[x] += S;
    energy += bulk_energy(Q, p);
    for (int gdir = 0; gdir < 3; gdir++) {
      rt Qn[3][3];
      q_full(Q5, N,
             neighbour(&g, c, UNIT[gdir][0], UNIT[gdir][1], UNIT[gdir][2]), Qn);
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
          energy += p[P_K] / 2.0 * (Qn[a][b] - Q[a][b]) * (Qn[a][b] - Q[a][b]);
    }
    for (int i = 0; i < q; i++)
      if (!isfinite(RE(f[i * N + c]))) nonfinite += 1;
    for (int k = 0; k < 5; k++)
      if (!isfinite(RE(Q5[k * N + c]))) nonfinite += 1;
  }
  double per_col = (double)ny * nz;
  for (int x = 0; x < nx; x++) prof[x] /= per_col;
  double half = s_ref / 2.0, xi_pos = -1.0;
  for (int x = 0; x < nx; x++) {
    double a = RE(prof[x]), b = RE(prof[(x + 1) % nx]);
    if (a >= half && b < half) {
      xi_pos = x + (a - half) / (a - b);
      break;
    }
  }
  rt radius;
  if (lattice == ORC_D2Q9 || nz == 1)
    radius = RSQRT(area / M_PI);
  else
    radius = RPOW(3.0 * area / (4.0 * M_PI), 1.0 / 3.0);
  out[0] = mass;
  out[1] = mom[0];
  out[2] = mom[1];
  out[3] = mom[2];
  out[4] = area;
  out[5] = radius;
  out[6] = xi_pos;
  out[7] = umax;
  out[8] = energy;
  out[9] = nonfinite;
  if (s_profile)
    for (int x = 0; x < nx; x++) s_profile[x] = prof[x];
  free(rho);
  free(u3);
  free(prof);
  return 0;
}

#ifndef ORC_COMPLEX
#ifdef _OPENMP
#include <omp.h>
#endif
/* Threads of the OpenMP cell loops (for timing; the results do not depend on
 * it: every loop writes disjoint cells and the reductions are serial).
 * n <= 0 leaves the count unchanged.  Returns the count now in effect. */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}
#endif
