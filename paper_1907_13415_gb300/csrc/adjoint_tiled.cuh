// adjoint_tiled.cuh -- the reverse sweep of one checkpoint segment on a
// single-plane lattice as owned tiles with recomputed halos.
//
// The five stages of a reverse step (adjoint.cuh) each gather the previous
// stage's output from the neighbouring cells, so the one-cell-per-thread
// segment kernel (adjoint_segment.cuh) needs a grid-wide barrier after
// every stage.  Here a block owns a 16 x 8 tile and keeps the stage
// outputs of a 24 x 16 box around it in shared memory: stage s is computed
// on every box cell within Chebyshev distance r_s of the tile
// (r = 4, 3, 2, 1, 0 for the corrector, predictor, lb, stress and stencil
// adjoints), which is exactly the support the next stage's gather reads.
// Only the adjoints of the state at the start of the step (of Q and of the
// populations), which the next reverse step reads around every tile, go
// through global memory, so one grid barrier per reverse step remains.
// A box cell's halo values are recomputed by every block whose box holds
// it; each block writes global adjoints and adds parameter adjoints for its
// own tile only.  Every cell value is formed by the same functions in the
// same order as in the segment kernel, so the state adjoints agree to
// rounding (the compiler may contract multiply-adds differently in the two
// kernels); the parameter adjoints are summed in another grouping.
#pragma once
#include "adjoint.cuh"
#include "adjoint_segment.cuh"

namespace nlc {

// The tile trades recomputation (the box holds 3 times the tile's cells)
// against the number of blocks: 16 x 8 tiles put one block on each of 128
// SMs for a 128^2 lattice (16 x 16 tiles: 64 blocks doing 1.65 times the
// work each, slower).
constexpr int ATX = 16, ATY = 8;                    // owned tile
constexpr int AHALO = 4;                            // halo of the box
constexpr int ABW = ATX + 2 * AHALO;                // box width (24)
constexpr int ABH = ATY + 2 * AHALO;                // box height (16)
constexpr int ABA = ABW * ABH;                      // box cells = threads per block

// stage outputs on the box, [component][box cell]
template <class T>
struct AdjTile {
  T qp[5][ABA];   // 1: adjoint of Q^P                 (r <= 4)
  T ua[2][ABA];   // 1-2: adjoint of u (advection)    (r <= 4, then r <= 3)
  T gv[4][ABA];   // 1-2: adjoint of grad u            (r <= 4, then r <= 3)
  T f[2][ABA];    // 3: adjoint of the force           (r <= 2)
  T dq[10][ABA];  // 4: adjoint of the first derivatives (r <= 1)
  T lap[5][ABA];  // 4: adjoint of the Laplacian       (r <= 1)
};

__device__ __forceinline__ int pmod(int v, int n) {
  const int r = v % n;
  return r < 0 ? r + n : r;
}

// the R-stencil gather of adjoint.cuh (rhs_stencil_gather) for
// rbar = a * A + b * B with A a global dense array and B a box array
template <class T>
__device__ __forceinline__ void rhs_gather_box(const Field<T>& U, const T* __restrict__ A, T a,
                                               const T (*B)[ABA], T b, const Dims& d, int x,
                                               int y, int t, const Par<T>& p, T out[5]) {
  constexpr int DIM = 2;
  const int64_t c = cell_of(d, x, y, 0);
  const T gk = p.Gamma * p.K;
#pragma unroll
  for (int k = 0; k < 5; k++) {
    const T r0 = a * A[k * d.n + c] + b * B[k][t];
    out[k] += -T(2) * DIM * gk * r0;
  }
#pragma unroll
  for (int g = 0; g < DIM; g++) {
    const int64_t cp = nbr(d, x, y, 0, g, +1), cm = nbr(d, x, y, 0, g, -1);
    const int tp = g == 0 ? t + 1 : t + ABW, tm = g == 0 ? t - 1 : t - ABW;
    const int xp = g == 0 ? x + 1 : x, yp = g == 1 ? y + 1 : y;
    const int xm = g == 0 ? x - 1 : x, ym = g == 1 ? y - 1 : y;
    const T up = U.at(g, xp, yp, 0), um = U.at(g, xm, ym, 0);
#pragma unroll
    for (int k = 0; k < 5; k++) {
      const T rp = a * A[k * d.n + cp] + b * B[k][tp];
      const T rm = a * A[k * d.n + cm] + b * B[k][tm];
      out[k] += (up * rp - um * rm) / T(2) + gk * (rp + rm);
    }
  }
}

// Reverse sweep of the segment recorded in a (as k_seg_reverse), one block
// per owned tile of a tiles_x-wide grid of tiles; cooperative launch.  At
// most 96 registers per thread, so that a block of the record kernel of the
// previous segment (k_seg_record_tiled, at most 72 registers per thread),
// which runs at the same time on another stream, fits beside it on an SM.
template <class Lat, class T>
__global__ void __maxnreg__(96) k_seg_reverse_tiled(SegArgs<T> a, int tiles_x) {
  static_assert(Lat::DIM == 2, "single-plane lattices");
  constexpr int DIM = 2;
  extern __shared__ __align__(16) unsigned char adj_smem[];
  AdjTile<T>& S = *reinterpret_cast<AdjTile<T>*>(adj_smem);
  const SegSlots<Lat, T> R{a};
  const Dims d = a.d;
  const Par<T> p = a.p;
  const int t = threadIdx.x;
  const int lx = t % ABW - AHALO, ly = t / ABW - AHALO;  // offset from the tile origin
  const int x0 = (int)(blockIdx.x % (unsigned)tiles_x) * ATX;
  const int y0 = (int)(blockIdx.x / (unsigned)tiles_x) * ATY;
  const int x = pmod(x0 + lx, d.nx), y = pmod(y0 + ly, d.ny);
  const int64_t idx = cell_of(d, x, y, 0);
  // Chebyshev distance from the tile (0 inside it)
  const int r = max(max(max(-lx, lx - (ATX - 1)), max(-ly, ly - (ATY - 1))), 0);
  const bool own = r == 0 && x0 + lx < d.nx && y0 + ly < d.ny;
  double acc3[3] = {0.0, 0.0, 0.0};
  auto take = [&](const ParBar<T>& pb) {
    acc3[0] += (double)pb.gamma;
    acc3[1] += (double)pb.K;
    acc3[2] += (double)pb.Gamma;
  };
  unsigned gen = 0;
  int lc = a.lc0;
  bool ok = true;
  for (int j = a.len - 1; j >= 0 && ok; j--) {
    const Field<T> Q = R.q(j), U = R.u(j), QP = R.qp(j);
    const T* __restrict__ lQn = a.lQ[lc];
    T* __restrict__ lQo = a.lQ[lc ^ 1];
    const T* __restrict__ lGn = a.lG[lc];
    T* __restrict__ lGo = a.lG[lc ^ 1];
    T lq[5];  // adjoint of Q^j at this cell (kept for an owned cell)
    // 1. corrector evaluation (adj_be2_at)
    if (r <= 4) {
      T q[5], dq[3][5], lap[5], u[3], G[3][3], rb[5];
      q_stencil<T, DIM>(QP, x, y, 0, q, dq, lap);
      u_stencil<T, DIM>(U, x, y, 0, u, G);
#pragma unroll
      for (int k = 0; k < 5; k++) rb[k] = lQn[k * d.n + idx] / T(2);
      T qb[5] = {}, dqb[3][5] = {}, lapb[5] = {}, ub[3] = {}, Gb[3][3] = {};
      ParBar<T> pb{T(0), T(0), T(0)};
      be_rhs_vjp<T, DIM>(q, dq, lap, u, G, p, rb, qb, dqb, lapb, ub, Gb, pb);
      rhs_stencil_gather<T, DIM>(U, lQn, T(0.5), nullptr, T(0), d, x, y, 0, p, qb);
#pragma unroll
      for (int k = 0; k < 5; k++) S.qp[k][t] = qb[k];
#pragma unroll
      for (int c = 0; c < DIM; c++) {
        S.ua[c][t] = ub[c];
#pragma unroll
        for (int b = 0; b < DIM; b++) S.gv[c * DIM + b][t] = Gb[c][b];
      }
      if (own) take(pb);
    }
    __syncthreads();
    // 2. predictor evaluation (adj_be1_at)
    if (r <= 3) {
      T q[5], dq[3][5], lap[5], u[3], G[3][3], rb[5];
      q_stencil<T, DIM>(Q, x, y, 0, q, dq, lap);
      u_stencil<T, DIM>(U, x, y, 0, u, G);
#pragma unroll
      for (int k = 0; k < 5; k++) rb[k] = lQn[k * d.n + idx] / T(2) + S.qp[k][t];
      T qb[5] = {}, dqb[3][5] = {}, lapb[5] = {}, ub[3] = {}, Gb[3][3] = {};
      ParBar<T> pb{T(0), T(0), T(0)};
      be_rhs_vjp<T, DIM>(q, dq, lap, u, G, p, rb, qb, dqb, lapb, ub, Gb, pb);
      rhs_gather_box<T>(U, lQn, T(0.5), S.qp, T(1), d, x, y, t, p, qb);
#pragma unroll
      for (int k = 0; k < 5; k++) lq[k] = lQn[k * d.n + idx] + S.qp[k][t] + qb[k];
#pragma unroll
      for (int c = 0; c < DIM; c++) {
        S.ua[c][t] += ub[c];
#pragma unroll
        for (int b = 0; b < DIM; b++) S.gv[c * DIM + b][t] += Gb[c][b];
      }
      if (own) take(pb);
    }
    __syncthreads();
    // 3. lb update (adj_lb_at): the pulled-back population adjoints are
    // written for the targets in this block's own tile only
    if (r <= 2) {
      T F[3], g[Lat::Q], rho, u[3];
      force_at<T, DIM>(R.pi(j), d, x, y, 0, F);
      pull<Lat, T>(R.g(j), d, x, y, 0, g);
      moments<Lat, T>(g, F, p, rho, u);
      T ub[3] = {T(0), T(0), T(0)}, Fb[3] = {T(0), T(0), T(0)}, rhob = T(0), gb[Lat::Q];
#pragma unroll
      for (int c = 0; c < DIM; c++) {
        T s = S.ua[c][t];
#pragma unroll
        for (int b = 0; b < DIM; b++) {
          const int e = b == 0 ? 1 : ABW;
          s += (S.gv[c * DIM + b][t - e] - S.gv[c * DIM + b][t + e]) / T(2);
        }
        ub[c] = s;
      }
#pragma unroll
      for (int i = 0; i < Lat::Q; i++) gb[i] = lGn[(int64_t)i * d.n + idx];
      collide_bgk_vjp<Lat, T>(gb, rho, u, F, p, rhob, ub, Fb);
      moments_vjp<Lat, T>(rho, u, rhob, ub, gb, Fb);
#pragma unroll
      for (int i = 0; i < Lat::Q; i++) {
        const int tx = lx - Lat::c(i, 0), ty = ly - Lat::c(i, 1);
        if (tx >= 0 && tx < ATX && ty >= 0 && ty < ATY && x0 + tx < d.nx && y0 + ty < d.ny)
          lGo[(int64_t)i * d.n + cell_of(d, x0 + tx, y0 + ty, 0)] = gb[i];
      }
#pragma unroll
      for (int c = 0; c < DIM; c++) S.f[c][t] = Fb[c];
    }
    __syncthreads();
    // 4. stress (adj_stress_at)
    if (r <= 1) {
      T Pib[3][3] = {};
#pragma unroll
      for (int c = 0; c < DIM; c++)
#pragma unroll
        for (int b = 0; b < DIM; b++) {
          const int e = b == 0 ? 1 : ABW;
          Pib[c][b] = (S.f[c][t - e] - S.f[c][t + e]) / T(2);
        }
      T q[5], dq[3][5], lap[5], h[5];
      q_stencil<T, DIM>(Q, x, y, 0, q, dq, lap);
      molecular_field(q, lap, p, h);
      T qb[5] = {}, hb[5] = {}, dqb[3][5] = {}, lapb[5] = {};
      ParBar<T> pb{T(0), T(0), T(0)};
      stress_vjp<T, DIM>(q, h, dq, p, Pib, qb, hb, dqb, pb);
      molecular_field_vjp(q, lap, p, hb, qb, lapb, pb);
#pragma unroll
      for (int k = 0; k < 5; k++) {
        lq[k] += qb[k];
        S.lap[k][t] = lapb[k];
#pragma unroll
        for (int g = 0; g < DIM; g++) S.dq[g * 5 + k][t] = dqb[g][k];
      }
      if (own) take(pb);
    }
    __syncthreads();
    // 5. stencil transposes (adj_stencil_at) on the owned cells
    if (own) {
#pragma unroll
      for (int k = 0; k < 5; k++) {
        T s = -T(2) * DIM * S.lap[k][t];
#pragma unroll
        for (int g = 0; g < DIM; g++) {
          const int e = g == 0 ? 1 : ABW;
          s += (S.dq[g * 5 + k][t - e] - S.dq[g * 5 + k][t + e]) / T(2);
          s += S.lap[k][t + e] + S.lap[k][t - e];
        }
        lQo[k * d.n + idx] = lq[k] + s;
      }
    }
    // the adjoints of step j's state are complete everywhere before the
    // next reverse step reads them around every tile
    if (!(ok = grid_sync(a.bar, gen, a.err, a.wait_ns))) break;
    lc ^= 1;
  }
  if (!ok) return;
  __shared__ double sh[32];
  const double g0 = block_sum(acc3[0], sh);
  const double g1 = block_sum(acc3[1], sh);
  const double g2 = block_sum(acc3[2], sh);
  if (threadIdx.x == 0) {
    a.acc[3 * blockIdx.x + 0] += g0;
    a.acc[3 * blockIdx.x + 1] += g1;
    a.acc[3 * blockIdx.x + 2] += g2;
  }
}

// ---------------------------------------------------------------------------
// record of a segment on the same tiles
// ---------------------------------------------------------------------------
// The forward recomputation of a segment (as k_seg_record: the stress, lb,
// predictor and corrector stages of step_unfused.cuh, keeping Pi, u, Q^P
// and the next state in the record slots) with the intermediates of a step
// in shared memory on the tile's box: the stress on r <= 3, the lb update
// (u) on r <= 2, the predictor (Q^P) on r <= 1, the corrector on the tile,
// one grid barrier per step.  Records are written for the owned cells
// (with the periodic images of the padded fields).
template <class T>
struct RecTile {
  T pi[4][ABA];  // stress                (r <= 3)
  T u[2][ABA];   // velocity of Eq. 6     (r <= 2)
  T qp[5][ABA];  // predictor Q^P         (r <= 1)
};

template <class Lat, class T>
__global__ void __maxnreg__(72) k_seg_record_tiled(SegArgs<T> a, int tiles_x) {
  static_assert(Lat::DIM == 2, "single-plane lattices");
  constexpr int DIM = 2;
  extern __shared__ __align__(16) unsigned char rec_smem[];
  RecTile<T>& S = *reinterpret_cast<RecTile<T>*>(rec_smem);
  const SegSlots<Lat, T> R{a};
  const Dims d = a.d;
  const Par<T> p = a.p;
  const int t = threadIdx.x;
  const int lx = t % ABW - AHALO, ly = t / ABW - AHALO;
  const int x0 = (int)(blockIdx.x % (unsigned)tiles_x) * ATX;
  const int y0 = (int)(blockIdx.x / (unsigned)tiles_x) * ATY;
  const int x = pmod(x0 + lx, d.nx), y = pmod(y0 + ly, d.ny);
  const int64_t idx = cell_of(d, x, y, 0);
  const int r = max(max(max(-lx, lx - (ATX - 1)), max(-ly, ly - (ATY - 1))), 0);
  const bool own = r == 0 && x0 + lx < d.nx && y0 + ly < d.ny;
  // u and its gradient (u_stencil) from the box
  auto u_box = [&](T u[3], T G[3][3]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      if (c < DIM) {
        u[c] = S.u[c][t];
        G[c][0] = (S.u[c][t + 1] - S.u[c][t - 1]) / T(2);
        G[c][1] = (S.u[c][t + ABW] - S.u[c][t - ABW]) / T(2);
        G[c][2] = T(0);
      } else {
        u[c] = T(0);
        G[c][0] = G[c][1] = G[c][2] = T(0);
      }
    }
  };
  unsigned gen = 0;
  for (int j = 0; j < a.len; j++) {
    const Field<T> Q = R.q(j), U = R.u(j), QP = R.qp(j), Qn = R.q(j + 1);
    T r1[5];
    // 1. stress (stress_at)
    if (r <= 3) {
      T q[5], dq[3][5], lap[5], h[5], P[3][3];
      q_stencil<T, DIM>(Q, x, y, 0, q, dq, lap);
      molecular_field(q, lap, p, h);
      stress<T, DIM>(q, h, dq, p, P);
#pragma unroll
      for (int c = 0; c < DIM; c++)
#pragma unroll
        for (int b = 0; b < DIM; b++) {
          S.pi[c * DIM + b][t] = P[c][b];
          if (own) R.pi(j)[(c * DIM + b) * d.n + idx] = P[c][b];
        }
    }
    __syncthreads();
    // 2. lb update (lb_at, BGK)
    if (r <= 2) {
      T F[3], g[Lat::Q], rho, u[3];
#pragma unroll
      for (int c = 0; c < 3; c++) {
        T s = T(0);
        if (c < DIM) {
#pragma unroll
          for (int b = 0; b < DIM; b++) {
            const int e = b == 0 ? 1 : ABW;
            s += (S.pi[c * DIM + b][t + e] - S.pi[c * DIM + b][t - e]) / T(2);
          }
        }
        F[c] = s;
      }
      pull<Lat, T>(R.g(j), d, x, y, 0, g);
      moments<Lat, T>(g, F, p, rho, u);
      collide_bgk<Lat, T>(g, rho, u, F, p);
#pragma unroll
      for (int c = 0; c < DIM; c++) S.u[c][t] = u[c];
      if (own) {
        T* gout = R.g(j + 1);
#pragma unroll
        for (int i = 0; i < Lat::Q; i++) gout[(int64_t)i * d.n + idx] = g[i];
        store_with_images<T, DIM, DIM>(U, d, x, y, 0, u);
      }
    }
    __syncthreads();
    // 3. predictor (predict_at)
    if (r <= 1) {
      T q[5], dq[3][5], lap[5], u[3], G[3][3], qp[5];
      q_stencil<T, DIM>(Q, x, y, 0, q, dq, lap);
      u_box(u, G);
      be_rhs<T, DIM>(q, dq, lap, u, G, p, r1);
#pragma unroll
      for (int k = 0; k < 5; k++) {
        qp[k] = q[k] + r1[k];
        S.qp[k][t] = qp[k];
      }
      if (own) store_with_images<T, 5, DIM>(QP, d, x, y, 0, qp);
    }
    __syncthreads();
    // 4. corrector (correct_at) on the owned cells
    if (own) {
      T qp[5], dq[3][5], lap[5], u[3], G[3][3], r2[5], out[5];
#pragma unroll
      for (int k = 0; k < 5; k++) {
        const T v = S.qp[k][t];
        const T xp = S.qp[k][t + 1], xm = S.qp[k][t - 1];
        const T yp = S.qp[k][t + ABW], ym = S.qp[k][t - ABW];
        qp[k] = v;
        dq[0][k] = (xp - xm) / T(2);
        dq[1][k] = (yp - ym) / T(2);
        dq[2][k] = T(0);
        lap[k] = (xp + xm - T(2) * v) + (yp + ym - T(2) * v);
      }
      u_box(u, G);
      be_rhs<T, DIM>(qp, dq, lap, u, G, p, r2);
#pragma unroll
      for (int k = 0; k < 5; k++) out[k] = Q.at(k, x, y, 0) + (r1[k] + r2[k]) / T(2);
      store_with_images<T, 5, DIM>(Qn, d, x, y, 0, out);
    }
    // the step's records are complete everywhere before the next step
    // reads them around every tile
    if (!grid_sync(a.bar, gen, a.err, a.wait_ns)) return;
  }
}

}  // namespace nlc
