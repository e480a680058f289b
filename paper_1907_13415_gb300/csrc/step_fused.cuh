// step_fused.cuh -- one time step as two tiled kernels.
//
//   lb kernel : Q^n halo tile in shared memory -> H (Eq. 3) and the stress Pi
//               (Eq. 5 without P0) on the tile plus a one-cell ring, also in
//               shared memory -> F = div Pi -> pull-stream the populations,
//               rho and u (Eq. 6), BGK collision with the source term
//               (Sec. 1.2.1); stores the post-collision deviations g* and u^n.
//   be kernel : Q^n and u^n halo tiles in shared memory -> R(Q^n) and the
//               predictor Q^P on the tile plus a one-cell ring (shared memory)
//               -> R(Q^P) and the corrector Q^{n+1} (Sec. 1.2.2, steps 1-5).
//
// Each thread block owns a TX x TY tile of the (x, y) plane.  On D3Q19 it
// marches along z through a chunk of planes, keeping rings of the last three
// (or four) planes of each staged field in shared memory, so the z halo is
// read once per chunk instead of once per plane.  On D2Q9 there is a single
// plane.  Periodic wrap-around is applied when the halo tiles are gathered, so
// tiles at the domain edge, ragged tiles and lattices smaller than a tile all
// take the same path.
#pragma once
#include "common.cuh"
#include "lattice.cuh"
#include "physics.cuh"
#include "step_unfused.cuh"

namespace nlc {

constexpr int FTX = 32;   // tile width (x), one warp
constexpr int FTY = 8;    // tile height (y)
constexpr int FNT = FTX * FTY;
constexpr int RX2 = FTX + 4, RY2 = FTY + 4;  // tile + 2-cell ring
constexpr int RX1 = FTX + 2, RY1 = FTY + 2;  // tile + 1-cell ring
constexpr int A2 = RX2 * RY2;
constexpr int A1 = RX1 * RY1;

__device__ __forceinline__ int wrapm(int v, int n) {
  int r = v % n;
  return r < 0 ? r + n : r;
}

// gather `ncomp` planes of field F (plane stride n) at z into a shared tile
// of the 2-cell ring region, periodic
template <class T>
__device__ __forceinline__ void stage_plane(const T* __restrict__ F, int ncomp,
                                            const Dims& d, int x0, int y0,
                                            int z, T* __restrict__ s) {
  const int zz = wrapm(z, d.nz);
  for (int c = threadIdx.x; c < A2; c += FNT) {
    const int rx = c % RX2, ry = c / RX2;
    const int gx = wrapm(x0 - 2 + rx, d.nx), gy = wrapm(y0 - 2 + ry, d.ny);
    const int64_t cell = cell_of(d, gx, gy, zz);
    for (int k = 0; k < ncomp; k++) s[k * A2 + c] = F[k * d.n + cell];
  }
}

// ---------------------------------------------------------------------------
// lb kernel
// ---------------------------------------------------------------------------
template <class Lat, class T>
struct LbSmem {
  static constexpr int NP = Lat::DIM == 3 ? 3 : 1;
  static constexpr int NPI = Lat::DIM * Lat::DIM;
  static constexpr size_t bytes = sizeof(T) * (size_t)NP * (5 * A2 + NPI * A1);
};

// stress on the 1-ring region of plane slot `s` (z neighbours in slots sm, sp)
template <class Lat, class T>
__device__ __forceinline__ void stress_plane(const T* __restrict__ sQ, int s,
                                             int sm, int sp,
                                             T* __restrict__ sPi,
                                             const Par<T>& p) {
  constexpr int DIM = Lat::DIM;
  constexpr int NPI = DIM * DIM;
  const T* Qc = sQ + s * 5 * A2;
  const T* Qm = sQ + sm * 5 * A2;
  const T* Qp = sQ + sp * 5 * A2;
  for (int c = threadIdx.x; c < A1; c += FNT) {
    const int hx = c % RX1 + 1, hy = c / RX1 + 1;
    const int o = hy * RX2 + hx;
    T q[5], dq[3][5], lap[5], h[5], P[3][3];
#pragma unroll
    for (int k = 0; k < 5; k++) {
      const T* F = Qc + k * A2;
      const T v = F[o], xp = F[o + 1], xm = F[o - 1], yp = F[o + RX2], ym = F[o - RX2];
      q[k] = v;
      dq[0][k] = (xp - xm) / T(2);
      dq[1][k] = (yp - ym) / T(2);
      T l = (xp + xm - T(2) * v) + (yp + ym - T(2) * v);
      if (DIM == 3) {
        const T zp = Qp[k * A2 + o], zm = Qm[k * A2 + o];
        dq[2][k] = (zp - zm) / T(2);
        l += zp + zm - T(2) * v;
      } else {
        dq[2][k] = T(0);
      }
      lap[k] = l;
    }
    molecular_field(q, lap, p, h);
    stress<T, DIM>(q, h, dq, p, P);
#pragma unroll
    for (int a = 0; a < DIM; a++)
#pragma unroll
      for (int b = 0; b < DIM; b++) sPi[(a * DIM + b) * A1 + c] = P[a][b];
  }
  (void)NPI;
}

template <class Lat, class T>
__global__ void __launch_bounds__(FNT) k_fused_lb(const T* __restrict__ gin,
                                                  T* __restrict__ gout,
                                                  const T* __restrict__ Q,
                                                  T* __restrict__ U, Dims d,
                                                  Par<T> p, int tz) {
  constexpr int DIM = Lat::DIM;
  constexpr int NPI = DIM * DIM;
  constexpr int NP = LbSmem<Lat, T>::NP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sQ = reinterpret_cast<T*>(smem_raw);   // [NP][5][A2]
  T* sPi = sQ + NP * 5 * A2;                // [NP][NPI][A1]

  const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
  const int tx = threadIdx.x % FTX, ty = threadIdx.x / FTX;
  const int x = x0 + tx, y = y0 + ty;
  const bool inside = x < d.nx && y < d.ny;
  const int ic = (ty + 1) * RX1 + (tx + 1);  // own cell in the 1-ring region

  auto lb_cell = [&](int z, const T* Pc, const T* Pm, const T* Pp) {
    if (!inside || z >= d.nz) return;
    T F[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int a = 0; a < DIM; a++) {
      T s = (Pc[(a * DIM + 0) * A1 + ic + 1] - Pc[(a * DIM + 0) * A1 + ic - 1]) / T(2);
      s += (Pc[(a * DIM + 1) * A1 + ic + RX1] - Pc[(a * DIM + 1) * A1 + ic - RX1]) / T(2);
      if (DIM == 3) s += (Pp[(a * DIM + 2) * A1 + ic] - Pm[(a * DIM + 2) * A1 + ic]) / T(2);
      F[a] = s;
    }
    T g[Lat::Q], rho, u[3];
    pull<Lat, T>(gin, d, x, y, z, g);
    moments<Lat, T>(g, F, p, rho, u);
    collide_bgk<Lat, T>(g, rho, u, F, p);
    const int64_t cell = cell_of(d, x, y, z);
#pragma unroll
    for (int i = 0; i < Lat::Q; i++) gout[(int64_t)i * d.n + cell] = g[i];
#pragma unroll
    for (int a = 0; a < DIM; a++) U[a * d.n + cell] = u[a];
  };

  if constexpr (DIM == 2) {
    stage_plane<T>(Q, 5, d, x0, y0, 0, sQ);
    __syncthreads();
    stress_plane<Lat, T>(sQ, 0, 0, 0, sPi, p);
    __syncthreads();
    lb_cell(0, sPi, sPi, sPi);
  } else {
    const int z0 = blockIdx.z * tz;
    const int z1 = min(z0 + tz, d.nz);
    // plane z lives in slot (z - z0 + 3) % 3 of both rings
    auto slot = [&](int z) { return (z - z0 + 6) % 3; };
    auto Qs = [&](int z) { return sQ + slot(z) * 5 * A2; };
    auto Ps = [&](int z) { return sPi + slot(z) * NPI * A1; };
    stage_plane<T>(Q, 5, d, x0, y0, z0 - 2, Qs(z0 - 2));
    stage_plane<T>(Q, 5, d, x0, y0, z0 - 1, Qs(z0 - 1));
    stage_plane<T>(Q, 5, d, x0, y0, z0, Qs(z0));
    __syncthreads();
    stress_plane<Lat, T>(sQ, slot(z0 - 1), slot(z0 - 2), slot(z0), Ps(z0 - 1), p);
    __syncthreads();
    stage_plane<T>(Q, 5, d, x0, y0, z0 + 1, Qs(z0 + 1));
    __syncthreads();
    stress_plane<Lat, T>(sQ, slot(z0), slot(z0 - 1), slot(z0 + 1), Ps(z0), p);
    for (int z = z0; z < z1; z++) {
      __syncthreads();
      stage_plane<T>(Q, 5, d, x0, y0, z + 2, Qs(z + 2));
      __syncthreads();
      stress_plane<Lat, T>(sQ, slot(z + 1), slot(z), slot(z + 2), Ps(z + 1), p);
      __syncthreads();
      lb_cell(z, Ps(z), Ps(z - 1), Ps(z + 1));
    }
  }
}

// ---------------------------------------------------------------------------
// Beris-Edwards kernel
// ---------------------------------------------------------------------------
template <class Lat, class T>
struct BeSmem {
  static constexpr int NQ = Lat::DIM == 3 ? 3 : 1;   // Q^n ring
  static constexpr int NU = Lat::DIM == 3 ? 4 : 1;   // u ring
  static constexpr int NQP = Lat::DIM == 3 ? 3 : 1;  // Q^P ring
  static constexpr int NR = Lat::DIM == 3 ? 2 : 1;   // R(Q^n) ring
  static constexpr size_t bytes =
      sizeof(T) * ((size_t)NQ * 5 * A2 + (size_t)NU * Lat::DIM * A2 +
                   (size_t)NQP * 5 * A1 + (size_t)NR * 5 * A1);
};

// central differences + Laplacian of a 5-component tile field at offset o of
// a tile with row length RX (z neighbours from the planes above and below)
template <class T, int DIM, int RX, int AREA>
__device__ __forceinline__ void tile_stencil5(const T* __restrict__ c,
                                              const T* __restrict__ m,
                                              const T* __restrict__ pp, int o,
                                              T q[5], T dq[3][5], T lap[5]) {
#pragma unroll
  for (int k = 0; k < 5; k++) {
    const T* F = c + k * AREA;
    const T v = F[o], xp = F[o + 1], xm = F[o - 1], yp = F[o + RX], ym = F[o - RX];
    q[k] = v;
    dq[0][k] = (xp - xm) / T(2);
    dq[1][k] = (yp - ym) / T(2);
    T l = (xp + xm - T(2) * v) + (yp + ym - T(2) * v);
    if (DIM == 3) {
      const T zp = pp[k * AREA + o], zm = m[k * AREA + o];
      dq[2][k] = (zp - zm) / T(2);
      l += zp + zm - T(2) * v;
    } else {
      dq[2][k] = T(0);
    }
    lap[k] = l;
  }
}

// u and G[a][b] = d_b u_a at offset o of the 2-ring u tile
template <class T, int DIM>
__device__ __forceinline__ void tile_ugrad(const T* __restrict__ c,
                                           const T* __restrict__ m,
                                           const T* __restrict__ pp, int o,
                                           T u[3], T G[3][3]) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    if (a < DIM) {
      const T* F = c + a * A2;
      u[a] = F[o];
      G[a][0] = (F[o + 1] - F[o - 1]) / T(2);
      G[a][1] = (F[o + RX2] - F[o - RX2]) / T(2);
      G[a][2] = DIM == 3 ? (pp[a * A2 + o] - m[a * A2 + o]) / T(2) : T(0);
    } else {
      u[a] = T(0);
      G[a][0] = G[a][1] = G[a][2] = T(0);
    }
  }
}

template <class Lat, class T>
__global__ void __launch_bounds__(FNT) k_fused_be(const T* __restrict__ Q,
                                                  const T* __restrict__ U,
                                                  T* __restrict__ Qout, Dims d,
                                                  Par<T> p, int tz) {
  constexpr int DIM = Lat::DIM;
  using S = BeSmem<Lat, T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sQ = reinterpret_cast<T*>(smem_raw);  // [NQ][5][A2]
  T* sU = sQ + S::NQ * 5 * A2;             // [NU][DIM][A2]
  T* sQP = sU + S::NU * DIM * A2;          // [NQP][5][A1]
  T* sR = sQP + S::NQP * 5 * A1;           // [NR][5][A1]

  const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
  const int tx = threadIdx.x % FTX, ty = threadIdx.x / FTX;
  const int x = x0 + tx, y = y0 + ty;
  const bool inside = x < d.nx && y < d.ny;
  const int z0 = DIM == 3 ? blockIdx.z * tz : 0;

  auto sq = [&](int z) { return sQ + ((z - z0 + 6) % S::NQ) * 5 * A2; };
  auto su = [&](int z) { return sU + ((z - z0 + 8) % S::NU) * DIM * A2; };
  auto sqp = [&](int z) { return sQP + ((z - z0 + 6) % S::NQP) * 5 * A1; };
  auto sr = [&](int z) { return sR + ((z - z0 + 6) % S::NR) * 5 * A1; };

  // predictor on the 1-ring region of plane z: R(Q^n) and Q^P = Q^n + R
  auto predict_plane = [&](int z) {
    const T* qc = sq(z);
    const T* qm = DIM == 3 ? sq(z - 1) : qc;
    const T* qpn = DIM == 3 ? sq(z + 1) : qc;
    const T* uc = su(z);
    const T* um = DIM == 3 ? su(z - 1) : uc;
    const T* upn = DIM == 3 ? su(z + 1) : uc;
    T* qp_out = sqp(z);
    T* r_out = sr(z);
    for (int c = threadIdx.x; c < A1; c += FNT) {
      const int o = (c / RX1 + 1) * RX2 + (c % RX1 + 1);
      T q[5], dq[3][5], lap[5], u[3], G[3][3], r[5];
      tile_stencil5<T, DIM, RX2, A2>(qc, qm, qpn, o, q, dq, lap);
      tile_ugrad<T, DIM>(uc, um, upn, o, u, G);
      be_rhs<T, DIM>(q, dq, lap, u, G, p, r);
#pragma unroll
      for (int k = 0; k < 5; k++) {
        r_out[k * A1 + c] = r[k];
        qp_out[k * A1 + c] = q[k] + r[k];
      }
    }
  };

  // corrector at the tile cells of plane z
  auto correct_cell = [&](int z) {
    if (!inside || z >= d.nz) return;
    const int ic = (ty + 1) * RX1 + (tx + 1);
    const int o2 = (ty + 2) * RX2 + (tx + 2);
    const T* pc = sqp(z);
    const T* pm = DIM == 3 ? sqp(z - 1) : pc;
    const T* ppn = DIM == 3 ? sqp(z + 1) : pc;
    T qp[5], dq[3][5], lap[5], u[3], G[3][3], r2[5];
    tile_stencil5<T, DIM, RX1, A1>(pc, pm, ppn, ic, qp, dq, lap);
    tile_ugrad<T, DIM>(su(z), DIM == 3 ? su(z - 1) : su(z),
                       DIM == 3 ? su(z + 1) : su(z), o2, u, G);
    be_rhs<T, DIM>(qp, dq, lap, u, G, p, r2);
    const T* qn = sq(z);
    const T* r1 = sr(z);
    const int64_t cell = cell_of(d, x, y, z);
#pragma unroll
    for (int k = 0; k < 5; k++)
      Qout[k * d.n + cell] = qn[k * A2 + o2] + (r1[k * A1 + ic] + r2[k]) / T(2);
  };

  if constexpr (DIM == 2) {
    stage_plane<T>(Q, 5, d, x0, y0, 0, sq(0));
    stage_plane<T>(U, DIM, d, x0, y0, 0, su(0));
    __syncthreads();
    predict_plane(0);
    __syncthreads();
    correct_cell(0);
  } else {
    const int z1 = min(z0 + tz, d.nz);
    for (int z = z0 - 2; z <= z0; z++) {
      stage_plane<T>(Q, 5, d, x0, y0, z, sq(z));
      stage_plane<T>(U, DIM, d, x0, y0, z, su(z));
    }
    __syncthreads();
    predict_plane(z0 - 1);
    __syncthreads();
    stage_plane<T>(Q, 5, d, x0, y0, z0 + 1, sq(z0 + 1));
    stage_plane<T>(U, DIM, d, x0, y0, z0 + 1, su(z0 + 1));
    __syncthreads();
    predict_plane(z0);
    for (int z = z0; z < z1; z++) {
      __syncthreads();
      stage_plane<T>(Q, 5, d, x0, y0, z + 2, sq(z + 2));
      stage_plane<T>(U, DIM, d, x0, y0, z + 2, su(z + 2));
      __syncthreads();
      predict_plane(z + 1);
      __syncthreads();
      correct_cell(z);
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <class Lat>
__host__ inline dim3 fused_grid(const Dims& d, int tz) {
  return dim3((unsigned)((d.nx + FTX - 1) / FTX), (unsigned)((d.ny + FTY - 1) / FTY),
              Lat::DIM == 3 ? (unsigned)((d.nz + tz - 1) / tz) : 1u);
}

template <class Lat>
__host__ inline int fused_tz(const Dims& d) {
  if (Lat::DIM == 2) return 1;
  // enough blocks for several waves over the SMs while amortising the
  // z ring prologue
  const int64_t tiles = (int64_t)((d.nx + FTX - 1) / FTX) * ((d.ny + FTY - 1) / FTY);
  int tz = 16;
  while (tz > 4 && tiles * ((d.nz + tz - 1) / tz) < 1200) tz /= 2;
  return tz < d.nz ? tz : d.nz;
}

template <class Lat, class T>
cudaError_t launch_fused_lb(const T* gin, T* gout, const T* Q, T* U,
                            const Dims& d, const Par<T>& p, cudaStream_t st) {
  static unsigned long long configured = 0;  // one bit per device
  const size_t smem = LbSmem<Lat, T>::bytes;
  int dev = 0;
  cudaGetDevice(&dev);
  if (!(configured >> (dev & 63) & 1ull)) {
    cudaError_t e = cudaFuncSetAttribute(k_fused_lb<Lat, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    configured |= 1ull << (dev & 63);
  }
  const int tz = fused_tz<Lat>(d);
  k_fused_lb<Lat, T><<<fused_grid<Lat>(d, tz), FNT, smem, st>>>(gin, gout, Q, U, d, p, tz);
  return cudaGetLastError();
}

template <class Lat, class T>
cudaError_t launch_fused_be(const T* Q, const T* U, T* Qout, const Dims& d,
                            const Par<T>& p, cudaStream_t st) {
  static unsigned long long configured = 0;  // one bit per device
  const size_t smem = BeSmem<Lat, T>::bytes;
  int dev = 0;
  cudaGetDevice(&dev);
  if (!(configured >> (dev & 63) & 1ull)) {
    cudaError_t e = cudaFuncSetAttribute(k_fused_be<Lat, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    configured |= 1ull << (dev & 63);
  }
  const int tz = fused_tz<Lat>(d);
  k_fused_be<Lat, T><<<fused_grid<Lat>(d, tz), FNT, smem, st>>>(Q, U, Qout, d, p, tz);
  return cudaGetLastError();
}

}  // namespace nlc
