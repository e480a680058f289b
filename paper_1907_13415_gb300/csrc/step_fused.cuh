// step_fused.cuh -- one time step as two tiled kernels.
//
//   lb kernel : Q^n tile (+2-cell halo) in shared memory -> H (Eq. 3) and the
//               stress Pi (Eq. 5 without P0) on the tile plus a one-cell
//               ring, in shared memory -> F = div Pi -> pull-stream the
//               populations, rho and u (Eq. 6), BGK collision with the
//               source term (Sec. 1.2.1); stores the post-collision
//               deviations g* and u^n.
//   be kernel : Q^n and u^n tiles (+2 halo) in shared memory -> R(Q^n) and
//               the predictor Q^P on the tile plus a one-cell ring (shared
//               memory) -> R(Q^P) and the corrector Q^{n+1} (Sec. 1.2.2,
//               steps 1-5).
//
// Each thread block owns a 32 x 8 tile of the (x, y) plane of one lattice
// (a batched context lists the tiles of all its lattices, so one launch
// advances all of them).  On D3Q19 it
// marches along z through a chunk of planes; the halo planes of Q and u
// arrive by TMA (one cp.async.bulk.tensor per plane and field) into rings of
// shared-memory slots, each completed on its own mbarrier, issued one plane
// ahead of use so the copy overlaps the computation of the current plane.
// On a single plane (D2Q9) it works the same way through a chunk of tiles
// stacked along y instead, the next tile's boxes in flight while the
// current tile is computed.
// Q and u are padded fields with periodic ghost rings (common.cuh), so every
// tile box is a plain rectangle; the kernels that write them also write the
// images.  Populations are read by pull with precomputed periodic offsets.
//
// Block = 11 warps.  Per plane, a ring phase gives each of the 340 cells of
// the tile plus its one-cell ring one thread (whole rows per warp), and a
// cell phase gives each of the 256 tile cells one thread; one barrier per
// plane separates them, with enough plane slots in shared memory that the
// ring phase of plane z+1 may overlap slower threads still in the cell phase
// of plane z.  FP32 runs the collision on packed pairs of opposite
// populations (packed.cuh).
#pragma once
#include "aux_kernels.cuh"
#include "chunks.h"
#include "common.cuh"
#include "grid_sync.cuh"
#include "lattice.cuh"
#include "packed.cuh"
#include "physics.cuh"
#include "step_unfused.cuh"
#include "tma.cuh"

#include <type_traits>
#include <vector>

namespace nlc {

constexpr int FTX = 32;                  // tile width (x)
constexpr int FTY = 8;                   // tile height (y)
constexpr int RX1 = FTX + 2, RY1 = FTY + 2;  // tile + 1-cell ring
constexpr int A1 = RX1 * RY1;            // 340 ring-region cells
constexpr int BXW = FTX + 8;             // TMA box width: x0-4 .. x0+35
constexpr int BYH = FTY + 4;             // TMA box height: y0-2 .. y0+9
constexpr int BA = BXW * BYH;            // box plane area (480)

// box index of lattice offset (dx, dy) from the tile origin (x0, y0)
__host__ __device__ constexpr int box_at(int dx, int dy) { return (dy + 2) * BXW + dx + 4; }

// slot s + k of a ring of N plane slots, 0 <= s < N, 0 <= k < N
template <int N>
__device__ __forceinline__ int slot_add(int s, int k) {
  const int r = s + k;
  return r >= N ? r - N : r;
}

// Ring-phase thread t -> cell (cx, cy) of the tile plus its one-cell ring,
// cx in [-1, FTX], cy in [-1, FTY], and its index ri = (cy + 1) RX1 + cx + 1
// in the ring-region arrays.  The first FTX (FTY + 2) threads take whole rows
// of FTX cells, one warp per row, so every shared-memory access of those
// warps is one contiguous run (no bank conflicts); the last 2 (FTY + 2)
// threads take the left and right ring columns.
static_assert(FTX == 32, "one warp per ring row");
__device__ __forceinline__ void ring_cell(int t, int& cx, int& cy, int& ri) {
  constexpr int NROW = FTX * RY1;
  if (t < NROW) {
    cx = t % FTX;
    cy = t / FTX - 1;
  } else {
    const int k = t - NROW;
    cx = (k & 1) ? FTX : -1;
    cy = (k >> 1) - 1;
  }
  ri = (cy + 1) * RX1 + cx + 1;
}

template <class T>
constexpr size_t align128(size_t bytes) {
  return (bytes + 127) / 128 * 128;
}

// One lattice of a (possibly batched) context, as the step kernels see it.
// T: arithmetic and the Q and u fields; G: storage of the populations.
template <class T, class G = T>
struct InstDev {
  Dims d;
  Par<T> p;
  G* g[2];         // populations (deviations), ping-pong
  Field<T> q[2];   // Q, ping-pong
  Field<T> u;      // u^n handed from the lb to the Beris-Edwards kernel
  const T* mrt;    // Q coefficients s_k / |v_k|^2 of the MRT collision, or nullptr
};

// One thread block's work: a 32 x 8 (x, y) tile of instance `inst`, planes
// z0 .. z1 - 1; on a single plane, z1 tiles stacked along y from row y0
// (z0 = 0).
struct TileRef {
  int inst, x0, y0, z0, z1;
};

// ---------------------------------------------------------------------------
// lb kernel
// ---------------------------------------------------------------------------
template <class Lat, class T>
struct LbCfg {
  static constexpr int DIM = Lat::DIM;
  static constexpr int NPI = DIM * DIM;
  // ring phase on threads [0, RING_T), cell phase on [CELL0, CELL0 + 256)
  static constexpr int RING_T = A1;
  static constexpr int CELL0 = 0;
  static constexpr int THREADS = 352;  // 11 warps
  static constexpr int MINB = sizeof(T) == 4 ? 2 : 1;
  static_assert(THREADS >= RING_T && THREADS >= CELL0 + FTX * FTY, "block too small");
  // Q plane slots (on a single plane: tile slots, the next tile's copy in
  // flight while the current one is used)
  static constexpr int NSQ = DIM == 3 ? 4 : 2;
  // Pi plane slots: the ring phase of plane z+1 may start while slower
  // threads still read Pi(z-2..z) for plane z-1, so four slots let one
  // barrier per plane suffice (on a single plane, two tile slots)
  static constexpr int NSP = DIM == 3 ? 4 : 2;
  static constexpr size_t q_slot = align128<T>(sizeof(T) * 5 * BA);
  static constexpr size_t p_slot = align128<T>(sizeof(T) * NPI * A1);
  static constexpr size_t off_p = NSQ * q_slot;
  // D3Q19: the force of the tile's cells, two plane slots [3][FTX FTY]
  // (formed by the warps without a tile cell, read by the cell phase one
  // plane later)
  static constexpr int NSF = DIM == 3 ? 2 : 0;
  static constexpr size_t f_slot = align128<T>(sizeof(T) * 3 * FTX * FTY);
  static constexpr size_t off_f = off_p + NSP * p_slot;
  static constexpr size_t off_bar = off_f + NSF * f_slot;
  static constexpr size_t bytes = off_bar + 8 * NSQ;
  static constexpr uint32_t tx_bytes = sizeof(T) * 5 * BA;
};

// 2d+1-point Laplacian from the centre value and its axis neighbours (zp, zm
// unused on a single plane).  FP64 keeps the per-axis form; FP32 sums the
// neighbours first and removes 2d v with one fused multiply-add.
template <class T, int DIM>
__device__ __forceinline__ T lap_points(T v, T xp, T xm, T yp, T ym, T zp, T zm) {
  if constexpr (std::is_same<T, double>::value) {
    T l = (xp + xm - T(2) * v) + (yp + ym - T(2) * v);
    if (DIM == 3) l += zp + zm - T(2) * v;
    return l;
  } else {
    T s = (xp + xm) + (yp + ym);
    if (DIM == 3) s += zp + zm;
    return fma_(T(-2.0 * DIM), v, s);
  }
}

// Isotropic stencils on the lattice's neighbour set (the remedy the paper
// points to for spurious currents, Sec. 2.2): twice the gradient,
// 2 d_a phi = 6 sum_i w_i c_ia phi(x + c_i), and the Laplacian,
// lap phi = 6 sum_i w_i [phi(x + c_i) - phi(x)], from at(cx, cy, cz), the
// value at neighbour offset c_i, and v = phi(x).
template <class Lat, class T, class At>
__device__ __forceinline__ void lattice_stencil(const At& at, T v, T d2[3], T& lap) {
  d2[0] = d2[1] = d2[2] = T(0);
  T s = T(0);
#pragma unroll
  for (int i = 1; i < Lat::Q; i++) {
    const T vi = at(Lat::c(i, 0), Lat::c(i, 1), Lat::c(i, 2));
    const T w = T(Lat::w(i));
    s = fma_(w, vi, s);
#pragma unroll
    for (int a = 0; a < 3; a++)
      if (Lat::c(i, a) != 0) d2[a] = fma_(T(Lat::c(i, a)) * w, vi, d2[a]);
  }
#pragma unroll
  for (int a = 0; a < 3; a++) d2[a] = d2[a] * T(6);
  lap = T(6) * fma_(T(-(1.0 - Lat::w(0))), v, s);
}

// stress on the ring-region cell of ring-phase thread t of a plane whose Q
// box is in sq (z neighbours in sqm, sqp), into the Pi slot sp.  The first
// derivatives are kept as plain differences (twice the central difference);
// the stress sees them with K/4, which gives K dQ:dQ exactly (scalings by
// powers of two are exact).
template <class Lat, class T, bool ISO>
__device__ __forceinline__ void stress_ring_cell(int t, const T* __restrict__ sq,
                                                 const T* __restrict__ sqm,
                                                 const T* __restrict__ sqp,
                                                 T* __restrict__ sp, const Par<T>& p) {
  constexpr int DIM = Lat::DIM;
  int cx, cy, c;
  ring_cell(t, cx, cy, c);
  const int o = box_at(cx, cy);
  T q[5], dq2[3][5], lap[5], h[5], P[3][3];
  // FP32: components (0, 1) and (2, 3) as packed pairs (same operations in
  // the same order as the scalar form, lane by lane)
  constexpr int KP = (std::is_same<T, float>::value && !ISO) ? 4 : 0;
  if constexpr (KP == 4) {
#pragma unroll
    for (int k = 0; k < 4; k += 2) {
      const float* F0 = sq + k * BA;
      const float* F1 = F0 + BA;
      const float2 v = pk(F0[o], F1[o]);
      const float2 xp = pk(F0[o + 1], F1[o + 1]), xm = pk(F0[o - 1], F1[o - 1]);
      const float2 yp = pk(F0[o + BXW], F1[o + BXW]), ym = pk(F0[o - BXW], F1[o - BXW]);
      float2 sum = padd(padd(xp, xm), padd(yp, ym));
      float2 dz = bc(0.0f);
      if (DIM == 3) {
        const float2 zp = pk(sqp[k * BA + o], sqp[(k + 1) * BA + o]);
        const float2 zm = pk(sqm[k * BA + o], sqm[(k + 1) * BA + o]);
        sum = padd(sum, padd(zp, zm));
        dz = psub(zp, zm);
      }
      const float2 dx = psub(xp, xm), dy = psub(yp, ym);
      const float2 l = pfma(bc(-2.0f * DIM), v, sum);
      q[k] = v.x, q[k + 1] = v.y;
      dq2[0][k] = dx.x, dq2[0][k + 1] = dx.y;
      dq2[1][k] = dy.x, dq2[1][k + 1] = dy.y;
      dq2[2][k] = dz.x, dq2[2][k + 1] = dz.y;
      lap[k] = l.x, lap[k + 1] = l.y;
    }
  }
#pragma unroll
  for (int k = KP; k < 5; k++) {
    if constexpr (ISO) {
      const int ok = k * BA + o;
      auto at = [&](int dx, int dy, int dz) {
        const T* pl = dz == 0 ? sq : (dz > 0 ? sqp : sqm);
        return pl[ok + dx + dy * BXW];
      };
      T d2[3];
      q[k] = sq[ok];
      lattice_stencil<Lat, T>(at, q[k], d2, lap[k]);
      dq2[0][k] = d2[0];
      dq2[1][k] = d2[1];
      dq2[2][k] = d2[2];
      continue;
    }
    const T* F = sq + k * BA;
    const T v = F[o], xp = F[o + 1], xm = F[o - 1];
    const T yp = F[o + BXW], ym = F[o - BXW];
    q[k] = v;
    dq2[0][k] = xp - xm;
    dq2[1][k] = yp - ym;
    T zp = T(0), zm = T(0);
    if (DIM == 3) {
      zp = (sqp + k * BA)[o];
      zm = (sqm + k * BA)[o];
    }
    dq2[2][k] = zp - zm;
    lap[k] = lap_points<T, DIM>(v, xp, xm, yp, ym, zp, zm);
  }
  molecular_field(q, lap, p, h);
  Par<T> p4 = p;
  p4.K = p.K * T(0.25);
  stress<T, DIM>(q, h, dq2, p4, P);
#pragma unroll
  for (int a = 0; a < DIM; a++)
#pragma unroll
    for (int b = 0; b < DIM; b++) sp[(a * DIM + b) * A1 + c] = P[a][b];
}

// Populations of one cell as the lb kernel holds them in registers: FP32
// keeps the rest value and the opposite pairs (packed arithmetic), FP64 a
// plain array.
template <class Lat, class T>
struct CellPops {
  T g[Lat::Q];
};
template <class Lat>
struct CellPops<Lat, float> {
  float g0;
  float2 gp[(Lat::Q - 1) / 2];
};

// Element offset i n + o of cell o in population plane i.  When every
// lattice of the launch has Q n < 2^32 (IX32) the sum stays in 32 bits,
// which saves the wide arithmetic on each of the Q loads and stores of a
// cell; larger lattices take the 64-bit form.
template <bool IX32>
__device__ __forceinline__ size_t pop_off(int i, unsigned n, unsigned o) {
  if constexpr (IX32)
    return (unsigned)(i * n + o);
  else
    return (size_t)i * n + o;
}

// MRT: the multiple-relaxation-time collision (physics.cuh: collide_mrt);
// a lattice of the launch without its own rates gets the BGK rates 1/tau.
// IX32: population offsets in 32 bits (pop_off).
// OBS: instead of a step, the observables of the current state (the terms
// of aux_kernels.cuh: rho and u of Eq. 6 in the cell phase, the Q terms of
// the tile's cells in the ring phase), summed per block into
// obs_partial[block][OBS_SLOTS]; nothing is stored.
// PERSIST: called repeatedly by the blocks of the persistent kernel, which
// rewrites the populations it reads within one launch: the pulls then go
// through L2 only (ld.global.cg) instead of the read-only path.
// Returns false when a bounded wait ran out (the error word is set and the
// block's copies are drained).
template <class Lat, class T, class G, bool MRT, bool ISO, bool IX32, bool OBS = false,
          bool PERSIST = false>
__device__ __forceinline__ bool fused_lb_tile(const TileRef tile,
                                              const InstDev<T, G>* __restrict__ insts,
                                              const CUtensorMap* __restrict__ qmaps, int cur,
                                              unsigned* __restrict__ err,
                                              double* __restrict__ obs_partial) {
  using C = LbCfg<Lat, T>;
  constexpr int DIM = Lat::DIM;
  constexpr int NPI = C::NPI;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::off_bar);
  auto sQ = [&](int slot) { return reinterpret_cast<T*>(smem + slot * C::q_slot); };
  auto sP = [&](int slot) { return reinterpret_cast<T*>(smem + C::off_p + slot * C::p_slot); };

  const InstDev<T, G>& I = insts[tile.inst];
  const Dims d = I.d;
  const Par<T> p = I.p;
  const G* __restrict__ gin = I.g[cur];
  G* __restrict__ gout = I.g[cur ^ 1];
  const Field<T> U = I.u;
  const int zoff = U.L.zoff;
  const CUtensorMap* qmap = &qmaps[2 * tile.inst + cur];

  const int tid = threadIdx.x;
  const int x0 = tile.x0, y0 = tile.y0;
  const int z0 = tile.z0;
  const int z1 = DIM == 3 ? tile.z1 : 1;
  const int zq0 = DIM == 3 ? z0 - 2 : 0;  // first Q plane loaded
  const int zp0 = DIM == 3 ? z0 - 1 : 0;  // first Pi plane computed
  // z - zq0 and z - zp0 are never negative: unsigned arithmetic lets the
  // power-of-two slot counts reduce to masks and shifts
  static_assert((C::NSQ & (C::NSQ - 1)) == 0 && (C::NSP & (C::NSP - 1)) == 0,
                "power-of-two slot counts");
  auto qslot = [&](int z) { return (int)((unsigned)(z - zq0) % C::NSQ); };
  auto qpar = [&](int z) { return ((unsigned)(z - zq0) / C::NSQ) & 1u; };
  auto pslot = [&](int z) { return (int)((unsigned)(z - zp0) % C::NSP); };

  __shared__ T s_mrt[MRT ? Lat::Q : 1];
  if constexpr (MRT) {
    if (tid < Lat::Q) {
      constexpr MomentBasis<Lat> B = make_moment_basis<Lat>();
      s_mrt[tid] = I.mrt ? I.mrt[tid] : T(double(p.inv_tau) / B.n2[tid]);
    }
  }
  if (tid == 0) {
    for (int s = 0; s < C::NSQ; s++) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int z) {  // thread 0 only
    const int s = qslot(z);
    mbar_expect_tx(&bars[s], C::tx_bytes);
    tma_load_4d(sQ(s), qmap, x0, y0, z + zoff, 0, &bars[s]);
  };
  bool late = false;
  auto wait = [&](int z) { late |= !mbar_wait(&bars[qslot(z)], qpar(z)); };
  auto abort_block = [&]() {
    // a wait ran out: report, and let thread 0 drain the copies still in
    // flight (bounded) before the block exits
    if (tid == 0) {
      atomicExch(err, DEV_ERR_TMA_TIMEOUT);
      for (int s = 0; s < C::NSQ; s++) (void)mbar_wait(&bars[s], 0), (void)mbar_wait(&bars[s], 1);
    }
  };

  // per-thread pull offsets (x fixed for the block; y fixed for a chunk of
  // planes, and set per tile on a single plane, where a block works through
  // tiles stacked along y: set_tile)
  const int ct = tid - C::CELL0;
  const int tx = ct % FTX, ty = ct / FTX;
  const int x = x0 + tx;
  int y = y0 + ty;
  bool cell = false;
  // source offsets within a plane for c_x, c_y in {-1, 0, 1} (index c + 1);
  // a lattice holds fewer than 2^31 cells, so 32-bit offsets suffice
  int colx[3] = {0, 0, 0};
  int rowy[3] = {0, 0, 0};
  // every cell of the tile lies GHOST or more away from the x and y faces:
  // its stores of u have no periodic images there (the same for the whole
  // block)
  bool tile_inner = false;
  auto set_tile = [&](int yt0) {  // tile rows yt0 .. yt0 + FTY - 1
    y = yt0 + ty;
    cell = ct >= 0 && ct < FTX * FTY && x < d.nx && y < d.ny;
    if (cell) {
      colx[0] = wrap_inc(x, d.nx);
      colx[1] = x;
      colx[2] = wrap_dec(x, d.nx);
      rowy[0] = wrap_inc(y, d.ny) * d.nx;
      rowy[1] = y * d.nx;
      rowy[2] = wrap_dec(y, d.ny) * d.nx;
    }
    tile_inner = x0 >= GHOST && x0 + FTX <= d.nx - GHOST && yt0 >= GHOST &&
                 yt0 + FTY <= d.ny - GHOST;
  };
  set_tile(y0);
  const int nxy = d.nx * d.ny;
  const int ic = (ty + 1) * RX1 + (tx + 1);

  // OBS: running sums of this thread (float-float for FP32), the
  // non-finite count and the maximum of |u|
  typename AccFor<T>::type oacc[OBS_SLOTS - 1];
  int onbad = 0;
  T oumax = T(0);
  const ObsConst<T> oconst(p, 1.0 / 3.0);
  // OBS: the Q terms of the tile cell (if any) of ring-phase thread t on
  // plane zr (rows from yt0), whose Q box is in sq, the plane above in sqp
  auto obs_ring = [&](int t, int zr, int yt0, const T* sq, const T* sqp) {
    int cx, cy, c;
    ring_cell(t, cx, cy, c);
    if (cx < 0 || cx >= FTX || cy < 0 || cy >= FTY || x0 + cx >= d.nx || yt0 + cy >= d.ny ||
        zr < z0 || zr >= z1)
      return;
    const T* qc = sq + box_at(cx, cy);
    const int64_t st[3] = {1, BXW, (int64_t)(sqp - sq)};
    obs_q_terms<DIM>(qc, (int64_t)BA, st, oconst, oacc, onbad);
  };

  // The populations of the next plane are pulled into registers (gn) as
  // soon as the current plane is done, so their loads are in flight while
  // the block computes the next plane's stress.
  constexpr bool kPacked = std::is_same<T, float>::value;
  constexpr int NP = (Lat::Q - 1) / 2;
  CellPops<Lat, T> gn;
  auto pull_next = [&](int z) {
    if (!cell) return;
    int plane[3];
    plane[1] = z * nxy;
    plane[0] = DIM == 3 ? wrap_inc(z, d.nz) * nxy : plane[1];
    plane[2] = DIM == 3 ? wrap_dec(z, d.nz) * nxy : plane[1];
    // 32-bit element offsets within a population plane; the plane of
    // population i starts i * n elements after gin
    const unsigned n32 = (unsigned)d.n;
    auto ld = [&](int i) {
      const unsigned off = (unsigned)(plane[Lat::c(i, 2) + 1] + rowy[Lat::c(i, 1) + 1] +
                                      colx[Lat::c(i, 0) + 1]);
      if constexpr (PERSIST)
        return T(__ldcg(gin + pop_off<IX32>(i, n32, off)));
      else
        return T(__ldg(gin + pop_off<IX32>(i, n32, off)));
    };
    if constexpr (kPacked) {
      gn.g0 = ld(0);
#pragma unroll
      for (int q = 0; q < NP; q++) {
        const int i = pair_first<Lat>(q);
        gn.gp[q] = make_float2(ld(i), ld(Lat::opp(i)));
      }
    } else {
#pragma unroll
      for (int i = 0; i < Lat::Q; i++) gn.g[i] = ld(i);
    }
  };

  // moments, collision and stores of this thread's cell on plane z, whose
  // stress is in Pi slot ps (the planes above and below in the slots of
  // z -+ 1)
  // F at the tile cell with ring index icc from the stress of its plane in
  // Pi slot ps (the planes below and above in slots psm, psp)
  auto force_cell = [&](int icc, int ps, int psm, int psp, T F[3]) {
    const T* Pc = sP(ps);
    const T* Pm = sP(psm);
    const T* Pp = sP(psp);
    const int ic = icc;
    F[0] = F[1] = F[2] = T(0);
    if constexpr (ISO) {
      // F_a = 3 sum_i w_i sum_b c_ib Pi_ab(x + c_i)
#pragma unroll
      for (int i = 1; i < Lat::Q; i++) {
        const T* Pi = Lat::c(i, 2) == 0 ? Pc : (Lat::c(i, 2) > 0 ? Pp : Pm);
        const int oi = ic + Lat::c(i, 0) + Lat::c(i, 1) * RX1;
        const T w3 = T(3.0 * Lat::w(i));
#pragma unroll
        for (int a = 0; a < DIM; a++) {
          T sb = T(0);
#pragma unroll
          for (int b = 0; b < DIM; b++)
            if (Lat::c(i, b) != 0) sb = fma_(T(Lat::c(i, b)), Pi[(a * DIM + b) * A1 + oi], sb);
          F[a] = fma_(w3, sb, F[a]);
        }
      }
    } else {
#pragma unroll
      for (int a = 0; a < DIM; a++) {
        // F_a = sum_b [Pi_ab(x + e_b) - Pi_ab(x - e_b)] / 2
        T s = Pc[(a * DIM + 0) * A1 + ic + 1] - Pc[(a * DIM + 0) * A1 + ic - 1];
        s += Pc[(a * DIM + 1) * A1 + ic + RX1] - Pc[(a * DIM + 1) * A1 + ic - RX1];
        if (DIM == 3) s += Pp[(a * DIM + 2) * A1 + ic] - Pm[(a * DIM + 2) * A1 + ic];
        F[a] = s * T(0.5);
      }
    }
  };

  // moments, collision and stores of this thread's cell on plane z, with the
  // force F of the cell
  auto lb_cell_F = [&](int z, T F[3]) {
    if (!cell) return;
    if constexpr (OBS) {
      T rho, u[3];
      if constexpr (kPacked) {
        float g0 = gn.g0, drho;
        float2 gp[NP];
        onbad += !isfinite(g0);
#pragma unroll
        for (int q = 0; q < NP; q++) {
          gp[q] = gn.gp[q];
          onbad += !isfinite(gp[q].x) + !isfinite(gp[q].y);
        }
        moments_pairs<Lat>(g0, gp, F, p.rho0, rho, drho, u);
      } else {
        T g[Lat::Q];
#pragma unroll
        for (int i = 0; i < Lat::Q; i++) {
          g[i] = gn.g[i];
          onbad += !isfinite(g[i]);
        }
        moments<Lat, T>(g, F, p, rho, u);
      }
      obs_u_terms(rho, u, oacc, oumax);
      if (z + 1 < z1) pull_next(z + 1);
      return;
    }
    const unsigned o = (unsigned)(z * nxy + rowy[1] + x);
    const unsigned n32 = (unsigned)d.n;
    T rho, u[3];
    if constexpr (MRT) {
      T g[Lat::Q];
      if constexpr (kPacked) {
        g[0] = gn.g0;
#pragma unroll
        for (int q = 0; q < NP; q++) {
          g[pair_first<Lat>(q)] = gn.gp[q].x;
          g[Lat::opp(pair_first<Lat>(q))] = gn.gp[q].y;
        }
      } else {
#pragma unroll
        for (int i = 0; i < Lat::Q; i++) g[i] = gn.g[i];
      }
      moments<Lat, T>(g, F, p, rho, u);
      collide_mrt<Lat, T>(g, rho, u, F, p, s_mrt);
#pragma unroll
      for (int i = 0; i < Lat::Q; i++) gout[pop_off<IX32>(i, n32, o)] = G(g[i]);
    } else if constexpr (kPacked) {
      float g0 = gn.g0, drho;
      float2 gp[NP];
#pragma unroll
      for (int q = 0; q < NP; q++) gp[q] = gn.gp[q];
      moments_pairs<Lat>(g0, gp, F, p.rho0, rho, drho, u);
      collide_bgk_pairs<Lat>(g0, gp, rho, drho, u, F, p.inv_tau, p.guo);
      gout[o] = g0;
#pragma unroll
      for (int q = 0; q < NP; q++) {
        const int i = pair_first<Lat>(q);
        gout[pop_off<IX32>(i, n32, o)] = gp[q].x;
        gout[pop_off<IX32>(Lat::opp(i), n32, o)] = gp[q].y;
      }
    } else {
      T g[Lat::Q];
#pragma unroll
      for (int i = 0; i < Lat::Q; i++) g[i] = gn.g[i];
      moments<Lat, T>(g, F, p, rho, u);
      collide_bgk<Lat, T>(g, rho, u, F, p);
#pragma unroll
      for (int i = 0; i < Lat::Q; i++) gout[pop_off<IX32>(i, n32, o)] = G(g[i]);
    }
    if (tile_inner && (DIM == 2 || (z >= GHOST && z < d.nz - GHOST)))
      store_interior<T, DIM>(U, x, y, z, u);
    else
      store_with_images<T, DIM, DIM>(U, d, x, y, z, u);
    if (z + 1 < z1) pull_next(z + 1);
  };

  // the same with F formed here from the stress of the plane (single plane)
  auto lb_cell = [&](int z, int ps) {
    if (!cell) return;
    T F[3];
    force_cell(ic, ps, ps, ps, F);
    lb_cell_F(z, F);
  };

  if constexpr (DIM == 2) {
    // tile.z1 tiles stacked along y: tile t (rows y0 + FTY t ..) has its Q box
    // in slot t & 1 and its stress in Pi slot t & 1; the copy of tile t + 1
    // is in flight while tile t is computed
    const int nt = tile.z1;
    auto issue2 = [&](int t) {  // thread 0 only
      const int sl = t & 1;
      mbar_expect_tx(&bars[sl], C::tx_bytes);
      tma_load_4d(sQ(sl), qmap, x0, y0 + FTY * t, 0, 0, &bars[sl]);
    };
    if (tid == 0) issue2(0);
    pull_next(0);
    for (int t = 0; t < nt; t++) {
      // tile t + 1 goes to the slot of tile t - 1, whose ring phase every
      // thread finished before the previous barrier
      if (tid == 0 && t + 1 < nt) issue2(t + 1);
      late |= !mbar_wait(&bars[t & 1], (unsigned)(t >> 1) & 1u);
      if (tid < C::RING_T) {
        stress_ring_cell<Lat, T, ISO>(tid, sQ(t & 1), sQ(t & 1), sQ(t & 1), sP(t & 1), p);
        if constexpr (OBS) obs_ring(tid, 0, y0 + FTY * t, sQ(t & 1), sQ(t & 1));
      }
      if (__syncthreads_or(late)) {
        abort_block();
        return false;
      }
      lb_cell(0, t & 1);
      if (t + 1 < nt) {
        set_tile(y0 + FTY * (t + 1));
        pull_next(0);
      }
    }
  } else {
    if (tid == 0)
      for (int z = z0 - 2; z <= z0 + 1; z++) issue(z);
    pull_next(z0);
    wait(z0 - 2);
    wait(z0 - 1);
    wait(z0);
    if (tid < C::RING_T)
      stress_ring_cell<Lat, T, ISO>(tid, sQ(qslot(z0 - 1)), sQ(qslot(z0 - 2)), sQ(qslot(z0)),
                               sP(pslot(z0 - 1)), p);
    if (__syncthreads_or(late)) {
      abort_block();
      return false;
    }
    if (tid == 0) issue(z0 + 2);
    wait(z0 + 1);
    if (tid < C::RING_T) {
      stress_ring_cell<Lat, T, ISO>(tid, sQ(qslot(z0)), sQ(qslot(z0 - 1)), sQ(qslot(z0 + 1)),
                               sP(pslot(z0)), p);
      if constexpr (OBS) obs_ring(tid, z0, y0, sQ(qslot(z0)), sQ(qslot(z0 + 1)));
    }
    // the first copy of the loop (plane z0 + 3) goes to the slot of Q(z0 - 1),
    // which the ring phase of plane z0 just above still reads
    __syncthreads();
    // After the barrier of plane z, the warps without a tile cell form the
    // force F(z) of the tile's cells into F slot z & 1, while the cell warps
    // update plane z - 1 with F(z - 1), formed one plane earlier.  F(z) reads
    // Pi(z - 1 .. z + 1), which the ring phase of plane z + 2 (the slot of
    // Pi(z - 2)) leaves alone; F slot z & 1 held F(z - 2), which the cell
    // warps read before the previous barrier.
    T* sF = reinterpret_cast<T*>(smem + C::off_f);
    constexpr int NT = FTX * FTY;
    auto force_plane = [&](int z) {  // threads NT .. THREADS - 1
      T* Fo = sF + (z & 1) * (C::f_slot / sizeof(T));
      for (int k = tid - NT; k < NT; k += C::THREADS - NT) {
        T F[3];
        force_cell((k / FTX + 1) * RX1 + (k % FTX) + 1, pslot(z), pslot(z - 1), pslot(z + 1), F);
        Fo[k] = F[0], Fo[NT + k] = F[1], Fo[2 * NT + k] = F[2];
      }
    };
    auto cell_plane = [&](int z) {  // threads 0 .. NT - 1
      const T* Fi = sF + (z & 1) * (C::f_slot / sizeof(T));
      T F[3] = {Fi[ct], Fi[NT + ct], Fi[2 * NT + ct]};
      lb_cell_F(z, F);
    };
    for (int z = z0; z < z1; z++) {
      // Q(z+3) reuses the slot of Q(z-1), last read by the ring phase of
      // plane z, which every thread finished before the previous barrier
      if (tid == 0 && z + 3 <= z1 + 1) issue(z + 3);
      wait(z + 2);
      if (tid < C::RING_T) {
        stress_ring_cell<Lat, T, ISO>(tid, sQ(qslot(z + 1)), sQ(qslot(z)), sQ(qslot(z + 2)),
                                 sP(pslot(z + 1)), p);
        if constexpr (OBS) obs_ring(tid, z + 1, y0, sQ(qslot(z + 1)), sQ(qslot(z + 2)));
      }
      if (__syncthreads_or(late)) {
        abort_block();
        return false;
      }
      if (tid >= NT)
        force_plane(z);
      else if (z > z0)
        cell_plane(z - 1);
    }
    __syncthreads();  // F(z1 - 1) is complete
    if (tid < NT) cell_plane(z1 - 1);
  }
  if constexpr (OBS) {
    __shared__ double s_obs[32];
    obs_block_out<T>(oacc, onbad, oumax, s_obs, obs_partial);
  }
  // every copy issued was waited on: retire the barriers, so that the
  // block's next tile (persistent kernel) can initialise them again
  __syncthreads();
  if (tid == 0)
    for (int s = 0; s < C::NSQ; s++) mbar_inval(&bars[s]);
  (void)NPI;
  return true;
}

// pdl_early: the launch fits in one wave of resident blocks, so the next
// kernel of the stream (launched with programmatic serialisation) may be
// scheduled at once and wait for this one on the device; otherwise its
// blocks would hold SM slots that this kernel's later waves need.
template <class Lat, class T, class G, bool MRT, bool ISO, bool IX32, bool OBS = false>
__global__ void __launch_bounds__(LbCfg<Lat, T>::THREADS, LbCfg<Lat, T>::MINB)
    k_fused_lb(const InstDev<T, G>* __restrict__ insts,
               const CUtensorMap* __restrict__ qmaps,
               const TileRef* __restrict__ tiles, int cur,
               unsigned* __restrict__ err, double* __restrict__ obs_partial, int pdl_early) {
  grid_dep_wait();
  if (pdl_early) grid_dep_trigger();
  (void)fused_lb_tile<Lat, T, G, MRT, ISO, IX32, OBS>(tiles[blockIdx.x], insts, qmaps, cur, err,
                                                      obs_partial);
}


// ---------------------------------------------------------------------------
// Beris-Edwards kernel
// ---------------------------------------------------------------------------
template <class Lat, class T>
struct BeCfg {
  static constexpr int DIM = Lat::DIM;
  // Plane slots, sized so that one barrier per plane suffices: at plane z
  // the predictor of z+1 and the copies of plane z+3 may overlap slower
  // threads still correcting plane z-1 (which reads Q^n(z-1), u(z-2..z) and
  // Q^P(z-2..z)).
  // predictor on threads [0, RING_T), corrector on [CELL0, CELL0 + CELL_T)
  static constexpr int RING_T = A1;
  static constexpr int CELL_T = FTX * FTY;
  static constexpr int CELL0 = 0;
  static constexpr int THREADS = 352;  // 11 warps
  static constexpr int MINB = sizeof(T) == 4 ? 2 : 1;
  static_assert(THREADS >= RING_T && THREADS >= CELL0 + CELL_T, "block too small");
  // On a single plane the slots hold stacked tiles instead: the copies of
  // tile t + 1 are in flight while tile t is computed, and they may not
  // overwrite tile t - 1, whose corrector can still run (three Q^n and u
  // slots, two Q^P slots).
  static constexpr int NSQ = DIM == 3 ? 5 : 3;   // Q^n plane slots
  static constexpr int NSU = DIM == 3 ? 6 : 3;   // u plane slots
  static constexpr int NSP = DIM == 3 ? 4 : 2;   // Q^P plane slots
  static constexpr size_t q_slot = align128<T>(sizeof(T) * 5 * BA);
  static constexpr size_t u_slot = align128<T>(sizeof(T) * DIM * BA);
  static constexpr size_t p_slot = align128<T>(sizeof(T) * 5 * A1);
  static constexpr size_t off_u = NSQ * q_slot;
  static constexpr size_t off_p = off_u + NSU * u_slot;
  static constexpr size_t off_bar = off_p + NSP * p_slot;
  static constexpr size_t bytes = off_bar + 8 * (NSQ + NSU);
  static constexpr uint32_t q_tx = sizeof(T) * 5 * BA;
  static constexpr uint32_t u_tx = sizeof(T) * DIM * BA;
};

// u and G2[a][b] = 2 d_b u_a (plain differences, twice the central
// difference) at box offset o (z neighbours from the planes above and
// below); the caller halves the factors that multiply G2, which gives the
// same products as the gradient with its halved coefficients, exactly
template <class Lat, class T, bool ISO>
__device__ __forceinline__ void box_ugrad(const T* __restrict__ c,
                                          const T* __restrict__ m,
                                          const T* __restrict__ pp, int o,
                                          T u[3], T G2[3][3]) {
  constexpr int DIM = Lat::DIM;
  // FP32: u_x and u_y as a packed pair
  constexpr int AP = (std::is_same<T, float>::value && !ISO) ? 2 : 0;
  if constexpr (AP == 2) {
    const float* F0 = c;
    const float* F1 = c + BA;
    const float2 gx = psub(pk(F0[o + 1], F1[o + 1]), pk(F0[o - 1], F1[o - 1]));
    const float2 gy = psub(pk(F0[o + BXW], F1[o + BXW]), pk(F0[o - BXW], F1[o - BXW]));
    u[0] = F0[o], u[1] = F1[o];
    G2[0][0] = gx.x, G2[1][0] = gx.y;
    G2[0][1] = gy.x, G2[1][1] = gy.y;
    if (DIM == 3) {
      const float2 gz = psub(pk(pp[o], pp[BA + o]), pk(m[o], m[BA + o]));
      G2[0][2] = gz.x, G2[1][2] = gz.y;
    } else {
      G2[0][2] = G2[1][2] = 0.0f;
    }
  }
#pragma unroll
  for (int a = AP; a < 3; a++) {
    if (ISO && a < DIM) {
      const int oa = a * BA + o;
      auto at = [&](int dx, int dy, int dz) {
        const T* pl = dz == 0 ? c : (dz > 0 ? pp : m);
        return pl[oa + dx + dy * BXW];
      };
      T d2[3], unused;
      u[a] = c[oa];
      lattice_stencil<Lat, T>(at, u[a], d2, unused);
      G2[a][0] = d2[0];
      G2[a][1] = d2[1];
      G2[a][2] = d2[2];
    } else if (a < DIM) {
      const T* F = c + a * BA;
      u[a] = F[o];
      G2[a][0] = F[o + 1] - F[o - 1];
      G2[a][1] = F[o + BXW] - F[o - BXW];
      G2[a][2] = DIM == 3 ? (pp + a * BA)[o] - (m + a * BA)[o] : T(0);
    } else {
      u[a] = T(0);
      G2[a][0] = G2[a][1] = G2[a][2] = T(0);
    }
  }
}

// Q, twice the advection, u.(2 dQ) = 2 u.grad Q, and the Laplacian at
// offset o of a plane array c (row stride row, component stride comp; z
// neighbours in m and pp).  The differences are kept plain (twice the
// central difference); the caller takes the advection with the factor -1/2
// (be_rhs_adv), which is exact.
template <class Lat, class T, bool ISO>
__device__ __forceinline__ void stencil_adv(const T* __restrict__ c, const T* __restrict__ m,
                                            const T* __restrict__ pp, int o, int row, int comp,
                                            const T u[3], T q[5], T adv[5], T lap[5]) {
  constexpr int DIM = Lat::DIM;
  const T u0 = u[0], u1 = u[1], u2 = u[2];
  // FP32: components (0, 1) and (2, 3) as packed pairs (same operations in
  // the same order as the scalar form, lane by lane)
  constexpr int KP = (std::is_same<T, float>::value && !ISO) ? 4 : 0;
  if constexpr (KP == 4) {
    const float2 a0 = bc(u0), a1 = bc(u1), a2 = bc(u2);
#pragma unroll
    for (int k = 0; k < 4; k += 2) {
      const float* F0 = c + k * comp;
      const float* F1 = F0 + comp;
      const float2 v = pk(F0[o], F1[o]);
      const float2 xp = pk(F0[o + 1], F1[o + 1]), xm = pk(F0[o - 1], F1[o - 1]);
      const float2 yp = pk(F0[o + row], F1[o + row]), ym = pk(F0[o - row], F1[o - row]);
      float2 a = pfma(a0, psub(xp, xm), pmul(a1, psub(yp, ym)));
      float2 sum = padd(padd(xp, xm), padd(yp, ym));
      if (DIM == 3) {
        const float2 zp = pk(pp[k * comp + o], pp[(k + 1) * comp + o]);
        const float2 zm = pk(m[k * comp + o], m[(k + 1) * comp + o]);
        a = pfma(a2, psub(zp, zm), a);
        sum = padd(sum, padd(zp, zm));
      }
      const float2 l = pfma(bc(-2.0f * DIM), v, sum);
      q[k] = v.x, q[k + 1] = v.y;
      adv[k] = a.x, adv[k + 1] = a.y;
      lap[k] = l.x, lap[k + 1] = l.y;
    }
  }
#pragma unroll
  for (int k = KP; k < 5; k++) {
    if constexpr (ISO) {
      const int ok = k * comp + o;
      auto at = [&](int dx, int dy, int dz) {
        const T* pl = dz == 0 ? c : (dz > 0 ? pp : m);
        return pl[ok + dx + dy * row];
      };
      T d2[3];
      q[k] = c[ok];
      lattice_stencil<Lat, T>(at, q[k], d2, lap[k]);
      T a = fma_(u0, d2[0], u1 * d2[1]);
      if (DIM == 3) a = fma_(u2, d2[2], a);
      adv[k] = a;
      continue;
    }
    const T* F = c + k * comp;
    const T v = F[o], xp = F[o + 1],
            xm = F[o - 1];
    const T yp = F[o + row], ym = F[o - row];
    q[k] = v;
    T a = fma_(u0, xp - xm, u1 * (yp - ym));
    T zp = T(0), zm = T(0);
    if (DIM == 3) {
      zp = (pp + k * comp)[o];
      zm = (m + k * comp)[o];
      a = fma_(u2, zp - zm, a);
    }
    adv[k] = a;
    lap[k] = lap_points<T, DIM>(v, xp, xm, yp, ym, zp, zm);
  }
}

// Returns false when a bounded wait ran out (the error word is set and the
// block's copies are drained).
template <class Lat, class T, class G, bool ISO>
__device__ __forceinline__ bool fused_be_tile(const TileRef tile,
                                              const InstDev<T, G>* __restrict__ insts,
                                              const CUtensorMap* __restrict__ qmaps,
                                              const CUtensorMap* __restrict__ umaps, int cur,
                                              unsigned* __restrict__ err) {
  using C = BeCfg<Lat, T>;
  constexpr int DIM = Lat::DIM;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* qbar = reinterpret_cast<uint64_t*>(smem + C::off_bar);
  uint64_t* ubar = qbar + C::NSQ;
  auto sQ = [&](int s) { return reinterpret_cast<T*>(smem + s * C::q_slot); };
  auto sU = [&](int s) { return reinterpret_cast<T*>(smem + C::off_u + s * C::u_slot); };
  auto sQP = [&](int s) { return reinterpret_cast<T*>(smem + C::off_p + s * C::p_slot); };

  const InstDev<T, G>& I = insts[tile.inst];
  const Dims d = I.d;
  const Par<T> p = I.p;
  // the factors of Eq. 1 that multiply the velocity gradient, halved: the
  // gradient arrives doubled (box_ugrad)
  Par<T> p2 = p;
  p2.hp = p.hp * T(0.5);
  p2.hm = p.hm * T(0.5);
  p2.x2 = p.x2 * T(0.5);
  p2.x29 = p.x29 * T(0.5);
  const Field<T> Qout = I.q[cur ^ 1];
  const int zoff = Qout.L.zoff;
  const CUtensorMap* qmap = &qmaps[2 * tile.inst + cur];
  const CUtensorMap* umap = &umaps[tile.inst];

  const int tid = threadIdx.x;
  const int x0 = tile.x0, y0 = tile.y0;
  const int z0 = tile.z0;
  const int z1 = DIM == 3 ? tile.z1 : 1;
  // Plane z of Q^n and u lives in slot (z - z0 + 2) mod NSQ (NSU), Q^P of
  // plane z in slot (z - z0 + 1) mod NSP.  The loop carries the slots of its
  // current plane and steps them with slot_add; every plane's copy is waited
  // on once, in z order, so one phase bit per slot (flipped at each wait)
  // gives the parity to wait for.

  if (tid == 0) {
    for (int s = 0; s < C::NSQ + C::NSU; s++) mbar_init(&qbar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // copies of plane z of the tile at rows yt0 .. into Q slot s and u slot t
  // (thread 0)
  auto issue = [&](int z, int s, int t, int yt0) {
    mbar_expect_tx(&qbar[s], C::q_tx);
    tma_load_4d(sQ(s), qmap, x0, yt0, z + zoff, 0, &qbar[s]);
    mbar_expect_tx(&ubar[t], C::u_tx);
    tma_load_4d(sU(t), umap, x0, yt0, z + zoff, 0, &ubar[t]);
  };
  bool late = false;
  uint32_t qph = 0, uph = 0;  // phase bit per slot
  auto wait = [&](int s, int t) {
    late |= !mbar_wait(&qbar[s], (qph >> s) & 1u);
    late |= !mbar_wait(&ubar[t], (uph >> t) & 1u);
    qph ^= 1u << s;
    uph ^= 1u << t;
  };
  auto abort_block = [&]() {
    if (tid == 0) {
      atomicExch(err, DEV_ERR_TMA_TIMEOUT);
      for (int s = 0; s < C::NSQ + C::NSU; s++)
        (void)mbar_wait(&qbar[s], 0), (void)mbar_wait(&qbar[s], 1);
    }
  };

  // predictor on the ring cell of ring-phase thread t of a plane whose Q^n
  // and u slots are sq, su (the planes below and above in sqm, sqp, sum,
  // sup): R(Q^n) and Q^P = Q^n + R into Q^P slot spo
  auto predict = [&](int t, int sq, int sqm, int sqp, int su, int sum, int sup, int spo) {
    int cx, cy, c;
    ring_cell(t, cx, cy, c);
    const int o = box_at(cx, cy);
    T q[5], adv[5], lap[5], u[3], G2[3][3], r[5];
    box_ugrad<Lat, T, ISO>(sU(su), sU(sum), sU(sup), o, u, G2);
    stencil_adv<Lat, T, ISO>(sQ(sq), sQ(sqm), sQ(sqp), o, BXW, BA, u, q, adv, lap);
    be_rhs_adv<T>(q, adv, lap, G2, p2, r, T(-0.5));
    T* qpo = sQP(spo);
    if constexpr (std::is_same<T, float>::value) {
      // components (0, 1) and (2, 3) as packed pairs
      const float2 a = padd(pk(q[0], q[1]), pk(r[0], r[1]));
      const float2 b = padd(pk(q[2], q[3]), pk(r[2], r[3]));
      qpo[c] = a.x, qpo[A1 + c] = a.y;
      qpo[2 * A1 + c] = b.x, qpo[3 * A1 + c] = b.y;
      qpo[4 * A1 + c] = q[4] + r[4];
    } else {
#pragma unroll
      for (int k = 0; k < 5; k++) qpo[k * A1 + c] = q[k] + r[k];
    }
  };

  // corrector threads: one tile cell each (on a single plane, of the tile
  // at rows yt0 .., set per stacked tile)
  const int ct = tid - C::CELL0;
  const int tx = ct % FTX, ty = ct / FTX;
  const int x = x0 + tx;
  int y = y0 + ty;
  bool cell = ct >= 0 && ct < C::CELL_T && x < d.nx && y < d.ny;
  auto set_tile = [&](int yt0) {
    y = yt0 + ty;
    cell = ct >= 0 && ct < C::CELL_T && x < d.nx && y < d.ny;
  };
  const int ic = (ty + 1) * RX1 + (tx + 1);
  const int o2 = box_at(tx, ty);

  // corrector at the tile cell of this thread on plane z, whose Q^n, u and
  // Q^P slots are sq, su, sp (neighbouring planes in sum, sup, spm, spp)
  auto correct = [&](int z, int sq, int su, int sum, int sup, int sp, int spm, int spp) {
    if (!cell) return;
    T qp[5], adv[5], lap[5], u[3], G2[3][3], r2[5];
    box_ugrad<Lat, T, ISO>(sU(su), sU(sum), sU(sup), o2, u, G2);
    stencil_adv<Lat, T, ISO>(sQP(sp), sQP(spm), sQP(spp), ic, RX1, A1, u, qp, adv, lap);
    be_rhs_adv<T>(qp, adv, lap, G2, p2, r2, T(-0.5));
    // Q^{n+1} = Q^n + [R(Q^n) + R(Q^P)]/2 = [Q^n + Q^P + R(Q^P)]/2, since
    // Q^P = Q^n + R(Q^n)
    const T* qn = sQ(sq);
    T out[5];
    if constexpr (std::is_same<T, float>::value) {
      // components (0, 1) and (2, 3) as packed pairs, lane by lane the
      // same operations as the scalar form
      const float2 h = bc(0.5f);
#pragma unroll
      for (int k = 0; k < 4; k += 2) {
        const float2 v = pmul(padd(padd(pk(qn[k * BA + o2], qn[(k + 1) * BA + o2]),
                                        pk(qp[k], qp[k + 1])),
                                   pk(r2[k], r2[k + 1])),
                              h);
        out[k] = v.x, out[k + 1] = v.y;
      }
      out[4] = (qn[4 * BA + o2] + qp[4] + r2[4]) * 0.5f;
    } else {
#pragma unroll
      for (int k = 0; k < 5; k++) out[k] = (qn[k * BA + o2] + qp[k] + r2[k]) * T(0.5);
    }
    store_with_images<T, 5, DIM>(Qout, d, x, y, z, out);
  };

  if constexpr (DIM == 2) {
    // tile.z1 tiles stacked along y: tile t (rows y0 + FTY t ..) has its Q^n
    // and u boxes in slots t mod 3 and its Q^P in slot t & 1
    const int nt = tile.z1;
    if (tid == 0) issue(0, 0, 0, y0);
    int sq = 0;  // Q^n and u slot of tile t
    for (int t = 0; t < nt; t++) {
      // tile t + 1 goes to the slots of tile t - 2, whose predictor and
      // corrector every thread finished before the previous barrier
      const int sn = slot_add<3>(sq, 1);
      if (tid == 0 && t + 1 < nt) issue(0, sn, sn, y0 + FTY * (t + 1));
      wait(sq, sq);
      if (tid < C::RING_T) predict(tid, sq, sq, sq, sq, sq, sq, t & 1);
      if (__syncthreads_or(late)) {
        abort_block();
        return false;
      }
      set_tile(y0 + FTY * t);
      correct(0, sq, sq, sq, sq, t & 1, t & 1, t & 1);
      sq = sn;
    }
  } else {
    constexpr int NQ = C::NSQ, NU = C::NSU, NP = C::NSP;
    // planes z0-2 .. z0+2 go to Q and u slots 0..4
    if (tid == 0)
      for (int k = 0; k <= 4; k++) issue(z0 - 2 + k, k, k, y0);
    wait(0, 0);
    wait(1, 1);
    wait(2, 2);
    if (tid < C::RING_T) predict(tid, 1, 0, 2, 1, 0, 2, 0);  // plane z0-1
    if (__syncthreads_or(late)) {
      abort_block();
      return false;
    }
    wait(3, 3);
    if (tid < C::RING_T) predict(tid, 2, 1, 3, 2, 1, 3, 1);  // plane z0
    // slots of plane z: Q^n sq, u su, Q^P sp
    int sq = 2, su = 2, sp = 1;
    for (int z = z0; z < z1; z++) {
      const int sq1 = slot_add<NQ>(sq, 1), sq2 = slot_add<NQ>(sq, 2);
      const int su1 = slot_add<NU>(su, 1), su2 = slot_add<NU>(su, 2);
      const int sp1 = slot_add<NP>(sp, 1);
      if (tid == 0 && z + 3 <= z1 + 1)
        issue(z + 3, slot_add<NQ>(sq, 3), slot_add<NU>(su, 3), y0);
      wait(sq2, su2);
      if (tid < C::RING_T) predict(tid, sq1, sq, sq2, su1, su, su2, sp1);  // plane z+1
      if (__syncthreads_or(late)) {
        abort_block();
        return false;
      }
      correct(z, sq, su, slot_add<NU>(su, NU - 1), su1, sp, slot_add<NP>(sp, NP - 1), sp1);
      sq = sq1;
      su = su1;
      sp = sp1;
    }
  }
  // every copy issued was waited on: retire the barriers (see fused_lb_tile)
  __syncthreads();
  if (tid == 0)
    for (int s = 0; s < C::NSQ + C::NSU; s++) mbar_inval(&qbar[s]);
  return true;
}

template <class Lat, class T, class G, bool ISO>
__global__ void __launch_bounds__(BeCfg<Lat, T>::THREADS, BeCfg<Lat, T>::MINB)
    k_fused_be(const InstDev<T, G>* __restrict__ insts,
               const CUtensorMap* __restrict__ qmaps,
               const CUtensorMap* __restrict__ umaps,
               const TileRef* __restrict__ tiles, int cur,
               unsigned* __restrict__ err, int pdl_early) {
  grid_dep_wait();
  if (pdl_early) grid_dep_trigger();
  (void)fused_be_tile<Lat, T, G, ISO>(tiles[blockIdx.x], insts, qmaps, umaps, cur, err);
}

// ---------------------------------------------------------------------------
// persistent form: several steps in one cooperative launch
// ---------------------------------------------------------------------------
// Every block stays resident (cooperative launch) and runs nsteps steps: in
// each, the lb phase and then the Beris-Edwards phase work through the
// tiles of the joint tile list, block b taking tiles b, b + G, b + 2G, ...
// (G = gridDim.x; the list is ordered so that neighbouring tiles run
// together), and a grid-wide barrier (grid_sync.cuh, bounded by wait_ns)
// separates the phases.  The tiles compute exactly what the two kernels
// compute.  (Handing the tiles out one by one from an atomic counter, to
// balance uneven tiles, was measured slower: each claim costs a round trip
// to L2 and two block barriers.)
struct PersistArgs {
  GridBarrier* bar;
  uint64_t wait_ns;
};

template <class Lat, class T>
struct PersistCfg {
  static constexpr int THREADS = LbCfg<Lat, T>::THREADS;
  static_assert(THREADS == BeCfg<Lat, T>::THREADS, "one block shape for both phases");
  static constexpr size_t bytes =
      LbCfg<Lat, T>::bytes > BeCfg<Lat, T>::bytes ? LbCfg<Lat, T>::bytes : BeCfg<Lat, T>::bytes;
  static constexpr int MINB = LbCfg<Lat, T>::MINB;
};

template <class Lat, class T, class G, bool ISO, bool IX32>
__global__ void __launch_bounds__(PersistCfg<Lat, T>::THREADS, PersistCfg<Lat, T>::MINB)
    k_fused_persistent(const InstDev<T, G>* __restrict__ insts,
                       const CUtensorMap* __restrict__ qmaps,
                       const CUtensorMap* __restrict__ umaps,
                       const TileRef* __restrict__ tiles, int ntiles, int cur0, int nsteps,
                       unsigned* __restrict__ err, PersistArgs pa) {
  unsigned gen = 0;
  int cur = cur0;
  for (int step = 0; step < nsteps; step++) {
#pragma unroll 1
    for (int ph = 0; ph < 2; ph++) {
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const bool ok =
            ph == 0 ? fused_lb_tile<Lat, T, G, false, ISO, IX32, false, true>(
                          tiles[t], insts, qmaps, cur, err, nullptr)
                    : fused_be_tile<Lat, T, G, ISO>(tiles[t], insts, qmaps, umaps, cur, err);
        if (!ok) return;
      }
      // the phase's global writes are read by TMA copies after the barrier
      fence_proxy_async_global();
      if (!grid_sync(pa.bar, gen, err, pa.wait_ns)) return;
      fence_proxy_async_global();
    }
    cur ^= 1;
  }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------

// Length of a column in chunk units: z planes on D3Q19, 32 x 8 tiles along
// y on a single plane (where a block works through tiles stacked along y).
template <class Lat>
__host__ inline int column_length(const Dims& d) {
  return Lat::DIM == 3 ? d.nz : (d.ny + FTY - 1) / FTY;
}

// Default chunk depth: enough blocks for several waves over the SMs while
// amortising the two-plane prologue of each chunk (D3Q19), or the wait for
// the first tile's copy (a single plane)
template <class Lat>
__host__ inline int fused_tz(const Dims& d, int64_t other_tiles) {
  const int len = column_length<Lat>(d);
  const int64_t columns = (int64_t)((d.nx + FTX - 1) / FTX) *
                          (Lat::DIM == 3 ? (d.ny + FTY - 1) / FTY : 1);
  const int lo = Lat::DIM == 3 ? 4 : 1;
  int tz = Lat::DIM == 3 ? 32 : 8;
  while (tz > lo && other_tiles + columns * ((len + tz - 1) / tz) < 1200) tz /= 2;
  return tz < len ? tz : len;
}

// tile list of one instance: chunk by chunk along z (tiles stacked along y
// on a single plane), x fastest within a chunk, so neighbouring blocks run
// together and share halos in L2.  On a single plane a tile's z0 is 0 and
// z1 the number of tiles stacked from y0.
template <class Lat>
__host__ inline void append_tiles(int inst, const Dims& d, int tz, bool taper,
                                  std::vector<TileRef>* out) {
  const std::vector<int> b = chunk_bounds(column_length<Lat>(d), tz, taper);
  for (size_t zc = 0; zc + 1 < b.size(); zc++) {
    if (Lat::DIM == 3) {
      for (int y0 = 0; y0 < d.ny; y0 += FTY)
        for (int x0 = 0; x0 < d.nx; x0 += FTX)
          out->push_back({inst, x0, y0, b[zc], b[zc + 1]});
    } else {
      for (int x0 = 0; x0 < d.nx; x0 += FTX)
        out->push_back({inst, x0, FTY * b[zc], 0, b[zc + 1] - b[zc]});
    }
  }
}

template <class K>
inline cudaError_t set_smem(K kernel, size_t bytes, unsigned long long* done_mask) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (*done_mask & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) *done_mask |= bit;
  return e;
}

// Blocks of `kernel` resident on the whole device at once (SMs times blocks
// per SM), found once per kernel and device; 0 if the query fails.
struct ResidentCache {
  int v[64];
  ResidentCache() {
    for (int& x : v) x = -1;
  }
};
template <class K>
inline int resident_blocks(K kernel, int threads, size_t smem, ResidentCache& c) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return 0;
  int* cache = c.v;
  if (cache[dev] < 0) {
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
            cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cache[dev] = sms * per_sm;
  }
  return cache[dev];
}

// A step kernel launched with programmatic stream serialisation (see
// grid_dep_wait): it may be scheduled while the previous kernel of the
// stream finishes, and waits for it on the device before its first global
// access.  Inside a stream capture the dependency becomes a programmatic
// edge of the graph.
template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int threads, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <class Lat, class T, class G, bool MRT, bool ISO, bool IX32>
cudaError_t launch_fused_lb_as(const InstDev<T, G>* insts, const CUtensorMap* qmaps,
                               const TileRef* tiles, int ntiles, int cur, unsigned* err,
                               cudaStream_t st) {
  static unsigned long long configured = 0;
  static ResidentCache resident;
  auto kernel = k_fused_lb<Lat, T, G, MRT, ISO, IX32>;
  constexpr int threads = LbCfg<Lat, T>::THREADS;
  constexpr size_t smem = LbCfg<Lat, T>::bytes;
  cudaError_t e = set_smem(kernel, smem, &configured);
  if (e != cudaSuccess) return e;
  const int early = ntiles <= resident_blocks(kernel, threads, smem, resident) ? 1 : 0;
  return launch_pdl(kernel, ntiles, threads, smem, st, insts, qmaps, tiles, cur, err,
                    (double*)nullptr, early);
}

// the observables of the current state (buffers cur) over the tiles given
// (standard stencils, 32-bit population offsets): per-block partial sums
// into partial[ntiles][OBS_SLOTS]
template <class Lat, class T, class G>
cudaError_t launch_fused_obs(const InstDev<T, G>* insts, const CUtensorMap* qmaps,
                             const TileRef* tiles, int ntiles, int cur, unsigned* err,
                             double* partial, cudaStream_t st) {
  static unsigned long long configured = 0;
  cudaError_t e = set_smem(k_fused_lb<Lat, T, G, false, false, true, true>, LbCfg<Lat, T>::bytes,
                           &configured);
  if (e != cudaSuccess) return e;
  k_fused_lb<Lat, T, G, false, false, true, true>
      <<<ntiles, LbCfg<Lat, T>::THREADS, LbCfg<Lat, T>::bytes, st>>>(insts, qmaps, tiles, cur,
                                                                      err, partial, 0);
  return cudaGetLastError();
}

// mrt: MRT collision; iso: isotropic stencils; ix32: every lattice of the
// launch has Q n < 2^32 (32-bit population offsets, taken by the BGK
// kernel with the standard stencils)
template <class Lat, class T, class G>
cudaError_t launch_fused_lb(const InstDev<T, G>* insts, const CUtensorMap* qmaps,
                            const TileRef* tiles, int ntiles, int cur, unsigned* err,
                            cudaStream_t st, bool mrt, bool iso, bool ix32) {
  if (iso)
    return mrt ? launch_fused_lb_as<Lat, T, G, true, true, false>(insts, qmaps, tiles, ntiles,
                                                                  cur, err, st)
               : launch_fused_lb_as<Lat, T, G, false, true, false>(insts, qmaps, tiles, ntiles,
                                                                   cur, err, st);
  if (mrt)
    return launch_fused_lb_as<Lat, T, G, true, false, false>(insts, qmaps, tiles, ntiles, cur,
                                                             err, st);
  return ix32 ? launch_fused_lb_as<Lat, T, G, false, false, true>(insts, qmaps, tiles, ntiles,
                                                                  cur, err, st)
              : launch_fused_lb_as<Lat, T, G, false, false, false>(insts, qmaps, tiles, ntiles,
                                                                   cur, err, st);
}

template <class Lat, class T, class G, bool ISO>
cudaError_t launch_fused_be_as(const InstDev<T, G>* insts, const CUtensorMap* qmaps,
                               const CUtensorMap* umaps, const TileRef* tiles, int ntiles,
                               int cur, unsigned* err, cudaStream_t st) {
  static unsigned long long configured = 0;
  static ResidentCache resident;
  auto kernel = k_fused_be<Lat, T, G, ISO>;
  constexpr int threads = BeCfg<Lat, T>::THREADS;
  constexpr size_t smem = BeCfg<Lat, T>::bytes;
  cudaError_t e = set_smem(kernel, smem, &configured);
  if (e != cudaSuccess) return e;
  const int early = ntiles <= resident_blocks(kernel, threads, smem, resident) ? 1 : 0;
  return launch_pdl(kernel, ntiles, threads, smem, st, insts, qmaps, umaps, tiles, cur, err,
                    early);
}

template <class Lat, class T, class G>
cudaError_t launch_fused_be(const InstDev<T, G>* insts, const CUtensorMap* qmaps,
                            const CUtensorMap* umaps, const TileRef* tiles, int ntiles,
                            int cur, unsigned* err, cudaStream_t st, bool iso) {
  return iso ? launch_fused_be_as<Lat, T, G, true>(insts, qmaps, umaps, tiles, ntiles, cur, err, st)
             : launch_fused_be_as<Lat, T, G, false>(insts, qmaps, umaps, tiles, ntiles, cur, err, st);
}

// Blocks of a cooperative launch of the persistent kernel: every block must
// be resident, so at most the SM count times the blocks per SM that fit
// (0 if the device cannot launch cooperatively).
template <class Lat, class T, class G>
int persistent_grid_max(bool iso, bool ix32) {
  int dev = 0, sms = 0, coop = 0, nb = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
    return 0;
  auto occ = [&](auto kernel) {
    static unsigned long long configured = 0;
    if (set_smem(kernel, PersistCfg<Lat, T>::bytes, &configured) != cudaSuccess) return -1;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
               &nb, kernel, PersistCfg<Lat, T>::THREADS, PersistCfg<Lat, T>::bytes) ==
                   cudaSuccess
               ? nb
               : -1;
  };
  int r;
  if (iso)
    r = occ(k_fused_persistent<Lat, T, G, true, false>);
  else
    r = ix32 ? occ(k_fused_persistent<Lat, T, G, false, true>)
             : occ(k_fused_persistent<Lat, T, G, false, false>);
  return r > 0 ? r * sms : 0;
}

// nsteps steps of every lattice of the tile list in one cooperative launch
// of `grid` blocks (at most persistent_grid_max); pa.bar must be zero (the
// caller clears it on the stream first)
template <class Lat, class T, class G>
cudaError_t launch_fused_persistent(const InstDev<T, G>* insts, const CUtensorMap* qmaps,
                                    const CUtensorMap* umaps, const TileRef* tiles, int ntiles,
                                    int cur, int nsteps, unsigned* err, PersistArgs pa, int grid,
                                    cudaStream_t st, bool iso, bool ix32) {
  void* args[] = {(void*)&insts, (void*)&qmaps, (void*)&umaps, (void*)&tiles, (void*)&ntiles,
                  (void*)&cur, (void*)&nsteps, (void*)&err, (void*)&pa};
  const void* k = iso ? (const void*)k_fused_persistent<Lat, T, G, true, false>
                      : (ix32 ? (const void*)k_fused_persistent<Lat, T, G, false, true>
                              : (const void*)k_fused_persistent<Lat, T, G, false, false>);
  return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(PersistCfg<Lat, T>::THREADS), args,
                                     PersistCfg<Lat, T>::bytes, st);
}

}  // namespace nlc
