// packed.cuh -- two-lane FP32 arithmetic for the FP32 step kernels.
//
// sm_100-family GPUs execute a float2 fused multiply-add, add or multiply
// (both lanes, each rounded to nearest like its scalar form) as ONE
// instruction.  The FMA pipe does the same work either way, but the step
// kernels are bound by instruction issue, so pairing independent lanes of
// arithmetic frees issue slots for their loads, stores and index math.
//
// On the host (tests compile the physics for the CPU), and in device passes
// for GPUs without the paired instructions, the pairs fall back to two
// scalar operations with the same rounding.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
#define NLC_PAIRED_FP32 1
#else
#define NLC_PAIRED_FP32 0
#endif

namespace nlc {

__host__ __device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }

__host__ __device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
#if NLC_PAIRED_FP32
  return __ffma2_rn(a, b, c);
#else
  return make_float2(std::fma(a.x, b.x, c.x), std::fma(a.y, b.y, c.y));
#endif
}

__host__ __device__ __forceinline__ float2 padd(float2 a, float2 b) {
#if NLC_PAIRED_FP32
  return __fadd2_rn(a, b);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}

// a - b as one fused multiply-add, fma(b, -1, a), exact like a subtraction
__host__ __device__ __forceinline__ float2 psub(float2 a, float2 b) {
#if NLC_PAIRED_FP32
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
#else
  return make_float2(a.x - b.x, a.y - b.y);
#endif
}

__host__ __device__ __forceinline__ float2 pmul(float2 a, float2 b) {
#if NLC_PAIRED_FP32
  return __fmul2_rn(a, b);
#else
  return make_float2(a.x * b.x, a.y * b.y);
#endif
}

// Index of the first velocity of the p-th opposite pair (i, opp(i)) with
// opp(i) > i, in the lattice's own ordering (the rest velocity is index 0).
template <class Lat>
__host__ __device__ constexpr int pair_first(int p) {
  int k = 0;
  for (int i = 1; i < Lat::Q; i++)
    if (Lat::opp(i) > i) {
      if (k == p) return i;
      k++;
    }
  return -1;
}

// rho and u of Eq. 6 from the deviations g_i = f_i - w_i rho0 held as the
// rest value g0 and NP = (q-1)/2 opposite pairs gp[p] = (g_i, g_opp(i)):
//   rho = rho0 + g0 + sum_p (gp.x + gp.y),
//   sum_i c_ia g_i = sum_p c_ia (gp.x - gp.y),
//   u = (sum_i c_i g_i + F/2) / rho.
template <class Lat>
__host__ __device__ __forceinline__ void moments_pairs(float g0, const float2* gp,
                                                       const float F[3], float rho0,
                                                       float& rho, float& drho, float u[3]) {
  constexpr int NP = (Lat::Q - 1) / 2;
  float2 s = gp[0];
#pragma unroll
  for (int p = 1; p < NP; p++) s = padd(s, gp[p]);
  drho = g0 + (s.x + s.y);
  rho = rho0 + drho;
#ifdef __CUDA_ARCH__
  const float inv = __fdividef(1.0f, rho);  // hardware reciprocal, 2 ulp, no slow path
#else
  const float inv = 1.0f / rho;
#endif
#pragma unroll
  for (int a = 0; a < 3; a++) {
    if (a >= Lat::DIM) {
      u[a] = 0.0f;
      continue;
    }
    float2 J = make_float2(0.0f, 0.0f);
    bool first = true;
#pragma unroll
    for (int p = 0; p < NP; p++) {
      const int c = Lat::c(pair_first<Lat>(p), a);
      if (c == 0) continue;
      if (first) {
        J = c > 0 ? gp[p] : make_float2(-gp[p].x, -gp[p].y);
        first = false;
      } else {
        J = c > 0 ? padd(J, gp[p]) : psub(J, gp[p]);
      }
    }
    u[a] = std::fma(F[a], 0.5f, J.x - J.y) * inv;
  }
}

// c_i.X of the first velocity of pair p as a packed (c_i.X, -c_i.X) from the
// packed axis values X2[a] = (X_a, -X_a); the sum starts at a positive
// component (every pair's first velocity has one in both lattices).
template <class Lat>
__host__ __device__ __forceinline__ float2 pair_dot(int i, const float2* X2) {
  float2 v = make_float2(0.0f, 0.0f);
  int start = -1;
#pragma unroll
  for (int a = 0; a < Lat::DIM; a++)
    if (start < 0 && Lat::c(i, a) > 0) start = a;
  v = X2[start];
#pragma unroll
  for (int a = 0; a < Lat::DIM; a++) {
    if (a == start) continue;
    const int c = Lat::c(i, a);
    if (c > 0) v = padd(v, X2[a]);
    if (c < 0) v = psub(v, X2[a]);
  }
  return v;
}

// BGK collision with the source term of Sec. 1.2.1 on the pair layout.
// For the pair (i, opp(i)) with v = c_i.u, f = c_i.F the post-collision
// deviation is
//   g_i* = (1 - 1/tau) g_i + w [C + v (A v + B f + R) + G f],
//   C = (drho - 3/2 rho u.u)/tau - 3 k u.F,  A = 9/2 rho/tau,  R = 3 rho/tau,
//   B = 9 k,  G = 3 k,  k = 1 - 1/(2 tau),
// and g_opp* is the same with (v, f) -> (-v, -f); one packed chain computes
// both lanes.  The rest population keeps only w0 C.
template <class Lat>
__host__ __device__ __forceinline__ void collide_bgk_pairs(float& g0, float2* gp, float rho,
                                                           float drho, const float u[3],
                                                           const float F[3], float inv_tau,
                                                           float guo) {
  constexpr int NP = (Lat::Q - 1) / 2;
  constexpr int D = Lat::DIM;
  const float uu = D == 3 ? std::fma(u[2], u[2], std::fma(u[1], u[1], u[0] * u[0]))
                          : std::fma(u[1], u[1], u[0] * u[0]);
  const float uF = D == 3 ? std::fma(u[2], F[2], std::fma(u[1], F[1], u[0] * F[0]))
                          : std::fma(u[1], F[1], u[0] * F[0]);
  const float C = std::fma(std::fma(-1.5f * rho, uu, drho), inv_tau, -3.0f * guo * uF);
  const float rt = rho * inv_tau;
  const float keep = 1.0f - inv_tau;
  g0 = std::fma(keep, g0, float(Lat::w(0)) * C);
  float2 U[3], Fp[3];
#pragma unroll
  for (int a = 0; a < D; a++) {
    U[a] = pk(u[a], -u[a]);
    Fp[a] = pk(F[a], -F[a]);
  }
  const float2 K2 = bc(keep);
#pragma unroll
  for (int p = 0; p < NP; p++) {
    const int i = pair_first<Lat>(p);
    const float w = float(Lat::w(i));
    const float2 v = pair_dot<Lat>(i, U);
    const float2 f = pair_dot<Lat>(i, Fp);
    float2 x = pfma(bc(4.5f * w * rt), v, bc(3.0f * w * rt));
    x = pfma(bc(9.0f * w * guo), f, x);
    x = pfma(v, x, bc(w * C));
    x = pfma(bc(3.0f * w * guo), f, x);
    gp[p] = pfma(K2, gp[p], x);
  }
}

}  // namespace nlc
