// adjoint_segment.cuh -- one checkpoint segment of the adjoint as two
// persistent kernels.
//
// A segment of len steps starts from a checkpointed state (g^0, Q^0) held in
// record slot 0.  The record kernel re-runs the segment's steps with the
// four stages of step_unfused.cuh (stress, lb, predict, correct) and keeps
// what the reverse sweep reads in per-step slots: g^j, Q^j, Pi^j, u^j and
// Q^{P,j}.  The reverse kernel then walks j = len-1 .. 0 through the five
// adjoint stages of adjoint.cuh (corrector and predictor evaluations, lb,
// stress, stencil transposes).  Every stage covers all cells before the next
// one starts; within a kernel the stages are separated by a grid-wide
// barrier instead of a kernel boundary, so one launch replaces 4 (record) or
// 5 (reverse) launches per step.  The kernels are launched cooperatively,
// which guarantees that every block is resident, and each barrier wait is
// bounded in wall-clock time by the context's wait budget (SegArgs::wait_ns,
// nlc_set_wait_budget; 200 ms by default): a wait that runs out records
// DEV_ERR_GRID_TIMEOUT and the block returns.
//
// Parameter adjoints are accumulated per thread in FP64 over all cells and
// steps the thread handles (a fixed cell-to-thread map, so the order is
// fixed), then reduced per block in a fixed order into acc[block][3].
#pragma once
#include "adjoint.cuh"
#include "common.cuh"
#include "grid_sync.cuh"
#include "step_unfused.cuh"
#include "tma.cuh"

namespace nlc {

template <class T>
struct SegArgs {
  Dims d;
  Par<T> p;
  Layout L;   // padded layout of Q, Q^P (5 components) and u (d components)
  int len;    // steps in the segment
  int lc0;    // lQ[lc0], lG[lc0] hold the adjoint of the state at the segment end
  // records: slot j at g + j Q n, q + j 5 comp, pi + j d^2 n, u + j d comp,
  // qp + j 5 comp
  T* g;
  T* q;
  T* pi;
  T* u;
  T* qp;
  T* r1;  // 5 n scratch of the record kernel
  // adjoint work arrays (adjoint.cuh)
  T* lQ[2];
  T* lG[2];
  T *lQP, *lUa, *lGv, *lF, *lDq, *lLap;
  double* acc;  // [gridDim.x][3], added to
  GridBarrier* bar;
  unsigned* err;
  uint64_t wait_ns;  // budget of each grid-barrier wait
};

template <class Lat, class T>
struct SegSlots {
  const SegArgs<T>& a;
  __device__ T* g(int j) const { return a.g + (int64_t)j * Lat::Q * a.d.n; }
  __device__ T* pi(int j) const { return a.pi + (int64_t)j * Lat::DIM * Lat::DIM * a.d.n; }
  __device__ Field<T> q(int j) const { return Field<T>{a.q + (int64_t)j * 5 * a.L.comp, a.L}; }
  __device__ Field<T> qp(int j) const {
    return Field<T>{a.qp + (int64_t)j * 5 * a.L.comp, a.L};
  }
  __device__ Field<T> u(int j) const {
    return Field<T>{a.u + (int64_t)j * Lat::DIM * a.L.comp, a.L};
  }
};

// every cell handled by this thread (fixed map), with its coordinates
#define NLC_FOR_CELLS(d)                                                            \
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (d).n; \
       idx += (int64_t)gridDim.x * blockDim.x)                                      \
    if (int x, y, z; decode((d), idx, x, y, z))

constexpr int SEG_THREADS = 128;

template <class Lat, class T>
__global__ void __launch_bounds__(SEG_THREADS) k_seg_record(SegArgs<T> a) {
  const SegSlots<Lat, T> S{a};
  const Dims d = a.d;
  const Par<T> p = a.p;
  unsigned gen = 0;
  for (int j = 0; j < a.len; j++) {
    const Field<T> Q = S.q(j), U = S.u(j), QP = S.qp(j);
    NLC_FOR_CELLS(d) stress_at<Lat, T>(Q, S.pi(j), d, p, false, idx, x, y, z);
    if (!grid_sync(a.bar, gen, a.err, a.wait_ns)) return;
    NLC_FOR_CELLS(d)
    lb_at<Lat, T>(S.g(j), S.g(j + 1), S.pi(j), U, d, p, nullptr, false, idx, x, y, z);
    if (!grid_sync(a.bar, gen, a.err, a.wait_ns)) return;
    NLC_FOR_CELLS(d) predict_at<Lat, T>(Q, U, QP, a.r1, d, p, false, idx, x, y, z);
    if (!grid_sync(a.bar, gen, a.err, a.wait_ns)) return;
    NLC_FOR_CELLS(d) correct_at<Lat, T>(Q, QP, a.r1, U, S.q(j + 1), d, p, false, idx, x, y, z);
    if (!grid_sync(a.bar, gen, a.err, a.wait_ns)) return;
  }
}

template <class Lat, class T>
__global__ void __launch_bounds__(SEG_THREADS) k_seg_reverse(SegArgs<T> a) {
  const SegSlots<Lat, T> S{a};
  const Dims d = a.d;
  const Par<T> p = a.p;
  unsigned gen = 0;
  double acc3[3] = {0.0, 0.0, 0.0};
  auto take = [&](const ParBar<T>& pb) {
    acc3[0] += (double)pb.gamma;
    acc3[1] += (double)pb.K;
    acc3[2] += (double)pb.Gamma;
  };
  int lc = a.lc0;
  bool ok = true;
  for (int j = a.len - 1; j >= 0 && ok; j--) {
    const Field<T> Q = S.q(j), U = S.u(j), QP = S.qp(j);
    T* lQn = a.lQ[lc];
    T* lQo = a.lQ[lc ^ 1];
    NLC_FOR_CELLS(d) {
      ParBar<T> pb{T(0), T(0), T(0)};
      adj_be2_at<Lat, T>(QP, U, lQn, a.lQP, a.lUa, a.lGv, d, p, pb, idx, x, y, z);
      take(pb);
    }
    if (!(ok = grid_sync(a.bar, gen, a.err, a.wait_ns))) break;
    NLC_FOR_CELLS(d) {
      ParBar<T> pb{T(0), T(0), T(0)};
      adj_be1_at<Lat, T>(Q, U, lQn, a.lQP, lQo, a.lUa, a.lGv, d, p, pb, idx, x, y, z);
      take(pb);
    }
    if (!(ok = grid_sync(a.bar, gen, a.err, a.wait_ns))) break;
    NLC_FOR_CELLS(d)
    adj_lb_at<Lat, T>(S.g(j), S.pi(j), a.lG[lc], a.lUa, a.lGv, a.lG[lc ^ 1], a.lF, d, p,
                      T(0), idx, x, y, z);
    if (!(ok = grid_sync(a.bar, gen, a.err, a.wait_ns))) break;
    NLC_FOR_CELLS(d) {
      ParBar<T> pb{T(0), T(0), T(0)};
      adj_stress_at<Lat, T>(Q, a.lF, lQo, a.lDq, a.lLap, d, p, pb, idx, x, y, z);
      take(pb);
    }
    if (!(ok = grid_sync(a.bar, gen, a.err, a.wait_ns))) break;
    NLC_FOR_CELLS(d) adj_stencil_at<Lat, T>(a.lDq, a.lLap, lQo, d, idx, x, y, z);
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

#undef NLC_FOR_CELLS

}  // namespace nlc
