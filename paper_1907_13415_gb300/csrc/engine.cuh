// engine.cuh -- the templated engine: device buffers of one or more lattices
// (a batch: same lattice type and precision, any extents and parameters) and
// the launch sequences of the step, set-up, read-back and observables.
#pragma once
#include <cmath>
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "adjoint.cuh"
#include "adjoint_segment.cuh"
#include "adjoint_tiled.cuh"
#include "aux_kernels.cuh"
#include "engine.h"
#include "nvtx_range.h"
#include "obs_finish.h"
#include "step_fused.cuh"
#include "step_unfused.cuh"

namespace nlc {

// parameters of one lattice in the arithmetic type T; the derived factors
// are formed in float64 and rounded once
template <class T>
inline Par<T> make_par(const nlc_params& q) {
  Par<double> d;
  d.A0 = q.A0;
  d.K = q.K;
  d.gamma = q.gamma;
  d.Gamma = q.Gamma;
  d.xi = q.xi;
  d.tau = q.tau;
  d.rho0 = q.rho0;
  derive(d);
  Par<T> p;
  p.A0 = (T)d.A0;
  p.K = (T)d.K;
  p.gamma = (T)d.gamma;
  p.Gamma = (T)d.Gamma;
  p.xi = (T)d.xi;
  p.tau = (T)d.tau;
  p.rho0 = (T)d.rho0;
  p.inv_tau = (T)d.inv_tau;
  p.guo = (T)d.guo;
  p.Ag = (T)d.Ag;
  p.A1 = (T)d.A1;
  p.Ag3 = (T)d.Ag3;
  p.xm1 = (T)d.xm1;
  p.xp1 = (T)d.xp1;
  p.x23 = (T)d.x23;
  p.x2 = (T)d.x2;
  p.hp = (T)d.hp;
  p.hm = (T)d.hm;
  p.x29 = (T)d.x29;
  return p;
}

#define NLC_CK(call)                                                       \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      err = std::string(#call) + ": " + cudaGetErrorString(e_);            \
      return e_ == cudaErrorMemoryAllocation ? NLC_ENOMEM : NLC_ECUDA;     \
    }                                                                      \
  } while (0)

#define NLC_CK_LAUNCH(what)                                                \
  do {                                                                     \
    cudaError_t e_ = cudaGetLastError();                                   \
    if (e_ != cudaSuccess) {                                               \
      err = std::string(what) + ": " + cudaGetErrorString(e_);             \
      return NLC_ECUDA;                                                    \
    }                                                                      \
  } while (0)

// host-side record of one lattice (T: arithmetic, Q and u; G: populations)
template <class T, class G = T>
struct InstHost {
  Dims d;
  Layout L;
  Par<T> p;
  G* g[2] = {nullptr, nullptr};
  Field<T> q[2];
  Field<T> u;
  int tz = 1;
  T* mrt = nullptr;  // MRT coefficients s_k / |v_k|^2 on the device, or nullptr (BGK)
  // lazily allocated: unfused schedule, read-back staging, checkpoints
  T* pi = nullptr;
  Field<T> qp;
  T* r1 = nullptr;
  T* raw = nullptr;
  double* stage = nullptr;
  double* fstage = nullptr;
  double* partial = nullptr;
  double* prof_partial = nullptr;
  // observables by the fused lb kernel (k_fused_lb with OBS): this
  // lattice's own tile list and one partial row per tile (+ the total)
  TileRef* obs_tiles = nullptr;
  int obs_ntiles = 0;
  size_t obs_cap = 0;        // tiles the obs_tiles / obs_part allocations hold
  int obs_tz = 0;            // chunk list the obs_tiles were built for
  bool obs_taper = false;
  double* obs_part = nullptr;
  double* prof = nullptr;
  int obs_blocks = 1;
  // adjoint work arrays (dense [comp][n])
  T* lQ[2] = {nullptr, nullptr};
  T* lG[2] = {nullptr, nullptr};
  T *lQP = nullptr, *lUa = nullptr, *lGv = nullptr, *lF = nullptr, *lDq = nullptr,
    *lLap = nullptr;
  double* acc = nullptr;  // [3 kernels][blocks][3]
  T* ck = nullptr;        // checkpoints, (Q + 5) n each
  int64_t ck_count = 0;
  // segment records of the persistent adjoint kernels (adjoint_segment.cuh),
  // two sets: the record of segment k-1 is written while segment k reverses
  T *rec_g[2] = {}, *rec_q[2] = {}, *rec_pi[2] = {}, *rec_u[2] = {}, *rec_qp[2] = {},
    *rec_r1[2] = {};
  int64_t rec_len = 0;
  GridBarrier* bar = nullptr;  // [0], [1]: record kernels; [2]: reverse kernel
  int seg_grid = 0;            // blocks of the cooperative launches (0: not available)
  // single-plane lattices: the reverse sweep as owned tiles with recomputed
  // halos (adjoint_tiled.cuh), tiles_x x tiles_y blocks; 0: not used
  int rev_tiles_x = 0, rev_grid = 0;
  int acc_slots = 0;  // parameter-adjoint slots of the segment kernels
};

// T: arithmetic and the Q, u fields; G: storage of the populations (float
// with T = double is the FP32-population, FP64-Q mode)
template <class Lat, class T, class G = T>
class Engine final : public EngineBase {
 public:
  static constexpr int Q = Lat::Q;
  static constexpr int DIM = Lat::DIM;

  explicit Engine(const EngineArgs& a) : args_(a) {}

  ~Engine() override {
    for (int c = 0; c < 2; c++)
      if (graph_[c]) cudaGraphExecDestroy(graph_[c]);
    if (cap_stream_) cudaStreamDestroy(cap_stream_);
    for (const SweepGraph& e : sweep_graphs_) cudaGraphExecDestroy(e.exec);
    if (side_stream_) cudaStreamDestroy(side_stream_);
    for (cudaEvent_t e : seg_ev_)
      if (e) cudaEventDestroy(e);
    for (void* ptr : allocs_) cudaFree(ptr);
  }

  nlc_status init() {
    const int n = args_.n;
    inst_.resize(n);
    mrt_on_.assign(n, false);
    std::vector<InstDev<T, G>> dev(n);
    std::vector<CUtensorMap> qmaps(2 * n), umaps(n);
    maps_ok_ = true;
    cudaStream_t st = args_.stream;
    nlc_status s;
    for (int i = 0; i < n; i++) {
      InstHost<T, G>& I = inst_[i];
      const nlc_grid& g = args_.grids[i];
      const nlc_params& q = args_.params[i];
      I.d = Dims{g.nx, g.ny, g.nz, (int64_t)g.nx * g.ny * g.nz};
      I.L = make_layout(I.d, DIM == 3);
      I.p = make_par<T>(q);
      T *q0, *q1, *u;
      if ((s = alloc(&I.g[0], (size_t)Q * I.d.n)) || (s = alloc(&I.g[1], (size_t)Q * I.d.n)) ||
          (s = alloc(&q0, (size_t)5 * I.L.comp)) || (s = alloc(&q1, (size_t)5 * I.L.comp)) ||
          (s = alloc(&u, (size_t)DIM * I.L.comp)))
        return s;
      I.q[0] = Field<T>{q0, I.L};
      I.q[1] = Field<T>{q1, I.L};
      I.u = Field<T>{u, I.L};
      NLC_CK(cudaMemsetAsync(I.g[0], 0, sizeof(G) * Q * I.d.n, st));
      NLC_CK(cudaMemsetAsync(I.g[1], 0, sizeof(G) * Q * I.d.n, st));
      NLC_CK(cudaMemsetAsync(q0, 0, sizeof(T) * 5 * I.L.comp, st));
      NLC_CK(cudaMemsetAsync(q1, 0, sizeof(T) * 5 * I.L.comp, st));
      NLC_CK(cudaMemsetAsync(u, 0, sizeof(T) * DIM * I.L.comp, st));
      maps_ok_ = maps_ok_ &&
                 encode_field_map<T>(&qmaps[2 * i], q0, I.L.nxp, I.L.nyp, I.L.nzp, 5, BXW, BYH) &&
                 encode_field_map<T>(&qmaps[2 * i + 1], q1, I.L.nxp, I.L.nyp, I.L.nzp, 5, BXW, BYH) &&
                 encode_field_map<T>(&umaps[i], u, I.L.nxp, I.L.nyp, I.L.nzp, DIM, BXW, BYH);
      dev[i].d = I.d;
      dev[i].p = I.p;
      dev[i].g[0] = I.g[0];
      dev[i].g[1] = I.g[1];
      dev[i].q[0] = I.q[0];
      dev[i].q[1] = I.q[1];
      dev[i].u = I.u;
      dev[i].mrt = nullptr;
    }
    ix32_ = true;
    for (const InstHost<T, G>& I : inst_)
      ix32_ = ix32_ && (uint64_t)Q * (uint64_t)I.d.n < (1ull << 32);
    if (const char* w = std::getenv("NLC_POP_INDEX64"))
      if (w[0] == '1') ix32_ = false;
    if ((s = alloc(&bad_, 1)) || (s = alloc(&derr_, 1)) || (s = alloc(&insts_dev_, (size_t)n)) ||
        (s = alloc(&qmaps_dev_, (size_t)2 * n)) || (s = alloc(&umaps_dev_, (size_t)n)))
      return s;
    NLC_CK(cudaMemsetAsync(derr_, 0, sizeof(unsigned), st));
    NLC_CK(cudaMemcpyAsync(insts_dev_, dev.data(), sizeof(InstDev<T, G>) * n, cudaMemcpyHostToDevice, st));
    NLC_CK(cudaMemcpyAsync(qmaps_dev_, qmaps.data(), sizeof(CUtensorMap) * 2 * n, cudaMemcpyHostToDevice, st));
    NLC_CK(cudaMemcpyAsync(umaps_dev_, umaps.data(), sizeof(CUtensorMap) * n, cudaMemcpyHostToDevice, st));
    return set_chunk(0, false);
  }

  // ---------------------------------------------------------------- chunks
  // Rebuilds the joint tile list with chunk depth tz (0: the default per
  // lattice), tapered or not (chunk_bounds), and drops captured step graphs
  // (they hold the old list).  Synchronises the stream.
  nlc_status set_chunk(int tz, bool taper) override {
    cudaStream_t st = args_.stream;
    std::vector<TileRef> tiles;
    taper_ = taper;
    for (size_t i = 0; i < inst_.size(); i++) {
      InstHost<T, G>& I = inst_[i];
      I.tz = tz > 0 ? std::min(tz, column_length<Lat>(I.d))
                    : fused_tz<Lat>(I.d, (int64_t)tiles.size());
      append_tiles<Lat>((int)i, I.d, I.tz, taper_, &tiles);
    }
    NLC_CK(cudaStreamSynchronize(st));  // no step may still read the old list
    if (tiles.size() > tiles_cap_) {
      if (tiles_dev_) {
        cudaFree(tiles_dev_);
        allocs_.erase(std::remove(allocs_.begin(), allocs_.end(), (void*)tiles_dev_),
                      allocs_.end());
        tiles_dev_ = nullptr;
      }
      nlc_status s = alloc(&tiles_dev_, tiles.size());
      if (s) return s;
      tiles_cap_ = tiles.size();
    }
    ntiles_ = (int)tiles.size();
    NLC_CK(cudaMemcpyAsync(tiles_dev_, tiles.data(), sizeof(TileRef) * tiles.size(),
                           cudaMemcpyHostToDevice, st));
    NLC_CK(cudaStreamSynchronize(st));
    drop_graphs();
    return NLC_OK;
  }

  int chunk(int i) const override { return inst_[i].tz; }
  bool tapered() const override { return taper_; }

  // Candidate depths are timed on the current state, which is saved first
  // and restored afterwards (the populations and Q of buffer parity cur_;
  // the other buffers are rewritten by every step before they are read).
  nlc_status autotune(int trial_steps, nlc_tune* out) override {
    cudaStream_t st = args_.stream;
    *out = nlc_tune{};
    out->trial_steps = trial_steps;
    if (!maps_ok_) {
      err = "TMA tensor maps unavailable: the fused schedule cannot run";
      return NLC_EUNSUPPORTED;
    }
    int maxz = 1;
    for (const auto& I : inst_) maxz = std::max(maxz, column_length<Lat>(I.d));
    // (depth, taper); depth 0: the default choice.  Depths count z planes on
    // D3Q19 and stacked tiles on a single plane.
    std::vector<std::pair<int, bool>> cand = {{0, false}};
    const std::vector<int> uni = DIM == 3 ? std::vector<int>{4, 6, 8, 12, 16, 24, 32, 48, 64}
                                          : std::vector<int>{1, 2, 4, 8, 16, 32};
    const std::vector<int> tap = DIM == 3 ? std::vector<int>{16, 24, 32, 48, 64, 96, 128}
                                          : std::vector<int>{4, 8, 16, 32};
    for (int c : uni)
      if (c <= maxz) cand.push_back({c, false});
    for (int c : tap)
      if (c <= maxz) cand.push_back({c, true});
    // saved state
    const int cur0 = cur_;
    std::vector<G*> gsave(inst_.size(), nullptr);
    std::vector<T*> qsave(inst_.size(), nullptr);
    auto release = [&]() {
      for (G* p : gsave) cudaFree(p);
      for (T* p : qsave) cudaFree(p);
    };
    for (size_t i = 0; i < inst_.size(); i++) {
      InstHost<T, G>& I = inst_[i];
      const size_t gb = sizeof(G) * Q * I.d.n, qb = sizeof(T) * 5 * I.L.comp;
      if (cudaMalloc(&gsave[i], gb) != cudaSuccess || cudaMalloc(&qsave[i], qb) != cudaSuccess) {
        cudaGetLastError();
        release();
        err = "nlc_autotune: no device memory for the saved state";
        return NLC_ENOMEM;
      }
      cudaMemcpyAsync(gsave[i], I.g[cur0], gb, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(qsave[i], I.q[cur0].base, qb, cudaMemcpyDeviceToDevice, st);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    nlc_status s = NLC_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      err = "nlc_autotune: cudaEventCreate failed";
      s = NLC_ECUDA;
    }
    const bool timing = timer.on;
    timer.on = false;
    double best = 0.0;
    int best_k = -1;
    // per-lattice chunk boundaries already timed
    std::vector<std::vector<std::vector<int>>> timed;
    for (size_t k = 0; k < cand.size() && s == NLC_OK; k++) {
      if ((s = set_chunk(cand[k].first, cand[k].second))) break;
      std::vector<std::vector<int>> bounds;
      for (const auto& I : inst_)
        bounds.push_back(chunk_bounds(column_length<Lat>(I.d), I.tz, taper_));
      if (std::find(timed.begin(), timed.end(), bounds) != timed.end()) continue;
      timed.push_back(bounds);
      if ((s = step_fused(st))) break;  // warm-up
      float ms = 0.f;
      if (cudaEventRecord(e0, st) != cudaSuccess) s = NLC_ECUDA;
      for (int j = 0; j < trial_steps && s == NLC_OK; j++) s = step_fused(st);
      if (s) break;
      if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        err = "nlc_autotune: event timing failed";
        s = NLC_ECUDA;
        break;
      }
      const double per = ms / trial_steps;
      out->candidates++;
      if (k == 0) out->default_ms = per;
      if (best_k < 0 || per < best) {
        best = per;
        best_k = (int)k;
      }
    }
    timer.on = timing;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    // restore the state whatever happened above
    cur_ = cur0;
    for (size_t i = 0; i < inst_.size(); i++) {
      InstHost<T, G>& I = inst_[i];
      cudaMemcpyAsync(I.g[cur0], gsave[i], sizeof(G) * Q * I.d.n, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(I.q[cur0].base, qsave[i], sizeof(T) * 5 * I.L.comp,
                      cudaMemcpyDeviceToDevice, st);
    }
    const cudaError_t ce = cudaStreamSynchronize(st);
    release();
    if (s) return s;
    if (ce != cudaSuccess) {
      err = std::string("nlc_autotune: ") + cudaGetErrorString(ce);
      return NLC_ECUDA;
    }
    if ((s = device_error())) return s;
    if ((s = set_chunk(cand[best_k].first, cand[best_k].second))) return s;
    out->best_ms = best;
    out->chunk = 1;
    for (const auto& I : inst_) out->chunk = std::max(out->chunk, I.tz);
    out->taper = taper_ ? 1 : 0;
    return NLC_OK;
  }

  int count() const override { return (int)inst_.size(); }

  nlc_status check_finite(int* bad) override {
    cudaStream_t st = args_.stream;
    *bad = -1;
    for (size_t i = 0; i < inst_.size(); i++) {
      InstHost<T, G>& I = inst_[i];
      NLC_CK(cudaMemsetAsync(bad_, 0, sizeof(unsigned long long), st));
      k_count_nonfinite<Lat, T><<<grid1(I.d.n), 256, 0, st>>>(I.g[cur_], I.q[cur_], I.d, bad_);
      NLC_CK_LAUNCH("k_count_nonfinite");
      unsigned long long nb = 0;
      NLC_CK(cudaMemcpyAsync(&nb, bad_, sizeof(nb), cudaMemcpyDeviceToHost, st));
      NLC_CK(cudaStreamSynchronize(st));
      if (nb) {
        *bad = (int)i;
        err = std::to_string(nb) + " non-finite values in lattice " + std::to_string(i);
        return NLC_EUNSTABLE;
      }
    }
    return device_error();
  }

  // MRT collision for lattice i with q rates in the moment order of
  // lattice.cuh, or BGK again (rates == nullptr).  Captured step graphs hold
  // the kernel variant, so they are dropped.
  nlc_status set_mrt(int i, const double* rates) override {
    InstHost<T, G>& I = inst_[i];
    cudaStream_t st = args_.stream;
    nlc_status s;
    if (rates) {
      if (!I.mrt && (s = alloc(&I.mrt, (size_t)Q))) return s;
      constexpr MomentBasis<Lat> B = make_moment_basis<Lat>();
      T a[Q];
      for (int k = 0; k < Q; k++) a[k] = (T)(rates[k] / B.n2[k]);
      NLC_CK(cudaMemcpyAsync(I.mrt, a, sizeof(a), cudaMemcpyHostToDevice, st));
    }
    const T* ptr = rates ? I.mrt : nullptr;
    NLC_CK(cudaMemcpyAsync(&insts_dev_[i].mrt, &ptr, sizeof(ptr), cudaMemcpyHostToDevice, st));
    NLC_CK(cudaStreamSynchronize(st));
    mrt_on_[i] = rates != nullptr;
    any_mrt_ = false;
    for (bool b : mrt_on_) any_mrt_ = any_mrt_ || b;
    drop_graphs();
    return NLC_OK;
  }

  void invalidate_graphs() override { drop_graphs(); }

  void drop_graphs() {
    for (int c = 0; c < 2; c++)
      if (graph_[c]) {
        cudaGraphExecDestroy(graph_[c]);
        graph_[c] = nullptr;
        graph_len_[c] = 0;
      }
    for (const SweepGraph& e : sweep_graphs_) cudaGraphExecDestroy(e.exec);
    sweep_graphs_.clear();
  }

  // stencils of every lattice: standard (false) or isotropic (true)
  nlc_status set_stencil(bool iso) override {
    if (iso != iso_) drop_graphs();
    iso_ = iso;
    return NLC_OK;
  }

  nlc_status set_params(int i, const nlc_params& q) override {
    InstHost<T, G>& I = inst_[i];
    I.p = make_par<T>(q);
    args_.params[i] = q;
    // the device descriptor holds the parameters: update it in place
    NLC_CK(cudaMemcpyAsync(&insts_dev_[i].p, &I.p, sizeof(Par<T>), cudaMemcpyHostToDevice,
                           args_.stream));
    NLC_CK(cudaStreamSynchronize(args_.stream));
    return NLC_OK;
  }

  // ---------------------------------------------------------------- step
  nlc_status step(int64_t n, int schedule) override {
    if (n <= 0) return NLC_OK;
    nlc_status s;
    if (schedule == NLC_SCHED_UNFUSED) {
      for (auto& I : inst_)
        if ((s = ensure_unfused(I))) return s;
      for (int64_t k = 0; k < n; k++)
        if ((s = step_unfused())) return s;
      return NLC_OK;
    }
    if (!maps_ok_) {
      err = "TMA tensor maps unavailable (driver entry point missing); use the "
            "unfused schedule";
      return NLC_EUNSUPPORTED;
    }
    // the persistent kernel's occupancy and counters are set up here, not
    // inside a stream capture (no allocation may happen there)
    if (persistent_steps > 0 && !any_mrt_) {
      int grid;
      if ((s = persist_grid(&grid))) return s;
    }
    // whole chunks of steps replay a captured CUDA graph (not while timing)
    if (graph_steps > 0 && !timer.on) {
      while (n >= graph_steps) {
        if ((s = ensure_graph(cur_))) return s;
        NLC_CK(cudaGraphLaunch(graph_[cur_], args_.stream));
        if (graph_steps % 2) cur_ ^= 1;
        n -= graph_steps;
      }
    }
    return fused_launches(n, args_.stream);
  }

  // n fused steps launched on st: two kernels per step, or cooperative
  // launches of the persistent kernel of up to persistent_steps steps each
  nlc_status fused_launches(int64_t n, cudaStream_t st) {
    nlc_status s;
    int grid = 0;
    if (persistent_steps > 0 && !any_mrt_ && (s = persist_grid(&grid))) return s;
    if (grid > 0) {
      while (n > 0) {
        const int m = (int)std::min<int64_t>(n, persistent_steps);
        if ((s = step_persistent(st, m, grid))) return s;
        n -= m;
      }
      return NLC_OK;
    }
    for (int64_t k = 0; k < n; k++)
      if ((s = step_fused(st))) return s;
    return NLC_OK;
  }

  // blocks of the persistent kernel (0: not available on this device)
  nlc_status persist_grid(int* grid) {
    const int v = (iso_ ? 2 : 0) + (ix32_ ? 1 : 0);
    if (pgrid_max_[v] < 0)
      pgrid_max_[v] = persistent_grid_max<Lat, T, G>(iso_, ix32_);
    if (pgrid_max_[v] > 0 && !pbar_) {
      nlc_status s;
      if ((s = alloc(&pbar_, 1))) return s;
    }
    *grid = std::min(pgrid_max_[v], ntiles_);
    return NLC_OK;
  }

  // m steps of every lattice in one cooperative launch
  nlc_status step_persistent(cudaStream_t st, int m, int grid) {
    NLC_CK(cudaMemsetAsync(pbar_, 0, sizeof(GridBarrier), st));
    const int e0 = mark();
    PersistArgs pa{pbar_, wait_ns};
    cudaError_t e = launch_fused_persistent<Lat, T, G>(insts_dev_, qmaps_dev_, umaps_dev_,
                                                       tiles_dev_, ntiles_, cur_, m, derr_, pa,
                                                       grid, st, iso_, ix32_);
    if (e != cudaSuccess) {
      err = std::string("persistent step kernel: ") + cudaGetErrorString(e);
      cudaGetLastError();
      return NLC_ECUDA;
    }
    const int e1 = mark();
    if (timer.on) timer.span(KID_PERSIST, e0, e1);
    if (m & 1) cur_ ^= 1;
    return NLC_OK;
  }

  // ---------------------------------------------------------------- I/O
  // Device-side address of a page-locked (pinned) host array, which the
  // kernels can read in place over the host link, or nullptr for any other
  // memory (pageable host memory goes through a staging copy instead).
  // true for memory the device can read directly (device or managed)
  template <class V>
  static bool device_array(const V* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
  }

  template <class V>
  static const V* mapped_host(const V* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? static_cast<const V*>(a.devicePointer) : nullptr;
  }

  // Q from float32 (pinned: read in place; else through the staging
  // buffer), rho = rho0, u = 0
  nlc_status set_fields_f32(int i, const float* Q5) override {
    InstHost<T, G>& I = inst_[i];
    nlc_status s;
    if ((s = ensure_staging(I))) return s;
    const int64_t n = I.d.n;
    cudaStream_t st = args_.stream;
    // device arrays are read in place too (a caller that uploads the next
    // state on its own copy stream while the current one is stepped)
    const float* qs = device_array(Q5) ? Q5 : mapped_host(Q5);
    if (!qs) {
      float* stage = reinterpret_cast<float*>(I.stage);  // 9 n doubles >= 5 n floats
      NLC_CK(cudaMemcpyAsync(stage, Q5, sizeof(float) * 5 * n, cudaMemcpyHostToDevice, st));
      qs = stage;
    }
    NLC_CK(cudaMemsetAsync(bad_, 0, sizeof(unsigned long long), st));
    k_set_fields<Lat, T, G, float><<<grid1(n), 256, 0, st>>>(
        qs, nullptr, nullptr, I.q[cur_], I.g[cur_], I.d, args_.params[i].rho0, bad_);
    NLC_CK_LAUNCH("k_set_fields");
    unsigned long long nbad = 0;
    NLC_CK(cudaMemcpyAsync(&nbad, bad_, sizeof(nbad), cudaMemcpyDeviceToHost, st));
    NLC_CK(cudaStreamSynchronize(st));
    if (nbad) {
      err = "nlc_set_fields_f32: " + std::to_string(nbad) + " non-finite input values";
      return NLC_EUNSTABLE;
    }
    return NLC_OK;
  }

  nlc_status set_fields(int i, const double* Q5, const double* rho,
                        const double* u) override {
    InstHost<T, G>& I = inst_[i];
    nlc_status s;
    if ((s = ensure_staging(I))) return s;
    const int64_t n = I.d.n;
    cudaStream_t st = args_.stream;
    // pinned inputs are read in place by the kernel (the transfer then
    // overlaps the conversion); others are copied to the staging buffer
    auto source = [&](const double* h, double* stage, int64_t count,
                      const double** out) -> nlc_status {
      *out = nullptr;
      if (!h) return NLC_OK;
      if ((*out = mapped_host(h))) return NLC_OK;
      NLC_CK(cudaMemcpyAsync(stage, h, sizeof(double) * count, cudaMemcpyHostToDevice, st));
      *out = stage;
      return NLC_OK;
    };
    const double *qs, *rs, *us;
    if ((s = source(Q5, I.stage, 5 * n, &qs)) || (s = source(rho, I.stage + 5 * n, n, &rs)) ||
        (s = source(u, I.stage + 6 * n, 3 * n, &us)))
      return s;
    NLC_CK(cudaMemsetAsync(bad_, 0, sizeof(unsigned long long), st));
    k_set_fields<Lat, T><<<grid1(n), 256, 0, st>>>(qs, rs, us, I.q[cur_], I.g[cur_], I.d,
                                                   args_.params[i].rho0, bad_);
    NLC_CK_LAUNCH("k_set_fields");
    unsigned long long nbad = 0;
    NLC_CK(cudaMemcpyAsync(&nbad, bad_, sizeof(nbad), cudaMemcpyDeviceToHost, st));
    NLC_CK(cudaStreamSynchronize(st));
    if (nbad) {
      err = "nlc_set_fields: " + std::to_string(nbad) +
            " non-finite (or non-positive density) input values";
      return NLC_EUNSTABLE;
    }
    return NLC_OK;
  }

  nlc_status get_fields(int i, double* Q5, double* rho, double* u) override {
    InstHost<T, G>& I = inst_[i];
    nlc_status s;
    if ((s = ensure_staging(I))) return s;
    const int64_t n = I.d.n;
    cudaStream_t st = args_.stream;
    if (Q5) {
      k_field_out<T><<<grid1(n), 256, 0, st>>>(I.q[cur_], 5, I.d, I.stage);
      NLC_CK_LAUNCH("k_field_out");
      NLC_CK(cudaMemcpyAsync(Q5, I.stage, sizeof(double) * 5 * n, cudaMemcpyDeviceToHost, st));
    }
    if (rho || u) {
      if ((s = moments_to_stage(I))) return s;
      if (rho)
        NLC_CK(cudaMemcpyAsync(rho, I.stage + 5 * n, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
      if (u)
        NLC_CK(cudaMemcpyAsync(u, I.stage + 6 * n, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    }
    NLC_CK(cudaStreamSynchronize(st));
    return device_error();
  }

  nlc_status get_populations(int i, double* f) override {
    InstHost<T, G>& I = inst_[i];
    if (!I.fstage) {
      nlc_status s = alloc(&I.fstage, (size_t)Q * I.d.n);
      if (s) return s;
    }
    const int64_t n = I.d.n;
    cudaStream_t st = args_.stream;
    k_populations_out<Lat, T><<<grid1(n), 256, 0, st>>>(I.g[cur_], I.d, args_.params[i].rho0,
                                                         I.fstage);
    NLC_CK_LAUNCH("k_populations_out");
    NLC_CK(cudaMemcpyAsync(f, I.fstage, sizeof(double) * Q * n, cudaMemcpyDeviceToHost, st));
    NLC_CK(cudaStreamSynchronize(st));
    return device_error();
  }

  size_t state_bytes() const override {
    size_t b = 0;
    for (const auto& I : inst_) b += (sizeof(G) * Q + sizeof(T) * 5) * (size_t)I.d.n;
    return b;
  }

  nlc_status save_state(void* dst) override {
    cudaStream_t st = args_.stream;
    char* out = (char*)dst;
    for (auto& I : inst_) {
      nlc_status s;
      if (!I.raw && (s = alloc(&I.raw, (size_t)5 * I.d.n))) return s;
      const int64_t n = I.d.n;
      k_field_raw_out<T><<<grid1(n), 256, 0, st>>>(I.q[cur_], 5, I.d, I.raw);
      NLC_CK_LAUNCH("k_field_raw_out");
      NLC_CK(cudaMemcpyAsync(out, I.g[cur_], sizeof(G) * Q * n, cudaMemcpyDeviceToHost, st));
      out += sizeof(G) * Q * n;
      NLC_CK(cudaMemcpyAsync(out, I.raw, sizeof(T) * 5 * n, cudaMemcpyDeviceToHost, st));
      out += sizeof(T) * 5 * n;
    }
    NLC_CK(cudaStreamSynchronize(st));
    return device_error();
  }

  nlc_status load_state(const void* src) override {
    cudaStream_t st = args_.stream;
    const char* in = (const char*)src;
    for (auto& I : inst_) {
      nlc_status s;
      if (!I.raw && (s = alloc(&I.raw, (size_t)5 * I.d.n))) return s;
      const int64_t n = I.d.n;
      NLC_CK(cudaMemcpyAsync(I.g[0], in, sizeof(G) * Q * n, cudaMemcpyHostToDevice, st));
      in += sizeof(G) * Q * n;
      NLC_CK(cudaMemcpyAsync(I.raw, in, sizeof(T) * 5 * n, cudaMemcpyHostToDevice, st));
      in += sizeof(T) * 5 * n;
      k_field_raw_in<T, DIM><<<grid1(n), 256, 0, st>>>(I.raw, I.d, I.q[0]);
      NLC_CK_LAUNCH("k_field_raw_in");
    }
    NLC_CK(cudaStreamSynchronize(st));
    cur_ = 0;
    return NLC_OK;
  }


  // ------------------------------------------------------------- adjoint
  nlc_status adjoint(const nlc_loss* loss, int64_t nsteps, int ckpt_every, nlc_grad* out,
                     double* dQ0) override {
    if constexpr (!std::is_same<T, G>::value) {
      err = "the adjoint needs the populations in the arithmetic precision";
      return NLC_EUNSUPPORTED;
    }
    InstHost<T, G>& I = inst_[0];
    const int64_t n = I.d.n;
    const int64_t nseg = (nsteps + ckpt_every - 1) / ckpt_every;
    const int64_t S = (int64_t)(Q + 5) * n;  // one state
    cudaStream_t st = args_.stream;
    nlc_status s;
    if ((s = ensure_staging(I)) || (s = ensure_segment(I, ckpt_every)) ||
        (s = ensure_adjoint(I, nseg + 1)))
      return s;
    if (I.seg_grid <= 0) {
      err = "the adjoint needs cooperative launches of its segment kernels";
      return NLC_EUNSUPPORTED;
    }
    if (any_mrt_ || iso_) {
      err = "the adjoint covers the BGK collision with the standard stencils only";
      return NLC_EUNSUPPORTED;
    }
    if (!maps_ok_) {
      err = "TMA tensor maps unavailable; the adjoint needs the fused step";
      return NLC_EUNSUPPORTED;
    }
    {
      NvtxRange nvtx_fwd("adjoint: forward sweep");
      // forward sweep, keeping the state at the start of every segment; the
      // record of the last segment, which the backward sweep needs first, runs
      // on the side stream from its checkpoint while the forward sweep
      // finishes that segment
      for (int64_t k = 0; k < nseg; k++) {
        if ((s = state_out(I, I.ck + k * S))) return s;
        const int64_t len = std::min<int64_t>(ckpt_every, nsteps - k * ckpt_every);
        if (k == nseg - 1) {
          NLC_CK(cudaEventRecord(seg_ev_[0], st));
          NLC_CK(cudaStreamWaitEvent(side_stream_, seg_ev_[0], 0));
          const int b = (int)(k & 1);
          if ((s = segment_record(I, b, I.ck + k * S, (int)len, side_stream_))) return s;
          NLC_CK(cudaEventRecord(seg_ev_[1 + b], side_stream_));
        }
        if ((s = fused_steps(len))) return s;
      }
    }
    if ((s = state_out(I, I.ck + nseg * S))) return s;  // final state
    // loss and its seed on the final state
    nlc_obs obs;
    if ((s = observables(0, &obs, nullptr))) return s;
    const double R = obs.radius, A = obs.s_area;
    const double dRdA = (DIM == 2 || I.d.nz == 1) ? (R > 0 ? 1.0 / (2.0 * M_PI * R) : 0.0)
                                                   : (A > 0 ? R / (3.0 * A) : 0.0);
    const double s_ref = 1.0 / 3.0;
    const double cR = loss->w_radius * 2.0 * (R - loss->target_radius) * dRdA / s_ref;
    const double cu = obs.u_l2 > 0 ? loss->w_velocity / obs.u_l2 : 0.0;
    out->radius = R;
    out->u_l2 = obs.u_l2;
    out->loss = loss->w_radius * (R - loss->target_radius) * (R - loss->target_radius) +
                loss->w_velocity * obs.u_l2;
    NLC_CK(cudaMemsetAsync(I.acc, 0, sizeof(double) * 3 * (3 * grid1(n) + I.acc_slots), st));
    int lc = 0;  // lQ[lc], lG[lc] hold the adjoint of the current state
    {
      const unsigned gb = grid1(n);
      k_stress<Lat, T><<<gb, 256, 0, st>>>(I.q[cur_], I.pi, I.d, I.p, false);
      k_adj_seed_q<T><<<gb, 256, 0, st>>>(I.q[cur_], (T)cR, I.lQ[lc], I.d);
      k_adj_lb<Lat, T><<<gb, 256, 0, st>>>(I.g[cur_], I.pi, nullptr, nullptr, nullptr,
                                           I.lG[lc], I.lF, I.d, I.p, (T)cu);
      k_adj_stress<Lat, T><<<gb, 256, 0, st>>>(I.q[cur_], I.lF, I.lQ[lc], I.lDq, I.lLap,
                                               I.d, I.p, I.acc + 2 * 3 * gb);
      k_adj_stencil<Lat, T><<<gb, 256, 0, st>>>(I.lDq, I.lLap, I.lQ[lc], I.d);
      NLC_CK_LAUNCH("adjoint seed");
    }
    // backward sweep, segment by segment (adjoint_segment.cuh)
    {
      NvtxRange nvtx_bwd("adjoint: backward segments");
      if ((s = segments_backward(I, nsteps, ckpt_every, nseg, S, lc))) return s;
    }
    // gradients: every block slot of every kernel, summed in a fixed order
    const unsigned gb = grid1(n);
    std::vector<double> acc((size_t)3 * (3 * gb + I.acc_slots));
    NLC_CK(cudaMemcpyAsync(acc.data(), I.acc, sizeof(double) * acc.size(),
                           cudaMemcpyDeviceToHost, st));
    if (dQ0) {
      k_dense_to_double<T><<<grid1(5 * n), 256, 0, st>>>(I.lQ[lc], I.stage, 5 * n);
      NLC_CK_LAUNCH("k_dense_to_double");
      NLC_CK(cudaMemcpyAsync(dQ0, I.stage, sizeof(double) * 5 * n, cudaMemcpyDeviceToHost, st));
    }
    // leave the context at the final state
    if ((s = state_in(I, I.ck + nseg * S))) return s;
    NLC_CK(cudaStreamSynchronize(st));
    if ((s = device_error())) return s;
    double g3[3] = {0, 0, 0};
    for (size_t i = 0; i < acc.size(); i++) g3[i % 3] += acc[i];
    out->dgamma = g3[0];
    out->dK = g3[1];
    out->dGamma = g3[2];
    return NLC_OK;
  }

  nlc_status observables(int i, nlc_obs* out, double* s_profile) override {
    InstHost<T, G>& I = inst_[i];
    nlc_status s;
    if ((s = ensure_staging(I))) return s;
    const int64_t n = I.d.n;
    const Dims& d = I.d;
    cudaStream_t st = args_.stream;
    const double s_ref = 1.0 / 3.0;
    const double* total;
    if (maps_ok_ && !iso_ && ix32_) {
      // one pass of the fused lb kernel in its observing form over this
      // lattice's tiles (the step's tile machinery, nothing stored)
      // the lattice's tiles in the chunk list the step runs with (the
      // autotuner's choice when it ran)
      if (!I.obs_tiles || I.obs_tz != I.tz || I.obs_taper != taper_) {
        std::vector<TileRef> tl;
        append_tiles<Lat>(i, I.d, I.tz, taper_, &tl);
        if (tl.size() > I.obs_cap) {
          for (void* old : {(void*)I.obs_tiles, (void*)I.obs_part})
            if (old) {
              NLC_CK(cudaStreamSynchronize(st));
              cudaFree(old);
              allocs_.erase(std::remove(allocs_.begin(), allocs_.end(), old), allocs_.end());
            }
          I.obs_tiles = nullptr;
          I.obs_part = nullptr;
          if ((s = alloc(&I.obs_tiles, tl.size())) ||
              (s = alloc(&I.obs_part, (tl.size() + 1) * OBS_SLOTS)))
            return s;
          I.obs_cap = tl.size();
        }
        NLC_CK(cudaMemcpyAsync(I.obs_tiles, tl.data(), sizeof(TileRef) * tl.size(),
                               cudaMemcpyHostToDevice, st));
        I.obs_ntiles = (int)tl.size();
        I.obs_tz = I.tz;
        I.obs_taper = taper_;
      }
      cudaError_t e = launch_fused_obs<Lat, T>(insts_dev_, qmaps_dev_, I.obs_tiles, I.obs_ntiles,
                                               cur_, derr_, I.obs_part, st);
      if (e != cudaSuccess) {
        err = std::string("fused observables kernel: ") + cudaGetErrorString(e);
        return NLC_ECUDA;
      }
      k_obs_final<<<OBS_SLOTS, 256, 0, st>>>(I.obs_part, I.obs_ntiles,
                                             I.obs_part + (int64_t)I.obs_ntiles * OBS_SLOTS);
      NLC_CK_LAUNCH("k_obs_final");
      total = I.obs_part + (int64_t)I.obs_ntiles * OBS_SLOTS;
    } else {
      // stress of the current Q, then rho, u and the observables in one pass
      k_stress<Lat, T><<<grid1(n), 256, 0, st>>>(I.q[cur_], I.pi, I.d, I.p, iso_);
      NLC_CK_LAUNCH("k_stress");
      k_obs_state<Lat, T><<<I.obs_blocks, 256, 0, st>>>(I.q[cur_], I.g[cur_], I.pi, d, I.p,
                                                        s_ref, iso_, I.partial);
      NLC_CK_LAUNCH("k_obs_state");
      k_obs_final<<<OBS_SLOTS, 256, 0, st>>>(I.partial, I.obs_blocks,
                                             I.partial + I.obs_blocks * OBS_SLOTS);
      NLC_CK_LAUNCH("k_obs_final");
      total = I.partial + I.obs_blocks * OBS_SLOTS;
    }
    const int64_t rows = (int64_t)d.ny * d.nz;
    const int rows_per_chunk = profile_rows_per_chunk(d);
    const int nchunks = (int)((rows + rows_per_chunk - 1) / rows_per_chunk);
    dim3 pg((d.nx + 127) / 128, nchunks);
    k_profile_partial<T><<<pg, 128, 0, st>>>(I.q[cur_], d, rows_per_chunk, I.prof_partial);
    NLC_CK_LAUNCH("k_profile_partial");
    k_profile_final<<<d.nx, 256, 0, st>>>(I.prof_partial, nchunks, d, I.prof);
    NLC_CK_LAUNCH("k_profile_final");
    double tot[OBS_SLOTS];
    std::vector<double> prof(d.nx);
    NLC_CK(cudaMemcpyAsync(tot, total, sizeof(tot), cudaMemcpyDeviceToHost, st));
    NLC_CK(cudaMemcpyAsync(prof.data(), I.prof, sizeof(double) * d.nx, cudaMemcpyDeviceToHost, st));
    NLC_CK(cudaStreamSynchronize(st));
    if ((s = device_error())) return s;
    obs_from_totals(tot, prof.data(), d.nx, DIM == 2 || d.nz == 1, s_ref, out);
    if (s_profile)
      for (int x = 0; x < d.nx; x++) s_profile[x] = prof[x];
    return NLC_OK;
  }

 private:
  static unsigned grid1(int64_t count) { return (unsigned)((count + 255) / 256); }

  // rows (y, z) per block of the S-profile pass: about 2048 blocks over the
  // lattice, so that small lattices still spread over the SMs
  static int profile_rows_per_chunk(const Dims& d) {
    const int64_t xb = (d.nx + 127) / 128, rows = (int64_t)d.ny * d.nz;
    const int64_t chunks = std::max<int64_t>(1, 2048 / xb);
    return (int)std::max<int64_t>(1, (rows + chunks - 1) / chunks);
  }

  template <class U>
  nlc_status alloc(U** p, size_t count) {
    void* ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, sizeof(U) * (count ? count : 1));
    if (e != cudaSuccess) {
      err = std::string("cudaMalloc(") + std::to_string(sizeof(U) * count) +
            " bytes): " + cudaGetErrorString(e);
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? NLC_ENOMEM : NLC_ECUDA;
    }
    allocs_.push_back(ptr);
    *p = (U*)ptr;
    return NLC_OK;
  }

  // device-side error word (bounded waits that ran out); read after a
  // sync, and cleared once reported, so that the context can run again
  nlc_status device_error() {
    unsigned e = 0;
    NLC_CK(cudaMemcpy(&e, derr_, sizeof(e), cudaMemcpyDeviceToHost));
    if (e != DEV_ERR_NONE) {
      err = e == DEV_ERR_GRID_TIMEOUT
                ? "a bounded grid-barrier wait ran out inside a persistent kernel"
                : "a bounded wait on a tile copy ran out inside a step kernel (code " +
                      std::to_string(e) + ")";
      NLC_CK(cudaMemset(derr_, 0, sizeof(unsigned)));
      return NLC_ETIMEOUT;
    }
    return NLC_OK;
  }

  nlc_status ensure_unfused(InstHost<T, G>& I) {
    if (I.pi) return NLC_OK;
    nlc_status s;
    const int64_t n = I.d.n;
    T* qp;
    if ((s = alloc(&I.pi, (size_t)DIM * DIM * n)) || (s = alloc(&qp, (size_t)5 * I.L.comp)) ||
        (s = alloc(&I.r1, (size_t)5 * n)))
      return s;
    I.qp = Field<T>{qp, I.L};
    return NLC_OK;
  }

  nlc_status ensure_staging(InstHost<T, G>& I) {
    if (I.stage) return NLC_OK;
    nlc_status s;
    const int64_t n = I.d.n;
    if ((s = alloc(&I.stage, (size_t)9 * n))) return s;
    if ((s = ensure_unfused(I))) return s;
    int dev = 0, sms = 0;
    NLC_CK(cudaGetDevice(&dev));
    NLC_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t want = (n + 255) / 256;
    I.obs_blocks = (int)(want < 16 * sms ? want : 16 * sms);
    if (I.obs_blocks < 1) I.obs_blocks = 1;
    if ((s = alloc(&I.partial, (size_t)(I.obs_blocks + 1) * OBS_SLOTS))) return s;
    const int64_t rows = (int64_t)I.d.ny * I.d.nz;
    const int rpc = profile_rows_per_chunk(I.d);
    const int64_t nchunks = (rows + rpc - 1) / rpc;
    if ((s = alloc(&I.prof_partial, (size_t)(nchunks * I.d.nx)))) return s;
    if ((s = alloc(&I.prof, (size_t)I.d.nx))) return s;
    return NLC_OK;
  }

  nlc_status ensure_adjoint(InstHost<T, G>& I, int64_t ck_count) {
    nlc_status s;
    const int64_t n = I.d.n;
    const int64_t S = (int64_t)(Q + 5) * n;
    if ((s = ensure_unfused(I))) return s;  // Pi for the loss seed
    if (!I.lQP) {
      if ((s = alloc(&I.lQ[0], (size_t)5 * n)) || (s = alloc(&I.lQ[1], (size_t)5 * n)) ||
          (s = alloc(&I.lG[0], (size_t)Q * n)) || (s = alloc(&I.lG[1], (size_t)Q * n)) ||
          (s = alloc(&I.lQP, (size_t)5 * n)) || (s = alloc(&I.lUa, (size_t)DIM * n)) ||
          (s = alloc(&I.lGv, (size_t)DIM * DIM * n)) || (s = alloc(&I.lF, (size_t)DIM * n)) ||
          (s = alloc(&I.lDq, (size_t)DIM * 5 * n)) || (s = alloc(&I.lLap, (size_t)5 * n)) ||
          (s = alloc(&I.acc, (size_t)3 * (3 * grid1(n) + seg_grid_max()))))
        return s;
    }
    if (I.ck_count < ck_count) {
      if ((s = alloc(&I.ck, (size_t)(ck_count * S)))) return s;
      I.ck_count = ck_count;
    }
    return NLC_OK;
  }

  // blocks of a cooperative launch of the segment kernels: every block must
  // be resident, so at most the SM count times the blocks per SM that fit
  int seg_grid_max() {
    int dev = 0, sms = 0, nb1 = 0, nb2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb1, k_seg_record<Lat, T>, SEG_THREADS,
                                                      0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb2, k_seg_reverse<Lat, T>,
                                                      SEG_THREADS, 0) != cudaSuccess)
      return 0;
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
      return 0;
    return sms * std::min(nb1, nb2);
  }

  // Single-plane lattices record and reverse each segment as owned 16 x 8
  // tiles with recomputed halos (one grid barrier per step,
  // adjoint_tiled.cuh) when every tile's block can be resident;
  // NLC_ADJ_TILED=0 keeps the one-cell-per-thread segment kernels.
  nlc_status plan_tiled_reverse(InstHost<T, G>& I) {
    I.rev_tiles_x = I.rev_grid = 0;
    if constexpr (DIM == 2) {
      const char* env = std::getenv("NLC_ADJ_TILED");
      if (env && env[0] == '0') return NLC_OK;
      const int tx = (I.d.nx + ATX - 1) / ATX, ty = (I.d.ny + ATY - 1) / ATY;
      const int64_t want = (int64_t)tx * ty;
      if (I.seg_grid <= 0 || want > seg_grid_max()) return NLC_OK;
      const size_t bytes = sizeof(AdjTile<T>);
      NLC_CK(cudaFuncSetAttribute(k_seg_reverse_tiled<Lat, T>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
      int dev = 0, sms = 0, nb = 0;
      NLC_CK(cudaGetDevice(&dev));
      NLC_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      NLC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_seg_reverse_tiled<Lat, T>, ABA,
                                                           bytes));
      if ((int64_t)nb * sms < want) return NLC_OK;
      NLC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_seg_record_tiled<Lat, T>, ABA,
                                                           sizeof(RecTile<T>)));
      if ((int64_t)nb * sms < want) return NLC_OK;
      I.rev_tiles_x = tx;
      I.rev_grid = (int)want;
      I.acc_slots = std::max(I.seg_grid, I.rev_grid);
    }
    return NLC_OK;
  }

  // record slots (two sets) for segments of up to len steps
  nlc_status ensure_segment(InstHost<T, G>& I, int64_t len) {
    nlc_status s;
    if (!I.bar) {
      if ((s = alloc(&I.bar, 3))) return s;
      const int64_t want = (I.d.n + SEG_THREADS - 1) / SEG_THREADS;
      I.seg_grid = (int)std::min<int64_t>(seg_grid_max(), want);
      I.acc_slots = I.seg_grid;
      if ((s = plan_tiled_reverse(I))) return s;
    }
    if (I.seg_grid <= 0 || I.rec_len >= len) return NLC_OK;
    const int64_t n = I.d.n, comp = I.L.comp;
    for (int b = 0; b < 2; b++)
      if ((s = alloc(&I.rec_g[b], (size_t)((len + 1) * Q * n))) ||
          (s = alloc(&I.rec_q[b], (size_t)((len + 1) * 5 * comp))) ||
          (s = alloc(&I.rec_pi[b], (size_t)(len * DIM * DIM * n))) ||
          (s = alloc(&I.rec_u[b], (size_t)(len * DIM * comp))) ||
          (s = alloc(&I.rec_qp[b], (size_t)(len * 5 * comp))) ||
          (s = alloc(&I.rec_r1[b], (size_t)(5 * n))))
        return s;
    I.rec_len = len;
    if (!side_stream_) {
      NLC_CK(cudaStreamCreateWithFlags(&side_stream_, cudaStreamNonBlocking));
      for (int k = 0; k < 5; k++)
        NLC_CK(cudaEventCreateWithFlags(&seg_ev_[k], cudaEventDisableTiming));
    }
    return NLC_OK;
  }

  SegArgs<T> seg_args(InstHost<T, G>& I, int b, int len, int lc) {
    SegArgs<T> a;
    a.d = I.d;
    a.p = I.p;
    a.L = I.L;
    a.len = len;
    a.lc0 = lc;
    a.g = I.rec_g[b];
    a.q = I.rec_q[b];
    a.pi = I.rec_pi[b];
    a.u = I.rec_u[b];
    a.qp = I.rec_qp[b];
    a.r1 = I.rec_r1[b];
    a.lQ[0] = I.lQ[0];
    a.lQ[1] = I.lQ[1];
    a.lG[0] = I.lG[0];
    a.lG[1] = I.lG[1];
    a.lQP = I.lQP;
    a.lUa = I.lUa;
    a.lGv = I.lGv;
    a.lF = I.lF;
    a.lDq = I.lDq;
    a.lLap = I.lLap;
    a.acc = I.acc + (size_t)3 * 3 * grid1(I.d.n);
    a.err = derr_;
    a.wait_ns = wait_ns;
    return a;
  }

  // record of a segment of len steps from the checkpoint at ck into set b,
  // on stream ss
  nlc_status segment_record(InstHost<T, G>& I, int b, const T* ck, int len, cudaStream_t ss) {
    const int64_t n = I.d.n;
    NLC_CK(cudaMemcpyAsync(I.rec_g[b], ck, sizeof(T) * Q * n, cudaMemcpyDeviceToDevice, ss));
    k_field_raw_in<T, DIM><<<grid1(n), 256, 0, ss>>>(ck + (int64_t)Q * n, I.d,
                                                       Field<T>{I.rec_q[b], I.L});
    NLC_CK_LAUNCH("k_field_raw_in");
    SegArgs<T> a = seg_args(I, b, len, 0);
    a.bar = I.bar + b;
    void* args[] = {&a};
    NLC_CK(cudaMemsetAsync(a.bar, 0, sizeof(GridBarrier), ss));
    if constexpr (DIM == 2) {
      if (I.rev_grid > 0) {
        int tiles_x = I.rev_tiles_x;
        void* targs[] = {&a, &tiles_x};
        NLC_CK(cudaLaunchCooperativeKernel((const void*)k_seg_record_tiled<Lat, T>,
                                           dim3(I.rev_grid), dim3(ABA), targs,
                                           sizeof(RecTile<T>), ss));
        return NLC_OK;
      }
    }
    NLC_CK(cudaLaunchCooperativeKernel((const void*)k_seg_record<Lat, T>, dim3(I.seg_grid),
                                       dim3(SEG_THREADS), args, 0, ss));
    return NLC_OK;
  }

  // reverse of the segment recorded in set b; the adjoint of its end state
  // is in (lQ[lc], lG[lc])
  nlc_status segment_reverse(InstHost<T, G>& I, int b, int len, int lc, cudaStream_t st) {
    SegArgs<T> a = seg_args(I, b, len, lc);
    a.bar = I.bar + 2;
    void* args[] = {&a};
    NLC_CK(cudaMemsetAsync(a.bar, 0, sizeof(GridBarrier), st));
    if constexpr (DIM == 2) {
      if (I.rev_grid > 0) {
        int tiles_x = I.rev_tiles_x;
        void* targs[] = {&a, &tiles_x};
        NLC_CK(cudaLaunchCooperativeKernel((const void*)k_seg_reverse_tiled<Lat, T>,
                                           dim3(I.rev_grid), dim3(ABA), targs,
                                           sizeof(AdjTile<T>), st));
        return NLC_OK;
      }
    }
    NLC_CK(cudaLaunchCooperativeKernel((const void*)k_seg_reverse<Lat, T>, dim3(I.seg_grid),
                                       dim3(SEG_THREADS), args, 0, st));
    return NLC_OK;
  }

  // All segments, last to first: the record of segment k-1 runs on the side
  // stream while segment k reverses on the main stream (the record of the
  // last segment was queued by the forward sweep).  Record set k % 2
  // is rewritten only after the reverse that read it (segment k+2) is done.
  nlc_status segments_backward(InstHost<T, G>& I, int64_t nsteps, int ckpt_every, int64_t nseg,
                               int64_t S, int& lc) {
    cudaStream_t st = args_.stream, ss = side_stream_;
    cudaEvent_t ev_main = seg_ev_[0], ev_rec[2] = {seg_ev_[1], seg_ev_[2]},
                ev_rev[2] = {seg_ev_[3], seg_ev_[4]};
    auto seg_len = [&](int64_t k) {
      return (int)std::min<int64_t>(ckpt_every, nsteps - k * ckpt_every);
    };
    nlc_status s;
    const int e0 = mark();
    // the record of the last segment was queued on the side stream during
    // the forward sweep (event ev_rec[(nseg - 1) & 1])
    for (int64_t k = nseg - 1; k >= 0; k--) {
      const int b = (int)(k & 1);
      NLC_CK(cudaStreamWaitEvent(st, ev_rec[b], 0));
      if (k > 0) {
        const int bp = (int)((k - 1) & 1);
        if (k + 1 < nseg) NLC_CK(cudaStreamWaitEvent(ss, ev_rev[bp], 0));
        if ((s = segment_record(I, bp, I.ck + (k - 1) * S, seg_len(k - 1), ss))) return s;
        NLC_CK(cudaEventRecord(ev_rec[bp], ss));
      }
      if ((s = segment_reverse(I, b, seg_len(k), lc, st))) return s;
      NLC_CK(cudaEventRecord(ev_rev[b], st));
      if (seg_len(k) & 1) lc ^= 1;
    }
    NLC_CK(cudaEventRecord(ev_main, ss));
    NLC_CK(cudaStreamWaitEvent(st, ev_main, 0));
    const int e1 = mark();
    if (timer.on) timer.span(KID_ADJOINT, e0, e1);
    return NLC_OK;
  }

  // current state of instance I <-> a dense (g, Q) record
  nlc_status state_out(InstHost<T, G>& I, T* dst) {
    const int64_t n = I.d.n;
    cudaStream_t st = args_.stream;
    NLC_CK(cudaMemcpyAsync(dst, I.g[cur_], sizeof(T) * Q * n, cudaMemcpyDeviceToDevice, st));
    k_field_raw_out<T><<<grid1(n), 256, 0, st>>>(I.q[cur_], 5, I.d, dst + (int64_t)Q * n);
    NLC_CK_LAUNCH("k_field_raw_out");
    return NLC_OK;
  }

  nlc_status state_in(InstHost<T, G>& I, const T* src) {
    const int64_t n = I.d.n;
    cudaStream_t st = args_.stream;
    NLC_CK(cudaMemcpyAsync(I.g[cur_], src, sizeof(T) * Q * n, cudaMemcpyDeviceToDevice, st));
    k_field_raw_in<T, DIM><<<grid1(n), 256, 0, st>>>(src + (int64_t)Q * n, I.d, I.q[cur_]);
    NLC_CK_LAUNCH("k_field_raw_in");
    return NLC_OK;
  }

  // rho, u of Eq. 6 at the current state into stage[5n..9n)
  nlc_status moments_to_stage(InstHost<T, G>& I) {
    const int64_t n = I.d.n;
    cudaStream_t st = args_.stream;
    k_stress<Lat, T><<<grid1(n), 256, 0, st>>>(I.q[cur_], I.pi, I.d, I.p, iso_);
    NLC_CK_LAUNCH("k_stress");
    k_moments_out<Lat, T><<<grid1(n), 256, 0, st>>>(I.g[cur_], I.pi, I.d, I.p, I.stage + 5 * n,
                                                     I.stage + 6 * n, iso_);
    NLC_CK_LAUNCH("k_moments_out");
    return NLC_OK;
  }

  int mark() { return timer.on ? timer.mark(args_.stream) : -1; }

  nlc_status step_unfused() {
    cudaStream_t st = args_.stream;
    const int a = cur_, b = cur_ ^ 1;
    for (auto& I : inst_) {
      const int64_t n = I.d.n;
      const int e0 = mark();
      k_stress<Lat, T><<<grid1(n), 256, 0, st>>>(I.q[a], I.pi, I.d, I.p, iso_);
      NLC_CK_LAUNCH("k_stress");
      const int e1 = mark();
      k_lb<Lat, T><<<grid1(n), 256, 0, st>>>(I.g[a], I.g[b], I.pi, I.u, I.d, I.p,
                                             mrt_on_[&I - inst_.data()] ? I.mrt : nullptr, iso_);
      NLC_CK_LAUNCH("k_lb");
      const int e2 = mark();
      k_predict<Lat, T><<<grid1(n), 256, 0, st>>>(I.q[a], I.u, I.qp, I.r1, I.d, I.p, iso_);
      NLC_CK_LAUNCH("k_predict");
      const int e3 = mark();
      k_correct<Lat, T><<<grid1(n), 256, 0, st>>>(I.q[a], I.qp, I.r1, I.u, I.q[b], I.d, I.p,
                                                  iso_);
      NLC_CK_LAUNCH("k_correct");
      const int e4 = mark();
      if (timer.on) {
        timer.span(KID_STRESS, e0, e1);
        timer.span(KID_LB, e1, e2);
        timer.span(KID_PREDICT, e2, e3);
        timer.span(KID_CORRECT, e3, e4);
      }
    }
    cur_ = b;
    return NLC_OK;
  }

  // one step of every lattice: two launches over the joint tile list
  nlc_status step_fused(cudaStream_t st) {
    const int a = cur_;
    const int e0 = mark();
    cudaError_t e = launch_fused_lb<Lat, T>(insts_dev_, qmaps_dev_, tiles_dev_, ntiles_, a,
                                            derr_, st, any_mrt_, iso_, ix32_);
    if (e != cudaSuccess) {
      err = std::string("fused lb kernel: ") + cudaGetErrorString(e);
      return NLC_ECUDA;
    }
    const int e1 = mark();
    e = launch_fused_be<Lat, T>(insts_dev_, qmaps_dev_, umaps_dev_, tiles_dev_, ntiles_, a,
                                derr_, st, iso_);
    if (e != cudaSuccess) {
      err = std::string("fused Beris-Edwards kernel: ") + cudaGetErrorString(e);
      return NLC_ECUDA;
    }
    const int e2 = mark();
    if (timer.on) {
      timer.span(KID_FUSED_LB, e0, e1);
      timer.span(KID_FUSED_BE, e1, e2);
    }
    cur_ ^= 1;
    return NLC_OK;
  }

  // len fused steps on the context's stream; runs of a few steps or more
  // replay a captured graph of exactly len steps (cached per buffer parity
  // and length) instead of launching kernel by kernel
  nlc_status fused_steps(int64_t len) {
    if (len < 4 || timer.on) {
      for (int64_t j = 0; j < len; j++) {
        nlc_status s = step_fused(args_.stream);
        if (s) return s;
      }
      return NLC_OK;
    }
    cudaGraphExec_t ex = nullptr;
    for (const SweepGraph& e : sweep_graphs_)
      if (e.parity == cur_ && e.len == len) ex = e.exec;
    if (!ex) {
      nlc_status s = capture_steps(cur_, (int)len, &ex);
      if (s) return s;
      sweep_graphs_.push_back(SweepGraph{cur_, len, ex});
    }
    NLC_CK(cudaGraphLaunch(ex, args_.stream));
    if (len & 1) cur_ ^= 1;
    return NLC_OK;
  }

  // captures len fused steps starting from buffer parity c
  nlc_status capture_steps(int c, int len, cudaGraphExec_t* out) {
    if (!cap_stream_) NLC_CK(cudaStreamCreateWithFlags(&cap_stream_, cudaStreamNonBlocking));
    // the persistent kernel's occupancy query and barrier allocation happen
    // before the capture (no allocation may happen inside one)
    if (persistent_steps > 0 && !any_mrt_) {
      int grid;
      nlc_status ps = persist_grid(&grid);
      if (ps) return ps;
    }
    const int saved = cur_;
    cur_ = c;
    NLC_CK(cudaStreamBeginCapture(cap_stream_, cudaStreamCaptureModeThreadLocal));
    nlc_status s = NLC_OK;
    s = fused_launches(len, cap_stream_);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap_stream_, &g);
    cur_ = saved;
    if (s != NLC_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) {
      err = std::string("stream capture: ") + cudaGetErrorString(e);
      return NLC_ECUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      err = std::string("graph instantiate: ") + cudaGetErrorString(e);
      return NLC_ECUDA;
    }
    return NLC_OK;
  }

  // captures graph_steps fused steps starting from buffer parity c
  nlc_status ensure_graph(int c) {
    if (graph_[c] && graph_len_[c] == graph_steps && graph_pers_[c] == persistent_steps)
      return NLC_OK;
    if (graph_[c]) {
      cudaGraphExecDestroy(graph_[c]);
      graph_[c] = nullptr;
    }
    nlc_status s = capture_steps(c, graph_steps, &graph_[c]);
    if (s) return s;
    graph_len_[c] = graph_steps;
    graph_pers_[c] = persistent_steps;
    return NLC_OK;
  }

  EngineArgs args_;
  std::vector<InstHost<T, G>> inst_;
  std::vector<void*> allocs_;
  InstDev<T, G>* insts_dev_ = nullptr;
  CUtensorMap* qmaps_dev_ = nullptr;
  CUtensorMap* umaps_dev_ = nullptr;
  TileRef* tiles_dev_ = nullptr;
  size_t tiles_cap_ = 0;
  bool taper_ = false;  // tapered chunk lists (chunk_bounds)
  int ntiles_ = 0;
  bool maps_ok_ = false;
  unsigned long long* bad_ = nullptr;
  unsigned* derr_ = nullptr;
  int cur_ = 0;
  cudaStream_t cap_stream_ = nullptr;
  cudaGraphExec_t graph_[2] = {nullptr, nullptr};
  struct SweepGraph {
    int parity;
    int64_t len;
    cudaGraphExec_t exec;
  };
  std::vector<SweepGraph> sweep_graphs_;  // the adjoint's forward sweeps
  cudaStream_t side_stream_ = nullptr;    // adjoint segment records
  std::vector<bool> mrt_on_;              // per lattice: MRT collision
  bool any_mrt_ = false;
  bool iso_ = false;                      // isotropic stencils
  bool ix32_ = false;                     // Q n < 2^32 on every lattice (pop_off)
  cudaEvent_t seg_ev_[5] = {};
  int graph_len_[2] = {0, 0};
  int graph_pers_[2] = {0, 0};           // persistent_steps the graphs hold
  int pgrid_max_[4] = {-1, -1, -1, -1};  // persistent blocks per (iso, ix32)
  GridBarrier* pbar_ = nullptr;          // persistent kernel's grid barrier
};

template <class Lat, class T, class G = T>
std::unique_ptr<EngineBase> make_engine(const EngineArgs& a, nlc_status* st,
                                        std::string* msg) {
  auto e = std::make_unique<Engine<Lat, T, G>>(a);
  *st = e->init();
  if (*st != NLC_OK) {
    *msg = e->err;
    return nullptr;
  }
  return e;
}

}  // namespace nlc
