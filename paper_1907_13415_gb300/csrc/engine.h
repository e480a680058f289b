// engine.h -- host-side interface between the C ABI and the templated
// per-lattice, per-precision engines.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "../../include/nlc.h"

namespace nlc {

// kernel ids of the timing log (names in nlc_timing_name)
enum KernelId { KID_FUSED_LB = 0, KID_FUSED_BE, KID_STRESS, KID_LB, KID_PREDICT,
                KID_CORRECT, KID_ADJOINT, KID_PERSIST, KID_COUNT };

// CUDA events recorded around kernel launches while timing is on.
class KernelTimer {
 public:
  ~KernelTimer() {
    for (cudaEvent_t e : pool_) cudaEventDestroy(e);
  }
  bool on = false;
  void reset() {
    used_ = 0;
    spans_.clear();
  }
  // records an event on st and returns its index (or -1 when out of events)
  int mark(cudaStream_t st) {
    if (used_ == pool_.size()) {
      if (pool_.size() >= kMaxEvents) return -1;
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      pool_.push_back(e);
    }
    if (cudaEventRecord(pool_[used_], st) != cudaSuccess) return -1;
    return (int)used_++;
  }
  void span(int kid, int a, int b) {
    if (a >= 0 && b >= 0) spans_.push_back({kid, a, b});
  }
  cudaError_t totals(double* ms, int64_t* launches) {
    for (int k = 0; k < KID_COUNT; k++) {
      ms[k] = 0.0;
      launches[k] = 0;
    }
    for (const Span& s : spans_) {
      float t = 0.f;
      cudaError_t e = cudaEventSynchronize(pool_[s.b]);
      if (e != cudaSuccess) return e;
      e = cudaEventElapsedTime(&t, pool_[s.a], pool_[s.b]);
      if (e != cudaSuccess) return e;
      ms[s.kid] += t;
      launches[s.kid] += 1;
    }
    return cudaSuccess;
  }

 private:
  struct Span {
    int kid, a, b;
  };
  static constexpr size_t kMaxEvents = 1 << 16;
  std::vector<cudaEvent_t> pool_;
  size_t used_ = 0;
  std::vector<Span> spans_;
};

struct EngineBase {
  virtual ~EngineBase() = default;
  KernelTimer timer;
  int graph_steps = 0;  // >0: whole chunks of this many steps replay a CUDA graph
  // budget in nanoseconds of every grid-barrier wait of the persistent
  // kernels (a wait that runs out ends the call with NLC_ETIMEOUT)
  uint64_t wait_ns = 200ull * 1000 * 1000;
  // >0: fused steps run as cooperative launches of the persistent kernel,
  // each advancing up to this many steps (nlc_set_persistent)
  int persistent_steps = 0;
  virtual int count() const = 0;
  // drops the captured step graphs (after a change of how steps launch)
  virtual void invalidate_graphs() = 0;
  // number of non-finite stored values of each lattice (syncs); first bad
  // lattice in *bad (-1 if none)
  virtual nlc_status check_finite(int* bad) = 0;
  virtual nlc_status set_params(int inst, const nlc_params& p) = 0;
  virtual nlc_status set_mrt(int inst, const double* rates) = 0;
  virtual nlc_status set_stencil(bool isotropic) = 0;
  // z planes per block of the fused kernels on three-dimensional lattices:
  // tz > 0 for every lattice (capped at its nz), 0 for the default choice;
  // taper: the last chunks of every column shrink (chunk_bounds)
  virtual nlc_status set_chunk(int tz, bool taper) = 0;
  virtual int chunk(int inst) const = 0;
  virtual bool tapered() const = 0;
  // times `trial_steps` fused steps for each candidate chunk depth on the
  // current state, restores the state and keeps the fastest depth
  virtual nlc_status autotune(int trial_steps, nlc_tune* out) = 0;
  virtual nlc_status step(int64_t n, int schedule) = 0;
  virtual nlc_status set_fields(int inst, const double* Q5, const double* rho,
                                const double* u) = 0;
  // Q from float32, rho = rho0, u = 0
  virtual nlc_status set_fields_f32(int inst, const float* Q5) = 0;
  virtual nlc_status get_fields(int inst, double* Q5, double* rho, double* u) = 0;
  virtual nlc_status get_populations(int inst, double* f) = 0;
  virtual nlc_status observables(int inst, nlc_obs* out, double* s_profile) = 0;
  virtual nlc_status adjoint(const nlc_loss* loss, int64_t nsteps, int ckpt_every,
                             nlc_grad* out, double* dQ0) = 0;
  // raw device state: populations (current buffer) then Q interior
  virtual size_t state_bytes() const = 0;
  virtual nlc_status save_state(void* dst) = 0;
  virtual nlc_status load_state(const void* src) = 0;
  std::string err;
};

struct EngineArgs {
  int n;                           // lattices in the context
  std::vector<nlc_grid> grids;     // n entries, same lattice and precision
  std::vector<nlc_params> params;  // n entries
  cudaStream_t stream;
};

// factories, one per translation unit (lattice x precision)
std::unique_ptr<EngineBase> make_engine_d2q9_f64(const EngineArgs&, nlc_status*, std::string*);
std::unique_ptr<EngineBase> make_engine_d2q9_f32(const EngineArgs&, nlc_status*, std::string*);
std::unique_ptr<EngineBase> make_engine_d3q19_f64(const EngineArgs&, nlc_status*, std::string*);
std::unique_ptr<EngineBase> make_engine_d3q19_f32(const EngineArgs&, nlc_status*, std::string*);
std::unique_ptr<EngineBase> make_engine_d2q9_f64f32(const EngineArgs&, nlc_status*, std::string*);
std::unique_ptr<EngineBase> make_engine_d3q19_f64f32(const EngineArgs&, nlc_status*, std::string*);

}  // namespace nlc
