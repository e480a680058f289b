// engine.cuh -- the templated engine: device buffers of one lattice and the
// launch sequences of the step, set-up, read-back and observables.
#pragma once
#include <cmath>
#include <cstdio>
#include <vector>

#include "aux_kernels.cuh"
#include "engine.h"
#include "step_fused.cuh"
#include "step_unfused.cuh"

namespace nlc {

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

template <class Lat, class T>
class Engine final : public EngineBase {
 public:
  static constexpr int Q = Lat::Q;
  static constexpr int DIM = Lat::DIM;

  explicit Engine(const EngineArgs& a) : args_(a) {
    d_.nx = a.grid.nx;
    d_.ny = a.grid.ny;
    d_.nz = a.grid.nz;
    d_.n = (int64_t)a.grid.nx * a.grid.ny * a.grid.nz;
    L_ = make_layout(d_, DIM == 3);
    const nlc_params& q = a.params;
    p_.A0 = (T)q.A0;
    p_.K = (T)q.K;
    p_.gamma = (T)q.gamma;
    p_.Gamma = (T)q.Gamma;
    p_.xi = (T)q.xi;
    p_.tau = (T)q.tau;
    p_.rho0 = (T)q.rho0;
    p_.inv_tau = (T)(1.0 / q.tau);
    p_.guo = (T)(1.0 - 1.0 / (2.0 * q.tau));
  }

  ~Engine() override {
    for (void* ptr : allocs_) cudaFree(ptr);
  }

  nlc_status init() {
    const int64_t n = d_.n;
    nlc_status s;
    T *q0, *q1, *u;
    if ((s = alloc(&g_[0], (size_t)Q * n)) || (s = alloc(&g_[1], (size_t)Q * n)) ||
        (s = alloc(&q0, (size_t)5 * L_.comp)) || (s = alloc(&q1, (size_t)5 * L_.comp)) ||
        (s = alloc(&u, (size_t)DIM * L_.comp)) || (s = alloc(&bad_, 1)) ||
        (s = alloc(&derr_, 1)))
      return s;
    q_[0] = Field<T>{q0, L_};
    q_[1] = Field<T>{q1, L_};
    u_ = Field<T>{u, L_};
    cudaStream_t st = args_.stream;
    NLC_CK(cudaMemsetAsync(g_[0], 0, sizeof(T) * Q * n, st));
    NLC_CK(cudaMemsetAsync(q0, 0, sizeof(T) * 5 * L_.comp, st));
    NLC_CK(cudaMemsetAsync(q1, 0, sizeof(T) * 5 * L_.comp, st));
    NLC_CK(cudaMemsetAsync(u, 0, sizeof(T) * DIM * L_.comp, st));
    NLC_CK(cudaMemsetAsync(derr_, 0, sizeof(unsigned), st));
    // TMA descriptors of the three padded fields (pointers never change)
    maps_ok_ = encode_field_map<T>(&qmap_[0], q0, L_.nxp, L_.nyp, L_.nzp, 5, BXW, BYH) &&
               encode_field_map<T>(&qmap_[1], q1, L_.nxp, L_.nyp, L_.nzp, 5, BXW, BYH) &&
               encode_field_map<T>(&umap_, u, L_.nxp, L_.nyp, L_.nzp, DIM, BXW, BYH);
    return NLC_OK;
  }

  // ---------------------------------------------------------------- step
  nlc_status step(int64_t n, int schedule) override {
    if (n <= 0) return NLC_OK;
    nlc_status s;
    if (schedule == NLC_SCHED_UNFUSED) {
      if ((s = ensure_unfused())) return s;
      for (int64_t k = 0; k < n; k++)
        if ((s = step_unfused())) return s;
      return NLC_OK;
    }
    if (!maps_ok_) {
      err = "TMA tensor maps unavailable (driver entry point missing); use the "
            "unfused schedule";
      return NLC_EUNSUPPORTED;
    }
    for (int64_t k = 0; k < n; k++)
      if ((s = step_fused())) return s;
    return NLC_OK;
  }

  // ---------------------------------------------------------------- I/O
  nlc_status set_fields(const double* Q5, const double* rho,
                        const double* u) override {
    nlc_status s;
    if ((s = ensure_staging())) return s;
    const int64_t n = d_.n;
    cudaStream_t st = args_.stream;
    NLC_CK(cudaMemcpyAsync(stage_, Q5, sizeof(double) * 5 * n, cudaMemcpyHostToDevice, st));
    if (rho)
      NLC_CK(cudaMemcpyAsync(stage_ + 5 * n, rho, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    if (u)
      NLC_CK(cudaMemcpyAsync(stage_ + 6 * n, u, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    NLC_CK(cudaMemsetAsync(bad_, 0, sizeof(unsigned long long), st));
    cur_ = 0;
    k_set_fields<Lat, T><<<grid1(n), 256, 0, st>>>(
        stage_, rho ? stage_ + 5 * n : nullptr, u ? stage_ + 6 * n : nullptr,
        q_[0], g_[0], d_, args_.params.rho0, bad_);
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

  nlc_status get_fields(double* Q5, double* rho, double* u) override {
    nlc_status s;
    if ((s = ensure_staging())) return s;
    const int64_t n = d_.n;
    cudaStream_t st = args_.stream;
    if (Q5) {
      k_field_out<T><<<grid1(n), 256, 0, st>>>(q_[cur_], 5, d_, stage_);
      NLC_CK_LAUNCH("k_field_out");
      NLC_CK(cudaMemcpyAsync(Q5, stage_, sizeof(double) * 5 * n, cudaMemcpyDeviceToHost, st));
    }
    if (rho || u) {
      if ((s = moments_to_stage())) return s;
      if (rho)
        NLC_CK(cudaMemcpyAsync(rho, stage_ + 5 * n, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
      if (u)
        NLC_CK(cudaMemcpyAsync(u, stage_ + 6 * n, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    }
    NLC_CK(cudaStreamSynchronize(st));
    return device_error();
  }

  nlc_status get_populations(double* f) override {
    nlc_status s;
    if ((s = ensure_fstage())) return s;
    const int64_t n = d_.n;
    cudaStream_t st = args_.stream;
    k_populations_out<Lat, T><<<grid1(n), 256, 0, st>>>(g_[cur_], d_, args_.params.rho0, fstage_);
    NLC_CK_LAUNCH("k_populations_out");
    NLC_CK(cudaMemcpyAsync(f, fstage_, sizeof(double) * Q * n, cudaMemcpyDeviceToHost, st));
    NLC_CK(cudaStreamSynchronize(st));
    return device_error();
  }

  size_t state_bytes() const override { return sizeof(T) * (size_t)(Q + 5) * (size_t)d_.n; }

  nlc_status save_state(void* dst) override {
    nlc_status s;
    if ((s = ensure_raw())) return s;
    const int64_t n = d_.n;
    cudaStream_t st = args_.stream;
    k_field_raw_out<T><<<grid1(n), 256, 0, st>>>(q_[cur_], 5, d_, raw_);
    NLC_CK_LAUNCH("k_field_raw_out");
    NLC_CK(cudaMemcpyAsync(dst, g_[cur_], sizeof(T) * Q * n, cudaMemcpyDeviceToHost, st));
    NLC_CK(cudaMemcpyAsync((char*)dst + sizeof(T) * Q * n, raw_, sizeof(T) * 5 * n,
                           cudaMemcpyDeviceToHost, st));
    NLC_CK(cudaStreamSynchronize(st));
    return device_error();
  }

  nlc_status load_state(const void* src) override {
    nlc_status s;
    if ((s = ensure_raw())) return s;
    const int64_t n = d_.n;
    cudaStream_t st = args_.stream;
    NLC_CK(cudaMemcpyAsync(g_[0], src, sizeof(T) * Q * n, cudaMemcpyHostToDevice, st));
    NLC_CK(cudaMemcpyAsync(raw_, (const char*)src + sizeof(T) * Q * n, sizeof(T) * 5 * n,
                           cudaMemcpyHostToDevice, st));
    k_field_raw_in<T, DIM><<<grid1(n), 256, 0, st>>>(raw_, d_, q_[0]);
    NLC_CK_LAUNCH("k_field_raw_in");
    NLC_CK(cudaStreamSynchronize(st));
    cur_ = 0;
    return NLC_OK;
  }

  nlc_status observables(nlc_obs* out, double* s_profile) override {
    nlc_status s;
    if ((s = ensure_staging())) return s;
    const int64_t n = d_.n;
    cudaStream_t st = args_.stream;
    if ((s = moments_to_stage())) return s;
    const double s_ref = 1.0 / 3.0;
    k_obs_partial<Lat, T><<<obs_blocks_, 256, 0, st>>>(
        q_[cur_], g_[cur_], stage_ + 5 * n, stage_ + 6 * n, d_, p_, s_ref, partial_);
    NLC_CK_LAUNCH("k_obs_partial");
    k_obs_final<<<1, 256, 0, st>>>(partial_, obs_blocks_, partial_ + obs_blocks_ * OBS_SLOTS);
    NLC_CK_LAUNCH("k_obs_final");
    const int64_t rows = (int64_t)d_.ny * d_.nz;
    const int rows_per_chunk = 64;
    const int nchunks = (int)((rows + rows_per_chunk - 1) / rows_per_chunk);
    dim3 pg((d_.nx + 127) / 128, nchunks);
    k_profile_partial<T><<<pg, 128, 0, st>>>(q_[cur_], d_, rows_per_chunk, prof_partial_);
    NLC_CK_LAUNCH("k_profile_partial");
    k_profile_final<<<(d_.nx + 127) / 128, 128, 0, st>>>(prof_partial_, nchunks, d_, prof_);
    NLC_CK_LAUNCH("k_profile_final");
    double tot[OBS_SLOTS];
    std::vector<double> prof(d_.nx);
    NLC_CK(cudaMemcpyAsync(tot, partial_ + obs_blocks_ * OBS_SLOTS, sizeof(tot), cudaMemcpyDeviceToHost, st));
    NLC_CK(cudaMemcpyAsync(prof.data(), prof_, sizeof(double) * d_.nx, cudaMemcpyDeviceToHost, st));
    NLC_CK(cudaStreamSynchronize(st));
    if ((s = device_error())) return s;
    out->mass = tot[0];
    out->mom[0] = tot[1];
    out->mom[1] = tot[2];
    out->mom[2] = tot[3];
    out->s_area = tot[4];
    out->free_energy = tot[5];
    out->nonfinite = (int64_t)tot[6];
    out->max_u = tot[7];
    out->radius = (DIM == 2 || d_.nz == 1) ? std::sqrt(tot[4] / M_PI)
                                           : std::cbrt(3.0 * tot[4] / (4.0 * M_PI));
    const double half = s_ref / 2.0;
    out->x_iface = -1.0;
    for (int x = 0; x < d_.nx; x++) {
      const double a = prof[x], b = prof[(x + 1) % d_.nx];
      if (a >= half && b < half) {
        out->x_iface = x + (a - half) / (a - b);
        break;
      }
    }
    if (s_profile)
      for (int x = 0; x < d_.nx; x++) s_profile[x] = prof[x];
    return NLC_OK;
  }

 private:
  static unsigned grid1(int64_t count) { return (unsigned)((count + 255) / 256); }

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

  // device-side error word (bounded waits that ran out); read after a sync
  nlc_status device_error() {
    unsigned e = 0;
    NLC_CK(cudaMemcpy(&e, derr_, sizeof(e), cudaMemcpyDeviceToHost));
    if (e != DEV_ERR_NONE) {
      err = "a bounded wait on a tile copy ran out inside a step kernel (code " +
            std::to_string(e) + ")";
      return NLC_ETIMEOUT;
    }
    return NLC_OK;
  }

  nlc_status ensure_unfused() {
    if (pi_) return NLC_OK;
    nlc_status s;
    const int64_t n = d_.n;
    T* qp;
    if ((s = alloc(&pi_, (size_t)DIM * DIM * n)) || (s = alloc(&qp, (size_t)5 * L_.comp)) ||
        (s = alloc(&r1_, (size_t)5 * n)))
      return s;
    qp_ = Field<T>{qp, L_};
    return NLC_OK;
  }

  nlc_status ensure_staging() {
    if (stage_) return NLC_OK;
    nlc_status s;
    const int64_t n = d_.n;
    if ((s = alloc(&stage_, (size_t)9 * n))) return s;
    if ((s = ensure_unfused())) return s;
    int dev = 0, sms = 0;
    NLC_CK(cudaGetDevice(&dev));
    NLC_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int64_t want = (n + 255) / 256;
    obs_blocks_ = (int)(want < 4 * sms ? want : 4 * sms);
    if (obs_blocks_ < 1) obs_blocks_ = 1;
    if ((s = alloc(&partial_, (size_t)(obs_blocks_ + 1) * OBS_SLOTS))) return s;
    const int64_t rows = (int64_t)d_.ny * d_.nz;
    const int64_t nchunks = (rows + 63) / 64;
    if ((s = alloc(&prof_partial_, (size_t)(nchunks * d_.nx)))) return s;
    if ((s = alloc(&prof_, (size_t)d_.nx))) return s;
    return NLC_OK;
  }

  nlc_status ensure_raw() {
    if (raw_) return NLC_OK;
    return alloc(&raw_, (size_t)5 * d_.n);
  }

  nlc_status ensure_fstage() {
    if (fstage_) return NLC_OK;
    return alloc(&fstage_, (size_t)Q * d_.n);
  }

  // rho, u of Eq. 6 at the current state into stage_[5n..9n)
  nlc_status moments_to_stage() {
    const int64_t n = d_.n;
    cudaStream_t st = args_.stream;
    k_stress<Lat, T><<<grid1(n), 256, 0, st>>>(q_[cur_], pi_, d_, p_);
    NLC_CK_LAUNCH("k_stress");
    k_moments_out<Lat, T><<<grid1(n), 256, 0, st>>>(g_[cur_], pi_, d_, p_,
                                                     stage_ + 5 * n, stage_ + 6 * n);
    NLC_CK_LAUNCH("k_moments_out");
    return NLC_OK;
  }

  int mark() { return timer.on ? timer.mark(args_.stream) : -1; }

  nlc_status step_unfused() {
    const int64_t n = d_.n;
    cudaStream_t st = args_.stream;
    const int a = cur_, b = cur_ ^ 1;
    const int e0 = mark();
    k_stress<Lat, T><<<grid1(n), 256, 0, st>>>(q_[a], pi_, d_, p_);
    NLC_CK_LAUNCH("k_stress");
    const int e1 = mark();
    k_lb<Lat, T><<<grid1(n), 256, 0, st>>>(g_[a], g_[b], pi_, u_, d_, p_);
    NLC_CK_LAUNCH("k_lb");
    const int e2 = mark();
    k_predict<Lat, T><<<grid1(n), 256, 0, st>>>(q_[a], u_, qp_, r1_, d_, p_);
    NLC_CK_LAUNCH("k_predict");
    const int e3 = mark();
    k_correct<Lat, T><<<grid1(n), 256, 0, st>>>(q_[a], qp_, r1_, u_, q_[b], d_, p_);
    NLC_CK_LAUNCH("k_correct");
    const int e4 = mark();
    if (timer.on) {
      timer.span(KID_STRESS, e0, e1);
      timer.span(KID_LB, e1, e2);
      timer.span(KID_PREDICT, e2, e3);
      timer.span(KID_CORRECT, e3, e4);
    }
    cur_ = b;
    return NLC_OK;
  }

  nlc_status step_fused() {
    cudaStream_t st = args_.stream;
    const int a = cur_, b = cur_ ^ 1;
    const int e0 = mark();
    cudaError_t e = launch_fused_lb<Lat, T>(qmap_[a], g_[a], g_[b], u_, d_, p_, derr_, st);
    if (e != cudaSuccess) {
      err = std::string("fused lb kernel: ") + cudaGetErrorString(e);
      return NLC_ECUDA;
    }
    const int e1 = mark();
    e = launch_fused_be<Lat, T>(qmap_[a], umap_, q_[b], d_, p_, derr_, st);
    if (e != cudaSuccess) {
      err = std::string("fused Beris-Edwards kernel: ") + cudaGetErrorString(e);
      return NLC_ECUDA;
    }
    const int e2 = mark();
    if (timer.on) {
      timer.span(KID_FUSED_LB, e0, e1);
      timer.span(KID_FUSED_BE, e1, e2);
    }
    cur_ = b;
    return NLC_OK;
  }

  EngineArgs args_;
  Dims d_;
  Layout L_;
  Par<T> p_;
  std::vector<void*> allocs_;
  T* g_[2] = {nullptr, nullptr};
  Field<T> q_[2];
  Field<T> u_;
  Field<T> qp_;
  CUtensorMap qmap_[2];
  CUtensorMap umap_;
  bool maps_ok_ = false;
  T* pi_ = nullptr;
  T* r1_ = nullptr;
  T* raw_ = nullptr;
  double* stage_ = nullptr;
  double* fstage_ = nullptr;
  double* partial_ = nullptr;
  double* prof_partial_ = nullptr;
  double* prof_ = nullptr;
  unsigned long long* bad_ = nullptr;
  unsigned* derr_ = nullptr;
  int obs_blocks_ = 1;
  int cur_ = 0;
};

template <class Lat, class T>
std::unique_ptr<EngineBase> make_engine(const EngineArgs& a, nlc_status* st,
                                        std::string* msg) {
  auto e = std::make_unique<Engine<Lat, T>>(a);
  *st = e->init();
  if (*st != NLC_OK) {
    *msg = e->err;
    return nullptr;
  }
  return e;
}

}  // namespace nlc
