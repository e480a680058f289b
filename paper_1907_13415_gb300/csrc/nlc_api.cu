// nlc_api.cpp -- the C ABI of libnlc (declared in include/nlc.h).
//
// Argument checking, context ownership and error reporting; the work is done
// by the templated engines (engine.cuh), one per lattice and precision.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/nlc.h"
#include "engine.h"
#include "lattice.cuh"
#include "tune_cache.h"
#include "nvtx_range.h"

using nlc::NvtxRange;

static_assert(nlc::KID_COUNT == NLC_N_KERNELS, "kernel id table out of sync");

struct nlc_ctx {
  std::vector<nlc_grid> grids;
  std::vector<nlc_params> params;
  cudaStream_t stream = nullptr;
  int device = 0;
  int schedule = NLC_SCHED_FUSED;
  int check_every = 0;
  std::vector<int64_t> steps;  // per lattice, since its last nlc_set_fields
  std::vector<char> mrt;       // per lattice: MRT collision on
  bool iso = false;            // isotropic stencils
  std::unique_ptr<nlc::EngineBase> eng;
  std::string err;
};

namespace {

nlc_status fail(nlc_ctx* ctx, nlc_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

bool finite(double v) { return std::isfinite(v); }

nlc_status check_grid(const nlc_grid* g, std::string* msg) {
  if (!g) {
    *msg = "grid is NULL";
    return NLC_EINVAL;
  }
  if (g->lattice != NLC_D2Q9 && g->lattice != NLC_D3Q19) {
    *msg = "unknown lattice " + std::to_string(g->lattice);
    return NLC_EINVAL;
  }
  if (g->precision != NLC_FP64 && g->precision != NLC_FP32 && g->precision != NLC_FP32_QF64) {
    *msg = "unknown precision " + std::to_string(g->precision);
    return NLC_EINVAL;
  }
  if (g->nx < 1 || g->ny < 1 || g->nz < 1) {
    *msg = "lattice extents must be >= 1";
    return NLC_EINVAL;
  }
  if (g->lattice == NLC_D2Q9 && g->nz != 1) {
    *msg = "D2Q9 needs nz = 1";
    return NLC_EINVAL;
  }
  const double cells = (double)g->nx * g->ny * g->nz;
  if (cells > 4.0e9) {
    *msg = "lattice too large";
    return NLC_EINVAL;
  }
  return NLC_OK;
}

nlc_status check_params(const nlc_params* p, std::string* msg) {
  if (!p) {
    *msg = "params is NULL";
    return NLC_EINVAL;
  }
  const double v[7] = {p->A0, p->K, p->gamma, p->Gamma, p->xi, p->tau, p->rho0};
  for (double x : v)
    if (!finite(x)) {
      *msg = "parameters must be finite";
      return NLC_EINVAL;
    }
  if (!(p->tau > 0.5)) {
    *msg = "tau must exceed 1/2";
    return NLC_EINVAL;
  }
  if (!(p->rho0 > 0.0)) {
    *msg = "rho0 must be positive";
    return NLC_EINVAL;
  }
  if (p->K < 0.0 || p->Gamma < 0.0) {
    *msg = "K and Gamma must be non-negative";
    return NLC_EINVAL;
  }
  return NLC_OK;
}

}  // namespace

extern "C" {

nlc_status nlc_create_batch(int32_t n, const nlc_grid* grids,
                            const nlc_params* params, void* stream,
                            nlc_ctx** out) {
  if (!out) return NLC_EINVAL;
  *out = nullptr;
  if (n < 1 || !grids || !params) return NLC_EINVAL;
  std::string msg;
  for (int i = 0; i < n; i++) {
    nlc_status st = check_grid(&grids[i], &msg);
    if (st == NLC_OK) st = check_params(&params[i], &msg);
    if (st != NLC_OK) return st;
    if (grids[i].lattice != grids[0].lattice || grids[i].precision != grids[0].precision)
      return NLC_EINVAL;  // one lattice type and precision per context
  }
  nlc_ctx* ctx = new (std::nothrow) nlc_ctx();
  if (!ctx) return NLC_ENOMEM;
  ctx->grids.assign(grids, grids + n);
  ctx->params.assign(params, params + n);
  ctx->steps.assign(n, 0);
  ctx->mrt.assign(n, 0);
  ctx->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&ctx->device) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return NLC_ECUDA;
  }
  nlc::EngineArgs a{n, ctx->grids, ctx->params, ctx->stream};
  const bool d3 = grids[0].lattice == NLC_D3Q19;
  const int32_t prec = grids[0].precision;
  nlc_status st = NLC_OK;
  if (d3)
    ctx->eng = prec == NLC_FP64   ? nlc::make_engine_d3q19_f64(a, &st, &msg)
               : prec == NLC_FP32 ? nlc::make_engine_d3q19_f32(a, &st, &msg)
                                  : nlc::make_engine_d3q19_f64f32(a, &st, &msg);
  else
    ctx->eng = prec == NLC_FP64   ? nlc::make_engine_d2q9_f64(a, &st, &msg)
               : prec == NLC_FP32 ? nlc::make_engine_d2q9_f32(a, &st, &msg)
                                  : nlc::make_engine_d2q9_f64f32(a, &st, &msg);
  if (!ctx->eng) {
    delete ctx;
    return st != NLC_OK ? st : NLC_ECUDA;
  }
  *out = ctx;
  return NLC_OK;
}

nlc_status nlc_create(const nlc_grid* grid, const nlc_params* params,
                      void* stream, nlc_ctx** out) {
  return nlc_create_batch(1, grid, params, stream, out);
}

nlc_status nlc_set_params(nlc_ctx* ctx, int32_t inst, const nlc_params* params) {
  if (!ctx) return NLC_EINVAL;
  if (inst < 0 || inst >= (int32_t)ctx->grids.size())
    return fail(ctx, NLC_EINVAL, "instance out of range");
  std::string msg;
  nlc_status st = check_params(params, &msg);
  if (st != NLC_OK) return fail(ctx, st, msg);
  st = ctx->eng->set_params(inst, *params);
  if (st != NLC_OK) return fail(ctx, st, ctx->eng->err);
  ctx->params[inst] = *params;
  return NLC_OK;
}

nlc_status nlc_set_mrt(nlc_ctx* ctx, int32_t inst, const double* rates, int32_t n) {
  if (!ctx) return NLC_EINVAL;
  if (inst < 0 || inst >= (int32_t)ctx->grids.size())
    return fail(ctx, NLC_EINVAL, "instance out of range");
  if (rates) {
    const int32_t q = ctx->grids[inst].lattice == NLC_D2Q9 ? 9 : 19;
    if (n != q) return fail(ctx, NLC_EINVAL, "one rate per velocity (moment) is needed");
    for (int32_t k = 0; k < n; k++)
      if (!(rates[k] > 0.0 && rates[k] < 2.0))
        return fail(ctx, NLC_EINVAL, "relaxation rates must lie in (0, 2)");
  }
  nlc_status st = ctx->eng->set_mrt(inst, rates);
  if (st != NLC_OK) return fail(ctx, st, ctx->eng->err);
  ctx->mrt[inst] = rates != nullptr;
  return NLC_OK;
}

nlc_status nlc_set_stencil(nlc_ctx* ctx, int32_t kind) {
  if (!ctx) return NLC_EINVAL;
  if (kind != NLC_STENCIL_STANDARD && kind != NLC_STENCIL_ISOTROPIC)
    return fail(ctx, NLC_EINVAL, "unknown stencil");
  nlc_status st = ctx->eng->set_stencil(kind == NLC_STENCIL_ISOTROPIC);
  if (st != NLC_OK) return fail(ctx, st, ctx->eng->err);
  ctx->iso = kind == NLC_STENCIL_ISOTROPIC;
  return NLC_OK;
}

nlc_status nlc_set_graph(nlc_ctx* ctx, int32_t steps) {
  if (!ctx) return NLC_EINVAL;
  if (steps < 0) return fail(ctx, NLC_EINVAL, "negative graph length");
  ctx->eng->graph_steps = steps;
  return NLC_OK;
}

nlc_status nlc_set_persistent(nlc_ctx* ctx, int32_t steps) {
  if (!ctx) return NLC_EINVAL;
  if (steps < 0) return fail(ctx, NLC_EINVAL, "negative persistent step count");
  if (steps != ctx->eng->persistent_steps) ctx->eng->invalidate_graphs();
  ctx->eng->persistent_steps = steps;
  return NLC_OK;
}

int32_t nlc_count(const nlc_ctx* ctx) { return ctx ? (int32_t)ctx->grids.size() : -1; }

nlc_status nlc_set_schedule(nlc_ctx* ctx, int32_t schedule) {
  if (!ctx) return NLC_EINVAL;
  if (schedule != NLC_SCHED_FUSED && schedule != NLC_SCHED_UNFUSED)
    return fail(ctx, NLC_EINVAL, "unknown schedule");
  ctx->schedule = schedule;
  return NLC_OK;
}

nlc_status nlc_set_chunk(nlc_ctx* ctx, int32_t chunk, int32_t taper) {
  if (!ctx) return NLC_EINVAL;
  if (chunk < 0) return fail(ctx, NLC_EINVAL, "negative chunk depth");
  if (taper != 0 && taper != 1) return fail(ctx, NLC_EINVAL, "taper must be 0 or 1");
  nlc_status st = ctx->eng->set_chunk(chunk, taper != 0);
  if (st != NLC_OK) return fail(ctx, st, ctx->eng->err);
  return NLC_OK;
}

int32_t nlc_get_chunk(const nlc_ctx* ctx, int32_t inst, int32_t* taper) {
  if (!ctx || inst < 0 || inst >= (int32_t)ctx->grids.size()) return -1;
  if (taper) *taper = ctx->eng->tapered() ? 1 : 0;
  return ctx->eng->chunk(inst);
}

// Cache key of the autotuner: what the timing depends on (lattice type,
// precision, extents, collision and stencils of every lattice, the GPU).
static std::string tune_key(const nlc_ctx* ctx) {
  const nlc_grid& g0 = ctx->grids[0];
  std::string k = g0.lattice == NLC_D2Q9 ? "D2Q9" : "D3Q19";
  k += g0.precision == NLC_FP64 ? "/fp64" : (g0.precision == NLC_FP32 ? "/fp32" : "/fp32_qf64");
  k += "/n" + std::to_string(ctx->grids.size()) + "/";
  for (size_t i = 0; i < ctx->grids.size(); i++) {
    const nlc_grid& g = ctx->grids[i];
    if (i) k += ",";
    k += std::to_string(g.nx) + "x" + std::to_string(g.ny) + "x" + std::to_string(g.nz);
    if (ctx->mrt[i]) k += "m";
  }
  k += ctx->iso ? "/iso" : "/std";
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, ctx->device) == cudaSuccess)
    k += std::string("/") + prop.name + "/" + std::to_string(prop.multiProcessorCount);
  else
    cudaGetLastError();
  return k;
}

nlc_status nlc_autotune(nlc_ctx* ctx, int32_t trial_steps, nlc_tune* out) {
  NvtxRange nvtx_range("nlc_autotune");
  if (!ctx) return NLC_EINVAL;
  if (trial_steps < 1) return fail(ctx, NLC_EINVAL, "trial_steps must be at least 1");
  nlc_tune res{};
  res.trial_steps = trial_steps;
  const char* env = std::getenv("NLC_TUNE_CACHE");
  const std::string path = env ? env : "";
  const std::string key = tune_key(ctx);
  long cached = 0;
  nlc_status st;
  // cached value: the chunk depth, negated for a tapered list
  if (!path.empty() && nlc::tune_cache_get(path, key, &cached) && cached != 0) {
    const bool taper = cached < 0;
    const int depth = (int)(cached < 0 ? -cached : cached);
    if ((st = ctx->eng->set_chunk(depth, taper)) != NLC_OK) return fail(ctx, st, ctx->eng->err);
    res.from_cache = 1;
    res.chunk = 1;
    for (size_t i = 0; i < ctx->grids.size(); i++)
      res.chunk = std::max(res.chunk, (int32_t)ctx->eng->chunk((int)i));
    res.taper = ctx->eng->tapered() ? 1 : 0;
  } else {
    if ((st = ctx->eng->autotune(trial_steps, &res)) != NLC_OK)
      return fail(ctx, st, ctx->eng->err);
    if (!path.empty() &&
        !nlc::tune_cache_put(path, key, res.taper ? -(long)res.chunk : (long)res.chunk))
      return fail(ctx, NLC_EINVAL, "nlc_autotune: cannot write the cache file " + path);
  }
  if (out) *out = res;
  return NLC_OK;
}

static bool bad_inst(const nlc_ctx* ctx, int32_t inst) {
  return inst < 0 || inst >= (int32_t)ctx->grids.size();
}

nlc_status nlc_set_fields(nlc_ctx* ctx, int32_t inst, const double* Q5,
                          const double* rho, const double* u) {
  NvtxRange nvtx_range("nlc_set_fields");
  if (!ctx) return NLC_EINVAL;
  if (bad_inst(ctx, inst)) return fail(ctx, NLC_EINVAL, "instance out of range");
  if (!Q5) return fail(ctx, NLC_EINVAL, "Q5 is NULL");
  nlc_status st = ctx->eng->set_fields(inst, Q5, rho, u);
  if (st != NLC_OK) return fail(ctx, st, ctx->eng->err);
  ctx->steps[inst] = 0;
  return NLC_OK;
}

nlc_status nlc_set_fields_f32(nlc_ctx* ctx, int32_t inst, const float* Q5) {
  NvtxRange nvtx_range("nlc_set_fields_f32");
  if (!ctx) return NLC_EINVAL;
  if (bad_inst(ctx, inst)) return fail(ctx, NLC_EINVAL, "instance out of range");
  if (!Q5) return fail(ctx, NLC_EINVAL, "Q5 is NULL");
  nlc_status st = ctx->eng->set_fields_f32(inst, Q5);
  if (st != NLC_OK) return fail(ctx, st, ctx->eng->err);
  ctx->steps[inst] = 0;
  return NLC_OK;
}

nlc_status nlc_get_fields(nlc_ctx* ctx, int32_t inst, double* Q5, double* rho,
                          double* u) {
  if (!ctx) return NLC_EINVAL;
  if (bad_inst(ctx, inst)) return fail(ctx, NLC_EINVAL, "instance out of range");
  nlc_status st = ctx->eng->get_fields(inst, Q5, rho, u);
  return st == NLC_OK ? st : fail(ctx, st, ctx->eng->err);
}

nlc_status nlc_get_populations(nlc_ctx* ctx, int32_t inst, double* f) {
  if (!ctx) return NLC_EINVAL;
  if (bad_inst(ctx, inst)) return fail(ctx, NLC_EINVAL, "instance out of range");
  if (!f) return fail(ctx, NLC_EINVAL, "f is NULL");
  nlc_status st = ctx->eng->get_populations(inst, f);
  return st == NLC_OK ? st : fail(ctx, st, ctx->eng->err);
}

nlc_status nlc_step(nlc_ctx* ctx, int64_t n) {
  NvtxRange nvtx_range("nlc_step");
  if (!ctx) return NLC_EINVAL;
  if (n < 0) return fail(ctx, NLC_EINVAL, "negative step count");
  const int64_t chunk = ctx->check_every > 0 ? ctx->check_every : n;
  for (int64_t done = 0; done < n;) {
    const int64_t k = std::min<int64_t>(chunk, n - done);
    nlc_status st = ctx->eng->step(k, ctx->schedule);
    if (st != NLC_OK) return fail(ctx, st, ctx->eng->err);
    for (auto& s : ctx->steps) s += k;
    done += k;
    if (ctx->check_every > 0) {
      int bad = -1;
      st = ctx->eng->check_finite(&bad);
      if (st != NLC_OK)
        return fail(ctx, st, ctx->eng->err + " after step " +
                                 std::to_string(bad >= 0 ? ctx->steps[bad] : ctx->steps[0]));
    }
  }
  return NLC_OK;
}

nlc_status nlc_set_check(nlc_ctx* ctx, int32_t every) {
  if (!ctx) return NLC_EINVAL;
  if (every < 0) return fail(ctx, NLC_EINVAL, "negative check interval");
  ctx->check_every = every;
  return NLC_OK;
}

nlc_status nlc_set_wait_budget(nlc_ctx* ctx, int64_t ns) {
  if (!ctx) return NLC_EINVAL;
  ctx->eng->wait_ns = ns < 0 ? 200ull * 1000 * 1000 : (uint64_t)ns;
  return NLC_OK;
}

nlc_status nlc_observables(nlc_ctx* ctx, int32_t inst, nlc_obs* out,
                           double* s_profile) {
  NvtxRange nvtx_range("nlc_observables");
  if (!ctx) return NLC_EINVAL;
  if (bad_inst(ctx, inst)) return fail(ctx, NLC_EINVAL, "instance out of range");
  if (!out) return fail(ctx, NLC_EINVAL, "out is NULL");
  nlc_status st = ctx->eng->observables(inst, out, s_profile);
  if (st != NLC_OK) return fail(ctx, st, ctx->eng->err);
  out->step = ctx->steps[inst];
  return NLC_OK;
}

namespace {

struct SaveHeader {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  int32_t count;         // lattices
  int32_t pad0;
  uint64_t desc_hash;    // checksum of the lattices' grids and parameters
  uint64_t payload_bytes;
  uint64_t checksum;     // of the payload (step counters, then the state)
};

const char kMagic[8] = {'N', 'L', 'C', 'S', 'T', 'A', 'T', 'E'};

// 64-bit FNV-1a over 8-byte little-endian words, then the tail bytes
uint64_t checksum64(const unsigned char* p, size_t n) {
  uint64_t h = 14695981039346656037ull;
  const uint64_t prime = 1099511628211ull;
  size_t i = 0;
  for (; i + 8 <= n; i += 8) {
    uint64_t w = 0;
    for (int b = 7; b >= 0; b--) w = (w << 8) | p[i + b];
    h ^= w;
    h *= prime;
  }
  for (; i < n; i++) {
    h ^= p[i];
    h *= prime;
  }
  return h;
}

uint64_t desc_hash(const nlc_ctx* ctx) {
  std::vector<unsigned char> b;
  for (size_t i = 0; i < ctx->grids.size(); i++) {
    const unsigned char* g = (const unsigned char*)&ctx->grids[i];
    const unsigned char* q = (const unsigned char*)&ctx->params[i];
    b.insert(b.end(), g, g + sizeof(nlc_grid));
    b.insert(b.end(), q, q + sizeof(nlc_params));
  }
  return checksum64(b.data(), b.size());
}

}  // namespace

nlc_status nlc_save(nlc_ctx* ctx, void* buf, size_t* len) {
  if (!ctx) return NLC_EINVAL;
  if (!len) return fail(ctx, NLC_EINVAL, "len is NULL");
  const size_t nst = sizeof(int64_t) * ctx->steps.size();
  const size_t payload = nst + ctx->eng->state_bytes();
  const size_t need = sizeof(SaveHeader) + payload;
  if (!buf) {
    *len = need;
    return NLC_OK;
  }
  if (*len < need) return fail(ctx, NLC_EINVAL, "buffer too small for the state");
  unsigned char* out = (unsigned char*)buf;
  std::memcpy(out + sizeof(SaveHeader), ctx->steps.data(), nst);
  nlc_status st = ctx->eng->save_state(out + sizeof(SaveHeader) + nst);
  if (st != NLC_OK) return fail(ctx, st, ctx->eng->err);
  SaveHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kMagic, 8);
  h.version = 1;
  h.header_bytes = sizeof(SaveHeader);
  h.count = (int32_t)ctx->grids.size();
  h.desc_hash = desc_hash(ctx);
  h.payload_bytes = payload;
  h.checksum = checksum64(out + sizeof(SaveHeader), payload);
  std::memcpy(out, &h, sizeof(h));
  *len = need;
  return NLC_OK;
}

nlc_status nlc_load(nlc_ctx* ctx, const void* buf, size_t len) {
  if (!ctx) return NLC_EINVAL;
  if (!buf || len < sizeof(SaveHeader)) return fail(ctx, NLC_EINVAL, "not a checkpoint");
  SaveHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != 1 ||
      h.header_bytes != sizeof(SaveHeader))
    return fail(ctx, NLC_EINVAL, "not a checkpoint of this format");
  if (h.count != (int32_t)ctx->grids.size() || h.desc_hash != desc_hash(ctx))
    return fail(ctx, NLC_EINVAL, "checkpoint is for other lattices or parameters");
  const size_t nst = sizeof(int64_t) * ctx->steps.size();
  const size_t payload = nst + ctx->eng->state_bytes();
  if (h.payload_bytes != payload || len < sizeof(SaveHeader) + payload)
    return fail(ctx, NLC_EINVAL, "checkpoint is truncated");
  const unsigned char* p = (const unsigned char*)buf + sizeof(SaveHeader);
  if (checksum64(p, payload) != h.checksum)
    return fail(ctx, NLC_ECORRUPT, "checkpoint checksum mismatch");
  nlc_status st = ctx->eng->load_state(p + nst);
  if (st != NLC_OK) return fail(ctx, st, ctx->eng->err);
  std::memcpy(ctx->steps.data(), p, nst);
  return NLC_OK;
}

nlc_status nlc_adjoint(nlc_ctx* ctx, const nlc_loss* loss, int64_t nsteps,
                       int32_t ckpt_every, nlc_grad* out, double* dQ0) {
  NvtxRange nvtx_range("nlc_adjoint");
  if (!ctx) return NLC_EINVAL;
  if (!loss || !out) return fail(ctx, NLC_EINVAL, "loss or out is NULL");
  if (nsteps < 1 || ckpt_every < 1) return fail(ctx, NLC_EINVAL, "nsteps and ckpt_every must be >= 1");
  if (ctx->grids.size() != 1) return fail(ctx, NLC_EINVAL, "the adjoint needs a single-lattice context");
  nlc_status st = ctx->eng->adjoint(loss, nsteps, ckpt_every, out, dQ0);
  if (st != NLC_OK) return fail(ctx, st, ctx->eng->err);
  ctx->steps[0] += nsteps;
  return NLC_OK;
}

nlc_status nlc_set_timing(nlc_ctx* ctx, int32_t enable) {
  if (!ctx) return NLC_EINVAL;
  if (enable) ctx->eng->timer.reset();
  ctx->eng->timer.on = enable != 0;
  return NLC_OK;
}

nlc_status nlc_get_timing(nlc_ctx* ctx, int32_t max_kernels, double* total_ms,
                          int64_t* launches, int32_t* n_kernels) {
  if (!ctx) return NLC_EINVAL;
  if (max_kernels < 0) return fail(ctx, NLC_EINVAL, "max_kernels < 0");
  double ms[nlc::KID_COUNT];
  int64_t cnt[nlc::KID_COUNT];
  cudaError_t e = ctx->eng->timer.totals(ms, cnt);
  if (e != cudaSuccess)
    return fail(ctx, NLC_ECUDA, std::string("timing: ") + cudaGetErrorString(e));
  for (int k = 0; k < nlc::KID_COUNT && k < max_kernels; k++) {
    if (total_ms) total_ms[k] = ms[k];
    if (launches) launches[k] = cnt[k];
  }
  if (n_kernels) *n_kernels = nlc::KID_COUNT;
  return NLC_OK;
}

const char* nlc_timing_name(int32_t k) {
  static const char* names[nlc::KID_COUNT] = {
      "fused_lb", "fused_be", "stress", "lb", "predict", "correct", "adjoint_step",
      "fused_persistent"};
  return (k >= 0 && k < nlc::KID_COUNT) ? names[k] : "?";
}

const char* nlc_last_error(const nlc_ctx* ctx) {
  return ctx ? ctx->err.c_str() : "context is NULL";
}

void nlc_destroy(nlc_ctx* ctx) { delete ctx; }

int32_t nlc_lattice_velocities(int32_t lattice, int32_t* c, double* w) {
  if (lattice != NLC_D2Q9 && lattice != NLC_D3Q19) return -1;
  const int q = lattice == NLC_D2Q9 ? nlc::LatD2Q9::Q : nlc::LatD3Q19::Q;
  for (int i = 0; i < q; i++) {
    for (int a = 0; a < 3; a++) {
      const int v = lattice == NLC_D2Q9 ? nlc::LatD2Q9::c(i, a) : nlc::LatD3Q19::c(i, a);
      if (c) c[3 * i + a] = v;
    }
    if (w) w[i] = lattice == NLC_D2Q9 ? nlc::LatD2Q9::w(i) : nlc::LatD3Q19::w(i);
  }
  return q;
}

const char* nlc_version(void) { return "nlc 0.1 (sm_103a)"; }

}  // extern "C"
