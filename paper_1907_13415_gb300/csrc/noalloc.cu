// noalloc.cu -- nlc_observables_static: the observables of a state that the
// caller holds in device memory, computed without allocating any device
// memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a host
// application which owns all device memory through its own pool and forbids
// raw allocations (a solver framework, a serving process with a fixed memory
// budget), or monitoring code that runs between time steps where the implicit
// device-wide synchronisation of cudaMalloc/cudaFree would stall other work.
// For them this entry point keeps every intermediate (the padded copy of Q,
// the stress, rho and u, the reduction partials and the S profile) in
// file-scope __device__ arrays of fixed size, which every GPU that loads the
// library holds until the process exits.  The first call on a device looks
// up the arrays' device addresses with cudaGetSymbolAddress.  Every call
// ends by copying the totals to the host and synchronising the stream, so
// the entry point cannot run inside a stream capture; it refuses a
// capturing stream with NLC_EINVAL.  Every call shares the arrays: two
// calls whose work overlaps on the GPU (different streams or threads) race
// and give undefined results.  Nothing here needs clearing between calls:
// each call overwrites every scratch value it later reads.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "../../include/nlc.h"
#include "aux_kernels.cuh"
#include "common.cuh"
#include "lattice.cuh"
#include "obs_finish.h"
#include "physics.cuh"
#include "step_unfused.cuh"

namespace nlc {
namespace {

// capacity of the static scratch (float64 elements)
constexpr int64_t kMaxCells = NLC_STATIC_MAX_CELLS;
constexpr int kMaxNx = NLC_STATIC_MAX_NX;
constexpr int64_t kMaxPadded = 262144;          // nxp * nyp * nzp of one component
constexpr int kObsBlocks = 256;                 // reduction blocks
constexpr int64_t kProfile = kMaxCells / 64 + 2 * kMaxNx;

constexpr int64_t kOffQ = 0;                              // padded Q, 5 components
constexpr int64_t kOffPi = kOffQ + 5 * kMaxPadded;        // stress, up to 9 planes
constexpr int64_t kOffRho = kOffPi + 9 * kMaxCells;       // rho, then u (3 planes)
constexpr int64_t kOffPart = kOffRho + 4 * kMaxCells;     // reduction partials + total
constexpr int64_t kOffProfP = kOffPart + (kObsBlocks + 1) * OBS_SLOTS;
constexpr int64_t kOffProf = kOffProfP + kProfile;
constexpr int64_t kTotal = kOffProf + kMaxNx;

static __device__ __align__(256) double g_scratch[kTotal];

// device address of g_scratch per device (host-side table)
double* g_scratch_ptr[64] = {nullptr};

// rho and u (Eq. 6, with F/2) from pre-collision populations f (float64)
template <class Lat>
__global__ void __launch_bounds__(256) k_moments_pre(const double* __restrict__ f,
                                                     const double* __restrict__ Pi, Dims d,
                                                     Par<double> p, double* __restrict__ rho,
                                                     double* __restrict__ u) {
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!decode(d, idx, x, y, z)) return;
  double F[3], g[Lat::Q], r, uu[3];
  force_at<double, Lat::DIM>(Pi, d, x, y, z, F);
#pragma unroll
  for (int i = 0; i < Lat::Q; i++) g[i] = f[(int64_t)i * d.n + idx] - Lat::w(i) * p.rho0;
  moments<Lat, double>(g, F, p, r, uu);
  rho[idx] = r;
#pragma unroll
  for (int a = 0; a < 3; a++) u[a * d.n + idx] = uu[a];
}

template <class Lat>
nlc_status run(const Dims& d, const Par<double>& p, const double* f, const double* Q5,
               cudaStream_t st, double* scratch, nlc_obs* out) {
  constexpr int DIM = Lat::DIM;
  const int64_t n = d.n;
  const Layout L = make_layout(d, DIM == 3);
  Field<double> Qf{scratch + kOffQ, L};
  double* Pi = scratch + kOffPi;
  double* rho = scratch + kOffRho;
  double* u = rho + n;
  double* part = scratch + kOffPart;
  double* profp = scratch + kOffProfP;
  double* prof = scratch + kOffProf;
  const unsigned gb = (unsigned)((n + 255) / 256);
  k_field_raw_in<double, DIM><<<gb, 256, 0, st>>>(Q5, d, Qf);
  k_stress<Lat, double><<<gb, 256, 0, st>>>(Qf, Pi, d, p, false);
  k_moments_pre<Lat><<<gb, 256, 0, st>>>(f, Pi, d, p, rho, u);
  const int blocks = (int)(gb < (unsigned)kObsBlocks ? gb : (unsigned)kObsBlocks);
  const double s_ref = 1.0 / 3.0;
  k_obs_partial<Lat, double><<<blocks, 256, 0, st>>>(Qf, f, rho, u, d, p, s_ref, part);
  k_obs_final<<<OBS_SLOTS, 256, 0, st>>>(part, blocks, part + blocks * OBS_SLOTS);
  const int64_t rows = (int64_t)d.ny * d.nz;
  const int rows_per_chunk = 64;
  const int nchunks = (int)((rows + rows_per_chunk - 1) / rows_per_chunk);
  k_profile_partial<double><<<dim3((d.nx + 127) / 128, nchunks), 128, 0, st>>>(
      Qf, d, rows_per_chunk, profp);
  k_profile_final<<<d.nx, 256, 0, st>>>(profp, nchunks, d, prof);
  if (cudaGetLastError() != cudaSuccess) return NLC_ECUDA;
  double tot[OBS_SLOTS];
  double hprof[kMaxNx];
  if (cudaMemcpyAsync(tot, part + blocks * OBS_SLOTS, sizeof(tot), cudaMemcpyDeviceToHost,
                      st) != cudaSuccess ||
      cudaMemcpyAsync(hprof, prof, sizeof(double) * d.nx, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return NLC_ECUDA;
  obs_from_totals(tot, hprof, d.nx, DIM == 2 || d.nz == 1, s_ref, out);
  out->step = 0;
  return NLC_OK;
}

}  // namespace
}  // namespace nlc

extern "C" NLC_API nlc_status nlc_observables_static(const nlc_grid* grid,
                                                     const nlc_params* params,
                                                     const double* f, const double* Q5,
                                                     void* stream, nlc_obs* out) {
  using namespace nlc;
  if (!grid || !params || !f || !Q5 || !out) return NLC_EINVAL;
  if (grid->lattice != NLC_D2Q9 && grid->lattice != NLC_D3Q19) return NLC_EINVAL;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return NLC_EINVAL;
  if (grid->lattice == NLC_D2Q9 && grid->nz != 1) return NLC_EINVAL;
  if (!(params->tau > 0.5) || !(params->rho0 > 0.0)) return NLC_EINVAL;
  Dims d{grid->nx, grid->ny, grid->nz, (int64_t)grid->nx * grid->ny * grid->nz};
  const Layout L = make_layout(d, grid->lattice == NLC_D3Q19);
  // sizes beyond the fixed scratch are refused (no fallback allocation)
  if (d.n > kMaxCells || d.nx > kMaxNx || L.comp > kMaxPadded) return NLC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // the call ends with a copy to the host and a stream synchronisation,
  // which a stream capture cannot hold
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return NLC_ECUDA;
  if (cap != cudaStreamCaptureStatusNone) return NLC_EINVAL;
  // a launch error left pending by earlier work of the calling thread is
  // cleared here, so that it is not reported as this call's failure
  (void)cudaGetLastError();
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return NLC_ECUDA;
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return NLC_ECUDA;
    }
    g_scratch_ptr[dev] = (double*)p;
  }
  Par<double> p;
  p.A0 = params->A0;
  p.K = params->K;
  p.gamma = params->gamma;
  p.Gamma = params->Gamma;
  p.xi = params->xi;
  p.tau = params->tau;
  p.rho0 = params->rho0;
  derive(p);
  return grid->lattice == NLC_D2Q9
             ? run<LatD2Q9>(d, p, f, Q5, st, g_scratch_ptr[dev], out)
             : run<LatD3Q19>(d, p, f, Q5, st, g_scratch_ptr[dev], out);
}
