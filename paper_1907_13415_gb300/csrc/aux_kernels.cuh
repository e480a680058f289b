// aux_kernels.cuh -- state set-up, read-back and FP64 observables.
#pragma once
#include "common.cuh"
#include "lattice.cuh"
#include "physics.cuh"
#include "step_unfused.cuh"

namespace nlc {

// Q from float64 (or, QIn = float, float32) input; populations to the
// pull-layout image of f^eq(rho, u): the deviation stored at y for
// direction i is g^eq_i evaluated at y + c_i, so that pulling reproduces
// f^eq at every cell.  Counts non-finite inputs.
template <class Lat, class T, class G, class QIn = double>
__global__ void __launch_bounds__(256) k_set_fields(
    const QIn* __restrict__ q_in, const double* __restrict__ rho_in,
    const double* __restrict__ u_in, Field<T> Q, G* __restrict__ g,
    Dims d, double rho0, unsigned long long* __restrict__ bad) {
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!decode(d, idx, x, y, z)) return;
  int nbad = 0;
  T qv[5];
#pragma unroll
  for (int k = 0; k < 5; k++) {
    const QIn v = q_in[k * d.n + idx];
    nbad += !isfinite(v);
    qv[k] = (T)v;
  }
  store_with_images<T, 5, Lat::DIM>(Q, d, x, y, z, qv);
  if (rho_in) nbad += !isfinite(rho_in[idx]) || !(rho_in[idx] > 0.0);
  if (u_in)
    for (int a = 0; a < 3; a++) nbad += !isfinite(u_in[a * d.n + idx]);
  if (!rho_in && !u_in) {
    // rho = rho0 and u = 0 everywhere: every deviation is exactly zero
#pragma unroll
    for (int i = 0; i < Lat::Q; i++) g[(int64_t)i * d.n + idx] = G(0);
    if (nbad) atomicAdd(bad, (unsigned long long)nbad);
    return;
  }
#pragma unroll
  for (int i = 0; i < Lat::Q; i++) {
    const int xs = wrap_add(x, Lat::c(i, 0), d.nx);
    const int ys = wrap_add(y, Lat::c(i, 1), d.ny);
    const int zs = Lat::DIM == 3 ? wrap_add(z, Lat::c(i, 2), d.nz) : z;
    const int64_t src = cell_of(d, xs, ys, zs);
    const double rho = rho_in ? rho_in[src] : rho0;
    double u[3] = {0.0, 0.0, 0.0};
    if (u_in)
      for (int a = 0; a < Lat::DIM; a++) u[a] = u_in[a * d.n + src];
    double cu = 0.0, uu = 0.0;
    for (int a = 0; a < Lat::DIM; a++) {
      cu += Lat::c(i, a) * u[a];
      uu += u[a] * u[a];
    }
    const double w = Lat::w(i);
    const double geq = w * ((rho - rho0) + rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
    g[(int64_t)i * d.n + idx] = (G)geq;
  }
  if (nbad) atomicAdd(bad, (unsigned long long)nbad);
}

// rho and u of Eq. 6 (with F/2) at the current time, into float64 arrays
template <class Lat, class T, class G>
__global__ void __launch_bounds__(256) k_moments_out(
    const G* __restrict__ gin, const T* __restrict__ Pi, Dims d, Par<T> p,
    double* __restrict__ rho_out, double* __restrict__ u_out, bool iso) {
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!decode(d, idx, x, y, z)) return;
  T F[3], g[Lat::Q], rho, u[3];
  if (iso)
    force_at_iso<Lat, T>(Pi, d, x, y, z, F);
  else
    force_at<T, Lat::DIM>(Pi, d, x, y, z, F);
  pull<Lat, T>(gin, d, x, y, z, g);
  moments<Lat, T>(g, F, p, rho, u);
  rho_out[idx] = (double)rho;
#pragma unroll
  for (int a = 0; a < 3; a++) u_out[a * d.n + idx] = (double)u[a];
}

// pre-collision populations f_i = w_i rho0 + g*_i(x - c_i) as float64
template <class Lat, class T, class G>
__global__ void __launch_bounds__(256) k_populations_out(
    const G* __restrict__ gin, Dims d, double rho0, double* __restrict__ f) {
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!decode(d, idx, x, y, z)) return;
  T g[Lat::Q];
  pull<Lat, T>(gin, d, x, y, z, g);
#pragma unroll
  for (int i = 0; i < Lat::Q; i++)
    f[(int64_t)i * d.n + idx] = Lat::w(i) * rho0 + (double)g[i];
}

// interior of a padded NC-component field into a dense float64 array
template <class T>
__global__ void __launch_bounds__(256) k_field_out(Field<T> F, int nc, Dims d,
                                                   double* __restrict__ out) {
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!decode(d, idx, x, y, z)) return;
  for (int k = 0; k < nc; k++) out[k * d.n + idx] = (double)F.at(k, x, y, z);
}

// counts non-finite populations and Q components
template <class Lat, class T, class G>
__global__ void __launch_bounds__(256) k_count_nonfinite(const G* __restrict__ g, Field<T> Q,
                                                         Dims d,
                                                         unsigned long long* __restrict__ bad) {
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!decode(d, idx, x, y, z)) return;
  int nbad = 0;
#pragma unroll
  for (int i = 0; i < Lat::Q; i++) nbad += !isfinite((double)g[(int64_t)i * d.n + idx]);
#pragma unroll
  for (int k = 0; k < 5; k++) nbad += !isfinite((double)Q.at(k, x, y, z));
  if (nbad) atomicAdd(bad, (unsigned long long)nbad);
}

// interior of a padded 5-component field to a dense array of the same type
// (checkpoints: bit-exact)
template <class T>
__global__ void __launch_bounds__(256) k_field_raw_out(Field<T> F, int nc, Dims d,
                                                       T* __restrict__ out) {
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!decode(d, idx, x, y, z)) return;
  for (int k = 0; k < nc; k++) out[k * d.n + idx] = F.at(k, x, y, z);
}

// dense 5-component array into a padded field, with periodic images
template <class T, int DIM>
__global__ void __launch_bounds__(256) k_field_raw_in(const T* __restrict__ in, Dims d,
                                                      Field<T> F) {
  int x, y, z;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!decode(d, idx, x, y, z)) return;
  T v[5];
  for (int k = 0; k < 5; k++) v[k] = in[k * d.n + idx];
  store_with_images<T, 5, DIM>(F, d, x, y, z, v);
}

// Observables, pass 1: per-block FP64 partial sums over cells.
// partial[block][OBS_SLOTS]: mass, mom x/y/z, sum S/s_ref, free energy,
// non-finite count, sum |u|^2, max |u| (last).
constexpr int OBS_SLOTS = 9;

// Running sum of float32 terms as the unevaluated pair hi + lo: every
// addition is made exact by Knuth's TwoSum, its rounding error collected in
// lo, so a thread's sum over its cells keeps roughly twice the float32
// precision at float32 speed (GB300 runs float64 arithmetic at a small fraction of its
// float32 rate); the pair is read out in float64 for the block and grid
// sums.
struct AccFF {
  float hi = 0.0f, lo = 0.0f;
  __host__ __device__ __forceinline__ void add(float v) {
    const float s = hi + v;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (v - bp);
    hi = s;
    lo += err;
  }
  // a b, exactly: the fused multiply-add gives the product's rounding error
  __host__ __device__ __forceinline__ void add_prod(float a, float b) {
    const float pr = a * b;
    const float e = fmaf(a, b, -pr);
    add(pr);
    lo += e;
  }
  __host__ __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// plain float64 running sum (float64 state)
struct AccD {
  double v = 0.0;
  __host__ __device__ __forceinline__ void add(double x) { v += x; }
  __host__ __device__ __forceinline__ void add_prod(double a, double b) { v += a * b; }
  __host__ __device__ __forceinline__ double value() const { return v; }
};

template <class T>
struct AccFor {
  using type = AccD;
};
template <>
struct AccFor<float> {
  using type = AccFF;
};

// One cell's contributions to the observables: rho and u (of Eq. 6), the
// cell's Q, and nbad non-finite stored values found by the caller.
// Per-cell terms in the arithmetic type T of the state (float for the FP32
// engine, whose state carries no more digits); acc (AccFor<T>: float-float
// for float, float64 for double) and umax collect them.
template <class T>
struct ObsConst {
  T c2, c3, c4, kh, inv_sref;
  __device__ ObsConst(const Par<T>& p, double s_ref) {
    c2 = p.A0 / T(2) * (T(1) - p.gamma / T(3));
    c3 = p.A0 * p.gamma / T(3);
    c4 = p.A0 * p.gamma / T(4);
    kh = p.K / T(2);
    inv_sref = T(1.0 / s_ref);
  }
};

// The flow terms of one cell from rho and u of Eq. 6: mass (acc[0]),
// momentum (acc[1..3]), |u|^2 (acc[7]) and the maximum of |u|.
template <class T, class A>
__device__ __forceinline__ void obs_u_terms(T r, const T u[3], A acc[OBS_SLOTS - 1], T& umax) {
  T uu = T(0);
  acc[0].add(r);
#pragma unroll
  for (int a = 0; a < 3; a++) {
    acc[1 + a].add_prod(r, u[a]);
    uu += u[a] * u[a];
  }
  umax = fmax(umax, sqrt(uu));
  acc[7].add(uu);
}

// The Q terms of one cell: S/s_ref (acc[4]), the free energy of Eq. 2 with
// its forward-difference gradient term (acc[5]) and the non-finite count.
// qc: component 0 of the cell, component k at qc[k cs]; st[g]: offset of
// the forward neighbour along axis g (DIM axes).
template <int DIM, class T, class A>
__device__ __forceinline__ void obs_q_terms(const T* qc, int64_t cs, const int64_t st[3],
                                            const ObsConst<T>& c, A acc[OBS_SLOTS - 1],
                                            int& nbad) {
  T q[5];
#pragma unroll
  for (int k = 0; k < 5; k++) {
    q[k] = qc[k * cs];
    nbad += !isfinite(q[k]);
  }
  const T qzz = -q[0] - q[3];
  const T tr2 = q[0] * q[0] + q[3] * q[3] + qzz * qzz +
                T(2) * (q[1] * q[1] + q[2] * q[2] + q[4] * q[4]);
  // Tr Q^3 = 3 det Q for traceless Q (Cayley-Hamilton)
  const T tr3 = T(3) * (q[0] * (q[3] * qzz - q[4] * q[4]) - q[1] * (q[1] * qzz - q[4] * q[2]) +
                        q[2] * (q[1] * q[4] - q[3] * q[2]));
  T en = c.c2 * tr2 - c.c3 * tr3 + c.c4 * tr2 * tr2;
  // forward-difference gradient energy K/2 sum_g |Q(x+e_g) - Q(x)|^2
#pragma unroll
  for (int g = 0; g < DIM; g++) {
    const T* qn = qc + st[g];
    T dv[5];
#pragma unroll
    for (int k = 0; k < 5; k++) dv[k] = qn[k * cs] - q[k];
    const T dzz = -dv[0] - dv[3];
    en += c.kh * (dv[0] * dv[0] + dv[3] * dv[3] + dzz * dzz +
                  T(2) * (dv[1] * dv[1] + dv[2] * dv[2] + dv[4] * dv[4]));
  }
  acc[4].add(sqrt(T(1.5) * tr2) * c.inv_sref);
  acc[5].add(en);
}

// (The non-finite count is kept as an integer and the maximum of |u| in T,
// where both are exact; GB300 runs float64 arithmetic at a small fraction of
// its float32 rate.)
template <int DIM, class T, class A>
__device__ __forceinline__ void obs_cell(const Field<T>& Q, const Dims& d, int x, int y, int z,
                                         T r, const T u[3], int& nbad,
                                         const ObsConst<T>& c, A acc[OBS_SLOTS - 1],
                                         T& umax) {
  obs_u_terms(r, u, acc, umax);
  // Q is stored padded with its periodic images (common.cuh), so the
  // forward neighbours are plain offsets from the cell
  const int64_t st[3] = {1, Q.L.nxp, Q.L.plane};
  obs_q_terms<DIM>(Q.base + Q.off(0, x, y, z), Q.L.comp, st, c, acc, nbad);
}

// per-block float64 partials of the accumulators into partial[block]
// (slot 6, the non-finite count, from the integer count nbad)
template <class T, class A>
__device__ __forceinline__ void obs_block_out(const A acc[OBS_SLOTS - 1], int nbad, T umax,
                                              double* sh, double* __restrict__ partial) {
  double tot[OBS_SLOTS];
  for (int k = 0; k < OBS_SLOTS - 1; k++)
    tot[k] = block_sum(k == 6 ? (double)nbad : acc[k].value(), sh);
  tot[OBS_SLOTS - 1] = block_max((double)umax, sh);
  if (threadIdx.x == 0)
    for (int k = 0; k < OBS_SLOTS; k++) partial[blockIdx.x * OBS_SLOTS + k] = tot[k];
}

// Observables, pass 1, from rho and u given as float64 arrays: per-block
// float64 partial sums over cells.  partial[block][OBS_SLOTS]: mass,
// mom x/y/z, sum S/s_ref, free energy, non-finite count, sum |u|^2,
// max |u| (last).
template <class Lat, class T, class G>
__global__ void __launch_bounds__(256) k_obs_partial(
    Field<T> Q, const G* __restrict__ gpost,
    const double* __restrict__ rho, const double* __restrict__ u, Dims d,
    Par<T> p, double s_ref, double* __restrict__ partial) {
  __shared__ double sh[32];
  typename AccFor<T>::type acc[OBS_SLOTS - 1];
  T umax = T(0);
  int nbad = 0;
  const ObsConst<T> c(p, s_ref);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < d.n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z;
    decode(d, idx, x, y, z);
#pragma unroll
    for (int i = 0; i < Lat::Q; i++) nbad += !isfinite((T)gpost[(int64_t)i * d.n + idx]);
    const T uc[3] = {(T)u[idx], (T)u[d.n + idx], (T)u[2 * d.n + idx]};
    obs_cell<Lat::DIM>(Q, d, x, y, z, (T)rho[idx], uc, nbad, c, acc, umax);
  }
  obs_block_out<T>(acc, nbad, umax, sh, partial);
}

// The same from the state itself: rho and u of Eq. 6 are formed per cell
// from the pulled populations and the force of the stress Pi (k_stress);
// every stored population is pulled by exactly one cell, so the non-finite
// count covers each once.
template <class Lat, class T, class G>
__global__ void __launch_bounds__(256) k_obs_state(
    Field<T> Q, const G* __restrict__ gin, const T* __restrict__ Pi, Dims d, Par<T> p,
    double s_ref, bool iso, double* __restrict__ partial) {
  __shared__ double sh[32];
  typename AccFor<T>::type acc[OBS_SLOTS - 1];
  T umax = T(0);
  int nbad = 0;
  const ObsConst<T> c(p, s_ref);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < d.n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z;
    decode(d, idx, x, y, z);
    T F[3], g[Lat::Q], rho, u[3];
    if (iso)
      force_at_iso<Lat, T>(Pi, d, x, y, z, F);
    else
      force_at<T, Lat::DIM>(Pi, d, x, y, z, F);
    pull<Lat, T>(gin, d, x, y, z, g);
#pragma unroll
    for (int i = 0; i < Lat::Q; i++) nbad += !isfinite(g[i]);
    moments<Lat, T>(g, F, p, rho, u);
    obs_cell<Lat::DIM>(Q, d, x, y, z, rho, u, nbad, c, acc, umax);
  }
  obs_block_out<T>(acc, nbad, umax, sh, partial);
}

namespace {  // non-template kernels: one private copy per translation unit

// pass 2: block k (launch OBS_SLOTS blocks) sums slot k of the partials in a
// fixed order
__global__ void __launch_bounds__(256) k_obs_final(const double* __restrict__ partial,
                                                   int nblocks,
                                                   double* __restrict__ out) {
  __shared__ double sh[32];
  const int k = blockIdx.x;
  double v = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    const double pv = partial[b * OBS_SLOTS + k];
    v = (k == OBS_SLOTS - 1) ? fmax(v, pv) : v + pv;
  }
  const double t = (k == OBS_SLOTS - 1) ? block_max(v, sh) : block_sum(v, sh);
  if (threadIdx.x == 0) out[k] = t;
}

}  // namespace

// y,z-mean of S per x: partial sums over row chunks, then a fixed-order sum
template <class T>
__global__ void __launch_bounds__(128) k_profile_partial(
    Field<T> Q, Dims d, int rows_per_chunk,
    double* __restrict__ partial) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int chunk = blockIdx.y;
  if (x >= d.nx) return;
  const int64_t rows = (int64_t)d.ny * d.nz;
  const int64_t r0 = (int64_t)chunk * rows_per_chunk;
  const int64_t r1 = r0 + rows_per_chunk < rows ? r0 + rows_per_chunk : rows;
  // S per cell in the state's type T, summed in float64
  double s = 0.0;
  for (int64_t r = r0; r < r1; r++) {
    const int yy = (int)((unsigned)r % (unsigned)d.ny), zz = (int)((unsigned)r / (unsigned)d.ny);
    T q[5];
    for (int k = 0; k < 5; k++) q[k] = Q.at(k, x, yy, zz);
    const T qzz = -q[0] - q[3];
    const T tr2 = q[0] * q[0] + q[3] * q[3] + qzz * qzz +
                  T(2) * (q[1] * q[1] + q[2] * q[2] + q[4] * q[4]);
    s += (double)sqrt(T(1.5) * tr2);
  }
  partial[(int64_t)chunk * d.nx + x] = s;
}

namespace {
// block x (launch nx blocks of 256 threads) sums the chunk partials of
// column x in a fixed order
__global__ void __launch_bounds__(256) k_profile_final(
    const double* __restrict__ partial, int nchunks, Dims d,
    double* __restrict__ out) {
  __shared__ double sh[32];
  const int x = blockIdx.x;
  double s = 0.0;
  for (int c = threadIdx.x; c < nchunks; c += blockDim.x) s += partial[(int64_t)c * d.nx + x];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[x] = s / ((double)d.ny * (double)d.nz);
}
}  // namespace

}  // namespace nlc
