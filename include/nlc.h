/*
 * nlc.h -- C ABI of libnlc: one GPU time step of the hybrid lattice-Boltzmann
 * (LB) / finite-difference Beris-Edwards method for nematic liquid crystals of
 * Coelho, Araujo & Telo da Gama, "Lattice-Boltzmann simulation of free
 * nematic-isotropic interfaces" (arxiv 1907.13415).
 *
 * The problem statement the calls follow (Sec. 1.1, Sec. 1.2, Sec. 2):
 *   - a periodic lattice (Sec. 2: periodic boundaries in every direction),
 *     D2Q9 (nz = 1) or D3Q19, lattice units (dx = dt = 1);
 *   - parameters A0, K, gamma (Eq. 2), Gamma, xi (Eq. 1), the LB relaxation
 *     time tau (Sec. 1.2.1) and the reference density rho0;
 *   - initial fields Q (the order-parameter tensor of Eq. 1), rho and u
 *     (Sec. 2: rho = 1, u = 0 by default);
 *   - time stepping; read-back of Q, rho, u and of observables (scalar order
 *     parameter profile, interface position, droplet radius, maximum speed).
 *
 * One call of nlc_step(ctx, 1) performs, on the GPU, per lattice cell:
 *   H from Eq. 3, the stress of Eq. 5 (without P0) and its central-difference
 *   divergence F (Sec. 1.2.1), rho and u from Eq. 6, BGK collision with the
 *   source term S_i of Sec. 1.2.1 and streaming, and the predictor-corrector
 *   update of Q by Eq. 1 with central differences (Sec. 1.2.2, steps 1-5),
 *   using the velocity of Eq. 6 held fixed over both evaluations.
 *
 * Conventions shared by every call:
 *   - Every call returns an nlc_status; nothing else crosses the ABI.  On
 *     failure nlc_last_error(ctx) gives a message owned by the context.
 *   - The caller owns every host array passed in or out; the library copies
 *     what it needs before returning.  The context owns all device memory.
 *   - Work is queued on the CUDA stream given to nlc_create (NULL = the legacy
 *     default stream).  nlc_step does not synchronise; nlc_set_fields,
 *     nlc_get_fields, nlc_get_populations and nlc_observables do.
 *   - Host field arrays are float64, structure of arrays, x fastest:
 *       Q5  [5][nz][ny][nx]   components (xx, xy, xz, yy, yz); Qzz = -Qxx-Qyy
 *       rho [nz][ny][nx]
 *       u   [3][nz][ny][nx]   (u_z is zero on D2Q9)
 *   - A context is not thread-safe; use one per host thread.
 */
#ifndef NLC_H
#define NLC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define NLC_API __attribute__((visibility("default")))
#else
#define NLC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NLC_OK = 0,
  NLC_EINVAL = -1,      /* bad argument (sizes, parameters, null pointer)  */
  NLC_ENOMEM = -2,      /* device or host allocation failed                */
  NLC_ECUDA = -3,       /* a CUDA call or kernel launch failed             */
  NLC_EUNSTABLE = -4,   /* non-finite values found in the state            */
  NLC_ETIMEOUT = -5,    /* a bounded device wait ran out                   */
  NLC_ECORRUPT = -6,    /* a saved state failed its checksum               */
  NLC_EUNSUPPORTED = -7 /* valid request this build does not implement     */
} nlc_status;

enum { NLC_D2Q9 = 0, NLC_D3Q19 = 1 };

/* Arithmetic and storage precision of the step.  Observables are always
 * accumulated in FP64. */
enum {
  NLC_FP64 = 0,     /* everything in double                                 */
  NLC_FP32 = 1,     /* populations (as deviations from w_i rho0) and Q stored
                       and computed in float                                */
  NLC_FP32_QF64 = 2 /* populations stored in float (as deviations), Q, u and
                       all arithmetic in double: halves the population
                       traffic of FP64 while Q keeps double precision.
                       nlc_adjoint returns NLC_EUNSUPPORTED.               */
};

/* Kernel schedule of one step.  Both compute the same step. */
enum {
  NLC_SCHED_FUSED = 0,  /* two tiled kernels per step (default)            */
  NLC_SCHED_UNFUSED = 1 /* four one-cell-per-thread kernels per step        */
};

typedef struct {
  int32_t nx, ny, nz; /* lattice extent; nz = 1 for D2Q9                    */
  int32_t lattice;    /* NLC_D2Q9 | NLC_D3Q19                               */
  int32_t precision;  /* NLC_FP64 | NLC_FP32 | NLC_FP32_QF64                */
} nlc_grid;

/* Eq. 2 (A0, K, gamma), Eq. 1 (Gamma, xi), Sec. 1.2.1 (tau), reference
 * density rho0 (Sec. 2 uses rho = 1).  tau must exceed 1/2. */
typedef struct {
  double A0, K, gamma, Gamma, xi, tau, rho0;
} nlc_params;

/* Observables of the current state (all accumulated in FP64).
 *   mass        sum of rho
 *   mom         sum of rho u, with u of Eq. 6
 *   s_area      sum of S / s_ref, S = sqrt(3/2 Tr Q^2), s_ref = 1/3 (the
 *               nematic order at coexistence, Sec. 2.1)
 *   radius      sqrt(s_area/pi) on a single plane, (3 s_area/(4 pi))^(1/3)
 *               in 3D (droplet radius, Sec. 2.2)
 *   x_iface     first x (scanning up from 0) where the y,z-mean of S falls
 *               through s_ref/2, linearly interpolated; -1 if none (flat
 *               interface position, Sec. 2.1)
 *   max_u       largest |u| (spurious-velocity measure, Sec. 2.2)
 *   free_energy Eq. 2 summed over cells, gradient term by forward differences
 *   nonfinite   count of non-finite stored values (populations and Q)
 *   step        time steps taken since the last nlc_set_fields             */
typedef struct {
  double mass, mom[3], s_area, radius, x_iface, max_u, free_energy;
  double u_l2;  /* sqrt(sum over cells of |u|^2) */
  int64_t nonfinite;
  int64_t step;
} nlc_obs;

/* Loss of the droplet problem: L = w_radius (radius - target_radius)^2
 * + w_velocity sqrt(sum_x |u(x)|^2), evaluated on the state after the run
 * (radius and u as in nlc_obs). */
typedef struct {
  double target_radius, w_radius, w_velocity;
} nlc_loss;

/* Result of nlc_adjoint: the loss, its parts, and dL/dgamma, dL/dK,
 * dL/dGamma (FP64 accumulations). */
typedef struct {
  double loss, radius, u_l2;
  double dgamma, dK, dGamma;
} nlc_grad;

/* Result of nlc_autotune. */
typedef struct {
  int32_t chunk;         /* z planes per block chosen for the fused kernels */
  int32_t taper;         /* 1: the chosen chunk list is tapered             */
  int32_t from_cache;    /* 1: taken from the cache file, nothing was timed */
  int32_t candidates;    /* chunk depths timed                              */
  int32_t trial_steps;   /* steps timed per candidate                       */
  double best_ms;        /* time per step of the chosen depth (0 if cached) */
  double default_ms;     /* time per step of the default depth (0 if cached)*/
} nlc_tune;

typedef struct nlc_ctx nlc_ctx;

/* Creates a context for one lattice on the current CUDA device and
 * allocates its device state (two copies of the q populations and of the 5 Q
 * components, plus work arrays).  The state starts at Q = 0, rho = rho0,
 * u = 0.  stream: a cudaStream_t (may be NULL).  *out is set on success.
 * The fused kernels address the populations with 32-bit offsets when every
 * lattice of the context has q nx ny nz < 2^32, else with 64-bit ones; the
 * environment variable NLC_POP_INDEX64=1, read here, forces the 64-bit form
 * (both give the same step bit for bit).
 * Errors: NLC_EINVAL (bad sizes or parameters, D2Q9 with nz != 1),
 * NLC_ENOMEM, NLC_ECUDA. */
NLC_API nlc_status nlc_create(const nlc_grid* grid, const nlc_params* params,
                      void* stream, nlc_ctx** out);

/* Creates one context holding n independent lattices that nlc_step advances
 * together (for example a sweep over gamma, Sec. 2.1's interface velocity
 * against temperature): every kernel launch of a step covers the tiles of
 * all n lattices.  The lattices share the lattice type and precision; their
 * extents and parameters may differ.  grids and params are arrays of n
 * entries (copied).  Instance i (0 <= i < n) is addressed by the inst
 * argument of the calls below.  Errors as nlc_create, and NLC_EINVAL for
 * n < 1 or mixed lattice types or precisions. */
NLC_API nlc_status nlc_create_batch(int32_t n, const nlc_grid* grids,
                                    const nlc_params* params, void* stream,
                                    nlc_ctx** out);

/* Number of lattices in the context (-1 for NULL). */
NLC_API int32_t nlc_count(const nlc_ctx* ctx);

/* steps > 0: nlc_step replays whole chunks of `steps` fused time steps as
 * one captured CUDA graph (captured on first use, on a private stream, and
 * launched on the context's stream); 0 (default) launches kernels directly.
 * Not used while timing is enabled. */
NLC_API nlc_status nlc_set_graph(nlc_ctx* ctx, int32_t steps);

/* steps > 0: nlc_step runs the fused schedule as cooperative launches of
 * one persistent kernel, each advancing every lattice of the context by up
 * to `steps` time steps (the paper has no counterpart; for batched sweeps of
 * many small lattices, where launch gaps dominate).  Its blocks stay
 * resident and take the tiles of the joint tile list one by one, with a
 * grid-wide barrier, bounded by the wait budget (nlc_set_wait_budget),
 * between the lb and Beris-Edwards phases of each step; the results equal
 * the two-kernel form bit for bit.  Combines with nlc_set_graph (a graph
 * then holds the cooperative launches).  0 (default): two kernel launches
 * per step.  The MRT collision and devices without cooperative launch keep
 * the two-kernel form.  Errors: NLC_EINVAL (steps < 0). */
NLC_API nlc_status nlc_set_persistent(nlc_ctx* ctx, int32_t steps);

/* Finite-difference stencils of the context (every lattice).
 * NLC_STENCIL_STANDARD (default): central first derivatives and the
 * 2d+1-point Laplacian (Sec. 1.2.2, second order).  NLC_STENCIL_ISOTROPIC:
 * the lattice's own neighbour set and weights (9 points on D2Q9, 19 on
 * D3Q19), d_a v = 3 sum_i w_i c_ia v(x + c_i) and
 * lap v = 6 sum_i w_i [v(x + c_i) - v(x)], also second order but with a
 * leading error that does not depend on direction -- the remedy Sec. 2.2
 * names for the spurious currents.  Applies to every derivative of the
 * step (grad Q, lap Q, grad u, div Pi) and to the force in the observables;
 * nlc_observables_static keeps the standard stencils.  nlc_adjoint returns
 * NLC_EUNSUPPORTED with the isotropic stencils.  Errors: NLC_EINVAL. */
#define NLC_STENCIL_STANDARD 0
#define NLC_STENCIL_ISOTROPIC 1
NLC_API nlc_status nlc_set_stencil(nlc_ctx* ctx, int32_t kind);

/* Collision operator of lattice inst.  The paper (Sec. 1.2.1) uses a
 * multiple-relaxation-time (MRT) collision but gives neither its moment
 * matrices nor its rates; the default is BGK with the single tau of
 * nlc_params.  With rates != NULL the collision becomes
 *   f* = f - M^-1 S M (f - f^eq + Ft/2) + Ft,   S = diag(rates),
 * with Ft_i = w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F (the source term of
 * Sec. 1.2.1 without its BGK prefactor) and M the orthogonal moment basis
 * obtained by Gram-Schmidt (unit weights) from, in this order,
 *   D2Q9 : 1, c^2, c^4, cx, c^2 cx, cy, c^2 cy, cx^2 - cy^2, cx cy
 *   D3Q19: 1, c^2, c^4, cx, c^2 cx, cy, c^2 cy, cz, c^2 cz, 3cx^2 - c^2,
 *          (3cx^2 - c^2) c^2, cy^2 - cz^2, (cy^2 - cz^2) c^2, cx cy, cy cz,
 *          cx cz, cx (cy^2 - cz^2), cy (cz^2 - cx^2), cz (cx^2 - cy^2).
 * rates: n = q host doubles in that order (copied; the rates of the
 * conserved moments 1, cx, cy, cz have no effect), each in (0, 2); the
 * shear viscosity is (1/s - 1/2)/3 for the rate s of the second-order
 * traceless moments.  With every rate 1/tau this is the BGK step.
 * rates == NULL returns to BGK.  Errors: NLC_EINVAL (instance, n, a rate
 * outside (0, 2)).  nlc_adjoint returns NLC_EUNSUPPORTED while any lattice of
 * the context uses MRT.  Synchronises the stream. */
NLC_API nlc_status nlc_set_mrt(nlc_ctx* ctx, int32_t inst, const double* rates, int32_t n);

/* Replaces the parameters of lattice inst (same checks as nlc_create);
 * the state is kept.  The step kernels (and captured step graphs) read the
 * parameters from device memory, so the change applies to the next step.
 * Synchronises the stream. */
NLC_API nlc_status nlc_set_params(nlc_ctx* ctx, int32_t inst, const nlc_params* params);

/* every > 0: nlc_step checks the state for non-finite values after every
 * `every` steps of each call (one extra pass over the populations and Q, and
 * a stream synchronisation) and stops with NLC_EUNSTABLE, naming the lattice
 * and the step, when it finds any; 0 (default) never checks. */
NLC_API nlc_status nlc_set_check(nlc_ctx* ctx, int32_t every);

/* Budget, in nanoseconds of the GPU's global timer, of every wait at a
 * grid-wide barrier of this context's persistent kernels (the segment
 * kernels of nlc_adjoint; the paper has no counterpart: it is the failure
 * detection of a kernel whose blocks wait on one another).  A wait that runs
 * out makes the kernel record the fault and return, and the call that
 * launched it fails with NLC_ETIMEOUT; the fault is cleared once reported
 * and the context stays usable (its state is that of the last completed
 * call, except for the adjoint's own work arrays).  ns < 0 restores the
 * default, 200 ms; 0 makes any wait that does not find the barrier already
 * complete run out (a test of the path).  Waits on tile copies inside the
 * step kernels keep their own fixed 200 ms bound. */
NLC_API nlc_status nlc_set_wait_budget(nlc_ctx* ctx, int64_t ns);

/* Selects the kernel schedule (NLC_SCHED_*) for later nlc_step calls. */
NLC_API nlc_status nlc_set_schedule(nlc_ctx* ctx, int32_t schedule);

/* Depth of the chunks of the fused schedule.  On D3Q19 each thread block of
 * the two step kernels marches through the z planes of one chunk of one
 * 32 x 8 column of the lattice, and the depth trades the two extra planes
 * every chunk recomputes against the number of blocks the GPU spreads over
 * its SMs.  On D2Q9 each block works through a chunk of 32 x 8 tiles
 * stacked along y, loading the next tile while it computes the current one;
 * the depth counts those tiles.  chunk > 0: chunks of that many planes
 * (tiles), capped at the column's length; chunk = 0: the library's default
 * depth.  taper = 1: chunks of `chunk` until at most 2 chunk of the column
 * remain, then chunks halving down to about 8 planes (tiles); the blocks run
 * chunk by chunk, so the last blocks are short and the last wave over the
 * SMs idles less of the GPU.  Neither changes any result: every chunk list
 * computes the same step bit for bit.  A runtime choice of this library;
 * the paper has no counterpart.  Synchronises the stream.  Errors:
 * NLC_EINVAL (chunk < 0, taper not 0 or 1). */
NLC_API nlc_status nlc_set_chunk(nlc_ctx* ctx, int32_t chunk, int32_t taper);

/* Chunk depth in use for lattice inst, or -1 for a NULL context
 * or an instance out of range; *taper (may be NULL) gets 1 for a tapered
 * chunk list. */
NLC_API int32_t nlc_get_chunk(const nlc_ctx* ctx, int32_t inst, int32_t* taper);

/* Autotuner of the fused schedule (a runtime choice of this library; the
 * paper has no counterpart).  Times trial_steps fused steps of the context's
 * own state for each candidate chunk list (uniform and tapered depths, see
 * nlc_set_chunk) with CUDA events, restores the state bit for bit afterwards
 * (populations and Q of every lattice, buffer parity; the step counters are
 * not touched) and keeps the fastest.  If the environment variable
 * NLC_TUNE_CACHE names a file, results are cached there as a flat JSON
 * object keyed by lattice, precision, extents, collision, stencils and GPU
 * (name, SM count), with the chunk depth as value (negative for a tapered
 * list): a key found there is applied without timing (out->from_cache = 1),
 * a new result is added.  Needs two extra copies of the populations and Q of the whole
 * context in device memory while it runs (freed before it returns).  out may
 * be NULL.  Synchronises the stream.
 * Errors: NLC_EINVAL (trial_steps < 1), NLC_ENOMEM, NLC_ECUDA,
 * NLC_ETIMEOUT. */
NLC_API nlc_status nlc_autotune(nlc_ctx* ctx, int32_t trial_steps, nlc_tune* out);

/* Replaces the state of lattice inst with Q5, rho and u (host float64,
 * layouts above).  The populations are set to the equilibrium
 * f_i^eq(rho, u) of Sec. 1.2.1.  rho may be NULL (rho0 everywhere) and u may
 * be NULL (at rest).  The lattice's step counter restarts at 0.
 * Page-locked (pinned) host arrays are read in place by the device, which
 * overlaps the transfer with the conversion; other host arrays are first
 * copied to a device staging buffer.  Either way the arrays are no longer
 * needed once the call returns.
 * Synchronises the stream.  Errors: NLC_EINVAL (null Q5, inst out of range),
 * NLC_EUNSTABLE (a non-finite input value; the state is then undefined),
 * NLC_ECUDA. */
NLC_API nlc_status nlc_set_fields(nlc_ctx* ctx, int32_t inst, const double* Q5,
                          const double* rho, const double* u);

/* The same with Q given in float32 (same layout, caller-owned; pinned host
 * arrays and device arrays are read in place, pageable host arrays go
 * through a staging copy) and the fluid at rest with rho = rho0, the initial state of
 * Sec. 2 (populations f_i^eq(rho0, 0) = w_i rho0), for contexts whose state
 * is float32 (NLC_FP32): half the host bytes of nlc_set_fields.  The values
 * are stored as given; in a context with float64 Q they are widened
 * exactly.  The lattice's step counter restarts at 0.  Synchronises the
 * stream.  Errors: NLC_EINVAL (null Q5, inst out of range), NLC_EUNSTABLE (a
 * non-finite input value; the state is then undefined), NLC_ECUDA. */
NLC_API nlc_status nlc_set_fields_f32(nlc_ctx* ctx, int32_t inst, const float* Q5);

/* Copies the current Q, rho and u (u of Eq. 6, including F/2) to host
 * arrays; any output may be NULL.  Synchronises the stream. */
NLC_API nlc_status nlc_get_fields(nlc_ctx* ctx, int32_t inst, double* Q5,
                          double* rho, double* u);

/* Copies the pre-collision populations f_i(x, t) of the current time to a
 * host array f[q][nz][ny][nx], in the order nlc_lattice_velocities gives.
 * Synchronises the stream. */
NLC_API nlc_status nlc_get_populations(nlc_ctx* ctx, int32_t inst, double* f);

/* Advances every lattice of the context by n time steps (n >= 0).  Queued
 * on the context's stream; returns launch errors only.  The two kernels of
 * a step are launched with programmatic dependent launch: each may be
 * scheduled while the kernel before it in the stream (the caller's own,
 * too) is finishing, and waits on the device for that kernel to complete
 * before it touches memory, so stream order holds for every buffer. */
NLC_API nlc_status nlc_step(nlc_ctx* ctx, int64_t n);

/* Computes the observables of the current state of instance inst into *out
 * and, if s_profile is not NULL, the y,z-mean of S for each x (nx values).
 * Synchronises the stream. */
NLC_API nlc_status nlc_observables(nlc_ctx* ctx, int32_t inst, nlc_obs* out,
                           double* s_profile);

/* Checkpoint of a context: a header (magic "NLCSTATE", format version,
 * lattice count, a hash of the grids and parameters), then the payload: the
 * per-lattice step counters and, lattice by lattice, the populations and the
 * Q components exactly as stored on the device (bitwise, in the context's
 * precision); the header carries a checksum of the payload (64-bit FNV-1a
 * over 8-byte little-endian words, then the tail bytes).  buf == NULL: *len receives the size needed.  Otherwise
 * *len must be at least that size and receives the bytes written.  The
 * caller owns buf.  Synchronises the stream.  Errors: NLC_EINVAL (small
 * buffer, null len), NLC_ECUDA. */
NLC_API nlc_status nlc_save(nlc_ctx* ctx, void* buf, size_t* len);

/* Restores a checkpoint written by nlc_save into a context of the same
 * lattices (extents, lattice type, precision) and parameters; continuing from it gives the
 * same results, bit for bit, as never having stopped.  Errors: NLC_EINVAL
 * (not a checkpoint, other grid or parameters, short buffer), NLC_ECORRUPT
 * (checksum mismatch; the state is left unchanged), NLC_ECUDA. */
NLC_API nlc_status nlc_load(nlc_ctx* ctx, const void* buf, size_t len);

/* Per-kernel device timing (CUDA events recorded on the context's stream
 * around each kernel launch of nlc_step).  enable = 1 clears the log and
 * starts recording; enable = 0 stops.  Meant for profiling: while enabled,
 * each step records one extra event per kernel. */
NLC_API nlc_status nlc_set_timing(nlc_ctx* ctx, int32_t enable);

/* Totals since timing was enabled, per kernel id (0 .. NLC_N_KERNELS-1):
 * total_ms[k] milliseconds and launches[k] launch counts (arrays of at least
 * max_kernels entries; either may be NULL).  *n_kernels (may be NULL) gets
 * NLC_N_KERNELS.  Synchronises the stream. */
#define NLC_N_KERNELS 8
NLC_API nlc_status nlc_get_timing(nlc_ctx* ctx, int32_t max_kernels,
                                  double* total_ms, int64_t* launches,
                                  int32_t* n_kernels);

/* Name of kernel id k for nlc_get_timing ("?" when out of range). */
NLC_API const char* nlc_timing_name(int32_t k);

/* Gradient of the loss after nsteps time steps with respect to gamma, K,
 * Gamma and the Q field of the current state, by a hand-written adjoint of
 * the time step (the reverse of Sec. 1.2's update, step by step) with
 * checkpointed recomputation: the forward run stores the state every
 * ckpt_every steps, and the backward sweep recomputes each segment from its
 * checkpoint into a ring of ckpt_every states before stepping back through
 * it.  The context must hold one lattice whose populations were set by
 * nlc_set_fields (they do not depend on Q).  On return the context holds
 * the state after the nsteps steps (as nlc_step would leave it), *out the
 * loss and parameter gradients, and dQ0 (host float64 [5][nz][ny][nx], may
 * be NULL) dL/dQ of the starting state.  Device memory: about
 * (nsteps/ckpt_every + ckpt_every + 12) states.  Synchronises the stream.
 * Errors: NLC_EINVAL (nsteps < 1, ckpt_every < 1, batch context, null
 * loss/out), NLC_ENOMEM, NLC_ECUDA, NLC_ETIMEOUT. */
NLC_API nlc_status nlc_adjoint(nlc_ctx* ctx, const nlc_loss* loss, int64_t nsteps,
                               int32_t ckpt_every, nlc_grad* out, double* dQ0);

/* Observables of a state held by the caller in device memory, computed
 * without allocating any device memory.  The paper has no counterpart: this
 * serves callers that may not call cudaMalloc, such as code inside a host
 * application that owns all device memory through its own pool, or
 * monitoring code that must not trigger the device-wide synchronisation of
 * an allocation.  Inputs (device pointers, float64, layouts as the host
 * arrays above): f the pre-collision populations [q][nz][ny][nx] in the
 * order nlc_lattice_velocities gives (as nlc_get_populations returns them),
 * Q5 [5][nz][ny][nx].  *out (host) gets the same values nlc_observables
 * reports for that state (step = 0).  All intermediates live in one fixed
 * block of device memory inside the library (about 17 MB, held by every
 * device that loads the library until the process exits); hence the limits
 * nx*ny*nz <= NLC_STATIC_MAX_CELLS, nx <= NLC_STATIC_MAX_NX and
 * (nx + 8)(ny + 4)(nz + 4) <= 262144 on D3Q19 ((nx + 8)(ny + 4) on D2Q9,
 * nx + 8 rounded up to a multiple of 4); larger lattices get NLC_EINVAL.
 * The first call on a device looks up that block's device address.  Queued
 * on stream, and ends by copying the totals to the host and synchronising
 * the stream: it cannot run inside a stream capture, and a capturing stream
 * gets NLC_EINVAL.  A launch error left pending by earlier work of the
 * calling thread is cleared on entry.  Calls share the block: calls that
 * overlap on the GPU race. */
#define NLC_STATIC_MAX_CELLS 65536
#define NLC_STATIC_MAX_NX 4096
NLC_API nlc_status nlc_observables_static(const nlc_grid* grid, const nlc_params* params,
                                          const double* f, const double* Q5, void* stream,
                                          nlc_obs* out);

/* Message of the last failed call on ctx (empty if none).  Owned by ctx. */
NLC_API const char* nlc_last_error(const nlc_ctx* ctx);

/* Frees the context and its device memory.  NULL is allowed. */
NLC_API void nlc_destroy(nlc_ctx* ctx);

/* Velocity set of a lattice: writes q vectors c[i][3] and weights w[i] (both
 * may be NULL) and returns q (9 or 19), or -1 for an unknown lattice. */
NLC_API int32_t nlc_lattice_velocities(int32_t lattice, int32_t* c, double* w);

/* Library version string. */
NLC_API const char* nlc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NLC_H */
