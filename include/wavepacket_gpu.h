/*
 * wavepacket_gpu.h -- C ABI of the GB300 (sm_103a) split-operator propagator.
 *
 * The library advances a wave function psi(x, t) on a periodic 1-, 2- or 3-D grid
 * under the time-dependent Schroedinger equation  i hbar dpsi/dt = (P^2/2m + V(x,t)) psi
 * (Dion, Hashemloo, Rahali, arXiv:1306.3247, Sec. 2.1, eqs. (1)-(2)) with the
 * symmetric split-operator step of eq. (splitop), the kinetic factor applied in
 * momentum space through forward/inverse FFTs (eq. (ft)).
 *
 * Conventions used by every call:
 *  - Grid (eq. (grid), Sec. 2.1): x_{d,i} = xmin[d] + i * L[d]/n[d], i = 0..n[d]-1,
 *    periodic with period L[d]. A paper-style closed interval [x_min, x_max] with n
 *    points maps to L = n (x_max - x_min)/(n - 1).
 *  - Layout (Sec. 3.2.4): psi is row-major psi[n0][n1][n2], the last axis fastest.
 *    1-D problems lie along x, 2-D problems in the xy plane (Sec. 2.2).
 *  - Every n[d] is a power of two, 2 <= n[d]; other sizes return WP_EUNSUPPORTED.
 *  - Momentum grid (Sec. 2.1): k_{d,j} = 2 pi j'/L[d], j' = j for j < n/2, j - n otherwise.
 *  - Times: t_s = t0 + s dt for step index s (a product, never a running sum).
 *  - Errors: every call returns a wp_status; nothing aborts (replaces abort() of
 *    Sec. 3.2.6). wp_last_error() gives the handle's last message.
 *  - Streams: all device work of a handle is ordered on the stream given at creation
 *    (NULL = the legacy default stream). Calls that return host data synchronise it.
 *  - Ownership: the library owns every buffer it allocates; caller buffers passed in
 *    are only read or written during the call.
 */
#ifndef WAVEPACKET_GPU_H
#define WAVEPACKET_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  WP_OK = 0,
  WP_EINVAL = 1,        /* bad argument (null pointer, nprint > nt as in Sec. 3.4, ...) */
  WP_EUNSUPPORTED = 2,  /* size not a power of two, ndim outside 1..3, too large a line */
  WP_ENOMEM = 3,        /* device allocation failed */
  WP_ENONFINITE = 4,    /* the norm became NaN or infinite */
  WP_ETIMEOUT = 5,      /* a bounded device wait gave up */
  WP_ECUDA = 6,         /* any other CUDA error; see wp_last_error */
  WP_EBUSY = 7          /* the handle is in use (e.g. a batch slot is occupied) */
} wp_status;

/* Arithmetic form of the propagation.
 *  WP_C128:       complex128 state, FP64 FFT and phases (the plain FP64 method).
 *  WP_C64:        complex64 state and FFT in FP32; twiddles, phase-argument reductions
 *                 modulo 2 pi and all observable reductions in FP64.
 *  WP_C128_F32X2: complex128 accuracy computed in float-float (pairs of FP32, about 48
 *                 significant bits) on the FP32 pipes, which GB300 runs about 58x faster
 *                 than FP64; 16 bytes per point in HBM. States enter and leave as
 *                 complex128. */
typedef enum { WP_C128 = 0, WP_C64 = 1, WP_C128_F32X2 = 2 } wp_precision;

/* Operator order of one step (eq. (splitop)).
 *  WP_ORDER_VKV: e^{-iV(t_{s+1})dt/2hbar} e^{-iK dt/hbar} e^{-iV(t_s)dt/2hbar}
 *                (trapezoid rule for the integral of V).
 *  WP_ORDER_KVK: e^{-iK dt/2hbar} e^{-iV(t_s + dt/2)dt/hbar} e^{-iK dt/2hbar}
 *                (the paper's order, mid-point rule, Algorithm 1).
 * Adjacent half-steps of consecutive steps are merged on the device; the result
 * differs from the unmerged product only by rounding. */
typedef enum { WP_ORDER_VKV = 0, WP_ORDER_KVK = 1 } wp_order;

/* Problem statement: the grid, mass and hbar, and the time step of Tab. 1
 * (units = the value of hbar: 1 for atomic units, 1.054571726e-34 for SI). */
typedef struct {
  int32_t ndim;       /* 1, 2 or 3 */
  int32_t precision;  /* wp_precision */
  int32_t order;      /* wp_order */
  int32_t autocorr;   /* nonzero: keep psi(t0) on the device for |<psi(0)|psi(t)>|^2 */
  int64_t n[3];       /* grid points per axis; axes >= ndim are ignored */
  double xmin[3];     /* first grid point per axis */
  double L[3];        /* period per axis (dx = L/n) */
  double mass, hbar, dt, t0;
} wp_problem;

/* Potential V(x,t) = sum over terms of f(t) * shape(x,t), evaluated on the device
 * every step. It plays the role of the user potential() of Sec. 3.2.3.
 * shape (centre c_d(t) = c0[d] + v[d] t):
 *   WP_SHAPE_CONST   1
 *   WP_SHAPE_QUAD    0.5 * sum_d a[d] (x_d - c_d)^2
 *   WP_SHAPE_LINEAR  sum_d a[d] (x_d - c_d)
 *   WP_SHAPE_GAUSS   exp(-sum_{d: a[d] > 0} (x_d - c_d)^2 / a[d]^2)
 *   WP_SHAPE_MORSE   a[0] (1 - exp(-a[1] (x_k - c_k)))^2 along axis k = (int)a[2]
 * time coefficient: f(t) = A0 + A env(t) sin(omega t + phi), with
 *   WP_ENV_NONE   env = 1
 *   WP_ENV_GAUSS  env = exp(-(t - t0)^2 / tau^2)
 *   WP_ENV_SIN2   env = sin^2(pi t / tau) for t0 <= t <= t0 + tau, else 0 (Sec. 4.1)
 * At most WP_MAX_TERMS terms, of which at most WP_MAX_GAUSS Gaussian shapes. */
enum { WP_SHAPE_CONST = 0, WP_SHAPE_QUAD = 1, WP_SHAPE_LINEAR = 2, WP_SHAPE_GAUSS = 3, WP_SHAPE_MORSE = 4 };
enum { WP_ENV_NONE = 0, WP_ENV_GAUSS = 1, WP_ENV_SIN2 = 2 };
#define WP_MAX_TERMS 8
#define WP_MAX_GAUSS 2

typedef struct {
  int32_t shape, env;
  double a[3], c0[3], v[3];
  double A0, A, omega, phi, t0, tau;
} wp_pot_term;

typedef struct {
  int32_t nterms;
  int32_t reserved;
  wp_pot_term term[WP_MAX_TERMS];
} wp_potential;

/* Observables of Tab. 3 at one time (Sec. 3.4: at t0 and every nprint steps).
 * Expectation values are the plain integrals <psi|A|psi> (not divided by the
 * norm squared): x[d] = <x_d>, x2[d] = <x_d^2> (so the width of Tab. 3 is
 * x2 - x^2), p[d] = <p_d>, energy = ekin + epot = <psi|H|psi>.
 * autocorr = |<psi(t0)|psi(t)>|^2 when enabled, else 0. */
typedef struct {
  double t, norm;
  double x[3], p[3], x2[3];
  double energy, ekin, epot, autocorr;
  int64_t step;
} wp_obs;

typedef struct wp_handle wp_handle;

/* Create a propagator for one problem (Sec. 3.2.1 parameters). Allocates the state,
 * one state-sized scratch buffer for the momentum-space observables, and small tables.
 * stream: a cudaStream_t or NULL. On success *out owns the handle. */
wp_status wp_create(const wp_problem* problem, void* stream, wp_handle** out);

/* The same, with all device memory of the handle (state, scratch, tables, records)
 * taken from mem_pool, a cudaMemPool_t of the current device, by stream-ordered
 * allocations on `stream`; wp_destroy returns it to the pool. A caller that reserves
 * its device memory up front (a pool whose release threshold keeps it) creates and
 * destroys handles without cudaMalloc or cudaFree. mem_pool = NULL is wp_create. The
 * pool must outlive the handle. The paper has no counterpart of this call. Errors as
 * wp_create (WP_ECUDA when the pool cannot serve an allocation). */
wp_status wp_create_pooled(const wp_problem* problem, void* stream, void* mem_pool, wp_handle** out);

/* Set the potential (Sec. 3.2.2-3.2.3). Copied; may be called again between steps. */
wp_status wp_set_potential(wp_handle* h, const wp_potential* pot);

/* A static potential given on the grid: the user potential() of Sec. 3.2.3 evaluated
 * once at every grid point. V holds n[0]*n[1]*n[2] FP64 energies in the state's layout
 * (row-major, last axis fastest), a host pointer (on_device = 0) or a device pointer
 * (on_device = 1); it is copied, and added to the analytic terms at every step and in
 * the potential energy. V = NULL removes the grid. Device memory: 8 bytes per point, plus
 * two 16-byte phase records per point for 2-D and 3-D grids (WP_ENOMEM if that fails).
 * A handle with a grid is run on its own sequence inside a batch (not in the batched
 * 2-D passes). Synchronises the handle's stream. */
wp_status wp_set_potential_grid(wp_handle* h, const double* V, int on_device);

/* The same grid from CUDA C source compiled at run time (NVRTC) for this GPU. src must
 * define
 *     __device__ double wp_user_potential(double x, double y, double z)
 * (unused coordinates are 0); it is evaluated once at every grid point in FP64 and the
 * result installed as by wp_set_potential_grid. A compilation error returns WP_EINVAL
 * with the compiler log in wp_last_error. */
wp_status wp_set_potential_source(wp_handle* h, const char* src);

/* Copy a complex128 row-major psi into the state (Sec. 3.2.4 initialize_wf).
 * on_device = 0: psi is host memory; 1: device memory. The step index is kept. */
wp_status wp_set_state(wp_handle* h, const void* psi, int on_device);

/* Fill the state with the normalised Gaussian packet of Sec. 4.2:
 * (2/pi)^{d/4} prod_d sigma_d^{-1/2} e^{i p0_d (x_d - x0_d)/hbar} e^{-(x_d - x0_d)^2/sigma_d^2}. */
wp_status wp_init_gaussian(wp_handle* h, const double x0[3], const double p0[3], const double sigma[3]);

/* Copy the state out as complex128 row-major (on_device as in wp_set_state). */
wp_status wp_get_state(wp_handle* h, void* dst, int on_device);

/* Advance nsteps >= 0 split-operator steps (eq. (splitop), Algorithm 1 inner loop).
 * Asynchronous on the handle's stream. */
wp_status wp_step(wp_handle* h, int64_t nsteps);

/* CUDA-graph replay of wp_step: the second call with a given nsteps captures that chunk's
 * launches as a graph and every later call replays it (the launches read the step index
 * and the potential from device memory, so a replay advances from the current step).
 * On by default for a handle created with a stream, unavailable on the legacy default
 * stream (WP_EINVAL). Setting the potential, a grid or a schedule, or profiling, drops
 * the captured graphs. This part has no counterpart in the paper. */
wp_status wp_set_graphs(wp_handle* h, int enable);

/* Evaluate the observables of Tab. 3 at the current step (synchronises). */
wp_status wp_observe(wp_handle* h, wp_obs* out);

/* User observables (Sec. 3.2.5: user_observe is called every nprint steps with the time
 * and the wave function).
 * wp_expect_grid: <psi|A|psi> = sum_j A_j |psi_j|^2 dV for a position-space operator given
 * on the grid (FP64, n[0]*n[1]*n[2] values in the state's layout; host pointer when
 * on_device = 0, device pointer when 1), at the current step; FP64 reduction in a fixed
 * order (bitwise reproducible). Allocates a small temporary; synchronises.
 * wp_run_callback: Algorithm 1 with a host function called on every record (the
 * record of the current step first, then one after every nprint steps) with the handle,
 * whose state is the state of the record (read it with wp_get_state, wp_state_ptr or
 * wp_expect_grid; do not step it inside fn); fn returns 0 to continue, nonzero to stop
 * after that record. *nrec receives the records delivered. The records equal wp_run's
 * to rounding. */
wp_status wp_expect_grid(wp_handle* h, const double* A, int on_device, double* out);
typedef int (*wp_record_fn)(wp_handle* h, const wp_obs* rec, void* user);
wp_status wp_run_callback(wp_handle* h, int64_t nt, int64_t nprint, wp_record_fn fn, void* user, int64_t* nrec);

/* Algorithm 1: observables at the current step and after every nprint steps,
 * nt steps in all (all nt run even when nprint does not divide nt, Sec. 3.4).
 * obs: caller-owned host array of at least 1 + nt/nprint records; *nobs gets the count.
 * nprint > nt or nprint <= 0 -> WP_EINVAL. A NaN/Inf norm -> WP_ENONFINITE. */
wp_status wp_run(wp_handle* h, int64_t nt, int64_t nprint, wp_obs* obs, int64_t* nobs);

/* Unnormalised in-place FFT of the state over all axes (eq. (ft)); sign -1 forward,
 * +1 inverse. The step index is unchanged. */
wp_status wp_fft(wp_handle* h, int sign);

/* Borrowed device pointer to the state, valid until wp_destroy. Element type is
 * complex128 (WP_C128), complex64 (WP_C64) or, for WP_C128_F32X2, four floats per
 * point (re_hi, re_lo, im_hi, im_lo), row-major. */
void* wp_state_ptr(wp_handle* h);

/* Current step index s (t_s = t0 + s dt); settable for checkpoint/resume (the setter
 * also updates the device copy, ordered on the handle's stream). */
int64_t wp_get_step_index(const wp_handle* h);
wp_status wp_set_step_index(wp_handle* h, int64_t s);

/* ---------------------------------------------------------------- schedules and autotuning
 * The paper fixes what a step computes (Sec. 2.1), not how the transforms are scheduled;
 * this part has no counterpart there. A schedule selects how the FFT passes are run:
 *   tile_log       log2 of the elements of a multi-dimensional pass tile (lines x points
 *                  held in shared memory): 10, 11 or 12;
 *   ept            minimum elements per thread, 8 or 16 (raised to 16 when a tile or a
 *                  1-D line needs it);
 *   max_radix_log  largest butterfly of the run-time-shape kernels: 2 (radix 4) or 3
 *                  (radix 8);
 *   fixed          1: use the compile-time-shape kernels where the shape allows (passes
 *                  of 64..1024 points with 2048-element tiles; 1-D lines of 256..16384
 *                  points), 0: always the run-time-shape kernels.
 * The default is {11, 8, 3, 1}. Every schedule computes the same step; results differ
 * only by rounding order.
 *
 * wp_set_schedule rebuilds the handle's pass plans (WP_EUNSUPPORTED when the schedule
 * does not fit the grid: too many threads or too much shared memory; the handle keeps its
 * previous schedule). It synchronises the handle's stream and must not be called during
 * stream capture.
 *
 * wp_autotune times every candidate schedule on the handle (`steps` steps each after one
 * warm-up step, CUDA events on the handle's stream), on a device copy of the state that
 * is put back afterwards together with the step index, applies the fastest (the default
 * unless another is more than 2 % faster), and stores it
 * in a process-wide cache keyed by (precision, ndim, extents, order). wp_create applies a
 * cached schedule to every later handle of the same key (batched and served instances
 * included). best_ms is the best time per step; ncandidates counts the schedules timed.
 * Allocates a temporary state copy (WP_ENOMEM if that fails). steps >= 1. */
typedef struct {
  int32_t tile_log;
  int32_t ept;
  int32_t max_radix_log;
  int32_t fixed;
} wp_schedule;

wp_status wp_get_schedule(const wp_handle* h, wp_schedule* out);
wp_status wp_set_schedule(wp_handle* h, const wp_schedule* s);
wp_status wp_autotune(wp_handle* h, int32_t steps, wp_schedule* best, double* best_ms, int32_t* ncandidates);
int64_t wp_autotune_cache_size(void);
void wp_autotune_cache_clear(void);

/* Kernel timing for measurement: while enabled, every launch is bracketed by CUDA
 * events on the handle's stream (CUDA-graph replay is off). wp_profile_read returns
 * the launch count and total milliseconds recorded for one kernel class (names as in
 * wp_kernel_name; index < wp_kernel_count()) and clears it. */
wp_status wp_profile_enable(wp_handle* h, int enable);
wp_status wp_profile_read(wp_handle* h, int kernel, int64_t* launches, double* total_ms);
int wp_kernel_count(void);
const char* wp_kernel_name(int kernel);

/* Launches of the library's kernels issued by this handle since creation. */
int64_t wp_launch_count(const wp_handle* h);

/* Batched instances (many independent propagations, e.g. uneven 1-D and 2-D grids).
 * A batch owns its instances' handles, all on one stream (the given one, or a new
 * non-blocking stream for NULL). wp_batch_add creates an instance (its precision must be
 * the batch's) and returns its index; wp_batch_handle gives the borrowed handle for
 * wp_init_gaussian / wp_set_state / wp_get_state / wp_observe (valid until
 * wp_batch_destroy). wp_batch_step advances every instance by nsteps steps (the chunk
 * semantics of wp_step): 1-D instances run in one resident launch per line length for
 * the whole chunk, 2-D instances whose axes tile into 2048-point tiles share one launch
 * per pass kind per step, others run their own sequence. With use_graph != 0 the chunk
 * is captured once per chunk length as a CUDA graph (on its second use) and replayed.
 * Each instance's result equals what the instance gives alone. */
typedef struct wp_batch wp_batch;
wp_status wp_batch_create(int32_t precision, void* stream, wp_batch** out);
wp_status wp_batch_add(wp_batch* b, const wp_problem* problem, const wp_potential* pot, int64_t* index);
wp_handle* wp_batch_handle(wp_batch* b, int64_t index);
int64_t wp_batch_size(const wp_batch* b);
wp_status wp_batch_step(wp_batch* b, int64_t nsteps, int use_graph);
int64_t wp_batch_launch_count(const wp_batch* b);  /* kernel launches issued (graph replays count 0) */
wp_status wp_batch_destroy(wp_batch* b);
const char* wp_batch_last_error(const wp_batch* b);

/* Serving: a continuous-batching request loop. Requests (a problem, its potential, the
 * Sec. 4.2 Gaussian packet parameters and a step count) queue in arrival order.
 * wp_server_progress (non-blocking) admits queued requests while a stream slot is free
 * and the estimated device bytes of the running requests stay within budget_bytes,
 * issues the next chunk of at most chunk_steps steps for every running request whose
 * previous chunk completed, and writes the ids of requests that finished since the last
 * call to done_ids (up to cap; *ndone gets the count). Each running request owns one of
 * nslots streams, so kernels of different requests overlap on the device; a request's
 * result is the one its handle gives alone. wp_server_fetch copies a finished request's
 * state (complex128, host, may be NULL) and final observables (may be NULL), returns
 * its submit / admit / finish times (seconds, steady clock, may be NULL) and releases
 * it. Errors: WP_EINVAL, WP_ENOMEM (a request above the budget), WP_EBUSY (fetch of an
 * unfinished request), WP_ECUDA; message in wp_server_last_error. */
typedef struct wp_server wp_server;
wp_status wp_server_create(int64_t budget_bytes, int32_t nslots, int64_t chunk_steps, wp_server** out);
wp_status wp_server_submit(wp_server* s, int64_t id, const wp_problem* problem, const wp_potential* pot,
                           const double x0[3], const double p0[3], const double sigma[3], int64_t nt);
wp_status wp_server_progress(wp_server* s, int64_t* done_ids, int64_t cap, int64_t* ndone);
wp_status wp_server_fetch(wp_server* s, int64_t id, void* psi_host, wp_obs* obs, double* times);
int64_t wp_server_pending(const wp_server* s);     /* queued + running + finished, not fetched */
int64_t wp_server_bytes_in_use(const wp_server* s);
int32_t wp_server_running(const wp_server* s);
wp_status wp_server_destroy(wp_server* s);
const char* wp_server_last_error(const wp_server* s);

/* Arithmetic-rate probe. The paper has no counterpart of this call. It measures the
 * fused multiply-add throughput of the current device in TFLOP/s (one FMA = 2 FLOPs):
 * fp64 != 0 for FP64, 0 for FP32, with 8 independent FMA chains per thread in 8 blocks
 * of 256 threads per SM, timed with CUDA events on `stream` (NULL = legacy default)
 * around the second of two launches of about 0.1 s each. The native FP64 form of the
 * split step is bound by the FP64 rate on GB300, so this is the peak its roofline
 * fraction is stated against. Synchronises the stream. Errors: WP_EINVAL (NULL
 * tflops), WP_ECUDA. */
wp_status wp_probe_fma_rate(int32_t fp64, void* stream, double* tflops);

/* Accuracy probe of the complex64 tables' phase factors. The paper has no counterpart of
 * this call. The complex64 form forms exp(-i A tau/hbar) with FP64 only in the reduction
 * of the argument modulo pi/2 and the cosine and sine as float-float pairs (Taylor series
 * on the FP32 pipe). This call evaluates that factor on the current device for n
 * arguments spread evenly over [-amax, amax] and returns in *max_err the largest absolute
 * difference of its cosine or sine (high + low part, summed in FP64) from the FP64
 * sincos of the same argument. Runs on `stream` (NULL = legacy default) and synchronises
 * it. Errors: WP_EINVAL (n < 1, amax not positive and finite, NULL max_err), WP_ECUDA. */
wp_status wp_probe_phase_ff(int64_t n, double amax, void* stream, double* max_err);

/* Allocation-free moments. The paper has no counterpart of this call: it exists for
 * callers that cannot call cudaMalloc (a host application whose device memory is held
 * by its own pool or reserved up front, code in a callback where allocation is not
 * allowed, a loop that cannot take the synchronisation an allocation may cause).
 * Computes, with FP64 sums over the grid of `problem` (cell volume dV = prod dx_d,
 * x_d = xmin_d + i dx_d), the moments of a caller-owned complex128 row-major state
 * psi_dev: norm = sqrt(sum |psi|^2 dV), x[d] = sum x_d |psi|^2 dV and
 * x2[d] = sum x_d^2 |psi|^2 dV, written to the host record *out (other fields 0,
 * t = problem->t0). It allocates nothing: the partial sums go to a fixed 256 KiB device
 * array inside the library, present on every device that loads it until the process
 * exits. Limit: at most 16,777,216 grid points (e.g. 256^3); larger grids return
 * WP_EUNSUPPORTED with a message naming the limit. The first call on a device (with
 * that device current) looks up the array's device address. Every call shares the one
 * array and overwrites it (no slot needs to start at zero), so calls whose kernels
 * overlap on the GPU (different streams or host threads) race: serialise them.
 * Runs on `stream` (NULL = legacy default), copies the record into pageable host memory
 * and synchronises the stream before returning, so it cannot be called on a stream that
 * is being captured into a CUDA graph.
 * Errors: WP_EINVAL (NULL argument, extent < 1), WP_EUNSUPPORTED (too many points),
 * WP_ECUDA (a failed launch, copy or synchronisation); the message of the calling
 * thread's last failure is in wp_moments_noalloc_error(). */
wp_status wp_moments_noalloc(const wp_problem* problem, const void* psi_dev, void* stream, wp_obs* out);
const char* wp_moments_noalloc_error(void);

/* Release everything the handle owns. NULL is accepted. */
wp_status wp_destroy(wp_handle* h);

/* The handle's last error message ("" if none); a static string for NULL. */
const char* wp_last_error(const wp_handle* h);
const char* wp_status_string(wp_status s);

#ifdef __cplusplus
}
#endif

#endif /* WAVEPACKET_GPU_H */
