// Internal host/device declarations of the split-operator library.
#pragma once

#include <cstdint>

#include "wavepacket_gpu.h"

namespace wp {

// Flags of one FFT pass over a tile of lines along one axis. The operations run in
// this order: IFFT, potential phase, position sums, FFT, kinetic round trip,
// momentum sums, store.
enum PassFlags : uint32_t {
  F_IFFT = 1u << 0,      // inverse FFT along the pass axis
  F_PHASE = 1u << 1,     // multiply by exp(-i V tau/hbar) (all axes in position space)
  F_OBS_POS = 1u << 2,   // position-space partial sums (after the phase)
  F_FFT = 1u << 3,       // forward FFT along the pass axis
  F_KIN = 1u << 4,       // forward FFT, kinetic factor, inverse FFT (all axes in k space)
  F_OBS_MOM = 1u << 5,   // momentum-space partial sums (after the forward FFT)
  F_NO_STORE = 1u << 6,  // keep the tile (used by the momentum sums)
  F_AUTOCORR = 1u << 7,  // add <psi0|psi> to the position sums
};

// Partial-sum slots per CTA.
enum Quantity : int {
  Q_RHO = 0,       // sum |psi|^2
  Q_X = 1,         // sum x_d |psi|^2, d = 0..2
  Q_XX = 4,        // sum x_d^2 |psi|^2
  Q_V = 7,         // sum V |psi|^2
  Q_AC_RE = 8,     // sum conj(psi0) psi
  Q_AC_IM = 9,
  Q_K = 10,        // sum k_d |psi_hat|^2
  Q_K2 = 13,       // sum |k|^2 |psi_hat|^2
  Q_RHOK = 14,     // sum |psi_hat|^2
  NQ = 16
};

template <class T>
struct alignas(2 * sizeof(T)) cx {
  T re, im;
};

// Stockham stage plan shared by the device FFT and the host table builder: the stage
// starting at span 2^logNs of a 2^logn transform has radix 2^wp_stage_radix_log (8 while
// at least 5 or exactly 3 factors of two remain, then 4, then 2).
__host__ __device__ constexpr int wp_stage_radix_log(int logn, int logNs) {
  return (logn - logNs >= 5 || logn - logNs == 3) ? 3 : (logn - logNs >= 2 ? 2 : 1);
}
// Offset of a stage's entries in the per-stage twiddle table (Ns (R - 1) entries each,
// none for the first stage).
__host__ __device__ constexpr int wp_stage_tw_offset(int logn, int logNs) {
  int off = 0, ls = 0;
  while (ls < logNs) {
    const int lr = wp_stage_radix_log(logn, ls);
    if (ls > 0) off += (1 << ls) * ((1 << lr) - 1);
    ls += lr;
  }
  return off;
}
constexpr int kFixedLogMin = 6, kFixedLogMax = 10;  // fixed-size pass kernels: n = 64..1024
constexpr int kRes1dLogMin = 8, kRes1dLogMax = 14;  // fixed-length resident lines: n = 256..16384
// elements per thread of a fixed-length resident line (1024 threads at most)
__host__ __device__ constexpr int wp_res1d_fixed_ept(int logn) { return logn >= 14 ? 16 : 8; }

// A table factor as one 16-byte record: the value for FP64 and float-float, the high
// and low FP32 parts for the complex64 form.
template <class T>
struct alignas(16) TwE {
  cx<T> w;
};
template <>
struct alignas(16) TwE<float> {
  cx<float> h, l;
};

// A factor value (FP64) as a 16-byte record of precision T.
template <class T>
__host__ __device__ inline TwE<T> make_rec(double re, double im) {
  TwE<T> r;
  r.w = cx<T>{(T)re, (T)im};
  return r;
}
template <>
__host__ __device__ inline TwE<float> make_rec<float>(double re, double im) {
  TwE<float> r;
  const float hr = (float)re, hi = (float)im;
  r.h = cx<float>{hr, hi};
  r.l = cx<float>{(float)(re - (double)hr), (float)(im - (double)hi)};
  return r;
}

// Per-line record of a pass: the product of the other axes' factors (potential phase in
// the contiguous pass, kinetic factor in the kinetic pass) and, for the potential, the
// per-line Gaussian-term phase coefficients f_g tau/hbar prod_{d != axis} G_d.
template <class T>
struct alignas(16) LineRec {
  TwE<T> L;
  T g[WP_MAX_GAUSS];
};

// Per-handle device control block. The time base lives on the device so that a
// captured CUDA graph replays correctly for any step index.
struct Ctrl {
  int64_t step;                  // step index s of the state (t_s = t0 + s dt)
  int64_t nobs;                  // observation records written by the current run
  double t_tab;                  // time of the current potential tables
  double gphase[WP_MAX_GAUSS];   // f_g(t) tau / hbar for the Gaussian terms
  double gcoef[WP_MAX_GAUSS];    // f_g(t)
  int32_t err;                   // first error raised by a kernel (0 = none)
  uint32_t prep_done;            // blocks of the current k_prep launch that have finished
};

// Potential descriptor as the kernels read it (same field meaning as wp_potential).
struct DevPot {
  int32_t nterms;
  int32_t ngauss;
  int32_t gauss_term[WP_MAX_GAUSS];  // indices of the Gaussian terms
  wp_pot_term term[WP_MAX_TERMS];
};

// Geometry shared by the kernels of one problem.
struct Geom {
  int32_t ndim;
  int32_t ln[3];       // log2 of the extents (0 for axes >= ndim)
  double xmin[3], dx[3];
  double kscale[3];    // 2 pi / L
  double mass, hbar, dt, t0;
  double dv;           // cell volume
  // Powers of two at or above the largest |x_i| and |k_i| of each axis. The observable
  // tables of the line sums (Ox, Ok) hold x / oscale_x and k / oscale_k, so that sums
  // formed in FP32 range stay finite in any units (in SI units k^2 |psi_hat|^2 alone
  // exceeds the FP32 range); the FP64 combination multiplies the scale back, exactly.
  double oscale_x[3], oscale_k[3];
  // Scaled FP32 geometry of the complex64 two-stage kernels' per-line observable rows:
  // x_i / oscale_x = xr0 + i dxr, k_j / oscale_k = j kr (j the signed index),
  // k2r = oscale_k^2 / k2s with k2s = the largest oscale_k^2 (powers of two: exact).
  float xr0[3], dxr[3], kr[3], k2r[3];
  double k2s;
};

// Device tables of one axis for precision T.
template <class T>
struct AxisTab {
  cx<T>* W;                   // exp(-2 pi i k/n), k < n (FP64-generated)
  cx<T>* Kfull;               // exp(-i hbar k^2 dt/2m) (axis 0 also carries 1/N)
  cx<T>* Khalf;               // the same for dt/2
  cx<T>* P;                   // exp(-i A(x,t) tau/hbar): additive potential phase
  cx<T>* W_lo;
  void* Wst;                  // per-stage twiddle records (fixed-size kernels), 16 B each
  cx<T>* Kfull_lo;            // low parts: value - (double)high, so that high + low
  cx<T>* Khalf_lo;            // carries the factor to about twice the precision of T
  cx<T>* P_lo;
  TwE<T>* Prec;               // the same factors as 16-byte records (fixed-size kernels)
  TwE<T>* Kfull_rec;
  TwE<T>* Khalf_rec;
  T* G[WP_MAX_GAUSS];         // Gaussian-term factors exp(-((x - c)/w)^2)
  double* A;                  // additive potential A(x,t), FP64
  double* Gd[WP_MAX_GAUSS];   // Gaussian factors, FP64
  cx<T>* Ox;                  // (x_i, x_i^2) in T: line sums of the position moments
  cx<T>* Ok;                  // (k_i, k_i^2) in T: line sums of the momentum moments
  T* AT;                      // A(x,t) rounded to T: line sums of the potential energy
  void* W256;                 // complex64 and float-float, n = 256: records exp(-2 pi i t k1/256) at k1 * 16 + t
  void* W2s;                  // complex64, n = 64 or 128: two-stage twiddle records (wp_pass2s.cuh)
};

template <class T>
struct PassParams {
  cx<T>* in;
  cx<T>* out;
  const cx<T>* psi0;
  Geom g;
  int32_t axis;        // axis the pass transforms
  int32_t logn;        // log2 of its length
  int32_t logC;        // log2 of the lines per tile
  int32_t LS;          // shared-memory row stride in elements (lines are rows' columns)
  int32_t log_inner;   // log2 of the element stride of the axis (0: contiguous)
  int32_t nthreads;    // block size; nthreads * ept >= tile elements
  int32_t ept;         // elements per thread (8 or 16): selects the kernel variant
  uint32_t flags;
  int32_t ngauss;
  int32_t khalf;       // kinetic factor for dt/2 instead of dt
  const cx<T>* W;
  const cx<T>* W_lo;
  const void* Wst;     // per-stage twiddle records of the pass axis
  int32_t fixed;       // use the fixed-size kernel (n = 2^logn, 2048-element tiles)
  int32_t max_radix_log;  // largest butterfly of the run-time-shape kernel (2 or 3)
  int32_t sep;            // the potential has additive (non-Gaussian) terms: apply the P factors
  const cx<T>* K[3];
  const cx<T>* K_lo[3];
  const cx<T>* P[3];
  const cx<T>* P_lo[3];
  const T* G[WP_MAX_GAUSS][3];
  const double* A[3];
  const double* Gd[WP_MAX_GAUSS][3];
  const Ctrl* ctrl;
  double* partials;    // [gridDim.x][NQ]
  const TwE<T>* Prec;      // pass-axis potential-phase records
  const TwE<T>* Krec;      // pass-axis kinetic records
  const cx<T>* Khalf_axes[3];     // dt/2 kinetic factors (batched kinetic pass, KVK ends)
  const cx<T>* Khalf_lo_axes[3];
  const TwE<T>* Krec_half;        // dt/2 records of the pass axis
  const LineRec<T>* lines_kin_half;
  const LineRec<T>* lines_phase;
  const LineRec<T>* lines_kin;
  const cx<T>* Ox;     // pass-axis observable tables (fixed-size kernels)
  const cx<T>* Ok;
  const T* AT;
  const T* ATax[3];    // A(x,t) rounded to T on every axis (two-stage kernels' line rows)
  const TwE<T>* grid_rec;  // static grid potential: phase records of this pass's tau, or NULL
  const double* grid_v;    // static grid potential (observables), or NULL
  const void* W256;        // two-stage 256-point kernels: twiddle records of the pass axis, or NULL
  const void* W2s;         // two-stage 64- and 128-point kernels: twiddle records, or NULL
};

// Per-line records of one pass (k_lines).
template <class T>
struct LinesParams {
  Geom g;
  int32_t axis;            // pass axis; lines run over the other axes
  int32_t gauss;           // also form the Gaussian-term coefficients
  int32_t ngauss;
  int64_t nlines;
  const cx<T>* H[3];
  const cx<T>* Lo[3];
  const double* Gd[WP_MAX_GAUSS][3];
  const Ctrl* ctrl;
  LineRec<T>* out;
};

template <class T>
struct PrepParams {
  Geom g;
  int64_t n[3];
  AxisTab<T> tab[3];
  const DevPot* pot;
  Ctrl* ctrl;
  int32_t step_add;    // added to ctrl->step before the time is formed
  double t_shift;      // added to t0 + step dt (dt/2 for the mid-point order)
  double tau;          // phase length (dt, dt/2 or 0 for observables only)
};

template <class T>
struct Res1dParams {
  cx<T>* psi;
  const cx<T>* psi0;
  Geom g;
  int32_t logn;
  int32_t nthreads;
  int32_t ept;         // elements per thread (8 or 16)
  int32_t order;       // wp_order
  int32_t obs;         // evaluate observables after the chunk
  int32_t autocorr;
  int64_t nsteps;      // steps in this chunk
  const cx<T>* W;
  const cx<T>* W_lo;
  const cx<T>* Kfull;
  const cx<T>* Khalf;
  const cx<T>* Kfull_lo;
  const cx<T>* Khalf_lo;
  const DevPot* pot;
  Ctrl* ctrl;
  double* obs_out;     // [..][16] records; written at ctrl->nobs
  int64_t obs_cap;
  // Potential phase split by time dependence (term masks, bit k = term k):
  // static terms as FP64 tables S[0] (phase length dt) and S[1] (dt/2); linear and
  // constant terms as a plane wave exp(-i (beta x - gamma) tau / hbar) built per step
  // from two short tables; the rest evaluated point by point.
  const TwE<T>* S[2];
  uint32_t static_mask;
  uint32_t plane_mask;
  uint32_t gen_mask;
  const double* vgrid;       // static grid potential (observables; the phase is in S), or NULL
  int32_t fixed;             // compile-time line length (k_res1d_fixed), n = 2^8 .. 2^14
  int32_t max_radix_log;     // largest butterfly of the run-time-length kernel (2 or 3)
  const void* Wst;           // per-stage twiddle records (fixed)
  const TwE<T>* Krec[2];     // kinetic factors dt, dt/2 as records (fixed)
};

// Static phase tables of a 1-D handle (k_static_phase), formed in FP64 and stored as records.
template <class T>
struct StaticPhaseParams {
  Geom g;
  int64_t n;
  const DevPot* pot;
  uint32_t static_mask;
  const double* vgrid; // static grid potential added to V_s, or NULL
  TwE<T>* S[2];        // exp(-i V_s dt / hbar), exp(-i V_s (dt/2) / hbar)
};

// <psi|A|psi> partial sums per block (k_expect_partial) and their fixed-order total.
template <class T>
struct ExpectParams {
  const cx<T>* psi;
  const double* A;
  int64_t n;
  int64_t per_block;   // points per block
  double* partial;     // [gridDim.x]
};

// Phase records of a static grid potential for dt and dt/2 (k_grid_phase).
template <class T>
struct GridPhaseParams {
  const double* V;
  int64_t n;
  double dt, hbar;
  TwE<T>* rec[2];
};

struct ReduceParams {
  const double* pos;   // [npos][NQ], rows pos_stride apart
  int64_t npos;
  const double* mom;   // [nmom][NQ], rows mom_stride apart
  int64_t nmom;
  int64_t pos_stride, mom_stride;
  Geom g;
  int64_t ntotal;      // grid points
  int32_t autocorr;
  Ctrl* ctrl;
  double* obs_out;     // [cap][16]
  int64_t obs_cap;
};

template <class T>
struct ConvParams {
  const void* src;
  void* dst;
  int64_t n;
  int32_t dir;         // 0: complex128 -> state, 1: state -> complex128
};

template <class T>
struct GaussParams {
  cx<T>* psi;
  Geom g;
  double x0[3], p0[3], sigma[3];
  double pref;
  cx<double>* tab;     // per-axis factors, axis d at tab + off[d] (k_gaussian_axes)
  int64_t off[3];
  int64_t nsum;        // sum of the extents
};

// Launchers (defined per precision in the kernel translation units).
template <class T> int launch_pass(const PassParams<T>& p, int64_t ntiles, size_t smem, void* stream);
template <class T> int launch_prep(const PrepParams<T>& p, void* stream);
template <class T> int launch_res1d(const Res1dParams<T>& p, size_t smem, void* stream);
template <class T> int launch_convert(const ConvParams<T>& p, void* stream);
template <class T> int launch_gaussian(const GaussParams<T>& p, int64_t n, void* stream);
template <class T> int launch_lines(const LinesParams<T>& p, void* stream);
// batched launches (one block range per instance)
template <class T> int launch_pass_batch(const PassParams<T>* params, const int64_t* tile_start, const int* block_inst,
                                         int logn, int64_t block_off, int64_t nblocks, uint32_t flags, int khalf,
                                         size_t smem, void* stream);
template <class T> int launch_lines_batch(const LinesParams<T>* params, int ninst, int64_t max_lines,
                                          void* stream);
template <class T> int launch_prep_batch(const PrepParams<T>* params, int ninst, int step_add, double shift_dt,
                                         double tau_dt, void* stream);
template <class T> int launch_res1d_batch(const Res1dParams<T>* params, int ninst, int nthreads, int ept,
                                          int64_t nsteps, size_t smem, void* stream);
// The record's reduction in two launches: launch_reduce_rows sums fixed runs of partial
// rows in place (adjusting p to the remaining rows; a no-op for few rows), launch_reduce
// sums the rest and writes the record.
int launch_reduce_rows(ReduceParams& p, void* stream);
int launch_reduce(const ReduceParams& p, void* stream);
template <class T> int launch_static_phase(const StaticPhaseParams<T>& p, void* stream);
template <class T> int launch_grid_phase(const GridPhaseParams<T>& p, void* stream);
template <class T> int launch_expect(const ExpectParams<T>& p, int nblocks, double dv, double* out, void* stream);
int launch_set_step(Ctrl* ctrl, int64_t step, void* stream);
int launch_add_step(Ctrl* ctrl, int64_t add, void* stream);
template <class T> int pass_smem_limit_set(size_t smem);
// fixed-size pass kernels (their own translation units, wp_fixed_*.cu)
template <class T> int launch_fixed(const PassParams<T>& p, unsigned ntiles, size_t smem, void* stream);
// One launch per batched pass (wp_batch_merged.cuh): class c of the pass covers launch
// blocks start[c] .. start[c + 1] - 1 and block-list entries list_off[c] on; key[c] is its
// line-length class (6..10 fixed-shape, kBatchClassP256 + v two-stage), counted after nprep
// leading blocks that form the per-instance tables (and, with lines, the line records) of
// the next step, with the step increment, time shift and phase length (units of dt) given.
constexpr int kMergedMaxClasses = 8;
struct MergedLaunch {
  int32_t ncls;
  int32_t key[kMergedMaxClasses];
  int64_t start[kMergedMaxClasses + 1];
  int64_t list_off[kMergedMaxClasses];
  int32_t nprep;
  int32_t step_add;
  double shift_dt, tau_dt;
  int32_t lines;
};
template <class T>
int launch_merged_contig(const PassParams<T>* params, const int64_t* tile_start, const int* block_inst,
                         const MergedLaunch& ml, uint32_t flags, int khalf, const PrepParams<T>* pp,
                         const LinesParams<T>* lp, size_t smem, void* stream);
template <class T>
int launch_merged_strided(const PassParams<T>* params, const int64_t* tile_start, const int* block_inst,
                          const MergedLaunch& ml, uint32_t flags, int khalf, const PrepParams<T>* pp,
                          const LinesParams<T>* lp, size_t smem, void* stream);

// two-stage kernels for 256-point lines, complex64 and float-float (wp_pass256_*.cu)
template <class T> bool pass256_applies(const PassParams<T>& p);
template <class T> int launch_pass256(const PassParams<T>& p, void* stream);
template <class T> int64_t pass256_blocks(const PassParams<T>& p);  // blocks (partial rows) of a launch
// complex64 two-stage kernels for 64- and 128-point lines (wp_pass2s_f32.cu), single and
// batched (class keys kBatchClassP2S + 100 (logn - 6) + v, v as for the 256-point class)
constexpr int kBatchClassP2S = 1100;
constexpr size_t kPass2sSmem = 136 * 16 + 16 * 137 * 8;  // the larger of their two shared-memory sizes
bool pass2s_applies(const PassParams<float>& p);
int launch_pass2s(const PassParams<float>& p, void* stream);
int launch_pass2s_batch(const PassParams<float>* params, const int64_t* tile_start, const int* block_inst, int logn,
                        int variant, int64_t block_off, int64_t nblocks, uint32_t flags, int khalf, void* stream);
// their batched form: one launch over a class of blocks (16-line or 16-column tiles).
// Class keys kBatchClassP256 + v in a batch's block lists, v = 2 x (largest Gaussian-term
// count) + (any additive terms) for the contiguous pass, 0 for the strided one; variant
// -1 selects the strided FFT-only kernel.
constexpr int kBatchClassP256 = 1000;
constexpr size_t kPass256Smem = 256 * 16 + 16 * 273 * 8;  // their dynamic shared memory
template <class T>
int launch_pass256_batch(const PassParams<T>* params, const int64_t* tile_start, const int* block_inst, int variant,
                         int64_t block_off, int64_t nblocks, uint32_t flags, int khalf, void* stream);
template <class T> int fixed_smem_limit_set(size_t smem);
// batched pass kernels, contiguous and strided axis (wp_batch_*.cu): one launch per
// line-length class, blocks block_off .. block_off + nblocks - 1 of the class-sorted list
template <class T> int launch_pass_batch_contig(const PassParams<T>* params, const int64_t* tile_start,
                                                const int* block_inst, int logn, int64_t block_off, int64_t nblocks,
                                                uint32_t flags, int khalf, size_t smem, void* stream);
template <class T> int launch_pass_batch_strided(const PassParams<T>* params, const int64_t* tile_start,
                                                 const int* block_inst, int logn, int64_t block_off, int64_t nblocks,
                                                 uint32_t flags, int khalf, size_t smem, void* stream);
template <class T> int launch_fixed_obs(const PassParams<T>& p, unsigned ntiles, size_t smem, void* stream);
template <class T> int fixed_obs_smem_limit_set(size_t smem);
template <class T> int launch_fixed_grid(const PassParams<T>& p, unsigned ntiles, size_t smem, void* stream);
template <class T> int fixed_grid_smem_limit_set(size_t smem);
template <class T> int launch_fixed_grid_obs(const PassParams<T>& p, unsigned ntiles, size_t smem, void* stream);
template <class T> int fixed_grid_obs_smem_limit_set(size_t smem);
template <class T> int res1d_smem_limit_set(size_t smem);
// fixed-length resident-line kernels (their own translation units, wp_res1d_*.cu)
template <class T> int launch_res1d_fixed(const Res1dParams<T>& p, size_t smem, void* stream);
template <class T> int launch_res1d_fixed_batch(const Res1dParams<T>* params, int ninst, int logn, int64_t nsteps,
                                                size_t smem, void* stream);
template <class T> int res1d_fixed_smem_limit_set(size_t smem);

// Handle access for the run-time compiled potentials (wp_jit.cu).
wp_status handle_set_error(wp_handle* h, wp_status st, const char* msg);
void handle_geometry(const wp_handle* h, int* ndim, int64_t n[3], double xmin[3], double dx[3], void** stream);

// Kernel classes for timing and launch counting.
enum KernelClass : int {
  K_PASS_CONTIG = 0,
  K_PASS_STRIDED = 1,
  K_PASS_KIN = 2,
  K_PREP = 3,
  K_RES1D = 4,
  K_REDUCE = 5,
  K_AUX = 6,
  K_LINES = 7,
  K_NCLASSES = 8
};

}  // namespace wp
