// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the C ABI (include/lbm.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lbm.h"

namespace lbm_gb300 {

constexpr int Q = 19;
constexpr int MAX_SPECIES = 4;
// partial slots per diagnostics quantity (k_diag)
constexpr int DIAG_SPREAD = 64;
// quantities of the per-CTA diagnostics partials of the stream/collide
// kernel: MAX_SPECIES mass deviations, momentum x, y, z, charge, count of
// non-finite or non-positive densities
constexpr int DIAG_NQ = MAX_SPECIES + 5;

// Potential psi is held on the device as a signed 64-bit fixed-point number
// with 52 fractional bits: psi = k * 2^-52 (|psi| < 2^11 = 2048, far beyond
// any potential of a lattice electrolyte in units of k_B T / e).  Sums and
// differences of neighbouring values are then exact integer operations, so
// the Poisson residual s - A psi is computed without cancellation error and
// without FP64 arithmetic (FP64 throughput on GB300 is a small fraction of
// FP32).  The Poisson source s = 4 pi l_B (rho_e + w) uses the same scale
// (|s| < 2048).  The smoothers work on FP32 corrections.
constexpr double PSI_SCALE = 4503599627370496.0;        // 2^52
constexpr double PSI_INV_SCALE = 1.0 / 4503599627370496.0;
constexpr float PSI_SCALE_F = 4503599627370496.0f;
constexpr float PSI_INV_SCALE_F = 1.0f / 4503599627370496.0f;
constexpr double PSI_MAX = 2048.0;                      // 2^11
// Absolute convergence floor of the Poisson solvers, as an rms residual in
// fixed-point units: rounding psi to the 2^-52 grid alone leaves a residual
// of rms sqrt((36 + 6) / 12) = 1.9 units under the 7-point operator, so a
// source of vanishing norm is solved once the residual is within twice that.
constexpr double RES_FLOOR_RMS = 4.0;

// Extrapolation in time of a fixed-point potential from its last values
// a = psi(t-1), b = psi(t-2), c = psi(t-3), d = psi(t-4), `order` of the
// older ones being valid:
//   order 0   a
//   order 1   2a - b             (line)
//   order 2   3a - 3b + c        (parabola)
//   order 3   2a - 2c + d        (exact for quadratics and for the
//                                 alternation (-1)^t, which the parabola
//                                 amplifies sevenfold; it needs no b)
// Exact in 128-bit integers; a value outside 2^61 units keeps a.
__device__ __forceinline__ int64_t extrapolate1(int64_t a, int64_t b, int64_t c, int64_t d,
                                                int order) {
  if (order <= 0) return a;
  const __int128 A = a;
  const __int128 g = order == 1   ? 2 * A - b
                     : order == 2 ? 3 * (A - b) + c
                                  : 2 * (A - c) + d;
  const __int128 lim = (__int128)1 << 61;
  return (g > lim || g < -lim) ? a : (int64_t)g;
}
// The history of the extrapolation: HIST_SLOTS lattice-sized buffers used as
// a ring.  With ring position r, psi(t-2) is in slot (r + 2) % 3, psi(t-3)
// in (r + 1) % 3 and psi(t-4) in r % 3; the start of a solve overwrites
// slot r % 3 with psi(t-1), and r advances by one.
constexpr int HIST_SLOTS = 3;
constexpr int HIST_ORDER = 3;  // valid entries of a full history

#ifdef __CUDACC__
// Conversions between 64-bit integers and FP32 on the 32-bit integer and FP32
// pipes: the instructions for 64-bit conversions issue on the FP64 pipe,
// which is narrow on this GPU (ncu shows the residual kernels bound by it).
//
// i64_to_f32: |v| = hi 2^32 + lo; hi, lo >> 16 and lo & 0xffff (each below
// 2^23) become floats exactly by placing them in the mantissa of 2^23 and
// subtracting 2^23; two FMAs join them (two roundings: within about one ulp
// of the correctly rounded value).  |v| >= 2^55 takes the plain conversion.
__device__ __forceinline__ float i64_to_f32(int64_t v) {
  const bool neg = v < 0;
  const uint64_t a = neg ? 0ull - (uint64_t)v : (uint64_t)v;
  const uint32_t hi = (uint32_t)(a >> 32), lo = (uint32_t)a;
  if (hi >= (1u << 23)) return (float)v;
  const float fh = __uint_as_float(0x4B000000u | hi) - 8388608.0f;
  const float fm = __uint_as_float(0x4B000000u | (lo >> 16)) - 8388608.0f;
  const float fl = __uint_as_float(0x4B000000u | (lo & 0xFFFFu)) - 8388608.0f;
  const float f = fmaf(fh, 4294967296.0f, fmaf(fm, 65536.0f, fl));
  return neg ? -f : f;
}

// f32_to_i64_rn: nearest integer (ties to even), |f| < 2^63.  |f| < 2^22:
// adding 1.5 * 2^23 rounds f to an integer in the low mantissa bits.  Else
// |f| rounded to an integer (exactly, by adding and subtracting 2^23 below
// 2^23) is mantissa * 2^e, shifted into place.
__device__ __forceinline__ int64_t f32_to_i64_rn(float f) {
  const float a = fabsf(f);
  if (a < 4194304.0f) return (int64_t)(__float_as_int(f + 12582912.0f) - 0x4B400000);
  const float r = a < 8388608.0f ? (a + 8388608.0f) - 8388608.0f : a;
  const uint32_t b = __float_as_uint(r);
  const int e = (int)(b >> 23) - 150;
  const uint64_t mant = (uint64_t)((b & 0x7FFFFFu) | 0x800000u);
  const int64_t m = (int64_t)(e >= 0 ? mant << e : mant >> 1);
  return f < 0.f ? -m : m;
}
#endif

// Per-node link word (only allocated when walls exist):
//   bit 0      node is a wall node
//   bit p      (p = 1..18) the upstream node r - c_p is a wall node
constexpr uint32_t LINK_SOLID = 1u;

struct StepArgs {
  const void* fin;
  void* fout;
  const uint32_t* links;   // NULL without walls
  const int64_t* psi;      // fixed point, lattice-sized; NULL when neutral
  const float* wallq;      // face charge share of each wall node; may be NULL
  int nx, ny, nz;
  int64_t N;
  float omega_visc, omega_drag;
  const float* omega_drag_z;  // per z-plane drag frequency (stacked instances) or NULL
  float fourpi_lb;
  float eext[3];
  float valence[MAX_SPECIES];
  float nref[MAX_SPECIES];  // reference density of the 16-bit shifted storage
  uint32_t step;            // time step (seeds the stochastic rounding)
  const uint32_t* step_dev; // device copy of the step (graph replays) or NULL
  double* diag;             // per-CTA diagnostics partials (DIAG_NQ per CTA) or NULL
};

struct PoissonLevel {
  int nx, ny, nz;
  int64_t n;
  int per[3];        // periodic flags
  int coarsened[3];  // 1 if this level halves that axis of the finer level
  float* e = nullptr;     // correction
  float* rhs = nullptr;   // right-hand side
  float* K = nullptr;     // [3][n] conductance to the + neighbour (levels >= 1)
  float* Dinv = nullptr;  // 1 / diagonal, 0 for an inactive cell (levels >= 1)
};

struct Poisson {
  static constexpr int NSLOT = 8;  // residual norm slots (batched spectral applications)
  // box of the fine grid inside the lattice: x, y full, z in [zlo, zlo+nzb)
  int zlo = 0, nzb = 0, perz = 1;
  std::vector<PoissonLevel> lev;
  int64_t* psi[2] = {nullptr, nullptr};  // lattice-sized fixed-point buffers
  int64_t* hist = nullptr;  // multigrid / SOR: HIST_SLOTS x N, the ring of older potentials
  int hist_n = 0;           // valid entries of hist (0..HIST_ORDER)
  int hist_ring = 0;        // ring position
  int cur = 0;
  int64_t* src = nullptr; // 4 pi l_B (rho_e + w) per lattice node (fixed point), no mean removed
  double* dsum = nullptr; // [0] sum of src over fluid, [1 + 2k] sum r^2, [2 + 2k] sum s^2 (fixed-point units), k < NSLOT
  double* hsum = nullptr; // pinned mirror of dsum
  long long* part = nullptr; // per-CTA partial sums of the charge kernel
  // connected fluid components (face neighbours): label per lattice node
  // (0 = largest component), allocated only when there is more than one
  int ncomp = 1;
  int* label = nullptr;
  unsigned long long* comp_sum = nullptr;  // source sums of components >= 1
  long long* comp_size = nullptr;           // cells per component
  long long* comp_mean = nullptr;           // source mean per component (fixed point)
  int64_t nfluid = 0;
  int coarse_sweeps = 16;
  double conv = 0.15;    // measured residual reduction per V-cycle (last solve)
  // one V-cycle plus the residual, captured as a CUDA graph per starting
  // potential buffer (the cycle ping-pongs the two buffers)
  cudaGraphExec_t cyc[2] = {nullptr, nullptr};
  int cyc_kernels = 0;
  bool cyc_failed = false;
  int nu1 = 2, nu2 = 2;
};

}  // namespace lbm_gb300

namespace lbm_gb300 {
struct SpectralPlan;
struct NNet;
}

struct lbm {
  lbm_config cfg;
  int S = 0;
  int64_t N = 0;
  int dev = 0;
  cudaStream_t own = nullptr;
  cudaStream_t st = nullptr;  // stream of the call in progress
  // ordering between a caller's stream and the library's own stream: the
  // last lbm_step on a caller's stream records this event there, and the
  // next call on the own stream waits for it (foreign_pending)
  cudaEvent_t order_ev = nullptr;
  bool foreign_pending = false;
  size_t esize = 4;
  void* f[2] = {nullptr, nullptr};
  int cur = 0;
  float mass[lbm_gb300::MAX_SPECIES] = {0};
  float valence[lbm_gb300::MAX_SPECIES] = {0};
  float nref[lbm_gb300::MAX_SPECIES] = {1, 1, 1, 1};
  unsigned species_set = 0;
  double mass0 = 0.0;
  bool has_walls = false;
  uint32_t* links = nullptr;
  float* wallq = nullptr;
  int64_t* wsrc = nullptr;  // 4 pi l_B w_i in fixed point (wall charge of each fluid cell)
  int64_t nfluid = 0;
  lbm_gb300::Poisson ps;
  lbm_gb300::SpectralPlan* spec = nullptr;  // spectral Poisson plan (LBM_POISSON_FFT)
  lbm_gb300::NNet* nn = nullptr;            // learned Poisson initial guess
  bool psi_valid = false;
  double* dred = nullptr;   // diagnostics partials, (MAX_SPECIES + 4) x DIAG_SPREAD (device)
  // per-CTA diagnostics partials written by every stream/collide launch
  // (DIAG_NQ doubles per CTA); diag_valid: they describe the current state
  double* dpart = nullptr;
  int64_t dpart_ctas = 0;   // CTAs of the last stream/collide launch
  bool diag_valid = false;
  // set by the spectral plan when the fluid is one periodic run: the charge
  // kernel's partial sum writes the source mean of every plane there, and
  // sets charge_means_ready for the next solve (which consumes it)
  long long* charge_mean_z = nullptr;
  bool charge_means_ready = false;
  // step counter advanced by the charge path while graph steps are captured
  uint32_t* charge_step = nullptr;
  double* hred = nullptr;   // pinned mirror
  int* dflag = nullptr;
  int last_iters = 0;
  double last_res = 0.0;
  int64_t tstep = 0;
  // phase timing (lbm_set_timing)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<int, int>>> ev_marks;  // phase, (start, stop)
  size_t ev_used = 0;
  double t_acc[3] = {0, 0, 0};
  int64_t t_cnt[3] = {0, 0, 0};
  int64_t launches = 0;
  int grid_cap = 1216;   // CTAs of the grid-stride reduction kernels (8 per SM)
  float* omega_drag_z = nullptr;  // per-plane drag frequency (lbm_set_plane_omega_drag)
  int collide_threads = 128;      // CTA size of the stream-collide kernel (autotuned)
  // whole-step CUDA graphs (LBM_FLAG_STEP_GRAPH), one per population parity
  cudaGraphExec_t step_graph[2] = {nullptr, nullptr};
  void* gstatus = nullptr;        // device status of graph steps
  void* hstatus = nullptr;        // pinned mirror
  int graph_kernels_fixed = 0;    // kernels per step outside the Poisson loop
  int graph_kernels_iter = 0;     // kernels per Poisson iteration
  int graph_kernels_redo = 0;     // kernels of the stream/collide run again after the loop
  std::vector<int> instance_z0;   // first plane of each stacked instance
  int charge_threads = 256;       // CTA size of the charge kernel (autotuned)  // kernels launched since timing was (re)set
  std::string err;
};

namespace lbm_gb300 {

// ---- lbm_api.cu ----
// Makes the library's own stream the stream of the call in progress, after
// the work that the last lbm_step queued on a caller's stream.
cudaError_t own_stream(lbm_t* h);

// ---- lbm_kernels.cu ----
cudaError_t launch_init_species(lbm_t* h, int s, const double* n0_dev,
                                const double* u0_dev);
cudaError_t launch_stream_collide(lbm_t* h);
// Stream-collide into the spare lattice with a given CTA size, without
// advancing the state (autotuning).
cudaError_t launch_stream_collide_probe(lbm_t* h, int threads);
cudaError_t launch_charge(lbm_t* h);
cudaError_t launch_gather(lbm_t* h, int s, double* n_dev, double* u_dev,
                          double* f_dev);
cudaError_t launch_diagnostics(lbm_t* h);
// Plane sums of n and of the mid-step flux per species (lbm_plane_fluxes):
// nz * S * 4 doubles, device.
cudaError_t launch_plane_fluxes(lbm_t* h, double* out_dev);
// Checks an initial species field in device memory (lbm_set_species_dev):
// per-CTA fluid sums of n0 and counts of invalid entries, 2 doubles per CTA
// in out (at most 256 CTAs, *nblk of them).
cudaError_t launch_species_check(lbm_t* h, const double* n0_dev, const double* u0_dev, double* out,
                                 int* nblk);
// Sums the stream/collide kernel's per-CTA diagnostics partials into out
// (DIAG_NQ doubles, device).
cudaError_t launch_diag_reduce(lbm_t* h, double* out);
cudaError_t launch_links(lbm_t* h, const uint8_t* solid_dev);
cudaError_t launch_psi_to_double(lbm_t* h, const int64_t* psi, double* out);
cudaError_t launch_psi_from_double(lbm_t* h, const double* in, int64_t* psi);
cudaError_t launch_src_from_rho(lbm_t* h, const double* rho_dev);

// ---- lbm_poisson.cu ----
lbm_status poisson_setup(lbm_t* h, const uint8_t* solid_host);
void poisson_free(lbm_t* h);
// Solves A psi = src - mean starting from the current psi buffer.
lbm_status poisson_solve(lbm_t* h, double tol, int maxit, int* iters,
                         double* rel_res);
// Multigrid / SOR host-driven steps: psi <- its extrapolation from the
// previous steps before the step's solve (as spectral_step_start).
lbm_status poisson_step_start(lbm_t* h);

// ---- lbm_spectral.cu ----
lbm_status spectral_setup(lbm_t* h, const uint8_t* solid_host);
void spectral_free(lbm_t* h);
lbm_status spectral_solve(lbm_t* h, double tol, int maxit, int* iters,
                          double* rel_res);
// Whole-step graphs: build (if needed) and replay nsteps steps; reads the
// device status once at the end.
lbm_status spectral_graph_steps(lbm_t* h, int nsteps);
void spectral_graph_free(lbm_t* h);
// Host-driven steps: psi <- its extrapolation from the previous steps
// before the step's solve (LBM_FLAG_NO_EXTRAPOLATION off, no learned guess).
lbm_status spectral_step_start(lbm_t* h);
// Restarts the potential history of every solver (psi was set from outside
// the steps).
lbm_status potential_history_reset(lbm_t* h);

// ---- lbm_nn.cu ----
lbm_status nn_init(lbm_t* h, int hidden, uint64_t seed);
void nn_free(lbm_t* h);
lbm_status nn_collect(lbm_t* h, int capacity);
lbm_status nn_train(lbm_t* h, int epochs, double lr, double* losses);
lbm_status nn_loss_grad_host(lbm_t* h, const float* x0, double* loss, float* grad);
lbm_status nn_params(lbm_t* h, float* get, const float* set, int* np);
// Solver hooks: given the initial FP32 residual (planes [zlo, zlo+nzb)),
// stores it for training and/or applies the learned correction to psi.
lbm_status nn_before_solve(lbm_t* h, const float* r, int zlo, int nzb, double rms,
                           bool* applied, float** dpsi);
lbm_status nn_revert(lbm_t* h, const float* dpsi);
void nn_record(lbm_t* h, double ratio);
bool nn_active(const lbm_t* h);
void nn_stats(const lbm_t* h, double* out);
lbm_status nn_set_use(lbm_t* h, int enable);

}  // namespace lbm_gb300

#define LBM_CUDA_TRY(h, call)                                              \
  do {                                                                     \
    cudaError_t _e = (call);                                               \
    if (_e != cudaSuccess) {                                               \
      (h)->err = std::string(#call) + ": " + cudaGetErrorString(_e);       \
      return _e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;     \
    }                                                                      \
  } while (0)
