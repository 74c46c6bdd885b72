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
// per-step record of lbm_step_record: the DIAG_NQ diagnostics sums, the
// step's Poisson applications and final relative residual
constexpr int REC_LEN = DIAG_NQ + 2;
constexpr int REC_CHUNK = 4096;  // steps recorded between two host waits

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

// Differences of the source and potential history kept for the start of
// each step's Poisson solve (lbm_start.cu).
constexpr int START_K = 5;
// index of the ring position in the history's device state
constexpr int START_RING_IDX = 1;
// starts fitted on at least this many differences count as steady-state
// steps for the graph steps' choice of the number of applications
constexpr int START_FULL_TERMS = START_K;

#ifdef __CUDACC__
// Conversions between 64-bit integers and FP32 on the 32-bit integer and FP32
// pipes: the instructions for 64-bit conversions issue on the FP64 pipe,
// which is narrow on this GPU (ncu shows the residual kernels bound by it).
//
// Compensated FP32 accumulation (Knuth's two-sum): hi + lo carries the sum
// to about twice the FP32 precision without FP64 arithmetic, which is slow
// on this GPU.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += e;
}

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
  const int* skip;          // device flag: nonzero makes the launch return at once (or NULL)
  // matrix of pair drag frequencies omega^{ab} (Sec. 2, general gamma^{ab}
  // for equal masses; zero diagonal), used instead of omega_drag when pair_on
  int pair_on;
  float pair[MAX_SPECIES][MAX_SPECIES];
  // charge scatter (periodic lattices without walls, nx a multiple of 32):
  // each node's stored charged populations are added, in fixed point, to
  // the next step's Poisson source at the node they stream to; NULL when a
  // separate pass computes the source
  int64_t* scat_acc;
  float scat_k[MAX_SPECIES];  // 4 pi l_B z n_ref 2^52 (0 for a neutral species)
  long long src_ref;          // 4 pi l_B sum_a z_a n_ref_a in fixed point, once per node
};

// The start's first pass fused into the charge pass: the source difference
// D_0 = s(t) - s(t-1) (s(t-1): what the source buffer holds before the pass
// overwrites it) into the ring slot of the current position, and its
// products with D_0 and the stored D_1 .. D_K per CTA into part.
struct DotsArgs {
  float* ring_d;       // START_K x N differences of consecutive sources
  const int* state;    // history state (ring position at START_RING_IDX)
  float* part;         // (START_K + 1) floats per CTA
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
  int cur = 0;
  int64_t* src = nullptr; // 4 pi l_B (rho_e + w) per lattice node (fixed point), no mean removed
  double* dsum = nullptr; // [0] sum of src over fluid, [1 + 2k] sum r^2, [2 + 2k] sum s^2 (fixed-point units), k < NSLOT
  double* hsum = nullptr; // pinned mirror of dsum
  uint8_t* face = nullptr; // face mask of the fine box (colour-split), walls only
  float* nacc = nullptr;   // norm slots of the multigrid residual (|r|^2, then |s|^2)
  float* hacc = nullptr;   // pinned mirror of nacc
  double snorm = 0.0;      // ||s - <s>|| of the current solve (fixed-point units)
  bool snorm_pending = false;  // the queued residual also carries the source norm
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
  // smoothing sweeps before / after the coarse correction: fine box and the
  // shared-memory sub-cycle (nu), the grid-kernel coarse levels between them
  // (nuc).  1 / 1 on the grid coarse levels saved 7% per V-cycle at 256^3
  // but cost cycles: less Poisson time for long solves from the previous
  // potential (13.9 cycles a step), more for the ~2-cycle solves from the
  // history start (porous 256^3: 1.78 against 1.74 ms a step; bulk 128^3:
  // 3.35 against 2.82 cycles), so all levels keep 2 / 2.
  int nu1 = 2, nu2 = 2;
  int nuc1 = 2, nuc2 = 2;
};

// History of the start of the Poisson solves (lbm_start.cu), device memory.
struct StartHistory {
  int64_t* s_prev = nullptr;    // source of the previous step (fixed point)
  int64_t* psi_prev = nullptr;  // potential of the step before the previous one
  float* ring_d = nullptr;      // START_K x N: differences of consecutive sources
  float* ring_p = nullptr;      // START_K x N: differences of consecutive potentials
  float* part = nullptr;        // per-CTA inner products, START_K + 1 per CTA
  double* gram = nullptr;       // START_K x START_K Gram matrix of the stored differences
  float* coef = nullptr;        // START_K coefficients of the current step
  int* state = nullptr;         // valid steps, ring position, terms of coef, terms used
  int ctas = 0;
  // the charge scatter's source take also ran the fit's first pass (the
  // differences and inner products) for this step, with dots_ctas partials
  bool dots_done = false;
  int dots_ctas = 0;
  // it also applied the start of the potential (and cleared the first norm
  // slot when psi_cleared), which start_apply then skips
  bool psi_done = false;
  bool psi_cleared = false;
  int part_ctas = 0;            // CTAs part has room for
  cudaStream_t side = nullptr;  // the fit runs here, beside the solve (lowest priority)
  cudaEvent_t fork = nullptr, join = nullptr;
  bool pending = false;         // a fit was queued on side and not yet joined
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
  lbm_gb300::StartHistory start;  // start of each step's Poisson solve
  lbm_gb300::SpectralPlan* spec = nullptr;  // spectral Poisson plan (LBM_POISSON_FFT)
  lbm_gb300::NNet* nn = nullptr;            // learned Poisson initial guess
  bool psi_valid = false;
  double* dred = nullptr;   // diagnostics partials, (MAX_SPECIES + 4) x DIAG_SPREAD (device)
  // per-CTA diagnostics partials written by every stream/collide launch
  // (DIAG_NQ doubles per CTA); diag_valid: they describe the current state
  double* dpart = nullptr;
  int64_t dpart_ctas = 0;   // CTAs of the last stream/collide launch
  double* dmid = nullptr;   // second level of the partials' reduction (k_diag_reduce)
  unsigned* ddone = nullptr;  // CTAs of k_diag_reduce done (reset by its last CTA)
  bool diag_valid = false;
  // set by the spectral plan when the fluid is one periodic run: the charge
  // kernel's partial sum writes the source mean of every plane there, and
  // sets charge_means_ready for the next solve (which consumes it)
  long long* charge_mean_z = nullptr;
  bool charge_means_ready = false;
  // step counter advanced by the charge path while graph steps are captured
  uint32_t* charge_step = nullptr;
  const int* collide_skip = nullptr;  // skip flag of the stream/collide being captured
  // extra duties of the start's bookkeeping kernel while a step graph is
  // captured: the speculation flag and the first norm slot to clear
  int* mark_skip_out = nullptr;
  const int* mark_prev_iters = nullptr;  // the previous step's applications (graph status)
  int mark_k = 0;                        // applications baked into the graph being captured
  float* mark_clear = nullptr;
  int mark_nclear = 0;
  bool slot0_cleared = false;  // the start's kernel cleared norm slot 0 (spec_fwd skips it)
  double* hred = nullptr;   // pinned mirror
  // per-step records (lbm_step_record): mapped pinned host slots (hrec,
  // its device address hrec_dev), written by the reduce kernel behind each
  // step; rec_dev / rec_host are set while a recording call steps (else
  // NULL)
  double* hrec = nullptr;
  double* hrec_dev = nullptr;
  int rec_cap = 0;
  double* rec_dev = nullptr;
  double* rec_host = nullptr;
  int* dflag = nullptr;
  int last_iters = 0;
  double last_res = 0.0;
  // start residuals of the Poisson solves (lbm_poisson_stats): the last
  // one, and the sum of log10 and the count since lbm_set_timing
  double last_start = 0.0;
  double start_log_sum = 0.0;
  int64_t start_count = 0;
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
  // matrix of pair drag frequencies (lbm_set_drag_matrix; three or more
  // species), and the config's omega_drag before a binary matrix replaced it
  bool pair_on = false;
  float pair[lbm_gb300::MAX_SPECIES][lbm_gb300::MAX_SPECIES] = {};
  double omega_drag_cfg = 0.0;
  int collide_threads = 128;      // CTA size of the stream-collide kernel (autotuned)
  // whole-step CUDA graphs (LBM_FLAG_STEP_GRAPH), one per population parity
  // [parity] and stream/collide variant [diag]
  cudaGraphExec_t step_graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  // the species' reference densities and valences the graphs were built with
  float graph_nref[lbm_gb300::MAX_SPECIES] = {0};
  float graph_valence[lbm_gb300::MAX_SPECIES] = {0};
  void* gstatus = nullptr;        // device status of graph steps
  void* hstatus = nullptr;        // pinned mirror
  int graph_kernels_fixed = 0;    // kernels per step outside the Poisson loop
  int graph_kernels_iter = 0;     // kernels per Poisson iteration
  int graph_kernels_redo = 0;     // kernels of the stream/collide run again after the loop
  std::vector<int> instance_z0;   // first plane of each stacked instance
  int charge_threads = 256;       // CTA size of the charge kernel (autotuned)
  // charge scatter (LBM_FLAG_CHARGE_PASS off, periodic lattice without
  // walls, nx a multiple of 32): scat_acc
  // accumulates the next step's Poisson source in the stream/collide;
  // scat_valid: it holds the source of the current populations (the step
  // then takes it instead of running the charge pass)
  bool scat_on = false;
  bool scat_valid = false;
  int64_t* scat_acc = nullptr;
  unsigned long long* scat_tot = nullptr;  // running 128-bit source total and CTA count (k_src_take)
  std::string err;
};

namespace lbm_gb300 {

// ---- lbm_api.cu ----
// Makes the library's own stream the stream of the call in progress, after
// the work that the last lbm_step queued on a caller's stream.
cudaError_t own_stream(lbm_t* h);

// ---- lbm_collide.cu (one object per storage format) ----
// Launches the fused stream/collide of storage format ST from a to a.fout:
// S species, walls w, charged c, `threads` per CTA, diagnostics variant d.
// (a.pair_on selects the pair-frequency drag; three or more species).
template <int ST>
cudaError_t collide_dispatch(const StepArgs& a, int S, bool w, bool c, cudaStream_t st,
                             int threads, bool d);
template <>
cudaError_t collide_dispatch<LBM_FP32>(const StepArgs&, int, bool, bool, cudaStream_t, int, bool);
template <>
cudaError_t collide_dispatch<LBM_FP16_SHIFT>(const StepArgs&, int, bool, bool, cudaStream_t, int,
                                             bool);
template <>
cudaError_t collide_dispatch<LBM_BF16_SHIFT>(const StepArgs&, int, bool, bool, cudaStream_t, int,
                                             bool);

// Records the relative residual at the start of a Poisson solve.
void note_start_residual(lbm_t* h, double rel);

// ---- lbm_kernels.cu ----
cudaError_t launch_init_species(lbm_t* h, int s, const double* n0_dev,
                                const double* u0_dev);
// diag: the variant that also writes the FP64 diagnostics partials of the
// state it stores (the last step of an lbm_step call)
cudaError_t launch_stream_collide(lbm_t* h, bool diag);
// Stream-collide into the spare lattice with a given CTA size, without
// advancing the state (autotuning).
cudaError_t launch_stream_collide_probe(lbm_t* h, int threads);
cudaError_t launch_charge(lbm_t* h);
// With the charge scatter on and no valid scattered source, runs the charge
// pass into the accumulator (so that the next step's launch_charge takes it).
cudaError_t charge_prepare(lbm_t* h);

// ---- lbm_start.cu: the source take fused with the fit's first pass ----
// With the start from the history on, moves the scattered source into the
// Poisson source (as k_src_take: accumulator cleared, exact total, mean,
// step counter) and forms the step's source difference and its inner
// products in the same pass; returns false (launching nothing) when the
// start is off.
bool launch_take_dots(lbm_t* h, unsigned ctas, double inv_nfluid);
// The arguments for fusing the start's first pass into a charge pass of
// `ctas` CTAs that writes the Poisson source; marks the step's pass as done.
// False when the start is off.
bool charge_dots_args(lbm_t* h, int ctas, DotsArgs* out);
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
// Reduces the stream/collide's per-CTA diagnostics partials into out (may
// be mapped pinned host memory); iters / rel (device, or NULL) are copied
// behind them.
cudaError_t launch_diag_reduce(lbm_t* h, double* out, const int* iters = nullptr,
                               const double* rel = nullptr);
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

// ---- lbm_spectral.cu ----
lbm_status spectral_setup(lbm_t* h, const uint8_t* solid_host);
void spectral_free(lbm_t* h);
lbm_status spectral_solve(lbm_t* h, double tol, int maxit, int* iters,
                          double* rel_res);
// Whole-step graphs: build (if needed) and replay nsteps steps; reads the
// device status once at the end.
lbm_status spectral_graph_steps(lbm_t* h, int nsteps);
// Device addresses of the current step's Poisson applications and final
// relative residual in the graph status.
void graph_status_ptrs(lbm_t* h, const int** iters, const double** rel);
void spectral_graph_free(lbm_t* h);
// Restarts the potential history of every solver (psi was set from outside
// the steps).
lbm_status potential_history_reset(lbm_t* h);

// ---- lbm_start.cu ----
lbm_status start_setup(lbm_t* h);
void start_free(lbm_t* h);
// The start is used (LBM_FLAG_NO_EXTRAPOLATION off).
bool start_enabled(const lbm_t* h);
// After the step's charge density: psi <- the start from the history.
// lagged: with the coefficients of the previous step's fit, this step's
// fit then queued on the side stream (start_join orders h->st after it);
// otherwise this step's fit first, on h->st.  The history restarts when
// the start is disabled.
cudaError_t start_step(lbm_t* h, bool lagged);
cudaError_t start_join(lbm_t* h);
// The two halves for graph capture: the start on h->st, the fit on st;
// `last` marks the step's last pass (it advances the history ring).
cudaError_t start_apply(lbm_t* h, bool last);
cudaError_t start_fit(lbm_t* h, cudaStream_t st, bool last);
// The history restarts (psi or the state was set from outside the steps).
cudaError_t start_reset(lbm_t* h);
// Device address of the number of terms the current step's start used
// (START_K: the full history).
const int* start_terms_dev(const lbm_t* h);

// ---- lbm_nn.cu ----
lbm_status nn_init(lbm_t* h, int hidden, uint64_t seed);
void nn_free(lbm_t* h);
lbm_status nn_collect(lbm_t* h, int capacity);
lbm_status nn_train(lbm_t* h, int epochs, double lr, double* losses);
lbm_status nn_loss_grad_host(lbm_t* h, const float* x0, double* loss, float* grad);
lbm_status nn_infer_host(lbm_t* h, const float* x0, float* y);
lbm_status nn_params(lbm_t* h, float* get, const float* set, int* np);
// Solver hooks: given the initial FP32 residual (planes [zlo, zlo+nzb);
// natural order when hx = 0, else colour-split with hx cells of a colour per
// x row), stores it for training and/or applies the learned correction.
lbm_status nn_before_solve(lbm_t* h, const float* r, int zlo, int nzb, int hx, double rms,
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
