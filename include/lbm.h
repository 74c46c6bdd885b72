/*
 * lbm.h -- C ABI of the GB300 two-timescale multicomponent lattice
 * Boltzmann library (D3Q19).
 *
 * The model is the discrete kinetic equation of Monteferrante, Melchionna
 * and Marini Bettolo Marconi, "Lattice Boltzmann Method for mixtures at
 * variable Schmidt number": for every species alpha and direction p,
 *
 *   f_p(r + c_p, t + 1) = f_p(r, t) - omega_visc [f_p - phi_perp,p] + g_p
 *
 * (Eq. latboeq), with the orthogonalised equilibrium phi_perp (Appendix,
 * final expression), the second-order forcing term g_p (Eq. ourforc) carrying
 * the interspecies drag of frequency omega_drag (Sec. 2, drag force) and the
 * mean-field electric force of the potential that solves the Poisson
 * equation nabla^2 psi = -4 pi l_B sum_alpha z^alpha n^alpha with the
 * surface-charge boundary condition (Eq. Poisson and the condition after it).
 *
 * Conventions shared by every entry point
 *   - Lattice: nx * ny * nz nodes on a 3-torus, index (z*ny + y)*nx + x,
 *     x fastest.  Walls are solid nodes; a non-periodic face is closed by
 *     a layer of solid nodes.  Halfway bounce-back at solid nodes.
 *   - D3Q19 order: 0 rest, 1..6 = +x,-x,+y,-y,+z,-z, 7..18 the 12 edge
 *     vectors in opposite pairs (2k-1, 2k).
 *   - Units: lattice units, v_T^2 = c_s^2 = 1/3, unit time step.
 *   - Host pointers are caller-owned, read or written during the call only
 *     and never retained.  Device memory is owned by the handle.
 *   - Every call returns an lbm_status; nothing throws across the ABI.
 *     The message of the last failure is lbm_last_error(h).
 *   - All calls on one handle must come from one host thread at a time.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm lbm_t; /* opaque, owned by the library */

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,    /* bad argument or call order                      */
  LBM_ENOMEM = 2,    /* device allocation failed                        */
  LBM_ECUDA = 3,     /* CUDA runtime error (message has the CUDA text)  */
  LBM_ENOCONV = 4,   /* Poisson solve hit its iteration limit           */
  LBM_EUNSTABLE = 5, /* non-finite or non-positive density detected     */
  LBM_ETIMEOUT = 6   /* reserved for a bounded device wait that gives up;
                        no call of this version returns it (no kernel of
                        the library waits on another CTA or device)     */
} lbm_status;

/* Population storage.  Every format stores the deviation of a population
 * from the reference equilibrium at rest, h = f / (w_p n_ref) - 1, with
 * n_ref the species' mean initial density (set by lbm_set_species), in
 * FP32, FP16 or BF16; the step computes in FP32 on deviations.  16-bit
 * stores round stochastically.                                            */
enum { LBM_FP32 = 0, LBM_FP16_SHIFT = 1, LBM_BF16_SHIFT = 2 };
/* Poisson solvers.  MG: geometric multigrid (any wall geometry).  SOR:
 * red-black successive over-relaxation (any geometry; slow, a reference).
 * FFT: 2-D FFT in x, y with an FFT (periodic power-of-two nz, 8..256) or
 * tridiagonal solves along z, exact in one pass up to FP32 rounding; needs
 * power-of-two nx, ny in [8, 256] with nx*ny <= 16384 and every z-plane
 * all fluid or all wall (periodic boxes, slits, stacks of slits); the
 * source mean is removed per run of fluid planes.                        */
enum { LBM_POISSON_MG = 0, LBM_POISSON_SOR = 1, LBM_POISSON_FFT = 2 };

typedef struct {
  int nx, ny, nz;        /* lattice extents, each >= 1                       */
  int nspecies;          /* 1..4                                             */
  double omega_visc;     /* 0 < w < 2: nu = c_s^2 (1/w - 1/2), Sec. 4        */
  double omega_drag;     /* 0 < w < 2: D = c_s^2 (1/w - 1/2), Sec. 4         */
  double bjerrum;        /* l_B of Eq. (Poisson); 0 = neutral, no Poisson    */
  double e_ext[3];       /* applied field, acceleration per unit valence     */
  int storage;           /* LBM_FP32 | LBM_FP16_SHIFT | LBM_BF16_SHIFT       */
  int poisson;           /* LBM_POISSON_MG | LBM_POISSON_SOR | LBM_POISSON_FFT */
  double poisson_tol;    /* ||s - A psi||_2 / ||s||_2 target, e.g. 1e-8, or
                            rms residual <= 4 * 2^-52 (psi's resolution)  */
  int poisson_maxit;     /* iteration cap (V-cycles or SOR sweeps)           */
  int device;            /* CUDA device ordinal                              */
  int flags;             /* LBM_FLAG_* bits                                  */
} lbm_config;

/* LBM_FLAG_STEP_GRAPH: every time step (charge density, spectral Poisson
 * solve with a device-side loop for extra applications, stream/collide) is
 * one CUDA graph replay; the host reads a small status after every 16
 * steps (and at the end of each lbm_step call) to report failures and to
 * adapt the number of applications baked into the graphs.  Needs
 * LBM_POISSON_FFT and l_B > 0.  Per-phase timings (lbm_get_timing) then
 * cover whole steps only.                                                 */
#define LBM_FLAG_STEP_GRAPH 1

/* LBM_FLAG_NO_EXTRAPOLATION: each step's Poisson solve (every solver)
 * starts from the previous step's potential.  Without the flag it starts
 * from the previous potential advanced along the recent history of the
 * solves: with the differences D_j = s(t-j) - s(t-j-1) of the last five
 * Poisson sources and P_j of the potentials, the coefficients c that fit
 * the new difference s(t) - s(t-1) best in least squares by sum c_j D_j
 * give psi(t-1) + sum c_j P_j (the projection of the new right-hand side on
 * the recent ones; fewer terms while the history fills after lbm_create,
 * lbm_set_species, lbm_set_state or lbm_solve_poisson, which restart it).
 * The solve still iterates to poisson_tol.  The learned guess, when in
 * use, corrects this start.  The paper has no counterpart: a property of
 * this library's solver.                                                  */
#define LBM_FLAG_NO_EXTRAPOLATION 2

/* LBM_FLAG_CHARGE_PASS: the charge density rho_e(t) of Eq. (Poisson) is
 * computed at the start of every step by a pass that pulls the charged
 * species' populations f(t).  Without the flag, on periodic FP32 lattices
 * without walls whose nx is a multiple of 32, the stream/collide of step
 * t - 1 adds each stored charged population to the node it streams to
 * (rho_e(r, t) = sum_a z_a sum_p f*_p^a(r - c_p, t - 1)), in 64-bit fixed
 * point, so the step reads those populations once; the results agree with
 * the pass up to FP32 rounding of the per-node sums.  The paper has no
 * counterpart: a property of this library's step.                        */
#define LBM_FLAG_CHARGE_PASS 4

/* Fills *cfg with defaults: omega_visc = 1, omega_drag = 1, l_B = 0,
 * FP32 storage, multigrid Poisson, tol 1e-8, maxit 200, device 0.        */
void lbm_config_default(lbm_config* cfg);

/* Creates a lattice.  Allocates two population lattices and the Poisson
 * hierarchy on cfg->device.  Returns LBM_EINVAL for extents < 1, species
 * outside 1..4, omega outside (0, 2), storage/poisson codes unknown;
 * LBM_ENOMEM when device memory runs out.  *out is NULL on failure.      */
lbm_status lbm_create(const lbm_config* cfg, lbm_t** out);

/* Batched instances.  Creates one lattice that stacks `count` independent
 * instances along z (each instance closes itself with its own wall planes,
 * set by the caller through lbm_set_walls on the stacked arrays).  All
 * cfgs share nx, ny, nspecies, omega_visc, bjerrum, e_ext, storage,
 * poisson, tolerances, device and flags; each brings its own nz and
 * omega_drag (the drag frequency becomes a per-plane field).  Instance i
 * occupies planes [lbm_instance_z0(h, i), lbm_instance_z0(h, i) + cfgs[i].nz).
 * LBM_EINVAL if the shared fields differ.                                 */
lbm_status lbm_create_stack(int count, const lbm_config* cfgs, lbm_t** out);
int lbm_instance_z0(const lbm_t* h, int i);

/* Per-plane drag frequency: omega (nz doubles, each in (0, 2)) replaces
 * the config's omega_drag on every node of plane z; NULL restores the
 * config value.                                                           */
lbm_status lbm_set_plane_omega_drag(lbm_t* h, const double* omega);

/* Drag between every pair of species (Sec. 2: the drag coefficient
 * gamma^{ab} of species of equal mass and diameters sigma_a, written as
 * omega^{ab} n_b / n): F_drag^a = -sum_b omega^{ab} (n_b / n)(v_a - v_b),
 * v the species velocities shifted by half the electric acceleration, as
 * for the single omega_drag (which is the case of equal omega^{ab}).  omega:
 * S*S doubles, row-major, symmetric (momentum is conserved), off-diagonal
 * entries in (0, 2), the diagonal is not used; NULL restores the config's
 * omega_drag.  For two species the drag depends on omega^{01} only, which
 * replaces omega_drag.  The relaxation rates of the species velocities are
 * then within (0, 2 max omega^{ab} (1 - x_a)) (Gershgorin), so entries below 1
 * are stable at any composition.  LBM_EINVAL for an entry out of range, an
 * asymmetric matrix, or per-plane drag frequencies (lbm_create_stack,
 * lbm_set_plane_omega_drag) on the same lattice.                           */
lbm_status lbm_set_drag_matrix(lbm_t* h, const double* omega);

/* Autotuner: times the stream/collide and charge kernels of the current
 * state at several CTA sizes (64, 128, 256) and keeps the fastest; the
 * populations do not advance, and the Poisson start's history restarts.
 * out (may be NULL) receives the chosen sizes and their times in ms:
 * [collide_threads, collide_ms, charge_threads, charge_ms]; with the charge
 * scatter (LBM_FLAG_CHARGE_PASS off, see there) the charge pass runs only
 * after new populations and is not timed (charge_ms 0, charge_threads
 * unchanged).                                                             */
lbm_status lbm_autotune(lbm_t* h, double* out);

/* Learned initial guess of the Poisson solve.  The paper has no
 * counterpart: this is an addition of this library.  A small periodic 3-D
 * convolutional network (two 3x3x3 layers, `hidden` channels, tanh) maps
 * the normalised residual of the solve's start (the history start of
 * LBM_FLAG_NO_EXTRAPOLATION's note, or the previous potential with that
 * flag) and the fluid mask to a correction of psi.  The solver applies it
 * before iterating, keeps it only if the residual drops, and always
 * iterates to the same tolerance.
 *   lbm_nn_init     random initialisation (seeded), hidden in 1..16;
 *                   requires l_B > 0 and host-driven steps
 *   lbm_nn_collect  store the initial residual of each following solve in
 *                   a ring of `capacity` fields (0 stops collecting)
 *   lbm_nn_train    `epochs` passes of Adam (rate lr) over the collected
 *                   fields on the GPU; losses[e] (may be NULL) receives the
 *                   mean loss ||r - A dpsi||^2 / ||r||^2 of each epoch
 *   lbm_nn_use      enable / disable the guess (FP16 inference)
 *   lbm_nn_params   copy the FP32 parameters out (get) or in (set), either
 *                   may be NULL; *nparams receives their count
 *   lbm_nn_loss_grad  loss and parameter gradient (FP32) on a given
 *                   normalised residual field x0 (N floats, host)
 *   lbm_nn_infer    the inference pass the solver uses (FP16 weights and
 *                   activations) on a given normalised residual x0: the
 *                   correction y in units of the residual's rms (N floats,
 *                   host; zero at wall nodes)
 *   lbm_nn_stats    out[0] guesses tried, out[1] kept, out[2] mean residual
 *                   ratio after/before of the kept ones, out[3] collected
 *                   fields, out[4] parameter count                        */
lbm_status lbm_nn_init(lbm_t* h, int hidden, uint64_t seed);
lbm_status lbm_nn_collect(lbm_t* h, int capacity);
lbm_status lbm_nn_train(lbm_t* h, int epochs, double lr, double* losses);
lbm_status lbm_nn_use(lbm_t* h, int enable);
lbm_status lbm_nn_params(lbm_t* h, float* get, const float* set, int* nparams);
lbm_status lbm_nn_loss_grad(lbm_t* h, const float* x0, double* loss, float* grad);
lbm_status lbm_nn_infer(lbm_t* h, const float* x0, float* y);
lbm_status lbm_nn_stats(lbm_t* h, double* out);

/* Releases every device buffer of h.  NULL is accepted.                  */
void lbm_destroy(lbm_t* h);

/* Walls (optional; must precede lbm_set_species).  solid: N bytes, non-zero
 * marks a wall node.  sigma: N doubles, the surface charge (units of e)
 * carried by each wall node, or NULL for uncharged walls; entries at fluid
 * nodes are ignored.  A wall node with k fluid face neighbours hands
 * sigma/k to each (boundary condition after Eq. Poisson).  LBM_EINVAL if
 * species were already set or every node is solid.                        */
lbm_status lbm_set_walls(lbm_t* h, const uint8_t* solid, const double* sigma);

/* Species s (0 <= s < nspecies): particle mass (equal for all species:
 * one thermal speed on the lattice), valence z^alpha, initial density n0
 * (N doubles, > 0 at fluid nodes) and velocity u0 (3N doubles laid out as
 * [3][N], or NULL for rest).  Sets f_p(r, 0) = phi_perp,p(n0, u0) at every
 * fluid node (local equilibrium, Appendix).  LBM_EINVAL for a bad index, a
 * different mass than an earlier species, or n0 <= 0 at a fluid node.     */
lbm_status lbm_set_species(lbm_t* h, int s, double mass, double valence,
                           const double* n0, const double* u0);

/* As lbm_set_species, with n0 (N doubles) and u0 (3N doubles, [3][N], or
 * NULL) in device memory of the handle's device: caller-owned (for example
 * torch tensors' data pointers), read by work queued on `stream` (a
 * cudaStream_t, or NULL for the library's stream) during the call, never
 * retained or freed.  Pass the stream on which the fields were written:
 * the library's own stream is a non-blocking stream and does not wait for
 * work on the legacy default stream.  The checks of lbm_set_species (n0
 * finite and > 0, u0 finite at every fluid node) run on the device; the
 * call returns after they were read back and the initialisation was
 * queued.  LBM_EINVAL as for lbm_set_species, and for a pointer the device
 * cannot reach (pinned host memory is accepted and read in place).        */
lbm_status lbm_set_species_dev(lbm_t* h, int s, double mass, double valence,
                               const double* n0_dev, const double* u0_dev, void* stream);

/* Advances nsteps >= 0 time steps of Eq. (latboeq).  Each step: charge
 * density and Poisson solve (if l_B > 0), fused stream + moments + forces +
 * collision of all species.  stream: a cudaStream_t, or NULL for the
 * library's own stream; the call returns after the work is queued except
 * that the Poisson convergence test reads one value back per iteration.
 * Work on a caller's stream starts after the work queued on the library's
 * stream, and every later call that runs on the library's stream (all
 * calls without a stream argument) waits for it: no lbm_synchronize is
 * needed between lbm_step(h, n, s) and lbm_get_moments(h, ...).
 * LBM_ENOCONV if a Poisson solve reached poisson_maxit (the state has then
 * advanced with the unconverged potential).                               */
lbm_status lbm_step(lbm_t* h, int nsteps, void* stream);

/* Blocks until all queued work of h is done.                             */
lbm_status lbm_synchronize(lbm_t* h);

/* Moments of the current state f(t) of species s: n (N doubles) and the
 * bare species velocity u = sum_p c_p f_p / n (3N doubles, [3][N]); either
 * pointer may be NULL.  Zero at wall nodes.  Host buffers.                */
lbm_status lbm_get_moments(lbm_t* h, int s, double* n, double* u);

/* As lbm_get_moments, into memory the handle's device can write: n_dev
 * (N doubles) and u_dev (3N doubles, [3][N]), either may be NULL,
 * caller-owned and never retained.  Device (or managed) memory, or pinned
 * host memory, which the gather kernel then writes directly (no separate
 * copy); any other pointer is refused with LBM_EINVAL before a kernel runs.
 * The gather is queued on `stream` (a cudaStream_t, or NULL for the
 * library's stream) after the last step and the call returns without
 * waiting for it; the caller orders its reads of the buffers on that
 * stream.                                                                  */
lbm_status lbm_get_moments_dev(lbm_t* h, int s, double* n_dev, double* u_dev, void* stream);

/* Plane sums of the current state, for the slit currents of Sec. 4 (mass
 * flow, electric and convective currents along the walls): for every
 * z-plane and species, over the plane's fluid nodes,
 *   out[(z*S + s)*4 + 0]      sum of n^s
 *   out[(z*S + s)*4 + 1..3]   sum of n^s (u^s + F^s / 2), x, y, z
 * with u^s the bare species velocity and F^s the force per unit mass of
 * Sec. 2 that the collision applies (applied and induced electric field,
 * drag on the force-shifted velocities): u^s + F^s / 2 is the velocity of
 * the second-order forcing of Eq. ourforc.  The induced field is the one of
 * the last Poisson solve (the potential the last step's collision used;
 * the same as the current one in a steady state).  out: nz*S*4 doubles,
 * host.                                                                     */
lbm_status lbm_plane_fluxes(lbm_t* h, double* out);

/* Moments as lbm_get_moments, for callers that must not allocate device
 * memory while they run (a device pool reserved by another framework, a
 * loop that cannot afford the device synchronisation of cudaMalloc).  The
 * paper has no counterpart: this is a library convenience.  It calls no
 * cudaMalloc / cudaFree: the device staging of the result is a static
 * device array of LBM_NOALLOC_MAX_NODES nodes x 4 doubles (8 MiB) that every
 * GPU loading the library holds until the process exits.  LBM_EINVAL when
 * the lattice has more nodes.  The first call on a device looks up the
 * array's device address; make that first call before any stream capture.
 * Like every call without a stream argument it runs after the last
 * lbm_step, also one queued on a caller's stream.  All calls share the
 * array: calls that overlap on the GPU (two handles or host threads on one
 * device) race on it.                                                      */
#define LBM_NOALLOC_MAX_NODES (1 << 18)
lbm_status lbm_get_moments_noalloc(lbm_t* h, int s, double* n, double* u);

/* Populations f_p(r, t) of species s (19*N doubles, [19][N]); zero at wall
 * nodes.  Host buffer.                                                    */
lbm_status lbm_get_populations(lbm_t* h, int s, double* f);

/* Potential psi (N doubles, zero at wall nodes) used by the last step's
 * collision.  Host buffer.                                                */
lbm_status lbm_get_potential(lbm_t* h, double* psi);

/* Standalone Poisson solve on the lattice's geometry (Eq. Poisson with the
 * wall charges of lbm_set_walls): A psi = 4 pi l_B (rho_e + w - mean).
 * rho_e: N doubles (host).  psi: N doubles (host), initial guess on entry,
 * solution on exit (zero mean over fluid cells is not enforced: the guess
 * fixes the constant).  tol, maxit as in the config (maxit <= 0 uses the
 * config's).  *iters and *rel_res (may be NULL) report the outcome.
 * Requires l_B > 0.  LBM_ENOCONV when the cap was hit (psi still written). */
lbm_status lbm_solve_poisson(lbm_t* h, const double* rho_e, double* psi,
                             double tol, int maxit, int* iters,
                             double* rel_res);

/* FP64 global diagnostics of the current state f(t).  After a step they
 * come from sums that the stream/collide kernel formed over what it stored
 * (per CTA, combined in FP64 in a fixed order: no pass over the lattice);
 * otherwise (after lbm_set_species or lbm_set_state) from a pass over the
 * populations.  Written to out:
 *   out[0 .. S-1]   total number of particles of each species
 *   out[S .. S+2]   total momentum sum_alpha sum_r m n^alpha u^alpha
 *   out[S+3]        net fluid charge sum_r sum_alpha z^alpha n^alpha
 *   out[S+4]        Poisson iterations of the last step
 *   out[S+5]        final relative Poisson residual of the last step
 *   out[S+6]        number of time steps taken
 * out must hold LBM_DIAG_LEN(S) doubles.  LBM_EUNSTABLE if a sum is not
 * finite or a density is non-finite or non-positive (after a step: a
 * density entering the last step; the values are still written).        */
#define LBM_DIAG_LEN(S) ((S) + 7)
lbm_status lbm_diagnostics(lbm_t* h, double* out);

/* nsteps time steps as lbm_step, each followed by the read-back of its
 * diagnostics: row k of out (LBM_DIAG_LEN(S) doubles per row, host memory,
 * nsteps rows) holds what lbm_diagnostics would return right after step k,
 * with that step's Poisson applications and final residual.  Every step
 * sums the state it stores in the stream/collide kernel (no pass over the
 * lattice); its sums are reduced on the device and copied to pinned
 * library memory with an asynchronous copy queued behind the step, so the
 * steps are not serialised by host waits: the call waits once per chunk
 * of up to 4096 steps and converts the rows.  stream as in lbm_step.
 * Returns as lbm_step; on an error the rows of the steps taken are
 * written.  LBM_EUNSTABLE when a row would make lbm_diagnostics return it
 * (all rows written).                                                     */
lbm_status lbm_step_record(lbm_t* h, int nsteps, double* out, void* stream);

/* Raw state for checkpointing (FP32 storage): the stored values of all
 * species, S*19*N floats in the library's internal order and form (post-
 * collision populations of the last step, before streaming, as
 * h = f / (w_p n_ref) - 1), plus the step counter.  lbm_set_state restores
 * exactly what lbm_get_state returned, into a lattice whose species were
 * set with the same initial densities (hence the same n_ref).  The
 * potential is not part of the state: the next solve starts from the
 * lattice's current psi, and its history restarts.                       */
lbm_status lbm_get_state(lbm_t* h, float* state, int64_t* step);
lbm_status lbm_set_state(lbm_t* h, const float* state, int64_t step);

/* The drag frequency of a Schmidt number Sc = nu / D, with the lattice
 * viscosity nu = c_s^2 (1/omega_visc - 1/2) and mutual diffusivity
 * D = c_s^2 (1/omega_drag - 1/2) of Sec. 4:
 *   omega_drag = 1 / (1/2 + (1/omega_visc - 1/2) / Sc).
 * Returns 0 when omega_visc is outside (0, 2) or Sc is not finite and
 * positive.                                                                */
double lbm_omega_drag_for_schmidt(double omega_visc, double schmidt);

/* Number of lattice nodes N = nx*ny*nz, and the element count of the raw
 * state (S*19*N).                                                          */
int64_t lbm_num_nodes(const lbm_t* h);
int64_t lbm_state_len(const lbm_t* h);

/* Start residuals of the Poisson solves (how good each solve's initial
 * potential was), written to out (5 doubles):
 *   out[0] iterations of the last solve (V-cycles, sweeps or applications)
 *   out[1] relative residual ||s - A psi|| / ||s|| at the start of the last
 *          solve (graph steps: the geometric mean over the last call's steps)
 *   out[2] relative residual at its end
 *   out[3] solves counted since lbm_set_timing
 *   out[4] mean of log10 of their start residuals
 * The paper has no counterpart: a measurement of this library's solver.   */
lbm_status lbm_poisson_stats(lbm_t* h, double* out);

/* Phase timing.  lbm_set_timing(h, 1) makes every following lbm_step record
 * CUDA events around its phases on the stream it runs on; lbm_get_timing
 * waits for them and writes, accumulated since timing was enabled:
 *   out[0] charge-density kernel ms    out[3] its launch count
 *   out[1] Poisson solve ms            out[4] Poisson iterations
 *   out[2] stream-collide kernel ms    out[5] its launch count
 *   out[6] kernels the library launched (all kinds)
 * out must hold 7 doubles.  lbm_set_timing(h, 0) stops recording and
 * clears the sums.                                                        */
lbm_status lbm_set_timing(lbm_t* h, int enable);
lbm_status lbm_get_timing(lbm_t* h, double* out);

/* The library's CUDA stream (a cudaStream_t), for callers that record
 * events around lbm_step on it.                                           */
void* lbm_stream(lbm_t* h);

/* Message of the last failure on h (or of the last failed lbm_create when
 * h is NULL).  Valid until the next call on h.                            */
const char* lbm_last_error(const lbm_t* h);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
