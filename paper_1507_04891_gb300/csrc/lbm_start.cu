// Start of each step's Poisson solve (every solver): the potential of the
// previous step advanced by an autoregression over the recent history of
// the solver's own (source, potential) pairs.
//
// The Poisson operator A is linear and fixed (the geometry does not change),
// so the change of the potential between steps answers the change of the
// source: A (psi(t) - psi(t-1)) = s(t) - s(t-1) up to the previous solves'
// residuals.  With the differences of the last K steps, D_j = s(t-j) -
// s(t-j-1) and P_j = psi(t-j) - psi(t-j-1), the coefficients c minimising
// || D_0 - sum_j c_j D_j ||_2 (D_0 = s(t) - s(t-1), known once the step's
// charge density is) give the start
//     psi_start = psi(t-1) + sum_j c_j P_j,
// whose residual is that least-squares residual (plus the previous solves'
// residuals carried along).  This is the projection of the new right-hand
// side onto the span of recent ones (the initial-guess technique of
// P. F. Fischer, Comput. Methods Appl. Mech. Engrg. 163 (1998) 193,
// "Projection techniques for iterative solution of Ax = b with successive
// right-hand sides"), written on differences so that it reproduces a
// potential constant in time exactly, and with the Gram matrix of the
// differences carried from step to step (each step adds one row, the inner
// products of D_0 with the stored differences).  Where the solve is short
// (the spectral solver: about one application a step) the start uses the
// coefficients of the previous step's fit, so that the fit of step t runs
// beside step t's solve instead of before it (the differences evolve
// slowly: in oracle runs of a charged porous box the start residual is the
// same to two digits with this one-step lag); before a multigrid or SOR
// solve, which takes milliseconds, the fit of the step itself comes first.
// Any start is valid: the solve still iterates to its tolerance from it.
//
// Storage: the previous source and the potential before the previous one
// (int64 fixed point), and rings of the last K differences of each as FP32
// (a difference is ~1e-3 of the field: FP32 keeps it to ~1e-10 of the
// field, far below the solver tolerance).  All bookkeeping (valid steps,
// ring position, Gram matrix, coefficients) lives in device memory, so the
// kernels replay unchanged inside the whole-step graphs.
#include <math.h>

#include <algorithm>

#include "lbm_internal.cuh"

namespace lbm_gb300 {
namespace {

constexpr int K = START_K;
// CTAs of the dot-product pass: a few cells per thread, FP32 per thread,
// FP64 across threads
constexpr int DOT_THREADS = 256;

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// state[0] steps of valid history since the last reset (0 .. K + 1)
// state[1] ring position of the current step (both rings; the fit advances
//          it after the step's passes have used it)
// state[2] autoregression terms of the coefficients in coef (0 .. K): the
//          next start uses this many
// state[3] terms the current step's start used (for the graph's decisions)
enum { ST_VALID = 0, ST_RING = 1, ST_TERMS = 2, ST_USED = 3 };
static_assert(ST_RING == START_RING_IDX, "ring position index shared with the charge pass");

// Least-squares coefficients over the first m stored differences:
// Cholesky of the Gram matrix G (K x K, row-major) with a relative diagonal
// load of 1e-10 against rounding, rows and columns from m on replaced by the
// identity so that every loop has the compile-time bound K (the factors stay
// in registers).  Returns false when a pivot is not positive or a
// coefficient is not finite.
__device__ bool solve_gram(const double* __restrict__ G, const double* __restrict__ rhs, int m,
                           double* c) {
  double L[K][K];
  double load = 0.0;
#pragma unroll
  for (int i = 0; i < K; ++i)
    if (i < m) load += G[i * K + i];
  load = 1e-10 * load / m + 1e-300;
  bool ok = true;
#pragma unroll
  for (int i = 0; i < K; ++i) {
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      double v;
      if (i < m && j < m) v = G[i * K + j] + (i == j ? load : 0.0);
      else v = (i == j) ? 1.0 : 0.0;
#pragma unroll
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
      if (i == j) {
        ok = ok && v > 0.0;
        L[i][i] = sqrt(v > 0.0 ? v : 1.0);
      } else {
        L[i][j] = v / L[j][j];
      }
    }
  }
  double y[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    double v = i < m ? rhs[i] : 0.0;
#pragma unroll
    for (int k = 0; k < i; ++k) v -= L[i][k] * y[k];
    y[i] = v / L[i][i];
  }
#pragma unroll
  for (int i = K - 1; i >= 0; --i) {
    double v = y[i];
#pragma unroll
    for (int k = i + 1; k < K; ++k) v -= L[k][i] * c[k];
    c[i] = v / L[i][i];
    ok = ok && isfinite(c[i]);
  }
  return ok;
}

// Pass 1 (one cell per thread): D_0 = s(t) - s(t-1) against D_0 and the
// stored D_1 .. D_K (ring slot of age j: (r - j) mod K); s(t) becomes the
// previous source and D_0 replaces D_K (slot r mod K).  Products in FP32
// (the differences carry ~7 significant digits of the field, far more than
// the start needs), summed per CTA in FP32 into part.
__global__ void __launch_bounds__(DOT_THREADS) k_start_dots(const int64_t* __restrict__ src,
                                                            int64_t* __restrict__ s_prev,
                                                            float* __restrict__ ring_d,
                                                            const int* __restrict__ state, int64_t N,
                                                            float* __restrict__ part) {
  const int r = state[ST_RING];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float acc[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) acc[j] = 0.f;
  if (i < N) {
    const int64_t s0 = src[i];
    const int64_t sp = s_prev[i];
    float dj[K + 1];
#pragma unroll
    for (int j = 1; j <= K; ++j) dj[j] = ring_d[(int64_t)((r - j + 2 * K) % K) * N + i];
    const float d0 = i64_to_f32(s0 - sp);
    acc[0] = d0 * d0;
#pragma unroll
    for (int j = 1; j <= K; ++j) acc[j] = d0 * dj[j];
    s_prev[i] = s0;
    ring_d[(int64_t)(r % K) * N + i] = d0;
  }
  __shared__ float red[DOT_THREADS / 32][K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    float v = acc[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][j] = v;
  }
  __syncthreads();
  if (threadIdx.x <= K) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < DOT_THREADS / 32; ++w) t += red[w][threadIdx.x];
    part[(int64_t)blockIdx.x * (K + 1) + threadIdx.x] = t;
  }
}

// Pass 2 (one CTA): the inner products g_j = <D_0, D_j> from the partials
// (compensated FP32 sums in a fixed order), the coefficients over the
// m = min(K, valid - 1) stored differences (fewer when the factorisation
// fails; the 5 x 5 factorisation is the only FP64 arithmetic), the Gram
// matrix of the next step (D_0 becomes D_1) and the bookkeeping.
__global__ void __launch_bounds__(256) k_start_solve(const float* __restrict__ part, int nctas,
                                                     double* __restrict__ gram,
                                                     float* __restrict__ coef,
                                                     int* __restrict__ state, int advance) {
  float hi[K + 1], lo[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) hi[j] = lo[j] = 0.f;
  for (int c0 = threadIdx.x; c0 < nctas; c0 += 8 * blockDim.x) {
    float x[8][K + 1];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = c0 + u * blockDim.x;
#pragma unroll
      for (int j = 0; j <= K; ++j) x[u][j] = c < nctas ? part[(int64_t)c * (K + 1) + j] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int j = 0; j <= K; ++j) two_sum_add(hi[j], lo[j], x[u][j]);
  }
#pragma unroll
  for (int j = 0; j <= K; ++j) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float oh = __shfl_down_sync(0xffffffffu, hi[j], off);
      const float ol = __shfl_down_sync(0xffffffffu, lo[j], off);
      two_sum_add(hi[j], lo[j], oh);
      lo[j] += ol;
    }
  }
  __shared__ float rh[8][K + 1], rl[8][K + 1];
  __shared__ double Gs[K * K];
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      rh[threadIdx.x >> 5][j] = hi[j];
      rl[threadIdx.x >> 5][j] = lo[j];
    }
  if (threadIdx.x < K * K) Gs[threadIdx.x] = gram[threadIdx.x];
  __syncthreads();
  if (threadIdx.x != 0) return;
  double g[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    float h = 0.f, l = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      two_sum_add(h, l, rh[w][j]);
      l += rl[w][j];
    }
    g[j] = (double)h + (double)l;
  }
  double G[K * K];
#pragma unroll
  for (int q = 0; q < K * K; ++q) G[q] = Gs[q];
  const int valid = state[ST_VALID];
  int m = min(K, valid - 1);
  double c[K];
#pragma unroll
  for (int j = 0; j < K; ++j) c[j] = 0.0;
  // rhs[j] = <D_0, D_{j+1}> = g[j + 1]; G[i][j] = <D_{i+1}, D_{j+1}>
  for (; m > 0; --m)
    if (solve_gram(G, g + 1, m, c)) break;
#pragma unroll
  for (int j = 0; j < K; ++j) coef[j] = (m > 0 && j < m) ? (float)c[j] : 0.0f;
  // the next step's Gram matrix: D_0 .. D_{K-2} become D_1 .. D_{K-1}
#pragma unroll
  for (int i = 1; i < K; ++i)
#pragma unroll
    for (int j = 1; j < K; ++j) gram[i * K + j] = G[(i - 1) * K + (j - 1)];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    gram[j] = g[j];
    gram[j * K] = g[j];
  }
  const int r = state[ST_RING];
  state[ST_TERMS] = max(m, 0);
  if (advance) state[ST_RING] = (r + 1) % K;
  state[ST_VALID] = min(valid + 1, K + 1);
}

// Pass 3: psi(t-1) + sum_j c_j P_j with P_1 = psi(t-1) - psi(t-2) (fresh)
// and P_j, j >= 2, from the ring (age j in slot (r - j + 1) mod K); psi(t-1)
// becomes the stored previous potential and P_1 replaces the slot of age
// K + 1 (slot r mod K).  The correction is formed in FP32 and rounded to the
// fixed-point grid; one too large for it keeps psi(t-1).
__global__ void __launch_bounds__(256) k_start_psi(int64_t* __restrict__ psi,
                                                   int64_t* __restrict__ psi_prev,
                                                   float* __restrict__ ring_p,
                                                   const float* __restrict__ coef,
                                                   int* __restrict__ state, int64_t N,
                                                   int advance) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int r = state[ST_RING];
  const int m = state[ST_TERMS];
  const int64_t a = psi[i];
  const float p1 = i64_to_f32(a - psi_prev[i]);
  if (m > 0) {
    float corr = coef[0] * p1;
#pragma unroll
    for (int j = 2; j <= K; ++j)
      if (j <= m) corr += coef[j - 1] * ring_p[(int64_t)((r - j + 1 + K) % K) * N + i];
    if (fabsf(corr) < 2.3e18f) psi[i] = a + f32_to_i64_rn(corr);
  }
  psi_prev[i] = a;
  ring_p[(int64_t)(r % K) * N + i] = p1;
}

// The step's bookkeeping after the start: the terms it used (for the
// graph's decisions) and, when it is the step's last pass, the ring
// position; after every thread of the start read them.  In a step graph it
// also writes whether the step speculates and clears the norm slot of the
// first application, which saves two graph nodes on the step's critical
// path.  The step does not speculate when the start used fewer than
// START_FULL_TERMS differences, or when the previous step needed more than
// the k applications baked into the graph (prev_iters: its count): steps
// that need more come in runs (the first steps after a restart, a change
// in the source the history does not follow), and a step that does not
// speculate only serialises its stream/collide behind the convergence
// test, while a failed speculation runs the stream/collide twice.
__global__ void k_start_mark(int* __restrict__ state, int advance, int* __restrict__ skip_out,
                             const int* __restrict__ prev_iters, int kbaked,
                             float* __restrict__ clear, int nclear) {
  if (threadIdx.x == 0) {
    const int used = state[ST_TERMS];
    state[ST_USED] = used;
    if (advance) state[ST_RING] = (state[ST_RING] + 1) % K;
    if (skip_out)
      *skip_out = (used < START_FULL_TERMS || (prev_iters && *prev_iters > kbaked)) ? 1 : 0;
  }
  for (int k = threadIdx.x; k < nclear; k += blockDim.x) clear[k] = 0.f;
}

// The charge scatter's source take fused with pass 1 (the step's source
// s(t) is the accumulator, and the source buffer still holds s(t-1), so the
// stored previous source is not needed: in a lattice with the scatter,
// k_start_dots never runs, and the first difference after a restart of the
// history is never used).  Node pairs over a grid of a few CTAs per SM:
// src = acc, acc = 0, D_0 = s(t) - s(t-1) into the ring slot r mod K, its
// products with D_0 .. D_K per CTA into part, and the exact 128-bit source
// total with the last CTA's work of k_src_take (FP64 total, mean over the
// fluid into mean_z, graph step counter, tot cleared).
// PSI (the spectral solver, whose start uses the previous step's fit): the
// start of the potential in the same pass (pass 3, as k_start_psi: the
// coefficients are known at the step's start), and the last CTA does
// k_start_mark's bookkeeping (terms used, the speculation flag, the first
// norm slot cleared; no ring advance: the fit advances it).
struct PsiArgs {
  int64_t* psi;
  int64_t* psi_prev;
  float* ring_p;
  const float* coef;
  int* skip_out;          // speculation flag of a step graph, or NULL
  const int* prev_iters;  // the previous step's applications (with skip_out)
  int kbaked;
  float* clear;           // norm slot to clear, or NULL
  int nclear;
};

template <bool PSI>
__global__ void __launch_bounds__(256) k_take_dots(int64_t* __restrict__ acc,
                                                   int64_t* __restrict__ src,
                                                   float* __restrict__ ring_d,
                                                   int* __restrict__ state, int64_t N,
                                                   float* __restrict__ part,
                                                   unsigned long long* tot, double* out,
                                                   long long* mean_z, int nz, double inv_nfluid,
                                                   uint32_t* step, const PsiArgs pa) {
  const int r = state[ST_RING];
  const int m = PSI ? state[ST_TERMS] : 0;
  const int64_t np = N / 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  longlong2* a2 = reinterpret_cast<longlong2*>(acc);
  longlong2* s2 = reinterpret_cast<longlong2*>(src);
  float2* rw = reinterpret_cast<float2*>(ring_d + (int64_t)(r % K) * N);
  float dp[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) dp[j] = 0.f;
  long long v = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < np; k += stride) {
    const longlong2 q = a2[k];
    const longlong2 o = s2[k];
    float2 dj[K + 1];
#pragma unroll
    for (int j = 1; j <= K; ++j)
      dj[j] = reinterpret_cast<const float2*>(ring_d + (int64_t)((r - j + 2 * K) % K) * N)[k];
    longlong2 pv = make_longlong2(0, 0), pp = make_longlong2(0, 0);
    float2 pj[K + 1];
    if (PSI) {
      pv = reinterpret_cast<const longlong2*>(pa.psi)[k];
      pp = reinterpret_cast<const longlong2*>(pa.psi_prev)[k];
#pragma unroll
      for (int j = 2; j <= K; ++j)
        pj[j] = j <= m ? reinterpret_cast<const float2*>(
                             pa.ring_p + (int64_t)((r - j + 1 + K) % K) * N)[k]
                       : make_float2(0.f, 0.f);
    }
    s2[k] = q;
    a2[k] = make_longlong2(0, 0);
    v += q.x + q.y;
    const float d0x = i64_to_f32(q.x - o.x), d0y = i64_to_f32(q.y - o.y);
    rw[k] = make_float2(d0x, d0y);
    dp[0] += d0x * d0x + d0y * d0y;
#pragma unroll
    for (int j = 1; j <= K; ++j) dp[j] += d0x * dj[j].x + d0y * dj[j].y;
    if (PSI) {
      const float p1x = i64_to_f32(pv.x - pp.x), p1y = i64_to_f32(pv.y - pp.y);
      longlong2 nv = pv;
      if (m > 0) {
        float cx = pa.coef[0] * p1x, cy = pa.coef[0] * p1y;
#pragma unroll
        for (int j = 2; j <= K; ++j)
          if (j <= m) {
            cx += pa.coef[j - 1] * pj[j].x;
            cy += pa.coef[j - 1] * pj[j].y;
          }
        if (fabsf(cx) < 2.3e18f) nv.x = pv.x + f32_to_i64_rn(cx);
        if (fabsf(cy) < 2.3e18f) nv.y = pv.y + f32_to_i64_rn(cy);
      }
      reinterpret_cast<longlong2*>(pa.psi)[k] = nv;
      reinterpret_cast<longlong2*>(pa.psi_prev)[k] = pv;
      reinterpret_cast<float2*>(pa.ring_p + (int64_t)(r % K) * N)[k] = make_float2(p1x, p1y);
    }
  }
  __shared__ float red[8][K + 1];
  __shared__ long long redv[8];
  __shared__ int last;
  __shared__ long long s_mean;
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    float t = dp[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][j] = t;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) redv[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x <= K) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w][threadIdx.x];
    part[(int64_t)blockIdx.x * (K + 1) + threadIdx.x] = t;
  }
  if (threadIdx.x == 0) {
    long long c = 0;
    for (int w = 0; w < 8; ++w) c += redv[w];
    const unsigned long long lo = (unsigned long long)c;
    const unsigned long long old = atomicAdd(&tot[0], lo);
    const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
    atomicAdd(&tot[1], carry + (c < 0 ? ~0ull : 0ull));
    __threadfence();
    last = atomicAdd(&tot[2], 1ull) == (unsigned long long)(gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long lo = atomicExch(&tot[0], 0ull);
    const unsigned long long hi = atomicExch(&tot[1], 0ull);
    atomicExch(&tot[2], 0ull);
    const __int128 t = (__int128)(((unsigned __int128)hi << 64) | (unsigned __int128)lo);
    const double td = (double)t;
    *out = td;
    s_mean = llrint(td * inv_nfluid);
    if (step) *step += 1u;
    if (PSI) {
      // every CTA read the terms and the ring position before counting itself
      const int used = state[ST_TERMS];
      state[ST_USED] = used;
      if (pa.skip_out)
        *pa.skip_out = (used < START_FULL_TERMS || (pa.prev_iters && *pa.prev_iters > pa.kbaked)) ? 1 : 0;
    }
  }
  if (PSI)
    for (int k = threadIdx.x; k < pa.nclear; k += blockDim.x) pa.clear[k] = 0.f;
  if (mean_z) {
    __syncthreads();
    for (int z = threadIdx.x; z < nz; z += blockDim.x) mean_z[z] = s_mean;
  }
}

}  // namespace

bool charge_dots_args(lbm_t* h, int ctas, DotsArgs* out) {
  StartHistory& H = h->start;
  if (!start_enabled(h) || ctas > H.part_ctas) return false;
  out->ring_d = H.ring_d;
  out->state = H.state;
  out->part = H.part;
  H.dots_done = true;
  H.dots_ctas = ctas;
  return true;
}

bool launch_take_dots(lbm_t* h, unsigned ctas, double inv_nfluid) {
  StartHistory& H = h->start;
  if (!start_enabled(h)) return false;
  ctas = std::min<unsigned>(ctas, (unsigned)H.ctas);
  // the spectral solver's start uses the previous step's fit, so the
  // start of the potential comes along (its bookkeeping in the last CTA)
  const bool psi = h->spec != nullptr;
  PsiArgs pa{};
  if (psi) {
    pa.psi = h->ps.psi[h->ps.cur];
    pa.psi_prev = H.psi_prev;
    pa.ring_p = H.ring_p;
    pa.coef = H.coef;
    pa.skip_out = h->mark_skip_out;
    pa.prev_iters = h->mark_prev_iters;
    pa.kbaked = h->mark_k;
    pa.clear = h->mark_clear;
    pa.nclear = h->mark_clear ? h->mark_nclear : 0;
    k_take_dots<true><<<ctas, 256, 0, h->st>>>(h->scat_acc, h->ps.src, H.ring_d, H.state, h->N,
                                               H.part, h->scat_tot, h->ps.dsum, h->charge_mean_z,
                                               h->cfg.nz, inv_nfluid, h->charge_step, pa);
  } else {
    k_take_dots<false><<<ctas, 256, 0, h->st>>>(h->scat_acc, h->ps.src, H.ring_d, H.state, h->N,
                                                H.part, h->scat_tot, h->ps.dsum, h->charge_mean_z,
                                                h->cfg.nz, inv_nfluid, h->charge_step, pa);
  }
  H.dots_done = true;
  H.dots_ctas = (int)ctas;
  H.psi_done = psi;
  H.psi_cleared = psi && h->mark_clear != nullptr;
  return true;
}

lbm_status start_setup(lbm_t* h) {
  start_free(h);
  StartHistory& H = h->start;
  const int64_t N = h->N;
  H.ctas = (int)nblk(N, DOT_THREADS);
  // partials for the largest grid that forms them: a charge pass of 64-thread CTAs
  H.part_ctas = std::max<int>(H.ctas, (int)nblk(N, 64));
  auto al = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return cudaMemset(*p, 0, bytes) == cudaSuccess;
  };
  const bool ok = al((void**)&H.s_prev, N * sizeof(int64_t)) &&
                  al((void**)&H.psi_prev, N * sizeof(int64_t)) &&
                  al((void**)&H.ring_d, (size_t)K * N * sizeof(float)) &&
                  al((void**)&H.ring_p, (size_t)K * N * sizeof(float)) &&
                  al((void**)&H.part, (size_t)H.part_ctas * (K + 1) * sizeof(float)) &&
                  al((void**)&H.gram, K * K * sizeof(double)) &&
                  al((void**)&H.coef, K * sizeof(float)) && al((void**)&H.state, 4 * sizeof(int));
  if (!ok) {
    start_free(h);
    h->err = "allocation of the Poisson start history failed";
    return LBM_ENOMEM;
  }
  int lo = 0, hi = 0;
  if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
      cudaStreamCreateWithPriority(&H.side, cudaStreamNonBlocking, lo) != cudaSuccess ||
      cudaEventCreateWithFlags(&H.fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&H.join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    start_free(h);
    h->err = "stream or event creation for the Poisson start failed";
    return LBM_ECUDA;
  }
  return LBM_OK;
}

void start_free(lbm_t* h) {
  StartHistory& H = h->start;
  cudaFree(H.s_prev);
  cudaFree(H.psi_prev);
  cudaFree(H.ring_d);
  cudaFree(H.ring_p);
  cudaFree(H.part);
  cudaFree(H.gram);
  cudaFree(H.coef);
  cudaFree(H.state);
  if (H.side) cudaStreamDestroy(H.side);
  if (H.fork) cudaEventDestroy(H.fork);
  if (H.join) cudaEventDestroy(H.join);
  H = StartHistory();
}

bool start_enabled(const lbm_t* h) {
  return h->start.state && !(h->cfg.flags & LBM_FLAG_NO_EXTRAPOLATION);
}

cudaError_t start_apply(lbm_t* h, bool last) {
  StartHistory& H = h->start;
  // without the start the history goes stale: it restarts when enabled again
  if (!start_enabled(h)) return start_reset(h);
  if (H.psi_done && !last) {
    // the step's source take applied the start (k_take_dots)
    H.psi_done = false;
    h->slot0_cleared = H.psi_cleared;
    return cudaSuccess;
  }
  H.psi_done = false;
  k_start_psi<<<nblk(h->N, 256), 256, 0, h->st>>>(h->ps.psi[h->ps.cur], H.psi_prev, H.ring_p, H.coef,
                                                   H.state, h->N, last ? 1 : 0);
  k_start_mark<<<1, 128, 0, h->st>>>(H.state, last ? 1 : 0, h->mark_skip_out, h->mark_prev_iters,
                                     h->mark_k, h->mark_clear, h->mark_clear ? h->mark_nclear : 0);
  h->slot0_cleared = h->mark_clear != nullptr;
  h->launches += 2;
  return cudaGetLastError();
}

cudaError_t start_fit(lbm_t* h, cudaStream_t st, bool last) {
  StartHistory& H = h->start;
  if (!start_enabled(h)) return cudaSuccess;
  int nparts = H.ctas;
  if (H.dots_done) {
    // the source take of this step formed the differences and products
    nparts = H.dots_ctas;
    H.dots_done = false;
  } else {
    k_start_dots<<<H.ctas, DOT_THREADS, 0, st>>>(h->ps.src, H.s_prev, H.ring_d, H.state, h->N,
                                                 H.part);
    ++h->launches;
  }
  k_start_solve<<<1, 256, 0, st>>>(H.part, nparts, H.gram, H.coef, H.state, last ? 1 : 0);
  ++h->launches;
  return cudaGetLastError();
}

cudaError_t start_step(lbm_t* h, bool lagged) {
  StartHistory& H = h->start;
  if (!lagged) {
    // the fit of this step, then the start from its coefficients
    cudaError_t e = start_fit(h, h->st, false);
    return e == cudaSuccess ? start_apply(h, true) : e;
  }
  cudaError_t e = start_apply(h, false);
  if (e != cudaSuccess || !start_enabled(h)) return e;
  // the fit of this step for the next start, beside the solve, on the
  // library's side stream
  e = cudaEventRecord(H.fork, h->st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(H.side, H.fork, 0);
  if (e == cudaSuccess) e = start_fit(h, H.side, true);
  if (e == cudaSuccess) e = cudaEventRecord(H.join, H.side);
  if (e == cudaSuccess) H.pending = true;
  return e;
}

cudaError_t start_join(lbm_t* h) {
  StartHistory& H = h->start;
  if (!H.pending) return cudaSuccess;
  H.pending = false;
  return cudaStreamWaitEvent(h->st, H.join, 0);
}

cudaError_t start_reset(lbm_t* h) {
  if (!h->start.state) return cudaSuccess;
  // no valid history, no terms for the next start
  return cudaMemsetAsync(h->start.state, 0, 3 * sizeof(int), h->st);
}

const int* start_terms_dev(const lbm_t* h) { return h->start.state ? h->start.state + ST_USED : nullptr; }

}  // namespace lbm_gb300
