// Learned initial guess for the Poisson solve (an addition to the paper's
// method; the plain solver still iterates to the same tolerance afterwards).
//
// A small periodic 3-D convolutional network maps the residual of the
// warm-start potential, r = s - A psi(t-1), to a correction:
//   x0 = r / sigma_r (sigma_r: rms of r over fluid cells), x1 = fluid mask
//   h_c = tanh(b_c + sum_{ci, o in 3x3x3} W1[c][ci][o] x_ci(cell + o))
//   y   = sum_{c, o} W2[c][o] h_c(cell + o),   delta psi = sigma_r y (fluid)
// Training pairs come from the solver itself: the initial residual of each
// step and the correction the plain solve found, A dpsi* = r.  The loss is
// the normalised residual left after the guess,
//   L = sum_fluid (x0 - A y)^2 / sum_fluid x0^2  = ||A (dpsi* - dpsi)||^2 / ||r||^2,
// with A the finite-volume operator of the Poisson solve.  Forward, backward
// (weight gradients as correlations) and Adam run in the kernels below;
// inference stores weights and activations in FP16 with FP32 accumulation.
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <random>
#include <string>
#include <vector>

#include "lbm_internal.cuh"

namespace lbm_gb300 {

struct NNet {
  int C = 8;                 // hidden channels
  static constexpr int CI = 2;
  int np = 0;                // parameter count
  float* p = nullptr;        // FP32 master parameters [W1 | b1 | W2]
  float* g = nullptr;        // gradients
  float* m = nullptr;        // Adam first moment
  float* v = nullptr;        // Adam second moment
  __half* ph = nullptr;      // FP16 copy for inference
  int adam_t = 0;
  float* x0 = nullptr;       // normalised residual (N)
  float* hid = nullptr;      // hidden activations (C x N), FP32 (training)
  __half* hid16 = nullptr;   // hidden activations (C x N), FP16 (inference)
  float* y = nullptr;        // output (N)
  float* res = nullptr;      // x0 - A y (N)
  float* gy = nullptr;       // dL/dy (N)
  float* ga = nullptr;       // dL/d(pre-activation) (C x N)
  double* red = nullptr;     // reductions [0] sum x0^2 [1] sum res^2
  double* hred = nullptr;    // pinned mirror
  // collected training residuals (ring buffer of full lattice fields)
  float* pool = nullptr;
  int cap = 0, count = 0, next = 0;
  bool collect = false, use = false;
  // inference on channel pairs: input packed per cell as (x0, fluid mask),
  // hidden activations stored per cell ([N][C] halves), and a host copy of
  // the parameters for the kernels' arguments (stale after training)
  __half2* xin = nullptr;
  std::vector<float> hp;
  bool hp_stale = true;
  // statistics of the guesses applied by the solver
  long long tried = 0, accepted = 0;
  double sum_ratio = 0.0;    // sum of residual ratio after/before over accepted guesses
};

namespace {

inline unsigned nb(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

struct Geo {
  int nx, ny, nz;
  int64_t N;
  const uint32_t* links;  // NULL: all fluid
};

__device__ __forceinline__ void xyz(int64_t i, const Geo& G, int& x, int& y, int& z) {
  const int64_t t = i / G.nx;
  x = (int)(i - t * G.nx);
  z = (int)(t / G.ny);
  y = (int)(t - (int64_t)z * G.ny);
}

__device__ __forceinline__ int64_t wrap_idx(const Geo& G, int x, int y, int z) {
  x = (x + G.nx) % G.nx;
  y = (y + G.ny) % G.ny;
  z = (z + G.nz) % G.nz;
  return ((int64_t)z * G.ny + y) * G.nx + x;
}

// The 27 neighbours of a cell from six wrapped axis offsets (no modulo per
// tap): offset of (dx, dy, dz) = ox[dx+1] + oy[dy+1] + oz[dz+1].
struct Taps {
  int ox[3], oy[3], oz[3];
};
__device__ __forceinline__ Taps taps_of(const Geo& G, int x, int y, int z) {
  Taps t;
  const int nxy = G.nx * G.ny;
  t.ox[0] = x == 0 ? G.nx - 1 : -1;
  t.ox[1] = 0;
  t.ox[2] = x == G.nx - 1 ? -(G.nx - 1) : 1;
  t.oy[0] = (y == 0 ? G.ny - 1 : -1) * G.nx;
  t.oy[1] = 0;
  t.oy[2] = (y == G.ny - 1 ? -(G.ny - 1) : 1) * G.nx;
  t.oz[0] = (z == 0 ? G.nz - 1 : -1) * nxy;
  t.oz[1] = 0;
  t.oz[2] = (z == G.nz - 1 ? -(G.nz - 1) : 1) * nxy;
  return t;
}

__device__ __forceinline__ bool fluid_at(const Geo& G, int64_t i) {
  return !G.links || !(G.links[i] & LINK_SOLID);
}

// (A v)_i over open faces (face open iff both cells fluid).
__device__ float apply_A(const float* v, const Geo& G, int64_t i, int x, int y, int z) {
  const float vc = v[i];
  float acc = 0.f;
  const int d[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int64_t j = wrap_idx(G, x + d[f][0], y + d[f][1], z + d[f][2]);
    if (j == i || !fluid_at(G, j)) continue;
    acc += vc - v[j];
  }
  return acc;
}

// x0 = r / sigma (fluid), 0 at wall nodes.  The residual of a trimmed
// multigrid box covers planes [zlo, zlo + nzb); with hx > 0 it is stored
// colour-split: cell (x, y, zb) of colour q = (x + y + zb) mod 2 at
// q H + (zb ny + y) hx + floor(x / 2), H = nzb ny hx.
// When xin is given, the same input packed for inference: (x0, fluid mask)
// as one FP16 pair per cell.
__global__ void k_nn_input(const float* __restrict__ r, int zlo, int nzb, int hx, float inv_sigma,
                           Geo G, float* __restrict__ x0, __half2* __restrict__ xin) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= G.N) return;
  const int64_t nxy = (int64_t)G.nx * G.ny;
  const int z = (int)(i / nxy);
  const bool fl = fluid_at(G, i);
  float v = 0.f;
  if (z >= zlo && z < zlo + nzb && fl) {
    int64_t j = i - (int64_t)zlo * nxy;
    if (hx > 0) {
      const int zb = z - zlo;
      const int64_t rem = i - (int64_t)z * nxy;
      const int y = (int)(rem / G.nx), x = (int)(rem - (int64_t)y * G.nx);
      const int64_t H = (int64_t)nzb * G.ny * hx;
      j = (((x + y + zb) & 1) ? H : 0) + ((int64_t)zb * G.ny + y) * hx + (x >> 1);
    }
    v = r[j] * inv_sigma;
  }
  x0[i] = v;
  if (xin) xin[i] = __floats2half2_rn(v, fl ? 1.f : 0.f);
}

__global__ void k_sum_sq(const float* __restrict__ a, int64_t n, double* out) {
  __shared__ float red[8];
  float v = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v += a[i] * a[i];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(out, t);
  }
}

// Layer 1 (FP32): hid[c][i] = tanh(b1[c] + sum W1[c][ci][o] x_ci(i + o)).
__global__ void __launch_bounds__(256) k_nn_layer1(const float* __restrict__ x0, const float* __restrict__ p,
                                                   int C, Geo G, float* __restrict__ hid) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= G.N) return;
  int x, y, z;
  xyz(i, G, x, y, z);
  float acc[16];
  for (int c = 0; c < C; ++c) acc[c] = p[C * 2 * 27 + c];
  for (int o = 0; o < 27; ++o) {
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    const int64_t j = wrap_idx(G, x + dx, y + dy, z + dz);
    const float a0 = x0[j];
    const float a1 = fluid_at(G, j) ? 1.f : 0.f;
    for (int c = 0; c < C; ++c) acc[c] += p[(c * 2 + 0) * 27 + o] * a0 + p[(c * 2 + 1) * 27 + o] * a1;
  }
  for (int c = 0; c < C; ++c) hid[(int64_t)c * G.N + i] = tanhf(acc[c]);
}

// Layer 2 (FP32): y = sum W2[c][o] hid_c(i + o), zero at wall nodes.
__global__ void __launch_bounds__(256) k_nn_layer2(const float* __restrict__ hid, const float* __restrict__ p,
                                                   int C, Geo G, float* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= G.N) return;
  if (!fluid_at(G, i)) {
    y[i] = 0.f;
    return;
  }
  int x, yy, z;
  xyz(i, G, x, yy, z);
  const float* W2 = p + C * 2 * 27 + C;
  float acc = 0.f;
  for (int o = 0; o < 27; ++o) {
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    const int64_t j = wrap_idx(G, x + dx, yy + dy, z + dz);
    for (int c = 0; c < C; ++c) acc += W2[c * 27 + o] * hid[(int64_t)c * G.N + j];
  }
  y[i] = acc;
}

// FP16 inference: the same two layers with half weights and activations,
// FP32 accumulation; writes the fixed-point correction sigma * y to dpsi.
__global__ void __launch_bounds__(256) k_nn_infer1(const float* __restrict__ x0, const __half* __restrict__ ph,
                                                   int C, Geo G, __half* __restrict__ hid) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= G.N) return;
  int x, y, z;
  xyz(i, G, x, y, z);
  const Taps T = taps_of(G, x, y, z);
  float acc[16];
  for (int c = 0; c < C; ++c) acc[c] = __half2float(ph[C * 2 * 27 + c]);
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    const int64_t j = i + T.ox[o % 3] + T.oy[(o / 3) % 3] + T.oz[o / 9];
    const __half a0 = __float2half(x0[j]);
    const __half a1 = __float2half(fluid_at(G, j) ? 1.f : 0.f);
    for (int c = 0; c < C; ++c)
      acc[c] += __half2float(__hfma(ph[(c * 2 + 0) * 27 + o], a0, __hmul(ph[(c * 2 + 1) * 27 + o], a1)));
  }
  for (int c = 0; c < C; ++c) hid[(int64_t)c * G.N + i] = __float2half(tanhf(acc[c]));
}

__global__ void __launch_bounds__(256) k_nn_infer2(const __half* __restrict__ hid, const __half* __restrict__ ph,
                                                   int C, Geo G, float sigma, float* __restrict__ dpsi) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= G.N) return;
  if (!fluid_at(G, i)) {
    dpsi[i] = 0.f;
    return;
  }
  int x, yy, z;
  xyz(i, G, x, yy, z);
  const Taps T = taps_of(G, x, yy, z);
  const __half* W2 = ph + C * 2 * 27 + C;
  float acc = 0.f;
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    const int64_t j = i + T.ox[o % 3] + T.oy[(o / 3) % 3] + T.oz[o / 9];
    for (int c = 0; c < C; ++c) acc += __half2float(__hmul(W2[c * 27 + o], hid[(int64_t)c * G.N + j]));
  }
  dpsi[i] = sigma * acc;
}

// Inference on channel pairs (C even, up to 16): the weights are kernel
// arguments (constant-bank operands of the FP16 pair FMAs, no loads), the
// input is one (x0, mask) pair per cell, the hidden activations one vector
// of C halves per cell.  Same network as k_nn_infer1/2: layer 1 with bias
// and tanh (the hardware's approximate tanh of FP16 pairs), layer 2
// accumulated per channel pair in FP16 and over pairs in FP32.
template <int C>
struct InferW {
  __half2 w1x[27][C / 2];  // W1[c][0][o] for c = 2k, 2k + 1
  __half2 w1m[27][C / 2];  // W1[c][1][o]
  __half2 b1[C / 2];
  __half2 w2[27][C / 2];   // W2[c][o]
};

template <int C>
struct HidVec {  // the C hidden halves of one cell
  __half2 v[C / 2];
};

__device__ __forceinline__ __half2 tanh_approx_h2(__half2 x) {
  uint32_t r;
  asm("tanh.approx.f16x2 %0, %1;" : "=r"(r) : "r"(*reinterpret_cast<const uint32_t*>(&x)));
  return *reinterpret_cast<const __half2*>(&r);
}

template <int C>
__global__ void __launch_bounds__(256) k_nn_fast1(const __half2* __restrict__ xin, const InferW<C> w,
                                                  Geo G, HidVec<C>* __restrict__ hid) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= G.N) return;
  int x, y, z;
  xyz(i, G, x, y, z);
  const Taps T = taps_of(G, x, y, z);
  __half2 acc[C / 2];
#pragma unroll
  for (int k = 0; k < C / 2; ++k) acc[k] = w.b1[k];
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    const __half2 v = xin[i + T.ox[o % 3] + T.oy[(o / 3) % 3] + T.oz[o / 9]];
    const __half2 xx = __low2half2(v), mm = __high2half2(v);
#pragma unroll
    for (int k = 0; k < C / 2; ++k) acc[k] = __hfma2(w.w1m[o][k], mm, __hfma2(w.w1x[o][k], xx, acc[k]));
  }
  HidVec<C> out;
#pragma unroll
  for (int k = 0; k < C / 2; ++k) out.v[k] = tanh_approx_h2(acc[k]);
  hid[i] = out;
}

// Layer 2 and the correction: dpsi = sigma y on fluid cells (kept for a
// revert), psi += round(dpsi) in fixed point.
template <int C>
__global__ void __launch_bounds__(256) k_nn_fast2(const HidVec<C>* __restrict__ hid, const InferW<C> w,
                                                  Geo G, float sigma, float* __restrict__ dpsi,
                                                  int64_t* __restrict__ psi) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= G.N) return;
  if (!fluid_at(G, i)) {
    dpsi[i] = 0.f;
    return;
  }
  int x, y, z;
  xyz(i, G, x, y, z);
  const Taps T = taps_of(G, x, y, z);
  __half2 acc[C / 2];
#pragma unroll
  for (int k = 0; k < C / 2; ++k) acc[k] = __float2half2_rn(0.f);
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    const HidVec<C> h = hid[i + T.ox[o % 3] + T.oy[(o / 3) % 3] + T.oz[o / 9]];
#pragma unroll
    for (int k = 0; k < C / 2; ++k) acc[k] = __hfma2(w.w2[o][k], h.v[k], acc[k]);
  }
  float yv = 0.f;
#pragma unroll
  for (int k = 0; k < C / 2; ++k) {
    const float2 f = __half22float2(acc[k]);
    yv += f.x + f.y;
  }
  const float d = sigma * yv;
  dpsi[i] = d;
  psi[i] += f32_to_i64_rn(d * PSI_SCALE_F);
}

template <int C>
InferW<C> infer_weights(const std::vector<float>& p) {
  InferW<C> w;
  const int b1 = C * 2 * 27, w2 = b1 + C;
  for (int o = 0; o < 27; ++o)
    for (int k = 0; k < C / 2; ++k) {
      const int c0 = 2 * k, c1 = 2 * k + 1;
      w.w1x[o][k] = __floats2half2_rn(p[(c0 * 2 + 0) * 27 + o], p[(c1 * 2 + 0) * 27 + o]);
      w.w1m[o][k] = __floats2half2_rn(p[(c0 * 2 + 1) * 27 + o], p[(c1 * 2 + 1) * 27 + o]);
      w.w2[o][k] = __floats2half2_rn(p[w2 + c0 * 27 + o], p[w2 + c1 * 27 + o]);
    }
  for (int k = 0; k < C / 2; ++k) w.b1[k] = __floats2half2_rn(p[b1 + 2 * k], p[b1 + 2 * k + 1]);
  return w;
}

template <int C>
cudaError_t fast_infer(NNet* n, const Geo& G, float sigma, int64_t* psi, cudaStream_t st) {
  const InferW<C> w = infer_weights<C>(n->hp);
  const unsigned b = nb(G.N, 256);
  HidVec<C>* hid = reinterpret_cast<HidVec<C>*>(n->hid16);
  k_nn_fast1<C><<<b, 256, 0, st>>>(n->xin, w, G, hid);
  k_nn_fast2<C><<<b, 256, 0, st>>>(hid, w, G, sigma, n->y, psi);
  return cudaGetLastError();
}

// res = x0 - A y and its squared sum.
__global__ void k_nn_res(const float* __restrict__ x0, const float* __restrict__ y, Geo G,
                         float* __restrict__ res, double* red) {
  __shared__ float sm[8];
  float v = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < G.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    float rv = 0.f;
    if (fluid_at(G, i)) {
      int x, yy, z;
      xyz(i, G, x, yy, z);
      rv = x0[i] - apply_A(y, G, i, x, yy, z);
    }
    res[i] = rv;
    v += rv * rv;
  }
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
    atomicAdd(red + 1, t);
  }
}

// dL/dy = -2 A res / sum x0^2 (A symmetric), zero at wall nodes.
__global__ void k_nn_gy(const float* __restrict__ res, Geo G, const double* __restrict__ red,
                        float* __restrict__ gy) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= G.N) return;
  float v = 0.f;
  if (fluid_at(G, i)) {
    int x, yy, z;
    xyz(i, G, x, yy, z);
    v = -2.0f / (float)red[0] * apply_A(res, G, i, x, yy, z);
  }
  gy[i] = v;
}

// dL/d(pre-activation)_c = (1 - h_c^2) sum_o W2[c][o] gy(i - o).
__global__ void __launch_bounds__(256) k_nn_ga(const float* __restrict__ gy, const float* __restrict__ hid,
                                               const float* __restrict__ p, int C, Geo G,
                                               float* __restrict__ ga) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= G.N) return;
  int x, yy, z;
  xyz(i, G, x, yy, z);
  const float* W2 = p + C * 2 * 27 + C;
  float acc[16];
  for (int c = 0; c < C; ++c) acc[c] = 0.f;
  for (int o = 0; o < 27; ++o) {
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    const int64_t j = wrap_idx(G, x - dx, yy - dy, z - dz);
    const float gj = gy[j];
    for (int c = 0; c < C; ++c) acc[c] += W2[c * 27 + o] * gj;
  }
  for (int c = 0; c < C; ++c) {
    const float h = hid[(int64_t)c * G.N + i];
    ga[(int64_t)c * G.N + i] = acc[c] * (1.f - h * h);
  }
}

// Weight gradients as correlations over cells:
//   g[W1 c,ci,o] = sum_i ga_c(i) x_ci(i + o),  g[b1 c] = sum_i ga_c(i),
//   g[W2 c,o]    = sum_i gy(i) hid_c(i + o).
// Each warp takes 32 cells at a time; every product is reduced across the
// warp and accumulated per CTA in shared memory, then added to g once per CTA.
__global__ void __launch_bounds__(256) k_nn_wgrad(const float* __restrict__ gy, const float* __restrict__ ga,
                                                  const float* __restrict__ hid,
                                                  const float* __restrict__ x0, int C, Geo G,
                                                  float* __restrict__ g) {
  extern __shared__ float acc[];  // np floats
  const int np = C * 2 * 27 + C + C * 27;
  for (int k = threadIdx.x; k < np; k += blockDim.x) acc[k] = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warps_total = gridDim.x * (blockDim.x >> 5);
  const int64_t nwork = (G.N + 31) / 32;
  auto wsum = [](float v) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
  };
  for (int64_t wk = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wk < nwork; wk += warps_total) {
    const int64_t i = wk * 32 + lane;
    const bool valid = i < G.N;
    int x = 0, yy = 0, z = 0;
    if (valid) xyz(i, G, x, yy, z);
    float gac[16];
    for (int c = 0; c < C; ++c) gac[c] = valid ? ga[(int64_t)c * G.N + i] : 0.f;
    const float gyi = valid ? gy[i] : 0.f;
    for (int c = 0; c < C; ++c) {
      const float t = wsum(gac[c]);
      if (lane == 0) acc[C * 2 * 27 + c] += t;
    }
    for (int o = 0; o < 27; ++o) {
      const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
      int64_t j = 0;
      float a0 = 0.f, a1 = 0.f;
      if (valid) {
        j = wrap_idx(G, x + dx, yy + dy, z + dz);
        a0 = x0[j];
        a1 = fluid_at(G, j) ? 1.f : 0.f;
      }
      for (int c = 0; c < C; ++c) {
        const float t0 = wsum(gac[c] * a0);
        const float t1 = wsum(gac[c] * a1);
        const float hv = valid ? hid[(int64_t)c * G.N + j] : 0.f;
        const float t2 = wsum(gyi * hv);
        if (lane == 0) {
          acc[(c * 2 + 0) * 27 + o] += t0;
          acc[(c * 2 + 1) * 27 + o] += t1;
          acc[C * 2 * 27 + C + c * 27 + o] += t2;
        }
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < np; k += blockDim.x) atomicAdd(g + k, acc[k]);
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1,
                       float b2, float eps, int t, __half* ph) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.f - b1) * gk;
  const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  const float mh = mk / (1.f - powf(b1, (float)t));
  const float vh = vk / (1.f - powf(b2, (float)t));
  p[k] -= lr * mh / (sqrtf(vh) + eps);
  ph[k] = __float2half(p[k]);
}

__global__ void k_to_half(const float* p, __half* ph, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) ph[k] = __float2half(p[k]);
}

// psi += round(dpsi) on fluid nodes (fixed point), or -= to revert.
__global__ void k_nn_apply(int64_t* psi, const float* __restrict__ dpsi, int64_t n, int sign) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t d = f32_to_i64_rn(dpsi[i] * PSI_SCALE_F);
  psi[i] += sign > 0 ? d : -d;
}

Geo geo_of(const lbm_t* h) {
  Geo G;
  G.nx = h->cfg.nx;
  G.ny = h->cfg.ny;
  G.nz = h->cfg.nz;
  G.N = h->N;
  G.links = h->links;
  return G;
}

// Forward + loss (+ backward into nn.g when grad) on the field in nn.x0.
// Returns the loss.
lbm_status loss_grad(lbm_t* h, bool grad, double* loss) {
  NNet& n = *h->nn;
  const Geo G = geo_of(h);
  const unsigned b = nb(G.N, 256);
  const unsigned gr = (unsigned)std::min<int64_t>(b, h->grid_cap);
  LBM_CUDA_TRY(h, cudaMemsetAsync(n.red, 0, 2 * sizeof(double), h->st));
  k_sum_sq<<<gr, 256, 0, h->st>>>(n.x0, G.N, n.red);
  k_nn_layer1<<<b, 256, 0, h->st>>>(n.x0, n.p, n.C, G, n.hid);
  k_nn_layer2<<<b, 256, 0, h->st>>>(n.hid, n.p, n.C, G, n.y);
  k_nn_res<<<gr, 256, 0, h->st>>>(n.x0, n.y, G, n.res, n.red);
  h->launches += 4;
  if (grad) {
    k_nn_gy<<<b, 256, 0, h->st>>>(n.res, G, n.red, n.gy);
    k_nn_ga<<<b, 256, 0, h->st>>>(n.gy, n.hid, n.p, n.C, G, n.ga);
    LBM_CUDA_TRY(h, cudaMemsetAsync(n.g, 0, n.np * sizeof(float), h->st));
    // CTAs of one warp: lane 0 alone writes the CTA's shared accumulators
    k_nn_wgrad<<<(unsigned)std::min<int64_t>(nb(G.N, 32), 152), 32, n.np * sizeof(float), h->st>>>(
        n.gy, n.ga, n.hid, n.x0, n.C, G, n.g);
    h->launches += 3;
  }
  LBM_CUDA_TRY(h, cudaGetLastError());
  LBM_CUDA_TRY(h, cudaMemcpyAsync(n.hred, n.red, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  *loss = n.hred[0] > 0 ? n.hred[1] / n.hred[0] : 0.0;
  return LBM_OK;
}

}  // namespace

void nn_free(lbm_t* h) {
  NNet* n = h->nn;
  if (!n) return;
  cudaFree(n->p);
  cudaFree(n->g);
  cudaFree(n->m);
  cudaFree(n->v);
  cudaFree(n->ph);
  cudaFree(n->x0);
  cudaFree(n->hid);
  cudaFree(n->hid16);
  cudaFree(n->xin);
  cudaFree(n->y);
  cudaFree(n->res);
  cudaFree(n->gy);
  cudaFree(n->ga);
  cudaFree(n->red);
  cudaFree(n->pool);
  if (n->hred) cudaFreeHost(n->hred);
  delete n;
  h->nn = nullptr;
}

lbm_status nn_init(lbm_t* h, int hidden, uint64_t seed) {
  if (hidden < 1 || hidden > 16) {
    h->err = "hidden channels must be in 1..16";
    return LBM_EINVAL;
  }
  nn_free(h);
  NNet* n = new NNet();
  h->nn = n;
  n->C = hidden;
  n->np = hidden * 2 * 27 + hidden + hidden * 27;
  const int64_t N = h->N;
  bool ok = cudaMalloc(&n->p, n->np * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->g, n->np * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->m, n->np * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->v, n->np * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->ph, n->np * sizeof(__half)) == cudaSuccess &&
            cudaMalloc(&n->x0, N * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->hid, (size_t)hidden * N * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->hid16, (size_t)hidden * N * sizeof(__half)) == cudaSuccess &&
            cudaMalloc(&n->xin, N * sizeof(__half2)) == cudaSuccess &&
            cudaMalloc(&n->y, N * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->res, N * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->gy, N * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->ga, (size_t)hidden * N * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->red, 2 * sizeof(double)) == cudaSuccess &&
            cudaMallocHost(&n->hred, 2 * sizeof(double)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    nn_free(h);
    h->err = "network allocation failed";
    return LBM_ENOMEM;
  }
  // He-style uniform initialisation, seeded; small output layer
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<float> U(-1.f, 1.f);
  std::vector<float> p(n->np, 0.f);
  const float a1 = sqrtf(3.f / (2.f * 27.f)), a2 = 0.1f * sqrtf(3.f / (hidden * 27.f));
  for (int k = 0; k < hidden * 2 * 27; ++k) p[k] = a1 * U(rng);
  for (int k = 0; k < hidden * 27; ++k) p[hidden * 2 * 27 + hidden + k] = a2 * U(rng);
  LBM_CUDA_TRY(h, cudaMemcpy(n->p, p.data(), n->np * sizeof(float), cudaMemcpyHostToDevice));
  LBM_CUDA_TRY(h, cudaMemset(n->m, 0, n->np * sizeof(float)));
  LBM_CUDA_TRY(h, cudaMemset(n->v, 0, n->np * sizeof(float)));
  k_to_half<<<nb(n->np, 256), 256, 0, h->st>>>(n->p, n->ph, n->np);
  LBM_CUDA_TRY(h, cudaGetLastError());
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return LBM_OK;
}

lbm_status nn_collect(lbm_t* h, int capacity) {
  NNet* n = h->nn;
  if (!n) {
    h->err = "network not initialised";
    return LBM_EINVAL;
  }
  if (capacity <= 0) {
    n->collect = false;
    return LBM_OK;
  }
  if (capacity != n->cap) {
    cudaFree(n->pool);
    n->pool = nullptr;
    if (cudaMalloc(&n->pool, (size_t)capacity * h->N * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      n->cap = 0;
      h->err = "training pool allocation failed";
      return LBM_ENOMEM;
    }
    n->cap = capacity;
    n->count = n->next = 0;
  }
  n->collect = true;
  return LBM_OK;
}

// Called by the solver with the initial residual (FP32, box-indexed: planes
// [zlo, zlo + nzb); colour-split when hx > 0) and its rms.  Stores it when collecting; applies the
// learned correction when in use.  Returns the relative change of the
// residual norm the caller must verify (the caller reverts on failure).
lbm_status nn_before_solve(lbm_t* h, const float* r, int zlo, int nzb, int hx, double rms,
                           bool* applied, float** dpsi_out) {
  *applied = false;
  NNet* n = h->nn;
  if (!n || rms <= 0.0 || !isfinite(rms)) return LBM_OK;
  const Geo G = geo_of(h);
  const unsigned b = nb(G.N, 256);
  const bool fast = n->C == 2 || n->C == 4 || n->C == 8 || n->C == 16;
  if (n->collect || n->use) {
    k_nn_input<<<b, 256, 0, h->st>>>(r, zlo, nzb, hx, (float)(1.0 / rms), G, n->x0,
                                      n->use && fast ? n->xin : nullptr);
    ++h->launches;
  }
  if (n->collect && n->cap > 0) {
    LBM_CUDA_TRY(h, cudaMemcpyAsync(n->pool + (size_t)n->next * G.N, n->x0, G.N * sizeof(float),
                                    cudaMemcpyDeviceToDevice, h->st));
    n->next = (n->next + 1) % n->cap;
    n->count = std::min(n->count + 1, n->cap);
  }
  if (n->use) {
    if (fast) {
      if (n->hp_stale) {
        n->hp.resize(n->np);
        LBM_CUDA_TRY(h, cudaMemcpyAsync(n->hp.data(), n->p, n->np * sizeof(float), cudaMemcpyDeviceToHost,
                                        h->st));
        LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
        n->hp_stale = false;
      }
      int64_t* psi = h->ps.psi[h->ps.cur];
      cudaError_t e = n->C == 2   ? fast_infer<2>(n, G, (float)rms, psi, h->st)
                      : n->C == 4 ? fast_infer<4>(n, G, (float)rms, psi, h->st)
                      : n->C == 8 ? fast_infer<8>(n, G, (float)rms, psi, h->st)
                                  : fast_infer<16>(n, G, (float)rms, psi, h->st);
      LBM_CUDA_TRY(h, e);
      h->launches += 2;
    } else {
      k_nn_infer1<<<b, 256, 0, h->st>>>(n->x0, n->ph, n->C, G, n->hid16);
      k_nn_infer2<<<b, 256, 0, h->st>>>(n->hid16, n->ph, n->C, G, (float)rms, n->y);
      k_nn_apply<<<b, 256, 0, h->st>>>(h->ps.psi[h->ps.cur], n->y, G.N, +1);
      h->launches += 3;
    }
    LBM_CUDA_TRY(h, cudaGetLastError());
    *applied = true;
    *dpsi_out = n->y;
    ++n->tried;
  }
  return LBM_OK;
}

lbm_status nn_revert(lbm_t* h, const float* dpsi) {
  k_nn_apply<<<nb(h->N, 256), 256, 0, h->st>>>(h->ps.psi[h->ps.cur], dpsi, h->N, -1);
  ++h->launches;
  LBM_CUDA_TRY(h, cudaGetLastError());
  return LBM_OK;
}

bool nn_active(const lbm_t* h) { return h->nn && (h->nn->collect || h->nn->use); }

void nn_stats(const lbm_t* h, double* out) {
  const NNet* n = h->nn;
  out[0] = n ? (double)n->tried : 0.0;
  out[1] = n ? (double)n->accepted : 0.0;
  out[2] = (n && n->accepted) ? n->sum_ratio / n->accepted : 0.0;
  out[3] = n ? (double)n->count : 0.0;
  out[4] = n ? (double)n->np : 0.0;
}

lbm_status nn_set_use(lbm_t* h, int enable) {
  if (!h->nn) {
    h->err = "network not initialised";
    return LBM_EINVAL;
  }
  h->nn->use = enable != 0;
  return LBM_OK;
}

void nn_record(lbm_t* h, double ratio) {
  if (!h->nn) return;
  h->nn->accepted += 1;
  h->nn->sum_ratio += ratio;
}

lbm_status nn_train(lbm_t* h, int epochs, double lr, double* losses) {
  NNet* n = h->nn;
  if (!n || n->count == 0) {
    h->err = "no network or no collected training residuals";
    return LBM_EINVAL;
  }
  for (int e = 0; e < epochs; ++e) {
    double tot = 0.0;
    for (int k = 0; k < n->count; ++k) {
      LBM_CUDA_TRY(h, cudaMemcpyAsync(n->x0, n->pool + (size_t)k * h->N, h->N * sizeof(float),
                                      cudaMemcpyDeviceToDevice, h->st));
      double L = 0.0;
      lbm_status s = loss_grad(h, true, &L);
      if (s != LBM_OK) return s;
      tot += L;
      ++n->adam_t;
      k_adam<<<nb(n->np, 256), 256, 0, h->st>>>(n->p, n->g, n->m, n->v, n->np, (float)lr, 0.9f,
                                                0.999f, 1e-8f, n->adam_t, n->ph);
      n->hp_stale = true;
      ++h->launches;
      LBM_CUDA_TRY(h, cudaGetLastError());
    }
    if (losses) losses[e] = tot / n->count;
  }
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return LBM_OK;
}

lbm_status nn_loss_grad_host(lbm_t* h, const float* x0_host, double* loss, float* grad_host) {
  NNet* n = h->nn;
  if (!n) {
    h->err = "network not initialised";
    return LBM_EINVAL;
  }
  LBM_CUDA_TRY(h, cudaMemcpyAsync(n->x0, x0_host, h->N * sizeof(float), cudaMemcpyHostToDevice, h->st));
  lbm_status s = loss_grad(h, grad_host != nullptr, loss);
  if (s != LBM_OK) return s;
  if (grad_host) {
    LBM_CUDA_TRY(h, cudaMemcpy(grad_host, n->g, n->np * sizeof(float), cudaMemcpyDeviceToHost));
  }
  return LBM_OK;
}

lbm_status nn_infer_host(lbm_t* h, const float* x0_host, float* y_host) {
  NNet* n = h->nn;
  if (!n) {
    h->err = "network not initialised";
    return LBM_EINVAL;
  }
  const Geo G = geo_of(h);
  const unsigned b = nb(G.N, 256);
  const bool fast = n->C == 2 || n->C == 4 || n->C == 8 || n->C == 16;
  LBM_CUDA_TRY(h, cudaMemcpyAsync(n->x0, x0_host, h->N * sizeof(float), cudaMemcpyHostToDevice, h->st));
  // the same packing as for a solver residual (sigma 1, every plane)
  k_nn_input<<<b, 256, 0, h->st>>>(n->x0, 0, h->cfg.nz, 0, 1.0f, G, n->x0, fast ? n->xin : nullptr);
  ++h->launches;
  if (fast) {
    int64_t* scratch = nullptr;
    LBM_CUDA_TRY(h, cudaMalloc(&scratch, h->N * sizeof(int64_t)));
    cudaMemsetAsync(scratch, 0, h->N * sizeof(int64_t), h->st);
    if (n->hp_stale) {
      n->hp.resize(n->np);
      cudaMemcpyAsync(n->hp.data(), n->p, n->np * sizeof(float), cudaMemcpyDeviceToHost, h->st);
      cudaStreamSynchronize(h->st);
      n->hp_stale = false;
    }
    cudaError_t e = n->C == 2   ? fast_infer<2>(n, G, 1.0f, scratch, h->st)
                    : n->C == 4 ? fast_infer<4>(n, G, 1.0f, scratch, h->st)
                    : n->C == 8 ? fast_infer<8>(n, G, 1.0f, scratch, h->st)
                                : fast_infer<16>(n, G, 1.0f, scratch, h->st);
    cudaStreamSynchronize(h->st);
    cudaFree(scratch);
    LBM_CUDA_TRY(h, e);
    h->launches += 2;
  } else {
    k_nn_infer1<<<b, 256, 0, h->st>>>(n->x0, n->ph, n->C, G, n->hid16);
    k_nn_infer2<<<b, 256, 0, h->st>>>(n->hid16, n->ph, n->C, G, 1.0f, n->y);
    h->launches += 2;
    LBM_CUDA_TRY(h, cudaGetLastError());
  }
  LBM_CUDA_TRY(h, cudaMemcpyAsync(y_host, n->y, h->N * sizeof(float), cudaMemcpyDeviceToHost, h->st));
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return LBM_OK;
}

lbm_status nn_params(lbm_t* h, float* get, const float* set, int* np) {
  NNet* n = h->nn;
  if (!n) {
    h->err = "network not initialised";
    return LBM_EINVAL;
  }
  if (np) *np = n->np;
  if (get) LBM_CUDA_TRY(h, cudaMemcpy(get, n->p, n->np * sizeof(float), cudaMemcpyDeviceToHost));
  if (set) {
    LBM_CUDA_TRY(h, cudaMemcpy(n->p, set, n->np * sizeof(float), cudaMemcpyHostToDevice));
    n->hp_stale = true;
    k_to_half<<<nb(n->np, 256), 256, 0, h->st>>>(n->p, n->ph, n->np);
    LBM_CUDA_TRY(h, cudaGetLastError());
    LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  }
  return LBM_OK;
}

}  // namespace lbm_gb300
