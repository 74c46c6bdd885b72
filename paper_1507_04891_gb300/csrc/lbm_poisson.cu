// Poisson solve for the mean-field potential of the charged mixture:
//   nabla^2 psi = -4 pi l_B sum_alpha z^alpha n^alpha          (Eq. Poisson)
// with the surface-charge Neumann condition at wall faces.  Discretised by
// finite volumes on the lattice cells:
//   (A psi)_i = sum_{open faces j} (psi_i - psi_j) = s_i - <s>,
//   s_i = 4 pi l_B (rho_e,i + w_i)
// (w_i: wall charge handed to cell i).  The mean <s> over fluid cells is
// removed (neutralising background), which makes the periodic / Neumann
// problem solvable.
//
// psi is a 64-bit fixed-point field (see lbm_internal.cuh), so the residual
// s - A psi is exact integer arithmetic and the 1e-8 relative residual is
// reached without FP64 arithmetic.  Two solvers work on FP32 corrections:
//   - geometric multigrid used for defect correction: cell-centred V(2,2)
//     cycles, red-black Gauss-Seidel smoothing, restriction by summing the
//     8 children, trilinear prolongation, coarse face conductances
//     (sum of the crossing fine ones) * h_fine/h_coarse, one-CTA coarsest
//     solve;
//   - red-black SOR directly on the fixed-point psi.
// Convergence is tested on the FP64 norm ratio ||s - A psi||_2 / ||s||_2.
#include <math.h>

#include <algorithm>
#include <vector>

#include "lbm_internal.cuh"

namespace lbm_gb300 {
namespace {

struct Box {
  int nx, ny, nzb, zlo, perz;
  int64_t nxy;
};

// open-face bits from the link word: bit 2 of the link word = +x neighbour
// is a wall node, 1 = -x, 4 = +y, 3 = -y, 6 = +z, 5 = -z.
__device__ __forceinline__ bool open_face(uint32_t lk, int face) {
  // face: 0 +x, 1 -x, 2 +y, 3 -y, 4 +z, 5 -z
  const int bit = (face & 1) ? face : face + 2;  // 0->2, 1->1, 2->4, 3->3, 4->6, 5->5
  return !((lk >> bit) & 1u);
}

// box-cell neighbour offsets (periodic x, y; z periodic only if perz)
__device__ __forceinline__ void box_nbr(const Box& b, int x, int y, int z,
                                        int (&d)[6]) {
  d[0] = (x == b.nx - 1) ? -(b.nx - 1) : 1;
  d[1] = (x == 0) ? (b.nx - 1) : -1;
  d[2] = ((y == b.ny - 1) ? -(b.ny - 1) : 1) * b.nx;
  d[3] = ((y == 0) ? (b.ny - 1) : -1) * b.nx;
  const int nxy = b.nx * b.ny;
  if (b.perz) {
    d[4] = ((z == b.nzb - 1) ? -(b.nzb - 1) : 1) * nxy;
    d[5] = ((z == 0) ? (b.nzb - 1) : -1) * nxy;
  } else {
    d[4] = (z == b.nzb - 1) ? 0 : nxy;
    d[5] = (z == 0) ? 0 : -nxy;
  }
}

__device__ __forceinline__ void box_xyz(uint32_t c, const Box& b, int& x,
                                        int& y, int& z) {
  const uint32_t t = c / (uint32_t)b.nx;
  x = (int)(c - t * (uint32_t)b.nx);
  z = (int)(t / (uint32_t)b.ny);
  y = (int)(t - (uint32_t)z * (uint32_t)b.ny);
}

__device__ __forceinline__ int64_t fx_of(float e) {
  return f32_to_i64_rn(e * PSI_SCALE_F);
}

// Residual on the fine box, r = s - <s> - A psi, exact in 64-bit integers.
// Writes r (FP32) to rhs and block sums of r^2 and (s - <s>)^2 (fixed-point
// units) to dsum[1], dsum[2].
template <bool WALLS>
__global__ void __launch_bounds__(256) k_res0(
    const int64_t* __restrict__ psi, const int64_t* __restrict__ src,
    const uint32_t* __restrict__ links, float* __restrict__ r, double* dsum,
    Box b, int64_t nbox, double inv_nfluid, const int* __restrict__ label,
    const long long* __restrict__ comp_mean) {
  __shared__ long long s_mean;
  __shared__ float red_r[8], red_s[8];
  if (threadIdx.x == 0) s_mean = llrint(dsum[0] * inv_nfluid);
  __syncthreads();
  float rr = 0.f, ss = 0.f;
  // grid-stride loop over a grid capped at a few CTAs per SM: one pair of
  // FP64 atomics per CTA instead of per 256 cells
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < (uint32_t)nbox;
       c += gridDim.x * blockDim.x) {
    const int64_t i = (int64_t)c + (int64_t)b.zlo * b.nxy;  // lattice node
    uint32_t lk = 0;
    if (WALLS) lk = links[i];
    if (WALLS && (lk & LINK_SOLID)) {
      r[c] = 0.f;
      continue;
    }
    int x, y, z;
    box_xyz(c, b, x, y, z);
    int d[6];
    box_nbr(b, x, y, z, d);
    const int64_t pc = psi[i];
    int64_t Ap = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      if (WALLS && !open_face(lk, f)) continue;
      Ap += pc - psi[i + d[f]];
    }
    const int64_t sfx = src[i] - (label ? comp_mean[label[i]] : (int64_t)s_mean);
    const float rf = i64_to_f32(sfx - Ap);
    r[c] = rf * PSI_INV_SCALE_F;
    rr += rf * rf;
    const float sf = i64_to_f32(sfx);
    ss += sf * sf;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    rr += __shfl_down_sync(0xffffffffu, rr, off);
    ss += __shfl_down_sync(0xffffffffu, ss, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red_r[threadIdx.x >> 5] = rr;
    red_s[threadIdx.x >> 5] = ss;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, ts = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tr += (double)red_r[w];
      ts += (double)red_s[w];
    }
    atomicAdd(dsum + 1, tr);
    atomicAdd(dsum + 2, ts);
  }
}

// Cell of colour `color` handled by thread t when the x extent is even:
// every x row holds nx/2 cells of each colour.  With an odd x extent every
// thread takes one cell and skips the other colour.
__device__ __forceinline__ bool rb_cell(uint32_t t, int nx, int ny, int64_t n,
                                        int color, bool compact, uint32_t& c,
                                        int& x, int& y, int& z) {
  if (compact) {
    const uint32_t half = (uint32_t)nx >> 1;
    if (t >= (uint32_t)(n >> 1)) return false;
    const uint32_t row = t / half;
    const uint32_t k = t - row * half;
    z = (int)(row / (uint32_t)ny);
    y = (int)(row - (uint32_t)z * (uint32_t)ny);
    x = (int)(2 * k) + ((y + z + color) & 1);
    c = row * (uint32_t)nx + (uint32_t)x;
    return true;
  }
  if (t >= (uint32_t)n) return false;
  c = t;
  const uint32_t q = t / (uint32_t)nx;
  x = (int)(t - q * (uint32_t)nx);
  z = (int)(q / (uint32_t)ny);
  y = (int)(q - (uint32_t)z * (uint32_t)ny);
  return ((x + y + z) & 1) == color;
}

// Red-black Gauss-Seidel on the fine box for A e = r (FP32).  With APPLY
// (the last sweep of a V-cycle) each cell also writes its final correction
// into the other potential buffer: psi_out = psi_in + round(e).
template <bool WALLS, bool APPLY>
__global__ void __launch_bounds__(256) k_smooth0(
    float* __restrict__ e, const float* __restrict__ r,
    const uint32_t* __restrict__ links, Box b, int64_t nbox, int color,
    int compact, const int64_t* __restrict__ psi_in, int64_t* __restrict__ psi_out) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t c;
  int x, y, z;
  if (!rb_cell(t, b.nx, b.ny, nbox, color, compact, c, x, y, z)) return;
  const int64_t i = (int64_t)c + (int64_t)b.zlo * b.nxy;
  uint32_t lk = 0;
  if (WALLS) {
    lk = links[i];
    if (lk & LINK_SOLID) return;
  }
  int d[6];
  box_nbr(b, x, y, z, d);
  float sum = r[c];
  int cnt = 0;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    if (WALLS && !open_face(lk, f)) continue;
    sum += e[(int64_t)c + d[f]];
    ++cnt;
  }
  float ev = e[c];
  if (cnt > 0) {
    ev = sum / (float)cnt;
    e[c] = ev;
  }
  if (APPLY) psi_out[i] = psi_in[i] + fx_of(ev);
}

// Red-black SOR directly on the fixed-point psi (in place).
template <bool WALLS>
__global__ void __launch_bounds__(256) k_sor0(
    int64_t* __restrict__ psi, const int64_t* __restrict__ src,
    const uint32_t* __restrict__ links, const double* dsum, Box b,
    int64_t nbox, double inv_nfluid, int color, float omega, const int* __restrict__ label,
    const long long* __restrict__ comp_mean) {
  __shared__ long long s_mean;
  if (threadIdx.x == 0) s_mean = llrint(dsum[0] * inv_nfluid);
  __syncthreads();
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= (uint32_t)nbox) return;
  int x, y, z;
  box_xyz(c, b, x, y, z);
  if (((x + y + z) & 1) != color) return;
  const int64_t i = (int64_t)c + (int64_t)b.zlo * b.nxy;
  uint32_t lk = 0;
  if (WALLS) {
    lk = links[i];
    if (lk & LINK_SOLID) return;
  }
  int d[6];
  box_nbr(b, x, y, z, d);
  const int64_t pc = psi[i];
  int64_t Ap = 0;
  int cnt = 0;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    if (WALLS && !open_face(lk, f)) continue;
    Ap += pc - psi[i + d[f]];
    ++cnt;
  }
  if (cnt == 0) return;
  const int64_t rfx = src[i] - (label ? comp_mean[label[i]] : (int64_t)s_mean) - Ap;
  psi[i] = pc + f32_to_i64_rn(omega * i64_to_f32(rfx) / (float)cnt);
}

struct CL {  // coarse level view
  int nx, ny, nz;
  int64_t n;
  int px, py, pz;
};

__device__ __forceinline__ void cl_xyz(uint32_t c, const CL& l, int& x, int& y,
                                       int& z) {
  const uint32_t t = c / (uint32_t)l.nx;
  x = (int)(c - t * (uint32_t)l.nx);
  z = (int)(t / (uint32_t)l.ny);
  y = (int)(t - (uint32_t)z * (uint32_t)l.ny);
}

// + and - neighbour offsets on a coarse level (0 when not periodic and at
// the boundary: the conductance there is zero anyway).
__device__ __forceinline__ void cl_nbr(const CL& l, int x, int y, int z,
                                       int (&d)[6]) {
  const int nxy = l.nx * l.ny;
  d[0] = (x == l.nx - 1) ? (l.px ? -(l.nx - 1) : 0) : 1;
  d[1] = (x == 0) ? (l.px ? l.nx - 1 : 0) : -1;
  d[2] = ((y == l.ny - 1) ? (l.py ? -(l.ny - 1) : 0) : 1) * l.nx;
  d[3] = ((y == 0) ? (l.py ? l.ny - 1 : 0) : -1) * l.nx;
  d[4] = ((z == l.nz - 1) ? (l.pz ? -(l.nz - 1) : 0) : 1) * nxy;
  d[5] = ((z == 0) ? (l.pz ? l.nz - 1 : 0) : -1) * nxy;
}

// Neighbour sum sum_faces K x_nb on a coarse level.  The + face of a cell
// carries K[axis][c]; the - face the + conductance of the - neighbour, which
// does not exist at the low end of a non-periodic axis.
__device__ __forceinline__ float cl_nsum(const float* __restrict__ x,
                                         const float* __restrict__ K, const CL& l,
                                         uint32_t c, int xx, int yy, int zz,
                                         const int (&d)[6]) {
  const int64_t n = l.n;
  float s = 0.f;
  s += K[c] * x[(int64_t)c + d[0]];
  s += K[n + c] * x[(int64_t)c + d[2]];
  s += K[2 * n + c] * x[(int64_t)c + d[4]];
  if (l.px || xx > 0) s += K[(int64_t)c + d[1]] * x[(int64_t)c + d[1]];
  if (l.py || yy > 0) s += K[n + (int64_t)c + d[3]] * x[(int64_t)c + d[3]];
  if (l.pz || zz > 0) s += K[2 * n + (int64_t)c + d[5]] * x[(int64_t)c + d[5]];
  return s;
}

__device__ __forceinline__ void gs_cell(float* x, const float* rhs, const float* K,
                                        const float* Dinv, const CL& l, uint32_t c,
                                        int xx, int yy, int zz) {
  const float di = Dinv[c];
  if (di == 0.f) return;
  int d[6];
  cl_nbr(l, xx, yy, zz, d);
  x[c] = di * (rhs[c] + cl_nsum(x, K, l, c, xx, yy, zz, d));
}

__global__ void __launch_bounds__(256) k_smooth(float* __restrict__ x,
                                                const float* __restrict__ rhs,
                                                const float* __restrict__ K,
                                                const float* __restrict__ Dinv,
                                                CL l, int color, int compact) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t c;
  int xx, yy, zz;
  if (!rb_cell(t, l.nx, l.ny, l.n, color, compact, c, xx, yy, zz)) return;
  gs_cell(x, rhs, K, Dinv, l, c, xx, yy, zz);
}

// One CTA: many red-black sweeps over the whole coarsest level.
__global__ void __launch_bounds__(1024) k_coarse_solve(
    float* __restrict__ x, const float* __restrict__ rhs,
    const float* __restrict__ K, const float* __restrict__ Dinv, CL l,
    int sweeps) {
  for (int it = 0; it < sweeps; ++it) {
    for (int color = 0; color < 2; ++color) {
      for (uint32_t c = threadIdx.x; c < (uint32_t)l.n; c += blockDim.x) {
        int xx, yy, zz;
        cl_xyz(c, l, xx, yy, zz);
        if (((xx + yy + zz) & 1) != color) continue;
        const float di = Dinv[c];
        if (di == 0.f) continue;
        int d[6];
        cl_nbr(l, xx, yy, zz, d);
        x[c] = di * (rhs[c] + cl_nsum(x, K, l, c, xx, yy, zz, d));
      }
      __syncthreads();
    }
  }
}

// Restriction from the fine box: rhs_c(J) = sum over children i of
// (r_i - (A e)_i).
template <bool WALLS>
__global__ void __launch_bounds__(256) k_restrict0(
    const float* __restrict__ e, const float* __restrict__ r,
    const uint32_t* __restrict__ links, Box b, CL cl, int cxs, int cys,
    int czs, float* __restrict__ rhs_c) {
  const uint32_t J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= (uint32_t)cl.n) return;
  int X, Y, Z;
  cl_xyz(J, cl, X, Y, Z);
  float acc = 0.f;
  for (int kz = 0; kz <= czs; ++kz)
    for (int ky = 0; ky <= cys; ++ky)
      for (int kx = 0; kx <= cxs; ++kx) {
        const int x = (X << cxs) + kx, y = (Y << cys) + ky, z = (Z << czs) + kz;
        const uint32_t c = ((uint32_t)z * b.ny + y) * b.nx + x;
        uint32_t lk = 0;
        if (WALLS) {
          lk = links[(int64_t)c + (int64_t)b.zlo * b.nxy];
          if (lk & LINK_SOLID) continue;
        }
        int d[6];
        box_nbr(b, x, y, z, d);
        const float ec = e[c];
        float Ae = 0.f;
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          if (WALLS && !open_face(lk, f)) continue;
          Ae += ec - e[(int64_t)c + d[f]];
        }
        acc += r[c] - Ae;
      }
  rhs_c[J] = acc;
}

__global__ void __launch_bounds__(256) k_restrict(
    const float* __restrict__ x, const float* __restrict__ rhs,
    const float* __restrict__ K, const float* __restrict__ Dinv, CL f, CL cl,
    int cxs, int cys, int czs, float* __restrict__ rhs_c) {
  const uint32_t J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= (uint32_t)cl.n) return;
  int X, Y, Z;
  cl_xyz(J, cl, X, Y, Z);
  float acc = 0.f;
  for (int kz = 0; kz <= czs; ++kz)
    for (int ky = 0; ky <= cys; ++ky)
      for (int kx = 0; kx <= cxs; ++kx) {
        const int xx = (X << cxs) + kx, yy = (Y << cys) + ky, zz = (Z << czs) + kz;
        const uint32_t c = ((uint32_t)zz * f.ny + yy) * f.nx + xx;
        const float di = Dinv[c];
        if (di == 0.f) continue;
        int d[6];
        cl_nbr(f, xx, yy, zz, d);
        const float Ax = x[c] / di - cl_nsum(x, K, f, c, xx, yy, zz, d);
        acc += rhs[c] - Ax;
      }
  rhs_c[J] = acc;
}

// Trilinear (cell-centred) prolongation of the coarse correction, added to
// the fine correction.  A coarse cell outside a non-periodic boundary or
// inactive is replaced by the parent cell.
__device__ __forceinline__ void prol_axis(int i, int n_c, int per, int coarsened,
                                          int& p0, int& p1, float& w0) {
  if (!coarsened) {
    p0 = p1 = i;
    w0 = 1.f;
    return;
  }
  p0 = i >> 1;
  int q = (i & 1) ? p0 + 1 : p0 - 1;
  if (q < 0 || q >= n_c) {
    if (per) q = (q + n_c) % n_c;
    else q = p0;
  }
  p1 = q;
  w0 = 0.75f;
}

template <bool FINE0, bool WALLS>
__global__ void __launch_bounds__(256) k_prolong(
    float* __restrict__ ef, const float* __restrict__ Dinv_f,
    const uint32_t* __restrict__ links, Box b, CL f, const float* __restrict__ xc,
    const float* __restrict__ Dinv_c, CL cl, int cxs, int cys, int czs) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= (uint32_t)f.n) return;
  int x, y, z;
  cl_xyz(c, f, x, y, z);
  if (FINE0) {
    if (WALLS && (links[(int64_t)c + (int64_t)b.zlo * b.nxy] & LINK_SOLID)) return;
  } else {
    if (Dinv_f[c] == 0.f) return;
  }
  int ax[2], ay[2], az[2];
  float wx0, wy0, wz0;
  prol_axis(x, cl.nx, cl.px, cxs, ax[0], ax[1], wx0);
  prol_axis(y, cl.ny, cl.py, cys, ay[0], ay[1], wy0);
  prol_axis(z, cl.nz, cl.pz, czs, az[0], az[1], wz0);
  const float wx[2] = {wx0, 1.f - wx0}, wy[2] = {wy0, 1.f - wy0},
              wz[2] = {wz0, 1.f - wz0};
  const int64_t parent = ((int64_t)az[0] * cl.ny + ay[0]) * cl.nx + ax[0];
  const float vp = xc[parent];
  float acc = 0.f;
#pragma unroll
  for (int kz = 0; kz < 2; ++kz)
#pragma unroll
    for (int ky = 0; ky < 2; ++ky)
#pragma unroll
      for (int kx = 0; kx < 2; ++kx) {
        const float w = wx[kx] * wy[ky] * wz[kz];
        if (w == 0.f) continue;
        const int64_t J = ((int64_t)az[kz] * cl.ny + ay[ky]) * cl.nx + ax[kx];
        const float v = (Dinv_c[J] != 0.f) ? xc[J] : vp;
        acc += w * v;
      }
  ef[c] += acc;
}

// Restricted residual of one coarse cell J: sum over its children i of
// (rhs_i - (A x)_i) on the finer level f.
__device__ __forceinline__ float restrict_cell(const float* x, const float* rhs,
                                              const float* K, const float* Dinv,
                                              const CL& f, int X, int Y, int Z,
                                              int cxs, int cys, int czs) {
  float acc = 0.f;
  for (int kz = 0; kz <= czs; ++kz)
    for (int ky = 0; ky <= cys; ++ky)
      for (int kx = 0; kx <= cxs; ++kx) {
        const int xx = (X << cxs) + kx, yy = (Y << cys) + ky, zz = (Z << czs) + kz;
        const uint32_t c = ((uint32_t)zz * f.ny + yy) * f.nx + xx;
        const float di = Dinv[c];
        if (di == 0.f) continue;
        int d[6];
        cl_nbr(f, xx, yy, zz, d);
        acc += rhs[c] - (x[c] / di - cl_nsum(x, K, f, c, xx, yy, zz, d));
      }
  return acc;
}

// Trilinear interpolation of the coarse correction at fine cell (x, y, z).
__device__ __forceinline__ float prolong_cell(const float* xc, const float* Dinv_c,
                                             const CL& cl, int x, int y, int z,
                                             int cxs, int cys, int czs) {
  int ax[2], ay[2], az[2];
  float wx0, wy0, wz0;
  prol_axis(x, cl.nx, cl.px, cxs, ax[0], ax[1], wx0);
  prol_axis(y, cl.ny, cl.py, cys, ay[0], ay[1], wy0);
  prol_axis(z, cl.nz, cl.pz, czs, az[0], az[1], wz0);
  const float wx[2] = {wx0, 1.f - wx0}, wy[2] = {wy0, 1.f - wy0},
              wz[2] = {wz0, 1.f - wz0};
  const int parent = (az[0] * cl.ny + ay[0]) * cl.nx + ax[0];
  const float vp = xc[parent];
  float acc = 0.f;
#pragma unroll
  for (int kz = 0; kz < 2; ++kz)
#pragma unroll
    for (int ky = 0; ky < 2; ++ky)
#pragma unroll
      for (int kx = 0; kx < 2; ++kx) {
        const float w = wx[kx] * wy[ky] * wz[kz];
        if (w == 0.f) continue;
        const int J = (az[kz] * cl.ny + ay[ky]) * cl.nx + ax[kx];
        acc += w * ((Dinv_c[J] != 0.f) ? xc[J] : vp);
      }
  return acc;
}

constexpr int SUB_MAX_LEVELS = 8;
constexpr int64_t SUB_MAX_CELLS = 4096;  // finest level handled in shared memory

struct SubLevel {
  CL l;
  int cx, cy, cz;  // halved axes relative to the next finer level
  const float* K;
  const float* Dinv;
};
struct SubHier {
  SubLevel lev[SUB_MAX_LEVELS];
  int nlev;
  const float* rhs_in;  // right-hand side of the first level (global)
  float* e_out;         // its correction (global)
};

// The whole V-cycle below and including a level of at most 4096 cells, in
// one CTA, every array in shared memory: smoothing, restriction, the
// coarsest-level sweeps and prolongation, separated by __syncthreads.
__global__ void __launch_bounds__(1024) k_sub_cycle(const SubHier H, int nu1, int nu2,
                                                    int sweeps) {
  extern __shared__ float sm[];
  __shared__ int offs[SUB_MAX_LEVELS];
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) {
    int off = 0;
    for (int l = 0; l < H.nlev; ++l) {
      offs[l] = off;
      off += 6 * (int)H.lev[l].l.n;
    }
  }
  __syncthreads();
  // level l occupies [e | rhs | K (3n) | Dinv] at sm + offs[l]
  struct Lv {
    float *e, *r, *K, *D;
  };
  auto lv = [&](int l) {
    const int n = (int)H.lev[l].l.n;
    Lv v;
    v.e = sm + offs[l];
    v.r = v.e + n;
    v.K = v.r + n;
    v.D = v.K + 3 * n;
    return v;
  };
  for (int l = 0; l < H.nlev; ++l) {
    const int n = (int)H.lev[l].l.n;
    const Lv v = lv(l);
    for (int c = tid; c < n; c += nt) {
      v.e[c] = 0.f;
      v.r[c] = l == 0 ? H.rhs_in[c] : 0.f;
      v.D[c] = H.lev[l].Dinv[c];
      v.K[c] = H.lev[l].K[c];
      v.K[n + c] = H.lev[l].K[n + c];
      v.K[2 * n + c] = H.lev[l].K[2 * n + c];
    }
  }
  __syncthreads();
  auto smooth = [&](int l, int count) {
    const CL L = H.lev[l].l;
    const Lv v = lv(l);
    const int compact = (L.nx % 2 == 0);
    const int work = compact ? (int)(L.n >> 1) : (int)L.n;
    for (int k = 0; k < count; ++k)
      for (int color = 0; color < 2; ++color) {
        for (int t = tid; t < work; t += nt) {
          uint32_t c;
          int xx, yy, zz;
          if (rb_cell((uint32_t)t, L.nx, L.ny, L.n, color, compact, c, xx, yy, zz))
            gs_cell(v.e, v.r, v.K, v.D, L, c, xx, yy, zz);
        }
        __syncthreads();
      }
  };
  for (int l = 0; l + 1 < H.nlev; ++l) {
    smooth(l, nu1);
    const SubLevel& C = H.lev[l + 1];
    const Lv f = lv(l), cv = lv(l + 1);
    const CL F = H.lev[l].l;
    for (int J = tid; J < (int)C.l.n; J += nt) {
      int X, Y, Z;
      cl_xyz((uint32_t)J, C.l, X, Y, Z);
      cv.r[J] = restrict_cell(f.e, f.r, f.K, f.D, F, X, Y, Z, C.cx, C.cy, C.cz);
    }
    __syncthreads();
  }
  smooth(H.nlev - 1, sweeps);
  for (int l = H.nlev - 2; l >= 0; --l) {
    const SubLevel& C = H.lev[l + 1];
    const CL L = H.lev[l].l;
    const Lv f = lv(l), cv = lv(l + 1);
    for (int c = tid; c < (int)L.n; c += nt) {
      if (f.D[c] == 0.f) continue;
      int xx, yy, zz;
      cl_xyz((uint32_t)c, L, xx, yy, zz);
      f.e[c] += prolong_cell(cv.e, cv.D, C.l, xx, yy, zz, C.cx, C.cy, C.cz);
    }
    __syncthreads();
    smooth(l, nu2);
  }
  const Lv v0 = lv(0);
  for (int c = tid; c < (int)H.lev[0].l.n; c += nt) H.e_out[c] = v0.e[c];
}

inline unsigned nblocks(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

Box make_box(lbm_t* h) {
  Box b;
  b.nx = h->cfg.nx;
  b.ny = h->cfg.ny;
  b.nzb = h->ps.nzb;
  b.zlo = h->ps.zlo;
  b.perz = h->ps.perz;
  b.nxy = (int64_t)b.nx * b.ny;
  return b;
}

CL make_cl(const PoissonLevel& l) {
  CL c;
  c.nx = l.nx;
  c.ny = l.ny;
  c.nz = l.nz;
  c.n = l.n;
  c.px = l.per[0];
  c.py = l.per[1];
  c.pz = l.per[2];
  return c;
}

}  // namespace

namespace {
void drop_graphs(Poisson& P) {
  for (int k = 0; k < 2; ++k) {
    if (P.cyc[k]) cudaGraphExecDestroy(P.cyc[k]);
    P.cyc[k] = nullptr;
  }
  P.cyc_failed = false;
}
}  // namespace

void poisson_free(lbm_t* h) {
  Poisson& P = h->ps;
  drop_graphs(P);
  for (auto& l : P.lev) {
    cudaFree(l.e);
    cudaFree(l.rhs);
    cudaFree(l.K);
    cudaFree(l.Dinv);
  }
  P.lev.clear();
  cudaFree(P.psi[0]);
  cudaFree(P.psi[1]);
  cudaFree(P.src);
  cudaFree(P.dsum);
  cudaFree(P.part);
  P.part = nullptr;
  cudaFree(P.label);
  cudaFree(P.comp_sum);
  cudaFree(P.comp_size);
  cudaFree(P.comp_mean);
  P.label = nullptr;
  P.comp_sum = nullptr;
  P.comp_size = nullptr;
  P.comp_mean = nullptr;
  P.ncomp = 1;
  if (P.hsum) cudaFreeHost(P.hsum);
  P.psi[0] = P.psi[1] = nullptr;
  P.src = nullptr;
  P.dsum = nullptr;
  P.hsum = nullptr;
}

namespace {
int sub_level(const Poisson& P);
size_t sub_smem(const Poisson& P, int lc);
}  // namespace

// Builds the grid hierarchy.  solid_host: lattice mask or NULL.
lbm_status poisson_setup(lbm_t* h, const uint8_t* solid) {
  Poisson& P = h->ps;
  drop_graphs(P);
  const int nx = h->cfg.nx, ny = h->cfg.ny, nz = h->cfg.nz;
  const int64_t nxy = (int64_t)nx * ny;
  // Trim fully solid bottom and top planes (slit geometry): the Poisson box
  // is then non-periodic in z.
  P.zlo = 0;
  P.nzb = nz;
  P.perz = 1;
  if (solid && nz >= 3) {
    auto plane_solid = [&](int z) {
      for (int64_t k = 0; k < nxy; ++k)
        if (!solid[(int64_t)z * nxy + k]) return false;
      return true;
    };
    if (plane_solid(0) && plane_solid(nz - 1)) {
      P.zlo = 1;
      P.nzb = nz - 2;
      P.perz = 0;
    }
  }
  // free old levels (walls may be reset)
  for (auto& l : P.lev) {
    cudaFree(l.e);
    cudaFree(l.rhs);
    cudaFree(l.K);
    cudaFree(l.Dinv);
  }
  P.lev.clear();

  // Level 0 conductances on the host (face open iff both cells fluid).
  PoissonLevel L0;
  L0.nx = nx;
  L0.ny = ny;
  L0.nz = P.nzb;
  L0.n = nxy * P.nzb;
  L0.per[0] = 1;
  L0.per[1] = 1;
  L0.per[2] = P.perz;
  L0.coarsened[0] = L0.coarsened[1] = L0.coarsened[2] = 0;
  auto fl0 = [&](int x, int y, int z) -> bool {
    return !solid || !solid[((int64_t)(z + P.zlo) * ny + y) * nx + x];
  };
  // host conductances of the current finest level: Kh[3][n], active flags
  std::vector<float> Kh(3 * L0.n, 0.f);
  std::vector<char> act(L0.n, 0);
  for (int z = 0; z < P.nzb; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int64_t c = ((int64_t)z * ny + y) * nx + x;
        act[c] = fl0(x, y, z);
        if (!act[c]) continue;
        if (nx > 1 && fl0((x + 1) % nx, y, z)) Kh[c] = 1.f;
        if (ny > 1 && fl0(x, (y + 1) % ny, z)) Kh[L0.n + c] = 1.f;
        if (P.nzb > 1 && (z + 1 < P.nzb || P.perz)) {
          if (fl0(x, y, (z + 1) % P.nzb)) Kh[2 * L0.n + c] = 1.f;
        }
      }
  if (cudaMalloc(&L0.e, L0.n * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&L0.rhs, L0.n * sizeof(float)) != cudaSuccess) {
    h->err = "Poisson level 0 allocation failed";
    return LBM_ENOMEM;
  }
  P.lev.push_back(L0);

  // Coarsen while the level has more than 64 cells and an axis can halve.
  int lx = nx, ly = ny, lz = P.nzb;
  int per[3] = {1, 1, P.perz};
  while ((int64_t)lx * ly * lz > 64 && P.lev.size() < 12) {
    int cx = (lx % 2 == 0 && lx >= 4), cy = (ly % 2 == 0 && ly >= 4),
        cz = (lz % 2 == 0 && lz >= 4);
    if (!cx && !cy && !cz) break;
    const int Lx = cx ? lx / 2 : lx, Ly = cy ? ly / 2 : ly, Lz = cz ? lz / 2 : lz;
    const int64_t n = (int64_t)Lx * Ly * Lz, nf = (int64_t)lx * ly * lz;
    std::vector<float> Kc(3 * n, 0.f);
    std::vector<char> ac(n, 0);
    const float sc[3] = {cx ? 0.5f : 1.f, cy ? 0.5f : 1.f, cz ? 0.5f : 1.f};
    for (int z = 0; z < lz; ++z)
      for (int y = 0; y < ly; ++y)
        for (int x = 0; x < lx; ++x) {
          const int64_t c = ((int64_t)z * ly + y) * lx + x;
          if (!act[c]) continue;
          const int X = cx ? x / 2 : x, Y = cy ? y / 2 : y, Z = cz ? z / 2 : z;
          const int64_t J = ((int64_t)Z * Ly + Y) * Lx + X;
          ac[J] = 1;
          // a fine face crossing the + face of J: the child on the + side
          // of J along that axis (last child), or any child if not coarsened
          if (!cx || (x & 1)) Kc[J] += sc[0] * Kh[c];
          if (!cy || (y & 1)) Kc[n + J] += sc[1] * Kh[nf + c];
          if (!cz || (z & 1)) Kc[2 * n + J] += sc[2] * Kh[2 * nf + c];
        }
    // inner faces of a non-coarsened axis are within J only if coarsened;
    // for a non-coarsened axis every child's + face is the coarse + face.
    std::vector<float> Dv(n, 0.f);
    for (int Z = 0; Z < Lz; ++Z)
      for (int Y = 0; Y < Ly; ++Y)
        for (int X = 0; X < Lx; ++X) {
          const int64_t J = ((int64_t)Z * Ly + Y) * Lx + X;
          if (!ac[J]) continue;
          const int Xm = (X - 1 + Lx) % Lx, Ym = (Y - 1 + Ly) % Ly, Zm = (Z - 1 + Lz) % Lz;
          float D = Kc[J] + Kc[n + J] + Kc[2 * n + J];
          if (per[0] || X > 0) D += Kc[((int64_t)Z * Ly + Y) * Lx + Xm];
          if (per[1] || Y > 0) D += Kc[n + ((int64_t)Z * Ly + Ym) * Lx + X];
          if (per[2] || Z > 0) D += Kc[2 * n + ((int64_t)Zm * Ly + Y) * Lx + X];
          Dv[J] = D > 0.f ? 1.f / D : 0.f;
          if (D == 0.f) ac[J] = 0;
        }
    PoissonLevel L;
    L.nx = Lx;
    L.ny = Ly;
    L.nz = Lz;
    L.n = n;
    L.per[0] = per[0];
    L.per[1] = per[1];
    L.per[2] = per[2];
    L.coarsened[0] = cx;
    L.coarsened[1] = cy;
    L.coarsened[2] = cz;
    if (cudaMalloc(&L.e, n * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&L.rhs, n * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&L.K, 3 * n * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&L.Dinv, n * sizeof(float)) != cudaSuccess) {
      h->err = "Poisson level allocation failed";
      P.lev.push_back(L);
      return LBM_ENOMEM;
    }
    cudaMemcpy(L.K, Kc.data(), 3 * n * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(L.Dinv, Dv.data(), n * sizeof(float), cudaMemcpyHostToDevice);
    P.lev.push_back(L);
    Kh.swap(Kc);
    act.swap(ac);
    lx = Lx;
    ly = Ly;
    lz = Lz;
  }
  const int lc = sub_level(P);
  if (lc > 0) {
    // allow the largest dynamic shared memory the device offers, so that
    // lattices created later with bigger sub-hierarchies also fit
    int optin = 0;
    LBM_CUDA_TRY(h, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev));
    if ((int)sub_smem(P, lc) > optin) {
      h->err = "coarse Poisson levels exceed the shared memory of one CTA";
      return LBM_EINVAL;
    }
    cudaFuncAttributes fa;
    LBM_CUDA_TRY(h, cudaFuncGetAttributes(&fa, k_sub_cycle));
    const int dyn_max = optin - (int)fa.sharedSizeBytes;
    if ((int)sub_smem(P, lc) > dyn_max) {
      h->err = "coarse Poisson levels exceed the shared memory of one CTA";
      return LBM_EINVAL;
    }
    LBM_CUDA_TRY(h, cudaFuncSetAttribute(k_sub_cycle, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         dyn_max));
  }
  LBM_CUDA_TRY(h, cudaGetLastError());
  return LBM_OK;
}

namespace {

// Queues the fine-box residual of the current potential and the
// device-to-host copy of its norms; does not wait.
cudaError_t residual_launch(lbm_t* h) {
  Poisson& P = h->ps;
  const Box b = make_box(h);
  const int64_t nbox = P.lev[0].n;
  const double inv_nf = 1.0 / (double)h->nfluid;
  cudaError_t e = cudaMemsetAsync(P.dsum + 1, 0, 2 * sizeof(double), h->st);
  if (e != cudaSuccess) return e;
  const unsigned nb = (unsigned)std::min<int64_t>(nblocks(nbox, 256), h->grid_cap);
  if (h->has_walls)
    k_res0<true><<<nb, 256, 0, h->st>>>(P.psi[P.cur], P.src, h->links, P.lev[0].rhs, P.dsum,
                                        b, nbox, inv_nf, P.label, P.comp_mean);
  else
    k_res0<false><<<nb, 256, 0, h->st>>>(P.psi[P.cur], P.src, nullptr, P.lev[0].rhs, P.dsum,
                                         b, nbox, inv_nf, nullptr, nullptr);
  ++h->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaMemcpyAsync(P.hsum, P.dsum, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->st);
}

// Waits for the last queued residual.  Returns ||r|| / ||s|| in *rel and
// whether the solve has converged: relative residual <= tol, or a residual
// at the fixed-point resolution of psi (rms below 2 units of 2^-52), which
// is all a charge-neutral source of vanishing norm allows.
lbm_status residual_read(lbm_t* h, double tol, double* rel, bool* done) {
  Poisson& P = h->ps;
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  const double rn = sqrt(P.hsum[1]), sn = sqrt(P.hsum[2]);
  *rel = sn > 0.0 ? rn / sn : (rn > 0.0 ? INFINITY : 0.0);
  if (!isfinite(rn) || !isfinite(sn)) {
    h->err = "Poisson residual is not finite";
    return LBM_EUNSTABLE;
  }
  *done = rn <= tol * sn || rn <= RES_FLOOR_RMS * sqrt((double)h->nfluid);
  return LBM_OK;
}

cudaError_t smooth_level(lbm_t* h, int l, int sweeps, bool apply = false) {
  Poisson& P = h->ps;
  PoissonLevel& L = P.lev[l];
  const int compact = (L.nx % 2 == 0) ? 1 : 0;
  const unsigned nb = nblocks(compact ? L.n / 2 : L.n, 256);
  if (l == 0) {
    const Box b = make_box(h);
    const int64_t* pin = P.psi[P.cur];
    int64_t* pout = P.psi[P.cur ^ 1];
    for (int k = 0; k < sweeps; ++k)
      for (int color = 0; color < 2; ++color) {
        const bool last = apply && k == sweeps - 1;
        if (h->has_walls) {
          if (last)
            k_smooth0<true, true><<<nb, 256, 0, h->st>>>(L.e, L.rhs, h->links, b, L.n, color,
                                                         compact, pin, pout);
          else
            k_smooth0<true, false><<<nb, 256, 0, h->st>>>(L.e, L.rhs, h->links, b, L.n, color,
                                                          compact, pin, pout);
        } else {
          if (last)
            k_smooth0<false, true><<<nb, 256, 0, h->st>>>(L.e, L.rhs, nullptr, b, L.n, color,
                                                          compact, pin, pout);
          else
            k_smooth0<false, false><<<nb, 256, 0, h->st>>>(L.e, L.rhs, nullptr, b, L.n, color,
                                                           compact, pin, pout);
        }
        ++h->launches;
      }
    if (apply) P.cur ^= 1;
  } else {
    const CL c = make_cl(L);
    for (int k = 0; k < sweeps; ++k)
      for (int color = 0; color < 2; ++color) {
        k_smooth<<<nb, 256, 0, h->st>>>(L.e, L.rhs, L.K, L.Dinv, c, color, compact);
        ++h->launches;
      }
  }
  return cudaGetLastError();
}

// First level (>= 1) small enough for the shared-memory sub-cycle.
int sub_level(const Poisson& P) {
  for (int l = 1; l < (int)P.lev.size(); ++l)
    if (P.lev[l].n <= SUB_MAX_CELLS && (int)P.lev.size() - l <= SUB_MAX_LEVELS) return l;
  return -1;
}

size_t sub_smem(const Poisson& P, int lc) {
  size_t n = 0;
  for (int l = lc; l < (int)P.lev.size(); ++l) n += 6 * (size_t)P.lev[l].n;
  return n * sizeof(float);
}

cudaError_t launch_sub_cycle(lbm_t* h, int lc) {
  Poisson& P = h->ps;
  SubHier H;
  H.nlev = (int)P.lev.size() - lc;
  for (int k = 0; k < H.nlev; ++k) {
    const PoissonLevel& L = P.lev[lc + k];
    H.lev[k].l = make_cl(L);
    H.lev[k].cx = L.coarsened[0];
    H.lev[k].cy = L.coarsened[1];
    H.lev[k].cz = L.coarsened[2];
    H.lev[k].K = L.K;
    H.lev[k].Dinv = L.Dinv;
  }
  H.rhs_in = P.lev[lc].rhs;
  H.e_out = P.lev[lc].e;
  const size_t smem = sub_smem(P, lc);
  const int threads = (int)std::min<int64_t>(1024, std::max<int64_t>(64, ((P.lev[lc].n / 2 + 31) / 32) * 32));
  k_sub_cycle<<<1, threads, smem, h->st>>>(H, P.nu1, P.nu2, P.coarse_sweeps);
  ++h->launches;
  return cudaGetLastError();
}

cudaError_t vcycle(lbm_t* h) {
  Poisson& P = h->ps;
  const int nl = (int)P.lev.size();
  const Box b = make_box(h);
  cudaError_t e = cudaMemsetAsync(P.lev[0].e, 0, P.lev[0].n * sizeof(float), h->st);
  if (e != cudaSuccess) return e;
  if (nl == 1) return smooth_level(h, 0, 8, true);
  const int lc = sub_level(P);
  if ((e = smooth_level(h, 0, P.nu1)) != cudaSuccess) return e;
  {
    PoissonLevel& C = P.lev[1];
    const CL cl = make_cl(C);
    if (h->has_walls)
      k_restrict0<true><<<nblocks(C.n, 256), 256, 0, h->st>>>(
          P.lev[0].e, P.lev[0].rhs, h->links, b, cl, C.coarsened[0], C.coarsened[1],
          C.coarsened[2], C.rhs);
    else
      k_restrict0<false><<<nblocks(C.n, 256), 256, 0, h->st>>>(
          P.lev[0].e, P.lev[0].rhs, nullptr, b, cl, C.coarsened[0], C.coarsened[1],
          C.coarsened[2], C.rhs);
    ++h->launches;
  }
  const int last = lc > 0 ? lc : nl - 1;  // levels 1..last-1 use grid kernels
  for (int l = 1; l < last; ++l) {
    PoissonLevel& L = P.lev[l];
    if ((e = cudaMemsetAsync(L.e, 0, L.n * sizeof(float), h->st)) != cudaSuccess) return e;
    if ((e = smooth_level(h, l, P.nu1)) != cudaSuccess) return e;
    PoissonLevel& C = P.lev[l + 1];
    k_restrict<<<nblocks(C.n, 256), 256, 0, h->st>>>(L.e, L.rhs, L.K, L.Dinv, make_cl(L),
                                                     make_cl(C), C.coarsened[0],
                                                     C.coarsened[1], C.coarsened[2], C.rhs);
    ++h->launches;
  }
  if (lc > 0) {
    if ((e = launch_sub_cycle(h, lc)) != cudaSuccess) return e;
  } else {
    PoissonLevel& L = P.lev[last];
    if ((e = cudaMemsetAsync(L.e, 0, L.n * sizeof(float), h->st)) != cudaSuccess) return e;
    if ((e = smooth_level(h, last, 50)) != cudaSuccess) return e;
  }
  for (int l = last - 1; l >= 0; --l) {
    PoissonLevel& F = P.lev[l];
    PoissonLevel& C = P.lev[l + 1];
    const unsigned nb = nblocks(F.n, 256);
    if (l == 0) {
      if (h->has_walls)
        k_prolong<true, true><<<nb, 256, 0, h->st>>>(F.e, nullptr, h->links, b, make_cl(F),
                                                     C.e, C.Dinv, make_cl(C), C.coarsened[0],
                                                     C.coarsened[1], C.coarsened[2]);
      else
        k_prolong<true, false><<<nb, 256, 0, h->st>>>(F.e, nullptr, nullptr, b, make_cl(F),
                                                      C.e, C.Dinv, make_cl(C), C.coarsened[0],
                                                      C.coarsened[1], C.coarsened[2]);
    } else {
      k_prolong<false, false><<<nb, 256, 0, h->st>>>(F.e, F.Dinv, nullptr, b, make_cl(F),
                                                     C.e, C.Dinv, make_cl(C), C.coarsened[0],
                                                     C.coarsened[1], C.coarsened[2]);
    }
    ++h->launches;
    if ((e = smooth_level(h, l, P.nu2, l == 0)) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace

namespace {

// One V-cycle followed by the residual of the corrected potential.  Replays
// a CUDA graph captured on first use (one per starting potential buffer);
// falls back to direct launches if capture is unavailable on the stream.
cudaError_t cycle(lbm_t* h) {
  Poisson& P = h->ps;
  const int start = P.cur;
  if (!P.cyc[start] && !P.cyc_failed) {
    cudaStreamCaptureStatus cs;
    cudaError_t e = cudaStreamIsCapturing(h->st, &cs);
    if (e == cudaSuccess && cs == cudaStreamCaptureStatusNone && h->st != nullptr &&
        cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int64_t before = h->launches;
      cudaError_t e1 = vcycle(h);
      cudaError_t e2 = e1 == cudaSuccess ? residual_launch(h) : e1;
      cudaGraph_t g = nullptr;
      cudaError_t e3 = cudaStreamEndCapture(h->st, &g);
      P.cur = start;                 // capture only recorded the work
      const int nk = (int)(h->launches - before);
      h->launches = before;
      cudaGraphExec_t ex = nullptr;
      if (e2 == cudaSuccess && e3 == cudaSuccess && g &&
          cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
        P.cyc[start] = ex;
        P.cyc_kernels = nk;
      } else {
        P.cyc_failed = true;
      }
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
    } else {
      cudaGetLastError();
      P.cyc_failed = true;
    }
  }
  if (P.cyc[start]) {
    cudaError_t e = cudaGraphLaunch(P.cyc[start], h->st);
    if (e != cudaSuccess) return e;
    P.cur ^= 1;
    h->launches += P.cyc_kernels;
    return cudaSuccess;
  }
  cudaError_t e = vcycle(h);
  if (e != cudaSuccess) return e;
  return residual_launch(h);
}

}  // namespace

lbm_status poisson_solve(lbm_t* h, double tol, int maxit, int* iters,
                         double* rel_res) {
  if (h->cfg.poisson == LBM_POISSON_FFT) return spectral_solve(h, tol, maxit, iters, rel_res);
  Poisson& P = h->ps;
  double rel = 0.0, rel0 = 0.0;
  bool done = false;
  LBM_CUDA_TRY(h, residual_launch(h));
  lbm_status s = residual_read(h, tol, &rel, &done);
  if (s != LBM_OK) return s;
  if (!done && nn_active(h)) {
    // learned initial guess: apply, keep it only if the residual drops
    const double rn = sqrt(P.hsum[1]) * PSI_INV_SCALE;
    bool applied = false;
    float* dpsi = nullptr;
    s = nn_before_solve(h, P.lev[0].rhs, P.zlo, P.nzb, rn / sqrt((double)h->nfluid), &applied, &dpsi);
    if (s != LBM_OK) return s;
    if (applied) {
      double rel_nn = 0.0;
      bool done_nn = false;
      LBM_CUDA_TRY(h, residual_launch(h));
      s = residual_read(h, tol, &rel_nn, &done_nn);
      if (s != LBM_OK) return s;
      if (rel_nn < rel) {
        nn_record(h, rel_nn / rel);
        rel = rel_nn;
        done = done_nn;
      } else {
        s = nn_revert(h, dpsi);
        if (s != LBM_OK) return s;
        LBM_CUDA_TRY(h, residual_launch(h));
        s = residual_read(h, tol, &rel, &done);
        if (s != LBM_OK) return s;
      }
    }
  }
  rel0 = rel;
  note_start_residual(h, rel0);
  int it = 0;
  if (h->cfg.poisson == LBM_POISSON_MG) {
    // Queue the predicted number of cycles (from the initial residual and
    // the reduction per cycle measured in the last solve) minus one before
    // the first host read-back, then test after every cycle.
    int batch = 1;
    if (!done && rel0 > 0.0 && isfinite(rel0)) {
      const double need = std::log(tol / rel0) / std::log(P.conv);
      batch = std::max(1, std::min(maxit, (int)std::ceil(need) - 1));
    }
    while (!done && it < maxit) {
      const int nb = std::min(batch, maxit - it);
      for (int k = 0; k < nb; ++k) LBM_CUDA_TRY(h, cycle(h));
      it += nb;
      batch = 1;
      s = residual_read(h, tol, &rel, &done);
      if (s != LBM_OK) return s;
    }
    if (it > 0 && rel > 0.0 && rel0 > 0.0 && isfinite(rel) && rel < rel0)
      P.conv = std::min(0.6, std::max(0.01, std::pow(rel / rel0, 1.0 / it)));
  } else {
    const Box b = make_box(h);
    const int64_t nbox = P.lev[0].n;
    const double inv_nf = 1.0 / (double)h->nfluid;
    const int L = std::max(std::max(h->cfg.nx, h->cfg.ny), P.nzb);
    // Red-black ordering is a true two-colouring only when every periodic
    // extent is even; otherwise same-colour neighbours meet across the wrap
    // and are updated together, which over-relaxation does not tolerate:
    // fall back to Gauss-Seidel weights there.
    const bool odd_wrap = (h->cfg.nx > 1 && (h->cfg.nx & 1)) ||
                          (h->cfg.ny > 1 && (h->cfg.ny & 1)) ||
                          (P.perz && P.nzb > 1 && (P.nzb & 1));
    const float omega =
        odd_wrap ? 1.0f : (float)(2.0 / (1.0 + sin(3.14159265358979323846 / L)));
    const int check = 10;
    while (!done && it < maxit) {
      for (int k = 0; k < check; ++k)
        for (int color = 0; color < 2; ++color) {
          if (h->has_walls)
            k_sor0<true><<<nblocks(nbox, 256), 256, 0, h->st>>>(
                P.psi[P.cur], P.src, h->links, P.dsum, b, nbox, inv_nf, color, omega, P.label,
                P.comp_mean);
          else
            k_sor0<false><<<nblocks(nbox, 256), 256, 0, h->st>>>(
                P.psi[P.cur], P.src, nullptr, P.dsum, b, nbox, inv_nf, color, omega, nullptr,
                nullptr);
          ++h->launches;
        }
      LBM_CUDA_TRY(h, cudaGetLastError());
      it += check;
      LBM_CUDA_TRY(h, residual_launch(h));
      s = residual_read(h, tol, &rel, &done);
      if (s != LBM_OK) return s;
    }
  }
  if (iters) *iters = it;
  if (rel_res) *rel_res = rel;
  if (!done) {
    h->err = "Poisson solve did not reach the tolerance within the iteration cap";
    return LBM_ENOCONV;
  }
  return LBM_OK;
}

}  // namespace lbm_gb300
