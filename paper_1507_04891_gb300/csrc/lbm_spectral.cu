// Spectral Poisson solver for lattices whose every z-plane is either all
// fluid or all wall (periodic boxes, slits, stacks of slits).  It solves the
// same finite-volume problem as the multigrid (Eq. Poisson with the
// surface-charge condition):
//   A psi = s - <s>_run,   (A psi)_i = sum_open faces (psi_i - psi_j),
// where <s>_run is the mean of the source over each run of consecutive
// fluid planes (each run is a separate connected fluid domain).
//
// The x and y directions are periodic and uniform, so a 2-D discrete
// Fourier transform diagonalises them: for the mode (kx, ky) the operator
// becomes lambda(kx, ky) + (1-D operator along z), and the z operator of a
// run is tridiagonal (walls at both ends: one open face there) or cyclic
// (a run that is the whole periodic z axis).  One application solves the
// problem to FP32 accuracy; it is used for defect correction on the exact
// fixed-point residual, so two applications usually reach 1e-8.
//
// Kernels per application: forward FFT of the residual, two real planes per
// complex transform (shared memory, radix 2); along z an FFT (periodic
// power-of-two z) or one tridiagonal solve per mode and run; inverse FFT
// fused with the update psi += round(e).
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "lbm_internal.cuh"

namespace lbm_gb300 {
namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ unsigned brev(unsigned v, int bits) {
  return __brev(v) >> (32 - bits);
}

// In-place radix-2 FFTs of `count` rows of length n = 2^lg stored with
// element stride `es` and row stride `rs` in shared memory (count = 2^lgc).
// Input in bit-reversed order.  tw[k] = exp(-2 pi i k / n) (k < n/2); sign
// -1 forward, +1 inverse (conjugate twiddles).  Consecutive threads take
// consecutive butterflies of one row when the elements are contiguous
// (es == 1) and the same butterfly of consecutive rows otherwise, so that
// shared-memory accesses never stride by a row.
__device__ void fft_rows(float2* a, int lg, int lgc, int es, int rs,
                         const float2* tw, float sign) {
  if (lg == 0) return;
  const int half = 1 << (lg - 1);
  const int total = half << lgc;
  for (int s = 1; s <= lg; ++s) {
    const int mh = 1 << (s - 1);
    const int tshift = lg - s;  // twiddle index step n/m = 2^(lg - s)
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      int row, b;
      if (es == 1) {
        row = t >> (lg - 1);
        b = t & (half - 1);
      } else {
        row = t & ((1 << lgc) - 1);
        b = t >> lgc;
      }
      const int j = b & (mh - 1);
      const int i0 = ((b >> (s - 1)) << s) + j, i1 = i0 + mh;
      float2 w = tw[j << tshift];
      w.y *= -sign;
      float2* p0 = a + row * rs + i0 * es;
      float2* p1 = a + row * rs + i1 * es;
      const float2 u = *p0;
      const float2 v = cmul(w, *p1);
      *p0 = make_float2(u.x + v.x, u.y + v.y);
      *p1 = make_float2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
  }
}

struct SpecArgs {
  int nx, ny, nz, lgx, lgy;
  const float2* twx;
  const float2* twy;
  const float* lam_xy;  // eigenvalue of the x-y Laplacian per mode (nx*ny)
  const float* lam_z;   // eigenvalue along a periodic z per kz (nz) or NULL
};

// The 2-D transform runs as separate passes with many small CTAs: rows
// along x (two real rows packed in one complex FFT), then columns along y.
//
// Forward x pass: rows y0 = 2q and y1 = 2q + 1 of a fluid plane form
// C = r_y0 + i r_y1; after the FFT, R_y0(k) = (C(k) + conj C(-k)) / 2 and
// R_y1(k) = (C(k) - conj C(-k)) / (2i) by the symmetry of real data.  One CTA
// handles RXP row pairs.
__global__ void __launch_bounds__(256) k_fft_x_fwd(const float* __restrict__ r,
                                                   float2* __restrict__ spec,
                                                   const int* __restrict__ planes, int npairs_row,
                                                   int64_t total_pairs, SpecArgs a, int lgr) {
  extern __shared__ float2 rb[];
  const int nx = a.nx, lgx = a.lgx;
  const int rxp = 1 << lgr;  // row pairs per CTA
  const int64_t p0 = (int64_t)blockIdx.x * rxp;
  const int cnt = (int)min((int64_t)rxp, total_pairs - p0);
#pragma unroll 4
  for (int idx = threadIdx.x; idx < cnt * nx; idx += blockDim.x) {
    const int q = idx >> lgx, x = idx & (nx - 1);
    const int64_t pp = p0 + q;
    const int z = planes[pp / npairs_row];
    const int y0 = 2 * (int)(pp % npairs_row), y1 = y0 + 1;
    const float* row = r + ((int64_t)z * a.ny) * nx;
    const float v0 = row[(int64_t)y0 * nx + x];
    const float v1 = (y1 < a.ny) ? row[(int64_t)y1 * nx + x] : 0.f;
    rb[q * nx + (lgx ? (int)brev(x, lgx) : 0)] = make_float2(v0, v1);
  }
  __syncthreads();
  fft_rows(rb, lgx, lgr, 1, nx, a.twx, -1.f);
  for (int idx = threadIdx.x; idx < cnt * nx; idx += blockDim.x) {
    const int q = idx >> lgx, k = idx & (nx - 1);
    const int64_t pp = p0 + q;
    const int z = planes[pp / npairs_row];
    const int y0 = 2 * (int)(pp % npairs_row), y1 = y0 + 1;
    const float2 c = rb[q * nx + k], cm = rb[q * nx + ((nx - k) & (nx - 1))];
    float2* out = spec + ((int64_t)z * a.ny) * nx;
    out[(int64_t)y0 * nx + k] = make_float2(0.5f * (c.x + cm.x), 0.5f * (c.y - cm.y));
    if (y1 < a.ny) out[(int64_t)y1 * nx + k] = make_float2(0.5f * (c.y + cm.y), -0.5f * (c.x - cm.x));
  }
}

// y pass (in place): one CTA takes CYC consecutive kx columns of one plane,
// staged in shared memory as [y][column] (coalesced), FFT along y.
__global__ void __launch_bounds__(256) k_fft_y(float2* __restrict__ spec,
                                               const int* __restrict__ planes, int cols_per_plane,
                                               SpecArgs a, float sign, int lgc) {
  extern __shared__ float2 cb[];
  const int ny = a.ny, lgy = a.lgy, nx = a.nx;
  const int CYC = 1 << lgc;  // columns per CTA
  const int z = planes[blockIdx.x / cols_per_plane];
  const int k0 = (blockIdx.x % cols_per_plane) * CYC;
  const int w = min(CYC, nx - k0);
  float2* base = spec + (int64_t)z * ny * nx + k0;
#pragma unroll 4
  for (int idx = threadIdx.x; idx < ny * CYC; idx += blockDim.x) {
    const int y = idx >> lgc, j = idx & (CYC - 1);
    if (j < w) cb[(lgy ? (int)brev(y, lgy) : 0) * CYC + j] = base[(int64_t)y * nx + j];
  }
  __syncthreads();
  fft_rows(cb, lgy, lgc, CYC, 1, a.twy, sign);
  for (int idx = threadIdx.x; idx < ny * CYC; idx += blockDim.x) {
    const int y = idx >> lgc, j = idx & (CYC - 1);
    if (j < w) base[(int64_t)y * nx + j] = cb[y * CYC + j];
  }
}

// Inverse x pass fused with the update: rows y0, y1 of the corrections
// (Hermitian spectra) form C = E_y0 + i E_y1; the inverse FFT gives e_y0 in
// the real and e_y1 in the imaginary part; psi += round(e / (nx ny)).
__global__ void __launch_bounds__(256) k_fft_x_inv_apply(const float2* __restrict__ spec,
                                                         const int* __restrict__ planes,
                                                         int npairs_row, int64_t total_pairs,
                                                         SpecArgs a, int64_t* psi, int lgr) {
  extern __shared__ float2 rb[];
  const int nx = a.nx, lgx = a.lgx;
  const int rxp = 1 << lgr;
  const int64_t p0 = (int64_t)blockIdx.x * rxp;
  const int cnt = (int)min((int64_t)rxp, total_pairs - p0);
  for (int idx = threadIdx.x; idx < cnt * nx; idx += blockDim.x) {
    const int q = idx >> lgx, k = idx & (nx - 1);
    const int64_t pp = p0 + q;
    const int z = planes[pp / npairs_row];
    const int y0 = 2 * (int)(pp % npairs_row), y1 = y0 + 1;
    const float2* row = spec + ((int64_t)z * a.ny) * nx;
    const float2 e0 = row[(int64_t)y0 * nx + k];
    const float2 e1 = (y1 < a.ny) ? row[(int64_t)y1 * nx + k] : make_float2(0.f, 0.f);
    rb[q * nx + (lgx ? (int)brev(k, lgx) : 0)] = make_float2(e0.x - e1.y, e0.y + e1.x);
  }
  __syncthreads();
  fft_rows(rb, lgx, lgr, 1, nx, a.twx, 1.f);
  const float scale = PSI_SCALE_F / (float)(nx * a.ny);
  for (int idx = threadIdx.x; idx < cnt * nx; idx += blockDim.x) {
    const int q = idx >> lgx, x = idx & (nx - 1);
    const int64_t pp = p0 + q;
    const int z = planes[pp / npairs_row];
    const int y0 = 2 * (int)(pp % npairs_row), y1 = y0 + 1;
    const float2 c = rb[q * nx + x];
    int64_t* row = psi + ((int64_t)z * a.ny) * nx;
    row[(int64_t)y0 * nx + x] += llrintf(c.x * scale);
    if (y1 < a.ny) row[(int64_t)y1 * nx + x] += llrintf(c.y * scale);
  }
}

// Mean of the source over the whole fluid (one run, periodic z), from the
// charge kernel's total in dsum[0].
__global__ void k_global_mean(const double* dsum, double inv_nfluid, long long* mean_z, int nz) {
  const long long m = llrint(dsum[0] * inv_nfluid);
  for (int z = threadIdx.x; z < nz; z += blockDim.x) mean_z[z] = m;
}

// Tridiagonal solve along z for one Fourier mode of one run:
//   -x_{z-1} + (lambda + d_z) x_z - x_{z+1} = rhat_z,
// d_z = 2 inside, 1 at a wall end; a cyclic run closes the chain
// (Sherman-Morrison).  The mode (0,0) is singular: its run mean is free, so
// x at the first plane of the run is pinned to 0 and the remaining planes
// are solved (the pinned plane's equation is redundant once the run sum of
// the right-hand side is zero, which the run-mean removal guarantees).
// X, C, Qv: the pencil's values, elimination factors and the Sherman-
// Morrison auxiliary vector, element k at index k * st (shared memory).
struct Run {
  int z0, len, cyclic;
};

__device__ void solve_pencil(float2* X, float* C, float* Qv, int st, int L, float lam,
                             bool singular, bool cyclic) {
  auto thomas = [&](int k0, int k1, auto diagf, bool with_q, auto qrhs) {
    // forward elimination on planes k0..k1-1 (off-diagonals -1)
    float c = 0.f, dq = 0.f;
    float2 d = make_float2(0.f, 0.f);
    for (int k = k0; k < k1; ++k) {
      const float den = diagf(k) + (k > k0 ? c : 0.f);
      const float inv = 1.0f / den;
      const float2 rk = X[k * st];
      d = make_float2((rk.x + (k > k0 ? d.x : 0.f)) * inv, (rk.y + (k > k0 ? d.y : 0.f)) * inv);
      if (with_q) {
        dq = (qrhs(k) + (k > k0 ? dq : 0.f)) * inv;
        Qv[k * st] = dq;
      }
      c = -inv;
      X[k * st] = d;
      C[k * st] = c;
    }
    float2 nx_ = X[(k1 - 1) * st];
    float nq = with_q ? Qv[(k1 - 1) * st] : 0.f;
    for (int k = k1 - 2; k >= k0; --k) {
      const float ck = C[k * st];
      const float2 dk = X[k * st];
      nx_ = make_float2(dk.x - ck * nx_.x, dk.y - ck * nx_.y);
      X[k * st] = nx_;
      if (with_q) {
        nq = Qv[k * st] - ck * nq;
        Qv[k * st] = nq;
      }
    }
  };
  auto noq = [](int) { return 0.f; };
  if (!cyclic) {
    auto diag = [&](int k) { return lam + (float)((k > 0) + (k < L - 1)); };
    if (singular) {
      X[0] = make_float2(0.f, 0.f);
      if (L > 1) thomas(1, L, diag, false, noq);
    } else {
      thomas(0, L, diag, false, noq);
    }
    return;
  }
  if (singular) {
    // pin x_0 = 0; planes 1..L-1 form a Dirichlet chain (diagonal 2)
    X[0] = make_float2(0.f, 0.f);
    thomas(1, L, [](int) { return 2.f; }, false, noq);
    return;
  }
  // Sherman-Morrison: A = T + u v^T, corners -1, gamma = -b,
  // T = A without corners, T_00 = b - gamma, T_LL = b - 1/gamma,
  // u = (gamma, 0, .., 0, -1), v = (1, 0, .., 0, -1/gamma).
  const float b = lam + 2.f;
  const float gam = -b;
  auto tdiag = [&](int k) {
    return k == 0 ? b - gam : (k == L - 1 ? b - 1.0f / gam : b);
  };
  auto urhs = [&](int k) { return k == 0 ? gam : (k == L - 1 ? -1.f : 0.f); };
  thomas(0, L, tdiag, true, urhs);
  const float2 y0 = X[0], yl = X[(L - 1) * st];
  const float q0 = Qv[0], ql = Qv[(L - 1) * st];
  const float den = 1.f + q0 - ql / gam;
  const float2 f = make_float2((y0.x - yl.x / gam) / den, (y0.y - yl.y / gam) / den);
  for (int k = 0; k < L; ++k) {
    const float qk = Qv[k * st];
    const float2 yk = X[k * st];
    X[k * st] = make_float2(yk.x - qk * f.x, yk.y - qk * f.y);
  }
}

constexpr int ZP = 32;  // pencils (Fourier modes) per CTA of the z solve

// One CTA: ZP consecutive modes of one run.  The pencils are staged in
// shared memory (coalesced: consecutive modes are contiguous in each
// plane), solved one per thread, and written back in place.
__global__ void __launch_bounds__(128) k_zsolve(float2* __restrict__ x,
                                                const Run* __restrict__ runs,
                                                SpecArgs a) {
  extern __shared__ float zsm[];
  const Run R = runs[blockIdx.y];
  const int L = R.len;
  const int nxy = a.nx * a.ny;
  const int m0 = blockIdx.x * ZP;
  float2* X = reinterpret_cast<float2*>(zsm);
  float* C = zsm + 2 * ZP * L;
  float* Qv = C + ZP * L;
  for (int idx = threadIdx.x; idx < ZP * L; idx += blockDim.x) {
    const int k = idx / ZP, j = idx - k * ZP;
    int z = R.z0 + k;
    if (z >= a.nz) z -= a.nz;
    if (m0 + j < nxy) X[idx] = x[(int64_t)z * nxy + m0 + j];
  }
  __syncthreads();
  const int j = threadIdx.x;
  if (j < ZP && m0 + j < nxy) {
    const int m = m0 + j;
    solve_pencil(X + j, C + j, Qv + j, ZP, L, a.lam_xy[m], m == 0, R.cyclic != 0);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < ZP * L; idx += blockDim.x) {
    const int k = idx / ZP, jj = idx - k * ZP;
    int z = R.z0 + k;
    if (z >= a.nz) z -= a.nz;
    if (m0 + jj < nxy) x[(int64_t)z * nxy + m0 + jj] = X[idx];
  }
}

// Periodic z axis of power-of-two length: the z operator is circulant, so an
// FFT along z diagonalises it too (eigenvalue 2 - 2 cos(2 pi kz / nz)).
// One CTA: ZP consecutive modes; forward FFT of each pencil in shared
// memory, division by lambda_xy + lambda_z (the (0,0,0) mode, the free mean,
// set to 0), inverse FFT, store.
__global__ void __launch_bounds__(256) k_zfft(float2* __restrict__ x, const float2* __restrict__ twz,
                                              int lgz, SpecArgs a) {
  extern __shared__ float2 zb[];
  const int L = 1 << lgz;
  const int nxy = a.nx * a.ny;
  const int m0 = blockIdx.x * ZP;
  const int lgp = 5;  // log2(ZP)
  // stage: plane k of pencil j at zb[brev(k) * ZP + j] (coalesced loads)
#pragma unroll 8
  for (int idx = threadIdx.x; idx < ZP * L; idx += 256) {
    const int k = idx >> lgp, j = idx & (ZP - 1);
    zb[(int)brev(k, lgz) * ZP + j] =
        (m0 + j < nxy) ? x[(int64_t)k * nxy + m0 + j] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_rows(zb, lgz, lgp, ZP, 1, twz, -1.f);
  // divide by the eigenvalue and put the spectrum back in bit-reversed
  // order for the inverse transform (through registers, one buffer)
  const float invL = 1.0f / (float)L;
  constexpr int PER = 32;  // elements per thread for L <= 256 (ZP * L / 256)
  float2 v[PER];
  int dst[PER];
  int cnt = 0;
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int idx = threadIdx.x + t * 256;
    if (idx < ZP * L) {
      const int kz = idx >> lgp, j = idx & (ZP - 1);
      const int m = m0 + j;
      const float lam = (m < nxy ? a.lam_xy[m] : 1.f) + a.lam_z[kz];
      const float sc = (m == 0 && kz == 0) ? 0.f : invL / lam;
      const float2 c = zb[idx];
      v[t] = make_float2(c.x * sc, c.y * sc);
      dst[t] = (int)brev(kz, lgz) * ZP + j;
      cnt = t + 1;
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < PER; ++t)
    if (t < cnt) zb[dst[t]] = v[t];
  __syncthreads();
  fft_rows(zb, lgz, lgp, ZP, 1, twz, 1.f);
#pragma unroll 8
  for (int idx = threadIdx.x; idx < ZP * L; idx += 256) {
    const int k = idx >> lgp, j = idx & (ZP - 1);
    if (m0 + j < nxy) x[(int64_t)k * nxy + m0 + j] = zb[idx];
  }
}

// Per-plane sums of the fixed-point source (one CTA per plane, exact).
__global__ void __launch_bounds__(256) k_plane_sums(const int64_t* __restrict__ src,
                                                    long long* __restrict__ psum,
                                                    int nxy) {
  __shared__ long long red[8];
  const int64_t base = (int64_t)blockIdx.x * nxy;
  long long v = 0;
  for (int k = threadIdx.x; k < nxy; k += blockDim.x) v += src[base + k];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    psum[blockIdx.x] = t;
  }
}

// Mean of the source over each run, broadcast to its planes (wall planes: 0).
__global__ void k_run_means(const long long* __restrict__ psum, const Run* __restrict__ runs,
                            int nruns, long long* __restrict__ mean_z, int nz, int nxy) {
  for (int z = threadIdx.x; z < nz; z += blockDim.x) mean_z[z] = 0;
  __syncthreads();
  for (int r = threadIdx.x; r < nruns; r += blockDim.x) {
    const Run R = runs[r];
    double tot = 0.0;
    for (int k = 0; k < R.len; ++k) {
      int z = R.z0 + k;
      if (z >= nz) z -= nz;
      tot += (double)psum[z];
    }
    const long long mean = llrint(tot / ((double)R.len * nxy));
    for (int k = 0; k < R.len; ++k) {
      int z = R.z0 + k;
      if (z >= nz) z -= nz;
      mean_z[z] = mean;
    }
  }
}

// Residual with per-plane means: r = s - mean_z - A psi (exact), norms into
// dsum[1], dsum[2].  Wall planes contribute nothing.
__global__ void __launch_bounds__(256) k_res_planes(
    const int64_t* __restrict__ psi, const int64_t* __restrict__ src,
    const long long* __restrict__ mean_z, const unsigned char* __restrict__ plane_fluid,
    float* __restrict__ r, double* dsum, int nx, int ny, int nz, int lgx, int lgxy) {
  __shared__ float red_r[8], red_s[8];
  const int nxy = nx * ny;
  const int64_t N = (int64_t)nxy * nz;
  float rr = 0.f, ss = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    // nx, ny are powers of two: plane, row and column by shifts
    const int z = (int)(i >> lgxy);
    const int k = (int)(i & (nxy - 1));
    if (!plane_fluid[z]) {
      r[i] = 0.f;
      continue;
    }
    const int y = k >> lgx, x = k & (nx - 1);
    const int64_t pc = psi[i];
    int64_t Ap = 0;
    if (nx > 1) {
      Ap += pc - psi[i + (x == nx - 1 ? -(nx - 1) : 1)];
      Ap += pc - psi[i + (x == 0 ? nx - 1 : -1)];
    }
    if (ny > 1) {
      Ap += pc - psi[i + (y == ny - 1 ? -(int64_t)(ny - 1) * nx : nx)];
      Ap += pc - psi[i + (y == 0 ? (int64_t)(ny - 1) * nx : -nx)];
    }
    if (nz > 1) {
      const int zp = (z == nz - 1) ? 0 : z + 1, zm = (z == 0) ? nz - 1 : z - 1;
      if (plane_fluid[zp] && zp != z) Ap += pc - psi[(int64_t)zp * nxy + k];
      if (plane_fluid[zm] && zm != z) Ap += pc - psi[(int64_t)zm * nxy + k];
    }
    const int64_t sfx = src[i] - mean_z[z];
    const float rf = (float)(sfx - Ap);
    r[i] = rf * PSI_INV_SCALE_F;
    rr += rf * rf;
    const float sf = (float)sfx;
    ss += sf * sf;
  }
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

int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return (1 << l) == n ? l : -1;
}

}  // namespace

struct SpectralPlan {
  int nx, ny, nz, lgx, lgy;
  int nplanes = 0, nruns = 0;
  int* planes = nullptr;           // indices of fluid planes
  Run* runs = nullptr;
  unsigned char* plane_fluid = nullptr;
  float2* twx = nullptr;
  float2* twy = nullptr;
  float2* spec = nullptr;          // N complex
  size_t zsmem = 0;                // shared memory of the z solve
  int lgz = -1;                    // log2(nz) when the z axis is one periodic run
  float2* twz = nullptr;           // z twiddles (periodic power-of-two z)
  float* lam_xy = nullptr;         // x-y Laplacian eigenvalues per mode
  float* lam_z = nullptr;          // z Laplacian eigenvalues (periodic power-of-two z)
  int last_iters = 2;              // applications of the previous solve
  bool runs_fit = true;            // z solve fits in shared memory
  float* r = nullptr;              // N
  long long* psum = nullptr;       // nz
  long long* mean_z = nullptr;     // nz
  size_t smem = 0;
};

void spectral_free(lbm_t* h) {
  SpectralPlan* s = h->spec;
  if (!s) return;
  cudaFree(s->planes);
  cudaFree(s->runs);
  cudaFree(s->plane_fluid);
  cudaFree(s->twx);
  cudaFree(s->twy);
  cudaFree(s->twz);
  cudaFree(s->lam_xy);
  cudaFree(s->lam_z);
  cudaFree(s->spec);
  cudaFree(s->r);
  cudaFree(s->psum);
  cudaFree(s->mean_z);
  delete s;
  h->spec = nullptr;
}

lbm_status spectral_setup(lbm_t* h, const uint8_t* solid) {
  spectral_free(h);
  const int nx = h->cfg.nx, ny = h->cfg.ny, nz = h->cfg.nz;
  const int lgx = ilog2(nx), lgy = ilog2(ny);
  if (lgx < 0 || lgy < 0) {
    h->err = "spectral Poisson solver needs power-of-two nx, ny";
    return LBM_EINVAL;
  }
  const int64_t nxy = (int64_t)nx * ny;
  std::vector<unsigned char> pf(nz, 1);
  if (solid) {
    for (int z = 0; z < nz; ++z) {
      int64_t cnt = 0;
      for (int64_t k = 0; k < nxy; ++k) cnt += solid[(int64_t)z * nxy + k] ? 1 : 0;
      if (cnt != 0 && cnt != nxy) {
        h->err = "spectral Poisson solver needs every z-plane all fluid or all wall";
        return LBM_EINVAL;
      }
      pf[z] = cnt == 0;
    }
  }
  std::vector<int> planes;
  for (int z = 0; z < nz; ++z)
    if (pf[z]) planes.push_back(z);
  if (planes.empty()) {
    h->err = "no fluid plane";
    return LBM_EINVAL;
  }
  std::vector<Run> runs;
  if ((int)planes.size() == nz) {
    Run R;
    R.z0 = 0;
    R.len = nz;
    R.cyclic = nz >= 3 ? 1 : 0;
    runs.push_back(R);
  } else {
    // start the scan after a wall plane so that runs never straddle it
    int zs = 0;
    while (pf[zs]) ++zs;
    for (int k = 1; k <= nz; ++k) {
      const int z = (zs + k) % nz;
      if (!pf[z]) continue;
      const int prev = (z - 1 + nz) % nz;
      if (!pf[prev]) {
        Run R;
        R.z0 = z;
        R.len = 0;
        R.cyclic = 0;
        runs.push_back(R);
      }
      runs.back().len++;
    }
  }
  SpectralPlan* s = new SpectralPlan();
  h->spec = s;
  s->nx = nx;
  s->ny = ny;
  s->nz = nz;
  s->lgx = lgx;
  s->lgy = lgy;
  s->nplanes = (int)planes.size();
  s->nruns = (int)runs.size();
  const int64_t N = h->N;
  auto al = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  bool ok = al((void**)&s->planes, planes.size() * sizeof(int)) &&
            al((void**)&s->runs, runs.size() * sizeof(Run)) &&
            al((void**)&s->plane_fluid, nz) && al((void**)&s->twx, std::max(1, nx / 2) * sizeof(float2)) &&
            al((void**)&s->twy, std::max(1, ny / 2) * sizeof(float2)) &&
            al((void**)&s->spec, N * sizeof(float2)) &&
            al((void**)&s->r, N * sizeof(float)) && al((void**)&s->psum, nz * sizeof(long long)) &&
            al((void**)&s->mean_z, nz * sizeof(long long));
  if (!ok) {
    spectral_free(h);
    h->err = "spectral Poisson allocation failed";
    return LBM_ENOMEM;
  }
  auto twiddles = [](int n) {
    std::vector<float2> t(std::max(1, n / 2));
    for (int k = 0; k < n / 2; ++k) {
      const double ang = -2.0 * 3.14159265358979323846 * k / n;
      t[k] = make_float2((float)cos(ang), (float)sin(ang));
    }
    return t;
  };
  auto tx = twiddles(nx), ty = twiddles(ny);
  LBM_CUDA_TRY(h, cudaMemcpy(s->planes, planes.data(), planes.size() * sizeof(int), cudaMemcpyHostToDevice));
  LBM_CUDA_TRY(h, cudaMemcpy(s->runs, runs.data(), runs.size() * sizeof(Run), cudaMemcpyHostToDevice));
  LBM_CUDA_TRY(h, cudaMemcpy(s->plane_fluid, pf.data(), nz, cudaMemcpyHostToDevice));
  LBM_CUDA_TRY(h, cudaMemcpy(s->twx, tx.data(), tx.size() * sizeof(float2), cudaMemcpyHostToDevice));
  LBM_CUDA_TRY(h, cudaMemcpy(s->twy, ty.data(), ty.size() * sizeof(float2), cudaMemcpyHostToDevice));
  {
    // eigenvalues of the periodic x-y Laplacian, 2 - 2 cos(2 pi k / n) per
    // axis, computed once in double precision
    std::vector<float> lxy(nxy);
    for (int ky = 0; ky < ny; ++ky)
      for (int kx = 0; kx < nx; ++kx)
        lxy[(int64_t)ky * nx + kx] =
            (float)((2.0 - 2.0 * cos(2.0 * 3.14159265358979323846 * kx / nx)) +
                    (2.0 - 2.0 * cos(2.0 * 3.14159265358979323846 * ky / ny)));
    std::vector<float> lz(nz);
    for (int kz = 0; kz < nz; ++kz)
      lz[kz] = (float)(2.0 - 2.0 * cos(2.0 * 3.14159265358979323846 * kz / nz));
    if (!al((void**)&s->lam_xy, nxy * sizeof(float)) || !al((void**)&s->lam_z, nz * sizeof(float))) {
      spectral_free(h);
      h->err = "spectral Poisson allocation failed";
      return LBM_ENOMEM;
    }
    LBM_CUDA_TRY(h, cudaMemcpy(s->lam_xy, lxy.data(), nxy * sizeof(float), cudaMemcpyHostToDevice));
    LBM_CUDA_TRY(h, cudaMemcpy(s->lam_z, lz.data(), nz * sizeof(float), cudaMemcpyHostToDevice));
  }
  int optin = 0;
  LBM_CUDA_TRY(h, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev));
  if (runs.size() == 1 && runs[0].cyclic && ilog2(nz) > 0 && nz >= 4 && nz <= 256 &&
      (size_t)ZP * nz * sizeof(float2) <= (size_t)optin) {
    s->lgz = ilog2(nz);
    auto tz = twiddles(nz);
    if (!al((void**)&s->twz, tz.size() * sizeof(float2))) {
      spectral_free(h);
      h->err = "spectral Poisson allocation failed";
      return LBM_ENOMEM;
    }
    LBM_CUDA_TRY(h, cudaMemcpy(s->twz, tz.data(), tz.size() * sizeof(float2), cudaMemcpyHostToDevice));
    const size_t zf = (size_t)ZP * nz * sizeof(float2);
    if (zf > 48 * 1024)
      LBM_CUDA_TRY(h, cudaFuncSetAttribute(k_zfft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zf));
  }
  int lmax = 0;
  for (const Run& R : runs) lmax = std::max(lmax, R.len);
  s->zsmem = (size_t)ZP * lmax * (2 + 1 + 1) * sizeof(float);
  s->runs_fit = s->lgz > 0 || (int)s->zsmem <= optin;
  if (!s->runs_fit && solid) {
    h->err = "spectral Poisson solver: fluid run along z too long for shared memory";
    return LBM_EINVAL;
  }
  // (without walls yet the plan is provisional: set_walls rebuilds it)
  if (s->runs_fit && s->zsmem > 48 * 1024)
    LBM_CUDA_TRY(h, cudaFuncSetAttribute(k_zsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->zsmem));
  s->smem = (size_t)nxy * sizeof(float2);
  {
    const int lgr = std::max(0, 10 - lgx), lgc = std::max(0, 10 - lgy);
    const int xs = (int)(((size_t)nx << lgr) * sizeof(float2)), ys = (int)(((size_t)ny << lgc) * sizeof(float2));
    if (xs > optin || ys > optin) {
      h->err = "spectral Poisson solver: lattice rows too long for shared memory";
      return LBM_EINVAL;
    }
    if (xs > 48 * 1024) {
      LBM_CUDA_TRY(h, cudaFuncSetAttribute(k_fft_x_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, xs));
      LBM_CUDA_TRY(h, cudaFuncSetAttribute(k_fft_x_inv_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, xs));
    }
    if (ys > 48 * 1024)
      LBM_CUDA_TRY(h, cudaFuncSetAttribute(k_fft_y, cudaFuncAttributeMaxDynamicSharedMemorySize, ys));
  }
  return LBM_OK;
}

namespace {

SpecArgs args_of(const SpectralPlan* s) {
  SpecArgs a;
  a.nx = s->nx;
  a.ny = s->ny;
  a.nz = s->nz;
  a.lgx = s->lgx;
  a.lgy = s->lgy;
  a.twx = s->twx;
  a.twy = s->twy;
  a.lam_xy = s->lam_xy;
  a.lam_z = s->lam_z;
  return a;
}

// Residual of the current potential; its norms go to dsum[1 + 2 slot] and
// dsum[2 + 2 slot] (slot 0 is the one the host reads by default).
cudaError_t spec_residual(lbm_t* h, bool to_host = true, int slot = 0) {
  SpectralPlan* s = h->spec;
  Poisson& P = h->ps;
  double* out = P.dsum + 2 * slot;
  cudaError_t e = cudaMemsetAsync(out + 1, 0, 2 * sizeof(double), h->st);
  if (e != cudaSuccess) return e;
  const unsigned nb = (unsigned)std::min<int64_t>(nblk(h->N, 256), h->grid_cap);
  k_res_planes<<<nb, 256, 0, h->st>>>(P.psi[P.cur], P.src, s->mean_z, s->plane_fluid, s->r,
                                      out, s->nx, s->ny, s->nz, s->lgx, s->lgx + s->lgy);
  ++h->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (!to_host) return cudaSuccess;
  return cudaMemcpyAsync(P.hsum, P.dsum, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->st);
}

cudaError_t spec_means(lbm_t* h) {
  SpectralPlan* s = h->spec;
  Poisson& P = h->ps;
  if (s->nruns == 1 && (int)s->nplanes == s->nz) {
    // one periodic run: the mean over all fluid, already summed by the
    // source kernel
    k_global_mean<<<1, 256, 0, h->st>>>(P.dsum, 1.0 / (double)h->nfluid, s->mean_z, s->nz);
    ++h->launches;
    return cudaGetLastError();
  }
  k_plane_sums<<<s->nz, 256, 0, h->st>>>(P.src, s->psum, s->nx * s->ny);
  k_run_means<<<1, 256, 0, h->st>>>(s->psum, s->runs, s->nruns, s->mean_z, s->nz, s->nx * s->ny);
  h->launches += 2;
  return cudaGetLastError();
}

cudaError_t spec_apply(lbm_t* h) {
  SpectralPlan* s = h->spec;
  Poisson& P = h->ps;
  const SpecArgs a = args_of(s);
  const int npairs_row = (s->ny + 1) / 2;
  const int64_t total_pairs = (int64_t)s->nplanes * npairs_row;
  // about 1024 complex values per CTA in each pass
  const int lgr = std::max(0, 10 - s->lgx), lgc = std::max(0, 10 - s->lgy);
  const unsigned gx = (unsigned)((total_pairs + (1 << lgr) - 1) >> lgr);
  const size_t xs = ((size_t)s->nx << lgr) * sizeof(float2);
  const int cols = (s->nx + (1 << lgc) - 1) >> lgc;
  const size_t ys = ((size_t)s->ny << lgc) * sizeof(float2);
  k_fft_x_fwd<<<gx, 256, xs, h->st>>>(s->r, s->spec, s->planes, npairs_row, total_pairs, a, lgr);
  k_fft_y<<<s->nplanes * cols, 256, ys, h->st>>>(s->spec, s->planes, cols, a, -1.f, lgc);
  if (s->lgz > 0) {
    k_zfft<<<nblk((int64_t)s->nx * s->ny, ZP), 256, (size_t)ZP * s->nz * sizeof(float2), h->st>>>(
        s->spec, s->twz, s->lgz, a);
  } else {
    dim3 g(nblk((int64_t)s->nx * s->ny, ZP), s->nruns);
    k_zsolve<<<g, 128, s->zsmem, h->st>>>(s->spec, s->runs, a);
  }
  k_fft_y<<<s->nplanes * cols, 256, ys, h->st>>>(s->spec, s->planes, cols, a, 1.f, lgc);
  k_fft_x_inv_apply<<<gx, 256, xs, h->st>>>(s->spec, s->planes, npairs_row, total_pairs, a,
                                             P.psi[P.cur], lgr);
  h->launches += 5;
  return cudaGetLastError();
}

}  // namespace

lbm_status spectral_solve(lbm_t* h, double tol, int maxit, int* iters, double* rel_res) {
  SpectralPlan* s = h->spec;
  Poisson& P = h->ps;
  if (!s->runs_fit) {
    h->err = "spectral Poisson solver: fluid run along z too long for shared memory";
    return LBM_EINVAL;
  }
  LBM_CUDA_TRY(h, spec_means(h));
  LBM_CUDA_TRY(h, spec_residual(h));
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  double rn = sqrt(P.hsum[1]), sn = sqrt(P.hsum[2]);
  auto conv = [&]() { return rn <= tol * sn || rn <= 2.0 * sqrt((double)h->nfluid); };
  if (!conv() && nn_active(h)) {
    bool applied = false;
    float* dpsi = nullptr;
    lbm_status st = nn_before_solve(h, s->r, 0, s->nz, rn * PSI_INV_SCALE / sqrt((double)h->nfluid),
                                    &applied, &dpsi);
    if (st != LBM_OK) return st;
    if (applied) {
      const double rn_old = rn;
      LBM_CUDA_TRY(h, spec_residual(h));
      LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
      rn = sqrt(P.hsum[1]);
      if (rn < rn_old) {
        nn_record(h, rn / rn_old);
      } else {
        st = nn_revert(h, dpsi);
        if (st != LBM_OK) return st;
        LBM_CUDA_TRY(h, spec_residual(h));
        LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
        rn = sqrt(P.hsum[1]);
      }
    }
  }
  int it = 0;
  if (!nn_active(h) && !conv()) {
    // Queue the number of applications the previous solve needed, each
    // followed by its residual in its own slot, and read all norms with one
    // host synchronisation.
    const int k = std::max(1, std::min(std::min(s->last_iters, maxit), Poisson::NSLOT - 1));
    for (int i = 1; i <= k; ++i) {
      LBM_CUDA_TRY(h, spec_apply(h));
      LBM_CUDA_TRY(h, spec_residual(h, false, i));
    }
    LBM_CUDA_TRY(h, cudaMemcpyAsync(P.hsum, P.dsum, (3 + 2 * k) * sizeof(double),
                                    cudaMemcpyDeviceToHost, h->st));
    LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
    int need = k;
    for (int i = 1; i <= k; ++i) {
      const double ri = sqrt(P.hsum[1 + 2 * i]), si = sqrt(P.hsum[2 + 2 * i]);
      if (ri <= tol * si || ri <= 2.0 * sqrt((double)h->nfluid)) {
        need = i;
        break;
      }
    }
    rn = sqrt(P.hsum[1 + 2 * k]);
    sn = sqrt(P.hsum[2 + 2 * k]);
    it = k;
    s->last_iters = need;
  }
  while (!conv() && it < maxit) {
    LBM_CUDA_TRY(h, spec_apply(h));
    LBM_CUDA_TRY(h, spec_residual(h));
    LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
    rn = sqrt(P.hsum[1]);
    sn = sqrt(P.hsum[2]);
    if (!isfinite(rn) || !isfinite(sn)) {
      h->err = "Poisson residual is not finite";
      return LBM_EUNSTABLE;
    }
    ++it;
    s->last_iters = it;
  }
  if (iters) *iters = it;
  if (rel_res) *rel_res = sn > 0.0 ? rn / sn : 0.0;
  if (!conv()) {
    h->err = "Poisson solve did not reach the tolerance within the iteration cap";
    return LBM_ENOCONV;
  }
  return LBM_OK;
}


// ---------------------------------------------------------------------------
// Whole-step CUDA graphs.  One graph per population parity holds a full time
// step: charge density, run means, residual, a device-side while loop
// (conditional graph node) of spectral applications + residual + test, and
// the fused stream/collide.  Steps are replayed back to back with no host
// round trip; the test kernel keeps the per-step status on the device.
// ---------------------------------------------------------------------------
namespace {

struct GraphStatus {
  uint32_t step;       // time step (read by the stream/collide kernel)
  int iters;           // Poisson iterations of the current step
  long long total;     // iterations summed over replayed steps
  int fails;           // steps whose solve stopped at the iteration cap
  int pad;
  double rel;          // final relative residual of the last step
};

// Convergence test of the last residual (one thread): sets the loop
// condition of the enclosing conditional node.
__global__ void k_graph_check(const double* __restrict__ dsum, GraphStatus* st, double tol,
                              double floor2, int maxit, int first,
                              cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double rn2 = dsum[1], sn2 = dsum[2];
  const bool conv = rn2 <= tol * tol * sn2 || rn2 <= floor2;
  if (first) {
    st->iters = 0;
    st->step += 1;
  } else {
    st->iters += 1;
  }
  const bool more = !conv && st->iters < maxit;
  cudaGraphSetConditional(cond, more ? 1u : 0u);
  st->rel = sn2 > 0.0 ? sqrt(rn2 / sn2) : 0.0;
  if (!more) {
    st->total += st->iters;
    if (!conv) st->fails += 1;
  }
}

}  // namespace

void spectral_graph_free(lbm_t* h) {
  for (int k = 0; k < 2; ++k) {
    if (h->step_graph[k]) cudaGraphExecDestroy(h->step_graph[k]);
    h->step_graph[k] = nullptr;
  }
}

namespace {

lbm_status build_step_graph(lbm_t* h, int parity) {
  Poisson& P = h->ps;
  const int saved_cur = h->cur;
  h->cur = parity;
  GraphStatus* gs = reinterpret_cast<GraphStatus*>(h->gstatus);
  const double tol = h->cfg.poisson_tol;
  const double floor2 = 4.0 * (double)h->nfluid;
  const int maxit = h->cfg.poisson_maxit;
  cudaGraph_t G = nullptr;
  LBM_CUDA_TRY(h, cudaGraphCreate(&G, 0));
  cudaGraphConditionalHandle cond;
  LBM_CUDA_TRY(h, cudaGraphConditionalHandleCreate(&cond, G, 0, cudaGraphCondAssignDefault));
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  const int64_t l0 = h->launches;
  // part A: source, means, first residual and test
  LBM_CUDA_TRY(h, cudaStreamBeginCaptureToGraph(h->st, G, nullptr, nullptr, 0, mode));
  cudaError_t e = cudaMemsetAsync(P.dsum, 0, 3 * sizeof(double), h->st);
  if (e == cudaSuccess) e = launch_charge(h);
  if (e == cudaSuccess) e = spec_means(h);
  if (e == cudaSuccess) e = spec_residual(h, false);
  if (e == cudaSuccess) {
    k_graph_check<<<1, 32, 0, h->st>>>(P.dsum, gs, tol, floor2, maxit, 1, cond);
    ++h->launches;
    e = cudaGetLastError();
  }
  std::vector<cudaGraphNode_t> deps;
  if (e == cudaSuccess) {
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    e = cudaStreamGetCaptureInfo(h->st, &cs, nullptr, nullptr, &d, nullptr, &nd);
    if (e == cudaSuccess) deps.assign(d, d + nd);
  }
  cudaGraph_t Gc = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(h->st, &Gc);
  if (e == cudaSuccess) e = e2;
  // the conditional while node and its body
  cudaGraphNode_t cnode = nullptr;
  cudaGraph_t body = nullptr;
  if (e == cudaSuccess) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&cnode, G, deps.data(), nullptr, deps.size(), &cp);
    if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
  }
  const int64_t l1 = h->launches;
  if (e == cudaSuccess) {
    e = cudaStreamBeginCaptureToGraph(h->st, body, nullptr, nullptr, 0, mode);
    if (e == cudaSuccess) {
      cudaError_t eb = spec_apply(h);
      if (eb == cudaSuccess) eb = spec_residual(h, false);
      if (eb == cudaSuccess) {
        k_graph_check<<<1, 32, 0, h->st>>>(P.dsum, gs, tol, floor2, maxit, 0, cond);
        ++h->launches;
        eb = cudaGetLastError();
      }
      cudaGraph_t bb = nullptr;
      e = cudaStreamEndCapture(h->st, &bb);
      if (e == cudaSuccess) e = eb;
    }
  }
  const int64_t l2 = h->launches;
  // part B: fused stream/collide after the loop
  if (e == cudaSuccess) {
    e = cudaStreamBeginCaptureToGraph(h->st, G, &cnode, nullptr, 1, mode);
    if (e == cudaSuccess) {
      cudaError_t eb = launch_stream_collide(h);
      cudaGraph_t gg = nullptr;
      e = cudaStreamEndCapture(h->st, &gg);
      if (e == cudaSuccess) e = eb;
    }
  }
  const int64_t l3 = h->launches;
  h->launches = l0;
  h->cur = saved_cur;
  cudaGraphExec_t ex = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, G, 0);
  cudaGraphDestroy(G);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->err = std::string("step graph construction failed: ") + cudaGetErrorString(e);
    return LBM_ECUDA;
  }
  h->step_graph[parity] = ex;
  h->graph_kernels_fixed = (int)((l1 - l0) + (l3 - l2));
  h->graph_kernels_iter = (int)(l2 - l1);
  return LBM_OK;
}

}  // namespace

lbm_status spectral_graph_steps(lbm_t* h, int nsteps) {
  if (!h->spec->runs_fit) {
    h->err = "spectral Poisson solver: fluid run along z too long for shared memory";
    return LBM_EINVAL;
  }
  if (!h->gstatus) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(GraphStatus)) != cudaSuccess) {
      cudaGetLastError();
      h->err = "graph status allocation failed";
      return LBM_ENOMEM;
    }
    GraphStatus z = {};
    z.step = (uint32_t)h->tstep;
    cudaMemcpy(p, &z, sizeof z, cudaMemcpyHostToDevice);
    h->gstatus = p;
    if (cudaMallocHost(&h->hstatus, sizeof(GraphStatus)) != cudaSuccess) {
      h->err = "pinned allocation failed";
      return LBM_ENOMEM;
    }
  }
  for (int k = 0; k < 2; ++k)
    if (!h->step_graph[k]) {
      lbm_status s = build_step_graph(h, k);
      if (s != LBM_OK) return s;
    }
  GraphStatus* hs = reinterpret_cast<GraphStatus*>(h->hstatus);
  // status before, to count this call's iterations and failures
  LBM_CUDA_TRY(h, cudaMemcpyAsync(hs, h->gstatus, sizeof(GraphStatus), cudaMemcpyDeviceToHost, h->st));
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  const long long total0 = hs->total;
  const int fails0 = hs->fails;
  for (int k = 0; k < nsteps; ++k) {
    LBM_CUDA_TRY(h, cudaGraphLaunch(h->step_graph[h->cur], h->st));
    h->cur ^= 1;
    ++h->tstep;
  }
  LBM_CUDA_TRY(h, cudaMemcpyAsync(hs, h->gstatus, sizeof(GraphStatus), cudaMemcpyDeviceToHost, h->st));
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  const long long iters = hs->total - total0;
  h->launches += (int64_t)nsteps * h->graph_kernels_fixed + iters * h->graph_kernels_iter;
  h->t_cnt[1] += iters;
  h->t_cnt[0] += nsteps;
  h->t_cnt[2] += nsteps;
  h->last_iters = hs->iters;
  h->last_res = hs->rel;
  h->psi_valid = true;
  if (hs->fails != fails0) {
    h->err = "a Poisson solve inside the step graph stopped at the iteration cap";
    return LBM_ENOCONV;
  }
  return LBM_OK;
}

}  // namespace lbm_gb300
