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
// fixed-point residual: one or two applications reach 1e-8.
//
// One application is three kernels:
//   k_plane_fwd  one CTA per fluid plane (or several small planes): the
//                exact residual of the plane, its real-to-complex 2-D FFT
//                (two real rows per complex transform along x, then the
//                nx/2 + 1 columns along y), the half spectrum to memory;
//   k_zfft / k_zsolve  along z for every mode: FFT, division by the
//                eigenvalue, inverse FFT (one periodic power-of-two run),
//                else one tridiagonal solve per mode and run;
//   k_plane_inv  inverse 2-D FFT of each plane fused with psi += round(e).
// The FFTs keep eight values per thread in registers (Stockham stages of
// radix 8, then 4 or 2) and exchange through shared memory between stages.
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
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// a * (sign i)
__device__ __forceinline__ float2 cmul_si(float2 a, float sign) {
  return make_float2(-sign * a.y, sign * a.x);
}

// Small DFTs in place, X_q = sum_r a_r exp(sign 2 pi i r q / R).
__device__ __forceinline__ void dft2(float2& a0, float2& a1) {
  const float2 t = a0;
  a0 = cadd(t, a1);
  a1 = csub(t, a1);
}
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3, float sign) {
  const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
  const float2 t2 = cadd(a1, a3), t3 = cmul_si(csub(a1, a3), sign);
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}
// radix 8 as two radix-4 transforms of the even and odd inputs joined by
// the twiddles exp(sign 2 pi i q / 8), q = 0..3
__device__ __forceinline__ void dft8(float2 (&v)[8], float sign) {
  dft4(v[0], v[2], v[4], v[6], sign);
  dft4(v[1], v[3], v[5], v[7], sign);
  const float c = 0.70710678118654752f;
  const float2 o0 = v[1];
  const float2 o1 = cmul(v[3], make_float2(c, sign * c));
  const float2 o2 = cmul_si(v[5], sign);
  const float2 o3 = cmul(v[7], make_float2(-c, sign * c));
  const float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}

// Shared-memory line of one transform.  PadLine: contiguous, one spare slot
// after every eight elements (the first Stockham stage writes with stride 8,
// which would hit two banks only).  StrideLine: element d at d * es, used
// when the lanes of a warp belong to different transforms (consecutive
// lanes, consecutive lines).
struct PadLine {
  float2* p;
  __device__ __forceinline__ float2& operator[](int d) const { return p[d + (d >> 3)]; }
};
struct StrideLine {
  float2* p;
  int es;
  __device__ __forceinline__ float2& operator[](int d) const { return p[d * es]; }
};
__host__ __device__ constexpr int padded_len(int L) { return L + (L >> 3); }

template <bool CTA>
__device__ __forceinline__ void line_sync() {
  if (CTA)
    __syncthreads();
  else
    __syncwarp();
}

// FFT of length L = 2^LG (8 <= L <= 256) held by T = L / 8 threads, thread t
// holding elements t + u T (u = 0..7) before and after.  Stockham autosort
// stages (the formulation of Stockham's self-sorting FFT used for GPUs by
// Govindaraju et al., SC 2008): the stage of radix R after earlier radices
// of product Ns takes butterfly j's inputs x[j + r L/R], multiplies input r
// by w^(r (j mod Ns) L / (Ns R)) with w = exp(sign 2 pi i / L), transforms
// them, and writes output q to (j div Ns) Ns R + (j mod Ns) + q Ns.  With
// eight values per thread a radix-R stage is 8/R butterflies j = t + s T per
// thread; the last stage's outputs fall on j + q L/R = t + (s + q 8/R) T,
// the starting distribution, so they stay in registers.  tw[m] =
// exp(-2 pi i m / L), m < L (the inverse conjugates it).  CTA: the T
// threads are in different warps (barrier), else in one warp.  LG is a
// template parameter so that every stage's radix, shifts and offsets are
// constants.
template <int LG, bool CTA, class Line>
__device__ __forceinline__ void fft_regs(float2 (&v)[8], int t, Line line,
                                         const float2* __restrict__ tw, float sign) {
  constexpr int T = 1 << (LG - 3);
  constexpr int NST = (LG + 2) / 3;
#pragma unroll
  for (int st = 0; st < NST; ++st) {
    const int lns = 3 * st;                              // log2 Ns
    const int lr = LG - lns >= 3 ? 3 : LG - lns;         // log2 R
    const int Ns = 1 << lns;
    const int tws = LG - lns - lr;                       // log2(L / (Ns R))
    if (lr == 3) {
      if (lns > 0) {
        const int k = t & (Ns - 1);
#pragma unroll
        for (int r = 1; r < 8; ++r) {
          float2 w = __ldg(tw + ((r * k) << tws));
          w.y *= -sign;
          v[r] = cmul(v[r], w);
        }
      }
      dft8(v, sign);
    } else if (lr == 2) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (lns > 0) {
          const int k = (t + s * T) & (Ns - 1);
#pragma unroll
          for (int r = 1; r < 4; ++r) {
            float2 w = __ldg(tw + ((r * k) << tws));
            w.y *= -sign;
            v[s + 2 * r] = cmul(v[s + 2 * r], w);
          }
        }
        dft4(v[s], v[s + 2], v[s + 4], v[s + 6], sign);
      }
    } else {
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if (lns > 0) {
          const int k = (t + s * T) & (Ns - 1);
          float2 w = __ldg(tw + (k << tws));
          w.y *= -sign;
          v[s + 4] = cmul(v[s + 4], w);
        }
        dft2(v[s], v[s + 4]);
      }
    }
    if (st == NST - 1) break;
    // slot u = s + G q holds output q of butterfly j = t + s T (G = 8 / R)
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int s = u & ((8 >> lr) - 1), q = u >> (3 - lr);
      const int j = t + s * T;
      line[((j >> lns) << (lns + lr)) + (j & (Ns - 1)) + (q << lns)] = v[u];
    }
    line_sync<CTA>();
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = line[t + u * T];
    line_sync<CTA>();
  }
}

// Calls F<LG>(args...) for the runtime lg in [3, 8].
#define LBM_LG_DISPATCH(lg, F, ...) \
  switch (lg) {                     \
    case 3: F<3>(__VA_ARGS__); break; \
    case 4: F<4>(__VA_ARGS__); break; \
    case 5: F<5>(__VA_ARGS__); break; \
    case 6: F<6>(__VA_ARGS__); break; \
    case 7: F<7>(__VA_ARGS__); break; \
    default: F<8>(__VA_ARGS__); break; \
  }

// Squared norms are accumulated by CTA b into partial NACC slot b mod NACC:
// one FP32 atomic per CTA and quantity (FP64 atomics are slow on this GPU),
// spread over addresses so that thousands of CTAs do not queue on one, and
// scaled by 2^-40 so that sums of squares of fixed-point values stay far
// inside the FP32 range.  A norm slot holds NACC partials of |r|^2 followed
// by NACC of |s - <s>|^2; the reader sums them in FP64 and scales back.  The
// norms only decide convergence, so FP32 partials (relative error ~1e-6)
// are ample.
constexpr int NACC = 64;
constexpr float NORM_SCALE = 1.0f / 1099511627776.0f;  // 2^-40

__device__ __forceinline__ void add_norms(float* acc, float rr, float ss, float* red_r,
                                          float* red_s) {
  for (int off = 16; off > 0; off >>= 1) {
    rr += __shfl_down_sync(0xffffffffu, rr, off);
    ss += __shfl_down_sync(0xffffffffu, ss, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red_r[threadIdx.x >> 5] = rr * NORM_SCALE;
    red_s[threadIdx.x >> 5] = ss * NORM_SCALE;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float tr = 0.f, ts = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      tr += red_r[i];
      ts += red_s[i];
    }
    const int k = blockIdx.x & (NACC - 1);
    atomicAdd(acc + k, tr);
    atomicAdd(acc + NACC + k, ts);
  }
}

struct SpecArgs {
  int nx, ny, nz, lgx, lgy, lgz;
  int H;       // nx / 2: the half spectrum keeps kx = 0..H
  int mxy;     // modes per plane, (H + 1) ny, mode m = ky (H + 1) + kx
  int lgtp;    // log2 of the threads per plane in the plane kernels (nx ny / 16)
  const float2* twx;  // exp(-2 pi i m / n), m < n, per axis
  const float2* twy;
  const float2* twz;
  const float* lamx;  // 2 - 2 cos(2 pi k / n): H + 1, ny and nz values
  const float* lamy;
  const float* lamz;
};

template <int G>
__device__ __forceinline__ void loadg(const int64_t* __restrict__ p, int64_t (&v)[G]) {
#pragma unroll
  for (int k = 0; k < G / 2; ++k) {
    const longlong2 a = __ldg(reinterpret_cast<const longlong2*>(p) + k);
    v[2 * k] = a.x;
    v[2 * k + 1] = a.y;
  }
}

// Plane data for the residual: offsets of the planes z +- 1, whether their
// faces are open (fluid planes), and the plane's source mean.
struct PlaneNbr {
  int64_t dup, ddn;
  bool up, dn;
  long long mean;
};

__device__ __forceinline__ PlaneNbr plane_nbr(const unsigned char* __restrict__ plane_fluid,
                                              const long long* __restrict__ mean_z, int z,
                                              int nxy, int nz) {
  PlaneNbr g;
  const int zp = (z == nz - 1) ? 0 : z + 1, zm = (z == 0) ? nz - 1 : z - 1;
  g.dup = (int64_t)(zp - z) * nxy;
  g.ddn = (int64_t)(zm - z) * nxy;
  g.up = nz > 1 && zp != z && __ldg(plane_fluid + zp);
  g.dn = nz > 1 && zm != z && __ldg(plane_fluid + zm);
  g.mean = __ldg(mean_z + z);
  return g;
}

// Exact residual r = s - <s> - A psi at the G (2 or 4) consecutive nodes
// x0..x0+G-1 (x0 a multiple of G) of row y of a plane, i0 the index of
// (x0, y): 16-byte loads of the row, the rows y +- 1 and the planes z +- 1
// (loaded whether or not their faces are open, so that no load waits on
// the plane data), two scalar loads for the x neighbours at the ends.  r in
// fixed-point units (FP32); rr, ss accumulate |r|^2 and |s - <s>|^2.
template <int G>
__device__ __forceinline__ void residual_g(const int64_t* __restrict__ psi,
                                           const int64_t* __restrict__ src, int64_t i0, int x0,
                                           int y, int nx, int ny, const PlaneNbr& g,
                                           float (&r)[G], float& rr, float& ss) {
  int64_t c[G], yp[G], ym[G], up[G], dn[G], sv[G];
  loadg<G>(psi + i0, c);
  const int64_t row = i0 - x0;
  const int64_t xl = __ldg(psi + row + ((x0 - 1) & (nx - 1)));
  const int64_t xr = __ldg(psi + row + ((x0 + G) & (nx - 1)));
  loadg<G>(psi + (y == ny - 1 ? i0 - (int64_t)(ny - 1) * nx : i0 + nx), yp);
  loadg<G>(psi + (y == 0 ? i0 + (int64_t)(ny - 1) * nx : i0 - nx), ym);
  loadg<G>(psi + i0 + g.dup, up);
  loadg<G>(psi + i0 + g.ddn, dn);
  loadg<G>(src + i0, sv);
#pragma unroll
  for (int j = 0; j < G; ++j) {
    const int64_t left = j == 0 ? xl : c[j - 1], right = j == G - 1 ? xr : c[j + 1];
    int64_t Ap = 4 * c[j] - left - right - yp[j] - ym[j];
    if (g.up) Ap += c[j] - up[j];
    if (g.dn) Ap += c[j] - dn[j];
    const int64_t sfx = sv[j] - g.mean;
    const float rf = i64_to_f32(sfx - Ap);
    const float sf = i64_to_f32(sfx);
    rr += rf * rf;
    ss += sf * sf;
    r[j] = rf;
  }
}

// Shared memory of one plane in the plane kernels: the half spectrum
// (mxy values, row stride H + 1, odd) and the padded lines of the row or
// column transforms (nx ny / 2 elements with padding).
__host__ __device__ constexpr int plane_smem_words(int nx, int ny) {
  return (nx / 2 + 1) * ny + (nx * ny / 16) * 9;
}

// Phases of the plane kernels, templated on the transform's log2 length.
// S: the plane's half spectrum (row stride rs = nx/2 + 1); scr: the padded
// lines (one per row pair along x, one per packed column along y).

// x forward: rows 2q, 2q + 1 (residual rows staged in the pair's own line,
// row 2q at float offset 0, row 2q + 1 at nx) -> one complex FFT -> half
// spectra R_2q(k) = (C(k) + conj C(-k)) / 2, R_2q+1(k) = (C(k) - conj C(-k)) / 2i.
template <int LGX>
__device__ __forceinline__ void xphase_fwd(float2* S, float2* scr, int w, bool valid,
                                           const float2* __restrict__ twx) {
  constexpr int NX = 1 << LGX, TX = NX >> 3, H = NX >> 1, RS = H + 1;
  const int q = w >> (LGX - 3), t = w & (TX - 1);
  const PadLine line{scr + q * padded_len(NX)};
  const int y0 = 2 * q;
  float2 v[8];
  {
    const float* rb = reinterpret_cast<const float*>(scr + q * padded_len(NX));
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int x = t + u * TX;
      v[u] = valid ? make_float2(rb[x], rb[NX + x]) : make_float2(0.f, 0.f);
    }
    __syncwarp();
  }
  fft_regs<LGX, false>(v, t, line, twx, -1.f);
#pragma unroll
  for (int u = 0; u < 8; ++u) line[t + u * TX] = v[u];
  __syncwarp();
#pragma unroll
  for (int u = 0; u < 5; ++u) {
    const int k = t + u * TX;  // k <= H: u < 4, or u == 4 and t == 0
    if (u < 4 || t == 0) {
      const float2 c = v[u], cm = line[(NX - k) & (NX - 1)];
      S[y0 * RS + k] = make_float2(0.5f * (c.x + cm.x), 0.5f * (c.y - cm.y));
      S[(y0 + 1) * RS + k] = make_float2(0.5f * (c.y + cm.y), -0.5f * (c.x - cm.x));
    }
  }
}

// y forward: columns kx = 1..H-1, and kx = 0, H packed as one complex column
// (both real), unpacked after the FFT: F0 = (Z + conj Z(-k)) / 2,
// FH = (Z - conj Z(-k)) / 2i.
template <int LGY>
__device__ __forceinline__ void yphase_fwd(float2* S, float2* scr, int w, int H,
                                           const float2* __restrict__ twy) {
  constexpr int NY = 1 << LGY, TY = NY >> 3;
  const int rs = H + 1;
  const int c = w >> (LGY - 3), t = w & (TY - 1);
  const PadLine line{scr + c * padded_len(NY)};
  float2 v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int y = t + u * TY;
    v[u] = c == 0 ? make_float2(S[y * rs].x, S[y * rs + H].x) : S[y * rs + c];
  }
  fft_regs<LGY, false>(v, t, line, twy, -1.f);
#pragma unroll
  for (int u = 0; u < 8; ++u) line[t + u * TY] = v[u];
  __syncwarp();
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int ky = t + u * TY;
    if (c == 0) {
      const float2 zk = v[u], zm = line[(NY - ky) & (NY - 1)];
      S[ky * rs] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      S[ky * rs + H] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    } else {
      S[ky * rs + c] = v[u];
    }
  }
}

// y inverse: column 0 carries kx = 0 and H packed as F0 + i FH, whose
// inverse is f0 + i fH with both real.
template <int LGY>
__device__ __forceinline__ void yphase_inv(float2* S, float2* scr, int w, int H,
                                           const float2* __restrict__ twy) {
  constexpr int NY = 1 << LGY, TY = NY >> 3;
  const int rs = H + 1;
  const int c = w >> (LGY - 3), t = w & (TY - 1);
  const PadLine line{scr + c * padded_len(NY)};
  float2 v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int y = t + u * TY;
    if (c == 0) {
      const float2 f0 = S[y * rs], fh = S[y * rs + H];
      v[u] = make_float2(f0.x - fh.y, f0.y + fh.x);
    } else {
      v[u] = S[y * rs + c];
    }
  }
  fft_regs<LGY, false>(v, t, line, twy, 1.f);
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int y = t + u * TY;
    if (c == 0) {
      S[y * rs] = make_float2(v[u].x, 0.f);
      S[y * rs + H] = make_float2(v[u].y, 0.f);
    } else {
      S[y * rs + c] = v[u];
    }
  }
}

// x inverse: rows 2q, 2q+1 as C(k) = E_2q(k) + i E_2q+1(k) over the full k
// range (E(k) = conj E(nx - k) above H); the inverse gives e_2q + i e_2q+1;
// psi += round(e / (nx ny)) in fixed point (rows of the plane at psi_z).
template <int LGX>
__device__ __forceinline__ void xphase_inv(const float2* S, float2* scr, int w, int ny,
                                           bool valid, int64_t* __restrict__ psi_z,
                                           const float2* __restrict__ twx) {
  constexpr int NX = 1 << LGX, TX = NX >> 3, H = NX >> 1, RS = H + 1;
  const int q = w >> (LGX - 3), t = w & (TX - 1);
  const PadLine line{scr + q * padded_len(NX)};
  const int y0 = 2 * q;
  float2 v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int k = t + u * TX;
    float2 e0, e1;
    if (k <= H) {
      e0 = S[y0 * RS + k];
      e1 = S[(y0 + 1) * RS + k];
    } else {
      e0 = S[y0 * RS + NX - k];
      e1 = S[(y0 + 1) * RS + NX - k];
      e0.y = -e0.y;
      e1.y = -e1.y;
    }
    v[u] = make_float2(e0.x - e1.y, e0.y + e1.x);
  }
  fft_regs<LGX, false>(v, t, line, twx, 1.f);
  if (valid) {
    const float scale = PSI_SCALE_F / (float)(NX * ny);
    int64_t* row0 = psi_z + (int64_t)y0 * NX;
    int64_t* row1 = row0 + NX;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int x = t + u * TX;
      row0[x] += f32_to_i64_rn(v[u].x * scale);
      row1[x] += f32_to_i64_rn(v[u].y * scale);
    }
  }
}

// Forward plane kernel.  Thread w of a plane's TP = nx ny / 16 threads is,
// along x, thread t = w mod (nx/8) of row pair q = w div (nx/8) (rows 2q and
// 2q + 1 packed as C = r_2q + i r_2q+1), and along y thread w mod (ny/8) of
// column c = w div (ny/8) (c = 0 carries the real columns kx = 0 and kx = H
// packed the same way).  The residual r = s - <s> - A psi is computed
// exactly in int64 (two nodes per thread and step); its squared norms (and
// the source's) are added to the norm slot given.  planes: the fluid
// planes' indices, or NULL when every plane is fluid (plane index = CTA slot
// index).
__global__ void __launch_bounds__(1024, 1) k_plane_fwd(
    const int64_t* __restrict__ psi, const int64_t* __restrict__ src,
    const long long* __restrict__ mean_z, const unsigned char* __restrict__ plane_fluid,
    const int* __restrict__ planes, int nplanes, float2* __restrict__ spec, float* norms,
    SpecArgs a) {
  extern __shared__ __align__(16) float2 sm[];
  __shared__ float red_r[32], red_s[32];
  const int nx = a.nx, ny = a.ny;
  const int tp = 1 << a.lgtp;
  const int slot = threadIdx.x >> a.lgtp, w = threadIdx.x & (tp - 1);
  const int pi = blockIdx.x * (blockDim.x >> a.lgtp) + slot;
  const bool valid = pi < nplanes;
  const int z = !valid ? 0 : (planes ? planes[pi] : pi);
  float2* S = sm + (size_t)slot * plane_smem_words(nx, ny);
  float2* scr = S + a.mxy;
  float rr = 0.f, ss = 0.f;

  // residual of the plane, two consecutive x per thread and step, into the
  // line of its row pair; a transform later overwrites only its own line,
  // after reading it
  if (valid) {
    const PlaneNbr g = plane_nbr(plane_fluid, mean_z, z, nx * ny, a.nz);
    const int64_t* psi_z = psi + (int64_t)z * nx * ny;
    const int64_t* src_z = src + (int64_t)z * nx * ny;
    const int lgp = a.lgx - 1;  // pairs per row
    // nx ny / 2 pairs over nx ny / 16 threads: eight per thread
#pragma unroll 2
    for (int j = 0; j < 8; ++j) {
      const int gi = w + j * tp;
      const int y = gi >> lgp, x0 = (gi & ((1 << lgp) - 1)) << 1;
      float r2[2];
      residual_g<2>(psi_z, src_z, y * nx + x0, x0, y, nx, ny, g, r2, rr, ss);
      float* rb = reinterpret_cast<float*>(scr + (y >> 1) * padded_len(nx)) + (y & 1) * nx + x0;
      rb[0] = r2[0] * PSI_INV_SCALE_F;
      rb[1] = r2[1] * PSI_INV_SCALE_F;
    }
  }
  __syncthreads();
  LBM_LG_DISPATCH(a.lgx, xphase_fwd, S, scr, w, valid, a.twx)
  __syncthreads();
  LBM_LG_DISPATCH(a.lgy, yphase_fwd, S, scr, w, a.H, a.twy)
  __syncthreads();
  if (valid) {
    float4* dst = reinterpret_cast<float4*>(spec + (int64_t)z * a.mxy);
    const float4* s4 = reinterpret_cast<const float4*>(S);
    // mxy / 2 = 4 tp + ny / 2 pairs of values (mxy even, plane offset even)
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const int i = w + k * tp;
      if (k < 4 || i < (a.mxy >> 1)) dst[i] = s4[i];
    }
  }
  add_norms(norms, rr, ss, red_r, red_s);
}

// Inverse plane kernel: load the plane's half spectrum, y inverse, x inverse
// with the update of psi.
__global__ void __launch_bounds__(1024, 1) k_plane_inv(const float2* __restrict__ spec,
                                                      const int* __restrict__ planes,
                                                      int nplanes, int64_t* __restrict__ psi,
                                                      SpecArgs a) {
  extern __shared__ __align__(16) float2 sm[];
  const int nx = a.nx, ny = a.ny;
  const int tp = 1 << a.lgtp;
  const int slot = threadIdx.x >> a.lgtp, w = threadIdx.x & (tp - 1);
  const int pi = blockIdx.x * (blockDim.x >> a.lgtp) + slot;
  const bool valid = pi < nplanes;
  const int z = !valid ? 0 : (planes ? planes[pi] : pi);
  float2* S = sm + (size_t)slot * plane_smem_words(nx, ny);
  float2* scr = S + a.mxy;
  {
    float4* s4 = reinterpret_cast<float4*>(S);
    const float4* src4 = reinterpret_cast<const float4*>(spec + (int64_t)z * a.mxy);
    float4 t4[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const int i = w + k * tp;
      t4[k] = valid && (k < 4 || i < (a.mxy >> 1)) ? src4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const int i = w + k * tp;
      if (k < 4 || i < (a.mxy >> 1)) s4[i] = t4[k];
    }
  }
  __syncthreads();
  LBM_LG_DISPATCH(a.lgy, yphase_inv, S, scr, w, a.H, a.twy)
  __syncthreads();
  LBM_LG_DISPATCH(a.lgx, xphase_inv, S, scr, w, ny, valid, psi + (int64_t)z * nx * ny, a.twx)
}

// Periodic z axis of power-of-two length (8..256): the z operator is
// circulant, so an FFT along z diagonalises it too (eigenvalue
// 2 - 2 cos(2 pi kz / nz)).  One CTA: 32 consecutive modes, thread
// (t, p) = threadIdx.x = 32 t + p, so every warp reads 32 consecutive modes
// of one plane; the pencil of mode p exchanges through column p of a
// [z][33] shared array.  Forward FFT, division by lambda (the free mean,
// mode (0,0,0), set to 0), inverse FFT, all in registers between exchanges.
template <int LGZ>
__global__ void __launch_bounds__(4 << LGZ, LGZ <= 7 ? 2 : 1) k_zfft(float2* __restrict__ spec, SpecArgs a) {
  extern __shared__ __align__(16) float2 zb[];
  constexpr int L = 1 << LGZ, T = L >> 3;
  const int p = threadIdx.x & 31, t = threadIdx.x >> 5;
  const int m = blockIdx.x * 32 + p;
  const bool ok = m < a.mxy;
  const int64_t mxy = a.mxy;
  float2 v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u)
    v[u] = ok ? spec[(int64_t)(t + u * T) * mxy + m] : make_float2(0.f, 0.f);
  const StrideLine line{zb + p, 33};
  fft_regs<LGZ, true>(v, t, line, a.twz, -1.f);
  const int ky = ok ? m / (a.H + 1) : 0, kx = ok ? m - ky * (a.H + 1) : 0;
  const float lxy = a.lamx[kx] + a.lamy[ky];
  constexpr float invL = 1.0f / (float)L;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int kz = t + u * T;
    const float sc = (m == 0 && kz == 0) ? 0.f : invL / (lxy + a.lamz[kz]);
    v[u] = make_float2(v[u].x * sc, v[u].y * sc);
  }
  fft_regs<LGZ, true>(v, t, line, a.twz, 1.f);
  if (ok) {
#pragma unroll
    for (int u = 0; u < 8; ++u) spec[(int64_t)(t + u * T) * mxy + m] = v[u];
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
  const int nxy = a.mxy;  // modes per plane of the half spectrum
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
    const int ky = m / (a.H + 1), kx = m - ky * (a.H + 1);
    solve_pencil(X + j, C + j, Qv + j, ZP, L, a.lamx[kx] + a.lamy[ky], m == 0, R.cyclic != 0);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < ZP * L; idx += blockDim.x) {
    const int k = idx / ZP, jj = idx - k * ZP;
    int z = R.z0 + k;
    if (z >= a.nz) z -= a.nz;
    if (m0 + jj < nxy) x[(int64_t)z * nxy + m0 + jj] = X[idx];
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

// Residual with per-plane means: r = s - mean_z - A psi (exact), its
// squared norms (and the source's) added to the norm slot acc; r (scaled to
// real units) is stored only when r != NULL.  One thread per two consecutive
// x (residual_g), no loop: every load of a thread is in flight at once.
// Wall planes contribute nothing.
__global__ void __launch_bounds__(256, 4) k_res_planes(
    const int64_t* __restrict__ psi, const int64_t* __restrict__ src,
    const long long* __restrict__ mean_z, const unsigned char* __restrict__ plane_fluid,
    float* __restrict__ r, float* acc, int nx, int ny, int nz, int lgx, int lgxy) {
  __shared__ float red_r[8], red_s[8];
  const int64_t npairs = ((int64_t)nx * ny * nz) >> 1;
  const int lgg = lgxy - 1, lgr = lgx - 1;  // pairs per plane, per row
  float rr = 0.f, ss = 0.f;
  const int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gi < npairs) {
    const int z = (int)(gi >> lgg);
    const int k = (int)(gi & ((1 << lgg) - 1));
    const int y = k >> lgr, x0 = (k & ((1 << lgr) - 1)) << 1;
    const int64_t i0 = ((int64_t)z * ny + y) * nx + x0;
    const bool fluid = __ldg(plane_fluid + z);
    const PlaneNbr g = plane_nbr(plane_fluid, mean_z, z, nx * ny, nz);
    float r2[2], a = 0.f, b = 0.f;
    residual_g<2>(psi, src, i0, x0, y, nx, ny, g, r2, a, b);
    if (fluid) {
      rr = a;
      ss = b;
    } else {
      r2[0] = r2[1] = 0.f;
    }
    if (r) *reinterpret_cast<float2*>(r + i0) = make_float2(r2[0] * PSI_INV_SCALE_F, r2[1] * PSI_INV_SCALE_F);
  }
  add_norms(acc, rr, ss, red_r, red_s);
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
  float2* tw = nullptr;            // twiddles: nx, then ny, then nz values
  float* lam = nullptr;            // eigenvalues: H + 1, then ny, then nz values
  float2* spec = nullptr;          // half spectrum, nz * mxy values
  int mxy = 0;
  int lgtp = 0;                    // log2 of the threads per plane
  int ppc = 1;                     // planes per CTA of the plane kernels
  size_t plane_smem = 0;           // shared memory of a plane-kernel CTA
  size_t zsmem = 0;                // shared memory of the z solve
  int lgz = -1;                    // log2(nz) when the z axis is one periodic run
  int last_iters = 2;              // applications of the previous solve
  int graph_k = 0;                 // applications baked into the step graphs
  int graph_pred = 0;              // applications the last graph steps suggest (0: none yet)
  int need_acc[4] = {0, 0, 0, 0};  // steps needing 1, 2, 3, >= 4 applications, not yet decided on
  bool status_read = false;        // the host copy of the graph status is current
  bool runs_fit = true;            // z solve fits in shared memory
  float* r = nullptr;              // N (residual for the learned guess)
  long long* psum = nullptr;       // nz
  long long* mean_z = nullptr;     // nz
  float* nacc = nullptr;           // norm slots, Poisson::NSLOT x 2 NACC
  float* hacc = nullptr;           // pinned mirror
};

void spectral_free(lbm_t* h) {
  SpectralPlan* s = h->spec;
  if (!s) return;
  cudaFree(s->planes);
  cudaFree(s->runs);
  cudaFree(s->plane_fluid);
  cudaFree(s->tw);
  cudaFree(s->lam);
  cudaFree(s->spec);
  cudaFree(s->r);
  cudaFree(s->psum);
  cudaFree(s->mean_z);
  h->charge_mean_z = nullptr;
  h->charge_means_ready = false;
  cudaFree(s->nacc);
  if (s->hacc) cudaFreeHost(s->hacc);
  delete s;
  h->spec = nullptr;
}

lbm_status spectral_setup(lbm_t* h, const uint8_t* solid) {
  spectral_free(h);
  const int nx = h->cfg.nx, ny = h->cfg.ny, nz = h->cfg.nz;
  const int lgx = ilog2(nx), lgy = ilog2(ny);
  if (lgx < 3 || lgy < 3 || lgx > 8 || lgy > 8 || nx * ny > 16384) {
    h->err = "spectral Poisson solver needs power-of-two nx, ny in [8, 256] with nx*ny <= 16384";
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
  s->mxy = (nx / 2 + 1) * ny;
  s->lgtp = lgx + lgy - 4;
  s->ppc = std::max(1, 256 >> s->lgtp);
  const int64_t N = h->N;
  auto al = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  const size_t ntw = (size_t)nx + ny + nz, nlam = (size_t)nx / 2 + 1 + ny + nz;
  bool ok = al((void**)&s->planes, planes.size() * sizeof(int)) &&
            al((void**)&s->runs, runs.size() * sizeof(Run)) && al((void**)&s->plane_fluid, nz) &&
            al((void**)&s->tw, ntw * sizeof(float2)) && al((void**)&s->lam, nlam * sizeof(float)) &&
            al((void**)&s->spec, (size_t)nz * s->mxy * sizeof(float2)) &&
            al((void**)&s->r, N * sizeof(float)) && al((void**)&s->psum, nz * sizeof(long long)) &&
            al((void**)&s->mean_z, nz * sizeof(long long)) &&
            al((void**)&s->nacc, (size_t)Poisson::NSLOT * 2 * NACC * sizeof(float));
  if (ok && cudaMallocHost((void**)&s->hacc, (size_t)Poisson::NSLOT * 2 * NACC * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    s->hacc = nullptr;
    ok = false;
  }
  if (!ok) {
    spectral_free(h);
    h->err = "spectral Poisson allocation failed";
    return LBM_ENOMEM;
  }
  // twiddles exp(-2 pi i m / n), m < n, and eigenvalues 2 - 2 cos(2 pi k / n)
  // of the periodic second difference, in double precision, rounded once;
  // the eigenvalue of k and n - k is the same number
  const double twopi = 2.0 * 3.14159265358979323846;
  std::vector<float2> tw;
  std::vector<float> lam;
  for (int n : {nx, ny, nz})
    for (int m = 0; m < n; ++m)
      tw.push_back(make_float2((float)cos(-twopi * m / n), (float)sin(-twopi * m / n)));
  auto eig = [&](int k, int n) {
    const int kk = std::min(k, n - k);
    return (float)(2.0 - 2.0 * cos(twopi * kk / n));
  };
  for (int k = 0; k <= nx / 2; ++k) lam.push_back(eig(k, nx));
  for (int k = 0; k < ny; ++k) lam.push_back(eig(k, ny));
  for (int k = 0; k < nz; ++k) lam.push_back(eig(k, nz));
  LBM_CUDA_TRY(h, cudaMemcpy(s->planes, planes.data(), planes.size() * sizeof(int), cudaMemcpyHostToDevice));
  LBM_CUDA_TRY(h, cudaMemcpy(s->runs, runs.data(), runs.size() * sizeof(Run), cudaMemcpyHostToDevice));
  LBM_CUDA_TRY(h, cudaMemcpy(s->plane_fluid, pf.data(), nz, cudaMemcpyHostToDevice));
  LBM_CUDA_TRY(h, cudaMemcpy(s->tw, tw.data(), ntw * sizeof(float2), cudaMemcpyHostToDevice));
  LBM_CUDA_TRY(h, cudaMemcpy(s->lam, lam.data(), nlam * sizeof(float), cudaMemcpyHostToDevice));
  int optin = 0;
  LBM_CUDA_TRY(h, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev));
  const int lgz = ilog2(nz);
  if (runs.size() == 1 && runs[0].cyclic && lgz >= 3 && lgz <= 8) {
    s->lgz = lgz;
    const size_t zf = (size_t)nz * 33 * sizeof(float2);
    if (zf > 48 * 1024)
    {
      cudaError_t e = cudaSuccess;
      switch (lgz) {
        case 3: e = cudaFuncSetAttribute(k_zfft<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zf); break;
        case 4: e = cudaFuncSetAttribute(k_zfft<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zf); break;
        case 5: e = cudaFuncSetAttribute(k_zfft<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zf); break;
        case 6: e = cudaFuncSetAttribute(k_zfft<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zf); break;
        case 7: e = cudaFuncSetAttribute(k_zfft<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zf); break;
        default: e = cudaFuncSetAttribute(k_zfft<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zf); break;
      }
      LBM_CUDA_TRY(h, e);
    }
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
  if (s->runs_fit && s->lgz < 0 && s->zsmem > 48 * 1024)
    LBM_CUDA_TRY(h, cudaFuncSetAttribute(k_zsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->zsmem));
  h->charge_mean_z = (s->nruns == 1 && s->nplanes == nz) ? s->mean_z : nullptr;
  h->charge_means_ready = false;
  s->plane_smem = (size_t)s->ppc * plane_smem_words(nx, ny) * sizeof(float2);
  if ((int)s->plane_smem > optin - 256) {
    h->err = "spectral Poisson solver: x-y plane too large for shared memory";
    return LBM_EINVAL;
  }
  if (s->plane_smem > 48 * 1024) {
    LBM_CUDA_TRY(h, cudaFuncSetAttribute(k_plane_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->plane_smem));
    LBM_CUDA_TRY(h, cudaFuncSetAttribute(k_plane_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->plane_smem));
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
  a.lgz = s->lgz;
  a.H = s->nx / 2;
  a.mxy = s->mxy;
  a.lgtp = s->lgtp;
  a.twx = s->tw;
  a.twy = s->tw + s->nx;
  a.twz = s->tw + s->nx + s->ny;
  a.lamx = s->lam;
  a.lamy = s->lam + s->nx / 2 + 1;
  a.lamz = a.lamy + s->ny;
  return a;
}

// Norm slot i: 2 NACC partial sums (residual^2, then source^2, in
// fixed-point units squared).
float* norm_slot(lbm_t* h, int slot) { return h->spec->nacc + (size_t)slot * 2 * NACC; }

cudaError_t clear_slot(lbm_t* h, int slot) {
  return cudaMemsetAsync(norm_slot(h, slot), 0, 2 * NACC * sizeof(float), h->st);
}

// Copies norm slots 0..n-1 to the host and waits.
cudaError_t read_slots(lbm_t* h, int n) {
  cudaError_t e = cudaMemcpyAsync(h->spec->hacc, h->spec->nacc, (size_t)n * 2 * NACC * sizeof(float),
                                  cudaMemcpyDeviceToHost, h->st);
  return e == cudaSuccess ? cudaStreamSynchronize(h->st) : e;
}

// Norms |r|_2, |s - <s>|_2 of a slot read by read_slots.
void slot_norms(const lbm_t* h, int slot, double* rn, double* sn) {
  const float* p = h->spec->hacc + (size_t)slot * 2 * NACC;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < NACC; ++k) {
    a += (double)p[k];
    b += (double)p[NACC + k];
  }
  *rn = sqrt(a * 1099511627776.0);
  *sn = sqrt(b * 1099511627776.0);
}

// Residual of the current potential (exact, k_res_planes) with its norms in
// the slot; stores r (for the learned guess) when with_r.
cudaError_t spec_residual(lbm_t* h, int slot, bool with_r) {
  SpectralPlan* s = h->spec;
  Poisson& P = h->ps;
  cudaError_t e = clear_slot(h, slot);
  if (e != cudaSuccess) return e;
  k_res_planes<<<nblk(h->N / 2, 256), 256, 0, h->st>>>(P.psi[P.cur], P.src, s->mean_z, s->plane_fluid,
                                                     with_r ? s->r : nullptr, norm_slot(h, slot),
                                                     s->nx, s->ny, s->nz, s->lgx, s->lgx + s->lgy);
  ++h->launches;
  return cudaGetLastError();
}

cudaError_t spec_means(lbm_t* h) {
  SpectralPlan* s = h->spec;
  Poisson& P = h->ps;
  if (s->nruns == 1 && (int)s->nplanes == s->nz) {
    // one periodic run: the mean over all fluid, written by the charge
    // path's partial sum, or here from its total
    if (h->charge_means_ready) {
      h->charge_means_ready = false;
      return cudaSuccess;
    }
    k_global_mean<<<1, 256, 0, h->st>>>(P.dsum, 1.0 / (double)h->nfluid, s->mean_z, s->nz);
    ++h->launches;
    return cudaGetLastError();
  }
  k_plane_sums<<<s->nz, 256, 0, h->st>>>(P.src, s->psum, s->nx * s->ny);
  k_run_means<<<1, 256, 0, h->st>>>(s->psum, s->runs, s->nruns, s->mean_z, s->nz, s->nx * s->ny);
  h->launches += 2;
  return cudaGetLastError();
}

// First kernel of an application: the residual of the current potential
// (norms into the slot) and its 2-D half spectrum.
cudaError_t spec_fwd(lbm_t* h, int slot) {
  SpectralPlan* s = h->spec;
  Poisson& P = h->ps;
  const SpecArgs a = args_of(s);
  float* out = norm_slot(h, slot);
  cudaError_t e = cudaSuccess;
  if (slot == 0 && h->slot0_cleared) h->slot0_cleared = false;  // cleared with the start
  else e = clear_slot(h, slot);
  if (e != cudaSuccess) return e;
  const unsigned gp = (unsigned)((s->nplanes + s->ppc - 1) / s->ppc);
  k_plane_fwd<<<gp, s->ppc << s->lgtp, s->plane_smem, h->st>>>(
      P.psi[P.cur], P.src, s->mean_z, s->plane_fluid, s->nplanes == s->nz ? nullptr : s->planes,
      s->nplanes, s->spec, out, a);
  ++h->launches;
  return cudaGetLastError();
}

// Rest of an application: the z solve and the inverse transform with the
// update of psi.
cudaError_t spec_zinv(lbm_t* h) {
  SpectralPlan* s = h->spec;
  Poisson& P = h->ps;
  const SpecArgs a = args_of(s);
  if (s->lgz > 0) {
    const unsigned g = nblk(s->mxy, 32);
    const size_t zs = (size_t)s->nz * 33 * sizeof(float2);
    switch (s->lgz) {
      case 3: k_zfft<3><<<g, 4 * s->nz, zs, h->st>>>(s->spec, a); break;
      case 4: k_zfft<4><<<g, 4 * s->nz, zs, h->st>>>(s->spec, a); break;
      case 5: k_zfft<5><<<g, 4 * s->nz, zs, h->st>>>(s->spec, a); break;
      case 6: k_zfft<6><<<g, 4 * s->nz, zs, h->st>>>(s->spec, a); break;
      case 7: k_zfft<7><<<g, 4 * s->nz, zs, h->st>>>(s->spec, a); break;
      default: k_zfft<8><<<g, 4 * s->nz, zs, h->st>>>(s->spec, a); break;
    }
  } else {
    dim3 g(nblk(s->mxy, ZP), s->nruns);
    k_zsolve<<<g, 128, s->zsmem, h->st>>>(s->spec, s->runs, a);
  }
  const unsigned gp = (unsigned)((s->nplanes + s->ppc - 1) / s->ppc);
  k_plane_inv<<<gp, s->ppc << s->lgtp, s->plane_smem, h->st>>>(
      s->spec, s->nplanes == s->nz ? nullptr : s->planes, s->nplanes, P.psi[P.cur], a);
  h->launches += 2;
  return cudaGetLastError();
}

cudaError_t spec_apply(lbm_t* h, int slot) {
  cudaError_t e = spec_fwd(h, slot);
  return e == cudaSuccess ? spec_zinv(h) : e;
}

}  // namespace

lbm_status spectral_solve(lbm_t* h, double tol, int maxit, int* iters, double* rel_res) {
  SpectralPlan* s = h->spec;
  if (!s->runs_fit) {
    h->err = "spectral Poisson solver: fluid run along z too long for shared memory";
    return LBM_EINVAL;
  }
  const double floor = RES_FLOOR_RMS * sqrt((double)h->nfluid);
  auto conv_of = [&](double rn, double sn) { return rn <= tol * sn || rn <= floor; };
  LBM_CUDA_TRY(h, spec_means(h));
  double rn = 0.0, sn = 0.0;
  int it = 0;
  bool known = false;  // rn, sn hold the norms of the current potential
  if (nn_active(h)) {
    LBM_CUDA_TRY(h, spec_residual(h, 0, true));
    LBM_CUDA_TRY(h, read_slots(h, 1));
    slot_norms(h, 0, &rn, &sn);
    note_start_residual(h, sn > 0.0 ? rn / sn : 0.0);
    known = true;
    if (!conv_of(rn, sn)) {
      bool applied = false;
      float* dpsi = nullptr;
      lbm_status st = nn_before_solve(h, s->r, 0, s->nz, 0, rn * PSI_INV_SCALE / sqrt((double)h->nfluid),
                                      &applied, &dpsi);
      if (st != LBM_OK) return st;
      if (applied) {
        const double rn_old = rn;
        LBM_CUDA_TRY(h, spec_residual(h, 0, false));
        LBM_CUDA_TRY(h, read_slots(h, 1));
        slot_norms(h, 0, &rn, &sn);
        if (rn < rn_old) {
          nn_record(h, rn / rn_old);
        } else {
          st = nn_revert(h, dpsi);
          if (st != LBM_OK) return st;
          LBM_CUDA_TRY(h, spec_residual(h, 0, false));
          LBM_CUDA_TRY(h, read_slots(h, 1));
          slot_norms(h, 0, &rn, &sn);
        }
      }
    }
  } else if (maxit > 0) {
    // Queue the number of applications the previous solve needed without
    // looking at the first residual (each application computes the norms
    // of the residual it transforms), the final residual's norms, and read
    // all norms with one host synchronisation.  An application beyond the
    // one that reached the tolerance only refines psi further.
    const int k = std::max(1, std::min(std::min(s->last_iters, maxit), Poisson::NSLOT - 1));
    for (int i = 0; i < k; ++i) LBM_CUDA_TRY(h, spec_apply(h, i));
    LBM_CUDA_TRY(h, spec_residual(h, k, false));
    LBM_CUDA_TRY(h, read_slots(h, k + 1));
    int need = k;
    slot_norms(h, 0, &rn, &sn);
    note_start_residual(h, sn > 0.0 ? rn / sn : 0.0);
    for (int i = 0; i <= k; ++i) {
      slot_norms(h, i, &rn, &sn);
      if (conv_of(rn, sn)) {
        need = i;
        break;
      }
    }
    slot_norms(h, k, &rn, &sn);
    known = true;
    it = k;
    s->last_iters = std::max(1, need);
  }
  if (!known) {
    LBM_CUDA_TRY(h, spec_residual(h, 0, false));
    LBM_CUDA_TRY(h, read_slots(h, 1));
    slot_norms(h, 0, &rn, &sn);
  }
  while (!conv_of(rn, sn) && it < maxit) {
    LBM_CUDA_TRY(h, spec_apply(h, 0));
    LBM_CUDA_TRY(h, spec_residual(h, 1, false));
    LBM_CUDA_TRY(h, read_slots(h, 2));
    slot_norms(h, 1, &rn, &sn);
    if (!isfinite(rn) || !isfinite(sn)) {
      h->err = "Poisson residual is not finite";
      return LBM_EUNSTABLE;
    }
    ++it;
    s->last_iters = it;
  }
  if (!isfinite(rn) || !isfinite(sn)) {
    h->err = "Poisson residual is not finite";
    return LBM_EUNSTABLE;
  }
  if (iters) *iters = it;
  if (rel_res) *rel_res = sn > 0.0 ? rn / sn : 0.0;
  if (!conv_of(rn, sn)) {
    h->err = "Poisson solve did not reach the tolerance within the iteration cap";
    return LBM_ENOCONV;
  }
  return LBM_OK;
}


// ---------------------------------------------------------------------------
// Whole-step CUDA graphs.  One graph per population parity holds a full time
// step: charge density, run means, k spectral applications, then side by
// side the fused stream/collide on that potential and the final residual
// with its test; a device-side while loop (conditional graph node) of
// [application, residual, test] for a step that needs more, and an if node
// that runs the stream/collide again on the refined potential (it writes
// the spare lattice, so running it twice is harmless).  The graphs are
// rebuilt when the applications steps need change (k from the distribution
// of the previous call's steps).
// Steps are replayed back to back with no host round trip; the test kernel
// keeps the per-step status on the device.
// ---------------------------------------------------------------------------
namespace {

struct GraphStatus {
  uint32_t step;       // time step (read by the stream/collide kernel)
  int iters;           // Poisson applications of the current step
  long long total;     // applications summed over replayed steps
  int fails;           // steps whose solve stopped at the iteration cap
  double rel;          // final relative residual of the last step
  int need[4];         // steps that needed 1, 2, 3, >= 4 applications since the host reset it
  int needf[4];        // the same, counting only steps whose start had the full history
  int full;            // the current step's start had the full history
  double start_log;    // sum of log10 of the steps' start residuals
  long long starts;    // steps counted in start_log
  int spec_skip;       // the current step does not speculate (start from a short history)
  long long redos;     // steps that ran the stream/collide after the loop
  int more;            // the first test of the step asks for more applications
};

// First node of the rerun branch: the loop runs when the step's first test
// asked for more applications (it reruns the stream/collide also when the
// step did not speculate and the baked applications were enough).
__global__ void k_loop_seed(const GraphStatus* st, cudaGraphConditionalHandle cond) {
  cudaGraphSetConditional(cond, st->more ? 1u : 0u);
}

// Whether the step runs its stream/collide speculatively, beside the test
// after the k baked applications: only when the start used the full
// history.  A start from a short history (the first steps after a restart)
// usually needs more applications, and the speculative stream/collide would
// be discarded; then the stream/collide runs once, after the loop.
// The step after one that needed more than the k baked applications does
// not speculate either (such steps come in runs; see k_start_mark).  This
// kernel decides when the start from the history is off; otherwise the
// start's bookkeeping kernel does.
__global__ void k_spec_decide(const int* __restrict__ start_terms, GraphStatus* st, int k) {
  st->spec_skip = ((start_terms && *start_terms < START_FULL_TERMS) || st->iters > k) ? 1 : 0;
}

// Convergence test (one warp).  first: after the k applications queued
// unconditionally (norm slots 0..k hold the residual before each and after
// the last); records how many a step needed and sets `redo` when the loop
// will run.  Otherwise after one more application (slot k).  Sets the
// condition of the while node.
__global__ void k_graph_check(const float* __restrict__ acc, GraphStatus* st, double tol,
                              double floor2, int maxit, int k, int first,
                              const int* __restrict__ start_terms,
                              cudaGraphConditionalHandle cond, cudaGraphConditionalHandle redo) {
  if (blockIdx.x != 0) return;
  const int lane = threadIdx.x;
  // lane i < k + 1 tests slot i
  bool conv_i = false;
  double rn2 = 0.0, sn2 = 0.0;
  if (lane <= k) {
    const float* a = acc + (size_t)lane * 2 * NACC;
    for (int j = 0; j < NACC; ++j) {
      rn2 += (double)a[j];
      sn2 += (double)a[NACC + j];
    }
    rn2 *= 1099511627776.0;
    sn2 *= 1099511627776.0;
    conv_i = rn2 <= tol * tol * sn2 || rn2 <= floor2;
  }
  const unsigned convmask = __ballot_sync(0xffffffffu, conv_i);
  const double rnk = __shfl_sync(0xffffffffu, rn2, k), snk = __shfl_sync(0xffffffffu, sn2, k);
  if (lane != 0) return;
  const bool conv = (convmask >> k) & 1u;
  // the step counts towards the choice of k when its start was near the
  // one of the steady state: fitted on at least START_FULL_TERMS stored
  // differences (the first starts after a restart have fewer), or any step
  // when the history start is off
  if (first) {
    st->full = !start_terms || *start_terms >= START_FULL_TERMS;
    st->iters = k;
    // slot 0 holds the residual the first application transformed (the
    // start), lane 0 read it
    if (rn2 >= 0.0 && sn2 > 0.0) {
      st->start_log += 0.5 * log10(fmax(rn2 / sn2, 1e-300));
      st->starts += 1;
    }
  } else {
    st->iters += 1;
  }
  const bool more = !conv && st->iters < maxit;
  // the stream/collide ran beside this test on the potential after k
  // applications: it runs again after the loop when the loop runs, or when
  // the step did not speculate.  The first test opens that branch (its loop
  // condition is seeded from `more` inside it); the tests in the loop
  // continue it.
  if (first) {
    st->more = more ? 1 : 0;
    const bool again = more || st->spec_skip;
    cudaGraphSetConditional(redo, again ? 1u : 0u);
    if (again) st->redos += 1;
  } else {
    cudaGraphSetConditional(cond, more ? 1u : 0u);
  }
  st->rel = snk > 0.0 ? sqrt(rnk / snk) : 0.0;
  // applications this step needed, recorded once per step: at the first
  // test when slot k converged (the earliest converged slot), else when the
  // loop ends
  int needed = 0;
  if (first && conv)
    needed = max(1, __ffs(convmask) - 1);
  else if (!more)
    needed = st->iters;
  if (needed) {
    const int j = min(needed, 4) - 1;
    st->need[j] += 1;
    if (st->full) st->needf[j] += 1;
  }
  if (!more) {
    st->total += st->iters;
    if (!conv) st->fails += 1;
  }
}

}  // namespace

void spectral_graph_free(lbm_t* h) {
  for (int k = 0; k < 2; ++k)
    for (int d = 0; d < 2; ++d) {
      if (h->step_graph[k][d]) cudaGraphExecDestroy(h->step_graph[k][d]);
      h->step_graph[k][d] = nullptr;
    }
}

lbm_status potential_history_reset(lbm_t* h) {
  LBM_CUDA_TRY(h, start_join(h));  // a fit still queued writes the history
  LBM_CUDA_TRY(h, start_reset(h));
  return LBM_OK;
}

namespace {

lbm_status build_step_graph(lbm_t* h, int parity, bool diag) {
  const int saved_cur = h->cur;
  const bool saved_diag = h->diag_valid;  // capture runs nothing
  const bool saved_scat = h->scat_valid;
  h->cur = parity;
  GraphStatus* gs = reinterpret_cast<GraphStatus*>(h->gstatus);
  const double tol = h->cfg.poisson_tol;
  const double floor2 = RES_FLOOR_RMS * RES_FLOOR_RMS * (double)h->nfluid;
  const int maxit = h->cfg.poisson_maxit;
  // steps count towards the choice of k once their start used the full
  // history (any step when the start is off)
  const int* terms = start_enabled(h) ? start_terms_dev(h) : nullptr;
  cudaGraph_t G = nullptr;
  LBM_CUDA_TRY(h, cudaGraphCreate(&G, 0));
  // redo: the if node of the rerun branch (in G); cond: the loop inside it
  // (created on the branch's body graph below)
  cudaGraphConditionalHandle cond = 0, redo;
  LBM_CUDA_TRY(h, cudaGraphConditionalHandleCreate(&redo, G, 0, cudaGraphCondAssignDefault));
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  cudaStream_t main = h->st, side = nullptr, side2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr, fork2 = nullptr, join2 = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
  // the fit of the Poisson start for the next step runs at the lowest
  // priority, beside the latency-bound transforms (node priorities are
  // kept at instantiation)
  if (e == cudaSuccess) {
    int lo = 0, hi = 0;
    e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&side2, cudaStreamNonBlocking, lo);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork2, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join2, cudaEventDisableTiming);
  const int64_t l0 = h->launches;
  int64_t lc = 0;  // launches of the stream/collide
  // part A: the source (advancing the step counter), the start of the
  // solve from the history (lbm_start.cu), the means, the predicted number
  // k of applications (each records the norms of the residual it
  // transforms); then, side by side, the stream/collide on that potential
  // and the final residual with the test
  const int k = h->spec->graph_k;
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(main, G, nullptr, nullptr, 0, mode);
  if (e == cudaSuccess) {
    cudaError_t ec = cudaSuccess;
    h->charge_step = &gs->step;
    // the start from the history, then the fit for the next step on the
    // second side stream, beside the applications; the start's
    // bookkeeping (its own kernel, or the last CTA of the source take when
    // that applies the start) also decides the speculation and clears the
    // first norm slot (when the start is on)
    const bool fit = start_enabled(h);
    if (fit) {
      h->mark_skip_out = &gs->spec_skip;
      h->mark_prev_iters = &gs->iters;
      h->mark_k = k;
      h->mark_clear = norm_slot(h, 0);
      h->mark_nclear = 2 * NACC;
    }
    // with the charge scatter, a replay finds the source of its input
    // populations in the accumulator (spectral_graph_steps sees to it
    // before the first replay; every step's stream/collide scatters the
    // next one)
    h->scat_valid = true;
    ec = launch_charge(h);
    h->charge_step = nullptr;
    if (ec == cudaSuccess) ec = start_apply(h, false);
    h->mark_skip_out = nullptr;
    h->mark_prev_iters = nullptr;
    h->mark_clear = nullptr;
    if (ec == cudaSuccess && fit) ec = cudaEventRecord(fork2, main);
    if (ec == cudaSuccess && fit) ec = cudaStreamWaitEvent(side2, fork2, 0);
    if (ec == cudaSuccess && fit) ec = start_fit(h, side2, true);
    if (ec == cudaSuccess && fit) ec = cudaEventRecord(join2, side2);
    if (ec == cudaSuccess) ec = spec_means(h);
    if (ec == cudaSuccess && !fit) {
      k_spec_decide<<<1, 1, 0, main>>>(terms, gs, k);
      ++h->launches;
      ec = cudaGetLastError();
    }
    for (int i = 0; i < k && ec == cudaSuccess; ++i) ec = spec_apply(h, i);
    if (ec == cudaSuccess) ec = cudaEventRecord(fork, main);
    if (ec == cudaSuccess) ec = cudaStreamWaitEvent(side, fork, 0);
    if (ec == cudaSuccess) {
      const int64_t a = h->launches;
      h->st = side;
      h->collide_skip = &gs->spec_skip;
      ec = launch_stream_collide(h, diag);
      h->collide_skip = nullptr;
      h->st = main;
      lc = h->launches - a;
    }
    if (ec == cudaSuccess) ec = cudaEventRecord(join, side);
    if (ec == cudaSuccess) ec = spec_residual(h, k, false);
    if (ec == cudaSuccess) {
      k_graph_check<<<1, 32, 0, main>>>(norm_slot(h, 0), gs, tol, floor2, maxit, k, 1, terms, cond,
                                        redo);
      ++h->launches;
      ec = cudaGetLastError();
    }
    if (ec == cudaSuccess) ec = cudaStreamWaitEvent(main, join, 0);
    if (ec == cudaSuccess && fit) ec = cudaStreamWaitEvent(main, join2, 0);
    std::vector<cudaGraphNode_t> deps;
    if (ec == cudaSuccess) {
      cudaStreamCaptureStatus cs;
      const cudaGraphNode_t* d = nullptr;
      size_t nd = 0;
      ec = cudaStreamGetCaptureInfo(main, &cs, nullptr, nullptr, &d, nullptr, &nd);
      if (ec == cudaSuccess) deps.assign(d, d + nd);
    }
    cudaGraph_t Gc = nullptr;
    e = cudaStreamEndCapture(main, &Gc);
    if (e == cudaSuccess) e = ec;
    // The rerun branch, an if node after the speculative stream/collide and
    // the fit: a kernel that seeds the loop condition from the first test,
    // the while loop of [application, residual, test], then the
    // stream/collide again on the refined potential.  A step that converged
    // after its baked applications evaluates this one conditional node only.
    const int64_t l1 = h->launches;
    cudaGraphNode_t inode = nullptr;
    cudaGraph_t ibody = nullptr;
    if (e == cudaSuccess) {
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = redo;
      cp.conditional.type = cudaGraphCondTypeIf;
      cp.conditional.size = 1;
      e = cudaGraphAddNode(&inode, G, deps.data(), nullptr, deps.size(), &cp);
      if (e == cudaSuccess) ibody = cp.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess)
      e = cudaGraphConditionalHandleCreate(&cond, ibody, 0, cudaGraphCondAssignDefault);
    std::vector<cudaGraphNode_t> sdeps;
    if (e == cudaSuccess) {
      e = cudaStreamBeginCaptureToGraph(main, ibody, nullptr, nullptr, 0, mode);
      if (e == cudaSuccess) {
        k_loop_seed<<<1, 1, 0, main>>>(gs, cond);
        ++h->launches;
        cudaError_t eb = cudaGetLastError();
        if (eb == cudaSuccess) {
          cudaStreamCaptureStatus cs;
          const cudaGraphNode_t* d = nullptr;
          size_t nd = 0;
          eb = cudaStreamGetCaptureInfo(main, &cs, nullptr, nullptr, &d, nullptr, &nd);
          if (eb == cudaSuccess) sdeps.assign(d, d + nd);
        }
        cudaGraph_t sg = nullptr;
        e = cudaStreamEndCapture(main, &sg);
        if (e == cudaSuccess) e = eb;
      }
    }
    cudaGraphNode_t cnode = nullptr;
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess) {
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = cond;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      e = cudaGraphAddNode(&cnode, ibody, sdeps.data(), nullptr, sdeps.size(), &cp);
      if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
    }
    const int64_t l2 = h->launches;
    if (e == cudaSuccess) {
      e = cudaStreamBeginCaptureToGraph(main, body, nullptr, nullptr, 0, mode);
      if (e == cudaSuccess) {
        cudaError_t eb = spec_apply(h, 0);
        if (eb == cudaSuccess) eb = spec_residual(h, k, false);
        if (eb == cudaSuccess) {
          k_graph_check<<<1, 32, 0, main>>>(norm_slot(h, 0), gs, tol, floor2, maxit, k, 0, terms,
                                            cond, redo);
          ++h->launches;
          eb = cudaGetLastError();
        }
        cudaGraph_t bb = nullptr;
        e = cudaStreamEndCapture(main, &bb);
        if (e == cudaSuccess) e = eb;
      }
    }
    const int64_t l3 = h->launches;
    if (e == cudaSuccess) {
      e = cudaStreamBeginCaptureToGraph(main, ibody, &cnode, nullptr, 1, mode);
      if (e == cudaSuccess) {
        // from the step's input populations again, into the same output as
        // the speculative launch (which flipped the parity while capturing);
        // the scatter of the speculative launch is cleared first
        h->cur = parity;
        cudaError_t eb = cudaSuccess;
        if (h->scat_on) eb = cudaMemsetAsync(h->scat_acc, 0, (size_t)h->N * sizeof(int64_t), main);
        if (eb == cudaSuccess) eb = launch_stream_collide(h, diag);
        cudaGraph_t gg = nullptr;
        e = cudaStreamEndCapture(main, &gg);
        if (e == cudaSuccess) e = eb;
      }
    }
    h->graph_kernels_fixed = (int)(l1 - l0);
    h->graph_kernels_iter = (int)(l3 - l2);
    h->graph_kernels_redo = (int)lc + 1;  // the seed and the stream/collide
  }
  h->launches = l0;
  h->cur = saved_cur;
  h->diag_valid = saved_diag;
  h->scat_valid = saved_scat;
  h->slot0_cleared = false;
  h->mark_skip_out = nullptr;
  h->mark_prev_iters = nullptr;
  h->mark_clear = nullptr;
  h->st = main;
  cudaGraphExec_t ex = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, G, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(G);
  if (fork) cudaEventDestroy(fork);
  if (join) cudaEventDestroy(join);
  if (fork2) cudaEventDestroy(fork2);
  if (join2) cudaEventDestroy(join2);
  if (side) cudaStreamDestroy(side);
  if (side2) cudaStreamDestroy(side2);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->err = std::string("step graph construction failed: ") + cudaGetErrorString(e);
    return LBM_ECUDA;
  }
  h->step_graph[parity][diag ? 1 : 0] = ex;
  return LBM_OK;
}

// Builds the missing step graphs (both parities, both stream/collide
// variants).
lbm_status build_step_graphs(lbm_t* h) {
  // the kernels' arguments bake every species' reference density and
  // valence (decoding of the stored deviations, charge, forces): a change
  // by lbm_set_species / lbm_set_species_dev rebuilds the graphs
  bool same = true;
  for (int s = 0; s < MAX_SPECIES; ++s)
    same = same && h->graph_nref[s] == h->nref[s] && h->graph_valence[s] == h->valence[s];
  if (!same) spectral_graph_free(h);
  for (int s = 0; s < MAX_SPECIES; ++s) {
    h->graph_nref[s] = h->nref[s];
    h->graph_valence[s] = h->valence[s];
  }
  for (int k = 0; k < 2; ++k)
    for (int d = 0; d < 2; ++d)
      if (!h->step_graph[k][d]) {
        lbm_status s = build_step_graph(h, k, d == 1);
        if (s != LBM_OK) return s;
      }
  return LBM_OK;
}

}  // namespace

void graph_status_ptrs(lbm_t* h, const int** iters, const double** rel) {
  GraphStatus* g = reinterpret_cast<GraphStatus*>(h->gstatus);
  *iters = g ? &g->iters : nullptr;
  *rel = g ? &g->rel : nullptr;
}

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
  SpectralPlan* sp = h->spec;
  GraphStatus* hs = reinterpret_cast<GraphStatus*>(h->hstatus);
  GraphStatus* ds = reinterpret_cast<GraphStatus*>(h->gstatus);
  // status before, to count this call's applications and failures (the
  // host copy from the end of the previous call is current: only these
  // graphs write the status)
  if (!sp->status_read) {
    LBM_CUDA_TRY(h, cudaMemcpyAsync(hs, ds, sizeof(GraphStatus), cudaMemcpyDeviceToHost, h->st));
    LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
    sp->status_read = true;
  }
  // the charge scatter: the source of the current populations into the
  // accumulator, where the first replay takes it
  LBM_CUDA_TRY(h, charge_prepare(h));
  const long long total0 = hs->total;
  const int fails0 = hs->fails;
  const double slog0 = hs->start_log;
  const long long starts0 = hs->starts;
  // Steps are replayed in chunks.  The distribution of the applications
  // the steps needed (accumulated over at least CHUNK steps whose start had
  // the full history) sets the number k baked into the graphs (rebuilt only
  // when k changes): the k of least expected cost per step.  With the start
  // from the history that is one in FP32; 16-bit storage, whose rounding
  // noise in the charge the history cannot predict, often needs two.  A step costs its k applications; one that
  // needs m > k also runs the while loop, m - k applications and residuals,
  // and the stream/collide again.  In units of a residual an application
  // costs about 4 and the stream/collide about 3.3 per FP32 species (3 per
  // 16-bit one), all three streaming the lattice at similar rates.
  constexpr int CHUNK = 16;
  const double costA = 4.0, costR = 1.0;
  const double costC = (h->cfg.storage == LBM_FP32 ? 3.3 : 3.0) * h->S;
  int done = 0;
  while (done < nsteps) {
    // the choice from the steps seen so far; before any, one application
    // with the start from the history (its steady state), else the last
    // solve's count
    const int pred = sp->graph_pred > 0 ? sp->graph_pred : (start_enabled(h) ? 1 : sp->last_iters);
    const int want = std::max(1, std::min(std::min(pred, h->cfg.poisson_maxit), Poisson::NSLOT - 1));
    if (sp->graph_k != want) {
      spectral_graph_free(h);
      sp->graph_k = want;
    }
    {
      lbm_status s = build_step_graphs(h);
      if (s != LBM_OK) return s;
    }
    const int n = std::min(CHUNK, nsteps - done);
    const long long tot_before = hs->total;
    const long long redos_before = hs->redos;
    LBM_CUDA_TRY(h, cudaMemsetAsync(ds->need, 0, 8 * sizeof(int), h->st));  // need, needf
    // the call's last step replays the variant that sums the state it
    // stores (diagnostics); every step does when the call records them,
    // and its record (the sums, applications and residual) is reduced and
    // copied to the host slot right after the step
    for (int k = 0; k < n; ++k) {
      const int d = (h->rec_dev || done + k == nsteps - 1) ? 1 : 0;
      LBM_CUDA_TRY(h, cudaGraphLaunch(h->step_graph[h->cur][d], h->st));
      h->cur ^= 1;
      ++h->tstep;
      h->diag_valid = d == 1;
      if (h->rec_dev)
        LBM_CUDA_TRY(h, launch_diag_reduce(h, h->rec_dev + (size_t)(done + k) * REC_LEN,
                                           &ds->iters, &ds->rel));
    }
    LBM_CUDA_TRY(h, cudaMemcpyAsync(hs, ds, sizeof(GraphStatus), cudaMemcpyDeviceToHost, h->st));
    LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
    // the body of the while node ran once per application beyond the k
    // baked into every step; steps that needed more than k, or did not
    // speculate, ran the stream/collide again
    const long long redo_steps = hs->redos - redos_before;
    h->launches += (int64_t)n * h->graph_kernels_fixed +
                   (hs->total - tot_before - (long long)n * sp->graph_k) * h->graph_kernels_iter +
                   (int64_t)redo_steps * h->graph_kernels_redo;
    // decide from the steady-state steps (full history at their start)
    // since the last decision once there are at least CHUNK of them (across
    // chunks and calls), or at the first chance
    for (int j = 0; j < 4; ++j) sp->need_acc[j] += hs->needf[j];
    const int tot = sp->need_acc[0] + sp->need_acc[1] + sp->need_acc[2] + sp->need_acc[3];
    // (with the start from the history the first decision also waits for
    // CHUNK such steps: the first ones after a restart are not typical)
    if (tot >= CHUNK || (sp->graph_pred == 0 && tot > 0 && !start_enabled(h))) {
      int best = 1;
      double best_cost = 0.0;
      for (int k = 1; k <= 4; ++k) {
        double c = costA * k * tot;
        for (int j = k; j < 4; ++j) c += sp->need_acc[j] * ((j + 1 - k) * (costA + costR) + costC);
        if (k == 1 || c < best_cost) {
          best = k;
          best_cost = c;
        }
      }
      sp->graph_pred = best;
      for (int j = 0; j < 4; ++j) sp->need_acc[j] = 0;
    }
    done += n;
    if (hs->fails != fails0) break;
  }
  // a new choice of k is built now, so that the next call starts replaying
  // at once
  if (sp->graph_pred > 0) {
    const int want = std::max(1, std::min(std::min(sp->graph_pred, h->cfg.poisson_maxit),
                                          Poisson::NSLOT - 1));
    if (sp->graph_k != want) {
      spectral_graph_free(h);
      sp->graph_k = want;
      lbm_status s = build_step_graphs(h);
      if (s != LBM_OK) return s;
    }
  }
  const long long iters = hs->total - total0;
  if (hs->starts > starts0) {
    // start residuals of the replayed steps (their geometric mean stands
    // for the last one)
    const double dl = hs->start_log - slog0;
    const long long dn = hs->starts - starts0;
    h->start_log_sum += dl;
    h->start_count += dn;
    h->last_start = pow(10.0, dl / (double)dn);
  }
  if (h->scat_on) h->scat_valid = true;  // each replay ends with a scattering stream/collide
  h->t_cnt[1] += iters;
  h->t_cnt[0] += done;
  h->t_cnt[2] += done;
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
