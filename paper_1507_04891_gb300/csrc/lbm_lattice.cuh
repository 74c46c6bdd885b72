// Device helpers of the lattice kernels, shared by the translation units
// that hold them (lbm_kernels.cu and the per-storage stream/collide units
// built from lbm_collide.cu): the D3Q19 velocity set, the population storage
// formats, streaming addresses with bounce-back, the potential gradient and
// the forces.  Internal to the library.
//
// Storage: structure of arrays, one plane of N values per (species,
// direction), f[(s*19 + p)*N + node], x fastest.  The stored lattice holds
// post-collision populations before streaming; every kernel that needs
// f(t) pulls them from the upstream node r - c_p (halfway bounce-back when
// that node is a wall node), so streaming costs no separate pass.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_internal.cuh"

namespace lbm_gb300 {
namespace {

// ---------------------------------------------------------------------------
// D3Q19 velocity set (Sec. 4 of the paper: D3Q19 discretisation).  Written as
// compile-time functions so that fully unrolled loops fold them away.
//   0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 edge vectors, opposite pairs.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ constexpr int CX(int p) {
  return (p == 1 || p == 7 || p == 9 || p == 11 || p == 13)    ? 1
         : (p == 2 || p == 8 || p == 10 || p == 12 || p == 14) ? -1
                                                               : 0;
}
__host__ __device__ __forceinline__ constexpr int CY(int p) {
  return (p == 3 || p == 7 || p == 10 || p == 15 || p == 17)   ? 1
         : (p == 4 || p == 8 || p == 9 || p == 16 || p == 18)  ? -1
                                                               : 0;
}
__host__ __device__ __forceinline__ constexpr int CZ(int p) {
  return (p == 5 || p == 11 || p == 14 || p == 15 || p == 18)  ? 1
         : (p == 6 || p == 12 || p == 13 || p == 16 || p == 17) ? -1
                                                                : 0;
}
__host__ __device__ __forceinline__ constexpr int OPP(int p) {
  return p == 0 ? 0 : ((p & 1) ? p + 1 : p - 1);
}
// Lattice weights Gamma_0(c_p) (Appendix): 1/3, 1/18, 1/36.
__host__ __device__ __forceinline__ constexpr float WT(int p) {
  return p == 0 ? (1.0f / 3.0f) : (p <= 6 ? (1.0f / 18.0f) : (1.0f / 36.0f));
}
// 1 / w_p, exact in FP32
__host__ __device__ __forceinline__ constexpr float INV_WT(int p) {
  return p == 0 ? 3.0f : (p <= 6 ? 18.0f : 36.0f);
}
constexpr float CS2 = 1.0f / 3.0f;

// ---------------------------------------------------------------------------
// Population storage formats.  The 16-bit formats store the relative
// deviation from the rest state of the species, h = f / (w_p n_ref) - 1, so
// that dilute ions keep their relative precision.
// ---------------------------------------------------------------------------
template <int ST>
struct Fmt;
// Every format stores the population's deviation from the reference
// equilibrium at rest, h = f / (w_p n_ref) - 1 (n_ref: the species' mean
// initial density).  The arithmetic of the step works on deviations
// d = f - w_p n_ref = w_p n_ref h, so FP32 rounding is relative to the
// deviation, not to f: a drift far below one ulp of f (the ion current of a
// high-Schmidt-number run) is still resolved.  ld returns f, ldd returns d;
// the stores take d.
template <>
struct Fmt<LBM_FP32> {
  using T = float;
  static __device__ __forceinline__ float ld(const T* p, float wn) { return wn * (1.0f + *p); }
  static __device__ __forceinline__ float ldd(const T* p, float wn) { return wn * *p; }
  static __device__ __forceinline__ float ldh(const T* p) { return *p; }
  static __device__ __forceinline__ void st(T* p, float d, float inv_wn) { *p = d * inv_wn; }
  // stores h (and a second value hb at pb); returns the stored values
  static __device__ __forceinline__ float sth_sr(T* p, float h, uint32_t) {
    *p = h;
    return h;
  }
  static __device__ __forceinline__ float2 sth_sr2(T* pa, float ha, T* pb, float hb, uint32_t) {
    *pa = ha;
    *pb = hb;
    return make_float2(ha, hb);
  }
};

// Two values rounded stochastically into a packed 16-bit pair by the
// hardware conversion with random bits (cvt.rs, sm_100 family); the first
// operand lands in the upper half.
__device__ __forceinline__ uint32_t cvt_rs_f16x2(float hi, float lo, uint32_t rbits) {
  uint32_t d;
  asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
  return d;
}
__device__ __forceinline__ uint32_t cvt_rs_bf16x2(float hi, float lo, uint32_t rbits) {
  uint32_t d;
  asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
  return d;
}
// 16-bit formats: the same h.  st() rounds to nearest; sth_sr() and sth_sr2()
// round stochastically (the hardware conversion draws on random bits to
// round up with probability equal to the dropped fraction), so the stored
// value is unbiased.  The per-step change of a slowly diffusing mode is a
// fraction of one 16-bit ulp of h; round-to-nearest would return the same
// value every step and freeze the mode.
template <>
struct Fmt<LBM_FP16_SHIFT> {
  using T = __half;
  static __device__ __forceinline__ float ld(const T* p, float wn) {
    return wn * (1.0f + __half2float(*p));
  }
  static __device__ __forceinline__ float ldd(const T* p, float wn) { return wn * __half2float(*p); }
  static __device__ __forceinline__ float ldh(const T* p) { return __half2float(*p); }
  static __device__ __forceinline__ void st(T* p, float d, float inv_wn) {
    *p = __float2half_rn(d * inv_wn);
  }
  // stochastic rounding; returns the stored values
  static __device__ __forceinline__ float sth_sr(T* p, float h, uint32_t rnd) {
    const uint32_t v = cvt_rs_f16x2(h, 0.0f, rnd);
    *reinterpret_cast<unsigned short*>(p) = (unsigned short)(v >> 16);
    return __high2float(*reinterpret_cast<const __half2*>(&v));
  }
  static __device__ __forceinline__ float2 sth_sr2(T* pa, float ha, T* pb, float hb, uint32_t rnd) {
    const uint32_t v = cvt_rs_f16x2(ha, hb, rnd);
    *reinterpret_cast<unsigned short*>(pa) = (unsigned short)(v >> 16);
    *reinterpret_cast<unsigned short*>(pb) = (unsigned short)(v & 0xFFFFu);
    const float2 r = __half22float2(*reinterpret_cast<const __half2*>(&v));
    return make_float2(r.y, r.x);  // ha sits in the upper half
  }
};
template <>
struct Fmt<LBM_BF16_SHIFT> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ float ld(const T* p, float wn) {
    return wn * (1.0f + __bfloat162float(*p));
  }
  static __device__ __forceinline__ float ldd(const T* p, float wn) {
    return wn * __bfloat162float(*p);
  }
  static __device__ __forceinline__ float ldh(const T* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ void st(T* p, float d, float inv_wn) {
    *p = __float2bfloat16_rn(d * inv_wn);
  }
  // stochastic rounding; returns the stored values (a bfloat16 is the upper
  // half of the float it rounds)
  static __device__ __forceinline__ float sth_sr(T* p, float h, uint32_t rnd) {
    const uint32_t v = cvt_rs_bf16x2(h, 0.0f, rnd);
    *reinterpret_cast<unsigned short*>(p) = (unsigned short)(v >> 16);
    return __uint_as_float(v & 0xFFFF0000u);
  }
  static __device__ __forceinline__ float2 sth_sr2(T* pa, float ha, T* pb, float hb, uint32_t rnd) {
    const uint32_t v = cvt_rs_bf16x2(ha, hb, rnd);
    *reinterpret_cast<unsigned short*>(pa) = (unsigned short)(v >> 16);
    *reinterpret_cast<unsigned short*>(pb) = (unsigned short)(v & 0xFFFFu);
    return make_float2(__uint_as_float(v & 0xFFFF0000u), __uint_as_float(v << 16));
  }
};

// Counter-based random bits for stochastic rounding: one 32-bit mix of the
// node index and the step per node, then one LCG step per stored value
// (only the high bits of the LCG state are used).  The mix is the
// low-bias 32-bit integer hash (xor-shift 16, multiply 0x7feb352d,
// xor-shift 15, multiply 0x846ca68b, xor-shift 16) published by
// C. Wellons' "hash prospector" search (2018); the LCG multiplier and
// increment are the Numerical Recipes pair (Press et al.).
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}
__device__ __forceinline__ uint32_t lcg_next(uint32_t& r) {
  r = r * 1664525u + 1013904223u;
  return r;
}

struct Nbr {
  // signed offsets to the upstream node along each axis for c = +1 / -1
  int dxm, dxp, dym, dyp, dzm, dzp;
};

__device__ __forceinline__ Nbr neighbours(int x, int y, int z, int nx, int ny,
                                          int nz) {
  const int nxy = nx * ny;
  Nbr o;
  o.dxm = (x == 0) ? nx - 1 : -1;  // node x-1
  o.dxp = (x == nx - 1) ? -(nx - 1) : 1;
  o.dym = ((y == 0) ? ny - 1 : -1) * nx;
  o.dyp = ((y == ny - 1) ? -(ny - 1) : 1) * nx;
  o.dzm = ((z == 0) ? nz - 1 : -1) * nxy;
  o.dzp = ((z == nz - 1) ? -(nz - 1) : 1) * nxy;
  return o;
}

// Offset from node r to the upstream node r - c_p.
__device__ __forceinline__ int upstream(const Nbr& o, int p) {
  const int cx = CX(p), cy = CY(p), cz = CZ(p);
  int d = 0;
  d += cx == 1 ? o.dxm : (cx == -1 ? o.dxp : 0);
  d += cy == 1 ? o.dym : (cy == -1 ? o.dyp : 0);
  d += cz == 1 ? o.dzm : (cz == -1 ? o.dzp : 0);
  return d;
}

// Pulls the deviation d_p = f_p(r, t) - w_p n_ref of species s: the
// post-collision value of r - c_p, or the reversed population of r itself
// when r - c_p is a wall node (w_p is the same for p and its opposite).
template <int ST, bool WALLS>
__device__ __forceinline__ float pull(const typename Fmt<ST>::T* __restrict__ f,
                                      int64_t N, int s, int p, uint32_t i,
                                      int d, uint32_t lk, float nref) {
  const float wn = WT(p) * nref;
  // branch-free: the bounce-back source only changes the address, so the
  // loads of all directions stay independent and are issued together
  int64_t idx = (int64_t)(s * Q + p) * N + (int64_t)((int)i + d);
  if (WALLS) {
    const int64_t bb = (int64_t)(s * Q + OPP(p)) * N + i;
    idx = ((lk >> p) & 1u) ? bb : idx;
  }
  return Fmt<ST>::ldd(f + idx, wn);
}

// Pulls the stored h_p = d_p / (w_p n_ref) (same addressing as pull).
template <int ST, bool WALLS>
__device__ __forceinline__ float pull_h(const typename Fmt<ST>::T* __restrict__ f,
                                        int64_t N, int s, int p, uint32_t i, int d,
                                        uint32_t lk) {
  int64_t idx = (int64_t)(s * Q + p) * N + (int64_t)((int)i + d);
  if (WALLS) {
    const int64_t bb = (int64_t)(s * Q + OPP(p)) * N + i;
    idx = ((lk >> p) & 1u) ? bb : idx;
  }
  return Fmt<ST>::ldh(f + idx);
}

__device__ __forceinline__ void site_xyz(uint32_t i, int nx, int ny, int& x,
                                         int& y, int& z) {
  const uint32_t t = i / (uint32_t)nx;
  x = (int)(i - t * (uint32_t)nx);
  z = (int)(t / (uint32_t)ny);
  y = (int)(t - (uint32_t)z * (uint32_t)ny);
}

// Gradient of psi at node i: mean of the two face gradients along each axis.
// A wall face takes the Neumann value of the surface-charge condition,
// d psi / d n_out = 4 pi l_B q (q: charge share of the wall node).
template <bool WALLS>
__device__ __forceinline__ void psi_gradient(const StepArgs& a, uint32_t i,
                                             const Nbr& o, uint32_t lk,
                                             float& gx, float& gy, float& gz) {
  const int64_t pc = a.psi[i];
  const int ii = (int)i;
  const int64_t pxp = a.psi[ii + o.dxp], pxm = a.psi[ii + o.dxm];
  const int64_t pyp = a.psi[ii + o.dyp], pym = a.psi[ii + o.dym];
  const int64_t pzp = a.psi[ii + o.dzp], pzm = a.psi[ii + o.dzm];
  float gpx = (float)(pxp - pc) * PSI_INV_SCALE_F;
  float gmx = (float)(pc - pxm) * PSI_INV_SCALE_F;
  float gpy = (float)(pyp - pc) * PSI_INV_SCALE_F;
  float gmy = (float)(pc - pym) * PSI_INV_SCALE_F;
  float gpz = (float)(pzp - pc) * PSI_INV_SCALE_F;
  float gmz = (float)(pc - pzm) * PSI_INV_SCALE_F;
  if (WALLS) {
    // bit 2: r + x is a wall node; bit 1: r - x; 4: +y; 3: -y; 6: +z; 5: -z
    const float k = a.fourpi_lb;
    if (lk & (1u << 2)) gpx = a.wallq ? k * a.wallq[ii + o.dxp] : 0.0f;
    if (lk & (1u << 1)) gmx = a.wallq ? -k * a.wallq[ii + o.dxm] : 0.0f;
    if (lk & (1u << 4)) gpy = a.wallq ? k * a.wallq[ii + o.dyp] : 0.0f;
    if (lk & (1u << 3)) gmy = a.wallq ? -k * a.wallq[ii + o.dym] : 0.0f;
    if (lk & (1u << 6)) gpz = a.wallq ? k * a.wallq[ii + o.dzp] : 0.0f;
    if (lk & (1u << 5)) gmz = a.wallq ? -k * a.wallq[ii + o.dzm] : 0.0f;
  }
  gx = 0.5f * (gpx + gmx);
  gy = 0.5f * (gpy + gmy);
  gz = 0.5f * (gpz + gmz);
}

// Block sum of 64-bit integers (exact), written to part[blockIdx.x].
__device__ __forceinline__ void block_partial(long long v, long long* part) {
  __shared__ long long red[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    part[blockIdx.x] = tot;
  }
}

// Block sum of 64-bit integers (exact), added to *out as one FP64 value per
// block (a block's sum is far below 2^53, so the conversion is exact).
__device__ __forceinline__ void block_sum_to(long long v, double* out) {
  __shared__ long long red[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    atomicAdd(out, (double)tot);
  }
}

// Force per unit mass on species a (Sec. 2): the electric acceleration
// z_a E (E: applied field minus c_s^2 grad psi) and the drag
// -omega_drag sum_b (n_b / n)(v_a - v_b) on the velocities shifted by half
// the electric acceleration, v = u + z E / 2, written with the number-
// weighted mean vb of the v_b (equal masses).
__device__ __forceinline__ void species_force(float usx, float usy, float usz, float zs, float Ex,
                                              float Ey, float Ez, float vbx, float vby, float vbz,
                                              float omd, float& Fx, float& Fy, float& Fz) {
  const float ex = zs * Ex, ey = zs * Ey, ez = zs * Ez;
  Fx = ex - omd * (usx + 0.5f * ex - vbx);
  Fy = ey - omd * (usy + 0.5f * ey - vby);
  Fz = ez - omd * (usz + 0.5f * ez - vbz);
}

// The same with a matrix of pair frequencies (Sec. 2, the general
// gamma^{ab} for equal masses): F_drag^a = -sum_b omega^{ab} x_b (v_a - v_b),
// x_b = n_b / n, written as -(W v_a - M) with W = sum_b omega^{ab} x_b and
// M = sum_b omega^{ab} x_b v_b (xv[b] = x_b v_b; omega^{aa} = 0).
template <int S>
__device__ __forceinline__ void species_force_pair(int sa, float usx, float usy, float usz, float zs,
                                                   float Ex, float Ey, float Ez, const float* x,
                                                   const float (*xv)[3], const StepArgs& a,
                                                   float& Fx, float& Fy, float& Fz) {
  float W = 0.f, Mx = 0.f, My = 0.f, Mz = 0.f;
#pragma unroll
  for (int b = 0; b < S; ++b) {
    const float w = a.pair[sa][b];
    W += w * x[b];
    Mx += w * xv[b][0];
    My += w * xv[b][1];
    Mz += w * xv[b][2];
  }
  const float ex = zs * Ex, ey = zs * Ey, ez = zs * Ez;
  Fx = ex - (W * (usx + 0.5f * ex) - Mx);
  Fy = ey - (W * (usy + 0.5f * ey) - My);
  Fz = ez - (W * (usz + 0.5f * ez) - Mz);
}

inline unsigned nblocks(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace
}  // namespace lbm_gb300
