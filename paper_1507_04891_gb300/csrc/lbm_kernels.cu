// Lattice Boltzmann kernels of the two-timescale multicomponent scheme:
// fused stream + moments + forces + collision, initialisation, charge
// density, moment gathers and FP64 diagnostics.
//
// Storage: structure of arrays, one plane of N values per (species,
// direction), f[(s*19 + p)*N + node], x fastest.  The stored lattice holds
// post-collision populations before streaming; every kernel that needs
// f(t) pulls them from the upstream node r - c_p (halfway bounce-back when
// that node is a wall node), so streaming costs no separate pass.
#include <algorithm>

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
// (only the high bits of the LCG state are used).
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

// ---------------------------------------------------------------------------
// Fused stream + collide, one thread per node, all S species in registers.
//   1. pull the 19*S populations f_p^alpha(r, t), as deviations from
//      w_p n_ref                                            (Eq. latboeq, lhs)
//   2. n^alpha, bare u^alpha = sum c f / n, barycentric u   (Sec. 3 definitions)
//   3. F^alpha = F_el + F_drag: electric z(-c_s^2 grad psi + E) and the drag
//      -omega_drag sum_beta (n_beta/n)(u^a - u^b) on velocities shifted by
//      half the electric acceleration                       (Sec. 2)
//   4. f* = f - omega_visc (f - phi_perp) + g_p              (Eq. latboeq, rhs)
//      phi_perp in its reduced form n w [1 + 3 a + 4.5 a^2 - 1.5 |u^a|^2],
//      a = u^a . c (algebraically equal to the Appendix expression);
//      g_p = n w [3 F.c + 9 (F.c)(u.c) - 3 F.u]             (Eq. ourforc)
//   5. store f* at r.
//   6. FP64 diagnostics of the state after the step (Sec. 3: species
//      continuity, total momentum): every stored value is pulled by exactly
//      one fluid node at the next step (by r + c_p, or by r itself in the
//      opposite direction when r + c_p is a wall node), so the sums of the
//      stored values give the next state's species masses, and the stored
//      values signed by the direction they are pulled in give its momentum.
//      Per CTA: the deviation sums (FP32 within a warp, FP64 across warps)
//      and a count of nodes whose density entering the step was not finite
//      and positive, written to a[blockIdx.x * DIAG_NQ + k].
// ---------------------------------------------------------------------------
template <int S, bool WALLS, bool CHARGED, int ST>
__global__ void __launch_bounds__(256, WALLS ? 2 : 1) k_stream_collide(const StepArgs a) {
  using T = typename Fmt<ST>::T;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  // deviation sums of the state after the step: masses, momentum, charge
  float qm[S], qjx = 0.f, qjy = 0.f, qjz = 0.f, qbad = 0.f;
#pragma unroll
  for (int s = 0; s < S; ++s) qm[s] = 0.f;
  uint32_t lk = 0;
  bool active = i < (uint32_t)a.N;
  if (WALLS && active) {
    lk = a.links[i];
    active = !(lk & LINK_SOLID);
  }
  if (active) {
    int x, y, z;
    site_xyz(i, a.nx, a.ny, x, y, z);
    const Nbr o = neighbours(x, y, z, a.nx, a.ny, a.nz);
    const T* __restrict__ fin = static_cast<const T*>(a.fin);
    T* __restrict__ fout = static_cast<T*>(a.fout);
    const int64_t N = a.N;

    // stored h_p = (f_p - w_p n_ref) / (w_p n_ref) of every species
    float f[S][Q];
#pragma unroll
    for (int p = 0; p < Q; ++p) {
      const int d = upstream(o, p);
#pragma unroll
      for (int s = 0; s < S; ++s) {
        f[s][p] = pull_h<ST, WALLS>(fin, N, s, p, i, d, lk);
      }
    }

    // n = n_ref (1 + sum w h), j = n_ref sum c w h  (sum w = 1, sum w c = 0)
    float mh[S], dn[S], n[S], jx[S], jy[S], jz[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      float m0 = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
      for (int p = 0; p < Q; ++p) {
        const float wh = WT(p) * f[s][p];
        m0 += wh;
        if (CX(p)) mx += CX(p) * wh;
        if (CY(p)) my += CY(p) * wh;
        if (CZ(p)) mz += CZ(p) * wh;
      }
      const float r = a.nref[s];
      mh[s] = m0;
      dn[s] = r * m0;
      n[s] = r + dn[s];
      jx[s] = r * mx;
      jy[s] = r * my;
      jz[s] = r * mz;
      if (!(n[s] > 0.f) || !isfinite(n[s])) qbad = 1.f;
    }

    float ntot = 0.f, Jx = 0.f, Jy = 0.f, Jz = 0.f;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      ntot += n[s];
      Jx += jx[s];
      Jy += jy[s];
      Jz += jz[s];
    }
    const float inv_ntot = 1.0f / ntot;
    // barycentric velocity (equal masses: mass-weighted = number-weighted)
    const float ux = Jx * inv_ntot, uy = Jy * inv_ntot, uz = Jz * inv_ntot;

    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (CHARGED) psi_gradient<WALLS>(a, i, o, lk, gx, gy, gz);
    const float Ex = -CS2 * gx + a.eext[0];
    const float Ey = -CS2 * gy + a.eext[1];
    const float Ez = -CS2 * gz + a.eext[2];

    // number-weighted mean of the drag velocities u^a + F_el^a / 2
    float zn = 0.f;
#pragma unroll
    for (int s = 0; s < S; ++s) zn += a.valence[s] * n[s];
    const float vbx = (Jx + 0.5f * zn * Ex) * inv_ntot;
    const float vby = (Jy + 0.5f * zn * Ey) * inv_ntot;
    const float vbz = (Jz + 0.5f * zn * Ez) * inv_ntot;

    const float om = a.omega_visc;
    const float omd = a.omega_drag_z ? a.omega_drag_z[z] : a.omega_drag;
    uint32_t rnd = 0;
    if (ST != LBM_FP32) rnd = mix32(i * 0x9E3779B9u ^ mix32(a.step_dev ? *a.step_dev : a.step));
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const float inv_n = 1.0f / n[s];
      const float usx = jx[s] * inv_n, usy = jy[s] * inv_n, usz = jz[s] * inv_n;
      float Fx, Fy, Fz;
      species_force(usx, usy, usz, a.valence[s], Ex, Ey, Ez, vbx, vby, vbz, omd, Fx, Fy, Fz);
      const float usq = usx * usx + usy * usy + usz * usz;
      const float Fu = Fx * ux + Fy * uy + Fz * uz;
      // In deviations, d*_p = (1 - omega) d_p + [omega phi_p + g_p - omega w_p n_ref]
      // with, per weight w_p,
      //   omega phi_p + g_p - omega w_p n_ref
      //     = w_p [omega dn + n (-1.5 omega |u^a|^2 - 3 F.u
      //                          + 4.5 omega a^2 + 9 (F.c)(u.c))]      (even in c)
      //     + w_p n 3 (omega a + F.c)                                 (odd in c)
      // a = u^a.c (phi_perp in its reduced form, the Appendix expression;
      // g_p of Eq. ourforc).  Divided by w_p n_ref this updates the stored
      // h = d / (w_p n_ref) directly: h*_p = (1 - omega) h_p + (even' +/- odd') / n_ref,
      // with the bracket values even', odd' free of w_p.  Every term is of
      // the size of the deviations.
      const float base = n[s] * (-1.5f * om * usq - 3.0f * Fu);
      const float odn = om * dn[s];
      const float inr = 1.0f / a.nref[s];
      // moving populations first; the rest population then takes
      // d*_0 = dn - sum_{p>0} d*_p over the stored (rounded) moving values,
      // i.e. h*_0 = (sum w h - sum_{p>0} w h*_p) / w_0, which holds exactly
      // in real arithmetic (phi_perp carries mass n, g_p none) and keeps the
      // rounding of the weights and of 16-bit stores from drifting the
      // species mass.
      // Directions come in opposite pairs (p, p+1), c_{p+1} = -c_p: a = u^a.c,
      // F.c and u.c flip sign, so each pair shares the even part and takes
      // +/- the odd part.
      const float omm = 1.0f - om;
      float moved = 0.f, mjx = 0.f, mjy = 0.f, mjz = 0.f;
#pragma unroll
      for (int p = 1; p < Q; p += 2) {
        const float av = CX(p) * usx + CY(p) * usy + CZ(p) * usz;
        const float fc = CX(p) * Fx + CY(p) * Fy + CZ(p) * Fz;
        const float uc = CX(p) * ux + CY(p) * uy + CZ(p) * uz;
        const float even = inr * (odn + base + n[s] * (4.5f * om * av * av + 9.0f * fc * uc));
        const float odd = inr * n[s] * 3.0f * (om * av + fc);
        const float2 hs = Fmt<ST>::sth_sr2(fout + (int64_t)(s * Q + p) * N + i,
                                           omm * f[s][p] + (even + odd),
                                           fout + (int64_t)(s * Q + p + 1) * N + i,
                                           omm * f[s][p + 1] + (even - odd), lcg_next(rnd));
        moved += WT(p) * (hs.x + hs.y);  // same weight for p and p+1
        // momentum carried by the pair at the next step: h*_p moves along
        // c_p unless r + c_p is a wall node (bit p+1), then it is pulled
        // back along -c_p; h*_{p+1} likewise with bit p
        float mj = hs.x - hs.y;
        if (WALLS) mj = (((lk >> (p + 1)) & 1u) ? -hs.x : hs.x) - (((lk >> p) & 1u) ? -hs.y : hs.y);
        if (CX(p)) mjx += CX(p) * WT(p) * mj;
        if (CY(p)) mjy += CY(p) * WT(p) * mj;
        if (CZ(p)) mjz += CZ(p) * WT(p) * mj;
      }
      const float h0 = Fmt<ST>::sth_sr(fout + (int64_t)(s * Q) * N + i, (mh[s] - moved) * INV_WT(0),
                                       lcg_next(rnd));
      const float r = a.nref[s];
      qm[s] = r * (WT(0) * h0 + moved);
      qjx += r * mjx;
      qjy += r * mjy;
      qjz += r * mjz;
    }
  }

  // per-CTA partial sums of the diagnostics (inactive threads add zeros)
  if (a.diag) {
    float q[DIAG_NQ];
#pragma unroll
    for (int k = 0; k < DIAG_NQ; ++k) q[k] = 0.f;
    float qc = 0.f;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      q[s] = qm[s];
      qc += a.valence[s] * qm[s];
    }
    q[MAX_SPECIES + 0] = qjx;
    q[MAX_SPECIES + 1] = qjy;
    q[MAX_SPECIES + 2] = qjz;
    q[MAX_SPECIES + 3] = qc;
    q[MAX_SPECIES + 4] = qbad;
    __shared__ float red[8][DIAG_NQ];
#pragma unroll
    for (int k = 0; k < DIAG_NQ; ++k) {
      float v = q[k];
      if (k >= S && k < MAX_SPECIES) continue;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < DIAG_NQ) {
      const int k = threadIdx.x;
      double tot = 0.0;
      if (k < S || k >= MAX_SPECIES)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += (double)red[w][k];
      a.diag[(int64_t)blockIdx.x * DIAG_NQ + k] = tot;
    }
  }
}

// ---------------------------------------------------------------------------
// Initialisation: f_p(r, 0) = phi_perp,p(n0, u0), i.e. the equilibrium at the
// species velocity, written to the stored lattice at the upstream node so
// that the next pull returns it (inverse streaming).
// ---------------------------------------------------------------------------
template <bool WALLS, int ST>
__global__ void k_init(int s, const double* __restrict__ n0,
                       const double* __restrict__ u0, const uint32_t* links,
                       void* fout_v, int nx, int ny, int nz, int64_t N,
                       float nref) {
  using T = typename Fmt<ST>::T;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (uint32_t)N) return;
  uint32_t lk = 0;
  if (WALLS) {
    lk = links[i];
    if (lk & LINK_SOLID) return;
  }
  int x, y, z;
  site_xyz(i, nx, ny, x, y, z);
  const Nbr o = neighbours(x, y, z, nx, ny, nz);
  T* fout = static_cast<T*>(fout_v);
  const float n = (float)n0[i];
  const float dn = (float)(n0[i] - (double)nref);  // deviation from n_ref, exact in FP64
  float vx = 0.f, vy = 0.f, vz = 0.f;
  if (u0) {
    vx = (float)u0[i];
    vy = (float)u0[N + i];
    vz = (float)u0[2 * N + i];
  }
  const float usq = vx * vx + vy * vy + vz * vz;
#pragma unroll
  for (int p = 0; p < Q; ++p) {
    const float av = CX(p) * vx + CY(p) * vy + CZ(p) * vz;
    // phi_p - w_p n_ref = w_p [dn + n (3 a + 4.5 a^2 - 1.5 |u|^2)]
    const float deq = WT(p) * (dn + n * (3.0f * av + 4.5f * av * av - 1.5f * usq));
    int64_t dst;
    int q = p;
    if (WALLS && ((lk >> p) & 1u)) {
      q = OPP(p);
      dst = i;
    } else {
      dst = (int64_t)((int)i + upstream(o, p));
    }
    Fmt<ST>::st(fout + (int64_t)(s * Q + q) * N + dst, deq, INV_WT(q) / nref);
  }
}

// ---------------------------------------------------------------------------
// Charge density for the Poisson source: s_r = 4 pi l_B (rho_e + w_r) with
// rho_e = sum_alpha z^alpha n^alpha(r, t) from the pulled populations of the
// charged species; per-CTA sums of s over fluid nodes (exact, int64).
// ---------------------------------------------------------------------------
// NC charged species, species indices cs, valences val, reference densities
// nref (the neutral species are not read).
template <int NC, bool WALLS, int ST>
__global__ void __launch_bounds__(256) k_charge(
    const void* fin_v, const uint32_t* links, const int64_t* wsrc, int64_t* src,
    long long* part, const int* label, unsigned long long* comp_sum, int nx, int ny,
    int nz, int64_t N, int4 cs, float4 val, float4 nref, float fourpi_lb, long long src_ref) {
  using T = typename Fmt<ST>::T;
  const T* fin = static_cast<const T*>(fin_v);
  const int sp[4] = {cs.x, cs.y, cs.z, cs.w};
  const float vz[4] = {val.x, val.y, val.z, val.w};
  const float nr[4] = {nref.x, nref.y, nref.z, nref.w};
  long long acc = 0;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (uint32_t)N) {
    uint32_t lk = 0;
    bool fluid = true;
    if (WALLS) {
      lk = links[i];
      fluid = !(lk & LINK_SOLID);
    }
    long long sv = 0;
    if (fluid) {
      int x, y, z;
      site_xyz(i, nx, ny, x, y, z);
      const Nbr o = neighbours(x, y, z, nx, ny, nz);
      // rho_e = sum z n_ref + sum z dn: the first part is the same at every
      // node (src_ref, fixed point, from the host); the deviations carry
      // the local charge at full FP32 precision
      // all pulls of the charged species are independent and in one basic
      // block, so that they are in flight together
      float v[NC > 0 ? NC : 1][Q];
#pragma unroll
      for (int p = 0; p < Q; ++p) {
        const int d = upstream(o, p);
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c][p] = pull<ST, WALLS>(fin, N, sp[c], p, i, d, lk, nr[c]);
      }
      float drho = 0.f;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float m0 = 0.f;
#pragma unroll
        for (int p = 0; p < Q; ++p) m0 += v[c][p];
        drho += vz[c] * m0;
      }
      // exact conversion: a float times a power of two, to a 64-bit integer;
      // the wall charge is already in fixed point
      sv = src_ref + (long long)(fourpi_lb * drho * PSI_SCALE_F);
      if (wsrc) sv += wsrc[i];
    }
    src[i] = sv;
    // the largest fluid component (label 0) is summed per CTA; the cells of
    // other components (rare: pockets closed off by walls) add to their own
    // sum (two's-complement wrap-around keeps the 64-bit sum exact)
    if (label && fluid && label[i] != 0)
      atomicAdd(comp_sum + label[i], (unsigned long long)sv);
    else
      acc = sv;
  }
  block_partial(acc, part);
}

// Sums the per-CTA partials of k_charge into *out exactly in 128-bit
// integers (FP64 arithmetic is slow on this GPU), converted to FP64 once.
// When mean_z is given (one periodic run of fluid planes), the source mean
// over the fluid, rounded to the fixed-point grid, is written to its nz
// planes; when step is given, the step counter of the graph steps is
// advanced (both save a launch per step).
__global__ void __launch_bounds__(1024) k_sum_partials(const long long* part, int n,
                                                       double* out, long long* mean_z, int nz,
                                                       double inv_nfluid, uint32_t* step) {
  __shared__ long long red_hi[32];
  __shared__ unsigned long long red_lo[32];
  __shared__ long long s_mean;
  __int128 v = 0;
#pragma unroll 8
  for (int k = threadIdx.x; k < n; k += blockDim.x) v += (__int128)part[k];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const long long hi = __shfl_down_sync(0xffffffffu, (long long)(v >> 64), off);
    const unsigned long long lo = __shfl_down_sync(0xffffffffu, (unsigned long long)v, off);
    v += ((__int128)hi << 64) | (__int128)lo;
  }
  if ((threadIdx.x & 31) == 0) {
    red_hi[threadIdx.x >> 5] = (long long)(v >> 64);
    red_lo[threadIdx.x >> 5] = (unsigned long long)v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __int128 tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      tot += ((__int128)red_hi[w] << 64) | (__int128)red_lo[w];
    const double t = (double)tot;
    *out = t;
    s_mean = llrint(t * inv_nfluid);
    if (step) *step += 1u;
  }
  if (mean_z) {
    __syncthreads();
    for (int z = threadIdx.x; z < nz; z += blockDim.x) mean_z[z] = s_mean;
  }
}

// Gathers f(t) of species s and its moments n, u = sum c f / n (doubles,
// from the deviations: n = n_ref + sum d, j = sum c d).
template <bool WALLS, int ST>
__global__ void k_gather(const void* fin_v, const uint32_t* links, int s,
                         int nx, int ny, int nz, int64_t N, float nref,
                         double* n_out, double* u_out, double* f_out) {
  using T = typename Fmt<ST>::T;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (uint32_t)N) return;
  uint32_t lk = 0;
  if (WALLS) lk = links[i];
  if (WALLS && (lk & LINK_SOLID)) {
    if (n_out) n_out[i] = 0.0;
    if (u_out) u_out[i] = u_out[N + i] = u_out[2 * N + i] = 0.0;
    if (f_out)
      for (int p = 0; p < Q; ++p) f_out[(int64_t)p * N + i] = 0.0;
    return;
  }
  int x, y, z;
  site_xyz(i, nx, ny, x, y, z);
  const Nbr o = neighbours(x, y, z, nx, ny, nz);
  const T* fin = static_cast<const T*>(fin_v);
  double m0 = nref, mx = 0, my = 0, mz = 0;
#pragma unroll
  for (int p = 0; p < Q; ++p) {
    const float v = pull<ST, WALLS>(fin, N, s, p, i, upstream(o, p), lk, nref);
    if (f_out) f_out[(int64_t)p * N + i] = (double)WT(p) * nref + (double)v;
    m0 += v;
    mx += CX(p) * (double)v;
    my += CY(p) * (double)v;
    mz += CZ(p) * (double)v;
  }
  if (n_out) n_out[i] = m0;
  if (u_out) {
    u_out[i] = mx / m0;
    u_out[N + i] = my / m0;
    u_out[2 * N + i] = mz / m0;
  }
}

// Diagnostics: per species the sum over fluid nodes of dn = n - n_ref, the
// total momentum and the net charge of the deviations (the host adds the
// reference parts n_ref x fluid nodes, exactly); flags non-finite or
// non-positive densities.  One node per thread, all species' loads in
// flight; deviations summed per warp in FP32 (they are small next to the
// reference part, so their rounding is far below the FP64 resolution of the
// total), per CTA in FP64, and added to one of DIAG_SPREAD partial slots per
// quantity (slot b mod DIAG_SPREAD for CTA b: FP64 atomics of thousands of
// CTAs on one address queue).  out layout: quantity k in
// [k * DIAG_SPREAD, (k + 1) * DIAG_SPREAD), k < MAX_SPECIES: dn per species,
// then momentum x, y, z, then charge.
template <int S, bool WALLS, int ST>
__global__ void __launch_bounds__(256) k_diag(const void* fin_v,
                                              const uint32_t* links, int nx,
                                              int ny, int nz, int64_t N,
                                              float4 val, float4 nref,
                                              double* out, int* bad) {
  using T = typename Fmt<ST>::T;
  constexpr int NQ = MAX_SPECIES + 4;
  float acc[NQ];
#pragma unroll
  for (int k = 0; k < NQ; ++k) acc[k] = 0.f;
  const float vz[4] = {val.x, val.y, val.z, val.w};
  const float nr[4] = {nref.x, nref.y, nref.z, nref.w};
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (uint32_t)N) {
    uint32_t lk = 0;
    bool fluid = true;
    if (WALLS) {
      lk = links[i];
      fluid = !(lk & LINK_SOLID);
    }
    if (fluid) {
      int x, y, z;
      site_xyz(i, nx, ny, x, y, z);
      const Nbr o = neighbours(x, y, z, nx, ny, nz);
      const T* fin = static_cast<const T*>(fin_v);
      float v[S][Q];
#pragma unroll
      for (int p = 0; p < Q; ++p) {
        const int d = upstream(o, p);
#pragma unroll
        for (int s = 0; s < S; ++s) v[s][p] = pull<ST, WALLS>(fin, N, s, p, i, d, lk, nr[s]);
      }
#pragma unroll
      for (int s = 0; s < S; ++s) {
        float m0 = 0, mx = 0, my = 0, mz = 0;
#pragma unroll
        for (int p = 0; p < Q; ++p) {
          m0 += v[s][p];
          mx += CX(p) * v[s][p];
          my += CY(p) * v[s][p];
          mz += CZ(p) * v[s][p];
        }
        if (!(nr[s] + m0 > 0.f) || !isfinite(m0) || !isfinite(mx) || !isfinite(my) ||
            !isfinite(mz))
          atomicOr(bad, 1);
        acc[s] += m0;
        acc[MAX_SPECIES + 0] += mx;
        acc[MAX_SPECIES + 1] += my;
        acc[MAX_SPECIES + 2] += mz;
        acc[MAX_SPECIES + 3] += vz[s] * m0;
      }
    }
  }
  __shared__ double red[8][NQ];
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    float v = acc[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = (double)v;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w][threadIdx.x];
    atomicAdd(out + threadIdx.x * DIAG_SPREAD + (blockIdx.x & (DIAG_SPREAD - 1)), tot);
  }
}

// Plane sums of the current state f(t): one CTA per z-plane; for each
// species the sum over the plane's fluid nodes of n^a and of the mid-step
// flux n^a (u^a + F^a / 2) (the velocity of the second-order forcing,
// Eq. ourforc), F^a the force of the stream/collide kernel (species_force)
// on f(t) with the potential in a.psi.  out[(z S + s) 4 + k], k = 0: n,
// 1..3: flux x, y, z.  Node values in FP32 (as in the step), sums in FP64.
template <int S, bool WALLS, bool CHARGED, int ST>
__global__ void __launch_bounds__(256) k_plane_fluxes(const StepArgs a, double* __restrict__ out) {
  using T = typename Fmt<ST>::T;
  const int z = blockIdx.x;
  const int nxy = a.nx * a.ny;
  double acc[S][4];
#pragma unroll
  for (int s = 0; s < S; ++s)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[s][k] = 0.0;
  const T* __restrict__ fin = static_cast<const T*>(a.fin);
  for (int k = threadIdx.x; k < nxy; k += blockDim.x) {
    const uint32_t i = (uint32_t)z * (uint32_t)nxy + (uint32_t)k;
    uint32_t lk = 0;
    if (WALLS) {
      lk = a.links[i];
      if (lk & LINK_SOLID) continue;
    }
    int x, y, zz;
    site_xyz(i, a.nx, a.ny, x, y, zz);
    const Nbr o = neighbours(x, y, zz, a.nx, a.ny, a.nz);
    float n[S], jx[S], jy[S], jz[S];
    float ntot = 0.f, Jx = 0.f, Jy = 0.f, Jz = 0.f, zn = 0.f;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      float m0 = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
      for (int p = 0; p < Q; ++p) {
        const float wh = WT(p) * pull_h<ST, WALLS>(fin, a.N, s, p, i, upstream(o, p), lk);
        m0 += wh;
        if (CX(p)) mx += CX(p) * wh;
        if (CY(p)) my += CY(p) * wh;
        if (CZ(p)) mz += CZ(p) * wh;
      }
      const float r = a.nref[s];
      n[s] = r + r * m0;
      jx[s] = r * mx;
      jy[s] = r * my;
      jz[s] = r * mz;
      ntot += n[s];
      Jx += jx[s];
      Jy += jy[s];
      Jz += jz[s];
      zn += a.valence[s] * n[s];
    }
    const float inv_ntot = 1.0f / ntot;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (CHARGED) psi_gradient<WALLS>(a, i, o, lk, gx, gy, gz);
    const float Ex = -CS2 * gx + a.eext[0];
    const float Ey = -CS2 * gy + a.eext[1];
    const float Ez = -CS2 * gz + a.eext[2];
    const float vbx = (Jx + 0.5f * zn * Ex) * inv_ntot;
    const float vby = (Jy + 0.5f * zn * Ey) * inv_ntot;
    const float vbz = (Jz + 0.5f * zn * Ez) * inv_ntot;
    const float omd = a.omega_drag_z ? a.omega_drag_z[zz] : a.omega_drag;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const float inv_n = 1.0f / n[s];
      float Fx, Fy, Fz;
      species_force(jx[s] * inv_n, jy[s] * inv_n, jz[s] * inv_n, a.valence[s], Ex, Ey, Ez, vbx, vby,
                    vbz, omd, Fx, Fy, Fz);
      acc[s][0] += (double)n[s];
      acc[s][1] += (double)(jx[s] + 0.5f * n[s] * Fx);
      acc[s][2] += (double)(jy[s] + 0.5f * n[s] * Fy);
      acc[s][3] += (double)(jz[s] + 0.5f * n[s] * Fz);
    }
  }
  __shared__ double red[8][S * 4];
#pragma unroll
  for (int s = 0; s < S; ++s)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double v = acc[s][k];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][s * 4 + k] = v;
    }
  __syncthreads();
  if (threadIdx.x < S * 4) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
    out[(int64_t)z * S * 4 + threadIdx.x] = t;
  }
}

// Checks an initial density (and velocity) field in device memory: per CTA
// (grid-stride) the sum of n0 over fluid nodes and the number of fluid nodes
// where n0 is not finite and positive or u0 not finite, written to
// out[2 b], out[2 b + 1].
__global__ void __launch_bounds__(256) k_species_check(const double* __restrict__ n0,
                                                       const double* __restrict__ u0,
                                                       const uint32_t* __restrict__ links,
                                                       int64_t N, double* __restrict__ out) {
  double sum = 0.0, bad = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (links && (links[i] & LINK_SOLID)) continue;
    const double v = n0[i];
    bool ok = v > 0.0 && isfinite(v);
    if (u0) ok = ok && isfinite(u0[i]) && isfinite(u0[N + i]) && isfinite(u0[2 * N + i]);
    if (ok) sum += v;
    else bad += 1.0;
  }
  __shared__ double red[2][8];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sum += __shfl_down_sync(0xffffffffu, sum, off);
    bad += __shfl_down_sync(0xffffffffu, bad, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sum;
    red[1][threadIdx.x >> 5] = bad;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
    out[2 * blockIdx.x + threadIdx.x] = t;
  }
}

// Sums the per-CTA diagnostics partials of the stream/collide kernel: one
// CTA per quantity, FP64, in a fixed order (the result does not depend on
// scheduling).
__global__ void __launch_bounds__(256) k_diag_reduce(const double* __restrict__ part,
                                                     int64_t nctas, double* __restrict__ out) {
  const int k = blockIdx.x;
  double v = 0.0;
  for (int64_t c = threadIdx.x; c < nctas; c += blockDim.x) v += part[c * DIAG_NQ + k];
  __shared__ double red[8];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[k] = t;
  }
}

// Link words from the wall mask: bit 0 = wall node, bit p = r - c_p is wall.
__global__ void k_links(const uint8_t* solid, uint32_t* links, int nx, int ny,
                        int nz, int64_t N) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (uint32_t)N) return;
  int x, y, z;
  site_xyz(i, nx, ny, x, y, z);
  const Nbr o = neighbours(x, y, z, nx, ny, nz);
  uint32_t w = solid[i] ? LINK_SOLID : 0u;
#pragma unroll
  for (int p = 1; p < Q; ++p)
    if (solid[(int)i + upstream(o, p)]) w |= 1u << p;
  links[i] = w;
}

__global__ void k_psi_to_double(const int64_t* psi, double* out, int64_t N) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) out[i] = (double)psi[i] * PSI_INV_SCALE;
}

__global__ void k_psi_from_double(const double* in, int64_t* psi,
                                  const uint32_t* links, int64_t N) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const bool solid = links && (links[i] & LINK_SOLID);
  psi[i] = solid ? 0 : llrint(in[i] * PSI_SCALE);
}

__global__ void __launch_bounds__(256) k_src_from_rho(
    const double* rho, const uint32_t* links, const int64_t* wsrc, int64_t* src,
    double* dsum, const int* label, unsigned long long* comp_sum, int64_t N,
    double fourpi_lb) {
  long long acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool solid = links && (links[i] & LINK_SOLID);
    long long sv = 0;
    if (!solid) sv = llrint(fourpi_lb * rho[i] * PSI_SCALE) + (wsrc ? wsrc[i] : 0);
    src[i] = sv;
    if (label && !solid && label[i] != 0)
      atomicAdd(comp_sum + label[i], (unsigned long long)sv);
    else
      acc += sv;
  }
  block_sum_to(acc, dsum);
}

// Mean of the source over each fluid component, in fixed point:
// component 0 from the CTA sums in dsum[0], the others from comp_sum.
__global__ void k_comp_means(const double* dsum, const unsigned long long* comp_sum,
                             const long long* comp_size, int ncomp, long long* comp_mean) {
  for (int k = threadIdx.x; k < ncomp; k += blockDim.x) {
    if (k == 0)
      comp_mean[0] = llrint(dsum[0] / (double)comp_size[0]);
    else
      comp_mean[k] = llrint((double)(long long)comp_sum[k] / (double)comp_size[k]);
  }
}

inline unsigned nblocks(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <int S, bool W, bool C, int ST>
cudaError_t launch_sc(const StepArgs& a, cudaStream_t st, int threads) {
  k_stream_collide<S, W, C, ST><<<nblocks(a.N, threads), threads, 0, st>>>(a);
  return cudaGetLastError();
}

template <int S, int ST>
cudaError_t dispatch_wc(const StepArgs& a, bool w, bool c, cudaStream_t st, int t) {
  if (w) return c ? launch_sc<S, true, true, ST>(a, st, t) : launch_sc<S, true, false, ST>(a, st, t);
  return c ? launch_sc<S, false, true, ST>(a, st, t) : launch_sc<S, false, false, ST>(a, st, t);
}

template <int ST>
cudaError_t dispatch_s(const StepArgs& a, int S, bool w, bool c, cudaStream_t st, int t) {
  switch (S) {
    case 1: return dispatch_wc<1, ST>(a, w, c, st, t);
    case 2: return dispatch_wc<2, ST>(a, w, c, st, t);
    case 3: return dispatch_wc<3, ST>(a, w, c, st, t);
    case 4: return dispatch_wc<4, ST>(a, w, c, st, t);
  }
  return cudaErrorInvalidValue;
}

float4 as_f4(const float* v) { return make_float4(v[0], v[1], v[2], v[3]); }

}  // namespace

namespace {
StepArgs step_args(lbm_t* h) {
  StepArgs a;
  a.fin = h->f[h->cur];
  a.fout = h->f[h->cur ^ 1];
  a.links = h->links;
  const bool charged = h->cfg.bjerrum > 0.0;
  a.psi = charged ? h->ps.psi[h->ps.cur] : nullptr;
  a.wallq = h->wallq;
  a.nx = h->cfg.nx;
  a.ny = h->cfg.ny;
  a.nz = h->cfg.nz;
  a.N = h->N;
  a.omega_visc = (float)h->cfg.omega_visc;
  a.omega_drag = (float)h->cfg.omega_drag;
  a.omega_drag_z = h->omega_drag_z;
  a.fourpi_lb = (float)(4.0 * 3.14159265358979323846 * h->cfg.bjerrum);
  for (int d = 0; d < 3; ++d) a.eext[d] = (float)h->cfg.e_ext[d];
  for (int s = 0; s < MAX_SPECIES; ++s) {
    a.valence[s] = h->valence[s];
    a.nref[s] = h->nref[s];
  }
  a.step = (uint32_t)h->tstep;
  a.step_dev = nullptr;
  if (h->gstatus) a.step_dev = reinterpret_cast<const uint32_t*>(h->gstatus);
  a.diag = h->dpart;
  return a;
}

cudaError_t collide_into_spare(lbm_t* h, int threads) {
  const StepArgs a = step_args(h);
  const bool charged = h->cfg.bjerrum > 0.0;
  h->dpart_ctas = (int64_t)nblocks(h->N, threads);
  switch (h->cfg.storage) {
    case LBM_FP32: return dispatch_s<LBM_FP32>(a, h->S, h->has_walls, charged, h->st, threads);
    case LBM_FP16_SHIFT: return dispatch_s<LBM_FP16_SHIFT>(a, h->S, h->has_walls, charged, h->st, threads);
    case LBM_BF16_SHIFT: return dispatch_s<LBM_BF16_SHIFT>(a, h->S, h->has_walls, charged, h->st, threads);
  }
  return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_stream_collide(lbm_t* h) {
  cudaError_t e = collide_into_spare(h, h->collide_threads);
  if (e == cudaSuccess) {
    h->cur ^= 1;
    ++h->launches;
    h->diag_valid = true;
  }
  return e;
}

cudaError_t launch_stream_collide_probe(lbm_t* h, int threads) {
  cudaError_t e = collide_into_spare(h, threads);
  if (e == cudaSuccess) ++h->launches;
  h->diag_valid = false;  // the partials describe the spare lattice
  return e;
}

cudaError_t launch_species_check(lbm_t* h, const double* n0_dev, const double* u0_dev, double* out,
                                 int* nblk) {
  const int nb = (int)std::min<int64_t>(nblocks(h->N, 256), 256);
  k_species_check<<<nb, 256, 0, h->st>>>(n0_dev, u0_dev, h->links, h->N, out);
  ++h->launches;
  *nblk = nb;
  return cudaGetLastError();
}

cudaError_t launch_diag_reduce(lbm_t* h, double* out) {
  k_diag_reduce<<<DIAG_NQ, 256, 0, h->st>>>(h->dpart, h->dpart_ctas, out);
  ++h->launches;
  return cudaGetLastError();
}

#define LBM_DISPATCH_WS(h, KERNEL_CALL)                                        \
  do {                                                                         \
    const bool _w = (h)->has_walls;                                            \
    switch ((h)->cfg.storage) {                                                \
      case LBM_FP32:                                                           \
        if (_w) { constexpr bool W_ = true; constexpr int ST_ = LBM_FP32; KERNEL_CALL; } \
        else { constexpr bool W_ = false; constexpr int ST_ = LBM_FP32; KERNEL_CALL; } \
        break;                                                                 \
      case LBM_FP16_SHIFT:                                                     \
        if (_w) { constexpr bool W_ = true; constexpr int ST_ = LBM_FP16_SHIFT; KERNEL_CALL; } \
        else { constexpr bool W_ = false; constexpr int ST_ = LBM_FP16_SHIFT; KERNEL_CALL; } \
        break;                                                                 \
      default:                                                                 \
        if (_w) { constexpr bool W_ = true; constexpr int ST_ = LBM_BF16_SHIFT; KERNEL_CALL; } \
        else { constexpr bool W_ = false; constexpr int ST_ = LBM_BF16_SHIFT; KERNEL_CALL; } \
        break;                                                                 \
    }                                                                          \
  } while (0)

cudaError_t launch_plane_fluxes(lbm_t* h, double* out_dev) {
  const StepArgs a = step_args(h);
  const bool c = h->cfg.bjerrum > 0.0;
  const unsigned nb = (unsigned)h->cfg.nz;
#define LBM_PF(SS)                                                                   \
  LBM_DISPATCH_WS(h, (c ? k_plane_fluxes<SS, W_, true, ST_><<<nb, 256, 0, h->st>>>(a, out_dev)  \
                        : k_plane_fluxes<SS, W_, false, ST_><<<nb, 256, 0, h->st>>>(a, out_dev)))
  switch (h->S) {
    case 1: LBM_PF(1); break;
    case 2: LBM_PF(2); break;
    case 3: LBM_PF(3); break;
    default: LBM_PF(4); break;
  }
#undef LBM_PF
  ++h->launches;
  return cudaGetLastError();
}

cudaError_t launch_init_species(lbm_t* h, int s, const double* n0,
                                const double* u0) {
  const int nb = nblocks(h->N, 256);
  LBM_DISPATCH_WS(h, (k_init<W_, ST_><<<nb, 256, 0, h->st>>>(
                         s, n0, u0, h->links, h->f[h->cur], h->cfg.nx,
                         h->cfg.ny, h->cfg.nz, h->N, h->nref[s])));
  ++h->launches;
  return cudaGetLastError();
}

cudaError_t launch_charge(lbm_t* h) {
  // one node per thread (the pulled loads of a node are independent and all
  // in flight); per-CTA partial sums instead of same-address atomics
  const int ct = h->charge_threads;
  const int nb = (int)nblocks(h->N, ct);
  const float k = (float)(4.0 * 3.14159265358979323846 * h->cfg.bjerrum);
  // reference part of the source, 4 pi l_B sum_alpha z^alpha n_ref^alpha,
  // in fixed point (FP64 on the host, the same at every fluid node)
  double zref = 0.0;
  for (int s = 0; s < h->S; ++s) zref += (double)h->valence[s] * (double)h->nref[s];
  const long long src_ref = llrint(4.0 * 3.14159265358979323846 * h->cfg.bjerrum * zref * PSI_SCALE);
  // the charged species, packed
  int csi[4] = {0, 0, 0, 0};
  float cval[4] = {0.f, 0.f, 0.f, 0.f}, cref[4] = {1.f, 1.f, 1.f, 1.f};
  int nc = 0;
  for (int s = 0; s < h->S; ++s)
    if (h->valence[s] != 0.f) {
      csi[nc] = s;
      cval[nc] = h->valence[s];
      cref[nc] = h->nref[s];
      ++nc;
    }
  const int4 cs4 = make_int4(csi[0], csi[1], csi[2], csi[3]);
  const float4 cv4 = make_float4(cval[0], cval[1], cval[2], cval[3]);
  const float4 cr4 = make_float4(cref[0], cref[1], cref[2], cref[3]);
#define LBM_CHARGE_S(NC)                                                        \
  LBM_DISPATCH_WS(h, (k_charge<NC, W_, ST_><<<nb, ct, 0, h->st>>>(               \
                         h->f[h->cur], h->links, h->wsrc, h->ps.src, h->ps.part, \
                         h->ps.label, h->ps.comp_sum,                            \
                         h->cfg.nx, h->cfg.ny, h->cfg.nz, h->N,                  \
                         cs4, cv4, cr4, k, src_ref)))
  switch (nc) {
    case 0: LBM_CHARGE_S(0); break;
    case 1: LBM_CHARGE_S(1); break;
    case 2: LBM_CHARGE_S(2); break;
    case 3: LBM_CHARGE_S(3); break;
    default: LBM_CHARGE_S(4); break;
  }
#undef LBM_CHARGE_S
  // the spectral solver's source mean for one periodic run is written here;
  // the solve then skips its own mean kernel once (charge_means_ready)
  long long* mz = h->charge_mean_z;
  k_sum_partials<<<1, 1024, 0, h->st>>>(h->ps.part, nb, h->ps.dsum, mz, h->cfg.nz,
                                        1.0 / (double)h->nfluid, h->charge_step);
  h->charge_means_ready = mz != nullptr;
  h->launches += 2;
  if (h->ps.label) {
    k_comp_means<<<1, 256, 0, h->st>>>(h->ps.dsum, h->ps.comp_sum, h->ps.comp_size,
                                        h->ps.ncomp, h->ps.comp_mean);
    ++h->launches;
  }
  return cudaGetLastError();
}

cudaError_t launch_gather(lbm_t* h, int s, double* n_dev, double* u_dev,
                          double* f_dev) {
  const int nb = nblocks(h->N, 256);
  LBM_DISPATCH_WS(h, (k_gather<W_, ST_><<<nb, 256, 0, h->st>>>(
                         h->f[h->cur], h->links, s, h->cfg.nx, h->cfg.ny,
                         h->cfg.nz, h->N, h->nref[s], n_dev, u_dev, f_dev)));
  ++h->launches;
  return cudaGetLastError();
}

cudaError_t launch_diagnostics(lbm_t* h) {
  const int nb = (int)nblocks(h->N, 256);
#define LBM_DIAG_S(SS)                                                         \
  LBM_DISPATCH_WS(h, (k_diag<SS, W_, ST_><<<nb, 256, 0, h->st>>>(               \
                         h->f[h->cur], h->links, h->cfg.nx, h->cfg.ny,         \
                         h->cfg.nz, h->N, as_f4(h->valence),                   \
                         as_f4(h->nref), h->dred, h->dflag)))
  switch (h->S) {
    case 1: LBM_DIAG_S(1); break;
    case 2: LBM_DIAG_S(2); break;
    case 3: LBM_DIAG_S(3); break;
    default: LBM_DIAG_S(4); break;
  }
#undef LBM_DIAG_S
  ++h->launches;
  return cudaGetLastError();
}

cudaError_t launch_links(lbm_t* h, const uint8_t* solid_dev) {
  k_links<<<nblocks(h->N, 256), 256, 0, h->st>>>(solid_dev, h->links, h->cfg.nx,
                                                h->cfg.ny, h->cfg.nz, h->N);
  ++h->launches;
  return cudaGetLastError();
}

cudaError_t launch_psi_to_double(lbm_t* h, const int64_t* psi, double* out) {
  k_psi_to_double<<<nblocks(h->N, 256), 256, 0, h->st>>>(psi, out, h->N);
  ++h->launches;
  return cudaGetLastError();
}

cudaError_t launch_psi_from_double(lbm_t* h, const double* in, int64_t* psi) {
  k_psi_from_double<<<nblocks(h->N, 256), 256, 0, h->st>>>(in, psi, h->links, h->N);
  ++h->launches;
  return cudaGetLastError();
}

cudaError_t launch_src_from_rho(lbm_t* h, const double* rho_dev) {
  const double k = 4.0 * 3.14159265358979323846 * h->cfg.bjerrum;
  k_src_from_rho<<<(unsigned)std::min<int64_t>(nblocks(h->N, 256), h->grid_cap), 256, 0,
                   h->st>>>(rho_dev, h->links, h->wsrc, h->ps.src, h->ps.dsum, h->ps.label,
                            h->ps.comp_sum, h->N, k);
  if (h->ps.label) {
    k_comp_means<<<1, 256, 0, h->st>>>(h->ps.dsum, h->ps.comp_sum, h->ps.comp_size,
                                        h->ps.ncomp, h->ps.comp_mean);
    ++h->launches;
  }
  ++h->launches;
  return cudaGetLastError();
}

}  // namespace lbm_gb300
