// Lattice Boltzmann kernels of the two-timescale multicomponent scheme other
// than the fused stream/collide (lbm_collide.cu): initialisation, charge
// density, moment gathers, plane sums, FP64 diagnostics, wall links and
// potential conversions, and the host-side launchers of all of them.
#include <algorithm>

#include "lbm_lattice.cuh"

namespace lbm_gb300 {
namespace {

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
// The start's first pass fused into the charge pass (DotsArgs): for this
// thread's NV consecutive nodes from i0 (i0 a multiple of NV), the source
// differences d0 against the stored D_1 .. D_K (ring slot of age j:
// (r - j) mod K, read before d0 replaces the oldest, slot r mod K), summed
// per CTA in FP32 into part (K + 1 values per CTA), as k_start_dots does.
// The stored differences of this thread's nodes, loaded before the pulls
// so that they are in flight with them.
template <int NV>
__device__ __forceinline__ void dots_load(const DotsArgs& dk, int64_t N, int64_t i0, int r,
                                          float (&dj)[START_K + 1][NV]) {
  constexpr int K = START_K;
#pragma unroll
  for (int j = 1; j <= K; ++j) {
    const float* rs = dk.ring_d + (int64_t)((r - j + 2 * K) % K) * N + i0;
    if (NV == 4) {
      const float4 w = *reinterpret_cast<const float4*>(rs);
      dj[j][0] = w.x; dj[j][NV > 1 ? 1 : 0] = w.y; dj[j][NV > 2 ? 2 : 0] = w.z;
      dj[j][NV > 3 ? 3 : 0] = w.w;
    } else {
#pragma unroll
      for (int u = 0; u < NV; ++u) dj[j][u] = rs[u];
    }
  }
}

template <int NV>
__device__ __forceinline__ void fused_dots(const DotsArgs& dk, int64_t N, int64_t i0, int r,
                                           const float (&dj)[START_K + 1][NV],
                                           const float (&d0)[NV], bool valid) {
  constexpr int K = START_K;
  float acc[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) acc[j] = 0.f;
  if (valid) {
#pragma unroll
    for (int u = 0; u < NV; ++u) acc[0] += d0[u] * d0[u];
#pragma unroll
    for (int j = 1; j <= K; ++j)
#pragma unroll
      for (int u = 0; u < NV; ++u) acc[j] += d0[u] * dj[j][u];
    float* rw = dk.ring_d + (int64_t)(r % K) * N + i0;
    if (NV == 4) {
      *reinterpret_cast<float4*>(rw) = make_float4(d0[0], d0[NV > 1 ? 1 : 0], d0[NV > 2 ? 2 : 0],
                                                   d0[NV > 3 ? 3 : 0]);
    } else {
#pragma unroll
      for (int u = 0; u < NV; ++u) rw[u] = d0[u];
    }
  }
  __shared__ float red[8][K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    float t = acc[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][j] = t;
  }
  __syncthreads();
  if (threadIdx.x <= K) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
    dk.part[(int64_t)blockIdx.x * (K + 1) + threadIdx.x] = t;
  }
}

// NC charged species, species indices cs, valences val, reference densities
// nref (the neutral species are not read).  DOTS: the start's first pass in
// the same kernel (the source buffer holds s(t-1) until this pass writes
// s(t)).
template <int NC, bool WALLS, int ST, bool DOTS>
__global__ void __launch_bounds__(256) k_charge(
    const void* fin_v, const uint32_t* links, const int64_t* wsrc, int64_t* src,
    long long* part, const int* label, unsigned long long* comp_sum, int nx, int ny,
    int nz, int64_t N, int4 cs, float4 val, float4 nref, float fourpi_lb, long long src_ref,
    DotsArgs dk) {
  using T = typename Fmt<ST>::T;
  const T* fin = static_cast<const T*>(fin_v);
  const int sp[4] = {cs.x, cs.y, cs.z, cs.w};
  const float vz[4] = {val.x, val.y, val.z, val.w};
  const float nr[4] = {nref.x, nref.y, nref.z, nref.w};
  long long acc = 0;
  float d0[1] = {0.f};
  float dj[START_K + 1][1];
  const int r = DOTS ? dk.state[START_RING_IDX] : 0;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (uint32_t)N) {
    uint32_t lk = 0;
    bool fluid = true;
    if (WALLS) {
      lk = links[i];
      fluid = !(lk & LINK_SOLID);
    }
    long long sv = 0;
    long long old = 0;
    if (DOTS) {
      old = src[i];
      dots_load<1>(dk, N, i, r, dj);
    }
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
    if (DOTS) d0[0] = i64_to_f32(sv - old);
    // the largest fluid component (label 0) is summed per CTA; the cells of
    // other components (rare: pockets closed off by walls) add to their own
    // sum (two's-complement wrap-around keeps the 64-bit sum exact)
    if (label && fluid && label[i] != 0)
      atomicAdd(comp_sum + label[i], (unsigned long long)sv);
    else
      acc = sv;
  }
  block_partial(acc, part);
  if (DOTS) fused_dots<1>(dk, N, i, r, dj, d0, i < (uint32_t)N);
}

// Four consecutive stored values of one direction plane starting at an
// element index that is a multiple of four, as floats (one 16-byte load in
// FP32, one 8-byte load in the 16-bit formats).
template <int ST>
__device__ __forceinline__ void ld4h(const typename Fmt<ST>::T* p, float (&v)[4]) {
  if (ST == LBM_FP32) {
    const float4 w = *reinterpret_cast<const float4*>(p);
    v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
  } else {
    const uint2 w = *reinterpret_cast<const uint2*>(p);
    const uint32_t lo = w.x, hi = w.y;
    if (ST == LBM_FP16_SHIFT) {
      const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&lo));
      const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&hi));
      v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
      v[0] = __uint_as_float(lo << 16);
      v[1] = __uint_as_float(lo & 0xFFFF0000u);
      v[2] = __uint_as_float(hi << 16);
      v[3] = __uint_as_float(hi & 0xFFFF0000u);
    }
  }
}

// The charge density of k_charge for lattices without walls and nx a
// multiple of four, four consecutive nodes of one x row per thread: the
// four upstream values of a direction are one aligned vector load when the
// direction has no x component, two when it has (the row's wrap included).
// The same sums in the same order as k_charge, so the source is the same.
template <int NC, int ST, bool DOTS>
__global__ void __launch_bounds__(256) k_charge_quad(
    const void* fin_v, int64_t* src, long long* part, int nx, int ny, int nz, int64_t N, int4 cs,
    float4 val, float4 nref, float fourpi_lb, long long src_ref, DotsArgs dk) {
  using T = typename Fmt<ST>::T;
  const T* fin = static_cast<const T*>(fin_v);
  const int sp[4] = {cs.x, cs.y, cs.z, cs.w};
  const float vz[4] = {val.x, val.y, val.z, val.w};
  const float nr[4] = {nref.x, nref.y, nref.z, nref.w};
  long long acc = 0;
  float d0[4] = {0.f, 0.f, 0.f, 0.f};
  float dj[START_K + 1][4];
  longlong2 o0 = make_longlong2(0, 0), o1 = make_longlong2(0, 0);
  const int r = DOTS ? dk.state[START_RING_IDX] : 0;
  const uint32_t qd = blockIdx.x * blockDim.x + threadIdx.x;
  if (qd < (uint32_t)(N >> 2)) {
    const uint32_t i0 = 4u * qd;
    if (DOTS) {
      // s(t-1) and the stored differences, in flight with the pulls
      const longlong2* so = reinterpret_cast<const longlong2*>(src + i0);
      o0 = so[0];
      o1 = so[1];
      dots_load<4>(dk, N, i0, r, dj);
    }
    int x0, y, z;
    site_xyz(i0, nx, ny, x0, y, z);
    const Nbr o = neighbours(x0, y, z, nx, ny, nz);
    const int prevq = (x0 == 0) ? nx - 4 : -4;      // the quad before (x0 - 4 .. x0 - 1)
    const int nextq = (x0 + 4 == nx) ? -(nx - 4) : 4;  // the quad after
    float drho[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float m0[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int p = 0; p < Q; ++p) {
        const int dyz = (CY(p) == 1 ? o.dym : (CY(p) == -1 ? o.dyp : 0)) +
                        (CZ(p) == 1 ? o.dzm : (CZ(p) == -1 ? o.dzp : 0));
        const T* b = fin + (int64_t)(sp[c] * Q + p) * N + ((int)i0 + dyz);
        float v[4];
        if (CX(p) == 0) {
          ld4h<ST>(b, v);
        } else if (CX(p) == 1) {  // pulled from x - 1: x0 - 1 .. x0 + 2
          float a[4], h[4];
          ld4h<ST>(b + prevq, a);
          ld4h<ST>(b, h);
          v[0] = a[3]; v[1] = h[0]; v[2] = h[1]; v[3] = h[2];
        } else {  // pulled from x + 1: x0 + 1 .. x0 + 4
          float h[4], a[4];
          ld4h<ST>(b, h);
          ld4h<ST>(b + nextq, a);
          v[0] = h[1]; v[1] = h[2]; v[2] = h[3]; v[3] = a[0];
        }
        const float wn = WT(p) * nr[c];
#pragma unroll
        for (int j = 0; j < 4; ++j) m0[j] += wn * v[j];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) drho[j] += vz[c] * m0[j];
    }
    long long sv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      sv[j] = src_ref + (long long)(fourpi_lb * drho[j] * PSI_SCALE_F);
      acc += sv[j];
    }
    longlong2* d = reinterpret_cast<longlong2*>(src + i0);
    if (DOTS) {
      d0[0] = i64_to_f32(sv[0] - o0.x);
      d0[1] = i64_to_f32(sv[1] - o0.y);
      d0[2] = i64_to_f32(sv[2] - o1.x);
      d0[3] = i64_to_f32(sv[3] - o1.y);
    }
    d[0] = make_longlong2(sv[0], sv[1]);
    d[1] = make_longlong2(sv[2], sv[3]);
  }
  block_partial(acc, part);
  if (DOTS) fused_dots<4>(dk, N, 4 * (int64_t)qd, r, dj, d0, qd < (uint32_t)(N >> 2));
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

// Takes the Poisson source that the previous step's stream/collide
// scattered (the charge scatter): src = acc, acc = 0 for the next
// scatter; node pairs (16-byte loads and stores; N is even: nx is a
// multiple of 32) over a grid of a few CTAs per SM, four pairs in flight
// per thread.  The total of the source is summed exactly as a 128-bit
// integer: each CTA adds its sum to tot[0] (low word; the carry is known
// from the old value) and tot[1] (high word), then counts itself in tot[2];
// the last CTA converts the total to FP64 into *out, writes the source mean
// over the fluid to mean_z[0 .. nz) (when given), advances the graph step
// counter (when given) and clears tot for the next launch.  Integer sums do
// not depend on the order in which CTAs add, so the result is the same in
// every run (the work of k_sum_partials, without a second launch; few CTAs,
// so few same-address atomics).
__global__ void __launch_bounds__(256) k_src_take(int64_t* __restrict__ acc,
                                                  int64_t* __restrict__ src, int64_t N,
                                                  unsigned long long* tot, double* out,
                                                  long long* mean_z, int nz, double inv_nfluid,
                                                  uint32_t* step) {
  const int64_t np = N / 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  longlong2* a2 = reinterpret_cast<longlong2*>(acc);
  longlong2* s2 = reinterpret_cast<longlong2*>(src);
  long long v = 0;
  for (int64_t k0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k0 < np; k0 += 4 * stride) {
    longlong2 q[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = k0 + u * stride;
      q[u] = k < np ? a2[k] : make_longlong2(0, 0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = k0 + u * stride;
      if (k < np) {
        s2[k] = q[u];
        a2[k] = make_longlong2(0, 0);
        v += q[u].x + q[u].y;
      }
    }
  }
  __shared__ long long red[32];
  __shared__ int last;
  __shared__ long long s_mean;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long c = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) c += red[w];
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
  }
  if (mean_z) {
    __syncthreads();
    for (int z = threadIdx.x; z < nz; z += blockDim.x) mean_z[z] = s_mean;
  }
}

// Gathers f(t) of species s and its moments n, u = sum c f / n (doubles,
// from the deviations: n = n_ref + sum d, j = sum c d).  The deviation sums
// are compensated FP32 sums (about twice FP32 precision), 1/n an FP32
// reciprocal refined by one Newton step r (2 - n r) in FP64: FP64-grade
// moments with a handful of FP64 operations per node (FP64 arithmetic is
// slow on this GPU).
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
  float m0h = 0.f, m0l = 0.f, mxh = 0.f, mxl = 0.f, myh = 0.f, myl = 0.f, mzh = 0.f, mzl = 0.f;
#pragma unroll
  for (int p = 0; p < Q; ++p) {
    const float v = pull<ST, WALLS>(fin, N, s, p, i, upstream(o, p), lk, nref);
    if (f_out) f_out[(int64_t)p * N + i] = (double)WT(p) * nref + (double)v;
    two_sum_add(m0h, m0l, v);
    if (CX(p)) two_sum_add(mxh, mxl, CX(p) * v);
    if (CY(p)) two_sum_add(myh, myl, CY(p) * v);
    if (CZ(p)) two_sum_add(mzh, mzl, CZ(p) * v);
  }
  const double n = (double)nref + ((double)m0h + (double)m0l);
  if (n_out) n_out[i] = n;
  if (u_out) {
    double r = (double)__frcp_rn((float)n);
    r = r * fma(-n, r, 2.0);
    u_out[i] = ((double)mxh + (double)mxl) * r;
    u_out[N + i] = ((double)myh + (double)myl) * r;
    u_out[2 * N + i] = ((double)mzh + (double)mzl) * r;
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
    float px[S], pxv[S][3];
#pragma unroll
    for (int b = 0; b < S; ++b) {
      px[b] = n[b] * inv_ntot;
      const float hz = 0.5f * a.valence[b] * n[b];
      pxv[b][0] = (jx[b] + hz * Ex) * inv_ntot;
      pxv[b][1] = (jy[b] + hz * Ey) * inv_ntot;
      pxv[b][2] = (jz[b] + hz * Ez) * inv_ntot;
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const float inv_n = 1.0f / n[s];
      float Fx, Fy, Fz;
      if (S >= 3 && a.pair_on)
        species_force_pair<S>(s, jx[s] * inv_n, jy[s] * inv_n, jz[s] * inv_n, a.valence[s], Ex, Ey,
                              Ez, px, pxv, a, Fx, Fy, Fz);
      else
        species_force(jx[s] * inv_n, jy[s] * inv_n, jz[s] * inv_n, a.valence[s], Ex, Ey, Ez, vbx,
                      vby, vbz, omd, Fx, Fy, Fz);
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

// Sums the per-CTA diagnostics partials of the stream/collide kernel in
// FP64, in a fixed order (the result does not depend on scheduling):
// DIAG_REDUCE_G CTAs per quantity each sum a contiguous share of the
// partials into mid, and the CTA that finishes last (counted in *done,
// which it resets) adds the DIAG_REDUCE_G values of each quantity in order.
// out may be mapped pinned host memory (a per-step record).  With iters /
// rel given (device), the last CTA also copies them to out[DIAG_NQ],
// out[DIAG_NQ + 1].
constexpr int DIAG_REDUCE_G = 8;
__global__ void __launch_bounds__(256) k_diag_reduce(const double* __restrict__ part,
                                                     int64_t nctas, double* __restrict__ mid,
                                                     unsigned* done, double* __restrict__ out,
                                                     const int* __restrict__ iters,
                                                     const double* __restrict__ rel) {
  const int k = blockIdx.x / DIAG_REDUCE_G, g = blockIdx.x % DIAG_REDUCE_G;
  const int64_t chunk = (nctas + DIAG_REDUCE_G - 1) / DIAG_REDUCE_G;
  const int64_t c0 = g * chunk, c1 = min(nctas, c0 + chunk);
  double v = 0.0;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) v += part[c * DIAG_NQ + k];
  __shared__ double red[8];
  __shared__ int last;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    mid[blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < DIAG_NQ) {
    double t = 0.0;
    for (int q = 0; q < DIAG_REDUCE_G; ++q)
      t += __ldcg(mid + threadIdx.x * DIAG_REDUCE_G + q);  // other CTAs' sums, from the L2
    out[threadIdx.x] = t;
  }
  if (threadIdx.x == 0) {
    if (iters) {
      out[DIAG_NQ] = (double)*iters;
      out[DIAG_NQ + 1] = *rel;
    }
    *done = 0u;
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
  a.skip = h->collide_skip;
  a.pair_on = h->pair_on ? 1 : 0;
  for (int i = 0; i < MAX_SPECIES; ++i)
    for (int j = 0; j < MAX_SPECIES; ++j) a.pair[i][j] = h->pair[i][j];
  a.scat_acc = nullptr;
  a.src_ref = 0;
  for (int s = 0; s < MAX_SPECIES; ++s) a.scat_k[s] = 0.f;
  return a;
}

// 4 pi l_B sum_a z_a n_ref_a in fixed point (FP64 on the host): the part
// of the Poisson source that is the same at every fluid node
long long source_reference(const lbm_t* h) {
  double zref = 0.0;
  for (int s = 0; s < h->S; ++s) zref += (double)h->valence[s] * (double)h->nref[s];
  return llrint(4.0 * 3.14159265358979323846 * h->cfg.bjerrum * zref * PSI_SCALE);
}

cudaError_t collide_into_spare(lbm_t* h, int threads, bool d, bool scatter) {
  StepArgs a = step_args(h);
  const bool c = h->cfg.bjerrum > 0.0;
  const bool w = h->has_walls;
  if (scatter) {
    // the next step's source, accumulated into scat_acc (zero here: the
    // step took the previous one out)
    a.scat_acc = h->scat_acc;
    a.src_ref = source_reference(h);
    for (int s = 0; s < h->S; ++s)
      a.scat_k[s] = (float)(4.0 * 3.14159265358979323846 * h->cfg.bjerrum * (double)h->valence[s] *
                            (double)h->nref[s] * PSI_SCALE);
  }
  if (d) h->dpart_ctas = (int64_t)nblocks(h->N, threads);
  switch (h->cfg.storage) {
    case LBM_FP32: return collide_dispatch<LBM_FP32>(a, h->S, w, c, h->st, threads, d);
    case LBM_FP16_SHIFT: return collide_dispatch<LBM_FP16_SHIFT>(a, h->S, w, c, h->st, threads, d);
    case LBM_BF16_SHIFT: return collide_dispatch<LBM_BF16_SHIFT>(a, h->S, w, c, h->st, threads, d);
  }
  return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_stream_collide(lbm_t* h, bool diag) {
  cudaError_t e = collide_into_spare(h, h->collide_threads, diag, h->scat_on);
  if (e == cudaSuccess) {
    h->cur ^= 1;
    ++h->launches;
    h->diag_valid = diag;
    if (h->scat_on) h->scat_valid = true;
  }
  return e;
}

cudaError_t launch_stream_collide_probe(lbm_t* h, int threads) {
  cudaError_t e = collide_into_spare(h, threads, false, false);
  if (e == cudaSuccess) ++h->launches;
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

cudaError_t launch_diag_reduce(lbm_t* h, double* out, const int* iters, const double* rel) {
  k_diag_reduce<<<DIAG_NQ * DIAG_REDUCE_G, 256, 0, h->st>>>(h->dpart, h->dpart_ctas, h->dmid,
                                                            h->ddone, out, iters, rel);
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
  h->scat_valid = false;  // new populations: the next step runs the charge pass
  const int nb = nblocks(h->N, 256);
  LBM_DISPATCH_WS(h, (k_init<W_, ST_><<<nb, 256, 0, h->st>>>(
                         s, n0, u0, h->links, h->f[h->cur], h->cfg.nx,
                         h->cfg.ny, h->cfg.nz, h->N, h->nref[s])));
  ++h->launches;
  return cudaGetLastError();
}

namespace {
// The charge pass: the source of the current populations into out (the
// Poisson source, or the scatter's accumulator), per-CTA partial sums into
// ps.part; returns the number of partials.
int charge_pass(lbm_t* h, int64_t* out) {
  // one node per thread (the pulled loads of a node are independent and all
  // in flight); per-CTA partial sums instead of same-address atomics
  const int ct = h->charge_threads;
  const int nb = (int)nblocks(h->N, ct);
  const float k = (float)(4.0 * 3.14159265358979323846 * h->cfg.bjerrum);
  // reference part of the source, 4 pi l_B sum_alpha z^alpha n_ref^alpha,
  // in fixed point (FP64 on the host, the same at every fluid node)
  const long long src_ref = source_reference(h);
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
  // the start's first pass rides along when the pass writes the Poisson
  // source (not the scatter's accumulator) of a lattice without walls
  DotsArgs dk{};
#define LBM_CHARGE_S(NC)                                                                    \
  LBM_DISPATCH_WS(h, (dots ? k_charge<NC, W_, ST_, true><<<nb, ct, 0, h->st>>>(             \
                                 h->f[h->cur], h->links, h->wsrc, out, h->ps.part,           \
                                 h->ps.label, h->ps.comp_sum, h->cfg.nx, h->cfg.ny,          \
                                 h->cfg.nz, h->N, cs4, cv4, cr4, k, src_ref, dk)             \
                           : k_charge<NC, W_, ST_, false><<<nb, ct, 0, h->st>>>(            \
                                 h->f[h->cur], h->links, h->wsrc, out, h->ps.part,           \
                                 h->ps.label, h->ps.comp_sum, h->cfg.nx, h->cfg.ny,          \
                                 h->cfg.nz, h->N, cs4, cv4, cr4, k, src_ref, dk)))
  // 16-bit storage without walls: four nodes per thread (the two-byte
  // loads of one node per thread made the pass request-bound; in FP32 the
  // one-node pass is faster, 53 against 61 us at 128^3)
  const bool quad = !h->has_walls && h->cfg.storage != LBM_FP32 && h->cfg.nx % 4 == 0;
  int nbq = nb;
  if (quad) nbq = (int)nblocks(h->N / 4, ct);
  // (not with walls: there the pass's registers grow from 62 to 80 and it
  // lost more than the separate pass cost, 0.18 against 0.12 ms per step on
  // the porous 256^3 box)
  const bool dots = out == h->ps.src && !h->has_walls && charge_dots_args(h, nbq, &dk);
  if (quad) {
#define LBM_CHARGE_Q1(NC, ST, D)                                                            \
  k_charge_quad<NC, ST, D><<<nbq, ct, 0, h->st>>>(h->f[h->cur], out, h->ps.part, h->cfg.nx, \
                                                  h->cfg.ny, h->cfg.nz, h->N, cs4, cv4, cr4,  \
                                                  k, src_ref, dk)
#define LBM_CHARGE_Q(NC)                                                                   \
  do {                                                                                     \
    if (h->cfg.storage == LBM_FP16_SHIFT) {                                                \
      if (dots) LBM_CHARGE_Q1(NC, LBM_FP16_SHIFT, true);                                   \
      else LBM_CHARGE_Q1(NC, LBM_FP16_SHIFT, false);                                       \
    } else {                                                                               \
      if (dots) LBM_CHARGE_Q1(NC, LBM_BF16_SHIFT, true);                                   \
      else LBM_CHARGE_Q1(NC, LBM_BF16_SHIFT, false);                                       \
    }                                                                                      \
  } while (0)
    switch (nc) {
      case 0: LBM_CHARGE_Q(0); break;
      case 1: LBM_CHARGE_Q(1); break;
      case 2: LBM_CHARGE_Q(2); break;
      case 3: LBM_CHARGE_Q(3); break;
      default: LBM_CHARGE_Q(4); break;
    }
#undef LBM_CHARGE_Q
#undef LBM_CHARGE_Q1
  } else {
    switch (nc) {
      case 0: LBM_CHARGE_S(0); break;
      case 1: LBM_CHARGE_S(1); break;
      case 2: LBM_CHARGE_S(2); break;
      case 3: LBM_CHARGE_S(3); break;
      default: LBM_CHARGE_S(4); break;
    }
  }
#undef LBM_CHARGE_S
  ++h->launches;
  return nbq;
}
}  // namespace

cudaError_t charge_prepare(lbm_t* h) {
  if (h->scat_on && !h->scat_valid) {
    charge_pass(h, h->scat_acc);
    h->scat_valid = true;
  }
  return cudaGetLastError();
}

cudaError_t launch_charge(lbm_t* h) {
  int nbq;
  if (h->scat_on) {
    // the source the previous stream/collide scattered (computed by the
    // pass into the accumulator when the populations came from elsewhere),
    // moved into the Poisson source; the accumulator is then zero for the
    // scatter of this step
    if (!h->scat_valid) charge_pass(h, h->scat_acc);
    const int tb = 256;
    const unsigned nbt = (unsigned)std::min<int64_t>(nblocks(h->N / 2, tb), h->grid_cap / 2);
    // with the start from the history on, the take also forms the fit's
    // source difference and its inner products (one pass over the source)
    if (!launch_take_dots(h, nbt, 1.0 / (double)h->nfluid))
      k_src_take<<<nbt, tb, 0, h->st>>>(
        h->scat_acc, h->ps.src, h->N, h->scat_tot, h->ps.dsum, h->charge_mean_z, h->cfg.nz,
        1.0 / (double)h->nfluid, h->charge_step);
    ++h->launches;
    h->scat_valid = false;
  } else {
    nbq = charge_pass(h, h->ps.src);
    k_sum_partials<<<1, 1024, 0, h->st>>>(h->ps.part, nbq, h->ps.dsum, h->charge_mean_z,
                                          h->cfg.nz, 1.0 / (double)h->nfluid, h->charge_step);
    ++h->launches;
  }
  // the spectral solver's source mean for one periodic run is written
  // there; the solve then skips its own mean kernel once
  // (charge_means_ready)
  h->charge_means_ready = h->charge_mean_z != nullptr;
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
