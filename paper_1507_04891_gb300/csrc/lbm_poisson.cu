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

// Fine box of the multigrid: the lattice planes [zlo, zlo + nzb).  Its FP32
// correction e and residual r are stored colour-split: cell (x, y, z) of
// colour q = (x + y + z) mod 2 sits at q H + (z ny + y) hx + floor(x / 2),
// hx = ceil(nx / 2), H = nzb ny hx.  A red-black half-sweep then reads the
// other colour's array and whole sectors of its own instead of every line of
// both colours interleaved.  The one-byte face mask uses the same layout.
struct Box {
  int nx, ny, nzb, zlo, perz;
  int hx;        // cells of one colour per x row (with one pad cell if nx is odd)
  uint32_t H;    // cells of one colour array
  int64_t nxy;   // lattice plane
};

// Face mask of a fine-box cell: bit f set when face f (0 +x, 1 -x, 2 +y,
// 3 -y, 4 +z, 5 -z) joins two fluid cells; FACE_SOLID for a wall cell.
constexpr uint32_t FACE_SOLID = 0x80u;
constexpr uint32_t FACES_OPEN = 0x3fu;

// open-face bits from the link word: bit 2 of the link word = +x neighbour
// is a wall node, 1 = -x, 4 = +y, 3 = -y, 6 = +z, 5 = -z.
__device__ __forceinline__ bool open_face(uint32_t lk, int face) {
  const int bit = (face & 1) ? face : face + 2;  // 0->2, 1->1, 2->4, 3->3, 4->6, 5->5
  return !((lk >> bit) & 1u);
}

// box-cell neighbour offsets in natural order (periodic x, y; z periodic
// only if perz, else the cell itself at the ends, where the face is closed)
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

// colour-split index of box cell (x, y, z)
__device__ __forceinline__ uint32_t sp_idx(const Box& b, int x, int y, int z) {
  return (((x + y + z) & 1) ? b.H : 0u) + ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.hx +
         (uint32_t)(x >> 1);
}

// colour-split indices of the six face neighbours (order of the mask bits)
__device__ __forceinline__ void sp_nbrs(const Box& b, int x, int y, int z, uint32_t (&j)[6]) {
  const int xp = (x == b.nx - 1) ? 0 : x + 1, xm = (x == 0) ? b.nx - 1 : x - 1;
  const int yp = (y == b.ny - 1) ? 0 : y + 1, ym = (y == 0) ? b.ny - 1 : y - 1;
  int zp, zm;
  if (b.perz) {
    zp = (z == b.nzb - 1) ? 0 : z + 1;
    zm = (z == 0) ? b.nzb - 1 : z - 1;
  } else {
    zp = (z == b.nzb - 1) ? z : z + 1;
    zm = (z == 0) ? z : z - 1;
  }
  j[0] = sp_idx(b, xp, y, z);
  j[1] = sp_idx(b, xm, y, z);
  j[2] = sp_idx(b, x, yp, z);
  j[3] = sp_idx(b, x, ym, z);
  j[4] = sp_idx(b, x, y, zp);
  j[5] = sp_idx(b, x, y, zm);
}

__device__ __forceinline__ int64_t fx_of(float e) {
  return f32_to_i64_rn(e * PSI_SCALE_F);
}

// Face mask of the fine box from the lattice link words.
__global__ void __launch_bounds__(256) k_face_mask(const uint32_t* __restrict__ links, Box b,
                                                   uint32_t nbox, uint8_t* __restrict__ mask) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nbox) return;
  int x, y, z;
  box_xyz(c, b, x, y, z);
  const uint32_t lk = links[(int64_t)c + (int64_t)b.zlo * b.nxy];
  uint32_t m = 0;
  if (lk & LINK_SOLID) {
    m = FACE_SOLID;
  } else {
#pragma unroll
    for (int f = 0; f < 6; ++f)
      if (open_face(lk, f)) m |= 1u << f;
  }
  mask[sp_idx(b, x, y, z)] = (uint8_t)m;
}

// Norm partials of the fine residual: CTA k adds its sums into slot
// k mod MG_NACC (FP32 atomics spread over addresses; FP64 atomics are slow
// on this GPU).  Values are scaled by 2^-20 before squaring so that sums of
// squared fixed-point values stay inside the FP32 range; the reader adds the
// slots in FP64 and scales by 2^40.  The norms only decide convergence, so
// FP32 partials are ample.
constexpr int MG_NACC = 64;
constexpr float MG_NORM_PRE = 1.0f / 1048576.0f;  // 2^-20

// Residual on the fine box, r = s - <s> - A psi, exact in 64-bit integers;
// one cell per thread.  Writes r (FP32, colour-split) and adds |r|^2 and,
// with SNORM (the first residual of a solve: the source does not change
// during one), |s - <s>|^2 (fixed-point units, scaled) to the norm slots.
template <bool WALLS, bool SNORM>
__global__ void __launch_bounds__(256) k_res0(
    const int64_t* __restrict__ psi, const int64_t* __restrict__ src,
    const uint8_t* __restrict__ mask, float* __restrict__ r, const double* __restrict__ dsum,
    float* __restrict__ acc, Box b, uint32_t nbox, double inv_nfluid,
    const int* __restrict__ label, const long long* __restrict__ comp_mean) {
  __shared__ long long s_mean;
  __shared__ float red_r[8], red_s[8];
  if (threadIdx.x == 0) s_mean = llrint(dsum[0] * inv_nfluid);
  __syncthreads();
  float rr = 0.f, ss = 0.f;
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nbox) {
    int x, y, z;
    box_xyz(c, b, x, y, z);
    const uint32_t q = sp_idx(b, x, y, z);
    const uint32_t m = WALLS ? (uint32_t)mask[q] : FACES_OPEN;
    if (m & FACE_SOLID) {
      r[q] = 0.f;
    } else {
      const int64_t i = (int64_t)c + (int64_t)b.zlo * b.nxy;  // lattice node
      int d[6];
      box_nbr(b, x, y, z, d);
      const int64_t pc = psi[i];
      int64_t Ap = 0;
#pragma unroll
      for (int f = 0; f < 6; ++f)
        if ((m >> f) & 1u) Ap += pc - psi[i + d[f]];
      const int64_t sfx = src[i] - (label ? comp_mean[label[i]] : (int64_t)s_mean);
      const float rf = i64_to_f32(sfx - Ap);
      r[q] = rf * PSI_INV_SCALE_F;
      const float rs = rf * MG_NORM_PRE;
      rr = rs * rs;
      if (SNORM) {
        const float sf = i64_to_f32(sfx) * MG_NORM_PRE;
        ss = sf * sf;
      }
    }
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
    float tr = 0.f, ts = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tr += red_r[w];
      ts += red_s[w];
    }
    const int k = blockIdx.x & (MG_NACC - 1);
    atomicAdd(acc + k, tr);
    if (SNORM) atomicAdd(acc + MG_NACC + k, ts);
  }
}

// Red-black Gauss-Seidel half-sweep on the fine box for A e = r (FP32), one
// cell of colour `color` per thread (colour index t).  MODE 1, the first
// half-sweep of a cycle: starts from e = 0, so no neighbour is read and the
// thread clears the other colour's cell at the same index.  MODE 2, the last
// half-sweep of a cycle: also writes the corrected potential
// psi_out = psi_in + round(e) for the x pair (2k, 2k + 1) its cell shares
// with the other colour's cell t, whose sweep has finished; wall cells keep
// psi_in.
template <bool WALLS, int MODE>
__global__ void __launch_bounds__(256) k_smooth0(
    float* __restrict__ e, const float* __restrict__ r, const uint8_t* __restrict__ mask,
    Box b, int color, const int64_t* __restrict__ psi_in, int64_t* __restrict__ psi_out) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= b.H) return;
  const uint32_t row = t / (uint32_t)b.hx;
  const uint32_t k = t - row * (uint32_t)b.hx;
  const int z = (int)(row / (uint32_t)b.ny);
  const int y = (int)(row - (uint32_t)z * (uint32_t)b.ny);
  const int x = 2 * (int)k + ((y + z + color) & 1);
  const uint32_t self = (color ? b.H : 0u) + t;
  const uint32_t other = (color ? 0u : b.H) + t;
  if (MODE == 1) e[other] = 0.f;
  float ev = 0.f;
  if (x < b.nx) {
    const uint32_t m = WALLS ? (uint32_t)mask[self] : FACES_OPEN;
    if (!(m & FACE_SOLID)) {
      float sum = r[self];
      if (MODE != 1) {
        uint32_t j[6];
        sp_nbrs(b, x, y, z, j);
#pragma unroll
        for (int f = 0; f < 6; ++f)
          if ((m >> f) & 1u) sum += e[j[f]];
      }
      const int cnt = __popc(m & FACES_OPEN);
      if (cnt > 0) {
        ev = __fdividef(sum, (float)cnt);
        e[self] = ev;
      } else if (MODE == 1) {
        e[self] = 0.f;
      } else {
        ev = e[self];
      }
    }
  }
  if (MODE == 2) {
    const int xo = x ^ 1;  // the other colour's cell of the pair
    float eo = 0.f;
    if (xo < b.nx) {
      const uint32_t mo = WALLS ? (uint32_t)mask[other] : FACES_OPEN;
      if (!(mo & FACE_SOLID)) eo = e[other];
    }
    const int x0 = 2 * (int)k;
    const float e0 = (x == x0) ? ev : eo, e1 = (x == x0) ? eo : ev;
    const int64_t base = ((int64_t)(z + b.zlo) * b.ny + y) * b.nx + x0;
    if ((b.nx & 1) == 0) {
      const longlong2 pin = *reinterpret_cast<const longlong2*>(psi_in + base);
      longlong2 po;
      po.x = pin.x + fx_of(e0);
      po.y = pin.y + fx_of(e1);
      *reinterpret_cast<longlong2*>(psi_out + base) = po;
    } else {
      if (x0 < b.nx) psi_out[base] = psi_in[base] + fx_of(e0);
      if (x0 + 1 < b.nx) psi_out[base + 1] = psi_in[base + 1] + fx_of(e1);
    }
  }
}

// Red-black cell of colour `color` handled by thread t on a coarse level in
// natural order: with an even x extent every x row holds nx/2 cells of each
// colour; with an odd one every thread takes one cell and skips the other
// colour.
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

// ---------------------------------------------------------------------------
// z-marching fine-box kernels.  Used when the red-black ordering is a true
// two-colouring (nx, ny even; nzb even or z not periodic): every face
// neighbour of a cell then has the other colour, and the other colour's
// entry at the same pair index k in a neighbouring row or plane is the
// cell's own y or z neighbour.  A thread owns the x pair (2k, 2k + 1) of row
// y and walks a run of zc planes, keeping the column below, here and above
// in registers; 2-D thread blocks over (k, y) need no integer division.
// ---------------------------------------------------------------------------

// Half-sweep of colour `color` (MODE as k_smooth0).  The planes are taken
// ZM_BATCH at a time: every load of a batch is issued before the first is
// used (the mask only selects among loaded values), so a thread keeps
// several DRAM requests in flight instead of waiting on the mask first.
constexpr int ZM_BATCH = 4;

template <bool WALLS, int MODE>
__global__ void __launch_bounds__(256) k_smooth0_zm(
    float* __restrict__ e, const float* __restrict__ r, const uint8_t* __restrict__ mask,
    Box b, int color, int zc, const int64_t* __restrict__ psi_in, int64_t* __restrict__ psi_out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (k >= b.hx || y >= b.ny) return;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, b.nzb);
  const uint32_t own = color ? b.H : 0u, oth = color ? 0u : b.H;
  float* __restrict__ eo = e + oth;
  float* __restrict__ ec = e + own;
  const float* __restrict__ rc = r + own;
  const uint32_t plane = (uint32_t)b.ny * (uint32_t)b.hx;
  const int yp = (y == b.ny - 1) ? 0 : y + 1, ym = (y == 0) ? b.ny - 1 : y - 1;
  const int kp = (k == b.hx - 1) ? 0 : k + 1, km = (k == 0) ? b.hx - 1 : k - 1;
  const uint32_t oc = (uint32_t)y * b.hx + k;
  const uint32_t oyp = (uint32_t)yp * b.hx + k, oym = (uint32_t)ym * b.hx + k;
  const uint32_t oxp = (uint32_t)y * b.hx + kp, oxm = (uint32_t)y * b.hx + km;
  // other colour of this pair column: plane below, here (rolling)
  float ob = 0.f, oh = 0.f;
  if (MODE != 1) {
    const int zb = (z0 > 0) ? z0 - 1 : (b.perz ? b.nzb - 1 : 0);
    ob = eo[(uint32_t)zb * plane + oc];
    oh = eo[(uint32_t)z0 * plane + oc];
  }
  for (int zs = z0; zs < z1; zs += ZM_BATCH) {
    float OA[ZM_BATCH], RC[ZM_BATCH], EX[ZM_BATCH], EYP[ZM_BATCH], EYM[ZM_BATCH];
    uint32_t M[ZM_BATCH], MO[ZM_BATCH];
    longlong2 PIN[ZM_BATCH];
#pragma unroll
    for (int u = 0; u < ZM_BATCH; ++u) {
      const int z = min(zs + u, z1 - 1);  // past the run: a repeat, unused
      const uint32_t pz = (uint32_t)z * plane;
      RC[u] = rc[pz + oc];
      M[u] = WALLS ? (uint32_t)mask[own + pz + oc] : FACES_OPEN;
      if (MODE != 1) {
        const int za = (z < b.nzb - 1) ? z + 1 : (b.perz ? 0 : z);
        OA[u] = eo[(uint32_t)za * plane + oc];
        const int p = (y + z + color) & 1;
        EX[u] = eo[pz + (p ? oxp : oxm)];
        EYP[u] = eo[pz + oyp];
        EYM[u] = eo[pz + oym];
      }
      if (MODE == 2) {
        MO[u] = WALLS ? (uint32_t)mask[oth + pz + oc] : FACES_OPEN;
        PIN[u] = *reinterpret_cast<const longlong2*>(
            psi_in + ((int64_t)(z + b.zlo) * b.ny + y) * b.nx + 2 * k);
      }
    }
#pragma unroll
    for (int u = 0; u < ZM_BATCH; ++u) {
      const int z = zs + u;
      if (z >= z1) break;
      const uint32_t pz = (uint32_t)z * plane;
      if (MODE == 1) eo[pz + oc] = 0.f;
      const int p = (y + z + color) & 1;  // own cell at x = 2k + p
      const uint32_t m = M[u];
      float ev = 0.f;
      if (!(m & FACE_SOLID)) {
        float sum = RC[u];
        if (MODE != 1) {
          // the x neighbour outside the pair: 2k + 2 (pair k + 1) when the
          // own cell is 2k + 1, else 2k - 1 (pair k - 1)
          const float exp1 = p ? EX[u] : oh, exm1 = p ? oh : EX[u];
          if (m & 1u) sum += exp1;
          if (m & 2u) sum += exm1;
          if (m & 4u) sum += EYP[u];
          if (m & 8u) sum += EYM[u];
          if (m & 16u) sum += OA[u];
          if (m & 32u) sum += ob;
        }
        const int cnt = __popc(m & FACES_OPEN);
        if (cnt > 0) {
          ev = __fdividef(sum, (float)cnt);
          ec[pz + oc] = ev;
        } else if (MODE == 1) {
          ec[pz + oc] = 0.f;
        } else {
          ev = ec[pz + oc];
        }
      }
      if (MODE == 2) {
        // pair update: the other colour's cell (x ^ 1) has its final value oh
        const float eo_v = (MO[u] & FACE_SOLID) ? 0.f : oh;
        const float e0 = p ? eo_v : ev, e1 = p ? ev : eo_v;
        longlong2 po;
        po.x = PIN[u].x + fx_of(e0);
        po.y = PIN[u].y + fx_of(e1);
        *reinterpret_cast<longlong2*>(psi_out + ((int64_t)(z + b.zlo) * b.ny + y) * b.nx + 2 * k) = po;
      }
      if (MODE != 1) {
        ob = oh;
        oh = OA[u];
      }
    }
  }
}

// Half-sweep (MODE as k_smooth0) with two x pairs per thread: cells
// 4j .. 4j + 3 of row y (pairs 2j and 2j + 1), colour arrays read as float2.
// Needs nx a multiple of 4.  Batches of planes as k_smooth0_zm.  Wall cells
// get e = 0 written (their correction is never read, and stays 0).
template <bool WALLS, int MODE>
__global__ void __launch_bounds__(256) k_smooth0_zq(
    float* __restrict__ e, const float* __restrict__ r, const uint8_t* __restrict__ mask,
    Box b, int color, int zc, const int64_t* __restrict__ psi_in, int64_t* __restrict__ psi_out) {
  constexpr int NB = (MODE == 2) ? 2 : ZM_BATCH;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (j >= (b.hx >> 1) || y >= b.ny) return;
  const int k0 = 2 * j;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, b.nzb);
  const uint32_t own = color ? b.H : 0u, oth = color ? 0u : b.H;
  float* __restrict__ eo = e + oth;
  float* __restrict__ ec = e + own;
  const float* __restrict__ rc = r + own;
  const uint32_t plane = (uint32_t)b.ny * (uint32_t)b.hx;
  const int yp = (y == b.ny - 1) ? 0 : y + 1, ym = (y == 0) ? b.ny - 1 : y - 1;
  const int kl = (k0 == 0) ? b.hx - 1 : k0 - 1;       // pair left of the two
  const int kr = (k0 + 2 == b.hx) ? 0 : k0 + 2;        // pair right of the two
  const uint32_t oc = (uint32_t)y * b.hx + k0;
  const uint32_t oyp = (uint32_t)yp * b.hx + k0, oym = (uint32_t)ym * b.hx + k0;
  const uint32_t oxl = (uint32_t)y * b.hx + kl, oxr = (uint32_t)y * b.hx + kr;
  auto ld2 = [](const float* p) { return *reinterpret_cast<const float2*>(p); };
  float2 ob = make_float2(0.f, 0.f), oh = make_float2(0.f, 0.f);
  if (MODE != 1) {
    const int zb = (z0 > 0) ? z0 - 1 : (b.perz ? b.nzb - 1 : 0);
    ob = ld2(eo + (uint32_t)zb * plane + oc);
    oh = ld2(eo + (uint32_t)z0 * plane + oc);
  }
  for (int zs = z0; zs < z1; zs += NB) {
    float2 OA[NB], RC[NB], EYP[NB], EYM[NB];
    float EX[NB];
    uint32_t M[NB], MO[NB];
    longlong2 P0[NB], P1[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int z = min(zs + u, z1 - 1);  // past the run: a repeat, unused
      const uint32_t pz = (uint32_t)z * plane;
      RC[u] = ld2(rc + pz + oc);
      M[u] = WALLS ? (uint32_t)*reinterpret_cast<const uint16_t*>(mask + own + pz + oc)
                   : (FACES_OPEN | (FACES_OPEN << 8));
      if (MODE != 1) {
        const int za = (z < b.nzb - 1) ? z + 1 : (b.perz ? 0 : z);
        OA[u] = ld2(eo + (uint32_t)za * plane + oc);
        const int p = (y + z + color) & 1;
        EX[u] = eo[pz + (p ? oxr : oxl)];
        EYP[u] = ld2(eo + pz + oyp);
        EYM[u] = ld2(eo + pz + oym);
      }
      if (MODE == 2) {
        MO[u] = WALLS ? (uint32_t)*reinterpret_cast<const uint16_t*>(mask + oth + pz + oc)
                      : (FACES_OPEN | (FACES_OPEN << 8));
        const int64_t base = ((int64_t)(z + b.zlo) * b.ny + y) * b.nx + 4 * j;
        P0[u] = *reinterpret_cast<const longlong2*>(psi_in + base);
        P1[u] = *reinterpret_cast<const longlong2*>(psi_in + base + 2);
      }
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int z = zs + u;
      if (z >= z1) break;
      const uint32_t pz = (uint32_t)z * plane;
      const int p = (y + z + color) & 1;  // own cells at 4j + p and 4j + 2 + p
      if (MODE == 1) *reinterpret_cast<float2*>(eo + pz + oc) = make_float2(0.f, 0.f);
      float val[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t m = (M[u] >> (8 * h)) & 0xffu;
        float v = 0.f;
        if (!(m & FACE_SOLID)) {
          float sum = h ? RC[u].y : RC[u].x;
          if (MODE != 1) {
            // x neighbours: A (h = 0) at 4j + p, B (h = 1) at 4j + 2 + p;
            // the other colour's cells of the two pairs are oh.x, oh.y
            float xp, xm;
            if (h == 0) {
              xp = p ? oh.y : oh.x;
              xm = p ? oh.x : EX[u];
            } else {
              xp = p ? EX[u] : oh.y;
              xm = p ? oh.y : oh.x;
            }
            if (m & 1u) sum += xp;
            if (m & 2u) sum += xm;
            if (m & 4u) sum += h ? EYP[u].y : EYP[u].x;
            if (m & 8u) sum += h ? EYM[u].y : EYM[u].x;
            if (m & 16u) sum += h ? OA[u].y : OA[u].x;
            if (m & 32u) sum += h ? ob.y : ob.x;
          }
          const int cnt = __popc(m & FACES_OPEN);
          if (cnt > 0) v = __fdividef(sum, (float)cnt);
          else if (MODE != 1) v = ec[pz + oc + h];  // isolated cell: unchanged
        }
        val[h] = v;
      }
      *reinterpret_cast<float2*>(ec + pz + oc) = make_float2(val[0], val[1]);
      if (MODE == 2) {
        const float ox = (MO[u] & FACE_SOLID) ? 0.f : oh.x;
        const float oy = ((MO[u] >> 8) & FACE_SOLID) ? 0.f : oh.y;
        const float e0 = p ? ox : val[0], e1 = p ? val[0] : ox;
        const float e2 = p ? oy : val[1], e3 = p ? val[1] : oy;
        const int64_t base = ((int64_t)(z + b.zlo) * b.ny + y) * b.nx + 4 * j;
        longlong2 q0, q1;
        q0.x = P0[u].x + fx_of(e0);
        q0.y = P0[u].y + fx_of(e1);
        q1.x = P1[u].x + fx_of(e2);
        q1.y = P1[u].y + fx_of(e3);
        *reinterpret_cast<longlong2*>(psi_out + base) = q0;
        *reinterpret_cast<longlong2*>(psi_out + base + 2) = q1;
      }
      if (MODE != 1) {
        ob = oh;
        oh = OA[u];
      }
    }
  }
}

// Fine-box residual r = s - <s> - A psi (exact integers), pair per thread
// and plane, planes ZM_RES_BATCH at a time with every load of a batch issued
// first; norms as in k_res0.
constexpr int ZM_RES_BATCH = 2;

template <bool WALLS, bool SNORM>
__global__ void __launch_bounds__(256, 3) k_res0_zm(
    const int64_t* __restrict__ psi, const int64_t* __restrict__ src,
    const uint8_t* __restrict__ mask, float* __restrict__ r, const double* __restrict__ dsum,
    float* __restrict__ acc, Box b, int zc, double inv_nfluid, const int* __restrict__ label,
    const long long* __restrict__ comp_mean) {
  __shared__ long long s_mean;
  __shared__ float red_r[8], red_s[8];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid == 0) s_mean = llrint(dsum[0] * inv_nfluid);
  __syncthreads();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  float rr = 0.f, ss = 0.f;
  if (k < b.hx && y < b.ny) {
    const int z0 = blockIdx.z * zc;
    const int z1 = min(z0 + zc, b.nzb);
    const int x0 = 2 * k;
    const int yp = (y == b.ny - 1) ? 0 : y + 1, ym = (y == 0) ? b.ny - 1 : y - 1;
    const int64_t oc = (int64_t)y * b.nx + x0;
    const int64_t oyp = (int64_t)yp * b.nx + x0, oym = (int64_t)ym * b.nx + x0;
    const int64_t oxm = (int64_t)y * b.nx + (x0 == 0 ? b.nx - 1 : x0 - 1);
    const int64_t oxp = (int64_t)y * b.nx + (x0 + 2 == b.nx ? 0 : x0 + 2);
    const uint32_t plane = (uint32_t)b.ny * (uint32_t)b.hx;
    const uint32_t sc = (uint32_t)y * b.hx + k;
    const int zb0 = (z0 > 0) ? z0 - 1 : (b.perz ? b.nzb - 1 : 0);
    longlong2 pb = *reinterpret_cast<const longlong2*>(psi + (int64_t)(zb0 + b.zlo) * b.nxy + oc);
    longlong2 ph = *reinterpret_cast<const longlong2*>(psi + (int64_t)(z0 + b.zlo) * b.nxy + oc);
    const int64_t mean0 = label ? (int64_t)comp_mean[0] : 0;
    for (int zs = z0; zs < z1; zs += ZM_RES_BATCH) {
      longlong2 PA[ZM_RES_BATCH], PYP[ZM_RES_BATCH], PYM[ZM_RES_BATCH], SV[ZM_RES_BATCH];
      int64_t PXM[ZM_RES_BATCH], PXP[ZM_RES_BATCH];
      int2 LB[ZM_RES_BATCH];
      uint32_t M0[ZM_RES_BATCH], M1[ZM_RES_BATCH];
#pragma unroll
      for (int u = 0; u < ZM_RES_BATCH; ++u) {
        const int z = min(zs + u, z1 - 1);  // past the run: a repeat, unused
        const int za = (z < b.nzb - 1) ? z + 1 : (b.perz ? 0 : z);
        const int64_t pl = (int64_t)(z + b.zlo) * b.nxy;
        PA[u] = *reinterpret_cast<const longlong2*>(psi + (int64_t)(za + b.zlo) * b.nxy + oc);
        PYP[u] = *reinterpret_cast<const longlong2*>(psi + pl + oyp);
        PYM[u] = *reinterpret_cast<const longlong2*>(psi + pl + oym);
        PXM[u] = psi[pl + oxm];
        PXP[u] = psi[pl + oxp];
        SV[u] = *reinterpret_cast<const longlong2*>(src + pl + oc);
        if (label) LB[u] = *reinterpret_cast<const int2*>(label + pl + oc);
        const uint32_t q0 = ((y + z) & 1) ? b.H : 0u, q1 = b.H - q0;
        const uint32_t si = (uint32_t)z * plane + sc;
        M0[u] = WALLS ? (uint32_t)mask[q0 + si] : FACES_OPEN;
        M1[u] = WALLS ? (uint32_t)mask[q1 + si] : FACES_OPEN;
      }
#pragma unroll
      for (int u = 0; u < ZM_RES_BATCH; ++u) {
        const int z = zs + u;
        if (z >= z1) break;
        int64_t s0, s1;
        if (label) {
          // component 0 (the largest) from a register: the gather is only
          // issued for cells of the other components
          s0 = SV[u].x - (LB[u].x ? comp_mean[LB[u].x] : mean0);
          s1 = SV[u].y - (LB[u].y ? comp_mean[LB[u].y] : mean0);
        } else {
          s0 = SV[u].x - (int64_t)s_mean;
          s1 = SV[u].y - (int64_t)s_mean;
        }
        const uint32_t q0 = ((y + z) & 1) ? b.H : 0u, q1 = b.H - q0;  // colour arrays of x0, x0 + 1
        const uint32_t si = (uint32_t)z * plane + sc;
        const longlong2 pa = PA[u], pyp = PYP[u], pym = PYM[u];
        const uint32_t m0 = M0[u], m1 = M1[u];
        // cell x0: +x = x0 + 1, -x = x0 - 1; cell x0 + 1: +x = x0 + 2, -x = x0
        if (!(m0 & FACE_SOLID)) {
          int64_t Ap = 0;
          const int64_t c = ph.x;
          if (m0 & 1u) Ap += c - ph.y;
          if (m0 & 2u) Ap += c - PXM[u];
          if (m0 & 4u) Ap += c - pyp.x;
          if (m0 & 8u) Ap += c - pym.x;
          if (m0 & 16u) Ap += c - pa.x;
          if (m0 & 32u) Ap += c - pb.x;
          const float rf = i64_to_f32(s0 - Ap);
          r[q0 + si] = rf * PSI_INV_SCALE_F;
          const float rs = rf * MG_NORM_PRE;
          rr = fmaf(rs, rs, rr);
          if (SNORM) {
            const float sf = i64_to_f32(s0) * MG_NORM_PRE;
            ss = fmaf(sf, sf, ss);
          }
        } else {
          r[q0 + si] = 0.f;
        }
        if (!(m1 & FACE_SOLID)) {
          int64_t Ap = 0;
          const int64_t c = ph.y;
          if (m1 & 1u) Ap += c - PXP[u];
          if (m1 & 2u) Ap += c - ph.x;
          if (m1 & 4u) Ap += c - pyp.y;
          if (m1 & 8u) Ap += c - pym.y;
          if (m1 & 16u) Ap += c - pa.y;
          if (m1 & 32u) Ap += c - pb.y;
          const float rf = i64_to_f32(s1 - Ap);
          r[q1 + si] = rf * PSI_INV_SCALE_F;
          const float rs = rf * MG_NORM_PRE;
          rr = fmaf(rs, rs, rr);
          if (SNORM) {
            const float sf = i64_to_f32(s1) * MG_NORM_PRE;
            ss = fmaf(sf, sf, ss);
          }
        } else {
          r[q1 + si] = 0.f;
        }
        pb = ph;
        ph = pa;
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    rr += __shfl_down_sync(0xffffffffu, rr, off);
    ss += __shfl_down_sync(0xffffffffu, ss, off);
  }
  if ((tid & 31) == 0) {
    red_r[tid >> 5] = rr;
    red_s[tid >> 5] = ss;
  }
  __syncthreads();
  if (tid == 0) {
    float tr = 0.f, ts = 0.f;
    const int nw = (int)(blockDim.x * blockDim.y) >> 5;
    for (int w = 0; w < nw; ++w) {
      tr += red_r[w];
      ts += red_s[w];
    }
    const int kk = (blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)) & (MG_NACC - 1);
    atomicAdd(acc + kk, tr);
    if (SNORM) atomicAdd(acc + MG_NACC + kk, ts);
  }
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

// Restriction from the fine box: rhs_c(J) = sum over the children i of J of
// (r_i - (A e)_i).
template <bool WALLS>
__global__ void __launch_bounds__(256) k_restrict0(
    const float* __restrict__ e, const float* __restrict__ r,
    const uint8_t* __restrict__ mask, Box b, CL cl, int cxs, int cys,
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
        const uint32_t q = sp_idx(b, x, y, z);
        const uint32_t m = WALLS ? (uint32_t)mask[q] : FACES_OPEN;
        if (m & FACE_SOLID) continue;
        uint32_t j[6];
        sp_nbrs(b, x, y, z, j);
        const float ec = e[q];
        float Ae = 0.f;
#pragma unroll
        for (int f = 0; f < 6; ++f)
          if ((m >> f) & 1u) Ae += ec - e[j[f]];
        acc += r[q] - Ae;
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

// Coarse coordinates along one axis for the prolongation: [0] the neighbour
// below, [1] the parent, [2] the neighbour above; a neighbour outside a
// non-periodic boundary, or along an axis the coarse level does not halve,
// is the parent's coordinate.
__device__ __forceinline__ void prol_axis(int X, int n_c, int per, int coarsened, int (&c)[3]) {
  c[0] = c[1] = c[2] = X;
  if (!coarsened) return;
  if (X > 0) c[0] = X - 1;
  else if (per) c[0] = n_c - 1;
  if (X < n_c - 1) c[2] = X + 1;
  else if (per) c[2] = 0;
}

// Trilinear (cell-centred) prolongation of the coarse correction, added to
// the fine correction; one thread per coarse cell J writes its children.
// Along an axis the coarse level halves, child k of J takes 3/4 of J's
// coordinate and 1/4 of the neighbour on its side (k = 0 below, k = 1
// above); an inactive coarse cell contributes the parent's value instead.
// FINE0: the fine level is the fine box (colour-split, face mask);
// otherwise a level in natural order, Dinv_f = 0 marking inactive cells.
template <bool FINE0, bool WALLS>
__global__ void __launch_bounds__(256) k_prolong(
    float* __restrict__ ef, const float* __restrict__ Dinv_f,
    const uint8_t* __restrict__ mask, Box b, CL f, const float* __restrict__ xc,
    const float* __restrict__ Dinv_c, CL cl, int cxs, int cys, int czs) {
  const uint32_t J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= (uint32_t)cl.n) return;
  int X, Y, Z;
  cl_xyz(J, cl, X, Y, Z);
  int ax[3], ay[3], az[3];
  prol_axis(X, cl.nx, cl.px, cxs, ax);
  prol_axis(Y, cl.ny, cl.py, cys, ay);
  prol_axis(Z, cl.nz, cl.pz, czs, az);
  const float vp = xc[J];
  float v[3][3][3];
#pragma unroll
  for (int dz = 0; dz < 3; ++dz)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const uint32_t Jn = ((uint32_t)az[dz] * (uint32_t)cl.ny + (uint32_t)ay[dy]) * (uint32_t)cl.nx +
                            (uint32_t)ax[dx];
        v[dz][dy][dx] = (Dinv_c[Jn] != 0.f) ? xc[Jn] : vp;
      }
  // weight of the parent's coordinate and of the side neighbour per axis
  const float wx[2] = {cxs ? 0.75f : 1.f, cxs ? 0.25f : 0.f};
  const float wy[2] = {cys ? 0.75f : 1.f, cys ? 0.25f : 0.f};
  const float wz[2] = {czs ? 0.75f : 1.f, czs ? 0.25f : 0.f};
#pragma unroll
  for (int kz = 0; kz < 2; ++kz)
#pragma unroll
    for (int ky = 0; ky < 2; ++ky)
#pragma unroll
      for (int kx = 0; kx < 2; ++kx) {
        if (kx > cxs || ky > cys || kz > czs) continue;
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int bb = 0; bb < 2; ++bb)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
              const int sz = c ? (kz ? 2 : 0) : 1, sy = bb ? (ky ? 2 : 0) : 1,
                        sx = a ? (kx ? 2 : 0) : 1;
              acc = fmaf(wx[a] * wy[bb] * wz[c], v[sz][sy][sx], acc);
            }
        const int x = (X << cxs) + kx, y = (Y << cys) + ky, z = (Z << czs) + kz;
        if (FINE0) {
          const uint32_t q = sp_idx(b, x, y, z);
          if (WALLS && (mask[q] & FACE_SOLID)) continue;
          ef[q] += acc;
        } else {
          const uint32_t c = ((uint32_t)z * (uint32_t)f.ny + (uint32_t)y) * (uint32_t)f.nx + (uint32_t)x;
          if (Dinv_f[c] == 0.f) continue;
          ef[c] += acc;
        }
      }
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

// Restriction from the fine box when the coarse level halves every axis
// (z-marching form of k_restrict0): one thread per coarse (X, Y) walks zc
// coarse planes.  Faces between two children of one coarse cell cancel in
// the sum of (A e)_i over the children, so rhs_c = sum over fluid children of
// r_i minus (e_i - e_out) over the open faces leaving the block.  The e of
// fine planes 2Z - 1 .. 2Z + 2 of the pair column are kept in registers.
template <bool WALLS>
__global__ void __launch_bounds__(256) k_restrict0_zm(
    const float* __restrict__ e, const float* __restrict__ r,
    const uint8_t* __restrict__ mask, Box b, CL cl, int zc, float* __restrict__ rhs_c) {
  const int X = blockIdx.x * blockDim.x + threadIdx.x;
  const int Y = blockIdx.y * blockDim.y + threadIdx.y;
  if (X >= cl.nx || Y >= cl.ny) return;
  const int Z0 = blockIdx.z * zc;
  const int Z1 = min(Z0 + zc, cl.nz);
  const uint32_t plane = (uint32_t)b.ny * (uint32_t)b.hx;
  const int Xm = (X == 0) ? b.hx - 1 : X - 1, Xp = (X == b.hx - 1) ? 0 : X + 1;
  const int y0 = 2 * Y;
  const int ym = (y0 == 0) ? b.ny - 1 : y0 - 1, yp = (y0 + 2 == b.ny) ? 0 : y0 + 2;
  // fine plane index with wrap (periodic) or clamp (the face is closed)
  auto zf = [&](int z) -> int {
    if (z < 0) return b.perz ? z + b.nzb : 0;
    if (z >= b.nzb) return b.perz ? z - b.nzb : b.nzb - 1;
    return z;
  };
  // e of fine cell (2X + kx, y0 + ky, z) of the pair column
  auto ecol = [&](int z, int ky, int kx) -> float {
    const uint32_t q = ((kx + ky + z) & 1) ? b.H : 0u;
    return e[q + (uint32_t)z * plane + (uint32_t)(y0 + ky) * b.hx + X];
  };
  float E[4][2][2];  // fine planes 2Z - 1, 2Z, 2Z + 1, 2Z + 2
  {
    const int za = zf(2 * Z0 - 1), zb = 2 * Z0;
#pragma unroll
    for (int ky = 0; ky < 2; ++ky)
#pragma unroll
      for (int kx = 0; kx < 2; ++kx) {
        E[0][ky][kx] = ecol(za, ky, kx);
        E[1][ky][kx] = ecol(zb, ky, kx);
      }
  }
  for (int Z = Z0; Z < Z1; ++Z) {
    const int z2 = 2 * Z + 1, z3 = zf(2 * Z + 2);
#pragma unroll
    for (int ky = 0; ky < 2; ++ky)
#pragma unroll
      for (int kx = 0; kx < 2; ++kx) {
        E[2][ky][kx] = ecol(z2, ky, kx);
        E[3][ky][kx] = ecol(z3, ky, kx);
      }
    // every load first (the masks only select among loaded values)
    uint32_t M[2][2][2];
    float RI[2][2][2], EXO[2][2][2], EYO[2][2][2];
#pragma unroll
    for (int kz = 0; kz < 2; ++kz)
#pragma unroll
      for (int ky = 0; ky < 2; ++ky)
#pragma unroll
        for (int kx = 0; kx < 2; ++kx) {
          const int z = 2 * Z + kz, y = y0 + ky;
          const uint32_t q = ((kx + ky + kz) & 1) ? b.H : 0u;  // colour of the child
          const uint32_t qo = b.H - q;                          // its face neighbours
          const uint32_t row = (uint32_t)z * plane + (uint32_t)y * b.hx;
          M[kz][ky][kx] = WALLS ? (uint32_t)mask[q + row + X] : FACES_OPEN;
          RI[kz][ky][kx] = r[q + row + X];
          // x face leaving the block: -x for kx = 0 (pair X - 1), +x for kx = 1
          EXO[kz][ky][kx] = e[qo + row + (kx ? Xp : Xm)];
          // y face leaving the block: row y0 - 1 or y0 + 2, same pair
          EYO[kz][ky][kx] = e[qo + (uint32_t)z * plane + (uint32_t)(ky ? yp : ym) * b.hx + X];
        }
    float acc = 0.f;
#pragma unroll
    for (int kz = 0; kz < 2; ++kz)
#pragma unroll
      for (int ky = 0; ky < 2; ++ky)
#pragma unroll
        for (int kx = 0; kx < 2; ++kx) {
          const uint32_t m = M[kz][ky][kx];
          if (m & FACE_SOLID) continue;
          const float ei = E[1 + kz][ky][kx];
          float Ae = 0.f;
          if (m & (kx ? 1u : 2u)) Ae += ei - EXO[kz][ky][kx];
          if (m & (ky ? 4u : 8u)) Ae += ei - EYO[kz][ky][kx];
          // z face leaving the block: planes 2Z - 1 or 2Z + 2 (registers)
          if (m & (kz ? 16u : 32u)) Ae += ei - (kz ? E[3][ky][kx] : E[0][ky][kx]);
          acc += RI[kz][ky][kx] - Ae;
        }
    rhs_c[((uint32_t)Z * cl.ny + Y) * cl.nx + X] = acc;
#pragma unroll
    for (int ky = 0; ky < 2; ++ky)
#pragma unroll
      for (int kx = 0; kx < 2; ++kx) {
        E[0][ky][kx] = E[2][ky][kx];
        E[1][ky][kx] = E[3][ky][kx];
      }
  }
}

// Prolongation to the fine box when the coarse level halves every axis
// (z-marching form of k_prolong<true, WALLS>): one thread per coarse (X, Y)
// walks zc coarse planes, keeping the 3 x 3 coarse neighbourhood of the
// planes below, here and above in registers (values, and a bit per cell for
// "active").  The eight children of a plane are loaded before any is
// stored, so that their loads overlap.
template <bool WALLS>
__global__ void __launch_bounds__(256) k_prolong0_zm(
    float* __restrict__ ef, const uint8_t* __restrict__ mask, Box b,
    const float* __restrict__ xc, const float* __restrict__ Dinv_c, CL cl, int zc) {
  const int X = blockIdx.x * blockDim.x + threadIdx.x;
  const int Y = blockIdx.y * blockDim.y + threadIdx.y;
  if (X >= cl.nx || Y >= cl.ny) return;
  const int Z0 = blockIdx.z * zc;
  const int Z1 = min(Z0 + zc, cl.nz);
  int ax[3], ay[3];
  prol_axis(X, cl.nx, cl.px, 1, ax);
  prol_axis(Y, cl.ny, cl.py, 1, ay);
  const uint32_t cplane = (uint32_t)cl.nx * (uint32_t)cl.ny;
  const uint32_t plane = (uint32_t)b.ny * (uint32_t)b.hx;
  float R[3][3][3];
  uint32_t act = 0;  // bit (dz * 9 + dy * 3 + dx): coarse cell active
  auto load_plane = [&](int Zp, int dz) {
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const uint32_t j = (uint32_t)Zp * cplane + (uint32_t)ay[dy] * cl.nx + (uint32_t)ax[dx];
        R[dz][dy][dx] = xc[j];
        if (Dinv_c[j] != 0.f) act |= 1u << (dz * 9 + dy * 3 + dx);
      }
  };
  auto zcl = [&](int Zq) -> int {  // coarse plane: wrap (periodic) or the parent's
    if (Zq < 0) return cl.pz ? Zq + cl.nz : Zq + 1;
    if (Zq >= cl.nz) return cl.pz ? Zq - cl.nz : Zq - 1;
    return Zq;
  };
  load_plane(zcl(Z0 - 1), 0);
  load_plane(Z0, 1);
  for (int Z = Z0; Z < Z1; ++Z) {
    act &= (1u << 18) - 1u;
    load_plane(zcl(Z + 1), 2);
    float EF[2][2][2];
    uint32_t MK[2][2][2];
#pragma unroll
    for (int kz = 0; kz < 2; ++kz)
#pragma unroll
      for (int ky = 0; ky < 2; ++ky)
#pragma unroll
        for (int kx = 0; kx < 2; ++kx) {
          const uint32_t q = ((kx + ky + kz) & 1) ? b.H : 0u;
          const uint32_t i = q + (uint32_t)(2 * Z + kz) * plane + (uint32_t)(2 * Y + ky) * b.hx + X;
          EF[kz][ky][kx] = ef[i];
          MK[kz][ky][kx] = WALLS ? (uint32_t)mask[i] : FACES_OPEN;
        }
    const float vp = R[1][1][1];
#pragma unroll
    for (int kz = 0; kz < 2; ++kz)
#pragma unroll
      for (int ky = 0; ky < 2; ++ky)
#pragma unroll
        for (int kx = 0; kx < 2; ++kx) {
          float acc = 0.f;
#pragma unroll
          for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int bb = 0; bb < 2; ++bb)
#pragma unroll
              for (int a = 0; a < 2; ++a) {
                const int sz = c ? (kz ? 2 : 0) : 1, sy = bb ? (ky ? 2 : 0) : 1,
                          sx = a ? (kx ? 2 : 0) : 1;
                const float w = (a ? 0.25f : 0.75f) * (bb ? 0.25f : 0.75f) * (c ? 0.25f : 0.75f);
                const float v = ((act >> (sz * 9 + sy * 3 + sx)) & 1u) ? R[sz][sy][sx] : vp;
                acc = fmaf(w, v, acc);
              }
          if (MK[kz][ky][kx] & FACE_SOLID) continue;
          const uint32_t q = ((kx + ky + kz) & 1) ? b.H : 0u;
          const uint32_t i = q + (uint32_t)(2 * Z + kz) * plane + (uint32_t)(2 * Y + ky) * b.hx + X;
          ef[i] = EF[kz][ky][kx] + acc;
        }
    act >>= 9;
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        R[0][dy][dx] = R[1][dy][dx];
        R[1][dy][dx] = R[2][dy][dx];
      }
  }
}

// Coarse pair interpolated at fine coordinate i along one axis: p0 the
// parent, p1 the neighbour on the child's side (the parent outside a
// non-periodic boundary), w0 the parent's weight.
__device__ __forceinline__ void prol_pair(int i, int n_c, int per, int coarsened,
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

// Trilinear interpolation of the coarse correction at fine cell (x, y, z).
__device__ __forceinline__ float prolong_cell(const float* xc, const float* Dinv_c,
                                             const CL& cl, int x, int y, int z,
                                             int cxs, int cys, int czs) {
  int ax[2], ay[2], az[2];
  float wx0, wy0, wz0;
  prol_pair(x, cl.nx, cl.px, cxs, ax[0], ax[1], wx0);
  prol_pair(y, cl.ny, cl.py, cys, ay[0], ay[1], wy0);
  prol_pair(z, cl.nz, cl.pz, czs, az[0], az[1], wz0);
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
  b.hx = (b.nx + 1) / 2;
  b.H = (uint32_t)((int64_t)b.nzb * b.ny * b.hx);
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
  cudaFree(P.face);
  cudaFree(P.nacc);
  if (P.hacc) cudaFreeHost(P.hacc);
  P.face = nullptr;
  P.nacc = nullptr;
  P.hacc = nullptr;
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
  // level 0 fields are colour-split: two arrays of nzb ny ceil(nx / 2)
  const size_t split = 2 * (size_t)P.nzb * ny * ((nx + 1) / 2);
  if (cudaMalloc(&L0.e, split * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&L0.rhs, split * sizeof(float)) != cudaSuccess) {
    h->err = "Poisson level 0 allocation failed";
    return LBM_ENOMEM;
  }
  // wall cells and pad cells are never read; cleared once so that no
  // uninitialised value is ever visible
  cudaMemset(L0.e, 0, split * sizeof(float));
  cudaMemset(L0.rhs, 0, split * sizeof(float));
  P.lev.push_back(L0);
  cudaFree(P.face);
  P.face = nullptr;
  if (h->has_walls) {
    if (cudaMalloc(&P.face, split) != cudaSuccess) {
      h->err = "Poisson face mask allocation failed";
      return LBM_ENOMEM;
    }
    cudaMemset(P.face, (int)FACE_SOLID, split);
    const Box b = make_box(h);
    k_face_mask<<<nblocks(L0.n, 256), 256, 0, h->st>>>(h->links, b, (uint32_t)L0.n, P.face);
    LBM_CUDA_TRY(h, cudaGetLastError());
  }
  if (!P.nacc) {
    if (cudaMalloc(&P.nacc, 2 * MG_NACC * sizeof(float)) != cudaSuccess ||
        cudaMallocHost(&P.hacc, 2 * MG_NACC * sizeof(float)) != cudaSuccess) {
      h->err = "Poisson norm slot allocation failed";
      return LBM_ENOMEM;
    }
  }

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

// The z-marching fine-box kernels need a true red-black two-colouring: x
// and y extents even, z extent even unless z is not periodic.
bool zm_fine(const Box& b) {
  return (b.nx % 2 == 0) && (b.ny % 2 == 0) && (!b.perz || b.nzb % 2 == 0);
}

// ... and, for the restriction and prolongation, a first coarse level that
// halves every axis.
bool zm_coarse(const Poisson& P, const Box& b) {
  return zm_fine(b) && P.lev.size() > 1 && P.lev[1].coarsened[0] && P.lev[1].coarsened[1] &&
         P.lev[1].coarsened[2];
}

constexpr int ZM_PLANES = 8;         // fine planes per thread
constexpr int ZM_COARSE_PLANES = 4;  // coarse planes per thread (restriction, prolongation)

// Launch shape of a z-marching kernel over nxp x nyp columns and nz planes:
// 256 threads as TX x TY with TX (up to 32) along x, runs of zc planes.
struct ZmShape {
  dim3 grid, block;
  int zc;
};
ZmShape zm_shape(int nxp, int nyp, int nz, int zc) {
  int tx = 1;
  while (tx < nxp && tx < 32) tx <<= 1;
  const int ty = 256 / tx;
  ZmShape z;
  z.block = dim3((unsigned)tx, (unsigned)ty, 1);
  z.zc = std::max(1, std::min(zc, nz));
  z.grid = dim3((unsigned)((nxp + tx - 1) / tx), (unsigned)((nyp + ty - 1) / ty),
                (unsigned)((nz + z.zc - 1) / z.zc));
  return z;
}

// Queues the fine-box residual of the current potential and the
// device-to-host copy of its norm slots; does not wait.  snorm: also the
// source norm (the first residual of a solve; later ones reuse it).
template <bool SNORM>
void residual_kernel(lbm_t* h, const Box& b) {
  Poisson& P = h->ps;
  const int64_t nbox = P.lev[0].n;
  const double inv_nf = 1.0 / (double)h->nfluid;
  const unsigned nb = nblocks(nbox, 256);
  if (zm_fine(b)) {
    const ZmShape z = zm_shape(b.hx, b.ny, b.nzb, ZM_PLANES);
    if (h->has_walls)
      k_res0_zm<true, SNORM><<<z.grid, z.block, 0, h->st>>>(P.psi[P.cur], P.src, P.face,
                                                            P.lev[0].rhs, P.dsum, P.nacc, b, z.zc,
                                                            inv_nf, P.label, P.comp_mean);
    else
      k_res0_zm<false, SNORM><<<z.grid, z.block, 0, h->st>>>(P.psi[P.cur], P.src, nullptr,
                                                             P.lev[0].rhs, P.dsum, P.nacc, b, z.zc,
                                                             inv_nf, nullptr, nullptr);
  } else if (h->has_walls) {
    k_res0<true, SNORM><<<nb, 256, 0, h->st>>>(P.psi[P.cur], P.src, P.face, P.lev[0].rhs, P.dsum,
                                               P.nacc, b, (uint32_t)nbox, inv_nf, P.label,
                                               P.comp_mean);
  } else {
    k_res0<false, SNORM><<<nb, 256, 0, h->st>>>(P.psi[P.cur], P.src, nullptr, P.lev[0].rhs,
                                                P.dsum, P.nacc, b, (uint32_t)nbox, inv_nf, nullptr,
                                                nullptr);
  }
}

cudaError_t residual_launch(lbm_t* h, bool snorm = false) {
  Poisson& P = h->ps;
  const Box b = make_box(h);
  cudaError_t e = cudaMemsetAsync(P.nacc, 0, 2 * MG_NACC * sizeof(float), h->st);
  if (e != cudaSuccess) return e;
  if (snorm) residual_kernel<true>(h, b);
  else residual_kernel<false>(h, b);
  P.snorm_pending = snorm;
  ++h->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaMemcpyAsync(P.hacc, P.nacc, 2 * MG_NACC * sizeof(float), cudaMemcpyDeviceToHost,
                         h->st);
}

// Norms ||r||_2 and ||s - <s>||_2 (fixed-point units) of the last residual
// read back.
void residual_norms(Poisson& P, double* rn, double* sn) {
  double a = 0.0, c = 0.0;
  for (int k = 0; k < MG_NACC; ++k) {
    a += (double)P.hacc[k];
    c += (double)P.hacc[MG_NACC + k];
  }
  *rn = sqrt(a) * 1048576.0;
  if (P.snorm_pending) {
    P.snorm = sqrt(c) * 1048576.0;
    P.snorm_pending = false;
  }
  *sn = P.snorm;
}

// Waits for the last queued residual.  Returns ||r|| / ||s|| in *rel and
// whether the solve has converged: relative residual <= tol, or a residual
// at the fixed-point resolution of psi (rms below 2 units of 2^-52), which
// is all a charge-neutral source of vanishing norm allows.
lbm_status residual_read(lbm_t* h, double tol, double* rel, bool* done) {
  Poisson& P = h->ps;
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  double rn, sn;
  residual_norms(P, &rn, &sn);
  *rel = sn > 0.0 ? rn / sn : (rn > 0.0 ? INFINITY : 0.0);
  if (!isfinite(rn) || !isfinite(sn)) {
    h->err = "Poisson residual is not finite";
    return LBM_EUNSTABLE;
  }
  *done = rn <= tol * sn || rn <= RES_FLOOR_RMS * sqrt((double)h->nfluid);
  return LBM_OK;
}

template <int MODE>
void smooth0_launch(lbm_t* h, const Box& b, unsigned nb, int color) {
  Poisson& P = h->ps;
  PoissonLevel& L = P.lev[0];
  const int64_t* pin = P.psi[P.cur];
  int64_t* pout = P.psi[P.cur ^ 1];
  if (zm_fine(b) && b.nx % 4 == 0) {
    const ZmShape z = zm_shape(b.hx / 2, b.ny, b.nzb, ZM_PLANES);
    if (h->has_walls)
      k_smooth0_zq<true, MODE><<<z.grid, z.block, 0, h->st>>>(L.e, L.rhs, P.face, b, color, z.zc,
                                                              pin, pout);
    else
      k_smooth0_zq<false, MODE><<<z.grid, z.block, 0, h->st>>>(L.e, L.rhs, nullptr, b, color,
                                                               z.zc, pin, pout);
  } else if (zm_fine(b)) {
    const ZmShape z = zm_shape(b.hx, b.ny, b.nzb, ZM_PLANES);
    if (h->has_walls)
      k_smooth0_zm<true, MODE><<<z.grid, z.block, 0, h->st>>>(L.e, L.rhs, P.face, b, color, z.zc,
                                                              pin, pout);
    else
      k_smooth0_zm<false, MODE><<<z.grid, z.block, 0, h->st>>>(L.e, L.rhs, nullptr, b, color,
                                                               z.zc, pin, pout);
  } else if (h->has_walls) {
    k_smooth0<true, MODE><<<nb, 256, 0, h->st>>>(L.e, L.rhs, P.face, b, color, pin, pout);
  } else {
    k_smooth0<false, MODE><<<nb, 256, 0, h->st>>>(L.e, L.rhs, nullptr, b, color, pin, pout);
  }
  ++h->launches;
}

// `sweeps` red-black sweeps on level l.  On the fine box: zero_start, the
// first half-sweep starts from e = 0; apply, the last half-sweep writes the
// corrected potential into the other buffer, which becomes current.
cudaError_t smooth_level(lbm_t* h, int l, int sweeps, bool apply = false,
                         bool zero_start = false) {
  Poisson& P = h->ps;
  PoissonLevel& L = P.lev[l];
  if (l == 0) {
    const Box b = make_box(h);
    const unsigned nb = nblocks(b.H, 256);
    for (int k = 0; k < sweeps; ++k)
      for (int color = 0; color < 2; ++color) {
        if (zero_start && k == 0 && color == 0) smooth0_launch<1>(h, b, nb, color);
        else if (apply && k == sweeps - 1 && color == 1) smooth0_launch<2>(h, b, nb, color);
        else smooth0_launch<0>(h, b, nb, color);
      }
    if (apply) P.cur ^= 1;
  } else {
    const int compact = (L.nx % 2 == 0) ? 1 : 0;
    const unsigned nb = nblocks(compact ? L.n / 2 : L.n, 256);
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
  cudaError_t e = cudaSuccess;
  // the first half-sweep starts from e = 0 (no clearing pass)
  if (nl == 1) return smooth_level(h, 0, 8, true, true);
  const int lc = sub_level(P);
  if (P.nu1 > 0) {
    if ((e = smooth_level(h, 0, P.nu1, false, true)) != cudaSuccess) return e;
  } else if ((e = cudaMemsetAsync(P.lev[0].e, 0, 2 * (size_t)b.H * sizeof(float), h->st)) !=
             cudaSuccess) {
    return e;
  }
  {
    PoissonLevel& C = P.lev[1];
    const CL cl = make_cl(C);
    const ZmShape zs = zm_shape(cl.nx, cl.ny, cl.nz, ZM_COARSE_PLANES);
    if (zm_coarse(P, b) && h->has_walls)
      k_restrict0_zm<true><<<zs.grid, zs.block, 0, h->st>>>(P.lev[0].e, P.lev[0].rhs, P.face, b,
                                                            cl, zs.zc, C.rhs);
    else if (zm_coarse(P, b))
      k_restrict0_zm<false><<<zs.grid, zs.block, 0, h->st>>>(P.lev[0].e, P.lev[0].rhs, nullptr, b,
                                                             cl, zs.zc, C.rhs);
    else if (h->has_walls)
      k_restrict0<true><<<nblocks(C.n, 256), 256, 0, h->st>>>(
          P.lev[0].e, P.lev[0].rhs, P.face, b, cl, C.coarsened[0], C.coarsened[1],
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
    if ((e = smooth_level(h, l, P.nuc1)) != cudaSuccess) return e;
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
    const unsigned nb = nblocks(C.n, 256);  // one thread per coarse cell
    if (l == 0 && zm_coarse(P, b)) {
      const CL cl = make_cl(C);
      const ZmShape zs = zm_shape(cl.nx, cl.ny, cl.nz, ZM_COARSE_PLANES);
      if (h->has_walls)
        k_prolong0_zm<true><<<zs.grid, zs.block, 0, h->st>>>(F.e, P.face, b, C.e, C.Dinv, cl,
                                                             zs.zc);
      else
        k_prolong0_zm<false><<<zs.grid, zs.block, 0, h->st>>>(F.e, nullptr, b, C.e, C.Dinv, cl,
                                                              zs.zc);
    } else if (l == 0) {
      if (h->has_walls)
        k_prolong<true, true><<<nb, 256, 0, h->st>>>(F.e, nullptr, P.face, b, make_cl(F),
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
    if ((e = smooth_level(h, l, l == 0 ? std::max(P.nu2, 1) : P.nuc2, l == 0)) != cudaSuccess) return e;
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
  LBM_CUDA_TRY(h, residual_launch(h, true));
  lbm_status s = residual_read(h, tol, &rel, &done);
  if (s != LBM_OK) return s;
  if (!done && nn_active(h)) {
    // learned initial guess: apply, keep it only if the residual drops
    double rn, sn;
    residual_norms(P, &rn, &sn);
    rn *= PSI_INV_SCALE;
    bool applied = false;
    float* dpsi = nullptr;
    s = nn_before_solve(h, P.lev[0].rhs, P.zlo, P.nzb, (h->cfg.nx + 1) / 2,
                        rn / sqrt((double)h->nfluid), &applied, &dpsi);
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
