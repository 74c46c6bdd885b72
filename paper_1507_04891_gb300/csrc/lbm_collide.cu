// The fused stream/collide kernel of one population storage format.  This
// file is compiled once per format (LBM_COLLIDE_STORAGE = LBM_FP32,
// LBM_FP16_SHIFT, LBM_BF16_SHIFT), so that the instances of the kernel (species
// count, walls, charge, diagnostics) build in parallel; each object defines
// collide_dispatch<LBM_COLLIDE_STORAGE>.
#include "lbm_lattice.cuh"

#ifndef LBM_COLLIDE_STORAGE
#error "compile with -DLBM_COLLIDE_STORAGE=<storage code>"
#endif

namespace lbm_gb300 {
namespace {

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
//   6. (DIAG) FP64 diagnostics of the state after the step (Sec. 3: species
//      continuity, total momentum): every stored value is pulled by exactly
//      one fluid node at the next step (by r + c_p, or by r itself in the
//      opposite direction when r + c_p is a wall node), so the sums of the
//      stored values give the next state's species masses, and the stored
//      values signed by the direction they are pulled in give its momentum.
//      Per CTA: the deviation sums (FP32 within a warp, FP64 across warps)
//      and a count of nodes whose density entering the step was not finite
//      and positive, written to a[blockIdx.x * DIAG_NQ + k].
// ---------------------------------------------------------------------------
// Charge scatter: the target of a stored population h*_p(r) is r + c_p
// (it is pulled there at the next step).  Targets are grouped by their row
// offset (dy, dz) = (c_y, c_z), nine groups; GRP numbers them.  Five groups
// also hold directions with an x component (dy = 0 or dz = 0); XGRP numbers
// those.  Per node: q0[GRP] sums the contributions to (x, y + dy, z + dz),
// qp[XGRP] those to x + 1, qm[XGRP] those to x - 1.
__host__ __device__ __forceinline__ constexpr int GRP(int p) { return (CZ(p) + 1) * 3 + (CY(p) + 1); }
__host__ __device__ __forceinline__ constexpr int XGRP_OF(int dy, int dz) {
  return dz == 0 ? (dy == 0 ? 0 : (dy == 1 ? 1 : 2)) : (dz == 1 ? 3 : 4);
}
__host__ __device__ __forceinline__ constexpr int XGRP(int p) { return XGRP_OF(CY(p), CZ(p)); }

// (p is a constant once the direction loops are unrolled, so the sums stay
// in registers)
__device__ __forceinline__ void scat_add(int p, float (&q0)[9], float (&qp)[5], float (&qm)[5],
                                         float v) {
  if (CX(p) == 0) q0[GRP(p)] += v;
  else if (CX(p) == 1) qp[XGRP(p)] += v;
  else qm[XGRP(p)] += v;
}

// A warp holds 32 consecutive nodes of one x row (nx is a multiple of 32).
// Per target group (dy, dz) a lane adds the contributions that reach its own
// x: its own ones with c_x = 0, those of lane - 1 with c_x = +1 and of
// lane + 1 with c_x = -1 (register shuffles); rows of one warp wrap inside
// the warp, and for wider rows the first and last lane send the
// contributions that cross into the neighbouring warp themselves.  Each
// sum goes to the next step's source with one 64-bit integer atomic per
// target (exact, so the order in which warps add does not matter; the
// FP32 sums are formed in a fixed order, so every run gives the same
// source).  The node's own target also receives the reference part of the
// source, once per node.  (x, y, z): the lane's node.
__device__ __forceinline__ void scatter_charge(const StepArgs& a, int x, int y, int z,
                                               float (&c0)[9], const float (&cp)[5],
                                               const float (&cm)[5]) {
  const int lane = threadIdx.x & 31;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const bool one = nx == 32;  // the row is this warp: the shuffles wrap it
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const float fl = __shfl_sync(0xffffffffu, cp[j], (lane + 31) & 31);  // lane - 1 sends to x
    const float fr = __shfl_sync(0xffffffffu, cm[j], (lane + 1) & 31);   // lane + 1 sends to x
    const int g = j == 0 ? 4 : (j == 1 ? 5 : (j == 2 ? 3 : (j == 3 ? 7 : 1)));  // GRP of XGRP j
    if (one || lane != 0) c0[g] += fl;
    if (one || lane != 31) c0[g] += fr;
  }
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(a.scat_acc);
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
  const int64_t nxy = (int64_t)nx * ny;
  const int64_t rowz[3] = {(int64_t)zm * nxy, (int64_t)z * nxy, (int64_t)zp * nxy};
  const int rowy[3] = {ym * nx, y * nx, yp * nx};
#pragma unroll
  for (int g = 0; g < 9; ++g) {
    long long q = (long long)f32_to_i64_rn(c0[g]);
    if (g == 4) q += a.src_ref;
    atomicAdd(acc + rowz[g / 3] + rowy[g % 3] + x, (unsigned long long)q);
  }
  if (!one && (lane == 0 || lane == 31)) {
    // the contributions that cross into the neighbouring warp of the row
    const int xt = lane == 0 ? (x == 0 ? nx - 1 : x - 1) : (x == nx - 1 ? 0 : x + 1);
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const int g = j == 0 ? 4 : (j == 1 ? 5 : (j == 2 ? 3 : (j == 3 ? 7 : 1)));
      const float v = lane == 0 ? cm[j] : cp[j];
      atomicAdd(acc + rowz[g / 3] + rowy[g % 3] + xt, (unsigned long long)(long long)f32_to_i64_rn(v));
    }
  }
}

// Registers: up to 128 per thread (two 256-thread CTAs per SM), 255 for four
// species.  The 16-bit ternary kernel without walls is capped at 96: it is
// bound by instruction issue, and 20 warps per SM (128-thread CTAs) instead
// of 16 issue more often than the few spilled registers cost (measured at
// 128^3: 133 -> 127 us per launch; 88 registers: 130 us).
template <int S, bool WALLS, int ST>
constexpr int collide_maxnreg() {
  return S >= 4 ? 255 : ((ST != LBM_FP32 && !WALLS && S == 3) ? 96 : 128);
}

template <int S, bool WALLS, bool CHARGED, int ST, bool DIAG, bool PAIR, bool SCAT>
__global__ void __launch_bounds__(256) __maxnreg__((collide_maxnreg<S, WALLS, ST>()))
    k_stream_collide(const StepArgs a) {
  using T = typename Fmt<ST>::T;
  // a speculative launch the step has decided against (same for every
  // thread of the grid)
  if (a.skip && *a.skip) return;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  // deviation sums of the state after the step: masses, momentum, charge
  float qm[S], qjx = 0.f, qjy = 0.f, qjz = 0.f, qbad = 0.f;
#pragma unroll
  for (int s = 0; s < S; ++s) qm[s] = 0.f;
  // (SCAT) charge sent to the next step's source, per target group
  float c0[9], cp[5], cm[5];
#pragma unroll
  for (int g = 0; g < 9; ++g) c0[g] = 0.f;
#pragma unroll
  for (int g = 0; g < 5; ++g) cp[g] = cm[g] = 0.f;
  uint32_t lk = 0;
  const bool inrange = i < (uint32_t)a.N;
  bool active = inrange;
  if (WALLS && inrange) {
    lk = a.links[i];
    active = !(lk & LINK_SOLID);
  }
  // Wall nodes in a warp with fluid nodes run the same instructions with
  // their loads switched off and store what they computed from zeros into
  // their own slots (which no pull reads): every store of the warp then
  // covers whole sectors, so the L2 need not fetch the rest of a sector a
  // partial write leaves (measured on the porous box: about 130 MB of DRAM
  // reads per launch at 128^3).  A warp of wall nodes only does nothing.
  const bool any_fluid = WALLS ? __any_sync(0xffffffffu, active) : true;  // every lane votes
  const bool work = inrange && any_fluid;
  if (work) {
    int x, y, z;
    site_xyz(i, a.nx, a.ny, x, y, z);
    const Nbr o = neighbours(x, y, z, a.nx, a.ny, a.nz);
    const T* __restrict__ fin = static_cast<const T*>(a.fin);
    T* __restrict__ fout = static_cast<T*>(a.fout);
    const int64_t N = a.N;

    // stored h_p = (f_p - w_p n_ref) / (w_p n_ref) of every species, pulled
    // from r - c_p.  The addresses do not wait for the link word: every
    // lane loads from its upstream nodes at once; then, in a warp with a
    // fluid node next to a wall, the directions whose upstream node is a
    // wall node take the node's own reversed value (halfway bounce-back).
    // Wall lanes compute from zeros.
    float f[S][Q];
#pragma unroll
    for (int p = 0; p < Q; ++p) {
      const int d = upstream(o, p);
#pragma unroll
      for (int s = 0; s < S; ++s) f[s][p] = pull_h<ST, false>(fin, N, s, p, i, d, 0u);
    }
    if (WALLS) {
      const uint32_t wb = active ? (lk & ~LINK_SOLID) : 0u;
      if (__any_sync(__activemask(), wb != 0u)) {
#pragma unroll
        for (int p = 1; p < Q; ++p)
#pragma unroll
          for (int s = 0; s < S; ++s)
            if ((wb >> p) & 1u) f[s][p] = Fmt<ST>::ldh(fin + (int64_t)(s * Q + OPP(p)) * N + i);
      }
      if (!active) {
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
          for (int p = 0; p < Q; ++p) f[s][p] = 0.f;
      }
    }

    // n = n_ref (1 + sum w h), j = n_ref sum c w h  (sum w = 1, sum w c = 0),
    // summed per weight class (faces p = 1..6, edges 7..18) so that each
    // population costs additions only
    float mh[S], dn[S], n[S], jx[S], jy[S], jz[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      float sf = 0.f, se = 0.f, xf = 0.f, xe = 0.f, yf = 0.f, ye = 0.f, zf = 0.f, ze = 0.f;
#pragma unroll
      for (int p = 1; p < Q; ++p) {
        const float hp = f[s][p];
        if (p <= 6) {
          sf += hp;
          if (CX(p)) xf += CX(p) * hp;
          if (CY(p)) yf += CY(p) * hp;
          if (CZ(p)) zf += CZ(p) * hp;
        } else {
          se += hp;
          if (CX(p)) xe += CX(p) * hp;
          if (CY(p)) ye += CY(p) * hp;
          if (CZ(p)) ze += CZ(p) * hp;
        }
      }
      const float m0 = fmaf(WT(0), f[s][0], fmaf(WT(1), sf, WT(7) * se));
      const float mx = fmaf(WT(1), xf, WT(7) * xe);
      const float my = fmaf(WT(1), yf, WT(7) * ye);
      const float mz = fmaf(WT(1), zf, WT(7) * ze);
      const float r = a.nref[s];
      mh[s] = m0;
      dn[s] = r * m0;
      n[s] = r + dn[s];
      jx[s] = r * mx;
      jy[s] = r * my;
      jz[s] = r * mz;
      if (DIAG && active && (!(n[s] > 0.f) || !isfinite(n[s]))) qbad = 1.f;
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
    // pair frequencies: the fractions x_b and x_b v_b of every species
    float px[PAIR ? S : 1], pxv[PAIR ? S : 1][3];
    if (PAIR) {
#pragma unroll
      for (int b = 0; b < S; ++b) {
        px[b] = n[b] * inv_ntot;
        const float hz = 0.5f * a.valence[b] * n[b];
        pxv[b][0] = (jx[b] + hz * Ex) * inv_ntot;
        pxv[b][1] = (jy[b] + hz * Ey) * inv_ntot;
        pxv[b][2] = (jz[b] + hz * Ez) * inv_ntot;
      }
    }

    const float om = a.omega_visc;
    const float omd = a.omega_drag_z ? a.omega_drag_z[z] : a.omega_drag;
    uint32_t rnd = 0;
    if (ST != LBM_FP32) rnd = mix32(i * 0x9E3779B9u ^ mix32(a.step_dev ? *a.step_dev : a.step));
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const float inv_n = 1.0f / n[s];
      const float usx = jx[s] * inv_n, usy = jy[s] * inv_n, usz = jz[s] * inv_n;
      float Fx, Fy, Fz;
      if (PAIR)
        species_force_pair<S>(s, usx, usy, usz, a.valence[s], Ex, Ey, Ez, px, pxv, a, Fx, Fy, Fz);
      else
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
      // the per-species factors of the bracket values, once per species:
      // even' = Ce + Ae a^2 + Be (F.c)(u.c), odd' = Do (omega a + F.c)
      const float nin = n[s] * inr;
      const float Ae = nin * (4.5f * om), Be = nin * 9.0f, Ce = inr * (odn + base);
      const float Do = nin * 3.0f, Dom = Do * om;
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
        const float even = fmaf(Ae, av * av, fmaf(Be, fc * uc, Ce));
        const float odd = fmaf(Dom, av, Do * fc);
        const float2 hs = Fmt<ST>::sth_sr2(fout + (int64_t)(s * Q + p) * N + i,
                                           omm * f[s][p] + (even + odd),
                                           fout + (int64_t)(s * Q + p + 1) * N + i,
                                           omm * f[s][p + 1] + (even - odd), lcg_next(rnd));
        moved += WT(p) * (hs.x + hs.y);  // same weight for p and p+1
        if constexpr (SCAT) {
          // charge these two stored values carry to r + c_p and r - c_p
          // (zero for a neutral species)
          const float kw = a.scat_k[s] * WT(p);
          scat_add(p, c0, cp, cm, kw * hs.x);
          scat_add(p + 1, c0, cp, cm, kw * hs.y);
        }
        // momentum carried by the pair at the next step: h*_p moves along
        // c_p unless r + c_p is a wall node (bit p+1), then it is pulled
        // back along -c_p; h*_{p+1} likewise with bit p
        if (DIAG) {
          float mj = hs.x - hs.y;
          if (WALLS) mj = (((lk >> (p + 1)) & 1u) ? -hs.x : hs.x) - (((lk >> p) & 1u) ? -hs.y : hs.y);
          if (CX(p)) mjx += CX(p) * WT(p) * mj;
          if (CY(p)) mjy += CY(p) * WT(p) * mj;
          if (CZ(p)) mjz += CZ(p) * WT(p) * mj;
        }
      }
      const float h0 = Fmt<ST>::sth_sr(fout + (int64_t)(s * Q) * N + i, (mh[s] - moved) * INV_WT(0),
                                       lcg_next(rnd));
      if constexpr (SCAT) c0[GRP(0)] += a.scat_k[s] * WT(0) * h0;
      if (DIAG && active) {
        const float r = a.nref[s];
        qm[s] = r * (WT(0) * h0 + moved);
        qjx += r * mjx;
        qjy += r * mjy;
        qjz += r * mjz;
      }
    }
    if constexpr (SCAT) scatter_charge(a, x, y, z, c0, cp, cm);
  }


  // per-CTA partial sums of the diagnostics (inactive threads add zeros)
  if (DIAG) {
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

template <int S, bool W, bool C, int ST, bool SC>
cudaError_t launch_sc2(const StepArgs& a, cudaStream_t st, int threads, bool diag) {
  const unsigned nb = nblocks(a.N, threads);
  // the pair-frequency drag exists for three or more species (a binary
  // depends on its one cross frequency, which the host passes as omega_drag)
  constexpr bool CAN_PAIR = S >= 3;
  if (CAN_PAIR && a.pair_on) {
    if (diag)
      k_stream_collide<S, W, C, ST, true, CAN_PAIR, SC><<<nb, threads, 0, st>>>(a);
    else
      k_stream_collide<S, W, C, ST, false, CAN_PAIR, SC><<<nb, threads, 0, st>>>(a);
  } else {
    if (diag)
      k_stream_collide<S, W, C, ST, true, false, SC><<<nb, threads, 0, st>>>(a);
    else
      k_stream_collide<S, W, C, ST, false, false, SC><<<nb, threads, 0, st>>>(a);
  }
  return cudaGetLastError();
}

// The charge scatter: a.scat_acc is set by the host only for charged FP32
// lattices without walls whose nx is a multiple of 32.
template <int S, bool W, bool C, int ST>
cudaError_t launch_sc(const StepArgs& a, cudaStream_t st, int threads, bool diag) {
  if constexpr (!W && C && ST == LBM_FP32) {
    if (a.scat_acc) return launch_sc2<S, W, C, ST, true>(a, st, threads, diag);
  }
  return launch_sc2<S, W, C, ST, false>(a, st, threads, diag);
}

template <int S, int ST>
cudaError_t dispatch_wc(const StepArgs& a, bool w, bool c, cudaStream_t st, int t, bool d) {
  if (w) return c ? launch_sc<S, true, true, ST>(a, st, t, d) : launch_sc<S, true, false, ST>(a, st, t, d);
  return c ? launch_sc<S, false, true, ST>(a, st, t, d) : launch_sc<S, false, false, ST>(a, st, t, d);
}

}  // namespace

template <>
cudaError_t collide_dispatch<LBM_COLLIDE_STORAGE>(const StepArgs& a, int S, bool w, bool c,
                                                  cudaStream_t st, int threads, bool d) {
  constexpr int ST = LBM_COLLIDE_STORAGE;
  switch (S) {
    case 1: return dispatch_wc<1, ST>(a, w, c, st, threads, d);
    case 2: return dispatch_wc<2, ST>(a, w, c, st, threads, d);
    case 3: return dispatch_wc<3, ST>(a, w, c, st, threads, d);
    case 4: return dispatch_wc<4, ST>(a, w, c, st, threads, d);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm_gb300
