// C ABI of the library (declared in include/lbm.h): argument checking,
// device memory ownership and the per-step launch sequence.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.cuh"

using namespace lbm_gb300;

namespace {

thread_local std::string g_create_error;

lbm_status fail(lbm_t* h, lbm_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

template <typename T>
lbm_status dev_alloc(lbm_t* h, T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(h, LBM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return LBM_OK;
}

// RAII scratch buffer for one call.
struct Scratch {
  void* p = nullptr;
  ~Scratch() {
    if (p) cudaFree(p);
  }
};

bool species_complete(const lbm_t* h) {
  return h->species_set == ((1u << h->S) - 1u);
}

// Returns the index of a recorded event (from a reusable pool).
cudaError_t mark(lbm_t* h, int* idx) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    h->ev_pool.push_back(e);
  }
  *idx = (int)h->ev_used++;
  return cudaEventRecord(h->ev_pool[*idx], h->st);
}

// Adds the elapsed times of all recorded phase pairs to the sums.
cudaError_t drain_timing(lbm_t* h) {
  for (auto& m : h->ev_marks) {
    cudaError_t r = cudaEventSynchronize(h->ev_pool[m.second.second]);
    if (r != cudaSuccess) return r;
    float ms = 0.f;
    r = cudaEventElapsedTime(&ms, h->ev_pool[m.second.first], h->ev_pool[m.second.second]);
    if (r != cudaSuccess) return r;
    h->t_acc[m.first] += ms;
  }
  h->ev_marks.clear();
  h->ev_used = 0;
  return cudaSuccess;
}

struct Phase {
  lbm_t* h;
  int phase, a = -1;
  Phase(lbm_t* hh, int p) : h(hh), phase(p) {
    if (h->timing) mark(h, &a);
  }
  cudaError_t stop() {
    if (!h->timing || a < 0) return cudaSuccess;
    int b;
    cudaError_t r = mark(h, &b);
    if (r == cudaSuccess) h->ev_marks.push_back({phase, {a, b}});
    a = -1;
    return r;
  }
};

}  // namespace

namespace lbm_gb300 {

void note_start_residual(lbm_t* h, double rel) {
  if (!(rel >= 0.0) || !isfinite(rel)) return;
  h->last_start = rel;
  h->start_log_sum += log10(std::max(rel, 1e-300));
  h->start_count += 1;
}

cudaError_t own_stream(lbm_t* h) {
  h->st = h->own;
  if (!h->foreign_pending) return cudaSuccess;
  h->foreign_pending = false;
  return cudaStreamWaitEvent(h->own, h->order_ev, 0);
}

}  // namespace lbm_gb300

namespace {

// The stream of a call with a stream argument (NULL: the library's own
// stream).  A caller's stream first waits for the work queued on the own
// stream; when the call ends, an event recorded on the caller's stream
// makes the next call on the own stream wait for this call's work.
struct CallStream {
  lbm_t* h;
  cudaError_t err = cudaSuccess;
  CallStream(lbm_t* hh, void* stream) : h(hh) {
    err = own_stream(h);
    if (err == cudaSuccess && stream && (cudaStream_t)stream != h->own) {
      err = cudaEventRecord(h->order_ev, h->own);
      if (err == cudaSuccess) err = cudaStreamWaitEvent((cudaStream_t)stream, h->order_ev, 0);
      if (err == cudaSuccess) h->st = (cudaStream_t)stream;
    }
  }
  ~CallStream() {
    if (h->st != h->own && cudaEventRecord(h->order_ev, h->st) == cudaSuccess)
      h->foreign_pending = true;
  }
};

// Argument checks shared by lbm_set_species and lbm_set_species_dev.
// The address under which the handle's device reaches caller memory p:
// device or managed memory of any device as is, pinned host memory through
// its mapped device address.  Anything else (pageable host memory, an
// unknown pointer) is refused here, before a kernel could touch it.
lbm_status device_view(lbm_t* h, const void* p, void** out, const char* what) {
  *out = nullptr;
  if (!p) return LBM_OK;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, LBM_EINVAL, std::string(what) + " is not memory the device can reach");
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    *out = const_cast<void*>(p);
    return LBM_OK;
  }
  if (at.type == cudaMemoryTypeHost && at.devicePointer) {
    *out = at.devicePointer;
    return LBM_OK;
  }
  return fail(h, LBM_EINVAL,
              std::string(what) + " must be device memory or pinned (mapped) host memory");
}

lbm_status species_args(lbm_t* h, int s, double mass, double valence, const void* n0) {
  if (!h) return LBM_EINVAL;
  if (s < 0 || s >= h->S) return fail(h, LBM_EINVAL, "species index out of range");
  if (!n0) return fail(h, LBM_EINVAL, "n0 is NULL");
  if (!(mass > 0.0) || !isfinite(mass) || !isfinite(valence))
    return fail(h, LBM_EINVAL, "mass must be > 0 and valence finite");
  if (h->species_set && fabs(mass - h->mass0) > 1e-12 * h->mass0)
    return fail(h, LBM_EINVAL,
                "all species must have the same mass (one thermal speed on the lattice)");
  return LBM_OK;
}

// Bookkeeping after species s was initialised: the state restarts at step 0.
lbm_status species_done(lbm_t* h, int s, double mass, double valence) {
  h->mass[s] = (float)mass;
  h->valence[s] = (float)valence;
  if (!h->species_set) h->mass0 = mass;
  h->species_set |= 1u << s;
  h->tstep = 0;
  h->psi_valid = false;
  h->diag_valid = false;
  return potential_history_reset(h);
}

}  // namespace

extern "C" {

void lbm_config_default(lbm_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->nx = c->ny = c->nz = 1;
  c->nspecies = 1;
  c->omega_visc = 1.0;
  c->omega_drag = 1.0;
  c->bjerrum = 0.0;
  c->storage = LBM_FP32;
  c->poisson = LBM_POISSON_MG;
  c->poisson_tol = 1e-8;
  c->poisson_maxit = 200;
  c->device = 0;
  c->flags = 0;
}

lbm_status lbm_create(const lbm_config* cfg, lbm_t** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (!cfg) {
    g_create_error = "cfg is NULL";
    return LBM_EINVAL;
  }
  const lbm_config& c = *cfg;
  if (c.nx < 1 || c.ny < 1 || c.nz < 1) {
    g_create_error = "lattice extents must be >= 1";
    return LBM_EINVAL;
  }
  const int64_t N = (int64_t)c.nx * c.ny * c.nz;
  if (N > (int64_t)1 << 30) {
    g_create_error = "lattice larger than 2^30 nodes";
    return LBM_EINVAL;
  }
  if (c.nspecies < 1 || c.nspecies > MAX_SPECIES) {
    g_create_error = "nspecies must be in 1..4";
    return LBM_EINVAL;
  }
  if (!(c.omega_visc > 0.0 && c.omega_visc < 2.0) ||
      !(c.omega_drag > 0.0 && c.omega_drag < 2.0)) {
    g_create_error = "omega_visc and omega_drag must lie in (0, 2)";
    return LBM_EINVAL;
  }
  if (c.storage != LBM_FP32 && c.storage != LBM_FP16_SHIFT && c.storage != LBM_BF16_SHIFT) {
    g_create_error = "unknown storage code";
    return LBM_EINVAL;
  }
  if (c.poisson != LBM_POISSON_MG && c.poisson != LBM_POISSON_SOR && c.poisson != LBM_POISSON_FFT) {
    g_create_error = "unknown Poisson solver code";
    return LBM_EINVAL;
  }
  if (!(c.bjerrum >= 0.0) || !isfinite(c.bjerrum)) {
    g_create_error = "bjerrum must be finite and >= 0";
    return LBM_EINVAL;
  }
  if (c.bjerrum > 0.0 && (!(c.poisson_tol > 0.0) || c.poisson_maxit < 1)) {
    g_create_error = "poisson_tol must be > 0 and poisson_maxit >= 1";
    return LBM_EINVAL;
  }
  if ((c.flags & LBM_FLAG_STEP_GRAPH) && (c.poisson != LBM_POISSON_FFT || !(c.bjerrum > 0.0))) {
    g_create_error = "LBM_FLAG_STEP_GRAPH needs the spectral Poisson solver and bjerrum > 0";
    return LBM_EINVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) {
    cudaGetLastError();
    g_create_error = "no CUDA device with the requested ordinal";
    return LBM_ECUDA;
  }
  lbm_t* h = new (std::nothrow) lbm_t();
  if (!h) return LBM_ENOMEM;
  h->cfg = c;
  h->omega_drag_cfg = c.omega_drag;
  h->S = c.nspecies;
  h->N = N;
  h->dev = c.device;
  h->nfluid = N;
  h->esize = (c.storage == LBM_FP32) ? 4 : 2;
  lbm_status s = LBM_OK;
  // the library's stream at the greatest priority: kernels of lower-priority
  // side work (the fit of the Poisson start) yield SMs to it
  int prio_lo = 0, prio_hi = 0;
  if (cudaSetDevice(h->dev) != cudaSuccess ||
      cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess ||
      cudaStreamCreateWithPriority(&h->own, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->order_ev, cudaEventDisableTiming) != cudaSuccess) {
    g_create_error = "CUDA context or stream creation failed";
    lbm_destroy(h);
    return LBM_ECUDA;
  }
  h->st = h->own;
  {
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->dev) == cudaSuccess && nsm > 0)
      h->grid_cap = 8 * nsm;
  }
  const size_t pops = (size_t)h->S * Q * N * h->esize;
  for (int k = 0; k < 2 && s == LBM_OK; ++k) {
    if (cudaMalloc(&h->f[k], pops) != cudaSuccess) {
      cudaGetLastError();
      s = LBM_ENOMEM;
    } else {
      cudaMemset(h->f[k], 0, pops);
    }
  }
  if (s == LBM_OK) s = dev_alloc(h, &h->dred, (MAX_SPECIES + 4) * DIAG_SPREAD);
  // diagnostics partials for the smallest CTA size the stream/collide uses (64)
  if (s == LBM_OK) s = dev_alloc(h, &h->dpart, (size_t)((N + 63) / 64) * DIAG_NQ);
  if (s == LBM_OK) s = dev_alloc(h, &h->dmid, (size_t)DIAG_NQ * 64);
  if (s == LBM_OK) s = dev_alloc(h, &h->ddone, 1);
  if (s == LBM_OK) cudaMemset(h->ddone, 0, sizeof(unsigned));
  if (s == LBM_OK) s = dev_alloc(h, &h->dflag, 1);
  if (s == LBM_OK && cudaMallocHost(&h->hred, (MAX_SPECIES + 4) * DIAG_SPREAD * sizeof(double)) != cudaSuccess)
    s = LBM_ENOMEM;
  if (s == LBM_OK && c.bjerrum > 0.0) {
    s = dev_alloc(h, &h->ps.psi[0], N);
    if (s == LBM_OK) s = dev_alloc(h, &h->ps.psi[1], N);
    if (s == LBM_OK) s = dev_alloc(h, &h->ps.src, N);
    // the charge scatter: FP32 storage (for 16-bit storage the pass is
    // faster: its stream/collide is bound by instruction issue, and the
    // scatter's instructions cost more than the pass), periodic (walls may
    // still come, lbm_set_walls turns it off), x rows of whole warps
    h->scat_on = !(c.flags & LBM_FLAG_CHARGE_PASS) && c.storage == LBM_FP32 && c.nx % 32 == 0;
    if (s == LBM_OK && h->scat_on) {
      s = dev_alloc(h, &h->scat_acc, N);
      if (s == LBM_OK) s = dev_alloc(h, &h->scat_tot, 3);
      if (s == LBM_OK) {
        cudaMemset(h->scat_acc, 0, N * sizeof(int64_t));
        cudaMemset(h->scat_tot, 0, 3 * sizeof(unsigned long long));
      }
    }
    if (s == LBM_OK) s = dev_alloc(h, &h->ps.dsum, 1 + 2 * Poisson::NSLOT);
    if (s == LBM_OK) s = dev_alloc(h, &h->ps.part, (size_t)((N + 63) / 64));
    if (s == LBM_OK && cudaMallocHost(&h->ps.hsum, (1 + 2 * Poisson::NSLOT) * sizeof(double)) != cudaSuccess)
      s = LBM_ENOMEM;
    if (s == LBM_OK) {
      cudaMemset(h->ps.psi[0], 0, N * sizeof(int64_t));
      cudaMemset(h->ps.psi[1], 0, N * sizeof(int64_t));
      cudaMemset(h->ps.dsum, 0, (1 + 2 * Poisson::NSLOT) * sizeof(double));
      s = poisson_setup(h, nullptr);
      if (s == LBM_OK) s = start_setup(h);
      if (s == LBM_OK && c.poisson == LBM_POISSON_FFT) s = spectral_setup(h, nullptr);
    }
  }
  if (s == LBM_OK && cudaDeviceSynchronize() != cudaSuccess) s = LBM_ECUDA;
  if (s != LBM_OK) {
    g_create_error = h->err.empty() ? "device allocation failed" : h->err;
    lbm_destroy(h);
    return s;
  }
  *out = h;
  return LBM_OK;
}

void lbm_destroy(lbm_t* h) {
  if (!h) return;
  cudaSetDevice(h->dev);
  if (h->own) cudaStreamSynchronize(h->own);
  cudaFree(h->f[0]);
  cudaFree(h->f[1]);
  cudaFree(h->scat_acc);
  cudaFree(h->scat_tot);
  cudaFree(h->links);
  cudaFree(h->wallq);
  cudaFree(h->wsrc);
  cudaFree(h->dred);
  if (h->hrec) cudaFreeHost(h->hrec);
  cudaFree(h->dpart);
  cudaFree(h->dmid);
  cudaFree(h->ddone);
  cudaFree(h->dflag);
  if (h->hred) cudaFreeHost(h->hred);
  spectral_graph_free(h);
  poisson_free(h);
  spectral_free(h);
  start_free(h);
  nn_free(h);
  cudaFree(h->omega_drag_z);
  cudaFree(h->gstatus);
  if (h->hstatus) cudaFreeHost(h->hstatus);
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  if (h->order_ev) cudaEventDestroy(h->order_ev);
  if (h->own) cudaStreamDestroy(h->own);
  delete h;
}

lbm_status lbm_set_walls(lbm_t* h, const uint8_t* solid, const double* sigma) {
  if (!h) return LBM_EINVAL;
  if (!solid) return fail(h, LBM_EINVAL, "solid mask is NULL");
  if (h->species_set) return fail(h, LBM_EINVAL, "walls must be set before any species");
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, own_stream(h));  // calls without a stream argument use the library's stream
  const int nx = h->cfg.nx, ny = h->cfg.ny, nz = h->cfg.nz;
  const int64_t N = h->N;
  int64_t nfluid = 0;
  for (int64_t i = 0; i < N; ++i) nfluid += solid[i] ? 0 : 1;
  if (nfluid == 0) return fail(h, LBM_EINVAL, "every node is a wall node");
  // Face charge share q_j = sigma_j / k_j of each wall node (k_j = number of
  // fluid face neighbours) and the wall charge w_i handed to each fluid cell.
  std::vector<float> q(N, 0.f);
  std::vector<double> qd(N, 0.0), wd(N, 0.0);
  auto idx = [&](int x, int y, int z) -> int64_t {
    x = (x + nx) % nx;
    y = (y + ny) % ny;
    z = (z + nz) % nz;
    return ((int64_t)z * ny + y) * nx + x;
  };
  const int fd[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
  bool charged_walls = false;
  if (sigma) {
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          const int64_t i = idx(x, y, z);
          if (!solid[i] || sigma[i] == 0.0) continue;
          if (!isfinite(sigma[i])) return fail(h, LBM_EINVAL, "sigma is not finite");
          int k = 0;
          for (auto& d : fd)
            if (!solid[idx(x + d[0], y + d[1], z + d[2])]) ++k;
          if (k == 0) continue;
          qd[i] = sigma[i] / k;
          q[i] = (float)qd[i];
          charged_walls = true;
        }
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          const int64_t i = idx(x, y, z);
          if (solid[i]) continue;
          double acc = 0.0;
          for (auto& d : fd) {
            const int64_t j = idx(x + d[0], y + d[1], z + d[2]);
            if (solid[j]) acc += qd[j];
          }
          wd[i] = acc;
        }
  }
  Scratch sc;
  if (cudaMalloc(&sc.p, N) != cudaSuccess) return fail(h, LBM_ENOMEM, "scratch allocation failed");
  lbm_status s = LBM_OK;
  if (!h->links) s = dev_alloc(h, &h->links, N);
  if (s != LBM_OK) return s;
  LBM_CUDA_TRY(h, cudaMemcpy(sc.p, solid, N, cudaMemcpyHostToDevice));
  h->has_walls = true;
  h->scat_on = false;  // the charge pass handles walls
  h->scat_valid = false;
  LBM_CUDA_TRY(h, launch_links(h, (const uint8_t*)sc.p));
  if (charged_walls) {
    if (!h->wallq && (s = dev_alloc(h, &h->wallq, N)) != LBM_OK) return s;
    if (!h->wsrc && (s = dev_alloc(h, &h->wsrc, N)) != LBM_OK) return s;
    std::vector<int64_t> wfx(N, 0);
    const double k4 = 4.0 * 3.14159265358979323846 * h->cfg.bjerrum;
    for (int64_t i = 0; i < N; ++i) wfx[i] = llrint(k4 * wd[i] * PSI_SCALE);
    LBM_CUDA_TRY(h, cudaMemcpy(h->wallq, q.data(), N * sizeof(float), cudaMemcpyHostToDevice));
    LBM_CUDA_TRY(h, cudaMemcpy(h->wsrc, wfx.data(), N * sizeof(int64_t), cudaMemcpyHostToDevice));
  } else {
    cudaFree(h->wallq);
    cudaFree(h->wsrc);
    h->wallq = nullptr;
    h->wsrc = nullptr;
  }
  h->nfluid = nfluid;
  if (h->cfg.bjerrum > 0.0) {
    h->ps.nfluid = nfluid;
    // connected fluid components over face neighbours (periodic): each is a
    // separate Poisson domain with its own neutralising mean (the spectral
    // solver takes the mean per run of fluid planes instead)
    std::vector<int> lab(h->cfg.poisson == LBM_POISSON_FFT ? 0 : N, -1);
    std::vector<long long> sizes;
    std::vector<int64_t> stack;
    for (int64_t i0 = 0; i0 < (int64_t)lab.size(); ++i0) {
      if (solid[i0] || lab[i0] >= 0) continue;
      const int c = (int)sizes.size();
      long long cnt = 0;
      lab[i0] = c;
      stack.push_back(i0);
      while (!stack.empty()) {
        const int64_t i = stack.back();
        stack.pop_back();
        ++cnt;
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
        for (auto& d : fd) {
          const int64_t j = idx(x + d[0], y + d[1], z + d[2]);
          if (!solid[j] && lab[j] < 0) {
            lab[j] = c;
            stack.push_back(j);
          }
        }
      }
      sizes.push_back(cnt);
    }
    Poisson& P = h->ps;
    cudaFree(P.label);
    cudaFree(P.comp_sum);
    cudaFree(P.comp_size);
    cudaFree(P.comp_mean);
    P.label = nullptr;
    P.comp_sum = nullptr;
    P.comp_size = nullptr;
    P.comp_mean = nullptr;
    P.ncomp = (int)sizes.size();
    if (P.ncomp > 1) {
      // relabel so that the largest component is 0
      int big = 0;
      for (int c = 1; c < P.ncomp; ++c)
        if (sizes[c] > sizes[big]) big = c;
      for (int64_t i = 0; i < N; ++i) {
        if (lab[i] == big) lab[i] = 0;
        else if (lab[i] == 0) lab[i] = big;
      }
      std::swap(sizes[0], sizes[big]);
      if ((s = dev_alloc(h, &P.label, N)) != LBM_OK) return s;
      if ((s = dev_alloc(h, &P.comp_sum, P.ncomp)) != LBM_OK) return s;
      if ((s = dev_alloc(h, &P.comp_size, P.ncomp)) != LBM_OK) return s;
      if ((s = dev_alloc(h, &P.comp_mean, P.ncomp)) != LBM_OK) return s;
      for (int64_t i = 0; i < N; ++i)
        if (lab[i] < 0) lab[i] = 0;  // wall nodes: unused
      LBM_CUDA_TRY(h, cudaMemcpy(P.label, lab.data(), N * sizeof(int), cudaMemcpyHostToDevice));
      LBM_CUDA_TRY(h, cudaMemcpy(P.comp_size, sizes.data(), P.ncomp * sizeof(long long),
                                 cudaMemcpyHostToDevice));
    }
    s = poisson_setup(h, solid);
    if (s != LBM_OK) return s;
    if (h->cfg.poisson == LBM_POISSON_FFT && (s = spectral_setup(h, solid)) != LBM_OK) return s;
  }
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  LBM_CUDA_TRY(h, cudaDeviceSynchronize());
  return LBM_OK;
}

lbm_status lbm_set_species(lbm_t* h, int s, double mass, double valence,
                           const double* n0, const double* u0) {
  lbm_status sa = species_args(h, s, mass, valence, n0);
  if (sa != LBM_OK) return sa;
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, own_stream(h));  // calls without a stream argument use the library's stream
  const int64_t N = h->N;
  // host checks and the reference density of the 16-bit shifted storage
  std::vector<uint8_t> solid;
  if (h->has_walls) {
    std::vector<uint32_t> lk(N);
    LBM_CUDA_TRY(h, cudaMemcpy(lk.data(), h->links, N * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    solid.resize(N);
    for (int64_t i = 0; i < N; ++i) solid[i] = (lk[i] & LINK_SOLID) ? 1 : 0;
  }
  double tot = 0.0;
  int64_t cnt = 0;
  for (int64_t i = 0; i < N; ++i) {
    if (!solid.empty() && solid[i]) continue;
    if (!(n0[i] > 0.0) || !isfinite(n0[i]))
      return fail(h, LBM_EINVAL, "n0 must be finite and > 0 at every fluid node");
    if (u0 && (!isfinite(u0[i]) || !isfinite(u0[N + i]) || !isfinite(u0[2 * N + i])))
      return fail(h, LBM_EINVAL, "u0 must be finite");
    tot += n0[i];
    ++cnt;
  }
  h->nref[s] = (float)(tot / (double)cnt);
  Scratch sc;
  const size_t bytes = (size_t)N * sizeof(double) * (u0 ? 4 : 1);
  if (cudaMalloc(&sc.p, bytes) != cudaSuccess) return fail(h, LBM_ENOMEM, "scratch allocation failed");
  double* dn = (double*)sc.p;
  double* du = u0 ? dn + N : nullptr;
  LBM_CUDA_TRY(h, cudaMemcpy(dn, n0, N * sizeof(double), cudaMemcpyHostToDevice));
  if (u0) LBM_CUDA_TRY(h, cudaMemcpy(du, u0, 3 * N * sizeof(double), cudaMemcpyHostToDevice));
  LBM_CUDA_TRY(h, launch_init_species(h, s, dn, du));
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return species_done(h, s, mass, valence);
}

lbm_status lbm_set_species_dev(lbm_t* h, int s, double mass, double valence,
                               const double* n0_arg, const double* u0_arg, void* stream) {
  lbm_status st = species_args(h, s, mass, valence, n0_arg);
  if (st != LBM_OK) return st;
  cudaSetDevice(h->dev);
  void *n0v = nullptr, *u0v = nullptr;
  if ((st = device_view(h, n0_arg, &n0v, "n0_dev")) != LBM_OK) return st;
  if ((st = device_view(h, u0_arg, &u0v, "u0_dev")) != LBM_OK) return st;
  const double* n0_dev = static_cast<const double*>(n0v);
  const double* u0_dev = static_cast<const double*>(u0v);
  CallStream cs(h, stream);
  LBM_CUDA_TRY(h, cs.err);
  // fluid-node sum of n0 (the reference density) and a count of invalid
  // entries, per CTA, summed on the host in a fixed order
  int nb = 0;
  LBM_CUDA_TRY(h, launch_species_check(h, n0_dev, u0_dev, h->dred, &nb));
  LBM_CUDA_TRY(h, cudaMemcpyAsync(h->hred, h->dred, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost,
                                  h->st));
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  double tot = 0.0, bad = 0.0;
  for (int b = 0; b < nb; ++b) {
    tot += h->hred[2 * b];
    bad += h->hred[2 * b + 1];
  }
  if (bad != 0.0)
    return fail(h, LBM_EINVAL, "n0 must be finite and > 0 at every fluid node, u0 finite");
  h->nref[s] = (float)(tot / (double)h->nfluid);
  LBM_CUDA_TRY(h, launch_init_species(h, s, n0_dev, u0_dev));
  return species_done(h, s, mass, valence);
}

lbm_status lbm_get_moments_dev(lbm_t* h, int s, double* n_arg, double* u_arg, void* stream) {
  if (!h) return LBM_EINVAL;
  if (s < 0 || s >= h->S) return fail(h, LBM_EINVAL, "species index out of range");
  if (!(h->species_set >> s & 1u)) return fail(h, LBM_EINVAL, "species not set");
  if (!n_arg && !u_arg) return LBM_OK;
  cudaSetDevice(h->dev);
  void *nv = nullptr, *uv = nullptr;
  lbm_status st = device_view(h, n_arg, &nv, "n_dev");
  if (st == LBM_OK) st = device_view(h, u_arg, &uv, "u_dev");
  if (st != LBM_OK) return st;
  double* n_dev = static_cast<double*>(nv);
  double* u_dev = static_cast<double*>(uv);
  CallStream cs(h, stream);
  LBM_CUDA_TRY(h, cs.err);
  LBM_CUDA_TRY(h, launch_gather(h, s, n_dev, u_dev, nullptr));
  return LBM_OK;
}

double lbm_omega_drag_for_schmidt(double omega_visc, double schmidt) {
  // Sc = nu / D with nu = c_s^2 (1/omega_visc - 1/2) and
  // D = c_s^2 (1/omega_drag - 1/2) (Sec. 4)
  if (!(omega_visc > 0.0 && omega_visc < 2.0) || !(schmidt > 0.0) || !isfinite(schmidt)) return 0.0;
  return 1.0 / (0.5 + (1.0 / omega_visc - 0.5) / schmidt);
}

}  // extern "C"

namespace {

// The steps of lbm_step / lbm_step_record on the library's stream (the
// caller's stream is ordered by the entry point).  While a recording call
// steps (h->rec_dev set), every step sums the state it stores and its
// record goes to slot k of the call's chunk.
lbm_status step_impl(lbm_t* h, int nsteps) {
  const bool charged = h->cfg.bjerrum > 0.0;
  if (h->cfg.flags & LBM_FLAG_STEP_GRAPH) {
    Phase pg(h, 1);
    lbm_status s = spectral_graph_steps(h, nsteps);
    LBM_CUDA_TRY(h, pg.stop());
    return s;
  }
  // bound the number of outstanding timing events
  if (h->timing && h->ev_used > 4096) LBM_CUDA_TRY(h, drain_timing(h));
  for (int k = 0; k < nsteps; ++k) {
    lbm_status s = LBM_OK;
    if (charged) {
      Phase pc(h, 0);
      LBM_CUDA_TRY(h, cudaMemsetAsync(h->ps.dsum, 0, 3 * sizeof(double), h->st));
      if (h->ps.comp_sum)
        LBM_CUDA_TRY(h, cudaMemsetAsync(h->ps.comp_sum, 0, h->ps.ncomp * sizeof(long long), h->st));
      LBM_CUDA_TRY(h, launch_charge(h));
      LBM_CUDA_TRY(h, pc.stop());
      h->t_cnt[0] += 1;
      int it = 0;
      double rel = 0.0;
      Phase pp(h, 1);
      // spectral: the start from the previous fit, this step's fit beside
      // the solve (joined before the next step); multigrid / SOR: the fit
      // first
      LBM_CUDA_TRY(h, start_step(h, h->spec != nullptr));
      s = poisson_solve(h, h->cfg.poisson_tol, h->cfg.poisson_maxit, &it, &rel);
      LBM_CUDA_TRY(h, pp.stop());
      h->t_cnt[1] += it;
      h->last_iters = it;
      h->last_res = rel;
      if (s != LBM_OK && s != LBM_ENOCONV) return s;
      h->psi_valid = true;
    }
    Phase ps(h, 2);
    // the last step of the call also sums the state it stores (diagnostics)
    LBM_CUDA_TRY(h, launch_stream_collide(h, h->rec_dev != nullptr || k == nsteps - 1));
    LBM_CUDA_TRY(h, ps.stop());
    LBM_CUDA_TRY(h, start_join(h));
    h->t_cnt[2] += 1;
    ++h->tstep;
    if (h->rec_dev) {
      // the sums straight into the host slot; the Poisson figures are known
      // here
      LBM_CUDA_TRY(h, launch_diag_reduce(h, h->rec_dev + (size_t)k * REC_LEN));
      double* hslot = h->rec_host + (size_t)k * REC_LEN;
      hslot[DIAG_NQ] = charged ? (double)h->last_iters : 0.0;
      hslot[DIAG_NQ + 1] = charged ? h->last_res : 0.0;
    }
    if (s == LBM_ENOCONV) return s;
  }
  if (h->timing && h->ev_used > 4096) LBM_CUDA_TRY(h, drain_timing(h));
  return LBM_OK;
}

// The diagnostics of lbm_diagnostics from the deviation sums (DIAG_NQ
// layout: species, momentum x y z, charge, bad flag).  Returns whether a
// value is not finite or the flag is set.
bool diag_from_sums(const lbm_t* h, const double* sums, double iters, double rel, double steps,
                    double* out) {
  const int S = h->S;
  const double nf = (double)h->nfluid;
  double zref = 0.0;
  bool bad = sums[MAX_SPECIES + 4] != 0.0;
  for (int s = 0; s < S; ++s) {
    out[s] = nf * (double)h->nref[s] + sums[s];
    zref += (double)h->valence[s] * (double)h->nref[s];
  }
  for (int d = 0; d < 3; ++d) out[S + d] = h->mass0 * sums[MAX_SPECIES + d];
  out[S + 3] = nf * zref + sums[MAX_SPECIES + 3];
  out[S + 4] = iters;
  out[S + 5] = rel;
  out[S + 6] = steps;
  for (int k = 0; k < S + 4; ++k) bad = bad || !isfinite(out[k]);
  return bad;
}

}  // namespace

extern "C" {

lbm_status lbm_step(lbm_t* h, int nsteps, void* stream) {
  if (!h) return LBM_EINVAL;
  if (nsteps < 0) return fail(h, LBM_EINVAL, "nsteps must be >= 0");
  if (!species_complete(h)) return fail(h, LBM_EINVAL, "every species must be set before stepping");
  cudaSetDevice(h->dev);
  CallStream cs(h, stream);
  LBM_CUDA_TRY(h, cs.err);
  return step_impl(h, nsteps);
}

lbm_status lbm_step_record(lbm_t* h, int nsteps, double* out, void* stream) {
  if (!h) return LBM_EINVAL;
  if (nsteps < 0) return fail(h, LBM_EINVAL, "nsteps must be >= 0");
  if (nsteps > 0 && !out) return fail(h, LBM_EINVAL, "out is NULL");
  if (!species_complete(h)) return fail(h, LBM_EINVAL, "every species must be set before stepping");
  cudaSetDevice(h->dev);
  CallStream cs(h, stream);
  LBM_CUDA_TRY(h, cs.err);
  const int want = std::min(nsteps, REC_CHUNK);
  if (want > h->rec_cap) {
    if (h->hrec) cudaFreeHost(h->hrec);
    h->hrec = nullptr;
    h->hrec_dev = nullptr;
    h->rec_cap = 0;
    void* dp = nullptr;
    if (cudaHostAlloc(&h->hrec, (size_t)want * REC_LEN * sizeof(double), cudaHostAllocMapped) !=
            cudaSuccess ||
        cudaHostGetDevicePointer(&dp, h->hrec, 0) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, LBM_ENOMEM, "record buffer allocation failed");
    }
    h->hrec_dev = static_cast<double*>(dp);
    h->rec_cap = want;
  }
  const int L = LBM_DIAG_LEN(h->S);
  bool bad = false;
  int done = 0;
  while (done < nsteps) {
    const int n = std::min(h->rec_cap, nsteps - done);
    const int64_t t0 = h->tstep;
    h->rec_dev = h->hrec_dev;
    h->rec_host = h->hrec;
    const lbm_status s = step_impl(h, n);
    h->rec_dev = nullptr;
    h->rec_host = nullptr;
    // the steps taken (all n unless one failed) and their records
    const int m = (int)(h->tstep - t0);
    LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
    for (int k = 0; k < m; ++k) {
      const double* r = h->hrec + (size_t)k * REC_LEN;
      bad = diag_from_sums(h, r, r[DIAG_NQ], r[DIAG_NQ + 1], (double)(t0 + k + 1),
                           out + (size_t)(done + k) * L) || bad;
    }
    done += m;
    if (s != LBM_OK) return s;
    if (m < n) break;
  }
  if (bad) return fail(h, LBM_EUNSTABLE, "non-finite or non-positive density detected");
  return LBM_OK;
}

lbm_status lbm_synchronize(lbm_t* h) {
  if (!h) return LBM_EINVAL;
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->own));
  return LBM_OK;
}

lbm_status lbm_get_moments(lbm_t* h, int s, double* n, double* u) {
  if (!h) return LBM_EINVAL;
  if (s < 0 || s >= h->S) return fail(h, LBM_EINVAL, "species index out of range");
  if (!(h->species_set >> s & 1u)) return fail(h, LBM_EINVAL, "species not set");
  if (!n && !u) return LBM_OK;
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, own_stream(h));  // calls without a stream argument use the library's stream
  const int64_t N = h->N;
  Scratch sc;
  if (cudaMalloc(&sc.p, 4 * N * sizeof(double)) != cudaSuccess)
    return fail(h, LBM_ENOMEM, "scratch allocation failed");
  double* dn = (double*)sc.p;
  double* du = dn + N;
  LBM_CUDA_TRY(h, launch_gather(h, s, dn, du, nullptr));
  if (n) LBM_CUDA_TRY(h, cudaMemcpyAsync(n, dn, N * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  if (u) LBM_CUDA_TRY(h, cudaMemcpyAsync(u, du, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return LBM_OK;
}

lbm_status lbm_plane_fluxes(lbm_t* h, double* out) {
  if (!h || !out) return LBM_EINVAL;
  if (!species_complete(h)) return fail(h, LBM_EINVAL, "every species must be set first");
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, own_stream(h));  // calls without a stream argument use the library's stream
  const size_t len = (size_t)h->cfg.nz * h->S * 4;
  Scratch sc;
  if (cudaMalloc(&sc.p, len * sizeof(double)) != cudaSuccess)
    return fail(h, LBM_ENOMEM, "scratch allocation failed");
  LBM_CUDA_TRY(h, launch_plane_fluxes(h, (double*)sc.p));
  LBM_CUDA_TRY(h, cudaMemcpyAsync(out, sc.p, len * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return LBM_OK;
}

lbm_status lbm_get_populations(lbm_t* h, int s, double* f) {
  if (!h) return LBM_EINVAL;
  if (s < 0 || s >= h->S || !f) return fail(h, LBM_EINVAL, "bad species index or NULL buffer");
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, own_stream(h));  // calls without a stream argument use the library's stream
  const int64_t N = h->N;
  Scratch sc;
  if (cudaMalloc(&sc.p, (size_t)Q * N * sizeof(double)) != cudaSuccess)
    return fail(h, LBM_ENOMEM, "scratch allocation failed");
  LBM_CUDA_TRY(h, launch_gather(h, s, nullptr, nullptr, (double*)sc.p));
  LBM_CUDA_TRY(h, cudaMemcpyAsync(f, sc.p, (size_t)Q * N * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return LBM_OK;
}

lbm_status lbm_get_potential(lbm_t* h, double* psi) {
  if (!h || !psi) return LBM_EINVAL;
  if (!(h->cfg.bjerrum > 0.0)) return fail(h, LBM_EINVAL, "neutral lattice has no potential");
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, own_stream(h));  // calls without a stream argument use the library's stream
  const int64_t N = h->N;
  Scratch sc;
  if (cudaMalloc(&sc.p, N * sizeof(double)) != cudaSuccess)
    return fail(h, LBM_ENOMEM, "scratch allocation failed");
  LBM_CUDA_TRY(h, launch_psi_to_double(h, h->ps.psi[h->ps.cur], (double*)sc.p));
  LBM_CUDA_TRY(h, cudaMemcpyAsync(psi, sc.p, N * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return LBM_OK;
}

lbm_status lbm_solve_poisson(lbm_t* h, const double* rho_e, double* psi,
                             double tol, int maxit, int* iters, double* rel_res) {
  if (!h) return LBM_EINVAL;
  if (!(h->cfg.bjerrum > 0.0)) return fail(h, LBM_EINVAL, "requires bjerrum > 0");
  if (!rho_e || !psi) return fail(h, LBM_EINVAL, "NULL buffer");
  if (!(tol > 0.0)) return fail(h, LBM_EINVAL, "tol must be > 0");
  if (maxit <= 0) maxit = h->cfg.poisson_maxit;
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, own_stream(h));  // calls without a stream argument use the library's stream
  const int64_t N = h->N;
  for (int64_t i = 0; i < N; ++i)
    if (!isfinite(rho_e[i]) || !isfinite(psi[i]) || fabs(psi[i]) >= PSI_MAX)
      return fail(h, LBM_EINVAL, "rho_e and psi must be finite, |psi| < 2048");
  Scratch sc;
  if (cudaMalloc(&sc.p, 2 * N * sizeof(double)) != cudaSuccess)
    return fail(h, LBM_ENOMEM, "scratch allocation failed");
  double* drho = (double*)sc.p;
  double* dpsi = drho + N;
  LBM_CUDA_TRY(h, cudaMemcpyAsync(drho, rho_e, N * sizeof(double), cudaMemcpyHostToDevice, h->st));
  LBM_CUDA_TRY(h, cudaMemcpyAsync(dpsi, psi, N * sizeof(double), cudaMemcpyHostToDevice, h->st));
  LBM_CUDA_TRY(h, cudaMemsetAsync(h->ps.dsum, 0, 3 * sizeof(double), h->st));
  if (h->ps.comp_sum)
    LBM_CUDA_TRY(h, cudaMemsetAsync(h->ps.comp_sum, 0, h->ps.ncomp * sizeof(long long), h->st));
  LBM_CUDA_TRY(h, launch_src_from_rho(h, drho));
  LBM_CUDA_TRY(h, launch_psi_from_double(h, dpsi, h->ps.psi[h->ps.cur]));
  int it = 0;
  double rel = 0.0;
  lbm_status s = poisson_solve(h, tol, maxit, &it, &rel);
  if (iters) *iters = it;
  if (rel_res) *rel_res = rel;
  if (s != LBM_OK && s != LBM_ENOCONV) return s;
  const lbm_status sr = potential_history_reset(h);
  if (sr != LBM_OK) return sr;
  LBM_CUDA_TRY(h, launch_psi_to_double(h, h->ps.psi[h->ps.cur], dpsi));
  LBM_CUDA_TRY(h, cudaMemcpyAsync(psi, dpsi, N * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return s;
}

lbm_status lbm_diagnostics(lbm_t* h, double* out) {
  if (!h || !out) return LBM_EINVAL;
  if (!species_complete(h)) return fail(h, LBM_EINVAL, "every species must be set first");
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, own_stream(h));  // calls without a stream argument use the library's stream
  // deviation sums: species masses, momentum x, y, z, charge
  double sums[MAX_SPECIES + 4];
  bool bad = false;
  if (h->diag_valid) {
    // the last stream/collide launch summed the state it wrote, per CTA
    LBM_CUDA_TRY(h, launch_diag_reduce(h, h->dred));
    LBM_CUDA_TRY(h, cudaMemcpyAsync(h->hred, h->dred, DIAG_NQ * sizeof(double),
                                    cudaMemcpyDeviceToHost, h->st));
    LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
    for (int k = 0; k < MAX_SPECIES + 4; ++k) sums[k] = h->hred[k];
    bad = h->hred[MAX_SPECIES + 4] != 0.0;
  } else {
    // a full pass over the populations of the current state
    LBM_CUDA_TRY(h, cudaMemsetAsync(h->dred, 0, (MAX_SPECIES + 4) * DIAG_SPREAD * sizeof(double), h->st));
    LBM_CUDA_TRY(h, cudaMemsetAsync(h->dflag, 0, sizeof(int), h->st));
    LBM_CUDA_TRY(h, launch_diagnostics(h));
    LBM_CUDA_TRY(h, cudaMemcpyAsync(h->hred, h->dred, (MAX_SPECIES + 4) * DIAG_SPREAD * sizeof(double),
                                    cudaMemcpyDeviceToHost, h->st));
    int flag = 0;
    LBM_CUDA_TRY(h, cudaMemcpyAsync(&flag, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
    // the kernel sums deviations from n_ref into DIAG_SPREAD partials per
    // quantity
    for (int k = 0; k < MAX_SPECIES + 4; ++k) {
      double t = 0.0;
      for (int j = 0; j < DIAG_SPREAD; ++j) t += h->hred[k * DIAG_SPREAD + j];
      sums[k] = t;
    }
    bad = flag != 0;
  }
  // the reference parts n_ref x fluid nodes are exact
  double full[DIAG_NQ];
  for (int k = 0; k < MAX_SPECIES + 4; ++k) full[k] = sums[k];
  full[MAX_SPECIES + 4] = bad ? 1.0 : 0.0;
  bad = diag_from_sums(h, full, (double)h->last_iters, h->last_res, (double)h->tstep, out);
  if (bad) return fail(h, LBM_EUNSTABLE, "non-finite or non-positive density detected");
  return LBM_OK;
}

lbm_status lbm_get_state(lbm_t* h, float* state, int64_t* step) {
  if (!h || !state) return LBM_EINVAL;
  if (h->cfg.storage != LBM_FP32)
    return fail(h, LBM_EINVAL, "raw state access needs FP32 storage");
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, own_stream(h));  // calls without a stream argument use the library's stream
  LBM_CUDA_TRY(h, cudaMemcpyAsync(state, h->f[h->cur], (size_t)h->S * Q * h->N * sizeof(float),
                                  cudaMemcpyDeviceToHost, h->st));
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  if (step) *step = h->tstep;
  return LBM_OK;
}

lbm_status lbm_set_state(lbm_t* h, const float* state, int64_t step) {
  if (!h || !state) return LBM_EINVAL;
  if (h->cfg.storage != LBM_FP32)
    return fail(h, LBM_EINVAL, "raw state access needs FP32 storage");
  if (!species_complete(h)) return fail(h, LBM_EINVAL, "every species must be set first");
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, own_stream(h));  // calls without a stream argument use the library's stream
  LBM_CUDA_TRY(h, cudaMemcpyAsync(h->f[h->cur], state, (size_t)h->S * Q * h->N * sizeof(float),
                                  cudaMemcpyHostToDevice, h->st));
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  h->tstep = step;
  h->diag_valid = false;
  h->scat_valid = false;
  return potential_history_reset(h);
}

lbm_status lbm_create_stack(int count, const lbm_config* cfgs, lbm_t** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (count < 1 || !cfgs) {
    g_create_error = "count must be >= 1 and cfgs non-NULL";
    return LBM_EINVAL;
  }
  lbm_config c = cfgs[0];
  int64_t nz = 0;
  for (int i = 0; i < count; ++i) {
    const lbm_config& k = cfgs[i];
    if (k.nx != c.nx || k.ny != c.ny || k.nspecies != c.nspecies || k.omega_visc != c.omega_visc ||
        k.bjerrum != c.bjerrum || k.e_ext[0] != c.e_ext[0] || k.e_ext[1] != c.e_ext[1] ||
        k.e_ext[2] != c.e_ext[2] || k.storage != c.storage || k.poisson != c.poisson ||
        k.poisson_tol != c.poisson_tol || k.poisson_maxit != c.poisson_maxit ||
        k.device != c.device || k.flags != c.flags) {
      g_create_error = "stacked instances must share every field but nz and omega_drag";
      return LBM_EINVAL;
    }
    if (k.nz < 1 || !(k.omega_drag > 0.0 && k.omega_drag < 2.0)) {
      g_create_error = "instance nz must be >= 1 and omega_drag in (0, 2)";
      return LBM_EINVAL;
    }
    nz += k.nz;
  }
  if (nz > (1 << 30)) {
    g_create_error = "stack too tall";
    return LBM_EINVAL;
  }
  c.nz = (int)nz;
  lbm_t* h = nullptr;
  lbm_status s = lbm_create(&c, &h);
  if (s != LBM_OK) return s;
  std::vector<double> om;
  om.reserve(nz);
  h->instance_z0.clear();
  for (int i = 0; i < count; ++i) {
    h->instance_z0.push_back((int)om.size());
    for (int z = 0; z < cfgs[i].nz; ++z) om.push_back(cfgs[i].omega_drag);
  }
  s = lbm_set_plane_omega_drag(h, om.data());
  if (s != LBM_OK) {
    g_create_error = h->err;
    lbm_destroy(h);
    return s;
  }
  *out = h;
  return LBM_OK;
}

int lbm_instance_z0(const lbm_t* h, int i) {
  if (!h) return -1;
  if (h->instance_z0.empty()) return i == 0 ? 0 : -1;
  if (i < 0 || i >= (int)h->instance_z0.size()) return -1;
  return h->instance_z0[i];
}

lbm_status lbm_set_plane_omega_drag(lbm_t* h, const double* omega) {
  if (!h) return LBM_EINVAL;
  cudaSetDevice(h->dev);
  if (!omega) {
    cudaFree(h->omega_drag_z);
    h->omega_drag_z = nullptr;
    spectral_graph_free(h);
    return LBM_OK;
  }
  if (h->pair_on)
    return fail(h, LBM_EINVAL, "a drag matrix and per-plane drag frequencies exclude each other");
  const int nz = h->cfg.nz;
  std::vector<float> w(nz);
  for (int z = 0; z < nz; ++z) {
    if (!(omega[z] > 0.0 && omega[z] < 2.0)) return fail(h, LBM_EINVAL, "omega_drag must lie in (0, 2)");
    w[z] = (float)omega[z];
  }
  if (!h->omega_drag_z) {
    lbm_status s = dev_alloc(h, &h->omega_drag_z, nz);
    if (s != LBM_OK) return s;
  }
  LBM_CUDA_TRY(h, cudaMemcpy(h->omega_drag_z, w.data(), nz * sizeof(float), cudaMemcpyHostToDevice));
  spectral_graph_free(h);
  return LBM_OK;
}

lbm_status lbm_set_drag_matrix(lbm_t* h, const double* omega) {
  if (!h) return LBM_EINVAL;
  const int S = h->S;
  if (!omega) {
    if (h->pair_on || h->cfg.omega_drag != h->omega_drag_cfg) spectral_graph_free(h);
    h->pair_on = false;
    h->cfg.omega_drag = h->omega_drag_cfg;
    return LBM_OK;
  }
  if (h->omega_drag_z)
    return fail(h, LBM_EINVAL, "a drag matrix and per-plane drag frequencies exclude each other");
  for (int i = 0; i < S; ++i)
    for (int j = 0; j < S; ++j) {
      if (i == j) continue;
      const double w = omega[i * S + j];
      if (!(w > 0.0 && w < 2.0)) return fail(h, LBM_EINVAL, "pair drag frequencies must lie in (0, 2)");
      if (fabs(w - omega[j * S + i]) > 1e-12 * w)
        return fail(h, LBM_EINVAL, "the drag matrix must be symmetric");
    }
  spectral_graph_free(h);
  if (S == 2) {
    // a binary depends on its cross frequency only: the scalar form
    h->pair_on = false;
    h->cfg.omega_drag = omega[1];
  } else if (S >= 3) {
    h->pair_on = true;
    for (int i = 0; i < MAX_SPECIES; ++i)
      for (int j = 0; j < MAX_SPECIES; ++j)
        h->pair[i][j] = (i < S && j < S && i != j) ? (float)omega[i * S + j] : 0.0f;
  }
  return LBM_OK;
}

lbm_status lbm_autotune(lbm_t* h, double* out) {
  if (!h) return LBM_EINVAL;
  if (!species_complete(h)) return fail(h, LBM_EINVAL, "every species must be set first");
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, own_stream(h));  // calls without a stream argument use the library's stream
  cudaEvent_t e0, e1;
  LBM_CUDA_TRY(h, cudaEventCreate(&e0));
  LBM_CUDA_TRY(h, cudaEventCreate(&e1));
  const int sizes[3] = {64, 128, 256};
  double best_c = 1e30, best_q = 1e30;
  int tc = h->collide_threads, tq = h->charge_threads;
  const int reps = 5;
  for (int k = 0; k < 3; ++k) {
    LBM_CUDA_TRY(h, launch_stream_collide_probe(h, sizes[k]));  // warm
    LBM_CUDA_TRY(h, cudaEventRecord(e0, h->st));
    for (int r = 0; r < reps; ++r) LBM_CUDA_TRY(h, launch_stream_collide_probe(h, sizes[k]));
    LBM_CUDA_TRY(h, cudaEventRecord(e1, h->st));
    LBM_CUDA_TRY(h, cudaEventSynchronize(e1));
    float ms = 0.f;
    LBM_CUDA_TRY(h, cudaEventElapsedTime(&ms, e0, e1));
    if (ms / reps < best_c) {
      best_c = ms / reps;
      tc = sizes[k];
    }
  }
  // (with the charge scatter the pass runs only after a restart, and the
  // step's source take would apply the potential's start on every timed
  // launch: nothing to time)
  if (h->cfg.bjerrum > 0.0 && !h->scat_on) {
    const int saved = h->charge_threads;
    for (int k = 0; k < 3; ++k) {
      h->charge_threads = sizes[k];
      LBM_CUDA_TRY(h, launch_charge(h));
      LBM_CUDA_TRY(h, cudaEventRecord(e0, h->st));
      for (int r = 0; r < reps; ++r) LBM_CUDA_TRY(h, launch_charge(h));
      LBM_CUDA_TRY(h, cudaEventRecord(e1, h->st));
      LBM_CUDA_TRY(h, cudaEventSynchronize(e1));
      float ms = 0.f;
      LBM_CUDA_TRY(h, cudaEventElapsedTime(&ms, e0, e1));
      if (ms / reps < best_q) {
        best_q = ms / reps;
        tq = sizes[k];
      }
    }
    h->charge_threads = saved;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->collide_threads = tc;
  h->charge_threads = tq;
  spectral_graph_free(h);  // graphs baked the old sizes
  h->psi_valid = false;
  h->scat_valid = false;  // the timed charge launches took the scattered source
  // (and, with the scatter, wrote source differences into the history)
  {
    lbm_status sr = potential_history_reset(h);
    if (sr != LBM_OK) return sr;
  }
  if (out) {
    out[0] = tc;
    out[1] = best_c;
    out[2] = tq;
    out[3] = best_q < 1e29 ? best_q : 0.0;
  }
  return LBM_OK;
}

lbm_status lbm_nn_init(lbm_t* h, int hidden, uint64_t seed) {
  if (!h) return LBM_EINVAL;
  if (!(h->cfg.bjerrum > 0.0)) return fail(h, LBM_EINVAL, "requires bjerrum > 0");
  if (h->cfg.flags & LBM_FLAG_STEP_GRAPH)
    return fail(h, LBM_EINVAL, "the learned guess runs in host-driven steps only");
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, own_stream(h));  // calls without a stream argument use the library's stream
  return nn_init(h, hidden, seed);
}

lbm_status lbm_nn_collect(lbm_t* h, int capacity) {
  if (!h) return LBM_EINVAL;
  cudaSetDevice(h->dev);
  return nn_collect(h, capacity);
}

lbm_status lbm_nn_train(lbm_t* h, int epochs, double lr, double* losses) {
  if (!h) return LBM_EINVAL;
  if (epochs < 0 || !(lr > 0.0)) return fail(h, LBM_EINVAL, "epochs >= 0 and lr > 0 required");
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, own_stream(h));  // calls without a stream argument use the library's stream
  return nn_train(h, epochs, lr, losses);
}

lbm_status lbm_nn_use(lbm_t* h, int enable) {
  if (!h) return LBM_EINVAL;
  return nn_set_use(h, enable);
}

lbm_status lbm_nn_params(lbm_t* h, float* get, const float* set, int* nparams) {
  if (!h) return LBM_EINVAL;
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, own_stream(h));  // calls without a stream argument use the library's stream
  return nn_params(h, get, set, nparams);
}

lbm_status lbm_nn_loss_grad(lbm_t* h, const float* x0, double* loss, float* grad) {
  if (!h || !x0 || !loss) return LBM_EINVAL;
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, own_stream(h));  // calls without a stream argument use the library's stream
  return nn_loss_grad_host(h, x0, loss, grad);
}

lbm_status lbm_nn_infer(lbm_t* h, const float* x0, float* y) {
  if (!h || !x0 || !y) return LBM_EINVAL;
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, own_stream(h));  // calls without a stream argument use the library's stream
  return nn_infer_host(h, x0, y);
}

lbm_status lbm_nn_stats(lbm_t* h, double* out) {
  if (!h || !out) return LBM_EINVAL;
  nn_stats(h, out);
  return LBM_OK;
}

lbm_status lbm_poisson_stats(lbm_t* h, double* out) {
  if (!h || !out) return LBM_EINVAL;
  out[0] = (double)h->last_iters;
  out[1] = h->last_start;
  out[2] = h->last_res;
  out[3] = (double)h->start_count;
  out[4] = h->start_count ? h->start_log_sum / (double)h->start_count : 0.0;
  return LBM_OK;
}

lbm_status lbm_set_timing(lbm_t* h, int enable) {
  if (!h) return LBM_EINVAL;
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, drain_timing(h));
  h->timing = enable != 0;
  h->launches = 0;
  h->start_log_sum = 0.0;
  h->start_count = 0;
  for (int k = 0; k < 3; ++k) {
    h->t_acc[k] = 0.0;
    h->t_cnt[k] = 0;
  }
  return LBM_OK;
}

lbm_status lbm_get_timing(lbm_t* h, double* out) {
  if (!h || !out) return LBM_EINVAL;
  cudaSetDevice(h->dev);
  LBM_CUDA_TRY(h, drain_timing(h));
  for (int k = 0; k < 3; ++k) {
    out[k] = h->t_acc[k];
    out[3 + k] = (double)h->t_cnt[k];
  }
  out[6] = (double)h->launches;
  return LBM_OK;
}

int64_t lbm_num_nodes(const lbm_t* h) { return h ? h->N : 0; }
int64_t lbm_state_len(const lbm_t* h) { return h ? (int64_t)h->S * Q * h->N : 0; }
void* lbm_stream(lbm_t* h) { return h ? (void*)h->own : nullptr; }

const char* lbm_last_error(const lbm_t* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
