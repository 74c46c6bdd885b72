// lbm_get_moments_noalloc: the moments of one species gathered into a
// fixed device staging array instead of a per-call device allocation.
//
// Who needs it: callers that must not allocate device memory while they run,
// for example a process whose device memory is fully reserved by another
// framework's pool, or a loop with hard latency limits that cannot afford
// an allocator call (cudaMalloc synchronises the device).  This entry point
// makes no cudaMalloc or cudaFree call and uses no allocating library routine.
//
// The staging array below is a file-scope device array: every GPU that loads
// the library holds its LBM_NOALLOC_MAX_NODES * 4 doubles (8 MiB) until the
// process exits.  All calls share it; calls that overlap on the GPU (two
// streams, two threads, two handles on one device) race on it.
#include <string.h>

#include <atomic>

#include "lbm_internal.cuh"

using namespace lbm_gb300;

namespace {

// n, u_x, u_y, u_z of up to LBM_NOALLOC_MAX_NODES nodes
static __device__ __align__(256) double g_moment_stage[4 * LBM_NOALLOC_MAX_NODES];

constexpr int kMaxDevices = 64;
// device address of g_moment_stage per device (host code cannot use the
// symbol itself: on the host it is only a stand-in, not a device address).
// Host threads that make their first call at the same time may both look
// the address up; they find the same value, and the atomic makes the
// concurrent stores well defined.
std::atomic<double*> g_stage_ptr[kMaxDevices] = {};

}  // namespace

extern "C" lbm_status lbm_get_moments_noalloc(lbm_t* h, int s, double* n, double* u) {
  if (!h) return LBM_EINVAL;
  if (s < 0 || s >= h->S) {
    h->err = "species index out of range";
    return LBM_EINVAL;
  }
  if (!(h->species_set >> s & 1u)) {
    h->err = "species not set";
    return LBM_EINVAL;
  }
  if (h->N > (int64_t)LBM_NOALLOC_MAX_NODES) {
    h->err = "lbm_get_moments_noalloc: lattice has more nodes than LBM_NOALLOC_MAX_NODES (262144)";
    return LBM_EINVAL;
  }
  if (h->dev < 0 || h->dev >= kMaxDevices) {
    h->err = "lbm_get_moments_noalloc: device ordinal beyond the supported range";
    return LBM_EINVAL;
  }
  if (!n && !u) return LBM_OK;
  LBM_CUDA_TRY(h, cudaSetDevice(h->dev));
  // first call on this device: look up the device address of the array
  // (with this device current)
  double* dn = g_stage_ptr[h->dev].load(std::memory_order_acquire);
  if (!dn) {
    LBM_CUDA_TRY(h, cudaGetSymbolAddress((void**)&dn, g_moment_stage));
    g_stage_ptr[h->dev].store(dn, std::memory_order_release);
  }
  const int64_t N = h->N;
  double* du = dn + N;
  // the gather runs on the library's stream after the last lbm_step, also
  // when that step ran on a caller's stream
  LBM_CUDA_TRY(h, own_stream(h));
  LBM_CUDA_TRY(h, launch_gather(h, s, dn, du, nullptr));
  if (n) LBM_CUDA_TRY(h, cudaMemcpyAsync(n, dn, N * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  if (u) LBM_CUDA_TRY(h, cudaMemcpyAsync(u, du, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  LBM_CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return LBM_OK;
}
