// noalloc.cu -- the Euler step of the master equation for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: a host framework whose caching
// allocator already holds the whole card, a process running under a fixed
// device-memory budget, or a latency-critical loop that must not pay the
// implicit device-wide synchronisation an allocation can cause.  For them,
// mxe_diffuse_step_noalloc runs the same kernels as mxe_diffuse_step (per-site
// factors, bond gather, conditional commit) on caller-owned inputs and
// outputs, with its scratch in one file-scope device array of fixed size
// instead of a context.  No context, no cudaMalloc / cudaFree, no allocating
// library call.
//
// The array lives on every device that loads this library until the process
// exits.  Every call shares it and it keeps the last call's contents; the
// flag words are cleared at the start of each call and the per-site scratch
// is fully written before it is read.  Calls that overlap on the GPU (on
// different streams, or from different host threads) race on the array.
#include <cuda_runtime.h>

#include <mutex>

#include "mxe_internal.cuh"

using namespace mxe;

namespace {

// 256 bytes of flag words, then MXE_NOALLOC_SCRATCH_DOUBLES doubles.
constexpr size_t kFlagBytes = 256;
constexpr size_t kScratchBytes = kFlagBytes + sizeof(double) * (size_t)MXE_NOALLOC_SCRATCH_DOUBLES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};  // device address of the array, per device

// Device address of the array on the current device.  Host code cannot pass
// the array's name to a kernel (on the host it names a stand-in), so the
// address is looked up once per device with that device current.
mxe_status scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return MXE_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return MXE_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return MXE_OK;
}

}  // namespace

extern "C" MXE_API mxe_status mxe_diffuse_step_noalloc(int64_t n, int32_t n_species, double* x_dev,
                                                       const double* T_dev, const double* mu_ex_dev,
                                                       const int32_t* bond_offsets_dev, const int32_t* bond_idx_dev,
                                                       double dt, double nu0, double Qm, void* cuda_stream) {
  if (n < 0 || n_species < 1 || n_species > 2) return MXE_ERR_ARG;
  if (n > MXE_NOALLOC_MAX_SITES(n_species)) return MXE_ERR_ARG;  // beyond the fixed scratch
  if (!(dt >= 0.0) || !(nu0 >= 0.0) || !(Qm == Qm)) return MXE_ERR_ARG;
  if (n > 0 && (!x_dev || !T_dev || !mu_ex_dev || !bond_offsets_dev || !bond_idx_dev)) return MXE_ERR_ARG;
  unsigned char* base = nullptr;
  mxe_status ms = scratch_address(&base);
  if (ms != MXE_OK) return ms;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int* step_flags = reinterpret_cast<int*>(base);
  int* sticky = step_flags + 1;
  double* factors = reinterpret_cast<double*>(base + kFlagBytes);
  double* x_new = factors + flux_scratch_len(n, n_species);
  cudaError_t e = cudaMemsetAsync(step_flags, 0, 2 * sizeof(int), st);
  if (e == cudaSuccess)
    e = launch_flux(x_dev, T_dev, mu_ex_dev, bond_offsets_dev, bond_idx_dev, n, n_species, dt, nu0, Qm, factors,
                    x_new, step_flags, st);
  if (e == cudaSuccess) e = launch_commit_x(x_dev, x_new, (int64_t)n_species * n, step_flags, sticky, nullptr, st);
  int flags_h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flags_h, step_flags, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? MXE_ERR_OOM : MXE_ERR_CUDA;
  }
  return (flags_h & kFlagXRange) ? MXE_ERR_X_RANGE : MXE_OK;
}
