// Objective of the discrete inverse problem computed without any device allocation,
// for callers that cannot call cudaMalloc (see lbm_objective_noalloc in
// include/lbm_solid.h).  Its per-block partial sums live in a fixed file-scope device
// array instead of handle-owned scratch.
#include <cuda_runtime.h>

#include <atomic>

#include "lbm_device.cuh"
#include "lbm_solid.h"

namespace {

constexpr int kThreads = 256;
constexpr long kMaxBlocks = LBM_NOALLOC_MAX_NODES / kThreads;

// Shared by every call on a device (two partial sums per block); held until exit.
static __device__ __align__(256) double g_noalloc_scratch[2 * kMaxBlocks];

constexpr int kMaxDevices = 64;
// Device address of g_noalloc_scratch per device, looked up on the first call on that
// device.  Atomic: concurrent first calls from several host threads may both look it
// up, and both store the same value.
static std::atomic<void *> g_scratch_addr[kMaxDevices];

// Per node: d = (m10 + dx^2 F_x / 2, m01 + dx^2 F_y / 2) of f_S; partial sums of
// w |d - d*|^2 and w |d*|^2 for this block.
__global__ void __launch_bounds__(kThreads) k_objective_noalloc(
    const double *__restrict__ fS, const double *__restrict__ F,
    const double *__restrict__ dstar, const double *__restrict__ obs, long N, double half_dx2,
    double *__restrict__ scratch) {
  const long n = blockIdx.x * (long)kThreads + threadIdx.x;
  double acc[2] = {0.0, 0.0};
  if (n < N) {
    double f[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] = fS[k * N + n];
    const double dx_ = (f[0] - f[2]) + (f[4] - f[6]) - (f[5] - f[7]) + half_dx2 * F[n];
    const double dy_ = (f[1] - f[3]) + (f[4] - f[6]) + (f[5] - f[7]) + half_dx2 * F[N + n];
    const double w = obs ? obs[n] : 1.0;
    const double ex = dx_ - dstar[n], ey = dy_ - dstar[N + n];
    acc[0] = w * (ex * ex + ey * ey);
    acc[1] = w * (dstar[n] * dstar[n] + dstar[N + n] * dstar[N + n]);
  }
  __shared__ double sm[64];
  lbm::block_sum<2>(acc, sm);
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x + 0] = acc[0];
    scratch[2 * blockIdx.x + 1] = acc[1];
  }
}

// J = (1/2) sum w |d - d*|^2 dx^2 / (sum w |d*|^2 dx^2), NaN when the weighted target
// norm is zero.
__global__ void __launch_bounds__(kThreads) k_objective_noalloc_finish(
    const double *__restrict__ scratch, long nb, double *__restrict__ J) {
  double acc[2] = {0.0, 0.0};
  for (long i = threadIdx.x; i < nb; i += kThreads) {
    acc[0] += scratch[2 * i + 0];
    acc[1] += scratch[2 * i + 1];
  }
  __shared__ double sm[64];
  lbm::block_sum<2>(acc, sm);
  if (threadIdx.x == 0)
    J[0] = acc[1] != 0.0 ? 0.5 * acc[0] / acc[1] : __longlong_as_double(0x7ff8000000000000ll);
}

}  // namespace

extern "C" lbm_status lbm_objective_noalloc(int nx, int ny, double dx, const double *fS_dev,
                                            const double *F_dev, const double *dstar_dev,
                                            const double *obs_dev, double *J_dev,
                                            void *stream) {
  if (nx < 1 || ny < 1 || !(dx > 0.0) || !fS_dev || !F_dev || !dstar_dev || !J_dev)
    return LBM_ERR_ARG;
  const long N = (long)nx * ny;
  if (N > LBM_NOALLOC_MAX_NODES) return LBM_ERR_ARG;  // beyond the fixed scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return LBM_ERR_ARG;
  void *addr = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!addr) {
    // Host code cannot use the array's name as a device address: look it up once per
    // device, with that device current.
    if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || !addr)
      return LBM_ERR_CUDA;
    g_scratch_addr[dev].store(addr, std::memory_order_release);
  }
  double *scratch = static_cast<double *>(addr);
  const long nb = (N + kThreads - 1) / kThreads;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_objective_noalloc<<<(unsigned)nb, kThreads, 0, s>>>(fS_dev, F_dev, dstar_dev, obs_dev, N,
                                                       0.5 * dx * dx, scratch);
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  k_objective_noalloc_finish<<<1, kThreads, 0, s>>>(scratch, nb, J_dev);
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  return LBM_OK;
}
