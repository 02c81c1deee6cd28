// Allocation-free CFL time step: mpm_cfl_dt_noalloc (declared in include/mpm2p.h).
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by another
// runtime (a framework with its own pre-sized pool that forbids foreign allocations), or a
// latency-critical loop that cannot afford an allocation's implicit device
// synchronisation or its failure mid-run.  This entry point computes the same transport
// time step as mpm_saturation_step from caller-owned flux arrays without allocating: its
// per-block partial maxima live in a fixed device array of this file, which every GPU
// that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/mpm2p.h"

namespace {

constexpr int kBlocksPerRealisation = 64;       // partial maxima per realisation
constexpr int kScratchDoubles = 64 * 1024;      // 512 KiB: R * 64 <= 65536, i.e. R <= 1024
constexpr int kMaxDevices = 64;

// Scratch of the reduction, shared by every call on a device.
static __device__ __align__(256) double g_noalloc_partials[kScratchDoubles];

// Device address of g_noalloc_partials per device (host side), set by the first call on
// that device.
double* g_scratch_addr[kMaxDevices] = {};

__global__ void k_cfl_partials(const double* __restrict__ ux, const double* __restrict__ uy, int nx, int ny,
                               double* partials) {
  __shared__ double sh[32];
  const int r = blockIdx.y;
  const long long n = (long long)nx * ny;
  const double* uxr = ux + (long long)r * ny * (nx + 1);
  const double* uyr = uy + (long long)r * (ny + 1) * nx;
  double m = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(c / nx), i = (int)(c - (long long)j * nx);
    const double f0 = -uxr[(long long)j * (nx + 1) + i], f1 = uxr[(long long)j * (nx + 1) + i + 1];
    const double f2 = -uyr[(long long)j * nx + i], f3 = uyr[(long long)(j + 1) * nx + i];
    const double out = fmax(f0, 0.0) + fmax(f1, 0.0) + fmax(f2, 0.0) + fmax(f3, 0.0);
    const double in = fmax(-f0, 0.0) + fmax(-f1, 0.0) + fmax(-f2, 0.0) + fmax(-f3, 0.0);
    m = fmax(m, fmax(out, in));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) partials[r * gridDim.x + blockIdx.x] = m;
  }
}

__global__ void k_cfl_from_partials(const double* partials, int R, double h, double cfl, double fmax_,
                                    double* dt) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  double m = 0.0;
  for (int b = 0; b < kBlocksPerRealisation; ++b) m = fmax(m, partials[r * kBlocksPerRealisation + b]);
  dt[r] = m > 0.0 ? cfl * h * h / (fmax_ * m) : 0.0;
}

// max_s f'(s) for f = M s^2 / (M s^2 + (1-s)^2): the stationary point is the root in (0,1)
// of 2(M+1)s^3 - 3(M+1)s^2 + 1 (strictly decreasing there), found by bisection.
double max_fprime(double M) {
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (2.0 * (M + 1.0) * mid * mid * mid - 3.0 * (M + 1.0) * mid * mid + 1.0 > 0.0) lo = mid;
    else hi = mid;
  }
  const double s = 0.5 * (lo + hi);
  const double den = M * s * s + (1.0 - s) * (1.0 - s);
  return 2.0 * M * s * (1.0 - s) / (den * den);
}

}  // namespace

extern "C" int mpm_cfl_dt_noalloc(const double* ux, const double* uy, int R, int nx, int ny, double h, double M,
                                  double cfl, double* dt, void* stream) {
  if (!ux || !uy || !dt || nx < 1 || ny < 1 || R < 1 || !(h > 0) || !(M > 0) || !(cfl > 0 && cfl <= 1))
    return MPM_ERR_ARG;
  if ((long long)R * kBlocksPerRealisation > kScratchDoubles) return MPM_ERR_TOO_LARGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MPM_ERR_CUDA;
  if (!g_scratch_addr[dev]) {
    double* p = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_partials) != cudaSuccess || !p)
      return MPM_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_cfl_partials<<<dim3(kBlocksPerRealisation, R), 256, 0, st>>>(ux, uy, nx, ny, g_scratch_addr[dev]);
  k_cfl_from_partials<<<(R + 127) / 128, 128, 0, st>>>(g_scratch_addr[dev], R, h, cfl, max_fprime(M), dt);
  return cudaGetLastError() == cudaSuccess ? MPM_OK : MPM_ERR_CUDA;
}
