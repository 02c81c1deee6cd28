// Fine-grid stencil kernels of the MPM-2P step (HBM-bound, FP64).
//
//  - kappa^n = lambda(s) K and the partial sums of epsilon (Section 4.1, Algorithm 1).
//  - the Algorithm 1 decision and the new epsilon after it.
//  - CFL time step (from per-subdomain maxima) and explicit upwind transport (Section 4,
//    Eq. BL2D).
#include "mpm2p_internal.cuh"

namespace mpm {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double mobility(double s, double M) {
  const double o = 1.0 - s;
  return M * s * s + o * o;
}

__device__ __forceinline__ double fracflow(double s, double M) {
  const double lw = M * s * s;
  const double o = 1.0 - s;
  return lw / (lw + o * o);
}

__device__ __forceinline__ double harm(double a, double b) { return 2.0 * a * b / (a + b); }


__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  return v;  // valid in thread 0
}

__device__ double block_max(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  return v;
}

// kappa^n = lambda(s) K and the interior-face transmissibilities of kappa^n (the east and
// north faces of each cell; the neighbour's kappa is recomputed from its s and K);
// optional partial sums of (kappa^n - kappa^m)^2 and (kappa^m)^2.
__global__ void k_mobility_eps(Grid g, DevState d, int with_eps) {
  __shared__ double sh[32];
  const int r = blockIdx.y;
  const int nx = g.nx, ny = g.ny;
  const long long n = g.ncell();
  const long long base = (long long)r * n;
  double num = 0.0, den = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const double sc = d.s[base + c];
    const double kn = mobility(sc, g.M) * d.K[base + c];
    d.kap_n[base + c] = kn;
    d.fs[base + c] = fracflow(sc, g.M);
    const int j = (int)(c / nx), i = (int)(c - (long long)j * nx);
    if (i < nx - 1) {
      const double ke = mobility(d.s[base + c + 1], g.M) * d.K[base + c + 1];
      d.tx[(long long)r * g.nfx() + (long long)j * (nx + 1) + i + 1] = harm(kn, ke);
    }
    if (j < ny - 1) {
      const double kt = mobility(d.s[base + c + nx], g.M) * d.K[base + c + nx];
      d.ty[(long long)r * g.nfy() + (long long)(j + 1) * nx + i] = harm(kn, kt);
    }
    if (with_eps) {
      const double km = d.kap_m[base + c];
      num += (kn - km) * (kn - km);
      den += km * km;
    }
  }
  if (!with_eps) return;
  num = block_sum(num, sh);
  den = block_sum(den, sh);
  if (threadIdx.x == 0) {
    d.eps_part[((long long)r * gridDim.x + blockIdx.x) * 2 + 0] = num;
    d.eps_part[((long long)r * gridDim.x + blockIdx.x) * 2 + 1] = den;
  }
}

__global__ void k_eps_finalize(Grid g, DevState d, int nblk) {
  __shared__ double sh[32];
  const int r = blockIdx.x;
  double num = 0.0, den = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    num += d.eps_part[((long long)r * nblk + b) * 2 + 0];
    den += d.eps_part[((long long)r * nblk + b) * 2 + 1];
  }
  num = block_sum(num, sh);
  den = block_sum(den, sh);
  if (threadIdx.x == 0) d.eps[r] = den > 0.0 ? sqrt(num) / sqrt(den) : 0.0;
}

__global__ void k_choose(Grid g, DevState d, double eta) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < g.R) d.rebuild[r] = d.eps[r] > eta ? 1 : 0;
}

// Algorithm 1 decision for every realisation (one CTA): rebuild_r = eps_r > eta; counts
// the branches taken and, inside a CUDA graph, sets the conditional handles of the
// rebuild body (any realisation rebuilds) and of the MPM-2P body (any reuses).
__global__ void k_choose_graph(Grid g, DevState d, double eta, cudaGraphConditionalHandle h_reb,
                               cudaGraphConditionalHandle h_mpm, int set_handles) {
  __shared__ int tot;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  int mine = 0;
  for (int r = threadIdx.x; r < g.R; r += blockDim.x) {
    const int f = d.eps[r] > eta ? 1 : 0;
    d.rebuild[r] = f;
    mine += f;
  }
  atomicAdd(&tot, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    d.counts[0] += tot;
    d.counts[1] += g.R - tot;
    if (set_handles) {
      cudaGraphSetConditional(h_reb, tot > 0 ? 1u : 0u);
      cudaGraphSetConditional(h_mpm, tot < g.R ? 1u : 0u);
      d.counts[2] += tot > 0;
      d.counts[3] += tot < g.R;
    }
  }
}

// New epsilon after the update of this step (Algorithm 1, update of epsilon): 0 where the basis was
// rebuilt (kappa^m := kappa^n), else ||kappa^n - kappa^m|| / ||kappa^m|| from the partial sums
// taken in the transport's mobility pass (kappa^m unchanged by an MPM-2P update).
__global__ void k_eps_after_choose(Grid g, DevState d, int nblk) {
  __shared__ double sh[32];
  const int r = blockIdx.x;
  double num = 0.0, den = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    num += d.eps_part[((long long)r * nblk + b) * 2 + 0];
    den += d.eps_part[((long long)r * nblk + b) * 2 + 1];
  }
  num = block_sum(num, sh);
  den = block_sum(den, sh);
  if (threadIdx.x == 0) d.eps[r] = d.rebuild[r] ? 0.0 : (den > 0.0 ? sqrt(num) / sqrt(den) : 0.0);
}

__global__ void k_fill_flags(Grid g, DevState d, int v) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < g.R) d.rebuild[r] = v;
}

__global__ void k_copy_kappa_m(Grid g, DevState d) {
  const int r = blockIdx.y;
  if (d.rebuild[r] != 1) return;
  const long long n = g.ncell();
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x)
    d.kap_m[(long long)r * n + c] = d.kap_n[(long long)r * n + c];
}

// dt per realisation from the per-subdomain maxima of max(total outflow, total inflow)
// over cells that the downscaling wrote (rate_part[r][subdomain]).
__global__ void k_cfl_finalize(Grid g, DevState d, int nsub, double cfl, double fmax_) {
  __shared__ double sh[32];
  const int r = blockIdx.x;
  double m = 0.0;
  for (int b = threadIdx.x; b < nsub; b += blockDim.x) m = fmax(m, d.rate_part[(long long)r * d.st_sub + b]);
  m = block_max(m, sh);
  if (threadIdx.x == 0) d.dt[r] = m > 0.0 ? cfl * g.h * g.h / (fmax_ * m) : 0.0;
}

// s2_c = s_c - dt/h^2 sum_faces F_out f(s_upwind); inflow through the boundary carries
// s_inflow.  f(s) is read from fs (computed once per cell where s was produced); the
// kernel writes f(s2) to fs2 for the next substep.
__global__ void k_upwind(Grid g, DevState d) {
  const int r = blockIdx.y;
  const int nx = g.nx, ny = g.ny;
  const long long n = g.ncell(), base = (long long)r * n;
  const double lam = d.dt[r] / (g.h * g.h);
  const double* ux = d.ux + (long long)r * g.nfx();
  const double* uy = d.uy + (long long)r * g.nfy();
  const double* fs = d.fs + base;
  const double f_in = fracflow(g.s_inflow, g.M);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(c / nx), i = (int)(c - (long long)j * nx);
    const double fc = fs[c];
    double acc = 0.0, F;
    F = -ux[(long long)j * (nx + 1) + i];
    if (F > 0.0) acc += F * fc;
    else if (F < 0.0) acc += F * (i > 0 ? fs[c - 1] : f_in);
    F = ux[(long long)j * (nx + 1) + i + 1];
    if (F > 0.0) acc += F * fc;
    else if (F < 0.0) acc += F * (i < nx - 1 ? fs[c + 1] : f_in);
    F = -uy[(long long)j * nx + i];
    if (F > 0.0) acc += F * fc;
    else if (F < 0.0) acc += F * (j > 0 ? fs[c - nx] : f_in);
    F = uy[(long long)(j + 1) * nx + i];
    if (F > 0.0) acc += F * fc;
    else if (F < 0.0) acc += F * (j < ny - 1 ? fs[c + nx] : f_in);
    const double s_new = d.s[base + c] - lam * acc;
    d.s2[base + c] = s_new;
    d.fs2[base + c] = fracflow(s_new, g.M);
  }
}

int cell_blocks(const Grid& g) {
  long long nb = (g.ncell() + kThreads - 1) / kThreads;
  return (int)(nb < 1024 ? nb : 1024);
}

}  // namespace

int grid_cell_blocks(const Grid& g) { return cell_blocks(g); }

void launch_mobility_eps(const Grid& g, const DevState& d, bool with_eps, cudaStream_t st) {
  dim3 grid(cell_blocks(g), g.R);
  k_mobility_eps<<<grid, kThreads, 0, st>>>(g, d, with_eps ? 1 : 0);
  ++g_launches;
  if (with_eps) {
    k_eps_finalize<<<g.R, kThreads, 0, st>>>(g, d, grid.x);
    ++g_launches;
  }
}

void launch_mobility_partials(const Grid& g, const DevState& d, cudaStream_t st) {
  k_mobility_eps<<<dim3(cell_blocks(g), g.R), kThreads, 0, st>>>(g, d, 1);
  ++g_launches;
}

void launch_eps_after_choose(const Grid& g, const DevState& d, cudaStream_t st) {
  k_eps_after_choose<<<g.R, kThreads, 0, st>>>(g, d, cell_blocks(g));
  ++g_launches;
}

void launch_choose(const Grid& g, const DevState& d, double eta, cudaStream_t st) {
  k_choose<<<(g.R + 127) / 128, 128, 0, st>>>(g, d, eta);
  ++g_launches;
}

void launch_choose_graph(const Grid& g, const DevState& d, double eta, cudaGraphConditionalHandle h_reb,
                         cudaGraphConditionalHandle h_mpm, int set_handles, cudaStream_t st) {
  k_choose_graph<<<1, 256, 0, st>>>(g, d, eta, h_reb, h_mpm, set_handles);
  ++g_launches;
}

void launch_fill_flags(const Grid& g, const DevState& d, int v, cudaStream_t st) {
  k_fill_flags<<<(g.R + 127) / 128, 128, 0, st>>>(g, d, v);
  ++g_launches;
}

void launch_copy_kappa_m(const Grid& g, const DevState& d, cudaStream_t st) {
  k_copy_kappa_m<<<dim3(cell_blocks(g), g.R), kThreads, 0, st>>>(g, d);
  ++g_launches;
}

void launch_cfl(const Grid& g, const DevState& d, double cfl, double fmax_, int nsub, cudaStream_t st) {
  k_cfl_finalize<<<g.R, kThreads, 0, st>>>(g, d, nsub, cfl, fmax_);
  ++g_launches;
}

void launch_upwind(const Grid& g, const DevState& d, cudaStream_t st) {
  k_upwind<<<dim3(cell_blocks(g), g.R), kThreads, 0, st>>>(g, d);
  ++g_launches;
}

}  // namespace mpm
