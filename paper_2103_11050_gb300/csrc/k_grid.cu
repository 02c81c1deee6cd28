// Fine-grid stencil kernels of the MPM-2P step (HBM-bound, FP64).
//
//  - kappa^n = lambda(s) K and the partial sums of epsilon (Section 4.1, Algorithm 1).
//  - explicit upwind transport with its CFL time step (Section 4, Eq. BL2D), the last
//    substep fused with kappa^n, the epsilon partial sums and the Algorithm 1 decision.
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
  return div64(lw, lw + o * o);
}

__device__ __forceinline__ double harm(double a, double b) { return div64(2.0 * a * b, a + b); }


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

__global__ void k_fill_flags(Grid g, DevState d, int v) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < g.R) d.rebuild[r] = v;
}

// lambda = dt / h^2 = (cfl / max f') / rate_max with rate_max the largest total in- or outflow
// of a cell (reduced by the downscaling, which also stores its reciprocal); cfl_fmax = cfl /
// max f' from the host; 0 when nothing flows.
__device__ __forceinline__ double cfl_lambda(const DevState& d, int r, double cfl_fmax) {
  return cfl_fmax * d.inv_rate[r];
}

// Explicit upwind update of cell (i, j) (Eq. BL2D): s - dt/h^2 sum_faces F_out f(s_upwind),
// with f(s) read from fs; inflow through the boundary carries f(s_inflow) = f_in.  The sign
// of each face flux is read from its bit pattern (integer compares instead of float64 ones;
// -0 counts as zero like +0), and the outward flux enters through a fused multiply-add.
__device__ __forceinline__ double upwind_cell(const Grid& g, const double* ux, const double* uy, const double* fs,
                                              const double* s, double lam, double f_in, int i, int j) {
  const int nx = g.nx, ny = g.ny;
  const long long c = (long long)j * nx + i;
  const double fc = fs[c];
  const double uw = ux[(long long)j * (nx + 1) + i], ue = ux[(long long)j * (nx + 1) + i + 1];
  const double us = uy[(long long)j * nx + i], un = uy[(long long)(j + 1) * nx + i];
  double acc = 0.0;
  // outward fluxes: west -uw, east ue, south -us, north un
  if (dneg(uw)) acc = fma(-uw, fc, acc);
  else if (dpos(uw)) acc = fma(-uw, i > 0 ? fs[c - 1] : f_in, acc);
  if (dpos(ue)) acc = fma(ue, fc, acc);
  else if (dneg(ue)) acc = fma(ue, i < nx - 1 ? fs[c + 1] : f_in, acc);
  if (dneg(us)) acc = fma(-us, fc, acc);
  else if (dpos(us)) acc = fma(-us, j > 0 ? fs[c - nx] : f_in, acc);
  if (dpos(un)) acc = fma(un, fc, acc);
  else if (dneg(un)) acc = fma(un, j < ny - 1 ? fs[c + nx] : f_in, acc);
  return fma(-lam, acc, s[c]);
}

// One upwind substep s -> s2 with f(s2) -> fs2 (all substeps but the last).
__global__ void k_upwind(Grid g, DevState d, double cfl_fmax) {
  const int r = blockIdx.y;
  const long long n = g.ncell(), base = (long long)r * n;
  const double lam = cfl_lambda(d, r, cfl_fmax);
  if (blockIdx.x == 0 && threadIdx.x == 0) d.dt[r] = lam * g.h * g.h;
  const double* ux = d.ux + (long long)r * g.nfx();
  const double* uy = d.uy + (long long)r * g.nfy();
  const double f_in = g.f_in;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(c / g.nx), i = (int)(c - (long long)j * g.nx);
    const double s_new = upwind_cell(g, ux, uy, d.fs + base, d.s + base, lam, f_in, i, j);
    d.s2[base + c] = s_new;
    d.fs2[base + c] = fracflow(s_new, g.M);
  }
}

constexpr int kTX = 32;  // columns of the cell tile of the last transport substep; its rows kTY are a
                        // template parameter (4, 8 or 16), two rows per thread: small tiles spread the
                        // FP64 work over the SMs, tall tiles recompute fewer halo cells

// Last upwind substep fused with kappa^n (Algorithm 1: transport, then kappa^n): each CTA
// updates a kTX x kTY tile plus its east column and north row, with the water mobility
// M s^2, the total mobility lambda(s) and kappa^n = lambda(s) K of each of these cells, into
// shared memory, then writes s2, f(s2) = M s^2 / lambda(s) (from the stored mobilities),
// kappa^n and the east / north transmissibilities of its cells.  A thread takes two cells of
// one column (rows lj and lj + kTY / 2).
// decide = 1 (mpm_step): also the partial sums of ||kappa^n - kappa^m||^2, ||kappa^m||^2 per
// CTA; the last CTA to finish takes the Algorithm 1 decision for every realisation with the
// epsilon of the previous pass (rebuild_r = eps_r > eta), stores the new epsilon (0 where
// the basis is rebuilt, else sqrt(num / den)), counts the branches and, in a CUDA graph
// (set_handle), sets the conditional handle of the rebuild body.
template <int kTY>
__global__ void __launch_bounds__(kTX * kTY / 2) k_upwind_kappa(Grid g, DevState d, double cfl_fmax, int decide,
                                                                double eta, cudaGraphConditionalHandle h_reb,
                                                                int set_handle) {
  __shared__ double sn[kTY + 1][kTX + 1];  // s2
  __shared__ double sw[kTY + 1][kTX + 1];  // M s2^2
  __shared__ double sl[kTY + 1][kTX + 1];  // lambda(s2)
  __shared__ double sk[kTY + 1][kTX + 1];  // kappa^n of s2
  __shared__ double sh[32];
  __shared__ int last, tot;
  const int r = blockIdx.y;
  const int nx = g.nx, ny = g.ny;
  const int ntx = (nx + kTX - 1) / kTX;
  const int tx0 = (blockIdx.x % ntx) * kTX, ty0 = (blockIdx.x / ntx) * kTY;
  const long long base = (long long)r * g.ncell();
  const double lam = cfl_lambda(d, r, cfl_fmax), f_in = g.f_in;  // every thread: two loads, one multiply
  if (blockIdx.x == 0 && threadIdx.x == 0) d.dt[r] = lam * g.h * g.h;
  const double* ux = d.ux + (long long)r * g.nfx();
  const double* uy = d.uy + (long long)r * g.nfy();
  for (int e = threadIdx.x; e < (kTX + 1) * (kTY + 1); e += blockDim.x) {
    const int li = e % (kTX + 1), lj = e / (kTX + 1);
    const int i = tx0 + li, j = ty0 + lj;
    if (i < nx && j < ny && !(li == kTX && lj == kTY)) {
      const double v = upwind_cell(g, ux, uy, d.fs + base, d.s + base, lam, f_in, i, j);
      const double o = 1.0 - v;
      const double lw = g.M * v * v;
      const double lt = lw + o * o;  // lambda(v), as mobility()
      sn[lj][li] = v;
      sw[lj][li] = lw;
      sl[lj][li] = lt;
      sk[lj][li] = lt * d.K[base + (long long)j * nx + i];
    }
  }
  __syncthreads();
  double num = 0.0, den = 0.0;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int li = threadIdx.x % kTX, lj = threadIdx.x / kTX + half * (kTY / 2);
    const int i = tx0 + li, j = ty0 + lj;
    if (i < nx && j < ny) {
      const long long c = base + (long long)j * nx + i;
      d.s2[c] = sn[lj][li];
      d.fs2[c] = div64(sw[lj][li], sl[lj][li]);  // fracflow(s2)
      const double kn = sk[lj][li];
      d.kap_n[c] = kn;
      if (i < nx - 1) d.tx[(long long)r * g.nfx() + (long long)j * (nx + 1) + i + 1] = harm(kn, sk[lj][li + 1]);
      if (j < ny - 1) d.ty[(long long)r * g.nfy() + (long long)(j + 1) * nx + i] = harm(kn, sk[lj + 1][li]);
      if (decide) {
        const double km = d.kap_m[c];
        num += (kn - km) * (kn - km);
        den += km * km;
      }
    }
  }
  if (!decide) return;
  num = block_sum(num, sh);
  den = block_sum(den, sh);
  const int nblk = gridDim.x;
  if (threadIdx.x == 0) {
    d.eps_part[((long long)r * nblk + blockIdx.x) * 2 + 0] = num;
    d.eps_part[((long long)r * nblk + blockIdx.x) * 2 + 1] = den;
    __threadfence();
    last = atomicAdd(&d.ticket[1], 1u) == (unsigned int)(nblk * gridDim.y) - 1u;
    tot = 0;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // one warp per realisation
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slot = (int)(__ldcg(d.hist_n) % kEpsHist);  // history slot of this decision
  int mine = 0;
  constexpr int kBatch = 8;  // partials loaded together before they are summed (same order)
  for (int rr = warp; rr < g.R; rr += blockDim.x >> 5) {
    double a = 0.0, b = 0.0;
    const double* ep = d.eps_part + (long long)rr * nblk * 2;
    for (int k0 = lane; k0 < nblk; k0 += 32 * kBatch) {
      double va[kBatch], vb[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int k = k0 + 32 * u;
        va[u] = k < nblk ? __ldcg(&ep[2 * k]) : 0.0;
        vb[u] = k < nblk ? __ldcg(&ep[2 * k + 1]) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        if (k0 + 32 * u < nblk) {
          a += va[u];
          b += vb[u];
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      const int f = d.eps[rr] > eta ? 1 : 0;
      d.rebuild[rr] = f;
      const double e = f ? 0.0 : (b > 0.0 ? sqrt(a) / sqrt(b) : 0.0);
      d.eps[rr] = e;
      d.eps_hist[(long long)rr * kEpsHist + slot] = e;
      d.reb_hist[(long long)rr * kEpsHist + slot] = f;
      mine += f;
    }
  }
  if (lane == 0 && mine) atomicAdd(&tot, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    d.hist_n[0] += 1;
    d.counts[0] += tot;
    d.counts[1] += g.R - tot;
    if (set_handle) {
      cudaGraphSetConditional(h_reb, tot > 0 ? 1u : 0u);
      d.counts[2] += tot > 0;
      d.counts[3] += tot < g.R;
    }
    d.ticket[1] = 0;
  }
}

// Host-visible transfers without a copy engine: src / dst is pinned host memory addressed
// from the device (the device address CUDA reports for it).  k_load_checked copies n values
// in and raises *bad (also pinned host memory) when one lies outside [0,1];
// k_store_host copies n values out and, from one thread, the two status words after them in
// stream order.
__global__ void k_load_checked(const double* __restrict__ src, double* __restrict__ dst, long long n, int* bad) {
  int found = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = src[i];
    dst[i] = v;
    found |= !(v >= 0.0 && v <= 1.0);
  }
  if (__syncthreads_or(found) && threadIdx.x == 0) *reinterpret_cast<volatile int*>(bad) = 1;
}

// k_load_checked that also writes the fractional flow f(s) of every value loaded (the one
// quantity of the saturation that the next transport step reads besides s itself).
__global__ void k_load_checked_fs(const double* __restrict__ src, double* __restrict__ dst,
                                  double* __restrict__ fs_dst, long long n, double M, int* bad) {
  int found = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = src[i];
    dst[i] = v;
    fs_dst[i] = fracflow(v, M);
    found |= !(v >= 0.0 && v <= 1.0);
  }
  if (__syncthreads_or(found) && threadIdx.x == 0) *reinterpret_cast<volatile int*>(bad) = 1;
}

__global__ void k_store_host(const double* __restrict__ src, double* __restrict__ dst, long long n,
                             const int* status, int* status_host) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    status_host[0] = status[0];
    status_host[1] = status[1];
  }
}

int transfer_blocks(long long n) {
  const long long nb = (n + kThreads - 1) / kThreads;
  return (int)(nb < 1 ? 1 : nb < 1216 ? nb : 1216);  // up to 8 CTAs per SM of 152
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

void launch_choose(const Grid& g, const DevState& d, double eta, cudaStream_t st) {
  k_choose<<<(g.R + 127) / 128, 128, 0, st>>>(g, d, eta);
  ++g_launches;
}

void launch_load_checked(const double* src_dev, double* dst, long long n, int* bad_dev, cudaStream_t st) {
  k_load_checked<<<transfer_blocks(n), kThreads, 0, st>>>(src_dev, dst, n, bad_dev);
  ++g_launches;
}

void launch_load_checked_fs(const double* src_dev, double* dst, double* fs_dst, long long n, double M, int* bad_dev,
                            cudaStream_t st) {
  k_load_checked_fs<<<transfer_blocks(n), kThreads, 0, st>>>(src_dev, dst, fs_dst, n, M, bad_dev);
  ++g_launches;
}

void launch_store_host(const double* src, double* dst_dev, long long n, const int* status, int* status_host_dev,
                       cudaStream_t st) {
  k_store_host<<<transfer_blocks(n), kThreads, 0, st>>>(src, dst_dev, n, status, status_host_dev);
  ++g_launches;
}

void launch_fill_flags(const Grid& g, const DevState& d, int v, cudaStream_t st) {
  k_fill_flags<<<(g.R + 127) / 128, 128, 0, st>>>(g, d, v);
  ++g_launches;
}

void launch_upwind(const Grid& g, const DevState& d, double cfl, double fmax_, cudaStream_t st) {
  k_upwind<<<dim3(cell_blocks(g), g.R), kThreads, 0, st>>>(g, d, cfl / fmax_);
  ++g_launches;
}

int upwind_kappa_blocks_rows(const Grid& g, int rows) { return ((g.nx + kTX - 1) / kTX) * ((g.ny + rows - 1) / rows); }

// the largest grid over the tile shapes (sizes the per-block partial sums)
int upwind_kappa_blocks(const Grid& g) { return upwind_kappa_blocks_rows(g, 4); }

void launch_upwind_kappa(const Grid& g, const DevState& d, double cfl, double fmax_, bool decide, double eta,
                         cudaGraphConditionalHandle h_reb, bool set_handle, int rows, cudaStream_t st) {
  const dim3 grid(upwind_kappa_blocks_rows(g, rows), g.R);
  const int dec = decide ? 1 : 0, sh = set_handle ? 1 : 0;
  const double cf = cfl / fmax_;
  if (rows >= 16) k_upwind_kappa<16><<<grid, kTX * 8, 0, st>>>(g, d, cf, dec, eta, h_reb, sh);
  else if (rows >= 8) k_upwind_kappa<8><<<grid, kTX * 4, 0, st>>>(g, d, cf, dec, eta, h_reb, sh);
  else k_upwind_kappa<4><<<grid, kTX * 2, 0, st>>>(g, d, cf, dec, eta, h_reb, sh);
  ++g_launches;
}

}  // namespace mpm
