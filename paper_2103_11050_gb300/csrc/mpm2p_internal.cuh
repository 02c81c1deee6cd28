// Internal declarations shared by the translation units of libmpm2p.
//
// Geometry tables (per subdomain, shared by all realisations) and per-realisation
// pools live in device memory owned by the context.  Kernels are grouped by stage:
//   k_grid.cu   fine-grid stencils: kappa / epsilon, decision, CFL, transport
//   k_local.cu  local Robin and Neumann problems (block-tridiagonal factorisation with
//               explicit inverse pivot blocks, multi-RHS solves, FP64 refinement)
//   k_iface.cu  interface (skeleton) system: element matrices, nested-dissection sweep
//               factorisation and solves
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <utility>

#include "fp64_div.cuh"

namespace mpm {

constexpr int kMaxRealisations = 65535;  // realisations per context (a grid y / z dimension)
constexpr int kMaxSide = 24;     // largest subdomain width / height in cells
constexpr int kPivotChunk = 16;  // pivot block of the interface sweeps
constexpr int kEpsHist = 4096;   // steps of epsilon history kept per realisation (MPM_EPS_HISTORY)

// Padded width A of the stored local factors ([b][A][A] per subdomain): 8, 16 or 32.
__host__ __device__ inline int pad_width(int max_a) { return max_a <= 8 ? 8 : max_a <= 16 ? 16 : 32; }

// Face numbering inside a subdomain of a x b cells: left side (b faces, bottom to top),
// right side (b), bottom side (a faces, left to right), top side (a): 2(a+b) faces.
__host__ __device__ inline int face_side_off(int side, int a, int b) {
  return side == 0 ? 0 : side == 1 ? b : side == 2 ? 2 * b : 2 * b + a;
}

struct DevSub {
  int x0, y0, a, b;
  int A;             // padded width of this subdomain's factor blocks, pad_width(a)
  int ndof;          // interface DOFs on the sides of this subdomain
  int dof_off;       // offset in per-DOF tables (sum of ndof of previous subdomains)
  int face_off;      // offset in per-face tables (sum of 2(a+b))
  int cell_off;      // offset in per-cell local tables (sum of a*b)
  int side_kind[4];  // 0 physical boundary, 1 interface
  int side_iface[4]; // interface id or -1
  int side_dof0[4];  // first local DOF of this side (U block, then P block)
  int side_nb[4];    // U DOFs on this side (= P DOFs)
  int side_nbr[4];   // subdomain on the other side of the interface, or -1
  double side_sign[4];  // n_check . n_check^i
  long long q_off;   // Robin factor (b*A*A values of the factor type, A = pad_width) in the factor pool
  long long t_off;   // b*a values: vertical transmissibilities + scaling (see k_local.cu)
  long long tr_off;  // (2(a+b)) x ndof BF traces
  long long pf_off;  // a*b x ndof BF pressures (temporary, rebuild only)
};

struct Grid {
  int R, nx, ny;
  double h;
  int bc_type[4];
  double bc_val[4];
  double s_inflow;
  double M;
  double f_in;  // f(s_inflow) = M s_inflow^2 / (M s_inflow^2 + (1 - s_inflow)^2), set with s_inflow and M
  int seg_len, degree;
  double inv_seg;  // 1 / seg_len
  double alpha;
  int order;  // MPM-2P perturbation order: 0 (Eq. mpm_tf_3 only) or 1 (plus Eq. mpm_tf_4, l = 1)
  // The subdomains of one launch of a local kernel: blockIdx.x indexes this list (device
  // memory), or the subdomains themselves when it is null.  Decompositions with subdomain
  // widths of more than one padded width (8, 16, 32) launch the local kernels once per width,
  // each over its own list, so that every factor is padded to its own width only.
  const int* sub_list;
  __host__ __device__ long long ncell() const { return (long long)nx * ny; }
  __host__ __device__ long long nfx() const { return (long long)ny * (nx + 1); }
  __host__ __device__ long long nfy() const { return (long long)(ny + 1) * nx; }
};

#ifdef __CUDACC__
// Subdomain handled by this CTA of a local kernel (see Grid::sub_list).
__device__ __forceinline__ int sub_index(const Grid& g) { return g.sub_list ? g.sub_list[blockIdx.x] : (int)blockIdx.x; }

// Programmatic dependent launch.  A kernel launched with the programmatic-serialisation
// attribute may start once every block of its predecessor in the stream has called
// pdl_trigger(), i.e. while the predecessor still runs.  Before pdl_wait() such a kernel
// reads only data that no kernel of the running chain writes (operators, factors, index
// maps, and fields finished before the chain's first, fully ordered launch) and writes
// only registers and shared memory; pdl_wait() returns once the predecessor grid has
// completed and its memory operations are visible.  Without the attribute both are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Sign of a float64 from its bit pattern (integer compares; -0 and +0 are neither).
__device__ __forceinline__ bool dpos(double v) { return __double_as_longlong(v) > 0; }
__device__ __forceinline__ bool dneg(double v) {
  const long long b = __double_as_longlong(v);
  return b < 0 && b != (long long)0x8000000000000000ull;
}

// Outward integrated flux of pressure p through a physical boundary face of a cell with
// values (kc, pc) on side `side` (Dirichlet: 2 kc (pc - g); Neumann: z h).
__device__ __forceinline__ double phys_flux(const Grid& g, int side, double kc, double pc) {
  return g.bc_type[side] == 0 ? 2.0 * kc * (pc - g.bc_val[side]) : g.bc_val[side] * g.h;
}
#endif

// Launch shapes that depend on the geometry (the number and size of the subdomains against
// the SM count): defaults below, or the choice of the autotuner (mpm_autotune), which times
// every candidate on the context's own data.
struct Tuning {
  int local_threads = 256;  // threads per CTA of the MPM-2P local solve (64, 128 or 256; warps 0-1 run
                            // the twisted chains, all warps the cell-parallel phases)
  int local_stage = 1;      // 1: stage the stored factor in shared memory (cp.async), 0: read it from
                            // global memory inside the chains (smaller CTAs, more of them per SM)
  int ds_threads = 256;     // the same two for the downscaling solve
  int ds_stage = 1;
  int transport_rows = 8;   // rows of the 32-column tile of the fused transport kernel (4, 8 or 16)
  int sweep_terms = 16;     // interface sweeps: terms of a row's sum per thread (4, 8 or 16; fewer terms,
                            // more threads per row and more CTAs per level)
};

// Nested-dissection node of the interface system.  Leaves are subdomains (no
// separator, frontal = element matrix over the subdomain's DOFs).
struct DevNode {
  int nsep, nbnd, nf;
  int leaf_sub;        // subdomain id for leaves, -1 otherwise
  int child[2];        // node ids, -1 for leaves
  int parent;          // -1 for the root
  long long f_off;     // frontal matrix (nf x nf, row major) in the frontal pool
  long long v_off;     // vectors (nf) in the g / x pools
  int src_off;         // internal nodes: 2*nf ints: child0 / child1 boundary index per frontal index (-1 none)
  int pmap_off;        // nbnd ints: frontal index in the parent of each boundary DOF
  int level;           // 0 for leaves, 1 + the larger level of the children otherwise
};

// Per-realisation device state (all pointers are device pointers; pools are indexed
// r * st_x + offset).
struct DevState {
  // cells [R][ny][nx]
  double *K, *q, *s, *s2, *kap_n, *kap_m, *p_m, *p_down;
  double* x_ds;        // pinned Neumann solution of the last refined downscaling (initial iterate of the next)
  double* dp0;         // MRCM-level pressure of the epsilon^0 solve (first-order MPM-2P only)
  double *fs, *fs2;    // fractional flow f(s) of s / s2
  // faces
  double *ux, *uy;
  double *tx, *ty;     // transmissibilities of kappa^n: tx [R][ny][nx+1], ty [R][ny+1][nx] (interior faces)
  // per realisation scalars
  double *eps, *dt, *eps_part;
  double* rate_part;  // [R][st_sub] per subdomain: max over its cells of max(outflow, inflow), by the downscaling
  double* rate_max;   // [R] max over rate_part, by the last block of the downscaling
  double* inv_rate;   // [R] 1 / rate_max (0 when nothing flows), by the same block
  unsigned int* ticket;  // [4] block-completion counters (0: downscaling, 1: transport); back to 0 after each launch
  int* rebuild;        // [R] branch of the current update: 1 = basis build, 0 = MPM-2P reuse
  int* status;         // [1] bitmask: 1 = a refinement did not reach its tolerance
  int* ir_iters;       // [1] max refinement sweeps used
  long long* counts;   // [5] rebuild / MPM-2P updates taken by the device-side decision; graph steps
                       //     that ran the rebuild body / the MPM-2P body; downscaling factorisations
                       //     computed (subdomains, all realisations)
  double* eps_hist;    // [R][kEpsHist] epsilon after each decision (ring, slot = step % kEpsHist)
  int* reb_hist;       // [R][kEpsHist] the decision of that step (1 = rebuild)
  long long* hist_n;   // [1] decisions recorded so far
  // per subdomain pools
  void* fac;           // Robin factors (float or double), st_fac values per realisation
  double* tvec;        // [ex, wE, wN, sc] per subdomain (4 m), st_t
  void* nfac;          // downscaling (pinned Neumann) factors of kappa^n, same layout as fac
  double* ntvec;       // their [ex, wE, wN, sc] of the current kappa^n (sc: of the stored factor), same
                       // layout as tvec
  double* nfw;         // [wE, wN] of kappa^n when the stored downscaling factor was computed (first 2 m of
                       // each subdomain's tvec-layout block)
  int* npin;           // [R][st_sub] pinned cell of the stored downscaling factor, -1: none stored
  double* npin_k;      // [R][st_sub] kappa^n of that cell when the factor was computed
  double* tr;          // BF traces, one column of 2(a+b) faces per BF (ndof x 2(a+b)), st_tr
  double* pf;          // BF pressures, one column of m cells per BF ((ndof + 1) x m), st_pf
  double* mu_hat;      // BF means, st_dof
  double* fbar;        // non-homogeneous / perturbation traces, st_face
  double* trace;       // one-sided traces of the current update, st_face
  double* trace1;      // one-sided traces of the first-order (epsilon^1) solve, st_face
  double* bhat;        // beta_hat = rho / kappa^m per face (interface faces), st_face
  double* rho_f;       // rho_e = alpha_e H_e / h per subdomain face (0 on physical faces), shared by all
                       // realisations (indexed face_off + f, no realisation stride)
  double* sub_mean;    // mean of the non-homogeneous local solution, st_sub
  double* sub_target;  // target mean of the downscaled pressure, st_sub
  double* pm_mean;     // mean of p^m over the subdomain, st_sub
  // interface system
  double *front, *gvec, *xvec;  // st_front, st_vec, st_vec
  double *pivinv, *colold;      // st_lvl * 256, st_col
  const int* srcmap;         // extend-add maps of the internal nodes (DevNode::src_off)
  unsigned int* nd_ticket;   // [R][st_nodes] children of each level-1 node done so far (see phase::fold_up)
  long long st_fac, st_t, st_tr, st_pf, st_dof, st_face, st_sub, st_front, st_vec, st_col, st_lvl, st_nodes;
};

// Kernels launched by this process through the wrappers below (host side, not thread safe).
extern long long g_launches;

// cudaLaunchKernelEx with the programmatic-serialisation attribute when pdl is set.
template <typename... KArgs, typename... Args>
void launch_ex(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
               Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);  // errors surface via cudaGetLastError
  ++g_launches;
}

// Host-side launch wrappers (defined in the .cu files).
// SMs of the current device (queried once per device).
inline int sm_count() {
  static int n[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (n[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    n[dev] = v > 0 ? v : 1;
  }
  return n[dev];
}

int grid_cell_blocks(const Grid& g);
void launch_mobility_eps(const Grid& g, const DevState& d, bool with_eps, cudaStream_t st);
void launch_choose(const Grid& g, const DevState& d, double eta, cudaStream_t st);
void launch_fill_flags(const Grid& g, const DevState& d, int v, cudaStream_t st);
// transfers with pinned host memory addressed from the device (no copy engine)
void launch_load_checked(const double* src_dev, double* dst, long long n, int* bad_dev, cudaStream_t st);
void launch_load_checked_fs(const double* src_dev, double* dst, double* fs_dst, long long n, double M, int* bad_dev,
                            cudaStream_t st);
void launch_store_host(const double* src, double* dst_dev, long long n, const int* status, int* status_host_dev,
                       cudaStream_t st);
void launch_upwind(const Grid& g, const DevState& d, double cfl, double fmax, cudaStream_t st);
int upwind_kappa_blocks(const Grid& g);
void launch_upwind_kappa(const Grid& g, const DevState& d, double cfl, double fmax, bool decide, double eta,
                         cudaGraphConditionalHandle h_reb, bool set_handle, int rows, cudaStream_t st);
int upwind_kappa_blocks_rows(const Grid& g, int rows);

int local_smem_limit();
void launch_robin_factor(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a,
                         int max_b, bool fp32, cudaStream_t st);
void launch_basis_solve(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a,
                        int max_b, int tc_kind, bool fp32, double ir_tol, int ir_max, const DevNode* nodes,
                        const int* leaf_node, cudaStream_t st);
void launch_mpm_local(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a,
                      int max_b, bool fp32, double ir_tol, int ir_max, const DevNode* nodes, const int* leaf_node,
                      int threads, int stage, int pass, cudaStream_t st);
void launch_reconstruct(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_face,
                        int max_dof, int max_nf1, const DevNode* nodes, const int* leaf_node, const int* pmap,
                        int branch, int pass, bool pdl, cudaStream_t st);
void launch_downscale_factor(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a,
                             int max_b, bool fp32, double reuse_tol, cudaStream_t st);
void launch_downscale(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a,
                      int max_b, bool fp32, double ir_tol, int ir_max, bool pdl, int threads, int stage,
                      cudaStream_t st);

void launch_element_matrix(const Grid& g, const DevState& d, const DevSub* subs, int nsub,
                           const DevNode* nodes, const int* leaf_node, cudaStream_t st);
void launch_nd_factor_level(const Grid& g, const DevState& d, const DevNode* nodes, const int* level_nodes,
                            int nlev, int max_nf, int max_nsep, const int* srcmap, cudaStream_t st);
void launch_nd_up(const Grid& g, const DevState& d, const DevNode* nodes, const int* level_nodes, int nlev,
                  int max_nf, int max_nsep, const int* srcmap, bool pdl, int terms, cudaStream_t st,
                  int branch = -1);
void launch_nd_down(const Grid& g, const DevState& d, const DevNode* nodes, const int* level_nodes, int nlev,
                    int max_nsep, int max_nbnd, const int* pmap, bool pdl, int terms, cudaStream_t st);

}  // namespace mpm
