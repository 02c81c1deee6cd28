// C ABI of the MRCM / MPM-2P hot path (declarations and argument contracts in
// include/mpm2p.h).  Host-side context: geometry tables, the nested-dissection tree of
// the interface system, device pools, and the launch sequences of Algorithm 1.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/mpm2p.h"
#include "mpm2p_internal.cuh"

using namespace mpm;

namespace mpm {
long long g_launches = 0;
}

// The subdomains of one padded factor width A: one launch of each local kernel, over the
// device list d_list (null when every subdomain has this width).
struct SubClass {
  int A, count, max_a, max_b;
  int* d_list;
};

struct mpm_ctx {
  Grid g{};
  cudaStream_t stream = nullptr;
  int device = 0;
  std::string err;
  int prec = MPM_PREC_FP64;
  double ir_tol = 1e-14;
  double ds_reuse = -1.0;  // relative transmissibility change up to which a float32 downscaling factor is
                           // kept; negative: the default of ds_reuse_tol
  int ir_max = 20;
  int fac_prec = -1;  // precision the stored factor was built with
  bool have_K = false, have_s = false, have_dec = false, have_basis = false;
  // kappa^n, f(s) and the transmissibilities of kappa^n lag the current saturation: set by a
  // pinned-memory mpm_set_saturation, which computes f(s) only (all a step needs); the other
  // entry points bring them up to date first (ensure_derived)
  bool derived_stale = false;
  double eta_init = 0.0;
  // decomposition
  int ncx = 0, ncy = 0;
  std::vector<int> col_w, row_h;
  std::vector<DevSub> subs;
  int max_a = 0, max_b = 0, max_dof = 0, max_face = 0, n_dof = 0, n_hat = 0;
  // nested dissection
  std::vector<DevNode> nodes;
  std::vector<int> leaf_node;
  std::vector<std::vector<int>> levels;  // node ids per level (level 0 = leaves)
  std::vector<int> lev_max_nf, lev_max_nsep, lev_max_nbnd;
  std::vector<int> lev_off;              // offset of each level in d_level_nodes
  // device tables
  DevSub* d_subs = nullptr;
  DevNode* d_nodes = nullptr;
  int* d_leaf_node = nullptr;
  int* d_level_nodes = nullptr;
  int* d_srcmap = nullptr;
  int* d_pmap = nullptr;
  DevState d{};
  std::vector<void*> grid_allocs, dec_allocs;
  // host staging for flags
  int* h_flags = nullptr;
  int* h_status = nullptr;  // pinned: status word and refinement sweep count, then a range flag
  int* h_status_dev = nullptr;  // the device address of h_status
  mpm_stats stats{};
  long long launches0 = 0;  // g_launches when the context was created
  long long init_rebuilds = 0;
  // kernel nodes of the step graph: always run / rebuild body / MPM-2P body; kernels only
  // recorded by captures (not executed at that time)
  long long gk_base = 0, gk_reb = 0, gk_mpm = 0, capture_launches = 0, graph_steps = 0;
  // CUDA graph of one Algorithm 1 step (conditional bodies for the two branches)
  bool use_graph = true;
  bool use_pdl = true;    // programmatic dependent launch along the interface-solve chain
  Tuning tune;            // launch shapes (defaults, mpm_set_tuning or mpm_autotune)
  std::vector<SubClass> classes;  // subdomains by padded factor width (one launch of a local kernel each)
  int next_pass = 0;      // pass of the next stand-alone interface solve (1 after mpm_perturbation_correction)
  // The saturation (and f(s)) live in two buffers that swap at every transport substep; a
  // graph reads and writes fixed buffers, so one graph is kept per buffer parity (slot 0:
  // the current saturation is in s_buf0).
  double* s_buf0 = nullptr;
  bool graph_valid[2] = {false, false};
  double g_eta = 0.0, g_cfl = 0.0;
  int g_nsub = 0;
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
  cudaStream_t cap_stream = nullptr, body_stream = nullptr;
  // side stream of the downscaling factorisation (forked after kappa^n, joined before the
  // downscaling solve)
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool factor_forked = false;  // a fork not yet joined into the main stream
  // branch of the rebuild body inside a step graph (forked after the decision, joined
  // before the interface solve)
  cudaStream_t reb_stream = nullptr;
  cudaEvent_t ev_reb_fork = nullptr, ev_reb_join = nullptr;
  bool reb_forked = false;
  // stage profiler
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_rec[MPM_NSTAGES];
  cudaEvent_t ev_open[MPM_NSTAGES] = {};
};

namespace {

int fail(mpm_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

#define CK(call)                                                                               \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(c, MPM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

int dalloc(mpm_ctx* c, std::vector<void*>& list, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(c, MPM_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  list.push_back(*p);
  cudaMemsetAsync(*p, 0, bytes, c->stream);
  return MPM_OK;
}

template <typename T>
int dalloc_t(mpm_ctx* c, std::vector<void*>& list, T** p, size_t n) {
  return dalloc(c, list, reinterpret_cast<void**>(p), n * sizeof(T));
}

void free_list(std::vector<void*>& list) {
  for (void* p : list) cudaFree(p);
  list.clear();
}

int check_launch(mpm_ctx* c) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, MPM_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return MPM_OK;
}

int copy_in(mpm_ctx* c, double* dst, const double* src, size_t n, int mem) {
  if (!src) return fail(c, MPM_ERR_ARG, "null input pointer");
  if (mem == MPM_MEM_HOST) {
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  } else if (mem == MPM_MEM_DEVICE) {
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  } else {
    return fail(c, MPM_ERR_ARG, "mem must be MPM_MEM_HOST or MPM_MEM_DEVICE");
  }
  return MPM_OK;
}

// The device address of pinned (page-locked, registered) host memory, or null for any other
// pointer; kernels read and write such memory directly, without a copy engine.
void* pinned_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear the query's error: the caller takes the copy path
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

int check_status(mpm_ctx* c);

int sync_status(mpm_ctx* c) {
  // status word and refinement sweep count (adjacent on the device), read in stream order
  // behind the work they report on, so that one host wait covers both
  CK(cudaMemcpyAsync(c->h_status, c->d.status, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return check_status(c);
}

// Acts on the status words already in h_status (after a host wait).
int check_status(mpm_ctx* c) {
  const int st = reinterpret_cast<volatile int*>(c->h_status)[0];
  const int it = reinterpret_cast<volatile int*>(c->h_status)[1];
  c->stats.ir_iters_max = std::max(c->stats.ir_iters_max, it);
  if (st & 1) {
    CK(cudaMemsetAsync(c->d.status, 0, sizeof(int), c->stream));
    return fail(c, MPM_ERR_NOT_CONVERGED, "local iterative refinement stopped above ir_tol=%g (ir_max=%d sweeps)",
                c->ir_tol, c->ir_max);
  }
  return MPM_OK;
}

int copy_out(mpm_ctx* c, double* dst, const double* src, size_t n, int mem) {
  if (!dst) return fail(c, MPM_ERR_ARG, "null output pointer");
  if (mem == MPM_MEM_HOST) {
    if (void* dd = pinned_device_ptr(dst)) {  // pinned: one kernel writes the values and the status words
      launch_store_host(src, static_cast<double*>(dd), (long long)n, c->d.status, c->h_status_dev, c->stream);
      CK(cudaGetLastError());
      CK(cudaStreamSynchronize(c->stream));
      return check_status(c);
    }
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  } else if (mem == MPM_MEM_DEVICE) {
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  } else {
    return fail(c, MPM_ERR_ARG, "mem must be MPM_MEM_HOST or MPM_MEM_DEVICE");
  }
  return sync_status(c);
}

// max_s f'(s) of f = M s^2 / (M s^2 + (1-s)^2): the stationary point solves
// 2(M+1)s^3 - 3(M+1)s^2 + 1 = 0, strictly decreasing on (0,1); bisection.
double max_fprime(double M) {
  double lo = 0.0, hi = 1.0;
  const double cM = M + 1.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (2.0 * cM * mid * mid * mid - 3.0 * cM * mid * mid + 1.0 > 0.0) lo = mid;
    else hi = mid;
  }
  const double s = 0.5 * (lo + hi);
  const double den = M * s * s + (1.0 - s) * (1.0 - s);
  return 2.0 * M * s * (1.0 - s) / (den * den);
}

// Factor precision per kernel: the per-step Neumann downscaling factors in FP32 in both
// mixed modes; the Robin factors (reused by every BF solve and MPM-2P step) only in
// MPM_PREC_FP32_IR_ALL.
bool fp32(const mpm_ctx* c) { return c->prec != MPM_PREC_FP64; }

// Fractional flow f(s) = M s^2 / (M s^2 + (1 - s)^2) (Eq. BL2D) on the host (inflow boundary).
double host_fracflow(double s, double M) {
  const double lw = M * s * s, o = 1.0 - s;
  return lw / (lw + o * o);
}
// Relative change of the transmissibilities up to which a stored float32 downscaling factor is
// kept (0: refactor every step; float64 factors are never kept: nothing refines them).  The
// default keeps factors within 0.5 % on decompositions with at least 4 subdomains per SM
// (over all realisations), where the factorisation competes with the step's other kernels
// for the SMs; on smaller ones it runs beside them for free and a kept factor would only add
// refinement sweeps (measured: 1024^2 and the 256-realisation ensemble 10-13 % faster per
// MPM-2P step, 256^2 6 % slower).
// kappa^n, f(s) and the transmissibilities of the current saturation (k_mobility_eps).
void recompute_derived(mpm_ctx* c) {
  launch_mobility_eps(c->g, c->d, false, c->stream);
  c->derived_stale = false;
}

// Brings them up to date when a pinned-memory mpm_set_saturation left them behind.
void ensure_derived(mpm_ctx* c) {
  if (c->derived_stale && c->have_s && c->have_K) recompute_derived(c);
}

double ds_reuse_tol(const mpm_ctx* c) {
  if (!fp32(c)) return 0.0;
  if (c->ds_reuse >= 0.0) return c->ds_reuse;
  return (long long)c->subs.size() * c->g.R >= 4LL * sm_count() ? 0.005 : 0.0;
}
bool robin_fp32_mode(int prec) { return prec == MPM_PREC_FP32_IR_ALL || prec >= MPM_PREC_TF32_IR; }
bool fp32_robin(const mpm_ctx* c) { return robin_fp32_mode(c->prec); }
// Tensor-core kind of the basis-function solves (0: CUDA cores), k_local_tc.cuh.
int tc_kind(const mpm_ctx* c) {
  return c->prec == MPM_PREC_TF32_IR ? 1 : c->prec == MPM_PREC_TF32X3_IR ? 2 : c->prec == MPM_PREC_BF16_IR ? 3 : 0;
}

cudaEvent_t take_event(mpm_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void prof_begin(mpm_ctx* c, int stage) {
  if (!c->prof) return;
  cudaEvent_t e = take_event(c);
  cudaEventRecord(e, c->stream);
  c->ev_open[stage] = e;
}

void prof_end(mpm_ctx* c, int stage) {
  if (!c->prof || !c->ev_open[stage]) return;
  cudaEvent_t e = take_event(c);
  cudaEventRecord(e, c->stream);
  c->ev_rec[stage].push_back({c->ev_open[stage], e});
  c->ev_open[stage] = nullptr;
}

// ---------------------------------------------------------------------------------------
// Nested dissection tree over the subdomain grid.
struct HostNode {
  int I0, I1, J0, J1;
  int child[2] = {-1, -1};
  int parent = -1;
  int level = 0;
  int leaf_sub = -1;
  std::vector<int> dofs;  // frontal order: separator DOFs, then boundary DOFs
  int nsep = 0;
};

struct Iface {
  int L, dof0, nb;  // length (cells), first global DOF, U DOFs (= P DOFs)
};

int v_id(const mpm_ctx* c, int I, int J) { return J * (c->ncx - 1) + I; }  // between (I,J) and (I+1,J)
int h_id(const mpm_ctx* c, int I, int J) { return c->ncy * (c->ncx - 1) + J * c->ncx + I; }  // (I,J)-(I,J+1)

void append_iface(std::vector<int>& out, const Iface& f) {
  for (int k = 0; k < 2 * f.nb; ++k) out.push_back(f.dof0 + k);
}

int build_tree(mpm_ctx* c, const std::vector<Iface>& ifs, std::vector<HostNode>& hn, int I0, int I1, int J0,
               int J1) {
  const int id = (int)hn.size();
  hn.push_back(HostNode{I0, I1, J0, J1});
  std::vector<int> sep;  // interface ids
  if (I1 - I0 == 1 && J1 - J0 == 1) {
    hn[id].leaf_sub = J0 * c->ncx + I0;
  } else {
    int ch0, ch1;
    if (I1 - I0 >= J1 - J0) {
      const int Im = (I0 + I1) / 2;
      ch0 = build_tree(c, ifs, hn, I0, Im, J0, J1);
      ch1 = build_tree(c, ifs, hn, Im, I1, J0, J1);
      for (int J = J0; J < J1; ++J) sep.push_back(v_id(c, Im - 1, J));
    } else {
      const int Jm = (J0 + J1) / 2;
      ch0 = build_tree(c, ifs, hn, I0, I1, J0, Jm);
      ch1 = build_tree(c, ifs, hn, I0, I1, Jm, J1);
      for (int I = I0; I < I1; ++I) sep.push_back(h_id(c, I, Jm - 1));
    }
    hn[id].child[0] = ch0;
    hn[id].child[1] = ch1;
    hn[ch0].parent = id;
    hn[ch1].parent = id;
    hn[id].level = 1 + std::max(hn[ch0].level, hn[ch1].level);
  }
  // boundary interfaces of the rectangle (interior to the domain)
  std::vector<int> bnd;
  if (hn[id].leaf_sub >= 0) {
    // leaf: subdomain side order left, right, bottom, top
    if (I0 > 0) bnd.push_back(v_id(c, I0 - 1, J0));
    if (I1 < c->ncx) bnd.push_back(v_id(c, I0, J0));
    if (J0 > 0) bnd.push_back(h_id(c, I0, J0 - 1));
    if (J1 < c->ncy) bnd.push_back(h_id(c, I0, J0));
  } else {
    for (int J = J0; J < J1; ++J) {
      if (I0 > 0) bnd.push_back(v_id(c, I0 - 1, J));
      if (I1 < c->ncx) bnd.push_back(v_id(c, I1 - 1, J));
    }
    for (int I = I0; I < I1; ++I) {
      if (J0 > 0) bnd.push_back(h_id(c, I, J0 - 1));
      if (J1 < c->ncy) bnd.push_back(h_id(c, I, J1 - 1));
    }
    std::sort(sep.begin(), sep.end());
    std::sort(bnd.begin(), bnd.end());
  }
  std::vector<int> dofs;
  for (int e : sep) append_iface(dofs, ifs[e]);
  const int nsep = (int)dofs.size();
  for (int e : bnd) append_iface(dofs, ifs[e]);
  hn[id].dofs = dofs;
  hn[id].nsep = nsep;
  return id;
}

void drop_graph(mpm_ctx* c);
int join_branches(mpm_ctx* c, bool factor);
bool late_factor_join(const mpm_ctx* c);

int release_decomposition(mpm_ctx* c) {
  if (!c->dec_allocs.empty()) cudaStreamSynchronize(c->stream);
  drop_graph(c);
  free_list(c->dec_allocs);
  c->d_subs = nullptr;
  c->d_nodes = nullptr;
  c->d_leaf_node = c->d_level_nodes = c->d_srcmap = c->d_pmap = nullptr;
  c->classes.clear();
  c->have_dec = false;
  c->have_basis = false;
  return MPM_OK;
}

// ---------------------------------------------------------------------------------------
// Launch sequences.

// Calls f(grid, count, max_a, max_b) once per width class: the local kernels run one launch
// per padded factor width, each over its class's subdomains (Grid::sub_list).
template <typename F>
void per_class(const mpm_ctx* c, F f) {
  for (const SubClass& k : c->classes) {
    Grid gk = c->g;
    gk.sub_list = c->classes.size() > 1 ? k.d_list : nullptr;
    f(gk, k.count, k.max_a, k.max_b);
  }
}

int run_build(mpm_ctx* c) {
  const Grid& g = c->g;
  DevState& d = c->d;
  cudaStream_t st = c->stream;
  const int nsub = (int)c->subs.size();
  prof_begin(c, MPM_STAGE_BASIS);
  per_class(c, [&](const Grid& gk, int n, int ma, int mb) {
    launch_robin_factor(gk, d, c->d_subs, n, ma, mb, fp32_robin(c), st);
  });
  per_class(c, [&](const Grid& gk, int n, int ma, int mb) {
    launch_basis_solve(gk, d, c->d_subs, n, ma, mb, tc_kind(c), fp32_robin(c), c->ir_tol, c->ir_max, c->d_nodes,
                       c->d_leaf_node, st);
  });
  if (c->n_dof > 0) launch_element_matrix(g, d, c->d_subs, nsub, c->d_nodes, c->d_leaf_node, st);
  prof_end(c, MPM_STAGE_BASIS);
  if (c->n_dof > 0) {
    prof_begin(c, MPM_STAGE_IFACE_FACTOR);
    for (size_t L = 1; L < c->levels.size(); ++L)
      launch_nd_factor_level(g, d, c->d_nodes, c->d_level_nodes + c->lev_off[L], (int)c->levels[L].size(),
                             c->lev_max_nf[L], c->lev_max_nsep[L], c->d_srcmap, st);
    prof_end(c, MPM_STAGE_IFACE_FACTOR);
    // level 1 of the upward sweep with the new fronts, for the rebuilding realisations (the
    // MPM-2P local solve does it for the others, phase::fold_up)
    if (c->levels.size() > 1)
      launch_nd_up(g, d, c->d_nodes, c->d_level_nodes + c->lev_off[1], (int)c->levels[1].size(), c->lev_max_nf[1],
                   c->lev_max_nsep[1], c->d_srcmap, false, c->tune.sweep_terms, st, 1);
  }
  c->fac_prec = c->prec;
  c->have_basis = true;
  return check_launch(c);
}

// MPM-2P local solves: pass 0 the epsilon^0 problem (Eq. mpm_tf_3), pass 1 the first-order
// problem (Eq. mpm_tf_4, l = 1; needs the reconstruction of pass 0).  The interface solve
// that follows uses the same pass.
int run_perturbation(mpm_ctx* c, int pass = 0) {
  const Grid& g = c->g;
  const int nsub = (int)c->subs.size();
  prof_begin(c, MPM_STAGE_PERTURB);
  per_class(c, [&](const Grid& gk, int n, int ma, int mb) {
    launch_mpm_local(gk, c->d, c->d_subs, n, ma, mb, robin_fp32_mode(c->fac_prec), c->ir_tol, c->ir_max, c->d_nodes,
                     c->d_leaf_node, c->tune.local_threads, c->tune.local_stage, pass, c->stream);
  });
  prof_end(c, MPM_STAGE_PERTURB);
  c->next_pass = pass;
  return check_launch(c);
}

// Interface solve: up and down sweeps over the nested-dissection levels, reconstruction.
// The first sweep kernel is fully ordered after what precedes it; the rest of the chain
// (and the downscaling after it, see run_downscale) uses programmatic dependent launch when
// enabled.
int run_interface(mpm_ctx* c, int pass = 0) {
  const Grid& g = c->g;
  DevState& d = c->d;
  cudaStream_t st = c->stream;
  const int nsub = (int)c->subs.size();
  int jrc = join_branches(c, !late_factor_join(c));
  if (jrc) return jrc;
  prof_begin(c, MPM_STAGE_IFACE_SOLVE);
  bool chained = false;
  if (c->n_dof > 0) {
    prof_begin(c, MPM_STAGE_IFACE_UP);
    // level 1 (nodes with two leaf children) was done by the local kernels that wrote the
    // leaves' right-hand sides (phase::fold_up)
    for (size_t L = 2; L < c->levels.size(); ++L) {
      launch_nd_up(g, d, c->d_nodes, c->d_level_nodes + c->lev_off[L], (int)c->levels[L].size(), c->lev_max_nf[L],
                   c->lev_max_nsep[L], c->d_srcmap, chained && c->use_pdl, c->tune.sweep_terms, st);
      chained = true;
    }
    prof_end(c, MPM_STAGE_IFACE_UP);
    // the top level holds the root alone, whose separator values the upward sweep leaves
    // final (no launch); level 1 (nodes with two leaf children) is done inside the
    // reconstruction
    prof_begin(c, MPM_STAGE_IFACE_DOWN);
    for (int L = (int)c->levels.size() - 2; L >= 2; --L)
      launch_nd_down(g, d, c->d_nodes, c->d_level_nodes + c->lev_off[L], (int)c->levels[L].size(),
                     c->lev_max_nsep[L], c->lev_max_nbnd[L], c->d_pmap, c->use_pdl, c->tune.sweep_terms, st);
    prof_end(c, MPM_STAGE_IFACE_DOWN);
  }
  prof_begin(c, MPM_STAGE_RECONSTRUCT);
  // the first-order pass concerns the MPM-2P realisations only (branch 0)
  launch_reconstruct(g, d, c->d_subs, nsub, c->max_face, c->max_dof, c->levels.size() > 1 ? c->lev_max_nf[1] : 0,
                     c->d_nodes, c->d_leaf_node, c->d_pmap, pass == 0 ? -1 : 0, pass, chained && c->use_pdl, st);
  prof_end(c, MPM_STAGE_RECONSTRUCT);
  prof_end(c, MPM_STAGE_IFACE_SOLVE);
  return check_launch(c);
}

// Downscaling factorisation of kappa^n on the side stream (fork): it overlaps whatever the
// main stream runs until join_downscale_factor.
int fork_downscale_factor(mpm_ctx* c) {
  if (c->prof) {  // the stage profiler times the factorisation alone, on the main stream
    prof_begin(c, MPM_STAGE_DS_FACTOR);
    per_class(c, [&](const Grid& gk, int n, int ma, int mb) {
      launch_downscale_factor(gk, c->d, c->d_subs, n, ma, mb, fp32(c), ds_reuse_tol(c), c->stream);
    });
    prof_end(c, MPM_STAGE_DS_FACTOR);
    return check_launch(c);
  }
  CK(cudaEventRecord(c->ev_fork, c->stream));
  CK(cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0));
  per_class(c, [&](const Grid& gk, int n, int ma, int mb) {
    launch_downscale_factor(gk, c->d, c->d_subs, n, ma, mb, fp32(c), ds_reuse_tol(c), c->side_stream);
  });
  CK(cudaEventRecord(c->ev_join, c->side_stream));
  c->factor_forked = true;
  return check_launch(c);
}

// Join every forked branch into the main stream (no-op when none is pending).
int join_branches(mpm_ctx* c, bool factor = true) {
  if (factor && c->factor_forked) CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  if (c->reb_forked) CK(cudaStreamWaitEvent(c->stream, c->ev_reb_join, 0));
  if (factor) c->factor_forked = false;
  c->reb_forked = false;
  return MPM_OK;
}

// A float64 downscaling factorisation takes longer than the perturbation solve: it is joined
// right before the downscaling solve (which then starts without programmatic launch), not
// before the interface solve.
bool late_factor_join(const mpm_ctx* c) { return !fp32(c); }

// Downscaling solve.  after_interface: launched right behind run_interface's chain, whose
// first kernel was ordered after the forked factorisation, so it may use programmatic
// dependent launch (before waiting it reads only the factor).  forked: the factor was forked
// by fork_downscale_factor; otherwise it is computed here on the main stream.
int run_downscale(mpm_ctx* c, bool after_interface, bool forked) {
  const bool joined_before = forked && !c->factor_forked;  // run_interface joined it
  if (forked) {
    int rc = join_branches(c, true);
    if (rc) return rc;
  }
  prof_begin(c, MPM_STAGE_DOWNSCALE);
  if (!forked) {
    per_class(c, [&](const Grid& gk, int n, int ma, int mb) {
      launch_downscale_factor(gk, c->d, c->d_subs, n, ma, mb, fp32(c), ds_reuse_tol(c), c->stream);
    });
  }
  per_class(c, [&](const Grid& gk, int n, int ma, int mb) {
    launch_downscale(gk, c->d, c->d_subs, n, ma, mb, fp32(c), c->ir_tol, c->ir_max,
                     after_interface && joined_before && c->use_pdl, c->tune.ds_threads, c->tune.ds_stage, c->stream);
  });
  prof_end(c, MPM_STAGE_DOWNSCALE);
  return check_launch(c);
}

// n_sub upwind substeps; the last one is fused with kappa^n (and, with decide, with the
// epsilon partial sums and the Algorithm 1 decision, see launch_upwind_kappa; needs a stored
// basis).  The saturation buffers swap at every substep: d.s is the new saturation after.
int run_transport(mpm_ctx* c, double cfl, int n_sub, bool decide, double eta, cudaGraphConditionalHandle h_reb,
                  bool set_handle) {
  prof_begin(c, MPM_STAGE_TRANSPORT);
  c->derived_stale = false;  // the transport writes kappa^n and its transmissibilities of the new saturation
  const double fmax_ = max_fprime(c->g.M);
  for (int k = 0; k < n_sub; ++k) {
    if (k + 1 < n_sub) launch_upwind(c->g, c->d, cfl, fmax_, c->stream);
    else launch_upwind_kappa(c->g, c->d, cfl, fmax_, decide, eta, h_reb, set_handle, c->tune.transport_rows, c->stream);
    std::swap(c->d.s, c->d.s2);
    std::swap(c->d.fs, c->d.fs2);
  }
  prof_end(c, MPM_STAGE_TRANSPORT);
  return check_launch(c);
}

void drop_graph(mpm_ctx* c) {
  for (int k = 0; k < 2; ++k) {
    if (c->graph_exec[k]) cudaGraphExecDestroy(c->graph_exec[k]);
    if (c->graph[k]) cudaGraphDestroy(c->graph[k]);
    c->graph_exec[k] = nullptr;
    c->graph[k] = nullptr;
    c->graph_valid[k] = false;
  }
}

int graph_slot(const mpm_ctx* c) { return c->d.s == c->s_buf0 ? 0 : 1; }

void destroy_streams(mpm_ctx* c) {
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->body_stream) cudaStreamDestroy(c->body_stream);
  if (c->side_stream) cudaStreamDestroy(c->side_stream);
  if (c->reb_stream) cudaStreamDestroy(c->reb_stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_reb_fork) cudaEventDestroy(c->ev_reb_fork);
  if (c->ev_reb_join) cudaEventDestroy(c->ev_reb_join);
  c->cap_stream = c->body_stream = c->side_stream = c->reb_stream = nullptr;
  c->ev_fork = c->ev_join = c->ev_reb_fork = c->ev_reb_join = nullptr;
}

#define CKG(call)                                                                                         \
  do {                                                                                                    \
    cudaError_t e_ = (call);                                                                              \
    if (e_ != cudaSuccess) {                                                                              \
      c->stream = user;                                                                                   \
      c->d = saved;                                                                                       \
      c->factor_forked = c->reb_forked = false;                                                           \
      return fail(c, MPM_ERR_CUDA, "graph capture: %s: %s", #call, cudaGetErrorString(e_));              \
    }                                                                                                     \
  } while (0)

// Capture one pass of the Algorithm 1 loop as a CUDA graph for the current saturation
// buffer parity: transport with kappa^n, the device-side decision and new epsilon; then
// three branches: the downscaling factorisation, IF(any rebuild){basis build}, and the
// perturbation solve (a no-op for rebuilding realisations); joined before the interface
// solve; the downscaling solve.  Kernel arguments (grid data, pointers, eta, cfl, n_sub) are captured by
// value, so setters that change them drop the graph.  The host-side buffer pointers are
// restored after the capture (nothing has run yet).
int build_step_graph(mpm_ctx* c, double eta, double cfl, int n_sub) {
  const int slot = graph_slot(c);
  if (c->graph_exec[slot]) cudaGraphExecDestroy(c->graph_exec[slot]);
  if (c->graph[slot]) cudaGraphDestroy(c->graph[slot]);
  c->graph_exec[slot] = nullptr;
  c->graph[slot] = nullptr;
  c->graph_valid[slot] = false;
  cudaStream_t user = c->stream;
  cudaStream_t cs = c->cap_stream, bs = c->body_stream;
  const bool prof = c->prof;
  const DevState saved = c->d;
  c->prof = false;
  c->stream = cs;
  const long long L0 = g_launches;
  long long Lb[3] = {L0, L0, L0};
  cudaStreamCaptureStatus stt;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndep = 0;
  cudaGraphConditionalHandle h_reb = 0;
  CKG(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  CKG(cudaStreamGetCaptureInfo(cs, &stt, nullptr, &cg, &deps, nullptr, &ndep));
  CKG(cudaGraphConditionalHandleCreate(&h_reb, cg, 0, cudaGraphCondAssignDefault));
  int rc = run_transport(c, cfl, n_sub, true, eta, h_reb, true);
  if (!rc) rc = fork_downscale_factor(c);
  Lb[0] = g_launches;
  if (!rc) {
    // rebuild body: IF(any realisation rebuilds) on its own branch, joined before the
    // interface solve, so that evaluating the condition overlaps the perturbation solve
    cudaStream_t rs = c->reb_stream;
    CKG(cudaEventRecord(c->ev_reb_fork, cs));
    CKG(cudaStreamWaitEvent(rs, c->ev_reb_fork, 0));
    CKG(cudaStreamGetCaptureInfo(rs, &stt, nullptr, &cg, &deps, nullptr, &ndep));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h_reb;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CKG(cudaGraphAddNode(&node, cg, deps, nullptr, ndep, &np));
    CKG(cudaStreamUpdateCaptureDependencies(rs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CKG(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    c->stream = bs;
    rc = run_build(c);
    c->stream = cs;
    cudaGraph_t body_out = nullptr;
    CKG(cudaStreamEndCapture(bs, &body_out));
    CKG(cudaEventRecord(c->ev_reb_join, rs));
    c->reb_forked = true;
  }
  Lb[1] = g_launches;
  // perturbation solve: every realisation's kernel returns at once where it rebuilds
  if (!rc) rc = run_perturbation(c);
  Lb[2] = Lb[1];
  if (!rc) rc = run_interface(c);
  if (!rc && c->g.order >= 1) {  // first-order term (its kernels skip rebuilding realisations)
    rc = run_perturbation(c, 1);
    if (!rc) rc = run_interface(c, 1);
  }
  if (!rc) rc = run_downscale(c, true, true);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  c->stream = user;
  c->prof = prof;
  c->d = saved;
  c->factor_forked = c->reb_forked = false;
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return fail(c, MPM_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  c->graph[slot] = graph;
  e = cudaGraphInstantiate(&c->graph_exec[slot], graph, 0);
  if (e != cudaSuccess) {
    drop_graph(c);
    return fail(c, MPM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  c->graph_valid[slot] = true;
  c->gk_reb = Lb[1] - Lb[0];
  c->gk_mpm = 0;  // the perturbation kernel is launched at every step (counted in gk_base)
  c->gk_base = (g_launches - L0) - c->gk_reb;
  c->capture_launches += g_launches - L0;
  c->g_eta = eta;
  c->g_cfl = cfl;
  c->g_nsub = n_sub;
  return MPM_OK;
}

int need_ready(mpm_ctx* c, bool basis) {
  if (!c->have_K) return fail(c, MPM_ERR_STATE, "permeability not set");
  if (!c->have_dec) return fail(c, MPM_ERR_STATE, "decomposition not set");
  if (!c->have_s) return fail(c, MPM_ERR_STATE, "saturation not set");
  if (basis && !c->have_basis) return fail(c, MPM_ERR_STATE, "no stored basis (call mpm_build_basis or mpm_init)");
  return MPM_OK;
}

}  // namespace

// =======================================================================================
extern "C" {

int mpm_create(mpm_ctx** out, int R, int nx, int ny, double Lx, double Ly, void* stream) {
  if (!out) return MPM_ERR_ARG;
  *out = nullptr;
  if (R < 1 || nx < 1 || ny < 1 || !(Lx > 0) || !(Ly > 0)) return MPM_ERR_ARG;
  if (R > kMaxRealisations) return MPM_ERR_ARG;  // realisations index grid y / z of the launches
  const double hx = Lx / nx, hy = Ly / ny;
  if (std::fabs(hx - hy) > 1e-12 * std::max(hx, hy)) return MPM_ERR_ARG;
  mpm_ctx* c = new mpm_ctx();
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  cudaGetDevice(&c->device);
  Grid& g = c->g;
  g.R = R;
  g.nx = nx;
  g.ny = ny;
  g.h = hx;
  g.bc_type[0] = g.bc_type[1] = MPM_BC_DIRICHLET;
  g.bc_type[2] = g.bc_type[3] = MPM_BC_NEUMANN;
  g.bc_val[0] = 1.0;
  g.bc_val[1] = g.bc_val[2] = g.bc_val[3] = 0.0;
  g.s_inflow = 1.0;
  g.M = 1.0;
  g.f_in = host_fracflow(g.s_inflow, g.M);
  g.seg_len = 1;
  g.inv_seg = 1.0;
  g.degree = 0;
  g.alpha = 1.0;
  g.order = 0;
  g.sub_list = nullptr;
  const size_t nc = (size_t)R * nx * ny;
  DevState& d = c->d;
  int rc = MPM_OK;
  double** cells[] = {&d.K, &d.q, &d.s, &d.s2, &d.kap_n, &d.kap_m, &d.p_m, &d.p_down, &d.fs, &d.fs2, &d.x_ds, &d.dp0};
  for (double** p : cells)
    if ((rc = dalloc_t(c, c->grid_allocs, p, nc)) != MPM_OK) break;
  c->s_buf0 = d.s;
  const int nblk = std::max(1024, upwind_kappa_blocks(g));
  if (rc == MPM_OK) rc = dalloc_t(c, c->grid_allocs, &d.ux, (size_t)R * g.nfx());
  if (rc == MPM_OK) rc = dalloc_t(c, c->grid_allocs, &d.uy, (size_t)R * g.nfy());
  if (rc == MPM_OK) rc = dalloc_t(c, c->grid_allocs, &d.tx, (size_t)R * g.nfx());
  if (rc == MPM_OK) rc = dalloc_t(c, c->grid_allocs, &d.ty, (size_t)R * g.nfy());
  if (rc == MPM_OK) rc = dalloc_t(c, c->grid_allocs, &d.eps, (size_t)R);
  if (rc == MPM_OK) rc = dalloc_t(c, c->grid_allocs, &d.dt, (size_t)R);
  if (rc == MPM_OK) rc = dalloc_t(c, c->grid_allocs, &d.eps_part, (size_t)R * nblk * 2);
  if (rc == MPM_OK) rc = dalloc_t(c, c->grid_allocs, &d.ticket, (size_t)4);
  if (rc == MPM_OK) rc = dalloc_t(c, c->grid_allocs, &d.rebuild, (size_t)R);
  if (rc == MPM_OK) rc = dalloc_t(c, c->grid_allocs, &d.status, 2);  // status word, then the sweep count
  if (rc == MPM_OK) d.ir_iters = d.status + 1;
  if (rc == MPM_OK) rc = dalloc_t(c, c->grid_allocs, &d.counts, 5);
  if (rc == MPM_OK) rc = dalloc_t(c, c->grid_allocs, &d.eps_hist, (size_t)R * kEpsHist);
  if (rc == MPM_OK) rc = dalloc_t(c, c->grid_allocs, &d.reb_hist, (size_t)R * kEpsHist);
  if (rc == MPM_OK) rc = dalloc_t(c, c->grid_allocs, &d.hist_n, 1);
  if (rc == MPM_OK && (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
                       cudaStreamCreateWithFlags(&c->body_stream, cudaStreamNonBlocking) != cudaSuccess ||
                       cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
                       cudaStreamCreateWithFlags(&c->reb_stream, cudaStreamNonBlocking) != cudaSuccess ||
                       cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventCreateWithFlags(&c->ev_reb_fork, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventCreateWithFlags(&c->ev_reb_join, cudaEventDisableTiming) != cudaSuccess))
    rc = MPM_ERR_CUDA;
  if (rc == MPM_OK && cudaMallocHost(&c->h_flags, sizeof(int) * R) != cudaSuccess) rc = MPM_ERR_OOM;
  if (rc == MPM_OK && cudaMallocHost(&c->h_status, sizeof(int) * 4) != cudaSuccess) rc = MPM_ERR_OOM;
  if (rc == MPM_OK && cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->h_status_dev), c->h_status, 0) != cudaSuccess)
    rc = MPM_ERR_CUDA;
  if (rc != MPM_OK) {
    destroy_streams(c);
    free_list(c->grid_allocs);
    if (c->h_flags) cudaFreeHost(c->h_flags);
    delete c;
    return rc;
  }
  cudaStreamSynchronize(c->stream);
  c->launches0 = g_launches;
  *out = c;
  return MPM_OK;
}

int mpm_destroy(mpm_ctx* c) {
  if (!c) return MPM_OK;
  cudaStreamSynchronize(c->stream);
  for (int k = 0; k < MPM_NSTAGES; ++k) {
    for (auto& pr : c->ev_rec[k]) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    if (c->ev_open[k]) cudaEventDestroy(c->ev_open[k]);
  }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  drop_graph(c);
  if (c->side_stream) cudaStreamSynchronize(c->side_stream);
  destroy_streams(c);
  release_decomposition(c);
  free_list(c->grid_allocs);
  if (c->h_flags) cudaFreeHost(c->h_flags);
  if (c->h_status) cudaFreeHost(c->h_status);
  delete c;
  return MPM_OK;
}

const char* mpm_last_error(const mpm_ctx* c) { return c ? c->err.c_str() : "null context"; }

int mpm_set_precision(mpm_ctx* c, int mode, double ir_tol, int ir_max) {
  if (!c) return MPM_ERR_ARG;
  if (mode < MPM_PREC_FP64 || mode > MPM_PREC_BF16_IR)
    return fail(c, MPM_ERR_ARG, "unknown precision mode %d", mode);
  if (!(ir_tol > 0) || ir_max < 1 || ir_max > 1000) return fail(c, MPM_ERR_ARG, "need ir_tol > 0 and 1 <= ir_max <= 1000");
  c->prec = mode;
  c->ir_tol = ir_tol;
  c->ir_max = ir_max;
  c->have_basis = false;  // the stored factors have the old type
  if (c->have_dec && c->d.npin)  // so do the stored downscaling factors
    CK(cudaMemsetAsync(c->d.npin, 0xff, (size_t)c->g.R * c->subs.size() * sizeof(int), c->stream));
  drop_graph(c);
  return MPM_OK;
}

int mpm_set_permeability(mpm_ctx* c, const double* K, int mem) {
  if (!c) return MPM_ERR_ARG;
  const size_t n = (size_t)c->g.R * c->g.nx * c->g.ny;
  if (mem == MPM_MEM_HOST && K) {
    for (size_t i = 0; i < n; ++i)
      if (!(K[i] > 0) || !std::isfinite(K[i])) return fail(c, MPM_ERR_ARG, "permeability must be positive and finite (index %zu)", i);
  }
  int rc = copy_in(c, c->d.K, K, n, mem);
  if (rc) return rc;
  c->have_K = true;
  if (c->have_s) recompute_derived(c);
  return check_launch(c);
}

int mpm_set_source(mpm_ctx* c, const double* q, int mem) {
  if (!c) return MPM_ERR_ARG;
  const size_t n = (size_t)c->g.R * c->g.nx * c->g.ny;
  if (!q) {
    CK(cudaMemsetAsync(c->d.q, 0, n * sizeof(double), c->stream));
    return MPM_OK;
  }
  return copy_in(c, c->d.q, q, n, mem);
}

int mpm_set_fluids(mpm_ctx* c, double M) {
  if (!c) return MPM_ERR_ARG;
  if (!(M > 0) || !std::isfinite(M)) return fail(c, MPM_ERR_ARG, "viscosity ratio must be positive");
  c->g.M = M;
  c->g.f_in = host_fracflow(c->g.s_inflow, M);
  drop_graph(c);
  if (c->have_s && c->have_K) recompute_derived(c);
  return check_launch(c);
}

int mpm_set_boundary(mpm_ctx* c, const int type[4], const double val[4], double s_inflow) {
  if (!c) return MPM_ERR_ARG;
  if (!type || !val) return fail(c, MPM_ERR_ARG, "null boundary arrays");
  bool any_d = false;
  for (int k = 0; k < 4; ++k) {
    if (type[k] != MPM_BC_DIRICHLET && type[k] != MPM_BC_NEUMANN) return fail(c, MPM_ERR_ARG, "bad boundary type on side %d", k);
    if (!std::isfinite(val[k])) return fail(c, MPM_ERR_ARG, "boundary value must be finite");
    any_d |= type[k] == MPM_BC_DIRICHLET;
  }
  if (!any_d) return fail(c, MPM_ERR_ARG, "at least one side must be Dirichlet");
  if (!(s_inflow >= 0 && s_inflow <= 1)) return fail(c, MPM_ERR_ARG, "s_inflow must be in [0,1]");
  for (int k = 0; k < 4; ++k) {
    c->g.bc_type[k] = type[k];
    c->g.bc_val[k] = val[k];
  }
  c->g.s_inflow = s_inflow;
  c->g.f_in = host_fracflow(s_inflow, c->g.M);
  c->have_basis = false;
  drop_graph(c);
  return MPM_OK;
}

int mpm_set_decomposition(mpm_ctx* c, int ncx, const int* col_w, int ncy, const int* row_h, int seg_len, int degree,
                          double alpha, const double* alpha_face) {
  if (!c) return MPM_ERR_ARG;
  if (ncx < 1 || ncy < 1 || !col_w || !row_h) return fail(c, MPM_ERR_ARG, "bad decomposition arrays");
  if (seg_len < 1 || (degree != 0 && degree != 1) || !(alpha > 0) || !std::isfinite(alpha))
    return fail(c, MPM_ERR_ARG, "need seg_len >= 1, degree in {0,1}, alpha > 0");
  if (degree == 1 && seg_len < 2)  // a linear function sampled at one edge midpoint vanishes
    return fail(c, MPM_ERR_ARG, "degree 1 needs seg_len >= 2");
  long long sx = 0, sy = 0;
  for (int I = 0; I < ncx; ++I) {
    if (col_w[I] < 1 || col_w[I] > kMaxSide || col_w[I] % seg_len)
      return fail(c, MPM_ERR_ARG, "column width %d must be in [1,%d] and a multiple of seg_len", col_w[I], kMaxSide);
    sx += col_w[I];
  }
  for (int J = 0; J < ncy; ++J) {
    if (row_h[J] < 1 || row_h[J] > kMaxSide || row_h[J] % seg_len)
      return fail(c, MPM_ERR_ARG, "row height %d must be in [1,%d] and a multiple of seg_len", row_h[J], kMaxSide);
    sy += row_h[J];
  }
  if (sx != c->g.nx || sy != c->g.ny) return fail(c, MPM_ERR_ARG, "widths/heights must sum to nx/ny");
  // alpha per interface face (x faces [ny][nx+1], then y faces [ny+1][nx]); checked on the
  // interface faces, the only ones read
  const long long nfx = (long long)c->g.ny * (c->g.nx + 1);
  auto alpha_at = [&](bool xface, int j, int i) {
    if (!alpha_face) return alpha;
    return xface ? alpha_face[(long long)j * (c->g.nx + 1) + i] : alpha_face[nfx + (long long)j * c->g.nx + i];
  };
  if (alpha_face) {
    for (int I = 1, x = col_w[0]; I < ncx; x += col_w[I], ++I)
      for (int j = 0; j < c->g.ny; ++j)
        if (!(alpha_at(true, j, x) > 0) || !std::isfinite(alpha_at(true, j, x)))
          return fail(c, MPM_ERR_ARG, "alpha must be positive and finite on interface x-face (%d, %d)", x, j);
    for (int J = 1, y = row_h[0]; J < ncy; y += row_h[J], ++J)
      for (int i = 0; i < c->g.nx; ++i)
        if (!(alpha_at(false, y, i) > 0) || !std::isfinite(alpha_at(false, y, i)))
          return fail(c, MPM_ERR_ARG, "alpha must be positive and finite on interface y-face (%d, %d)", i, y);
  }
  release_decomposition(c);
  c->ncx = ncx;
  c->ncy = ncy;
  c->col_w.assign(col_w, col_w + ncx);
  c->row_h.assign(row_h, row_h + ncy);
  Grid& g = c->g;
  g.seg_len = seg_len;
  g.inv_seg = 1.0 / seg_len;
  g.degree = degree;
  g.alpha = alpha;
  // interfaces
  const int nv = ncy * (ncx - 1), nh = (ncy - 1) * ncx;
  std::vector<Iface> ifs(nv + nh);
  int off = 0;
  for (int e = 0; e < nv + nh; ++e) {
    int L;
    if (e < nv) L = row_h[e / (ncx - 1)];
    else L = col_w[(e - nv) % ncx];
    const int nb = (L / seg_len) * (degree + 1);
    ifs[e] = Iface{L, off, nb};
    off += 2 * nb;
  }
  c->n_dof = off;
  // subdomains
  std::vector<int> xo(ncx + 1, 0), yo(ncy + 1, 0);
  for (int I = 0; I < ncx; ++I) xo[I + 1] = xo[I] + col_w[I];
  for (int J = 0; J < ncy; ++J) yo[J + 1] = yo[J] + row_h[J];
  c->subs.assign(ncx * ncy, DevSub{});
  long long q_off = 0, t_off = 0, tr_off = 0, pf_off = 0;
  int dof_off = 0, face_off = 0, cell_off = 0;
  c->max_a = c->max_b = c->max_dof = c->max_face = 0;
  c->n_hat = 0;
  std::vector<double> rho_host;  // per subdomain face, in face order (left, right, bottom, top)
  for (int J = 0; J < ncy; ++J) {
    for (int I = 0; I < ncx; ++I) {
      DevSub& s = c->subs[J * ncx + I];
      s.x0 = xo[I];
      s.y0 = yo[J];
      s.a = col_w[I];
      s.b = row_h[J];
      const int ids[4] = {I > 0 ? v_id(c, I - 1, J) : -1, I < ncx - 1 ? v_id(c, I, J) : -1,
                          J > 0 ? h_id(c, I, J - 1) : -1, J < ncy - 1 ? h_id(c, I, J) : -1};
      const int nbr[4] = {I > 0 ? J * ncx + I - 1 : -1, I < ncx - 1 ? J * ncx + I + 1 : -1,
                          J > 0 ? (J - 1) * ncx + I : -1, J < ncy - 1 ? (J + 1) * ncx + I : -1};
      const double sgn[4] = {-1.0, 1.0, -1.0, 1.0};
      int nd = 0;
      for (int q = 0; q < 4; ++q) {
        s.side_iface[q] = ids[q];
        s.side_nbr[q] = nbr[q];
        s.side_sign[q] = sgn[q];
        const int len = q < 2 ? s.b : s.a;
        if (ids[q] >= 0) {
          s.side_kind[q] = 1;
          s.side_dof0[q] = nd;
          s.side_nb[q] = ifs[ids[q]].nb;
          nd += 2 * ifs[ids[q]].nb;
          // rho_e = alpha_e H_e / h of each face of the side (H_e: the interface length)
          for (int t = 0; t < len; ++t) {
            const double ae = q == 0   ? alpha_at(true, s.y0 + t, s.x0)
                              : q == 1 ? alpha_at(true, s.y0 + t, s.x0 + s.a)
                              : q == 2 ? alpha_at(false, s.y0, s.x0 + t)
                                       : alpha_at(false, s.y0 + s.b, s.x0 + t);
            rho_host.push_back(ae * ifs[ids[q]].L);
          }
        } else {
          s.side_kind[q] = 0;
          s.side_dof0[q] = nd;
          s.side_nb[q] = 0;
          for (int t = 0; t < len; ++t) rho_host.push_back(0.0);
        }
      }
      s.ndof = nd;
      s.dof_off = dof_off;
      s.face_off = face_off;
      s.cell_off = cell_off;
      const int m = s.a * s.b, nface = 2 * (s.a + s.b);
      s.q_off = q_off;
      s.t_off = t_off;
      s.tr_off = tr_off;
      s.pf_off = pf_off;
      s.A = pad_width(s.a);
      q_off += (long long)s.b * s.A * s.A;
      t_off += 4LL * m;
      tr_off += (long long)nface * nd;
      pf_off += (long long)m * (nd + 1);
      dof_off += nd;
      face_off += nface;
      cell_off += m;
      c->max_a = std::max(c->max_a, s.a);
      c->max_b = std::max(c->max_b, s.b);
      c->max_dof = std::max(c->max_dof, nd);
      c->max_face = std::max(c->max_face, nface);
      c->n_hat += nd;
    }
  }
  // width classes of the local kernels (Grid::sub_list): one per padded width present
  std::vector<std::vector<int>> cls_lists;
  c->classes.clear();
  for (int A : {8, 16, 32}) {
    SubClass k{A, 0, 0, 0, nullptr};
    std::vector<int> lst;
    for (int i = 0; i < (int)c->subs.size(); ++i)
      if (c->subs[i].A == A) {
        lst.push_back(i);
        k.max_a = std::max(k.max_a, c->subs[i].a);
        k.max_b = std::max(k.max_b, c->subs[i].b);
      }
    if (lst.empty()) continue;
    k.count = (int)lst.size();
    c->classes.push_back(k);
    cls_lists.push_back(lst);
  }
  // nested dissection tree
  std::vector<HostNode> hn;
  build_tree(c, ifs, hn, 0, ncx, 0, ncy);
  const int nn = (int)hn.size();
  int nlev = 0;
  for (auto& n : hn) nlev = std::max(nlev, n.level + 1);
  c->levels.assign(nlev, {});
  for (int i = 0; i < nn; ++i) c->levels[hn[i].level].push_back(i);
  c->nodes.assign(nn, DevNode{});
  c->leaf_node.assign(ncx * ncy, -1);
  std::vector<int> srcmap, pmap;
  long long f_off = 0, v_off = 0;
  for (int i = 0; i < nn; ++i) {
    DevNode& dn = c->nodes[i];
    const HostNode& h = hn[i];
    dn.nf = (int)h.dofs.size();
    dn.nsep = h.nsep;
    dn.nbnd = dn.nf - dn.nsep;
    dn.leaf_sub = h.leaf_sub;
    dn.child[0] = h.child[0];
    dn.child[1] = h.child[1];
    dn.parent = h.parent;
    dn.level = h.level;
    dn.f_off = f_off;
    dn.v_off = v_off;
    f_off += (long long)dn.nf * dn.nf;
    v_off += dn.nf;
    if (h.leaf_sub >= 0) {
      c->leaf_node[h.leaf_sub] = i;
      if (dn.nf != c->subs[h.leaf_sub].ndof) return fail(c, MPM_ERR_ARG, "internal: leaf DOF mismatch");
    }
    dn.src_off = (int)srcmap.size();
    if (h.child[0] >= 0) {
      for (int ch = 0; ch < 2; ++ch) {
        const HostNode& hc = hn[h.child[ch]];
        std::map<int, int> pos;
        for (int k = hc.nsep; k < (int)hc.dofs.size(); ++k) pos[hc.dofs[k]] = k - hc.nsep;
        for (int k = 0; k < dn.nf; ++k) {
          auto it = pos.find(h.dofs[k]);
          srcmap.push_back(it == pos.end() ? -1 : it->second);
        }
      }
    }
  }
  for (int i = 0; i < nn; ++i) {
    DevNode& dn = c->nodes[i];
    const HostNode& h = hn[i];
    dn.pmap_off = (int)pmap.size();
    if (h.parent >= 0) {
      std::map<int, int> pos;
      const HostNode& hp = hn[h.parent];
      for (int k = 0; k < (int)hp.dofs.size(); ++k) pos[hp.dofs[k]] = k;
      for (int k = h.nsep; k < (int)h.dofs.size(); ++k) {
        auto it = pos.find(h.dofs[k]);
        if (it == pos.end()) return fail(c, MPM_ERR_ARG, "internal: boundary DOF missing in parent");
        pmap.push_back(it->second);
      }
    }
  }
  std::vector<int> level_nodes;
  c->lev_off.assign(nlev, 0);
  c->lev_max_nf.assign(nlev, 0);
  c->lev_max_nsep.assign(nlev, 0);
  c->lev_max_nbnd.assign(nlev, 0);
  long long st_lvl = 1;
  for (int L = 0; L < nlev; ++L) {
    c->lev_off[L] = (int)level_nodes.size();
    for (int i : c->levels[L]) {
      level_nodes.push_back(i);
      c->lev_max_nf[L] = std::max(c->lev_max_nf[L], c->nodes[i].nf);
      c->lev_max_nsep[L] = std::max(c->lev_max_nsep[L], c->nodes[i].nsep);
      c->lev_max_nbnd[L] = std::max(c->lev_max_nbnd[L], c->nodes[i].nbnd);
    }
    st_lvl = std::max(st_lvl, (long long)c->levels[L].size());
  }
  if (srcmap.empty()) srcmap.push_back(-1);
  if (pmap.empty()) pmap.push_back(-1);
  // device pools
  DevState& d = c->d;
  const int R = g.R, nsub = ncx * ncy;
  d.st_fac = q_off;
  d.st_t = t_off;
  d.st_tr = tr_off;
  d.st_pf = pf_off;
  d.st_dof = dof_off;
  d.st_face = face_off;
  d.st_sub = nsub;
  d.st_front = f_off;
  d.st_vec = v_off;
  d.st_col = v_off * kPivotChunk;
  d.st_lvl = st_lvl;
  d.st_nodes = nn;
  auto& A = c->dec_allocs;
  int rc = MPM_OK;
  if (!rc) rc = dalloc(c, A, &d.fac, (size_t)R * q_off * sizeof(double));
  if (!rc) rc = dalloc_t(c, A, &d.tvec, (size_t)R * t_off);
  if (!rc) rc = dalloc(c, A, &d.nfac, (size_t)R * q_off * sizeof(double));
  if (!rc) rc = dalloc_t(c, A, &d.ntvec, (size_t)R * t_off);
  if (!rc) rc = dalloc_t(c, A, &d.nfw, (size_t)R * t_off);
  if (!rc) rc = dalloc_t(c, A, &d.npin, (size_t)R * nsub);
  if (!rc) rc = dalloc_t(c, A, &d.npin_k, (size_t)R * nsub);
  if (!rc) rc = dalloc_t(c, A, &d.tr, (size_t)R * tr_off);
  if (!rc) rc = dalloc_t(c, A, &d.pf, (size_t)R * pf_off);
  if (!rc) rc = dalloc_t(c, A, &d.mu_hat, (size_t)R * dof_off);
  if (!rc) rc = dalloc_t(c, A, &d.fbar, (size_t)R * face_off);
  if (!rc) rc = dalloc_t(c, A, &d.trace, (size_t)R * face_off);
  if (!rc) rc = dalloc_t(c, A, &d.trace1, (size_t)R * face_off);
  if (!rc) rc = dalloc_t(c, A, &d.bhat, (size_t)R * face_off);
  if (!rc) rc = dalloc_t(c, A, &d.rho_f, (size_t)face_off);
  if (!rc) rc = dalloc_t(c, A, &d.sub_mean, (size_t)R * nsub);
  if (!rc) rc = dalloc_t(c, A, &d.sub_target, (size_t)R * nsub);
  if (!rc) rc = dalloc_t(c, A, &d.pm_mean, (size_t)R * nsub);
  if (!rc) rc = dalloc_t(c, A, &d.rate_part, (size_t)R * nsub);
  if (!rc) rc = dalloc_t(c, A, &d.rate_max, (size_t)R);
  if (!rc) rc = dalloc_t(c, A, &d.inv_rate, (size_t)R);
  if (!rc) rc = dalloc_t(c, A, &d.front, (size_t)R * f_off);
  if (!rc) rc = dalloc_t(c, A, &d.gvec, (size_t)R * v_off);
  if (!rc) rc = dalloc_t(c, A, &d.xvec, (size_t)R * v_off);
  if (!rc) rc = dalloc_t(c, A, &d.pivinv, (size_t)R * st_lvl * kPivotChunk * kPivotChunk);
  if (!rc) rc = dalloc_t(c, A, &d.colold, (size_t)R * d.st_col);
  if (!rc) rc = dalloc_t(c, A, &c->d_subs, (size_t)nsub);
  if (!rc) rc = dalloc_t(c, A, &c->d_nodes, (size_t)nn);
  if (!rc) rc = dalloc_t(c, A, &d.nd_ticket, (size_t)R * nn);  // zeroed
  if (!rc) rc = dalloc_t(c, A, &c->d_leaf_node, (size_t)nsub);
  if (!rc) rc = dalloc_t(c, A, &c->d_level_nodes, level_nodes.size());
  if (!rc) rc = dalloc_t(c, A, &c->d_srcmap, srcmap.size());
  if (!rc) d.srcmap = c->d_srcmap;
  if (!rc) rc = dalloc_t(c, A, &c->d_pmap, pmap.size());
  if (c->classes.size() > 1)
    for (size_t k = 0; k < c->classes.size() && !rc; ++k) rc = dalloc_t(c, A, &c->classes[k].d_list, cls_lists[k].size());
  if (rc) {
    release_decomposition(c);
    return rc;
  }
  CK(cudaMemsetAsync(d.npin, 0xff, (size_t)R * nsub * sizeof(int), c->stream));  // no stored factor: -1
  CK(cudaMemcpyAsync(c->d_subs, c->subs.data(), nsub * sizeof(DevSub), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(d.rho_f, rho_host.data(), rho_host.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  if (c->classes.size() > 1)
    for (size_t k = 0; k < c->classes.size(); ++k)
      CK(cudaMemcpyAsync(c->classes[k].d_list, cls_lists[k].data(), cls_lists[k].size() * sizeof(int),
                         cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_nodes, c->nodes.data(), nn * sizeof(DevNode), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_leaf_node, c->leaf_node.data(), nsub * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_level_nodes, level_nodes.data(), level_nodes.size() * sizeof(int), cudaMemcpyHostToDevice,
                     c->stream));
  CK(cudaMemcpyAsync(c->d_srcmap, srcmap.data(), srcmap.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_pmap, pmap.data(), pmap.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->have_dec = true;
  c->have_basis = false;
  c->stats.interface_dofs = c->n_dof;
  c->stats.subdomains = nsub;
  c->stats.n_hat = c->n_hat;
  return MPM_OK;
}

int mpm_set_saturation(mpm_ctx* c, const double* s, int mem) {
  if (!c) return MPM_ERR_ARG;
  const size_t n = (size_t)c->g.R * c->g.nx * c->g.ny;
  if (mem == MPM_MEM_HOST && s && c->have_K && pinned_device_ptr(s)) {
    // Pinned memory: one kernel loads the values into the scratch saturation, range-checks
    // them and writes their f(s) into the scratch f buffer; when every value lies in [0,1] the
    // current and scratch buffers swap (the step graph of the other buffer parity serves
    // from then on).  kappa^n and the transmissibilities are left for the next step's
    // transport (which recomputes them from the new saturation) or for ensure_derived.
    volatile int* flag = reinterpret_cast<volatile int*>(c->h_status) + 2;
    *flag = 0;
    launch_load_checked_fs(static_cast<const double*>(pinned_device_ptr(s)), c->d.s2, c->d.fs2, (long long)n, c->g.M,
                           c->h_status_dev + 2, c->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    if (*flag != 0)
      for (size_t i = 0; i < n; ++i)
        if (!(s[i] >= 0 && s[i] <= 1)) return fail(c, MPM_ERR_ARG, "saturation must lie in [0,1] (index %zu)", i);
    std::swap(c->d.s, c->d.s2);
    std::swap(c->d.fs, c->d.fs2);
    c->have_s = true;
    c->derived_stale = true;
    return MPM_OK;
  }
  if (mem == MPM_MEM_HOST && s) {
    // The copy goes to the scratch saturation buffer (every step writes it before reading
    // it) and is range-checked on the way; the current saturation is replaced, by a device
    // copy, only when every value lies in [0,1].  Pinned memory is read by a kernel that
    // also checks the values; other host memory takes a copy while the host checks them.
    size_t bad = 0;
    if (void* ds = pinned_device_ptr(s)) {
      volatile int* flag = reinterpret_cast<volatile int*>(c->h_status) + 2;
      *flag = 0;
      launch_load_checked(static_cast<const double*>(ds), c->d.s2, (long long)n, c->h_status_dev + 2, c->stream);
      CK(cudaGetLastError());
      CK(cudaStreamSynchronize(c->stream));
      bad = *flag != 0;
    } else {
      CK(cudaMemcpyAsync(c->d.s2, s, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      for (size_t i = 0; i < n; ++i) bad += !(s[i] >= 0 && s[i] <= 1);  // branch-free (vectorises)
      CK(cudaStreamSynchronize(c->stream));  // the caller's buffer is free again
    }
    if (bad)  // locate the first offender
      for (size_t i = 0; i < n; ++i)
        if (!(s[i] >= 0 && s[i] <= 1)) return fail(c, MPM_ERR_ARG, "saturation must lie in [0,1] (index %zu)", i);
    CK(cudaMemcpyAsync(c->d.s, c->d.s2, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  } else {
    int rc = copy_in(c, c->d.s, s, n, mem);
    if (rc) return rc;
  }
  c->have_s = true;
  if (c->have_K) recompute_derived(c);
  return check_launch(c);
}

int mpm_build_basis(mpm_ctx* c) {
  if (!c) return MPM_ERR_ARG;
  int rc = need_ready(c, false);
  if (rc) return rc;
  ensure_derived(c);
  launch_fill_flags(c->g, c->d, 1, c->stream);
  return run_build(c);
}

int mpm_eval_epsilon(mpm_ctx* c, double* eps) {
  if (!c) return MPM_ERR_ARG;
  int rc = need_ready(c, true);
  if (rc) return rc;
  launch_mobility_eps(c->g, c->d, true, c->stream);
  c->derived_stale = false;
  if ((rc = check_launch(c))) return rc;
  if (eps) return copy_out(c, eps, c->d.eps, c->g.R, MPM_MEM_HOST);
  return MPM_OK;
}

int mpm_choose(mpm_ctx* c, double eta, int* rebuild) {
  if (!c) return MPM_ERR_ARG;
  if (!std::isfinite(eta)) return fail(c, MPM_ERR_ARG, "eta must be finite");
  launch_choose(c->g, c->d, eta, c->stream);
  int rc = check_launch(c);
  if (rc) return rc;
  if (rebuild) {
    CK(cudaMemcpyAsync(rebuild, c->d.rebuild, sizeof(int) * c->g.R, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return MPM_OK;
}

int mpm_perturbation_solve(mpm_ctx* c) {
  if (!c) return MPM_ERR_ARG;
  int rc = need_ready(c, true);
  if (rc) return rc;
  ensure_derived(c);
  launch_fill_flags(c->g, c->d, 0, c->stream);
  return run_perturbation(c);
}

int mpm_perturbation_correction(mpm_ctx* c) {
  if (!c) return MPM_ERR_ARG;
  int rc = need_ready(c, true);
  if (rc) return rc;
  ensure_derived(c);
  if (c->g.order < 1) return fail(c, MPM_ERR_STATE, "the first-order term needs mpm_set_mpm_order(ctx, 1)");
  launch_fill_flags(c->g, c->d, 0, c->stream);
  return run_perturbation(c, 1);
}

int mpm_set_mpm_order(mpm_ctx* c, int order) {
  if (!c) return MPM_ERR_ARG;
  if (order != 0 && order != 1) return fail(c, MPM_ERR_ARG, "order must be 0 or 1");
  c->g.order = order;
  drop_graph(c);
  return MPM_OK;
}

int mpm_interface_solve(mpm_ctx* c) {
  if (!c) return MPM_ERR_ARG;
  int rc = need_ready(c, true);
  if (rc) return rc;
  ensure_derived(c);
  const int pass = c->next_pass;
  c->next_pass = 0;
  return run_interface(c, pass);
}

int mpm_downscale(mpm_ctx* c) {
  if (!c) return MPM_ERR_ARG;
  int rc = need_ready(c, true);
  if (rc) return rc;
  ensure_derived(c);
  return run_downscale(c, false, false);
}

int mpm_saturation_step(mpm_ctx* c, double cfl, int n_sub, double* dt) {
  if (!c) return MPM_ERR_ARG;
  if (!(cfl > 0 && cfl <= 1) || n_sub < 1) return fail(c, MPM_ERR_ARG, "need 0 < cfl <= 1 and n_sub >= 1");
  int rc = need_ready(c, false);
  if (rc) return rc;
  if ((rc = run_transport(c, cfl, n_sub, false, 0.0, 0, false))) return rc;
  if (dt) return copy_out(c, dt, c->d.dt, c->g.R, MPM_MEM_HOST);
  return MPM_OK;
}

int mpm_init(mpm_ctx* c, double eta) {
  if (!c) return MPM_ERR_ARG;
  if (!std::isfinite(eta)) return fail(c, MPM_ERR_ARG, "eta must be finite");
  int rc = need_ready(c, false);
  if (rc) return rc;
  recompute_derived(c);
  launch_fill_flags(c->g, c->d, 1, c->stream);
  // a fresh start: no stored downscaling factor is kept (their type may have changed)
  CK(cudaMemsetAsync(c->d.npin, 0xff, (size_t)c->g.R * c->subs.size() * sizeof(int), c->stream));
  if ((rc = fork_downscale_factor(c))) return rc;
  if ((rc = run_build(c))) return rc;
  if ((rc = run_interface(c))) return rc;
  if ((rc = run_downscale(c, true, true))) return rc;
  std::vector<double> e(c->g.R, eta);
  CK(cudaMemcpyAsync(c->d.eps, e.data(), sizeof(double) * c->g.R, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->init_rebuilds += c->g.R;
  return MPM_OK;
}

int mpm_step(mpm_ctx* c, double eta, double cfl, int n_sub) {
  if (!c) return MPM_ERR_ARG;
  if (!(cfl > 0 && cfl <= 1) || n_sub < 1 || !std::isfinite(eta))
    return fail(c, MPM_ERR_ARG, "need 0 < cfl <= 1, n_sub >= 1 and finite eta");
  int rc = need_ready(c, true);
  if (rc) return rc;
  if (c->use_graph && !c->prof) {
    if (c->g_eta != eta || c->g_cfl != cfl || c->g_nsub != n_sub) drop_graph(c);
    const int slot = graph_slot(c);
    if (!c->graph_valid[slot] && (rc = build_step_graph(c, eta, cfl, n_sub))) return rc;
    CK(cudaGraphLaunch(c->graph_exec[slot], c->stream));
    c->derived_stale = false;  // its transport wrote kappa^n and the transmissibilities
    if (n_sub & 1) {  // the graph left the new saturation in the other buffer
      std::swap(c->d.s, c->d.s2);
      std::swap(c->d.fs, c->d.fs2);
    }
    c->stats.steps += 1;
    c->graph_steps += 1;
    return MPM_OK;
  }
  // eager path: the host reads the device decision to skip the branch nobody takes
  if ((rc = run_transport(c, cfl, n_sub, true, eta, 0, false))) return rc;
  if ((rc = fork_downscale_factor(c))) return rc;
  CK(cudaMemcpyAsync(c->h_flags, c->d.rebuild, sizeof(int) * c->g.R, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  int nreb = 0;
  for (int r = 0; r < c->g.R; ++r) nreb += c->h_flags[r] != 0;
  if (nreb > 0 && (rc = run_build(c))) return rc;
  if (nreb < c->g.R && (rc = run_perturbation(c))) return rc;
  if ((rc = run_interface(c))) return rc;
  if (nreb < c->g.R && c->g.order >= 1) {
    if ((rc = run_perturbation(c, 1))) return rc;
    if ((rc = run_interface(c, 1))) return rc;
  }
  if ((rc = run_downscale(c, true, true))) return rc;
  c->stats.steps += 1;
  return check_launch(c);
}

int mpm_set_downscale_reuse(mpm_ctx* c, double tol) {
  if (!c) return MPM_ERR_ARG;
  if (!(tol <= 0.5)) return fail(c, MPM_ERR_ARG, "need tol <= 0.5 (negative: the default)");
  c->ds_reuse = tol;
  drop_graph(c);
  return MPM_OK;
}

int mpm_set_execution(mpm_ctx* c, int flags) {
  if (!c) return MPM_ERR_ARG;
  if (flags & ~(MPM_EXEC_GRAPH | MPM_EXEC_PDL)) return fail(c, MPM_ERR_ARG, "unknown execution flags %d", flags);
  c->use_graph = (flags & MPM_EXEC_GRAPH) != 0;
  c->use_pdl = (flags & MPM_EXEC_PDL) != 0;
  drop_graph(c);
  return MPM_OK;
}

int mpm_get_pressure(mpm_ctx* c, double* p, int which, int mem) {
  if (!c) return MPM_ERR_ARG;
  const size_t n = (size_t)c->g.R * c->g.nx * c->g.ny;
  if (which == MPM_P_MRCM) return copy_out(c, p, c->d.p_m, n, mem);
  if (which == MPM_P_DOWNSCALED) return copy_out(c, p, c->d.p_down, n, mem);
  return fail(c, MPM_ERR_ARG, "which must be MPM_P_MRCM or MPM_P_DOWNSCALED");
}

int mpm_get_flux(mpm_ctx* c, double* ux, double* uy, int mem) {
  if (!c) return MPM_ERR_ARG;
  int rc = copy_out(c, ux, c->d.ux, (size_t)c->g.R * c->g.nfx(), mem);
  if (rc) return rc;
  return copy_out(c, uy, c->d.uy, (size_t)c->g.R * c->g.nfy(), mem);
}

int mpm_get_saturation(mpm_ctx* c, double* s, int mem) {
  if (!c) return MPM_ERR_ARG;
  return copy_out(c, s, c->d.s, (size_t)c->g.R * c->g.nx * c->g.ny, mem);
}

int mpm_get_conductivity(mpm_ctx* c, double* kappa, int mem) {
  if (!c) return MPM_ERR_ARG;
  ensure_derived(c);
  return copy_out(c, kappa, c->d.kap_n, (size_t)c->g.R * c->g.nx * c->g.ny, mem);
}

int mpm_get_stats(mpm_ctx* c, mpm_stats* out) {
  if (!c || !out) return MPM_ERR_ARG;
  int rc = sync_status(c);
  std::vector<double> e(c->g.R), dt(c->g.R);
  CK(cudaMemcpy(e.data(), c->d.eps, sizeof(double) * c->g.R, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(dt.data(), c->d.dt, sizeof(double) * c->g.R, cudaMemcpyDeviceToHost));
  c->stats.last_eps_max = *std::max_element(e.begin(), e.end());
  c->stats.last_dt_min = *std::min_element(dt.begin(), dt.end());
  long long cnt[5] = {0, 0, 0, 0, 0};
  CK(cudaMemcpy(cnt, c->d.counts, sizeof(cnt), cudaMemcpyDeviceToHost));
  c->stats.ds_factorisations = cnt[4];
  c->stats.rebuilds = c->init_rebuilds + cnt[0];
  c->stats.mpm_updates = cnt[1];
  c->stats.kernel_launches = g_launches - c->launches0 - c->capture_launches + c->graph_steps * c->gk_base +
                             cnt[2] * c->gk_reb + cnt[3] * c->gk_mpm;
  *out = c->stats;
  return rc;
}

int mpm_get_eps_history(mpm_ctx* c, double* eps, int* rebuilt, int cap, int* n_out) {
  if (!c || !n_out) return MPM_ERR_ARG;
  if (cap < 0 || (cap > 0 && !eps)) return fail(c, MPM_ERR_ARG, "need cap >= 0 and an eps array");
  int rc = sync_status(c);
  long long n = 0;
  CK(cudaMemcpy(&n, c->d.hist_n, sizeof(n), cudaMemcpyDeviceToHost));
  const int R = c->g.R;
  const long long k = std::min<long long>(std::min<long long>(n, cap), kEpsHist);
  std::vector<double> eh((size_t)R * kEpsHist);
  std::vector<int> rh((size_t)R * kEpsHist);
  CK(cudaMemcpy(eh.data(), c->d.eps_hist, eh.size() * sizeof(double), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(rh.data(), c->d.reb_hist, rh.size() * sizeof(int), cudaMemcpyDeviceToHost));
  for (int r = 0; r < R; ++r)
    for (long long q = 0; q < k; ++q) {
      const long long step = n - k + q;  // chronological: the oldest of the k kept decisions first
      const size_t src = (size_t)r * kEpsHist + (size_t)(step % kEpsHist);
      eps[(size_t)r * cap + q] = eh[src];
      if (rebuilt) rebuilt[(size_t)r * cap + q] = rh[src];
    }
  *n_out = (int)k;
  return rc;
}

}  // extern "C"

namespace {

bool valid_tuning(const Tuning& t) {
  auto nt = [](int v) { return v == 64 || v == 128 || v == 256; };
  return nt(t.local_threads) && nt(t.ds_threads) && (t.local_stage == 0 || t.local_stage == 1) &&
         (t.ds_stage == 0 || t.ds_stage == 1) && (t.transport_rows == 4 || t.transport_rows == 8 || t.transport_rows == 16) &&
         (t.sweep_terms == 4 || t.sweep_terms == 8 || t.sweep_terms == 16);
}

// Median device time (ms) of `reps` launches of fn on the context's stream, after one untimed launch.
template <typename F>
double time_launches(mpm_ctx* c, F fn, int reps, cudaEvent_t e0, cudaEvent_t e1) {
  fn();
  std::vector<float> t(reps);
  for (int k = 0; k < reps; ++k) {
    cudaEventRecord(e0, c->stream);
    fn();
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&t[k], e0, e1);
  }
  std::sort(t.begin(), t.end());
  return t[reps / 2];
}

}  // namespace

extern "C" {

int mpm_get_tuning(mpm_ctx* c, int* v, int n) {
  if (!c || !v || n < MPM_TUNE_N) return MPM_ERR_ARG;
  const Tuning& t = c->tune;
  const int vals[MPM_TUNE_N] = {t.local_threads, t.local_stage, t.ds_threads, t.ds_stage, t.transport_rows,
                                t.sweep_terms};
  for (int k = 0; k < MPM_TUNE_N; ++k) v[k] = vals[k];
  return MPM_OK;
}

int mpm_set_tuning(mpm_ctx* c, const int* v, int n) {
  if (!c || !v || n < MPM_TUNE_N) return MPM_ERR_ARG;
  Tuning t;
  t.local_threads = v[0];
  t.local_stage = v[1];
  t.ds_threads = v[2];
  t.ds_stage = v[3];
  t.transport_rows = v[4];
  t.sweep_terms = v[5];
  if (!valid_tuning(t)) return fail(c, MPM_ERR_ARG, "invalid tuning values");
  c->tune = t;
  drop_graph(c);
  return MPM_OK;
}

int mpm_autotune(mpm_ctx* c, int reps, double* ms_out) {
  if (!c) return MPM_ERR_ARG;
  if (reps < 1 || reps > 100) return fail(c, MPM_ERR_ARG, "need 1 <= reps <= 100");
  int rc = need_ready(c, true);
  if (rc) return rc;
  ensure_derived(c);
  const Grid& g = c->g;
  DevState& d = c->d;
  const int nsub = (int)c->subs.size();
  cudaEvent_t e0 = take_event(c), e1 = take_event(c);
  const bool saved_prof = c->prof;
  c->prof = false;
  CK(cudaStreamSynchronize(c->stream));
  Tuning best = c->tune;
  double best_ms[4] = {1e300, 1e300, 1e300, 1e300};
  // 1. the fused transport tile: without the decision its outputs (s2, f(s2), kappa^n and the
  //    transmissibilities of s2) depend only on s, f(s) and the fluxes, so repeated launches
  //    write the same values; kappa^n and the transmissibilities of the current s are restored
  //    afterwards
  const double fmax_ = max_fprime(g.M);
  for (int rows : {4, 8, 16}) {
    const double ms = time_launches(c, [&] { launch_upwind_kappa(g, d, 0.5, fmax_, false, 0.0, 0, false, rows, c->stream); },
                                    reps, e0, e1);
    if (ms < best_ms[0]) { best_ms[0] = ms; best.transport_rows = rows; }
  }
  recompute_derived(c);
  // 2. the MPM-2P local solve (every realisation takes the reuse branch while timed; the
  //    branch flags of the last update are put back afterwards: the downscaling reads them)
  std::vector<int> flags(g.R);
  CK(cudaMemcpyAsync(flags.data(), d.rebuild, sizeof(int) * g.R, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  launch_fill_flags(g, d, 0, c->stream);
  // (timed as the epsilon^0 solve, which leaves the first-order pressure dp0 alone)
  for (int nt : {64, 128, 256})
    for (int stage : {0, 1}) {
      const double ms = time_launches(c, [&] {
        per_class(c, [&](const Grid& gk, int n, int ma, int mb) {
          Grid g0k = gk;
          g0k.order = 0;
          launch_mpm_local(g0k, d, c->d_subs, n, ma, mb, robin_fp32_mode(c->fac_prec), c->ir_tol, c->ir_max,
                           c->d_nodes, c->d_leaf_node, nt, stage, 0, c->stream);
        });
      }, reps, e0, e1);
      if (ms < best_ms[1]) { best_ms[1] = ms; best.local_threads = nt; best.local_stage = stage; }
    }
  CK(cudaMemcpyAsync(d.rebuild, flags.data(), sizeof(int) * g.R, cudaMemcpyHostToDevice, c->stream));
  // 3. the downscaling solve with the factor of the current kappa^n (its inputs, the traces and
  //    targets of the last interface solve, are left unchanged; its outputs are recomputed)
  per_class(c, [&](const Grid& gk, int n, int ma, int mb) {
    launch_downscale_factor(gk, d, c->d_subs, n, ma, mb, fp32(c), ds_reuse_tol(c), c->stream);
  });
  for (int nt : {64, 128, 256})
    for (int stage : {0, 1}) {
      const double ms = time_launches(c, [&] {
        per_class(c, [&](const Grid& gk, int n, int ma, int mb) {
          launch_downscale(gk, d, c->d_subs, n, ma, mb, fp32(c), c->ir_tol, c->ir_max, false, nt, stage, c->stream);
        });
      }, reps, e0, e1);
      if (ms < best_ms[2]) { best_ms[2] = ms; best.ds_threads = nt; best.ds_stage = stage; }
    }
  // 4. the interface sweeps (up and down, every level; they only read the leaves' right-hand
  //    sides and rewrite the internal nodes' vectors, so repeating them changes nothing)
  if (c->n_dof > 0)
    for (int terms : {4, 8, 16}) {
      const double ms = time_launches(c, [&] {
        for (size_t L = 2; L < c->levels.size(); ++L)
          launch_nd_up(g, d, c->d_nodes, c->d_level_nodes + c->lev_off[L], (int)c->levels[L].size(),
                       c->lev_max_nf[L], c->lev_max_nsep[L], c->d_srcmap, false, terms, c->stream);
        for (int L = (int)c->levels.size() - 2; L >= 2; --L)
          launch_nd_down(g, d, c->d_nodes, c->d_level_nodes + c->lev_off[L], (int)c->levels[L].size(),
                         c->lev_max_nsep[L], c->lev_max_nbnd[L], c->d_pmap, false, terms, c->stream);
      }, reps, e0, e1);
      if (ms < best_ms[3]) { best_ms[3] = ms; best.sweep_terms = terms; }
    }
  c->ev_pool.push_back(e0);
  c->ev_pool.push_back(e1);
  c->prof = saved_prof;
  rc = check_launch(c);
  if (rc) return rc;
  rc = sync_status(c);
  c->tune = best;
  drop_graph(c);
  if (ms_out)
    for (int k = 0; k < 4; ++k) ms_out[k] = best_ms[k] < 1e300 ? best_ms[k] : 0.0;
  return rc;
}

int mpm_sync(mpm_ctx* c) {
  if (!c) return MPM_ERR_ARG;
  return sync_status(c);
}

int mpm_profile_enable(mpm_ctx* c, int enable) {
  if (!c) return MPM_ERR_ARG;
  c->prof = enable != 0;
  return MPM_OK;
}

int mpm_profile_read(mpm_ctx* c, double* ms, long long* count) {
  if (!c) return MPM_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < MPM_NSTAGES; ++k) {
    double tot = 0.0;
    for (auto& pr : c->ev_rec[k]) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, pr.first, pr.second));
      tot += t;
      c->ev_pool.push_back(pr.first);
      c->ev_pool.push_back(pr.second);
    }
    if (ms) ms[k] = tot;
    if (count) count[k] = (long long)c->ev_rec[k].size();
    c->ev_rec[k].clear();
  }
  return MPM_OK;
}

}  // extern "C"
