/*
 * mpm2p.h -- C ABI of the GB300 (sm_103a) MRCM / MPM-2P pressure-update hot path.
 *
 * Method: Rocha, Mankad, Sousa, Pereira, "The Multiscale Perturbation Method for
 * Two-Phase Reservoir Flow Problems", arXiv 2103.11050.
 *
 * Problem (Section 2, Eq. Darcy and Eq. BL2D): on the rectangle [0, nx h] x [0, ny h]
 * with square cells of side h, u = -lambda(s) K grad p, div u = q, with per-side
 * Dirichlet (p = g) or Neumann (u.n = z) data, coupled with ds/dt + div(f(s) u) = 0.
 * lambda(s) = M s^2 + (1 - s)^2 and f(s) = M s^2 / lambda(s) (Section 5, k_rw = s^2,
 * k_ro = (1 - s)^2, M = mu_o / mu_w).  kappa = lambda(s) K (Section 2).
 *
 * The fine grid is cell centred with P0 edge fluxes (Section 3): two-point fluxes with
 * harmonic transmissibilities 2 ka kb / (ka + kb); half-cell transmissibility 2 kc on
 * Dirichlet faces.  The domain is split into a tensor product of rectangular subdomains
 * (Section 3); the interface spaces are discontinuous polynomials of degree 0 or 1 on
 * segments of seg_len fine edges (Section 3.1).
 *
 * Conventions shared by all calls
 *  - Every call returns an int status (MPM_OK on success) and never aborts the process.
 *    After an error, mpm_last_error(ctx) returns a one-line message.  A CUDA error
 *    (MPM_ERR_CUDA) leaves the context unusable; destroy it.
 *  - Arrays are float64, C order.  Cell arrays are [R][ny][nx] (R independent
 *    realisations, row j = y index).  Face fluxes are INTEGRATED over the face (h times
 *    the normal velocity): ux is [R][ny][nx+1] (x-face left of cell (i,j), +x positive),
 *    uy is [R][ny+1][nx] (+y positive).
 *  - mem = MPM_MEM_HOST: the pointer is host memory (pageable or pinned); the call copies
 *    synchronously.  Pinned (page-locked, CUDA-registered) host memory is read or written
 *    directly by a kernel, through the device address CUDA reports for it, instead of a
 *    copy-engine transfer; pageable memory takes cudaMemcpyAsync.  Either way the buffer
 *    is free again when the call returns.  mem = MPM_MEM_DEVICE: the pointer is device
 *    memory of the context's device (for instance a torch CUDA tensor's data_ptr()); the
 *    copy is enqueued on the context's stream.
 *  - The caller owns every pointer it passes; setters copy into library-owned device
 *    memory, getters copy out.  Changing the precision, fluids, boundary data or
 *    decomposition discards the stored basis (call mpm_init or mpm_build_basis again).
 *    The library allocates its device memory at mpm_set_decomposition (and frees it in
 *    mpm_destroy); compute calls allocate nothing.
 *  - All work is enqueued on the stream given to mpm_create; compute calls do not
 *    synchronise the host unless stated (mpm_get_*, mpm_get_stats and calls that return
 *    values through host pointers synchronise the stream).
 */
#ifndef MPM2P_H
#define MPM2P_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MPM_OK = 0,
  MPM_ERR_ARG = 1,            /* invalid argument or inconsistent sizes */
  MPM_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  MPM_ERR_OOM = 3,            /* device allocation failed */
  MPM_ERR_NOT_CONVERGED = 4,  /* iterative refinement hit its iteration cap */
  MPM_ERR_STATE = 5,          /* call out of order (e.g. solve before build) */
  MPM_ERR_TOO_LARGE = 6       /* request exceeds a fixed capacity (mpm_cfl_dt_noalloc) */
};

enum { MPM_MEM_HOST = 0, MPM_MEM_DEVICE = 1 };
enum { MPM_BC_DIRICHLET = 0, MPM_BC_NEUMANN = 1 };
enum { MPM_SIDE_LEFT = 0, MPM_SIDE_RIGHT = 1, MPM_SIDE_BOTTOM = 2, MPM_SIDE_TOP = 3 };

/* Precision of the local factorisations and solves.
 *  FP64:          everything in float64.
 *  FP32_IR:       the per-step Neumann downscaling (a new factorisation every step) in
 *                 float32 with float64 refinement to ir_tol; the Robin factors, built once
 *                 per basis rebuild and reused by every BF solve and every MPM-2P step, in
 *                 float64 (on GB300 a float64 solve with a stored factor costs less than
 *                 float32 solves plus float64 refinement residuals).
 *  FP32_IR_ALL:   every local factorisation and solve in float32 with float64 refinement.
 *  TF32_IR, TF32X3_IR, BF16_IR: as FP32_IR_ALL, with the multi-right-hand-side basis-function
 *                 solves of a rebuild (all ndof + 1 right-hand sides of a subdomain) on the
 *                 tensor cores (mma.sync, float32 accumulation) and refined in float64:
 *                 TF32_IR rounds both operands to tf32; TF32X3_IR splits each operand into two
 *                 tf32 parts and sums three products (about float32 accuracy); BF16_IR rounds
 *                 both operands to bf16.  With too little precision for the local conditioning
 *                 the refinement stalls and the next synchronising call returns
 *                 MPM_ERR_NOT_CONVERGED.  Subdomains whose tensor-core tables do not fit in
 *                 shared memory (sides of 20 x 24 cells and larger) take the float32
 *                 CUDA-core basis solve of FP32_IR_ALL instead.
 * The interface (skeleton) system, residuals, fluxes and transport are float64 in all modes. */
enum {
  MPM_PREC_FP64 = 0,
  MPM_PREC_FP32_IR = 1,
  MPM_PREC_FP32_IR_ALL = 2,
  MPM_PREC_TF32_IR = 3,
  MPM_PREC_TF32X3_IR = 4,
  MPM_PREC_BF16_IR = 5
};

/* Which pressure mpm_get_pressure returns. */
enum {
  MPM_P_MRCM = 0,        /* MRCM-level pressure p^m of the last basis build (Section 3) */
  MPM_P_DOWNSCALED = 1   /* pressure of the last downscaling, Eq. (mpm_upd) */
};

typedef struct mpm_ctx mpm_ctx;

typedef struct mpm_stats {
  long long steps;            /* Algorithm 1 iterations run by mpm_step */
  long long rebuilds;         /* basis builds (all realisations summed) */
  long long mpm_updates;      /* MPM-2P reuse updates (all realisations summed) */
  double last_eps_max;        /* max over realisations of the last epsilon */
  double last_dt_min;         /* min over realisations of the last transport dt */
  int ir_iters_max;           /* max refinement sweeps used by any local solve */
  int interface_dofs;         /* interface unknowns per realisation */
  int subdomains;             /* subdomains per realisation */
  int n_hat;                  /* homogeneous BFs per realisation (Section 4.3) */
  long long kernel_launches;  /* CUDA kernels launched by this context so far */
  long long ds_factorisations; /* downscaling factorisations computed (subdomains, all
                                  realisations summed); see mpm_set_downscale_reuse */
} mpm_stats;

/* Stages timed by the profiler (each is the set of kernels of one step of the path). */
enum {
  MPM_STAGE_TRANSPORT = 0,     /* upwind substeps (CFL step), kappa^n, epsilon and
                                  the decision (all in the transport kernel)         */
  MPM_STAGE_DS_FACTOR = 1,     /* downscaling factorisation of kappa^n (Eq. mpm_upd);
                                  a step overlaps it with the perturbation and
                                  interface solves on a second stream, the profiler
                                  runs it alone on the context's stream              */
  MPM_STAGE_BASIS = 2,         /* Robin factorisation, BF solves, element matrices   */
  MPM_STAGE_IFACE_FACTOR = 3,  /* nested-dissection factorisation of the interface   */
  MPM_STAGE_PERTURB = 4,       /* MPM-2P residual, local solve, interface RHS        */
  MPM_STAGE_IFACE_SOLVE = 5,   /* interface sweeps and traces                        */
  MPM_STAGE_DOWNSCALE = 6,     /* u_bar, Neumann downscaling, CFL maxima (one kernel) */
  MPM_STAGE_IFACE_UP = 7,      /* parts of MPM_STAGE_IFACE_SOLVE: upward sweep ...    */
  MPM_STAGE_IFACE_DOWN = 8,    /* ... downward sweep ...                              */
  MPM_STAGE_RECONSTRUCT = 9,   /* ... traces and targets (with the level-1 step)      */
  MPM_NSTAGES = 10
};

/* Create a context for R realisations of an nx x ny grid on [0,Lx]x[0,Ly].
 * Cells must be square: Lx/nx == Ly/ny (relative 1e-12).  stream is a cudaStream_t
 * (NULL = legacy default stream) of the current device, which becomes the context's
 * device.  Defaults: M = 1, left p = 1, right p = 0, top/bottom no flow, s_inflow = 1,
 * q = 0, FP64.  Errors: MPM_ERR_ARG for non-positive sizes, R > 65535 or non-square
 * cells. */
int mpm_create(mpm_ctx** ctx, int R, int nx, int ny, double Lx, double Ly, void* stream);

/* Free all device memory of ctx (after synchronising its stream). NULL is a no-op. */
int mpm_destroy(mpm_ctx* ctx);

/* Message of the last failed call on ctx ("" if none). Owned by ctx. */
const char* mpm_last_error(const mpm_ctx* ctx);

/* Local solver precision (enum above).  ir_tol: target of the refinement, as a backward
 * error in flux units (max |residual| / max(|rhs| + sum |face fluxes|) over the subdomain,
 * the face fluxes of the first iterate;
 * default 1e-14; ignored for FP64), ir_max: sweep cap (>= 1).  Refinement stops at ir_tol
 * (1e-3 ir_tol for the basis-function solves, whose traces are combined with the interface
 * coefficients), or when a sweep no longer halves the error (the FP64 rounding floor of the
 * residual) if the error is then <= 1e3 ir_tol.  A local solve that reaches neither within
 * ir_max sweeps makes the next mpm_sync / getter return MPM_ERR_NOT_CONVERGED.  Takes
 * effect at the next basis build. */
int mpm_set_precision(mpm_ctx* ctx, int mode, double ir_tol, int ir_max);

/* Reuse of float32 downscaling factors (Eq. mpm_upd, left-hand side; the refined precision
 * modes only).  The pinned Neumann operator of kappa^n changes every step, but little in most
 * subdomains (the premise of MPM-2P, Section 4).  A subdomain whose stored float32 factor was
 * computed from transmissibilities within a relative tol of the current ones on every face
 * (and with the pinned cell's kappa within tol) keeps it: its float64 refinement runs against
 * the current operator, so the solution is that of the current operator to the same ir_tol,
 * and the refinement's contraction per sweep grows by at most about tol.  tol <= 0.5; 0
 * refactors every subdomain every step; negative (the default) means 0.005 on decompositions
 * with at least 4 subdomains per SM (realisations included), where the factorisation competes
 * with the rest of the step for the SMs, else 0.  mpm_stats.ds_factorisations counts the
 * factorisations computed.  MPM_ERR_ARG above 0.5 or NaN.  Drops a captured graph. */
int mpm_set_downscale_reuse(mpm_ctx* ctx, double tol);

/* Absolute permeability K [R][ny][nx], every entry > 0 and finite (checked for host
 * input; device input is trusted). */
int mpm_set_permeability(mpm_ctx* ctx, const double* K, int mem);

/* Source q [R][ny][nx] per unit area (Eq. Darcy); NULL resets it to zero. */
int mpm_set_source(mpm_ctx* ctx, const double* q, int mem);

/* Viscosity ratio M = mu_o / mu_w > 0 (Section 5). */
int mpm_set_fluids(mpm_ctx* ctx, double M);

/* Boundary data per side (MPM_SIDE_*): type[k] is MPM_BC_DIRICHLET (val = pressure g)
 * or MPM_BC_NEUMANN (val = outward normal velocity z; z < 0 injects).  At least one side
 * must be Dirichlet (otherwise the pressure is defined up to a constant).  s_inflow is
 * the saturation carried by inflow through any boundary face (Eq. BL2D). */
int mpm_set_boundary(mpm_ctx* ctx, const int type[4], const double val[4], double s_inflow);

/* Tensor-product decomposition (Section 3): ncx column widths col_w (cells, summing to
 * nx) and ncy row heights row_h (summing to ny); every width and height <= 24 and a
 * multiple of seg_len; degree 0 or 1 (Section 3.1), degree 1 with seg_len >= 2 (its linear
 * basis function, sampled at the midpoint of a single edge, would vanish and leave the
 * interface system singular); MPM_ERR_ARG otherwise.  alpha > 0 is the constant of
 * Eq. (beta) (beta = alpha H / kappa, H = length of the interface carrying the face).
 * alpha_face (host memory, may be NULL) gives alpha per fine face instead, the aMRCM's
 * alpha(x) of Section 3.1: ny (nx + 1) values for the x-faces in the layout of ux, then
 * (ny + 1) nx values for the y-faces in the layout of uy (one field for all realisations);
 * only its values on interface faces are read, and each of those must be > 0 and finite
 * (else MPM_ERR_ARG).  NULL means alpha on every face.  The array is copied.
 * (Re)allocates every per-subdomain device buffer; invalidates the stored basis. */
int mpm_set_decomposition(mpm_ctx* ctx, int ncx, const int* col_w, int ncy, const int* row_h,
                          int seg_len, int degree, double alpha, const double* alpha_face);

/* Water saturation s [R][ny][nx] in [0,1]; also recomputes kappa^n = lambda(s) K.  Host
 * values are range-checked (on the device for pinned memory, on the host otherwise) before
 * they replace the current saturation: MPM_ERR_ARG, naming the first index outside [0,1],
 * leaves the context unchanged. */
int mpm_set_saturation(mpm_ctx* ctx, const double* s, int mem);

/* MRCM basis build at the current kappa^n (Algorithm 1, initialisation and rebuild branch; Eqs. mrc1,
 * mrc_homogeneous, mrc_non_homogeneous, mrc2): factor every local Robin problem, one
 * local solve per interface DOF plus the non-homogeneous one, assemble and factor the
 * interface system and form its right-hand side (mpm_interface_solve solves it).  Stores
 * kappa^m := kappa^n.  Enqueued, no host sync.  Needs mpm_set_permeability,
 * mpm_set_decomposition and mpm_set_saturation first. */
int mpm_build_basis(mpm_ctx* ctx);

/* Recompute kappa^n = lambda(s) K from the current saturation and
 * epsilon_r = ||kappa^n - kappa^m||_2 / ||kappa^m||_2 per realisation (Section 4.1,
 * Algorithm 1, update of epsilon).  eps (host, [R]) may be NULL (then no host sync). */
int mpm_eval_epsilon(mpm_ctx* ctx, double* eps);

/* Algorithm 1 decision per realisation: rebuild_r = (epsilon_r > eta) with the
 * epsilon of the last mpm_eval_epsilon.  rebuild (host, [R]) may be NULL (no host sync). */
int mpm_choose(mpm_ctx* ctx, double eta, int* rebuild);

/* MPM-2P perturbation solve (Section 4.1, Eq. mpm_tf_3): fine residual
 * r = q h^2 - sum_faces F(kappa^n, p^m), then one local solve per subdomain with the
 * stored Robin factor of kappa^m (zero Robin data, homogeneous physical data), and the
 * interface right-hand side from its traces.  Needs a stored basis. */
int mpm_perturbation_solve(mpm_ctx* ctx);

/* Order of the MPM-2P perturbation expansion (Section 4.1): 0 (default, as in the paper) keeps
 * the epsilon^0 problem only (Eq. mpm_tf_3); 1 adds the first-order term (Eq. mpm_tf_4 with
 * l = 1): a second local solve per subdomain with the stored Robin factors, source
 * div(kappa_eps grad delta p_0) = -(A(kappa^n) - A(kappa^m)) delta p_0 on the fine grid
 * (delta p_0 the MRCM-level pressure of the epsilon^0 solve, homogeneous data), a second
 * interface solve, and the flux increment u_hat_1 + (kappa^n - kappa^m) grad delta p_0 in
 * u_bar.  mpm_step applies it to every MPM-2P update; it roughly doubles the cost of the
 * perturbation and interface stages.  Drops a captured graph. */
int mpm_set_mpm_order(mpm_ctx* ctx, int order);

/* The first-order local solves (order 1 only; MPM_ERR_STATE otherwise), for the stand-alone
 * sequence mpm_perturbation_solve, mpm_interface_solve, mpm_perturbation_correction,
 * mpm_interface_solve, mpm_downscale.  The interface solve after it solves the first-order
 * interface problem; the one after mpm_perturbation_solve also forms delta p_0. */
int mpm_perturbation_correction(mpm_ctx* ctx);

/* Interface (skeleton) solve with the stored factorisation for the right-hand side of the
 * last mpm_build_basis, mpm_perturbation_solve or mpm_perturbation_correction, then the one-sided traces of every
 * subdomain (and, after a build, the MRCM-level pressure p^m).  The interface fluxes
 * u_bar are formed from these traces by mpm_downscale. */
int mpm_interface_solve(mpm_ctx* ctx);

/* Downscaling (Eq. mpm_upd).  First the interface / boundary fluxes u_bar from the traces
 * of the last mpm_interface_solve: after a build, the mean of the one-sided MRCM traces;
 * after a perturbation solve, the mean of the one-sided traces of the epsilon^0 problem
 * plus the fine flux of p^m with kappa^n (Section 4.1, u_bar = u^m + delta u^n).  Then per
 * subdomain the Neumann problem with kappa^n and u_bar on all its boundary faces; pressure
 * constant fixed by mean(p~) = mean of the MRCM-level pressure of the same update over the
 * subdomain.  Writes the conservative fine fluxes ux, uy (boundary and interior faces),
 * p~, and the per-subdomain maxima of cell in/outflow that the next mpm_saturation_step
 * turns into its time step. */
int mpm_downscale(mpm_ctx* ctx);

/* Explicit upwind transport (Section 4, Eq. BL2D): n_sub >= 1 explicit Euler steps with
 * the fine fluxes of the last mpm_downscale frozen and
 * dt = cfl h^2 / (max f' * max_c max(out_c, in_c)), out_c / in_c the total integrated
 * outflow / inflow of cell c (taken by mpm_downscale; dt = 0 before any downscaling),
 * 0 < cfl <= 1.  Then recomputes kappa^n.  dt (host, [R]) may be NULL (no host sync). */
int mpm_saturation_step(mpm_ctx* ctx, double cfl, int n_sub, double* dt);

/* Algorithm 1 initialisation: kappa^0, MRCM solve + downscale, store the
 * basis, epsilon := eta.  Enqueued, no host sync. */
int mpm_init(mpm_ctx* ctx, double eta);

/* One pass of the while loop of Algorithm 1 for every realisation:
 * n_sub transport steps, kappa^n, MRCM rebuild where epsilon > eta (the epsilon of the
 * previous pass) else an MPM-2P update, downscaling, new epsilon.  By default the pass is
 * one CUDA graph launch: the decision is taken on the device and selects conditional graph
 * bodies (rebuild / reuse), with no host synchronisation.  The graph is captured at the
 * first call and again whenever eta, cfl, n_sub, the fluids, the boundary data, the
 * precision or the decomposition change. */
int mpm_step(mpm_ctx* ctx, double eta, double cfl, int n_sub);

/* Execution of the path (bitmask, default MPM_EXEC_GRAPH | MPM_EXEC_PDL):
 *  MPM_EXEC_GRAPH       mpm_step is one captured CUDA graph launch with device-side
 *                       branching; without it mpm_step runs kernel by kernel and the host
 *                       reads the decision to skip the branch no realisation takes (the
 *                       stage profiler requires this).
 *  MPM_EXEC_PDL         inside mpm_step and mpm_init, the kernels after the first one of the
 *                       interface solve (every nested-dissection level, reconstruction, the
 *                       downscaling) use programmatic dependent launch: each may start while
 *                       its predecessor runs and loads its operators (factor rows, index maps)
 *                       or, for the downscaling, factors its Neumann problems before waiting
 *                       for the predecessor's results.
 * Results are identical up to rounding order.  Any other bit is MPM_ERR_ARG.  Drops a
 * captured graph. */
enum { MPM_EXEC_GRAPH = 1, MPM_EXEC_PDL = 4 };
int mpm_set_execution(mpm_ctx* ctx, int flags);

/* Launch shapes that depend on the geometry (the count and size of the subdomains against the
 * GPU's SM count).  The values, in order (MPM_TUNE_N ints):
 *   [0] threads per CTA of the MPM-2P local solve (64, 128 or 256)
 *   [1] 1: that kernel stages the stored Robin factor in shared memory, 0: reads it from global
 *       memory (smaller CTAs, more subdomains resident per SM)
 *   [2], [3] the same for the downscaling solve
 *   [4] rows (4, 8 or 16) of the 32-column cell tile of the fused transport kernel (two rows
 *       per thread)
 *   [5] interface sweeps: terms of a row's sum per thread (4, 8 or 16)
 * Defaults: 256, 1, 256, 1, 8, 16.  mpm_get_tuning / mpm_set_tuning read and write them (n >=
 * MPM_TUNE_N; invalid values: MPM_ERR_ARG); results do not depend on them beyond rounding.
 * mpm_autotune times every candidate of each kernel on the context's current data (reps
 * timed launches each, the median taken; 1 <= reps <= 100) and keeps the fastest.  It needs a
 * stored basis (after mpm_init); it leaves the state of the current step as it was (it
 * recomputes the downscaled fluxes and pressure of the last update from the same traces, equal
 * up to refinement rounding), synchronises, and writes the best times (ms: transport, MPM-2P
 * local solve, downscaling solve, interface sweeps; 0 when not timed) to ms (host, 4 values)
 * unless NULL.  Setting or tuning
 * drops a captured graph. */
enum { MPM_TUNE_N = 6 };
int mpm_get_tuning(mpm_ctx* ctx, int* values, int n);
int mpm_set_tuning(mpm_ctx* ctx, const int* values, int n);
int mpm_autotune(mpm_ctx* ctx, int reps, double* ms);

/* Copy out pressure [R][ny][nx] (which = MPM_P_*), fluxes ux [R][ny][nx+1],
 * uy [R][ny+1][nx], saturation [R][ny][nx] or conductivity kappa^n.  Synchronise. */
int mpm_get_pressure(mpm_ctx* ctx, double* p, int which, int mem);
int mpm_get_flux(mpm_ctx* ctx, double* ux, double* uy, int mem);
int mpm_get_saturation(mpm_ctx* ctx, double* s, int mem);
int mpm_get_conductivity(mpm_ctx* ctx, double* kappa, int mem);

/* Counters (synchronises the stream and reports a pending MPM_ERR_NOT_CONVERGED). */
int mpm_get_stats(mpm_ctx* ctx, mpm_stats* out);

/* History of the dimensionless MPM-2P parameter (Section 4.1, Algorithm 1): for each of the
 * last steps of mpm_step, the epsilon computed at its end (0 after a rebuild) and its
 * decision (1 = basis rebuilt, 0 = MPM-2P update).  The device keeps the last
 * MPM_EPS_HISTORY steps per realisation.  eps ([R][cap], host) and rebuilt ([R][cap], host,
 * may be NULL) receive per realisation the k = min(steps so far, cap, MPM_EPS_HISTORY) most
 * recent entries in chronological order (row stride cap); *n_out = k.  Synchronises. */
enum { MPM_EPS_HISTORY = 4096 };
int mpm_get_eps_history(mpm_ctx* ctx, double* eps, int* rebuilt, int cap, int* n_out);

/* Synchronise the context's stream; returns a pending device-side status. */
int mpm_sync(mpm_ctx* ctx);

/* Stage profiler: enable != 0 records a CUDA event pair on the context's stream around
 * every stage launch (small overhead); 0 disables it.  mpm_profile_read synchronises,
 * writes per stage the summed device time in ms (ms[MPM_NSTAGES]) and the number of
 * recorded stage executions (count[MPM_NSTAGES]) since enabling or the last read, and
 * resets them.  Either output may be NULL. */
int mpm_profile_enable(mpm_ctx* ctx, int enable);
int mpm_profile_read(mpm_ctx* ctx, double* ms, long long* count);

/* Allocation-free transport time step (the paper has no counterpart: this is a service
 * for callers that cannot allocate device memory).  Some callers cannot call cudaMalloc:
 * code whose device memory belongs to another runtime's pre-sized pool, or a
 * latency-critical loop that cannot afford an allocation's implicit device
 * synchronisation or its failure mid-run.  For them this computes, without any context
 * and without allocating, the same dt per realisation as mpm_saturation_step:
 *   dt_r = cfl h^2 / (max f' * max_c max(out_c, in_c))  (0 when there is no flow),
 * out_c / in_c the total integrated outflow / inflow of cell c, f' for viscosity ratio M.
 * ux [R][ny][nx+1], uy [R][ny+1][nx] (integrated face fluxes, as mpm_get_flux) and dt [R]
 * are caller-owned DEVICE pointers of the current device; the work is enqueued on stream
 * (a cudaStream_t, NULL = legacy default stream) and the call does not synchronise.
 * Scratch: a fixed 512 KiB device array inside the library (64 partial maxima per
 * realisation), held by every GPU that loads the library until the process exits; hence
 * R <= 1024, and larger R returns MPM_ERR_TOO_LARGE without launching anything.  The
 * first call on a device looks up that array's device address (cudaGetSymbolAddress), so
 * make the first call on each device before any stream capture, from one host thread.
 * Every call overwrites the scratch slots it reads, so nothing has to be cleared, but all
 * calls share the array: calls that may overlap on the GPU (different streams without
 * ordering) race and must be serialised by the caller.  Returns MPM_ERR_ARG for null
 * pointers, non-positive sizes, h, M or cfl outside (0,1]; MPM_ERR_CUDA if a CUDA call fails. */
int mpm_cfl_dt_noalloc(const double* ux, const double* uy, int R, int nx, int ny, double h, double M,
                       double cfl, double* dt, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MPM2P_H */
