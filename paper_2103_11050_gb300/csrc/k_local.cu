// Local problems on the subdomains: Robin problems of the MRCM (Eq. mrc1 with the
// split Eqs. mrc_homogeneous / mrc_non_homogeneous), the MPM-2P epsilon^0 local solve
// (Eq. mpm_tf_3 with zero Robin data) and the Neumann downscaling (Eq. mpm_upd).
//
// Discretisation (two-point fluxes on the a x b cells of a subdomain, row-major local
// index c = jl * a + il):
//   interior face (harmonic):     T = 2 ka kb / (ka + kb)
//   Robin interface face:         r_e = kappa_c / (1/2 + rho), rho = alpha H / h
//   Dirichlet physical face:      2 kappa_c          Neumann face: 0
// The matrix is block tridiagonal over grid rows: A = tridiag(-diag(t_{j-1}), D_j,
// -diag(t_j)), D_j tridiagonal.  The block LDL^T with explicit inverse pivots
//   S_0 = D_0,  S_j = D_j - diag(t_{j-1}) Q_{j-1} diag(t_{j-1}),  Q_j = S_j^{-1}
// only needs elementwise updates between pivots (the coupling blocks are diagonal),
// and each Q_j comes from an in-place Gauss-Jordan inversion held one entry per thread.
// Solves are 2b dependent dense a x a block products (GEMV / small GEMM per block row):
//   forward  W_j = Q_j (f_j + t_{j-1} o W_{j-1})
//   backward X_j = W_j + Q_j (t_j o X_{j+1})
// In FP32 mode the factor is built from the Jacobi-scaled matrix S A S,
// S = diag(A)^{-1/2}, and FP64 iterative refinement against the FP64 stencil recovers
// FP64 accuracy.  Factorisations and single-RHS solves run two warps per subdomain,
// factoring from both ends (twisted, k_local_warp.cuh); the multi-RHS basis solve runs one
// CTA per subdomain with the same twisted sweeps.  Factors are stored padded as
// [b][A][A] (A = pad_width(max a)).
#include "mpm2p_internal.cuh"
#include "k_iface_phases.cuh"
#include "k_local_tc.cuh"
#include "k_local_warp.cuh"

#include <algorithm>
#include <type_traits>

namespace mpm {

namespace {

constexpr int kSmemBudget = 200 * 1024;

// Asynchronous 16-byte global -> shared copies (cp.async), completed by cp_async_wait_all().
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}
// Stage `bytes` (a multiple of 16, both addresses 16-byte aligned) into shared memory.
__device__ __forceinline__ void stage_async(void* smem_dst, const void* gsrc, size_t bytes) {
  char* dst = reinterpret_cast<char*>(smem_dst);
  const char* src = reinterpret_cast<const char*>(gsrc);
  for (size_t o = (size_t)threadIdx.x * 16; o < bytes; o += (size_t)blockDim.x * 16) cp_async16(dst + o, src + o);
}

using phase::side_basis;

// Local cell adjacent to face f, and the side / position of the face.
__device__ __forceinline__ void face_info(const DevSub& sd, int f, int& side, int& t, int& cl) {
  if (f < sd.b) { side = 0; t = f; cl = t * sd.a; }
  else if (f < 2 * sd.b) { side = 1; t = f - sd.b; cl = t * sd.a + sd.a - 1; }
  else if (f < 2 * sd.b + sd.a) { side = 2; t = f - 2 * sd.b; cl = t; }
  else { side = 3; t = f - 2 * sd.b - sd.a; cl = (sd.b - 1) * sd.a + t; }
}

// Shared-memory layout of one subdomain problem.
struct Stencil {
  double* kap;   // m
  double* ex;    // m   diagonal part not due to interior faces (Robin, Dirichlet, pin)
  double* wE;    // m   transmissibility to the east neighbour (0 on the last column)
  double* wN;    // m   transmissibility to the north neighbour (0 on the last row)
  double* sc;    // m   Jacobi scaling (1 in FP64 mode)
};

// Multi-RHS twisted block solve  (S A S) X = Z  in place on Z ([m][ncol], column stride
// ncol) with the factor of k_local_warp.cuh (top chain j < mid, bottom chain j > mid,
// middle row mid = b/2).  W: workspace of the same shape.  Q: [b][A][A] factor and
// th[m] = scaled north couplings (factor type), both in shared memory.  The coupling of a
// block row to its neighbour (an elementwise product, the inter-row blocks of a 5-point
// operator being diagonal) is formed once per entry in shared memory before the row's
// products with its a x a block, not once per output row inside them.
template <typename T>
__device__ void block_solve(const DevSub& sd, const T* th, const T* Q, int A, T* Z, T* W, int ncol) {
  const int a = sd.a, b = sd.b, mid = b / 2;
  const int nwork = a * ncol;
  // W_j = Q_j Y_j,  Y_j = Z_j + th_{jp} o W_{jp} (formed in place in Z_j),  jp = previous
  // row of the chain (-1: none)
  auto product = [&](int j, const T* Y) {  // W_j = Q_j Y
    const T* Qj = Q + (long long)j * A * A;
    for (int w = threadIdx.x; w < nwork; w += blockDim.x) {
      const int i = w / ncol, col = w - (w / ncol) * ncol;
      T acc = T(0);
      for (int k = 0; k < a; ++k) acc += Qj[i * A + k] * Y[k * ncol + col];
      W[(j * a + i) * ncol + col] = acc;
    }
    __syncthreads();
  };
  auto fwd = [&](int j, int jp) {
    if (jp >= 0) {
      const T* tj = th + min(j, jp) * a;
      for (int w = threadIdx.x; w < nwork; w += blockDim.x) {
        const int k = w / ncol, col = w - (w / ncol) * ncol;
        Z[(j * a + k) * ncol + col] += tj[k] * W[(jp * a + k) * ncol + col];
      }
      __syncthreads();
    }
    product(j, Z + (long long)j * a * ncol);
  };
  for (int j = 0; j < mid; ++j) fwd(j, j - 1);
  for (int j = b - 1; j > mid; --j) fwd(j, j + 1 < b ? j + 1 : -1);
  // middle: X_mid = Q_mid (Z_mid + th_{mid-1} o W_{mid-1} + th_mid o W_{mid+1})
  if (mid > 0 || mid < b - 1) {
    for (int w = threadIdx.x; w < nwork; w += blockDim.x) {
      const int k = w / ncol, col = w - (w / ncol) * ncol;
      const int ck = mid * a + k;
      T zk = Z[ck * ncol + col];
      if (mid > 0) zk += th[ck - a] * W[(ck - a) * ncol + col];
      if (mid < b - 1) zk += th[ck] * W[(ck + a) * ncol + col];
      Z[ck * ncol + col] = zk;
    }
    __syncthreads();
  }
  product(mid, Z + (long long)mid * a * ncol);  // W_mid holds X_mid
  // backward: X_j = W_j + Q_j (th_{jc} o X_{jn}), jn = the row solved before.  The products
  // th_{jc} o X_{jn} go into W_{jn} (no longer needed once X_{jn} is final), except for
  // jn = mid, whose row serves both chains with different couplings.
  auto bwd = [&](int j, int jn) {
    const T* Qj = Q + (long long)j * A * A;
    const T* tj = th + min(j, jn) * a;
    if (jn != mid) {
      for (int w = threadIdx.x; w < nwork; w += blockDim.x) {
        const int k = w / ncol, col = w - (w / ncol) * ncol;
        W[(jn * a + k) * ncol + col] = tj[k] * Z[(jn * a + k) * ncol + col];
      }
      __syncthreads();
      for (int w = threadIdx.x; w < nwork; w += blockDim.x) {
        const int i = w / ncol, col = w - (w / ncol) * ncol;
        T acc = T(0);
        for (int k = 0; k < a; ++k) acc += Qj[i * A + k] * W[(jn * a + k) * ncol + col];
        Z[(j * a + i) * ncol + col] = W[(j * a + i) * ncol + col] + acc;
      }
    } else {
      for (int w = threadIdx.x; w < nwork; w += blockDim.x) {
        const int i = w / ncol, col = w - (w / ncol) * ncol;
        T acc = T(0);
        for (int k = 0; k < a; ++k) acc += Qj[i * A + k] * (tj[k] * Z[(jn * a + k) * ncol + col]);
        Z[(j * a + i) * ncol + col] = W[(j * a + i) * ncol + col] + acc;
      }
    }
    __syncthreads();
  };
  for (int w = threadIdx.x; w < nwork; w += blockDim.x) {
    const int i = w / ncol, col = w - (w / ncol) * ncol;
    Z[(mid * a + i) * ncol + col] = W[(mid * a + i) * ncol + col];
  }
  __syncthreads();
  for (int j = mid - 1; j >= 0; --j) bwd(j, j + 1);
  for (int j = mid + 1; j < b; ++j) bwd(j, j - 1);
}

// (A x)_c in flux form: sum over interior faces of T (x_c - x_nb) plus ex_c x_c, so that
// b - A x is the mass-balance defect of the cell; absx = sum of the magnitudes of the
// terms (the flux scale of the cell).  x has column stride ncol.
__device__ __forceinline__ double apply_A(const DevSub& sd, const Stencil& S, const double* x, int c,
                                          int col, int ncol, double& absx) {
  const int a = sd.a, b = sd.b;
  const int jl = c / a, il = c - jl * a;
  const double xc = x[c * ncol + col];
  double t = S.ex[c] * xc;
  double v = t;
  absx = fabs(t);
  if (il < a - 1) { t = S.wE[c] * (xc - x[(c + 1) * ncol + col]); v += t; absx += fabs(t); }
  if (il > 0) { t = S.wE[c - 1] * (xc - x[(c - 1) * ncol + col]); v += t; absx += fabs(t); }
  if (jl < b - 1) { t = S.wN[c] * (xc - x[(c + a) * ncol + col]); v += t; absx += fabs(t); }
  if (jl > 0) { t = S.wN[c - a] * (xc - x[(c - a) * ncol + col]); v += t; absx += fabs(t); }
  return v;
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), __double_as_longlong(v));
}

// Solve A X = B for ncol right-hand sides (B, X FP64 [m][ncol]).  FP64 mode: one block
// solve.  FP32 mode: refinement  x += S solve(S r),  r = b - A x (FP64, flux form), with
// the backward error in flux units  eta = max_col max|r| / max(|b| + sum|fluxes|).
// Stops when eta <= target, or when a sweep no longer halves eta (the FP64 rounding floor
// of the residual) provided eta <= 1e3 tol; after ir_max sweeps without either, the status
// bit is set.  colmax holds per column [max|r|, max(|b|+sum|fluxes|)].
template <typename T>
__device__ void solve_refined(const DevSub& sd, Stencil S, const T* th, const T* Q, int A, const double* B,
                              double* X, double* Rr, T* Zw, T* Ww, int ncol, bool refine, double target, double tol,
                              int ir_max, double* colmax /* 2*ncol */, int* status, int* ir_used) {
  const int m = sd.a * sd.b;
  const int n = m * ncol;
  if (std::is_same<T, double>::value && !refine) {
    // float64 factor, unscaled (S.sc = 1): one block solve, without the scaling products (in
    // place when B and X are the workspace Zw itself)
    const bool in_place = reinterpret_cast<const void*>(B) == reinterpret_cast<const void*>(Zw);
    if (!in_place)
      for (int e = threadIdx.x; e < n; e += blockDim.x) Zw[e] = T(B[e]);
    __syncthreads();
    block_solve<T>(sd, th, Q, A, Zw, Ww, ncol);
    if (!in_place)
      for (int e = threadIdx.x; e < n; e += blockDim.x) X[e] = double(Zw[e]);
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(ir_used, 1);
    __syncthreads();
    return;
  }
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    X[e] = 0.0;
    Rr[e] = B[e];
  }
  __syncthreads();
  const int sweeps = refine ? ir_max : 1;
  int it = 0;
  bool ok = false;
  double eta_prev = 1e300;
  for (; it < sweeps; ++it) {
    for (int e = threadIdx.x; e < n; e += blockDim.x) Zw[e] = T(Rr[e] * S.sc[e / ncol]);
    __syncthreads();
    block_solve<T>(sd, th, Q, A, Zw, Ww, ncol);
    for (int e = threadIdx.x; e < n; e += blockDim.x) X[e] += double(Zw[e]) * S.sc[e / ncol];
    __syncthreads();
    if (!refine) { it = 1; ok = true; break; }
    for (int c = threadIdx.x; c < 2 * ncol; c += blockDim.x) colmax[c] = 0.0;
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int c = e / ncol, col = e - c * ncol;
      double absx;
      const double r = B[e] - apply_A(sd, S, X, c, col, ncol, absx);
      Rr[e] = r;
      atomic_max_nonneg(&colmax[col], fabs(r));
      atomic_max_nonneg(&colmax[ncol + col], absx + fabs(B[e]));
    }
    __syncthreads();
    double eta = 0.0;
    for (int col = 0; col < ncol; ++col)
      if (colmax[ncol + col] > 0.0) eta = fmax(eta, colmax[col] / colmax[ncol + col]);
    __syncthreads();
    if (eta <= target) { ok = true; ++it; break; }
    if (eta > 0.5 * eta_prev && eta <= 1e3 * tol) { ok = true; ++it; break; }  // FP64 floor reached
    eta_prev = eta;
  }
  if (threadIdx.x == 0) {
    if (!ok) atomicOr(status, 1);
    atomicMax(ir_used, it);
  }
  __syncthreads();
}

struct SmemPlan {
  int ncol;
  size_t bytes;
};

__host__ __device__ inline size_t stencil_bytes(int m) { return (size_t)5 * m * sizeof(double); }

template <typename T>
size_t fixed_bytes(int a, int b, int A) {
  const int m = a * b;
  return stencil_bytes(m) + (size_t)b * A * A * sizeof(T) + (size_t)m * sizeof(T) + 64 * sizeof(double) + 256;
}

// direct: the float64 solve without refinement, whose right-hand side is built in the block
// solve's workspace and whose solution is read from it (no separate right-hand-side, solution
// and residual blocks: 16 instead of 40 bytes per cell and column).
template <typename T>
SmemPlan plan_smem(int a, int b, int A, int ncol_max, bool q_global = false, bool direct = false) {
  const int m = a * b;
  const size_t fixed = fixed_bytes<T>(a, b, A) - (q_global ? (size_t)b * A * A * sizeof(T) : 0);
  const size_t per_col = direct ? (size_t)m * 2 * sizeof(T) + 2 * sizeof(double)
                                : (size_t)m * (3 * sizeof(double) + 2 * sizeof(T)) + 2 * sizeof(double);
  // signed: the fixed part alone may exceed the budget (a staged 32-wide float64 factor of
  // 24 block rows), which leaves no column and sends the caller to the in-place factor
  const long long room = (long long)kSmemBudget - (long long)fixed;
  int ncol = room > 0 ? (int)(room / (long long)per_col) : 0;
  if (ncol > ncol_max) ncol = ncol_max;
  if (ncol < 1) ncol = 1;
  return {ncol, fixed + per_col * ncol};
}

template <typename T>
struct Carve {
  Stencil S;
  T* Q;
  T* th;
  double* colmax;
  double *B, *X, *Rr;
  T *Zw, *Ww;
};

template <typename T>
__device__ Carve<T> carve(char* base, int a, int b, int A, int ncol, bool q_global = false, bool direct = false) {
  const int m = a * b;
  Carve<T> c;
  double* p = reinterpret_cast<double*>(base);
  c.S.kap = p; p += m;
  c.S.ex = p; p += m;
  c.S.wE = p; p += m;
  c.S.wN = p; p += m;
  c.S.sc = p; p += m;
  c.colmax = p; p += 64;
  if (!direct) {
    c.B = p; p += (size_t)m * ncol;
    c.X = p; p += (size_t)m * ncol;
    c.Rr = p; p += (size_t)m * ncol;
  }
  T* q = reinterpret_cast<T*>(p);
  c.Q = q; q += q_global ? 0 : (size_t)b * A * A;  // the factor stays in global memory when q_global
  c.Zw = q; q += (size_t)m * ncol;
  c.Ww = q; q += (size_t)m * ncol;
  c.th = q;
  if (direct) {  // float64 only (plan_smem): right-hand side and solution live in Zw
    c.B = c.X = reinterpret_cast<double*>(c.Zw);
    c.Rr = nullptr;
  }
  return c;
}


// Load the stored Robin factor (padded) and FP64 stencil of kappa^m into shared memory (CTA).
template <typename T>
__device__ void load_robin(const DevState& d, const DevSub& sd, int r, Carve<T>& cv, const Grid& g, int A,
                           bool q_global = false) {
  const int a = sd.a, b = sd.b, m = a * b;
  const T* Qg = reinterpret_cast<const T*>(d.fac) + (long long)r * d.st_fac + sd.q_off;
  if (q_global) cv.Q = const_cast<T*>(Qg);  // read in place (only read by the solves)
  else
    for (int e = threadIdx.x; e < b * A * A; e += blockDim.x) cv.Q[e] = Qg[e];
  const double* tv = d.tvec + (long long)r * d.st_t + sd.t_off;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    cv.S.ex[c] = tv[c];
    cv.S.wE[c] = tv[m + c];
    cv.S.wN[c] = tv[2 * m + c];
    cv.S.sc[c] = tv[3 * m + c];
    const int jl = c / a, il = c - jl * a;
    cv.S.kap[c] = d.kap_m[(long long)r * g.ncell() + (long long)(sd.y0 + jl) * g.nx + sd.x0 + il];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < m; c += blockDim.x)
    cv.th[c] = c + a < m ? T(cv.S.wN[c] * cv.S.sc[c] * cv.S.sc[c + a]) : T(0);
  __syncthreads();
}

// Right-hand side of the local problem for column `col` of the basis set: col < ndof is the
// homogeneous BF of local DOF col (Robin datum g = -bh s phi on U-DOFs, g = psi on P-DOFs,
// entering as r_e g_e; zero source and physical data), col == ndof the non-homogeneous BF
// (source q h^2 and physical data, zero Robin data).
__device__ double basis_rhs(const Grid& g, const DevState& d, const DevSub& sd, const Stencil& S, int r,
                            int c, int col) {
  const int a = sd.a, b = sd.b;
  const int jl = c / a, il = c - jl * a;
  const double kc = S.kap[c];
  double v = 0.0;
  if (col == sd.ndof) {
    v = d.q[(long long)r * g.ncell() + (long long)(sd.y0 + jl) * g.nx + sd.x0 + il] * g.h * g.h;
    const int sides[4] = {il == 0 ? 0 : -1, il == a - 1 ? 1 : -1, jl == 0 ? 2 : -1, jl == b - 1 ? 3 : -1};
    for (int q = 0; q < 4; ++q) {
      const int sdx = sides[q];
      if (sdx < 0 || sd.side_kind[sdx] == 1) continue;
      if (g.bc_type[sdx] == 0) v += 2.0 * kc * g.bc_val[sdx];
      else v -= g.bc_val[sdx] * g.h;
    }
    return v;
  }
  // find the side of DOF col
  for (int q = 0; q < 4; ++q) {
    if (sd.side_kind[q] != 1) continue;
    const int d0 = sd.side_dof0[q], nb = sd.side_nb[q];
    if (col < d0 || col >= d0 + 2 * nb) continue;
    const bool on_side = (q == 0 && il == 0) || (q == 1 && il == a - 1) || (q == 2 && jl == 0) ||
                         (q == 3 && jl == b - 1);
    if (!on_side) return 0.0;
    const int t = (q < 2) ? jl : il;
    const double rho = d.rho_f[sd.face_off + face_side_off(q, a, b) + t];
    const bool isU = col < d0 + nb;
    const double phi = side_basis(isU ? col - d0 : col - d0 - nb, t, g.seg_len, g.degree, g.inv_seg);
    // r_e g_e with r_e = kc/(1/2+rho): U: g = -(rho/kc) s phi -> -rho s phi/(1/2+rho); P: kc phi/(1/2+rho)
    return isU ? div64(-rho * sd.side_sign[q] * phi, 0.5 + rho) : div64(kc * phi, 0.5 + rho);
  }
  return 0.0;
}

// Robin datum g_e of basis column col on face f (0 for the non-homogeneous column).
__device__ double basis_g(const Grid& g, const DevState& d, const DevSub& sd, const Stencil& S, int f, int col) {
  if (col == sd.ndof) return 0.0;
  int side, t, cl;
  face_info(sd, f, side, t, cl);
  if (sd.side_kind[side] != 1) return 0.0;
  const int d0 = sd.side_dof0[side], nb = sd.side_nb[side];
  if (col < d0 || col >= d0 + 2 * nb) return 0.0;
  const bool isU = col < d0 + nb;
  const double phi = side_basis(isU ? col - d0 : col - d0 - nb, t, g.seg_len, g.degree, g.inv_seg);
  return isU ? -div64(d.rho_f[sd.face_off + f], S.kap[cl]) * sd.side_sign[side] * phi : phi;
}

// Robin coefficient r_e = kappa_c / (1/2 + rho_e) of every interface face of the subdomain
// (unused on physical faces), formed once per CTA for the traces of all its basis columns.
__device__ void robin_coeffs(const DevState& d, const DevSub& sd, const Stencil& S, double* rface) {
  const int nface = 2 * (sd.a + sd.b);
  for (int f = threadIdx.x; f < nface; f += blockDim.x) {
    int side, t, cl;
    face_info(sd, f, side, t, cl);
    rface[f] = sd.side_kind[side] == 1 ? div64(S.kap[cl], 0.5 + d.rho_f[sd.face_off + f]) : 0.0;
  }
}

// Outward trace on face f of the local solution x (column col of X) of basis column bcol;
// rface from robin_coeffs.
__device__ double basis_trace(const Grid& g, const DevState& d, const DevSub& sd, const Stencil& S, const double* X,
                              const double* rface, int ncol, int f, int col, int bcol, bool homogeneous_phys) {
  int side, t, cl;
  face_info(sd, f, side, t, cl);
  const double kc = S.kap[cl], pc = X[cl * ncol + col];
  if (sd.side_kind[side] == 1) return rface[f] * (pc - basis_g(g, d, sd, S, f, bcol));
  if (g.bc_type[side] == 0) return 2.0 * kc * (pc - (homogeneous_phys ? 0.0 : g.bc_val[side]));
  return homogeneous_phys ? 0.0 : g.bc_val[side] * g.h;
}

// All BF solves of a subdomain (rebuild): the ndof homogeneous BFs and the non-homogeneous
// one, in column chunks of ncol_max; chunk k goes to the CTA with blockIdx.z = k mod gridDim.z
// (on grids with few subdomains several CTAs share a subdomain's columns, each with its own
// copy of the factor).  Outputs: traces (tr, fbar), pressures (pf incl. the
// non-homogeneous column), means (mu_hat, sub_mean); the CTA of the non-homogeneous column
// also writes the subdomain's interface right-hand side.
template <typename T>
__global__ void k_basis_solve(Grid g, DevState d, const DevSub* subs, int A, int ncol_max, int refine,
                              double tol, int ir_max, const DevNode* nodes, const int* leaf_node, int q_global) {
  extern __shared__ __align__(16) char smem[];
  const int r = blockIdx.y;
  if (d.rebuild[r] != 1) return;
  __shared__ DevSub sd_s;  // the subdomain record, staged once per CTA (indexed by side)
  const int sidx = sub_index(g);
  if (threadIdx.x == 0) sd_s = subs[sidx];
  __syncthreads();
  const DevSub& sd = sd_s;
  const int a = sd.a, b = sd.b, m = a * b;
  const int nface = 2 * (a + b);
  const int ntot = sd.ndof + 1;
  if ((int)blockIdx.z * ncol_max >= ntot) return;  // no chunk for this CTA
  const bool direct = std::is_same<T, double>::value && refine == 0;  // the layout of plan_smem
  Carve<T> cv = carve<T>(smem, a, b, A, ncol_max, q_global != 0, direct);
  load_robin<T>(d, sd, r, cv, g, A, q_global != 0);
  __shared__ double rface[4 * kMaxSide];
  robin_coeffs(d, sd, cv.S, rface);  // read after the barriers of the first chunk's solve
  double* tr = d.tr + (long long)r * d.st_tr + sd.tr_off;       // [ndof][nface]
  double* pf = d.pf + (long long)r * d.st_pf + sd.pf_off;       // [ndof+1][m]
  double* fbar = d.fbar + (long long)r * d.st_face + sd.face_off;
  double* muh = d.mu_hat + (long long)r * d.st_dof + sd.dof_off;
  for (int c0 = blockIdx.z * ncol_max; c0 < ntot; c0 += gridDim.z * ncol_max) {
    const int ncol = min(ncol_max, ntot - c0);
    for (int e = threadIdx.x; e < m * ncol; e += blockDim.x) {
      const int c = e / ncol, col = e - c * ncol;
      cv.B[e] = basis_rhs(g, d, sd, cv.S, r, c, c0 + col);
    }
    __syncthreads();
    // The BF traces are combined with possibly large interface coefficients, so their local
    // conservation defect (sum of residuals) is driven to the FP64 rounding floor.
    solve_refined<T>(sd, cv.S, cv.th, cv.Q, A, cv.B, cv.X, cv.Rr, cv.Zw, cv.Ww, ncol, refine != 0, 1e-3 * tol, tol,
                     ir_max, cv.colmax, d.status, d.ir_iters);
    for (int e = threadIdx.x; e < m * ncol; e += blockDim.x) {
      const int col = e / m, c = e - col * m;
      pf[(long long)(c0 + col) * m + c] = cv.X[c * ncol + col];
    }
    for (int e = threadIdx.x; e < nface * ncol; e += blockDim.x) {
      const int f = e / ncol, col = e - f * ncol, bcol = c0 + col;
      const double v = basis_trace(g, d, sd, cv.S, cv.X, rface, ncol, f, col, bcol, bcol < sd.ndof);
      if (bcol < sd.ndof) tr[(long long)bcol * nface + f] = v;
      else fbar[f] = v;
    }
    // column means
    for (int col = threadIdx.x >> 5; col < ncol; col += blockDim.x >> 5) {
      double s = 0.0;
      for (int c = threadIdx.x & 31; c < m; c += 32) s += cv.X[c * ncol + col];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if ((threadIdx.x & 31) == 0) {
        const int bcol = c0 + col;
        if (bcol < sd.ndof) muh[bcol] = s / m;
        else d.sub_mean[(long long)r * d.st_sub + sidx] = s / m;
      }
    }
    __syncthreads();
  }
  // Interface right-hand side (Eq. mrc2) from the non-homogeneous traces just written.
  if ((ntot - 1) / ncol_max % (int)gridDim.z == (int)blockIdx.z)
    for (int k = threadIdx.x; k < sd.ndof; k += blockDim.x)
      phase::element_rhs(g, d, sd, nodes[leaf_node[sidx]], r, k, fbar);
}

// ---------------------------------------------------------------------------------------------
// Tensor-core basis-function solves (k_local_tc.cuh): the float32 Robin factor, every block
// product on the tensor cores, float64 refinement with the same residual, scale and stopping
// rule as solve_refined.  Z / W are [m][ld] floats, ncp = ncol rounded up to 8 (the padding
// columns hold zeros).

template <int A, int KIND>
__device__ void solve_refined_tc(const DevSub& sd, Stencil S, const float* th, const float* Q, const double* B,
                                 double* X, double* Rr, float* Zw, float* Ww, int ncol, int ld, double target, double tol,
                                 int ir_max, double* colmax, int* status, int* ir_used) {
  const int m = sd.a * sd.b;
  const int n = m * ncol, ncp = (ncol + 7) / 8 * 8;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    X[e] = 0.0;
    Rr[e] = B[e];
  }
  __syncthreads();
  int it = 0;
  bool ok = false;
  double eta_prev = 1e300;
  for (; it < ir_max; ++it) {
    for (int e = threadIdx.x; e < m * ncp; e += blockDim.x) {
      const int c = e / ncp, col = e - c * ncp;
      Zw[c * ld + col] = col < ncol ? (float)(Rr[c * ncol + col] * S.sc[c]) : 0.0f;
    }
    __syncthreads();
    tc::block_solve_tc<A, KIND>(sd, th, Q, Zw, Ww, ld, ncp);
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int c = e / ncol, col = e - c * ncol;
      X[e] += (double)Zw[c * ld + col] * S.sc[c];
    }
    for (int c = threadIdx.x; c < 2 * ncol; c += blockDim.x) colmax[c] = 0.0;
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int c = e / ncol, col = e - c * ncol;
      double absx;
      const double r = B[e] - apply_A(sd, S, X, c, col, ncol, absx);
      Rr[e] = r;
      atomic_max_nonneg(&colmax[col], fabs(r));
      atomic_max_nonneg(&colmax[ncol + col], absx + fabs(B[e]));
    }
    __syncthreads();
    double eta = 0.0;
    for (int col = 0; col < ncol; ++col)
      if (colmax[ncol + col] > 0.0) eta = fmax(eta, colmax[col] / colmax[ncol + col]);
    __syncthreads();
    if (eta <= target) { ok = true; ++it; break; }
    if (eta > 0.5 * eta_prev && eta <= 1e3 * tol) { ok = true; ++it; break; }  // float64 floor reached
    eta_prev = eta;
  }
  if (threadIdx.x == 0) {
    if (!ok) atomicOr(status, 1);
    atomicMax(ir_used, it);
  }
  __syncthreads();
}

// Shared memory of the tensor-core basis solve: the stencil, colmax, B / X / Rr ([m][ncol]
// doubles), the factor ([b][A][A] floats), th (m floats), Z / W ([m][ld] floats).
struct TcPlan {
  int ncol, ld;
  size_t bytes;
};

inline TcPlan plan_tc(int a, int b, int A) {
  const int m = a * b;
  for (int ncol = 32; ncol >= 8; ncol -= 8) {
    const int ld = tc::tc_ld(ncol);
    const size_t bytes = stencil_bytes(m) + 64 * sizeof(double) + (size_t)3 * m * ncol * sizeof(double) +
                         (size_t)b * A * A * sizeof(float) + (size_t)m * sizeof(float) +
                         (size_t)2 * m * ld * sizeof(float) + 256;
    if (bytes <= (size_t)kSmemBudget || ncol == 8) return {ncol, ld, bytes};
  }
  return {8, tc::tc_ld(8), 0};
}

// All BF solves of a subdomain on the tensor cores (same outputs as k_basis_solve).
template <int A, int KIND>
__global__ void __launch_bounds__(256) k_basis_solve_tc(Grid g, DevState d, const DevSub* subs, int ncol_max, int ld,
                                                        double tol, int ir_max, const DevNode* nodes,
                                                        const int* leaf_node) {
  extern __shared__ __align__(16) char smem[];
  const int r = blockIdx.y;
  if (d.rebuild[r] != 1) return;
  __shared__ DevSub sd_s;
  const int sidx = sub_index(g);
  if (threadIdx.x == 0) sd_s = subs[sidx];
  __syncthreads();
  const DevSub& sd = sd_s;
  const int a = sd.a, b = sd.b, m = a * b;
  const int nface = 2 * (a + b);
  const int ntot = sd.ndof + 1;
  // carve: the float32 part of the layout (Q, Zw, Ww, th) after the float64 part
  Carve<float> cv;
  {
    double* p = reinterpret_cast<double*>(smem);
    cv.S.kap = p; p += m;
    cv.S.ex = p; p += m;
    cv.S.wE = p; p += m;
    cv.S.wN = p; p += m;
    cv.S.sc = p; p += m;
    cv.colmax = p; p += 64;
    cv.B = p; p += (size_t)m * ncol_max;
    cv.X = p; p += (size_t)m * ncol_max;
    cv.Rr = p; p += (size_t)m * ncol_max;
    float* q = reinterpret_cast<float*>(p);
    cv.Q = q; q += (size_t)b * A * A;
    cv.th = q; q += m;
    q += (16 - ((uintptr_t)q & 15) / 4) & 3;  // 16-byte alignment of the right-hand-side blocks
    cv.Zw = q; q += (size_t)m * ld;
    cv.Ww = q;
  }
  load_robin<float>(d, sd, r, cv, g, A);
  __shared__ double rface[4 * kMaxSide];
  robin_coeffs(d, sd, cv.S, rface);  // read after the barriers of the first chunk's solve
  double* tr = d.tr + (long long)r * d.st_tr + sd.tr_off;
  double* pf = d.pf + (long long)r * d.st_pf + sd.pf_off;
  double* fbar = d.fbar + (long long)r * d.st_face + sd.face_off;
  double* muh = d.mu_hat + (long long)r * d.st_dof + sd.dof_off;
  for (int c0 = blockIdx.z * ncol_max; c0 < ntot; c0 += gridDim.z * ncol_max) {
    const int ncol = min(ncol_max, ntot - c0);
    for (int e = threadIdx.x; e < m * ncol; e += blockDim.x) {
      const int c = e / ncol, col = e - c * ncol;
      cv.B[e] = basis_rhs(g, d, sd, cv.S, r, c, c0 + col);
    }
    __syncthreads();
    solve_refined_tc<A, KIND>(sd, cv.S, cv.th, cv.Q, cv.B, cv.X, cv.Rr, cv.Zw, cv.Ww, ncol, ld, 1e-3 * tol, tol, ir_max,
                              cv.colmax, d.status, d.ir_iters);
    for (int e = threadIdx.x; e < m * ncol; e += blockDim.x) {
      const int col = e / m, c = e - col * m;
      pf[(long long)(c0 + col) * m + c] = cv.X[c * ncol + col];
    }
    for (int e = threadIdx.x; e < nface * ncol; e += blockDim.x) {
      const int f = e / ncol, col = e - f * ncol, bcol = c0 + col;
      const double v = basis_trace(g, d, sd, cv.S, cv.X, rface, ncol, f, col, bcol, bcol < sd.ndof);
      if (bcol < sd.ndof) tr[(long long)bcol * nface + f] = v;
      else fbar[f] = v;
    }
    for (int col = threadIdx.x >> 5; col < ncol; col += blockDim.x >> 5) {
      double sum = 0.0;
      for (int c = threadIdx.x & 31; c < m; c += 32) sum += cv.X[c * ncol + col];
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
      if ((threadIdx.x & 31) == 0) {
        const int bcol = c0 + col;
        if (bcol < sd.ndof) muh[bcol] = sum / m;
        else d.sub_mean[(long long)r * d.st_sub + sidx] = sum / m;
      }
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < sd.ndof; k += blockDim.x)
    phase::element_rhs(g, d, sd, nodes[leaf_node[sidx]], r, k, fbar);
}

// ---------------------------------------------------------------------------------------------
// Warp-per-subdomain kernels (k_local_warp.cuh).  WPB warps per CTA, one subdomain each.

__device__ __forceinline__ void load_kappa_cta(const Grid& g, const DevSub& sd, const double* kap, double* dst) {
  for (int c = threadIdx.x; c < sd.a * sd.b; c += blockDim.x) {
    const int jl = c / sd.a, il = c - jl * sd.a;
    dst[c] = kap[(long long)(sd.y0 + jl) * g.nx + sd.x0 + il];
  }
  __syncthreads();
}

// Robin factorisation at kappa^n (rebuild realisations), stored for reuse by MPM-2P:
// twisted Q blocks [b][A][A] (factor type), [ex, wE, wN, sc] (FP64) and beta_hat per face;
// also stores kappa^m := kappa^n on the subdomain's cells.
template <typename T, int A>
__global__ void k_robin_factor_w(Grid g, DevState d, const DevSub* subs, int scale) {
  extern __shared__ __align__(16) char smem[];
  const int sidx = sub_index(g);
  const int r = blockIdx.y;
  if (d.rebuild[r] != 1) return;
  __shared__ DevSub sd_s;  // the subdomain record, staged once per CTA (indexed by side)
  if (threadIdx.x == 0) sd_s = subs[sidx];
  __syncthreads();
  const DevSub& sd = sd_s;
  const int m = sd.a * sd.b;
  warp::Tables<T> t = warp::carve<T, A>(smem, m, sd.b);
  load_kappa_cta(g, sd, d.kap_n + (long long)r * g.ncell(), t.kap);
  for (int c = threadIdx.x; c < m; c += blockDim.x) {  // kappa^m := kappa^n on this subdomain
    const int jl = c / sd.a, il = c - jl * sd.a;
    d.kap_m[(long long)r * g.ncell() + (long long)(sd.y0 + jl) * g.nx + sd.x0 + il] = t.kap[c];
  }
  warp::build<T, A>(g, sd, t, d.tx + (long long)r * g.nfx(), d.ty + (long long)r * g.nfy(), d.rho_f + sd.face_off,
                    0, scale != 0);
  T* Qg = reinterpret_cast<T*>(d.fac) + (long long)r * d.st_fac + sd.q_off;
  warp::factor<T, A>(sd, t, Qg);
  double* tv = d.tvec + (long long)r * d.st_t + sd.t_off;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    tv[c] = t.ex[c];
    tv[m + c] = t.wE[c];
    tv[2 * m + c] = t.wN[c];
    tv[3 * m + c] = t.sc[c];
  }
  double* bh = d.bhat + (long long)r * d.st_face + sd.face_off;
  for (int f = threadIdx.x; f < 2 * (sd.a + sd.b); f += blockDim.x) {
    int side, tt, cl;
    face_info(sd, f, side, tt, cl);
    bh[f] = sd.side_kind[side] == 1 ? div64(d.rho_f[sd.face_off + f], t.kap[cl]) : 0.0;
  }
}

// MPM-2P local solve: A_i(kappa^m) dp = r_i with zero Robin data and homogeneous physical
// data, using the stored factor (staged into shared memory when qoff != 0, else read from
// global memory).  pass 0 (Eq. mpm_tf_3): r_i is the fine residual
// q h^2 - sum_faces F(kappa^n, p^m) on the subdomain's cells; with store_x the local solution
// is also written to dp0 (the reconstruction adds the BF combination to it).  pass 1 (Eq.
// mpm_tf_4, l = 1): r_i = -(A(kappa^n) - A(kappa^m)) dp0 with homogeneous data, dp0 the
// MRCM-level pressure of the epsilon^0 solve: minus the sum over the cell's faces of
// (T^n - T^m)(dp0_c - dp0_nb) (harmonic transmissibilities; the neighbour across an
// interface from its own subdomain) and, on Dirichlet faces, 2 (kappa^n - kappa^m)_c dp0_c.
// Outputs the perturbation traces (fbar), mean(dp) and the interface right-hand side of the
// subdomain.
// Resident CTAs per SM that the register allocation of the MPM-2P local solve must allow: 768
// threads per SM for factor widths up to 16 (at most 80 registers a thread, no spills; the
// chains of more subdomains in flight hide the latency of the factor loads and shuffles), no
// bound for width 32 (its register-held blocks would spill).
template <int A, int NT>
constexpr int kLocalMinBlocks = A <= 16 ? 768 / NT : 1;

template <typename T, int A, int NT>
__global__ void __launch_bounds__(NT, kLocalMinBlocks<A, NT>) k_mpm_local_w(Grid g, DevState d, const DevSub* subs, size_t qoff,
                                                    int refine, double tol, int ir_max, const DevNode* nodes,
                                                    const int* leaf_node, int pass, int store_x) {
  extern __shared__ __align__(16) char smem[];
  __shared__ double red[64];
  __shared__ double fb[4 * kMaxSide];
  const int sidx = sub_index(g);
  const int r = blockIdx.y;
  if (d.rebuild[r] != 0) return;
  __shared__ DevSub sd_s;  // the subdomain record, staged once per CTA (indexed by side)
  if (threadIdx.x == 0) sd_s = subs[sidx];
  __syncthreads();
  const DevSub& sd = sd_s;
  const int a = sd.a, b = sd.b, m = a * b;
  warp::Tables<T> t = warp::carve<T, A>(smem, m, b);
  const T* Qg = reinterpret_cast<const T*>(d.fac) + (long long)r * d.st_fac + sd.q_off;
  const T* Q = Qg;
  if (qoff != 0) {
    T* Qs = reinterpret_cast<T*>(smem + qoff);
    stage_async(Qs, Qg, (size_t)b * A * A * sizeof(T));
    Q = Qs;
  }
  const double* tv = d.tvec + (long long)r * d.st_t + sd.t_off;
  const int nx = g.nx, ny = g.ny;
  const long long cb = (long long)r * g.ncell();
  const double* tx = d.tx + (long long)r * g.nfx();
  const double* ty = d.ty + (long long)r * g.nfy();
  const double* pm = d.p_m + cb;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    const int jl = c / a, il = c - jl * a;
    const int i = sd.x0 + il, j = sd.y0 + jl;
    const long long gc = (long long)j * nx + i;
    t.kap[c] = d.kap_m[cb + gc];
    t.ex[c] = tv[c];
    t.wE[c] = tv[m + c];
    t.wN[c] = tv[2 * m + c];
    t.sc[c] = tv[3 * m + c];
    const double kc = d.kap_n[cb + gc];
    if (pass == 0) {
      // fine residual r_c = q_c h^2 - sum_faces F_out(kappa^n, p^m)
      const double pc = pm[gc];
      double out = 0.0;
      if (i > 0) out += tx[(long long)j * (nx + 1) + i] * (pc - pm[gc - 1]);
      else out += phys_flux(g, 0, kc, pc);
      if (i < nx - 1) out += tx[(long long)j * (nx + 1) + i + 1] * (pc - pm[gc + 1]);
      else out += phys_flux(g, 1, kc, pc);
      if (j > 0) out += ty[gc] * (pc - pm[gc - nx]);
      else out += phys_flux(g, 2, kc, pc);
      if (j < ny - 1) out += ty[gc + nx] * (pc - pm[gc + nx]);
      else out += phys_flux(g, 3, kc, pc);
      t.B[c] = d.q[cb + gc] * g.h * g.h - out;
    } else {
      // r_c = -sum_faces (T^n - T^m)(x_c - x_nb) - Dirichlet 2 (kappa^n - kappa^m)_c x_c, x = dp0
      const double* x = d.dp0 + cb;
      const double* km = d.kap_m + cb;
      const double xc = x[gc], kmc = km[gc];
      double out = 0.0;
      auto face = [&](double Tn, long long nb) {
        const double kmn = km[nb];
        out += (Tn - div64(2.0 * kmc * kmn, kmc + kmn)) * (xc - x[nb]);
      };
      auto phys = [&](int side) {
        if (g.bc_type[side] == 0) out += 2.0 * (kc - kmc) * xc;
      };
      if (i > 0) face(tx[(long long)j * (nx + 1) + i], gc - 1);
      else phys(0);
      if (i < nx - 1) face(tx[(long long)j * (nx + 1) + i + 1], gc + 1);
      else phys(1);
      if (j > 0) face(ty[gc], gc - nx);
      else phys(2);
      if (j < ny - 1) face(ty[gc + nx], gc + nx);
      else phys(3);
      t.B[c] = -out;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < b * A; e += blockDim.x) {
    const int j = e / A, i = e - j * A;
    t.th[e] = (i < a && j < b - 1) ? warp::scaled_coupling<T>(t.wN[j * a + i], t.sc[j * a + i], t.sc[j * a + i + a])
                                   : T(0);
  }
  if (qoff != 0) cp_async_wait_all();
  __syncthreads();
  warp::solve_refined<T, A>(sd, t, Q, refine != 0, tol, ir_max, d.status, d.ir_iters, red);
  if (store_x)
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
      const int jl = c / a, il = c - jl * a;
      d.dp0[cb + (long long)(sd.y0 + jl) * nx + sd.x0 + il] = t.X[c];
    }
  double* fbar = d.fbar + (long long)r * d.st_face + sd.face_off;
  const int nface = 2 * (a + b);
  for (int f = threadIdx.x; f < nface; f += blockDim.x) {
    int side, tt, cl;
    face_info(sd, f, side, tt, cl);
    const double kc = t.kap[cl], pc = t.X[cl];
    double v;
    if (sd.side_kind[side] == 1) v = div64(kc, 0.5 + d.rho_f[sd.face_off + f]) * pc;
    else v = g.bc_type[side] == 0 ? 2.0 * kc * pc : 0.0;
    fbar[f] = v;
    fb[f] = v;
  }
  double s = 0.0;
  for (int c = threadIdx.x; c < m; c += blockDim.x) s += t.X[c];
  s = warp::cta_sum0(s, red);  // its barrier also orders the fb writes before the reads below
  if (threadIdx.x == 0) d.sub_mean[(long long)r * d.st_sub + sidx] = s / m;
  // Interface right-hand side (Eq. mrc2) from the perturbation traces.
  if (sd.ndof > 0) {
    const DevNode& leaf = nodes[leaf_node[sidx]];
    for (int k = threadIdx.x; k < sd.ndof; k += blockDim.x) phase::element_rhs(g, d, sd, leaf, r, k, fb);
    phase::fold_up(d, nodes, leaf_node[sidx], r);
  }
}

// Downscaling factorisation (Eq. mpm_upd, left-hand side): the pinned Neumann operator of
// kappa^n of every subdomain, factored (twisted block factorisation) into nfac, with its
// FP64 stencil [ex, wE, wN, sc] into ntvec.  It depends only on kappa^n, so the step runs it
// on a side stream concurrently with the perturbation and interface solves.
// reuse_tol > 0 (float32 factors, which the downscaling solve refines in float64 against the
// current operator anyway): a subdomain whose stored factor was computed from transmissibilities
// within a relative reuse_tol of the current ones on every face (and the pinned cell's kappa
// likewise) keeps that factor, its scaling and its pinned cell; only the float64 stencil of
// the current kappa^n is written.  The generalised eigenvalues of the current operator
// against the stored one then lie within 1 -+ reuse_tol, so the refinement's contraction per
// sweep grows by at most about reuse_tol.
template <typename T, int A>
__global__ void k_downscale_factor_w(Grid g, DevState d, const DevSub* subs, int scale, double reuse_tol) {
  extern __shared__ __align__(16) char smem[];
  const int sidx = sub_index(g);
  const int r = blockIdx.y;
  __shared__ DevSub sd_s;  // the subdomain record, staged once per CTA (indexed by side)
  if (threadIdx.x == 0) sd_s = subs[sidx];
  __syncthreads();
  const DevSub& sd = sd_s;
  const int m = sd.a * sd.b;
  warp::Tables<T> t = warp::carve<T, A>(smem, m, sd.b);
  load_kappa_cta(g, sd, d.kap_n + (long long)r * g.ncell(), t.kap);
  const double* txr = d.tx + (long long)r * g.nfx();
  const double* tyr = d.ty + (long long)r * g.nfy();
  double* tv = d.ntvec + (long long)r * d.st_t + sd.t_off;
  double* fw = d.nfw + (long long)r * d.st_t + sd.t_off;
  const long long si = (long long)r * d.st_sub + sidx;
  const int pin_old = reuse_tol > 0.0 ? d.npin[si] : -1;
  if (pin_old >= 0) {
    // |T - T_factor| > reuse_tol T_factor on some face?  (non-negative values compared as bit
    // patterns: integer compares)
    bool far = false;
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
      const int jl = c / sd.a, il = c - jl * sd.a;
      const int i = sd.x0 + il, j = sd.y0 + jl;
      const double we = il < sd.a - 1 ? txr[(long long)j * (g.nx + 1) + i + 1] : 0.0;
      const double wn = jl < sd.b - 1 ? tyr[(long long)(j + 1) * g.nx + i] : 0.0;
      const double fe = fw[c], fn = fw[m + c];
      far |= nn_bits(fabs(we - fe)) > nn_bits(reuse_tol * fe);
      far |= nn_bits(fabs(wn - fn)) > nn_bits(reuse_tol * fn);
      tv[c] = c == pin_old ? t.kap[c] : 0.0;  // ex of the pinned operator, pinned where the factor was
      tv[m + c] = we;
      tv[2 * m + c] = wn;
    }
    if (threadIdx.x == 0) {
      const double kp = d.npin_k[si];
      far |= nn_bits(fabs(t.kap[pin_old] - kp)) > nn_bits(reuse_tol * kp);
    }
    if (!__syncthreads_or(far)) return;  // reused: ntvec holds the current stencil, the stored scaling
  }
  // the pinned cell: the one of largest kappa^n (first on ties).  The pin fixes the pressure
  // constant only (the mean is shifted afterwards), so its place changes no result, but a pin in
  // a low-conductivity cell of a high-contrast field leaves a badly conditioned system that the
  // float32 factor then refines slowly.
  __shared__ int pin_s;
  if (threadIdx.x == 0) {
    int p = 0;
    for (int c = 1; c < m; ++c)
      if (__double_as_longlong(t.kap[c]) > __double_as_longlong(t.kap[p])) p = c;  // positive doubles
    pin_s = p;
  }
  __syncthreads();
  warp::build<T, A>(g, sd, t, d.tx + (long long)r * g.nfx(), d.ty + (long long)r * g.nfy(), d.rho_f + sd.face_off,
                    1 + pin_s, scale != 0);
  warp::factor<T, A>(sd, t, reinterpret_cast<T*>(d.nfac) + (long long)r * d.st_fac + sd.q_off);
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    tv[c] = t.ex[c];
    tv[m + c] = t.wE[c];
    tv[2 * m + c] = t.wN[c];
    tv[3 * m + c] = t.sc[c];
    fw[c] = t.wE[c];
    fw[m + c] = t.wN[c];
  }
  if (threadIdx.x == 0) {
    d.npin[si] = pin_s;
    d.npin_k[si] = t.kap[pin_s];
    atomicAdd(reinterpret_cast<unsigned long long*>(&d.counts[4]), 1ull);
  }
}

// Downscaling solve (Eq. mpm_upd) with the factor of k_downscale_factor_w: u_bar is formed
// from the traces of the interface solve (each realisation with the branch it took), written
// to ux / uy on the faces this subdomain owns (its physical sides, its right and top
// interfaces) and used as Neumann data; solve + FP64 refinement; the pressure constant
// makes mean(p~) equal the target.  Writes p~, the interior fluxes and the subdomain's
// maximum over its cells of max(total outflow, total inflow); the last block to finish
// reduces these maxima per realisation into rate_max (CFL step).  The factor and stencil
// are loaded before pdl_wait() (they come from a stream joined before the launch).
// Resident CTAs per SM that the register allocation of the downscaling solve must allow, for
// factor widths up to 16: 896 threads per SM with float32 factors (at most 72 registers a
// thread), 640 with float64 ones (at most 102); no bound for 32-wide blocks (they would spill).
template <typename T, int A, int NT>
constexpr int kDownscaleMinBlocks = A > 16 ? 1 : (std::is_same<T, float>::value ? 896 : 640) / NT;

template <typename T, int A, int NT>
__global__ void __launch_bounds__(NT, kDownscaleMinBlocks<T, A, NT>) k_downscale_w(Grid g, DevState d, const DevSub* subs, size_t qoff,
                                                               int refine, double tol, int ir_max) {
  extern __shared__ __align__(16) char smem[];
  __shared__ double red[64];
  __shared__ double ub[4 * kMaxSide];  // u_bar per boundary face (face order), +x / +y
  __shared__ int last;
  const int sidx = sub_index(g);
  const int r = blockIdx.y;
  __shared__ DevSub sd_s;  // the subdomain record, staged once per CTA (indexed by side)
  if (threadIdx.x == 0) sd_s = subs[sidx];
  __syncthreads();
  const DevSub& sd = sd_s;
  const int a = sd.a, b = sd.b, m = a * b, nx = g.nx;
  warp::Tables<T> t = warp::carve<T, A>(smem, m, b);
  const T* Qg = reinterpret_cast<const T*>(d.nfac) + (long long)r * d.st_fac + sd.q_off;
  const T* Q = Qg;  // staged into shared memory when qoff != 0, else read from global memory
  if (qoff != 0) {
    T* Qs = reinterpret_cast<T*>(smem + qoff);
    stage_async(Qs, Qg, (size_t)b * A * A * sizeof(T));
    Q = Qs;
  }
  const bool warm = refine != 0;  // refined solves start from the previous step's solution
  {
    const double* tv = d.ntvec + (long long)r * d.st_t + sd.t_off;
    const double* xw = d.x_ds + (long long)r * g.ncell();
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
      t.ex[c] = tv[c];
      t.wE[c] = tv[m + c];
      t.wN[c] = tv[2 * m + c];
      t.sc[c] = tv[3 * m + c];
      if (warm) {
        const int jl = c / a, il = c - jl * a;
        t.X[c] = xw[(long long)(sd.y0 + jl) * g.nx + sd.x0 + il];
      }
    }
  }
  __syncthreads();
  // the factor's own couplings: the north transmissibilities it was computed from (equal to the
  // current ones unless the factor was kept, see k_downscale_factor_w)
  const double* fwN = d.nfw + (long long)r * d.st_t + sd.t_off + m;
  for (int e = threadIdx.x; e < b * A; e += blockDim.x) {
    const int j = e / A, i = e - j * A;
    t.th[e] = (i < a && j < b - 1) ? warp::scaled_coupling<T>(fwN[j * a + i], t.sc[j * a + i], t.sc[j * a + i + a])
                                   : T(0);
  }
  const double* qc = d.q + (long long)r * g.ncell();
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    const int jl = c / a, il = c - jl * a;
    t.B[c] = qc[(long long)(sd.y0 + jl) * nx + sd.x0 + il] * g.h * g.h;
  }
  if (qoff != 0) cp_async_wait_all();
  pdl_wait();
  double* uxw = d.ux + (long long)r * g.nfx();
  double* uyw = d.uy + (long long)r * g.nfy();
  const int branch = d.rebuild[r] != 0 ? 1 : 0;
  for (int f = threadIdx.x; f < 2 * (a + b); f += blockDim.x) {
    int side, tt, cl;
    face_info(sd, f, side, tt, cl);
    const double v = phase::ubar_face(g, d, subs, sd, r, side, tt, branch);
    ub[f] = v;
    if (sd.side_kind[side] == 1 && (side == 0 || side == 2)) continue;  // written by the neighbour
    const int il = cl % a, jl = cl / a;
    const int i = sd.x0 + il, j = sd.y0 + jl;
    if (side == 0) uxw[(long long)j * (nx + 1) + i] = v;
    else if (side == 1) uxw[(long long)j * (nx + 1) + i + 1] = v;
    else if (side == 2) uyw[(long long)j * nx + i] = v;
    else uyw[(long long)(j + 1) * nx + i] = v;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    const int jl = c / a, il = c - jl * a;
    double v = t.B[c];
    if (il == 0) v += ub[jl];
    if (il == a - 1) v -= ub[b + jl];
    if (jl == 0) v += ub[2 * b + il];
    if (jl == b - 1) v -= ub[2 * b + a + il];
    t.B[c] = v;
  }
  __syncthreads();
  warp::solve_refined<T, A>(sd, t, Q, refine != 0, tol, ir_max, d.status, d.ir_iters, red, warm);
  double s = 0.0;
  for (int c = threadIdx.x; c < m; c += blockDim.x) s += t.X[c];
  s = warp::cta_sum0(s, red);
  __shared__ double shift_s;
  if (threadIdx.x == 0) shift_s = d.sub_target[(long long)r * d.st_sub + sidx] - s / m;
  __syncthreads();
  const double shift = shift_s;
  // east / north face fluxes of every cell (along +x / +y, as stored in ux / uy), each
  // computed once; the residual and right-hand side buffers are free after the solve
  double* FE = t.Rr;
  double* FN = t.B;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    const int jl = c / a, il = c - jl * a;
    const int i = sd.x0 + il, j = sd.y0 + jl;
    d.p_down[(long long)r * g.ncell() + (long long)j * nx + i] = t.X[c] + shift;
    if (warm) d.x_ds[(long long)r * g.ncell() + (long long)j * nx + i] = t.X[c];
    const double fe = il == a - 1 ? ub[b + jl] : t.wE[c] * (t.X[c] - t.X[c + 1]);
    const double fn = jl == b - 1 ? ub[2 * b + a + il] : t.wN[c] * (t.X[c] - t.X[c + a]);
    if (il < a - 1) uxw[(long long)j * (nx + 1) + i + 1] = fe;
    if (jl < b - 1) uyw[(long long)(j + 1) * nx + i] = fn;
    FE[c] = fe;
    FN[c] = fn;
  }
  __syncthreads();
  // max over the cells of max(total outflow, total inflow); signs from the bit patterns, and
  // the maxima (of non-negative sums) on the bit patterns too
  unsigned long long rate_b = 0;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    const int jl = c / a, il = c - jl * a;
    const double o[4] = {-(il == 0 ? ub[jl] : FE[c - 1]), FE[c], -(jl == 0 ? ub[2 * b + il] : FN[c - a]), FN[c]};
    double out = 0.0, in = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (dpos(o[k])) out += o[k];
      else if (dneg(o[k])) in -= o[k];
    }
    const unsigned long long uo = nn_bits(out), ui = nn_bits(in);
    const unsigned long long u = uo > ui ? uo : ui;
    rate_b = u > rate_b ? u : rate_b;
  }
  const double rate = nn_from_bits(warp::cta_max_bits(rate_b, red));
  // last-block reduction of the per-subdomain maxima (threadfence-reduction pattern)
  if (threadIdx.x == 0) {
    d.rate_part[(long long)r * d.st_sub + sidx] = rate;
    __threadfence();
    const unsigned int nblk = (unsigned int)d.st_sub * gridDim.y;  // every subdomain, over all launches
    last = atomicAdd(&d.ticket[0], 1u) == nblk - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int nsub = d.st_sub;
  for (int rr = 0; rr < (int)gridDim.y; ++rr) {
    unsigned long long mb = 0;
    for (int k = threadIdx.x; k < nsub; k += blockDim.x) {
      const unsigned long long u = nn_bits(__ldcg(&d.rate_part[(long long)rr * d.st_sub + k]));
      mb = u > mb ? u : mb;
    }
    const double mx = nn_from_bits(warp::cta_max_bits(mb, red));
    if (threadIdx.x == 0) {
      d.rate_max[rr] = mx;
      d.inv_rate[rr] = mx > 0.0 ? 1.0 / mx : 0.0;
    }
  }
  if (threadIdx.x == 0) d.ticket[0] = 0;
}

template <typename K>
void set_smem(K kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  // all of the unified L1 / shared storage that shared memory may take: the occupancy of these
  // kernels is bounded by their shared tables, and their global loads are read-once streams
  cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}

size_t align16(size_t v) { return (v + 15) / 16 * 16; }

// Launch geometry of the two-warp kernels: one subdomain per CTA of 64 threads (spreads
// the subdomains over all SMs); dynamic shared memory = tables (+ the factor for the
// downscaling).
template <typename T, int A>
void pair_geometry(int max_a, int max_b, bool with_q, size_t& bytes, size_t& qoff) {
  const int m = max_a * max_b;
  qoff = align16(warp::table_bytes<T, A>(m, max_b));
  bytes = align16(qoff + (with_q ? (size_t)max_b * A * A * sizeof(T) : 0));
}

template <typename T, int A>
void robin_factor_t(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a, int max_b,
                    cudaStream_t st) {
  size_t bytes, qoff;
  pair_geometry<T, A>(max_a, max_b, false, bytes, qoff);
  set_smem(k_robin_factor_w<T, A>, bytes);
  k_robin_factor_w<T, A><<<dim3(nsub, g.R), 64, bytes, st>>>(g, d, subs, std::is_same<T, float>::value ? 1 : 0);
  ++g_launches;
}

template <typename T, int A, int NT>
void mpm_local_nt(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a, int max_b, int refine,
                  double tol, int ir_max, const DevNode* nodes, const int* leaf_node, int stage, int pass,
                  cudaStream_t st) {
  size_t bytes, qoff;
  pair_geometry<T, A>(max_a, max_b, stage != 0, bytes, qoff);  // stored factor staged in shared memory ...
  if (stage == 0 || bytes > (size_t)kSmemBudget) {              // ... or read from global memory
    pair_geometry<T, A>(max_a, max_b, false, bytes, qoff);
    qoff = 0;
  }
  set_smem(k_mpm_local_w<T, A, NT>, bytes);
  k_mpm_local_w<T, A, NT><<<dim3(nsub, g.R), NT, bytes, st>>>(g, d, subs, qoff, refine, tol, ir_max, nodes, leaf_node,
                                                               pass, pass == 0 && g.order >= 1 ? 1 : 0);
  ++g_launches;
}

template <typename T, int A>
void mpm_local_t(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a, int max_b, int refine,
                 double tol, int ir_max, const DevNode* nodes, const int* leaf_node, int threads, int stage, int pass,
                 cudaStream_t st) {
  if (threads <= 64)
    mpm_local_nt<T, A, 64>(g, d, subs, nsub, max_a, max_b, refine, tol, ir_max, nodes, leaf_node, stage, pass, st);
  else if (threads <= 128)
    mpm_local_nt<T, A, 128>(g, d, subs, nsub, max_a, max_b, refine, tol, ir_max, nodes, leaf_node, stage, pass, st);
  else mpm_local_nt<T, A, 256>(g, d, subs, nsub, max_a, max_b, refine, tol, ir_max, nodes, leaf_node, stage, pass, st);
}

template <typename T, int A>
void downscale_factor_t(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a, int max_b,
                        double reuse_tol, cudaStream_t st) {
  size_t bytes, qoff;
  pair_geometry<T, A>(max_a, max_b, false, bytes, qoff);
  set_smem(k_downscale_factor_w<T, A>, bytes);
  k_downscale_factor_w<T, A><<<dim3(nsub, g.R), 64, bytes, st>>>(g, d, subs, std::is_same<T, float>::value ? 1 : 0,
                                                                   reuse_tol);
  ++g_launches;
}

template <typename T, int A, int NT>
void downscale_nt(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a, int max_b, int refine,
                  double tol, int ir_max, bool pdl, int stage, cudaStream_t st) {
  size_t bytes, qoff;
  pair_geometry<T, A>(max_a, max_b, stage != 0, bytes, qoff);
  if (stage == 0 || bytes > (size_t)kSmemBudget) {  // factor read from global memory
    pair_geometry<T, A>(max_a, max_b, false, bytes, qoff);
    qoff = 0;
  }
  set_smem(k_downscale_w<T, A, NT>, bytes);
  launch_ex(k_downscale_w<T, A, NT>, dim3(nsub, g.R), dim3(NT), bytes, st, pdl, g, d, subs, qoff, refine, tol, ir_max);
}

template <typename T, int A>
void downscale_t(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a, int max_b, int refine,
                 double tol, int ir_max, bool pdl, int threads, int stage, cudaStream_t st) {
  if (threads <= 64) downscale_nt<T, A, 64>(g, d, subs, nsub, max_a, max_b, refine, tol, ir_max, pdl, stage, st);
  else if (threads <= 128) downscale_nt<T, A, 128>(g, d, subs, nsub, max_a, max_b, refine, tol, ir_max, pdl, stage, st);
  else downscale_nt<T, A, 256>(g, d, subs, nsub, max_a, max_b, refine, tol, ir_max, pdl, stage, st);
}

template <int A, int KIND>
void basis_tc_launch(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a, int max_b, double tol,
                     int ir_max, const DevNode* nodes, const int* leaf_node, cudaStream_t st) {
  const TcPlan pl = plan_tc(max_a, max_b, A);
  set_smem(k_basis_solve_tc<A, KIND>, pl.bytes);
  k_basis_solve_tc<A, KIND><<<dim3(nsub, g.R), 256, pl.bytes, st>>>(g, d, subs, pl.ncol, pl.ld, tol, ir_max, nodes,
                                                                    leaf_node);
  ++g_launches;
}

template <int A>
void basis_tc_kind(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a, int max_b, int kind,
                   double tol, int ir_max, const DevNode* nodes, const int* leaf_node, cudaStream_t st) {
  if (kind == tc::kTf32) basis_tc_launch<A, tc::kTf32>(g, d, subs, nsub, max_a, max_b, tol, ir_max, nodes, leaf_node, st);
  else if (kind == tc::kTf32x3)
    basis_tc_launch<A, tc::kTf32x3>(g, d, subs, nsub, max_a, max_b, tol, ir_max, nodes, leaf_node, st);
  else basis_tc_launch<A, tc::kBf16>(g, d, subs, nsub, max_a, max_b, tol, ir_max, nodes, leaf_node, st);
}

}  // namespace

int local_smem_limit() { return kSmemBudget; }

#define MPM_DISPATCH_A(FN, T, ...)                         \
  do {                                                     \
    const int A_ = pad_width(max_a);                       \
    if (A_ == 8) FN<T, 8>(__VA_ARGS__);                    \
    else if (A_ == 16) FN<T, 16>(__VA_ARGS__);             \
    else FN<T, 32>(__VA_ARGS__);                           \
  } while (0)

void launch_robin_factor(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a, int max_b,
                         bool fp32, cudaStream_t st) {
  if (fp32) MPM_DISPATCH_A(robin_factor_t, float, g, d, subs, nsub, max_a, max_b, st);
  else MPM_DISPATCH_A(robin_factor_t, double, g, d, subs, nsub, max_a, max_b, st);
}

void launch_basis_solve(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a, int max_b,
                        int tc_kind, bool fp32, double ir_tol, int ir_max, const DevNode* nodes,
                        const int* leaf_node, cudaStream_t st) {
  dim3 grid(nsub, g.R);
  const int thr = 256;
  const int A = pad_width(max_a);
  // tensor cores (float32 factor), unless the class's tables exceed shared memory (sides of
  // 20 x 24 cells and up): those take the float32 CUDA-core solve below, same factor and outputs
  if (tc_kind != 0 && plan_tc(max_a, max_b, A).bytes <= (size_t)kSmemBudget) {
    if (A == 8) basis_tc_kind<8>(g, d, subs, nsub, max_a, max_b, tc_kind, ir_tol, ir_max, nodes, leaf_node, st);
    else if (A == 16) basis_tc_kind<16>(g, d, subs, nsub, max_a, max_b, tc_kind, ir_tol, ir_max, nodes, leaf_node, st);
    else basis_tc_kind<32>(g, d, subs, nsub, max_a, max_b, tc_kind, ir_tol, ir_max, nodes, leaf_node, st);
    return;
  }
  // the stored factor is staged in shared memory unless that leaves room for fewer than 8
  // right-hand-side columns per pass (large padded blocks): then it is read in place.  With
  // fewer than 4 CTAs per SM, the column chunks of a subdomain are spread over up to 4 CTAs.
  const int per = nsub * g.R;
  grid.z = per >= 4 * sm_count() ? 1 : std::min(4, (4 * sm_count() + per - 1) / per);
  if (fp32) {
    SmemPlan pl = plan_smem<float>(max_a, max_b, A, 32);
    const bool qg = pl.ncol < 8;
    if (qg) pl = plan_smem<float>(max_a, max_b, A, 32, true);
    set_smem(k_basis_solve<float>, pl.bytes);
    k_basis_solve<float><<<grid, thr, pl.bytes, st>>>(g, d, subs, A, pl.ncol, 1, ir_tol, ir_max, nodes, leaf_node,
                                                       qg ? 1 : 0);
  } else {
    // float64 without refinement: the direct layout (right-hand side and solution in the
    // workspace), up to 64 columns per pass, or as many as spread the columns of the widest
    // subdomain (2 (a + b) / seg_len segments of degree + 1 functions, U and P, plus the
    // non-homogeneous column) evenly over the CTAs of a subdomain
    const int ntot = 2 * (g.degree + 1) * (2 * max_a + 2 * max_b) / g.seg_len + 1;
    const int cap = grid.z > 1 ? std::min(64, ((int)(ntot + grid.z - 1) / (int)grid.z)) : 64;
    SmemPlan pl = plan_smem<double>(max_a, max_b, A, cap, false, true);
    const bool qg = pl.ncol < 8 && pl.ncol < cap;
    if (qg) pl = plan_smem<double>(max_a, max_b, A, cap, true, true);
    set_smem(k_basis_solve<double>, pl.bytes);
    k_basis_solve<double><<<grid, thr, pl.bytes, st>>>(g, d, subs, A, pl.ncol, 0, ir_tol, ir_max, nodes,
                                                         leaf_node, qg ? 1 : 0);
  }
  ++g_launches;
}

void launch_mpm_local(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a, int max_b,
                      bool fp32, double ir_tol, int ir_max, const DevNode* nodes, const int* leaf_node, int threads,
                      int stage, int pass, cudaStream_t st) {
  if (fp32)
    MPM_DISPATCH_A(mpm_local_t, float, g, d, subs, nsub, max_a, max_b, 1, ir_tol, ir_max, nodes, leaf_node, threads,
                   stage, pass, st);
  else
    MPM_DISPATCH_A(mpm_local_t, double, g, d, subs, nsub, max_a, max_b, 0, ir_tol, ir_max, nodes, leaf_node, threads,
                   stage, pass, st);
}

void launch_downscale_factor(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a, int max_b,
                             bool fp32, double reuse_tol, cudaStream_t st) {
  if (fp32) MPM_DISPATCH_A(downscale_factor_t, float, g, d, subs, nsub, max_a, max_b, reuse_tol, st);
  else MPM_DISPATCH_A(downscale_factor_t, double, g, d, subs, nsub, max_a, max_b, 0.0, st);
}

void launch_downscale(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_a, int max_b,
                      bool fp32, double ir_tol, int ir_max, bool pdl, int threads, int stage, cudaStream_t st) {
  if (fp32) MPM_DISPATCH_A(downscale_t, float, g, d, subs, nsub, max_a, max_b, 1, ir_tol, ir_max, pdl, threads, stage, st);
  else MPM_DISPATCH_A(downscale_t, double, g, d, subs, nsub, max_a, max_b, 0, ir_tol, ir_max, pdl, threads, stage, st);
}

}  // namespace mpm
