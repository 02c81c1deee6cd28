// Warp-per-subdomain local solver for single right-hand sides (MPM-2P local solve and
// downscaling).  Same block-tridiagonal LDL^T with explicit inverse pivots as the
// CTA-wide path in k_local.cu, but one warp owns one subdomain:
//   - the a x a pivot block S_j is held in registers, identity-padded to A x A
//     (A in {8, 16, 32}): lane l holds column c = l % A, rows r = (l / A) * NR + q,
//     q < NR = A*A/32;
//   - Gauss-Jordan inversion exchanges the pivot row / column by warp shuffles, with no
//     block barrier (an inverted padded block is [S^-1 0; 0 I]);
//   - S_j = D_j - t_{j-1} o Q_{j-1} o t_{j-1} is formed in the registers that still hold
//     Q_{j-1} (the couplings between grid rows are diagonal);
//   - a solve is 2b dependent A x A products, each lane reducing its rows by shuffles.
// All inner loops run in the factor type T; the scaled couplings are precomputed once.
#pragma once
#include "mpm2p_internal.cuh"

namespace mpm {
namespace warp {

// Per-warp shared-memory tables of one subdomain (a x b cells, m = a b, padded width A).
template <typename T>
struct Tables {
  double* kap;  // m
  double* ex;   // m  diagonal part not due to interior faces
  double* wE;   // m  east transmissibility (0 on the last column)
  double* wN;   // m  north transmissibility (0 on the last row)
  double* sc;   // m  Jacobi scaling
  double* X;    // m  FP64 solution
  double* B;    // m  FP64 right-hand side
  double* Rr;   // m  FP64 residual
  T* dh;        // b*A  scaled diagonal (padding: 1)
  T* eh;        // b*A  scaled coupling to the east neighbour (padding: 0)
  T* th;        // b*A  scaled coupling to the north neighbour, positive (padding: 0)
  T* V;         // b*A  work vector (padded)
  T* W;         // b*A  forward products
};

template <typename T, int A>
__host__ __device__ constexpr size_t table_bytes(int m, int b) {
  return (size_t)8 * m * sizeof(double) + (size_t)5 * b * A * sizeof(T);
}

template <typename T, int A>
__device__ Tables<T> carve(char* base, int m, int b) {
  Tables<T> t;
  double* p = reinterpret_cast<double*>(base);
  t.kap = p; p += m;
  t.ex = p; p += m;
  t.wE = p; p += m;
  t.wN = p; p += m;
  t.sc = p; p += m;
  t.X = p; p += m;
  t.B = p; p += m;
  t.Rr = p; p += m;
  T* q = reinterpret_cast<T*>(p);
  t.dh = q; q += b * A;
  t.eh = q; q += b * A;
  t.th = q; q += b * A;
  t.V = q; q += b * A;
  t.W = q;
  return t;
}

// FP64 stencil of the Robin (neumann = 0) or pinned Neumann (neumann = 1) operator of
// kappa^n (transmissibilities tx / ty of the current kappa^n, r-th realisation pointers),
// and the scaled T tables.  kap must already hold the subdomain's kappa^n.
template <typename T, int A>
__device__ void build(const Grid& g, const DevSub& sd, Tables<T> t, const double* tx, const double* ty,
                      int neumann, bool scale, int lane) {
  const int a = sd.a, b = sd.b, m = a * b;
  for (int c = lane; c < m; c += 32) {
    const int jl = c / a, il = c - jl * a;
    const int i = sd.x0 + il, j = sd.y0 + jl;
    const double kc = t.kap[c];
    t.wE[c] = il < a - 1 ? tx[(long long)j * (g.nx + 1) + i + 1] : 0.0;
    t.wN[c] = jl < b - 1 ? ty[(long long)(j + 1) * g.nx + i] : 0.0;
    double dg = 0.0;
    if (!neumann) {
      if (il == 0) dg += sd.side_kind[0] == 1 ? kc / (0.5 + sd.side_rho[0]) : (g.bc_type[0] == 0 ? 2.0 * kc : 0.0);
      if (il == a - 1) dg += sd.side_kind[1] == 1 ? kc / (0.5 + sd.side_rho[1]) : (g.bc_type[1] == 0 ? 2.0 * kc : 0.0);
      if (jl == 0) dg += sd.side_kind[2] == 1 ? kc / (0.5 + sd.side_rho[2]) : (g.bc_type[2] == 0 ? 2.0 * kc : 0.0);
      if (jl == b - 1) dg += sd.side_kind[3] == 1 ? kc / (0.5 + sd.side_rho[3]) : (g.bc_type[3] == 0 ? 2.0 * kc : 0.0);
    } else if (c == 0) {
      dg += kc;  // pin: A + kappa_0 e_0 e_0^T
    }
    t.ex[c] = dg;
  }
  __syncwarp();
  for (int c = lane; c < m; c += 32) {
    const int jl = c / a, il = c - jl * a;
    double d = t.ex[c] + t.wE[c] + t.wN[c];
    if (il > 0) d += t.wE[c - 1];
    if (jl > 0) d += t.wN[c - a];
    t.sc[c] = scale ? rsqrt(d) : 1.0;
    t.Rr[c] = d;  // full diagonal, consumed below
  }
  __syncwarp();
  for (int e = lane; e < b * A; e += 32) {
    const int j = e / A, i = e - j * A;
    if (i < a) {
      const int c = j * a + i;
      t.dh[e] = T(t.Rr[c] * t.sc[c] * t.sc[c]);
      t.eh[e] = i < a - 1 ? T(-t.wE[c] * t.sc[c] * t.sc[c + 1]) : T(0);
      t.th[e] = j < b - 1 ? T(t.wN[c] * t.sc[c] * t.sc[c + a]) : T(0);
    } else {
      t.dh[e] = T(1);
      t.eh[e] = T(0);
      t.th[e] = T(0);
    }
  }
  __syncwarp();
}

// Reciprocal of a pivot: FP32 uses the hardware approximation (<= 2 ulp), which the FP64
// refinement absorbs; FP64 keeps the correctly rounded division.
__device__ __forceinline__ float pivot_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double pivot_rcp(double x) { return 1.0 / x; }

// In-register Gauss-Jordan inversion of the padded A x A block.  Pivot p:
//   M[p][p] <- 1/M[p][p],  M[p][c] <- M[p][c]/M[p][p],  M[r][p] <- -M[r][p]/M[p][p],
//   M[r][c] <- M[r][c] - M[r][p] M[p][c]/M[p][p]  otherwise.
// Row p is held in slot p % NR of the lanes with h == p / NR, so only that slot needs the
// pivot-row case; the pivot-column case is folded into a per-lane multiplier.
template <typename T, int A>
__device__ __forceinline__ void gj_invert(T (&v)[A * A / 32], int lane) {
  constexpr int NR = A * A / 32;
  const int c = lane % A, h = lane / A;
#pragma unroll
  for (int p = 0; p < A; ++p) {
    const T rowv = __shfl_sync(0xffffffffu, v[p % NR], c + A * (p / NR));  // M[p][c]
    const T piv = __shfl_sync(0xffffffffu, rowv, p);                       // M[p][p]
    const T ip = pivot_rcp(piv);
    const bool pc = c == p;
    const T keep = pc ? T(0) : T(1);        // the pivot column is replaced, not updated
    const T sc = pc ? ip : rowv * ip;       // M[p][c] / M[p][p], or 1/M[p][p] in the pivot column
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const T colv = __shfl_sync(0xffffffffu, v[q], p + A * h);  // M[r][p]
      if (q == p % NR && h == p / NR) v[q] = sc;                  // pivot row
      else v[q] = keep * v[q] - colv * sc;
    }
  }
}

// Factor: Q_j = S_j^-1 for j = 0..b-1, written to Q ([b][A][A], padded).
template <typename T, int A>
__device__ void factor(const DevSub& sd, Tables<T> t, T* Q, int lane) {
  constexpr int NR = A * A / 32;
  const int c = lane % A, h = lane / A;
  T v[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) v[q] = T(0);
  for (int j = 0; j < sd.b; ++j) {
    const T tc = j > 0 ? t.th[(j - 1) * A + c] : T(0);
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const int r = h * NR + q;
      T s = r == c ? t.dh[j * A + r] : (c == r + 1 ? t.eh[j * A + r] : (r == c + 1 ? t.eh[j * A + c] : T(0)));
      if (j > 0) s -= t.th[(j - 1) * A + r] * v[q] * tc;
      v[q] = s;
    }
    gj_invert<T, A>(v, lane);
    T* Qj = Q + (size_t)j * A * A;
#pragma unroll
    for (int q = 0; q < NR; ++q) Qj[(h * NR + q) * A + c] = v[q];
  }
  __syncwarp();
}

// y[c] = sum_r Q[r][c] x[r] for the lane's column c (Q symmetric), x held as x[lane % A].
template <typename T, int A>
__device__ __forceinline__ T matvec(const T* Qj, T x, int lane) {
  constexpr int NR = A * A / 32;
  const int c = lane % A, h = lane / A;
  T acc = T(0);
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    const int r = h * NR + q;
    acc += Qj[r * A + c] * __shfl_sync(0xffffffffu, x, r);
  }
#pragma unroll
  for (int o = A; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// Solve (S A S) y = V in place (V, W: [b][A] padded, W workspace).
template <typename T, int A>
__device__ void solve(const DevSub& sd, Tables<T> t, const T* Q, int lane) {
  const int c = lane % A;
  const int b = sd.b;
  T w = T(0);
  for (int j = 0; j < b; ++j) {
    T u = t.V[j * A + c];
    if (j > 0) u += t.th[(j - 1) * A + c] * w;
    w = matvec<T, A>(Q + (size_t)j * A * A, u, lane);
    if (lane < A) t.W[j * A + c] = w;
  }
  __syncwarp();
  T x = w;  // X_{b-1} = W_{b-1}
  if (lane < A) t.V[(b - 1) * A + c] = x;
  for (int j = b - 2; j >= 0; --j) {
    const T u = t.th[j * A + c] * x;
    x = t.W[j * A + c] + matvec<T, A>(Q + (size_t)j * A * A, u, lane);
    if (lane < A) t.V[j * A + c] = x;
  }
  __syncwarp();
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// (A x)_c in flux form (see k_local.cu) and the cell's flux scale.
__device__ __forceinline__ double apply_A(const DevSub& sd, const double* ex, const double* wE, const double* wN,
                                          const double* x, int c, double& absx) {
  const int a = sd.a, b = sd.b;
  const int jl = c / a, il = c - jl * a;
  const double xc = x[c];
  double t0 = ex[c] * xc, t1 = 0.0, t2 = 0.0, t3 = 0.0, t4 = 0.0;
  if (il < a - 1) t1 = wE[c] * (xc - x[c + 1]);
  if (il > 0) t2 = wE[c - 1] * (xc - x[c - 1]);
  if (jl < b - 1) t3 = wN[c] * (xc - x[c + a]);
  if (jl > 0) t4 = wN[c - a] * (xc - x[c - a]);
  absx = fabs(t0) + fabs(t1) + fabs(t2) + fabs(t3) + fabs(t4);
  return (t0 + t1) + (t2 + t3) + t4;
}

// Refined solve of A x = B (FP64, t.B) into t.X; same stopping rule as the CTA path
// with target = tol.
template <typename T, int A>
__device__ void solve_refined(const DevSub& sd, Tables<T> t, const T* Q, bool refine, double tol, int ir_max,
                              int* status, int* ir_used, int lane) {
  const double target = tol;
  const int a = sd.a, b = sd.b, m = a * b;
  for (int c = lane; c < m; c += 32) {
    t.X[c] = 0.0;
    t.Rr[c] = t.B[c];
  }
  __syncwarp();
  const int sweeps = refine ? ir_max : 1;
  int it = 0;
  bool ok = false;
  double eta_prev = 1e300;
  for (; it < sweeps; ++it) {
    for (int e = lane; e < b * A; e += 32) {
      const int j = e / A, i = e - j * A;
      t.V[e] = i < a ? T(t.Rr[j * a + i] * t.sc[j * a + i]) : T(0);
    }
    __syncwarp();
    solve<T, A>(sd, t, Q, lane);
    for (int c = lane; c < m; c += 32) {
      const int j = c / a, i = c - j * a;
      t.X[c] += double(t.V[j * A + i]) * t.sc[c];
    }
    __syncwarp();
    if (!refine) { it = 1; ok = true; break; }
    double rmax = 0.0, smax = 0.0;
    for (int c = lane; c < m; c += 32) {
      double absx;
      const double r = t.B[c] - apply_A(sd, t.ex, t.wE, t.wN, t.X, c, absx);
      t.Rr[c] = r;
      rmax = fmax(rmax, fabs(r));
      smax = fmax(smax, absx + fabs(t.B[c]));
    }
    rmax = warp_max(rmax);
    smax = warp_max(smax);
    __syncwarp();
    const double eta = smax > 0.0 ? rmax / smax : 0.0;
    if (eta <= target) { ok = true; ++it; break; }
    if (eta > 0.5 * eta_prev && eta <= 1e3 * tol) { ok = true; ++it; break; }  // FP64 floor reached
    eta_prev = eta;
  }
  if (lane == 0) {
    if (!ok) atomicOr(status, 1);
    atomicMax(ir_used, it);
  }
  __syncwarp();
}

}  // namespace warp
}  // namespace mpm
