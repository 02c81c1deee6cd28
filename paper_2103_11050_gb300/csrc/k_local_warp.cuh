// Two-warp-per-subdomain local solver for single right-hand sides (Robin factorisation,
// MPM-2P local solve and downscaling).  Block-tridiagonal LDL^T with explicit inverse
// pivots, factored from both ends (twisted); each warp owns one chain:
//   - the a x a pivot block S_j is held in registers, identity-padded to A x A
//     (A in {8, 16, 32}): lane l holds column c = l % A, rows r = (l / A) * NR + q,
//     q < NR = A*A/32;
//   - Gauss-Jordan inversion exchanges the pivot row / column by warp shuffles, with no
//     block barrier (an inverted padded block is [S^-1 0; 0 I]);
//   - S_j = D_j - t_{j-1} o Q_{j-1} o t_{j-1} is formed in the registers that still hold
//     Q_{j-1} (the couplings between grid rows are diagonal);
//   - a solve is ~b + 1 dependent A x A products per warp chain, each lane reducing its rows
//     by shuffles.
// All inner loops run in the factor type T; the scaled couplings are precomputed once.
#pragma once
#include "mpm2p_internal.cuh"

namespace mpm {
namespace warp {

// float64 -> factor type T and back.  For float32 both run on the integer units
// (fp_bits.cuh): rounding to nearest even, and exact widening, over the float32 normal range,
// which holds the scaled factors, residuals and corrections; anything smaller than 2^-126
// becomes zero.
template <typename T>
__device__ __forceinline__ T to_T(double x);
template <>
__device__ __forceinline__ double to_T<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_T<float>(double x) { return f64_to_f32_rn(x); }
__device__ __forceinline__ double from_T(double v) { return v; }
__device__ __forceinline__ double from_T(float v) { return f32_to_f64(v); }

// Float64 factors are built from the unscaled operator (Jacobi scaling only for float32).
template <typename T>
constexpr bool kUnscaled = sizeof(T) == sizeof(double);

// The scaled north coupling t_j sc_c sc_c+a of the padded tables (T = float), or t_j itself.
template <typename T>
__device__ __forceinline__ T scaled_coupling(double wN, double sc0, double sc1) {
  if constexpr (kUnscaled<T>) return wN;
  else return to_T<T>(wN * sc0 * sc1);
}

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
  double* fE;   // m  east face flux wE (x_c - x_east) of the current iterate (0 on the last column)
  double* fN;   // m  north face flux wN (x_c - x_north) (0 on the last row)
  T* dh;        // b*A  scaled diagonal (padding: 1)
  T* eh;        // b*A  scaled coupling to the east neighbour (padding: 0)
  T* th;        // b*A  scaled coupling to the north neighbour, positive (padding: 0)
  T* V;         // b*A  work vector (padded)
  T* W;         // b*A  forward products
};

template <typename T, int A>
__host__ __device__ constexpr size_t table_bytes(int m, int b) {
  return (size_t)10 * m * sizeof(double) + (size_t)5 * b * A * sizeof(T);
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
  t.fE = p; p += m;
  t.fN = p; p += m;
  T* q = reinterpret_cast<T*>(p);
  t.dh = q; q += b * A;
  t.eh = q; q += b * A;
  t.th = q; q += b * A;
  t.V = q; q += b * A;
  t.W = q;
  return t;
}

// FP64 stencil of the Robin (neumann = 0) or pinned Neumann (neumann = 1 + the pinned cell) operator of
// kappa^n (transmissibilities tx / ty of the current kappa^n, r-th realisation pointers;
// rho: the subdomain's per-face rho_e = alpha_e H_e / h), and the scaled T tables.  kap must
// already hold the subdomain's kappa^n.
template <typename T, int A>
__device__ void build(const Grid& g, const DevSub& sd, Tables<T> t, const double* tx, const double* ty,
                      const double* rho, int neumann, bool scale) {
  const int a = sd.a, b = sd.b, m = a * b;
  const int lane = threadIdx.x;
  for (int c = lane; c < m; c += blockDim.x) {
    const int jl = c / a, il = c - jl * a;
    const int i = sd.x0 + il, j = sd.y0 + jl;
    const double kc = t.kap[c];
    t.wE[c] = il < a - 1 ? tx[(long long)j * (g.nx + 1) + i + 1] : 0.0;
    t.wN[c] = jl < b - 1 ? ty[(long long)(j + 1) * g.nx + i] : 0.0;
    double dg = 0.0;
    if (!neumann) {
      // rho of this cell's face on each side (face numbering: left, right, bottom, top)
      if (il == 0) dg += sd.side_kind[0] == 1 ? div64(kc, 0.5 + rho[jl]) : (g.bc_type[0] == 0 ? 2.0 * kc : 0.0);
      if (il == a - 1) dg += sd.side_kind[1] == 1 ? div64(kc, 0.5 + rho[b + jl]) : (g.bc_type[1] == 0 ? 2.0 * kc : 0.0);
      if (jl == 0) dg += sd.side_kind[2] == 1 ? div64(kc, 0.5 + rho[2 * b + il]) : (g.bc_type[2] == 0 ? 2.0 * kc : 0.0);
      if (jl == b - 1)
        dg += sd.side_kind[3] == 1 ? div64(kc, 0.5 + rho[2 * b + a + il]) : (g.bc_type[3] == 0 ? 2.0 * kc : 0.0);
    } else if (c == neumann - 1) {
      dg += kc;  // pin: A + kappa_p e_p e_p^T at the pinned cell p = neumann - 1
    }
    t.ex[c] = dg;
  }
  __syncthreads();
  for (int c = lane; c < m; c += blockDim.x) {
    const int jl = c / a, il = c - jl * a;
    double d = t.ex[c] + t.wE[c] + t.wN[c];
    if (il > 0) d += t.wE[c - 1];
    if (jl > 0) d += t.wN[c - a];
    t.sc[c] = scale ? rsqrt(d) : 1.0;
    t.Rr[c] = d;  // full diagonal, consumed below
  }
  __syncthreads();
  for (int e = lane; e < b * A; e += blockDim.x) {
    const int j = e / A, i = e - j * A;
    if (i < a) {
      const int c = j * a + i;
      t.dh[e] = to_T<T>(t.Rr[c] * t.sc[c] * t.sc[c]);
      t.eh[e] = i < a - 1 ? to_T<T>(-t.wE[c] * t.sc[c] * t.sc[c + 1]) : T(0);
      t.th[e] = j < b - 1 ? to_T<T>(t.wN[c] * t.sc[c] * t.sc[c + a]) : T(0);
    } else {
      t.dh[e] = T(1);
      t.eh[e] = T(0);
      t.th[e] = T(0);
    }
  }
  __syncthreads();
}

// Reciprocal of a pivot: FP32 uses the hardware approximation (<= 2 ulp), which the FP64
// refinement absorbs; FP64 the Newton-Raphson reciprocal of fp64_div.cuh (<= 1 ulp).
__device__ __forceinline__ float pivot_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double pivot_rcp(double x) { return rcp64(x); }

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

// Twisted block factorisation with two warps (warp 0 from the top, warp 1 from the
// bottom, meeting at block row mid = b/2):
//   top     S_0 = D_0,        S_j = D_j - t_{j-1} o Q_{j-1} o t_{j-1},  j < mid
//   bottom  S_{b-1} = D_{b-1}, S_j = D_j - t_j o Q_{j+1} o t_j,          j > mid
//   middle  S_mid = D_mid - t_{mid-1} o Q_{mid-1} o t_{mid-1} - t_mid o Q_{mid+1} o t_mid
// with Q_j = S_j^-1 written to Q ([b][A][A], padded).  The critical path is
// max(mid, b-1-mid) + 1 inversions instead of b.  Warps 0 and 1 work; any further warps of
// the CTA (blockDim.x a multiple of 64) only join the barriers.
template <typename T, int A>
__device__ void factor(const DevSub& sd, Tables<T> t, T* Q) {
  constexpr int NR = A * A / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = lane % A, h = lane / A;
  const int b = sd.b, mid = b / 2;
  T v[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) v[q] = T(0);
  // D_j entry (r, c) of the scaled operator (identity padding)
  auto dentry = [&](int j, int r) -> T {
    return r == c ? t.dh[j * A + r] : (c == r + 1 ? t.eh[j * A + r] : (r == c + 1 ? t.eh[j * A + c] : T(0)));
  };
  const int nsteps = warp == 0 ? mid : warp == 1 ? b - 1 - mid : 0;  // warps >= 2 idle here
  for (int k = 0; k < nsteps; ++k) {
    const int j = warp == 0 ? k : b - 1 - k;
    const int jc = warp == 0 ? j - 1 : j;  // coupling row to the previous block (top: j-1, bottom: j)
    const T tc = k > 0 ? t.th[jc * A + c] : T(0);
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const int r = h * NR + q;
      T s = dentry(j, r);
      if (k > 0) s -= t.th[jc * A + r] * v[q] * tc;
      v[q] = s;
    }
    gj_invert<T, A>(v, lane);
    T* Qj = Q + (size_t)j * A * A;
#pragma unroll
    for (int q = 0; q < NR; ++q) Qj[(h * NR + q) * A + c] = v[q];
  }
  __syncthreads();
  if (warp == 0) {
    const T* Qb = Q + (size_t)(mid + 1) * A * A;
    const T ta = mid > 0 ? t.th[(mid - 1) * A + c] : T(0);
    const T tb = mid < b - 1 ? t.th[mid * A + c] : T(0);
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const int r = h * NR + q;
      T s = dentry(mid, r);
      if (mid > 0) s -= t.th[(mid - 1) * A + r] * v[q] * ta;
      if (mid < b - 1) s -= t.th[mid * A + r] * Qb[r * A + c] * tb;
      v[q] = s;
    }
    gj_invert<T, A>(v, lane);
    T* Qm = Q + (size_t)mid * A * A;
#pragma unroll
    for (int q = 0; q < NR; ++q) Qm[(h * NR + q) * A + c] = v[q];
  }
  __syncthreads();
}

// The lane's part of an A x A block (column c = lane % A, rows (lane / A) NR + q): loaded into
// registers one block row ahead of its use, so that the load latency of the stored factor
// (shared or global memory) overlaps the previous product of the chain.
template <typename T, int A>
__device__ __forceinline__ void load_block(const T* Qj, T (&q)[A * A / 32], int lane) {
  constexpr int NR = A * A / 32;
  const int c = lane % A, h = lane / A;
#pragma unroll
  for (int k = 0; k < NR; ++k) q[k] = Qj[(h * NR + k) * A + c];
}

// y[c] = sum_r Q[r][c] x[r] for the lane's column c (Q symmetric), x held as x[lane % A], Q in
// the registers of load_block.
template <typename T, int A>
__device__ __forceinline__ T matvec_regs(const T (&q)[A * A / 32], T x, int lane) {
  constexpr int NR = A * A / 32;
  const int h = lane / A;
  T acc0 = T(0), acc1 = T(0);
#pragma unroll
  for (int k = 0; k < NR; k += 2) {
    const int r = h * NR + k;
    acc0 += q[k] * __shfl_sync(0xffffffffu, x, r);
    if (k + 1 < NR) acc1 += q[k + 1] * __shfl_sync(0xffffffffu, x, r + 1);
  }
  T acc = acc0 + acc1;
#pragma unroll
  for (int o = A; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

template <typename T, int A>
__device__ __forceinline__ T matvec(const T* Qj, T x, int lane) {
  T q[A * A / 32];
  load_block<T, A>(Qj, q, lane);
  return matvec_regs<T, A>(q, x, lane);
}

// Twisted solve (S A S) y = V in place (V, W: [b][A] padded, W workspace), two warps:
//   forward   W_j = Q_j (V_j + t_{j-1} o W_{j-1}) (top, j < mid),
//             W_j = Q_j (V_j + t_j o W_{j+1})     (bottom, j > mid),
//   middle    y_mid = Q_mid (V_mid + t_{mid-1} o W_{mid-1} + t_mid o W_{mid+1}),
//   backward  y_j = W_j + Q_j (t_j o y_{j+1}) (top),  y_j = W_j + Q_j (t_{j-1} o y_{j-1}) (bottom).
// Each chain prefetches the next block of its factor while it multiplies with the current one.
template <typename T, int A>
__device__ void solve(const DevSub& sd, Tables<T> t, const T* Q) {
  constexpr int NR = A * A / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = lane % A;
  const int b = sd.b, mid = b / 2;
  const int nsteps = warp == 0 ? mid : warp == 1 ? b - 1 - mid : 0;  // warps >= 2 idle here
  T qc[NR], qn[NR];
  T w = T(0);
  if (nsteps > 0) load_block<T, A>(Q + (size_t)(warp == 0 ? 0 : b - 1) * A * A, qc, lane);
  for (int k = 0; k < nsteps; ++k) {
    const int j = warp == 0 ? k : b - 1 - k;
    const int jc = warp == 0 ? j - 1 : j;
    if (k + 1 < nsteps) load_block<T, A>(Q + (size_t)(warp == 0 ? j + 1 : j - 1) * A * A, qn, lane);
    T u = t.V[j * A + c];
    if (k > 0) u += t.th[jc * A + c] * w;
    w = matvec_regs<T, A>(qc, u, lane);
    if (lane < A) t.W[j * A + c] = w;
#pragma unroll
    for (int q = 0; q < NR; ++q) qc[q] = qn[q];
  }
  __syncthreads();
  if (warp == 0) {
    T u = t.V[mid * A + c];
    if (mid > 0) u += t.th[(mid - 1) * A + c] * t.W[(mid - 1) * A + c];
    if (mid < b - 1) u += t.th[mid * A + c] * t.W[(mid + 1) * A + c];
    const T x = matvec<T, A>(Q + (size_t)mid * A * A, u, lane);
    if (lane < A) t.V[mid * A + c] = x;
  }
  __syncthreads();
  T x = warp < 2 ? t.V[mid * A + c] : T(0);
  if (nsteps > 0) load_block<T, A>(Q + (size_t)(warp == 0 ? mid - 1 : mid + 1) * A * A, qc, lane);
  for (int k = 0; k < nsteps; ++k) {
    const int j = warp == 0 ? mid - 1 - k : mid + 1 + k;
    const int jc = warp == 0 ? j : j - 1;  // coupling to the row solved before
    if (k + 1 < nsteps) load_block<T, A>(Q + (size_t)(warp == 0 ? j - 1 : j + 1) * A * A, qn, lane);
    x = t.W[j * A + c] + matvec_regs<T, A>(qc, t.th[jc * A + c] * x, lane);
    if (lane < A) t.V[j * A + c] = x;
#pragma unroll
    for (int q = 0; q < NR; ++q) qc[q] = qn[q];
  }
  __syncthreads();
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA, complete in thread 0 only (the other threads return their warp's sum).
// One barrier, which also orders every shared-memory write issued before the call ahead of
// every read after it; red (one double per warp) may be reused after the caller's next
// barrier.
__device__ __forceinline__ double cta_sum0(double v, double* red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v += red[w];
  return v;
}

// Maxima of non-negative doubles (+0, never -0) on their bit patterns (fp_bits.cuh): integer
// compares instead of float64 ones; a NaN propagates.
__device__ __forceinline__ unsigned long long warp_max_bits(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Max over the CTA of a non-negative value (red: one double of shared memory per warp).
__device__ __forceinline__ double cta_max(double v, double* red) {
  unsigned long long* ru = reinterpret_cast<unsigned long long*>(red);
  const unsigned long long u = warp_max_bits(nn_bits(v));
  if ((threadIdx.x & 31) == 0) ru[threadIdx.x >> 5] = u;
  __syncthreads();
  unsigned long long r = ru[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = ru[w] > r ? ru[w] : r;
  __syncthreads();
  return nn_from_bits(r);
}

// Max over the CTA of two non-negative values at once (one pair of barriers), as bit patterns.
__device__ __forceinline__ void cta_max2_bits(unsigned long long& v1, unsigned long long& v2, double* red) {
  unsigned long long* ru = reinterpret_cast<unsigned long long*>(red);
  v1 = warp_max_bits(v1);
  v2 = warp_max_bits(v2);
  const int nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    ru[threadIdx.x >> 5] = v1;
    ru[nw + (threadIdx.x >> 5)] = v2;
  }
  __syncthreads();
  unsigned long long r1 = ru[0], r2 = ru[nw];
  for (int w = 1; w < nw; ++w) {
    r1 = ru[w] > r1 ? ru[w] : r1;
    r2 = ru[nw + w] > r2 ? ru[nw + w] : r2;
  }
  __syncthreads();
  v1 = r1;
  v2 = r2;
}

// Max over the CTA of one non-negative value, as a bit pattern.
__device__ __forceinline__ unsigned long long cta_max_bits(unsigned long long v, double* red) {
  unsigned long long* ru = reinterpret_cast<unsigned long long*>(red);
  v = warp_max_bits(v);
  if ((threadIdx.x & 31) == 0) ru[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long r = ru[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = ru[w] > r ? ru[w] : r;
  __syncthreads();
  return r;
}

// Half of a non-negative double, on its bit pattern: the exponent field minus one for normal
// numbers from 2^-1021 up; a shift of the pattern (exact halving, truncated) below that.
__device__ __forceinline__ unsigned long long half_bits(unsigned long long u) {
  return (u >> 52) >= 2ull ? u - (1ull << 52) : u >> 1;
}

// East and north face fluxes of the iterate x, each face computed once: fE[c] = wE_c (x_c -
// x_east), fN[c] = wN_c (x_c - x_north), 0 on the subdomain's last column / row.  All threads
// of the CTA; a barrier must follow before apply_A reads them.
__device__ __forceinline__ void face_fluxes(const DevSub& sd, const double* wE, const double* wN, const double* x,
                                            double* fE, double* fN) {
  const int a = sd.a, b = sd.b, m = a * b;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    const int jl = c / a, il = c - jl * a;
    fE[c] = il < a - 1 ? wE[c] * (x[c] - x[c + 1]) : 0.0;
    fN[c] = jl < b - 1 ? wN[c] * (x[c] - x[c + a]) : 0.0;
  }
}

// (A x)_c in flux form (see k_local.cu) from the face fluxes of face_fluxes: ex_c x_c plus the
// cell's four outward face fluxes (the west and south ones are the neighbours' east / north
// fluxes negated, which is exact), summed in a fixed order; absx: the cell's flux scale.
__device__ __forceinline__ double apply_A(const DevSub& sd, const double* ex, const double* fE, const double* fN,
                                          const double* x, int c, double& absx) {
  const int a = sd.a;
  const int jl = c / a, il = c - jl * a;
  const double t0 = ex[c] * x[c], t1 = fE[c], t3 = fN[c];
  const double t2 = il > 0 ? -fE[c - 1] : 0.0, t4 = jl > 0 ? -fN[c - a] : 0.0;
  absx = fabs(t0) + fabs(t1) + fabs(t2) + fabs(t3) + fabs(t4);
  return (t0 + t1) + (t2 + t3) + t4;
}

__device__ __forceinline__ double apply_A(const DevSub& sd, const double* ex, const double* fE, const double* fN,
                                          const double* x, int c) {
  const int a = sd.a;
  const int jl = c / a, il = c - jl * a;
  const double t0 = ex[c] * x[c], t1 = fE[c], t3 = fN[c];
  const double t2 = il > 0 ? -fE[c - 1] : 0.0, t4 = jl > 0 ? -fN[c - a] : 0.0;
  return (t0 + t1) + (t2 + t3) + t4;
}

// Refined solve of A x = B (FP64, t.B) into t.X; same stopping rule as the CTA path with
// target = tol.  warm: start from the iterate already in t.X (otherwise from zero).  All
// threads of the CTA; red: two doubles of shared memory per warp.
template <typename T, int A>
__device__ void solve_refined(const DevSub& sd, Tables<T> t, const T* Q, bool refine, double tol, int ir_max,
                              int* status, int* ir_used, double* red, bool warm = false) {
  const double target = tol;
  const int a = sd.a, b = sd.b, m = a * b;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (warm) {  // t.X holds an initial iterate: start from its residual
    face_fluxes(sd, t.wE, t.wN, t.X, t.fE, t.fN);
    __syncthreads();
    for (int c = tid; c < m; c += nt) t.Rr[c] = t.B[c] - apply_A(sd, t.ex, t.fE, t.fN, t.X, c);
  } else {
    for (int c = tid; c < m; c += nt) {
      t.X[c] = 0.0;
      t.Rr[c] = t.B[c];
    }
  }
  __syncthreads();
  const int sweeps = refine ? ir_max : 1;
  int it = 0;
  bool ok = false;
  // The stopping rule on bit patterns of non-negative doubles (integer compares): rmax <=
  // tol * smax, or stagnation (rmax > rmax_prev / 2) with rmax <= 1e3 tol * smax.  Both
  // thresholds are fixed by the scale smax of the first iterate.
  unsigned long long thr_tol = 0, thr_floor = 0, half_prev = nn_bits(0.5e300);
  for (; it < sweeps; ++it) {
    for (int e = tid; e < b * A; e += nt) {
      const int j = e / A, i = e - j * A;
      // float64 factors are built unscaled (sc = 1): no multiplication by the scaling there
      if constexpr (kUnscaled<T>) t.V[e] = i < a ? t.Rr[j * a + i] : T(0);
      else t.V[e] = i < a ? to_T<T>(t.Rr[j * a + i] * t.sc[j * a + i]) : T(0);
    }
    __syncthreads();
    solve<T, A>(sd, t, Q);
    for (int c = tid; c < m; c += nt) {
      const int j = c / a, i = c - j * a;
      if constexpr (kUnscaled<T>) t.X[c] += t.V[j * A + i];
      else t.X[c] += from_T(t.V[j * A + i]) * t.sc[c];
    }
    __syncthreads();
    if (!refine) { it = 1; ok = true; break; }
    face_fluxes(sd, t.wE, t.wN, t.X, t.fE, t.fN);
    __syncthreads();
    unsigned long long rb = 0;  // max |r| as a bit pattern
    if (it == 0) {  // the scale max(|A||x| + |b|) is taken once, at the first iterate
      unsigned long long sb = 0;
      for (int c = tid; c < m; c += nt) {
        double absx;
        const double r = t.B[c] - apply_A(sd, t.ex, t.fE, t.fN, t.X, c, absx);
        t.Rr[c] = r;
        const unsigned long long ur = nn_bits(fabs(r)), us = nn_bits(absx + fabs(t.B[c]));
        rb = ur > rb ? ur : rb;
        sb = us > sb ? us : sb;
      }
      cta_max2_bits(rb, sb, red);
      const double smax = nn_from_bits(sb);
      thr_tol = nn_bits(target * smax);
      thr_floor = nn_bits(1e3 * tol * smax);
    } else {
      for (int c = tid; c < m; c += nt) {
        const double r = t.B[c] - apply_A(sd, t.ex, t.fE, t.fN, t.X, c);
        t.Rr[c] = r;
        const unsigned long long ur = nn_bits(fabs(r));
        rb = ur > rb ? ur : rb;
      }
      rb = cta_max_bits(rb, red);
    }
    if (rb <= thr_tol) { ok = true; ++it; break; }
    if (rb > half_prev && rb <= thr_floor) { ok = true; ++it; break; }  // FP64 floor reached
    half_prev = half_bits(rb);
  }
  if (tid == 0) {
    if (!ok) atomicOr(status, 1);
    atomicMax(ir_used, it);
  }
  __syncthreads();
}

}  // namespace warp
}  // namespace mpm
