// Interface (skeleton) system of the MRCM, Eq. (mrc2), FP64.
//
// Element matrices.  Subdomain i contributes, for every test function on one of its
// interface sides (psi for the flux balance, phi for the Robin-weighted pressure
// continuity, the latter multiplied by -1 so that the assembled matrix is symmetric),
//   psi_k rows:  sum_e psi_k(e) F_e
//   phi_k rows: -sum_e bh_e s phi_k(e) F_e + sum_e bh_e phi_k(e) U_e,   bh_e = rho / kappa_c,
// with F_e = Fbar_e + sum_l c_l Fhat_e,l (traces of the BFs) and U_e = sum_l c_l phi_l(e).
// The global matrix is the sum of these element matrices (each interface is shared by two
// subdomains), like a finite-element assembly with subdomains as elements and interfaces
// as nodes.
//
// Factorisation: nested dissection over the subdomain grid (recursive bisection; the
// separator of a node is the line of interfaces between its two halves).  Each node's
// frontal matrix (separator DOFs first, then boundary DOFs) is the extend-add of its
// children's Schur complements; the separator pivots are eliminated by a blocked
// Gauss-Jordan sweep, which leaves
//   [ F_ss^-1          F_ss^-1 F_sb            ]
//   [ -F_bs F_ss^-1    F_bb - F_bs F_ss^-1 F_sb ]   (Schur complement -> parent)
// in place.  The frontal matrices are stored transposed (the sweep then produces the
// transposes of these blocks), so that the solve reads them along rows.  With the flux rows negated the system is symmetric quasi-definite
// (Robin-weighted U block positive definite, P block negative definite when a Dirichlet
// side exists), so the sweep needs no pivoting.
// Solve: upward  y_s = F_ss^-1 g_s, g_b += (-F_bs F_ss^-1) g_s  (g_b -> parent);
//        downward x_s = y_s - (F_ss^-1 F_sb) x_b  (x_b from the parent).
#include <algorithm>

#include "k_iface_phases.cuh"
#include "k_local_warp.cuh"
#include "mpm2p_internal.cuh"

namespace mpm {

namespace {

constexpr int kTile = 32;

using phase::dof_info;
using phase::side_basis;

__device__ __forceinline__ int side_len(const DevSub& sd, int side) { return side < 2 ? sd.b : sd.a; }

__global__ void k_element_matrix(Grid g, DevState d, const DevSub* subs, const DevNode* nodes,
                                 const int* leaf_node) {
  const int r = blockIdx.y;
  if (d.rebuild[r] != 1) return;
  const int sidx = blockIdx.x;
  __shared__ DevSub sd_s;  // the subdomain record, staged once per CTA (indexed by side)
  if (threadIdx.x == 0) sd_s = subs[sidx];
  __syncthreads();
  const DevSub& sd = sd_s;
  const int nd = sd.ndof;
  if (nd == 0) return;
  const DevNode leaf = nodes[leaf_node[sidx]];
  double* E = d.front + (long long)r * d.st_front + leaf.f_off;
  const double* tr = d.tr + (long long)r * d.st_tr + sd.tr_off;  // [nd][nface]
  const double* bhat = d.bhat + (long long)r * d.st_face + sd.face_off;
  const int nface = 2 * (sd.a + sd.b);
  for (int e = threadIdx.x; e < nd * nd; e += blockDim.x) {
    const int k = e / nd, l = e - k * nd;
    int side, isP, kk;
    dof_info(sd, k, side, isP, kk);
    int lside, lisP, ll;
    dof_info(sd, l, lside, lisP, ll);
    const int L = side_len(sd, side);
    const int f0 = face_side_off(side, sd.a, sd.b);
    const double s = sd.side_sign[side];
    double v = 0.0;
    for (int t = 0; t < L; ++t) {
      const double w = side_basis(kk, t, g.seg_len, g.degree, g.inv_seg);
      if (w == 0.0) continue;
      const double F = tr[(long long)l * nface + f0 + t];
      if (isP) {
        v += w * F;
      } else {
        const double bh = bhat[f0 + t];
        v -= bh * s * w * F;
        if (!lisP && lside == side) v += bh * w * side_basis(ll, t, g.seg_len, g.degree, g.inv_seg);
      }
    }
    E[(long long)l * nd + k] = v;  // stored transposed (see the per-level solve kernels)
  }
}

// Frontal matrix of an internal node: extend-add of the children's Schur complements.
__global__ void k_nd_assemble(Grid g, DevState d, const DevNode* nodes, const int* level_nodes,
                              const int* srcmap) {
  const int r = blockIdx.z;
  if (d.rebuild[r] != 1) return;
  const DevNode nd = nodes[level_nodes[blockIdx.x]];
  const int nf = nd.nf;
  const long long total = (long long)nf * nf;
  const long long start = (long long)blockIdx.y * blockDim.x * 8;
  if (start >= total) return;
  double* F = d.front + (long long)r * d.st_front + nd.f_off;  // transposed storage, mapped entry by entry
  const int* s0 = srcmap + nd.src_off;
  const int* s1 = s0 + nf;
  const DevNode c0 = nodes[nd.child[0]], c1 = nodes[nd.child[1]];
  const double* C0 = d.front + (long long)r * d.st_front + c0.f_off;
  const double* C1 = d.front + (long long)r * d.st_front + c1.f_off;
  for (long long e = start + threadIdx.x; e < total && e < start + (long long)blockDim.x * 8; e += blockDim.x) {
    const int i = (int)(e / nf), j = (int)(e - (long long)i * nf);
    double v = 0.0;
    const int a0 = s0[i], b0 = s0[j];
    if (a0 >= 0 && b0 >= 0) v += C0[(long long)(c0.nsep + a0) * c0.nf + c0.nsep + b0];
    const int a1 = s1[i], b1 = s1[j];
    if (a1 >= 0 && b1 >= 0) v += C1[(long long)(c1.nsep + a1) * c1.nf + c1.nsep + b1];
    F[e] = v;
  }
}

// The factorisation of one level runs, for every pivot chunk P = [k0, k0 + nb) (nb <= 16),
// two launches: k_sweep_rowcol (pivot rows and columns) and k_sweep_trailing (the rest).  The
// inverse of the chunk's pivot block is ready before k_sweep_rowcol: the first chunk's from
// k_sweep_pivot0, every later chunk's from the k_sweep_trailing launch of the chunk before,
// whose diagonal tile holding that block finishes it and inverts it at once.  The inverse is
// written into the front (where the solve reads it) and to pivinv (read by k_sweep_rowcol).

// One warp inverts the pivot block [k1, k1 + nb) of a front in registers (Gauss-Jordan, the
// block padded with the identity to 16 x 16), src(i, k) giving its entries.
template <typename Src>
__device__ __forceinline__ void invert_pivot(Src src, double* F, int nf, int k1, int nb, double* pv, int lane) {
  constexpr int A = kPivotChunk, NR = A * A / 32;
  const int c = lane % A, h = lane / A;
  double v[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    const int i = h * NR + q;
    v[q] = (i < nb && c < nb) ? src(i, c) : (i == c ? 1.0 : 0.0);
  }
  warp::gj_invert<double, A>(v, lane);
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    const int i = h * NR + q;
    if (i < nb && c < nb) F[(long long)(k1 + i) * nf + k1 + c] = v[q];
    pv[i * A + c] = v[q];
  }
}

// Inverse of the first pivot block of every front of a level (one warp per front).
__global__ void __launch_bounds__(32) k_sweep_pivot0(Grid g, DevState d, const DevNode* nodes, const int* level_nodes) {
  const int r = blockIdx.y;
  if (d.rebuild[r] != 1) return;
  const DevNode nd = nodes[level_nodes[blockIdx.x]];
  if (nd.nsep <= 0) return;
  const int nf = nd.nf;
  double* F = d.front + (long long)r * d.st_front + nd.f_off;
  double* pv = d.pivinv + ((long long)r * d.st_lvl + blockIdx.x) * kPivotChunk * kPivotChunk;
  invert_pivot([&](int i, int k) { return F[(long long)i * nf + k]; }, F, nf, 0, min(kPivotChunk, nd.nsep), pv,
               threadIdx.x);
}

constexpr int kRcIdx = 32;  // front indices per CTA of k_sweep_rowcol

// Pivot rows and columns of chunk P for every index c outside P:  M_Pc <- Pinv M_Pc  and
// M_cP <- -M_cP Pinv, the old M_cP saved to colold for k_sweep_trailing.  The symmetric
// pattern of the partial inverse (see k_sweep_trailing) gives the column from the row:
// before the step M_cP = s M_Pc^T with s = +1 for c not yet eliminated (c >= k0 + nb) and
// s = -1 for c < k0, so with Pinv symmetric the new column is -s (Pinv M_Pc)^T and the old
// one s M_Pc^T: one product of Pinv with the CTA's 16 x 32 slab of pivot rows, staged in
// shared memory.  The pivot rows are read and written along rows (coalesced), the columns
// 16 consecutive entries per index.
__global__ void __launch_bounds__(256) k_sweep_rowcol(Grid g, DevState d, const DevNode* nodes,
                                                       const int* level_nodes, int k0) {
  __shared__ double P[kPivotChunk][kPivotChunk + 1];
  __shared__ double S[kPivotChunk][kRcIdx + 1];  // old pivot rows of the CTA's indices
  __shared__ double Y[kPivotChunk][kRcIdx + 1];  // new pivot rows
  const int r = blockIdx.z;
  if (d.rebuild[r] != 1) return;
  const DevNode nd = nodes[level_nodes[blockIdx.x]];
  if (k0 >= nd.nsep) return;
  const int nb = min(kPivotChunk, nd.nsep - k0);
  const int nf = nd.nf;
  const int i0 = blockIdx.y * kRcIdx;
  if (i0 >= nf) return;
  const int tid = threadIdx.x;
  const double* Pg = d.pivinv + ((long long)r * d.st_lvl + blockIdx.x) * kPivotChunk * kPivotChunk;
  double* F = d.front + (long long)r * d.st_front + nd.f_off;
  for (int e = tid; e < kPivotChunk * kPivotChunk; e += blockDim.x) P[e / kPivotChunk][e % kPivotChunk] = Pg[e];
  for (int e = tid; e < kPivotChunk * kRcIdx; e += blockDim.x) {
    const int l = e / kRcIdx, j = e - l * kRcIdx, idx = i0 + j;
    S[l][j] = (l < nb && idx < nf) ? F[(long long)(k0 + l) * nf + idx] : 0.0;
  }
  __syncthreads();
  auto outside = [&](int idx) { return idx < nf && !(idx >= k0 && idx < k0 + nb); };
  for (int e = tid; e < kPivotChunk * kRcIdx; e += blockDim.x) {
    const int l = e / kRcIdx, j = e - l * kRcIdx, idx = i0 + j;
    if (l >= nb || !outside(idx)) continue;
    double a = 0.0;
#pragma unroll
    for (int q = 0; q < kPivotChunk; ++q) a += P[l][q] * S[q][j];  // S is 0 past nb
    Y[l][j] = a;
    F[(long long)(k0 + l) * nf + idx] = a;
  }
  __syncthreads();
  double* Cold = d.colold + (long long)r * d.st_col + (long long)nd.v_off * kPivotChunk;
  for (int e = tid; e < kPivotChunk * kRcIdx; e += blockDim.x) {
    const int j = e / kPivotChunk, l = e - j * kPivotChunk, idx = i0 + j;
    if (!outside(idx)) continue;
    // sign flips on the bit pattern (no float64 instruction): s = -1 below k0
    const unsigned long long sflip = idx < k0 ? 0x8000000000000000ull : 0ull;
    if (l < nb)
      F[(long long)idx * nf + k0 + l] =
          __longlong_as_double(__double_as_longlong(Y[l][j]) ^ sflip ^ 0x8000000000000000ull);
    Cold[(long long)idx * kPivotChunk + l] = l < nb ? __longlong_as_double(__double_as_longlong(S[l][j]) ^ sflip) : 0.0;
  }
}

// Trailing update of chunk P:  M_rc -= Mold_rP M_Pc(new)  for r, c outside P.
// The frontal matrices are symmetric, and Gauss-Jordan elimination keeps a fixed pattern:
// with E the pivots eliminated so far and R the rest, M_EE and M_RR stay symmetric and
// M_ER = -M_RE^T (the partial inverse [A^-1, A^-1 B; -B^T A^-1, C - B^T A^-1 B]).  So only the
// tiles on and above the diagonal are computed (blockIdx.y enumerates the pairs ty <= tx); an
// off-diagonal tile also writes its mirror, negated where exactly one of row and column lies in
// E, i.e. below k0 (through shared memory, so that both writes are coalesced).  This halves the
// float64 work of the factorisation.  The diagonal tile that holds the next chunk's pivot
// block (final once this update is done) also inverts it (invert_pivot).
__global__ void k_sweep_trailing(Grid g, DevState d, const DevNode* nodes, const int* level_nodes, int k0,
                                 int tiles_x) {
  __shared__ double A[kTile][kPivotChunk + 1];
  __shared__ double B[kPivotChunk][kTile + 1];
  __shared__ double Tn[kTile][kTile + 1];
  const int r = blockIdx.z;
  if (d.rebuild[r] != 1) return;
  const DevNode nd = nodes[level_nodes[blockIdx.x]];
  if (k0 >= nd.nsep) return;
  const int nb = min(kPivotChunk, nd.nsep - k0);
  const int nf = nd.nf;
  int ty = 0, rem = blockIdx.y;  // (ty, tx) from the upper-triangle index
  while (rem >= tiles_x - ty) {
    rem -= tiles_x - ty;
    ++ty;
  }
  const int tx = ty + rem;
  const int r0 = ty * kTile, c0 = tx * kTile;
  if (r0 >= nf || c0 >= nf) return;
  double* F = d.front + (long long)r * d.st_front + nd.f_off;
  const double* Cold = d.colold + (long long)r * d.st_col + (long long)nd.v_off * kPivotChunk;
  for (int e = threadIdx.x; e < kTile * kPivotChunk; e += blockDim.x) {
    const int i = e / kPivotChunk, l = e - i * kPivotChunk;
    const int row = r0 + i;
    A[i][l] = (row < nf && l < nb && !(row >= k0 && row < k0 + nb)) ? Cold[(long long)row * kPivotChunk + l] : 0.0;
    const int l2 = e / kTile, j = e - l2 * kTile;
    const int colx = c0 + j;
    B[l2][j] = (colx < nf && l2 < nb && !(colx >= k0 && colx < k0 + nb)) ? F[(long long)(k0 + l2) * nf + colx] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
    const int i = e / kTile, j = e - i * kTile;
    const int row = r0 + i, colx = c0 + j;
    if (row >= nf || colx >= nf) continue;
    if ((row >= k0 && row < k0 + nb) || (colx >= k0 && colx < k0 + nb)) continue;
    double acc = 0.0;
#pragma unroll
    for (int l = 0; l < kPivotChunk; ++l) acc += A[i][l] * B[l][j];
    const double v = F[(long long)row * nf + colx] - acc;
    F[(long long)row * nf + colx] = v;
    Tn[i][j] = ((row < k0) == (colx < k0)) ? v : -v;
  }
  if (tx == ty) {
    const int k1 = k0 + kPivotChunk;  // the next chunk: its pivot block lies inside tile k1 / kTile
    if (k1 < nd.nsep && ty == k1 / kTile) {
      __syncthreads();  // the tile's values complete, its writes to F ordered before the inverse's
      if (threadIdx.x < 32) {
        const int o = k1 - r0;
        double* pv = d.pivinv + ((long long)r * d.st_lvl + blockIdx.x) * kPivotChunk * kPivotChunk;
        invert_pivot([&](int i, int k) { return Tn[o + i][o + k]; }, F, nf, k1, min(kPivotChunk, nd.nsep - k1), pv,
                     threadIdx.x);
      }
    }
    return;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
    const int j = e / kTile, i = e - j * kTile;  // consecutive threads: consecutive columns of row c0 + j
    const int row = r0 + i, colx = c0 + j;
    if (row >= nf || colx >= nf) continue;
    if ((row >= k0 && row < k0 + nb) || (colx >= k0 && colx < k0 + nb)) continue;
    F[(long long)colx * nf + row] = Tn[i][j];
  }
}

// Per-level solve kernels.  Every frontal matrix is stored transposed, G = F^T (the element
// matrices are written transposed and the extend-add maps entries index by index), and the
// sweep runs on G, which leaves
//   [ G_ss^-1 = (F_ss^-1)^T         G_ss^-1 G_sb = (F_bs F_ss^-1)^T      ]
//   [ -G_bs G_ss^-1 = -(F_ss^-1 F_sb)^T   S_G = (F_bb - F_bs F_ss^-1 F_sb)^T ]
// so the solve with F reads G along its rows: output r is a sum over k of G[k][r] (up) or
// G[ns + k][r] (down).  Consecutive threads take consecutive r, so every load is coalesced
// and no cross-lane reduction is needed (float64 instructions are scarce on this part).  KS
// threads share a row, each summing every KS-th k (its first kKpt terms held in registers,
// loaded before pdl_wait()), and combine in shared memory.
constexpr int kKpt = 16;

// Upward solve at one level: y_s = F_ss^-1 g_s, y_s[r] = sum_k G[k][r] g_s[k] (r < ns, into
// x), and g_b += -F_bs F_ss^-1 g_s, g_b[r] = gather(r) - sum_k G[k][r] g_s[k] (r >= ns), with
// g gathered from the children.
template <int KS>
__global__ void __launch_bounds__(256) k_nd_up(Grid g, DevState d, const DevNode* nodes, const int* level_nodes,
                                               const int* srcmap, int branch) {
  constexpr int ROWS = 256 / KS;
  extern __shared__ __align__(16) double nd_smem[];
  pdl_trigger();
  const int r = blockIdx.z;
  if (branch >= 0 && d.rebuild[r] != branch) return;  // branch >= 0: only the realisations that took it
  const DevNode nd = nodes[level_nodes[blockIdx.x]];
  const int row0 = blockIdx.y * ROWS;
  if (row0 >= nd.nf) return;
  const int nf = nd.nf, ns = nd.nsep;
  double* part = nd_smem;                            // [KS][ROWS]
  double* gs = nd_smem + KS * ROWS;                  // ns
  const int i = threadIdx.x % ROWS, q = threadIdx.x / ROWS;
  const int row = row0 + i;
  const long long vb = (long long)r * d.st_vec;
  const int* s0 = srcmap + nd.src_off;
  const int* s1 = s0 + nf;
  const DevNode& c0 = nodes[nd.child[0]];
  const DevNode& c1 = nodes[nd.child[1]];
  const double* g0 = d.gvec + vb + c0.v_off + c0.nsep;
  const double* g1 = d.gvec + vb + c1.v_off + c1.nsep;
  int own0 = -1, own1 = -1;
  if (q == 0 && row < nf && row >= ns) {
    own0 = s0[row];
    own1 = s1[row];
  }
  // this thread's first kKpt terms G[q + u KS][row]: operator data, loaded before the wait
  const double* F = d.front + (long long)r * d.st_front + nd.f_off;
  double v[kKpt];
#pragma unroll
  for (int u = 0; u < kKpt; ++u) {
    const int k = q + u * KS;
    v[u] = (row < nf && k < ns) ? F[(long long)k * nf + row] : 0.0;
  }
  // gather indices of the first separator entry of this thread (index maps are static)
  const int p0 = threadIdx.x < ns ? s0[threadIdx.x] : -1, p1 = threadIdx.x < ns ? s1[threadIdx.x] : -1;
  pdl_wait();
  for (int k = threadIdx.x; k < ns; k += blockDim.x) {
    const bool first = k == (int)threadIdx.x;
    const int a0 = first ? p0 : s0[k], a1 = first ? p1 : s1[k];
    gs[k] = (a0 >= 0 ? g0[a0] : 0.0) + (a1 >= 0 ? g1[a1] : 0.0);
  }
  __syncthreads();
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int u = 0; u < kKpt; ++u) {
    const int k = q + u * KS;
    if (k < ns) acc[u & 3] += v[u] * gs[k];
  }
  if (row < nf)
    for (int k = q + kKpt * KS; k < ns; k += KS) acc[0] += F[(long long)k * nf + row] * gs[k];
  part[q * ROWS + i] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  __syncthreads();
  if (q == 0 && row < nf) {
    double sum = part[i];
#pragma unroll
    for (int u = 1; u < KS; ++u) sum += part[u * ROWS + i];
    if (row < ns) d.xvec[vb + nd.v_off + row] = sum;
    else d.gvec[vb + nd.v_off + row] = ((own0 >= 0 ? g0[own0] : 0.0) + (own1 >= 0 ? g1[own1] : 0.0)) - sum;
  }
}

// Downward solve at one level: x_s = y_s - F_ss^-1 F_sb x_b,
// x_s[r] = y_s[r] + sum_k G[ns + k][r] x_b[k], with x_b gathered
// from the parent's x; the CTA of row block 0 also stores x_b in the node's own vector for
// its children.  Leaves are not visited: the reconstruction gathers their x from the parent.
template <int KS>
__global__ void __launch_bounds__(256) k_nd_down(Grid g, DevState d, const DevNode* nodes, const int* level_nodes,
                                                 const int* pmap) {
  constexpr int ROWS = 256 / KS;
  extern __shared__ __align__(16) double nd_smem[];
  pdl_trigger();
  const int r = blockIdx.z;
  const DevNode nd = nodes[level_nodes[blockIdx.x]];
  if (nd.parent < 0) return;
  const int nf = nd.nf, ns = nd.nsep, nbd = nd.nbnd;
  const int row0 = blockIdx.y * ROWS;
  if (row0 >= ns && blockIdx.y != 0) return;
  double* part = nd_smem;                            // [KS][ROWS]
  double* xb = nd_smem + KS * ROWS;                  // nbd
  const int i = threadIdx.x % ROWS, q = threadIdx.x / ROWS;
  const int row = row0 + i;
  const long long vb = (long long)r * d.st_vec;
  const int* pm = pmap + nd.pmap_off;
  const double* xp = d.xvec + vb + nodes[nd.parent].v_off;
  double* xo = d.xvec + vb + nd.v_off;
  const double* F = d.front + (long long)r * d.st_front + nd.f_off + (long long)ns * nf;
  double v[kKpt];
#pragma unroll
  for (int u = 0; u < kKpt; ++u) {
    const int k = q + u * KS;
    v[u] = (row < ns && k < nbd) ? F[(long long)k * nf + row] : 0.0;
  }
  const int p0 = threadIdx.x < nbd ? pm[threadIdx.x] : 0;  // static index map, loaded before the wait
  pdl_wait();
  for (int k = threadIdx.x; k < nbd; k += blockDim.x) {
    const double x = xp[k == (int)threadIdx.x ? p0 : pm[k]];
    xb[k] = x;
    if (blockIdx.y == 0) xo[ns + k] = x;
  }
  __syncthreads();
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int u = 0; u < kKpt; ++u) {
    const int k = q + u * KS;
    if (k < nbd) acc[u & 3] += v[u] * xb[k];
  }
  if (row < ns)
    for (int k = q + kKpt * KS; k < nbd; k += KS) acc[0] += F[(long long)k * nf + row] * xb[k];
  part[q * ROWS + i] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  __syncthreads();
  if (q == 0 && row < ns) {
    double sum = part[i];
#pragma unroll
    for (int u = 1; u < KS; ++u) sum += part[u * ROWS + i];
    xo[row] += sum;
  }
}

// Reconstruction from the interface solution c of one subdomain per CTA: the one-sided
// traces F = Fbar + F_hat c, then the target mean of the downscaled pressure, and at a
// rebuild the MRCM-level pressure p^m = pbar + P_hat c:
//   rebuild: target = mean(p^m);  MPM-2P: target = mean(p^m) + mean(dpbar) + mu_hat . dc.
// c is gathered from the leaf's parent P.  When P is a level-1 node (two leaf children) its
// downward step is done here, redundantly by both children, instead of by a sweep kernel:
// x_P = [y_s + sum_k G[ns + k][r] x_b[k] ; x_b], x_b from P's parent.
// F_hat and P_hat are stored one column per BF, so thread (face f, chunk q) sums F_hat[l][f]
// c[l] over l = q, q + KS, ... with coalesced loads (its first kKpt terms loaded before
// pdl_wait()), and the KS chunks combine in shared memory.  branch >= 0 restricts the launch
// to the realisations that took that branch.
constexpr int kKpt1 = 8;  // register-held terms per thread of the fused level-1 step

template <int KS>
__global__ void __launch_bounds__(256) k_reconstruct(Grid g, DevState d, const DevSub* subs, const DevNode* nodes,
                                                     const int* leaf_node, const int* pmap, int branch, int pass) {
  constexpr int FACES = 256 / KS;
  extern __shared__ __align__(16) double nd_smem[];
  __shared__ double red[32];
  pdl_trigger();
  const int sidx = blockIdx.x, r = blockIdx.y;
  const int br = d.rebuild[r];
  if (branch >= 0 && br != branch) return;
  const DevSub& sd = subs[sidx];
  const int a = sd.a, b = sd.b, m = a * b, nd = sd.ndof, nface = 2 * (a + b);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double* part = nd_smem;                            // [KS][FACES], then the level-1 partial sums
  double* cs = nd_smem + 256;                        // nd
  double* xP = cs + nd;                              // the parent's frontal solution (fused case)
  const int f = threadIdx.x % FACES, q = threadIdx.x / FACES;
  const long long vb = (long long)r * d.st_vec;
  const double* trb = d.tr + (long long)r * d.st_tr + sd.tr_off;
  double v[kKpt];
#pragma unroll
  for (int u = 0; u < kKpt; ++u) {
    const int l = q + u * KS;
    v[u] = (f < nface && l < nd) ? trb[(long long)l * nface + f] : 0.0;
  }
  const double fbar = f < nface && q == 0 ? d.fbar[(long long)r * d.st_face + sd.face_off + f] : 0.0;
  const int* pm = nullptr;
  int p0 = 0;
  bool fused = false;
  DevNode P{};
  // fused level-1 step: thread (row i1, chunk q1) of P's separator rows; its first terms
  // G[ns + k][i1] and P's boundary index map are operator data, loaded before the wait
  int rows1 = 1, i1 = 0, q1 = 0, pp0 = 0;
  double v1[kKpt1];
  if (nd > 0) {
    const DevNode& leaf = nodes[leaf_node[sidx]];
    P = nodes[leaf.parent];
    pm = pmap + leaf.pmap_off;
    if ((int)threadIdx.x < nd) p0 = pm[threadIdx.x];
    fused = P.level == 1;
    if (fused) {
      while (rows1 < P.nsep) rows1 <<= 1;
      const int kc = 256 / rows1;
      i1 = threadIdx.x % rows1;
      q1 = threadIdx.x / rows1;
      const double* G = d.front + (long long)r * d.st_front + P.f_off + (long long)P.nsep * P.nf;
#pragma unroll
      for (int u = 0; u < kKpt1; ++u) {
        const int k = q1 + u * kc;
        v1[u] = (i1 < P.nsep && k < P.nbnd) ? G[(long long)k * P.nf + i1] : 0.0;
      }
      if (P.parent >= 0 && (int)threadIdx.x < P.nbnd) pp0 = pmap[P.pmap_off + threadIdx.x];
    }
  }
  pdl_wait();
  if (fused) {
    const int kc = 256 / rows1;
    const double* xpp = P.parent >= 0 ? d.xvec + vb + nodes[P.parent].v_off : nullptr;
    for (int k = threadIdx.x; k < P.nbnd; k += blockDim.x)
      xP[P.nsep + k] = xpp[k == (int)threadIdx.x ? pp0 : pmap[P.pmap_off + k]];
    __syncthreads();
    const double* G = d.front + (long long)r * d.st_front + P.f_off + (long long)P.nsep * P.nf;
    double a1[2] = {0.0, 0.0};
#pragma unroll
    for (int u = 0; u < kKpt1; ++u) {
      const int k = q1 + u * kc;
      if (k < P.nbnd) a1[u & 1] += v1[u] * xP[P.nsep + k];
    }
    if (i1 < P.nsep)
      for (int k = q1 + kKpt1 * kc; k < P.nbnd; k += kc) a1[0] += G[(long long)k * P.nf + i1] * xP[P.nsep + k];
    part[q1 * rows1 + i1] = a1[0] + a1[1];
    __syncthreads();
    if (q1 == 0 && i1 < P.nsep) {
      double sum = d.xvec[vb + P.v_off + i1];  // y_s of the upward sweep
      for (int u = 0; u < kc; ++u) sum += part[u * rows1 + i1];
      xP[i1] = sum;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < nd; l += blockDim.x) cs[l] = xP[l == (int)threadIdx.x ? p0 : pm[l]];
  } else if (nd > 0) {
    const double* xp = d.xvec + vb + P.v_off;
    for (int l = threadIdx.x; l < nd; l += blockDim.x) cs[l] = xp[l == (int)threadIdx.x ? p0 : pm[l]];
  }
  __syncthreads();
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int u = 0; u < kKpt; ++u) {
    const int l = q + u * KS;
    if (l < nd) acc[u & 3] += v[u] * cs[l];
  }
  if (f < nface)
    for (int l = q + kKpt * KS; l < nd; l += KS) acc[0] += trb[(long long)l * nface + f] * cs[l];
  part[q * FACES + f] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  __syncthreads();
  if (q == 0 && f < nface) {
    double sum = part[f];
#pragma unroll
    for (int u = 1; u < KS; ++u) sum += part[u * FACES + f];
    (pass == 0 ? d.trace : d.trace1)[(long long)r * d.st_face + sd.face_off + f] = fbar + sum;
  }
  double pt = 0.0;
  if (br == 0 && pass == 0 && g.order >= 1) {
    // first-order MPM-2P: the MRCM-level pressure of the epsilon^0 solve, dp0 = dpbar + P_hat c
    // (dpbar stored in dp0 by the local solve), the source of the first-order problem
    const double* pf = d.pf + (long long)r * d.st_pf + sd.pf_off;
    double* x = d.dp0 + (long long)r * g.ncell();
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
      const int jl = c / a, il = c - jl * a;
      const long long gc = (long long)(sd.y0 + jl) * g.nx + sd.x0 + il;
      double pv = x[gc];
      for (int l = 0; l < nd; ++l) pv += pf[(long long)l * m + c] * cs[l];
      x[gc] = pv;
    }
  }
  if (br == 1) {
    const double* pf = d.pf + (long long)r * d.st_pf + sd.pf_off;  // [nd + 1][m]
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
      double pv = pf[(long long)nd * m + c];
      for (int l = 0; l < nd; ++l) pv += pf[(long long)l * m + c] * cs[l];
      const int jl = c / a, il = c - jl * a;
      d.p_m[(long long)r * g.ncell() + (long long)(sd.y0 + jl) * g.nx + sd.x0 + il] = pv;
      pt += pv;
    }
  } else {
    const double* muh = d.mu_hat + (long long)r * d.st_dof + sd.dof_off;
    for (int l = threadIdx.x; l < nd; l += blockDim.x) pt += muh[l] * cs[l];
    pt *= m;
  }
  pt = phase::warp_sum(pt);
  if (lane == 0) red[warp] = pt;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    const long long si = (long long)r * d.st_sub + sidx;
    if (br == 1) {
      d.pm_mean[si] = s / m;
      d.sub_target[si] = s / m;
    } else if (pass == 0) {
      d.sub_target[si] = d.pm_mean[si] + (d.sub_mean[si] * m + s) / m;
    } else {  // the first-order term adds its own mean
      d.sub_target[si] += (d.sub_mean[si] * m + s) / m;
    }
  }
}

}  // namespace

void launch_element_matrix(const Grid& g, const DevState& d, const DevSub* subs, int nsub, const DevNode* nodes,
                           const int* leaf_node, cudaStream_t st) {
  k_element_matrix<<<dim3(nsub, g.R), 256, 0, st>>>(g, d, subs, nodes, leaf_node);
  ++g_launches;
}

void launch_nd_factor_level(const Grid& g, const DevState& d, const DevNode* nodes, const int* level_nodes,
                            int nlev, int max_nf, int max_nsep, const int* srcmap, cudaStream_t st) {
  const int thr = 256;
  const long long per = (long long)thr * 8;
  const int ablk = (int)(((long long)max_nf * max_nf + per - 1) / per);
  k_nd_assemble<<<dim3(nlev, ablk, g.R), thr, 0, st>>>(g, d, nodes, level_nodes, srcmap);
  ++g_launches;
  const int tiles_x = (max_nf + kTile - 1) / kTile;
  k_sweep_pivot0<<<dim3(nlev, g.R), 32, 0, st>>>(g, d, nodes, level_nodes);
  ++g_launches;
  for (int k0 = 0; k0 < max_nsep; k0 += kPivotChunk) {
    k_sweep_rowcol<<<dim3(nlev, (max_nf + kRcIdx - 1) / kRcIdx, g.R), 256, 0, st>>>(g, d, nodes, level_nodes, k0);
    ++g_launches;
    k_sweep_trailing<<<dim3(nlev, tiles_x * (tiles_x + 1) / 2, g.R), 256, 0, st>>>(g, d, nodes, level_nodes, k0,
                                                                                  tiles_x);
    ++g_launches;
  }
}

namespace {
// k-chunks per output row: each thread sums about `terms` of the n terms, with at most 16
// chunks (more chunks mean fewer rows per CTA and more CTAs, but a longer serial combination of
// the partial sums: 32 and 64 chunks were measured slower on the 1024^2 workload).
int k_split(int n, int terms) {
  const int q = (n + terms - 1) / terms;
  return q <= 1 ? 1 : q <= 2 ? 2 : q <= 4 ? 4 : q <= 8 ? 8 : 16;
}
}  // namespace

#define MPM_DISPATCH_KS(KERNEL, ks, ...)                        \
  do {                                                          \
    switch (ks) {                                               \
      case 1: launch_ex(KERNEL<1>, __VA_ARGS__); break;         \
      case 2: launch_ex(KERNEL<2>, __VA_ARGS__); break;         \
      case 4: launch_ex(KERNEL<4>, __VA_ARGS__); break;         \
      case 8: launch_ex(KERNEL<8>, __VA_ARGS__); break;         \
      default: launch_ex(KERNEL<16>, __VA_ARGS__); break;       \
    }                                                           \
  } while (0)

void launch_nd_up(const Grid& g, const DevState& d, const DevNode* nodes, const int* level_nodes, int nlev,
                  int max_nf, int max_nsep, const int* srcmap, bool pdl, int terms, cudaStream_t st, int branch) {
  const int ks = k_split(max_nsep, terms), rows = 256 / ks;
  const dim3 grid(nlev, (max_nf + rows - 1) / rows, g.R);
  const size_t smem = (size_t)(256 + max_nsep) * sizeof(double);
  MPM_DISPATCH_KS(k_nd_up, ks, grid, dim3(256), smem, st, pdl, g, d, nodes, level_nodes, srcmap, branch);
}

void launch_nd_down(const Grid& g, const DevState& d, const DevNode* nodes, const int* level_nodes, int nlev,
                    int max_nsep, int max_nbnd, const int* pmap, bool pdl, int terms, cudaStream_t st) {
  const int ks = k_split(max_nbnd, terms), rows = 256 / ks;
  const dim3 grid(nlev, max_nsep > 0 ? (max_nsep + rows - 1) / rows : 1, g.R);
  const size_t smem = (size_t)(256 + max_nbnd) * sizeof(double);
  MPM_DISPATCH_KS(k_nd_down, ks, grid, dim3(256), smem, st, pdl, g, d, nodes, level_nodes, pmap);
}

void launch_reconstruct(const Grid& g, const DevState& d, const DevSub* subs, int nsub, int max_face, int max_dof,
                        int max_nf1, const DevNode* nodes, const int* leaf_node, const int* pmap, int branch, int pass,
                        bool pdl, cudaStream_t st) {
  const int faces = max_face <= 16 ? 16 : max_face <= 32 ? 32 : max_face <= 64 ? 64 : 128;
  const int ks = 256 / faces;
  const size_t smem = (size_t)(256 + (max_dof > 0 ? max_dof : 1) + max_nf1) * sizeof(double);
  MPM_DISPATCH_KS(k_reconstruct, ks, dim3(nsub, g.R), dim3(256), smem, st, pdl, g, d, subs, nodes, leaf_node, pmap,
                  branch, pass);
}

}  // namespace mpm
