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
// in place.  With the flux rows negated the system is symmetric quasi-definite
// (Robin-weighted U block positive definite, P block negative definite when a Dirichlet
// side exists), so the sweep needs no pivoting.
// Solve: upward  y_s = F_ss^-1 g_s, g_b += (-F_bs F_ss^-1) g_s  (g_b -> parent);
//        downward x_s = y_s - (F_ss^-1 F_sb) x_b  (x_b from the parent).
#include "mpm2p_internal.cuh"

namespace mpm {

namespace {

constexpr int kTile = 32;

__device__ __forceinline__ double side_basis(int kk, int t, int seg_len, int degree) {
  const int nb = degree + 1;
  const int seg = kk / nb, pw = kk - seg * nb;
  if (t / seg_len != seg) return 0.0;
  if (pw == 0) return 1.0;
  const double xi = ((t % seg_len) + 0.5) / seg_len;
  return 2.0 * xi - 1.0;
}

// Side, kind (0 = U, 1 = P) and index within the side's space of local DOF k.
__device__ __forceinline__ bool dof_info(const DevSub& sd, int k, int& side, int& isP, int& kk) {
  for (int q = 0; q < 4; ++q) {
    if (sd.side_kind[q] != 1) continue;
    const int d0 = sd.side_dof0[q], nb = sd.side_nb[q];
    if (k >= d0 && k < d0 + 2 * nb) {
      side = q;
      isP = k >= d0 + nb;
      kk = isP ? k - d0 - nb : k - d0;
      return true;
    }
  }
  return false;
}

__device__ __forceinline__ int side_len(const DevSub& sd, int side) { return side < 2 ? sd.b : sd.a; }

__global__ void k_element_matrix(Grid g, DevState d, const DevSub* subs, const DevNode* nodes,
                                 const int* leaf_node) {
  const int r = blockIdx.y;
  if (d.rebuild[r] != 1) return;
  const int sidx = blockIdx.x;
  const DevSub sd = subs[sidx];
  const int nd = sd.ndof;
  if (nd == 0) return;
  const DevNode leaf = nodes[leaf_node[sidx]];
  double* E = d.front + (long long)r * d.st_front + leaf.f_off;
  const double* tr = d.tr + (long long)r * d.st_tr + sd.tr_off;
  const double* bhat = d.bhat + (long long)r * d.st_face + sd.face_off;
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
      const double w = side_basis(kk, t, g.seg_len, g.degree);
      if (w == 0.0) continue;
      const double F = tr[(long long)(f0 + t) * nd + l];
      if (isP) {
        v += w * F;
      } else {
        const double bh = bhat[f0 + t];
        v -= bh * s * w * F;
        if (!lisP && lside == side) v += bh * w * side_basis(ll, t, g.seg_len, g.degree);
      }
    }
    E[e] = v;
  }
}

// Element right-hand side from the non-homogeneous (rebuild) or perturbation (MPM-2P)
// traces fbar, moved to the right-hand side: psi rows -sum psi F, phi rows +sum bh s phi F.
__global__ void k_element_rhs(Grid g, DevState d, const DevSub* subs, const DevNode* nodes,
                              const int* leaf_node) {
  const int r = blockIdx.y;
  const int sidx = blockIdx.x;
  const DevSub sd = subs[sidx];
  const int nd = sd.ndof;
  if (nd == 0) return;
  const DevNode leaf = nodes[leaf_node[sidx]];
  double* gv = d.gvec + (long long)r * d.st_vec + leaf.v_off;
  const double* fb = d.fbar + (long long)r * d.st_face + sd.face_off;
  const double* bhat = d.bhat + (long long)r * d.st_face + sd.face_off;
  for (int k = threadIdx.x; k < nd; k += blockDim.x) {
    int side, isP, kk;
    dof_info(sd, k, side, isP, kk);
    const int L = side_len(sd, side);
    const int f0 = face_side_off(side, sd.a, sd.b);
    const double s = sd.side_sign[side];
    double v = 0.0;
    for (int t = 0; t < L; ++t) {
      const double w = side_basis(kk, t, g.seg_len, g.degree);
      if (w == 0.0) continue;
      const double F = fb[f0 + t];
      if (isP) v -= w * F;
      else v += bhat[f0 + t] * s * w * F;
    }
    gv[k] = v;
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
  double* F = d.front + (long long)r * d.st_front + nd.f_off;
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

// Sweep step 1: invert the pivot block P = [k0, k0+nb) of every node (one CTA per node).
__global__ void k_sweep_pivot(Grid g, DevState d, const DevNode* nodes, const int* level_nodes, int k0) {
  __shared__ double piv[2][2 * kPivotChunk + 1];
  const int r = blockIdx.y;
  if (d.rebuild[r] != 1) return;
  const int nid = level_nodes[blockIdx.x];
  const DevNode nd = nodes[nid];
  if (k0 >= nd.nsep) return;
  const int nb = min(kPivotChunk, nd.nsep - k0);
  double* F = d.front + (long long)r * d.st_front + nd.f_off;
  const int tid = threadIdx.x;
  const int i = tid / kPivotChunk, k = tid - i * kPivotChunk;
  const bool active = i < nb && k < nb;
  double v = active ? F[(long long)(k0 + i) * nd.nf + k0 + k] : 0.0;
  for (int p = 0; p < nb; ++p) {
    double* buf = piv[p & 1];
    if (active) {
      if (k == p) buf[i] = v;
      if (i == p) buf[kPivotChunk + k] = v;
      if (i == p && k == p) buf[2 * kPivotChunk] = 1.0 / v;
    }
    __syncthreads();
    if (active) {
      const double ip = buf[2 * kPivotChunk];
      const double mip = buf[i], mpk = buf[kPivotChunk + k];
      if (i == p && k == p) v = ip;
      else if (i == p) v = mpk * ip;
      else if (k == p) v = -mip * ip;
      else v = v - mip * (mpk * ip);
    }
  }
  if (active) {
    F[(long long)(k0 + i) * nd.nf + k0 + k] = v;
    d.pivinv[((long long)r * d.st_lvl + blockIdx.x) * kPivotChunk * kPivotChunk + i * kPivotChunk + k] = v;
  }
}

// Sweep step 2: pivot rows  M_Pc <- Pinv M_Pc  and pivot columns  M_rP <- -M_rP Pinv
// (old M_rP saved for step 3), for every index outside P.
__global__ void k_sweep_rowcol(Grid g, DevState d, const DevNode* nodes, const int* level_nodes, int k0) {
  __shared__ double P[kPivotChunk][kPivotChunk];
  const int r = blockIdx.z;
  if (d.rebuild[r] != 1) return;
  const DevNode nd = nodes[level_nodes[blockIdx.x]];
  if (k0 >= nd.nsep) return;
  const int nb = min(kPivotChunk, nd.nsep - k0);
  const int nf = nd.nf;
  const int idx = blockIdx.y * blockDim.x + threadIdx.x;
  const double* Pg = d.pivinv + ((long long)r * d.st_lvl + blockIdx.x) * kPivotChunk * kPivotChunk;
  for (int e = threadIdx.x; e < kPivotChunk * kPivotChunk; e += blockDim.x) P[e / kPivotChunk][e % kPivotChunk] = Pg[e];
  __syncthreads();
  if (idx >= nf || (idx >= k0 && idx < k0 + nb)) return;
  double* F = d.front + (long long)r * d.st_front + nd.f_off;
  double* Cold = d.colold + (long long)r * d.st_col + (long long)nd.v_off * kPivotChunk;
  double col[kPivotChunk], row[kPivotChunk];
#pragma unroll
  for (int l = 0; l < kPivotChunk; ++l) {
    col[l] = l < nb ? F[(long long)(k0 + l) * nf + idx] : 0.0;
    row[l] = l < nb ? F[(long long)idx * nf + k0 + l] : 0.0;
  }
#pragma unroll
  for (int l = 0; l < kPivotChunk; ++l) {
    if (l >= nb) break;
    double a = 0.0, c = 0.0;
#pragma unroll
    for (int q = 0; q < kPivotChunk; ++q) {
      if (q >= nb) break;
      a += P[l][q] * col[q];
      c += row[q] * P[q][l];
    }
    F[(long long)(k0 + l) * nf + idx] = a;
    F[(long long)idx * nf + k0 + l] = -c;
    Cold[(long long)idx * kPivotChunk + l] = row[l];
  }
}

// Sweep step 3: trailing update  M_rc -= Mold_rP M_Pc(new)  for r, c outside P.
__global__ void k_sweep_trailing(Grid g, DevState d, const DevNode* nodes, const int* level_nodes, int k0,
                                 int tiles_x) {
  __shared__ double A[kTile][kPivotChunk + 1];
  __shared__ double B[kPivotChunk][kTile + 1];
  const int r = blockIdx.z;
  if (d.rebuild[r] != 1) return;
  const DevNode nd = nodes[level_nodes[blockIdx.x]];
  if (k0 >= nd.nsep) return;
  const int nb = min(kPivotChunk, nd.nsep - k0);
  const int nf = nd.nf;
  const int ty = blockIdx.y / tiles_x, tx = blockIdx.y - ty * tiles_x;
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
    F[(long long)row * nf + colx] -= acc;
  }
}

constexpr int kRowsPerCta = 8;  // frontal rows per CTA of the solve kernels (one row per warp)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Upward solve at one level: gather g from the children, y_s = M_ss g_s -> x, g_b += M_bs g_s.
// One warp per frontal row (lane-strided dot product, shuffle reduction).
__global__ void k_nd_up(Grid g, DevState d, const DevNode* nodes, const int* level_nodes, const int* srcmap) {
  extern __shared__ double gs[];
  const int r = blockIdx.z;
  const DevNode nd = nodes[level_nodes[blockIdx.x]];
  const int nf = nd.nf, ns = nd.nsep;
  const int row0 = blockIdx.y * kRowsPerCta;
  if (row0 >= nf) return;
  const int* s0 = srcmap + nd.src_off;
  const int* s1 = s0 + nf;
  const DevNode c0 = nodes[nd.child[0]], c1 = nodes[nd.child[1]];
  const double* g0 = d.gvec + (long long)r * d.st_vec + c0.v_off;
  const double* g1 = d.gvec + (long long)r * d.st_vec + c1.v_off;
  for (int k = threadIdx.x; k < ns; k += blockDim.x) {
    double v = 0.0;
    if (s0[k] >= 0) v += g0[c0.nsep + s0[k]];
    if (s1[k] >= 0) v += g1[c1.nsep + s1[k]];
    gs[k] = v;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const double* F = d.front + (long long)r * d.st_front + nd.f_off;
  for (int row = row0 + warp; row < min(nf, row0 + kRowsPerCta); row += nw) {
    const double* Fr = F + (long long)row * nf;
    double acc = 0.0;
    for (int k = lane; k < ns; k += 32) acc += Fr[k] * gs[k];
    acc = warp_sum(acc);
    if (lane == 0) {
      if (row < ns) {
        d.xvec[(long long)r * d.st_vec + nd.v_off + row] = acc;
      } else {
        double v = 0.0;
        if (s0[row] >= 0) v += g0[c0.nsep + s0[row]];
        if (s1[row] >= 0) v += g1[c1.nsep + s1[row]];
        d.gvec[(long long)r * d.st_vec + nd.v_off + row] = v + acc;
      }
    }
  }
}

// Downward solve at one level: x_b from the parent, x_s = y_s - M_sb x_b (one warp per row).
__global__ void k_nd_down(Grid g, DevState d, const DevNode* nodes, const int* level_nodes, const int* pmap) {
  extern __shared__ double xb[];
  const int r = blockIdx.z;
  const DevNode nd = nodes[level_nodes[blockIdx.x]];
  const int nf = nd.nf, ns = nd.nsep, nbd = nd.nbnd;
  if (nd.parent < 0) return;
  const int row0 = blockIdx.y * kRowsPerCta;
  if (row0 > 0 && row0 >= ns) return;
  double* x = d.xvec + (long long)r * d.st_vec + nd.v_off;
  const DevNode pa = nodes[nd.parent];
  const double* xp = d.xvec + (long long)r * d.st_vec + pa.v_off;
  const int* pm = pmap + nd.pmap_off;
  for (int k = threadIdx.x; k < nbd; k += blockDim.x) {
    const double v = xp[pm[k]];
    xb[k] = v;
    if (blockIdx.y == 0) x[ns + k] = v;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const double* F = d.front + (long long)r * d.st_front + nd.f_off;
  for (int row = row0 + warp; row < min(ns, row0 + kRowsPerCta); row += nw) {
    const double* Fr = F + (long long)row * nf + ns;
    double acc = 0.0;
    for (int k = lane; k < nbd; k += 32) acc += Fr[k] * xb[k];
    acc = warp_sum(acc);
    if (lane == 0) x[row] -= acc;
  }
}

}  // namespace

void launch_element_matrix(const Grid& g, const DevState& d, const DevSub* subs, int nsub, const DevNode* nodes,
                           const int* leaf_node, cudaStream_t st) {
  k_element_matrix<<<dim3(nsub, g.R), 256, 0, st>>>(g, d, subs, nodes, leaf_node);
  ++g_launches;
}

void launch_element_rhs(const Grid& g, const DevState& d, const DevSub* subs, int nsub, const DevNode* nodes,
                        const int* leaf_node, cudaStream_t st) {
  k_element_rhs<<<dim3(nsub, g.R), 128, 0, st>>>(g, d, subs, nodes, leaf_node);
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
  for (int k0 = 0; k0 < max_nsep; k0 += kPivotChunk) {
    k_sweep_pivot<<<dim3(nlev, g.R), kPivotChunk * kPivotChunk, 0, st>>>(g, d, nodes, level_nodes, k0);
    ++g_launches;
    k_sweep_rowcol<<<dim3(nlev, (max_nf + 127) / 128, g.R), 128, 0, st>>>(g, d, nodes, level_nodes, k0);
    ++g_launches;
    k_sweep_trailing<<<dim3(nlev, tiles_x * tiles_x, g.R), 256, 0, st>>>(g, d, nodes, level_nodes, k0, tiles_x);
    ++g_launches;
  }
}

void launch_nd_up(const Grid& g, const DevState& d, const DevNode* nodes, const int* level_nodes, int nlev,
                  int max_nf, int max_nsep, const int* srcmap, cudaStream_t st) {
  k_nd_up<<<dim3(nlev, (max_nf + kRowsPerCta - 1) / kRowsPerCta, g.R), 256, (size_t)max_nsep * sizeof(double), st>>>(
      g, d, nodes, level_nodes, srcmap);
  ++g_launches;
}

void launch_nd_down(const Grid& g, const DevState& d, const DevNode* nodes, const int* level_nodes, int nlev,
                    int max_nsep, int max_nbnd, const int* pmap, cudaStream_t st) {
  const int ny = max_nsep > 0 ? (max_nsep + kRowsPerCta - 1) / kRowsPerCta : 1;
  k_nd_down<<<dim3(nlev, ny, g.R), 256, (size_t)(max_nbnd > 0 ? max_nbnd : 1) * sizeof(double), st>>>(
      g, d, nodes, level_nodes, pmap);
  ++g_launches;
}

}  // namespace mpm
