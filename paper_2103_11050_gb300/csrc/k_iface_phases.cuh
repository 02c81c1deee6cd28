// Per-item device functions of the interface-solve stage (Eq. mrc2 right-hand side,
// nested-dissection up / down sweeps, reconstruction of traces and p^m, interface fluxes
// u_bar).  The sweeps are called both by one-kernel-per-level launches and by the
// persistent cooperative kernel that runs the whole sweep in one launch (k_iface.cu); the
// right-hand side is formed by the local-solve kernels that produce the traces, u_bar by
// the downscaling kernel that consumes it (k_local.cu).
#pragma once
#include "mpm2p_internal.cuh"

namespace mpm {
namespace phase {

__device__ __forceinline__ double side_basis(int kk, int t, int seg_len, int degree) {
  const int nb = degree + 1;
  const int seg = kk / nb, pw = kk - seg * nb;
  if (t / seg_len != seg) return 0.0;
  if (pw == 0) return 1.0;
  const double xi = div64((t % seg_len) + 0.5, (double)seg_len);
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

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Element right-hand side of local DOF k of subdomain sd from the non-homogeneous
// (rebuild) or perturbation (MPM-2P) traces fb (this subdomain's, face order), moved to the
// right-hand side: psi rows -sum psi F, phi rows +sum bh s phi F, over the edges of the
// DOF's segment (its support).  Written to the leaf's g vector.
__device__ __forceinline__ void element_rhs(const Grid& g, const DevState& d, const DevSub& sd, const DevNode& leaf,
                                            int r, int k, const double* fb) {
  int side, isP, kk;
  dof_info(sd, k, side, isP, kk);
  const int f0 = face_side_off(side, sd.a, sd.b);
  const double s = sd.side_sign[side];
  const double* bhat = d.bhat + (long long)r * d.st_face + sd.face_off;
  const int t0 = (kk / (g.degree + 1)) * g.seg_len;
  double v = 0.0;
  for (int t = t0; t < t0 + g.seg_len; ++t) {
    const double w = side_basis(kk, t, g.seg_len, g.degree);
    if (w == 0.0) continue;
    const double F = fb[f0 + t];
    if (isP) v -= w * F;
    else v += bhat[f0 + t] * s * w * F;
  }
  d.gvec[(long long)r * d.st_vec + leaf.v_off + k] = v;
}

// Value of the gathered right-hand side of node nd at frontal index k (children's g).
__device__ __forceinline__ double gather_g(const DevState& d, const DevNode* nodes, const DevNode& nd, int r,
                                           const int* srcmap, int k) {
  const int* s0 = srcmap + nd.src_off;
  const int* s1 = s0 + nd.nf;
  double v = 0.0;
  if (s0[k] >= 0) {
    const DevNode& c0 = nodes[nd.child[0]];
    v += d.gvec[(long long)r * d.st_vec + c0.v_off + c0.nsep + s0[k]];
  }
  if (s1[k] >= 0) {
    const DevNode& c1 = nodes[nd.child[1]];
    v += d.gvec[(long long)r * d.st_vec + c1.v_off + c1.nsep + s1[k]];
  }
  return v;
}

// Upward solve, one frontal row per warp, from the transposed sweep G (k_iface.cu):
// y_s[row] = sum_k G[k][row] g_s[k] -> x (row < nsep), or
// g_b[row] = gather(row) - sum_k G[k][row] g_s[k] (row >= nsep).  gs: the node's gathered
// separator right-hand side (shared memory), or nullptr to gather from the children on the fly.
__device__ __forceinline__ void nd_up_row(const DevState& d, const DevNode* nodes, const DevNode& nd, int r, int row,
                                          const int* srcmap, int lane, const double* gs) {
  const int nf = nd.nf, ns = nd.nsep;
  const double* G = d.front + (long long)r * d.st_front + nd.f_off;
  double acc = 0.0;
  if (gs)
    for (int k = lane; k < ns; k += 32) acc += G[(long long)k * nf + row] * gs[k];
  else
    for (int k = lane; k < ns; k += 32) acc += G[(long long)k * nf + row] * gather_g(d, nodes, nd, r, srcmap, k);
  acc = warp_sum(acc);
  if (lane == 0) {
    if (row < ns) d.xvec[(long long)r * d.st_vec + nd.v_off + row] = acc;
    else d.gvec[(long long)r * d.st_vec + nd.v_off + row] = gather_g(d, nodes, nd, r, srcmap, row) - acc;
  }
}

// Downward solve, one separator row per warp: x_s[row] = y_s[row] + sum_k G[ns + k][row] x_b[k],
// x_b read from the parent.
__device__ __forceinline__ void nd_down_row(const DevState& d, const DevNode* nodes, const DevNode& nd, int r,
                                            int row, const int* pmap, int lane) {
  const int nf = nd.nf, ns = nd.nsep, nbd = nd.nbnd;
  const DevNode& pa = nodes[nd.parent];
  const double* xp = d.xvec + (long long)r * d.st_vec + pa.v_off;
  const int* pm = pmap + nd.pmap_off;
  const double* G = d.front + (long long)r * d.st_front + nd.f_off + (long long)ns * nf;
  double acc = 0.0;
  for (int k = lane; k < nbd; k += 32) acc += G[(long long)k * nf + row] * xp[pm[k]];
  acc = warp_sum(acc);
  if (lane == 0) d.xvec[(long long)r * d.st_vec + nd.v_off + row] += acc;
}

// Downward solve, boundary copy: x_b[k] = parent's x at the matching frontal index.
__device__ __forceinline__ void nd_down_copy(const DevState& d, const DevNode* nodes, const DevNode& nd, int r,
                                             const int* pmap, int k) {
  const DevNode& pa = nodes[nd.parent];
  d.xvec[(long long)r * d.st_vec + nd.v_off + nd.nsep + k] =
      d.xvec[(long long)r * d.st_vec + pa.v_off + pmap[nd.pmap_off + k]];
}

// Traces (and at a rebuild the MRCM-level pressure p^m) of subdomain sidx from the
// interface solution (whole CTA; cs: >= ndof doubles, red: 32 doubles of shared memory):
//   rebuild: p^m = pbar + P_hat c, F = Fbar + F_hat c, target mean = mean(p^m)
//   MPM-2P : F = dFbar + F_hat dc, target mean = mean(p^m) + mean(dpbar) + mu_hat . dc
__device__ inline void reconstruct(const Grid& g, const DevState& d, const DevSub* subs, const DevNode* nodes,
                            const int* leaf_node, int sidx, int r, int branch, double* cs, double* red) {
  const DevSub& sd = subs[sidx];
  const int a = sd.a, b = sd.b, m = a * b, nd = sd.ndof;
  const int nface = 2 * (a + b);
  if (nd > 0) {
    const DevNode& leaf = nodes[leaf_node[sidx]];
    const double* x = d.xvec + (long long)r * d.st_vec + leaf.v_off;
    for (int l = threadIdx.x; l < nd; l += blockDim.x) cs[l] = x[l];
  }
  __syncthreads();
  const double* tr = d.tr + (long long)r * d.st_tr + sd.tr_off;
  const double* fbar = d.fbar + (long long)r * d.st_face + sd.face_off;
  double* trace = d.trace + (long long)r * d.st_face + sd.face_off;
  for (int f = threadIdx.x; f < nface; f += blockDim.x) {
    double v = fbar[f];
    for (int l = 0; l < nd; ++l) v += tr[(long long)l * nface + f] * cs[l];
    trace[f] = v;
  }
  double part = 0.0;
  if (branch == 1) {
    const double* pf = d.pf + (long long)r * d.st_pf + sd.pf_off;
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
      double v = pf[(long long)nd * m + c];
      for (int l = 0; l < nd; ++l) v += pf[(long long)l * m + c] * cs[l];
      const int jl = c / a, il = c - jl * a;
      d.p_m[(long long)r * g.ncell() + (long long)(sd.y0 + jl) * g.nx + sd.x0 + il] = v;
      part += v;
    }
  } else if (threadIdx.x == 0) {
    const double* muh = d.mu_hat + (long long)r * d.st_dof + sd.dof_off;
    part = d.sub_mean[(long long)r * d.st_sub + sidx] * m;
    for (int l = 0; l < nd; ++l) part += muh[l] * cs[l] * m;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    const long long si = (long long)r * d.st_sub + sidx;
    if (branch == 1) {
      d.pm_mean[si] = s / m;
      d.sub_target[si] = s / m;
    } else {
      d.sub_target[si] = d.pm_mean[si] + s / m;
    }
  }
  __syncthreads();
}

// u_bar on face t of side `side` of subdomain sd, oriented along +x / +y (Section 4.1,
// u_bar = uhat_0 + delta u^n).  branch = 1 (after a basis build): the mean of the two
// one-sided MRCM traces on an interface, the trace itself on a physical side.  branch = 0
// (after a perturbation solve): the same from the epsilon^0 traces, plus
// F_n(p^m) = -kappa^n grad p^m.  Both subdomains of an interface face get bit-identical
// values: the outward flux is formed with explicitly rounded operations whose operands
// swap sign exactly when the two sides swap.
__device__ __forceinline__ double ubar_face(const Grid& g, const DevState& d, const DevSub* subs, const DevSub& sd,
                                            int r, int side, int t, int branch) {
  const int nx = g.nx;
  const long long cb = (long long)r * g.ncell();
  int ci, cj;  // cell of sd adjacent to the face
  if (side == 0) { ci = sd.x0; cj = sd.y0 + t; }
  else if (side == 1) { ci = sd.x0 + sd.a - 1; cj = sd.y0 + t; }
  else if (side == 2) { ci = sd.x0 + t; cj = sd.y0; }
  else { ci = sd.x0 + t; cj = sd.y0 + sd.b - 1; }
  const long long c = (long long)cj * nx + ci;
  const double Fo = d.trace[(long long)r * d.st_face + sd.face_off + face_side_off(side, sd.a, sd.b) + t];
  double out;  // outward from sd
  if (sd.side_kind[side] == 1) {
    const DevSub& nb = subs[sd.side_nbr[side]];
    const int opp = side ^ 1;  // 0 <-> 1, 2 <-> 3: the same face seen from the neighbour
    const double Fn = d.trace[(long long)r * d.st_face + nb.face_off + face_side_off(opp, nb.a, nb.b) + t];
    out = 0.5 * __dsub_rn(Fo, Fn);
    if (branch == 0) {
      long long cn, fi;
      double T;
      if (side == 0) { cn = c - 1; fi = (long long)cj * (nx + 1) + ci; }
      else if (side == 1) { cn = c + 1; fi = (long long)cj * (nx + 1) + ci + 1; }
      else if (side == 2) { cn = c - nx; fi = (long long)cj * nx + ci; }
      else { cn = c + nx; fi = (long long)(cj + 1) * nx + ci; }
      T = side < 2 ? d.tx[(long long)r * g.nfx() + fi] : d.ty[(long long)r * g.nfy() + fi];
      out = __dadd_rn(out, __dmul_rn(T, __dsub_rn(d.p_m[cb + c], d.p_m[cb + cn])));
    }
  } else {
    out = Fo;
    // the perturbation traces carry homogeneous physical data; add F_n(p^m)
    if (branch == 0) out += phys_flux(g, side, d.kap_n[cb + c], d.p_m[cb + c]);
  }
  return (side == 0 || side == 2) ? -out : out;
}

}  // namespace phase
}  // namespace mpm
