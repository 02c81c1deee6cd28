// Per-item device functions shared by the interface-solve stage and the local kernels:
// interface basis values, the element right-hand side of Eq. (mrc2) (formed by the
// local-solve kernels that produce the traces) and the interface fluxes u_bar (formed by
// the downscaling kernel that consumes them, k_local.cu).
#pragma once
#include "mpm2p_internal.cuh"

namespace mpm {
namespace phase {

// Value at edge t of interface basis function kk (Legendre {1, 2 xi - 1} on segments of
// seg_len edges, xi of the edge midpoint).  2 xi - 1 = (2 (t mod seg_len) + 1 - seg_len) / seg_len:
// an integer numerator (exact) times inv_seg = 1 / seg_len (computed on the host; exact for
// powers of two).
__device__ __forceinline__ double side_basis(int kk, int t, int seg_len, int degree, double inv_seg) {
  const int nb = degree + 1;
  const int seg = kk / nb, pw = kk - seg * nb;
  if (t / seg_len != seg) return 0.0;
  if (pw == 0) return 1.0;
  return (double)(2 * (t % seg_len) + 1 - seg_len) * inv_seg;
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
    const double w = side_basis(kk, t, g.seg_len, g.degree, g.inv_seg);
    if (w == 0.0) continue;
    const double F = fb[f0 + t];
    if (isP) v -= w * F;
    else v += bhat[f0 + t] * s * w * F;
  }
  d.gvec[(long long)r * d.st_vec + leaf.v_off + k] = v;
}

// u_bar on face t of side `side` of subdomain sd, oriented along +x / +y (Section 4.1,
// u_bar = uhat_0 + delta u^n; with g.order = 1 also the first-order term of Eq. mpm_tf_4).  branch = 1 (after a basis build): the mean of the two
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
      if (g.order >= 1) {
        // first-order term: the mean of the one-sided epsilon^1 traces plus
        // (T^n - T^m)(dp0_c - dp0_nb), T^m the harmonic transmissibility of kappa^m (symmetric
        // in its two cells, so both sides round identically)
        const double F1o = d.trace1[(long long)r * d.st_face + sd.face_off + face_side_off(side, sd.a, sd.b) + t];
        const double F1n = d.trace1[(long long)r * d.st_face + nb.face_off + face_side_off(opp, nb.a, nb.b) + t];
        const double km0 = d.kap_m[cb + c], km1 = d.kap_m[cb + cn];
        const double Tm = div64(2.0 * (km0 * km1), km0 + km1);
        out = __dadd_rn(out, 0.5 * __dsub_rn(F1o, F1n));
        out = __dadd_rn(out, __dmul_rn(__dsub_rn(T, Tm), __dsub_rn(d.dp0[cb + c], d.dp0[cb + cn])));
      }
    }
  } else {
    out = Fo;
    // the perturbation traces carry homogeneous physical data; add F_n(p^m)
    if (branch == 0) out += phys_flux(g, side, d.kap_n[cb + c], d.p_m[cb + c]);
    if (branch == 0 && g.order >= 1) {
      // first-order term: its trace (homogeneous data) and, on a Dirichlet face,
      // 2 (kappa^n - kappa^m)_c dp0_c
      out += d.trace1[(long long)r * d.st_face + sd.face_off + face_side_off(side, sd.a, sd.b) + t];
      if (g.bc_type[side] == 0) out += 2.0 * (d.kap_n[cb + c] - d.kap_m[cb + c]) * d.dp0[cb + c];
    }
  }
  return (side == 0 || side == 2) ? -out : out;
}

// Upward step of the nested-dissection solve at one level-1 node nid (two leaf children) for
// realisation r, by all threads of one CTA: g_s gathered from the children's right-hand sides,
// then for every frontal row y[row] = sum_k G[k][row] g_s[k] into x (separator rows) or
// g_b[row] = gather(row) - y[row] into g (boundary rows), as the level kernels do (k_iface.cu).
// The children's vectors were written by other CTAs: read past L1.
__device__ __forceinline__ void nd_up_leaf_parent(const DevState& d, const DevNode* nodes, int nid, int r) {
  __shared__ double gs[4 * kMaxSide];  // a level-1 separator is one interface: at most 4 kMaxSide DOFs
  const DevNode nd = nodes[nid];
  const int nf = nd.nf, ns = nd.nsep;
  const long long vb = (long long)r * d.st_vec;
  const int* s0 = d.srcmap + nd.src_off;
  const int* s1 = s0 + nf;
  const double* g0 = d.gvec + vb + nodes[nd.child[0]].v_off;  // leaves: no separator part
  const double* g1 = d.gvec + vb + nodes[nd.child[1]].v_off;
  for (int k = threadIdx.x; k < ns; k += blockDim.x) {
    const int a0 = s0[k], a1 = s1[k];
    gs[k] = (a0 >= 0 ? __ldcg(g0 + a0) : 0.0) + (a1 >= 0 ? __ldcg(g1 + a1) : 0.0);
  }
  __syncthreads();
  const double* F = d.front + (long long)r * d.st_front + nd.f_off;
  for (int row = threadIdx.x; row < nf; row += blockDim.x) {
    double acc0 = 0.0, acc1 = 0.0;
    int k = 0;
    for (; k + 1 < ns; k += 2) {
      acc0 += F[(long long)k * nf + row] * gs[k];
      acc1 += F[(long long)(k + 1) * nf + row] * gs[k + 1];
    }
    if (k < ns) acc0 += F[(long long)k * nf + row] * gs[k];
    const double y = acc0 + acc1;
    if (row < ns) {
      d.xvec[vb + nd.v_off + row] = y;
    } else {
      const int a0 = s0[row], a1 = s1[row];
      d.gvec[vb + nd.v_off + row] = ((a0 >= 0 ? __ldcg(g0 + a0) : 0.0) + (a1 >= 0 ? __ldcg(g1 + a1) : 0.0)) - y;
    }
  }
}

// Called by every thread of a CTA of the MPM-2P local solve right after it wrote leaf lid's
// interface right-hand side (realisation r): the CTA that completes the second child of a
// level-1 node does that node's upward step (nd_up_leaf_parent), so the level-1 sweep of an
// MPM-2P update needs no launch of its own.  (After a basis build the level-1 step is launched
// behind the new factorisation instead, for the rebuilding realisations only.)  A ticket
// per node and realisation counts the completed children (last-arriving-block pattern: no CTA
// waits for another); the second arrival resets it for the next solve.
__device__ __forceinline__ void fold_up(const DevState& d, const DevNode* nodes, int lid, int r) {
  __shared__ int last;
  const int p = nodes[lid].parent;
  if (p < 0 || nodes[p].level != 1) return;
  __syncthreads();  // every write of this leaf's right-hand side issued
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int* t = d.nd_ticket + (long long)r * d.st_nodes + p;
    last = atomicAdd(t, 1u) == 1u;
    if (last) *t = 0u;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  nd_up_leaf_parent(d, nodes, p, r);
}

}  // namespace phase
}  // namespace mpm
