// Tensor-core multi-right-hand-side block solves for the basis-function solves of an MRCM
// rebuild (Eqs. mrc_homogeneous, mrc_non_homogeneous): all ndof + 1 right-hand sides of a
// subdomain against its stored Robin factor.
//
// The twisted block substitution of k_local.cu,
//   forward   W_j = Q_j (Z_j + t o W_prev),   middle  X_mid = Q_mid (Z_mid + t o W_mid-1 + t o W_mid+1),
//   backward  X_j = W_j + Q_j (t o X_next),
// is a chain of dense products of the a x a explicit inverse pivot Q_j with an a x ncol block of
// right-hand sides: the dense contraction of the rebuild.  Here each product runs on the tensor
// cores with warp-level mma.sync (operands from shared memory, float32 accumulation):
//   kTf32    m16n8k8 tf32: both operands rounded to tf32 (10-bit mantissa);
//   kTf32x3  the same instruction three times on split operands, x = hi + lo with hi = tf32(x) and
//            lo = tf32(x - hi), accumulating hi.hi + hi.lo + lo.hi (the lo.lo term is below float32
//            rounding): products accurate to about float32;
//   kBf16    m16n8k16 bf16: both operands rounded to bf16 (7-bit mantissa).
// The float64 iterative refinement around it (k_local.cu) recovers float64 accuracy, or reports
// that it cannot.  Warps come in pairs: warp 2g runs the top chain and warp 2g + 1 the bottom
// chain of column group g, so the two chains run concurrently and a warp only waits for its
// own previous product (a __syncwarp); the middle row and the switch from the forward to the
// backward sweep take three block barriers.
//
// Fragment layouts (PTX ISA, mma.m16n8k8 / m16n8k16, g = lane / 4, t = lane % 4):
//   A (16 x k, row major)   tf32: a0 = A[g][t], a1 = A[g+8][t], a2 = A[g][t+4], a3 = A[g+8][t+4]
//                           bf16: a0 = A[g][2t..2t+1], a1 = A[g+8][2t..], a2 = A[g][2t+8..], a3 = A[g+8][2t+8..]
//   B (k x 8, column major) tf32: b0 = B[t][g], b1 = B[t+4][g]
//                           bf16: b0 = B[2t..2t+1][g], b1 = B[2t+8..2t+9][g]
//   C (16 x 8)              c0 = C[g][2t], c1 = C[g][2t+1], c2 = C[g+8][2t], c3 = C[g+8][2t+1]
#pragma once
#include <cuda_bf16.h>

#include "mpm2p_internal.cuh"

namespace mpm {
namespace tc {

enum Kind { kTf32 = 1, kTf32x3 = 2, kBf16 = 3 };

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Row stride (floats) of the right-hand-side blocks for ncp columns: at least ncp, and 8 more
// than a multiple of 32 so that the B-fragment loads of a warp hit 32 distinct banks.
__host__ __device__ inline int tc_ld(int ncp) { return (ncp + 23) / 32 * 32 + 8; }

// One product  Out_j[r][col] = sum_k Q_j[r][k] Zt[k][col]  for the rows r < a of block row j and
// the n-tiles [nt0, nt1) of 8 columns, with Zt[k][col] = Z[j][k][col] + tp[k] * P[k][col]
// (P = the neighbouring block row of the chain, tp its coupling; both skipped when P is null),
// and a second neighbour term for the middle row; if add, Out += (the backward step adds
// W_j).  Z, P, P2 and Out are block rows of [m][ld] float arrays; Q_j is [A][A] (identity
// padded).  All 32 lanes of the warp take part.
template <int A, int KIND>
__device__ __forceinline__ void block_product(const float* Qj, int a, const float* Z, const float* P, const float* tp,
                                              const float* P2, const float* tp2, float* Out, const float* Add, int ld,
                                              int nt0, int nt1) {
  constexpr int MT = (A + 15) / 16;             // 16-row tiles
  constexpr int KS = KIND == kBf16 ? 16 : 8;    // k per instruction
  constexpr int KT = (A + KS - 1) / KS;         // k-steps (A = 8 with bf16: one step, upper half zero)
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  auto zt = [&](int k, int col) -> float {     // the right-hand side with its neighbour terms
    if (k >= a) return 0.0f;
    float v = Z ? Z[k * ld + col] : 0.0f;
    if (P) v = fmaf(tp[k], P[k * ld + col], v);
    if (P2) v = fmaf(tp2[k], P2[k * ld + col], v);
    return v;
  };
  auto qv = [&](int r, int k) -> float { return (r < a && k < A) ? Qj[r * A + k] : 0.0f; };
#pragma unroll
  for (int mt = 0; mt < MT; ++mt) {
    const int r0 = mt * 16 + g, r1 = r0 + 8;
    // A fragments of this m-tile for every k-step (held in registers over the n-tiles)
    uint32_t ah[KT][4], al[KT][4];
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
      if (KIND == kBf16) {
        const int k = kt * 16 + 2 * t;
        ah[kt][0] = pack_bf16(qv(r0, k), qv(r0, k + 1));
        ah[kt][1] = pack_bf16(qv(r1, k), qv(r1, k + 1));
        ah[kt][2] = pack_bf16(qv(r0, k + 8), qv(r0, k + 9));
        ah[kt][3] = pack_bf16(qv(r1, k + 8), qv(r1, k + 9));
      } else {
        const int k = kt * 8 + t;
        const float v[4] = {qv(r0, k), qv(r1, k), qv(r0, k + 4), qv(r1, k + 4)};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ah[kt][q] = to_tf32(v[q]);
          al[kt][q] = KIND == kTf32x3 ? to_tf32(v[q] - __uint_as_float(ah[kt][q])) : 0u;
        }
      }
    }
    for (int nt = nt0; nt < nt1; ++nt) {
      const int col = nt * 8 + g;
      float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int kt = 0; kt < KT; ++kt) {
        if (KIND == kBf16) {
          const int k = kt * 16 + 2 * t;
          const uint32_t b0 = pack_bf16(zt(k, col), zt(k + 1, col));
          const uint32_t b1 = pack_bf16(zt(k + 8, col), zt(k + 9, col));
          mma_bf16(acc, ah[kt][0], ah[kt][1], ah[kt][2], ah[kt][3], b0, b1);
        } else {
          const int k = kt * 8 + t;
          const float z0 = zt(k, col), z1 = zt(k + 4, col);
          const uint32_t bh0 = to_tf32(z0), bh1 = to_tf32(z1);
          if (KIND == kTf32x3) {
            const uint32_t bl0 = to_tf32(z0 - __uint_as_float(bh0)), bl1 = to_tf32(z1 - __uint_as_float(bh1));
            mma_tf32(acc, al[kt][0], al[kt][1], al[kt][2], al[kt][3], bh0, bh1);
            mma_tf32(acc, ah[kt][0], ah[kt][1], ah[kt][2], ah[kt][3], bl0, bl1);
          }
          mma_tf32(acc, ah[kt][0], ah[kt][1], ah[kt][2], ah[kt][3], bh0, bh1);
        }
      }
      const int cc = nt * 8 + 2 * t;
      if (r0 < a) {
        Out[r0 * ld + cc] = acc[0] + (Add ? Add[r0 * ld + cc] : 0.0f);
        Out[r0 * ld + cc + 1] = acc[1] + (Add ? Add[r0 * ld + cc + 1] : 0.0f);
      }
      if (r1 < a) {
        Out[r1 * ld + cc] = acc[2] + (Add ? Add[r1 * ld + cc] : 0.0f);
        Out[r1 * ld + cc + 1] = acc[3] + (Add ? Add[r1 * ld + cc + 1] : 0.0f);
      }
    }
  }
}

// Twisted multi-right-hand-side solve  (S A S) X = Z  in place on Z ([m][ld] floats, ncp
// columns, ncp a multiple of 8), W: workspace of the same shape; Q: [b][A][A] factor, th[m]: the
// scaled north couplings (th[j a + i] couples rows j and j + 1).  blockDim.x / 64 column groups,
// each a pair of warps (top chain, bottom chain).  Ends with a block barrier.
template <int A, int KIND>
__device__ void block_solve_tc(const DevSub& sd, const float* th, const float* Q, float* Z, float* W, int ld, int ncp) {
  const int a = sd.a, b = sd.b, mid = b / 2;
  const int warp = threadIdx.x >> 5, chain = warp & 1, grp = warp >> 1, ngrp = blockDim.x >> 6;
  const int ntile = ncp / 8;
  const int nt0 = grp * ntile / ngrp, nt1 = (grp + 1) * ntile / ngrp;  // this group's n-tiles
  auto row = [&](float* M, int j) { return M + (size_t)j * a * ld; };
  auto crow = [&](const float* M, int j) { return M + (size_t)j * a * ld; };
  // forward: top chain j = 0 .. mid-1 (coupling th row j-1), bottom chain j = b-1 .. mid+1 (th row j)
  const int nsteps = chain == 0 ? mid : b - 1 - mid;
  for (int k = 0; k < nsteps; ++k) {
    const int j = chain == 0 ? k : b - 1 - k;
    const int jp = chain == 0 ? j - 1 : j + 1;  // previous row of the chain
    const int jc = chain == 0 ? j - 1 : j;      // its coupling row in th
    block_product<A, KIND>(Q + (size_t)j * A * A, a, crow(Z, j), k > 0 ? crow(W, jp) : nullptr,
                           k > 0 ? th + (size_t)jc * a : nullptr, nullptr, nullptr, row(W, j), nullptr, ld, nt0, nt1);
    __syncwarp();
  }
  __syncthreads();
  // middle row: X_mid = Q_mid (Z_mid + th_{mid-1} o W_{mid-1} + th_mid o W_{mid+1}), by the top-chain
  // warps, into the free row W_mid (with two m-tiles the second one still reads Z_mid after the
  // first has written), then copied to Z_mid
  if (chain == 0)
    block_product<A, KIND>(Q + (size_t)mid * A * A, a, crow(Z, mid), mid > 0 ? crow(W, mid - 1) : nullptr,
                           mid > 0 ? th + (size_t)(mid - 1) * a : nullptr, mid < b - 1 ? crow(W, mid + 1) : nullptr,
                           mid < b - 1 ? th + (size_t)mid * a : nullptr, row(W, mid), nullptr, ld, nt0, nt1);
  __syncthreads();
  for (int e = threadIdx.x; e < a * ncp; e += blockDim.x) {
    const int i = e / ncp, col = e - i * ncp;
    row(Z, mid)[i * ld + col] = crow(W, mid)[i * ld + col];
  }
  __syncthreads();
  // backward: X_j = W_j + Q_j (th o X_next), top j = mid-1 .. 0 (next j+1, th row j), bottom j = mid+1 .. b-1
  for (int k = 0; k < nsteps; ++k) {
    const int j = chain == 0 ? mid - 1 - k : mid + 1 + k;
    const int jn = chain == 0 ? j + 1 : j - 1;
    const int jc = chain == 0 ? j : j - 1;
    // Zt = 0 + th o X_next: the product of Q_j with the coupled neighbour alone, plus W_j
    block_product<A, KIND>(Q + (size_t)j * A * A, a, nullptr, crow(Z, jn), th + (size_t)jc * a, nullptr, nullptr,
                           row(Z, j), crow(W, j), ld, nt0, nt1);
    __syncwarp();
  }
  __syncthreads();
}

}  // namespace tc
}  // namespace mpm
