// Device set-up of one operator of a structured square mesh, and the
// per-block reductions of a stacked context (serving with an operator per
// request).
//
// Mesh: N x N vertices of the unit square, vertex (x, y) = y N + x, every
// cell split by its SW->NE diagonal into a lower triangle (SW, SE, NE) and
// an upper one (SW, NE, NW); element coefficients ke[2 (cy (N-1) + cx) + t]
// (t = 0 lower, 1 upper), the order of the square meshes' element lists.
// Operators are kept over ALL vertices as 7-point stencils per vertex,
// slots 0 diagonal, 1 SW (-N-1), 2 S (-N), 3 W (-1), 4 E (+1), 5 N (+N),
// 6 NE (+N+1); a slot whose neighbour lies outside the grid holds 0.
//
//  k_sq_assemble   the P1 stiffness A_ab = sum_T k_T |T| grad phi_a . grad phi_b
//                  (Sec. 2.1's P1 discretisation): on a right isosceles
//                  triangle the element matrix is k_T/2 [[1,-1,0],[-1,2,-1],
//                  [0,-1,1]] in the order (acute, right-angle, acute), so the
//                  hypotenuse couplings (SW, NE slots) are exactly zero.
//  k_sq_galerkin   A_{l+1} = P^T A_l P (Sec. 2.2) with P the natural
//                  inclusion: coarse vertex (X, Y) sits on fine vertex
//                  (2X, 2Y) (weight 1) and is an end of the six coarse edges
//                  whose fine midpoints (2X +- 1, 2Y), (2X, 2Y +- 1),
//                  (2X + 1, 2Y + 1), (2X - 1, 2Y - 1) carry weight 1/2.
//  k_sq_write      one block of a stacked level: the drop rule |a_ij| <=
//                  1e-12 max(|a_ii|, |a_jj|) on the full operator, deg_i =
//                  kept neighbours before Dirichlet elimination, and the
//                  interior rows' DIA values, diagonal, 1/diagonal, 1/deg.
//  k_sq_coarse     the coarsest level of one block is one vertex: its entry
//                  of the context's explicit coarse inverse is 1/a.
#pragma once

#include "kernels.cuh"

namespace mgk {

constexpr int kSqSlots = 7;

__device__ __forceinline__ void sq_slot_offset(int k, int& dx, int& dy) {
  // slots 1..6: SW, S, W, E, N, NE
  const int tx[kSqSlots] = {0, -1, 0, -1, 1, 0, 1};
  const int ty[kSqSlots] = {0, -1, -1, 0, 0, 1, 1};
  dx = tx[k];
  dy = ty[k];
}

// slot of the offset (dx, dy), or -1
__device__ __forceinline__ int sq_slot_of(int dx, int dy) {
  if (dx == 0 && dy == 0) return 0;
  if (dx == -1 && dy == -1) return 1;
  if (dx == 0 && dy == -1) return 2;
  if (dx == -1 && dy == 0) return 3;
  if (dx == 1 && dy == 0) return 4;
  if (dx == 0 && dy == 1) return 5;
  if (dx == 1 && dy == 1) return 6;
  return -1;
}

__global__ void k_sq_assemble(int N, const double* __restrict__ ke, double* __restrict__ S) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N * N) return;
  const int x = v % N, y = v / N, nc = N - 1;
  auto kc = [&](int cx, int cy, int t) -> double {
    return (cx < 0 || cy < 0 || cx >= nc || cy >= nc) ? 0.0 : ke[2 * ((size_t)cy * nc + cx) + t];
  };
  // the six elements at (x, y): the lower and upper triangles of the cell to
  // the SW, the upper one of the cell to the SE, the lower one of the cell to
  // the NW, both of the cell to the NE
  const double sw_lo = kc(x - 1, y - 1, 0), sw_up = kc(x - 1, y - 1, 1);
  const double se_up = kc(x, y - 1, 1), nw_lo = kc(x - 1, y, 0);
  const double ne_lo = kc(x, y, 0), ne_up = kc(x, y, 1);
  double* s = S + (size_t)v * kSqSlots;
  s[0] = 0.5 * sw_lo + 0.5 * sw_up + se_up + nw_lo + 0.5 * ne_lo + 0.5 * ne_up;
  s[1] = 0.0;
  s[2] = -0.5 * sw_lo - 0.5 * se_up;  // S (x, y-1)
  s[3] = -0.5 * sw_up - 0.5 * nw_lo;  // W (x-1, y)
  s[4] = -0.5 * se_up - 0.5 * ne_lo;  // E (x+1, y)
  s[5] = -0.5 * nw_lo - 0.5 * ne_up;  // N (x, y+1)
  s[6] = 0.0;
  if (y == 0) s[2] = 0.0;
  if (x == 0) s[3] = 0.0;
  if (x == N - 1) s[4] = 0.0;
  if (y == N - 1) s[5] = 0.0;
}

__global__ void k_sq_galerkin(int Nf, const double* __restrict__ Sf, int Nc,
                              double* __restrict__ Sc) {
  const int V = blockIdx.x * blockDim.x + threadIdx.x;
  if (V >= Nc * Nc) return;
  const int X = V % Nc, Y = V / Nc;
  double acc[kSqSlots];
#pragma unroll
  for (int k = 0; k < kSqSlots; ++k) acc[k] = 0.0;
  // children of (X, Y): itself, then the six edge midpoints
  const int cdx[kSqSlots] = {0, -1, 0, -1, 1, 0, 1};
  const int cdy[kSqSlots] = {0, -1, -1, 0, 0, 1, 1};
  auto add = [&](int JX, int JY, double w) {
    const int k = sq_slot_of(JX - X, JY - Y);
    if (k >= 0 && JX >= 0 && JY >= 0 && JX < Nc && JY < Nc) acc[k] += w;
  };
  for (int c = 0; c < kSqSlots; ++c) {
    const int ix = 2 * X + cdx[c], iy = 2 * Y + cdy[c];
    if (ix < 0 || iy < 0 || ix >= Nf || iy >= Nf) continue;
    const double wi = c == 0 ? 1.0 : 0.5;
    const double* s = Sf + ((size_t)iy * Nf + ix) * kSqSlots;
    for (int k = 0; k < kSqSlots; ++k) {
      int dx, dy;
      sq_slot_offset(k, dx, dy);
      const int jx = ix + dx, jy = iy + dy;
      const double a = s[k];
      if (a == 0.0 || jx < 0 || jy < 0 || jx >= Nf || jy >= Nf) continue;
      const double wa = wi * a;
      const int px = jx & 1, py = jy & 1;
      if (!px && !py) {
        add(jx / 2, jy / 2, wa);
      } else if (px && !py) {
        add((jx - 1) / 2, jy / 2, 0.5 * wa);
        add((jx + 1) / 2, jy / 2, 0.5 * wa);
      } else if (!px && py) {
        add(jx / 2, (jy - 1) / 2, 0.5 * wa);
        add(jx / 2, (jy + 1) / 2, 0.5 * wa);
      } else {
        add((jx - 1) / 2, (jy - 1) / 2, 0.5 * wa);
        add((jx + 1) / 2, (jy + 1) / 2, 0.5 * wa);
      }
    }
  }
  double* out = Sc + (size_t)V * kSqSlots;
#pragma unroll
  for (int k = 0; k < kSqSlots; ++k) out[k] = acc[k];
}

// DIA offsets of one stacked level (ascending) and the slot each reads.
struct SqDia {
  int ndia;
  int slot[kMaxDia];
};

template <class T>
__global__ void k_sq_write(int N, const double* __restrict__ S, int block, SqDia dia,
                           int n_stacked, T* __restrict__ dval, T* __restrict__ diag,
                           T* __restrict__ dinv, T* __restrict__ invdeg,
                           unsigned char* __restrict__ nbm, double* __restrict__ dval64,
                           double* __restrict__ diag64, double* __restrict__ dinv64,
                           unsigned char* __restrict__ nbm64) {
  const int w = N - 2, m = w * w;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  const int x = r % w + 1, y = r / w + 1;
  const double* s = S + ((size_t)y * N + x) * kSqSlots;
  const double aii = s[0];
  double vals[kSqSlots];
  int deg = 0;
#pragma unroll
  for (int k = 1; k < kSqSlots; ++k) {
    int dx, dy;
    sq_slot_offset(k, dx, dy);
    const int jx = x + dx, jy = y + dy;  // always inside the full grid here
    const double a = s[k];
    const double ajj = S[((size_t)jy * N + jx) * kSqSlots];
    const bool keep = fabs(a) > 1e-12 * fmax(fabs(aii), fabs(ajj));
    deg += keep ? 1 : 0;
    const bool interior = jx > 0 && jy > 0 && jx < N - 1 && jy < N - 1;
    vals[k] = keep && interior ? a : 0.0;
  }
  const size_t R = (size_t)block * m + r;
  unsigned msk = 0, msk64 = 0;  // the rows' neighbour masks (bit d: value d nonzero)
  for (int d = 0; d < dia.ndia; ++d) {
    const double v = vals[dia.slot[d]];
    dval[(size_t)d * n_stacked + R] = (T)v;
    msk |= ((T)v != T(0) ? 1u : 0u) << d;
    if (dval64) dval64[(size_t)d * n_stacked + R] = v;
    msk64 |= (v != 0.0 ? 1u : 0u) << d;
  }
  if (nbm) nbm[R] = (unsigned char)msk;
  if (nbm64) nbm64[R] = (unsigned char)msk64;
  const double di = 1.0 / aii;
  diag[R] = (T)aii;
  dinv[R] = (T)di;
  invdeg[R] = (T)(1.0 / (double)deg);
  if (diag64) {
    diag64[R] = aii;
    dinv64[R] = di;
  }
}

// The coarsest level of a block is its one interior vertex (N = 3).
__global__ void k_sq_coarse(const double* __restrict__ S, int block, int slots,
                            double* __restrict__ cinv) {
  if (threadIdx.x == 0) cinv[(size_t)block * slots + block] = 1.0 / S[4 * kSqSlots];
}

// ----------------------------------------------------- per-block sums ----
// A stacked level-0 vector holds `slots` blocks of m rows.  Grid (chunks,
// slots): block (c, b) sums rows [c R, min((c+1) R, m)) of block b, R =
// kThreads, in a fixed tree; partial[c * slots + b] (the layout k_reduce and
// k_reduce_check read with B = slots).  A block's sums do not depend on the
// other blocks.

// The block's kThreads values summed in a fixed order: a butterfly within
// each warp, then warp 0 adds the kThreads / 32 warp sums the same way.
// Valid in thread 0.
__device__ __forceinline__ double block_tree_sum(double v, double* sh) {
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = lane < kThreads / 32 ? sh[lane] : 0.0;
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;
}

// The per-block norms take kBlkRows rows per thread: a thread adds its
// rows' squares in row order (fma), then the block adds the threads by a
// fixed tree.  B300's FP64 pipe bounds these kernels, and one tree per row
// (ten FP64 shuffle-adds) cost more than the residual itself.  Grid:
// (ceil(m / (kThreads * kBlkRows)), slots); partial[chunk][slot].
constexpr int kBlkRows = 4;

__global__ void __launch_bounds__(kThreads) k_blk_sumsq(const double* __restrict__ x, int m,
                                                        int slots,
                                                        double* __restrict__ partial) {
  pdl_wait();
  __shared__ double sh[kThreads];
  const int b = blockIdx.y;
  const int r0 = blockIdx.x * kThreads * kBlkRows + threadIdx.x;
  double v = 0.0;
#pragma unroll
  for (int k = 0; k < kBlkRows; ++k) {
    const int r = r0 + k * kThreads;
    if (r < m) {
      const double e = x[(size_t)b * m + r];
      v = fma(e, e, v);
    }
  }
  const double s = block_tree_sum(v, sh);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * slots + b] = s;
}

// The rows of one thread of k_blk_resid64.  kP2: rhat = float(r * p2) with
// p2 = 2^e exactly (scale2's in-range form); otherwise scale2 itself.  The
// slot's exponent is uniform, so the choice is one branch per thread and
// the FP64 pipe, which bounds this kernel on B300, never sees the other
// form.
template <bool kP2>
__device__ __forceinline__ double blk_resid_rows(const LV<double>& L, const double* __restrict__ f,
                                                 const double* __restrict__ u,
                                                 float* __restrict__ rhat, int se, double p2,
                                                 int m, int b, int r0, float* __restrict__ d0,
                                                 const float* __restrict__ dinv0, float theta0) {
  double ss = 0.0;
#pragma unroll
  for (int k = 0; k < kBlkRows; ++k) {
    const int r = r0 + k * kThreads;
    if (r < m) {
      const int i = b * m + r;
      const double ax = row_ax(L, i, u, 1, 0);
      const double rv = fma(-L.diag[i], u[i], f[i]) - ax;
      if (rhat) {
        const float rh = (float)(kP2 ? rv * p2 : scale2(rv, se));
        rhat[i] = rh;
        if (d0) d0[i] = theta0 * (rh * dinv0[i]);
      }
      ss = fma(rv, rv, ss);
    }
  }
  return ss;
}

// r = f - A u in FP64 (the arithmetic of k_resid64), rhat = float(2^-sexp_b r)
// (may be NULL), and the block's partial sums of r^2; kBlkRows rows per
// thread, grid as k_blk_sumsq.  d0 (may be NULL): the next FP32 cycle's first
// level-0 smoothing delta, as k_resid64's.
__global__ void __launch_bounds__(kThreads) k_blk_resid64(LV<double> L, const double* __restrict__ f,
                                                          const double* __restrict__ u,
                                                          float* __restrict__ rhat,
                                                          const int* __restrict__ sexp, int m,
                                                          int slots,
                                                          double* __restrict__ partial,
                                                          float* __restrict__ d0,
                                                          const float* __restrict__ dinv0,
                                                          const float* __restrict__ prm0) {
  pdl_wait();
  __shared__ double sh[kThreads];
  const int b = blockIdx.y;
  const int r0 = blockIdx.x * kThreads * kBlkRows + threadIdx.x;
  const int se = rhat ? -sexp[b] : 0;
  const bool p2ok = se >= -1022 && se <= 1023;
  const double p2 = p2ok ? __longlong_as_double((long long)(se + 1023) << 52) : 0.0;
  const float theta0 = d0 ? prm0[P_THETA] : 0.0f;
  const double ss =
      p2ok ? blk_resid_rows<true>(L, f, u, rhat, se, p2, m, b, r0, d0, dinv0, theta0)
           : blk_resid_rows<false>(L, f, u, rhat, se, p2, m, b, r0, d0, dinv0, theta0);
  const double s = block_tree_sum(ss, sh);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * slots + b] = s;
}

// u += 2^sexp_b c on the rows of the blocks still active; iteration counts.
// Grid (chunks of kThreads rows, slots): block b of the stack is blockIdx.y.
__global__ void __launch_bounds__(kThreads) k_blk_refine_update(double* __restrict__ u,
                                                                const float* __restrict__ c,
                                                                const int* __restrict__ sexp,
                                                                const int* __restrict__ active,
                                                                int m, int slots,
                                                                int* __restrict__ iters) {
  pdl_wait();
  const int b = blockIdx.y;
  const int r = blockIdx.x * kThreads + threadIdx.x;
  if (r == 0 && active[b]) iters[b] += 1;
  if (r >= m || !active[b]) return;
  const size_t t = (size_t)b * m + r;
  u[t] += scale2((double)c[t], sexp[b]);
}

// u <- w on the rows of the blocks still active (stationary FP64 solve);
// grid as k_blk_refine_update.
__global__ void __launch_bounds__(kThreads) k_blk_masked_copy(double* __restrict__ u,
                                                              const double* __restrict__ w,
                                                              const int* __restrict__ active,
                                                              int m, int slots,
                                                              int* __restrict__ iters) {
  pdl_wait();
  const int b = blockIdx.y;
  const int r = blockIdx.x * kThreads + threadIdx.x;
  if (r == 0 && active[b]) iters[b] += 1;
  if (r >= m || !active[b]) return;
  const size_t t = (size_t)b * m + r;
  u[t] = w[t];
}

}  // namespace mgk
