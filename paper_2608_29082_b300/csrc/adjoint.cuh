// Adjoint (reverse-mode) kernels of the learnable V-cycle, for training
// (Algorithm 3's "compute gradients via backpropagation").
//
// Notation per level: M = D_g^{-1} A_g is the mean over graph neighbours,
// (M x)_i = invdeg_i sum_{j in N(i)} x_j, and its transpose gathers
// (M^T x)_i = sum_{j in N(i)} invdeg_j x_j (the graph is symmetric).
// A is symmetric (SPD), so A^T = A.  For a step y = g(x; p) with adjoint
// ybar, each kernel produces xbar and the dot products <ybar, dg/dp> that
// make the parameter gradients; the dots are reduced per block in a fixed
// order and summed over blocks in a fixed order (deterministic).
//
// Forward smoothing step (Sec. 3):  r = f - A u,  delta = theta D^{-1} r,
//   u' = u + eta (w1 delta + w2 M delta)
// Adjoint given ubar' (adjoint of u'):
//   phibar = eta ubar',  deltabar = w1 phibar + w2 M^T phibar,
//   rbar = theta D^{-1} deltabar,  ubar = ubar' - A rbar,  fbar += rbar,
//   d eta = <ubar', w1 delta + w2 M delta>, d w1 = eta <ubar', delta>,
//   d w2 = eta <ubar', M delta>,  d theta = <deltabar, D^{-1} r>.
// Restriction r_c = P^T (w1 r + w2 M r), r = f - A u: given rcbar,
//   phibar = P rcbar, rbar = w1 phibar + w2 M^T phibar,
//   d w1 = <phibar, r>, d w2 = <phibar, M r>; then ubar -= A rbar, fbar += rbar.
// Prolongation u' = u + w1 P e + w2 M P e: given ubar',
//   ebar = P^T (w1 ubar' + w2 M^T ubar'),  d w1 = <ubar', P e>,
//   d w2 = <ubar', M P e>.
#pragma once

#include "kernels.cuh"
#include "multi_rhs.cuh"

namespace mgk {

template <class W>
__device__ __forceinline__ W warp_sum(W v) {
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums Q values over the block (fixed order) and writes partial[blk*Q + q].
// Each thread's terms and the sum within a warp are in the context precision
// W; the warp sums and everything after are FP64.  (Forming the terms in FP64
// for an FP32 context put the whole kernel on the B300's FP64 pipe, which
// made it 8x slower than its neighbours.)
template <int Q, class W>
__device__ __forceinline__ void block_dots(const W (&v)[Q], double* __restrict__ partial) {
  __shared__ double sh[Q][kThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const W s = warp_sum(v[q]);
    if (lane == 0) sh[q][warp] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x < Q) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[threadIdx.x][w];
    partial[(size_t)blockIdx.x * Q + threadIdx.x] = s;
  }
}

// grad[idx] += sum_k partial[k*Q + q] by one block of kThreads threads
// (strided per thread, then a fixed tree).
__device__ __forceinline__ void grad_accum_block(const double* __restrict__ partial, int nblk,
                                                 int Q, int q, double* __restrict__ grad,
                                                 int idx) {
  __shared__ double sh[kThreads];
  double s = 0.0;
  for (int k = threadIdx.x; k < nblk; k += kThreads) s += partial[(size_t)k * Q + q];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w >= 1; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) grad[idx] += sh[0];
}

// grad[idx_q] += sum_k partial[k*Q + q]; one block per q.
__global__ void __launch_bounds__(kThreads) k_grad_accum(const double* __restrict__ partial,
                                                         int nblk, int Q, double* __restrict__ grad,
                                                         int i0, int i1, int i2, int i3) {
  const int q = blockIdx.x;
  grad_accum_block(partial, nblk, Q, q, grad, q == 0 ? i0 : q == 1 ? i1 : q == 2 ? i2 : i3);
}

// Parameter-gradient sums folded into the kernel that follows their
// producers: up to two jobs, each the cross-block sum of a dot kernel's
// partials into Q gradient entries (k_grad_accum's work, block by block).
// The host kernel runs its own nwork blocks and Q[0] + Q[1] more, one per
// entry.  Folding saves a launch per job; every entry still receives its
// sums in the order the jobs were issued.
struct GradJobs {
  const double* partial[2];
  int nblk[2], Q[2];
  int idx[2][4];
  int nwork;
  double* grad;
};

// true (and the job's block done) for the extra blocks of a host kernel
__device__ __forceinline__ bool grad_job_block(const GradJobs& a) {
  const int k = (int)blockIdx.x - a.nwork;
  if (k < 0) return false;
  if (k < a.Q[0])
    grad_accum_block(a.partial[0], a.nblk[0], a.Q[0], k, a.grad, a.idx[0][k]);
  else if (k < a.Q[0] + a.Q[1])
    grad_accum_block(a.partial[1], a.nblk[1], a.Q[1], k - a.Q[0], a.grad, a.idx[1][k - a.Q[0]]);
  return true;
}

// sum_{j in N(i)} invdeg_j x_j   (row i of M^T x, without the outer factor)
template <class T>
__device__ __forceinline__ T row_mt(const LV<T>& L, int i, const T* __restrict__ x, int B, int b) {
  T s = T(0);
  for_nb<T, false>(L, i, [&](int c, T, bool nb) {
    const T w = nb ? L.invdeg[c] : T(0);
    s = fma(w, x[(size_t)c * B + b], s);
  });
  return s;
}

// sum_{j in N(i)} dinv_j x_j
template <class T>
__device__ __forceinline__ T row_sum_dinv(const LV<T>& L, int i, const T* __restrict__ x, int B,
                                          int b) {
  T s = T(0);
  for_nb<T, false>(L, i, [&](int c, T, bool nb) {
    const T w = nb ? L.dinv[c] : T(0);
    s = fma(w, x[(size_t)c * B + b], s);
  });
  return s;
}

// Smoothing step, part 1: from ubar' and the step's residual r, write
// rbar = theta D^{-1} deltabar and the dots (eta, w1, w2, theta).
template <class T>
__global__ void __launch_bounds__(kThreads) k_adj_smooth(LV<T> L, const T* __restrict__ ubar,
                                                         const T* __restrict__ r,
                                                         T* __restrict__ rbar, int B,
                                                         const T* __restrict__ prm,
                                                         double* __restrict__ partial) {
  pdl_wait();
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  T v[4] = {T(0), T(0), T(0), T(0)};
  if (t < (size_t)L.n * B) {
    int i, b;
    split_rb(t, B, i, b);
    const T theta = prm[P_THETA], eta = prm[P_ETA], w1 = prm[P_WB1], w2 = prm[P_WB2];
    const T ub = ubar[t];
    const T phib = eta * ub;
    const T mtphib = eta * row_mt(L, i, ubar, B, b);          // M^T phibar
    const T deltab = fma(w1, phib, w2 * mtphib);
    const T dr = L.dinv[i] * r[t];                             // D^{-1} r
    rbar[t] = theta * (L.dinv[i] * deltab);
    const T delta = theta * dr;
    const T mdelta = L.invdeg[i] * (theta * row_sum_dinv(L, i, r, B, b));  // M delta
    v[0] = ub * (w1 * delta + w2 * mdelta);  // d eta
    v[1] = eta * (ub * delta);               // d w1
    v[2] = eta * (ub * mdelta);              // d w2
    v[3] = deltab * dr;                      // d theta
  }
  block_dots<4>(v, partial);
}

// ubar <- ubar - A rbar ; fbar (+)= rbar   (fbar_set: overwrite instead)
template <class T>
__global__ void __launch_bounds__(kThreads) k_adj_apply_a(LV<T> L, T* __restrict__ ubar,
                                                          const T* __restrict__ rbar,
                                                          T* __restrict__ fbar, int B,
                                                          int fbar_set, GradJobs acc) {
  pdl_wait();
  if (grad_job_block(acc)) return;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)L.n * B) return;
  const int i = (int)(t / B), b = (int)(t - (size_t)i * B);
  const T rb = rbar[t];
  if (ubar) {
    const T ax = row_ax(L, i, rbar, B, b);
    ubar[t] = ubar[t] - fma(L.diag[i], rb, ax);
  }
  fbar[t] = fbar_set ? rb : fbar[t] + rb;
}

// Restriction adjoint, fine rows: given pb = P rcbar (fine rows, computed by
// the prolongation kernel), phibar = pb, rbar = w1 phibar + w2 M^T phibar;
// dots (wR1, wR2) with the residual r.
template <class T>
__global__ void __launch_bounds__(kThreads) k_adj_restrict(LV<T> L, const T* __restrict__ pb,
                                                           const T* __restrict__ r,
                                                           T* __restrict__ rbar, int B,
                                                           const T* __restrict__ prm,
                                                           double* __restrict__ partial) {
  pdl_wait();
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  T v[2] = {T(0), T(0)};
  if (t < (size_t)L.n * B) {
    int i, b;
    split_rb(t, B, i, b);
    const T w1 = prm[P_WR1], w2 = prm[P_WR2];
    const T phib = pb[t];
    T mt = T(0), sr = T(0);
    for_nb<T, false>(L, i, [&](int c, T, bool nb) {
      const T w = nb ? L.invdeg[c] : T(0);
      mt = fma(w, pb[(size_t)c * B + b], mt);
      const T rv = r[(size_t)c * B + b];
      sr += nb ? rv : T(0);
    });
    rbar[t] = fma(w1, phib, w2 * mt);
    v[0] = phib * r[t];
    v[1] = phib * (L.invdeg[i] * sr);
  }
  block_dots<2>(v, partial);
}

// Prolongation adjoint, fine rows: g_i = w1 ubar_i + w2 (M^T ubar)_i; the
// coarse adjoint ebar = P^T g is then the restriction gather.
template <class T>
__global__ void __launch_bounds__(kThreads) k_adj_prolong_fine(LV<T> L, const T* __restrict__ ubar,
                                                               T* __restrict__ g, int B,
                                                               const T* __restrict__ prm) {
  pdl_wait();
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)L.n * B) return;
  int i, b;
  split_rb(t, B, i, b);
  const T w1 = prm[P_WP1], w2 = prm[P_WP2];
  g[t] = fma(w1, ubar[t], w2 * row_mt(L, i, ubar, B, b));
}

// Prolongation parameter dots, fine rows: <ubar, P e>, <ubar, M P e>, given
// pe = P e (fine rows, computed by the prolongation kernel).
template <class T>
__global__ void __launch_bounds__(kThreads) k_adj_prolong_dots(LV<T> L, const T* __restrict__ ubar,
                                                               const T* __restrict__ pe, int B,
                                                               double* __restrict__ partial) {
  pdl_wait();
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  T v[2] = {T(0), T(0)};
  if (t < (size_t)L.n * B) {
    int i, b;
    split_rb(t, B, i, b);
    T s = T(0);
    for_nb<T, false>(L, i, [&](int c, T, bool nb) {
      const T pv = pe[(size_t)c * B + b];
      s += nb ? pv : T(0);
    });
    const T ub = ubar[t];
    v[0] = ub * pe[t];
    v[1] = ub * (L.invdeg[i] * s);
  }
  block_dots<2>(v, partial);
}

// Residual loss: r = f - A u; per block, per rhs partial sums of r^2 (the
// batch-independent tiling of k_resid64); optionally keeps r for the gradient.
template <class T>
__global__ void __launch_bounds__(kRedMax) k_loss_resid(LV<T> L, const T* __restrict__ f,
                                                        const T* __restrict__ u, T* __restrict__ r,
                                                        int B, double* __restrict__ partial) {
  __shared__ double sh[kRedMax];
  int i, b;
  bool ok;
  red_tile(L.n, B, i, b, ok);
  double rv = 0.0;
  if (ok) {
    const size_t k = (size_t)i * B + b;
    const T ax = row_ax(L, i, u, B, b);
    const T rr = fma(-L.diag[i], u[k], f[k]) - ax;
    if (r) r[k] = rr;
    rv = (double)rr;
  }
  sh[threadIdx.x] = rv * rv;
  __syncthreads();
  block_rows_reduce32(sh);
  red_store(sh, B, partial);
}

// ubar = -2 w_b A r  (gradient of sum_b w_b ||f_b - A u_b||^2 w.r.t. u)
template <class T>
__global__ void __launch_bounds__(kThreads) k_loss_grad(LV<T> L, const T* __restrict__ r,
                                                        const double* __restrict__ w,
                                                        T* __restrict__ ubar, int B) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)L.n * B) return;
  const int i = (int)(t / B), b = (int)(t - (size_t)i * B);
  const T ar = fma(L.diag[i], r[t], row_ax(L, i, r, B, b));
  ubar[t] = (T)(-2.0 * w[b]) * ar;
}

// loss = sum_b w_b s_b ; per_rhs[b] = s_b (optional)
__global__ void k_loss_combine(const double* __restrict__ s, const double* __restrict__ w, int B,
                               double* __restrict__ loss, double* __restrict__ per_rhs) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double acc = 0.0;
  for (int b = 0; b < B; ++b) {
    if (per_rhs) per_rhs[b] = s[b];
    if (w) acc += w[b] * s[b];
  }
  if (loss) *loss = acc;
}

// Multi-right-hand-side forms (one thread per row and BV consecutive rhs,
// the B / BV threads of a row adjacent, as in multi_rhs.cuh; launch:
// 1-D grid of ceil(n * (B / BV) / kThreads) blocks).  rbar, ubar and fbar
// are computed with the arithmetic of the one-thread-per-(row, rhs) kernels
// above; each thread adds its BV terms of a parameter dot before the block
// sum, so the dots round differently (still in a fixed order).
template <class T, int BV>
__global__ void __launch_bounds__(kThreads) k_adj_smooth_mb(LV<T> L, const T* __restrict__ ubar,
                                                            const T* __restrict__ r,
                                                            T* __restrict__ rbar, int B,
                                                            const T* __restrict__ prm,
                                                            double* __restrict__ partial) {
  pdl_wait();
  const int nq = B / BV;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = g / nq;
  T v[4] = {T(0), T(0), T(0), T(0)};
  if (i < L.n) {
    const int b0 = (g - i * nq) * BV;
    const size_t base = (size_t)i * B + b0;
    const T theta = prm[P_THETA], eta = prm[P_ETA], w1 = prm[P_WB1], w2 = prm[P_WB2];
    T ub[BV], rr[BV], mt[BV], sd[BV], rb[BV];
    ldg<T, BV>(ubar, base, ub);
    ldg<T, BV>(r, base, rr);
#pragma unroll
    for (int b = 0; b < BV; ++b) mt[b] = sd[b] = T(0);
    // M^T ubar and sum_{N(i)} dinv_j r_j, each accumulated in row_mt's and
    // row_sum_dinv's order
    for_nb<T, false, true>(L, i, [&](int c, T, bool nb) {
      const T wm = nb ? L.invdeg[c] : T(0);
      const T wd = nb ? L.dinv[c] : T(0);
      T uc[BV], rc[BV];
      ldg<T, BV>(ubar, (size_t)c * B + b0, uc);
      ldg<T, BV>(r, (size_t)c * B + b0, rc);
#pragma unroll
      for (int b = 0; b < BV; ++b) {
        mt[b] = fma(wm, uc[b], mt[b]);
        sd[b] = fma(wd, rc[b], sd[b]);
      }
    });
    const T di = L.dinv[i], id = L.invdeg[i];
#pragma unroll
    for (int b = 0; b < BV; ++b) {
      const T phib = eta * ub[b];
      const T mtphib = eta * mt[b];
      const T deltab = fma(w1, phib, w2 * mtphib);
      const T dr = di * rr[b];
      rb[b] = theta * (di * deltab);
      const T delta = theta * dr;
      const T mdelta = id * (theta * sd[b]);
      v[0] += ub[b] * (w1 * delta + w2 * mdelta);
      v[1] += eta * (ub[b] * delta);
      v[2] += eta * (ub[b] * mdelta);
      v[3] += deltab * dr;
    }
    stg<T, BV>(rbar, base, rb);
  }
  block_dots<4>(v, partial);
}

// ubar <- ubar - A rbar (when ubar is given); fbar (+)= rbar
template <class T, int BV>
__global__ void __launch_bounds__(kThreads) k_adj_apply_a_mb(LV<T> L, T* __restrict__ ubar,
                                                             const T* __restrict__ rbar,
                                                             T* __restrict__ fbar, int B,
                                                             int fbar_set, GradJobs acc) {
  pdl_wait();
  if (grad_job_block(acc)) return;
  const int nq = B / BV;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = g / nq;
  if (i >= L.n) return;
  const int b0 = (g - i * nq) * BV;
  const size_t base = (size_t)i * B + b0;
  T rb[BV];
  ldg<T, BV>(rbar, base, rb);
  if (ubar) {
    T ax[BV], ub[BV];
    row_ax_mb<T, BV>(L, i, rbar, B, b0, ax);
    ldg<T, BV>(ubar, base, ub);
    const T d = L.diag[i];
#pragma unroll
    for (int b = 0; b < BV; ++b) ub[b] = ub[b] - fma(d, rb[b], ax[b]);
    stg<T, BV>(ubar, base, ub);
  }
  T fb[BV];
  if (fbar_set) {
#pragma unroll
    for (int b = 0; b < BV; ++b) fb[b] = rb[b];
  } else {
    ldg<T, BV>(fbar, base, fb);
#pragma unroll
    for (int b = 0; b < BV; ++b) fb[b] = fb[b] + rb[b];
  }
  stg<T, BV>(fbar, base, fb);
}

}  // namespace mgk
