// Kernels of restarted flexible GMRES, FGMRES(m), with right preconditioning
// (Saad 1993): the outer Krylov method the paper pairs with its V-cycle and
// full-multigrid preconditioners (Sec. 4.2, tab:helmholtz-results-precond).
// Vectors are [n][B]; the Arnoldi basis V_0..V_m and the preconditioned directions Z_0..Z_{m-1} are stored
// vstride = n * B apart.  Orthogonalisation is classical Gram-Schmidt
// applied twice (CGS2): each pass forms all dot products from the same
// vector, so a step needs two multi-dot reductions instead of j + 1
// dependent ones.  All reductions group their terms independently of the
// batch (k_gm_dots below, k_reduce), so each right-hand side's iteration
// does not depend on what else is in the batch.
//
// Vector type T: double in an FP64 context.  In an FP32 context the whole
// Arnoldi cycle (basis, directions, operator, Gram-Schmidt) is FP32 and only
// the restart (true residual, u += Z y) is FP64: B300's FP64 pipe (about
// 0.6 T FMA/s) would bound CGS2's 4 (j + 1) multiply-adds per entry and
// step, while FP32 runs at the memory rate.  The Hessenberg problem is FP64
// throughout.
//
// Per right-hand side b, small[b * gm_stride(m)] holds
//   H  (m+1) x m Hessenberg matrix, column j at j * (m + 1)
//   cs, sn  the m Givens rotations
//   g  the rotated right-hand side of the least-squares problem, m + 1
//   y  its solution at the end of a cycle, m
//   beta  the cycle's initial residual norm
#pragma once

#include "kernels.cuh"

namespace mgk {

__host__ __device__ inline int gm_stride(int m) { return m * (m + 1) + 4 * m + 2; }

// The Gram-Schmidt kernels stream the whole basis once per pass.  A block
// covers kGmTile = 256 rows and bt = min(B, 16) right-hand-side columns
// (blockDim = 32 * bt); thread (r, c) owns rows base + r + 32 k, k <
// kGmRows, of column c.  Loads use clamped in-range addresses (their values
// are masked afterwards) so that all kGmRows * kGmQ of a round are issued
// before the arithmetic; w and the first round are issued together, and
// each next round is issued before the current round's reduction tree.
// Each thread sums its rows in k order and the 32 row-threads of a column
// are added by a fixed tree, so a right-hand side's results do not depend
// on the batch.  partial[blk][q][b] as read by k_reduce (nblk = ceil(n /
// 256)).
constexpr int kGmRows = 8;
constexpr int kGmQ = 4;
constexpr int kGmTile = kRedRows * kGmRows;
constexpr int kGmBt = 16;
constexpr int kGmThreads = kRedRows * kGmBt;

struct GmTile {
  int bt, t, r, b, bc;  // bc: b clamped into [0, B)
  bool okb;
  int i0;
  __device__ GmTile(int B) {
    bt = blockDim.x / kRedRows;
    t = threadIdx.x;
    r = t / bt;
    b = blockIdx.y * bt + t % bt;
    okb = b < B;
    bc = okb ? b : B - 1;
    i0 = blockIdx.x * kGmTile + r;
  }
  // clamped element offset of row k of this thread, and whether it is real
  __device__ size_t off(int k, int n, int B) const {
    return (size_t)min(i0 + k * kRedRows, n - 1) * B + bc;
  }
  __device__ bool ok(int k, int n) const { return okb && i0 + k * kRedRows < n; }
};

// Right-hand side of entry t of an [n][B] vector (32-bit modulo when the
// vector has fewer than 2^32 entries).
__device__ __forceinline__ int gm_col(size_t t, int n, int B) {
  return (size_t)n * B <= 0xffffffffull ? (int)((unsigned)t % (unsigned)B) : (int)(t % B);
}

// sh[qq][r * bt + c] summed over the 32 rows r into sh[qq][c], qq < nv
template <class T>
__device__ __forceinline__ void gm_rows_reduce(T (*sh)[kGmThreads], int nv) {
  const int bt = blockDim.x / kRedRows;
  const int t = threadIdx.x;
  const int r = t / bt;
  for (int s = kRedRows / 2; s >= 1; s >>= 1) {
    if (r < s)
      for (int qq = 0; qq < nv; ++qq) sh[qq][t] += sh[qq][t + s * bt];
    __syncthreads();
  }
}

// v[qq][k] = V_{min(q0 + qq, nq - 1)} at this thread's clamped row k
template <class T>
__device__ __forceinline__ void gm_load_round(const GmTile& g, const T* __restrict__ V,
                                              size_t vstride, int q0, int nq, int n, int B,
                                              T (&v)[kGmQ][kGmRows]) {
#pragma unroll
  for (int qq = 0; qq < kGmQ; ++qq) {
    const T* Vq = V + (size_t)min(q0 + qq, nq - 1) * vstride;
#pragma unroll
    for (int k = 0; k < kGmRows; ++k) v[qq][k] = Vq[g.off(k, n, B)];
  }
}

// partial[blk][q][b] = the block's rows of V_q . w, q < nq (sums in T)
template <class T>
__global__ void __launch_bounds__(kGmThreads) k_gm_dots(const T* __restrict__ V, size_t vstride,
                                                        const T* __restrict__ w, int nq, int n,
                                                        int B, double* __restrict__ partial) {
  pdl_wait();
  __shared__ T sh[kGmQ][kGmThreads];
  const GmTile g(B);
  T wk[kGmRows];
#pragma unroll
  for (int k = 0; k < kGmRows; ++k) wk[k] = w[g.off(k, n, B)];
  T v[kGmQ][kGmRows];
  gm_load_round(g, V, vstride, 0, nq, n, B, v);
#pragma unroll
  for (int k = 0; k < kGmRows; ++k) wk[k] = g.ok(k, n) ? wk[k] : T(0);
  for (int q0 = 0; q0 < nq; q0 += kGmQ) {
    const int nv = min(kGmQ, nq - q0);
#pragma unroll
    for (int qq = 0; qq < kGmQ; ++qq) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < kGmRows; ++k) acc = fma(v[qq][k], wk[k], acc);
      sh[qq][g.t] = acc;
    }
    if (q0 + kGmQ < nq) gm_load_round(g, V, vstride, q0 + kGmQ, nq, n, B, v);
    __syncthreads();
    gm_rows_reduce(sh, nv);
    if (g.r == 0 && g.okb)
      for (int qq = 0; qq < nv; ++qq)
        partial[((size_t)blockIdx.x * nq + q0 + qq) * B + g.b] = (double)sh[qq][g.t];
    __syncthreads();
  }
}

// w -= sum_{q < nq} h[q][b] V_q (q in order); partial[blk][b] of |w|^2
template <class T>
__global__ void __launch_bounds__(kGmThreads) k_gm_orth(const T* __restrict__ V, size_t vstride,
                                                        T* __restrict__ w,
                                                        const double* __restrict__ h, int nq,
                                                        int n, int B,
                                                        double* __restrict__ partial) {
  pdl_wait();
  __shared__ T sh[1][kGmThreads];
  const GmTile g(B);
  T wk[kGmRows];
#pragma unroll
  for (int k = 0; k < kGmRows; ++k) wk[k] = w[g.off(k, n, B)];
  T v[kGmQ][kGmRows];
  gm_load_round(g, V, vstride, 0, nq, n, B, v);
  for (int q0 = 0; q0 < nq; q0 += kGmQ) {
    T hq[kGmQ];
#pragma unroll
    for (int qq = 0; qq < kGmQ; ++qq) hq[qq] = (T)h[(size_t)min(q0 + qq, nq - 1) * B + g.bc];
#pragma unroll
    for (int qq = 0; qq < kGmQ; ++qq) {
      const bool live = q0 + qq < nq;
#pragma unroll
      for (int k = 0; k < kGmRows; ++k) wk[k] = live ? fma(-hq[qq], v[qq][k], wk[k]) : wk[k];
    }
    if (q0 + kGmQ < nq) gm_load_round(g, V, vstride, q0 + kGmQ, nq, n, B, v);
  }
  T ss = T(0);
#pragma unroll
  for (int k = 0; k < kGmRows; ++k) {
    if (g.ok(k, n)) {
      w[g.off(k, n, B)] = wk[k];
      ss = fma(wk[k], wk[k], ss);
    }
  }
  sh[0][g.t] = ss;
  __syncthreads();
  gm_rows_reduce(sh, 1);
  if (g.r == 0 && g.okb) partial[(size_t)blockIdx.x * B + g.b] = (double)sh[0][g.t];
}

// Restart: beta = ||r||, relres = beta / ||f||; right-hand sides whose
// relres met tol (or is not finite) leave the active set; g = beta e_1;
// inv = 1 / beta (v_0 = r * inv); every right-hand side starts the cycle
// (done = 0).  state[0] = active count, state[1] = 1 if a residual is not
// finite.  One block.
__global__ void k_gm_restart(const double* __restrict__ rsum, const double* __restrict__ fsum,
                             const double* __restrict__ ctl, int m, int B, int* __restrict__ active,
                             double* __restrict__ relres, double* __restrict__ small,
                             double* __restrict__ inv, int* __restrict__ done,
                             int* __restrict__ state) {
  pdl_wait();
  __shared__ int cnt, bad;
  if (threadIdx.x == 0) { cnt = 0; bad = 0; }
  __syncthreads();
  const double tol = ctl[0];
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const double beta = sqrt(rsum[b]), fn = sqrt(fsum[b]);
    const double rel = fn > 0.0 ? beta / fn : beta;
    relres[b] = rel;
    if (!isfinite(rel)) atomicAdd(&bad, 1);
    if (active[b] && !(rel < tol) && isfinite(rel)) atomicAdd(&cnt, 1);
    else active[b] = 0;
    double* sb = small + (size_t)b * gm_stride(m);
    double* g = sb + m * (m + 1) + 2 * m;
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    sb[m * (m + 1) + 4 * m + 1] = beta;
    inv[b] = beta > 0.0 && isfinite(beta) ? 1.0 / beta : 0.0;
    done[b] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    state[0] = cnt;
    state[1] = bad;
  }
}

// Arnoldi step j: column j of H = h1 + h2 (the two Gram-Schmidt passes) and
// ||w||, the previous rotations applied, a new rotation, the residual
// estimate |g_{j+1}| / ||f||.  inv = 1 / ||w|| (v_{j+1} = w * inv).  A
// right-hand side still in its cycle counts the step; it finishes the cycle
// (done = j + 1, the columns it uses) when the estimate meets tol, is not
// finite, or |g_{j+1}| < rho * beta (rho > 0: the accuracy an FP32 cycle
// can resolve; the restart's FP64 residual continues from there).
// state[3] = right-hand sides still in their cycle.  One block.
__global__ void k_gm_arnoldi(double* __restrict__ small, const double* __restrict__ h1,
                             const double* __restrict__ h2, const double* __restrict__ wn,
                             const double* __restrict__ fsum, const double* __restrict__ ctl, int m,
                             int j, int B, double rho, const int* __restrict__ active,
                             int* __restrict__ iters, double* __restrict__ inv,
                             double* __restrict__ relres, int* __restrict__ done,
                             int* __restrict__ state) {
  pdl_wait();
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  const double tol = ctl[0];
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    double* sb = small + (size_t)b * gm_stride(m);
    double* cs = sb + m * (m + 1);
    double* sn = cs + m;
    double* g = sn + m;
    const double beta = sb[m * (m + 1) + 4 * m + 1];
    double* Hj = sb + (size_t)j * (m + 1);
    for (int i = 0; i <= j; ++i) Hj[i] = h1[(size_t)i * B + b] + h2[(size_t)i * B + b];
    const double hn = sqrt(wn[b]);
    Hj[j + 1] = hn;
    inv[b] = hn > 0.0 && isfinite(hn) ? 1.0 / hn : 0.0;
    for (int i = 0; i < j; ++i) {
      const double t = cs[i] * Hj[i] + sn[i] * Hj[i + 1];
      Hj[i + 1] = -sn[i] * Hj[i] + cs[i] * Hj[i + 1];
      Hj[i] = t;
    }
    const double a = Hj[j], c2 = Hj[j + 1];
    const double r = sqrt(a * a + c2 * c2);
    cs[j] = r > 0.0 ? a / r : 1.0;
    sn[j] = r > 0.0 ? c2 / r : 0.0;
    Hj[j] = r;
    Hj[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    if (active[b] && !done[b]) {
      const double fn = sqrt(fsum[b]);
      const double est = fn > 0.0 ? fabs(g[j + 1]) / fn : fabs(g[j + 1]);
      iters[b] += 1;
      relres[b] = est;
      if (est < tol || !isfinite(est) || fabs(g[j + 1]) < rho * beta) done[b] = j + 1;
      else atomicAdd(&cnt, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) state[3] = cnt;
}

// End of a cycle of jl + 1 steps: y = H^{-1} g by back substitution (upper
// triangular after the rotations) over the columns the right-hand side
// used (done, else jl + 1); y = 0 beyond them.  One block.
__global__ void k_gm_solve_y(double* __restrict__ small, int m, int jl, int B,
                             const int* __restrict__ active, const int* __restrict__ done) {
  pdl_wait();
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    if (!active[b]) continue;
    double* sb = small + (size_t)b * gm_stride(m);
    const double* g = sb + m * (m + 1) + 2 * m;
    double* y = sb + m * (m + 1) + 3 * m + 1;
    const int jb = done[b] ? min(done[b] - 1, jl) : jl;
    for (int i = jl; i > jb; --i) y[i] = 0.0;
    for (int i = jb; i >= 0; --i) {
      double t = g[i];
      for (int k = i + 1; k <= jb; ++k) t -= sb[(size_t)k * (m + 1) + i] * y[k];
      const double d = sb[(size_t)i * (m + 1) + i];
      y[i] = d != 0.0 ? t / d : 0.0;
    }
  }
}

// u += sgn * sum_{q < nq} y_q Z_q for the active right-hand sides (FP64 u)
template <class T>
__global__ void __launch_bounds__(kThreads) k_gm_update(double* __restrict__ u,
                                                        const T* __restrict__ Z, size_t vstride,
                                                        const double* __restrict__ small, int m,
                                                        int nq, double sgn,
                                                        const int* __restrict__ active, int n,
                                                        int B) {
  pdl_wait();
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * B) return;
  const int b = gm_col(t, n, B);
  if (!active[b]) return;
  const double* y = small + (size_t)b * gm_stride(m) + m * (m + 1) + 3 * m + 1;
  double acc = 0.0;
#pragma unroll 4
  for (int q = 0; q < nq; ++q) acc = fma(y[q], (double)Z[(size_t)q * vstride + t], acc);
  u[t] = fma(sgn, acc, u[t]);
}

// v = w * inv[b] (v may be w), rounded to V's type
template <class T, class V>
__global__ void __launch_bounds__(kThreads) k_gm_scale(const T* w, const double* __restrict__ inv,
                                                       V* v, int n, int B) {
  pdl_wait();
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * B) return;
  v[t] = (V)(w[t] * (T)inv[gm_col(t, n, B)]);
}

}  // namespace mgk
