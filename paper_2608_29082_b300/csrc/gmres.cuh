// Kernels of restarted flexible GMRES, FGMRES(m), with right preconditioning
// (Saad 1993): the outer Krylov method the paper pairs with its V-cycle and
// full-multigrid preconditioners (Sec. 5).  Vectors are FP64 [n][B]; the
// Arnoldi basis V_0..V_m and the preconditioned directions Z_0..Z_{m-1} are
// stored vstride = n * B apart.  Orthogonalisation is classical Gram-Schmidt
// applied twice (CGS2): each pass forms all dot products from the same
// vector, so a step needs two multi-dot reductions instead of j + 1
// dependent ones.  Dots use the batch-independent reduction tiling of
// kernels.cuh (red_tile) and k_reduce, so each right-hand side's iteration
// does not depend on the batch.
//
// Per right-hand side b, small[b * gm_stride(m)] holds
//   H  (m+1) x m Hessenberg matrix, column j at j * (m + 1)
//   cs, sn  the m Givens rotations
//   g  the rotated right-hand side of the least-squares problem, m + 1
//   y  its solution at the end of a cycle, m
#pragma once

#include "kernels.cuh"

namespace mgk {

__host__ __device__ inline int gm_stride(int m) { return m * (m + 1) + 4 * m + 1; }

// partial[blk][q][b] = the block's rows of V_q . w, q < nq
__global__ void __launch_bounds__(kRedMax) k_gm_dots(const double* __restrict__ V, size_t vstride,
                                                     const double* __restrict__ w, int nq, int n,
                                                     int B, double* __restrict__ partial) {
  pdl_wait();
  __shared__ double sh[kRedMax];
  int i, b;
  bool ok;
  red_tile(n, B, i, b, ok);
  const size_t k = (size_t)i * B + b;
  const double wk = ok ? w[k] : 0.0;
  for (int q = 0; q < nq; ++q) {
    sh[threadIdx.x] = ok ? V[(size_t)q * vstride + k] * wk : 0.0;
    __syncthreads();
    block_rows_reduce32(sh);
    red_store(sh, B, partial + (size_t)blockIdx.x * (nq - 1) * B + (size_t)q * B);
    __syncthreads();
  }
}

// w -= sum_{q < nq} h[q][b] V_q (fixed q order); partial[blk][b] of |w|^2
__global__ void __launch_bounds__(kRedMax) k_gm_orth(const double* __restrict__ V, size_t vstride,
                                                     double* __restrict__ w,
                                                     const double* __restrict__ h, int nq, int n,
                                                     int B, double* __restrict__ partial) {
  pdl_wait();
  __shared__ double sh[kRedMax];
  int i, b;
  bool ok;
  red_tile(n, B, i, b, ok);
  double wk = 0.0;
  if (ok) {
    const size_t k = (size_t)i * B + b;
    wk = w[k];
    for (int q = 0; q < nq; ++q) wk = fma(-h[(size_t)q * B + b], V[(size_t)q * vstride + k], wk);
    w[k] = wk;
  }
  sh[threadIdx.x] = wk * wk;
  __syncthreads();
  block_rows_reduce32(sh);
  red_store(sh, B, partial);
}

// Restart: beta = ||r||, relres = beta / ||f||; right-hand sides whose
// relres met tol (or is not finite) leave the active set; g = beta e_1;
// inv = 1 / beta (v_0 = r * inv).  state[0] = active count, state[1] = 1 if
// a residual is not finite.  One block.
__global__ void k_gm_restart(const double* __restrict__ rsum, const double* __restrict__ fsum,
                             const double* __restrict__ ctl, int m, int B, int* __restrict__ active,
                             double* __restrict__ relres, double* __restrict__ small,
                             double* __restrict__ inv, int* __restrict__ state) {
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
    double* g = small + (size_t)b * gm_stride(m) + m * (m + 1) + 2 * m;
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    inv[b] = beta > 0.0 && isfinite(beta) ? 1.0 / beta : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    state[0] = cnt;
    state[1] = bad;
  }
}

// Arnoldi step j: column j of H = h1 + h2 (the two Gram-Schmidt passes) and
// ||w||, the previous rotations applied, a new rotation, the residual
// estimate |g_{j+1}| / ||f||.  inv = 1 / ||w|| (v_{j+1} = w * inv).  Counts
// the step for every active right-hand side not yet below tol in this cycle;
// state[3] = those still >= tol after it.  One block.
__global__ void k_gm_arnoldi(double* __restrict__ small, const double* __restrict__ h1,
                             const double* __restrict__ h2, const double* __restrict__ wn,
                             const double* __restrict__ fsum, const double* __restrict__ ctl, int m,
                             int j, int B, const int* __restrict__ active, int* __restrict__ iters,
                             double* __restrict__ inv, double* __restrict__ relres,
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
    // a right-hand side whose estimate met tol earlier in this cycle rides
    // along until the cycle ends but is not counted (relres holds its
    // estimate at that step; at a restart, its true relres >= tol)
    if (active[b] && !(relres[b] < tol)) {
      const double fn = sqrt(fsum[b]);
      const double est = fn > 0.0 ? fabs(g[j + 1]) / fn : fabs(g[j + 1]);
      iters[b] += 1;
      relres[b] = est;
      if (!(est < tol) && isfinite(est)) atomicAdd(&cnt, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) state[3] = cnt;
}

// End of a cycle with jl + 1 directions: y = H^{-1} g by back substitution
// (upper triangular after the rotations), active right-hand sides.  One block.
__global__ void k_gm_solve_y(double* __restrict__ small, int m, int jl, int B,
                             const int* __restrict__ active) {
  pdl_wait();
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    if (!active[b]) continue;
    double* sb = small + (size_t)b * gm_stride(m);
    const double* g = sb + m * (m + 1) + 2 * m;
    double* y = sb + m * (m + 1) + 3 * m + 1;
    for (int i = jl; i >= 0; --i) {
      double t = g[i];
      for (int k = i + 1; k <= jl; ++k) t -= sb[(size_t)k * (m + 1) + i] * y[k];
      const double d = sb[(size_t)i * (m + 1) + i];
      y[i] = d != 0.0 ? t / d : 0.0;
    }
  }
}

// u += sum_{q < nq} y_q Z_q for the active right-hand sides
__global__ void __launch_bounds__(kThreads) k_gm_update(double* __restrict__ u,
                                                        const double* __restrict__ Z,
                                                        size_t vstride,
                                                        const double* __restrict__ small, int m,
                                                        int nq, const int* __restrict__ active,
                                                        int n, int B) {
  pdl_wait();
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * B) return;
  const int b = (int)(t % B);
  if (!active[b]) return;
  const double* y = small + (size_t)b * gm_stride(m) + m * (m + 1) + 3 * m + 1;
  double acc = u[t];
  for (int q = 0; q < nq; ++q) acc = fma(y[q], Z[(size_t)q * vstride + t], acc);
  u[t] = acc;
}

// v = w * inv[b] (v may be w)
__global__ void __launch_bounds__(kThreads) k_gm_scale(const double* w,
                                                       const double* __restrict__ inv, double* v,
                                                       int n, int B) {
  pdl_wait();
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * B) return;
  v[t] = w[t] * inv[t % B];
}

}  // namespace mgk
