// Kernels of the flexible conjugate-gradient outer loop (FCG with one stored
// direction) that uses the learnable V-cycle as a variable preconditioner.
// All vectors FP64 [n][B]; per-right-hand-side dot products use the
// batch-independent reduction tiling of kernels.cuh and k_reduce.
#pragma once

#include "kernels.cuh"

namespace mgk {

// Per-block partial sums of NQ dot products per rhs, x_q . y_q, in the
// batch-independent reduction tiling (red_tile): partial[blk][q][b].
template <int NQ>
__global__ void __launch_bounds__(kRedMax) k_dots(const double* __restrict__ x0,
                                                  const double* __restrict__ y0,
                                                  const double* __restrict__ x1,
                                                  const double* __restrict__ y1, int n, int B,
                                                  double* __restrict__ partial) {
  pdl_wait();
  __shared__ double sh[NQ][kRedMax];
  int i, b;
  bool ok;
  red_tile(n, B, i, b, ok);
  const size_t k = (size_t)i * B + b;
  sh[0][threadIdx.x] = ok ? x0[k] * y0[k] : 0.0;
  if (NQ > 1) sh[NQ - 1][threadIdx.x] = ok ? x1[k] * y1[k] : 0.0;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    block_rows_reduce32(sh[q]);
    red_store(sh[q], B, partial + (size_t)blockIdx.x * (NQ - 1) * B + (size_t)q * B);
  }
}

// q = A p (FP64, level 0) and per-block partials of (p, q) and (p, r):
// partial[blk][0][b] = (p, q), partial[blk][1][b] = (p, r).
__global__ void __launch_bounds__(kRedMax) k_spmv_dots(LV<double> L, const double* __restrict__ p,
                                                       const double* __restrict__ r,
                                                       double* __restrict__ q, int B,
                                                       double* __restrict__ partial) {
  pdl_wait();
  __shared__ double sh[2][kRedMax];
  int i, b;
  bool ok;
  red_tile(L.n, B, i, b, ok);
  double pq = 0.0, pr = 0.0;
  if (ok) {
    const size_t k = (size_t)i * B + b;
    const double pk = p[k];
    const double qk = fma(L.diag[i], pk, row_ax(L, i, p, B, b));
    q[k] = qk;
    pq = pk * qk;
    pr = pk * r[k];
  }
  sh[0][threadIdx.x] = pq;
  sh[1][threadIdx.x] = pr;
  __syncthreads();
  block_rows_reduce32(sh[0]);
  block_rows_reduce32(sh[1]);
  red_store(sh[0], B, partial + (size_t)blockIdx.x * B);
  red_store(sh[1], B, partial + (size_t)blockIdx.x * B + B);
}

// alpha_b = (p, r) / (p, q) for the active right-hand sides (else 0).
// sums = [pq(B), pr(B)].
__global__ void k_fcg_alpha(const double* __restrict__ sums, const int* __restrict__ active, int B,
                            double* __restrict__ alpha, double* __restrict__ pq_keep) {
  pdl_wait();
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const double pq = sums[b], pr = sums[B + b];
    alpha[b] = (active[b] && pq != 0.0) ? pr / pq : 0.0;
    pq_keep[b] = pq;
  }
}

// u += alpha p, r -= alpha q for the active right-hand sides; per-block
// partials of r.r (for the convergence test) over all right-hand sides.
__global__ void __launch_bounds__(kRedMax) k_fcg_update(double* __restrict__ u,
                                                        double* __restrict__ r,
                                                        const double* __restrict__ p,
                                                        const double* __restrict__ q,
                                                        const double* __restrict__ alpha,
                                                        const int* __restrict__ active, int n,
                                                        int B, double* __restrict__ partial) {
  pdl_wait();
  __shared__ double sh[kRedMax];
  int i, b;
  bool ok;
  red_tile(n, B, i, b, ok);
  double rr = 0.0;
  if (ok) {
    const size_t k = (size_t)i * B + b;
    double rk = r[k];
    if (active[b]) {
      const double a = alpha[b];
      u[k] = fma(a, p[k], u[k]);
      rk = fma(-a, q[k], rk);
      r[k] = rk;
    }
    rr = rk * rk;
  }
  sh[threadIdx.x] = rr;
  __syncthreads();
  block_rows_reduce32(sh);
  red_store(sh, B, partial);
}

// p = z + beta p with beta_b = -(z, q)/(p, q)_previous; first: p = z.
__global__ void __launch_bounds__(kThreads) k_fcg_direction(double* __restrict__ p,
                                                            const double* __restrict__ z,
                                                            const double* __restrict__ zq,
                                                            const double* __restrict__ pq,
                                                            int n, int B, int first) {
  pdl_wait();
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * B) return;
  const int b = (int)(t % B);
  if (first) {
    p[t] = z[t];
  } else {
    const double beta = pq[b] != 0.0 ? -zq[b] / pq[b] : 0.0;
    p[t] = fma(beta, p[t], z[t]);
  }
}

// rhat = float(r * 2^-sexp[b]) (preconditioner input of an FP32 cycle).
__global__ void __launch_bounds__(kThreads) k_scale_to_f32(const double* __restrict__ r,
                                                           const int* __restrict__ sexp,
                                                           float* __restrict__ rhat, int n, int B) {
  pdl_wait();
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * B) return;
  rhat[t] = (float)scale2(r[t], -sexp[t % B]);
}

// z = 2^sexp[b] * c (preconditioner output back in FP64).
__global__ void __launch_bounds__(kThreads) k_scale_from_f32(const float* __restrict__ c,
                                                             const int* __restrict__ sexp,
                                                             double* __restrict__ z, int n, int B) {
  pdl_wait();
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * B) return;
  z[t] = scale2((double)c[t], sexp[t % B]);
}

}  // namespace mgk
