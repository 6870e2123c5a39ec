// Kernels of the flexible conjugate-gradient outer loop (FCG with one stored
// direction) that uses the learnable V-cycle as a variable preconditioner.
// All vectors FP64 [n][B]; per-right-hand-side dot products use the
// batch-independent reduction tiling of kernels.cuh and k_reduce.
#pragma once

#include "kernels.cuh"
#include "multi_rhs.cuh"

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

// ---------------------------------------------------------------------------
// FCG with FP32 vectors in a precision-32 context (the Krylov counterpart of
// the FP32 cycle inside FP64 refinement).  An inner FCG(1) phase solves the
// scaled correction equation A e = rhat, rhat = 2^-s r, with FP32 vectors
// r, z, p, q, e and the context's FP32 operator; when its recurrence
// residual has fallen by the floor factor, or its scaled estimate says the
// tolerance may be met, or the last iteration comes, the phase ends for that
// right-hand side: u += 2^s e in FP64, the true residual f - A u is formed in
// FP64 and tested, and a new phase starts from it with a fresh direction.
// Only those restarts decide convergence.
//
// Reductions: a block covers 32 x kF32Rows rows and bt = min(B, 32)
// right-hand sides; thread (g, b) (g = threadIdx.x / bt) owns rows
// blk * 32 kF32Rows + g + 32 k, k < kF32Rows, sums its products in that
// order in FP32, and the block sums its 32 row groups with the fixed tree of
// block_rows_reduce32 in FP64.  The grouping depends on the rows only, so
// every right-hand side's sums are the same whatever else is in the batch.
// ---------------------------------------------------------------------------

constexpr int kF32Rows = 8;
constexpr int kF32BlockRows = kRedRows * kF32Rows;

// Row group g, right-hand side b of this thread, first row of the block.
__device__ __forceinline__ void f32_tile(int B, int& g, int& b, int& i0) {
  const int bt = blockDim.x / kRedRows;
  g = threadIdx.x / bt;
  b = blockIdx.y * bt + threadIdx.x % bt;
  i0 = blockIdx.x * kF32BlockRows + g;
}

// partial[blk][b] = sum of x_ib * y_ib over the block's rows.
__global__ void __launch_bounds__(kRedMax) k32_dot(const float* __restrict__ x,
                                                   const float* __restrict__ y, int n, int B,
                                                   double* __restrict__ partial) {
  pdl_wait();
  __shared__ double sh[kRedMax];
  int g, b, i0;
  f32_tile(B, g, b, i0);
  float acc = 0.0f;
  if (b < B) {
#pragma unroll
    for (int k = 0; k < kF32Rows; ++k) {
      const int i = i0 + kRedRows * k;
      if (i < n) {
        const size_t t = (size_t)i * B + b;
        acc = fmaf(x[t], y[t], acc);
      }
    }
  }
  sh[threadIdx.x] = (double)acc;
  __syncthreads();
  block_rows_reduce32(sh);
  red_store(sh, B, partial);
}

// p = z for a fresh direction, else p = z + beta_b p (beta from
// k32_reduce_beta); rows of the f32 tiling.
__global__ void __launch_bounds__(kRedMax) k32_direction(float* __restrict__ p,
                                                         const float* __restrict__ z,
                                                         const double* __restrict__ beta,
                                                         const int* __restrict__ fresh, int n,
                                                         int B) {
  pdl_wait();
  int g, b, i0;
  f32_tile(B, g, b, i0);
  if (b >= B) return;
  const bool f = fresh[b] != 0;
  const float be = (float)beta[b];
#pragma unroll
  for (int k = 0; k < kF32Rows; ++k) {
    const int i = i0 + kRedRows * k;
    if (i < n) {
      const size_t t = (size_t)i * B + b;
      p[t] = f ? z[t] : fmaf(be, p[t], z[t]);
    }
  }
}

// q = A p with the FP32 operator, partials of (p, q) and (p, r):
// partial[2 blk][b] = (p, q), partial[2 blk + 1][b] = (p, r).
__global__ void __launch_bounds__(kRedMax) k32_spmv_dots(LV<float> L, const float* __restrict__ p,
                                                         const float* __restrict__ r,
                                                         float* __restrict__ q, int B,
                                                         double* __restrict__ partial) {
  pdl_wait();
  __shared__ double sh[2][kRedMax];
  int g, b, i0;
  f32_tile(B, g, b, i0);
  float pq = 0.0f, pr = 0.0f;
  if (b < B) {
#pragma unroll 2
    for (int k = 0; k < kF32Rows; ++k) {
      const int i = i0 + kRedRows * k;
      if (i < L.n) {
        const size_t t = (size_t)i * B + b;
        const float pk = p[t];
        const float qk = fmaf(L.diag[i], pk, row_ax(L, i, p, B, b));
        q[t] = qk;
        pq = fmaf(pk, qk, pq);
        pr = fmaf(pk, r[t], pr);
      }
    }
  }
  sh[0][threadIdx.x] = (double)pq;
  sh[1][threadIdx.x] = (double)pr;
  __syncthreads();
  block_rows_reduce32(sh[0]);
  block_rows_reduce32(sh[1]);
  red_store(sh[0], B, partial + (size_t)blockIdx.x * B);
  red_store(sh[1], B, partial + (size_t)blockIdx.x * B + B);
}

// k32_spmv_dots with right-hand-side tiles: thread (g, tile) owns the rows
// of row group g and BV consecutive right-hand sides (BV | B, BV | 32), so a
// row's matrix entries are read once per BV columns and its neighbours'
// values in 32-byte pieces (row_ax_mb) instead of once per column.  Every
// (row, rhs) value and every per-column sum is computed in the order of
// k32_spmv_dots, so the results are the same.
// The rows are read with the launch-wide 32-byte alignment answer of
// multi_rhs.cuh (mb_aligned).  For BV = 8 eight blocks per SM are asked of
// the compiler: its former 64 registers (a small spill) instead of 70 and
// one block fewer; the 16-rhs L-shape FCG solves took 1-2 % less time.
template <int BV>
__global__ void __launch_bounds__(kRedRows * 32 / BV, BV == 8 ? 8 : 1) k32_spmv_dots_mb(LV<float> L,
                                                            const float* __restrict__ p,
                                                            const float* __restrict__ r,
                                                            float* __restrict__ q, int B,
                                                            double* __restrict__ partial) {
  pdl_wait();
  __shared__ double sh[2][kRedMax];
  const int nt = blockDim.x / kRedRows;  // tiles per row group
  const int bt = nt * BV;                 // right-hand sides of this block column
  const int g = threadIdx.x / nt;
  const int tile = threadIdx.x - g * nt;
  const int b0 = blockIdx.y * bt + tile * BV;
  float pq[BV], pr[BV];
#pragma unroll
  for (int j = 0; j < BV; ++j) pq[j] = pr[j] = 0.0f;
  auto body = [&](auto A) {
    constexpr int kA = decltype(A)::value;
    if (b0 < B) {
      const int i0 = blockIdx.x * kF32BlockRows + g;
#pragma unroll 1
      for (int k = 0; k < kF32Rows; ++k) {
        const int i = i0 + kRedRows * k;
        if (i >= L.n) break;
        const size_t base = (size_t)i * B + b0;
        float pv[BV], ax[BV];
        row_ax_mb<float, BV, kA>(L, i, p, B, b0, ax);
        ldg<float, BV, kA>(p, base, pv);
        const float d = L.diag[i];
#pragma unroll
        for (int j = 0; j < BV; ++j) {
          ax[j] = fmaf(d, pv[j], ax[j]);  // q
          pq[j] = fmaf(pv[j], ax[j], pq[j]);
        }
        stg<float, BV, kA>(q, base, ax);
        ldg<float, BV, kA>(r, base, ax);  // r, in the registers q no longer needs
#pragma unroll
        for (int j = 0; j < BV; ++j) pr[j] = fmaf(pv[j], ax[j], pr[j]);
      }
    }
  };
  if (mb_aligned<float>(B, p, q, r))
    body(std::integral_constant<int, 1>{});
  else
    body(std::integral_constant<int, 0>{});
  // column c of the block is right-hand side blockIdx.y * bt + c; row g of
  // sh[w] holds row group g's sums (the layout block_rows_reduce32 uses)
#pragma unroll
  for (int j = 0; j < BV; ++j) {
    sh[0][g * bt + tile * BV + j] = (double)pq[j];
    sh[1][g * bt + tile * BV + j] = (double)pr[j];
  }
  __syncthreads();
  for (int s = kRedRows / 2; s >= 1; s >>= 1) {
    for (int e = threadIdx.x; e < 2 * s * bt; e += blockDim.x) {
      const int w = e / (s * bt), x = e - w * s * bt;
      sh[w][x] += sh[w][x + s * bt];
    }
    __syncthreads();
  }
  for (int c = threadIdx.x; c < bt; c += blockDim.x) {
    const int b = blockIdx.y * bt + c;
    if (b < B) {
      partial[(size_t)blockIdx.x * 2 * B + b] = sh[0][c];
      partial[(size_t)blockIdx.x * 2 * B + B + b] = sh[1][c];
    }
  }
}

// e += alpha_b p, r -= alpha_b q for the right-hand sides in a phase;
// partials of r.r.
__global__ void __launch_bounds__(kRedMax) k32_fcg_update(float* __restrict__ e,
                                                          float* __restrict__ r,
                                                          const float* __restrict__ p,
                                                          const float* __restrict__ q,
                                                          const double* __restrict__ alpha,
                                                          const int* __restrict__ active, int n,
                                                          int B, double* __restrict__ partial) {
  pdl_wait();
  __shared__ double sh[kRedMax];
  int g, b, i0;
  f32_tile(B, g, b, i0);
  float rr = 0.0f;
  if (b < B) {
    const bool on = active[b] != 0;
    const float a = (float)alpha[b];
#pragma unroll
    for (int k = 0; k < kF32Rows; ++k) {
      const int i = i0 + kRedRows * k;
      if (i < n) {
        const size_t t = (size_t)i * B + b;
        float rk = r[t];
        if (on) {
          e[t] = fmaf(a, p[t], e[t]);
          rk = fmaf(-a, q[t], rk);
          r[t] = rk;
        }
        rr = fmaf(rk, rk, rr);
      }
    }
  }
  sh[threadIdx.x] = (double)rr;
  __syncthreads();
  block_rows_reduce32(sh);
  red_store(sh, B, partial);
}

// One block per right-hand side b: zq = the sum of its (z, q) partials,
// beta_b = -zq / (p, q)_previous (0 for a fresh direction).
__global__ void __launch_bounds__(kThreads) k32_reduce_beta(const double* __restrict__ partial,
                                                            int nblk, int B,
                                                            const double* __restrict__ pq,
                                                            const int* __restrict__ fresh,
                                                            double* __restrict__ beta) {
  pdl_wait();
  __shared__ double sh[kThreads];
  const int b = blockIdx.x;
  const double zq = block_sum_partials(partial, nblk, B, b, sh);
  if (threadIdx.x == 0) beta[b] = (fresh[b] || pq[b] == 0.0) ? 0.0 : -zq / pq[b];
}

// One block per right-hand side b: (p, q) and (p, r) from k32_spmv_dots'
// partials (read as 2B columns), alpha_b = (p, r)/(p, q) in a phase (else 0);
// keeps (p, q) for the next beta and ends the fresh state of b.
__global__ void __launch_bounds__(kThreads) k32_reduce_alpha(const double* __restrict__ partial,
                                                             int nblk, int B,
                                                             const int* __restrict__ active,
                                                             double* __restrict__ alpha,
                                                             double* __restrict__ pq,
                                                             int* __restrict__ fresh) {
  pdl_wait();
  __shared__ double sh[kThreads];
  const int b = blockIdx.x;
  const double sq = block_sum_partials(partial, nblk, 2 * B, b, sh);
  const double sr = block_sum_partials(partial, nblk, 2 * B, B + b, sh);
  if (threadIdx.x == 0) {
    alpha[b] = (active[b] && sq != 0.0) ? sr / sq : 0.0;
    pq[b] = sq;
    fresh[b] = 0;
  }
}

// One block per right-hand side b after the update: rr = ||r_b||^2 of the
// recurrence, the step counted, and the end of b's phase decided: rr at most
// floor^2 times the phase's initial rr0, the scaled estimate
// rr 4^sexp_prev at most (tol ||f||)^2, a non-finite rr, or the last
// iteration (state[2] + 1 >= max_iter).  Sets restart[b] and *any.
// ctl = (tol, max_iter, floor^2).
__global__ void __launch_bounds__(kThreads) k32_phase_check(
    const double* __restrict__ partial, int nblk, int B, const int* __restrict__ active,
    const double* __restrict__ rr0, const double* __restrict__ fsum,
    const int* __restrict__ sexp_prev, const double* __restrict__ ctl,
    const int* __restrict__ state, int* __restrict__ iters, int* __restrict__ restart,
    int* __restrict__ any) {
  pdl_wait();
  __shared__ double sh[kThreads];
  const int b = blockIdx.x;
  const double rr = block_sum_partials(partial, nblk, B, b, sh);
  if (threadIdx.x != 0 || !active[b]) return;
  iters[b] += 1;
  const double tol = ctl[0], floor2 = ctl[2];
  const double est = scale2(scale2(rr, sexp_prev[b]), sexp_prev[b]);
  const bool last = (double)(state[2] + 1) >= ctl[1];
  const bool end = !isfinite(rr) || rr <= floor2 * rr0[b] || est <= tol * tol * fsum[b] || last;
  if (end) {
    restart[b] = 1;
    atomicExch(any, 1);
  }
}

// u += 2^sexp_prev[b] e, e = 0 for the right-hand sides whose phase ends
// (nothing when no phase ends).
__global__ void __launch_bounds__(kRedMax) k32_fold(double* __restrict__ u, float* __restrict__ e,
                                                    const int* __restrict__ sexp_prev,
                                                    const int* __restrict__ restart,
                                                    const int* __restrict__ any, int n, int B) {
  pdl_wait();
  if (!*any) return;
  int g, b, i0;
  f32_tile(B, g, b, i0);
  if (b >= B || !restart[b]) return;
  const int s = sexp_prev[b];
#pragma unroll
  for (int k = 0; k < kF32Rows; ++k) {
    const int i = i0 + kRedRows * k;
    if (i < n) {
      const size_t t = (size_t)i * B + b;
      u[t] += scale2((double)e[t], s);
      e[t] = 0.0f;
    }
  }
}

// k_resid64 for a restart: r = f - A u in FP64 and the partials of r.r for
// every right-hand side, rhat = float(2^-sexp[b] r) written only where b's
// phase ends (the others keep their recurrence residual); nothing when no
// phase ends.
__global__ void __launch_bounds__(kRedMax) k_resid64_restart(
    LV<double> L, const double* __restrict__ f, const double* __restrict__ u,
    float* __restrict__ rhat, const int* __restrict__ sexp, const int* __restrict__ restart,
    const int* __restrict__ any, int B, double* __restrict__ partial) {
  pdl_wait();
  if (!*any) return;
  __shared__ double sh[kRedMax];
  int i, b;
  bool ok;
  red_tile(L.n, B, i, b, ok);
  double r = 0.0;
  if (ok) {
    const size_t k = (size_t)i * B + b;
    r = fma(-L.diag[i], u[k], f[k]) - row_ax(L, i, u, B, b);
    if (restart[b]) rhat[k] = (float)scale2(r, -sexp[b]);
  }
  sh[threadIdx.x] = r * r;
  __syncthreads();
  block_rows_reduce32(sh);
  red_store(sh, B, partial);
}

// k_reduce when some phase ends (nothing otherwise).
__global__ void __launch_bounds__(kThreads) k_reduce_if(const double* __restrict__ partial,
                                                        int nblk, int B,
                                                        const int* __restrict__ any,
                                                        double* __restrict__ out) {
  pdl_wait();
  if (!*any) return;
  __shared__ double sh[kThreads];
  const int b = blockIdx.x;
  const double r = block_sum_partials(partial, nblk, B, b, sh);
  if (threadIdx.x == 0) out[b] = r;
}

// One block: the restart's convergence test for the right-hand sides whose
// phase ended (check_block's rule on them only): relres from the FP64
// residual, active cleared at tol or on a non-finite residual, sexp_prev =
// the exponent rhat was scaled with, sexp = ilogb ||r||, rr0 = ||rhat||^2,
// a fresh direction next.  Then, for all, the loop state as check_block
// (inc: count this iteration) and the while-node condition; clears the
// restart flags.
__global__ void __launch_bounds__(kThreads) k32_restart_check(
    const double* __restrict__ rsum, const double* __restrict__ fsum, int B,
    const double* __restrict__ ctl, int* __restrict__ active, double* __restrict__ relres,
    int* __restrict__ sexp, int* __restrict__ sexp_prev, double* __restrict__ rr0,
    int* __restrict__ fresh, int* __restrict__ restart, int* __restrict__ any,
    int* __restrict__ state, int inc, cudaGraphConditionalHandle h, int set_cond) {
  pdl_wait();
  __shared__ int cnt, bad;
  const double tol = ctl[0];
  if (threadIdx.x == 0) { cnt = 0; bad = 0; }
  __syncthreads();
  const bool some = *any != 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    if (some && restart[b]) {
      const double rn = sqrt(rsum[b]), fn = sqrt(fsum[b]);
      const double rel = fn > 0.0 ? rn / fn : rn;
      relres[b] = rel;
      if (!isfinite(rel)) atomicAdd(&bad, 1);
      if (!(active[b] && !(rel < tol) && isfinite(rel))) active[b] = 0;
      const int sp = sexp[b];
      sexp_prev[b] = sp;
      sexp[b] = rn > 0.0 && isfinite(rn) ? ilogb(rn) : 0;
      rr0[b] = scale2(scale2(rsum[b], -sp), -sp);
      fresh[b] = 1;
      restart[b] = 0;
    }
    if (active[b]) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *any = 0;
    const int it = inc ? state[2] + 1 : 0;
    state[0] = cnt;
    state[1] = bad;
    state[2] = it;
    const int go = cnt > 0 && bad == 0 && (double)it < ctl[1];
    state[3] = go;
    if (set_cond) cudaGraphSetConditional(h, go ? 1u : 0u);
  }
}

// Start of a solve: every right-hand side active with a phase ending now
// (e = 0, so the first restart only forms r = f - A u), sexp = ilogb ||f||.
__global__ void k32_init(const double* __restrict__ fsum, int B, int* __restrict__ active,
                         int* __restrict__ iters, int* __restrict__ sexp,
                         int* __restrict__ restart, int* __restrict__ any) {
  pdl_wait();
  const int b = threadIdx.x + blockIdx.x * blockDim.x;
  if (b == 0) *any = 1;
  if (b >= B) return;
  active[b] = 1;
  iters[b] = 0;
  restart[b] = 1;
  const double fn = sqrt(fsum[b]);
  sexp[b] = fn > 0.0 && isfinite(fn) ? ilogb(fn) : 0;
}

}  // namespace mgk
