// mg_solve_fcg: flexible conjugate gradients with the context's learnable
// V-cycle (FP32 or FP64) as a variable preconditioner.  Included at the end
// of mg_api.cu (same translation unit).
//
// Notay's flexible CG with one stored direction, per right-hand side:
//   r = f - A u, z = M(r), p = z, q = A p, alpha = (p, r)/(p, q)
//   repeat: u += alpha p, r -= alpha q, test ||r||/||f|| < tol,
//           z = M(r), beta = -(z, q)/(p, q), p = z + beta p,
//           q = A p, alpha = (p, r)/(p, q)
// fcg64: FP64 vectors; an FP32 cycle sees r scaled by an exact power of two
// (2^-ilogb||r||).  fcg32 (precision-32 contexts, the default there): the
// same recurrence in FP32 on the scaled correction equation, in phases
// ended by FP64 restarts that form and test the true residual.  One CUDA
// graph holds the set-up and a while-node around the iteration.

namespace {

__global__ void k_fcg_count(const int* __restrict__ active, int* __restrict__ iters, int B) {
  mgk::pdl_wait();
  const int b = threadIdx.x;
  if (b < B && active[b]) iters[b] += 1;
}

__global__ void k_true_relres(const double* __restrict__ rsum, const double* __restrict__ fsum,
                              int B, double* __restrict__ relres) {
  mgk::pdl_wait();
  const int b = threadIdx.x;
  if (b >= B) return;
  const double rn = sqrt(rsum[b]), fn = sqrt(fsum[b]);
  relres[b] = fn > 0.0 ? rn / fn : rn;
}

mg_status fcg_buffers(mg_ctx* c) {
  if (c->k_r) return MG_OK;
  const size_t v = (size_t)c->n[0] * c->maxB * sizeof(double);
  for (double** q : {&c->k_r, &c->k_z, &c->k_p, &c->k_q}) MG_CUDA(cudaMalloc(q, v));
  MG_CUDA(cudaMalloc(&c->k_partial, (size_t)c->nblk_max * 2 * c->maxB * sizeof(double)));
  MG_CUDA(cudaMalloc(&c->k_small, (size_t)6 * c->maxB * sizeof(double)));
  return MG_OK;
}

// MG_OPT_FCG_FP32 = 2: FP32 vectors from this many level-0 rows on
constexpr int kFcg32Rows = 1 << 20;

mg_status fcg32_buffers(mg_ctx* c) {
  if (c->k32_p) return MG_OK;
  const size_t v = (size_t)c->n[0] * c->maxB * sizeof(float);
  for (float** q : {&c->k32_p, &c->k32_q, &c->k32_e}) MG_CUDA(cudaMalloc(q, v));
  MG_CUDA(cudaMalloc(&c->k32_small, (size_t)4 * c->maxB * sizeof(double) +
                                        (size_t)(2 * c->maxB + 1) * sizeof(int)));
  return MG_OK;
}

// mg_solve_fcg of a precision-32 context with FP32 vectors: phases of FCG(1)
// on the scaled correction equation A e = 2^-s r in FP32, ended per
// right-hand side by an FP64 restart (kernels in krylov.cuh).  One graph: the
// first restart (r = f - A u, the test) before a while node whose body is one
// FP32 step, the phase test and the (predicated) restart.
mg_status fcg32(mg_ctx* c, const double* f, double* u, int B, cudaStream_t s) {
  mg_status st = fcg32_buffers(c);
  if (st != MG_OK) return st;
  const int n0 = c->n[0];
  const int bt = std::min(B, 32);
  const int nblk = (n0 + mgk::kRedRows - 1) / mgk::kRedRows;
  const dim3 rgrid(nblk, (B + bt - 1) / bt), rblock(mgk::kRedRows * bt);
  const int nb32 = (n0 + mgk::kF32BlockRows - 1) / mgk::kF32BlockRows;
  const dim3 g32(nb32, (B + bt - 1) / bt);
  const LV<double> L0 = c->d64[0].view();
  const LV<float> L32 = c->d32[0].view();
  double* alpha = (double*)c->k32_small;
  double* beta = alpha + c->maxB;
  double* pq = beta + c->maxB;
  double* rr0 = pq + c->maxB;
  int* fresh = (int*)(rr0 + c->maxB);
  int* restart = fresh + c->maxB;
  int* any = restart + c->maxB;
  float* r = c->rhat32;  // the phase's recurrence residual (the cycle's input)
  float* z = c->c32;     // the preconditioned residual (the cycle's output)
  // the FP64 restart for the right-hand sides whose phase ends: u += 2^s e,
  // r = f - A u, the test, rhat = 2^-s r, a fresh direction
  auto restart_step = [&](Issue<double>& is, cudaGraphConditionalHandle h, int inc, int cond) {
    is.launch(mgk::k32_fold, g32, rblock, 0, u, c->k32_e, (const int*)c->sexp_prev,
              (const int*)restart, (const int*)any, n0, B);
    is.launch(mgk::k_resid64_restart, rgrid, rblock, 0, L0, f, (const double*)u, r,
              (const int*)c->sexp, (const int*)restart, (const int*)any, B, c->partial);
    is.launch(mgk::k_reduce_if, dim3(B), dim3(kThreads), 0, (const double*)c->partial, nblk, B,
              (const int*)any, c->rsum);
    is.launch(mgk::k32_restart_check, dim3(1), dim3(kThreads), 0, (const double*)c->rsum,
              (const double*)c->fsum, B, (const double*)c->tol_dev, c->active, c->relres, c->sexp,
              c->sexp_prev, rr0, fresh, restart, any, c->state, inc, h, cond);
  };
  auto pre = [&](cudaStream_t cs, cudaGraphConditionalHandle h, int cond) {
    Issue<double> is{c, c->d64, c->prm64, cs, B};
    is.launch(mgk::k_sumsq64, rgrid, rblock, 0, f, n0, B, c->partial);
    is.launch(mgk::k_reduce, dim3(B), dim3(kThreads), 0, (const double*)c->partial, nblk, B,
              c->fsum);
    is.launch(mgk::k32_init, dim3((B + kThreads - 1) / kThreads), dim3(kThreads), 0,
              (const double*)c->fsum, B, c->active, c->iters, c->sexp, restart, any);
    cudaMemsetAsync(c->k32_e, 0, (size_t)n0 * B * sizeof(float), cs);
    restart_step(is, h, 0, cond);
    return is.nk;
  };
  auto body = [&](cudaStream_t cs, cudaGraphConditionalHandle h, int cond) {
    int nk = 0;
    Issue<float> is{c, c->d32, c->prm32, cs, B};
    if (c->opt_fcg_precond == 1)
      is.fmg(r, z);
    else
      is.vcycle(r, z, true);
    // beta from (z, q_prev), the direction, q = A p and alpha, the update
    is.launch(mgk::k32_dot, g32, rblock, 0, (const float*)z, (const float*)c->k32_q, n0, B,
              c->partial);
    is.launch(mgk::k32_reduce_beta, dim3(B), dim3(kThreads), 0, (const double*)c->partial, nb32,
              B, (const double*)pq, (const int*)fresh, beta);
    is.launch(mgk::k32_direction, g32, rblock, 0, c->k32_p, (const float*)z, (const double*)beta,
              (const int*)fresh, n0, B);
    // q = A p on right-hand-side tiles of BV columns (BV | B)
    const int bv = B % 8 == 0 ? 8 : B % 4 == 0 ? 4 : B % 2 == 0 ? 2 : 1;
    const dim3 tblock(mgk::kRedRows * bt / bv);
    auto spmv = [&](auto kern) {
      is.launch(kern, g32, tblock, 0, L32, (const float*)c->k32_p, (const float*)r, c->k32_q, B,
                c->partial);
    };
    if (bv == 8)
      spmv(mgk::k32_spmv_dots_mb<8>);
    else if (bv == 4)
      spmv(mgk::k32_spmv_dots_mb<4>);
    else if (bv == 2)
      spmv(mgk::k32_spmv_dots_mb<2>);
    else
      spmv(mgk::k32_spmv_dots_mb<1>);
    is.launch(mgk::k32_reduce_alpha, dim3(B), dim3(kThreads), 0, (const double*)c->partial, nb32,
              B, (const int*)c->active, alpha, pq, fresh);
    is.launch(mgk::k32_fcg_update, g32, rblock, 0, c->k32_e, r, (const float*)c->k32_p,
              (const float*)c->k32_q, (const double*)alpha, (const int*)c->active, n0, B,
              c->partial);
    is.launch(mgk::k32_phase_check, dim3(B), dim3(kThreads), 0, (const double*)c->partial, nb32,
              B, (const int*)c->active, (const double*)rr0, (const double*)c->fsum,
              (const int*)c->sexp_prev, (const double*)c->tol_dev, (const int*)c->state,
              c->iters, restart, any);
    nk += is.nk;
    Issue<double> is2{c, c->d64, c->prm64, cs, B};
    restart_step(is2, h, 1, cond);
    return nk + is2.nk;
  };
  return run_loop(c, 45, f, u, B, s, "mg_solve_fcg", pre, body,
                  [](cudaStream_t) { return 0; }, false);
}

}  // namespace

namespace {

// mg_solve_fcg with FP64 vectors (FP64 contexts, and precision-32 contexts
// with MG_OPT_FCG_FP32 = 0): the FP32 cycle, if any, on the scaled residual.
mg_status fcg64(mg_ctx* c, const double* f, double* u, int B, double tol, int max_iter,
                cudaStream_t s) {
  mg_status st = fcg_buffers(c);
  if (st != MG_OK) return st;
  const int n0 = c->n[0];
  const int bt = std::min((int)B, 32);  // reduction tiling (kernels.cuh red_tile)
  const int nblk = (n0 + mgk::kRedRows - 1) / mgk::kRedRows;
  const dim3 rgrid(nblk, (B + bt - 1) / bt), rblock(mgk::kRedRows * bt);
  const LV<double> L0 = c->d64[0].view();
  const bool p32 = c->prec == 32;
  const size_t N = (size_t)n0 * B;
  double* alpha = c->k_small;
  double* pq = c->k_small + c->maxB;
  double* zq = c->k_small + 2 * c->maxB;
  double* sums = c->k_small + 3 * c->maxB;  // [2B]
  c->solve_ctl[0] = tol;
  c->solve_ctl[1] = (double)max_iter;
  MG_CUDA(cudaMemcpyAsync(c->tol_dev, c->solve_ctl, 2 * sizeof(double), cudaMemcpyHostToDevice, s));

  // z = M(r): one V-cycle from zero, or one full multigrid
  // (MG_OPT_FCG_PRECOND), on the (scaled) residual
  auto precondition = [&](cudaStream_t cs) {
    int nk = 0;
    if (p32) {
      Issue<double> is0{c, c->d64, c->prm64, cs, B};
      is0.launch(mgk::k_scale_to_f32, grid_for(N), dim3(kThreads), 0, (const double*)c->k_r,
                 (const int*)c->sexp, c->rhat32, n0, (int)B);
      Issue<float> is{c, c->d32, c->prm32, cs, B};
      if (c->opt_fcg_precond == 1)
        is.fmg(c->rhat32, c->c32);
      else
        is.vcycle(c->rhat32, c->c32, true);
      is.launch(mgk::k_scale_from_f32, grid_for(N), dim3(kThreads), 0, (const float*)c->c32,
                (const int*)c->sexp, c->k_z, n0, (int)B);
      nk += is0.nk + is.nk;
    } else {
      Issue<double> is{c, c->d64, c->prm64, cs, B};
      if (c->opt_fcg_precond == 1)
        is.fmg(c->k_r, c->k_z);
      else
        is.vcycle(c->k_r, c->k_z, true);
      nk += is.nk;
    }
    return nk;
  };
  // q = A p, (p, q), (p, r), alpha
  auto direction_tail = [&](Issue<double>& is) {
    is.launch(mgk::k_spmv_dots, rgrid, rblock, 0, L0, (const double*)c->k_p,
              (const double*)c->k_r, c->k_q, (int)B, c->k_partial);
    is.launch(mgk::k_reduce, dim3(2 * B), dim3(kThreads), 0, (const double*)c->k_partial, nblk,
              (int)(2 * B), sums);
    is.launch(mgk::k_fcg_alpha, dim3(1), dim3(kThreads), 0, (const double*)sums,
              (const int*)c->active, (int)B, alpha, pq);
  };
  // ||f||, r = f - A u, the first test, z = M r, p = z and its direction terms
  auto pre = [&](cudaStream_t cs, cudaGraphConditionalHandle h, int cond) {
    int nk = 0;
    Issue<double> is{c, c->d64, c->prm64, cs, B};
    is.launch(mgk::k_sumsq64, rgrid, rblock, 0, f, n0, (int)B, c->partial);
    is.launch(mgk::k_reduce, dim3(B), dim3(kThreads), 0, (const double*)c->partial, nblk, (int)B,
              c->fsum);
    is.launch(k_init_solve, dim3(1), dim3(kThreads), 0, (const double*)c->fsum, (int)B, c->active,
              c->iters, c->sexp);
    is.launch(mgk::k_outer_residual64, rgrid, rblock, 0, L0, f, (const double*)u, c->k_r, (int)B);
    is.launch(mgk::k_dots<1>, rgrid, rblock, 0, (const double*)c->k_r, (const double*)c->k_r,
              (const double*)nullptr, (const double*)nullptr, n0, (int)B, c->partial);
    reduce_and_check(is, c, nblk, (int)B, (int*)nullptr, 0, h, cond);
    nk += is.nk;
    nk += precondition(cs);
    Issue<double> is2{c, c->d64, c->prm64, cs, B};
    is2.launch(mgk::k_fcg_direction, grid_for(N), dim3(kThreads), 0, c->k_p, (const double*)c->k_z,
               (const double*)zq, (const double*)pq, n0, (int)B, 1);
    direction_tail(is2);
    return nk + is2.nk;
  };
  // u += alpha p, r -= alpha q, the test, z = M r, the new direction
  auto body = [&](cudaStream_t cs, cudaGraphConditionalHandle h, int cond) {
    int nk = 0;
    Issue<double> is{c, c->d64, c->prm64, cs, B};
    is.launch(k_fcg_count, dim3(1), dim3(kThreads), 0, (const int*)c->active, c->iters, (int)B);
    is.launch(mgk::k_fcg_update, rgrid, rblock, 0, u, c->k_r, (const double*)c->k_p,
              (const double*)c->k_q, (const double*)alpha, (const int*)c->active, n0, (int)B,
              c->partial);
    reduce_and_check(is, c, nblk, (int)B, (int*)nullptr, 1, h, cond);
    nk += is.nk;
    nk += precondition(cs);
    Issue<double> is2{c, c->d64, c->prm64, cs, B};
    is2.launch(mgk::k_dots<1>, rgrid, rblock, 0, (const double*)c->k_z, (const double*)c->k_q,
               (const double*)nullptr, (const double*)nullptr, n0, (int)B, c->partial);
    is2.launch(mgk::k_reduce, dim3(B), dim3(kThreads), 0, (const double*)c->partial, nblk, (int)B,
               zq);
    is2.launch(mgk::k_fcg_direction, grid_for(N), dim3(kThreads), 0, c->k_p, (const double*)c->k_z,
               (const double*)zq, (const double*)pq, n0, (int)B, 0);
    direction_tail(is2);
    return nk + is2.nk;
  };
  // after the loop: the true residual of the final iterate
  auto post = [&](cudaStream_t cs) {
    Issue<double> is{c, c->d64, c->prm64, cs, B};
    is.launch(mgk::k_outer_residual64, rgrid, rblock, 0, L0, f, (const double*)u, c->k_r, (int)B);
    is.launch(mgk::k_dots<1>, rgrid, rblock, 0, (const double*)c->k_r, (const double*)c->k_r,
              (const double*)nullptr, (const double*)nullptr, n0, (int)B, c->partial);
    is.launch(mgk::k_reduce, dim3(B), dim3(kThreads), 0, (const double*)c->partial, nblk, (int)B,
              c->rsum);
    is.launch(k_true_relres, dim3(1), dim3(kThreads), 0, (const double*)c->rsum,
              (const double*)c->fsum, (int)B, c->relres);
    return is.nk;
  };
  return run_loop(c, 40, f, u, B, s, "mg_solve_fcg", pre, body, post, true);
}

}  // namespace

extern "C" mg_status mg_solve_fcg(mg_ctx* c, const double* f, double* u, int32_t B, double tol,
                                  int32_t max_iter, int32_t* iters_out, double* relres_out,
                                  void* stream) {
  if (!c) return mgi::set_global_error(MG_ERR_INVALID, "mg_solve_fcg: ctx is NULL");
  if (!f || !u || B < 1 || B > c->maxB || max_iter < 0 || !(tol > 0.0))
    return c->fail(MG_ERR_INVALID, "mg_solve_fcg: bad arguments");
  if ((const void*)f == (const void*)u) return c->fail(MG_ERR_INVALID, "mg_solve_fcg: f and u alias");
  cudaStream_t s = (cudaStream_t)stream;
  mg_status st = sync_params(c, s);
  if (st != MG_OK) return st;
  // FP32 vectors where the FP64 vector work is large (it is bound by B300's
  // FP64 pipe); on smaller levels the FP64 form converges in fewer steps.
  // The choice depends on the operator only, never on the batch.
  const bool fp32_vectors =
      c->prec == 32 && (c->opt_fcg_fp32 == 1 || (c->opt_fcg_fp32 == 2 && c->n[0] >= kFcg32Rows));
  if (fp32_vectors) {
    const double fl = c->opt_fcg_floor > 0 ? std::pow(10.0, -c->opt_fcg_floor) : 0.0;
    c->solve_ctl[0] = tol;
    c->solve_ctl[1] = (double)max_iter;
    c->solve_ctl[2] = fl * fl;
    MG_CUDA(cudaMemcpyAsync(c->tol_dev, c->solve_ctl, 3 * sizeof(double), cudaMemcpyHostToDevice,
                            s));
    st = fcg32(c, f, u, (int)B, s);
  } else {
    st = fcg64(c, f, u, (int)B, tol, max_iter, s);
  }
  if (st != MG_OK) return st;
  mg_status result = MG_OK;
  if (c->h_state[1])
    result = MG_ERR_DIVERGED;
  else if (c->h_state[0] > 0)
    result = MG_NOT_CONVERGED;
  if ((st = read_results(c, s, (int)B, iters_out, relres_out)) != MG_OK) return st;
  if (result == MG_ERR_DIVERGED) c->err = "mg_solve_fcg: non-finite residual";
  if (result == MG_NOT_CONVERGED) c->err = "mg_solve_fcg: tolerance not met within max_iter";
  return result;
}
