// mg_solve_fcg: flexible conjugate gradients in FP64 with the context's
// learnable V-cycle (FP32 or FP64) as a variable preconditioner.  Included at
// the end of mg_api.cu (same translation unit).
//
// Notay's flexible CG with one stored direction, per right-hand side:
//   r = f - A u, z = M(r), p = z, q = A p, alpha = (p, r)/(p, q)
//   repeat: u += alpha p, r -= alpha q, test ||r||/||f|| < tol,
//           z = M(r), beta = -(z, q)/(p, q), p = z + beta p,
//           q = A p, alpha = (p, r)/(p, q)
// The FP32 cycle sees r scaled by an exact power of two (2^-ilogb||r||).
// One CUDA graph holds the set-up and a while-node around the iteration.

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
  st = fcg_buffers(c);
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
  st = run_loop(c, 40, f, u, (int)B, s, "mg_solve_fcg", pre, body, post, true);
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
