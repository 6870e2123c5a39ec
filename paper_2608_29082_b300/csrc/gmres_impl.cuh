// mg_solve_fgmres: restarted flexible GMRES (gmres.cuh) with the learnable
// V-cycle or full multigrid as the right preconditioner.  Included at the end
// of mg_api.cu (same translation unit), after krylov_impl.cuh.
//
// The host drives the restart cycle: a restart graph (FP64 true residual,
// beta, v_0), one graph per Arnoldi step j (preconditioner, K z_j, CGS2, the
// rotations) in the context precision, and an end-of-cycle graph (y, u += Z
// y in FP64).  After the restart and after every step the host reads the
// convergence counts.  In an FP32 context this is FGMRES-based iterative
// refinement: FP32 cycles, each ending at most MG_OPT_FGMRES_FLOOR decades
// below its starting residual, corrected by FP64 restarts.

namespace {

mg_status gm_buffers(mg_ctx* c, int m) {
  if (c->gm_m == m && c->gm_V) return MG_OK;
  // graphs captured earlier point at the old workspace
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
  c->graphs.clear();
  for (void* p : {c->gm_V, c->gm_Z, (void*)c->gm_zero32, (void*)c->gm_small, (void*)c->gm_h,
                  (void*)c->gm_vec, (void*)c->gm_partial, (void*)c->gm_done})
    if (p) cudaFree(p);
  c->gm_V = c->gm_Z = nullptr;
  c->gm_zero32 = nullptr;
  c->gm_small = c->gm_h = c->gm_vec = c->gm_partial = nullptr;
  c->gm_done = nullptr;
  c->gm_m = 0;
  const size_t N = (size_t)c->n[0] * c->maxB;
  const size_t v = N * (c->prec == 32 ? sizeof(float) : sizeof(double));
  const size_t nblk = ((size_t)c->n[0] + mgk::kGmTile - 1) / mgk::kGmTile;
  const size_t mb = (size_t)c->maxB;
  MG_CUDA(cudaMalloc(&c->gm_V, v * (m + 1)));
  MG_CUDA(cudaMalloc(&c->gm_Z, v * m));
  if (c->prec == 32) {
    MG_CUDA(cudaMalloc(&c->gm_zero32, N * sizeof(float)));
    MG_CUDA(cudaMemset(c->gm_zero32, 0, N * sizeof(float)));
  }
  MG_CUDA(cudaMalloc(&c->gm_small, mb * mgk::gm_stride(m) * sizeof(double)));
  MG_CUDA(cudaMalloc(&c->gm_h, 2 * (m + 1) * mb * sizeof(double)));
  MG_CUDA(cudaMalloc(&c->gm_vec, 2 * mb * sizeof(double)));
  MG_CUDA(cudaMalloc(&c->gm_partial, nblk * (m + 1) * mb * sizeof(double)));
  MG_CUDA(cudaMalloc(&c->gm_done, mb * sizeof(int)));
  c->gm_m = m;
  return MG_OK;
}

// Launch shapes and scratch of one FGMRES solve.
struct GmShape {
  int m, B, n0, gblk;
  size_t vs;  // stride between basis vectors
  dim3 ggrid, gblock, rgrid, rblock;
  double *h1, *h2, *wn, *inv;
  double rho;
};

// Arnoldi step j in vector type T: z_j = M(v_j), w = K z_j into the slot of
// v_{j+1} (K = A in FP64; K = -A in FP32, as 0 - A z from the residual
// kernel, undone by the update's sign), CGS2, the rotations, v_{j+1}.
template <class T>
void gm_step(mg_ctx* c, Issue<T>& is, const GmShape& g, int j, const LV<double>& L0) {
  T* V = (T*)c->gm_V;
  T* Z = (T*)c->gm_Z;
  T* Vj = V + (size_t)j * g.vs;
  T* Vn = V + (size_t)(j + 1) * g.vs;
  T* Zj = Z + (size_t)j * g.vs;
  if (c->opt_fcg_precond == 1)
    is.fmg(Vj, Zj);
  else
    is.vcycle(Vj, Zj, true);
  if constexpr (sizeof(T) == sizeof(float))
    is.op_residual(0, c->gm_zero32, Zj, Vn, 0, 0);
  else
    is.launch(mgk::k_spmv_dots, g.rgrid, g.rblock, 0, L0, (const double*)Zj, (const double*)Vj,
              (double*)Vn, g.B, c->k_partial);
  for (int pass = 0; pass < 2; ++pass) {
    double* h = pass == 0 ? g.h1 : g.h2;
    is.launch(mgk::k_gm_dots<T>, g.ggrid, g.gblock, 0, (const T*)V, g.vs, (const T*)Vn, j + 1,
              g.n0, g.B, c->gm_partial);
    is.launch(mgk::k_reduce, dim3((j + 1) * g.B), dim3(kThreads), 0,
              (const double*)c->gm_partial, g.gblk, (int)((j + 1) * g.B), h);
    is.launch(mgk::k_gm_orth<T>, g.ggrid, g.gblock, 0, (const T*)V, g.vs, Vn, (const double*)h,
              j + 1, g.n0, g.B, c->partial);
  }
  is.launch(mgk::k_reduce, dim3(g.B), dim3(kThreads), 0, (const double*)c->partial, g.gblk, g.B,
            g.wn);
  is.launch(mgk::k_gm_arnoldi, dim3(1), dim3(kThreads), 0, c->gm_small, (const double*)g.h1,
            (const double*)g.h2, (const double*)g.wn, (const double*)c->fsum,
            (const double*)c->tol_dev, g.m, j, g.B, g.rho, (const int*)c->active, c->iters, g.inv,
            c->relres, c->gm_done, c->state);
  is.launch(mgk::k_gm_scale<T, T>, grid_for((size_t)g.n0 * g.B), dim3(kThreads), 0,
            (const T*)Vn, (const double*)g.inv, Vn, g.n0, g.B);
}

}  // namespace

extern "C" mg_status mg_solve_fgmres(mg_ctx* c, const double* f, double* u, int32_t B, double tol,
                                     int32_t max_iter, int32_t restart, int32_t* iters_out,
                                     double* relres_out, void* stream) {
  if (!c) return mgi::set_global_error(MG_ERR_INVALID, "mg_solve_fgmres: ctx is NULL");
  if (!f || !u || B < 1 || B > c->maxB || max_iter < 0 || !(tol > 0.0) || restart < 1 ||
      restart > 64)
    return c->fail(MG_ERR_INVALID, "mg_solve_fgmres: bad arguments");
  if ((const void*)f == (const void*)u)
    return c->fail(MG_ERR_INVALID, "mg_solve_fgmres: f and u alias");
  cudaStream_t s = (cudaStream_t)stream;
  mg_status st = sync_params(c, s);
  if (st != MG_OK) return st;
  st = fcg_buffers(c);
  if (st != MG_OK) return st;
  const int m = restart;
  st = gm_buffers(c, m);
  if (st != MG_OK) return st;
  const int n0 = c->n[0];
  const int bt = std::min((int)B, 32);  // reduction tiling (kernels.cuh red_tile)
  const int nblk = (n0 + mgk::kRedRows - 1) / mgk::kRedRows;
  const dim3 rgrid(nblk, (B + bt - 1) / bt), rblock(mgk::kRedRows * bt);
  const LV<double> L0 = c->d64[0].view();
  const bool p32 = c->prec == 32;
  const size_t N = (size_t)n0 * B;
  GmShape g;
  g.m = m;
  g.B = B;
  g.n0 = n0;
  // Gram-Schmidt tiling (gmres.cuh): 256 rows x min(B, 16) columns a block
  const int gbt = std::min((int)B, mgk::kGmBt);
  g.gblk = (n0 + mgk::kGmTile - 1) / mgk::kGmTile;
  g.ggrid = dim3(g.gblk, (B + gbt - 1) / gbt);
  g.gblock = dim3(mgk::kRedRows * gbt);
  g.rgrid = rgrid;
  g.rblock = rblock;
  g.vs = N;
  g.h1 = c->gm_h;
  g.h2 = c->gm_h + (size_t)(m + 1) * B;
  g.wn = c->gm_vec;
  g.inv = c->gm_vec + B;
  // an FP32 cycle resolves its residual to about 1e-4..1e-7 of its start
  // (CGS2 and K z in FP32, depending on the operator's conditioning); below
  // that the FP64 restart takes over
  g.rho = p32 && c->opt_fgmres_floor > 0 ? std::pow(10.0, -c->opt_fgmres_floor) : 0.0;
  const double sgn = p32 ? -1.0 : 1.0;
  c->solve_ctl[0] = tol;
  c->solve_ctl[1] = (double)max_iter;
  MG_CUDA(cudaMemcpyAsync(c->tol_dev, c->solve_ctl, 2 * sizeof(double), cudaMemcpyHostToDevice, s));
  auto key = [&](int id) {
    return std::make_tuple(id, (const void*)f, (const void*)u, (int)B, c->structure);
  };
  auto read_state = [&]() -> mg_status {
    MG_CUDA(cudaMemcpyAsync(c->h_state, c->state, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaStreamSynchronize(s));
    return MG_OK;
  };

  // ||f||, every right-hand side active, no iterations yet
  st = run_graph(c, key(7000), s, [&](cudaStream_t cs) {
    Issue<double> is{c, c->d64, c->prm64, cs, B};
    is.launch(mgk::k_sumsq64, rgrid, rblock, 0, f, n0, (int)B, c->partial);
    is.launch(mgk::k_reduce, dim3(B), dim3(kThreads), 0, (const double*)c->partial, nblk, (int)B,
              c->fsum);
    is.launch(k_init_solve, dim3(1), dim3(kThreads), 0, (const double*)c->fsum, (int)B, c->active,
              c->iters, c->sexp);
    return is.nk;
  });
  if (st != MG_OK) return st;
  int total = 0;
  bool diverged = false;
  for (;;) {
    // restart: r = f - A u, beta = ||r||, the test, v_0 = r / beta
    st = run_graph(c, key(7001), s, [&](cudaStream_t cs) {
      Issue<double> is{c, c->d64, c->prm64, cs, B};
      is.launch(mgk::k_outer_residual64, rgrid, rblock, 0, L0, f, (const double*)u, c->k_r,
                (int)B);
      is.launch(mgk::k_dots<1>, rgrid, rblock, 0, (const double*)c->k_r, (const double*)c->k_r,
                (const double*)nullptr, (const double*)nullptr, n0, (int)B, c->partial);
      is.launch(mgk::k_reduce, dim3(B), dim3(kThreads), 0, (const double*)c->partial, nblk, (int)B,
                c->rsum);
      is.launch(mgk::k_gm_restart, dim3(1), dim3(kThreads), 0, (const double*)c->rsum,
                (const double*)c->fsum, (const double*)c->tol_dev, m, (int)B, c->active,
                c->relres, c->gm_small, g.inv, c->gm_done, c->state);
      if (p32)
        is.launch(mgk::k_gm_scale<double, float>, grid_for(N), dim3(kThreads), 0,
                  (const double*)c->k_r, (const double*)g.inv, (float*)c->gm_V, n0, (int)B);
      else
        is.launch(mgk::k_gm_scale<double, double>, grid_for(N), dim3(kThreads), 0,
                  (const double*)c->k_r, (const double*)g.inv, (double*)c->gm_V, n0, (int)B);
      return is.nk;
    });
    if (st != MG_OK) return st;
    if ((st = read_state()) != MG_OK) return st;
    if (c->h_state[1]) {
      diverged = true;
      break;
    }
    if (c->h_state[0] == 0 || total >= max_iter) break;
    int jl = -1;
    for (int j = 0; j < m && total < max_iter; ++j) {
      st = run_graph(c, key(7100 + j), s, [&](cudaStream_t cs) {
        if (p32) {
          Issue<float> is{c, c->d32, c->prm32, cs, B};
          gm_step(c, is, g, j, L0);
          return is.nk;
        }
        Issue<double> is{c, c->d64, c->prm64, cs, B};
        gm_step(c, is, g, j, L0);
        return is.nk;
      });
      if (st != MG_OK) return st;
      ++total;
      jl = j;
      if ((st = read_state()) != MG_OK) return st;
      if (c->h_state[3] == 0) break;
    }
    if (jl < 0) break;
    // end of the cycle: y, u += Z y
    st = run_graph(c, key(7300 + jl), s, [&](cudaStream_t cs) {
      Issue<double> is{c, c->d64, c->prm64, cs, B};
      is.launch(mgk::k_gm_solve_y, dim3(1), dim3(kThreads), 0, c->gm_small, m, jl, (int)B,
                (const int*)c->active, (const int*)c->gm_done);
      if (p32)
        is.launch(mgk::k_gm_update<float>, grid_for(N), dim3(kThreads), 0, u,
                  (const float*)c->gm_Z, g.vs, (const double*)c->gm_small, m, jl + 1, sgn,
                  (const int*)c->active, n0, (int)B);
      else
        is.launch(mgk::k_gm_update<double>, grid_for(N), dim3(kThreads), 0, u,
                  (const double*)c->gm_Z, g.vs, (const double*)c->gm_small, m, jl + 1, sgn,
                  (const int*)c->active, n0, (int)B);
      return is.nk;
    });
    if (st != MG_OK) return st;
  }
  // the true residual of the final iterate
  st = run_graph(c, key(7002), s, [&](cudaStream_t cs) {
    Issue<double> is{c, c->d64, c->prm64, cs, B};
    is.launch(mgk::k_outer_residual64, rgrid, rblock, 0, L0, f, (const double*)u, c->k_r, (int)B);
    is.launch(mgk::k_dots<1>, rgrid, rblock, 0, (const double*)c->k_r, (const double*)c->k_r,
              (const double*)nullptr, (const double*)nullptr, n0, (int)B, c->partial);
    is.launch(mgk::k_reduce, dim3(B), dim3(kThreads), 0, (const double*)c->partial, nblk, (int)B,
              c->rsum);
    is.launch(k_true_relres, dim3(1), dim3(kThreads), 0, (const double*)c->rsum,
              (const double*)c->fsum, (int)B, c->relres);
    return is.nk;
  });
  if (st != MG_OK) return st;
  std::vector<double> rel(B);
  if ((st = read_results(c, s, (int)B, iters_out, rel.data())) != MG_OK) return st;
  if (relres_out) std::copy(rel.begin(), rel.end(), relres_out);
  mg_status result = MG_OK;
  for (double r : rel)
    if (!(r < tol)) result = MG_NOT_CONVERGED;
  if (diverged) result = MG_ERR_DIVERGED;
  if (result == MG_ERR_DIVERGED) c->err = "mg_solve_fgmres: non-finite residual";
  if (result == MG_NOT_CONVERGED) c->err = "mg_solve_fgmres: tolerance not met within max_iter";
  return result;
}
