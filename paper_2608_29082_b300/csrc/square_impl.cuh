// Stacked contexts for serving: one operator per request on a structured
// square mesh.  Included at the end of mg_api.cu (same translation unit).
//
// A context for `slots` requests of size class N holds, on every level, the
// block-diagonal stack of `slots` interior operators (block b = rows
// [b m_l, (b+1) m_l), m_l = (N_l - 2)^2).  The DIA offsets of a level are the
// same for every block and the entries that would couple two blocks are
// zero, so the cycle's kernels run on the stack unchanged; a block's rows
// see only their own block.  mg_setup_square builds the structure once
// (transfers, offsets, device arrays); mg_square_set_block writes one
// request's operator into its block on the device (assembly, Galerkin
// coarsening, drop rule, degrees, coarsest inverse); mg_solve_blocks solves
// every block to its own tolerance with per-block norms, scaling, masking
// and convergence.

namespace {

struct SquareLevels {
  std::vector<int> N;  // vertices per side, finest first
};

// Host CSR of one stacked level with placeholder values on the operator's
// pattern (interior 5-point on the finest level, 7-point on Galerkin
// levels); transfers of the natural inclusion between interior grids.
struct StackCsr {
  std::vector<int> rp, ci;
  std::vector<double> v;
  mg_csr csr() const {
    mg_csr c;
    c.n_rows = (int)rp.size() - 1;
    c.n_cols = c.n_rows;
    c.nnz = (int)ci.size();
    c.rowptr = rp.data();
    c.col = ci.data();
    c.val = v.data();
    return c;
  }
};

void stack_operator(int N, int slots, bool seven, StackCsr& A) {
  const int w = N - 2, m = w * w;
  A.rp.assign(1, 0);
  A.ci.clear();
  A.v.clear();
  const int dx7[7] = {-1, 0, -1, 0, 1, 0, 1}, dy7[7] = {-1, -1, 0, 0, 0, 1, 1};
  for (int b = 0; b < slots; ++b)
    for (int r = 0; r < m; ++r) {
      const int x = r % w, y = r / w;
      for (int k = 0; k < 7; ++k) {
        if (!seven && (k == 0 || k == 6)) continue;
        const int jx = x + dx7[k], jy = y + dy7[k];
        if (jx < 0 || jy < 0 || jx >= w || jy >= w) continue;
        A.ci.push_back(b * m + jy * w + jx);
        A.v.push_back(k == 3 ? (seven ? 8.0 : 4.0) : -1.0);
      }
      A.rp.push_back((int)A.ci.size());
    }
}

void stack_prolongation(int Nf, int slots, StackCsr& P) {
  const int Nc = (Nf - 1) / 2 + 1;
  const int wf = Nf - 2, wc = Nc - 2, mf = wf * wf, mc = wc * wc;
  P.rp.assign(1, 0);
  P.ci.clear();
  P.v.clear();
  auto cidx = [&](int X, int Y) {  // interior coarse index or -1
    return (X <= 0 || Y <= 0 || X >= Nc - 1 || Y >= Nc - 1) ? -1 : (Y - 1) * wc + (X - 1);
  };
  for (int b = 0; b < slots; ++b)
    for (int r = 0; r < mf; ++r) {
      const int x = r % wf + 1, y = r / wf + 1;
      int pa[2] = {-1, -1};
      double wt = 0.5;
      if (x % 2 == 0 && y % 2 == 0) {
        pa[0] = cidx(x / 2, y / 2);
        wt = 1.0;
      } else if (x % 2 == 1 && y % 2 == 0) {
        pa[0] = cidx((x - 1) / 2, y / 2);
        pa[1] = cidx((x + 1) / 2, y / 2);
      } else if (x % 2 == 0 && y % 2 == 1) {
        pa[0] = cidx(x / 2, (y - 1) / 2);
        pa[1] = cidx(x / 2, (y + 1) / 2);
      } else {
        pa[0] = cidx((x - 1) / 2, (y - 1) / 2);
        pa[1] = cidx((x + 1) / 2, (y + 1) / 2);
      }
      if (pa[0] >= 0 && pa[1] >= 0 && pa[1] < pa[0]) std::swap(pa[0], pa[1]);
      for (int k = 0; k < 2; ++k)
        if (pa[k] >= 0) {
          P.ci.push_back(b * mc + pa[k]);
          P.v.push_back(wt);
        }
      P.rp.push_back((int)P.ci.size());
    }
}

// DIA slot of each offset of a stacked level (interior width w).
mgk::SqDia square_dia(const int* doff, int ndia, int w) {
  mgk::SqDia d;
  d.ndia = ndia;
  const int dx[7] = {0, -1, 0, -1, 1, 0, 1}, dy[7] = {0, -1, -1, 0, 0, 1, 1};
  for (int k = 0; k < ndia; ++k) {
    d.slot[k] = 0;
    for (int s = 1; s < 7; ++s)
      if (dy[s] * w + dx[s] == doff[k]) d.slot[k] = s;
  }
  for (int k = ndia; k < mgk::kMaxDia; ++k) d.slot[k] = 0;
  return d;
}

}  // namespace

extern "C" mg_status mg_setup_square(mg_ctx** out, int32_t N, int32_t J, int32_t slots,
                                     const mg_params* p, int32_t precision, void* stream) {
  std::lock_guard<std::recursive_mutex> lk(mgi::setup_mutex());
  if (!out) return mgi::set_global_error(MG_ERR_INVALID, "mg_setup_square: out is NULL");
  *out = nullptr;
  if (J < 2 || J > 16 || slots < 1 || slots > 2048 || N < 5)
    return mgi::set_global_error(MG_ERR_INVALID, "mg_setup_square: bad sizes");
  std::vector<int> Ns{N};
  for (int l = 1; l < J; ++l) {
    if ((Ns.back() - 1) % 2) return mgi::set_global_error(MG_ERR_INVALID, "mg_setup_square: N - 1 must be divisible by 2^(J-1)");
    Ns.push_back((Ns.back() - 1) / 2 + 1);
  }
  if (Ns.back() != 3)
    return mgi::set_global_error(MG_ERR_INVALID,
                                 "mg_setup_square: the coarsest level must be 3 x 3 vertices");
  if ((int64_t)(N - 2) * (N - 2) * slots >= ((int64_t)1 << 31))
    return mgi::set_global_error(MG_ERR_INVALID, "mg_setup_square: too many rows");
  std::vector<StackCsr> A(J), P(J - 1);
  std::vector<std::vector<double>> deg(J);
  for (int l = 0; l < J; ++l) {
    stack_operator(Ns[l], slots, l > 0, A[l]);
    deg[l].assign(A[l].rp.size() - 1, l > 0 ? 1.0 / 6.0 : 0.25);
    if (l < J - 1) stack_prolongation(Ns[l], slots, P[l]);
  }
  std::vector<mg_csr> Ac(J), Pc(std::max(J - 1, 1));
  std::vector<const double*> dp(J);
  for (int l = 0; l < J; ++l) {
    Ac[l] = A[l].csr();
    dp[l] = deg[l].data();
    if (l < J - 1) {
      Pc[l] = P[l].csr();
      Pc[l].n_cols = (int)A[l + 1].rp.size() - 1;
    }
  }
  mg_hierarchy h;
  h.n_levels = J;
  h.P = Pc.data();
  h.inv_deg = dp.data();
  const int keep_policy = g_layout_policy;
  g_layout_policy = 0;  // every stacked level is DIA
  mg_ctx* c = nullptr;
  mg_status st = mg_setup(&c, &h, Ac.data(), p, 1, precision, stream);
  g_layout_policy = keep_policy;
  if (st != MG_OK) return st;
  c->sq_slots = slots;
  c->sq_N = Ns;
  size_t scratch = 0;
  for (int n : Ns) scratch += (size_t)n * n * mgk::kSqSlots;
  cudaError_t e;
  if ((e = cudaMalloc(&c->sq_scratch, scratch * sizeof(double))) != cudaSuccess ||
      (e = cudaMemset(c->sq_scratch, 0, scratch * sizeof(double))) != cudaSuccess ||
      (c->cholInv == nullptr &&
       (e = cudaMalloc(&c->cholInv, (size_t)slots * slots * sizeof(double))) != cudaSuccess) ||
      (e = cudaMemset(c->cholInv, 0, (size_t)slots * slots * sizeof(double))) != cudaSuccess ||
      (e = cudaStreamSynchronize(cudaStreamLegacy)) != cudaSuccess) {
    mg_destroy(c);
    return mgi::set_global_error(e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,
                                 std::string("mg_setup_square: ") + cudaGetErrorString(e));
  }
  // the block-diagonal coarsest level is solved by its explicit inverse,
  // one 1 x 1 block per request
  c->coarse_inv = true;
  for (int l = 0; l < J; ++l)
    if ((l < (int)c->d64.size() && c->d64[l].ndia == 0 && c->d64[l].n > slots) ||
        (l < (int)c->d32.size() && c->d32[l].ndia == 0 && c->d32[l].n > slots)) {
      mg_destroy(c);
      return mgi::set_global_error(MG_ERR_CUDA, "mg_setup_square: a stacked level is not DIA");
    }
  *out = c;
  return MG_OK;
}

extern "C" mg_status mg_square_set_block(mg_ctx* c, int32_t block, const double* ke,
                                         void* stream) {
  if (!c) return mgi::set_global_error(MG_ERR_INVALID, "mg_square_set_block: ctx is NULL");
  if (c->sq_slots <= 0) return c->fail(MG_ERR_INVALID, "mg_square_set_block: not a square context");
  if (!ke || block < 0 || block >= c->sq_slots)
    return c->fail(MG_ERR_INVALID, "mg_square_set_block: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const int J = c->J, S = c->sq_slots;
  std::vector<double*> Sl(J);
  size_t off = 0;
  for (int l = 0; l < J; ++l) {
    Sl[l] = c->sq_scratch + off;
    off += (size_t)c->sq_N[l] * c->sq_N[l] * mgk::kSqSlots;
  }
  auto blocks = [](size_t n) { return dim3((unsigned)((n + kThreads - 1) / kThreads)); };
  const int N0 = c->sq_N[0];
  mgk::k_sq_assemble<<<blocks((size_t)N0 * N0), kThreads, 0, s>>>(N0, ke, Sl[0]);
  for (int l = 0; l < J; ++l) {
    const int Nl = c->sq_N[l], w = Nl - 2;
    if (l < J - 1) {
      auto write = [&](auto& D, auto* dummy, DevLevel<double>* D64) {
        using T = std::remove_pointer_t<decltype(dummy)>;
        const mgk::SqDia dia = square_dia(D.doff, D.ndia, w);
        mgk::k_sq_write<T><<<blocks((size_t)w * w), kThreads, 0, s>>>(
            Nl, Sl[l], block, dia, D.n, D.dval, D.diag, D.dinv, D.invdeg, D.nbm,
            D64 ? D64->dval : nullptr, D64 ? D64->diag : nullptr, D64 ? D64->dinv : nullptr,
            D64 ? D64->nbm : nullptr);
      };
      if (c->prec == 64)
        write(c->d64[l], (double*)nullptr, (DevLevel<double>*)nullptr);
      else
        write(c->d32[l], (float*)nullptr, l == 0 ? &c->d64[0] : nullptr);
      const int Nc = c->sq_N[l + 1];
      mgk::k_sq_galerkin<<<blocks((size_t)Nc * Nc), kThreads, 0, s>>>(Nl, Sl[l], Nc, Sl[l + 1]);
    } else {
      mgk::k_sq_coarse<<<1, 32, 0, s>>>(Sl[l], block, S, c->cholInv);
    }
  }
  MG_CUDA(cudaGetLastError());
  c->launches += 2 * J;
  return MG_OK;
}

extern "C" mg_status mg_solve_blocks(mg_ctx* c, int32_t nblocks, const double* f, double* u,
                                     double tol, int32_t max_iter, int32_t* iters_out,
                                     double* relres_out, void* stream) {
  if (!c) return mgi::set_global_error(MG_ERR_INVALID, "mg_solve_blocks: ctx is NULL");
  if (c->sq_slots <= 0) return c->fail(MG_ERR_INVALID, "mg_solve_blocks: not a square context");
  if (!f || !u || max_iter < 0 || !(tol > 0.0) || nblocks < 1 || nblocks > c->sq_slots)
    return c->fail(MG_ERR_INVALID, "mg_solve_blocks: bad arguments");
  if ((const void*)f == (const void*)u) return c->fail(MG_ERR_INVALID, "mg_solve_blocks: f and u alias");
  if (!c->coarse_inv) return c->fail(MG_ERR_INVALID, "mg_solve_blocks: no coarsest inverse");
  cudaStream_t s = (cudaStream_t)stream;
  mg_status st = sync_params(c, s);
  if (st != MG_OK) return st;
  // The leading S of the context's blocks: at every level they are its
  // leading rows, so the cycle runs on views of the levels with fewer rows
  // and the strides of the whole level (blocks never couple).
  const int S = nblocks;
  const int m = c->n[0] / c->sq_slots;
  const int n0 = m * S;
  auto lead = [&](auto& all) {
    auto v = all;
    if (S == c->sq_slots) return v;
    for (auto& D : v) {
      D.ld = D.n;
      D.ldc = D.nc;
      D.n = D.n / c->sq_slots * S;
      D.nc = D.nc / c->sq_slots * S;
    }
    return v;
  };
  std::vector<DevLevel<float>> v32 = lead(c->d32);
  std::vector<DevLevel<double>> v64 = lead(c->d64);
  const dim3 bgrid((unsigned)((m + kThreads - 1) / kThreads), (unsigned)S);
  // the norm kernels: kBlkRows rows per thread
  const dim3 ngrid((unsigned)((m + kThreads * mgk::kBlkRows - 1) / (kThreads * mgk::kBlkRows)),
                   (unsigned)S);
  const int nchunk = (int)ngrid.x;
  const LV<double> L0 = v64[0].view();
  const bool p32 = c->prec == 32;
  c->solve_ctl[0] = tol;
  c->solve_ctl[1] = (double)max_iter;
  MG_CUDA(cudaMemcpyAsync(c->tol_dev, c->solve_ctl, 2 * sizeof(double), cudaMemcpyHostToDevice, s));
  if ((int64_t)nchunk * S > (int64_t)c->nblk_max * c->maxB)
    return c->fail(MG_ERR_INVALID, "mg_solve_blocks: partial-sum workspace too small");
  // per-block state arrays (active, iters, sexp, norms), allocated once for
  // all the context's blocks: the captured graphs of every block count keep
  // these pointers
  if (!c->blk_state) {
    MG_CUDA(cudaMalloc(&c->blk_state,
                       (size_t)c->sq_slots * (4 * sizeof(int) + 3 * sizeof(double))));
    c->maxB_blocks = c->sq_slots;
  }
  // per-block state in its own arrays (the context's per-rhs arrays are
  // sized for one column)
  const int SA = c->sq_slots;
  int* active = (int*)c->blk_state;
  int* iters = active + SA;
  int* sexp = iters + SA;
  int* sexp_prev = sexp + SA;
  double* rsum = (double*)(sexp_prev + SA);
  double* fsum = rsum + SA;
  double* relres = fsum + SA;
  auto check = [&](Issue<double>& is, cudaGraphConditionalHandle h, int inc, int cond) {
    is.launch(mgk::k_blk_resid64, ngrid, dim3(kThreads), 0, L0, f, (const double*)u,
              p32 ? c->rhat32 : (float*)nullptr, (const int*)sexp, m, S, c->partial,
              p32 ? c->d32[0].t : (float*)nullptr,
              p32 ? (const float*)c->d32[0].dinv : (const float*)nullptr, (const float*)c->prm32);
    if ((int64_t)S * nchunk <= kMergeReduceMax) {
      is.launch(mgk::k_reduce_check, dim3(1), dim3(kThreads), 0, (const double*)c->partial, nchunk,
                rsum, p32 ? sexp_prev : (int*)nullptr, (const double*)fsum, S,
                (const double*)c->tol_dev, active, relres, sexp, c->state, inc, h, cond);
    } else {
      is.launch(mgk::k_reduce, dim3(S), dim3(kThreads), 0, (const double*)c->partial, nchunk, S,
                rsum);
      if (p32) is.launch(k_shift_sexp, dim3(1), dim3(kThreads), 0, sexp, sexp_prev, S);
      is.launch(mgk::k_check, dim3(1), dim3(kThreads), 0, (const double*)rsum,
                (const double*)fsum, S, (const double*)c->tol_dev, active, relres, sexp,
                c->state, inc, h, cond);
    }
  };
  auto pre = [&](cudaStream_t cs, cudaGraphConditionalHandle h, int cond) {
    Issue<double> is{c, v64, c->prm64, cs, 1};
    is.launch(mgk::k_blk_sumsq, ngrid, dim3(kThreads), 0, f, m, S, c->partial);
    is.launch(mgk::k_reduce, dim3(S), dim3(kThreads), 0, (const double*)c->partial, nchunk, S,
              fsum);
    is.launch(k_init_solve, dim3((S + kThreads - 1) / kThreads), dim3(kThreads), 0,
              (const double*)fsum, S, active, iters, sexp);
    check(is, h, 0, cond);
    return is.nk;
  };
  auto body = [&](cudaStream_t cs, cudaGraphConditionalHandle h, int cond) {
    int nk = 0;
    if (p32) {
      Issue<float> is{c, v32, c->prm32, cs, 1};
      is.delta0_ready = true;  // check's k_blk_resid64 wrote the first step's delta
      is.rfold = mgk::RefineEp{u, sexp_prev, active, iters, m};
      is.vcycle(c->rhat32, c->c32, true);
      if (!is.rfold_done)
        is.launch(mgk::k_blk_refine_update, bgrid, dim3(kThreads), 0, u,
                  (const float*)c->c32, (const int*)sexp_prev, (const int*)active, m, S, iters);
      nk += is.nk;
      Issue<double> is2{c, v64, c->prm64, cs, 1};
      check(is2, h, 1, cond);
      nk += is2.nk;
    } else {
      Issue<double> is{c, v64, c->prm64, cs, 1};
      is.launch(mgk::k_copy<double>, grid_for((size_t)n0), dim3(kThreads), 0, (const double*)u,
                c->w64, (size_t)n0);
      is.vcycle(f, c->w64, false);
      is.launch(mgk::k_blk_masked_copy, bgrid, dim3(kThreads), 0, u,
                (const double*)c->w64, (const int*)active, m, S, iters);
      check(is, h, 1, cond);
      nk += is.nk;
    }
    return nk;
  };
  st = run_loop(c, 60, f, u, S, s, "mg_solve_blocks", pre, body,
                [](cudaStream_t) { return 0; }, false);
  if (st != MG_OK) return st;
  mg_status result = MG_OK;
  if (c->h_state[1])
    result = MG_ERR_DIVERGED;
  else if (c->h_state[0] > 0)
    result = MG_NOT_CONVERGED;
  if (iters_out) MG_CUDA(cudaMemcpyAsync(iters_out, iters, S * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (relres_out)
    MG_CUDA(cudaMemcpyAsync(relres_out, relres, S * sizeof(double), cudaMemcpyDeviceToHost, s));
  MG_CUDA(cudaStreamSynchronize(s));
  if (result == MG_ERR_DIVERGED) c->err = "mg_solve_blocks: non-finite residual";
  if (result == MG_NOT_CONVERGED) c->err = "mg_solve_blocks: tolerance not met within max_iter";
  return result;
}
