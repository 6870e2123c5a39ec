// Training entry points of libmg.so: checkpointed forward of K unrolled
// cycles, the hand-written adjoint of those cycles, and the residual loss.
// Included at the end of mg_api.cu (same translation unit).
//
// Checkpoints per cycle k (context precision T):
//   ck_u[k]      level-0 iterate entering cycle k
//   ck_f[k][l]   right-hand side of level l >= 1 (the restricted residual)
//   ck_e[k][l]   output of level l >= 1 (the coarse correction e_c)
// plus one copy of f.  The backward pass recomputes, level by level, the
// smoothing iterates from these (per-level checkpointing), so memory is
// O(K * sum_l n_l * B) instead of O(K * steps * n * B).

namespace {

template <class T>
std::vector<DevLevel<T>>& levels_of(mg_ctx* c);
template <>
std::vector<DevLevel<double>>& levels_of<double>(mg_ctx* c) { return c->d64; }
template <>
std::vector<DevLevel<float>>& levels_of<float>(mg_ctx* c) { return c->d32; }
template <class T>
const T* prm_of(mg_ctx* c);
template <>
const double* prm_of<double>(mg_ctx* c) { return c->prm64; }
template <>
const float* prm_of<float>(mg_ctx* c) { return c->prm32; }

mg_status train_alloc(mg_ctx* c, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess)
    return c->fail(e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,
                   std::string("training workspace: ") + cudaGetErrorString(e));
  c->tr_alloc.push_back(*p);
  return MG_OK;
}

void train_free(mg_ctx* c) {
  for (void* p : c->tr_alloc)
    if (p) cudaFree(p);
  c->tr_alloc.clear();
  c->ck_f.clear();
  c->ck_e.clear();
  c->bw_it.clear();
  c->ck_u.clear();
  c->bw_ubar.clear();
  c->bw_fbar.clear();
  c->bw_r.clear();
  c->bw_rbar.clear();
  c->ck_f0 = nullptr;
  c->bw_partial = nullptr;
  c->bw_partial_p = nullptr;
  c->bw_nblk = 0;
  c->bw_gp = nullptr;
  c->trK = c->trB = 0;
  c->tr_recorded = false;
}

mg_status ensure_train(mg_ctx* c, int K, int B) {
  if (c->trK == K && c->trB == B && c->tr_nu_pre == c->nu_pre && c->tr_nu_post == c->nu_post)
    return MG_OK;
  std::lock_guard<std::recursive_mutex> lk(mgi::setup_mutex());
  cudaDeviceSynchronize();
  // captured forward graphs point at the old checkpoint buffers
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
  c->graphs.clear();
  train_free(c);
  const size_t tb = c->prec == 64 ? 8 : 4;
  const int J = c->J;
  mg_status st;
  auto vec = [&](int lev, void** p) { return train_alloc(c, p, (size_t)c->n[lev] * B * tb); };
  c->ck_u.assign(K, nullptr);
  c->ck_f.assign(K, std::vector<void*>(J, nullptr));
  c->ck_e.assign(K, std::vector<void*>(J, nullptr));
  for (int k = 0; k < K; ++k) {
    if ((st = vec(0, &c->ck_u[k])) != MG_OK) return st;
    for (int l = 1; l < J; ++l) {
      if ((st = vec(l, &c->ck_f[k][l])) != MG_OK) return st;
      if ((st = vec(l, &c->ck_e[k][l])) != MG_OK) return st;
    }
  }
  if ((st = vec(0, &c->ck_f0)) != MG_OK) return st;
  const int nit = c->nu_pre + c->nu_post + 2;
  c->bw_it.assign(J, std::vector<void*>(nit, nullptr));
  c->bw_ubar.assign(J, nullptr);
  c->bw_fbar.assign(J, nullptr);
  c->bw_r.assign(J, nullptr);
  c->bw_rbar.assign(J, nullptr);
  for (int l = 0; l < J; ++l) {
    for (int k = 0; k < nit; ++k)
      if ((st = vec(l, &c->bw_it[l][k])) != MG_OK) return st;
    if ((st = vec(l, &c->bw_ubar[l])) != MG_OK) return st;
    if ((st = vec(l, &c->bw_fbar[l])) != MG_OK) return st;
    if ((st = vec(l, &c->bw_r[l])) != MG_OK) return st;
    if ((st = vec(l, &c->bw_rbar[l])) != MG_OK) return st;
  }
  const size_t nblk = ((size_t)c->n[0] * B + kThreads - 1) / kThreads + 1;
  if ((st = train_alloc(c, (void**)&c->bw_partial, nblk * 4 * sizeof(double))) != MG_OK) return st;
  if ((st = train_alloc(c, (void**)&c->bw_partial_p, (size_t)J * nblk * 2 * sizeof(double))) !=
      MG_OK)
    return st;
  c->bw_nblk = nblk;
  if ((st = train_alloc(c, (void**)&c->bw_gp, (size_t)(J - 1) * mgk::P_COUNT * sizeof(double))) !=
      MG_OK)
    return st;
  c->trK = K;
  c->trB = B;
  c->tr_nu_pre = c->nu_pre;
  c->tr_nu_post = c->nu_post;
  return MG_OK;
}

template <class T>
struct Backward {
  mg_ctx* c;
  Issue<T>& is;
  std::vector<DevLevel<T>>& L;
  cudaStream_t s;
  int B;
  double* grad;  // device [J-1][P_COUNT]
  int k = 0;     // cycle being reversed

  T* V(void* p) const { return (T*)p; }
  size_t vbytes(int lev) const { return (size_t)c->n[lev] * B * sizeof(T); }

  // One forward smoothing step uin -> uout (uout != uin), same arithmetic as
  // the forward cycle (the Issue launch forms: multi-rhs kernels when B > 1).
  // zero: uin is the zero vector (not read).
  void step(int lev, const T* f, const T* uin, T* uout, bool zero) {
    DevLevel<T>& D = L[lev];
    if (!is.conv(lev, mgk::P_WB2)) {
      is.op_jacobi(lev, f, uin, uout, zero);
    } else {
      if (zero)
        cudaMemsetAsync(uout, 0, vbytes(lev), s);
      else
        cudaMemcpyAsync(uout, uin, vbytes(lev), cudaMemcpyDeviceToDevice, s);
      is.op_residual(lev, f, uout, D.t, 1, zero);
      is.op_conv_update(lev, D.t, uout, zero);
    }
  }

  // A gradient job (adjoint.cuh GradJobs): the cross-block sums of a dot
  // kernel's nblk x Q partials into the level's entries a, b2, c2, d.
  void job(mgk::GradJobs& g, int j, const double* partial, int lev, int Q, size_t nblk, int a,
           int b2, int c2, int d) const {
    const int base = lev * mgk::P_COUNT;
    g.partial[j] = partial;
    g.nblk[j] = (int)nblk;
    g.Q[j] = Q;
    g.idx[j][0] = base + a;
    g.idx[j][1] = base + b2;
    g.idx[j][2] = base + (c2 < 0 ? a : c2);
    g.idx[j][3] = base + (d < 0 ? a : d);
    g.grad = grad;
  }
  static mgk::GradJobs no_jobs() {
    mgk::GradJobs g;
    std::memset(&g, 0, sizeof(g));
    return g;
  }
  // ubar -= A rbar, fbar += rbar, with the gradient jobs' sums in extra blocks
  void apply_a(int lev, T* ubar, const T* rbar, T* fbar, mgk::GradJobs acc) {
    DevLevel<T>& D = L[lev];
    if (const int bv = is.mbv()) {
      is.with_bv(bv, [&](auto kk) {
        const dim3 gm = is.mb_grid(D.n, bv);
        acc.nwork = (int)gm.x;
        is.launch(mgk::k_adj_apply_a_mb<T, decltype(kk)::value>,
                  dim3(gm.x + acc.Q[0] + acc.Q[1]), dim3(kThreads), 0, D.view(), ubar, rbar, fbar,
                  B, 0, acc);
      });
    } else {
      const dim3 g = grid_for((size_t)D.n * B);
      acc.nwork = (int)g.x;
      is.launch(mgk::k_adj_apply_a<T>, dim3(g.x + acc.Q[0] + acc.Q[1]), dim3(kThreads), 0,
                D.view(), ubar, rbar, fbar, B, 0, acc);
    }
  }

  // Adjoint of the smoothing step uin -> (next); ubar holds the adjoint of
  // the step's output on entry and of uin on exit; fbar accumulates.
  void adj_step(int lev, const T* f, const T* uin, bool zero, T* ubar, T* fbar) {
    DevLevel<T>& D = L[lev];
    const size_t work = (size_t)D.n * B;
    const dim3 g = grid_for(work);
    T* r = V(c->bw_r[lev]);
    T* rbar = V(c->bw_rbar[lev]);
    is.op_residual(lev, f, uin, r, 0, zero);
    mgk::GradJobs acc = no_jobs();
    if (const int bv = is.mbv()) {  // multi-rhs forms (B > 1)
      is.with_bv(bv, [&](auto kk) {
        constexpr int BV = decltype(kk)::value;
        const dim3 gm = is.mb_grid(D.n, bv);
        is.launch(mgk::k_adj_smooth_mb<T, BV>, gm, dim3(kThreads), 0, D.view(), (const T*)ubar,
                  (const T*)r, rbar, B, is.P(lev), c->bw_partial);
        job(acc, 0, c->bw_partial, lev, 4, gm.x, mgk::P_ETA, mgk::P_WB1, mgk::P_WB2,
            mgk::P_THETA);
      });
    } else {
      is.launch(mgk::k_adj_smooth<T>, g, dim3(kThreads), 0, D.view(), (const T*)ubar,
                (const T*)r, rbar, B, is.P(lev), c->bw_partial);
      job(acc, 0, c->bw_partial, lev, 4, g.x, mgk::P_ETA, mgk::P_WB1, mgk::P_WB2, mgk::P_THETA);
    }
    apply_a(lev, ubar, rbar, fbar, acc);
  }

  // Level lev of cycle k: ubar (adjoint of the level's output) -> adjoint of
  // its input u_in; fbar (zeroed by the caller) accumulates the adjoint of f.
  void level(int lev, const T* f, const T* uin, T* ubar, T* fbar) {
    const int J = c->J;
    if (lev == J - 1) {  // e = A_J^{-1} f  =>  fbar = A_J^{-1} ebar
      is.coarse(ubar, fbar);
      return;
    }
    DevLevel<T>& D = L[lev];
    const int np = c->nu_pre, nq = c->nu_post;
    std::vector<void*>& it = c->bw_it[lev];
    const bool zero_in = uin == nullptr;
    // forward recompute of this level's iterates
    if (zero_in)
      cudaMemsetAsync(it[0], 0, vbytes(lev), s);
    else
      cudaMemcpyAsync(it[0], uin, vbytes(lev), cudaMemcpyDeviceToDevice, s);
    for (int j = 0; j < np; ++j) step(lev, f, V(it[j]), V(it[j + 1]), zero_in && j == 0);
    const T* ec = V(c->ck_e[k][lev + 1]);
    if (is.conv(lev, mgk::P_WP2)) {  // P e_c per fine row, then Phi_P and the update
      is.op_pe(lev, ec, D.t);
      is.op_prolong(lev, D.t, V(it[np]), V(it[np + 1]), 1);
    } else {
      is.op_prolong(lev, ec, V(it[np]), V(it[np + 1]), 0);
    }
    for (int j = 0; j < nq; ++j) step(lev, f, V(it[np + 1 + j]), V(it[np + 2 + j]), false);
    // reverse: post-smoothing
    for (int j = nq - 1; j >= 0; --j) adj_step(lev, f, V(it[np + 1 + j]), false, ubar, fbar);
    // prolongation: ebar = P^T Phi_P^T ubar, dots <ubar, P e>, <ubar, M P e>
    T* ebar = V(c->bw_ubar[lev + 1]);
    const dim3 gf = grid_for((size_t)D.n * B);
    // g = Phi_P^T ubar per fine row, ebar = P^T g (the gather of the
    // restriction), P e per fine row for the dots; D.t and D.u2 are free here
    is.launch(mgk::k_adj_prolong_fine<T>, gf, dim3(kThreads), 0, D.view(), (const T*)ubar, D.t, B,
              is.P(lev));
    is.op_gather(lev, D.t, ebar, 0);
    is.op_pe(lev, ec, D.u2);
    // the dots go to this level's own partials: the coarse levels below
    // reuse bw_partial before the restriction adjoint sums them
    double* pdots = c->bw_partial_p + (size_t)lev * c->bw_nblk * 2;
    is.launch(mgk::k_adj_prolong_dots<T>, gf, dim3(kThreads), 0, D.view(), (const T*)ubar,
              (const T*)D.u2, B, pdots);
    // coarse level (its input iterate is zero)
    T* fcbar = V(c->bw_fbar[lev + 1]);
    cudaMemsetAsync(fcbar, 0, vbytes(lev + 1), s);
    level(lev + 1, V(c->ck_f[k][lev + 1]), nullptr, ebar, fcbar);
    // restriction: r = f - A u_pre, r_c = P^T Phi_R r
    T* r = V(c->bw_r[lev]);
    T* rbar = V(c->bw_rbar[lev]);
    is.op_residual(lev, f, V(it[np]), r, 0, zero_in && np == 0);
    is.op_pe(lev, fcbar, D.t);  // P rcbar per fine row
    is.launch(mgk::k_adj_restrict<T>, gf, dim3(kThreads), 0, D.view(), (const T*)D.t,
              (const T*)r, rbar, B, is.P(lev), c->bw_partial);
    mgk::GradJobs acc = no_jobs();
    job(acc, 0, c->bw_partial, lev, 2, gf.x, mgk::P_WR1, mgk::P_WR2, -1, -1);
    job(acc, 1, pdots, lev, 2, gf.x, mgk::P_WP1, mgk::P_WP2, -1, -1);
    apply_a(lev, ubar, rbar, fbar, acc);
    // reverse: pre-smoothing
    for (int j = np - 1; j >= 0; --j) adj_step(lev, f, V(it[j]), zero_in && j == 0, ubar, fbar);
  }
};

template <class T>
mg_status forward_record(mg_ctx* c, const T* f, T* u, int B, int K, cudaStream_t s) {
  mg_status st = ensure_train(c, K, B);
  if (st != MG_OK) return st;
  MG_CUDA(cudaMemcpyAsync(c->ck_f0, f, (size_t)c->n[0] * B * sizeof(T), cudaMemcpyDeviceToDevice,
                          s));
  const int J = c->J;
  std::vector<std::vector<T*>> fo(K, std::vector<T*>(J, nullptr)), uo(K, std::vector<T*>(J, nullptr));
  for (int k = 0; k < K; ++k)
    for (int l = 1; l < J; ++l) {
      fo[k][l] = (T*)c->ck_f[k][l];
      uo[k][l] = (T*)c->ck_e[k][l];
    }
  auto key = std::make_tuple(1000 + K, (const void*)f, (const void*)u, B, c->structure);
  st = run_graph(c, key, s, [&](cudaStream_t cs) {
    Issue<T> is{c, levels_of<T>(c), prm_of<T>(c), cs, B};
    for (int k = 0; k < K; ++k) {
      cudaMemcpyAsync(c->ck_u[k], u, (size_t)c->n[0] * B * sizeof(T), cudaMemcpyDeviceToDevice, cs);
      is.fov = fo[k].data();
      is.uov = uo[k].data();
      is.vcycle((const T*)c->ck_f0, u, false);
    }
    return is.nk;
  });
  if (st != MG_OK) return st;
  c->tr_recorded = true;
  c->rec_version = c->param_version;
  return MG_OK;
}

template <class T>
mg_status backward(mg_ctx* c, int K, const T* gout, T* gin, T* gf, double* gparams,
                   cudaStream_t s) {
  const int B = c->trB;
  const size_t v0 = (size_t)c->n[0] * B * sizeof(T);
  const size_t gpb = (size_t)(c->J - 1) * mgk::P_COUNT * sizeof(double);
  T* ubar = (T*)c->bw_ubar[0];
  T* fbar0 = (T*)c->bw_fbar[0];
  MG_CUDA(cudaMemcpyAsync(ubar, gout, v0, cudaMemcpyDeviceToDevice, s));
  // The reverse pass (about 40 kernels per level and cycle) touches context
  // buffers only, so it is captured once per (K, B, convolution structure)
  // and replayed; the caller's buffers are copied in before and out after.
  auto key = std::make_tuple(2000 + K, (const void*)c->bw_gp, (const void*)ubar, B, c->structure);
  mg_status st = run_graph(c, key, s, [&](cudaStream_t cs) {
    cudaMemsetAsync(c->bw_gp, 0, gpb, cs);
    cudaMemsetAsync(fbar0, 0, v0, cs);
    Issue<T> is{c, levels_of<T>(c), prm_of<T>(c), cs, B};
    Backward<T> bw{c, is, levels_of<T>(c), cs, B, c->bw_gp};
    for (int k = K - 1; k >= 0; --k) {
      bw.k = k;
      bw.level(0, (const T*)c->ck_f0, (const T*)c->ck_u[k], ubar, fbar0);
    }
    return is.nk;
  });
  if (st != MG_OK) return st;
  MG_CUDA(cudaMemcpyAsync(gparams, c->bw_gp, gpb, cudaMemcpyDeviceToDevice, s));
  if (gf) MG_CUDA(cudaMemcpyAsync(gf, fbar0, v0, cudaMemcpyDeviceToDevice, s));
  if (gin) MG_CUDA(cudaMemcpyAsync(gin, ubar, v0, cudaMemcpyDeviceToDevice, s));
  return MG_OK;
}

template <class T>
mg_status residual_loss(mg_ctx* c, const T* f, const T* u, int B, const double* w, double* loss,
                        double* per_rhs, T* grad_u, cudaStream_t s) {
  DevLevel<T>& D = levels_of<T>(c)[0];
  const int bt = std::min(B, 32);
  const int nblk = (D.n + mgk::kRedRows - 1) / mgk::kRedRows;
  T* r = grad_u ? D.t : nullptr;
  mgk::k_loss_resid<T><<<dim3(nblk, (B + bt - 1) / bt), mgk::kRedRows * bt, 0, s>>>(
      D.view(), f, u, r, B, c->partial);
  mgk::k_reduce<<<B, kThreads, 0, s>>>(c->partial, nblk, B, c->rsum);
  mgk::k_loss_combine<<<1, 32, 0, s>>>(c->rsum, w, B, loss, per_rhs);
  int nk = 3;
  if (grad_u) {
    mgk::k_loss_grad<T><<<grid_for((size_t)D.n * B), kThreads, 0, s>>>(D.view(), D.t, w, grad_u, B);
    ++nk;
  }
  MG_CUDA(cudaGetLastError());
  c->launches += nk;
  return MG_OK;
}

}  // namespace

extern "C" mg_status mg_forward_record(mg_ctx* c, const void* f, void* u, int32_t B, int32_t K,
                                       void* stream) {
  if (!c) return mgi::set_global_error(MG_ERR_INVALID, "mg_forward_record: ctx is NULL");
  if (!f || !u || f == u || B < 1 || B > c->maxB || K < 1 || K > 1000)
    return c->fail(MG_ERR_INVALID, "mg_forward_record: bad arguments");
  if (c->cheb_K > 0)
    return c->fail(MG_ERR_INVALID,
                   "mg_forward_record: the adjoint covers the SAGEConv smoother, not ChebConv "
                   "(mg_set_cheb degree > 0)");
  cudaStream_t s = (cudaStream_t)stream;
  mg_status st = sync_params(c, s);
  if (st != MG_OK) return st;
  if (c->prec == 64) return forward_record<double>(c, (const double*)f, (double*)u, B, K, s);
  return forward_record<float>(c, (const float*)f, (float*)u, B, K, s);
}

extern "C" mg_status mg_vcycle_backward(mg_ctx* c, int32_t K, const void* gout, void* gin, void* gf,
                                        double* gparams, void* stream) {
  if (!c) return mgi::set_global_error(MG_ERR_INVALID, "mg_vcycle_backward: ctx is NULL");
  if (!c->tr_recorded) return c->fail(MG_ERR_STATE, "mg_vcycle_backward: no recorded forward");
  if (K != c->trK) return c->fail(MG_ERR_STATE, "mg_vcycle_backward: n_cycles differs from the recorded forward");
  if (c->rec_version != c->param_version)
    return c->fail(MG_ERR_STATE, "mg_vcycle_backward: parameters changed since the forward");
  if (!gout || !gparams) return c->fail(MG_ERR_INVALID, "mg_vcycle_backward: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  if (c->prec == 64)
    return backward<double>(c, K, (const double*)gout, (double*)gin, (double*)gf, gparams, s);
  return backward<float>(c, K, (const float*)gout, (float*)gin, (float*)gf, gparams, s);
}

extern "C" mg_status mg_residual_loss(mg_ctx* c, const void* f, const void* u, int32_t B,
                                      const double* w, double* loss, double* per_rhs, void* grad_u,
                                      void* stream) {
  if (!c) return mgi::set_global_error(MG_ERR_INVALID, "mg_residual_loss: ctx is NULL");
  if (!f || !u || B < 1 || B > c->maxB || (grad_u && !w) || (loss && !w))
    return c->fail(MG_ERR_INVALID, "mg_residual_loss: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  if (c->prec == 64)
    return residual_loss<double>(c, (const double*)f, (const double*)u, B, w, loss, per_rhs,
                                 (double*)grad_u, s);
  return residual_loss<float>(c, (const float*)f, (const float*)u, B, w, loss, per_rhs,
                              (float*)grad_u, s);
}
