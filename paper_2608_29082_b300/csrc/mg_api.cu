// libmg.so: context, device set-up and the learnable V-cycle driver.
//
// One mg_ctx holds a hierarchy on one GPU.  The V-cycle (Algorithm 2) is
// issued as a fixed sequence of level kernels, captured once per (buffers,
// batch) into a CUDA graph and replayed; parameters live in device memory so
// that changing Theta (training) does not invalidate the graphs.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "adjoint.cuh"
#include "gmres.cuh"
#include "halo.cuh"
#include "halo_sell.cuh"
#include "kernels.cuh"
#include "krylov.cuh"
#include "multi_rhs.cuh"
#include "square.cuh"
#include "mg.h"
#include "mg_internal.h"

using mgk::kThreads;
using mgk::LV;

// ------------------------------------------------------------ errors ------

namespace {
std::mutex g_err_mu;
std::string g_err;
}  // namespace

namespace mgi {
std::recursive_mutex& setup_mutex() {
  static std::recursive_mutex m;
  return m;
}

mg_status set_global_error(mg_status s, const std::string& msg) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err = msg;
  return s;
}
const std::string& global_error() { return g_err; }
}  // namespace mgi

// ------------------------------------------------------- host packing -----

namespace {

struct HostLevel {
  int n = 0, nc = 0, KR = 0, ndia = 0;
  int doff[mgk::kMaxDia] = {0};
  std::vector<int> sl_ptr, col, p_idx, r_idx;
  std::vector<double> val, diag, dinv, invdeg, p_w, r_w, dval;
};

// 0: DIA where a level's off-diagonals lie on at most kMaxDia diagonals,
// SELL-32 elsewhere; 1: SELL-32 everywhere (mg_set_layout_policy).
int g_layout_policy = 0;

template <class T>
struct DevLevel {
  int n = 0, nc = 0, KR = 0, nsl = 0, ndia = 0;
  // row strides of the [k][.] arrays when they differ from n / nc (a view of
  // the leading blocks of a stacked level; 0: n / nc)
  int ld = 0, ldc = 0;
  int doff[mgk::kMaxDia] = {0};
  size_t nent = 0;
  int *sl_ptr = nullptr, *col = nullptr, *p_idx = nullptr, *r_idx = nullptr;
  T *val = nullptr, *diag = nullptr, *dinv = nullptr, *invdeg = nullptr, *p_w = nullptr,
    *r_w = nullptr, *dval = nullptr;
  unsigned char* nbm = nullptr;  // DIA levels: per-row mask of the nonzero off-diagonals (in T)
  T *u = nullptr, *f = nullptr, *t = nullptr, *u2 = nullptr;  // workspace [n][maxB]
  // SELL levels: halo tables of the fused steps (halo_sell.cuh) for tiles of
  // hs_tr rows (0: none), and the host copy of the SELL pattern they are
  // rebuilt from when the tile size changes
  int hs_tr = 0, hs_hmax = 0;
  int *hs_ptr = nullptr, *hs_row = nullptr;
  int16_t* hs_lcol = nullptr;
  std::vector<int> h_slptr, h_col;
  mgk::SellHalo halo() const { return mgk::SellHalo{hs_tr, hs_ptr, hs_row, hs_lcol}; }
  LV<T> view() const {
    LV<T> v;
    v.n = n;
    v.nc = nc;
    v.ld = ld ? ld : n;
    v.ldc = ldc ? ldc : nc;
    v.KR = KR;
    v.ndia = ndia;
    for (int k = 0; k < mgk::kMaxDia; ++k) v.doff[k] = doff[k];
    v.dval = dval;
    v.sl_ptr = sl_ptr;
    v.col = col;
    v.val = val;
    v.diag = diag;
    v.dinv = dinv;
    v.invdeg = invdeg;
    v.p_idx = p_idx;
    v.p_w = p_w;
    v.r_idx = r_idx;
    v.r_w = r_w;
    v.nbm = nbm;
    return v;
  }
};

template <class T>
void free_level(DevLevel<T>& L) {
  void* ptrs[] = {L.sl_ptr, L.col, L.p_idx, L.r_idx, L.val,  L.diag,   L.dinv,  L.invdeg, L.p_w,
                  L.r_w,    L.u,   L.f,     L.t,     L.u2,   L.dval,   L.hs_ptr, L.hs_row,
                  L.hs_lcol, L.nbm};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  L = DevLevel<T>();
}

std::string csr_check(const mg_csr& A, int nr, int nc, const char* what) {
  char buf[256];
  if (A.n_rows != nr || A.n_cols != nc) {
    snprintf(buf, sizeof buf, "%s: expected %d x %d, got %d x %d", what, nr, nc, A.n_rows,
             A.n_cols);
    return buf;
  }
  if (!A.rowptr || (A.nnz > 0 && (!A.col || !A.val)) || A.rowptr[0] != 0 ||
      A.rowptr[nr] != A.nnz)
    return std::string(what) + ": inconsistent CSR arrays";
  for (int i = 0; i < nr; ++i)
    if (A.rowptr[i + 1] < A.rowptr[i]) return std::string(what) + ": rowptr not monotone";
  for (int k = 0; k < A.nnz; ++k)
    if (A.col[k] < 0 || A.col[k] >= nc) return std::string(what) + ": column out of range";
  return "";
}

// SELL-32 packing of the off-diagonal part; transfer lists.
std::string pack_level(const mg_csr& A, const double* invdeg, const mg_csr* P, HostLevel& H) {
  const int n = A.n_rows;
  H.n = n;
  H.diag.assign(n, 0.0);
  H.dinv.assign(n, 0.0);
  H.invdeg.assign(invdeg, invdeg + n);
  std::vector<int> cnt(n, 0);
  for (int i = 0; i < n; ++i)
    for (int k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
      if (A.col[k] == i)
        H.diag[i] += A.val[k];
      else if (A.val[k] != 0.0)
        cnt[i]++;
    }
  for (int i = 0; i < n; ++i) {
    if (!(H.diag[i] > 0.0)) return "operator has a non-positive diagonal entry";
    if (!(invdeg[i] > 0.0) || !std::isfinite(invdeg[i])) return "inv_deg must be positive";
    H.dinv[i] = 1.0 / H.diag[i];
  }
  // DIA when the off-diagonals lie on few diagonals (ascending offsets keep
  // the column order of the CSR rows, hence the same accumulation order)
  std::vector<int> offs;
  bool dia = g_layout_policy == 0;
  for (int i = 0; i < n && dia; ++i)
    for (int k = A.rowptr[i]; k < A.rowptr[i + 1] && dia; ++k) {
      if (k > A.rowptr[i] && A.col[k] <= A.col[k - 1]) dia = false;  // unsorted or duplicate
      if (!dia || A.col[k] == i || A.val[k] == 0.0) continue;
      const int o = A.col[k] - i;
      if (std::find(offs.begin(), offs.end(), o) == offs.end()) {
        if ((int)offs.size() == mgk::kMaxDia)
          dia = false;
        else
          offs.push_back(o);
      }
    }
  if (dia && !offs.empty()) {
    std::sort(offs.begin(), offs.end());
    H.ndia = (int)offs.size();
    for (int k = 0; k < H.ndia; ++k) H.doff[k] = offs[k];
    H.dval.assign((size_t)H.ndia * n, 0.0);
    for (int i = 0; i < n; ++i)
      for (int k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
        if (A.col[k] == i || A.val[k] == 0.0) continue;
        const int d = (int)(std::find(offs.begin(), offs.end(), A.col[k] - i) - offs.begin());
        H.dval[(size_t)d * n + i] = A.val[k];
      }
  }
  const int nsl = H.ndia > 0 ? 0 : (n + mgk::kSlice - 1) / mgk::kSlice;
  H.sl_ptr.assign(nsl + 1, 0);
  for (int s = 0; s < nsl; ++s) {
    int K = 0;
    for (int i = s * 32; i < std::min(n, s * 32 + 32); ++i) K = std::max(K, cnt[i]);
    H.sl_ptr[s + 1] = H.sl_ptr[s] + 32 * K;
  }
  H.col.assign(H.sl_ptr[nsl], -1);
  H.val.assign(H.sl_ptr[nsl], 0.0);
  for (int i = 0; i < n && H.ndia == 0; ++i) {
    int k = 0;
    const int base = H.sl_ptr[i / 32] + (i % 32);
    for (int e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      if (A.col[e] == i || A.val[e] == 0.0) continue;
      H.col[base + 32 * k] = A.col[e];
      H.val[base + 32 * k] = A.val[e];
      ++k;
    }
  }
  if (P) {
    const int nc = P->n_cols;
    H.nc = nc;
    H.p_idx.assign(2 * (size_t)n, -1);
    H.p_w.assign(2 * (size_t)n, 0.0);
    std::vector<int> ccount(nc, 0);
    for (int i = 0; i < n; ++i) {
      int k = 0;
      for (int e = P->rowptr[i]; e < P->rowptr[i + 1]; ++e) {
        if (P->val[e] == 0.0) continue;
        if (k == 2) return "prolongation rows may hold at most 2 entries";
        H.p_idx[(size_t)k * n + i] = P->col[e];
        H.p_w[(size_t)k * n + i] = P->val[e];
        ccount[P->col[e]]++;
        ++k;
      }
    }
    int KR = 0;
    for (int I = 0; I < nc; ++I) KR = std::max(KR, ccount[I]);
    H.KR = KR;
    H.r_idx.assign((size_t)KR * nc, -1);
    H.r_w.assign((size_t)KR * nc, 0.0);
    std::vector<int> fill(nc, 0);
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < 2; ++k) {
        const int I = H.p_idx[(size_t)k * n + i];
        if (I < 0) continue;
        H.r_idx[(size_t)fill[I] * nc + I] = i;
        H.r_w[(size_t)fill[I] * nc + I] = H.p_w[(size_t)k * n + i];
        fill[I]++;
      }
  }
  return "";
}

// Halo tables of a SELL level for tiles of TR rows (halo_sell.cuh): per tile
// the ascending list of outside rows that neighbour a tile row, and per SELL
// entry of a tile row the local slot of its column.  Returns false when a
// tile's slots would not fit int16 (the kernel then is not used).
bool build_sell_halo(int n, const std::vector<int>& sl_ptr, const std::vector<int>& col, int TR,
                     std::vector<int>& hptr, std::vector<int>& hrow, std::vector<int16_t>& lcol,
                     int& hmax) {
  const int ntiles = (n + TR - 1) / TR;
  hptr.assign(1, 0);
  hrow.clear();
  lcol.assign(col.size(), (int16_t)-1);
  hmax = 0;
  std::vector<int> ext;
  for (int t = 0; t < ntiles; ++t) {
    const int r0 = t * TR, r1 = std::min(n, r0 + TR);
    ext.clear();
    for (int i = r0; i < r1; ++i)
      for (int e = sl_ptr[i >> 5] + (i & 31); e < sl_ptr[(i >> 5) + 1]; e += mgk::kSlice) {
        const int c = col[e];
        if (c >= 0 && (c < r0 || c >= r1)) ext.push_back(c);
      }
    std::sort(ext.begin(), ext.end());
    ext.erase(std::unique(ext.begin(), ext.end()), ext.end());
    if ((r1 - r0) + (int64_t)ext.size() > 32767) return false;
    for (int i = r0; i < r1; ++i)
      for (int e = sl_ptr[i >> 5] + (i & 31); e < sl_ptr[(i >> 5) + 1]; e += mgk::kSlice) {
        const int c = col[e];
        if (c < 0) continue;
        const int slot = (c >= r0 && c < r1)
                             ? c - r0
                             : (r1 - r0) + (int)(std::lower_bound(ext.begin(), ext.end(), c) -
                                                 ext.begin());
        lcol[e] = (int16_t)slot;
      }
    hrow.insert(hrow.end(), ext.begin(), ext.end());
    hptr.push_back((int)hrow.size());
    hmax = std::max(hmax, (int)ext.size());
  }
  return true;
}

// Dense FP64 Cholesky A = L L^T (column-major L).  Returns false if A is not
// numerically SPD.
bool cholesky(const mg_csr& A, std::vector<double>& Lc) {
  const int n = A.n_rows;
  Lc.assign((size_t)n * n, 0.0);
  std::vector<double> M((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) M[(size_t)i * n + A.col[k]] += A.val[k];
  for (int j = 0; j < n; ++j) {
    double d = M[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= Lc[j + (size_t)k * n] * Lc[j + (size_t)k * n];
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    Lc[j + (size_t)j * n] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double s = M[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= Lc[i + (size_t)k * n] * Lc[j + (size_t)k * n];
      Lc[i + (size_t)j * n] = s / ljj;
    }
  }
  return true;
}

// Explicit inverse of the coarsest operator from its Cholesky factor
// (column-major L): A^{-1} e_k by the two substitutions for every k, then
// symmetrised; row-major.  Empty when the 1-norm condition number
// ||A||_1 ||A^{-1}||_1 exceeds 1e6 (the substitutions are kept there: an
// explicit inverse loses about cond(A) units of rounding).
std::vector<double> coarse_inverse(const mg_csr& A, const std::vector<double>& Lc, int n) {
  std::vector<double> X((size_t)n * n, 0.0), y(n);
  for (int k = 0; k < n; ++k) {
    std::fill(y.begin(), y.end(), 0.0);
    y[k] = 1.0;
    for (int j = 0; j < n; ++j) {  // L y = e_k
      y[j] /= Lc[j + (size_t)j * n];
      for (int i = j + 1; i < n; ++i) y[i] -= Lc[i + (size_t)j * n] * y[j];
    }
    for (int j = n - 1; j >= 0; --j) {  // L^T x = y
      y[j] /= Lc[j + (size_t)j * n];
      for (int i = 0; i < j; ++i) y[i] -= Lc[j + (size_t)i * n] * y[j];
    }
    for (int i = 0; i < n; ++i) X[(size_t)i * n + k] = y[i];
  }
  double an = 0.0, in = 0.0;
  std::vector<double> colsum(n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) colsum[A.col[k]] += std::fabs(A.val[k]);
  for (double v : colsum) an = std::max(an, v);
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += std::fabs(X[(size_t)i * n + k]);
    in = std::max(in, s);
  }
  if (!(an * in <= 1e6)) return {};
  for (int i = 0; i < n; ++i)
    for (int k = i + 1; k < n; ++k) {
      const double m = 0.5 * (X[(size_t)i * n + k] + X[(size_t)k * n + i]);
      X[(size_t)i * n + k] = X[(size_t)k * n + i] = m;
    }
  return X;
}

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  int nkernels = 0;  // kernels per launch (outside any loop body)
  int nbody = 0;     // kernels per iteration of a while-node body
};

}  // namespace

// ------------------------------------------------------------ context -----

struct mg_ctx {
  int J = 0, prec = 64, maxB = 1, nJ = 0;
  std::vector<int> n;
  std::vector<DevLevel<double>> d64;
  std::vector<DevLevel<float>> d32;
  double *cholL = nullptr, *cholU = nullptr, *cholDinv = nullptr;
  double* cholP = nullptr;  // packed column-major lower triangle of the factor
  // explicit inverse of A_J (row-major), formed at set-up when the coarsest
  // level is 32..512 rows and well conditioned; used when coarse_inv is set
  double* cholInv = nullptr;
  bool coarse_inv = false;
  // stacked square-mesh contexts (square_impl.cuh): requests per context
  // (0: an ordinary context), vertices per side per level, the set-up
  // scratch (7-point stencils over all vertices of every level) and the
  // per-block solve state
  int sq_slots = 0;
  std::vector<int> sq_N;
  double* sq_scratch = nullptr;
  void* blk_state = nullptr;
  int maxB_blocks = 0;
  // flexible-CG workspace (allocated on first use): r, z, p, q [n0][maxB]
  double *k_r = nullptr, *k_z = nullptr, *k_p = nullptr, *k_q = nullptr;
  double *k_partial = nullptr, *k_small = nullptr;
  // FCG with FP32 vectors (precision-32 contexts): p, q, e [n0][maxB] in
  // FP32 (r and z are rhat32 and c32), per-rhs alpha, beta, (p, q), rr0
  // (double) and fresh, restart flags and the any-restart flag (int)
  float *k32_p = nullptr, *k32_q = nullptr, *k32_e = nullptr;
  void* k32_small = nullptr;
  // flexible GMRES workspace (mg_solve_fgmres), for restart length gm_m:
  // basis and directions in the context precision (gm_V, gm_Z: void), an
  // FP32 zero vector (the right-hand side of w = 0 - A z), per-rhs cycle ends
  int gm_m = 0;
  void *gm_V = nullptr, *gm_Z = nullptr;
  float* gm_zero32 = nullptr;
  double *gm_small = nullptr, *gm_h = nullptr, *gm_vec = nullptr, *gm_partial = nullptr;
  int* gm_done = nullptr;
  int nu_pre = 2, nu_post = 2;
  std::vector<double> prm;  // [J-1][P_COUNT]
  double* prm64 = nullptr;
  float* prm32 = nullptr;
  bool prm_dirty = true;
  // ChebConv smoother (mg_set_cheb): degree (0: SAGEConv), coefficients
  // [J][MG_CHEB_MAX_DEGREE + 1] on the host and, in the context precision,
  // on the device
  int cheb_K = 0;
  std::vector<double> cheb_host;
  void* cheb_dev = nullptr;
  bool cheb_dirty = false;
  uint32_t structure = 0;
  // outer-loop workspace
  int nblk_max = 0;
  double *partial = nullptr, *rsum = nullptr, *fsum = nullptr, *relres = nullptr, *w64 = nullptr;
  int *active = nullptr, *iters = nullptr, *sexp = nullptr, *sexp_prev = nullptr,
      *state = nullptr;
  float *c32 = nullptr, *rhat32 = nullptr;
  int* h_state = nullptr;  // pinned [2]
  double* tol_dev = nullptr;      // device [3]: tol, max_iter, and a loop's own bound
  double solve_ctl[3] = {0, 0, 0};  // host staging of tol_dev
  double *hf = nullptr, *hu = nullptr;  // device buffers for mg_solve_host
  cudaStream_t cap = nullptr;
  std::map<std::tuple<int, const void*, const void*, int, uint32_t>, GraphEntry> graphs;
  std::string err;
  int64_t launches = 0;
  // options (mg_set_option)
  int64_t opt_tail_work = 2048;  // rows x rhs at or below which levels run in k_tail
  int opt_tail_teams = 1;  // k_tail levels by teams of warps, entries per thread (0: whole block)
  int opt_pdl = 1;               // programmatic dependent launch between kernels
  int opt_multi_rhs = 1;         // multi-rhs kernels: 0 off, 1 widest tile, else max tile
  int opt_device_loop = 1;       // solve loops as while nodes (0: host-driven plain graphs)
  int opt_fcg_precond = 0;       // preconditioner of mg_solve_fcg: 0 V-cycle, 1 full multigrid
  int opt_fgmres_floor = 4;      // FP32 FGMRES cycle floor, 10^-value (0: none)
  // precision-32 FCG: 1 FP32 vectors + FP64 restarts, 0 FP64 vectors, 2 FP32
  // vectors from kFcg32Rows level-0 rows on
  int opt_fcg_fp32 = 2;
  int opt_fcg_floor = 2;         // its phase floor, 10^-value (0: none)
  int64_t opt_halo_rows = 256;   // rows per block of the halo-fused DIA steps (0: unfused)
  // DIA levels whose vectors (rows x rhs x value bytes) are at least this
  // large use the 2D-tiled fused steps (0: never; measured slower than the
  // two-kernel form on the large stacked levels, so off)
  int64_t opt_halo2d_bytes = 0;
  int opt_dia_two_rows = 1;  // one rhs: two rows per thread (k_*_dia2r, k_pe2r)
  int opt_sell_halo_rows = 0;  // rows per tile of the halo-fused SELL steps (0: unfused)
  int opt_sell_halo_threads = 256;  // threads per block of those steps
  // largest level vector (rows x rhs x value bytes) whose smoothing and
  // restriction steps use the SELL halo form (prolongation: every level)
  int64_t opt_sell_halo_max_bytes = INT64_MAX;
  int64_t wave_threads = 148 * 2048;  // SMs x resident threads per SM (set in mg_setup)
  // training state (device buffers in the context precision)
  int64_t param_version = 0, rec_version = -1;
  int trK = 0, trB = 0, tr_nu_pre = -1, tr_nu_post = -1;
  bool tr_recorded = false;
  std::vector<void*> tr_alloc;
  std::vector<std::vector<void*>> ck_f, ck_e, bw_it;  // [K][J], [K][J], [J][nu_pre+nu_post+2]
  std::vector<void*> ck_u, bw_ubar, bw_fbar, bw_r, bw_rbar;
  void* ck_f0 = nullptr;
  double* bw_partial = nullptr;
  // per level: the prolongation-adjoint dots, summed into the gradient by
  // the same level's restriction adjoint (after the coarse levels ran)
  double* bw_partial_p = nullptr;
  size_t bw_nblk = 0;
  double* bw_gp = nullptr;  // parameter gradients of the captured backward [J-1][P_COUNT]

  mg_status fail(mg_status s, const std::string& m) {
    err = m;
    return s;
  }
};

#define MG_CUDA(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return c->fail(e_ == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,          \
                     std::string(#call) + ": " + cudaGetErrorString(e_));                 \
  } while (0)

namespace {

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
  if (src.empty()) {
    *dst = nullptr;
    return cudaSuccess;
  }
  cudaError_t e = cudaMalloc((void**)dst, src.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

template <class T>
std::vector<T> cast(const std::vector<double>& v) {
  return std::vector<T>(v.begin(), v.end());
}

template <class T>
cudaError_t upload_level(const HostLevel& H, DevLevel<T>& D, int maxB, bool vectors) {
  cudaError_t e;
  D.n = H.n;
  D.nc = H.nc;
  D.KR = H.KR;
  D.nsl = (int)H.sl_ptr.size() - 1;
  D.nent = H.col.size();
  D.ndia = H.ndia;
  for (int k = 0; k < mgk::kMaxDia; ++k) D.doff[k] = H.doff[k];
  if ((e = upload(&D.dval, cast<T>(H.dval))) != cudaSuccess) return e;
  if (H.ndia > 0) {  // bit k: off-diagonal k of the row is nonzero once rounded to T
    std::vector<unsigned char> m((size_t)H.n, 0);
    for (int k = 0; k < H.ndia; ++k)
      for (int i = 0; i < H.n; ++i)
        if ((T)H.dval[(size_t)k * H.n + i] != T(0)) m[i] |= (unsigned char)(1u << k);
    if ((e = upload(&D.nbm, m)) != cudaSuccess) return e;
  }
  if ((e = upload(&D.sl_ptr, H.sl_ptr)) != cudaSuccess) return e;
  if ((e = upload(&D.col, H.col)) != cudaSuccess) return e;
  if ((e = upload(&D.val, cast<T>(H.val))) != cudaSuccess) return e;
  if ((e = upload(&D.diag, cast<T>(H.diag))) != cudaSuccess) return e;
  if ((e = upload(&D.dinv, cast<T>(H.dinv))) != cudaSuccess) return e;
  if ((e = upload(&D.invdeg, cast<T>(H.invdeg))) != cudaSuccess) return e;
  if ((e = upload(&D.p_idx, H.p_idx)) != cudaSuccess) return e;
  if ((e = upload(&D.p_w, cast<T>(H.p_w))) != cudaSuccess) return e;
  if ((e = upload(&D.r_idx, H.r_idx)) != cudaSuccess) return e;
  if ((e = upload(&D.r_w, cast<T>(H.r_w))) != cudaSuccess) return e;
  if (vectors) {
    const size_t bytes = (size_t)H.n * maxB * sizeof(T);
    for (T** p : {&D.u, &D.f, &D.t, &D.u2}) {
      if ((e = cudaMalloc((void**)p, bytes)) != cudaSuccess) return e;
      if ((e = cudaMemset(*p, 0, bytes)) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// (Re)builds the SELL halo tables of levels 0..J-2 for tiles of TR rows (0:
// frees them).  Levels stored as DIA, levels without workspace vectors (the
// FP64 finest copy of an FP32 context) and levels whose tiles do not fit the
// kernel's int16 slots keep the two-kernel form.  The caller makes sure no
// work that reads the old tables is in flight.
template <class T>
cudaError_t upload_sell_halo(std::vector<DevLevel<T>>& Ls, int TR, int J) {
  for (int l = 0; l < J - 1 && l < (int)Ls.size(); ++l) {
    DevLevel<T>& D = Ls[l];
    for (void* p : {(void*)D.hs_ptr, (void*)D.hs_row, (void*)D.hs_lcol})
      if (p) cudaFree(p);
    D.hs_ptr = D.hs_row = nullptr;
    D.hs_lcol = nullptr;
    D.hs_tr = D.hs_hmax = 0;
    if (TR <= 0 || D.ndia > 0 || D.h_col.empty() || !D.u) continue;
    std::vector<int> hptr, hrow;
    std::vector<int16_t> lcol;
    int hmax = 0;
    if (!build_sell_halo(D.n, D.h_slptr, D.h_col, TR, hptr, hrow, lcol, hmax)) continue;
    cudaError_t e;
    if ((e = upload(&D.hs_ptr, hptr)) != cudaSuccess) return e;
    if ((e = upload(&D.hs_row, hrow)) != cudaSuccess) return e;
    if ((e = upload(&D.hs_lcol, lcol)) != cudaSuccess) return e;
    D.hs_tr = TR;
    D.hs_hmax = hmax;
  }
  return cudaSuccess;
}

uint32_t structure_of(const std::vector<double>& prm, int J) {
  uint32_t s = 0;
  for (int l = 0; l < J - 1 && l < 10; ++l) {
    const double* p = &prm[(size_t)l * mgk::P_COUNT];
    s |= (p[mgk::P_WB2] != 0.0 ? 1u : 0u) << (3 * l);
    s |= (p[mgk::P_WR2] != 0.0 ? 1u : 0u) << (3 * l + 1);
    s |= (p[mgk::P_WP2] != 0.0 ? 1u : 0u) << (3 * l + 2);
  }
  if (J - 1 > 10) s |= 1u << 31;  // deep hierarchies: recapture on every change
  return s;
}

std::string read_params(const mg_params* p, int J, std::vector<double>& out, int& nu_pre,
                        int& nu_post) {
  if (!p) return "params is NULL";
  if (p->n_levels != J) return "params.n_levels does not match the hierarchy";
  if (p->nu_pre < 0 || p->nu_post < 0 || p->nu_pre > 64 || p->nu_post > 64)
    return "smoothing step counts must be in [0, 64]";
  if (!p->theta || !p->eta || !p->wB || !p->wR || !p->wP) return "params arrays are NULL";
  out.assign((size_t)(J - 1) * mgk::P_COUNT, 0.0);
  for (int l = 0; l < J - 1; ++l) {
    double* q = &out[(size_t)l * mgk::P_COUNT];
    q[mgk::P_THETA] = p->theta[l];
    q[mgk::P_ETA] = p->eta[l];
    q[mgk::P_WB1] = p->wB[2 * l];
    q[mgk::P_WB2] = p->wB[2 * l + 1];
    q[mgk::P_WR1] = p->wR[2 * l];
    q[mgk::P_WR2] = p->wR[2 * l + 1];
    q[mgk::P_WP1] = p->wP[2 * l];
    q[mgk::P_WP2] = p->wP[2 * l + 1];
  }
  for (double v : out)
    if (!std::isfinite(v)) return "params must be finite";
  nu_pre = p->nu_pre;
  nu_post = p->nu_post;
  return "";
}

inline dim3 grid_for(size_t work) { return dim3((unsigned)((work + kThreads - 1) / kThreads)); }

// Dynamic shared memory the small-level block may use (of 227 KB per block).
constexpr size_t kTailSmemMax = 200 * 1024;
// Shared memory of a halo-fused block (default limit, no opt-in needed).
constexpr size_t kHaloSmemMax = 48 * 1024;
// Shared memory of a SELL halo tile (opted in at set-up for every instance).
constexpr size_t kSellHaloSmemMax = 160 * 1024;

// Issues the kernels of one V-cycle (or one level step) on a stream.
template <class T>
struct Issue {
  mg_ctx* c;
  std::vector<DevLevel<T>>& L;
  const T* prm;  // device [J-1][P_COUNT]
  cudaStream_t s;
  int B;
  int nk = 0;
  // level 0's first smoothing step from zero has its delta in L[0].t already
  // (written by k_resid64 with the scaled residual): skip its launch
  bool delta0_ready = false;
  // rfold.u set: level 0's last smoothing step also applies the refinement
  // update (MEAN_CONV_UPDATE_REFINE) when it is the two-row kernel; then
  // rfold_done tells the caller to skip its own update launch
  mgk::RefineEp rfold{};
  bool rfold_done = false;
  // optional per-kernel timing: an event pair around every launch
  std::vector<std::tuple<int, int, cudaEvent_t, cudaEvent_t>>* rec = nullptr;

  void pre(int kind, int lev) {
    if (!rec) return;
    // an NVTX range per step and level around its launch (host timeline of
    // a tracing tool), next to the CUDA event pair on the stream
    char name[64];
    snprintf(name, sizeof name, "L%d %s", lev, mg_kernel_name(kind));
    nvtxRangePushA(name);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
    rec->emplace_back(kind, lev, a, b);
  }
  void post() {
    if (!rec) return;
    cudaEventRecord(std::get<3>(rec->back()), s);
    nvtxRangePop();
  }

  const T* P(int lev) const { return prm + (size_t)lev * mgk::P_COUNT; }
  const T* chebc(int lev) const {
    return (const T*)c->cheb_dev + (size_t)lev * (MG_CHEB_MAX_DEGREE + 1);
  }
  bool conv(int lev, int which) const {
    return c->prm[(size_t)lev * mgk::P_COUNT + which] != 0.0;
  }

  // Kernel launch; with programmatic dependent launch enabled the next
  // kernel in the stream (or captured graph) is scheduled while this one
  // drains and waits in griddepcontrol.wait for its completion.
  template <class... KArgs, class... Args>
  void launch(void (*kern)(KArgs...), dim3 g, dim3 b, size_t smem, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = c->opt_pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kern, args...);
    ++nk;
  }

  // Right-hand sides per thread of the multi-rhs kernels (0: one thread per
  // (row, rhs)): the widest tile of at most 8 values that divides B, or of at
  // most the option's value.  8 is the measured optimum on the 3.1M-row
  // L-shape with 16 rhs in both precisions: 16 FP32 values per thread cost
  // occupancy (64 registers), fewer values cost matrix re-reads.
  int mbv() const {
    if (B < 2 || !c->opt_multi_rhs) return 0;
    int vmax = 8;
    if (c->opt_multi_rhs > 1) vmax = std::min(sizeof(T) == 4 ? 16 : 8, c->opt_multi_rhs);
    if (c->opt_multi_rhs > 1) vmax = std::min(vmax, c->opt_multi_rhs);
    for (int bv = vmax; bv >= 2; bv >>= 1)
      if (B % bv == 0) return bv;
    return 0;
  }
  dim3 mb_grid(int rows, int bv) const {
    const size_t threads = (size_t)rows * (size_t)(B / bv);
    return dim3((unsigned)((threads + kThreads - 1) / kThreads));
  }
  // Calls fn(std::integral_constant<int, BV>) for the chosen tile width.
  template <class F>
  void with_bv(int bv, F&& fn) {
    switch (bv) {
      case 16: fn(std::integral_constant<int, 16>{}); break;
      case 8: fn(std::integral_constant<int, 8>{}); break;
      case 4: fn(std::integral_constant<int, 4>{}); break;
      default: fn(std::integral_constant<int, 2>{}); break;
    }
  }

  // One rhs on a DIA level whose offsets fit 32 bits: the two-row kernels.
  bool two_rows(const DevLevel<T>& D) const {
    const LV<T> v = D.view();
    return B == 1 && c->opt_dia_two_rows && v.ndia > 0 && (int64_t)v.ndia * v.ld < INT32_MAX;
  }
  static dim3 two_row_grid(int n) { return grid_for(((size_t)n + 1) / 2); }
  void op_residual(int lev, const T* f, const T* u, T* out, int scale, int zero) {
    DevLevel<T>& D = L[lev];
    if (two_rows(D)) {
      launch(mgk::k_residual_dia2r<T>, two_row_grid(D.n), kThreads, 0, D.view(), f, u, out,
             P(lev), scale, zero);
    } else if (const int bv = mbv()) {
      with_bv(bv, [&](auto k) {
        launch(mgk::k_residual_mb<T, decltype(k)::value>, mb_grid(D.n, bv), kThreads, 0,
               D.view(), f, u, out, B, P(lev), scale, zero);
      });
    } else {
      launch(B == 1 ? mgk::k_residual<T, 1> : mgk::k_residual<T, 0>, grid_for((size_t)D.n * B), kThreads, 0, D.view(), f, u, out, B,
             P(lev), scale, zero);
    }
  }
  void op_conv_update(int lev, const T* x, T* u, int zero) {
    DevLevel<T>& D = L[lev];
    if (two_rows(D)) {
      launch(mgk::k_mean_dia2r<T, mgk::MEAN_CONV_UPDATE>, two_row_grid(D.n), kThreads, 0,
             D.view(), x, (const T*)nullptr, u, P(lev), zero, mgk::RefineEp{});
    } else if (const int bv = mbv()) {
      with_bv(bv, [&](auto k) {
        launch(mgk::k_conv_update_mb<T, decltype(k)::value>, mb_grid(D.n, bv), kThreads, 0,
               D.view(), x, u, B, P(lev), zero);
      });
    } else {
      launch(B == 1 ? mgk::k_conv_update<T, 1> : mgk::k_conv_update<T, 0>, grid_for((size_t)D.n * B), kThreads, 0, D.view(), x, u, B,
             P(lev), zero);
    }
  }
  // One ChebConv recurrence pass (k_cheb_step); out may be tpp.
  void op_cheb(int lev, const T* tprev, const T* tpp, T* out, T* u, int k, int zero) {
    DevLevel<T>& D = L[lev];
    if (const int bv = mbv()) {
      with_bv(bv, [&](auto kk) {
        launch(mgk::k_cheb_step_mb<T, decltype(kk)::value>, mb_grid(D.n, bv), kThreads, 0,
               D.view(), tprev, tpp, out, u, B, P(lev), chebc(lev), k, zero);
      });
    } else {
      launch(B == 1 ? mgk::k_cheb_step<T, 1> : mgk::k_cheb_step<T, 0>, grid_for((size_t)D.n * B), kThreads, 0, D.view(), tprev, tpp,
             out, u, B, P(lev), chebc(lev), k, zero);
    }
  }
  void op_jacobi(int lev, const T* f, const T* uin, T* uout, int zero) {
    DevLevel<T>& D = L[lev];
    if (const int bv = mbv()) {
      with_bv(bv, [&](auto k) {
        launch(mgk::k_jacobi_mb<T, decltype(k)::value>, mb_grid(D.n, bv), kThreads, 0, D.view(),
               f, uin, uout, B, P(lev), zero);
      });
    } else {
      launch(B == 1 ? mgk::k_jacobi<T, 1> : mgk::k_jacobi<T, 0>, grid_for((size_t)D.n * B), kThreads, 0, D.view(), f, uin, uout, B,
             P(lev), zero);
    }
  }
  void op_conv_r(int lev, const T* r, T* phi) {
    DevLevel<T>& D = L[lev];
    if (two_rows(D)) {
      launch(mgk::k_mean_dia2r<T, mgk::MEAN_CONV_R>, two_row_grid(D.n), kThreads, 0, D.view(), r,
             (const T*)nullptr, phi, P(lev), 0, mgk::RefineEp{});
    } else if (const int bv = mbv()) {
      with_bv(bv, [&](auto k) {
        launch(mgk::k_conv_r_mb<T, decltype(k)::value>, mb_grid(D.n, bv), kThreads, 0, D.view(),
               r, phi, B, P(lev));
      });
    } else {
      launch(B == 1 ? mgk::k_conv_r<T, 1> : mgk::k_conv_r<T, 0>, grid_for((size_t)D.n * B), kThreads, 0, D.view(), r, phi, B,
             P(lev));
    }
  }
  // fc = P^T x (after Phi_R) or P^T (wR1 x) (plain restriction)
  void op_gather(int lev, const T* x, T* fc, int scale) {
    DevLevel<T>& D = L[lev];
    if (const int bv = mbv()) {
      with_bv(bv, [&](auto k) {
        launch(mgk::k_gather_mb<T, decltype(k)::value>, mb_grid(D.nc, bv), kThreads, 0,
               D.view(), x, fc, B, P(lev), scale);
      });
    } else if (scale) {
      launch(B == 1 ? mgk::k_restrict<T, 1> : mgk::k_restrict<T, 0>, grid_for((size_t)D.nc * B), kThreads, 0, D.view(), x, fc, B,
             P(lev), 0);
    } else {
      launch(B == 1 ? mgk::k_gather<T, 1> : mgk::k_gather<T, 0>, grid_for((size_t)D.nc * B), kThreads, 0, D.view(), x, fc, B);
    }
  }
  void op_pe(int lev, const T* ec, T* pe) {
    DevLevel<T>& D = L[lev];
    if (B == 1 && c->opt_dia_two_rows) {
      launch(mgk::k_pe2r<T>, two_row_grid(D.n), kThreads, 0, D.view(), ec, pe);
    } else if (const int bv = mbv()) {
      with_bv(bv, [&](auto k) {
        launch(mgk::k_pe_mb<T, decltype(k)::value>, mb_grid(D.n, bv), kThreads, 0, D.view(), ec,
               pe, B);
      });
    } else {
      launch(B == 1 ? mgk::k_pe<T, 1> : mgk::k_pe<T, 0>, grid_for((size_t)D.n * B), kThreads, 0, D.view(), ec, pe, B);
    }
  }
  // u = uin + Phi_P(x) with x = P e_c (conv), or u = uin + wP1 P x (plain)
  void op_prolong(int lev, const T* x, const T* uin, T* u, int conv_p) {
    DevLevel<T>& D = L[lev];
    if (conv_p && two_rows(D)) {
      launch(mgk::k_mean_dia2r<T, mgk::MEAN_PROLONG_CONV>, two_row_grid(D.n), kThreads, 0,
             D.view(), x, uin, u, P(lev), 0, mgk::RefineEp{});
    } else if (const int bv = mbv()) {
      with_bv(bv, [&](auto k) {
        launch(mgk::k_prolong_mb<T, decltype(k)::value>, mb_grid(D.n, bv), kThreads, 0,
               D.view(), x, uin, u, B, P(lev), conv_p);
      });
    } else if (conv_p) {
      launch(B == 1 ? mgk::k_prolong_conv<T, 1> : mgk::k_prolong_conv<T, 0>, grid_for((size_t)D.n * B), kThreads, 0, D.view(), x, uin, u,
             B, P(lev));
    } else {
      launch(B == 1 ? mgk::k_prolong<T, 1> : mgk::k_prolong<T, 0>, grid_for((size_t)D.n * B), kThreads, 0, D.view(), x, uin, u, B,
             P(lev), 0);
    }
  }

  // nu smoothing steps on level lev; u updated in place.  zero: u is 0 on entry.
  // Halo-fused steps (halo.cuh) on a DIA level: rows per block TR and halo
  // H, or 0 (two-kernel form) when the level is SELL or the option is off;
  // when a tile would be narrower than its halo (each block redoing more
  // than 3x its rows); when the tile does not fit kHaloSmemMax for B
  // right-hand sides; or when the first stage over all tiles and halos
  // exceeds one wave of the GPU.  Past that point the level fills the GPU
  // and the redundant halo work costs more than the kernel boundary it
  // saves (measured: the 511^2-row level of the 513^2 mesh runs faster
  // unfused, its coarser levels fused).
  int halo_rows(int lev, int& H, size_t& smem, int& threads) const {
    const DevLevel<T>& D = L[lev];
    if (c->opt_halo_rows <= 0 || D.ndia == 0) return 0;
    H = 0;
    for (int k = 0; k < D.ndia; ++k) H = std::max(H, std::abs(D.doff[k]));
    const size_t per_row = (size_t)B * sizeof(T);
    const int64_t cap_rows = (int64_t)(kHaloSmemMax / per_row);
    int64_t tr = std::min<int64_t>(c->opt_halo_rows, cap_rows - 2 * (int64_t)H);
    if (tr >= D.n) {
      tr = D.n;  // one block, no halo
    } else if (tr < std::max<int64_t>(H, 1)) {
      return 0;
    }
    const int64_t span = std::min<int64_t>(tr + 2 * (int64_t)H, D.n);
    if (span > cap_rows) return 0;
    const int64_t nblk = (D.n + tr - 1) / tr;
    if (nblk * span * B > c->wave_threads) return 0;
    smem = (size_t)span * per_row;
    threads = (int)std::min<int64_t>(mgk::kTailThreads, (span * B + 31) / 32 * 32);
    return (int)tr;
  }
  // 2D-tiled fused steps (k_halo_dia2) on a DIA level whose vectors are at
  // least opt_halo2d_bytes: its grid width w (the offsets must be 0, +-1,
  // +-w, +-(w-1) or +-(w+1)), the tiles and every diagonal's grid shift;
  // false (another form) otherwise, or when the tile's shared memory for B
  // right-hand sides exceeds kHaloSmemMax.
  struct Halo2 {
    int w = 0, tiles_x = 0;
    unsigned tiles = 0;
    size_t smem = 0;
    mgk::DiaShift sh;
  };
  bool halo2d(int lev, Halo2& h) const {
    const DevLevel<T>& D = L[lev];
    if (c->opt_halo2d_bytes <= 0 || D.ndia == 0) return false;
    if ((int64_t)D.n * B * (int64_t)sizeof(T) < c->opt_halo2d_bytes) return false;
    h.smem = (size_t)mgk::kH2RX * mgk::kH2RY * B * sizeof(T);
    if (h.smem > kHaloSmemMax) return false;
    int m = INT_MAX;
    for (int k = 0; k < D.ndia; ++k)
      if (std::abs(D.doff[k]) > 1) m = std::min(m, std::abs(D.doff[k]));
    if (m == INT_MAX) return false;
    for (int w : {m, m + 1, m - 1}) {
      if (w < 3) continue;
      bool ok = true;
      for (int k = 0; k < D.ndia && ok; ++k) {
        ok = false;
        for (int dy = -1; dy <= 1 && !ok; ++dy) {
          const int dx = D.doff[k] - dy * w;
          if (dx >= -1 && dx <= 1) {
            h.sh.dx[k] = (int8_t)dx;
            h.sh.dy[k] = (int8_t)dy;
            ok = true;
          }
        }
      }
      if (!ok) continue;
      for (int k = D.ndia; k < mgk::kMaxDia; ++k) h.sh.dx[k] = h.sh.dy[k] = 0;
      h.w = w;
      h.tiles_x = (w + mgk::kH2X - 1) / mgk::kH2X;
      const int64_t rows = (D.n + (int64_t)w - 1) / w;
      const int64_t tiles = h.tiles_x * ((rows + mgk::kH2Y - 1) / mgk::kH2Y);
      if (tiles >= ((int64_t)1 << 31)) return false;
      h.tiles = (unsigned)tiles;
      return true;
    }
    return false;
  }
  template <int MODE>
  void op_halo2(int lev, const Halo2& h, const T* f, const T* x, T* y, int zero) {
    DevLevel<T>& D = L[lev];
    launch(B == 1 ? mgk::k_halo_dia2<T, MODE, 1> : mgk::k_halo_dia2<T, MODE, 0>, dim3(h.tiles),
           dim3(mgk::kH2Threads), h.smem, D.view(), f, x, y, B, P(lev), h.w, h.tiles_x, h.sh, zero);
  }
  // Halo-tiled fused steps on a SELL level (halo_sell.cuh): the tile's
  // shared bytes, or 0 (two-kernel form) when the level has no halo tables
  // or the tile does not fit kSellHaloSmemMax for B right-hand sides.
  size_t sell_halo(int lev, bool size_cap = true) const {
    const DevLevel<T>& D = L[lev];
    if (D.ndia > 0 || D.hs_tr <= 0 || !D.hs_ptr) return 0;
    if (size_cap && (int64_t)D.n * B * (int64_t)sizeof(T) > c->opt_sell_halo_max_bytes) return 0;
    const size_t smem = (size_t)(D.hs_tr + D.hs_hmax) * B * sizeof(T);
    return smem <= kSellHaloSmemMax ? smem : 0;
  }
  template <int MODE>
  void op_halo_sell(int lev, size_t smem, const T* f, const T* x, T* y, int zero) {
    DevLevel<T>& D = L[lev];
    const dim3 grid((unsigned)((D.n + D.hs_tr - 1) / D.hs_tr));
    if (const int bv = mbv()) {
      with_bv(bv, [&](auto k) {
        launch(mgk::k_halo_sell<T, decltype(k)::value, MODE>, grid,
               dim3(c->opt_sell_halo_threads), smem, D.view(), D.halo(), f, x, y, B, P(lev),
               zero);
      });
    } else {
      launch(mgk::k_halo_sell<T, 1, MODE>, grid, dim3(c->opt_sell_halo_threads), smem, D.view(),
             D.halo(), f, x, y, B, P(lev), zero);
    }
  }
  // fine, phi, fout: HALO_SMOOTH_GATHER's finer level, its Phi_R values and
  // this level's right-hand side (the level itself and NULLs otherwise).
  template <int MODE>
  void op_halo(int lev, int TR, int H, size_t smem, int threads, const T* f, const T* x, T* y,
               int zero, int fine = -1, const T* phi = nullptr, T* fout = nullptr) {
    DevLevel<T>& D = L[lev];
    launch(B == 1 ? mgk::k_halo_dia<T, MODE, 1> : mgk::k_halo_dia<T, MODE, 0>,
           dim3((unsigned)((D.n + TR - 1) / TR)), dim3(threads), smem, D.view(), f, x, y, B,
           P(lev), TR, H, zero, L[fine >= 0 ? fine : lev].view(), phi, fout);
  }
  // The restriction from level lev leaves its gather to the first smoothing
  // step of level lev + 1 when that step is a 1D halo-fused kernel from zero
  // (every level of the descent below the cycle's first starts from zero).
  bool gather_in_next_smooth(int lev) const {
    const int nxt = lev + 1;
    if (c->cheb_K > 0 || c->nu_pre < 1 || nxt >= c->J - 1 || nxt >= tail_level()) return false;
    if (!conv(nxt, mgk::P_WB2)) return false;
    int H = 0, nth = 0;
    size_t smem = 0;
    return halo_rows(nxt, H, smem, nth) > 0;
  }
  int pending_gather = -1;  // the level whose gather the next smoothing does (-1: none)

  void smooth(int lev, const T* f, T* u, int nu, bool zero) {
    DevLevel<T>& D = L[lev];
    const size_t N = (size_t)D.n * B;
    const dim3 g = grid_for(N);
    if (nu == 0) {
      if (zero) cudaMemsetAsync(u, 0, N * sizeof(T), s);
      return;
    }
    if (c->cheb_K > 0) {  // ChebConv smoother: delta, then K recurrence passes
      for (int k = 0; k < nu; ++k) {
        const int z = zero && k == 0;
        pre(MG_K_RESIDUAL_SCALED, lev);
        op_residual(lev, f, u, D.t, 1, z);
        post();
        T* tpp = D.t;  // T_{j-2}
        T* tp = D.u2;  // T_{j-1}
        pre(MG_K_CHEB_STEP, lev);
        op_cheb(lev, D.t, D.t, D.u2, u, 1, z);
        post();
        for (int j = 2; j <= c->cheb_K; ++j) {
          pre(MG_K_CHEB_STEP, lev);
          op_cheb(lev, tp, tpp, tpp, u, j, 0);
          post();
          std::swap(tp, tpp);
        }
      }
      return;
    }
    if (!conv(lev, mgk::P_WB2)) {
      T* cur = u;
      T* oth = D.u2;
      for (int k = 0; k < nu; ++k) {
        pre(MG_K_JACOBI, lev);
        op_jacobi(lev, f, cur, oth, (int)(zero && k == 0));
        post();
        std::swap(cur, oth);
      }
      if (cur != u) launch(mgk::k_copy<T>, g, kThreads, 0, (const T*)cur, u, N);
      return;
    }
    int H = 0, nth = 0;
    size_t smem = 0;
    if (const int TR = halo_rows(lev, H, smem, nth)) {  // one fused kernel per step
      T* cur = u;
      T* oth = D.u2;
      for (int k = 0; k < nu; ++k) {
        pre(MG_K_SMOOTH_HALO, lev);
        if (k == 0 && zero && lev > 0 && pending_gather == lev - 1) {  // f gathered here
          op_halo<mgk::HALO_SMOOTH_GATHER>(lev, TR, H, smem, nth, f, cur, oth, 1, lev - 1,
                                           L[lev - 1].u2, (T*)f);
          pending_gather = -1;
        } else {
          op_halo<mgk::HALO_SMOOTH>(lev, TR, H, smem, nth, f, cur, oth, (int)(zero && k == 0));
        }
        post();
        std::swap(cur, oth);
      }
      if (cur != u) launch(mgk::k_copy<T>, g, kThreads, 0, (const T*)cur, u, N);
      return;
    }
    Halo2 h2;
    if (halo2d(lev, h2)) {  // large DIA level: one 2D-tiled fused kernel per step
      T* cur = u;
      T* oth = D.u2;
      for (int k = 0; k < nu; ++k) {
        pre(MG_K_SMOOTH_HALO, lev);
        op_halo2<mgk::HALO_SMOOTH>(lev, h2, f, cur, oth, (int)(zero && k == 0));
        post();
        std::swap(cur, oth);
      }
      if (cur != u) launch(mgk::k_copy<T>, g, kThreads, 0, (const T*)cur, u, N);
      return;
    }
    if (const size_t hsm = sell_halo(lev)) {  // SELL: one fused kernel per step
      T* cur = u;
      T* oth = D.u2;
      for (int k = 0; k < nu; ++k) {
        pre(MG_K_SMOOTH_HALO, lev);
        op_halo_sell<mgk::HALO_SMOOTH>(lev, hsm, f, cur, oth, (int)(zero && k == 0));
        post();
        std::swap(cur, oth);
      }
      if (cur != u) launch(mgk::k_copy<T>, g, kThreads, 0, (const T*)cur, u, N);
      return;
    }
    for (int k = 0; k < nu; ++k) {
      const int z = zero && k == 0;
      if (!(z && lev == 0 && delta0_ready)) {
        pre(MG_K_RESIDUAL_SCALED, lev);
        op_residual(lev, f, u, D.t, 1, z);
        post();
      }
      pre(MG_K_CONV_UPDATE, lev);
      if (k == nu - 1 && lev == 0 && !zero && rfold.u && two_rows(D)) {
        launch(mgk::k_mean_dia2r<T, mgk::MEAN_CONV_UPDATE_REFINE>, two_row_grid(D.n), kThreads,
               0, D.view(), (const T*)D.t, (const T*)nullptr, u, P(lev), 0, rfold);
        rfold_done = true;
      } else {
        op_conv_update(lev, D.t, u, z);
      }
      post();
    }
  }

  // f_{lev+1} = P^T phi with phi = Phi_R(r) in L[lev].u2: now, or in the
  // first smoothing step of level lev + 1 (gather_in_next_smooth).
  void gather_phi(int lev) {
    if (gather_in_next_smooth(lev)) {
      pending_gather = lev;
      return;
    }
    pre(MG_K_RESTRICT, lev);
    op_gather(lev, L[lev].u2, Fl(lev + 1), 0);
    post();
  }

  void restrict_(int lev, const T* f, const T* u) {
    DevLevel<T>& D = L[lev];
    int H = 0, nth = 0;
    size_t smem = 0;
    const int TR = conv(lev, mgk::P_WR2) ? halo_rows(lev, H, smem, nth) : 0;
    if (TR) {  // residual and Phi_R in one kernel, then the gather P^T
      pre(MG_K_RESTRICT_HALO, lev);
      op_halo<mgk::HALO_RESTRICT>(lev, TR, H, smem, nth, f, u, D.u2, 0);
      post();
      gather_phi(lev);
      return;
    }
    Halo2 h2;
    if (conv(lev, mgk::P_WR2) && halo2d(lev, h2)) {  // large DIA level: 2D tiles
      pre(MG_K_RESTRICT_HALO, lev);
      op_halo2<mgk::HALO_RESTRICT>(lev, h2, f, u, D.u2, 0);
      post();
      gather_phi(lev);
      return;
    }
    if (conv(lev, mgk::P_WR2)) {
      if (const size_t hsm = sell_halo(lev)) {  // SELL: r and Phi_R(r) in one kernel
        pre(MG_K_RESTRICT_HALO, lev);
        op_halo_sell<mgk::HALO_RESTRICT>(lev, hsm, f, u, D.u2, 0);
        post();
        gather_phi(lev);
        return;
      }
    }
    pre(MG_K_RESIDUAL, lev);
    op_residual(lev, f, u, D.t, 0, 0);
    post();
    if (conv(lev, mgk::P_WR2)) {  // Phi_R per fine row, then the gather P^T
      pre(MG_K_CONV_R, lev);
      op_conv_r(lev, D.t, D.u2);
      post();
      gather_phi(lev);
    } else {
      pre(MG_K_RESTRICT, lev);
      op_gather(lev, D.t, Fl(lev + 1), 1);
      post();
    }
  }

  void prolong(int lev, const T* ec, T* u) {
    DevLevel<T>& D = L[lev];
    int H = 0, nth = 0;
    size_t smem = 0;
    const int TR = conv(lev, mgk::P_WP2) ? halo_rows(lev, H, smem, nth) : 0;
    if (TR) {  // P e_c, Phi_P and the update in one kernel
      pre(MG_K_PROLONG_HALO, lev);
      op_halo<mgk::HALO_PROLONG>(lev, TR, H, smem, nth, (const T*)nullptr, ec, u, 0);
      post();
      return;
    }
    Halo2 h2;
    if (conv(lev, mgk::P_WP2) && halo2d(lev, h2)) {  // large DIA level: 2D tiles
      pre(MG_K_PROLONG_HALO, lev);
      op_halo2<mgk::HALO_PROLONG>(lev, h2, (const T*)nullptr, ec, u, 0);
      post();
      return;
    }
    if (conv(lev, mgk::P_WP2)) {
      if (const size_t hsm = sell_halo(lev, false)) {  // SELL: P e_c, Phi_P and the update
        pre(MG_K_PROLONG_HALO, lev);
        op_halo_sell<mgk::HALO_PROLONG>(lev, hsm, (const T*)nullptr, ec, u, 0);
        post();
        return;
      }
    }
    if (conv(lev, mgk::P_WP2)) {  // P e_c per fine row, then Phi_P and the update
      pre(MG_K_PE, lev);
      op_pe(lev, ec, D.t);
      post();
      pre(MG_K_PROLONG, lev);
      op_prolong(lev, D.t, u, u, 1);
      post();
    } else {
      pre(MG_K_PROLONG, lev);
      op_prolong(lev, ec, u, u, 0);
      post();
    }
  }

  // rows of the coarsest level in this issue's view (fewer than the
  // context's in a view of the leading blocks of a stacked context, which
  // always solves with the explicit inverse)
  int rowsJ() const { return L[c->J - 1].n; }

  int coarse_warps(int cap) const {
    return std::max(1, std::min(std::min(B, cap), 6144 / std::max(1, rowsJ())));
  }

  void coarse(const T* f, T* u) {
    const size_t nJ = (size_t)rowsJ();
    if (c->coarse_inv) {  // one FP64 dot per (row, rhs), spread over SMs
      pre(MG_K_COARSE_CHOL, c->J - 1);
      launch(mgk::k_coarse_inv<T>,
             dim3((unsigned)((nJ * B + mgk::kCoarseInvThreads - 1) / mgk::kCoarseInvThreads)),
             dim3(mgk::kCoarseInvThreads), 0, (const double*)c->cholInv, (int)nJ, c->nJ, f, u,
             B);
      post();
      return;
    }
    const size_t fixed = mgk::tail_align(nJ * (nJ + 1) / 2 * sizeof(double)) +
                         mgk::tail_align(nJ * sizeof(double));
    // factor staged in shared memory as a packed triangle; past a few rows
    // the FP64 substitutions of one SM bound the step, so each right-hand
    // side gets a block (one warp) of its own on another SM
    const int nwp = nJ >= 32 ? 1 : std::max(1, std::min(B, 32));
    if (fixed + (size_t)nwp * nJ * sizeof(double) <= kTailSmemMax) {
      pre(MG_K_COARSE_CHOL, c->J - 1);
      launch(mgk::k_coarse_chol_packed<T>, dim3((unsigned)((B + nwp - 1) / nwp)), dim3(32 * nwp),
             fixed + (size_t)nwp * nJ * sizeof(double), (const double*)c->cholP,
             (const double*)c->cholDinv, c->nJ, f, u, B);
      post();
      return;
    }
    const int nw = coarse_warps(8);
    pre(MG_K_COARSE_CHOL, c->J - 1);
    launch(mgk::k_coarse_chol<T>, dim3(1), dim3(32 * nw), (size_t)nw * c->nJ * sizeof(double),
           (const double*)c->cholL, (const double*)c->cholU, (const double*)c->cholDinv, c->nJ,
           f, u, B);
    post();
  }

  // First level handled by the single-block tail for this batch size (J-1:
  // no tail, only the coarse solve).
  // Small-level arguments for every level (lt chosen by the caller).
  // l0: the level whose vectors are (f0, u0) (the cycle's first level).
  void tail_args(mgk::TailArgs<T>& a, const T* f0, T* u0, bool u0_zero, int l0 = 0) const {
    std::memset(&a, 0, sizeof(a));
    a.J = c->J;
    a.B = B;
    a.nu_pre = c->nu_pre;
    a.nu_post = c->nu_post;
    a.nJ = rowsJ();
    a.cwarps = coarse_warps(32);
    a.lt_zero = (int)u0_zero;
    for (int l = 0; l < c->J; ++l) {
      a.L[l] = L[l].view();
      a.nsl[l] = L[l].ndia > 0 ? 0 : L[l].nsl;
      a.nent[l] = L[l].ndia > 0 ? 0 : (int)L[l].nent;
      a.f[l] = l == l0 ? f0 : Fl(l);
      a.u[l] = l == l0 ? u0 : Ul(l);
      a.t[l] = L[l].t;
      a.u2[l] = L[l].u2;
      if (l < c->J - 1) {
        a.convB |= (conv(l, mgk::P_WB2) ? 1u : 0u) << l;
        a.convR |= (conv(l, mgk::P_WR2) ? 1u : 0u) << l;
        a.convP |= (conv(l, mgk::P_WP2) ? 1u : 0u) << l;
      }
    }
    a.prm = prm;
    a.cL = c->cholL;
    a.cU = c->cholU;
    a.cDinv = c->cholDinv;
    a.cInv = c->coarse_inv ? c->cholInv : nullptr;
    a.cInvLd = c->nJ;
    // the team of a small level: about opt_tail_teams entries (row, rhs) per
    // thread, a power of two of warps, never more warps than the finer
    // level's team
    int prev = mgk::kTailBlock / 32;
    for (int l = 0; l < mgk::kMaxLevels; ++l) {
      int w = mgk::kTailBlock / 32;
      if (c->opt_tail_teams > 0 && l < c->J) {
        const int64_t per_warp = 32 * (int64_t)c->opt_tail_teams;
        const int64_t need = ((int64_t)L[l].n * B + per_warp - 1) / per_warp;
        w = 1;
        while (w < mgk::kTailBlock / 32 && w < need) w *= 2;
      }
      a.tw[l] = std::min(w, prev);
      prev = a.tw[l];
    }
    // a recorded forward must leave every level's f and u in its checkpoint
    // buffers, so it keeps the small levels' vectors in global memory
    a.smem_vectors = fov == nullptr && uov == nullptr ? 1 : 0;
    a.smem_matrix = 1;
  }

  // First level run by the single-block kernel (J-1: none): levels with
  // rows x rhs <= the threshold, reduced until their data fits in shared
  // memory.
  int tail_level() const {
    if (c->opt_tail_work <= 0 || c->J > mgk::kMaxLevels || c->cheb_K > 0) return c->J - 1;
    int lt = c->J - 1;
    while (lt > 0 && (int64_t)L[lt - 1].n * B <= c->opt_tail_work) --lt;
    if (lt == c->J - 1) return lt;
    mgk::TailArgs<T> a;
    tail_args(a, nullptr, nullptr, false);
    while (lt < c->J - 1 && mgk::tail_smem_bytes<T>(a, lt) > kTailSmemMax) ++lt;
    return lt;
  }

  void tail(int lt, const T* f0, T* u0, bool u0_zero, int l0 = 0) {
    mgk::TailArgs<T> a;
    tail_args(a, f0, u0, u0_zero, l0);
    a.lt = lt;
    if (lt > l0) a.lt_zero = 1;  // levels below the cycle's first start from zero
    pre(MG_K_TAIL, lt);
    launch(a.B == 1 ? mgk::k_tail<T, 1> : mgk::k_tail<T, 0>, dim3(1), dim3(mgk::kTailBlock),
           mgk::tail_smem_bytes<T>(a, lt), a);
    post();
  }

  // Level vectors of levels >= 1; training points them at checkpoint storage.
  T* const* fov = nullptr;
  T* const* uov = nullptr;
  T* Fl(int lev) const { return fov ? fov[lev] : L[lev].f; }
  T* Ul(int lev) const { return uov ? uov[lev] : L[lev].u; }

  void vcycle(const T* f0, T* u0, bool u0_zero) { vcycle_from(0, f0, u0, u0_zero); }

  // Algorithm 2 started on level l0 with right-hand side f0 and iterate u0
  // (the vectors of levels below l0 are the level buffers).
  void vcycle_from(int l0, const T* f0, T* u0, bool u0_zero) {
    const int J = c->J;
    if (l0 == J - 1) {  // the coarsest level: the exact solve
      coarse(f0, u0);
      return;
    }
    const int lt = std::max(tail_level(), l0);
    for (int lev = l0; lev < lt; ++lev) {
      const T* f = lev == l0 ? f0 : Fl(lev);
      T* u = lev == l0 ? u0 : Ul(lev);
      smooth(lev, f, u, c->nu_pre, lev == l0 ? u0_zero : true);
      restrict_(lev, f, u);
    }
    if (lt < J - 1)
      tail(lt, lt == l0 ? f0 : Fl(lt), lt == l0 ? u0 : Ul(lt), lt == l0 ? u0_zero : true, lt);
    else
      coarse(Fl(J - 1), Ul(J - 1));
    for (int lev = lt - 1; lev >= l0; --lev) {
      const T* f = lev == l0 ? f0 : Fl(lev);
      T* u = lev == l0 ? u0 : Ul(lev);
      prolong(lev, Ul(lev + 1), u);
      smooth(lev, f, u, c->nu_post, false);
    }
  }

  // f_{l+1} = P^T Phi_R(f_l) into the level buffer Fl(lev + 1): the cycle's
  // restriction applied to a right-hand side.
  void restrict_f(int lev, const T* f) {
    DevLevel<T>& D = L[lev];
    if (conv(lev, mgk::P_WR2)) {
      pre(MG_K_CONV_R, lev);
      op_conv_r(lev, f, D.u2);
      post();
      pre(MG_K_RESTRICT, lev);
      op_gather(lev, D.u2, Fl(lev + 1), 0);
      post();
    } else {
      pre(MG_K_RESTRICT, lev);
      op_gather(lev, f, Fl(lev + 1), 1);
      post();
    }
  }

  // Full multigrid (nested iteration, the preconditioner of the paper's
  // Sec. 4.2 Krylov experiments, tab:helmholtz-results-precond): f
  // restricted to every level by the cycle's restriction, the coarsest
  // level solved exactly, then on each finer level
  // the coarser solution through the cycle's prolongation (Phi_P P, from a
  // zero iterate) is the initial guess of one V-cycle started on that level.
  // The V-cycle on level l reuses the buffers of levels > l, whose FMG
  // values (f_{l+1}, u_{l+1}) are consumed by then.
  void fmg(const T* f0, T* u0) {
    const int J = c->J;
    for (int lev = 0; lev < J - 1; ++lev) restrict_f(lev, lev == 0 ? f0 : Fl(lev));
    coarse(Fl(J - 1), Ul(J - 1));
    for (int lev = J - 2; lev >= 0; --lev) {
      const T* f = lev == 0 ? f0 : Fl(lev);
      T* u = lev == 0 ? u0 : Ul(lev);
      cudaMemsetAsync(u, 0, (size_t)L[lev].n * B * sizeof(T), s);
      prolong(lev, Ul(lev + 1), u);
      vcycle_from(lev, f, u, false);
    }
  }
};

mg_status sync_params(mg_ctx* c, cudaStream_t s) {
  if (c->cheb_dirty) {
    // pageable sources that go out of scope: make each copy complete
    if (c->prec == 64) {
      MG_CUDA(cudaMemcpyAsync(c->cheb_dev, c->cheb_host.data(),
                              c->cheb_host.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    } else {
      std::vector<float> f(c->cheb_host.begin(), c->cheb_host.end());
      MG_CUDA(cudaMemcpyAsync(c->cheb_dev, f.data(), f.size() * sizeof(float),
                              cudaMemcpyHostToDevice, s));
    }
    MG_CUDA(cudaStreamSynchronize(s));
    c->cheb_dirty = false;
  }
  if (!c->prm_dirty) return MG_OK;
  if (c->prec == 64) {
    MG_CUDA(cudaMemcpyAsync(c->prm64, c->prm.data(), c->prm.size() * sizeof(double),
                            cudaMemcpyHostToDevice, s));
  } else {
    std::vector<float> f(c->prm.begin(), c->prm.end());
    MG_CUDA(cudaMemcpyAsync(c->prm32, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice,
                            s));
    // the FP32 copy is pageable and goes out of scope: make the copy complete
    MG_CUDA(cudaStreamSynchronize(s));
  }
  c->prm_dirty = false;
  return MG_OK;
}

// Debug build (-DMG_BOUNDS_CHECK): the first out-of-range index a kernel met
// (kernels.cuh idx_ok) becomes MG_ERR_INVALID of the call that launched it;
// the record is cleared.  Synchronises s.  Other builds: MG_OK.
mg_status bounds_status(mg_ctx* c, cudaStream_t s, const char* who) {
#ifdef MG_BOUNDS_CHECK
  unsigned long long w = 0;
  MG_CUDA(cudaStreamSynchronize(s));
  MG_CUDA(cudaMemcpyFromSymbol(&w, mgk::g_bounds_error, sizeof(w)));
  if (w) {
    const unsigned long long zero = 0;
    MG_CUDA(cudaMemcpyToSymbol(mgk::g_bounds_error, &zero, sizeof(zero)));
    char buf[192];
    snprintf(buf, sizeof buf, "%s: index out of range (check site %llu, index %d)", who,
             (w - 1) >> 32, (int)(unsigned)((w - 1) & 0xffffffffull));
    return c->fail(MG_ERR_INVALID, buf);
  }
#else
  (void)c;
  (void)s;
  (void)who;
#endif
  return MG_OK;
}

// Captures fn(stream) into a graph stored under key (or reuses it) and
// launches it on s.
template <class Fn>
mg_status run_graph(mg_ctx* c, const std::tuple<int, const void*, const void*, int, uint32_t>& key,
                    cudaStream_t s, Fn&& fn) {
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    std::lock_guard<std::recursive_mutex> lk(mgi::setup_mutex());
    cudaGraph_t g = nullptr;
    MG_CUDA(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    int nk = fn(c->cap);
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return c->fail(MG_ERR_CUDA, std::string("graph capture failed: ") +
                                      cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    }
    GraphEntry ge;
    ge.nkernels = nk;
    cudaError_t e3 = cudaGraphInstantiate(&ge.exec, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess)
      return c->fail(MG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e3));
    if (c->graphs.size() > 512) {  // bounded cache
      for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
      c->graphs.clear();
    }
    it = c->graphs.emplace(key, ge).first;
  }
  MG_CUDA(cudaGraphLaunch(it->second.exec, s));
  c->launches += it->second.nkernels;
  return bounds_status(c, s, "mg_vcycle / mg_fmg / a solve step");
}

// An iterative solve: pre once (it ends with k_check), then body while
// k_check says continue, then post (when has_post).  Each of pre/body is
// fn(stream, while-node handle, set_cond) -> kernels issued; post is
// fn(stream) -> kernels issued.
//   device loop (default): one graph, the body inside a conditional while
//     node whose condition k_check sets; one launch and one host sync per solve.
//   host loop (MG_OPT_DEVICE_LOOP = 0): three plain graphs; the host reads
//     state[3] after pre and after every body launch.  Same kernels in the
//     same order with the same arguments, so the same results; a profiler
//     that cannot see inside conditional nodes sees every kernel.
// On return state[0..3] is in c->h_state.
template <class Pre, class Body, class Post>
mg_status run_loop(mg_ctx* c, int id, const void* f, const void* u, int B, cudaStream_t s,
                   const char* who, Pre&& pre, Body&& body, Post&& post, bool has_post) {
  if (!c->opt_device_loop) {
    auto key = [&](int sub) { return std::make_tuple(id + sub, f, u, B, c->structure); };
    const cudaGraphConditionalHandle h0 = 0;
    mg_status st = run_graph(c, key(1), s, [&](cudaStream_t cs) { return pre(cs, h0, 0); });
    for (;;) {
      if (st != MG_OK) return st;
      MG_CUDA(cudaMemcpyAsync(c->h_state, c->state, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
      MG_CUDA(cudaStreamSynchronize(s));
      if (!c->h_state[3]) break;
      st = run_graph(c, key(2), s, [&](cudaStream_t cs) { return body(cs, h0, 0); });
    }
    if (has_post) {
      st = run_graph(c, key(3), s, [&](cudaStream_t cs) { return post(cs); });
      if (st != MG_OK) return st;
      MG_CUDA(cudaStreamSynchronize(s));
    }
    return bounds_status(c, s, who);
  }
  auto key = std::make_tuple(id, f, u, B, c->structure);
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    std::lock_guard<std::recursive_mutex> lk(mgi::setup_mutex());
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle h;
    int nk_init = 0, nk_body = 0;
    MG_CUDA(cudaGraphCreate(&g, 0));
    MG_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
    MG_CUDA(cudaStreamBeginCaptureToGraph(c->cap, g, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
    nk_init += pre(c->cap, h, 1);
    cudaStreamCaptureStatus cst;
    cudaGraph_t capg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t ndeps = 0;
    cudaGraphNode_t wnode;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaError_t e = cudaStreamGetCaptureInfo(c->cap, &cst, nullptr, &capg, &deps, &edges, &ndeps);
    // a capture invalidated on the way (status not active) has no graph to add to
    if (e == cudaSuccess && (cst != cudaStreamCaptureStatusActive || !capg))
      e = cudaErrorStreamCaptureInvalidated;
    if (e == cudaSuccess) e = cudaGraphAddNode(&wnode, capg, deps, edges, ndeps, &np);
    if (e == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(c->cap, &wnode, nullptr, 1,
                                              cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess && has_post) nk_init += post(c->cap);
    cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return c->fail(MG_ERR_CUDA, std::string(who) + ": graph build: " +
                                      cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraph_t bodyg = np.conditional.phGraph_out[0];
    MG_CUDA(cudaStreamBeginCaptureToGraph(c->cap, bodyg, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
    nk_body += body(c->cap, h, 1);
    cudaGraph_t body_out = nullptr;
    e = cudaGetLastError();
    e2 = cudaStreamEndCapture(c->cap, &body_out);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      cudaGraphDestroy(g);
      return c->fail(MG_ERR_CUDA, std::string(who) + ": body capture: " +
                                      cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    GraphEntry ge;
    ge.nkernels = nk_init;
    ge.nbody = nk_body;
    e = cudaGraphInstantiate(&ge.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess)
      return c->fail(MG_ERR_CUDA, std::string(who) + ": instantiate: " + cudaGetErrorString(e));
    if (c->graphs.size() > 512) {
      for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
      c->graphs.clear();
    }
    it = c->graphs.emplace(key, ge).first;
  }
  MG_CUDA(cudaGraphLaunch(it->second.exec, s));
  MG_CUDA(cudaMemcpyAsync(c->h_state, c->state, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
  MG_CUDA(cudaStreamSynchronize(s));
  c->launches += it->second.nkernels + (int64_t)c->h_state[2] * it->second.nbody;
  return bounds_status(c, s, who);
}

// Copies the per-right-hand-side iteration counts and relative residuals of
// a finished solve to the host (either pointer may be NULL), ordered on the
// solve's stream s and waited for: s may be a non-blocking stream, which a
// plain cudaMemcpy on the legacy default stream would not wait for.
mg_status read_results(mg_ctx* c, cudaStream_t s, int B, int32_t* iters_out, double* relres_out) {
  if (iters_out)
    MG_CUDA(cudaMemcpyAsync(iters_out, c->iters, B * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (relres_out)
    MG_CUDA(cudaMemcpyAsync(relres_out, c->relres, B * sizeof(double), cudaMemcpyDeviceToHost, s));
  MG_CUDA(cudaStreamSynchronize(s));
  return MG_OK;
}

}  // namespace

// ------------------------------------------------------------ C ABI -------

extern "C" mg_status mg_last_error(const mg_ctx* ctx, char* buf, size_t len) {
  if (!buf || len == 0) return MG_ERR_INVALID;
  std::string m;
  if (ctx) {
    m = ctx->err;
  } else {
    std::lock_guard<std::mutex> lk(g_err_mu);
    m = g_err;
  }
  snprintf(buf, len, "%s", m.c_str());
  return MG_OK;
}

extern "C" int64_t mg_kernel_launches(const mg_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" void mg_destroy(mg_ctx* c) {
  if (!c) return;
  std::lock_guard<std::recursive_mutex> lk(mgi::setup_mutex());
  if (c->cap) cudaStreamSynchronize(c->cap);
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
  for (auto& L : c->d64) free_level(L);
  for (auto& L : c->d32) free_level(L);
  for (void* p : {(void*)c->cholP, (void*)c->cholInv, (void*)c->sq_scratch, c->blk_state,
                  (void*)c->k_r, (void*)c->k_z, (void*)c->k_p, (void*)c->k_q,
                  (void*)c->k_partial, (void*)c->k_small, (void*)c->k32_p, (void*)c->k32_q,
                  (void*)c->k32_e, c->k32_small, (void*)c->gm_V, (void*)c->gm_Z,
                  (void*)c->gm_small, (void*)c->gm_h, (void*)c->gm_vec, (void*)c->gm_partial,
                  (void*)c->gm_zero32, (void*)c->gm_done, c->cheb_dev})
    if (p) cudaFree(p);
  void* ptrs[] = {c->cholL,  c->cholU,  c->cholDinv, c->prm64,  c->prm32, c->partial,
                  c->rsum,   c->fsum,   c->relres,   c->w64,    c->active, c->iters,
                  c->sexp,   c->sexp_prev, c->state, c->c32,    c->rhat32, c->hf, c->hu,
                  c->tol_dev};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (void* p : c->tr_alloc)
    if (p) cudaFree(p);
  if (c->h_state) cudaFreeHost(c->h_state);
  if (c->cap) cudaStreamDestroy(c->cap);
  delete c;
}

// Opts every SELL halo kernel instance in to kSellHaloSmemMax bytes of
// dynamic shared memory.
template <class T, int MODE>
static cudaError_t sell_halo_attrs_mode() {
  const int bytes = (int)kSellHaloSmemMax;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(mgk::k_halo_sell<T, 1, MODE>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(mgk::k_halo_sell<T, 2, MODE>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(mgk::k_halo_sell<T, 4, MODE>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(mgk::k_halo_sell<T, 8, MODE>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(mgk::k_halo_sell<T, 16, MODE>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <class T>
static cudaError_t sell_halo_attrs() {
  cudaError_t e;
  if ((e = sell_halo_attrs_mode<T, mgk::HALO_SMOOTH>()) != cudaSuccess) return e;
  if ((e = sell_halo_attrs_mode<T, mgk::HALO_RESTRICT>()) != cudaSuccess) return e;
  return sell_halo_attrs_mode<T, mgk::HALO_PROLONG>();
}

static mg_status validate_hierarchy(const mg_hierarchy* h, const mg_csr* A, int32_t maxB,
                                    int32_t precision, std::string& why) {
  if (!h || !A) { why = "hierarchy or A_levels is NULL"; return MG_ERR_INVALID; }
  if (h->n_levels < 2 || h->n_levels > 32) { why = "n_levels must be in [2, 32]"; return MG_ERR_INVALID; }
  if (!h->P || !h->inv_deg) { why = "hierarchy arrays are NULL"; return MG_ERR_INVALID; }
  if (maxB < 1 || maxB > kThreads) { why = "max_batch must be in [1, 256]"; return MG_ERR_INVALID; }
  if (precision != 64 && precision != 32) { why = "precision must be 64 or 32"; return MG_ERR_INVALID; }
  const int J = h->n_levels;
  for (int l = 0; l < J; ++l) {
    const int n = A[l].n_rows;
    if (n < 1) { why = "empty level"; return MG_ERR_INVALID; }
    if ((int64_t)n * maxB >= ((int64_t)1 << 31)) {
      why = "rows x max_batch must stay below 2^31";
      return MG_ERR_INVALID;
    }
    std::string m = csr_check(A[l], n, n, "A_levels");
    if (!m.empty()) { why = m + " (level " + std::to_string(l) + ")"; return MG_ERR_INVALID; }
    if (!h->inv_deg[l]) { why = "inv_deg is NULL"; return MG_ERR_INVALID; }
    if (l < J - 1) {
      m = csr_check(h->P[l], n, A[l + 1].n_rows, "P");
      if (!m.empty()) { why = m + " (level " + std::to_string(l) + ")"; return MG_ERR_INVALID; }
    }
  }
  if (A[J - 1].n_rows > 2048) { why = "coarsest level larger than 2048 rows"; return MG_ERR_INVALID; }
  return MG_OK;
}

extern "C" mg_status mg_footprint_bytes(const mg_hierarchy* h, const mg_csr* A, int32_t maxB,
                                        int32_t precision, size_t* bytes) {
  std::string why;
  if (!bytes) return mgi::set_global_error(MG_ERR_INVALID, "bytes is NULL");
  mg_status st = validate_hierarchy(h, A, maxB, precision, why);
  if (st != MG_OK) return mgi::set_global_error(st, "mg_footprint_bytes: " + why);
  const size_t tb = precision == 64 ? 8 : 4;
  size_t total = 0;
  for (int l = 0; l < h->n_levels; ++l) {
    const size_t n = A[l].n_rows;
    const size_t nnz = A[l].nnz;
    // SELL (padding bounded by slice maxima: estimate with nnz), diag/dinv/invdeg,
    // transfer lists, 4 work vectors.
    total += nnz * (4 + tb) + 3 * n * tb + 2 * n * (4 + tb) + 8 * n * (4 + tb) +
             4 * n * maxB * tb;
    if (precision == 32 && l == 0) total += nnz * 12 + 3 * n * 8;
  }
  const size_t nJ = A[h->n_levels - 1].n_rows;
  total += 3 * nJ * nJ * 8;
  const size_t n0 = A[0].n_rows;
  total += 3 * n0 * maxB * 8 + n0 * maxB * 8;  // outer-loop vectors
  *bytes = total;
  return MG_OK;
}

extern "C" mg_status mg_setup(mg_ctx** out, const mg_hierarchy* h, const mg_csr* A,
                              const mg_params* p, int32_t maxB, int32_t precision, void* stream) {
  std::lock_guard<std::recursive_mutex> lk(mgi::setup_mutex());
  if (!out) return mgi::set_global_error(MG_ERR_INVALID, "mg_setup: out is NULL");
  *out = nullptr;
  std::string why;
  mg_status st = validate_hierarchy(h, A, maxB, precision, why);
  if (st != MG_OK) return mgi::set_global_error(st, "mg_setup: " + why);
  const int J = h->n_levels;
  mg_ctx* c = new mg_ctx();
  c->J = J;
  c->prec = precision;
  c->maxB = maxB;
  {
    int dev = 0, sms = 0, tpm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&tpm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) == cudaSuccess &&
        sms > 0 && tpm > 0)
      c->wave_threads = (int64_t)sms * tpm;
  }
  why = read_params(p, J, c->prm, c->nu_pre, c->nu_post);
  if (!why.empty()) {
    delete c;
    return mgi::set_global_error(MG_ERR_INVALID, "mg_setup: " + why);
  }
  c->structure = structure_of(c->prm, J);
  // pack on the host
  std::vector<HostLevel> H(J);
  for (int l = 0; l < J; ++l) {
    why = pack_level(A[l], h->inv_deg[l], l < J - 1 ? &h->P[l] : nullptr, H[l]);
    if (!why.empty()) {
      delete c;
      return mgi::set_global_error(MG_ERR_INVALID,
                                   "mg_setup: level " + std::to_string(l) + ": " + why);
    }
    c->n.push_back(H[l].n);
  }
  std::vector<double> Lc;
  if (!cholesky(A[J - 1], Lc)) {
    delete c;
    return mgi::set_global_error(MG_ERR_NOT_SPD, "mg_setup: coarsest operator is not SPD");
  }
  const int nJ = A[J - 1].n_rows;
  c->nJ = nJ;
  std::vector<double> Ainv;
  if (nJ >= 32 && nJ <= 512) Ainv = coarse_inverse(A[J - 1], Lc, nJ);
  std::vector<double> Uc((size_t)nJ * nJ), dj(nJ);
  for (int i = 0; i < nJ; ++i)
    for (int j = 0; j < nJ; ++j) Uc[i + (size_t)j * nJ] = Lc[j + (size_t)i * nJ];
  for (int j = 0; j < nJ; ++j) dj[j] = 1.0 / Lc[j + (size_t)j * nJ];

  auto bail = [&](cudaError_t e) {
    std::string m = std::string("mg_setup: ") + cudaGetErrorString(e);
    mg_destroy(c);
    return mgi::set_global_error(e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA, m);
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking)) != cudaSuccess) return bail(e);
  for (const void* k : {(const void*)mgk::k_tail<float, 0>, (const void*)mgk::k_tail<float, 1>,
                        (const void*)mgk::k_tail<double, 0>, (const void*)mgk::k_tail<double, 1>})
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kTailSmemMax)) != cudaSuccess)
      return bail(e);
  if ((e = cudaFuncSetAttribute(mgk::k_coarse_chol_packed<float>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax)) !=
      cudaSuccess)
    return bail(e);
  if ((e = cudaFuncSetAttribute(mgk::k_coarse_chol_packed<double>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax)) !=
      cudaSuccess)
    return bail(e);
  if ((e = sell_halo_attrs<float>()) != cudaSuccess) return bail(e);
  if ((e = sell_halo_attrs<double>()) != cudaSuccess) return bail(e);
  // host copies of the SELL patterns the halo tables are built from
  auto keep_pattern = [&](auto& levels) {
    for (int l = 0; l < J - 1; ++l)
      if (H[l].ndia == 0) {
        levels[l].h_slptr = H[l].sl_ptr;
        levels[l].h_col = H[l].col;
      }
  };
  if (precision == 64) {
    c->d64.resize(J);
    for (int l = 0; l < J; ++l)
      if ((e = upload_level(H[l], c->d64[l], maxB, true)) != cudaSuccess) return bail(e);
    keep_pattern(c->d64);
    if ((e = upload_sell_halo(c->d64, c->opt_sell_halo_rows, J)) != cudaSuccess) return bail(e);
    if ((e = cudaMalloc(&c->prm64, c->prm.size() * sizeof(double))) != cudaSuccess) return bail(e);
  } else {
    c->d32.resize(J);
    for (int l = 0; l < J; ++l)
      if ((e = upload_level(H[l], c->d32[l], maxB, true)) != cudaSuccess) return bail(e);
    keep_pattern(c->d32);
    if ((e = upload_sell_halo(c->d32, c->opt_sell_halo_rows, J)) != cudaSuccess) return bail(e);
    c->d64.resize(1);  // FP64 finest operator for the refinement residual
    HostLevel H0 = H[0];
    H0.p_idx.clear(); H0.p_w.clear(); H0.r_idx.clear(); H0.r_w.clear(); H0.nc = 0; H0.KR = 0;
    if ((e = upload_level(H0, c->d64[0], maxB, false)) != cudaSuccess) return bail(e);
    if ((e = cudaMalloc(&c->prm32, c->prm.size() * sizeof(float))) != cudaSuccess) return bail(e);
  }
  if ((e = upload(&c->cholL, Lc)) != cudaSuccess) return bail(e);
  if ((e = upload(&c->cholU, Uc)) != cudaSuccess) return bail(e);
  if ((e = upload(&c->cholDinv, dj)) != cudaSuccess) return bail(e);
  if (!Ainv.empty()) {
    if ((e = upload(&c->cholInv, Ainv)) != cudaSuccess) return bail(e);
    c->coarse_inv = true;
  }
  {
    std::vector<double> Pk;
    Pk.reserve((size_t)nJ * (nJ + 1) / 2);
    for (int j = 0; j < nJ; ++j)
      for (int i = j; i < nJ; ++i) Pk.push_back(Lc[i + (size_t)j * nJ]);
    if ((e = upload(&c->cholP, Pk)) != cudaSuccess) return bail(e);
  }
  // outer-loop workspace
  const int n0 = H[0].n;
  c->nblk_max = n0;  // R >= 1 rows per block
  const size_t v64 = (size_t)n0 * maxB * sizeof(double);
  if ((e = cudaMalloc(&c->partial, (size_t)c->nblk_max * maxB * sizeof(double))) != cudaSuccess) return bail(e);
  for (double** q : {&c->rsum, &c->fsum, &c->relres})
    if ((e = cudaMalloc(q, maxB * sizeof(double))) != cudaSuccess) return bail(e);
  for (int** q : {&c->active, &c->iters, &c->sexp, &c->sexp_prev})
    if ((e = cudaMalloc(q, maxB * sizeof(int))) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&c->state, 4 * sizeof(int))) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&c->tol_dev, 3 * sizeof(double))) != cudaSuccess) return bail(e);
  if ((e = cudaMallocHost(&c->h_state, 4 * sizeof(int))) != cudaSuccess) return bail(e);
  if (precision == 64) {
    if ((e = cudaMalloc(&c->w64, v64)) != cudaSuccess) return bail(e);
  } else {
    if ((e = cudaMalloc(&c->c32, (size_t)n0 * maxB * sizeof(float))) != cudaSuccess) return bail(e);
    if ((e = cudaMalloc(&c->rhat32, (size_t)n0 * maxB * sizeof(float))) != cudaSuccess) return bail(e);
  }
  // the synchronous copies are complete; wait for the memsets on the legacy
  // stream only (a device-wide synchronisation would also wait on, and could
  // disturb, other threads' streams)
  if ((e = cudaStreamSynchronize(cudaStreamLegacy)) != cudaSuccess) return bail(e);
  *out = c;
  (void)stream;
  return MG_OK;
}

extern "C" mg_status mg_set_params(mg_ctx* c, const mg_params* p) {
  if (!c) return mgi::set_global_error(MG_ERR_INVALID, "mg_set_params: ctx is NULL");
  std::vector<double> prm;
  int a, b;
  std::string why = read_params(p, c->J, prm, a, b);
  if (!why.empty()) return c->fail(MG_ERR_INVALID, "mg_set_params: " + why);
  if (a != c->nu_pre || b != c->nu_post) {  // the cycle's shape changed
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
    c->graphs.clear();
  }
  c->prm = prm;
  c->nu_pre = a;
  c->nu_post = b;
  c->structure = structure_of(prm, c->J);
  c->prm_dirty = true;
  c->param_version++;
  return MG_OK;
}

extern "C" mg_status mg_set_cheb(mg_ctx* c, int32_t K, const double* coef) {
  if (!c) return mgi::set_global_error(MG_ERR_INVALID, "mg_set_cheb: ctx is NULL");
  if (K < 0 || K > MG_CHEB_MAX_DEGREE)
    return c->fail(MG_ERR_INVALID, "mg_set_cheb: degree out of range");
  if (K > 0 && !coef) return c->fail(MG_ERR_INVALID, "mg_set_cheb: coef is NULL");
  const int S = MG_CHEB_MAX_DEGREE + 1;
  std::vector<double> v((size_t)c->J * S, 0.0);
  for (int l = 0; K > 0 && l < c->J - 1; ++l)
    for (int k = 0; k <= K; ++k) {
      const double x = coef[(size_t)l * (K + 1) + k];
      if (!std::isfinite(x)) return c->fail(MG_ERR_INVALID, "mg_set_cheb: non-finite coef");
      v[(size_t)l * S + k] = x;
    }
  if (!c->cheb_dev)
    MG_CUDA(cudaMalloc(&c->cheb_dev, v.size() * (c->prec == 64 ? sizeof(double) : sizeof(float))));
  if (K != c->cheb_K) {  // other kernels in the cycle
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
    c->graphs.clear();
  }
  c->cheb_host = v;
  c->cheb_K = K;
  c->cheb_dirty = true;
  c->param_version++;
  return MG_OK;
}

extern "C" mg_status mg_level_sizes(const mg_ctx* c, int32_t* J, int32_t* n) {
  if (!c || !J) return MG_ERR_INVALID;
  *J = c->J;
  if (n)
    for (int l = 0; l < c->J; ++l) n[l] = c->n[l];
  return MG_OK;
}

extern "C" mg_status mg_vcycle(mg_ctx* c, const void* f, void* u, int32_t B, void* stream) {
  if (!c) return mgi::set_global_error(MG_ERR_INVALID, "mg_vcycle: ctx is NULL");
  if (!f || !u || B < 1 || B > c->maxB) return c->fail(MG_ERR_INVALID, "mg_vcycle: bad arguments");
  if (f == u) return c->fail(MG_ERR_INVALID, "mg_vcycle: f and u must not alias");
  cudaStream_t s = (cudaStream_t)stream;
  mg_status st = sync_params(c, s);
  if (st != MG_OK) return st;
  auto key = std::make_tuple(0, f, (const void*)u, (int)B, c->structure);
  if (c->prec == 64)
    return run_graph(c, key, s, [&](cudaStream_t cs) {
      Issue<double> is{c, c->d64, c->prm64, cs, B};
      is.vcycle((const double*)f, (double*)u, false);
      return is.nk;
    });
  return run_graph(c, key, s, [&](cudaStream_t cs) {
    Issue<float> is{c, c->d32, c->prm32, cs, B};
    is.vcycle((const float*)f, (float*)u, false);
    return is.nk;
  });
}

extern "C" mg_status mg_fmg(mg_ctx* c, const void* f, void* u, int32_t B, void* stream) {
  if (!c) return mgi::set_global_error(MG_ERR_INVALID, "mg_fmg: ctx is NULL");
  if (!f || !u || B < 1 || B > c->maxB) return c->fail(MG_ERR_INVALID, "mg_fmg: bad arguments");
  if (f == u) return c->fail(MG_ERR_INVALID, "mg_fmg: f and u must not alias");
  cudaStream_t s = (cudaStream_t)stream;
  mg_status st = sync_params(c, s);
  if (st != MG_OK) return st;
  auto key = std::make_tuple(6, f, (const void*)u, (int)B, c->structure);
  if (c->prec == 64)
    return run_graph(c, key, s, [&](cudaStream_t cs) {
      Issue<double> is{c, c->d64, c->prm64, cs, B};
      is.fmg((const double*)f, (double*)u);
      return is.nk;
    });
  return run_graph(c, key, s, [&](cudaStream_t cs) {
    Issue<float> is{c, c->d32, c->prm32, cs, B};
    is.fmg((const float*)f, (float*)u);
    return is.nk;
  });
}

namespace {

__global__ void k_init_solve(const double* __restrict__ fsum, int B, int* __restrict__ active,
                             int* __restrict__ iters, int* __restrict__ sexp) {
  mgk::pdl_wait();
  const int b = threadIdx.x + blockIdx.x * blockDim.x;
  if (b >= B) return;
  active[b] = 1;
  iters[b] = 0;
  const double fn = sqrt(fsum[b]);
  sexp[b] = fn > 0.0 && isfinite(fn) ? ilogb(fn) : 0;
}

__global__ void k_shift_sexp(int* __restrict__ sexp, int* __restrict__ sexp_prev, int B) {
  mgk::pdl_wait();
  const int b = threadIdx.x;
  if (b < B) sexp_prev[b] = sexp[b];
}

__global__ void k_bump_iters(const int* __restrict__ active, int* __restrict__ iters, int B) {
  mgk::pdl_wait();
  const int b = threadIdx.x;
  if (b < B && active[b]) iters[b] += 1;
}

// Per-right-hand-side sums of c->partial into c->rsum, the copy
// sexp_prev = sexp (when given) and the convergence test.  For small
// B * nblk one block does all three (k_reduce_check: the same sums in the
// same order, two launches fewer per iteration of a latency-bound solve);
// otherwise k_reduce over B blocks, the copy and k_check.
constexpr int64_t kMergeReduceMax = 32768;
void reduce_and_check(Issue<double>& is, mg_ctx* c, int nblk, int B, int* sexp_prev, int inc,
                      cudaGraphConditionalHandle h, int cond) {
  if ((int64_t)B * nblk <= kMergeReduceMax) {
    is.launch(mgk::k_reduce_check, dim3(1), dim3(kThreads), 0, (const double*)c->partial, nblk,
              c->rsum, sexp_prev, (const double*)c->fsum, B, (const double*)c->tol_dev, c->active,
              c->relres, c->sexp, c->state, inc, h, cond);
    return;
  }
  is.launch(mgk::k_reduce, dim3(B), dim3(kThreads), 0, (const double*)c->partial, nblk, B,
            c->rsum);
  if (sexp_prev) is.launch(k_shift_sexp, dim3(1), dim3(kThreads), 0, c->sexp, sexp_prev, B);
  is.launch(mgk::k_check, dim3(1), dim3(kThreads), 0, (const double*)c->rsum,
            (const double*)c->fsum, B, (const double*)c->tol_dev, c->active, c->relres, c->sexp,
            c->state, inc, h, cond);
}

}  // namespace

extern "C" mg_status mg_solve(mg_ctx* c, const double* f, double* u, int32_t B, double tol,
                              int32_t max_iter, int32_t* iters_out, double* relres_out,
                              void* stream) {
  if (!c) return mgi::set_global_error(MG_ERR_INVALID, "mg_solve: ctx is NULL");
  if (!f || !u || B < 1 || B > c->maxB || max_iter < 0 || !(tol > 0.0))
    return c->fail(MG_ERR_INVALID, "mg_solve: bad arguments");
  if ((const void*)f == (const void*)u) return c->fail(MG_ERR_INVALID, "mg_solve: f and u alias");
  cudaStream_t s = (cudaStream_t)stream;
  mg_status st = sync_params(c, s);
  if (st != MG_OK) return st;
  const int n0 = c->n[0];
  const int bt = std::min((int)B, 32);  // reduction tiling (kernels.cuh red_tile)
  const int nblk = (n0 + mgk::kRedRows - 1) / mgk::kRedRows;
  const dim3 rgrid(nblk, (B + bt - 1) / bt), rblock(mgk::kRedRows * bt);
  const LV<double> L0 = c->d64[0].view();
  const bool p32 = c->prec == 32;
  c->solve_ctl[0] = tol;
  c->solve_ctl[1] = (double)max_iter;
  MG_CUDA(cudaMemcpyAsync(c->tol_dev, c->solve_ctl, 2 * sizeof(double), cudaMemcpyHostToDevice, s));

  // residual of the current iterate, its norms and the convergence test
  auto check_tail = [&](Issue<double>& is, cudaGraphConditionalHandle h, int inc, int cond) {
    is.launch(mgk::k_resid64, rgrid, rblock, 0, L0, (const double*)f, (const double*)u,
              p32 ? c->rhat32 : (float*)nullptr, (const int*)c->sexp, (int)B, c->partial,
              p32 ? c->d32[0].t : (float*)nullptr,
              p32 ? (const float*)c->d32[0].dinv : (const float*)nullptr, (const float*)c->prm32);
    reduce_and_check(is, c, nblk, (int)B, p32 ? c->sexp_prev : (int*)nullptr, inc, h, cond);
  };
  auto pre = [&](cudaStream_t cs, cudaGraphConditionalHandle h, int cond) {
    Issue<double> is{c, c->d64, c->prm64, cs, B};
    is.launch(mgk::k_sumsq64, rgrid, rblock, 0, f, n0, (int)B, c->partial);
    is.launch(mgk::k_reduce, dim3(B), dim3(kThreads), 0, (const double*)c->partial, nblk, (int)B,
              c->fsum);
    is.launch(k_init_solve, dim3(1), dim3(kThreads), 0, (const double*)c->fsum, (int)B, c->active,
              c->iters, c->sexp);
    check_tail(is, h, 0, cond);
    return is.nk;
  };
  auto body = [&](cudaStream_t cs, cudaGraphConditionalHandle h, int cond) {
    int nk = 0;
    if (p32) {
      Issue<float> is{c, c->d32, c->prm32, cs, B};
      is.delta0_ready = true;  // check_tail's k_resid64 wrote the first step's delta
      if (B == 1) is.rfold = mgk::RefineEp{u, c->sexp_prev, c->active, c->iters, n0};
      is.vcycle(c->rhat32, c->c32, true);
      if (!is.rfold_done)
        is.launch(mgk::k_refine_update, grid_for((size_t)n0 * B), dim3(kThreads), 0, u,
                  (const float*)c->c32, (const int*)c->sexp_prev, (const int*)c->active, n0,
                  (int)B, c->iters);
      nk += is.nk;
      Issue<double> is2{c, c->d64, c->prm64, cs, B};
      check_tail(is2, h, 1, cond);
      nk += is2.nk;
    } else {
      Issue<double> is{c, c->d64, c->prm64, cs, B};
      if (B == 1) {
        is.vcycle(f, u, false);
        is.launch(k_bump_iters, dim3(1), dim3(kThreads), 0, (const int*)c->active, c->iters,
                  (int)B);
      } else {
        is.launch(mgk::k_copy<double>, grid_for((size_t)n0 * B), dim3(kThreads), 0,
                  (const double*)u, c->w64, (size_t)n0 * B);
        is.vcycle(f, c->w64, false);
        is.launch(mgk::k_masked_copy, grid_for((size_t)n0 * B), dim3(kThreads), 0, u,
                  (const double*)c->w64, (const int*)c->active, n0, (int)B, c->iters);
      }
      check_tail(is, h, 1, cond);
      nk += is.nk;
    }
    return nk;
  };
  st = run_loop(c, 30, f, u, (int)B, s, "mg_solve", pre, body,
                [](cudaStream_t) { return 0; }, false);
  if (st != MG_OK) return st;
  mg_status result = MG_OK;
  if (c->h_state[1])
    result = MG_ERR_DIVERGED;
  else if (c->h_state[0] > 0)
    result = MG_NOT_CONVERGED;
  if ((st = read_results(c, s, (int)B, iters_out, relres_out)) != MG_OK) return st;
  if (result == MG_ERR_DIVERGED) c->err = "mg_solve: non-finite residual";
  if (result == MG_NOT_CONVERGED) c->err = "mg_solve: tolerance not met within max_iter";
  return result;
}

extern "C" mg_status mg_solve_host(mg_ctx* c, const double* fh, double* uh, int32_t B, double tol,
                                   int32_t max_iter, int32_t* iters_out, double* relres_out,
                                   void* stream) {
  if (!c) return mgi::set_global_error(MG_ERR_INVALID, "mg_solve_host: ctx is NULL");
  if (!fh || !uh || B < 1 || B > c->maxB) return c->fail(MG_ERR_INVALID, "mg_solve_host: bad arguments");
  const size_t bytes = (size_t)c->n[0] * B * sizeof(double);
  if (!c->hf) {
    MG_CUDA(cudaMalloc(&c->hf, (size_t)c->n[0] * c->maxB * sizeof(double)));
    MG_CUDA(cudaMalloc(&c->hu, (size_t)c->n[0] * c->maxB * sizeof(double)));
  }
  cudaStream_t s = (cudaStream_t)stream;
  MG_CUDA(cudaMemcpyAsync(c->hf, fh, bytes, cudaMemcpyHostToDevice, s));
  MG_CUDA(cudaMemcpyAsync(c->hu, uh, bytes, cudaMemcpyHostToDevice, s));
  mg_status st = mg_solve(c, c->hf, c->hu, B, tol, max_iter, iters_out, relres_out, stream);
  if (st < 0) return st;
  MG_CUDA(cudaMemcpyAsync(uh, c->hu, bytes, cudaMemcpyDeviceToHost, s));
  MG_CUDA(cudaStreamSynchronize(s));
  return st;
}

extern "C" mg_status mg_level_apply(mg_ctx* c, int32_t lev, int32_t op, const void* x,
                                    const void* y, void* out, int32_t B, void* stream) {
  if (!c) return mgi::set_global_error(MG_ERR_INVALID, "mg_level_apply: ctx is NULL");
  if (lev < 0 || lev >= c->J || B < 1 || B > c->maxB || !x || !out)
    return c->fail(MG_ERR_INVALID, "mg_level_apply: bad arguments");
  if ((op == MG_OP_SMOOTH || op == MG_OP_RESIDUAL || op == MG_OP_PROLONG) && !y)
    return c->fail(MG_ERR_INVALID, "mg_level_apply: y is required for this op");
  if ((op == MG_OP_RESTRICT || op == MG_OP_PROLONG || op == MG_OP_SMOOTH) && lev == c->J - 1)
    return c->fail(MG_ERR_INVALID, "mg_level_apply: no transfer/smoother on the coarsest level");
  if (op == MG_OP_COARSE && lev != c->J - 1)
    return c->fail(MG_ERR_INVALID, "mg_level_apply: coarse solve only on the coarsest level");
  if (op < MG_OP_SMOOTH || op > MG_OP_REFINE_RESIDUAL)
    return c->fail(MG_ERR_INVALID, "mg_level_apply: op");
  if (op == MG_OP_REFINE_RESIDUAL) {
    // the pre-loop kernels of mg_solve's refinement with the FP32 copy
    // written to out: ||f||, s = ilogb ||f||, r = f - A u, float(2^-s r)
    if (lev != 0 || !y) return c->fail(MG_ERR_INVALID, "mg_level_apply: refine residual needs level 0, f, u");
    if (out == x || out == y) return c->fail(MG_ERR_INVALID, "mg_level_apply: out aliases an input");
    cudaStream_t s = (cudaStream_t)stream;
    const int n0 = c->n[0];
    const int bt = std::min((int)B, 32);
    const int nblk = (n0 + mgk::kRedRows - 1) / mgk::kRedRows;
    const dim3 rgrid(nblk, (B + bt - 1) / bt), rblock(mgk::kRedRows * bt);
    Issue<double> is{c, c->d64, c->prm64, s, B};
    is.launch(mgk::k_sumsq64, rgrid, rblock, 0, (const double*)x, n0, (int)B, c->partial);
    is.launch(mgk::k_reduce, dim3(B), dim3(kThreads), 0, (const double*)c->partial, nblk, (int)B,
              c->fsum);
    is.launch(k_init_solve, dim3(1), dim3(kThreads), 0, (const double*)c->fsum, (int)B, c->active,
              c->iters, c->sexp);
    is.launch(mgk::k_resid64, rgrid, rblock, 0, c->d64[0].view(), (const double*)x,
              (const double*)y, (float*)out, (const int*)c->sexp, (int)B, c->partial,
              (float*)nullptr, (const float*)nullptr, (const float*)nullptr);
    MG_CUDA(cudaGetLastError());
    c->launches += is.nk;
    return MG_OK;
  }
  if (op == MG_OP_OUTER_RESIDUAL) {
    if (lev != 0 || !y) return c->fail(MG_ERR_INVALID, "mg_level_apply: outer residual needs level 0, f, u");
    if (out == x || out == y) return c->fail(MG_ERR_INVALID, "mg_level_apply: out aliases an input");
    cudaStream_t s = (cudaStream_t)stream;
    const int bt = std::min((int)B, 32);
    const dim3 rgrid((c->n[0] + mgk::kRedRows - 1) / mgk::kRedRows, (B + bt - 1) / bt);
    mgk::k_outer_residual64<<<rgrid, mgk::kRedRows * bt, 0, s>>>(
        c->d64[0].view(), (const double*)x, (const double*)y, (double*)out, B);
    MG_CUDA(cudaGetLastError());
    c->launches += 1;
    return MG_OK;
  }
  if (out == x || out == y) return c->fail(MG_ERR_INVALID, "mg_level_apply: out aliases an input");
  cudaStream_t s = (cudaStream_t)stream;
  mg_status st = sync_params(c, s);
  if (st != MG_OK) return st;
  auto go = [&](auto& levels, auto* prm) -> mg_status {
    using T = std::remove_pointer_t<decltype(prm)>;
    Issue<T> is{c, levels, prm, s, B};
    auto& D = levels[lev];
    const T* X = (const T*)x;
    const T* Y = (const T*)y;
    T* O = (T*)out;
    const size_t vb = (size_t)D.n * B * sizeof(T);
    switch (op) {
      case MG_OP_SMOOTH:
        MG_CUDA(cudaMemcpyAsync(O, Y, vb, cudaMemcpyDeviceToDevice, s));
        is.smooth(lev, X, O, 1, false);
        break;
      case MG_OP_RESIDUAL:
        (B == 1 ? mgk::k_residual<T, 1> : mgk::k_residual<T, 0>)<<<grid_for((size_t)D.n * B), kThreads, 0, s>>>(D.view(), X, Y, O, B,
                                                                          is.P(lev), 0, 0);
        is.nk++;
        break;
      case MG_OP_RESTRICT:
        (B == 1 ? mgk::k_restrict<T, 1> : mgk::k_restrict<T, 0>)<<<grid_for((size_t)D.nc * B), kThreads, 0, s>>>(
            D.view(), X, O, B, is.P(lev), is.conv(lev, mgk::P_WR2));
        is.nk++;
        break;
      case MG_OP_PROLONG:
        (B == 1 ? mgk::k_prolong<T, 1> : mgk::k_prolong<T, 0>)<<<grid_for((size_t)D.n * B), kThreads, 0, s>>>(
            D.view(), X, Y, O, B, is.P(lev), is.conv(lev, mgk::P_WP2));
        is.nk++;
        break;
      case MG_OP_COARSE:
        is.coarse(X, O);
        break;
    }
    MG_CUDA(cudaGetLastError());
    c->launches += is.nk;
    return MG_OK;
  };
  if (c->prec == 64) return go(c->d64, c->prm64);
  return go(c->d32, c->prm32);
}

extern "C" const char* mg_kernel_name(int32_t kind) {
  switch (kind) {
    case MG_K_JACOBI: return "jacobi_smooth";
    case MG_K_RESIDUAL_SCALED: return "residual_scaled";
    case MG_K_CONV_UPDATE: return "sage_conv_update";
    case MG_K_RESIDUAL: return "residual";
    case MG_K_RESTRICT: return "restrict_conv";
    case MG_K_PROLONG: return "prolong_conv";
    case MG_K_COARSE_CHOL: return "coarse_cholesky";
    case MG_K_OUTER_RESIDUAL: return "outer_residual_fp64";
    case MG_K_TAIL: return "small_levels_block";
    case MG_K_CONV_R: return "restrict_conv_fine";
    case MG_K_PE: return "prolong_fine";
    case MG_K_SMOOTH_HALO: return "smooth_halo";
    case MG_K_RESTRICT_HALO: return "restrict_conv_halo";
    case MG_K_PROLONG_HALO: return "prolong_halo";
    case MG_K_CHEB_STEP: return "cheb_conv_update";
    default: return "unknown";
  }
}

extern "C" mg_status mg_vcycle_profile(mg_ctx* c, const void* f, void* u, int32_t B,
                                       mg_kernel_time* out, int32_t max_out, int32_t* n_out,
                                       void* stream) {
  if (!c) return mgi::set_global_error(MG_ERR_INVALID, "mg_vcycle_profile: ctx is NULL");
  if (!f || !u || B < 1 || B > c->maxB || !out || !n_out || max_out < 0)
    return c->fail(MG_ERR_INVALID, "mg_vcycle_profile: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  mg_status st = sync_params(c, s);
  if (st != MG_OK) return st;
  std::vector<std::tuple<int, int, cudaEvent_t, cudaEvent_t>> rec;
  if (c->prec == 64) {
    Issue<double> is{c, c->d64, c->prm64, s, B};
    is.rec = &rec;
    is.vcycle((const double*)f, (double*)u, false);
    c->launches += is.nk;
  } else {
    Issue<float> is{c, c->d32, c->prm32, s, B};
    is.rec = &rec;
    is.vcycle((const float*)f, (float*)u, false);
    c->launches += is.nk;
  }
  cudaError_t e = cudaStreamSynchronize(s);
  int k = 0;
  for (auto& r : rec) {
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, std::get<2>(r), std::get<3>(r));
    if (k < max_out) {
      out[k].kernel = std::get<0>(r);
      out[k].level = std::get<1>(r);
      out[k].ms = ms;
    }
    ++k;
    cudaEventDestroy(std::get<2>(r));
    cudaEventDestroy(std::get<3>(r));
  }
  *n_out = std::min(k, max_out);
  MG_CUDA(e);
  return MG_OK;
}

#include "train_impl.cuh"
#include "krylov_impl.cuh"
#include "gmres_impl.cuh"
#include "square_impl.cuh"

extern "C" mg_status mg_set_option(mg_ctx* c, int32_t option, int64_t value) {
  if (!c) return mgi::set_global_error(MG_ERR_INVALID, "mg_set_option: ctx is NULL");
  std::lock_guard<std::recursive_mutex> lk(mgi::setup_mutex());
  switch (option) {
    case MG_OPT_TAIL_WORK:
      if (value < 0) return c->fail(MG_ERR_INVALID, "mg_set_option: tail work must be >= 0");
      c->opt_tail_work = value;
      break;
    case MG_OPT_PDL:
      c->opt_pdl = value != 0;
      break;
    case MG_OPT_MULTI_RHS:
      if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != 16)
        return c->fail(MG_ERR_INVALID, "mg_set_option: multi-rhs tile must be 0, 1, 2, 4, 8 or 16");
      c->opt_multi_rhs = (int)value;
      break;
    case MG_OPT_DEVICE_LOOP:
      c->opt_device_loop = value != 0;
      break;
    case MG_OPT_FCG_PRECOND:
      if (value != 0 && value != 1)
        return c->fail(MG_ERR_INVALID, "mg_set_option: FCG preconditioner must be 0 or 1");
      c->opt_fcg_precond = (int)value;
      break;
    case MG_OPT_FGMRES_FLOOR:
      if (value < 0 || value > 15)
        return c->fail(MG_ERR_INVALID, "mg_set_option: FGMRES floor must be in [0, 15]");
      c->opt_fgmres_floor = (int)value;
      break;
    case MG_OPT_FCG_FP32:
      if (value != 0 && value != 1 && value != 2)
        return c->fail(MG_ERR_INVALID, "mg_set_option: FCG FP32 must be 0, 1 or 2");
      c->opt_fcg_fp32 = (int)value;
      break;
    case MG_OPT_FCG_FLOOR:
      if (value < 0 || value > 15)
        return c->fail(MG_ERR_INVALID, "mg_set_option: FCG floor must be in [0, 15]");
      c->opt_fcg_floor = (int)value;
      break;
    case MG_OPT_HALO_ROWS:
      if (value < 0 || value > (1 << 30))
        return c->fail(MG_ERR_INVALID, "mg_set_option: halo rows must be in [0, 2^30]");
      c->opt_halo_rows = value;
      break;
    case MG_OPT_HALO2D_BYTES:
      if (value < 0) return c->fail(MG_ERR_INVALID, "mg_set_option: 2D halo bytes must be >= 0");
      c->opt_halo2d_bytes = value;
      break;
    case MG_OPT_DIA_TWO_ROWS:
      if (value != 0 && value != 1)
        return c->fail(MG_ERR_INVALID, "mg_set_option: DIA two rows must be 0 or 1");
      c->opt_dia_two_rows = (int)value;
      break;
    case MG_OPT_TAIL_TEAMS:
      if (value < 0 || value > 64)
        return c->fail(MG_ERR_INVALID, "mg_set_option: tail teams must be in [0, 64]");
      c->opt_tail_teams = (int)value;
      break;
    case MG_OPT_COARSE_INVERSE:
      if (value != 0 && value != 1)
        return c->fail(MG_ERR_INVALID, "mg_set_option: coarse inverse must be 0 or 1");
      c->coarse_inv = value == 1 && c->cholInv != nullptr;
      break;
    case MG_OPT_SELL_HALO_MAX_BYTES:
      if (value < 0) return c->fail(MG_ERR_INVALID, "mg_set_option: byte cap must be >= 0");
      c->opt_sell_halo_max_bytes = value;
      break;
    case MG_OPT_SELL_HALO_THREADS:
      if (value < 32 || value > mgk::kTailThreads || value % 32 != 0)
        return c->fail(MG_ERR_INVALID,
                       "mg_set_option: SELL halo threads must be a multiple of 32 up to 1024");
      c->opt_sell_halo_threads = (int)value;
      break;
    case MG_OPT_SELL_HALO_ROWS: {
      if (value < 0 || value > 8192 || value % mgk::kSlice != 0)
        return c->fail(MG_ERR_INVALID,
                       "mg_set_option: SELL halo rows must be 0 or a multiple of 32 up to 8192");
      if (value == c->opt_sell_halo_rows) return MG_OK;
      // work in flight may read the old tables
      MG_CUDA(cudaDeviceSynchronize());
      c->opt_sell_halo_rows = (int)value;
      MG_CUDA(c->prec == 64 ? upload_sell_halo(c->d64, (int)value, c->J)
                            : upload_sell_halo(c->d32, (int)value, c->J));
      break;
    }
    default:
      return c->fail(MG_ERR_INVALID, "mg_set_option: unknown option");
  }
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
  c->graphs.clear();
  return MG_OK;
}

extern "C" int32_t mg_debug_bounds(uint64_t* word) {
#ifdef MG_BOUNDS_CHECK
  unsigned long long w = 0;
  if (cudaMemcpyFromSymbol(&w, mgk::g_bounds_error, sizeof(w)) != cudaSuccess) return -1;
  const unsigned long long zero = 0;
  if (w && cudaMemcpyToSymbol(mgk::g_bounds_error, &zero, sizeof(zero)) != cudaSuccess) return -1;
  if (word) *word = w;
  return 1;
#else
  if (word) *word = 0;
  return 0;
#endif
}

extern "C" mg_status mg_set_layout_policy(int32_t policy) {
  if (policy != 0 && policy != 1)
    return mgi::set_global_error(MG_ERR_INVALID, "mg_set_layout_policy: policy must be 0 or 1");
  g_layout_policy = policy;
  return MG_OK;
}
