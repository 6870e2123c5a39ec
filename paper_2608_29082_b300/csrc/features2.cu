// Learnable multigrid with two features per node (d = 2).
//
// The paper's Helmholtz experiment (Sec. 4.3) solves a complex system and
// carries the real and imaginary parts of the solution as two node features;
// each SAGEConv then holds W_1, W_2 in R^{2x2} (Sec. 3.2) and may mix them.
// This translation unit is that cycle (Algorithm 2) on complex operators:
//   delta = theta D_A^{-1}(f - A u)          complex arithmetic
//   u <- u + eta Phi_B(delta)                Phi(x)_i = W_1 x_i + W_2 mean x_j
//   r_c = P^T Phi_R(f - A u),  u <- u + Phi_P(P e_c)    (real P)
//   coarsest level: e = A_J^{-1} r, A_J inverted once on the host (FP64)
// Vectors are [n][nrhs] complex, (Re, Im) adjacent, in the context's
// precision; operators are CSR with complex values.  One thread per (row,
// right-hand side).  The context owns every device buffer it allocates.
// A cycle is captured once per (f, u, nrhs) into a CUDA graph on a private
// stream and replayed on the caller's stream; parameters are kernel
// arguments, so mg2_set_params drops the captured graphs.
#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "mg.h"
#include "mg_internal.h"

namespace {

constexpr int kF2Threads = 256;

template <class T>
struct Pair;
template <>
struct Pair<float> {
  using type = float2;
};
template <>
struct Pair<double> {
  using type = double2;
};

// (W_1, W_2) of one SAGEConv, row-major 2 x 2 each: w[0] = W_1, w[1] = W_2
template <class T>
struct Conv2 {
  T w[2][2][2];
};

// out = f - A u (u_zero: u = 0), then optionally out = theta * out / A_ii
// (dinv = 1 / A_ii, complex)
template <class T>
__global__ void __launch_bounds__(kF2Threads)
    k2_residual(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                const typename Pair<T>::type* __restrict__ av,
                const typename Pair<T>::type* __restrict__ f,
                const typename Pair<T>::type* __restrict__ u, typename Pair<T>::type* __restrict__ out,
                int B, const typename Pair<T>::type* __restrict__ dinv, T theta, int scale,
                int u_zero) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * B) return;
  const int i = (int)(t / B), b = (int)(t - (size_t)i * B);
  typename Pair<T>::type r = f[t];
  if (!u_zero) {
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const typename Pair<T>::type a = av[e];
      const typename Pair<T>::type x = u[(size_t)ci[e] * B + b];
      r.x -= a.x * x.x - a.y * x.y;
      r.y -= a.x * x.y + a.y * x.x;
    }
  }
  if (scale) {
    const typename Pair<T>::type d = dinv[i];
    const T re = r.x * d.x - r.y * d.y, im = r.x * d.y + r.y * d.x;
    r.x = theta * re;
    r.y = theta * im;
  }
  out[t] = r;
}

// phi_i = W_1 x_i + W_2 inv_deg_i sum_{j != i in row i} x_j; mode 0: y = phi,
// 1: y += eta phi, 2: y += phi.  x and y are distinct buffers.
template <class T>
__global__ void __launch_bounds__(kF2Threads)
    k2_conv(int n, const int* __restrict__ rp, const int* __restrict__ ci,
            const T* __restrict__ invdeg, const typename Pair<T>::type* __restrict__ x,
            typename Pair<T>::type* __restrict__ y, int B, Conv2<T> w, T eta, int mode) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * B) return;
  const int i = (int)(t / B), b = (int)(t - (size_t)i * B);
  T sx = T(0), sy = T(0);
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const int c = ci[e];
    if (c == i) continue;
    const typename Pair<T>::type v = x[(size_t)c * B + b];
    sx += v.x;
    sy += v.y;
  }
  const T mx = invdeg[i] * sx, my = invdeg[i] * sy;
  const typename Pair<T>::type xi = x[t];
  typename Pair<T>::type phi;
  phi.x = w.w[0][0][0] * xi.x + w.w[0][0][1] * xi.y + (w.w[1][0][0] * mx + w.w[1][0][1] * my);
  phi.y = w.w[0][1][0] * xi.x + w.w[0][1][1] * xi.y + (w.w[1][1][0] * mx + w.w[1][1][1] * my);
  if (mode == 0) {
    y[t] = phi;
  } else {
    typename Pair<T>::type o = y[t];
    const T s = mode == 1 ? eta : T(1);
    o.x += s * phi.x;
    o.y += s * phi.y;
    y[t] = o;
  }
}

// y = M x for a real CSR matrix M (n rows) on complex vectors
template <class T>
__global__ void __launch_bounds__(kF2Threads)
    k2_spmv_real(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                 const T* __restrict__ mv, const typename Pair<T>::type* __restrict__ x,
                 typename Pair<T>::type* __restrict__ y, int B) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * B) return;
  const int i = (int)(t / B), b = (int)(t - (size_t)i * B);
  T sx = T(0), sy = T(0);
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const T m = mv[e];
    const typename Pair<T>::type v = x[(size_t)ci[e] * B + b];
    sx += m * v.x;
    sy += m * v.y;
  }
  typename Pair<T>::type o;
  o.x = sx;
  o.y = sy;
  y[t] = o;
}

// e = A_J^{-1} r with the dense inverse (row-major, complex)
template <class T>
__global__ void __launch_bounds__(kF2Threads)
    k2_dense(int n, const typename Pair<T>::type* __restrict__ inv,
             const typename Pair<T>::type* __restrict__ r, typename Pair<T>::type* __restrict__ e,
             int B) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * B) return;
  const int i = (int)(t / B), b = (int)(t - (size_t)i * B);
  T sx = T(0), sy = T(0);
  for (int j = 0; j < n; ++j) {
    const typename Pair<T>::type a = inv[(size_t)i * n + j];
    const typename Pair<T>::type v = r[(size_t)j * B + b];
    sx += a.x * v.x - a.y * v.y;
    sy += a.x * v.y + a.y * v.x;
  }
  typename Pair<T>::type o;
  o.x = sx;
  o.y = sy;
  e[t] = o;
}

dim3 grid_of(size_t work) { return dim3((unsigned)((work + kF2Threads - 1) / kF2Threads)); }

}  // namespace

struct mg2_ctx {
  int J = 0, prec = 64, maxB = 1;
  struct Lev {
    int n = 0, nnz = 0, nnzP = 0;
    int *rp = nullptr, *ci = nullptr;        // A (complex values in av)
    void *av = nullptr, *dinv = nullptr;     // Pair<T>
    void* invdeg = nullptr;                  // T
    int *prp = nullptr, *pci = nullptr;      // P: n x n_next
    void* pv = nullptr;                      // T
    int *trp = nullptr, *tci = nullptr;      // P^T: n_next x n
    void* tv = nullptr;                      // T
    void *f = nullptr, *u = nullptr, *t = nullptr, *t2 = nullptr;  // Pair<T>, n * maxB
  };
  std::vector<Lev> lev;
  void* cinv = nullptr;  // Pair<T>, n_J x n_J
  std::vector<double> theta, eta, WB, WR, WP;
  int nu_pre = 1, nu_post = 1;
  std::vector<void*> owned;
  cudaStream_t cap = nullptr;  // capture stream
  std::map<std::tuple<const void*, const void*, int>, cudaGraphExec_t> graphs;
  void drop_graphs() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
  }
};

namespace {

mg_status fail(const std::string& m, mg_status s = MG_ERR_INVALID) {
  return mgi::set_global_error(s, m);
}

template <class X>
bool upload(mg2_ctx* c, void** dst, const X* src, size_t count) {
  if (count == 0) {
    *dst = nullptr;
    return true;
  }
  if (cudaMalloc(dst, count * sizeof(X)) != cudaSuccess) return false;
  c->owned.push_back(*dst);
  return cudaMemcpy(*dst, src, count * sizeof(X), cudaMemcpyHostToDevice) == cudaSuccess;
}

// Transpose of a CSR matrix (rows x cols) by counting sort: columns of each
// output row in ascending order.
void transpose(int rows, int cols, const int32_t* rp, const int32_t* ci, const double* v,
               std::vector<int>& trp, std::vector<int>& tci, std::vector<double>& tv) {
  const int nnz = rp[rows];
  trp.assign(cols + 1, 0);
  for (int e = 0; e < nnz; ++e) trp[ci[e] + 1]++;
  for (int j = 0; j < cols; ++j) trp[j + 1] += trp[j];
  tci.resize(nnz);
  tv.resize(nnz);
  std::vector<int> pos(trp.begin(), trp.end() - 1);
  for (int i = 0; i < rows; ++i)
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const int k = pos[ci[e]]++;
      tci[k] = i;
      tv[k] = v[e];
    }
}

// Dense complex inverse by Gauss-Jordan elimination with partial pivoting.
bool invert(int n, std::vector<std::complex<double>>& a, std::vector<std::complex<double>>& inv) {
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::abs(a[(size_t)i * n + k]) > std::abs(a[(size_t)p * n + k])) p = i;
    if (!(std::abs(a[(size_t)p * n + k]) > 0.0)) return false;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        std::swap(a[(size_t)p * n + j], a[(size_t)k * n + j]);
        std::swap(inv[(size_t)p * n + j], inv[(size_t)k * n + j]);
      }
    const std::complex<double> d = 1.0 / a[(size_t)k * n + k];
    for (int j = 0; j < n; ++j) {
      a[(size_t)k * n + j] *= d;
      inv[(size_t)k * n + j] *= d;
    }
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const std::complex<double> m = a[(size_t)i * n + k];
      if (m == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        a[(size_t)i * n + j] -= m * a[(size_t)k * n + j];
        inv[(size_t)i * n + j] -= m * inv[(size_t)k * n + j];
      }
    }
  }
  return true;
}

template <class T>
mg_status setup_typed(mg2_ctx* c, const mg2_level* L) {
  using P2 = typename Pair<T>::type;
  const int J = c->J;
  for (int l = 0; l < J; ++l) {
    const mg2_level& s = L[l];
    mg2_ctx::Lev& d = c->lev[l];
    d.n = s.n;
    d.nnz = s.A_indptr[s.n];
    std::vector<P2> av(d.nnz), dinv(d.n);
    std::vector<T> invdeg(d.n);
    for (int i = 0; i < d.n; ++i) {
      std::complex<double> diag = 0.0;
      for (int e = s.A_indptr[i]; e < s.A_indptr[i + 1]; ++e) {
        av[e].x = (T)s.A_vals[2 * e];
        av[e].y = (T)s.A_vals[2 * e + 1];
        if (s.A_indices[e] == i) diag += std::complex<double>(s.A_vals[2 * e], s.A_vals[2 * e + 1]);
      }
      if (!(std::abs(diag) > 0.0)) return fail("mg2_setup: zero diagonal");
      const std::complex<double> di = 1.0 / diag;
      dinv[i].x = (T)di.real();
      dinv[i].y = (T)di.imag();
      invdeg[i] = (T)s.inv_deg[i];
    }
    std::vector<int> rp(s.A_indptr, s.A_indptr + d.n + 1), ci(s.A_indices, s.A_indices + d.nnz);
    if (!upload(c, (void**)&d.rp, rp.data(), rp.size()) ||
        !upload(c, (void**)&d.ci, ci.data(), ci.size()) || !upload(c, &d.av, av.data(), av.size()) ||
        !upload(c, &d.dinv, dinv.data(), dinv.size()) ||
        !upload(c, &d.invdeg, invdeg.data(), invdeg.size()))
      return fail("mg2_setup: device allocation or copy failed", MG_ERR_CUDA);
    const size_t vec = (size_t)d.n * c->maxB;
    for (void** v : {&d.f, &d.u, &d.t, &d.t2}) {
      if (cudaMalloc(v, vec * sizeof(P2)) != cudaSuccess)
        return fail("mg2_setup: device allocation failed", MG_ERR_OOM);
      c->owned.push_back(*v);
    }
    if (l < J - 1) {
      const int nc = L[l + 1].n;
      d.nnzP = s.P_indptr[d.n];
      std::vector<int> prp(s.P_indptr, s.P_indptr + d.n + 1), pci(s.P_indices, s.P_indices + d.nnzP);
      std::vector<T> pv(d.nnzP);
      for (int e = 0; e < d.nnzP; ++e) pv[e] = (T)s.P_vals[e];
      std::vector<int> trp, tci;
      std::vector<double> tvd;
      transpose(d.n, nc, s.P_indptr, s.P_indices, s.P_vals, trp, tci, tvd);
      std::vector<T> tv(tvd.begin(), tvd.end());
      if (!upload(c, (void**)&d.prp, prp.data(), prp.size()) ||
          !upload(c, (void**)&d.pci, pci.data(), pci.size()) ||
          !upload(c, &d.pv, pv.data(), pv.size()) ||
          !upload(c, (void**)&d.trp, trp.data(), trp.size()) ||
          !upload(c, (void**)&d.tci, tci.data(), tci.size()) ||
          !upload(c, &d.tv, tv.data(), tv.size()))
        return fail("mg2_setup: device allocation or copy failed", MG_ERR_CUDA);
    }
  }
  // the coarsest operator, inverted in FP64 on the host
  const mg2_level& s = L[J - 1];
  const int n = s.n;
  std::vector<std::complex<double>> a((size_t)n * n, 0.0), inv;
  for (int i = 0; i < n; ++i)
    for (int e = s.A_indptr[i]; e < s.A_indptr[i + 1]; ++e)
      a[(size_t)i * n + s.A_indices[e]] += std::complex<double>(s.A_vals[2 * e], s.A_vals[2 * e + 1]);
  if (!invert(n, a, inv)) return fail("mg2_setup: coarsest operator is singular", MG_ERR_NOT_SPD);
  std::vector<P2> ci(inv.size());
  for (size_t k = 0; k < inv.size(); ++k) {
    ci[k].x = (T)inv[k].real();
    ci[k].y = (T)inv[k].imag();
  }
  if (!upload(c, &c->cinv, ci.data(), ci.size()))
    return fail("mg2_setup: device allocation or copy failed", MG_ERR_CUDA);
  return MG_OK;
}

template <class T>
Conv2<T> conv_of(const std::vector<double>& W, int l) {
  Conv2<T> w;
  for (int m = 0; m < 2; ++m)
    for (int p = 0; p < 2; ++p)
      for (int q = 0; q < 2; ++q) w.w[m][p][q] = (T)W[(size_t)l * 8 + m * 4 + p * 2 + q];
  return w;
}

// Algorithm 2 on level l with two-feature convolutions.
template <class T>
void cycle(mg2_ctx* c, int l, const typename Pair<T>::type* f, typename Pair<T>::type* u, int B,
           cudaStream_t s) {
  using P2 = typename Pair<T>::type;
  mg2_ctx::Lev& L = c->lev[l];
  const dim3 g = grid_of((size_t)L.n * B);
  if (l == c->J - 1) {
    k2_dense<T><<<g, kF2Threads, 0, s>>>(L.n, (const P2*)c->cinv, f, u, B);
    return;
  }
  const T theta = (T)c->theta[l], eta = (T)c->eta[l];
  const Conv2<T> wb = conv_of<T>(c->WB, l), wr = conv_of<T>(c->WR, l), wp = conv_of<T>(c->WP, l);
  P2* t = (P2*)L.t;
  P2* t2 = (P2*)L.t2;
  auto smooth = [&](int nu) {
    for (int k = 0; k < nu; ++k) {
      k2_residual<T><<<g, kF2Threads, 0, s>>>(L.n, L.rp, L.ci, (const P2*)L.av, f, u, t, B,
                                              (const P2*)L.dinv, theta, 1, 0);
      k2_conv<T><<<g, kF2Threads, 0, s>>>(L.n, L.rp, L.ci, (const T*)L.invdeg, t, u, B, wb, eta, 1);
    }
  };
  smooth(c->nu_pre);
  k2_residual<T><<<g, kF2Threads, 0, s>>>(L.n, L.rp, L.ci, (const P2*)L.av, f, u, t, B,
                                          (const P2*)L.dinv, theta, 0, 0);
  k2_conv<T><<<g, kF2Threads, 0, s>>>(L.n, L.rp, L.ci, (const T*)L.invdeg, t, t2, B, wr, T(1), 0);
  mg2_ctx::Lev& C = c->lev[l + 1];
  const dim3 gc = grid_of((size_t)C.n * B);
  k2_spmv_real<T><<<gc, kF2Threads, 0, s>>>(C.n, L.trp, L.tci, (const T*)L.tv, t2, (P2*)C.f, B);
  cudaMemsetAsync(C.u, 0, (size_t)C.n * B * sizeof(P2), s);
  cycle<T>(c, l + 1, (const P2*)C.f, (P2*)C.u, B, s);
  k2_spmv_real<T><<<g, kF2Threads, 0, s>>>(L.n, L.prp, L.pci, (const T*)L.pv, (const P2*)C.u, t, B);
  k2_conv<T><<<g, kF2Threads, 0, s>>>(L.n, L.rp, L.ci, (const T*)L.invdeg, t, u, B, wp, T(1), 2);
  smooth(c->nu_post);
}

}  // namespace

extern "C" mg_status mg2_setup(mg2_ctx** out, int32_t J, const mg2_level* levels,
                               int32_t max_batch, int32_t precision) {
  if (!out) return fail("mg2_setup: out is NULL");
  *out = nullptr;
  if (J < 1 || J > 32 || !levels || max_batch < 1 || (precision != 32 && precision != 64))
    return fail("mg2_setup: bad arguments");
  for (int l = 0; l < J; ++l) {
    const mg2_level& s = levels[l];
    if (s.n < 1 || !s.A_indptr || !s.A_indices || !s.A_vals || !s.inv_deg)
      return fail("mg2_setup: level " + std::to_string(l) + " is incomplete");
    const int nn = l < J - 1 ? levels[l + 1].n : 0;
    if (l < J - 1 && (!s.P_indptr || !s.P_indices || !s.P_vals))
      return fail("mg2_setup: level " + std::to_string(l) + " has no prolongation");
    for (int e = 0; e < s.A_indptr[s.n]; ++e)
      if (s.A_indices[e] < 0 || s.A_indices[e] >= s.n)
        return fail("mg2_setup: column index out of range");
    if (l < J - 1)
      for (int e = 0; e < s.P_indptr[s.n]; ++e)
        if (s.P_indices[e] < 0 || s.P_indices[e] >= nn)
          return fail("mg2_setup: prolongation column out of range");
  }
  if (levels[J - 1].n > 4096) return fail("mg2_setup: coarsest level larger than 4096 rows");
  mg2_ctx* c = new mg2_ctx;
  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return fail("mg2_setup: stream creation failed", MG_ERR_CUDA);
  }
  c->J = J;
  c->prec = precision;
  c->maxB = max_batch;
  c->lev.resize(J);
  c->theta.assign(std::max(J - 1, 0), 2.0 / 3.0);
  c->eta.assign(std::max(J - 1, 0), 1.0);
  for (std::vector<double>* W : {&c->WB, &c->WR, &c->WP}) {
    W->assign((size_t)std::max(J - 1, 0) * 8, 0.0);
    for (int l = 0; l < J - 1; ++l) (*W)[(size_t)l * 8 + 0] = (*W)[(size_t)l * 8 + 3] = 1.0;
  }
  const mg_status st = precision == 64 ? setup_typed<double>(c, levels) : setup_typed<float>(c, levels);
  if (st != MG_OK) {
    mg2_destroy(c);
    return st;
  }
  *out = c;
  return MG_OK;
}

extern "C" mg_status mg2_set_params(mg2_ctx* c, const double* theta, const double* eta,
                                    const double* WB, const double* WR, const double* WP,
                                    int32_t nu_pre, int32_t nu_post) {
  if (!c) return fail("mg2_set_params: ctx is NULL");
  if (!theta || !eta || !WB || !WR || !WP || nu_pre < 0 || nu_post < 0 || nu_pre > 16 ||
      nu_post > 16)
    return fail("mg2_set_params: bad arguments");
  const int m = c->J - 1;
  for (int l = 0; l < m; ++l) {
    if (!std::isfinite(theta[l]) || !std::isfinite(eta[l])) return fail("mg2_set_params: non-finite");
    for (int k = 0; k < 8; ++k)
      if (!std::isfinite(WB[l * 8 + k]) || !std::isfinite(WR[l * 8 + k]) ||
          !std::isfinite(WP[l * 8 + k]))
        return fail("mg2_set_params: non-finite");
  }
  c->theta.assign(theta, theta + m);
  c->eta.assign(eta, eta + m);
  c->WB.assign(WB, WB + (size_t)m * 8);
  c->WR.assign(WR, WR + (size_t)m * 8);
  c->WP.assign(WP, WP + (size_t)m * 8);
  c->nu_pre = nu_pre;
  c->nu_post = nu_post;
  c->drop_graphs();
  return MG_OK;
}

extern "C" mg_status mg2_vcycle(mg2_ctx* c, const void* f, void* u, int32_t nrhs, void* stream) {
  if (!c) return fail("mg2_vcycle: ctx is NULL");
  if (!f || !u || f == u || nrhs < 1 || nrhs > c->maxB) return fail("mg2_vcycle: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const auto key = std::make_tuple(f, (const void*)u, (int)nrhs);
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail(std::string("mg2_vcycle: ") + cudaGetErrorString(e), MG_ERR_CUDA);
    if (c->prec == 64)
      cycle<double>(c, 0, (const double2*)f, (double2*)u, nrhs, c->cap);
    else
      cycle<float>(c, 0, (const float2*)f, (float2*)u, nrhs, c->cap);
    const cudaError_t e1 = cudaGetLastError();
    const cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return fail(std::string("mg2_vcycle: capture: ") +
                      cudaGetErrorString(e1 != cudaSuccess ? e1 : e2),
                  MG_ERR_CUDA);
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e3 = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess)
      return fail(std::string("mg2_vcycle: instantiate: ") + cudaGetErrorString(e3), MG_ERR_CUDA);
    if (c->graphs.size() >= 256) c->drop_graphs();  // bounded cache
    it = c->graphs.emplace(key, exec).first;
  }
  const cudaError_t e = cudaGraphLaunch(it->second, s);
  if (e != cudaSuccess)
    return fail(std::string("mg2_vcycle: ") + cudaGetErrorString(e), MG_ERR_CUDA);
  return MG_OK;
}

extern "C" void mg2_destroy(mg2_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  c->drop_graphs();
  if (c->cap) cudaStreamDestroy(c->cap);
  for (void* p : c->owned)
    if (p) cudaFree(p);
  delete c;
}
