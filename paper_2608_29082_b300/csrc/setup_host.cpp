// Host-side hierarchy construction for nested P1 meshes (FP64, single pass,
// no GPU).  Implements the Galerkin coarsening A_{l+1} = P_l^T A_l P_l with
// P_l the natural inclusion of the coarse finite-element space (Sec. 2.2),
// Dirichlet elimination, and the algebraic graph degree of Sec. 2.1 used by
// the mean aggregation of the SAGEConv (Sec. 3.2).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "mg.h"
#include "mg_internal.h"

namespace {

// vw: doubles per value (1 real, 2 complex with (Re, Im) adjacent)
bool alloc_csr(mg_csr_owned* o, int nr, int nc, long long nnz, int vw = 1) {
  o->n_rows = nr;
  o->n_cols = nc;
  o->nnz = (int32_t)nnz;
  o->rowptr = (int32_t*)std::malloc(sizeof(int32_t) * (size_t)(nr + 1));
  o->col = (int32_t*)std::malloc(sizeof(int32_t) * (size_t)std::max<long long>(nnz, 1));
  o->val = (double*)std::malloc(sizeof(double) * vw * (size_t)std::max<long long>(nnz, 1));
  if (!o->rowptr || !o->col || !o->val) {
    mg_csr_owned_free(o);
    return false;
  }
  return true;
}

bool csr_ok(const mg_csr* A) {
  if (!A || A->n_rows < 0 || A->n_cols < 0 || A->nnz < 0 || !A->rowptr) return false;
  if (A->nnz > 0 && (!A->col || !A->val)) return false;
  if (A->rowptr[0] != 0 || A->rowptr[A->n_rows] != A->nnz) return false;
  for (int i = 0; i < A->n_rows; ++i)
    if (A->rowptr[i + 1] < A->rowptr[i]) return false;
  for (int k = 0; k < A->nnz; ++k)
    if (A->col[k] < 0 || A->col[k] >= A->n_cols) return false;
  return true;
}

// Row-wise sparse accumulator: values for columns touched in the current row.
template <class V>
struct Spa {
  std::vector<V> acc;
  std::vector<int> mark, cols;
  explicit Spa(int n) : acc(n, V(0)), mark(n, -1) {}
  void add(int row, int j, V v) {
    if (mark[j] != row) {
      mark[j] = row;
      acc[j] = V(0);
      cols.push_back(j);
    }
    acc[j] += v;
  }
};

template <class V>
struct Csr {
  int nr = 0, nc = 0;
  std::vector<int> ptr, col;
  std::vector<V> val;
};

// Magnitude used by the drop rule: |a| for real values, the complex modulus
// for complex ones.
inline double mag(double a) { return std::fabs(a); }
inline double mag(const std::complex<double>& a) { return std::abs(a); }

template <class V>
constexpr int value_width() {
  return sizeof(V) / sizeof(double);
}

}  // namespace

extern "C" void mg_csr_owned_free(mg_csr_owned* m) {
  if (!m) return;
  std::free(m->rowptr);
  std::free(m->col);
  std::free(m->val);
  m->rowptr = nullptr;
  m->col = nullptr;
  m->val = nullptr;
  m->n_rows = m->n_cols = m->nnz = 0;
}

namespace {

// P^T A P over all vertices with P from the parent map; values V (real, or
// complex (Re, Im) adjacent: P is real, so both parts go through the same
// sums in the same order as two real products would).
template <class V>
mg_status galerkin_impl(const mg_csr* A, const V* Aval, const int32_t* parent, int32_t nv_c,
                        double drop_tol, mg_csr_owned* out, const char* who) {
  if (!out) return mgi::set_global_error(MG_ERR_INVALID, std::string(who) + ": out is NULL");
  std::memset(out, 0, sizeof(*out));
  if (!csr_ok(A) || A->n_rows != A->n_cols || !parent || nv_c <= 0)
    return mgi::set_global_error(MG_ERR_INVALID,
                                 std::string(who) + ": invalid matrix or parent map");
  const int nf = A->n_rows;
  // P rows from the parent map (natural inclusion).
  std::vector<int> pc(2 * (size_t)nf);
  std::vector<double> pw(2 * (size_t)nf);
  for (int i = 0; i < nf; ++i) {
    int a = parent[2 * i], b = parent[2 * i + 1];
    if (a < 0 || a >= nv_c || b >= nv_c)
      return mgi::set_global_error(MG_ERR_INVALID,
                                   std::string(who) + ": parent index out of range");
    pc[2 * i] = a;
    pc[2 * i + 1] = b;
    pw[2 * i] = b < 0 ? 1.0 : 0.5;
    pw[2 * i + 1] = b < 0 ? 0.0 : 0.5;
  }
  // AP = A P, row by row.
  Csr<V> AP;
  AP.nr = nf;
  AP.nc = nv_c;
  AP.ptr.assign(nf + 1, 0);
  {
    Spa<V> spa(nv_c);
    for (int i = 0; i < nf; ++i) {
      spa.cols.clear();
      for (int k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) {
        int j = A->col[k];
        const V a = Aval[k];
        spa.add(i, pc[2 * j], a * pw[2 * j]);
        if (pc[2 * j + 1] >= 0) spa.add(i, pc[2 * j + 1], a * pw[2 * j + 1]);
      }
      std::sort(spa.cols.begin(), spa.cols.end());
      for (int j : spa.cols) {
        AP.col.push_back(j);
        AP.val.push_back(spa.acc[j]);
      }
      AP.ptr[i + 1] = (int)AP.col.size();
    }
  }
  // P^T as coarse-row lists of (fine row, weight), fine rows ascending.
  std::vector<int> tcount(nv_c + 1, 0);
  for (int i = 0; i < nf; ++i) {
    tcount[pc[2 * i] + 1]++;
    if (pc[2 * i + 1] >= 0) tcount[pc[2 * i + 1] + 1]++;
  }
  for (int I = 0; I < nv_c; ++I) tcount[I + 1] += tcount[I];
  std::vector<int> trow(tcount[nv_c]);
  std::vector<double> tw(tcount[nv_c]);
  {
    std::vector<int> fill(tcount.begin(), tcount.end() - 1);
    for (int i = 0; i < nf; ++i)
      for (int s = 0; s < 2; ++s) {
        int I = pc[2 * i + s];
        if (I < 0) continue;
        trow[fill[I]] = i;
        tw[fill[I]] = pw[2 * i + s];
        fill[I]++;
      }
  }
  // C = P^T (A P).
  Csr<V> C;
  C.nr = C.nc = nv_c;
  C.ptr.assign(nv_c + 1, 0);
  {
    Spa<V> spa(nv_c);
    for (int I = 0; I < nv_c; ++I) {
      spa.cols.clear();
      for (int t = tcount[I]; t < tcount[I + 1]; ++t) {
        int i = trow[t];
        double w = tw[t];
        for (int k = AP.ptr[i]; k < AP.ptr[i + 1]; ++k) spa.add(I, AP.col[k], w * AP.val[k]);
      }
      std::sort(spa.cols.begin(), spa.cols.end());
      for (int j : spa.cols) {
        C.col.push_back(j);
        C.val.push_back(spa.acc[j]);
      }
      C.ptr[I + 1] = (int)C.col.size();
    }
  }
  // Diagonal, then drop round-off off-diagonals.
  std::vector<double> d(nv_c, 0.0);
  for (int I = 0; I < nv_c; ++I)
    for (int k = C.ptr[I]; k < C.ptr[I + 1]; ++k)
      if (C.col[k] == I) d[I] = mag(C.val[k]);
  long long keep = 0;
  std::vector<char> kept(C.col.size(), 0);
  for (int I = 0; I < nv_c; ++I)
    for (int k = C.ptr[I]; k < C.ptr[I + 1]; ++k) {
      int Jc = C.col[k];
      bool ok = Jc == I || mag(C.val[k]) > drop_tol * std::max(d[I], d[Jc]);
      kept[k] = ok;
      keep += ok;
    }
  if (!alloc_csr(out, nv_c, nv_c, keep, value_width<V>()))
    return mgi::set_global_error(MG_ERR_OOM, std::string(who) + ": host allocation failed");
  V* oval = reinterpret_cast<V*>(out->val);
  long long w = 0;
  out->rowptr[0] = 0;
  for (int I = 0; I < nv_c; ++I) {
    for (int k = C.ptr[I]; k < C.ptr[I + 1]; ++k)
      if (kept[k]) {
        out->col[w] = C.col[k];
        oval[w] = C.val[k];
        ++w;
      }
    out->rowptr[I + 1] = (int32_t)w;
  }
  return MG_OK;
}

// Dirichlet elimination and graph degrees; values V as galerkin_impl.
template <class V>
mg_status eliminate_impl(const mg_csr* A, const V* Aval, const uint8_t* bnd, double drop_tol,
                         mg_csr_owned* out, double* inv_deg, const char* who) {
  if (!out) return mgi::set_global_error(MG_ERR_INVALID, std::string(who) + ": out is NULL");
  std::memset(out, 0, sizeof(*out));
  if (!csr_ok(A) || A->n_rows != A->n_cols || !bnd || !inv_deg)
    return mgi::set_global_error(MG_ERR_INVALID, std::string(who) + ": invalid arguments");
  const int nv = A->n_rows;
  std::vector<int> id(nv, -1);
  int ni = 0;
  for (int i = 0; i < nv; ++i)
    if (!bnd[i]) id[i] = ni++;
  std::vector<double> d(nv, 0.0);
  for (int i = 0; i < nv; ++i)
    for (int k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k)
      if (A->col[k] == i) d[i] = mag(Aval[k]);
  auto edge = [&](int i, int k) {
    int j = A->col[k];
    return j != i && mag(Aval[k]) > drop_tol * std::max(d[i], d[j]);
  };
  long long nnz = 0;
  for (int i = 0; i < nv; ++i) {
    if (id[i] < 0) continue;
    int deg = 0;
    for (int k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) {
      bool e = edge(i, k);
      deg += e;
      int j = A->col[k];
      if (id[j] >= 0 && (j == i || e)) ++nnz;
    }
    if (deg == 0)
      return mgi::set_global_error(MG_ERR_INVALID, std::string(who) + ": isolated vertex");
    inv_deg[id[i]] = 1.0 / (double)deg;
  }
  if (!alloc_csr(out, ni, ni, nnz, value_width<V>()))
    return mgi::set_global_error(MG_ERR_OOM, std::string(who) + ": host allocation failed");
  V* oval = reinterpret_cast<V*>(out->val);
  long long w = 0;
  out->rowptr[0] = 0;
  for (int i = 0; i < nv; ++i) {
    if (id[i] < 0) continue;
    for (int k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) {
      int j = A->col[k];
      if (id[j] >= 0 && (j == i || edge(i, k))) {
        out->col[w] = id[j];
        oval[w] = Aval[k];
        ++w;
      }
    }
    out->rowptr[id[i] + 1] = (int32_t)w;
  }
  return MG_OK;
}

}  // namespace

extern "C" mg_status mg_galerkin(const mg_csr* A, const int32_t* parent, int32_t nv_c,
                                 double drop_tol, mg_csr_owned* out) {
  return galerkin_impl<double>(A, A ? A->val : nullptr, parent, nv_c, drop_tol, out,
                               "mg_galerkin");
}

extern "C" mg_status mg_galerkin_complex(const mg_csr* A, const int32_t* parent, int32_t nv_c,
                                         double drop_tol, mg_csr_owned* out) {
  return galerkin_impl<std::complex<double>>(
      A, A ? reinterpret_cast<const std::complex<double>*>(A->val) : nullptr, parent, nv_c,
      drop_tol, out, "mg_galerkin_complex");
}

extern "C" mg_status mg_eliminate(const mg_csr* A, const uint8_t* bnd, double drop_tol,
                                  mg_csr_owned* out, double* inv_deg) {
  return eliminate_impl<double>(A, A ? A->val : nullptr, bnd, drop_tol, out, inv_deg,
                                "mg_eliminate");
}

extern "C" mg_status mg_eliminate_complex(const mg_csr* A, const uint8_t* bnd, double drop_tol,
                                          mg_csr_owned* out, double* inv_deg) {
  return eliminate_impl<std::complex<double>>(
      A, A ? reinterpret_cast<const std::complex<double>*>(A->val) : nullptr, bnd, drop_tol, out,
      inv_deg, "mg_eliminate_complex");
}

extern "C" mg_status mg_prolongation(const int32_t* parent, int32_t nv_f, const uint8_t* bnd_f,
                                     int32_t nv_c, const uint8_t* bnd_c, mg_csr_owned* out) {
  if (!out) return mgi::set_global_error(MG_ERR_INVALID, "mg_prolongation: out is NULL");
  std::memset(out, 0, sizeof(*out));
  if (!parent || !bnd_f || !bnd_c || nv_f <= 0 || nv_c <= 0)
    return mgi::set_global_error(MG_ERR_INVALID, "mg_prolongation: invalid arguments");
  std::vector<int> idc(nv_c, -1);
  int nic = 0;
  for (int I = 0; I < nv_c; ++I)
    if (!bnd_c[I]) idc[I] = nic++;
  int nif = 0;
  long long nnz = 0;
  for (int i = 0; i < nv_f; ++i) {
    int a = parent[2 * i], b = parent[2 * i + 1];
    if (a < 0 || a >= nv_c || b >= nv_c)
      return mgi::set_global_error(MG_ERR_INVALID, "mg_prolongation: parent out of range");
    if (bnd_f[i]) continue;
    ++nif;
    nnz += (idc[a] >= 0) + (b >= 0 && idc[b] >= 0);
  }
  if (!alloc_csr(out, nif, nic, nnz))
    return mgi::set_global_error(MG_ERR_OOM, "mg_prolongation: host allocation failed");
  long long w = 0;
  int r = 0;
  out->rowptr[0] = 0;
  for (int i = 0; i < nv_f; ++i) {
    if (bnd_f[i]) continue;
    int a = parent[2 * i], b = parent[2 * i + 1];
    double wt = b < 0 ? 1.0 : 0.5;
    int ia = idc[a], ib = b >= 0 ? idc[b] : -1;
    if (ia >= 0 && ib >= 0 && ib < ia) std::swap(ia, ib);
    if (ia >= 0) { out->col[w] = ia; out->val[w] = wt; ++w; }
    if (ib >= 0) { out->col[w] = ib; out->val[w] = wt; ++w; }
    out->rowptr[++r] = (int32_t)w;
  }
  return MG_OK;
}
