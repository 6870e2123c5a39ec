// Device kernels of the learnable V-cycle (Algorithm 2) for sm_103a.
//
// Data layout per level (n rows, B right-hand sides):
//   vectors      X[n][B], right-hand-side index fastest
//   off-diagonal SELL-32: rows grouped in slices of 32; entry k of row i at
//                sl_ptr[i/32] + 32*k + i%32 (column-major inside a slice, so a
//                warp's loads of one k are contiguous); col = -1 pads a slice
//   diag, dinv   A_ii and 1/A_ii
//   invdeg       1/|N(i)|, the mean of the SAGEConv (Sec. 3.2)
//   p_idx, p_w   prolongation rows, [2][n] (second parent -1 when absent)
//   r_idx, r_w   restriction R = P^T as coarse-row gather lists, [KR][nc]
//
// The off-diagonal pattern of A is the convolution graph (Sec. 2.1), so the
// same column array serves the residual and the mean aggregation.
// Arithmetic uses explicit fma() so that every right-hand side is computed in
// the same order whatever the batch size: results do not depend on B.
//
// Every step is a per-element device function (one (row, rhs) pair) used by
// two launch forms: a grid kernel per step for large levels, and k_tail,
// one thread block that runs all small levels of a cycle with block
// barriers between the steps.  Every kernel starts with griddepcontrol.wait
// followed by griddepcontrol.launch_dependents: with programmatic dependent
// launch the next kernel of a captured cycle is scheduled while this one
// runs, and its own griddepcontrol.wait holds it until this grid has
// completed and its memory is visible.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mgk {

// Index checks of the debug build (-DMG_BOUNDS_CHECK).  idx_ok(v, n, site)
// returns v when 0 <= v < n, else -1 (the entry is then treated as absent,
// so the access is skipped) and records the first violation in
// g_bounds_error as ((site << 32) | (uint32_t)v) + 1; -1 passes unchanged
// (padding).  Sites: 1 SELL column, 2 prolongation parent, 3 restriction
// child, 4 halo row, 5 halo local column.  Without the macro idx_ok is v.
#ifdef MG_BOUNDS_CHECK
__device__ unsigned long long g_bounds_error = 0;
__device__ __forceinline__ int idx_ok(int v, int n, int site) {
  if (v == -1 || (v >= 0 && v < n)) return v;
  atomicCAS(&g_bounds_error, 0ull,
            (((unsigned long long)site << 32) | (unsigned long long)(unsigned)v) + 1ull);
  return -1;
}
#else
__device__ __forceinline__ int idx_ok(int v, int, int) { return v; }
#endif

constexpr int kThreads = 256;
constexpr int kSlice = 32;
constexpr int kMaxLevels = 16;
constexpr int kTailThreads = 1024;
// The small-levels block (k_tail): 512 threads, so that each level's view
// (offsets, sizes, array pointers) stays in registers across its steps'
// barriers (up to 128 registers per thread; at 1024 threads the 64-register
// limit spilled them, and re-reading them from shared memory after every
// barrier put those loads on each step's dependent chain: 41 against 33 us
// per 513^2 cycle).
constexpr int kTailBlock = 512;

// Parameter block per level, in the order used everywhere:
// theta, eta, wB1, wB2, wR1, wR2, wP1, wP2.
enum { P_THETA = 0, P_ETA, P_WB1, P_WB2, P_WR1, P_WR2, P_WP1, P_WP2, P_COUNT };

constexpr int kMaxDia = 8;
constexpr int kMaxKR = 8;  // restriction children handled with a fixed trip count

// Level view.  Off-diagonals are stored either as SELL-32 (sl_ptr, col, val)
// or, when every off-diagonal of the level lies on at most kMaxDia diagonals
// (structured meshes), as DIA: ndia > 0, offsets doff[k] in ascending order
// and values dval[k][n] (zero where row i has no entry on diagonal k).  The
// graph neighbours of i are exactly its nonzero off-diagonals in either form,
// visited in ascending column order, so both forms give the same arithmetic.
// ld and ldc are the row strides of the [k][.] arrays (dval, p_idx, p_w with
// ld; r_idx, r_w with ldc): n and nc, except in a view of the leading rows of
// a stacked level, where they stay those of the whole level.
template <class T>
struct LV {
  int n, nc, KR;
  int ld, ldc;
  int ndia;
  int doff[kMaxDia];
  const T* __restrict__ dval;
  const int* __restrict__ sl_ptr;
  const int* __restrict__ col;
  const T* __restrict__ val;
  const T* __restrict__ diag;
  const T* __restrict__ dinv;
  const T* __restrict__ invdeg;
  const int* __restrict__ p_idx;
  const T* __restrict__ p_w;
  const int* __restrict__ r_idx;
  const T* __restrict__ r_w;
  // DIA levels: bit k of nbm[i] is set iff off-diagonal k of row i is
  // nonzero (in T), the neighbour test of the mean aggregation, so that
  // the mean-only steps read one byte per row instead of the ndia values;
  // NULL: the test reads the values
  const unsigned char* __restrict__ nbm;
};

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch() { asm volatile("griddepcontrol.launch_dependents;"); }

// (row, rhs) of a flat index t into X[n][B]; n * B < 2^31 is checked at set-up.
__device__ __forceinline__ void split_rb(size_t t, int B, int& i, int& b) {
  if (B == 1) {
    i = (int)t;
    b = 0;
  } else {
    const unsigned tt = (unsigned)t;
    i = (int)(tt / (unsigned)B);
    b = (int)(tt - (unsigned)i * (unsigned)B);
  }
}

// ldexp out of line: a call is never evaluated speculatively, so the FP64
// arithmetic of its special cases stays off the common path of scale2.
__device__ __noinline__ double ldexp_rare(double x, int e) { return ldexp(x, e); }

// x * 2^e.  For -1022 <= e <= 1023, 2^e is a normal binary64 number (biased
// exponent e + 1023, zero fraction), so one multiply gives the exact scaled
// value, rounded once if it is subnormal: bitwise what ldexp returns, without
// ldexp's FP64 special-case arithmetic (B300's FP64 pipe is narrow).  Other e
// go through ldexp.
__device__ __forceinline__ double scale2(double x, int e) {
  if (e >= -1022 && e <= 1023) return x * __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp_rare(x, e);
}

__device__ __forceinline__ int slice_begin(const int* sl_ptr, int i) {
  return sl_ptr[i >> 5] + (i & 31);
}

// Read-only operator data is fetched towards L1 before griddepcontrol.wait:
// it never depends on the preceding kernel (only vectors do), so its latency
// overlaps that kernel's drain.  These are hints; the values are loaded
// again where they are used.
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Row i's off-diagonals (DIA values, or the SELL slice pointer), diagonal,
// its inverse and 1/deg.
template <class T>
__device__ __forceinline__ void prefetch_row(const LV<T>& L, int i) {
  if (L.ndia > 0) {
#pragma unroll
    for (int k = 0; k < kMaxDia; ++k)
      if (k < L.ndia) prefetch_l1(L.dval + (size_t)k * L.ld + i);
  } else {
    prefetch_l1(L.sl_ptr + (i >> 5));
  }
  prefetch_l1(L.diag + i);
  prefetch_l1(L.dinv + i);
  prefetch_l1(L.invdeg + i);
}

// What a mean-only step reads of row i: its neighbour mask (DIA values
// without one, or the SELL slice pointer) and 1/deg.
template <class T>
__device__ __forceinline__ void prefetch_mean(const LV<T>& L, int i) {
  if (L.ndia > 0) {
    if (L.nbm) {
      prefetch_l1(L.nbm + i);
    } else {
#pragma unroll
      for (int k = 0; k < kMaxDia; ++k)
        if (k < L.ndia) prefetch_l1(L.dval + (size_t)k * L.ld + i);
    }
  } else {
    prefetch_l1(L.sl_ptr + (i >> 5));
  }
  prefetch_l1(L.invdeg + i);
}

// Fine row i's prolongation entries.
template <class T>
__device__ __forceinline__ void prefetch_p(const LV<T>& L, int i) {
  prefetch_l1(L.p_idx + i);
  prefetch_l1(L.p_idx + (size_t)L.ld + i);
  prefetch_l1(L.p_w + i);
  prefetch_l1(L.p_w + (size_t)L.ld + i);
}

// Coarse row I's restriction gather list.
template <class T>
__device__ __forceinline__ void prefetch_r(const LV<T>& L, int I) {
  for (int k = 0; k < L.KR && k < kMaxKR; ++k) {
    prefetch_l1(L.r_idx + (size_t)k * L.ldc + I);
    prefetch_l1(L.r_w + (size_t)k * L.ldc + I);
  }
}

// Row of flat index t into X[n][B].
__device__ __forceinline__ int row_of(size_t t, int B) {
  return B == 1 ? (int)t : (int)((unsigned)t / (unsigned)B);
}

// Calls fn(c, a_ic, is_neighbour) for the off-diagonals of row i in ascending
// column order.  DIA: every diagonal is visited; absent entries have a_ic = 0,
// is_neighbour = false and a clamped in-range c, so the value and the
// neighbour loads of a row are independent of each other.  SELL: a loop
// over the row's slice entries; with kPreload and a slice at most kMaxDia
// wide (every mesh here), all column indices (and, with kVal, values) are
// loaded before the first call, so the neighbour loads inside fn do not
// wait on one another's index loads.  kPreload is used by the multi-rhs
// kernels, where it is measured faster; it costs registers that the
// one-value-per-thread kernels (also used on DIA levels) cannot spare.
// kVal = false: fn ignores a_ic (mean aggregation), SELL values are not read.
template <class T, bool kVal = true, bool kPreload = false, class F>
__device__ __forceinline__ void for_nb(const LV<T>& L, int i, F&& fn) {
  if (L.ndia > 0) {
    if (!kVal && L.nbm) {  // the neighbour test from the row's mask
      const unsigned msk = L.nbm[i];
#pragma unroll
      for (int k = 0; k < kMaxDia; ++k) {
        if (k < L.ndia) {
          const int c = min(max(i + L.doff[k], 0), L.n - 1);
          fn(c, T(0), ((msk >> k) & 1u) != 0u);
        }
      }
      return;
    }
#pragma unroll
    for (int k = 0; k < kMaxDia; ++k) {
      if (k < L.ndia) {
        const T v = L.dval[(size_t)k * L.ld + i];
        const int c = min(max(i + L.doff[k], 0), L.n - 1);
        fn(c, v, v != T(0));
      }
    }
  } else {
    const int s0 = L.sl_ptr[i >> 5];
    const int end = L.sl_ptr[(i >> 5) + 1];
    const int beg = s0 + (i & 31);
    if (kPreload && end - s0 <= kMaxDia * kSlice) {
      int cs[kMaxDia];
      T vs[kMaxDia];
#pragma unroll
      for (int k = 0; k < kMaxDia; ++k) {
        const int e = beg + k * kSlice;
        cs[k] = e < end ? idx_ok(L.col[e], L.n, 1) : -1;
        vs[k] = kVal && e < end ? L.val[e] : T(0);
      }
#pragma unroll
      for (int k = 0; k < kMaxDia; ++k)
        if (cs[k] >= 0) fn(cs[k], vs[k], true);
    } else {
      for (int e = beg; e < end; e += kSlice) {
        const int c = idx_ok(L.col[e], L.n, 1);
        if (c >= 0) fn(c, kVal ? L.val[e] : T(0), true);
      }
    }
  }
}

// Neighbour bits of DIA row i (bit k: off-diagonal k nonzero): the
// level's mask, or the test on the values.
template <class T>
__device__ __forceinline__ unsigned nb_mask(const LV<T>& L, int i) {
  if (L.nbm) return L.nbm[i];
  unsigned m = 0;
#pragma unroll
  for (int k = 0; k < kMaxDia; ++k)
    if (k < L.ndia && L.dval[(size_t)k * L.ld + i] != T(0)) m |= 1u << k;
  return m;
}

// sum_{j != i} a_ij x_j
template <class T>
__device__ __forceinline__ T row_ax(const LV<T>& L, int i, const T* __restrict__ x, int B, int b) {
  T a_acc = T(0);
  for_nb(L, i, [&](int c, T v, bool) { a_acc = fma(v, x[(size_t)c * B + b], a_acc); });
  return a_acc;
}

// sum_{j in N(i)} x_j
template <class T>
__device__ __forceinline__ T row_sum(const LV<T>& L, int i, const T* __restrict__ x, int B, int b) {
  T s_acc = T(0);
  for_nb<T, false>(L, i, [&](int c, T, bool nb) {
    const T xv = x[(size_t)c * B + b];
    s_acc += nb ? xv : T(0);
  });
  return s_acc;
}

template <class T>
__device__ __forceinline__ T prolong_at(const LV<T>& L, int j, const T* __restrict__ ec, int B,
                                        int b) {
  const int a = idx_ok(L.p_idx[j], L.nc, 2), c = idx_ok(L.p_idx[(size_t)L.ld + j], L.nc, 2);
  T v = T(0);
  if (a >= 0) v = L.p_w[j] * ec[(size_t)a * B + b];
  if (c >= 0) v = fma(L.p_w[(size_t)L.ld + j], ec[(size_t)c * B + b], v);
  return v;
}

// ------------------------------------------------------ element steps ----
// t indexes (row, rhs) = (t / B, t % B) of the level the step writes.

// out = [theta dinv] (f - A u).  u_zero: u is taken as 0 and not read.
template <class T>
__device__ __forceinline__ void residual_el(const LV<T>& L, const T* __restrict__ f,
                                            const T* __restrict__ u, T* __restrict__ out, int B,
                                            const T* __restrict__ prm, int scale, int u_zero,
                                            size_t t) {
  int i, b;
  split_rb(t, B, i, b);
  T r = f[t];
  if (!u_zero) {
    const T ax = row_ax(L, i, u, B, b);
    r = fma(-L.diag[i], u[t], r) - ax;
  }
  if (scale) r = prm[P_THETA] * (r * L.dinv[i]);
  out[t] = r;
}

// u <- u + eta * (wB1 * x + wB2 * mean_{N(i)} x)   (Phi_B applied to delta = x)
template <class T>
__device__ __forceinline__ void conv_update_el(const LV<T>& L, const T* __restrict__ x,
                                               T* __restrict__ u, int B, const T* __restrict__ prm,
                                               int u_zero, size_t t) {
  int i, b;
  split_rb(t, B, i, b);
  const T s = row_sum(L, i, x, B, b);
  const T phi = fma(prm[P_WB1], x[t], prm[P_WB2] * (L.invdeg[i] * s));
  const T u0 = u_zero ? T(0) : u[t];
  u[t] = fma(prm[P_ETA], phi, u0);
}

// Smoothing step with Phi_B = w1 I (w2 = 0) in one pass; Jacobi needs the
// old iterate everywhere, so the result goes to a second buffer.
// uout = uin + eta * w1 * theta * dinv * (f - A uin)
template <class T>
__device__ __forceinline__ void jacobi_el(const LV<T>& L, const T* __restrict__ f,
                                          const T* __restrict__ uin, T* __restrict__ uout, int B,
                                          const T* __restrict__ prm, int u_zero, size_t t) {
  int i, b;
  split_rb(t, B, i, b);
  T r = f[t];
  T u0 = T(0);
  if (!u_zero) {
    u0 = uin[t];
    const T ax = row_ax(L, i, uin, B, b);
    r = fma(-L.diag[i], u0, r) - ax;
  }
  const T delta = prm[P_THETA] * (r * L.dinv[i]);
  uout[t] = fma(prm[P_ETA], prm[P_WB1] * delta, u0);
}

// fc_I = sum_{i in children(I)} P_iI * (wR1 r_i + wR2 mean_{N(i)} r); t over nc*B
template <class T>
__device__ __forceinline__ void restrict_el(const LV<T>& L, const T* __restrict__ r,
                                            T* __restrict__ fc, int B, const T* __restrict__ prm,
                                            int conv, size_t t) {
  int I, b;
  split_rb(t, B, I, b);
  const T w1 = prm[P_WR1], w2 = prm[P_WR2];
  T acc = T(0);
  if (L.KR <= kMaxKR) {
    // fixed trip count, no early exit: every child's loads issue together
    int idx[kMaxKR];
    T wk[kMaxKR];
#pragma unroll
    for (int k = 0; k < kMaxKR; ++k) {
      idx[k] = k < L.KR ? idx_ok(L.r_idx[(size_t)k * L.ldc + I], L.n, 3) : -1;
      wk[k] = k < L.KR ? L.r_w[(size_t)k * L.ldc + I] : T(0);
    }
#pragma unroll
    for (int k = 0; k < kMaxKR; ++k) {
      if (idx[k] >= 0) {
        const int i = idx[k];
        T phi = w1 * r[(size_t)i * B + b];
        if (conv) phi = fma(w2, L.invdeg[i] * row_sum(L, i, r, B, b), phi);
        acc = fma(wk[k], phi, acc);
      }
    }
  } else {
    for (int k = 0; k < L.KR; ++k) {
      const int i = idx_ok(L.r_idx[(size_t)k * L.ldc + I], L.n, 3);
      if (i < 0) break;
      T phi = w1 * r[(size_t)i * B + b];
      if (conv) phi = fma(w2, L.invdeg[i] * row_sum(L, i, r, B, b), phi);
      acc = fma(L.r_w[(size_t)k * L.ldc + I], phi, acc);
    }
  }
  fc[t] = acc;
}

// u_i = uin_i + wP1 (P ec)_i + wP2 mean_{N(i)} (P ec)   (uin may equal u)
template <class T>
__device__ __forceinline__ void prolong_el(const LV<T>& L, const T* __restrict__ ec, const T* uin,
                                           T* u, int B, const T* __restrict__ prm, int conv,
                                           size_t t) {
  int i, b;
  split_rb(t, B, i, b);
  T phi = prm[P_WP1] * prolong_at(L, i, ec, B, b);
  if (conv) {
    T s = T(0);
    for_nb<T, false>(L, i, [&](int c, T, bool nb) {
      const T pv = prolong_at(L, c, ec, B, b);
      s += nb ? pv : T(0);
    });
    phi = fma(prm[P_WP2], L.invdeg[i] * s, phi);
  }
  u[t] = uin[t] + phi;
}

// Split forms of the convolution transfers: the fused steps above evaluate
// the convolution of every child (restriction) or neighbour (prolongation)
// inside one thread; these evaluate it once per fine row in its own pass.
// Values and summation order are those of restrict_el / prolong_el.

// phi_i = wR1 r_i + wR2 mean_{N(i)} r   (fine rows)
template <class T>
__device__ __forceinline__ void conv_r_el(const LV<T>& L, const T* __restrict__ r,
                                          T* __restrict__ phi, int B, const T* __restrict__ prm,
                                          size_t t) {
  int i, b;
  split_rb(t, B, i, b);
  T p = prm[P_WR1] * r[t];
  p = fma(prm[P_WR2], L.invdeg[i] * row_sum(L, i, r, B, b), p);
  phi[t] = p;
}

// fc_I = sum_{i in children(I)} P_iI phi_i   (coarse rows)
template <class T>
__device__ __forceinline__ T gather_at(const LV<T>& L, const T* __restrict__ phi, int B, int I,
                                       int b) {
  T acc = T(0);
  if (L.KR <= kMaxKR) {
    int idx[kMaxKR];
    T wk[kMaxKR];
#pragma unroll
    for (int k = 0; k < kMaxKR; ++k) {
      idx[k] = k < L.KR ? idx_ok(L.r_idx[(size_t)k * L.ldc + I], L.n, 3) : -1;
      wk[k] = k < L.KR ? L.r_w[(size_t)k * L.ldc + I] : T(0);
    }
#pragma unroll
    for (int k = 0; k < kMaxKR; ++k)
      if (idx[k] >= 0) acc = fma(wk[k], phi[(size_t)idx[k] * B + b], acc);
  } else {
    for (int k = 0; k < L.KR; ++k) {
      const int i = idx_ok(L.r_idx[(size_t)k * L.ldc + I], L.n, 3);
      if (i < 0) break;
      acc = fma(L.r_w[(size_t)k * L.ldc + I], phi[(size_t)i * B + b], acc);
    }
  }
  return acc;
}

template <class T>
__device__ __forceinline__ void gather_el(const LV<T>& L, const T* __restrict__ phi,
                                          T* __restrict__ fc, int B, size_t t) {
  int I, b;
  split_rb(t, B, I, b);
  fc[t] = gather_at(L, phi, B, I, b);
}

// pe_i = (P ec)_i   (fine rows)
template <class T>
__device__ __forceinline__ void pe_el(const LV<T>& L, const T* __restrict__ ec,
                                      T* __restrict__ pe, int B, size_t t) {
  int i, b;
  split_rb(t, B, i, b);
  pe[t] = prolong_at(L, i, ec, B, b);
}

// u_i = uin_i + wP1 pe_i + wP2 mean_{N(i)} pe   (uin may equal u)
template <class T>
__device__ __forceinline__ void prolong_conv_el(const LV<T>& L, const T* __restrict__ pe,
                                                const T* uin, T* u, int B,
                                                const T* __restrict__ prm, size_t t) {
  int i, b;
  split_rb(t, B, i, b);
  T phi = prm[P_WP1] * pe[t];
  phi = fma(prm[P_WP2], L.invdeg[i] * row_sum(L, i, pe, B, b), phi);
  u[t] = uin[t] + phi;
}

// Coarsest level: u = A_J^{-1} f by the FP64 Cholesky factor A_J = L L^T.
// Lc: L column-major (L[i + j n]); Uc: L^T column-major; dinv: 1/L_jj.
// Warps 0..nw-1 of the block take one right-hand side each in turn; column-
// oriented substitution in shared memory ys[nw][n].
template <class T>
__device__ __forceinline__ void coarse_chol_block(const double* __restrict__ Lc,
                                                  const double* __restrict__ Uc,
                                                  const double* __restrict__ dinv, int n,
                                                  const T* __restrict__ f, T* __restrict__ u,
                                                  int B, int nw, double* ys) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp >= nw) return;
  double* y = ys + (size_t)warp * n;
  for (int b = warp; b < B; b += nw) {
    for (int i = lane; i < n; i += 32) y[i] = (double)f[(size_t)i * B + b];
    __syncwarp();
    for (int j = 0; j < n; ++j) {  // L y = f
      const double yj = y[j] * dinv[j];
      __syncwarp();
      for (int i = j + 1 + lane; i < n; i += 32) y[i] = fma(-Lc[i + (size_t)j * n], yj, y[i]);
      if (lane == 0) y[j] = yj;
      __syncwarp();
    }
    for (int j = n - 1; j >= 0; --j) {  // L^T x = y
      const double xj = y[j] * dinv[j];
      __syncwarp();
      for (int i = lane; i < j; i += 32) y[i] = fma(-Uc[i + (size_t)j * n], xj, y[i]);
      if (lane == 0) y[j] = xj;
      __syncwarp();
    }
    for (int i = lane; i < n; i += 32) u[(size_t)i * B + b] = (T)y[i];
    __syncwarp();
  }
}

// ------------------------------------------------------- grid kernels ----

// Blocks of the first wave of a 256-thread grid on B300 (148 SMs x 8
// resident blocks).  Only they can run while the predecessor drains; later
// blocks start after it, so their prefetches would only add instructions.
constexpr unsigned kPrefetchBlocks = 148 * 8;

// PF: prefetch statement for the thread's row (read-only data only), run
// before griddepcontrol.wait by the first wave's blocks.  The grid kernels
// below take kB = 1 for one right-hand side known at compile time (the
// row/column split and the neighbour index products fold) and kB = 0 for
// B_ of them.
#define MG_GRID_PROLOGUE(N, PF)                                             \
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;           \
  const bool in_range = t < (size_t)(N);                                    \
  if (in_range && blockIdx.x < kPrefetchBlocks) { PF; }                     \
  pdl_wait();                                                               \
  pdl_launch();

template <class T, int kB = 0>
__global__ void __launch_bounds__(kThreads) k_residual(LV<T> L, const T* __restrict__ f,
                                                       const T* __restrict__ u, T* __restrict__ out,
                                                       int B_, const T* __restrict__ prm, int scale,
                                                       int u_zero) {
  const int B = kB ? kB : B_;
  MG_GRID_PROLOGUE((size_t)L.n * B, prefetch_row(L, row_of(t, B)))
  if (in_range) residual_el(L, f, u, out, B, prm, scale, u_zero, t);
  pdl_launch();
}

template <class T, int kB = 0>
__global__ void __launch_bounds__(kThreads) k_conv_update(LV<T> L, const T* __restrict__ x,
                                                          T* __restrict__ u, int B_,
                                                          const T* __restrict__ prm, int u_zero) {
  const int B = kB ? kB : B_;
  MG_GRID_PROLOGUE((size_t)L.n * B, prefetch_mean(L, row_of(t, B)))
  if (in_range) conv_update_el(L, x, u, B, prm, u_zero, t);
  pdl_launch();
}

// One pass of the ChebConv smoother (polynomial smoother of Sec. 3.3): with
// Lhat = D_g^{-1} L_g - I = -D_g^{-1} A_g (mean aggregation, lambda_max = 2)
// and the Chebyshev recurrence,
//   k = 1:   T_1 = Lhat T_0;                  u <- u + eta (c_0 T_0 + c_1 T_1)
//   k >= 2:  T_k = 2 Lhat T_{k-1} - T_{k-2};  u <- u + eta c_k T_k
// tprev = T_{k-1}, tpp = T_{k-2} (T_0 when k = 1), out = T_k.  out may be tpp:
// each entry of tpp is read, then overwritten, by the same thread.
template <class T, int kB = 0>
__global__ void __launch_bounds__(kThreads) k_cheb_step(LV<T> L, const T* __restrict__ tprev,
                                                        const T* tpp, T* out, T* __restrict__ u,
                                                        int B_, const T* __restrict__ prm,
                                                        const T* __restrict__ coef, int k,
                                                        int u_zero) {
  const int B = kB ? kB : B_;
  MG_GRID_PROLOGUE((size_t)L.n * B, prefetch_mean(L, row_of(t, B)))
  if (in_range) {
    int i, b;
    split_rb(t, B, i, b);
    const T lt = -(L.invdeg[i] * row_sum(L, i, tprev, B, b));
    const T q = tpp[t];
    T tk, upd;
    if (k == 1) {
      tk = lt;
      upd = fma(coef[1], tk, coef[0] * q);
    } else {
      tk = fma(T(2), lt, -q);
      upd = coef[k] * tk;
    }
    out[t] = tk;
    const T u0 = u_zero ? T(0) : u[t];
    u[t] = fma(prm[P_ETA], upd, u0);
  }
  pdl_launch();
}

template <class T, int kB = 0>
__global__ void __launch_bounds__(kThreads) k_jacobi(LV<T> L, const T* __restrict__ f,
                                                     const T* __restrict__ uin, T* __restrict__ uout,
                                                     int B_, const T* __restrict__ prm, int u_zero) {
  const int B = kB ? kB : B_;
  MG_GRID_PROLOGUE((size_t)L.n * B, prefetch_row(L, row_of(t, B)))
  if (in_range) jacobi_el(L, f, uin, uout, B, prm, u_zero, t);
  pdl_launch();
}

template <class T, int kB = 0>
__global__ void __launch_bounds__(kThreads) k_restrict(LV<T> L, const T* __restrict__ r,
                                                       T* __restrict__ fc, int B_,
                                                       const T* __restrict__ prm, int conv) {
  const int B = kB ? kB : B_;
  MG_GRID_PROLOGUE((size_t)L.nc * B, prefetch_r(L, row_of(t, B)))
  if (in_range) restrict_el(L, r, fc, B, prm, conv, t);
  pdl_launch();
}

template <class T, int kB = 0>
__global__ void __launch_bounds__(kThreads) k_prolong(LV<T> L, const T* __restrict__ ec,
                                                      const T* uin, T* u, int B_,
                                                      const T* __restrict__ prm, int conv) {
  const int B = kB ? kB : B_;
  MG_GRID_PROLOGUE((size_t)L.n * B, prefetch_p(L, row_of(t, B)))
  if (in_range) prolong_el(L, ec, uin, u, B, prm, conv, t);
  pdl_launch();
}

template <class T, int kB = 0>
__global__ void __launch_bounds__(kThreads) k_conv_r(LV<T> L, const T* __restrict__ r,
                                                     T* __restrict__ phi, int B_,
                                                     const T* __restrict__ prm) {
  const int B = kB ? kB : B_;
  MG_GRID_PROLOGUE((size_t)L.n * B, prefetch_mean(L, row_of(t, B)))
  if (in_range) conv_r_el(L, r, phi, B, prm, t);
  pdl_launch();
}

template <class T, int kB = 0>
__global__ void __launch_bounds__(kThreads) k_gather(LV<T> L, const T* __restrict__ phi,
                                                     T* __restrict__ fc, int B_) {
  const int B = kB ? kB : B_;
  MG_GRID_PROLOGUE((size_t)L.nc * B, prefetch_r(L, row_of(t, B)))
  if (in_range) gather_el(L, phi, fc, B, t);
  pdl_launch();
}

template <class T, int kB = 0>
__global__ void __launch_bounds__(kThreads) k_pe(LV<T> L, const T* __restrict__ ec,
                                                 T* __restrict__ pe, int B_) {
  const int B = kB ? kB : B_;
  MG_GRID_PROLOGUE((size_t)L.n * B, prefetch_p(L, row_of(t, B)))
  if (in_range) pe_el(L, ec, pe, B, t);
  pdl_launch();
}

template <class T, int kB = 0>
__global__ void __launch_bounds__(kThreads) k_prolong_conv(LV<T> L, const T* __restrict__ pe,
                                                           const T* uin, T* u, int B_,
                                                           const T* __restrict__ prm) {
  const int B = kB ? kB : B_;
  MG_GRID_PROLOGUE((size_t)L.n * B, prefetch_mean(L, row_of(t, B)))
  if (in_range) prolong_conv_el(L, pe, uin, u, B, prm, t);
  pdl_launch();
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_copy(const T* __restrict__ x, T* __restrict__ y,
                                                   size_t n) {
  MG_GRID_PROLOGUE(n, (void)0)
  if (in_range) y[t] = x[t];
  pdl_launch();
}

// ------------------------------------- one rhs on a DIA level, two rows --
// A thread takes rows i0 = 2g and i0 + 1: the rows share each diagonal's
// address arithmetic (32-bit offsets; the host checks ndia * ld < 2^31)
// and keep twice the loads in flight.  Row by row the arithmetic is that of
// residual_el, conv_update_el, conv_r_el and prolong_conv_el (same
// operations in the same order), so the results are bitwise those of the
// one-row kernels.  Launch: ceil(ceil(n / 2) / kThreads) blocks.

template <class T>
__global__ void __launch_bounds__(kThreads)
    k_residual_dia2r(LV<T> L, const T* __restrict__ f, const T* __restrict__ u,
                     T* __restrict__ out, const T* __restrict__ prm, int scale, int u_zero) {
  const int i0 = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i0 < L.n && blockIdx.x < kPrefetchBlocks) prefetch_row(L, i0);
  pdl_wait();
  pdl_launch();
  if (i0 >= L.n) return;
  const bool two = i0 + 1 < L.n;
  const int i1 = two ? i0 + 1 : i0;  // the second row, or the first again
  T r0 = f[i0], r1 = f[i1];
  if (!u_zero) {
    T a0 = T(0), a1 = T(0);
#pragma unroll
    for (int k = 0; k < kMaxDia; ++k) {
      if (k < L.ndia) {
        const T* dk = L.dval + k * L.ld;
        const T v0 = dk[i0], v1 = dk[i1];
        const int c0 = min(max(i0 + L.doff[k], 0), L.n - 1);
        const int c1 = min(max(i1 + L.doff[k], 0), L.n - 1);
        a0 = fma(v0, u[c0], a0);
        a1 = fma(v1, u[c1], a1);
      }
    }
    r0 = fma(-L.diag[i0], u[i0], r0) - a0;
    r1 = fma(-L.diag[i1], u[i1], r1) - a1;
  }
  if (scale) {
    r0 = prm[P_THETA] * (r0 * L.dinv[i0]);
    r1 = prm[P_THETA] * (r1 * L.dinv[i1]);
  }
  out[i0] = r0;
  if (two) out[i1] = r1;
  pdl_launch();
}

enum { MEAN_CONV_UPDATE = 0, MEAN_CONV_R = 1, MEAN_PROLONG_CONV = 2, MEAN_CONV_UPDATE_REFINE = 3 };

// The refinement update u += 2^sexp_b c of an FP32 cycle's result c, for
// blocks of m rows (m = n: one system; the stacked contexts' slots
// otherwise), applied by the cycle's last level-0 kernel to the rows it
// writes (MEAN_CONV_UPDATE_REFINE): the arithmetic of k_refine_update and
// k_blk_refine_update, which it replaces.
struct RefineEp {
  double* u;
  const int* sexp;
  const int* active;
  int* iters;
  int m;
};

// The mean-only steps: CONV_UPDATE u = u0 + eta (wB1 x + wB2 mean x) (u0 =
// 0 when u_zero); CONV_R y = wR1 x + wR2 mean x; PROLONG_CONV u = uin + wP1 x
// + wP2 mean x.  The neighbour test comes from the level's mask.
template <class T, int MODE>
__global__ void __launch_bounds__(kThreads)
    k_mean_dia2r(LV<T> L, const T* __restrict__ x, const T* uin, T* y,
                 const T* __restrict__ prm, int u_zero, RefineEp ep) {
  const int i0 = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i0 < L.n && blockIdx.x < kPrefetchBlocks) prefetch_mean(L, i0);
  pdl_wait();
  pdl_launch();
  if (i0 >= L.n) return;
  const bool two = i0 + 1 < L.n;
  const int i1 = two ? i0 + 1 : i0;
  const unsigned m0 = nb_mask(L, i0), m1 = nb_mask(L, i1);
  T s0 = T(0), s1 = T(0);
#pragma unroll
  for (int k = 0; k < kMaxDia; ++k) {
    if (k < L.ndia) {
      const int c0 = min(max(i0 + L.doff[k], 0), L.n - 1);
      const int c1 = min(max(i1 + L.doff[k], 0), L.n - 1);
      const T x0 = x[c0], x1 = x[c1];
      s0 += ((m0 >> k) & 1u) ? x0 : T(0);
      s1 += ((m1 >> k) & 1u) ? x1 : T(0);
    }
  }
  const T d0 = L.invdeg[i0], d1 = L.invdeg[i1];
  if constexpr (MODE == MEAN_CONV_UPDATE || MODE == MEAN_CONV_UPDATE_REFINE) {
    const T p0 = fma(prm[P_WB1], x[i0], prm[P_WB2] * (d0 * s0));
    const T p1 = fma(prm[P_WB1], x[i1], prm[P_WB2] * (d1 * s1));
    const T u0 = u_zero ? T(0) : y[i0];
    const T u1 = u_zero ? T(0) : y[i1];
    const T c0 = fma(prm[P_ETA], p0, u0), c1 = fma(prm[P_ETA], p1, u1);
    y[i0] = c0;
    if (two) y[i1] = c1;
    if constexpr (MODE == MEAN_CONV_UPDATE_REFINE) {
      const int b0 = i0 / ep.m, b1 = i1 / ep.m;
      if (ep.active[b0]) {
        ep.u[i0] += scale2((double)c0, ep.sexp[b0]);
        if (i0 - b0 * ep.m == 0) ep.iters[b0] += 1;
      }
      if (two && ep.active[b1]) {
        ep.u[i1] += scale2((double)c1, ep.sexp[b1]);
        if (i1 - b1 * ep.m == 0) ep.iters[b1] += 1;
      }
    }
  } else if constexpr (MODE == MEAN_CONV_R) {
    T p0 = prm[P_WR1] * x[i0], p1 = prm[P_WR1] * x[i1];
    p0 = fma(prm[P_WR2], d0 * s0, p0);
    p1 = fma(prm[P_WR2], d1 * s1, p1);
    y[i0] = p0;
    if (two) y[i1] = p1;
  } else {
    T p0 = prm[P_WP1] * x[i0], p1 = prm[P_WP1] * x[i1];
    p0 = fma(prm[P_WP2], d0 * s0, p0);
    p1 = fma(prm[P_WP2], d1 * s1, p1);
    const T v0 = uin[i0] + p0, v1 = uin[i1] + p1;
    y[i0] = v0;
    if (two) y[i1] = v1;
  }
  pdl_launch();
}

// P e_c per fine row (prolong_at's arithmetic), one rhs, two rows per
// thread; any layout (the prolongation lists are per row).
template <class T>
__global__ void __launch_bounds__(kThreads)
    k_pe2r(LV<T> L, const T* __restrict__ ec, T* __restrict__ pe) {
  const int i0 = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i0 < L.n && blockIdx.x < kPrefetchBlocks) prefetch_p(L, i0);
  pdl_wait();
  pdl_launch();
  if (i0 >= L.n) return;
  const bool two = i0 + 1 < L.n;
  const int i1 = two ? i0 + 1 : i0;
  const T v0 = prolong_at(L, i0, ec, 1, 0), v1 = prolong_at(L, i1, ec, 1, 0);
  pe[i0] = v0;
  if (two) pe[i1] = v1;
  pdl_launch();
}

template <class T>
__global__ void k_coarse_chol(const double* __restrict__ Lc, const double* __restrict__ Uc,
                              const double* __restrict__ dinv, int n, const T* __restrict__ f,
                              T* __restrict__ u, int B) {
  extern __shared__ double ys[];
  pdl_wait();
  pdl_launch();
  coarse_chol_block(Lc, Uc, dinv, n, f, u, B, (int)(blockDim.x >> 5), ys);
  pdl_launch();
}


// ------------------------------------------------------ small levels -----

// All levels lt..J-1 of one V-cycle in a single block: down (smoothing,
// residual, restriction), the coarsest Cholesky solve, up (prolongation,
// smoothing).  Level lt's right-hand side is f[lt]; its result is u[lt].
template <class T>
struct TailArgs {
  int lt, J, B, nu_pre, nu_post, nJ, cwarps, lt_zero, smem_vectors, smem_matrix;
  unsigned convB, convR, convP;  // bit l: w2 != 0 on level l
  int nsl[kMaxLevels];           // SELL slices per level (0 for DIA levels)
  int nent[kMaxLevels];          // SELL entries per level
  LV<T> L[kMaxLevels];
  const T* f[kMaxLevels];
  T* u[kMaxLevels];
  T* t[kMaxLevels];
  T* u2[kMaxLevels];
  const T* prm;  // [J-1][P_COUNT]
  const double* cL;
  const double* cU;
  const double* cDinv;
  const double* cInv;  // explicit inverse of A_J (row-major), or NULL: substitutions
  int cInvLd;          // its row stride
  int tw[kMaxLevels];  // warps of the team that runs level l (a power of two <= 32)
};

// The threads that run one small level of k_tail: the first W warps of the
// block.  A level's steps are separated by a barrier among exactly those
// threads: __syncthreads for the whole block, the named barrier log2(W)
// (bar.sync with W * 32 threads) for 2..8 warps, __syncwarp for one warp.
// Coarser levels have no more warps than finer ones, so a level's team
// contains the teams of all coarser levels; a level small enough for a few
// warps thus pays for cheap barriers instead of a barrier of the whole block.
// Which thread computes an entry never changes its value.
struct Team {
  int W;
  __device__ __forceinline__ bool member() const { return (int)(threadIdx.x >> 5) < W; }
  __device__ __forceinline__ int size() const { return W * 32; }
  __device__ __forceinline__ void sync() const {
    if (W * 32 >= (int)blockDim.x) {
      __syncthreads();
    } else if (W == 1) {
      __syncwarp();
    } else {
      const int id = 31 - __clz(W);  // 1..4
      asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(W * 32) : "memory");
    }
  }
};

// Vectors of the small levels: in shared memory when a.smem_vectors (the
// usual case), else the global level buffers.
template <class T>
struct TailVecs {
  T* u[kMaxLevels];
  T* f[kMaxLevels];
  T* t[kMaxLevels];
  T* u2[kMaxLevels];
};

__host__ __device__ inline size_t tail_align(size_t x) { return (x + 15) & ~size_t(15); }

// Shared-memory bytes of nchunk rows of count elements whose global row
// stride is ld: one block when the rows are contiguous (ld == count), else
// rows padded to a multiple of 4 elements (smem_take_rows).
template <class U>
__host__ __device__ inline size_t rows_bytes(int count, int ld, int nchunk) {
  if (ld == count) return tail_align((size_t)nchunk * count * sizeof(U));
  return (size_t)nchunk * ((count + 3) & ~3) * sizeof(U);
}

// Shared-memory bytes of one small level: its four vectors (vec) and its
// read-only arrays (mat): DIA values or SELL slices, diag, dinv, invdeg and,
// above the coarsest level, the prolongation and restriction lists.
template <class T>
__host__ __device__ inline size_t tail_level_bytes(const LV<T>& L, int nsl, int nent, int B,
                                                   bool last, bool vec, bool mat) {
  const int n = L.n, nc = L.nc;
  size_t s = 0;
  if (vec) s += 4 * tail_align((size_t)n * B * sizeof(T));
  if (mat) {
    if (L.ndia > 0) {
      s += rows_bytes<T>(n, L.ld, L.ndia);
    } else {
      s += tail_align((size_t)(nsl + 1) * sizeof(int)) + tail_align((size_t)nent * sizeof(int)) +
           tail_align((size_t)nent * sizeof(T));
    }
    s += 3 * tail_align((size_t)n * sizeof(T));
    if (!last) {
      s += rows_bytes<int>(n, L.ld, 2) + rows_bytes<T>(n, L.ld, 2);
      s += rows_bytes<int>(nc, L.ldc, L.KR) + rows_bytes<T>(nc, L.ldc, L.KR);
    }
  }
  return s;
}

// Dynamic shared memory of k_tail: Cholesky scratch, the parameters of
// levels 0..J-2, then every level lt..J-1 as laid out by tail_level_bytes.
template <class T>
__host__ __device__ inline size_t tail_head_bytes(const TailArgs<T>& a) {
  return tail_align((size_t)a.cwarps * a.nJ * sizeof(double)) +
         tail_align((size_t)(a.J - 1) * P_COUNT * sizeof(T));
}
template <class T>
__host__ __device__ inline size_t tail_smem_bytes(const TailArgs<T>& a, int lt) {
  size_t off = tail_head_bytes(a);
  for (int l = lt; l < a.J; ++l)
    off += tail_level_bytes<T>(a.L[l], a.nsl[l], a.nent[l], a.B, l == a.J - 1,
                               a.smem_vectors != 0, a.smem_matrix != 0);
  return off;
}

// The copies carry no compiler memory clobber: their destinations are read
// only after cp_async_wait_all (which has one) and a barrier, and without
// it the loads of the next copy's source pointer need not wait for the
// issue of the previous copy.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem_src));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}
// One element of 4 or 8 bytes (both addresses aligned to its size).
template <class U>
__device__ __forceinline__ void cp_async_el(U* smem_dst, const U* gmem_src) {
  static_assert(sizeof(U) == 4 || sizeof(U) == 8, "cp.async element of 4 or 8 bytes");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  if constexpr (sizeof(U) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem_src));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem_src));
}

// Starts copying count elements into shared memory at base + off (all
// threads of the block take part) and advances off; returns the
// shared-memory copy.  Every transfer is a cp.async that stays in flight
// until cp_async_wait_all: 16-byte chunks from a 16-byte aligned source, and
// element-sized ones for the elements past the last whole chunk or from an
// unaligned source, so nothing beyond src + count is read and no copy
// waits for another (a plain load per array would put one memory round trip
// per array on the block's path).
// The copies are spread over nlanes threads, this one being lane (the whole
// block by default).
template <class U>
__device__ __forceinline__ U* smem_take(unsigned char* base, size_t& off, const U* src,
                                        size_t count, unsigned lane = threadIdx.x,
                                        unsigned nlanes = blockDim.x) {
  U* dst = (U*)(base + off);
  off += tail_align(count * sizeof(U));
  size_t first = 0;  // first element copied one by one
  if ((((uintptr_t)src) & 15) == 0) {
    const size_t nchunk = count * sizeof(U) / 16;
    const char* s = (const char*)src;
    char* d = (char*)dst;
    for (size_t k = lane; k < nchunk; k += nlanes) cp_async16(d + 16 * k, s + 16 * k);
    first = nchunk * 16 / sizeof(U);
  }
  for (size_t k = first + lane; k < count; k += nlanes) cp_async_el(dst + k, src + k);
  return dst;
}

// smem_take of nchunk rows of count elements, row k at src + k * ld: one
// copy when the rows are contiguous, else row by row into rows padded to a
// multiple of 4 elements (16 bytes for 4- and 8-byte types).  ld_out is the
// shared-memory row stride (the layout rows_bytes counts).
template <class U>
__device__ __forceinline__ U* smem_take_rows(unsigned char* base, size_t& off, const U* src,
                                             int count, int ld, int nchunk, int& ld_out,
                                             unsigned lane = threadIdx.x,
                                             unsigned nlanes = blockDim.x) {
  if (ld == count) {
    ld_out = count;
    return smem_take(base, off, src, (size_t)nchunk * count, lane, nlanes);
  }
  const int lds = (count + 3) & ~3;
  U* dst = (U*)(base + off);
  for (int k = 0; k < nchunk; ++k) {
    size_t o = off + (size_t)k * lds * sizeof(U);
    smem_take(base, o, src + (size_t)k * ld, (size_t)count, lane, nlanes);
  }
  off += (size_t)nchunk * lds * sizeof(U);
  ld_out = lds;
  return dst;
}

// Offset of column j of a packed column-major lower triangle of order n.
__device__ __forceinline__ size_t packed_col(int n, int j) {
  return (size_t)j * n - (size_t)j * (j - 1) / 2;
}

// u = A_J^{-1} f with the explicit FP64 inverse (row-major n x n with row
// stride ld, formed on the host from the Cholesky factor; a leading block of
// it for the leading blocks of a stacked context): one thread per (row, rhs) output,
// the products summed in column order.  Every output is independent, so the
// step spreads over many SMs instead of running the 2n dependent steps of
// the substitutions on one (B300's FP64 pipe makes those slow).
template <class T>
__device__ __forceinline__ void coarse_inv_el(const double* __restrict__ Ainv, int n, int ld,
                                              const T* __restrict__ f, T* __restrict__ u, int B,
                                              size_t t) {
  int i, b;
  split_rb(t, B, i, b);
  const double* row = Ainv + (size_t)i * ld;
  double acc = 0.0;
#pragma unroll 8
  for (int j = 0; j < n; ++j) acc = fma(row[j], (double)f[(size_t)j * B + b], acc);
  u[t] = (T)acc;
}

constexpr int kCoarseInvThreads = 64;

template <class T>
__global__ void __launch_bounds__(kCoarseInvThreads)
    k_coarse_inv(const double* __restrict__ Ainv, int n, int ld, const T* __restrict__ f,
                 T* __restrict__ u, int B) {
  pdl_wait();
  pdl_launch();
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < (size_t)n * B) coarse_inv_el(Ainv, n, ld, f, u, B, t);
}

// The same substitutions as coarse_chol_block with the factor staged in
// shared memory as a packed lower triangle (column j holds rows j..n-1):
// every step reads the factor at shared-memory latency.  Same values and
// order, hence the same results.  Warp w of block k takes right-hand sides
// k * nw + w, + nw * gridDim.x, ...: a grid of several blocks spreads the
// right-hand sides over SMs, whose FP64 pipes bound the substitutions.
template <class T>
__global__ void k_coarse_chol_packed(const double* __restrict__ Lp, const double* __restrict__ dinv,
                                     int n, const T* __restrict__ f, T* __restrict__ u, int B) {
  extern __shared__ __align__(16) unsigned char cs_smem[];
  pdl_wait();
  pdl_launch();
  size_t off = 0;
  const double* P = smem_take(cs_smem, off, Lp, (size_t)n * (n + 1) / 2);
  const double* di = smem_take(cs_smem, off, dinv, (size_t)n);
  double* ys = (double*)(cs_smem + off);
  cp_async_wait_all();
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double* y = ys + (size_t)warp * n;
  for (int b = blockIdx.x * nw + warp; b < B; b += nw * gridDim.x) {
    for (int i = lane; i < n; i += 32) y[i] = (double)f[(size_t)i * B + b];
    __syncwarp();
    for (int j = 0; j < n; ++j) {  // L y = f
      const double yj = y[j] * di[j];
      const double* col = P + packed_col(n, j) - j;  // col[i] = L_ij
      __syncwarp();
      for (int i = j + 1 + lane; i < n; i += 32) y[i] = fma(-col[i], yj, y[i]);
      if (lane == 0) y[j] = yj;
      __syncwarp();
    }
    for (int j = n - 1; j >= 0; --j) {  // L^T x = y
      const double xj = y[j] * di[j];
      __syncwarp();
      for (int i = lane; i < j; i += 32) y[i] = fma(-P[packed_col(n, i) + (j - i)], xj, y[i]);
      if (lane == 0) y[j] = xj;
      __syncwarp();
    }
    for (int i = lane; i < n; i += 32) u[(size_t)i * B + b] = (T)y[i];
    __syncwarp();
  }
  pdl_launch();
}

template <class T>
__device__ __forceinline__ void tail_smooth(const TailArgs<T>& a, const LV<T>* Ls,
                                            const T* prm_all, const TailVecs<T>& v, int l, int nu,
                                            bool zero, const Team& tm, int B) {
  const LV<T> L = Ls[l];  // in registers across the steps' barriers
  const size_t N = (size_t)L.n * B;
  const T* prm = prm_all + (size_t)l * P_COUNT;
  const size_t t0 = threadIdx.x, dt = tm.size();
  if ((a.convB >> l) & 1u) {
    for (int k = 0; k < nu; ++k) {
      const int z = zero && k == 0;
      for (size_t t = t0; t < N; t += dt)
        residual_el(L, (const T*)v.f[l], (const T*)v.u[l], v.t[l], B, prm, 1, z, t);
      tm.sync();
      for (size_t t = t0; t < N; t += dt)
        conv_update_el(L, (const T*)v.t[l], v.u[l], B, prm, z, t);
      tm.sync();
    }
  } else {
    T* cur = v.u[l];
    T* oth = v.u2[l];
    for (int k = 0; k < nu; ++k) {
      const int z = zero && k == 0;
      for (size_t t = t0; t < N; t += dt)
        jacobi_el(L, (const T*)v.f[l], (const T*)cur, oth, B, prm, z, t);
      tm.sync();
      T* tmp = cur;
      cur = oth;
      oth = tmp;
    }
    if (cur != v.u[l]) {
      for (size_t t = t0; t < N; t += dt) v.u[l][t] = cur[t];
      tm.sync();
    }
  }
  if (nu == 0 && zero) {
    for (size_t t = t0; t < N; t += dt) v.u[l][t] = T(0);
    tm.sync();
  }
}

// kB = 1: one right-hand side, known at compile time (the index arithmetic
// of every step folds); kB = 0: B right-hand sides.
template <class T, int kB>
__global__ void __launch_bounds__(kTailBlock, 1) k_tail(const __grid_constant__ TailArgs<T> a) {
  extern __shared__ __align__(16) unsigned char tail_smem[];
  // The arguments, the staged level views and the vector pointers live in
  // shared memory, one copy per block.  Levels are indexed at run time: as
  // per-thread tables they would sit in local memory (1024 copies, which L1
  // does not hold, so every step would reload them from L2), and reading
  // each array's pointer from the argument space after the previous
  // cp.async would put one argument fetch per array on the block's path.
  __shared__ TailArgs<T> sa;
  __shared__ LV<T> sL[kMaxLevels];
  __shared__ TailVecs<T> v;
  {
    const unsigned* src = reinterpret_cast<const unsigned*>(&a);
    unsigned* dst = reinterpret_cast<unsigned*>(&sa);
    for (int k = threadIdx.x; k < (int)(sizeof(TailArgs<T>) / 4); k += blockDim.x) dst[k] = src[k];
  }
  __syncthreads();
  double* ys = (double*)tail_smem;
  const int J = a.J, lt = a.lt;
  const int B = kB ? kB : a.B;
  {
    const unsigned* src = reinterpret_cast<const unsigned*>(&sa.L[lt]);
    unsigned* dst = reinterpret_cast<unsigned*>(&sL[lt]);
    const int words = (int)((J - lt) * sizeof(LV<T>) / 4);
    for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
  }
  __syncthreads();
  // Lay out every small level in shared memory (the same order as
  // tail_level_bytes): vectors first, then the read-only arrays, copied
  // once per cycle.  Warp l - lt stages level l (its offset is the head
  // plus the sizes of levels lt..l-1), so the levels' copy loops
  // run side by side instead of each warp stepping through all of them
  // (warps take further levels in turn if there are more levels than warps).
  // The read-only arrays never depend on the preceding kernel, so their
  // copies are issued before griddepcontrol.wait and overlap its drain; the
  // level-lt vectors it writes are copied after the wait.  Lane 0 of the
  // warp records the level's pointers; the barrier after the copies
  // publishes them.
  const size_t off_lt_vec = tail_head_bytes(a);
  for (int l = lt + (int)(threadIdx.x >> 5); l < J; l += (int)(blockDim.x >> 5)) {
    const unsigned lane = threadIdx.x & 31;
    const bool w0 = lane == 0;
    {
      size_t off = off_lt_vec;
      for (int k = lt; k < l; ++k)
        off += tail_level_bytes<T>(sa.L[k], sa.nsl[k], sa.nent[k], B, k == J - 1,
                                   a.smem_vectors != 0, a.smem_matrix != 0);
      const LV<T>& G = sa.L[l];
      LV<T>& S = sL[l];
      const size_t nB = (size_t)G.n * B;
      if (a.smem_vectors) {
        const size_t bytes = tail_align(nB * sizeof(T));
        if (w0) {
          v.u[l] = (T*)(tail_smem + off);
          v.f[l] = (T*)(tail_smem + off + bytes);
          v.t[l] = (T*)(tail_smem + off + 2 * bytes);
          v.u2[l] = (T*)(tail_smem + off + 3 * bytes);
        }
        off += 4 * bytes;
      } else if (w0) {
        v.u[l] = sa.u[l];
        v.f[l] = (T*)sa.f[l];
        v.t[l] = sa.t[l];
        v.u2[l] = sa.u2[l];
      }
      if (a.smem_matrix) {
        int ld = G.ld, ldc = G.ldc;
        if (G.ndia > 0) {
          const T* dv = smem_take_rows(tail_smem, off, G.dval, G.n, G.ld, G.ndia, ld, lane, 32);
          if (w0) S.dval = dv;
        } else {
          const int* sp = smem_take(tail_smem, off, G.sl_ptr, (size_t)sa.nsl[l] + 1, lane, 32);
          const int* cl = smem_take(tail_smem, off, G.col, (size_t)sa.nent[l], lane, 32);
          const T* vl = smem_take(tail_smem, off, G.val, (size_t)sa.nent[l], lane, 32);
          if (w0) {
            S.sl_ptr = sp;
            S.col = cl;
            S.val = vl;
          }
        }
        const T* dg = smem_take(tail_smem, off, G.diag, (size_t)G.n, lane, 32);
        const T* di = smem_take(tail_smem, off, G.dinv, (size_t)G.n, lane, 32);
        const T* ig = smem_take(tail_smem, off, G.invdeg, (size_t)G.n, lane, 32);
        if (w0) {
          S.diag = dg;
          S.dinv = di;
          S.invdeg = ig;
        }
        if (l < J - 1) {
          const int* pi = smem_take_rows(tail_smem, off, G.p_idx, G.n, G.ld, 2, ld, lane, 32);
          const T* pw = smem_take_rows(tail_smem, off, G.p_w, G.n, G.ld, 2, ld, lane, 32);
          const int* ri = smem_take_rows(tail_smem, off, G.r_idx, G.nc, G.ldc, G.KR, ldc, lane, 32);
          const T* rw = smem_take_rows(tail_smem, off, G.r_w, G.nc, G.ldc, G.KR, ldc, lane, 32);
          if (w0) {
            S.p_idx = pi;
            S.p_w = pw;
            S.r_idx = ri;
            S.r_w = rw;
          }
        }
        if (w0) {
          S.ld = ld;
          S.ldc = ldc;
          S.nbm = nullptr;  // the staged values give the neighbour test
        }
      }
    }
  }
  pdl_wait();
  pdl_launch();
  // the parameters of levels 0..J-2 (a training step may write them),
  // after the wait
  size_t off_prm = tail_align((size_t)a.cwarps * a.nJ * sizeof(double));
  const T* prm_all = smem_take(tail_smem, off_prm, a.prm, (size_t)(J - 1) * P_COUNT);
  if (a.smem_vectors) {
    const size_t nB = (size_t)sa.L[lt].n * B;
    size_t o2 = off_lt_vec + tail_align(nB * sizeof(T));
    smem_take(tail_smem, o2, sa.f[lt], nB);
    if (!a.lt_zero) {
      o2 = off_lt_vec;
      smem_take(tail_smem, o2, (const T*)sa.u[lt], nB);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // descent: level l by its team (teams shrink towards the coarsest level)
  for (int l = lt; l < J - 1; ++l) {
    const Team tm{sa.tw[l]};
    if (!tm.member()) break;
    const LV<T> L = sL[l];
    const T* prm = prm_all + (size_t)l * P_COUNT;
    const size_t t0 = threadIdx.x, dt = tm.size();
    tail_smooth(a, sL, prm_all, v, l, a.nu_pre, l == lt ? (a.lt_zero != 0) : true, tm, B);
    const size_t N = (size_t)L.n * B;
    for (size_t t = t0; t < N; t += dt)
      residual_el(L, (const T*)v.f[l], (const T*)v.u[l], v.t[l], B, prm, 0, 0, t);
    tm.sync();
    const size_t Nc = (size_t)L.nc * B;
    if ((a.convR >> l) & 1u) {  // Phi_R per fine row, then the gather P^T
      for (size_t t = t0; t < N; t += dt) conv_r_el(L, (const T*)v.t[l], v.u2[l], B, prm, t);
      tm.sync();
      for (size_t t = t0; t < Nc; t += dt) gather_el(L, (const T*)v.u2[l], v.f[l + 1], B, t);
    } else {
      for (size_t t = t0; t < Nc; t += dt)
        restrict_el(L, (const T*)v.t[l], v.f[l + 1], B, prm, 0, t);
    }
    tm.sync();
  }
  {
    const Team tm{sa.tw[J - 1]};
    if (tm.member()) {
      if (a.cInv) {
        for (size_t t = threadIdx.x; t < (size_t)a.nJ * B; t += tm.size())
          coarse_inv_el(a.cInv, a.nJ, a.cInvLd, (const T*)v.f[J - 1], v.u[J - 1], B, t);
      } else {
        coarse_chol_block(a.cL, a.cU, a.cDinv, a.nJ, (const T*)v.f[J - 1], v.u[J - 1], B,
                          min(a.cwarps, tm.W), ys);
      }
    }
  }
  // ascent: each team first waits for the coarser levels' (sub-)team
  for (int l = J - 2; l >= lt; --l) {
    const Team tm{sa.tw[l]};
    if (!tm.member()) continue;
    tm.sync();
    const LV<T> L = sL[l];
    const T* prm = prm_all + (size_t)l * P_COUNT;
    const size_t t0 = threadIdx.x, dt = tm.size();
    const size_t N = (size_t)L.n * B;
    if ((a.convP >> l) & 1u) {  // P e_c per fine row, then Phi_P and the update
      for (size_t t = t0; t < N; t += dt) pe_el(L, (const T*)v.u[l + 1], v.t[l], B, t);
      tm.sync();
      for (size_t t = t0; t < N; t += dt)
        prolong_conv_el(L, (const T*)v.t[l], (const T*)v.u[l], v.u[l], B, prm, t);
    } else {
      for (size_t t = t0; t < N; t += dt)
        prolong_el(L, (const T*)v.u[l + 1], (const T*)v.u[l], v.u[l], B, prm, 0, t);
    }
    tm.sync();
    tail_smooth(a, sL, prm_all, v, l, a.nu_post, false, tm, B);
  }
  __syncthreads();
  if (a.smem_vectors) {
    const size_t N = (size_t)sa.L[lt].n * B;
    T* ug = sa.u[lt];
    for (size_t t = threadIdx.x; t < N; t += blockDim.x) ug[t] = v.u[lt][t];
  }
  pdl_launch();
}

// ---------------------------------------------------------------------------
// FP64 outer loops (refinement, plain solve, flexible CG) with deterministic
// per-right-hand-side reductions whose grouping does not depend on the batch:
// a block covers kRedRows = 32 rows and bt = min(B, 32) right-hand-side
// columns (blockDim = 32 * bt, grid = (ceil(n / 32), ceil(B / bt))), sums its
// 32 rows per column with a fixed tree into partial[blockIdx.x * B + b], and
// k_reduce adds the blocks in a fixed order.  So every right-hand side's
// norms and dot products are bitwise the same whatever else is in the batch.
// ---------------------------------------------------------------------------

constexpr int kRedRows = 32;
constexpr int kRedMax = 1024;  // kRedRows x 32 columns

// (row, rhs) of this thread in the reduction tiling.
__device__ __forceinline__ void red_tile(int n, int B, int& i, int& b, bool& ok) {
  const int bt = blockDim.x / kRedRows;
  const int t = threadIdx.x;
  i = blockIdx.x * kRedRows + t / bt;
  b = blockIdx.y * bt + t % bt;
  ok = i < n && b < B;
}

// sh[r * bt + c] summed over the 32 rows r (fixed tree) into sh[c].
__device__ __forceinline__ void block_rows_reduce32(double* sh) {
  const int bt = blockDim.x / kRedRows;
  const int t = threadIdx.x;
  const int r = t / bt;
  for (int s = kRedRows / 2; s >= 1; s >>= 1) {
    if (r < s) sh[t] += sh[t + s * bt];
    __syncthreads();
  }
}

// Writes the block's column sums (row 0 of sh) to partial[blk * B + b].
__device__ __forceinline__ void red_store(const double* sh, int B, double* __restrict__ partial) {
  const int bt = blockDim.x / kRedRows;
  const int t = threadIdx.x;
  const int b = blockIdx.y * bt + t;
  if (t < bt && b < B) partial[(size_t)blockIdx.x * B + b] = sh[t];
}

// r = f - A u in FP64; optionally rhat = float(r * 2^-sexp[b]); partial sums
// of r^2.
// d0 (may be NULL): also the first smoothing step's delta of the next FP32
// cycle, which starts from zero on level 0: theta_0 (rhat dinv_0), the
// arithmetic of residual_el with u_zero (FP32 level-0 dinv0, parameters
// prm0 of level 0), so that cycle skips that launch.
__global__ void __launch_bounds__(kRedMax) k_resid64(LV<double> L, const double* __restrict__ f,
                                                     const double* __restrict__ u,
                                                     float* __restrict__ rhat,
                                                     const int* __restrict__ sexp, int B,
                                                     double* __restrict__ partial,
                                                     float* __restrict__ d0,
                                                     const float* __restrict__ dinv0,
                                                     const float* __restrict__ prm0) {
  pdl_wait();
  __shared__ double sh[kRedMax];
  int i, b;
  bool ok;
  red_tile(L.n, B, i, b, ok);
  double r = 0.0;
  if (ok) {
    const size_t k = (size_t)i * B + b;
    const double ax = row_ax(L, i, u, B, b);
    r = fma(-L.diag[i], u[k], f[k]) - ax;
    if (rhat) {
      const float rh = (float)scale2(r, -sexp[b]);
      rhat[k] = rh;
      if (d0) d0[k] = prm0[P_THETA] * (rh * dinv0[i]);
    }
  }
  sh[threadIdx.x] = r * r;
  __syncthreads();
  block_rows_reduce32(sh);
  red_store(sh, B, partial);
}

// r = f - A u in FP64 with the same arithmetic as k_resid64.
__global__ void __launch_bounds__(kRedMax) k_outer_residual64(LV<double> L,
                                                              const double* __restrict__ f,
                                                              const double* __restrict__ u,
                                                              double* __restrict__ out, int B) {
  pdl_wait();
  int i, b;
  bool ok;
  red_tile(L.n, B, i, b, ok);
  if (ok) {
    const size_t k = (size_t)i * B + b;
    out[k] = fma(-L.diag[i], u[k], f[k]) - row_ax(L, i, u, B, b);
  }
}

// partial sums of x^2 (FP64), same tiling as k_resid64.
__global__ void __launch_bounds__(kRedMax) k_sumsq64(const double* __restrict__ x, int n, int B,
                                                     double* __restrict__ partial) {
  pdl_wait();
  __shared__ double sh[kRedMax];
  int i, b;
  bool ok;
  red_tile(n, B, i, b, ok);
  const double v = ok ? x[(size_t)i * B + b] : 0.0;
  sh[threadIdx.x] = v * v;
  __syncthreads();
  block_rows_reduce32(sh);
  red_store(sh, B, partial);
}

// out[b] = sum over blocks of partial[blk * B + b]; grid = B blocks.
// Sum of the partials of right-hand side b in a fixed order (strided per
// thread, then a fixed tree); one block of kThreads threads; every thread
// returns the sum.
__device__ __forceinline__ double block_sum_partials(const double* __restrict__ partial,
                                                     int nblk, int B, int b, double* sh) {
  double s = 0.0;
  for (int k = threadIdx.x; k < nblk; k += kThreads) s += partial[(size_t)k * B + b];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w >= 1; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// out[b] = sum of the partials of right-hand side b; one block per b.
__global__ void __launch_bounds__(kThreads) k_reduce(const double* __restrict__ partial, int nblk,
                                                     int B, double* __restrict__ out) {
  pdl_wait();
  __shared__ double sh[kThreads];
  const int b = blockIdx.x;
  const double r = block_sum_partials(partial, nblk, B, b, sh);
  if (threadIdx.x == 0) out[b] = r;
}

// Convergence test per right-hand side (body of k_check and k_reduce_check,
// one block).  ctl = (tol, max_iter).  state[0] = right-hand sides still
// active, state[1] = 1 if a residual is not finite, state[2] = iterations
// done (reset when inc == 0, else +1), state[3] = continue: some right-hand
// side is active, all residuals are finite and fewer than max_iter
// iterations ran.  With set_cond the same value becomes the enclosing
// while-node's condition (h is ignored otherwise).
__device__ __forceinline__ void check_block(const double* __restrict__ rsum,
                                            const double* __restrict__ fsum, int B,
                                            const double* __restrict__ ctl,
                                            int* __restrict__ active, double* __restrict__ relres,
                                            int* __restrict__ sexp, int* __restrict__ state,
                                            int inc, cudaGraphConditionalHandle h, int set_cond) {
  __shared__ int cnt, bad;
  const double tol = ctl[0];
  if (threadIdx.x == 0) { cnt = 0; bad = 0; }
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const double rn = sqrt(rsum[b]), fn = sqrt(fsum[b]);
    const double rel = fn > 0.0 ? rn / fn : rn;
    relres[b] = rel;
    if (!isfinite(rel)) atomicAdd(&bad, 1);
    if (active[b] && !(rel < tol) && isfinite(rel)) atomicAdd(&cnt, 1);
    else active[b] = 0;
    sexp[b] = rn > 0.0 && isfinite(rn) ? ilogb(rn) : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int it = inc ? state[2] + 1 : 0;
    state[0] = cnt;
    state[1] = bad;
    state[2] = it;
    const int go = cnt > 0 && bad == 0 && (double)it < ctl[1];
    state[3] = go;  // read by the host when it drives the loop
    if (set_cond) cudaGraphSetConditional(h, go ? 1u : 0u);
  }
}

__global__ void k_check(const double* __restrict__ rsum, const double* __restrict__ fsum, int B,
                        const double* __restrict__ ctl, int* __restrict__ active,
                        double* __restrict__ relres, int* __restrict__ sexp,
                        int* __restrict__ state, int inc, cudaGraphConditionalHandle h,
                        int set_cond) {
  pdl_wait();
  check_block(rsum, fsum, B, ctl, active, relres, sexp, state, inc, h, set_cond);
}

// k_reduce, the copy sexp_prev = sexp (when sexp_prev is given) and k_check
// in one block of kThreads threads, for small B * nblk (the sums run one
// right-hand side after another, each in k_reduce's order, so the results
// are those of the three kernels).
__global__ void __launch_bounds__(kThreads)
    k_reduce_check(const double* __restrict__ partial, int nblk, double* __restrict__ rsum,
                   int* __restrict__ sexp_prev, const double* __restrict__ fsum, int B,
                   const double* __restrict__ ctl, int* __restrict__ active,
                   double* __restrict__ relres, int* __restrict__ sexp, int* __restrict__ state,
                   int inc, cudaGraphConditionalHandle h, int set_cond) {
  pdl_wait();
  __shared__ double sh[kThreads];
  for (int b = 0; b < B; ++b) {
    const double r = block_sum_partials(partial, nblk, B, b, sh);
    if (threadIdx.x == 0) rsum[b] = r;
  }
  if (sexp_prev)
    for (int b = threadIdx.x; b < B; b += blockDim.x) sexp_prev[b] = sexp[b];
  __syncthreads();
  check_block(rsum, fsum, B, ctl, active, relres, sexp, state, inc, h, set_cond);
}

// u += 2^sexp[b] * c for the right-hand sides still active (refinement update).
__global__ void __launch_bounds__(kThreads) k_refine_update(double* __restrict__ u,
                                                            const float* __restrict__ c,
                                                            const int* __restrict__ sexp,
                                                            const int* __restrict__ active, int n,
                                                            int B, int* __restrict__ iters) {
  pdl_wait();
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < (size_t)B && active[t]) iters[t] += 1;
  if (t >= (size_t)n * B) return;
  const int b = (int)(t % B);
  if (active[b]) u[t] += scale2((double)c[t], sexp[b]);
}

// u <- w for the right-hand sides still active (plain solve, B > 1).
__global__ void __launch_bounds__(kThreads) k_masked_copy(double* __restrict__ u,
                                                          const double* __restrict__ w,
                                                          const int* __restrict__ active, int n,
                                                          int B, int* __restrict__ iters) {
  pdl_wait();
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < (size_t)B && active[t]) iters[t] += 1;
  if (t >= (size_t)n * B) return;
  if (active[t % B]) u[t] = w[t];
}

}  // namespace mgk
