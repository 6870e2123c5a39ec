// Learnable multigrid with two features per node (d = 2).
//
// The paper's Helmholtz experiment (Sec. 4.2) solves a complex system and
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
// arguments, so mg2_set_params drops the captured graphs.  mg2_solve_fgmres
// wraps the cycle (or full multigrid) in restarted flexible GMRES on the
// equivalent real system of size 2n.
#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include <cstdint>
#include <cstring>

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

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch() { asm volatile("griddepcontrol.launch_dependents;"); }

// BV consecutive complex values x[off .. off+BV) (Pair<T> = (Re, Im)): one
// 32-byte access where BV pairs are 32 bytes and the address is 32-byte
// aligned (ld.global.v8.b32), else pair by pair.  kA: -1 tests each
// address; 1 or 0 is a launch-wide answer (pairs_aligned), so an access
// carries no alignment branch.
template <class T, int BV, int kA = -1>
__device__ __forceinline__ void ld_pairs(const typename Pair<T>::type* __restrict__ x, size_t off,
                                         typename Pair<T>::type (&out)[BV]) {
  const typename Pair<T>::type* p = x + off;
  if constexpr (BV * sizeof(typename Pair<T>::type) == 32 && kA != 0) {
    if (kA == 1 || ((uintptr_t)p & 31) == 0) {
      uint32_t w[8];
      asm("ld.global.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
          : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
            "=r"(w[7])
          : "l"(p));
      memcpy(out, w, 32);
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < BV; ++j) out[j] = p[j];
}

template <class T, int BV, int kA = -1>
__device__ __forceinline__ void st_pairs(typename Pair<T>::type* __restrict__ x, size_t off,
                                         const typename Pair<T>::type (&in)[BV]) {
  typename Pair<T>::type* p = x + off;
  if constexpr (BV * sizeof(typename Pair<T>::type) == 32 && kA != 0) {
    if (kA == 1 || ((uintptr_t)p & 31) == 0) {
      uint32_t w[8];
      memcpy(w, in, 32);
      asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(w[0]),
                   "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                   : "memory");
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < BV; ++j) p[j] = in[j];
}

// Thread layout of the cycle kernels: thread g owns row i = g / (B / BV) and
// the BV consecutive right-hand sides b0.. (BV | B); the B / BV threads of a
// row are adjacent lanes, so a warp reads whole runs of a neighbour's values
// and a row's matrix entries once per BV columns.  For every (row, rhs) the
// arithmetic is the same as with BV = 1.  Every kernel waits on its
// predecessor (griddepcontrol.wait) before touching memory, so it may be
// launched with programmatic dependent launch.
#define MG2_PROLOGUE(NROWS)                              \
  pdl_wait();                                             \
  pdl_launch();                                           \
  const int nq = B / BV;                                  \
  const int g = blockIdx.x * blockDim.x + threadIdx.x;    \
  const int i = g / nq;                                   \
  if (i >= (NROWS)) return;                               \
  const int b0 = (g - i * nq) * BV;

// Whether every [n][B] complex access of a launch is 32-byte aligned (the
// vectors' bases and the row pitch B * sizeof(pair); a thread's column
// offset is a multiple of the 32-byte tile).  The grid kernels run their
// element step with that launch-wide answer in FP32 (the form measured on
// the real-valued path's multi-rhs kernels) and with a test per access in
// FP64.
template <class T>
__device__ __forceinline__ bool pairs_aligned(int B, const void* a, const void* b,
                                              const void* c = nullptr) {
  return ((size_t)B * sizeof(typename Pair<T>::type)) % 32 == 0 &&
         ((((uintptr_t)a) | ((uintptr_t)b) | ((uintptr_t)c)) & 31) == 0;
}
#define MG2_DISPATCH(AL, CALL)          \
  if constexpr (sizeof(T) != 4) {       \
    CALL(-1);                           \
  } else if (AL) {                      \
    CALL(1);                            \
  } else {                              \
    CALL(0);                            \
  }

// ---- element steps: row i, right-hand sides b0 .. b0 + BV - 1 ----------
// (the grid kernels below and the single-block small-levels kernel k2_tail
// run the same functions, so every launch form rounds alike)

// out = f - A u (u_zero: u = 0), then optionally out = theta * out / A_ii
// (dinv = 1 / A_ii, complex)
template <class T, int BV, int kA = -1>
__device__ __forceinline__ void res2_el(int i, int b0, const int* __restrict__ rp,
                                        const int* __restrict__ ci,
                                        const typename Pair<T>::type* __restrict__ av,
                                        const typename Pair<T>::type* __restrict__ f,
                                        const typename Pair<T>::type* __restrict__ u,
                                        typename Pair<T>::type* __restrict__ out, int B,
                                        const typename Pair<T>::type* __restrict__ dinv, T theta,
                                        int scale, int u_zero) {
  using P2 = typename Pair<T>::type;
  const size_t base = (size_t)i * B + b0;
  P2 r[BV];
  ld_pairs<T, BV, kA>(f, base, r);
  if (!u_zero) {
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const P2 a = av[e];
      P2 x[BV];
      ld_pairs<T, BV, kA>(u, (size_t)ci[e] * B + b0, x);
#pragma unroll
      for (int j = 0; j < BV; ++j) {
        r[j].x -= a.x * x[j].x - a.y * x[j].y;
        r[j].y -= a.x * x[j].y + a.y * x[j].x;
      }
    }
  }
  if (scale) {
    const P2 d = dinv[i];
#pragma unroll
    for (int j = 0; j < BV; ++j) {
      const T re = r[j].x * d.x - r[j].y * d.y, im = r[j].x * d.y + r[j].y * d.x;
      r[j].x = theta * re;
      r[j].y = theta * im;
    }
  }
  st_pairs<T, BV, kA>(out, base, r);
}

// phi_i = W_1 x_i + W_2 inv_deg_i sum_{j != i in row i} x_j; mode 0: y = phi,
// 1: y += eta phi, 2: y += phi.  x and y are distinct buffers.
template <class T, int BV, int kA = -1>
__device__ __forceinline__ void conv2_el(int i, int b0, const int* __restrict__ rp,
                                         const int* __restrict__ ci, const T* __restrict__ invdeg,
                                         const typename Pair<T>::type* __restrict__ x,
                                         typename Pair<T>::type* __restrict__ y, int B,
                                         const Conv2<T>& w, T eta, int mode) {
  using P2 = typename Pair<T>::type;
  const size_t base = (size_t)i * B + b0;
  T sx[BV], sy[BV];
#pragma unroll
  for (int j = 0; j < BV; ++j) sx[j] = sy[j] = T(0);
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const int c = ci[e];
    if (c == i) continue;
    P2 v[BV];
    ld_pairs<T, BV, kA>(x, (size_t)c * B + b0, v);
#pragma unroll
    for (int j = 0; j < BV; ++j) {
      sx[j] += v[j].x;
      sy[j] += v[j].y;
    }
  }
  const T id = invdeg[i];
  P2 xi[BV], o[BV];
  ld_pairs<T, BV, kA>(x, base, xi);
  if (mode != 0) ld_pairs<T, BV, kA>(y, base, o);
#pragma unroll
  for (int j = 0; j < BV; ++j) {
    const T mx = id * sx[j], my = id * sy[j];
    P2 phi;
    phi.x = w.w[0][0][0] * xi[j].x + w.w[0][0][1] * xi[j].y + (w.w[1][0][0] * mx + w.w[1][0][1] * my);
    phi.y = w.w[0][1][0] * xi[j].x + w.w[0][1][1] * xi[j].y + (w.w[1][1][0] * mx + w.w[1][1][1] * my);
    if (mode == 0) {
      o[j] = phi;
    } else {
      const T s = mode == 1 ? eta : T(1);
      o[j].x += s * phi.x;
      o[j].y += s * phi.y;
    }
  }
  st_pairs<T, BV, kA>(y, base, o);
}

// y = M x for a real CSR matrix M on complex vectors
template <class T, int BV, int kA = -1>
__device__ __forceinline__ void spmv2_el(int i, int b0, const int* __restrict__ rp,
                                         const int* __restrict__ ci, const T* __restrict__ mv,
                                         const typename Pair<T>::type* __restrict__ x,
                                         typename Pair<T>::type* __restrict__ y, int B) {
  using P2 = typename Pair<T>::type;
  P2 o[BV];
#pragma unroll
  for (int j = 0; j < BV; ++j) o[j].x = o[j].y = T(0);
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const T m = mv[e];
    P2 v[BV];
    ld_pairs<T, BV, kA>(x, (size_t)ci[e] * B + b0, v);
#pragma unroll
    for (int j = 0; j < BV; ++j) {
      o[j].x += m * v[j].x;
      o[j].y += m * v[j].y;
    }
  }
  st_pairs<T, BV, kA>(y, (size_t)i * B + b0, o);
}

// e = A_J^{-1} r with the dense inverse (row-major, complex) for row i,
// right-hand sides b0..: called by the 32 lanes of a warp; lane l sums the
// products of columns l, l + 32, ... in order, then the lanes' sums are added
// by a fixed butterfly and lane 0 stores.  The order of every (row, rhs) sum
// does not depend on BV.
template <class T, int BV>
__device__ __forceinline__ void dense2_warp(int i, int b0, int lane, int n,
                                            const typename Pair<T>::type* __restrict__ inv,
                                            const typename Pair<T>::type* __restrict__ r,
                                            typename Pair<T>::type* __restrict__ e, int B) {
  using P2 = typename Pair<T>::type;
  T sx[BV], sy[BV];
#pragma unroll
  for (int j = 0; j < BV; ++j) sx[j] = sy[j] = T(0);
  for (int k = lane; k < n; k += 32) {
    const P2 a = inv[(size_t)i * n + k];
    P2 v[BV];
    ld_pairs<T, BV>(r, (size_t)k * B + b0, v);
#pragma unroll
    for (int j = 0; j < BV; ++j) {
      sx[j] += a.x * v[j].x - a.y * v[j].y;
      sy[j] += a.x * v[j].y + a.y * v[j].x;
    }
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1)
#pragma unroll
    for (int j = 0; j < BV; ++j) {
      sx[j] += __shfl_xor_sync(0xffffffffu, sx[j], m);
      sy[j] += __shfl_xor_sync(0xffffffffu, sy[j], m);
    }
  if (lane == 0) {
    P2 o[BV];
#pragma unroll
    for (int j = 0; j < BV; ++j) {
      o[j].x = sx[j];
      o[j].y = sy[j];
    }
    st_pairs<T, BV>(e, (size_t)i * B + b0, o);
  }
}

// ---- grid kernels ---------------------------------------------------------
template <class T, int BV>
__global__ void __launch_bounds__(kF2Threads)
    k2_residual(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                const typename Pair<T>::type* __restrict__ av,
                const typename Pair<T>::type* __restrict__ f,
                const typename Pair<T>::type* __restrict__ u, typename Pair<T>::type* __restrict__ out,
                int B, const typename Pair<T>::type* __restrict__ dinv, T theta, int scale,
                int u_zero) {
  MG2_PROLOGUE(n)
#define MG2_CALL(A) res2_el<T, BV, A>(i, b0, rp, ci, av, f, u, out, B, dinv, theta, scale, u_zero)
  MG2_DISPATCH(pairs_aligned<T>(B, f, u, out), MG2_CALL)
#undef MG2_CALL
}

template <class T, int BV>
__global__ void __launch_bounds__(kF2Threads)
    k2_conv(int n, const int* __restrict__ rp, const int* __restrict__ ci,
            const T* __restrict__ invdeg, const typename Pair<T>::type* __restrict__ x,
            typename Pair<T>::type* __restrict__ y, int B, Conv2<T> w, T eta, int mode) {
  MG2_PROLOGUE(n)
#define MG2_CALL(A) conv2_el<T, BV, A>(i, b0, rp, ci, invdeg, x, y, B, w, eta, mode)
  MG2_DISPATCH(pairs_aligned<T>(B, x, y), MG2_CALL)
#undef MG2_CALL
}

template <class T, int BV>
__global__ void __launch_bounds__(kF2Threads)
    k2_spmv_real(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                 const T* __restrict__ mv, const typename Pair<T>::type* __restrict__ x,
                 typename Pair<T>::type* __restrict__ y, int B) {
  MG2_PROLOGUE(n)
#define MG2_CALL(A) spmv2_el<T, BV, A>(i, b0, rp, ci, mv, x, y, B)
  MG2_DISPATCH(pairs_aligned<T>(B, x, y), MG2_CALL)
#undef MG2_CALL
}

// one warp per (row, tile of BV right-hand sides)
template <class T, int BV>
__global__ void __launch_bounds__(kF2Threads)
    k2_dense(int n, const typename Pair<T>::type* __restrict__ inv,
             const typename Pair<T>::type* __restrict__ r, typename Pair<T>::type* __restrict__ e,
             int B) {
  pdl_wait();
  pdl_launch();
  const int nq = B / BV;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int i = w / nq;
  if (i >= n) return;
  dense2_warp<T, BV>(i, (w - i * nq) * BV, lane, n, inv, r, e, B);
}

// ---- single-block small levels ---------------------------------------------
// Levels lt .. J-2 of a cycle (rows x rhs at most the tail threshold on
// level lt) in one block of kT2Threads threads, steps separated by block
// barriers, in two launches around the coarsest product: the descent
// (smoothing, restriction, down to f_J) and, after the grid kernel of the
// dense coarsest product (a warp per output over many SMs: on one SM its
// FP64 products took longer than the launches it saved), the ascent.  The
// same element steps as the grid kernels (one rhs per thread step).
// Operator arrays stay in global memory (L2).  Slot k holds level lt + k.
constexpr int kT2Max = 8;
constexpr int kT2Threads = 1024;

template <class T>
struct Tail2 {
  using P2 = typename Pair<T>::type;
  int lt, J, B, nu_pre, nu_post, nJ;
  int ascent;  // 0: the descent to f_J, 1: the ascent from u_J
  int n[kT2Max];
  const int *rp[kT2Max], *ci[kT2Max], *prp[kT2Max], *pci[kT2Max], *trp[kT2Max], *tci[kT2Max];
  const P2 *av[kT2Max], *dinv[kT2Max];
  const T *invdeg[kT2Max], *pv[kT2Max], *tv[kT2Max];
  const P2* f[kT2Max];
  P2 *u[kT2Max], *t[kT2Max], *t2[kT2Max];
  T theta[kT2Max], eta[kT2Max];
  Conv2<T> wb[kT2Max], wr[kT2Max], wp[kT2Max];
  const P2* cinv;
};

template <class T>
__global__ void __launch_bounds__(kT2Threads) k2_tail(Tail2<T> a) {
  using P2 = typename Pair<T>::type;
  pdl_wait();
  pdl_launch();
  const int B = a.B;
  // fn(i, b) for every (row, rhs) of a level, then a block barrier
  auto each = [&](int n, auto&& fn) {
    for (int e = threadIdx.x; e < n * B; e += blockDim.x) fn(e / B, e - (e / B) * B);
    __syncthreads();
  };
  auto smooth = [&](int k, int nu) {
    for (int q = 0; q < nu; ++q) {
      each(a.n[k], [&](int i, int b) {
        res2_el<T, 1>(i, b, a.rp[k], a.ci[k], a.av[k], a.f[k], a.u[k], a.t[k], B, a.dinv[k],
                      a.theta[k], 1, 0);
      });
      each(a.n[k], [&](int i, int b) {
        conv2_el<T, 1>(i, b, a.rp[k], a.ci[k], a.invdeg[k], a.t[k], a.u[k], B, a.wb[k],
                       a.eta[k], 1);
      });
    }
  };
  const int kJ = a.J - 1 - a.lt;
  if (a.ascent) {
    for (int k = kJ - 1; k >= 0; --k) {
      each(a.n[k], [&](int i, int b) {
        spmv2_el<T, 1>(i, b, a.prp[k], a.pci[k], a.pv[k], a.u[k + 1], a.t[k], B);
      });
      each(a.n[k], [&](int i, int b) {
        conv2_el<T, 1>(i, b, a.rp[k], a.ci[k], a.invdeg[k], a.t[k], a.u[k], B, a.wp[k], T(1),
                       2);
      });
      smooth(k, a.nu_post);
    }
    return;
  }
  for (int k = 0; k < kJ; ++k) {
    smooth(k, a.nu_pre);
    each(a.n[k], [&](int i, int b) {
      res2_el<T, 1>(i, b, a.rp[k], a.ci[k], a.av[k], a.f[k], a.u[k], a.t[k], B, a.dinv[k],
                    a.theta[k], 0, 0);
    });
    each(a.n[k], [&](int i, int b) {
      conv2_el<T, 1>(i, b, a.rp[k], a.ci[k], a.invdeg[k], a.t[k], a.t2[k], B, a.wr[k], T(1), 0);
    });
    each(a.n[k + 1], [&](int i, int b) {
      spmv2_el<T, 1>(i, b, a.trp[k], a.tci[k], a.tv[k], a.t2[k], (P2*)a.f[k + 1], B);
      P2 z;
      z.x = z.y = T(0);
      a.u[k + 1][(size_t)i * B + b] = z;
    });
  }
}

dim3 grid_of(size_t work) { return dim3((unsigned)((work + kF2Threads - 1) / kF2Threads)); }

// ---- FGMRES on the real form (FP64 vectors, double2 = (Re, Im)) ----------
// A right-hand side's vectors are real 2n vectors [Re; Im]; inner products
// are sum_i Re x_i Re y_i + Im x_i Im y_i.  Each (vector, rhs) sum is one
// block over the rows in a fixed order, so results do not depend on B.

// w = A z (complex CSR, FP64)
__global__ void __launch_bounds__(kF2Threads)
    k2g_apply(int n, const int* __restrict__ rp, const int* __restrict__ ci,
              const double2* __restrict__ av, const double2* __restrict__ z,
              double2* __restrict__ w, int B) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * B) return;
  const int i = (int)(t / B), b = (int)(t - (size_t)i * B);
  double sx = 0.0, sy = 0.0;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const double2 a = av[e];
    const double2 x = z[(size_t)ci[e] * B + b];
    sx += a.x * x.x - a.y * x.y;
    sy += a.x * x.y + a.y * x.x;
  }
  w[t] = make_double2(sx, sy);
}

// out[q * B + b] = <V_q, w>_b for block (q, b); V_q = V + q * vstride
// (w = nullptr: <V_q, V_q>)
__global__ void __launch_bounds__(kF2Threads)
    k2g_dots(const double2* __restrict__ V, size_t vstride, const double2* __restrict__ w,
             int n, int B, double* __restrict__ out) {
  __shared__ double sh[kF2Threads];
  const int q = blockIdx.x, b = blockIdx.y;
  const double2* x = V + (size_t)q * vstride;
  const double2* y = w ? w : x;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 a = x[(size_t)i * B + b], c = y[(size_t)i * B + b];
    s += a.x * c.x + a.y * c.y;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k >= 1; k >>= 1) {
    if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[(size_t)q * B + b] = sh[0];
}

// w -= sum_{q < nq} h[q * B + b] V_q
__global__ void __launch_bounds__(kF2Threads)
    k2g_orth(const double2* __restrict__ V, size_t vstride, double2* __restrict__ w,
             const double* __restrict__ h, int nq, int n, int B) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * B) return;
  const int b = (int)(t % B);
  double2 o = w[t];
  for (int q = 0; q < nq; ++q) {
    const double hq = h[(size_t)q * B + b];
    const double2 v = V[(size_t)q * vstride + t];
    o.x -= hq * v.x;
    o.y -= hq * v.y;
  }
  w[t] = o;
}

// v = w * inv[b]
__global__ void __launch_bounds__(kF2Threads)
    k2g_scale(const double2* w, const double* __restrict__ inv, double2* v, int n, int B) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * B) return;
  const double s = inv[t % B];
  const double2 x = w[t];
  v[t] = make_double2(x.x * s, x.y * s);
}

// u += sum_{q < nq} y_q Z_q for the active right-hand sides
__global__ void __launch_bounds__(kF2Threads)
    k2g_update(double2* __restrict__ u, const double2* __restrict__ Z, size_t vstride,
               const double* __restrict__ y, int ystride, int nq, const int* __restrict__ active,
               int n, int B) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * B) return;
  const int b = (int)(t % B);
  if (!active[b]) return;
  const double* yb = y + (size_t)b * ystride;
  double2 o = u[t];
  for (int q = 0; q < nq; ++q) {
    const double2 z = Z[(size_t)q * vstride + t];
    o.x += yb[q] * z.x;
    o.y += yb[q] * z.y;
  }
  u[t] = o;
}

// FP64 <-> context precision copies of level-0 vectors
template <class T>
__global__ void __launch_bounds__(kF2Threads)
    k2g_convert(const void* __restrict__ x, void* __restrict__ y, size_t N, int to_ctx) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  using P2 = typename Pair<T>::type;
  if (to_ctx) {
    const double2 v = ((const double2*)x)[t];
    P2 o;
    o.x = (T)v.x;
    o.y = (T)v.y;
    ((P2*)y)[t] = o;
  } else {
    const P2 v = ((const P2*)x)[t];
    ((double2*)y)[t] = make_double2((double)v.x, (double)v.y);
  }
}

// Per right-hand side b, small[b * stride]: H (m+1) x m (column j at
// j (m+1)), cs[m], sn[m], g[m+1], y[m].
__host__ __device__ inline int k2g_stride(int m) { return m * (m + 1) + 4 * m + 1; }

// Restart: beta = ||r||, relres, the active set, g = beta e_1, inv = 1/beta,
// done = 0; state[0] = active count, state[1] = 1 if non-finite.  One block.
__global__ void k2g_restart(const double* __restrict__ rsum, const double* __restrict__ fsum,
                            double tol, int m, int B, int* __restrict__ active,
                            double* __restrict__ relres, double* __restrict__ small,
                            double* __restrict__ inv, int* __restrict__ done,
                            int* __restrict__ state) {
  __shared__ int cnt, bad;
  if (threadIdx.x == 0) {
    cnt = 0;
    bad = 0;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const double beta = sqrt(rsum[b]), fn = sqrt(fsum[b]);
    const double rel = fn > 0.0 ? beta / fn : beta;
    relres[b] = rel;
    if (!isfinite(rel)) atomicAdd(&bad, 1);
    if (active[b] && !(rel < tol) && isfinite(rel))
      atomicAdd(&cnt, 1);
    else
      active[b] = 0;
    double* g = small + (size_t)b * k2g_stride(m) + m * (m + 1) + 2 * m;
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    inv[b] = beta > 0.0 && isfinite(beta) ? 1.0 / beta : 0.0;
    done[b] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    state[0] = cnt;
    state[1] = bad;
  }
}

// Arnoldi step j: H column j = h1 + h2 and ||w||, rotations, the estimate;
// a right-hand side in its cycle counts the step and finishes it (done =
// j + 1) when the estimate meets tol or is not finite.  state[3] = right-hand
// sides still in their cycle.  One block.
__global__ void k2g_arnoldi(double* __restrict__ small, const double* __restrict__ h1,
                            const double* __restrict__ h2, const double* __restrict__ wn,
                            const double* __restrict__ fsum, double tol, int m, int j, int B,
                            const int* __restrict__ active, int* __restrict__ iters,
                            double* __restrict__ inv, double* __restrict__ relres,
                            int* __restrict__ done, int* __restrict__ state) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    double* sb = small + (size_t)b * k2g_stride(m);
    double* cs = sb + m * (m + 1);
    double* sn = cs + m;
    double* g = sn + m;
    double* Hj = sb + (size_t)j * (m + 1);
    for (int i = 0; i <= j; ++i) Hj[i] = h1[(size_t)i * B + b] + h2[(size_t)i * B + b];
    const double hn = sqrt(wn[b]);
    Hj[j + 1] = hn;
    inv[b] = hn > 0.0 && isfinite(hn) ? 1.0 / hn : 0.0;
    for (int i = 0; i < j; ++i) {
      const double t = cs[i] * Hj[i] + sn[i] * Hj[i + 1];
      Hj[i + 1] = -sn[i] * Hj[i] + cs[i] * Hj[i + 1];
      Hj[i] = t;
    }
    const double a = Hj[j], c2 = Hj[j + 1];
    const double r = sqrt(a * a + c2 * c2);
    cs[j] = r > 0.0 ? a / r : 1.0;
    sn[j] = r > 0.0 ? c2 / r : 0.0;
    Hj[j] = r;
    Hj[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    if (active[b] && !done[b]) {
      const double fn = sqrt(fsum[b]);
      const double est = fn > 0.0 ? fabs(g[j + 1]) / fn : fabs(g[j + 1]);
      iters[b] += 1;
      relres[b] = est;
      if (est < tol || !isfinite(est))
        done[b] = j + 1;
      else
        atomicAdd(&cnt, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) state[3] = cnt;
}

// y = H^{-1} g over the columns each right-hand side used; y = 0 beyond.
__global__ void k2g_solve_y(double* __restrict__ small, int m, int jl, int B,
                            const int* __restrict__ active, const int* __restrict__ done) {
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    if (!active[b]) continue;
    double* sb = small + (size_t)b * k2g_stride(m);
    const double* g = sb + m * (m + 1) + 2 * m;
    double* y = sb + m * (m + 1) + 3 * m + 1;
    const int jb = done[b] ? min(done[b] - 1, jl) : jl;
    for (int i = jl; i > jb; --i) y[i] = 0.0;
    for (int i = jb; i >= 0; --i) {
      double t = g[i];
      for (int k = i + 1; k <= jb; ++k) t -= sb[(size_t)k * (m + 1) + i] * y[k];
      const double d = sb[(size_t)i * (m + 1) + i];
      y[i] = d != 0.0 ? t / d : 0.0;
    }
  }
}

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
  int opt_pdl = 1;   // programmatic dependent launch between the cycle's kernels
  int opt_tile = 1;  // right-hand-side tiles of the cycle's kernels (0: one per thread)
  // levels with rows x rhs at most this (and all coarser) run in k2_tail
  // (0: never, the default: measured no faster in FP32 and slower in FP64,
  // where one SM's FP64 pipe carries the small levels' complex products)
  int64_t opt_tail_work = 0;
  // mg2_vcycle_profile: (kind, level, start, end) per launch while set
  std::vector<std::tuple<int, int, cudaEvent_t, cudaEvent_t>>* prof = nullptr;
  std::vector<void*> owned;
  cudaStream_t cap = nullptr;  // capture stream
  // FGMRES (mg2_solve_fgmres): the FP64 level-0 operator, and the workspace
  // for restart length gm_m (allocated on first use)
  void* av64 = nullptr;  // double2, level 0 (= lev[0].av in FP64 contexts)
  int gm_m = 0;
  double *gmV = nullptr, *gmZ = nullptr, *gmR = nullptr, *gmSmall = nullptr, *gmH = nullptr;
  double* gmVec = nullptr;  // fsum, rsum, wn, inv, relres: 5 * maxB
  int* gmInt = nullptr;     // active, iters, done: 3 * maxB; state: 4
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
mg_status setup_typed(mg2_ctx* c, const mg2_level* L,
                      const std::vector<std::complex<double>>& inv) {
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
      const std::complex<double> di = 1.0 / diag;  // nonzero: checked in mg2_setup
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
  // the level-0 operator in FP64 for FGMRES's outer products
  if (sizeof(T) == sizeof(double)) {
    c->av64 = c->lev[0].av;
  } else {
    std::vector<double> a64(2 * (size_t)c->lev[0].nnz);
    std::copy(L[0].A_vals, L[0].A_vals + a64.size(), a64.begin());
    if (!upload(c, &c->av64, a64.data(), a64.size()))
      return fail("mg2_setup: device allocation or copy failed", MG_ERR_CUDA);
  }
  // the coarsest operator's inverse (computed on the host by mg2_setup)
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

// Launches of the cycle kernels: right-hand-side tiles of BV columns (the
// widest of 4 (FP32) or 2 (FP64) complex values, 32 bytes, that divides B;
// 1 with tiling off) and programmatic dependent launch (option).
template <class T>
struct Launch2 {
  mg2_ctx* c;
  cudaStream_t s;
  int B;
  int bv() const {
    if (!c->opt_tile) return 1;
    for (int v = sizeof(T) == 4 ? 4 : 2; v > 1; v /= 2)
      if (B % v == 0) return v;
    return 1;
  }
  template <class... KArgs, class... Args>
  void go(int kind, int lev, void (*k)(KArgs...), int n, Args... args) const {
    if (c->prof) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, s);
      c->prof->emplace_back(kind, lev, a, b);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid_of((size_t)n * (B / bv()));
    cfg.blockDim = dim3(kF2Threads);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = c->opt_pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k, args...);
    if (c->prof) cudaEventRecord(std::get<3>(c->prof->back()), s);
  }
  // f(std::integral_constant<int, BV>) for this launch's tile width
  template <class F>
  void with_bv(F&& f) const {
    const int v = bv();
    if constexpr (sizeof(T) == 4) {
      if (v == 4) return f(std::integral_constant<int, 4>{});
    }
    if (v == 2) return f(std::integral_constant<int, 2>{});
    f(std::integral_constant<int, 1>{});
  }
  using P2 = typename Pair<T>::type;
  // profile kinds (mg_kernel_kind): the smoothing residual, the smoothing
  // conv, the restriction's residual and Phi_R, the P^T gather, P e_c, the
  // prolongation's Phi_P and the coarsest product
  void residual(int lev, const mg2_ctx::Lev& L, const P2* f, const P2* u, P2* out, T theta,
                int scale, int u_zero) const {
    with_bv([&](auto V) {
      go(scale ? MG_K_RESIDUAL_SCALED : MG_K_RESIDUAL, lev, k2_residual<T, decltype(V)::value>,
         L.n, L.n, (const int*)L.rp, (const int*)L.ci, (const P2*)L.av, f, u, out, B,
         (const P2*)L.dinv, theta, scale, u_zero);
    });
  }
  void conv(int lev, const mg2_ctx::Lev& L, const P2* x, P2* y, Conv2<T> w, T eta,
            int mode) const {
    const int kind = mode == 1 ? MG_K_CONV_UPDATE : mode == 0 ? MG_K_CONV_R : MG_K_PROLONG;
    with_bv([&](auto V) {
      go(kind, lev, k2_conv<T, decltype(V)::value>, L.n, L.n, (const int*)L.rp,
         (const int*)L.ci, (const T*)L.invdeg, x, y, B, w, eta, mode);
    });
  }
  void spmv(int kind, int lev, int n, const int* rp, const int* ci, const void* mv, const P2* x,
            P2* y) const {
    with_bv([&](auto V) {
      go(kind, lev, k2_spmv_real<T, decltype(V)::value>, n, n, rp, ci, (const T*)mv, x, y, B);
    });
  }
  // first level the single-block kernel runs for this batch (J - 1: none;
  // it needs a level above the coarsest)
  int tail_level() const {
    const int J = c->J;
    if (c->opt_tail_work <= 0 || J < 2) return J - 1;
    int lt = J - 1;
    while (lt > 0 && (int64_t)c->lev[lt - 1].n * B <= c->opt_tail_work) --lt;
    if (lt == J - 1 || J - lt > kT2Max) return J - 1;
    return lt;
  }
  // the descent (ascent = 0) or ascent (1) of the cycle from level l
  // (>= tail_level()) on (f, u), in one block
  void tail(int l, const P2* f, P2* u, int ascent) const {
    Tail2<T> a;
    std::memset(&a, 0, sizeof(a));
    a.lt = l;
    a.ascent = ascent;
    a.J = c->J;
    a.B = B;
    a.nu_pre = c->nu_pre;
    a.nu_post = c->nu_post;
    a.nJ = c->lev[c->J - 1].n;
    a.cinv = (const P2*)c->cinv;
    for (int lv = l; lv < c->J; ++lv) {
      const int k = lv - l;
      const mg2_ctx::Lev& L = c->lev[lv];
      a.n[k] = L.n;
      a.rp[k] = L.rp;
      a.ci[k] = L.ci;
      a.av[k] = (const P2*)L.av;
      a.dinv[k] = (const P2*)L.dinv;
      a.invdeg[k] = (const T*)L.invdeg;
      a.prp[k] = L.prp;
      a.pci[k] = L.pci;
      a.pv[k] = (const T*)L.pv;
      a.trp[k] = L.trp;
      a.tci[k] = L.tci;
      a.tv[k] = (const T*)L.tv;
      a.f[k] = k == 0 ? f : (const P2*)L.f;
      a.u[k] = k == 0 ? u : (P2*)L.u;
      a.t[k] = (P2*)L.t;
      a.t2[k] = (P2*)L.t2;
      if (lv < c->J - 1) {
        a.theta[k] = (T)c->theta[lv];
        a.eta[k] = (T)c->eta[lv];
        a.wb[k] = conv_of<T>(c->WB, lv);
        a.wr[k] = conv_of<T>(c->WR, lv);
        a.wp[k] = conv_of<T>(c->WP, lv);
      }
    }
    if (c->prof) {
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, s);
      c->prof->emplace_back(MG_K_TAIL, l, e0, e1);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(kT2Threads);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = c->opt_pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k2_tail<T>, a);
    if (c->prof) cudaEventRecord(std::get<3>(c->prof->back()), s);
  }
  void dense(int lev, int n, const P2* r, P2* e) const {
    // one warp per (row, tile): 32 threads per output
    with_bv([&](auto V) {
      go(MG_K_COARSE_CHOL, lev, k2_dense<T, decltype(V)::value>, 32 * n, n, (const P2*)c->cinv,
         r, e, B);
    });
  }
};

// Algorithm 2 on level l with two-feature convolutions.
template <class T>
void cycle(mg2_ctx* c, int l, const typename Pair<T>::type* f, typename Pair<T>::type* u, int B,
           cudaStream_t s) {
  using P2 = typename Pair<T>::type;
  const Launch2<T> k{c, s, B};
  mg2_ctx::Lev& L = c->lev[l];
  if (l == c->J - 1) {
    k.dense(l, L.n, f, u);
    return;
  }
  if (l >= k.tail_level()) {  // this level and every coarser one in one block,
    k.tail(l, f, u, 0);        // in two launches around the coarsest product
    k.dense(c->J - 1, c->lev[c->J - 1].n, (const P2*)c->lev[c->J - 1].f,
            (P2*)c->lev[c->J - 1].u);
    k.tail(l, f, u, 1);
    return;
  }
  const T theta = (T)c->theta[l], eta = (T)c->eta[l];
  const Conv2<T> wb = conv_of<T>(c->WB, l), wr = conv_of<T>(c->WR, l), wp = conv_of<T>(c->WP, l);
  P2* t = (P2*)L.t;
  P2* t2 = (P2*)L.t2;
  auto smooth = [&](int nu) {
    for (int q = 0; q < nu; ++q) {
      k.residual(l, L, f, u, t, theta, 1, 0);
      k.conv(l, L, t, u, wb, eta, 1);
    }
  };
  smooth(c->nu_pre);
  k.residual(l, L, f, u, t, theta, 0, 0);
  k.conv(l, L, t, t2, wr, T(1), 0);
  mg2_ctx::Lev& C = c->lev[l + 1];
  k.spmv(MG_K_RESTRICT, l, C.n, L.trp, L.tci, L.tv, t2, (P2*)C.f);
  cudaMemsetAsync(C.u, 0, (size_t)C.n * B * sizeof(P2), s);
  cycle<T>(c, l + 1, (const P2*)C.f, (P2*)C.u, B, s);
  k.spmv(MG_K_PE, l, L.n, L.prp, L.pci, L.pv, (const P2*)C.u, t);
  k.conv(l, L, t, u, wp, T(1), 2);
  smooth(c->nu_post);
}

// Full multigrid with two-feature convolutions: f restricted to every level
// by P^T Phi_R, the coarsest level solved exactly, then on each finer level
// Phi_P(P u_{l+1}) (from a zero iterate) starts one cycle on that level.
// Levels below 0 use their own f / u buffers; a level's cycle reuses the
// buffers of the levels below it once their FMG values are consumed.
template <class T>
void fmg(mg2_ctx* c, const typename Pair<T>::type* f0, typename Pair<T>::type* u0, int B,
         cudaStream_t s) {
  using P2 = typename Pair<T>::type;
  const Launch2<T> k{c, s, B};
  const int J = c->J;
  for (int l = 0; l < J - 1; ++l) {
    mg2_ctx::Lev& L = c->lev[l];
    mg2_ctx::Lev& C = c->lev[l + 1];
    const P2* fl = l == 0 ? f0 : (const P2*)L.f;
    k.conv(l, L, fl, (P2*)L.t2, conv_of<T>(c->WR, l), T(1), 0);
    k.spmv(MG_K_RESTRICT, l, C.n, L.trp, L.tci, L.tv, (const P2*)L.t2, (P2*)C.f);
  }
  mg2_ctx::Lev& LJ = c->lev[J - 1];
  const P2* fJ = J == 1 ? f0 : (const P2*)LJ.f;
  P2* uJ = J == 1 ? u0 : (P2*)LJ.u;
  k.dense(J - 1, LJ.n, fJ, uJ);
  for (int l = J - 2; l >= 0; --l) {
    mg2_ctx::Lev& L = c->lev[l];
    mg2_ctx::Lev& C = c->lev[l + 1];
    const P2* fl = l == 0 ? f0 : (const P2*)L.f;
    P2* ul = l == 0 ? u0 : (P2*)L.u;
    k.spmv(MG_K_PE, l, L.n, L.prp, L.pci, L.pv, (const P2*)C.u, (P2*)L.t);
    k.conv(l, L, (const P2*)L.t, ul, conv_of<T>(c->WP, l), T(1), 0);
    cycle<T>(c, l, fl, ul, B, s);
  }
}

// z = M(v) for FP64 level-0 vectors: one cycle from zero (which = 0) or one
// FMG (1) in the context precision.
template <class T>
void precondition(mg2_ctx* c, int which, const double2* v, double2* z, int B, cudaStream_t s) {
  using P2 = typename Pair<T>::type;
  mg2_ctx::Lev& L0 = c->lev[0];
  const size_t N = (size_t)L0.n * B;
  const bool fp64 = sizeof(T) == sizeof(double);
  const P2* fin = fp64 ? (const P2*)v : (const P2*)L0.f;
  P2* uout = fp64 ? (P2*)z : (P2*)L0.u;
  if (!fp64) k2g_convert<T><<<grid_of(N), kF2Threads, 0, s>>>(v, L0.f, N, 1);
  if (which == 1) {
    fmg<T>(c, fin, uout, B, s);
  } else {
    cudaMemsetAsync(uout, 0, N * sizeof(P2), s);
    cycle<T>(c, 0, fin, uout, B, s);
  }
  if (!fp64) k2g_convert<T><<<grid_of(N), kF2Threads, 0, s>>>(L0.u, z, N, 0);
}

void free_gm(mg2_ctx* c) {
  for (void* p : {(void*)c->gmV, (void*)c->gmZ, (void*)c->gmR, (void*)c->gmSmall, (void*)c->gmH,
                  (void*)c->gmVec, (void*)c->gmInt})
    if (p) cudaFree(p);
  c->gmV = c->gmZ = c->gmR = c->gmSmall = c->gmH = c->gmVec = nullptr;
  c->gmInt = nullptr;
  c->gm_m = 0;
}

}  // namespace

extern "C" mg_status mg2_setup(mg2_ctx** out, int32_t J, const mg2_level* levels,
                               int32_t max_batch, int32_t precision) {
  std::lock_guard<std::recursive_mutex> lk(mgi::setup_mutex());
  if (!out) return fail("mg2_setup: out is NULL");
  *out = nullptr;
  // max_batch: FGMRES's per-(vector, rhs) sums run on a grid with nrhs rows
  if (J < 1 || J > 32 || !levels || max_batch < 1 || max_batch > 65535 ||
      (precision != 32 && precision != 64))
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
  // the host inverts the coarsest operator in O(n^3): keep it a coarse level
  if (levels[J - 1].n > 2048) return fail("mg2_setup: coarsest level larger than 2048 rows");
  // host checks before the first CUDA call: every diagonal nonzero (the
  // smoother divides by it), the coarsest operator invertible (FP64 dense
  // inverse by Gauss-Jordan)
  for (int l = 0; l < J; ++l) {
    const mg2_level& s = levels[l];
    for (int i = 0; i < s.n; ++i) {
      std::complex<double> diag = 0.0;
      for (int e = s.A_indptr[i]; e < s.A_indptr[i + 1]; ++e)
        if (s.A_indices[e] == i) diag += std::complex<double>(s.A_vals[2 * e], s.A_vals[2 * e + 1]);
      if (!(std::abs(diag) > 0.0))
        return fail("mg2_setup: zero diagonal on level " + std::to_string(l));
    }
  }
  std::vector<std::complex<double>> inv;
  {
    const mg2_level& s = levels[J - 1];
    const int n = s.n;
    std::vector<std::complex<double>> a((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
      for (int e = s.A_indptr[i]; e < s.A_indptr[i + 1]; ++e)
        a[(size_t)i * n + s.A_indices[e]] +=
            std::complex<double>(s.A_vals[2 * e], s.A_vals[2 * e + 1]);
    if (!invert(n, a, inv)) return fail("mg2_setup: coarsest operator is singular", MG_ERR_NOT_SPD);
  }
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
  const mg_status st =
      precision == 64 ? setup_typed<double>(c, levels, inv) : setup_typed<float>(c, levels, inv);
  if (st != MG_OK) {
    mg2_destroy(c);
    return st;
  }
  *out = c;
  return MG_OK;
}

extern "C" mg_status mg2_set_option(mg2_ctx* c, int32_t option, int64_t value) {
  if (!c) return fail("mg2_set_option: ctx is NULL");
  switch (option) {
    case MG_OPT_PDL:
      c->opt_pdl = value != 0;
      break;
    case MG_OPT_MULTI_RHS:
      if (value != 0 && value != 1) return fail("mg2_set_option: tile option must be 0 or 1");
      c->opt_tile = (int)value;
      break;
    case MG_OPT_TAIL_WORK:
      if (value < 0) return fail("mg2_set_option: tail work must be >= 0");
      c->opt_tail_work = value;
      break;
    default:
      return fail("mg2_set_option: unknown option");
  }
  c->drop_graphs();
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
    std::lock_guard<std::recursive_mutex> lk(mgi::setup_mutex());
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

extern "C" mg_status mg2_vcycle_profile(mg2_ctx* c, const void* f, void* u, int32_t nrhs,
                                        mg_kernel_time* out, int32_t max_out, int32_t* n_out,
                                        void* stream) {
  if (!c) return fail("mg2_vcycle_profile: ctx is NULL");
  if (!f || !u || f == u || nrhs < 1 || nrhs > c->maxB || !out || max_out < 0 || !n_out)
    return fail("mg2_vcycle_profile: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<std::tuple<int, int, cudaEvent_t, cudaEvent_t>> rec;
  c->prof = &rec;
  if (c->prec == 64)
    cycle<double>(c, 0, (const double2*)f, (double2*)u, nrhs, s);
  else
    cycle<float>(c, 0, (const float2*)f, (float2*)u, nrhs, s);
  c->prof = nullptr;
  cudaError_t e = cudaStreamSynchronize(s);
  int k = 0;
  for (auto& r : rec) {
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, std::get<2>(r), std::get<3>(r));
    if (k < max_out) {
      out[k].kernel = std::get<0>(r);
      out[k].level = std::get<1>(r);
      out[k].ms = ms;
      ++k;
    }
    cudaEventDestroy(std::get<2>(r));
    cudaEventDestroy(std::get<3>(r));
  }
  *n_out = k;
  if (e != cudaSuccess)
    return fail(std::string("mg2_vcycle_profile: ") + cudaGetErrorString(e), MG_ERR_CUDA);
  return MG_OK;
}

extern "C" mg_status mg2_solve_fgmres(mg2_ctx* c, const void* f, void* u, int32_t B, double tol,
                                      int32_t max_iter, int32_t restart, int32_t precond,
                                      int32_t* iters_out, double* relres_out, void* stream) {
  if (!c) return fail("mg2_solve_fgmres: ctx is NULL");
  if (!f || !u || f == u || B < 1 || B > c->maxB || !(tol > 0.0) || max_iter < 0 || restart < 1 ||
      restart > 64 || (precond != 0 && precond != 1))
    return fail("mg2_solve_fgmres: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const int m = restart;
  const int n0 = c->lev[0].n;
  const size_t N0 = (size_t)n0 * c->maxB;
  const size_t mb = (size_t)c->maxB;
  if (c->gm_m != m) {
    std::lock_guard<std::recursive_mutex> lk(mgi::setup_mutex());
    cudaDeviceSynchronize();
    free_gm(c);
    const bool ok =
        cudaMalloc(&c->gmV, (m + 1) * N0 * sizeof(double2)) == cudaSuccess &&
        cudaMalloc(&c->gmZ, m * N0 * sizeof(double2)) == cudaSuccess &&
        cudaMalloc(&c->gmR, N0 * sizeof(double2)) == cudaSuccess &&
        cudaMalloc(&c->gmSmall, mb * k2g_stride(m) * sizeof(double)) == cudaSuccess &&
        cudaMalloc(&c->gmH, 2 * (m + 1) * mb * sizeof(double)) == cudaSuccess &&
        cudaMalloc(&c->gmVec, 5 * mb * sizeof(double)) == cudaSuccess &&
        cudaMalloc(&c->gmInt, (3 * mb + 4) * sizeof(int)) == cudaSuccess;
    if (!ok) {
      free_gm(c);
      return fail("mg2_solve_fgmres: device allocation failed", MG_ERR_OOM);
    }
    c->gm_m = m;
  }
  const size_t vs = (size_t)n0 * B;  // stride between basis vectors (double2)
  double2* V = (double2*)c->gmV;
  double2* Z = (double2*)c->gmZ;
  double2* r = (double2*)c->gmR;
  double* h1 = c->gmH;
  double* h2 = c->gmH + (size_t)(m + 1) * B;
  double *fsum = c->gmVec, *rsum = c->gmVec + mb, *wn = c->gmVec + 2 * mb;
  double *inv = c->gmVec + 3 * mb, *relres = c->gmVec + 4 * mb;
  int *active = c->gmInt, *iters = c->gmInt + mb, *done = c->gmInt + 2 * mb;
  int* state = c->gmInt + 3 * mb;
  const mg2_ctx::Lev& L0 = c->lev[0];
  const dim3 g = grid_of(vs), gb(1, B);
  const double2* fd = (const double2*)f;
  double2* ud = (double2*)u;
  std::vector<int> ones(B, 1);
  int hs[4] = {0, 0, 0, 0};
  auto read_state = [&]() -> bool {
    return cudaMemcpyAsync(hs, state, sizeof(hs), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
           cudaStreamSynchronize(s) == cudaSuccess;
  };
  k2g_dots<<<gb, kF2Threads, 0, s>>>(fd, 0, nullptr, n0, B, fsum);
  cudaMemsetAsync(iters, 0, B * sizeof(int), s);
  cudaMemcpyAsync(active, ones.data(), B * sizeof(int), cudaMemcpyHostToDevice, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail("mg2_solve_fgmres: set-up failed", MG_ERR_CUDA);
  int total = 0;
  bool diverged = false;
  for (;;) {
    k2_residual<double, 1><<<g, kF2Threads, 0, s>>>(n0, L0.rp, L0.ci, (const double2*)c->av64, fd,
                                                 ud, r, B, (const double2*)nullptr, 0.0, 0, 0);
    k2g_dots<<<gb, kF2Threads, 0, s>>>(r, 0, nullptr, n0, B, rsum);
    k2g_restart<<<1, kF2Threads, 0, s>>>(rsum, fsum, tol, m, B, active, relres, c->gmSmall, inv,
                                         done, state);
    k2g_scale<<<g, kF2Threads, 0, s>>>(r, inv, V, n0, B);
    if (!read_state()) return fail("mg2_solve_fgmres: restart failed", MG_ERR_CUDA);
    if (hs[1]) {
      diverged = true;
      break;
    }
    if (hs[0] == 0 || total >= max_iter) break;
    int jl = -1;
    for (int j = 0; j < m && total < max_iter; ++j) {
      double2* Vj = V + (size_t)j * vs;
      double2* Vn = V + (size_t)(j + 1) * vs;
      double2* Zj = Z + (size_t)j * vs;
      if (c->prec == 64)
        precondition<double>(c, precond, Vj, Zj, B, s);
      else
        precondition<float>(c, precond, Vj, Zj, B, s);
      k2g_apply<<<g, kF2Threads, 0, s>>>(n0, L0.rp, L0.ci, (const double2*)c->av64, Zj, Vn, B);
      for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
        double* h = pass == 0 ? h1 : h2;
        k2g_dots<<<dim3(j + 1, B), kF2Threads, 0, s>>>(V, vs, Vn, n0, B, h);
        k2g_orth<<<g, kF2Threads, 0, s>>>(V, vs, Vn, h, j + 1, n0, B);
      }
      k2g_dots<<<gb, kF2Threads, 0, s>>>(Vn, 0, nullptr, n0, B, wn);
      k2g_arnoldi<<<1, kF2Threads, 0, s>>>(c->gmSmall, h1, h2, wn, fsum, tol, m, j, B, active,
                                           iters, inv, relres, done, state);
      k2g_scale<<<g, kF2Threads, 0, s>>>(Vn, inv, Vn, n0, B);
      ++total;
      jl = j;
      if (!read_state()) return fail("mg2_solve_fgmres: Arnoldi step failed", MG_ERR_CUDA);
      if (hs[3] == 0) break;
    }
    if (jl < 0) break;
    k2g_solve_y<<<1, kF2Threads, 0, s>>>(c->gmSmall, m, jl, B, active, done);
    k2g_update<<<g, kF2Threads, 0, s>>>(ud, Z, vs, c->gmSmall + m * (m + 1) + 3 * m + 1,
                                        k2g_stride(m), jl + 1, active, n0, B);
  }
  // the true residual of the final iterate
  k2_residual<double, 1><<<g, kF2Threads, 0, s>>>(n0, L0.rp, L0.ci, (const double2*)c->av64, fd, ud,
                                               r, B, (const double2*)nullptr, 0.0, 0, 0);
  k2g_dots<<<gb, kF2Threads, 0, s>>>(r, 0, nullptr, n0, B, rsum);
  std::vector<double> hr(B), hf(B);
  std::vector<int> hi(B);
  if (cudaMemcpyAsync(hr.data(), rsum, B * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(hf.data(), fsum, B * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(hi.data(), iters, B * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(std::string("mg2_solve_fgmres: ") + cudaGetErrorString(cudaGetLastError()),
                MG_ERR_CUDA);
  mg_status st = MG_OK;
  for (int b = 0; b < B; ++b) {
    const double rel = hf[b] > 0.0 ? std::sqrt(hr[b] / hf[b]) : std::sqrt(hr[b]);
    if (relres_out) relres_out[b] = rel;
    if (iters_out) iters_out[b] = hi[b];
    if (!(rel < tol)) st = MG_NOT_CONVERGED;
  }
  if (diverged) return fail("mg2_solve_fgmres: non-finite residual", MG_ERR_DIVERGED);
  if (st == MG_NOT_CONVERGED) mgi::set_global_error(st, "mg2_solve_fgmres: tolerance not met");
  return st;
}

extern "C" void mg2_destroy(mg2_ctx* c) {
  if (!c) return;
  std::lock_guard<std::recursive_mutex> lk(mgi::setup_mutex());
  cudaDeviceSynchronize();
  free_gm(c);
  c->drop_graphs();
  if (c->cap) cudaStreamDestroy(c->cap);
  for (void* p : c->owned)
    if (p) cudaFree(p);
  delete c;
}
