// Multi-right-hand-side forms of the level steps: one thread owns a row i
// and BV consecutive right-hand sides b0..b0+BV-1.  The B / BV threads of a
// row are adjacent lanes (b0 = (thread % (B / BV)) * BV), so a warp's 16-byte
// loads of a neighbour's values cover whole contiguous runs of X[n][B]
// rather than one piece of each of 32 rows.  The row's matrix entries are
// read once per BV columns.  For every (row, rhs) the arithmetic is the
// sequence of the scalar element functions in kernels.cuh, so results are
// identical to the one-thread-per-(row, rhs) form.
#pragma once

#include <cstring>
#include <type_traits>

#include "kernels.cuh"

namespace mgk {

// BV values of row r (offset r * B + b0), vectorised when 16-byte aligned:
// B * sizeof(T) and b0 * sizeof(T) are multiples of 16 whenever BV * sizeof(T)
// is (launches use BV | B).
template <class T, int BV>
__device__ __forceinline__ void ldv(const T* __restrict__ x, size_t off, T (&out)[BV]) {
  constexpr int W = 16 / (int)sizeof(T);
  if constexpr (BV % W == 0) {
    const uint4* q = reinterpret_cast<const uint4*>(x + off);
#pragma unroll
    for (int k = 0; k < BV / W; ++k) {
      const uint4 w = q[k];
      memcpy(&out[k * W], &w, 16);
    }
  } else {
#pragma unroll
    for (int b = 0; b < BV; ++b) out[b] = x[off + b];
  }
}

template <class T, int BV>
__device__ __forceinline__ void stv(T* __restrict__ x, size_t off, const T (&in)[BV]) {
  constexpr int W = 16 / (int)sizeof(T);
  if constexpr (BV % W == 0) {
    uint4* q = reinterpret_cast<uint4*>(x + off);
#pragma unroll
    for (int k = 0; k < BV / W; ++k) {
      uint4 w;
      memcpy(&w, &in[k * W], 16);
      q[k] = w;
    }
  } else {
#pragma unroll
    for (int b = 0; b < BV; ++b) x[off + b] = in[b];
  }
}

// Global-memory forms of ldv / stv.  A thread's BV values are 32 bytes for
// BV = 8 in FP32 (4 in FP64); one 256-bit access (ld/st.global.v8.b32)
// moves them where the address is 32-byte aligned, so that the two threads
// of a row fill whole 32-byte sectors with one request each, instead of two
// 16-byte requests that each use half of every sector they touch (the
// neighbour gathers of the level steps are bound by L1 sector throughput).
// Other sizes and alignments take the 16-byte path.  The values are the
// same either way.  kA: -1 tests each address; 1 or 0 is a launch-wide
// answer (mb_aligned below), so an access carries no alignment branch and
// the gathers of a row can be issued back to back.
__device__ __forceinline__ void ld256(const void* p, uint32_t (&w)[8]) {
  asm("ld.global.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
        "=r"(w[7])
      : "l"(p));
}

__device__ __forceinline__ void st256(void* p, const uint32_t (&w)[8]) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(w[0]),
               "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
               : "memory");
}

template <class T, int BV, int kA = -1>
__device__ __forceinline__ void ldg(const T* __restrict__ x, size_t off, T (&out)[BV]) {
  constexpr int W32 = 32 / (int)sizeof(T);
  if constexpr (BV % W32 == 0 && kA != 0) {
    const T* p = x + off;
    if (kA == 1 || __builtin_expect(((uintptr_t)p & 31) == 0, 1)) {
#pragma unroll
      for (int k = 0; k < BV / W32; ++k) {
        uint32_t w[8];
        ld256(p + k * W32, w);
        memcpy(&out[k * W32], w, 32);
      }
      return;
    }
  }
  ldv<T, BV>(x, off, out);
}

template <class T, int BV, int kA = -1>
__device__ __forceinline__ void stg(T* __restrict__ x, size_t off, const T (&in)[BV]) {
  constexpr int W32 = 32 / (int)sizeof(T);
  if constexpr (BV % W32 == 0 && kA != 0) {
    T* p = x + off;
    if (kA == 1 || ((uintptr_t)p & 31) == 0) {
#pragma unroll
      for (int k = 0; k < BV / W32; ++k) {
        uint32_t w[8];
        memcpy(w, &in[k * W32], 32);
        st256(p + k * W32, w);
      }
      return;
    }
  }
  stv<T, BV>(x, off, in);
}

// Whether every [n][B] access of a launch is 32-byte aligned: the vectors'
// base addresses are, and so is a row (B * sizeof(T)); a thread's column
// offset b0 * sizeof(T) is a multiple of BV * sizeof(T), which the 256-bit
// path requires to be 32 (ldg / stg).
template <class T>
__device__ __forceinline__ bool mb_aligned(int B, const void* a, const void* b = nullptr,
                                           const void* c = nullptr, const void* d = nullptr) {
  return ((size_t)B * sizeof(T)) % 32 == 0 &&
         ((((uintptr_t)a) | ((uintptr_t)b) | ((uintptr_t)c) | ((uintptr_t)d)) & 31) == 0;
}

// Runs BODY, a generic lambda over the alignment mode (its argument's
// ::value is the kA of ldg / stg), once.  FP32: with kA = 1 when AL holds
// for the launch, else with kA = 0 (on the 16-rhs L-shape level 0 the
// residual, the SAGEConv update, Phi_R and P e_c took 3-5 % less time than
// with a test per access; the prolongation update, which needs more
// registers in this form, keeps the test per access).  FP64: kA = -1,
// the test per access.
#define MG_MB_DISPATCH(AL, BODY)                 \
  if constexpr (sizeof(T) != 4)                  \
    BODY(std::integral_constant<int, -1>{});     \
  else if (AL)                                   \
    BODY(std::integral_constant<int, 1>{});      \
  else                                           \
    BODY(std::integral_constant<int, 0>{});

// The per-access form, for the kernels not moved to the launch-wide answer.
#define MG_MB_PER_ACCESS(BODY) BODY(std::integral_constant<int, -1>{});

// Launch: 1-D grid of ceil(NROWS * (B / BV) / kThreads) blocks.  PF: the
// row's read-only prefetch (kernels.cuh), before griddepcontrol.wait.
#define MG_MB_PROLOGUE(NROWS, PF)                               \
  const int nq = B / BV;                                        \
  const int g = blockIdx.x * blockDim.x + threadIdx.x;          \
  const int i = g / nq;                                         \
  const bool in_rows = i < (NROWS);                             \
  if (in_rows && blockIdx.x < kPrefetchBlocks) { PF; }         \
  pdl_wait();                                                   \
  pdl_launch();                                                 \
  if (!in_rows) return;                                         \
  const int b0 = (g - i * nq) * BV;                             \
  const size_t base = (size_t)i * B + b0;

// sum_{j != i} a_ij x_j for BV columns
template <class T, int BV, int kA = -1>
__device__ __forceinline__ void row_ax_mb(const LV<T>& L, int i, const T* __restrict__ x, int B,
                                          int b0, T (&ax)[BV]) {
#pragma unroll
  for (int b = 0; b < BV; ++b) ax[b] = T(0);
  for_nb<T, true, true>(L, i, [&](int c, T v, bool) {
    T xv[BV];
    ldg<T, BV, kA>(x, (size_t)c * B + b0, xv);
#pragma unroll
    for (int b = 0; b < BV; ++b) ax[b] = fma(v, xv[b], ax[b]);
  });
}

// sum_{j in N(i)} x_j for BV columns (kPre: SELL column preload, see for_nb;
// measured faster in the prolongation, slower in the two mean-only steps,
// whose extra registers cost occupancy)
template <class T, int BV, bool kPre = false, int kA = -1>
__device__ __forceinline__ void row_sum_mb(const LV<T>& L, int i, const T* __restrict__ x, int B,
                                           int b0, T (&s)[BV]) {
#pragma unroll
  for (int b = 0; b < BV; ++b) s[b] = T(0);
  for_nb<T, false, kPre>(L, i, [&](int c, T, bool nb) {
    T xv[BV];
    ldg<T, BV, kA>(x, (size_t)c * B + b0, xv);
#pragma unroll
    for (int b = 0; b < BV; ++b) s[b] += nb ? xv[b] : T(0);
  });
}

// Resident blocks asked of the compiler for 32-byte tiles of the residual
// (FP32: 48 registers) and of Phi_R (32 registers): in the launch-wide form
// the compiler would otherwise take 52 and 40 and lose a block per SM, which
// measured slower; Phi_R keeps its 32 registers in FP64 too.
template <class T, int BV>
constexpr int kResMinBlocks = sizeof(T) == 4 && BV * sizeof(T) == 32 ? 5 : 1;
template <class T, int BV>
constexpr int kConvRMinBlocks = BV * sizeof(T) == 32 ? 8 : 1;

template <class T, int BV>
__global__ void __launch_bounds__(kThreads, kResMinBlocks<T, BV>) k_residual_mb(LV<T> L, const T* __restrict__ f,
                                                          const T* __restrict__ u,
                                                          T* __restrict__ out, int B,
                                                          const T* __restrict__ prm, int scale,
                                                          int u_zero) {
  MG_MB_PROLOGUE(L.n, prefetch_row(L, i))
  auto body = [&](auto A) {
    constexpr int kA = decltype(A)::value;
    T r[BV];
    ldg<T, BV, kA>(f, base, r);
    if (!u_zero) {
      T ax[BV], uu[BV];
      row_ax_mb<T, BV, kA>(L, i, u, B, b0, ax);
      ldg<T, BV, kA>(u, base, uu);
      const T d = L.diag[i];
#pragma unroll
      for (int b = 0; b < BV; ++b) r[b] = fma(-d, uu[b], r[b]) - ax[b];
    }
    if (scale) {
      const T th = prm[P_THETA], di = L.dinv[i];
#pragma unroll
      for (int b = 0; b < BV; ++b) r[b] = th * (r[b] * di);
    }
    stg<T, BV, kA>(out, base, r);
  };
  MG_MB_DISPATCH(mb_aligned<T>(B, f, u, out), body)
}

// Resident blocks asked of the compiler for the mean-only step: it is
// bound by the latency of its neighbour gathers, so tiles of up to 32
// bytes a thread keep 7 blocks (36 registers) per SM.
template <class T, int BV>
constexpr int kConvMinBlocks = BV * sizeof(T) <= 32 ? 7 : 1;

template <class T, int BV>
__global__ void __launch_bounds__(kThreads, kConvMinBlocks<T, BV>)
    k_conv_update_mb(LV<T> L, const T* __restrict__ x,
                                                             T* __restrict__ u, int B,
                                                             const T* __restrict__ prm,
                                                             int u_zero) {
  MG_MB_PROLOGUE(L.n, prefetch_mean(L, i))
  auto body = [&](auto A) {
    constexpr int kA = decltype(A)::value;
    T s[BV], xi[BV], uu[BV];
    row_sum_mb<T, BV, false, kA>(L, i, x, B, b0, s);
    ldg<T, BV, kA>(x, base, xi);
    if (u_zero) {
#pragma unroll
      for (int b = 0; b < BV; ++b) uu[b] = T(0);
    } else {
      ldg<T, BV, kA>(u, base, uu);
    }
    const T w1 = prm[P_WB1], w2 = prm[P_WB2], eta = prm[P_ETA], id = L.invdeg[i];
#pragma unroll
    for (int b = 0; b < BV; ++b) {
      const T phi = fma(w1, xi[b], w2 * (id * s[b]));
      uu[b] = fma(eta, phi, uu[b]);
    }
    stg<T, BV, kA>(u, base, uu);
  };
  MG_MB_DISPATCH(mb_aligned<T>(B, x, u), body)
}

// k_cheb_step (kernels.cuh) for a tile of BV right-hand sides: the row's
// neighbour pattern is read once for the tile; same arithmetic per entry.
template <class T, int BV>
__global__ void __launch_bounds__(kThreads) k_cheb_step_mb(LV<T> L, const T* __restrict__ tprev,
                                                           const T* tpp, T* out,
                                                           T* __restrict__ u, int B,
                                                           const T* __restrict__ prm,
                                                           const T* __restrict__ coef, int k,
                                                           int u_zero) {
  MG_MB_PROLOGUE(L.n, prefetch_mean(L, i))
  auto body = [&](auto A) {
    constexpr int kA = decltype(A)::value;
    T s[BV], q[BV], uu[BV];
    row_sum_mb<T, BV, false, kA>(L, i, tprev, B, b0, s);
    ldg<T, BV, kA>(tpp, base, q);
    if (u_zero) {
#pragma unroll
      for (int b = 0; b < BV; ++b) uu[b] = T(0);
    } else {
      ldg<T, BV, kA>(u, base, uu);
    }
    const T id = L.invdeg[i], eta = prm[P_ETA], c0 = coef[0], ck = coef[k];
#pragma unroll
    for (int b = 0; b < BV; ++b) {
      const T lt = -(id * s[b]);
      T tk, upd;
      if (k == 1) {
        tk = lt;
        upd = fma(ck, tk, c0 * q[b]);
      } else {
        tk = fma(T(2), lt, -q[b]);
        upd = ck * tk;
      }
      q[b] = tk;
      uu[b] = fma(eta, upd, uu[b]);
    }
    stg<T, BV, kA>(out, base, q);
    stg<T, BV, kA>(u, base, uu);
  };
  MG_MB_DISPATCH(mb_aligned<T>(B, tprev, tpp, out, u), body)
}

// FP32 32-byte tiles of the fused Jacobi step: 64 registers (4 blocks per
// SM), as in the per-access form; unbounded, the launch-wide form takes 66
// and loses a block.  Measured with the bound (a small spill): the classical
// FP32 FCG solve of the 16-rhs L-shape, 282 -> 277 ms.
template <class T, int BV>
constexpr int kJacMinBlocks = sizeof(T) == 4 && BV * sizeof(T) == 32 ? 4 : 1;

template <class T, int BV>
__global__ void __launch_bounds__(kThreads, kJacMinBlocks<T, BV>) k_jacobi_mb(LV<T> L, const T* __restrict__ f,
                                                        const T* __restrict__ uin,
                                                        T* __restrict__ uout, int B,
                                                        const T* __restrict__ prm, int u_zero) {
  MG_MB_PROLOGUE(L.n, prefetch_row(L, i))
  auto body = [&](auto A) {
    constexpr int kA = decltype(A)::value;
    T r[BV], u0[BV];
    ldg<T, BV, kA>(f, base, r);
    if (u_zero) {
#pragma unroll
      for (int b = 0; b < BV; ++b) u0[b] = T(0);
    } else {
      T ax[BV];
      ldg<T, BV, kA>(uin, base, u0);
      row_ax_mb<T, BV, kA>(L, i, uin, B, b0, ax);
      const T d = L.diag[i];
#pragma unroll
      for (int b = 0; b < BV; ++b) r[b] = fma(-d, u0[b], r[b]) - ax[b];
    }
    const T th = prm[P_THETA], eta = prm[P_ETA], w1 = prm[P_WB1], di = L.dinv[i];
#pragma unroll
    for (int b = 0; b < BV; ++b) {
      const T delta = th * (r[b] * di);
      r[b] = fma(eta, w1 * delta, u0[b]);
    }
    stg<T, BV, kA>(uout, base, r);
  };
  MG_MB_DISPATCH(mb_aligned<T>(B, f, uin, uout), body)
}

// phi_i = wR1 r_i + wR2 mean_{N(i)} r
template <class T, int BV>
__global__ void __launch_bounds__(kThreads, kConvRMinBlocks<T, BV>) k_conv_r_mb(LV<T> L, const T* __restrict__ r,
                                                        T* __restrict__ phi, int B,
                                                        const T* __restrict__ prm) {
  MG_MB_PROLOGUE(L.n, prefetch_mean(L, i))
  auto body = [&](auto A) {
    constexpr int kA = decltype(A)::value;
    T s[BV], ri[BV];
    row_sum_mb<T, BV, false, kA>(L, i, r, B, b0, s);
    ldg<T, BV, kA>(r, base, ri);
    const T w1 = prm[P_WR1], w2 = prm[P_WR2], id = L.invdeg[i];
#pragma unroll
    for (int b = 0; b < BV; ++b) {
      T p = w1 * ri[b];
      ri[b] = fma(w2, id * s[b], p);
    }
    stg<T, BV, kA>(phi, base, ri);
  };
  MG_MB_DISPATCH(mb_aligned<T>(B, r, phi), body)
}

// fc_I = sum_children P_iI phi_i (coarse rows); scale: phi = w1 * x (plain
// restriction), else phi = x (after k_conv_r_mb)
template <class T, int BV>
__global__ void __launch_bounds__(kThreads) k_gather_mb(LV<T> L, const T* __restrict__ x,
                                                        T* __restrict__ fc, int B,
                                                        const T* __restrict__ prm, int scale) {
  MG_MB_PROLOGUE(L.nc, prefetch_r(L, i))
  auto body = [&](auto A) {
    constexpr int kA = decltype(A)::value;
    T acc[BV];
#pragma unroll
    for (int b = 0; b < BV; ++b) acc[b] = T(0);
    const T w1 = prm[P_WR1];
    for (int k = 0; k < L.KR; ++k) {
      const int c = idx_ok(L.r_idx[(size_t)k * L.ldc + i], L.n, 3);
      if (c < 0) break;
      const T w = L.r_w[(size_t)k * L.ldc + i];
      T xv[BV];
      ldg<T, BV, kA>(x, (size_t)c * B + b0, xv);
#pragma unroll
      for (int b = 0; b < BV; ++b) acc[b] = fma(w, scale ? w1 * xv[b] : xv[b], acc[b]);
    }
    stg<T, BV, kA>(fc, base, acc);
  };
  MG_MB_DISPATCH(mb_aligned<T>(B, x, fc), body)
}

// pe_i = (P ec)_i
template <class T, int BV, int kA = -1>
__device__ __forceinline__ void prolong_at_mb(const LV<T>& L, int j, const T* __restrict__ ec,
                                              int B, int b0, T (&v)[BV]) {
  const int a = idx_ok(L.p_idx[j], L.nc, 2), c = idx_ok(L.p_idx[(size_t)L.ld + j], L.nc, 2);
#pragma unroll
  for (int b = 0; b < BV; ++b) v[b] = T(0);
  if (a >= 0) {
    T e[BV];
    ldg<T, BV, kA>(ec, (size_t)a * B + b0, e);
    const T w = L.p_w[j];
#pragma unroll
    for (int b = 0; b < BV; ++b) v[b] = w * e[b];
  }
  if (c >= 0) {
    T e[BV];
    ldg<T, BV, kA>(ec, (size_t)c * B + b0, e);
    const T w = L.p_w[(size_t)L.ld + j];
#pragma unroll
    for (int b = 0; b < BV; ++b) v[b] = fma(w, e[b], v[b]);
  }
}

template <class T, int BV>
__global__ void __launch_bounds__(kThreads) k_pe_mb(LV<T> L, const T* __restrict__ ec,
                                                    T* __restrict__ pe, int B) {
  MG_MB_PROLOGUE(L.n, prefetch_p(L, i))
  auto body = [&](auto A) {
    constexpr int kA = decltype(A)::value;
    T v[BV];
    prolong_at_mb<T, BV, kA>(L, i, ec, B, b0, v);
    stg<T, BV, kA>(pe, base, v);
  };
  MG_MB_DISPATCH(mb_aligned<T>(B, ec, pe), body)
}

// u_i = uin_i + wP1 x_i + wP2 mean_{N(i)} x with x = pe (conv), or
// u_i = uin_i + wP1 (P ec)_i (plain prolongation: x = ec, conv = 0)
template <class T, int BV>
__global__ void __launch_bounds__(kThreads) k_prolong_mb(LV<T> L, const T* __restrict__ x,
                                                         const T* uin, T* u, int B,
                                                         const T* __restrict__ prm, int conv) {
  MG_MB_PROLOGUE(L.n, if (conv) prefetch_mean(L, i); prefetch_p(L, i))
  auto body = [&](auto A) {
    constexpr int kA = decltype(A)::value;
    T phi[BV], ui[BV];
    const T w1 = prm[P_WP1];
    if (conv) {
      T s[BV], xi[BV];
      ldg<T, BV, kA>(x, base, xi);
      row_sum_mb<T, BV, true, kA>(L, i, x, B, b0, s);
      const T w2 = prm[P_WP2], id = L.invdeg[i];
#pragma unroll
      for (int b = 0; b < BV; ++b) {
        T p = w1 * xi[b];
        phi[b] = fma(w2, id * s[b], p);
      }
    } else {
      T v[BV];
      prolong_at_mb<T, BV, kA>(L, i, x, B, b0, v);
#pragma unroll
      for (int b = 0; b < BV; ++b) phi[b] = w1 * v[b];
    }
    ldg<T, BV, kA>(uin, base, ui);
#pragma unroll
    for (int b = 0; b < BV; ++b) ui[b] = ui[b] + phi[b];
    stg<T, BV, kA>(u, base, ui);
  };
  MG_MB_PER_ACCESS(body)
}

#undef MG_MB_PROLOGUE

}  // namespace mgk
