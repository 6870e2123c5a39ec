// Halo-tiled fused level steps for DIA levels (structured meshes).
//
// Each of the learnable steps of Algorithm 2 that apply a SAGEConv mean
// (Sec. 3.2) is a two-stage map: a per-row first stage x -> z, then
// y_i = F(z_i, mean_{N(i)} z).  Unfused, the two stages are two grid
// kernels with z in global memory.  On a DIA level the neighbours of row i
// lie within H = max_k |offset_k| rows, so a block that owns rows [r0, r1)
// evaluates the first stage on rows [lo, hi) = [r0 - H, r1 + H) clamped to
// [0, n) into shared memory, synchronises, and applies the second stage to
// its own rows from there.  Halo rows are evaluated by both neighbouring
// blocks (redundant work, 2H / (r1 - r0) extra), which trades a kernel
// boundary for a block barrier.
//
//   HALO_SMOOTH    z = theta D^{-1}(f - A x)          (x = u_in, or 0 if zero)
//                  y = x + eta (wB1 z + wB2 mean z)   (y = u_out, y != x)
//   HALO_RESTRICT  z = f - A x                        (x = u)
//                  y = wR1 z + wR2 mean z             (y = Phi_R(r), fine rows)
//   HALO_PROLONG   z = P x                            (x = e_c)
//                  y = y + wP1 z + wP2 mean z         (y = u, in place per row)
//
// Each stage is the arithmetic of the unfused element functions in
// kernels.cuh (same operations, same order), so results are bitwise those
// of the two-kernel form.  Launch: grid ceil(n / TR), kTailThreads threads,
// (min(TR + 2H, n)) * B * sizeof(T) bytes of dynamic shared memory.
#pragma once

#include "kernels.cuh"

namespace mgk {

enum { HALO_SMOOTH = 0, HALO_RESTRICT = 1, HALO_PROLONG = 2 };

template <class T, int MODE>
__global__ void __launch_bounds__(kTailThreads)
    k_halo_dia(LV<T> L, const T* __restrict__ f, const T* __restrict__ x, T* y, int B,
               const T* __restrict__ prm, int TR, int H, int zero) {
  extern __shared__ __align__(16) unsigned char halo_raw[];
  T* sz = reinterpret_cast<T*>(halo_raw);
  const int r0 = blockIdx.x * TR;
  const int r1 = min(r0 + TR, L.n);
  const int lo = max(r0 - H, 0), hi = min(r1 + H, L.n);
  const size_t base = (size_t)lo * B;
  const size_t nz = (size_t)(hi - lo) * B;
  // read-only operator rows of the tile before waiting for the predecessor
  for (int j = lo + (int)threadIdx.x; j < hi; j += blockDim.x) {
    if constexpr (MODE == HALO_PROLONG) prefetch_p(L, j);
    prefetch_row(L, j);
  }
  pdl_wait();
  pdl_launch();

  // first stage on own rows and halo
  for (size_t e = threadIdx.x; e < nz; e += blockDim.x) {
    const size_t t = base + e;
    int j, b;
    split_rb(t, B, j, b);
    T z;
    if constexpr (MODE == HALO_PROLONG) {
      z = prolong_at(L, j, x, B, b);
    } else {
      z = f[t];
      if (!zero) {
        const T ax = row_ax(L, j, x, B, b);
        z = fma(-L.diag[j], x[t], z) - ax;
      }
      if constexpr (MODE == HALO_SMOOTH) z = prm[P_THETA] * (z * L.dinv[j]);
    }
    sz[e] = z;
  }
  __syncthreads();

  // second stage on own rows; every neighbour (clamped index included) is
  // inside [lo, hi)
  const size_t e1 = (size_t)(r1 - lo) * B;
  for (size_t e = (size_t)(r0 - lo) * B + threadIdx.x; e < e1; e += blockDim.x) {
    const size_t t = base + e;
    int i, b;
    split_rb(t, B, i, b);
    T s = T(0);
    for_nb<T, false>(L, i, [&](int c, T, bool nb) {
      const T zv = sz[(size_t)(c - lo) * B + b];
      s += nb ? zv : T(0);
    });
    if constexpr (MODE == HALO_SMOOTH) {
      const T phi = fma(prm[P_WB1], sz[e], prm[P_WB2] * (L.invdeg[i] * s));
      const T u0 = zero ? T(0) : x[t];
      y[t] = fma(prm[P_ETA], phi, u0);
    } else if constexpr (MODE == HALO_RESTRICT) {
      T p = prm[P_WR1] * sz[e];
      p = fma(prm[P_WR2], L.invdeg[i] * s, p);
      y[t] = p;
    } else {
      T phi = prm[P_WP1] * sz[e];
      phi = fma(prm[P_WP2], L.invdeg[i] * s, phi);
      y[t] = y[t] + phi;
    }
  }
}

}  // namespace mgk
