// Halo-tiled fused level steps for SELL-32 levels (unstructured meshes).
//
// The same two-stage steps as halo.cuh (a per-row first stage x -> z, then
// y_i = F(z_i, mean_{N(i)} z) with the SAGEConv mean of Sec. 3.2), for
// levels whose off-diagonals are stored as SELL-32 slices.  On an
// unstructured level the neighbours of a row are not within a fixed offset,
// so the tiles carry explicit halos built on the host at set-up:
//  - a tile is TR consecutive rows [r0, r1) (TR a multiple of the slice
//    height; on a locality-preserving row order, such as the Morton order
//    of the meshes here, most neighbours of a tile lie inside it);
//  - hrow[hptr[t] .. hptr[t+1]) lists, ascending, the rows outside the tile
//    that are neighbours of a tile row (the tile's halo);
//  - lcol[e], parallel to the SELL column array, gives for every entry of a
//    tile row the local slot of its column: c - r0 inside the tile, else
//    (r1 - r0) + k for the halo row hrow[hptr[t] + k]; -1 for padding.
// A block evaluates the first stage on its rows and its halo rows into
// shared memory (slot l holds row r0 + l for l < r1 - r0, halo row k at
// r1 - r0 + k), synchronises, and applies the second stage to its own rows,
// reading the neighbours' z through lcol.  Halo rows are evaluated by every
// tile that borders them (redundant work, from L2 in the common case); in
// exchange z never goes to global memory and the kernel boundary between
// the two stages disappears.  Modes and arithmetic are those of halo.cuh
// and of the multi-rhs element forms (multi_rhs.cuh): results are bitwise
// those of the two-kernel form.
//
//   HALO_SMOOTH    z = theta D^{-1}(f - A x)          (x = u_in, or 0 if zero)
//                  y = x + eta (wB1 z + wB2 mean z)   (y = u_out, y != x)
//   HALO_RESTRICT  z = f - A x                        (x = u)
//                  y = wR1 z + wR2 mean z             (y = Phi_R(r), fine rows)
//   HALO_PROLONG   z = P x                            (x = e_c)
//                  y = y + wP1 z + wP2 mean z         (y = u, in place per row)
//
// Launch: one block per tile, of at most kTailThreads threads (a launch-shape
// choice: results do not depend on it); a thread takes items (slot, tile of
// BV right-hand sides) in turn.  Dynamic shared memory
// (TR + max halo) * B * sizeof(T).
#pragma once

#include <cstdint>

#include "halo.cuh"
#include "multi_rhs.cuh"

namespace mgk {

struct SellHalo {
  int TR;                             // rows per tile
  const int* __restrict__ hptr;       // [tiles + 1]
  const int* __restrict__ hrow;       // halo rows per tile, ascending
  const int16_t* __restrict__ lcol;   // local slot per SELL entry, -1 padding
};

template <class T, int BV, int MODE>
__global__ void __launch_bounds__(kTailThreads)
    k_halo_sell(LV<T> L, SellHalo hs, const T* __restrict__ f, const T* __restrict__ x, T* y,
                int B, const T* __restrict__ prm, int zero) {
  extern __shared__ __align__(16) unsigned char halo_raw[];
  T* sz = reinterpret_cast<T*>(halo_raw);
  const int nq = B / BV;
  const int t = blockIdx.x;
  const int r0 = t * hs.TR;
  const int nown = min(hs.TR, L.n - r0);
  const int h0 = hs.hptr[t];
  const int nh = hs.hptr[t + 1] - h0;
  const int nitem = (nown + nh) * nq;
  // read-only operator data of the tile's rows before waiting for the
  // predecessor (halo tables and SELL arrays never depend on it)
  for (int l = threadIdx.x; l < nown; l += blockDim.x) {
    if constexpr (MODE == HALO_PROLONG) prefetch_p(L, r0 + l);
    prefetch_row(L, r0 + l);
  }
  pdl_wait();
  pdl_launch();

  // first stage on the tile's rows and its halo rows
  for (int it = threadIdx.x; it < nitem; it += blockDim.x) {
    const int l = it / nq;
    const int b0 = (it - l * nq) * BV;
    const int j = l < nown ? r0 + l : idx_ok(hs.hrow[h0 + (l - nown)], L.n, 4);
#ifdef MG_BOUNDS_CHECK
    if (j < 0) continue;  // recorded; the slot is never read through a valid lcol
#endif
    const size_t base = (size_t)j * B + b0;
    T z[BV];
    if constexpr (MODE == HALO_PROLONG) {
      prolong_at_mb<T, BV>(L, j, x, B, b0, z);
    } else {
      ldg<T, BV>(f, base, z);
      if (!zero) {
        T ax[BV], uu[BV];
        row_ax_mb<T, BV>(L, j, x, B, b0, ax);
        ldg<T, BV>(x, base, uu);
        const T d = L.diag[j];
#pragma unroll
        for (int b = 0; b < BV; ++b) z[b] = fma(-d, uu[b], z[b]) - ax[b];
      }
      if constexpr (MODE == HALO_SMOOTH) {
        const T th = prm[P_THETA], di = L.dinv[j];
#pragma unroll
        for (int b = 0; b < BV; ++b) z[b] = th * (z[b] * di);
      }
    }
    stv<T, BV>(sz, (size_t)l * B + b0, z);
  }
  __syncthreads();

  // second stage on the tile's rows; neighbour slots through lcol, in the
  // row's SELL order (ascending column), as row_sum_mb visits them
  for (int it = threadIdx.x; it < nown * nq; it += blockDim.x) {
    const int l = it / nq;
    const int b0 = (it - l * nq) * BV;
    const int i = r0 + l;
    const size_t base = (size_t)i * B + b0;
    T s[BV], zi[BV];
#pragma unroll
    for (int b = 0; b < BV; ++b) s[b] = T(0);
    const int end = L.sl_ptr[(i >> 5) + 1];
    for (int e = L.sl_ptr[i >> 5] + (i & 31); e < end; e += kSlice) {
      const int lc = idx_ok(hs.lcol[e], nown + nh, 5);
      if (lc >= 0) {
        T zv[BV];
        ldv<T, BV>(sz, (size_t)lc * B + b0, zv);
#pragma unroll
        for (int b = 0; b < BV; ++b) s[b] += zv[b];
      }
    }
    ldv<T, BV>(sz, (size_t)l * B + b0, zi);
    const T id = L.invdeg[i];
    if constexpr (MODE == HALO_SMOOTH) {
      T uu[BV];
      if (zero) {
#pragma unroll
        for (int b = 0; b < BV; ++b) uu[b] = T(0);
      } else {
        ldg<T, BV>(x, base, uu);
      }
      const T w1 = prm[P_WB1], w2 = prm[P_WB2], eta = prm[P_ETA];
#pragma unroll
      for (int b = 0; b < BV; ++b) {
        const T phi = fma(w1, zi[b], w2 * (id * s[b]));
        uu[b] = fma(eta, phi, uu[b]);
      }
      stg<T, BV>(y, base, uu);
    } else if constexpr (MODE == HALO_RESTRICT) {
      const T w1 = prm[P_WR1], w2 = prm[P_WR2];
#pragma unroll
      for (int b = 0; b < BV; ++b) {
        const T p = w1 * zi[b];
        zi[b] = fma(w2, id * s[b], p);
      }
      stg<T, BV>(y, base, zi);
    } else {
      T uu[BV];
      ldg<T, BV>(y, base, uu);
      const T w1 = prm[P_WP1], w2 = prm[P_WP2];
#pragma unroll
      for (int b = 0; b < BV; ++b) {
        const T p = w1 * zi[b];
        uu[b] = uu[b] + fma(w2, id * s[b], p);
      }
      stg<T, BV>(y, base, uu);
    }
  }
}

}  // namespace mgk
