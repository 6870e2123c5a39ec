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

// HALO_SMOOTH_GATHER: the first smoothing step of a level that starts from
// zero, with the level's right-hand side gathered in the first stage from
// the finer level's Phi_R values (f_j = (P^T phi)_j, gather_el's arithmetic,
// for the tile's rows and halo; written to fout for the tile's own rows), so
// the restriction's separate gather launch is not needed.
enum { HALO_SMOOTH = 0, HALO_RESTRICT = 1, HALO_PROLONG = 2, HALO_SMOOTH_GATHER = 3 };

// kB = 1: one right-hand side known at compile time; kB = 0: B of them.
// Lf, phi, fout: the finer level, its Phi_R values and this level's
// right-hand side (HALO_SMOOTH_GATHER only).
template <class T, int MODE, int kB>
__global__ void __launch_bounds__(kTailThreads)
    k_halo_dia(LV<T> L, const T* __restrict__ f, const T* __restrict__ x, T* y, int B_,
               const T* __restrict__ prm, int TR, int H, int zero, LV<T> Lf,
               const T* __restrict__ phi, T* __restrict__ fout) {
  constexpr bool kSmooth = MODE == HALO_SMOOTH || MODE == HALO_SMOOTH_GATHER;
  const int B = kB ? kB : B_;
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
    if constexpr (MODE == HALO_SMOOTH_GATHER) prefetch_r(Lf, j);
    prefetch_row(L, j);
  }
  pdl_wait();
  pdl_launch();

  // The operands of this thread's first second-stage element (its row's
  // neighbour bits, 1/deg and the value it updates), loaded before the
  // barrier so that they travel with the first stage's loads instead of
  // costing a second memory round trip after it.
  const size_t eo = (size_t)(r0 - lo) * B;  // the tile's own rows: [eo, e1)
  const size_t e0 = eo + threadIdx.x;
  const size_t e1 = (size_t)(r1 - lo) * B;
  unsigned m0 = 0;
  T id0 = T(0), v0 = T(0);
  if (e0 < e1) {
    const size_t t = base + e0;
    int i, b;
    split_rb(t, B, i, b);
    m0 = nb_mask(L, i);
    id0 = L.invdeg[i];
    if constexpr (MODE == HALO_SMOOTH) v0 = zero ? T(0) : x[t];
    if constexpr (MODE == HALO_PROLONG) v0 = y[t];
  }

  // first stage on own rows and halo
  for (size_t e = threadIdx.x; e < nz; e += blockDim.x) {
    const size_t t = base + e;
    int j, b;
    split_rb(t, B, j, b);
    T z;
    if constexpr (MODE == HALO_PROLONG) {
      z = prolong_at(L, j, x, B, b);
    } else if constexpr (MODE == HALO_SMOOTH_GATHER) {  // from zero: delta = theta dinv f
      const T fj = gather_at(Lf, phi, B, j, b);
      if (e >= eo && e < e1) fout[t] = fj;
      z = prm[P_THETA] * (fj * L.dinv[j]);
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
  // inside [lo, hi).  The neighbour sum is row_sum's (ascending offsets,
  // absent entries adding +0).
  for (size_t e = e0; e < e1; e += blockDim.x) {
    const size_t t = base + e;
    int i, b;
    split_rb(t, B, i, b);
    const bool first = e == e0;
    const unsigned m = first ? m0 : nb_mask(L, i);
    const T id = first ? id0 : L.invdeg[i];
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kMaxDia; ++k) {
      if (k < L.ndia) {
        const int c = min(max(i + L.doff[k], 0), L.n - 1);
        const T zv = sz[(size_t)(c - lo) * B + b];
        s += ((m >> k) & 1u) ? zv : T(0);
      }
    }
    if constexpr (kSmooth) {
      const T ph = fma(prm[P_WB1], sz[e], prm[P_WB2] * (id * s));
      const T u0 = MODE == HALO_SMOOTH_GATHER ? T(0) : (first ? v0 : (zero ? T(0) : x[t]));
      y[t] = fma(prm[P_ETA], ph, u0);
    } else if constexpr (MODE == HALO_RESTRICT) {
      T p = prm[P_WR1] * sz[e];
      p = fma(prm[P_WR2], id * s, p);
      y[t] = p;
    } else {
      T ph = prm[P_WP1] * sz[e];
      ph = fma(prm[P_WP2], id * s, ph);
      y[t] = (first ? v0 : y[t]) + ph;
    }
  }
}

// The same fused steps with 2D tiles, for DIA levels laid out on a grid of
// width w whose offsets are 0, +-1, +-w, +-(w-1) or +-(w+1) (every square
// mesh here; the stacked contexts are grids of width w and slots * w rows).
// A 1D tile of TR rows needs a halo of H = w + 1 rows on each side, which
// for a large level is several times the tile; a tile of kH2X x kH2Y grid
// points needs a ring of one point: (kH2X + 2)(kH2Y + 2) first-stage points
// for kH2X * kH2Y outputs.  Neighbour k of row i sits at grid shift
// (dx[k], dy[k]); a region point outside the grid's columns or rows holds 0
// and is only ever met through an absent (zero) entry.  Same arithmetic as
// k_halo_dia and the two-kernel form.  Launch: tiles_x * tiles_y blocks of
// kH2Threads, (kH2X + 2)(kH2Y + 2) * B * sizeof(T) bytes of dynamic shared
// memory.
// Measured on the 8-slot stacked 1025^2 context (8.4M rows, one rhs per
// block): the fused smoothing step takes 167 us against 96 us for the
// two-row pair (k_residual_dia2r + k_mean_dia2r), although it moves about
// 40 instead of 68 bytes per row: every region point repeats a full
// residual, so it issues more instructions per output than the pair, which
// is no longer DRAM-bound either.  Off by default (MG_OPT_HALO2D_BYTES).
constexpr int kH2X = 32, kH2Y = 8;
constexpr int kH2RX = kH2X + 2, kH2RY = kH2Y + 2;

struct DiaShift {
  int8_t dx[kMaxDia], dy[kMaxDia];
};

// One thread per region point for one right-hand side, so that the first
// stage is a single round of loads per block.
constexpr int kH2Threads = (kH2RX * kH2RY + 31) / 32 * 32;

// kB = 1: one right-hand side known at compile time; kB = 0: B of them.
// No prefetch before the wait: the level spans many waves of blocks, and
// only the first wave would overlap its predecessor.
template <class T, int MODE, int kB>
__global__ void __launch_bounds__(kH2Threads, 4)
    k_halo_dia2(LV<T> L, const T* __restrict__ f, const T* __restrict__ x, T* y, int B_,
                const T* __restrict__ prm, int w, int tiles_x, DiaShift sh, int zero) {
  const int B = kB ? kB : B_;
  extern __shared__ __align__(16) unsigned char halo_raw[];
  T* sz = reinterpret_cast<T*>(halo_raw);
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int gx0 = tx * kH2X - 1, gy0 = ty * kH2Y - 1;  // grid point of region (0, 0)
  auto row_at = [&](int lx, int ly) -> int {  // row of a region point, or -1
    const int gx = gx0 + lx, gy = gy0 + ly;
    if (gx < 0 || gx >= w || gy < 0) return -1;
    const long long r = (long long)gy * w + gx;
    return r < L.n ? (int)r : -1;
  };
  const int npts = kH2RX * kH2RY;
  pdl_wait();
  pdl_launch();

  // The operands of this thread's first second-stage output (its
  // neighbour bits, 1/deg and the value it updates), loaded before the
  // barrier so that they travel with the first stage's loads.
  const int nown = kH2X * kH2Y * B;
  int i0 = -1;
  unsigned m0 = 0;
  T id0 = T(0), v0 = T(0);
  if ((int)threadIdx.x < nown) {
    const int pt = threadIdx.x / B, b = threadIdx.x - pt * B;
    i0 = row_at(1 + pt % kH2X, 1 + pt / kH2X);
    if (i0 >= 0) {
      const size_t t = (size_t)i0 * B + b;
      m0 = nb_mask(L, i0);
      id0 = L.invdeg[i0];
      if constexpr (MODE == HALO_SMOOTH) v0 = zero ? T(0) : x[t];
      if constexpr (MODE == HALO_PROLONG) v0 = y[t];
    }
  }

  // first stage on the region (own points and the one-point ring)
  const int nz = npts * B;
  for (int e = threadIdx.x; e < nz; e += blockDim.x) {
    const int pt = e / B, b = e - pt * B;
    const int j = row_at(pt % kH2RX, pt / kH2RX);
    T z = T(0);
    if (j >= 0) {
      const size_t t = (size_t)j * B + b;
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
    }
    sz[e] = z;
  }
  __syncthreads();

  // second stage on the own points
  for (int e = threadIdx.x; e < nown; e += blockDim.x) {
    const int pt = e / B, b = e - pt * B;
    const int lx = 1 + pt % kH2X, ly = 1 + pt / kH2X;
    const bool first = e == (int)threadIdx.x;
    const int i = first ? i0 : row_at(lx, ly);
    if (i < 0) continue;
    const size_t t = (size_t)i * B + b;
    const unsigned m = first ? m0 : nb_mask(L, i);
    const T id = first ? id0 : L.invdeg[i];
    const int me = ly * kH2RX + lx;
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kMaxDia; ++k) {
      if (k < L.ndia) {
        const bool nb = ((m >> k) & 1u) != 0u;
        const T zv = nb ? sz[(size_t)(me + sh.dy[k] * kH2RX + sh.dx[k]) * B + b] : T(0);
        s += nb ? zv : T(0);
      }
    }
    const T zi = sz[(size_t)me * B + b];
    if constexpr (MODE == HALO_SMOOTH) {
      const T phi = fma(prm[P_WB1], zi, prm[P_WB2] * (id * s));
      const T u0 = first ? v0 : (zero ? T(0) : x[t]);
      y[t] = fma(prm[P_ETA], phi, u0);
    } else if constexpr (MODE == HALO_RESTRICT) {
      T p = prm[P_WR1] * zi;
      p = fma(prm[P_WR2], id * s, p);
      y[t] = p;
    } else {
      T phi = prm[P_WP1] * zi;
      phi = fma(prm[P_WP2], id * s, phi);
      y[t] = (first ? v0 : y[t]) + phi;
    }
  }
}

}  // namespace mgk
