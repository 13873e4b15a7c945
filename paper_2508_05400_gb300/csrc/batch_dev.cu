// Batched rKS in one persistent launch.
//
// Each thread-block cluster (G CTAs, G = 1, 2, 4 or 8) takes problems from a
// device work queue sorted by cost, largest first, and runs the whole of
// Algorithm 1 for each on the device, with no host round trip (the launch
// configuration, one kernel or two taking problems from the two ends of the
// queue with different G, is picked by timing at creation):
//   - the expansions of Algorithm 2: SpMV, sketch, randomized Gram-Schmidt in
//     the sketch (CGS2 on the d-dimensional sketches), update, sketch of the
//     update; the rows of the problem are split over the G CTAs by tiles of
//     kBR rows, and the sketch partial sums are exchanged through global
//     memory at the cluster barrier;
//   - the contraction: Hessenberg reduction, Francis QR, reordering of the
//     wanted Schur blocks to the top, truncation to k columns (pairs kept
//     whole), whitening of the kept sketches when their Gram matrix drifted
//     (Sec. 3.3), Ritz pairs and the estimates of Sec. 4.1, by one warp of
//     every CTA with the routines of dense_dev.cuh (every CTA of a cluster
//     holds the same small matrices and takes the same decisions);
//   - the restart product U_k = U Q' (Eq. 3.5) row by row;
//   - at convergence the Ritz vectors x = U y and their FP64 residuals
//     ||A x - l x|| / (||A||_1 ||x||) and Rayleigh quotients; if a residual
//     is above `verify` the tolerance is divided by 4 and the restarts go on.
// The restart keeps the max(k, min(keep, m / 2)) best Schur vectors (a thick
// restart) and locks nothing.
//
// Arithmetic: basis and matrix values as double-float pairs (48-bit
// significand, error-free products and sums on the FP32 pipes); the sketch
// sums, least squares, dense steps and residuals in FP64.  The basis columns
// are stored unnormalised, u_c = sig_c * U[:, c] with sig_c = 1 / beta_c, so
// that no pass over the basis is spent on the normalisation: the scale enters
// the next SpMV and the coefficients of the update and restart products.
//
// The sketch Omega is the library's sparse-sign embedding (the same hash as
// rks_sketch_pairs).  For every tile of kBR rows the rows of each sketch row
// are listed in increasing order (built on the host at creation); a tile's
// sums are formed from its vector values staged in shared memory by 8 lanes
// per sketch row in a fixed order, written to global memory, and the tiles
// are added in a fixed order after the cluster barrier.  No result depends on
// G, so the autotuned choice does not change a bit of any output, and a
// problem's results are the same in any batch.
//
// Every loop is bounded (restarts by maxit, the QR sweeps by 60 m + 100); the
// only waits are __syncthreads and the hardware cluster barrier, reached by
// every CTA of a cluster in the same order because their decisions are made
// from identical data.

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <thread>
#include <vector>

#include "../../include/rks.h"
#include "dense_dev.cuh"
#include "rks_impl.h"

namespace cg = cooperative_groups;

namespace {

constexpr int kBT = 512;                 // threads per CTA
constexpr int kBR = 2048;                // rows per sketch tile (an entry holds the row in 15 bits)
constexpr int kBH = 8;                   // lanes per sketch row in the tile sums
constexpr int kBRowsPerThread = kBR / kBT;
constexpr int kBMaxM = rks_dd::kMaxM;    // largest Krylov dimension m
constexpr int kBMaxKa = 32;              // largest kept dimension (k + 1)
constexpr int kBInfo = 8;                // ints of every problem's record
constexpr int kBSlot = 6;                // doubles per reported pair: lre, lim, resid, rq_re, rq_im, est

enum { kIStatus = 0, kIRestarts, kIMatvec, kINw, kIConv, kIWhiten, kINconv };

// Scalar type of the warp-level dense step (Hessenberg, Francis QR,
// reordering, Ritz pairs).  The step is latency-bound on one warp: FP64 and
// the double-float type of dense_dev.cuh take the same time here, and FP64 is
// the more accurate.
using DenseR = double;
__device__ __forceinline__ DenseR dense_from(double x) { return DenseR(x); }

// Phases of the per-CTA cycle counters (clock64 deltas taken by thread 0 at
// the CTA barriers that end each phase, summed over CTAs and problems).
enum {
  kPhStart = 0, kPhSpmvRows, kPhHess, kPhExchange, kPhLs, kPhUpdRows, kPhSchur, kPhBeta, kPhDense,
  kPhKept, kPhRestart, kPhRitz, kPhFinal, kPhQueue, kPhases
};

// ---------------------------------------------------------------------------
// double-float arithmetic (error-free transformations)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void bd_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// (s, t) += (ah + al) * (bh + bl)
__device__ __forceinline__ void bd_mac(float ah, float al, float bh, float bl, float& s, float& t) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  float s2, e2;
  bd_two_sum(s, p, s2, e2);
  s = s2;
  t += e2 + e;
}
// (s, t) += (bh + bl)
__device__ __forceinline__ void bd_add(float bh, float bl, float& s, float& t) {
  float s2, e2;
  bd_two_sum(s, bh, s2, e2);
  s = s2;
  t += e2 + bl;
}
__device__ __forceinline__ float2 bd_norm(float s, float t) {
  const float h = s + t;
  return make_float2(h, t - (h - s));
}
__host__ __device__ __forceinline__ float2 bd_from(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}
__device__ __forceinline__ double bd_to(float2 v) { return (double)v.x + (double)v.y; }

// butterfly over the kBH lanes of a group (fixed order)
__device__ __forceinline__ void bd_group_sum(float& s, float& t) {
#pragma unroll
  for (int o = kBH / 2; o; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float t2 = __shfl_xor_sync(0xffffffffu, t, o);
    float ss, e;
    bd_two_sum(s, s2, ss, e);
    s = ss;
    t = t + t2 + e;
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ uint64_t bd_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Entry i of the default start vector: N(0,1) from SplitMix64(seed) draws
// 2i + 1 and 2i + 2 and Box-Muller (the generator of rks_create).
__device__ double bd_normal(uint64_t seed, int64_t i) {
  const uint64_t g = 0x9E3779B97F4A7C15ull;
  const uint64_t h1 = bd_mix64(seed + (uint64_t)(2 * i + 1) * g);
  const uint64_t h2 = bd_mix64(seed + (uint64_t)(2 * i + 2) * g);
  const double u1 = (double)(h1 >> 11) * (1.0 / 9007199254740992.0);
  const double u2 = (double)(h2 >> 11) * (1.0 / 9007199254740992.0);
  return sqrt(-2.0 * log1p(-u1)) * cospi(2.0 * u2);
}

// ---------------------------------------------------------------------------
// problem records and the shared-memory layout
// ---------------------------------------------------------------------------

constexpr int kBMaxDiag = 8;   // diagonals of the diagonal storage

struct BdProb {
  int64_t n;
  int ntile;
  const int32_t* rowptr;
  const int32_t* colind;
  const float2* vals;     // double-float values (CSR)
  int D;                  // > 0: A also by diagonals, offsets doff[e] increasing,
  int doff[kBMaxDiag];    //   row i's entry on diagonal e at dvals[e * ldu + i] (0 where A has none)
  const float2* dvals;
  int dv32;               // 1: every value of A is an FP32 number and dvals holds FP32 values
                          //   (const float*, the pairs' low words being zero)
  const int32_t* tbin;    // ntile x (d + 1): start of every (tile, sketch row) entry block
  const uint16_t* ent;    // entry blocks: 8 lane chunks of equal padded length,
                          //   entry = row in tile | 0x8000 if negative, 0xFFFF = none
  float2* U;              // the basis, unnormalised, by tiles: row r of tile t, column c at
                          //   U[(t (m + 1) + c) kBR + r]
  int64_t ldu;            // leading dimension of X and of the diagonal storage
  float2* tsum;           // 2 x ntile x d tile sums (double buffered)
  double* rsum;           // ntile x (k + 1) x 4 residual partials
  double* X;              // ldu x (k + 1) Ritz vectors (real packing)
  double norm1;
  double* out;            // (k + 1) x kBSlot, then max_est, max_resid
  int* info;              // kBInfo
};

struct BdArgs {
  const BdProb* probs;
  const int* order;       // problems, largest first
  unsigned long long* queue;   // positions taken from the front (low 32 bits) and the back (high 32 bits)
  int dir;                // 0: this kernel takes problems from the front of order, 1: from the back
  int tune;               // > 0: a tuning run, every problem stops after `tune` restarts
  int64_t nmax;
  int count, k, m, d, zeta, which, maxit, conv;
  int want;               // Schur vectors kept by a restart (thick restart, >= k)
  double tol, verify;
  uint64_t seed;
  unsigned long long* phase;   // kPhases cycle sums (zeroed before the launch)
};

struct BdLayout {
  int S, B, T, Q, Td, Qd, W, G, Ri, QC, z, sv, r, sig, coef, bk, lre, lim, est, scr, xs, total;
};

__host__ __device__ inline int bd_take(int& o, int cnt) {
  const int at = o;
  o += (cnt + 1) & ~1;   // 16-byte aligned regions
  return at;
}

// Offsets (in 8-byte words) of the per-CTA arrays in dynamic shared memory.
// The arrays of the contraction share their space with the two tile buffers
// of the expansions (never live at the same time).
__host__ __device__ inline BdLayout bd_layout(int m, int d) {
  BdLayout L;
  int o = 0;
  L.S = bd_take(o, d * (m + 1));         // sketches of the basis (orthonormal), FP64
  L.B = bd_take(o, (m + 1) * m);         // [B; b^T] of the decomposition, FP64
  L.z = bd_take(o, d);
  L.sv = bd_take(o, d);
  L.r = bd_take(o, m + 1);
  L.sig = bd_take(o, m + 1);
  L.coef = bd_take(o, m + 1);            // update coefficients (double-float)
  L.bk = bd_take(o, m);
  L.lre = bd_take(o, m);
  L.lim = bd_take(o, m);
  L.est = bd_take(o, m);
  L.scr = bd_take(o, 4 * m + 64);
  const int u0 = o;                      // contraction / finalisation only:
  L.T = bd_take(o, m * m);               // Hessenberg / Schur form, double-float
  L.Q = bd_take(o, m * m);               // Schur vectors, double-float
  L.Td = bd_take(o, m * m);              // kept block of the Schur form, FP64
  L.Qd = bd_take(o, m * m);              // kept Schur vectors, FP64
  L.W = bd_take(o, d * m > 2 * m * m ? d * m : 2 * m * m);   // kept sketches; Ritz vectors of T
  L.G = bd_take(o, m * m);               // Gram matrix, then R
  L.Ri = bd_take(o, m * m);              // R^{-1}
  L.QC = bd_take(o, m * m);              // restart coefficients (double-float); packed Y
  L.xs = u0;                             // expansions only: two tiles of one column (double-float)
  if (o < u0 + 2 * kBR) o = u0 + 2 * kBR;
  L.total = o;
  return L;
}

struct BdShared {
  int prob;
  int flag[8];
  int ord[kBMaxM];
  double red[8 + (kBT / 32) * 4];
};

// ---------------------------------------------------------------------------
// passes over the rows of one CTA
// ---------------------------------------------------------------------------

// Tile sums of the sketch of one column for tile t (xt: that column of the
// tile, rows written by this CTA): ts[t * d + b] = sum of the signed xt[row]
// listed for sketch row b.  8 lanes
// per sketch row, lane h adds its chunk of the list in order, then the
// butterfly; loop bounds are warp-uniform (4 groups a warp).
__device__ __forceinline__ void bd_bins_tile(const BdProb& P, int d, int t, const float2* __restrict__ xt,
                                          float2* __restrict__ ts) {
  const int g = threadIdx.x / kBH, h = threadIdx.x % kBH;
  const int32_t* off = P.tbin + (size_t)t * (d + 1);
  for (int bb = g & ~3; bb < d; bb += kBT / kBH) {
    const int b = bb + (g & 3);
    float s = 0.f, e = 0.f;
    if (b < d) {
      const int e0 = off[b], len = (off[b + 1] - e0) / kBH;   // per lane, a multiple of 8
      const uint4* ev = reinterpret_cast<const uint4*>(P.ent + e0 + (size_t)h * len);
      // branch-free: the padding entries gather row 0 with sign 0 (adding an
      // exact zero changes no bit), so that all 8 gathers are in flight at once
#pragma unroll 2
      for (int v = 0; v < len / 8; ++v) {
        const uint4 w = ev[v];
        const uint32_t word[4] = {w.x, w.y, w.z, w.w};
        float2 xv[8];
        float sg[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const uint32_t en = (word[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
          const bool pad = en == 0xFFFFu;
          xv[q] = xt[pad ? 0u : (en & 0x7FFFu)];
          sg[q] = pad ? 0.f : ((en & 0x8000u) ? -1.f : 1.f);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) bd_add(sg[q] * xv[q].x, sg[q] * xv[q].y, s, e);
      }
    }
    bd_group_sum(s, e);
    if (b < d && h == 0) ts[(size_t)t * d + b] = bd_norm(s, e);
  }
}

// out[b] = scale * sum over tiles of ts[t * d + b]: tile t on lane t % 8 of
// the group of b, then the butterfly (the same order for every G).
__device__ void bd_tiles_reduce(const float2* ts, int ntile, int d, double scale, double* out) {
  const int g = threadIdx.x / kBH, h = threadIdx.x % kBH;
  for (int bb = g & ~3; bb < d; bb += kBT / kBH) {
    const int b = bb + (g & 3);
    float s = 0.f, e = 0.f;
    if (b < d) {
#pragma unroll 4
      for (int t = h; t < ntile; t += kBH) {
        const float2 v = __ldcg(ts + (size_t)t * d + b);
        bd_add(v.x, v.y, s, e);
      }
    }
    bd_group_sum(s, e);
    if (b < d && h == 0) out[b] = bd_to(bd_norm(s, e)) * scale;
  }
}

template <bool L2>
__device__ __forceinline__ float2 bd_ld(const float2* p) {
  return L2 ? __ldcg(p) : *p;
}

// Position of row i, column c of the tiled basis (m1 = m + 1 columns a tile).
__device__ __forceinline__ int64_t bd_uix(int64_t i, int c, int m1) {
  return ((i / kBR) * m1 + c) * (int64_t)kBR + (i % kBR);
}

// w = sg * A x for the rows of tile t (CSR), x = column j, w = column j + 1
// of the tiled basis; kBRowsPerThread rows per thread at a time.  L2: read x
// through L2 only (rows written by other CTAs).
template <bool L2>
__device__ __forceinline__ void bd_spmv_csr(const BdProb& P, int t, int m1, int j, float2 sg, float2* xs) {
  const int64_t r0 = (int64_t)t * kBR;
  const int rows = (int)min((int64_t)kBR, P.n - r0);
  float2* w = P.U + ((int64_t)t * m1 + j + 1) * kBR;
  int p0[kBRowsPerThread], len[kBRowsPerThread];
  int lmax = 0;
#pragma unroll
  for (int q = 0; q < kBRowsPerThread; ++q) {
    const int rr = threadIdx.x + q * kBT;
    p0[q] = 0;
    len[q] = 0;
    if (rr < rows) {
      p0[q] = P.rowptr[r0 + rr];
      len[q] = P.rowptr[r0 + rr + 1] - p0[q];
    }
    lmax = max(lmax, len[q]);
  }
  float s[kBRowsPerThread], e[kBRowsPerThread];
#pragma unroll
  for (int q = 0; q < kBRowsPerThread; ++q) { s[q] = 0.f; e[q] = 0.f; }
  for (int l = 0; l < lmax; ++l) {
    float2 a[kBRowsPerThread], v[kBRowsPerThread];
#pragma unroll
    for (int q = 0; q < kBRowsPerThread; ++q) {   // past a row's end: its last entry times 0
      const bool in = l < len[q];
      const int p = p0[q] + (in ? l : max(len[q] - 1, 0));
      const int col = len[q] > 0 ? P.colind[p] : 0;
      a[q] = len[q] > 0 ? P.vals[p] : make_float2(0.f, 0.f);
      if (!in) a[q] = make_float2(0.f, 0.f);
      v[q] = bd_ld<L2>(P.U + bd_uix(col, j, m1));
    }
#pragma unroll
    for (int q = 0; q < kBRowsPerThread; ++q) bd_mac(a[q].x, a[q].y, v[q].x, v[q].y, s[q], e[q]);
  }
#pragma unroll
  for (int q = 0; q < kBRowsPerThread; ++q) {
    const int rr = threadIdx.x + q * kBT;
    if (rr < rows) {
      const float2 y = bd_norm(s[q], e[q]);
      float s2 = 0.f, e2 = 0.f;
      bd_mac(y.x, y.y, sg.x, sg.y, s2, e2);
      const float2 o = bd_norm(s2, e2);
      w[rr] = o;
      xs[rr] = o;
    }
  }
}

// The same product from the diagonal storage (columns i + doff[e] in
// increasing order, as the CSR rows), ND diagonals.
template <bool L2, int ND, bool V32>
__device__ __forceinline__ void bd_spmv_dia_n(const BdProb& P, int t, int m1, int j, float2 sg, float2* xs) {
  const int64_t r0 = (int64_t)t * kBR, n = P.n, ld = P.ldu;
  const int rows = (int)min((int64_t)kBR, n - r0);
  float2* w = P.U + ((int64_t)t * m1 + j + 1) * kBR;
#pragma unroll
  for (int q = 0; q < kBRowsPerThread; ++q) {
    const int rq = threadIdx.x + q * kBT;
    const int rr = min(rq, rows - 1);   // rows past n read row n - 1 (never stored)
    float2 a[ND], v[ND];
#pragma unroll
    for (int dg = 0; dg < ND; ++dg) {
      const int64_t c = min(max(r0 + rr + P.doff[dg], (int64_t)0), n - 1);   // value 0 outside A
      const size_t ia = (size_t)dg * ld + r0 + rr;
      a[dg] = V32 ? make_float2(reinterpret_cast<const float*>(P.dvals)[ia], 0.f) : P.dvals[ia];
      v[dg] = bd_ld<L2>(P.U + bd_uix(c, j, m1));
    }
    float s = 0.f, e = 0.f;
#pragma unroll
    for (int dg = 0; dg < ND; ++dg) bd_mac(a[dg].x, a[dg].y, v[dg].x, v[dg].y, s, e);
    if (rq < rows) {
      const float2 y = bd_norm(s, e);
      float s2 = 0.f, e2 = 0.f;
      bd_mac(y.x, y.y, sg.x, sg.y, s2, e2);
      const float2 o = bd_norm(s2, e2);
      w[rq] = o;
      xs[rq] = o;
    }
  }
}

// Dispatch on the number of diagonals.
template <bool L2, bool V32>
__device__ __forceinline__ void bd_spmv_dia(const BdProb& P, int t, int m1, int j, float2 sg, float2* xs) {
  switch (P.D) {   // a compile-time number of diagonals: all loads of a row issued together
    case 1: bd_spmv_dia_n<L2, 1, V32>(P, t, m1, j, sg, xs); return;
    case 2: bd_spmv_dia_n<L2, 2, V32>(P, t, m1, j, sg, xs); return;
    case 3: bd_spmv_dia_n<L2, 3, V32>(P, t, m1, j, sg, xs); return;
    case 4: bd_spmv_dia_n<L2, 4, V32>(P, t, m1, j, sg, xs); return;
    case 5: bd_spmv_dia_n<L2, 5, V32>(P, t, m1, j, sg, xs); return;
    case 6: bd_spmv_dia_n<L2, 6, V32>(P, t, m1, j, sg, xs); return;
    case 7: bd_spmv_dia_n<L2, 7, V32>(P, t, m1, j, sg, xs); return;
    default: bd_spmv_dia_n<L2, 8, V32>(P, t, m1, j, sg, xs); return;
  }
}

// u~ = w + sum_c U[:, c] coef[c] (c <= j) for the rows of tile t, in place on
// column j + 1 (which holds w).  Thread p takes the row pairs (2 p, 2 p + 1),
// p = threadIdx.x, threadIdx.x + kBT (16-byte loads).
__device__ __forceinline__ void bd_update_full(float2* __restrict__ Ut, int j, const float2* coef, float2* xs) {
  constexpr int kPairs = kBR / (2 * kBT);
  float2* wcol = Ut + (size_t)(j + 1) * kBR;
  float s[2 * kPairs], e[2 * kPairs];
#pragma unroll
  for (int q = 0; q < kPairs; ++q) {
    const float4 w = *reinterpret_cast<const float4*>(wcol + 2 * (threadIdx.x + q * kBT));
    s[2 * q] = w.x; e[2 * q] = w.y; s[2 * q + 1] = w.z; e[2 * q + 1] = w.w;
  }
#pragma unroll 4
  for (int c = 0; c <= j; ++c) {
    const float2 cf = coef[c];
    const float2* col = Ut + (size_t)c * kBR;
    float4 u[kPairs];
#pragma unroll
    for (int q = 0; q < kPairs; ++q) u[q] = *reinterpret_cast<const float4*>(col + 2 * (threadIdx.x + q * kBT));
#pragma unroll
    for (int q = 0; q < kPairs; ++q) {
      bd_mac(u[q].x, u[q].y, cf.x, cf.y, s[2 * q], e[2 * q]);
      bd_mac(u[q].z, u[q].w, cf.x, cf.y, s[2 * q + 1], e[2 * q + 1]);
    }
  }
#pragma unroll
  for (int q = 0; q < kPairs; ++q) {
    const float2 a = bd_norm(s[2 * q], e[2 * q]), b = bd_norm(s[2 * q + 1], e[2 * q + 1]);
    const float4 o = make_float4(a.x, a.y, b.x, b.y);
    *reinterpret_cast<float4*>(wcol + 2 * (threadIdx.x + q * kBT)) = o;
    *reinterpret_cast<float4*>(xs + 2 * (threadIdx.x + q * kBT)) = o;
  }
}

__device__ __forceinline__ void bd_update_tile(const BdProb& P, int t, int m1, int j, const float2* coef,
                                              float2* xs) {
  constexpr int kPairs = kBR / (2 * kBT);
  const int rows = (int)min((int64_t)kBR, P.n - (int64_t)t * kBR);
  if (rows == kBR) {   // a full tile: no bounds tests between the loads
    bd_update_full(P.U + (int64_t)t * m1 * kBR, j, coef, xs);
    return;
  }
  const float2* Ut = P.U + (int64_t)t * m1 * kBR;
  float2* wcol = P.U + ((int64_t)t * m1 + j + 1) * kBR;
  float s[2 * kPairs], e[2 * kPairs];
#pragma unroll
  for (int q = 0; q < kPairs; ++q) {
    const int r = 2 * (threadIdx.x + q * kBT);
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r + 1 < rows) w = *reinterpret_cast<const float4*>(wcol + r);
    else if (r < rows) { const float2 w1 = wcol[r]; w.x = w1.x; w.y = w1.y; }
    s[2 * q] = w.x; e[2 * q] = w.y; s[2 * q + 1] = w.z; e[2 * q + 1] = w.w;
  }
#pragma unroll 4
  for (int c = 0; c <= j; ++c) {
    const float2 cf = coef[c];
    const float2* col = Ut + (size_t)c * kBR;
#pragma unroll
    for (int q = 0; q < kPairs; ++q) {
      const int r = 2 * (threadIdx.x + q * kBT);
      if (r + 1 < rows) {
        const float4 u = *reinterpret_cast<const float4*>(col + r);
        bd_mac(u.x, u.y, cf.x, cf.y, s[2 * q], e[2 * q]);
        bd_mac(u.z, u.w, cf.x, cf.y, s[2 * q + 1], e[2 * q + 1]);
      } else if (r < rows) {
        const float2 u = col[r];
        bd_mac(u.x, u.y, cf.x, cf.y, s[2 * q], e[2 * q]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kPairs; ++q) {
    const int r = 2 * (threadIdx.x + q * kBT);
    const float2 a = bd_norm(s[2 * q], e[2 * q]), b = bd_norm(s[2 * q + 1], e[2 * q + 1]);
    if (r + 1 < rows) {
      *reinterpret_cast<float4*>(wcol + r) = make_float4(a.x, a.y, b.x, b.y);
      *reinterpret_cast<float4*>(xs + r) = make_float4(a.x, a.y, b.x, b.y);
    } else if (r < rows) {
      wcol[r] = a;
      xs[r] = a;
    }
  }
}

// Restart product of the rows of tile t: U[:, l] = sum_c U[:, c] qc[c * ka + l]
// (l < ka, c < m), then U[:, ka] = U[:, m].  Each row is read whole before
// its first write.
template <int KM>
__device__ __noinline__ void bd_restart_tile(const BdProb& P, int t, int m, int ka, const float2* qc) {
  const int rows = (int)min((int64_t)kBR, P.n - (int64_t)t * kBR);
  float2* Ut = P.U + (int64_t)t * (m + 1) * kBR;
  for (int r = threadIdx.x; r < rows; r += kBT) {
    float s[KM], e[KM];
#pragma unroll
    for (int l = 0; l < KM; ++l) { s[l] = 0.f; e[l] = 0.f; }
#pragma unroll 4
    for (int c = 0; c < m; ++c) {
      const float2 u = Ut[(size_t)c * kBR + r];
#pragma unroll
      for (int l = 0; l < KM; ++l)
        if (l < ka) {
          const float2 q = qc[c * ka + l];
          bd_mac(u.x, u.y, q.x, q.y, s[l], e[l]);
        }
    }
    const float2 last = Ut[(size_t)m * kBR + r];
#pragma unroll
    for (int l = 0; l < KM; ++l)
      if (l < ka) Ut[(size_t)l * kBR + r] = bd_norm(s[l], e[l]);
    Ut[(size_t)ka * kBR + r] = last;
  }
}

// The passes over the tiles t0..t1-1 of this CTA, each a function of its own
// (own register allocation, one call per pass).  The sketch sums of tile t - 1
// are formed while the rows of tile t are computed; one barrier per tile.
// xs: two tile buffers in shared memory (tile t in buffer t % 2).
template <bool L2, bool V32>
__device__ __noinline__ void bd_pass_spmv(const BdProb& P, int t0, int t1, int m1, int j, float2 sg, int d,
                                          float2* ts, float2* xs) {
  for (int t = t0; t <= t1; ++t) {
    if (t < t1) {
      if (V32) bd_spmv_dia<L2, true>(P, t, m1, j, sg, xs + (t & 1) * kBR);
      else if (P.D > 0) bd_spmv_dia<L2, false>(P, t, m1, j, sg, xs + (t & 1) * kBR);
      else bd_spmv_csr<L2>(P, t, m1, j, sg, xs + (t & 1) * kBR);
    }
    if (t > t0) bd_bins_tile(P, d, t - 1, xs + ((t - 1) & 1) * kBR, ts);
    __syncthreads();
  }
}
__device__ __noinline__ void bd_pass_update(const BdProb& P, int t0, int t1, int m1, int j, const float2* coef, int d,
                                            float2* ts, float2* xs) {
  for (int t = t0; t <= t1; ++t) {
    if (t < t1) bd_update_tile(P, t, m1, j, coef, xs + (t & 1) * kBR);
    if (t > t0) bd_bins_tile(P, d, t - 1, xs + ((t - 1) & 1) * kBR, ts);
    __syncthreads();
  }
}
__device__ __noinline__ void bd_pass_start(const BdProb& P, int t0, int t1, int m1, uint64_t seed, int d, float2* ts,
                                           float2* xs) {
  for (int t = t0; t <= t1; ++t) {
    if (t < t1) {
      const int64_t r0 = (int64_t)t * kBR;
      const int rows = (int)min((int64_t)kBR, P.n - r0);
      float2* col = P.U + (int64_t)t * m1 * kBR;
      float2* x = xs + (t & 1) * kBR;
      for (int r = threadIdx.x; r < rows; r += kBT) {
        const float2 v = bd_from(bd_normal(seed, r0 + r));
        col[r] = v;
        x[r] = v;
      }
    }
    if (t > t0) bd_bins_tile(P, d, t - 1, xs + ((t - 1) & 1) * kBR, ts);
    __syncthreads();
  }
}

// cluster-wide barrier; the fence orders this thread's global writes before it
__device__ __forceinline__ void bd_cluster_sync(cg::cluster_group& cl) {
  __threadfence();
  cl.sync();
}

// Fixed-order sum over the CTA of 4 doubles per thread (warp butterflies,
// then the warps in order); the result in v[] of every thread.
__device__ void bd_block_sum4(double v[4], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = warp_sum(v[q]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 4; ++q) red[warp * 4 + q] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double a = 0.0;
    for (int w = 0; w < kBT / 32; ++w) a += red[w * 4 + q];
    v[q] = a;
  }
  __syncthreads();
}

// The residual sums of one tile for the Ritz vector in X column col (and
// col + 1 for a pair): ||A x - l x||^2, ||x||^2, Re and Im of x^H A x.
__device__ __noinline__ void bd_resid_tile(const BdProb& P, int64_t r0, int rows, const double* xr, const double* xi,
                                           bool pair, double lr, double li, double* red, double* out4) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int rr = threadIdx.x; rr < rows; rr += kBT) {
    const int64_t i = r0 + rr;
    double ar = 0.0, ai = 0.0;
    for (int p = P.rowptr[i]; p < P.rowptr[i + 1]; ++p) {
      const double a = bd_to(P.vals[p]);
      const int cc = P.colind[p];
      ar += a * __ldcg(xr + cc);
      if (pair) ai += a * __ldcg(xi + cc);
    }
    const double x0 = __ldcg(xr + i), x1 = pair ? __ldcg(xi + i) : 0.0;
    const double re = ar - lr * x0 + li * x1, im = ai - li * x0 - lr * x1;
    v[0] += re * re + im * im;
    v[1] += x0 * x0 + x1 * x1;
    v[2] += x0 * ar + x1 * ai;
    v[3] += x0 * ai - x1 * ar;
  }
  bd_block_sum4(v, red);
  if (threadIdx.x < 4) out4[threadIdx.x] = v[threadIdx.x];
}

// The warp-0 stages of the contraction, each with its own register
// allocation: Hessenberg reduction, Francis QR, reordering with the kept size
// (blocks covering `want` columns, pairs whole, at most m - 1), Ritz pairs.
__device__ __noinline__ void bd_hess(int m, DenseR* T, DenseR* Q, DenseR* v, int lane) {
  rks_dd::hessenberg(m, T, m, Q, m, v, lane);
}
__device__ __noinline__ int bd_francis(int m, DenseR* T, DenseR* Q, int lane) {
  return rks_dd::schur(m, T, m, Q, m, m, lane);
}
__device__ __noinline__ int bd_reorder_truncate(int m, DenseR* T, DenseR* Q, int which, int want,
                                                DenseR* keys, int lane) {
  return min(rks_dd::reorder_select(m, T, m, Q, m, m, which, want, keys, lane), m - 1);
}
__device__ __noinline__ void bd_quasi_eig(int ka, int m, const DenseR* T, DenseR* lre, DenseR* lim,
                                          DenseR* Yr, DenseR* Yi, int lane) {
  rks_dd::quasi_eig(ka, T, m, lre, lim, Yr, Yi, m, lane);
}

// ---------------------------------------------------------------------------
// one problem, by one cluster
// ---------------------------------------------------------------------------

__device__ void bd_solve(const BdArgs& A, const BdProb& P, double* sm, BdShared& sh, cg::cluster_group& cl,
                         long long* pacc, long long& tlast) {
  using df = DenseR;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#define BD_MARK(ph)                     \
  if (tid == 0) {                       \
    const long long tnow = clock64();   \
    pacc[ph] += tnow - tlast;           \
    tlast = tnow;                       \
  }
  const int m = A.m, d = A.d, k = A.k;
  const int G = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const BdLayout L = bd_layout(m, d);
  double* S = sm + L.S;
  double* B = sm + L.B;
  df* T = reinterpret_cast<df*>(sm + L.T);
  df* Q = reinterpret_cast<df*>(sm + L.Q);
  double* Td = sm + L.Td;
  double* Qd = sm + L.Qd;
  double* W = sm + L.W;
  double* Gm = sm + L.G;
  double* Ri = sm + L.Ri;
  double* Yp = sm + L.QC;
  float2* qc = reinterpret_cast<float2*>(sm + L.QC);
  double* z = sm + L.z;
  double* sv = sm + L.sv;
  double* r = sm + L.r;
  double* sig = sm + L.sig;
  float2* coef = reinterpret_cast<float2*>(sm + L.coef);
  double* bk = sm + L.bk;
  double* lre = sm + L.lre;
  double* lim = sm + L.lim;
  double* est = sm + L.est;
  double* scr = sm + L.scr;
  df* scr_df = reinterpret_cast<df*>(scr);
  float2* xs = reinterpret_cast<float2*>(sm + L.xs);
  df* Yr = reinterpret_cast<df*>(W);
  df* Yi = reinterpret_cast<df*>(W) + m * m;
  const int ldb = m + 1;
  const int kp1 = k + 1;
  const int64_t n = P.n, ld = P.ldu;
  const int m1 = m + 1;
  const int t0 = (int)((int64_t)P.ntile * rank / G), t1 = (int)((int64_t)P.ntile * (rank + 1) / G);
  const int64_t lo = min((int64_t)t0 * kBR, n), hi = min((int64_t)t1 * kBR, n);
  const double zscale = 1.0 / sqrt((double)A.zeta);
  const double tiny = 2.2250738585072014e-308;
  int ex = 0;
  double tol = A.tol;
  const int maxit = A.tune > 0 ? A.tune : A.maxit;
  int restarts = 0, status = RKS_OK, nw = 0, converged = 0, whit = 0, ka = 0, nconv = 0;
  int64_t nmatvec = 0;
  double max_est = 0.0, max_res = 0.0;
  bool have_ritz = false;

  // ---- start (Sec. 3.1 with k = 0): U[:, 0] = u~_1, S[:, 0] = Omega u~_1 / beta
  {
    float2* ts = P.tsum + (size_t)(ex & 1) * P.ntile * d;
    bd_pass_start(P, t0, t1, m1, A.seed + 1, d, ts, xs);
    bd_cluster_sync(cl);
    bd_tiles_reduce(ts, P.ntile, d, zscale, sv);
    ++ex;
    __syncthreads();
    if (warp == 0) {
      double a = 0.0;
      for (int i = lane; i < d; i += 32) a += sv[i] * sv[i];
      a = warp_sum(a);
      if (lane == 0) sh.red[0] = sqrt(a);
    }
    for (int t = tid; t < (m + 1) * m; t += kBT) B[t] = 0.0;
    __syncthreads();
    const double beta = sh.red[0];
    if (!(beta > 0.0) || !isfinite(beta)) status = isfinite(beta) ? RKS_EBREAKDOWN : RKS_ENAN;
    for (int i = tid; i < d; i += kBT) S[i] = sv[i] / beta;
    if (tid == 0) sig[0] = 1.0 / beta;
    __syncthreads();
    BD_MARK(kPhStart);
  }
  int ja = 0;
  while (status == RKS_OK) {
    // ---- Algorithm 2: extension from ja to m columns
    for (int j = ja; j < m; ++j) {
      float2* ts = P.tsum + (size_t)(ex & 1) * P.ntile * d;
      const float2 sg = bd_from(sig[j]);
      // w = A u_j, partial z = Omega w (FP32 diagonals when A's values are FP32 numbers)
      if (P.dv32) {
        if (G > 1) bd_pass_spmv<true, true>(P, t0, t1, m1, j, sg, d, ts, xs);
        else bd_pass_spmv<false, true>(P, t0, t1, m1, j, sg, d, ts, xs);
      } else {
        if (G > 1) bd_pass_spmv<true, false>(P, t0, t1, m1, j, sg, d, ts, xs);
        else bd_pass_spmv<false, false>(P, t0, t1, m1, j, sg, d, ts, xs);
      }
      BD_MARK(kPhSpmvRows);
      bd_cluster_sync(cl);
      bd_tiles_reduce(ts, P.ntile, d, zscale, z);
      ++ex;
      __syncthreads();
      BD_MARK(kPhExchange);
      // b = S_j^+ z by CGS2 on the sketches: r1 = S^T z, r = r1 + S^T (z - S r1)
      for (int c = warp; c <= j; c += kBT / 32) {
        double a = 0.0;
        for (int i = lane; i < d; i += 32) a += S[i + (size_t)c * d] * z[i];
        a = warp_sum(a);
        if (lane == 0) r[c] = a;
      }
      __syncthreads();
      for (int i = tid; i < d; i += kBT) {
        double a = z[i];
        for (int c = 0; c <= j; ++c) a -= S[i + (size_t)c * d] * r[c];
        sv[i] = a;
      }
      __syncthreads();
      for (int c = warp; c <= j; c += kBT / 32) {
        double a = 0.0;
        for (int i = lane; i < d; i += 32) a += S[i + (size_t)c * d] * sv[i];
        a = warp_sum(a);
        if (lane == 0) {
          r[c] += a;
          coef[c] = bd_from(-sig[c] * r[c]);
        }
      }
      __syncthreads();
      BD_MARK(kPhLs);
      ts = P.tsum + (size_t)(ex & 1) * P.ntile * d;
      bd_pass_update(P, t0, t1, m1, j, coef, d, ts, xs);   // u~ = w - U b, partial s~ = Omega u~
      BD_MARK(kPhUpdRows);
      bd_cluster_sync(cl);
      bd_tiles_reduce(ts, P.ntile, d, zscale, sv);
      ++ex;
      ++nmatvec;
      __syncthreads();
      BD_MARK(kPhExchange);
      if (warp == 0) {                                  // beta = ||s~||
        double a = 0.0, zz = 0.0;
        for (int i = lane; i < d; i += 32) { a += sv[i] * sv[i]; zz += z[i] * z[i]; }
        a = warp_sum(a);
        zz = warp_sum(zz);
        if (lane == 0) { sh.red[0] = sqrt(a); sh.red[1] = sqrt(zz); }
      }
      __syncthreads();
      const double beta = sh.red[0];
      if (!(beta > 1e-14 * sh.red[1]) || !isfinite(beta)) {
        status = isfinite(beta) ? RKS_EBREAKDOWN : RKS_ENAN;
        break;
      }
      for (int i = tid; i < d; i += kBT) S[i + (size_t)(j + 1) * d] = sv[i] / beta;
      for (int c = tid; c <= j; c += kBT) B[c + (size_t)j * ldb] = r[c];
      if (tid == 0) {
        B[(j + 1) + (size_t)j * ldb] = beta;
        sig[j + 1] = 1.0 / beta;
      }
      __syncthreads();
      BD_MARK(kPhBeta);
    }
    if (status != RKS_OK) break;

    // ---- contraction (Algorithm 1): Schur form, reordering, truncation (warp 0, double-float)
    if (warp == 0) {
      for (int t = lane; t < m * m; t += 32) T[t] = df(B[(t % m) + (size_t)(t / m) * ldb]);
      __syncwarp();
      bd_hess(m, T, Q, scr_df, lane);
      BD_MARK(kPhHess);
      const int rc = bd_francis(m, T, Q, lane);
      BD_MARK(kPhSchur);
      const int kt = rc == 0 ? bd_reorder_truncate(m, T, Q, A.which, A.want, reinterpret_cast<df*>(W), lane) : 0;
      if (lane == 0) {
        sh.flag[0] = rc ? RKS_EDENSE : RKS_OK;
        sh.flag[1] = kt;
      }
    }
    __syncthreads();
    BD_MARK(kPhDense);
    if (sh.flag[0] != RKS_OK) { status = sh.flag[0]; break; }
    ka = sh.flag[1];
    // FP64 copies of the kept part: Q_k (m x ka, ld m) and T_a (ka x ka, ld m)
    for (int t = tid; t < m * ka; t += kBT) Qd[t] = (double)Q[t];
    for (int t = tid; t < m * ka; t += kBT) Td[t] = (double)T[t];
    __syncthreads();
    // kept sketches S Q_k and b^T Q_k
    for (int t = tid; t < d * ka; t += kBT) {
      const int i = t % d, l = t / d;
      double a = 0.0;
      for (int c = 0; c < m; ++c) a += S[i + (size_t)c * d] * Qd[c + l * m];
      W[t] = a;
    }
    for (int l = tid; l < ka; l += kBT) {
      double a = 0.0;
      for (int c = 0; c < m; ++c) a += B[m + (size_t)c * ldb] * Qd[c + l * m];
      bk[l] = a;
    }
    __syncthreads();
    // Gram matrix of the kept sketches; whitening when it drifted (Sec. 3.3)
    for (int t = tid; t < ka * ka; t += kBT) {
      const int a = t % ka, b = t / ka;
      double s = 0.0;
      for (int i = 0; i < d; ++i) s += W[i + (size_t)a * d] * W[i + (size_t)b * d];
      Gm[t] = s;
    }
    __syncthreads();
    if (warp == 0) {
      double e2 = 0.0;
      for (int t = lane; t < ka * ka; t += 32) {
        const double e = Gm[t] - ((t % ka) == (t / ka) ? 1.0 : 0.0);
        e2 += e * e;
      }
      e2 = warp_sum(e2);
      if (lane == 0) sh.flag[2] = sqrt(e2) > 1e-10 ? 1 : 0;
    }
    __syncthreads();
    if (sh.flag[2]) {
      // G = R^T R (Cholesky; R is the triangular factor of S Q_k = Q_s R with
      // a positive diagonal); T_a <- R T_a R^{-1}, b <- b R^{-1},
      // Q_k <- Q_k R^{-1}, S Q_k <- S Q_k R^{-1} = Q_s
      if (tid == 0) {
        int ok = 1;
        for (int j = 0; j < ka && ok; ++j) {
          double dd = Gm[j + j * ka];
          for (int l = 0; l < j; ++l) dd -= Gm[l + j * ka] * Gm[l + j * ka];
          if (!(dd > 0.0)) { ok = 0; break; }
          const double rjj = sqrt(dd);
          Gm[j + j * ka] = rjj;
          for (int c = j + 1; c < ka; ++c) {
            double a = Gm[j + c * ka];
            for (int l = 0; l < j; ++l) a -= Gm[l + j * ka] * Gm[l + c * ka];
            Gm[j + c * ka] = a / rjj;
          }
        }
        if (ok) {
          for (int j = 0; j < ka; ++j) {
            for (int i = 0; i < ka; ++i) Ri[i + j * ka] = 0.0;
            Ri[j + j * ka] = 1.0 / Gm[j + j * ka];
            for (int i = j - 1; i >= 0; --i) {
              double a = 0.0;
              for (int l = i + 1; l <= j; ++l) a += Gm[i + l * ka] * Ri[l + j * ka];
              Ri[i + j * ka] = -a / Gm[i + i * ka];
            }
          }
        }
        sh.flag[3] = ok;
      }
      __syncthreads();
      if (!sh.flag[3]) { status = RKS_EDENSE; break; }
      for (int i = tid; i < ka; i += kBT) {          // T_a R^{-1}: row i by thread i
        double row[kBMaxKa];
        for (int c = 0; c < ka; ++c) {
          double a = 0.0;
          for (int l = 0; l <= c; ++l) a += Td[i + l * m] * Ri[l + c * ka];
          row[c] = a;
        }
        for (int c = 0; c < ka; ++c) Td[i + c * m] = row[c];
      }
      __syncthreads();
      for (int c = tid; c < ka; c += kBT) {          // R (T_a R^{-1}): column c by thread c
        double col[kBMaxKa];
        for (int i = 0; i < ka; ++i) {
          double a = 0.0;
          for (int l = i; l < ka; ++l) a += Gm[i + l * ka] * Td[l + c * m];
          col[i] = a;
        }
        for (int i = 0; i < ka; ++i) Td[i + c * m] = col[i];
      }
      for (int i = tid; i < m + d + 1; i += kBT) {   // rows of Q_k, of S Q_k, and b^T Q_k
        double* base;
        int ldx;
        if (i < m) { base = Qd + i; ldx = m; }
        else if (i < m + d) { base = W + (i - m); ldx = d; }
        else { base = bk; ldx = 1; }
        double row[kBMaxKa];
        for (int c = 0; c < ka; ++c) {
          double a = 0.0;
          for (int l = 0; l <= c; ++l) a += base[(size_t)l * ldx] * Ri[l + c * ka];
          row[c] = a;
        }
        for (int c = 0; c < ka; ++c) base[(size_t)c * ldx] = row[c];
      }
      __syncthreads();
      for (int t = tid; t < m * ka; t += kBT) {      // the whitened T_a for the Ritz step
        if (t % m < ka) T[t] = df(Td[t]);
      }
      ++whit;
      __syncthreads();
    }
    // restart coefficients sig_c Q'[c, l] and the restart product (Eq. 3.5)
    for (int t = tid; t < m * ka; t += kBT) {
      const int c = t / ka, l = t % ka;
      qc[t] = bd_from(sig[c] * Qd[c + l * m]);
    }
    __syncthreads();
    BD_MARK(kPhKept);
    for (int t = t0; t < t1; ++t) {
      if (ka <= 16) bd_restart_tile<16>(P, t, m, ka, qc);
      else bd_restart_tile<kBMaxKa>(P, t, m, ka, qc);
    }
    // S <- [S Q', s], B <- [T_a; b^T Q'], sig <- [1 .. 1, sig_m]
    for (int i = tid; i < d; i += kBT) {
      const double last = S[i + (size_t)m * d];
      for (int l = 0; l < ka; ++l) S[i + (size_t)l * d] = W[i + (size_t)l * d];
      S[i + (size_t)ka * d] = last;
    }
    for (int t = tid; t < (m + 1) * m; t += kBT) {
      const int row = t % ldb, col = t / ldb;
      double v = 0.0;
      if (col < ka) v = row < ka ? Td[row + col * m] : (row == ka ? bk[col] : 0.0);
      B[t] = v;
    }
    __syncthreads();
    if (tid == 0) {
      sig[ka] = sig[m];
      for (int l = 0; l < ka; ++l) sig[l] = 1.0;
    }
    ++restarts;
    __syncthreads();
    BD_MARK(kPhRestart);
    // Ritz pairs of T_a (double-float) and the estimates |b^T y| / scale, best first (warp 0)
    if (warp == 0) {
      bd_quasi_eig(ka, m, T, scr_df, scr_df + m, Yr, Yi, lane);
      for (int t = lane; t < ka; t += 32) {
        lre[t] = (double)scr_df[t];
        lim[t] = (double)scr_df[m + t];
        double br = 0.0, bi = 0.0;
        for (int c = 0; c < ka; ++c) {
          br += bk[c] * (double)Yr[c + t * m];
          bi += bk[c] * (double)Yi[c + t * m];
        }
        const double den = A.conv == RKS_CONV_NORM1 ? P.norm1 : fmax(hypot(lre[t], lim[t]), tiny);
        est[t] = hypot(br, bi) / den;
      }
      __syncwarp();
      if (lane == 0) {   // stable sort by key
        for (int t = 0; t < ka; ++t) sh.ord[t] = t;
        for (int t = 1; t < ka; ++t) {
          const int o = sh.ord[t];
          const double kv = rks_dd::key(lre[o], lim[o], A.which);
          int u = t - 1;
          while (u >= 0 && rks_dd::key(lre[sh.ord[u]], lim[sh.ord[u]], A.which) > kv) {
            sh.ord[u + 1] = sh.ord[u];
            --u;
          }
          sh.ord[u + 1] = o;
        }
        int nwl = min(k, ka);
        if (nwl > 0 && nwl < ka && lim[sh.ord[nwl - 1]] > 0.0) ++nwl;
        double mx = 0.0;
        int nc = 0;
        for (int t = 0; t < nwl; ++t) {
          mx = fmax(mx, est[sh.ord[t]]);
          nc += est[sh.ord[t]] <= tol;
        }
        sh.flag[4] = nwl;
        sh.flag[5] = nc;
        sh.red[2] = mx;
      }
    }
    __syncthreads();
    nw = sh.flag[4];
    nconv = sh.flag[5];
    max_est = sh.red[2];
    have_ritz = true;
    const bool conv_now = max_est <= tol;
    bd_cluster_sync(cl);   // restarted rows visible to the cluster
    BD_MARK(kPhRitz);
    if (!conv_now && restarts < maxit) {
      ja = ka;
      continue;
    }
    // ---- Ritz vectors X = U_k Y (real packing) and their FP64 residuals
    for (int t = tid; t < nw * ka; t += kBT) {
      const int c = t % ka, col = t / ka;
      const int o = sh.ord[col];
      Yp[c + col * ka] = lim[o] < 0.0 ? (double)Yi[c + sh.ord[col - 1] * m] : (double)Yr[c + o * m];
    }
    __syncthreads();
    for (int64_t i = lo + tid; i < hi; i += kBT) {
      double u[kBMaxKa];
      for (int c = 0; c < ka; ++c) u[c] = bd_to(P.U[bd_uix(i, c, m1)]);
      for (int col = 0; col < nw; ++col) {
        double a = 0.0;
        for (int c = 0; c < ka; ++c) a += u[c] * Yp[c + col * ka];
        P.X[i + (size_t)col * ld] = a;
      }
    }
    bd_cluster_sync(cl);
    for (int t = t0; t < t1; ++t) {
      const int64_t r0 = (int64_t)t * kBR;
      const int rows = (int)min((int64_t)kBR, n - r0);
      for (int col = 0; col < nw; ++col) {
        const int o = sh.ord[col];
        if (lim[o] < 0.0) continue;                     // the first member covers the pair
        const bool pair = lim[o] > 0.0;
        const double* xr = P.X + (size_t)col * ld;
        const double* xi = pair ? P.X + (size_t)(col + 1) * ld : xr;
        bd_resid_tile(P, r0, rows, xr, xi, pair, lre[o], lim[o], sh.red + 8, P.rsum + ((size_t)t * kp1 + col) * 4);
      }
    }
    bd_cluster_sync(cl);
    for (int q = tid; q < nw * 4; q += kBT) {          // sum over tiles, in tile order
      const int col = q / 4, qq = q % 4;
      double a = 0.0;
      if (lim[sh.ord[col]] >= 0.0)
        for (int t = 0; t < P.ntile; ++t) a += __ldcg(P.rsum + ((size_t)t * kp1 + col) * 4 + qq);
      scr[q] = a;
    }
    __syncthreads();
    max_res = 0.0;
    for (int col = 0; col < nw; ++col) {
      const int base = (lim[sh.ord[col]] < 0.0 ? col - 1 : col) * 4;
      const double res = sqrt(scr[base]) / (P.norm1 * sqrt(scr[base + 1]));
      max_res = fmax(max_res, isfinite(res) ? res : INFINITY);
    }
    const bool verified = !(A.verify > 0.0) || max_res <= A.verify;
    if (conv_now && !verified && restarts < maxit) {
      tol *= 0.25;
      bd_cluster_sync(cl);   // every CTA has read rsum before it is written again
      BD_MARK(kPhFinal);
      ja = ka;
      continue;
    }
    BD_MARK(kPhFinal);
    converged = conv_now && verified;
    if (rank == 0) {
      for (int col = tid; col < nw; col += kBT) {
        const int o = sh.ord[col];
        const bool second = lim[o] < 0.0;
        const int base = (second ? col - 1 : col) * 4;
        const double xx = scr[base + 1];
        double* slot = P.out + (size_t)col * kBSlot;
        slot[0] = lre[o];
        slot[1] = lim[o];
        slot[2] = sqrt(scr[base]) / (P.norm1 * sqrt(xx));
        slot[3] = scr[base + 2] / xx;
        slot[4] = (second ? -1.0 : 1.0) * scr[base + 3] / xx;
        slot[5] = est[o];
      }
    }
    break;
  }
  if (rank == 0 && tid == 0) {
    if (status == RKS_OK && !converged) status = RKS_ENOCONV;
    P.info[kIStatus] = status;
    P.info[kIRestarts] = restarts;
    P.info[kIMatvec] = (int)nmatvec;
    P.info[kINw] = have_ritz && (status == RKS_OK || status == RKS_ENOCONV) ? nw : 0;
    P.info[kIConv] = converged;
    P.info[kIWhiten] = whit;
    P.info[kINconv] = nconv;
    P.out[(size_t)kp1 * kBSlot] = max_est;
    P.out[(size_t)kp1 * kBSlot + 1] = max_res;
  }
#undef BD_MARK
}

__global__ void __launch_bounds__(kBT, 2) k_batch_rks(BdArgs A) {
  extern __shared__ __align__(16) double bd_dyn[];
  __shared__ BdShared sh;
  double* sm = bd_dyn;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned G = cl.num_blocks();
  long long pacc[kPhases];
  for (int q = 0; q < kPhases; ++q) pacc[q] = 0;
  long long tlast = clock64();
  for (int guard = 0; guard <= A.count; ++guard) {
    if (cl.block_rank() == 0 && threadIdx.x == 0) {
      // one atomic add on both counters: the old value tells how many
      // positions either end had taken, so the two ends never overlap
      const unsigned long long old = atomicAdd(A.queue, A.dir ? (1ull << 32) : 1ull);
      const int head = (int)(old & 0xffffffffull), tail = (int)(old >> 32);
      const int p = head + tail < A.count ? A.order[A.dir ? A.count - 1 - tail : head] : -1;
      for (unsigned r = 0; r < G; ++r) *cl.map_shared_rank(&sh.prob, r) = p;
    }
    cl.sync();
    const int p = sh.prob;
    if (threadIdx.x == 0) {
      const long long tnow = clock64();
      pacc[kPhQueue] += tnow - tlast;
      tlast = tnow;
    }
    if (p < 0) break;
    bd_solve(A, A.probs[p], sm, sh, cl, pacc, tlast);
    cl.sync();   // every CTA has read sh.prob before rank 0 writes the next one
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < kPhases; ++q) atomicAdd(A.phase + q, (unsigned long long)pacc[q]);
}

// The device dense step on one matrix (test entry point): one warp, the
// matrices in global memory, double-float arithmetic (as in the solver).
__global__ void k_dense_test(int m, const double* B, DenseR* T, DenseR* Q, int which, int nsort,
                             DenseR* lre, DenseR* lim, DenseR* Yr, DenseR* Yi, DenseR* scratch,
                             int* status) {
  const int lane = threadIdx.x;
  for (int t = lane; t < m * m; t += 32) T[t] = dense_from(B[t]);
  __syncwarp();
  rks_dd::hessenberg(m, T, m, Q, m, scratch, lane);
  const int rc = rks_dd::schur(m, T, m, Q, m, m, lane);
  int fails = 0;
  if (rc == 0) {
    const int top = rks_dd::reorder_select(m, T, m, Q, m, m, which, nsort, scratch + m, lane);
    fails = top < min(nsort, m) ? 1 : 0;
    rks_dd::quasi_eig(m, T, m, lre, lim, Yr, Yi, m, lane);
  }
  if (lane == 0) status[0] = rc ? RKS_EDENSE : fails;
}

__global__ void k_df_to_double(int64_t count, const DenseR* in, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

uint64_t mix64_host(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Tile bin lists of Omega for one problem.  For tile t (rows t kBR ..) and
// sketch row b, the rows of the tile with Omega[b, row] != 0 in increasing
// order are cut into kBH consecutive chunks of ceil(c / kBH) entries (chunk
// h for lane h), each padded with 0xFFFF to a common length P, a multiple of
// 8 (one 16-byte load per 8 entries); the block of (t, b) starts at
// tbin[t * (d + 1) + b] and holds kBH * P entries.  Entry = row in tile |
// 0x8000 for a negative sign.  Column i of Omega: base = mix(seed * gamma +
// i), draws mix(base + (r + 1) gamma), row = high 32 bits * d >> 32, sign =
// low bit, repeated rows skipped (the hash of rks_sketch_pairs).  false if a
// column could not draw zeta distinct rows.
bool build_bins(int64_t n, int d, int zeta, uint64_t seed, std::vector<int32_t>& tbin, std::vector<uint16_t>& ent) {
  const uint64_t gamma = 0x9E3779B97F4A7C15ull;
  const int ntile = (int)((n + kBR - 1) / kBR);
  tbin.assign((size_t)ntile * (d + 1), 0);
  ent.clear();
  ent.reserve((size_t)n * zeta * 5 / 4 + 64);
  std::vector<int> rows((size_t)kBR * zeta);
  std::vector<uint16_t> tag((size_t)kBR * zeta);
  std::vector<int> cnt(d + 1), cur(d);
  std::vector<uint16_t> list((size_t)kBR * zeta);
  for (int t = 0; t < ntile; ++t) {
    const int64_t r0 = (int64_t)t * kBR;
    const int nr = (int)std::min<int64_t>(kBR, n - r0);
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int q = 0; q < nr; ++q) {
      const uint64_t base = mix64_host(seed * gamma + (uint64_t)(r0 + q));
      int got = 0;
      for (int r = 0; r < 32 * zeta && got < zeta; ++r) {
        const uint64_t h = mix64_host(base + (uint64_t)(r + 1) * gamma);
        const int row = (int)(((h >> 32) * (uint64_t)d) >> 32);
        bool dup = false;
        for (int u = 0; u < got; ++u) dup |= rows[(size_t)q * zeta + u] == row;
        if (dup) continue;
        rows[(size_t)q * zeta + got] = row;
        tag[(size_t)q * zeta + got] = (uint16_t)(q | ((h & 1ull) ? 0x8000 : 0));
        ++got;
      }
      if (got < zeta) return false;
      for (int u = 0; u < zeta; ++u) ++cnt[rows[(size_t)q * zeta + u] + 1];
    }
    // the plain lists, increasing row within every list
    std::vector<int> loff(d + 1, 0);
    for (int b = 0; b < d; ++b) loff[b + 1] = loff[b] + cnt[b + 1];
    for (int b = 0; b < d; ++b) cur[b] = loff[b];
    for (int q = 0; q < nr; ++q)
      for (int u = 0; u < zeta; ++u) list[cur[rows[(size_t)q * zeta + u]]++] = tag[(size_t)q * zeta + u];
    // padded lane chunks
    int32_t* off = tbin.data() + (size_t)t * (d + 1);
    for (int b = 0; b < d; ++b) {
      const int c = loff[b + 1] - loff[b];
      const int s = (c + kBH - 1) / kBH;
      const int P = (s + 7) / 8 * 8;
      off[b] = (int32_t)ent.size();
      for (int h = 0; h < kBH; ++h)
        for (int u = 0; u < P; ++u) {
          const int e = h * s + u;
          ent.push_back(u < s && e < c ? list[loff[b] + e] : (uint16_t)0xFFFF);
        }
    }
    off[d] = (int32_t)ent.size();
  }
  if (ent.size() >= ((size_t)1 << 31)) return false;
  if (ent.empty()) ent.push_back(0xFFFF);
  return true;
}

// Diagonal storage of a CSR matrix with at most kBMaxDiag distinct offsets
// column - row, each row's columns increasing and distinct: doff (increasing)
// and dv[e * ldu + i] (zero where the row has no entry on diagonal e).
// Returns the number of diagonals, or 0 when the matrix does not qualify.
int build_dia(int64_t n, int64_t ldu, const int32_t* rowptr, const int32_t* colind, const std::vector<float2>& vals,
              int* doff, std::vector<float2>& dv) {
  int D = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      if (p > rowptr[i] && colind[p] <= colind[p - 1]) return 0;
      const int o = (int)((int64_t)colind[p] - i);
      bool have = false;
      for (int e = 0; e < D; ++e) have |= doff[e] == o;
      if (have) continue;
      if (D == kBMaxDiag) return 0;
      doff[D++] = o;
    }
  std::sort(doff, doff + D);
  dv.assign((size_t)std::max(D, 1) * ldu, make_float2(0.f, 0.f));
  for (int64_t i = 0; i < n; ++i)
    for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const int o = (int)((int64_t)colind[p] - i);
      const int e = (int)(std::lower_bound(doff, doff + D, o) - doff);
      dv[(size_t)e * ldu + i] = vals[p];
    }
  return D;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct rks_dbatch {
  int device = 0, count = 0, k = 0, p = 0, m = 0, d = 0, zeta = 8, which = 0, maxit = 1000, conv = 0, want = 0;
  double tol = 0.0, verify = 0.0;
  uint64_t seed = 0;
  // launch configuration: nL clusters of GL CTAs take problems from the
  // front (largest first), nS clusters of GS CTAs from the back (nS = 0: one kernel)
  int GL = 1, nL = 0, GS = 0, nS = 0;
  size_t smem = 0;
  int64_t nmax = 0;
  std::vector<int64_t> n;
  std::vector<BdProb> probs;
  std::vector<float> tune_ms;   // tuning runs, one per candidate configuration
  char* pool = nullptr;
  BdProb* d_probs = nullptr;
  int* d_order = nullptr;
  unsigned long long* d_queue = nullptr;
  int* d_info = nullptr;
  double* d_out = nullptr;
  unsigned long long* d_phase = nullptr;
  unsigned long long phase[kPhases] = {};
  cudaStream_t stream = nullptr, stream2 = nullptr;
  bool own_stream = false;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr, fork = nullptr, join = nullptr;
  std::vector<int> info;
  std::vector<double> out;
  bool solved = false;
  float last_ms = 0.f;
};

namespace {

int out_stride(const rks_dbatch* b) { return (b->k + 1) * kBSlot + 2; }

void cluster_cfg(const rks_dbatch* b, int G, int grid, cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr) {
  cfg = cudaLaunchConfig_t{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBT);
  cfg.dynamicSmemBytes = b->smem;
  cfg.stream = b->stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = G;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
}

cudaError_t launch_kernel(rks_dbatch* b, cudaStream_t st, int G, int nclusters, int dir, int tune) {
  BdArgs a;
  a.probs = b->d_probs;
  a.order = b->d_order;
  a.queue = b->d_queue;
  a.dir = dir;
  a.tune = tune;
  a.nmax = b->nmax;
  a.count = b->count;
  a.k = b->k;
  a.m = b->m;
  a.d = b->d;
  a.zeta = b->zeta;
  a.which = b->which;
  a.maxit = b->maxit;
  a.want = b->want;
  a.conv = b->conv;
  a.tol = b->tol;
  a.verify = b->verify;
  a.seed = b->seed;
  a.phase = b->d_phase;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cluster_cfg(b, G, nclusters * G, cfg, attr);
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, k_batch_rks, a);
}

// The whole launch on b->stream: queue and counters reset, the front kernel,
// and the back kernel (if any) on a second stream forked and joined by events.
cudaError_t launch_batch(rks_dbatch* b, int GL, int nL, int GS, int nS, int tune) {
  cudaError_t e = cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long), b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_phase, 0, sizeof(unsigned long long) * kPhases, b->stream);
  if (e != cudaSuccess) return e;
  if (nS > 0) {
    if ((e = cudaEventRecord(b->fork, b->stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(b->stream2, b->fork, 0)) != cudaSuccess) return e;
    if ((e = launch_kernel(b, b->stream2, GS, nS, 1, tune)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(b->join, b->stream2)) != cudaSuccess) return e;
  }
  if ((e = launch_kernel(b, b->stream, GL, nL, 0, tune)) != cudaSuccess) return e;
  if (nS > 0) e = cudaStreamWaitEvent(b->stream, b->join, 0);
  return e;
}

// Clusters of G CTAs resident on the device at once (0: G not possible).
int resident_clusters(const rks_dbatch* b, int G) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cluster_cfg(b, G, G * 64, cfg, attr);
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, k_batch_rks, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nc;
}

double csr_val(const void* vals, int dtype, int64_t q) {
  return dtype == RKS_F64 ? ((const double*)vals)[q] : (double)((const float*)vals)[q];
}

}  // namespace

extern "C" int rks_create_batched_dev(rks_dbatch** out, int count, const int64_t* n, const int32_t* const* rowptr,
                                      const int32_t* const* colind, const void* const* vals, int vals_dtype, int k,
                                      int p, int d, int which, double tol, uint64_t seed, const rks_opts* opts,
                                      int ctas_per_problem) {
  if (!out) return RKS_EINVAL;
  *out = nullptr;
  rks_opts o;
  rks_opts_default(&o);
  if (opts) o = *opts;
  const int m = k + p;
  if (count < 1 || !n || !rowptr || !colind || !vals || (vals_dtype != RKS_F64 && vals_dtype != RKS_F32))
    return RKS_EINVAL;
  if (k < 1 || p < 2 || m > kBMaxM || k + 1 > kBMaxKa || o.keep < 0 || o.keep >= m) return RKS_EINVAL;
  const int want = std::max(k, std::min(o.keep, m / 2));
  if (want + 1 > kBMaxKa) return RKS_EINVAL;
  if (o.zeta < 1 || d < m + 1 || d < 2 * o.zeta || !(tol > 0.0) || which < 0 || which > 3 || o.maxit < 1)
    return RKS_EINVAL;
  if (o.mem_device || o.u1 || (o.conv != RKS_CONV_EIG && o.conv != RKS_CONV_NORM1) || !(o.verify >= 0.0))
    return RKS_EINVAL;
  if (!(ctas_per_problem == 0 || ctas_per_problem == 1 || ctas_per_problem == 2 || ctas_per_problem == 4 ||
        ctas_per_problem == 8))
    return RKS_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (n[i] < m + 1 || n[i] >= ((int64_t)1 << 31) || !rowptr[i] || !colind[i] || !vals[i]) return RKS_EINVAL;
    if (rowptr[i][0] != 0) return RKS_EINVAL;
    for (int64_t r = 0; r < n[i]; ++r)
      if (rowptr[i][r + 1] < rowptr[i][r]) return RKS_EINVAL;
    const int64_t nnz = rowptr[i][n[i]];
    for (int64_t q = 0; q < nnz; ++q) {
      if (colind[i][q] < 0 || colind[i][q] >= n[i]) return RKS_EINVAL;
      const double v = csr_val(vals[i], vals_dtype, q);
      if (!std::isfinite(v) || std::fabs(v) > 3.0e38) return RKS_EINVAL;   // double-float range
    }
  }
  const BdLayout L = bd_layout(m, d);
  rks_dbatch* b = new (std::nothrow) rks_dbatch();
  if (!b) return RKS_ENOMEM;
  b->count = count;
  b->k = k;
  b->p = p;
  b->m = m;
  b->d = d;
  b->zeta = o.zeta;
  b->which = which;
  b->maxit = o.maxit;
  b->want = want;
  b->conv = o.conv;
  b->tol = tol;
  b->verify = o.verify;
  b->seed = seed;
  b->smem = (size_t)L.total * sizeof(double);
  b->n.assign(n, n + count);
  auto fail = [&](int rc) {
    rks_destroy_batched_dev(b);
    return rc;
  };
  if (cudaGetDevice(&b->device) != cudaSuccess) return fail(RKS_ECUDA);
  int smem_max = 0;
  if (cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device) != cudaSuccess)
    return fail(RKS_ECUDA);
  if (b->smem + sizeof(BdShared) > (size_t)smem_max) return fail(RKS_EINVAL);
  if (cudaFuncSetAttribute(k_batch_rks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem) != cudaSuccess)
    return fail(RKS_ECUDA);
  // host images (threads over problems): Omega's tile bin lists, the
  // double-float values, ||A||_1 (largest column sum), the diagonal storage
  std::vector<std::vector<int32_t>> tbin(count);
  std::vector<std::vector<uint16_t>> ent(count);
  std::vector<std::vector<float2>> dvals(count), diag(count);
  std::vector<std::vector<float>> diag32(count);
  std::vector<double> norm1(count, 0.0);
  std::vector<int> ndiag(count, 0);
  std::vector<std::array<int, kBMaxDiag>> doffs(count);
  std::vector<char> okv(count, 1);
  b->probs.resize(count);
  {
    std::atomic<int> next(0);
    auto work = [&]() {
      for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) {
        const int64_t ni = n[i], nnz = rowptr[i][ni];
        const int64_t ldu = (ni + 63) / 64 * 64;
        okv[i] = build_bins(n[i], d, o.zeta, seed, tbin[i], ent[i]) ? 1 : 0;
        std::vector<double> colsum(ni, 0.0);
        dvals[i].assign(std::max<int64_t>(nnz, 1), make_float2(0.f, 0.f));
        for (int64_t q = 0; q < nnz; ++q) {
          const double v = csr_val(vals[i], vals_dtype, q);
          colsum[colind[i][q]] += std::fabs(v);
          dvals[i][q] = bd_from(v);
        }
        norm1[i] = *std::max_element(colsum.begin(), colsum.end());
        if (!(norm1[i] > 0.0)) okv[i] = 0;
        doffs[i].fill(0);
        ndiag[i] = build_dia(ni, ldu, rowptr[i], colind[i], dvals[i], doffs[i].data(), diag[i]);
        // FP32 values (zero low words): the diagonal storage in FP32
        bool f32 = ndiag[i] > 0;
        for (int64_t q = 0; q < nnz && f32; ++q) f32 = dvals[i][q].y == 0.f;
        if (f32) {
          diag32[i].resize(diag[i].size());
          for (size_t q = 0; q < diag[i].size(); ++q) diag32[i][q] = diag[i][q].x;
          diag[i].clear();
        }
      }
    };
    const int nt = std::max(1, std::min<int>(count, (int)std::thread::hardware_concurrency()));
    std::vector<std::thread> workers;
    for (int t = 1; t < nt; ++t) workers.emplace_back(work);
    work();
    for (auto& th : workers) th.join();
  }
  for (int i = 0; i < count; ++i)
    if (!okv[i]) return fail(RKS_EINVAL);
  // one device allocation for everything
  constexpr int kParts = 10;
  std::vector<size_t> off((size_t)count * kParts);
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    const int64_t ni = n[i], nnz = std::max<int64_t>(rowptr[i][ni], 1);
    const int ntile = (int)((ni + kBR - 1) / kBR);
    const int64_t ldu = (ni + 63) / 64 * 64;
    const size_t sz[kParts] = {(size_t)(ni + 1) * 4, (size_t)nnz * 4, (size_t)nnz * 8, tbin[i].size() * 4,
                               ent[i].size() * 2, (size_t)ntile * kBR * (m + 1) * 8, (size_t)2 * ntile * d * 8,
                               (size_t)ntile * (k + 1) * 4 * 8, (size_t)ldu * (k + 1) * 8,
                               ndiag[i] ? (diag32[i].empty() ? diag[i].size() * 8 : diag32[i].size() * 4) : 0};
    for (int q = 0; q < kParts; ++q) {
      off[(size_t)i * kParts + q] = total;
      total += align_up(sz[q]);
    }
    b->probs[i].n = ni;
    b->probs[i].ntile = ntile;
    b->probs[i].ldu = ldu;
  }
  const size_t off_probs = total;
  total += align_up(sizeof(BdProb) * count);
  const size_t off_order = total;
  total += align_up(sizeof(int) * count);
  const size_t off_queue = total;
  total += 256;
  const size_t off_phase = total;
  total += align_up(sizeof(unsigned long long) * kPhases);
  const size_t off_info = total;
  total += align_up(sizeof(int) * kBInfo * count);
  const size_t off_out = total;
  total += align_up(sizeof(double) * out_stride(b) * count);
  if (cudaMalloc(&b->pool, total) != cudaSuccess) {
    cudaGetLastError();
    return fail(RKS_ENOMEM);
  }
  b->d_probs = (BdProb*)(b->pool + off_probs);
  b->d_order = (int*)(b->pool + off_order);
  b->d_queue = (unsigned long long*)(b->pool + off_queue);
  b->d_phase = (unsigned long long*)(b->pool + off_phase);
  b->d_info = (int*)(b->pool + off_info);
  b->d_out = (double*)(b->pool + off_out);
  for (int i = 0; i < count; ++i) {
    const int64_t ni = n[i], nnz = rowptr[i][ni];
    BdProb& P = b->probs[i];
    char* base = b->pool;
    const size_t* of = off.data() + (size_t)i * kParts;
    P.rowptr = (const int32_t*)(base + of[0]);
    P.colind = (const int32_t*)(base + of[1]);
    P.vals = (const float2*)(base + of[2]);
    P.tbin = (const int32_t*)(base + of[3]);
    P.ent = (const uint16_t*)(base + of[4]);
    P.U = (float2*)(base + of[5]);
    P.tsum = (float2*)(base + of[6]);
    P.rsum = (double*)(base + of[7]);
    P.X = (double*)(base + of[8]);
    P.D = ndiag[i];
    for (int e = 0; e < kBMaxDiag; ++e) P.doff[e] = doffs[i][e];
    P.dvals = ndiag[i] ? (const float2*)(base + of[9]) : nullptr;
    P.dv32 = ndiag[i] && !diag32[i].empty() ? 1 : 0;
    P.out = b->d_out + (size_t)i * out_stride(b);
    P.info = b->d_info + (size_t)i * kBInfo;
    P.norm1 = norm1[i];
    if (cudaMemcpy((void*)P.rowptr, rowptr[i], (ni + 1) * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        (nnz && cudaMemcpy((void*)P.colind, colind[i], nnz * 4, cudaMemcpyHostToDevice) != cudaSuccess) ||
        (nnz && cudaMemcpy((void*)P.vals, dvals[i].data(), nnz * 8, cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemcpy((void*)P.tbin, tbin[i].data(), tbin[i].size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy((void*)P.ent, ent[i].data(), ent[i].size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
        (P.D && !P.dv32 &&
         cudaMemcpy((void*)P.dvals, diag[i].data(), diag[i].size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) ||
        (P.D && P.dv32 &&
         cudaMemcpy((void*)P.dvals, diag32[i].data(), diag32[i].size() * 4, cudaMemcpyHostToDevice) != cudaSuccess))
      return fail(RKS_ECUDA);
  }
  // largest first (cost ~ nnz + n m), ties by index
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    const double ca = (double)rowptr[a][n[a]] + (double)n[a] * m, cc = (double)rowptr[c][n[c]] + (double)n[c] * m;
    return ca > cc;
  });
  if (cudaMemcpy(b->d_probs, b->probs.data(), sizeof(BdProb) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(RKS_ECUDA);
  if (o.stream) {
    b->stream = (cudaStream_t)o.stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(RKS_ECUDA);
    b->own_stream = true;
  }
  if (cudaEventCreate(&b->e0) != cudaSuccess || cudaEventCreate(&b->e1) != cudaSuccess) return fail(RKS_ECUDA);
  if (cudaStreamCreateWithFlags(&b->stream2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess)
    return fail(RKS_ECUDA);
  b->nmax = *std::max_element(n, n + count);
  // launch configuration: the one asked for (one kernel, ctas_per_problem
  // CTAs a problem), else the fastest candidate on a tuning run of two
  // restarts of every problem (the throughput of the configuration)
  {
    struct Cand { int GL, nL, GS, nS; };
    std::vector<Cand> cands;
    const int slots1 = resident_clusters(b, 1);   // CTAs resident at once
    auto single = [&](int G) {
      const int nc = resident_clusters(b, G);
      if (nc > 0) cands.push_back({G, std::min(nc, count), 0, 0});
    };
    auto dual = [&](int GL, int GS, int num, int den) {   // num / den of the CTA slots for the front kernel
      if (resident_clusters(b, GL) <= 0 || resident_clusters(b, GS) <= 0 || count < 2) return;
      const int nL = std::max(1, slots1 * num / den / GL);
      const int nS = std::max(1, (slots1 - nL * GL) / GS);
      cands.push_back({GL, std::min(nL, count), GS, std::min(nS, count)});
    };
    if (ctas_per_problem) {
      single(ctas_per_problem);
    } else {
      single(2);
      single(4);
      single(8);
      dual(8, 2, 1, 4);
      dual(8, 2, 1, 2);
      dual(8, 4, 1, 2);
      dual(4, 2, 1, 2);
    }
    if (cands.empty()) return fail(RKS_EINVAL);
    b->tune_ms.assign(cands.size(), 0.f);
    int best = 0;
    if (cands.size() > 1) {
      for (size_t c = 0; c < cands.size(); ++c) {
        const Cand& cd = cands[c];
        if (cudaEventRecord(b->e0, b->stream) != cudaSuccess ||
            launch_batch(b, cd.GL, cd.nL, cd.GS, cd.nS, 2) != cudaSuccess ||
            cudaEventRecord(b->e1, b->stream) != cudaSuccess || cudaStreamSynchronize(b->stream) != cudaSuccess)
          return fail(RKS_ECUDA);
        cudaEventElapsedTime(&b->tune_ms[c], b->e0, b->e1);
        if (b->tune_ms[c] < b->tune_ms[best]) best = (int)c;
      }
    }
    b->GL = cands[best].GL;
    b->nL = cands[best].nL;
    b->GS = cands[best].GS;
    b->nS = cands[best].nS;
  }
  // the launch (queue reset + kernel) as a CUDA graph
  {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail(RKS_ECUDA);
    const cudaError_t le = launch_batch(b, b->GL, b->nL, b->GS, b->nS, 0);
    const cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
    if (le != cudaSuccess || ce != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      return fail(RKS_ECUDA);
    }
    const cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return fail(RKS_ECUDA);
  }
  b->info.assign((size_t)kBInfo * count, 0);
  b->out.assign((size_t)out_stride(b) * count, 0.0);
  *out = b;
  return RKS_OK;
}

extern "C" int rks_solve_batched_dev(rks_dbatch* b, rks_info* infos) {
  if (!b) return RKS_EINVAL;
  if (cudaEventRecord(b->e0, b->stream) != cudaSuccess || cudaGraphLaunch(b->graph, b->stream) != cudaSuccess ||
      cudaEventRecord(b->e1, b->stream) != cudaSuccess || cudaStreamSynchronize(b->stream) != cudaSuccess)
    return RKS_ECUDA;
  cudaEventElapsedTime(&b->last_ms, b->e0, b->e1);
  if (cudaMemcpy(b->info.data(), b->d_info, sizeof(int) * b->info.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(b->out.data(), b->d_out, sizeof(double) * b->out.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(b->phase, b->d_phase, sizeof(b->phase), cudaMemcpyDeviceToHost) != cudaSuccess)
    return RKS_ECUDA;
  b->solved = true;
  const int os = out_stride(b);
  int first_err = RKS_OK;
  bool noconv = false;
  for (int i = 0; i < b->count; ++i) {
    const int* inf = b->info.data() + (size_t)i * kBInfo;
    const double* o = b->out.data() + (size_t)i * os;
    if (infos) {
      rks_info& r = infos[i];
      r.nconv = inf[kINconv];
      r.nlocked = 0;
      r.restarts = inf[kIRestarts];
      r.nmatvec = inf[kIMatvec];
      r.converged = inf[kIConv];
      r.max_est = o[(b->k + 1) * kBSlot];
      r.max_resid = o[(b->k + 1) * kBSlot + 1];
      r.t_solve_ms = b->last_ms;
    }
    const int s = inf[kIStatus];
    if (s == RKS_ENOCONV) noconv = true;
    else if (s != RKS_OK && first_err == RKS_OK) first_err = s;
  }
  if (first_err != RKS_OK) return first_err;
  return noconv ? RKS_ENOCONV : RKS_OK;
}

extern "C" int rks_dbatch_config(const rks_dbatch* b, int* cfg4, float* tune_ms, int ntune, float* last_ms) {
  if (!b) return RKS_EINVAL;
  if (cfg4) {
    cfg4[0] = b->GL;
    cfg4[1] = b->nL;
    cfg4[2] = b->GS;
    cfg4[3] = b->nS;
  }
  if (tune_ms)
    for (int c = 0; c < ntune && c < (int)b->tune_ms.size(); ++c) tune_ms[c] = b->tune_ms[c];
  if (last_ms) *last_ms = b->last_ms;
  return (int)b->tune_ms.size();
}

extern "C" int rks_dbatch_phase_cycles(const rks_dbatch* b, int64_t* cycles, int count) {
  if (!b || !cycles || count < 1) return RKS_EINVAL;
  if (!b->solved) return RKS_ESTATE;
  const int nc = std::min(count, (int)kPhases);
  for (int q = 0; q < nc; ++q) cycles[q] = (int64_t)b->phase[q];
  return nc;
}

extern "C" int rks_dbatch_status(const rks_dbatch* b, int i) {
  if (!b || i < 0 || i >= b->count) return RKS_EINVAL;
  if (!b->solved) return RKS_ESTATE;
  return b->info[(size_t)i * kBInfo + kIStatus];
}

extern "C" int rks_dbatch_eigpairs(rks_dbatch* b, int i, double* lam_re, double* lam_im, double* resid,
                                   double* rq_re, double* rq_im, double* est, double* X) {
  if (!b || i < 0 || i >= b->count) return RKS_EINVAL;
  if (!b->solved) return RKS_ESTATE;
  const int nw = b->info[(size_t)i * kBInfo + kINw];
  const double* o = b->out.data() + (size_t)i * out_stride(b);
  for (int t = 0; t < nw; ++t) {
    const double* s = o + (size_t)t * kBSlot;
    if (lam_re) lam_re[t] = s[0];
    if (lam_im) lam_im[t] = s[1];
    if (resid) resid[t] = s[2];
    if (rq_re) rq_re[t] = s[3];
    if (rq_im) rq_im[t] = s[4];
    if (est) est[t] = s[5];
  }
  if (X && nw > 0) {
    const BdProb& P = b->probs[i];
    if (cudaMemcpy2D(X, sizeof(double) * P.n, P.X, sizeof(double) * P.ldu, sizeof(double) * P.n, nw,
                     cudaMemcpyDeviceToHost) != cudaSuccess)
      return RKS_ECUDA;
  }
  return nw;
}

extern "C" void rks_destroy_batched_dev(rks_dbatch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->e0) cudaEventDestroy(b->e0);
  if (b->e1) cudaEventDestroy(b->e1);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  if (b->stream2) cudaStreamDestroy(b->stream2);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  if (b->pool) cudaFree(b->pool);
  delete b;
}

extern "C" int rks_dev_ordered_schur(int m, const double* Bh, int which, int nsort, double* T, double* Q,
                                     double* lam_re, double* lam_im, double* Y_re, double* Y_im) {
  using df = DenseR;
  if (m < 1 || m > kBMaxM || !Bh || !T || !Q || which < 0 || which > 3 || nsort < 0) return RKS_EINVAL;
  const size_t mm = (size_t)m * m;
  const size_t nout = 4 * mm + 2 * (size_t)m;   // T, Q, Yr, Yi, lre, lim
  double* dB = nullptr;
  df* dv = nullptr;
  double* dout = nullptr;
  int* ds = nullptr;
  if (cudaMalloc(&dB, sizeof(double) * mm) != cudaSuccess || cudaMalloc(&dv, sizeof(df) * (nout + 2 * m)) != cudaSuccess ||
      cudaMalloc(&dout, sizeof(double) * nout) != cudaSuccess || cudaMalloc(&ds, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(dB);
    cudaFree(dv);
    cudaFree(dout);
    cudaFree(ds);
    return RKS_ENOMEM;
  }
  df *dT = dv, *dQ = dv + mm, *dYr = dv + 2 * mm, *dYi = dv + 3 * mm, *dl = dv + 4 * mm;
  int rc = RKS_OK, st = 0;
  if (cudaMemcpy(dB, Bh, sizeof(double) * mm, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(dv, 0, sizeof(df) * (nout + 2 * m)) != cudaSuccess)
    rc = RKS_ECUDA;
  if (!rc) {
    k_dense_test<<<1, 32>>>(m, dB, dT, dQ, which, std::min(nsort, m), dl, dl + m, dYr, dYi, dl + 2 * m, ds);
    k_df_to_double<<<8, 256>>>((int64_t)nout, dv, dout);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) rc = RKS_ECUDA;
  }
  const double* ho = nullptr;
  std::vector<double> h(nout);
  if (!rc && (cudaMemcpy(&st, ds, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
              cudaMemcpy(h.data(), dout, sizeof(double) * nout, cudaMemcpyDeviceToHost) != cudaSuccess))
    rc = RKS_ECUDA;
  if (!rc && st != 0) rc = RKS_EDENSE;
  if (!rc) {
    ho = h.data();
    std::memcpy(T, ho, sizeof(double) * mm);
    std::memcpy(Q, ho + mm, sizeof(double) * mm);
    if (Y_re) std::memcpy(Y_re, ho + 2 * mm, sizeof(double) * mm);
    if (Y_im) std::memcpy(Y_im, ho + 3 * mm, sizeof(double) * mm);
    if (lam_re) std::memcpy(lam_re, ho + 4 * mm, sizeof(double) * m);
    if (lam_im) std::memcpy(lam_im, ho + 4 * mm + m, sizeof(double) * m);
  }
  cudaFree(dB);
  cudaFree(dv);
  cudaFree(dout);
  cudaFree(ds);
  return rc;
}
