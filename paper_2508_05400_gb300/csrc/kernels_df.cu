// Double-float (DF) kernels of the rKS hot path: FP64-class accuracy on the
// FP32 pipes of sm_103a.
//
// GB300 executes FP64 at about 2 FMA/clock/SM (measured: 0.6 T FMA/s for the
// whole GPU), 60x below FP32, so FP64 arithmetic, not HBM, bounds an FP64
// Arnoldi step.  Here every n-dimensional quantity keeps 8 bytes per value but
// as an unevaluated sum of two floats (hi + lo, |lo| <= ulp(hi)/2, a 48-bit
// significand), and products/sums use error-free transformations (TwoSum,
// TwoProd via fmaf) on the FP32 pipes.  The d-dimensional sketch data and the
// host-side dense work stay FP64; final residuals are computed in FP64.
//
// One Arnoldi step of Algorithm 2 (Sec. 3.1), new column c = j + 1, is three
// kernels:
//   k_df_spmv_ell / k_df_spmv_sketch
//                     w' = A u~_j (unscaled, u_j = u~_j / beta_j), z' = Omega w'
//                     (A as interleaved ELLPACK when that is compact, else CSR)
//   k_df_ls_coop      fold of the sketch partials, finish column j (beta_j =
//                     ||s~_j||, S, scale, coefficient column), then b = S^+ z by
//                     CGS2 in the sketch against the locked and active columns
//                     (Thm 4.3), z = z' / beta_j (k_df_fold + k_df_ls1 +
//                     k_df_ls_gram when a cooperative launch is unavailable)
//   k_df_update_sketch u~_{j+1} = w'/beta_j - U b, s~_{j+1} = Omega u~_{j+1}
//
// Sketch accumulation is deterministic: no atomics.  Each CTA owns a fixed,
// contiguous range of rows, cut into tiles of at most kTileRows rows.  For
// every tile a transposed copy of Omega restricted to the tile (the "bin
// lists", built once by k_tiles_build) gives, per sketch row, the tile rows
// that contribute to it and their signs, in a fixed order.  A tile's values
// are staged in shared memory; then the threads that own the tile's sketch
// rows sum their lists (DF, TwoSum) into per-CTA DF accumulators.  Each CTA
// writes its d partial sums; the consumer adds the CTA partials in a fixed
// order (fold_row).  The result is the same bits on every run.

#include <algorithm>
#include <type_traits>
#include <vector>

#include "rks_impl.h"

namespace rks {

// ---------------------------------------------------------------------------
// double-float helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

// (s, t) += (ah + al) * (bh + bl), (s, t) an unnormalised accumulator
__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float& s, float& t) {
  float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  float s2, e2;
  two_sum(s, p, s2, e2);
  s = s2;
  t += e2 + e;
}

// (s, t) += (bh + bl)
__device__ __forceinline__ void df_add(float bh, float bl, float& s, float& t) {
  float s2, e2;
  two_sum(s, bh, s2, e2);
  s = s2;
  t += e2 + bl;
}

// (s, t) += a * b for values stored as TA and TB: an FP32 value has no low
// word, so its terms are left out (df_mac's operations otherwise, in its
// order; the sums differ from df_mac's at most in the sign of a zero)
template <class TA, class TB>
__device__ __forceinline__ void mac_st(float2 a, float2 b, float& s, float& t) {
  constexpr bool A1 = sizeof(TA) == 4, B1 = sizeof(TB) == 4;
  if constexpr (!A1 && !B1) {
    df_mac(a.x, a.y, b.x, b.y, s, t);
  } else {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    if constexpr (!B1) e = fmaf(a.x, b.y, e);
    if constexpr (!A1) e = fmaf(a.y, b.x, e);
    float s2, e2;
    two_sum(s, p, s2, e2);
    s = s2;
    t += e2 + e;
  }
}

__device__ __forceinline__ float2 df_norm(float s, float t) {
  float h, l;
  fast_two_sum(s, t, h, l);
  return make_float2(h, l);
}

__device__ __forceinline__ float2 df_from_double(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return make_float2(h, l);
}

__device__ __forceinline__ double df_to_double(float2 v) { return (double)v.x + (double)v.y; }

// DF warp reduction of (s, t) pairs
__device__ __forceinline__ void df_warp_sum(float& s, float& t) {
  for (int o = 16; o; o >>= 1) {
    float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    float t2 = __shfl_xor_sync(0xffffffffu, t, o);
    float ss, e;
    two_sum(s, s2, ss, e);
    s = ss;
    t = t + t2 + e;
  }
}

// Basis / matrix storage: float2 = double-float pair, float = FP32 (the
// mixed-precision basis of the paper's future-work direction, Sec. 6).  Loads
// widen to a pair; stores round the pair to the stored type, and the sketch
// is always taken of the value as stored.
__device__ __forceinline__ float2 ldv(const float2* p) { return *p; }
__device__ __forceinline__ float2 ldv(const float* p) { return make_float2(*p, 0.f); }
__device__ __forceinline__ float2 stv(float2* p, float2 v) { *p = v; return v; }
__device__ __forceinline__ float2 stv(float* p, float2 v) {
  float r = v.x + v.y;
  *p = r;
  return make_float2(r, 0.f);
}

// ---------------------------------------------------------------------------
// sketch (same hash as kernels.cu; see rks.h)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t mix64_df(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Packed Omega table: for column i, MAXZ uint16 entries (row in bits 0..14,
// bit 15 set for a negative sign), written once by k_omega_table from the same
// hash; unused slots (t >= zeta) are 0xFFFF.  The tile bin lists are built
// from it.

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// The packed Omega table from the hash of rks.h.
template <int MAXZ>
__global__ void k_omega_table(int64_t n, int d, int zeta, uint64_t seed, uint16_t* __restrict__ tab, int* flag) {
  const uint64_t gamma = 0x9E3779B97F4A7C15ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t base = mix64_df(seed * gamma + (uint64_t)i);
    int rows[MAXZ];
    uint16_t ent[MAXZ];
#pragma unroll
    for (int t = 0; t < MAXZ; ++t) { rows[t] = -1; ent[t] = 0xFFFF; }
    int cnt = 0;
    const int cap = 32 * zeta;
    for (int r = 0; r < cap && cnt < zeta; ++r) {
      uint64_t h = mix64_df(base + (uint64_t)(r + 1) * gamma);
      int row = (int)(((h >> 32) * (uint64_t)d) >> 32);
      bool dup = false;
#pragma unroll
      for (int t = 0; t < MAXZ; ++t) dup |= (rows[t] == row);
      if (dup) continue;
#pragma unroll
      for (int t = 0; t < MAXZ; ++t)
        if (t == cnt) { rows[t] = row; ent[t] = (uint16_t)(row | ((h & 1ull) ? 0x8000 : 0)); }
      ++cnt;
    }
    if (cnt < zeta) atomicOr(flag, RKS_FLAG_HASH);
#pragma unroll
    for (int t = 0; t < MAXZ; ++t) tab[i * MAXZ + t] = ent[t];
  }
}

// ---------------------------------------------------------------------------
// tile bin lists (built once per context from the packed table)
// ---------------------------------------------------------------------------

// Largest number of entries of one sketch row within one tile (atomicMax into
// *lmax; the per-bin counts are integers, so their order does not matter).
template <int MAXZ>
__global__ void __launch_bounds__(256) k_tiles_count(const int64_t* __restrict__ trow, int d,
                                                     const uint16_t* __restrict__ otab, int* lmax) {
  extern __shared__ int cnt[];   // d
  const int64_t t = blockIdx.x;
  for (int b = threadIdx.x; b < d; b += blockDim.x) cnt[b] = 0;
  __syncthreads();
  const int64_t q1 = trow[t + 1] * MAXZ;
  for (int64_t q = trow[t] * MAXZ + threadIdx.x; q < q1; q += blockDim.x) {
    const uint32_t e = otab[q];
    if (e != 0xFFFFu) atomicAdd(&cnt[e & 0x7FFF], 1);
  }
  __syncthreads();
  int m = 0;
  for (int b = threadIdx.x; b < d; b += blockDim.x) m = max(m, cnt[b]);
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(lmax, m);
}

// Bin lists of one tile (one CTA per tile), jagged-diagonal layout:
//   positions p = 0..d-1 rank the sketch rows by entry count (descending,
//   ties by row index); meta[t*d + p] = row | count << 16;
//   slot s holds entry s of every position whose count exceeds s, the
//   positions in order, from off[t*(L+1) + s] = sum_p min(count_p, s);
//   an entry is (tile row) | 0x8000 for a negative sign.
// The entries of a sketch row are listed in (32-row chunk, slot, lane) order,
// fixed by the table alone.
template <int MAXZ>
__global__ void __launch_bounds__(256) k_tiles_build(const int64_t* __restrict__ trow, int d, int zeta, int L,
                                                     const uint16_t* __restrict__ otab, uint32_t* __restrict__ meta,
                                                     int* __restrict__ off, uint16_t* __restrict__ ent) {
  extern __shared__ int sm[];
  int* cnt = sm;          // d: entries per sketch row
  int* rank = cnt + d;    // d: position of each sketch row
  int* scnt = rank + d;   // d: counts by position
  int* cur = scnt + d;    // d: fill cursor per sketch row
  int* offs = cur + d;    // L + 1
  const int64_t t = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t r0 = trow[t], r1 = trow[t + 1];
  for (int b = tid; b < d; b += nt) { cnt[b] = 0; cur[b] = 0; }
  __syncthreads();
  for (int64_t q = r0 * MAXZ + tid; q < r1 * MAXZ; q += nt) {
    const uint32_t e = otab[q];
    if (e != 0xFFFFu) atomicAdd(&cnt[e & 0x7FFF], 1);
  }
  __syncthreads();
  for (int b = tid; b < d; b += nt) {
    const int cb = cnt[b];
    int r = 0;
    for (int b2 = 0; b2 < d; ++b2) {
      const int c2 = cnt[b2];
      r += (c2 > cb) || (c2 == cb && b2 < b);
    }
    rank[b] = r;
  }
  __syncthreads();
  for (int b = tid; b < d; b += nt) {
    scnt[rank[b]] = cnt[b];
    meta[t * d + rank[b]] = (uint32_t)b | ((uint32_t)cnt[b] << 16);
  }
  __syncthreads();
  for (int s = tid; s <= L; s += nt) {
    int o = 0;
    for (int p = 0; p < d; ++p) o += min(scnt[p], s);
    offs[s] = o;
    off[t * (L + 1) + s] = o;
  }
  __syncthreads();
  if (tid < 32) {
    const int lane = tid;
    uint16_t* et = ent + r0 * zeta;
    const int rows = (int)(r1 - r0);
    for (int c0 = 0; c0 < rows; c0 += 32) {
      const int l = c0 + lane;
      for (int s = 0; s < MAXZ; ++s) {
        const uint32_t e = l < rows ? (uint32_t)otab[(r0 + l) * MAXZ + s] : 0xFFFFu;
        const bool v = e != 0xFFFFu;
        const uint32_t key = v ? (e & 0x7FFFu) : (0x10000u + lane);   // no two invalid lanes match
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        if (v) {
          const int b = (int)(e & 0x7FFFu);
          const int kk = cur[b] + __popc(grp & ((1u << lane) - 1u));
          et[offs[kk] + rank[b]] = (uint16_t)(l | (e & 0x8000u));
        }
        __syncwarp();
        if (v && lane == __ffs(grp) - 1) cur[e & 0x7FFFu] += __popc(grp);
        __syncwarp();
      }
    }
  }
}

// (s, e) += sign * vals[row] for one bin-list entry; LO = false: the tile
// holds FP32 values (zero low words), whose low words are left out
template <bool LO>
__device__ __forceinline__ void tile_add(uint32_t x, const float2* vals, float& s, float& e) {
  const float2 v = vals[x & 0x7FFFu];
  const uint32_t sg = (x & 0x8000u) << 16;
  if (LO) {
    df_add(__uint_as_float(__float_as_uint(v.x) ^ sg), __uint_as_float(__float_as_uint(v.y) ^ sg), s, e);
  } else {
    float s2, e2;
    two_sum(s, __uint_as_float(__float_as_uint(v.x) ^ sg), s2, e2);
    s = s2;
    e += e2;
  }
}

// Sketch of one staged tile: acc[row] += sum over the row's bin list of
// sign * vals[tile row], entries in their stored order.  The tile's slot
// offsets (offs), positions (ms) and entries (es) are in shared memory.
// H adjacent lanes share a position (each takes every H-th entry) when d is
// small; their sums are combined by a fixed xor tree.  A sketch row has one
// position per tile, so acc[row] has one writer per tile.
template <bool LO>
__device__ __forceinline__ void tile_gather(int d, int H, const float2* vals, const int* offs, const uint32_t* ms,
                                            const uint16_t* es, float2* acc) {
  const int total = d * H;
  const int lane = threadIdx.x & 31;
  for (int base = threadIdx.x & ~31; base < total; base += blockDim.x) {
    const int pp = base + lane;
    const int p = pp / H, h = pp - p * H;
    float s = 0.f, e = 0.f;
    int b = -1, cnt = 0;
    if (pp < total) {
      const uint32_t mt = ms[p];
      b = (int)(mt & 0xFFFFu);
      cnt = (int)(mt >> 16);
      int q = h;
      for (; q + 3 * H < cnt; q += 4 * H) {
        const uint32_t x0 = es[offs[q] + p], x1 = es[offs[q + H] + p];
        const uint32_t x2 = es[offs[q + 2 * H] + p], x3 = es[offs[q + 3 * H] + p];
        tile_add<LO>(x0, vals, s, e);
        tile_add<LO>(x1, vals, s, e);
        tile_add<LO>(x2, vals, s, e);
        tile_add<LO>(x3, vals, s, e);
      }
      for (; q < cnt; q += H) tile_add<LO>(es[offs[q] + p], vals, s, e);
    }
    for (int o = 1; o < H; o <<= 1) {
      const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
      const float e2 = __shfl_xor_sync(0xffffffffu, e, o);
      float ss, er;
      two_sum(s, s2, ss, er);
      s = ss;
      e = e + e2 + er;
    }
    if (h == 0 && cnt > 0) {
      const float2 a = acc[b];
      float as = a.x, ae = a.y;
      df_add(s, e, as, ae);
      acc[b] = df_norm(as, ae);
    }
  }
}

// Shared memory of a tile kernel: DF accumulators (d), two value buffers,
// the update's coefficients (c), then two buffers each of the tile's entries,
// positions and slot offsets.
struct TileSmem {
  size_t acc, vb, rsh, es, ms, offs, total;
};

__host__ __device__ inline TileSmem tile_smem_layout(int d, int L, int c, int zeta) {
  TileSmem s;
  size_t o = 0;
  s.acc = o; o += (size_t)d * sizeof(float2);
  s.vb = o; o += (size_t)2 * kTileRows * sizeof(float2);
  s.rsh = o; o += (size_t)c * sizeof(float2);
  o = (o + 15) & ~(size_t)15;
  s.es = o; o += (size_t)2 * kTileRows * zeta * sizeof(uint16_t);
  s.ms = o; o += (size_t)2 * d * sizeof(uint32_t);
  s.offs = o; o += (size_t)2 * (L + 1) * sizeof(int);
  s.total = o;
  return s;
}

__host__ __device__ inline size_t tile_smem_bytes(int d, int L, int c, int zeta) {
  return tile_smem_layout(d, L, c, zeta).total;
}

// Stage tile t's slot offsets, positions and entries (coalesced copies; the
// entries with 16-byte loads when aligned).
__device__ __forceinline__ void tile_stage(const SketchTiles& tv, int64_t t, int64_t r0, int rows, int* of,
                                           uint32_t* ms, uint16_t* es) {
  const int L1 = tv.L + 1, d = tv.d;
  for (int q = threadIdx.x; q < L1; q += blockDim.x) of[q] = tv.off[t * L1 + q];
  const uint32_t* mg = tv.meta + t * d;
  for (int q = threadIdx.x; q < d; q += blockDim.x) ms[q] = __ldg(mg + q);
  const uint16_t* src = tv.ent + r0 * tv.zeta;
  const int cnt = rows * tv.zeta;
  int q0 = 0;
  if (((r0 * tv.zeta) & 7) == 0) {
    const int nv = cnt >> 3;
    for (int q = threadIdx.x; q < nv; q += blockDim.x)
      reinterpret_cast<uint4*>(es)[q] = __ldg(reinterpret_cast<const uint4*>(src) + q);
    q0 = nv << 3;
  }
  for (int q = q0 + threadIdx.x; q < cnt; q += blockDim.x) es[q] = src[q];
}

// The bin lists of one tile held in registers between their load and their
// store into shared memory, so that the loads of the next tile's lists are in
// flight while this tile's rows are computed.  Valid when every per-thread
// count fits (tile_regs_fit); the stored bytes are those of tile_stage.
constexpr int kStageRegs = 2;   // uint4 of entries per thread (zeta <= 8)
struct TileRegs {
  uint4 e[kStageRegs];
  int of[2];
  uint32_t ms[2];
};
__host__ __device__ inline bool tile_regs_fit(const SketchTiles& tv) {
  return tv.L + 1 <= 2 * 512 && tv.d <= 2 * 512 && kTileRows * tv.zeta / 8 <= kStageRegs * 512;
}
__device__ __forceinline__ void tile_regs_load(const SketchTiles& tv, int64_t t, TileRegs& R) {
  const int L1 = tv.L + 1, d = tv.d;
  const int64_t r0 = tv.row[t];
  const int cnt = (int)(tv.row[t + 1] - r0) * tv.zeta;
  const uint4* src = reinterpret_cast<const uint4*>(tv.ent + r0 * tv.zeta);   // r0 is a multiple of kTileRows
#pragma unroll
  for (int u = 0; u < kStageRegs; ++u) {
    const int q = threadIdx.x + u * 512;
    R.e[u] = q * 8 < cnt ? __ldg(src + q) : make_uint4(0u, 0u, 0u, 0u);
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int q = threadIdx.x + u * 512;
    R.of[u] = q < L1 ? tv.off[t * L1 + q] : 0;
    R.ms[u] = q < d ? __ldg(tv.meta + t * d + q) : 0u;
  }
}
__device__ __forceinline__ void tile_regs_store(const SketchTiles& tv, int64_t t, const TileRegs& R, int* of,
                                                uint32_t* ms, uint16_t* es) {
  const int L1 = tv.L + 1, d = tv.d;
  const int cnt = (int)(tv.row[t + 1] - tv.row[t]) * tv.zeta;
#pragma unroll
  for (int u = 0; u < kStageRegs; ++u) {
    const int q = threadIdx.x + u * 512;
    if (q * 8 + 8 <= cnt) reinterpret_cast<uint4*>(es)[q] = R.e[u];
    else if (q * 8 < cnt) {   // the ragged end of the last tile
      const uint32_t wd[4] = {R.e[u].x, R.e[u].y, R.e[u].z, R.e[u].w};
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (q * 8 + k < cnt) es[q * 8 + k] = (uint16_t)((wd[k >> 1] >> (16 * (k & 1))) & 0xFFFFu);
    }
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int q = threadIdx.x + u * 512;
    if (q < L1) of[q] = R.of[u];
    if (q < d) ms[q] = R.ms[u];
  }
}

__device__ __forceinline__ void tile_write_part(const float2* acc, int d, double* part) {
  __syncthreads();
  for (int r = threadIdx.x; r < d; r += blockDim.x) part[(size_t)blockIdx.x * d + r] = df_to_double(acc[r]);
}

// w'[i] = sum_p A_p x[col_p] (DF) over the CTA's tiles; part[cta] = the
// CTA's Omega-sums of w' as stored.  512 threads; thread l takes the tile
// rows l and l + 512 together, four entries of each per round, so that the
// loads of both rows are in flight at once (the products of a row are still
// accumulated in entry order).
// SK = false: the plain SpMV (Krylov-Schur with Euclidean CGS2), no sketch.
template <class TA, class TU, bool SK>
__global__ void __launch_bounds__(512) k_df_spmv_sketch(
    const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind, const TA* __restrict__ vals,
    const TU* __restrict__ x, TU* __restrict__ w, const SketchTiles tv, double* __restrict__ part) {
  static_assert(kTileRows == 1024, "two rows per thread of a 512-thread CTA");
  extern __shared__ __align__(16) uint8_t smraw[];
  const int d = tv.d, L1 = tv.L + 1;
  const TileSmem lay = tile_smem_layout(d, tv.L, 0, tv.zeta);
  float2* acc = reinterpret_cast<float2*>(smraw + lay.acc);
  if (SK)
    for (int r = threadIdx.x; r < d; r += blockDim.x) acc[r] = make_float2(0.f, 0.f);
  const int t0 = tv.ctile[blockIdx.x], t1 = tv.ctile[blockIdx.x + 1];
  for (int t = t0; t < t1; ++t) {
    const int buf = (t - t0) & 1;
    float2* v = reinterpret_cast<float2*>(smraw + lay.vb) + buf * kTileRows;
    int* of = reinterpret_cast<int*>(smraw + lay.offs) + buf * L1;
    uint32_t* ms = reinterpret_cast<uint32_t*>(smraw + lay.ms) + buf * d;
    uint16_t* es = reinterpret_cast<uint16_t*>(smraw + lay.es) + (size_t)buf * kTileRows * tv.zeta;
    const int64_t r0 = tv.row[t];
    const int rows = (int)(tv.row[t + 1] - r0);
    if (SK) tile_stage(tv, t, r0, rows, of, ms, es);
    const int la = threadIdx.x, lb = threadIdx.x + 512;
    int pa = 0, ea = 0, pb = 0, eb = 0;
    if (la < rows) { pa = rowptr[r0 + la]; ea = rowptr[r0 + la + 1]; }
    if (lb < rows) { pb = rowptr[r0 + lb]; eb = rowptr[r0 + lb + 1]; }
    float sa = 0.f, ta = 0.f, sb = 0.f, tb = 0.f;
    const int len = max(ea - pa, eb - pb);
    for (int q = 0; q < len; q += 4) {
      int ca[4], cb[4];
      float2 va[4], vbv[4], xa[4], xb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int p = pa + q + u, p2 = pb + q + u;
        ca[u] = p < ea ? colind[p] : -1;
        cb[u] = p2 < eb ? colind[p2] : -1;
        va[u] = p < ea ? ldv(vals + p) : make_float2(0.f, 0.f);
        vbv[u] = p2 < eb ? ldv(vals + p2) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        xa[u] = ca[u] >= 0 ? ldv(x + ca[u]) : make_float2(0.f, 0.f);
        xb[u] = cb[u] >= 0 ? ldv(x + cb[u]) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (ca[u] >= 0) mac_st<TA, TU>(va[u], xa[u], sa, ta);
        if (cb[u] >= 0) mac_st<TA, TU>(vbv[u], xb[u], sb, tb);
      }
    }
    if (la < rows) v[la] = stv(w + r0 + la, df_norm(sa, ta));
    if (lb < rows) v[lb] = stv(w + r0 + lb, df_norm(sb, tb));
    if (SK) {
      __syncthreads();
      tile_gather<sizeof(TU) == 8>(d, tv.H, v, of, ms, es, acc);
    }
  }
  if (SK) tile_write_part(acc, d, part);
}

// The SpMV+sketch of k_df_spmv_sketch on the ELLPACK copy of A (CsrDF): a
// thread's entries sit at fixed offsets from its row index, so the loads of a
// round need no row pointer first and each is one contiguous segment per warp.
// Entries are taken in CSR order and padding (column -1) is skipped, so the
// products and sums are those of the CSR kernel, bit for bit.
// WC > 0: rows of at most WC entries, all of a row's loads in one round
// (5-point stencils: W = 5 fits WC = 6 without spilling at two CTAs per SM).
template <class TA, class TU, bool SK, int WC>
__global__ void __launch_bounds__(512) k_df_spmv_ell(
    const int32_t* __restrict__ ecol, const TA* __restrict__ evals, int W,
    const TU* __restrict__ x, TU* __restrict__ w, const SketchTiles tv, double* __restrict__ part) {
  static_assert(kTileRows == 1024, "two rows per thread of a 512-thread CTA");
  extern __shared__ __align__(16) uint8_t smraw[];
  const int d = tv.d, L1 = tv.L + 1;
  const TileSmem lay = tile_smem_layout(d, tv.L, 0, tv.zeta);
  float2* acc = reinterpret_cast<float2*>(smraw + lay.acc);
  if (SK)
    for (int r = threadIdx.x; r < d; r += blockDim.x) acc[r] = make_float2(0.f, 0.f);
  const int t0 = tv.ctile[blockIdx.x], t1 = tv.ctile[blockIdx.x + 1];
  for (int t = t0; t < t1; ++t) {
    const int buf = (t - t0) & 1;
    float2* v = reinterpret_cast<float2*>(smraw + lay.vb) + buf * kTileRows;
    int* of = reinterpret_cast<int*>(smraw + lay.offs) + buf * L1;
    uint32_t* ms = reinterpret_cast<uint32_t*>(smraw + lay.ms) + buf * d;
    uint16_t* es = reinterpret_cast<uint16_t*>(smraw + lay.es) + (size_t)buf * kTileRows * tv.zeta;
    const int64_t r0 = tv.row[t];
    const int rows = (int)(tv.row[t + 1] - r0);
    if (SK) tile_stage(tv, t, r0, rows, of, ms, es);
    const int la = threadIdx.x, lb = threadIdx.x + 512;
    const bool oka = la < rows, okb = lb < rows;
    const int64_t ia = r0 + la, ib = r0 + lb;
    const int64_t ba = (((ia >> 5) * W) << 5) + (ia & 31), bb = (((ib >> 5) * W) << 5) + (ib & 31);
    float sa = 0.f, ta = 0.f, sb = 0.f, tb = 0.f;
    if (WC > 0) {                                 // one round: every column and value, then x
      constexpr int R1 = WC > 0 ? WC : 1;
      int ca[R1], cb[R1];
      float2 va[R1], vbv[R1];
#pragma unroll
      for (int e = 0; e < R1; ++e) {
        const int64_t oa = ba + ((int64_t)e << 5), ob = bb + ((int64_t)e << 5);
        ca[e] = (oka && e < W) ? ecol[oa] : -1;
        cb[e] = (okb && e < W) ? ecol[ob] : -1;
        va[e] = (oka && e < W) ? ldv(evals + oa) : make_float2(0.f, 0.f);
        vbv[e] = (okb && e < W) ? ldv(evals + ob) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int e = 0; e < R1; ++e) {
        const float2 xa = ca[e] >= 0 ? ldv(x + ca[e]) : make_float2(0.f, 0.f);
        const float2 xb = cb[e] >= 0 ? ldv(x + cb[e]) : make_float2(0.f, 0.f);
        if (ca[e] >= 0) mac_st<TA, TU>(va[e], xa, sa, ta);
        if (cb[e] >= 0) mac_st<TA, TU>(vbv[e], xb, sb, tb);
      }
    }
    constexpr int RU = 4;                         // rounds of four entries
    for (int q = 0; WC == 0 && q < W; q += RU) {
      int ca[RU], cb[RU];
      float2 va[RU], vbv[RU], xa[RU], xb[RU];
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const int e = q + u;
        const int64_t oa = ba + ((int64_t)e << 5), ob = bb + ((int64_t)e << 5);
        ca[u] = (oka && e < W) ? ecol[oa] : -1;
        cb[u] = (okb && e < W) ? ecol[ob] : -1;
        va[u] = (oka && e < W) ? ldv(evals + oa) : make_float2(0.f, 0.f);
        vbv[u] = (okb && e < W) ? ldv(evals + ob) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        xa[u] = ca[u] >= 0 ? ldv(x + ca[u]) : make_float2(0.f, 0.f);
        xb[u] = cb[u] >= 0 ? ldv(x + cb[u]) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        if (ca[u] >= 0) mac_st<TA, TU>(va[u], xa[u], sa, ta);
        if (cb[u] >= 0) mac_st<TA, TU>(vbv[u], xb[u], sb, tb);
      }
    }
    if (oka) v[la] = stv(w + ia, df_norm(sa, ta));
    if (okb) v[lb] = stv(w + ib, df_norm(sb, tb));
    if (SK) {
      __syncthreads();
      tile_gather<sizeof(TU) == 8>(d, tv.H, v, of, ms, es, acc);
    }
  }
  if (SK) tile_write_part(acc, d, part);
}

// w = A x (+ partial sketches) with one warp per row inside each sketch tile
// (rows of many entries): lanes take the row's entries with a stride of 32,
// then a fixed xor tree adds the lanes' double-float sums.
template <class TA, class TU, bool SK, int LPR>
__global__ void __launch_bounds__(512) k_df_spmv_warp(const int32_t* __restrict__ rowptr,
                                                      const int32_t* __restrict__ colind, const TA* __restrict__ vals,
                                                      const TU* __restrict__ x, TU* __restrict__ w,
                                                      const SketchTiles tv, double* __restrict__ part) {
  extern __shared__ __align__(16) uint8_t smraw[];
  const int d = tv.d, L1 = tv.L + 1;
  const TileSmem lay = tile_smem_layout(d, tv.L, 0, tv.zeta);
  float2* acc = reinterpret_cast<float2*>(smraw + lay.acc);
  if (SK)
    for (int r = threadIdx.x; r < d; r += blockDim.x) acc[r] = make_float2(0.f, 0.f);
  // groups of LPR lanes per row (LPR = 32: a warp per row)
  const int grp = threadIdx.x / LPR, lane = threadIdx.x % LPR, ngrp = blockDim.x / LPR;
  const int t0 = tv.ctile[blockIdx.x], t1 = tv.ctile[blockIdx.x + 1];
  for (int t = t0; t < t1; ++t) {
    const int buf = (t - t0) & 1;
    float2* v = reinterpret_cast<float2*>(smraw + lay.vb) + buf * kTileRows;
    int* of = reinterpret_cast<int*>(smraw + lay.offs) + buf * L1;
    uint32_t* ms = reinterpret_cast<uint32_t*>(smraw + lay.ms) + buf * d;
    uint16_t* es = reinterpret_cast<uint16_t*>(smraw + lay.es) + (size_t)buf * kTileRows * tv.zeta;
    const int64_t r0 = tv.row[t];
    const int rows = (int)(tv.row[t + 1] - r0);
    if (SK) tile_stage(tv, t, r0, rows, of, ms, es);
    const int nit = (rows + ngrp - 1) / ngrp;        // the same trip count for every lane
    for (int it = 0; it < nit; ++it) {
      const int l = it * ngrp + grp;
      float sh = 0.f, sl = 0.f;
      if (l < rows) {
        const int p0 = rowptr[r0 + l], p1 = rowptr[r0 + l + 1];
        for (int p = p0 + lane; p < p1; p += LPR) {
          const float2 a = ldv(vals + p), xv = ldv(x + colind[p]);
          mac_st<TA, TU>(a, xv, sh, sl);
        }
      }
#pragma unroll
      for (int o = LPR / 2; o; o >>= 1) {              // fixed xor tree inside the group
        const float s2 = __shfl_xor_sync(0xffffffffu, sh, o);
        const float t2 = __shfl_xor_sync(0xffffffffu, sl, o);
        float ss, e;
        two_sum(sh, s2, ss, e);
        sh = ss;
        sl = sl + t2 + e;
      }
      if (l < rows && lane == 0) v[l] = stv(w + r0 + l, df_norm(sh, sl));
    }
    if (SK) {
      __syncthreads();
      tile_gather<sizeof(TU) == 8>(d, tv.H, v, of, ms, es, acc);
    }
  }
  if (SK) tile_write_part(acc, d, part);
}

// Merge-path split: the number of rows i whose end marker lies before merge
// position dd (marker of row i at rowptr[i + 1] + i); dd - i entries precede.
__device__ __forceinline__ int64_t merge_split(int64_t dd, int64_t n, int64_t nnz, const int32_t* __restrict__ rowptr) {
  int64_t lo = dd > nnz ? dd - nnz : 0, hi = dd < n ? dd : n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)rowptr[mid + 1] + mid < dd) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

constexpr int kMergeBlk = kMergeCta * kMergeItems;   // merge items per CTA

// part_row[b] = rows whose end precedes merge position b * kMergeBlk, b <= nb
__global__ void k_merge_partition(int64_t n, int64_t nnz, const int32_t* __restrict__ rowptr, int64_t nb,
                                  int64_t* __restrict__ part_row) {
  const int64_t total = n + nnz;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b <= nb; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t dd = b * kMergeBlk < total ? b * kMergeBlk : total;
    part_row[b] = merge_split(dd, n, nnz, rowptr);
  }
}

// w' = A x by merge path.  CTA b owns merge positions [b B, (b + 1) B)
// (B = kMergeBlk rows + entries): first its entries' double-float products
// a_p x[col_p] (coalesced, many loads in flight) and its rows' end offsets go
// to shared memory, then thread t walks positions [t K, (t + 1) K) of them
// (K = kMergeItems): a row ending in its range is written to wd (partial when
// it began before), the row still open at its end goes to (mp_row, mp_val).
// The products and their order within a row are those of the CSR kernel.
template <class TA>
__global__ void __launch_bounds__(kMergeCta) k_df_spmv_merge(
    int64_t n, int64_t nnz, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
    const TA* __restrict__ vals, const float2* __restrict__ x2, const float* __restrict__ x1,
    const int64_t* __restrict__ part_row, float2* __restrict__ wd, int* __restrict__ mp_row,
    float2* __restrict__ mp_val, int64_t nthreads) {
  __shared__ float2 prod[kMergeBlk];
  __shared__ int32_t rend[kMergeBlk + 1];
  __shared__ int crow[kMergeCta];       // row open at the end of each thread's range (-1: none)
  __shared__ float2 cval[kMergeCta];    // its partial sum
  __shared__ float2 fval[kMergeCta];    // partial sum of the first row the thread completes
  __shared__ int fhas[kMergeCta];       // whether the thread completes a row
  const int64_t total = n + nnz;
  const int64_t b = blockIdx.x;
  const int64_t rlo = part_row[b], rhi = part_row[b + 1];
  const int64_t dlo = b * kMergeBlk, dhi = dlo + kMergeBlk < total ? dlo + kMergeBlk : total;
  const int64_t jlo = dlo - rlo, jhi = dhi - rhi;     // entries of the CTA's range
  const int ne = (int)(jhi - jlo), nr = (int)(rhi - rlo);
  // products a_p x[col_p], eight entries per thread in flight at a time
  for (int e0 = threadIdx.x; e0 < ne; e0 += 8 * kMergeCta) {
    int c[8];
    float2 a[8], xv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * kMergeCta;
      c[u] = e < ne ? colind[jlo + e] : 0;
      a[u] = e < ne ? ldv(vals + jlo + e) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) xv[u] = x2 ? x2[c[u]] : make_float2(x1[c[u]], 0.f);   // c = 0 past the end
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * kMergeCta;
      if (e < ne) {
        const float pr = a[u].x * xv[u].x;
        float er = fmaf(a[u].x, xv[u].x, -pr);
        er = fmaf(a[u].x, xv[u].y, er);
        er = fmaf(a[u].y, xv[u].x, er);
        prod[e] = make_float2(pr, er);
      }
    }
  }
  for (int r = threadIdx.x; r <= nr; r += kMergeCta) rend[r] = rowptr[rlo + r + 1 <= n ? rlo + r + 1 : n];
  crow[threadIdx.x] = -1;
  cval[threadIdx.x] = make_float2(0.f, 0.f);
  fval[threadIdx.x] = make_float2(0.f, 0.f);
  fhas[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t = b * kMergeCta + threadIdx.x;
  const int64_t d0 = t * kMergeItems;
  const int64_t d1 = d0 + kMergeItems < total ? d0 + kMergeItems : total;
  if (t < nthreads && d0 < total) {
    // split inside the CTA's rows: marker of row rlo + q at rend[q] + rlo + q
    auto split = [&](int64_t dd) {
      int lo = 0, hi = nr;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int64_t)rend[mid] + rlo + mid < dd) lo = mid + 1;
        else hi = mid;
      }
      return lo;
    };
    int q = split(d0);
    const int qe = split(d1);
    int64_t j = d0 - (rlo + q);
    const int64_t je = d1 - (rlo + qe);
    float sh = 0.f, sl = 0.f;
    bool first = true;
    for (; q < qe; ++q) {
      const int64_t pe = rend[q];
      for (; j < pe; ++j) {
        const float2 v = prod[j - jlo];
        df_add(v.x, v.y, sh, sl);
      }
      // the first row this thread completes is the one it started in, which
      // may have begun in earlier ranges: its sum is finished by the fold
      if (first) {
        fval[threadIdx.x] = df_norm(sh, sl);
        fhas[threadIdx.x] = 1;
        first = false;
      } else {
        wd[rlo + q] = df_norm(sh, sl);
      }
      sh = 0.f;
      sl = 0.f;
    }
    for (; j < je; ++j) {
      const float2 v = prod[j - jlo];
      df_add(v.x, v.y, sh, sl);
    }
    crow[threadIdx.x] = rlo + qe < n ? (int)(rlo + qe) : -1;
    cval[threadIdx.x] = df_norm(sh, sl);
  }
  __syncthreads();
  // Fold in thread order, by warp 0: lane L folds the records of threads
  // 8L .. 8L+7 (the partial sums of the row it enters with, up to and with
  // its first completion, and the rows it completes after that, written
  // here), then lane 0 chains the 32 lanes: the running row collects each
  // lane's leading partial and is written at the lane's first completion.
  // The row open at the CTA's end becomes the CTA's carry (mp_row[b],
  // mp_val[b]; -1: none), added by k_df_merge_fix.  A fixed order: the sums
  // are the same bits on every run.
  if (threadIdx.x < 32) {
    constexpr int kSeg = kMergeCta / 32;
    const int lane = threadIdx.x;
    float ph = 0.f, pl = 0.f;          // contribution to the row the lane enters with
    float oh = 0.f, ol = 0.f;          // partial of the row open at the lane's end (after a completion)
    int has = 0, orow = -1;
    for (int q = 0; q < kSeg; ++q) {
      const int u = lane * kSeg + q;
      if (fhas[u]) {
        const float2 f = fval[u];
        if (!has) {
          df_add(f.x, f.y, ph, pl);
          has = 1;
        } else {
          df_add(f.x, f.y, oh, ol);
          if (orow >= 0) wd[orow] = df_norm(oh, ol);
        }
        orow = crow[u];
        const float2 v = cval[u];
        oh = 0.f;
        ol = 0.f;
        df_add(v.x, v.y, oh, ol);
      } else if (crow[u] >= 0) {
        const float2 v = cval[u];
        if (has) df_add(v.x, v.y, oh, ol);
        else df_add(v.x, v.y, ph, pl);
      }
    }
    const float2 pre = df_norm(ph, pl), post = df_norm(oh, ol);
    __shared__ float2 s_pre[32], s_post[32];
    __shared__ int s_has[32], s_orow[32];
    s_pre[lane] = pre;
    s_post[lane] = post;
    s_has[lane] = has;
    s_orow[lane] = orow;
    __syncwarp();
    if (lane == 0) {
      int rc = (int)rlo;
      float ch = 0.f, cl = 0.f;
      for (int L = 0; L < 32; ++L) {
        const float2 v = s_pre[L];
        df_add(v.x, v.y, ch, cl);
        if (s_has[L]) {
          if (rc >= 0) wd[rc] = df_norm(ch, cl);
          rc = s_orow[L];
          const float2 w2 = s_post[L];
          ch = 0.f;
          cl = 0.f;
          df_add(w2.x, w2.y, ch, cl);
        }
      }
      mp_row[b] = rc >= 0 && rc < n ? rc : -1;
      mp_val[b] = df_norm(ch, cl);
    }
  }
}

// Fold of the merge-path carries of the CTAs: the first CTA of each run of
// equal carry rows adds the run's partial sums, in CTA order, to that row.
__global__ void k_df_merge_fix(const int* __restrict__ mp_row, const float2* __restrict__ mp_val, int64_t nthreads,
                               float2* __restrict__ wd) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nthreads;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int r = mp_row[t];
    if (r < 0 || (t > 0 && mp_row[t - 1] == r)) continue;
    float sh = 0.f, sl = 0.f;
    for (int64_t u = t; u < nthreads && mp_row[u] == r; ++u) df_add(mp_val[u].x, mp_val[u].y, sh, sl);
    const float2 cur = wd[r];
    df_add(cur.x, cur.y, sh, sl);
    wd[r] = df_norm(sh, sl);
  }
}

// FP32 copy of a double-float vector (the stored basis vector of the FP32 phase)
__global__ void k_df_round_f32(int64_t n, const float2* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i].x + a[i].y;
}

// Offsets of the diagonal copy, passed by value.
struct DiaOffs {
  int o[16];
  int lo = 0, hi = 0;   // smallest and largest offset (the SpMV's interior-tile test)
};

// w = A x (+ the per-CTA partial sketches of w when SK) on the diagonal copy
// of A: every load independent of the others and coalesced (value of
// diagonal e at row i, x at i + off_e), the products in increasing column
// order (the CSR kernel's order, the same bits); two rows per thread, the
// tiles and the sketch gather of k_df_spmv_ell.
template <class TU, class TA, bool SK, int DMAX>
__global__ void __launch_bounds__(512, 2) k_df_spmv_dia(const DiaOffs offs, int D, const TA* __restrict__ dv,
                                                     int64_t ldd, int64_t n, const TU* __restrict__ x,
                                                     TU* __restrict__ w, const SketchTiles tv,
                                                     double* __restrict__ part) {
  static_assert(kTileRows == 1024, "two rows per thread of a 512-thread CTA");
  extern __shared__ __align__(16) uint8_t smraw[];
  const int d = tv.d, L1 = tv.L + 1;
  const TileSmem lay = tile_smem_layout(d, tv.L, 0, tv.zeta);
  float2* acc = reinterpret_cast<float2*>(smraw + lay.acc);
  if (SK)
    for (int r = threadIdx.x; r < d; r += blockDim.x) acc[r] = make_float2(0.f, 0.f);
  const int t0 = tv.ctile[blockIdx.x], t1 = tv.ctile[blockIdx.x + 1];
  const bool regs = SK && tile_regs_fit(tv);
  TileRegs R;
  if (regs && t0 < t1) tile_regs_load(tv, t0, R);
  for (int t = t0; t < t1; ++t) {
    const int buf = (t - t0) & 1;
    float2* v = reinterpret_cast<float2*>(smraw + lay.vb) + buf * kTileRows;
    int* of = reinterpret_cast<int*>(smraw + lay.offs) + buf * L1;
    uint32_t* ms = reinterpret_cast<uint32_t*>(smraw + lay.ms) + buf * d;
    uint16_t* es = reinterpret_cast<uint16_t*>(smraw + lay.es) + (size_t)buf * kTileRows * tv.zeta;
    const int64_t r0 = tv.row[t];
    const int rows = (int)(tv.row[t + 1] - r0);
    if (regs) {            // this tile's lists were loaded during the previous tile
      tile_regs_store(tv, t, R, of, ms, es);
      if (t + 1 < t1) tile_regs_load(tv, t + 1, R);
    } else if (SK) {
      tile_stage(tv, t, r0, rows, of, ms, es);
    }
    const int la = threadIdx.x, lb = threadIdx.x + 512;
    const bool oka = la < rows, okb = lb < rows;
    const int64_t ia = r0 + la, ib = r0 + lb;
    // rounds of four diagonals (eight for FP32 vectors and values): the loads
    // of a round are all in flight at once, and the registers stay within
    // two CTAs per SM
    constexpr int RU = sizeof(TU) == 4 && sizeof(TA) == 4 && DMAX == 8 ? 8 : 4;
    float sa = 0.f, ta = 0.f, sb = 0.f, tb = 0.f;
    // an interior tile (every x[i + off] of its rows inside 0 .. n-1, the
    // usual case) needs no bounds test: 32-bit offsets from the row pointers
    // (D <= 8 and FP32 values; the other kernels keep one path within their
    // registers)
    const bool interior = DMAX == 8 && sizeof(TA) == 4 && r0 + offs.lo >= 0 && r0 + kTileRows + offs.hi <= n;
    if (interior) {
      const TA* dva = dv + ia;
      const TU* xpa = x + ia;
#pragma unroll
      for (int e0 = 0; e0 < DMAX; e0 += RU) {
        float2 va[RU], vb[RU], xa[RU], xb[RU];
#pragma unroll
        for (int u = 0; u < RU; ++u) {
          const int e = e0 + u;
          const bool on = e < D;
          const TA* pv = dva + e * ldd;
          const TU* px = xpa + offs.o[e];
          va[u] = (on && oka) ? ldv(pv) : make_float2(0.f, 0.f);
          vb[u] = (on && okb) ? ldv(pv + 512) : make_float2(0.f, 0.f);
          xa[u] = (on && oka) ? ldv(px) : make_float2(0.f, 0.f);
          xb[u] = (on && okb) ? ldv(px + 512) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < RU; ++u) {
          if (e0 + u < D) {
            mac_st<TA, TU>(va[u], xa[u], sa, ta);
            mac_st<TA, TU>(vb[u], xb[u], sb, tb);
          }
        }
      }
    } else {
#pragma unroll
      for (int e0 = 0; e0 < DMAX; e0 += RU) {
        float2 va[RU], vb[RU], xa[RU], xb[RU];
#pragma unroll
        for (int u = 0; u < RU; ++u) {
          const int e = e0 + u;
          const bool on = e < D;
          const int64_t ja = ia + offs.o[e], jb = ib + offs.o[e];
          va[u] = (on && oka) ? ldv(dv + e * ldd + ia) : make_float2(0.f, 0.f);
          vb[u] = (on && okb) ? ldv(dv + e * ldd + ib) : make_float2(0.f, 0.f);
          xa[u] = (on && oka && ja >= 0 && ja < n) ? ldv(x + ja) : make_float2(0.f, 0.f);
          xb[u] = (on && okb && jb >= 0 && jb < n) ? ldv(x + jb) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < RU; ++u) {
          if (e0 + u < D) {
            mac_st<TA, TU>(va[u], xa[u], sa, ta);
            mac_st<TA, TU>(vb[u], xb[u], sb, tb);
          }
        }
      }
    }
    if (oka) v[la] = stv(w + ia, df_norm(sa, ta));
    if (okb) v[lb] = stv(w + ib, df_norm(sb, tb));
    if (SK) {
      __syncthreads();
      tile_gather<sizeof(TU) == 8>(d, tv.H, v, of, ms, es, acc);
    }
  }
  if (SK) tile_write_part(acc, d, part);
}

// Row i's entries into the diagonal copy (dv cleared before)
template <class TV>
__global__ void k_dia_fill(int64_t n, const DiaOffs offs, int D, int64_t ldd, const int32_t* __restrict__ rowptr,
                           const int32_t* __restrict__ colind, const TV* __restrict__ vals, TV* __restrict__ dv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const int64_t off = (int64_t)colind[p] - i;
      for (int e = 0; e < D; ++e)
        if (offs.o[e] == off) { dv[e * ldd + i] = vals[p]; break; }
    }
  }
}

// ELLPACK slots of row i (and the padding rows of the last slice)
template <class TV>
__global__ void k_ell_fill(int64_t n, int W, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                           const TV* __restrict__ vals, int32_t* __restrict__ ecol, TV* __restrict__ evals) {
  const int64_t nrow = (n + 31) / 32 * 32;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrow; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p0 = i < n ? rowptr[i] : 0;
    const int len = i < n ? (int)(rowptr[i + 1] - p0) : 0;
    const int64_t b = (((i >> 5) * W) << 5) + (i & 31);
    for (int e = 0; e < W; ++e) {
      const int64_t o = b + ((int64_t)e << 5);
      ecol[o] = e < len ? colind[p0 + e] : -1;
      evals[o] = e < len ? vals[p0 + e] : TV();
    }
  }
}

// Vector load of two consecutive rows (i even, ld even): float4 = two pairs,
// float2 = two FP32 values.
__device__ __forceinline__ void ld2(const float2* p, float2& a, float2& b) {
  float4 v = __ldcs(reinterpret_cast<const float4*>(p));
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld2(const float* p, float2& a, float2& b) {
  float2 v = __ldcs(reinterpret_cast<const float2*>(p));
  a = make_float2(v.x, 0.f);
  b = make_float2(v.y, 0.f);
}

// u~ = sj * w' + sum_{col < c} U[:, col] * nrs[col]  (nrs = -b .* scale, DF)
// written to U[:, c]; part[cta] = the CTA's Omega-sums of u~ as stored.
// A thread takes two consecutive rows (tile starts are even and ld is a
// multiple of 32, so the pair load stays aligned and inside the column).
// MODE 1: with the sketch; MODE 0: plain update (Euclidean CGS2); MODE 2:
// plain update, and part[cta] = the CTA's sum of squares of u~ as stored
// (FP64, fixed reduction order).
template <class TU, int UNR, int MINB, int MODE>
__global__ void __launch_bounds__(512, MINB) k_df_update_sketch(
    TU* __restrict__ U, int64_t ldu, int c, const float2* __restrict__ nrs, const float2* __restrict__ sj,
    const SketchTiles tv, double* __restrict__ part) {
  constexpr bool SK = MODE == 1;
  extern __shared__ __align__(16) uint8_t smraw[];
  const int d = tv.d, L1 = tv.L + 1;
  const TileSmem lay = tile_smem_layout(d, tv.L, c, tv.zeta);
  float2* acc = reinterpret_cast<float2*>(smraw + lay.acc);
  float2* rsh = reinterpret_cast<float2*>(smraw + lay.rsh);
  for (int col = threadIdx.x; col < c; col += blockDim.x) rsh[col] = nrs[col];
  if (SK)
    for (int r = threadIdx.x; r < d; r += blockDim.x) acc[r] = make_float2(0.f, 0.f);
  double ss = 0.0;
  __syncthreads();
  const float2 sc = sj[0];
  const int t0 = tv.ctile[blockIdx.x], t1 = tv.ctile[blockIdx.x + 1];
  // The second half of the grid takes its tiles last to first: the two CTAs
  // an SM holds (blocks b and b + G/2) then meet their short last tile at
  // different times, and the SM keeps more loads in flight.
  const bool rev = blockIdx.x >= gridDim.x / 2;
  for (int tt = t0; tt < t1; ++tt) {
    const int t = rev ? t1 - 1 - (tt - t0) : tt;
    const int buf = (tt - t0) & 1;
    float2* v = reinterpret_cast<float2*>(smraw + lay.vb) + buf * kTileRows;
    int* of = reinterpret_cast<int*>(smraw + lay.offs) + buf * L1;
    uint32_t* ms = reinterpret_cast<uint32_t*>(smraw + lay.ms) + buf * d;
    uint16_t* es = reinterpret_cast<uint16_t*>(smraw + lay.es) + (size_t)buf * kTileRows * tv.zeta;
    const int64_t r0 = tv.row[t];
    const int rows = (int)(tv.row[t + 1] - r0);
    if (SK) tile_stage(tv, t, r0, rows, of, ms, es);
    for (int l = 2 * threadIdx.x; l < rows; l += 2 * blockDim.x) {
      const int64_t i = r0 + l;
      float s0 = 0.f, t0a = 0.f, s1 = 0.f, t1a = 0.f;
      {
        float2 w0, w1;
        ld2(U + i + (int64_t)c * ldu, w0, w1);
        mac_st<TU, float2>(w0, sc, s0, t0a);
        mac_st<TU, float2>(w1, sc, s1, t1a);
      }
      const TU* up = U + i;
      int col = 0;
      for (; col + UNR <= c; col += UNR) {
        float2 a[UNR], bb[UNR];
#pragma unroll
        for (int q = 0; q < UNR; ++q) ld2(up + (int64_t)(col + q) * ldu, a[q], bb[q]);
#pragma unroll
        for (int q = 0; q < UNR; ++q) {
          const float2 r = rsh[col + q];
          mac_st<TU, float2>(a[q], r, s0, t0a);
          mac_st<TU, float2>(bb[q], r, s1, t1a);
        }
      }
      for (; col < c; ++col) {
        float2 a, bb;
        ld2(up + (int64_t)col * ldu, a, bb);
        const float2 r = rsh[col];
        mac_st<TU, float2>(a, r, s0, t0a);
        mac_st<TU, float2>(bb, r, s1, t1a);
      }
      const float2 v0 = stv(U + i + (int64_t)c * ldu, df_norm(s0, t0a));
      v[l] = v0;
      if (MODE == 2) { const double x = df_to_double(v0); ss = fma(x, x, ss); }
      if (l + 1 < rows) {
        const float2 v1 = stv(U + i + 1 + (int64_t)c * ldu, df_norm(s1, t1a));
        v[l + 1] = v1;
        if (MODE == 2) { const double x = df_to_double(v1); ss = fma(x, x, ss); }
      }
    }
    if (SK) {
      __syncthreads();
      tile_gather<sizeof(TU) == 8>(d, tv.H, v, of, ms, es, acc);
    }
  }
  if (SK) tile_write_part(acc, d, part);
  if (MODE == 2) {
    __shared__ double red[32];
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
      part[blockIdx.x] = s;
    }
  }
}

// Euclidean CGS2 (Krylov-Schur baseline): part[cta * c + l] = the CTA's
// partial of U[:, l]^T U[:, cv] for l < c (DF products, FP64 per CTA, fixed
// order).  Columns go in groups of 8 (U read once); U[:, cv] is re-read per
// group (from L2).
template <class TU>
__global__ void __launch_bounds__(512) k_df_dots(const TU* __restrict__ U, int64_t ldu, int c, int cv,
                                                 const SketchTiles tv, double* __restrict__ part) {
  __shared__ float2 red[16][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t0 = tv.ctile[blockIdx.x], t1 = tv.ctile[blockIdx.x + 1];
  const TU* vcol = U + (int64_t)cv * ldu;
  for (int g0 = 0; g0 < c; g0 += 8) {
    const int ng = min(8, c - g0);
    float s[8], e[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) { s[q] = 0.f; e[q] = 0.f; }
    for (int t = t0; t < t1; ++t) {
      const int64_t r0 = tv.row[t];
      const int rows = (int)(tv.row[t + 1] - r0);
      for (int l = 2 * threadIdx.x; l < rows; l += 2 * blockDim.x) {
        const int64_t i = r0 + l;
        float2 x0, x1;
        ld2(vcol + i, x0, x1);
        if (l + 1 >= rows) x1 = make_float2(0.f, 0.f);
        float2 a[8], b[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q < ng) ld2(U + i + (int64_t)(g0 + q) * ldu, a[q], b[q]);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q < ng) {
            df_mac(a[q].x, a[q].y, x0.x, x0.y, s[q], e[q]);
            df_mac(b[q].x, b[q].y, x1.x, x1.y, s[q], e[q]);
          }
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      df_warp_sum(s[q], e[q]);
      if (lane == 0) red[warp][q] = df_norm(s[q], e[q]);
    }
    __syncthreads();
    if (threadIdx.x < ng) {
      double v = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += df_to_double(red[w][threadIdx.x]);
      part[(size_t)blockIdx.x * c + g0 + threadIdx.x] = v;
    }
    __syncthreads();
  }
}

// Coefficients of one CGS2 pass from the folded dots g_l = u~_l^T v:
// pass 1 (v = w' = A u~_j): b_l = cs_l cs_j g_l, rprev = b, sj = cs_j;
// pass 2 (v = u~): b_l = cs_l g_l, rprev += b, sj = 1; nrs_l = -b_l cs_l.
// One CTA; the G partials of each l are added in CTA order.
__global__ void __launch_bounds__(256) k_ks_coef(int pass, int j, int c, int G, const double* __restrict__ part,
                                                 const double* __restrict__ colscale, double* __restrict__ rprev,
                                                 float2* __restrict__ nrs, float2* __restrict__ sj) {
  for (int l = threadIdx.x; l < c; l += blockDim.x) {
    double g = 0.0;
    for (int q = 0; q < G; ++q) g += part[(size_t)q * c + l];
    const double b = pass == 1 ? colscale[l] * colscale[j] * g : colscale[l] * g;
    rprev[l] = pass == 1 ? b : rprev[l] + b;
    nrs[l] = df_from_double(-b * colscale[l]);
  }
  if (threadIdx.x == 0) sj[0] = df_from_double(pass == 1 ? colscale[j] : 1.0);
}

// End of a CGS2 step j: beta = ||u~|| from the G sum-of-squares partials,
// colscale[j + 1] = 1/beta, coefficient column j = (rprev_0..j, beta); beta
// <= thr is a breakdown.  With j < 0 only the start vector's scale.
__global__ void k_ks_finish(int j, int G, const double* __restrict__ part, double thr,
                            double* __restrict__ colscale, const double* __restrict__ rprev, double* __restrict__ coef,
                            int ldcoef, int* flag) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double ss = 0.0;
  for (int q = 0; q < G; ++q) ss += part[q];
  const double beta = sqrt(ss);
  const bool finite = isfinite(beta);
  const bool brk = finite && !(beta > thr);
  colscale[j + 1] = (finite && !brk) ? 1.0 / beta : 0.0;
  if (j >= 0) {
    double* cc = coef + (size_t)j * ldcoef;
    for (int i = 0; i <= j; ++i) cc[i] = rprev[i];
    cc[j + 1] = beta;
  }
  if (!finite) atomicOr(flag, RKS_FLAG_NAN);
  else if (brk) atomicOr(flag, RKS_FLAG_BREAKDOWN);
}

// sum over g < G of part[g * d + r] by one warp: lane l adds g = l, l + 32,
// ... in order, then a fixed xor tree adds the 32 lane sums (every lane ends
// with the total).  The same order on every run.
__device__ __forceinline__ double fold_row(const double* __restrict__ part, int d, int G, int r, int lane) {
  double v = 0.0;
#pragma unroll 8
  for (int g = lane; g < G; g += 32) v += part[(size_t)g * d + r];
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// out = the CTA-ordered sum of the sketch kernels' partials (warp per row)
__global__ void __launch_bounds__(256) k_df_fold(const double* __restrict__ part, int d, int G,
                                                 double* __restrict__ out) {
  const int r = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= d) return;
  const double v = fold_row(part, d, G, r, lane);
  if (lane == 0) out[r] = v;
}

// Least squares b = S^+ z of one Arnoldi step (Alg. 2, Thm 4.3: against the
// locked and active sketches together), CGS2 in the sketch written through the
// Gram matrix M = S^T S: r1 = S^T z, r = r1 + S^T (z - S r1) = 2 r1 - M r1
// (the same quantity; M is the identity up to rounding).  M is kept on the
// device: the host sets it after every restart, and finishing column j adds
// its row M[:, j] = S^T s_j.  Phases (8 warps per CTA):
//   A  finish column j if requested (beta_j = ||s~_j||, S[:, j] in FP64 and
//      DF, colscale[j] = 1/beta_j, coefficient column j-1, flags: every CTA
//      computes beta_j itself, CTA 0 writes); then per column (one warp)
//      r1 = S^T z and, when finishing, the new row of M;
//   B  per column (one warp) r = 2 r1 - M r1, rprev = r (FP64),
//      nrs = -r .* colscale (DF), sj = colscale[j].
// k_df_ls_coop runs the fold of the sketch partials, A and B in one
// cooperative launch (two grid barriers); k_df_ls1 (A) and k_df_ls_gram (B)
// are the separate-launch form.
// z = z_raw * zscale * colscale[j] (z_raw is the sketch of the unscaled w').

__device__ double block_sum_d(double v, double* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[32] = v;
  }
  __syncthreads();
  return red[32];
}

// Phase A for one column (one warp): r1[col] = S[:, col]^T z (if want_r1)
// and, when column j is being finished (sjd = its DF values), the Gram entries
// M[col, j] = M[j, col] = S[:, col]^T s_j.  Column j itself reads sjd.
__device__ __forceinline__ void ls_phase_a(int col, int j, int d, int finish, int want_r1, const float2* S2,
                                           const float2* zd, const float2* sjd, float2* r1, float2* M2, int ldm,
                                           int lane) {
  const float2* sc = (finish && col == j) ? sjd : S2 + (size_t)col * d;
  float s = 0.f, t = 0.f, g = 0.f, ge = 0.f;
#pragma unroll 4
  for (int r = lane; r < d; r += 32) {
    const float2 a = sc[r];
    if (want_r1) {
      const float2 b = zd[r];
      df_mac(a.x, a.y, b.x, b.y, s, t);
    }
    if (finish) {
      const float2 b = sjd[r];
      df_mac(a.x, a.y, b.x, b.y, g, ge);
    }
  }
  if (want_r1) df_warp_sum(s, t);
  if (finish) df_warp_sum(g, ge);
  if (lane == 0) {
    if (want_r1) r1[col] = df_norm(s, t);
    if (finish) {
      const float2 m = df_norm(g, ge);
      M2[col + (size_t)j * ldm] = m;
      M2[j + (size_t)col * ldm] = m;
    }
  }
}

// Phase B for one column (one warp): r = 2 r1[col] - sum_l M[l, col] r1[l].
__device__ __forceinline__ void ls_phase_b(int col, int c, const float2* M2, int ldm, const float2* r1,
                                           const double* colscale, double* rprev, float2* nrs, int lane) {
  const float2* mc = M2 + (size_t)col * ldm;
  float s = 0.f, t = 0.f;
#pragma unroll 4
  for (int l = lane; l < c; l += 32) {
    const float2 a = mc[l], b = r1[l];
    df_mac(a.x, a.y, b.x, b.y, s, t);
  }
  df_warp_sum(s, t);
  if (lane == 0) {
    const float2 rc = r1[col];
    float hs = 2.f * rc.x, ht = 2.f * rc.y;   // exact doubling
    df_add(-s, -t, hs, ht);
    const double rd = df_to_double(df_norm(hs, ht));
    rprev[col] = rd;
    nrs[col] = df_from_double(-rd * colscale[col]);
  }
}

__global__ void __launch_bounds__(256) k_df_ls1(
    int j, int d, double zscale, int finish, int ls, double* __restrict__ s_raw, const double* __restrict__ z_raw,
    double* __restrict__ S64, float2* __restrict__ S2, double* __restrict__ colscale,
    const double* __restrict__ rprev, double* __restrict__ coef, int ldcoef, double* __restrict__ znorm_prev,
    float2* __restrict__ r1, float2* __restrict__ M2, int ldm, int* flag) {
  extern __shared__ float2 zd[];   // d: z; then d: s_j (when finishing)
  float2* sjd = zd + d;
  __shared__ double red[33];
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  double inv = 0.0;
  if (finish) {
    double ss = 0.0;
    for (int r = tid; r < d; r += nt) { double v = s_raw[r] * zscale; ss = fma(v, v, ss); }
    ss = block_sum_d(ss, red);
    const double beta = sqrt(ss);
    const bool finite = isfinite(beta);
    const bool brk = finite && !(beta > 1e-14 * znorm_prev[0]);
    inv = (finite && !brk) ? 1.0 / beta : 0.0;
    for (int r = tid; r < d; r += nt) sjd[r] = df_from_double(s_raw[r] * zscale * inv);
    if (blockIdx.x == 0) {
      for (int r = tid; r < d; r += nt) {
        double v = s_raw[r] * zscale * inv;
        S64[r + (size_t)j * d] = v;
        S2[r + (size_t)j * d] = df_from_double(v);
      }
      if (j >= 1) {
        double* cc = coef + (size_t)(j - 1) * ldcoef;
        for (int i = tid; i < j; i += nt) cc[i] = rprev[i];
        if (tid == 0) cc[j] = beta;
      }
      if (tid == 0) {
        colscale[j] = inv;
        if (!finite) atomicOr(flag, RKS_FLAG_NAN);
        else if (brk) atomicOr(flag, RKS_FLAG_BREAKDOWN);
      }
    }
  }
  if (!ls && !finish) return;
  if (ls) {
    const double scj = finish ? inv : colscale[j];
    double zz = 0.0;
    for (int r = tid; r < d; r += nt) {
      double v = z_raw[r] * zscale * scj;
      zz = fma(v, v, zz);
      zd[r] = df_from_double(v);
    }
    zz = block_sum_d(zz, red);
    if (blockIdx.x == 0 && tid == 0) znorm_prev[0] = sqrt(zz);
  }
  __syncthreads();
  const int c = j + 1;
  for (int col = blockIdx.x * nw + warp; col < c; col += gridDim.x * nw)
    ls_phase_a(col, j, d, finish, ls, S2, zd, sjd, r1, M2, ldm, lane);
}

// Phase B as its own launch (warp per column); CTA 0 also sets sj.
__global__ void __launch_bounds__(256) k_df_ls_gram(int j, const float2* __restrict__ M2, int ldm,
                                                    const float2* __restrict__ r1,
                                                    const double* __restrict__ colscale,
                                                    double* __restrict__ rprev, float2* __restrict__ nrs,
                                                    float2* __restrict__ sj) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int c = j + 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) sj[0] = df_from_double(colscale[j]);
  const int col = blockIdx.x * nw + warp;
  if (col < c) ls_phase_b(col, c, M2, ldm, r1, colscale, rprev, nrs, lane);
}

// Grid-wide barrier of the cooperative least-squares kernel.  bar[0] counts
// arrivals, bar[1] is the generation.  The wait is bounded (about a second of
// clock cycles): on timeout the kernel records RKS_FLAG_TIMEOUT and goes on,
// and the host reports the failure instead of the device hanging.  The
// cooperative launch guarantees that all CTAs are resident, so the bound is
// never reached in a correct run.
__device__ __forceinline__ void grid_barrier(unsigned* bar, unsigned nblocks, int* flag, long long limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    if (arrived == nblocks) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (clock64() - t0 > limit) { atomicOr(flag, RKS_FLAG_TIMEOUT); break; }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// Fold of the sketch partials, phase A and phase B in one cooperative launch.
// The kernel is a chain of L2 round trips, so everything that does not
// depend on the fold is loaded before it: each warp's column of S (phase A)
// and of M (phase B) into registers, z_raw together with s_raw.  The order of
// every sum is that of ls_phase_a / ls_phase_b, so the results are the same
// bits as theirs.
constexpr int kLsPre = 12;          // entries per lane prefetched for phase A (d <= 384 fully)
constexpr int kLsPreB = 4;          // for phase B (c <= 128 fully)
constexpr int kLsStageMax = 2048;   // d up to which z_raw / s_raw are staged in shared memory

__global__ void __launch_bounds__(256) k_df_ls_coop(
    int j, int d, double zscale, int finish, double* __restrict__ s_raw, double* __restrict__ z_raw,
    double* __restrict__ S64, float2* __restrict__ S2, double* __restrict__ colscale, double* __restrict__ rprev,
    double* __restrict__ coef, int ldcoef, double* __restrict__ znorm_prev, float2* __restrict__ nrs,
    float2* __restrict__ sj, float2* __restrict__ r1, float2* __restrict__ M2, int ldm,
    const double* __restrict__ part_z, const double* __restrict__ part_s, int G, unsigned* bar, int* flag,
    int stall) {
  extern __shared__ float2 zd[];   // d: z; d: s_j (when finishing); then 2d doubles: z_raw, s_raw
  float2* sjd = zd + d;
  double* zst = reinterpret_cast<double*>(sjd + d);
  double* sst = zst + d;
  __shared__ double red[33];
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  const int gw = blockIdx.x * nw + warp, tw = gridDim.x * nw;   // global warp index, warps in grid
  const int c = j + 1;
  // stall (a test hook) waits for one CTA more than the grid holds, so every
  // barrier runs out its short limit and the solve reports RKS_ETIMEOUT
  const unsigned expect = gridDim.x + (stall ? 1u : 0u);
  const long long limit = stall ? 2000000ll : 4000000000ll;
  const bool stage = d <= kLsStageMax;
  // prefetch (independent of the fold): this warp's first column
  const int col0 = gw;
  float2 pa[kLsPre], pb[kLsPreB];
  double cs0 = 0.0;
  const bool pre_a = col0 < c && !(finish && col0 == j);      // column j of S is new when finishing
  const bool pre_b = col0 < c && !(finish && col0 == j);      // so is column j of M
  if (pre_a) {
    const float2* sc = S2 + (size_t)col0 * d;
#pragma unroll
    for (int i = 0; i < kLsPre; ++i) {
      const int r = lane + 32 * i;
      pa[i] = r < d ? sc[r] : make_float2(0.f, 0.f);
    }
  }
  if (pre_b) {
    const float2* mc = M2 + (size_t)col0 * ldm;
#pragma unroll
    for (int i = 0; i < kLsPreB; ++i) {
      const int l = lane + 32 * i;
      pb[i] = (l < c && !(finish && l == j)) ? mc[l] : make_float2(0.f, 0.f);
    }
    cs0 = colscale[col0];
  }
  const double zn_prev = znorm_prev[0];
  // z' and s~_j from the sketch kernels' per-CTA partial sums
  {
    const int nb = finish ? 2 * d : d;
    for (int r = gw; r < nb; r += tw) {
      const bool isz = r < d;
      const double v = fold_row(isz ? part_z : part_s, d, G, isz ? r : r - d, lane);
      if (lane == 0) {
        if (isz) z_raw[r] = v;
        else s_raw[r - d] = v;
      }
    }
    grid_barrier(bar, expect, flag, limit);
  }
  // z_raw and s_raw in one round trip
  const double cs_j = finish ? 0.0 : colscale[j];
  if (stage) {
    for (int r = tid; r < d; r += nt) {
      zst[r] = z_raw[r];
      if (finish) sst[r] = s_raw[r];
    }
    __syncthreads();
  }
  const double* zsrc = stage ? zst : z_raw;
  const double* ssrc = stage ? sst : s_raw;
  double inv = 0.0;
  if (finish) {
    double ss = 0.0;
    for (int r = tid; r < d; r += nt) { double v = ssrc[r] * zscale; ss = fma(v, v, ss); }
    ss = block_sum_d(ss, red);
    const double beta = sqrt(ss);
    const bool finite = isfinite(beta);
    const bool brk = finite && !(beta > 1e-14 * zn_prev);
    inv = (finite && !brk) ? 1.0 / beta : 0.0;
    for (int r = tid; r < d; r += nt) sjd[r] = df_from_double(ssrc[r] * zscale * inv);
    if (blockIdx.x == 0) {
      for (int r = tid; r < d; r += nt) {
        double v = ssrc[r] * zscale * inv;
        S64[r + (size_t)j * d] = v;
        S2[r + (size_t)j * d] = df_from_double(v);
      }
      if (j >= 1) {
        double* cc = coef + (size_t)(j - 1) * ldcoef;
        for (int i = tid; i < j; i += nt) cc[i] = rprev[i];
        if (tid == 0) cc[j] = beta;
      }
      if (tid == 0) {
        colscale[j] = inv;
        if (!finite) atomicOr(flag, RKS_FLAG_NAN);
        else if (brk) atomicOr(flag, RKS_FLAG_BREAKDOWN);
      }
    }
  }
  const double scj = finish ? inv : cs_j;
  double zz = 0.0;
  for (int r = tid; r < d; r += nt) {
    double v = zsrc[r] * zscale * scj;
    zz = fma(v, v, zz);
    zd[r] = df_from_double(v);
  }
  zz = block_sum_d(zz, red);            // also orders the zd and sjd writes before their use
  // phase A: r1[col] = S[:, col]^T z and, when finishing, M[col, j] = S[:, col]^T s_j
  float2 mnew = make_float2(0.f, 0.f);  // M[j, col0] computed here (finishing)
  for (int col = gw; col < c; col += tw) {
    if (col == col0 && pre_a) {
      float s_ = 0.f, t_ = 0.f, g = 0.f, ge = 0.f;
      int i = 0;
#pragma unroll
      for (int ii = 0; ii < kLsPre; ++ii, ++i) {
        const int r = lane + 32 * ii;
        if (r < d) {
          const float2 a = pa[ii], b = zd[r];
          df_mac(a.x, a.y, b.x, b.y, s_, t_);
          if (finish) { const float2 e = sjd[r]; df_mac(a.x, a.y, e.x, e.y, g, ge); }
        }
      }
      for (int r = lane + 32 * kLsPre; r < d; r += 32) {
        const float2 a = S2[(size_t)col * d + r], b = zd[r];
        df_mac(a.x, a.y, b.x, b.y, s_, t_);
        if (finish) { const float2 e = sjd[r]; df_mac(a.x, a.y, e.x, e.y, g, ge); }
      }
      df_warp_sum(s_, t_);
      if (finish) df_warp_sum(g, ge);
      if (lane == 0) r1[col] = df_norm(s_, t_);
      if (finish) {
        mnew = df_norm(g, ge);
        if (lane == 0) {
          M2[col + (size_t)j * ldm] = mnew;
          M2[j + (size_t)col * ldm] = mnew;
        }
      }
    } else {
      ls_phase_a(col, j, d, finish, 1, S2, zd, sjd, r1, M2, ldm, lane);
    }
  }
  grid_barrier(bar, expect, flag, limit);
  // phase B
  if (blockIdx.x == 0 && tid == 0) { sj[0] = df_from_double(scj); znorm_prev[0] = sqrt(zz); }
  for (int col = gw; col < c; col += tw) {
    if (col == col0 && pre_b) {
      float s_ = 0.f, t_ = 0.f;
#pragma unroll
      for (int ii = 0; ii < kLsPreB; ++ii) {
        const int l = lane + 32 * ii;
        if (l < c) {
          const float2 a = (finish && l == j) ? mnew : pb[ii], b = r1[l];
          df_mac(a.x, a.y, b.x, b.y, s_, t_);
        }
      }
      for (int l = lane + 32 * kLsPreB; l < c; l += 32) {
        const float2 a = (finish && l == j) ? mnew : M2[l + (size_t)col * ldm], b = r1[l];
        df_mac(a.x, a.y, b.x, b.y, s_, t_);
      }
      df_warp_sum(s_, t_);
      if (lane == 0) {
        const float2 rc = r1[col];
        float hs = 2.f * rc.x, ht = 2.f * rc.y;   // exact doubling
        df_add(-s_, -t_, hs, ht);
        const double rd = df_to_double(df_norm(hs, ht));
        rprev[col] = rd;
        nrs[col] = df_from_double(-rd * cs0);
      }
    } else {
      ls_phase_b(col, c, M2, ldm, r1, colscale, rprev, nrs, lane);
    }
  }
}

// y = x (FP64) in the storage type
template <class TU>
__global__ void k_d2df(int64_t n, const double* __restrict__ x, TU* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    stv(y + i, df_from_double(x[i]));
}

// stored columns -> FP64 columns (ncols, with leading dimensions)
template <class TU>
__global__ void k_df2d_cols(int64_t n, const TU* __restrict__ x, int64_t ldx, double* __restrict__ y,
                            int64_t ldy, int ncols) {
  const int j = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i + (int64_t)j * ldy] = df_to_double(ldv(x + i + (int64_t)j * ldx));
}

// part[cta] = the CTA's Omega-sums of a stored vector (start vector)
template <class TU>
__global__ void __launch_bounds__(512) k_df_sketch_vec(const TU* __restrict__ x, const SketchTiles tv,
                                                       double* __restrict__ part) {
  extern __shared__ __align__(16) uint8_t smraw[];
  const int d = tv.d, L1 = tv.L + 1;
  const TileSmem lay = tile_smem_layout(d, tv.L, 0, tv.zeta);
  float2* acc = reinterpret_cast<float2*>(smraw + lay.acc);
  for (int r = threadIdx.x; r < d; r += blockDim.x) acc[r] = make_float2(0.f, 0.f);
  const int t0 = tv.ctile[blockIdx.x], t1 = tv.ctile[blockIdx.x + 1];
  for (int t = t0; t < t1; ++t) {
    const int buf = (t - t0) & 1;
    float2* v = reinterpret_cast<float2*>(smraw + lay.vb) + buf * kTileRows;
    int* of = reinterpret_cast<int*>(smraw + lay.offs) + buf * L1;
    uint32_t* ms = reinterpret_cast<uint32_t*>(smraw + lay.ms) + buf * d;
    uint16_t* es = reinterpret_cast<uint16_t*>(smraw + lay.es) + (size_t)buf * kTileRows * tv.zeta;
    const int64_t r0 = tv.row[t];
    const int rows = (int)(tv.row[t + 1] - r0);
    tile_stage(tv, t, r0, rows, of, ms, es);
    for (int l = threadIdx.x; l < rows; l += blockDim.x) v[l] = ldv(x + r0 + l);
    __syncthreads();
    tile_gather<sizeof(TU) == 8>(d, tv.H, v, of, ms, es, acc);
  }
  tile_write_part(acc, d, part);
}

// U[i, c0 + l] -= coef[l] * U[i, src] for l < ncols (double-float): one
// reflector applied to a block of columns (randomized Householder QR).
__global__ void __launch_bounds__(256) k_df_axpy_cols(int64_t n, float2* __restrict__ U, int64_t ldu, int src,
                                                      int c0, int ncols, const float2* __restrict__ coef) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 u = U[i + (int64_t)src * ldu];
    for (int l = 0; l < ncols; ++l) {
      float2* y = U + i + (int64_t)(c0 + l) * ldu;
      const float2 yv = *y, c = coef[l];
      float sh = yv.x, sl = yv.y;
      df_mac(-c.x, -c.y, u.x, u.y, sh, sl);
      *y = df_norm(sh, sl);
    }
  }
}

// Row-blocked DF product, in place: U[i, c0 + o] = sum_l U[i, a0 + l] Q[l, o]
// (Q DF, nin x nout column-major), then U[i, c0 + nout] = U[i, move_src].
template <class TU>
__global__ void __launch_bounds__(128) k_df_rows_gemm(int64_t n, TU* U, int64_t ldu, int a0, int nin,
                                                      const float2* __restrict__ Q, int nout, int c0,
                                                      int move_src) {
  extern __shared__ float2 shq[];
  float2* Qs = shq;
  float2* tmp = shq + (size_t)nin * nout;
  for (int t = threadIdx.x; t < nin * nout; t += blockDim.x) Qs[t] = Q[t];
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const TU* up = U + i + (int64_t)a0 * ldu;
  for (int o0 = 0; o0 < nout; o0 += 4) {
    float s[4] = {0.f, 0.f, 0.f, 0.f}, t[4] = {0.f, 0.f, 0.f, 0.f};
    const int no = min(4, nout - o0);
    for (int l = 0; l < nin; ++l) {
      float2 a = ldv(up + (int64_t)l * ldu);
#pragma unroll
      for (int o = 0; o < 4; ++o)
        if (o < no) {
          float2 q = Qs[l + (size_t)(o0 + o) * nin];
          df_mac(a.x, a.y, q.x, q.y, s[o], t[o]);
        }
    }
#pragma unroll
    for (int o = 0; o < 4; ++o)
      if (o < no) tmp[(size_t)(o0 + o) * blockDim.x + threadIdx.x] = df_norm(s[o], t[o]);
  }
  const TU mv = move_src >= 0 ? U[i + (int64_t)move_src * ldu] : TU();
  for (int o = 0; o < nout; ++o) stv(U + i + (int64_t)(c0 + o) * ldu, tmp[(size_t)o * blockDim.x + threadIdx.x]);
  if (move_src >= 0) U[i + (int64_t)(c0 + nout) * ldu] = mv;
}

// y = sum_{j < ncols} U[:, j] (FP32 columns), in FP64
__global__ void k_sum_cols_f32(int64_t n, const float* __restrict__ U, int64_t ldu, int ncols,
                               double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < ncols; ++j) s += (double)U[i + (int64_t)j * ldu];
    y[i] = s;
  }
}

// Restart product, in place: U[i, c0 + o] = sum_l U[i, a0 + l] Q[l, o] for
// o < nout (<= 4 * MAXOP), then U[i, c0 + nout] = U[i, move_src].  A CTA of
// 256 threads owns 64 rows; the 4 threads of a row split the outputs (up to
// MAXOP DF accumulators each, in registers).  Every read of the CTA's rows
// precedes the barrier, every write follows it, and no other CTA touches
// these rows, so the in-place update is safe.
template <class TU, int MAXOP>
__global__ void __launch_bounds__(256) k_df_restart(int64_t n, TU* U, int64_t ldu, int a0, int nin,
                                                    const float2* __restrict__ Q, int nout, int c0, int move_src) {
  extern __shared__ float2 qs[];                  // nin x nout, column-major
  for (int t = threadIdx.x; t < nin * nout; t += blockDim.x) qs[t] = Q[t];
  __syncthreads();
  const int r = threadIdx.x & 63, g = threadIdx.x >> 6;       // row in tile, output group
  const int64_t i = blockIdx.x * (int64_t)64 + r;
  const int per = (nout + 3) / 4;
  const int o0 = g * per;
  const int no = max(0, min(per, nout - o0));
  float s[MAXOP], t[MAXOP];
#pragma unroll
  for (int o = 0; o < MAXOP; ++o) { s[o] = 0.f; t[o] = 0.f; }
  TU mv{};
  if (i < n) {
    const TU* up = U + i + (int64_t)a0 * ldu;
    int l = 0;
    for (; l + 4 <= nin; l += 4) {          // four loads in flight per thread
      float2 a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = ldv(up + (int64_t)(l + u) * ldu);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float2* ql = qs + (l + u) + (size_t)o0 * nin;
#pragma unroll
        for (int o = 0; o < MAXOP; ++o)
          if (o < no) {
            const float2 q = ql[(size_t)o * nin];
            df_mac(a[u].x, a[u].y, q.x, q.y, s[o], t[o]);
          }
      }
    }
    for (; l < nin; ++l) {
      const float2 a = ldv(up + (int64_t)l * ldu);
      const float2* ql = qs + l + (size_t)o0 * nin;
#pragma unroll
      for (int o = 0; o < MAXOP; ++o)
        if (o < no) {
          const float2 q = ql[(size_t)o * nin];
          df_mac(a.x, a.y, q.x, q.y, s[o], t[o]);
        }
    }
    if (move_src >= 0 && g == 0) mv = U[i + (int64_t)move_src * ldu];
  }
  __syncthreads();
  if (i < n) {
#pragma unroll
    for (int o = 0; o < MAXOP; ++o)
      if (o < no) stv(U + i + (int64_t)(c0 + o0 + o) * ldu, df_norm(s[o], t[o]));
    if (move_src >= 0 && g == 0) U[i + (int64_t)(c0 + nout) * ldu] = mv;
  }
}

// ---------------------------------------------------------------------------
// Hand-over of the mixed path's FP32 Krylov-Schur decomposition
// A U = U T + u b^T to double-float: the FP32 basis promoted exactly, the
// relation error E = A U - U T - u b^T of the promoted columns, and damped
// Jacobi sweeps on A X - X T = -E for the correction U <- U + X.
// ---------------------------------------------------------------------------

// U2[:, j] = Uf[:, j], j < ncols (exact: the pairs' low words are zero)
__global__ void k_f32_to_df_cols(int64_t n, const float* __restrict__ Uf, int64_t ldu, int ncols,
                                 float2* __restrict__ U2) {
  const int64_t total = (int64_t)ncols * ldu;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q % ldu;
    if (i < n) U2[q] = make_float2(Uf[q], 0.f);
  }
}

// e = w - v - beta u in double-float, rounded to FP32 (column j of E:
// w = A u_j, v = (U T)_j, beta = b_j times the column scale of u)
__global__ void k_relation_resid(int64_t n, const float2* __restrict__ w, const float2* __restrict__ v,
                                 const float2* __restrict__ u, double beta, float* __restrict__ e) {
  const float2 nb = df_from_double(-beta);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 a = w[i], b = v[i], c = u[i];
    float s = a.x, t = a.y;
    df_add(-b.x, -b.y, s, t);
    df_mac(nb.x, nb.y, c.x, c.y, s, t);
    e[i] = s + t;
  }
}

// 1 / a_ii (0 where row i has no diagonal entry or a zero one)
__global__ void k_diag_inv(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                           const float* __restrict__ vals, float* __restrict__ dinv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float a = 0.f;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p)
      if (colind[p] == i) a += vals[p];
    dinv[i] = a != 0.f ? 1.0f / a : 0.f;
  }
}

// One damped Jacobi sweep on A X - X T = -E for all kk columns:
//   R = E + A X - Y (Y = X T, given),  Xn = X - omega D^{-1} R,
// a thread per row (the row's entries loaded once, up to 16 kept in
// registers), FP32 with FMA.  With part: the per-CTA sums of R^2 per column
// (warp sums by a fixed butterfly, then the warps in order) in
// part[blockIdx.x * kk + j].
constexpr int kJacobiCta = 256;
__global__ void __launch_bounds__(kJacobiCta) k_jacobi_sweep(int64_t n, const int32_t* __restrict__ rowptr,
                                                             const int32_t* __restrict__ colind,
                                                             const float* __restrict__ vals,
                                                             const float* __restrict__ dinv, int kk, int64_t ld,
                                                             const float* __restrict__ X,
                                                             const float* __restrict__ E,
                                                             const float* __restrict__ Y, float omega,
                                                             float* __restrict__ Xn, double* __restrict__ part) {
  constexpr int RM = 16;
  __shared__ double wsum[kJacobiCta / 32];
  const int64_t i = blockIdx.x * (int64_t)kJacobiCta + threadIdx.x;
  const bool on = i < n;
  int p0 = 0, len = 0;
  float di = 0.f;
  int cj[RM];
  float aj[RM];
  if (on) {
    p0 = rowptr[i];
    len = rowptr[i + 1] - p0;
    di = dinv[i];
  }
#pragma unroll
  for (int e = 0; e < RM; ++e) {
    const bool h = e < len;
    cj[e] = h ? colind[p0 + e] : 0;
    aj[e] = h ? vals[p0 + e] : 0.f;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j = 0; j < kk; ++j) {
    const int64_t o = (int64_t)j * ld;
    double r2 = 0.0;
    if (on) {
      float acc = E[o + i] - Y[o + i];
#pragma unroll
      for (int e = 0; e < RM; ++e)
        if (e < len) acc = fmaf(aj[e], X[o + cj[e]], acc);
      for (int e = RM; e < len; ++e) acc = fmaf(vals[p0 + e], X[o + colind[p0 + e]], acc);
      Xn[o + i] = fmaf(-omega * di, acc, X[o + i]);
      r2 = (double)acc * (double)acc;
    }
    if (part) {
      for (int s = 16; s; s >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, s);
      if (lane == 0) wsum[wid] = r2;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kJacobiCta / 32; ++w) t += wsum[w];
        part[(int64_t)blockIdx.x * kk + j] = t;
      }
      __syncthreads();
    }
  }
}

// U2[:, j] += X[:, j] (double-float + FP32), j < kk
__global__ void k_df_add_f32_cols(int64_t n, float2* __restrict__ U2, int64_t ldu, int kk,
                                  const float* __restrict__ X, int64_t ldx) {
  const int64_t total = (int64_t)kk * n;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = q / n, i = q - j * n;
    const float2 u = U2[j * ldu + i];
    float s = u.x, t = u.y;
    df_add(X[j * ldx + i], 0.f, s, t);
    U2[j * ldu + i] = df_norm(s, t);
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

static int df_grid(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  const int cap = kDfCtas;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

static cudaError_t configure_df_kernels_once() {
  const int big = 200 * 1024;
  cudaError_t e = cudaSuccess;
#define RKS_SMEM(f) if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, big)
  RKS_SMEM((k_df_spmv_sketch<float2, float2, true>)); RKS_SMEM((k_df_spmv_sketch<float, float, true>));
  RKS_SMEM((k_df_spmv_sketch<float2, float2, false>));
  RKS_SMEM((k_df_spmv_ell<float2, float2, true, 0>)); RKS_SMEM((k_df_spmv_ell<float, float, true, 0>));
  RKS_SMEM((k_df_spmv_warp<float2, float2, true, 32>)); RKS_SMEM((k_df_spmv_warp<float, float, true, 32>));
  RKS_SMEM((k_df_spmv_warp<float2, float2, false, 32>)); RKS_SMEM((k_df_spmv_warp<float2, float2, true, 8>));
  RKS_SMEM((k_df_spmv_warp<float, float, true, 8>)); RKS_SMEM((k_df_spmv_warp<float2, float2, false, 8>));
  RKS_SMEM((k_df_spmv_dia<float2, float2, true, 8>)); RKS_SMEM((k_df_spmv_dia<float, float, true, 8>));
  RKS_SMEM((k_df_spmv_dia<float2, float2, true, 16>)); RKS_SMEM((k_df_spmv_dia<float, float, true, 16>));
  RKS_SMEM((k_df_spmv_dia<float2, float2, false, 8>)); RKS_SMEM((k_df_spmv_dia<float2, float2, false, 16>));
  RKS_SMEM((k_df_spmv_dia<float2, float, true, 8>)); RKS_SMEM((k_df_spmv_dia<float2, float, false, 8>));
  RKS_SMEM((k_df_spmv_ell<float2, float2, false, 0>)); RKS_SMEM((k_df_spmv_ell<float2, float2, true, 6>));
  RKS_SMEM((k_df_spmv_ell<float, float, true, 6>)); RKS_SMEM((k_df_spmv_ell<float2, float2, false, 6>));
  constexpr int U8 = kDfUpdUnroll, MB = kDfUpdMinBlocks;
  RKS_SMEM((k_df_update_sketch<float2, U8, MB, 1>)); RKS_SMEM((k_df_update_sketch<float, 2 * U8, MB, 1>));
  RKS_SMEM((k_df_update_sketch<float2, U8, MB, 0>)); RKS_SMEM((k_df_update_sketch<float2, U8, MB, 2>));
  RKS_SMEM(k_df_sketch_vec<float2>); RKS_SMEM(k_df_sketch_vec<float>);
  RKS_SMEM(k_tiles_count<4>); RKS_SMEM(k_tiles_count<8>); RKS_SMEM(k_tiles_count<16>);
  RKS_SMEM(k_tiles_build<4>); RKS_SMEM(k_tiles_build<8>); RKS_SMEM(k_tiles_build<16>);
  RKS_SMEM(k_df_ls1);
  RKS_SMEM(k_df_ls_coop);
  RKS_SMEM(k_df_rows_gemm<float2>);
  RKS_SMEM(k_df_rows_gemm<float>);
  RKS_SMEM((k_df_restart<float2, 4>)); RKS_SMEM((k_df_restart<float2, 8>)); RKS_SMEM((k_df_restart<float2, 16>));
  RKS_SMEM((k_df_restart<float, 4>)); RKS_SMEM((k_df_restart<float, 8>)); RKS_SMEM((k_df_restart<float, 16>));
#undef RKS_SMEM
  return e;
}

cudaError_t configure_df_kernels() { return once_per_device(kCfgDf, configure_df_kernels_once); }

int df_small_smem(int d, int c) { return (int)((size_t)2 * d * sizeof(float2)); }
int df_gemm_smem(int nin, int nout) { return (int)(((size_t)nin * nout + (size_t)128 * nout) * sizeof(float2)); }

void launch_ell_fill(int64_t n, int W, const int32_t* rowptr, const int32_t* colind, const void* vals, bool f32,
                     int32_t* ecol, void* evals, cudaStream_t st) {
  const int g = df_grid((n + 31) / 32 * 32, 256);
  if (f32)
    k_ell_fill<float><<<g, 256, 0, st>>>(n, W, rowptr, colind, static_cast<const float*>(vals), ecol,
                                         static_cast<float*>(evals));
  else
    k_ell_fill<float2><<<g, 256, 0, st>>>(n, W, rowptr, colind, static_cast<const float2*>(vals), ecol,
                                          static_cast<float2*>(evals));
}

void launch_dia_fill(int64_t n, int D, const int* doff, int64_t ldd, const int32_t* rowptr, const int32_t* colind,
                     const void* vals, bool f32, void* dvals, cudaStream_t st) {
  DiaOffs o{};
  for (int e = 0; e < D && e < 16; ++e) o.o[e] = doff[e];
  const int g = df_grid(n, 256);
  cudaMemsetAsync(dvals, 0, (size_t)D * ldd * (f32 ? sizeof(float) : sizeof(float2)), st);
  if (f32)
    k_dia_fill<float><<<g, 256, 0, st>>>(n, o, D, ldd, rowptr, colind, static_cast<const float*>(vals),
                                         static_cast<float*>(dvals));
  else
    k_dia_fill<float2><<<g, 256, 0, st>>>(n, o, D, ldd, rowptr, colind, static_cast<const float2*>(vals),
                                          static_cast<float2*>(dvals));
}

template <class TU, bool SK>
static void launch_dia(const CsrDF& A, const void* x, void* w, const SketchTiles& t, double* part, size_t sm,
                       cudaStream_t st) {
  DiaOffs o{};
  for (int e = 0; e < A.D; ++e) o.o[e] = A.doff[e];
  o.lo = A.D ? A.doff[0] : 0;
  o.hi = A.D ? A.doff[A.D - 1] : 0;
  const TU* xx = static_cast<const TU*>(x);
  TU* ww = static_cast<TU*>(w);
  const TU* dv = static_cast<const TU*>(A.dvals);
  if (A.D > 8) {
    k_df_spmv_dia<TU, TU, SK, 16><<<t.G, 512, sm, st>>>(o, A.D, dv, A.ldd, A.n, xx, ww, t, part);
  } else if constexpr (std::is_same<TU, float2>::value) {
    // double-float vectors: the FP32 copy of the diagonals when every value
    // of A is an FP32 number (the pairs' low words are zero: the same bits)
    if (A.dvals_f32)
      k_df_spmv_dia<float2, float, SK, 8><<<t.G, 512, sm, st>>>(o, A.D, static_cast<const float*>(A.dvals_f32),
                                                                A.ldd, A.n, xx, ww, t, part);
    else
      k_df_spmv_dia<float2, float2, SK, 8><<<t.G, 512, sm, st>>>(o, A.D, dv, A.ldd, A.n, xx, ww, t, part);
  } else {
    k_df_spmv_dia<TU, TU, SK, 8><<<t.G, 512, sm, st>>>(o, A.D, dv, A.ldd, A.n, xx, ww, t, part);
  }
}

// The merge-path partition of A (the first row of every CTA's range), once per
// matrix: it depends on the row pointers only.
void launch_merge_partition(const CsrDF& A, cudaStream_t st) {
  const int64_t nb = (A.mp_threads + kMergeCta - 1) / kMergeCta;
  k_merge_partition<<<df_grid(nb + 1, 256), 256, 0, st>>>(A.n, A.nnz, A.rowptr, nb, A.mp_part);
}

// merge path: w = A x (double-float partials folded), then rounded to FP32 (f32)
static void launch_merge(const CsrDF& A, const void* x, void* w, cudaStream_t st) {
  float2* wd = A.f32 ? A.mp_w : static_cast<float2*>(w);
  const int64_t nb = (A.mp_threads + kMergeCta - 1) / kMergeCta;
  const float2* x2 = A.f32 ? nullptr : static_cast<const float2*>(x);
  const float* x1 = A.f32 ? static_cast<const float*>(x) : nullptr;
  if (A.f32)
    k_df_spmv_merge<float><<<(unsigned)nb, kMergeCta, 0, st>>>(A.n, A.nnz, A.rowptr, A.colind,
                                                              static_cast<const float*>(A.vals), x2, x1, A.mp_part,
                                                              wd, A.mp_row, A.mp_val, A.mp_threads);
  else
    k_df_spmv_merge<float2><<<(unsigned)nb, kMergeCta, 0, st>>>(A.n, A.nnz, A.rowptr, A.colind,
                                                               static_cast<const float2*>(A.vals), x2, x1, A.mp_part,
                                                               wd, A.mp_row, A.mp_val, A.mp_threads);
  k_df_merge_fix<<<df_grid(nb, 256), 256, 0, st>>>(A.mp_row, A.mp_val, nb, wd);
  if (A.f32) k_df_round_f32<<<df_grid(A.n, 256), 256, 0, st>>>(A.n, wd, static_cast<float*>(w));
}

void launch_df_spmv_sketch(const CsrDF& A, const void* x, void* w, const SketchTiles& t, double* part,
                           cudaStream_t st) {
  const size_t sm = tile_smem_bytes(t.d, t.L, 0, t.zeta);
  if (A.fmt == kSpmvMerge) {
    launch_merge(A, x, w, st);
    launch_df_sketch_vec(w, t, part, A.f32, st);
    return;
  }
  if (A.fmt == kSpmvWarp) {
    const bool wide = A.nnz >= 64 * A.n;   // mean row length >= 64: a warp per row, else 8 lanes
    if (A.f32) {
      auto k = wide ? k_df_spmv_warp<float, float, true, 32> : k_df_spmv_warp<float, float, true, 8>;
      k<<<t.G, 512, sm, st>>>(A.rowptr, A.colind, static_cast<const float*>(A.vals), static_cast<const float*>(x),
                              static_cast<float*>(w), t, part);
    } else {
      auto k = wide ? k_df_spmv_warp<float2, float2, true, 32> : k_df_spmv_warp<float2, float2, true, 8>;
      k<<<t.G, 512, sm, st>>>(A.rowptr, A.colind, static_cast<const float2*>(A.vals), static_cast<const float2*>(x),
                              static_cast<float2*>(w), t, part);
    }
    return;
  }
  if (A.dvals) {
    if (A.f32) launch_dia<float, true>(A, x, w, t, part, sm, st);
    else launch_dia<float2, true>(A, x, w, t, part, sm, st);
    return;
  }
  if (A.ecol) {
    const bool narrow = A.W <= 6;
    if (A.f32) {
      auto k = narrow ? k_df_spmv_ell<float, float, true, 6> : k_df_spmv_ell<float, float, true, 0>;
      k<<<t.G, 512, sm, st>>>(A.ecol, static_cast<const float*>(A.evals), A.W, static_cast<const float*>(x),
                              static_cast<float*>(w), t, part);
    } else {
      auto k = narrow ? k_df_spmv_ell<float2, float2, true, 6> : k_df_spmv_ell<float2, float2, true, 0>;
      k<<<t.G, 512, sm, st>>>(A.ecol, static_cast<const float2*>(A.evals), A.W, static_cast<const float2*>(x),
                              static_cast<float2*>(w), t, part);
    }
    return;
  }
  if (A.f32)
    k_df_spmv_sketch<float, float, true><<<t.G, 512, sm, st>>>(
        A.rowptr, A.colind, static_cast<const float*>(A.vals), static_cast<const float*>(x), static_cast<float*>(w),
        t, part);
  else
    k_df_spmv_sketch<float2, float2, true><<<t.G, 512, sm, st>>>(
        A.rowptr, A.colind, static_cast<const float2*>(A.vals), static_cast<const float2*>(x),
        static_cast<float2*>(w), t, part);
}

void launch_df_spmv(const CsrDF& A, const void* x, void* w, const SketchTiles& t, cudaStream_t st) {
  const size_t sm = tile_smem_bytes(t.d, t.L, 0, t.zeta);
  if (A.fmt == kSpmvMerge && !A.f32) {
    launch_merge(A, x, w, st);
    return;
  }
  if (A.fmt == kSpmvWarp && !A.f32) {
    auto k = A.nnz >= 64 * A.n ? k_df_spmv_warp<float2, float2, false, 32> : k_df_spmv_warp<float2, float2, false, 8>;
    k<<<t.G, 512, sm, st>>>(A.rowptr, A.colind, static_cast<const float2*>(A.vals), static_cast<const float2*>(x),
                            static_cast<float2*>(w), t, nullptr);
    return;
  }
  if (A.dvals && !A.f32) {
    launch_dia<float2, false>(A, x, w, t, nullptr, sm, st);
    return;
  }
  if (A.ecol && !A.f32) {
    auto k = A.W <= 6 ? k_df_spmv_ell<float2, float2, false, 6> : k_df_spmv_ell<float2, float2, false, 0>;
    k<<<t.G, 512, sm, st>>>(A.ecol, static_cast<const float2*>(A.evals), A.W, static_cast<const float2*>(x),
                            static_cast<float2*>(w), t, nullptr);
    return;
  }
  k_df_spmv_sketch<float2, float2, false><<<t.G, 512, sm, st>>>(
      A.rowptr, A.colind, static_cast<const float2*>(A.vals), static_cast<const float2*>(x), static_cast<float2*>(w),
      t, nullptr);
}

void launch_df_update_plain(void* U, int64_t ldu, int c, const float2* nrs, const float2* sj, const SketchTiles& t,
                            double* norm_part, cudaStream_t st) {
  constexpr int U8 = kDfUpdUnroll, MB = kDfUpdMinBlocks;
  const size_t sm = tile_smem_bytes(t.d, t.L, c, t.zeta);
  float2* u = static_cast<float2*>(U);
  if (norm_part) k_df_update_sketch<float2, U8, MB, 2><<<t.G, 512, sm, st>>>(u, ldu, c, nrs, sj, t, norm_part);
  else k_df_update_sketch<float2, U8, MB, 0><<<t.G, 512, sm, st>>>(u, ldu, c, nrs, sj, t, nullptr);
}

void launch_df_fold(const double* part, int d, int G, double* out, cudaStream_t st) {
  k_df_fold<<<(d + 7) / 8, 256, 0, st>>>(part, d, G, out);
}

void launch_df_dots(const void* U, int64_t ldu, int c, int cv, const SketchTiles& t, double* part, cudaStream_t st) {
  k_df_dots<float2><<<t.G, 512, 0, st>>>(static_cast<const float2*>(U), ldu, c, cv, t, part);
}

void launch_ks_coef(int pass, int j, int c, int G, const double* part, const double* colscale, double* rprev,
                    float2* nrs, float2* sj, cudaStream_t st) {
  k_ks_coef<<<1, 256, 0, st>>>(pass, j, c, G, part, colscale, rprev, nrs, sj);
}

void launch_ks_finish(int j, int G, const double* part, double thr, double* colscale,
                      const double* rprev, double* coef, int ldcoef, int* flag, cudaStream_t st) {
  k_ks_finish<<<1, 32, 0, st>>>(j, G, part, thr, colscale, rprev, coef, ldcoef, flag);
}

void launch_df_update_sketch(void* U, int64_t ldu, int c, const float2* nrs, const float2* sj, const SketchTiles& t,
                             double* part, bool f32, cudaStream_t st) {
  constexpr int U8 = kDfUpdUnroll, MB = kDfUpdMinBlocks;
  const size_t sm = tile_smem_bytes(t.d, t.L, c, t.zeta);
  // FP32 basis: twice the columns per batch, so that a thread has as many
  // bytes of loads in flight as with pairs (same order of the sums)
  if (f32)
    k_df_update_sketch<float, 2 * U8, MB, 1><<<t.G, 512, sm, st>>>(static_cast<float*>(U), ldu, c, nrs, sj, t,
                                                                   part);
  else
    k_df_update_sketch<float2, U8, MB, 1><<<t.G, 512, sm, st>>>(static_cast<float2*>(U), ldu, c, nrs, sj, t, part);
}

int launch_df_small(int j, int d, double zscale, int finish, int ls, double* s_raw, double* z_raw, double* S64,
                    float2* S2, double* colscale, double* rprev, double* coef, int ldcoef, double* znorm_prev,
                    float2* nrs, float2* sj, float2* r1, float2* M2, int ldm, const double* part_z,
                    const double* part_s, int G, int* flag, unsigned* bar, cudaStream_t st, int stall) {
  const size_t sm = (size_t)2 * d * sizeof(float2);
  const size_t sm_coop = sm + (d <= kLsStageMax ? (size_t)2 * d * sizeof(double) : 0);
  const int c = j + 1;
  if (ls && bar) {
    // one cooperative launch: partial-sum fold, phases A and B, two grid
    // barriers; a warp per folded row (the fold's L2 latency dominates, so one
    // row per warp beats fewer CTAs with less barrier traffic)
    const int nb = finish ? 2 * d : d;
    int g = (std::max(c, nb) + 7) / 8;
    g = std::min(g, 96);
    // a small problem (less than one wave of sketch CTAs) shares the GPU with
    // other solves: fewer CTAs are easier to co-schedule for the cooperative
    // launch (the fold of a row is the same whichever warp does it)
    if (G < 152) g = std::min((std::max(c, d) + 7) / 8, 48);
    void* args[] = {&j, &d, &zscale, &finish, &s_raw, &z_raw, &S64, &S2, &colscale, &rprev, &coef, &ldcoef,
                    &znorm_prev, &nrs, &sj, &r1, &M2, &ldm, &part_z, &part_s, &G, &bar, &flag, &stall};
    if (cudaLaunchCooperativeKernel((const void*)k_df_ls_coop, dim3(g), dim3(256), args, sm_coop, st) == cudaSuccess)
      return 1;
    (void)cudaGetLastError();   // not available: fall back to the kernels below
  }
  const int gf = (d + 7) / 8;
  int nl = 0;
  if (finish) { k_df_fold<<<gf, 256, 0, st>>>(part_s, d, G, s_raw); ++nl; }
  if (ls) { k_df_fold<<<gf, 256, 0, st>>>(part_z, d, G, z_raw); ++nl; }
  const int g1 = ls ? (c + 7) / 8 : 1;
  k_df_ls1<<<g1, 256, sm, st>>>(j, d, zscale, finish, ls, s_raw, z_raw, S64, S2, colscale, rprev, coef, ldcoef,
                                znorm_prev, r1, M2, ldm, flag);
  if (!ls) return nl + 1;
  k_df_ls_gram<<<(c + 7) / 8, 256, 0, st>>>(j, M2, ldm, r1, colscale, rprev, nrs, sj);
  return nl + 2;
}

void launch_omega_table(int64_t n, int d, int zeta, uint64_t seed, uint16_t* tab, int* flag, cudaStream_t st) {
  const int g = df_grid(n, 256) * 4;
  if (zeta <= 4) k_omega_table<4><<<g, 256, 0, st>>>(n, d, zeta, seed, tab, flag);
  else if (zeta <= 8) k_omega_table<8><<<g, 256, 0, st>>>(n, d, zeta, seed, tab, flag);
  else k_omega_table<16><<<g, 256, 0, st>>>(n, d, zeta, seed, tab, flag);
}

int omega_slots(int zeta) { return zeta <= 4 ? 4 : (zeta <= 8 ? 8 : 16); }

void launch_sum_cols_f32(int64_t n, const float* U, int64_t ldu, int ncols, double* y, cudaStream_t st) {
  k_sum_cols_f32<<<df_grid(n, 256) * 2, 256, 0, st>>>(n, U, ldu, ncols, y);
}

void launch_d2df(int64_t n, const double* x, void* y, bool f32, cudaStream_t st) {
  if (f32) k_d2df<float><<<df_grid(n, 256) * 2, 256, 0, st>>>(n, x, static_cast<float*>(y));
  else k_d2df<float2><<<df_grid(n, 256) * 2, 256, 0, st>>>(n, x, static_cast<float2*>(y));
}

void launch_df2d_cols(int64_t n, const void* x, int64_t ldx, double* y, int64_t ldy, int ncols, bool f32,
                      cudaStream_t st) {
  dim3 grid((unsigned)df_grid(n, 256), (unsigned)ncols);
  if (f32) k_df2d_cols<float><<<grid, 256, 0, st>>>(n, static_cast<const float*>(x), ldx, y, ldy, ncols);
  else k_df2d_cols<float2><<<grid, 256, 0, st>>>(n, static_cast<const float2*>(x), ldx, y, ldy, ncols);
}

void launch_df_axpy_cols(int64_t n, float2* U, int64_t ldu, int src, int c0, int ncols, const float2* coef,
                         cudaStream_t st) {
  if (ncols <= 0) return;
  const int g = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  k_df_axpy_cols<<<g, 256, 0, st>>>(n, U, ldu, src, c0, ncols, coef);
}

void launch_df_sketch_vec(const void* x, const SketchTiles& t, double* part, bool f32, cudaStream_t st) {
  const size_t sm = tile_smem_bytes(t.d, t.L, 0, t.zeta);
  if (f32) k_df_sketch_vec<float><<<t.G, 512, sm, st>>>(static_cast<const float*>(x), t, part);
  else k_df_sketch_vec<float2><<<t.G, 512, sm, st>>>(static_cast<const float2*>(x), t, part);
}

// Row ranges: G CTAs (at most kSketchCtas) own contiguous, even-aligned row
// ranges of equal length (to within two rows); each range is cut into tiles
// of at most kTileRows rows.  The partition depends on n only.
int build_sketch_tiles(int64_t n, int d, int zeta, const uint16_t* otab, SketchTiles* out, cudaStream_t st) {
  SketchTiles t;
  t.n = n; t.d = d; t.zeta = zeta;
  const int64_t npair = (n + 1) / 2;
  int64_t G = std::min<int64_t>(kSketchCtas, std::max<int64_t>(1, (n + kTileRows - 1) / kTileRows));
  G = std::max<int64_t>(1, std::min(G, npair));
  std::vector<int> ctile(G + 1);
  std::vector<int64_t> row;
  for (int64_t g = 0; g < G; ++g) {
    const int64_t a = 2 * (g * npair / G), b = std::min<int64_t>(n, 2 * ((g + 1) * npair / G));
    ctile[g] = (int)row.size();
    for (int64_t r = a; r < b; r += kTileRows) row.push_back(r);
  }
  ctile[G] = (int)row.size();
  row.push_back(n);
  t.G = (int)G;
  t.ntile = (int)row.size() - 1;
  t.H = 1;
  while (t.H < 8 && (int64_t)d * t.H * 2 <= 512) t.H *= 2;
  cudaError_t e = cudaMalloc(&t.row, row.size() * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc(&t.ctile, ctile.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(t.row, row.data(), row.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(t.ctile, ctile.data(), ctile.size() * sizeof(int), cudaMemcpyHostToDevice);
  int* lmax = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&lmax, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(lmax, 0, sizeof(int), st);
  const int slots = omega_slots(zeta);
  const size_t smc = (size_t)d * sizeof(int);
  if (e == cudaSuccess) {
    if (slots == 4) k_tiles_count<4><<<t.ntile, 256, smc, st>>>(t.row, d, otab, lmax);
    else if (slots == 8) k_tiles_count<8><<<t.ntile, 256, smc, st>>>(t.row, d, otab, lmax);
    else k_tiles_count<16><<<t.ntile, 256, smc, st>>>(t.row, d, otab, lmax);
    e = cudaGetLastError();
  }
  int L = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&L, lmax, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(lmax);
  t.L = L;
  if (e == cudaSuccess) e = cudaMalloc(&t.meta, (size_t)t.ntile * d * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&t.off, (size_t)t.ntile * (L + 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&t.ent, (size_t)n * zeta * sizeof(uint16_t));
  const size_t smb = ((size_t)4 * d + L + 1) * sizeof(int);
  if (e == cudaSuccess) {
    if (slots == 4) k_tiles_build<4><<<t.ntile, 256, smb, st>>>(t.row, d, zeta, L, otab, t.meta, t.off, t.ent);
    else if (slots == 8) k_tiles_build<8><<<t.ntile, 256, smb, st>>>(t.row, d, zeta, L, otab, t.meta, t.off, t.ent);
    else k_tiles_build<16><<<t.ntile, 256, smb, st>>>(t.row, d, zeta, L, otab, t.meta, t.off, t.ent);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  *out = t;
  return (int)e;
}

void free_sketch_tiles(SketchTiles* t) {
  cudaFree(t->row); cudaFree(t->ctile); cudaFree(t->meta); cudaFree(t->off); cudaFree(t->ent);
  *t = SketchTiles();
}

size_t sketch_tile_smem(const SketchTiles& t, int c) { return tile_smem_bytes(t.d, t.L, c, t.zeta); }

template <class TU>
static void restart_t(int64_t n, TU* U, int64_t ldu, int a0, int nin, const float2* Q, int nout, int c0,
                      int move_src, cudaStream_t st) {
  const size_t sm = (size_t)nin * nout * sizeof(float2);
  const int g = (int)((n + 63) / 64);
  const int per = (nout + 3) / 4;
  if (per <= 4) k_df_restart<TU, 4><<<g, 256, sm, st>>>(n, U, ldu, a0, nin, Q, nout, c0, move_src);
  else if (per <= 8) k_df_restart<TU, 8><<<g, 256, sm, st>>>(n, U, ldu, a0, nin, Q, nout, c0, move_src);
  else k_df_restart<TU, 16><<<g, 256, sm, st>>>(n, U, ldu, a0, nin, Q, nout, c0, move_src);
}

void launch_df_rows_gemm(int64_t n, void* U, int64_t ldu, int a0, int nin, const float2* Q, int nout, int c0,
                         int move_src, bool f32, cudaStream_t st) {
  if (nout <= 64) {        // register-tiled restart product
    if (f32) restart_t<float>(n, static_cast<float*>(U), ldu, a0, nin, Q, nout, c0, move_src, st);
    else restart_t<float2>(n, static_cast<float2*>(U), ldu, a0, nin, Q, nout, c0, move_src, st);
    return;
  }
  const size_t sm = (size_t)df_gemm_smem(nin, nout);
  const int g = (int)((n + 127) / 128);
  if (f32) k_df_rows_gemm<float><<<g, 128, sm, st>>>(n, static_cast<float*>(U), ldu, a0, nin, Q, nout, c0, move_src);
  else k_df_rows_gemm<float2><<<g, 128, sm, st>>>(n, static_cast<float2*>(U), ldu, a0, nin, Q, nout, c0, move_src);
}


void launch_f32_to_df_cols(int64_t n, const float* Uf, int64_t ldu, int ncols, float2* U2, cudaStream_t st) {
  k_f32_to_df_cols<<<df_grid((int64_t)ncols * ldu, 256), 256, 0, st>>>(n, Uf, ldu, ncols, U2);
}

void launch_relation_resid(int64_t n, const float2* w, const float2* v, const float2* u, double beta, float* e,
                           cudaStream_t st) {
  k_relation_resid<<<df_grid(n, 256), 256, 0, st>>>(n, w, v, u, beta, e);
}

void launch_diag_inv(int64_t n, const int32_t* rowptr, const int32_t* colind, const float* vals, float* dinv,
                     cudaStream_t st) {
  k_diag_inv<<<df_grid(n, 256), 256, 0, st>>>(n, rowptr, colind, vals, dinv);
}

int jacobi_sweep_ctas(int64_t n) { return (int)((n + kJacobiCta - 1) / kJacobiCta); }

void launch_jacobi_sweep(int64_t n, const int32_t* rowptr, const int32_t* colind, const float* vals,
                         const float* dinv, int kk, int64_t ld, const float* X, const float* E, const float* Y,
                         float omega, float* Xn, double* part, cudaStream_t st) {
  k_jacobi_sweep<<<jacobi_sweep_ctas(n), kJacobiCta, 0, st>>>(n, rowptr, colind, vals, dinv, kk, ld, X, E, Y, omega,
                                                              Xn, part);
}

void launch_df_add_f32_cols(int64_t n, float2* U2, int64_t ldu, int kk, const float* X, int64_t ldx,
                            cudaStream_t st) {
  k_df_add_f32_cols<<<df_grid((int64_t)kk * n, 256), 256, 0, st>>>(n, U2, ldu, kk, X, ldx);
}

}  // namespace rks
