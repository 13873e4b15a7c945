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
//   k_df_spmv_sketch  w' = A u~_j (unscaled, u_j = u~_j / beta_j), z' = Omega w'
//   k_df_small        finish column j (beta_j = ||s~_j||, S, scale, coefficient
//                     column), then b = S^+ z by CGS2 in the sketch against the
//                     locked and active columns (Thm 4.3), z = z' / beta_j
//   k_df_update_sketch u~_{j+1} = w'/beta_j - U b, s~_{j+1} = Omega u~_{j+1}
//
// Sketch accumulation: per-CTA bins hold (hi, lo) float pairs in shared
// memory.  A contribution x = xh + xl is added with a returning FP32 atomic on
// hi: from the returned old value the exact rounding error of old + xh is
// recovered (TwoSum) and added, with xl, to lo.  The bins are folded into the
// global FP64 d-vector with one FP64 atomic add per bin and CTA.

#include <algorithm>

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
// hash; unused slots (t >= zeta) are 0xFFFF.
template <int MAXZ>
struct OmegaRow { uint16_t e[MAXZ]; };

template <int MAXZ>
__device__ __forceinline__ OmegaRow<MAXZ> omega_load(const uint16_t* __restrict__ tab, int64_t i) {
  OmegaRow<MAXZ> r;
  if constexpr (MAXZ == 4) {
    uint2 v = __ldg(reinterpret_cast<const uint2*>(tab) + i);
    r.e[0] = v.x & 0xFFFF; r.e[1] = v.x >> 16; r.e[2] = v.y & 0xFFFF; r.e[3] = v.y >> 16;
  } else {
    const uint4* p = reinterpret_cast<const uint4*>(tab) + i * (MAXZ / 8);
#pragma unroll
    for (int q = 0; q < MAXZ / 8; ++q) {
      uint4 v = __ldg(p + q);
      r.e[8 * q + 0] = v.x & 0xFFFF; r.e[8 * q + 1] = v.x >> 16;
      r.e[8 * q + 2] = v.y & 0xFFFF; r.e[8 * q + 3] = v.y >> 16;
      r.e[8 * q + 4] = v.z & 0xFFFF; r.e[8 * q + 5] = v.z >> 16;
      r.e[8 * q + 6] = v.w & 0xFFFF; r.e[8 * q + 7] = v.w >> 16;
    }
  }
  return r;
}

// Add sign * (vh + vl) into the bins of the rows listed in `o`.
template <int MAXZ>
__device__ __forceinline__ void df_sketch_add_tab(float* bh, float* bl, const OmegaRow<MAXZ>& o, float vh,
                                                  float vl) {
#pragma unroll
  for (int t = 0; t < MAXZ; ++t) {
    const uint32_t e = o.e[t];
    if (e == 0xFFFFu) continue;
    const int row = e & 0x7FFF;
    const float xh = (e & 0x8000u) ? -vh : vh;
    const float xl = (e & 0x8000u) ? -vl : vl;
    float old = atomicAdd(&bh[row], xh);
    float s, er;
    two_sum(old, xh, s, er);
    atomicAdd(&bl[row], er + xl);
  }
}

__device__ __forceinline__ void df_bins_zero(float* bh, float* bl, int d) {
  for (int r = threadIdx.x; r < d; r += blockDim.x) { bh[r] = 0.f; bl[r] = 0.f; }
  __syncthreads();
}

__device__ __forceinline__ void df_bins_flush(const float* bh, const float* bl, double* out, int d) {
  __syncthreads();
  for (int r = threadIdx.x; r < d; r += blockDim.x) {
    double v = (double)bh[r] + (double)bl[r];
    if (v != 0.0) atomicAdd(&out[r], v);
  }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// The packed Omega table (see OmegaRow) from the hash of rks.h.
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

// w'[i] = sum_p A_p x[col_p]  (A and x in DF); out_raw += Omega-sums of w'.
template <int MAXZ, class TA, class TU>
__global__ void __launch_bounds__(512) k_df_spmv_sketch(
    int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
    const TA* __restrict__ vals, const TU* __restrict__ x, TU* __restrict__ w, int d,
    const uint16_t* __restrict__ otab, double* out_raw) {
  extern __shared__ float shf[];
  float* bh = shf;
  float* bl = shf + d;
  df_bins_zero(bh, bl, d);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f, t = 0.f;
    const int p0 = rowptr[i], p1 = rowptr[i + 1];
    for (int p = p0; p < p1; ++p) {
      float2 a = ldv(vals + p);
      float2 xv = ldv(x + colind[p]);
      df_mac(a.x, a.y, xv.x, xv.y, s, t);
    }
    const OmegaRow<MAXZ> o = omega_load<MAXZ>(otab, i);
    float2 v = stv(w + i, df_norm(s, t));
    df_sketch_add_tab<MAXZ>(bh, bl, o, v.x, v.y);
  }
  df_bins_flush(bh, bl, out_raw, d);
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
// written to U[:, c]; out_raw += Omega-sums of u~.
template <int MAXZ, class TU, int UNR, int MINB>
__global__ void __launch_bounds__(512, MINB) k_df_update_sketch(
    int64_t n, TU* __restrict__ U, int64_t ldu, int c, const float2* __restrict__ nrs,
    const float2* __restrict__ sj, int d, const uint16_t* __restrict__ otab, double* out_raw) {
  extern __shared__ float shf[];
  float* bh = shf;
  float* bl = shf + d;
  float2* rsh = reinterpret_cast<float2*>(shf + 2 * d);
  for (int col = threadIdx.x; col < c; col += blockDim.x) rsh[col] = nrs[col];
  df_bins_zero(bh, bl, d);
  const float2 sc = sj[0];
  const int64_t npair = (n + 1) / 2;
  for (int64_t pi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pi < npair;
       pi += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = 2 * pi;          // rows i, i + 1 (ld is a multiple of 32: the pair stays aligned)
    float s0 = 0.f, t0 = 0.f, s1 = 0.f, t1 = 0.f;
    {
      float2 w0, w1;
      ld2(U + i + (int64_t)c * ldu, w0, w1);
      df_mac(w0.x, w0.y, sc.x, sc.y, s0, t0);
      df_mac(w1.x, w1.y, sc.x, sc.y, s1, t1);
    }
    const TU* up = U + i;
    int col = 0;
    for (; col + UNR <= c; col += UNR) {
      float2 a[UNR], b[UNR];
#pragma unroll
      for (int q = 0; q < UNR; ++q) ld2(up + (int64_t)(col + q) * ldu, a[q], b[q]);
#pragma unroll
      for (int q = 0; q < UNR; ++q) {
        const float2 r = rsh[col + q];
        df_mac(a[q].x, a[q].y, r.x, r.y, s0, t0);
        df_mac(b[q].x, b[q].y, r.x, r.y, s1, t1);
      }
    }
    for (; col < c; ++col) {
      float2 a, b;
      ld2(up + (int64_t)col * ldu, a, b);
      const float2 r = rsh[col];
      df_mac(a.x, a.y, r.x, r.y, s0, t0);
      df_mac(b.x, b.y, r.x, r.y, s1, t1);
    }
    const float2 v0 = stv(U + i + (int64_t)c * ldu, df_norm(s0, t0));
    df_sketch_add_tab<MAXZ>(bh, bl, omega_load<MAXZ>(otab, i), v0.x, v0.y);
    if (i + 1 < n) {
      const float2 v1 = stv(U + i + 1 + (int64_t)c * ldu, df_norm(s1, t1));
      df_sketch_add_tab<MAXZ>(bh, bl, omega_load<MAXZ>(otab, i + 1), v1.x, v1.y);
    }
  }
  df_bins_flush(bh, bl, out_raw, d);
}


// Least squares b = S^+ z of one Arnoldi step, CGS2 in the sketch, in three
// multi-CTA kernels (8 warps per CTA):
//   k_df_ls1  finish column j if requested (beta_j = ||s~_j||, S[:, j] in FP64
//             and DF, colscale[j] = 1/beta_j, coefficient column j-1, flags:
//             every CTA computes beta_j itself, CTA 0 writes), then
//             r1 = S^T z (warp per column; column j read from s_raw directly);
//   k_df_ls2  z1 = z - S r1 (warp per row);
//   k_df_ls3  r = r1 + S^T z1 (warp per column), rprev = r (FP64),
//             nrs = -r .* colscale (DF), sj = colscale[j].
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

__global__ void __launch_bounds__(256) k_df_ls1(
    int j, int d, double zscale, int finish, int ls, double* __restrict__ s_raw, const double* __restrict__ z_raw,
    double* __restrict__ S64, float2* __restrict__ S2, double* __restrict__ colscale,
    const double* __restrict__ rprev, double* __restrict__ coef, int ldcoef, double* __restrict__ znorm_prev,
    float2* __restrict__ r1, int* flag) {
  extern __shared__ float2 zd[];   // d
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
      if (!ls) {                      // finish only (single CTA): clear the sums here
        __syncthreads();
        for (int r = tid; r < d; r += nt) s_raw[r] = 0.0;
      }
    }
  }
  if (!ls) return;
  const double scj = finish ? inv : colscale[j];
  double zz = 0.0;
  for (int r = tid; r < d; r += nt) {
    double v = z_raw[r] * zscale * scj;
    zz = fma(v, v, zz);
    zd[r] = df_from_double(v);
  }
  zz = block_sum_d(zz, red);            // also orders the zd writes before their use
  if (blockIdx.x == 0 && tid == 0) znorm_prev[0] = sqrt(zz);
  const int c = j + 1;
  const int col = blockIdx.x * nw + warp;
  if (col >= c) return;
  float s = 0.f, t = 0.f;
  if (finish && col == j) {             // the column finished above, straight from the sums
    for (int r = lane; r < d; r += 32) {
      float2 a = df_from_double(s_raw[r] * zscale * inv), b = zd[r];
      df_mac(a.x, a.y, b.x, b.y, s, t);
    }
  } else {
    const float2* sc = S2 + (size_t)col * d;
    for (int r = lane; r < d; r += 32) {
      float2 a = sc[r], b = zd[r];
      df_mac(a.x, a.y, b.x, b.y, s, t);
    }
  }
  df_warp_sum(s, t);
  if (lane == 0) r1[col] = df_norm(s, t);
}

// Grid-wide barrier of the cooperative least-squares kernel.  bar[0] counts
// arrivals, bar[1] is the generation.  The wait is bounded (about a second of
// clock cycles): on timeout the kernel records RKS_FLAG_TIMEOUT and goes on,
// and the host reports the failure instead of the device hanging.  The
// cooperative launch guarantees that all CTAs are resident, so the bound is
// never reached in a correct run.
__device__ __forceinline__ void grid_barrier(unsigned* bar, unsigned nblocks, int* flag) {
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
        if (clock64() - t0 > 4000000000ll) { atomicOr(flag, RKS_FLAG_TIMEOUT); break; }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// sum_r S2[r, col] * v[r] over r = lane, lane + 32, ... < d (DF), with the
// loads of four rows issued before their products (L2 latency overlap).
__device__ __forceinline__ void df_col_dot(const float2* __restrict__ sc, const float2* v, int d, int lane,
                                           float& s, float& t) {
  int r = lane;
  for (; r + 96 < d; r += 128) {
    const float2 a0 = sc[r], a1 = sc[r + 32], a2 = sc[r + 64], a3 = sc[r + 96];
    const float2 b0 = v[r], b1 = v[r + 32], b2 = v[r + 64], b3 = v[r + 96];
    df_mac(a0.x, a0.y, b0.x, b0.y, s, t);
    df_mac(a1.x, a1.y, b1.x, b1.y, s, t);
    df_mac(a2.x, a2.y, b2.x, b2.y, s, t);
    df_mac(a3.x, a3.y, b3.x, b3.y, s, t);
  }
  for (; r < d; r += 32) {
    const float2 a = sc[r], b = v[r];
    df_mac(a.x, a.y, b.x, b.y, s, t);
  }
}

// The three least-squares phases of k_df_ls1/2/3 in one cooperative launch.
__global__ void __launch_bounds__(256) k_df_ls_coop(
    int j, int d, double zscale, int finish, double* __restrict__ s_raw, double* __restrict__ z_raw,
    double* __restrict__ S64, float2* __restrict__ S2, double* __restrict__ colscale, double* __restrict__ rprev,
    double* __restrict__ coef, int ldcoef, double* __restrict__ znorm_prev, float2* __restrict__ nrs,
    float2* __restrict__ sj, float2* __restrict__ r1, float2* __restrict__ z1, unsigned* bar, int* flag) {
  extern __shared__ float2 zd[];   // d
  __shared__ double red[33];
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  const int gw = blockIdx.x * nw + warp, tw = gridDim.x * nw;   // global warp index, warps in grid
  const int c = j + 1;
  double inv = 0.0;
  if (finish) {
    double ss = 0.0;
    for (int r = tid; r < d; r += nt) { double v = s_raw[r] * zscale; ss = fma(v, v, ss); }
    ss = block_sum_d(ss, red);
    const double beta = sqrt(ss);
    const bool finite = isfinite(beta);
    const bool brk = finite && !(beta > 1e-14 * znorm_prev[0]);
    inv = (finite && !brk) ? 1.0 / beta : 0.0;
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
  const double scj = finish ? inv : colscale[j];
  double zz = 0.0;
  for (int r = tid; r < d; r += nt) {
    double v = z_raw[r] * zscale * scj;
    zz = fma(v, v, zz);
    zd[r] = df_from_double(v);
  }
  zz = block_sum_d(zz, red);
  // phase 1: r1 = S^T z (column j straight from the sums when just finished)
  for (int col = gw; col < c; col += tw) {
    float s = 0.f, t = 0.f;
    if (finish && col == j) {
      for (int r = lane; r < d; r += 32) {
        float2 a = df_from_double(s_raw[r] * zscale * inv), b = zd[r];
        df_mac(a.x, a.y, b.x, b.y, s, t);
      }
    } else {
      df_col_dot(S2 + (size_t)col * d, zd, d, lane, s, t);
    }
    df_warp_sum(s, t);
    if (lane == 0) r1[col] = df_norm(s, t);
  }
  grid_barrier(bar, gridDim.x, flag);
  // phase 2: z1 = z - S r1 (S[:, j] was written by CTA 0 before the barrier)
  for (int r = gw; r < d; r += tw) {
    float s = 0.f, t = 0.f;
    for (int col = lane; col < c; col += 32) {
      float2 a = S2[r + (size_t)col * d], b = r1[col];
      df_mac(a.x, a.y, b.x, b.y, s, t);
    }
    df_warp_sum(s, t);
    if (lane == 0) {
      float s2 = zd[r].x, t2 = zd[r].y;
      df_add(-s, -t, s2, t2);
      z1[r] = df_norm(s2, t2);
    }
  }
  grid_barrier(bar, gridDim.x, flag);
  // phase 3: r = r1 + S^T z1; clear the sums (no longer read)
  if (blockIdx.x == 0) {
    for (int r = tid; r < d; r += nt) { z_raw[r] = 0.0; s_raw[r] = 0.0; }
    if (tid == 0) { sj[0] = df_from_double(scj); znorm_prev[0] = sqrt(zz); }
  }
  for (int col = gw; col < c; col += tw) {
    float s = 0.f, t = 0.f;
    df_col_dot(S2 + (size_t)col * d, z1, d, lane, s, t);
    df_warp_sum(s, t);
    if (lane == 0) {
      df_add(r1[col].x, r1[col].y, s, t);
      const double rd = df_to_double(df_norm(s, t));
      rprev[col] = rd;
      nrs[col] = df_from_double(-rd * colscale[col]);
    }
  }
}

__global__ void __launch_bounds__(256) k_df_ls2(int j, int d, double zscale, double* __restrict__ s_raw,
                                                const double* __restrict__ z_raw, const float2* __restrict__ S2,
                                                const double* __restrict__ colscale, const float2* __restrict__ r1,
                                                float2* __restrict__ z1) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  const int c = j + 1;
  if (blockIdx.x == 0)
    for (int r = tid; r < d; r += blockDim.x) s_raw[r] = 0.0;   // no kernel of this step reads it again
  const int r = blockIdx.x * nw + warp;
  if (r >= d) return;
  float s = 0.f, t = 0.f;
  for (int col = lane; col < c; col += 32) {
    float2 a = S2[r + (size_t)col * d], b = r1[col];
    df_mac(a.x, a.y, b.x, b.y, s, t);
  }
  df_warp_sum(s, t);
  if (lane == 0) {
    float2 zr = df_from_double(z_raw[r] * zscale * colscale[j]);
    float s2 = zr.x, t2 = zr.y;
    df_add(-s, -t, s2, t2);
    z1[r] = df_norm(s2, t2);
  }
}

__global__ void __launch_bounds__(256) k_df_ls3(int j, int d, double* __restrict__ z_raw,
                                                const float2* __restrict__ S2, const double* __restrict__ colscale,
                                                const float2* __restrict__ r1, const float2* __restrict__ z1,
                                                double* __restrict__ rprev, float2* __restrict__ nrs,
                                                float2* __restrict__ sj) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  const int c = j + 1;
  if (blockIdx.x == 0) {
    for (int r = tid; r < d; r += blockDim.x) z_raw[r] = 0.0;   // read for the last time in k_df_ls2
    if (tid == 0) sj[0] = df_from_double(colscale[j]);
  }
  const int col = blockIdx.x * nw + warp;
  if (col >= c) return;
  float s = 0.f, t = 0.f;
  const float2* sc = S2 + (size_t)col * d;
  for (int r = lane; r < d; r += 32) {
    float2 a = sc[r], b = z1[r];
    df_mac(a.x, a.y, b.x, b.y, s, t);
  }
  df_warp_sum(s, t);
  if (lane == 0) {
    df_add(r1[col].x, r1[col].y, s, t);
    const double rd = df_to_double(df_norm(s, t));
    rprev[col] = rd;
    nrs[col] = df_from_double(-rd * colscale[col]);
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

// sketch of a DF vector (start vector)
template <int MAXZ, class TU>
__global__ void __launch_bounds__(512) k_df_sketch_vec(int64_t n, const TU* __restrict__ x, int d,
                                                       const uint16_t* __restrict__ otab, double* out_raw) {
  extern __shared__ float shf[];
  float* bh = shf;
  float* bl = shf + d;
  df_bins_zero(bh, bl, d);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float2 v = ldv(x + i);
    df_sketch_add_tab<MAXZ>(bh, bl, omega_load<MAXZ>(otab, i), v.x, v.y);
  }
  df_bins_flush(bh, bl, out_raw, d);
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
// launchers
// ---------------------------------------------------------------------------

static int df_grid(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  const int cap = kDfCtas;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t configure_df_kernels() {
  static bool done = false;
  if (done) return cudaSuccess;
  const int big = 200 * 1024;
  cudaError_t e = cudaSuccess;
#define RKS_SMEM(f) if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, big)
#define RKS_SMEM_T(TA, TU)                                                                          \
  RKS_SMEM((k_df_spmv_sketch<4, TA, TU>)); RKS_SMEM((k_df_spmv_sketch<8, TA, TU>));                  \
  RKS_SMEM((k_df_spmv_sketch<16, TA, TU>));
  RKS_SMEM_T(float2, float2) RKS_SMEM_T(float, float)
#undef RKS_SMEM_T
  constexpr int U8 = kDfUpdUnroll, MB = kDfUpdMinBlocks;
  RKS_SMEM((k_df_update_sketch<4, float2, U8, MB>)); RKS_SMEM((k_df_update_sketch<8, float2, U8, MB>));
  RKS_SMEM((k_df_update_sketch<16, float2, U8, MB>)); RKS_SMEM((k_df_update_sketch<4, float, U8, MB>));
  RKS_SMEM((k_df_update_sketch<8, float, U8, MB>)); RKS_SMEM((k_df_update_sketch<16, float, U8, MB>));
  RKS_SMEM((k_df_sketch_vec<4, float2>)); RKS_SMEM((k_df_sketch_vec<8, float2>)); RKS_SMEM((k_df_sketch_vec<16, float2>));
  RKS_SMEM((k_df_sketch_vec<4, float>)); RKS_SMEM((k_df_sketch_vec<8, float>)); RKS_SMEM((k_df_sketch_vec<16, float>));
  RKS_SMEM(k_df_ls1);
  RKS_SMEM(k_df_ls_coop);
  RKS_SMEM(k_df_rows_gemm<float2>);
  RKS_SMEM(k_df_rows_gemm<float>);
  RKS_SMEM((k_df_restart<float2, 4>)); RKS_SMEM((k_df_restart<float2, 8>)); RKS_SMEM((k_df_restart<float2, 16>));
  RKS_SMEM((k_df_restart<float, 4>)); RKS_SMEM((k_df_restart<float, 8>)); RKS_SMEM((k_df_restart<float, 16>));
#undef RKS_SMEM
  if (e == cudaSuccess) done = true;
  return e;
}

int df_small_smem(int d, int c) { return (int)((size_t)d * sizeof(float2)); }
int df_gemm_smem(int nin, int nout) { return (int)(((size_t)nin * nout + (size_t)128 * nout) * sizeof(float2)); }

template <class TA, class TU>
static void spmv_t(const CsrDF& A, const void* x, void* w, int d, int zeta, const uint16_t* otab, double* out_raw,
                   cudaStream_t st) {
  const int g = df_grid(A.n, 512);
  const size_t sm = (size_t)2 * d * sizeof(float);
  const TA* v = static_cast<const TA*>(A.vals);
  const TU* xx = static_cast<const TU*>(x);
  TU* ww = static_cast<TU*>(w);
  if (zeta <= 4)
    k_df_spmv_sketch<4, TA, TU><<<g, 512, sm, st>>>(A.n, A.rowptr, A.colind, v, xx, ww, d, otab, out_raw);
  else if (zeta <= 8)
    k_df_spmv_sketch<8, TA, TU><<<g, 512, sm, st>>>(A.n, A.rowptr, A.colind, v, xx, ww, d, otab, out_raw);
  else
    k_df_spmv_sketch<16, TA, TU><<<g, 512, sm, st>>>(A.n, A.rowptr, A.colind, v, xx, ww, d, otab, out_raw);
}

void launch_df_spmv_sketch(const CsrDF& A, const void* x, void* w, int d, int zeta, const uint16_t* otab,
                           double* out_raw, cudaStream_t st) {
  if (A.f32) spmv_t<float, float>(A, x, w, d, zeta, otab, out_raw, st);
  else spmv_t<float2, float2>(A, x, w, d, zeta, otab, out_raw, st);
}

template <class TU>
static void update_t(int64_t n, void* U, int64_t ldu, int c, const float2* nrs, const float2* sj, int d, int zeta,
                     const uint16_t* otab, double* out_raw, cudaStream_t st) {
  constexpr int U8 = kDfUpdUnroll, MB = kDfUpdMinBlocks;
  int64_t g64 = ((n + 1) / 2 + 511) / 512;
  if (g64 > 152 * MB) g64 = 152 * MB;
  const int g = (int)std::max<int64_t>(g64, 1);
  const size_t sm = (size_t)2 * d * sizeof(float) + (size_t)c * sizeof(float2) + 16;
  TU* u = static_cast<TU*>(U);
  if (zeta <= 4) k_df_update_sketch<4, TU, U8, MB><<<g, 512, sm, st>>>(n, u, ldu, c, nrs, sj, d, otab, out_raw);
  else if (zeta <= 8) k_df_update_sketch<8, TU, U8, MB><<<g, 512, sm, st>>>(n, u, ldu, c, nrs, sj, d, otab, out_raw);
  else k_df_update_sketch<16, TU, U8, MB><<<g, 512, sm, st>>>(n, u, ldu, c, nrs, sj, d, otab, out_raw);
}

void launch_df_update_sketch(int64_t n, void* U, int64_t ldu, int c, const float2* nrs, const float2* sj,
                             int d, int zeta, const uint16_t* otab, double* out_raw, bool f32, cudaStream_t st) {
  if (f32) update_t<float>(n, U, ldu, c, nrs, sj, d, zeta, otab, out_raw, st);
  else update_t<float2>(n, U, ldu, c, nrs, sj, d, zeta, otab, out_raw, st);
}

int launch_df_small(int j, int d, double zscale, int finish, int ls, double* s_raw, double* z_raw, double* S64,
                    float2* S2, double* colscale, double* rprev, double* coef, int ldcoef, double* znorm_prev,
                    float2* nrs, float2* sj, float2* r1, float2* z1, int* flag, unsigned* bar, cudaStream_t st) {
  const size_t sm = (size_t)d * sizeof(float2);
  const int c = j + 1;
  if (ls && bar) {
    // one cooperative launch: warps over columns / rows, two grid barriers
    int g = (std::max(c, d) + 7) / 8;
    g = std::min(g, 48);
    void* args[] = {&j, &d, &zscale, &finish, &s_raw, &z_raw, &S64, &S2, &colscale, &rprev, &coef, &ldcoef,
                    &znorm_prev, &nrs, &sj, &r1, &z1, &bar, &flag};
    if (cudaLaunchCooperativeKernel((const void*)k_df_ls_coop, dim3(g), dim3(256), args, sm, st) == cudaSuccess)
      return 1;
    (void)cudaGetLastError();   // not available: fall back to the three-kernel form below
  }
  const int g1 = ls ? (c + 7) / 8 : 1;
  k_df_ls1<<<g1, 256, sm, st>>>(j, d, zscale, finish, ls, s_raw, z_raw, S64, S2, colscale, rprev, coef, ldcoef,
                                znorm_prev, r1, flag);
  if (!ls) return 1;
  k_df_ls2<<<(d + 7) / 8, 256, 0, st>>>(j, d, zscale, s_raw, z_raw, S2, colscale, r1, z1);
  k_df_ls3<<<(c + 7) / 8, 256, 0, st>>>(j, d, z_raw, S2, colscale, r1, z1, rprev, nrs, sj);
  return 3;
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

template <class TU>
static void sketch_vec_t(int64_t n, const void* x, int d, int zeta, const uint16_t* otab, double* out_raw,
                         cudaStream_t st) {
  const int g = df_grid(n, 512);
  const size_t sm = (size_t)2 * d * sizeof(float);
  const TU* xx = static_cast<const TU*>(x);
  if (zeta <= 4) k_df_sketch_vec<4, TU><<<g, 512, sm, st>>>(n, xx, d, otab, out_raw);
  else if (zeta <= 8) k_df_sketch_vec<8, TU><<<g, 512, sm, st>>>(n, xx, d, otab, out_raw);
  else k_df_sketch_vec<16, TU><<<g, 512, sm, st>>>(n, xx, d, otab, out_raw);
}

void launch_df_sketch_vec(int64_t n, const void* x, int d, int zeta, const uint16_t* otab, double* out_raw,
                          bool f32, cudaStream_t st) {
  if (f32) sketch_vec_t<float>(n, x, d, zeta, otab, out_raw, st);
  else sketch_vec_t<float2>(n, x, d, zeta, otab, out_raw, st);
}

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

}  // namespace rks
