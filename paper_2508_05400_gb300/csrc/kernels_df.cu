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

// ---------------------------------------------------------------------------
// sketch (same hash as kernels.cu; see rks.h)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t mix64_df(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Add sign * (vh + vl) of column i of Omega into the (hi, lo) bins.
template <int MAXZ>
__device__ __forceinline__ void df_sketch_add(float* bh, float* bl, uint64_t seed, uint64_t i, int d, int zeta,
                                              float vh, float vl, int* flag) {
  const uint64_t gamma = 0x9E3779B97F4A7C15ull;
  const uint64_t base = mix64_df(seed * gamma + i);
  int rows[MAXZ];
#pragma unroll
  for (int t = 0; t < MAXZ; ++t) rows[t] = -1;
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
      if (t == cnt) rows[t] = row;
    ++cnt;
    const float xh = (h & 1ull) ? -vh : vh;
    const float xl = (h & 1ull) ? -vl : vl;
    float old = atomicAdd(&bh[row], xh);
    float s, e;
    two_sum(old, xh, s, e);
    atomicAdd(&bl[row], e + xl);
  }
  if (cnt < zeta) atomicOr(flag, RKS_FLAG_HASH);
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

// w'[i] = sum_p A_p x[col_p]  (A and x in DF); out_raw += Omega-sums of w'.
template <int MAXZ>
__global__ void __launch_bounds__(512) k_df_spmv_sketch(
    int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
    const float2* __restrict__ vals, const float2* __restrict__ x, float2* __restrict__ w, int d, int zeta,
    uint64_t seed, double* out_raw, int* flag) {
  extern __shared__ float shf[];
  float* bh = shf;
  float* bl = shf + d;
  df_bins_zero(bh, bl, d);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f, t = 0.f;
    const int p0 = rowptr[i], p1 = rowptr[i + 1];
    for (int p = p0; p < p1; ++p) {
      float2 a = vals[p];
      float2 xv = x[colind[p]];
      df_mac(a.x, a.y, xv.x, xv.y, s, t);
    }
    float2 v = df_norm(s, t);
    w[i] = v;
    df_sketch_add<MAXZ>(bh, bl, seed, (uint64_t)i, d, zeta, v.x, v.y, flag);
  }
  df_bins_flush(bh, bl, out_raw, d);
}

// u~ = sj * w' + sum_{col < c} U[:, col] * nrs[col]  (nrs = -b .* scale, DF)
// written to U[:, c]; out_raw += Omega-sums of u~.
template <int MAXZ>
__global__ void __launch_bounds__(512) k_df_update_sketch(
    int64_t n, float2* __restrict__ U, int64_t ldu, int c, const float2* __restrict__ nrs,
    const float2* __restrict__ sj, int d, int zeta, uint64_t seed, double* out_raw, int* flag) {
  extern __shared__ float shf[];
  float* bh = shf;
  float* bl = shf + d;
  float2* rsh = reinterpret_cast<float2*>(shf + 2 * d + (2 * d & 1));
  for (int col = threadIdx.x; col < c; col += blockDim.x) rsh[col] = nrs[col];
  df_bins_zero(bh, bl, d);
  const float2 sc = sj[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f, t = 0.f;
    float2 wv = U[i + (int64_t)c * ldu];
    df_mac(wv.x, wv.y, sc.x, sc.y, s, t);
    const float2* up = U + i;
    int col = 0;
    for (; col + 4 <= c; col += 4) {
      float2 a0 = up[(int64_t)(col + 0) * ldu];
      float2 a1 = up[(int64_t)(col + 1) * ldu];
      float2 a2 = up[(int64_t)(col + 2) * ldu];
      float2 a3 = up[(int64_t)(col + 3) * ldu];
      float2 r0 = rsh[col + 0], r1 = rsh[col + 1], r2 = rsh[col + 2], r3 = rsh[col + 3];
      df_mac(a0.x, a0.y, r0.x, r0.y, s, t);
      df_mac(a1.x, a1.y, r1.x, r1.y, s, t);
      df_mac(a2.x, a2.y, r2.x, r2.y, s, t);
      df_mac(a3.x, a3.y, r3.x, r3.y, s, t);
    }
    for (; col < c; ++col) {
      float2 a = up[(int64_t)col * ldu];
      float2 r = rsh[col];
      df_mac(a.x, a.y, r.x, r.y, s, t);
    }
    float2 v = df_norm(s, t);
    U[i + (int64_t)c * ldu] = v;
    df_sketch_add<MAXZ>(bh, bl, seed, (uint64_t)i, d, zeta, v.x, v.y, flag);
  }
  df_bins_flush(bh, bl, out_raw, d);
}

// Block-wide sum of a double (blockDim multiple of 32, <= 1024).
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

// Single CTA.  (1) If finish: column j from s_raw (beta_j, S[:, j] in FP64
// and DF, colscale[j] = 1/beta_j, coefficient column j-1 = (r_prev, beta_j),
// breakdown / NaN flags).  (2) If ls: z = z_raw * zscale * colscale[j];
// r = S^+ z by CGS2 over the c = j + 1 columns; r -> rprev (FP64),
// nrs = -r .* colscale (DF), sj = colscale[j] (DF); zero z_raw.
__global__ void __launch_bounds__(1024) k_df_small(
    int j, int d, double zscale, int finish, int ls, double* __restrict__ s_raw, double* __restrict__ z_raw,
    double* __restrict__ S64, float2* __restrict__ S2, double* __restrict__ colscale,
    double* __restrict__ rprev, double* __restrict__ coef, int ldcoef, double* __restrict__ znorm_prev,
    float2* __restrict__ nrs, float2* __restrict__ sj, int* flag) {
  extern __shared__ float2 sh2[];
  float2* zd = sh2;            // d   : z (DF)
  float2* r1 = sh2 + d;        // c   : first pass coefficients
  float2* z1 = r1 + (j + 1);   // d   : z - S r1
  __shared__ double red[33];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  if (finish) {
    double ss = 0.0;
    for (int r = tid; r < d; r += nt) { double v = s_raw[r] * zscale; ss = fma(v, v, ss); }
    ss = block_sum_d(ss, red);
    const double beta = sqrt(ss);
    const double zn = znorm_prev[0];
    const bool finite = isfinite(beta);
    const bool brk = finite && !(beta > 1e-14 * zn);
    const double inv = (finite && !brk) ? 1.0 / beta : 0.0;
    for (int r = tid; r < d; r += nt) {
      double v = s_raw[r] * zscale * inv;
      S64[r + (size_t)j * d] = v;
      S2[r + (size_t)j * d] = df_from_double(v);
      s_raw[r] = 0.0;
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
    __syncthreads();
  }
  if (!ls) return;
  const int c = j + 1;
  const double scj = colscale[j];
  double zz = 0.0;
  for (int r = tid; r < d; r += nt) {
    double v = z_raw[r] * zscale * scj;
    zz = fma(v, v, zz);
    zd[r] = df_from_double(v);
    z_raw[r] = 0.0;
  }
  zz = block_sum_d(zz, red);   // also orders the zd writes before their use
  if (tid == 0) znorm_prev[0] = sqrt(zz);
  // pass 1: r1 = S^T z (warp per column)
  for (int col = warp; col < c; col += nw) {
    float s = 0.f, t = 0.f;
    const float2* sc = S2 + (size_t)col * d;
    for (int r = lane; r < d; r += 32) {
      float2 a = sc[r], b = zd[r];
      df_mac(a.x, a.y, b.x, b.y, s, t);
    }
    df_warp_sum(s, t);
    if (lane == 0) r1[col] = df_norm(s, t);
  }
  __syncthreads();
  // pass 2: z1 = z - S r1 (thread per row)
  for (int r = tid; r < d; r += nt) {
    float s = zd[r].x, t = zd[r].y;
    for (int col = 0; col < c; ++col) {
      float2 a = S2[r + (size_t)col * d], b = r1[col];
      df_mac(a.x, a.y, -b.x, -b.y, s, t);
    }
    z1[r] = df_norm(s, t);
  }
  __syncthreads();
  // pass 3: r = r1 + S^T z1
  for (int col = warp; col < c; col += nw) {
    float s = 0.f, t = 0.f;
    const float2* sc = S2 + (size_t)col * d;
    for (int r = lane; r < d; r += 32) {
      float2 a = sc[r], b = z1[r];
      df_mac(a.x, a.y, b.x, b.y, s, t);
    }
    df_warp_sum(s, t);
    if (lane == 0) {
      df_add(r1[col].x, r1[col].y, s, t);
      float2 rv = df_norm(s, t);
      double rd = df_to_double(rv);
      rprev[col] = rd;
      nrs[col] = df_from_double(-rd * colscale[col]);
    }
  }
  if (tid == 0) sj[0] = df_from_double(scj);
}

// u = x (FP64) as DF
__global__ void k_d2df(int64_t n, const double* __restrict__ x, float2* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = df_from_double(x[i]);
}

// DF columns -> FP64 columns (ncols, with leading dimensions)
__global__ void k_df2d_cols(int64_t n, const float2* __restrict__ x, int64_t ldx, double* __restrict__ y,
                            int64_t ldy, int ncols) {
  const int j = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i + (int64_t)j * ldy] = df_to_double(x[i + (int64_t)j * ldx]);
}

// sketch of a DF vector (start vector)
template <int MAXZ>
__global__ void __launch_bounds__(512) k_df_sketch_vec(int64_t n, const float2* __restrict__ x, int d, int zeta,
                                                       uint64_t seed, double* out_raw, int* flag) {
  extern __shared__ float shf[];
  float* bh = shf;
  float* bl = shf + d;
  df_bins_zero(bh, bl, d);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float2 v = x[i];
    df_sketch_add<MAXZ>(bh, bl, seed, (uint64_t)i, d, zeta, v.x, v.y, flag);
  }
  df_bins_flush(bh, bl, out_raw, d);
}

// Row-blocked DF product, in place: U[i, c0 + o] = sum_l U[i, a0 + l] Q[l, o]
// (Q DF, nin x nout column-major), then U[i, c0 + nout] = U[i, move_src].
__global__ void __launch_bounds__(128) k_df_rows_gemm(int64_t n, float2* U, int64_t ldu, int a0, int nin,
                                                      const float2* __restrict__ Q, int nout, int c0,
                                                      int move_src) {
  extern __shared__ float2 shq[];
  float2* Qs = shq;
  float2* tmp = shq + (size_t)nin * nout;
  for (int t = threadIdx.x; t < nin * nout; t += blockDim.x) Qs[t] = Q[t];
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2* up = U + i + (int64_t)a0 * ldu;
  for (int o0 = 0; o0 < nout; o0 += 4) {
    float s[4] = {0.f, 0.f, 0.f, 0.f}, t[4] = {0.f, 0.f, 0.f, 0.f};
    const int no = min(4, nout - o0);
    for (int l = 0; l < nin; ++l) {
      float2 a = up[(int64_t)l * ldu];
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
  const float2 mv = move_src >= 0 ? U[i + (int64_t)move_src * ldu] : make_float2(0.f, 0.f);
  for (int o = 0; o < nout; ++o) U[i + (int64_t)(c0 + o) * ldu] = tmp[(size_t)o * blockDim.x + threadIdx.x];
  if (move_src >= 0) U[i + (int64_t)(c0 + nout) * ldu] = mv;
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
  RKS_SMEM(k_df_spmv_sketch<4>); RKS_SMEM(k_df_spmv_sketch<8>); RKS_SMEM(k_df_spmv_sketch<16>);
  RKS_SMEM(k_df_update_sketch<4>); RKS_SMEM(k_df_update_sketch<8>); RKS_SMEM(k_df_update_sketch<16>);
  RKS_SMEM(k_df_sketch_vec<4>); RKS_SMEM(k_df_sketch_vec<8>); RKS_SMEM(k_df_sketch_vec<16>);
  RKS_SMEM(k_df_small);
  RKS_SMEM(k_df_rows_gemm);
#undef RKS_SMEM
  if (e == cudaSuccess) done = true;
  return e;
}

int df_small_smem(int d, int c) { return (int)((size_t)(2 * d + c) * sizeof(float2)); }
int df_gemm_smem(int nin, int nout) { return (int)(((size_t)nin * nout + (size_t)128 * nout) * sizeof(float2)); }

void launch_df_spmv_sketch(const CsrDF& A, const float2* x, float2* w, int d, int zeta, uint64_t seed,
                           double* out_raw, int* flag, cudaStream_t st) {
  const int g = df_grid(A.n, 512);
  const size_t sm = (size_t)2 * d * sizeof(float);
  if (zeta <= 4)
    k_df_spmv_sketch<4><<<g, 512, sm, st>>>(A.n, A.rowptr, A.colind, A.vals, x, w, d, zeta, seed, out_raw, flag);
  else if (zeta <= 8)
    k_df_spmv_sketch<8><<<g, 512, sm, st>>>(A.n, A.rowptr, A.colind, A.vals, x, w, d, zeta, seed, out_raw, flag);
  else
    k_df_spmv_sketch<16><<<g, 512, sm, st>>>(A.n, A.rowptr, A.colind, A.vals, x, w, d, zeta, seed, out_raw, flag);
}

void launch_df_update_sketch(int64_t n, float2* U, int64_t ldu, int c, const float2* nrs, const float2* sj,
                             int d, int zeta, uint64_t seed, double* out_raw, int* flag, cudaStream_t st) {
  const int g = df_grid(n, 512);
  const size_t sm = (size_t)(2 * d + 1) * sizeof(float) + (size_t)c * sizeof(float2) + 8;
  if (zeta <= 4)
    k_df_update_sketch<4><<<g, 512, sm, st>>>(n, U, ldu, c, nrs, sj, d, zeta, seed, out_raw, flag);
  else if (zeta <= 8)
    k_df_update_sketch<8><<<g, 512, sm, st>>>(n, U, ldu, c, nrs, sj, d, zeta, seed, out_raw, flag);
  else
    k_df_update_sketch<16><<<g, 512, sm, st>>>(n, U, ldu, c, nrs, sj, d, zeta, seed, out_raw, flag);
}

void launch_df_small(int j, int d, double zscale, int finish, int ls, double* s_raw, double* z_raw, double* S64,
                     float2* S2, double* colscale, double* rprev, double* coef, int ldcoef, double* znorm_prev,
                     float2* nrs, float2* sj, int* flag, cudaStream_t st) {
  const size_t sm = (size_t)df_small_smem(d, j + 1);
  k_df_small<<<1, 1024, sm, st>>>(j, d, zscale, finish, ls, s_raw, z_raw, S64, S2, colscale, rprev, coef, ldcoef,
                                  znorm_prev, nrs, sj, flag);
}

void launch_d2df(int64_t n, const double* x, float2* y, cudaStream_t st) {
  k_d2df<<<df_grid(n, 256) * 2, 256, 0, st>>>(n, x, y);
}

void launch_df2d_cols(int64_t n, const float2* x, int64_t ldx, double* y, int64_t ldy, int ncols, cudaStream_t st) {
  dim3 grid((unsigned)df_grid(n, 256), (unsigned)ncols);
  k_df2d_cols<<<grid, 256, 0, st>>>(n, x, ldx, y, ldy, ncols);
}

void launch_df_sketch_vec(int64_t n, const float2* x, int d, int zeta, uint64_t seed, double* out_raw, int* flag,
                          cudaStream_t st) {
  const int g = df_grid(n, 512);
  const size_t sm = (size_t)2 * d * sizeof(float);
  if (zeta <= 4) k_df_sketch_vec<4><<<g, 512, sm, st>>>(n, x, d, zeta, seed, out_raw, flag);
  else if (zeta <= 8) k_df_sketch_vec<8><<<g, 512, sm, st>>>(n, x, d, zeta, seed, out_raw, flag);
  else k_df_sketch_vec<16><<<g, 512, sm, st>>>(n, x, d, zeta, seed, out_raw, flag);
}

void launch_df_rows_gemm(int64_t n, float2* U, int64_t ldu, int a0, int nin, const float2* Q, int nout, int c0,
                         int move_src, cudaStream_t st) {
  const size_t sm = (size_t)df_gemm_smem(nin, nout);
  const int g = (int)((n + 127) / 128);
  k_df_rows_gemm<<<g, 128, sm, st>>>(n, U, ldu, a0, nin, Q, nout, c0, move_src);
}

}  // namespace rks
