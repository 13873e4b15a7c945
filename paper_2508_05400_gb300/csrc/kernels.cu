// CUDA kernels of the rKS hot path (sm_103a), FP64 basis.
//
// One Arnoldi step of Algorithm 2 (Sec. 3.1) for the new column c = j + 1:
//   k_spmv_sketch   w = A u_j (u_j = U[:, j] * colscale[j]) -> U[:, c];
//                   z_raw += sum_i sign * w_i  (z = Omega w, Sec. 5 sketch)
//   k_ls_dot        r1 = S^T z                    (S = Omega U[:, 0..j])
//   k_ls_resid      z1 = z - S r1
//   k_ls_dot2       r = r1 + S^T z1, rs = r .* colscale   (CGS2 in the sketch
//                   for b_{j+1} = S^+ z; locked columns included: Thm 4.3)
//   k_update_sketch U[:, c] <- U[:, c] - U[:, 0..j] rs   (u~ = w - U b);
//                   s_raw += sum_i sign * u~_i            (s~ = Omega u~)
//   k_finish        beta = ||s~||, S[:, c] = s~/beta, colscale[c] = 1/beta,
//                   coefficient column, zero the accumulators.
// The basis is stored unnormalised: column c holds u~_c and colscale[c] =
// 1/beta_c (u_c = u~_c / beta_c), so no pass over n is spent on scaling.
//
// Restart (Algorithm 1, truncation; Eqs. 3.5-3.6): k_restart_gemm computes
// U[:, q..q+ka-1] = U[:, q..m-1] Q' in place, row by row, and moves the last
// vector u to column q + ka.
//
// Sketch: column i of Omega has zeta distinct rows from the SplitMix64 hash
// of (seed, i) (see rks.h); entries are sign/sqrt(zeta).  The kernels
// accumulate sign * v in FP64 shared-memory bins per CTA and fold the bins
// into a global d-vector with one atomic add per bin; the 1/sqrt(zeta) scale
// is applied by the consumers of the sums.

#include <mutex>

#include "rks_impl.h"

namespace rks {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

// Rows and signs (+1/-1) of column i of Omega.  Returns false if the draw cap
// was reached (cannot happen for d >= 2*zeta in practice).
template <int MAXZ>
__device__ __forceinline__ bool omega_column(uint64_t seed, uint64_t i, int d, int zeta,
                                             int (&rows)[MAXZ], double (&sgn)[MAXZ]) {
  const uint64_t base = mix64(seed * kGamma + i);
  int cnt = 0;
  const int cap = 32 * zeta;
#pragma unroll
  for (int t = 0; t < MAXZ; ++t) { rows[t] = -1; sgn[t] = 0.0; }
  for (int r = 0; r < cap && cnt < zeta; ++r) {
    uint64_t h = mix64(base + (uint64_t)(r + 1) * kGamma);
    int row = (int)(((h >> 32) * (uint64_t)d) >> 32);
    bool dup = false;
#pragma unroll
    for (int t = 0; t < MAXZ; ++t) dup |= (rows[t] == row);
    if (dup) continue;
    double s = (h & 1ull) ? -1.0 : 1.0;
#pragma unroll
    for (int t = 0; t < MAXZ; ++t) {
      if (t == cnt) { rows[t] = row; sgn[t] = s; }
    }
    ++cnt;
  }
  return cnt == zeta;
}

template <int MAXZ>
__device__ __forceinline__ void sketch_add(double* bins, uint64_t seed, uint64_t i, int d, int zeta,
                                           double v, int* flag) {
  int rows[MAXZ];
  double sgn[MAXZ];
  if (!omega_column<MAXZ>(seed, i, d, zeta, rows, sgn)) atomicOr(flag, RKS_FLAG_HASH);
#pragma unroll
  for (int t = 0; t < MAXZ; ++t)
    if (t < zeta && rows[t] >= 0) atomicAdd(&bins[rows[t]], sgn[t] * v);
}

__device__ __forceinline__ void bins_zero(double* bins, int d) {
  for (int r = threadIdx.x; r < d; r += blockDim.x) bins[r] = 0.0;
  __syncthreads();
}

__device__ __forceinline__ void bins_flush(const double* bins, double* out, int d) {
  __syncthreads();
  for (int r = threadIdx.x; r < d; r += blockDim.x) {
    double v = bins[r];
    if (v != 0.0) atomicAdd(&out[r], v);
  }
}

// ---------------------------------------------------------------------------

template <int MAXZ>
__global__ void k_sketch_pairs(int64_t n, int d, int zeta, uint64_t seed, int32_t* rows_out,
                               int8_t* signs_out, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int rows[MAXZ];
    double sgn[MAXZ];
    if (!omega_column<MAXZ>(seed, (uint64_t)i, d, zeta, rows, sgn)) atomicOr(flag, RKS_FLAG_HASH);
#pragma unroll
    for (int t = 0; t < MAXZ; ++t)
      if (t < zeta) {
        rows_out[i * zeta + t] = rows[t];
        signs_out[i * zeta + t] = (int8_t)(sgn[t] > 0 ? 1 : -1);
      }
  }
}

// out_raw += sum_i sign * (x_i * xscale)
template <int MAXZ>
__global__ void k_sketch_vec(int64_t n, const double* __restrict__ x, double xscale, int d, int zeta,
                             uint64_t seed, double* out_raw, int* flag) {
  extern __shared__ double bins[];
  bins_zero(bins, d);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    sketch_add<MAXZ>(bins, seed, (uint64_t)i, d, zeta, x[i] * xscale, flag);
  bins_flush(bins, out_raw, d);
}

// w = A (x * xscale[0]); out_raw += Omega-sums of w.
template <int MAXZ>
__global__ void k_spmv_sketch(int64_t n, const int32_t* __restrict__ rowptr,
                              const int32_t* __restrict__ colind, const double* __restrict__ vals,
                              const double* __restrict__ x, const double* __restrict__ xscale,
                              double* __restrict__ w, int d, int zeta, uint64_t seed,
                              double* out_raw, int* flag) {
  extern __shared__ double bins[];
  bins_zero(bins, d);
  const double sc = xscale[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) acc = fma(vals[p], x[colind[p]], acc);
    acc *= sc;
    w[i] = acc;
    sketch_add<MAXZ>(bins, seed, (uint64_t)i, d, zeta, acc, flag);
  }
  bins_flush(bins, out_raw, d);
}

// r[col] = sum_row S[row, col] * z_raw[row] * zscale, one warp per column.
__global__ void k_ls_dot(int c, int d, const double* __restrict__ S, const double* __restrict__ z,
                         double zscale, double* __restrict__ r) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= c) return;
  const double* s = S + (size_t)warp * d;
  double acc = 0.0;
  for (int row = lane; row < d; row += 32) acc = fma(s[row], z[row], acc);
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) r[warp] = acc * zscale;
}

// z1[row] = z_raw[row] * zscale - sum_col S[row, col] r1[col], one warp per row.
__global__ void k_ls_resid(int c, int d, const double* __restrict__ S, const double* __restrict__ z,
                           double zscale, const double* __restrict__ r1, double* __restrict__ z1) {
  int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (row >= d) return;
  double acc = 0.0;
  for (int col = lane; col < c; col += 32) acc = fma(S[row + (size_t)col * d], r1[col], acc);
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) z1[row] = z[row] * zscale - acc;
}

// r = r1 + S^T z1 ; rs = r .* colscale
__global__ void k_ls_dot2(int c, int d, const double* __restrict__ S, const double* __restrict__ z1,
                          const double* __restrict__ r1, const double* __restrict__ colscale,
                          double* __restrict__ r, double* __restrict__ rs) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= c) return;
  const double* s = S + (size_t)warp * d;
  double acc = 0.0;
  for (int row = lane; row < d; row += 32) acc = fma(s[row], z1[row], acc);
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    double v = r1[warp] + acc;
    r[warp] = v;
    rs[warp] = v * colscale[warp];
  }
}

// U[:, c] <- U[:, c] - U[:, 0..c-1] rs ; out_raw += Omega-sums of the result.
template <int MAXZ>
__global__ void k_update_sketch(int64_t n, double* __restrict__ U, int64_t ldu, int c,
                                const double* __restrict__ rs, int d, int zeta, uint64_t seed,
                                double* out_raw, int* flag) {
  extern __shared__ double sh[];
  double* bins = sh;
  double* rsh = sh + d;
  for (int col = threadIdx.x; col < c; col += blockDim.x) rsh[col] = rs[col];
  bins_zero(bins, d);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = U[i + (int64_t)c * ldu];
    const double* up = U + i;
    int col = 0;
    for (; col + 4 <= c; col += 4) {
      double a0 = up[(int64_t)(col + 0) * ldu], a1 = up[(int64_t)(col + 1) * ldu];
      double a2 = up[(int64_t)(col + 2) * ldu], a3 = up[(int64_t)(col + 3) * ldu];
      acc = fma(-a0, rsh[col + 0], acc);
      acc = fma(-a1, rsh[col + 1], acc);
      acc = fma(-a2, rsh[col + 2], acc);
      acc = fma(-a3, rsh[col + 3], acc);
    }
    for (; col < c; ++col) acc = fma(-up[(int64_t)col * ldu], rsh[col], acc);
    U[i + (int64_t)c * ldu] = acc;
    sketch_add<MAXZ>(bins, seed, (uint64_t)i, d, zeta, acc, flag);
  }
  bins_flush(bins, out_raw, d);
}

// One CTA: finish step c (see file header).  coef column c-1 gets (r, beta).
__global__ void k_finish(int c, int d, double zscale, double* __restrict__ s_raw,
                         double* __restrict__ z_raw, double* __restrict__ S,
                         double* __restrict__ colscale, const double* __restrict__ r,
                         double* __restrict__ coef, int ldcoef, int* flag) {
  __shared__ double red[2][32];
  double ss = 0.0, zz = 0.0;
  for (int row = threadIdx.x; row < d; row += blockDim.x) {
    double v = s_raw[row] * zscale;
    double w = z_raw[row] * zscale;
    ss = fma(v, v, ss);
    zz = fma(w, w, zz);
  }
  for (int o = 16; o; o >>= 1) {
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
    zz += __shfl_xor_sync(0xffffffffu, zz, o);
  }
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[0][warp] = ss; red[1][warp] = zz; }
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
    ss = lane < nw ? red[0][lane] : 0.0;
    zz = lane < nw ? red[1][lane] : 0.0;
    for (int o = 16; o; o >>= 1) {
      ss += __shfl_xor_sync(0xffffffffu, ss, o);
      zz += __shfl_xor_sync(0xffffffffu, zz, o);
    }
    if (lane == 0) { red[0][0] = ss; red[1][0] = zz; }
  }
  __syncthreads();
  const double beta = sqrt(red[0][0]);
  const double znorm = sqrt(red[1][0]);
  const bool finite = isfinite(beta) && isfinite(znorm);
  const bool brk = finite && !(beta > 1e-14 * znorm);
  const double inv = (finite && !brk) ? 1.0 / beta : 0.0;
  for (int row = threadIdx.x; row < d; row += blockDim.x) {
    S[row + (size_t)c * d] = s_raw[row] * zscale * inv;
    s_raw[row] = 0.0;
    z_raw[row] = 0.0;
  }
  double* cc = coef + (size_t)(c - 1) * ldcoef;
  for (int i = threadIdx.x; i < c; i += blockDim.x) cc[i] = r[i];
  if (threadIdx.x == 0) {
    cc[c] = beta;
    colscale[c] = inv;
    if (!finite) atomicOr(flag, RKS_FLAG_NAN);
    else if (brk) atomicOr(flag, RKS_FLAG_BREAKDOWN);
  }
}

// Initial vector: S[:, 0] = s/beta, colscale[0] = 1/beta from s_raw.
__global__ void k_start_finish(int d, double zscale, double* __restrict__ s_raw, double* __restrict__ S,
                               double* __restrict__ colscale, int* flag) {
  __shared__ double red[32];
  double ss = 0.0;
  for (int row = threadIdx.x; row < d; row += blockDim.x) {
    double v = s_raw[row] * zscale;
    ss = fma(v, v, ss);
  }
  for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = ss;
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
    ss = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) red[0] = ss;
  }
  __syncthreads();
  double beta = sqrt(red[0]);
  bool ok = isfinite(beta) && beta > 0.0;
  double inv = ok ? 1.0 / beta : 0.0;
  for (int row = threadIdx.x; row < d; row += blockDim.x) {
    S[row] = s_raw[row] * zscale * inv;
    s_raw[row] = 0.0;
  }
  if (threadIdx.x == 0) {
    colscale[0] = inv;
    if (!ok) atomicOr(flag, isfinite(beta) ? RKS_FLAG_BREAKDOWN : RKS_FLAG_NAN);
  }
}

// Default start vector: N(0,1) entries, SplitMix64 stream of `seed`
// (draw r = mix(seed + (r+1) gamma)), Box-Muller on draws (2i, 2i+1).
__global__ void k_start_vector(int64_t n, uint64_t seed, double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t h1 = mix64(seed + (uint64_t)(2 * i + 1) * kGamma);
    uint64_t h2 = mix64(seed + (uint64_t)(2 * i + 2) * kGamma);
    double u1 = (double)(h1 >> 11) * (1.0 / 9007199254740992.0);
    double u2 = (double)(h2 >> 11) * (1.0 / 9007199254740992.0);
    x[i] = sqrt(-2.0 * log1p(-u1)) * cospi(2.0 * u2);
  }
}

// Row-blocked small GEMM: C[i, 0..nout-1] = sum_l A[i, l] * B[l, o] for the
// rows of this CTA, A = columns a0..a0+nin-1 of (lda), C = columns c0.. of
// (ldc).  All reads of a row happen before its writes, so C may alias A.
// If move_src >= 0, column move_src of A is copied to column c0 + nout after.
// Dynamic shared memory: B (nin * nout) then tmp (blockDim * nout).
__global__ void k_rows_gemm(int64_t n, const double* A, int64_t lda, int a0, int nin,
                            const double* __restrict__ B, int nout, double* C, int64_t ldc, int c0,
                            int move_src) {
  extern __shared__ double sh[];
  double* Bs = sh;
  double* tmp = sh + (size_t)nin * nout;
  for (int t = threadIdx.x; t < nin * nout; t += blockDim.x) Bs[t] = B[t];
  __syncthreads();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* ap = A + i + (int64_t)a0 * lda;
  for (int o0 = 0; o0 < nout; o0 += 8) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int no = min(8, nout - o0);
    for (int l = 0; l < nin; ++l) {
      double a = ap[(int64_t)l * lda];
      const double* b = Bs + l + (size_t)o0 * nin;
#pragma unroll
      for (int o = 0; o < 8; ++o)
        if (o < no) acc[o] = fma(a, b[(size_t)o * nin], acc[o]);
    }
#pragma unroll
    for (int o = 0; o < 8; ++o)
      if (o < no) tmp[(size_t)(o0 + o) * blockDim.x + threadIdx.x] = acc[o];
  }
  double mv = move_src >= 0 ? A[i + (int64_t)move_src * lda] : 0.0;
  for (int o = 0; o < nout; ++o) C[i + (int64_t)(c0 + o) * ldc] = tmp[(size_t)o * blockDim.x + threadIdx.x];
  if (move_src >= 0) C[i + (int64_t)(c0 + nout) * ldc] = mv;
}

// y = A x for several columns: Y[:, j] = A X[:, j], j < ncols.
__global__ void k_spmm(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                       const double* __restrict__ vals, const double* __restrict__ X, int64_t ldx,
                       double* __restrict__ Y, int64_t ldy, int ncols) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int j = blockIdx.y;
  if (i >= n || j >= ncols) return;
  const double* x = X + (int64_t)j * ldx;
  double acc = 0.0;
  for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) acc = fma(vals[p], x[colind[p]], acc);
  Y[i + (int64_t)j * ldy] = acc;
}

// Residual sums of eigenpair column pair t (blockIdx.y): col[t] (re part),
// colim[t] (im part column or -1), lam (a, b).  out[t*6 + ...] +=
// {||r||^2, ||x||^2, Re x^H A x, Im x^H A x}.
__global__ void k_resid_sums(int64_t n, const double* __restrict__ X, const double* __restrict__ AX,
                             int64_t ld, const int* __restrict__ col, const int* __restrict__ colim,
                             const double* __restrict__ lre, const double* __restrict__ lim,
                             double* __restrict__ out) {
  int t = blockIdx.y;
  int cr = col[t], ci = colim[t];
  double a = lre[t], b = lim[t];
  double s[4] = {0, 0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double xr = X[i + (int64_t)cr * ld], axr = AX[i + (int64_t)cr * ld];
    double xi = ci >= 0 ? X[i + (int64_t)ci * ld] : 0.0;
    double axi = ci >= 0 ? AX[i + (int64_t)ci * ld] : 0.0;
    double rre = axr - a * xr + b * xi;
    double rim = axi - a * xi - b * xr;
    s[0] += rre * rre + rim * rim;
    s[1] += xr * xr + xi * xi;
    s[2] += xr * axr + xi * axi;
    s[3] += xr * axi - xi * axr;
  }
  __shared__ double red[4][32];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double v = s[q];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double v = lane < nw ? red[q][lane] : 0.0;
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) out[((size_t)t * 4 + q) * gridDim.x + blockIdx.x] = v;   // summed on the host in CTA order
    }
  }
}

__global__ void k_f32_to_f64(int64_t n, const float* __restrict__ a, double* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

__global__ void k_check_csr(int64_t n, int64_t nnz, const int32_t* __restrict__ rowptr,
                            const int32_t* __restrict__ colind, int* bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int a = rowptr[i], b = rowptr[i + 1];
    if (a > b || a < 0 || b > nnz) { atomicOr(bad, 1); continue; }
    for (int p = a; p < b; ++p)
      if (colind[p] < 0 || colind[p] >= n) { atomicOr(bad, 2); break; }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (rowptr[0] != 0 || rowptr[n] != nnz)) atomicOr(bad, 4);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

static int grid_for(int64_t n, int threads, int max_ctas) {
  int64_t g = (n + threads - 1) / threads;
  if (g > max_ctas) g = max_ctas;
  if (g < 1) g = 1;
  return (int)g;
}


void launch_sketch_pairs(int64_t n, int d, int zeta, uint64_t seed, int32_t* rows, int8_t* signs,
                         int* flag, cudaStream_t st) {
  int g = grid_for(n, 256, 152 * 8);
  if (zeta <= 4) k_sketch_pairs<4><<<g, 256, 0, st>>>(n, d, zeta, seed, rows, signs, flag);
  else if (zeta <= 8) k_sketch_pairs<8><<<g, 256, 0, st>>>(n, d, zeta, seed, rows, signs, flag);
  else k_sketch_pairs<16><<<g, 256, 0, st>>>(n, d, zeta, seed, rows, signs, flag);
}

void launch_sketch_vec(int64_t n, const double* x, double xscale, int d, int zeta, uint64_t seed,
                       double* out_raw, int* flag, cudaStream_t st) {
  int g = grid_for(n, 256, kSketchCtas);
  size_t sm = (size_t)d * sizeof(double);
  if (zeta <= 4) k_sketch_vec<4><<<g, 256, sm, st>>>(n, x, xscale, d, zeta, seed, out_raw, flag);
  else if (zeta <= 8) k_sketch_vec<8><<<g, 256, sm, st>>>(n, x, xscale, d, zeta, seed, out_raw, flag);
  else k_sketch_vec<16><<<g, 256, sm, st>>>(n, x, xscale, d, zeta, seed, out_raw, flag);
}

void launch_spmv_sketch(const Csr& A, const double* x, const double* xscale, double* w, int d, int zeta,
                        uint64_t seed, double* out_raw, int* flag, cudaStream_t st) {
  int g = grid_for(A.n, 256, kSketchCtas);
  size_t sm = (size_t)d * sizeof(double);
  if (zeta <= 4)
    k_spmv_sketch<4><<<g, 256, sm, st>>>(A.n, A.rowptr, A.colind, A.vals, x, xscale, w, d, zeta, seed, out_raw, flag);
  else if (zeta <= 8)
    k_spmv_sketch<8><<<g, 256, sm, st>>>(A.n, A.rowptr, A.colind, A.vals, x, xscale, w, d, zeta, seed, out_raw, flag);
  else
    k_spmv_sketch<16><<<g, 256, sm, st>>>(A.n, A.rowptr, A.colind, A.vals, x, xscale, w, d, zeta, seed, out_raw, flag);
}

void launch_ls(int c, int d, const double* S, const double* z_raw, double zscale, const double* colscale,
               double* r1, double* z1, double* r, double* rs, cudaStream_t st) {
  int warps_per_cta = 4;
  int g1 = (c + warps_per_cta - 1) / warps_per_cta;
  k_ls_dot<<<g1, 32 * warps_per_cta, 0, st>>>(c, d, S, z_raw, zscale, r1);
  int g2 = (d + warps_per_cta - 1) / warps_per_cta;
  k_ls_resid<<<g2, 32 * warps_per_cta, 0, st>>>(c, d, S, z_raw, zscale, r1, z1);
  k_ls_dot2<<<g1, 32 * warps_per_cta, 0, st>>>(c, d, S, z1, r1, colscale, r, rs);
}

void launch_update_sketch(int64_t n, double* U, int64_t ldu, int c, const double* rs, int d, int zeta,
                          uint64_t seed, double* out_raw, int* flag, cudaStream_t st) {
  int g = grid_for(n, 256, kSketchCtas);
  size_t sm = (size_t)(d + c) * sizeof(double);
  if (zeta <= 4) k_update_sketch<4><<<g, 256, sm, st>>>(n, U, ldu, c, rs, d, zeta, seed, out_raw, flag);
  else if (zeta <= 8) k_update_sketch<8><<<g, 256, sm, st>>>(n, U, ldu, c, rs, d, zeta, seed, out_raw, flag);
  else k_update_sketch<16><<<g, 256, sm, st>>>(n, U, ldu, c, rs, d, zeta, seed, out_raw, flag);
}

void launch_finish(int c, int d, double zscale, double* s_raw, double* z_raw, double* S, double* colscale,
                   const double* r, double* coef, int ldcoef, int* flag, cudaStream_t st) {
  k_finish<<<1, 512, 0, st>>>(c, d, zscale, s_raw, z_raw, S, colscale, r, coef, ldcoef, flag);
}

void launch_start_finish(int d, double zscale, double* s_raw, double* S, double* colscale, int* flag,
                         cudaStream_t st) {
  k_start_finish<<<1, 512, 0, st>>>(d, zscale, s_raw, S, colscale, flag);
}

void launch_start_vector(int64_t n, uint64_t seed, double* x, cudaStream_t st) {
  k_start_vector<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, seed, x);
}

// Opt every kernel with dynamic shared memory into the large carve-out
// (sketch bins of up to d = 8192 doubles, restart product tiles).
cudaError_t once_per_device(int slot, cudaError_t (*f)()) {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static bool done[kCfgSlots][kMaxDev] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (slot < 0 || slot >= kCfgSlots || dev < 0 || dev >= kMaxDev) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lock(mu);
  if (done[slot][dev]) return cudaSuccess;
  e = f();
  if (e == cudaSuccess) done[slot][dev] = true;
  return e;
}

static cudaError_t configure_kernels_once() {
  const int big = 200 * 1024;
  cudaError_t e = cudaSuccess;
#define RKS_SMEM(f) if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, big)
  RKS_SMEM(k_sketch_vec<4>); RKS_SMEM(k_sketch_vec<8>); RKS_SMEM(k_sketch_vec<16>);
  RKS_SMEM(k_spmv_sketch<4>); RKS_SMEM(k_spmv_sketch<8>); RKS_SMEM(k_spmv_sketch<16>);
  RKS_SMEM(k_update_sketch<4>); RKS_SMEM(k_update_sketch<8>); RKS_SMEM(k_update_sketch<16>);
  RKS_SMEM(k_rows_gemm);
#undef RKS_SMEM
  return e;
}

cudaError_t configure_kernels() { return once_per_device(kCfgBase, configure_kernels_once); }

int rows_gemm_smem(int nin, int nout, int threads) {
  return (int)(((size_t)nin * nout + (size_t)threads * nout) * sizeof(double));
}

void launch_rows_gemm(int64_t n, const double* A, int64_t lda, int a0, int nin, const double* B, int nout,
                      double* C, int64_t ldc, int c0, int move_src, cudaStream_t st) {
  const int threads = 128;
  size_t sm = (size_t)rows_gemm_smem(nin, nout, threads);
  int g = (int)((n + threads - 1) / threads);
  k_rows_gemm<<<g, threads, sm, st>>>(n, A, lda, a0, nin, B, nout, C, ldc, c0, move_src);
}

void launch_spmm(const Csr& A, const double* X, int64_t ldx, double* Y, int64_t ldy, int ncols, cudaStream_t st) {
  dim3 grid((unsigned)((A.n + 255) / 256), (unsigned)ncols);
  k_spmm<<<grid, 256, 0, st>>>(A.n, A.rowptr, A.colind, A.vals, X, ldx, Y, ldy, ncols);
}

int launch_resid_sums(int64_t n, const double* X, const double* AX, int64_t ld, int npairs, const int* col,
                      const int* colim, const double* lre, const double* lim, double* out, cudaStream_t st) {
  const int g = grid_for(n, 256, kResidCtas);
  dim3 grid((unsigned)g, (unsigned)npairs);
  k_resid_sums<<<grid, 256, 0, st>>>(n, X, AX, ld, col, colim, lre, lim, out);
  return g;
}

void launch_f32_to_f64(int64_t n, const float* a, double* b, cudaStream_t st) {
  k_f32_to_f64<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, a, b);
}

void launch_check_csr(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colind, int* bad,
                      cudaStream_t st) {
  k_check_csr<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, nnz, rowptr, colind, bad);
}

}  // namespace rks
