// Randomized QR factorisations of a tall and skinny block K = Q R (Sec. 2 of
// the paper: the randomized orthogonalisation processes an rKS basis can be
// built with), on the double-float kernels of the solver:
//
//  * RKS_QR_RGS: randomized Gram-Schmidt, the process of Algorithm 2 without
//    the product with A.  The sketches z_j = Omega k_j of all columns first
//    (tile sketch kernel); per column r = S_j^T z_j with a second pass in the
//    sketch (host, FP64: S_j is d x j),
//    q~ = k_j - Q_j r fused with the partial sketches of q~ (the solver's
//    update kernel), beta = ||Omega q~||.  Columns stay unscaled on the
//    device (their scale 1/beta goes into the next coefficients and the
//    final conversion), as in the solver.
//  * RKS_QR_WHITEN: sketch and whiten (the whitening of Sec. 3.3 on a whole
//    block): Omega K = Q_s R by Householder QR on the host, Q = K R^{-1} by
//    one double-float product.
//  * RKS_QR_RCHOLQR: randomized Cholesky QR: Q_1 = K R_1^{-1} as above, the
//    Gram matrix Q_1^T Q_1 (double-float dot kernel), its Cholesky factor R_2,
//    Q = Q_1 R_2^{-1}, R = R_2 R_1: a Euclidean-orthonormal Q.
//  * RKS_QR_RHQR: randomized Householder QR: Householder QR of the sketched
//    block Theta K, Theta = [[I_s, 0], [0, Omega']] (rows 0..s-1 kept,
//    Omega' the embedding of dimension n - s on the others), on the host,
//    with every reflector applied to the double-float columns on the device
//    and Q accumulated from the reflectors: Theta Q orthonormal.
//
// Omega is the solver's sparse-sign embedding (SplitMix64 hash, zeta rows per
// column, values +-1/sqrt(zeta)), applied through the deterministic per-tile
// bin lists, so the results do not depend on scheduling.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/rks.h"
#include "dense.h"
#include "rks_impl.h"

namespace {

// Q[i, j] = (x.hi + x.lo)[i, j] * scale[j] in FP64
__global__ void k_df2d_scaled(int64_t n, const float2* __restrict__ x, int64_t ldx, const double* __restrict__ scale,
                              double* __restrict__ y, int64_t ldy) {
  const int j = blockIdx.y;
  const double sc = scale[j];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = x[i + (int64_t)j * ldx];
    y[i + (int64_t)j * ldy] = ((double)v.x + (double)v.y) * sc;
  }
}

float2 to_df(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

// Device state of one call, freed on every exit path.
struct QrWork {
  int64_t n = 0, ldu = 0;
  int s = 0, d = 0, zeta = 0;
  double zscale = 0.0;
  cudaStream_t st = nullptr;
  float2* U = nullptr;        // ldu x 2s double-float columns: [0, s) and [s, 2s)
  uint16_t* otab = nullptr;
  rks::SketchTiles tiles;
  bool have_tiles = false;
  double* part = nullptr;     // G x max(d, s) partial sums
  double* sums = nullptr;     // s x max(d, s) folded sums (a column per sketch or dot group)
  float2* Q2 = nullptr;       // s x s double-float factor
  float2* nrs = nullptr;      // s update coefficients
  float2* sj = nullptr;       // scale of the updated column
  double* scale = nullptr;    // s column scales for the output
  int* flag = nullptr;
  std::vector<double> host;   // s x max(d, s) sums read back
  ~QrWork() {
    cudaFree(U); cudaFree(otab); cudaFree(part); cudaFree(sums); cudaFree(Q2); cudaFree(nrs); cudaFree(sj);
    cudaFree(scale); cudaFree(flag);
    if (have_tiles) rks::free_sketch_tiles(&tiles);
  }
};

#define QK(x)                                   \
  do {                                          \
    if ((x) != cudaSuccess) return RKS_ECUDA;   \
  } while (0)

// nsk: rows the sketch covers (n, or n - s for RHQR's Omega' on rows s..n-1)
int setup(QrWork& w, int64_t n, int s, int d, int zeta, uint64_t seed, cudaStream_t st, int64_t nsk) {
  w.n = n; w.s = s; w.d = d; w.zeta = zeta; w.st = st;
  w.zscale = 1.0 / std::sqrt((double)zeta);
  w.ldu = (n + 31) / 32 * 32;
  const int wide = std::max(d, s);
  if (cudaMalloc(&w.U, (size_t)w.ldu * 2 * s * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&w.otab, (size_t)nsk * rks::omega_slots(zeta) * sizeof(uint16_t)) != cudaSuccess ||
      cudaMalloc(&w.sums, (size_t)wide * s * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&w.Q2, (size_t)s * s * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&w.nrs, (size_t)2 * s * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&w.sj, sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&w.scale, (size_t)s * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&w.flag, sizeof(int)) != cudaSuccess)
    return RKS_ENOMEM;
  w.host.assign((size_t)wide * s, 0.0);
  QK(cudaMemsetAsync(w.flag, 0, sizeof(int), st));
  rks::launch_omega_table(nsk, d, zeta, seed, w.otab, w.flag, st);
  int bad = 0;
  QK(cudaMemcpyAsync(&bad, w.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  QK(cudaStreamSynchronize(st));
  if (bad) return RKS_EINVAL;
  if (rks::configure_df_kernels() != cudaSuccess) return RKS_ECUDA;
  if (rks::build_sketch_tiles(nsk, d, zeta, w.otab, &w.tiles, st) != 0) return RKS_ECUDA;
  w.have_tiles = true;
  cudaFree(w.otab);
  w.otab = nullptr;
  if (rks::sketch_tile_smem(w.tiles, s) > 200 * 1024) return RKS_EINVAL;
  if (cudaMalloc(&w.part, (size_t)w.tiles.G * wide * sizeof(double)) != cudaSuccess) return RKS_ENOMEM;
  return RKS_OK;
}

float2* col(QrWork& w, int j) { return w.U + (size_t)j * w.ldu; }

// host <- the folded sums of the last kernel's per-CTA partials (rows < cnt)
int fold_to_host(QrWork& w, int cnt) {
  rks::launch_df_fold(w.part, cnt, w.tiles.G, w.sums, w.st);
  QK(cudaGetLastError());
  QK(cudaMemcpyAsync(w.host.data(), w.sums, (size_t)cnt * sizeof(double), cudaMemcpyDeviceToHost, w.st));
  QK(cudaStreamSynchronize(w.st));
  return RKS_OK;
}

// U[:, c0 + o] = sum_l U[:, a0 + l] F[l, o] for o < s (F s x s, host FP64),
// out of place, in blocks of at most 64 outputs
int product(QrWork& w, int a0, const std::vector<double>& F, int c0) {
  const int s = w.s;
  std::vector<float2> F2((size_t)s * s);
  for (size_t t = 0; t < F2.size(); ++t) F2[t] = to_df(F[t]);
  QK(cudaMemcpyAsync(w.Q2, F2.data(), F2.size() * sizeof(float2), cudaMemcpyHostToDevice, w.st));
  for (int o0 = 0; o0 < s; o0 += 64) {
    const int nb = std::min(64, s - o0);
    rks::launch_df_rows_gemm(w.n, w.U, w.ldu, a0, s, w.Q2 + (size_t)o0 * s, nb, c0 + o0, -1, false, w.st);
  }
  QK(cudaGetLastError());
  QK(cudaStreamSynchronize(w.st));   // F2 is a host temporary
  return RKS_OK;
}

// inverse of an upper-triangular s x s R (back substitution)
std::vector<double> upper_inverse(int s, const std::vector<double>& R) {
  std::vector<double> X((size_t)s * s, 0.0);
  for (int j = 0; j < s; ++j) {
    X[j + (size_t)j * s] = 1.0 / R[j + (size_t)j * s];
    for (int i = j - 1; i >= 0; --i) {
      double acc = 0.0;
      for (int l = i + 1; l <= j; ++l) acc += R[i + (size_t)l * s] * X[l + (size_t)j * s];
      X[i + (size_t)j * s] = -acc / R[i + (size_t)i * s];
    }
  }
  return X;
}

// Sk (d x s) = Omega U[:, c0 .. c0+s): the sketches of s columns, folded on
// the device one after the other (stream order protects the partials), read
// back at once
int sketch_block(QrWork& w, int c0, std::vector<double>& Sk) {
  const int s = w.s, d = w.d;
  for (int j = 0; j < s; ++j) {
    rks::launch_df_sketch_vec(col(w, c0 + j), w.tiles, w.part, false, w.st);
    rks::launch_df_fold(w.part, d, w.tiles.G, w.sums + (size_t)j * d, w.st);
  }
  QK(cudaGetLastError());
  QK(cudaMemcpyAsync(w.host.data(), w.sums, (size_t)d * s * sizeof(double), cudaMemcpyDeviceToHost, w.st));
  QK(cudaStreamSynchronize(w.st));
  Sk.assign((size_t)d * s, 0.0);
  for (size_t t = 0; t < Sk.size(); ++t) Sk[t] = w.host[t] * w.zscale;
  return RKS_OK;
}

// Omega K = Q_s R1 (host); U[:, s..2s) = K R1^{-1}.  Sk receives Q_s.
int whiten(QrWork& w, std::vector<double>& R1, std::vector<double>& Sk) {
  const int s = w.s, d = w.d;
  int rc = sketch_block(w, 0, Sk);
  if (rc) return rc;
  R1.assign((size_t)s * s, 0.0);
  rks_dense::house_qr(d, s, Sk.data(), R1.data());
  for (int j = 0; j < s; ++j)
    if (!(R1[j + (size_t)j * s] > 0.0) || !std::isfinite(R1[j + (size_t)j * s])) return RKS_EBREAKDOWN;
  return product(w, 0, upper_inverse(s, R1), s);
}

int rgs(QrWork& w, std::vector<double>& R, std::vector<double>& S) {
  const int s = w.s, d = w.d;
  R.assign((size_t)s * s, 0.0);
  S.assign((size_t)d * s, 0.0);
  std::vector<double> Z, zr(d), r(s), cs(s, 0.0);
  std::vector<float2> nrs(s);
  const float2 one = make_float2(1.f, 0.f);
  QK(cudaMemcpyAsync(w.sj, &one, sizeof(float2), cudaMemcpyHostToDevice, w.st));
  // z_j = Omega k_j does not depend on the process: all of them at once
  int rc = sketch_block(w, 0, Z);
  if (rc) return rc;
  for (int j = 0; j < s; ++j) {
    if (j > 0) {
      // r = S_j^+ z: S_j is sketch-orthonormal; its projection twice
      // (r1 = S^T z, r = r1 + S^T (z - S r1))
      const double* z = &Z[(size_t)j * d];
      std::copy(z, z + d, zr.begin());
      for (int c = 0; c < j; ++c) {
        const double* sc = &S[(size_t)c * d];
        double a = 0.0;
        for (int i = 0; i < d; ++i) a += sc[i] * z[i];
        r[c] = a;
      }
      for (int c = 0; c < j; ++c)
        for (int i = 0; i < d; ++i) zr[i] -= S[i + (size_t)c * d] * r[c];
      for (int c = 0; c < j; ++c) {
        const double* sc = &S[(size_t)c * d];
        double a = 0.0;
        for (int i = 0; i < d; ++i) a += sc[i] * zr[i];
        r[c] += a;
      }
    }
    // q~ = k_j - sum_c (q~_c / beta_c) r_c, fused with its partial sketches
    for (int c = 0; c < j; ++c) nrs[c] = to_df(-r[c] * cs[c]);
    if (j > 0) QK(cudaMemcpyAsync(w.nrs, nrs.data(), (size_t)j * sizeof(float2), cudaMemcpyHostToDevice, w.st));
    rks::launch_df_update_sketch(w.U, w.ldu, j, w.nrs, w.sj, w.tiles, w.part, false, w.st);
    rc = fold_to_host(w, d);
    if (rc) return rc;
    double bb = 0.0;
    for (int i = 0; i < d; ++i) { const double v = w.host[i] * w.zscale; bb += v * v; }
    const double beta = std::sqrt(bb);
    if (!(beta > 0.0) || !std::isfinite(beta)) return RKS_EBREAKDOWN;
    for (int i = 0; i < d; ++i) S[i + (size_t)j * d] = w.host[i] * w.zscale / beta;
    for (int c = 0; c < j; ++c) R[c + (size_t)j * s] = r[c];
    R[j + (size_t)j * s] = beta;
    cs[j] = 1.0 / beta;
  }
  QK(cudaMemcpyAsync(w.scale, cs.data(), (size_t)s * sizeof(double), cudaMemcpyHostToDevice, w.st));
  return RKS_OK;
}

// Randomized Householder QR: Householder QR of Theta K ((s + d) x s, Theta =
// [[I_s, 0], [0, Omega']], Omega' on rows s..n-1) on the host in FP64, its
// reflectors H_j = I - beta_j u_j (Theta u_j)^T Theta applied to the
// double-float columns on the device (u_j is column j after the earlier
// reflectors with its entries above j dropped and rho_j taken off entry j,
// so Theta u_j = v_j), then Q = H_0 ... H_{s-1} [I_s; 0] accumulated
// backwards into columns s..2s-1.  The coefficient of every column update is
// a sketched inner product: the sketches of the later columns are updated on
// the host (Theta H_j = (I - beta v v^T) Theta), each pivot column is
// re-read and re-sketched from the device before its reflector is formed.
int rhqr(QrWork& w, std::vector<double>& R, std::vector<double>& scale) {
  const int s = w.s, d = w.d, ns = s + d;
  const int64_t nb = w.n - s;
  std::vector<double> Y((size_t)ns * s, 0.0), V((size_t)ns * s, 0.0), beta(s, 0.0);
  std::vector<float2> top((size_t)s * s), cf(s), colv(s);
  // top blocks (rows 0..s-1) and sketches of the bottom rows of every column
  QK(cudaMemcpy2DAsync(top.data(), s * sizeof(float2), w.U, w.ldu * sizeof(float2), s * sizeof(float2), s,
                       cudaMemcpyDeviceToHost, w.st));
  for (int l = 0; l < s; ++l) {
    rks::launch_df_sketch_vec(col(w, l) + s, w.tiles, w.part, false, w.st);
    rks::launch_df_fold(w.part, d, w.tiles.G, w.sums + (size_t)l * d, w.st);
  }
  QK(cudaGetLastError());
  QK(cudaMemcpyAsync(w.host.data(), w.sums, (size_t)d * s * sizeof(double), cudaMemcpyDeviceToHost, w.st));
  QK(cudaStreamSynchronize(w.st));
  for (int l = 0; l < s; ++l) {
    for (int i = 0; i < s; ++i) {
      const float2 t = top[i + (size_t)l * s];
      Y[i + (size_t)l * ns] = (double)t.x + (double)t.y;
    }
    for (int i = 0; i < d; ++i) Y[s + i + (size_t)l * ns] = w.host[i + (size_t)l * d] * w.zscale;
  }
  R.assign((size_t)s * s, 0.0);
  for (int j = 0; j < s; ++j) {
    double* y = &Y[(size_t)j * ns];
    double* v = &V[(size_t)j * ns];
    if (j > 0) {
      // the pivot column as the device holds it (its top rows and the sketch
      // of the others), so that the reflector is consistent with the vector
      // it is built from: Theta u_j = v_j to rounding
      QK(cudaMemcpyAsync(colv.data(), col(w, j), (size_t)s * sizeof(float2), cudaMemcpyDeviceToHost, w.st));
      rks::launch_df_sketch_vec(col(w, j) + s, w.tiles, w.part, false, w.st);
      rks::launch_df_fold(w.part, d, w.tiles.G, w.sums, w.st);
      QK(cudaGetLastError());
      QK(cudaMemcpyAsync(w.host.data(), w.sums, (size_t)d * sizeof(double), cudaMemcpyDeviceToHost, w.st));
      QK(cudaStreamSynchronize(w.st));
      for (int i = 0; i < s; ++i) y[i] = (double)colv[i].x + (double)colv[i].y;
      for (int i = 0; i < d; ++i) y[s + i] = w.host[i] * w.zscale;
    }
    double nn = 0.0;
    for (int i = j; i < ns; ++i) nn += y[i] * y[i];
    const double nrm = std::sqrt(nn);
    if (!(nrm > 0.0) || !std::isfinite(nrm)) return RKS_EBREAKDOWN;
    const double rho = y[j] >= 0.0 ? -nrm : nrm;     // -sign(y_j) ||y(j:)||
    for (int i = 0; i < j; ++i) R[i + (size_t)j * s] = y[i];
    R[j + (size_t)j * s] = rho;
    for (int i = j; i < ns; ++i) v[i] = y[i];
    v[j] -= rho;
    double vv = 0.0;
    for (int i = j; i < ns; ++i) vv += v[i] * v[i];
    beta[j] = 2.0 / vv;
    // column j becomes u_j: its top rows are v's (zeros above j)
    for (int i = 0; i < s; ++i) colv[i] = to_df(v[i]);
    QK(cudaMemcpyAsync(col(w, j), colv.data(), (size_t)s * sizeof(float2), cudaMemcpyHostToDevice, w.st));
    // H_j on the later columns: y_l -= c_l u_j, c_l = beta v^T Theta y_l
    const int nl = s - 1 - j;
    for (int l = j + 1; l < s; ++l) {
      double* yl = &Y[(size_t)l * ns];
      double a = 0.0;
      for (int i = j; i < ns; ++i) a += v[i] * yl[i];
      const double c = beta[j] * a;
      for (int i = j; i < ns; ++i) yl[i] -= c * v[i];
      cf[l - j - 1] = to_df(c);
    }
    if (nl > 0) {
      QK(cudaMemcpyAsync(w.nrs, cf.data(), (size_t)nl * sizeof(float2), cudaMemcpyHostToDevice, w.st));
      rks::launch_df_axpy_cols(w.n, w.U, w.ldu, j, j + 1, nl, w.nrs, w.st);
    }
  }
  // Q = H_0 ... H_{s-1} [I_s; 0] in columns s..2s-1, Theta Q tracked on the host
  QK(cudaMemsetAsync(col(w, s), 0, (size_t)w.ldu * s * sizeof(float2), w.st));
  std::vector<float2> eye((size_t)s * s, make_float2(0.f, 0.f));
  for (int l = 0; l < s; ++l) eye[l + (size_t)l * s] = make_float2(1.f, 0.f);
  QK(cudaMemcpy2DAsync(col(w, s), w.ldu * sizeof(float2), eye.data(), s * sizeof(float2), s * sizeof(float2), s,
                       cudaMemcpyHostToDevice, w.st));
  std::vector<double> Z((size_t)ns * s, 0.0);
  for (int l = 0; l < s; ++l) Z[l + (size_t)l * ns] = 1.0;
  for (int j = s - 1; j >= 0; --j) {
    const double* v = &V[(size_t)j * ns];
    for (int l = j; l < s; ++l) {
      double* zl = &Z[(size_t)l * ns];
      double a = 0.0;
      for (int i = j; i < ns; ++i) a += v[i] * zl[i];
      const double c = beta[j] * a;
      for (int i = j; i < ns; ++i) zl[i] -= c * v[i];
      cf[l - j] = to_df(c);
    }
    QK(cudaMemcpyAsync(w.nrs + s, cf.data(), (size_t)(s - j) * sizeof(float2), cudaMemcpyHostToDevice, w.st));
    rks::launch_df_axpy_cols(w.n, w.U, w.ldu, j, s + j, s - j, w.nrs + s, w.st);
  }
  QK(cudaGetLastError());
  // positive diagonal: flip Q's column j and R's row j where rho_j < 0
  scale.assign(s, 1.0);
  for (int j = 0; j < s; ++j)
    if (R[j + (size_t)j * s] < 0.0) {
      scale[j] = -1.0;
      for (int c = j; c < s; ++c) R[j + (size_t)c * s] = -R[j + (size_t)c * s];
    }
  (void)nb;
  QK(cudaStreamSynchronize(w.st));
  return RKS_OK;
}

}  // namespace

extern "C" int rks_sketch_qr(int64_t n, int s, const double* K, int64_t ldk, int d, int zeta, uint64_t seed,
                             int method, double* Q, int64_t ldq, double* R, double* S, void* stream) {
  if (n < 2 || s < 1 || s > RKS_SKETCH_QR_MAX_S || zeta < 1 || zeta > 16 || d < 2 * zeta || d > 8192 || s > d ||
      s > n || !K || !Q || !R || ldk < n || ldq < n)
    return RKS_EINVAL;
  if (method != RKS_QR_RGS && method != RKS_QR_WHITEN && method != RKS_QR_RCHOLQR && method != RKS_QR_RHQR)
    return RKS_EINVAL;
  if (method == RKS_QR_RHQR && n - s < 2) return RKS_EINVAL;
  if (Q == K && ldq != ldk) return RKS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  QrWork w;
  int rc = setup(w, n, s, d, zeta, seed, st, method == RKS_QR_RHQR ? n - s : n);
  if (rc) return rc;
  for (int j = 0; j < s; ++j) rks::launch_d2df(n, K + (size_t)j * ldk, col(w, j), false, st);
  QK(cudaGetLastError());
  std::vector<double> Rh, Sh;
  int out0 = 0;                 // first column of the result in U
  std::vector<double> ones(s, 1.0);
  if (method == RKS_QR_RGS) {
    rc = rgs(w, Rh, Sh);
    if (rc) return rc;
  } else if (method == RKS_QR_RHQR) {
    std::vector<double> sc;
    rc = rhqr(w, Rh, sc);
    if (rc) return rc;
    out0 = s;
    QK(cudaMemcpyAsync(w.scale, sc.data(), (size_t)s * sizeof(double), cudaMemcpyHostToDevice, st));
    if (S) {                    // Omega' Q[s:, :], measured: the sketched rows of Theta Q
      Sh.assign((size_t)d * s, 0.0);
      for (int j = 0; j < s; ++j) {
        rks::launch_df_sketch_vec(col(w, s + j) + s, w.tiles, w.part, false, st);
        rks::launch_df_fold(w.part, d, w.tiles.G, w.sums + (size_t)j * d, st);
      }
      QK(cudaGetLastError());
      QK(cudaMemcpyAsync(w.host.data(), w.sums, (size_t)d * s * sizeof(double), cudaMemcpyDeviceToHost, st));
      QK(cudaStreamSynchronize(st));
      for (int j = 0; j < s; ++j)
        for (int i = 0; i < d; ++i) Sh[i + (size_t)j * d] = w.host[i + (size_t)j * d] * w.zscale * sc[j];
    }
  } else {
    std::vector<double> R1;
    rc = whiten(w, R1, Sh);
    if (rc) return rc;
    out0 = s;
    Rh = R1;
    if (method == RKS_QR_RCHOLQR) {
      // G = Q1^T Q1 (columns s .. 2s-1), upper triangle by columns
      std::vector<double> G((size_t)s * s, 0.0);
      for (int cv = 0; cv < s; ++cv) {
        rks::launch_df_dots(col(w, s), w.ldu, cv + 1, cv, w.tiles, w.part, st);
        rks::launch_df_fold(w.part, cv + 1, w.tiles.G, w.sums + (size_t)cv * s, st);
      }
      QK(cudaGetLastError());
      QK(cudaMemcpyAsync(w.host.data(), w.sums, (size_t)s * s * sizeof(double), cudaMemcpyDeviceToHost, st));
      QK(cudaStreamSynchronize(st));
      for (int cv = 0; cv < s; ++cv)
        for (int l = 0; l <= cv; ++l) G[l + (size_t)cv * s] = G[cv + (size_t)l * s] = w.host[l + (size_t)cv * s];
      // Cholesky G = R2^T R2 (R2 upper)
      std::vector<double> R2((size_t)s * s, 0.0);
      for (int j = 0; j < s; ++j) {
        double dd = G[j + (size_t)j * s];
        for (int l = 0; l < j; ++l) dd -= R2[l + (size_t)j * s] * R2[l + (size_t)j * s];
        if (!(dd > 0.0) || !std::isfinite(dd)) return RKS_EDENSE;
        const double rjj = std::sqrt(dd);
        R2[j + (size_t)j * s] = rjj;
        for (int c = j + 1; c < s; ++c) {
          double a = G[j + (size_t)c * s];
          for (int l = 0; l < j; ++l) a -= R2[l + (size_t)j * s] * R2[l + (size_t)c * s];
          R2[j + (size_t)c * s] = a / rjj;
        }
      }
      rc = product(w, s, upper_inverse(s, R2), 0);   // Q = Q1 R2^{-1} into columns 0 .. s-1
      if (rc) return rc;
      out0 = 0;
      for (int j = 0; j < s; ++j)                   // R = R2 R1
        for (int i = 0; i <= j; ++i) {
          double a = 0.0;
          for (int l = i; l <= j; ++l) a += R2[i + (size_t)l * s] * R1[l + (size_t)j * s];
          Rh[i + (size_t)j * s] = a;
        }
    }
    QK(cudaMemcpyAsync(w.scale, ones.data(), (size_t)s * sizeof(double), cudaMemcpyHostToDevice, st));
    if (S) {                    // the sketch of the computed Q, measured
      rc = sketch_block(w, out0, Sh);
      if (rc) return rc;
    }
  }
  dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 1024), (unsigned)s);
  k_df2d_scaled<<<grid, 256, 0, st>>>(n, col(w, out0), w.ldu, w.scale, Q, ldq);
  QK(cudaGetLastError());
  QK(cudaStreamSynchronize(st));
  std::copy(Rh.begin(), Rh.end(), R);
  if (S) std::copy(Sh.begin(), Sh.end(), S);
  return RKS_OK;
}
