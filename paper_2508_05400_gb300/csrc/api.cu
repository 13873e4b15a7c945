// C ABI of librks: context management and the rKS driver (Algorithm 1).
//
// Device: all n-dimensional work (SpMV, sketches, the RGS update, the restart
// product U Q, eigenvectors and residuals) runs in the kernels of kernels.cu
// on the context's stream.  Host: the m x m FP64 contraction (Schur form,
// reordering, truncation, whitening, locking, Ritz pairs and estimates) runs
// in dense.cpp between expansions, on the Rayleigh quotient copied back from
// the device.
//
// Column layout of the basis U (n x (m+1), column-major, ld = n rounded up
// to 32): columns 0..q-1 are the locked Schur vectors U_q (Sec. 4.3), columns
// q..q+ja-1 the active basis, column q+ja the last vector u.  S = Omega U is
// kept both on the device (d x (m+1)) and on the host.

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/rks.h"
#include "dense.h"
#include "rks_impl.h"

using rks::Csr;
typedef std::complex<double> cd;

struct rks_ctx {
  // problem
  int64_t n = 0, nnz = 0;
  int k = 0, p = 0, m = 0, d = 0, zeta = 8, which = 0;
  double tol = 0, eta_lock = 0, zscale = 1;
  uint64_t seed = 0;
  rks_opts opts;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // device
  int32_t* rowptr = nullptr;
  int32_t* colind = nullptr;
  double* vals = nullptr;
  Csr A;
  double* U = nullptr;
  int64_t ldu = 0;
  double* S = nullptr;
  double* colscale = nullptr;
  double *z_raw = nullptr, *s_raw = nullptr, *z1 = nullptr, *r1 = nullptr, *r = nullptr, *rs = nullptr;
  double* coef = nullptr;
  int* flag = nullptr;
  double* Qd = nullptr;
  double* u1 = nullptr;
  double* X = nullptr;
  double* AX = nullptr;
  double* rsum = nullptr;
  int* pcol = nullptr;
  double* plam = nullptr;
  // double-float path (opts.prec == RKS_PREC_DF)
  int prec = RKS_PREC_DF;
  rks::CsrDF A2;        // the value array and basis in use (DF pairs or FP32)
  float2* vals2 = nullptr;
  float2* U2 = nullptr;
  float* valsf = nullptr;  // mixed precision: FP32 values and basis
  int ell_w = 0;           // ELLPACK copy of A for the SpMV (0: not used)
  bool spmv_merge = false, spmv_warp = false;   // CSR SpMV variants chosen by row lengths
  bool vals_f32 = false;   // every value of A is an FP32 number (the double-float copies' low words are 0)
  int dia_d = 0;           // diagonal copy of A for the SpMV (0: not used), its offsets
  int dia_off[16] = {};
  float2* dia_val2 = nullptr;
  float* dia_valf = nullptr;
  int32_t* ell_col = nullptr;
  float2* ell_val2 = nullptr;
  float* ell_valf = nullptr;
  float* Uf = nullptr;
  void* qimg = nullptr;     // mixed precision: bf16 split image of Q' for the tensor-core restart
  std::vector<uint16_t> qimg_h;
  void* qimg_df = nullptr;  // double-float basis: digit image of Q', column exponents, row exponents
  int* fexp_d = nullptr;
  int* pexp_d = nullptr;     // power-of-two part of the input columns' scales
  int* rexp_d = nullptr;     // per-row exponents (n)
  std::vector<int> fexp_h, pexp_h;
  std::vector<double> Qr_h;
  // rotation of the kept columns still to be applied on the device after the
  // restart's host work (whitening, aggressive reorder): columns corr_q ..
  // corr_q + corr_ka - 1 times corr (corr_ka x corr_ka); empty: none
  std::vector<double> corr;
  int corr_q = 0, corr_ka = 0;
  bool up_M2 = false;      // the Gram matrix changed at the restart: upload it
  void* Ub = nullptr;      // basis in use: U2 or Uf
  bool f32 = false;        // basis in use is FP32
  int phase_restarts = 0;
  float2* S2 = nullptr;
  float2* nrs = nullptr;
  float2* sj = nullptr;
  float2* Q2 = nullptr;
  double* rprev = nullptr;
  double* znorm = nullptr;
  uint16_t* otab = nullptr;  // packed Omega (rows + signs) from the hash; freed once the tiles are built
  rks::SketchTiles tiles;    // per-tile bin lists of Omega (deterministic sketch accumulation)
  double* part_z = nullptr;  // G x d per-CTA partial sketches of A u (z') and of u~ (s~)
  double* part_s = nullptr;
  double* part_d = nullptr;  // Euclidean CGS2 baseline: G x (m+1) partial dot products
  unsigned* bar = nullptr;   // grid-barrier state of the cooperative least squares
  float2* lsr1 = nullptr;    // least-squares scratch: first-pass coefficients (m+1)
  float2* M2 = nullptr;      // Gram matrix S^T S of the sketched basis (DF, (m+1) x (m+1))
  std::vector<float2> M2_h;
  double* tmp64 = nullptr;
  // host state
  double norm1 = 0;
  std::vector<double> S_h, cs_h, coef_h, Ba, Tqq, Tqa;
  std::vector<float2> S2_h;
  int q = 0, ja = 0;
  int brow = 0;            // row of b in the active Rayleigh quotient (active columns kept at the last restart)
  int64_t nmatvec = 0;
  int restarts = 0;
  int last_expand_from = 0;
  // instrumentation (rks_get_stats)
  rks_stats stats;
  std::vector<cudaEvent_t> evpool;   // pairs: [2i] start, [2i+1] stop
  std::vector<int> evclass;
  int evused = 0;
  // results
  bool solved = false;
  int kk = 0;               // columns of the kept decomposition (locked + active)
  int nw = 0;               // reported Ritz pairs: the best k (k + 1 for a pair at the cut)
  std::vector<double> Tfull, bfull, lre, lim, est, resid;
  std::vector<double> rq_re, rq_im;   // Rayleigh quotients x^H A x / x^H x of the Ritz vectors
  std::vector<double> hist;
  std::vector<int> hist_lock;
  std::vector<cd> Y;
};

namespace {

#define CK(x)                                                              \
  do {                                                                     \
    cudaError_t e_ = (x);                                                  \
    if (e_ != cudaSuccess) {                                               \
      std::fprintf(stderr, "librks: %s failed: %s\n", #x, cudaGetErrorString(e_)); \
      return e_ == cudaErrorMemoryAllocation ? RKS_ENOMEM : RKS_ECUDA;    \
    }                                                                      \
  } while (0)

template <class T>
int dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) { *p = nullptr; return e == cudaErrorMemoryAllocation ? RKS_ENOMEM : RKS_ECUDA; }
  return RKS_OK;
}

int launch_err() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::fprintf(stderr, "librks: kernel launch failed: %s\n", cudaGetErrorString(e));
    return RKS_ECUDA;
  }
  return RKS_OK;
}

inline double& M(std::vector<double>& a, int ld, int i, int j) { return a[i + (size_t)j * ld]; }

// Launch accounting: every kernel launch is counted; with opts.profile the
// launches of a class are bracketed by CUDA events on the context's stream.
int prof_begin(rks_ctx* c, int cls) {
  if (!c->opts.profile) return -1;
  if (c->opts.profile > 1 && !((c->opts.profile >> (cls + 1)) & 1)) return -1;   // class not timed
  if ((size_t)(2 * c->evused + 2) > c->evpool.size()) {
    for (int t = 0; t < 64; ++t) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      c->evpool.push_back(e);
    }
    c->evclass.resize(c->evpool.size() / 2);
  }
  int slot = c->evused++;
  c->evclass[slot] = cls + (c->f32 ? RKS_NK : 0);   // FP32-basis launches counted apart as well
  cudaEventRecord(c->evpool[2 * slot], c->stream);
  return slot;
}

void prof_end(rks_ctx* c, int slot, int cls, int nlaunch, double bytes, double flops) {
  c->stats.launches[cls] += nlaunch;
  c->stats.bytes[cls] += bytes;
  c->stats.flops[cls] += flops;
  if (c->f32) {
    c->stats.launches_f32[cls] += nlaunch;
    c->stats.bytes_f32[cls] += bytes;
  }
  if (slot >= 0) cudaEventRecord(c->evpool[2 * slot + 1], c->stream);
}

// Called after a stream synchronisation: fold the recorded event pairs.
void prof_flush(rks_ctx* c) {
  for (int s = 0; s < c->evused; ++s) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->evpool[2 * s], c->evpool[2 * s + 1]) == cudaSuccess) {
      const int cls = c->evclass[s] % RKS_NK;
      c->stats.ms[cls] += ms;
      if (c->evclass[s] >= RKS_NK) c->stats.ms_f32[cls] += ms;
    }
  }
  c->evused = 0;
}

// Append column j (global index) of the expansion to the host Rayleigh quotient.
void absorb_columns(rks_ctx* c, int from, int to) {
  const int ldc = c->m + 1;
  const int ldb = c->m + 1;
  const int ldt = c->k + 2;
  for (int j = from; j < to; ++j) {
    int a = j - c->q;
    for (int i = 0; i < c->q; ++i) M(c->Tqa, ldt, i, a) = c->coef_h[i + (size_t)j * ldc];
    for (int i = 0; i <= a; ++i) M(c->Ba, ldb, i, a) = c->coef_h[c->q + i + (size_t)j * ldc];
    M(c->Ba, ldb, a + 1, a) = c->coef_h[j + 1 + (size_t)j * ldc];
    for (int i = a + 2; i <= c->m; ++i) M(c->Ba, ldb, i, a) = 0.0;
  }
}

int read_flag(rks_ctx* c, int* f) {
  CK(cudaMemcpyAsync(f, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return RKS_OK;
}

int flag_status(int f) {
  if (f & rks::RKS_FLAG_TIMEOUT) return RKS_ETIMEOUT;
  if (f & rks::RKS_FLAG_NAN) return RKS_ENAN;
  if (f & rks::RKS_FLAG_HASH) return RKS_EINVAL;
  if (f & rks::RKS_FLAG_BREAKDOWN) return RKS_EBREAKDOWN;
  return RKS_OK;
}

// Algorithm 2 in double-float: three kernels per step (see kernels_df.cu).
void expand_df_launches(rks_ctx* c, int c0) {
  const double n = (double)c->n, P = 8.0, PV = c->f32 ? 4.0 : 8.0;
  // algorithmic bytes of the storage the SpMV reads: CSR/ELLPACK values and
  // columns (and row pointers), or the D diagonals (FP32 copies when A's
  // values are FP32 numbers); x read once, w written
  const double PA = (c->A2.dvals && c->A2.dvals_f32 && c->A2.D <= 8) ? 4.0 : PV;
  const double spmv_bytes = c->A2.dvals ? (double)c->A2.D * PA * n + 2 * PV * n
                                        : (double)c->nnz * (PV + 4) + 4.0 * (n + 1) + 2 * PV * n;
  for (int j = c0; j < c->m; ++j) {
    const int col = j + 1;
    int s = prof_begin(c, RKS_K_SPMV);
    const size_t es = c->f32 ? sizeof(float) : sizeof(float2);
    char* ub = static_cast<char*>(c->Ub);
    rks::launch_df_spmv_sketch(c->A2, ub + (size_t)j * c->ldu * es, ub + (size_t)col * c->ldu * es, c->tiles,
                               c->part_z, c->stream);
    prof_end(c, s, RKS_K_SPMV, 1, spmv_bytes, 2.0 * c->nnz);
    s = prof_begin(c, RKS_K_LS);
    const int nls = rks::launch_df_small(j, c->d, c->zscale, j > c0 ? 1 : 0, 1, c->s_raw, c->z_raw, c->S, c->S2,
                                         c->colscale, c->rprev, c->coef, c->m + 1, c->znorm, c->nrs, c->sj, c->lsr1,
                                         c->M2, c->m + 1, c->part_z, c->part_s, c->tiles.G, c->flag, c->bar, c->stream, c->opts.debug_stall);
    prof_end(c, s, RKS_K_LS, nls, 3.0 * P * c->d * col, 6.0 * c->d * col);
    s = prof_begin(c, RKS_K_UPDATE);
    rks::launch_df_update_sketch(c->Ub, c->ldu, col, c->nrs, c->sj, c->tiles, c->part_s, c->f32, c->stream);
    prof_end(c, s, RKS_K_UPDATE, 1, (col + 2) * (c->f32 ? 4.0 : P) * n, 2.0 * n * col);
    ++c->nmatvec;
  }
  int s = prof_begin(c, RKS_K_FINISH);
  const int nf = rks::launch_df_small(c->m, c->d, c->zscale, 1, 0, c->s_raw, c->z_raw, c->S, c->S2, c->colscale,
                                      c->rprev, c->coef, c->m + 1, c->znorm, c->nrs, c->sj, c->lsr1, c->M2, c->m + 1,
                                      c->part_z, c->part_s, c->tiles.G, c->flag, c->bar, c->stream, c->opts.debug_stall);
  prof_end(c, s, RKS_K_FINISH, nf, 3.0 * P * c->d, 2.0 * c->d);
}

// Krylov-Schur with Euclidean CGS2 (the paper's KS-CGS2 comparison method,
// Sec. 5), same storage and kernels without the sketch: per step the SpMV,
// two passes of (dot products with every basis column, update), and the norm.
void expand_ks_launches(rks_ctx* c, int c0) {
  const double n = (double)c->n, P = 8.0;
  const double PA = (c->A2.dvals && c->A2.dvals_f32 && c->A2.D <= 8) ? 4.0 : P;
  const double spmv_bytes = c->A2.dvals ? (double)c->A2.D * PA * n + 2 * P * n
                                        : (double)c->nnz * (P + 4) + 4.0 * (n + 1) + 2 * P * n;
  const int G = c->tiles.G;
  for (int j = c0; j < c->m; ++j) {
    const int col = j + 1;
    char* ub = static_cast<char*>(c->Ub);
    const size_t es = sizeof(float2);
    int s = prof_begin(c, RKS_K_SPMV);
    rks::launch_df_spmv(c->A2, ub + (size_t)j * c->ldu * es, ub + (size_t)col * c->ldu * es, c->tiles, c->stream);
    prof_end(c, s, RKS_K_SPMV, 1, spmv_bytes, 2.0 * c->nnz);
    for (int pass = 1; pass <= 2; ++pass) {
      s = prof_begin(c, RKS_K_LS);
      rks::launch_df_dots(c->Ub, c->ldu, col, col, c->tiles, c->part_d, c->stream);
      rks::launch_ks_coef(pass, j, col, G, c->part_d, c->colscale, c->rprev, c->nrs, c->sj, c->stream);
      prof_end(c, s, RKS_K_LS, 2, (col + 1) * P * n, 2.0 * n * col);
      s = prof_begin(c, RKS_K_UPDATE);
      rks::launch_df_update_plain(c->Ub, c->ldu, col, c->nrs, c->sj, c->tiles, pass == 2 ? c->part_s : nullptr,
                                  c->stream);
      prof_end(c, s, RKS_K_UPDATE, 1, (col + 2) * P * n, 2.0 * n * col);
    }
    s = prof_begin(c, RKS_K_FINISH);
    rks::launch_ks_finish(j, G, c->part_s, 1e-14 * c->norm1, c->colscale, c->rprev, c->coef, c->m + 1, c->flag,
                          c->stream);
    prof_end(c, s, RKS_K_FINISH, 1, 8.0 * G, 2.0 * G);
    ++c->nmatvec;
  }
}

// Algorithm 2: extend from the last vector at column q+ja to column m.
int expand(rks_ctx* c) {
  const int c0 = c->q + c->ja;
  c->brow = c->ja;
  if (c->opts.ortho == RKS_ORTHO_CGS2) {
    expand_ks_launches(c, c0);
  } else if (c->prec != RKS_PREC_FP64) {
    expand_df_launches(c, c0);
  } else
  {
  const double n = (double)c->n, P = sizeof(double);
  const double spmv_bytes = (double)c->nnz * (P + 4) + 4.0 * (n + 1) + 2 * P * n;
  for (int j = c0; j < c->m; ++j) {
    const int col = j + 1;
    int s = prof_begin(c, RKS_K_SPMV);
    rks::launch_spmv_sketch(c->A, c->U + (int64_t)j * c->ldu, c->colscale + j, c->U + (int64_t)col * c->ldu,
                            c->d, c->zeta, c->seed, c->z_raw, c->flag, c->stream);
    prof_end(c, s, RKS_K_SPMV, 1, spmv_bytes, 2.0 * c->nnz);
    s = prof_begin(c, RKS_K_LS);
    rks::launch_ls(col, c->d, c->S, c->z_raw, c->zscale, c->colscale, c->r1, c->z1, c->r, c->rs, c->stream);
    prof_end(c, s, RKS_K_LS, 3, 3.0 * P * c->d * col, 6.0 * c->d * col);
    s = prof_begin(c, RKS_K_UPDATE);
    rks::launch_update_sketch(c->n, c->U, c->ldu, col, c->rs, c->d, c->zeta, c->seed, c->s_raw, c->flag,
                              c->stream);
    prof_end(c, s, RKS_K_UPDATE, 1, (col + 2) * P * n, 2.0 * n * col);
    s = prof_begin(c, RKS_K_FINISH);
    rks::launch_finish(col, c->d, c->zscale, c->s_raw, c->z_raw, c->S, c->colscale, c->r, c->coef, c->m + 1,
                       c->flag, c->stream);
    prof_end(c, s, RKS_K_FINISH, 1, 3.0 * P * c->d, 2.0 * c->d);
    ++c->nmatvec;
  }
  }
  int rc = launch_err();
  if (rc) return rc;
  c->last_expand_from = c0;
  // bring back coefficients, scales and sketches
  CK(cudaMemcpyAsync(c->coef_h.data(), c->coef, c->coef_h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaMemcpyAsync(c->cs_h.data(), c->colscale, c->cs_h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaMemcpyAsync(c->S_h.data(), c->S, c->S_h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  int f = 0;
  rc = read_flag(c, &f);
  if (rc) return rc;
  prof_flush(c);
  if ((f & rks::RKS_FLAG_TIMEOUT) && c->bar) {
    // a grid barrier gave up: its arrival count no longer matches the grid,
    // so start the next cooperative launch from a clean state
    CK(cudaMemsetAsync(c->bar, 0, 2 * sizeof(unsigned), c->stream));
    CK(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  rc = flag_status(f);
  if (rc) return rc;
  absorb_columns(c, c0, c->m);
  c->ja = c->m - c->q;
  return RKS_OK;
}


// Algorithm 1 contraction + whitening (Sec. 3.3) + locking (Sec. 4.4) +
// restart product on the device.  Sets c->kk results of the Ritz step.
// Locking threshold of an active block with eigenvalue modulus lam (Sec. 4.4):
// eta_lock * |lambda| (floored at eps ||T_a||_F), or eta_lock * ||A||_1.
double lock_threshold(const rks_ctx* c, double lam, double tn) {
  const double scale = c->opts.conv == RKS_CONV_NORM1 ? c->norm1 : std::max(lam, 2.220446049250313e-16 * tn);
  return c->eta_lock * scale;
}

// Aggressive deflation (Sec. 4.3, after Thm 4.3): reorder the active Schur
// form T_a (ka x ka) so that the blocks whose Ritz estimate |b^T y| (unit y,
// eigenvector of T_a) is below the locking threshold lead, in their order,
// followed by the others in theirs.  The rotation Z goes onto b (Z^T b), the
// pending right factor Cm of the kept columns (ka x ka; empty = identity),
// the coupling T_qa (q x ka, leading dimension ldt) and the kept sketches
// S_a (d x ka).  Returns true when something moved; a refused swap leaves
// everything unchanged.
bool aggressive_reorder(const rks_ctx* c, int ka, std::vector<double>& Ta, std::vector<double>& bk,
                        std::vector<double>& Cm, int q, int ldt, std::vector<double>& Tqa, int d,
                        std::vector<double>& Sa) {
  if (ka < 2) return false;
  const auto bl = rks_dense::blocks(ka, Ta.data(), ka);
  std::vector<double> lre(ka), lim(ka);
  std::vector<std::complex<double>> Y((size_t)ka * ka);
  rks_dense::quasi_eig(ka, Ta.data(), ka, lre.data(), lim.data(), Y.data(), ka);
  double tn = 0.0;
  for (double v : Ta) tn += v * v;
  tn = std::sqrt(tn);
  std::vector<char> sel(bl.size(), 0);
  for (size_t t = 0; t < bl.size(); ++t) {
    std::complex<double> e = 0.0;   // column bl[t].start of Y: the block's eigenvector (Im >= 0)
    for (int i = 0; i < ka; ++i) e += bk[i] * Y[i + (size_t)bl[t].start * ka];
    sel[t] = std::abs(e) <= lock_threshold(c, std::hypot(bl[t].re, bl[t].im), tn);
  }
  size_t first_open = 0;
  while (first_open < bl.size() && sel[first_open]) ++first_open;
  bool behind = false;
  for (size_t t = first_open; t < bl.size(); ++t) behind = behind || sel[t];
  if (!behind) return false;
  std::vector<double> T2 = Ta, Z((size_t)ka * ka, 0.0);
  for (int i = 0; i < ka; ++i) Z[i + (size_t)i * ka] = 1.0;
  if (rks_dense::reorder_select(ka, T2.data(), ka, Z.data(), ka, ka, sel) != 0) return false;
  Ta = T2;
  auto right = [&](std::vector<double>& X, int rows, int ldx) {   // X (rows x ka) <- X Z
    std::vector<double> row(ka);
    for (int r = 0; r < rows; ++r) {
      for (int j = 0; j < ka; ++j) {
        double acc = 0.0;
        for (int l = 0; l < ka; ++l) acc += X[r + (size_t)l * ldx] * Z[l + (size_t)j * ka];
        row[j] = acc;
      }
      for (int j = 0; j < ka; ++j) X[r + (size_t)j * ldx] = row[j];
    }
  };
  if (Cm.empty()) {
    Cm.assign((size_t)ka * ka, 0.0);
    for (int i = 0; i < ka; ++i) Cm[i + (size_t)i * ka] = 1.0;
  }
  right(Cm, ka, ka);
  right(Tqa, q, ldt);
  right(Sa, d, d);
  std::vector<double> b2(ka, 0.0);
  for (int j = 0; j < ka; ++j)
    for (int l = 0; l < ka; ++l) b2[j] += bk[l] * Z[l + (size_t)j * ka];
  bk = b2;
  return true;
}

// U[:, a0 .. a0+nout-1] <- U[:, a0 .. a0+nin-1] diag(cs) Q in place (Eq. 3.5),
// Q nin x nout (host FP64, column-major), cs the column scales of the inputs
// (nullptr: ones); move_src >= 0 also copies column move_src to a0 + nout.
// Tensor cores where the sizes allow, else the SIMT kernels.  The host images
// are pageable, so each copy has taken its source when cudaMemcpyAsync
// returns and nothing here waits for the kernel.
int restart_launch(rks_ctx* c, int a0, int nin, const std::vector<double>& Q, const double* cs, int nout,
                   int move_src) {
  std::vector<double> Qp((size_t)nin * nout);
  for (int j = 0; j < nout; ++j)
    for (int l = 0; l < nin; ++l) Qp[l + (size_t)j * nin] = (cs ? cs[l] : 1.0) * Q[l + (size_t)j * nin];
  const int ps = prof_begin(c, RKS_K_RESTART);
  if (c->f32 && c->qimg && rks::tc_restart_supported(nin, nout)) {
    // FP32 basis: split-BF16 product on the tensor cores
    rks::tc_restart_bimage(nin, nout, Qp.data(), c->qimg_h);
    CK(cudaMemcpyAsync(c->qimg, c->qimg_h.data(), c->qimg_h.size() * sizeof(uint16_t), cudaMemcpyHostToDevice,
                       c->stream));
    float* U0 = c->Uf + (size_t)a0 * c->ldu;
    rks::launch_tc_restart_f32(c->n, U0, U0, c->ldu, nin, nout, c->qimg,
                               move_src >= 0 ? c->Uf + (size_t)move_src * c->ldu : nullptr,
                               move_src >= 0 ? c->Uf + (size_t)(a0 + nout) * c->ldu : nullptr, c->flag, c->stream);
  } else if (c->prec != RKS_PREC_FP64 && !c->f32 && c->qimg_df && rks::tc_restart_df_supported(nin, nout)) {
    // double-float basis: exact digit products on the tensor cores.  The power
    // of two of each column scale goes onto U (an exact exponent offset in the
    // digit split), the rest (in [1, 2)) stays in Q'.
    c->pexp_h.assign(nin, 0);
    c->Qr_h.assign(Qp.size(), 0.0);
    for (int l = 0; l < nin; ++l) {
      const double sc = cs ? cs[l] : 1.0;
      int E = 0;
      if (sc != 0.0) std::frexp(sc, &E);
      c->pexp_h[l] = sc != 0.0 ? E - 1 : 0;
      for (int j = 0; j < nout; ++j)
        c->Qr_h[l + (size_t)j * nin] = std::ldexp(Qp[l + (size_t)j * nin], -c->pexp_h[l]);
    }
    rks::tc_restart_df_bimage(nin, nout, c->Qr_h.data(), c->qimg_h, c->fexp_h);
    CK(cudaMemcpyAsync(c->pexp_d, c->pexp_h.data(), c->pexp_h.size() * sizeof(int), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(c->qimg_df, c->qimg_h.data(), c->qimg_h.size() * sizeof(uint16_t), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(c->fexp_d, c->fexp_h.data(), c->fexp_h.size() * sizeof(int), cudaMemcpyHostToDevice,
                       c->stream));
    float2* U0 = c->U2 + (size_t)a0 * c->ldu;
    rks::launch_tc_restart_df(c->n, U0, U0, c->ldu, nin, nout, c->qimg_df, c->fexp_d, c->pexp_d, c->rexp_d,
                              move_src >= 0 ? c->U2 + (size_t)move_src * c->ldu : nullptr,
                              move_src >= 0 ? c->U2 + (size_t)(a0 + nout) * c->ldu : nullptr, c->flag, c->stream);
  } else if (c->prec != RKS_PREC_FP64) {
    std::vector<float2> Q2h(Qp.size());
    for (size_t t = 0; t < Qp.size(); ++t) {
      float h = (float)Qp[t];
      Q2h[t] = make_float2(h, (float)(Qp[t] - (double)h));
    }
    CK(cudaMemcpyAsync(c->Q2, Q2h.data(), Q2h.size() * sizeof(float2), cudaMemcpyHostToDevice, c->stream));
    rks::launch_df_rows_gemm(c->n, c->Ub, c->ldu, a0, nin, c->Q2, nout, a0, move_src, c->f32, c->stream);
  } else {
    CK(cudaMemcpyAsync(c->Qd, Qp.data(), Qp.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    rks::launch_rows_gemm(c->n, c->U, c->ldu, a0, nin, c->Qd, nout, c->U, c->ldu, a0, move_src, c->stream);
  }
  prof_end(c, ps, RKS_K_RESTART, 1, (double)(nin + nout + (move_src >= 0 ? 2 : 0)) * (c->f32 ? 4.0 : 8.0) * c->n,
           2.0 * c->n * nin * nout);
  return launch_err();
}

int contract(rks_ctx* c) {
  const int m = c->m, q = c->q, ma = c->ja, d = c->d;
  const int ldb = m + 1, ldt = c->k + 2;
  std::vector<double> H((size_t)ma * ma), Q((size_t)ma * ma), b(ma);
  for (int j = 0; j < ma; ++j) {
    for (int i = 0; i < ma; ++i) H[i + (size_t)j * ma] = M(c->Ba, ldb, i, j);
    b[j] = M(c->Ba, ldb, ma, j);
  }
  rks_dense::hessenberg_arrow(ma, c->brow, H.data(), ma, Q.data(), ma);
  if (rks_dense::schur(ma, H.data(), ma, Q.data(), ma) != 0) return RKS_EDENSE;
  // Algorithm 1 keeps the k - q best active Schur vectors; with opts.keep > 0
  // the restart is thick: up to keep active vectors even after locking
  int want = c->k - q;
  if (c->opts.keep > 0) want = std::max(want, std::min(c->opts.keep, ma / 2));
  rks_dense::reorder(ma, H.data(), ma, Q.data(), ma, ma, c->which, std::min(want + 1, ma));
  // truncation size: blocks covering `want` columns, pairs kept whole
  int ka = 0;
  for (const auto& B : rks_dense::blocks(ma, H.data(), ma)) {
    if (ka >= want) break;
    ka = B.start + B.size;
  }
  ka = std::min(ka, ma - 1);
  // truncated pieces
  std::vector<double> Ta((size_t)ka * ka), bk(ka, 0.0), Qk((size_t)ma * ka);
  for (int j = 0; j < ka; ++j) {
    for (int i = 0; i < ka; ++i) Ta[i + (size_t)j * ka] = H[i + (size_t)j * ma];
    for (int i = 0; i < ma; ++i) Qk[i + (size_t)j * ma] = Q[i + (size_t)j * ma];
    double acc = 0.0;
    for (int i = 0; i < ma; ++i) acc += b[i] * Q[i + (size_t)j * ma];
    bk[j] = acc;
  }
  std::vector<double> Tqa_new((size_t)ldt * ka, 0.0);
  for (int j = 0; j < ka; ++j)
    for (int i = 0; i < q; ++i) {
      double acc = 0.0;
      for (int l = 0; l < ma; ++l) acc += M(c->Tqa, ldt, i, l) * Qk[l + (size_t)j * ma];
      Tqa_new[i + (size_t)j * ldt] = acc;
    }
  // The device restart (Eq. 3.5) starts now, with the truncated Schur vectors
  // as they are; the host work below (sketches, whitening, aggressive reorder,
  // Gram matrix, locking and, in the caller, the Ritz pairs) overlaps it.
  // Whitening and the aggressive reorder rotate the kept columns once more:
  // that ka x ka factor C goes to the device in upload_restart, as a second
  // in-place product, before the next expansion.
  int rc = restart_launch(c, q, ma, Qk, &c->cs_h[q], ka, m);
  if (rc) return rc;
  // sketches of the kept columns: S_a <- S_a Qk ; last column moves to q+ka
  std::vector<double> Sa((size_t)d * ka, 0.0);
  for (int j = 0; j < ka; ++j)
    for (int l = 0; l < ma; ++l) {
      double w = Qk[l + (size_t)j * ma];
      const double* src = &c->S_h[(size_t)(q + l) * d];
      double* dst = &Sa[(size_t)j * d];
      for (int i = 0; i < d; ++i) dst[i] += w * src[i];
    }
  // whitening when the sketch lost orthonormality (Sec. 3.3, Eqs. 3.7-3.8)
  // (the Gram matrix of the kept sketches, reused below for the device copy
  // of S^T S unless whitening or the reorder changes them)
  const bool sketched = c->opts.ortho != RKS_ORTHO_CGS2;
  std::vector<double> Gsa((size_t)ka * ka, 0.0);
  double gerr = 0.0;
  if (sketched)
    for (int bb = 0; bb < ka; ++bb)
      for (int a = 0; a <= bb; ++a) {
        double acc = 0.0;
        for (int i = 0; i < d; ++i) acc += Sa[i + (size_t)a * d] * Sa[i + (size_t)bb * d];
        Gsa[a + (size_t)bb * ka] = Gsa[bb + (size_t)a * ka] = acc;
        const double e = acc - ((a == bb) ? 1.0 : 0.0);
        gerr += (a == bb ? 1.0 : 2.0) * e * e;
      }
  std::vector<double> Cm;   // pending right factor of the kept columns (empty: none)
  bool whitened = false;
  if (sketched && ka > 0 && std::sqrt(gerr) > 1e-10) {
    whitened = true;
    ++c->stats.whitenings;
    std::vector<double> R((size_t)ka * ka), Rinv((size_t)ka * ka, 0.0);
    rks_dense::house_qr(d, ka, Sa.data(), R.data());
    for (int j = 0; j < ka; ++j) {          // Rinv by back substitution
      Rinv[j + (size_t)j * ka] = 1.0 / R[j + (size_t)j * ka];
      for (int i = j - 1; i >= 0; --i) {
        double acc = 0.0;
        for (int l = i + 1; l <= j; ++l) acc += R[i + (size_t)l * ka] * Rinv[l + (size_t)j * ka];
        Rinv[i + (size_t)j * ka] = -acc / R[i + (size_t)i * ka];
      }
    }
    auto matmul = [](int r, int inner, int cc, const double* X, int ldx, const double* Yv, int ldy,
                     double* Z, int ldz) {
      for (int j = 0; j < cc; ++j)
        for (int i = 0; i < r; ++i) {
          double acc = 0.0;
          for (int l = 0; l < inner; ++l) acc += X[i + (size_t)l * ldx] * Yv[l + (size_t)j * ldy];
          Z[i + (size_t)j * ldz] = acc;
        }
    };
    Cm = Rinv;
    std::vector<double> t2((size_t)ka * ka);
    matmul(ka, ka, ka, Ta.data(), ka, Rinv.data(), ka, t2.data(), ka);
    matmul(ka, ka, ka, R.data(), ka, t2.data(), ka, Ta.data(), ka);
    std::vector<double> b2(ka);
    for (int j = 0; j < ka; ++j) {
      double acc = 0.0;
      for (int l = 0; l < ka; ++l) acc += bk[l] * Rinv[l + (size_t)j * ka];
      b2[j] = acc;
    }
    bk = b2;
    if (q) {
      std::vector<double> t3((size_t)ldt * ka, 0.0);
      matmul(q, ka, ka, Tqa_new.data(), ldt, Rinv.data(), ka, t3.data(), ldt);
      Tqa_new = t3;
    }
  }
  const bool reordered = c->opts.lock && c->opts.aggressive &&
                         aggressive_reorder(c, ka, Ta, bk, Cm, q, ldt, Tqa_new, d, Sa);
  if (reordered) ++c->stats.reorders;
  c->corr = Cm;
  c->corr_q = q;
  c->corr_ka = ka;
  // host copies of the new scales and sketches (uploaded in upload_restart)
  const double s_last_scale = c->cs_h[m];
  for (int j = 0; j < ka; ++j) c->cs_h[q + j] = 1.0;
  c->cs_h[q + ka] = s_last_scale;
  for (int j = q + ka + 1; j <= m; ++j) c->cs_h[j] = 0.0;
  for (int j = 0; j < ka; ++j) std::memcpy(&c->S_h[(size_t)(q + j) * d], &Sa[(size_t)j * d], d * sizeof(double));
  std::memmove(&c->S_h[(size_t)(q + ka) * d], &c->S_h[(size_t)m * d], d * sizeof(double));
  c->up_M2 = c->M2 && sketched;
  if (c->up_M2) {
    // Gram matrix of the kept sketches (locked, active and the last vector)
    // for the least squares of the next expansion
    const int nc = q + ka + 1, ldm = m + 1;
    c->M2_h.assign((size_t)ldm * ldm, make_float2(0.f, 0.f));
    for (int b2 = 0; b2 < nc; ++b2)
      for (int a2 = 0; a2 <= b2; ++a2) {
        double acc = 0.0;
        if (!whitened && !reordered && a2 >= q && b2 < q + ka) {
          acc = Gsa[(a2 - q) + (size_t)(b2 - q) * ka];   // both active: computed above
        } else {
          const double* x = &c->S_h[(size_t)a2 * d];
          const double* y = &c->S_h[(size_t)b2 * d];
          for (int i = 0; i < d; ++i) acc += x[i] * y[i];
        }
        const float h = (float)acc;
        const float2 v = make_float2(h, (float)(acc - (double)h));
        c->M2_h[a2 + (size_t)b2 * ldm] = v;
        c->M2_h[b2 + (size_t)a2 * ldm] = v;
      }
  }
  if (c->prec != RKS_PREC_FP64) {
    c->S2_h.resize(c->S_h.size());
    for (size_t t = 0; t < c->S_h.size(); ++t) {
      float h = (float)c->S_h[t];
      c->S2_h[t] = make_float2(h, (float)(c->S_h[t] - (double)h));
    }
  }
  // locking: leading active blocks with small |b| (relative to |lambda|)
  int r = 0;
  if (c->opts.lock) {
    double tn = 0.0;
    for (double v : Ta) tn += v * v;
    tn = std::sqrt(tn);
    for (const auto& B : rks_dense::blocks(ka, Ta.data(), ka)) {
      if (q + r + B.size > c->k) break;
      const double thr = lock_threshold(c, std::hypot(B.re, B.im), tn);
      bool ok = true;
      for (int t = 0; t < B.size; ++t) ok = ok && std::fabs(bk[B.start + t]) <= thr;
      if (!ok) break;
      r = B.start + B.size;
    }
  }
  if (r > 0) {
    const int qn = q + r;
    std::vector<double> Tqq2((size_t)ldt * ldt, 0.0), Tqa2((size_t)ldt * ka, 0.0);
    for (int j = 0; j < q; ++j)
      for (int i = 0; i <= j + 1 && i < q; ++i) Tqq2[i + (size_t)j * ldt] = M(c->Tqq, ldt, i, j);
    for (int j = 0; j < r; ++j) {
      for (int i = 0; i < q; ++i) Tqq2[i + (size_t)(q + j) * ldt] = Tqa_new[i + (size_t)j * ldt];
      for (int i = 0; i < r; ++i) Tqq2[q + i + (size_t)(q + j) * ldt] = Ta[i + (size_t)j * ka];
    }
    for (int j = r; j < ka; ++j) {
      for (int i = 0; i < q; ++i) Tqa2[i + (size_t)(j - r) * ldt] = Tqa_new[i + (size_t)j * ldt];
      for (int i = 0; i < r; ++i) Tqa2[q + i + (size_t)(j - r) * ldt] = Ta[i + (size_t)j * ka];
    }
    std::vector<double> Ta2((size_t)(ka - r) * (ka - r));
    for (int j = r; j < ka; ++j)
      for (int i = r; i < ka; ++i) Ta2[(i - r) + (size_t)(j - r) * (ka - r)] = Ta[i + (size_t)j * ka];
    std::vector<double> b2(bk.begin() + r, bk.end());
    c->Tqq = Tqq2;
    c->Tqa.assign((size_t)ldt * (m + 1), 0.0);
    std::copy(Tqa2.begin(), Tqa2.end(), c->Tqa.begin());
    Ta = Ta2;
    bk = b2;
    c->q = qn;
    ka -= r;
  } else {
    c->Tqa.assign((size_t)ldt * (m + 1), 0.0);
    std::copy(Tqa_new.begin(), Tqa_new.end(), c->Tqa.begin());
  }
  c->ja = ka;
  std::fill(c->Ba.begin(), c->Ba.end(), 0.0);
  for (int j = 0; j < ka; ++j) {
    for (int i = 0; i < ka; ++i) M(c->Ba, ldb, i, j) = Ta[i + (size_t)j * ka];
    M(c->Ba, ldb, ka, j) = bk[j];
  }
  return RKS_OK;
}

// Second half of a restart, after the host work: the pending rotation of the
// kept columns (whitening, aggressive reorder) as an in-place product, then
// the new column scales, sketches and Gram matrix to the device.
int upload_restart(rks_ctx* c) {
  if (!c->corr.empty()) {
    int rc = restart_launch(c, c->corr_q, c->corr_ka, c->corr, nullptr, c->corr_ka, -1);
    if (rc) return rc;
    c->corr.clear();
  }
  CK(cudaMemcpyAsync(c->colscale, c->cs_h.data(), c->cs_h.size() * sizeof(double), cudaMemcpyHostToDevice,
                     c->stream));
  CK(cudaMemcpyAsync(c->S, c->S_h.data(), c->S_h.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  if (c->up_M2)
    CK(cudaMemcpyAsync(c->M2, c->M2_h.data(), c->M2_h.size() * sizeof(float2), cudaMemcpyHostToDevice,
                       c->stream));
  if (c->prec != RKS_PREC_FP64)
    CK(cudaMemcpyAsync(c->S2, c->S2_h.data(), c->S2_h.size() * sizeof(float2), cudaMemcpyHostToDevice, c->stream));
  return launch_err();
}

// Ritz pairs of the full T = [[Tqq, Tqa], [0, T_a]] and estimates (Eq. 4.8).
void ritz(rks_ctx* c) {
  const int q = c->q, ja = c->ja, kk = q + ja, ldt = c->k + 2, ldb = c->m + 1;
  c->kk = kk;
  c->Tfull.assign((size_t)kk * kk, 0.0);
  c->bfull.assign(kk, 0.0);
  for (int j = 0; j < q; ++j)
    for (int i = 0; i < q; ++i) c->Tfull[i + (size_t)j * kk] = M(c->Tqq, ldt, i, j);
  for (int j = 0; j < ja; ++j) {
    for (int i = 0; i < q; ++i) c->Tfull[i + (size_t)(q + j) * kk] = M(c->Tqa, ldt, i, j);
    for (int i = 0; i < ja; ++i) c->Tfull[q + i + (size_t)(q + j) * kk] = M(c->Ba, ldb, i, j);
    c->bfull[q + j] = M(c->Ba, ldb, ja, j);
  }
  std::vector<double> lre(kk), lim(kk);
  std::vector<cd> Y((size_t)kk * kk);
  rks_dense::quasi_eig(kk, c->Tfull.data(), kk, lre.data(), lim.data(), Y.data(), kk);
  std::vector<int> order(kk);
  for (int i = 0; i < kk; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return rks_dense::key(lre[a], lim[a], c->which) < rks_dense::key(lre[b], lim[b], c->which);
  });
  c->lre.resize(kk); c->lim.resize(kk); c->est.resize(kk); c->Y.resize((size_t)kk * kk);
  for (int t = 0; t < kk; ++t) {
    int o = order[t];
    c->lre[t] = lre[o];
    c->lim[t] = lim[o];
    cd bty = 0.0;
    for (int i = 0; i < kk; ++i) {
      c->Y[i + (size_t)t * kk] = Y[i + (size_t)o * kk];
      bty += c->bfull[i] * Y[i + (size_t)o * kk];
    }
    double al = std::hypot(lre[o], lim[o]);
    c->est[t] = std::abs(bty) / std::max(c->opts.conv == RKS_CONV_NORM1 ? c->norm1 : al, 1e-300);
  }
  int nw = std::min(c->k, kk);
  if (nw > 0 && nw < kk && c->lim[nw - 1] > 0) ++nw;   // never split a complex pair
  c->nw = nw;
}

// Ritz vectors X = U Y (real packing), A X and FP64 residuals.
int finalize(rks_ctx* c) {
  const int kk = c->kk, nw = c->nw;
  if (!c->X) {
    // X holds the nw <= k + 1 Ritz vectors; AX also serves as FP64 scratch
    // for the kk <= min(m, 2k + 1) kept basis columns
    const int ncx = std::min(c->m + 1, 2 * c->k + 2);
    int rc = dalloc(&c->X, (size_t)c->ldu * ncx);
    if (rc) return rc;
    rc = dalloc(&c->AX, (size_t)c->ldu * ncx);
    if (rc) return rc;
    rc = dalloc(&c->rsum, (size_t)4 * (c->k + 1) * rks::kResidCtas);
    if (rc) return rc;
    rc = dalloc(&c->pcol, (size_t)2 * (c->k + 1));
    if (rc) return rc;
    rc = dalloc(&c->plam, (size_t)2 * (c->k + 1));
    if (rc) return rc;
  }
  std::vector<double> Yr((size_t)kk * nw);
  std::vector<int> col, colim;
  std::vector<double> pl_re, pl_im;
  for (int t = 0; t < nw;) {
    bool pair = c->lim[t] > 0 && t + 1 < nw;
    for (int i = 0; i < kk; ++i) {
      Yr[i + (size_t)t * kk] = c->Y[i + (size_t)t * kk].real();
      if (pair) Yr[i + (size_t)(t + 1) * kk] = c->Y[i + (size_t)t * kk].imag();
    }
    col.push_back(t);
    colim.push_back(pair ? t + 1 : -1);
    pl_re.push_back(c->lre[t]);
    pl_im.push_back(pair ? c->lim[t] : 0.0);
    t += pair ? 2 : 1;
  }
  const int np = (int)col.size();
  CK(cudaMemcpyAsync(c->Qd, Yr.data(), Yr.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  int ps = prof_begin(c, RKS_K_OTHER);
  if (c->prec != RKS_PREC_FP64) {
    rks::launch_df2d_cols(c->n, c->Ub, c->ldu, c->AX, c->ldu, kk, c->f32, c->stream);
    rks::launch_rows_gemm(c->n, c->AX, c->ldu, 0, kk, c->Qd, nw, c->X, c->ldu, 0, -1, c->stream);
  } else {
    rks::launch_rows_gemm(c->n, c->U, c->ldu, 0, kk, c->Qd, nw, c->X, c->ldu, 0, -1, c->stream);
  }
  rks::launch_spmm(c->A, c->X, c->ldu, c->AX, c->ldu, nw, c->stream);
  std::vector<int> pc(2 * np);
  std::vector<double> pv(2 * np);
  for (int t = 0; t < np; ++t) { pc[t] = col[t]; pc[np + t] = colim[t]; pv[t] = pl_re[t]; pv[np + t] = pl_im[t]; }
  CK(cudaMemcpyAsync(c->pcol, pc.data(), pc.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->plam, pv.data(), pv.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  const int rg = rks::launch_resid_sums(c->n, c->X, c->AX, c->ldu, np, c->pcol, c->pcol + np, c->plam,
                                        c->plam + np, c->rsum, c->stream);
  prof_end(c, ps, RKS_K_OTHER, 3, 0.0, 0.0);
  int rc = launch_err();
  if (rc) return rc;
  std::vector<double> part((size_t)4 * np * rg), sums(4 * np, 0.0);
  CK(cudaMemcpyAsync(part.data(), c->rsum, part.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int q = 0; q < 4 * np; ++q)
    for (int g = 0; g < rg; ++g) sums[q] += part[(size_t)q * rg + g];
  prof_flush(c);
  c->resid.assign(nw, 0.0);
  c->rq_re.assign(nw, 0.0);
  c->rq_im.assign(nw, 0.0);
  for (int t = 0; t < np; ++t) {
    const double xx = std::max(sums[4 * t + 1], 1e-300);
    double res = std::sqrt(sums[4 * t]) / (c->norm1 * std::sqrt(xx));
    c->resid[col[t]] = res;
    // x^H A x / x^H x for x = X[:, col] + i X[:, colim] (the member with
    // Im lambda > 0); its conjugate partner gets the conjugate quotient
    c->rq_re[col[t]] = sums[4 * t + 2] / xx;
    c->rq_im[col[t]] = colim[t] >= 0 ? sums[4 * t + 3] / xx : 0.0;
    if (colim[t] >= 0) {
      c->resid[colim[t]] = res;
      c->rq_re[colim[t]] = c->rq_re[col[t]];
      c->rq_im[colim[t]] = -c->rq_im[col[t]];
    }
  }
  return RKS_OK;
}

void free_ctx(rks_ctx* c) {
  if (!c) return;
  cudaFree(c->rowptr); cudaFree(c->colind); cudaFree(c->vals);
  cudaFree(c->U); cudaFree(c->S); cudaFree(c->colscale);
  cudaFree(c->z_raw); cudaFree(c->s_raw); cudaFree(c->z1); cudaFree(c->r1); cudaFree(c->r); cudaFree(c->rs);
  cudaFree(c->coef); cudaFree(c->flag); cudaFree(c->Qd); cudaFree(c->u1);
  cudaFree(c->X); cudaFree(c->AX); cudaFree(c->rsum); cudaFree(c->pcol); cudaFree(c->plam);
  cudaFree(c->ell_col); cudaFree(c->ell_val2); cudaFree(c->ell_valf); cudaFree(c->dia_val2); cudaFree(c->dia_valf);
  cudaFree(c->A2.mp_row); cudaFree(c->A2.mp_val); cudaFree(c->A2.mp_w); cudaFree(c->A2.mp_part);
  cudaFree(c->vals2); cudaFree(c->U2); cudaFree(c->S2); cudaFree(c->nrs); cudaFree(c->sj); cudaFree(c->Q2);
  cudaFree(c->rprev); cudaFree(c->znorm); cudaFree(c->tmp64); cudaFree(c->valsf); cudaFree(c->Uf);
  cudaFree(c->otab); cudaFree(c->lsr1); cudaFree(c->M2); cudaFree(c->bar); cudaFree(c->qimg);
  cudaFree(c->qimg_df); cudaFree(c->fexp_d); cudaFree(c->pexp_d); cudaFree(c->rexp_d);
  rks::free_sketch_tiles(&c->tiles);
  cudaFree(c->part_z); cudaFree(c->part_s); cudaFree(c->part_d);
  for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // namespace

extern "C" {

void rks_opts_default(rks_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->zeta = 8;
  o->maxit = 1000;
  o->lock = 1;
  o->tc_restart = 1;
}

const char* rks_strerror(int s) {
  switch (s) {
    case RKS_OK: return "ok";
    case RKS_EINVAL: return "invalid argument";
    case RKS_ENOMEM: return "out of memory";
    case RKS_ECUDA: return "CUDA error";
    case RKS_ENOCONV: return "not converged within maxit restarts (results are partial)";
    case RKS_EBREAKDOWN: return "breakdown: invariant subspace reached";
    case RKS_ENAN: return "non-finite value encountered";
    case RKS_ESTATE: return "call out of order";
    case RKS_EDENSE: return "small dense Schur iteration failed";
    case RKS_ETIMEOUT: return "a bounded device-side wait timed out";
    default: return "unknown status";
  }
}

int rks_create(rks_ctx** out, int64_t n, const int32_t* rowptr, const int32_t* colind, const void* vals,
               int vals_dtype, int k, int p, int d, int which, double tol, uint64_t seed, const rks_opts* opts) {
  if (!out) return RKS_EINVAL;
  *out = nullptr;
  rks_opts o;
  rks_opts_default(&o);
  if (opts) o = *opts;
  if (o.zeta == 0) o.zeta = 8;
  if (o.conv != RKS_CONV_EIG && o.conv != RKS_CONV_NORM1) return RKS_EINVAL;
  if (o.prec != RKS_PREC_DF && o.prec != RKS_PREC_FP64 && o.prec != RKS_PREC_MIXED) return RKS_EINVAL;
  if (o.debug_stall != 0 && o.debug_stall != 1) return RKS_EINVAL;
  if (o.maxit <= 0) o.maxit = 1000;
  if (o.keep < 0 || o.keep > k) return RKS_EINVAL;
  if (o.aggressive != 0 && o.aggressive != 1) return RKS_EINVAL;
  if (o.ortho != RKS_ORTHO_SKETCH && o.ortho != RKS_ORTHO_CGS2) return RKS_EINVAL;
  if (o.ortho == RKS_ORTHO_CGS2 && o.prec != RKS_PREC_DF) return RKS_EINVAL;
  const int m = k + p;
  if (n <= 0 || !rowptr || !colind || !vals || k < 1 || p < 2 || (int64_t)m + 1 > n || d < m + 1 ||
      o.zeta < 1 || o.zeta > 16 || d < 2 * o.zeta || d > 8192 || which < 0 || which > 3 || !(tol > 0) ||
      (vals_dtype != RKS_F64 && vals_dtype != RKS_F32) || n > (int64_t)INT32_MAX)
    return RKS_EINVAL;
  // the restart product keeps an (m x (k+2)) tile of Q' and 128 x (k+2) outputs in shared memory
  if (rks::rows_gemm_smem(m, k + 2, 128) > 200 * 1024) return RKS_EINVAL;
  rks_ctx* c = new (std::nothrow) rks_ctx();
  if (!c) return RKS_ENOMEM;
  c->n = n; c->k = k; c->p = p; c->m = m; c->d = d; c->zeta = o.zeta; c->which = which;
  c->tol = tol; c->seed = seed; c->opts = o; c->prec = o.prec;
  c->eta_lock = o.eta_lock > 0 ? o.eta_lock : tol;
  c->zscale = 1.0 / std::sqrt((double)o.zeta);
  const cudaMemcpyKind kind = o.mem_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  int rc = RKS_OK;
  auto fail = [&](int code) { free_ctx(c); return code; };
  if (o.stream) {
    c->stream = (cudaStream_t)o.stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(RKS_ECUDA);
    c->own_stream = true;
  }
  if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) return fail(RKS_ECUDA);
  // CSR: read nnz from rowptr[n]
  int32_t nnz32 = 0;
  if (cudaMemcpy(&nnz32, rowptr + n, sizeof(int32_t), o.mem_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost) !=
      cudaSuccess)
    return fail(RKS_ECUDA);
  if (nnz32 < 0) return fail(RKS_EINVAL);
  c->nnz = nnz32;
  if ((rc = dalloc(&c->rowptr, n + 1)) || (rc = dalloc(&c->colind, c->nnz)) || (rc = dalloc(&c->vals, c->nnz)))
    return fail(rc);
  if (cudaMemcpyAsync(c->rowptr, rowptr, (n + 1) * sizeof(int32_t), kind, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->colind, colind, c->nnz * sizeof(int32_t), kind, c->stream) != cudaSuccess)
    return fail(RKS_ECUDA);
  if (vals_dtype == RKS_F64) {
    if (cudaMemcpyAsync(c->vals, vals, c->nnz * sizeof(double), kind, c->stream) != cudaSuccess) return fail(RKS_ECUDA);
  } else {
    float* tmp = nullptr;
    if ((rc = dalloc(&tmp, c->nnz))) return fail(rc);
    if (cudaMemcpyAsync(tmp, vals, c->nnz * sizeof(float), kind, c->stream) != cudaSuccess) { cudaFree(tmp); return fail(RKS_ECUDA); }
    rks::launch_f32_to_f64(c->nnz, tmp, c->vals, c->stream);
    cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
  }
  if ((rc = dalloc(&c->flag, 4))) return fail(rc);
  if (cudaMemsetAsync(c->flag, 0, 4 * sizeof(int), c->stream) != cudaSuccess) return fail(RKS_ECUDA);
  rks::launch_check_csr(n, c->nnz, c->rowptr, c->colind, c->flag, c->stream);
  int bad = 0;
  if (cudaMemcpyAsync(&bad, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(RKS_ECUDA);
  if (bad) return fail(RKS_EINVAL);
  c->A.n = n; c->A.nnz = c->nnz; c->A.rowptr = c->rowptr; c->A.colind = c->colind; c->A.vals = c->vals;
  // ||A||_1: column sums of |a_ij| on the host, entries in storage order (the
  // same bits on every run; FP64 atomics would add them in varying order)
  {
    std::vector<int32_t> ci(c->nnz);
    std::vector<double> cv(c->nnz);
    cudaError_t e = cudaMemcpyAsync(ci.data(), c->colind, c->nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(cv.data(), c->vals, c->nnz * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(RKS_ECUDA);
    std::vector<double> colsum(n, 0.0);
    for (int64_t p = 0; p < c->nnz; ++p) colsum[ci[p]] += std::fabs(cv[p]);
    if (c->prec != RKS_PREC_FP64) {
      // the double-float and FP32 copies need every value inside the FP32
      // exponent range: above FLT_MAX a value becomes inf, below FLT_MIN it
      // loses significand bits silently
      bool exact = true;
      for (int64_t p = 0; p < c->nnz; ++p) {
        const double a = std::fabs(cv[p]);
        if (!std::isfinite(a)) return fail(RKS_ENAN);
        if (a > 3.4028234663852886e38 || (a != 0.0 && a < 1.1754943508222875e-38)) return fail(RKS_EINVAL);
        exact = exact && (double)(float)cv[p] == cv[p];
      }
      c->vals_f32 = exact;
    }
    // widest row: an ELLPACK copy for the SpMV when the padding stays small
    std::vector<int32_t> rp(n + 1);
    if (cudaMemcpyAsync(rp.data(), c->rowptr, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return fail(RKS_ECUDA);
    int wmax = 0;
    for (int64_t i = 0; i < n; ++i) wmax = std::max(wmax, rp[i + 1] - rp[i]);
    const int64_t slots = (n + 31) / 32 * 32 * (int64_t)wmax;
    c->ell_w = (wmax >= 1 && wmax <= 16 && (double)slots <= 1.25 * (double)std::max<int64_t>(c->nnz, 1)) ? wmax : 0;
    // row-length statistics for the CSR kernels: a warp per row for long
    // rows, merge path when the longest row is far above the mean
    {
      const double mean = n ? (double)c->nnz / (double)n : 0.0;
      c->spmv_merge = wmax > 128 && (double)wmax > 16.0 * mean;
      c->spmv_warp = !c->spmv_merge && mean >= 16.0;
    }
    // at most 16 distinct diagonals with little padding (stencils): a
    // diagonal copy for the SpMV instead
    {
      std::vector<int64_t> offs;
      bool fits = c->nnz > 0;
      for (int64_t i = 0; i < n && fits; ++i)
        for (int32_t q = rp[i]; q < rp[i + 1]; ++q) {
          const int64_t o = (int64_t)ci[q] - i;
          if (std::find(offs.begin(), offs.end(), o) == offs.end()) {
            offs.push_back(o);
            if (offs.size() > 16) { fits = false; break; }
          }
        }
      if (fits && (double)offs.size() * (double)n <= 1.3 * (double)c->nnz) {
        std::sort(offs.begin(), offs.end());
        c->dia_d = (int)offs.size();
        for (int e = 0; e < c->dia_d; ++e) c->dia_off[e] = (int)offs[e];
      }
    }
    c->norm1 = n ? *std::max_element(colsum.begin(), colsum.end()) : 0.0;
    if (!std::isfinite(c->norm1)) return fail(RKS_ENAN);
    if (c->norm1 == 0.0) c->norm1 = 1.0;
  }
  c->ldu = (n + 31) / 32 * 32;
  if (c->prec != RKS_PREC_FP64) {
    if (c->prec == RKS_PREC_MIXED) {
      if ((rc = dalloc(&c->Uf, (size_t)c->ldu * (m + 1))) || (rc = dalloc(&c->valsf, c->nnz))) return fail(rc);
      if (o.tc_restart && cudaMalloc(&c->qimg, rks::kTcImageBytes) != cudaSuccess) return fail(RKS_ENOMEM);
      if (rks::configure_tc_kernels() != cudaSuccess) return fail(RKS_ECUDA);
      rks::launch_d2df(c->nnz, c->vals, c->valsf, true, c->stream);
    }
    if ((rc = dalloc(&c->U2, (size_t)c->ldu * (m + 1))) || (rc = dalloc(&c->vals2, c->nnz)) ||
        (rc = dalloc(&c->S2, (size_t)d * (m + 1))) || (rc = dalloc(&c->nrs, m + 1)) || (rc = dalloc(&c->sj, 1)) ||
        (rc = dalloc(&c->Q2, (size_t)(m + 1) * (m + 1))) || (rc = dalloc(&c->rprev, m + 1)) ||
        (rc = dalloc(&c->znorm, 1)) || (rc = dalloc(&c->tmp64, n)) ||
        (rc = dalloc(&c->otab, (size_t)n * rks::omega_slots(o.zeta))) || (rc = dalloc(&c->lsr1, m + 1)) ||
        (rc = dalloc(&c->M2, (size_t)(m + 1) * (m + 1))) || (rc = dalloc(&c->bar, 2)))
      return fail(rc);
    if (o.tc_restart && rks::tc_restart_df_supported(m, k + 1)) {
      if (rks::configure_tc_kernels() != cudaSuccess) return fail(RKS_ECUDA);
      if (cudaMalloc(&c->qimg_df, rks::kTcDfImageBytes) != cudaSuccess ||
          cudaMalloc(&c->fexp_d, 64 * sizeof(int)) != cudaSuccess ||
          cudaMalloc(&c->pexp_d, 256 * sizeof(int)) != cudaSuccess ||
          cudaMalloc(&c->rexp_d, (size_t)n * sizeof(int)) != cudaSuccess)
        return fail(RKS_ENOMEM);
    }
    if (cudaMemsetAsync(c->bar, 0, 2 * sizeof(unsigned), c->stream) != cudaSuccess) return fail(RKS_ECUDA);
    {
      int bad = 0;
      if (cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream) != cudaSuccess) return fail(RKS_ECUDA);
      rks::launch_omega_table(n, d, o.zeta, seed, c->otab, c->flag, c->stream);
      if (cudaMemcpyAsync(&bad, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess)
        return fail(RKS_ECUDA);
      if (bad) return fail(RKS_EINVAL);
    }
    if (rks::configure_df_kernels() != cudaSuccess) return fail(RKS_ECUDA);
    if (rks::build_sketch_tiles(n, d, o.zeta, c->otab, &c->tiles, c->stream) != 0) return fail(RKS_ECUDA);
    cudaFree(c->otab);
    c->otab = nullptr;
    if (rks::sketch_tile_smem(c->tiles, m + 1) > 200 * 1024) return fail(RKS_EINVAL);
    if ((rc = dalloc(&c->part_z, (size_t)c->tiles.G * d)) || (rc = dalloc(&c->part_s, (size_t)c->tiles.G * d)) ||
        (rc = dalloc(&c->part_d, (size_t)c->tiles.G * (m + 1))))
      return fail(rc);
    rks::launch_d2df(c->nnz, c->vals, c->vals2, false, c->stream);
    c->A2.n = n; c->A2.nnz = c->nnz; c->A2.rowptr = c->rowptr; c->A2.colind = c->colind; c->A2.vals = c->vals2;
    if (c->dia_d) {
      const int64_t ldd = (n + 31) / 32 * 32;
      if ((rc = dalloc(&c->dia_val2, (size_t)c->dia_d * ldd))) return fail(rc);
      rks::launch_dia_fill(n, c->dia_d, c->dia_off, ldd, c->rowptr, c->colind, c->vals2, false, c->dia_val2,
                           c->stream);
      if (c->prec == RKS_PREC_MIXED) {
        if ((rc = dalloc(&c->dia_valf, (size_t)c->dia_d * ldd))) return fail(rc);
        rks::launch_dia_fill(n, c->dia_d, c->dia_off, ldd, c->rowptr, c->colind, c->valsf, true, c->dia_valf,
                             c->stream);
      } else if (c->vals_f32 && c->dia_d <= 8) {
        // FP32 values: the double-float SpMV reads them from an FP32 copy
        float* vf = nullptr;
        if ((rc = dalloc(&vf, c->nnz))) return fail(rc);
        rks::launch_d2df(c->nnz, c->vals, vf, true, c->stream);
        if ((rc = dalloc(&c->dia_valf, (size_t)c->dia_d * ldd))) { cudaFree(vf); return fail(rc); }
        rks::launch_dia_fill(n, c->dia_d, c->dia_off, ldd, c->rowptr, c->colind, vf, true, c->dia_valf, c->stream);
        cudaStreamSynchronize(c->stream);
        cudaFree(vf);
      }
      if (c->vals_f32 && c->dia_d <= 8) c->A2.dvals_f32 = c->dia_valf;
      if ((rc = launch_err())) return fail(rc);
      c->A2.D = c->dia_d;
      for (int e = 0; e < c->dia_d; ++e) c->A2.doff[e] = c->dia_off[e];
      c->A2.ldd = ldd;
      c->A2.dvals = c->dia_val2;
      c->A2.fmt = rks::kSpmvDia;
    } else if (!c->ell_w && c->spmv_merge) {
      // rows of very uneven length: merge path (rows + entries split evenly)
      c->A2.fmt = rks::kSpmvMerge;
      c->A2.mp_threads = (n + c->nnz + rks::kMergeItems - 1) / rks::kMergeItems;
      const int64_t nbm = (c->A2.mp_threads + rks::kMergeCta - 1) / rks::kMergeCta;
      if ((rc = dalloc(&c->A2.mp_row, (size_t)c->A2.mp_threads)) ||
          (rc = dalloc(&c->A2.mp_val, (size_t)c->A2.mp_threads)) || (rc = dalloc(&c->A2.mp_part, (size_t)nbm + 1)))
        return fail(rc);
      if (c->prec == RKS_PREC_MIXED && (rc = dalloc(&c->A2.mp_w, (size_t)n))) return fail(rc);
      rks::launch_merge_partition(c->A2, c->stream);
      if ((rc = launch_err())) return fail(rc);
    } else if (!c->ell_w && c->spmv_warp) {
      c->A2.fmt = rks::kSpmvWarp;          // long rows: a warp per row
    } else if (c->ell_w) {
      const size_t slots = (size_t)((n + 31) / 32 * 32) * c->ell_w;
      if ((rc = dalloc(&c->ell_col, slots)) || (rc = dalloc(&c->ell_val2, slots))) return fail(rc);
      rks::launch_ell_fill(n, c->ell_w, c->rowptr, c->colind, c->vals2, false, c->ell_col, c->ell_val2, c->stream);
      if (c->prec == RKS_PREC_MIXED) {
        if ((rc = dalloc(&c->ell_valf, slots))) return fail(rc);
        rks::launch_ell_fill(n, c->ell_w, c->rowptr, c->colind, c->valsf, true, c->ell_col, c->ell_valf, c->stream);
      }
      if ((rc = launch_err())) return fail(rc);
      c->A2.W = c->ell_w;
      c->A2.ecol = c->ell_col;
      c->A2.evals = c->ell_val2;
      c->A2.fmt = rks::kSpmvEll;
    }
    c->Ub = c->U2;
    if (rks::configure_df_kernels() != cudaSuccess) return fail(RKS_ECUDA);
    if (rks::df_gemm_smem(m, k + 2) > 200 * 1024 || rks::df_small_smem(d, m + 1) > 200 * 1024) return fail(RKS_EINVAL);
  } else if ((rc = dalloc(&c->U, (size_t)c->ldu * (m + 1)))) {
    return fail(rc);
  }
  if ((rc = dalloc(&c->S, (size_t)d * (m + 1))) ||
      (rc = dalloc(&c->colscale, m + 1)) || (rc = dalloc(&c->z_raw, d)) || (rc = dalloc(&c->s_raw, d)) ||
      (rc = dalloc(&c->z1, d)) || (rc = dalloc(&c->r1, m + 1)) || (rc = dalloc(&c->r, m + 1)) ||
      (rc = dalloc(&c->rs, m + 1)) || (rc = dalloc(&c->coef, (size_t)(m + 1) * m)) ||
      (rc = dalloc(&c->Qd, (size_t)(m + 1) * (m + 1))))
    return fail(rc);
  if (o.u1) {
    if ((rc = dalloc(&c->u1, n))) return fail(rc);
    if (cudaMemcpyAsync(c->u1, o.u1, n * sizeof(double), kind, c->stream) != cudaSuccess) return fail(RKS_ECUDA);
  }
  c->opts.u1 = nullptr;  // the caller's pointer is not kept
  c->S_h.assign((size_t)d * (m + 1), 0.0);
  c->cs_h.assign(m + 1, 0.0);
  c->coef_h.assign((size_t)(m + 1) * m, 0.0);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(RKS_ECUDA);
  if (rks::configure_kernels() != cudaSuccess) return fail(RKS_ECUDA);
  *out = c;
  return RKS_OK;
}

// Mixed path: carry the FP32 phase's Krylov-Schur decomposition
// A U = U T + u b^T (q = 0, ka = ja kept columns, u at column ka) over to
// double-float, so that the double-float restarts continue from it instead of
// from one start vector.  The FP32 columns are promoted exactly; their
// relation error E = A U - U T - u b^T (the FP32 rounding of the stored basis
// vectors, of the order of 2^-24 ||A|| per column) is formed in double-float
// and reduced by damped Jacobi sweeps on the correction equation
// A X - X T = -E, U <- U + X; the corrected columns are sketched again and
// [U u] is made sketch-orthonormal once more (the R of the QR of
// [Omega U, Omega u], Sec. 3.3), T and b following the change of basis
// exactly: with [U u] = [V v] R, A V = V (R11 T + r12 b^T) R11^-1 +
// v r22 b^T R11^-1.  The sweeps stop once the largest column norm of the
// relation error, over ||A||_1 (*rel, measured every kHandoverCheck sweeps
// at the sweep's input), is at most thr / 2, stops falling, or after
// kHandoverSweeps; above thr the decomposition is not accurate enough for the
// target: RKS_EDENSE, the basis is left promoted but not rotated.
// RKS_EINVAL: the state does not allow it (nothing in the basis has changed).
constexpr int kHandoverSweeps = 48;
constexpr int kHandoverCheck = 8;
constexpr float kJacobiOmega = 0.67f;

static int handover_df(rks_ctx* c, double thr, double* rel) {
  const int ka = c->ja, m = c->m, d = c->d, ldb = m + 1;
  const int64_t n = c->n, ldu = c->ldu;
  if (c->prec != RKS_PREC_MIXED || c->q != 0 || ka < 1 || ka + 1 > m + 1 || !c->valsf ||
      c->opts.ortho != RKS_ORTHO_SKETCH)
    return RKS_EINVAL;
  std::vector<double> T((size_t)ka * ka), b(ka);
  for (int j = 0; j < ka; ++j) {
    for (int i = 0; i < ka; ++i) T[i + (size_t)j * ka] = M(c->Ba, ldb, i, j);
    b[j] = M(c->Ba, ldb, ka, j);
  }
  const double cs_u = c->cs_h[ka];
  for (int j = 0; j < ka; ++j)
    if (c->cs_h[j] != 1.0) return RKS_EINVAL;
  // the double-float basis and storage of A from here on
  c->f32 = false;
  c->Ub = c->U2;
  c->A2.vals = c->vals2;
  c->A2.evals = c->ell_val2;
  if (c->dia_d) c->A2.dvals = c->dia_val2;
  c->A2.f32 = false;
  float *work = nullptr, *dinv = nullptr;
  float2* dfw = nullptr;
  double* part = nullptr;
  const int gj = rks::jacobi_sweep_ctas(n);
  int rc = dalloc(&work, (size_t)4 * ka * ldu);
  if (!rc) rc = dalloc(&dinv, (size_t)n);
  if (!rc) rc = dalloc(&part, (size_t)gj * ka);
  if (!rc) rc = dalloc(&dfw, (size_t)(2 * ka + 1) * ldu);
  auto release = [&]() { cudaFree(work); cudaFree(dinv); cudaFree(part); cudaFree(dfw); };
  if (rc) {
    release();
    cudaGetLastError();   // a failed allocation leaves its error for the next launch check
    return rc;
  }
  const int ps = prof_begin(c, RKS_K_OTHER);
  rks::launch_f32_to_df_cols(n, c->Uf, ldu, ka + 1, c->U2, c->stream);
  // double-float scratch: U in columns 0 .. ka-1, V = U T in ka .. 2ka-1,
  // w = A u_j in 2ka
  std::vector<float2> T2((size_t)ka * ka);
  for (size_t t = 0; t < T.size(); ++t) {
    const float h = (float)T[t];
    T2[t] = make_float2(h, (float)(T[t] - (double)h));
  }
  CK(cudaMemcpyAsync(c->Q2, T2.data(), T2.size() * sizeof(float2), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(dfw, c->U2, (size_t)ka * ldu * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
  rks::launch_df_rows_gemm(n, dfw, ldu, 0, ka, c->Q2, ka, ka, -1, false, c->stream);
  float* Xa = work;
  float* Xb = work + (size_t)ka * ldu;
  float* Y = work + (size_t)2 * ka * ldu;
  float* E = work + (size_t)3 * ka * ldu;
  float2* wcol = dfw + (size_t)(2 * ka) * ldu;
  for (int j = 0; j < ka; ++j) {
    rks::launch_df_spmv(c->A2, c->U2 + (size_t)j * ldu, wcol, c->tiles, c->stream);
    rks::launch_relation_resid(n, wcol, dfw + (size_t)(ka + j) * ldu, c->U2 + (size_t)ka * ldu, b[j] * cs_u,
                               E + (size_t)j * ldu, c->stream);
  }
  // Jacobi sweeps in FP32 (E is formed in double-float; X is a correction of
  // relative size 2^-24, so FP32 carries it far below the target)
  rks::launch_diag_inv(n, c->rowptr, c->colind, c->valsf, dinv, c->stream);
  CK(cudaMemsetAsync(Xa, 0, (size_t)ka * ldu * sizeof(float), c->stream));
  int cur = 0;   // the iterate is in columns cur .. cur + ka - 1 of the work array, the next in the other half
  std::vector<double> ph((size_t)gj * ka);
  double prev = 1e300;
  *rel = 1e300;
  int sweeps = 0;
  for (int it = 0; it < kHandoverSweeps; ++it) {
    rks::launch_df_rows_gemm(n, work, ldu, cur, ka, c->Q2, ka, 2 * ka, -1, true, c->stream);   // Y = X T
    const bool check = (it + 1) % kHandoverCheck == 0;
    rks::launch_jacobi_sweep(n, c->rowptr, c->colind, c->valsf, dinv, ka, ldu, cur ? Xb : Xa, E, Y, kJacobiOmega,
                             cur ? Xa : Xb, check ? part : nullptr, c->stream);
    cur = ka - cur;
    ++sweeps;
    if (!check) continue;
    rc = launch_err();
    if (rc) { release(); return rc; }
    CK(cudaMemcpyAsync(ph.data(), part, ph.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    double worst = 0.0;
    for (int j = 0; j < ka; ++j) {
      double acc = 0.0;
      for (int g = 0; g < gj; ++g) acc += ph[(size_t)g * ka + j];
      worst = std::max(worst, std::sqrt(acc));
    }
    *rel = worst / c->norm1;
    if (*rel <= 0.5 * thr || *rel > 0.9 * prev) break;
    prev = *rel;
  }
  rks::launch_df_add_f32_cols(n, c->U2, ldu, ka, cur ? Xb : Xa, ldu, c->stream);
  rc = launch_err();
  if (rc) { release(); return rc; }
  if (!(*rel <= thr)) {
    prof_end(c, ps, RKS_K_OTHER, 4 + 2 * ka + 2 * sweeps, 0.0, 0.0);
    release();
    return RKS_EDENSE;
  }
  // sketches of the corrected columns and of u (the per-CTA partials summed in
  // CTA order); u's must agree with the one the FP32 phase kept
  std::vector<double> Sall((size_t)d * (ka + 1)), pz((size_t)c->tiles.G * d);
  for (int j = 0; j <= ka; ++j) {
    rks::launch_df_sketch_vec(c->U2 + (size_t)j * ldu, c->tiles, c->part_s, false, c->stream);
    CK(cudaMemcpyAsync(pz.data(), c->part_s, pz.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const double sc = c->zscale * (j == ka ? cs_u : 1.0);
    for (int r = 0; r < d; ++r) {
      double acc = 0.0;
      for (int g = 0; g < c->tiles.G; ++g) acc += pz[(size_t)g * d + r];
      Sall[r + (size_t)j * d] = sc * acc;
    }
  }
  prof_end(c, ps, RKS_K_OTHER, 5 + 2 * ka + 2 * sweeps + ka + 1, 0.0, 0.0);
  release();
  {
    double du = 0.0, nu = 0.0;
    for (int r = 0; r < d; ++r) {
      const double a = Sall[r + (size_t)ka * d], e = c->S_h[r + (size_t)ka * d];
      du += (a - e) * (a - e);
      nu += e * e;
    }
    if (!(du <= 1e-6 * nu)) return RKS_EINVAL;   // not the decomposition the FP32 phase left
  }
  const int kb = ka + 1;
  std::vector<double> Rinv((size_t)kb * kb), Tn((size_t)ka * ka), bn(ka);
  if (rks_dense::sketch_reorthonormalize(d, ka, Sall.data(), T.data(), b.data(), Rinv.data(), Tn.data(),
                                         bn.data()) != 0)
    return RKS_EINVAL;
  // [V v] = [U u] diag(cs) R^-1 in place
  rc = restart_launch(c, 0, kb, Rinv, c->cs_h.data(), kb, -1);
  if (rc) return rc;
  for (int j = 0; j <= m; ++j) c->cs_h[j] = j < kb ? 1.0 : 0.0;
  std::fill(c->S_h.begin(), c->S_h.end(), 0.0);
  std::copy(Sall.begin(), Sall.end(), c->S_h.begin());
  std::fill(c->Ba.begin(), c->Ba.end(), 0.0);
  for (int j = 0; j < ka; ++j) {
    for (int i = 0; i < ka; ++i) M(c->Ba, ldb, i, j) = Tn[i + (size_t)j * ka];
    M(c->Ba, ldb, ka, j) = bn[j];
  }
  c->Tqq.assign((size_t)(c->k + 2) * (c->k + 2), 0.0);
  c->Tqa.assign((size_t)(c->k + 2) * (m + 1), 0.0);
  c->corr.clear();
  c->up_M2 = c->M2 != nullptr;
  if (c->up_M2) {
    const int ldm = m + 1;
    c->M2_h.assign((size_t)ldm * ldm, make_float2(0.f, 0.f));
    for (int b2 = 0; b2 < kb; ++b2)
      for (int a2 = 0; a2 <= b2; ++a2) {
        double acc = 0.0;
        for (int i = 0; i < d; ++i) acc += c->S_h[i + (size_t)a2 * d] * c->S_h[i + (size_t)b2 * d];
        const float h = (float)acc;
        const float2 v = make_float2(h, (float)(acc - (double)h));
        c->M2_h[a2 + (size_t)b2 * ldm] = v;
        c->M2_h[b2 + (size_t)a2 * ldm] = v;
      }
  }
  c->S2_h.resize(c->S_h.size());
  for (size_t t = 0; t < c->S_h.size(); ++t) {
    const float h = (float)c->S_h[t];
    c->S2_h[t] = make_float2(h, (float)(c->S_h[t] - (double)h));
  }
  rc = upload_restart(c);
  if (rc) return rc;
  ritz(c);
  return RKS_OK;
}

// Algorithm 1's initial state: the start vector u_1 = u~_1 / ||Omega u~_1||
// (Sec. 3.1, k = 0) in column 0, nothing kept.
static int start_alg1(rks_ctx* c, const double* start) {
  const int m = c->m, d = c->d;
  c->q = 0; c->ja = 0; c->kk = 0; c->nw = 0;
  c->Ba.assign((size_t)(m + 1) * m, 0.0);
  c->Tqq.assign((size_t)(c->k + 2) * (c->k + 2), 0.0);
  c->Tqa.assign((size_t)(c->k + 2) * (m + 1), 0.0);
  CK(cudaMemsetAsync(c->flag, 0, 4 * sizeof(int), c->stream));
  CK(cudaMemsetAsync(c->z_raw, 0, d * sizeof(double), c->stream));
  CK(cudaMemsetAsync(c->s_raw, 0, d * sizeof(double), c->stream));
  CK(cudaMemsetAsync(c->coef, 0, (size_t)(m + 1) * m * sizeof(double), c->stream));
  CK(cudaMemsetAsync(c->S, 0, (size_t)d * (m + 1) * sizeof(double), c->stream));
  CK(cudaMemsetAsync(c->colscale, 0, (m + 1) * sizeof(double), c->stream));
  // start vector (Sec. 3.1, k = 0): u_1 = u~_1 / ||Omega u~_1||
  int ps = prof_begin(c, RKS_K_OTHER);
  if (c->prec != RKS_PREC_FP64) {
    const double* src = start ? start : c->u1;
    if (!src) { rks::launch_start_vector(c->n, c->seed + 1, c->tmp64, c->stream); src = c->tmp64; }
    rks::launch_d2df(c->n, src, c->Ub, c->f32, c->stream);
    if (c->opts.ortho == RKS_ORTHO_CGS2) {   // Euclidean normalisation of the start vector
      rks::launch_df_dots(c->Ub, c->ldu, 1, 0, c->tiles, c->part_d, c->stream);
      rks::launch_ks_finish(-1, c->tiles.G, c->part_d, 0.0, c->colscale, c->rprev, c->coef, m + 1, c->flag,
                            c->stream);
      prof_end(c, ps, RKS_K_OTHER, src == c->tmp64 && !start ? 4 : 3, 0.0, 0.0);
    } else {
      rks::launch_df_sketch_vec(c->Ub, c->tiles, c->part_s, c->f32, c->stream);
      CK(cudaMemsetAsync(c->znorm, 0, sizeof(double), c->stream));
      const int nf = rks::launch_df_small(0, d, c->zscale, 1, 0, c->s_raw, c->z_raw, c->S, c->S2, c->colscale,
                                          c->rprev, c->coef, m + 1, c->znorm, c->nrs, c->sj, c->lsr1, c->M2, c->m + 1,
                                          c->part_z, c->part_s, c->tiles.G, c->flag, c->bar, c->stream, c->opts.debug_stall);
      prof_end(c, ps, RKS_K_OTHER, (src == c->tmp64 && !start ? 3 : 2) + nf, 0.0, 0.0);
    }
  } else {
    if (c->u1) CK(cudaMemcpyAsync(c->U, c->u1, c->n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    else rks::launch_start_vector(c->n, c->seed + 1, c->U, c->stream);
    rks::launch_sketch_vec(c->n, c->U, 1.0, d, c->zeta, c->seed, c->s_raw, c->flag, c->stream);
    rks::launch_start_finish(d, c->zscale, c->s_raw, c->S, c->colscale, c->flag, c->stream);
    prof_end(c, ps, RKS_K_OTHER, c->u1 ? 2 : 3, 0.0, 0.0);
  }
  return launch_err();
}

// Algorithm 1 from the start vector `start` (NULL: the user's u1 or the
// library's generator) until the estimates reach c->tol (with the FP64
// verification when verify > 0), `limit` restarts, or stagnation (if
// stall > 0: no decrease of the largest estimate over `stall` restarts).
// Sets *converged; leaves the Ritz pairs of the last contraction in c.
static int run_alg1(rks_ctx* c, const double* start, int limit, double verify, int stall, bool* converged,
                    bool resume = false) {
  const int m = c->m, d = c->d;
  *converged = false;
  int rc = RKS_OK;
  if (resume) {                        // from the decomposition in c (the mixed path's hand-over)
    CK(cudaMemsetAsync(c->flag, 0, 4 * sizeof(int), c->stream));
    CK(cudaMemsetAsync(c->z_raw, 0, d * sizeof(double), c->stream));
    CK(cudaMemsetAsync(c->s_raw, 0, d * sizeof(double), c->stream));
  } else {
    rc = start_alg1(c, start);
    if (rc) return rc;
  }
  rc = expand(c);                      // Algorithm 1, initial expansion to m
  if (rc) return rc;
  if (c->opts.max_restarts < 0) { c->solved = true; return RKS_OK; }
  int done = 0;
  double best = 1e300;
  int since_best = 0, q_seen = c->q;
  while (true) {
    auto h0 = std::chrono::steady_clock::now();
    rc = contract(c);                  // Schur, reorder, truncate, whiten, lock, restart
    if (rc) return rc;
    ++c->restarts;
    ++done;
    ritz(c);
    c->stats.host_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - h0).count();
    rc = upload_restart(c);            // pending rotation, scales, sketches, Gram matrix
    if (rc) return rc;
    double mx = 0.0;
    for (int t = 0; t < c->nw; ++t) mx = std::max(mx, c->est[t]);
    c->hist.push_back(mx);
    c->hist_lock.push_back(c->q);
    if (mx <= c->tol) {
      *converged = true;
      if (verify > 0) {                // FP64 verification of the true residuals
        rc = finalize(c);
        if (rc) return rc;
        double mr = 0.0;
        for (double v : c->resid) mr = std::max(mr, v);
        if (mr > verify && c->q < c->k && done < limit) {   // locked vectors are final
          c->tol *= 0.25;
          c->eta_lock *= 0.25;
          *converged = false;
          rc = expand(c);
          if (rc) return rc;
          continue;
        }
        if (mr > verify) *converged = false;
      }
      return RKS_OK;
    }
    // stagnation: no halving of the largest estimate over `stall` restarts,
    // counted afresh when vectors lock (the next wanted pair enters the set)
    if (c->q > q_seen) { q_seen = c->q; best = mx; since_best = 0; }
    else if (mx < 0.5 * best) { best = mx; since_best = 0; }
    else if (++since_best >= stall && stall > 0) return RKS_OK;
    if (done >= limit) return RKS_OK;
    rc = expand(c);                    // Algorithm 2 from k to m
    if (rc) return rc;
  }
}

static int solve_impl(rks_ctx* c) {
  c->solved = false;
  c->nmatvec = 0; c->restarts = 0;
  std::memset(&c->stats, 0, sizeof(c->stats));
  c->evused = 0;
  c->hist.clear();
  c->hist_lock.clear();
  c->rq_re.clear();
  c->rq_im.clear();
  const int limit = c->opts.max_restarts > 0 ? std::min(c->opts.maxit, c->opts.max_restarts) : c->opts.maxit;
  const double tol0 = c->tol, eta0 = c->eta_lock;
  bool converged = false, fp32_done = false;
  int rc = RKS_OK;
  if (c->prec == RKS_PREC_MIXED) {
    // Phase 1: FP32 basis and values (compensated arithmetic), down to the
    // FP32 floor or until the estimates stagnate.  With a thick restart
    // (keep > 0) phase 2 continues from this phase's decomposition, so there
    // is no locking here: a locked vector's dropped residual would stay in
    // the decomposition that phase 2 continues from.  With keep = 0 (the
    // truncation of Algorithm 1) this phase locks and phase 2 starts afresh.
    c->f32 = true;
    c->Ub = c->Uf;
    c->A2.vals = c->valsf;
    c->A2.evals = c->ell_valf;
    if (c->dia_d) c->A2.dvals = c->dia_valf;
    c->A2.f32 = true;
    const int lock0 = c->opts.lock, aggr0 = c->opts.aggressive;
    const bool carry = c->opts.keep > 0 && c->opts.ortho == RKS_ORTHO_SKETCH;
    // target of this phase: 32 u_32 when phase 2 continues from it (every
    // FP32 restart counts), 64 u_32 (just above the FP32 floor) otherwise
    const double floor32 = c->opts.mixed_tol > 0 ? c->opts.mixed_tol
                                                 : (carry ? 32.0 : 64.0) * 5.9604644775390625e-08;
    c->tol = std::max(tol0, floor32);
    c->eta_lock = std::max(eta0, 0.5 * floor32);
    if (carry) {
      c->opts.lock = 0;
      c->opts.aggressive = 0;
    }
    bool conv1 = false;
    // (with the hand-over every FP32 restart counts toward the double-float
    // phase, so a long stagnation window: 40 restarts)
    rc = run_alg1(c, nullptr, limit, 0.0, carry ? 40 : 20, &conv1);
    c->opts.lock = lock0;
    c->opts.aggressive = aggr0;
    c->phase_restarts = c->restarts;
    c->stats.fp32_restarts = c->restarts;
    const int kk32 = c->kk;
    // The FP32 result may already meet the target: its Ritz vectors checked
    // in FP64 (finalize promotes the FP32 basis exactly); then no
    // double-float phase is needed.
    const bool near = c->opts.conv != RKS_CONV_NORM1 || c->hist.empty() || c->hist.back() <= c->opts.verify;
    if (rc == RKS_OK && c->opts.max_restarts >= 0 && c->opts.verify > 0 && c->kk > 0 && near) {
      rc = finalize(c);
      if (rc == RKS_OK) {
        double mr = 0.0;
        for (double v : c->resid) mr = std::max(mr, v);
        fp32_done = mr <= c->opts.verify;
      }
    }
    c->tol = tol0;
    c->eta_lock = eta0;
    if (fp32_done) {
      converged = true;
    } else if (rc == RKS_OK && c->opts.max_restarts >= 0) {
      // Phase 2: double-float, continuing from the FP32 decomposition made
      // exact (handover_df); if that is not possible or does not converge,
      // from the sum of the FP32 Schur vectors (all wanted directions to
      // FP32 accuracy), verified in FP64 either way.
      // The relation error left must be below what the target asks of the
      // residuals (on the ||A||_1 scale): the estimate tolerance, or with
      // the FP64 check what the verified bound leaves above it; on the
      // |lambda| scale, tol times the smallest wanted |lambda|.
      double thr = tol0;
      if (c->opts.conv == RKS_CONV_NORM1) {
        if (c->opts.verify > 0) thr = std::max(tol0, c->opts.verify - tol0);
      } else {
        double lmin = 1e300;
        for (int t = 0; t < c->nw; ++t) lmin = std::min(lmin, std::hypot(c->lre[t], c->lim[t]));
        thr = c->nw > 0 ? tol0 * lmin / c->norm1 : 0.0;
      }
      double rel = 0.0;
      const int h = carry ? handover_df(c, thr, &rel) : RKS_EINVAL;
      c->stats.handover_rel = carry ? rel : 0.0;
      const bool cont = h == RKS_OK;
      if (cont) {
        c->stats.mixed_phase2 = 1;
        rc = run_alg1(c, nullptr, std::max(1, limit - c->restarts), c->opts.verify, 60, &converged, true);
      } else if (h != RKS_EINVAL && h != RKS_EDENSE && h != RKS_ENOMEM) {
        rc = h;                          // a CUDA error; the others fall back below
      }
      // a fresh double-float phase: without the hand-over (at least one
      // restart, as a partial result must be a double-float decomposition),
      // or after a continuation that stagnated before the limit
      if (rc == RKS_OK && !converged && (!cont || c->restarts < limit)) {
        c->stats.mixed_phase2 = 2;
        c->tol = tol0;
        c->eta_lock = eta0;
        rks::launch_sum_cols_f32(c->n, c->Uf, c->ldu, kk32, c->tmp64, c->stream);
        rc = launch_err();
        c->f32 = false;
        c->Ub = c->U2;
        c->A2.vals = c->vals2;
        c->A2.evals = c->ell_val2;
        if (c->dia_d) c->A2.dvals = c->dia_val2;
        c->A2.f32 = false;
        if (rc == RKS_OK)
          rc = run_alg1(c, c->tmp64, std::max(1, limit - c->restarts), c->opts.verify, 0, &converged);
      }
    }
  } else {
    rc = run_alg1(c, nullptr, limit, c->opts.verify, 0, &converged);
  }
  c->tol = tol0;
  c->eta_lock = eta0;
  if (rc) return rc;
  if (c->opts.max_restarts < 0) { c->solved = true; return RKS_OK; }
  if (!fp32_done) {
    rc = finalize(c);
    if (rc) return rc;
  }
  c->solved = true;
  if (converged && c->opts.verify > 0) {
    double mr = 0.0;
    for (double v : c->resid) mr = std::max(mr, v);
    if (mr > c->opts.verify) converged = false;
  }
  return converged ? RKS_OK : RKS_ENOCONV;
}

int rks_solve(rks_ctx* c, rks_info* info) {
  if (!c) return RKS_EINVAL;
  cudaEventRecord(c->ev0, c->stream);
  int rc = solve_impl(c);
  cudaEventRecord(c->ev1, c->stream);
  cudaEventSynchronize(c->ev1);
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->nlocked = c->q;
    info->restarts = c->restarts;
    info->nmatvec = c->nmatvec;
    double me = 0.0, mr = 0.0;
    int nc = 0;
    for (size_t i = 0; i < (size_t)c->nw && i < c->est.size() && c->restarts > 0; ++i) {
      me = std::max(me, c->est[i]);
      if (c->est[i] <= c->tol) ++nc;
    }
    for (double v : c->resid) mr = std::max(mr, v);
    info->nconv = nc;
    info->max_est = me;
    info->max_resid = mr;
    info->converged = (rc == RKS_OK && c->restarts > 0) ? 1 : 0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    info->t_solve_ms = ms;
  }
  return rc;
}

int rks_spmv_format(const rks_ctx* c) {
  if (!c) return RKS_EINVAL;
  return c->prec == RKS_PREC_FP64 ? RKS_SPMV_CSR : c->A2.fmt;
}

int rks_nkept(const rks_ctx* c) { return c ? c->kk : 0; }

int rks_nwanted(const rks_ctx* c) { return c ? c->nw : 0; }

int rks_get_history(const rks_ctx* c, double* hist, int* nlock, int cap) {
  if (!c || cap < 0) return RKS_EINVAL;
  int nh = std::min((int)c->hist.size(), cap);
  for (int i = 0; i < nh; ++i) {
    if (hist) hist[i] = c->hist[i];
    if (nlock) nlock[i] = c->hist_lock[i];
  }
  return nh;
}

int rks_get_stats(const rks_ctx* c, rks_stats* out) {
  if (!c || !out) return RKS_EINVAL;
  *out = c->stats;
  return RKS_OK;
}
double rks_norm1(const rks_ctx* c) { return c ? c->norm1 : 0.0; }

int rks_get_schur(rks_ctx* c, double* T, double* U, double* b) {
  if (!c) return RKS_EINVAL;
  if (!c->solved || c->kk == 0) return RKS_ESTATE;
  const int kk = c->kk;
  if (T) std::memcpy(T, c->Tfull.data(), sizeof(double) * kk * kk);
  if (b) std::memcpy(b, c->bfull.data(), sizeof(double) * kk);
  if (U) {
    const double* src = c->U;
    if (c->prec != RKS_PREC_FP64) {
      rks::launch_df2d_cols(c->n, c->Ub, c->ldu, c->AX, c->ldu, kk, c->f32, c->stream);
      src = c->AX;
    }
    CK(cudaMemcpy2DAsync(U, c->n * sizeof(double), src, c->ldu * sizeof(double), c->n * sizeof(double), kk,
                         c->opts.mem_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return RKS_OK;
}

int rks_get_rayleigh(rks_ctx* c, double* rq_re, double* rq_im) {
  if (!c) return RKS_EINVAL;
  if (!c->solved || c->kk == 0 || c->rq_re.size() != (size_t)c->nw) return RKS_ESTATE;
  if (rq_re) std::memcpy(rq_re, c->rq_re.data(), sizeof(double) * c->nw);
  if (rq_im) std::memcpy(rq_im, c->rq_im.data(), sizeof(double) * c->nw);
  return RKS_OK;
}

int rks_get_eigpairs(rks_ctx* c, double* lam_re, double* lam_im, double* X, double* resid) {
  if (!c) return RKS_EINVAL;
  if (!c->solved || c->kk == 0) return RKS_ESTATE;
  const int nw = c->nw;
  if (lam_re) std::memcpy(lam_re, c->lre.data(), sizeof(double) * nw);
  if (lam_im) std::memcpy(lam_im, c->lim.data(), sizeof(double) * nw);
  if (resid) std::memcpy(resid, c->resid.data(), sizeof(double) * nw);
  if (X) {
    CK(cudaMemcpy2DAsync(X, c->n * sizeof(double), c->X, c->ldu * sizeof(double), c->n * sizeof(double), nw,
                         c->opts.mem_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return RKS_OK;
}

int rks_get_estimates(rks_ctx* c, double* est) {
  if (!c || !est) return RKS_EINVAL;
  if (!c->solved || c->kk == 0) return RKS_ESTATE;
  std::memcpy(est, c->est.data(), sizeof(double) * c->nw);
  return RKS_OK;
}

int rks_get_krylov(rks_ctx* c, int* ncols_out, double* U, double* S, double* H) {
  if (!c) return RKS_EINVAL;
  if (!c->solved) return RKS_ESTATE;
  const int nc = c->q + c->ja + 1;
  if (ncols_out) *ncols_out = nc;
  if (U && c->prec != RKS_PREC_FP64 && !c->f32) {
    std::vector<float2> tmp((size_t)c->n * nc);
    CK(cudaMemcpy2DAsync(tmp.data(), c->n * sizeof(float2), c->U2, c->ldu * sizeof(float2), c->n * sizeof(float2), nc,
                         cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (size_t t = 0; t < tmp.size(); ++t) U[t] = (double)tmp[t].x + (double)tmp[t].y;
  } else if (U && c->f32) {
    std::vector<float> tmp((size_t)c->n * nc);
    CK(cudaMemcpy2DAsync(tmp.data(), c->n * sizeof(float), c->Uf, c->ldu * sizeof(float), c->n * sizeof(float), nc,
                         cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (size_t t = 0; t < tmp.size(); ++t) U[t] = (double)tmp[t];
  } else if (U) {
    CK(cudaMemcpy2DAsync(U, c->n * sizeof(double), c->U, c->ldu * sizeof(double), c->n * sizeof(double), nc,
                         cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  if (U) {
    for (int j = 0; j < nc; ++j) {
      double s = c->cs_h[j];
      double* col = U + (size_t)j * c->n;
      for (int64_t i = 0; i < c->n; ++i) col[i] *= s;
    }
  }
  if (S) std::memcpy(S, c->S_h.data(), sizeof(double) * (size_t)c->d * nc);
  if (H) {
    std::memset(H, 0, sizeof(double) * (size_t)nc * (nc - 1));
    for (int j = c->last_expand_from; j < nc - 1; ++j)
      for (int i = 0; i <= j + 1; ++i) H[i + (size_t)j * nc] = c->coef_h[i + (size_t)j * (c->m + 1)];
  }
  return RKS_OK;
}

void rks_destroy(rks_ctx* c) { free_ctx(c); }

int rks_host_ordered_schur(int m, const double* B, int which, int nsort, double* T, double* Q) {
  if (m <= 0 || !B || !T || !Q || which < 0 || which > 3) return RKS_EINVAL;
  std::memcpy(T, B, sizeof(double) * (size_t)m * m);
  rks_dense::hessenberg(m, T, m, Q, m);
  if (rks_dense::schur(m, T, m, Q, m) != 0) return RKS_EDENSE;
  rks_dense::reorder(m, T, m, Q, m, m, which, std::min(std::max(nsort, 0), m));
  return RKS_OK;
}

int rks_host_reorder_select(int n, double* T, const int* select, double* Z) {
  if (n < 1 || !T || !select || !Z) return RKS_EINVAL;
  const auto bl = rks_dense::blocks(n, T, n);
  std::vector<char> sel(bl.size());
  for (size_t t = 0; t < bl.size(); ++t) sel[t] = select[bl[t].start] != 0;
  return rks_dense::reorder_select(n, T, n, Z, n, n, sel) == 0 ? RKS_OK : RKS_EDENSE;
}

int rks_host_sketch_reorthonormalize(int d, int ka, double* S, const double* T, const double* b, double* Rinv,
                                     double* Tn, double* bn) {
  if (d < 1 || ka < 1 || ka + 1 > d || !S || !T || !b || !Rinv || !Tn || !bn) return RKS_EINVAL;
  return rks_dense::sketch_reorthonormalize(d, ka, S, T, b, Rinv, Tn, bn) == 0 ? RKS_OK : RKS_EDENSE;
}

int rks_host_quasi_eig(int n, const double* T, double* lam_re, double* lam_im, double* Y_re, double* Y_im) {
  if (n <= 0 || !T || !lam_re || !lam_im) return RKS_EINVAL;
  std::vector<cd> Y((size_t)n * n);
  rks_dense::quasi_eig(n, T, n, lam_re, lam_im, Y.data(), n);
  for (size_t i = 0; i < Y.size(); ++i) {
    if (Y_re) Y_re[i] = Y[i].real();
    if (Y_im) Y_im[i] = Y[i].imag();
  }
  return RKS_OK;
}

int rks_sketch_pairs(int64_t n, int d, int zeta, uint64_t seed, int32_t* rows, int8_t* signs, void* stream) {
  if (n <= 0 || zeta < 1 || zeta > 16 || d < 2 * zeta || !rows || !signs) return RKS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int* flag = nullptr;
  int rc = dalloc(&flag, 1);
  if (rc) return rc;
  cudaMemsetAsync(flag, 0, sizeof(int), st);
  rks::launch_sketch_pairs(n, d, zeta, seed, rows, signs, flag, st);
  int f = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&f, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(flag);
  if (e != cudaSuccess) return RKS_ECUDA;
  return f ? RKS_EINVAL : RKS_OK;
}

int rks_basis_product_f32(int64_t n, const float* U, int64_t ldu, int nin, const double* Q, int nout, float* out,
                          void* stream) {
  if (n <= 0 || ldu < n || !U || !Q || !out || !rks::tc_restart_supported(nin, nout)) return RKS_EINVAL;
  if (rks::configure_tc_kernels() != cudaSuccess) return RKS_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<uint16_t> img;
  rks::tc_restart_bimage(nin, nout, Q, img);
  void* dimg = nullptr;
  int* flag = nullptr;
  if (cudaMalloc(&dimg, img.size() * sizeof(uint16_t)) != cudaSuccess) return RKS_ENOMEM;
  if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) { cudaFree(dimg); return RKS_ENOMEM; }
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dimg, img.data(), img.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    rks::launch_tc_restart_f32(n, U, out, ldu, nin, nout, dimg, nullptr, nullptr, flag, st);
    e = cudaGetLastError();
  }
  int f = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&f, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dimg);
  cudaFree(flag);
  if (e != cudaSuccess) return RKS_ECUDA;
  return (f & rks::RKS_FLAG_TIMEOUT) ? RKS_ETIMEOUT : RKS_OK;
}

int rks_basis_product_df(int64_t n, const double* U, int64_t ldu, int nin, const double* Q, int nout, double* out,
                         void* stream) {
  if (n <= 0 || ldu < n || !U || !Q || !out || !rks::tc_restart_df_supported(nin, nout)) return RKS_EINVAL;
  if (rks::configure_tc_kernels() != cudaSuccess) return RKS_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<uint16_t> img;
  std::vector<int> fexp;
  rks::tc_restart_df_bimage(nin, nout, Q, img, fexp);
  float2 *Ud = nullptr, *Od = nullptr;
  void* dimg = nullptr;
  int *dfexp = nullptr, *flag = nullptr, *pexp = nullptr, *rexp = nullptr;
  int rc = RKS_OK;
  if (cudaMalloc(&Ud, (size_t)ldu * nin * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&Od, (size_t)ldu * nout * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&dimg, img.size() * sizeof(uint16_t)) != cudaSuccess ||
      cudaMalloc(&dfexp, fexp.size() * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&pexp, (size_t)nin * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&rexp, (size_t)n * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&flag, sizeof(int)) != cudaSuccess)
    rc = RKS_ENOMEM;
  int f = 0;
  if (rc == RKS_OK) {
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(pexp, 0, (size_t)nin * sizeof(int), st);   // unscaled columns
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dimg, img.data(), img.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dfexp, fexp.data(), fexp.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      rks::launch_d2df((int64_t)ldu * nin, U, Ud, false, st);   // the basis as double-float pairs
      rks::launch_tc_restart_df(n, Ud, Od, ldu, nin, nout, dimg, dfexp, pexp, rexp, nullptr, nullptr, flag, st);
      rks::launch_df2d_cols(n, Od, ldu, out, ldu, nout, false, st);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&f, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = RKS_ECUDA;
  }
  cudaFree(Ud); cudaFree(Od); cudaFree(dimg); cudaFree(dfexp); cudaFree(pexp); cudaFree(rexp); cudaFree(flag);
  if (rc != RKS_OK) return rc;
  return (f & rks::RKS_FLAG_TIMEOUT) ? RKS_ETIMEOUT : RKS_OK;
}

int rks_sketch_apply(int64_t n, int d, int zeta, uint64_t seed, const double* x, double* z, void* stream) {
  if (n <= 0 || zeta < 1 || zeta > 16 || d < 2 * zeta || d > 8192 || !x || !z) return RKS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (rks::configure_kernels() != cudaSuccess) return RKS_ECUDA;
  int* flag = nullptr;
  int rc = dalloc(&flag, 1);
  if (rc) return rc;
  cudaMemsetAsync(flag, 0, sizeof(int), st);
  cudaMemsetAsync(z, 0, d * sizeof(double), st);
  rks::launch_sketch_vec(n, x, 1.0, d, zeta, seed, z, flag, st);
  // the kernel sums sign * x_i; the 1/sqrt(zeta) scale is applied here
  std::vector<double> h(d);
  int f = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), z, d * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&f, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    const double sc = 1.0 / std::sqrt((double)zeta);
    for (double& v : h) v *= sc;
    e = cudaMemcpyAsync(z, h.data(), d * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(flag);
  if (e != cudaSuccess) return RKS_ECUDA;
  return f ? RKS_EINVAL : RKS_OK;
}

}  // extern "C"
