// Internal declarations of librks (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace rks {

enum : int { RKS_FLAG_NAN = 1, RKS_FLAG_BREAKDOWN = 2, RKS_FLAG_HASH = 4, RKS_FLAG_TIMEOUT = 8 };

// CTAs of the kernels that carry a sketch (FP64 path: one shared-memory bin
// set each, folded with one atomic per bin; DF path: one row range each).
constexpr int kSketchCtas = 152 * 2;
// CTAs of the double-float streaming kernels (512 threads each).
constexpr int kDfCtas = 152 * 2;
// CTAs of the final residual sums (partials added on the host in CTA order).
constexpr int kResidCtas = 152 * 2;
// Update kernel: columns loaded per batch and resident CTAs per SM it is
// compiled for (register budget 65536 / (512 * kDfUpdMinBlocks) per thread).
constexpr int kDfUpdUnroll = 10;
constexpr int kDfUpdMinBlocks = 2;

// Deterministic sketch accumulation: per-tile bin lists of Omega (built once
// by build_sketch_tiles; layout in kernels_df.cu).  Device arrays:
//   row[ntile + 1]          first row of each tile (row[ntile] = n)
//   ctile[G + 1]            CTA g owns tiles ctile[g] .. ctile[g + 1] - 1
//   meta[ntile * d]         per tile and position: sketch row | count << 16
//   off[ntile * (L + 1)]    per tile: slot offsets of its entries
//   ent[n * zeta]           tile t's entries at row[t] * zeta .. row[t + 1] * zeta
// The sketch kernels run G CTAs and write G x d partial sums (FP64), which
// are added in CTA order.
constexpr int kTileRows = 1024;
struct SketchTiles {
  int64_t n = 0;
  int d = 0, zeta = 0, G = 0, ntile = 0, L = 0, H = 1;   // L: largest list; H: threads per list
  int64_t* row = nullptr;
  int* ctile = nullptr;
  uint32_t* meta = nullptr;
  int* off = nullptr;
  uint16_t* ent = nullptr;
};

struct Csr {
  int64_t n = 0, nnz = 0;
  const int32_t* rowptr = nullptr;
  const int32_t* colind = nullptr;
  const double* vals = nullptr;
};

struct CsrDF {
  int64_t n = 0, nnz = 0;
  const int32_t* rowptr = nullptr;
  const int32_t* colind = nullptr;
  const void* vals = nullptr;   // float2 pairs, or float when f32
  bool f32 = false;             // FP32 values and FP32 basis (mixed precision)
  // The same matrix as ELLPACK interleaved by 32-row slices (optional): row i
  // has its W slots at ((i / 32) * W + e) * 32 + i % 32, e < W, in CSR order,
  // padded with column -1.  Used by the SpMV when set.
  int W = 0;
  const int32_t* ecol = nullptr;
  const void* evals = nullptr;  // float2 pairs, or float when f32
  // The same matrix by diagonals (optional; used first when set): D <= 16
  // offsets doff[e] = column - row, increasing; row i's entry on diagonal e
  // at dvals[e * ldd + i], zero where A has none.  In increasing column
  // order, as a CSR row with sorted columns.
  int D = 0;
  int doff[16] = {};
  int64_t ldd = 0;
  const void* dvals = nullptr;  // float2 pairs, or float when f32
  // FP32 copy of the diagonals for double-float vectors (optional, D <= 8):
  // set when every value of A is an FP32 number, so that the pairs' low
  // words are zero and the products are the same bits
  const void* dvals_f32 = nullptr;
  // Irregular rows (CSR only; see rks_spmv_format): kSpmvWarp takes a row
  // per warp inside the sketch tiles; kSpmvMerge splits rows + entries evenly
  // over threads (merge path), then folds the partial rows and sketches w.
  int fmt = 0;
  int64_t* mp_part = nullptr;   // merge path: first row of every CTA's range
  int* mp_row = nullptr;        // merge path: carry row of every thread (-1: none)
  float2* mp_val = nullptr;     // its partial sum (double-float)
  float2* mp_w = nullptr;       // double-float result before rounding to FP32 (f32 only)
  int64_t mp_threads = 0;
};

// SpMV formats (CsrDF::fmt, rks_spmv_format)
enum { kSpmvCsr = 0, kSpmvEll = 1, kSpmvDia = 2, kSpmvWarp = 3, kSpmvMerge = 4 };
constexpr int kMergeItems = 12;  // rows + entries per thread of the merge-path SpMV
constexpr int kMergeCta = 256;   // threads per CTA of the merge path (a CTA stages 12 x 256 items)

// Diagonal copy of a CSR matrix (see CsrDF); dvals (D * ldd values) is
// cleared first.
void launch_merge_partition(const CsrDF& A, cudaStream_t st);
void launch_dia_fill(int64_t n, int D, const int* doff, int64_t ldd, const int32_t* rowptr, const int32_t* colind,
                     const void* vals, bool f32, void* dvals, cudaStream_t st);

// ELLPACK copy of a CSR matrix (see CsrDF): ecol and evals hold
// ceil(n / 32) * 32 * W slots; vals are float2 pairs or float (f32).
void launch_ell_fill(int64_t n, int W, const int32_t* rowptr, const int32_t* colind, const void* vals, bool f32,
                     int32_t* ecol, void* evals, cudaStream_t st);

cudaError_t configure_df_kernels();
int df_small_smem(int d, int c);
int df_gemm_smem(int nin, int nout);
void launch_df_spmv_sketch(const CsrDF& A, const void* x, void* w, const SketchTiles& t, double* part,
                           cudaStream_t st);
void launch_df_update_sketch(void* U, int64_t ldu, int c, const float2* nrs, const float2* sj, const SketchTiles& t,
                             double* part, bool f32, cudaStream_t st);
int launch_df_small(int j, int d, double zscale, int finish, int ls, double* s_raw, double* z_raw, double* S64,
                    float2* S2, double* colscale, double* rprev, double* coef, int ldcoef, double* znorm_prev,
                    float2* nrs, float2* sj, float2* r1, float2* M2, int ldm, const double* part_z,
                    const double* part_s, int G, int* flag, unsigned* bar, cudaStream_t st, int stall = 0);
// Krylov-Schur baseline with Euclidean CGS2 (no sketch), DF basis.
void launch_df_spmv(const CsrDF& A, const void* x, void* w, const SketchTiles& t, cudaStream_t st);
void launch_df_update_plain(void* U, int64_t ldu, int c, const float2* nrs, const float2* sj, const SketchTiles& t,
                            double* norm_part, cudaStream_t st);
void launch_df_dots(const void* U, int64_t ldu, int c, int cv, const SketchTiles& t, double* part, cudaStream_t st);
// out[r] = sum over g < G of part[g * d + r] in a fixed order (r < d)
void launch_df_fold(const double* part, int d, int G, double* out, cudaStream_t st);
// U[:, c0 + l] -= coef[l] * U[:, src], l < ncols (double-float columns, coef device)
void launch_df_axpy_cols(int64_t n, float2* U, int64_t ldu, int src, int c0, int ncols, const float2* coef,
                         cudaStream_t st);
void launch_ks_coef(int pass, int j, int c, int G, const double* part, const double* colscale, double* rprev,
                    float2* nrs, float2* sj, cudaStream_t st);
void launch_ks_finish(int j, int G, const double* part, double thr, double* colscale,
                      const double* rprev, double* coef, int ldcoef, int* flag, cudaStream_t st);
int build_sketch_tiles(int64_t n, int d, int zeta, const uint16_t* otab, SketchTiles* out, cudaStream_t st);
void free_sketch_tiles(SketchTiles* t);
size_t sketch_tile_smem(const SketchTiles& t, int c);
void launch_omega_table(int64_t n, int d, int zeta, uint64_t seed, uint16_t* tab, int* flag, cudaStream_t st);
int omega_slots(int zeta);
void launch_d2df(int64_t n, const double* x, void* y, bool f32, cudaStream_t st);
void launch_sum_cols_f32(int64_t n, const float* U, int64_t ldu, int ncols, double* y, cudaStream_t st);
void launch_df2d_cols(int64_t n, const void* x, int64_t ldx, double* y, int64_t ldy, int ncols, bool f32,
                      cudaStream_t st);
void launch_df_sketch_vec(const void* x, const SketchTiles& t, double* part, bool f32, cudaStream_t st);
void launch_df_rows_gemm(int64_t n, void* U, int64_t ldu, int a0, int nin, const float2* Q, int nout, int c0,
                         int move_src, bool f32, cudaStream_t st);
// Hand-over of the mixed path's FP32 decomposition to double-float
// (kernels_df.cu): exact promotion of FP32 columns, the relation error
// e = w - v - beta u rounded to FP32, 1 / a_ii, damped Jacobi sweeps on
// A X - X T = -E (Y = X T given; with part, the per-CTA sums of the squared
// residual per column, jacobi_sweep_ctas(n) x kk), and U2 += X.
void launch_f32_to_df_cols(int64_t n, const float* Uf, int64_t ldu, int ncols, float2* U2, cudaStream_t st);
void launch_relation_resid(int64_t n, const float2* w, const float2* v, const float2* u, double beta, float* e,
                           cudaStream_t st);
void launch_diag_inv(int64_t n, const int32_t* rowptr, const int32_t* colind, const float* vals, float* dinv,
                     cudaStream_t st);
int jacobi_sweep_ctas(int64_t n);
void launch_jacobi_sweep(int64_t n, const int32_t* rowptr, const int32_t* colind, const float* vals,
                         const float* dinv, int kk, int64_t ld, const float* X, const float* E, const float* Y,
                         float omega, float* Xn, double* part, cudaStream_t st);
void launch_df_add_f32_cols(int64_t n, float2* U2, int64_t ldu, int kk, const float* X, int64_t ldx,
                            cudaStream_t st);

// Tensor-core restart product for an FP32 basis (restart_tc.cu):
// out[:, o] = sum_l in[:, l] Q[l, o], in place allowed, then mvdst = mvsrc.
bool tc_restart_supported(int nin, int nout);
size_t tc_restart_smem(int nin, int nout);
void tc_restart_bimage(int nin, int nout, const double* Q, std::vector<uint16_t>& img);
cudaError_t configure_tc_kernels();
void launch_tc_restart_f32(int64_t n, const float* in, float* out, int64_t ldu, int nin, int nout, const void* bimg,
                           const float* mvsrc, float* mvdst, int* flag, cudaStream_t st);
constexpr size_t kTcImageBytes = (size_t)3 * 256 * 64 * 2;   // largest split image of Q'
// Double-float basis: exact digit products on the tensor cores (restart_tc.cu).
constexpr size_t kTcDfSmemMax = 227 * 1024;
constexpr size_t kTcDfImageBytes = (size_t)8 * 256 * 64 * 2;  // largest digit image of Q'
bool tc_restart_df_supported(int nin, int nout);
size_t tc_restart_df_smem(int nin, int nout);
void tc_restart_df_bimage(int nin, int nout, const double* Q, std::vector<uint16_t>& img, std::vector<int>& fexp);
// out = in diag(2^pexp) Q (pexp: nin device ints, the input columns'
// power-of-two scales; rexp: n device ints of scratch).
void launch_tc_restart_df(int64_t n, const float2* in, float2* out, int64_t ldu, int nin, int nout, const void* bimg,
                          const int* fexp, const int* pexp, int* rexp, const float2* mvsrc, float2* mvdst, int* flag,
                          cudaStream_t st);

void launch_sketch_pairs(int64_t n, int d, int zeta, uint64_t seed, int32_t* rows, int8_t* signs, int* flag,
                         cudaStream_t st);
void launch_sketch_vec(int64_t n, const double* x, double xscale, int d, int zeta, uint64_t seed, double* out_raw,
                       int* flag, cudaStream_t st);
void launch_spmv_sketch(const Csr& A, const double* x, const double* xscale, double* w, int d, int zeta,
                        uint64_t seed, double* out_raw, int* flag, cudaStream_t st);
void launch_ls(int c, int d, const double* S, const double* z_raw, double zscale, const double* colscale,
               double* r1, double* z1, double* r, double* rs, cudaStream_t st);
void launch_update_sketch(int64_t n, double* U, int64_t ldu, int c, const double* rs, int d, int zeta,
                          uint64_t seed, double* out_raw, int* flag, cudaStream_t st);
void launch_finish(int c, int d, double zscale, double* s_raw, double* z_raw, double* S, double* colscale,
                   const double* r, double* coef, int ldcoef, int* flag, cudaStream_t st);
void launch_start_finish(int d, double zscale, double* s_raw, double* S, double* colscale, int* flag,
                         cudaStream_t st);
void launch_start_vector(int64_t n, uint64_t seed, double* x, cudaStream_t st);
cudaError_t configure_kernels();
// Run f() once per CUDA device (the device current at the call), safe to call
// from several host threads: slot names the configuration; a failure is
// returned and f() retried at the next call.  The record is per process and
// is not reset by cudaDeviceReset.
enum { kCfgBase = 0, kCfgDf = 1, kCfgTc = 2, kCfgWs = 3, kCfgSlots = 4 };
cudaError_t once_per_device(int slot, cudaError_t (*f)());
int rows_gemm_smem(int nin, int nout, int threads);
void launch_rows_gemm(int64_t n, const double* A, int64_t lda, int a0, int nin, const double* B, int nout,
                      double* C, int64_t ldc, int c0, int move_src, cudaStream_t st);
void launch_spmm(const Csr& A, const double* X, int64_t ldx, double* Y, int64_t ldy, int ncols, cudaStream_t st);
// Writes per-CTA partial sums out[(pair * 4 + q) * G + cta]; returns G (<= kResidCtas).
int launch_resid_sums(int64_t n, const double* X, const double* AX, int64_t ld, int npairs, const int* col,
                      const int* colim, const double* lre, const double* lim, double* out, cudaStream_t st);
void launch_f32_to_f64(int64_t n, const float* a, double* b, cudaStream_t st);
void launch_check_csr(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colind, int* bad,
                      cudaStream_t st);

}  // namespace rks
