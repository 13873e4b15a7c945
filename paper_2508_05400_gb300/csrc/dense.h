// Small dense FP64 routines of the rKS contraction step (host side).
// Column-major storage; see dense.cpp for the methods.
#pragma once
#include <complex>
#include <vector>

namespace rks_dense {

struct Block { int start, size; double re, im; };   // im >= 0 for a 2x2 pair

// A (n x n) <- Q^T A Q upper Hessenberg; Q (n x n) is overwritten with Q.
void hessenberg(int n, double* A, int lda, double* Q, int ldq);
// Same result for a matrix that is upper Hessenberg except for row ka, which
// may be full in columns 0..ka-1 (the restarted Rayleigh quotient
// [T_k; b^T] of Algorithm 2 followed by Arnoldi columns): O(ka^3) work.
void hessenberg_arrow(int n, int ka, double* A, int lda, double* Q, int ldq);
// Real Schur form of an upper Hessenberg H (in place), Z <- Z * (QR rotations).
// 2x2 blocks are standardised.  Returns 0, or -1 if the iteration did not converge.
int schur(int n, double* H, int ldh, double* Z, int ldz);
// Standardise the 2x2 diagonal block at i (rotation applied to T and to the
// first nz rows of Z).  Returns the resulting block size at i (1 or 2).
int standardize_2x2(int n, double* T, int ldt, double* Z, int ldz, int nz, int i);
// Diagonal blocks of a quasi-triangular T with their eigenvalues.
std::vector<Block> blocks(int n, const double* T, int ldt);
// Ordering key, smaller = more wanted: which 0 LM, 1 SM, 2 LR, 3 SR.
double key(double re, double im, int which);
// Swap the adjacent diagonal blocks at j (sizes p then q).  0 on success.
int swap_blocks(int n, double* T, int ldt, double* Z, int ldz, int nz, int j, int p, int q);
// Move the best `nsort` blocks (by key) to the top, best first.  Returns the
// number of rejected swaps (0 when the ordering is complete).
int reorder(int n, double* T, int ldt, double* Z, int ldz, int nz, int which, int nsort);
// Move the diagonal blocks flagged in sel (one flag per block, in the order
// of blocks(T)) to the top, keeping the order among the flagged blocks and
// among the others (the ordering of LAPACK's dtrsen).  Z (nz rows) takes the
// rotations.  Returns 0, or -1 (T and Z unchanged) if a swap is refused or
// rounding splits a 2x2 block.
int reorder_select(int n, double* T, int ldt, double* Z, int ldz, int nz, const std::vector<char>& sel);
// Householder QR of the d x ka matrix S (column-major, ld d): R (ka x ka,
// upper triangular, positive diagonal); S is overwritten by the explicit Q.
void house_qr(int d, int ka, double* S, double* R);
// A Krylov-Schur decomposition A U = U T + u b^T (U: ka columns) whose basis
// [U u] has drifted from sketch-orthonormality: S (d x (ka+1), column-major,
// in: [Omega U, Omega u], out: Q) -> R from S = Q R, Rinv = R^-1 ((ka+1)^2),
// and the decomposition of [V v] = [U u] R^-1, A V = V Tn + v bn^T with
// Tn = (R11 T + r12 b^T) R11^-1 and bn^T = r22 b^T R11^-1 (Tn: ka x ka, bn:
// ka).  Returns 0, or -1 if R is singular (outputs undefined).
int sketch_reorthonormalize(int d, int ka, double* S, const double* T, const double* b, double* Rinv, double* Tn,
                            double* bn);
// Eigenvalues and unit 2-norm eigenvectors of a quasi-triangular T; a 2x2
// block at (i, i+1) gives columns i (Im > 0) and i+1 (its conjugate).
int quasi_eig(int n, const double* T, int ldt, double* lam_re, double* lam_im,
              std::complex<double>* Y, int ldy);

}  // namespace rks_dense
