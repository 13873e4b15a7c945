// Small dense FP64 linear algebra for the rKS restart (host side).
//
// The contraction step of Algorithm 1 (Sec. 3.1) needs, on an m x m Rayleigh
// quotient B (m <= a few hundred): the real Schur form B = Q T Q^T (Prop. 2.8),
// a reordering that moves the wanted eigenvalues to the leading diagonal
// blocks, and the eigenvectors of the truncated quasi-triangular T_k for the
// Ritz pairs and the residual estimates |b^T y| / |lambda| (Sec. 4.1).
//
// Methods (textbook, written for this library):
//  * Householder reduction to Hessenberg form, accumulating Q;
//  * implicit double-shift (Francis) QR with deflation and exceptional shifts,
//    applied to the whole matrix so that T is a full real Schur form;
//  * 2x2 blocks standardised by one rotation: equal diagonal and opposite-sign
//    off-diagonals for a complex pair, upper triangular for a real pair;
//  * swapping of adjacent 1x1/2x2 diagonal blocks by the direct method of
//    Bai & Demmel (1993): solve the small Sylvester equation
//    T11 X - X T22 = -T12, take the QR factorisation of [X; I], and apply it
//    as an orthogonal similarity; the swap is rejected if the new
//    sub-diagonal block is not negligible;
//  * eigenvectors of a quasi-triangular matrix by back substitution (complex
//    arithmetic for pairs), each normalised to unit 2-norm.
// Matrices are column-major with explicit leading dimensions.

#include "dense.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

namespace rks_dense {

namespace {

constexpr double kEps = 2.220446049250313e-16;

inline double& at(double* A, int lda, int i, int j) { return A[i + (size_t)j * lda]; }
inline double at(const double* A, int lda, int i, int j) { return A[i + (size_t)j * lda]; }

// Householder vector for x (length len): P = I - beta v v^T, v[0] = 1,
// P x = alpha e_1.  beta = 0 when x is already a multiple of e_1.
void house(const double* x, int len, double* v, double* beta) {
  double s = 0.0;
  for (int i = 1; i < len; ++i) s += x[i] * x[i];
  v[0] = 1.0;
  for (int i = 1; i < len; ++i) v[i] = x[i];
  if (s == 0.0) { *beta = 0.0; return; }
  double nrm = std::sqrt(x[0] * x[0] + s);
  double v0 = x[0] >= 0.0 ? x[0] + nrm : x[0] - nrm;
  for (int i = 1; i < len; ++i) v[i] /= v0;
  double vtv = 1.0;
  for (int i = 1; i < len; ++i) vtv += v[i] * v[i];
  *beta = 2.0 / vtv;
}

// rows r0..r0+len-1 of A, columns c0..c1 (inclusive): A <- (I - beta v v^T) A
void apply_left(double* A, int lda, int r0, int len, int c0, int c1, const double* v, double beta) {
  if (beta == 0.0) return;
  for (int j = c0; j <= c1; ++j) {
    double s = 0.0;
    for (int i = 0; i < len; ++i) s += v[i] * at(A, lda, r0 + i, j);
    s *= beta;
    for (int i = 0; i < len; ++i) at(A, lda, r0 + i, j) -= s * v[i];
  }
}

// columns c0..c0+len-1 of A, rows r0..r1: A <- A (I - beta v v^T).
// Column-major friendly: w = A v by columns, then A -= beta w v^T by columns.
void apply_right(double* A, int lda, int c0, int len, int r0, int r1, const double* v, double beta) {
  if (beta == 0.0 || r1 < r0) return;
  if (len <= 3) {   // short reflectors (QR sweeps): row by row
    for (int i = r0; i <= r1; ++i) {
      double s = 0.0;
      for (int j = 0; j < len; ++j) s += at(A, lda, i, c0 + j) * v[j];
      s *= beta;
      for (int j = 0; j < len; ++j) at(A, lda, i, c0 + j) -= s * v[j];
    }
    return;
  }
  const int nr = r1 - r0 + 1;
  thread_local std::vector<double> w;
  w.assign(nr, 0.0);
  double* wp = w.data();
  for (int j = 0; j < len; ++j) {
    const double vj = v[j];
    const double* col = A + r0 + (size_t)(c0 + j) * lda;
    for (int i = 0; i < nr; ++i) wp[i] += col[i] * vj;
  }
  for (int j = 0; j < len; ++j) {
    const double f = beta * v[j];
    double* col = A + r0 + (size_t)(c0 + j) * lda;
    for (int i = 0; i < nr; ++i) col[i] -= wp[i] * f;
  }
}

// Plane rotation on rows (i, i+1) / columns (i, i+1): new basis columns
// q1 = (cs, sn), q2 = (-sn, cs).  T <- R^T T R over the full matrix, Z <- Z R.
// Only the structurally nonzero part is touched (columns >= i on the left,
// rows <= i+1 on the right), so exact zeros left of / below the block stay zero.
void rotate_pair(int n, double* T, int ldt, double* Z, int ldz, int nz, int i, double cs, double sn) {
  for (int j = i; j < n; ++j) {          // left: R^T
    double a = at(T, ldt, i, j), b = at(T, ldt, i + 1, j);
    at(T, ldt, i, j) = cs * a + sn * b;
    at(T, ldt, i + 1, j) = -sn * a + cs * b;
  }
  for (int r = 0; r <= i + 1; ++r) {     // right: R
    double a = at(T, ldt, r, i), b = at(T, ldt, r, i + 1);
    at(T, ldt, r, i) = cs * a + sn * b;
    at(T, ldt, r, i + 1) = -sn * a + cs * b;
  }
  if (Z) {
    for (int r = 0; r < nz; ++r) {
      double a = at(Z, ldz, r, i), b = at(Z, ldz, r, i + 1);
      at(Z, ldz, r, i) = cs * a + sn * b;
      at(Z, ldz, r, i + 1) = -sn * a + cs * b;
    }
  }
}

}  // namespace

void hessenberg(int n, double* A, int lda, double* Q, int ldq) {
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) at(Q, ldq, i, j) = (i == j) ? 1.0 : 0.0;
  std::vector<double> x(n), v(n);
  for (int k = 0; k + 2 < n; ++k) {
    int len = n - k - 1;
    for (int i = 0; i < len; ++i) x[i] = at(A, lda, k + 1 + i, k);
    double beta;
    house(x.data(), len, v.data(), &beta);
    apply_left(A, lda, k + 1, len, k, n - 1, v.data(), beta);
    apply_right(A, lda, k + 1, len, 0, n - 1, v.data(), beta);
    apply_right(Q, ldq, k + 1, len, 0, n - 1, v.data(), beta);
    for (int i = k + 2; i < n; ++i) at(A, lda, i, k) = 0.0;
  }
}

void hessenberg_arrow(int n, int ka, double* A, int lda, double* Q, int ldq) {
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) at(Q, ldq, i, j) = (i == j) ? 1.0 : 0.0;
  if (ka < 2 || ka >= n) {
    if (ka >= n) hessenberg(n, A, lda, Q, ldq);
    return;
  }
  // Row ka holds b in columns 0..ka-1; rows > ka are zero there.  Reduce from
  // the bottom: for row i = ka, ka-1, ..., 2 zero (i, 0..i-2) with a reflector
  // acting on columns (and, as a similarity, rows) 0..i-1.  Entries of rows
  // > i in those columns are already zero, so they stay zero.
  std::vector<double> x(n), v(n);
  for (int i = ka; i >= 2; --i) {
    const int len = i;              // indices 0..i-1, pivot at i-1
    // reflector on the reversed row segment so that the last entry survives
    for (int t = 0; t < len; ++t) x[t] = at(A, lda, i, len - 1 - t);
    double beta;
    house(x.data(), len, v.data(), &beta);
    if (beta == 0.0) continue;
    std::vector<double> vr(len);
    for (int t = 0; t < len; ++t) vr[t] = v[len - 1 - t];
    // A <- A P on columns 0..len-1 (rows 0..n-1), then A <- P A on rows 0..len-1
    apply_right(A, lda, 0, len, 0, n - 1, vr.data(), beta);
    apply_left(A, lda, 0, len, 0, n - 1, vr.data(), beta);
    apply_right(Q, ldq, 0, len, 0, n - 1, vr.data(), beta);
    for (int t = 0; t < len - 1; ++t) at(A, lda, i, t) = 0.0;
  }
}

int standardize_2x2(int n, double* T, int ldt, double* Z, int ldz, int nz, int i) {
  double a = at(T, ldt, i, i), b = at(T, ldt, i, i + 1);
  double c = at(T, ldt, i + 1, i), d = at(T, ldt, i + 1, i + 1);
  if (c == 0.0) return 1;  // already triangular: two real eigenvalues
  double cs, sn;
  int is_pair;
  if (b == 0.0) {
    cs = 0.0; sn = 1.0; is_pair = 0;
  } else {
    double p = 0.5 * (a - d);
    double disc = p * p + b * c;
    if (disc >= 0.0) {
      // real pair: first basis vector = eigenvector of lambda1
      double z = p + (p >= 0.0 ? 1.0 : -1.0) * std::sqrt(disc);
      double l1 = d + z;
      double v1 = b, v2 = l1 - a;          // from the first row
      double w1 = l1 - d, w2 = c;          // from the second row
      if (std::hypot(w1, w2) > std::hypot(v1, v2)) { v1 = w1; v2 = w2; }
      double nv = std::hypot(v1, v2);
      cs = v1 / nv; sn = v2 / nv; is_pair = 0;
    } else {
      if (a == d && (b + c) == 0.0) return 2;  // already standard
      double th = 0.5 * std::atan2(-(a - d), (b + c));
      cs = std::cos(th); sn = std::sin(th); is_pair = 1;
    }
  }
  rotate_pair(n, T, ldt, Z, ldz, nz, i, cs, sn);
  if (is_pair) {
    double m = 0.5 * (at(T, ldt, i, i) + at(T, ldt, i + 1, i + 1));
    at(T, ldt, i, i) = m;
    at(T, ldt, i + 1, i + 1) = m;
    if (at(T, ldt, i, i + 1) * at(T, ldt, i + 1, i) >= 0.0) {
      // rounding made the pair look real: keep it as a triangular real pair
      at(T, ldt, i + 1, i) = 0.0;
      return 1;
    }
    return 2;
  }
  at(T, ldt, i + 1, i) = 0.0;
  return 1;
}

int schur(int n, double* H, int ldh, double* Z, int ldz) {
  // H is upper Hessenberg on entry; Z holds the Hessenberg transformation.
  if (n <= 0) return 0;
  double anorm = 0.0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i <= std::min(j + 1, n - 1); ++i) anorm = std::max(anorm, std::fabs(at(H, ldh, i, j)));
  if (anorm == 0.0) return 0;
  int hi = n - 1;
  int its = 0, total = 0;
  const int max_total = 60 * n + 100;
  double v[3];
  while (hi >= 0) {
    // look for a negligible sub-diagonal entry
    int l = hi;
    while (l > 0) {
      double s = std::fabs(at(H, ldh, l - 1, l - 1)) + std::fabs(at(H, ldh, l, l));
      if (s == 0.0) s = anorm;
      if (std::fabs(at(H, ldh, l, l - 1)) <= kEps * s) { at(H, ldh, l, l - 1) = 0.0; break; }
      --l;
    }
    if (l == hi) { --hi; its = 0; continue; }
    if (l == hi - 1) {
      standardize_2x2(n, H, ldh, Z, ldz, n, hi - 1);
      hi -= 2; its = 0; continue;
    }
    if (++total > max_total) return -1;
    ++its;
    double s, t;
    if (its % 11 == 10) {   // exceptional shift
      double ex = std::fabs(at(H, ldh, hi, hi - 1)) + std::fabs(at(H, ldh, hi - 1, hi - 2));
      double h11 = 0.75 * ex + at(H, ldh, hi, hi);
      s = 2.0 * h11;
      t = h11 * h11 + 0.4375 * ex * ex;
    } else {
      s = at(H, ldh, hi - 1, hi - 1) + at(H, ldh, hi, hi);
      t = at(H, ldh, hi - 1, hi - 1) * at(H, ldh, hi, hi) - at(H, ldh, hi - 1, hi) * at(H, ldh, hi, hi - 1);
    }
    double x = at(H, ldh, l, l) * at(H, ldh, l, l) + at(H, ldh, l, l + 1) * at(H, ldh, l + 1, l)
               - s * at(H, ldh, l, l) + t;
    double y = at(H, ldh, l + 1, l) * (at(H, ldh, l, l) + at(H, ldh, l + 1, l + 1) - s);
    double z = at(H, ldh, l + 1, l) * at(H, ldh, l + 2, l + 1);
    for (int k = l; k <= hi - 2; ++k) {
      double xv[3] = {x, y, z}, beta;
      house(xv, 3, v, &beta);
      int c0 = std::max(l, k - 1);
      apply_left(H, ldh, k, 3, c0, n - 1, v, beta);
      int r1 = std::min(k + 3, hi);
      apply_right(H, ldh, k, 3, 0, r1, v, beta);
      apply_right(Z, ldz, k, 3, 0, n - 1, v, beta);
      if (k > l) { at(H, ldh, k + 1, k - 1) = 0.0; at(H, ldh, k + 2, k - 1) = 0.0; }
      x = at(H, ldh, k + 1, k);
      y = at(H, ldh, k + 2, k);
      if (k < hi - 2) z = at(H, ldh, k + 3, k);
    }
    double xv[2] = {x, y}, beta;
    house(xv, 2, v, &beta);
    apply_left(H, ldh, hi - 1, 2, hi - 2, n - 1, v, beta);
    apply_right(H, ldh, hi - 1, 2, 0, hi, v, beta);
    apply_right(Z, ldz, hi - 1, 2, 0, n - 1, v, beta);
    if (hi - 2 > l) at(H, ldh, hi, hi - 2) = 0.0;
  }
  // clean: everything below the first sub-diagonal is zero
  for (int j = 0; j < n; ++j)
    for (int i = j + 2; i < n; ++i) at(H, ldh, i, j) = 0.0;
  return 0;
}

// Diagonal blocks of T starting in [i0, i1) (a 2x2 block is never split).
static void scan_blocks(const double* T, int ldt, int i0, int i1, int n, std::vector<Block>& out) {
  int i = i0;
  while (i < i1) {
    if (i + 1 < n && at(T, ldt, i + 1, i) != 0.0) {
      double a = at(T, ldt, i, i), b = at(T, ldt, i, i + 1), c = at(T, ldt, i + 1, i), d = at(T, ldt, i + 1, i + 1);
      double p = 0.5 * (a - d), disc = p * p + b * c;
      out.push_back({i, 2, 0.5 * (a + d), disc < 0 ? std::sqrt(-disc) : 0.0});
      i += 2;
    } else {
      out.push_back({i, 1, at(T, ldt, i, i), 0.0});
      i += 1;
    }
  }
}

std::vector<Block> blocks(int n, const double* T, int ldt) {
  std::vector<Block> out;
  int i = 0;
  while (i < n) {
    if (i + 1 < n && at(T, ldt, i + 1, i) != 0.0) {
      double a = at(T, ldt, i, i), b = at(T, ldt, i, i + 1), c = at(T, ldt, i + 1, i), d = at(T, ldt, i + 1, i + 1);
      double p = 0.5 * (a - d), disc = p * p + b * c;
      double re = 0.5 * (a + d);
      double im = disc < 0 ? std::sqrt(-disc) : 0.0;
      out.push_back({i, 2, re, im});
      i += 2;
    } else {
      out.push_back({i, 1, at(T, ldt, i, i), 0.0});
      i += 1;
    }
  }
  return out;
}

double key(double re, double im, int which) {
  switch (which) {
    case 0: return -std::hypot(re, im);  // LM
    case 1: return std::hypot(re, im);   // SM
    case 2: return -re;                  // LR
    default: return re;                  // SR
  }
}

namespace {

// Solve the small dense system M x = r (size s <= 4) by Gaussian elimination
// with partial pivoting.  Returns false if M is numerically singular.
bool small_solve(int s, double M[4][4], double r[4]) {
  for (int k = 0; k < s; ++k) {
    int p = k;
    for (int i = k + 1; i < s; ++i) if (std::fabs(M[i][k]) > std::fabs(M[p][k])) p = i;
    if (M[p][k] == 0.0) return false;
    if (p != k) { for (int j = 0; j < s; ++j) std::swap(M[k][j], M[p][j]); std::swap(r[k], r[p]); }
    for (int i = k + 1; i < s; ++i) {
      double f = M[i][k] / M[k][k];
      for (int j = k; j < s; ++j) M[i][j] -= f * M[k][j];
      r[i] -= f * r[k];
    }
  }
  for (int k = s - 1; k >= 0; --k) {
    double acc = r[k];
    for (int j = k + 1; j < s; ++j) acc -= M[k][j] * r[j];
    r[k] = acc / M[k][k];
  }
  return true;
}

}  // namespace

// Exchange of two adjacent 1x1 blocks a = T(j,j), c = T(j+1,j+1): the rotation
// whose first column is the eigenvector (b, c - a) of [[a, b], [0, c]] for c
// brings c to the top (G^T T G = [[c, *], [0, a]]).
static void swap_singles(int n, double* T, int ldt, double* Z, int ldz, int nz, int j) {
  const double a = at(T, ldt, j, j), b = at(T, ldt, j, j + 1), c = at(T, ldt, j + 1, j + 1);
  const double x = b, y = c - a;
  const double r = std::hypot(x, y);
  if (r == 0.0) return;                       // equal diagonal, b = 0: already in order
  const double cs = x / r, sn = y / r;
  for (int col = j; col < n; ++col) {         // rows j, j+1 <- G^T rows
    const double t0 = at(T, ldt, j, col), t1 = at(T, ldt, j + 1, col);
    at(T, ldt, j, col) = cs * t0 + sn * t1;
    at(T, ldt, j + 1, col) = -sn * t0 + cs * t1;
  }
  for (int row = 0; row <= j + 1; ++row) {    // columns j, j+1 <- columns G
    const double t0 = at(T, ldt, row, j), t1 = at(T, ldt, row, j + 1);
    at(T, ldt, row, j) = cs * t0 + sn * t1;
    at(T, ldt, row, j + 1) = -sn * t0 + cs * t1;
  }
  if (Z) {
    double* z0 = Z + (size_t)j * ldz;
    double* z1 = Z + (size_t)(j + 1) * ldz;
    for (int row = 0; row < nz; ++row) {
      const double t0 = z0[row], t1 = z1[row];
      z0[row] = cs * t0 + sn * t1;
      z1[row] = -sn * t0 + cs * t1;
    }
  }
  at(T, ldt, j, j) = c;
  at(T, ldt, j + 1, j + 1) = a;
  at(T, ldt, j + 1, j) = 0.0;
}

int swap_blocks(int n, double* T, int ldt, double* Z, int ldz, int nz, int j, int p, int q) {
  if (p == 1 && q == 1) {
    swap_singles(n, T, ldt, Z, ldz, nz, j);
    return 0;
  }
  const int s = p + q;
  // Sylvester: T11 X - X T22 = -T12, X is p x q; unknown index x(i,l) = i + p*l
  double M[4][4] = {{0}}, r[4] = {0};
  for (int l = 0; l < q; ++l)
    for (int i = 0; i < p; ++i) {
      int row = i + p * l;
      for (int ii = 0; ii < p; ++ii) M[row][ii + p * l] += at(T, ldt, j + i, j + ii);
      for (int ll = 0; ll < q; ++ll) M[row][i + p * ll] -= at(T, ldt, j + p + ll, j + p + l);
      r[row] = -at(T, ldt, j + i, j + p + l);
    }
  if (!small_solve(p * q, M, r)) return -1;
  // W = [X; I_q] (s x q); Householder QR, Q = H_1 H_2 ... (first q columns span W)
  double W[4][2];
  for (int l = 0; l < q; ++l) {
    for (int i = 0; i < p; ++i) W[i][l] = r[i + p * l];
    for (int i = 0; i < q; ++i) W[p + i][l] = (i == l) ? 1.0 : 0.0;
  }
  double Qs[4][4];
  for (int a = 0; a < s; ++a) for (int b = 0; b < s; ++b) Qs[a][b] = (a == b) ? 1.0 : 0.0;
  for (int l = 0; l < q; ++l) {
    double x[4], v[4], beta;
    int len = s - l;
    for (int i = 0; i < len; ++i) x[i] = W[l + i][l];
    house(x, len, v, &beta);
    if (beta == 0.0) continue;
    for (int c = l; c < q; ++c) {            // W <- H W
      double acc = 0.0;
      for (int i = 0; i < len; ++i) acc += v[i] * W[l + i][c];
      acc *= beta;
      for (int i = 0; i < len; ++i) W[l + i][c] -= acc * v[i];
    }
    for (int a = 0; a < s; ++a) {            // Qs <- Qs H
      double acc = 0.0;
      for (int i = 0; i < len; ++i) acc += Qs[a][l + i] * v[i];
      acc *= beta;
      for (int i = 0; i < len; ++i) Qs[a][l + i] -= acc * v[i];
    }
  }
  double wnorm = 0.0;
  for (int a = 0; a < s; ++a) for (int b = 0; b < s; ++b) wnorm = std::max(wnorm, std::fabs(at(T, ldt, j + a, j + b)));
  // T <- Qs^T T Qs on rows/columns j..j+s-1 of the full matrix, Z <- Z Qs
  std::vector<double> tmp(s);
  for (int c = j; c < n; ++c) {
    for (int a = 0; a < s; ++a) {
      double acc = 0.0;
      for (int b = 0; b < s; ++b) acc += Qs[b][a] * at(T, ldt, j + b, c);
      tmp[a] = acc;
    }
    for (int a = 0; a < s; ++a) at(T, ldt, j + a, c) = tmp[a];
  }
  auto right = [&](double* A, int lda, int rows) {
    for (int rr = 0; rr < rows; ++rr) {
      for (int a = 0; a < s; ++a) {
        double acc = 0.0;
        for (int b = 0; b < s; ++b) acc += at(A, lda, rr, j + b) * Qs[b][a];
        tmp[a] = acc;
      }
      for (int a = 0; a < s; ++a) at(A, lda, rr, j + a) = tmp[a];
    }
  };
  right(T, ldt, j + s);
  if (Z) right(Z, ldz, nz);
  // the p x q... now q x p block below the new leading block must be negligible
  double lower = 0.0;
  for (int a = q; a < s; ++a) for (int b = 0; b < q; ++b) lower = std::max(lower, std::fabs(at(T, ldt, j + a, j + b)));
  if (lower > 1e3 * kEps * std::max(wnorm, 1e-300)) {
    // reject: undo the similarity (Qs is orthogonal) so T keeps its structure
    for (int c = j; c < n; ++c) {
      for (int a = 0; a < s; ++a) {
        double acc = 0.0;
        for (int b = 0; b < s; ++b) acc += Qs[a][b] * at(T, ldt, j + b, c);
        tmp[a] = acc;
      }
      for (int a = 0; a < s; ++a) at(T, ldt, j + a, c) = tmp[a];
    }
    auto undo_right = [&](double* A, int lda, int rows) {
      for (int rr = 0; rr < rows; ++rr) {
        for (int a = 0; a < s; ++a) {
          double acc = 0.0;
          for (int b = 0; b < s; ++b) acc += at(A, lda, rr, j + b) * Qs[a][b];
          tmp[a] = acc;
        }
        for (int a = 0; a < s; ++a) at(A, lda, rr, j + a) = tmp[a];
      }
    };
    undo_right(T, ldt, j + s);
    if (Z) undo_right(Z, ldz, nz);
    return -2;
  }
  for (int a = q; a < s; ++a) for (int b = 0; b < q; ++b) at(T, ldt, j + a, j + b) = 0.0;
  for (int c = 0; c < j; ++c) for (int a = 0; a < s; ++a) at(T, ldt, j + a, c) = 0.0;
  if (q == 1 && s > 1) { /* single leading block: nothing to standardise */ }
  if (q == 2) standardize_2x2(n, T, ldt, Z, ldz, nz, j);
  if (p == 2) standardize_2x2(n, T, ldt, Z, ldz, nz, j + q);
  // a 2x2 block that became triangular leaves zeros; re-clean below-diagonal
  for (int a = 0; a < s; ++a)
    for (int b = 0; b < s; ++b)
      if (a > b + 1) at(T, ldt, j + a, j + b) = 0.0;
  return 0;
}

int reorder(int n, double* T, int ldt, double* Z, int ldz, int nz, int which, int nsort) {
  int top = 0;   // first position not yet fixed
  int placed = 0;
  int fails = 0;
  while (placed < nsort && top < n) {
    std::vector<Block> bl = blocks(n, T, ldt);
    int best = -1;
    double bk = 0.0;
    for (size_t t = 0; t < bl.size(); ++t) {
      if (bl[t].start < top) continue;
      double kk = key(bl[t].re, bl[t].im, which);
      if (best < 0 || kk < bk) { best = (int)t; bk = kk; }
    }
    if (best < 0) break;
    // bubble block `best` up to position `top`
    int t = best;
    std::vector<Block> loc;
    while (bl[t].start > top) {
      const int up_start = bl[t - 1].start, up_size = bl[t - 1].size, s = up_size + bl[t].size;
      int rc = swap_blocks(n, T, ldt, Z, ldz, nz, up_start, up_size, bl[t].size);
      if (rc != 0) { ++fails; break; }
      // only the two swapped blocks changed: rescan their rows (the moved
      // block now starts at up_start; a 2x2 block may have split)
      loc.clear();
      scan_blocks(T, ldt, up_start, up_start + s, n, loc);
      bl.erase(bl.begin() + (t - 1), bl.begin() + (t + 1));
      bl.insert(bl.begin() + (t - 1), loc.begin(), loc.end());
      t = t - 1;
    }
    if (t < 0) break;
    top = bl[t].start + bl[t].size;
    ++placed;
  }
  return fails;
}

int reorder_select(int n, double* T, int ldt, double* Z, int ldz, int nz, const std::vector<char>& sel) {
  std::vector<Block> bl = blocks(n, T, ldt);
  if (sel.size() != bl.size()) return -1;
  // work on copies so that a refused swap leaves T and Z as they were
  std::vector<double> T2((size_t)n * n), Z2((size_t)nz * n);
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) T2[i + (size_t)j * n] = at(T, ldt, i, j);
    for (int i = 0; i < nz; ++i) Z2[i + (size_t)j * nz] = at(Z, ldz, i, j);
  }
  std::vector<int> size(bl.size());
  for (size_t t = 0; t < bl.size(); ++t) size[t] = bl[t].size;
  std::vector<char> cur = sel;   // flags in the current block order
  int placed = 0;                // flagged blocks already at the top
  for (size_t t = 0; t < cur.size(); ++t) {
    if (!cur[t]) continue;
    int start = 0;                 // row of block t - 1 (recomputed as it moves)
    for (int v = 0; v + 1 < (int)t; ++v) start += size[v];
    for (int u = (int)t; u > placed; --u) {
      if (swap_blocks(n, T2.data(), n, Z2.data(), nz, nz, start, size[u - 1], size[u]) != 0) return -1;
      std::vector<Block> loc;
      scan_blocks(T2.data(), n, start, start + size[u - 1] + size[u], n, loc);
      if (loc.size() != 2 || loc[0].size != size[u] || loc[1].size != size[u - 1]) return -1;
      std::swap(size[u], size[u - 1]);
      std::swap(cur[u], cur[u - 1]);
      if (u - 2 >= 0) start -= size[u - 2];
    }
    ++placed;
  }
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) at(T, ldt, i, j) = T2[i + (size_t)j * n];
    for (int i = 0; i < nz; ++i) at(Z, ldz, i, j) = Z2[i + (size_t)j * nz];
  }
  return 0;
}

int sketch_reorthonormalize(int d, int ka, double* S, const double* T, const double* b, double* Rinv, double* Tn,
                            double* bn) {
  const int kb = ka + 1;
  std::vector<double> R((size_t)kb * kb);
  house_qr(d, kb, S, R.data());
  for (int j = 0; j < kb; ++j)
    for (int i = 0; i < kb; ++i) Rinv[i + (size_t)j * kb] = 0.0;
  for (int j = 0; j < kb; ++j) {          // R^-1 by back substitution
    if (R[j + (size_t)j * kb] == 0.0) return -1;
    Rinv[j + (size_t)j * kb] = 1.0 / R[j + (size_t)j * kb];
    for (int i = j - 1; i >= 0; --i) {
      double acc = 0.0;
      for (int l = i + 1; l <= j; ++l) acc += R[i + (size_t)l * kb] * Rinv[l + (size_t)j * kb];
      Rinv[i + (size_t)j * kb] = -acc / R[i + (size_t)i * kb];
    }
  }
  // P = R11 T + r12 b^T, Tn = P R11^-1 (R11^-1 is the leading block of R^-1)
  std::vector<double> P((size_t)ka * ka);
  for (int j = 0; j < ka; ++j)
    for (int i = 0; i < ka; ++i) {
      double acc = R[i + (size_t)ka * kb] * b[j];
      for (int l = i; l < ka; ++l) acc += R[i + (size_t)l * kb] * T[l + (size_t)j * ka];
      P[i + (size_t)j * ka] = acc;
    }
  for (int j = 0; j < ka; ++j) {
    for (int i = 0; i < ka; ++i) {
      double acc = 0.0;
      for (int l = 0; l <= j; ++l) acc += P[i + (size_t)l * ka] * Rinv[l + (size_t)j * kb];
      Tn[i + (size_t)j * ka] = acc;
    }
    double acc = 0.0;
    for (int l = 0; l <= j; ++l) acc += b[l] * Rinv[l + (size_t)j * kb];
    bn[j] = R[ka + (size_t)ka * kb] * acc;
  }
  return 0;
}

void house_qr(int d, int ka, double* S, double* R) {
  std::vector<double> V((size_t)d * ka, 0.0), beta(ka, 0.0);
  std::vector<double> A(S, S + (size_t)d * ka);
  for (int j = 0; j < ka; ++j) {
    double s = 0.0;
    for (int i = j; i < d; ++i) s += A[i + (size_t)j * d] * A[i + (size_t)j * d];
    double nrm = std::sqrt(s);
    double x0 = A[j + (size_t)j * d];
    double v0 = x0 >= 0 ? x0 + nrm : x0 - nrm;
    double* v = &V[(size_t)j * d];
    v[j] = 1.0;
    double vtv = 1.0;
    for (int i = j + 1; i < d; ++i) { v[i] = (v0 != 0.0) ? A[i + (size_t)j * d] / v0 : 0.0; vtv += v[i] * v[i]; }
    beta[j] = (nrm == 0.0) ? 0.0 : 2.0 / vtv;
    for (int cc = j; cc < ka; ++cc) {
      double acc = 0.0;
      for (int i = j; i < d; ++i) acc += v[i] * A[i + (size_t)cc * d];
      acc *= beta[j];
      for (int i = j; i < d; ++i) A[i + (size_t)cc * d] -= acc * v[i];
    }
  }
  // R and explicit Q (first ka columns)
  for (int j = 0; j < ka; ++j)
    for (int i = 0; i < ka; ++i) R[i + (size_t)j * ka] = (i <= j) ? A[i + (size_t)j * d] : 0.0;
  std::vector<double> Q((size_t)d * ka, 0.0);
  for (int j = 0; j < ka; ++j) Q[j + (size_t)j * d] = 1.0;
  for (int h = ka - 1; h >= 0; --h) {
    const double* v = &V[(size_t)h * d];
    for (int cc = 0; cc < ka; ++cc) {
      double acc = 0.0;
      for (int i = h; i < d; ++i) acc += v[i] * Q[i + (size_t)cc * d];
      acc *= beta[h];
      for (int i = h; i < d; ++i) Q[i + (size_t)cc * d] -= acc * v[i];
    }
  }
  for (int j = 0; j < ka; ++j) {      // positive diagonal of R
    if (R[j + (size_t)j * ka] < 0) {
      for (int cc = j; cc < ka; ++cc) R[j + (size_t)cc * ka] = -R[j + (size_t)cc * ka];
      for (int i = 0; i < d; ++i) Q[i + (size_t)j * d] = -Q[i + (size_t)j * d];
    }
  }
  std::memcpy(S, Q.data(), Q.size() * sizeof(double));
}

int quasi_eig(int n, const double* T, int ldt, double* lam_re, double* lam_im,
              std::complex<double>* Y, int ldy) {
  std::vector<Block> bl = blocks(n, T, ldt);
  typedef std::complex<double> cd;
  std::vector<cd> y(n);
  int col = 0;
  double tnorm = 0.0;
  for (int j = 0; j < n; ++j) for (int i = 0; i <= std::min(j + 1, n - 1); ++i) tnorm = std::max(tnorm, std::fabs(at(T, ldt, i, j)));
  const double small = std::max(tnorm * kEps, 1e-300);
  for (size_t bi = 0; bi < bl.size(); ++bi) {
    const Block& B = bl[bi];
    int nlam = B.size;           // a 2x2 block gives a conjugate pair
    for (int e = 0; e < nlam; ++e) {
      cd lam(B.re, B.size == 2 ? (e == 0 ? B.im : -B.im) : 0.0);
      std::fill(y.begin(), y.end(), cd(0.0));
      int top;
      if (B.size == 1) {
        y[B.start] = 1.0;
        top = B.start;
      } else {
        // eigenvector of the standardised block [[a, b], [c, a]]: (b, lam - a)
        double b = at(T, ldt, B.start, B.start + 1);
        y[B.start] = b;
        y[B.start + 1] = lam - at(T, ldt, B.start, B.start);
        top = B.start;
      }
      // back substitution over the blocks above
      for (int ci = (int)bi - 1; ci >= 0; --ci) {
        const Block& C = bl[ci];
        cd rhs[2];
        for (int a = 0; a < C.size; ++a) {
          cd acc = 0.0;
          for (int l = C.start + C.size; l <= top + B.size - 1; ++l) acc += at(T, ldt, C.start + a, l) * y[l];
          rhs[a] = -acc;
        }
        if (C.size == 1) {
          cd den = at(T, ldt, C.start, C.start) - lam;
          if (std::abs(den) < small) den = small;
          y[C.start] = rhs[0] / den;
        } else {
          cd m00 = at(T, ldt, C.start, C.start) - lam, m01 = at(T, ldt, C.start, C.start + 1);
          cd m10 = at(T, ldt, C.start + 1, C.start), m11 = at(T, ldt, C.start + 1, C.start + 1) - lam;
          cd det = m00 * m11 - m01 * m10;
          if (std::abs(det) < small * small) det = small * small;
          y[C.start] = (rhs[0] * m11 - m01 * rhs[1]) / det;
          y[C.start + 1] = (m00 * rhs[1] - m10 * rhs[0]) / det;
        }
      }
      double nrm = 0.0;
      for (int i = 0; i < n; ++i) nrm += std::norm(y[i]);
      nrm = std::sqrt(nrm);
      for (int i = 0; i < n; ++i) Y[i + (size_t)col * ldy] = y[i] / nrm;
      lam_re[col] = lam.real();
      lam_im[col] = lam.imag();
      ++col;
    }
  }
  return 0;
}

}  // namespace rks_dense
