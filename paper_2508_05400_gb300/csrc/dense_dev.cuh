// Small dense steps of the rKS contraction (Algorithm 1) on the device, for
// one problem per warp: Hessenberg reduction, Francis double-shift QR to the
// real Schur form, reordering of the wanted eigenvalues to the top by swaps
// of adjacent diagonal blocks (Bai & Demmel), eigenvectors of a
// quasi-triangular matrix.  The methods are those of dense.cpp (the host
// side); here every routine is executed by all 32 lanes of one warp
// together: the scalar decisions (reflectors, shifts, deflation tests) are
// computed by every lane from shared memory (the same values, so the same
// branches), and the row and column updates are split over the lanes, with
// __syncwarp() between the phases.  Matrices are column-major in shared (or
// global) memory with leading dimension ld.  Every loop is bounded; the QR
// iteration returns -1 after 60 n + 100 sweeps.
//
// The routines are templates on the scalar type R: double, or rks_dd::df, a
// double-float number (an unevaluated sum hi + lo of two floats, 48-bit
// significand) whose arithmetic runs on the FP32 pipes: Dekker's exact
// product (by fma) and Knuth's exact sum, with the accurate addition and the
// Newton-corrected division and square root of the double-double literature
// (Dekker 1971; Hida, Li & Bailey 2001) carried over to float pairs.  On a GPU
// whose FP64 rate is a small fraction of its FP32 rate the df instantiation
// is the fast one; its rounding unit 2^-48 is far below what the
// contraction needs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rks_dd {

constexpr int kMaxM = 64;   // largest matrix the per-lane block lists cover

// ---------------------------------------------------------------------------
// double-float numbers
// ---------------------------------------------------------------------------

struct df {
  float hi, lo;
  __host__ __device__ df() : hi(0.f), lo(0.f) {}
  __host__ __device__ df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ df(float x) : hi(x), lo(0.f) {}
  __host__ __device__ df(int x) : hi((float)x), lo(0.f) {}
  __host__ __device__ explicit df(double x) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  }
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void df_quick_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
__device__ __forceinline__ df operator+(df a, df b) {
  float s, e, t, f;
  df_two_sum(a.hi, b.hi, s, e);
  df_two_sum(a.lo, b.lo, t, f);
  e += t;
  df_quick_two_sum(s, e, s, e);
  e += f;
  df_quick_two_sum(s, e, s, e);
  return df(s, e);
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float s;
  df_quick_two_sum(p, e, s, e);
  return df(s, e);
}
// quotient by two correction steps on a fast float quotient: each step
// divides the exact-ish remainder, so the float quotients need only be
// accurate to a few units in the last place
__device__ __forceinline__ df operator/(df a, df b) {
  const float rb = __frcp_rn(b.hi);
  const float q1 = a.hi * rb;
  const df r = a - b * df(q1);
  const float q2 = r.hi * rb;
  const df r2 = r - b * df(q2);
  const float q3 = r2.hi * rb;
  float s, e;
  df_quick_two_sum(q1, q2, s, e);
  return df(s, e) + df(q3);
}
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__device__ __forceinline__ df& operator-=(df& a, df b) { return a = a - b; }
__device__ __forceinline__ df& operator*=(df& a, df b) { return a = a * b; }
__device__ __forceinline__ df& operator/=(df& a, df b) { return a = a / b; }
__device__ __forceinline__ bool operator<(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df a, df b) { return b < a; }
__device__ __forceinline__ bool operator<=(df a, df b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(df a, df b) { return !(a < b); }
__device__ __forceinline__ bool operator==(df a, df b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(df a, df b) { return !(a == b); }

// scalar functions for both types
__device__ __forceinline__ double rabs(double x) { return fabs(x); }
__device__ __forceinline__ df rabs(df x) { return x.hi < 0.f || (x.hi == 0.f && x.lo < 0.f) ? -x : x; }
__device__ __forceinline__ double rsqrt_(double x) { return sqrt(x); }
// square root by one Newton correction of the float root: y + (x - y^2) / (2 y)
__device__ __forceinline__ df rsqrt_(df x) {
  if (!(x.hi > 0.f)) return df(0.f);
  const float y = sqrtf(x.hi);
  const float p = y * y;
  const float pe = fmaf(y, y, -p);
  const df r = x - df(p, pe);
  const float c = r.hi / (2.f * y);
  float s, e;
  df_quick_two_sum(y, c, s, e);
  return df(s, e);
}
__device__ __forceinline__ double rmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ df rmax(df a, df b) { return a < b ? b : a; }
template <class R>
__device__ __forceinline__ bool rfinite(R x) { return isfinite((double)x); }
// sqrt(a^2 + b^2) without overflow or underflow of the squares
template <class R>
__device__ __forceinline__ R rhypot(R a, R b) {
  a = rabs(a);
  b = rabs(b);
  const R s = rmax(a, b);
  if (s == R(0)) return R(0);
  const R is = R(1) / s;
  const R x = a * is, y = b * is;
  return s * rsqrt_(x * x + y * y);
}
template <class R>
__device__ __forceinline__ R reps();
template <>
__device__ __forceinline__ double reps<double>() { return 2.220446049250313e-16; }
template <>
__device__ __forceinline__ df reps<df>() { return df(3.552713678800501e-15f); }   // 2^-48

template <class R>
__device__ __forceinline__ R& at(R* A, int ld, int i, int j) { return A[i + j * ld]; }
template <class R>
__device__ __forceinline__ R at(const R* A, int ld, int i, int j) { return A[i + j * ld]; }

// Butterfly sum / max over the 32 lanes (the same value in every lane: each
// step adds two partials in either order, and + and max commute exactly).
__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ df warp_allsum(df v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = v + df(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
  return v;
}
__device__ __forceinline__ double warp_allmax(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ df warp_allmax(df v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = rmax(v, df(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)));
  return v;
}

// ---------------------------------------------------------------------------
// reflectors and rotations
// ---------------------------------------------------------------------------

// Householder vector for x (LEN <= 4, in registers): P = I - beta v v^T, v[0] = 1.
template <int LEN, class R>
__device__ __forceinline__ void house(const R (&x)[LEN], R (&v)[LEN], R& beta) {
  R s = R(0);
#pragma unroll
  for (int i = 1; i < LEN; ++i) s += x[i] * x[i];
  v[0] = R(1);
#pragma unroll
  for (int i = 1; i < LEN; ++i) v[i] = x[i];
  beta = R(0);
  if (s == R(0)) return;
  const R nrm = rsqrt_(x[0] * x[0] + s);
  const R v0 = x[0] >= R(0) ? x[0] + nrm : x[0] - nrm;
  const R iv0 = R(1) / v0;
#pragma unroll
  for (int i = 1; i < LEN; ++i) v[i] *= iv0;
  R vtv = R(1);
#pragma unroll
  for (int i = 1; i < LEN; ++i) vtv += v[i] * v[i];
  beta = R(2) / vtv;
}

// rows r0..r0+LEN-1, columns c0..c1: A <- (I - beta v v^T) A (lanes over columns)
template <int LEN, class R>
__device__ __forceinline__ void apply_left_n(R* A, int ld, int r0, int c0, int c1, const R (&v)[LEN], R beta,
                                             int lane) {
  if (beta != R(0)) {
    for (int j = c0 + lane; j <= c1; j += 32) {
      R a[LEN];
      R s = R(0);
#pragma unroll
      for (int i = 0; i < LEN; ++i) {
        a[i] = at(A, ld, r0 + i, j);
        s += v[i] * a[i];
      }
      s *= beta;
#pragma unroll
      for (int i = 0; i < LEN; ++i) at(A, ld, r0 + i, j) = a[i] - s * v[i];
    }
  }
  __syncwarp();
}

// columns c0..c0+LEN-1, rows r0..r1: A <- A (I - beta v v^T) (lanes over rows)
template <int LEN, class R>
__device__ __forceinline__ void apply_right_n(R* A, int ld, int c0, int r0, int r1, const R (&v)[LEN], R beta,
                                              int lane) {
  if (beta != R(0)) {
    for (int i = r0 + lane; i <= r1; i += 32) {
      R a[LEN];
      R s = R(0);
#pragma unroll
      for (int j = 0; j < LEN; ++j) {
        a[j] = at(A, ld, i, c0 + j);
        s += a[j] * v[j];
      }
      s *= beta;
#pragma unroll
      for (int j = 0; j < LEN; ++j) at(A, ld, i, c0 + j) = a[j] - s * v[j];
    }
  }
  __syncwarp();
}

// apply_left_n on rows r0.. of A and, in the same phase, apply_right_n on
// columns r0.. of Z (nz rows): different arrays, one barrier.
template <int LEN, class R>
__device__ __forceinline__ void apply_left_right_n(R* A, int ld, int r0, int c0, int c1, R* Z, int ldz, int nz,
                                                   const R (&v)[LEN], R beta, int lane) {
  if (beta != R(0)) {
    for (int j = c0 + lane; j <= c1; j += 32) {
      R a[LEN];
      R s = R(0);
#pragma unroll
      for (int i = 0; i < LEN; ++i) {
        a[i] = at(A, ld, r0 + i, j);
        s += v[i] * a[i];
      }
      s *= beta;
#pragma unroll
      for (int i = 0; i < LEN; ++i) at(A, ld, r0 + i, j) = a[i] - s * v[i];
    }
    for (int i = lane; i < nz; i += 32) {
      R a[LEN];
      R s = R(0);
#pragma unroll
      for (int j = 0; j < LEN; ++j) {
        a[j] = at(Z, ldz, i, r0 + j);
        s += a[j] * v[j];
      }
      s *= beta;
#pragma unroll
      for (int j = 0; j < LEN; ++j) at(Z, ldz, i, r0 + j) = a[j] - s * v[j];
    }
  }
  __syncwarp();
}

// The same with a vector of any length in shared memory (Hessenberg reduction).
template <class R>
__device__ inline void apply_left(R* A, int ld, int r0, int len, int c0, int c1, const R* v, R beta, int lane) {
  if (beta != R(0)) {
    for (int j = c0 + lane; j <= c1; j += 32) {
      R s = R(0);
      for (int i = 0; i < len; ++i) s += v[i] * at(A, ld, r0 + i, j);
      s *= beta;
      for (int i = 0; i < len; ++i) at(A, ld, r0 + i, j) -= s * v[i];
    }
  }
  __syncwarp();
}
template <class R>
__device__ inline void apply_right(R* A, int ld, int c0, int len, int r0, int r1, const R* v, R beta, int lane) {
  if (beta != R(0)) {
    for (int i = r0 + lane; i <= r1; i += 32) {
      R s = R(0);
      for (int j = 0; j < len; ++j) s += at(A, ld, i, c0 + j) * v[j];
      s *= beta;
      for (int j = 0; j < len; ++j) at(A, ld, i, c0 + j) -= s * v[j];
    }
  }
  __syncwarp();
}

// Plane rotation on rows / columns (i, i+1) of T (n x n) and columns of Z (nz rows).
template <class R>
__device__ inline void rotate_pair(int n, R* T, int ldt, R* Z, int ldz, int nz, int i, R cs, R sn, int lane) {
  for (int j = i + lane; j < n; j += 32) {
    const R a = at(T, ldt, i, j), b = at(T, ldt, i + 1, j);
    at(T, ldt, i, j) = cs * a + sn * b;
    at(T, ldt, i + 1, j) = cs * b - sn * a;
  }
  __syncwarp();
  for (int r = lane; r <= i + 1; r += 32) {
    const R a = at(T, ldt, r, i), b = at(T, ldt, r, i + 1);
    at(T, ldt, r, i) = cs * a + sn * b;
    at(T, ldt, r, i + 1) = cs * b - sn * a;
  }
  if (Z)
    for (int r = lane; r < nz; r += 32) {
      const R a = at(Z, ldz, r, i), b = at(Z, ldz, r, i + 1);
      at(Z, ldz, r, i) = cs * a + sn * b;
      at(Z, ldz, r, i + 1) = cs * b - sn * a;
    }
  __syncwarp();
}

// A (n x n) <- Q^T A Q upper Hessenberg, Q = the reflectors (Q set to I first).
// v: scratch of n values in shared memory.  The norm of each column is a
// butterfly over the lanes (the same value in every lane).
template <class R>
__device__ inline void hessenberg(int n, R* A, int lda, R* Q, int ldq, R* v, int lane) {
  for (int t = lane; t < n * n; t += 32) at(Q, ldq, t % n, t / n) = (t % n == t / n) ? R(1) : R(0);
  __syncwarp();
  for (int k = 0; k + 2 < n; ++k) {
    const int len = n - k - 1;
    R s = R(0);
    for (int i = 1 + lane; i < len; i += 32) s += at(A, lda, k + 1 + i, k) * at(A, lda, k + 1 + i, k);
    s = warp_allsum(s);
    const R x0 = at(A, lda, k + 1, k);
    R beta = R(0), iv0 = R(1);
    if (s != R(0)) {
      const R nrm = rsqrt_(x0 * x0 + s);
      iv0 = R(1) / (x0 >= R(0) ? x0 + nrm : x0 - nrm);
    }
    __syncwarp();
    R vv = R(0);
    for (int i = lane; i < len; i += 32) {
      const R vi = i == 0 ? R(1) : (s != R(0) ? at(A, lda, k + 1 + i, k) * iv0 : R(0));
      v[i] = vi;
      if (i > 0) vv += vi * vi;
    }
    vv = warp_allsum(vv);
    __syncwarp();
    if (s != R(0)) beta = R(2) / (R(1) + vv);
    apply_left(A, lda, k + 1, len, k, n - 1, v, beta, lane);
    apply_right(A, lda, k + 1, len, 0, n - 1, v, beta, lane);
    apply_right(Q, ldq, k + 1, len, 0, n - 1, v, beta, lane);
    for (int i = k + 2 + lane; i < n; i += 32) at(A, lda, i, k) = R(0);
    __syncwarp();
  }
}

// Standardise the 2x2 block at i; returns its size (1: real pair, 2: complex).
template <class R>
__device__ inline int standardize_2x2(int n, R* T, int ldt, R* Z, int ldz, int nz, int i, int lane) {
  const R a = at(T, ldt, i, i), b = at(T, ldt, i, i + 1);
  const R c = at(T, ldt, i + 1, i), d = at(T, ldt, i + 1, i + 1);
  if (c == R(0)) return 1;
  R cs, sn;
  int is_pair;
  if (b == R(0)) {
    cs = R(0); sn = R(1); is_pair = 0;
  } else {
    const R p = R(0.5f) * (a - d);
    const R disc = p * p + b * c;
    if (disc >= R(0)) {
      const R z = p + (p >= R(0) ? R(1) : R(-1)) * rsqrt_(disc);
      const R l1 = d + z;
      R v1 = b, v2 = l1 - a;
      const R w1 = l1 - d, w2 = c;
      if (rhypot(w1, w2) > rhypot(v1, v2)) { v1 = w1; v2 = w2; }
      const R nv = rhypot(v1, v2);
      cs = v1 / nv; sn = v2 / nv; is_pair = 0;
    } else {
      if (a == d && (b + c) == R(0)) return 2;
      // the rotation by theta with 2 theta = atan2(d - a, b + c) equalises the
      // diagonal; cos and sin of theta from those of 2 theta by the
      // half-angle formulas (theta in (-pi/2, pi/2], so cos theta >= 0)
      const R X = b + c, Y = d - a;
      const R r2 = rhypot(X, Y);
      const R c2 = X / r2, s2 = Y / r2;
      if (c2 >= R(0)) {
        cs = rsqrt_(R(0.5f) * (R(1) + c2));
        sn = s2 / (R(2) * cs);
      } else {
        sn = rsqrt_(R(0.5f) * (R(1) - c2));
        if (s2 < R(0)) sn = -sn;
        cs = s2 / (R(2) * sn);
      }
      is_pair = 1;
    }
  }
  __syncwarp();
  rotate_pair(n, T, ldt, Z, ldz, nz, i, cs, sn, lane);
  int size = 1;
  if (is_pair) {
    const R mm = R(0.5f) * (at(T, ldt, i, i) + at(T, ldt, i + 1, i + 1));
    const bool real = at(T, ldt, i, i + 1) * at(T, ldt, i + 1, i) >= R(0);
    __syncwarp();
    if (lane == 0) {
      at(T, ldt, i, i) = mm;
      at(T, ldt, i + 1, i + 1) = mm;
      if (real) at(T, ldt, i + 1, i) = R(0);
    }
    size = real ? 1 : 2;
  } else {
    __syncwarp();
    if (lane == 0) at(T, ldt, i + 1, i) = R(0);
  }
  __syncwarp();
  return size;
}

// Real Schur form of the upper Hessenberg H (n x n) in place, Z <- Z * (rotations)
// (Z has nz rows).  Returns 0, or -1 if the iteration did not converge.
template <class R>
__device__ inline int schur(int n, R* H, int ldh, R* Z, int ldz, int nz, int lane) {
  if (n <= 0) return 0;
  const R eps = reps<R>();
  R anorm = R(0);
  for (int j = lane; j < n; j += 32)
    for (int i = 0; i <= min(j + 1, n - 1); ++i) anorm = rmax(anorm, rabs(at(H, ldh, i, j)));
  anorm = warp_allmax(anorm);
  if (anorm == R(0)) return 0;
  int hi = n - 1, its = 0, total = 0;
  const int max_total = 60 * n + 100;
  while (hi >= 0) {
    int l = hi;
    while (l > 0) {
      R s = rabs(at(H, ldh, l - 1, l - 1)) + rabs(at(H, ldh, l, l));
      if (s == R(0)) s = anorm;
      if (rabs(at(H, ldh, l, l - 1)) <= eps * s) break;
      --l;
    }
    __syncwarp();
    if (l > 0 && lane == 0) at(H, ldh, l, l - 1) = R(0);
    __syncwarp();
    if (l == hi) { --hi; its = 0; continue; }
    if (l == hi - 1) {
      standardize_2x2(n, H, ldh, Z, ldz, nz, hi - 1, lane);
      hi -= 2; its = 0; continue;
    }
    if (++total > max_total) return -1;
    ++its;
    R s, t;
    if (its % 11 == 10) {   // exceptional shift
      const R ex = rabs(at(H, ldh, hi, hi - 1)) + rabs(at(H, ldh, hi - 1, hi - 2));
      const R h11 = R(0.75f) * ex + at(H, ldh, hi, hi);
      s = R(2) * h11;
      t = h11 * h11 + R(0.4375f) * ex * ex;
    } else {
      s = at(H, ldh, hi - 1, hi - 1) + at(H, ldh, hi, hi);
      t = at(H, ldh, hi - 1, hi - 1) * at(H, ldh, hi, hi) - at(H, ldh, hi - 1, hi) * at(H, ldh, hi, hi - 1);
    }
    R x = at(H, ldh, l, l) * at(H, ldh, l, l) + at(H, ldh, l, l + 1) * at(H, ldh, l + 1, l)
          - s * at(H, ldh, l, l) + t;
    R y = at(H, ldh, l + 1, l) * (at(H, ldh, l, l) + at(H, ldh, l + 1, l + 1) - s);
    R z = at(H, ldh, l + 1, l) * at(H, ldh, l + 2, l + 1);
    for (int k = l; k <= hi - 2; ++k) {
      const R xv[3] = {x, y, z};
      R v[3], beta;
      house<3>(xv, v, beta);
      __syncwarp();
      apply_left_right_n<3>(H, ldh, k, max(l, k - 1), n - 1, Z, ldz, nz, v, beta, lane);
      apply_right_n<3>(H, ldh, k, 0, min(k + 3, hi), v, beta, lane);
      if (k > l && lane == 0) { at(H, ldh, k + 1, k - 1) = R(0); at(H, ldh, k + 2, k - 1) = R(0); }
      __syncwarp();
      x = at(H, ldh, k + 1, k);
      y = at(H, ldh, k + 2, k);
      if (k < hi - 2) z = at(H, ldh, k + 3, k);
      __syncwarp();
    }
    const R xv[2] = {x, y};
    R v[2], beta;
    house<2>(xv, v, beta);
    __syncwarp();
    apply_left_right_n<2>(H, ldh, hi - 1, hi - 2, n - 1, Z, ldz, nz, v, beta, lane);
    apply_right_n<2>(H, ldh, hi - 1, 0, hi, v, beta, lane);
    if (hi - 2 > l && lane == 0) at(H, ldh, hi, hi - 2) = R(0);
    __syncwarp();
  }
  for (int t = lane; t < n * n; t += 32) {
    const int i = t % n, j = t / n;
    if (i > j + 1) at(H, ldh, i, j) = R(0);
  }
  __syncwarp();
  return 0;
}

// ---------------------------------------------------------------------------
// diagonal blocks, reordering, eigenvectors
// ---------------------------------------------------------------------------

template <class R>
struct Block { int start, size; R re, im; };

template <class R>
__device__ inline Block<R> block_at(const R* T, int ldt, int i, int n) {
  if (i + 1 < n && at(T, ldt, i + 1, i) != R(0)) {
    const R a = at(T, ldt, i, i), b = at(T, ldt, i, i + 1), c = at(T, ldt, i + 1, i), d = at(T, ldt, i + 1, i + 1);
    const R p = R(0.5f) * (a - d), disc = p * p + b * c;
    return {i, 2, R(0.5f) * (a + d), disc < R(0) ? rsqrt_(-disc) : R(0)};
  }
  return {i, 1, at(T, ldt, i, i), R(0)};
}

// Ordering key of an eigenvalue (smaller is wanted first).
template <class R>
__device__ inline R key(R re, R im, int which) {
  switch (which) {
    case 0: return -rhypot(re, im);
    case 1: return rhypot(re, im);
    case 2: return -re;
    default: return re;
  }
}

// S x S linear system M x = r by Gaussian elimination with partial pivoting,
// in registers (the row exchanges are selects); false if singular.
template <int S, class R>
__device__ __forceinline__ bool small_solve(R (&M)[S][S], R (&r)[S]) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < S; ++k) {
    int p = k;
    R pv = rabs(M[k][k]);
#pragma unroll
    for (int i = k + 1; i < S; ++i)
      if (rabs(M[i][k]) > pv) { p = i; pv = rabs(M[i][k]); }
#pragma unroll
    for (int i = k + 1; i < S; ++i) {
      const bool sw = i == p;
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const R a = M[k][j], b = M[i][j];
        M[k][j] = sw ? b : a;
        M[i][j] = sw ? a : b;
      }
      const R a = r[k], b = r[i];
      r[k] = sw ? b : a;
      r[i] = sw ? a : b;
    }
    if (M[k][k] == R(0)) ok = false;
    const R inv = M[k][k] == R(0) ? R(0) : R(1) / M[k][k];
#pragma unroll
    for (int i = k + 1; i < S; ++i) {
      const R f = M[i][k] * inv;
#pragma unroll
      for (int j = k; j < S; ++j) M[i][j] -= f * M[k][j];
      r[i] -= f * r[k];
    }
  }
  if (!ok) return false;
#pragma unroll
  for (int k = S - 1; k >= 0; --k) {
    R acc = r[k];
#pragma unroll
    for (int j = k + 1; j < S; ++j) acc -= M[k][j] * r[j];
    r[k] = acc / M[k][k];
  }
  return true;
}

// Swap adjacent 1x1 blocks at j (the rotation with first column the eigenvector of c).
template <class R>
__device__ inline void swap_singles(int n, R* T, int ldt, R* Z, int ldz, int nz, int j, int lane) {
  const R a = at(T, ldt, j, j), b = at(T, ldt, j, j + 1), c = at(T, ldt, j + 1, j + 1);
  const R x = b, y = c - a;
  const R r = rhypot(x, y);
  __syncwarp();
  if (r == R(0)) return;
  const R ir = R(1) / r;
  const R cs = x * ir, sn = y * ir;
  for (int col = j + lane; col < n; col += 32) {
    const R t0 = at(T, ldt, j, col), t1 = at(T, ldt, j + 1, col);
    at(T, ldt, j, col) = cs * t0 + sn * t1;
    at(T, ldt, j + 1, col) = cs * t1 - sn * t0;
  }
  __syncwarp();
  for (int row = lane; row <= j + 1; row += 32) {
    const R t0 = at(T, ldt, row, j), t1 = at(T, ldt, row, j + 1);
    at(T, ldt, row, j) = cs * t0 + sn * t1;
    at(T, ldt, row, j + 1) = cs * t1 - sn * t0;
  }
  if (Z)
    for (int row = lane; row < nz; row += 32) {
      const R t0 = at(Z, ldz, row, j), t1 = at(Z, ldz, row, j + 1);
      at(Z, ldz, row, j) = cs * t0 + sn * t1;
      at(Z, ldz, row, j + 1) = cs * t1 - sn * t0;
    }
  __syncwarp();
  if (lane == 0) {
    at(T, ldt, j, j) = c;
    at(T, ldt, j + 1, j + 1) = a;
    at(T, ldt, j + 1, j) = R(0);
  }
  __syncwarp();
}

// Reflector L of the Householder QR of W (S x Q), accumulated into Qs.
template <int S, int Q, int L, class R>
__device__ __forceinline__ void qr_step(R (&W)[S][Q], R (&Qs)[S][S]) {
  constexpr int LEN = S - L;
  R x[LEN], v[LEN], beta;
#pragma unroll
  for (int i = 0; i < LEN; ++i) x[i] = W[L + i][L];
  house<LEN>(x, v, beta);
  if (beta == R(0)) return;
#pragma unroll
  for (int c = L; c < Q; ++c) {
    R acc = R(0);
#pragma unroll
    for (int i = 0; i < LEN; ++i) acc += v[i] * W[L + i][c];
    acc *= beta;
#pragma unroll
    for (int i = 0; i < LEN; ++i) W[L + i][c] -= acc * v[i];
  }
#pragma unroll
  for (int a = 0; a < S; ++a) {
    R acc = R(0);
#pragma unroll
    for (int i = 0; i < LEN; ++i) acc += Qs[a][L + i] * v[i];
    acc *= beta;
#pragma unroll
    for (int i = 0; i < LEN; ++i) Qs[a][L + i] -= acc * v[i];
  }
}

// T (rows / columns j..j+S-1) <- G^T T G and Z <- Z G for an orthogonal S x S G
// (transpose: G^T in place of G), lanes over columns, then rows.
template <int S, bool TR, class R>
__device__ __forceinline__ void apply_similarity(int n, R* T, int ldt, R* Z, int ldz, int nz, int j, const R (&G)[S][S],
                                                 int lane) {
  for (int c = j + lane; c < n; c += 32) {
    R tmp[S];
#pragma unroll
    for (int a = 0; a < S; ++a) {
      R acc = R(0);
#pragma unroll
      for (int b = 0; b < S; ++b) acc += (TR ? G[a][b] : G[b][a]) * at(T, ldt, j + b, c);
      tmp[a] = acc;
    }
#pragma unroll
    for (int a = 0; a < S; ++a) at(T, ldt, j + a, c) = tmp[a];
  }
  __syncwarp();
  for (int rr = lane; rr < j + S; rr += 32) {
    R tmp[S];
#pragma unroll
    for (int a = 0; a < S; ++a) {
      R acc = R(0);
#pragma unroll
      for (int b = 0; b < S; ++b) acc += at(T, ldt, rr, j + b) * (TR ? G[a][b] : G[b][a]);
      tmp[a] = acc;
    }
#pragma unroll
    for (int a = 0; a < S; ++a) at(T, ldt, rr, j + a) = tmp[a];
  }
  if (Z)
    for (int rr = lane; rr < nz; rr += 32) {
      R tmp[S];
#pragma unroll
      for (int a = 0; a < S; ++a) {
        R acc = R(0);
#pragma unroll
        for (int b = 0; b < S; ++b) acc += at(Z, ldz, rr, j + b) * (TR ? G[a][b] : G[b][a]);
        tmp[a] = acc;
      }
#pragma unroll
      for (int a = 0; a < S; ++a) at(Z, ldz, rr, j + a) = tmp[a];
    }
  __syncwarp();
}

// Swap the adjacent diagonal blocks at j (sizes P then Q, not both 1): the
// Sylvester equation T11 X - X T22 = -T12, then the orthogonal factor of the
// QR of [X; I] moves T22's block to the top (Bai & Demmel).  0 on success,
// -1 / -2 when refused (T and Z unchanged).
template <int P, int Q, class R>
__device__ inline int swap_pq(int n, R* T, int ldt, R* Z, int ldz, int nz, int j, int lane) {
  constexpr int S = P + Q, PQ = P * Q;
  R M[PQ][PQ], r[PQ];
#pragma unroll
  for (int a = 0; a < PQ; ++a) {
    r[a] = R(0);
#pragma unroll
    for (int b = 0; b < PQ; ++b) M[a][b] = R(0);
  }
#pragma unroll
  for (int l = 0; l < Q; ++l)
#pragma unroll
    for (int i = 0; i < P; ++i) {
      const int row = i + P * l;
#pragma unroll
      for (int ii = 0; ii < P; ++ii) M[row][ii + P * l] += at(T, ldt, j + i, j + ii);
#pragma unroll
      for (int ll = 0; ll < Q; ++ll) M[row][i + P * ll] -= at(T, ldt, j + P + ll, j + P + l);
      r[row] = -at(T, ldt, j + i, j + P + l);
    }
  if (!small_solve<PQ>(M, r)) { __syncwarp(); return -1; }
  R W[S][Q];
#pragma unroll
  for (int l = 0; l < Q; ++l) {
#pragma unroll
    for (int i = 0; i < P; ++i) W[i][l] = r[i + P * l];
#pragma unroll
    for (int i = 0; i < Q; ++i) W[P + i][l] = (i == l) ? R(1) : R(0);
  }
  R Qs[S][S];
#pragma unroll
  for (int a = 0; a < S; ++a)
#pragma unroll
    for (int b = 0; b < S; ++b) Qs[a][b] = (a == b) ? R(1) : R(0);
  qr_step<S, Q, 0>(W, Qs);
  if (Q == 2) qr_step<S, Q, (Q == 2 ? 1 : 0)>(W, Qs);
  R wnorm = R(0);
#pragma unroll
  for (int a = 0; a < S; ++a)
#pragma unroll
    for (int b = 0; b < S; ++b) wnorm = rmax(wnorm, rabs(at(T, ldt, j + a, j + b)));
  __syncwarp();
  apply_similarity<S, false>(n, T, ldt, Z, ldz, nz, j, Qs, lane);
  R lower = R(0);
#pragma unroll
  for (int a = Q; a < S; ++a)
#pragma unroll
    for (int b = 0; b < Q; ++b) lower = rmax(lower, rabs(at(T, ldt, j + a, j + b)));
  __syncwarp();
  if (lower > R(1000) * reps<R>() * rmax(wnorm, R(1e-30f))) {   // refused: undo
    apply_similarity<S, true>(n, T, ldt, Z, ldz, nz, j, Qs, lane);
    return -2;
  }
  if (lane == 0) {
    for (int a = Q; a < S; ++a) for (int b = 0; b < Q; ++b) at(T, ldt, j + a, j + b) = R(0);
    for (int c = 0; c < j; ++c) for (int a = 0; a < S; ++a) at(T, ldt, j + a, c) = R(0);
  }
  __syncwarp();
  if (Q == 2) standardize_2x2(n, T, ldt, Z, ldz, nz, j, lane);
  if (P == 2) standardize_2x2(n, T, ldt, Z, ldz, nz, j + Q, lane);
  if (lane == 0)
    for (int a = 0; a < S; ++a)
      for (int b = 0; b < S; ++b)
        if (a > b + 1) at(T, ldt, j + a, j + b) = R(0);
  __syncwarp();
  return 0;
}

// Swap the adjacent diagonal blocks at j (sizes p then q); 0 on success,
// -1 / -2 when refused (T and Z unchanged).
template <class R>
__device__ inline int swap_blocks(int n, R* T, int ldt, R* Z, int ldz, int nz, int j, int p, int q, int lane) {
  if (p == 1 && q == 1) {
    swap_singles(n, T, ldt, Z, ldz, nz, j, lane);
    return 0;
  }
  if (p == 1) return swap_pq<1, 2>(n, T, ldt, Z, ldz, nz, j, lane);
  if (q == 1) return swap_pq<2, 1>(n, T, ldt, Z, ldz, nz, j, lane);
  return swap_pq<2, 2>(n, T, ldt, Z, ldz, nz, j, lane);
}

// Move the best diagonal blocks (by key; ties by position) covering `want`
// columns, pairs whole, to the top, keeping their relative order (the
// selection of Algorithm 1's truncation): each selected block, top to bottom,
// is swapped up past the unselected blocks above it.  keys: scratch of n
// values (shared memory).  Returns the number of leading columns that hold
// selected blocks (want or want + 1, fewer only if a swap was refused).
// n <= kMaxM; the selection is a bit mask of rows.
template <class R>
__device__ inline int reorder_select(int n, R* T, int ldt, R* Z, int ldz, int nz, int which, int want, R* keys,
                                     int lane) {
  for (int i = lane; i < n; i += 32) {   // key of the block starting at i (rows that start none: unused)
    const bool second = i > 0 && at(T, ldt, i, i - 1) != R(0);
    if (!second) {
      const Block<R> b = block_at(T, ldt, i, n);
      keys[i] = key(b.re, b.im, which);
    }
  }
  __syncwarp();
  uint64_t sel = 0;
  int cols = 0;
  while (cols < want) {
    int best = -1, bsz = 0;
    R bk = R(0);
    for (int i = 0; i < n;) {
      const int sz = (i + 1 < n && at(T, ldt, i + 1, i) != R(0)) ? 2 : 1;
      if (!((sel >> i) & 1ull) && (best < 0 || keys[i] < bk)) { best = i; bk = keys[i]; bsz = sz; }
      i += sz;
    }
    if (best < 0) break;
    sel |= (bsz == 2 ? 3ull : 1ull) << best;
    cols += bsz;
  }
  __syncwarp();
  int top = 0;
  for (int placed = 0; placed < n && top < n; ++placed) {
    int i = top;   // the first selected block at or below top (the blocks between are unselected)
    while (i < n && !((sel >> i) & 1ull)) i += (i + 1 < n && at(T, ldt, i + 1, i) != R(0)) ? 2 : 1;
    if (i >= n) break;
    int size = (i + 1 < n && at(T, ldt, i + 1, i) != R(0)) ? 2 : 1;
    int cur = i;
    bool refused = false;
    for (int guard = 0; cur > top && guard < n; ++guard) {
      const int up_start = (cur - 2 >= top && at(T, ldt, cur - 1, cur - 2) != R(0)) ? cur - 2 : cur - 1;
      const int up_size = cur - up_start;
      const int rc = swap_blocks(n, T, ldt, Z, ldz, nz, up_start, up_size, size, lane);
      if (rc != 0) { refused = true; break; }
      sel |= ((1ull << size) - 1ull) << up_start;
      sel &= ~(((1ull << up_size) - 1ull) << (up_start + size));
      cur = up_start;
      size = (cur + 1 < n && at(T, ldt, cur + 1, cur) != R(0)) ? 2 : 1;   // a standardised pair may be real
    }
    __syncwarp();
    if (refused) break;
    top = cur + size;
  }
  return top;
}

// Eigenvalues and unit eigenvectors of a quasi-triangular T (n x n): column c
// of (Yre, Yim) (ld ldy) for eigenvalue c in block order (a pair: Im > 0
// first).  Lanes take one eigenvector each: back substitution through the
// blocks above the eigenvalue's own, read from T's subdiagonal.
template <class R>
__device__ inline void quasi_eig(int n, const R* T, int ldt, R* lre, R* lim, R* Yre, R* Yim, int ldy, int lane) {
  R tnorm = R(0);
  for (int j = lane; j < n; j += 32)
    for (int i = 0; i <= min(j + 1, n - 1); ++i) tnorm = rmax(tnorm, rabs(at(T, ldt, i, j)));
  tnorm = warp_allmax(tnorm);
  const R small = rmax(tnorm * reps<R>(), R(1e-30f));
  for (int c = lane; c < n; c += 32) {
    int start = 0;   // the block holding column c
    while (true) {
      const int sz = (start + 1 < n && at(T, ldt, start + 1, start) != R(0)) ? 2 : 1;
      if (c < start + sz) break;
      start += sz;
    }
    const Block<R> B = block_at(T, ldt, start, n);
    const int e = c - start;
    const R lr = B.re, li = B.size == 2 ? (e == 0 ? B.im : -B.im) : R(0);
    R* yr = Yre + c * ldy;
    R* yi = Yim + c * ldy;
    for (int i = 0; i < n; ++i) { yr[i] = R(0); yi[i] = R(0); }
    if (B.size == 1) {
      yr[B.start] = R(1);
    } else {
      yr[B.start] = at(T, ldt, B.start, B.start + 1);
      yr[B.start + 1] = lr - at(T, ldt, B.start, B.start);
      yi[B.start + 1] = li;
    }
    const int last = B.start + B.size - 1;
    int bot = B.start - 1;   // bottom row of the next block above
    while (bot >= 0) {
      const int csz = (bot >= 1 && at(T, ldt, bot, bot - 1) != R(0)) ? 2 : 1;
      const int cs0 = bot - csz + 1;
      R rr0 = R(0), ri0 = R(0), rr1 = R(0), ri1 = R(0);
      for (int l = cs0 + csz; l <= last; ++l) {
        const R t0 = at(T, ldt, cs0, l);
        rr0 -= t0 * yr[l];
        ri0 -= t0 * yi[l];
        if (csz == 2) {
          const R t1 = at(T, ldt, cs0 + 1, l);
          rr1 -= t1 * yr[l];
          ri1 -= t1 * yi[l];
        }
      }
      if (csz == 1) {
        R dr = at(T, ldt, cs0, cs0) - lr, di = -li;
        if (rhypot(dr, di) < small) { dr = small; di = R(0); }
        const R den = R(1) / (dr * dr + di * di);
        yr[cs0] = (rr0 * dr + ri0 * di) * den;
        yi[cs0] = (ri0 * dr - rr0 * di) * den;
      } else {
        const R m00r = at(T, ldt, cs0, cs0) - lr, m00i = -li;
        const R m01 = at(T, ldt, cs0, cs0 + 1), m10 = at(T, ldt, cs0 + 1, cs0);
        const R m11r = at(T, ldt, cs0 + 1, cs0 + 1) - lr, m11i = -li;
        R detr = m00r * m11r - m00i * m11i - m01 * m10, deti = m00r * m11i + m00i * m11r;
        if (rhypot(detr, deti) < small * small) { detr = small * small; deti = R(0); }
        const R dd = R(1) / (detr * detr + deti * deti);
        const R n0r = rr0 * m11r - ri0 * m11i - m01 * rr1, n0i = rr0 * m11i + ri0 * m11r - m01 * ri1;
        const R n1r = m00r * rr1 - m00i * ri1 - m10 * rr0, n1i = m00r * ri1 + m00i * rr1 - m10 * ri0;
        yr[cs0] = (n0r * detr + n0i * deti) * dd;
        yi[cs0] = (n0i * detr - n0r * deti) * dd;
        yr[cs0 + 1] = (n1r * detr + n1i * deti) * dd;
        yi[cs0 + 1] = (n1i * detr - n1r * deti) * dd;
      }
      bot = cs0 - 1;
    }
    // unit norm (scaled, so that the squares neither overflow nor underflow)
    R mx = R(0);
    for (int i = 0; i <= last; ++i) mx = rmax(mx, rmax(rabs(yr[i]), rabs(yi[i])));
    const R imx = R(1) / mx;
    R nrm = R(0);
    for (int i = 0; i <= last; ++i) {
      const R a = yr[i] * imx, b = yi[i] * imx;
      nrm += a * a + b * b;
    }
    const R inv = imx / rsqrt_(nrm);
    for (int i = 0; i <= last; ++i) { yr[i] *= inv; yi[i] *= inv; }
    lre[c] = lr;
    lim[c] = li;
  }
  __syncwarp();
}

}  // namespace rks_dd
