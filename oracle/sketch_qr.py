"""Randomized QR factorisations of a tall and skinny K: plain FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module.

Sec. 2 of the paper lists the randomized orthogonalisation processes an rKS
basis can be built with; each takes K (n x s) to K = Q R with R upper
triangular:

* RGS, randomized Gram-Schmidt (the process of Algorithm 2, without A): for
  each column k_j, r = S_j^+ (Omega k_j) (least squares in the sketch),
  q~ = k_j - Q_j r, s~ = Omega q~, beta = ||s~||, q_j = q~ / beta,
  s_j = s~ / beta, R[:j, j] = r, R[j, j] = beta.  Omega Q is orthonormal.
* Sketch and whiten (the whitening of Sec. 3.3 applied to a whole block):
  Omega K = Q_s R (Householder QR, positive diagonal), Q = K R^{-1}.
  Omega Q = Q_s is orthonormal.
* Randomized Cholesky QR: Q_1, R_1 from sketch and whiten, then Cholesky QR
  of the well-conditioned Q_1: Q_1^T Q_1 = R_2^T R_2, Q = Q_1 R_2^{-1},
  R = R_2 R_1.  Q is orthonormal (Euclidean).

A sketch-orthonormal factorisation K = Q R with R upper triangular and a
positive diagonal is unique (R is the R factor of Omega K), so RGS and sketch
and whiten compute the same Q and R in exact arithmetic; randomized Cholesky
QR computes the Euclidean QR factorisation of K.  The tests pin each function
against the other and against LAPACK's QR.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def _positive_qr(X: np.ndarray):
    """Householder QR with a positive diagonal of R (LAPACK, then signs)."""
    Qx, Rx = np.linalg.qr(X)
    sgn = np.sign(np.diag(Rx))
    sgn[sgn == 0] = 1.0
    return Qx * sgn, (Rx.T * sgn).T


def rgs(K: np.ndarray, Omega) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Randomized Gram-Schmidt, column by column.  Returns Q, R, S = Omega Q."""
    K = np.asarray(K, dtype=np.float64)
    n, s = K.shape
    d = Omega.shape[0]
    Q = np.zeros((n, s))
    S = np.zeros((d, s))
    R = np.zeros((s, s))
    for j in range(s):
        z = Omega @ K[:, j]                                  # sketch of the new column
        r = np.linalg.lstsq(S[:, :j], z, rcond=None)[0] if j else np.zeros(0)
        qt = K[:, j] - Q[:, :j] @ r                          # q~ = k_j - Q_j r
        st = Omega @ qt                                      # s~ = Omega q~
        beta = np.linalg.norm(st)
        Q[:, j] = qt / beta
        S[:, j] = st / beta
        R[:j, j] = r
        R[j, j] = beta
    return Q, R, S


def sketch_whiten(K: np.ndarray, Omega) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Omega K = Q_s R, Q = K R^{-1}.  Returns Q, R, S = Q_s."""
    K = np.asarray(K, dtype=np.float64)
    Qs, R = _positive_qr(Omega @ K)
    Q = sla.solve_triangular(R, K.T, trans="T", lower=False).T   # K R^{-1}
    return Q, R, Qs


def rcholqr(K: np.ndarray, Omega) -> tuple[np.ndarray, np.ndarray]:
    """Sketch and whiten, then Cholesky QR of Q_1.  Returns Q, R."""
    Q1, R1, _ = sketch_whiten(K, Omega)
    R2 = np.linalg.cholesky(Q1.T @ Q1).T                 # upper, positive diagonal
    Q = sla.solve_triangular(R2, Q1.T, trans="T", lower=False).T
    return Q, R2 @ R1
