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

* RHQR, randomized Householder QR: Householder QR carried out in the
  sketched space of Theta = [[I_s, 0], [0, Omega']] (the first s rows kept
  exactly, the other n - s sketched by Omega').  For column j the reflector
  of the sketched column y = Theta x (entries above j dropped) is
  v = y - rho e_j, rho = -sign(y_j) ||y||, beta = 2 / v^T v; its n-dimensional
  counterpart u (x with entries above j dropped and rho taken off entry j)
  has Theta u = v, and H_j = I - beta u (Theta u)^T Theta satisfies
  Theta H_j = (I - beta v v^T) Theta.  H_j is applied to the later columns,
  R[:j, j] = y[:j], R[j, j] = rho, and Q = H_0 ... H_{s-1} [I_s; 0]
  (accumulated backwards).  Theta Q is orthonormal.

A sketch-orthonormal factorisation K = Q R with R upper triangular and a
positive diagonal is unique (R is the R factor of Omega K), so RGS and sketch
and whiten compute the same Q and R in exact arithmetic, and RHQR the same as
both with Omega = Theta; randomized Cholesky QR computes the Euclidean QR
factorisation of K.  With Omega' = I (Theta = I) RHQR is Householder QR.  The
tests pin each function against the others and against LAPACK's QR.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


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


def theta_matrix(n: int, s: int, Omega_bottom):
    """Theta = [[I_s, 0], [0, Omega']] ((s + d) x n) for RHQR."""
    return sp.block_diag([sp.identity(s, format="csr"), sp.csr_matrix(Omega_bottom)], format="csr")


def rhqr(K: np.ndarray, Omega_bottom) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Randomized Householder QR with Theta = [[I_s, 0], [0, Omega_bottom]].

    Returns Q (n x s), R (s x s, positive diagonal) and Theta Q ((s + d) x s).
    The reflectors are applied to the n-dimensional columns themselves; their
    coefficients come from the sketched columns Theta x.
    """
    K = np.array(K, dtype=np.float64)
    n, s = K.shape
    Th = theta_matrix(n, s, Omega_bottom)
    X = K.copy()
    Us, Vs, betas = [], [], []
    R = np.zeros((s, s))
    for j in range(s):
        x = X[:, j]
        y = Th @ x                                   # sketched column
        yv = y.copy()
        yv[:j] = 0.0
        nrm = np.linalg.norm(yv)
        rho = -nrm if yv[j] >= 0 else nrm            # rho = -sign(y_j) ||y||
        v = yv.copy()
        v[j] -= rho                                  # v = y - rho e_j
        u = x.copy()
        u[:j] = 0.0
        u[j] -= rho                                  # Theta u = v
        beta = 2.0 / (v @ v)
        R[:j, j] = y[:j]
        R[j, j] = rho
        for l in range(j + 1, s):                    # H_j applied to the later columns
            X[:, l] -= beta * (v @ (Th @ X[:, l])) * u
        Us.append(u)
        Vs.append(v)
        betas.append(beta)
    Q = np.zeros((n, s))
    Q[np.arange(s), np.arange(s)] = 1.0              # [I_s; 0]
    for j in range(s - 1, -1, -1):                   # Q = H_0 ... H_{s-1} [I_s; 0]
        c = betas[j] * (Vs[j] @ (Th @ Q))
        Q -= np.outer(Us[j], c)
    sgn = np.sign(np.diag(R))
    sgn[sgn == 0] = 1.0
    Q = Q * sgn
    R = (R.T * sgn).T
    return Q, R, Th @ Q
