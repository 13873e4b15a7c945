"""Randomized Krylov-Schur with deflation: plain FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module.

The code follows the paper's algorithms step by step, in its notation:

* Algorithm 2 (extend an rKS factorization, Sec. 3.1): for j = k+1..m,
  w_j = A u_j; z_j = Omega w_j; b_{j+1} = S_j^+ z_j;
  u~_{j+1} = w_j - U_j b_{j+1}; s~_{j+1} = Omega u~_{j+1};
  beta_{j+1} = ||s~_{j+1}||; append u~/beta, s~/beta, and the column
  (b_{j+1}; beta_{j+1}) of B.  With k = 0 it starts from
  u_1 = u~_1/||Omega u~_1|| (Sec. 3.1, text before Algorithm 2).
* Deflation (Sec. 4.2-4.3, Thm 4.3): with q locked sketch-orthonormal Schur
  vectors U_q, the expansion applies the deflated operator
  A_q = (I - U_q (Omega U_q)^+ Omega) A, i.e. step "w_j = A u_j" becomes
  w_j = A u_j - U_q (Omega U_q)^+ Omega A u_j; the projections against U_q
  and U_j are taken as one least-squares problem (Thm 4.3: sequential and
  at-once deflation coincide).  The discarded coefficients
  (Omega U_q)^+ Omega A u_j are kept as the coupling block T_qa of the full
  upper-triangular Rayleigh quotient of A (reading: the paper leaves the
  recovery of A's eigenvectors implicit; Thm 4.3's third item guarantees that
  [U_q U_r] are Schur vectors of A).
* Algorithm 1 (rKS, Sec. 3.1): Schur form B = Q1 T Q1^T, reordering by an
  orthogonal Q2 so that the wanted eigenvalues lead, truncation
  U <- U Q1 Q2 (e_1..e_k), S <- S Q1 Q2 (e_1..e_k), b^T <- b^T Q1 Q2 (e_1..e_k),
  u and s unchanged (Eqs. 3.5-3.6), Ritz pairs of T and the residual
  estimates |b^T y| / |lambda| (Sec. 4.1, Eq. 4.8), then extension.
* Locking (Sec. 4.4, Eq. 4.21): a leading block of active Schur vectors whose
  entries of b are below the threshold is moved to U_q and its b set to zero.
* Aggressive deflation (option; Sec. 4.3, after Thm 4.3): before locking,
  the active Schur form is reordered so that every block whose Ritz
  estimate |b^T y| is below the locking threshold leads.
* Whitening (Sec. 3.3, Eqs. 3.7-3.8): S_k = QR (Householder),
  U <- U R^{-1}, T <- R T R^{-1}, b^T <- b^T R^{-1}.

Readings where the paper is silent (each also listed in the design notes):
* the locking threshold is relative: |b_i| <= eta_lock * max(|lambda_i|,
  eps ||T||_F), lambda_i the eigenvalue of the diagonal block holding i, and a
  2x2 block is locked whole;
* locked vectors count in the Krylov dimension: the expansion runs the active
  part from k - q to m - q columns and the restart keeps k columns in all;
* the truncation keeps k - q active columns, one more if that cut would split a
  2x2 block;
* wanted eigenvalues are ordered by key (LM: -|l|, SM: |l|, LR: -Re l,
  SR: Re l), best first; ties keep the order of the Schur form;
* convergence: every one of the k estimates |b^T y_i|/|lambda_i| <= tol
  (Sec. 5.1), or all k vectors locked;
* whitening is applied at a restart when ||S_a^T S_a - I||_F > 1e-10;
* an exact breakdown (beta <= 1e-14 ||Omega w||) raises ``Breakdown``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
from scipy.linalg.lapack import dtrsen

from .sketch import omega_matrix

WHICH = ("LM", "SM", "LR", "SR")


class Breakdown(RuntimeError):
    """beta_{j+1} vanished: an invariant subspace was found (Sec. 2.1)."""


def key(lam, which: str):
    """Ordering key of eigenvalues: smaller key = more wanted."""
    lam = np.asarray(lam)
    if which == "LM":
        return -np.abs(lam)
    if which == "SM":
        return np.abs(lam)
    if which == "LR":
        return -lam.real
    if which == "SR":
        return lam.real
    raise ValueError(which)


# ---------------------------------------------------------------------------
# Small dense FP64 pieces (library primitives: LAPACK via scipy)
# ---------------------------------------------------------------------------

def schur_blocks(T: np.ndarray):
    """Diagonal blocks of a real quasi-triangular T: list of (start, size)."""
    m = T.shape[0]
    out, i = [], 0
    while i < m:
        if i + 1 < m and T[i + 1, i] != 0.0:
            out.append((i, 2)); i += 2
        else:
            out.append((i, 1)); i += 1
    return out


def block_eigenvalue(T: np.ndarray, start: int, size: int) -> complex:
    """Eigenvalue of a diagonal block (the one with Im >= 0 for a 2x2 block)."""
    if size == 1:
        return complex(T[start, start])
    ev = np.linalg.eigvals(T[start:start + 2, start:start + 2])
    return complex(ev[np.argmax(ev.imag)])


def ordered_schur(B: np.ndarray, which: str, nsort: int):
    """Real Schur form B = Q T Q^T with the wanted eigenvalues leading.

    Alg. 1, Schur step and reordering step (Prop. 2.8: any order is reachable
    by orthogonal similarity).  The best ``nsort`` diagonal blocks by key are
    moved to the top, best first, by repeated LAPACK dtrsen calls (each call
    moves the selected set to the top and keeps its relative order, so
    selecting the best r blocks after the best r-1 are in place puts block r
    right below them).
    """
    T, Q = sla.schur(np.asarray(B, dtype=np.float64), output="real")
    for r in range(1, nsort + 1):
        blocks = schur_blocks(T)
        if r > len(blocks):
            break
        keys = np.array([key(block_eigenvalue(T, s, z), which) for s, z in blocks])
        best = np.argsort(keys, kind="stable")[:r]
        select = np.zeros(T.shape[0], dtype=np.int32)
        for b in best:
            s, z = blocks[b]
            select[s:s + z] = 1
        T, Q, _, _, _, _, _, info = dtrsen(select, T, Q, job="N")
        if info != 0:
            raise RuntimeError(f"dtrsen failed: info={info}")
    return T, Q


def truncation_size(T: np.ndarray, want: int) -> int:
    """Number of leading columns holding ``want`` eigenvalues, blocks kept whole."""
    size = 0
    for s, z in schur_blocks(T):
        if size >= want:
            break
        size = s + z
    return size


def ritz(T: np.ndarray, b: np.ndarray, which: str, norm_a: float | None = None):
    """Ritz values, unit-norm eigenvectors y of T, and the residual estimates.

    estimate_i = |b^T y_i| / |lambda_i| (Eq. 4.8), or |b^T y_i| / ||A||_1 (the
    non-relative bound of the Sec. 4.1 remark scaled by ||A||_1) when
    ``norm_a`` is given; sorted by key (best first).
    """
    lam, Y = sla.eig(T)
    Y = Y / np.linalg.norm(Y, axis=0)
    order = np.argsort(key(lam, which), kind="stable")
    lam, Y = lam[order], Y[:, order]
    den = norm_a if norm_a is not None else np.maximum(np.abs(lam), np.finfo(float).tiny)
    est = np.abs(b @ Y) / den
    return lam, Y, est


# ---------------------------------------------------------------------------
# The decomposition and its two operations
# ---------------------------------------------------------------------------

@dataclass
class RKSState:
    """A partitioned rKS decomposition (Thm 4.3 layout).

    A [U_q U_a] = [U_q U_a] [[T_qq, T_qa], [0, B_a]] + u [0, b_a]^T, with
    (Omega [U_q U_a u]) orthonormal.  Columns are stored column-major.
    During an expansion U_a holds the active basis plus its last vector.
    """
    A: sp.csr_matrix
    Omega: sp.csr_matrix
    Uq: np.ndarray          # n x q   locked vectors
    Sq: np.ndarray          # d x q   their sketches
    Tqq: np.ndarray         # q x q
    Tqa: np.ndarray         # q x ja  coupling of locked and active columns
    Ua: np.ndarray          # n x (ja+1) active basis and last vector u
    Sa: np.ndarray          # d x (ja+1)
    Ba: np.ndarray          # (ja+1) x ja: [B_a; b_a^T]
    nmatvec: int = 0

    @property
    def q(self) -> int:
        return self.Uq.shape[1]

    @property
    def ja(self) -> int:
        return self.Ba.shape[1]


def start(A, Omega, u1: np.ndarray) -> RKSState:
    """Initial vector of Alg. 2 with k = 0: u_1 = u~_1 / ||Omega u~_1||."""
    n = A.shape[0]
    d = Omega.shape[0]
    s = Omega @ u1
    beta = np.linalg.norm(s)
    return RKSState(A=A, Omega=Omega,
                    Uq=np.zeros((n, 0), order="F"), Sq=np.zeros((d, 0), order="F"),
                    Tqq=np.zeros((0, 0)), Tqa=np.zeros((0, 0)),
                    Ua=np.asfortranarray((u1 / beta)[:, None]),
                    Sa=np.asfortranarray((s / beta)[:, None]),
                    Ba=np.zeros((1, 0)))


def extend(st: RKSState, m_active: int) -> None:
    """Algorithm 2: extend the active factorization to ``m_active`` columns.

    Every step follows the algorithm's order; with locked vectors the product
    with A is replaced by the deflated operator of Sec. 4.3, and the two
    sketch-orthogonalisations (against U_q, then U_j) are done as one
    least-squares problem against [S_q S_j], which Thm 4.3 shows to be the same
    operator.  Done one after the other in floating point, a component along U_q
    left in U_j re-enters every new vector amplified by ||b||/beta; under LR/SM
    the zero eigenvalues of A_q are the wanted ones and the restart filter then
    grows that component exponentially.
    """
    A, Om = st.A, st.Omega
    n, d = A.shape[0], Om.shape[0]
    j0 = st.ja
    q = st.q
    U = np.zeros((n, m_active + 1), order="F"); U[:, :j0 + 1] = st.Ua
    S = np.zeros((d, m_active + 1), order="F"); S[:, :j0 + 1] = st.Sa
    B = np.zeros((m_active + 1, m_active)); B[:j0 + 1, :j0] = st.Ba
    Tqa = np.zeros((q, m_active)); Tqa[:, :j0] = st.Tqa
    for j in range(j0, m_active):          # 0-based: u_j is column j
        w = A @ U[:, j]                     # w_j = A u_j
        st.nmatvec += 1
        z = Om @ w                          # z_j = Omega w_j
        # b_{j+1} = S_j^+ z_j; with locked vectors the sketch-orthogonalisation
        # against U_q (deflated operator A_q, Sec. 4.3) is the same least-squares
        # problem taken against [S_q S_j] at once (Thm 4.3).
        y = np.linalg.lstsq(np.hstack([st.Sq, S[:, :j + 1]]), z, rcond=None)[0]
        cq, bj = y[:q], y[q:]
        Tqa[:, j] = cq                      # (Omega U_q)^+ Omega A u_j, kept as T_qa
        ut = w - st.Uq @ cq - U[:, :j + 1] @ bj   # u~_{j+1} = A_q u_j - U_j b_{j+1}
        st_ = Om @ ut                       # s~_{j+1} = Omega u~_{j+1}
        beta = np.linalg.norm(st_)          # beta_{j+1} = ||s~_{j+1}||
        if not beta > 1e-14 * np.linalg.norm(z):
            raise Breakdown(f"beta = {beta:.3e} at column {j + 1}")
        U[:, j + 1] = ut / beta
        S[:, j + 1] = st_ / beta
        B[:j + 1, j] = bj
        B[j + 1, j] = beta
    st.Ua, st.Sa, st.Ba, st.Tqa = U, S, B, Tqa


def whiten(st: RKSState) -> None:
    """Sec. 3.3: S_a = QR (Householder), U_a <- U_a R^{-1}, B <- R B R^{-1}, b <- R^{-T} b.

    Applied to the active columns of a contracted decomposition (the last
    vector u and the locked block are left as they are).
    """
    ja = st.ja
    Qs, R = np.linalg.qr(st.Sa[:, :ja])
    sgn = np.sign(np.diag(R)); sgn[sgn == 0] = 1.0
    Qs, R = Qs * sgn, (R.T * sgn).T       # positive diagonal
    Rinv = sla.solve_triangular(R, np.eye(ja))
    st.Ua[:, :ja] = st.Ua[:, :ja] @ Rinv
    st.Sa[:, :ja] = Qs
    Ta, b = st.Ba[:ja, :], st.Ba[ja, :]
    st.Ba = np.vstack([R @ Ta @ Rinv, b @ Rinv])
    st.Tqa = st.Tqa @ Rinv


def contract(st: RKSState, k: int, which: str, keep: int = 0):
    """Alg. 1 contraction: Schur form, reordering, truncation of the active part.

    The active part keeps its k - q best Schur vectors (Alg. 1 truncates to
    k), or, with ``keep`` > 0, max(k - q, min(keep, ma // 2)) of them: after
    q vectors are locked the restart still carries up to ``keep`` active
    directions (a thick restart, Sec. 2.3's truncation with a larger size).
    Returns (T_a, b_a, Q) where Q (ma x ka) are the kept Schur vectors.
    """
    ma = st.ja
    Ba, b = st.Ba[:ma, :], st.Ba[ma, :]
    want = k - st.q
    if keep:
        want = max(want, min(keep, ma // 2))
    # sort enough blocks to cover ``want`` columns plus a possible pair
    T, Q = ordered_schur(Ba, which, nsort=min(want + 1, ma))
    ka = min(truncation_size(T, want), ma - 1)
    Qk = Q[:, :ka]
    st.Ua = np.asfortranarray(np.hstack([st.Ua[:, :ma] @ Qk, st.Ua[:, ma:ma + 1]]))
    st.Sa = np.asfortranarray(np.hstack([st.Sa[:, :ma] @ Qk, st.Sa[:, ma:ma + 1]]))
    Ta = T[:ka, :ka]
    bk = b @ Qk
    st.Ba = np.vstack([Ta, bk])
    st.Tqa = st.Tqa @ Qk
    return Ta, bk, Qk


def block_eigvec(T: np.ndarray, start: int, size: int):
    """Eigenvalue and unit eigenvector y of a quasi-triangular T for its
    diagonal block at ``start`` (the Im >= 0 member of a pair).

    T is block upper triangular, so y is zero below the block, the block's own
    eigenvector inside it, and above it the solution of
    (T_11 - lambda I) x = -T_12 v (the first start + size entries are the only
    nonzero ones: the observation of the remark after Eq. 4.21).
    """
    lam = block_eigenvalue(T, start, size)
    e = start + size
    if size == 1:
        v = np.ones(1, dtype=complex)
    else:
        w, V = np.linalg.eig(T[start:e, start:e])
        v = V[:, np.argmax(w.imag)]
    y = np.zeros(T.shape[0], dtype=complex)
    y[start:e] = v
    if start:
        y[:start] = np.linalg.solve(T[:start, :start] - lam * np.eye(start), -(T[:start, start:e] @ v))
    return lam, y / np.linalg.norm(y)


def aggressive_reorder(st: RKSState, eta_lock: float, norm_a: float | None = None) -> int:
    """Aggressive deflation (Sec. 4.3, after Thm 4.3): reorder the active part
    so that every converged Schur block comes first, ready to be locked.

    The factorization can be reordered by any orthogonal similarity that keeps
    T_a quasi-triangular; moving a block to the front makes its eigenvector
    the leading Schur vector, whose entry of b is then b^T y (unit y).  A
    block counts as converged when |b^T y| is below the locking threshold of
    ``lock`` (the same scale).  Converged blocks move to the front in their
    current order and the others follow in theirs (LAPACK dtrsen); U_a, S_a,
    b and T_qa take the same rotation.  Returns the number of converged
    columns; nothing moves when they already lead or a swap is refused.
    """
    ja = st.ja
    if ja == 0:
        return 0
    Ta, b = st.Ba[:ja, :], st.Ba[ja, :]
    scale = np.finfo(float).eps * np.linalg.norm(Ta)
    select = np.zeros(ja, dtype=np.int32)
    for s, z in schur_blocks(Ta):
        lam, y = block_eigvec(Ta, s, z)
        thr = eta_lock * (norm_a if norm_a is not None else max(abs(lam), scale))
        if abs(b @ y) <= thr:
            select[s:s + z] = 1
    nsel = int(select.sum())
    if nsel == 0 or np.all(select[:nsel] == 1):
        return nsel
    T2, Z, _, _, _, _, _, info = dtrsen(select, Ta, np.eye(ja), job="N")
    if info != 0:
        return 0
    st.Ba = np.vstack([T2, b @ Z])
    st.Ua = np.asfortranarray(np.hstack([st.Ua[:, :ja] @ Z, st.Ua[:, ja:]]))
    st.Sa = np.asfortranarray(np.hstack([st.Sa[:, :ja] @ Z, st.Sa[:, ja:]]))
    st.Tqa = st.Tqa @ Z
    return nsel


def lock(st: RKSState, k: int, eta_lock: float, norm_a: float | None = None) -> int:
    """Sec. 4.4 locking: move the leading active blocks with small |b| to U_q.

    The threshold is eta_lock * |lambda| of the block, or the absolute
    threshold of Eq. 4.21 with eta = eta_lock * ||A||_1 when ``norm_a`` is
    given.  Returns the number of vectors locked now.
    """
    ja = st.ja
    Ta, b = st.Ba[:ja, :], st.Ba[ja, :]
    scale = np.finfo(float).eps * np.linalg.norm(Ta)
    r = 0
    for s, z in schur_blocks(Ta):
        if st.q + r + z > k:
            break
        lam = abs(block_eigenvalue(Ta, s, z))
        thr = eta_lock * (norm_a if norm_a is not None else max(lam, scale))
        if np.all(np.abs(b[s:s + z]) <= thr):
            r = s + z
        else:
            break
    if r == 0:
        return 0
    q = st.q
    Tqq = np.zeros((q + r, q + r))
    Tqq[:q, :q] = st.Tqq
    Tqq[:q, q:] = st.Tqa[:, :r]
    Tqq[q:, q:] = Ta[:r, :r]
    st.Tqq = Tqq
    st.Tqa = np.vstack([st.Tqa[:, r:], Ta[:r, r:]])
    st.Uq = np.asfortranarray(np.hstack([st.Uq, st.Ua[:, :r]]))
    st.Sq = np.asfortranarray(np.hstack([st.Sq, st.Sa[:, :r]]))
    st.Ua = np.asfortranarray(st.Ua[:, r:])
    st.Sa = np.asfortranarray(st.Sa[:, r:])
    st.Ba = np.vstack([Ta[r:, r:], b[r:]])   # b of locked vectors set to zero
    return r


def full_T(st: RKSState):
    """Full k x k Rayleigh quotient of A and its b (locked b entries are 0)."""
    q, ja = st.q, st.ja
    T = np.zeros((q + ja, q + ja))
    T[:q, :q] = st.Tqq
    T[:q, q:] = st.Tqa
    T[q:, q:] = st.Ba[:ja, :]
    b = np.concatenate([np.zeros(q), st.Ba[ja, :]])
    U = np.hstack([st.Uq, st.Ua[:, :ja]])
    return T, b, U


# ---------------------------------------------------------------------------
# Driver
# ---------------------------------------------------------------------------

@dataclass
class RKSResult:
    eigvals: np.ndarray       # k Ritz values, best first
    X: np.ndarray             # n x k complex Ritz vectors U Y (unit sketch norm of y)
    resid: np.ndarray         # ||A x - l x|| / (||A||_1 ||x||), FP64
    est: np.ndarray           # |b^T y| / |l|  (Eq. 4.8)
    lam_rq: np.ndarray        # Rayleigh quotients x^H A x / x^H x
    T: np.ndarray
    U: np.ndarray
    b: np.ndarray
    u: np.ndarray
    S: np.ndarray
    s: np.ndarray
    restarts: int
    nmatvec: int
    nlocked: int
    converged: bool
    history: list = field(default_factory=list)
    locked: list = field(default_factory=list)   # q after each restart


def n_wanted(lam: np.ndarray, k: int) -> int:
    """How many leading sorted Ritz values are reported: k, or k + 1 when the
    k-th is the first member of a complex pair (pairs are never split)."""
    nw = min(k, lam.size)
    if 0 < nw < lam.size and lam[nw - 1].imag > 0:
        nw += 1
    return nw


def norm1(A: sp.spmatrix) -> float:
    return float(np.abs(A).sum(axis=0).max())


def true_residuals(A, X: np.ndarray, lam: np.ndarray):
    """||A x_i - l_i x_i|| / (||A||_1 ||x_i||) and Rayleigh quotients, FP64."""
    AX = A @ X
    nrm = norm1(A)
    res = np.linalg.norm(AX - X * lam, axis=0) / (nrm * np.linalg.norm(X, axis=0))
    rq = np.einsum("ij,ij->j", X.conj(), AX) / np.einsum("ij,ij->j", X.conj(), X)
    return res, rq


def rks(A, k: int, p: int, d: int, u1: np.ndarray, *, zeta: int = 8, seed: int = 0,
        which: str = "LM", tol: float = 1e-10, lock_vectors: bool = True,
        eta_lock: float | None = None, maxit: int = 1000, Omega=None,
        whiten_tol: float = 1e-10, max_restarts: int | None = None,
        conv: str = "eig", keep: int = 0, aggressive: bool = False) -> RKSResult:
    """Algorithm 1 (rKS) with the deflation of Sec. 4.

    ``max_restarts`` (if given) stops after that many contractions whatever the
    estimates say (the paper's fixed-iteration runs, Sec. 5).  ``conv`` picks
    the convergence quantity: "eig" (|b^T y|/|lambda|, Eq. 4.8) or "norm1"
    (|b^T y|/||A||_1, see ``ritz``), and the matching locking threshold.
    ``keep`` > 0 selects the thick restart of ``contract``; ``aggressive``
    moves converged Schur blocks to the front before locking
    (``aggressive_reorder``).  Convergence and
    the returned pairs concern the n_wanted best Ritz pairs of the full T.
    """
    A = sp.csr_matrix(A, dtype=np.float64)
    norm_a = norm1(A) if conv == "norm1" else None
    n = A.shape[0]
    m = k + p
    if Omega is None:
        Omega = omega_matrix(n, d, zeta, seed)
    eta_lock = tol if eta_lock is None else eta_lock
    st = start(A, Omega, np.asarray(u1, dtype=np.float64))
    extend(st, m)                                # Alg. 1, first line
    history = []
    locked = []
    converged = False
    restarts = 0
    limit = maxit if max_restarts is None else min(maxit, max_restarts)
    while True:
        contract(st, k, which, keep)             # Schur, reorder, truncate
        restarts += 1
        ja = st.ja
        if ja and whiten_tol is not None:
            G = st.Sa[:, :ja].T @ st.Sa[:, :ja]
            if np.linalg.norm(G - np.eye(ja)) > whiten_tol:
                whiten(st)
        if lock_vectors:
            if aggressive:
                aggressive_reorder(st, eta_lock, norm_a)
            lock(st, k, eta_lock, norm_a)
        locked.append(st.q)
        T, b, _ = full_T(st)
        lam, Y, est = ritz(T, b, which, norm_a)  # Alg. 1, Ritz pairs + Eq. 4.8
        est = est[:n_wanted(lam, k)]
        history.append(float(est.max()) if est.size else 0.0)
        if np.all(est <= tol):
            converged = True
            break
        if restarts >= limit:
            break
        extend(st, m - st.q)                     # Alg. 1, extension
    T, b, U = full_T(st)
    lam, Y, est = ritz(T, b, which, norm_a)
    nw = n_wanted(lam, k)
    lam, Y, est = lam[:nw], Y[:, :nw], est[:nw]
    X = U @ Y
    res, rq = true_residuals(A, X, lam)
    return RKSResult(eigvals=lam, X=X, resid=res, est=est, lam_rq=rq, T=T, U=U, b=b,
                     u=st.Ua[:, st.ja].copy(), S=np.hstack([st.Sq, st.Sa[:, :st.ja]]),
                     s=st.Sa[:, st.ja].copy(), restarts=restarts, nmatvec=st.nmatvec,
                     nlocked=st.q, converged=converged, history=history, locked=locked)
