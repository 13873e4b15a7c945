"""Pins of the randomized QR oracle (Sec. 2's randomized orthogonalisations).

RGS and sketch-and-whiten must give the unique sketch-orthonormal QR
factorisation (R = the R factor of Omega K), randomized Cholesky QR the unique
Euclidean one (LAPACK's QR up to column signs); with Omega = I, RGS is
Gram-Schmidt.  Eq. 2.13 bounds the condition number of a sketch-orthonormal Q.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import sketch_qr as SQ
from oracle.sketch import omega_matrix
from paper_2508_05400_gb300 import inputs as I


def _graded_block(n, s, cond, seed):
    """K = U diag(sigma) V^T with singular values from 1 down to 1/cond."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, s)))
    V, _ = np.linalg.qr(rng.standard_normal((s, s)))
    return (U * np.logspace(0, -np.log10(cond), s)) @ V.T


@pytest.mark.parametrize("cond", [1e2, 1e8])
def test_rgs_and_whitening_give_the_unique_sketch_orthonormal_qr(cond):
    n, s, d = 3000, 24, 96
    K = _graded_block(n, s, cond, 1)
    Om = omega_matrix(n, d, 8, 0)
    Qg, Rg, Sg = SQ.rgs(K, Om)
    Qw, Rw, Sw = SQ.sketch_whiten(K, Om)
    # loss of sketch-orthonormality of the order of u * kappa(K) (the MGS-like
    # behaviour the paper attributes to RGS), exact for the whitened sketch
    lost = 10 * s * 1.1e-16 * cond
    for Q, R, S in ((Qg, Rg, Sg), (Qw, Rw, Sw)):
        assert np.linalg.norm(K - Q @ R) <= 1e-14 * np.linalg.norm(K) * s
        assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
        assert np.linalg.norm(S.T @ S - np.eye(s)) < lost
        assert np.linalg.norm(Om @ Q - S) < lost
    assert np.linalg.norm(Sw.T @ Sw - np.eye(s)) < 1e-13 * s
    # uniqueness: the same R (that of Omega K) and the same Q
    assert np.linalg.norm(Rg - Rw) <= 1e-13 * np.linalg.norm(Rw)
    assert np.linalg.norm(Qg - Qw) <= lost


def test_rgs_with_identity_sketch_is_gram_schmidt():
    # Omega = I: sketch-orthonormal is orthonormal, RGS is Gram-Schmidt, and
    # the factorisation is LAPACK's QR with a positive diagonal
    n, s = 200, 12
    K = _graded_block(n, s, 1e3, 2)
    Q, R, S = SQ.rgs(K, sp.identity(n, format="csr"))
    Qx, Rx = np.linalg.qr(K)
    sgn = np.sign(np.diag(Rx))
    assert np.allclose(Q, Qx * sgn, atol=1e-11)
    assert np.allclose(R, (Rx.T * sgn).T, atol=1e-12 * np.abs(Rx).max())


@pytest.mark.parametrize("cond", [1e2, 1e10])
def test_rcholqr_is_the_euclidean_qr(cond):
    n, s, d = 3000, 24, 96
    K = _graded_block(n, s, cond, 3)
    Om = omega_matrix(n, d, 8, 0)
    Q, R = SQ.rcholqr(K, Om)
    assert np.linalg.norm(Q.T @ Q - np.eye(s)) < 1e-13 * s          # orthonormal at any condition
    assert np.linalg.norm(K - Q @ R) <= 1e-14 * np.linalg.norm(K) * s
    Qx, Rx = np.linalg.qr(K)
    sgn = np.sign(np.diag(Rx))
    assert np.linalg.norm(Q - Qx * sgn) <= 1e-15 * cond * s * 10


def test_condition_of_sketch_orthonormal_q():
    # Eq. 2.13: kappa(Q) <= sqrt((1+eps)/(1-eps)) kappa(Omega Q) = sqrt((1+eps)/(1-eps))
    n, s, d = 4000, 16, 160
    K = _graded_block(n, s, 1e6, 4)
    Om = omega_matrix(n, d, 8, 0)
    Q, R, S = SQ.sketch_whiten(K, Om)
    Ub, _ = np.linalg.qr(K)
    sv = np.linalg.svd((Om @ Ub), compute_uv=False)
    eps = max(sv.max() ** 2 - 1, 1 - sv.min() ** 2)
    assert eps < 1
    svq = np.linalg.svd(Q, compute_uv=False)
    assert svq.max() / svq.min() <= np.sqrt((1 + eps) / (1 - eps)) * (1 + 1e-10)


def test_planted_mistake_in_rgs_is_caught(monkeypatch):
    # a dropped projection term (q~ = k_j - Q_{j-1} r without the last column)
    n, s, d = 500, 8, 48
    K = _graded_block(n, s, 10.0, 5)
    Om = omega_matrix(n, d, 8, 0)
    real = np.linalg.lstsq

    def bad(a, b, rcond=None):
        y = real(a, b, rcond=rcond)
        y[0][-1:] = 0.0
        return y
    monkeypatch.setattr(SQ.np.linalg, "lstsq", bad)
    Q, R, S = SQ.rgs(K, Om)
    monkeypatch.undo()
    assert np.linalg.norm(S.T @ S - np.eye(s)) > 1e-6


# ---------------------------------------------------------------------------
# RHQR: Householder QR in the sketched space of Theta = [[I_s, 0], [0, Omega']]
# ---------------------------------------------------------------------------

def test_rhqr_with_identity_sketch_is_householder_qr():
    # Omega' = I makes Theta = I: RHQR is Householder QR, LAPACK's up to signs
    n, s = 300, 16
    K = _graded_block(n, s, 1e6, 5)
    Q, R, TQ = SQ.rhqr(K, sp.identity(n - s, format="csr"))
    Ql, Rl = np.linalg.qr(K)
    sg = np.sign(np.diag(Rl))
    Ql, Rl = Ql * sg, (Rl.T * sg).T
    assert np.linalg.norm(R - Rl) <= 1e-13 * np.linalg.norm(Rl)
    assert np.linalg.norm(Q - Ql) <= 1e-10
    assert np.linalg.norm(Q.T @ Q - np.eye(s)) <= 1e-14 * s


@pytest.mark.parametrize("cond", [1e2, 1e6])
def test_rhqr_gives_the_unique_theta_orthonormal_qr(cond):
    # the same factorisation as RGS and sketch-and-whiten with Omega = Theta
    n, s, d = 3000, 24, 96
    K = _graded_block(n, s, cond, 6)
    Ob = omega_matrix(n - s, d, 8, 0)
    Th = SQ.theta_matrix(n, s, Ob)
    Q, R, TQ = SQ.rhqr(K, Ob)
    Qw, Rw, Sw = SQ.sketch_whiten(K, Th)
    Qg, Rg, Sg = SQ.rgs(K, Th)
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    assert np.linalg.norm(K - Q @ R) <= 1e-14 * np.linalg.norm(K) * s
    assert np.linalg.norm(TQ.T @ TQ - np.eye(s)) <= 1e-14 * s
    assert np.linalg.norm(Th @ Q - TQ) <= 1e-14 * s
    lost = 10 * s * 1.1e-16 * cond
    assert np.linalg.norm(R - Rw) <= 1e-13 * np.linalg.norm(Rw)
    assert np.linalg.norm(R - Rg) <= 1e-13 * np.linalg.norm(Rg)
    assert np.linalg.norm(Q - Qw) <= lost and np.linalg.norm(Q - Qg) <= lost


def test_rhqr_stays_orthonormal_where_whitening_does_not():
    # Householder-type stability: Theta Q orthonormal to rounding for
    # kappa(K) = 1e12, where K R^{-1} (sketch and whiten) loses ~u kappa
    n, s, d = 2000, 20, 80
    K = _graded_block(n, s, 1e12, 7)
    Ob = omega_matrix(n - s, d, 8, 0)
    Th = SQ.theta_matrix(n, s, Ob)
    Q, R, TQ = SQ.rhqr(K, Ob)
    Qw, _, _ = SQ.sketch_whiten(K, Th)
    TQw = Th @ Qw
    assert np.linalg.norm(TQ.T @ TQ - np.eye(s)) <= 1e-13 * s
    assert np.linalg.norm(TQw.T @ TQw - np.eye(s)) > 1e3 * np.linalg.norm(TQ.T @ TQ - np.eye(s))
    assert np.linalg.norm(K - Q @ R) <= 1e-14 * np.linalg.norm(K) * s


def test_rhqr_planted_mistake_is_caught():
    # a reflector whose n-dimensional vector keeps the entries above the
    # diagonal (Theta u != v) no longer factors K
    n, s, d = 500, 8, 40
    K = _graded_block(n, s, 1e2, 8)
    Ob = omega_matrix(n - s, d, 8, 0)
    good = SQ.rhqr(K, Ob)
    bad_src = open(SQ.__file__).read().replace("        u[:j] = 0.0\n", "")
    ns = {}
    exec(compile(bad_src, SQ.__file__, "exec"), ns)
    Q, R, TQ = ns["rhqr"](K, Ob)
    assert np.linalg.norm(K - Q @ R) > 1e-6 * np.linalg.norm(K)
    Q, R, TQ = good
    assert np.linalg.norm(K - Q @ R) <= 1e-13 * np.linalg.norm(K)
