"""Pins of the FP64 rKS oracle against the paper's invariants and closed forms.

Every pin checks the oracle against something other than itself: the
definitions and theorems of the paper (sketch-orthonormality Def. 2.3, the
Krylov relation Eq. 2.4 / 2.16, the Rayleigh quotient Thm 2.4, the residual
bounds of Sec. 4.1, the locking bound Eq. 4.21), brute force (MGS Arnoldi,
dense eigenvalues), and closed-form spectra.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import rks as R
from oracle.sketch import omega_matrix
from paper_2508_05400_gb300 import inputs as I


def _decomposition_errors(st):
    """Errors of the full decomposition A U = U T + u b^T and of its sketch."""
    T, b, U = R.full_T(st)
    u = st.Ua[:, st.ja]
    Sall = np.hstack([st.Sq, st.Sa])
    Uall = np.hstack([st.Uq, st.Ua])
    orth = np.linalg.norm(Sall.T @ Sall - np.eye(Sall.shape[1]))
    sketch = np.linalg.norm(st.Omega @ Uall - Sall) / np.linalg.norm(Sall)
    AU = st.A @ U
    rel = np.linalg.norm(AU - U @ T - np.outer(u, b)) / np.linalg.norm(AU)
    return orth, sketch, rel


def _expand_from_scratch(A, m, d, zeta=8, seed=0, Omega=None):
    A = sp.csr_matrix(A)
    n = A.shape[0]
    Om = omega_matrix(n, d, zeta, seed) if Omega is None else Omega
    st = R.start(A, Om, I.start_vector(n, 1))
    R.extend(st, m)
    return st


def test_expansion_invariants():
    # Alg. 2 from k = 0 yields a randomized Arnoldi factorization (Def. 2.1):
    # (Omega U)^T (Omega U) = I, A U = U B + u b^T, B upper Hessenberg with a
    # positive subdiagonal, and B = (Omega U)^T Omega A U (Thm 2.4, Eq. 2.9).
    A = I.convdiff_2d(20, 20, 1.0, 20.0, 10.0).to_scipy()
    st = _expand_from_scratch(A, 30, 64)
    orth, sketch, rel = _decomposition_errors(st)
    assert orth < 1e-12 and sketch < 1e-14 and rel < 1e-13
    B = st.Ba[:30, :]
    assert np.all(np.tril(B, -2) == 0)
    assert np.all(np.diag(B, -1) > 0)
    S = st.Sa[:, :30]
    rq = S.T @ (st.Omega @ (A @ st.Ua[:, :30]))
    assert np.linalg.norm(rq - B) < 1e-12 * np.linalg.norm(B)


def test_identity_sketch_reduces_to_arnoldi():
    # With Omega = I, sketch-orthonormal means orthonormal and Alg. 2 is the
    # Arnoldi process: B equals the Hessenberg matrix of a brute-force
    # modified Gram-Schmidt Arnoldi (unique for a positive subdiagonal).
    n, m = 60, 12
    A = I.paper_tridiag(n, "logarithmic", 4).to_scipy().toarray() + \
        0.05 * I.normal(9, n * n).reshape(n, n)
    st = _expand_from_scratch(A, m, n, Omega=sp.identity(n, format="csr"))
    V = np.zeros((n, m + 1)); H = np.zeros((m + 1, m))
    v = I.start_vector(n, 1)
    V[:, 0] = v / np.linalg.norm(v)
    for j in range(m):
        w = A @ V[:, j]
        for i in range(j + 1):
            H[i, j] = V[:, i] @ w
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        V[:, j + 1] = w / H[j + 1, j]
    assert np.allclose(st.Ba, H, atol=1e-12)
    assert np.allclose(st.Ua, V, atol=1e-12)


@pytest.mark.parametrize("which", R.WHICH)
def test_ordered_schur_against_numpy(which):
    rng = np.random.default_rng(5)
    for m in (10, 33, 80):
        B = rng.standard_normal((m, m))
        T, Q = R.ordered_schur(B, which, nsort=8)
        assert np.linalg.norm(Q.T @ Q - np.eye(m)) < 1e-13 * m
        assert np.linalg.norm(Q @ T @ Q.T - B) < 1e-13 * m * np.linalg.norm(B)
        assert np.all(np.tril(T, -2) == 0)
        blocks = R.schur_blocks(T)
        for s, z in blocks:
            if z == 2:   # standardised 2x2 block: equal diagonal, complex pair
                assert abs(T[s, s] - T[s + 1, s + 1]) < 1e-12 * np.linalg.norm(B)
                assert T[s, s + 1] * T[s + 1, s] < 0
        lam = np.array([R.block_eigenvalue(T, s, z) for s, z in blocks])
        ref = np.linalg.eigvals(B)
        ref = ref[ref.imag >= 0]
        ref_keys = np.sort(R.key(ref, which))
        keys = R.key(lam, which)
        assert np.allclose(keys[:8], ref_keys[:8], atol=1e-10 * np.abs(ref).max())
        assert np.all(np.diff(keys[:8]) >= -1e-10 * np.abs(ref).max())


def test_contraction_keeps_decomposition():
    # Truncation (Alg. 1; Eqs. 3.5-3.6): U Q(:,1:k), S Q(:,1:k), b^T Q(:,1:k),
    # u and s unchanged is again an rKS decomposition with S = Omega U.
    A = I.convdiff_2d(20, 20, 1.0, 20.0, 10.0).to_scipy()
    st = _expand_from_scratch(A, 30, 64)
    Ta, b, Q = R.contract(st, 8, "LR")
    assert st.ja in (8, 9)
    orth, sketch, rel = _decomposition_errors(st)
    assert orth < 1e-12 and sketch < 1e-13 and rel < 1e-12
    R.extend(st, 30)
    orth, sketch, rel = _decomposition_errors(st)
    assert orth < 1e-12 and sketch < 1e-13 and rel < 1e-12


def test_toeplitz_closed_form_small():
    # Non-symmetric Toeplitz (2, -1.3, -0.7) at n = 30, where the eigenvalue
    # condition numbers stay small enough for 1e-10 (LM, k = 4).
    n = 30
    A = I.toeplitz_tridiag(n).to_scipy()
    res = R.rks(A, 4, 12, 40, I.start_vector(n, 1), zeta=4, seed=0, which="LM", tol=1e-14)
    ex = I.toeplitz_eigenvalues(n, -1.3, 2.0, -0.7)
    ex = ex[np.argsort(-np.abs(ex))][:4]
    assert res.converged
    assert np.max(np.abs(res.eigvals - ex) / np.abs(ex)) < 1e-10
    assert res.resid.max() < 1e-11


def test_symmetric_toeplitz_closed_form():
    n = 100
    s = np.sqrt(0.91)
    A = I.toeplitz_tridiag(n, -s, 2.0, -s).to_scipy()
    res = R.rks(A, 4, 12, 40, I.start_vector(n, 1), zeta=4, seed=0, which="LM", tol=1e-12)
    ex = I.toeplitz_eigenvalues(n, -s, 2.0, -s)
    ex = ex[np.argsort(-np.abs(ex))][:4]
    assert res.converged
    assert np.max(np.abs(res.eigvals - ex) / np.abs(ex)) < 1e-10


@pytest.mark.parametrize("lock", [False, True])
def test_convdiff_kronecker_closed_form(lock):
    # The 2D upwind operator with constant nu is a Kronecker sum of 1D Toeplitz
    # operators; LR eigenvalues from rKS with deflation match it.
    N = 30
    A = I.convdiff_2d(N, N, 1.0, 20.0, 10.0).to_scipy()
    ex = np.sort(I.convdiff_2d_eigenvalues(N, N, 1.0, 20.0, 10.0))[::-1][:6]
    res = R.rks(A, 6, 18, 64, I.start_vector(N * N, 1), zeta=8, seed=0, which="LR",
                tol=1e-13, lock_vectors=lock)
    assert res.converged
    if lock:
        assert res.nlocked > 0
    assert np.max(np.abs(res.eigvals - ex) / np.abs(ex)) < 1e-10
    assert res.resid.max() < 1e-13


def test_thick_restart_keeps_closed_form_and_saves_matvecs():
    # keep > 0 retains extra active Schur vectors after locking: the same
    # closed-form eigenvalues, with fewer products with A than truncating to k
    N = 30
    A = I.convdiff_2d(N, N, 1.0, 20.0, 10.0).to_scipy()
    ex = np.sort(I.convdiff_2d_eigenvalues(N, N, 1.0, 20.0, 10.0))[::-1][:6]
    u1 = I.start_vector(N * N, 1)
    base = R.rks(A, 6, 18, 64, u1, zeta=8, seed=0, which="LR", tol=1e-13)
    thick = R.rks(A, 6, 18, 64, u1, zeta=8, seed=0, which="LR", tol=1e-13, keep=6)
    assert base.converged and thick.converged
    assert thick.eigvals.size == 6
    assert np.max(np.abs(thick.eigvals - ex) / np.abs(ex)) < 1e-10
    assert thick.resid.max() < 1e-13
    assert thick.nmatvec < base.nmatvec
    # the full decomposition it ends on is still a Krylov decomposition
    r = A @ thick.U - thick.U @ thick.T - np.outer(thick.u, thick.b)
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(A @ thick.U)


def test_contract_keep_size():
    # the kept active count is max(k - q, min(keep, ma // 2)) with ma = m - q
    # active columns, one more when a complex pair straddles the cut
    A = I.convdiff_2d(12, 11, 1.0, 20.0, 10.0).to_scipy()
    Om = omega_matrix(132, 48, 8, 0)
    for keep, qlock, expect in [(0, 0, 4), (4, 0, 4), (6, 0, 6), (4, 2, 4), (10, 2, 9), (20, 2, 9)]:
        st = R.start(A, Om, I.start_vector(132, 1))
        R.extend(st, 20)
        if qlock:   # lock the two leading vectors: the active part then has 18 columns
            R.contract(st, qlock, "LR")
            R.lock(st, qlock, 1e300)
            assert st.q == qlock
            R.extend(st, 20 - qlock)
        Ta, bk, Qk = R.contract(st, 4, "LR", keep)
        assert Qk.shape[1] - expect in (0, 1)
        if Qk.shape[1] == expect + 1:        # only for a pair at the cut
            assert R.schur_blocks(Ta)[-1][1] == 2


def _planted_spectrum_matrix(n, seed):
    """A = X D X^{-1} with known eigenvalues (including complex pairs), X well conditioned."""
    rng = np.random.default_rng(seed)
    lam = np.concatenate([np.linspace(1.0, 3.0, n - 6), [5.0, -4.5, 0.02]])
    D = np.diag(lam)
    Blk = np.zeros((n, n)); Blk[: n - 3, : n - 3] = D[: n - 3, : n - 3]
    # three complex pairs a +- ib as 2x2 blocks replace the last three singles
    pairs = [(4.0, 1.0), (-0.5, 3.5), (0.01, 0.05)]
    lam_all = list(np.linspace(1.0, 3.0, n - 6))
    Blk = np.zeros((n, n))
    Blk[: n - 6, : n - 6] = np.diag(lam_all)
    for t, (a, b) in enumerate(pairs):
        i = n - 6 + 2 * t
        Blk[i:i + 2, i:i + 2] = [[a, b], [-b, a]]
        lam_all += [a + 1j * b, a - 1j * b]
    Qx, _ = np.linalg.qr(rng.standard_normal((n, n)))
    X = Qx @ (np.eye(n) + 0.1 * np.triu(rng.standard_normal((n, n)), 1) / np.sqrt(n))
    A = X @ Blk @ np.linalg.inv(X)
    return A, np.array(lam_all), np.linalg.cond(X)


@pytest.mark.parametrize("which,k", [("LM", 4), ("SM", 3), ("LR", 4), ("SR", 2)])
def test_bruteforce_planted_spectrum(which, k):
    n = 150
    A, lam, condX = _planted_spectrum_matrix(n, 11)
    want = lam[np.argsort(R.key(lam, which), kind="stable")][:k]
    res = R.rks(A, k, 16, 64, I.start_vector(n, 1), zeta=8, seed=0, which=which, tol=1e-13)
    assert res.converged
    # each computed value matches a wanted one within cond(X) * 1e-12
    for lam_c in res.eigvals:
        assert np.min(np.abs(want - lam_c)) < condX * 1e-12 * max(1.0, abs(lam_c))
    # and the dense brute force agrees with the planted spectrum
    dense = np.linalg.eigvals(A)
    assert all(np.min(np.abs(dense - w)) < 1e-10 for w in want)


def test_residual_estimate_band():
    # Sec. 4.1 remark (exact bound): with eps the distortion of Omega on
    # span[U u], sqrt((1-eps)/(1+eps)) |b^T y| <= ||A x - l x|| / ||x||
    # <= sqrt((1+eps)/(1-eps)) |b^T y| for x = U y, ||y|| = 1.
    N = 20
    A = I.convdiff_2d(N, N, 1.0, 20.0, 10.0).to_scipy()
    n = N * N
    Om = omega_matrix(n, 256, 8, 0)      # eps < 1 needs d well above m
    st = R.start(sp.csr_matrix(A), Om, I.start_vector(n, 1))
    R.extend(st, 24)
    for _ in range(3):
        R.contract(st, 6, "LR")
        T, b, U = R.full_T(st)
        u = st.Ua[:, st.ja]
        Qb, _ = np.linalg.qr(np.hstack([U, u[:, None]]))
        sv = np.linalg.svd(Om @ Qb, compute_uv=False)
        eps = max(sv.max() ** 2 - 1, 1 - sv.min() ** 2)
        assert eps < 1
        lam, Y, est = R.ritz(T, b, "LR")
        X = U @ Y
        true = np.linalg.norm(A @ X - X * lam, axis=0) / np.linalg.norm(X, axis=0)
        bty = np.abs(b @ Y)
        lo = np.sqrt((1 - eps) / (1 + eps)) * bty
        hi = np.sqrt((1 + eps) / (1 - eps)) * bty
        assert np.all(true >= lo * (1 - 1e-9)) and np.all(true <= hi * (1 + 1e-9))
        R.extend(st, 24)


def test_locking_bound_and_deflated_operator():
    # Eq. 4.21: a locked Ritz pair (l, x = U_q y), ||y|| = 1, satisfies
    # ||A x - l x|| <= sqrt(q)/sqrt(1-eps) * max|b_locked|, and Thm 4.3:
    # (I - U_q (Omega U_q)^T Omega) A U_q = U_q T_qq - U_q T_qq + O(b) ~ 0.
    N = 30
    A = sp.csr_matrix(I.convdiff_2d(N, N, 1.0, 20.0, 10.0).to_scipy())
    n = N * N
    Om = omega_matrix(n, 64, 8, 0)
    st = R.start(A, Om, I.start_vector(n, 1))
    R.extend(st, 24)
    locked_total = 0
    for _ in range(60):
        R.contract(st, 6, "LR")
        ja = st.ja
        b_before = st.Ba[ja, :].copy()
        u = st.Ua[:, ja].copy()
        q0 = st.q
        r = R.lock(st, 6, 1e-11)
        if r:
            locked_total += r
            q = st.q
            bq = np.concatenate([np.zeros(q0), b_before[:r]])   # lock-time b of U_q
            Qb, _ = np.linalg.qr(np.hstack([st.Uq, u[:, None]]))
            sv = np.linalg.svd(Om @ Qb, compute_uv=False)
            eps = max(sv.max() ** 2 - 1, 1 - sv.min() ** 2)
            lam, W = np.linalg.eig(st.Tqq)
            W = W / np.linalg.norm(W, axis=0)
            X = st.Uq @ W
            res = np.linalg.norm(A @ X - X * lam, axis=0)
            bound = np.sqrt(q) / np.sqrt(1 - eps) * max(np.abs(bq).max(), 1e-300)
            # earlier locked vectors carry their own (smaller or equal) b
            assert np.all(res[-r:] <= bound * 1.0001 + 1e-10 * np.abs(lam[-r:]))
            P = st.Uq @ (st.Sq.T @ (Om @ (A @ st.Uq)))
            Aq_Uq = A @ st.Uq - P
            assert np.linalg.norm(Aq_Uq) < 1e-8 * np.linalg.norm(A @ st.Uq)
        T, b, U = R.full_T(st)
        lam, Y, est = R.ritz(T, b, "LR")
        if st.q >= 6 or np.all(est <= 1e-11):
            break
        R.extend(st, 24 - st.q)
    assert locked_total > 0
    orth, sketch, rel = _decomposition_errors(st)
    assert orth < 1e-11 and rel < 1e-11


def test_whitening_restores_orthonormal_sketch():
    # Sec. 3.3: S = QR, U <- U R^{-1}, T <- R T R^{-1}, b^T <- b^T R^{-1} keeps
    # the Krylov relation and the spectrum, and makes Omega U orthonormal.
    A = I.convdiff_2d(20, 20, 1.0, 20.0, 10.0).to_scipy()
    st = _expand_from_scratch(A, 30, 64)
    R.contract(st, 8, "LR")
    ja = st.ja
    G = np.eye(ja) + 0.05 * np.triu(np.ones((ja, ja)), 1)   # spoil orthonormality
    st.Ua[:, :ja] = st.Ua[:, :ja] @ G
    st.Sa[:, :ja] = st.Sa[:, :ja] @ G
    Ta = st.Ba[:ja, :]
    st.Ba = np.vstack([np.linalg.solve(G, Ta @ G), st.Ba[ja, :] @ G])
    ev0 = np.sort_complex(np.linalg.eigvals(st.Ba[:ja, :]))
    R.whiten(st)
    S = st.Sa[:, :ja]
    assert np.linalg.norm(S.T @ S - np.eye(ja)) < 1e-13
    _, sketch, rel = _decomposition_errors(st)
    assert sketch < 1e-13 and rel < 1e-12
    assert np.allclose(np.sort_complex(np.linalg.eigvals(st.Ba[:ja, :])), ev0, rtol=1e-10)


# ---------------------------------------------------------------------------
# Planted mistakes: each pin above must catch a plausible bug in the oracle.
# ---------------------------------------------------------------------------

def _extend_with(monkeypatch, mutation):
    """Run a mutated Alg. 2 (mistake planted in the oracle, on the CPU)."""
    orig_lstsq = np.linalg.lstsq

    def run():
        A = sp.csr_matrix(I.convdiff_2d(20, 20, 1.0, 20.0, 10.0).to_scipy())
        st = _expand_from_scratch(A, 20, 64)
        return st
    if mutation == "sign":
        def bad(a, b, rcond=None):
            x = orig_lstsq(a, b, rcond=rcond)
            return (-x[0],) + tuple(x[1:])
        monkeypatch.setattr(np.linalg, "lstsq", bad)
    elif mutation == "dropped_term":
        def bad(a, b, rcond=None):
            x = orig_lstsq(a, b, rcond=rcond)
            y = x[0].copy()
            if y.size > 1:
                y[0] = 0.0
            return (y,) + tuple(x[1:])
        monkeypatch.setattr(np.linalg, "lstsq", bad)
    elif mutation == "transposed":
        def bad(a, b, rcond=None):
            return orig_lstsq(a[::-1, :], b, rcond=rcond)
        monkeypatch.setattr(np.linalg, "lstsq", bad)
    st = run()
    monkeypatch.undo()
    return st


@pytest.mark.parametrize("mutation", ["sign", "dropped_term", "transposed"])
def test_planted_mistakes_are_caught(monkeypatch, mutation):
    st = _extend_with(monkeypatch, mutation)
    orth, sketch, rel = _decomposition_errors(st)
    B = st.Ba[:20, :]
    S = st.Sa[:, :20]
    rq = S.T @ (st.Omega @ (st.A @ st.Ua[:, :20]))
    rq_err = np.linalg.norm(rq - B) / np.linalg.norm(B)
    # the expansion invariant test would fail on at least one of its checks
    assert orth > 1e-6 or rq_err > 1e-6 or rel > 1e-6


def test_planted_missing_coupling_breaks_eigenvalues(monkeypatch):
    # Dropping T_qa (the coefficients of A u_j on the locked vectors, which the
    # lock step folds into T_qq) must break the true residuals once vectors
    # are locked.
    orig = R.lock

    def lock_without_coupling(st, k, eta_lock, norm_a=None):
        st.Tqa[:] = 0.0
        return orig(st, k, eta_lock, norm_a)
    monkeypatch.setattr(R, "lock", lock_without_coupling)
    N = 30
    A = I.convdiff_2d(N, N, 1.0, 20.0, 10.0).to_scipy()
    res = R.rks(A, 6, 18, 64, I.start_vector(N * N, 1), zeta=8, seed=0, which="LR",
                tol=1e-13, maxit=80)
    assert res.nlocked > 1
    assert res.resid.max() > 1e-8


def test_block_eigvec_against_library_eig():
    # The eigenvector of a quasi-triangular T for its i-th diagonal block is
    # zero below that block (remark after Eq. 4.21) and is, up to a phase, the
    # eigenvector LAPACK returns for the same eigenvalue.
    import scipy.linalg as sla
    rng = np.random.default_rng(3)
    T, _ = sla.schur(rng.standard_normal((14, 14)), output="real")
    lam_all, V = np.linalg.eig(T)
    nb2 = 0
    for s, z in R.schur_blocks(T):
        nb2 += z == 2
        lam, y = R.block_eigvec(T, s, z)
        assert np.linalg.norm(T @ y - lam * y) < 1e-12 * np.linalg.norm(T)
        assert np.all(y[s + z:] == 0) and abs(np.linalg.norm(y) - 1) < 1e-14
        v = V[:, np.argmin(np.abs(lam_all - lam))]
        assert abs(abs(np.vdot(v, y)) - 1) < 1e-10
    assert nb2 >= 2                       # the case covers complex pairs


def _exterior_pair_matrix(n=300, seed=5, isolated=None):
    """A normal matrix whose eigenvalue 1.0 sits just outside a disk of
    eigenvalues (slow to converge) and whose pair 0.9 +- 5i is isolated
    (fast): under LR the pair is wanted after 1.0 but converges first.
    ``isolated`` adds one more real eigenvalue far to the right (converges,
    and locks, first)."""
    rng = np.random.default_rng(seed)
    lead = ([isolated] if isolated is not None else []) + [1.0]
    h = len(lead) + 2
    nb = (n - h) // 2
    r = np.sqrt(rng.uniform(0, 1, nb)); th = rng.uniform(0, np.pi, nb)
    Blk = np.zeros((n, n))
    for i, v in enumerate(lead):
        Blk[i, i] = v
    Blk[h - 2:h, h - 2:h] = [[0.9, 5.0], [-5.0, 0.9]]
    for t in range(nb):
        a, b = -0.05 + r[t] * np.cos(th[t]), r[t] * np.sin(th[t])
        i = h + 2 * t
        Blk[i:i + 2, i:i + 2] = [[a, b], [-b, a]]
    if n - h - 2 * nb:
        Blk[n - 1, n - 1] = -0.5
    Qx, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return Qx @ Blk @ Qx.T


@pytest.mark.parametrize("isolated", [None, 3.0])
def test_aggressive_reorder_moves_converged_block(isolated):
    # Sec. 4.3 (after Thm 4.3): reordering the factorization to test another
    # leading vector.  The reorder is an orthogonal similarity: the
    # decomposition A U = U T + u b^T (locked part and coupling T_qa
    # included) still holds, the spectrum of T_a is unchanged, the converged
    # pair now leads, and its estimate |b^T y| is the same number before and
    # after (b' = Z^T b, y' = Z^T y).
    A = sp.csr_matrix(_exterior_pair_matrix(isolated=isolated))
    n = A.shape[0]
    k = 3 if isolated is None else 4
    st = R.start(A, omega_matrix(n, 48, 8, 0), I.start_vector(n, 1))
    R.extend(st, 15)
    moved = False
    for _ in range(8):
        R.contract(st, k, "LR")
        if isolated is not None and st.q == 0:
            R.lock(st, k, 1e-12)          # the isolated eigenvalue locks first
            R.extend(st, 15 - st.q)
            continue
        ja = st.ja
        Ta, b = st.Ba[:ja, :].copy(), st.Ba[ja, :].copy()
        blocks = R.schur_blocks(Ta)
        est = {}
        for s, z in blocks:
            lam, y = R.block_eigvec(Ta, s, z)
            est[s] = (lam, abs(b @ y))
        nsel = R.aggressive_reorder(st, 1e-12)
        Ta2, b2 = st.Ba[:ja, :], st.Ba[ja, :]
        assert np.allclose(np.sort_complex(np.linalg.eigvals(Ta2)), np.sort_complex(np.linalg.eigvals(Ta)),
                           atol=1e-12)
        orth, sketch, rel = _decomposition_errors(st)
        assert orth < 1e-11 and sketch < 1e-13 and rel < 1e-11
        conv = [s for s, z in blocks if est[s][1] <= 1e-12 * max(abs(est[s][0]), 1e-300)]
        assert nsel == sum(dict(blocks)[s] for s in conv)
        if conv and conv[0] != 0:         # a converged block behind an unconverged one
            lam0, y0 = R.block_eigvec(Ta2, 0, dict(R.schur_blocks(Ta2))[0])
            assert abs(lam0 - est[conv[0]][0]) < 1e-12 * abs(lam0)
            assert abs(abs(b2 @ y0) - est[conv[0]][1]) <= 1e-6 * est[conv[0]][1] + 1e-15
            moved = True
            break
        R.extend(st, 15 - st.q)
    assert moved and st.q == (0 if isolated is None else 1)


def test_aggressive_deflation_locks_earlier_same_result():
    # Plain locking waits for the leading Schur vector; aggressive deflation
    # locks the converged pair as soon as it converges.  Same eigenvalues,
    # same residual level (planted spectrum {1, 0.9 +- 5i}).
    A = _exterior_pair_matrix()
    n = A.shape[0]
    plain = R.rks(A, 3, 12, 48, I.start_vector(n, 1), which="LR", tol=1e-12)
    aggr = R.rks(A, 3, 12, 48, I.start_vector(n, 1), which="LR", tol=1e-12, aggressive=True)
    assert plain.converged and aggr.converged
    for res in (plain, aggr):
        assert np.allclose(np.sort_complex(res.eigvals), np.sort_complex([1.0, 0.9 + 5j, 0.9 - 5j]), atol=1e-11)
        assert res.resid.max() < 1e-13
    first = lambda hist: next(t for t, q in enumerate(hist) if q > 0)
    assert first(aggr.locked) < first(plain.locked)
    assert aggr.locked[first(aggr.locked)] == 2       # the pair, locked whole


@pytest.mark.parametrize("eta_lock", [1e-3, 1e-6])
def test_locking_bound_sqrt_i_at_lock_time(eta_lock):
    # Remark after Eq. 4.21: with |b_j| <= eta on the locked columns, the Ritz
    # pair of the i-th diagonal block of T_qq (its eigenvector lives in the
    # first i entries) has ||A U_q y - l U_q y|| = ||u|| |b^T y| (Eq. 4.20)
    # <= sqrt(i) eta ||u||, with ||u|| <= 1/sqrt(1-eps).  Planted spectrum
    # {1.6, 1.45, 1.3, 1.2} over a bulk in [-1, 1]; the first locking event
    # takes two vectors at once, with |b| far above rounding.
    n = 200
    rng = np.random.default_rng(7)
    lam_p = np.concatenate([[1.6, 1.45, 1.3, 1.2], rng.uniform(-1, 1, n - 4)])
    Qx, _ = np.linalg.qr(rng.standard_normal((n, n)))
    X = Qx @ (np.eye(n) + 0.3 * np.triu(rng.standard_normal((n, n)), 1) / np.sqrt(n))
    A = sp.csr_matrix(X @ np.diag(lam_p) @ np.linalg.inv(X))
    Om = omega_matrix(n, 48, 8, 0)
    st = R.start(A, Om, I.start_vector(n, 1))
    R.extend(st, 12)
    for _ in range(20):
        R.contract(st, 4, "LM")
        ja = st.ja
        b_before = st.Ba[ja, :].copy()
        u = st.Ua[:, ja].copy()
        r = R.lock(st, 4, eta_lock)
        if r:
            break
        R.extend(st, 12 - st.q)
    assert r >= 2 and st.q == r            # first locking event, several vectors
    eta = np.abs(b_before[:r]).max()
    Qb, _ = np.linalg.qr(np.hstack([st.Uq, u[:, None]]))
    sv = np.linalg.svd(Om @ Qb, compute_uv=False)
    eps = max(sv.max() ** 2 - 1, 1 - sv.min() ** 2)
    assert eps < 1 and np.linalg.norm(u) <= 1 / np.sqrt(1 - eps) * (1 + 1e-12)
    for s, z in R.schur_blocks(st.Tqq):
        lam, y = R.block_eigvec(st.Tqq, s, z)
        assert np.all(y[s + z:] == 0)
        x = st.Uq @ y
        res = np.linalg.norm(A @ x - lam * x)
        ident = np.linalg.norm(u) * abs(b_before[:r] @ y)
        assert abs(res - ident) <= 1e-7 * ident + 1e-13 * abs(lam)
        assert res <= np.sqrt(s + z) * eta / np.sqrt(1 - eps) * (1 + 1e-9)
