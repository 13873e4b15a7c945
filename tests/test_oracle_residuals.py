"""Pins of the oracle's FP64 residual and Rayleigh quotient (``true_residuals``).

The residual ||A x - l x|| / (||A||_1 ||x||) is the measure every full-size
test and the benchmark judge convergence by (the normwise residual of the
Sec. 4.1 remark, scaled by ||A||_1), and x^H A x / x^H x is the Rayleigh
quotient that refines a Ritz value.  These tests feed it vectors whose
residual and quotient are known without it:

* the closed-form eigenvectors of a tridiagonal Toeplitz matrix, x_i =
  r^i sin(i j pi / (n+1)) with r = sqrt(sub/sup) (residual zero, quotient
  the eigenvalue diag + 2 sqrt(sub*sup) cos(j pi/(n+1)) with the signs of
  the off-diagonals);
* such a vector plus delta e_1, whose residual is |delta| ||(A - l I) e_1||
  and whose quotient follows from x^T A x expanded by hand;
* a complex pair of a 2 x 2 rotation block [[a, b], [-b, a]] (eigenvectors
  (1, +-i)), exact and perturbed, which a missing conjugation turns into a
  0/0 quotient;
* columns of different residual side by side, which a wrong reduction axis
  mixes up.
"""
import numpy as np
import scipy.sparse as sp

from oracle import rks as R


def _toeplitz(n, sub, diag, sup):
    return sp.diags([np.full(n - 1, sub), np.full(n, diag), np.full(n - 1, sup)], [-1, 0, 1],
                    format="csr")


def _toeplitz_pair(n, j, sub, diag, sup):
    """Closed-form eigenpair j (1-based) of tridiag(sub, diag, sup), sub*sup > 0."""
    i = np.arange(1, n + 1)
    th = j * np.pi / (n + 1)
    r = np.sqrt(sub / sup)
    x = r ** i * np.sin(i * th)
    # (A x)_i = sub x_{i-1} + diag x_i + sup x_{i+1} = (diag + 2 s cos th) x_i,
    # s = sub / r = sup * r (both carry the sign of the off-diagonals)
    lam = diag + 2.0 * (sub / r) * np.cos(th)
    return x, lam


def test_toeplitz_eigenvectors_have_zero_residual_and_exact_quotient():
    sub, diag, sup = -1.3, 2.0, -0.7
    for n in (12, 25, 40):
        A = _toeplitz(n, sub, diag, sup)
        js = [1, 2, n // 2, n]
        X = np.column_stack([_toeplitz_pair(n, j, sub, diag, sup)[0] for j in js])
        lam = np.array([_toeplitz_pair(n, j, sub, diag, sup)[1] for j in js])
        res, rq = R.true_residuals(A, X, lam)
        assert res.shape == (len(js),) and rq.shape == (len(js),)
        assert np.all(res <= 4e-14), res        # rounding of the closed form only
        assert np.allclose(rq, lam, rtol=1e-13, atol=0), (rq, lam)


def test_perturbed_eigenvector_residual_and_quotient_by_hand():
    sub, diag, sup = -1.3, 2.0, -0.7
    n = 30
    A = _toeplitz(n, sub, diag, sup)
    norm1 = abs(sub) + abs(diag) + abs(sup)          # an interior column
    cols, lams, want_res, want_rq = [], [], [], []
    for j, delta in ((1, 1e-3), (3, -2.5e-2), (7, 0.5), (11, 0.0)):
        x0, lam = _toeplitz_pair(n, j, sub, diag, sup)
        x = x0.copy()
        x[0] += delta
        # A x - lam x = delta (A - lam I) e_1 = delta (diag - lam, sub, 0, ...)
        res = abs(delta) * np.hypot(diag - lam, sub) / (norm1 * np.linalg.norm(x))
        # x^T A x = lam x0.x0 + delta (e_1^T A x0 + x0^T A e_1) + delta^2 diag,
        # e_1^T A x0 = lam x0[0], x0^T A e_1 = diag x0[0] + sub x0[1]
        xAx = lam * (x0 @ x0) + delta * (lam * x0[0] + diag * x0[0] + sub * x0[1]) + delta ** 2 * diag
        cols.append(x)
        lams.append(lam)
        want_res.append(res)
        want_rq.append(xAx / (x @ x))
    res, rq = R.true_residuals(A, np.column_stack(cols), np.array(lams))
    assert np.allclose(res, want_res, rtol=1e-12, atol=1e-14), (res, want_res)
    assert np.allclose(rq, want_rq, rtol=1e-13, atol=0), (rq, want_rq)
    # ||A||_1 is the largest column sum (4.0 here), not the Frobenius norm
    assert abs(R.norm1(A) - norm1) < 1e-15


def _rotation_operator(a, b, tail):
    """Block diagonal [[a, b], [-b, a]] (+) diag(tail): eigenvalues a +- i b, tail."""
    n = 2 + len(tail)
    A = np.zeros((n, n))
    A[0, 0], A[0, 1], A[1, 0], A[1, 1] = a, b, -b, a
    A[2:, 2:] = np.diag(tail)
    return sp.csr_matrix(A)


def test_complex_pair_residual_and_quotient():
    a, b = 0.75, 2.0
    tail = np.array([1.5, -0.25, 3.0])
    A = _rotation_operator(a, b, tail)
    norm1 = max(abs(a) + abs(b), np.abs(tail).max())
    n = A.shape[0]
    # [[a, b], [-b, a]] (1, i) = (a + i b) (1, i): eigenvalue a + i b
    xp = np.zeros(n, dtype=complex)
    xp[0], xp[1] = 1.0, 1j
    xm = xp.conj()
    xt = np.zeros(n, dtype=complex)
    xt[3] = 1.0                                   # a real eigenvector of the tail
    lam = np.array([a + 1j * b, a - 1j * b, tail[1]])
    res, rq = R.true_residuals(A, np.column_stack([xp, xm, xt]), lam)
    assert np.all(res <= 1e-16)
    assert np.allclose(rq, lam, rtol=1e-15, atol=0)
    # perturbed: x = (1 + delta, i, 0, ...), (A - lam I) e_1 = (-i b, -b, 0, ...)
    delta = 0.3
    x = xp.copy()
    x[0] += delta
    want_res = abs(delta) * b * np.sqrt(2.0) / (norm1 * np.sqrt((1 + delta) ** 2 + 1))
    # x^H A x = conj(x0) (a x0 + b x1) + conj(x1) (-b x0 + a x1), x0 = 1 + delta, x1 = i
    x0, x1 = 1 + delta, 1j
    xAx = np.conj(x0) * (a * x0 + b * x1) + np.conj(x1) * (-b * x0 + a * x1)
    want_rq = xAx / ((1 + delta) ** 2 + 1)
    res, rq = R.true_residuals(A, x[:, None], np.array([lam[0]]))
    assert abs(res[0] - want_res) <= 1e-14 * want_res
    assert abs(rq[0] - want_rq) <= 1e-14 * abs(want_rq)


def test_planted_mistakes_in_residual_are_caught(monkeypatch):
    """Each plausible slip in true_residuals fails one of the pins above."""
    import pytest

    good = R.true_residuals

    def frobenius_norm(A, X, lam):          # ||A||_F instead of ||A||_1
        AX = A @ X
        res = np.linalg.norm(AX - X * lam, axis=0) / (sp.linalg.norm(A) * np.linalg.norm(X, axis=0))
        return res, good(A, X, lam)[1]

    def no_conjugate(A, X, lam):            # x^T A x / x^T x for complex x
        AX = A @ X
        return good(A, X, lam)[0], np.einsum("ij,ij->j", X, AX) / np.einsum("ij,ij->j", X, X)

    def plus_sign(A, X, lam):               # A x + l x
        AX = A @ X
        res = np.linalg.norm(AX + X * lam, axis=0) / (R.norm1(A) * np.linalg.norm(X, axis=0))
        return res, good(A, X, lam)[1]

    for bad, test in ((frobenius_norm, test_perturbed_eigenvector_residual_and_quotient_by_hand),
                      (no_conjugate, test_complex_pair_residual_and_quotient),
                      (plus_sign, test_toeplitz_eigenvectors_have_zero_residual_and_exact_quotient)):
        monkeypatch.setattr(R, "true_residuals", bad)
        with np.errstate(all="ignore"), pytest.raises(AssertionError):
            test()
        monkeypatch.setattr(R, "true_residuals", good)
