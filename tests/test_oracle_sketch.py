"""Pins of the sparse-sign embedding (oracle side) and of the random inputs.

The embedding is the paper's sparse-sign Omega (Sec. 5 setup; Sec. 1.1
oblivious subspace embeddings, Def. 1.1).  Pins: the published SplitMix64
outputs, the structural invariants of a sparse-sign matrix, its moments, and
the epsilon-embedding property of Def. 1.1 / Cor. 1.2 on random subspaces.
"""
import os

import numpy as np
import pytest

from oracle import sketch as SK
from paper_2508_05400_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_ints(name):
    with open(os.path.join(GOLD, name)) as f:
        return [int(x) for x in f.read().split("\n") if x and not x.startswith("#")]


def test_splitmix64_published_outputs():
    want = _golden_ints("splitmix64_seed1234567.txt")
    # oracle scalar form: state += gamma, output mix(state)
    s, got = 1234567, []
    for _ in range(5):
        s = (s + SK.GAMMA) & SK.MASK
        got.append(SK.mix64_scalar(s))
    assert got == want
    # input-module vector form
    assert [int(x) for x in I.splitmix64_draws(1234567, 0, 5)] == want


def test_hash_vectorised_equals_one_draw_at_a_time():
    n, d, zeta, seed = 700, 80, 4, 0
    rows, signs = SK.rows_signs(n, d, zeta, seed)
    for i in range(n):
        r, s = SK.column_rows_signs_scalar(i, d, zeta, seed)
        assert list(rows[i]) == r and list(signs[i]) == s
    rows8, _ = SK.rows_signs(300, 64, 8, 5)
    for i in range(300):
        assert list(rows8[i]) == SK.column_rows_signs_scalar(i, 64, 8, 5)[0]


@pytest.mark.parametrize("d,zeta", [(80, 4), (64, 8), (320, 8)])
def test_sparse_sign_structure(d, zeta):
    n = 20000
    rows, signs = SK.rows_signs(n, d, zeta, 0)
    assert rows.min() >= 0 and rows.max() < d
    srt = np.sort(rows, axis=1)
    assert np.all(np.diff(srt, axis=1) > 0), "rows of a column must be distinct"
    assert set(np.unique(signs)) == {-1, 1}
    Om = SK.omega_matrix(n, d, zeta, 0)
    col_nnz = np.diff(Om.tocsc().indptr)
    assert np.all(col_nnz == zeta)
    assert np.allclose(np.abs(Om.data), 1 / np.sqrt(zeta))
    # sign balance and uniform rows (chi-square, 6 sigma)
    frac = (signs == 1).mean()
    assert abs(frac - 0.5) < 6 * np.sqrt(0.25 / signs.size)
    hist = np.bincount(rows.ravel(), minlength=d)
    e = rows.size / d
    chi2 = ((hist - e) ** 2 / e).sum()
    assert abs(chi2 - (d - 1)) < 6 * np.sqrt(2 * (d - 1))


def test_seed_changes_embedding():
    a, _ = SK.rows_signs(1000, 80, 4, 0)
    b, _ = SK.rows_signs(1000, 80, 4, 1)
    assert (a != b).mean() > 0.9


def test_expected_squared_norm_is_preserved():
    # E ||Omega x||^2 = ||x||^2 for the 1/sqrt(zeta) scale: the cross terms have
    # zero mean because signs are independent and +-1 with equal probability.
    n, d, zeta = 400, 40, 4
    x = I.normal(7, n)
    r = np.array([np.linalg.norm(SK.omega_matrix(n, d, zeta, s) @ x) ** 2
                  for s in range(300)]) / (x @ x)
    assert abs(r.mean() - 1.0) < 5 * r.std() / np.sqrt(r.size)


@pytest.mark.parametrize("n,cols,d,zeta", [(20000, 41, 80, 4), (50000, 81, 320, 8)])
def test_embedding_of_random_subspace(n, cols, d, zeta):
    # Def. 1.1 / Cor. 1.2: Omega Q (Q orthonormal, n x cols) has singular values
    # near 1.  For an oblivious embedding the spectrum of (Omega Q)^T (Omega Q)
    # follows the Marchenko-Pastur law with edges (1 -+ sqrt(cols/d))^2, and
    # E ||Omega Q||_F^2 = cols exactly.  (The paper's "d = 2k gives eps = 1/sqrt 2"
    # is a rule of thumb: at cols/d = 1/2 the upper edge is ~2.9.)
    Q, _ = np.linalg.qr(I.normal(3, n * cols).reshape(n, cols))
    sv = np.linalg.svd(SK.omega_matrix(n, d, zeta, 0) @ Q, compute_uv=False)
    c = np.sqrt(cols / d)
    assert sv.min() > 0.7 * (1 - c)
    assert sv.max() < 1.15 * (1 + c)
    assert abs(np.mean(sv ** 2) - 1) < 4 * np.sqrt(2.0 / d) / np.sqrt(cols) + 0.01


def test_start_vector_moments():
    x = I.start_vector(200000, 1)
    assert abs(x.mean()) < 5 / np.sqrt(x.size)
    assert abs(x.var() - 1) < 5 * np.sqrt(2 / x.size)
    # fourth moment of N(0,1) is 3
    assert abs((x ** 4).mean() - 3) < 0.1
    assert np.array_equal(x, I.start_vector(200000, 1))
