"""Pins of the oracle's (eps, k) column / row ID (Sec. 2.1, Lemma 2.1)."""
import numpy as np
import pytest

from oracle import interp


def _cplx(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _reconstruct(A, r):
    out = np.empty_like(A)
    out[:, r.q] = A[:, r.q]
    out[:, r.p] = A[:, r.q] @ r.T
    return out


@pytest.mark.parametrize("m,n,rank", [(60, 40, 7), (30, 30, 1), (100, 12, 11)])
def test_column_id_is_exact_on_low_rank(m, n, rank):
    rng = np.random.default_rng(m + n)
    A = _cplx(rng, m, rank) @ _cplx(rng, rank, n)
    r = interp.column_id(A, 1e-12, 0)
    assert r.k == rank
    assert set(r.q.tolist()) | set(r.p.tolist()) == set(range(n))
    assert np.linalg.norm(A - _reconstruct(A, r)) < 1e-11 * np.linalg.norm(A)


def test_column_id_error_is_order_eps():
    rng = np.random.default_rng(1)
    m, n = 80, 50
    Uq, _ = np.linalg.qr(_cplx(rng, m, n))
    Vq, _ = np.linalg.qr(_cplx(rng, n, n))
    sig = 10.0 ** (-0.5 * np.arange(n))
    A = (Uq * sig) @ Vq.conj().T
    for eps in (1e-4, 1e-6, 1e-9):
        r = interp.column_id(A, eps, 0)
        err = np.linalg.norm(A - _reconstruct(A, r), 2)
        assert err <= 50 * eps * sig[0]
        svd_rank = int(np.sum(sig > eps * sig[0]))
        assert abs(r.k - svd_rank) <= 2


def _pivoted_gram_schmidt(A, k):
    """Textbook Businger-Golub pivoting: take the column of largest residual norm, then
    project it out of the others (classical Gram-Schmidt, reorthogonalised)."""
    R = A.copy()
    piv, diag = [], []
    for _ in range(k):
        norms = np.linalg.norm(R, axis=0)
        norms[piv] = -1
        j = int(np.argmax(norms))
        piv.append(j)
        diag.append(norms[j])
        qv = R[:, j] / norms[j]
        for _ in range(2):
            R = R - np.outer(qv, qv.conj() @ R)
    return piv, np.array(diag)


def test_pivots_and_diagonal_match_textbook_pivoting():
    rng = np.random.default_rng(7)
    A = _cplx(rng, 30, 12) * (3.0 ** -np.arange(12))[None, :] @ np.diag(np.exp(1j * np.arange(12)))
    r = interp.column_id(A, 0.0, 0)
    piv, diag = _pivoted_gram_schmidt(A, 12)
    assert list(r.q[:8]) == piv[:8]
    assert np.allclose(r.rdiag[:8], diag[:8], rtol=1e-10)
    norms = np.linalg.norm(A, axis=0)
    assert r.q[0] == int(np.argmax(norms))


def test_rank_rule():
    d = np.array([2.0, 1.0, 3e-6, 1e-6, 1e-9])
    assert interp.rank_from_diag(d, 1e-6, 10) == 3       # 3e-6 > 2e-6 kept; 1e-6 <= 2e-6 dropped
    assert interp.rank_from_diag(d, 1e-6, 2) == 2        # rank parameter k caps k_eps
    assert interp.rank_from_diag(d, 0.0, 10) == 5
    assert interp.rank_from_diag(np.zeros(4), 1e-6, 4) == 1
    assert interp.rank_from_diag(d, 10.0, 10) == 1       # at least one skeleton


def test_zero_block_gives_rank_one_and_zero_T():
    r = interp.column_id(np.zeros((5, 4), dtype=complex), 1e-6, 0)
    assert r.k == 1 and np.all(r.T == 0) and r.T.shape == (1, 3)


def test_row_id_reconstructs():
    rng = np.random.default_rng(3)
    A = _cplx(rng, 35, 5) @ _cplx(rng, 5, 70)
    r = interp.row_id(A, 1e-12, 0)
    assert r.k == 5
    U = np.zeros((35, r.k), dtype=complex)
    U[r.q, np.arange(r.k)] = 1.0
    U[r.p, :] = r.T.T
    assert np.linalg.norm(A - U @ A[r.q, :]) < 1e-11 * np.linalg.norm(A)


def test_sampled_rows_give_the_same_skeleton_on_low_rank():
    # Eq. pivotedQR2: the ID of a tall low-rank block from t*k sampled rows is exact
    rng = np.random.default_rng(9)
    A = _cplx(rng, 400, 6) @ _cplx(rng, 6, 30)
    s = np.sort(rng.choice(400, 12, replace=False))
    r = interp.column_id(A[s], 1e-12, 0)
    assert r.k == 6
    assert np.linalg.norm(A - _reconstruct(A, r)) < 1e-10 * np.linalg.norm(A)
