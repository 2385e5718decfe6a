"""Pins of the reference solvers (oracle/solvers.py) against facts that do not
come from the solvers themselves: least squares from numpy's SVD-based
lstsq, one-step solutions of a single equation and of a diagonal system, a
consistent nonnegative system whose residual must vanish, and the
subset partition."""
import numpy as np
import pytest

from oracle import solvers as S


def _ops(M):
    return (lambda x: M @ x), (lambda y: M.T @ y)


def test_cgls_reaches_least_squares():
    rng = np.random.default_rng(1)
    M = rng.normal(size=(40, 12))
    b = rng.normal(size=40)
    f, bt = _ops(M)
    x, hist = S.cgls(f, bt, b, np.zeros(12), 20)
    want = np.linalg.lstsq(M, b, rcond=None)[0]
    assert np.allclose(x, want, rtol=1e-9, atol=1e-11)
    # the normal-equations residual decreases to ~0 within n iterations
    assert np.linalg.norm(M.T @ (b - M @ hist[11])) < 1e-8 * np.linalg.norm(M.T @ b)


def test_cgls_first_step_is_exact_line_search():
    """After one step x1 = alpha A^T b with alpha minimising |A x - b| along A^T b."""
    rng = np.random.default_rng(2)
    M = rng.normal(size=(9, 5))
    b = rng.normal(size=9)
    f, bt = _ops(M)
    x1 = S.cgls(f, bt, b, np.zeros(5), 1)[0]
    d = M.T @ b
    ts = np.linspace(0.0, 2.0, 20001) * (x1 @ d) / (d @ d)
    best = ts[np.argmin([np.linalg.norm(M @ (t * d) - b) for t in ts])]
    assert np.allclose(x1, best * d, rtol=2e-4)


def test_sart_single_equation_one_step():
    """One equation a x = b in one unknown: SART lands on b / a in one step."""
    M = np.array([[2.5]])
    f, bt = _ops(M)
    x, _ = S.ossart([f], [bt], [np.array([7.0])], np.array([0.3]), 1, nonneg=False)
    assert x[0] == pytest.approx(7.0 / 2.5, rel=1e-15)


def test_sart_diagonal_system_one_iteration():
    rng = np.random.default_rng(3)
    d = rng.uniform(0.5, 2.0, size=7)
    M = np.diag(d)
    b = rng.uniform(0, 1, size=7)
    f, bt = _ops(M)
    x, _ = S.ossart([f], [bt], [b], np.zeros(7), 1)
    assert np.allclose(x, b / d, rtol=1e-14)


def test_ossart_consistent_nonnegative_system_converges():
    """Nonnegative A, b = A x_true with x_true >= 0, three subsets of rows:
    the residual goes to 0 and x to x_true (full column rank)."""
    rng = np.random.default_rng(4)
    M = rng.uniform(0, 1, size=(60, 10)) * (rng.uniform(size=(60, 10)) < 0.5)
    x_true = rng.uniform(0.2, 1.0, size=10)
    b = M @ x_true
    subsets = [np.arange(0, 20), np.arange(20, 40), np.arange(40, 60)]
    fs = [(lambda x, s=s: M[s] @ x) for s in subsets]
    bs = [(lambda y, s=s: M[s].T @ y) for s in subsets]
    x, hist = S.ossart(fs, bs, [b[s] for s in subsets], np.zeros(10), 400)
    assert np.linalg.norm(M @ x - b) < 1e-6 * np.linalg.norm(b)
    assert np.allclose(x, x_true, rtol=1e-4)
    res = [np.linalg.norm(M @ h - b) for h in hist]
    assert res[-1] < res[0] < np.linalg.norm(b)


def test_ossart_untouched_elements_keep_their_value():
    M = np.array([[1.0, 0.0], [2.0, 0.0]])  # no ray crosses element 1
    f, bt = _ops(M)
    x, _ = S.ossart([f], [bt], [np.array([1.0, 2.0])], np.array([0.0, 0.7]), 3)
    assert x[1] == 0.7 and x[0] == pytest.approx(1.0)


def test_angle_blocks_partition():
    bl = S.angle_blocks(100, 20)
    assert len(bl) == 5 and all(len(b) == 20 for b in bl)
    assert np.array_equal(np.concatenate(bl), np.arange(100))
    bl = S.angle_blocks(7, 3)
    assert [len(b) for b in bl] == [3, 3, 1]


def test_inverse_or_zero():
    assert np.array_equal(S.inverse_or_zero([0.0, 2.0, -1.0]), [0.0, 0.5, 0.0])
