"""Pins of the predictor's spectral features (oracle/features.py, entries
4..15) on inputs with closed forms, independent of the oracle's own path.

* A tridiagonal operator T applied to e_1: the (two-sided) Lanczos recurrence
  of App. A / B reproduces T itself (v_j = e_j), so the statistics of H(j,j)
  and |H(j+1,j)| are those of the chosen diagonals: the mean, the standard
  deviation, max |Im H(j,j)| and, for H(j+1,j) = c e^{s j}, the slope s.
* A = diag(w) on 32 dimensions with a generic source: H_32 is similar to A,
  and with well-separated extremes the 30 power / inverse iterations of
  Eq. popt give z_min = min|w|, z_max = max|w| and p = (z_min z_max)^-1/2.
* Entry 14 from sgn(T) e_1 by the eigendecomposition of T (the nested method
  with l = k reproduces the plain Krylov-Ritz value, Sec. 4.2).
* Entry 15 from the scalar Roberts-Higham iteration on the eigenvalues of the
  symmetric inner Ritz matrix H_l (the Frobenius norms of the stopping rule
  are then sums over the eigenvalues), not from the matrix iteration.
"""
import numpy as np
import pytest

from oracle import features as ofeat
from oracle import nested, signfun

K = ofeat.K_FEAT
J = np.arange(K)


def tridiag_op(d, e_sub, e_sup):
    """T as callables (apply, apply^dagger) on vectors of len(d)."""
    T = np.diag(d).astype(complex) + np.diag(e_sub, -1) + np.diag(e_sup, 1)
    return (lambda v: T @ v), (lambda v: T.conj().T @ v), T


def e1(n):
    v = np.zeros(n, complex)
    v[0] = 1.0
    return v


def _check_statistics(f, im_max):
    assert f[4] == pytest.approx(1.5 + 0.01 * 15.5, rel=1e-12)          # mean Re H(j,j)
    assert f[5] == pytest.approx(0.01 * np.sqrt((K * K - 1) / 12.0), rel=1e-9)
    assert f[6] == pytest.approx(im_max, abs=1e-12)
    sub = 0.8 * np.exp(-0.05 * np.arange(K - 1))
    q = np.exp(-0.05)
    mean = 0.8 * (1 - q ** (K - 1)) / (1 - q) / (K - 1)                # geometric sum
    assert f[7] == pytest.approx(mean, rel=1e-12)
    assert f[8] == pytest.approx(np.sqrt(np.mean(sub ** 2) - mean ** 2), rel=1e-9)
    assert f[9] == pytest.approx(-0.05, rel=1e-9)                      # slope of ln|H(j+1,j)|


def test_diagonal_statistics_and_slope_through_the_recurrence():
    """Hermitian: Lanczos on T from e_1 reproduces T (App. A)."""
    n = 40
    d = 1.5 + 0.01 * np.arange(n)
    e = 0.8 * np.exp(-0.05 * np.arange(n - 1))
    A, Ad, T = tridiag_op(d, e, e)
    _check_statistics(ofeat.features_of_operator(A, Ad, True, e1(n)), 0.0)


def test_diagonal_statistics_of_given_coefficients_two_sided():
    """Complex H(j,j): the statistics of given coefficients (the two-sided
    recurrence itself is pinned by its biorthogonality elsewhere)."""
    al = 1.5 + 0.01 * J - 0.002j * J          # negative: max |Im| needs the modulus
    be = (0.8 * np.exp(-0.05 * np.arange(K - 1))).astype(complex)
    _check_statistics(ofeat.spectral_features(al, be, be, False), 0.002 * 31)


def test_p_estimate_of_a_known_spectrum():
    w = np.concatenate([[0.1], np.linspace(1.0, 2.0, 30), [10.0]])
    A = lambda v: w * v
    b = np.random.default_rng(3).standard_normal(32) + 0j
    f = ofeat.features_of_operator(A, A, True, b)
    assert f[0] == pytest.approx(-1.0, abs=1e-10)        # log10 z_min
    assert f[1] == pytest.approx(1.0, abs=1e-10)         # log10 z_max
    assert f[2] == pytest.approx(2.0, abs=1e-10)
    assert f[3] == pytest.approx(0.0, abs=1e-10)         # log10 p, p = (0.1 * 10)^-1/2


def test_tail_weight_and_rhi_count_from_the_spectrum():
    d = np.array([(-1.0) ** j * (1.0 + 0.1 * j) for j in range(K)])
    e = np.full(K - 1, 0.3)
    A, Ad, T = tridiag_op(d, e, e)
    f = ofeat.features_of_operator(A, Ad, True, e1(K))
    lam, Q = np.linalg.eigh(T.real)
    c = Q @ (np.sign(lam) * Q[0])                       # sgn(T) e_1
    c2 = c ** 2
    assert f[10] == pytest.approx(0.5 * np.log10(c2[24:].sum() / c2.sum()), abs=1e-6)
    # RHi count: the scalar iteration x <- (x + 1/x)/2 on the eigenvalues of
    # the (symmetric) inner Ritz matrix H_l, with the Frobenius stopping rule
    # of the matrix iteration (orthogonal eigenvectors: the norms are sums
    # over the eigenvalues)
    p = 10.0 ** f[3]
    _, info = nested.inner_sign(d, e, e, K, p, True)
    x = np.linalg.eigvalsh(info["H_l"])
    for it in range(1, signfun.RHI_MAXIT + 1):
        xn = 0.5 * (x + 1.0 / x)
        done = np.linalg.norm(xn - x) <= signfun.RHI_STOP * np.linalg.norm(xn)
        x = xn
        if done:
            break
    assert f[11] == it
