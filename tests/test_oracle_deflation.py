"""Pins of the LR deflation oracle (oracle/deflation.py, App. C steps 1, 6).

* The eigenpairs from the dense eigendecomposition satisfy A R = R Lambda,
  L^dagger A = Lambda L^dagger and L^dagger R = I, and are those of smallest
  modulus (every other eigenvalue lies outside the deflation gap Delta).
* Step 1 removes exactly the deflated components: L^dagger x_minus = 0.
* With no eigenpairs the deflated method is the undeflated one.
* Against the dense truth sgn(A) x (spectral definition, Eqs. fAdef, sgnz) the
  deflated approximation is far more accurate at the same k (Sec. 3: the
  deflation gap lets the Krylov space stay small).
"""
import numpy as np
import pytest

import inputs
from oracle import deflation, dirac, nested, signfun

DIMS = (3, 3, 3, 4)
M_W = -2.0


@pytest.fixture(scope="module", params=[0.0, 0.3])
def case(request):
    mu = request.param
    U = inputs.su3_links(DIMS, 31)[0]
    a = dirac.dense_A(U, DIMS, mu, M_W)
    herm = mu == 0.0
    lam, R, L = deflation.smallest_eigenpairs(a, 16, herm)
    return mu, U, a, herm, lam, R, L


def test_eigenpairs_are_the_smallest_left_and_right(case):
    mu, U, a, herm, lam, R, L = case
    assert np.abs(a @ R - R * lam[None, :]).max() < 1e-10
    assert np.abs(L.conj().T @ a - lam[:, None] * L.conj().T).max() < 1e-10
    assert np.abs(L.conj().T @ R - np.eye(len(lam))).max() < 1e-10
    all_abs = np.sort(np.abs(np.linalg.eigvals(a)))
    assert np.abs(lam).max() == pytest.approx(all_abs[len(lam) - 1], rel=1e-10)
    assert all_abs[len(lam)] >= np.abs(lam).max()


def test_projection_removes_the_deflated_components(case):
    mu, U, a, herm, lam, R, L = case
    x = inputs.gaussian_sources(DIMS, 32)[0]
    xm, d = deflation.project(x, R, L)
    assert np.abs(L.conj().T @ xm).max() < 1e-12 * np.linalg.norm(x)
    assert np.allclose(x, xm + R @ d)


def test_no_eigenpairs_is_the_undeflated_method(case):
    mu, U, a, herm, lam, R, L = case
    x = inputs.gaussian_sources(DIMS, 32)[0]
    e = np.zeros((a.shape[0], 0), complex)
    y0, _ = nested.sign_apply(U, DIMS, mu, M_W, x, 96, 48)
    y1, _ = deflation.sign_apply(U, DIMS, mu, M_W, x, 96, 48, np.zeros(0, complex), e, e)
    assert np.allclose(y0, y1, rtol=0, atol=1e-14 * np.linalg.norm(y0))


def test_deflation_reaches_the_dense_truth_at_smaller_k(case):
    mu, U, a, herm, lam, R, L = case
    x = inputs.gaussian_sources(DIMS, 32)[0]
    truth = signfun.sign_spectral(a, herm) @ x
    err = lambda y: np.linalg.norm(y - truth) / np.linalg.norm(truth)
    y0, _ = nested.sign_apply(U, DIMS, mu, M_W, x, 144, 48)
    y1, _ = deflation.sign_apply(U, DIMS, mu, M_W, x, 144, 48, lam, R, L)
    assert err(y1) < err(y0) / 10
