"""Pins for the oracle's matrix sign function, Krylov recurrences and nesting.

* spectral sign vs scipy's independent ``signm``;
* RHi vs the spectral sign, and a 2x2 closed form;
* algebraic invariants of the dense truth on a lattice: sgn(A)^2 = 1,
  [sgn(A), A] = 0, Ginsparg-Wilson, and at mu = 0 the unit circle;
* Lanczos / two-sided Lanczos: (bi)orthonormality and W^dagger A V = H;
* Krylov-Ritz converges to the dense truth; nested with l = k equals plain
  (Sec. 4.2: "for l -> k the nested solution converges to the non-nested one").
"""
import numpy as np
import pytest
import scipy.linalg

import inputs
from oracle import dirac, freefield, krylov, nested, signfun

DIMS2 = (2, 2, 2, 2)


@pytest.fixture(scope="module")
def lattice2():
    U, _ = inputs.su3_links(DIMS2, seed=61)
    return U


def _rand_offaxis(n, rng, complex_=True, shift=1.0):
    """Random matrix whose eigenvalues stay away from the imaginary axis."""
    q = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if complex_ else 0)
    lam = rng.uniform(0.3, 3.0, n) * rng.choice([-1, 1], n)
    if complex_:
        lam = lam + 1j * rng.uniform(-0.5, 0.5, n)
    return q @ np.diag(lam) @ np.linalg.inv(q)


def test_spectral_sign_vs_scipy_signm():
    rng = np.random.default_rng(1)
    a = _rand_offaxis(12, rng)
    assert np.abs(signfun.sign_general(a) - scipy.linalg.signm(a)).max() < 1e-8
    h = rng.standard_normal((10, 10)) + 1j * rng.standard_normal((10, 10))
    h = h + h.conj().T
    assert np.abs(signfun.sign_hermitian(h) - scipy.linalg.signm(h)).max() < 1e-8


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_dense_lattice_sign_vs_scipy(lattice2, mu):
    a = dirac.dense_A(lattice2, DIMS2, mu, -2.0)
    s = signfun.sign_spectral(a, hermitian=(mu == 0.0))
    assert np.abs(s - scipy.linalg.signm(a)).max() < 1e-7


def test_rhi_vs_spectral_and_2x2_closed_form():
    rng = np.random.default_rng(2)
    a = _rand_offaxis(16, rng)
    s, it, conv = signfun.rhi(a)
    assert conv and it <= 20
    assert np.abs(s - signfun.sign_general(a)).max() < 1e-10
    # 2x2 with eigenvalues of opposite sign: sgn(M) = (2M - tr(M) 1) / (l1 - l2)
    m = np.array([[1.5, 2.0 - 1j], [0.3j, -0.7]])
    l1, l2 = np.linalg.eigvals(m)
    if l1.real < 0:
        l1, l2 = l2, l1
    closed = (2 * m - np.trace(m) * np.eye(2)) / (l1 - l2)
    s2, _, _ = signfun.rhi(m)
    assert np.abs(s2 - closed).max() < 1e-13


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_dense_truth_invariants(lattice2, mu):
    a = dirac.dense_A(lattice2, DIMS2, mu, -2.0)
    s = signfun.sign_spectral(a, hermitian=(mu == 0.0))
    n = a.shape[0]
    assert np.abs(s @ s - np.eye(n)).max() < 1e-11                  # sgn^2 = 1
    assert np.abs(s @ a - a @ s).max() < 1e-11                      # [sgn A, A] = 0
    g5 = np.kron(np.eye(n // 12), np.kron(dirac.GAMMA5, np.eye(3)))
    dov = np.eye(n) + g5 @ s                                        # Eq. Dovmu
    assert np.abs(g5 @ dov + dov @ g5 - dov @ g5 @ dov).max() < 1e-11   # Ginsparg-Wilson
    if mu == 0.0:
        lam = np.linalg.eigvals(dov)
        assert np.abs(np.abs(lam - 1.0) - 1.0).max() < 1e-10       # unit circle


def test_lanczos_orthonormal_and_projection(lattice2):
    a, _, _ = nested.operator(lattice2, DIMS2, 0.0, -2.0)
    x = inputs.gaussian_sources(DIMS2, seed=62)[0]
    k = 24
    res = krylov.lanczos(a, x, k)
    V = res.V
    assert np.abs(V.conj().T @ V - np.eye(k)).max() < 1e-10
    AV = np.stack([a(V[:, j]) for j in range(k)], axis=1)
    assert np.abs(V.conj().T @ AV - res.H()).max() < 1e-10
    assert np.allclose(res.beta, res.gamma) and np.isrealobj(res.H())
    assert np.abs(res.alpha_imag).max() < 1e-12


def test_two_sided_biorthonormal_and_projection(lattice2):
    a, adag, _ = nested.operator(lattice2, DIMS2, 0.3, -2.0)
    x = inputs.gaussian_sources(DIMS2, seed=63)[0]
    k = 24
    res = krylov.two_sided_lanczos(a, adag, x, k, store_left=True)
    V, W = res.V, res.W
    assert np.abs(W.conj().T @ V - np.eye(k)).max() < 1e-9         # w_j^dag v_i = delta_ij
    AV = np.stack([a(V[:, j]) for j in range(k)], axis=1)
    assert np.abs(W.conj().T @ AV - res.H()).max() < 1e-9          # H = W^dag A V
    # the coefficient choice makes |beta| = |gamma|
    assert np.allclose(np.abs(res.beta), np.abs(res.gamma))


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_krylov_ritz_converges_to_dense(lattice2, mu):
    x = inputs.gaussian_sources(DIMS2, seed=64)[0]
    truth, _ = nested.sign_apply(lattice2, DIMS2, mu, -2.0, x, method="dense")
    errs = []
    for k in (16, 96, 192):            # 192 = dim(A): the Krylov space is all of C^n
        y, _ = nested.sign_apply(lattice2, DIMS2, mu, -2.0, x, k, method="plain")
        errs.append(np.linalg.norm(y - truth) / np.linalg.norm(truth))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-10


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_nested_with_l_equal_k_is_plain(lattice2, mu):
    x = inputs.gaussian_sources(DIMS2, seed=65)[0]
    k = 40
    yp, _ = nested.sign_apply(lattice2, DIMS2, mu, -2.0, x, k, method="plain")
    yn, _ = nested.sign_apply(lattice2, DIMS2, mu, -2.0, x, k, k, method="nested")
    assert np.linalg.norm(yn - yp) / np.linalg.norm(yp) < 1e-10


@pytest.mark.parametrize("mu,k,ell", [(0.0, 64, 24), (0.3, 80, 32)])
def test_nested_reaches_plain_at_small_l(lattice2, mu, k, ell):
    """l << k already reaches the accuracy of the non-nested method (Sec. 4.2)."""
    x = inputs.gaussian_sources(DIMS2, seed=66)[0]
    truth, _ = nested.sign_apply(lattice2, DIMS2, mu, -2.0, x, method="dense")
    yp, _ = nested.sign_apply(lattice2, DIMS2, mu, -2.0, x, k, method="plain")
    yn, info = nested.sign_apply(lattice2, DIMS2, mu, -2.0, x, k, ell)
    ep = np.linalg.norm(yp - truth) / np.linalg.norm(truth)
    en = np.linalg.norm(yn - truth) / np.linalg.norm(truth)
    assert en < 2.0 * ep + 1e-13
    assert info["rhi_converged"] and info["rhi_iters"] <= 10        # "7 to 10" (Sec. 3)


def test_sgn2_estimate_tracks_true_error(lattice2):
    """The sgn^2 estimate of Sec. 3 is consistent with the true error."""
    x = inputs.ones_source(DIMS2)[0]
    truth, _ = nested.sign_apply(lattice2, DIMS2, 0.0, -2.0, x, method="dense")
    for k in (8, 16):
        y, _ = nested.sign_apply(lattice2, DIMS2, 0.0, -2.0, x, k, k)
        true_err = np.linalg.norm(y - truth) / np.linalg.norm(truth)
        est = nested.sgn2_error(lattice2, DIMS2, 0.0, -2.0, x, k, k)
        assert 0.05 * true_err < est < 20.0 * true_err


def test_overlap_unit_circle_via_nested(lattice2):
    """D_ov from the nested sign keeps the Ginsparg-Wilson relation on vectors."""
    x, z = inputs.gaussian_sources(DIMS2, seed=67, n_rhs=2)
    d = lambda v: nested.overlap_apply(lattice2, DIMS2, 0.0, -2.0, v, 192, 96, method="nested")[0]
    g5 = lambda v: dirac.gamma5(v, DIMS2)
    # <z, (g5 D + D g5 - D g5 D) x> = 0
    lhs = g5(d(x)) + d(g5(x)) - d(g5(d(x)))
    assert np.linalg.norm(lhs) < 1e-8 * np.linalg.norm(x)


# ---- free field and pure gauge: exact answers at any size (oracle/freefield.py)


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_free_field_sign_matches_dense_sign(mu):
    """Momentum-space sgn(A) b equals the dense spectral sgn of the
    real-space operator (a separate construction: the stencil's matrix and
    its eigendecomposition) on a lattice with four different extents."""
    dims = (2, 3, 2, 4)
    U = inputs.unit_links(dims)
    b = inputs.gaussian_sources(dims, seed=7)[0]
    exact = freefield.free_sign_apply(b, dims, mu, -1.5)
    dense = nested.sign_apply(U, dims, mu, -1.5, b, method="dense")[0]
    assert np.abs(exact - dense).max() < 1e-11 * np.abs(dense).max()


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_pure_gauge_sign_is_the_rotated_free_sign(mu):
    """sgn(A_U) W b = W sgn(A_1) b for U_nu(x) = W(x+nu) W(x)^+."""
    dims = (2, 2, 3, 4)
    W = inputs.gauge_transform(dims, seed=8)
    U = freefield.pure_gauge_links(W)
    b = inputs.gaussian_sources(dims, seed=9)[0]
    want = freefield.rotate(W, freefield.free_sign_apply(b, dims, mu, -1.5), dims)
    got = nested.sign_apply(U, dims, mu, -1.5, freefield.rotate(W, b, dims), method="dense")[0]
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()
    # the links are far from the identity
    assert np.abs(U - inputs.unit_links(dims)).max() > 0.5
