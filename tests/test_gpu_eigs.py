"""The eigensolver of the deflation (nk_eigs_smallest) against the oracle's
dense eigendecomposition of A on a 3^3 x 4 lattice (N = 1296).

The critical eigenpairs of LR deflation (App. C step 1; Sec. 3 deflates those
of smallest modulus) from k steps of the device's (two-sided) Lanczos
recurrence with both bases kept, Ritz values of H_k nearest zero and their
eigenvectors lifted through the bases:
* mu = 0 (Hermitian): the 16 eigenvalues are the 16 of smallest |lambda| of
  the dense A, the eigenvectors are those of the oracle up to a phase, and a
  solve deflated with them equals the solve deflated with the oracle's pairs;
* mu = 0.3 (two-sided): the m eigenvalues are those of smallest modulus of
  the dense A (the Rayleigh quotients <l, A r>, to 1e-12), the reported residual is the larger of the true right and
  left residuals, <l_i, r_i> = 1, and a solve deflated with them equals the
  solve deflated with the oracle's pairs.
At k = 1200 (mu = 0) the converged eigenvalues come in repeated copies (loss
of orthogonality of the unreorthogonalised recurrence), the case the refined
Ritz vectors of a cluster are for.
"""
import numpy as np
import pytest

import inputs
from oracle import deflation, dirac, signfun

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0912_4457_gb300 import nksign  # noqa: E402
from paper_0912_4457_gb300.nksign import NK_FP64, Context  # noqa: E402

DIMS = (3, 3, 3, 4)
M_W = -2.0


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def links():
    return inputs.su3_links(DIMS, 31)[0]


def make(U, mu):
    ctx = Context(DIMS)
    ctx.load_links(U)
    ctx.set_mu_mw(mu, M_W)
    return ctx


@pytest.mark.parametrize("k", [800, 1200])
def test_hermitian_eigenpairs_match_the_dense_oracle(links, k):
    m = 16
    a = dirac.dense_A(links, DIMS, 0.0, M_W)
    lam_or, R_or, _ = deflation.smallest_eigenpairs(a, m, True)
    ctx = make(links, 0.0)
    b = inputs.gaussian_sources(DIMS, 41)[0]
    lam, R, L, res, rc = ctx.eigs_smallest(b, k, m, tol=1e-9)
    assert rc == 0 and len(lam) == m
    assert np.all(np.abs(lam.imag) == 0.0)
    # the 16 smallest |lambda|, in that order
    assert np.allclose(np.abs(lam), np.sort(np.abs(lam_or)), rtol=0, atol=1e-12)
    assert np.all(res <= 1e-9)
    for i in range(m):
        r = R[i]
        assert np.linalg.norm(r) == pytest.approx(1.0, abs=1e-12)
        assert np.linalg.norm(a @ r - lam[i] * r) == pytest.approx(res[i], rel=1e-6, abs=1e-13)
        j = int(np.argmin(np.abs(lam_or - lam[i])))
        assert abs(np.vdot(R_or[:, j], r)) == pytest.approx(1.0, abs=1e-8)   # same vector up to a phase
        assert np.array_equal(L[i], r)
    ctx.close()


def test_hermitian_deflation_with_the_solver_pairs_matches_the_oracle_pairs(links):
    m, k_solve, ell = 16, 144, 48
    a = dirac.dense_A(links, DIMS, 0.0, M_W)
    lam_or, R_or, _ = deflation.smallest_eigenpairs(a, m, True)
    ctx = make(links, 0.0)
    lam, R, _, _, _ = ctx.eigs_smallest(inputs.gaussian_sources(DIMS, 41)[0], 800, m, tol=1e-9)
    b = inputs.gaussian_sources(DIMS, 32, n_rhs=2)
    ctx.set_deflation(lam, R, None)
    y, st, rc = ctx.sign_apply(b, k_solve, ell, flags=NK_FP64)
    ctx.set_deflation(lam_or, R_or.T, None)
    y_or, _, _ = ctx.sign_apply(b, k_solve, ell, flags=NK_FP64)
    truth = np.stack([signfun.sign_spectral(a, True) @ b[i] for i in range(2)])
    for i in range(2):
        # the same deflated space up to the eigenvectors' error (residual /
        # gap): the two solves reach the truth alike
        assert rel(y[i], y_or[i]) < 1e-6
        assert rel(y[i], truth[i]) < 2.0 * rel(y_or[i], truth[i]) + 1e-8
    ctx.close()


def test_two_sided_eigenpairs_are_eigenpairs_of_the_dense_operator(links):
    m, k, tol = 6, 1000, 1e-8
    a = dirac.dense_A(links, DIMS, 0.3, M_W)
    ev = np.linalg.eigvals(a)
    smallest = ev[np.argsort(np.abs(ev))][:m]
    ctx = make(links, 0.3)
    lam, R, L, res, rc = ctx.eigs_smallest(inputs.gaussian_sources(DIMS, 41)[0], k, m, tol=tol)
    assert rc == 0 and len(lam) == m
    assert np.all(np.diff(np.abs(lam)) >= 0)
    # the m eigenvalues of smallest modulus: Rayleigh quotients, far more
    # accurate than the residual (1e-9) that H_k's eigenvalues are limited to
    assert np.max(np.abs(np.sort_complex(lam) - np.sort_complex(smallest))) < 1e-12
    for i in range(m):
        r, l = R[i], L[i]
        res_r = np.linalg.norm(a @ r - lam[i] * r)
        res_l = np.linalg.norm(a.conj().T @ l - np.conj(lam[i]) * l) / np.linalg.norm(l)
        # the reported residual is the larger of the two, and it is <= tol
        assert res[i] <= tol
        assert max(res_r, res_l) == pytest.approx(res[i], rel=1e-6, abs=1e-13)
        assert np.linalg.norm(r) == pytest.approx(1.0, abs=1e-12)
        assert np.vdot(l, r) == pytest.approx(1.0, abs=1e-12)
    ctx.close()


def test_two_sided_deflation_with_the_solver_pairs_matches_the_oracle_pairs(links):
    m, k_solve, ell = 6, 144, 48
    a = dirac.dense_A(links, DIMS, 0.3, M_W)
    lam_or, R_or, L_or = deflation.smallest_eigenpairs(a, m, False)
    ctx = make(links, 0.3)
    lam, R, L, _, _ = ctx.eigs_smallest(inputs.gaussian_sources(DIMS, 41)[0], 1000, m, tol=1e-8)
    b = inputs.gaussian_sources(DIMS, 32, n_rhs=2)
    truth = np.stack([signfun.sign_spectral(a, False) @ b[i] for i in range(2)])
    y0, _, _ = ctx.sign_apply(b, k_solve, ell, flags=NK_FP64)
    ctx.set_deflation(lam, R, L)
    y, st, rc = ctx.sign_apply(b, k_solve, ell, flags=NK_FP64)
    assert rc == 0 and st["defl_m"] == m
    ctx.set_deflation(lam_or, R_or.T, L_or.T)
    y_or, _, _ = ctx.sign_apply(b, k_solve, ell, flags=NK_FP64)
    for i in range(2):
        # the same deflated space up to the eigenvectors' error: the solve
        # deflated with the solver's pairs is the one deflated with the exact
        # pairs, and both are closer to the truth than the undeflated one
        assert rel(y[i], y_or[i]) < 1e-6
        assert rel(y[i], truth[i]) < 1.01 * rel(y_or[i], truth[i]) + 1e-9
        assert rel(y[i], truth[i]) < rel(y0[i], truth[i])
    ctx.close()


def test_eigensolver_arguments_and_too_small_k(links):
    ctx = make(links, 0.0)
    b = inputs.gaussian_sources(DIMS, 41)[0]
    # k odd, k < 2 m + 2, m above the deflation maximum (256), tol not positive
    for k, m, tol in [(31, 4, 1e-9), (8, 4, 1e-9), (800, 257, 1e-9), (800, 4, 0.0)]:
        assert ctx.eigs_smallest(b, k, m, tol=tol, check=False)[4] == nksign.NK_EINVAL
    # too short a recurrence: fewer pairs converge, and the ones found are returned
    lam, R, L, res, rc = ctx.eigs_smallest(b, 300, 16, tol=1e-9, check=False)
    assert rc == nksign.NK_ENOTCONV and len(lam) < 16 and np.all(res <= 1e-9)
    ctx.close()
