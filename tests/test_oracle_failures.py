"""The oracle on the inputs that drive the failure statuses of the GPU path.

* A source that is an eigenvector of A leaves r = 0 after the first step:
  the recurrence stops (App. B serious breakdown; in the Hermitian case the
  undefined v_2 = r / 0 of App. A, reported the same way).  On the free field
  with periodic t, A = gamma5 (1 - 8 kappa) on constant vectors, so the
  constant spin-0 colour-0 vector is one (eigenvalue -1 at m_w = -2).
* A tridiagonal H with a purely imaginary spectrum (skew-symmetric: zero
  diagonal, H(j, j+1) = -H(j+1, j)) has no sign (Eq. sgnz leaves the
  imaginary axis undefined): H' = (pH + (pH)^-1) / 2 is skew as well, and the
  Roberts-Higham iteration stays on the imaginary axis and never converges.
"""
import numpy as np

import inputs
from oracle import krylov, nested

M_W = -2.0


def eigen_source(dims):
    b = np.zeros(12 * int(np.prod(dims)), complex)
    b[0::12] = 1.0        # spin 0, colour 0 on every site
    return b


def skew_tridiagonal():
    beta = np.array([0.5, 0.3, 2.0, 0.7, 1.3, 0.4, 1.1], dtype=complex)
    return np.zeros(8, complex), beta, -beta


def test_eigenvector_source_is_an_exact_eigenvector():
    dims = (4, 4, 4, 4)
    A, _, _ = nested.operator(inputs.unit_links(dims), dims, 0.0, M_W, antiperiodic_t=False)
    b = eigen_source(dims)
    assert np.array_equal(A(b), -b)


def test_eigenvector_source_breaks_the_recurrence_down():
    dims = (4, 4, 4, 4)
    b = eigen_source(dims)
    for mu in (0.0,):
        A, Ad, herm = nested.operator(inputs.unit_links(dims), dims, mu, M_W, antiperiodic_t=False)
        out = nested.outer_basis(A, Ad, b, 8, herm)
        assert out.breakdown and out.k_used == 1
        assert out.alpha[0] == -1.0
    # the two-sided recurrence on a Hermitian A from the same source (delta = 0)
    A, Ad, _ = nested.operator(inputs.unit_links(dims), dims, 0.0, M_W, antiperiodic_t=False)
    out = krylov.two_sided_lanczos(A, Ad, b, 8)
    assert out.breakdown and out.k_used == 1


def test_skew_tridiagonal_has_no_sign():
    al, be, ga = skew_tridiagonal()
    h = np.diag(al) + np.diag(be, -1) + np.diag(ga, 1)
    ev = np.linalg.eigvals(h)
    assert np.allclose(ev.real, 0.0, atol=1e-12)
    p, _, _ = nested.estimate_p(al, be, ga)
    for ell in (4, 8):
        _, info = nested.inner_sign(al, be, ga, ell, p, False)
        assert not info["rhi_converged"] and info["rhi_iters"] == 50
        assert not info["inner_breakdown"] and not info["lu_singular"]
