"""The identities behind the overlap inversion, on the dense oracle.

* D_ov(mu)^dagger = gamma5 D_ov(-mu) gamma5 (Eq. Dovmu; A(mu)^dagger = A(-mu)
  and sgn(A)^dagger = sgn(A^dagger)): the adjoint that the CG on the normal
  equations applies.
* At mu = 0, D_ov satisfies the Ginsparg-Wilson relation D + D^dagger =
  D^dagger D: D_ov is normal with its spectrum on the unit circle about 1, so
  the singular values of D_ov + m (m > 0) are at least m.
"""
import numpy as np
import pytest

import inputs
from oracle import dirac, signfun

DIMS = (3, 3, 3, 4)
M_W = -2.0


def dense_overlap(U, mu):
    a = dirac.dense_A(U, DIMS, mu, M_W)
    s = signfun.sign_spectral(a, mu == 0.0)
    n = a.shape[0]
    g5 = np.diag(np.tile([1.0] * 6 + [-1.0] * 6, n // 12)).astype(complex)
    return np.eye(n) + g5 @ s, g5


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_adjoint_is_gamma5_overlap_at_minus_mu_gamma5(mu):
    U = inputs.su3_links(DIMS, 31)[0]
    d, g5 = dense_overlap(U, mu)
    dm, _ = dense_overlap(U, -mu)
    assert np.abs(d.conj().T - g5 @ dm @ g5).max() < 1e-12


def test_ginsparg_wilson_and_shifted_singular_values():
    U = inputs.su3_links(DIMS, 31)[0]
    d, _ = dense_overlap(U, 0.0)
    assert np.abs(d + d.conj().T - d.conj().T @ d).max() < 1e-12
    m = 0.2
    sv = np.linalg.svd(d + m * np.eye(d.shape[0]), compute_uv=False)
    assert sv.min() >= m - 1e-12
