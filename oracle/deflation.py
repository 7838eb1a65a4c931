"""LR deflation (App. C steps 1 and 6; Sec. 3, deflation paragraph).

Test infrastructure only (see ``oracle/__init__.py``).

Given the m critical eigenvalues lambda_i of A with right eigenvectors r_i and
left eigenvectors l_i normalised to <l_i, r_j> = delta_ij (l_i = r_i for
Hermitian A):
  step 1:  x_minus = x - sum_i <l_i, x> r_i
  step 6:  sgn(A) x ~ sum_i sgn(lambda_i) <l_i, x> r_i + (nested approximation on x_minus)
with sgn(z) = sgn(Re z) (Eq. sgnz).  The paper deflates the eigenvalues of
smallest modulus (the footnote of Sec. 3) and calls the largest deflated
|lambda| the deflation gap Delta.
"""
from __future__ import annotations

import numpy as np

from . import nested, signfun


def smallest_eigenpairs(a_dense, m: int, hermitian: bool):
    """The m eigenvalues of smallest modulus of a dense A with right
    eigenvectors R (columns) and left eigenvectors L (columns) with
    L^dagger R = I (from the full eigendecomposition: the left vectors are the
    rows of the inverse eigenvector matrix)."""
    if hermitian:
        w, v = np.linalg.eigh(a_dense)
        idx = np.argsort(np.abs(w))[:m]
        return w[idx].astype(np.complex128), v[:, idx], v[:, idx]
    w, v = np.linalg.eig(a_dense)
    vinv = np.linalg.inv(v)
    idx = np.argsort(np.abs(w))[:m]
    return w[idx], v[:, idx], np.conj(vinv[idx, :]).T


def project(x, R, L):
    """Step 1: (x_minus, d) with d_i = <l_i, x>."""
    d = L.conj().T @ x
    return x - R @ d, d


def sign_apply(U, dims, mu, m_w, x, k, ell, lam, R, L, p=None, antiperiodic_t=True):
    """App. C steps 1-6: the deflated nested approximation to sgn(A) x."""
    a, adag, herm = nested.operator(U, dims, mu, m_w, antiperiodic_t)
    xm, d = project(np.asarray(x, dtype=np.complex128), R, L)
    y, info = nested.nested_sign(a, adag, xm, k, ell, herm, p)
    s = np.array([signfun.sgn_scalar(z) for z in lam])
    return y + R @ (s * d), dict(info, d=d, x_minus=xm)
