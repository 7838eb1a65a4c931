"""Matrix sign function: spectral definition and Roberts-Higham iteration.

Test infrastructure only (see ``oracle/__init__.py``).

* Spectral form f(A) = U f(Lambda) U^{-1}  (Sec. 2, Eq. fAdef), with the
  complex sign sgn(z) = z / sqrt(z^2) = sgn(Re z), square-root cut on the
  negative real axis  (Sec. 2, Eq. sgnz).  For Hermitian A the eigenvalues are
  real and sgn(x) = +-1.
* Roberts-Higham iteration (RHi): S_0 = H, S_{n+1} = (S_n + S_n^{-1}) / 2
  (Sec. 3, Eq. Roberts).  The paper iterates until the iterate is exact to
  working precision; the stopping rule here (a reading of that) stops once the relative
  Frobenius change ||S_{n+1} - S_n|| / ||S_{n+1}|| falls below ``RHI_STOP``
  = 1e-10.  In the quadratic regime the error of S_{n+1} is of the order of
  the square of that change, i.e. at rounding level.  At most ``RHI_MAXIT``
  = 50 iterations.
"""
from __future__ import annotations

import numpy as np

RHI_STOP = 1e-10
RHI_MAXIT = 50


def sgn_scalar(z):
    """sgn(z) = sgn(Re z) (Eq. sgnz); 0 on the imaginary axis (undefined there)."""
    return np.sign(np.real(z))


def sign_hermitian(a):
    """sgn(A) for Hermitian A: U diag(sgn lambda) U^dagger (Eq. fAdef)."""
    w, u = np.linalg.eigh(a)
    return (u * np.sign(w)[None, :]) @ u.conj().T


def sign_general(a):
    """sgn(A) for diagonalisable A: U diag(sgn Re lambda) U^{-1} (Eqs. fAdef, sgnz)."""
    w, u = np.linalg.eig(a)
    return np.linalg.solve(u.T, (u * sgn_scalar(w)[None, :]).T).T


def sign_spectral(a, hermitian: bool):
    return sign_hermitian(a) if hermitian else sign_general(a)


def rhi(h, stop: float = RHI_STOP, maxit: int = RHI_MAXIT):
    """Roberts-Higham iteration on a dense matrix (Eq. Roberts).

    Returns ``(S, n_iter, converged)``; ``S`` approximates sgn(h).
    """
    s = np.array(h, dtype=np.result_type(h, np.float64), copy=True)
    for it in range(1, maxit + 1):
        s_new = 0.5 * (s + np.linalg.inv(s))
        diff = np.linalg.norm(s_new - s)
        s = s_new
        if diff <= stop * np.linalg.norm(s):
            return s, it, True
    return s, maxit, False
