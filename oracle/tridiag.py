"""Preconditioned Ritz matrix H_k' = [p H_k + (p H_k)^{-1}] / 2 (Eq. precond).

Test infrastructure only (see ``oracle/__init__.py``).

App. C, steps 3-4: factor p H_k by LU with LAPACK gttrf (L unit lower
bidiagonal, U with a diagonal and two super-diagonals, partial pivoting) and
apply H_k' to a vector as
  (a) (p H_k)^{-1} v by the LU back substitution gttrs, and
  (b) (p H_k) v by a tridiagonal (band) matrix-vector product, added to (a).
For the two-sided inner recurrence H_k'^dagger is needed too; it uses the same
factors with gttrs in conjugate-transpose mode and the band product with H^dagger.
In the Hermitian case everything is real (dgttrf/dgttrs), as App. C states.

The tridiagonal is passed as its diagonals (see ``krylov``): ``alpha`` (k),
``beta`` = H(j+1, j) and ``gamma`` = H(j, j+1) (k-1 each).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import lapack


class PrecondLU:
    """LU factors of p H_k, in gttrf form (dl, d, du, du2, ipiv)."""

    def __init__(self, p, alpha, beta, gamma):
        alpha = np.asarray(alpha)
        self.real = not (np.iscomplexobj(alpha) or np.iscomplexobj(beta) or np.iscomplexobj(gamma))
        dt = np.float64 if self.real else np.complex128
        self.p = float(p)
        self.alpha = np.asarray(alpha, dtype=dt)
        self.beta = np.asarray(beta, dtype=dt)
        self.gamma = np.asarray(gamma, dtype=dt)
        gttrf = lapack.dgttrf if self.real else lapack.zgttrf
        dl, d, du, du2, ipiv, info = gttrf(self.p * self.beta, self.p * self.alpha, self.p * self.gamma)
        if info < 0:
            raise ValueError("gttrf: illegal argument %d" % -info)
        self.singular = info > 0
        self.factors = (dl, d, du, du2, ipiv)

    def solve(self, v, conj_trans: bool = False):
        """(p H)^{-1} v, or ((p H)^dagger)^{-1} v, by gttrs."""
        gttrs = lapack.dgttrs if self.real else lapack.zgttrs
        trans = "N" if not conj_trans else ("T" if self.real else "C")
        x, info = gttrs(*self.factors, np.asarray(v).reshape(-1, 1), trans=trans)
        if info != 0:
            raise ValueError("gttrs failed: %d" % info)
        return x[:, 0]

    def band_mv(self, v, dagger: bool = False):
        """(p H) v or (p H)^dagger v for the tridiagonal H."""
        v = np.asarray(v)
        if not dagger:
            sub, diag, sup = self.beta, self.alpha, self.gamma
        else:
            sub, diag, sup = np.conj(self.gamma), np.conj(self.alpha), np.conj(self.beta)
        y = diag * v
        y[1:] += sub * v[:-1]
        y[:-1] += sup * v[1:]
        return self.p * y

    def apply_hprime(self, v, dagger: bool = False):
        """H_k' v = [(pH) v + (pH)^{-1} v] / 2  (or the same with H^dagger)."""
        return 0.5 * (self.band_mv(v, dagger) + self.solve(v, conj_trans=dagger))


def hprime_dense(p, h):
    """Dense H' = [pH + (pH)^{-1}]/2, for tests on small matrices only."""
    ph = p * np.asarray(h)
    return 0.5 * (ph + np.linalg.inv(ph))
