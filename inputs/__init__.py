"""Seeded synthetic inputs for the nested Krylov-Ritz sign function.

This module is shared by the CPU oracle and by the GPU path. It produces
*data* only: gauge links, source vectors and gauge transformations. It holds
none of the method's arithmetic (no Wilson operator, no Krylov recurrence, no
sign function), so that the oracle and the CUDA path share inputs but no code.

Conventions (fixed by the C-ABI, see include/nksign.h):

* ``dims = (Lx, Ly, Lz, Lt)``; site index ``s = x + Lx*(y + Ly*(z + Lz*t))``.
* Link array: complex128, shape ``(Lt, Lz, Ly, Lx, 4, 3, 3)``; ``U[t,z,y,x,nu]``
  is the SU(3) matrix ``U_{x,+nu}`` for ``nu = 0, 1, 2, 3`` = x, y, z, t.  The
  flattened memory order is the ABI's ``[t][z][y][x][nu][3][3]``.
* Spinor vector: complex128, length ``12*V``, element ``12*s + 3*spin + colour``.
  As an array it has shape ``(Lt, Lz, Ly, Lx, 4, 3)``.

The paper's runs use Monte-Carlo gauge ensembles that are not available. The
stand-in is a field of independent links ``U = exp(i eps X)`` with ``X`` a random
traceless Hermitian 3x3 matrix and ``eps`` set by bisection so that the mean
plaquette hits a target (0.59 by default).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "volume",
    "plaquette",
    "su3_links",
    "gaussian_sources",
    "point_sources",
    "ones_source",
    "gauge_transform",
    "unit_links",
]


def volume(dims) -> int:
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def _shape(dims):
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def _dagger(m):
    return np.conj(np.swapaxes(m, -1, -2))


def plaquette(U: np.ndarray) -> float:
    """Mean plaquette (1/3) Re tr U_p over all sites and the 6 planes mu < nu."""
    total = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            ax_mu, ax_nu = 3 - mu, 3 - nu
            u_mu = U[..., mu, :, :]
            u_nu = U[..., nu, :, :]
            u_nu_xpmu = np.roll(u_nu, -1, axis=ax_mu)
            u_mu_xpnu = np.roll(u_mu, -1, axis=ax_nu)
            p = u_mu @ u_nu_xpmu @ _dagger(u_mu_xpnu) @ _dagger(u_nu)
            total += np.trace(p, axis1=-2, axis2=-1).real.mean() / 3.0
    return total / 6.0


def _traceless_hermitian(rng, shape):
    g = (rng.standard_normal(shape + (3, 3)) + 1j * rng.standard_normal(shape + (3, 3))) / np.sqrt(2.0)
    x = 0.5 * (g + _dagger(g))
    tr = np.trace(x, axis1=-2, axis2=-1)
    x = x - (tr / 3.0)[..., None, None] * np.eye(3)
    return x


def _expi(q, w, eps):
    """Q diag(exp(i eps w)) Q^dagger for a batch of eigen-decompositions."""
    ph = np.exp(1j * eps * w)
    return (q * ph[..., None, :]) @ _dagger(q)


def su3_links(dims, seed: int, target_plaquette: float = 0.59, tol: float = 1e-6,
              max_bisect: int = 60):
    """Random SU(3) links U = exp(i eps X), eps bisected for the mean plaquette.

    Returns ``(U, eps)`` with ``U`` complex128 of shape ``(Lt,Lz,Ly,Lx,4,3,3)``.
    ``X`` is traceless Hermitian, so ``det U = exp(i eps tr X) = 1``.
    """
    rng = np.random.default_rng(seed)
    shape = _shape(dims) + (4,)
    x = _traceless_hermitian(rng, shape)
    w, q = np.linalg.eigh(x)
    lo, hi = 0.0, 4.0
    # plaquette(eps) decreases from 1 as eps grows (for the range used here)
    while plaquette(_expi(q, w, hi)) > target_plaquette:
        hi *= 2.0
        if hi > 1e3:
            raise ValueError("cannot reach the target plaquette")
    eps = 0.5 * (lo + hi)
    for _ in range(max_bisect):
        eps = 0.5 * (lo + hi)
        p = plaquette(_expi(q, w, eps))
        if abs(p - target_plaquette) < tol:
            break
        if p > target_plaquette:
            lo = eps
        else:
            hi = eps
    return _expi(q, w, eps), eps


def unit_links(dims) -> np.ndarray:
    """Free field: every link is the 3x3 identity."""
    u = np.zeros(_shape(dims) + (4, 3, 3), dtype=np.complex128)
    u[..., :, :, :] = np.eye(3)
    return u


def gaussian_sources(dims, seed: int, n_rhs: int = 1) -> np.ndarray:
    """``n_rhs`` complex Gaussian vectors CN(0, 1), shape ``(n_rhs, 12V)``."""
    rng = np.random.default_rng(seed)
    n = 12 * volume(dims)
    re = rng.standard_normal((n_rhs, n))
    im = rng.standard_normal((n_rhs, n))
    return (re + 1j * im) / np.sqrt(2.0)


def point_sources(dims, site: int = 0) -> np.ndarray:
    """The 12 spin-colour point sources at one site, shape ``(12, 12V)``.

    Row ``3*spin + colour`` is the unit vector with a 1 at that component of
    ``site``.
    """
    n = 12 * volume(dims)
    b = np.zeros((12, n), dtype=np.complex128)
    for sc in range(12):
        b[sc, 12 * site + sc] = 1.0
    return b


def ones_source(dims) -> np.ndarray:
    """The test vector x = (1, ..., 1), shape ``(1, 12V)``."""
    return np.ones((1, 12 * volume(dims)), dtype=np.complex128)


def gauge_transform(dims, seed: int) -> np.ndarray:
    """Random SU(3) matrix per site (shape ``(Lt,Lz,Ly,Lx,3,3)``)."""
    rng = np.random.default_rng(seed)
    x = _traceless_hermitian(rng, _shape(dims))
    w, q = np.linalg.eigh(x)
    return _expi(q, w, 1.0)
