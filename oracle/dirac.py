"""Wilson-Dirac operator at chemical potential mu (Sec. 2 of the paper).

Test infrastructure only (see ``oracle/__init__.py``).

D_w(mu) = 1 - kappa sum_{i=1..3} (T_i^+ + T_i^-) - kappa (e^{mu} T_4^+ + e^{-mu} T_4^-)
with (T_nu^{+-})_{yx} = (1 +- gamma_nu) U_{x,+-nu} delta_{y, x +- nu},
U_{x,-nu} = U^dagger_{x-nu,+nu} and kappa = 1/(8 + 2 m_w)   (Sec. 2, eq. after Dovmu).

Written out per site y:
  (T_nu^+ psi)_y = (1 + gamma_nu) U_{y-nu,+nu} psi_{y-nu}
  (T_nu^- psi)_y = (1 - gamma_nu) U^dagger_{y,+nu} psi_{y+nu}

Readings where the paper is silent:
* gamma basis: chiral, gamma_k = [[0, -i s_k], [i s_k, 0]], gamma_4 = [[0, 1], [1, 0]],
  so gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1);
* boundary conditions: periodic in x, y, z, antiperiodic in t (a factor -1 on
  every hop that crosses the t boundary).

Array layout (shared with ``inputs``): spinors ``(Lt, Lz, Ly, Lx, 4, 3)``,
links ``(Lt, Lz, Ly, Lx, 4, 3, 3)``, direction nu = 0..3 (x, y, z, t) lives on
array axis ``3 - nu``.
"""
from __future__ import annotations

import numpy as np

_SIGMA = [
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def gamma_matrices():
    """Euclidean gamma_1..gamma_4 in the chiral basis, and gamma_5 = g1 g2 g3 g4."""
    g = [np.block([[_Z2, -1j * s], [1j * s, _Z2]]) for s in _SIGMA]
    g.append(np.block([[_Z2, _I2], [_I2, _Z2]]))
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


GAMMA, GAMMA5 = gamma_matrices()


def kappa_of(m_w: float) -> float:
    return 1.0 / (8.0 + 2.0 * m_w)


def _as_field(psi, dims):
    lx, ly, lz, lt = dims
    psi = np.asarray(psi, dtype=np.complex128)
    batch = psi.shape[1:] if psi.ndim > 1 else ()
    return psi.reshape((lt, lz, ly, lx, 4, 3) + batch), batch


def wilson_dirac(psi, U, dims, mu: float, m_w: float, antiperiodic_t: bool = True):
    """D_w(mu) psi for one vector (length 12V) or a block of vectors (12V, B)."""
    dims = tuple(int(d) for d in dims)
    field, batch = _as_field(psi, dims)
    kappa = kappa_of(m_w)
    extra = "".join(chr(ord("k") + i) for i in range(len(batch)))  # batch letters
    hop = np.zeros_like(field)
    for nu in range(4):
        ax = 3 - nu
        w_plus = np.exp(mu) if nu == 3 else 1.0
        w_minus = np.exp(-mu) if nu == 3 else 1.0
        u = U[..., nu, :, :]
        # backward neighbour: (1 + gamma_nu) U_{y-nu,+nu} psi_{y-nu}
        psi_m = np.roll(field, 1, axis=ax)
        u_m = np.roll(u, 1, axis=ax)
        if antiperiodic_t and nu == 3:
            psi_m[0] *= -1.0
        chi = np.einsum("tzyxab,tzyxsb" + extra + "->tzyxsa" + extra, u_m, psi_m)
        proj = np.eye(4) + GAMMA[nu]
        hop += w_plus * np.einsum("rs,tzyxsa" + extra + "->tzyxra" + extra, proj, chi)
        # forward neighbour: (1 - gamma_nu) U^dagger_{y,+nu} psi_{y+nu}
        psi_p = np.roll(field, -1, axis=ax)
        if antiperiodic_t and nu == 3:
            psi_p[-1] *= -1.0
        chi = np.einsum("tzyxba,tzyxsb" + extra + "->tzyxsa" + extra, np.conj(u), psi_p)
        proj = np.eye(4) - GAMMA[nu]
        hop += w_minus * np.einsum("rs,tzyxsa" + extra + "->tzyxra" + extra, proj, chi)
    out = field - kappa * hop
    return out.reshape(np.asarray(psi).shape)


def gamma5(psi, dims):
    """gamma_5 acting on the spin index of a vector (or block of vectors)."""
    field, batch = _as_field(psi, dims)
    extra = "".join(chr(ord("k") + i) for i in range(len(batch)))
    out = np.einsum("rs,tzyxsa" + extra + "->tzyxra" + extra, GAMMA5, field)
    return out.reshape(np.asarray(psi).shape)


def apply_A(psi, U, dims, mu: float, m_w: float, antiperiodic_t: bool = True):
    """A = gamma_5 D_w(mu), the argument of the sign function in Eq. Dovmu."""
    return gamma5(wilson_dirac(psi, U, dims, mu, m_w, antiperiodic_t), dims)


def apply_A_dagger(psi, U, dims, mu: float, m_w: float, antiperiodic_t: bool = True):
    """A^dagger psi = D_w(mu)^dagger (gamma_5 psi), from the adjoint of each hop.

    Taking the conjugate transpose of (T_nu^{+-})_{yx} of Sec. 2 (gamma_nu is
    Hermitian and commutes with the colour matrices; the weights e^{+-mu} are
    real and stay on their own term):
      ((T_nu^+)^dagger psi)_x = (1 + gamma_nu) U^dagger_{x,+nu} psi_{x+nu}
      ((T_nu^-)^dagger psi)_x = (1 - gamma_nu) U_{x-nu,+nu}    psi_{x-nu}
    This is the definition of the adjoint, not the identity
    A^dagger = gamma_5 D_w(-mu) that the GPU path relies on; the tests check
    that identity against this function.
    """
    dims = tuple(int(d) for d in dims)
    field, batch = _as_field(gamma5(psi, dims), dims)
    kappa = kappa_of(m_w)
    extra = "".join(chr(ord("k") + i) for i in range(len(batch)))
    hop = np.zeros_like(field)
    for nu in range(4):
        ax = 3 - nu
        w_plus = np.exp(mu) if nu == 3 else 1.0
        w_minus = np.exp(-mu) if nu == 3 else 1.0
        u = U[..., nu, :, :]
        # (T_nu^+)^dagger: (T^+)_{yx} nonzero for y = x + nu, so
        # ((T^+)^dagger psi)_x = (1 + gamma_nu) U^dagger_{x,+nu} psi_{x+nu}
        psi_p = np.roll(field, -1, axis=ax)
        if antiperiodic_t and nu == 3:
            psi_p[-1] *= -1.0
        chi = np.einsum("tzyxba,tzyxsb" + extra + "->tzyxsa" + extra, np.conj(u), psi_p)
        hop += w_plus * np.einsum("rs,tzyxsa" + extra + "->tzyxra" + extra, np.eye(4) + GAMMA[nu], chi)
        # (T_nu^-)^dagger: ((T^-)^dagger psi)_x = (1 - gamma_nu) U_{x-nu,+nu} psi_{x-nu}
        psi_m = np.roll(field, 1, axis=ax)
        u_m = np.roll(u, 1, axis=ax)
        if antiperiodic_t and nu == 3:
            psi_m[0] *= -1.0
        chi = np.einsum("tzyxab,tzyxsb" + extra + "->tzyxsa" + extra, u_m, psi_m)
        hop += w_minus * np.einsum("rs,tzyxsa" + extra + "->tzyxra" + extra, np.eye(4) - GAMMA[nu], chi)
    out = field - kappa * hop
    return out.reshape(np.asarray(psi).shape)


def dense_A(U, dims, mu: float, m_w: float, antiperiodic_t: bool = True):
    """The full 12V x 12V matrix of A = gamma_5 D_w(mu), column by column."""
    dims = tuple(int(d) for d in dims)
    n = 12 * int(np.prod(dims))
    eye = np.eye(n, dtype=np.complex128)
    return apply_A(eye, U, dims, mu, m_w, antiperiodic_t)
