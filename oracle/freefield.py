"""Exact sgn(A) b for the free field (all links 1) and for pure-gauge links,
in momentum space.

Test infrastructure only (see ``oracle/__init__.py``).  With U = 1 the
Wilson operator of Sec. 2 is diagonal in momentum: for the plane wave
psi_y = e^{i p.y} u,
    D(p) = 1 - 2 kappa sum_nu cos(pt_nu) + 2 i kappa sum_nu gamma_nu sin(pt_nu),
with pt_nu = p_nu for nu = 1..3 and pt_4 = p_4 + i mu (the weights e^{+-mu}
of the temporal hops), p_nu = 2 pi n / L_nu in space and, antiperiodic in t,
p_4 = (2 n + 1) pi / L_t.  A(p) = gamma5 D(p) is a 4 x 4 matrix (times the
colour identity) and sgn(A) acts on each momentum by sgn(A(p)), the
spectral definition (Eqs. fAdef, sgnz) applied to a 4 x 4 matrix.

Pure gauge links U_nu(x) = W(x + nu) W(x)^+ (W an SU(3) field) transform the
free operator to W A W^+ (the covariance of Sec. 2's hop convention), so
sgn(A_U) (W b) = W sgn(A_1) b: an exact answer for a link field that is not
trivial, at any lattice size.
"""
from __future__ import annotations

import numpy as np

from . import dirac, signfun


def momentum_sign_matrices(dims, mu, m_w, antiperiodic_t=True):
    """sgn(A(p)) for every momentum, shape (Lt, Lz, Ly, Lx, 4, 4) in FFT order
    (batched eigendecompositions: eigh for mu = 0, eig otherwise)."""
    lx, ly, lz, lt = dims
    kappa = dirac.kappa_of(m_w)
    pts = [2 * np.pi * np.fft.fftfreq(n, 1.0 / n) / n for n in (lt, lz, ly, lx)]
    if antiperiodic_t:
        pts[0] = pts[0] + np.pi / lt
    pt, pz, py, px = np.meshgrid(*pts, indexing="ij")
    d = np.zeros(pt.shape + (4, 4), dtype=np.complex128)
    d[..., :, :] = np.eye(4)
    for nu, p in enumerate((px, py, pz, pt + 1j * mu)):
        d = d - 2 * kappa * np.cos(p)[..., None, None] * np.eye(4) \
            + 2j * kappa * np.sin(p)[..., None, None] * dirac.GAMMA[nu]
    a = dirac.GAMMA5 @ d
    if mu == 0.0:
        w, v = np.linalg.eigh(a)
        return (v * np.sign(w)[..., None, :]) @ np.conj(np.swapaxes(v, -1, -2))
    w, v = np.linalg.eig(a)
    sv = v * signfun.sgn_scalar(w)[..., None, :]
    # sgn(A) = V sgn(L) V^{-1}:  X V = S V  ->  solve on the transposes
    return np.swapaxes(np.linalg.solve(np.swapaxes(v, -1, -2), np.swapaxes(sv, -1, -2)), -1, -2)


def free_sign_apply(b, dims, mu, m_w, antiperiodic_t=True, sgn_p=None):
    """sgn(A) b for U = 1; b of length 12 V (index 12 site + 3 spin + colour) or (n, 12 V)."""
    lx, ly, lz, lt = dims
    b = np.asarray(b, dtype=np.complex128)
    single = b.ndim == 1
    bs = b.reshape(-1, lt, lz, ly, lx, 4, 3)
    if sgn_p is None:
        sgn_p = momentum_sign_matrices(dims, mu, m_w, antiperiodic_t)
    t = np.arange(lt).reshape(lt, 1, 1, 1, 1, 1)
    twist = np.exp(-1j * np.pi * t / lt) if antiperiodic_t else np.ones_like(t, dtype=np.complex128)
    out = []
    for v in bs:
        f = np.fft.fftn(v * twist, axes=(0, 1, 2, 3))
        g = np.einsum("tzyxab,tzyxbc->tzyxac", sgn_p, f)
        out.append((np.fft.ifftn(g, axes=(0, 1, 2, 3)) / twist).reshape(-1))
    out = np.stack(out)
    return out[0] if single else out


def pure_gauge_links(W):
    """U_nu(x) = W(x + nu) W(x)^+ for W of shape (Lt, Lz, Ly, Lx, 3, 3)."""
    U = np.empty(W.shape[:4] + (4, 3, 3), dtype=np.complex128)
    Wd = np.conj(np.swapaxes(W, -1, -2))
    for nu in range(4):
        U[..., nu, :, :] = np.roll(W, -1, axis=3 - nu) @ Wd
    return U


def rotate(W, v, dims):
    """(W v)(x) = W(x) v(x) on the colour index, v of length 12 V or (n, 12 V)."""
    lx, ly, lz, lt = dims
    v = np.asarray(v, dtype=np.complex128)
    single = v.ndim == 1
    f = v.reshape(-1, lt, lz, ly, lx, 4, 3)
    r = np.einsum("tzyxab,ntzyxsb->ntzyxsa", W, f).reshape(f.shape[0], -1)
    return r[0] if single else r
