"""FP64 reference of the 16 predictor features of one source (the inputs of
the learned (k, l) predictor).

Test infrastructure only (see ``oracle/__init__.py``).  The features are the
library's choice, not the paper's; they are built from quantities the paper
defines:

  0 mu, 1 m_w, 2 log10 V,
  3 mean plaquette (1/3) Re tr U_mu(x)^+ U_nu(x+mu)^+ U_mu(x+nu) U_nu(x)
    over all sites and the six planes mu < nu.  In the hop convention of
    Sec. 2 the link U_{x,+nu} carries colour from x to x + nu and transforms
    as W(x+nu) U W(x)^+, so this is the closed loop that is gauge invariant
    (the textbook plaquette of the links U^+),
  then 32 steps of the outer recurrence (App. A for mu = 0, App. B otherwise)
  and the nested inner part on H_32 with l = 32 and p estimated (Eq. popt):
  4 log10 z_min, 5 log10 z_max, 6 their difference, 7 log10 p,
  8 mean Re H(j,j), 9 its standard deviation, 10 max |Im H(j,j)|,
  11 mean |H(j+1,j)|, 12 its standard deviation, 13 least-squares slope of
  ln |H(j+1,j)| against j, 14 log10(|c_24..31| / |c|) for c = V_l sgn(H_l) e_1
  (how much of the k = 32 answer sits in the last quarter of the basis),
  15 the number of Roberts-Higham iterations (Eq. Roberts).
"""
from __future__ import annotations

import numpy as np

from . import nested

K_FEAT = 32


def _dag(u):
    return np.conj(np.swapaxes(u, -1, -2))


def plaquette(U):
    """Mean plaquette of links U[t, z, y, x, nu, 3, 3] (direction nu = 0..3 is x, y, z, t)."""
    U = np.asarray(U)
    total = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            axis_mu, axis_nu = 3 - mu, 3 - nu        # array axis of direction mu, nu
            a = U[..., mu, :, :]
            b = np.roll(U[..., nu, :, :], -1, axis=axis_mu)   # U_nu(x + mu)
            c = np.roll(U[..., mu, :, :], -1, axis=axis_nu)   # U_mu(x + nu)
            d = U[..., nu, :, :]
            p = _dag(a) @ _dag(b) @ c @ d
            total += np.einsum("...ii->...", p).real.mean() / 3.0
    return total / 6.0


def spectral_features(alpha, beta, gamma, herm):
    """Features 4..15 from the K_FEAT = 32 step recurrence coefficients H_32
    (alpha = H(j,j), beta = H(j+1,j), gamma = H(j,j+1)): the p estimate of
    Eq. popt, the statistics of the diagonals and the nested inner part
    (App. C steps 3-5) on H_32 with l = 32."""
    k = K_FEAT
    p, z_min, z_max = nested.estimate_p(alpha, beta, gamma)
    c, info = nested.inner_sign(alpha, beta, gamma, K_FEAT, p, herm)
    if herm:
        re_a = np.asarray(alpha, dtype=np.float64)[:k]
        im_a = np.zeros(k)
    else:
        re_a = np.real(alpha[:k])
        im_a = np.imag(alpha[:k])
    sub = np.abs(np.asarray(beta)[: k - 1])
    j = np.arange(k - 1, dtype=np.float64)
    slope = np.polyfit(j, np.log(sub), 1)[0]
    cabs2 = np.abs(c) ** 2
    return np.array([
        np.log10(z_min), np.log10(z_max), np.log10(z_max) - np.log10(z_min), np.log10(p),
        re_a.mean(), re_a.std(), np.abs(im_a).max(),
        sub.mean(), sub.std(), slope,
        0.5 * np.log10(cabs2[24:].sum() / cabs2.sum()),
        float(info["rhi_iters"]),
    ])


def features_of_operator(apply_a, apply_adag, herm, b):
    """Features 4..15 of source b for an operator given as callables: 32 steps
    of the outer recurrence (App. A / B), then spectral_features."""
    outer = nested.outer_basis(apply_a, apply_adag, np.asarray(b, dtype=np.complex128), K_FEAT, herm)
    return spectral_features(outer.alpha, outer.beta, outer.gamma, herm)


def features(U, dims, mu, m_w, b, antiperiodic_t=True):
    """The 16 features (FP64) of source b; dims = (Lx, Ly, Lz, Lt)."""
    apply_a, apply_adag, herm = nested.operator(U, dims, mu, m_w, antiperiodic_t)
    head = np.array([mu, m_w, np.log10(np.prod(dims)), plaquette(U)])
    return np.concatenate([head, features_of_operator(apply_a, apply_adag, herm, b)])
