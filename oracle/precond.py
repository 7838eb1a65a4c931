"""Closed forms for the preconditioning factor p and the improvement factor F.

Test infrastructure only (see ``oracle/__init__.py``).

* Hermitian case (Sec. 4.1, Eq. popt): p_opt = (z_min z_max)^{-1/2}; the largest
  transformed eigenvalue is z'_max = [sqrt(z_max/z_min) + sqrt(z_min/z_max)]/2
  and the condition number drops by F = (z_max/z_min) / z'_max  (Eq. condimp),
  approximately 2 sqrt(z_max/z_min).
* Non-Hermitian, spectrum in circles C(+-m, r) (Sec. 4.1): p_opt = (m^2 - r^2)^{-1/2};
  with m_s = p_opt m the image circles have centre m' = (m_s + 1/m_s)/2 and
  radius r' = (m_s - 1/m_s)/2; d = (m-r)/(m+r), d' = 1/m_s^2 and
  F = d'/d = ((m+r)/m)^2 = (2 - Delta/m)^2 with r = m - Delta  (Eq. condimpNH).
* Ellipse E(m, a, b): p_opt = (m^2 - a^2)^{-1/2}.
* The map itself: z -> z' = (p z + 1/(p z)) / 2  (Fig. precond / Eq. precond).
"""
from __future__ import annotations

import numpy as np


def transform(z, p):
    return 0.5 * (p * z + 1.0 / (p * z))


def p_opt(z_min, z_max):
    return 1.0 / np.sqrt(z_min * z_max)


def zprime_max(z_min, z_max):
    q = np.sqrt(z_max / z_min)
    return 0.5 * (q + 1.0 / q)


def improvement_hermitian(z_min, z_max):
    return (z_max / z_min) / zprime_max(z_min, z_max)


def circle_p_opt(m, r):
    return 1.0 / np.sqrt(m * m - r * r)


def circle_image(m, r):
    """(m', r') of the transformed circle for p = p_opt."""
    ms = circle_p_opt(m, r) * m
    return 0.5 * (ms + 1.0 / ms), 0.5 * (ms - 1.0 / ms)


def circle_improvement(m, r):
    """F = d'/d from the definitions d = (m-r)/(m+r), d' = (m'-r')/(m'+r')."""
    mp, rp = circle_image(m, r)
    d = (m - r) / (m + r)
    dp = (mp - rp) / (mp + rp)
    return dp / d


def circle_improvement_closed(m, r):
    """F = ((m + r)/m)^2, the closed form of Eq. condimpNH."""
    return ((m + r) / m) ** 2


def ellipse_p_opt(m, a):
    return 1.0 / np.sqrt(m * m - a * a)
