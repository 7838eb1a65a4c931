"""Krylov-Ritz approximations to sgn(A) x: non-nested and nested.

Test infrastructure only (see ``oracle/__init__.py``).

* Non-nested (Sec. 3, Eqs. non-nested / non-nested-oblique):
      y = |x| V_k sgn(H_k) e_1,
  sgn(H_k) by the Roberts-Higham iteration (Eq. Roberts) or the spectral form.
* Nested (Sec. 4, Eqs. innersign, precond, nested; App. C steps 2-6, without
  the deflation of steps 1 and 6, which the synthetic workloads do not use):
      2. (two-sided) Lanczos with A and x           -> V_k, H_k
      3. LU of p H_k (gttrf)
      4. (two-sided) Lanczos with H_k' and e_1^(k)   -> V_l, H_l
      5. RHi on H_l                                 -> sgn(H_l)
      6. y = |x| V_k V_l sgn(H_l) e_1^(l)
  Steps 3-5 are real in the Hermitian case.
* p: Eq. popt, p = (z_min z_max)^{-1/2}.  The paper takes z_min, z_max from
  spectral information of A (footnote to Eq. popt; p need only be
  approximate).  Reading used here and on the GPU:
  z_max from P_EST_ITERS = 30 steps of power iteration with H_k and z_min
  from 30 steps of inverse iteration with the LU of H_k, both from the
  normalised all-ones start vector; the estimate is |H x| (resp. 1/|H^{-1} x|)
  at the last step.  A smallest Ritz value whose Ritz pair has not converged
  (a spurious value in the spectral gap) is skipped: see estimate_p.
* Error estimate (Sec. 3): x~ = approx(approx(x)) and eps = |x~ - x| / (2 |x|).
* Overlap operator (Eq. Dovmu): D_ov x = x + gamma_5 sgn(gamma_5 D_w(mu)) x.
"""
from __future__ import annotations

import numpy as np

from . import dirac, krylov, signfun, tridiag

P_EST_ITERS = 30
P_RESID_TOL = 0.1


def estimate_p(alpha, beta, gamma, iters: int = P_EST_ITERS, resid_tol: float = P_RESID_TOL):
    """(p, z_min, z_max) from power / inverse iteration with H_k (Eq. popt).

    The smallest Ritz value found by inverse iteration is accepted only if
    its Ritz pair has converged: residual |H(k-1,k-2)| |x_{k-1}| (x the unit
    eigenvector estimate) at most resid_tol times the value.  Otherwise it is
    a spurious Ritz value inside the spectral gap (the near-zero Ritz values
    the Fig. 7 caption mentions), not spectral information of A, and the
    inverse iteration is repeated with that direction projected out.
    """
    lu = tridiag.PrecondLU(1.0, alpha, beta, gamma)
    k = len(lu.alpha)
    dt = lu.alpha.dtype
    x = np.ones(k, dtype=dt) / np.sqrt(k)
    z_max = 0.0
    for _ in range(iters):
        y = lu.band_mv(x)
        z_max = np.sqrt(np.vdot(y, y).real)
        x = y / z_max
    x = np.ones(k, dtype=dt) / np.sqrt(k)
    t = 1.0
    for _ in range(iters):
        y = lu.solve(x)
        t = np.sqrt(np.vdot(y, y).real)
        x = y / t
    z_min = 1.0 / t
    resid = abs(lu.beta[k - 2]) * abs(x[k - 1]) if k >= 2 else 0.0
    if resid > resid_tol * z_min:
        x1 = x
        x = np.ones(k, dtype=dt) / np.sqrt(k)
        x = x - np.vdot(x1, x) * x1
        x = x / np.sqrt(np.vdot(x, x).real)
        for _ in range(iters):
            y = lu.solve(x)
            y = y - np.vdot(x1, y) * x1
            t = np.sqrt(np.vdot(y, y).real)
            x = y / t
        z_min = 1.0 / t
    return 1.0 / np.sqrt(z_min * z_max), z_min, z_max


def shared_p(estimates):
    """One p for a batch of right-hand sides that share A (Eq. popt).

    The footnote to Eq. popt takes z_min and z_max from spectral information
    of A.  Each RHS's H_k gives estimates (z_min, z_max) (``estimate_p``);
    their extremes over the batch, min z_min and max z_max, are the batch's
    estimates of A's.  ``estimates`` is a sequence of (p, z_min, z_max); entries
    without a positive finite z_min and z_max are skipped.
    """
    zmn, zmx = None, 0.0
    for _, a, b in estimates:
        if a > 0.0 and b > 0.0 and np.isfinite(a) and np.isfinite(b):
            zmn = a if zmn is None else min(zmn, a)
            zmx = max(zmx, b)
    if zmn is None:
        return 1.0
    return 1.0 / np.sqrt(zmn * zmx)


def inner_sign(alpha, beta, gamma, ell: int, p: float, hermitian: bool):
    """App. C steps 3-5 and the inner half of step 6: c = V_l sgn(H_l) e_1 (a k-vector).

    Returns ``(c, info)`` where info has the inner Ritz matrix ``H_l``, the
    number of RHi iterations and whether RHi converged.
    """
    lu = tridiag.PrecondLU(p, alpha, beta, gamma)              # step 3
    k = len(lu.alpha)
    e1 = np.zeros(k, dtype=np.float64 if hermitian else np.complex128)
    e1[0] = 1.0
    if hermitian:                                              # step 4
        inner = krylov.lanczos(lu.apply_hprime, e1, ell)
    else:
        inner = krylov.two_sided_lanczos(
            lu.apply_hprime, lambda v: lu.apply_hprime(v, dagger=True), e1, ell)
    h_l = inner.H()
    s, it, conv = signfun.rhi(h_l)                             # step 5
    c = inner.V[:, : inner.k_used] @ s[:, 0]
    return c, {"H_l": h_l, "rhi_iters": it, "rhi_converged": conv,
               "inner_breakdown": inner.breakdown, "lu_singular": lu.singular,
               "inner": inner}


def inner_sign_multilevel(alpha, beta, gamma, ells, p: float, hermitian: bool):
    """Multi-level nesting (Sec. 4.5): c = V_{l_1} V_{l_2} ... V_{l_n} sgn(H_{l_n}) e_1.

    Level i (i = 1..n) applies App. C steps 3-4 to the Ritz matrix of the level
    above (H_k for i = 1): the LU of p_i H, the (two-sided) Lanczos recurrence
    with H' = (p_i H + (p_i H)^-1)/2 from e_1 for l_i steps -> V_{l_i}, H_{l_i}.
    RHi runs on the deepest Ritz matrix only (step 5), and the product is
    lifted back through every level.  p_1 = p (the caller's, as in
    inner_sign); deeper levels estimate their own p_i by Eq. popt from the
    Ritz matrix of the level above (the footnote of Sec. 4.5).  With one
    level this is inner_sign.

    Returns (c, info) with the per-level p values and the RHi count."""
    h_al, h_be, h_ga = alpha, beta, gamma
    bases, ps = [], []
    for i, ell in enumerate(ells):
        p_i = p if i == 0 else estimate_p(h_al, h_be, h_ga)[0]
        lu = tridiag.PrecondLU(p_i, h_al, h_be, h_ga)          # step 3 at this level
        k_i = len(lu.alpha)
        e1 = np.zeros(k_i, dtype=np.float64 if hermitian else np.complex128)
        e1[0] = 1.0
        if hermitian:                                          # step 4 at this level
            inner = krylov.lanczos(lu.apply_hprime, e1, ell)
        else:
            inner = krylov.two_sided_lanczos(
                lu.apply_hprime, lambda v, lu=lu: lu.apply_hprime(v, dagger=True), e1, ell)
        bases.append(inner.V[:, : inner.k_used])
        ps.append(p_i)
        m = inner.k_used
        h_al = inner.alpha[:m]
        h_be = inner.beta[: m - 1]
        h_ga = inner.gamma[: m - 1]
    h = np.diag(h_al).astype(np.result_type(h_al, h_be, h_ga))
    if len(h_al) > 1:
        h = h + np.diag(h_be, -1) + np.diag(h_ga, 1)
    s, it, conv = signfun.rhi(h)                               # step 5, deepest level
    c = s[:, 0]
    for V in reversed(bases):                                  # lift back level by level
        c = V @ c
    return c, {"p": ps, "rhi_iters": it, "rhi_converged": conv}


def operator(U, dims, mu: float, m_w: float, antiperiodic_t: bool = True):
    """(apply A, apply A^dagger, hermitian) for A = gamma_5 D_w(mu)."""
    def a(v):
        return dirac.apply_A(v, U, dims, mu, m_w, antiperiodic_t)

    def adag(v):
        return dirac.apply_A_dagger(v, U, dims, mu, m_w, antiperiodic_t)

    return a, adag, (mu == 0.0)


def outer_basis(apply_a, apply_adag, x, k: int, hermitian: bool):
    """App. C step 2: the outer (two-sided) Lanczos recurrence."""
    if hermitian:
        return krylov.lanczos(apply_a, x, k)
    return krylov.two_sided_lanczos(apply_a, apply_adag, x, k)


def nested_sign(apply_a, apply_adag, x, k: int, ell: int, hermitian: bool, p=None, ells=()):
    """Nested approximation to sgn(A) x (Eq. nested, App. C steps 2-6); with
    ells = (l_2, l_3, ...) the inner part nests further levels below l
    (Sec. 4.5, inner_sign_multilevel)."""
    outer = outer_basis(apply_a, apply_adag, x, k, hermitian)
    if outer.breakdown:
        raise FloatingPointError("two-sided Lanczos: serious breakdown at step %d" % outer.k_used)
    alpha, beta, gamma = outer.alpha, outer.beta, outer.gamma
    if p is None:
        p, z_min, z_max = estimate_p(alpha, beta, gamma)
    else:
        z_min = z_max = float("nan")
    if ells:
        c, info = inner_sign_multilevel(alpha, beta, gamma, (ell, *ells), p, hermitian)
        info["p_levels"] = info.pop("p")
    else:
        c, info = inner_sign(alpha, beta, gamma, ell, p, hermitian)
    y = outer.xnorm * (outer.V @ c)                            # step 6
    info.update(p=p, z_min=z_min, z_max=z_max, outer=outer, c=c)
    return y, info


def plain_sign(apply_a, apply_adag, x, k: int, hermitian: bool, method: str = "rhi"):
    """Non-nested Krylov-Ritz approximation y = |x| V_k sgn(H_k) e_1."""
    outer = outer_basis(apply_a, apply_adag, x, k, hermitian)
    if outer.breakdown:
        raise FloatingPointError("two-sided Lanczos: serious breakdown at step %d" % outer.k_used)
    h = outer.H()
    if method == "rhi":
        s, it, conv = signfun.rhi(h)
    else:
        s, it, conv = signfun.sign_spectral(h, hermitian), 0, True
    y = outer.xnorm * (outer.V @ s[:, 0])
    return y, {"rhi_iters": it, "rhi_converged": conv, "outer": outer}


def sign_apply(U, dims, mu, m_w, x, k=None, ell=None, p=None, method="nested",
               antiperiodic_t=True, ells=()):
    """sgn(gamma_5 D_w(mu)) x by the nested (optionally multi-level, ells),
    plain or dense method."""
    a, adag, herm = operator(U, dims, mu, m_w, antiperiodic_t)
    x = np.asarray(x, dtype=np.complex128)
    if method == "nested":
        return nested_sign(a, adag, x, k, ell, herm, p, ells)
    if method == "plain":
        return plain_sign(a, adag, x, k, herm)
    if method == "dense":
        m = dirac.dense_A(U, dims, mu, m_w, antiperiodic_t)
        s = signfun.sign_spectral(m, herm)
        return s @ x, {"sign": s}
    raise ValueError(method)


def sgn2_error(U, dims, mu, m_w, x, k, ell, p=None, antiperiodic_t=True):
    """eps = |sgn(A) sgn(A) x - x| / (2 |x|), both signs nested (Sec. 3)."""
    y, _ = sign_apply(U, dims, mu, m_w, x, k, ell, p, "nested", antiperiodic_t)
    z, _ = sign_apply(U, dims, mu, m_w, y, k, ell, p, "nested", antiperiodic_t)
    return np.linalg.norm(z - x) / (2.0 * np.linalg.norm(x))


def overlap_apply(U, dims, mu, m_w, x, k=None, ell=None, p=None, method="nested",
                  antiperiodic_t=True):
    """D_ov(mu) x = x + gamma_5 sgn(gamma_5 D_w(mu)) x (Eq. Dovmu)."""
    y, info = sign_apply(U, dims, mu, m_w, x, k, ell, p, method, antiperiodic_t)
    return np.asarray(x) + dirac.gamma5(y, dims), info
