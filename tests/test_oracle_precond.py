"""Pins for the preconditioning step (Sec. 4.1) and the tridiagonal LU (App. C).

* the paper's printed p_opt / F values (tests/golden/paper_precond_values.txt);
* the circle map C(m, r) -> C(m', r') for p = p_opt, checked point by point;
* sgn(H') = sgn(H) and eig(H') = (p z + 1/(p z))/2 (Eq. proofprec) on dense
  tridiagonals;
* the gttrf/gttrs-based application of H' and H'^dagger vs dense algebra;
* the power / inverse iteration estimates of z_max / z_min vs eigenvalues.
"""
import os

import numpy as np
import pytest

from oracle import nested, precond, signfun, tridiag

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_precond_values.txt")


def _golden():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, args, value, tol, cite = [f.strip() for f in line.split("|")]
        kw = dict(a.split("=") for a in args.split())
        rows[name] = ({k: float(v) for k, v in kw.items()}, float(value), float(tol), cite)
    return rows


def test_paper_printed_values():
    g = _golden()
    kw, val, tol, _ = g["p_opt_hermitian"]
    assert abs(precond.p_opt(kw["z_min"], kw["z_max"]) - val) <= tol
    kw, val, tol, _ = g["F_hermitian"]
    assert abs(precond.improvement_hermitian(kw["z_min"], kw["z_max"]) - val) <= tol
    # and F ~ 2 sqrt(z_max/z_min) (Eq. condimp)
    assert precond.improvement_hermitian(kw["z_min"], kw["z_max"]) == pytest.approx(
        2 * np.sqrt(kw["z_max"] / kw["z_min"]), rel=0.02)
    kw, val, tol, _ = g["p_opt_nonhermitian"]
    assert abs(precond.p_opt(kw["z_min"], kw["z_max"]) - val) <= tol
    kw, val, tol, _ = g["F_circle"]
    assert abs(precond.circle_improvement(kw["m"], kw["r"]) - val) <= tol
    assert abs(precond.circle_improvement_closed(kw["m"], kw["r"]) - val) <= tol


def test_optimal_p_balances_extremes():
    """At p_opt the images of z_min and z_max coincide (Eq. popt)."""
    zmin, zmax = 0.055, 5.26
    p = precond.p_opt(zmin, zmax)
    assert precond.transform(zmin, p) == pytest.approx(precond.transform(zmax, p), rel=1e-14)
    assert precond.transform(zmin, p) == pytest.approx(precond.zprime_max(zmin, zmax), rel=1e-14)


@pytest.mark.parametrize("m,r", [(2.55, 2.45), (1.0, 0.6), (3.0, 0.5)])
def test_circle_maps_to_circle(m, r):
    p = precond.circle_p_opt(m, r)
    mp, rp = precond.circle_image(m, r)
    th = np.linspace(0, 2 * np.pi, 257)
    z = m + r * np.exp(1j * th)
    zp = precond.transform(z, p)
    assert np.abs(np.abs(zp - mp) - rp).max() < 1e-12
    # d' = 1/m_s^2
    ms = p * m
    assert (mp - rp) / (mp + rp) == pytest.approx(1 / ms ** 2, rel=1e-12)


def _rand_tridiag(k, rng, complex_):
    a = rng.uniform(-3, 3, k)
    b = rng.uniform(0.2, 1.5, k - 1)
    if not complex_:
        return a, b, b.copy()
    a = a + 1j * rng.uniform(-0.3, 0.3, k)
    b = b * np.exp(1j * rng.uniform(-0.5, 0.5, k - 1))
    g = np.conj(b) ** 2 / b            # the two-sided Lanczos choice |gamma| = |beta|
    return a, b, g


def _dense(a, b, g):
    return np.diag(a) + np.diag(b, -1) + np.diag(g, 1)


@pytest.mark.parametrize("complex_", [False, True])
def test_sign_invariant_under_precond(complex_):
    rng = np.random.default_rng(3)
    a, b, g = _rand_tridiag(14, rng, complex_)
    h = _dense(a, b, g)
    for p in (0.5, 1.0, 1.7):
        hp = tridiag.hprime_dense(p, h)
        herm = not complex_
        assert np.abs(signfun.sign_spectral(hp, herm) - signfun.sign_spectral(h, herm)).max() < 1e-9
        zs = np.sort_complex(np.linalg.eigvals(h))
        zps = np.sort_complex(np.linalg.eigvals(hp))
        mapped = np.sort_complex(precond.transform(zs, p))
        assert np.abs(zps - mapped).max() < 1e-9


@pytest.mark.parametrize("complex_", [False, True])
def test_lu_apply_matches_dense(complex_):
    rng = np.random.default_rng(4)
    k = 33
    a, b, g = _rand_tridiag(k, rng, complex_)
    h = _dense(a, b, g)
    p = 1.3
    lu = tridiag.PrecondLU(p, a, b, g)
    assert lu.real == (not complex_)
    v = rng.standard_normal(k) + (1j * rng.standard_normal(k) if complex_ else 0)
    hp = tridiag.hprime_dense(p, h)
    assert np.abs(lu.solve(v) - np.linalg.solve(p * h, v)).max() < 1e-11
    assert np.abs(lu.band_mv(v) - p * h @ v).max() < 1e-12
    assert np.abs(lu.apply_hprime(v) - hp @ v).max() < 1e-11
    assert np.abs(lu.apply_hprime(v, dagger=True) - hp.conj().T @ v).max() < 1e-11


def test_lu_partial_pivoting_reconstructs():
    """Rebuild P L U from the gttrf factors and compare with p H."""
    rng = np.random.default_rng(5)
    k = 9
    a, b, g = _rand_tridiag(k, rng, True)
    a[2] = 1e-3                        # force a row interchange
    p = 0.8
    lu = tridiag.PrecondLU(p, a, b, g)
    dl, d, du, du2, ipiv = lu.factors
    U = np.diag(d) + np.diag(du, 1) + np.diag(du2, 2)
    # apply the L factors and interchanges in order: A = P_1 L_1 P_2 L_2 ... U
    m = U.astype(np.complex128)
    for i in reversed(range(k - 1)):
        li = np.eye(k, dtype=np.complex128)
        li[i + 1, i] = dl[i]
        m = li @ m
        if ipiv[i] - 1 != i:
            m[[i, i + 1]] = m[[i + 1, i]]
    assert np.abs(m - p * _dense(a, b, g)).max() < 1e-12
    assert any(ipiv[i] - 1 != i for i in range(k - 1))


def test_p_estimate_skips_spurious_gap_ritz_value():
    """Spectrum symmetric about 0 with a gap (-0.5, 0.5): a Ritz matrix of odd
    size has a spurious Ritz value near zero (Fig. 7 caption); it has not
    converged, so z_min must come from the converged edge of the gap instead.
    With even size there is no such value and z_min is the smallest |Ritz value|."""
    from oracle import krylov
    rng = np.random.default_rng(9)
    pos = np.sort(rng.uniform(0.5, 3.0, 200))
    w = np.concatenate([pos, -pos])
    x = rng.standard_normal(w.size)
    for k in (41, 40):
        res = krylov.lanczos(lambda v: w * v, x, k)
        ritz = np.sort(np.abs(np.linalg.eigvalsh(res.H())))
        p, zmin, zmax = nested.estimate_p(res.alpha, res.beta, res.gamma, iters=60)
        if k % 2:
            assert ritz[0] < 0.3                  # the spurious value exists
            assert zmin > 0.45                    # and is skipped
        else:
            assert ritz[0] > 0.45
            assert zmin == pytest.approx(ritz[0], rel=2e-2)
        assert zmax == pytest.approx(ritz[-1], rel=1e-2)


def test_spectral_estimates_hermitian():
    """Power / inverse iteration converge to max|z| and min|z| of H."""
    rng = np.random.default_rng(6)
    k = 30
    a, b, g = _rand_tridiag(k, rng, False)
    z = np.sort(np.abs(np.linalg.eigvalsh(_dense(a, b, g))))
    assert z[-2] / z[-1] < 0.95 and z[0] / z[1] < 0.95      # gaps for fast convergence
    # a random tridiagonal is not a Lanczos matrix: no residual screening here
    p, zmin, zmax = nested.estimate_p(a, b, g, iters=400, resid_tol=np.inf)
    assert zmax == pytest.approx(z[-1], rel=1e-10)
    assert zmin == pytest.approx(z[0], rel=1e-10)
    assert p == pytest.approx(precond.p_opt(z[0], z[-1]), rel=1e-10)


@pytest.mark.parametrize("hermitian", [True, False])
def test_shared_p_is_p_opt_of_the_batch_spectrum(hermitian):
    """Two sources that each excite part of the spectrum of A = diag(w): each
    H_k (k = the size of its part, so its Ritz values are exact) sees only
    its part, and the batch's p (Eq. popt with z_min, z_max of A, footnote)
    is p_opt(min |w|, max |w|) over the whole spectrum."""
    from oracle import krylov
    lam1 = np.array([0.4, -0.55, 0.8, -1.1, 1.5])
    lam2 = np.array([1.0, -1.7, 2.2, -2.6, 3.0])
    w = np.concatenate([lam1, lam2]).astype(np.complex128)
    if not hermitian:
        w = w * np.exp(0.15j * np.arange(w.size))     # |w| unchanged, off the real axis
    rng = np.random.default_rng(4)
    wt = rng.uniform(0.5, 1.5, w.size)
    est = []
    for part in (slice(0, 5), slice(5, 10)):
        x = np.zeros(w.size, np.complex128)
        x[part] = wt[part]
        if hermitian:
            res = krylov.lanczos(lambda v: w.real * v, x.real, 5)
        else:
            res = krylov.two_sided_lanczos(lambda v: w * v, lambda v: np.conj(w) * v, x, 5)
        # exact Ritz values: no screening of unconverged ones needed
        est.append(nested.estimate_p(res.alpha, res.beta, res.gamma, iters=400, resid_tol=np.inf))
    assert est[0][1] == pytest.approx(0.4, rel=1e-8) and est[0][2] == pytest.approx(1.5, rel=1e-8)
    assert est[1][1] == pytest.approx(1.0, rel=1e-8) and est[1][2] == pytest.approx(3.0, rel=1e-8)
    assert nested.shared_p(est) == pytest.approx(precond.p_opt(0.4, 3.0), rel=1e-8)
    # one RHS: its own estimate; entries without an estimate are skipped
    assert nested.shared_p(est[:1]) == pytest.approx(est[0][0], rel=1e-15)
    assert nested.shared_p([(1.0, 0.0, 0.0)] + est) == nested.shared_p(est)
