"""Pins for the oracle's Wilson-Dirac operator (Sec. 2).

Each pin checks the oracle against something other than itself:
* the free-field closed form, derived in momentum space by hand;
* gauge covariance under the paper's link convention (catches a wrong link
  site, a missing dagger or a transposed colour index);
* gamma5-hermiticity at mu = 0 and the identity A^dagger = gamma5 D_w(-mu);
* the dense conjugate transpose (brute force) on a tiny lattice.
Lattices with four different extents catch axis mix-ups.
"""
import itertools

import numpy as np
import pytest

import inputs
from oracle import dirac

DIMS = (2, 3, 4, 6)   # Lx, Ly, Lz, Lt all different


def test_gamma_algebra():
    g, g5 = dirac.GAMMA, dirac.GAMMA5
    for a, b in itertools.product(range(4), range(4)):
        assert np.allclose(g[a] @ g[b] + g[b] @ g[a], 2.0 * (a == b) * np.eye(4), atol=1e-15)
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T)
        assert np.allclose(g5 @ g[a], -g[a] @ g5)
    # chiral basis: gamma5 = g1 g2 g3 g4 is diag(1, 1, -1, -1)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]), atol=1e-15)


def _free_field_dp(p, mu, m_w):
    """D(p) = 1 - 2 kappa sum cos(pt_nu) + 2 i kappa sum gamma_nu sin(pt_nu),
    pt_nu = p_nu for nu = 1..3 and pt_4 = p_4 + i mu.

    Derivation: with U = 1 and psi_y = e^{i p.y} u, the shift gives
    psi_{y -+ nu} = e^{-+ i p_nu} psi_y, so
    D(p) = 1 - kappa sum_nu [w+ (1 + g_nu) e^{-i p_nu} + w- (1 - g_nu) e^{i p_nu}],
    and e^{+-mu} e^{-+ i p_4} = e^{-+ i (p_4 + i mu)}.
    """
    kappa = 1.0 / (8.0 + 2.0 * m_w)
    d = np.eye(4, dtype=np.complex128)
    for nu in range(4):
        pt = p[nu] + (1j * mu if nu == 3 else 0.0)
        d = d - 2.0 * kappa * np.cos(pt) * np.eye(4) + 2j * kappa * np.sin(pt) * dirac.GAMMA[nu]
    return d


@pytest.mark.parametrize("mu,m_w", [(0.0, -2.0), (0.3, -2.0), (0.7, -1.5)])
def test_free_field_closed_form(mu, m_w):
    lx, ly, lz, lt = DIMS
    U = inputs.unit_links(DIMS)
    rng = np.random.default_rng(0)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    cols, expect = [], []
    for n in [(0, 0, 0, 0), (1, 2, 3, 5), (1, 1, 0, 2), (0, 2, 1, 3)]:
        # antiperiodic in t: p_4 = (2 n + 1) pi / Lt
        p = (2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz,
             (2 * n[3] + 1) * np.pi / lt)
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        cols.append((phase[..., None, None] * u).reshape(-1))
        expect.append((phase[..., None, None] * (_free_field_dp(p, mu, m_w) @ u)).reshape(-1))
    out = dirac.wilson_dirac(np.stack(cols, axis=1), U, DIMS, mu, m_w)
    assert np.abs(out - np.stack(expect, axis=1)).max() < 1e-13


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_gauge_covariance(mu):
    """U'_{x,nu} = Om_{x+nu} U_{x,nu} Om_x^dagger  =>  D'(Om psi) = Om (D psi).

    This is the transformation law of the paper's convention, in which the
    link U_{x,+nu} carries a quark from x to x + nu (Sec. 2).
    """
    U, _ = inputs.su3_links(DIMS, seed=21)
    om = inputs.gauge_transform(DIMS, seed=22)
    up = np.empty_like(U)
    for nu in range(4):
        om_fwd = np.roll(om, -1, axis=3 - nu)
        up[..., nu, :, :] = om_fwd @ U[..., nu, :, :] @ np.conj(np.swapaxes(om, -1, -2))
    psi = inputs.gaussian_sources(DIMS, seed=23)[0]
    field = psi.reshape(DIMS[3], DIMS[2], DIMS[1], DIMS[0], 4, 3)
    rot = np.einsum("tzyxab,tzyxsb->tzyxsa", om, field).reshape(-1)
    lhs = dirac.wilson_dirac(rot, up, DIMS, mu, -2.0)
    rhs = np.einsum("tzyxab,tzyxsb->tzyxsa", om,
                    dirac.wilson_dirac(psi, U, DIMS, mu, -2.0).reshape(field.shape)).reshape(-1)
    assert np.abs(lhs - rhs).max() < 1e-13
    # and the transformation is not trivial
    assert np.abs(dirac.wilson_dirac(rot, U, DIMS, mu, -2.0) - rhs).max() > 1e-3


def test_gamma5_hermiticity_mu0():
    U, _ = inputs.su3_links(DIMS, seed=31)
    u, v = inputs.gaussian_sources(DIMS, seed=32, n_rhs=2)
    lhs = np.vdot(u, dirac.apply_A(v, U, DIMS, 0.0, -2.0))
    rhs = np.vdot(dirac.apply_A(u, U, DIMS, 0.0, -2.0), v)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("mu", [0.0, 0.3, -0.5])
def test_adjoint_brute_force_and_mu_flip(mu):
    dims = (2, 2, 2, 4)
    U, _ = inputs.su3_links(dims, seed=41)
    a = dirac.dense_A(U, dims, mu, -2.0)
    n = a.shape[0]
    adag = dirac.apply_A_dagger(np.eye(n), U, dims, mu, -2.0)
    assert np.abs(adag - a.conj().T).max() < 1e-14
    # A^dagger = gamma5 D_w(-mu)
    flip = dirac.dense_A(U, dims, -mu, -2.0)
    assert np.abs(flip - a.conj().T).max() < 1e-14
    if mu != 0.0:
        assert np.abs(a - a.conj().T).max() > 1e-3


def test_dense_matches_explicit_hop_matrices():
    """Build D_w from the (y, x) blocks of T_nu^{+-} literally, site by site."""
    dims = (2, 2, 3, 2)
    mu, m_w = 0.4, -1.8
    U, _ = inputs.su3_links(dims, seed=51)
    lx, ly, lz, lt = dims
    V = lx * ly * lz * lt
    kappa = 1.0 / (8 + 2 * m_w)
    D = np.eye(12 * V, dtype=np.complex128)

    def idx(c):
        return c[0] + lx * (c[1] + ly * (c[2] + lz * c[3]))

    for c in itertools.product(range(lx), range(ly), range(lz), range(lt)):
        xs = idx(c)
        for nu in range(4):
            w_p = np.exp(mu) if nu == 3 else 1.0
            w_m = np.exp(-mu) if nu == 3 else 1.0
            # T^+: (y, x) block for y = x + nu, value (1 + g) U_{x,+nu}
            cp = list(c); cp[nu] += 1
            sign_p = -1.0 if (nu == 3 and cp[3] == lt) else 1.0
            cp[nu] %= dims[nu]
            yp = idx(cp)
            blk = np.kron(np.eye(4) + dirac.GAMMA[nu], U[c[3], c[2], c[1], c[0], nu])
            D[12 * yp:12 * yp + 12, 12 * xs:12 * xs + 12] -= kappa * w_p * sign_p * blk
            # T^-: (y, x) block for y = x - nu, value (1 - g) U_{x,-nu} = (1 - g) U^dagger_{x-nu,+nu}
            cm = list(c); cm[nu] -= 1
            sign_m = -1.0 if (nu == 3 and cm[3] < 0) else 1.0
            cm[nu] %= dims[nu]
            ym = idx(cm)
            blk = np.kron(np.eye(4) - dirac.GAMMA[nu], U[cm[3], cm[2], cm[1], cm[0], nu].conj().T)
            D[12 * ym:12 * ym + 12, 12 * xs:12 * xs + 12] -= kappa * w_m * sign_m * blk
    A = np.kron(np.eye(V), np.kron(dirac.GAMMA5, np.eye(3))) @ D
    assert np.abs(A - dirac.dense_A(U, dims, mu, m_w)).max() < 1e-14
