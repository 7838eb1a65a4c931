"""Seeded synthetic inputs: SU(3) links at a target plaquette, sources."""
import numpy as np
import pytest

import inputs


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 3, 4, 5)])
def test_links_are_su3_at_target_plaquette(dims):
    U, eps = inputs.su3_links(dims, seed=7)
    assert U.shape == (dims[3], dims[2], dims[1], dims[0], 4, 3, 3)
    uu = U @ np.conj(np.swapaxes(U, -1, -2))
    assert np.abs(uu - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1.0).max() < 1e-13
    assert abs(inputs.plaquette(U) - 0.59) < 1e-6
    assert 0.0 < eps < 2.0


def test_links_deterministic_per_seed():
    a, _ = inputs.su3_links((2, 2, 2, 4), seed=3)
    b, _ = inputs.su3_links((2, 2, 2, 4), seed=3)
    c, _ = inputs.su3_links((2, 2, 2, 4), seed=4)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def test_unit_links_plaquette_is_one():
    assert inputs.plaquette(inputs.unit_links((2, 3, 2, 4))) == pytest.approx(1.0, abs=1e-15)


def test_plaquette_brute_force_small():
    """Loop-by-loop plaquette on a 2x2x2x3 lattice equals the vectorised one."""
    dims = (2, 2, 2, 3)
    U, _ = inputs.su3_links(dims, seed=11)
    lx, ly, lz, lt = dims
    total, count = 0.0, 0
    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for x in range(lx):
                    c = [x, y, z, t]
                    for mu in range(4):
                        for nu in range(mu + 1, 4):
                            cm = list(c); cm[mu] = (cm[mu] + 1) % dims[mu]
                            cn = list(c); cn[nu] = (cn[nu] + 1) % dims[nu]
                            at = lambda q, d: U[q[3], q[2], q[1], q[0], d]
                            p = at(c, mu) @ at(cm, nu) @ at(cn, mu).conj().T @ at(c, nu).conj().T
                            total += np.trace(p).real / 3.0
                            count += 1
    assert total / count == pytest.approx(inputs.plaquette(U), abs=1e-14)


def test_sources():
    dims = (2, 2, 2, 2)
    b = inputs.point_sources(dims, site=3)
    assert b.shape == (12, 192)
    for sc in range(12):
        assert b[sc, 36 + sc] == 1.0 and np.count_nonzero(b[sc]) == 1
    g = inputs.gaussian_sources((4, 4, 4, 4), seed=1, n_rhs=2)
    assert g.shape == (2, 3072)
    assert abs(np.mean(np.abs(g) ** 2) - 1.0) < 0.05
    assert np.array_equal(g, inputs.gaussian_sources((4, 4, 4, 4), seed=1, n_rhs=2))


def test_gauge_transform_su3():
    om = inputs.gauge_transform((2, 2, 2, 2), seed=5)
    assert np.abs(om @ np.conj(np.swapaxes(om, -1, -2)) - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(om) - 1).max() < 1e-13
