"""Pins of the multi-level nested sign (oracle/nested.py, Sec. 4.5).

* One level is the single-level inner part (App. C steps 3-5) exactly.
* Several levels converge to sgn(H_k) e_1 of the outer Ritz matrix, taken here
  from scipy's matrix sign function (not from the oracle's RHi): Sec. 4.5
  reports that each nested level reproduces the level above once its size
  is inside its convergence region.
"""
import numpy as np
import pytest
import scipy.linalg

import inputs
from oracle import nested

M_W = -2.0


@pytest.fixture(scope="module", params=[0.0, 0.3])
def ritz(request):
    mu = request.param
    dims = (4, 4, 4, 4)
    U = inputs.su3_links(dims, 101)[0]
    A, Ad, herm = nested.operator(U, dims, mu, M_W)
    o = nested.outer_basis(A, Ad, inputs.gaussian_sources(dims, 201)[0], 256, herm)
    return mu, herm, o


def test_one_level_is_the_inner_sign(ritz):
    mu, herm, o = ritz
    p, _, _ = nested.estimate_p(o.alpha, o.beta, o.gamma)
    c1, _ = nested.inner_sign(o.alpha, o.beta, o.gamma, 64, p, herm)
    cm, info = nested.inner_sign_multilevel(o.alpha, o.beta, o.gamma, [64], p, herm)
    assert np.array_equal(c1, cm)
    assert info["p"] == [p]


@pytest.mark.parametrize("ells", [[96, 32], [96, 40, 16], [128, 48, 20, 10]])
def test_levels_converge_to_the_sign_of_h_k(ritz, ells):
    mu, herm, o = ritz
    H = o.H()
    truth = scipy.linalg.signm(H)[:, 0]
    p, _, _ = nested.estimate_p(o.alpha, o.beta, o.gamma)
    c, info = nested.inner_sign_multilevel(o.alpha, o.beta, o.gamma, ells, p, herm)
    assert info["rhi_converged"] and len(info["p"]) == len(ells)
    assert np.linalg.norm(c - truth) / np.linalg.norm(truth) < 1e-8


def test_nested_solve_with_levels_reaches_the_dense_sign():
    """sign_apply with further levels (ells) against the dense spectral sign
    of A on 2^4 (N = 192): k = 192 exhausts the space, so the levels are the
    only approximation left."""
    dims = (2, 2, 2, 2)
    U = inputs.su3_links(dims, 111)[0]
    x = inputs.gaussian_sources(dims, 211)[0]
    for mu in (0.0, 0.3):
        truth, _ = nested.sign_apply(U, dims, mu, M_W, x, method="dense")
        one, _ = nested.sign_apply(U, dims, mu, M_W, x, 192, 128)
        two, info = nested.sign_apply(U, dims, mu, M_W, x, 192, 128, ells=(64,))
        assert len(info["p_levels"]) == 2 and info["p_levels"][0] == info["p"]
        for y in (one, two):
            assert np.linalg.norm(y - truth) / np.linalg.norm(truth) < 1e-8
