"""Pins of the FP64 predictor oracle (oracle/mlp.py, oracle/features.py)
against facts other than itself: finite differences, closed forms at zero
weights and in the linear regime of tanh, the first Adam step, and the
plaquette of special gauge fields."""
import numpy as np
import pytest

import inputs
from oracle import features as ofeat
from oracle import mlp


def _params(seed, scale=0.3):
    return np.random.default_rng(seed).standard_normal(mlp.N_PARAMS) * scale


def _batch(seed, n):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, mlp.N_IN)), rng.standard_normal((n, mlp.N_OUT))


def test_parameter_count_matches_layer_sizes():
    assert mlp.N_PARAMS == 64 * 16 + 64 + 64 * 64 + 64 + 2 * 64 + 2
    w = _params(0)
    np.testing.assert_array_equal(mlp.pack(mlp.unpack(w)), w)


@pytest.mark.parametrize("n", [1, 5])
def test_gradient_matches_central_differences(n):
    w = _params(1)
    X, T = _batch(2, n)
    _, g = mlp.loss_grad(w, X, T)
    rng = np.random.default_rng(3)
    # every bias and a random sample of weights of each layer
    idx = np.unique(np.concatenate([rng.integers(0, mlp.N_PARAMS, 120),
                                    np.arange(1024, 1088), np.arange(5184, 5248), [5376, 5377]]))
    h = 1e-6
    for i in idx:
        e = np.zeros_like(w)
        e[i] = h
        fd = (mlp.loss(w + e, X, T) - mlp.loss(w - e, X, T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_zero_weights_closed_form():
    """With all weights and hidden biases zero the output is b3 for every
    input, L = mean |b3 - t|^2 / 2, dL/db3 = mean(b3 - t), and every other
    gradient vanishes (tanh(0) = 0 kills the W3 and deeper terms)."""
    P = {name: np.zeros(shp) for name, shp in mlp.SHAPES}
    P["b3"] = np.array([0.7, -1.2])
    w = mlp.pack(P)
    X, T = _batch(4, 9)
    L, g = mlp.loss_grad(w, X, T)
    assert L == pytest.approx(0.5 * np.mean(np.sum((P["b3"] - T) ** 2, axis=1)), rel=1e-14)
    G = mlp.unpack(g)
    np.testing.assert_allclose(G["b3"], (P["b3"] - T).mean(axis=0), rtol=1e-14)
    for name in ("W1", "b1", "W2", "b2", "W3"):
        assert np.all(G[name] == 0.0), name


def test_linear_regime_is_the_matrix_product():
    """For tiny first- and second-layer weights tanh is the identity to third
    order, so z = W3 W2 W1 x + W3 W2 b1 + W3 b2 + b3 up to O(scale^3); a
    transposed W1, W2 or W3 would break this."""
    rng = np.random.default_rng(5)
    s = 1e-4
    P = {"W1": rng.standard_normal((64, 16)) * s, "b1": rng.standard_normal(64) * s,
         "W2": rng.standard_normal((64, 64)) * s, "b2": rng.standard_normal(64) * s,
         "W3": rng.standard_normal((2, 64)), "b3": rng.standard_normal(2)}
    X = rng.standard_normal((7, 16))
    z, _ = mlp.forward(mlp.pack(P), X)
    lin = X @ (P["W3"] @ P["W2"] @ P["W1"]).T + P["W3"] @ (P["W2"] @ P["b1"] + P["b2"]) + P["b3"]
    np.testing.assert_allclose(z, lin, rtol=0, atol=1e-9)
    # and the output depends on x only through the product (a non-trivial value)
    assert np.abs(lin - P["b3"]).max() > 1e-8


def test_first_adam_step_is_a_signed_learning_rate_step():
    """From zero moments the bias-corrected moments are g and g^2, so the first
    step is -lr g / (|g| + eps)."""
    w = _params(6)
    g = np.random.default_rng(7).standard_normal(mlp.N_PARAMS)
    lr = 1e-2
    w1, m, v = mlp.adam_step(w, g, np.zeros_like(w), np.zeros_like(w), 1, lr)
    np.testing.assert_allclose(w1 - w, -lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)


def test_weight_decay_alone_shrinks_the_weights():
    """With zero gradient the moments stay zero and a step is w -> (1 - lr wd) w."""
    w = _params(10)
    z = np.zeros_like(w)
    w1, m, v = mlp.adam_step(w, z, z, z, 1, 1e-2, wd=0.1)
    np.testing.assert_allclose(w1, (1.0 - 1e-3) * w, rtol=1e-15)
    assert not m.any() and not v.any()


def test_training_fits_a_small_target():
    """Adam on a smooth target from 48 samples lowers the loss by a large factor."""
    rng = np.random.default_rng(8)
    X = rng.standard_normal((48, 16))
    T = np.stack([np.sin(X[:, 0]) + 0.5 * X[:, 1], X[:, 2] * X[:, 3] * 0.3], axis=1)
    w0 = _params(9, 0.2)
    _, hist = mlp.train(w0, X, T, 300, 1e-2)
    assert hist[-1] < 0.05 * hist[0]


def test_plaquette_of_unit_links_is_one():
    U = inputs.unit_links((2, 2, 2, 4))
    assert ofeat.plaquette(U) == pytest.approx(1.0, abs=1e-15)


def test_plaquette_is_gauge_invariant():
    """Invariant under U_nu(x) -> W(x+nu) U_nu(x) W(x)^+, the transformation
    under which the Wilson stencil of Sec. 2 is covariant."""
    dims = (4, 4, 2, 4)
    U, _ = inputs.su3_links(dims, seed=1, target_plaquette=0.59)
    om = inputs.gauge_transform(dims, seed=11)
    up = np.empty_like(U)
    for nu in range(4):
        om_fwd = np.roll(om, -1, axis=3 - nu)
        up[..., nu, :, :] = om_fwd @ U[..., nu, :, :] @ np.conj(np.swapaxes(om, -1, -2))
    P = ofeat.plaquette(U)
    assert ofeat.plaquette(up) == pytest.approx(P, abs=1e-13)
    assert np.abs(up - U).max() > 0.1
    # the generator's ensemble is symmetric under U -> U^+, so the value is
    # near its target (0.59 for the textbook loop of the stored links)
    assert abs(P - 0.59) < 0.02


def test_plaquette_of_an_abelian_constant_field():
    """U_x = diag(e^{i th}) on x links only, others 1: every plaquette in a
    plane containing x is U_x(x) U_x(x+nu)^+ = 1, so P = 1; with a
    position-dependent phase theta(y) on x links the (x, y) plaquette is
    e^{i (th(y) - th(y+1))} and P = (5 + mean cos(dth)) / 6."""
    dims = (2, 4, 2, 2)
    Lx, Ly, Lz, Lt = dims
    U = inputs.unit_links(dims).copy()
    th = np.array([0.0, 0.4, 1.1, 0.3])
    for y in range(Ly):
        U[:, :, y, :, 0] = np.exp(1j * th[y]) * np.eye(3)
    dth = th - np.roll(th, -1)
    assert ofeat.plaquette(U) == pytest.approx((5.0 + np.mean(np.cos(dth))) / 6.0, abs=1e-14)
