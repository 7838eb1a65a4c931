"""GPU parity of the learned (k, l) predictor: the FP32 kernels through the
C ABI against the FP64 oracle (oracle/mlp.py, oracle/features.py).

Tolerances: FP32 forward and backward passes over 64-wide dot products
carry relative rounding of order 1e-6 per layer; the loss is checked to 1e-5
relative and the gradient to 1e-4 of its largest component.  Adam divides by
the root of the second moment, so parameters with near-zero gradient may
move differently; training is compared through the loss history and the
norm of the parameter change.  Features: FP32 storage of FP64 values
(relative 1e-6) of quantities that the outer recurrence determines to
1e-11, except the integer RHi count, which must match exactly.
"""
import numpy as np
import pytest

import inputs
from oracle import features as ofeat
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0912_4457_gb300 import nksign  # noqa: E402
from paper_0912_4457_gb300.nksign import NK_EINVAL, Context, Mlp, NkError  # noqa: E402


def _batch(seed, n):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n, 16)).astype(np.float32),
            rng.standard_normal((n, 2)).astype(np.float32))


@pytest.mark.parametrize("n", [1, 37, 256])
def test_loss_and_gradient_match_oracle(n):
    m = Mlp(seed=n)
    w = m.get_params().astype(np.float64)
    X, T = _batch(100 + n, n)
    L, g = m.loss_grad(X, T)
    L_or, g_or = omlp.loss_grad(w, X.astype(np.float64), T.astype(np.float64))
    assert abs(L - L_or) <= 1e-5 * abs(L_or)
    assert np.abs(g - g_or).max() <= 1e-4 * np.abs(g_or).max()


def test_forward_with_standardisation_matches_oracle():
    m = Mlp(seed=3)
    rng = np.random.default_rng(4)
    xmu, xsd = rng.standard_normal(16), 0.5 + rng.random(16)
    ymu, ysd = np.array([9.0, 6.5]), np.array([0.7, 0.9])
    m.set_norm(xmu, xsd, ymu, ysd)
    X = (rng.standard_normal((20, 16)) * xsd + xmu).astype(np.float32)
    y = m.forward(X)
    xs = omlp.standardise(X.astype(np.float64), xmu.astype(np.float32), xsd.astype(np.float32))
    z, _ = omlp.forward(m.get_params(), xs)
    y_or = z * ysd.astype(np.float32) + ymu.astype(np.float32)
    assert np.abs(y - y_or).max() <= 1e-5 * np.abs(y_or).max()


def test_set_params_round_trip_and_training_matches_oracle():
    m = Mlp(seed=5)
    w0 = np.random.default_rng(6).standard_normal(nksign.NK_MLP_PARAMS).astype(np.float32) * 0.2
    m.set_params(w0)
    np.testing.assert_array_equal(m.get_params(), w0)
    rng = np.random.default_rng(7)
    X = rng.standard_normal((48, 16)).astype(np.float32)
    T = np.stack([np.sin(X[:, 0]) + 0.5 * X[:, 1], 0.3 * X[:, 2] * X[:, 3]], axis=1).astype(np.float32)
    hist = m.train(X, T, epochs=40, lr=3e-3)
    w_or, hist_or = omlp.train(w0.astype(np.float64), X.astype(np.float64), T.astype(np.float64), 40, 3e-3)
    np.testing.assert_allclose(hist, hist_or, rtol=1e-3)
    w = m.get_params().astype(np.float64)
    assert np.linalg.norm(w - w_or) <= 1e-2 * np.linalg.norm(w_or - w0)
    assert hist[-1] < 0.7 * hist[0]


def test_weight_decay_matches_oracle():
    m = Mlp(seed=11)
    w0 = m.get_params()
    m.set_weight_decay(0.05)
    X, T = _batch(12, 32)
    hist = m.train(X, T, epochs=20, lr=3e-3)
    w_or, hist_or = omlp.train(w0.astype(np.float64), X.astype(np.float64), T.astype(np.float64), 20, 3e-3,
                               wd=0.05)
    np.testing.assert_allclose(hist, hist_or, rtol=1e-3)
    w = m.get_params().astype(np.float64)
    assert np.linalg.norm(w - w_or) <= 1e-2 * np.linalg.norm(w_or - w0)
    with pytest.raises(NkError):
        m.set_weight_decay(-1.0)


def test_training_is_deterministic():
    X, T = _batch(8, 64)
    out = []
    for _ in range(2):
        m = Mlp(seed=9)
        m.train(X, T, epochs=10, lr=1e-3)
        out.append(m.get_params())
    np.testing.assert_array_equal(out[0], out[1])


def test_mlp_invalid_arguments():
    m = Mlp(seed=1)
    X, T = _batch(1, 257)
    with pytest.raises(NkError) as e:
        m.loss_grad(X, T)
    assert e.value.code == NK_EINVAL
    with pytest.raises(NkError):
        m.train(X[:4], T[:4], epochs=0)
    with pytest.raises(NkError):
        m.set_norm(np.zeros(16), np.zeros(16), np.zeros(2), np.ones(2))


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_features_match_oracle(mu):
    dims = (4, 4, 4, 4)
    U, _ = inputs.su3_links(dims, seed=31)
    b = inputs.gaussian_sources(dims, seed=32)[0]
    ctx = Context(dims)
    ctx.load_links(U)
    ctx.set_mu_mw(mu, -1.9)
    f = ctx.features(torch.from_numpy(b).cuda())
    f_or = ofeat.features(U, dims, mu, -1.9, b)
    assert f[15] == f_or[15]
    for i in range(15):
        assert abs(f[i] - f_or[i]) <= 2e-6 * max(1.0, abs(f_or[i])) + 1e-9, (i, f[i], f_or[i])


def test_predict_sizes_rounds_and_clamps():
    """Zero weights make the output b3 (de-standardised): the sizes are 2^b3
    rounded to even and clamped to k in [64, k_max], l in [16, min(k, 256)]."""
    dims = (4, 4, 4, 4)
    ctx = Context(dims)
    ctx.load_links(inputs.su3_links(dims, seed=31)[0])
    ctx.set_mu_mw(0.3, -2.0)
    b = torch.from_numpy(inputs.gaussian_sources(dims, seed=33)[0]).cuda()
    m = Mlp(seed=0)
    w = np.zeros(nksign.NK_MLP_PARAMS, np.float32)
    cases = [((np.log2(300.2), np.log2(47.2)), 1536, (300, 48)),
             ((20.0, 20.0), 1024, (1024, 256)),
             ((0.0, 0.0), 1024, (64, 16)),
             ((np.log2(200.0), np.log2(250.0)), 1536, (200, 200))]
    for (lk, ll), kmax, want in cases:
        w[-2:] = [lk, ll]
        m.set_params(w)
        assert ctx.predict_sizes(m, b, kmax) == want
    with pytest.raises(NkError):
        ctx.predict_sizes(m, b, 63)
