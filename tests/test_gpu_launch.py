"""Launch shapes of the outer recurrence and the autotuner.

Every shape computes the same method; shapes differ only in the order of
the floating-point sums, so each must meet the same bars as the default:
<= 1e-10 against the FP64 oracle at a converged k and <= 1e-8 for the mixed
schedule against the dense truth; and one shape is bitwise reproducible.
"""
import os

import numpy as np
import pytest

import inputs
from oracle import nested

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0912_4457_gb300.nksign import NK_EINVAL, NK_FP64, NK_MIXED, Context, NkError  # noqa: E402

DIMS = (4, 4, 4, 4)
KL = {0.0: (384, 96), 0.3: (512, 128)}   # converged sizes on this lattice
M_W = -2.0


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def case():
    U = inputs.su3_links(DIMS, seed=101)[0]
    b = inputs.gaussian_sources(DIMS, seed=302, n_rhs=3)
    y_or = {mu: nested.sign_apply(U, DIMS, mu, M_W, b[0], *KL[mu])[0] for mu in (0.0, 0.3)}
    return U, b, y_or


def ctx_for(U, mu):
    ctx = Context(DIMS)
    ctx.load_links(U)
    ctx.set_mu_mw(mu, M_W)
    return ctx


# (stencil threads, order, step-2 blocks, early threads, early order, split, early split)
SHAPES = [(64, 1, 1, 256, 1, 1, 3), (256, 0, 7, 64, 0, 3, 1), (128, 1, 40, 128, 1, 3, 3), (64, 0, 3, 64, 1, 1, 1)]


@pytest.mark.parametrize("mu", [0.0, 0.3])
@pytest.mark.parametrize("shape", SHAPES)
def test_every_shape_matches_oracle(case, mu, shape):
    U, b, y_or = case
    ctx = ctx_for(U, mu)
    ctx.set_launch(3, NK_FP64, *shape)
    assert ctx.get_launch(3, NK_FP64) == shape
    y, st, _ = ctx.sign_apply(b, *KL[mu], flags=NK_FP64)
    assert rel(y[0], y_or[mu]) <= 1e-10
    y2, _, _ = ctx.sign_apply(b, *KL[mu], flags=NK_FP64)
    np.testing.assert_array_equal(y, y2)
    ctx.close()


@pytest.mark.parametrize("shape", SHAPES[:2])
def test_mixed_schedule_under_other_shapes(case, shape):
    U, b, y_or = case
    ctx = ctx_for(U, 0.3)
    ctx.set_launch(3, NK_MIXED, *shape)
    y, _, _ = ctx.sign_apply(b, 512, 128, flags=NK_MIXED)
    assert rel(y[0], y_or[0.3]) <= 1e-8
    ctx.close()


def test_autotune_and_cache(case, tmp_path):
    U, b, y_or = case
    path = str(tmp_path / "tune.txt")
    ctx = ctx_for(U, 0.3)
    default = ctx.get_launch(3, NK_MIXED)
    assert default[:2] == (128, 0) and default[3:] == (128, 0, 1, 1)
    shape, ms = ctx.autotune(3, NK_MIXED, path)
    assert shape[0] in (64, 128, 256) and shape[1] in (0, 1) and shape[2] >= 1
    assert shape[3] in (64, 128, 256) and shape[4] in (0, 1) and shape[5] in (1, 3) and shape[6] in (1, 3)
    assert 0.0 < ms < 10.0
    assert ctx.get_launch(3, NK_MIXED) == shape
    lines = open(path).read().split("\n")
    assert lines[0].split()[:8] == ["nk_launch", "4", "4", "4", "4", "3", "1", "1"]
    # a second context reads the cache instead of timing
    ctx2 = ctx_for(U, 0.3)
    shape2, ms2 = ctx2.autotune(3, NK_MIXED, path)
    assert shape2 == shape and abs(ms2 - ms) <= 1e-6 * ms
    assert open(path).read().count("nk_launch") == 1
    # the tuned shape is used by the next solve, with the same accuracy
    y, _, _ = ctx.sign_apply(b, 512, 128, flags=NK_MIXED)
    assert rel(y[0], y_or[0.3]) <= 1e-8
    # the FP64 shape of the same context is separate and still the default
    assert ctx.get_launch(3, NK_FP64)[:2] == (128, 0)
    ctx.close()
    ctx2.close()


def test_invalid_shapes(case):
    U, _, _ = case
    ctx = ctx_for(U, 0.0)
    for bad in [(96, 0, 4), (128, 2, 4), (128, 0, 0), (128, 0, 5000), (128, 0, 4, 32, 0), (128, 0, 4, 64, 3),
                (128, 0, 4, 64, 0, 2, 1), (128, 0, 4, 64, 0, 1, 4)]:
        with pytest.raises(NkError) as e:
            ctx.set_launch(1, NK_FP64, *bad)
        assert e.value.code == NK_EINVAL
    with pytest.raises(NkError):
        ctx.set_launch(13, NK_FP64, 128, 0, 4)
    ctx.close()
