"""The learned (k, l) predictor in use: labels from runs of the method, a
predictor fitted to them, and the adaptive-k solve started from its
prediction, which must still meet the tolerance.

Accuracy is measured against a fixed-k all-FP64 solve 256 steps past the
accepted k (l = 256), whose own parity with the oracle is covered by the
converged-parity tests; the bar is 10 tol (the acceptance test bounds the
change of the coefficients, not the error itself).
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0912_4457_gb300 import nksign, predictor  # noqa: E402

TOL = 1e-8


def _ref(ctx, b, k):
    ref = torch.empty_like(b)
    kref = min(predictor.K_MAX, k + 256)
    ctx.sign_apply_dev(b, ref, 1, kref, min(kref, 256))
    return ref


def _small_instance(seed):
    inst = predictor.sample_instance(seed)
    while inst["dims"] not in [(4, 4, 4, 4), (4, 4, 4, 8)]:
        seed += 1000
        inst = predictor.sample_instance(seed)
    return inst


def test_label_and_fitted_prediction_meet_the_tolerance():
    inst = _small_instance(3)
    ctx = predictor._context(inst)
    b = torch.from_numpy(inst["b"]).cuda()
    k_star, l_star, info = predictor.label(ctx, b, TOL)
    assert k_star is not None, info
    assert k_star % 64 == 0 and 16 <= l_star <= min(k_star, 256)
    f = ctx.features(b)
    X = np.stack([f, f + 1e-3])
    Y = np.array([[np.log2(k_star), np.log2(l_star)]] * 2, np.float32)
    m, hist, _ = predictor.fit(X, Y, epochs=400, lr=1e-2)
    assert hist[-1] < 1e-2 * hist[0]
    kp, lp = ctx.predict_sizes(m, b, predictor.K_MAX)
    assert abs(kp - k_star) <= 8 and abs(lp - l_star) <= 4
    y = torch.empty_like(b)
    st, rc, _ = predictor.solve_predicted(ctx, m, b, y, TOL)
    assert rc == nksign.NK_OK
    assert st["checks"] <= 4
    err = predictor._rel(y, _ref(ctx, b, st["k_used"]))
    assert err <= 10 * TOL
    # an under-predicted k still converges: adaptive k carries on past it (with
    # the fallback l of solve_predicted: l_star is by definition the smallest l
    # that meets the tolerance at k_star, so checks at other k may sit just
    # above it)
    ctx.set_adapt_start(64)
    st2, rc2 = ctx.sign_apply_dev(b, y, 1, predictor.K_MAX, 256, tol=TOL, check=False)
    ctx.set_adapt_start(0)
    assert rc2 == nksign.NK_OK and st2["k_used"] >= k_star - 64
    assert predictor._rel(y, _ref(ctx, b, st2["k_used"])) <= 10 * TOL


@pytest.mark.skipif(not os.path.exists(predictor.WEIGHTS_PATH), reason="no trained predictor stored")
def test_stored_predictor_on_held_out_instance():
    m = predictor.load_model()
    inst = _small_instance(900)
    ctx = predictor._context(inst)
    b = torch.from_numpy(inst["b"]).cuda()
    y = torch.empty_like(b)
    st, rc, (kp, lp) = predictor.solve_predicted(ctx, m, b, y, TOL)
    assert rc == nksign.NK_OK
    assert 64 <= kp <= predictor.K_MAX and 16 <= lp <= min(kp, 256)
    assert predictor._rel(y, _ref(ctx, b, st["k_used"])) <= 10 * TOL
