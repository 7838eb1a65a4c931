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


# held-out instances of the stored predictor (its training used seeds below 144)
HELD_OUT = [145, 152, 158, 163, 168, 176, 190]


@pytest.mark.skipif(not os.path.exists(predictor.WEIGHTS_PATH), reason="no trained predictor stored")
def test_prediction_saves_checks_and_time_on_held_out_instances():
    """What the predictor gains over the method without it: adaptive k started
    from the prediction against adaptive k from the default start (checks every
    NK_ADAPT_STEP from NK_ADAPT_FIRST(l), l = 160), both at tol = 1e-8 on the
    same held-out instances.  Summed over them the predicted start needs fewer
    convergence checks and less device time, and every result meets the
    tolerance against a converged reference."""
    m = predictor.load_model()
    tot = {"default": [0, 0.0], "predicted": [0, 0.0]}
    for seed in HELD_OUT:
        inst = predictor.sample_instance(seed)
        ctx = predictor._context(inst)
        b = torch.from_numpy(inst["b"]).cuda()
        y_d, y_p = torch.empty_like(b), torch.empty_like(b)
        for rep in range(2):          # the second run of each is timed (warm)
            st_d, rc_d = ctx.sign_apply_dev(b, y_d, 1, predictor.K_MAX, 160, tol=TOL, check=False)
            st_p, rc_p, _ = predictor.solve_predicted(ctx, m, b, y_p, TOL)
        assert rc_d == nksign.NK_OK and rc_p == nksign.NK_OK, seed
        ref = _ref(ctx, b, max(st_d["k_used"], st_p["k_used"]))
        assert predictor._rel(y_d, ref) <= 10 * TOL and predictor._rel(y_p, ref) <= 10 * TOL, seed
        tot["default"][0] += st_d["checks"]
        tot["default"][1] += st_d["t_total_ms"]
        tot["predicted"][0] += st_p["checks"]
        tot["predicted"][1] += st_p["t_total_ms"]
        ctx.close()
    assert tot["predicted"][0] < tot["default"][0], tot
    assert tot["predicted"][1] < tot["default"][1], tot


@pytest.mark.skipif(not os.path.exists(predictor.WEIGHTS_PATH), reason="no trained predictor stored")
def test_library_runs_the_predictor_itself():
    """NK_PREDICT: the library predicts (k, l) from source 0 with the predictor
    set on the context and starts its adaptive checks there (nk_stats reports
    the prediction); the result meets the tolerance."""
    m = predictor.load_model()
    inst = predictor.sample_instance(163)
    ctx = predictor._context(inst)
    b = torch.from_numpy(inst["b"]).cuda()
    kp, lp = ctx.predict_sizes(m, b, predictor.K_MAX)
    ctx.set_predictor(m)
    y = torch.empty_like(b)
    st, rc = ctx.sign_apply_dev(b, y, 1, predictor.K_MAX, 256, tol=TOL, flags=nksign.NK_PREDICT, check=False)
    assert rc == nksign.NK_OK
    assert (st["k_pred"], st["ell_pred"]) == (kp, lp)
    # the same procedure as predictor.solve_predicted: the same k, checks and result
    y_py = torch.empty_like(b)
    st_py, rc_py, _ = predictor.solve_predicted(ctx, m, b, y_py, TOL)
    assert rc_py == nksign.NK_OK
    assert (st["k_used"], st["checks"], st["ell_used"]) == (st_py["k_used"], st_py["checks"], st_py["ell_used"])
    assert torch.equal(y, y_py)
    assert predictor._rel(y, _ref(ctx, b, st["k_used"])) <= 10 * TOL
    # the error estimate of Sec. 3 inside the same call
    st2, rc2 = ctx.sign_apply_dev(b, y, 1, predictor.K_MAX, 256, tol=TOL,
                                  flags=nksign.NK_PREDICT | nksign.NK_EPS_EST, check=False)
    assert rc2 == nksign.NK_OK and 0.0 < st2["eps_sgn2"][0] <= 10 * TOL
    ctx.set_predictor(None)
    ctx.close()
