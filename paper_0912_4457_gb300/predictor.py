"""Learned subspace sizes: training data, training and use of the (k, l)
predictor (the nk_mlp_* / nk_features / nk_predict_sizes entry points).

The paper sets the outer size k and the inner size l by hand for each
ensemble (Secs. 4.2-4.3).  Here a 16 -> 64 -> 64 -> 2 perceptron, trained on
runs of the method itself, predicts (log2 k, log2 l) for one operator and
source from features of the first 32 outer steps; the adaptive-k solve then
starts its convergence checks just below the predicted k and uses the
predicted l, and still runs on past k if the tolerance is not met there.

Labels of one instance (all-FP64 solves, one source):
  k*  the k at which adaptive k (checks every NK_ADAPT_STEP = 64 steps from
      k = 64 on, l = 256) accepts the result at tolerance tol;
  l*  the smallest l of L_GRID whose fixed-(k*, l) result agrees with the
      fixed-(k*, min(k*, 256)) result to tol (relative 2-norm), by bisection.

Every step of a solve runs in the library's kernels; this module only
samples instances, calls the C ABI through ``nksign`` and keeps the
bookkeeping.  Command line: ``python -m paper_0912_4457_gb300.predictor``
builds the data set, trains, evaluates on held-out instances and writes
``predictor_weights.npz`` (weights and standardisation) next to this file.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import nksign

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS_PATH = os.path.join(HERE, "predictor_weights.npz")

K_MAX = 1536
L_LABEL = 256
L_GRID = [16, 24, 32, 40, 48, 64, 80, 96, 128, 160, 192, 256]
DIMS_CHOICES = [(4, 4, 4, 4), (4, 4, 4, 8), (6, 6, 6, 6), (8, 8, 8, 8), (6, 6, 6, 12), (10, 10, 10, 10)]


def sample_instance(seed: int):
    """One synthetic operator and source: lattice from DIMS_CHOICES, mu ~ U[0, 1],
    m_w ~ U[-2.2, -1.8], plaquette ~ U[0.55, 0.62], one Gaussian source."""
    import inputs   # seeded synthetic generators (not part of the compute path)
    rng = np.random.default_rng([4457, seed])
    dims = DIMS_CHOICES[int(rng.integers(len(DIMS_CHOICES)))]
    mu = float(rng.uniform(0.0, 1.0))
    m_w = float(rng.uniform(-2.2, -1.8))
    plaq = float(rng.uniform(0.55, 0.62))
    U, _ = inputs.su3_links(dims, seed=10_000 + seed, target_plaquette=plaq)
    b = inputs.gaussian_sources(dims, seed=20_000 + seed)[0]
    return {"seed": seed, "dims": dims, "mu": mu, "m_w": m_w, "plaquette": plaq, "U": U, "b": b}


def _context(inst):
    ctx = nksign.Context(inst["dims"])
    ctx.load_links(inst["U"])
    ctx.set_mu_mw(inst["mu"], inst["m_w"])
    return ctx


def _rel(a, b):
    import torch
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def label(ctx, b_dev, tol: float):
    """(k*, l*, info) for one device source, or (None, None, info) if adaptive k
    does not meet tol by K_MAX or the recurrence breaks down."""
    import torch
    y = torch.empty_like(b_dev)
    ctx.set_adapt_start(64)
    try:
        st, rc = ctx.sign_apply_dev(b_dev, y, 1, K_MAX, L_LABEL, tol=tol, check=False)
    finally:
        ctx.set_adapt_start(0)
    info = {"rc": rc, "checks": st["checks"]}
    if rc != nksign.NK_OK:
        return None, None, info
    k_star = int(st["k_used"])
    ref = torch.empty_like(b_dev)
    ctx.sign_apply_dev(b_dev, ref, 1, k_star, min(k_star, L_LABEL))
    grid = [l for l in L_GRID if l <= k_star]
    lo, hi = 0, len(grid) - 1          # grid[hi] always passes (it is the reference)
    while lo < hi:
        mid = (lo + hi) // 2
        ctx.sign_apply_dev(b_dev, y, 1, k_star, grid[mid])
        if _rel(y, ref) <= tol:
            hi = mid
        else:
            lo = mid + 1
    return k_star, grid[lo], info


def build_dataset(n: int, tol: float = 1e-8, first_seed: int = 0, log=print):
    """Features X (n', 16), targets Y (n', 2) = (log2 k*, log2 l*) and per-instance
    records, skipping instances without a label."""
    import torch
    X, Y, recs = [], [], []
    for s in range(first_seed, first_seed + n):
        inst = sample_instance(s)
        ctx = _context(inst)
        b_dev = torch.from_numpy(inst["b"]).cuda()
        t0 = time.time()
        try:
            f = ctx.features(b_dev)
            k_star, l_star, info = label(ctx, b_dev, tol)
        except nksign.NkError as e:
            k_star, l_star, info, f = None, None, {"error": str(e)}, None
        rec = {k: inst[k] for k in ("seed", "dims", "mu", "m_w", "plaquette")}
        rec.update({"k": k_star, "l": l_star, "sec": round(time.time() - t0, 2), **info})
        recs.append(rec)
        log(json.dumps(rec))
        ctx.close()
        if k_star is None:
            continue
        X.append(f)
        Y.append([np.log2(k_star), np.log2(l_star)])
    return np.array(X, np.float32), np.array(Y, np.float32), recs


def fit(X, Y, epochs: int = 3000, lr: float = 3e-3, seed: int = 0):
    """(trained nksign.Mlp, loss history, standardisation (xmu, xsd, ymu, ysd))."""
    m = nksign.Mlp(seed)
    xsd = X.std(axis=0)
    xsd = np.where(xsd > 1e-6, xsd, 1.0)
    ysd = Y.std(axis=0)
    ysd = np.where(ysd > 1e-6, ysd, 1.0)
    norm = (X.mean(axis=0), xsd, Y.mean(axis=0), ysd)
    m.set_norm(*norm)
    hist = m.train(X, Y, epochs, lr)
    return m, hist, norm


def save_model(path, params, xmu, xsd, ymu, ysd, meta):
    np.savez(path, params=params, xmu=xmu, xsd=xsd, ymu=ymu, ysd=ysd, meta=json.dumps(meta))


def load_model(path: str = WEIGHTS_PATH):
    """The trained predictor stored by ``main`` as an nksign.Mlp."""
    z = np.load(path)
    m = nksign.Mlp(0)
    m.set_params(z["params"])
    m.set_norm(z["xmu"], z["xsd"], z["ymu"], z["ysd"])
    return m


def solve_predicted(ctx, m, b_dev, y_dev, tol: float, k_max: int = K_MAX, flags=nksign.NK_FP64):
    """Adaptive-k solve of one source with predicted sizes: l = l_pred and the
    checks start at k_pred - 2 * NK_ADAPT_STEP, so that an exact prediction is
    accepted at k_pred after three checks (the first only fills the previous
    coefficients).  Returns (stats, rc, (k_pred, l_pred))."""
    k_pred, l_pred = ctx.predict_sizes(m, b_dev, k_max)
    ctx.set_adapt_start(max(64, k_pred - 128))
    try:
        st, rc = ctx.sign_apply_dev(b_dev, y_dev, 1, k_max, l_pred, tol=tol, flags=flags, check=False)
    finally:
        ctx.set_adapt_start(0)
    return st, rc, (k_pred, l_pred)


def evaluate(m, seeds, tol: float = 1e-8, l_default: int = 160, log=print):
    """Held-out comparison: predicted sizes against adaptive k from its default
    start with l = l_default.  Accuracy of both is measured against a fixed-k
    solve at k_used + 256 (l = 256)."""
    import torch
    rows = []
    for s in seeds:
        inst = sample_instance(s)
        ctx = _context(inst)
        b = torch.from_numpy(inst["b"]).cuda()
        y0 = torch.empty_like(b)
        y1 = torch.empty_like(b)
        st0, rc0 = ctx.sign_apply_dev(b, y0, 1, K_MAX, l_default, tol=tol, check=False)
        st1, rc1, (kp, lp) = solve_predicted(ctx, m, b, y1, tol)
        if rc0 != nksign.NK_OK or rc1 != nksign.NK_OK:
            rows.append({"seed": s, "rc": [rc0, rc1]})
            ctx.close()
            continue
        kref = min(K_MAX, max(st0["k_used"], st1["k_used"]) + 256)
        ref = torch.empty_like(b)
        ctx.sign_apply_dev(b, ref, 1, kref, min(kref, L_LABEL))
        # warm timings: repeat each once more and keep the second
        st0, _ = ctx.sign_apply_dev(b, y0, 1, K_MAX, l_default, tol=tol, check=False)
        st1, _, _ = solve_predicted(ctx, m, b, y1, tol)
        row = {"seed": s, "dims": inst["dims"], "mu": round(inst["mu"], 3), "k_pred": kp, "l_pred": lp,
               "default": {"k": st0["k_used"], "checks": st0["checks"], "ms": round(st0["t_total_ms"], 2),
                           "err": _rel(y0, ref)},
               "predicted": {"k": st1["k_used"], "checks": st1["checks"], "ms": round(st1["t_total_ms"], 2),
                             "err": _rel(y1, ref)}}
        rows.append(row)
        log(json.dumps(row))
        ctx.close()
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=64, help="instances (the last quarter is held out)")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--out", default=WEIGHTS_PATH)
    ap.add_argument("--report", default=None, help="JSON summary path")
    a = ap.parse_args(argv)
    n_test = a.n // 4
    train_seeds = list(range(0, a.n - n_test))
    test_seeds = list(range(a.n - n_test, a.n))
    t0 = time.time()
    X, Y, recs = build_dataset(len(train_seeds), a.tol, 0)
    t_data = time.time() - t0
    m, hist, norm = fit(X, Y, a.epochs)
    pred = m.forward(X)
    train_rmse = np.sqrt(np.mean((pred - Y) ** 2, axis=0)).tolist()
    Xt, Yt, recs_t = build_dataset(n_test, a.tol, a.n - n_test)
    test_rmse = np.sqrt(np.mean((m.forward(Xt) - Yt) ** 2, axis=0)).tolist() if len(Xt) else None
    rows = evaluate(m, test_seeds, a.tol)
    ok = [r for r in rows if "default" in r]
    summ = {
        "n_train": int(len(X)), "n_test": int(len(Xt)), "tol": a.tol, "data_sec": round(t_data, 1),
        "loss_first_last": [float(hist[0]), float(hist[-1])],
        "rmse_log2_train": train_rmse, "rmse_log2_test": test_rmse,
        "default_ms": float(np.sum([r["default"]["ms"] for r in ok])),
        "predicted_ms": float(np.sum([r["predicted"]["ms"] for r in ok])),
        "default_checks": int(np.sum([r["default"]["checks"] for r in ok])),
        "predicted_checks": int(np.sum([r["predicted"]["checks"] for r in ok])),
        "max_err_default": float(max([r["default"]["err"] for r in ok], default=0.0)),
        "max_err_predicted": float(max([r["predicted"]["err"] for r in ok], default=0.0)),
        "labels_train": [[r["seed"], r["k"], r["l"]] for r in recs],
        "labels_test": [[r["seed"], r["k"], r["l"]] for r in recs_t],
        "rows": rows,
    }
    save_model(a.out, m.get_params(), *norm,
               {k: summ[k] for k in ("n_train", "n_test", "tol", "rmse_log2_train", "rmse_log2_test")})
    print(json.dumps({k: v for k, v in summ.items() if k != "rows"}))
    if a.report:
        with open(a.report, "w") as fh:
            json.dump(summ, fh, indent=1)


if __name__ == "__main__":
    main()
