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
# the 64-instance sweep: seeds 1000 + i on 4^4, 6^4, 8^4, 10^4 in turn (16 each),
# the first 48 for training and the last 16 held out
C5_LATTICES = [(4, 4, 4, 4), (6, 6, 6, 6), (8, 8, 8, 8), (10, 10, 10, 10)]
C5_FIRST_SEED, C5_N, C5_TEST = 1000, 64, 16
C5_REPORT = os.path.join(HERE, "c5_evaluation.json")


def sample_instance(seed: int, dims=None):
    """One synthetic operator and source: lattice `dims` (default: drawn from
    DIMS_CHOICES), mu ~ U[0, 1], m_w ~ U[-2.2, -1.8], plaquette ~ U[0.55, 0.62],
    one Gaussian source."""
    import inputs   # seeded synthetic generators (not part of the compute path)
    rng = np.random.default_rng([4457, seed])
    drawn = DIMS_CHOICES[int(rng.integers(len(DIMS_CHOICES)))]
    dims = tuple(dims) if dims is not None else drawn
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


def c5_dims(seed: int):
    return C5_LATTICES[(seed - C5_FIRST_SEED) % len(C5_LATTICES)]


def build_dataset(n: int, tol: float = 1e-8, first_seed: int = 0, log=print, dims_of=None):
    """Features X (n', 16), targets Y (n', 2) = (log2 k*, log2 l*) and per-instance
    records, skipping instances without a label.  dims_of(seed): the lattice of
    an instance (default: drawn by sample_instance)."""
    import torch
    X, Y, recs = [], [], []
    for s in range(first_seed, first_seed + n):
        inst = sample_instance(s, dims_of(s) if dims_of else None)
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


def fit(X, Y, epochs: int = 2000, lr: float = 1e-3, seed: int = 0, val_frac: float = 0.25, chunk: int = 10,
        weight_decays=(0.0, 1e-2, 1e-1)):
    """(trained nksign.Mlp, validation-loss history, standardisation (xmu, xsd, ymu, ysd)).

    A 16 -> 64 -> 64 -> 2 network has far more parameters than there are
    labelled instances, so training is regularised and stops early: a seeded
    fraction val_frac of the samples is held out, Adam (with each decoupled
    weight decay of weight_decays) runs in chunks of `chunk` epochs on the
    rest, and the parameters with the lowest held-out loss are kept."""
    n = len(X)
    order = np.random.default_rng([7, seed]).permutation(n)
    n_val = int(round(val_frac * n)) if n >= 8 else 0
    val, fit_idx = order[:n_val], order[n_val:]
    Xf, Yf = X[fit_idx], Y[fit_idx]
    xsd = Xf.std(axis=0)
    xsd = np.where(xsd > 1e-6, xsd, 1.0)
    ysd = Yf.std(axis=0)
    ysd = np.where(ysd > 1e-6, ysd, 1.0)
    norm = (Xf.mean(axis=0), xsd, Yf.mean(axis=0), ysd)
    m = nksign.Mlp(seed)
    m.set_norm(*norm)
    if n_val == 0:
        return m, m.train(Xf, Yf, epochs, lr), norm
    w_init = m.get_params()
    best, w_best, hist_best = np.inf, w_init, None
    for wd in weight_decays:
        m.set_params(w_init)
        m.set_weight_decay(wd)
        hist = []
        for _ in range(max(1, epochs // chunk)):
            m.train(Xf, Yf, chunk, lr)
            L, _ = m.loss_grad(X[val], Y[val])
            hist.append(L)
            if L < best:
                best, w_best, hist_best = L, m.get_params(), hist
    m.set_params(w_best)
    m.set_weight_decay(0.0)
    return m, np.array(hist_best), norm


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
    coefficients); l is the predicted l times 1.5.  An under-predicted k costs further checks only; if the
    tolerance is still not met at k_max (l too small for it), the solve is
    repeated once with l = 256 from the default start.  Returns
    (stats, rc, (k_pred, l_pred)); stats["fallback"] says whether the
    repeat ran."""
    k_pred, l_pred = ctx.predict_sizes(m, b_dev, k_max)
    # l too small never passes the test, so it gets a margin of 1.5x (the
    # inner part costs O(k l), little against a repeated solve)
    l_use = min(L_LABEL, k_pred, 2 * int(np.ceil(0.75 * l_pred)))
    ctx.set_adapt_start(max(64, k_pred - 128))
    try:
        st, rc = ctx.sign_apply_dev(b_dev, y_dev, 1, k_max, l_use, tol=tol, flags=flags, check=False)
    finally:
        ctx.set_adapt_start(0)
    st["fallback"] = False
    if rc == nksign.NK_ENOTCONV and l_use < L_LABEL:
        ms = st["t_total_ms"]
        st, rc = ctx.sign_apply_dev(b_dev, y_dev, 1, k_max, L_LABEL, tol=tol, flags=flags, check=False)
        st["t_total_ms"] += ms
        st["fallback"] = True
    return st, rc, (k_pred, l_pred)


def evaluate(m, seeds, tol: float = 1e-8, l_default: int = 160, mean_sizes=None, log=print, dims_of=None):
    """Held-out comparison of three ways to run adaptive k on each instance:
      default    checks from NK_ADAPT_FIRST(l_default) on, l = l_default;
      mean       the training set's geometric-mean (k, l) used like a prediction
                 (checks from k - 128, l x 1.5);
      predicted  the predictor's (k, l) (solve_predicted).
    Accuracy is measured against a fixed-k solve 256 steps past the largest
    accepted k (l = 256).  Times are CUDA-event times of warm repeats."""
    import torch
    rows = []
    for s in seeds:
        inst = sample_instance(s, dims_of(s) if dims_of else None)
        ctx = _context(inst)
        b = torch.from_numpy(inst["b"]).cuda()
        ys = {name: torch.empty_like(b) for name in ("default", "mean", "predicted")}

        def run(name):
            if name == "default":
                st, rc = ctx.sign_apply_dev(b, ys[name], 1, K_MAX, l_default, tol=tol, check=False)
                return st, rc
            if name == "mean":
                km, lm = mean_sizes
                l_use = min(L_LABEL, km, 2 * int(np.ceil(0.75 * lm)))
                ctx.set_adapt_start(max(64, km - 128))
                try:
                    st, rc = ctx.sign_apply_dev(b, ys[name], 1, K_MAX, l_use, tol=tol, check=False)
                finally:
                    ctx.set_adapt_start(0)
                return st, rc
            st, rc, _ = solve_predicted(ctx, m, b, ys[name], tol)
            return st, rc

        names = ["default", "predicted"] + (["mean"] if mean_sizes else [])
        out = {name: run(name) for name in names}
        if any(rc != nksign.NK_OK for _, rc in out.values()):
            rows.append({"seed": s, "rc": {name: rc for name, (_, rc) in out.items()}})
            ctx.close()
            continue
        kref = min(K_MAX, max(st["k_used"] for st, _ in out.values()) + 256)
        ref = torch.empty_like(b)
        ctx.sign_apply_dev(b, ref, 1, kref, min(kref, L_LABEL))
        kp, lp = ctx.predict_sizes(m, b, K_MAX)
        row = {"seed": s, "dims": inst["dims"], "mu": round(inst["mu"], 3), "k_pred": kp, "l_pred": lp}
        for name in names:
            st, _ = run(name)          # warm repeat for the time
            row[name] = {"k": st["k_used"], "checks": st["checks"], "ms": round(st["t_total_ms"], 2),
                         "err": _rel(ys[name], ref)}
            if name == "predicted":
                row[name]["fallback"] = st["fallback"]
        rows.append(row)
        log(json.dumps(row))
        ctx.close()
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=192, help="instances (the last quarter is held out)")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--epochs", type=int, default=2000)
    ap.add_argument("--out", default=WEIGHTS_PATH)
    ap.add_argument("--dataset", default=None,
                    help="npz of features and labels: read if it exists, else written after labelling")
    ap.add_argument("--report", default=None, help="JSON summary path")
    ap.add_argument("--c5", action="store_true",
                    help="the 64-instance sweep (seeds 1000 + i, 4^4 / 6^4 / 8^4 / 10^4 in turn, 48 train / 16 "
                         "held out); writes its record to c5_evaluation.json and its weights beside it")
    a = ap.parse_args(argv)
    first, dims_of = 0, None
    if a.c5:
        a.n, first, dims_of = C5_N, C5_FIRST_SEED, c5_dims
        a.report = a.report or C5_REPORT
        if a.out == WEIGHTS_PATH:
            a.out = os.path.join(HERE, "predictor_weights_c5.npz")
    n_test = C5_TEST if a.c5 else a.n // 4
    test_seeds = list(range(first + a.n - n_test, first + a.n))
    t0 = time.time()
    if a.dataset and os.path.exists(a.dataset):
        z = np.load(a.dataset, allow_pickle=False)
        X, Y, Xt, Yt = z["X"], z["Y"], z["Xt"], z["Yt"]
        recs, recs_t = json.loads(str(z["recs"])), json.loads(str(z["recs_t"]))
    else:
        X, Y, recs = build_dataset(a.n - n_test, a.tol, first, dims_of=dims_of)
        Xt, Yt, recs_t = build_dataset(n_test, a.tol, first + a.n - n_test, dims_of=dims_of)
        if a.dataset:
            np.savez(a.dataset, X=X, Y=Y, Xt=Xt, Yt=Yt, recs=json.dumps(recs), recs_t=json.dumps(recs_t))
    t_data = time.time() - t0
    m, hist, norm = fit(X, Y, a.epochs)
    train_rmse = np.sqrt(np.mean((m.forward(X) - Y) ** 2, axis=0)).tolist()
    test_rmse = np.sqrt(np.mean((m.forward(Xt) - Yt) ** 2, axis=0)).tolist() if len(Xt) else None
    mean_rmse = np.sqrt(np.mean((Y.mean(axis=0) - Yt) ** 2, axis=0)).tolist() if len(Xt) else None
    km = 2 * int(round(0.5 * 2 ** Y[:, 0].mean()))
    lm = 2 * int(round(0.5 * 2 ** Y[:, 1].mean()))
    rows = evaluate(m, test_seeds, a.tol, mean_sizes=(km, lm), dims_of=dims_of)
    ok = [r for r in rows if "default" in r]
    tot = lambda name, key: float(np.sum([r[name][key] for r in ok]))
    summ = {
        "n_train": int(len(X)), "n_test": int(len(Xt)), "n_evaluated": len(ok), "tol": a.tol,
        "data_sec": round(t_data, 1), "val_loss_first_best": [float(hist[0]), float(np.min(hist))],
        "rmse_log2_train": train_rmse, "rmse_log2_test": test_rmse, "rmse_log2_test_of_mean": mean_rmse,
        "mean_sizes": [km, lm],
        "ms": {name: tot(name, "ms") for name in ("default", "mean", "predicted")},
        "checks": {name: int(tot(name, "checks")) for name in ("default", "mean", "predicted")},
        "max_err": {name: float(max([r[name]["err"] for r in ok], default=0.0))
                    for name in ("default", "mean", "predicted")},
        "fallbacks": int(sum(1 for r in ok if r["predicted"].get("fallback"))),
        "labels_train": [[r["seed"], r["k"], r["l"]] for r in recs],
        "labels_test": [[r["seed"], r["k"], r["l"]] for r in recs_t],
        "rows": rows,
    }
    save_model(a.out, m.get_params(), *norm,
               {k: summ[k] for k in ("n_train", "n_test", "tol", "rmse_log2_train", "rmse_log2_test")})
    print(json.dumps({k: v for k, v in summ.items() if k not in ("rows", "labels_train", "labels_test")}))
    if a.report:
        with open(a.report, "w") as fh:
            json.dump(summ, fh, indent=1)


if __name__ == "__main__":
    main()
