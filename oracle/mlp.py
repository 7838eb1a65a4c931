"""FP64 reference of the learned (k, l) predictor: a 16 -> 64 -> 64 -> 2
multilayer perceptron (tanh, tanh, linear), its mean-squared-error loss, the
loss gradient by back-propagation and one Adam step (Kingma & Ba 2015).

Test infrastructure only (see ``oracle/__init__.py``).  The paper picks its
subspace sizes by hand (Secs. 4.2-4.3); the predictor belongs to the library,
so this module follows the textbook definitions:

* forward: h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), z = W3 h2 + b3;
* loss over n samples with targets t: L = (1/n) sum_s |z_s - t_s|^2 / 2;
* Adam with bias correction and optional decoupled weight decay;
* inputs and targets are standardised first: x -> (x - xmu)/xsd,
  y -> (y - ymu)/ysd, and predictions are de-standardised;
* parameters flattened as W1[64][16], b1[64], W2[64][64], b2[64], W3[2][64],
  b3[2] (row = output unit).

Pinned by central finite differences of the loss, by closed forms at zero
weights and in the linear regime of tanh, and by the first Adam step
(tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 16, 64, 2
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_OUT, N_H)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = w[o:o + n].reshape(shp)
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def forward(w, X):
    """Outputs z (n, 2) and the activations (h1, h2) for standardised inputs X (n, 16)."""
    P = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ P["W1"].T + P["b1"])
    h2 = np.tanh(h1 @ P["W2"].T + P["b2"])
    z = h2 @ P["W3"].T + P["b3"]
    return z, (h1, h2)


def loss(w, X, T):
    z, _ = forward(w, X)
    return 0.5 * np.sum((z - np.asarray(T, dtype=np.float64)) ** 2) / len(X)


def loss_grad(w, X, T):
    """(L, dL/dw) by back-propagation through the three layers."""
    P = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    n = len(X)
    z, (h1, h2) = forward(w, X)
    L = 0.5 * np.sum((z - T) ** 2) / n
    dz = (z - T) / n                        # dL/dz
    dW3 = dz.T @ h2
    db3 = dz.sum(axis=0)
    da2 = (dz @ P["W3"]) * (1.0 - h2 ** 2)  # through tanh: d tanh(a)/da = 1 - tanh^2
    dW2 = da2.T @ h1
    db2 = da2.sum(axis=0)
    da1 = (da2 @ P["W2"]) * (1.0 - h1 ** 2)
    dW1 = da1.T @ X
    db1 = da1.sum(axis=0)
    return L, pack({"W1": dW1, "b1": db1, "W2": dW2, "b2": db2, "W3": dW3, "b3": db3})


def adam_step(w, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One Adam update at step t (1-based) with decoupled weight decay wd
    (Loshchilov & Hutter): returns (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return w - lr * (mh / (np.sqrt(vh) + eps) + wd * w), m, v


def standardise(X, mu, sd):
    return (np.asarray(X, dtype=np.float64) - mu) / sd


def train(w, X, T, epochs, lr, wd=0.0):
    """Full-batch Adam from zero moments; returns (w, loss before each step)."""
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    hist = []
    for t in range(1, epochs + 1):
        L, g = loss_grad(w, X, T)
        hist.append(L)
        w, m, v = adam_step(w, g, m, v, t, lr, wd=wd)
    return w, np.array(hist)
