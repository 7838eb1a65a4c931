"""Lanczos (App. A) and two-sided Lanczos (App. B), step by step.

Test infrastructure only (see ``oracle/__init__.py``).

Both run k steps from the source x with v_1 = x/|x|, store the right basis
V_k = (v_1 .. v_k) column by column, and return the tridiagonal Ritz matrix
H_k as its three diagonals:

* ``alpha[j]`` = H(j, j), j = 0..k-1
* ``beta[j]``  = H(j+1, j), j = 0..k-2   (sub-diagonal)
* ``gamma[j]`` = H(j, j+1), j = 0..k-2   (super-diagonal)

Readings where the paper leaves a choice:
* Hermitian case: H(j,j) = v_j^dagger r is real in exact arithmetic; its real
  part is used both in H and in the update r <- r - H(j,j) v_j, in line with
  "steps 3-5 are done in real arithmetic" (App. C).  The imaginary part is
  returned as a diagnostic.
* Two-sided case: beta = sqrt(delta) on the principal branch (cut on the
  negative real axis, as in Eq. sgnz); gamma = conj(delta) / beta.
* Serious breakdown (App. B): delta == 0, or a non-finite delta, stops the
  recurrence with ``breakdown = True``.  In the Hermitian case (App. A) a zero
  (or non-finite) beta leaves v_{j+1} = r / beta undefined: the Krylov space
  is invariant, and the recurrence stops the same way.
* The inputs are the operator as callables, so the same code serves the outer
  recurrence on A (length 12V vectors) and the inner recurrence on H_k'
  (length-k vectors, real in the Hermitian case).
"""
from __future__ import annotations

import numpy as np


class LanczosResult:
    def __init__(self, V, alpha, beta, gamma, xnorm, k_used, breakdown=False,
                 alpha_imag=None, W=None):
        self.V = V
        self.alpha = alpha
        self.beta = beta
        self.gamma = gamma
        self.xnorm = xnorm
        self.k_used = k_used
        self.breakdown = breakdown
        self.alpha_imag = alpha_imag
        self.W = W

    def H(self):
        """Dense k x k tridiagonal Ritz matrix."""
        k = self.k_used
        h = np.zeros((k, k), dtype=np.result_type(self.alpha, self.beta, self.gamma))
        h[np.arange(k), np.arange(k)] = self.alpha[:k]
        if k > 1:
            h[np.arange(1, k), np.arange(k - 1)] = self.beta[: k - 1]
            h[np.arange(k - 1), np.arange(1, k)] = self.gamma[: k - 1]
        return h


def lanczos(apply_a, x, k: int, store_basis: bool = True) -> LanczosResult:
    """Hermitian Lanczos, App. A: k applications of A, three-term recurrence."""
    x = np.asarray(x)
    n = x.shape[0]
    xnorm = float(np.sqrt(np.vdot(x, x).real))
    V = np.zeros((n, k), dtype=x.dtype) if store_basis else None
    alpha = np.zeros(k)
    alpha_imag = np.zeros(k)
    beta = np.zeros(max(k - 1, 0))
    v_prev = None
    v = x / xnorm
    if store_basis:
        V[:, 0] = v
    r = apply_a(v)
    for j in range(k):
        a = np.vdot(v, r)                      # H(j,j) <- v_j^dagger r
        alpha[j] = a.real
        alpha_imag[j] = np.imag(a)
        r = r - alpha[j] * v                   # r <- r - H(j,j) v_j
        if j == k - 1:
            break
        b = np.sqrt(np.vdot(r, r).real)        # beta <- sqrt(r^dagger r)
        if b == 0 or not np.isfinite(b):
            return LanczosResult(V, alpha, beta, beta.copy(), xnorm, j + 1, True, alpha_imag)
        beta[j] = b
        v_prev, v = v, r / b                   # v_{j+1} <- r / beta
        if store_basis:
            V[:, j + 1] = v
        r = apply_a(v)                         # r <- A v_{j+1}
        r = r - b * v_prev                     # r <- r - beta v_j
    return LanczosResult(V, alpha, beta, beta.copy(), xnorm, k, False, alpha_imag)


def two_sided_lanczos(apply_a, apply_adag, x, k: int, store_basis: bool = True,
                      store_left: bool = False) -> LanczosResult:
    """Two-sided Lanczos, App. B: bases V_k, W_k with w_j^dagger v_i = delta_ij."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[0]
    xnorm = float(np.sqrt(np.vdot(x, x).real))
    V = np.zeros((n, k), dtype=np.complex128) if store_basis else None
    W = np.zeros((n, k), dtype=np.complex128) if store_left else None
    alpha = np.zeros(k, dtype=np.complex128)
    beta = np.zeros(max(k - 1, 0), dtype=np.complex128)
    gamma = np.zeros(max(k - 1, 0), dtype=np.complex128)
    v = x / xnorm
    w = v.copy()
    if store_basis:
        V[:, 0] = v
    if store_left:
        W[:, 0] = w
    r = apply_a(v)
    l = apply_adag(w)
    for j in range(k):
        a = np.vdot(w, r)                      # H(j,j) <- w_j^dagger r
        alpha[j] = a
        r = r - a * v                          # r <- r - H(j,j) v_j
        l = l - np.conj(a) * w                 # l <- l - H(j,j)^* w_j
        if j == k - 1:
            break
        delta = np.vdot(r, l)                  # delta <- r^dagger l
        if delta == 0 or not np.isfinite(delta):
            return LanczosResult(V, alpha, beta, gamma, xnorm, j + 1, True, None, W)
        b = np.sqrt(delta)                     # beta <- sqrt(delta), principal branch
        g = np.conj(delta) / b                 # gamma <- delta^* / beta
        beta[j] = b
        gamma[j] = g
        v_prev, w_prev = v, w
        v = r / b                              # v_{j+1} <- r / beta
        w = l / np.conj(g)                     # w_{j+1} <- l / gamma^*
        if store_basis:
            V[:, j + 1] = v
        if store_left:
            W[:, j + 1] = w
        r = apply_a(v)                         # r <- A v_{j+1}
        l = apply_adag(w)                      # l <- A^dagger w_{j+1}
        r = r - g * v_prev                     # r <- r - gamma v_j
        l = l - np.conj(b) * w_prev            # l <- l - beta^* w_j
    return LanczosResult(V, alpha, beta, gamma, xnorm, k, False, None, W)
