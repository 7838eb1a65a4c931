"""Failure statuses of the CUDA path, driven by host inputs only.

* NK_EBREAKDOWN: the source is an exact eigenvector of A (free field with
  periodic t, m_w = -2, constant spin-0 colour-0 vector: A b = -b), so the
  first residual is exactly zero (App. A / B: v_2 = r / beta undefined).
* NK_ERHI: nk_inner_sign on a skew-symmetric tridiagonal, whose spectrum lies
  on the imaginary axis where sgn is undefined (Eq. sgnz); the oracle's RHi
  does not converge either (tests/test_oracle_failures.py).  A second RHS of
  the same batch keeps its own status and its oracle result.
"""
import numpy as np
import pytest

import inputs
from oracle import nested

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0912_4457_gb300 import nksign  # noqa: E402
from paper_0912_4457_gb300.nksign import (  # noqa: E402
    NK_EBREAKDOWN, NK_ERHI, NK_FP64, NK_MIXED, NK_NO_GRAPH, NK_OK, Context,
)

M_W = -2.0


@pytest.mark.parametrize("flags", [NK_FP64, NK_MIXED, NK_MIXED | NK_NO_GRAPH])
def test_eigenvector_source_reports_breakdown(flags):
    dims = (4, 4, 4, 4)
    ctx = Context(dims, bc_t_antiperiodic=False)
    ctx.load_links(inputs.unit_links(dims))
    ctx.set_mu_mw(0.0, M_W)
    b = np.zeros((1, 12 * 256), complex)
    b[0, 0::12] = 1.0
    y, st, rc = ctx.sign_apply(b, 64, 16, flags=flags, check=False)
    assert rc == NK_EBREAKDOWN
    assert st["status"][0] == NK_EBREAKDOWN
    assert "breakdown" in nksign.load_library().nk_last_error(ctx.h).decode()
    ctx.close()


def test_imaginary_spectrum_reports_rhi_failure_per_rhs():
    # RHS 0: skew-symmetric tridiagonal (imaginary spectrum); RHS 1: a Ritz
    # matrix of the two-sided recurrence on 4^4 (mu = 0.3)
    k, ell = 8, 8
    beta = np.array([0.5, 0.3, 2.0, 0.7, 1.3, 0.4, 1.1], dtype=complex)
    dims = (4, 4, 4, 4)
    U = inputs.su3_links(dims, 101)[0]
    A, Ad, herm = nested.operator(U, dims, 0.3, M_W)
    o = nested.outer_basis(A, Ad, inputs.gaussian_sources(dims, 201)[0], k, herm)
    al = np.stack([np.zeros(k, complex), o.alpha])
    be = np.stack([np.append(beta, 0), np.append(o.beta, 0)])
    ga = np.stack([np.append(-beta, 0), np.append(o.gamma, 0)])
    ctx = Context(dims)
    c, st, rc = ctx.inner_sign(al, be, ga, ell, p=0.0, hermitian=False, check=False)
    assert rc == NK_ERHI
    assert st["status"][0] == NK_ERHI and st["status"][1] == NK_OK
    p1, _, _ = nested.estimate_p(o.alpha, o.beta, o.gamma)
    c_or, info = nested.inner_sign(o.alpha, o.beta, o.gamma, ell, p1, False)
    assert info["rhi_converged"]
    assert np.linalg.norm(c[1] - c_or) / np.linalg.norm(c_or) < 1e-11
    ctx.close()
