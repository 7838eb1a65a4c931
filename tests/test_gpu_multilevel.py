"""Multi-level nesting (Sec. 4.5) on the GPU against the oracle.

* nk_inner_sign with levels below the first against the oracle's
  inner_sign_multilevel on the same H_k (same p for the first level; deeper
  levels estimate theirs on both sides).
* A whole solve with three levels against the single-level solve and the
  oracle: the deeper levels sit inside their convergence region, so the
  result agrees with one level to the method's error level.
"""
import numpy as np
import pytest

import inputs
from oracle import nested

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0912_4457_gb300.nksign import NK_FP64, NK_MIXED, Context  # noqa: E402

M_W = -2.0
DIMS = (4, 4, 4, 4)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_inner_sign_multilevel_matches_oracle(mu):
    U = inputs.su3_links(DIMS, 101)[0]
    A, Ad, herm = nested.operator(U, DIMS, mu, M_W)
    o = nested.outer_basis(A, Ad, inputs.gaussian_sources(DIMS, 201)[0], 256, herm)
    p, _, _ = nested.estimate_p(o.alpha, o.beta, o.gamma)
    ells = [96, 32, 16]
    c_or, info = nested.inner_sign_multilevel(o.alpha, o.beta, o.gamma, ells, p, herm)
    ctx = Context(DIMS)
    ctx.set_nesting(ells[1:])
    c, st, rc = ctx.inner_sign(o.alpha, o.beta, o.gamma, ells[0], p=0.0, hermitian=herm)
    assert rc == 0
    assert st["p"][0] == pytest.approx(p, rel=1e-12)
    assert rel(c[0], c_or) < 1e-10
    assert abs(st["rhi_iters"][0] - info["rhi_iters"]) <= 1
    ctx.set_nesting(())
    c1, _, _ = ctx.inner_sign(o.alpha, o.beta, o.gamma, ells[0], p=0.0, hermitian=herm)
    c1_or, _ = nested.inner_sign(o.alpha, o.beta, o.gamma, ells[0], p, herm)
    assert rel(c1[0], c1_or) < 1e-11
    ctx.close()


@pytest.mark.parametrize("mu,k,flags", [(0.0, 384, NK_FP64), (0.3, 512, NK_FP64), (0.3, 512, NK_MIXED)])
def test_multilevel_solve_matches_single_level(mu, k, flags):
    U = inputs.su3_links(DIMS, 101)[0]
    b = inputs.gaussian_sources(DIMS, 201, n_rhs=2)
    ctx = Context(DIMS)
    ctx.load_links(U)
    ctx.set_mu_mw(mu, M_W)
    y1, st1, _ = ctx.sign_apply(b, k, 128)
    ctx.set_nesting([40, 16])
    y3, st3, _ = ctx.sign_apply(b, k, 128, flags=flags)
    p = st3["p"][0]
    y_or, _ = nested.sign_apply(U, DIMS, mu, M_W, b[0], k, 128, p=p)
    for i in range(2):
        assert rel(y3[i], y1[i]) < (1e-9 if flags == NK_FP64 else 1e-8)
    assert rel(y3[0], y_or) < (1e-9 if flags == NK_FP64 else 1e-8)
    ctx.close()
