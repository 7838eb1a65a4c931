"""Overlap inversion on the GPU (nk_overlap_solve) against the dense solve.

x = (D_ov(mu) + m)^-1 b from the dense overlap operator of the oracle
(numpy's solver on I + gamma5 sgn(A), sgn from the spectral definition)
against the CG on the normal equations, whose every iteration applies the
nested sign function twice.  The sign function's error (about 1e-8 at these
k, with deflation at mu = 0.3) bounds the agreement: cond(M) is about 5 here.
"""
import numpy as np
import pytest

import inputs
from oracle import deflation, dirac, signfun

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0912_4457_gb300.nksign import NK_FP64, NK_OK, Context  # noqa: E402

DIMS = (3, 3, 3, 4)
M_W = -2.0
MASS = 0.2


@pytest.mark.parametrize("mu,k,defl", [(0.0, 256, 0), (0.3, 256, 16)])
def test_overlap_cg_matches_the_dense_solve(mu, k, defl):
    U = inputs.su3_links(DIMS, 31)[0]
    b = inputs.gaussian_sources(DIMS, 33, n_rhs=2)
    a = dirac.dense_A(U, DIMS, mu, M_W)
    herm = mu == 0.0
    s = signfun.sign_spectral(a, herm)
    n = a.shape[0]
    g5 = np.tile([1.0] * 6 + [-1.0] * 6, n // 12)
    M = np.eye(n) + g5[:, None] * s + MASS * np.eye(n)
    ctx = Context(DIMS)
    ctx.load_links(U)
    ctx.set_mu_mw(mu, M_W)
    if defl:
        lam, R, L = deflation.smallest_eigenpairs(a, defl, herm)
        ctx.set_deflation(lam, R.T, None if herm else L.T)
    x, its, res, rc = ctx.overlap_solve(b, k, 64, mass=MASS, tol_cg=1e-10, maxit=200, flags=NK_FP64, check=False)
    assert rc == NK_OK, (its, res)
    for i in range(2):
        xt = np.linalg.solve(M, b[i])
        assert np.linalg.norm(x[i] - xt) / np.linalg.norm(xt) < 1e-6
        assert res[i] <= 1e-10 and 0 < its[i] < 200
    ctx.close()
