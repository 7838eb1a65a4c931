"""nk_inner_sign_noalloc against nk_inner_sign, through the C ABI.

The no-allocation entry point serves callers that must not allocate device
memory (code running where cudaMalloc is forbidden or unsafe, e.g. inside
another framework's memory budget).  It keeps its scratch in one static device
array of the library, so it is checked here against the ordinary entry point
on two calls in a row -- the second call must not see leftovers of the first
-- and for its size limit.  This file is collected last on purpose.
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

TOL = 1e-11   # the inner-sign parity tolerance of tests/test_gpu_parity.py


def _ritz(mu, k, seeds):
    dims = (4, 4, 4, 4)
    U, _ = inputs.su3_links(dims, 101)
    A, Ad, herm = nested.operator(U, dims, mu, -2.0)
    hs = [nested.outer_basis(A, Ad, inputs.gaussian_sources(dims, s)[0], k, herm) for s in seeds]
    pad = lambda x: np.concatenate([x, np.zeros(1, x.dtype)]) if len(x) < k else x
    al = np.stack([h.alpha for h in hs]).astype(np.complex128)
    be = np.stack([pad(h.beta) for h in hs]).astype(np.complex128)
    ga = np.stack([pad(h.gamma) for h in hs]).astype(np.complex128)
    return dims, U, al, be, ga, herm


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("first,second", [((0.3, 256, 64, (301, 302)), (0.0, 192, 48, (303,)))])
def test_noalloc_matches_inner_sign_two_calls(first, second):
    for mu, k, ell, seeds in (first, second):
        dims, U, al, be, ga, herm = _ritz(mu, k, seeds)
        ctx = nksign.Context(dims)
        c_ref, st, _ = ctx.inner_sign(al, be, ga, ell, p=0.0, hermitian=herm)
        ctx.close()
        n = len(seeds)
        c_dev = torch.full((n, k), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        rc, msg = nksign.inner_sign_noalloc(_dev(al), _dev(be), _dev(ga), c_dev, n, k, ell, 0.0, herm)
        assert rc == nksign.NK_OK, msg
        c = c_dev.cpu().numpy()
        for r in range(n):
            assert np.linalg.norm(c[r] - c_ref[r]) / np.linalg.norm(c_ref[r]) < TOL


def test_noalloc_rejects_sizes_beyond_its_scratch():
    k = 1026
    a = torch.zeros((1, k), dtype=torch.complex128, device="cuda")
    c = torch.zeros_like(a)
    rc, msg = nksign.inner_sign_noalloc(a, a, a, c, 1, k, 64, 1.0, True)
    assert rc == nksign.NK_EINVAL
    assert "static scratch" in msg and "1024" in msg
    rc, msg = nksign.inner_sign_noalloc(a[:, :64], a[:, :64], a[:, :64], c[:, :64], 3, 64, 16, 1.0, True)
    assert rc == nksign.NK_EINVAL
