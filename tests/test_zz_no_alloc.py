"""nk_inner_sign_noalloc through the C ABI.

The no-allocation entry point serves callers that may not allocate device
memory: code that runs inside another framework's memory budget, a process
whose allocator belongs to someone else, or a path that must not call
cudaMalloc.  It keeps its scratch in one static device array of the library,
so each case here runs two calls in a row -- the second must not see
leftovers of the first -- and compares each result with the ordinary entry
point nk_inner_sign and with the CPU oracle on the same H_k.  It also checks
the size limit.  This file is collected last on purpose.
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
TOL_ORACLE = 1e-10


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _ritz(mu, k, seeds):
    dims = (4, 4, 4, 4)
    U, _ = inputs.su3_links(dims, 101)
    A, Ad, herm = nested.operator(U, dims, mu, -2.0)
    hs = [nested.outer_basis(A, Ad, inputs.gaussian_sources(dims, s)[0], k, herm) for s in seeds]
    pad = lambda x: np.concatenate([x, np.zeros(1, x.dtype)]) if len(x) < k else x
    al = np.stack([h.alpha for h in hs]).astype(np.complex128)
    be = np.stack([pad(h.beta) for h in hs]).astype(np.complex128)
    ga = np.stack([pad(h.gamma) for h in hs]).astype(np.complex128)
    return dims, hs, al, be, ga, herm


def _oracle_c(hs, ell, p, herm):
    """The oracle's c for each RHS: p per RHS (p == 0), one p for the batch
    from the extremes of the per-RHS estimates (p < 0), or p itself."""
    est = [nested.estimate_p(h.alpha, h.beta, h.gamma) for h in hs]
    if p < 0:
        ps = [nested.shared_p(est)] * len(hs)
    elif p == 0:
        ps = [e[0] for e in est]
    else:
        ps = [p] * len(hs)
    return [nested.inner_sign(h.alpha, h.beta, h.gamma, ell, pp, herm)[0] for h, pp in zip(hs, ps)]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# (mu, k, l, source seeds, p): p == 0 one p per RHS, p < 0 one p for the batch
CASES = [((0.3, 256, 64, (301, 302), 0.0), (0.0, 192, 48, (303,), 0.0)),
         ((0.3, 256, 64, (301, 302), -1.0), (0.3, 192, 64, (304, 305), -1.0))]


@pytest.mark.parametrize("first,second", CASES)
def test_noalloc_matches_inner_sign_two_calls(first, second):
    for mu, k, ell, seeds, p in (first, second):
        dims, hs, al, be, ga, herm = _ritz(mu, k, seeds)
        ctx = nksign.Context(dims)
        c_ref, st, _ = ctx.inner_sign(al, be, ga, ell, p=p, hermitian=herm)
        ctx.close()
        c_or = _oracle_c(hs, ell, p, herm)
        n = len(seeds)
        c_dev = torch.full((n, k), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        rc, msg = nksign.inner_sign_noalloc(_dev(al), _dev(be), _dev(ga), c_dev, n, k, ell, p, herm)
        assert rc == nksign.NK_OK, msg
        c = c_dev.cpu().numpy()
        for r in range(n):
            assert _rel(c[r], c_ref[r]) < TOL
            assert _rel(c[r], c_or[r]) < TOL_ORACLE


def test_noalloc_rejects_sizes_beyond_its_scratch():
    k = 1026
    a = torch.zeros((1, k), dtype=torch.complex128, device="cuda")
    c = torch.zeros_like(a)
    rc, msg = nksign.inner_sign_noalloc(a, a, a, c, 1, k, 64, 1.0, True)
    assert rc == nksign.NK_EINVAL
    assert "static scratch" in msg and "1024" in msg
    b = torch.zeros((3, 64), dtype=torch.complex128, device="cuda")
    rc, msg = nksign.inner_sign_noalloc(b, b, b, torch.zeros_like(b), 3, 64, 16, 1.0, True)
    assert rc == nksign.NK_EINVAL and "n_rhs <= 2" in msg
