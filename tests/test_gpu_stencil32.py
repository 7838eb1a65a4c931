"""The multi-RHS FP32 stencil (nk_stencil32_dev) against the oracle's stencil.

The kernel takes 2 n_rhs FP32 vectors in its pair layout ([6][V] of four
floats per vector: components 2i and 2i + 1 of a site, re/im interleaved) and
applies A to the first n_rhs and A^dagger to the others.  Cases cover both
block shapes (8 sites above 12 vectors, 32 up to 12), a lattice whose
volume is not a multiple of the block (ragged last block), periodic and
antiperiodic t.  Tolerance: FP32 rounding of the input, the links and ~100
flops per component (2e-6 relative, as for the FP32 stencil elsewhere).
"""
import numpy as np
import pytest

import inputs
from oracle import dirac

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0912_4457_gb300.nksign import Context  # noqa: E402

M_W = -2.0


def to_pair_layout(x, V):
    """(n, 12 V) complex in the ABI layout [site][12] -> (n, 6, V, 4) float32."""
    n = x.shape[0]
    c = x.reshape(n, V, 6, 2)                   # site, pair, member
    out = np.empty((n, 6, V, 4), np.float32)
    out[..., 0] = c[..., 0].real.transpose(0, 2, 1)
    out[..., 1] = c[..., 0].imag.transpose(0, 2, 1)
    out[..., 2] = c[..., 1].real.transpose(0, 2, 1)
    out[..., 3] = c[..., 1].imag.transpose(0, 2, 1)
    return out


def from_pair_layout(p, V):
    n = p.shape[0]
    c = np.empty((n, V, 6, 2), np.complex128)
    c[..., 0] = (p[..., 0] + 1j * p[..., 1]).transpose(0, 2, 1)
    c[..., 1] = (p[..., 2] + 1j * p[..., 3]).transpose(0, 2, 1)
    return c.reshape(n, 12 * V)


@pytest.mark.parametrize("dims,n_rhs,mu,anti", [
    ((4, 4, 4, 4), 12, 0.3, True),       # 24 vectors: 16-site blocks
    ((3, 5, 2, 6), 12, 0.2, True),       # V = 180: ragged last block of 16
    ((3, 5, 2, 6), 5, 0.0, False),       # 10 vectors: 32-site blocks, ragged, periodic t
    ((6, 4, 4, 6), 1, 0.5, True),        # 2 vectors
])
def test_stencil32_native_layout_matches_oracle(dims, n_rhs, mu, anti):
    V = int(np.prod(dims))
    U = inputs.su3_links(dims, 21)[0]
    x = inputs.gaussian_sources(dims, 22, n_rhs=2 * n_rhs)
    ctx = Context(dims, anti)
    ctx.load_links(U)
    ctx.set_mu_mw(mu, M_W)
    xin = torch.from_numpy(to_pair_layout(x, V).reshape(-1)).cuda()
    out = torch.full_like(xin, float("nan"))
    ctx.stencil32_dev(xin, out, n_rhs)
    torch.cuda.synchronize()
    got = from_pair_layout(out.cpu().numpy().reshape(2 * n_rhs, 6, V, 4), V)
    for i in range(2 * n_rhs):
        f = dirac.apply_A if i < n_rhs else dirac.apply_A_dagger
        ref = f(x[i], U, dims, mu, M_W, antiperiodic_t=anti)
        assert np.linalg.norm(got[i] - ref) / np.linalg.norm(ref) < 2e-6, i
    ctx.close()


def test_dslash_fp32_24_vectors():
    """nk_dslash_dev precision 32 with 24 vectors (the 16-site block shape)."""
    dims = (4, 4, 4, 6)
    U = inputs.su3_links(dims, 23)[0]
    x = inputs.gaussian_sources(dims, 24, n_rhs=24)
    ctx = Context(dims)
    ctx.load_links(U)
    ctx.set_mu_mw(0.3, M_W)
    xd = torch.from_numpy(x).cuda()
    o = torch.zeros_like(xd)
    ctx.dslash_dev(xd, o, 24, dagger=True, precision=32)
    torch.cuda.synchronize()
    got = o.cpu().numpy()
    for i in (0, 7, 23):
        ref = dirac.apply_A_dagger(x[i], U, dims, 0.3, M_W)
        assert np.linalg.norm(got[i] - ref) / np.linalg.norm(ref) < 2e-6
    ctx.close()
