"""The bench workload itself: 10^4, mu = 0.2, the 12 spin-colour point sources
at the origin, k = 1024, l = 128 with a second nested level l_2 = 64
(Sec. 4.5), FP32 stencil from step 256 with an FP64 recurrence, one p for the
batch, one CUDA graph.

* every source against the same batch all in FP64 at k = 1536, l = 256 (which
  FP64 k = 1024 already matches to 1e-11): within 1e-8;
* source 0 against the nested oracle at the same (k, l, l_2, p): within 1e-8 (the
  oracle takes about two minutes at this volume);
* the labelled second schedule, the two-float recurrence from step 0, within
  1e-8 of the same FP64 reference.
"""
import numpy as np
import pytest

import bench
from oracle import nested

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0912_4457_gb300.nksign import NK_FP64, NK_MIXED, NK_SHARED_P, Context  # noqa: E402

TOL = 1e-8


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_bench_workload_every_source_and_the_oracle():
    w = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    U, b = bench.make_inputs(w)
    ctx = Context(w["dims"])
    ctx.load_links(U)
    ctx.set_mu_mw(w["mu"], w["m_w"])
    ctx.set_precision(w["j0"])
    ctx.set_nesting(w.get("nest", ()))
    bd = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    y = torch.zeros_like(bd)
    st, rc = ctx.sign_apply_dev(bd, y, 12, w["k"], w["ell"], flags=NK_MIXED | NK_SHARED_P)
    assert rc == 0 and len(set(st["p"])) == 1
    yref = torch.zeros_like(bd)
    ctx.sign_apply_dev(bd, yref, 12, w["k_ref"], w["ell_ref"], flags=NK_FP64 | NK_SHARED_P)
    ymx, yr = y.cpu().numpy(), yref.cpu().numpy()
    errs = [rel(ymx[i], yr[i]) for i in range(12)]
    assert max(errs) <= TOL, errs
    ctx.set_df_recurrence(0)
    y2 = torch.zeros_like(bd)
    ctx.sign_apply_dev(bd, y2, 12, w["k"], w["ell"], flags=NK_MIXED | NK_SHARED_P)
    y2h = y2.cpu().numpy()
    assert max(rel(y2h[i], yr[i]) for i in range(12)) <= TOL
    ctx.close()
    y_or, _ = nested.sign_apply(U, w["dims"], w["mu"], w["m_w"], b[0], w["k"], w["ell"], p=st["p"][0],
                                ells=w.get("nest", ()))
    assert rel(ymx[0], y_or) <= TOL
    assert rel(yr[0], y_or) <= 1e-10    # FP64 at k = 1536 against the oracle at k = 1024
