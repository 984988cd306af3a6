"""Map server: continuous batching under an HBM budget.

Each request's map must be the same when it runs alone (Context.build_smatrix +
inelastic_map) and when it runs in the mix, within the tolerance of its precision;
requests that do not fit the remaining budget wait for memory to free up; a request
larger than the whole budget is rejected at submission.
"""
import numpy as np
import pytest

import specimen as sp
from oracle import multislice as ms

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-4, "tf32": 1e-3, "bf16x3": 1e-3}


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_07628_gb300 import build
    build.build()
    import paper_1908_07628_gb300 as pkg
    return pkg


def _requests():
    specs = [(128, 1, 3, "fp32"), (256, 2, 5, "tf32"), (128, 2, 4, "bf16x3"),
             (256, 3, 6, "tf32"), (128, 1, 2, "tf32"), (256, 2, 3, "fp32")]
    out = []
    for k, (n, f, n_z, prec) in enumerate(specs):
        wl = sp.random_workload(n=n, n_z=n_z, f=f, cell=n * 0.05, n_sites=7, w=10, seed=40 + k,
                                scan_n=4, alpha=0.02, beta=0.03, dz=1.8)
        out.append((wl, prec))
    return out


def _req(g, wl, prec):
    return g.make_request(wl.vproj, wl.cell, wl.lam, wl.sigma, wl.dz, wl.f, wl.alpha, wl.H,
                          wl.site_slice, wl.win_x0, wl.win_y0, wl.site_x, wl.site_y, wl.scan,
                          wl.beta, precision=prec)


def _alone(g, ctx, wl, prec):
    sm = g.build_smatrix_for(ctx, wl)
    return g.inelastic_map_for(ctx, sm, wl, prec)


@pytest.mark.parametrize("slots,budget_kind", [(3, "two_largest"), (3, "largest_only")])
def test_results_same_alone_and_in_the_mix(g, slots, budget_kind):
    reqs = _requests()
    built = [_req(g, wl, prec) for wl, prec in reqs]
    fps = sorted(g.request_footprint(r) for r, _ in built)
    budget = fps[-1] + fps[-2] if budget_kind == "two_largest" else fps[-1]
    srv = g.Server(0, hbm_budget=budget, slots=slots)
    ids = [srv.submit(r, keep, wl.n_types, wl.scan) for (r, keep), (wl, _) in zip(built, reqs)]
    maps = [srv.wait(i, timeout=300)[0] for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"] and st["peak_bytes"] <= budget
    ctx = g.Context(0)
    for (wl, prec), got in zip(reqs, maps):
        ref = _alone(g, ctx, wl, prec)
        assert ref.max() > 0
        assert ms.relative_error(ref, got) < TOL[prec], prec


def test_oversize_request_is_rejected(g):
    wl, prec = _requests()[1]
    r, keep = _req(g, wl, prec)
    srv = g.Server(0, hbm_budget=g.request_footprint(r) - 1, slots=1)
    with pytest.raises(g.EelsError) as e:
        srv.submit(r, keep, wl.n_types, wl.scan)
    srv.close()
    assert e.value.status == 3
