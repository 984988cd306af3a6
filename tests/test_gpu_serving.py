"""Map server: continuous batching under an HBM budget, work issued in tiles.

Each request's map must be the same when it runs alone (Context.build_smatrix +
inelastic_map with the same deterministic grouping) and when its tiles interleave with
other requests' on the device: equal up to the order of the FP64 map sums (1e-12), and
equal to the alone map of every other precision within that precision's tolerance;
requests must overlap on the device (their first-tile-to-done intervals intersect);
requests that do not fit the remaining budget wait for memory to free up; a request
larger than the whole budget is rejected at submission; a cancelled request and one
past its deadline are dropped with EELS_ERR_CANCELLED while the others complete.
"""
import numpy as np
import pytest

import specimen as sp
from oracle import multislice as ms

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-4, "tf32": 1e-4, "bf16x3": 1e-3}
SAME = 1e-12   # the same request alone and in the mix: FP64 summation order only


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


def _req(g, wl, prec, deadline_s=0.0, sin_checkpoint=0):
    return g.make_request(wl.vproj, wl.cell, wl.lam, wl.sigma, wl.dz, wl.f, wl.alpha, wl.H,
                          wl.site_slice, wl.win_x0, wl.win_y0, wl.site_x, wl.site_y, wl.scan,
                          wl.beta, precision=prec, deadline_s=deadline_s,
                          sin_checkpoint=sin_checkpoint)


def _alone(g, ctx, wl, prec):
    """The request's map computed directly, with the server's grouping rule."""
    ctx.set_association("model")
    try:
        sm = g.build_smatrix_for(ctx, wl)
        return g.inelastic_map_for(ctx, sm, wl, prec)
    finally:
        ctx.set_association("auto")


@pytest.mark.parametrize("slots,budget_kind", [(3, "two_largest"), (3, "largest_only")])
def test_results_same_alone_and_in_the_mix(g, slots, budget_kind):
    reqs = _requests()
    # the fourth request keeps its probe waves every 3 slices and recomputes S_in
    built = [_req(g, wl, prec, sin_checkpoint=3 if k == 3 else 0)
             for k, (wl, prec) in enumerate(reqs)]
    fps = sorted(g.request_footprint(r) for r, _ in built)
    budget = fps[-1] + fps[-2] if budget_kind == "two_largest" else fps[-1]
    srv = g.Server(0, hbm_budget=budget, slots=slots)
    ids = [srv.submit(r, keep, wl.n_types, wl.scan) for (r, keep), (wl, _) in zip(built, reqs)]
    maps = [srv.wait(i, timeout=300)[0] for i in ids]
    info = [srv.info(i) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["cancelled"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"] and st["peak_bytes"] <= budget
    spans = sorted((r["t_first_tile"], r["t_done"]) for r in info)
    assert all(a >= 0 and b > a for a, b in spans)
    if budget_kind == "two_largest":
        # room for two requests at once: at least two were on the device together (their
        # intervals from the first issued tile to completion intersect)
        assert any(spans[k + 1][0] < spans[k][1] for k in range(len(spans) - 1)), spans
    assert all(r["tiles"] >= 2 for r in info)   # every request ran as several tiles
    ctx = g.Context(0)
    for (wl, prec), got in zip(reqs, maps):
        ref = _alone(g, ctx, wl, prec)
        assert ref.max() > 0
        assert ms.relative_error(ref, got) < SAME, prec
        for other in TOL:                          # and within tolerance of the others
            if other != prec:
                assert ms.relative_error(_alone(g, ctx, wl, other), got) < max(TOL[prec], TOL[other])


def test_oversize_request_is_rejected(g):
    wl, prec = _requests()[1]
    r, keep = _req(g, wl, prec)
    srv = g.Server(0, hbm_budget=g.request_footprint(r) - 1, slots=1)
    with pytest.raises(g.EelsError) as e:
        srv.submit(r, keep, wl.n_types, wl.scan)
    srv.close()
    assert e.value.status == 3


def test_cancelled_and_expired_requests_are_dropped(g):
    """A long request cancelled while it runs, one cancelled before admission and one
    whose deadline passes are dropped with EELS_ERR_CANCELLED and their memory is given
    back; the requests around them complete with their alone maps."""
    long_wl = sp.random_workload(n=512, n_z=80, f=2, cell=25.6, n_sites=7, w=10, seed=51,
                                 scan_n=4, alpha=0.02, beta=0.03, dz=1.8)
    reqs = _requests()[:3]
    built = [_req(g, wl, prec) for wl, prec in reqs]
    r_long, k_long = _req(g, long_wl, "tf32")
    r_late, k_late = _req(g, long_wl, "tf32", deadline_s=1e-3)
    fp = max(g.request_footprint(r) for r, _ in built + [(r_long, k_long)])
    srv = g.Server(0, hbm_budget=2 * fp, slots=1)
    i_long = srv.submit(r_long, k_long, long_wl.n_types, long_wl.scan)
    i_late = srv.submit(r_late, k_late, long_wl.n_types, long_wl.scan)
    ids = [srv.submit(r, keep, wl.n_types, wl.scan) for (r, keep), (wl, _) in zip(built, reqs)]
    i_pend = srv.submit(*_req(g, long_wl, "tf32"), long_wl.n_types, long_wl.scan)
    srv.cancel(i_pend)            # still queued behind the others: dropped before admission
    import time
    t0 = time.time()
    while srv.info(i_long)["tiles"] < 2 and time.time() - t0 < 60:
        time.sleep(0.002)
    srv.cancel(i_long)            # running: dropped at its next tile boundary
    for i in (i_long, i_late, i_pend):
        with pytest.raises(g.EelsError) as e:
            srv.wait(i, timeout=300)
        assert e.value.status == 6
    assert srv.info(i_pend)["tiles"] == 0 and srv.info(i_pend)["t_admit"] < 0
    assert srv.info(i_long)["tiles"] < 2 * long_wl.n_z // 4
    maps = [srv.wait(i, timeout=300)[0] for i in ids]
    st = srv.stats()
    srv.close()
    assert st["cancelled"] == 3 and st["completed"] == len(reqs) and st["failed"] == 0
    ctx = g.Context(0)
    for (wl, prec), got in zip(reqs, maps):
        assert ms.relative_error(_alone(g, ctx, wl, prec), got) < SAME, prec


def _window_count(coords, positions, cell, f):
    """Scan positions within a site's PRISM window along one axis (minimum image, half-open
    [-L/2f, L/2f))."""
    out = []
    for s in coords:
        d = s - positions
        d = d - cell * np.floor(d / cell + 0.5)
        out.append(int(np.sum((d >= -cell / (2 * f)) & (d < cell / (2 * f)))))
    return np.array(out)


def test_request_metrics_and_jsonl_log(g, tmp_path):
    """Per-request metrics: beams, pixel-slices, wave-steps (with and without S_in
    checkpoints) and the contraction's flops as the server groups it (8 per complex
    product, the grouping with fewer products), and one JSON line per request."""
    import json
    reqs = _requests()[:3]
    built = [_req(g, wl, prec, sin_checkpoint=3 if k == 1 else 0)
             for k, (wl, prec) in enumerate(reqs)]
    srv = g.Server(0, hbm_budget=sum(g.request_footprint(r) for r, _ in built), slots=2)
    ids = [srv.submit(r, keep, wl.n_types, wl.scan) for (r, keep), (wl, _) in zip(built, reqs)]
    for i in ids:
        srv.wait(i, timeout=300)
    infos = [srv.info(i) for i in ids]
    path = str(tmp_path / "requests.jsonl")
    srv.log_jsonl(path, ids, extra={ids[0]: {"tag": "first"}})
    srv.close()
    for k, ((wl, prec), d) in enumerate(zip(reqs, infos)):
        n_in = g.count_beams(wl.n, wl.cell, wl.lam, wl.f, wl.alpha)
        n_out = g.count_beams(wl.n, wl.cell, wl.lam, wl.f, wl.beta)
        assert (d["n_in"], d["n_out"]) == (n_in, n_out)
        n_sx, n_sy, x0, y0, sx, sy = wl.scan
        assert d["pixel_slices"] == n_sx * n_sy * wl.n_z
        assert d["wave_steps"] == (n_in * (2 if k == 1 else 1) + n_out) * wl.n_z
        nx = _window_count(wl.site_x, x0 + sx * np.arange(n_sx), wl.cell, wl.f)
        ny = _window_count(wl.site_y, y0 + sy * np.arange(n_sy), wl.cell, wl.f)
        nr = (nx * ny).astype(float)
        P, T = wl.H.shape[-1] ** 2, wl.n_types
        c_tr = float(np.sum((nr > 0) * T * (n_out * P * n_in + n_out * n_in * nr)))
        c_pr = float(np.sum(nr * n_in * P + T * n_out * P * nr))
        want = 8 * (c_tr if prec == "fp32" else min(c_tr, c_pr))
        assert want > 0 and abs(d["contraction_flops"] - want) <= 1e-9 * want, (prec, d, want)
    lines = [json.loads(ln) for ln in open(path)]
    assert [ln["id"] for ln in lines] == ids and lines[0]["tag"] == "first"
    for ln in lines:
        assert ln["status"] == 0 and ln["latency_s"] > 0 and ln["pixel_slices_per_s"] > 0
        assert ln["wait_s"] >= 0 and ln["contraction_flops"] > 0
