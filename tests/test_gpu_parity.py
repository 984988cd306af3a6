"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerance (FP32 multislice + FP32 contraction): normalised RMS map error
eps = ||I_gpu - I_ref|| / ||I_ref|| <= 1e-4, the bound the design states for
the FP32 path; S-matrix columns are compared with a relative tolerance of 1e-5
per depth (FP32 FFT round-off grows like sqrt(log N) per step).
"""
import math

import numpy as np
import pytest

import specimen as sp
from oracle import linear as lin
from oracle import multislice as ms

pytestmark = pytest.mark.gpu

EPS_FP32 = 1e-4
# TF32 tensor cores: FP32 multislice, operands rounded to TF32, FP32 accumulate; held to
# the FP32 bound
EPS_TF32 = 1e-4
# BF16 hi+lo split (three products): the reduced-precision bound
EPS_BF16X3 = 1e-3
EPS = {"fp32": EPS_FP32, "tf32": EPS_TF32, "bf16x3": EPS_BF16X3}
PRECS = ("fp32", "tf32", "bf16x3")


def variants():
    """(precision, association) pairs: both groupings of the tensor-core contraction."""
    out = [("fp32", "auto"), ("tf32", "auto")]
    for prec in ("tf32", "bf16x3"):
        out += [(prec, "transition_first"), (prec, "probe_first")]
    return out


def run_map(g, ctx, sm, wl, prec, assoc):
    ctx.set_association(assoc)
    try:
        return g.inelastic_map_for(ctx, sm, wl, prec)
    finally:
        ctx.set_association("auto")


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_07628_gb300 import build
    build.build()
    import paper_1908_07628_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def ctx(g):
    return g.Context(0)


def eps(ref, test):
    return ms.relative_error(ref, test)


def _rand(n, f, seed, n_z=4, n_sites=6, w=8, cell=None, scan_n=3, n_types=2):
    cell = cell if cell is not None else n * 0.05
    return sp.random_workload(n=n, n_z=n_z, f=f, cell=cell, n_sites=n_sites, w=w, seed=seed,
                              scan_n=scan_n, n_types=n_types, alpha=0.02, beta=0.03, dz=1.8)


# --- S_in ---------------------------------------------------------------------------------

@pytest.mark.parametrize("n,f,seed", [(64, 1, 1), (128, 2, 2), (384, 2, 3)])
def test_s_in_matches_oracle(g, ctx, n, f, seed):
    import torch
    wl = _rand(n, f, seed, n_z=3)
    sm = g.build_smatrix_for(ctx, wl)
    ref, (bp, bq) = lin.build_s_in(wl)
    p, q = sm.beams()
    assert np.array_equal(p, bp) and np.array_equal(q, bq)
    for depth in range(wl.n_z):
        out = torch.empty((sm.n_in, n // 2, n // 2), dtype=torch.complex64, device="cuda")
        sm.copy_depth(depth, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.complex128) / n
        err = np.linalg.norm(got - ref[depth]) / np.linalg.norm(ref[depth])
        assert err < 1e-5, (depth, err)


# --- maps -----------------------------------------------------------------------------------

@pytest.mark.parametrize("n,f,seed,w", [(64, 1, 4, 8), (64, 2, 5, 13), (128, 3, 6, 20),
                                        (256, 2, 7, 32), (384, 3, 8, 24)])
def test_linear_map_matches_oracle(g, ctx, n, f, seed, w):
    wl = _rand(n, f, seed, w=w, n_sites=8)
    ref = lin.linear_map(wl) if n >= 256 else ms.quadratic_map(wl)
    sm = g.build_smatrix_for(ctx, wl)
    assert ref.max() > 0
    for prec, assoc in variants():
        got = run_map(g, ctx, sm, wl, prec, assoc)
        assert eps(ref, got) < EPS[prec], (prec, assoc)


@pytest.mark.parametrize("width", [128, 256])
@pytest.mark.parametrize("n,f,seed,w", [(128, 3, 6, 20), (256, 2, 7, 32), (64, 2, 5, 13)])
def test_tile_widths_match_oracle(g, ctx, width, n, f, seed, w):
    """Both output tile widths of the tensor-core GEMMs (EELS_OPT_TILE_WIDTH), forced, in
    every grouping and precision; column counts that are and are not multiples of 128."""
    wl = _rand(n, f, seed, w=w, n_sites=8)
    ref = lin.linear_map(wl) if n >= 256 else ms.quadratic_map(wl)
    assert ref.max() > 0
    sm = g.build_smatrix_for(ctx, wl)
    ctx.set_tile_width(width)
    try:
        for prec, assoc in variants():
            got = run_map(g, ctx, sm, wl, prec, assoc)
            assert eps(ref, got) < EPS[prec], (width, prec, assoc, eps(ref, got))
    finally:
        ctx.set_tile_width(0)


def test_rocksalt_small_full_map(g, ctx):
    wl = sp.rocksalt_small()
    ref = lin.linear_map(wl)
    q = ms.quadratic_map(wl, positions=[(0, 0), (5, 2)])
    for iy, ix in [(0, 0), (5, 2)]:
        assert np.allclose(q[:, iy, ix], ref[:, iy, ix], rtol=1e-12, atol=0)
    sm = g.build_smatrix_for(ctx, wl)
    for prec, assoc in variants():
        got = run_map(g, ctx, sm, wl, prec, assoc)
        assert eps(ref, got) < EPS[prec], (prec, assoc)
        for m in range(wl.n_types):
            assert eps(ref[m], got[m]) < EPS[prec], (prec, assoc, m)


def test_quadratic_reference_map_matches_oracle(g, ctx):
    wl = _rand(64, 2, 9, n_sites=5)
    ref = ms.quadratic_map(wl)
    c = {}
    ms.quadratic_map(wl, positions=[(0, 0)], counter=c)
    got, steps = g.quadratic_reference_map_for(ctx, wl)
    assert eps(ref, got) < EPS_FP32
    # the GPU count is the paper's per-probe count summed over probes
    c_all = {}
    ms.quadratic_map(wl, counter=c_all)
    assert steps == c_all["steps"]


def test_quadratic_reference_subset_positions(g, ctx):
    wl = sp.rocksalt_small()
    pos = [(1, 3), (6, 7)]
    ref = ms.quadratic_map(wl, positions=pos)
    got, steps = g.quadratic_reference_map_for(ctx, wl, positions=pos)
    assert eps(ref, got) < EPS_FP32
    assert steps == 2 * (24 * 21 + 6)


# --- edge cases -------------------------------------------------------------------------

def test_no_sites_gives_zero_map(g, ctx):
    wl = _rand(64, 1, 10).with_sites([])
    sm = g.build_smatrix_for(ctx, wl)
    for prec, assoc in variants():
        got = run_map(g, ctx, sm, wl, prec, assoc)
        assert got.shape == (wl.n_types, wl.scan[1], wl.scan[0]) and not got.any()


def test_single_slice_and_extreme_windows(g, ctx):
    for w in (1, 32):
        wl = _rand(64, 1, 11 + w, n_z=1, w=w, n_sites=3)
        ref = ms.quadratic_map(wl)
        sm = g.build_smatrix_for(ctx, wl)
        for prec, assoc in variants():
            got = run_map(g, ctx, sm, wl, prec, assoc)
            assert eps(ref, got) < EPS[prec], (w, prec, assoc)


@pytest.mark.parametrize("n_types", [1, 6])
def test_channel_counts(g, ctx, n_types):
    """One channel and six (the serving stream's range): the per-channel planes of the
    spread epilogue, the transition lists and the map planes, in every variant."""
    wl = _rand(128, 2, 43, n_sites=5, w=12, n_types=n_types)
    ref = ms.quadratic_map(wl)
    assert ref.shape[0] == n_types and ref.max() > 0
    sm = g.build_smatrix_for(ctx, wl)
    for prec, assoc in variants():
        got = run_map(g, ctx, sm, wl, prec, assoc)
        assert eps(ref, got) < EPS[prec], (n_types, prec, assoc)
        for m in range(n_types):
            if ref[m].max() > 0:
                assert eps(ref[m], got[m]) < EPS[prec], (n_types, m, prec, assoc)


@pytest.mark.parametrize("scan", [(1, 1), (7, 1), (1, 9)])
def test_degenerate_scans(g, ctx, scan):
    """A single probe position and single-row / single-column scans (one-row phase tables,
    one-position windows, GEMM tiles with one valid column pair or row) in every variant."""
    wl = _rand(128, 2, 41, n_sites=6, w=10, scan_n=4)
    wl = wl.with_scan(scan + tuple(wl.scan[2:]))
    ref = ms.quadratic_map(wl)
    assert ref.shape[1:] == (scan[1], scan[0])
    sm = g.build_smatrix_for(ctx, wl)
    for prec, assoc in variants():
        got = run_map(g, ctx, sm, wl, prec, assoc)
        assert got.shape == ref.shape
        if ref.max() == 0:
            assert not got.any(), (prec, assoc)
        else:
            assert eps(ref, got) < EPS[prec], (scan, prec, assoc)


def test_site_outside_every_window_contributes_nothing(g, ctx):
    wl = _rand(128, 4, 12, n_sites=4)
    rx, ry = wl.scan_positions()
    far_x = (rx[0] + wl.cell / 2) % wl.cell      # half a cell away: outside the L/4 window
    wl.site_x[:] = far_x
    sm = g.build_smatrix_for(ctx, wl)
    got = g.inelastic_map_for(ctx, sm, wl, "fp32")
    assert not got.any()


def test_window_rule_tie_is_half_open(g, ctx):
    """A site exactly at -L/(2f) from a probe counts, one at +L/(2f) does not."""
    wl = _rand(64, 2, 13, n_sites=2, n_z=2)
    rx, ry = wl.scan_positions()
    h = wl.cell / (2 * wl.f)
    wl.site_x[:] = [rx[1] - h, rx[1] + h]
    wl.site_y[:] = ry[1]
    ref = ms.quadratic_map(wl)
    sm = g.build_smatrix_for(ctx, wl)
    got = g.inelastic_map_for(ctx, sm, wl, "fp32")
    assert eps(ref, got) < EPS_FP32


def test_errors_are_reported(g, ctx):
    wl = _rand(64, 1, 14)
    with pytest.raises(g.EelsError) as e:
        ctx.build_smatrix(np.zeros((2, 96, 96), np.float32), 10.0, 0.02508, 7e-4, 2.0, 1, 0.02)
    assert e.value.status == 2
    with pytest.raises(g.EelsError) as e:
        ctx.build_smatrix(wl.vproj, wl.cell, wl.lam, wl.sigma, wl.dz, 1, 0.5)  # beyond band
    assert e.value.status == 1
    sm = g.build_smatrix_for(ctx, wl)
    with pytest.raises(g.EelsError) as e:
        ctx.inelastic_map(sm, np.zeros((1, 1, 40, 40), np.complex64), [0], [0], [0], [0.0], [0.0],
                          wl.scan, wl.beta)
    assert e.value.status == 1


def test_non_finite_map_is_reported(g, ctx):
    """A NaN in one site's transition potential reaches the map: every precision returns
    EELS_ERR_NONFINITE (the map's sentinel); finite inputs on the same context then map
    normally."""
    wl = _rand(64, 1, 30, n_sites=3)
    sm = g.build_smatrix_for(ctx, wl)
    bad = wl.with_sites(np.arange(wl.n_sites))
    bad.H = bad.H.copy()
    bad.H[:, 0, 2, 3] = np.nan          # every site, so that a reached one carries it
    for prec, assoc in (("fp32", "auto"), ("tf32", "probe_first"), ("bf16x3", "transition_first")):
        with pytest.raises(g.EelsError) as e:
            run_map(g, ctx, sm, bad, prec, assoc)
        assert e.value.status == 7, prec
    assert eps(ms.quadratic_map(wl), g.inelastic_map_for(ctx, sm, wl, "fp32")) < EPS_FP32


# --- full-size workload, sampled outputs -----------------------------------------------------

def test_rocksalt_512_sampled_sites_and_probes(g, ctx):
    """The bench workload's S-matrix (512^2, 40 slices, f = 2) with three sites at three
    depths; the oracle evaluates the conventional algorithm at sampled probes."""
    wl = sp.rocksalt_fp32()
    rx, ry = wl.scan_positions()
    cx, cy = rx[16], ry[16]
    cand = [s for s in range(wl.n_sites)
            if abs(wl.site_x[s] - cx) < 3.0 and abs(wl.site_y[s] - cy) < 3.0]
    chosen = []
    for target in (0, 21, 39):
        for s in cand:
            if wl.site_slice[s] == target:
                chosen.append(s)
                break
    assert len(chosen) == 3
    sub = wl.with_sites(chosen)
    sm = g.build_smatrix_for(ctx, sub)
    pos = [(16, 16), (3, 29), (30, 5)]
    ref = ms.quadratic_map(sub, positions=pos)
    r = np.array([ref[:, iy, ix] for iy, ix in pos])
    assert r.max() > 0
    for prec, assoc in variants():
        got = run_map(g, ctx, sm, sub, prec, assoc)
        t = np.array([got[:, iy, ix] for iy, ix in pos])
        assert eps(r, t) < EPS[prec], (prec, assoc)


@pytest.mark.parametrize("name,targets,probes", [
    ("rocksalt_vacancy", (0, 40, 79), [(16, 16), (2, 29)]),
    ("nanoparticle", (12, 25, 44), [(64, 64), (60, 70)]),
])
def test_large_workloads_sampled(g, ctx, name, targets, probes):
    """768^2 vacancy crystal (80 slices, f = 2) and 1024^2 nanoparticle (50 slices, f = 4):
    the full S-matrix, three sites at three depths near the first probe, the m = 0
    channel; the conventional FP64 oracle evaluates the sampled probes."""
    wl = sp.WORKLOADS[name]()
    rx, ry = wl.scan_positions()
    cx, cy = rx[probes[0][1]], ry[probes[0][0]]
    chosen = []
    for target in targets:
        idx = np.nonzero(wl.site_slice == target)[0]
        assert idx.size, target
        d2 = (wl.site_x[idx] - cx) ** 2 + (wl.site_y[idx] - cy) ** 2
        chosen.append(int(idx[np.argmin(d2)]))
    sub = wl.with_sites(chosen)
    sub.H = np.ascontiguousarray(sub.H[:, 1:2])
    sm = g.build_smatrix_for(ctx, sub)
    ref = ms.quadratic_map(sub, positions=probes)
    r = np.array([ref[:, iy, ix] for iy, ix in probes])
    assert r.max() > 0
    for prec, assoc in variants():
        got = run_map(g, ctx, sm, sub, prec, assoc)
        t = np.array([got[:, iy, ix] for iy, ix in probes])
        assert eps(r, t) < EPS[prec], (prec, assoc, eps(r, t))


@pytest.mark.parametrize("name,prec", [("nanoparticle", "bf16x3"),
                                       ("rocksalt_vacancy", "bf16x3"),
                                       ("rocksalt_fp32", "tf32")])
def test_full_size_map_is_additive_over_its_sites(g, ctx, name, prec):
    """The full-size workloads with all their sites (13 571 on the 1024^2 nanoparticle,
    21 835 on the 768^2 vacancy crystal, 5 120 on the 512^2 crystal), in the launch
    configuration the bench times (batches of tens of sites, several per slice on the
    sphere): the map is a sum over sites (Eq. SHn0 summed over transitions), so the maps
    of the even- and odd-numbered sites add up to the full map, up to FP64 summation
    order (grouping and tile width fixed so that every site's contribution is computed
    the same way in all three calls).  The full map is finite and non-negative."""
    wl = sp.WORKLOADS[name]()
    sm = g.build_smatrix_for(ctx, wl)
    ctx.set_association("probe_first")
    ctx.set_tile_width(256)
    try:
        full = g.inelastic_map_for(ctx, sm, wl, prec)
        even = g.inelastic_map_for(ctx, sm, wl.with_sites(np.arange(0, wl.n_sites, 2)), prec)
        odd = g.inelastic_map_for(ctx, sm, wl.with_sites(np.arange(1, wl.n_sites, 2)), prec)
    finally:
        ctx.set_association("auto")
        ctx.set_tile_width(0)
    del sm
    assert np.all(np.isfinite(full)) and full.min() >= 0 and full.max() > 0
    assert np.abs(even + odd - full).max() <= 1e-12 * full.max()
    assert even.max() > 0 and odd.max() > 0


@pytest.mark.parametrize("cap", [1, 3])
def test_several_batches_per_slice_match_oracle(g, ctx, cap):
    """Sites of one slice contracted in several batches (EELS_OPT_BATCH_SITES): the
    batch offsets into the site, transition and tile lists are non-zero and the last
    batch is ragged.  Element by element against the oracle in both groupings."""
    wl = _rand(128, 2, 27, n_z=2, n_sites=14, w=12)
    rx, ry = wl.scan_positions()
    reached = [s for s in range(wl.n_sites)
               if any(ms.axis_in_window(wl.site_x[s], x, wl.cell, wl.f) for x in rx)
               and any(ms.axis_in_window(wl.site_y[s], y, wl.cell, wl.f) for y in ry)]
    counts = np.bincount(wl.site_slice[reached], minlength=wl.n_z)
    assert (counts > cap).all(), counts                            # every slice: > 1 batch
    assert cap == 1 or (counts % cap != 0).any(), counts           # a ragged last batch
    ref = lin.linear_map(wl)
    assert ref.max() > 0
    sm = g.build_smatrix_for(ctx, wl)
    whole = {}
    for prec, assoc in variants():
        whole[(prec, assoc)] = run_map(g, ctx, sm, wl, prec, assoc)
    ctx.set_batch_sites(cap)
    try:
        for prec, assoc in variants():
            got = run_map(g, ctx, sm, wl, prec, assoc)
            assert eps(ref, got) < EPS[prec], (prec, assoc, eps(ref, got))
            # batching changes only the order of the FP64 sums
            assert np.allclose(got, whole[(prec, assoc)], rtol=1e-12, atol=1e-15 * ref.max())
    finally:
        ctx.set_batch_sites(0)


def test_rocksalt_small_batches_of_three_sites(g, ctx):
    """The 128^2 rocksalt crystal (8 Fe sites per occupied slice, 3 channels) in batches
    of three sites: 3 + 3 + 2 per slice."""
    wl = sp.rocksalt_small()
    ref = lin.linear_map(wl)
    sm = g.build_smatrix_for(ctx, wl)
    ctx.set_batch_sites(3)
    try:
        for prec, assoc in variants():
            got = run_map(g, ctx, sm, wl, prec, assoc)
            assert eps(ref, got) < EPS[prec], (prec, assoc, eps(ref, got))
    finally:
        ctx.set_batch_sites(0)


# --- checkpointed S_in: segments recomputed during the backward sweep ---------------------

@pytest.mark.parametrize("k", [2, 3])
def test_checkpointed_s_in_gives_the_same_map(g, ctx, k):
    """A build that keeps the probe waves every k slices (EELS_OPT_SIN_CHECKPOINT) and a map
    that recomputes S_in segment by segment: 7 slices make a short last segment.  The map
    equals the one from the stored S_in up to the FP64 summation order, in every variant,
    and the oracle's within tolerance."""
    wl = _rand(128, 2, 29, n_z=7, n_sites=10, w=12)
    ref = lin.linear_map(wl)
    assert ref.max() > 0
    sm = g.build_smatrix_for(ctx, wl)
    whole = {v: run_map(g, ctx, sm, wl, *v) for v in variants()}
    ctx.set_sin_checkpoint(k)
    try:
        smc = g.build_smatrix_for(ctx, wl)
    finally:
        ctx.set_sin_checkpoint(0)
    for prec, assoc in variants():
        got = run_map(g, ctx, smc, wl, prec, assoc)
        assert np.allclose(got, whole[(prec, assoc)], rtol=1e-12, atol=1e-15 * ref.max()), \
            (prec, assoc)
        assert eps(ref, got) < EPS[prec], (prec, assoc)
    import torch
    out = torch.empty((smc.n_in, 64, 64), dtype=torch.complex64, device="cuda")
    with pytest.raises(g.EelsError) as e:
        smc.copy_depth(0, out)
    assert e.value.status == 2
    ctx.set_sout_scheme("recompute")
    try:
        with pytest.raises(g.EelsError) as e:
            g.inelastic_map_for(ctx, smc, wl, "fp32")
        assert e.value.status == 2
    finally:
        ctx.set_sout_scheme("stream")


def test_headline_checkpointed_s_in_gives_the_same_map(g, ctx):
    """The 1024^2 sphere with every site, S_in kept only as probe waves every 8 slices (the
    map server's choice for requests whose S-matrices would not fit, here 36 GB of
    checkpoints instead of 131 GB): the map recomputed segment by segment equals the map
    from the stored S_in up to FP64 summation order."""
    wl = sp.nanoparticle()
    ctx.set_association("probe_first")
    ctx.set_tile_width(256)
    try:
        sm = g.build_smatrix_for(ctx, wl)
        whole = g.inelastic_map_for(ctx, sm, wl, "bf16x3")
        del sm
        ctx.set_sin_checkpoint(8)
        try:
            smc = g.build_smatrix_for(ctx, wl)
        finally:
            ctx.set_sin_checkpoint(0)
        got = g.inelastic_map_for(ctx, smc, wl, "bf16x3")
        del smc
    finally:
        ctx.set_association("auto")
        ctx.set_tile_width(0)
    assert whole.max() > 0
    assert np.abs(got - whole).max() <= 1e-12 * whole.max()


# --- failure detection: a bounded device wait that runs out ------------------------------

def test_bounded_wait_timeout_is_reported_and_context_recovers(g, ctx):
    """EELS_OPT_WAIT_TEST withholds every TMA load of the tensor-core pipelines and cuts
    their waits to 2e6 cycles (about a millisecond): the consumers give up with nothing in
    flight, the kernels record it and return, and the map call reports EELS_ERR_TIMEOUT.
    The same context then computes a correct map."""
    wl = _rand(64, 2, 28, n_sites=4, w=8)
    ref = ms.quadratic_map(wl)
    sm = g.build_smatrix_for(ctx, wl)
    for prec, assoc in (("tf32", "probe_first"), ("bf16x3", "transition_first")):
        ctx.set_wait_test(2000)
        try:
            with pytest.raises(g.EelsError) as e:
                run_map(g, ctx, sm, wl, prec, assoc)
        finally:
            ctx.set_wait_test(0)
        assert e.value.status == 5 and "timed out" in str(e.value), str(e.value)
        got = run_map(g, ctx, sm, wl, prec, assoc)
        assert eps(ref, got) < EPS[prec], (prec, assoc)


def test_shared_transition_potentials_equal_per_site_copies(g, ctx):
    """h_shared: one [T][w][w] H for every site gives the map of the per-site copies."""
    wl = _rand(128, 2, 15, n_sites=6, w=12)
    Hs = np.ascontiguousarray(wl.H[0])
    wl_rep = wl.with_sites(np.arange(wl.n_sites))
    wl_rep.H = np.ascontiguousarray(np.broadcast_to(Hs, wl.H.shape))
    sm = g.build_smatrix_for(ctx, wl)
    for prec, assoc in variants():
        a = run_map(g, ctx, sm, wl_rep, prec, assoc)
        ctx.set_association(assoc)
        b = ctx.inelastic_map(sm, Hs, wl.site_slice, wl.win_x0, wl.win_y0, wl.site_x, wl.site_y,
                              wl.scan, wl.beta, precision=prec)
        ctx.set_association("auto")
        assert a.max() > 0 and np.allclose(a, b, rtol=1e-12, atol=0), (prec, assoc)
    qa, _ = g.quadratic_reference_map_for(ctx, wl_rep)
    qb, _ = ctx.quadratic_reference_map(wl.vproj, wl.cell, wl.lam, wl.sigma, wl.dz, wl.f,
                                        wl.alpha, Hs, wl.site_slice, wl.win_x0, wl.win_y0,
                                        wl.site_x, wl.site_y, wl.scan, wl.beta)
    assert np.allclose(qa, qb, rtol=1e-12, atol=0)


# --- detector-beam shards (the multi-GPU decomposition, run one after another) -------------

def test_detector_shards_run_in_sequence_sum_to_the_full_map(g, ctx):
    """G shards of the EELS aperture computed one after another on one GPU and added
    on the host in shard order equal the full map; each shard equals the oracle's map
    over the same detector beams."""
    from paper_1908_07628_gb300 import shard
    wl = _rand(128, 2, 16, n_sites=6, w=12)
    n_out = ms.lattice_beams(wl.n, wl.cell, wl.lam, wl.f, wl.beta)[0].size
    sm = g.build_smatrix_for(ctx, wl)
    try:
        for prec, assoc in variants():
            full = run_map(g, ctx, sm, wl, prec, assoc)
            parts = []
            for k in range(3):
                ctx.set_detector_shard(k, 3)
                parts.append(run_map(g, ctx, sm, wl, prec, assoc))
            ctx.set_detector_shard(0, 1)
            assert full.max() > 0 and eps(full, shard.sum_maps(parts)) < 1e-6, (prec, assoc)
            if prec == "fp32":
                for k in range(3):
                    ref = lin.linear_map(wl, detectors=np.array(shard.detector_shard(n_out, k, 3)))
                    assert eps(ref, parts[k]) < EPS_FP32, k
        # more shards than detector beams: the surplus shards are empty
        ctx.set_detector_shard(n_out + 1, n_out + 2)
        assert not g.inelastic_map_for(ctx, sm, wl, "tf32").any()
        ctx.set_detector_shard(3, 3)
        with pytest.raises(g.EelsError) as e:
            g.inelastic_map_for(ctx, sm, wl, "fp32")
        assert e.value.status == 1
    finally:
        ctx.set_detector_shard(0, 1)


# --- S_out schemes: the Sec. III listing and the inverse multislice retreat (Sec. IV C) ----

def _coarse(n, f, seed):
    """Strong random potentials sampled at 0.2 A: t_i reaches the band limit, so the
    inverse retreat loses a visible part of the detector waves."""
    return sp.random_workload(n=n, n_z=5, f=f, cell=n * 0.2, n_sites=8, w=12, seed=seed,
                              scan_n=3, alpha=0.0165, beta=0.025, dz=1.8, vscale=1200.0)


@pytest.mark.parametrize("scheme,n,f,seed", [("recompute", 128, 2, 17), ("inverse", 64, 2, 18),
                                             ("inverse", 128, 2, 26)])
def test_sout_schemes_match_oracle(g, ctx, scheme, n, f, seed):
    wl = _coarse(n, f, seed)
    ref = lin.linear_map(wl, scheme=scheme)
    exact = lin.linear_map(wl)
    assert exact.max() > 0
    if scheme == "inverse":
        assert eps(exact, ref) > 1e-3                   # the approximation is visible
    sm = g.build_smatrix_for(ctx, wl)
    ctx.set_sout_scheme(scheme)
    try:
        for prec, assoc in variants():
            got = run_map(g, ctx, sm, wl, prec, assoc)
            assert eps(ref, got) < EPS[prec], (prec, assoc, eps(ref, got))
    finally:
        ctx.set_sout_scheme("stream")


def test_inverse_scheme_on_rocksalt_matches_oracle(g, ctx):
    wl = sp.rocksalt_small()
    ref = lin.linear_map(wl, scheme="inverse")
    sm = g.build_smatrix_for(ctx, wl)
    ctx.set_sout_scheme("inverse")
    try:
        got = g.inelastic_map_for(ctx, sm, wl, "fp32")
    finally:
        ctx.set_sout_scheme("stream")
    assert eps(ref, got) < EPS_FP32


def test_inverse_scheme_is_exact_in_free_space(g, ctx):
    wl = _rand(128, 2, 20, n_sites=6, w=10, n_z=4)
    wl.vproj = np.zeros_like(wl.vproj)
    sm = g.build_smatrix_for(ctx, wl)
    exact = g.inelastic_map_for(ctx, sm, wl, "fp32")
    ctx.set_sout_scheme("inverse")
    try:
        got = g.inelastic_map_for(ctx, sm, wl, "fp32")
    finally:
        ctx.set_sout_scheme("stream")
    assert exact.max() > 0 and eps(exact, got) < 1e-5


# --- crop windows of a long-tailed transition potential (Sec. IV B) --------------------

def test_crop_series_matches_oracle(g, ctx):
    """The dopant slab (51.6 A) with its transition potential cut to 64 (the whole cell),
    30 and 15 pixels of the N/2 grid: each map equals the oracle's, and the GPU crop
    errors against the whole-cell map equal the oracle's."""
    maps, refs = {}, {}
    s_in = None
    sm = None
    for w in (64, 30, 15):
        wl = sp.dopant_slab(w, scan_n=12)
        if s_in is None:
            s_in = lin.build_s_in(wl)
            sm = g.build_smatrix_for(ctx, wl)
        refs[w] = lin.linear_map(wl, s_in=s_in)
        for prec in ("fp32", "tf32"):
            got = g.inelastic_map_for(ctx, sm, wl, prec)
            assert eps(refs[w], got) < EPS[prec], (w, prec)
            maps[(w, prec)] = got
    for w in (30, 15):
        e_ref = eps(refs[64], refs[w])
        e_gpu = eps(maps[(64, "fp32")], maps[(w, "fp32")])
        assert e_ref > 1e-3 and abs(e_gpu - e_ref) < 1e-3 * e_ref + 1e-6, (w, e_ref, e_gpu)


# --- frozen phonons -----------------------------------------------------------------------

def test_phonon_average_matches_oracle(g, ctx):
    from oracle import phonon
    cfg = sp.rocksalt_phonons(3, u_rms=0.1, ncell=2, nzc=3, n=128, f=2, scan_n=4, w=16)
    ref = phonon.average_map(cfg)
    assert ref.max() > 0
    for prec in ("fp32", "tf32", "bf16x3"):
        got = ctx.phonon_map(cfg, precision=prec)
        assert eps(ref, got) < EPS[prec], prec
    one = ctx.phonon_map(cfg[:1])
    assert eps(g.inelastic_map_for(ctx, g.build_smatrix_for(ctx, cfg[0]), cfg[0], "fp32"), one) < 1e-12
    with pytest.raises(g.EelsError) as e:
        ctx.phonon_map([cfg[0], sp.rocksalt_phonons(1, ncell=2, nzc=3, n=256, f=2, scan_n=4,
                                                     w=16)[0]])
    assert e.value.status == 1


@pytest.mark.parametrize("n,f,seed", [(512, 2, 24), (768, 2, 21), (768, 3, 22), (1024, 3, 25)])
def test_s_in_and_map_two_stage_plans(g, ctx, n, f, seed):
    """The two-stage FFT plans (512: radix 16 then 32; 768: 24 then 32; 1024: 32 then 32,
    second-stage twiddles from tables, pruned first inverse stage): S_in at every depth,
    and the map on 512 and 768.  A cell of 0.012 A per pixel keeps the peak host memory of
    the FP64 oracle near 4 GB at 768^2 (0.02 A per pixel took 10.9 GB there, enough for a
    memory-limited test process to be killed)."""
    import torch
    wl = _rand(n, f, seed, n_z=2, n_sites=4, w=12, cell=n * 0.012)
    s_in, beams = lin.build_s_in(wl)
    sm = g.build_smatrix_for(ctx, wl)
    nh = n // 2
    for depth in range(wl.n_z):
        out = torch.empty((sm.n_in, nh, nh), dtype=torch.complex64, device="cuda")
        sm.copy_depth(depth, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.complex128) / n
        err = np.linalg.norm(got - s_in[depth]) / np.linalg.norm(s_in[depth])
        assert err < 1e-5, (depth, err)
    if n > 768:
        return   # the 1024 map is checked on sampled probes of the nanoparticle
    # the FFT plan is what this checks: the map through the FP32 contraction (the
    # tensor-core contractions are checked on the other grids)
    ref = lin.linear_map(wl, s_in=(s_in, beams))
    assert ref.max() > 0
    assert eps(ref, g.inelastic_map_for(ctx, sm, wl, "fp32")) < EPS_FP32


def test_handle_freed_after_its_context(g):
    """A garbage collector may finalise a context before the S-matrix built on it; the
    handle must still free cleanly and leave no error for the next call."""
    wl = _rand(64, 1, 23)
    c = g.Context(0)
    sm = g.build_smatrix_for(c, wl)
    c.close()
    sm.free()
    c2 = g.Context(0)
    got = g.inelastic_map_for(c2, g.build_smatrix_for(c2, wl), wl, "fp32")
    assert eps(ms.quadratic_map(wl), got) < EPS_FP32
