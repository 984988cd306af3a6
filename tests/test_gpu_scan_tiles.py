"""Per-scan-tile resumable maps (eels_inelastic_map_tiles) against the one-call map.

A position's map value depends only on that position (its PRISM windows and probe
coefficients), so with the grouping and tile width fixed the tiled map equals the
one-call map up to FP64 summation order.  Checked: ragged tilings (edge tiles narrower,
one-position tiles, one tile covering the scan) in every precision; a map finished over
several calls of two tiles each; a call that fails in the middle (bounded-wait test
mode) keeps the finished tiles and the next call completes the map; a process that maps
two tiles into a checkpoint file and exits, after which this process resumes from the
file; and the argument checks.
"""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

import specimen as sp
from oracle import multislice as ms

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EPS = {"fp32": 1e-4, "tf32": 1e-4, "bf16x3": 1e-3}
SAME = 1e-11   # tiled against one-call map, relative to the map's largest value


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


def _workload():
    return sp.random_workload(n=128, n_z=5, f=2, cell=128 * 0.05, n_sites=10, w=16, seed=41,
                              scan_n=7, n_types=2, alpha=0.02, beta=0.03, dz=1.8)


def _fixed(ctx, assoc):
    ctx.set_association(assoc)
    ctx.set_tile_width(256)


def _reset(ctx):
    ctx.set_association("auto")
    ctx.set_tile_width(0)


def _close(a, b):
    return np.abs(a - b).max() <= SAME * np.abs(b).max()


@pytest.mark.parametrize("prec,assoc", [("fp32", "auto"), ("tf32", "probe_first"),
                                        ("tf32", "transition_first"), ("bf16x3", "probe_first")])
@pytest.mark.parametrize("tile", [(3, 2), (1, 1), (7, 7), (4, 7)])
def test_tiled_map_equals_one_call_map(g, ctx, prec, assoc, tile):
    wl = _workload()
    sm = g.build_smatrix_for(ctx, wl)
    _fixed(ctx, assoc)
    try:
        full = g.inelastic_map_for(ctx, sm, wl, prec)
        gx, gy = -(-wl.scan[0] // tile[0]), -(-wl.scan[1] // tile[1])
        out = np.zeros_like(full)
        done = np.zeros((gy, gx), dtype=np.uint8)
        left = g.inelastic_map_tiles_for(ctx, sm, wl, tile, out, done, prec)
    finally:
        _reset(ctx)
    assert left == 0 and done.all()
    assert full.max() > 0
    assert _close(out, full), (prec, assoc, tile, np.abs(out - full).max() / full.max())


def test_tiled_map_matches_oracle_in_pieces(g, ctx):
    """Two tiles per call until done; the remaining count falls by two each call."""
    wl = _workload()
    ref = ms.quadratic_map(wl)
    sm = g.build_smatrix_for(ctx, wl)
    tile = (3, 3)                       # 3 x 3 tiles on the 7 x 7 scan
    out = np.zeros_like(ref)
    done = np.zeros((3, 3), dtype=np.uint8)
    lefts = []
    while True:
        lefts.append(g.inelastic_map_tiles_for(ctx, sm, wl, tile, out, done, "tf32",
                                               max_tiles=2))
        if lefts[-1] == 0:
            break
    assert lefts == [7, 5, 3, 1, 0]
    assert ms.relative_error(ref, out) < EPS["tf32"]


def test_failed_call_keeps_finished_tiles_and_resumes(g, ctx):
    wl = _workload()
    sm = g.build_smatrix_for(ctx, wl)
    _fixed(ctx, "probe_first")
    try:
        full = g.inelastic_map_for(ctx, sm, wl, "tf32")
        out = np.zeros_like(full)
        done = np.zeros((2, 2), dtype=np.uint8)
        tile = (4, 4)
        assert g.inelastic_map_tiles_for(ctx, sm, wl, tile, out, done, "tf32", max_tiles=1) == 3
        first = out.copy()
        ctx.set_wait_test(2000)          # every later tile's waits run out
        try:
            with pytest.raises(g.EelsError) as e:
                g.inelastic_map_tiles_for(ctx, sm, wl, tile, out, done, "tf32")
        finally:
            ctx.set_wait_test(0)
        assert e.value.status == 5
        assert done.tolist() == [[1, 0], [0, 0]]
        assert np.array_equal(out, first)   # nothing outside the finished tile was written
        assert np.all(out[:, 4:, :] == 0) and np.all(out[:, :, 4:] == 0)
        assert g.inelastic_map_tiles_for(ctx, sm, wl, tile, out, done, "tf32") == 0
    finally:
        _reset(ctx)
    assert _close(out, full)


CHILD = r"""
import sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import paper_1908_07628_gb300 as g
from test_gpu_scan_tiles import _workload
wl = _workload()
ctx = g.Context(0)
ctx.set_association("probe_first")
ctx.set_tile_width(256)
sm = g.build_smatrix_for(ctx, wl)
_, left = g.resumable_map(ctx, sm, wl, (2, 3), {path!r}, "tf32", max_tiles=2)
assert left == 10, left
"""


def test_checkpoint_file_resumes_after_the_process_exits(g, ctx):
    wl = _workload()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "map.npz")
        code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), path=path)
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True,
                           text=True, timeout=600)
        assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
        with np.load(path) as z:
            assert int(z["done"].sum()) == 2
        sm = g.build_smatrix_for(ctx, wl)
        _fixed(ctx, "probe_first")
        try:
            out, left = g.resumable_map(ctx, sm, wl, (2, 3), path, "tf32")
            full = g.inelastic_map_for(ctx, sm, wl, "tf32")
        finally:
            _reset(ctx)
        assert left == 0
        assert _close(out, full), np.abs(out - full).max() / full.max()
        other = _workload()
        other.scan = (6,) + tuple(other.scan[1:])
        with pytest.raises(ValueError):
            g.resumable_map(ctx, sm, other, (2, 3), path, "tf32")


def test_tile_arguments_are_checked(g, ctx):
    wl = _workload()
    sm = g.build_smatrix_for(ctx, wl)
    out = np.zeros((wl.n_types, wl.scan[1], wl.scan[0]))
    with pytest.raises(ValueError):
        g.inelastic_map_tiles_for(ctx, sm, wl, (0, 2), out, np.zeros(4, np.uint8))
    with pytest.raises(TypeError):
        g.inelastic_map_tiles_for(ctx, sm, wl, (4, 4), out, np.zeros(3, np.uint8))
    with pytest.raises(TypeError):
        g.inelastic_map_tiles_for(ctx, sm, wl, (4, 4), out.astype(np.float32),
                                  np.zeros(4, np.uint8))
