"""The bounds-checked debug build (-DSTEM_CHECK) on the GPU.

In that build every kernel that derives an index from a device list (window origins,
beam columns, scan indices, transition types, the persistent GEMMs' tile decode and TMA
box coordinates) checks it first, records a violation in its unit's flag, skips the
access, and the call returns EELS_ERR_BOUNDS.  Checked here, in a child process that
loads the checked library (STEM_CHECK=1 selects it at import):

* valid inputs raise no check, and the maps, the quadratic baseline and the elastic
  images still match the FP64 oracle;
* EELS_OPT_CHECK_TEST gives the first site that some probe reaches the window origin N/2,
  one past its range (a walk from there still stays inside the plane, so nothing is read
  out of bounds even if a check were missing): every precision and grouping reports
  EELS_ERR_BOUNDS, and the same context maps correctly afterwards;
* the normal build refuses the test option (EELS_ERR_UNSUPPORTED).
"""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

import specimen as sp
from oracle import elastic as el
from oracle import multislice as ms

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EPS = {"fp32": 1e-4, "tf32": 1e-4, "bf16x3": 1e-3}
VARIANTS = [("fp32", "auto"), ("tf32", "transition_first"), ("tf32", "probe_first"),
            ("bf16x3", "transition_first"), ("bf16x3", "probe_first")]


def _workload():
    return sp.random_workload(n=128, n_z=4, f=2, cell=128 * 0.05, n_sites=8, w=20, seed=6,
                              scan_n=3, n_types=2, alpha=0.02, beta=0.03, dz=1.8)


def _dets(wl):
    return [(0.0, wl.beta), (0.6 * wl.lam * wl.n / (4 * wl.cell), 0.0)]


CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import paper_1908_07628_gb300 as g
from test_gpu_checked_build import VARIANTS, _dets, _workload

assert g.checked_build(), "the checked library was not loaded"
wl = _workload()
ctx = g.Context(0)
ctx.set_exit_plane(True)
sm = g.build_smatrix_for(ctx, wl)
out = {{}}
for prec, assoc in VARIANTS:
    ctx.set_association(assoc)
    out["map_%s_%s" % (prec, assoc)] = g.inelastic_map_for(ctx, sm, wl, prec)
ctx.set_association("auto")
out["quadratic"], _ = g.quadratic_reference_map_for(ctx, wl)
out["elastic"] = ctx.elastic_images(sm, wl.scan, _dets(wl))
ctx.set_check_test(1)
statuses, messages = [], []
for prec, assoc in VARIANTS:
    ctx.set_association(assoc)
    try:
        g.inelastic_map_for(ctx, sm, wl, prec)
        statuses.append(0)
        messages.append("")
    except g.EelsError as e:
        statuses.append(e.status)
        messages.append(str(e))
ctx.set_check_test(0)
ctx.set_association("probe_first")
out["after"] = g.inelastic_map_for(ctx, sm, wl, "tf32")
np.savez({path!r}, statuses=np.array(statuses), messages=np.array(messages), **out)
"""


@pytest.fixture(scope="module")
def checked_results():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_07628_gb300 import build
    build.build(check=True)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "checked.npz")
        env = dict(os.environ, STEM_CHECK="1")
        code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), path=path)
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env,
                           capture_output=True, text=True, timeout=900)
        assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
        with np.load(path) as z:
            return {k: z[k] for k in z.files}


def test_checked_build_raises_no_check_on_valid_inputs(checked_results):
    wl = _workload()
    ref = ms.quadratic_map(wl)
    assert ref.max() > 0
    for prec, assoc in VARIANTS:
        got = checked_results["map_%s_%s" % (prec, assoc)]
        assert ms.relative_error(ref, got) < EPS[prec], (prec, assoc)
    assert ms.relative_error(ref, checked_results["quadratic"]) < EPS["fp32"]
    dets = _dets(wl)
    eref = el.quadratic_images(wl, dets)
    for d in range(len(dets)):
        assert ms.relative_error(eref[d], checked_results["elastic"][d]) < EPS["fp32"], d


def test_bad_window_origin_is_reported_and_context_recovers(checked_results):
    statuses = checked_results["statuses"].tolist()
    messages = checked_results["messages"].tolist()
    assert statuses == [8] * len(VARIANTS), list(zip(statuses, messages))
    assert all("bounds check" in m for m in messages), messages
    ref = ms.quadratic_map(_workload())
    assert ms.relative_error(ref, checked_results["after"]) < EPS["tf32"]


def test_normal_build_refuses_the_check_test_option():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_07628_gb300 import build
    build.build()
    import paper_1908_07628_gb300 as g
    assert not g.checked_build()
    ctx = g.Context(0)
    with pytest.raises(g.EelsError) as e:
        ctx.set_check_test(1)
    assert e.value.status == 2
