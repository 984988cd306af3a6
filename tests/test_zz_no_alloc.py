"""The allocation-free S_in build (eels_build_smatrix_static) against eels_build_smatrix.

Callers that cannot allocate device memory (plug-ins inside a host application that
owns the memory pool, real-time loops that must not risk an allocation failure) use
the static entry point; it must store the same S_in as the regular build.  The
512^2 case has more probe beams than one chunk of the static work array holds, so
the beam offsets of later chunks and their restart at the entrance plane are
exercised too.  Two calls in a
row check that whatever the first call leaves in the shared static work array
does not leak into the second.  This file sorts last so that a failure here
leaves every other test already run.
"""
import numpy as np
import pytest

import specimen as sp

pytestmark = pytest.mark.gpu

TOL = 1e-5   # same bound as the S-matrix parity test


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_07628_gb300 import build
    build.build()
    import paper_1908_07628_gb300 as pkg
    return pkg


STATIC_BYTES = 64 << 20   # EELS_STATIC_SCRATCH_BYTES


@pytest.mark.parametrize("which", ["random64_f2", "rocksalt_small", "random256_f2_host",
                                   "random512_f2_chunks"])
def test_static_build_matches_allocating_build(g, which):
    import torch
    if which == "rocksalt_small":
        wl = sp.rocksalt_small()
    elif which == "random64_f2":
        wl = sp.random_workload(n=64, n_z=5, f=2, cell=6.4, n_sites=3, w=8, seed=31,
                                alpha=0.02, beta=0.03, dz=1.8)
    elif which == "random512_f2_chunks":
        wl = sp.random_workload(n=512, n_z=3, f=2, cell=12.8, n_sites=3, w=8, seed=33,
                                alpha=0.02, beta=0.03, dz=1.8)
    else:
        wl = sp.random_workload(n=256, n_z=3, f=2, cell=12.8, n_sites=3, w=8, seed=32,
                                alpha=0.02, beta=0.03, dz=1.8)
    ctx = g.Context(0)
    sm = g.build_smatrix_for(ctx, wl)
    nh = wl.n // 2
    if which == "random512_f2_chunks":
        # one chunk holds at most STATIC_BYTES / (two N x N/2 complex64 waves) beams
        assert sm.n_in > 2 * (STATIC_BYTES // (2 * wl.n * nh * 8)), sm.n_in
    ref = torch.empty((wl.n_z, sm.n_in, nh, nh), dtype=torch.complex64, device="cuda")
    for i in range(wl.n_z):
        sm.copy_depth(i, ref[i])
    vproj = wl.vproj if which.endswith("host") else torch.from_numpy(wl.vproj).cuda()
    for call in range(2):
        out = torch.full((wl.n_z, sm.n_in, nh, nh), complex(float("nan"), 0.0),
                         dtype=torch.complex64, device="cuda")
        n_in = g.build_smatrix_static(vproj, wl.cell, wl.lam, wl.sigma, wl.dz, wl.f, wl.alpha, out)
        torch.cuda.synchronize()
        assert n_in == sm.n_in
        err = (torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref)).item()
        assert np.isfinite(err) and err < TOL, (call, err)


def test_static_build_rejects_a_too_small_output_buffer(g):
    import torch
    wl = sp.rocksalt_small()
    small = torch.empty(16, dtype=torch.complex64, device="cuda")
    with pytest.raises(g.EelsError) as e:
        g.build_smatrix_static(wl.vproj, wl.cell, wl.lam, wl.sigma, wl.dz, wl.f, wl.alpha, small)
    assert e.value.status == 1 and "needs" in str(e.value)
    big = np.zeros((1, 1024, 1024), np.float32)
    out = torch.empty(1 << 20, dtype=torch.complex64, device="cuda")   # 1245 beams need 2.6 GB
    with pytest.raises(g.EelsError) as e:
        g.build_smatrix_static(big, 100.0, 0.02508, 7.3e-4, 2.0, 4, 0.02, out)
    assert e.value.status == 1 and "needs" in str(e.value)
