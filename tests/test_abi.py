"""The C-ABI library loads, exports every declared entry point, and its host-only
helpers agree with the oracle and with the paper's printed memory example.
No GPU needed (no compute call is made)."""
import json
import os
import re

import numpy as np
import pytest

import specimen as sp
from oracle import multislice as ms

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stem_eels.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1908_07628_gb300 import build
    build.build()
    import paper_1908_07628_gb300 as g
    return g


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(eels_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_three_calls_of_the_method():
    syms = declared_symbols()
    for name in ("eels_build_smatrix", "eels_inelastic_map", "eels_quadratic_reference_map"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(so, name), name
    assert set(declared_symbols()) == set(lib.EXPORTS)


def test_checked_build_compiles_and_exports_the_same_symbols(lib):
    """The bounds-checked variant (-DSTEM_CHECK) builds beside the normal library, says so
    through eels_checked_build, and exports every declared entry point; the normal
    library says it is not checked."""
    import ctypes
    from paper_1908_07628_gb300 import build
    path = build.build(check=True)
    assert path == build.lib_path(True) and path != lib.LIB_PATH
    checked, normal = ctypes.CDLL(path), ctypes.CDLL(lib.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(checked, name), name
    assert checked.eels_checked_build() == 1 and normal.eels_checked_build() == 0


def test_beam_counts_match_oracle_enumeration(lib):
    """Integer work: the library's aperture enumeration equals the oracle's exactly."""
    for (n, L, f, ang) in [(128, 8.6, 1, 0.02), (128, 8.6, 1, 0.03), (512, 34.4, 2, 0.02),
                           (512, 34.4, 2, 0.03), (768, 51.6, 2, 0.03), (1024, 100.0, 4, 0.02),
                           (1024, 100.0, 4, 0.03), (64, 6.0, 3, 0.05)]:
        try:
            ref = ms.lattice_beams(n, L, 0.02508, f, ang)[0].size
        except ValueError:
            continue
        assert lib.count_beams(n, L, 0.02508, f, ang) == ref


def test_memory_model_reproduces_paper_example(lib):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_memory_example.json")))
    conv, trans, smat = lib.memory_model(g["grid"], g["n_slices"], g["planes_s1"], g["planes_s2"])
    assert int(conv / 1e6) == g["conventional_minimum_MB"]
    assert round(trans / 1e9, 2) == g["transmission_GB"]
    assert round(smat / 1e9, 2) == g["smatrix_GB"]


def test_footprint_counts_stored_smatrix_and_one_sout_depth(lib):
    n, nz, nin, nout, chunk = 512, 40, 593, 1321, 64
    plane = 8 * (n // 2) ** 2
    expect = 8 * nz * n * n + plane * (nz * nin + nout) + 2 * 8 * chunk * n * (n // 2)
    assert lib.footprint_bytes(n, nz, nin, nout, chunk) == expect
    assert lib.footprint_bytes(-2, nz, nin, nout, chunk) == -1


def test_workload_beam_counts():
    wl = sp.rocksalt_small()
    assert ms.lattice_beams(wl.n, wl.cell, wl.lam, wl.f, wl.alpha)[0].size == 145
    assert ms.lattice_beams(wl.n, wl.cell, wl.lam, wl.f, wl.beta)[0].size == 333


def test_request_footprint_with_s_in_checkpoints(lib):
    """Host-only footprint model of the map server: S_in at every depth versus
    checkpoints every K slices (probe waves as N x N/2 row spectra) plus one recomputed
    segment and the forward work arrays during the map."""
    import ctypes
    import math
    req = {"n": 1024, "n_z": 120, "cell": 68.8, "f": 2}
    H = np.zeros((1, 2, 32, 32), np.complex64)
    vproj = np.zeros((req["n_z"], 8, 8), np.float32)   # only the pointer and n_z are read
    r, keep = lib.make_request(vproj, req["cell"], 0.02508, 7.29e-4, 2.15, req["f"], 0.02, H,
                               np.zeros(1, np.int32), np.zeros(1, np.int32),
                               np.zeros(1, np.int32), np.zeros(1), np.zeros(1),
                               (16, 16, 0.0, 0.0, 0.1, 0.1), 0.03)
    r.spec.n = req["n"]
    n, nz = req["n"], req["n_z"]
    n_in = lib.count_beams(n, req["cell"], 0.02508, req["f"], 0.02)
    n_out = lib.count_beams(n, req["cell"], 0.02508, req["f"], 0.03)
    c, nn, plane, wave = 8, n * n, (n // 2) ** 2 * 8, 8 * n * (n // 2)
    h = 1 * 2 * 32 * 32 * 8
    cap = 4 << 30
    whole = lib.request_footprint(r)
    expect_whole = (c * nz * nn + plane + nz * n_in * plane +
                    max(2 * n_in * wave + 4 * nz * nn,
                        2 * n_out * wave + n_out * plane + cap + h))
    assert whole == expect_whole
    k = math.ceil(math.sqrt(2 * nz))
    r.sin_checkpoint = k
    ck = lib.request_footprint(r)
    expect_ck = (c * nz * nn + plane + math.ceil(nz / k) * n_in * wave +
                 max(2 * n_in * wave + 4 * nz * nn,
                     2 * n_out * wave + n_out * plane + cap + h + 2 * n_in * wave +
                     k * n_in * plane))
    assert ck == expect_ck
    assert ck < whole / 2.5          # the largest request of the mixed stream fits in HBM
    del keep
