"""Pins of the elastic-image oracle (ADF / incoherent BF of Sec. IV D) against things
other than itself: closed forms in free space, the EELS detector's f-lattice sum, the
EELS aperture's beam count and the conventional multislice definition."""
import math

import numpy as np
import pytest

import specimen as sp
from oracle import elastic as el
from oracle import linear as lin
from oracle import multislice as ms


def _tiny(n, f, cell, seed, alpha=0.02, beta=0.03, n_z=3, scan_n=3):
    return sp.random_workload(n=n, n_z=n_z, f=f, cell=cell, n_sites=2, w=6, seed=seed,
                              alpha=alpha, beta=beta, dz=1.5, scan_n=scan_n)


def test_free_space_bright_field_is_one_and_dark_field_is_zero():
    """v = 0, f = 1: the exit wave is the aperture-limited probe with propagator phases
    only, so a detector covering the probe aperture collects exactly the probe's unit
    intensity and an annulus outside it collects nothing."""
    wl = _tiny(32, 1, 6.0, 3)
    wl.vproj = np.zeros_like(wl.vproj)
    img = el.quadratic_images(wl, [(0.0, wl.beta), (1.2 * wl.alpha, 0.0)])
    assert np.allclose(img[0], 1.0, rtol=0, atol=1e-12)
    assert np.abs(img[1]).max() < 1e-24


def test_cut_detector_equals_f_lattice_detector_for_a_localised_wave():
    """A band-limited wave well inside the L/f cell around R: the cut-and-DFT detector
    equals f^2 times the sum over f-lattice beams of |<k|psi>|^2 on the full grid (the
    EELS detector integral, computed here by a full-grid FFT)."""
    n, f, cell = 128, 2, 25.6
    wl = _tiny(n, f, cell, 5, beta=0.03)
    rx, ry = 9.3, 14.1
    x = np.arange(n) * cell / n
    dx = x[None, :] - rx
    dy = x[:, None] - ry
    # width 1 A: tails at the cut edge (6.4 A away) ~ e^-20; spectrum at the band edge ~ e^-15
    g = np.exp(-(dx ** 2 + dy ** 2) / 2.0) * np.exp(2j * math.pi * (0.3 * dx - 0.2 * dy))
    psi = np.fft.ifft2(np.fft.fft2(g) * ms.band_limit(n))
    det = ms.lattice_beams(n, cell, wl.lam, f, wl.beta)
    want = ms.detect(psi, f, det)
    got = el._images_of_exit(ms.decimate(psi), wl, [(0.0, wl.beta)], rx, ry)[0]
    assert want > 1e-3
    assert abs(got - want) < 1e-9 * want


@pytest.mark.parametrize("n,f,cell", [(64, 1, 6.4), (128, 2, 12.8), (96, 3, 15.0)])
def test_bright_field_detector_is_the_eels_aperture(n, f, cell):
    lam, beta = sp.LAM_200KEV, 0.03
    m = n // 2 // f
    mask = el.detector_mask(m, n, cell, lam, f, 0.0, beta)
    assert mask.sum() == ms.lattice_beams(n, cell, lam, f, beta)[0].size


def test_cut_is_centred_on_the_probe():
    """For R = (p + 0.3) h (h the N/2-grid pixel) the cut [R - L/2f, R + L/2f) holds the
    pixels p - M/2 + 1 .. p + M/2 (no pixel is at a tie)."""
    nh, cell, f = 64, 12.8, 2
    h = cell / nh
    m = nh // f
    for p in (0, 5, 40, 63):
        assert el.window_start(nh, cell, f, (p + 0.3) * h) == (p - m // 2 + 1) % nh


@pytest.mark.parametrize("n,f,cell,seed", [(32, 1, 6.0, 1), (64, 2, 12.0, 2)])
def test_prism_images_equal_the_conventional_definition(n, f, cell, seed):
    """S_in at the exit surface applied to the probe coefficients reproduces the probe
    carried through every slice (the linearity the S-matrix rests on, Sec. III)."""
    wl = _tiny(n, f, cell, seed)
    dets = [(0.0, wl.beta), (0.025, 0.0), (0.010, 0.025)]   # band edge here is 33 mrad
    q = el.quadratic_images(wl, dets)
    p = el.linear_images(wl, dets)
    assert q.min() >= 0 and q[0].max() > 0 and q[1].max() > 0
    assert ms.relative_error(q, p) < 1e-12


def test_bf_division_is_per_channel_ratio():
    m = np.arange(12.0).reshape(2, 2, 3) + 1
    bf = np.array([[1.0, 2.0, 4.0], [0.5, 0.25, 8.0]])
    out = el.bf_corrected(m, bf)
    assert np.array_equal(out[1, 1, 2] * bf[1, 2], m[1, 1, 2])
