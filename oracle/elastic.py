"""Elastic STEM images from the same calculation: annular dark field and incoherent
bright field, and the bright-field-divided EELS map (Sec. IV D).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. IV D forms, next to the EELS map, an ADF image (detector inner angle 60 mrad)
and an incoherent bright-field image whose detector has the angular extent of the
EELS aperture, and divides the EELS map by the latter.  The paper gives no formula;
the reading here (PRISM, Sec. III and Sec. IV D):

* the elastic exit wave of probe R is the conventional multislice result
  psi_R(exit) = A_{n_z-1} ... A_0 psi_R(0) with the probe of Eq. illum on the f-lattice
  (f^2 periodic images, each of unit norm);
* as in PRISM, it is cut to the L/f cell around R: the pixels of the N/2 grid (where
  the S-matrices live) whose minimum-image offset from R lies in [-L/2f, L/2f) on both
  axes, the half-open rule the EELS window uses for sites; that is M = N/(2f) pixels
  per axis, starting at the in-rule pixel whose cyclic predecessor is out of rule (at
  f = 1 every pixel is in rule and the cut is the whole cell, started at pixel 0);
* the detector integrates |.|^2 over the cut wave's own DFT lattice, k = f(a, b)/L:
  I_D(R) = 4 sum_{k in D} |DFT_unitary(cut)(k)|^2 = (16 f^2 / N^2) sum_{k in D} |sum_p
  cut(p) exp(-2 pi i k.x_p)|^2, which equals the EELS detector's f^2 sum over f-lattice
  beams for a wave that lies inside the cut;
* a detector D = {k : inner <= lambda |k| <= outer} (outer <= 0: no outer edge), always
  inside the band limit 16 f^2 (a^2 + b^2) < N^2 of the calculation.

The ADF detector of Sec. IV D is (0.060, 0); the incoherent bright field is (0, beta).
"""
from __future__ import annotations

import math

import numpy as np

from . import linear as lin
from . import multislice as ms


def window_start(nh: int, cell: float, f: int, r: float) -> int:
    """First pixel of the L/f cut around r on one axis of the N/2 grid."""
    x = np.arange(nh) * (cell / nh)
    ok = ms.axis_in_window(x, r, cell, f)
    if ok.all():            # f = 1: the whole cell (a cyclic shift leaves |DFT| unchanged)
        return 0
    starts = np.nonzero(ok & ~np.roll(ok, 1))[0]
    if starts.size != 1:
        raise ValueError("the cut is not one cyclic run of pixels")
    return int(starts[0])


def detector_mask(m: int, n: int, cell: float, lam: float, f: int, inner: float,
                  outer: float) -> np.ndarray:
    """bool [M][M] over the cut's DFT bins (numpy FFT order, [ky][kx])."""
    a = ms.fft_index(m)
    ka = a[None, :]
    kb = a[:, None]
    k = f * np.sqrt((ka * ka + kb * kb).astype(np.float64)) / cell
    band = 16 * f * f * (ka * ka + kb * kb) < n * n
    mask = band & (lam * k >= inner)
    if outer > 0:
        mask &= lam * k <= outer
    return mask


def _images_of_exit(dec_exit, wl, detectors, rx_i, ry_i):
    """I_D for one probe from its decimated exit wave (true scale)."""
    n, f = wl.n, wl.f
    nh = n // 2
    if nh % f:
        raise ValueError("the L/f cut needs N/2 divisible by f")
    m = nh // f
    x0 = window_start(nh, wl.cell, f, rx_i)
    y0 = window_start(nh, wl.cell, f, ry_i)
    rows, cols = ms.window_indices(nh, x0, y0, m)
    cut = dec_exit[np.ix_(rows, cols)]
    spec = np.abs(np.fft.fft2(cut)) ** 2
    out = []
    for inner, outer in detectors:
        mask = detector_mask(m, n, wl.cell, wl.lam, f, inner, outer)
        out.append(16.0 * f * f / (n * n) * float(np.sum(spec[mask])))
    return out


def quadratic_images(wl, detectors, positions=None):
    """Definition: each probe carried through all slices by multislice (Alg. 1 without
    ionisation), then cut and detected.  float64 [n_det][n_sy][n_sx]."""
    n, L = wl.n, wl.cell
    P = ms.propagator(n, L, wl.lam, wl.dz)
    ts = [ms.transmission(wl.vproj[i], wl.sigma) for i in range(wl.n_z)]
    rx, ry = wl.scan_positions()
    out = np.zeros((len(detectors), wl.scan[1], wl.scan[0]))
    pos = positions if positions is not None else [
        (iy, ix) for iy in range(wl.scan[1]) for ix in range(wl.scan[0])]
    for iy, ix in pos:
        psi = ms.probe(n, L, wl.lam, wl.f, wl.alpha, rx[ix], ry[iy])
        for t in ts:
            psi = ms.slice_step(psi, t, P)
        out[:, iy, ix] = _images_of_exit(ms.decimate(psi), wl, detectors, rx[ix], ry[iy])
    return out


def exit_s_matrix(wl):
    """Decimated exit waves of the probe beams, complex128 [n_in][N/2][N/2], and beams."""
    n, L, f = wl.n, wl.cell, wl.f
    beams = ms.lattice_beams(n, L, wl.lam, f, wl.alpha)
    P = ms.propagator(n, L, wl.lam, wl.dz)
    psi = lin.plane_waves(n, beams, f)
    for i in range(wl.n_z):
        psi = np.fft.ifft2(P[None] * np.fft.fft2(ms.transmission(wl.vproj[i], wl.sigma)[None]
                                                   * psi))
    return ms.decimate(psi), beams


def linear_images(wl, detectors):
    """PRISM form: psi_R(exit) = sum_j a_j(R) S_exit[j] (Sec. III), then cut and detected."""
    s_exit, beams = exit_s_matrix(wl)
    rx, ry = wl.scan_positions()
    a = lin.probe_coefficients(wl, beams, rx, ry)
    out = np.zeros((len(detectors), wl.scan[1], wl.scan[0]))
    for iy in range(wl.scan[1]):
        for ix in range(wl.scan[0]):
            dec = np.tensordot(a[:, iy, ix], s_exit, axes=(0, 0))
            out[:, iy, ix] = _images_of_exit(dec, wl, detectors, rx[ix], ry[iy])
    return out


def bf_corrected(eels_map, bf):
    """EELS map divided by the incoherent bright-field image (Sec. IV D), per channel."""
    return eels_map / bf[None]
