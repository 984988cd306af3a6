"""Conventional (quadratic) STEM-EELS multislice in FP64 -- the definition.

TEST INFRASTRUCTURE ONLY (see the package docstring): nothing in the CUDA
library imports or calls this module.

Conventions (the paper fixes the physics; where it is silent the reading taken
is stated here):

* Grid: N x N pixels over an L x L cell; arrays are [y][x].  Signed frequency
  indices p, q in FFT order; k = (p/L, q/L).  Forward transform uses
  exp(-2 pi i r.g) (Sec. II, footnote to Eq. 4).  Unitary normalisation.
* Slice operator (Eq. MSop): A_i psi = F^-1[ P . F[ t_i . psi ] ] with the
  transmission function t_i = exp(i sigma v_i(r)) (Eq. 3-4) and the Fresnel
  propagator P(k) = B(k) exp(-i pi lambda dz |k|^2); B is the band limit to
  half the array (Sec. III, below Eq. TPRISM1): B = 1 iff p^2 + q^2 < (N/4)^2.
* Probe (Eq. illum, chi = 0): psi_R = c sum_j exp(-2 pi i k_j.R) |k_j>, with
  k_j = f(p, q)/L on the PRISM interpolation lattice inside the aperture
  lambda |k| <= alpha (Sec. III, "the natural reciprocal space sampling ... L/f"),
  |k> the unit-norm plane wave, c = f / sqrt(n_in) so that each of the f^2
  periodic images of the probe carries unit norm.
* Ionisation (Eq. Hn0Psi): the transition potential H_n0 and t_i are both
  diagonal in real space, so they commute; the inelastic wave of a site in
  slice i is formed from the transmitted wave t_i psi_i on the half-resolution
  grid that the paper stores its scattering matrices on (Sec. III, "side-length
  of N/2"): x = H . Dec(t_i psi_i) inside the site's w x w window, zero outside,
  then Fourier-interpolated back to N x N (Interp), and the slice is finished
  by the propagator.
* Detection (first listing, "integrate over the detector"): with interpolation
  factor f the detector integral is sampled on the same f-lattice:
  I(R) += f^2 sum_{lambda |k_d| <= beta} |<k_d| psi_exit>|^2.
* PRISM window: a site contributes to I(R) iff the minimum-image displacement
  r_s - R lies in [-L/(2f), L/(2f)) along both axes (each probe of the
  interpolated S-matrix lives in an L/f cell).  At f = 1 every site counts.
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------------------
# grid, band limit, beam lists
# ---------------------------------------------------------------------------

def fft_index(n: int) -> np.ndarray:
    """Signed integer frequency index of each FFT bin: 0..N/2-1, -N/2..-1."""
    i = np.arange(n)
    return np.where(i < n - n // 2, i, i - n).astype(np.int64)


def band_limit(n: int) -> np.ndarray:
    """B(k): 1 inside p^2 + q^2 < (N/4)^2 (integer test, exact), else 0. [y][x]."""
    p = fft_index(n)
    return 16 * (p[None, :] ** 2 + p[:, None] ** 2) < n * n


def propagator(n: int, cell: float, lam: float, dz: float) -> np.ndarray:
    """P(k) = B(k) exp(-i pi lambda dz |k|^2), Eq. MSop, in FP64."""
    p = fft_index(n).astype(np.float64)
    k2 = (p[None, :] ** 2 + p[:, None] ** 2) / (cell * cell)
    return band_limit(n) * np.exp(-1j * math.pi * lam * dz * k2)


def transmission(v_slice: np.ndarray, sigma: float) -> np.ndarray:
    """t_i(r) = exp(i sigma v_i(r)) (Eq. 3-4)."""
    return np.exp(1j * sigma * v_slice.astype(np.float64))


def lattice_beams(n: int, cell: float, lam: float, f: int, angle: float):
    """Integer pairs (p, q) of the f-lattice points k = f(p,q)/L with lambda|k| <= angle.

    Sec. III: the aperture covers pi alpha^2 of reciprocal space, sampled with
    pitch f/L.  Returned in row-major (q, then p) order.  Every beam must lie
    strictly inside the band limit so that the plane wave is a valid
    band-limited wave.
    """
    pmax = int(math.ceil(angle * cell / (lam * f))) + 1
    ps, qs = [], []
    for q in range(-pmax, pmax + 1):
        for p in range(-pmax, pmax + 1):
            if lam * f * math.sqrt(p * p + q * q) / cell <= angle:
                ps.append(p)
                qs.append(q)
    ps = np.array(ps, dtype=np.int64)
    qs = np.array(qs, dtype=np.int64)
    if ps.size and np.any(16 * f * f * (ps * ps + qs * qs) >= n * n):
        raise ValueError("aperture extends beyond the band limit of the grid")
    return ps, qs


# ---------------------------------------------------------------------------
# operators
# ---------------------------------------------------------------------------

def slice_step(psi: np.ndarray, t: np.ndarray, P: np.ndarray) -> np.ndarray:
    """One multislice iteration, Eq. MSop: transmit through t, then propagate."""
    return np.fft.ifft2(P * np.fft.fft2(t * psi))


def propagate(psi: np.ndarray, P: np.ndarray) -> np.ndarray:
    """Fresnel propagation by one slice thickness (second half of Eq. MSop)."""
    return np.fft.ifft2(P * np.fft.fft2(psi))


def decimate(x: np.ndarray) -> np.ndarray:
    """Samples at even pixels: the N/2 representation of a band-limited wave."""
    return x[..., ::2, ::2]


def interpolate(xh: np.ndarray, n: int) -> np.ndarray:
    """Fourier interpolation from the N/2 grid back to N: zero-pad the spectrum.

    The N/2-grid spectrum (bins -N/4..N/4-1) is placed at the same signed
    frequencies of the N grid.  The factor 4 makes decimate(interpolate(x)) == x.
    """
    nh = n // 2
    X = np.fft.fft2(xh)
    Y = np.zeros(xh.shape[:-2] + (n, n), dtype=np.complex128)
    ph = fft_index(nh) % n
    Y[..., ph[:, None], ph[None, :]] = X
    return 4.0 * np.fft.ifft2(Y)


def window_indices(nh: int, x0: int, y0: int, w: int):
    """Row and column indices of a w x w window of the N/2 grid (periodic)."""
    return (y0 + np.arange(w)) % nh, (x0 + np.arange(w)) % nh


def ionise(alpha: np.ndarray, Hw: np.ndarray, x0: int, y0: int) -> np.ndarray:
    """Eq. Hn0Psi on the N/2 grid: H . Dec(alpha) inside the window, 0 outside."""
    n = alpha.shape[-1]
    nh = n // 2
    w = Hw.shape[-1]
    if w > nh:
        raise ValueError("transition window larger than the N/2 grid")
    rows, cols = window_indices(nh, x0, y0, w)
    d = decimate(alpha)
    x = np.zeros((nh, nh), dtype=np.complex128)
    x[np.ix_(rows, cols)] = Hw.astype(np.complex128) * d[np.ix_(rows, cols)]
    return x


def axis_in_window(s, r, cell: float, f: int):
    """PRISM window test along one axis: minimum-image s - r in [-L/(2f), L/(2f))."""
    d = s - r
    d = d - cell * np.floor(d / cell + 0.5)
    h = cell / (2 * f)
    return (d >= -h) & (d < h)


def probe(n: int, cell: float, lam: float, f: int, alpha: float, rx: float, ry: float,
          beams=None) -> np.ndarray:
    """Real-space STEM probe at R = (rx, ry), Eq. illum with chi = 0 on the f-lattice."""
    bp, bq = lattice_beams(n, cell, lam, f, alpha) if beams is None else beams
    c = f / math.sqrt(bp.size)
    Psi = np.zeros((n, n), dtype=np.complex128)
    phase = -2.0 * math.pi * f * (bp * rx + bq * ry) / cell
    Psi[(f * bq) % n, (f * bp) % n] = c * np.exp(1j * phase)
    return np.fft.ifft2(Psi, norm="ortho")


def detect(psi: np.ndarray, f: int, det_beams) -> float:
    """f^2 sum over detector beams of |<k_d|psi>|^2 (the detector integral)."""
    n = psi.shape[-1]
    dp, dq = det_beams
    c = np.fft.fft2(psi, norm="ortho")[(f * dq) % n, (f * dp) % n]
    return float(f * f * np.sum(np.abs(c) ** 2))


# ---------------------------------------------------------------------------
# the conventional algorithm (Sec. III, first listing)
# ---------------------------------------------------------------------------

def quadratic_map(wl, positions=None, counter=None):
    """Conventional quadratic STEM-EELS map.

    For every probe position: advance the elastic wave slice by slice; at each
    slice form the inelastic wave of every transition of the sites in that
    slice (inside the probe's PRISM window), propagate it to the exit surface
    with the multislice operator and add its detector integral to the map.

    positions: optional list of (iy, ix) scan indices to evaluate (others stay 0).
    counter:   optional dict; counter["steps"] accumulates multislice operations
               per the paper's count (n_z - i per transition in slice i, plus n_z
               for the elastic wave).
    Returns I float64 [n_types][n_sy][n_sx].
    """
    n, L, n_z, f = wl.n, wl.cell, wl.n_z, wl.f
    T = wl.n_types
    n_sx, n_sy = wl.scan[0], wl.scan[1]
    t = [transmission(wl.vproj[i], wl.sigma) for i in range(n_z)]
    P = propagator(n, L, wl.lam, wl.dz)
    probe_beams = lattice_beams(n, L, wl.lam, f, wl.alpha)
    det_beams = lattice_beams(n, L, wl.lam, f, wl.beta)
    rx, ry = wl.scan_positions()
    by_slice = [np.nonzero(wl.site_slice == i)[0] for i in range(n_z)]
    if positions is None:
        positions = [(iy, ix) for iy in range(n_sy) for ix in range(n_sx)]
    I = np.zeros((T, n_sy, n_sx))
    steps = 0
    for iy, ix in positions:
        psi = probe(n, L, wl.lam, f, wl.alpha, rx[ix], ry[iy], probe_beams)
        for i in range(n_z):
            alpha = t[i] * psi
            for s in by_slice[i]:
                if not (axis_in_window(wl.site_x[s], rx[ix], L, f)
                        and axis_in_window(wl.site_y[s], ry[iy], L, f)):
                    continue
                for m in range(T):
                    y = interpolate(ionise(alpha, wl.H[s, m], wl.win_x0[s], wl.win_y0[s]), n)
                    y = propagate(y, P)
                    for i2 in range(i + 1, n_z):
                        y = slice_step(y, t[i2], P)
                    I[m, iy, ix] += detect(y, f, det_beams)
                    steps += n_z - i
            psi = propagate(alpha, P)
            steps += 1
    if counter is not None:
        counter["steps"] = counter.get("steps", 0) + steps
    return I


def relative_error(ref: np.ndarray, test: np.ndarray) -> float:
    """Normalised RMS error, Eq. nrmsse read as sqrt(sum (I_ref - I)^2 / sum I_ref^2)."""
    ref = np.asarray(ref, dtype=np.float64)
    test = np.asarray(test, dtype=np.float64)
    return float(np.sqrt(np.sum((ref - test) ** 2) / np.sum(ref ** 2)))
