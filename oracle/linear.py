"""Scattering-matrix (PRISM-EELS) map in FP64, exact store-and-stream form.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. III, second listing: S_1 carries the plane waves of the probe aperture
forward to the ionisation depth, S_2 carries the plane waves of the EELS
aperture backwards from the exit surface with the transpose operator
(Eq. MSTop), and each transition contributes |S_n psi|^2 with
S_n = S_2 F H_n0 F^-1 S_1 (Eq. SHn0).

Here S_1 = S_in is stored at every depth; S_2 is produced by the adjoint step
A_i^dagger = conj(t_i) F^-1 conj(P) F, which is the complex conjugate of the
paper's transpose operator and therefore gives the same |.|^2.  Because the
stored waves are band-limited, the contraction can run on the N/2 grid inside
the transition window without loss:

  <k_d| U Interp(x)> = 4 <Dec beta_d, x>_{N/2}

for beta_d band-limited (the product of two waves limited to |p| < N/4 has no
component at the N/2-grid Nyquist frequency).  So

  M_n[d, j] = sum_{p in W} conj(Sout[d, p]) H_n[p] Sin[j, p],   Sout = 4 Dec beta
  I(R) += f^2 sum_d | sum_j M_n[d, j] a_j(R) |^2,   a_j(R) = c exp(-2 pi i k_j.R)

which the paper states carries no error relative to the conventional
algorithm (Abstract; Sec. IV A).
"""
from __future__ import annotations

import math

import numpy as np

from . import multislice as ms


def plane_waves(n: int, beams, f: int) -> np.ndarray:
    """Unit-norm plane waves |k> for the given f-lattice beams, [beam][y][x]."""
    bp, bq = beams
    Psi = np.zeros((bp.size, n, n), dtype=np.complex128)
    Psi[np.arange(bp.size), (f * bq) % n, (f * bp) % n] = 1.0
    return np.fft.ifft2(Psi, norm="ortho")


def adjoint_step(beta: np.ndarray, t: np.ndarray, P: np.ndarray) -> np.ndarray:
    """Adjoint of one slice step A = F^-1 P F t: A^dagger = conj(t) . F^-1[conj(P) . F[beta]]."""
    return np.conj(t) * np.fft.ifft2(np.conj(P) * np.fft.fft2(beta))


def build_s_in(wl):
    """S_in at every depth: Dec(t_i psi_j(i)) for every probe beam j.

    psi_j(0) = |k_j>;  psi_j(i+1) = F^-1 P F (t_i psi_j(i)).
    Returns complex128 [n_z][n_in][N/2][N/2] and the beam list.
    """
    n, L, f = wl.n, wl.cell, wl.f
    beams = ms.lattice_beams(n, L, wl.lam, f, wl.alpha)
    P = ms.propagator(n, L, wl.lam, wl.dz)
    psi = plane_waves(n, beams, f)
    out = np.empty((wl.n_z, psi.shape[0], n // 2, n // 2), dtype=np.complex128)
    for i in range(wl.n_z):
        alpha = ms.transmission(wl.vproj[i], wl.sigma)[None] * psi
        out[i] = ms.decimate(alpha)
        psi = np.fft.ifft2(P[None] * np.fft.fft2(alpha))
    return out, beams


def _exit_detector_waves(wl, detectors):
    """beta_d(n_z-1) = F^-1 conj(P) F |k_d> for the EELS aperture's beams, and P."""
    n, L, f = wl.n, wl.cell, wl.f
    det = ms.lattice_beams(n, L, wl.lam, f, wl.beta)
    if detectors is not None:
        det = (det[0][detectors], det[1][detectors])
    P = ms.propagator(n, L, wl.lam, wl.dz)
    return np.fft.ifft2(np.conj(P)[None] * np.fft.fft2(plane_waves(n, det, f))), P


def _back_one_slice(beta, wl, P, i):
    """beta(i-1) = F^-1 conj(P) F (conj(t_i) beta(i)): one slice towards the entrance."""
    t = ms.transmission(wl.vproj[i], wl.sigma)
    return np.fft.ifft2(np.conj(P)[None] * np.fft.fft2(np.conj(t)[None] * beta))


def iter_s_out(wl, detectors=None):
    """Yield (i, Sout_i) for i = n_z-1 .. 0 with Sout_i = 4 Dec(beta_d(i)).

    beta_d(n_z-1) = F^-1 conj(P) F |k_d>;  beta_d(i-1) = F^-1 conj(P) F (conj(t_i) beta_d(i)),
    i.e. the detector plane waves carried back through slices n_z-1 .. i+1 and the
    propagation half of slice i.  `detectors` (indices into the aperture's beam
    list) keeps only those detector beams.
    """
    beta, P = _exit_detector_waves(wl, detectors)
    for i in range(wl.n_z - 1, -1, -1):
        yield i, 4.0 * ms.decimate(beta)
        if i > 0:
            beta = _back_one_slice(beta, wl, P, i)


def iter_s_out_recompute(wl, detectors=None):
    """Yield (i, Sout_i) for i = 0 .. n_z-1, S_2 recalculated from the exit surface
    for every slice (Sec. III second listing, "Re-calculate S_2"): n_z - 1 - i
    backward slice steps for depth i.  Exact; equal to iter_s_out."""
    start, P = _exit_detector_waves(wl, detectors)
    for i in range(wl.n_z):
        beta = start
        for j in range(wl.n_z - 1, i, -1):
            beta = _back_one_slice(beta, wl, P, j)
        yield i, 4.0 * ms.decimate(beta)


def iter_s_out_inverse(wl, detectors=None):
    """Yield (i, Sout_i) for i = 0 .. n_z-1 with S_2 carried back to depth 0 once and
    then retreated one slice per depth with the inverse multislice operator
    (Sec. IV C, Eq. MSinvop).

    The backward step is beta(i) = G(conj(t_{i+1}) beta(i+1)) with G = F^-1 conj(P) F.
    Its inverse undoes the last operation first, with the conjugated factors:
    propagate with P, then multiply by t_{i+1}.  Both are exact on the band, but
    conj(t) beta carries content outside the band limit that G removed, and the
    inverse cannot restore it (the loss Sec. IV C describes); the retreated wave is
    projected onto the band, the space the S-matrices represent:

        beta~(0) = beta(0),   beta~(i+1) = B . F[t_{i+1} F^-1[P F beta~(i)]]  (in k).
    """
    beta, P = _exit_detector_waves(wl, detectors)
    for i in range(wl.n_z - 1, 0, -1):
        beta = _back_one_slice(beta, wl, P, i)
    B = ms.band_limit(wl.n)
    for i in range(wl.n_z):
        yield i, 4.0 * ms.decimate(beta)
        if i + 1 < wl.n_z:
            t = ms.transmission(wl.vproj[i + 1], wl.sigma)
            moved = t[None] * np.fft.ifft2(P[None] * np.fft.fft2(beta))
            beta = np.fft.ifft2(B[None] * np.fft.fft2(moved))


S_OUT_SCHEMES = {"stream": iter_s_out, "recompute": iter_s_out_recompute,
                 "inverse": iter_s_out_inverse}


def probe_coefficients(wl, beams, rx, ry) -> np.ndarray:
    """a_j(R) = c exp(-2 pi i k_j.R) for all scan positions, [n_in][n_sy][n_sx]."""
    bp, bq = beams
    c = wl.f / math.sqrt(bp.size)
    ph = (-2.0 * math.pi * wl.f / wl.cell) * (bp[:, None, None] * rx[None, None, :]
                                              + bq[:, None, None] * ry[None, :, None])
    return c * np.exp(1j * ph)


def linear_map(wl, s_in=None, detectors=None, scheme="stream"):
    """PRISM-EELS map, FP64: I float64 [n_types][n_sy][n_sx].

    With `detectors` (indices into the EELS aperture's beam list) the detector sum
    of Eq. SHn0 runs over those beams only.  `scheme` picks how S_out reaches each
    depth: "stream" (backwards once), "recompute" (from the exit surface for every
    slice) or "inverse" (retreated with the inverse multislice operator)."""
    n, L, f = wl.n, wl.cell, wl.f
    nh = n // 2
    if s_in is None:
        s_in, beams = build_s_in(wl)
    else:
        s_in, beams = s_in
    rx, ry = wl.scan_positions()
    a = probe_coefficients(wl, beams, rx, ry)
    T = wl.n_types
    I = np.zeros((T, wl.scan[1], wl.scan[0]))
    for i, sout in S_OUT_SCHEMES[scheme](wl, detectors):
        for s in np.nonzero(wl.site_slice == i)[0]:
            okx = ms.axis_in_window(wl.site_x[s], rx, L, f)
            oky = ms.axis_in_window(wl.site_y[s], ry, L, f)
            if not (okx.any() and oky.any()):
                continue
            rows, cols = ms.window_indices(nh, wl.win_x0[s], wl.win_y0[s], wl.w)
            A = sout[:, rows][:, :, cols].reshape(sout.shape[0], -1)
            B = s_in[i][:, rows][:, :, cols].reshape(s_in.shape[1], -1)
            aR = a[:, oky][:, :, okx].reshape(a.shape[0], -1)
            for m in range(T):
                h = wl.H[s, m].astype(np.complex128).ravel()
                M = np.conj(A) @ (h[:, None] * B.T)            # n_out x n_in
                V = M @ aR                                     # n_out x n_R
                contrib = f * f * np.sum(np.abs(V) ** 2, axis=0)
                I[m][np.ix_(oky, okx)] += contrib.reshape(int(oky.sum()), int(okx.sum()))
    return I
