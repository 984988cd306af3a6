"""Dense-matrix restatement of the conventional map for tiny grids (N <= 32).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Every operator of Sec. II-III is written out as an explicit matrix over the
flattened N x N grid (index iy*N + ix):

* F      unitary DFT matrix, F[k, r] = exp(-2 pi i (p ix + q iy)/N) / N,
* A_i    = F^H diag(P) F diag(t_i)                         (Eq. MSop),
* D      decimation to the even sub-grid,
* J      band-limited interpolation, J[n, m] = prod_axes (2/N) sum_{p=-N/4}^{N/4-1}
         exp(2 pi i p (n - 2m)/N),
* probe  evaluated point by point as c sum_j exp(2 pi i k_j.(r - R)) / N.

No FFT routine is called, and the beam lists are enumerated here again, so a
mistake in the FFT-based oracle (a sign, an index order, a normalisation, a
misplaced spectrum bin) shows up as a disagreement.
"""
from __future__ import annotations

import math

import numpy as np


def _signed(n):
    return np.array([i if i < n - n // 2 else i - n for i in range(n)], dtype=np.float64)


def dft_matrix(n: int) -> np.ndarray:
    p = _signed(n)
    x = np.arange(n, dtype=np.float64)
    F1 = np.exp(-2j * math.pi * np.outer(p, x) / n) / math.sqrt(n)    # [freq][pos]
    return np.kron(F1, F1)   # rows (q, p), cols (iy, ix)


def interpolation_matrix(n: int) -> np.ndarray:
    nh = n // 2
    nn = np.arange(n, dtype=np.float64)
    mm = np.arange(nh, dtype=np.float64)
    J1 = np.zeros((n, nh), dtype=np.complex128)
    for p in range(-(n // 4), n // 4):
        J1 += np.exp(2j * math.pi * p * (nn[:, None] - 2 * mm[None, :]) / n)
    J1 /= nh
    return np.kron(J1, J1)


def decimation_matrix(n: int) -> np.ndarray:
    nh = n // 2
    D = np.zeros((nh * nh, n * n))
    for my in range(nh):
        for mx in range(nh):
            D[my * nh + mx, (2 * my) * n + 2 * mx] = 1.0
    return D


def _beams(n, cell, lam, f, angle):
    out = []
    r = angle * cell / (lam * f)
    m = int(r) + 2
    for q in range(-m, m + 1):
        for p in range(-m, m + 1):
            if lam * f * math.hypot(p, q) / cell <= angle:
                out.append((f * p, f * q))
    return out


def dense_map(wl):
    """Map of the conventional algorithm built from dense operators. [T][n_sy][n_sx]."""
    n, L, f, n_z = wl.n, wl.cell, wl.f, wl.n_z
    nh = n // 2
    F = dft_matrix(n)
    Fh = F.conj().T
    p = _signed(n)
    K2 = (p[None, :] ** 2 + p[:, None] ** 2).ravel()        # (q, p) order, squared index
    band = (16 * K2 < n * n).astype(np.float64)
    Pdiag = band * np.exp(-1j * math.pi * wl.lam * wl.dz * K2 / (L * L))
    prop = Fh @ (Pdiag[:, None] * F)
    tdiag = [np.exp(1j * wl.sigma * wl.vproj[i].astype(np.float64).ravel()) for i in range(n_z)]
    A = [prop @ np.diag(t) for t in tdiag]
    D = decimation_matrix(n)
    J = interpolation_matrix(n)
    ix = np.arange(n, dtype=np.float64) * L / n
    X, Y = np.meshgrid(ix, ix)
    X = X.ravel()
    Y = Y.ravel()
    pb = _beams(n, L, wl.lam, f, wl.alpha)
    db = _beams(n, L, wl.lam, f, wl.beta)
    c = f / math.sqrt(len(pb))
    # detector rows <k_d| as explicit plane waves
    Det = np.array([np.exp(-2j * math.pi * (kp * X + kq * Y) / L) / n for kp, kq in db])
    n_sx, n_sy, x0, y0, sx, sy = wl.scan
    I = np.zeros((wl.n_types, n_sy, n_sx))
    for iy in range(n_sy):
        for jx in range(n_sx):
            rx = x0 + jx * sx
            ry = y0 + iy * sy
            psi = np.zeros(n * n, dtype=np.complex128)
            for kp, kq in pb:
                psi += c * np.exp(2j * math.pi * (kp * (X - rx) + kq * (Y - ry)) / L) / n
            for i in range(n_z):
                alpha = tdiag[i] * psi
                for s in range(wl.n_sites):
                    if wl.site_slice[s] != i:
                        continue
                    ok = True
                    for sc, rc in ((wl.site_x[s], rx), (wl.site_y[s], ry)):
                        d = sc - rc
                        d = d - L * math.floor(d / L + 0.5)
                        if not (-L / (2 * f) <= d < L / (2 * f)):
                            ok = False
                    if not ok:
                        continue
                    for m in range(wl.n_types):
                        hfull = np.zeros(nh * nh, dtype=np.complex128)
                        for v in range(wl.w):
                            for u in range(wl.w):
                                gy = (wl.win_y0[s] + v) % nh
                                gx = (wl.win_x0[s] + u) % nh
                                hfull[gy * nh + gx] = complex(wl.H[s, m, v, u])
                        y = prop @ (J @ (hfull * (D @ alpha)))
                        for i2 in range(i + 1, n_z):
                            y = A[i2] @ y
                        I[m, iy, jx] += f * f * float(np.sum(np.abs(Det @ y) ** 2))
                psi = prop @ alpha
    return I
