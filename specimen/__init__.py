"""Seeded synthetic specimens, beam parameters and scan grids.

This module only *prepares inputs*: atom coordinates, projected potentials
v_i(r) per slice, transition-potential windows H_n0 sampled around each
ionising site, and the scan raster.  It holds none of the multislice or
PRISM arithmetic (no transmission functions, propagators, beam lists or
window rules) so that the FP64 oracle and the CUDA library can both consume
exactly the same arrays without sharing any of the method's code.

Physical inputs stand in for data the paper takes from elsewhere:

* the paper's SrTiO3 / FePt structures (Sec. III) become rocksalt Fe-O
  supercells and a spherical Fe-O particle;
* the transition potentials H_n0 of Eq. (Hn0def), which the paper imports
  from muSTEM, become the analytic model
  H_m(r) = A (r/r0)^|m| exp(-r^2 / (2 r0^2)) exp(i m phi).

Array conventions: real-space arrays are indexed [y][x]; the pixel (ix, iy)
of an N x N grid over an L x L cell sits at (ix L/N, iy L/N).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Two-Gaussian projected-potential parameters per species:
# (amplitudes in V*A, Gaussian widths in A).  v(r) = sum_k A_k exp(-r^2/(2 s_k^2)).
POTENTIAL_PARAMS = {
    "Fe": ((80.0, 20.0), (0.25, 0.8)),
    "O": ((30.0, 8.0), (0.25, 0.8)),
}

# Physical constants (CODATA 2018, SI).
_M0 = 9.1093837015e-31      # electron rest mass, kg
_E = 1.602176634e-19        # elementary charge, C
_H = 6.62607015e-34         # Planck constant, J s
_C = 299792458.0            # speed of light, m/s


def electron_wavelength(e0_ev: float) -> float:
    """Relativistic electron wavelength in Angstrom for accelerating voltage e0_ev."""
    p = math.sqrt(2.0 * _M0 * _E * e0_ev * (1.0 + _E * e0_ev / (2.0 * _M0 * _C * _C)))
    return _H / p * 1e10


def interaction_constant(e0_ev: float, lam_a: float) -> float:
    """sigma = 2 pi m e lambda / h^2 (Sec. II, after Eq. Schro), in rad / (V A).

    m is the relativistic mass at e0_ev; lam_a is the wavelength in Angstrom.
    """
    m = _M0 + _E * e0_ev / (_C * _C)
    return 2.0 * math.pi * m * _E * (lam_a * 1e-10) / (_H * _H) * 1e-10


@dataclasses.dataclass
class Workload:
    """Everything a map request needs, as plain arrays.

    vproj     float32 [n_z][n][n]      projected potential of each slice, V*A
    H         complex64 [S][T][w][w]   transition potential windows on the N/2 grid
    site_*    per ionising site: slice index, position (A), window origin on the N/2 grid
    scan      (n_sx, n_sy, x0, y0, step_x, step_y); R(ix, iy) = (x0 + ix*step_x, y0 + iy*step_y)
    """

    name: str
    n: int
    cell: float
    n_z: int
    dz: float
    lam: float
    sigma: float
    f: int
    alpha: float
    beta: float
    vproj: np.ndarray
    w: int
    H: np.ndarray
    site_slice: np.ndarray
    site_x: np.ndarray
    site_y: np.ndarray
    win_x0: np.ndarray
    win_y0: np.ndarray
    scan: tuple

    @property
    def n_types(self) -> int:
        return int(self.H.shape[1])

    @property
    def n_sites(self) -> int:
        return int(self.H.shape[0])

    @property
    def n_scan(self) -> int:
        return int(self.scan[0] * self.scan[1])

    def scan_positions(self):
        """Scan coordinates as two FP64 vectors (x of each column, y of each row)."""
        n_sx, n_sy, x0, y0, sx, sy = self.scan
        rx = np.array([x0 + i * sx for i in range(n_sx)], dtype=np.float64)
        ry = np.array([y0 + i * sy for i in range(n_sy)], dtype=np.float64)
        return rx, ry

    def with_sites(self, idx) -> "Workload":
        """Copy restricted to a subset of ionising sites (same specimen and scan)."""
        idx = np.asarray(idx, dtype=np.int64)
        return dataclasses.replace(
            self, H=np.ascontiguousarray(self.H[idx]),
            site_slice=self.site_slice[idx].copy(), site_x=self.site_x[idx].copy(),
            site_y=self.site_y[idx].copy(), win_x0=self.win_x0[idx].copy(),
            win_y0=self.win_y0[idx].copy())

    def with_scan(self, scan) -> "Workload":
        return dataclasses.replace(self, scan=tuple(scan))


# ----------------------------------------------------------------------------
# structures
# ----------------------------------------------------------------------------

_FE_FRAC = ((0.0, 0.0, 0.0), (0.5, 0.5, 0.0), (0.5, 0.0, 0.5), (0.0, 0.5, 0.5))


def rocksalt_atoms(a: float, nx: int, ny: int, nzc: int, vacancy_frac: float = 0.0,
                   seed: int | None = None):
    """Rocksalt Fe-O supercell: Fe on the fcc sites, O shifted by a/2 along x.

    Returns (x, y, z, species, zlayer) with zlayer the index of the a/2 layer
    each atom lies in (exact integer, used for slicing with dz = a/2).
    A seeded fraction of Fe sites become vacancies (atom removed).
    """
    xs, ys, zs, sp, lay = [], [], [], [], []
    for k in range(nzc):
        for j in range(ny):
            for i in range(nx):
                for fx, fy, fz in _FE_FRAC:
                    for name, ox in (("Fe", 0.0), ("O", 0.5)):
                        gx = (fx + ox) % 1.0
                        xs.append((i + gx) * a)
                        ys.append((j + fy) * a)
                        zs.append((k + fz) * a)
                        sp.append(name)
                        lay.append(2 * k + int(round(2 * fz)))
    x = np.array(xs); y = np.array(ys); z = np.array(zs)
    sp = np.array(sp); lay = np.array(lay, dtype=np.int32)
    if vacancy_frac > 0.0:
        rng = np.random.default_rng(seed)
        fe = np.nonzero(sp == "Fe")[0]
        drop = fe[rng.random(fe.size) < vacancy_frac]
        keep = np.ones(x.size, dtype=bool)
        keep[drop] = False
        x, y, z, sp, lay = x[keep], y[keep], z[keep], sp[keep], lay[keep]
    return x, y, z, sp, lay


def nanoparticle_atoms(a: float, diameter: float, box: float):
    """Rocksalt Fe-O sphere of the given diameter centred in a cubic box.

    An Fe lattice site sits at the box centre; sites with |r - c| <= d/2 are kept.
    """
    c = box / 2.0
    n = int(math.ceil(diameter / a)) + 2
    xs, ys, zs, sp = [], [], [], []
    r2max = (diameter / 2.0) ** 2
    for k in range(-n, n + 1):
        for j in range(-n, n + 1):
            for i in range(-n, n + 1):
                for fx, fy, fz in _FE_FRAC:
                    for name, ox in (("Fe", 0.0), ("O", 0.5)):
                        px = (i + fx + ox) * a
                        py = (j + fy) * a
                        pz = (k + fz) * a
                        if px * px + py * py + pz * pz <= r2max:
                            xs.append(c + px); ys.append(c + py); zs.append(c + pz)
                            sp.append(name)
    return np.array(xs), np.array(ys), np.array(zs), np.array(sp)


# ----------------------------------------------------------------------------
# sampled fields
# ----------------------------------------------------------------------------

def _profile(n: int, px: float, pos: float, s: float, cut: float):
    """Indices and 1D Gaussian factors exp(-d^2/(2 s^2)) of a periodic patch."""
    m = min(int(math.ceil(cut / px)), (n - 1) // 2)
    c = int(math.floor(pos / px + 0.5))
    idx = np.arange(c - m, c + m + 1)
    d = idx * px - pos
    return idx % n, np.exp(-d * d / (2.0 * s * s))


def projected_potentials(n: int, cell: float, n_z: int, x, y, sp, slice_idx) -> np.ndarray:
    """v_i(r) for each slice: per-atom sums of two Gaussians on the N x N grid.

    Each Gaussian is evaluated on a periodic patch of half-width
    min(6 s_k, (N-1)/2 pixels) around the atom (displacements measured from the
    atom, patch wrapped onto the cell).  Returned as float32 V*A.
    """
    px = cell / n
    v = np.zeros((n_z, n, n), dtype=np.float64)
    for xa, ya, spa, si in zip(x, y, sp, slice_idx):
        amps, sigs = POTENTIAL_PARAMS[str(spa)]
        for amp, s in zip(amps, sigs):
            ix, gx = _profile(n, px, xa, s, 6.0 * s)
            iy, gy = _profile(n, px, ya, s, 6.0 * s)
            v[si][np.ix_(iy, ix)] += amp * np.outer(gy, gx)
    return v.astype(np.float32)


def transition_windows(n: int, cell: float, w: int, site_x, site_y, m_list=(-1, 0, 1),
                       amp: float = 0.01, r0: float = 0.3, tail: bool = False):
    """Synthetic L-edge-like transition potentials sampled on the N/2 grid.

    H_m(r) = amp (r/r0)^|m| exp(-r^2/(2 r0^2)) exp(i m phi) about each site, or with
    tail=True the long-tailed amp (r/r0)^|m| / (1 + (r/r0)^2)^((|m|+3)/2) exp(i m phi)
    (decaying as r^-3), on a w x w window of the N/2 grid whose origin is (nearest
    pixel - w/2), taken modulo N/2.  Returns (H complex64 [S][T][w][w], win_x0, win_y0).
    """
    nh = n // 2
    px = cell / nh
    S = len(site_x)
    H = np.zeros((S, len(m_list), w, w), dtype=np.complex128)
    x0 = np.zeros(S, dtype=np.int32)
    y0 = np.zeros(S, dtype=np.int32)
    u = np.arange(w)
    for s in range(S):
        cx = int(math.floor(site_x[s] / px + 0.5)) - w // 2
        cy = int(math.floor(site_y[s] / px + 0.5)) - w // 2
        dx = (cx + u) * px - site_x[s]
        dy = (cy + u) * px - site_y[s]
        DX, DY = np.meshgrid(dx, dy)
        r = np.hypot(DX, DY)
        phi = np.arctan2(DY, DX)
        for t, m in enumerate(m_list):
            if tail:
                radial = (r / r0) ** abs(m) / (1.0 + (r / r0) ** 2) ** ((abs(m) + 3) / 2.0)
            else:
                radial = (r / r0) ** abs(m) * np.exp(-r * r / (2 * r0 * r0))
            H[s, t] = amp * radial * np.exp(1j * m * phi)
        x0[s] = cx % nh
        y0[s] = cy % nh
    return H.astype(np.complex64), x0, y0


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

A_FEO = 4.3
LAM_200KEV = 0.02508


def _crystal_workload(name, n, ncell, nzc, f, w, scan_n, vacancy_frac=0.0, seed=None,
                      alpha=0.020, beta=0.030):
    a = A_FEO
    L = ncell * a
    x, y, z, sp, lay = rocksalt_atoms(a, ncell, ncell, nzc, vacancy_frac, seed)
    n_z = 2 * nzc
    vproj = projected_potentials(n, L, n_z, x, y, sp, lay)
    fe = sp == "Fe"
    sx, sy, ss = x[fe], y[fe], lay[fe]
    H, wx, wy = transition_windows(n, L, w, sx, sy)
    c0 = (ncell // 2) * a if ncell > 1 else 0.0
    scan = (scan_n, scan_n, c0, c0, a / scan_n, a / scan_n)
    return Workload(name=name, n=n, cell=L, n_z=n_z, dz=a / 2, lam=LAM_200KEV,
                    sigma=interaction_constant(200e3, LAM_200KEV), f=f, alpha=alpha,
                    beta=beta, vproj=vproj, w=w, H=H, site_slice=ss.astype(np.int32),
                    site_x=sx.copy(), site_y=sy.copy(), win_x0=wx, win_y0=wy, scan=scan)


def rocksalt_small():
    """Rocksalt Fe-O 2x2x3 cells, 128^2 grid, 6 slices, f=1, 8x8 scan over one cell."""
    return _crystal_workload("rocksalt_2x2x3_n128_f1", n=128, ncell=2, nzc=3, f=1, w=32, scan_n=8)


def rocksalt_fp32():
    """Rocksalt Fe-O 8x8x20 cells, 512^2 grid, 40 slices, f=2, 32x32 scan over the central cell."""
    return _crystal_workload("rocksalt_8x8x20_n512_f2", n=512, ncell=8, nzc=20, f=2, w=32,
                             scan_n=32)


def rocksalt_phonons(k: int, u_rms: float = 0.08, seed: int = 5, ncell: int = 4, nzc: int = 6,
                     n: int = 256, f: int = 2, scan_n: int = 16, w: int = 24):
    """k frozen-phonon configurations of a rocksalt Fe-O crystal (ncell x ncell x nzc
    cells, n^2 grid, f, scan_n^2 scan over the central cell).

    Every atom is displaced in x and y by independent Gaussian offsets of standard
    deviation u_rms (A), drawn from one seeded generator, configuration after
    configuration (z, and so the slice of each atom, is kept).  Potentials and the
    transition windows of the Fe sites follow the displaced atoms.  Returns a list of
    Workloads with the same shapes."""
    a = A_FEO
    L = ncell * a
    x0, y0, z, sp_, lay = rocksalt_atoms(a, ncell, ncell, nzc)
    n_z = 2 * nzc
    rng = np.random.default_rng(seed)
    c0 = (ncell // 2) * a if ncell > 1 else 0.0
    scan = (scan_n, scan_n, c0, c0, a / scan_n, a / scan_n)
    out = []
    for c in range(k):
        x = (x0 + rng.normal(0.0, u_rms, x0.size)) % L
        y = (y0 + rng.normal(0.0, u_rms, y0.size)) % L
        vproj = projected_potentials(n, L, n_z, x, y, sp_, lay)
        fe = sp_ == "Fe"
        H, wx, wy = transition_windows(n, L, w, x[fe], y[fe])
        out.append(Workload(name=f"rocksalt_{ncell}x{ncell}x{nzc}_n{n}_f{f}_fp{c}", n=n, cell=L,
                            n_z=n_z, dz=a / 2, lam=LAM_200KEV,
                            sigma=interaction_constant(200e3, LAM_200KEV), f=f, alpha=0.020,
                            beta=0.030, vproj=vproj, w=w, H=H,
                            site_slice=lay[fe].astype(np.int32), site_x=x[fe].copy(),
                            site_y=y[fe].copy(), win_x0=wx, win_y0=wy, scan=scan))
    return out


def rocksalt_slab(nzc: int, n: int = 256, ncell: int = 8, f: int = 2, scan_n: int = 16):
    """Rocksalt Fe-O ncell x ncell x nzc cells (2 nzc slices of a/2), n^2 grid, a scan of
    scan_n^2 over the central cell: the thickness series of the S_2 scheme study."""
    return _crystal_workload(f"rocksalt_{ncell}x{ncell}x{nzc}_n{n}_f{f}", n=n, ncell=ncell,
                             nzc=nzc, f=f, w=32, scan_n=scan_n)


def dopant_slab(w: int, n: int = 128, nzc: int = 12, scan_n: int = 32, r0: float = 0.4,
                every_fe: bool = False):
    """One dopant with a long-tailed transition potential in a rocksalt Fe-O slab.

    2x2 cells (8.6 A) x nzc cells (2 nzc slices of a/2; 51.6 A for nzc = 12), n^2 grid,
    f = 1.  The dopant replaces the Fe at the cell centre in the middle slice; its two
    transitions (m = +2, -2) have the r^-3 tail of transition_windows(tail=True) and
    are cut to a w x w window of the N/2 grid (w = n/2 is the whole cell).  The scan
    covers the cell with scan_n^2 positions: the crop-window series of Sec. IV B.
    every_fe=True puts the same transitions on every Fe of the slab (a contraction
    large enough to time)."""
    a = A_FEO
    L = 2 * a
    x, y, z, sp, lay = rocksalt_atoms(a, 2, 2, nzc)
    n_z = 2 * nzc
    vproj = projected_potentials(n, L, n_z, x, y, sp, lay)
    mid = 2 * (nzc // 2)     # an even a/2 layer: it holds an Fe at (a, a)
    if every_fe:
        pick = np.nonzero(sp == "Fe")[0]
    else:
        pick = np.nonzero((sp == "Fe") & (lay == mid) & (np.abs(x - a) < 1e-9)
                          & (np.abs(y - a) < 1e-9))[0]
    sx, sy = x[pick].copy(), y[pick].copy()
    H, wx, wy = transition_windows(n, L, w, sx, sy, m_list=(2, -2), r0=r0, tail=True)
    scan = (scan_n, scan_n, 0.0, 0.0, L / scan_n, L / scan_n)
    return Workload(name=f"dopant_2x2x{nzc}_n{n}_w{w}" + ("_allfe" if every_fe else ""), n=n,
                    cell=L, n_z=n_z, dz=a / 2, lam=LAM_200KEV,
                    sigma=interaction_constant(200e3, LAM_200KEV), f=1, alpha=0.020, beta=0.030,
                    vproj=vproj, w=w, H=H, site_slice=lay[pick].astype(np.int32), site_x=sx,
                    site_y=sy, win_x0=wx, win_y0=wy, scan=scan)


def rocksalt_vacancy():
    """Rocksalt Fe-O 12x12x40 cells, 768^2 grid, 80 slices, f=2, 5% Fe vacancies (seed 3)."""
    return _crystal_workload("rocksalt_12x12x40_n768_f2_vac5", n=768, ncell=12, nzc=40, f=2,
                             w=32, scan_n=32, vacancy_frac=0.05, seed=3)


def nanoparticle():
    """Fe-O sphere (80 A) in a 100 A box, dz = 2 A, 1024^2 grid, f=4, 128x128 scan."""
    a, box, n, f, w = A_FEO, 100.0, 1024, 4, 24
    dz = 2.0
    n_z = 50
    x, y, z, sp = nanoparticle_atoms(a, 80.0, box)
    lay = np.floor(z / dz + 1e-9).astype(np.int32)
    vproj = projected_potentials(n, box, n_z, x, y, sp, lay)
    fe = sp == "Fe"
    H, wx, wy = transition_windows(n, box, w, x[fe], y[fe])
    scan = (128, 128, 10.0, 10.0, 80.0 / 128, 80.0 / 128)
    return Workload(name="feo_sphere80_n1024_f4", n=n, cell=box, n_z=n_z, dz=dz,
                    lam=LAM_200KEV, sigma=interaction_constant(200e3, LAM_200KEV), f=f,
                    alpha=0.020, beta=0.030, vproj=vproj, w=w, H=H,
                    site_slice=lay[fe].astype(np.int32), site_x=x[fe].copy(),
                    site_y=y[fe].copy(), win_x0=wx, win_y0=wy, scan=scan)


def random_workload(n: int, n_z: int, f: int, cell: float, n_sites: int, w: int, seed: int,
                    lam: float = LAM_200KEV, alpha: float = 0.020, beta: float = 0.030,
                    dz: float = 2.0, scan_n: int = 4, vscale: float = 400.0, n_types: int = 2):
    """Random specimen for small tests: smooth random potentials and random-phase H windows.

    Potentials are random Gaussians (peak up to vscale V*A) at random positions;
    sites are random positions in random slices; H is a random complex window
    times a Gaussian envelope.  Everything is drawn from one seeded generator.
    """
    rng = np.random.default_rng(seed)
    n_atoms = 6 * n_z
    ax = rng.random(n_atoms) * cell
    ay = rng.random(n_atoms) * cell
    asl = rng.integers(0, n_z, n_atoms)
    px = cell / n
    v = np.zeros((n_z, n, n))
    for xa, ya, si in zip(ax, ay, asl):
        s = 0.2 + 0.4 * rng.random()
        amp = vscale * rng.random()
        ix, gx = _profile(n, px, xa, s, 6 * s)
        iy, gy = _profile(n, px, ya, s, 6 * s)
        v[si][np.ix_(iy, ix)] += amp * np.outer(gy, gx)
    step = cell / (f * scan_n)
    ox, oy = rng.random() * cell, rng.random() * cell
    # sites within reach of the scanned L/f cell, wrapped into the supercell
    sx = (ox + rng.uniform(-0.5, 1.5, n_sites) * cell / f) % cell
    sy = (oy + rng.uniform(-0.5, 1.5, n_sites) * cell / f) % cell
    ss = rng.integers(0, n_z, n_sites).astype(np.int32)
    nh = n // 2
    env = np.exp(-((np.arange(w) - w / 2) ** 2) / (2 * (w / 5) ** 2))
    H = (rng.standard_normal((n_sites, n_types, w, w))
         + 1j * rng.standard_normal((n_sites, n_types, w, w))) * 0.01
    H *= env[None, None, :, None] * env[None, None, None, :]
    wx = rng.integers(0, nh, n_sites).astype(np.int32)
    wy = rng.integers(0, nh, n_sites).astype(np.int32)
    scan = (scan_n, scan_n, ox, oy, step, step)
    return Workload(name=f"random_n{n}_z{n_z}_f{f}_s{seed}", n=n, cell=cell, n_z=n_z, dz=dz,
                    lam=lam, sigma=interaction_constant(200e3, lam), f=f, alpha=alpha,
                    beta=beta, vproj=v.astype(np.float32), w=w, H=H.astype(np.complex64),
                    site_slice=ss, site_x=sx, site_y=sy, win_x0=wx, win_y0=wy, scan=scan)


def nanoparticle_small():
    """Fe-O sphere (30 A) in a 40 A box, dz = 2 A, 20 slices, 512^2 grid, f = 4,
    48x48 scan at 0.625 A: a few-GB case of the nanoparticle workload for profiling."""
    a, box, n, f, w = A_FEO, 40.0, 512, 4, 24
    dz = 2.0
    n_z = 20
    x, y, z, sp = nanoparticle_atoms(a, 30.0, box)
    lay = np.floor(z / dz + 1e-9).astype(np.int32)
    keep = lay < n_z
    x, y, z, sp, lay = x[keep], y[keep], z[keep], sp[keep], lay[keep]
    vproj = projected_potentials(n, box, n_z, x, y, sp, lay)
    fe = sp == "Fe"
    H, wx, wy = transition_windows(n, box, w, x[fe], y[fe])
    scan = (48, 48, 5.0, 5.0, 0.625, 0.625)
    return Workload(name="feo_sphere30_n512_f4", n=n, cell=box, n_z=n_z, dz=dz,
                    lam=LAM_200KEV, sigma=interaction_constant(200e3, LAM_200KEV), f=f,
                    alpha=0.020, beta=0.030, vproj=vproj, w=w, H=H,
                    site_slice=lay[fe].astype(np.int32), site_x=x[fe].copy(),
                    site_y=y[fe].copy(), win_x0=wx, win_y0=wy, scan=scan)


def nanoparticle_small_1024():
    """The 30 A Fe-O sphere of nanoparticle_small on a 1024^2 grid (0.039 A pixels), 10
    slices, f = 4, 48x48 scan: a few-GB case of the 1024^2 FFT plan for profiling."""
    wl = nanoparticle_small()
    a, box, n, f, w = A_FEO, 40.0, 1024, 4, 24
    n_z = 10
    x, y, z, sp = nanoparticle_atoms(a, 30.0, box)
    lay = np.floor(z / 2.0 + 1e-9).astype(np.int32)
    keep = lay < n_z
    x, y, sp, lay = x[keep], y[keep], sp[keep], lay[keep]
    vproj = projected_potentials(n, box, n_z, x, y, sp, lay)
    fe = sp == "Fe"
    H, wx, wy = transition_windows(n, box, w, x[fe], y[fe])
    return Workload(name="feo_sphere30_n1024_f4", n=n, cell=box, n_z=n_z, dz=2.0,
                    lam=wl.lam, sigma=wl.sigma, f=f, alpha=wl.alpha, beta=wl.beta, vproj=vproj,
                    w=w, H=H, site_slice=lay[fe].astype(np.int32), site_x=x[fe].copy(),
                    site_y=y[fe].copy(), win_x0=wx, win_y0=wy, scan=wl.scan)


def nanoparticle_centre_512():
    """The four central slices (46-54 A deep) of the 80 A Fe-O sphere in its 100 A box on
    a 512^2 grid, f = 4, 64x64 scan over 80 A: the headline's contraction shapes (n_in,
    n_out and the 24-pixel windows depend on the box, not the grid) in a few GB, for
    profiling the GEMMs."""
    a, box, n, f, w = A_FEO, 100.0, 512, 4, 24
    dz, z0, n_z = 2.0, 46.0, 4
    x, y, z, sp = nanoparticle_atoms(a, 80.0, box)
    lay = np.floor((z - z0) / dz + 1e-9).astype(np.int32)
    keep = (lay >= 0) & (lay < n_z)
    x, y, sp, lay = x[keep], y[keep], sp[keep], lay[keep]
    vproj = projected_potentials(n, box, n_z, x, y, sp, lay)
    fe = sp == "Fe"
    H, wx, wy = transition_windows(n, box, w, x[fe], y[fe])
    scan = (64, 64, 10.0, 10.0, 80.0 / 64, 80.0 / 64)
    return Workload(name="feo_sphere80_n512_f4_centre4", n=n, cell=box, n_z=n_z, dz=dz,
                    lam=LAM_200KEV, sigma=interaction_constant(200e3, LAM_200KEV), f=f,
                    alpha=0.020, beta=0.030, vproj=vproj, w=w, H=H,
                    site_slice=lay[fe].astype(np.int32), site_x=x[fe].copy(),
                    site_y=y[fe].copy(), win_x0=wx, win_y0=wy, scan=scan)


WORKLOADS = {
    "rocksalt_small": rocksalt_small,
    "rocksalt_fp32": rocksalt_fp32,
    "rocksalt_vacancy": rocksalt_vacancy,
    "nanoparticle": nanoparticle,
    "nanoparticle_small": nanoparticle_small,
    "nanoparticle_small_1024": nanoparticle_small_1024,
    "nanoparticle_centre_512": nanoparticle_centre_512,
}


# ----------------------------------------------------------------------------
# mixed request stream for the map server
# ----------------------------------------------------------------------------

_M_ORDER = (0, 1, -1, 2, -2, 3)
_MASTERS = {}


def _master_crystal(n: int, max_slices: int = 120):
    """Rocksalt crystal of N/64 cells per side (0.0672 A pixels), max_slices thick.

    The crystal repeats every two slices (dz = a/2), so only two slices of potential
    are evaluated and then tiled.  Returns (vproj [max_slices][n][n], Fe sites x, y,
    slice) shared by every request on this grid.
    """
    if n in _MASTERS:
        return _MASTERS[n]
    ncell = n // 64
    a = A_FEO
    L = ncell * a
    x, y, z, sp, lay = rocksalt_atoms(a, ncell, ncell, 1)
    two = projected_potentials(n, L, 2, x, y, sp, lay)
    vproj = np.ascontiguousarray(np.tile(two, (max_slices // 2, 1, 1)))
    fe = sp == "Fe"
    fx, fy, fl = x[fe], y[fe], lay[fe]
    reps = max_slices // 2
    sx = np.tile(fx, reps)
    sy = np.tile(fy, reps)
    ss = (np.repeat(np.arange(reps), fx.size) * 2 + np.tile(fl, reps)).astype(np.int32)
    _MASTERS[n] = (vproj, sx, sy, ss, L)
    return _MASTERS[n]


def serving_request(rng, w: int = 32):
    """One map request of the mixed stream: grid 256^2..1024^2, 20..120 slices, 1..6
    transition channels, f in {2, 3, 4}, scan 16^2..64^2 over the central unit cell.

    Returns a dict of host arrays; vproj is a view of the first n_z slices of the
    grid's master crystal and H is one [T][w][w] set shared by all Fe sites (every
    site sits on a pixel of the N/2 grid, so the same samples apply to all of them).
    """
    n = int(rng.choice([256, 384, 512, 768, 1024]))
    n_z = int(rng.integers(10, 61)) * 2
    T = int(rng.integers(1, 7))
    f = int(rng.choice([2, 3, 4]))
    ns = int(rng.integers(16, 65))
    vproj, sx, sy, ss, L = _master_crystal(n)
    keep = ss < n_z
    nh = n // 2
    px = L / nh
    sxk, syk, ssk = sx[keep], sy[keep], ss[keep]
    wx = ((np.floor(sxk / px + 0.5).astype(np.int64) - w // 2) % nh).astype(np.int32)
    wy = ((np.floor(syk / px + 0.5).astype(np.int64) - w // 2) % nh).astype(np.int32)
    # shared H sampled about a site on a pixel: window origin at -w/2
    u = (np.arange(w) - w // 2) * px
    DX, DY = np.meshgrid(u, u)
    r = np.hypot(DX, DY)
    phi = np.arctan2(DY, DX)
    H = np.stack([0.01 * (r / 0.3) ** abs(m) * np.exp(-r * r / 0.18) * np.exp(1j * m * phi)
                  for m in _M_ORDER[:T]]).astype(np.complex64)
    c0 = (L // A_FEO // 2) * A_FEO
    return {"n": n, "n_z": n_z, "cell": L, "f": f, "n_types": T, "vproj": vproj[:n_z],
            "H": H, "site_slice": ssk.copy(), "site_x": sxk.copy(), "site_y": syk.copy(),
            "win_x0": wx, "win_y0": wy, "scan": (ns, ns, c0, c0, A_FEO / ns, A_FEO / ns),
            "lam": LAM_200KEV, "sigma": interaction_constant(200e3, LAM_200KEV),
            "dz": A_FEO / 2, "alpha": 0.020, "beta": 0.030}


def serving_stream(count: int, seed: int = 4, accept=None):
    """`count` requests with unit-mean exponential inter-arrival gaps (seeded).

    accept(request) -> bool may reject a draw (for example one whose device footprint
    exceeds the server budget); rejected draws are replaced by the next ones.
    """
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        req = serving_request(rng)
        gap = float(rng.exponential(1.0))
        if accept is None or accept(req):
            req["gap"] = gap
            out.append(req)
    return out
