"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a printed number, an invariant, a brute-force dense evaluation or a
direct (FFT-free) sum.  None needs a GPU.
"""
import json
import math
import os

import numpy as np
import pytest

import specimen as sp
from oracle import dense
from oracle import linear as lin
from oracle import multislice as ms

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tiny(n=16, f=1, seed=1, n_z=3, n_sites=3, w=6, alpha=0.0138, beta=0.018, cell=4.0,
          scan_n=3, dz=1.5):
    return sp.random_workload(n=n, n_z=n_z, f=f, cell=cell, n_sites=n_sites, w=w, seed=seed,
                              alpha=alpha, beta=beta, dz=dz, scan_n=scan_n)


def _band_limited(n, rng, batch=()):
    X = rng.standard_normal(batch + (n, n)) + 1j * rng.standard_normal(batch + (n, n))
    return np.fft.ifft2(X * ms.band_limit(n))


# --- beam constants (Sec. II, after Eq. Schro) ---------------------------------

def test_wavelength_and_interaction_constant_match_textbook():
    g = json.load(open(os.path.join(GOLDEN, "textbook_beam_constants.json")))
    lam = sp.electron_wavelength(g["e0_volts"])
    assert abs(lam - g["wavelength_A"]) < 5e-5
    sig = sp.interaction_constant(g["e0_volts"], g["wavelength_A"])
    assert abs(sig - g["sigma_rad_per_VA"]) / g["sigma_rad_per_VA"] < 2e-4


# --- band limit and half-resolution representation (Sec. III) -----------------

def test_band_limit_is_half_the_array():
    for n in (16, 64, 96, 128):
        B = ms.band_limit(n)
        p = ms.fft_index(n)
        on_axis = p[B[0, :]]
        assert on_axis.max() == n // 4 - 1 and on_axis.min() == -(n // 4 - 1)
        assert np.array_equal(B, B.T) and np.array_equal(B, B[::-1][np.r_[-1, 0:n - 1]])


def test_decimate_interpolate_roundtrip():
    rng = np.random.default_rng(0)
    for n in (16, 48, 64):
        x = _band_limited(n, rng)
        assert np.allclose(ms.interpolate(ms.decimate(x), n), x, atol=1e-13 * np.abs(x).max())
        xh = rng.standard_normal((n // 2, n // 2)) + 1j * rng.standard_normal((n // 2, n // 2))
        assert np.allclose(ms.decimate(ms.interpolate(xh, n)), xh, atol=1e-13)


def test_half_grid_inner_product_identity():
    """<b, Interp x>_N = 4 <Dec b, x>_{N/2} for band-limited b (used by the linear form)."""
    rng = np.random.default_rng(5)
    n = 32
    b = _band_limited(n, rng)
    xh = rng.standard_normal((n // 2, n // 2)) + 1j * rng.standard_normal((n // 2, n // 2))
    lhs = np.vdot(b, ms.interpolate(xh, n))
    rhs = 4 * np.vdot(ms.decimate(b), xh)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# --- multislice operator (Eqs. 3, 4, MSop) ------------------------------------

def test_norm_conserved_without_band_limit_and_nonincreasing_with_it():
    rng = np.random.default_rng(2)
    n, L = 64, 10.0
    v = rng.standard_normal((n, n)) * 50
    t = ms.transmission(v, 7.3e-4)
    P = ms.propagator(n, L, 0.02508, 2.0)
    P_open = np.exp(-1j * math.pi * 0.02508 * 2.0 * (ms.fft_index(n)[None] ** 2
                                                    + ms.fft_index(n)[:, None] ** 2) / L ** 2)
    psi = _band_limited(n, rng)
    nrm = np.linalg.norm(psi)
    y = psi
    for _ in range(5):
        y = ms.slice_step(y, t, P_open)
    assert abs(np.linalg.norm(y) - nrm) < 1e-13 * nrm
    y = psi
    prev = nrm
    for _ in range(5):
        y = ms.slice_step(y, t, P)
        assert np.linalg.norm(y) <= prev * (1 + 1e-14)
        prev = np.linalg.norm(y)


def test_free_space_equals_closed_form_propagator():
    rng = np.random.default_rng(3)
    n, L, lam, dz, nz = 64, 12.0, 0.02508, 1.7, 7
    psi = _band_limited(n, rng)
    P = ms.propagator(n, L, lam, dz)
    t = np.ones((n, n))
    y = psi
    for _ in range(nz):
        y = ms.slice_step(y, t, P)
    p = ms.fft_index(n).astype(float)
    closed = ms.band_limit(n) * np.exp(-1j * math.pi * lam * nz * dz
                                       * (p[None] ** 2 + p[:, None] ** 2) / L ** 2)
    ref = np.fft.ifft2(closed * np.fft.fft2(psi))
    assert np.allclose(y, ref, atol=1e-13 * np.abs(ref).max())


def test_paraxial_gaussian_beam_matches_fresnel_solution():
    """exp(-r^2/(2 w0^2)) spreads as (w0^2/w^2) exp(-r^2/(2 w^2)), w^2 = w0^2 + i lambda z/(2 pi)."""
    n, L, lam, dz, nz, w0 = 256, 16.0, 0.02508, 5.0, 20, 0.5
    x = np.arange(n) * L / n
    d = x - L / 2
    X, Y = np.meshgrid(d, d)
    r2 = X ** 2 + Y ** 2
    psi = np.exp(-r2 / (2 * w0 ** 2)).astype(np.complex128)
    P = ms.propagator(n, L, lam, dz)
    y = psi
    for _ in range(nz):
        y = ms.slice_step(y, np.ones((n, n)), P)
    w2 = w0 ** 2 + 1j * lam * nz * dz / (2 * math.pi)
    ref = (w0 ** 2 / w2) * np.exp(-r2 / (2 * w2))
    assert np.abs(y - ref).max() < 1e-10


def test_transmission_phase_focuses_like_a_converging_lens():
    """Eq. 3 with the propagator: a slice whose projected potential falls off as -kappa r^2
    is a thin converging lens of focal length pi / (lambda sigma kappa).  A Gaussian beam
    through it and 50 A of free space follows the complex-width solution, brightening on
    axis towards the focus (with the phase sign reversed it would spread instead)."""
    n, L, lam, dz, nz, w0 = 256, 16.0, 0.02508, 2.5, 20, 0.5
    sigma = 7.2886e-4
    kappa = math.pi / (lam * sigma * 50.0)          # focal length 50 A
    x = np.arange(n) * L / n
    d = x - L / 2
    X, Y = np.meshgrid(d, d)
    r2 = X ** 2 + Y ** 2
    psi = np.exp(-r2 / (2 * w0 ** 2)).astype(np.complex128)
    P = ms.propagator(n, L, lam, dz)
    y = ms.slice_step(psi, ms.transmission(-kappa * r2, sigma), P)
    for _ in range(nz - 1):
        y = ms.slice_step(y, np.ones((n, n)), P)
    a = 1 / (2 * w0 ** 2) + 1j * sigma * kappa        # exp(-a r^2) after the lens
    w2 = 1 / (2 * a) + 1j * lam * nz * dz / (2 * math.pi)
    ref = (1 / (2 * a * w2)) * np.exp(-r2 / (2 * w2))
    assert np.abs(y - ref).max() < 1e-10
    assert abs(y[n // 2, n // 2]) ** 2 > 1.5


def test_adjoint_of_slice_step():
    rng = np.random.default_rng(4)
    n = 48
    t = ms.transmission(rng.standard_normal((n, n)) * 80, 7.3e-4)
    P = ms.propagator(n, 9.0, 0.02508, 2.0)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    y = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    lhs = np.vdot(lin.adjoint_step(x, t, P), y)
    rhs = np.vdot(x, ms.slice_step(y, t, P))
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


# --- probe and detector (Eq. illum; PRISM interpolation) ------------------------

def test_probe_has_unit_norm_per_periodic_image():
    for f in (1, 2, 3):
        n, L = 96, 9.0
        psi = ms.probe(n, L, 0.02508, f, 0.025, 1.234, 4.321)
        assert abs(np.linalg.norm(psi) ** 2 - f * f) < 1e-12


def test_f_lattice_detector_integral_is_exact_for_a_localised_wave():
    """f^2 sum over the whole f-lattice of |<k|psi>|^2 = ||psi||^2 if psi fits in an L/f box."""
    rng = np.random.default_rng(6)
    n = 48
    for f in (2, 3, 4):
        b = n // f
        psi = np.zeros((n, n), dtype=complex)
        psi[5:5 + b, 7:7 + b] = rng.standard_normal((b, b)) + 1j * rng.standard_normal((b, b))
        c = np.fft.fft2(psi, norm="ortho")[::f, ::f]
        assert abs(f * f * np.sum(np.abs(c) ** 2) - np.linalg.norm(psi) ** 2) < 1e-10


# --- whole pipeline -------------------------------------------------------------

def test_thin_single_atom_limit_is_fourier_transform_of_H_times_probe():
    """n_z = 1, v = 0: I(R) = f^2 sum_d |(4/N) sum_m H(m) psi_R(2m) exp(-2 pi i f p_d.m/(N/2))|^2,
    evaluated as direct sums (no FFT)."""
    n, L, f = 32, 6.0, 1
    wl = _tiny(n=n, f=f, n_z=1, n_sites=1, w=10, alpha=0.02, beta=0.03, cell=L, scan_n=2, seed=7)
    wl.vproj[:] = 0.0
    wl.site_slice[:] = 0
    I = ms.quadratic_map(wl)
    nh = n // 2
    bp, bq = ms.lattice_beams(n, L, wl.lam, f, wl.alpha)
    dp, dq = ms.lattice_beams(n, L, wl.lam, f, wl.beta)
    c = f / math.sqrt(bp.size)
    rx, ry = wl.scan_positions()
    my, mx = np.meshgrid(np.arange(nh), np.arange(nh), indexing="ij")
    win = np.zeros((nh, nh), dtype=complex)
    rows = (wl.win_y0[0] + np.arange(wl.w)) % nh
    cols = (wl.win_x0[0] + np.arange(wl.w)) % nh
    for m in range(wl.n_types):
        win[:] = 0
        win[np.ix_(rows, cols)] = wl.H[0, m]
        for iy in range(2):
            for ix in range(2):
                X = 2 * mx * L / n
                Y = 2 * my * L / n
                psi = np.zeros((nh, nh), dtype=complex)
                for p, q in zip(bp, bq):
                    psi += c * np.exp(2j * math.pi * f * (p * (X - rx[ix]) + q * (Y - ry[iy])) / L) / n
                tot = 0.0
                for p, q in zip(dp, dq):
                    amp = (4.0 / n) * np.sum(win * psi * np.exp(-2j * math.pi * f * (p * mx + q * my) / nh))
                    tot += abs(amp) ** 2
                assert abs(f * f * tot - I[m, iy, ix]) < 1e-12 * I[m].max()


@pytest.mark.parametrize("f", [2, 3])
def test_thin_single_atom_limit_with_prism_windows(f):
    """f > 1, n_z = 1, v = 0 (Sec. III, Sec. IV C): probe R sees the site only when the
    minimum-image displacement r_s - R lies in [-L/2f, L/2f) on both axes; there I(R) is
    f^2 sum_d of the direct-sum Fourier transform of H times the f-lattice probe, elsewhere
    zero.  The window test and the sums are written out here, apart from the oracle."""
    n, L = 32, 6.0
    wl = _tiny(n=n, f=f, n_z=1, n_sites=1, w=10, alpha=0.02, beta=0.03, cell=L, scan_n=16,
               seed=1)
    wl.vproj[:] = 0.0
    wl.site_slice[:] = 0
    I = ms.quadratic_map(wl)
    nh = n // 2
    bp, bq = ms.lattice_beams(n, L, wl.lam, f, wl.alpha)
    dp, dq = ms.lattice_beams(n, L, wl.lam, f, wl.beta)
    c = f / math.sqrt(bp.size)
    rx, ry = wl.scan_positions()
    half = L / (2 * f)

    def inside(s, r):
        d = s - r
        d -= L * math.floor(d / L + 0.5)
        return -half <= d < half

    my, mx = np.meshgrid(np.arange(nh), np.arange(nh), indexing="ij")
    X, Y = 2 * mx * L / n, 2 * my * L / n
    rows = (wl.win_y0[0] + np.arange(wl.w)) % nh
    cols = (wl.win_x0[0] + np.arange(wl.w)) % nh
    seen = set()
    for m in range(wl.n_types):
        win = np.zeros((nh, nh), dtype=complex)
        win[np.ix_(rows, cols)] = wl.H[0, m]
        for iy in range(rx.size):
            for ix in range(rx.size):
                hit = inside(wl.site_x[0], rx[ix]) and inside(wl.site_y[0], ry[iy])
                seen.add(hit)
                if not hit:
                    assert I[m, iy, ix] == 0.0
                    continue
                psi = np.zeros((nh, nh), dtype=complex)
                for p, q in zip(bp, bq):
                    psi += c * np.exp(2j * math.pi * f * (p * (X - rx[ix]) + q * (Y - ry[iy])) / L) / n
                tot = 0.0
                for p, q in zip(dp, dq):
                    amp = (4.0 / n) * np.sum(win * psi * np.exp(-2j * math.pi * f * (p * mx + q * my) / nh))
                    tot += abs(amp) ** 2
                assert abs(f * f * tot - I[m, iy, ix]) < 1e-12 * I[m].max()
    assert seen == {True, False}   # the scan reaches both sides of the window edge


@pytest.mark.parametrize("n,f,cell,alpha,beta", [(16, 1, 4.0, 0.0138, 0.018),
                                                 (32, 2, 8.0, 0.0138, 0.018),
                                                 (32, 1, 6.0, 0.02, 0.03)])
def test_quadratic_equals_dense_matrix_evaluation(n, f, cell, alpha, beta):
    wl = _tiny(n=n, f=f, cell=cell, alpha=alpha, beta=beta, seed=11 + n + f)
    Iq = ms.quadratic_map(wl)
    Id = dense.dense_map(wl)
    assert Iq.max() > 0
    assert ms.relative_error(Id, Iq) < 1e-12


@pytest.mark.parametrize("n,f,cell,alpha,beta,seed", [(32, 1, 6.0, 0.02, 0.03, 1),
                                                      (64, 2, 12.0, 0.02, 0.03, 2),
                                                      (96, 3, 15.0, 0.02, 0.03, 3)])
def test_linear_algorithm_adds_no_error(n, f, cell, alpha, beta, seed):
    """Abstract / Sec. IV A: the scattering-matrix algorithm reproduces the conventional map."""
    wl = _tiny(n=n, f=f, cell=cell, alpha=alpha, beta=beta, seed=seed, n_z=4, n_sites=6, w=8,
               scan_n=3)
    Iq = ms.quadratic_map(wl)
    Il = lin.linear_map(wl)
    assert Iq.max() > 0
    assert ms.relative_error(Iq, Il) < 1e-12


# --- S_2 schemes of Alg. 2: recalculated per slice (Sec. III), inverse multislice (Sec. IV C)

@pytest.mark.parametrize("n,f,cell,seed", [(32, 1, 6.0, 1), (64, 2, 12.0, 2)])
def test_recalculated_s2_reproduces_the_conventional_map(n, f, cell, seed):
    """The listing recalculates S_2 from the exit surface at every slice: exact."""
    wl = _tiny(n=n, f=f, cell=cell, alpha=0.02, beta=0.03, seed=seed, n_z=4, n_sites=6, w=8,
               scan_n=3)
    Iq = ms.quadratic_map(wl)
    assert Iq.max() > 0
    assert ms.relative_error(Iq, lin.linear_map(wl, scheme="recompute")) < 1e-12


def test_inverse_multislice_is_exact_in_free_space():
    """With v = 0 nothing leaves the band, so the retreat undoes the backward step."""
    wl = _tiny(n=32, f=1, cell=6.0, alpha=0.02, beta=0.03, seed=6, n_z=4, n_sites=6, w=8)
    wl.vproj = np.zeros_like(wl.vproj)
    Iq = ms.quadratic_map(wl)
    assert Iq.max() > 0
    assert ms.relative_error(Iq, lin.linear_map(wl, scheme="inverse")) < 1e-12


def test_inverse_multislice_is_exact_at_the_entrance_slice():
    """S_2 at depth 0 comes from the full backward sweep; only deeper slices are retreated."""
    wl = _tiny(n=32, f=1, cell=6.0, alpha=0.02, beta=0.03, seed=7, n_z=4, n_sites=6, w=8)
    wl.vproj = (wl.vproj * 4.0).astype(np.float32)        # strong scattering
    first = wl.with_sites(np.arange(wl.n_sites))
    first.site_slice[:] = 0
    Iq = ms.quadratic_map(first)
    assert ms.relative_error(Iq, lin.linear_map(first, scheme="inverse")) < 1e-12
    deep = wl.with_sites(np.arange(wl.n_sites))
    deep.site_slice[:] = wl.n_z - 1
    Iq = ms.quadratic_map(deep)
    assert ms.relative_error(Iq, lin.linear_map(deep, scheme="inverse")) > 1e-4


def test_inverse_multislice_is_exact_while_the_waves_stay_in_band():
    """Slices of weak single-harmonic potentials v_i = A cos(2 pi (a_i x + b_i y)/L + phi_i)
    with sigma A = 0.1: t_i has harmonics of order m with weight ~ J_m(0.1), and reaching
    the band edge from the small apertures needs six orders (~1e-11).  The retreat must
    then reproduce the conventional map, which requires the transmission of the right
    slice at every retreat step (the potentials change the map by far more than 1e-6)."""
    n, cell = 32, 8.0
    wl = _tiny(n=n, f=1, cell=cell, alpha=0.008, beta=0.008, seed=8, n_z=4, n_sites=6, w=8,
               scan_n=3)
    x = np.arange(n) * cell / n
    amp = 0.1 / wl.sigma
    freqs = [(1, 0, 0.3), (0, 1, 1.7), (1, 1, 2.9), (1, -1, 4.1)]
    v = np.empty((wl.n_z, n, n))
    for i, (a, b, ph) in enumerate(freqs):
        v[i] = amp * np.cos(2 * math.pi * (a * x[None, :] + b * x[:, None]) / cell + ph)
    wl.vproj = v.astype(np.float32)
    Iq = ms.quadratic_map(wl)
    assert ms.relative_error(Iq, lin.linear_map(wl, scheme="inverse")) < 1e-6
    free = wl.with_sites(np.arange(wl.n_sites))
    free.vproj = np.zeros_like(wl.vproj)
    assert ms.relative_error(Iq, ms.quadratic_map(free)) > 1e-2


def test_linear_equals_quadratic_on_rocksalt_probes():
    wl = sp.rocksalt_small()
    pos = [(0, 0), (3, 5), (7, 2)]
    Iq = ms.quadratic_map(wl, positions=pos)
    Il = lin.linear_map(wl)
    for iy, ix in pos:
        assert np.abs(Iq[:, iy, ix] - Il[:, iy, ix]).max() < 1e-12 * Il.max()


def test_mirror_symmetry_of_rocksalt_map():
    """H_{-1}(x,-y) = H_{+1}(x,y); the crystal and probe are mirror-symmetric about an Fe
    column, so I_{-1}(x, y) = I_{+1}(x, -y) and I_0 is mirror-symmetric."""
    wl = sp.rocksalt_small()
    pos = [(1, 2), (7, 2), (3, 6), (5, 6)]     # pairs (iy, ix) and ((8 - iy) % 8, ix)
    I = ms.quadratic_map(wl, positions=pos)
    for (a, b) in ((pos[0], pos[1]), (pos[2], pos[3])):
        scale = I[:, a[0], a[1]].max()
        assert abs(I[0, a[0], a[1]] - I[2, b[0], b[1]]) < 1e-8 * scale
        assert abs(I[1, a[0], a[1]] - I[1, b[0], b[1]]) < 1e-8 * scale
        assert abs(I[0, a[0], a[1]] - I[2, a[0], a[1]]) > 1e-5 * scale  # not equal by accident


def test_map_scales_with_transition_amplitude_squared():
    wl = _tiny(n=32, f=1, cell=6.0, alpha=0.02, beta=0.03, seed=9)
    I1 = ms.quadratic_map(wl)
    wl.H = (wl.H * 3.0).astype(np.complex64)
    I3 = ms.quadratic_map(wl)
    assert ms.relative_error(9 * I1, I3) < 1e-6


def test_multislice_count_matches_paper_formula():
    """Sec. III: N_MS = sum_iz n_states (n_z - iz) + n_z per probe position."""
    wl = sp.rocksalt_small()
    c = {}
    ms.quadratic_map(wl, positions=[(2, 3)], counter=c)
    n_states = 8 * wl.n_types        # 8 Fe per slice in the 2x2 cell, every transition counted
    nz = wl.n_z
    assert c["steps"] == sum(n_states * (nz - i) for i in range(nz)) + nz


def test_window_rule_at_f1_admits_every_site_once():
    rng = np.random.default_rng(12)
    L = 7.0
    s = rng.random(200) * L * 3 - L
    r = rng.random(200) * L
    assert ms.axis_in_window(s, r, L, 1).all()
    # at f = 2, exactly one of the two half-cells of the periodic line admits a point
    a = ms.axis_in_window(s, r, L, 2)
    b = ms.axis_in_window(s, r + L / 2, L, 2)
    assert np.all(a ^ b)


# --- crop windows (Sec. IV B) -------------------------------------------------------

def test_cropped_window_equals_full_window_zeroed_outside_the_crop():
    """A w-pixel crop of the dopant's transition potential gives the map of the full
    (whole-cell) window with H set to zero outside the same w x w pixels, and the crop
    error falls as the crop grows (the long tail is cut less)."""
    full = sp.dopant_slab(64, n=64, nzc=3, scan_n=6)
    s_in = lin.build_s_in(full)
    ref = lin.linear_map(full, s_in=s_in)
    errs = []
    for w in (8, 16, 24):
        crop = sp.dopant_slab(w, n=64, nzc=3, scan_n=6)
        got = lin.linear_map(crop, s_in=s_in)
        # the same pixels inside the full window: offsets of the centred origins
        off = (full.w // 2) - (w // 2)
        zeroed = full.with_sites([0])
        Hz = np.zeros_like(full.H)
        Hz[:, :, off:off + w, off:off + w] = full.H[:, :, off:off + w, off:off + w]
        zeroed.H = Hz
        assert np.array_equal(Hz[:, :, off:off + w, off:off + w], crop.H)
        assert ms.relative_error(lin.linear_map(zeroed, s_in=s_in), got) < 1e-12
        errs.append(ms.relative_error(ref, got))
    assert errs[0] > errs[1] > errs[2] > 0


# --- frozen phonons ------------------------------------------------------------------

def test_phonon_configurations_have_the_requested_displacements():
    cfg = sp.rocksalt_phonons(4, u_rms=0.08, ncell=4, nzc=2, n=128, f=2, scan_n=4, w=16)
    ref = sp.rocksalt_phonons(1, u_rms=0.0, ncell=4, nzc=2, n=128, f=2, scan_n=4, w=16)[0]
    L = ref.cell
    d = np.concatenate([((c.site_x - ref.site_x + L / 2) % L - L / 2) for c in cfg] +
                       [((c.site_y - ref.site_y + L / 2) % L - L / 2) for c in cfg])
    assert abs(d.mean()) < 4 * 0.08 / math.sqrt(d.size)
    assert abs(d.std() / 0.08 - 1.0) < 4 / math.sqrt(2 * d.size)
    assert all(np.array_equal(c.site_slice, ref.site_slice) for c in cfg)


def test_phonon_average_is_the_mean_of_conventional_passes():
    """The average over configurations equals the mean of the conventional (quadratic)
    maps of the passes; with no displacement every pass is the static map."""
    from oracle import phonon
    cfg = sp.rocksalt_phonons(3, u_rms=0.1, ncell=2, nzc=2, n=64, f=1, scan_n=3, w=10)
    avg = phonon.average_map(cfg)
    quad = sum(ms.quadratic_map(c) for c in cfg) / len(cfg)
    assert avg.max() > 0 and ms.relative_error(quad, avg) < 1e-12
    assert ms.relative_error(lin.linear_map(cfg[0]), avg) > 1e-4     # the passes differ
    still = sp.rocksalt_phonons(2, u_rms=0.0, ncell=2, nzc=2, n=64, f=1, scan_n=3, w=10)
    assert ms.relative_error(ms.quadratic_map(still[0]), phonon.average_map(still)) < 1e-12
