"""ctypes binding of libstemeels.so (include/stem_eels.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Arrays may be numpy arrays (host) or torch CUDA tensors (device); the
binding passes their pointers and the matching host/device flag.  If the shared
object is missing or fails to load, every call raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# STEM_CHECK=1: the bounds-checked debug build (build.build(check=True))
LIB_PATH = (os.path.join(_HERE, "_build_check", "libstemeels_check.so")
            if os.environ.get("STEM_CHECK", "") == "1"
            else os.path.join(_HERE, "_build", "libstemeels.so"))

EELS_PREC = {"fp32": 0, "tf32": 1, "bf16x3": 2}
_STATUS = {0: "EELS_OK", 1: "EELS_ERR_ARG", 2: "EELS_ERR_UNSUPPORTED", 3: "EELS_ERR_OOM",
           4: "EELS_ERR_CUDA", 5: "EELS_ERR_TIMEOUT", 6: "EELS_ERR_CANCELLED",
           7: "EELS_ERR_NONFINITE", 8: "EELS_ERR_BOUNDS"}


class EelsError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Specimen(C.Structure):
    _fields_ = [("n", C.c_int), ("n_z", C.c_int), ("cell", C.c_double),
                ("vproj", C.c_void_p), ("vproj_on_device", C.c_int)]


class Optics(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("sigma", C.c_double), ("dz", C.c_double),
                ("f", C.c_int), ("alpha", C.c_double)]


class Transitions(C.Structure):
    _fields_ = [("n_sites", C.c_int), ("n_types", C.c_int), ("w", C.c_int),
                ("H", C.c_void_p), ("slice", C.c_void_p), ("win_x0", C.c_void_p),
                ("win_y0", C.c_void_p), ("x", C.c_void_p), ("y", C.c_void_p),
                ("on_device", C.c_int), ("h_shared", C.c_int)]


class Scan(C.Structure):
    _fields_ = [("n_sx", C.c_int), ("n_sy", C.c_int), ("x0", C.c_double), ("y0", C.c_double),
                ("step_x", C.c_double), ("step_y", C.c_double)]


class Request(C.Structure):
    _fields_ = [("spec", Specimen), ("optics", Optics), ("tr", Transitions), ("scan", Scan),
                ("beta", C.c_double), ("precision", C.c_int), ("deadline_s", C.c_double),
                ("sin_checkpoint", C.c_int)]


class RequestInfo(C.Structure):
    _fields_ = [("done", C.c_int), ("status", C.c_int), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_first_tile", C.c_double), ("t_done", C.c_double),
                ("tiles", C.c_int), ("footprint", C.c_int64), ("n_in", C.c_int),
                ("n_out", C.c_int), ("pixel_slices", C.c_int64), ("wave_steps", C.c_int64),
                ("contraction_flops", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("cancelled", C.c_int64), ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("max_ms", C.c_double), ("mean_wait_ms", C.c_double), ("makespan_s", C.c_double),
                ("pixel_slices_per_s", C.c_double), ("peak_bytes", C.c_int64)]


class Detector(C.Structure):
    _fields_ = [("inner", C.c_double), ("outer", C.c_double)]


EXPORTS = {
    "eels_create": (C.c_int, [C.c_int, C.POINTER(C.c_void_p)]),
    "eels_destroy": (None, [C.c_void_p]),
    "eels_last_error": (C.c_char_p, [C.c_void_p]),
    "eels_build_smatrix": (C.c_int, [C.c_void_p, C.POINTER(Specimen), C.POINTER(Optics),
                                     C.c_void_p, C.POINTER(C.c_void_p)]),
    "eels_smatrix_free": (None, [C.c_void_p]),
    "eels_smatrix_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                    C.POINTER(C.c_int)]),
    "eels_smatrix_beams": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "eels_smatrix_copy_depth": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "eels_fp32_fma_rate": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "eels_checked_build": (C.c_int, []),
    "eels_inelastic_map": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Transitions),
                                     C.POINTER(Scan), C.c_double, C.c_int, C.c_void_p, C.c_int,
                                     C.c_void_p]),
    "eels_inelastic_map_tiles": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Transitions),
                                           C.POINTER(Scan), C.c_double, C.c_int, C.c_int, C.c_int,
                                           C.c_void_p, C.c_void_p, C.c_int,
                                           C.POINTER(C.c_int), C.c_void_p]),
    "eels_quadratic_reference_map": (C.c_int, [C.c_void_p, C.POINTER(Specimen), C.POINTER(Optics),
                                               C.POINTER(Transitions), C.POINTER(Scan), C.c_double,
                                               C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                                               C.c_void_p, C.POINTER(C.c_int64)]),
    "eels_elastic_images": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Scan),
                                      C.POINTER(Detector), C.c_int, C.c_void_p, C.c_int,
                                      C.c_void_p]),
    "eels_divide_map": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int64,
                                  C.c_int, C.c_void_p]),
    "eels_phonon_map": (C.c_int, [C.c_void_p, C.POINTER(Specimen), C.POINTER(Transitions),
                                  C.c_int, C.POINTER(Optics), C.POINTER(Scan), C.c_double,
                                  C.c_int, C.c_void_p, C.c_int, C.c_void_p]),
    "eels_set_option": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "eels_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "eels_tuning_read": (C.c_int, [C.c_void_p, C.c_char_p, C.c_int]),
    "eels_profile_read": (C.c_int, [C.c_void_p, C.c_char_p, C.c_int]),
    "eels_build_smatrix_static": (C.c_int, [C.POINTER(Specimen), C.POINTER(Optics), C.c_void_p,
                                            C.c_int64, C.POINTER(C.c_int), C.c_void_p,
                                            C.c_char_p, C.c_int]),
    "eels_request_footprint": (C.c_int64, [C.POINTER(Request)]),
    "eels_server_create": (C.c_int, [C.c_int, C.c_int64, C.c_int, C.POINTER(C.c_void_p)]),
    "eels_server_submit": (C.c_int, [C.c_void_p, C.POINTER(Request), C.POINTER(C.c_int64)]),
    "eels_server_wait": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_double,
                                   C.POINTER(C.c_double)]),
    "eels_server_stats_get": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "eels_server_cancel": (C.c_int, [C.c_void_p, C.c_int64]),
    "eels_server_request_info": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(RequestInfo)]),
    "eels_server_destroy": (None, [C.c_void_p]),
    "eels_count_beams": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_int, C.c_double]),
    "eels_memory_model": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int64)]),
    "eels_footprint_bytes": (C.c_int64, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
}

_lib = None


def load():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libstemeels.so not built ({LIB_PATH}); run "
                               "paper_1908_07628_gb300.build.build()")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _is_cuda_tensor(a) -> bool:
    return type(a).__module__.startswith("torch") and getattr(a, "is_cuda", False)


def _ptr(a, dtype):
    """(pointer, on_device, keepalive) of a contiguous array of the given numpy dtype."""
    if _is_cuda_tensor(a):
        import torch
        want = {np.float32: torch.float32, np.complex64: torch.complex64, np.float64: torch.float64,
                np.int32: torch.int32}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"device array must be a contiguous {want} tensor")
        return C.c_void_p(a.data_ptr()), 1, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(C.c_void_p), 0, arr


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


class Context:
    """An eels_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        self._lib = load()
        h = C.c_void_p()
        st = self._lib.eels_create(device, C.byref(h))
        if st != 0:
            raise EelsError(st, f"eels_create(device={device})")
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            self._lib.eels_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != 0:
            msg = self._lib.eels_last_error(self._h)
            raise EelsError(st, f"{what}: {msg.decode() if msg else ''}")

    ASSOCIATIONS = {"auto": 0, "transition_first": 1, "probe_first": 2, "model": 3}

    def set_association(self, how: str = "auto"):
        """Grouping of the tensor-core contraction (EELS_OPT_ASSOCIATION)."""
        self._check(self._lib.eels_set_option(self._h, 1, self.ASSOCIATIONS[how]), "set_option")

    def set_detector_shard(self, index: int = 0, count: int = 1):
        """Restrict inelastic_map to detector beams d with d % count == index
        (EELS_OPT_SHARD_COUNT / EELS_OPT_SHARD_INDEX); (0, 1) is the whole aperture."""
        self._check(self._lib.eels_set_option(self._h, 2, int(count)), "set_option")
        self._check(self._lib.eels_set_option(self._h, 3, int(index)), "set_option")

    def set_exit_plane(self, on: bool = True):
        """Builds also keep S_in at the exit surface (EELS_OPT_EXIT_PLANE), for elastic_images."""
        self._check(self._lib.eels_set_option(self._h, 5, 1 if on else 0), "set_option")

    def set_batch_sites(self, cap: int = 0):
        """At most `cap` sites of a slice per tensor-core contraction batch
        (EELS_OPT_BATCH_SITES); 0 sizes batches by the operand memory budget."""
        self._check(self._lib.eels_set_option(self._h, 6, int(cap)), "set_option")

    def set_tile_width(self, cols: int = 0):
        """Output tile columns of the tensor-core GEMMs (EELS_OPT_TILE_WIDTH): 0 lets the
        library choose (measured under the AUTO grouping), 128 or 256 forces a width."""
        self._check(self._lib.eels_set_option(self._h, 10, int(cols)), "set_option")

    def set_operand_budget(self, mib: int = 8192):
        """Device memory (MiB) for one batch's tensor-core operands (EELS_OPT_OPERAND_MIB)."""
        self._check(self._lib.eels_set_option(self._h, 9, int(mib)), "set_option")

    def set_sin_checkpoint(self, k: int = 0):
        """Builds keep the probe waves every k slices instead of S_in at every depth
        (EELS_OPT_SIN_CHECKPOINT); maps recompute S_in segment by segment.  0: off."""
        self._check(self._lib.eels_set_option(self._h, 8, int(k)), "set_option")

    def set_wait_test(self, kcycles: int = 0):
        """Failure-detection test mode (EELS_OPT_WAIT_TEST): kcycles > 0 limits the
        tensor-core pipeline waits to 1000 * kcycles clock cycles and withholds every TMA
        load, so the waits run out; 0 restores normal operation."""
        self._check(self._lib.eels_set_option(self._h, 7, int(kcycles)), "set_option")

    def set_check_test(self, on: int = 1):
        """Bounds-checked build test (EELS_OPT_CHECK_TEST): the next maps get a window
        origin one past its range, which the checked kernels report (EELS_ERR_BOUNDS)."""
        self._check(self._lib.eels_set_option(self._h, 11, int(on)), "set_option")

    def elastic_images(self, sm, scan, detectors, out=None, stream=None):
        """Elastic images [n_det][n_sy][n_sx] (FP64) for detectors [(inner, outer), ...]
        (semi-angles in rad; outer <= 0: up to the band limit)."""
        dets = (Detector * len(detectors))(*[Detector(float(a), float(b)) for a, b in detectors])
        sc = Scan(*[int(v) for v in scan[:2]], *[float(v) for v in scan[2:]])
        shape = (len(detectors), int(scan[1]), int(scan[0]))
        out_arr = np.zeros(shape) if out is None else out
        o, o_dev, okeep = _ptr(out_arr, np.float64)
        st = self._lib.eels_elastic_images(self._h, sm._h, C.byref(sc), dets, len(detectors), o,
                                           o_dev, _stream(stream))
        self._check(st, "eels_elastic_images")
        if out is None or not o_dev:
            if o_dev == 0 and out is not None and okeep is not out:
                out[...] = okeep
            return okeep if out is None else out
        return out

    def phonon_map(self, configs, precision="fp32", out=None, stream=None):
        """eels_phonon_map over workload-like configurations (same grid, optics, scan,
        beta and channels; each with its own vproj, H and sites): the mean map."""
        c0 = configs[0]
        specs = (Specimen * len(configs))()
        trs = (Transitions * len(configs))()
        keep = []
        for i, wl in enumerate(configs):
            v, v_dev, vk = _ptr(wl.vproj, np.float32)
            specs[i] = Specimen(int(wl.n), int(wl.n_z), float(wl.cell), v, v_dev)
            tr, tk = _transitions(wl.H, wl.site_slice, wl.win_x0, wl.win_y0, wl.site_x, wl.site_y)
            trs[i] = tr
            keep += [vk, tk]
        op = Optics(float(c0.lam), float(c0.sigma), float(c0.dz), int(c0.f), float(c0.alpha))
        sc = Scan(*[int(v) for v in c0.scan[:2]], *[float(v) for v in c0.scan[2:]])
        shape = (int(c0.H.shape[-3]), int(c0.scan[1]), int(c0.scan[0]))
        out_arr = np.zeros(shape) if out is None else out
        o, o_dev, okeep = _ptr(out_arr, np.float64)
        st = self._lib.eels_phonon_map(self._h, specs, trs, len(configs), C.byref(op), C.byref(sc),
                                       float(c0.beta), EELS_PREC[precision], o, o_dev,
                                       _stream(stream))
        del keep
        self._check(st, "eels_phonon_map")
        if out is None or not o_dev:
            if o_dev == 0 and out is not None and okeep is not out:
                out[...] = okeep
            return okeep if out is None else out
        return out

    def divide_map(self, eels_map, bf, stream=None):
        """In place: eels_map[m] /= bf (the bright-field correction); both numpy FP64
        arrays or both CUDA FP64 tensors.  Returns eels_map."""
        m_ptr, m_dev, mkeep = _ptr(eels_map, np.float64)
        b_ptr, b_dev, bkeep = _ptr(bf, np.float64)
        if m_dev != b_dev:
            raise ValueError("map and bright field must both be on the host or the device")
        n_pix = int(bf.shape[-1] * bf.shape[-2])
        st = self._lib.eels_divide_map(self._h, m_ptr, b_ptr, int(eels_map.shape[0]), n_pix, m_dev,
                                       _stream(stream))
        self._check(st, "eels_divide_map")
        if not m_dev and mkeep is not eels_map:
            eels_map[...] = mkeep
        return eels_map

    SOUT_SCHEMES = {"stream": 0, "recompute": 1, "inverse": 2}

    def set_sout_scheme(self, how: str = "stream"):
        """How S_out reaches each depth (EELS_OPT_SOUT_SCHEME): "stream", "recompute"
        (the Sec. III listing) or "inverse" (inverse multislice, Sec. IV C)."""
        self._check(self._lib.eels_set_option(self._h, 4, self.SOUT_SCHEMES[how]), "set_option")

    def profile_enable(self, on: bool = True):
        self._check(self._lib.eels_profile_enable(self._h, 1 if on else 0), "profile_enable")

    def tuning_read(self) -> list:
        """The autotuner's choices per contraction shape (eels_tuning_read)."""
        import json
        need = self._lib.eels_tuning_read(self._h, None, 0)
        buf = C.create_string_buffer(max(need, 1))
        self._lib.eels_tuning_read(self._h, buf, need)
        return json.loads(buf.value.decode() or "[]")

    def profile_read(self) -> dict:
        """Per-kernel {launches, ms} recorded since the last read (clears the records)."""
        import json
        need = self._lib.eels_profile_read(self._h, None, 0)
        buf = C.create_string_buffer(max(need, 2))
        self._lib.eels_profile_read(self._h, buf, len(buf))
        return json.loads(buf.value.decode() or "{}")

    # -- the three calls of the method --------------------------------------------------

    def build_smatrix(self, vproj, cell, lam, sigma, dz, f, alpha, stream=None) -> "SMatrix":
        """eels_build_smatrix: S_in at every depth for the probe aperture alpha."""
        v, on_dev, keep = _ptr(vproj, np.float32)
        n_z, n = int(vproj.shape[0]), int(vproj.shape[-1])
        spec = Specimen(n, n_z, float(cell), v, on_dev)
        op = Optics(float(lam), float(sigma), float(dz), int(f), float(alpha))
        h = C.c_void_p()
        st = self._lib.eels_build_smatrix(self._h, C.byref(spec), C.byref(op), _stream(stream),
                                          C.byref(h))
        del keep
        self._check(st, "eels_build_smatrix")
        return SMatrix(self, h)

    def inelastic_map(self, sm, H, site_slice, win_x0, win_y0, site_x, site_y, scan, beta,
                      precision="fp32", out=None, stream=None):
        """eels_inelastic_map: FP64 map [n_types][n_sy][n_sx] (numpy, or into a CUDA tensor)."""
        tr, keep = _transitions(H, site_slice, win_x0, win_y0, site_x, site_y)
        sc = Scan(*[int(v) for v in scan[:2]], *[float(v) for v in scan[2:]])
        shape = (int(H.shape[-3]), int(scan[1]), int(scan[0]))
        out_arr = np.zeros(shape) if out is None else out
        o, o_dev, okeep = _ptr(out_arr, np.float64)
        st = self._lib.eels_inelastic_map(self._h, sm._h, C.byref(tr), C.byref(sc), float(beta),
                                          EELS_PREC[precision], o, o_dev, _stream(stream))
        del keep
        self._check(st, "eels_inelastic_map")
        if out is None or not o_dev:
            if o_dev == 0 and out is not None and okeep is not out:
                out[...] = okeep
            return okeep if out is None else out
        return out

    def inelastic_map_tiles(self, sm, H, site_slice, win_x0, win_y0, site_x, site_y, scan, beta,
                            tile, map_out, tile_done, precision="fp32", max_tiles=0,
                            stream=None):
        """eels_inelastic_map_tiles: maps the scan tiles (tile = (tile_nx, tile_ny)) not yet
        marked in tile_done into map_out, both numpy arrays updated in place (map_out float64
        [n_types][n_sy][n_sx], tile_done uint8 [gy][gx]); at most max_tiles tiles (0: all).
        Returns the number of tiles left.  On an error the finished tiles stay written and
        marked, and the EelsError is raised."""
        tnx, tny = int(tile[0]), int(tile[1])
        n_sx, n_sy = int(scan[0]), int(scan[1])
        if tnx < 1 or tny < 1:
            raise ValueError("scan tiles need at least one position")
        gx, gy = -(-n_sx // tnx), -(-n_sy // tny)
        shape = (int(H.shape[-3]), n_sy, n_sx)
        if not (isinstance(map_out, np.ndarray) and map_out.dtype == np.float64
                and map_out.shape == shape and map_out.flags.c_contiguous):
            raise TypeError(f"map_out must be a C-contiguous float64 numpy array {shape}")
        if not (isinstance(tile_done, np.ndarray) and tile_done.dtype == np.uint8
                and tile_done.size == gx * gy and tile_done.flags.c_contiguous):
            raise TypeError(f"tile_done must be a C-contiguous uint8 numpy array of {gx * gy}")
        tr, keep = _transitions(H, site_slice, win_x0, win_y0, site_x, site_y)
        sc = Scan(n_sx, n_sy, *[float(v) for v in scan[2:]])
        left = C.c_int(0)
        st = self._lib.eels_inelastic_map_tiles(
            self._h, sm._h, C.byref(tr), C.byref(sc), float(beta), EELS_PREC[precision], tnx,
            tny, map_out.ctypes.data, tile_done.ctypes.data, int(max_tiles), C.byref(left),
            _stream(stream))
        del keep
        self._check(st, "eels_inelastic_map_tiles")
        return int(left.value)

    def quadratic_reference_map(self, vproj, cell, lam, sigma, dz, f, alpha, H, site_slice,
                                win_x0, win_y0, site_x, site_y, scan, beta, positions=None,
                                stream=None):
        """eels_quadratic_reference_map: conventional algorithm on the GPU.  Returns (map, steps)."""
        v, on_dev, vkeep = _ptr(vproj, np.float32)
        n_z, n = int(vproj.shape[0]), int(vproj.shape[-1])
        spec = Specimen(n, n_z, float(cell), v, on_dev)
        op = Optics(float(lam), float(sigma), float(dz), int(f), float(alpha))
        tr, keep = _transitions(H, site_slice, win_x0, win_y0, site_x, site_y)
        sc = Scan(*[int(x) for x in scan[:2]], *[float(x) for x in scan[2:]])
        out = np.zeros((int(H.shape[-3]), int(scan[1]), int(scan[0])))
        steps = C.c_int64(0)
        if positions is None:
            pp, npos, pkeep = None, 0, None
        else:
            pkeep = np.ascontiguousarray(np.asarray(positions, dtype=np.int32).reshape(-1, 2))
            pp, npos = pkeep.ctypes.data_as(C.c_void_p), int(pkeep.shape[0])
        st = self._lib.eels_quadratic_reference_map(
            self._h, C.byref(spec), C.byref(op), C.byref(tr), C.byref(sc), float(beta), pp, npos,
            out.ctypes.data_as(C.c_void_p), 0, _stream(stream), C.byref(steps))
        del keep, vkeep, pkeep
        self._check(st, "eels_quadratic_reference_map")
        return out, int(steps.value)


class SMatrix:
    """Library-owned S_in handle (eels_smatrix)."""

    def __init__(self, ctx: Context, h):
        self.ctx = ctx
        self._h = h
        n, nz, nin = C.c_int(), C.c_int(), C.c_int()
        ctx._check(ctx._lib.eels_smatrix_info(h, C.byref(n), C.byref(nz), C.byref(nin)), "info")
        self.n, self.n_z, self.n_in = n.value, nz.value, nin.value

    def beams(self):
        p = np.zeros(self.n_in, dtype=np.int32)
        q = np.zeros(self.n_in, dtype=np.int32)
        self.ctx._check(self.ctx._lib.eels_smatrix_beams(self._h, p.ctypes.data_as(C.c_void_p),
                                                         q.ctypes.data_as(C.c_void_p)), "beams")
        return p, q

    def copy_depth(self, depth, dst, stream=None):
        """Copy S_in(depth) into a complex64 CUDA tensor [n_in][N/2][N/2]."""
        ptr, on_dev, _ = _ptr(dst, np.complex64)
        if not on_dev:
            raise TypeError("copy_depth needs a CUDA tensor")
        self.ctx._check(self.ctx._lib.eels_smatrix_copy_depth(self._h, int(depth), ptr,
                                                              _stream(stream)), "copy_depth")
        return dst

    def free(self):
        if self._h:
            self.ctx._lib.eels_smatrix_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _transitions(H, site_slice, win_x0, win_y0, site_x, site_y):
    """H is [S][T][w][w] (per site) or [T][w][w] (the same potentials at every site)."""
    h, h_dev, hk = _ptr(H, np.complex64)
    arrs = [np.ascontiguousarray(site_slice, dtype=np.int32),
            np.ascontiguousarray(win_x0, dtype=np.int32),
            np.ascontiguousarray(win_y0, dtype=np.int32),
            np.ascontiguousarray(site_x, dtype=np.float64),
            np.ascontiguousarray(site_y, dtype=np.float64)]
    ptrs = [a.ctypes.data_as(C.c_void_p) for a in arrs]
    shared = len(H.shape) == 3
    n_sites = int(arrs[0].shape[0])
    tshape = H.shape if shared else H.shape[1:]
    tr = Transitions(n_sites, int(tshape[0]), int(tshape[1]), h, *ptrs, h_dev, 1 if shared else 0)
    return tr, (hk, arrs)


def build_smatrix_static(vproj, cell, lam, sigma, dz, f, alpha, out, stream=None) -> int:
    """eels_build_smatrix_static: S_in into the complex64 CUDA tensor `out`
    ([n_z][n_in][N/2][N/2]) using only the library's static work array.  Returns n_in."""
    v, on_dev, keep = _ptr(vproj, np.float32)
    n_z, n = int(vproj.shape[0]), int(vproj.shape[-1])
    spec = Specimen(n, n_z, float(cell), v, on_dev)
    op = Optics(float(lam), float(sigma), float(dz), int(f), float(alpha))
    optr, o_dev, okeep = _ptr(out, np.complex64)
    if not o_dev:
        raise TypeError("out must be a CUDA tensor")
    n_in = C.c_int(0)
    err = C.create_string_buffer(256)
    st = load().eels_build_smatrix_static(C.byref(spec), C.byref(op), optr,
                                          int(out.numel() * out.element_size()), C.byref(n_in),
                                          _stream(stream), err, len(err))
    del keep, okeep
    if st != 0:
        raise EelsError(st, "eels_build_smatrix_static: " + err.value.decode())
    return int(n_in.value)


def fp32_fma_rate(device=0, iters=1 << 20) -> float:
    """eels_fp32_fma_rate: measured FP32 FMA flop/s of the device."""
    out = C.c_double(0.0)
    st = load().eels_fp32_fma_rate(int(device), int(iters), C.byref(out))
    if st != 0:
        raise EelsError(st, "eels_fp32_fma_rate")
    return out.value


def checked_build() -> bool:
    """True if the loaded library is the bounds-checked build (-DSTEM_CHECK)."""
    return bool(load().eels_checked_build())


def count_beams(n, cell, lam, f, angle) -> int:
    return int(load().eels_count_beams(int(n), float(cell), float(lam), int(f), float(angle)))


def memory_model(n, n_z, planes_in, planes_out):
    out = (C.c_int64 * 3)()
    st = load().eels_memory_model(int(n), int(n_z), int(planes_in), int(planes_out), out)
    if st != 0:
        raise EelsError(st, "eels_memory_model")
    return [int(v) for v in out]


def footprint_bytes(n, n_z, n_in, n_out, chunk) -> int:
    return int(load().eels_footprint_bytes(int(n), int(n_z), int(n_in), int(n_out), int(chunk)))


# -- convenience: unpack any object carrying the workload attributes ------------------------

def build_smatrix_for(ctx: Context, wl, vproj=None, stream=None) -> SMatrix:
    return ctx.build_smatrix(wl.vproj if vproj is None else vproj, wl.cell, wl.lam, wl.sigma,
                             wl.dz, wl.f, wl.alpha, stream=stream)


def inelastic_map_for(ctx: Context, sm: SMatrix, wl, precision="fp32", H=None, out=None,
                      stream=None):
    return ctx.inelastic_map(sm, wl.H if H is None else H, wl.site_slice, wl.win_x0, wl.win_y0,
                             wl.site_x, wl.site_y, wl.scan, wl.beta, precision=precision, out=out,
                             stream=stream)


def inelastic_map_tiles_for(ctx: Context, sm: SMatrix, wl, tile, map_out, tile_done,
                            precision="fp32", max_tiles=0, stream=None) -> int:
    return ctx.inelastic_map_tiles(sm, wl.H, wl.site_slice, wl.win_x0, wl.win_y0, wl.site_x,
                                   wl.site_y, wl.scan, wl.beta, tile, map_out, tile_done,
                                   precision=precision, max_tiles=max_tiles, stream=stream)


def resumable_map(ctx: Context, sm: SMatrix, wl, tile, path, precision="fp32", max_tiles=0,
                  stream=None):
    """Map of wl per scan tile with an FP64 checkpoint file at path (.npz): the partial
    map and the tile marks are loaded from it if it exists (it must belong to the same
    scan, tiling, channel count and precision), and written back (to a temporary file,
    then renamed) after every finished tile, so a process that stops between tiles loses
    no finished tile.  At most max_tiles tiles this call (0: all).  Returns (map, tiles
    left)."""
    tnx, tny = int(tile[0]), int(tile[1])
    n_sx, n_sy = int(wl.scan[0]), int(wl.scan[1])
    gx, gy = -(-n_sx // tnx), -(-n_sy // tny)
    key = np.array([n_sx, n_sy, tnx, tny, int(wl.H.shape[-3]), EELS_PREC[precision]],
                   dtype=np.int64)
    if os.path.exists(path):
        with np.load(path) as z:
            if not np.array_equal(z["key"], key):
                raise ValueError(f"checkpoint {path} belongs to another map")
            map_out = np.ascontiguousarray(z["map"], dtype=np.float64)
            done = np.ascontiguousarray(z["done"], dtype=np.uint8)
    else:
        map_out = np.zeros((int(wl.H.shape[-3]), n_sy, n_sx))
        done = np.zeros((gy, gx), dtype=np.uint8)
    left = int((done == 0).sum())
    mapped = 0
    while left > 0 and (max_tiles <= 0 or mapped < max_tiles):
        left = inelastic_map_tiles_for(ctx, sm, wl, tile, map_out, done, precision,
                                       max_tiles=1, stream=stream)
        mapped += 1
        tmp = path + ".tmp.npz"
        np.savez(tmp, key=key, map=map_out, done=done)
        os.replace(tmp, path)
    return map_out, left


def quadratic_reference_map_for(ctx: Context, wl, positions=None, stream=None):
    return ctx.quadratic_reference_map(wl.vproj, wl.cell, wl.lam, wl.sigma, wl.dz, wl.f, wl.alpha,
                                       wl.H, wl.site_slice, wl.win_x0, wl.win_y0, wl.site_x,
                                       wl.site_y, wl.scan, wl.beta, positions=positions,
                                       stream=stream)


# -- map server --------------------------------------------------------------------------

def make_request(vproj, cell, lam, sigma, dz, f, alpha, H, site_slice, win_x0, win_y0, site_x,
                 site_y, scan, beta, precision="tf32", deadline_s=0.0, sin_checkpoint=0):
    """eels_request over host arrays; returns (request, keepalive)."""
    v, on_dev, vkeep = _ptr(vproj, np.float32)
    if on_dev:
        raise TypeError("server requests take host arrays")
    n_z, n = int(vproj.shape[0]), int(vproj.shape[-1])
    tr, tkeep = _transitions(H, site_slice, win_x0, win_y0, site_x, site_y)
    req = Request(Specimen(n, n_z, float(cell), v, 0),
                  Optics(float(lam), float(sigma), float(dz), int(f), float(alpha)), tr,
                  Scan(*[int(x) for x in scan[:2]], *[float(x) for x in scan[2:]]), float(beta),
                  EELS_PREC[precision], float(deadline_s), int(sin_checkpoint))
    return req, (vkeep, tkeep)


def request_footprint(req) -> int:
    return int(load().eels_request_footprint(C.byref(req)))


class Server:
    """eels_server: continuous-batching map server on one device."""

    def __init__(self, device: int = 0, hbm_budget: int = 64 << 30, slots: int = 4):
        self._lib = load()
        h = C.c_void_p()
        st = self._lib.eels_server_create(int(device), int(hbm_budget), int(slots), C.byref(h))
        if st != 0:
            raise EelsError(st, "eels_server_create")
        self._h = h
        self._keep = {}
        self._shape = {}

    def submit(self, req, keep, n_types, scan) -> int:
        rid = C.c_int64(0)
        st = self._lib.eels_server_submit(self._h, C.byref(req), C.byref(rid))
        if st != 0:
            raise EelsError(st, "eels_server_submit")
        self._keep[rid.value] = (req, keep)
        self._shape[rid.value] = (int(n_types), int(scan[1]), int(scan[0]))
        return rid.value

    def wait(self, rid: int, timeout: float = 0.0):
        out = np.zeros(self._shape[rid])
        lat = C.c_double(0.0)
        st = self._lib.eels_server_wait(self._h, int(rid), out.ctypes.data_as(C.c_void_p),
                                        float(timeout), C.byref(lat))
        if st == 5:
            raise EelsError(st, "eels_server_wait timed out")
        self._keep.pop(rid, None)
        if st == 6:
            raise EelsError(st, f"request {rid} cancelled")
        if st != 0:
            raise EelsError(st, f"request {rid} failed")
        return out, float(lat.value)

    def cancel(self, rid: int):
        """eels_server_cancel: drop the request before admission or at its next tile."""
        st = self._lib.eels_server_cancel(self._h, int(rid))
        if st != 0:
            raise EelsError(st, "eels_server_cancel")

    def info(self, rid: int) -> dict:
        """eels_server_request_info: status, times (s since server start) and tiles."""
        r = RequestInfo()
        st = self._lib.eels_server_request_info(self._h, int(rid), C.byref(r))
        if st != 0:
            raise EelsError(st, "eels_server_request_info")
        return {name: getattr(r, name) for name, _ in RequestInfo._fields_}

    def log_jsonl(self, path, rids, extra=None):
        """Appends one JSON line per request (eels_server_request_info plus the derived
        latency, wait and pixel-slices/s) to path; extra (a dict per request id) is merged
        into its line."""
        import json
        with open(path, "a") as fh:
            for rid in rids:
                d = self.info(rid)
                d["id"] = int(rid)
                done, first, sub = d["t_done"], d["t_first_tile"], d["t_submit"]
                d["latency_s"] = done - sub if d["done"] and done >= 0 else None
                d["wait_s"] = first - sub if first >= 0 else None
                run = done - first if d["done"] and first >= 0 and done >= first else None
                d["pixel_slices_per_s"] = (d["pixel_slices"] / run
                                           if run and d["status"] == 0 else None)
                if extra and rid in extra:
                    d.update(extra[rid])
                fh.write(json.dumps(d) + "\n")

    def stats(self) -> dict:
        s = ServerStats()
        self._lib.eels_server_stats_get(self._h, C.byref(s))
        return {name: getattr(s, name) for name, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.eels_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
