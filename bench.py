"""Benchmark: EELS map pixel-slices/s of the linear S-matrix method on one GB300.

A step is one pass of the whole hot path over the workload: build S_in (all
depths), stream S_out backwards and contract every transition of every slice
into the FP64 map.  value = n_scan * n_z / step time, inputs resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the workload
(the method has no exchange step; replicas only): value = N * units / max time.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import specimen as sp  # noqa: E402

METRIC = "EELS map pixel-slices/s"
UNIT = "pixel-slices/s"
DEFAULT_WORKLOAD = "nanoparticle"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


def _peaks():
    try:
        return json.load(open(PEAKS))
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0, "fallback": True}


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for name, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle sample (the conventional algorithm, FP64, as it stands)
# ---------------------------------------------------------------------------

_POOL_WL = None


def _pool_init(name):
    """Worker initialiser: build the workload once per process."""
    global _POOL_WL
    import specimen as sp_
    os.environ["OMP_NUM_THREADS"] = "1"
    _POOL_WL = sp_.WORKLOADS[name]()


def _oracle_probe_sample(args):
    """One probe of the conventional oracle over the last `tail` slices of the specimen with
    the deepest `max_sites` sites of its window there: a few tens of multislice operations,
    each the same transmit-FFT-propagate-IFFT step the full run repeats."""
    iy, ix, tail, max_sites = args
    from oracle import multislice as ms
    wl = _POOL_WL
    first = max(0, wl.n_z - tail)
    rx, ry = wl.scan_positions()
    seen = [s for s in range(wl.n_sites)
            if wl.site_slice[s] >= first
            and ms.axis_in_window(wl.site_x[s], rx[ix], wl.cell, wl.f)
            and ms.axis_in_window(wl.site_y[s], ry[iy], wl.cell, wl.f)]
    seen.sort(key=lambda s: -int(wl.site_slice[s]))
    sub = wl.with_sites(seen[:max_sites])
    sub = dataclasses.replace(sub, vproj=wl.vproj[first:], n_z=wl.n_z - first,
                              site_slice=(sub.site_slice - first).astype(np.int32))
    c = {}
    t0 = time.perf_counter()
    ms.quadratic_map(sub, positions=[(iy, ix)], counter=c)
    return time.perf_counter() - t0, c["steps"]


def _full_probe_steps(wl, iy, ix):
    """Multislice operations of one probe in the conventional algorithm (Sec. III count)."""
    from oracle import multislice as ms
    rx, ry = wl.scan_positions()
    steps = wl.n_z
    for s in range(wl.n_sites):
        if (ms.axis_in_window(wl.site_x[s], rx[ix], wl.cell, wl.f)
                and ms.axis_in_window(wl.site_y[s], ry[iy], wl.cell, wl.f)):
            steps += wl.n_types * (wl.n_z - int(wl.site_slice[s]))
    return steps


class OracleSampler:
    """The FP64 conventional oracle on this host's cores, one worker process per core,
    each holding the workload.  sample() runs one probe per worker (spread over the
    scan) with the deepest sites of its window; the cost of the conventional algorithm
    is exactly linear in its multislice count, so the full-workload rate is the sampled
    time per operation times the full per-probe count."""

    def __init__(self, wl_name, procs=None, tail=8, max_sites=1):
        self.name = wl_name
        self.wl = sp.WORKLOADS[wl_name]()
        self.procs = procs or os.cpu_count() or 1
        self.tail = tail
        self.max_sites = max_sites
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_pool_init,
                                                 initargs=(wl_name,))
        self.k = 0

    def sample(self):
        wl = self.wl
        n_sx, n_sy = wl.scan[0], wl.scan[1]
        jobs = []
        for q in range(self.procs):
            k = self.k * self.procs + q
            jobs.append(((k * 7 + 3) % n_sy, (k * 13 + 5) % n_sx, self.tail, self.max_sites))
        self.k += 1
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_probe_sample, jobs)
        wall = time.perf_counter() - t0
        ops = sum(s for _, s in res)
        per_op = sum(t for t, _ in res) / ops            # seconds per op per core
        full = float(np.mean([_full_probe_steps(wl, j[0], j[1]) for j in jobs]))
        rate = self.procs * wl.n_z / (full * per_op)     # a core does n_z pixel-slices per probe
        sample = (f"{self.procs} processes x 1 probe of {wl.name}: the conventional algorithm over "
                  f"the last {self.tail} slices with the {self.max_sites} deepest sites of the "
                  f"probe's window there ({ops} multislice ops, {wall:.1f} s wall); rate scaled "
                  f"by the full per-probe count {full:.0f} ops")
        return rate, sample, {"wall_s": wall, "ops": int(ops), "full_ops_per_probe": full}

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_oracle_rate(wl_name, budget_procs=None):
    """Pixel-slices/s of the FP64 conventional oracle on this host's cores (one sample)."""
    smp = OracleSampler(wl_name, budget_procs)
    try:
        rate, sample, rec = smp.sample()
    finally:
        smp.close()
    return rate, smp.procs, sample, rec


def _oracle_full_probe(args):
    name, iy, ix = args
    import specimen as sp_
    from oracle import multislice as ms
    wl = sp_.WORKLOADS[name]()
    return ms.quadratic_map(wl, positions=[(iy, ix)])[:, iy, ix]


def cpu_oracle_full(wl_name):
    """The whole map of a small workload with the FP64 conventional oracle, probes spread
    over this host's cores: pixel-slices/s of a complete run, no extrapolation."""
    wl = sp.WORKLOADS[wl_name]()
    jobs = [(wl_name, iy, ix) for iy in range(wl.scan[1]) for ix in range(wl.scan[0])]
    cores = min(os.cpu_count() or 1, len(jobs))
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_full_probe, jobs)
    wall = time.perf_counter() - t0
    return {"workload": wl.name, "value": wl.n_scan * wl.n_z / wall, "unit": UNIT,
            "wall_s": wall, "cores": cores, "probes": len(jobs),
            "sample": "complete map (every probe, every site), conventional FP64 algorithm"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def _algorithmic(wl, n_in, n_out, prof, steps):
    """Algorithmic bytes of the multislice kernels per step of the default (stream)
    scheme.  Row pass: read W and write Phi (N x N/2 each) and store the even samples
    ((N/2)^2) per wave, plus the slice's t (N^2) once per launch; the last slice of each
    sweep stores without writing Phi.  Column pass: read Phi, write W.  Complex64."""
    n, nz = wl.n, wl.n_z
    nh = n // 2
    c = 8
    row = (2 * n * nh + nh * nh) * c
    last = (n * nh + nh * nh) * c
    col = 2 * n * nh * c
    t = n * n * c
    work = work_depths(wl)
    # the backward sweep stores S_out only at depths with transitions (and skips the
    # depth-0 pass when that depth has none)
    adj = sum((2 * n * nh + (nh * nh if i in work else 0)) * c for i in range(1, nz)) + \
        (last if 0 in work else 0)
    out = {}
    for name, waves, per_wave in (("row_pass", n_in, (nz - 1) * row + last),
                                  ("row_pass_adjoint", n_out, adj)):
        launches = prof.get(name, {}).get("launches", 0) / steps
        out[name] = ("hbm", waves * per_wave + launches * t)
    for name, waves in (("col_pass", n_in), ("col_pass_adjoint", n_out)):
        out[name] = ("hbm", waves * (nz - 1) * col)
    return out


def work_depths(wl):
    """Depths whose sites some probe of the scan reaches (the map contracts only those)."""
    rx, ry = wl.scan_positions()
    return {int(wl.site_slice[s]) for s in range(wl.n_sites)
            if _window_count(wl.site_x[s], rx, wl.cell, wl.f) and
            _window_count(wl.site_y[s], ry, wl.cell, wl.f)}


def crop_study(g, ctx, stream, widths=(64, 48, 30, 22, 15), reps=3):
    """Sec. IV B trade-off: one dopant with a long-tailed transition potential in a
    51.6 A rocksalt slab (2x2 cells, 128^2, f = 1, 32x32 scan over the cell); the
    potential is cut to w x w pixels of the N/2 grid (0.134 A each; 64 = the whole cell).
    Reports the contraction time (TF32, CUDA events of the gather and GEMM launches) and
    the errors against the whole-cell map (FP32): total, and in the 1 A window around
    the dopant (eps of the site pixels, and of their summed signal)."""
    import torch
    base = sp.dopant_slab(widths[0])
    vdev = torch.from_numpy(base.vproj).cuda()
    sm = g.build_smatrix_for(ctx, base, vproj=vdev, stream=stream)
    rx, ry = base.scan_positions()
    sx, sy = float(base.site_x[0]), float(base.site_y[0])
    win = (np.abs(ry - sy)[:, None] <= 0.5) & (np.abs(rx - sx)[None, :] <= 0.5)
    contraction = ("gemm", "tc_")

    def contraction_ms(wl):
        g.inelastic_map_for(ctx, sm, wl, "tf32", stream=stream)     # warm / tune
        torch.cuda.synchronize()
        ctx.profile_read()
        ctx.profile_enable(True)
        for _ in range(reps):
            g.inelastic_map_for(ctx, sm, wl, "tf32", stream=stream)
        ctx.profile_enable(False)
        prof = ctx.profile_read()
        return (sum(v["ms"] for k, v in prof.items() if k.startswith(contraction)) / reps,
                sum(v["ms"] for v in prof.values()) / reps)

    rows, ref = [], None
    for w in widths:
        wl = sp.dopant_slab(w)
        fp = g.inelastic_map_for(ctx, sm, wl, "fp32", stream=stream)
        t_c, t_all = contraction_ms(wl)
        t_every, _ = contraction_ms(sp.dopant_slab(w, every_fe=True))
        if ref is None:
            ref = fp
        d = fp - ref
        rows.append({"w": w, "side_A": round(w * base.cell / (base.n // 2), 2),
                     "contraction_ms": round(t_c, 3), "map_kernels_ms": round(t_all, 3),
                     "contraction_ms_every_fe": round(t_every, 3),
                     "eps_total": float(np.sqrt(np.sum(d ** 2) / np.sum(ref ** 2))),
                     "eps_site": float(np.sqrt(np.sum(d[:, win] ** 2) / np.sum(ref[:, win] ** 2))),
                     "site_signal_err": float(abs(fp[:, win].sum() - ref[:, win].sum())
                                              / ref[:, win].sum())})
    sm.free()
    t0 = rows[0]["contraction_ms"]
    t0e = rows[0]["contraction_ms_every_fe"]
    for r in rows:
        r["speedup_vs_whole_cell"] = round(t0 / r["contraction_ms"], 2)
        r["speedup_vs_whole_cell_every_fe"] = round(t0e / r["contraction_ms_every_fe"], 2)
    return {"workload": "dopant in rocksalt Fe-O 2x2x12 cells (51.6 A), 128^2, f=1, 32x32 scan",
            "every_fe_sites": int(sp.dopant_slab(widths[0], every_fe=True).n_sites),
            "site_pixels": int(win.sum()), "rows": rows}


def phonon_run(g, ctx, stream, k, precision, reps=2):
    """Frozen-phonon average over k seeded configurations of the 512^2 rocksalt crystal
    (8x8x20 cells, f = 2, 32x32 scan, u_rms = 0.08 A): pixel-slices/s counting every pass,
    host inputs (the configurations' potentials and transition windows) copied inside
    the timed region."""
    import torch
    cfg = sp.rocksalt_phonons(k, u_rms=0.08, ncell=8, nzc=20, n=512, f=2, scan_n=32, w=32)
    out = torch.zeros((cfg[0].n_types, 32, 32), dtype=torch.float64, device="cuda")
    ctx.phonon_map(cfg[:1], precision=precision, out=out, stream=stream)   # warm / tune
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        ctx.phonon_map(cfg, precision=precision, out=out, stream=stream)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    units = k * cfg[0].n_scan * cfg[0].n_z
    static = cfg[0]
    return {"configs": k, "u_rms_A": 0.08, "workload": "rocksalt Fe-O 8x8x20 cells, 512^2, f=2",
            "value": units / dt, "unit": UNIT, "ms_per_pass": 1e3 * dt / k,
            "precision": precision, "map_mean": float(out.mean().item()),
            "h2d_bytes_per_pass": int(static.vproj.nbytes + static.H.nbytes)}


def s2_study(g, ctx, stream, thickness_cells=(5, 12, 19, 23), reps=2):
    """Sec. IV C trade-off on a rocksalt thickness series (8x8 cells, 256^2, f = 2, 16x16
    scan): map time of each S_out scheme (TF32 contraction) and the error of the
    inverse retreat against the exact stream (FP32 contraction, so that the scheme's
    error is not hidden under tensor-core rounding)."""
    import torch
    rows = []
    for nzc in thickness_cells:
        wl = sp.rocksalt_slab(nzc)
        vdev = torch.from_numpy(wl.vproj).cuda()
        Hdev = torch.from_numpy(wl.H).cuda()
        sm = g.build_smatrix_for(ctx, wl, vproj=vdev, stream=stream)
        ms_, maps = {}, {}
        for scheme in ("stream", "recompute", "inverse"):
            ctx.set_sout_scheme(scheme)
            maps[scheme] = g.inelastic_map_for(ctx, sm, wl, "fp32", H=Hdev, stream=stream)
            g.inelastic_map_for(ctx, sm, wl, "tf32", H=Hdev, stream=stream)   # warm / tune
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                g.inelastic_map_for(ctx, sm, wl, "tf32", H=Hdev, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_[scheme] = e0.elapsed_time(e1) / reps
        ctx.set_sout_scheme("stream")
        sm.free()
        ref = maps["stream"]

        def err(m):
            return float(np.sqrt(np.sum((m - ref) ** 2) / np.sum(ref ** 2)))
        rows.append({"thickness_A": round(wl.n_z * wl.dz, 1), "n_z": wl.n_z,
                     "map_ms": {k: round(v, 2) for k, v in ms_.items()},
                     "eps_inverse_vs_exact": err(maps["inverse"]),
                     "eps_recompute_vs_exact": err(maps["recompute"]),
                     "inverse_speedup_vs_recompute_pct":
                         round(100.0 * (ms_["recompute"] / ms_["inverse"] - 1.0), 1),
                     "stream_speedup_vs_inverse_pct":
                         round(100.0 * (ms_["inverse"] / ms_["stream"] - 1.0), 1)})
    return {"workload": "rocksalt Fe-O 8x8 cells x thickness, 256^2, f=2, 16x16 scan",
            "rows": rows}


def _source_hash(kernel):
    import hashlib
    files = (["paper_1908_07628_gb300/csrc/multislice.cu", "paper_1908_07628_gb300/csrc/common.cuh"]
             if "pass" in kernel else
             ["paper_1908_07628_gb300/csrc/contract_tc.cu", "paper_1908_07628_gb300/csrc/tc_ptx.cuh"])
    m = hashlib.sha1()
    for f in files:
        m.update(open(os.path.join(ROOT, f), "rb").read())
    return m.hexdigest()[:12]


def measured_traffic(kernel, n, waves, operand_bytes=None):
    """DRAM bytes per launch from the committed ncu table, if the kernel is unchanged: a
    captured launch of the same size, or a measured ratio of DRAM bytes to operand bytes
    applied to this launch's operand bytes."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        if ln.startswith("#") or not ln.strip():
            continue
        name, nn, w, sha, val = ln.split()
        if name != kernel or sha != _source_hash(kernel):
            continue
        if w == "ratio" and operand_bytes:
            return float(val) * operand_bytes
        if nn != "any" and int(nn) == n and w == str(waves):
            return float(val)
    return None


def gemm_v_operand_bytes(wl, n_out, precision, launches):
    """Operand bytes GEMM-V reads per launch on average: the S_out window of every site
    and the H_t Y / -i H_t Y rows of every transition, both planes of the split."""
    rx, ry = wl.scan_positions()
    kal, vb = (64, 4) if precision == "bf16x3" else (32, 8)
    k1p = (2 * wl.w * wl.w + kal - 1) // kal * kal
    total = 0
    for s in range(wl.n_sites):
        nr = _window_count(wl.site_x[s], rx, wl.cell, wl.f) * \
            _window_count(wl.site_y[s], ry, wl.cell, wl.f)
        if nr:
            total += (n_out + wl.n_types * 2 * nr) * k1p * vb
    return total / max(launches, 1)


# precision each workload's configuration names: the 1024^2 sphere and the 768^2 vacancy
# crystal the BF16 hi + lo split, the 512^2 crystal ("FP32 on device") the TF32 tensor
# cores with the hi + lo split (FP32-class), the small parity case the CUDA-core FP32 path
CONFIG_PRECISION = {"rocksalt_small": "fp32", "rocksalt_fp32": "tf32", "rocksalt_vacancy": "bf16x3",
                    "nanoparticle": "bf16x3", "nanoparticle_small": "bf16x3"}
# extra workloads timed in the same run (same clocks record), each in its own precision
EXTRA_CONFIGS = (("rocksalt_fp32", "tf32"), ("rocksalt_vacancy", "bf16x3"))
# sampled-output accuracy against the FP64 oracle: three sites at three depths near the
# first probe, the m = 0 channel, the conventional algorithm at two probes
ORACLE_SAMPLES = {
    "rocksalt_fp32": ((0, 21, 39), ((16, 16), (3, 29))),
    "rocksalt_vacancy": ((0, 40, 79), ((16, 16), (2, 29))),
    "nanoparticle": ((12, 25, 44), ((64, 64), (60, 70))),
    "nanoparticle_small": ((4, 10, 17), ((24, 24), (20, 28))),
    "rocksalt_small": ((0, 2, 5), ((3, 3), (5, 2))),
}


def workload_config(wl, n_in, n_out, precision, association, world):
    """The configuration dict both arms report for a workload."""
    return {"workload": wl.name, "n": wl.n, "n_z": wl.n_z, "f": wl.f, "cell_A": wl.cell,
            "n_in": int(n_in), "n_out": int(n_out), "w": wl.w, "n_sites": int(wl.n_sites),
            "scan": [int(wl.scan[0]), int(wl.scan[1])], "n_types": int(wl.n_types),
            "precision": precision, "association": association,
            "parallelism": f"replicas{world}",
            "l2": "inputs larger than L2 (S_in alone is "
                  f"{wl.n_z * n_in * (wl.n // 2) ** 2 * 8 / 1e9:.1f} GB)"}


def oracle_sample_sub(wl, name):
    """The sampled sub-workload (sites and m = 0 channel) and its probes."""
    targets, probes = ORACLE_SAMPLES[name]
    rx, ry = wl.scan_positions()
    cx, cy = rx[probes[0][1]], ry[probes[0][0]]
    chosen = []
    for t in targets:
        idx = np.nonzero(wl.site_slice == t)[0]
        d2 = (wl.site_x[idx] - cx) ** 2 + (wl.site_y[idx] - cy) ** 2
        chosen.append(int(idx[np.argmin(d2)]))
    sub = wl.with_sites(chosen)
    sub.H = np.ascontiguousarray(sub.H[:, min(1, sub.H.shape[1] - 1):][:, :1])
    return sub, list(probes)


def _oracle_probe(args):
    """FP64 conventional oracle at one probe of a sampled sub-workload (a spawn worker)."""
    name, k = args
    import specimen as sp_
    from oracle import multislice as ms
    wl = sp_.WORKLOADS[name]()
    sub, probes = oracle_sample_sub(wl, name)
    iy, ix = probes[k]
    t0 = time.perf_counter()
    ref = ms.quadratic_map(sub, positions=[(iy, ix)])
    return name, k, ref[:, iy, ix].tolist(), time.perf_counter() - t0


def oracle_samples(names):
    """Reference values of every sampled probe, computed on the host before CUDA starts."""
    jobs = [(nm, k) for nm in names for k in range(len(ORACLE_SAMPLES[nm][1]))]
    if not jobs:
        return {}
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        res = pool.map(_oracle_probe, jobs)
    out = {}
    for nm, k, vals, sec in res:
        out.setdefault(nm, {})[k] = (vals, sec)
    return out


def sampled_eps(g, ctx, wl, name, precision, ref, stream):
    """eps of the GPU map against the FP64 oracle at the sampled probes (same sub-workload)."""
    from oracle import multislice as ms
    sub, probes = oracle_sample_sub(wl, name)
    sm = g.build_smatrix_for(ctx, sub, stream=stream)
    got = g.inelastic_map_for(ctx, sm, sub, precision=precision, stream=stream)
    sm.free()
    r = np.array([ref[k][0] for k in range(len(probes))])
    t = np.array([got[:, iy, ix] for iy, ix in probes])
    return {"eps_vs_fp64_oracle": float(ms.relative_error(r, t)),
            "sample": f"{len(probes)} probes x 3 sites at depths {ORACLE_SAMPLES[name][0]}, "
                      "m = 0 channel, full S-matrix; oracle: conventional FP64 algorithm",
            "oracle_s": float(sum(ref[k][1] for k in range(len(probes))))}


def measure_peaks(g, dev, seconds=3.0):
    """TF32 (cuBLAS, torch fp32 matmul with TF32 allowed) burst and sustained, and the
    FP32 FMA rate of the CUDA cores (eels_fp32_fma_rate), each with its SM clock."""
    import torch
    out = {}
    n = 8192
    a = torch.randn(n, n, device="cuda")
    b = torch.randn(n, n, device="cuda")
    prev = torch.get_float32_matmul_precision()
    torch.set_float32_matmul_precision("high")        # TF32 tensor cores
    try:
        torch.matmul(a, b)
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(10):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        out["tf32_tflops"] = 2.0 * n ** 3 / best / 1e12
        clk = ClockSampler(dev)
        clk.start()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 0
        e0.record()
        while time.perf_counter() - t0 < seconds:
            for _ in range(8):
                torch.matmul(a, b)
            reps += 8
            torch.cuda.synchronize()
        e1.record()
        torch.cuda.synchronize()
        out["tf32_tflops_sustained"] = 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) / 1e3) / 1e12
        out["tf32_clocks"] = clk.stop()
    finally:
        torch.set_float32_matmul_precision(prev)
    del a, b
    torch.cuda.empty_cache()
    clk = ClockSampler(dev)
    clk.start()
    rate = max(g.fp32_fma_rate(dev, 1 << 21) for _ in range(3))
    out["fp32_fma_tflops"] = rate / 1e12
    out["fp32_clocks"] = clk.stop()
    out["how"] = ("tf32: torch.matmul fp32 8192^3 with TF32 allowed (cuBLAS), best of 10 (burst) "
                  f"and back to back for {seconds:.0f} s (sustained); fp32: eels_fp32_fma_rate, "
                  "independent FMA chains on every SM, best of 3")
    return out


def _timed_steps(step, k, stream, world, dev):
    """k steps between CUDA events on the launch stream, barrier + synchronize on both
    sides, SM clocks sampled meanwhile.  Returns (ms total, clocks)."""
    import torch
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(k):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_total = e0.elapsed_time(e1)
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
        t = torch.tensor([ms_total], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(t.item())
    return ms_total, clk


def _profiled(ctx, step, k):
    """Per-kernel CUDA-event times of k steps run apart from the timed region."""
    import torch
    torch.cuda.synchronize()
    ctx.profile_read()
    ctx.profile_enable(True)
    for _ in range(k):
        step()
    torch.cuda.synchronize()
    ctx.profile_enable(False)
    return ctx.profile_read()


def _tensor_roof(kernel, wl, n_in, n_out, prof, steps, peak, peak_src):
    """Roofline of a tensor-core kernel: three real products per useful product (hi + lo)."""
    useful = contraction_flops(wl, n_in, n_out, kernel)
    launches = prof[kernel]["launches"]
    avg_s = prof[kernel]["ms"] / launches / 1e3
    per_step = launches / steps
    achieved = 3 * useful / per_step / avg_s / 1e12
    traffic = None
    if "gemm_v" in kernel:
        prec = "bf16x3" if "bf16x3" in kernel else "tf32"
        traffic = measured_traffic(kernel, wl.n, "batch",
                                   gemm_v_operand_bytes(wl, n_out, prec, per_step))
    return {"kernel": kernel, "bound": "tensor", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
            "traffic_note": "ncu DRAM bytes per operand byte of a captured batch x this launch's "
                            "operand bytes" if traffic else None,
            "useful_tflops": useful / per_step / avg_s / 1e12,
            "avg_launch_ms": avg_s * 1e3, "launches_per_step": per_step,
            "peak_source": peak_src}


def _roofline(dom, wl, n_in, n_out, prof, steps, peaks, tpk, clk):
    """Roofline entry of kernel `dom` from the profiled steps."""
    if dom is None:
        return None
    alg = _algorithmic(wl, n_in, n_out, prof, steps)
    launches = prof[dom]["launches"]
    avg_s = prof[dom]["ms"] / launches / 1e3
    per_step = launches / steps
    if dom in alg:
        bytes_launch = alg[dom][1] / per_step
        achieved = bytes_launch / avg_s / 1e9
        waves = n_out if "adjoint" in dom else n_in
        return {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "traffic": measured_traffic(dom, wl.n, waves), "algorithmic_bytes": bytes_launch,
                "avg_launch_ms": avg_s * 1e3,
                "peak_source": "measured" if "fallback" not in peaks else "fallback"}
    if "bf16x3" in dom:
        # the step runs for seconds: the sustained figure (measured under the power cap)
        return _tensor_roof(dom, wl, n_in, n_out, prof, steps, peaks["bf16_tflops_sustained"],
                            "measured bf16 sustained (MEASURED_PEAKS.json)")
    nominal = tpk.get("nominal", False)   # --no-peaks: nominal ratios, not measured
    if "tf32" in dom:
        return _tensor_roof(dom, wl, n_in, n_out, prof, steps, tpk["tf32_tflops_sustained"],
                            "nominal: measured bf16 sustained x 1.1/2.25 (--no-peaks)" if nominal
                            else "measured tf32 sustained (cuBLAS, this run)")
    flops = contraction_flops(wl, n_in, n_out, dom)
    peak = tpk["fp32_fma_tflops"]
    achieved = flops / per_step / avg_s / 1e12
    return {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None, "avg_launch_ms": avg_s * 1e3,
            "peak_source": "nominal: 152 x 128 x 2 x max clock (--no-peaks)" if nominal
            else "measured fp32 FMA rate (eels_fp32_fma_rate, this run)"}


def _multislice_bounds(wl, n_in, n_out, prof, steps, peaks, tpk):
    """Every multislice kernel against the HBM bound and the measured FP32 rate: per wave
    and slice the row pass runs two N-point FFTs on N rows and one complex multiply per
    pixel (10 N^2 log2 N + 6 N^2 flop), the column pass two FFTs on the N/2 band columns
    and the propagator multiply (5 N^2 log2 N + 3 N^2 flop)."""
    alg = _algorithmic(wl, n_in, n_out, prof, steps)
    lg = math.log2(wl.n)
    nn = float(wl.n) ** 2
    row_full, row_last = 10 * nn * lg + 6 * nn, 5 * nn * lg + 6 * nn
    col = 5 * nn * lg + 3 * nn
    work = work_depths(wl)
    fft = {"row_pass": n_in * ((wl.n_z - 1) * row_full + row_last),
           "row_pass_adjoint": n_out * ((wl.n_z - 1) * row_full + (row_last if 0 in work else 0)),
           "col_pass": n_in * (wl.n_z - 1) * col,
           "col_pass_adjoint": n_out * (wl.n_z - 1) * col}
    out = {}
    for k in alg:
        if k not in prof or prof[k]["ms"] <= 0:
            continue
        sec = prof[k]["ms"] / steps / 1e3
        out[k] = {"achieved_gbs": alg[k][1] / sec / 1e9,
                  "frac": alg[k][1] / sec / 1e9 / peaks["hbm_gbs"],
                  "fft_tflops": fft[k] / sec / 1e12,
                  "fp32_frac": fft[k] / sec / 1e12 / tpk["fp32_fma_tflops"]}
    # the whole slice step (row + column pass) against the minimum bytes a beam-step must
    # move: read and write the band-limited state, 2 (N/2)^2 complex64, plus the S store,
    # (N/2)^2 (the two-pass design moves about three times that)
    state, store = 2 * (wl.n // 2) ** 2 * 8, (wl.n // 2) ** 2 * 8
    for name, waves, r, c, stores in (
            ("forward_step", n_in, "row_pass", "col_pass", wl.n_z),
            ("adjoint_step", n_out, "row_pass_adjoint", "col_pass_adjoint", len(work))):
        if r in prof and c in prof and prof[r]["ms"] + prof[c]["ms"] > 0:
            sec = (prof[r]["ms"] + prof[c]["ms"]) / steps / 1e3
            total = waves * (wl.n_z * state + stores * store)
            gbs = total / sec / 1e9
            out[name + "_vs_min_bytes"] = {"min_bytes_per_beam_step": total / (waves * wl.n_z),
                                           "achieved_gbs": gbs, "frac": gbs / peaks["hbm_gbs"]}
    return out


# kernels behind one profiling record: a gather record brackets three gather kernels;
# every step also runs six small kernels outside the records (propagator table, four
# phase tables, the final scale-and-check of the map)
KERNELS_PER_RECORD = {"tc_gather_y": 3, "tc_gather": 3}
UNRECORDED_PER_STEP = 6


def kernel_launches(prof):
    """Kernel launches of one profiled step."""
    return sum(v["launches"] * KERNELS_PER_RECORD.get(k, 1) for k, v in prof.items()) + \
        UNRECORDED_PER_STEP


def _shares(prof, steps):
    tot = sum(v["ms"] for v in prof.values())
    return {k: {"launches_per_step": prof[k]["launches"] / steps,
                "ms_per_step": prof[k]["ms"] / steps,
                "share": prof[k]["ms"] / max(tot, 1e-9)} for k in sorted(prof)}


def time_workload(g, ctx, wl, precision, steps, warmup, stream, world, dev):
    """Warm-up, un-instrumented timed steps, then one profiled step.  Returns the figures."""
    import torch
    vdev = torch.from_numpy(wl.vproj).cuda()
    Hdev = torch.from_numpy(wl.H).cuda()
    mdev = torch.zeros((wl.n_types, wl.scan[1], wl.scan[0]), dtype=torch.float64, device="cuda")

    def step():
        sm = g.build_smatrix_for(ctx, wl, vproj=vdev, stream=stream)
        g.inelastic_map_for(ctx, sm, wl, precision=precision, H=Hdev, out=mdev, stream=stream)
        sm.free()

    for _ in range(warmup):
        step()
    ms_total, clk = _timed_steps(step, steps, stream, world, dev)
    prof = _profiled(ctx, step, 1)
    del vdev, Hdev
    return {"ms_total": ms_total, "clocks": clk, "prof": prof, "map": mdev}


def gpu_arm(args, rank, world, ref_samples):
    import torch
    from paper_1908_07628_gb300 import build
    build.build()
    import paper_1908_07628_gb300 as g

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    wl = load_workload(args)
    precision = args.precision or CONFIG_PRECISION.get(args.workload, "bf16x3")
    ctx = g.Context(dev)
    ctx.set_association(args.association)
    if args.operand_mib:
        ctx.set_operand_budget(args.operand_mib)
    if args.tile_width:
        ctx.set_tile_width(args.tile_width)
    ctx.set_sout_scheme(args.sout_scheme)
    stream = torch.cuda.current_stream()
    n_in = g.count_beams(wl.n, wl.cell, wl.lam, wl.f, wl.alpha)
    n_out = g.count_beams(wl.n, wl.cell, wl.lam, wl.f, wl.beta)

    # headline: un-instrumented timed steps; kernel shares from one profiled step after
    res = time_workload(g, ctx, wl, precision, args.steps, args.warmup, stream, world, dev)
    ms_step = res["ms_total"] / args.steps
    units = wl.n_scan * wl.n_z
    value = world * units / (ms_step / 1e3)
    prof, clk = res["prof"], res["clocks"]
    launches_per_step = kernel_launches(prof)
    tuning = ctx.tuning_read()

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    vh = torch.from_numpy(wl.vproj).pin_memory().numpy()
    Hh = torch.from_numpy(wl.H).pin_memory().numpy()
    mh = torch.zeros((wl.n_types, wl.scan[1], wl.scan[0]), dtype=torch.float64).pin_memory().numpy()

    def e2e_step():
        sm = g.build_smatrix_for(ctx, wl, vproj=vh, stream=stream)
        g.inelastic_map_for(ctx, sm, wl, precision=precision, H=Hh, out=mh, stream=stream)
        sm.free()

    e2e_step()
    torch.cuda.synchronize()
    k_e2e = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / k_e2e
    h2d = wl.vproj.nbytes + wl.H.nbytes + wl.n_sites * (3 * 4 + 2 * 8)
    d2h = wl.n_types * wl.n_scan * 8
    del vh, Hh

    out = {}
    if rank == 0:
        # measured denominators: TF32 tensor (cuBLAS) and the FP32 FMA rate, this run
        peaks = _peaks()
        if args.no_peaks:   # (profiling runs) nominal figures instead of measured ones
            tpk = {"tf32_tflops": peaks["bf16_tflops"] * 1.1 / 2.25,
                   "tf32_tflops_sustained": peaks["bf16_tflops_sustained"] * 1.1 / 2.25,
                   "fp32_fma_tflops": 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) / 1e6,
                   "how": "not measured (--no-peaks): bf16 x 1.1/2.25 and 152 x 128 x 2 x clock",
                   "nominal": True}
        else:
            tpk = measure_peaks(g, dev)
        tot = {k: v["ms"] for k, v in prof.items()}
        dom = max(tot, key=tot.get) if tot else None
        out["roofline"] = _roofline(dom, wl, n_in, n_out, prof, 1, peaks, tpk, clk)
        out["multislice_bounds"] = _multislice_bounds(wl, n_in, n_out, prof, 1, peaks, tpk)
        out["kernels"] = _shares(prof, 1)
        out["peaks_measured"] = tpk
        acc = {}
        if args.workload in ref_samples:
            acc = sampled_eps(g, ctx, wl, args.workload, precision, ref_samples[args.workload],
                              stream)
        out["accuracy"] = acc

        # the other configurations, timed the same way, each in its own precision
        extras = []
        for name, prec in EXTRA_CONFIGS:
            if args.no_extra or name == args.workload:
                continue
            w2 = sp.WORKLOADS[name]()
            r2 = time_workload(g, ctx, w2, prec, 3, 2, stream, 1, dev)
            ni2 = g.count_beams(w2.n, w2.cell, w2.lam, w2.f, w2.alpha)
            no2 = g.count_beams(w2.n, w2.cell, w2.lam, w2.f, w2.beta)
            t2 = {k: v["ms"] for k, v in r2["prof"].items()}
            d2 = max(t2, key=t2.get)
            e = {"workload": w2.name, "precision": prec, "n": w2.n, "n_z": w2.n_z, "f": w2.f,
                 "n_in": ni2, "n_out": no2, "scan": [w2.scan[0], w2.scan[1]],
                 "value": w2.n_scan * w2.n_z / (r2["ms_total"] / 3 / 1e3), "unit": UNIT,
                 "ms_per_step": r2["ms_total"] / 3, "steps": 3, "warmup": 2,
                 "clocks": r2["clocks"],
                 "roofline": _roofline(d2, w2, ni2, no2, r2["prof"], 1, peaks, tpk, r2["clocks"]),
                 "kernels": _shares(r2["prof"], 1)}
            if name in ref_samples:
                e["accuracy"] = sampled_eps(g, ctx, w2, name, prec, ref_samples[name], stream)
            extras.append(e)
            del r2
            torch.cuda.empty_cache()
        out["other_configs"] = extras

        # the conventional algorithm on the same GPU, seeded probe sample, per pixel-slice
        if not args.no_quadratic:
            rng = np.random.default_rng(16)
            npos = min(args.quad_probes, wl.n_scan)
            flat = rng.choice(wl.n_scan, size=npos, replace=False)
            pos = [(int(i // wl.scan[0]), int(i % wl.scan[0])) for i in flat]
            g.quadratic_reference_map_for(ctx, wl, positions=pos[:1], stream=stream)
            torch.cuda.synchronize()
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            _, qsteps = g.quadratic_reference_map_for(ctx, wl, positions=pos, stream=stream)
            q1.record(stream)
            torch.cuda.synchronize()
            qs = q0.elapsed_time(q1) / 1e3
            out["gpu_quadratic"] = {"value": npos * wl.n_z / qs, "unit": UNIT, "probes": npos,
                                    "multislice_ops": qsteps,
                                    "sample": f"{npos} seeded probes of the same scan"}
        if not args.no_elastic:
            vdev = torch.from_numpy(wl.vproj).cuda()
            out["elastic"] = elastic_run(g, ctx, wl, vdev, stream, precision)
            del vdev
        torch.cuda.empty_cache()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": precision, "data": "synthetic",
        "config": workload_config(wl, n_in, n_out, precision, args.association, world),
        "e2e": {"value": world * units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "steps": k_e2e},
        "gpu_launches": int(launches_per_step * args.steps),
        "timing": "value: steps between CUDA events on the launch stream, no per-kernel "
                  "instrumentation; kernel shares and the roofline from one more step with "
                  "events around every launch",
        "clocks": clk,
        "autotuner": tuning,
    }
    line.update(out)
    return line


def elastic_run(g, ctx, wl, vdev, stream, precision, reps=3):
    """Time the elastic images and the extra build work of the exit plane."""
    import torch
    dets = [(0.060, 0.0), (0.0, wl.beta)]
    edge = wl.lam * wl.n / (4 * wl.cell)
    if edge <= 0.060:
        return {"skipped": f"band edge {edge * 1e3:.0f} mrad is below the 60 mrad ADF detector"}

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def build():
        g.build_smatrix_for(ctx, wl, vproj=vdev, stream=stream).free()

    t_build = timed(build)
    ctx.set_exit_plane(True)
    try:
        t_build_exit = timed(build)
        sm = g.build_smatrix_for(ctx, wl, vproj=vdev, stream=stream)
        out = torch.zeros((2, wl.scan[1], wl.scan[0]), dtype=torch.float64, device="cuda")
        ctx.profile_read()
        ctx.profile_enable(True)
        t_img = timed(lambda: ctx.elastic_images(sm, wl.scan, dets, out=out, stream=stream))
        ctx.profile_enable(False)
        prof = ctx.profile_read()
        sm.free()
    finally:
        ctx.set_exit_plane(False)
    img = out.cpu().numpy()
    return {"detectors": {"adf": [0.060, None], "bf": [0.0, wl.beta]},
            "images_ms": t_img, "probes_per_s": wl.n_scan / (t_img / 1e3),
            "exit_plane_build_ms": t_build_exit - t_build, "build_ms": t_build,
            "kernels": {k: {"launches": v["launches"] // (reps + 1),
                            "ms": v["ms"] / (reps + 1)} for k, v in prof.items()},
            "adf_mean": float(img[0].mean()), "bf_mean": float(img[1].mean())}


def _window_count(s, r, cell, f):
    """Scan positions whose PRISM window (minimum image within [-L/2f, L/2f)) holds s."""
    d = s - r
    d = d - cell * np.floor(d / cell + 0.5)
    h = cell / (2 * f)
    return int(((d >= -h) & (d < h)).sum())


def contraction_flops(wl, n_in, n_out, kernel):
    """Real flops of the contraction kernels over the whole workload (8 per complex MAC)."""
    rx, ry = wl.scan_positions()
    g1 = g2 = gy = gv = 0
    P = wl.w * wl.w
    for s in range(wl.n_sites):
        nx = _window_count(wl.site_x[s], rx, wl.cell, wl.f)
        ny = _window_count(wl.site_y[s], ry, wl.cell, wl.f)
        if nx and ny:
            g1 += wl.n_types * n_out * P * n_in           # M_n = S_out^H diag(H) S_in
            g2 += wl.n_types * n_out * n_in * nx * ny     # M_n a(R)
            gy += nx * ny * n_in * P                      # Y = S_in a(R), once per site
            gv += wl.n_types * n_out * P * nx * ny        # S_out^H (H . Y)
    for key, val in (("gemm1", g1), ("gemm2", g2), ("gemm_y", gy), ("gemm_v", gv)):
        if key in kernel:
            return 8.0 * val
    return 8.0 * (g1 + g2)


def load_workload(args):
    wl = sp.WORKLOADS[args.workload]()
    if args.max_slices and args.max_slices < wl.n_z:
        k = args.max_slices
        keep = np.nonzero(wl.site_slice < k)[0]
        wl = wl.with_sites(keep)
        wl.vproj = np.ascontiguousarray(wl.vproj[:k])
        wl.n_z = k
        wl.name = f"{wl.name}_first{k}slices"
    return wl


def _request_arrays(req, g, precision):
    # sin_checkpoint -1: the server keeps only checkpoints of S_in for requests whose
    # S-matrices would take more than half of its budget
    return g.make_request(req["vproj"], req["cell"], req["lam"], req["sigma"], req["dz"], req["f"],
                          req["alpha"], req["H"], req["site_slice"], req["win_x0"], req["win_y0"],
                          req["site_x"], req["site_y"], req["scan"], req["beta"],
                          precision=precision, sin_checkpoint=-1)


def _predicted_service_s(req, g):
    """Work model used only to set the arrival rate: multislice beam-steps at the
    measured 512^2 cost scaled by N^2 log N, plus the smaller contraction flop count
    at 600 TFLOP/s."""
    n, nz, f = req["n"], req["n_z"], req["f"]
    n_in = g.count_beams(n, req["cell"], req["lam"], f, req["alpha"])
    n_out = g.count_beams(n, req["cell"], req["lam"], f, req["beta"])
    ms_s = 1.2e-6 * (n_in + n_out) * nz * (n / 512) ** 2 * math.log2(n) / 9.0
    rx = np.array([req["scan"][2] + i * req["scan"][4] for i in range(req["scan"][0])])
    ry = np.array([req["scan"][3] + i * req["scan"][5] for i in range(req["scan"][1])])
    P = req["H"].shape[-1] ** 2
    T = req["n_types"]
    tr = pr = 0.0
    for x, y in zip(req["site_x"], req["site_y"]):
        nr = _window_count(x, rx, req["cell"], f) * _window_count(y, ry, req["cell"], f)
        if nr:
            tr += T * (n_out * P * n_in + n_out * n_in * nr)
            pr += nr * n_in * P + T * n_out * P * nr
    return ms_s + 8 * min(tr, pr) / 600e12


def serving_run(g, n_requests, budget, slots, precision, load=1.5, seed=4, log_path=None):
    """Seeded Poisson stream of mixed map requests through the map server."""
    redrawn = []

    def footprint(req):
        # the server's own rule: S_in checkpointed every ceil(sqrt(2 n_z)) slices when
        # storing every depth would take more than half of the budget
        r, _ = _request_arrays(req, g, precision)
        r.sin_checkpoint = 0
        whole = g.request_footprint(r)
        if whole <= budget // 2:
            return whole, 0
        r.sin_checkpoint = max(2, math.ceil(math.sqrt(2.0 * req["n_z"])))
        return g.request_footprint(r), r.sin_checkpoint

    def accept(req):
        ok = footprint(req)[0] <= budget
        if not ok:
            redrawn.append((req["n"], req["n_z"], req["f"]))
        return ok
    stream = sp.serving_stream(n_requests, seed=seed, accept=accept)
    pred = [_predicted_service_s(r, g) for r in stream]
    srv = g.Server(0, hbm_budget=budget, slots=slots)
    # calibrate the work model: the three requests closest to the median prediction,
    # each run alone through the server, give the measured / predicted time ratio
    order = np.argsort(pred)
    mid = order[max(0, len(order) // 2 - 1): len(order) // 2 + 2]
    meas = []
    for k in mid:
        r, keep = _request_arrays(stream[k], g, precision)
        meas.append(srv.wait(srv.submit(r, keep, stream[k]["n_types"], stream[k]["scan"]))[1])
    scale = float(np.sum(meas) / np.sum([pred[k] for k in mid]))
    srv.close()
    mean_gap = scale * float(np.mean(pred)) / load
    srv = g.Server(0, hbm_budget=budget, slots=slots)
    ids = []
    t0 = time.perf_counter()
    arrival = 0.0
    for req in stream:
        arrival += req["gap"] * mean_gap
        delay = t0 + arrival - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        r, keep = _request_arrays(req, g, precision)
        ids.append(srv.submit(r, keep, req["n_types"], req["scan"]))
    errors = []
    for i in ids:
        try:
            srv.wait(i)
        except g.EelsError as e:
            errors.append(str(e)[:120])
    st = srv.stats()
    infos = [srv.info(i) for i in ids]
    if log_path:   # one JSON line per request
        srv.log_jsonl(log_path, ids, extra={i: {"n": req["n"], "n_z": req["n_z"],
                                                "n_types": req["n_types"], "f": req["f"],
                                                "precision": precision}
                                            for i, req in zip(ids, stream)})
    srv.close()
    fps = [footprint(req) for req in stream]
    return {"requests": n_requests, "slots": slots, "hbm_budget_gb": budget / 2 ** 30,
            "largest_footprint_gb": max(f for f, _ in fps) / 2 ** 30,
            "checkpointed_requests": sum(1 for _, k in fps if k),
            "errors": errors[:4],
            "precision": precision, "offered_load": load, "mean_interarrival_s": mean_gap,
            "model_scale": scale,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
            "mean_wait_ms": st["mean_wait_ms"], "makespan_s": st["makespan_s"],
            "pixel_slices_per_s": st["pixel_slices_per_s"], "completed": st["completed"],
            "failed": st["failed"], "peak_gb": st["peak_bytes"] / 2 ** 30,
            "wave_steps": sum(d["wave_steps"] for d in infos if d["status"] == 0),
            "contraction_tflop": sum(d["contraction_flops"] for d in infos) / 1e12,
            "redrawn_over_budget": len(redrawn), "redrawn_shapes": redrawn[:16],
            "stream": "seeded (4) mixed rocksalt requests: grids 256^2-1024^2, 20-120 slices, "
                      "1-6 channels, f 2-4, scans 16^2-64^2; Poisson arrivals at the offered "
                      "load of a work model calibrated on three requests run alone; draws over "
                      "the budget redrawn; tiles of 4 slices / depths interleaved over the "
                      "slots' issue tokens"}


def reference_arm(args, rank, world):
    """The oracle arm: the FP64 conventional algorithm on the host cores, each step one
    bounded sample of the same workload (its rate extrapolated by the exact multislice
    count), plus the complete map of the small 128^2 case timed without extrapolation."""
    if rank != 0:
        return None
    from oracle import multislice as ms
    smp = OracleSampler(args.workload)
    wl = smp.wl
    precision = args.precision or CONFIG_PRECISION.get(args.workload, "bf16x3")
    n_in = ms.lattice_beams(wl.n, wl.cell, wl.lam, wl.f, wl.alpha)[0].size
    n_out = ms.lattice_beams(wl.n, wl.cell, wl.lam, wl.f, wl.beta)[0].size
    try:
        for _ in range(args.warmup):
            smp.sample()
        vals, ops = [], 0
        t0 = time.perf_counter()
        for _ in range(args.steps):
            rate, sample, rec = smp.sample()
            vals.append(rate)
            ops += rec["ops"]
        total = time.perf_counter() - t0
    finally:
        smp.close()
    value = float(np.mean(vals))
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": workload_config(wl, n_in, n_out, precision, args.association, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": smp.procs, "kind": "oracle",
                             "sample": sample + f"; each step one such sample ({ops} ops over "
                                                f"{args.steps} steps, {total:.1f} s)"},
            "full_small_map": cpu_oracle_full("rocksalt_small"),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(sp.WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["fp32", "tf32", "bf16x3"],
                    help="contraction precision (default: the one the workload's configuration names)")
    ap.add_argument("--quad-probes", type=int, default=4)
    ap.add_argument("--association", default="auto",
                    choices=["auto", "transition_first", "probe_first"])
    ap.add_argument("--sout-scheme", default="stream", choices=["stream", "recompute", "inverse"],
                    help="how S_out reaches each depth (the paper's S_2 variants)")
    ap.add_argument("--s2-study", action="store_true",
                    help="print the S_out scheme thickness study instead of the bench line")
    ap.add_argument("--no-elastic", action="store_true", help="skip the ADF / BF images")
    ap.add_argument("--no-extra", action="store_true", help="skip the other configurations")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip the TF32 / FP32 peak measurements (nominal figures instead)")
    ap.add_argument("--phonons", type=int, default=0,
                    help="print the frozen-phonon average over this many configurations")
    ap.add_argument("--crop-study", action="store_true",
                    help="print the crop-window study (Sec. IV B) instead of the bench line")
    ap.add_argument("--no-quadratic", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-eps", action="store_true", help="skip the FP64-oracle accuracy samples")
    ap.add_argument("--no-serving", action="store_true", help="skip the request stream")
    ap.add_argument("--serving", action="store_true",
                    help="only run the mixed request stream through the map server")
    ap.add_argument("--serving-requests", type=int, default=64)
    ap.add_argument("--serving-budget-gb", type=float, default=240.0)
    ap.add_argument("--serving-slots", type=int, default=4)
    ap.add_argument("--serving-log", default=None,
                    help="append one JSON line per serving request to this file")
    ap.add_argument("--serving-load", type=float, default=1.5,
                    help="offered load of the request stream, as a multiple of the service rate")
    ap.add_argument("--tile-width", type=int, default=0, choices=[0, 128, 256],
                    help="force the output tile width of the tensor-core GEMMs (0: chosen)")
    ap.add_argument("--operand-mib", type=int, default=0,
                    help="device memory (MiB) for one batch's tensor-core operands (0: the "
                         "library's default); small profiling captures")
    ap.add_argument("--max-slices", type=int, default=0,
                    help="keep only the first K slices (smaller device footprint for profiling)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        line = reference_arm(args, rank, world)
        if line is not None:
            print(json.dumps(line))
        return
    # the host work forks worker processes: run it before the first CUDA call
    cpu, ref_samples = None, {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, sample, rec = cpu_oracle_rate(args.workload)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               **rec}
    if rank == 0 and not args.no_eps and not args.max_slices:
        names = [args.workload] + [n for n, _ in EXTRA_CONFIGS
                                   if not args.no_extra and n != args.workload]
        ref_samples = oracle_samples([n for n in names if n in ORACLE_SAMPLES])
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    if args.serving:
        import torch
        from paper_1908_07628_gb300 import build
        build.build()
        import paper_1908_07628_gb300 as g
        torch.cuda.init()
        res = serving_run(g, args.serving_requests, int(args.serving_budget_gb * 2 ** 30),
                          args.serving_slots, args.precision or "bf16x3", load=args.serving_load,
                          log_path=args.serving_log)
        print(json.dumps({"metric": "EELS map serving p99 latency", "value": res["p99_ms"],
                          "unit": "ms", "higher_is_better": False, "n_gpus": 1,
                          "data": "synthetic", "serving": res,
                          "config": {"workload": "mixed map request stream (seed 4)"}}))
        return
    if args.phonons:
        import torch
        from paper_1908_07628_gb300 import build
        build.build()
        import paper_1908_07628_gb300 as g
        res = phonon_run(g, g.Context(0), torch.cuda.current_stream(), args.phonons,
                         args.precision or "tf32")
        print(json.dumps({"study": "frozen-phonon average", "metric": METRIC, "data": "synthetic",
                          **res}))
        return
    if args.crop_study:
        import torch
        from paper_1908_07628_gb300 import build
        build.build()
        import paper_1908_07628_gb300 as g
        res = crop_study(g, g.Context(0), torch.cuda.current_stream())
        print(json.dumps({"study": "crop window of the transition potential (Sec. IV B)",
                          "data": "synthetic", **res}))
        return
    if args.s2_study:
        import torch
        from paper_1908_07628_gb300 import build
        build.build()
        import paper_1908_07628_gb300 as g
        ctx = g.Context(0)
        res = s2_study(g, ctx, torch.cuda.current_stream())
        print(json.dumps({"study": "S_out schemes (Sec. III listing, Sec. IV C inverse multislice)",
                          "data": "synthetic", **res}))
        return
    line = gpu_arm(args, rank, world, ref_samples)
    line["cpu_baseline"] = cpu
    if rank == 0 and not args.no_serving:
        import torch
        import paper_1908_07628_gb300 as g
        torch.cuda.empty_cache()
        line["serving"] = serving_run(g, args.serving_requests, int(args.serving_budget_gb * 2 ** 30),
                                      args.serving_slots, "bf16x3", load=args.serving_load,
                                      log_path=args.serving_log)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
