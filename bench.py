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
DEFAULT_WORKLOAD = "rocksalt_fp32"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x clock
SMS, FP32_LANES = 152, 128
TF32_PER_BF16 = 1.1 / 2.25


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

def _oracle_probe_sample(args):
    """One probe of the conventional oracle with the sites of the deepest slice that
    holds any site in the probe's window (a few hundred multislice operations)."""
    name, iy, ix = args
    import specimen as sp_
    from oracle import multislice as ms
    wl = sp_.WORKLOADS[name]()
    rx, ry = wl.scan_positions()
    seen = [s for s in range(wl.n_sites)
            if ms.axis_in_window(wl.site_x[s], rx[ix], wl.cell, wl.f)
            and ms.axis_in_window(wl.site_y[s], ry[iy], wl.cell, wl.f)]
    deepest = max((int(wl.site_slice[s]) for s in seen), default=0)
    keep = [s for s in seen if wl.site_slice[s] == deepest]
    sub = wl.with_sites(keep)
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


def cpu_oracle_rate(wl_name, budget_procs=None):
    """Pixel-slices/s of the FP64 conventional oracle on this host's cores.

    Sample: one probe per worker process (spread over the scan), each running the
    conventional algorithm with only the sites of one deep slice of its window,
    so every worker does a few hundred multislice operations.  The cost of the
    conventional algorithm is exactly linear in its multislice count, so the
    full-workload rate is the sampled time per operation times the full count.
    """
    wl = sp.WORKLOADS[wl_name]()
    cores = budget_procs or os.cpu_count() or 1
    n_sx, n_sy = wl.scan[0], wl.scan[1]
    jobs = []
    for k in range(cores):
        iy = (k * 7 + 3) % n_sy
        ix = (k * 13 + 5) % n_sx
        jobs.append((wl_name, iy, ix))
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_probe_sample, jobs)
    wall = time.perf_counter() - t0
    per_step = sum(t for t, _ in res) / sum(s for _, s in res)   # seconds per op per core
    full = np.mean([_full_probe_steps(wl, j[1], j[2]) for j in jobs])
    # one core finishes a probe (n_z pixel-slices) in full * per_step seconds
    rate = cores * wl.n_z / (full * per_step)
    sample = (f"{cores} processes x 1 probe of {wl.name}, sites of the deepest occupied slice only "
              f"({sum(s for _, s in res)} multislice ops, {wall:.1f} s wall); rate scaled by "
              f"the full per-probe count {full:.0f} ops")
    return rate, cores, sample


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
    out = {}
    for name, waves in (("row_pass", n_in), ("row_pass_adjoint", n_out)):
        launches = prof.get(name, {}).get("launches", 0) / steps
        out[name] = ("hbm", waves * ((nz - 1) * row + last) + launches * t)
    for name, waves in (("col_pass", n_in), ("col_pass_adjoint", n_out)):
        out[name] = ("hbm", waves * (nz - 1) * col)
    return out


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


def measured_traffic(kernel, n, waves):
    """DRAM bytes per launch from the committed ncu table, if the kernel is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        if ln.startswith("#") or not ln.strip():
            continue
        name, nn, w, sha, nbytes = ln.split()
        if name == kernel and int(nn) == n and w == str(waves) and sha == _source_hash(kernel):
            return float(nbytes)
    return None


def gpu_arm(args, rank, world):
    import torch
    from paper_1908_07628_gb300 import build
    build.build()
    import paper_1908_07628_gb300 as g

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    wl = load_workload(args)
    ctx = g.Context(dev)
    ctx.set_association(args.association)
    ctx.set_sout_scheme(args.sout_scheme)
    stream = torch.cuda.current_stream()
    vdev = torch.from_numpy(wl.vproj).cuda()
    Hdev = torch.from_numpy(wl.H).cuda()
    mdev = torch.zeros((wl.n_types, wl.scan[1], wl.scan[0]), dtype=torch.float64, device="cuda")

    def step():
        sm = g.build_smatrix_for(ctx, wl, vproj=vdev, stream=stream)
        g.inelastic_map_for(ctx, sm, wl, precision=args.precision, H=Hdev, out=mdev, stream=stream)
        sm.free()

    n_in = g.count_beams(wl.n, wl.cell, wl.lam, wl.f, wl.alpha)
    n_out = g.count_beams(wl.n, wl.cell, wl.lam, wl.f, wl.beta)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    ctx.profile_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_total = e0.elapsed_time(e1)
    ctx.profile_enable(False)
    prof = ctx.profile_read()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
        t = torch.tensor([ms_total], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    units = wl.n_scan * wl.n_z
    value = world * units / (ms_step / 1e3)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    vh = torch.from_numpy(wl.vproj).pin_memory().numpy()
    Hh = torch.from_numpy(wl.H).pin_memory().numpy()
    mh = torch.zeros((wl.n_types, wl.scan[1], wl.scan[0]), dtype=torch.float64).pin_memory().numpy()

    def e2e_step():
        sm = g.build_smatrix_for(ctx, wl, vproj=vh, stream=stream)
        g.inelastic_map_for(ctx, sm, wl, precision=args.precision, H=Hh, out=mh, stream=stream)
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

    # accuracy of the timed precision against the FP32 CUDA-core path on the same
    # workload (the FP32 path is pinned to the FP64 oracle by the parity tests)
    acc = None
    if rank == 0 and args.precision != "fp32" and not args.no_eps:
        sm = g.build_smatrix_for(ctx, wl, vproj=vdev, stream=stream)
        ref = g.inelastic_map_for(ctx, sm, wl, precision="fp32", H=Hdev, stream=stream)
        sm.free()
        got = mdev.cpu().numpy()
        acc = {"eps_vs_fp32_path": float(np.sqrt(np.sum((got - ref) ** 2) / np.sum(ref ** 2))),
               "max_abs_rel": float(np.abs(got - ref).max() / np.abs(ref).max())}

    # quadratic algorithm on the same GPU, seeded probe sample, scaled per pixel-slice
    quad = None
    if rank == 0 and not args.no_quadratic:
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
        quad = {"value": npos * wl.n_z / qs, "unit": UNIT, "probes": npos,
                "multislice_ops": qsteps, "sample": f"{npos} seeded probes of the same scan"}

    # elastic by-products (Sec. IV D) of the same S-matrix: ADF (60 mrad inner) and the
    # incoherent bright field with the EELS aperture, plus the exit-plane cost of the build
    elastic = None
    if rank == 0 and not args.no_elastic:
        elastic = elastic_run(g, ctx, wl, vdev, stream, args.precision)

    # roofline of the dominant kernel (CUDA-event times of every launch in the timed region).
    # Tensor peak: the measured burst figure when the sampled clocks show the GPU at its
    # maximum SM clock with no power cap during the timed region, else the sustained one
    # (measured under the power cap at a lower clock).
    peaks = _peaks()
    unthrottled = bool(clk) and "sw_power_cap" not in clk["reasons"] and \
        clk["sm_mhz"] >= 0.97 * clk["sm_max_mhz"]
    bf16_peak = peaks["bf16_tflops"] if unthrottled else peaks["bf16_tflops_sustained"]
    bf16_src = ("measured bf16 burst (clocks at max, no power cap)" if unthrottled
                else "measured bf16 sustained")
    alg = _algorithmic(wl, n_in, n_out, prof, args.steps)
    tot = {k: v["ms"] for k, v in prof.items()}
    dom = max(tot, key=tot.get) if tot else None
    roof = None
    if dom is not None:
        launches = prof[dom]["launches"]
        avg_s = prof[dom]["ms"] / launches / 1e3
        per_step = launches / args.steps          # launches of this kernel in one step
        if dom in alg and alg[dom][0] == "hbm":
            # per step = per launch x launches per step, for bytes and time alike
            bytes_launch = alg[dom][1] / per_step
            achieved = bytes_launch / avg_s / 1e9
            waves = n_out if "adjoint" in dom else n_in
            roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                    "traffic": measured_traffic(dom, wl.n, waves),
                    "algorithmic_bytes": bytes_launch,
                    "peak_source": "measured" if "fallback" not in peaks else "fallback"}
        elif "bf16x3" in dom:
            useful = contraction_flops(wl, n_in, n_out, dom)
            # the tensor pipe runs three BF16 products per real product (hi*hi, hi*lo, lo*hi)
            peak = bf16_peak
            achieved = 3 * useful / per_step / avg_s / 1e12
            roof = {"kernel": dom, "bound": "tensor", "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                    "useful_tflops": useful / per_step / avg_s / 1e12,
                    "peak_source": bf16_src}
        elif "tf32" in dom:
            flops = contraction_flops(wl, n_in, n_out, dom)
            # TF32 dense = 1.1 / 2.25 of BF16 (nominal)
            peak = bf16_peak * TF32_PER_BF16
            achieved = flops / per_step / avg_s / 1e12
            roof = {"kernel": dom, "bound": "tensor", "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": measured_traffic(dom, wl.n, "batch"),
                    "peak_source": bf16_src + " x nominal tf32/bf16 (1.1/2.25)"}
        else:
            flops = contraction_flops(wl, n_in, n_out, dom)
            mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
            peak = SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12
            achieved = flops / per_step / avg_s / 1e12
            roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                    "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz (sampled)"}
    # every multislice kernel against the HBM bound (the dominant one is in roofline) and
    # against the FP32 ALU bound: per wave and slice the row pass runs two N-point FFTs on
    # N rows and one complex multiply per pixel (10 N^2 log2 N + 6 N^2 flop), the column
    # pass two N-point FFTs on the N/2 band columns and the propagator multiply
    # (5 N^2 log2 N + 3 N^2 flop)
    mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = SMS * FP32_LANES * 2 * mhz * 1e6
    lg = math.log2(wl.n)
    nn = float(wl.n) ** 2
    # (the last row pass of each sweep stops after the inverse FFT and the multiply)
    row_full, row_last = 10 * nn * lg + 6 * nn, 5 * nn * lg + 6 * nn
    col = 5 * nn * lg + 3 * nn
    fft = {"row_pass": n_in * ((wl.n_z - 1) * row_full + row_last),
           "row_pass_adjoint": n_out * ((wl.n_z - 1) * row_full + row_last),
           "col_pass": n_in * (wl.n_z - 1) * col,
           "col_pass_adjoint": n_out * (wl.n_z - 1) * col}
    hbm = {}
    for k in alg:
        if k not in prof or prof[k]["ms"] <= 0:
            continue
        sec = prof[k]["ms"] / args.steps / 1e3
        hbm[k] = {"achieved_gbs": alg[k][1] / sec / 1e9,
                  "frac": alg[k][1] / sec / 1e9 / peaks["hbm_gbs"],
                  "fft_tflops": fft[k] / sec / 1e12,
                  "fp32_frac": fft[k] / sec / fp32_peak}
    share = {k: {"launches": prof[k]["launches"], "ms_per_step": prof[k]["ms"] / args.steps,
                 "share": prof[k]["ms"] / max(sum(tot.values()), 1e-9)} for k in prof}
    launches_per_step = sum(v["launches"] for v in prof.values()) / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"tf32": "tf32", "bf16x3": "bf16x3"}.get(args.precision, "f32"), "data": "synthetic",
        "config": {"workload": wl.name, "n": wl.n, "n_z": wl.n_z, "f": wl.f, "n_in": n_in,
                   "n_out": n_out, "scan": [wl.scan[0], wl.scan[1]], "n_types": wl.n_types,
                   "precision": args.precision, "association": args.association,
                   "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (S_in alone is "
                         f"{wl.n_z * n_in * (wl.n // 2) ** 2 * 8 / 1e9:.1f} GB)"},
        "e2e": {"value": world * units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "roofline": roof,
        "multislice_hbm": hbm,
        "kernels": share,
        "clocks": clk,
        "gpu_quadratic": quad,
        "accuracy": acc,
        "elastic": elastic,
    }
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
    return g.make_request(req["vproj"], req["cell"], req["lam"], req["sigma"], req["dz"], req["f"],
                          req["alpha"], req["H"], req["site_slice"], req["win_x0"], req["win_y0"],
                          req["site_x"], req["site_y"], req["scan"], req["beta"],
                          precision=precision)


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


def serving_run(g, n_requests, budget, slots, precision, load=1.5, seed=4):
    """Seeded Poisson stream of mixed map requests through the map server."""
    accept = lambda req: g.request_footprint(_request_arrays(req, g, precision)[0]) <= budget
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
    for i in ids:
        srv.wait(i)
    st = srv.stats()
    srv.close()
    return {"requests": n_requests, "slots": slots, "hbm_budget_gb": budget / 2 ** 30,
            "precision": precision, "offered_load": load, "mean_interarrival_s": mean_gap,
            "model_scale": scale,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
            "mean_wait_ms": st["mean_wait_ms"], "makespan_s": st["makespan_s"],
            "pixel_slices_per_s": st["pixel_slices_per_s"], "completed": st["completed"],
            "failed": st["failed"], "peak_gb": st["peak_bytes"] / 2 ** 30,
            "stream": "seeded (4) mixed rocksalt requests: grids 256^2-1024^2, 20-120 slices, "
                      "1-6 channels, f 2-4, scans 16^2-64^2; Poisson arrivals at the offered "
                      "load of a work model calibrated on three requests run alone; draws over "
                      "the budget redrawn"}


def reference_arm(args, rank, world):
    if rank != 0:
        return None
    wl = sp.WORKLOADS[args.workload]()
    vals = []
    for _ in range(args.warmup):
        cpu_oracle_rate(args.workload)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rate, cores, sample = cpu_oracle_rate(args.workload)
        vals.append(rate)
    wall = time.perf_counter() - t0
    value = float(np.mean(vals))
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": wl.n_scan * wl.n_z / value * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": wl.name, "precision": "fp64 oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(sp.WORKLOADS))
    ap.add_argument("--precision", default="tf32", choices=["fp32", "tf32", "bf16x3"])
    ap.add_argument("--quad-probes", type=int, default=8)
    ap.add_argument("--association", default="auto",
                    choices=["auto", "transition_first", "probe_first"])
    ap.add_argument("--sout-scheme", default="stream", choices=["stream", "recompute", "inverse"],
                    help="how S_out reaches each depth (the paper's S_2 variants)")
    ap.add_argument("--s2-study", action="store_true",
                    help="print the S_out scheme thickness study instead of the bench line")
    ap.add_argument("--no-elastic", action="store_true", help="skip the ADF / BF images")
    ap.add_argument("--phonons", type=int, default=0,
                    help="print the frozen-phonon average over this many configurations")
    ap.add_argument("--crop-study", action="store_true",
                    help="print the crop-window study (Sec. IV B) instead of the bench line")
    ap.add_argument("--no-quadratic", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-eps", action="store_true", help="skip the FP32 accuracy reference")
    ap.add_argument("--no-serving", action="store_true", help="skip the short serving stream")
    ap.add_argument("--serving", action="store_true",
                    help="only run the mixed request stream through the map server")
    ap.add_argument("--serving-requests", type=int, default=64)
    ap.add_argument("--serving-budget-gb", type=float, default=160.0)
    ap.add_argument("--serving-slots", type=int, default=4)
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
    # the CPU sample forks worker processes: run it before the first CUDA call
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, sample = cpu_oracle_rate(args.workload)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
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
                          args.serving_slots, args.precision)
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
                         args.precision)
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
    line = gpu_arm(args, rank, world)
    line["cpu_baseline"] = cpu
    if rank == 0 and not args.no_serving:
        import paper_1908_07628_gb300 as g
        line["serving"] = serving_run(g, 12, 48 << 30, 3, args.precision)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
