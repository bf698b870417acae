"""Benchmark: EC-curve throughput of a 512^3 float32 field with 1024 levels.

One step = one full curve request (EC, surface area and volume curves)
through the C ABI: scratch reset, the spacing check of the thresholds, the
histogram kernel over every voxel, the scan.  Inputs are resident in HBM
before the timed region (537 MB, larger than L2, so no flush is needed
between steps).  Prints one JSON line, which also carries the same step with
all four descriptors, the end-to-end number through the host-buffer call,
the same request streamed from a raw file, the contribution-type map of the
same field (22 vertex types x 1024 levels)
the batched-versus-per-field comparison on the served request mix, and
sensor frames of 36 small tiles served one frame at a time, and the 2048^3
low-memory workload streamed from its on-device generator under a 4 GB cap.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  python bench.py --profile-case [typemap|2d|rows|hashbox]
                                     (the curve kernel, or the type map, alone
                                      on a 256 x 512 x 512 slab of the field;
                                      the 2D kernel on the 16384^2 uint8 field;
                                      the curve kernel on a 256 x 511 x 511
                                      slab (rows not a multiple of 16 bytes);
                                      or one 66-plane slab of the 2048^2
                                      hash-box generator; for ncu captures)

--impl reference times the CPU oracle (the plain cell-counting reference) on
this machine's host cores, on a bounded sample of the same workload.
Under torchrun (N > 1) every rank processes its own copy of the workload
(independent fields, no data-path collective) and the slowest rank's time
is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EC-curve Gvoxels/s & % HBM peak (512³ f32, 1024 lvls); batched vs per-field"
WORKLOAD = ("512^3 float32 density: 2000 Gaussian blobs (r~U[3,12], a~U[0.5,1.5]) + N(0,0.05^2) noise, "
            "seed 3; 1024 uniform thresholds over [min,max]; EC, surface-area and volume curves (int64), "
            "26-connectivity")
N = 512
L = 1024
DESC = 13            # EC | AREA | VOLUME
DESC_ALL = 15        # EC | PERIMETER | AREA | VOLUME
KERNEL = "k_planar3d"
LAUNCHES_PER_STEP = 3   # spacing check, histogram kernel, scan
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_planar3d_512cube_f32.json")


# Files that define the profiled kernel (k_planar3d and what it inlines):
# the stored ncu traffic is used only while they are unchanged.
KERNEL_SOURCES = ("ec_planar3d.cu", "ec_slice.h", "ec_fast3d.cuh", "ec_swar.h", "ec_rules.h", "ec_internal.h")
# The contribution-type map's histogram kernel (k_types3) and its summary.
TYPEMAP_KERNEL = "k_types3"
TYPEMAP_SOURCES = ("ec_typemap.cu", "ec_types.h", "ec_fast3d.cuh", "ec_rules.h", "ec_internal.h")
TYPEMAP_SUMMARY = os.path.join(ROOT, "profiles", "k_types3_512cube_f32.json")


def kernel_source_hash(sources=KERNEL_SOURCES) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2311_11740_gb300", "csrc")
    for f in sources:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
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
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), active=parts[4],
                                     hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


def traffic_per_launch(summary=PROFILE_SUMMARY, sources=KERNEL_SOURCES):
    """DRAM bytes per launch of a kernel from its committed ncu summary, or
    None when the kernel's sources changed since the capture."""
    if not os.path.exists(summary):
        return None
    with open(summary) as f:
        d = json.load(f)
    if d.get("kernel_source_hash") != kernel_source_hash(sources):
        return None
    return d.get("dram_bytes_per_full_launch")


def cpu_baseline(field_cpu, thr_cpu, budget_s: float):
    """The oracle on all host cores and on one core, each for about half of
    `budget_s` (see cpu_baseline_once)."""
    import oracle
    full = cpu_baseline_once(field_cpu, thr_cpu, budget_s * 0.55)
    oracle.set_threads(1)
    try:
        one = cpu_baseline_once(field_cpu, thr_cpu, budget_s * 0.45)
    finally:
        oracle.set_threads(0)
    full["one_core"] = one
    return full


def cpu_baseline_once(field_cpu, thr_cpu, budget_s: float):
    """Time the oracle (as it stands) on a bounded sample of the workload:
    whole passes over the field (or over its first z-planes when one pass
    would exceed the budget), repeated until about `budget_s` seconds."""
    import numpy as np
    import oracle
    thr = thr_cpu.numpy()
    probe = np.ascontiguousarray(field_cpu[:4].numpy())
    t0 = time.perf_counter()
    oracle.ec_curves(probe, thr, L, 26, DESC)
    per_plane = (time.perf_counter() - t0) / 4
    planes = int(max(4, min(field_cpu.shape[0], budget_s / max(per_plane, 1e-6))))
    sample = np.ascontiguousarray(field_cpu[:planes].numpy())
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.ec_curves(sample, thr, L, 26, DESC)
        reps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    vox = sample.size * reps
    return {"value": vox / dt / 1e9, "unit": "Gvoxels/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{reps} pass(es) over the first {planes} z-planes ({sample.size} voxels each) of the same "
                      f"field and thresholds, EC+area+volume, {dt:.1f} s"}


def time_device(fn, steps):
    import torch
    stream = torch.cuda.current_stream()
    st, en = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    st.record(stream)
    for _ in range(steps):
        fn()
    en.record(stream)
    torch.cuda.synchronize()
    return st.elapsed_time(en) / steps


def stratified_subset(reqs, per_stratum, seed):
    """Indices of a stratified sample of the request stream: for each kind
    (2D, 3D) the requests split into side quartiles and per_stratum drawn
    from each, plus the largest field of each kind."""
    import numpy as np
    rng = np.random.default_rng(seed)
    pick = set()
    for nd in (2, 3):
        idx = [i for i, r in enumerate(reqs) if r["ndim"] == nd]
        idx.sort(key=lambda i: reqs[i]["side"])
        pick.add(idx[-1])
        for q in range(4):
            part = idx[len(idx) * q // 4:len(idx) * (q + 1) // 4]
            pick.update(int(i) for i in rng.choice(part, size=min(per_stratum, len(part)), replace=False))
    return sorted(pick)


def config5_section(ec, ctx, n_requests, seed=5, loads=(0.5, 0.9, 1.2), with_oracle=True):
    """The batched/served workload at its stated size: n_requests requests,
    70 % 2D uint8 (side log-uniform 64..4096, 256 levels, EC+perimeter+area)
    and 30 % 3D float32 (side log-uniform 32..512, 64..1024 uniform
    thresholds, EC+perimeter+area+volume), each a smoothed GRF generated on
    the device.  Timed three ways on the same device-resident fields: one
    ec_curve call per field; one ec_batch (persistent launch in a CUDA
    graph) with the autotuner choosing its plan (tuned on the first, untimed
    call) and with the default plan; and the continuous-admission server
    (slots tuned the same way, an untimed burst first) under Poisson
    arrivals at 0.5, 0.9 and 1.2 of its closed-loop capacity.  All paths
    must agree; a stratified subset of at least 256 requests (with the
    largest field of each kind) is checked against the oracle."""
    import numpy as np
    import torch
    from paper_2311_11740_gb300 import workloads
    reqs = workloads.request_stream(seed=seed, n=n_requests, max_2d=4096, max_3d=512)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fields, cells = [], 0
    for r in reqs:
        f, thr = workloads.request_field_device(r, device="cuda")
        fields.append(dict(field=f, thresholds=thr, L=r["L"], descriptors=7 if r["ndim"] == 2 else 15))
        cells += f.numel()
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    field_bytes = sum(d["field"].numel() * d["field"].element_size() for d in fields)

    # one launch sequence per field
    outs = [ec.curve(d["field"], d["thresholds"], L=d["L"], descriptors=d["descriptors"], ctx=ctx) for d in fields]
    per_ms = time_device(lambda: [ec.curve(d["field"], d["thresholds"], L=d["L"], descriptors=d["descriptors"],
                                           ctx=ctx, out=o) for d, o in zip(fields, outs)], 2)
    # one batched launch: default plan, then the autotuned plan
    plain = ec.Batch(fields, ctx=ctx)
    plain.run()
    plain_ms = time_device(plain.run, 3)
    same = all(torch.equal(a, b) for a, b in zip(outs, plain.outs))
    tctx = ec.Context(torch.cuda.current_device())
    tctx.set_option(ec.EC_OPT_AUTOTUNE, 1)
    tuned = ec.Batch(fields, ctx=tctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tuned.run()   # the first batch of its mix class times the candidate plans
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    tuned_ms = time_device(tuned.run, 3)
    same &= all(torch.equal(a, b) for a, b in zip(outs, tuned.outs))
    plan = tuned.tuned_plan()

    # served: device-resident fields, host thresholds and outputs
    host_thr = [None if d["thresholds"] is None else d["thresholds"].cpu().numpy() for d in fields]
    reqs_sv = [dict(field=d["field"], thresholds=t, L=d["L"], descriptors=d["descriptors"])
               for d, t in zip(fields, host_thr)]
    want = [o.cpu().numpy() for o in outs]
    sv = ec.Server(device_mem_budget=8 << 30, max_slots=8, ctx=tctx)
    served_ok = all(np.array_equal(sv.wait(t, 600000), w) for t, w in zip(sv.submit_many(reqs_sv), want))
    t0 = time.perf_counter()
    tickets = sv.submit_many(reqs_sv)   # closed loop: the whole stream at once
    sv.wait_all(600000)
    cap_s = time.perf_counter() - t0
    served_ok &= all(np.array_equal(sv.result(t), w) for t, w in zip(tickets, want))
    served = {"closed_loop_gcells_s": cells / cap_s / 1e9, "closed_loop_ms": cap_s * 1e3, "slots": 8,
              "fields": "device-resident (read in place); thresholds and outputs through host memory",
              "loads": []}
    rng = np.random.default_rng(seed)

    def poisson_pass(rho):
        rate = rho * len(reqs_sv) / cap_s
        gaps = rng.exponential(1.0 / rate, size=len(reqs_sv))
        t0 = time.perf_counter()
        due = t0
        tickets = []
        for r, g in zip(reqs_sv, gaps):
            due += g
            while time.perf_counter() < due:
                pass
            tickets.append(sv.submit(**r))
        ok = all(np.array_equal(sv.wait(t, 600000), w) for t, w in zip(tickets, want))
        return rate, time.perf_counter() - t0, ok

    # untimed pass at the lowest load: the groups that arrivals form (smaller
    # than the closed loop's) meet their mix classes, so tuning stays out of
    # the timed passes
    served_ok &= poisson_pass(loads[0])[2]
    for rho in loads:
        sv.reset_stats()
        rate, span, ok = poisson_pass(rho)
        served_ok &= ok
        st = sv.stats()
        served["loads"].append({"offered_load": rho, "offered_rate_req_s": rate, "gcells_s": cells / span / 1e9,
                                "p50_us": st["p50_us"], "p99_us": st["p99_us"], "mean_us": st["mean_us"]})
    sv.close()
    res = {"workload": f"{len(fields)} requests, seed {seed}: 70% 2D uint8 (side log-uniform 64..4096, 256 "
                       f"levels, EC+perimeter+area), 30% 3D float32 (side log-uniform 32..512, 64..1024 "
                       f"thresholds, all four descriptors), smoothed GRFs (sigma 2..10) generated on the device",
           "requests": len(fields), "cells": cells, "field_bytes": field_bytes, "generate_s": gen_s,
           "largest": {"2d_side": max(r["side"] for r in reqs if r["ndim"] == 2),
                       "3d_side": max(r["side"] for r in reqs if r["ndim"] == 3)},
           "per_field_ms": per_ms, "per_field_gcells_s": cells / per_ms / 1e6,
           "batched_default_ms": plain_ms, "batched_default_gcells_s": cells / plain_ms / 1e6,
           "batched_ms": tuned_ms, "batched_gcells_s": cells / tuned_ms / 1e6,
           "autotune": {"on": True, "tuning_call_s": tune_s,
                        "plan": None if plan is None else dict(zip(("tz3", "grid", "rows2d"), plan)),
                        "candidates": "3D item depth 16/32/64, 2D item rows 32/64/128, grid all-resident or "
                                      "one block per SM (coordinate descent)"},
           "served": served, "identical": bool(same and served_ok)}
    del tuned, plain
    tctx.close()
    if with_oracle:
        import oracle
        sub = stratified_subset(reqs, 32, seed)
        t0 = time.perf_counter()
        ok = True
        for i in sub:
            d = fields[i]
            f = d["field"].cpu().numpy()
            thr = None if d["thresholds"] is None else d["thresholds"].cpu().numpy()
            conn = 8 if f.ndim == 2 else 26
            ok &= bool(np.array_equal(oracle.ec_curves(f, thr, d["L"], conn, d["descriptors"]), want[i]))
        res["identical_to_oracle"] = ok
        res["oracle_subset"] = {"requests": len(sub), "cells": int(sum(fields[i]["field"].numel() for i in sub)),
                                "strata": "2D and 3D each split into side quartiles, 32 drawn per quartile, "
                                          "plus the largest field of each kind",
                                "oracle_s": time.perf_counter() - t0}
    del fields, outs
    torch.cuda.empty_cache()
    return res


def type_map_section(ec, ctx, field, thr, steps, with_cpu, budget_s):
    """The contribution-type map of the same field (ec_type_map: the 22
    Table 2 types at each of the 1024 levels), timed per call; the library's
    Table 2 weights applied to it (ec_apply_weights) must give the curve
    request's EC, perimeter, area and volume curves.  The CPU leg times the
    oracle (the definition, level by level) on one level pass over a
    bounded sample and scales it to all L levels."""
    import numpy as np
    import torch
    nt = ec.NTYPES[3]
    counts = torch.empty((nt, L), dtype=torch.int64, device="cuda")
    ec.type_map(field, thr, out=counts, ctx=ctx)
    # weights per type from the library's per-mask table: any mask of the type
    tt, vt = ec.type_table(3), ec.vertex_table_3d()
    W = np.stack([vt[int(np.flatnonzero(tt == t)[0])] for t in range(nt)], axis=1).astype(np.int32)
    curves = ec.apply_weights(counts, W, [8, 2, 4, 8], ctx=ctx)
    same = torch.equal(curves, ec.curve(field, thr, descriptors=DESC_ALL, ctx=ctx))
    torch.cuda.synchronize()
    ctx.profile_read()
    ms = time_device(lambda: ec.type_map(field, thr, out=counts, ctx=ctx), steps)
    kms, kl = ctx.profile_read()
    kus = kms / max(kl, 1) * 1e3
    wus = time_device(lambda: ec.apply_weights(counts, W, [8, 2, 4, 8], out=curves, ctx=ctx), steps) * 1e3
    peak, peak_kind = measured_peaks()
    vox = field.numel()
    out = {"workload": "the same 512^3 float32 field and 1024 thresholds; counts of the 22 Table 2 vertex types "
                       "at every level (int64 [22][1024]) over the 513^3 vertices",
           "ms_per_step": ms, "value": vox / ms / 1e6, "unit": "Gvoxels/s",
           "per_step": "ec_type_map: memset + k_types3 + k_type_scan + k_type_empty",
           "gpu_launches_per_step": 3,
           "roofline": {"bound": "hbm", "kernel": TYPEMAP_KERNEL, "achieved": vox * 4 / (kus * 1e-6) / 1e9,
                        "peak": peak, "unit": "GB/s", "frac": vox * 4 / (kus * 1e-6) / 1e9 / peak,
                        "peak_source": peak_kind,
                        "traffic": traffic_per_launch(TYPEMAP_SUMMARY, TYPEMAP_SOURCES),
                        "kernel_avg_us": kus, "algorithmic_bytes_per_launch": vox * 4},
           "apply_weights_us": wus, "weighted_equals_curves": bool(same)}
    if with_cpu:
        from oracle import typemap as tm
        import oracle
        f_cpu, t_np = field.cpu(), thr.cpu().numpy()
        planes = 8
        t0 = time.perf_counter()
        tm.type_counts_at(oracle.bin_field(np.ascontiguousarray(f_cpu[:planes].numpy()), t_np, L), L, L // 2)
        per_plane = (time.perf_counter() - t0) / planes
        planes = int(max(8, min(field.shape[0], budget_s / 3 / max(per_plane, 1e-6))))
        sample = np.ascontiguousarray(f_cpu[:planes].numpy())
        t0 = time.perf_counter()
        bins = oracle.bin_field(sample, t_np, L)
        t_bin = time.perf_counter() - t0
        ks = (0, L // 2, L - 1)
        t0 = time.perf_counter()
        for k in ks:
            tm.type_counts_at(bins, L, k)
        t_level = (time.perf_counter() - t0) / len(ks)
        est = t_bin + L * t_level
        out["cpu_baseline"] = {"value": sample.size / est / 1e9, "unit": "Gvoxels/s", "cores": 1, "kind": "oracle",
                               "sample": f"oracle binning + 3 of the 1024 level passes over the first {planes} "
                                         f"z-planes ({sample.size} voxels), scaled to 1024 levels "
                                         f"({t_bin:.2f} s + 1024 x {t_level:.3f} s)"}
    return out


def configs_2d_section(ec, ctx, steps=20, with_cpu=True):
    """The 2D workloads: a 256^2 uint8 field (256 identity levels; small,
    so launch-latency bound: microseconds per request) and the 16384^2
    field as uint8 (256 levels) and as float32 (1024 uniform thresholds),
    EC + perimeter + area, 8-connectivity.  Per request: device time of the
    whole request (memset, spacing check, histogram kernel, scan) and of the
    histogram kernel alone, with its HBM roofline (1 or 4 bytes per pixel).
    The oracle is timed on all host cores and on one core on a bounded
    sample (the first rows of the field)."""
    import numpy as np
    import oracle
    from paper_2311_11740_gb300 import workloads
    peak, peak_kind = measured_peaks()
    desc = ec.EC_DESC_EC | ec.EC_DESC_PERIMETER | ec.EC_DESC_AREA
    out = {}
    try:
        g1 = workloads.config1(device="cuda")
        o1 = torch_empty((3, 256))
        ec.curve(g1, None, L=256, descriptors=desc, out=o1, ctx=ctx)
        ctx.profile_read()
        ms = time_device(lambda: ec.curve(g1, None, L=256, descriptors=desc, out=o1, ctx=ctx), 200)
        kms, kl = ctx.profile_read()
        kus = kms / max(kl, 1) * 1e3
        want1 = oracle.ec_curves(g1.cpu().numpy(), None, 256, 8, desc)
        c1 = {"workload": "256^2 uint8 smoothed GRF (seed 1, sigma 4), 256 identity levels, EC+perimeter+area",
              "us_per_field": ms * 1e3, "kernel_avg_us": kus,
              "roofline": {"bound": "hbm", "kernel": "k_pixel2d_fast", "achieved": 65536 / (kus * 1e-6) / 1e9,
                           "peak": peak, "unit": "GB/s", "frac": 65536 / (kus * 1e-6) / 1e9 / peak,
                           "peak_source": peak_kind, "traffic": None, "algorithmic_bytes_per_launch": 65536,
                           "note": "64 KiB per request: launch-latency bound, not bandwidth bound"},
              "identical": bool(np.array_equal(o1.cpu().numpy(), want1))}
        if with_cpu:
            c1["cpu_baseline"] = {}
            for cores in (0, 1):
                oracle.set_threads(cores)
                h1 = g1.cpu().numpy()
                t0, reps = time.perf_counter(), 0
                while time.perf_counter() - t0 < 1.0:
                    oracle.ec_curves(h1, None, 256, 8, desc)
                    reps += 1
                c1["cpu_baseline"]["all_cores" if cores == 0 else "one_core"] = {
                    "us_per_field": (time.perf_counter() - t0) / reps * 1e6,
                    "cores": oracle.num_threads(), "kind": "oracle", "sample": f"{reps} whole fields"}
            oracle.set_threads(0)
        out["config1"] = c1
        u8, f32, thr = workloads.config2(device="cuda")
        c2 = {"workload": "16384^2 smoothed GRF (seed 2, sigma 16, periodic FFT): uint8 with 256 identity levels "
                          "and the float32 copy with 1024 uniform thresholds; EC+perimeter+area"}
        for name, fld, t, Lr, nbytes in (("u8", u8, None, 256, u8.numel()), ("f32", f32, thr, 1024, f32.numel() * 4)):
            o = torch_empty((3, Lr))
            ec.curve(fld, t, L=Lr, descriptors=desc, out=o, ctx=ctx)
            ctx.profile_read()
            ms = time_device(lambda: ec.curve(fld, t, L=Lr, descriptors=desc, out=o, ctx=ctx), steps)
            kms, kl = ctx.profile_read()
            kus = kms / max(kl, 1) * 1e3
            ach = nbytes / (kus * 1e-6) / 1e9
            c2[name] = {"ms_per_step": ms, "value": fld.numel() / ms / 1e6, "unit": "Gpixels/s",
                        "roofline": {"bound": "hbm", "kernel": "k_pixel2d_fast", "achieved": ach, "peak": peak,
                                     "unit": "GB/s", "frac": ach / peak, "peak_source": peak_kind, "traffic": None,
                                     "kernel_avg_us": kus, "algorithmic_bytes_per_launch": nbytes}}
            # invariants at full size: the top level holds every pixel
            top = o[:, -1].cpu().numpy()
            c2[name]["top_level_invariants"] = bool(top[0] == 1 and top[1] == 2 * (16384 + 16384)
                                                    and top[2] == 16384 * 16384)
        if with_cpu:
            rows = 1024
            sample = np.ascontiguousarray(u8[:rows].cpu().numpy())
            c2["cpu_baseline"] = {}
            for cores in (0, 1):
                oracle.set_threads(cores)
                t0 = time.perf_counter()
                oracle.ec_curves(sample, None, 256, 8, desc)
                dt = time.perf_counter() - t0
                c2["cpu_baseline"]["all_cores" if cores == 0 else "one_core"] = {
                    "value": sample.size / dt / 1e9, "unit": "Gpixels/s", "cores": oracle.num_threads(),
                    "kind": "oracle", "sample": f"the first {rows} rows of the uint8 field ({sample.size} pixels)"}
            oracle.set_threads(0)
        out["config2"] = c2
        del u8, f32, thr
    except Exception as e:   # the optional leg must not cost the line
        out["error"] = f"{type(e).__name__}: {e}"
    return out


def torch_empty(shape):
    import torch
    return torch.empty(shape, dtype=torch.int64, device="cuda")


def file_stream_section(ec, ctx, field, thr, want, reps=3):
    """Low-memory streaming straight from a raw file (ec_curve_3d_file): the
    field written to a temporary file (so it is served from the page cache),
    then 64-plane slabs read by pread into page-locked staging and counted
    while the next slab is read.  Wall-clock per call, results checked."""
    import numpy as np
    fd, path = tempfile.mkstemp(suffix=".raw")
    try:
        with os.fdopen(fd, "wb") as fh:
            fh.write(field.cpu().numpy().tobytes())
        thr_h = thr.cpu().numpy()
        got = ec.curve_3d_file(path, tuple(field.shape), np.float32, thresholds=thr_h, descriptors=DESC, ctx=ctx)
        t0 = time.perf_counter()
        for _ in range(reps):
            got = ec.curve_3d_file(path, tuple(field.shape), np.float32, thresholds=thr_h, descriptors=DESC,
                                   ctx=ctx)
        dt = (time.perf_counter() - t0) / reps
        return {"workload": "the same 512^3 float32 field as a raw file (page cache), 64-plane slabs, "
                            "EC+area+volume", "ms_per_call": dt * 1e3, "value": field.numel() / dt / 1e9,
                "unit": "Gvoxels/s", "file_bytes": field.numel() * 4,
                "identical": bool(np.array_equal(got, want))}
    except Exception as e:   # the optional leg must not cost the line
        return {"error": f"{type(e).__name__}: {e}"}
    finally:
        os.unlink(path)


def realtime_frames_section(ec, ctx, nframes=300, seed=7):
    """Real-time sensor frames (the microscopy case study, Sec. 3, and Sec. 4):
    each frame is 36 grid squares of 134 x 134 uint8 pixels (smoothed GRF
    stand-ins, the micrographs are not available), EC + perimeter + area over
    256 levels, submitted from page-locked host memory to the server one
    frame at a time; a frame's latency runs from its submission until all 36
    curves are back on the host.  The paper asks for 36 squares at 30 frames
    per second (19 Mpixels/s)."""
    import numpy as np
    import oracle
    from paper_2311_11740_gb300 import workloads
    try:
        tiles = [workloads.quantize_u8(workloads.grf_2d(seed * 1000 + i, 134, 134, 4.0)).contiguous()
                 for i in range(36)]
        want = [oracle.ec_curves(t.numpy(), None, 256, 8, 7) for t in tiles]
        t0 = time.perf_counter()
        for t in tiles:
            oracle.ec_curves(t.numpy(), None, 256, 8, 7)
        oracle_ms = (time.perf_counter() - t0) * 1e3
        reqs = [(t.pin_memory(), None, 256, 7) for t in tiles]
        sv = ec.Server(device_mem_budget=1 << 30, max_slots=4, ctx=ctx)
        try:
            ok = all(np.array_equal(sv.wait(t, 60000), w) for t, w in zip(sv.submit_many(reqs), want))
            lat = []
            for _ in range(nframes):
                t0 = time.perf_counter()
                tickets = sv.submit_many(reqs)
                sv.wait_all(60000)
                lat.append(time.perf_counter() - t0)
            ok &= all(np.array_equal(sv.result(t), w) for t, w in zip(tickets, want))
        finally:
            sv.close()
        us = sorted(x * 1e6 for x in lat)
        mean = sum(lat) / len(lat)
        px = 36 * 134 * 134
        return {"workload": "frames of 36 grid squares of 134 x 134 uint8 (smoothed GRFs, seed 7), 256 levels, "
                            "EC+perimeter+area, page-locked host tiles through ec_server, one frame in flight",
                "frames": nframes, "p50_us": us[len(us) // 2], "p99_us": us[min(len(us) - 1, int(0.99 * len(us)))],
                "frames_per_s": 1.0 / mean, "mpixels_s": px / mean / 1e6, "needed_mpixels_s_at_30fps": px * 30 / 1e6,
                "oracle_ms_per_frame": oracle_ms, "oracle_cores": oracle.num_threads(), "identical": bool(ok)}
    except Exception as e:   # the optional leg must not cost the line
        return {"error": f"{type(e).__name__}: {e}"}


def streamed_2048_section(ec, ctx, n=2048, cap=4 << 30):
    """The low-memory workload: a 2048^3 uint16 hash-box field (4096 identity
    levels, EC + volume) generated on the device slab by slab (64 planes and
    their halo planes) and counted under a 4 GB device-memory cap; the field
    (17.2 GB) is never resident.  Wall clock of the whole pass (generation
    included) and the summed device time of the histogram kernels alone."""
    import numpy as np
    try:
        spec = ec.HashboxSpec(4, 0, 0, 0, n, n)
        kw = dict(L=4096, descriptors=ec.EC_DESC_EC | ec.EC_DESC_VOLUME, slab_planes=64, device_mem_cap=cap,
                  ctx=ctx)
        ec.hashbox_stream(spec, n, **kw)          # warm-up (buffers, streams)
        ctx.profile_read()
        t0 = time.perf_counter()
        got = ec.hashbox_stream(spec, n, **kw)
        dt = time.perf_counter() - t0
        kms, kl = ctx.profile_read()
        vox = n ** 3
        peak, peak_kind = measured_peaks()
        ok = bool(got[0, -1] == 1 and got[1, -1] == vox and np.all(np.diff(got[1]) >= 0))
        return {"workload": f"{n}^3 uint16 hash-box field (seed 4, 5^3 box of a MurmurHash3-finaliser counter hash), 4096 identity "
                            f"levels, EC+volume, 64-plane slabs generated on the device, {cap >> 30} GB cap",
                "ms_per_pass": dt * 1e3, "value": vox / dt / 1e9, "unit": "Gvoxels/s",
                "histogram_kernel_ms": kms, "histogram_launches": kl,
                "histogram_gvox_s": vox / (kms * 1e-3) / 1e9 if kms > 0 else None,
                "histogram_hbm_frac": (vox * 2 / (kms * 1e-3) / 1e9) / peak if kms > 0 else None,
                "peak_source": peak_kind, "top_level_invariants": ok}
    except Exception as e:   # the optional leg must not cost the line
        return {"error": f"{type(e).__name__}: {e}"}


def run_reference(args):
    """--impl reference: the CPU oracle timed per step on a bounded sample."""
    import numpy as np
    import oracle
    from paper_2311_11740_gb300 import workloads
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    field, thr = workloads.config3(device="cpu") if args.small == 0 else workloads.config3(n=args.small)
    thr_np = thr.numpy()
    total_steps = args.steps + args.warmup
    budget = 150.0 / max(total_steps, 1)
    probe = np.ascontiguousarray(field[:2].numpy())
    t0 = time.perf_counter()
    oracle.ec_curves(probe, thr_np, L, 26, DESC)
    per_plane = (time.perf_counter() - t0) / 2
    planes = int(max(1, min(field.shape[0], budget / max(per_plane, 1e-6))))
    sample = np.ascontiguousarray(field[:planes].numpy())
    for _ in range(args.warmup):
        oracle.ec_curves(sample, thr_np, L, 26, DESC)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.ec_curves(sample, thr_np, L, 26, DESC)
    dt = time.perf_counter() - t0
    value = sample.size * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gvoxels/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{planes} z-planes of the 512^3 field per step"},
            "cpu_baseline": {"value": value, "unit": "Gvoxels/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"first {planes} z-planes ({sample.size} voxels) of the same field per step"},
            "e2e": {"value": value, "unit": "Gvoxels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--small", type=int, default=0, help="testing only: edge of a smaller cube")
    ap.add_argument("--batch-requests", type=int, default=4096)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-type-map", action="store_true")
    ap.add_argument("--profile-case", nargs="?", const="curve", choices=("curve", "typemap", "2d", "rows", "hashbox"),
                    help="run two curve requests (or two type maps) on the first 256 planes of the field, or "
                         "two 2D requests on the 16384^2 uint8 field (2d), and exit")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2311_11740_gb300 import ec, workloads

    if args.profile_case == "hashbox":
        for _ in range(2):
            slab = ec.gen_hashbox_u16(4, 0, 0, 0, 2048, 2048, 66, device=local)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "2048 x 2048 x 66 uint16 hash-box slab (seed 4)",
                          "value_at_origin": int(slab[0, 0, 0])}))
        return 0
    if args.profile_case == "2d":
        u8, _, _ = workloads.config2(device="cuda")
        ctx = ec.Context(local)
        desc2 = ec.EC_DESC_EC | ec.EC_DESC_PERIMETER | ec.EC_DESC_AREA
        for _ in range(2):
            res = ec.curve(u8, None, L=256, descriptors=desc2, ctx=ctx)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "16384^2 uint8 smoothed GRF, 256 levels, EC+perimeter+area",
                          "area_at_top": int(res[2, -1])}))
        return 0
    n = args.small or N
    field, thr = workloads.config3(device="cuda", n=n) if args.small else workloads.config3(device="cuda")
    if args.profile_case == "rows":
        slab = field[:256, :511, :511].contiguous()
        ctx = ec.Context(local)
        for _ in range(2):
            res = ec.curve(slab, thr, descriptors=DESC, ctx=ctx)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "256x511x511 float32 slab of the benchmark field (rows of 2044 bytes), "
                                          "EC+area+volume", "volume_at_top": int(res[2, -1])}))
        return 0
    if args.profile_case:
        slab = field[:256].contiguous()
        ctx = ec.Context(local)
        if args.profile_case == "typemap":
            for _ in range(2):
                res = ec.type_map(slab, thr, ctx=ctx)
            torch.cuda.synchronize()
            print(json.dumps({"profile_case": "256x512x512 float32 slab of the benchmark field, type map",
                              "full_vertices_at_top": int(res[21, -1])}))
            return 0
        for _ in range(2):
            res = ec.curve(slab, thr, descriptors=DESC, ctx=ctx)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "256x512x512 float32 slab of the benchmark field, EC+area+volume",
                          "volume_at_top": int(res[2, -1])}))
        return 0
    vox = field.numel()
    ctx = ec.Context(local)
    ctx.set_option(ec.EC_OPT_PROFILE, 1)
    out = torch.empty((3, L), dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ec.curve(field, thr, descriptors=DESC, out=out, ctx=ctx)
    torch.cuda.synchronize()
    ctx.profile_read()   # discard warm-up kernel times

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        ec.curve(field, thr, descriptors=DESC, out=out, ctx=ctx)
    stop.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    elapsed_ms = start.elapsed_time(stop)
    kernel_ms, kernel_launches = ctx.profile_read()
    if dist:
        t = torch.tensor([elapsed_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    ms_per_step = elapsed_ms / args.steps
    value = world * vox * args.steps / (elapsed_ms / 1e3) / 1e9

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if rank == 0 or world > 1:
        host = field.cpu().pin_memory()
        thr_h = thr.cpu().numpy()
        ec.curve_3d_stream(host, thresholds=thr_h, descriptors=DESC, ctx=ctx)     # warm-up
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            res = ec.curve_3d_stream(host, thresholds=thr_h, descriptors=DESC, ctx=ctx)
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        e2e = {"value": world * vox / e2e_s / 1e9, "unit": "Gvoxels/s",
               "h2d_bytes_per_step": int(host.numel() * 4 + thr_h.nbytes),
               "d2h_bytes_per_step": int(res.nbytes)}

    # the same step with all four descriptors (perimeter included)
    out_all = torch.empty((4, L), dtype=torch.int64, device="cuda")
    ec.curve(field, thr, descriptors=DESC_ALL, out=out_all, ctx=ctx)
    all_ms = time_device(lambda: ec.curve(field, thr, descriptors=DESC_ALL, out=out_all, ctx=ctx), 50)
    ctx.profile_read()
    file_stream = None if rank != 0 else file_stream_section(ec, ctx, field, thr, out.cpu().numpy())
    configs_2d = None if (args.no_batch or rank != 0) else configs_2d_section(ec, ctx,
                                                                               with_cpu=not args.no_cpu_baseline)
    type_map = None if (args.no_type_map or rank != 0) else type_map_section(
        ec, ctx, field, thr, 20, not args.no_cpu_baseline, args.cpu_budget)
    batched = None if (args.no_batch or rank != 0) else config5_section(ec, ctx, args.batch_requests,
                                                                         with_oracle=not args.no_cpu_baseline)
    frames = None if (args.no_batch or rank != 0) else realtime_frames_section(ec, ctx)
    streamed = None if (args.no_batch or rank != 0) else streamed_2048_section(ec, ctx)

    if rank != 0:
        return 0
    peak, peak_kind = measured_peaks()
    bytes_per_launch = vox * 4
    kernel_avg_s = kernel_ms / max(kernel_launches, 1) / 1e3
    achieved = bytes_per_launch / kernel_avg_s / 1e9
    traffic = traffic_per_launch()
    line = {
        "metric": METRIC, "value": value, "unit": "Gvoxels/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if not args.small else f"{n}^3 test cube", "field_bytes": vox * 4,
                   "l2": "inputs larger than L2 (537 MB field), no flush",
                   "per_step": "ec_curve_3d: memset + k_uniform_check + k_planar3d + k_scan"},
        "roofline": {"bound": "hbm", "kernel": KERNEL, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_kind, "traffic": traffic,
                     "kernel_avg_us": kernel_avg_s * 1e6, "algorithmic_bytes_per_launch": bytes_per_launch},
        "e2e": e2e,
        "gpu_launches": LAUNCHES_PER_STEP * args.steps,
        "clocks": clocks,
        "all_descriptors": {"descriptors": "EC+perimeter+area+volume", "ms_per_step": all_ms,
                            "value": vox / all_ms / 1e6, "unit": "Gvoxels/s"},
        "file_stream": file_stream,
        "config1": None if configs_2d is None else configs_2d.get("config1"),
        "config2": None if configs_2d is None else configs_2d.get("config2"),
        "type_map": type_map,
        "config5": batched,
        "realtime_frames": frames,
        "streamed_2048": streamed,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(field.cpu(), thr.cpu(), args.cpu_budget)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
