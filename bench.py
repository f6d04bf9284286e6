#!/usr/bin/env python
"""Benchmark: element Gram matrices per second on one GB300 (and N GPUs, weak scaling).

Workload ("seq_q5_8x8x8"): the full exact sequence in FP64 -- H1, H(curl), H(div) and L2
Gram matrices of 512 jittered trilinear hexahedra of an 8^3 unit-cube mesh (O(p^7)
sum-factorization path) and of the same 512 elements as sheared parallelepipeds (O(p^6)
affine path), test order q = 5, Gauss 7^3 points, per-element coefficient k_e in
[0.5, 2].  One step = the 8 calls (4 spaces x 2 maps) = 4096 element matrices, 4.56 GB
written.  Inputs are resident in HBM when a step starts; L2 is flushed (a 512 MiB
write) before every step, outside the timed events.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle (conventional
quadrature, the paper's Algorithms 1/4/6/8) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SPACES = ["H1", "HCURL", "HDIV", "L2"]
WORKLOAD = "seq_q5_8x8x8"
Q, L = 5, 7
METRIC = "element Gram matrices/s (H1+H(curl)+H(div)+L2, q=5, trilinear O(p^7) + affine O(p^6), FP64)"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant launch, the
# H(curl) general contraction of this workload, from one ncu capture of this script
# (command and figures in profiles/launches_seq_q5_8x8x8_fp64.md).  It is reported only
# while the source of that kernel (the text between the two markers below in
# dpg_kernels.cu) is the one the counters were taken on.
TRAFFIC = {"bytes": 127710976 + 1240180224,
           "kernel_sha256": "057a2fd106afd81cbdb9f51e9eea11cbd1d21527df77b94ab5490c2d35376ab1",
           "markers": ("// general sum factorization", "// FP32 general sum factorization")}


def dominant_traffic():
    import hashlib
    try:
        src = open(os.path.join(ROOT, "paper_1711_00984_gb300", "csrc", "dpg_kernels.cu")).read()
        a, b = src.index(TRAFFIC["markers"][0]), src.index(TRAFFIC["markers"][1])
    except (OSError, ValueError):
        return None
    return TRAFFIC["bytes"] if hashlib.sha256(src[a:b].encode()).hexdigest() == TRAFFIC["kernel_sha256"] else None
UNIT = "element matrices/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-form sub-measurement")
    ap.add_argument("--workload", default=None,
                    choices=sorted(SECONDARY) + ["hp_q2to8_16x16x16", "dpg_q6_p4_16x16x16"],
                    help="secondary workload record")
    ap.add_argument("--only", default=None, help="profiling case: run only this space's call (H1, HCURL, HDIV, L2)")
    ap.add_argument("--map", default="general", choices=["general", "affine"], help="map of the --only case")
    ap.add_argument("--elems", type=int, default=0,
                    help="elements of the --only case (default: all 512) or of the dpg_q6_p4_16x16x16 record")
    ap.add_argument("--fp32", action="store_true", help="FP32 form for the --only case")
    ap.add_argument("--condense", default="tc", choices=["tc", "fma"],
                    help="arithmetic of the condensation updates in the dpg_q6_p4_16x16x16 record")
    return ap.parse_args()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def workload_config():
    return {"workload": WORKLOAD + ": H1/H(curl)/H(div)/L2 Gram, q=5, L=7, 512 jittered trilinear "
                                   "+ 512 affine hexahedra per GPU, k_e~U[0.5,2]",
            "elements_per_step": 4096, "q": Q, "L": L,
            "l2": "flushed before every step (512 MiB write, outside the timed events)"}


# ---------------------------------------------------------------------------- oracle arm

def oracle_sample(n_per_call: int, offset: int = 0):
    """Time the oracle on n_per_call elements of every (space, map) of the workload."""
    import numpy as np
    import oracle
    from paper_1711_00984_gb300 import meshgen
    w = meshgen.workload(WORKLOAD)
    ne = w["verts"].shape[0]
    idx = (np.arange(n_per_call) * 37 + offset) % ne
    t0 = time.perf_counter()
    count = 0
    for verts in (w["verts"], w["verts_affine"]):
        for s in SPACES:
            c = meshgen.coeff_pairs(s, w["k"], ne)
            oracle.gram(s, Q, L, verts[idx], c[idx], nthreads=host_cores())
            count += len(idx)
    return count, time.perf_counter() - t0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = host_cores()
    n = max(1, cores)                           # one element per core per (space, map) call
    for i in range(args.warmup):
        oracle_sample(n, offset=i)
    tot_count, tot_t = 0, 0.0
    for i in range(args.steps):
        c, t = oracle_sample(n, offset=args.warmup + i)
        tot_count += c
        tot_t += t
    v = tot_count / tot_t
    sample = f"{n} elements x 8 (space, map) calls per step, seeded spread of the 512-element workload"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded meshgen)", "config": workload_config(),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- multi-rank host logic

def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest value of x over all ranks (the step time the whole job waited for); a
    no-op on one rank.  Any torch.distributed backend (NCCL on the GPUs, gloo on CPU)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank: int, seconds: float) -> float:
    """Whole-job rate of a weak-scaling step: every rank processes units_per_rank units, the
    job takes the slowest rank's time."""
    return world * units_per_rank / seconds


# ---------------------------------------------------------------------------- GPU arm

class ClockSampler:
    def __init__(self, index: int):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")
        self.index = index

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        import statistics
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1711_00984_gb300 as dpg
    from paper_1711_00984_gb300 import build as dbuild
    from paper_1711_00984_gb300 import meshgen

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        dbuild.build()
    if world > 1:
        dist.barrier()
    dpg.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    sh = int(stream.cuda_stream)

    w = meshgen.workload(WORKLOAD)
    ne = w["verts"].shape[0]
    tuned = {}
    for s in SPACES:
        dpg.dpg_tables_init_L(Q, L, s)
        # the library's autotuner picks each general-path program's stage-A chunk (set-up,
        # outside the timed region)
        tuned[s] = [dpg.dpg_autotune(Q, s, False, sh)] + ([] if args.no_fp32 else [dpg.dpg_autotune(Q, s, True, sh)])
    maps = [("general", torch.from_numpy(w["verts"]).to(dev), False),
            ("affine", torch.from_numpy(w["verts_affine"]).to(dev), True)]
    coeffs = {s: torch.from_numpy(meshgen.coeff_pairs(s, w["k"], ne)).to(dev) for s in SPACES}
    outs = {(m, s): torch.empty((ne,) + dpg.matrix_shape(s, Q), dtype=torch.float64, device=dev)
            for m, _, _ in maps for s in SPACES}
    out_bytes = sum(o.numel() * 8 for o in outs.values())
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def call(mname, v, aff, s):
        code = dpg.dpg_integrate(dpg.space_id(s, affine=aff), 0, Q, ne, v.data_ptr(), coeffs[s].data_ptr(),
                                 outs[(mname, s)].data_ptr(), sh)
        if code:
            raise dpg.DpgError(code, "dpg_integrate")

    dom_ev = []

    def step(record_dom=False):
        for mname, v, aff in maps:
            for s in SPACES:
                if record_dom and mname == "general" and s == "HCURL":
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    call(mname, v, aff, s)
                    b.record(stream)
                    dom_ev.append((a, b))
                else:
                    call(mname, v, aff, s)

    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    code, bad = dpg.dpg_sync_status(sh)
    if code:
        raise RuntimeError(f"device status {dpg.STATUS.get(code)} at element {bad}")

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            ev[i][0].record(stream)
            step(record_dom=True)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    dom_ms = float(np.mean([a.elapsed_time(b) for a, b in dom_ev]))
    total_ms = max_over_ranks(total_ms, world, dev)
    code, bad = dpg.dpg_sync_status(sh)
    if code:
        raise RuntimeError(f"device status {dpg.STATUS.get(code)} at element {bad}")

    elems_per_step = ne * len(SPACES) * len(maps)
    ms_per_step = total_ms / args.steps
    value = job_throughput(world, elems_per_step, ms_per_step * 1e-3)

    # ---- e2e through the host-buffer entry point (H2D + integrate + D2H per call)
    e2e = None
    if not args.no_e2e:
        hv = {m: v.cpu().pin_memory() for m, v, _ in maps}
        hc = {s: c.cpu().pin_memory() for s, c in coeffs.items()}
        ho = {k: torch.empty(o.shape, dtype=o.dtype).pin_memory() for k, o in outs.items()}

        def hstep():
            for mname, _, aff in maps:
                for s in SPACES:
                    code = dpg.dpg_integrate_host(dpg.space_id(s, affine=aff), 0, Q, ne, hv[mname].data_ptr(),
                                                  hc[s].data_ptr(), ho[(mname, s)].data_ptr(), sh)
                    if code:
                        raise dpg.DpgError(code, "dpg_integrate_host")
        hstep()
        ke = max(1, min(args.steps, 3))
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(ke):
            hstep()
        te = (time.perf_counter() - t0) / ke
        te = max_over_ranks(te, world, dev)
        in_bytes = sum(v.numel() * 8 for v in hv.values()) * len(SPACES) + sum(c.numel() * 8 for c in hc.values()) * 2
        e2e = {"value": job_throughput(world, elems_per_step, te), "unit": UNIT, "h2d_bytes_per_step": int(in_bytes),
               "d2h_bytes_per_step": int(out_bytes), "ms_per_step": 1e3 * te}

    # ---- roofline of the dominant kernel (H(curl) general: geometry + contraction launch pair)
    fpe = dpg.dpg_flops_per_element(dpg.space_id("HCURL"), 0, Q)
    peak64 = dpg.dpg_measure_fma_peak(64, sh)
    peak32 = dpg.dpg_measure_fma_peak(32, sh)
    peak_dmma = dpg.dpg_measure_fma_peak(65, sh)
    achieved = fpe * ne / (dom_ms * 1e-3)
    roof = {"bound": "alu", "kernel": "sf_general_kernel<double> (H(curl), with its geom_kernel launch)",
            "achieved": achieved / 1e12, "peak": peak64 / 1e12, "unit": "TFLOP/s",
            "frac": achieved / peak64, "traffic": dominant_traffic(),
            "traffic_unit": "bytes per launch (the contraction launch; its geom_kernel launch not included)",
            "peak_source": "FP64 FMA rate measured in this run by dpg_measure_fma_peak (MEASURED_PEAKS has no FP64 entry)",
            "flops_per_launch": fpe * ne, "launch_ms": dom_ms,
            "measured_alu_peaks_tflops": {"fp64_dfma": peak64 / 1e12, "fp32_ffma": peak32 / 1e12,
                                          "fp64_mma_m8n8k4": peak_dmma / 1e12}}

    # ---- the FP32 form on the same workload: time, speed-up, error against the FP64 result
    fp32 = None
    if not args.no_fp32:
        outs32 = {k: torch.empty(o.shape, dtype=torch.float32, device=dev) for k, o in outs.items()}

        def step32():
            for mname, v, aff in maps:
                for s_ in SPACES:
                    code = dpg.dpg_integrate(dpg.space_id(s_, fp32=True, affine=aff), 0, Q, ne, v.data_ptr(),
                                             coeffs[s_].data_ptr(), outs32[(mname, s_)].data_ptr(), sh)
                    if code:
                        raise dpg.DpgError(code, "dpg_integrate")
        for _ in range(args.warmup):
            flush.fill_(1)
            step32()
        ev32 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            ev32[i][0].record(stream)
            step32()
            ev32[i][1].record(stream)
        torch.cuda.synchronize()
        ms32 = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev32])), world, dev)
        errs = {}
        for k in outs:
            ref = outs[k]
            d = (outs32[k].double() - ref).flatten(1).norm(dim=1) / ref.flatten(1).norm(dim=1)
            errs[f"{k[1]}_{k[0]}"] = float(d.max())
        fp32 = {"ms_per_step": ms32, "value": job_throughput(world, elems_per_step, ms32 * 1e-3), "unit": UNIT,
                "speedup_vs_fp64": ms_per_step / ms32, "max_rel_frobenius_err_vs_fp64": max(errs.values()),
                "target_err": 1e-5, "err_per_call": errs}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        n = 4 * max(2, host_cores())             # about 10-30 s of oracle work
        cnt, t = oracle_sample(n)
        cpu = {"value": cnt / t, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
               "sample": f"{n} elements per (space, map) call x 8 calls = {cnt} element matrices, FP64"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded meshgen: jittered 8^3 mesh + sheared parallelepipeds)",
                "config": workload_config(), "output_gbs": world * out_bytes / (ms_per_step * 1e-3) / 1e9,
                "autotuned_nj": {s_: {"fp64": v_[0], **({"fp32": v_[1]} if len(v_) > 1 else {})}
                                 for s_, v_ in tuned.items()},
                "gpu_launches": 16 * args.steps, "clocks": clk.summary(), "roofline": roof,
                "cpu_baseline": cpu, "e2e": e2e, "fp32_form": fp32,
                "per_step_ms": {"min": min(step_ms), "max": max(step_ms)}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ultraweak acoustics (Sec. 3.3): the adjoint graph norm's diagonal blocks are H1 and H(div)
# Gram matrices with coefficients (omega^2 + alpha, 1) (Eq. 3.17); omega = 4 pi, alpha = 1
ACOUSTIC_OMEGA, ACOUSTIC_ALPHA = 4.0 * 3.141592653589793, 1.0
_AC = (ACOUSTIC_OMEGA ** 2 + ACOUSTIC_ALPHA, 1.0)

SECONDARY = {
    # name: (meshgen workload, q, L, [(space, p_trial, map, coefficients or None)]); map is
    # False (general), True (affine) or "extruded"
    "hcurl_q6_p4_16x16x16": ("hcurl_q6_p4_16x16x16", 6, 8, [("HCURL", 0, False, None), ("B", 4, False, None)]),
    "q9_8x8x4": ("q9_8x8x4", 9, 11, [("H1", 0, False, None), ("HDIV", 0, False, None),
                                     ("H1", 0, True, None), ("HDIV", 0, True, None)]),
    # the full element routine of the ultraweak acoustics formulation at the paper's
    # p0 = 4, p_r = 6 (Table 5) on the 16^3 jittered mesh: Gram blocks, cross block, stiffness
    "acoustics_q6_p4_16x16x16": ("hcurl_q6_p4_16x16x16", 6, 8,
                                 [("H1", 0, False, _AC), ("HDIV", 0, False, _AC),
                                  ("ACOUSTIC_CROSS", 0, False, None), ("ACOUSTIC_B", 4, False, None)]),
    # 512 elements extruded along x1 (Eq. 2.89, right): the O(p^6) extruded-map path
    # (Algorithm 11) and, on the same elements, the general O(p^7) path; unit coefficients
    "ext_q5_8x8x8": ("ext_q5_8x8x8", 5, 7, [(s_, 0, m_, None) for m_ in ("extruded", False)
                                            for s_ in ("H1", "HCURL", "HDIV", "L2")]),
}


def run_secondary(args):
    """Per-call FP64 and FP32 timings, rooflines and FP32 error of a secondary workload."""
    import numpy as np
    import torch
    import paper_1711_00984_gb300 as dpg
    from paper_1711_00984_gb300 import build as dbuild
    from paper_1711_00984_gb300 import meshgen
    dbuild.build()
    dpg.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    sh = int(stream.cuda_stream)
    wname, q, L, calls = SECONDARY[args.workload]
    w = meshgen.workload(wname)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    peak64 = dpg.dpg_measure_fma_peak(64, sh)
    peak32 = dpg.dpg_measure_fma_peak(32, sh)
    hbm = 6771.1e9
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] * 1e9
    except Exception:
        pass
    rec = {"workload": wname, "q": q, "L": L, "calls": []}
    tuned = {}
    for space, p, aff, cf in calls:
        ext = aff == "extruded"
        aff = aff is True
        dpg.dpg_tables_init_L(q, L, space)
        if space in SPACES and not aff and not ext and space not in tuned:
            tuned[space] = [dpg.dpg_autotune(q, space, False, sh), dpg.dpg_autotune(q, space, True, sh)]
        v = torch.from_numpy(w["verts_affine" if aff else "verts"]).to(dev)
        ne = v.shape[0]
        ct = None if cf is None else torch.tensor([list(cf)] * ne, dtype=torch.float64, device=dev)
        cptr = 0 if ct is None else ct.data_ptr()
        res = {"space": space, "p_trial": p, "map": "affine" if aff else ("extruded" if ext else "general"),
               "elements": ne}
        if cf is not None:
            res["coeffs"] = list(cf)
        outs = {}
        for fp32 in (False, True):
            sid = dpg.space_id(space, fp32=fp32, affine=aff, extruded=ext)
            shape = (ne,) + dpg.matrix_shape(space, q, p)
            out = torch.empty(shape, dtype=torch.float32 if fp32 else torch.float64, device=dev)

            def call():
                code = dpg.dpg_integrate(sid, p, q, ne, v.data_ptr(), cptr, out.data_ptr(), sh)
                if code:
                    raise dpg.DpgError(code, "dpg_integrate")
            for _ in range(args.warmup):
                call()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            for i in range(args.steps):
                flush.fill_(i & 0xff)
                ev[i][0].record(stream)
                call()
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            code, bad = dpg.dpg_sync_status(sh)
            assert code == 0, (code, bad)
            ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
            flops = dpg.dpg_flops_per_element(sid, p, q) * ne
            nbytes = out.numel() * out.element_size()
            t_alu = flops / (peak32 if fp32 else peak64)
            t_mem = nbytes / hbm
            key = "fp32" if fp32 else "fp64"
            res[key] = {"ms": ms, "element_matrices_per_s": ne / (ms * 1e-3), "output_gbs": nbytes / (ms * 1e-3) / 1e9,
                        "tflops": flops / (ms * 1e-3) / 1e12, "bound": "alu" if t_alu > t_mem else "hbm",
                        "roofline_frac": max(t_alu, t_mem) / (ms * 1e-3)}
            outs[key] = out
        errs = []
        for e0 in range(0, ne, 64):
            a = outs["fp32"][e0:e0 + 64].double()
            b = outs["fp64"][e0:e0 + 64]
            errs.append(((a - b).flatten(1).norm(dim=1) / b.flatten(1).norm(dim=1)).max().item())
        res["fp32_max_rel_frobenius_err_vs_fp64"] = max(errs)
        res["fp32_speedup"] = res["fp64"]["ms"] / res["fp32"]["ms"]
        rec["calls"].append(res)
        del outs
        torch.cuda.empty_cache()
    rec["measured_alu_peaks_tflops"] = {"fp64": peak64 / 1e12, "fp32": peak32 / 1e12}
    rec["autotuned_nj_fp64_fp32"] = tuned
    if args.workload.startswith("acoustics"):
        ne = rec["calls"][0]["elements"]
        tot64 = sum(c["fp64"]["ms"] for c in rec["calls"])
        tot32 = sum(c["fp32"]["ms"] for c in rec["calls"])
        rec["element_routine"] = {
            "calls": [c["space"] for c in rec["calls"]], "omega": ACOUSTIC_OMEGA, "alpha": ACOUSTIC_ALPHA,
            "fp64_ms": tot64, "fp32_ms": tot32, "fp64_s_per_element": tot64 * 1e-3 / ne,
            "fp32_s_per_element": tot32 * 1e-3 / ne,
            "paper_table5_context": {"p0": 4, "p_r": 6, "tensorization_s_per_element": 8.08e-2,
                                     "conventional_s_per_element": 1.900,
                                     "note": "G, B and l on the paper's CPU; here the G blocks, X and B (no load vector)"}}
        if not args.no_cpu:
            rec["element_routine"]["cpu_baseline"] = _acoustics_oracle_rate(w["verts"], q, L)
    print(json.dumps(rec), flush=True)


def _acoustics_oracle_rate(verts, q, L):
    """The oracle's rate for the same four calls on a bounded sample (2 elements)."""
    import numpy as np
    import oracle
    sample = np.ascontiguousarray(verts[:2])
    c = np.tile(np.array(_AC), (2, 1))
    t0 = time.perf_counter()
    oracle.gram("H1", q, L, sample, c)
    oracle.gram("HDIV", q, L, sample, c)
    oracle.acoustic_cross(q, L, sample)
    oracle.acoustic_b(q, 4, L, sample)
    dt = time.perf_counter() - t0
    return {"value": sample.shape[0] / dt, "unit": "element routines/s", "cores": len(os.sched_getaffinity(0)),
            "kind": "oracle", "sample": "2 elements of the workload, the four calls"}


def run_hp(args):
    """hp_q2to8_16x16x16: one dpg_integrate_hp call per space (graph-captured, replayed)."""
    import numpy as np
    import torch
    import paper_1711_00984_gb300 as dpg
    from paper_1711_00984_gb300 import build as dbuild
    from paper_1711_00984_gb300 import meshgen
    dbuild.build()
    dpg.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    sh = int(stream.cuda_stream)
    w = meshgen.workload("hp_q2to8_16x16x16")
    v = torch.from_numpy(w["verts"]).to(dev)
    qn = w["q_elem"].astype(np.int32)
    qt = torch.from_numpy(qn).to(dev)
    ne = len(qn)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    peak64 = dpg.dpg_measure_fma_peak(64, sh)
    peak32 = dpg.dpg_measure_fma_peak(32, sh)
    hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] * 1e9 if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6771.1e9
    rec = {"workload": "hp_q2to8_16x16x16", "elements": ne,
           "q_histogram": {int(q): int((qn == q).sum()) for q in range(2, 9)}, "calls": []}
    tuned = {}
    for space in SPACES:
        for q in range(2, 9):
            dpg.dpg_tables_init(q, space)
            tuned[f"{space}_q{q}"] = [dpg.dpg_autotune(q, space, False, sh), dpg.dpg_autotune(q, space, True, sh)]
        dims = np.array([dpg.dpg_matrix_rows(space, int(q)) for q in qn], dtype=np.int64)
        sizes = dims * dims
        off = np.zeros(ne, dtype=np.int64)
        off[1:] = np.cumsum(sizes)[:-1]
        offt = torch.from_numpy(off).to(dev)
        total = int(sizes.sum())
        flops = sum(int((qn == q).sum()) * dpg.dpg_flops_per_element(dpg.space_id(space), 0, q) for q in range(2, 9))
        res = {"space": space, "output_values": total}
        outs = {}
        for fp32 in (False, True):
            out = torch.empty(total, dtype=torch.float32 if fp32 else torch.float64, device=dev)
            sid = dpg.space_id(space, fp32=fp32)

            def call():
                code = dpg.dpg_integrate_hp(sid, ne, v.data_ptr(), 0, qt.data_ptr(), offt.data_ptr(), out.data_ptr(), sh)
                if code:
                    raise dpg.DpgError(code, "dpg_integrate_hp")
            for _ in range(args.warmup):
                call()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            for i in range(args.steps):
                flush.fill_(i & 0xff)
                ev[i][0].record(stream)
                call()
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            code, bad = dpg.dpg_sync_status(sh)
            assert code == 0, (code, bad)
            ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
            nbytes = out.numel() * out.element_size()
            t_alu = flops / (peak32 if fp32 else peak64)
            t_mem = nbytes / hbm
            res["fp32" if fp32 else "fp64"] = {
                "ms": ms, "element_matrices_per_s": ne / (ms * 1e-3), "output_gbs": nbytes / (ms * 1e-3) / 1e9,
                "tflops": flops / (ms * 1e-3) / 1e12, "bound": "alu" if t_alu > t_mem else "hbm",
                "roofline_frac": max(t_alu, t_mem) / (ms * 1e-3)}
            outs[fp32] = out
        err = 0.0
        for e0 in range(0, ne, 256):
            for e in range(e0, min(ne, e0 + 256), 37):
                a = outs[True][off[e]:off[e] + sizes[e]].double()
                b = outs[False][off[e]:off[e] + sizes[e]]
                err = max(err, float((a - b).norm() / b.norm()))
        res["fp32_max_rel_frobenius_err_vs_fp64_sampled"] = err
        res["fp32_speedup"] = res["fp64"]["ms"] / res["fp32"]["ms"]
        rec["calls"].append(res)
        del outs
        torch.cuda.empty_cache()
    rec["flops_note"] = "algorithmic flops of the FP64-order programs, summed over the elements' orders"
    rec["autotuned_nj_fp64_fp32"] = tuned
    print(json.dumps(rec), flush=True)


def condense_flops(n: int, mc: int) -> float:
    """Algorithmic flops of one condensation (2 per multiply-add): Cholesky n^3/6, the
    substitutions of mc right-hand sides mc n^2/2, the lower triangle of W^T W n mc(mc+1)/2."""
    return 2.0 * (n ** 3 / 6.0 + mc * n * n / 2.0 + n * mc * (mc + 1) / 2.0)


def run_dpg_chain(args):
    """The DPG element routine of the mixed-stiffness workload (Eqs. 3.7-3.8): Gram matrix G
    of H(curl) q = 6, enriched stiffness B (vector-L2 trial p = 4), load vector l (a
    degree-2 source), then the condensed K = B^T G^-1 B and F = B^T G^-1 l, per stage."""
    import numpy as np
    import torch
    import oracle
    import paper_1711_00984_gb300 as dpg
    from paper_1711_00984_gb300 import build as dbuild
    from paper_1711_00984_gb300 import meshgen
    dbuild.build()
    dpg.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    sh = int(stream.cuda_stream)
    q, p, L = 6, 4, 8
    w = meshgen.workload("hcurl_q6_p4_16x16x16")
    vn = np.ascontiguousarray(w["verts"][:args.elems] if args.elems > 0 else w["verts"])
    v = torch.from_numpy(vn).to(dev)
    ne = v.shape[0]
    src = np.random.default_rng(6).uniform(-1.0, 1.0, 30)
    ct = torch.from_numpy(src).to(dev)
    dpg.dpg_tables_init_L(q, L, "HCURL")
    dpg.dpg_tables_init_L(q, L, "B")
    tuned_hcurl = dpg.dpg_autotune(q, "HCURL", False, sh)
    dpg.dpg_condense_set_method(args.condense)
    n, m = dpg.dpg_matrix_rows("HCURL", q), dpg.dpg_matrix_cols("B", p, q)
    G = torch.empty((ne, n, n), dtype=torch.float64, device=dev)
    B = torch.empty((ne, n, m), dtype=torch.float64, device=dev)
    l = torch.empty((ne, n), dtype=torch.float64, device=dev)
    K = torch.empty((ne, m, m), dtype=torch.float64, device=dev)
    F = torch.empty((ne, m), dtype=torch.float64, device=dev)
    G0, B0, l0 = torch.empty_like(G), torch.empty_like(B), torch.empty_like(l)
    peak64 = dpg.dpg_measure_fma_peak(64, sh)
    stages = {
        "gram": lambda: dpg.integrate("HCURL", q, v, out=G0, stream=stream),
        "stiffness_b": lambda: dpg.integrate("B", q, v, p=p, out=B0, stream=stream),
        "load": lambda: dpg.integrate_load("HCURL", q, v, ct, out=l0, stream=stream),
        "condense": lambda: dpg.condense(G, B, l, K=K, F=F, stream=stream),
    }

    def refresh():                           # the condensation works in place on G, B, l
        G.copy_(G0); B.copy_(B0); l.copy_(l0)
    for f in ("gram", "stiffness_b", "load"):
        stages[f]()
    refresh()
    rec = {"workload": "dpg_q6_p4_16x16x16", "q": q, "p_trial": p, "L": L, "elements": ne, "n": n, "m": m,
           "autotuned_nj_hcurl_fp64": tuned_hcurl, "condense_method": args.condense, "stages": {}}
    steps = max(1, min(args.steps, 5))
    for name, fn in stages.items():
        for _ in range(max(1, min(args.warmup, 2))):
            if name == "condense":
                refresh()
            fn()
        ts = []
        for _ in range(steps):
            if name == "condense":
                refresh()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        code, bad = dpg.dpg_sync_status(sh)
        assert code == 0, (name, code, bad)
        rec["stages"][name] = {"ms": float(np.median(ts))}
    cf = condense_flops(n, m + 1) * ne
    cms = rec["stages"]["condense"]["ms"]
    cd = rec["stages"]["condense"]
    cd.update({"flops_per_element": cf / ne, "fp64_equivalent_tflops": cf / (cms * 1e-3) / 1e12})
    if args.condense == "fma":
        cd.update({"bound": "alu", "roofline_frac": cf / (cms * 1e-3) / peak64})
    else:
        # the O(n^3) part runs as BF16 digit products on the tensor cores: the FP64 FMA peak
        # is no longer its bound, only the yardstick of the FP64 work it stands for
        cd.update({"bound": "tensor digit products + FP64 panels",
                   "ratio_to_fp64_fma_peak": cf / (cms * 1e-3) / peak64})
    tot = sum(st["ms"] for st in rec["stages"].values())
    rec["element_routine_ms"] = tot
    rec["element_routines_per_s"] = ne / (tot * 1e-3)
    # the same routine through the one-call entry point (G, B, l in a library workspace)
    ts = []
    for i in range(1 + steps):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dpg.condensed_system(q, p, v, None, ct, K=K, F=F, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        if i:
            ts.append(a.elapsed_time(b))
    code, bad = dpg.dpg_sync_status(sh)
    assert code == 0, ("condensed_system", code, bad)
    rec["one_call"] = {"ms": float(np.median(ts)), "element_routines_per_s": ne / (float(np.median(ts)) * 1e-3),
                       "entry_point": "dpg_condensed_system"}
    rec["measured_fp64_fma_peak_tflops"] = peak64 / 1e12
    if args.no_cpu:
        print(json.dumps(rec), flush=True)
        return
    # the oracle's chain on a bounded sample: its rate and the agreement of K and F
    idx = [0, ne - 1]
    t0 = time.perf_counter()
    Go, _ = oracle.gram("HCURL", q, L, vn[idx])
    Bo, _ = oracle.mixed_b(q, p, L, vn[idx])
    lo, _ = oracle.load("HCURL", q, L, vn[idx], src)
    Ko, Fo, _ = oracle.condense(Go, Bo, lo)
    dt = time.perf_counter() - t0
    Kg, Fg = K[idx].cpu().numpy(), F[idx].cpu().numpy()
    rec["sample_rel_err"] = {"K": float(max(np.linalg.norm(Kg[i] - Ko[i]) / np.linalg.norm(Ko[i]) for i in range(2))),
                             "F": float(max(np.linalg.norm(Fg[i] - Fo[i]) / np.linalg.norm(Fo[i]) for i in range(2)))}
    rec["cpu_baseline"] = {"value": 2 / dt, "unit": "element routines/s", "cores": host_cores(), "kind": "oracle",
                           "sample": f"elements 0 and {ne - 1}: gram, mixed_b, load, condense"}
    print(json.dumps(rec), flush=True)


def run_case(args):
    """One (space, map, form) call of the workload on a subset of elements, for profilers."""
    import torch
    import paper_1711_00984_gb300 as dpg
    from paper_1711_00984_gb300 import build as dbuild
    from paper_1711_00984_gb300 import meshgen
    dbuild.build()
    dpg.load()
    torch.cuda.set_device(0)
    w = meshgen.workload(WORKLOAD)
    ne = args.elems or w["verts"].shape[0]
    aff = args.map == "affine"
    s = args.only
    dpg.dpg_tables_init_L(Q, L, s)
    v = torch.from_numpy(w["verts_affine" if aff else "verts"][:ne]).cuda()
    c = torch.from_numpy(meshgen.coeff_pairs(s, w["k"], w["verts"].shape[0])[:ne]).cuda()
    out = torch.empty((ne,) + dpg.matrix_shape(s, Q), dtype=torch.float32 if args.fp32 else torch.float64, device="cuda")
    for _ in range(args.warmup + args.steps):
        dpg.integrate(s, Q, v, c, affine=aff, fp32=args.fp32, out=out)
    code, bad = dpg.sync_status()
    assert code == 0, (code, bad)
    print(json.dumps({"profile_case": {"space": s, "map": args.map, "elems": ne, "fp32": args.fp32,
                                       "calls": args.warmup + args.steps}}))


def main():
    args = parse()
    if args.only:
        run_case(args)
    elif args.workload == "hp_q2to8_16x16x16":
        run_hp(args)
    elif args.workload == "dpg_q6_p4_16x16x16":
        run_dpg_chain(args)
    elif args.workload:
        run_secondary(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
