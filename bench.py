#!/usr/bin/env python
"""Benchmark: element matrices per second on one GB300 (and N GPUs, weak scaling).

Headline workload ("hp_q2to8_16x16x16"): the full exact sequence in FP64 on a jittered
16^3 trilinear mesh whose 4096 elements draw their test order q_e uniformly from
{2, ..., 8}: H1, H(curl), H(div) and L2 Gram matrices, one graph-captured persistent
launch per space (dpg_integrate_hp, output packed per element by an offset table).  One
step = the 4 calls = 16384 element matrices, 62.8 GB written.  Inputs are resident in HBM
when a step starts; L2 is flushed (a 512 MiB write) before every step, outside the timed
events (the outputs are far larger than L2 as well).

The same JSON line carries the rest of the metric ("element matrices/s and output GB/s vs
q per space; FP32-form vs FP64 speed-up at the stated error"):
  * fp32_form        : the headline step in the FP32 form, its speed-up and its error;
  * per_q            : the headline mesh split by order, one dpg_integrate call per (space,
                       q): element matrices/s, GB/s and roofline fraction per q per space,
                       both forms;
  * configs          : the 8^3 q = 5 workload (general O(p^7) and affine O(p^6) maps), the
                       16^3 H(curl) q = 6 Gram and mixed stiffness B (p = 4), the q = 9 H1 /
                       H(div) elements (general and affine): per call FP64 and FP32 times,
                       rooflines, FP32 error and speed-up, and a sampled oracle rate;
  * further_workloads: the extruded map (8^3, q = 5, every space, both forms), the
                       ultraweak acoustics element routine (16^3, q = 6, p = 4) and the DPG
                       element routine (G, B, l and the condensation K, F) on 912 elements of
                       the 16^3 H(curl) q = 6 / p = 4 mesh, with the condensation's other
                       digit route beside it and K, F against the oracle on two elements;
  * roofline         : the dominant kernel of the headline step against the FP64 FMA rate
                       measured in this run; rooflines elsewhere use the measured HBM copy
                       rate (MEASURED_PEAKS.json when present, else measured here), the
                       FP32 FMA rate and the tcgen05 TF32 rate (its third for 3xTF32 stages);
  * e2e              : the 8^3 q = 5 step through the host-buffer entry point
                       (dpg_integrate_host: host-to-device inputs, integration and
                       device-to-host output inside the timed region);
  * cpu_baseline     : the oracle (conventional quadrature) on a bounded sample of the
                       headline workload, on the host cores.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle (conventional
quadrature, the paper's Algorithms 1/4/6/8) on a bounded sample of the headline workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SPACES = ["H1", "HCURL", "HDIV", "L2"]
HEADLINE = "hp_q2to8_16x16x16"
HP_QS = list(range(2, 9))
METRIC = ("element Gram matrices/s (H1+H(curl)+H(div)+L2, 16^3 trilinear hexahedra with per-element "
          "q in {2..8}, L = q+2, one graph-captured persistent launch per space, FP64)")
UNIT = "element matrices/s"
# the 8^3 q = 5 workload (general + affine maps), its e2e record and the profiling case
WORKLOAD2, Q2, L2Q = "seq_q5_8x8x8", 5, 7

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the headline's
# dominant kernel (hp_contract_kernel<double>, the H(curl) call), from one ncu capture on the
# first 512 elements of the headline mesh scaled to the full launch by output bytes (command
# and figures under profiles/), reported only while the source of the kernel (the texts
# between the marker pairs below in dpg_kernels.cu) is the one the counters were taken on.
TRAFFIC = {"bytes": 36942101403, "kernel_sha256": "4f7badd1eec2a103122838fbb4c01331bf8a20e8733b71c9914e3fbc8dcf4a23",
           "markers": (("// general sum factorization", "// FP32 general sum factorization"),
                       ("// hp batching: elements of mixed order q", "// FMA-rate probe"))}


def kernel_source_hash():
    import hashlib
    try:
        src = open(os.path.join(ROOT, "paper_1711_00984_gb300", "csrc", "dpg_kernels.cu")).read()
        text = "".join(src[src.index(a):src.index(b)] for a, b in TRAFFIC["markers"])
    except (OSError, ValueError):
        return None
    return hashlib.sha256(text.encode()).hexdigest()


def dominant_traffic():
    if TRAFFIC["bytes"] is None:
        return None
    return TRAFFIC["bytes"] if kernel_source_hash() == TRAFFIC["kernel_sha256"] else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-form sub-measurements")
    ap.add_argument("--no-configs", action="store_true", help="headline only (no per-q sweep, no other configs)")
    ap.add_argument("--workload", default=None,
                    choices=sorted(SECONDARY) + ["hp_q2to8_16x16x16", "dpg_q6_p4_16x16x16"],
                    help="secondary workload record")
    ap.add_argument("--only", default=None, help="profiling case: run only this space's call (H1, HCURL, HDIV, L2)")
    ap.add_argument("--map", default="general", choices=["general", "affine", "extruded", "hp"],
                    help="map of the --only case (hp: the headline mesh through dpg_integrate_hp)")
    ap.add_argument("--elems", type=int, default=0,
                    help="elements of the --only case (default: all) or of the dpg_q6_p4_16x16x16 record")
    ap.add_argument("--fp32", action="store_true", help="FP32 form for the --only case")
    ap.add_argument("--condense", default="tcgen05", choices=["tcgen05", "tc", "fma"],
                    help="arithmetic of the condensation updates in the dpg_q6_p4_16x16x16 record")
    return ap.parse_args()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def workload_config():
    return {"workload": HEADLINE + ": H1/H(curl)/H(div)/L2 Gram matrices of a jittered 16^3 trilinear mesh, "
                                   "4096 elements per GPU per space, q_e ~ U{2..8} (seed 4), L_e = q_e + 2, "
                                   "unit coefficients, packed output (offset table)",
            "elements_per_step": 4 * 4096, "q": "2..8", "L": "q+2",
            "l2": "flushed before every step (512 MiB write, outside the timed events); outputs >> L2"}


# ---------------------------------------------------------------------------- oracle arm

def oracle_sample_hp(spaces, per_q: int, offset: int = 0):
    """Time the oracle on per_q elements of each order q = 2..8 of the headline mesh for
    each space in `spaces` (conventional quadrature with the element's own rule L = q + 2,
    OpenMP over the elements of a call on every host core)."""
    import numpy as np
    import oracle
    from paper_1711_00984_gb300 import meshgen
    w = meshgen.workload(HEADLINE)
    qe = w["q_elem"]
    count, t = 0, 0.0
    for s in spaces:
        for q in HP_QS:
            idx = np.flatnonzero(qe == q)
            pick = idx[(np.arange(per_q) * 97 + offset * 13) % len(idx)]
            t0 = time.perf_counter()
            oracle.gram(s, q, q + 2, w["verts"][pick], nthreads=host_cores())
            t += time.perf_counter() - t0
            count += len(pick)
    return count, t


def oracle_sample(n_per_call: int, offset: int = 0):
    """Time the oracle on n_per_call elements of every (space, map) of the 8^3 q = 5 workload."""
    import numpy as np
    import oracle
    from paper_1711_00984_gb300 import meshgen
    w = meshgen.workload(WORKLOAD2)
    ne = w["verts"].shape[0]
    idx = (np.arange(n_per_call) * 37 + offset) % ne
    t0 = time.perf_counter()
    count = 0
    for verts in (w["verts"], w["verts_affine"]):
        for s in SPACES:
            c = meshgen.coeff_pairs(s, w["k"], ne)
            oracle.gram(s, Q2, L2Q, verts[idx], c[idx], nthreads=host_cores())
            count += len(idx)
    return count, time.perf_counter() - t0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = host_cores()
    # one step = one space's elements at every order (cores elements per order, one
    # OpenMP call per order); the spaces rotate, so 4 consecutive steps cover the
    # headline step's mix (equal counts per space and per order)
    for i in range(args.warmup):
        oracle_sample_hp([SPACES[i % 4]], cores, offset=i)
    tot_count, tot_t = 0, 0.0
    for i in range(args.steps):
        c, t = oracle_sample_hp([SPACES[i % 4]], cores, offset=args.warmup + i)
        tot_count += c
        tot_t += t
    v = tot_count / tot_t
    sample = (f"step i: {cores} elements of each order q = 2..8 of the headline mesh (one OpenMP call per order "
              f"on {cores} threads) for space i mod 4 (H1, H(curl), H(div), L2), different elements every step")
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
    """nvidia-smi clock and throttle-reason samples (every 50 ms) while the block runs,
    written to a temporary file (removed afterwards)."""

    def __init__(self, index: int):
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="dpg_clocks_", suffix=".csv")
        os.close(fd)
        self.index = index
        self.rows = []

    def __enter__(self):
        try:
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
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    self.rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass

    def summary(self):
        import statistics
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measure_peaks(dpg, sh, dev):
    """Roofline denominators: FP64 / FP32 FMA, FP64 mma.sync and tcgen05 TF32 rates measured
    by the library's probes; the HBM copy rate from MEASURED_PEAKS.json, else measured
    here as a device-to-device copy of 2 GiB (read + write bytes, best of 10)."""
    import torch
    pk = {"fp64_dfma": dpg.dpg_measure_fma_peak(64, sh), "fp32_ffma": dpg.dpg_measure_fma_peak(32, sh),
          "fp64_mma_m8n8k4": dpg.dpg_measure_fma_peak(65, sh), "tf32_tcgen05": dpg.dpg_measure_fma_peak(19, sh)}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm = None
    if os.path.exists(path):
        try:
            hbm = float(json.load(open(path))["hbm_gbs"]) * 1e9
            pk["hbm_source"] = "MEASURED_PEAKS.json hbm_gbs"
        except Exception:
            hbm = None
    if hbm is None:
        a = torch.empty(1 << 31, dtype=torch.uint8, device=dev)
        b = torch.empty_like(a)
        a.fill_(1)
        stream = torch.cuda.current_stream()
        best = 0.0
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.copy_(a)
            e1.record(stream)
            torch.cuda.synchronize()
            best = max(best, 2 * a.numel() / (e0.elapsed_time(e1) * 1e-3))
        del a, b
        torch.cuda.empty_cache()
        hbm = best
        pk["hbm_source"] = "device-to-device copy of 2 GiB measured in this run (MEASURED_PEAKS.json absent)"
    pk["hbm"] = hbm
    return pk


def roof(flops, nbytes, ms, fp32, pk):
    """Roofline of one call: t_roof = max(flops / ALU peak, bytes / HBM); the ALU peak is the
    FP64 FMA rate (FP64 form) or the FP32 FMA rate (FP32 form: its FMA stages; its 3xTF32
    stages have the larger tcgen05 TF32 rate / 3)."""
    t_alu = flops / (pk["fp32_ffma"] if fp32 else pk["fp64_dfma"])
    t_mem = nbytes / pk["hbm"]
    return {"ms": ms, "tflops": flops / (ms * 1e-3) / 1e12, "output_gbs": nbytes / (ms * 1e-3) / 1e9,
            "bound": "alu" if t_alu > t_mem else "hbm", "roofline_frac": max(t_alu, t_mem) / (ms * 1e-3),
            "flops": flops, "bytes": nbytes}


def timed(fn, steps, warmup, flush, stream, median=True):
    """CUDA-event time of fn (ms): warm-up calls, then `steps` calls each after an L2 flush
    (outside the events); median (or mean) of the steps."""
    import numpy as np
    import torch
    for _ in range(warmup):
        fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(i & 0xff)
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    t = [a.elapsed_time(b) for a, b in ev]
    return float(np.median(t) if median else np.mean(t))


def rel_err_stats(a_list, b_list):
    """Max and median over elements of the relative Frobenius error of a against b."""
    import numpy as np
    errs = []
    for a, b in zip(a_list, b_list):
        errs.append(float((a.double() - b).norm() / b.norm()))
    return {"max": max(errs), "median": float(np.median(errs)), "elements": len(errs)}


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
    pk = measure_peaks(dpg, sh, dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    single = world == 1 and rank == 0

    # ---------------------------------------------------------------- headline: hp mesh
    w = meshgen.workload(HEADLINE)
    qn = w["q_elem"].astype(np.int32)
    ne = len(qn)
    v = torch.from_numpy(w["verts"]).to(dev)
    qt = torch.from_numpy(qn).to(dev)
    tuned = {}
    for s in SPACES:
        for q in HP_QS:
            dpg.dpg_tables_init(q, s)
            # the library's autotuner picks each program's stage-A chunk (set-up, untimed)
            tuned[f"{s}_q{q}"] = [dpg.dpg_autotune(q, s, False, sh)] + ([] if args.no_fp32 else
                                                                         [dpg.dpg_autotune(q, s, True, sh)])
    offs, sizes, offt, flops_hp = {}, {}, {}, {}
    for s in SPACES:
        dims = np.array([dpg.dpg_matrix_rows(s, int(q)) for q in qn], dtype=np.int64)
        sizes[s] = dims * dims
        off = np.zeros(ne, dtype=np.int64)
        off[1:] = np.cumsum(sizes[s])[:-1]
        offs[s] = off
        offt[s] = torch.from_numpy(off).to(dev)
        flops_hp[s] = sum(int((qn == q).sum()) * dpg.dpg_flops_per_element(dpg.space_id(s), 0, q) for q in HP_QS)
    out64 = {s: torch.empty(int(sizes[s].sum()), dtype=torch.float64, device=dev) for s in SPACES}
    out_bytes = sum(o.numel() * 8 for o in out64.values())

    def hp_call(s, out, fp32):
        code = dpg.dpg_integrate_hp(dpg.space_id(s, fp32=fp32), ne, v.data_ptr(), 0, qt.data_ptr(),
                                    offt[s].data_ptr(), out.data_ptr(), sh)
        if code:
            raise dpg.DpgError(code, "dpg_integrate_hp")

    dom_ev = []
    dom = "HCURL"

    def step(record_dom=False):
        for s in SPACES:
            if record_dom and s == dom:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                hp_call(s, out64[s], False)
                b.record(stream)
                dom_ev.append((a, b))
            else:
                hp_call(s, out64[s], False)

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
    total_ms = max_over_ranks(float(sum(step_ms)), world, dev)
    dom_ms = float(np.mean([a.elapsed_time(b) for a, b in dom_ev]))
    code, bad = dpg.dpg_sync_status(sh)
    if code:
        raise RuntimeError(f"device status {dpg.STATUS.get(code)} at element {bad}")
    elems_per_step = ne * len(SPACES)
    ms_per_step = total_ms / args.steps
    value = job_throughput(world, elems_per_step, ms_per_step * 1e-3)

    achieved = flops_hp[dom] / (dom_ms * 1e-3)
    roofline = {"bound": "alu", "kernel": "hp_contract_kernel<double> (H(curl) call, timed as its whole graph: "
                                          "work generation, geometry, persistent contraction)",
                "achieved": achieved / 1e12, "peak": pk["fp64_dfma"] / 1e12, "unit": "TFLOP/s",
                "frac": achieved / pk["fp64_dfma"], "traffic": dominant_traffic(),
                "traffic_unit": "DRAM bytes per launch of the contraction kernel",
                "peak_source": "FP64 FMA rate measured in this run by dpg_measure_fma_peak "
                               "(MEASURED_PEAKS.json has no FP64 entry)",
                "flops_per_launch": flops_hp[dom], "launch_ms": dom_ms,
                "measured_peaks": {"fp64_dfma_tflops": pk["fp64_dfma"] / 1e12, "fp32_ffma_tflops": pk["fp32_ffma"] / 1e12,
                                   "fp64_mma_m8n8k4_tflops": pk["fp64_mma_m8n8k4"] / 1e12,
                                   "tf32_tcgen05_tflops": pk["tf32_tcgen05"] / 1e12,
                                   "tf32_tcgen05_div3_tflops": pk["tf32_tcgen05"] / 3e12,
                                   "hbm_gbs": pk["hbm"] / 1e9, "hbm_source": pk["hbm_source"]}}
    hp_calls = {}
    for s in SPACES:
        hp_calls[s] = {"elements": ne, "output_gb": out64[s].numel() * 8 / 1e9}

    # ---- the headline step in the FP32 form: time, speed-up, error against the FP64 result
    fp32 = None
    if not args.no_fp32:
        out32 = {s: torch.empty(out64[s].numel(), dtype=torch.float32, device=dev) for s in SPACES}

        def step32():
            for s in SPACES:
                hp_call(s, out32[s], True)
        ms32 = max_over_ranks(timed(step32, args.steps, args.warmup, flush, stream, median=False), world, dev)
        code, bad = dpg.dpg_sync_status(sh)
        if code:
            raise RuntimeError(f"device status {dpg.STATUS.get(code)} at element {bad}")
        errs = {}
        sample = np.arange(0, ne, 17)
        for s in SPACES:
            a = [out32[s][offs[s][e]:offs[s][e] + sizes[s][e]] for e in sample]
            b = [out64[s][offs[s][e]:offs[s][e] + sizes[s][e]] for e in sample]
            errs[s] = rel_err_stats(a, b)
        fp32 = {"ms_per_step": ms32, "value": job_throughput(world, elems_per_step, ms32 * 1e-3), "unit": UNIT,
                "speedup_vs_fp64": ms_per_step / ms32, "target_err": 1e-5,
                "max_rel_frobenius_err_vs_fp64": max(e["max"] for e in errs.values()),
                "median_rel_frobenius_err_vs_fp64": float(np.median([e["median"] for e in errs.values()])),
                "err_per_space": errs, "err_sample": f"every 17th element ({len(sample)} per space)"}
        # per-space FP32 calls and their rooflines
        for s in SPACES:
            t = timed(lambda: hp_call(s, out32[s], True), min(args.steps, 5), 1, flush, stream)
            hp_calls[s]["fp32"] = roof(flops_hp[s], out32[s].numel() * 4, t, True, pk)
        del out32
    for s in SPACES:
        t = timed(lambda: hp_call(s, out64[s], False), min(args.steps, 5), 1, flush, stream)
        hp_calls[s]["fp64"] = roof(flops_hp[s], out64[s].numel() * 8, t, False, pk)
        if "fp32" in hp_calls[s]:
            hp_calls[s]["fp32_speedup"] = hp_calls[s]["fp64"]["ms"] / hp_calls[s]["fp32"]["ms"]
    del out64
    torch.cuda.empty_cache()

    # ---- end to end through the host-buffer entry point (the 8^3 q = 5 step), before the
    #      other records load the host
    e2e = None
    if not args.no_e2e:
        e2e = e2e_record(args, dpg, meshgen, world, dev, sh)
        torch.cuda.empty_cache()

    # ---- vs q: the headline mesh split by order, one dpg_integrate call per (space, q)
    per_q = None
    if single and not args.no_configs:
        per_q = {}
        for s in SPACES:
            rows = []
            for q in HP_QS:
                idx = np.flatnonzero(qn == q)
                vq = torch.from_numpy(np.ascontiguousarray(w["verts"][idx])).to(dev)
                nq = len(idx)
                n = dpg.dpg_matrix_rows(s, q)
                rec = {"q": q, "L": q + 2, "n": n, "elements": nq}
                outs = {}
                for f32 in ([False] if args.no_fp32 else [False, True]):
                    o = torch.empty((nq, n, n), dtype=torch.float32 if f32 else torch.float64, device=dev)
                    sid = dpg.space_id(s, fp32=f32)

                    def call():
                        code = dpg.dpg_integrate(sid, 0, q, nq, vq.data_ptr(), 0, o.data_ptr(), sh)
                        if code:
                            raise dpg.DpgError(code, "dpg_integrate")
                    t = timed(call, min(args.steps, 5), 1, flush, stream)
                    r = roof(dpg.dpg_flops_per_element(sid, 0, q) * nq, o.numel() * o.element_size(), t, f32, pk)
                    r["element_matrices_per_s"] = nq / (t * 1e-3)
                    rec["fp32" if f32 else "fp64"] = r
                    outs[f32] = o
                if True in outs:
                    rec["fp32_speedup"] = rec["fp64"]["ms"] / rec["fp32"]["ms"]
                    e = rel_err_stats(list(outs[True][::7]), list(outs[False][::7]))
                    rec["fp32_err_max"], rec["fp32_err_median"] = e["max"], e["median"]
                rows.append(rec)
                del outs
            per_q[s] = rows
        torch.cuda.empty_cache()
        code, bad = dpg.dpg_sync_status(sh)
        if code:
            raise RuntimeError(f"per-q sweep: device status {dpg.STATUS.get(code)} at element {bad}")

    # ---- the other configurations (rank 0 of a one-GPU run)
    configs = None
    if single and not args.no_configs:
        configs = {WORKLOAD2: config2_record(args, dpg, pk, flush, stream, sh, dev)}
        for name in ("hcurl_q6_p4_16x16x16", "q9_8x8x4"):
            configs[name] = secondary_record(args, name, dpg, pk, flush, stream, sh, dev)
            torch.cuda.empty_cache()

    # ---- the workloads past the Gram matrices (rank 0 of a one-GPU run): the extruded map,
    #      the ultraweak acoustics element routine, and the DPG element routine with the
    #      condensation on 912 elements of the 16^3 mesh (six waves of one CTA per SM)
    more = None
    if single and not args.no_configs:
        sub = argparse.Namespace(**vars(args))
        sub.steps, sub.warmup = min(args.steps, 5), min(args.warmup, 2)
        more = {}
        for name in ("ext_q5_8x8x8", "acoustics_q6_p4_16x16x16"):
            more[name] = secondary_full_record(sub, name, dpg, stream, sh, dev)
            torch.cuda.empty_cache()
        more["dpg_q6_p4_16x16x16"] = dpg_chain_record(sub, dpg, stream, sh, dev, 912)
        torch.cuda.empty_cache()
        code, bad = dpg.dpg_sync_status(sh)
        if code:
            raise RuntimeError(f"further workloads: device status {dpg.STATUS.get(code)} at element {bad}")

    cpu = None
    if single and not args.no_cpu:
        cnt, t = oracle_sample_hp(SPACES, host_cores())
        cpu = {"value": cnt / t, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
               "sample": f"{host_cores()} elements of each order q = 2..8 of the headline mesh for each space "
                         f"({cnt} element matrices; conventional FP64 quadrature, L = q+2, OpenMP over the "
                         f"elements of a call)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded meshgen: jittered 16^3 trilinear mesh, q_e ~ U{2..8})",
                "config": workload_config(), "output_gbs": world * out_bytes / (ms_per_step * 1e-3) / 1e9,
                "gpu_launches": 48 * args.steps, "clocks": clk.summary(), "roofline": roofline,
                "cpu_baseline": cpu, "e2e": e2e, "fp32_form": fp32, "hp_calls": hp_calls, "per_q": per_q,
                "configs": configs, "further_workloads": more, "autotuned_nj_fp64_fp32": tuned,
                "per_step_ms": {"min": min(step_ms), "max": max(step_ms)},
                "notes": {"gpu_launches": "12 library kernels per dpg_integrate_hp graph (work generation 10, "
                                          "geometry 1, persistent contraction 1) x 4 spaces per step",
                          "e2e": "covers the 8^3 q = 5 step (configs.seq_q5_8x8x8), not the headline mesh"}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def config2_record(args, dpg, pk, flush, stream, sh, dev):
    """The 8^3 q = 5 workload: 4 spaces x (general, affine) calls per step, FP64 and FP32."""
    import numpy as np
    import torch
    from paper_1711_00984_gb300 import meshgen
    w = meshgen.workload(WORKLOAD2)
    ne = w["verts"].shape[0]
    for s in SPACES:
        dpg.dpg_tables_init_L(Q2, L2Q, s)
        dpg.dpg_autotune(Q2, s, False, sh)
        if not args.no_fp32:
            dpg.dpg_autotune(Q2, s, True, sh)
    maps = [("general", torch.from_numpy(w["verts"]).to(dev), False),
            ("affine", torch.from_numpy(w["verts_affine"]).to(dev), True)]
    coeffs = {s: torch.from_numpy(meshgen.coeff_pairs(s, w["k"], ne)).to(dev) for s in SPACES}
    rec = {"workload": WORKLOAD2 + ": 512 jittered trilinear + 512 affine hexahedra, q = 5, L = 7, k_e ~ U[0.5,2]",
           "elements_per_step": 8 * ne, "calls": []}
    outs = {}
    tot = {False: 0.0, True: 0.0}
    for mname, vv, aff in maps:
        for s in SPACES:
            c = {"space": s, "map": mname, "elements": ne}
            for f32 in ([False] if args.no_fp32 else [False, True]):
                sid = dpg.space_id(s, fp32=f32, affine=aff)
                o = torch.empty((ne,) + dpg.matrix_shape(s, Q2), dtype=torch.float32 if f32 else torch.float64,
                                device=dev)

                def call():
                    code = dpg.dpg_integrate(sid, 0, Q2, ne, vv.data_ptr(), coeffs[s].data_ptr(), o.data_ptr(), sh)
                    if code:
                        raise dpg.DpgError(code, "dpg_integrate")
                t = timed(call, min(args.steps, 10), 2, flush, stream)
                r = roof(dpg.dpg_flops_per_element(sid, 0, Q2) * ne, o.numel() * o.element_size(), t, f32, pk)
                r["element_matrices_per_s"] = ne / (t * 1e-3)
                c["fp32" if f32 else "fp64"] = r
                tot[f32] += t
                outs[(mname, s, f32)] = o
            if not args.no_fp32:
                c["fp32_speedup"] = c["fp64"]["ms"] / c["fp32"]["ms"]
                e = rel_err_stats(list(outs[(mname, s, True)]), list(outs[(mname, s, False)]))
                c["fp32_err_max"], c["fp32_err_median"] = e["max"], e["median"]
                del outs[(mname, s, True)]
            del outs[(mname, s, False)]
            rec["calls"].append(c)
    code, bad = dpg.dpg_sync_status(sh)
    if code:
        raise RuntimeError(f"{WORKLOAD2}: device status {dpg.STATUS.get(code)} at element {bad}")
    rec["fp64_ms_per_step"] = tot[False]
    rec["element_matrices_per_s_fp64"] = 8 * ne / (tot[False] * 1e-3)
    if not args.no_fp32:
        rec["fp32_ms_per_step"] = tot[True]
        rec["fp32_speedup"] = tot[False] / tot[True]
    hc = [c for c in rec["calls"] if c["space"] == "HCURL" and c["map"] == "general"][0]["fp64"]
    rec["roofline"] = {"kernel": "sf_general_kernel<double> (H(curl), with its geom_kernel launch)",
                       "bound": "alu", "frac": hc["roofline_frac"], "achieved_tflops": hc["tflops"],
                       "peak_tflops": pk["fp64_dfma"] / 1e12, "flops_per_launch": hc["flops"], "launch_ms": hc["ms"]}
    for form in (["fp64"] if args.no_fp32 else ["fp64", "fp32"]):
        calls = [c[form] for c in rec["calls"] if c["map"] == "affine"]
        nbytes = sum(c["bytes"] for c in calls)
        ms = sum(c["ms"] for c in calls)
        roof_ms = sum(c["roofline_frac"] * c["ms"] for c in calls)     # sum of max(t_alu, t_mem)
        rec["affine_" + form] = {"bytes": nbytes, "ms": ms, "gbs": nbytes / (ms * 1e-3) / 1e9,
                                 "roofline_ms": roof_ms, "roofline_frac": roof_ms / ms,
                                 "hbm_only_frac": nbytes / (ms * 1e-3) / pk["hbm"],
                                 "note": "roofline: per call the slower of its FP64 (or FP32) FMA time for the "
                                         "algorithmic non-zero products and its output-write time, summed"}
    if not args.no_cpu:
        n = host_cores()
        cnt, t = oracle_sample(n)
        rec["cpu_baseline"] = {"value": cnt / t, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                               "sample": f"{n} elements per (space, map) call x 8 calls = {cnt} element matrices"}
    return rec


def secondary_record(args, name, dpg, pk, flush, stream, sh, dev):
    """One of the SECONDARY workloads as a record: per call FP64 and FP32 time, roofline,
    FP32 error (max and median) and speed-up, and the oracle's rate on a small sample."""
    import numpy as np
    import torch
    import oracle
    from paper_1711_00984_gb300 import meshgen
    wname, q, L, calls = SECONDARY[name]
    w = meshgen.workload(wname)
    rec = {"workload": wname, "q": q, "L": L, "calls": []}
    cpu_t, cpu_n = 0.0, 0
    for space, p, aff, cf in calls:
        aff = aff is True
        dpg.dpg_tables_init_L(q, L, space)
        if space in SPACES and not aff:
            dpg.dpg_autotune(q, space, False, sh)
            if not args.no_fp32:
                dpg.dpg_autotune(q, space, True, sh)
        vn = w["verts_affine" if aff else "verts"]
        vv = torch.from_numpy(vn).to(dev)
        ne = vv.shape[0]
        res = {"space": space, "p_trial": p, "map": "affine" if aff else "general", "elements": ne}
        outs = {}
        for f32 in ([False] if args.no_fp32 else [False, True]):
            sid = dpg.space_id(space, fp32=f32, affine=aff)
            o = torch.empty((ne,) + dpg.matrix_shape(space, q, p), dtype=torch.float32 if f32 else torch.float64,
                            device=dev)

            def call():
                code = dpg.dpg_integrate(sid, p, q, ne, vv.data_ptr(), 0, o.data_ptr(), sh)
                if code:
                    raise dpg.DpgError(code, "dpg_integrate")
            t = timed(call, min(args.steps, 5), 1, flush, stream)
            r = roof(dpg.dpg_flops_per_element(sid, p, q) * ne, o.numel() * o.element_size(), t, f32, pk)
            r["element_matrices_per_s"] = ne / (t * 1e-3)
            res["fp32" if f32 else "fp64"] = r
            outs[f32] = o
        code, bad = dpg.dpg_sync_status(sh)
        assert code == 0, (name, space, code, bad)
        if True in outs:
            res["fp32_speedup"] = res["fp64"]["ms"] / res["fp32"]["ms"]
            sample = list(range(0, ne, 9))
            e = rel_err_stats([outs[True][i] for i in sample], [outs[False][i] for i in sample])
            res["fp32_err_max"], res["fp32_err_median"] = e["max"], e["median"]
        if not args.no_cpu:
            pick = np.array([ne // 3])
            t0 = time.perf_counter()
            if space == "B":
                oracle.mixed_b(q, p, L, vn[pick], nthreads=host_cores())
            else:
                oracle.gram(space, q, L, vn[pick], nthreads=host_cores())
            cpu_t += time.perf_counter() - t0
            cpu_n += 1
        rec["calls"].append(res)
        del outs
        torch.cuda.empty_cache()
    if cpu_n:
        rec["cpu_baseline"] = {"value": cpu_n / cpu_t, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                               "sample": f"one element per call ({cpu_n} element matrices, sampled)"}
    return rec


def e2e_record(args, dpg, meshgen, world, dev, sh):
    """The 8^3 q = 5 step (4 spaces x 2 maps) through dpg_integrate_host: pinned host inputs
    and outputs, every copy inside the timed region."""
    import torch
    import torch.distributed as dist
    w = meshgen.workload(WORKLOAD2)
    ne = w["verts"].shape[0]
    for s in SPACES:
        dpg.dpg_tables_init_L(Q2, L2Q, s)
    hv = {"general": torch.from_numpy(w["verts"]).pin_memory(), "affine": torch.from_numpy(w["verts_affine"]).pin_memory()}
    hc = {s: torch.from_numpy(meshgen.coeff_pairs(s, w["k"], ne)).pin_memory() for s in SPACES}
    ho = {(m, s): torch.empty((ne,) + dpg.matrix_shape(s, Q2), dtype=torch.float64).pin_memory()
          for m in hv for s in SPACES}

    def hstep():
        for m in hv:
            for s in SPACES:
                code = dpg.dpg_integrate_host(dpg.space_id(s, affine=m == "affine"), 0, Q2, ne, hv[m].data_ptr(),
                                              hc[s].data_ptr(), ho[(m, s)].data_ptr(), sh)
                if code:
                    raise dpg.DpgError(code, "dpg_integrate_host")
    hstep()
    ke = max(1, min(args.steps, 3))
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        hstep()
    te = max_over_ranks((time.perf_counter() - t0) / ke, world, dev)
    in_bytes = sum(x.numel() * 8 for x in hv.values()) * len(SPACES) + sum(c.numel() * 8 for c in hc.values()) * 2
    out_bytes = sum(o.numel() * 8 for o in ho.values())
    return {"value": job_throughput(world, 8 * ne, te), "unit": UNIT, "h2d_bytes_per_step": int(in_bytes),
            "d2h_bytes_per_step": int(out_bytes), "ms_per_step": 1e3 * te,
            "workload": WORKLOAD2 + " (8 calls of 512 elements, q = 5, FP64): dpg_integrate_host, host buffers pinned"}


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
    import torch
    import paper_1711_00984_gb300 as dpg
    from paper_1711_00984_gb300 import build as dbuild
    dbuild.build()
    dpg.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    print(json.dumps(secondary_full_record(args, args.workload, dpg, stream, int(stream.cuda_stream), dev)), flush=True)


def secondary_full_record(args, name, dpg, stream, sh, dev):
    """The record of a named secondary workload (its calls in both forms; the acoustics
    workload also as its element routine)."""
    import numpy as np
    import torch
    from paper_1711_00984_gb300 import meshgen
    wname, q, L, calls = SECONDARY[name]
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
    if name.startswith("acoustics"):
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
    return rec


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
    """The DPG element routine of the mixed-stiffness workload, as its own record."""
    import torch
    import paper_1711_00984_gb300 as dpg
    from paper_1711_00984_gb300 import build as dbuild
    dbuild.build()
    dpg.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    print(json.dumps(dpg_chain_record(args, dpg, stream, int(stream.cuda_stream), dev, args.elems)), flush=True)


def dpg_chain_record(args, dpg, stream, sh, dev, elems):
    """The DPG element routine of the mixed-stiffness workload (Eqs. 3.7-3.8): Gram matrix G
    of H(curl) q = 6, enriched stiffness B (vector-L2 trial p = 4), load vector l (a
    degree-2 source), then the condensed K = B^T G^-1 B and F = B^T G^-1 l, per stage, on the
    first `elems` elements of the 16^3 mesh (all when 0)."""
    import numpy as np
    import torch
    import oracle
    from paper_1711_00984_gb300 import meshgen
    q, p, L = 6, 4, 8
    w = meshgen.workload("hcurl_q6_p4_16x16x16")
    vn = np.ascontiguousarray(w["verts"][:elems] if elems > 0 else w["verts"])
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
    # the other digit route (mma.sync) on the same inputs, for comparison
    other = "tc" if args.condense == "tcgen05" else ("tcgen05" if args.condense == "tc" else None)
    if other:
        dpg.dpg_condense_set_method(other)
        ts = []
        for i in range(2):
            refresh()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            stages["condense"]()
            b.record(stream)
            torch.cuda.synchronize()
            if i:
                ts.append(a.elapsed_time(b))
        dpg.dpg_condense_set_method(args.condense)
        refresh()
        cd["other_route"] = {"method": other, "ms": float(np.median(ts))}
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
        return rec
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
    return rec


def run_case(args):
    """One (space, map, form) call on a subset of elements, for profilers: the 8^3 q = 5
    workload (general, affine or extruded map) or, with --map hp, the first --elems
    elements of the headline mesh through dpg_integrate_hp."""
    import numpy as np
    import torch
    import paper_1711_00984_gb300 as dpg
    from paper_1711_00984_gb300 import build as dbuild
    from paper_1711_00984_gb300 import meshgen
    dbuild.build()
    dpg.load()
    torch.cuda.set_device(0)
    s = args.only
    if args.map == "hp":
        w = meshgen.workload(HEADLINE)
        ne = args.elems or w["verts"].shape[0]
        qn = np.ascontiguousarray(w["q_elem"][:ne].astype(np.int32))
        for q in sorted(set(qn.tolist())):
            dpg.dpg_tables_init(q, s)
        dims = np.array([dpg.dpg_matrix_rows(s, int(q)) for q in qn], dtype=np.int64)
        off = np.zeros(ne, dtype=np.int64)
        off[1:] = np.cumsum(dims * dims)[:-1]
        v = torch.from_numpy(np.ascontiguousarray(w["verts"][:ne])).cuda()
        qt, offt = torch.from_numpy(qn).cuda(), torch.from_numpy(off).cuda()
        out = torch.empty(int((dims * dims).sum()), dtype=torch.float32 if args.fp32 else torch.float64, device="cuda")
        sh = int(torch.cuda.current_stream().cuda_stream)
        for _ in range(args.warmup + args.steps):
            code = dpg.dpg_integrate_hp(dpg.space_id(s, fp32=args.fp32), ne, v.data_ptr(), 0, qt.data_ptr(),
                                        offt.data_ptr(), out.data_ptr(), sh)
            assert code == 0, code
    else:
        w = meshgen.workload("ext_q5_8x8x8" if args.map == "extruded" else WORKLOAD2)
        ne = args.elems or w["verts"].shape[0]
        aff = args.map == "affine"
        dpg.dpg_tables_init_L(Q2, L2Q, s)
        v = torch.from_numpy(w["verts_affine" if aff else "verts"][:ne]).cuda()
        c = torch.from_numpy(meshgen.coeff_pairs(s, w["k"], w["verts"].shape[0])[:ne]).cuda()
        out = torch.empty((ne,) + dpg.matrix_shape(s, Q2), dtype=torch.float32 if args.fp32 else torch.float64,
                          device="cuda")
        for _ in range(args.warmup + args.steps):
            dpg.integrate(s, Q2, v, c, affine=aff, extruded=args.map == "extruded", fp32=args.fp32, out=out)
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
