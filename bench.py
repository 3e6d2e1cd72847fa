#!/usr/bin/env python3
"""Throughput of the primal hybrid FEM path on one GB300 (or N replicas).

One step = the whole data-parallel path on one synthetic workload.  The
default is the jittered checkerboard (Kuhn 1^3 cube refined 6 levels =
17,915,904 tets, interior vertices moved by up to 0.2 h with seed 3,
a_K in {1, 1e4} on an 8^3 checkerboard, c = 1); the lognormal one (Kuhn 3^3
cube refined 4 levels = 3,359,232 tets, a_K = exp(N(0,1)) seed 2, c = 0.1) is
``--workload lognormal_3m``.  Both use f from u = sin(pi x) sin(pi y)
sin(pi z) and zero Dirichlet data.  The step:

    ph_mesh_create  face-to-tet connectivity, numbering, CSR pattern, geometry
    ph_assemble     local matrices + element condensation + CSR scatter
    ph_recover      element recovery from face multipliers (seeded Lambda)

The global solve is not part of the step (it is not data-parallel work of the
path and the metric counts assembled + condensed tets).  Inputs are resident
in HBM when timing starts; the e2e leg repeats the step through host (pinned)
buffers with the copies inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload, on every host core.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import meshgen  # noqa: E402

METRIC = "tets assembled+condensed/s"
UNIT = "tets/s"
WORKLOAD = "jitter_checker_18m"
# (Kuhn m, refinement levels) of each workload; lognormal_1m is a smaller case
# of the lognormal recipe (995,328 tets, working set above L2) for profiler
# captures
WORKLOADS = {"jitter_checker_18m": (1, 6), "lognormal_3m": (3, 4), "lognormal_1m": (2, 4)}
L2_BYTES = 129 * 2 ** 20
HBM_PEAK_FALLBACK = 6800.0
# FP64 peak derived from the recipe's nominal 1.25 TFLOP/s, 152 SMs and the
# 2070 MHz maximum SM clock: 2 FP64 instructions (DFMA, DADD or DMUL) per SM
# per clock -> 152 * 2 * 2.07e9 = 629.3e9 FP64 operations/s.  Context only:
# the roofline takes the peak measured by ph_fp64_peak in the same run.
FP64_PEAK_DERIVED_GOPS = 152 * 2 * 2.070
# DFMA iterations per thread of one ph_fp64_peak launch (tens of ms)
FP64_PEAK_ITERS = 4000
# FP64 operations per element in k_assemble's formulas (each fma, add, mul or
# div counted once): condensation kernel Qf 56, load and right-hand side 30,
# condensed entries 24 (d_k (Q_km d_m + e_m) for the 10 entries, e_m = d_m/(c|T|)).
ASSEMBLE_OPS_PER_TET = 110
# Method-level bytes per element of the numeric phase: coordinates, f and
# H counted once (136 + 24 nC/nE + 24 nF/nE).
def assemble_bytes_per_tet(nE, nC, nF):
    return 136.0 + 24.0 * nC / nE + 24.0 * nF / nE


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except OSError:
        return {}


# end-to-end leg: steps in flight at once (host threads, one stream each)
E_INFLIGHT = 2
# kernels timed with the library's CUDA events inside the timed region
TIMED_KERNELS = ("k_assemble", "zero_values", "k_recover_factored")
# mesh-build kernels, timed in a separate short loop (their timers add host
# work between the build's launches)
BUILD_KERNELS = ("k_face_count", "k_face_fill", "k_face_match", "k_face_emit", "k_row_fill", "k_scan")


def sources_sha256(sources):
    """sha256 over the named files of the library's csrc/, in order: the key
    a profile summary carries, so that its figures are used only while the
    kernels they were taken on are unchanged."""
    h = hashlib.sha256()
    for name in sources:
        with open(os.path.join(ROOT, "paper_2509_11133_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profile_kv(name):
    """key: value lines of a committed profile summary, or {} when it is
    missing or the sources it names changed after the counters were taken."""
    prof = os.path.join(ROOT, "profiles", name)
    try:
        kv = {}
        for line in open(prof):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    except OSError:
        return {}
    if kv.get("sources_sha256") != sources_sha256(kv.get("sources", "").split()):
        return {}
    return kv


def profile_figures(kernel="k_assemble"):
    """Per-element figures of the committed ncu capture of a kernel (taken
    on a smaller mesh of the lognormal recipe; the kernel's work and traffic
    per element do not depend on the mesh size): DRAM bytes and FP64
    instructions per element.  Empty when the kernel's sources changed after
    the counters were taken."""
    kv = profile_kv(f"{kernel}_lognormal_1m.txt")
    out = {}
    for key in ("dram_bytes_per_tet", "fp64_inst_per_tet", "fp32_inst_per_tet"):
        try:
            out[key] = float(kv[key])
        except (KeyError, ValueError):
            pass
    return out


def step_fp64_counts():
    """FP64 instructions per element of every kernel of the step (ncu's
    DFMA + DMUL + DADD counters of one build, assembly and recovery on the
    995,328-tet lognormal mesh, divided by its element count), or {} when
    the capture does not match the sources."""
    kv = profile_kv("fp64_step_lognormal_1m.txt")
    out = {}
    for k, v in kv.items():
        if k.startswith("fp64_per_tet "):
            out[k.split(" ", 1)[1]] = float(v)
    return out


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.12)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# ranks
# ---------------------------------------------------------------------------
def max_over_ranks(values, world, device):
    """Element-wise maximum of per-rank timings (all ranks get the result)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_rate(units_per_rank, world, ms):
    """Units processed by all ranks per second, timed by the slowest rank."""
    return world * units_per_rank / (ms * 1e-3)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def host_cores():
    """Host cores this process may run on (the box's, or its allotment)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def make_problem(name):
    if name in ("jitter_checker_18m", "lognormal_3m"):
        return meshgen.problem(name)
    m, k = WORKLOADS[name]
    coord, tet = meshgen.kuhn_cube(m)
    coord, tet, _ = meshgen.refined(coord, tet, k)
    return meshgen.Problem(name, coord, tet, meshgen.lognormal_field(tet.shape[0], 2), 0.1,
                           lambda x: meshgen.sin_source(x, 1.0, 1.0), info={"m": m, "k": k, "seed": 2})


def gpu_arm(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import paper_2509_11133_gb300 as ph
    from paper_2509_11133_gb300 import build as phbuild

    if not os.path.exists(phbuild.LIB):
        phbuild.build()
    ph.load()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()

    t0 = time.time()
    p = make_problem(args.workload)
    gen_s = time.time() - t0
    coord_h = torch.from_numpy(np.ascontiguousarray(p.coord)).pin_memory()
    tet_h = torch.from_numpy(np.ascontiguousarray(p.tet)).pin_memory()
    a_h = torch.from_numpy(np.ascontiguousarray(p.a)).pin_memory()
    coord_d, tet_d, a_d = coord_h.to(dev), tet_h.to(dev), a_h.to(dev)

    # counts and face centroids from the host arrays alone (the query a
    # host-only caller makes), face data at the centroids (input
    # preparation, untimed)
    info, cen = ph.ph_host_mesh_query(coord_h, tet_h)
    cen = cen.numpy()
    f_h = torch.from_numpy(np.asarray(p.f(cen), np.float64)).pin_memory()
    lam_h = torch.from_numpy(np.random.default_rng(7).standard_normal(info["L"])).pin_memory()
    f_d, lam_d = f_h.to(dev), lam_h.to(dev)
    nE, nF, L, nnz = info["nE"], info["nF"], info["L"], info["nnz"]
    values = torch.empty(nnz, dtype=torch.float64, device=dev)
    rhs = torch.empty(L, dtype=torch.float64, device=dev)
    u = torch.empty((nE, 4), dtype=torch.float64, device=dev)
    factor = torch.empty((nE, 10), dtype=torch.float64, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        m = ph.Mesh(coord_d, tet_d)
        if ev is not None:
            ev[1].record(stream)
        m.assemble(a_d, p.c, f_d, values=values, rhs=rhs, factor=factor)
        if ev is not None:
            ev[2].record(stream)
        m.recover_factored(factor, p.c, f_d, lam_d, u=u)
        if ev is not None:
            ev[3].record(stream)
        m.close()

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    n_launch0 = ph.ph_launch_count()
    for name in TIMED_KERNELS:
        ph.ph_kernel_time(name, reset=True)
    ph.ph_timing_enable(True)      # CUDA events around each element-kernel launch, on its stream
    for i in range(args.steps):
        step(evs[i])
        flush.zero_()          # L2 flush between timed steps (outside the event pairs)
    torch.cuda.synchronize()
    ph.ph_timing_enable(False)
    n_launch = ph.ph_launch_count() - n_launch0
    kern = {}
    for name in TIMED_KERNELS:
        ms, n = ph.ph_kernel_time(name, reset=True)
        kern[name] = ms / n if n else float("nan")
    # breakdown of the mesh build: a few more steps with its kernels timed
    # (not part of the headline timing)
    for name in BUILD_KERNELS:
        ph.ph_kernel_time(name, reset=True)
    ph.ph_timing_enable(2)
    for _ in range(5):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    ph.ph_timing_enable(False)
    build_kern = {}
    for name in BUILD_KERNELS:
        ms, n = ph.ph_kernel_time(name, reset=True)
        build_kern[name] = ms / 5 if n else float("nan")  # per build (k_scan: all scans of one build)
    # the precision variant: the same step with the element geometry, the face
    # areas and the condensation kernel in double-word arithmetic
    # (ph_mesh_create_dw + ph_assemble_dw), its own timed loop
    variant = None
    if not args.no_variant:
        def step_dw(ev=None):
            if ev is not None:
                ev[0].record(stream)
            m = ph.Mesh(coord_d, tet_d, geometry="dw")
            if ev is not None:
                ev[2].record(stream)
            m.assemble(a_d, p.c, f_d, values=values, rhs=rhs, factor=factor, variant="dw")
            if ev is not None:
                ev[3].record(stream)
            m.recover_factored(factor, p.c, f_d, lam_d, u=u, variant="dw")
            if ev is not None:
                ev[1].record(stream)
            m.close()

        for _ in range(args.warmup):
            step_dw()
            flush.zero_()
        torch.cuda.synchronize()
        evd = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
        ph.ph_kernel_time("k_assemble_dw", reset=True)
        ph.ph_kernel_time("k_recover_factored_dw", reset=True)
        ph.ph_timing_enable(True)
        for i in range(args.steps):
            step_dw(evd[i])
            flush.zero_()
        torch.cuda.synchronize()
        ph.ph_timing_enable(False)
        ms, n = ph.ph_kernel_time("k_assemble_dw", reset=True)
        rms, rn = ph.ph_kernel_time("k_recover_factored_dw", reset=True)
        # the double-word mesh build's kernels, in a short loop of their own
        for name in BUILD_KERNELS:
            ph.ph_kernel_time(name, reset=True)
        ph.ph_timing_enable(2)
        for _ in range(5):
            step_dw()
            flush.zero_()
        torch.cuda.synchronize()
        ph.ph_timing_enable(False)
        build_dw = {}
        for name in BUILD_KERNELS:
            bms, bn = ph.ph_kernel_time(name, reset=True)
            build_dw[name] = bms / 5 if bn else float("nan")
        variant = {"step_ms": float(np.mean([e[0].elapsed_time(e[1]) for e in evd])),
                   "mesh_build_kernels_ms": build_dw,
                   "phases_ms": {"mesh_create_dw": float(np.mean([e[0].elapsed_time(e[2]) for e in evd])),
                                 "assemble_dw": float(np.mean([e[2].elapsed_time(e[3]) for e in evd])),
                                 "recover_dw": float(np.mean([e[3].elapsed_time(e[1]) for e in evd]))},
                   "k_assemble_dw_ms": ms / n if n else float("nan"),
                   "k_recover_factored_dw_ms": rms / rn if rn else float("nan")}
    # the FP64 pipe's throughput on this GPU, measured now, under the same
    # clock sampling as the timed steps: best of 3 probe launches
    ph.ph_fp64_peak(FP64_PEAK_ITERS)
    peak_runs = [ph.ph_fp64_peak(FP64_PEAK_ITERS) for _ in range(3)]
    fp64_peak_gops = max(r[0] for r in peak_runs) / 1e9
    barrier()
    clk = clocks.stop()
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    create_ms = [e[0].elapsed_time(e[1]) for e in evs]
    asm_ms = [e[1].elapsed_time(e[2]) for e in evs]
    rec_ms = [e[2].elapsed_time(e[3]) for e in evs]
    ms_per_step = float(np.mean(step_ms))

    # e2e: host (pinned) inputs -> one C-ABI call per step (ph_assemble_host)
    # -> host outputs, every step's copies inside the timed region.  The host
    # link (~0.2 TB/s each way) binds one call, so E_INFLIGHT host threads run
    # steps concurrently, each on its own stream and output buffers: one
    # step's download overlaps the next one's upload and kernels.  Timed with
    # the host clock from the first call to the last return.
    def out_buffers():
        return {"rowptr": torch.empty(L + 1, dtype=torch.int32).pin_memory(),
                "colind": torch.empty(nnz, dtype=torch.int32).pin_memory(),
                "values": torch.empty(nnz, dtype=torch.float64).pin_memory(),
                "rhs": torch.empty(L, dtype=torch.float64).pin_memory(),
                "u": torch.empty((nE, 4), dtype=torch.float64).pin_memory()}

    def step_e2e(out, s):
        ph.ph_assemble_host(coord_h, tet_h, a_h, p.c, f_h, (nF, L, nnz), lam=lam_h, out=out, stream=s)

    def run_e2e(n_steps, inflight):
        outs = [out_buffers() for _ in range(inflight)]
        streams = [torch.cuda.Stream(device=dev) for _ in range(inflight)]
        errors = []

        def worker(w):
            try:
                torch.cuda.set_device(dev)
                for _ in range(w, n_steps, inflight):
                    step_e2e(outs[w], streams[w])
            except Exception as exc:  # reported after the join
                errors.append(exc)

        torch.cuda.synchronize()
        t0 = time.perf_counter()
        threads = [threading.Thread(target=worker, args=(w,)) for w in range(inflight)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        t1 = time.perf_counter()
        if errors:
            raise errors[0]
        return (t1 - t0) * 1e3 / n_steps

    h2d = 24 * p.nC + 16 * nE + 8 * nE + 8 * nF + 8 * L
    d2h = 4 * (L + 1) + 4 * nnz + 8 * nnz + 8 * L + 32 * nE
    e2e_ms = e2e_serial_ms = float("nan")
    if not args.no_e2e:
        e2e_steps = max(6, args.steps // 2)
        run_e2e(max(2, args.warmup), E_INFLIGHT)  # warm-up (pinned buffers, pool, streams)
        barrier()
        e2e_serial_ms = run_e2e(e2e_steps, 1)
        barrier()
        e2e_ms = run_e2e(e2e_steps, E_INFLIGHT)
        barrier()

    # max over ranks
    ms_per_step, e2e_ms, e2e_serial_ms, asm_max, k_asm = max_over_ranks(
        [ms_per_step, e2e_ms, e2e_serial_ms, float(np.mean(asm_ms)), kern["k_assemble"]], world, dev)
    # the lowest FP64 peak over the ranks
    fp64_peak_gops = -max_over_ranks([-fp64_peak_gops], world, dev)[0]

    if rank != 0:
        return None
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", HBM_PEAK_FALLBACK))
    asm_s = k_asm * 1e-3          # one k_assemble launch, CUDA events on its stream
    prof = profile_figures()
    if "fp64_inst_per_tet" in prof:
        ops_per_tet, ops_source = prof["fp64_inst_per_tet"], "ncu FP64 instructions (DFMA+DADD+DMUL) per element"
    else:
        ops_per_tet, ops_source = ASSEMBLE_OPS_PER_TET, "formula count (no capture of the current sources)"
    achieved_gops = ops_per_tet * nE / asm_s / 1e9
    traffic = prof["dram_bytes_per_tet"] * nE if "dram_bytes_per_tet" in prof else None
    bpt = assemble_bytes_per_tet(nE, p.nC, nF)
    value = whole_job_rate(nE, world, ms_per_step)
    cfg = workload_config(args.workload, p, world)
    if (cfg["nF"], cfg["L"], cfg["nnz"]) != (nF, L, nnz):
        raise RuntimeError(f"mesh counts {nF, L, nnz} differ from the closed forms {cfg['nF'], cfg['L'], cfg['nnz']}")
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": cfg,
        "phases_ms": {"mesh_create": float(np.mean(create_ms)), "assemble": float(np.mean(asm_ms)),
                      "recover": float(np.mean(rec_ms))},
        "kernels_ms": kern,
        "mesh_build_kernels_ms": build_kern,
        "roofline": {
            "kernel": "k_assemble (average launch over the timed steps, CUDA events on its stream)",
            "bound": "alu",
            "achieved": achieved_gops,
            "peak": fp64_peak_gops,
            "unit": "G FP64-op/s",
            "frac": achieved_gops / fp64_peak_gops,
            "traffic": traffic,
            "ops_per_tet": ops_per_tet,
            "ops_source": ops_source,
            "peak_source": "measured in this run: ph_fp64_peak (16 independent DFMA chains per thread, 8 x 256 "
                           "threads per SM, CUDA events), best of 3, during the clock sampling",
            "peak_runs_gops": [r[0] / 1e9 for r in peak_runs],
            "peak_derived_gops": FP64_PEAK_DERIVED_GOPS,
        },
        "roofline_hbm": {
            "achieved": bpt * nE / asm_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
            "frac": bpt * nE / asm_s / 1e9 / hbm_peak, "bytes_per_tet": bpt,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback",
        },
        "roofline_step": step_roofline(nE, ms_per_step, fp64_peak_gops),
        "e2e": None if args.no_e2e else {"value": whole_job_rate(nE, world, e2e_ms), "unit": UNIT,
                                         "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                                         "api": "ph_assemble_host (pinned host buffers, one call per step)",
                                         "in_flight": E_INFLIGHT, "timing": "host clock over all steps",
                                         "one_in_flight": {"value": whole_job_rate(nE, world, e2e_serial_ms),
                                                           "ms_per_step": e2e_serial_ms}},
        "gpu_launches": int(n_launch),
        "gpu_launches_per_step": n_launch / args.steps,
        "clocks": clk,
        "setup": {"host_mesh_generation_s": gen_s},
    }
    if variant is not None:
        line["variant_dw"] = variant_report(variant, nE, p.nC, nF, world, fp64_peak_gops, hbm_peak, ms_per_step,
                                            k_asm)
    if not args.no_extras:
        line["batched"] = batched_section(ph, dev, steps=max(3, args.steps // 10), warmup=3)
        line["adjoint"] = adjoint_section(ph, dev)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, args.workload, budget_s=args.cpu_budget)
    return line


def step_roofline(nE, step_ms, fp64_peak_gops):
    """The whole step against the FP64 pipe: every FP64 instruction of the
    step's kernels (per-element counts from the committed ncu capture) over
    the step's time; null when the capture does not match the sources."""
    counts = step_fp64_counts()
    if not counts:
        return None
    per_tet = sum(counts.values())
    g = per_tet * nE / (step_ms * 1e-3) / 1e9
    return {"what": "all FP64 instructions of one step (mesh build, assembly, recovery) over the step time",
            "bound": "alu", "achieved": g, "peak": fp64_peak_gops, "unit": "G FP64-op/s",
            "frac": g / fp64_peak_gops, "fp64_inst_per_tet": per_tet, "per_kernel": counts,
            "ops_source": "ncu FP64 instructions (DFMA+DADD+DMUL), profiles/fp64_step_lognormal_1m.txt"}


def variant_report(v, nE, nC, nF, world, fp64_peak_gops, hbm_peak, f64_step_ms, f64_k_asm_ms):
    """The precision variant's line: the step with ph_assemble_dw and its
    condensation kernel against the FP64 and HBM rooflines (per-element
    instruction and traffic figures from the kernel's committed ncu capture
    when it matches the sources)."""
    k_s = v["k_assemble_dw_ms"] * 1e-3
    prof = profile_figures("k_assemble_dw")
    bpt = assemble_bytes_per_tet(nE, nC, nF)
    out = {
        "what": "ph_mesh_create_dw + ph_assemble_dw + ph_recover_factored_dw: the element geometry (G_e, "
                "G_e T0^-1), the condensation kernel (the 3x3 algebra of A^-1) and the recovery's product "
                "(Qf/9) z' in double-word arithmetic (float pairs, ~48 bits) on the FP32 pipe; edge vectors, "
                "|det E|, face areas, the leading term d d'/(c|T|), every sum of H and rhs and the recovery's "
                "z' terms in fp64; flat or reaction-dominated elements take the fp64 kernel; tested against the "
                "oracle at the fp64 path's bars",
        "dtype": "f64 + f32x2 (double-word) geometry and condensation kernel",
        "value": whole_job_rate(nE, world, v["step_ms"]), "unit": UNIT, "ms_per_step": v["step_ms"],
        "phases_ms": v["phases_ms"], "mesh_build_kernels_ms": v["mesh_build_kernels_ms"],
        "speedup_step_vs_f64": f64_step_ms / v["step_ms"],
        "k_assemble_dw_ms": v["k_assemble_dw_ms"], "speedup_kernel_vs_f64": f64_k_asm_ms / v["k_assemble_dw_ms"],
        "k_recover_factored_dw_ms": v["k_recover_factored_dw_ms"],
        "roofline_hbm": {"achieved": bpt * nE / k_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                         "frac": bpt * nE / k_s / 1e9 / hbm_peak, "bytes_per_tet": bpt,
                         "traffic": prof["dram_bytes_per_tet"] * nE if "dram_bytes_per_tet" in prof else None},
    }
    if "fp64_inst_per_tet" in prof:
        g = prof["fp64_inst_per_tet"] * nE / k_s / 1e9
        out["roofline_fp64"] = {"achieved": g, "peak": fp64_peak_gops, "unit": "G FP64-op/s",
                                "frac": g / fp64_peak_gops, "ops_per_tet": prof["fp64_inst_per_tet"],
                                "ops_source": "ncu FP64 instructions (DFMA+DADD+DMUL) per element"}
    if "fp32_inst_per_tet" in prof:
        out["fp32_inst_per_tet"] = prof["fp32_inst_per_tet"]
    return out


# ---------------------------------------------------------------------------
# batched workload: 256 problems, Kuhn m_i^3 cubes refined once, m_i from
# sizes log-uniform in [1e4, 5e5] elements (seed 4), each its own lognormal a
# ---------------------------------------------------------------------------
def batched_section(ph, dev, steps, warmup):
    """The batched workload: 256 problems, each its own mesh (Kuhn m_i^3 cube
    refined once) and lognormal field.  Mesh builds: 256 ph_mesh_create calls
    against one ph_mesh_create_batch.  Numeric phase (assembly with the
    element factor and recovery from a seeded Lambda): one captured graph of
    three persistent launches against 256 sequential plain call pairs."""
    import torch
    rng = np.random.Generator(np.random.PCG64(4))
    sizes = np.exp(rng.uniform(np.log(1e4), np.log(5e5), 256))
    ms = np.clip(np.round((sizes / 72.0) ** (1.0 / 3.0)), 6, 19).astype(int)
    inputs = {}
    for m in sorted(set(ms.tolist())):
        coord, tet = meshgen.kuhn_cube(int(m))
        coord, tet, _ = meshgen.refined(coord, tet, 1)
        inputs[m] = (torch.as_tensor(coord, device=dev), torch.as_tensor(tet, device=dev))
    coords = [inputs[m][0] for m in ms]
    tets = [inputs[m][1] for m in ms]

    def build_separate():
        out = [ph.Mesh(c, t) for c, t in zip(coords, tets)]
        torch.cuda.synchronize()
        return out

    def build_batched():
        out = ph.create_meshes(coords, tets)
        torch.cuda.synchronize()
        return out

    build_ms = {}
    for name, fn in (("separate_calls", build_separate), ("one_batched_call", build_batched)):
        best = float("inf")
        for _ in range(3):
            t0 = time.perf_counter()
            built = fn()
            best = min(best, (time.perf_counter() - t0) * 1e3)
            if name == "separate_calls" or _ < 2:  # keep the last batched build
                for mm in built:
                    mm.close()
        build_ms[name] = best
    meshes = built  # the batched build's meshes
    fcache = {}
    probs = []
    for i, (m, mesh) in enumerate(zip(ms, meshes)):
        if m not in fcache:
            cen = mesh.faces()["face_centroid"].cpu().numpy()
            fcache[m] = torch.as_tensor(np.asarray(meshgen.sin_source(cen), np.float64), device=dev)
        probs.append(dict(mesh=mesh, f=fcache[m], a=torch.as_tensor(meshgen.lognormal_field(mesh.nE, 4000 + i),
                                                                     device=dev),
                          values=torch.empty(mesh.nnz, dtype=torch.float64, device=dev),
                          rhs=torch.empty(mesh.L, dtype=torch.float64, device=dev),
                          factor=torch.empty((mesh.nE, 10), dtype=torch.float64, device=dev),
                          lam=torch.as_tensor(np.random.default_rng(70 + i).standard_normal(mesh.L), device=dev),
                          u=torch.empty((mesh.nE, 4), dtype=torch.float64, device=dev)))
    total = sum(p["mesh"].nE for p in probs)
    batch = ph.Batch([p["mesh"] for p in probs])
    batch.bind([p["a"] for p in probs], [0.1] * len(probs), [p["f"] for p in probs], [p["values"] for p in probs],
               [p["rhs"] for p in probs], factor=[p["factor"] for p in probs])
    batch.bind_recovery([p["lam"] for p in probs], [p["u"] for p in probs])
    tune_ms = batch.autotune(reps=2)
    cfg = dict(batch.get_config(), best_ms=tune_ms)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    n0 = ph.ph_launch_count()
    graph_ms = timed(batch.graph_launch)
    launches_graph = (ph.ph_launch_count() - n0) / (steps + warmup)

    def plain():
        for p in probs:
            p["mesh"].assemble(p["a"], 0.1, p["f"], values=p["values"], rhs=p["rhs"], factor=p["factor"])
            p["mesh"].recover_factored(p["factor"], 0.1, p["f"], p["lam"], u=p["u"])

    n0 = ph.ph_launch_count()
    plain_ms = timed(plain)
    launches_plain = (ph.ph_launch_count() - n0) / (steps + warmup)
    batch.close()
    for p in probs:
        p["mesh"].close()
    return {
        "problems": len(probs), "tets": int(total), "distinct_mesh_shapes": len(inputs),
        "step": "assembly and condensation with the element factor + recovery from a seeded Lambda",
        "mesh_build_ms": build_ms, "mesh_build_speedup": build_ms["separate_calls"] / build_ms["one_batched_call"],
        "batched_graph_ms": graph_ms, "batched_tets_per_s": total / (graph_ms * 1e-3),
        "plain_sequential_ms": plain_ms, "plain_sequential_tets_per_s": total / (plain_ms * 1e-3),
        "speedup_vs_sequential": plain_ms / graph_ms, "autotuned": cfg,
        "launches_per_batch": {"graph": launches_graph, "sequential": launches_plain},
    }


# ---------------------------------------------------------------------------
# adjoint workload: Kuhn 6^3 cube refined 3 levels (2,239,488 tets), c = 0.1,
# U_obs from a lognormal a (seed 5), gradient at a lognormal a (seed 51)
# ---------------------------------------------------------------------------
def adjoint_section(ph, dev, rtol=1e-10):
    """One gradient dJ/dlog a on the adjoint workload (config 5): assembly,
    Schwarz-preconditioned PCG forward solve, recovery and misfit, adjoint
    right-hand side, adjoint solve with the same H and preconditioner, and the
    gradient kernel, each timed with CUDA events."""
    import torch
    p = meshgen.problem("kuhn_m6_k3")
    mesh = ph.Mesh(torch.as_tensor(p.coord, device=dev), torch.as_tensor(p.tet, device=dev))
    cen = mesh.faces()["face_centroid"].cpu().numpy()
    f = torch.as_tensor(np.asarray(meshgen.sin_source(cen), np.float64), device=dev)
    c = 0.1

    def forward(a):
        values, rhs, factor = mesh.assemble(a, c, f, factor=True)
        lam, it, P = ph.solve_system(mesh, values, rhs, rtol, 100000)
        P.close()
        return mesh.recover_factored(factor, c, f, lam)

    a_obs = torch.as_tensor(meshgen.lognormal_field(p.nE, 5), device=dev)
    u_obs = forward(a_obs)
    a = torch.as_tensor(meshgen.lognormal_field(p.nE, 51), device=dev)
    forward(a)  # warm-up
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    values, rhs, factor = mesh.assemble(a, c, f, factor=True)
    ev[1].record(stream)
    P = ph.Schwarz(mesh, values)
    ev[2].record(stream)
    lam, it1, _, _ = P.solve(values, rhs, rtol=rtol, maxit=100000)
    ev[3].record(stream)
    u = mesh.recover_factored(factor, c, f, lam)
    J = mesh.misfit(u, u_obs)
    ev[4].record(stream)
    rq = mesh.adjoint_rhs(factor, c, u, u_obs)
    ev[5].record(stream)
    q, it2, _, _ = P.solve(values, rq, rtol=rtol, maxit=100000)
    ev[6].record(stream)
    grad = mesh.adjoint_grad(a, factor, c, u, u_obs, q)
    ev[7].record(stream)
    torch.cuda.synchronize()
    P.close()
    t = [ev[i].elapsed_time(ev[i + 1]) for i in range(7)]
    total = sum(t)
    adj_kernels_ms = t[4] + t[6]
    out = {
        "workload": "Kuhn 6^3 cube, 3 refinement levels", "nE": p.nE, "L": mesh.L,
        "J": J.item(), "grad_norm": grad.norm().item(),
        "grads_per_s": 1000.0 / total, "ms_per_gradient": total,
        "ms": {"assemble": t[0], "schwarz_setup": t[1], "forward_solve": t[2], "recover_misfit": t[3],
               "adjoint_rhs": t[4], "adjoint_solve": t[5], "adjoint_grad": t[6]},
        "pcg_iterations": [it1, it2], "pcg_rtol": rtol, "preconditioner": "edge-patch additive Schwarz",
        "adjoint_kernels_tets_per_s": p.nE / (adj_kernels_ms * 1e-3),
        "note": "gradient time is dominated by the two PCG solves of the condensed system",
    }
    mesh.close()
    return out


# ---------------------------------------------------------------------------
# oracle (CPU) on a bounded sample of the workload
# ---------------------------------------------------------------------------
def oracle_sample(p, n_tets):
    """Sub-mesh of the first n_tets elements (vertices renumbered), its own
    face data, coefficients and a seeded Lambda."""
    tet = p.tet[:n_tets]
    used, inv = np.unique(tet.ravel(), return_inverse=True)
    tet_s = inv.reshape(-1, 4).astype(np.int32)
    coord_s = p.coord[used]
    return coord_s, tet_s, p.a[:n_tets]


def oracle_step(p, coord_s, tet_s, a_s, nthreads):
    """One pass of the oracle over a sub-mesh: faces, multipliers, CSR
    pattern, face data, assembly and condensation, recovery (element loops
    on nthreads host threads)."""
    import oracle
    fc = oracle.faces(tet_s, coord_s.shape[0])
    fm, L = oracle.multipliers(fc["face_kind"])
    rowptr, colind = oracle.csr_pattern(fc["tet_face"], fm, L)
    cen = oracle.face_centroids(coord_s, fc["face_vtx"])
    f = np.asarray(p.f(cen), np.float64)
    csr = {"face_mult": fm, "L": L, "rowptr": rowptr, "colind": colind}
    oracle.assemble(coord_s, tet_s, fc, csr, a_s, p.c, f, nthreads=nthreads)
    lam = np.random.default_rng(7).standard_normal(L)
    oracle.recover(coord_s, tet_s, fc, fm, a_s, p.c, f, lam, nthreads=nthreads)


def sized_oracle_run(p, budget_s, nthreads, steps=1):
    """Size a prefix sub-mesh to about budget_s seconds per pass at nthreads,
    then time `steps` passes.  Returns (tets, mean seconds per pass)."""
    n = 20000
    coord_s, tet_s, a_s = oracle_sample(p, n)
    t0 = time.perf_counter()
    oracle_step(p, coord_s, tet_s, a_s, nthreads)
    dt = time.perf_counter() - t0
    n = int(min(p.nE, max(20000, n * budget_s / max(dt, 1e-6))))
    coord_s, tet_s, a_s = oracle_sample(p, n)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle_step(p, coord_s, tet_s, a_s, nthreads)
        times.append(time.perf_counter() - t0)
    return n, float(np.mean(times))


def cpu_baseline(p, workload, budget_s=15.0):
    """Time the oracle as it stands on every host core (its element loops
    shared out by OpenMP; faces and CSR pattern are serial sorts), and on
    one core for the speed-up, each on a prefix sample sized to about
    budget_s/2 seconds of work."""
    import oracle
    oracle.build()
    cores = host_cores()
    n_all, t_all = sized_oracle_run(p, budget_s / 2, cores)
    n_one, t_one = sized_oracle_run(p, budget_s / 2, 1)
    what = ("faces, multipliers, CSR pattern, assembly+condensation (binary128 per element), recovery")
    return {"value": n_all / t_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {n_all} tets of the {workload} mesh as a sub-mesh: {what}; {t_all:.2f} s per pass "
                      f"on {cores} threads",
            "single_thread": {"value": n_one / t_one, "cores": 1,
                              "sample": f"first {n_one} tets, {t_one:.2f} s per pass"},
            "speedup": (n_all / t_all) / (n_one / t_one)}


def profile_pcg(iters):
    """A fixed number of Schwarz-preconditioned PCG iterations on the adjoint
    workload's system (Kuhn 6^3 cube, 3 levels, c = 0.1, lognormal a with
    seed 51): a target for profiler launch lists of the solve."""
    import torch
    import paper_2509_11133_gb300 as ph
    from paper_2509_11133_gb300 import build
    build.build()
    ph.load()
    dev = torch.device("cuda", 0)
    p = meshgen.problem("kuhn_m6_k3")
    mesh = ph.Mesh(torch.as_tensor(p.coord, device=dev), torch.as_tensor(p.tet, device=dev))
    cen = mesh.faces()["face_centroid"].cpu().numpy()
    f = torch.as_tensor(np.asarray(meshgen.sin_source(cen), np.float64), device=dev)
    a = torch.as_tensor(meshgen.lognormal_field(p.nE, 51), device=dev)
    values, rhs = mesh.assemble(a, 0.1, f)
    P = ph.Schwarz(mesh, values)
    _, it, _, _ = P.solve(values, rhs, rtol=0.0, maxit=iters, check=False)
    torch.cuda.synchronize()
    print(json.dumps({"profile_pcg": {"L": mesh.L, "iterations": it}}))
    P.close()
    mesh.close()
    return 0


def profile_kernels(workload, reps, variant="f64"):
    """Profiler target for the element kernels: on the given workload, `reps`
    rounds of assembly with the element factor and recovery from a seeded
    Lambda (ph_assemble and ph_recover_factored, or their double-word
    versions for variant "dw"), the
    misfit, the adjoint right-hand side and the adjoint gradient from a seeded
    q (no solves, so few launches)."""
    import torch
    import paper_2509_11133_gb300 as ph
    from paper_2509_11133_gb300 import build
    build.build()
    ph.load()
    dev = torch.device("cuda", 0)
    p = make_problem(workload)
    mesh = ph.Mesh(torch.as_tensor(p.coord, device=dev), torch.as_tensor(p.tet, device=dev),
                   geometry="dw" if variant == "dw" else "f64")
    cen = mesh.faces()["face_centroid"].cpu().numpy()
    f = torch.as_tensor(np.asarray(p.f(cen), np.float64), device=dev)
    a = torch.as_tensor(p.a, device=dev)
    rng = np.random.default_rng(7)
    lam = torch.as_tensor(rng.standard_normal(mesh.L), device=dev)
    q = torch.as_tensor(rng.standard_normal(mesh.L), device=dev)
    u_obs = torch.as_tensor(rng.standard_normal((mesh.nE, 4)), device=dev)
    for _ in range(reps):
        values, rhs, factor = mesh.assemble(a, p.c, f, factor=True, variant=variant)
        u = mesh.recover_factored(factor, p.c, f, lam, variant=variant)
        mesh.misfit(u, u_obs)
        mesh.adjoint_rhs(factor, p.c, u, u_obs)
        if variant == "f64":  # the gradient reads the fp64 geometry record
            mesh.adjoint_grad(a, factor, p.c, u, u_obs, q)
    torch.cuda.synchronize()
    mesh.check()
    print(json.dumps({"profile_kernels": {"workload": workload, "nE": mesh.nE, "reps": reps, "variant": variant}}))
    mesh.close()
    return 0


def workload_config(workload, p, world):
    """The config object of both arms.  Counts of the all-Dirichlet Kuhn
    mesh in closed form: 12 m^2 4^k boundary faces, nF = (4 nE + boundary)/2,
    L = nF, nnz = nF + 12 nE (each checked against the device build in the
    full-size tests)."""
    m, k = p.info["m"], p.info["k"]
    nE = p.nE
    nF = (4 * nE + 12 * m * m * 4 ** k) // 2
    if workload == "jitter_checker_18m":
        mesh = (f"Kuhn {m}^3 unit cube, {k} levels of the paper's 1->12 refinement, interior vertices moved "
                f"uniformly in a ball of 0.2 x their shortest edge (seed 3; {p.info.get('jitter_redrawn', 0)} "
                f"vertices redrawn with a halved radius)")
        coef = "a in {1, 1e4} on an 8^3 checkerboard of element centroids"
    else:
        mesh = f"Kuhn {m}^3 unit cube, {k} levels of the paper's 1->12 refinement"
        coef = "exp(N(0,1)) per element, seed 2"
    return {
        "workload": workload,
        "mesh": mesh,
        "nE": nE, "nC": p.nC, "nF": nF, "L": nF, "nnz": nF + 12 * nE,
        "a": coef, "c": p.c, "f": "(3 pi^2 + 1) sin(pi x) sin(pi y) sin(pi z)",
        "boundary": "zero Dirichlet",
        "step": "mesh build (faces, multipliers, CSR pattern, geometry) + assembly and condensation "
                "(with element factor) + element recovery from a seeded Lambda",
        "l2": "512 MiB buffer written between timed steps (outside the step events)",
        "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
    }


def reference_arm(args):
    p = make_problem(args.workload)
    import oracle
    oracle.build()
    cores = host_cores()
    # size one step to ~budget seconds on every core, then W + K steps
    budget = max(0.1, args.ref_step_s)
    n = 20000
    coord_s, tet_s, a_s = oracle_sample(p, n)
    t0 = time.perf_counter()
    oracle_step(p, coord_s, tet_s, a_s, cores)
    dt = time.perf_counter() - t0
    n = int(min(p.nE, max(20000, n * budget / max(dt, 1e-6))))
    coord_s, tet_s, a_s = oracle_sample(p, n)
    for _ in range(args.warmup):
        oracle_step(p, coord_s, tet_s, a_s, cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_step(p, coord_s, tet_s, a_s, cores)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = n / (ms * 1e-3)
    sample = (f"first {n} tets of the {args.workload} mesh as a sub-mesh per step: faces, multipliers, CSR pattern, "
              f"assembly+condensation, recovery (C oracle, binary128 per element, element loops on {cores} "
              f"threads)")
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.workload, p, 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiler runs)")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and adjoint sections")
    ap.add_argument("--no-variant", action="store_true", help="skip the double-word assembly variant's timed loop")
    ap.add_argument("--variant", default="f64", choices=["f64", "dw"],
                    help="assembly used by --profile-kernels")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-step-s", type=float, default=3.0)
    ap.add_argument("--profile-pcg", type=int, default=0, metavar="N",
                    help="profiler target: N Schwarz-PCG iterations on the adjoint workload, then exit")
    ap.add_argument("--profile-kernels", type=int, default=0, metavar="R",
                    help="profiler target: R rounds of the element kernels (assembly, recovery, misfit, adjoint) "
                         "on --workload, then exit")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.profile_pcg > 0:
        return profile_pcg(args.profile_pcg)
    if args.profile_kernels > 0:
        return profile_kernels(args.workload, args.profile_kernels, args.variant)
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(reference_arm(args)), flush=True)
        return 0
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        line = gpu_arm(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
