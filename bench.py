"""Benchmark: leap-frog triangle-steps per second on the ~4M-triangle scatterer workload.

One bench "step" is one full leap-frog step (E half-step over every interior edge, the line
source, B half-step over every triangle) of the graded unit-square mesh with an equilateral
PEC hole (h 2e-4 .. 8e-4, ~4M triangles, FP32 fields, FP64-built coefficients).  By default
the steps run temporally blocked: greedy tiles of <= 2500 triangles with each tile's boundary
rings stored first (--tiler greedy: the greedy method's own order; --tiler kd: KD tiles), 8
steps per launch, 512 threads per tile (--variant plain: two kernels per step in RCM order).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Prints one JSON line.  ``value`` = triangles * K / device time of the K timed steps (inputs
resident in HBM); ``e2e`` = the same work through the public API with host buffers: fields
written from pinned host memory, K steps, fields read back, all inside the timed region.
``roofline`` refers to the dominant kernel, timed per launch with CUDA events on the launch
stream in a window right after the timed region; ``cpu_baseline`` is the FP64 oracle on a
bounded window of the same workload.  ``--impl reference`` times that oracle alone.
N > 1 (torchrun): independent replicas, one per GPU, no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = ("scatterer-4M: unit square, PEC walls and PEC equilateral hole (side 0.2, centre "
            "(0.5,0.5)), spacing graded 2e-4..8e-4, jitter 0.2h, FP32 fields, line source "
            "x=0.35, w0=2*pi*20")
WORKLOAD_PLASMA = ("plasma-1M: unit square, PEC walls, uniform spacing (1M triangles), jitter 0.2h, "
                   "Gaussian density n = (0.8 w0)^2 exp(-|r-c|^2/(2*0.15^2)) on the nodes, cold-plasma "
                   "current on the edges, collision rate 0.01 w0, FP32 fields, line source x=0.35, "
                   "w0=2*pi*20")
METRIC = "cell-updates/s"
UNIT = "triangle-steps/s"
L2_BYTES = 129e6


# Counters of the dominant kernel per launch (DRAM bytes, shared-memory wavefronts, warp
# instructions), from one ncu capture of the bench command at its configuration, stored in
# profiles/ncu_counters.json with the sha1 of the sources they measured: used only while those
# sources are unchanged, else reported as null.
COUNTER_FILE = os.path.join(ROOT, "profiles", "ncu_counters.json")
COUNTER_SOURCES = ("paper_1812_01448_gb300/csrc/kernels_tb.cu", "paper_1812_01448_gb300/csrc/kernels_tbf.cu",
                   "paper_1812_01448_gb300/csrc/device.cuh", "paper_1812_01448_gb300/csrc/tiles_host.cpp",
                   "paper_1812_01448_gb300/csrc/mesh_host.cpp")


def sources_sha1(paths=COUNTER_SOURCES) -> str:
    import hashlib
    h = hashlib.sha1()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _counters(key: dict):
    """(counters per launch, why-null) for a configuration key, from COUNTER_FILE."""
    try:
        with open(COUNTER_FILE) as f:
            recs = json.load(f)["records"]
    except (OSError, ValueError, KeyError):
        return None, "no counter file"
    sha = sources_sha1()
    for r in recs:
        if r["config"] == key:
            if r["sources_sha1"] != sha:
                return None, "kernel sources changed since the capture"
            return r, None
    return None, "configuration not captured"


def onchip_roofline(c: dict, ms_per_launch: float, sm_mhz) -> dict:
    """The blocked kernel against its on-chip limits, from counters of one launch (ncu) over the
    launch time measured live: shared-memory wavefronts (one per SM per cycle: 32 banks x 4 B)
    and warp instructions issued (four schedulers per SM, one each per cycle)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    hz = (sm_mhz or 2070.0) * 1e6
    t = ms_per_launch * 1e-3
    wf, ins = float(c["smem_wavefronts"]), float(c["warp_instructions"])
    ideal = float(c["smem_instructions"])
    smem = {"achieved": wf / t, "peak": sms * hz, "unit": "wavefronts/s", "frac": wf / t / (sms * hz),
            "wavefronts_per_launch": wf}
    ld, st, misc = (c.get(k) for k in ("pipe_lsu_wavefronts_mem_shared_op_ld", "pipe_lsu_wavefronts_mem_shared_op_st",
                                       "pipe_lsu_wavefronts_mem_shared_op_misc"))
    if ld is not None and st is not None:
        # loads and stores against one wavefront per instruction (no bank conflict); the rest of
        # the wavefronts are the cp.async gathers' shared-memory writes (LDGSTS, "misc")
        smem.update({"load_store_wavefronts": ld + st, "load_store_instructions": ideal,
                     "bank_conflict_factor": (ld + st) / ideal if ideal else None,
                     "cp_async_wavefronts": misc})
    else:
        smem.update({"conflict_free_wavefronts_per_launch": ideal,
                     "bank_conflict_factor": wf / ideal if ideal else None})
    return {
        "bound": "shared-memory wavefronts",
        "smem": smem,
        "issue": {"achieved": ins / t, "peak": 4 * sms * hz, "unit": "warp instructions/s",
                  "frac": ins / t / (4 * sms * hz), "instructions_per_launch": ins},
        "clock_mhz": hz / 1e6, "sms": sms,
        "counters": "profiles/ncu_counters.json (one ncu capture of this configuration; "
                    "time is this run's CUDA-event launch time)",
    }


def partition_stats(m):
    """Fig. 6 quantities of a tiled mesh: parts, triangles per part (mean, rms deviation, max)
    and the shared boundary l_Sigma, the interior edges whose triangles lie in two parts."""
    import numpy as np

    off = m.tiles()
    sizes = np.diff(off)
    t = m.tables()
    tile = np.searchsorted(off, np.arange(m.n_tris), side="right") - 1
    et = t["edge_tri"]
    shared = int(np.count_nonzero(tile[et[:, 0]] != tile[et[:, 1]]))
    return {"parts": int(sizes.size), "tris_mean": float(sizes.mean()), "tris_rms": float(sizes.std()),
            "tris_max": int(sizes.max()), "shared_edges": shared}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def max_over_ranks(x: float, dist=None) -> float:
    """Maximum of x over all ranks (x itself without a process group).  Uses a CUDA tensor
    under NCCL and a CPU tensor under gloo."""
    if dist is None or not dist.is_initialized():
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def load_workload(name="scatterer"):
    """(mesh, source edge ids, amplitudes, w0, t0, tau, node density or None, nu, description)."""
    import meshgen
    w0 = 2 * math.pi * 20
    if name == "plasma":
        ms = meshgen.cached("plasma_1003", meshgen.plasma_square_mesh)
        ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.35, ms.h)
        dens = meshgen.plasma_density_nodes(ms.xy, w0)
        return ms, ids, amp, w0, 0.1, 0.05, dens, 0.01 * w0, WORKLOAD_PLASMA
    ms = meshgen.cached("scatterer_1002", meshgen.scatterer_mesh)
    ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.35, 2e-4)
    return ms, ids, amp, w0, 0.1, 0.05, None, 0.0, WORKLOAD


def _oracle_ops(ms):
    from oracle import mesh as om, operators
    return operators.Operators(om.canonicalize(ms.xy, ms.tris))


def cpu_oracle_rates(ms, ops, state, dt, budget_s, plasma=None, source=None, numpy_too=True):
    """Time the oracle on this workload from `state`: the compiled C step (oracle/cstep.c) on one
    host core and on all of them, and the numpy oracle on one core, each for about budget_s
    seconds.  Returns {"c1": (rate, steps, seconds, threads), "call": ..., "numpy": ...}."""
    from oracle import cstep, leapfrog as lf
    out = {}
    stepper = cstep.Stepper(ops)
    for key, threads in (("c1", 1), ("call", cstep.host_cores())):
        st, used = stepper.run(state, dt, 1, plasma, source, threads)      # first touch
        t = time.perf_counter()
        st, used = stepper.run(st, dt, 2, plasma, source, threads)
        per = (time.perf_counter() - t) / 2
        n = max(2, int(budget_s / max(per, 1e-6)))
        t = time.perf_counter()
        st, used = stepper.run(st, dt, n, plasma, source, threads)
        el = time.perf_counter() - t
        out[key] = (ms.n_tris * n / el, n, el, used)
    if numpy_too:
        nbar = plasma.nbar(ops) if plasma is not None else None
        cols = ops.col_of_edge[source.edge_ids] if source is not None else None
        st = lf.step(ops, state, dt, plasma, source, nbar, cols)
        n = 0
        t = time.perf_counter()
        while n < 3 or time.perf_counter() - t < budget_s:
            st = lf.step(ops, st, dt, plasma, source, nbar, cols)
            n += 1
        el = time.perf_counter() - t
        out["numpy"] = (ms.n_tris * n / el, n, el, 1)
    return out


def cpu_baseline_line(rates, what):
    """The bench line's cpu_baseline: the compiled oracle on all host cores, with the one-core
    and numpy figures beside it."""
    r, n, el, used = rates["call"]
    line = {"value": r, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"{n} leap-frog steps of {what} in {el:.1f} s (oracle/cstep.c, FP64, {used} threads)"}
    r1, n1, el1, _ = rates["c1"]
    line["single_core"] = {"value": r1, "cores": 1,
                           "sample": f"{n1} steps in {el1:.1f} s (oracle/cstep.c, FP64, one thread)"}
    if "numpy" in rates:
        r2, n2, el2, _ = rates["numpy"]
        line["numpy_oracle"] = {"value": r2, "cores": 1,
                                "sample": f"{n2} steps in {el2:.1f} s (oracle/leapfrog.py, numpy/scipy.sparse FP64)"}
    return line


def run_reference(args):
    """The oracle timed alone on the host cores (the reference arm): the compiled C step on all
    cores, over a bounded number of steps of the same workload."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import cstep, leapfrog as lf, spectral
    ms, ids, amp, w0, t0, tau, dens, nu, what = load_workload(args.workload)
    ops = _oracle_ops(ms)
    # the oracle takes the same dt the library would (dt = 0.5 * 2 / rho, rho by power iteration)
    rho, _ = spectral.power_iteration(ops, 200)
    dt = 1.0 / rho
    src = lf.Source(ids, amp, w0, t0, tau)
    pl = lf.Plasma(dens, nu) if dens is not None else None
    stepper = cstep.Stepper(ops)
    st = lf.initial_state(ops)
    st, _ = stepper.run(st, dt, 1, pl, src, threads=cstep.host_cores())    # first touch
    t = time.perf_counter()
    for _ in range(args.warmup):
        st, _ = stepper.run(st, dt, 1, pl, src, threads=cstep.host_cores())
    per = (time.perf_counter() - t) / max(1, args.warmup)
    # a bounded sample: at most about a minute of steps
    n = max(1, min(args.steps, int(60.0 / max(per, 1e-6))))
    t = time.perf_counter()
    st, used = stepper.run(st, dt, n, pl, src, threads=cstep.host_cores())
    el = time.perf_counter() - t
    rate = ms.n_tris * n / el
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / n,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": what, "n_tris": ms.n_tris},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": f"{n} of {args.steps} leap-frog steps on the full mesh after {args.warmup} warm-up steps "
                                   f"(oracle/cstep.c, FP64, {used} threads, {el:.1f} s)"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_native(args):
    import numpy as np
    import torch

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1812_01448_gb300 import build as b
    b.build()
    import paper_1812_01448_gb300 as ue

    ms, ids, amp, w0, t0, tau, dens, nu, what = load_workload(args.workload)
    stream = torch.cuda.current_stream()
    blocked = args.variant == "blocked"
    tiled = {"greedy": ue.UE_REORDER_GREEDY, "rings": ue.UE_REORDER_GREEDY_RINGS, "kd": ue.UE_REORDER_KD}[args.tiler]
    m = ue.Mesh(ms.xy, ms.tris, reorder=tiled if blocked else ue.UE_REORDER_RCM,
                tile_tris=args.tile_tris)
    if args.frame > 0:
        m.frame_attach(args.frame)
    variant = {"plain": ue.UE_VARIANT_PLAIN, "blocked": ue.UE_VARIANT_BLOCKED,
               "persistent": ue.UE_VARIANT_PERSISTENT}[args.variant]
    vopt = dict(variant=variant, block_depth=args.block_depth, graph_chunk=args.graph_chunk,
                tb_threads=args.tb_threads,
                tb_kernel=ue.UE_TB_FUSED if args.tb_kernel == "fused" else ue.UE_TB_SPLIT)
    if args.quick_setup:
        # profiling runs: a fixed dt instead of the 200-iteration power iteration, so that few
        # kernel launches precede the captured ones
        m.geometry_build(stream=stream, dt_mode=ue.UE_DT_GIVEN, dt=1e-5, **vopt)
    else:
        m.geometry_build(stream=stream, **vopt)
    dt, rho, _ = m.get_dt()
    m.set_source(ids, amp, w0, t0, tau)
    if dens is not None:
        m.set_plasma(dens, nu)
    st = m.stats()
    n_t, n_ei = st["n_tris"], st["n_interior_edges"]
    part_stats = partition_stats(m) if blocked else None
    frame = m.frame_info() if args.frame > 0 else None

    # warm-up, then the step graphs captured and uploaded (setup, like the tiles: a run of
    # fewer warm-up steps than one graph chunk would otherwise capture inside the timed call)
    m.step_n(args.warmup, stream)
    m.step_prepare(stream)
    torch.cuda.synchronize()
    if args.step_sweep:
        # the cost of one ue_step_n(n) call against n (median of 5 calls, CUDA events on the
        # launch stream): how a launch's fixed cost and its per-step cost split
        rows = []
        for n in [int(x) for x in args.step_sweep.split(",")]:
            ts = []
            for _ in range(5):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                m.step_n(n, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            rows.append({"steps": n, "ms_per_call": float(np.median(ts)), "us_per_step": 1e3 * float(np.median(ts)) / n})
        if rank == 0:
            print(json.dumps({"metric": "ue_step_n call time against its step count", "workload": what,
                              "variant": args.variant, "tiler": args.tiler, "block_depth": args.block_depth,
                              "rows": rows}), flush=True)
        m.close()
        return

    def barrier():
        if dist is not None:
            dist.barrier()

    launches0 = m.stats()["kernel_launches"]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        m.step_n(args.steps, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = m.stats()["kernel_launches"] - launches0
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), dist)
    value = world * n_t * args.steps / (ms_total * 1e-3)

    # per-kernel device times, CUDA events on the launch stream, right after the timed region
    nprof = min(200, max(20, args.steps // 10))
    if blocked:
        nprof = max(4, nprof // args.block_depth)
    prof_ms, prof_bytes = m.profile_steps(nprof, stream)
    names = ["k_edge_half: E half-step (eq. 3)", "k_source", "k_tri_half: B half-step (eq. 4)"]
    if blocked and args.frame > 0:
        names[2] = (f"frame region: gather, {args.block_depth} plain steps of the tiles next to the PML "
                    "frame with the frame, scatter (beside k_tbp on a second stream)")
    if blocked:
        used = m.stats()["tb_kernel_used"]
        kname = {1: "k_tb", 2: "k_tbs", 3: "k_tbp", 4: "k_tbf", 5: "k_tbf1"}.get(used, "?")
        form = {1: "one CTA per tile", 2: "one CTA per tile, records in shared memory",
                3: "one CTA per SM with the next tile's loads in flight",
                4: "fused edge and triangle phases, one CTA per SM with the next tile's loads in flight",
                5: "the whole mesh in one CTA"}.get(used, "")
        names[0] = f"{kname}: {args.block_depth} leap-frog steps per launch on {args.tiler} tiles, {form}"
    k = int(np.argmax(prof_ms))
    peak, peak_kind = _peaks()
    achieved = prof_bytes[k] / (prof_ms[k] * 1e-3) / 1e9
    ckey = {"workload": args.workload, "variant": args.variant, "tiler": args.tiler if blocked else "",
            "tile_tris": args.tile_tris if blocked else 0, "block_depth": args.block_depth if blocked else 1,
            "threads": (args.tb_threads or 512) if blocked else 0, "frame": args.frame,
            "kernel": args.tb_kernel if blocked else ""}
    crec, cwhy = _counters(ckey) if k == 0 else (None, "not the profiled kernel")
    traffic = float(crec["per_launch"]["dram_bytes"]) if crec else None
    traffic_src = "profiles/ncu_counters.json" if crec else cwhy
    step_bytes = st["bytes_per_step"]
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
            "kernel": names[k],
            "bytes_per_launch": prof_bytes[k], "ms_per_launch": prof_ms[k],
            "peak_kind": f"{peak_kind} (STREAM-style copy)",
            "step": {"bytes": step_bytes, "achieved_gbs": step_bytes * args.steps / (ms_total * 1e-3) / 1e9,
                     "frac": step_bytes * args.steps / (ms_total * 1e-3) / 1e9 / peak,
                     "kernel_ms": [float(x) for x in prof_ms]}}
    if blocked:
        roof["algorithmic_bytes_note"] = ("bytes of the same steps done by the plain kernels (an effective "
                                          "rate: temporal blocking keeps them on chip, so frac can exceed 1); "
                                          "the blocked kernel streams streamed_bytes_per_launch, and its "
                                          "binding resource is in onchip")
        roof["streamed_bytes_per_launch"] = prof_bytes[1]
        roof["streamed_gbs"] = prof_bytes[1] / (prof_ms[0] * 1e-3) / 1e9
    if crec is not None:
        roof["onchip"] = onchip_roofline(crec["per_launch"], prof_ms[k], clk.summary().get("sm_mhz"))

    # end to end through the public API with host buffers: the fields in the product's
    # precision (float32, ue_write_fields_f32 / ue_read_fields_f32) by default, or as doubles;
    # a framed mesh moves them as doubles (the float32 calls refuse it)
    f32 = args.e2e_fields == "f32" and args.frame <= 0
    wt = torch.float32 if f32 else torch.float64
    pinned = lambda n: torch.zeros(n, dtype=wt, pin_memory=True).numpy()
    E0, B0, Eo, Bo = pinned(m.n_edges), pinned(m.n_tris), pinned(m.n_edges), pinned(m.n_tris)
    J0 = Jo = None
    if dens is not None:
        J0, Jo = pinned(m.n_edges), pinned(m.n_edges)
    write = m.write_fields_f32 if f32 else m.write_fields
    read = m.read_fields_f32 if f32 else m.read_fields
    # warm-up of the transfer path: one untimed write and read of the same pinned buffers (the
    # GPU's first touch of freshly pinned pages costs address translation, not bandwidth)
    write(E0, B0, J0, stream=stream)
    read(j=dens is not None, out={"E": Eo, "B": Bo, "j": Jo}, stream=stream)
    barrier()
    torch.cuda.synchronize()
    d0 = m.stats()["direct_fields"]
    t_e2e = time.perf_counter()
    write(E0, B0, J0, stream=stream)
    m.set_step(0)
    m.step_n(args.steps, stream)
    read(j=dens is not None, out={"E": Eo, "B": Bo, "j": Jo}, stream=stream)
    t_e2e = max_over_ranks(time.perf_counter() - t_e2e, dist)
    io = (4.0 if f32 else 8.0) * (m.n_edges + m.n_tris + (m.n_edges if dens is not None else 0))
    api = "ue_write_fields_f32 / ue_read_fields_f32 (float32)" if f32 else "ue_write_fields / ue_read_fields (float64)"
    e2e = {"value": world * n_t * args.steps / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": io / args.steps, "d2h_bytes_per_step": io / args.steps,
           "what": f"{api}: fields written from pinned host arrays, K steps, fields read into pinned host arrays",
           "fields_moved_in_place": m.stats()["direct_fields"] - d0}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import leapfrog as lf
        ops = _oracle_ops(ms)
        rates = cpu_oracle_rates(ms, ops, lf.initial_state(ops), dt, args.cpu_seconds,
                                 plasma=lf.Plasma(dens, nu) if dens is not None else None,
                                 source=lf.Source(ids, amp, w0, t0, tau))
        cpu = cpu_baseline_line(rates, "the full mesh")

    # steps per replay of the captured graph: whole blocked launches, an even number of them
    # (the field buffers swap each launch), as ue_step_n forms them from graph_chunk
    kd = args.block_depth
    graph_steps = (2 * max(1, args.graph_chunk // (2 * kd)) * kd) if blocked else args.graph_chunk
    if rank == 0:
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": what, "n_tris": n_t, "n_interior_edges": n_ei,
                       "n_edges": m.n_edges, "dt": dt, "rho": rho,
                       "variant": (f"blocked k={args.block_depth} {args.tiler} tiles<={args.tile_tris} "
                                f"threads={args.tb_threads or 512} {args.tb_kernel} kernel" if blocked
                                else args.variant) + f", CUDA graph chunk {graph_steps} steps",
                       "l2": (f"working set {step_bytes / 1e6:.0f} MB per step > {L2_BYTES / 1e6:.0f} MB L2; no flush"
                              if step_bytes > L2_BYTES else
                              f"working set {step_bytes / 1e6:.0f} MB per step < {L2_BYTES / 1e6:.0f} MB L2: "
                              "no flush between steps, so the steps run largely from L2, as every step of a "
                              "long run of this mesh does"),
                       "parallelism": f"replicas x{world}",
                       "tiles": part_stats,
                       "pml_frame": frame},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    m.close()
    if dist is not None:
        dist.destroy_process_group()


def _time_steps(fn, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e-3


def run_cavity(args):
    """The 1,024-triangle PEC cavity (TE(1,1) start, dt = 1/rho) over --steps steps: the whole
    mesh is one tile without a halo, so all the steps run in one launch of one CTA with the mesh
    in shared memory; against the plain path (two kernels per step, CUDA graphs).  Both are
    bound by latency (launches, barriers, dependent shared loads), not by memory: the mesh's
    step touches 55 KB."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_1812_01448_gb300 import build as b
    b.build()
    import paper_1812_01448_gb300 as ue
    import meshgen
    from oracle import leapfrog as lf, mesh as om, operators
    ms = meshgen.cavity_te11_mesh()
    stream = torch.cuda.current_stream()
    probe = ue.Mesh(ms.xy, ms.tris)
    probe.geometry_build()
    dt, rho, _ = probe.get_dt()
    probe.close()
    ops = operators.Operators(om.canonicalize(ms.xy, ms.tris))
    B0 = meshgen.te_mode_b(ops.geom.O, 1, 1, 1.0, 0.5)
    res = {}
    for name, load, opts in (("one CTA", dict(reorder=ue.UE_REORDER_GREEDY, tile_tris=4096),
                              dict(variant=ue.UE_VARIANT_BLOCKED, block_depth=8)),
                             ("plain", dict(), dict(graph_chunk=32))):
        m = ue.Mesh(ms.xy, ms.tris, **load)
        m.geometry_build(stream=stream, dt_mode=ue.UE_DT_GIVEN, dt=dt, **opts)
        m.write_fields(E=np.zeros(m.n_edges), B=B0, stream=stream)
        m.step_n(args.warmup, stream)
        l0 = m.stats()["kernel_launches"]
        t = _time_steps(lambda: m.step_n(args.steps, stream), stream)
        launches = m.stats()["kernel_launches"] - l0
        m.write_fields(E=np.zeros(m.n_edges), B=B0, stream=stream)
        m.set_step(0)
        m.step_n(args.steps, stream)
        E, B, _ = m.read_fields(stream=stream)
        m.close()
        res[name] = (m.n_tris * args.steps / t, t, launches, E, B)
    st = lf.run(ops, lf.initial_state(ops, B=B0), dt, args.steps)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    v, t, launches, E, B = res["one CTA"]
    line = {
        "metric": "cell-updates/s (cavity, one CTA)", "value": v, "unit": UNIT, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "dtype": "f32",
        "data": "synthetic", "gpu_launches": launches,
        "plain": {"value": res["plain"][0], "ms_per_step": 1e3 * res["plain"][1] / args.steps,
                  "gpu_launches": res["plain"][2]},
        "ratio_vs_plain": v / res["plain"][0],
        "vs_oracle": {"E_rel_l2": rel(E, ops.extend(st.E)), "B_rel_l2": rel(B, st.B),
                      "plain_E_rel_l2": rel(res["plain"][3], ops.extend(st.E))},
        "roofline": {"bound": "latency", "ns_per_step": 1e9 * t / args.steps,
                     "what": "one CTA of 512 threads, one barrier per step; the step of the 1,024 triangles "
                             "is a chain of three shared loads and six floating-point operations per thread"},
        "config": {"workload": f"cavity-1k: PEC rectangle 1 x 0.5, 33x17 jittered lattice, {ms.tris.shape[0]} "
                               "triangles, TE(1,1) start, dt = 1/rho", "n_tris": int(ms.tris.shape[0]),
                   "dt": dt, "rho": rho},
    }
    print(json.dumps(line), flush=True)


def run_batch(args):
    """Many independent meshes advanced together, in the launch form the autotuner picks on a
    sample of them (tune.autotune_batch), against the plain form: each mesh stepped alone with
    its own E and B launches, no graph.  Every mesh keeps its own dt (power iteration) and
    line source."""
    import multiprocessing as mp

    import meshgen
    specs = meshgen.batch_specs(args.batch_meshes)
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        meshes = pool.map(meshgen.batch_mesh, specs, chunksize=2)
    t_gen = time.perf_counter() - t0
    import torch
    torch.cuda.set_device(0)
    from paper_1812_01448_gb300 import build as b
    b.build()
    import paper_1812_01448_gb300 as ue
    from paper_1812_01448_gb300 import tune
    stream = torch.cuda.current_stream()
    items = []
    for sp, ms in zip(specs, meshes):
        ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.35, ms.h)
        items.append((ms, ids, amp, sp["omega0"]))
    best, table = tune.autotune_batch(items, sample=args.tune_sample, stream=stream)
    variant = {"plain": ue.UE_VARIANT_PLAIN, "persistent": ue.UE_VARIANT_PERSISTENT,
               "blocked": ue.UE_VARIANT_BLOCKED}[best["variant"]]
    singles = []
    for ms, ids, amp, w0 in items:
        m = ue.Mesh(ms.xy, ms.tris, reorder=tune.TILERS[best["tiler"]], tile_tris=best["tile_tris"])
        m.geometry_build(stream=stream, graph_chunk=-1)          # own dt: power iteration
        m.set_source(ids, amp, w0, 0.1, 0.05)
        singles.append(m)
    n_t = sum(m.n_tris for m in singles)
    # plain form: every mesh alone, E and B launches per mesh per step (plus its g-table launch)
    for m in singles:
        m.step_n(2, stream)
    sp_steps = max(3, args.steps // 50)

    def plain():
        for _ in range(sp_steps):
            for m in singles:
                m.step_n(1, stream)
    t_plain = _time_steps(plain, stream)
    rate_plain = n_t * sp_steps / t_plain
    # the tuned form over the whole batch (rebuilt with each mesh's own dt)
    for m in singles:
        dt = m.get_dt()[0]
        m.geometry_build(stream=stream, dt_mode=ue.UE_DT_GIVEN, dt=dt, graph_chunk=args.graph_chunk,
                         variant=variant, block_depth=best["block_depth"], tb_threads=best["tb_threads"])
    bt = ue.batch_create(singles, stream)
    k = best["block_depth"]
    bt.step_n(max(k, args.warmup - args.warmup % k), stream)
    n_steps = max(k, args.steps - args.steps % k)
    t = _time_steps(lambda: bt.step_n(n_steps, stream), stream)
    rate = n_t * n_steps / t
    bt.close()
    line = {
        "metric": "cell-updates/s (batch of independent meshes)", "unit": UNIT,
        "value": rate, "n_meshes": len(singles), "n_tris_total": n_t, "steps": n_steps,
        "plain_steps": sp_steps, "plain_per_mesh": rate_plain,
        "ratio_batched_vs_plain": rate / rate_plain,
        "tuned": best, "tuning": table,
        "config": {"workload": f"{len(singles)} meshes, log-uniform 5k-200k triangles, random "
                               "scatterer each, own dt and source frequency",
                   "mesh_generation_s": t_gen},
    }
    print(json.dumps(line), flush=True)
    for m in singles:
        m.close()


def run_learned(args):
    """Learned rho (shipped weights) against the 200-iteration power iteration on held-out
    meshes (sizes log-uniform up to --learned-max triangles, plus the 4M scatterer mesh):
    dt-selection time, accuracy, acceptance by the certified bracket, stability."""
    import multiprocessing as mp

    import numpy as np

    import meshgen
    specs = meshgen.learned_specs(args.learned_meshes, seed=2200, n_min=10_000,
                                  n_max=args.learned_max)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        meshes = pool.map(meshgen.learned_mesh, specs, chunksize=1)
    meshes.append(meshgen.cached("scatterer_1002", meshgen.scatterer_mesh))
    import torch
    torch.cuda.set_device(0)
    from paper_1812_01448_gb300 import build as b
    b.build()
    import paper_1812_01448_gb300 as ue
    from paper_1812_01448_gb300 import learned
    p = learned.load_weights(args.weights) if args.weights else learned.load_weights()
    # first launches of each path (module load) outside the measurement
    for mode in (ue.UE_DT_POWER, ue.UE_DT_LEARNED):
        w = ue.Mesh(meshes[0].xy, meshes[0].tris)
        w.geometry_build(dt_mode=mode, mlp_params=p)
        w.close()
    rows = []
    for ms in meshes:
        a = ue.Mesh(ms.xy, ms.tris)
        a.geometry_build()
        _, rho_pi, _ = a.get_dt()
        t_pi = a.stats()["dt_setup_ms"]
        a.close()
        m = ue.Mesh(ms.xy, ms.tris)
        m.geometry_build(dt_mode=ue.UE_DT_LEARNED, mlp_params=p, watchdog_every=100)
        dt, rho, src = m.get_dt()
        st = m.stats()
        rng = np.random.default_rng(0)
        m.write_fields(E=rng.standard_normal(m.n_edges), B=rng.standard_normal(m.n_tris))
        m.step_n(2000)
        ok = m.check()[0]
        m.close()
        rows.append(dict(n_tris=ms.n_tris, rho_pi=rho_pi, rho_hat=st["rho_hat"], rho_lo=st["rho_lo"],
                         rho_hi=st["rho_hi"], accepted=src == ue.UE_RHO_LEARNED,
                         ms_learned=st["dt_setup_ms"], ms_power=t_pi, stable=bool(ok)))
    err = np.array([abs(r["rho_hat"] / r["rho_pi"] - 1) for r in rows])
    acc = [r for r in rows if r["accepted"]]
    big = [r for r in rows if r["n_tris"] >= 1_000_000 and r["accepted"]]
    line = {
        "metric": "learned dt: setup time vs 200-iteration power iteration", "n_meshes": len(rows),
        "median_rel_err": float(np.median(err)), "max_rel_err": float(err.max()),
        "within_2pct": int((err <= 0.02).sum()), "accepted": len(acc),
        "unstable_runs": sum(not r["stable"] for r in rows),
        "median_speedup_accepted": float(np.median([r["ms_power"] / r["ms_learned"] for r in acc])) if acc else None,
        "speedup_largest": (big[-1]["ms_power"] / big[-1]["ms_learned"]) if big else None,
        "rows": rows,
    }
    print(json.dumps(line), flush=True)


def run_modes(args):
    """Highest eigenmodes of the scatterer-4M mesh (ue_modes, the complex-time method with
    deflation in block form): block iterations per second.  Each iteration applies K to the
    block, forms the S-weighted Gram matrix and re-orthonormalises (Cholesky QR); the Gram
    matrix (upper triangle) and the triangular block update are FP64 multiply-adds, m (m+1) n_t
    flops each."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_1812_01448_gb300 import build as b
    b.build()
    import paper_1812_01448_gb300 as ue
    import meshgen
    ms = meshgen.cached("scatterer_1002", meshgen.scatterer_mesh)
    m = ue.Mesh(ms.xy, ms.tris)
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=1e-6)
    n_modes, iters = args.n_modes, max(1, args.steps)
    m.modes(n_modes, iters=max(3, args.warmup))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    om = m.modes(n_modes, iters=iters)
    t = time.perf_counter() - t0
    width = min(32, 2 * n_modes)
    flops = 2.0 * width * (width + 1) * m.n_tris * iters
    fp64_nominal = 1.25e12
    line = {
        "metric": "eigenmodes: block iterations/s", "value": iters / t, "unit": "iterations/s",
        "ms_per_iteration": 1e3 * t / iters, "n_modes": n_modes, "block_width": width, "iters": iters,
        "omega_top": [float(x) for x in om[:4]], "dtype": "f64", "data": "synthetic",
        "roofline": {"bound": "alu (fp64)", "achieved": flops / t / 1e12, "peak": fp64_nominal / 1e12,
                     "unit": "TFLOP/s", "frac": flops / t / fp64_nominal, "traffic": None,
                     "peak_kind": "nominal FP64 rate of GB300 (no measured FP64 peak)",
                     "what": "Gram matrix (upper triangle) and triangular block update, m (m+1) n_t flops each per iteration"},
        "config": {"workload": "scatterer-4M", "n_tris": m.n_tris},
    }
    m.close()
    print(json.dumps(line), flush=True)


def run_spectrum(args):
    """Both ends of the spectrum of a rectangular resonator of 101 x 70 lattice cells (Section 2,
    Fig. 4: the mesh's eigenvalues against the analytic ones), jittered and Delaunay-triangulated:
    the lowest modes from ue_modes_low (Chebyshev-filtered subspace iteration) against the
    analytic TE(m, n) frequencies pi sqrt((m/a)^2 + (n/b)^2), and the highest from ue_modes (the
    complex-time method with deflation), which set the stability bound of eq. 20."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_1812_01448_gb300 import build as b
    b.build()
    import paper_1812_01448_gb300 as ue
    import meshgen
    a_len, b_len = 1.01, 0.70
    ms = meshgen.cavity_lattice(102, 71, a_len, b_len, seed=1007)
    m = ue.Mesh(ms.xy, ms.tris)
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=1e-5)
    n_low = 16
    analytic = np.array(sorted(np.pi * np.hypot(i / a_len, j / b_len)
                               for i in range(40) for j in range(40) if i or j)[:n_low - 1])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    low = m.modes_low(n_low, iters=400, degree=32, seed=2)
    t_low = time.perf_counter() - t0
    t0 = time.perf_counter()
    top = m.modes(4, iters=3000, seed=2)
    t_top = time.perf_counter() - t0
    rel = low[1:] / analytic - 1.0
    line = {
        "metric": "resonator spectrum (Fig. 4): lowest and highest omegas", "unit": "rad/s (c = 1)",
        "value": float(low[1]), "dtype": "f64", "data": "synthetic",
        "omega_low": [float(x) for x in low], "omega_analytic": [0.0] + [float(x) for x in analytic],
        "rel_err_low": [float(x) for x in rel], "max_rel_err_low": float(np.abs(rel).max()),
        "omega_top": [float(x) for x in top], "dt_bound_eq20": 2.0 / float(top[0]),
        "seconds_low": t_low, "seconds_top": t_top,
        "config": {"workload": "resonator 1.01 x 0.70 (101 x 70 lattice cells, jitter 0.2h, Delaunay)",
                   "n_tris": m.n_tris, "n_low": n_low, "n_top": 4},
    }
    m.close()
    print(json.dumps(line), flush=True)


def run_relax(args):
    """Mesh optimisation (ue_mesh_relax: jello model, Section 3) on a Delaunay mesh of random
    points in the unit square: GPU time per relaxation step, the whole call with Lawson flips
    every 20 steps, and the spectral radius (hence dt, eq. 20) before and after, from the
    library's power iteration.  The oracle's relaxation, timed for 10 steps, is the CPU line."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_1812_01448_gb300 import build as b
    b.build()
    import paper_1812_01448_gb300 as ue
    import meshgen
    from oracle import relax as orelax
    ms = meshgen.random_delaunay(args.relax_points, seed=1006)
    iters = max(1, args.steps)
    ue.mesh_relax(ms.xy, ms.tris, max(3, args.warmup), flip_every=0)     # warm-up
    # per-step time without the call's fixed cost (host lists, allocation, transfers): the
    # difference between calls of N and N/2 steps (without flips, slivers would collapse over
    # much longer runs: the model needs its flips)
    half = max(1, iters // 2)
    t0 = time.perf_counter()
    ue.mesh_relax(ms.xy, ms.tris, half, flip_every=0)
    t_half = time.perf_counter() - t0
    t0 = time.perf_counter()
    ue.mesh_relax(ms.xy, ms.tris, iters, flip_every=0)
    t_call = time.perf_counter() - t0
    t_steps = (t_call - t_half) * iters / max(1, iters - half)
    t0 = time.perf_counter()
    xr, tr, flips = ue.mesh_relax(ms.xy, ms.tris, iters, flip_every=20)
    t_all = time.perf_counter() - t0
    rho = []
    for xy, tris in ((ms.xy, ms.tris), (xr, tr)):
        m = ue.Mesh(xy, tris)
        m.geometry_build()
        rho.append(m.get_dt()[1])
        m.close()
    t0 = time.perf_counter()
    orelax.relax(ms.xy, ms.tris, 10, flip_every=0)
    t_cpu = (time.perf_counter() - t0) / 10
    n_nodes = ms.xy.shape[0]
    line = {
        "metric": "mesh relaxation: node-steps/s", "value": n_nodes * iters / t_steps, "unit": "node-steps/s",
        "ms_per_step": 1e3 * t_steps / iters, "steps": iters, "call_seconds": t_call,
        "n_nodes": n_nodes, "n_tris": int(ms.tris.shape[0]),
        "with_flips": {"seconds": t_all, "flips": int(flips), "flip_every": 20},
        "rho_before": rho[0], "rho_after": rho[1], "dt_gain": rho[0] / rho[1],
        "dtype": "f64", "data": "synthetic",
        "cpu_baseline": {"value": n_nodes / t_cpu, "unit": "node-steps/s", "cores": 1, "kind": "oracle",
                         "sample": "10 relaxation steps of the same mesh (numpy, one thread)"},
        "config": {"workload": f"Delaunay mesh of {args.relax_points} uniform random points in the unit square, "
                               "jello-model relaxation, uniform target size"},
    }
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=8.0,
                    help="seconds of each CPU baseline sample (compiled oracle on one and on all "
                         "cores, numpy oracle)")
    ap.add_argument("--variant", choices=["plain", "blocked", "persistent"], default="blocked")
    ap.add_argument("--tile-tris", type=int, default=0,
                    help="largest tile (owned triangles); 0: 2500, and 2700 for the plasma workload, the "
                         "fastest measured for each")
    ap.add_argument("--frame", type=int, default=0,
                    help="scatterer workload: PML frame of this many cells (open boundary instead "
                         "of the PEC walls)")
    ap.add_argument("--tiler", choices=["kd", "greedy", "rings"], default="rings",
                    help="blocked variant: KD or greedy partition into tiles; rings: the greedy tiles "
                         "with each tile's boundary rings stored first, by angle")
    ap.add_argument("--block-depth", type=int, default=0,
                    help="steps per blocked launch (the tiles' halo depth); 0: 10 on scatterer-4M without a "
                         "frame, 8 otherwise (plasma tiles of 2700 and the frame region were measured at 8)")
    ap.add_argument("--graph-chunk", type=int, default=32)
    ap.add_argument("--tb-threads", type=int, default=0, choices=[0, 512, 1024])
    ap.add_argument("--e2e-fields", choices=["f32", "f64"], default="f32",
                    help="element type of the host field arrays of the end-to-end measurement")
    ap.add_argument("--tb-kernel", choices=["split", "fused"], default="split",
                    help="blocked variant: the split kernel (edges, then triangles) or the fused one")
    ap.add_argument("--workload", choices=["scatterer", "plasma", "cavity", "batch", "learned", "modes", "relax",
                                           "spectrum"],
                    default="scatterer",
                    help="scatterer: scatterer-4M (the default); plasma: plasma-1M (cold-plasma current); "
                         "cavity: the 1,024-triangle cavity in one CTA")
    ap.add_argument("--relax-points", type=int, default=100_000)
    ap.add_argument("--n-modes", type=int, default=8)
    ap.add_argument("--learned-meshes", type=int, default=40)
    ap.add_argument("--learned-max", type=int, default=1_000_000)
    ap.add_argument("--step-sweep", default="",
                    help="comma-separated step counts: time one ue_step_n call of each (after the warm-up) "
                         "and print that table instead of the bench line")
    ap.add_argument("--weights", default="", help="learned workload: a weight file other than the shipped one")
    ap.add_argument("--batch-meshes", type=int, default=512)
    ap.add_argument("--tune-sample", type=int, default=32)
    ap.add_argument("--quick-setup", action="store_true",
                    help="fixed dt instead of power iteration (for profiler runs)")
    args = ap.parse_args(argv)
    if args.tile_tris <= 0:
        args.tile_tris = 2700 if args.workload == "plasma" else 2500
    if args.block_depth <= 0:
        args.block_depth = 10 if args.workload == "scatterer" and args.frame == 0 else 8
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.frame > 0 and args.variant == "persistent":
        ap.error("--frame needs --variant plain or blocked")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "cavity":
        run_cavity(args)
    elif args.workload == "modes":
        run_modes(args)
    elif args.workload == "spectrum":
        run_spectrum(args)
    elif args.workload == "relax":
        run_relax(args)
    elif args.workload == "learned":
        run_learned(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
