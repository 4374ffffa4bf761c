#!/usr/bin/env python
"""Benchmark of the fused Simulation -> Hierarchy-Scan -> Bind MeshPose frame.

One step = one full frame of the 4,096 x 512-joint + 1,024-joint-dragon
workload (2,098,176 joints): per-character key sampling, slerp/lerp between
keys and between two clips, the Hierarchy-Scan and the bind product, as the
library's launches (the work queue, then the frame kernels) replayed from CUDA
graphs of four consecutive frames.  The output rotates over enough buffers
that consecutive steps touch more memory than the 129 MB L2 (inputs larger
than L2).

Printed (rank 0, one JSON line): joints/s of the whole job, the roofline of
the frame kernels (algorithmic bytes / CUDA-event duration against the
measured HBM copy bandwidth), the end-to-end rate through the public API
with host buffers, the plain level-synchronous kernel on the same frame, the
fused forward+adjoint (loss_backward) on the 1,024 x 256-joint workload, the
FP64 oracle on the host cores, and SM clocks sampled during the timed loop.

--impl reference times the FP64 CPU oracle on the host cores, one full frame
of the same workload per step.

Multi-GPU: characters are independent, so each rank runs its own batch of
the same size (weak scaling, no data-path collective); the timing is the
maximum over ranks.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import re
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "joint transforms/s fwd and fwd+bwd on 1 GB300, % of HBM roofline, vs plain kernel"
# The frame both arms time, named the same way in both JSON lines.
WORKLOAD = "frame: 4,096 x 512-joint biped (depth 70) + 1 x 1,024-joint dragon chain, 2 clips x 30 keys"
UNIT = "joints/s"
L2_BYTES = 129 * 1024 * 1024
FRAMES_PER_GRAPH = 4  # frames per captured CUDA graph in the timed frame loop
# DRAM bytes per launch of the frame's dominant kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by the hash of the
# kernel sources it was taken on (comments and whitespace aside); reported
# as null once the code changes.  Current: k_walk2 on the 4,096 bipeds.
NCU_TRAFFIC = {"9d28c9fadbd4aae7": 2654464 + 42383616}


# ------------------------------------------------------------------ helpers
# The sources the persistent frame kernel is compiled and launched from.
FRAME_KERNEL_SOURCES = ("anim_internal.h", "dev_math.cuh", "scan_core.cuh", "k_scan_qt.cu", "k_walk.cu", "k_walk2.cu",
                        "smem_limit.h", "host.cu")


def kernel_source_hash() -> str:
    """Hash of the frame kernel's sources with comments and whitespace
    removed, so that only a change of its code voids a stored ncu capture."""
    h = hashlib.sha256()
    for name in FRAME_KERNEL_SOURCES:
        f = os.path.join(ROOT, "paper_2505_06703_gb300", "csrc", name)
        with open(f, encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(os.path.basename(f).encode())
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def frame_algorithmic_bytes(w: dict) -> int:
    """Compulsory unique bytes of one frame: the skin matrices written (48 B
    per joint), each used type's tables read once (keys: 28 B of q and t per
    key record, inverse binds 48 B and parents 4 B per joint) and 12 B per
    character (time, blend weight, type id)."""
    types = w["types"]
    ct = w["char_type"]
    joints = sum(len(types[t]["parents"]) for t in ct)
    tables = 0
    for t in sorted(set(int(x) for x in ct)):
        ty = types[t]
        n = len(ty["parents"])
        nc, nk = ty["keys"].shape[:2]
        tables += nc * nk * n * 28 + n * 48 + n * 4
    return joints * 48 + tables + len(ct) * 12


def frame_touched_bytes(w: dict) -> int:
    """Bytes one frame would move if nothing were cached or shared, as
    context for the algorithmic bytes: per joint four 32-byte key records,
    the 48-byte inverse bind, a 4-byte table entry and the 48-byte output."""
    types = w["types"]
    return sum(len(types[t]["parents"]) for t in w["char_type"]) * (4 * 32 + 48 + 4 + 48)


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal


def add_nominal_fractions(obj) -> None:
    """Beside each HBM roofline's fraction of the measured peak, its fraction
    of the nominal 7.9 TB/s."""
    if isinstance(obj, dict):
        rf = obj.get("roofline")
        if isinstance(rf, dict) and rf.get("unit") == "GB/s" and "achieved" in rf:
            rf.setdefault("nominal_peak", NOMINAL_HBM_GBS)
            rf.setdefault("frac_of_nominal", round(rf["achieved"] / NOMINAL_HBM_GBS, 4))
        for v in obj.values():
            add_nominal_fractions(v)


def fwd_bwd_algorithmic_bytes(w: dict) -> int:
    """loss_backward: read q (16 B), t (12 B), target (12 B) and write dq
    (16 B), dt (12 B) per joint, plus the type's parent table."""
    types = w["types"]
    joints = len(w["q"])
    return joints * 68 + sum(len(t["parents"]) * 4 for t in types)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_workload(rank: int) -> dict:
    """The same skeletons and clips on every rank; each rank's characters get
    their own times and blend weights (an independent batch)."""
    w = synth.config2()
    if rank:
        rng = np.random.default_rng(1000 + rank)
        n = len(w["char_type"])
        w["time"] = rng.uniform(0.0, 1.0, n).astype(np.float32)
        w["weight"] = rng.uniform(0.0, 1.0, n).astype(np.float32)
    return w


def aggregate_max(x: float, world: int) -> float:
    """Maximum over ranks (timing only; no data crosses ranks)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except OSError:
            pass
        finally:
            if self.path:
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ our arm
def setup_ctx(w: dict, device: int):
    import paper_2505_06703_gb300 as pk
    ctx = pk.Context(device)
    types = w["types"]
    ids = ctx.create_skeletons([t["parents"] for t in types], rest_q=[t["rest_q"] for t in types],
                               rest_t=[t["rest_t"] for t in types])
    for i, t in zip(ids, types):
        if "keys" in t:
            ctx.upload_clips(i, t["keys"], t["rate_hz"])
    plan = ctx.plan(np.asarray(ids, np.int32)[w["char_type"]])
    return ctx, plan


def set_or_tune(ctx, plan, schedule, which: int):
    """Apply a given schedule, else run the library's autotuner (anim_tune
    mode `which`) for this workload."""
    if schedule:
        ctx.set_schedule(plan, schedule)
    else:
        ctx.tune(plan, which)


def time_events(fn, steps: int, warmup: int):
    """Run fn(s) warmup + steps times on the current stream; return the
    CUDA-event milliseconds of the timed steps (synchronized on both sides)."""
    import torch
    for s in range(warmup):
        fn(s)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for s in range(steps):
        fn(warmup + s)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_ours(args) -> dict:
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"

    w = rank_workload(rank)
    ctx, plan = setup_ctx(w, local)
    if args.schedule:
        ctx.set_schedule(plan, [int(x) for x in args.schedule.split(",")])
    else:
        ctx.tune(plan, 0)  # the library's autotuner picks the schedule for this mix
    schedule = ctx.get_schedule(plan)
    joints = plan.total
    n_chars = plan.n_chars
    out_bytes = joints * 48
    n_out = max(3, math.ceil(2.5 * L2_BYTES / out_bytes))
    outs = [torch.empty((joints, 12), dtype=torch.float32, device=dev) for _ in range(n_out)]
    # per-step inputs: times advance by 1/60 s per frame
    n_in = 6
    times = [torch.as_tensor(np.mod(w["time"] + k / 60.0, 1.0).astype(np.float32), device=dev) for k in range(n_in)]
    blend = torch.as_tensor(w["weight"], device=dev)

    # frames captured FRAMES_PER_GRAPH at a time (each frame its own work
    # queue + frame kernels, on its own times and output buffer), as a render
    # loop would submit them; single-frame graphs for the remainder, so that
    # exactly `steps` frames are timed
    n_frames = n_out * n_in // math.gcd(n_out, n_in)
    n_frames = FRAMES_PER_GRAPH * math.ceil(n_frames / FRAMES_PER_GRAPH)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for i in range(n_frames):  # warm once outside capture (sets kernel attributes)
            ctx.evaluate_frame(plan, times[i % n_in], blend, out=outs[i % n_out])
    stream.synchronize()

    def capture(first, count):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for i in range(first, first + count):
                ctx.evaluate_frame(plan, times[i % n_in], blend, out=outs[i % n_out])
        return g

    graphs = [capture(i, FRAMES_PER_GRAPH) for i in range(0, n_frames, FRAMES_PER_GRAPH)]
    singles = [capture(i, 1) for i in range(n_frames)]
    n_graph = len(graphs)
    torch.cuda.synchronize()

    steps, warmup = args.steps, args.warmup
    for s in range(warmup):
        singles[s % n_frames].replay()
    torch.cuda.synchronize()
    barrier(world)
    def load_for(seconds):
        t0 = time.perf_counter()
        k = 0
        while time.perf_counter() - t0 < seconds:
            for _ in range(16):
                graphs[k % n_graph].replay()
                k += 1
            torch.cuda.synchronize()

    # clocks are sampled over continuous load: ~0.7 s before, the timed
    # steps, ~0.7 s after (the sampler's period is 200 ms)
    with ClockSampler(local) as clocks:
        load_for(0.7)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for s in range(steps // FRAMES_PER_GRAPH):
            graphs[s % n_graph].replay()
        for s in range(steps % FRAMES_PER_GRAPH):
            singles[s % n_frames].replay()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        load_for(0.7)
    barrier(world)
    ms_max = aggregate_max(ms, world)
    ms_step = ms_max / steps
    value = world * joints / (ms_step / 1e3)
    clock = clocks.summary()

    # the frame kernels alone (the work queue built once and reused): one
    # CUDA graph of frame-kernel launches back to back, one per output
    # buffer, CUDA events around its replays on the launching stream
    with torch.cuda.stream(stream):
        ctx.frame_build_queue(plan, times[0])
    stream.synchronize()
    kg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(kg, stream=stream):
        for o in outs:
            ctx.frame_run_queue(plan, times[0], blend, o)
    k_reps = max(2, math.ceil(steps / n_out))
    with torch.cuda.stream(stream):
        k_ms = time_events(lambda s: kg.replay(), k_reps, max(3, warmup)) / (k_reps * n_out)
    alg = frame_algorithmic_bytes(w)
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    achieved = alg / (k_ms / 1e3) / 1e9
    tr = NCU_TRAFFIC.get(kernel_source_hash())
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": tr,
                "kernel": {0: "k_scan_qt<0> (persistent frame)", 1: "k_walk (chain walk in skin space)",
                           2: "k_walk2 (warp-specialized chain walk in skin space)"}[schedule[3]],
                "kernel_ms": round(k_ms, 5), "algorithmic_bytes": alg, "peak_source": peak_src,
                "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                "touched_bytes": frame_touched_bytes(w)}

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warmup,
              "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
              "dtype": "f32", "data": "synthetic (seeded skeletons, clips, times and blend weights)",
              "config": {"workload": WORKLOAD,
                         "steps_of_the_frame": "slerp keys, slerp 2-clip blend, hierarchy scan, bind",
                         "joints_per_step_per_gpu": joints, "characters_per_gpu": n_chars,
                         "l2": f"output rotated over {n_out} buffers ({n_out * out_bytes / 1e6:.0f} MB > 129 MB L2)",
                         "timing": f"CUDA graphs of {FRAMES_PER_GRAPH} consecutive frames (each frame: work queue + frame "
                                   "kernels, its own times and output buffer) replayed back to back, CUDA events; the "
                                   "roofline's kernel time from one graph of frame-kernel launches back to back",
                         "schedule": {"seg_len,ctas_per_sm,joints_per_item,walk,adj_ctas": schedule,
                                      "source": "--schedule" if args.schedule else "anim_tune"},
                         "parallelism": f"replicas x{world} (independent character batches)"},
              # per frame: the work queue, the frame kernel, and with a chain-walk
              # schedule the segmented kernel beside it (the dragon chain is never walked)
              "roofline": roofline, "gpu_launches": (3 if schedule[3] else 2) * steps, "clocks": clock}

    # end to end through the C-ABI call with host buffers
    # (anim_evaluate_frame_host): page-locked inputs copied in and the whole
    # skin output copied back inside the call, every step
    if True:
        h_times = [t.cpu().pin_memory() for t in times]
        h_blend = blend.cpu().pin_memory()
        h_out = torch.empty((joints, 12), dtype=torch.float32).pin_memory()
        ctx.evaluate_frame_host(plan, h_times[0], h_blend, out=h_out)  # allocates the plan's staging
        torch.cuda.synchronize()

        def e2e_step(s):
            ctx.evaluate_frame_host(plan, h_times[s % n_in], h_blend, out=h_out)

        e_steps = max(3, min(steps, 20))
        e_ms = aggregate_max(time_events(e2e_step, e_steps, 2), world)
        result["e2e"] = {"value": world * joints / (e_ms / e_steps / 1e3), "unit": UNIT,
                         "h2d_bytes_per_step": int(h_times[0].numel() * 4 + h_blend.numel() * 4),
                         "d2h_bytes_per_step": int(h_out.numel() * 4), "ms_per_step": e_ms / e_steps,
                         "call": "anim_evaluate_frame_host"}

    if not args.no_extras:
        # plain level-synchronous kernel on the same frame
        def plain_step(s):
            ctx.evaluate_frame(plan, times[s % n_in], blend, out=outs[s % n_out], levelsync=True)

        p_steps = max(3, min(steps, 20))
        p_ms = aggregate_max(time_events(plain_step, p_steps, 2), world)
        result["plain"] = {"value": world * joints / (p_ms / p_steps / 1e3), "unit": UNIT,
                           "ms_per_step": p_ms / p_steps, "kernel": "k_levelsync (1 CTA/char, barrier per level)",
                           "speedup_fused_vs_plain": (p_ms / p_steps) / ms_step}
        result["fwd_bwd"] = run_fwd_bwd(ctx_factory=setup_ctx, device=local, dev=dev, steps=steps,
                                        warmup=warmup, world=world, peak=peak, schedule=args.schedule_bwd)
        if not args.schedule:  # the extra workloads run the autotuner
            result["frame_mixed"] = run_mixed_frame(local, dev, world, peak)
            result["ik"] = run_ik(local, dev, world, peak)
            result["frame_skinned"] = run_skinned_frame(local, dev, world, peak)
            result["frame_layers"] = run_layered_frame(local, dev, world, peak)
            result["crowd_raster"] = run_crowd(local, dev, world)
            cmp_ = time_forward_methods(rank_workload(rank), local, dev, world)
            result["scan_comparison"] = {
                "workload": "forward from local poses (scan + bind) on the frame's 2,098,176 joints",
                "ms_per_launch": {k: v for k, v in cmp_.items() if k != "schedule"},
                "speedup_ours_vs": {k: v / cmp_["ours"] for k, v in cmp_.items() if k not in ("schedule", "ours")},
                "schedule": cmp_["schedule"]}
    del ctx
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return result


def run_mixed_frame(device, dev, world, peak, schedule=None, workload=None) -> dict:
    """Batched heterogeneous frame (10,000 characters of 5 types, 32 to 2,048
    joints, depths 8 to 2,048): the autotuned schedule, frames replayed from
    one CUDA graph with outputs rotated over buffers larger than L2."""
    import torch
    w = workload if workload is not None else synth.config3()
    ctx, plan = setup_ctx(w, device)
    set_or_tune(ctx, plan, schedule, 0)
    joints = plan.total
    n_out = max(2, math.ceil(2.5 * L2_BYTES / (joints * 48)))
    outs = [torch.empty((joints, 12), dtype=torch.float32, device=dev) for _ in range(n_out)]
    tm = torch.as_tensor(w["time"], device=dev)
    bw = torch.as_tensor(w["weight"], device=dev)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for o in outs:
            ctx.evaluate_frame(plan, tm, bw, out=o)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        for o in outs:
            ctx.evaluate_frame(plan, tm, bw, out=o)
    torch.cuda.synchronize()
    reps = 5
    ms = aggregate_max(time_events(lambda s: graph.replay(), reps, 2), world)
    ms_step = ms / (reps * n_out)
    alg = frame_algorithmic_bytes(w)
    achieved = alg / (ms_step / 1e3) / 1e9
    return {"value": world * joints / (ms_step / 1e3), "unit": UNIT, "ms_per_step": ms_step, "joints": joints,
            "workload": "frame: 10,000 chars of 32/128/512/1,024/2,048-joint types (depths 8/16/70/256/2,048) "
                        "at 40/30/15/10/5 %, shuffled",
            "schedule": ctx.get_schedule(plan),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "algorithmic_bytes": alg,
                         "note": "whole frame (work queue + kernels), frames back to back in one CUDA graph"}}


def run_mixed_split(device, dev, world, peak, schedule=None) -> dict:
    """The heterogeneous frame (config 3) type by type: the frame restricted
    to each type's characters, under the schedule the autotuner picks for the
    whole mix (or the given one), timed like run_mixed_frame; beside the whole
    mix.  Shows where the mixed frame's time goes."""
    import torch
    w = synth.config3()
    ctx, plan = setup_ctx(w, device)
    set_or_tune(ctx, plan, schedule, 0)
    sched = ctx.get_schedule(plan)
    out = {"schedule": sched, "types": []}
    for ty in list(range(len(w["types"]))) + [None]:
        chars = np.nonzero(w["char_type"] == ty)[0] if ty is not None else np.arange(len(w["char_type"]))
        ws = synth.subset(w, chars)
        r = run_mixed_frame(device, dev, world, peak, schedule=sched, workload=ws)
        ent = {"ms_per_step": r["ms_per_step"], "joints": int(r["joints"]), "frac": r["roofline"]["frac"]}
        if ty is None:
            out["whole_mix"] = ent
        else:
            ty_d = w["types"][ty]
            ent.update({"type_joints": len(ty_d["parents"]), "depth": int(ty_d["depth"]), "characters": len(chars)})
            out["types"].append(ent)
    return out


def run_skinned_frame(device, dev, world, peak, schedule=None) -> dict:
    """The frame with linear blend skinning fused in: the frame's characters
    with a 1,500-vertex mesh per type (about 3,000 faces), positions and
    normals written, skin matrices kept on chip; frames back to back in one
    CUDA graph, vertex buffers rotated past the L2 size."""
    import torch
    w = synth.with_meshes(synth.config2(), n_verts=1500)
    ctx, plan = setup_ctx(w, device)
    for i, t in enumerate(w["types"]):
        ctx.upload_mesh(i, t["mesh"])
    set_or_tune(ctx, plan, schedule, 3)  # the skinned frame's own schedule
    nv = int(ctx.vertex_offsets(plan)[-1])
    n_out = max(2, math.ceil(2.5 * L2_BYTES / (nv * 24)))
    outs = [torch.empty((nv, 6), dtype=torch.float32, device=dev) for _ in range(n_out)]
    tm = torch.as_tensor(w["time"], device=dev)
    bw = torch.as_tensor(w["weight"], device=dev)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for o in outs:
            ctx.evaluate_frame_skinned(plan, tm, bw, verts=o)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        for o in outs:
            ctx.evaluate_frame_skinned(plan, tm, bw, verts=o)
    torch.cuda.synchronize()
    reps = 5
    ms = aggregate_max(time_events(lambda s: graph.replay(), reps, 2), world)
    ms_step = ms / (reps * n_out)
    # vertices out (24 B), mesh records read once per type (48 B per vertex),
    # the frame's tables and per-character inputs; no skin matrices written
    alg = nv * 24 + sum(len(t["mesh"]["pos"]) * 48 for t in w["types"]) + \
        frame_algorithmic_bytes(w) - plan.total * 48
    achieved = alg / (ms_step / 1e3) / 1e9
    return {"value": world * nv / (ms_step / 1e3), "unit": "skinned vertices/s", "ms_per_step": ms_step,
            "joints_per_s": world * plan.total / (ms_step / 1e3), "vertices": nv,
            "workload": "frame + linear blend skinning: the frame's 4,097 characters, 1,500-vertex mesh per type, "
                        "4 bones per vertex, positions + normals out, skin matrices not written",
            "schedule": ctx.get_schedule(plan),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "algorithmic_bytes": alg}}


def run_layered_frame(device, dev, world, peak, schedule=None) -> dict:
    """The frame with layered blending: the frame's characters with 4 clips
    per type blended by per-character weights plus an additive layer;
    frames back to back in one CUDA graph, outputs rotated past L2."""
    import torch
    w = synth.with_layers(synth.config2(), n_clips=4)
    ctx, plan = setup_ctx(w, device)
    for i, t in enumerate(w["types"]):
        ctx.upload_additive(i, t["add_keys"], t["rate_hz"])
    set_or_tune(ctx, plan, schedule, 4)  # the layered frame's own schedule
    joints = plan.total
    n_out = max(2, math.ceil(2.5 * L2_BYTES / (joints * 48)))
    outs = [torch.empty((joints, 12), dtype=torch.float32, device=dev) for _ in range(n_out)]
    tm = torch.as_tensor(w["time"], device=dev)
    wts = torch.as_tensor(w["weights"], device=dev)
    aw = torch.as_tensor(w["add_w"], device=dev)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for o in outs:
            ctx.evaluate_frame_layers(plan, tm, wts, aw, out=o)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        for o in outs:
            ctx.evaluate_frame_layers(plan, tm, wts, aw, out=o)
    torch.cuda.synchronize()
    reps = 5
    ms = aggregate_max(time_events(lambda s: graph.replay(), reps, 2), world)
    ms_step = ms / (reps * n_out)
    # skin out, 4 clips + the additive layer of keys once, 28 B per character
    alg = frame_algorithmic_bytes(w) + sum(len(t["parents"]) * t["add_keys"].shape[0] * 28 for t in w["types"]) + \
        len(w["char_type"]) * 16
    achieved = alg / (ms_step / 1e3) / 1e9
    return {"value": world * joints / (ms_step / 1e3), "unit": UNIT, "ms_per_step": ms_step,
            "workload": "frame with 4 clips per type blended by per-character weights (incremental slerp) "
                        "+ an additive layer; the frame's 4,097 characters",
            "schedule": ctx.get_schedule(plan),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "algorithmic_bytes": alg}}


def run_crowd(device, dev, world) -> dict:
    """The whole picture per frame: the frame's 4,097 characters sampled,
    scanned, bound and skinned (1,500 vertices, about 1,500 triangles each),
    then rasterized headless at 1920x1080 (64 characters per grid row) into an
    RGBA buffer; frames back to back in one CUDA graph."""
    import torch
    w = synth.with_meshes(synth.config2(), n_verts=1500)
    ctx, plan = setup_ctx(w, device)
    for i, t in enumerate(w["types"]):
        ctx.upload_mesh(i, t["mesh"])
        ctx.upload_faces(i, t["mesh"]["faces"])
    ctx.tune(plan, 3)  # the skinned frame's schedule
    nv = int(ctx.vertex_offsets(plan)[-1])
    tris = sum(len(w["types"][int(t)]["mesh"]["faces"]) for t in w["char_type"])
    verts = torch.empty((nv, 6), dtype=torch.float32, device=dev)
    W, H, cols = 1920, 1080, 64
    vis = torch.empty((H, W), dtype=torch.int64, device=dev)
    rgba = torch.empty((H, W), dtype=torch.int32, device=dev)
    tm = torch.as_tensor(w["time"], device=dev)
    bw = torch.as_tensor(w["weight"], device=dev)
    scale, spacing = 11.0, 2.6

    def frame():
        ctx.evaluate_frame_skinned(plan, tm, bw, verts=verts)
        ctx.raster(plan, verts, W, H, cols, spacing, 15.0, 15.0, scale, ids=False, rgba=rgba, vis=vis)

    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        frame()
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        for _ in range(4):
            frame()
    torch.cuda.synchronize()
    reps = 5
    ms = aggregate_max(time_events(lambda s: graph.replay(), reps, 2), world) / (reps * 4)
    covered = int((rgba != 0xFF201810 - (1 << 32)).sum())
    return {"frames_per_s": world / (ms / 1e3), "ms_per_step": ms, "triangles": tris,
            "triangles_per_s": world * tris / (ms / 1e3), "image": f"{W}x{H} RGBA8", "covered_pixels": covered,
            "workload": "frame + skinning + headless raster of 4,097 characters (1,500 vertices, ~1,500 "
                        "triangles each) at 1920x1080", "schedule": ctx.get_schedule(plan)}


def run_ik(device, dev, world, peak, schedule=None) -> dict:
    """Batched IK (8,192 characters, 128- and 1,024-joint types, 8 effectors
    each): 200 Adam steps, each one fused launch (forward over the effector
    ancestors, effector loss, adjoint, Adam), the whole run one CUDA graph.
    The final effector error is the GPU run's own distance to its targets;
    the agreement with the FP64 run of the same schedule is a parity test."""
    import torch
    w = synth.config5()
    ctx, plan = setup_ctx(w, device)
    types, ct, eff = w["types"], np.asarray(w["char_type"]), np.asarray(w["effectors"])
    t = torch.as_tensor(w["t"], device=dev)
    _, mt = ctx.forward_local(plan, torch.as_tensor(w["q_target"], device=dev), t, skin=False, model=True)
    mt = mt.view(-1, 3, 4)[:, :, 3]
    off = torch.as_tensor(plan.row_off[:-1], device=dev)
    eff_t = torch.as_tensor(eff, device=dev).long()[torch.as_tensor(ct, device=dev).long()]
    targets = mt[off[:, None] + eff_t].contiguous()
    active = 0  # joints the step touches: the effectors' ancestors
    for ty in range(len(types)):
        par, act = types[ty]["parents"], set()
        for j in eff[ty]:
            a = int(j)
            while a >= 0 and a not in act:
                act.add(a)
                a = int(par[a])
        active += len(act) * int(np.sum(ct == ty))
    q0 = torch.as_tensor(w["q0"], device=dev)
    q = q0.clone()
    loss = torch.zeros(plan.n_chars, device=dev)
    if schedule:
        ctx.set_schedule(plan, schedule)
    else:
        ctx.tune_ik(plan, eff)  # the IK step's schedule; the IK object keeps it
    ik = ctx.ik(plan, eff)
    n_steps = int(w["n_steps"])
    stream = torch.cuda.Stream()

    def run_all():
        ik.reset()  # step counter and the object's own Adam state
        q.copy_(q0)
        for _ in range(n_steps):
            ik.step(q, None, None, t, targets, lr=w["lr"], betas=w["betas"], eps=w["eps"], loss=loss)

    with torch.cuda.stream(stream):
        run_all()  # warm outside capture (kernel attributes)
    stream.synchronize()

    def eff_err():
        _, mq = ctx.forward_local(plan, q, t, skin=False, model=True)
        pe = mq.view(-1, 3, 4)[:, :, 3][off[:, None] + eff_t]
        d = torch.linalg.norm(pe - targets, dim=-1)
        return float(d.mean()), float(d.max())

    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        run_all()
    torch.cuda.synchronize()
    reps = 3
    ms = aggregate_max(time_events(lambda s: graph.replay(), reps, 1), world)
    ms_step = ms / (reps * n_steps)
    e_mean, e_max = eff_err()
    q_final = q.cpu().numpy()  # the final pose of the timed run, for the FP64 comparison
    q.copy_(q0)
    e0_mean, _ = eff_err()
    alg = active * 108 + plan.n_chars * eff.shape[1] * 12
    achieved = alg / (ms_step / 1e3) / 1e9
    return {"steps_per_s": world / (ms_step / 1e3), "active_joints_per_s": world * active / (ms_step / 1e3),
            "ms_per_step": ms_step, "steps": n_steps, "active_joints": active, "characters": plan.n_chars,
            "workload": "IK: 4,096 x 128-joint (depth 16) + 4,096 x 1,024-joint (depth 256) chars, 8 effectors "
                        "each, 200 Adam steps (lr 1e-2)",
            "schedule": ctx.get_schedule(plan),
            "adam_state": "the IK object's own (active joints only, contiguous)",
            "effector_error": {"start_mean": e0_mean, "final_mean": e_mean, "final_max": e_max,
                               "note": "distance to targets (skeletons of unit extent)"},
            "_q_final": q_final,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "algorithmic_bytes_per_step": alg,
                         "note": "108 B per active joint (q, t, m, v in; q, m, v out) + targets"}}


def time_forward_methods(w: dict, device: int, dev: str, world: int, algs=(1, 2, 3, 4, 5), schedule=None) -> dict:
    """Hierarchy-Scan + bind from given local poses on workload w: our
    autotuned forward kernel, the plain level-synchronous kernel and the
    paper's Algorithms 1-4 (one CTA per character, one thread per joint), each
    as back-to-back launches in one CUDA graph over output buffers rotated
    past the L2 size.  Milliseconds per launch."""
    import torch
    ctx, plan = setup_ctx(w, device)
    set_or_tune(ctx, plan, schedule, 1)
    q, t = synth.local_poses(np.random.default_rng(7), plan.total, t_half=0.0005)
    q, t = torch.as_tensor(q, device=dev), torch.as_tensor(t, device=dev)
    n_out = max(2, math.ceil(2.5 * L2_BYTES / (plan.total * 48)))
    outs = [torch.empty((plan.total, 12), dtype=torch.float32, device=dev) for _ in range(n_out)]
    methods = {"ours": lambda o: ctx.forward_local(plan, q, t, skin=True),
               "levelsync": lambda o: ctx.forward_local(plan, q, t, levelsync=True)}
    for a in algs:
        name = f"paper_alg{a}" if a <= 4 else "leaf_walk"
        methods[name] = (lambda a: lambda o: ctx.forward_local_paper(plan, a, q, t, out=o))(a)
    res = {}
    for name, fn in methods.items():
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            for o in outs:
                fn(o)
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            for o in outs:
                fn(o)
        torch.cuda.synchronize()
        reps = 3
        res[name] = aggregate_max(time_events(lambda s: graph.replay(), reps, 1), world) / (reps * n_out)
    res["schedule"] = ctx.get_schedule(plan)
    return res


def run_paper_sweep(args) -> dict:
    """The paper's experiment shape (Sec. 4, Fig. 7): 10,000 characters of
    about 300 joints, the tree depth swept from 15 to 120 levels; per depth
    four seeded random 300-joint trees (a spine of that depth, the other
    joints on uniform earlier parents), 2,500 characters each.  Our forward
    kernel against the plain kernel and the paper's Algorithms 1-4."""
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    rows = []
    for depth in (15, 30, 60, 90, 120):
        rng = np.random.default_rng(1000 + depth)
        types = [synth.make_type(synth.relabel_dfs(synth.random_tree(300, depth, rng, spine=depth), rng)[0], rng,
                                 with_clips=False) for _ in range(4)]
        ct = np.repeat(np.arange(4, dtype=np.int32), 2500)
        rng.shuffle(ct)
        r = time_forward_methods({"types": types, "char_type": ct}, local, dev, world)
        joints = 10000 * 300
        rows.append({"depth": depth, "ms": {k: v for k, v in r.items() if k != "schedule"},
                     "g_joints_per_s": {k: joints / (v / 1e3) / 1e9 for k, v in r.items() if k != "schedule"},
                     "schedule": r["schedule"]})
    return {"metric": "Hierarchy-Scan + bind from local poses, ms per batch of 10,000 x 300-joint characters",
            "impl": "ours", "n_gpus": world, "sweep": rows,
            "config": {"workload": "depth sweep 15-120, 4 random 300-joint trees x 2,500 characters per depth",
                       "timing": "CUDA graphs, outputs rotated past L2, CUDA events"}}


def run_fwd_bwd(ctx_factory, device, dev, steps, warmup, world, peak, schedule=None):
    """Fused forward + adjoint (anim_loss_backward) on 1,024 characters of the
    256-joint type: read q, t, target; write dq, dt (and per-character loss)."""
    import torch
    w = synth.config4()
    ctx, plan = ctx_factory(w, device)
    if schedule:
        ctx.set_schedule(plan, [int(x) for x in schedule.split(",")])
    else:
        ctx.tune(plan, 2)
    joints = plan.total
    n_sets = max(2, math.ceil(2.5 * L2_BYTES / (joints * 68)))
    sets = []
    for k in range(n_sets):
        q = torch.as_tensor(w["q"], device=dev) * (1.0 + 0.01 * k)
        sets.append((q.contiguous(), torch.as_tensor(w["t"], device=dev), torch.as_tensor(w["target"], device=dev),
                     torch.empty((joints, 4), device=dev), torch.empty((joints, 3), device=dev),
                     torch.empty(plan.n_chars, device=dev)))

    # one CUDA graph holding one adjoint launch per input/output set, in
    # sequence (inputs cold in L2 at every launch); the timed region holds
    # GPU work only, not Python launch overhead
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for q, t, tg, gq, gt, loss in sets:  # warm outside capture (kernel attributes)
            ctx.loss_backward(plan, q, t, tg, grad_q=gq, grad_t=gt, loss=loss)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        for q, t, tg, gq, gt, loss in sets:
            ctx.loss_backward(plan, q, t, tg, grad_q=gq, grad_t=gt, loss=loss)
    torch.cuda.synchronize()
    reps = max(1, math.ceil(steps / n_sets))

    def step(s):
        graph.replay()

    ms = aggregate_max(time_events(step, reps, max(1, warmup // n_sets)), world)
    ms_step = ms / (reps * n_sets)
    alg = fwd_bwd_algorithmic_bytes(w)
    achieved = alg / (ms_step / 1e3) / 1e9
    return {"value": world * joints / (ms_step / 1e3), "unit": UNIT, "ms_per_step": ms_step,
            "launches_timed": reps * n_sets,
            "schedule": ctx.get_schedule(plan),
            "workload": "1,024 chars x 256-joint tree (depth 96), loss sum |p - target|^2",
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "algorithmic_bytes": alg,
                         "note": "adjoint launches back to back in one CUDA graph, one per rotated set"},
            "l2": f"inputs/outputs rotated over {n_sets} sets ({n_sets * joints * 68 / 1e6:.0f} MB)"}


def cpu_model() -> str:
    """The host CPU's model name (or, on Arm, implementer and part codes)."""
    import platform
    try:
        with open("/proc/cpuinfo") as f:
            txt = f.read()
    except OSError:
        return platform.machine()
    m = re.search(r"^model name\s*:\s*(.+)$", txt, re.M)
    if m:
        return m.group(1).strip()
    imp = re.search(r"^CPU implementer\s*:\s*(\S+)", txt, re.M)
    part = re.search(r"^CPU part\s*:\s*(\S+)", txt, re.M)
    if imp and part:
        return f"{platform.machine()} (implementer {imp.group(1)}, part {part.group(1)})"
    return platform.machine()


def host_cores() -> int:
    """Cores this process may run on (its affinity mask where the OS has one)."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _oracle_share(share: int, n_shares: int, warm: int, reps: int, ready, start, out) -> None:
    """One process of the all-cores oracle timing: its contiguous share of the
    frame's characters, `warm` untimed frames, then `reps` timed ones after the
    parent's start signal; reports its elapsed seconds."""
    import oracle
    w = synth.config2()
    idx = np.array_split(np.arange(len(w["char_type"])), n_shares)[share]
    ws = synth.subset(w, idx)
    for _ in range(max(1, warm)):
        oracle.frame(ws)
    ready.put(share)
    if not start.wait(300):
        out.put(-1.0)
        return
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.frame(ws)
    out.put(time.perf_counter() - t0)


def oracle_all_cores(reps: int, warm: int = 1, workers: int | None = None) -> tuple[float, int]:
    """The FP64 oracle as it stands on every host core: the frame's characters
    split into one share per process (spawned, so no process forks after CUDA
    has started), all shares run `reps` frames at once; returns (wall seconds
    from the start signal to the last share's end, processes)."""
    import multiprocessing as mp
    n = workers or host_cores()
    ctx = mp.get_context("spawn")
    ready, out, start = ctx.Queue(), ctx.Queue(), ctx.Event()
    procs = [ctx.Process(target=_oracle_share, args=(i, n, warm, reps, ready, start, out)) for i in range(n)]
    for p in procs:
        p.start()
    def collect(q, count, what):
        got, t_end = [], time.monotonic() + 600
        while len(got) < count:
            try:
                got.append(q.get(timeout=1.0))
            except Exception:  # queue.Empty: check that the processes still run
                if any(p.exitcode not in (None, 0) for p in procs) or time.monotonic() > t_end:
                    raise RuntimeError(f"oracle processes failed while {what}")
        return got

    try:
        collect(ready, n, "preparing their shares")
        t0 = time.perf_counter()
        start.set()
        times = collect(out, n, "timing")
        dt = time.perf_counter() - t0
    finally:
        start.set()
        for p in procs:
            p.join(60)
            if p.is_alive():
                p.terminate()
    if min(times) < 0:
        raise RuntimeError("an oracle process did not start")
    return dt, n


def ik_vs_oracle(q_gpu) -> dict:
    """The FP64 oracle's run of the same IK schedule (config 5: 8,192
    characters, 200 Adam steps, every host core) and the agreement of the
    GPU run's final effector positions with it (each side with its own
    targets); also the oracle's rate on this workload."""
    import oracle
    w = synth.config5()
    types, ct, eff = w["types"], w["char_type"], w["effectors"]
    tg = oracle.ik_targets(w)
    t0 = time.perf_counter()
    q_ref, _, procs = oracle.ik_all_cores(types, ct, w["t"], w["q0"], eff, tg, int(w["n_steps"]), lr=w["lr"],
                                          betas=w["betas"], eps=w["eps"])
    dt = time.perf_counter() - t0
    off = oracle.offsets(ct, types)
    rows = (off[:-1, None] + eff[ct]).ravel()
    pe = []
    for q in (np.asarray(q_gpu, np.float64), q_ref):
        _, M = oracle.forward_qt(types, ct, q, w["t"], with_skin=False)
        pe.append(M[rows, :, 3].reshape(len(ct), -1, 3))
    err_g = np.linalg.norm(pe[0] - tg, axis=-1)
    err_r = np.linalg.norm(pe[1] - tg, axis=-1)
    d = np.linalg.norm(pe[0] - pe[1], axis=-1)
    joints = int(off[-1])
    return {"final_mean_gpu": float(err_g.mean()), "final_max_gpu": float(err_g.max()),
            "final_mean_oracle": float(err_r.mean()), "final_max_oracle": float(err_r.max()),
            "max_abs_effector_diff": float(np.abs(pe[0] - pe[1]).max()),
            "frac_effectors_within_1pct": float((d <= 1e-2).mean()), "effectors": int(d.size),
            "bar": "mean and max remaining error within 25% of the FP64 run's, >= 99.5% of effectors within 1e-2 "
                   "(1% of the unit extent) of their FP64 positions",
            "oracle": {"seconds": dt, "cores": procs, "steps_per_s": int(w["n_steps"]) / dt,
                       "joint_steps_per_s": joints * int(w["n_steps"]) / dt, "kind": "oracle", "cpu": cpu_model(),
                       "sample": f"the whole run: {len(ct):,} characters x {int(w['n_steps'])} Adam steps, FP64, "
                                 f"characters split over {procs} processes (full trees each step)"}}


def cpu_baseline(min_seconds: float = 6.0) -> dict:
    """The FP64 oracle as it stands on the full frame: on every host core (one
    process per core, each on its share of the characters) and on one host
    thread."""
    import oracle
    w = synth.config2()
    joints = int(sum(len(w["types"][t]["parents"]) for t in w["char_type"]))
    oracle.frame(w)  # build + warm
    reps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < min_seconds:
        oracle.frame(w)
        reps += 1
    dt = time.perf_counter() - t0
    single = {"value": reps * joints / dt, "cores": 1,
              "sample": f"full frame ({joints:,} joints) x {reps} in {dt:.1f} s, FP64, one host thread"}
    n = host_cores()
    reps_all = max(1, math.ceil(min_seconds / (dt / reps) * n / 2))  # about min_seconds / 2 of wall time
    try:
        dt_all, n = oracle_all_cores(reps_all)
    except RuntimeError as e:  # report the one-thread figure alone
        return {"value": single["value"], "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": cpu_model(),
                "sample": single["sample"], "all_cores_error": str(e)}
    return {"value": reps_all * joints / dt_all, "unit": UNIT, "cores": n, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"full frame ({joints:,} joints) x {reps_all} in {dt_all:.1f} s, FP64, characters split "
                      f"over {n} processes (one per host core)",
            "single_thread": single}


# ------------------------------------------------------------------ reference arm
def run_reference(args) -> dict | None:
    """The reference arm: the FP64 oracle as it stands on the host cores, one
    step = the full frame with its characters split over one process per core
    (a bounded sample on one thread if the processes cannot run)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    import oracle
    w = synth.config2()
    joints = int(sum(len(w["types"][t]["parents"]) for t in w["char_type"]))
    try:
        dt, n = oracle_all_cores(args.steps, warm=args.warmup)
        desc = (f"full frame ({joints:,} joints) per step, characters split over {n} processes (one per host "
                f"core), FP64")
    except RuntimeError:
        w = synth.subset(w, list(range(0, 4096, 16)) + [4096])
        joints = int(sum(len(w["types"][t]["parents"]) for t in w["char_type"]))
        for _ in range(args.warmup):
            oracle.frame(w)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle.frame(w)
        dt, n = time.perf_counter() - t0, 1
        desc = f"every 16th character of the frame + the dragon ({joints:,} joints) per step, FP64, one host thread"
    value = args.steps * joints / dt
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": n, "kind": "oracle", "cpu": cpu_model(),
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_only(args) -> dict:
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    peak = measured_peaks().get("hbm_gbs") or 6800.0
    sched = [int(x) for x in args.schedule.split(",")] if args.schedule else None
    if args.only == "forward":
        res = time_forward_methods(rank_workload(rank), local, dev, world, algs=(), schedule=sched)
    elif args.only == "fwd_bwd":
        res = run_fwd_bwd(ctx_factory=setup_ctx, device=local, dev=dev, steps=args.steps, warmup=args.warmup,
                          world=world, peak=peak, schedule=args.schedule_bwd or None)
    else:
        fn = {"mixed": run_mixed_frame, "mixed_split": run_mixed_split, "ik": run_ik, "skinned": run_skinned_frame,
              "layers": run_layered_frame}
        res = fn[args.only](local, dev, world, peak, schedule=sched)
        res.pop("_q_final", None)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return {"only": args.only, "n_gpus": world, "result": res}


def summary(r: dict) -> dict:
    """The headline figures of every workload in one flat object: ms per step
    and the fraction of the measured HBM peak (frame kernel, fwd+bwd, mixed
    frame, IK step), the plain kernel's time and the fused frame's speedup
    over it, and the IK's agreement with the FP64 oracle run."""
    out = {"frame_ms": r.get("ms_per_step"), "frame_kernel_frac": r.get("roofline", {}).get("frac")}
    for key, name in (("fwd_bwd", "fwd_bwd"), ("frame_mixed", "mixed"), ("ik", "ik")):
        x = r.get(key)
        if isinstance(x, dict):
            out[f"{name}_ms"] = x.get("ms_per_step")
            out[f"{name}_frac"] = x.get("roofline", {}).get("frac")
    p = r.get("plain")
    if isinstance(p, dict):
        out["plain_ms"] = p.get("ms_per_step")
        out["fused_vs_plain"] = p.get("speedup_fused_vs_plain")
    ik = r.get("ik")
    if isinstance(ik, dict) and isinstance(ik.get("vs_oracle"), dict):
        v = ik["vs_oracle"]
        out["ik_max_dev_from_oracle"] = v.get("max_abs_effector_diff")
        out["ik_frac_within_1pct"] = v.get("frac_effectors_within_1pct")
        out["ik_final_err_gpu"] = v.get("final_mean_gpu")
        out["ik_final_err_oracle"] = v.get("final_mean_oracle")
    return {k: (round(v, 6) if isinstance(v, float) else v) for k, v in out.items()}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extras", action="store_true", help="skip the plain-kernel and fwd+bwd measurements")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--schedule", default="", help="seg_len,ctas_per_sm,joints_per_item,walk[,adj_ctas] for the frame "
                                                   "instead of running the autotuner")
    ap.add_argument("--schedule-bwd", default="", help="the same for the forward+adjoint measurement")
    ap.add_argument("--only", choices=["mixed", "mixed_split", "ik", "skinned", "layers", "forward", "fwd_bwd"],
                    default="",
                    help="run one of the extra workloads alone (under --schedule if given, else autotuned) and "
                         "print its result object; a short command for profiling its kernel")
    ap.add_argument("--paper-sweep", action="store_true",
                    help="print the depth sweep of the paper's experiment (our forward kernel, the plain kernel, "
                         "the paper's Algorithms 1-4) instead of the bench line")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        r = run_reference(args)
        if r is not None:
            print(json.dumps(r))
        return
    if args.paper_sweep:
        r = run_paper_sweep(args)
        if dist_env()[1] == 0:
            print(json.dumps(r))
        return
    if args.only:
        r = run_only(args)
        if dist_env()[1] == 0:
            print(json.dumps(r))
        return
    world, rank, _ = dist_env()
    r = run_ours(args)
    q_ik = r.get("ik", {}).pop("_q_final", None) if isinstance(r.get("ik"), dict) else None
    if rank == 0:
        if world == 1 and not args.no_cpu:
            r["cpu_baseline"] = cpu_baseline()
            if q_ik is not None:  # the oracle's IK run, part of the CPU-baseline leg
                r["ik"]["vs_oracle"] = ik_vs_oracle(q_ik)
        add_nominal_fractions(r)
        r["summary"] = summary(r)  # last, so that the end of the line carries it
        print(json.dumps(r))


if __name__ == "__main__":
    main()
