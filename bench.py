#!/usr/bin/env python
"""Throughput of the Vertex Block Descent sweep on one B300 (or N replicas).

Workload (default): a 100x100x100 grid of cubes split into 6 tets each
(1,030,301 vertices, 6,000,000 tets), vertices jittered by +-10% of the
0.01 m edge, E = 1e6 Pa, nu = 0.45, rho = 1000, dropped from 0.5 m onto a
ground plane with penalty stiffness 1e7, h = 1/60, 100 iterations per step,
20 steps (the warm-up steps run before and the state is reset to rest).
Synthetic inputs; the slot data streamed per iteration (1.3 GB) exceeds L2.

Metric: vertex-block updates per second = free vertices x iterations x steps
/ time, whole job.  One JSON line on rank 0.  ``--impl reference`` times the
FP64 CPU oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "vertex-block updates/sec and % HBM roofline (1M-vert mesh); batched & adjoint vs plain"
UNIT = "vertex-block updates/s"
# algorithmic bytes per vertex-block update (per-incidence rest data + own
# vertex I/O + one re-read of neighbour positions per colour pass)
B_INC, B_VTX, B_X = 52, 44, 12
B_SC = 24  # with self-collision: contact[i] and rev_off[i], rev_off[i+1], in the sweep and the copy-back
VARIANTS = {0: "plain", 1: "tma_staged", 2: "persistent", 3: "two_phase_scatter", 4: "fused_cluster_loop",
            5: "compact_rest_slots", 6: "compact_rest_slots_packed_pairs", 7: "warp_rows_tma_ring"}
KERNELS = {0: "k_sweep", 1: "k_sweep_pipe", 2: "k_sweep_persist", 3: "k_scatter_slots + k_scatter_reduce",
           4: "k_iterate_fused", 5: "k_sweep_rest", 6: "k_sweep_pair", 7: "k_sweep_rows"}
NOMINAL_HBM_GBS = 7700.0  # B300 HBM3e nominal bandwidth, for context beside the measured peak
DETECT_LAUNCHES = 20   # kernels and memsets of one self-collision detection (three prefix sums)
CCD_LAUNCHES = 20      # kernels and memsets of one CCD (two prefix sums)
EE_LAUNCHES = 17       # the edge-edge part of one CCD (two prefix sums)
EE_CARRY_LAUNCHES = 9  # carrying edge-edge pairs at the step start (one prefix sum)
CPU_SAMPLE_N = 32      # the CPU legs run a 32^3-cube crop of the same recipe
CPU_SAMPLE_ITERS = 100  # the workload's own iterations per step


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scene", choices=["cube", "slabs"], default="cube",
                    help="cube: the large-cube drop (default); slabs: the self-collision slab scene")
    ap.add_argument("--n", type=int, default=0, help="cubes per side (default 100 for cube, 300 for slabs)")
    ap.add_argument("--iters", type=int, default=0, help="iterations per step (default 100 cube, 20 slabs)")
    ap.add_argument("--coloring", choices=["kuhn", "greedy"], default="kuhn")
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--variant", type=int, default=-1,
                    help="sweep kernel: 0 plain, 1 TMA-staged, 2 persistent, 3 two-phase scatter, "
                         "4 fused loop (small meshes), 5 compact slots, 6 compact slots in packed pairs, "
                         "7 warp rows; -1 autotune")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default launch shape")
    ap.add_argument("--mu-c", type=float, default=0.0, help="ground friction coefficient (Eqs. 13-16)")
    ap.add_argument("--ccd-interval", type=int, default=0,
                    help="slabs scene: vertex-triangle CCD every n iterations (Sec. 3.5); 0 = DCD only")
    ap.add_argument("--ccd-edges", action="store_true", help="slabs scene: the CCD also pairs crossing edges")
    ap.add_argument("--line-search", action="store_true", help="local backtracking on G_i (Sec. 3.2)")
    ap.add_argument("--jacobi", action="store_true", help="block-Jacobi iterations")
    ap.add_argument("--young", type=float, default=0.0, help="override Young's modulus of the workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-per-mesh", action="store_true",
                    help="batched leg: skip the comparison with one context per mesh")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched, adjoint, self-collision and Chebyshev comparisons")
    ap.add_argument("--batch-meshes", type=int, default=4096)
    ap.add_argument("--only", choices=["batched", "adjoint", "self_collision", "chebyshev", "small_configs",
                                       "paper_scale", "parity"],
                    default=None,
                    help="run one of the comparisons alone and print it as the JSON line (for profiling)")
    ap.add_argument("--no-paper-scale", action="store_true", help="skip the 320^3-cube comparison")
    ap.add_argument("--oracle-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--budget", type=float, default=0.0, help=argparse.SUPPRESS)
    args = ap.parse_args(argv)
    if not args.n:
        args.n = 300 if args.scene == "slabs" else 100
    if not args.iters:
        args.iters = 20 if args.scene == "slabs" else 100
    return args


# ------------------------------------------------------------ distributed ---

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_job(seconds: float, units: float, world: int):
    """(max seconds over ranks, sum of units over ranks)."""
    if world <= 1:
        return seconds, units
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def any_rank(flag: bool, world: int) -> bool:
    """True on every rank if the flag is set on any rank (the ranks then take
    the same branch, so their collectives stay matched)."""
    if world <= 1:
        return flag
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([1.0 if flag else 0.0], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return bool(t.item() > 0)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ clocks ---

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gpu_id, "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "note": "nvidia-smi unavailable"}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def clocks_rejected(clk: dict) -> bool:
    """A timed region that saw a hardware or thermal slowdown, or SM clocks
    far below their maximum with no reason given (a leftover clock lock), is
    not a valid measurement; sw_power_cap alone is kept."""
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if bad & set(clk.get("reasons", [])):
        return True
    sm, smax = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    return bool(sm and smax and sm < 0.8 * smax and not clk.get("reasons"))


def gpu_id_of(dev: int) -> str:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


# ---------------------------------------------------------------- helpers ---

def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


def kernel_source_sha() -> str:
    """Hash of the forward kernels' code with comments and blank space removed,
    so that a profile stays attached to the code it measured."""
    import re
    h = hashlib.sha256()
    for f in ("vbd_kernels.cu", "vbd_kernels.h"):
        with open(os.path.join(ROOT, "paper_2403_06321_b300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("".join(src.split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(workload_key: str, updates_per_launch: float):
    """DRAM bytes per sweep launch from the committed ncu summary (bytes per
    vertex update, measured on a smaller case of the same recipe, times the
    updates of this launch), if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "sweep_%s.md" % workload_key)
    try:
        lines = open(p).read().splitlines()
    except OSError:
        return None
    kv = {}
    for ln in lines:
        if ln.startswith("- ") and ":" in ln:
            k, v = ln[2:].split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    if kv.get("kernel_source_sha") != kernel_source_sha():
        return None
    try:
        return float(kv["dram_bytes_per_update"]) * updates_per_launch
    except (KeyError, ValueError):
        return None


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def crop_description(n: int = CPU_SAMPLE_N, iters: int = CPU_SAMPLE_ITERS) -> str:
    return ("large_cube recipe on a %d^3-cube crop (%d verts, %d tets): jitter 10%% (seed 1), E=1e6 nu=0.45, "
            "0.5 m above ground k_c=1e7, h=1/60, %d iterations/step" % (n, (n + 1) ** 3, 6 * n ** 3, iters))


def oracle_child(args) -> int:
    """Child process of the CPU legs: times the oracle library named by
    VBD_ORACLE_LIB (the serial build, or the OpenMP build on OMP_NUM_THREADS
    threads) on the crop, `warmup` untimed steps then steps until `budget`
    seconds or `steps` steps, and prints one JSON line."""
    import numpy as np
    from oracle import oracle
    from paper_2403_06321_b300 import synth
    m, cfg = synth.large_cube(CPU_SAMPLE_N)
    model = oracle.Model.from_mesh(m)
    colors = synth.kuhn_coloring(m.grid_ijk)
    p = oracle.Params.make(gravity=cfg.gravity, ground_on=cfg.ground_on, k_c=cfg.k_c)
    x, v = m.rest.copy(), np.zeros_like(m.rest)
    vp = v.copy()
    n_free = int((m.pinned == 0).sum())
    for _ in range(args.warmup):
        model.step(p, colors, 4, cfg.h, CPU_SAMPLE_ITERS, x, v, vp)
    t0 = time.perf_counter()
    times = []
    while len(times) < args.steps:
        a = time.perf_counter()
        model.step(p, colors, 4, cfg.h, CPU_SAMPLE_ITERS, x, v, vp)
        times.append(time.perf_counter() - a)
        if args.budget > 0 and time.perf_counter() - t0 >= args.budget:
            break
    print(json.dumps({"n_free": n_free, "iters": CPU_SAMPLE_ITERS, "step_s": times}), flush=True)
    return 0


def run_oracle_child(threads: int, budget_s: float, steps: int, warmup: int) -> dict:
    """Runs oracle_child in a fresh interpreter (spawned, so no CUDA state is
    inherited) with the serial build (threads == 1) or the OpenMP build."""
    from oracle import oracle
    lib = oracle.build(openmp=threads > 1)
    env = dict(os.environ, VBD_ORACLE_LIB=lib, OMP_NUM_THREADS=str(threads), OMP_PROC_BIND="spread",
               OMP_PLACES="cores" if threads > 1 else "threads")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-child", "--steps", str(steps),
           "--warmup", str(warmup), "--budget", str(budget_s)]
    res = subprocess.run(cmd, env=env, capture_output=True, text=True, check=True)
    out = json.loads(res.stdout.strip().splitlines()[-1])
    out["threads"] = threads
    return out


def run_cpu_baseline(budget_s: float = 10.0) -> dict:
    """The FP64 oracle as it stands, on this host: the OpenMP build on every
    core (the vertices of one colour on all threads) and the serial build on
    one core, each for about budget_s seconds of steps of the crop."""
    cores = host_cores()
    res = {}
    for threads in sorted({1, cores}):
        r = run_oracle_child(threads, budget_s, 1000, 0)
        steps = len(r["step_s"])
        res[threads] = {"value": r["n_free"] * r["iters"] * steps / sum(r["step_s"]), "unit": UNIT,
                        "cores": threads, "kind": "oracle",
                        "sample": "%d step(s) of the %s FP64 oracle on %d thread(s): %s" % (
                            steps, "OpenMP" if threads > 1 else "serial", threads, crop_description())}
    out = dict(res[cores])
    if cores > 1:
        out["single_core"] = res[1]
        out["build"] = "oracle/vbd_oracle.c with -fopenmp (vertices of one colour on all threads)"
    return out


# --------------------------------------------------------------- reference ---

def run_reference(args):
    """The reference arm: the oracle (there is no other implementation of the
    paper), OpenMP build on every host core, timed step by step on a 32^3-cube
    crop of the benchmark recipe at the workload's 100 iterations per step."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    cores = host_cores()
    r = run_oracle_child(cores, 0.0, args.steps, args.warmup)
    dt = sum(r["step_s"])
    value = r["n_free"] * r["iters"] * args.steps / dt
    sample = ("each step: one time step (%d iterations) of the %s FP64 oracle on %d thread(s), %s" % (
        r["iters"], "OpenMP" if cores > 1 else "serial", cores, crop_description()))
    cfg = workload_config(args, None)
    cfg["workload"] = crop_description() + " (a bounded sample of: %s)" % cfg["workload"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(args, info, mesh=None) -> dict:
    n = args.n
    if args.scene == "slabs":
        nv = (n + 1) ** 2 * 5 + (n - 1) ** 2 * 5
        nt = 24 * (n * n + (n - 2) ** 2)
        desc = ("colliding_slabs: %dx%dx4 + %dx%dx4 cubes x 6 tets (%d verts, %d tets), jitter 5%%, E=1e5 "
                "nu=0.4, upper slab turned 0.15 rad and sunk 0.1 edge, self-collision r=0.5 edge k_c=1e5, "
                "h=1/60, %d iterations/step" % (n, n, n - 2, n - 2, nv, nt, args.iters))
    else:
        desc = ("large_cube: %d^3 cubes x 6 tets (%d verts, %d tets), jitter 10%%, E=1e6 nu=0.45, "
                "drop 0.5 m onto ground k_c=1e7, h=1/60, %d iterations/step" % (
                    n, (n + 1) ** 3, 6 * n ** 3, args.iters))
    n_tets = mesh.n_tets if mesh is not None else (nt if args.scene == "slabs" else 6 * n ** 3)
    cfg = {"workload": desc,
           "iters_per_step": args.iters, "h": 1.0 / 60.0, "coloring": args.coloring,
           "variant": {"mu_c": args.mu_c, "line_search": bool(args.line_search), "jacobi": bool(args.jacobi),
                       "young_override": args.young or None, "self_collision": args.scene == "slabs",
                       "ccd_interval": args.ccd_interval if args.scene == "slabs" else 0,
                       "ccd_edges": bool(args.ccd_edges) and args.scene == "slabs"},
           "l2": "inputs larger than L2 (slot stream %.2f GB per iteration)" % (n_tets * 4 * 48 / 1e9)}
    if info is not None:
        cfg.update({"n_colors": info.n_colors, "n_free_verts": info.n_free, "n_slots": int(info.n_slots),
                    "lanes_per_vertex": info.lanes_per_vertex, "block_threads": info.block_threads,
                    "sweep_variant": VARIANTS[info.pipeline], "stage_slots": info.pipe_stage_slots,
                    "ctas_per_sm": info.pipe_ctas_per_sm,
                    "cuda_graph": bool(info.use_graph), "parallelism": "replicas"})
    return cfg


# ------------------------------------------------------------------ extras ---

def _timed(stream, fn, reps):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def run_batched(args) -> dict:
    """4096 independent beams (cube counts U{4..40} x U{2..8} x U{2..8}) swept
    in one launch per colour, against the same beams each in its own context
    (its own launches and graph) on the same GPU, both on one stream."""
    import numpy as np
    import torch
    from paper_2403_06321_b300 import synth, vbd
    meshes, cfg = synth.beam_batch(args.batch_meshes)
    cat, voff, toff = synth.concat(meshes)
    colors = np.concatenate([synth.kuhn_coloring(m.grid_ijk) for m in meshes])
    params = vbd.make_params(gravity=cfg.gravity, init_mode=cfg.init_mode, det_eps=cfg.det_eps)
    stream = torch.cuda.Stream()
    sim = vbd.Sim(cat, params, colors=colors, stream=stream, vert_offset=voff, tet_offset=toff)
    sim.set_state(cat.rest, np.zeros_like(cat.rest))
    if args.lanes or args.block or args.variant >= 0:  # a given launch shape (profiling)
        vbd.vbd_set_launch(sim.ctx, args.lanes, args.block, args.variant)
    elif not args.no_autotune:
        vbd.vbd_autotune(sim.ctx, cfg.h, cfg.iters)  # launch shape for this batch
    info = vbd.vbd_get_info(sim.ctx)
    sim.set_state(cat.rest, np.zeros_like(cat.rest))
    steps = 5
    h, iters = cfg.h, cfg.iters
    for _ in range(2):
        sim.step(h, iters)
    t_ms, sweep_ms, _ = timed_steps(sim, h, iters, steps, stream)
    t_b = t_ms / 1e3
    sim.sync_status()
    v_batched = info.n_free * iters * steps / t_b
    sim.close()
    # roofline of the colour passes: the algorithmic byte model per update
    # (rest data 52 B per incidence, own vertex 44 B, neighbour re-reads
    # 12 B per colour) and, for the compact-slot kernels, their own (16 B of
    # ids per incidence, 60 B own vertex and rest position, 24 B per colour)
    C = info.n_colors
    inc = 4.0 * cat.n_tets / cat.n_verts
    avg_launch_s = sweep_ms / 1e3 / (steps * iters * C)
    peak, peak_kind = measured_peak_hbm()
    b_model = inc * B_INC + B_VTX + B_X * C
    roof = {"bound": "hbm", "peak": peak, "peak_source": peak_kind, "unit": "GB/s",
            "alg_bytes_per_update": b_model, "avg_launch_us": avg_launch_s * 1e6,
            "achieved": info.n_free / C * b_model / avg_launch_s / 1e9}
    roof["frac"] = roof["achieved"] / peak
    if info.pipeline in (5, 6):
        b_own = inc * 16 + 60 + 24 * C
        roof["own_model_bytes_per_update"] = b_own
        roof["own_model_frac"] = info.n_free / C * b_own / avg_launch_s / 1e9 / peak
    out = {"workload": "%d beams, %d verts, %d tets, Kuhn 4-colouring, h=1/60, %d iterations/step, "
                       "one launch per colour for all meshes, CUDA graph per step" % (
                           len(meshes), cat.n_verts, cat.n_tets, iters),
           "launch": {"sweep_variant": VARIANTS[info.pipeline], "lanes_per_vertex": info.lanes_per_vertex,
                      "block_threads": info.block_threads},
           "value": v_batched, "unit": UNIT, "ms_per_step": t_b * 1e3 / steps,
           "n_free_verts": int(info.n_free), "roofline": roof}
    if args.no_per_mesh:
        return out
    # per-mesh contexts
    sims = []
    for m in meshes:
        s_ = vbd.Sim(m, params, colors=synth.kuhn_coloring(m.grid_ijk), stream=stream)
        s_.set_state(m.rest, np.zeros_like(m.rest))
        sims.append(s_)
    n_free = sum(s_.info.n_free for s_ in sims)

    def all_step():
        for s_ in sims:
            s_.step(h, iters)
    all_step()
    psteps = 2
    t_p = _timed(stream, all_step, psteps)
    v_plain = n_free * iters * psteps / t_p
    for s_ in sims:
        s_.sync_status()
        s_.close()
    out.update({"per_mesh_value": v_plain, "per_mesh_ms_per_step": t_p * 1e3 / psteps,
                "speedup_vs_plain": v_batched / v_plain})
    return out


def run_adjoint(args, reps: int = 5) -> dict:
    """Adjoint block-GS sweeps (vbd_backward) on the benchmark cube against
    the forward sweeps on the same mesh: vertex-block updates per second of
    each, 2 recorded steps; forward and backward are each timed `reps` times
    and the medians are reported."""
    import numpy as np
    import torch
    from paper_2403_06321_b300 import synth, vbd
    m, cfg = synth.large_cube(args.n)
    steps, iters, adj_iters = 2, args.iters, args.iters
    params = vbd.make_params(gravity=cfg.gravity, ground_on=cfg.ground_on, k_c=cfg.k_c,
                             init_mode=cfg.init_mode, det_eps=cfg.det_eps, tape_steps=steps)
    stream = torch.cuda.Stream()
    sim = vbd.Sim(m, params, colors=synth.kuhn_coloring(m.grid_ijk), stream=stream)
    n_free = sim.info.n_free
    zeros = np.zeros_like(m.rest)
    dev = sim.workspace.device
    gx = torch.zeros(3 * m.n_verts, dtype=torch.float32, device=dev)
    gx[2::3] = 1.0 / m.n_verts
    gE = torch.empty(m.n_tets, dtype=torch.float32, device=dev)
    gv = torch.empty(3 * m.n_verts, dtype=torch.float32, device=dev)
    sim.set_state(m.rest, zeros)
    for _ in range(steps):
        sim.step(cfg.h, iters)
    vbd.vbd_backward(sim.ctx, gx, gE, gv, adj_iters)  # warm-up
    t_f, t_a = [], []
    for _ in range(reps):
        sim.set_state(m.rest, zeros)
        t_f.append(_timed(stream, lambda: sim.step(cfg.h, iters), steps))
        t_a.append(_timed(stream, lambda: vbd.vbd_backward(sim.ctx, gx, gE, gv, adj_iters), 1))
    # how converged the timed solves are (untimed): the adjoint's relative
    # residual per recorded step, and the forward's max |dG/dx| after each step
    adj_res = vbd.vbd_adjoint_residuals(sim.ctx, steps)
    sim.set_state(m.rest, zeros)
    fwd_res = []
    for _ in range(steps):
        sim.step(cfg.h, iters)
        fwd_res.append(vbd.vbd_gradient_norm(sim.ctx))
    sim.sync_status()
    sim.close()
    tf, ta = statistics.median(t_f), statistics.median(t_a)
    v_f = n_free * iters * steps / tf
    v_a = n_free * adj_iters * steps / ta
    return {"workload": "large_cube %d^3, %d recorded steps, %d adjoint block-GS iterations per step" % (
                args.n, steps, adj_iters),
            "value": v_a, "unit": "adjoint vertex-block updates/s", "forward_value": v_f,
            "ratio_vs_plain": v_a / v_f, "ms_backward": ta * 1e3, "ms_forward": tf * 1e3,
            "timing": "median of %d repetitions (backward %s ms)" % (
                reps, ", ".join("%.2f" % (t * 1e3) for t in t_a)),
            "convergence": {
                "adjoint_rel_residual_per_step": [float(r) for r in adj_res],
                "adjoint_rel_residual": "max |r - H lam| / max |r| after the sweeps (FP64 reduction)",
                "forward_grad_inf_per_step_N": [g for g, _ in fwd_res],
                "forward_weight_scale_N": fwd_res[0][1],
                "forward_grad": "max_i |dG/dx_i| at the end of each step (FP64 reduction); scale = max_i m_i |g|"}}


def _gpu_final(mesh, pdict, colors, h, iters, steps, v0, voff=None, toff=None, track_contact=False):
    """Final positions (float64, caller order) of `steps` steps through the C
    ABI; with track_contact, also the most vertices below z = 0 after a step."""
    import numpy as np
    from paper_2403_06321_b300 import vbd
    sim = vbd.Sim(mesh, vbd.make_params(**pdict), colors=colors, vert_offset=voff, tet_offset=toff)
    touched = 0
    try:
        sim.set_state(mesh.rest, v0)
        for _ in range(steps):
            sim.step(h, iters)
            if track_contact:
                x, _ = sim.get_state()
                touched = max(touched, int((x[:, 2] < 0).sum().item()))
        sim.sync_status()
        x, _ = sim.get_state()
        return x.cpu().numpy().astype(np.float64), touched
    finally:
        sim.close()


def _oracle_final(oracle, mesh, pdict, colors, h, iters, steps, v0):
    import numpy as np
    model = oracle.Model.from_mesh(mesh)
    p = oracle.Params.make(**pdict)
    x, v = mesh.rest.copy(), np.array(v0, np.float64)
    vp = v.copy()
    for _ in range(steps):
        model.step(p, colors, int(colors.max()) + 1, h, iters, x, v, vp)
    return x


def _pdict(cfg, **over):
    d = dict(gravity=cfg.gravity, ground_on=cfg.ground_on, ground_height=cfg.ground_height,
             ground_normal=cfg.ground_normal, k_c=cfg.k_c, cheby_rho=cfg.cheby_rho, init_mode=cfg.init_mode,
             det_eps=cfg.det_eps)
    d.update(over)
    return d


def run_parity() -> dict:
    """Part of the oracle (CPU) leg: the FP64 oracle runs a sample of every
    workload and the CUDA path the same sample; the error of each is
    max |x_gpu - x_oracle| over all vertices after the last step, divided by
    the bounding-box diagonal (bar 1e-5), and for the adjoint the worst
    |g_gpu - g_oracle| over max |g_oracle| per gradient column (bar 1e-3).
    Each line names its sample."""
    import numpy as np
    import torch
    from oracle import oracle
    from paper_2403_06321_b300 import synth, vbd
    os.environ.setdefault("VBD_ORACLE_LIB", oracle.build(openmp=True))
    t0 = time.perf_counter()
    out = {"bars": {"positions": "max |x_gpu - x_oracle| / bbox diagonal <= 1e-5",
                    "gradients": "max |g_gpu - g_oracle| / max |g_oracle| per column <= 1e-3"}}

    def diag(x):
        return float(np.linalg.norm(x.max(0) - x.min(0)))

    # cantilever beam: the whole recipe
    m, cfg = synth.cantilever_beam()
    col = synth.kuhn_coloring(m.grid_ijk)
    pd = _pdict(cfg)
    z = np.zeros_like(m.rest)
    xg, _ = _gpu_final(m, pd, col, cfg.h, cfg.iters, cfg.steps, z)
    xo = _oracle_final(oracle, m, pd, col, cfg.h, cfg.iters, cfg.steps, z)
    out["cantilever_beam"] = {"sample": "the whole workload (176 verts, 100 steps x 20 iterations)",
                              "err_over_bbox": float(np.abs(xg - xo).max()) / diag(xo)}
    # large cube: the benchmark recipe on a 12^3 crop started 5 mm above the ground
    m, cfg = synth.large_cube(12, drop_height=0.005)
    col = synth.kuhn_coloring(m.grid_ijk)
    pd = _pdict(cfg)
    z = np.zeros_like(m.rest)
    xg, touched = _gpu_final(m, pd, col, cfg.h, cfg.iters, cfg.steps, z, track_contact=True)
    xo = _oracle_final(oracle, m, pd, col, cfg.h, cfg.iters, cfg.steps, z)
    out["large_cube"] = {"sample": "benchmark recipe (jitter seed 1, E=1e6, nu=0.45, k_c=1e7, 20 steps x 100 "
                                   "iterations) on a 12^3-cube crop (2,197 verts) started 5 mm above the ground",
                         "err_over_bbox": float(np.abs(xg - xo).max()) / diag(xo),
                         "vertices_in_ground_contact_max": touched}
    # beam batch: the three smallest of the first 16 beams of the recipe, as one union
    meshes, cfg = synth.beam_batch(16)
    pick = sorted(range(16), key=lambda b: meshes[b].n_verts)[:3]
    sub = [meshes[b] for b in pick]
    cat, voff, toff = synth.concat(sub)
    col = np.concatenate([synth.kuhn_coloring(mm.grid_ijk) for mm in sub])
    pd = _pdict(cfg)
    xg, _ = _gpu_final(cat, pd, col, cfg.h, cfg.iters, cfg.steps, np.zeros_like(cat.rest), voff, toff)
    worst = 0.0
    for k, mm in enumerate(sub):
        xo = _oracle_final(oracle, mm, pd, synth.kuhn_coloring(mm.grid_ijk), cfg.h, cfg.iters, cfg.steps,
                           np.zeros_like(mm.rest))
        worst = max(worst, float(np.abs(xg[voff[k]:voff[k + 1]] - xo).max()) / diag(mm.rest))
    out["beam_batch"] = {"sample": "beams %s of the 4096-beam recipe (%d verts) swept as one union, 50 steps x 30 "
                                   "iterations" % (pick, cat.n_verts), "err_over_bbox": worst}
    # differentiable beam: its loss and 30 x 50 schedule on the cantilever mesh, adjoint gradients
    m, _ = synth.cantilever_beam()
    col = synth.kuhn_coloring(m.grid_ijk)
    h, iters, steps, adj_iters = 1 / 60, 50, 30, 150
    tip = np.nonzero(synth.face_mask(m.grid_ijk, (10, 3, 3), "x+"))[0]
    target = m.rest[tip] + np.random.default_rng(3).uniform(-0.1, 0.1, size=3)
    pd = _pdict(synth.SimConfig())
    sim = vbd.Sim(m, vbd.make_params(tape_steps=steps, **pd), colors=col)
    try:
        sim.set_state(m.rest, np.zeros_like(m.rest))
        for _ in range(steps):
            sim.step(h, iters)
        x, _ = sim.get_state()
        xg = x.cpu().numpy().astype(np.float64)
        g = np.zeros_like(xg)
        g[tip] = 2.0 / len(tip) * (xg[tip] - target)
        dev = sim.workspace.device
        gE = torch.empty(m.n_tets, dtype=torch.float32, device=dev)
        gv = torch.empty(3 * m.n_verts, dtype=torch.float32, device=dev)
        vbd.vbd_backward(sim.ctx, torch.tensor(g.reshape(-1), dtype=torch.float32, device=dev), gE, gv, adj_iters)
        sim.sync_status()
        gE = gE.cpu().numpy().astype(np.float64)
        gv = gv.cpu().numpy().astype(np.float64).reshape(-1, 3)
    finally:
        sim.close()
    model = oracle.Model.from_mesh(m)
    p = oracle.Params.make(**pd)
    x, v = m.rest.copy(), np.zeros_like(m.rest)
    vp = v.copy()
    xs = [x.copy()]
    for _ in range(steps):
        model.step(p, col, 4, h, iters, x, v, vp)
        xs.append(x.copy())
    go = np.zeros_like(x)
    go[tip] = 2.0 / len(tip) * (x[tip] - target)
    oE, ov, _ = oracle.dense_adjoint(model, p, h, xs, go)

    def worst_col(gg, oo):
        gg, oo = gg.reshape(len(gg), -1), oo.reshape(len(oo), -1)
        return max(float(np.abs(gg[:, c] - oo[:, c]).max()) / float(np.abs(oo[:, c]).max())
                   for c in range(oo.shape[1]) if np.abs(oo[:, c]).max() > 0)
    out["differentiable_beam"] = {
        "sample": "its loss (tip face to a seeded target) and schedule (30 steps x 50 iterations, %d adjoint "
                  "iterations) on the cantilever mesh (176 verts, 540 tets)" % adj_iters,
        "x_err_over_bbox": float(np.abs(xg - x).max()) / diag(x),
        "dlogE_worst": worst_col(gE, oE), "dv0_worst": worst_col(gv, ov)}
    # paper scale: the 33M-vertex recipe on a 12^3 crop
    m, cfg, v0 = synth.paper_scale_cube(12)
    v0 = v0.astype(np.float32).astype(np.float64)
    col = synth.kuhn_coloring(m.grid_ijk)
    pd = _pdict(cfg)
    xg, _ = _gpu_final(m, pd, col, cfg.h, cfg.iters, cfg.steps, v0)
    xo = _oracle_final(oracle, m, pd, col, cfg.h, cfg.iters, cfg.steps, v0)
    out["paper_scale"] = {"sample": "paper-scale recipe (seed 4, N(0, 0.5 m/s) velocities, 5 steps x 20 "
                                    "iterations) on a 12^3-cube crop", "err_over_bbox": float(np.abs(xg - xo).max())
                          / diag(xo)}
    out["seconds"] = time.perf_counter() - t0
    return out


def timed_steps(sim, h: float, iters: int, K: int, stream):
    """K steps with CUDA events on the sim's stream: (total ms, iteration
    phase ms, per-step ms)."""
    import torch
    from paper_2403_06321_b300 import vbd
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    ev_a = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    torch.cuda.synchronize()
    for k in range(K):
        ev[k].record(stream)
        vbd.vbd_begin_step(sim.ctx, h)
        ev_a[k].record(stream)
        vbd.vbd_iterate(sim.ctx, iters)
        ev_b[k].record(stream)
        vbd.vbd_end_step(sim.ctx)
    ev[K].record(stream)
    torch.cuda.synchronize()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(K)]
    return ev[0].elapsed_time(ev[K]), sum(a.elapsed_time(b) for a, b in zip(ev_a, ev_b)), per


def run_paper_scale(args) -> dict:
    """The paper-scale recipe at full size: 320^3 cubes (33,076,161 verts,
    196,608,000 tets, about 1e8 DoFs), N(0, 0.5 m/s) velocities (seed 4),
    h = 1/60, 20 iterations per step, 5 timed steps after 1 warm-up step,
    HBM resident (a 67 GB workspace).  Skipped, with the reason, when the host
    or the GPU lacks the memory."""
    import numpy as np
    import torch
    from paper_2403_06321_b300 import synth, vbd
    host_free = 0
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    host_free = int(ln.split()[1]) * 1024
    except (OSError, ValueError, IndexError):
        host_free = 0
    dev_free, _ = torch.cuda.mem_get_info()
    if host_free < 80e9 or dev_free < 80e9:
        return {"skipped": "needs 80 GB of free host and device memory (host %.0f GB, device %.0f GB free)" % (
            host_free / 1e9, dev_free / 1e9)}
    t0 = time.perf_counter()
    m, cfg, v0 = synth.paper_scale_cube(320)
    colors = synth.kuhn_coloring(m.grid_ijk)
    stream = torch.cuda.Stream()
    sim = vbd.Sim(m, vbd.make_params(**_pdict(cfg)), colors=colors, stream=stream)
    setup_s = time.perf_counter() - t0
    try:
        info = sim.info
        sim.set_state(m.rest, v0)
        vbd.vbd_autotune(sim.ctx, cfg.h, cfg.iters)  # trials of a whole step: long enough to show the power cap
        info = vbd.vbd_get_info(sim.ctx)
        sim.set_state(m.rest, v0)
        sim.step(cfg.h, cfg.iters)  # warm-up (graph capture)
        sim.set_state(m.rest, v0)
        clocks = ClockSampler(gpu_id_of(torch.cuda.current_device()))
        time.sleep(0.3)
        t_ms, sweep_ms, per = timed_steps(sim, cfg.h, cfg.iters, cfg.steps, stream)
        clk = clocks.stop()
        sim.sync_status()
    finally:
        sim.close()
    n_upd = float(info.n_free) * cfg.iters * cfg.steps
    C = info.n_colors
    b_upd = 4.0 * m.n_tets / m.n_verts * B_INC + B_VTX + B_X * C
    launches = cfg.steps * cfg.iters * C
    avg_launch_s = sweep_ms / 1e3 / launches
    achieved = info.n_free / C * b_upd / avg_launch_s / 1e9
    peak, peak_kind = measured_peak_hbm()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": peak_kind, "alg_bytes_per_update": b_upd, "avg_launch_us": avg_launch_s * 1e6}
    if info.pipeline in (5, 6):  # the compact-slot kernels' own byte model
        b_own = 4.0 * m.n_tets / m.n_verts * 16 + 60 + 24 * C
        roof["own_model_bytes_per_update"] = b_own
        roof["own_model_frac"] = info.n_free / C * b_own / avg_launch_s / 1e9 / peak
    return {"workload": "paper_scale: 320^3 cubes x 6 tets (%d verts, %d tets), N(0, 0.5 m/s) velocities, ground "
                        "k_c=1e7, h=1/60, %d iterations/step, %d steps" % (m.n_verts, m.n_tets, cfg.iters,
                                                                         cfg.steps),
            "value": n_upd / (t_ms / 1e3), "unit": UNIT, "ms_per_step": t_ms / cfg.steps,
            "ms_per_step_each": per, "setup_s": setup_s,
            "launch": {"sweep_variant": VARIANTS[info.pipeline], "lanes_per_vertex": info.lanes_per_vertex,
                       "block_threads": info.block_threads},
            "roofline": roof, "clocks": clk}


def run_chebyshev(args) -> dict:
    """Chebyshev acceleration (Sec. 3.8, Eqs. 18-19) with rho = 0.95 on the
    benchmark cube, against the same mesh, colouring and iterations without
    it: the extra k_cheby pass per iteration (x, the two previous iterates
    and the collision flags) is the whole cost."""
    import numpy as np
    import torch
    from paper_2403_06321_b300 import synth, vbd
    m, cfg = synth.large_cube(args.n)
    colors = synth.kuhn_coloring(m.grid_ijk)
    iters, steps = args.iters, 3
    out = {}
    for rho in (0.95, 0.0):
        params = vbd.make_params(gravity=cfg.gravity, ground_on=cfg.ground_on, k_c=cfg.k_c,
                                 init_mode=cfg.init_mode, det_eps=cfg.det_eps, cheby_rho=rho)
        stream = torch.cuda.Stream()
        sim = vbd.Sim(m, params, colors=colors, stream=stream)
        n_free = sim.info.n_free
        zeros = np.zeros_like(m.rest)
        sim.set_state(m.rest, zeros)
        sim.step(cfg.h, iters)  # warm-up (graph capture)
        sim.set_state(m.rest, zeros)
        t = _timed(stream, lambda: sim.step(cfg.h, iters), steps)
        sim.sync_status()
        sim.close()
        out[rho] = (n_free * iters * steps / t, t * 1e3 / steps)
    return {"workload": "large_cube %d^3, %d iterations/step, rho = 0.95" % (args.n, iters),
            "value": out[0.95][0], "unit": UNIT, "ms_per_step": out[0.95][1],
            "value_without": out[0.0][0], "ms_per_step_without": out[0.0][1],
            "ratio_vs_plain": out[0.95][0] / out[0.0][0]}


def run_self_collision(args) -> dict:
    """Self-collision (vertex-triangle DCD at each step start, contact forces
    in the sweep, x^new + copy-back per colour) on the slab scene at
    300x300x4 + 298x298x4 cubes, against the same mesh and iterations with
    self-collision off; plus the detection's own time per step."""
    import numpy as np
    import torch
    from paper_2403_06321_b300 import synth, vbd
    m, cfg, u0 = synth.colliding_slabs(n=300, layers=4, seed=31)
    colors = synth.kuhn_coloring(m.grid_ijk)
    h, iters, steps = cfg.h, cfg.iters, 5
    out = {}
    for sc in (True, False):
        params = vbd.make_params(gravity=cfg.gravity, k_c=cfg.k_c, self_collision=sc, dcd_radius=cfg.dcd_radius)
        stream = torch.cuda.Stream()
        sim = vbd.Sim(m, params, colors=colors, stream=stream)
        n_free = sim.info.n_free
        sim.set_state(m.rest, np.zeros_like(m.rest))
        for _ in range(2):
            sim.step(h, iters)
        vbd.vbd_sync_status(sim.ctx, with_contacts=True)
        t = _timed(stream, lambda: sim.step(h, iters), steps)
        _, pairs = vbd.vbd_sync_status(sim.ctx, with_contacts=True)
        out[sc] = (n_free * iters * steps / t, t * 1e3 / steps, pairs / steps)
        if sc:  # begin_step alone: detection + Eq. 3 prediction
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            tot = 0.0
            for _ in range(steps):
                torch.cuda.synchronize()
                e0.record(stream)
                vbd.vbd_begin_step(sim.ctx, h)
                e1.record(stream)
                vbd.vbd_iterate(sim.ctx, iters)
                vbd.vbd_end_step(sim.ctx)
                torch.cuda.synchronize()
                tot += e0.elapsed_time(e1)
            out["begin_ms"] = tot / steps
            info = sim.info
        sim.sync_status()
        sim.close()
    return {"workload": "colliding slabs 300x300x4 + 298x298x4 cubes (%d verts, %d tets, %d boundary tris), "
                        "r = 0.5 edge, k_c = 1e5, h=1/60, %d iterations/step, Kuhn 4-colouring" % (
                            m.n_verts, m.n_tets, info.n_surface_tris, iters),
            "value": out[True][0], "unit": UNIT, "ms_per_step": out[True][1],
            "pairs_per_step": out[True][2], "detect_and_predict_ms_per_step": out["begin_ms"],
            "value_without_self_collision": out[False][0], "ms_per_step_without": out[False][1],
            "ratio_vs_plain": out[True][0] / out[False][0]}


def launches_per_step(args, info, iters: int, C: int) -> int:
    """Kernels of one timed step: predict + finish, and per iteration the
    sweep launches of the chosen variant (self-collision: sweep + copy-back
    per colour, plus the detection; Jacobi: one pass + copy-back; the fused
    loop: one launch for all iterations)."""
    if args.scene == "slabs":
        n_ccd = -(-iters // args.ccd_interval) if args.ccd_interval > 0 else 0
        per_ccd = CCD_LAUNCHES + (EE_LAUNCHES if args.ccd_edges else 0)
        carry = EE_CARRY_LAUNCHES if (args.ccd_edges and args.ccd_interval > 0) else 0
        return 2 + DETECT_LAUNCHES + carry + n_ccd * per_ccd + iters * 2 * C
    if args.jacobi:
        return 2 + iters * 2
    per_colour = {3: 2}.get(info.pipeline, 1)
    if info.pipeline == 4:
        return 3
    return 2 + iters * C * per_colour


def run_small_configs(args) -> dict:
    """The two workloads that fit in L2 (cantilever beam, differentiable
    beam): latency- and launch-bound, so only time per step is reported,
    plus the differentiable beam's adjoint (vbd_backward) over its 30 steps."""
    import numpy as np
    import torch
    from paper_2403_06321_b300 import synth, vbd
    out = {}
    m, cfg = synth.cantilever_beam()
    stream = torch.cuda.Stream()
    sim = vbd.Sim(m, vbd.make_params(gravity=cfg.gravity), colors=synth.kuhn_coloring(m.grid_ijk), stream=stream)
    sim.set_state(m.rest, np.zeros_like(m.rest))
    vbd.vbd_autotune(sim.ctx, cfg.h, cfg.iters)
    chosen = VARIANTS[vbd.vbd_get_info(sim.ctx).pipeline]
    sim.set_state(m.rest, np.zeros_like(m.rest))
    for _ in range(5):
        sim.step(cfg.h, cfg.iters)
    t = _timed(stream, lambda: sim.step(cfg.h, cfg.iters), cfg.steps)
    sim.sync_status()
    sim.close()
    out["cantilever_beam"] = {"workload": "10x3x3 cubes (176 verts, 540 tets), x=0 face pinned, h=1/60, "
                                          "%d iterations/step" % cfg.iters,
                              "ms_per_step": t * 1e3 / cfg.steps, "sweep_variant": chosen}
    m, cfg, tip, target = synth.differentiable_beam()
    params = vbd.make_params(gravity=cfg.gravity, tape_steps=cfg.steps)
    sim = vbd.Sim(m, params, colors=synth.kuhn_coloring(m.grid_ijk), stream=stream)
    dev = sim.workspace.device
    zeros = np.zeros_like(m.rest)
    sim.set_state(m.rest, zeros)
    vbd.vbd_autotune(sim.ctx, cfg.h, cfg.iters)
    chosen = VARIANTS[vbd.vbd_get_info(sim.ctx).pipeline]
    gx = torch.zeros(3 * m.n_verts, dtype=torch.float32, device=dev)
    gE = torch.empty(m.n_tets, dtype=torch.float32, device=dev)
    gv = torch.empty(3 * m.n_verts, dtype=torch.float32, device=dev)

    def fwd():
        sim.set_state(m.rest, zeros)
        for _ in range(cfg.steps):
            sim.step(cfg.h, cfg.iters)
    fwd()
    vbd.vbd_backward(sim.ctx, gx, gE, gv, cfg.iters)
    t_f = _timed(stream, fwd, 1)
    gx.copy_(torch.tensor(np.random.default_rng(3).normal(0.0, 1.0, 3 * m.n_verts), dtype=torch.float32,
                          device=dev))
    t_b = _timed(stream, lambda: vbd.vbd_backward(sim.ctx, gx, gE, gv, cfg.iters), 1)
    adj_res = vbd.vbd_adjoint_residuals(sim.ctx, cfg.steps)
    sim.set_state(m.rest, zeros)
    fwd_res = []
    for _ in range(cfg.steps):
        sim.step(cfg.h, cfg.iters)
        fwd_res.append(vbd.vbd_gradient_norm(sim.ctx))
    sim.sync_status()
    sim.close()
    out["differentiable_beam"] = {"workload": "40x8x8 cubes (3,321 verts, 15,360 tets), %d steps x %d iterations, "
                                              "adjoint %d block-GS iterations per step" % (
                                                  cfg.steps, cfg.iters, cfg.iters),
                                  "ms_per_step": t_f * 1e3 / cfg.steps, "ms_backward_per_step": t_b * 1e3 / cfg.steps,
                                  "sweep_variant": chosen,
                                  "convergence": {
                                      "adjoint_rel_residual_max": float(max(adj_res)),
                                      "adjoint_rel_residual_last_step": float(adj_res[-1]),
                                      "forward_grad_inf_max_N": max(g for g, _ in fwd_res),
                                      "forward_weight_scale_N": fwd_res[0][1],
                                      "note": "adjoint for a seeded N(0, 1) dL/dx_T; max over the 30 steps"}}
    return out


# --------------------------------------------------------------------- ours ---

def run_ours(args):
    import numpy as np
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_2403_06321_b300 import synth, vbd
    from paper_2403_06321_b300.build import build
    if rank == 0:
        build()
    barrier(world)

    if args.scene == "slabs":
        m, cfg, _ = synth.colliding_slabs(n=args.n, layers=4, seed=31)
    else:
        m, cfg = synth.large_cube(args.n)
    if args.young > 0:
        m.young[:] = args.young
    colors = synth.kuhn_coloring(m.grid_ijk) if args.coloring == "kuhn" else None
    params = vbd.make_params(gravity=cfg.gravity, ground_on=cfg.ground_on, k_c=cfg.k_c,
                             init_mode=cfg.init_mode, det_eps=cfg.det_eps, mu_c=args.mu_c,
                             line_search=args.line_search, jacobi=args.jacobi,
                             self_collision=cfg.self_collision, dcd_radius=cfg.dcd_radius,
                             scatter_sweep=args.variant == 3, warp_rows=args.variant == 7,
                             ccd_interval=args.ccd_interval if args.scene == "slabs" else 0,
                             ccd_edges=bool(args.ccd_edges) and args.scene == "slabs")
    stream = torch.cuda.Stream()
    sim = vbd.Sim(m, params, colors=colors, stream=stream)
    if args.lanes or args.block or args.variant >= 0:
        vbd.vbd_set_launch(sim.ctx, args.lanes, args.block, args.variant)
    vbd.vbd_set_graph(sim.ctx, not args.no_graph)
    iters, h, K = args.iters, cfg.h, args.steps
    zeros = np.zeros_like(m.rest)
    sim.set_state(m.rest, zeros)
    if not (args.no_autotune or args.lanes or args.block or args.variant >= 0):
        vbd.vbd_autotune(sim.ctx, h, min(iters, 20))  # times each launch shape, keeps the fastest
    info = vbd.vbd_get_info(sim.ctx)

    # warm-up (graph capture happens here), then reset to the initial state
    sim.set_state(m.rest, zeros)
    for _ in range(args.warmup):
        sim.step(h, iters)
    sim.sync_status()
    sim.set_state(m.rest, zeros)
    torch.cuda.synchronize()

    def timed_region():
        clocks = ClockSampler(gpu_id_of(local))
        time.sleep(0.3)
        barrier(world)
        t_ms, sweep_ms, per_step = timed_steps(sim, h, iters, K, stream)
        barrier(world)
        clk = clocks.stop()
        sim.sync_status()  # raises on non-finite updates
        return t_ms, sweep_ms, per_step, clk

    t_ms, sweep_ms, per_step, clk = timed_region()
    if any_rank(clocks_rejected(clk), world):  # throttled or clock-locked: measure once more
        first = clk
        sim.set_state(m.rest, zeros)
        for _ in range(args.warmup):
            sim.step(h, iters)
        sim.set_state(m.rest, zeros)
        t_ms, sweep_ms, per_step, clk = timed_region()
        clk = dict(clk, remeasured_after=first)
    units = float(info.n_free) * iters * K
    t_job, units_job = reduce_job(t_ms / 1e3, units, world)
    value = units_job / t_job

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        N = m.n_verts
        xh = torch.from_numpy(m.rest.astype(np.float32).reshape(-1)).pin_memory()
        vh = torch.zeros(3 * N, dtype=torch.float32).pin_memory()
        vph = torch.zeros(3 * N, dtype=torch.float32).pin_memory()
        vout = torch.zeros(3 * N, dtype=torch.float32).pin_memory()
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(K):
            vbd.vbd_set_state(sim.ctx, xh, vh, vph)
            vbd.vbd_step(sim.ctx, h, iters)
            vbd.vbd_get_state(sim.ctx, xh, vout)  # synchronising (host destination)
            vph, vh, vout = vh, vout, vph
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        te_job, ue_job = reduce_job(te, units, world)
        e2e = {"value": ue_job / te_job, "unit": UNIT, "h2d_bytes_per_step": 3 * 12 * N,
               "d2h_bytes_per_step": 2 * 12 * N}
    sim.close()

    if rank != 0:
        return 0
    C = info.n_colors
    inc_per_vert = 4.0 * m.n_tets / m.n_verts
    if args.jacobi:
        # one pass over all vertices per iteration (+ its 32-byte copy-back)
        b_upd = inc_per_vert * B_INC + B_VTX + B_X + 32
        launches_sweep = K * iters
        bytes_per_launch = info.n_free * b_upd
    else:
        b_upd = inc_per_vert * B_INC + B_VTX + B_X * C
        if args.scene == "slabs":
            b_upd += B_SC  # pair index and corner-list offsets, read again by the copy-back
        launches_sweep = K * iters * C
        bytes_per_launch = info.n_free / C * b_upd
    avg_launch_s = sweep_ms / 1e3 / launches_sweep
    achieved = bytes_per_launch / avg_launch_s / 1e9
    peak, peak_kind = measured_peak_hbm()
    traffic = (profiled_traffic("large_cube", info.n_free / C)
               if args.scene == "cube" and not args.jacobi and info.pipeline in (0, 2) else None)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": t_job * 1e3 / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": workload_config(args, info, m),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_gbs": NOMINAL_HBM_GBS,
                     "kernel": ("k_sweep_sc" if args.scene == "slabs" else KERNELS[info.pipeline])
                     + " (one colour pass)", "alg_bytes_per_update": b_upd,
                     "avg_launch_us": avg_launch_s * 1e6,
                     "sweep_share_of_step": sweep_ms / t_ms},
        "e2e": e2e,
        "gpu_launches": K * launches_per_step(args, info, iters, C),
        "clocks": clk,
    }
    groups = [g for g in (per_step[k * K // 5:(k + 1) * K // 5] for k in range(5)) if g]
    if len(groups) == 5:
        rates = [info.n_free * iters * len(g) / (sum(g) / 1e3) for g in groups]
        line["median_of_5"] = {"value": statistics.median(rates), "unit": UNIT,
                               "groups": rates, "how": "the K timed steps split into 5 consecutive groups, "
                                                       "rate of each group, median (this rank)"}
    if not args.no_extras and world == 1 and args.scene == "cube":
        line["batched"] = run_batched(args)
        line["adjoint"] = run_adjoint(args)
        line["self_collision"] = run_self_collision(args)
        line["chebyshev"] = run_chebyshev(args)
        line["small_configs"] = run_small_configs(args)
        if not args.no_paper_scale:
            line["paper_scale"] = run_paper_scale(args)
    if not args.no_cpu_baseline and world == 1:
        # the oracle leg: timed on this host's cores, and compared with the
        # CUDA path on a sample of every workload
        line["cpu_baseline"] = run_cpu_baseline()
        if args.scene == "cube":
            line["parity"] = run_parity()
    print(json.dumps(line), flush=True)
    return 0


def run_only(args) -> int:
    import torch
    from paper_2403_06321_b300.build import build
    build()
    torch.cuda.set_device(0)
    fn = {"batched": run_batched, "adjoint": run_adjoint, "self_collision": run_self_collision,
          "chebyshev": run_chebyshev, "small_configs": run_small_configs, "paper_scale": run_paper_scale,
          "parity": lambda _a: run_parity()}[args.only]
    print(json.dumps({"only": args.only, args.only: fn(args)}), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.oracle_child:
        return oracle_child(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
