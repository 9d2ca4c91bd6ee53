"""Benchmark of the overset assembly + interpolation step on GB300.

One step = one time step of the moving-overset workload: set the frames of the moving grids
(ovs_set_motion), then find the donors of every fringe point and interpolate u, v, w, p with the frame
velocity transform in one call (ovs_assemble_interpolate).  Default workload: the school of 16 fish O-grids
(64^3 to 160x96x96) in a stretched curvilinear 512x384x256 background (~50 M nodes), FP64 coordinates,
FP32 fields, ~2.8 M fringe points a step, synthetic and seeded; --workload selects a smaller one.

Prints ONE JSON line (rank 0).  Metric: fringe points assembled + interpolated per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ovs|reference] [--workload cfg0..cfg4]

--impl reference times the plain FP64 CPU oracle (the method written out from the paper) on the host cores,
on a bounded sample of the same workload per step.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fringe pts assembled+interpolated/s per step (learned vs plain), % HBM peak"
UNIT = "pts/s"
# Algorithmic bytes per fringe point (no cache reuse credited): assembly reads the node id (4), the receiver
# coordinates (24), the previous donor (4) and the donor cell's 8 corners (8 x 3 x 8 = 192) and writes grid,
# cell, xi, status (33): 257 B; interpolation reads the donor record (32) and 8 x 4 FP32 field values (128)
# and writes 4 values (16): 176 B.
BYTES_ASSEMBLE = 257
BYTES_INTERP = 176
BYTES_POINT = BYTES_ASSEMBLE + BYTES_INTERP
# The fused kernel (ovs_assemble_interpolate: k_assemble interpolates each point as it decides its donor) moves the
# assembly's 257 B plus the interpolation's fields and outputs (128 + 16 B); the donor record is not re-read.
BYTES_FUSED = BYTES_ASSEMBLE + 128 + 16
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_assemble_cfg4.txt")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1910_09315_gb300", "csrc", f) for f in
                  ("ovs_assemble.cu", "ovs_internal.cuh", "ovs_fields.cuh", "ovs_mlp.cuh")]
WORKLOADS = {
    "cfg1": "moving ellipsoid: stretched curvilinear bg 128^3 + O-grid 96x64x64, 100 steps dt=1e-3, FP32 fields",
    "cfg0": "tiny: Cartesian bg 64^3 + rotated perturbed box 32^3, FP64 fields",
    "cfg2": "moving ellipsoid with bg 256^3 (plain guess), FP32 fields",
    "cfg3": "school of 8 fish O-grids (48x32x32..128x64x64) in a stretched bg 384x256x128, dt=1.39e-3, FP32 fields",
    "cfg4": "school of 16 fish O-grids (64^3..160x96x96) in a stretched bg 512x384x256 (~50M nodes), FP32 fields",
}
# distinct time steps a run cycles through at most (a triangle wave over the first ones beyond that): building the
# fringe sets of a school step takes seconds on the host, so they are built by a pool of host processes
DISTINCT_STEPS = {"cfg3": 64, "cfg4": 64}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ovs", choices=["ovs", "reference"])
    ap.add_argument("--workload", default="cfg4", choices=sorted(WORKLOADS))
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-vs-plain comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=0, help="oracle points per CPU-baseline sample (0: auto)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def combine_ranks(world: int, total_ms: float, e2e_ms: float, pts: float, device="cpu"):
    """Whole-job figures of a replicas run: the slowest rank's timed-region and end-to-end times (max over ranks)
    and the points of all ranks (sum).  One rank: the local figures."""
    if world == 1:
        return total_ms, e2e_ms, pts
    import torch

    t = torch.tensor([total_ms, e2e_ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    p = torch.tensor([pts], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(p, op=torch.distributed.ReduceOp.SUM)
    return float(t[0]), float(t[1]), float(p[0])


def rank0_choice(world: int, flag: bool, device="cpu") -> bool:
    """Every rank takes rank 0's choice (e.g. the launch mode), so that all replicas run the same way."""
    if world == 1:
        return flag
    import torch

    t = torch.tensor([1 if flag else 0], dtype=torch.int32, device=device)
    torch.distributed.broadcast(t, 0)
    return bool(t.item())


def _gen_surface(dims, periodic):
    """The closed shell between a body O-grid's two outer radial layers (all azimuths, all polar rings)."""
    import gen

    return gen.index_box_surface(dims, periodic, (0, 0, dims[2] - 2), (dims[0], dims[1] - 1, dims[2] - 1))


def guess_label(choice) -> str:
    if choice is None:
        return "plain: previous donor, else the control cell (--no-learned)"
    if choice["chosen_width"] == 0:
        return "learned guess requested; the guess autotuner kept no network (plain start was faster)"
    H = choice["chosen_width"]
    return f"learned: previous donor, else the 3-{H}-{H}-3 network of the donor grid (width chosen by ovs_autotune_guess)"


def host_workers() -> int:
    """Host processes for building the steps' fringe sets (at most 8: each holds a step's temporaries)."""
    return max(1, min(8, os.cpu_count() or 1))


def config_index(name: str) -> int:
    return int(name[3:])


def schedule(n: int, s: int) -> int:
    """Step s of the run -> time step of the workload; beyond the last step the motion runs back (a triangle
    wave keeps every step a small motion from the previous one)."""
    if n <= 1:
        return 0
    p = 2 * (n - 1)
    q = s % p
    return q if q < n else p - q


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def profile_traffic(workload: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, if the summary covers this
    workload and the kernel's source has not changed since the capture (the summary records the workload and
    the source hash); else None."""
    try:
        txt = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    m_tr = re.search(r"traffic_bytes_per_full_launch:\s*([0-9.eE+]+)", txt)
    m_wl = re.search(r"traffic_workload:\s*(\S+)", txt)
    if not m_hash or not m_tr or not m_wl or m_wl.group(1) != workload or m_hash.group(1) != kernel_hash():
        return None
    return float(m_tr.group(1))


def measured_peak():
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(mp["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = os.path.join("/tmp", f"ovs_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def lines(self) -> int:
        try:
            return sum(1 for _ in open(self.path))
        except OSError:
            return 0

    def stop(self):
        if self.proc is None:
            return None
        # one more sample after the timed region (the region is often shorter than the sampling interval)
        n0, t0 = self.lines(), time.time()
        while self.lines() <= n0 and time.time() - t0 < 1.0:
            time.sleep(0.02)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def build_workload(name: str):
    import gen

    sc = gen.config(config_index(name))
    return sc


_POOL_SC = None


def _step_job(ts):
    m = _POOL_SC.motion(ts)
    return ts, m, _POOL_SC.fringe_sets(ts, m)


def step_inputs(sc, nsteps_total: int, distinct: int = 0, workers: int = 0):
    """Motions and fringe sets of every step the run visits (host, precomputed outside the timed region).
    workers > 1: the distinct steps are built by forked host processes (call this before any CUDA work: a process
    forked after the first GPU call can hang)."""
    global _POOL_SC
    n = min(sc.nsteps, distinct) if distinct else sc.nsteps
    need = sorted({schedule(n, s) for s in range(nsteps_total)})
    cache = {}
    if workers > 1 and len(need) > 1:
        import multiprocessing as mp

        _POOL_SC = sc
        with mp.get_context("fork").Pool(min(workers, len(need))) as pool:
            for ts, m, fs in pool.imap_unordered(_step_job, need):
                cache[ts] = (m, fs)
        _POOL_SC = None
    for ts in need:
        if ts not in cache:
            m = sc.motion(ts)
            cache[ts] = (m, sc.fringe_sets(ts, m))
    return [cache[schedule(n, s)] for s in range(nsteps_total)], len(need)


# ----------------------------------------------------------------------------------------------------- ovs arm
def run_ovs(args, rank, world, local):
    import torch

    from paper_1910_09315_gb300 import build as ovs_build
    from paper_1910_09315_gb300 import ovs

    ovs_build.build()
    # host inputs first: the step builder forks worker processes, which must happen before any CUDA call
    sc = build_workload(args.workload)
    K, W = args.steps, args.warmup
    inputs, n_distinct = step_inputs(sc, W + K, DISTINCT_STEPS.get(args.workload, 0), workers=host_workers())
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    max_pts = max(sum(len(s.node_ids) for s in fs) for _, fs in inputs)
    xi_dtype = ovs.OVS_F64 if sc.field_dtype == np.float64 else ovs.OVS_F32
    stream = torch.cuda.current_stream(dev)
    ctx = ovs.Context(device=local, stream=stream, max_points=max_pts)
    gids = [ctx.add_grid(g.x, g.y, g.z, g.dims, g.periodic, g.role) for g in sc.grids]
    fdt = torch.float64 if sc.field_dtype == np.float64 else torch.float32
    fields = [tuple(torch.as_tensor(f[k]).to(dev, fdt) for k in ("u", "v", "w", "p")) for f in sc.fields]
    # device-resident inputs of every step (node ids); donors and outputs preallocated
    dev_sets = []
    host_sets = []
    for m, fs in inputs:
        dev_sets.append([(s.receiver, torch.as_tensor(s.node_ids).to(dev), s.donors) for s in fs])
        host_sets.append([(s.receiver, torch.as_tensor(s.node_ids).pin_memory(), s.donors) for s in fs])
    donors = ctx.alloc_donors(max_pts, xi_dtype)
    outs = [torch.empty(max_pts, dtype=fdt, device=dev) for _ in range(4)]
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (129 MB)

    def donors_view(n):
        return {"grid": donors["grid"][:n], "cell": donors["cell"][:n], "xi": donors["xi"][:3 * n],
                "status": donors["status"][:n], "xi_dtype": xi_dtype, "n": n}

    layout = [fields]  # the donor fields one_step passes: four arrays per grid (the headline), or records

    # Each resident step's call arguments are marshalled once, before any timing, as a C caller holds its
    # structs: the timed loop then makes only the library calls (ovs_set_motion per grid and one
    # ovs_assemble_interpolate), not the Python binding's per-call marshalling.
    lib = ovs.load()
    prep = []
    for s_, (m_, fs_) in enumerate(inputs):
        mot = []
        for gid, mo in zip(gids, m_):
            arrs = [(ctypes.c_double * k)(*[float(x) for x in np.ravel(a)])
                    for a, k in ((mo.R, 9), (mo.c, 3), (mo.V, 3), (mo.omega, 3))]
            mot.append((gid, arrs, [ctypes.cast(a, ctypes.c_void_p) for a in arrs]))
        n_ = sum(int(x[1].numel()) for x in dev_sets[s_])
        prep.append((mot, ovs.make_sets(dev_sets[s_]), len(dev_sets[s_]), ovs.Context.donors_struct(donors_view(n_)), n_))
    field_args = {}

    def fields_arg(fl):
        if id(fl) not in field_args:
            farr, o, _ = ctx._fields_structs(fl, 0, outs)
            field_args[id(fl)] = (fl, farr, o)
        return field_args[id(fl)][1:]

    def call(rc):
        if rc != ovs.OVS_OK:
            raise ovs.OvsError(rc, ovs.ovs_last_error(ctx.ctx))

    def one_step(s, sets, fused=True):
        if sets is not dev_sets[s]:  # inputs that are not the resident ones: the binding's own marshalling
            m, fs = inputs[s]
            for gid, mo in zip(gids, m):
                ctx.set_motion(gid, mo.R, mo.c, mo.V, mo.omega)
            n = sum(int(x[1].numel()) for x in sets)
            ctx.assemble_interpolate(sets, layout[0], donors=donors_view(n), out=[o[:n] for o in outs])
            return n
        mot, sarr, ns, dstruct, n = prep[s]
        for gid, _, ptrs in mot:
            call(lib.ovs_set_motion(ctx.ctx, gid, *ptrs))
        farr, ostruct = fields_arg(layout[0])
        if fused:
            call(lib.ovs_assemble_interpolate(ctx.ctx, sarr, ns, ctypes.byref(dstruct), farr, len(gids),
                                              ctypes.byref(ostruct)))
        else:
            call(lib.ovs_assemble(ctx.ctx, sarr, ns, ctypes.byref(dstruct)))
            call(lib.ovs_interpolate(ctx.ctx, sarr, ns, ctypes.byref(dstruct), farr, len(gids), ctypes.byref(ostruct)))
        return n

    # warm-up (hints become warm exactly as in a time loop)
    for s in range(W):
        one_step(s, dev_sets[s])
    torch.cuda.synchronize()
    def events(n):
        out = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        for e in out:
            e.record(stream)  # torch creates the CUDA event on its first record
        return out

    def timed(fused: bool, trace: bool):
        """K steps enqueued back to back (the host runs ahead as in a time loop) after the hints are reset and
        the W warm-up steps rerun; an L2 flush before each step sits outside its events; one synchronisation at
        the end.  trace: the library's trace events around its
        kernels (per-kernel times; launches are then direct, not the captured graph)."""
        # every pass starts from the same state: no previous donors, then the W warm-up steps (the hints of a
        # time loop that has run W steps); a pass never reuses hints from an earlier pass over the same steps
        ovs.ovs_reset_hints(ctx.ctx)
        for s in range(W):
            one_step(s, dev_sets[s], fused=fused)
        e0, e1 = events(K), events(K)
        tr = [events(5) for _ in range(K)] if trace else None
        torch.cuda.synchronize()
        n = 0
        for k, s in enumerate(range(W, W + K)):
            flush.zero_()
            if trace:
                ovs.ovs_set_trace_events(ctx.ctx, tr[k])
            e0[k].record(stream)
            n += one_step(s, dev_sets[s], fused=fused)
            e1[k].record(stream)
        torch.cuda.synchronize()
        ovs.ovs_set_trace_events(ctx.ctx, [])
        step = [e0[k].elapsed_time(e1[k]) for k in range(K)]
        if not trace:
            return n, step, None, None, None
        fast = [tr[k][0].elapsed_time(tr[k][1]) for k in range(K)]
        slow = [tr[k][1].elapsed_time(tr[k][2]) for k in range(K)]
        interp = [tr[k][3].elapsed_time(tr[k][4]) for k in range(K)]
        return n, step, fast, slow, interp

    nw = sum(int(x[1].numel()) for x in dev_sets[W - 1])
    # the learned guess (on unless --no-learned): every body grid's network trained by the library's own kernels on
    # samples of the grid itself, for each candidate width; the library's guess autotuner then picks the width, or
    # no network, on the last warm-up step, and leaves its choice installed
    guess_choice = None
    if not args.no_learned:
        guess_choice = train_and_pick_guess(args, sc, ctx, gids, dev_sets[W - 1], fields, donors_view(nw),
                                            [o[:nw] for o in outs], ovs, torch)
        for s in range(W):
            one_step(s, dev_sets[s])
    # launch shapes: the library's autotuner on the last warm-up step (its calls run for real)
    tuning = ctx.autotune(dev_sets[W - 1], fields, donors=donors_view(nw), out=[o[:nw] for o in outs], reps=3,
                          xi_dtype=xi_dtype)
    # launch mode: both modes timed on the (untimed) warm-up steps with the L2 flushed before each, as in the
    # timed region (the library's autotuner repeats one call with a warm L2, which can hide a mode's cost)
    calib = {ovs.OVS_LAUNCH_GRAPH: 0.0, ovs.OVS_LAUNCH_DIRECT: 0.0}
    for mode in (ovs.OVS_LAUNCH_GRAPH, ovs.OVS_LAUNCH_DIRECT) * 3:  # alternating, three rounds each
        ctx.set_options(launch=mode)
        one_step(0, dev_sets[0])  # (captures the graph)
        ovs.ovs_reset_hints(ctx.ctx)  # the same start for both modes
        ec0, ec1 = events(W), events(W)
        for s in range(W):
            flush.zero_()
            ec0[s].record(stream)
            one_step(s, dev_sets[s])
            ec1[s].record(stream)
        torch.cuda.synchronize()
        # (the first step after the reset starts cold in both modes: left out, it would dominate the sums)
        calib[mode] += float(np.sum([a.elapsed_time(b) for a, b in list(zip(ec0, ec1))[1:]]))
    use_graph = rank0_choice(world, calib[ovs.OVS_LAUNCH_GRAPH] <= calib[ovs.OVS_LAUNCH_DIRECT], dev)
    tuning["launch"] = ovs.OVS_LAUNCH_GRAPH if use_graph else ovs.OVS_LAUNCH_DIRECT
    ctx.set_options(launch=tuning["launch"])
    # the clock sampler starts before the timed region and has reported once before it begins (its start-up
    # must not overlap the timing); meanwhile the GPU keeps running warm-up steps
    clocks = Clocks(local)
    clocks.start()
    t_wait = time.time()
    while clocks.proc is not None and clocks.lines() == 0 and time.time() - t_wait < 5.0:
        for s in range(W):
            one_step(s, dev_sets[s])
        torch.cuda.synchronize()
    for s in range(W):
        one_step(s, dev_sets[s])
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # (an NVTX range around the headline pass, so that a profiler can select exactly its kernels)
    torch.cuda.nvtx.range_push("ovs_timed_steps")
    pts, step_ms, _, _, _ = timed(True, trace=False)
    torch.cuda.nvtx.range_pop()
    ck = clocks.stop()
    total_ms = float(np.sum(step_ms))
    # the same steps again with per-kernel events (direct launches): breakdown and roofline
    _, traced_ms, fast_ms, slow_ms, interp_ms = timed(True, trace=True)
    # both launch modes without tracing (the headline ran the autotuner's choice), and the two separate calls
    # (ovs_assemble, then ovs_interpolate) in the chosen mode
    tuned_launch = tuning["launch"]
    mode_ms = {}
    for name, mode in (("graph", ovs.OVS_LAUNCH_GRAPH), ("direct", ovs.OVS_LAUNCH_DIRECT)):
        if mode == tuned_launch:
            mode_ms[name] = total_ms / K
            continue
        ctx.set_options(launch=mode)
        for s in range(W):
            one_step(s, dev_sets[s])
        _, ms, _, _, _ = timed(True, trace=False)
        mode_ms[name] = float(np.mean(ms))
    ctx.set_options(launch=tuned_launch)
    for s in range(W):
        one_step(s, dev_sets[s], fused=False)
    _, sep_ms, _, _, _ = timed(False, trace=False)
    # the same steps with each grid's fields as one array of (u, v, w, p) records per node (ovs_fields.stride 4):
    # one 16-byte load per donor corner instead of four
    layout[0] = [torch.stack(f, 1).contiguous() for f in fields]
    for s in range(W):
        one_step(s, dev_sets[s])
    _, rec_ms, _, _, _ = timed(True, trace=False)
    _, _, rec_fast_ms, _, _ = timed(True, trace=True)
    layout[0] = fields
    interleaved = {"ms_per_step": float(np.mean(rec_ms)), "k_assemble_ms": float(np.mean(rec_fast_ms)),
                   "note": "fields as (u, v, w, p) records per node; the headline passes four arrays per grid"}
    # plain, unbatched: one ovs_assemble_interpolate per fringe set (direct launches, default launch shapes), the
    # same steps and start (previous donor, else control cell), for the batching comparison
    # (its call arguments, one call per set, marshalled before timing as for the batched calls)
    unb_prep = []
    for s_ in range(len(inputs)):
        calls, b = [], 0
        for st_ in dev_sets[s_]:
            n = int(st_[1].numel())
            d = {"grid": donors["grid"][b:b + n], "cell": donors["cell"][b:b + n], "xi": donors["xi"][3 * b:3 * (b + n)],
                 "status": donors["status"][b:b + n], "xi_dtype": xi_dtype, "n": n}
            farr, o, _ = ctx._fields_structs(fields, n, [x[b:b + n] for x in outs])
            calls.append((ovs.make_sets([st_]), ovs.Context.donors_struct(d), farr, o))
            b += n
        unb_prep.append((calls, b))

    def unbatched_step(s):
        for gid, _, ptrs in prep[s][0]:
            call(lib.ovs_set_motion(ctx.ctx, gid, *ptrs))
        calls, b = unb_prep[s]
        for sarr, dstruct, farr, o in calls:
            call(lib.ovs_assemble_interpolate(ctx.ctx, sarr, 1, ctypes.byref(dstruct), farr, len(gids), ctypes.byref(o)))
        return b

    saved_tuning = ovs.ovs_get_tuning(ctx.ctx)
    headline_guess = ovs.ovs_get_options(ctx.ctx).guess
    ctx.set_options(launch=ovs.OVS_LAUNCH_DIRECT, guess=ovs.OVS_GUESS_HINT)  # the plain start
    ctx.set_tuning(assemble_blocks_per_sm=0, interp_blocks_per_sm=0, slow_blocks_per_sm=0, guess_blocks_per_sm=0)
    ovs.ovs_reset_hints(ctx.ctx)  # the start of every timed pass
    for s in range(W):
        unbatched_step(s)
    e0u, e1u = events(K), events(K)
    torch.cuda.synchronize()
    for k, s in enumerate(range(W, W + K)):
        flush.zero_()
        e0u[k].record(stream)
        unbatched_step(s)
        e1u[k].record(stream)
    torch.cuda.synchronize()
    unbatched_ms = float(np.mean([a.elapsed_time(b) for a, b in zip(e0u, e1u)]))
    ovs.ovs_set_tuning(ctx.ctx, saved_tuning)  # the autotuned shapes and launch mode
    ctx.set_options(guess=headline_guess)
    for s in range(W):
        one_step(s, dev_sets[s])

    # the interpolation as a sparse matrix (paper Sec. 2.2.6): build it from the donors of one step and time
    # one matrix-vector product per field component (as an implicit solve would apply it)
    nW = one_step(W, dev_sets[W])
    dW = donors_view(nW)
    ev_m = events(3)
    ev_m[0].record(stream)
    row_ptr, col, val = ctx.interp_matrix(dW, ovs.OVS_F64 if fdt == torch.float64 else ovs.OVS_F32)
    ev_m[1].record(stream)
    xs = [torch.cat([f[c] for f in fields]) for c in range(4)]
    reps = 20
    for r in range(reps):
        for c in range(4):
            ctx.spmv(row_ptr, col, val, xs[c])
    ev_m[2].record(stream)
    torch.cuda.synchronize()
    matrix = {"points": nW, "nnz": int(row_ptr[-1].item()), "build_ms": ev_m[0].elapsed_time(ev_m[1]),
              "spmv_ms_per_component": ev_m[1].elapsed_time(ev_m[2]) / (4 * reps),
              "note": "rows = fringe points, 8 weights per found point; x = every grid's node values"}
    # hole cutting (paper Sec. 2.2.1): every body's closed wall surface blanks the background nodes in a box
    # around it (the box's nodes are listed once, outside the timing); time per step for all bodies
    import gen as _gen

    holes = None
    bodies = [q for q, g in enumerate(sc.grids) if g.role == 1 and g.meta.get("kind") in ("ogrid", "fish")]
    if bodies and sc.grids[0].meta.get("axes") is not None:
        mW = inputs[W][0]
        bg0 = sc.grids[0]
        cuts = []
        for q in bodies:
            V, T = _gen.body_surface(sc.grids[q])
            sid = ctx.add_surface(gids[q], V, T)
            ext = np.linalg.norm(V, axis=1).max() + 0.02  # the body's bounding sphere: any rotation
            cand = _gen.box_candidates(bg0, mW[q].c - ext, mW[q].c + ext).astype(np.int32)
            cuts.append((sid, torch.as_tensor(cand).to(dev)))
        iblank = torch.ones(bg0.n_nodes, dtype=torch.uint8, device=dev)
        for gid, mo in zip(gids, mW):
            ctx.set_motion(gid, mo.R, mo.c, mo.V, mo.omega)
        sids, cand_list = [c[0] for c in cuts], [c[1] for c in cuts]

        def cut_all(batched):
            iblank.fill_(1)
            if batched:
                ctx.hole_cut_many(sids, gids[0], iblank, cand_list)
            else:
                for sid, cand in cuts:
                    ctx.hole_cut(sid, gids[0], iblank, nodes=cand)

        ev_h = events(4)
        reps = 10
        for batched in (True, False):
            cut_all(batched)  # warm-up
        ev_h[0].record(stream)
        for r in range(reps):
            cut_all(True)
        ev_h[1].record(stream)
        blanked = int((iblank == 0).sum().item())
        ev_h[2].record(stream)
        for r in range(reps):
            cut_all(False)
        ev_h[3].record(stream)
        torch.cuda.synchronize()
        assert int((iblank == 0).sum().item()) == blanked
        holes = {"bodies": len(bodies), "candidate_nodes": int(sum(int(c.numel()) for _, c in cuts)),
                 "blanked": blanked, "ms_per_step": ev_h[0].elapsed_time(ev_h[1]) / reps,
                 "ms_per_step_one_call_per_body": ev_h[2].elapsed_time(ev_h[3]) / reps,
                 "note": "one ovs_hole_cut_many launch for all bodies (mask fill included)"}
        ovs.ovs_set_iblank(ctx.ctx, gids[0], None)
    # fluxes at the receivers (paper Sec. 2.1 eq. flux, Sec. 2.4 mass conservation): after one step, every body
    # grid's interpolated fringe velocities are placed in its node arrays (outside the timing) and the flux through
    # the closed shell between its two fringe layers is reconstructed and corrected, one call per body grid
    fluxes = None
    shells = []
    for q, g in enumerate(sc.grids):
        if g.role != 1 or g.meta.get("kind") not in ("ogrid", "fish"):
            continue
        n = g.dims
        faces_np, signs_np = _gen_surface(n, g.periodic)
        shells.append((q, torch.as_tensor(faces_np).to(dev), torch.as_tensor(signs_np).to(dev)))
    if shells:
        nW = one_step(W, dev_sets[W])
        vel = {q: [torch.zeros(sc.grids[q].n_nodes, dtype=fdt, device=dev) for _ in range(3)] for q, _, _ in shells}
        b = 0
        for r, ids, _ in dev_sets[W]:
            k = int(ids.numel())
            if r in vel:
                for c in range(3):
                    vel[r][c].index_copy_(0, ids.long(), outs[c][b:b + k])
            b += k
        ev_f = events(2)
        reps = 10
        nfaces = sum(int(f.numel()) for _, f, _ in shells)
        for r in range(reps + 1):
            if r == 1:
                ev_f[0].record(stream)
            for q, f, sg in shells:
                ctx.interface_flux(gids[q], f, tuple(vel[q]), signs=sg, surf_start=[0, int(f.numel())], correct=True)
        ev_f[1].record(stream)
        torch.cuda.synchronize()
        fluxes = {"grids": len(shells), "faces": nfaces, "ms_per_step": ev_f[0].elapsed_time(ev_f[1]) / reps,
                  "note": "each body grid's closed shell between its two fringe layers: face fluxes, net flux, "
                          "correction in proportion to area (one ovs_interface_flux per grid)"}
    learned = None if args.no_learned else learned_vs_plain(guess_choice, ctx, dev_sets, one_step, timed, stream,
                                                            flush, K, W, ovs, torch)
    e2e_ms, h2d, d2h, e2e_ref = end_to_end(ctx, lib, inputs, host_sets, dev_sets, prep, layout, max_pts, xi_dtype,
                                           fdt, W, K, flush, stream, dev, ovs, torch)
    total_ms, e2e_total, pts_all = combine_ranks(world, total_ms, e2e_ms, float(pts), dev)
    stats = None
    if rank == 0:
        # a warm step, as in the timed region: the hints are those of the step before
        one_step(W - 1, dev_sets[W - 1])
        ctx.set_options(collect_stats=1)
        ctx.stats(reset=True)
        one_step(W, dev_sets[W])
        stats = ctx.stats(reset=True)
        ctx.set_options(collect_stats=0)
    ctx.sync()
    value = pts_all / (total_ms / 1e3)
    peak, peak_kind = measured_peak()
    fast_avg_ms = float(np.mean(fast_ms))
    pts_per_step = pts / K
    achieved = BYTES_FUSED * pts_per_step / (fast_avg_ms / 1e3) / 1e9
    traffic = profile_traffic(args.workload)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 coords / f32 Newton+fields" if xi_dtype == ovs.OVS_F32 else "f64",
        "data": "synthetic (seeded generator, shapes of the stated workload)",
        "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "points_per_step": pts_per_step,
                   "guess": guess_label(guess_choice), "parallelism": f"replicas x{world}",
                   "l2": "flushed (256 MB write) between timed steps", "timing": "per-step CUDA events, steps enqueued back to back",
                   "call": "ovs_set_motion per grid + ovs_assemble_interpolate per step",
                   "launch": ("CUDA graph per step (captured once)" if tuning["launch"] == ovs.OVS_LAUNCH_GRAPH
                              else "direct launches") + ", persistent kernels, shapes autotuned, launch mode "
                             "picked on the warm-up steps (L2 flushed)",
                   "tuning": tuning, "grids": len(sc.grids), "sets_per_step": len(dev_sets[W]),
                   "distinct_time_steps": n_distinct},
        "hbm_frac_model": value / world * BYTES_POINT / (peak * 1e9),
        "breakdown_ms_per_step": {"k_assemble (with the interpolation of its points)": fast_avg_ms,
                                  "k_slow + k_slow_tail (with the interpolation of their points)":
                                      float(np.mean(slow_ms))},
        "launch_modes_ms_per_step": {"graph": mode_ms["graph"], "direct": mode_ms["direct"],
                                     "direct_traced": float(np.mean(traced_ms)),
                                     "separate_calls": float(np.mean(sep_ms))},
        "roofline": {"kernel": "k_assemble", "bound": "hbm", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": f"{peak_kind} hbm_gbs (copy)", "bytes_per_point": BYTES_FUSED,
                     "traffic": traffic},
        "e2e": {"value": pts_all / (e2e_total / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d // K,
                "d2h_bytes_per_step": d2h // K,
                "how": "a time loop through the C ABI: per step one H2D copy of its node ids (pinned), "
                       "ovs_set_motion per grid + ovs_assemble_interpolate, D2H of u, v, w, p and status (pinned); "
                       "copies on two copy streams, three device buffer sets in turn, so that step s+1's "
                       "copy-in and step s-1's copy-out overlap step s's kernels; host wall clock over the K "
                       "steps, L2 flushed once before",
                "serial_ms_per_step": e2e_ref},
        "gpu_launches": 3 * K,  # per step: k_assemble, k_slow, k_slow_tail (all interpolating)
        "clocks": ck,
        "walk_stats": stats,
        "plain_unbatched_ms_per_step": unbatched_ms,
        "batched_over_unbatched": unbatched_ms / (total_ms / K),
        "learned_vs_plain": learned,
        "interp_matrix": matrix,
        "interface_flux": fluxes,
        "hole_cut": holes,
        "interleaved_fields": interleaved,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sc, inputs[W], args.cpu_sample)
    return line


def end_to_end(ctx, lib, inputs, host_sets, dev_sets, prep, layout, max_pts, xi_dtype, fdt, W, K, flush, stream,
               dev, ovs, torch):
    """End to end: steps W .. W+K-1 from pinned host node ids to pinned host outputs.  The headline drives the
    C ABI as a C caller's time loop would (structs marshalled once; one H2D copy of the step's node ids on a copy
    stream; the library's calls on its stream after that copy; the D2H copies of u, v, w, p and status on a
    second copy stream after the call; three device buffer sets in turn, so that copies of neighbouring steps
    overlap a step's kernels), timed by the host wall clock over the K steps.  For reference, per-step
    synchronous figures (ms per step): the same C-ABI calls with each step's copies and kernels in sequence, and
    the Python binding (one copy per set, the binding's marshalling on every call).  Returns (total ms,
    H2D bytes, D2H bytes, references)."""
    ctypes_ = __import__("ctypes")
    host_ids = [torch.cat([ids for _, ids, _ in host_sets[s]]).pin_memory() for s in range(W + K)]
    nb = 3  # device buffer sets in turn (with two, a step's call waited on the copy-out of the step two before)
    dstage = [torch.empty(max_pts, dtype=torch.int32, device=dev) for _ in range(nb)]
    ddon = [ctx.alloc_donors(max_pts, xi_dtype) for _ in range(nb)]
    # a step's four output fields side by side in one buffer (u of its n points, then v, w, p), so that one copy
    # brings them back
    dout = [torch.empty(4 * max_pts, dtype=fdt, device=dev) for _ in range(nb)]
    hout = [torch.empty(4 * max_pts, dtype=fdt).pin_memory() for _ in range(nb)]
    hstat = [torch.empty(max_pts, dtype=torch.uint8).pin_memory() for _ in range(nb)]
    # each step's structs, marshalled before timing as a C caller holds them
    call_args = []
    for k in range(K):
        s, b = W + k, k % nb
        views, off = [], 0
        for r, ids, dn in dev_sets[s]:
            m = int(ids.numel())
            views.append((r, dstage[b][off:off + m], dn))
            off += m
        n = off
        dview = {"grid": ddon[b]["grid"][:n], "cell": ddon[b]["cell"][:n], "xi": ddon[b]["xi"][:3 * n],
                 "status": ddon[b]["status"][:n], "xi_dtype": xi_dtype, "n": n}
        farr, ostruct, _ = ctx._fields_structs(layout[0], n, [dout[b][c * n:(c + 1) * n] for c in range(4)])
        call_args.append((s, b, n, ovs.make_sets(views), len(views), ovs.Context.donors_struct(dview), farr, ostruct,
                          dview))

    def check(rc):
        if rc != ovs.OVS_OK:
            raise ovs.OvsError(rc, ovs.ovs_last_error(ctx.ctx))

    def c_call(k):
        s, b, n, sarr, ns, dstruct, farr, ostruct, _ = call_args[k]
        for gid, _, ptrs in prep[s][0]:
            check(lib.ovs_set_motion(ctx.ctx, gid, *ptrs))
        check(lib.ovs_assemble_interpolate(ctx.ctx, sarr, ns, ctypes_.byref(dstruct), farr, len(farr),
                                           ctypes_.byref(ostruct)))

    def copy_out(k):
        s, b, n = call_args[k][:3]
        hout[b][:4 * n].copy_(dout[b][:4 * n], non_blocking=True)
        hstat[b][:n].copy_(ddon[b]["status"][:n], non_blocking=True)

    h2d_st, d2h_st = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(K)]
    ev_call = [torch.cuda.Event() for _ in range(K)]
    ev_out = [torch.cuda.Event() for _ in range(K)]
    flush.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    host_s = 0.0
    for k in range(K):
        th = time.perf_counter()
        s, b, n = call_args[k][:3]
        with torch.cuda.stream(h2d_st):
            if k >= nb:
                h2d_st.wait_event(ev_call[k - nb])  # the call that read this staging buffer has run
            dstage[b][:n].copy_(host_ids[s], non_blocking=True)
            ev_in[k].record(h2d_st)
        stream.wait_event(ev_in[k])
        if k >= nb:
            stream.wait_event(ev_out[k - nb])  # this buffer set's outputs of step k-2 are copied out
        c_call(k)
        ev_call[k].record(stream)
        with torch.cuda.stream(d2h_st):
            d2h_st.wait_event(ev_call[k])
            copy_out(k)
            ev_out[k].record(d2h_st)
        host_s += time.perf_counter() - th
    torch.cuda.synchronize()
    total = (time.perf_counter() - t0) * 1e3
    h2d = sum(4 * call_args[k][2] for k in range(K))
    d2h = sum(call_args[k][2] * (4 * dout[0].element_size() + 1) for k in range(K))
    # per-step synchronous references
    serial, binding = [], []
    for k in range(K):
        s, b, n = call_args[k][:3]
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        dstage[b][:n].copy_(host_ids[s], non_blocking=True)
        c_call(k)
        copy_out(k)
        torch.cuda.synchronize()
        serial.append((time.perf_counter() - t) * 1e3)
    for k in range(K):
        s, b, n = call_args[k][:3]
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        sets = [(r, ids.to(dev, non_blocking=True), dn) for r, ids, dn in host_sets[s]]
        for gid, mo in enumerate(inputs[s][0]):
            ctx.set_motion(gid, mo.R, mo.c, mo.V, mo.omega)
        ctx.assemble_interpolate(sets, layout[0], donors=call_args[k][8],
                                 out=[dout[b][c * n:(c + 1) * n] for c in range(4)])
        copy_out(k)
        torch.cuda.synchronize()
        binding.append((time.perf_counter() - t) * 1e3)
    ref = {"c_abi_synchronous": float(np.median(serial)), "python_binding_synchronous": float(np.median(binding)),
           "pipelined_host_ms_per_step": host_s * 1e3 / K,
           "note": "synchronous figures: medians, each step's H2D copy, calls and D2H copies in sequence, then a "
                   "synchronisation; pipelined_host_ms_per_step: the host's mean time per step in the headline loop "
                   "(enqueueing, and waiting for a free parameter staging buffer)"}
    return total, h2d, d2h, ref


GUESS_WIDTHS = (32, 64)
GUESS_SAMPLES = 2_000_000
GUESS_EPOCHS = 40


def train_and_pick_guess(args, sc, ctx, gids, sets, fields, donors, outs, ovs, torch):
    """Train every body grid's guess network (3-H-H-3 SiLU, GUESS_SAMPLES samples of the grid itself, by the
    library's kernels) for each width of GUESS_WIDTHS, then let the library's guess autotuner (ovs_autotune_guess)
    pick one width or none on `sets`: its score is one cold plus one warm call.  Leaves options.guess = MLP and the
    chosen networks installed."""
    import gen

    bodies = [gi for gi, g in enumerate(sc.grids) if g.role == 1]
    params, train = {}, {}
    for H in GUESS_WIDTHS:
        t0 = time.perf_counter()
        losses = []
        per_grid = [None] * len(gids)
        for gi in bodies:
            g = sc.grids[gi]
            cells, xi = gen.mlp_training_samples(config_index(args.workload), g, GUESS_SAMPLES)
            rng = np.random.default_rng(100 + gi)
            init = np.concatenate([rng.normal(0, 0.8, 3 * H), np.zeros(H), rng.normal(0, 1 / np.sqrt(H), H * H),
                                   np.zeros(H), rng.normal(0, 1 / np.sqrt(H), 3 * H), np.zeros(3)]).astype(np.float32)
            losses.append(ctx.train_guess(gids[gi], cells, xi.astype(np.float32), init, hidden=H, epochs=GUESS_EPOCHS,
                                          batch=8192, lr=3e-3, lr_final=1e-5))
            p = torch.empty(ovs.ovs_guess_param_count(H), dtype=torch.float32, device=ctx.device)
            assert ovs.ovs_guess_get_params(ctx.ctx, gids[gi], p.data_ptr()) == H
            per_grid[gi] = p
        torch.cuda.synchronize()
        params[H] = per_grid
        train[H] = {"train_s": time.perf_counter() - t0, "train_mse": float(np.mean(losses))}
    ctx.set_options(guess=ovs.OVS_GUESS_MLP)
    hidden = list(GUESS_WIDTHS) + [0]
    cand = [params[H] for H in GUESS_WIDTHS] + [[None] * len(gids)]
    best, ms = ctx.autotune_guess(sets, fields, hidden, cand, donors=donors, out=outs, reps=3)
    return {"network": "3-H-H-3 SiLU per body grid, FP16 tensor-core inference (FP32 accumulation in layers 1 and 3)"
                       f" inside k_assemble, trained by the library's kernels on {GUESS_SAMPLES} samples x "
                       f"{GUESS_EPOCHS} epochs per body grid",
            "bodies": len(bodies), "training": {str(H): v for H, v in train.items()},
            "autotune_guess_ms_cold_warm": {str(h): list(m) for h, m in zip(hidden, ms)},
            "chosen_width": hidden[best]}


def learned_vs_plain(choice, ctx, dev_sets, one_step, timed, stream, flush, K, W, ovs, torch):
    """The same steps with the plain start (previous donor, else the control cell) and the learned one (previous
    donor, else the network), warm (a time loop: every pass from reset hints plus the W warm-up steps) and cold (no
    previous donors: a step after ovs_reset_hints), in the headline's launch mode; mean ms per step, L2 flushed
    before each step; walk statistics from one more pass of each.  Leaves options.guess = MLP."""
    out = dict(choice)

    def warm(mode):
        ctx.set_options(guess=mode)
        _, ms, _, _, _ = timed(True, trace=False)
        return float(np.mean(ms))

    def cold(mode, steps):
        ctx.set_options(guess=mode)
        e0 = [torch.cuda.Event(enable_timing=True) for _ in steps]
        e1 = [torch.cuda.Event(enable_timing=True) for _ in steps]
        for e in e0 + e1:
            e.record(stream)
        torch.cuda.synchronize()
        for k, s in enumerate(steps):
            flush.zero_()
            ovs.ovs_reset_hints(ctx.ctx)
            e0[k].record(stream)
            one_step(s, dev_sets[s])
            e1[k].record(stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in zip(e0, e1)]))

    def stats(mode, is_cold):
        ctx.set_options(guess=mode, collect_stats=1)
        ovs.ovs_reset_hints(ctx.ctx)
        for s in range(W):
            one_step(s, dev_sets[s])
        if is_cold:
            ovs.ovs_reset_hints(ctx.ctx)
        ctx.stats(reset=True)
        one_step(W, dev_sets[W])
        st = ctx.stats(reset=True)
        ctx.set_options(collect_stats=0)
        return st

    cold_steps = list(range(W, W + min(K, 5)))
    res = {}
    for name, mode in (("plain", ovs.OVS_GUESS_HINT), ("learned", ovs.OVS_GUESS_MLP)):
        res[name] = {"warm_ms_per_step": warm(mode), "cold_ms_per_step": cold(mode, cold_steps),
                     "warm_stats": stats(mode, False), "cold_stats": stats(mode, True)}
    ctx.set_options(guess=ovs.OVS_GUESS_MLP)
    out.update(res)
    out["warm_plain_over_learned"] = res["plain"]["warm_ms_per_step"] / res["learned"]["warm_ms_per_step"]
    out["cold_plain_over_learned"] = res["plain"]["cold_ms_per_step"] / res["learned"]["cold_ms_per_step"]
    return out


# ----------------------------------------------------------------------------------------------------- oracle
def oracle_points_per_s(sc, motions, fsets, sample_n: int, rng, grids=None):
    import oracle

    if grids is None:
        # the oracle's grids, every receiver grid's node coordinates and the donor fields in FP64 (the oracle's
        # precision): inputs, formed once before any timing
        fields64 = [{k: np.asarray(f[k], dtype=np.float64) for k in ("u", "v", "w", "p")} for f in sc.fields]
        grids = ([oracle.OracleGrid.from_gen(g) for g in sc.grids], [g.xyz() for g in sc.grids], fields64)
    ogrids, xyz, fields64 = grids
    frames = [oracle.frame_of(m) for m in motions]
    sizes = np.array([len(s.node_ids) for s in fsets], dtype=np.int64)
    tot = sizes.sum()
    t0 = time.perf_counter()
    n = 0
    for s, sz in zip(fsets, sizes):
        k = int(round(sample_n * sz / tot)) if sample_n < tot else int(sz)
        if k == 0:
            continue
        ids = s.node_ids if k >= sz else np.sort(rng.choice(s.node_ids, size=k, replace=False))
        d = oracle.assemble(ogrids, frames, xyz[s.receiver], s.receiver, ids, s.donors)
        oracle.interpolate(d, fields64, frames, s.receiver)
        n += len(ids)
    return n, time.perf_counter() - t0, grids


def cpu_baseline(sc, step_input, sample_n: int):
    import oracle

    motions, fsets = step_input
    rng = np.random.default_rng(7)
    tot = sum(len(s.node_ids) for s in fsets)
    if sample_n <= 0:
        sample_n = min(tot, 400_000)
    n, dt, grids = oracle_points_per_s(sc, motions, fsets, sample_n, rng)
    cores = oracle.num_threads()
    # the same oracle on one core, on a smaller sample (about 3 s of work)
    n1_want = int(max(2_000, min(25_000, 3.0 * n / dt / max(1, cores))))
    oracle.set_num_threads(1)
    try:
        n1, dt1, _ = oracle_points_per_s(sc, motions, fsets, n1_want, rng, grids)
    finally:
        oracle.set_num_threads(0)
    return {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} of the {tot} fringe points of one step (seeded random subset), bins built before timing",
            "seconds": dt,
            "single_core": {"value": n1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"{n1} fringe points of the same step (seeded random subset)", "seconds": dt1}}


def run_reference(args, rank, world):
    import oracle

    if rank != 0:
        return None
    oracle.build()
    sc = build_workload(args.workload)
    K, W = args.steps, args.warmup
    inputs, _ = step_inputs(sc, W + K, DISTINCT_STEPS.get(args.workload, 0), workers=host_workers())
    rng = np.random.default_rng(11)
    # each step a bounded sample of its fringe points, sized from a first probe step so that the K + W steps take
    # about 90 s of oracle time in all (at most 20 k points a step)
    n0, dt0, grids = oracle_points_per_s(sc, inputs[0][0], inputs[0][1], 2_000, rng, None)
    per_step = int(max(500, min(20_000, 90.0 * (n0 / max(dt0, 1e-9)) / max(1, W + K))))
    for s in range(W):
        _, _, grids = oracle_points_per_s(sc, inputs[s][0], inputs[s][1], per_step, rng, grids)
    tot_n, tot_t = 0, 0.0
    for s in range(W, W + K):
        n, dt, grids = oracle_points_per_s(sc, inputs[s][0], inputs[s][1], per_step, rng, grids)
        tot_n += n
        tot_t += dt
    value = tot_n / tot_t
    full = sum(len(x.node_ids) for x in inputs[W][1])
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": tot_t / K * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator)",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}",
                       "points_per_step": tot_n / K, "full_points_per_step": full},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{per_step} seeded random fringe points per step of {full}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        # the oracle runs on the host of rank 0 only; other ranks exit without work
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch

        torch.distributed.init_process_group("nccl")
    line = run_ovs(args, rank, world, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
