"""Benchmark: PERCH successor evaluation (renders + edge costs) per second at
640x480 on one GB300, plus time to the optimal scene.

One step = one pass of the hot path over one expansion batch of the
640x480 workload (three ~10k-triangle meshes, 50 x 50 x 16 pose grid): parent
z-buffers and residual sets for three parents (the root, one object placed,
two objects placed), then the successor evaluation of all their children
(120k + 80k + 40k = 240k hypotheses) in one launch. Inputs are resident on
the device when the timed region starts; L2 is flushed (a 256 MiB write)
before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank evaluates its own batch (independent
problems, weak scaling); there is no data-path collective. The reference arm
(--impl reference) times the CPU oracle on a bounded sample of the same batch.
"""
from __future__ import annotations

import argparse
import json
import math
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

from paper_1510_05613_gb300 import synth  # noqa: E402

METRIC = "successor renders+costs/sec at 640x480; time to optimal scene (1 GB300)"
UNIT = "hypotheses/s"
L2_FLUSH_BYTES = 256 << 20
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128
WORKLOADS = {
    "c2": "640x480 fx=525, 3 procedural meshes (box/cylinder/superquadric, ~10k triangles), 50x50x16 pose grid, "
          "sigma 3 mm, 5% dropout, delta 1 cm; one expansion batch = root + 1-object + 2-object parents, "
          "240000 hypotheses",
    "icp": "640x480 fx=525, the three ~10k-triangle meshes of c2 observed off the 50x50x16 grid (up to half a "
           "step in x, y and yaw), sigma 3 mm, 5% dropout, delta 1 cm; one step = ICP refinement (pairs within "
           "2 cm, at most 20 fits) of every successor of the root expansion, 120000 hypotheses",
    "c3": "640x480 fx=525, heavy occlusion: 5 of 8 procedural meshes of 2k-50k triangles, one object >70% occluded, "
          "50x50x16 pose grid, sigma 3 mm, 5% dropout, delta 1 cm; one expansion batch = the children of a "
          "2-object parent, 120000 hypotheses",
}


def c2_batch(wl):
    """(parents, hyp_parent, hyps) of one expansion batch of the 640x480
    workload: the root's children (every pose of every type), the children of
    the first ground-truth object, and the last-level children of the first
    two ground-truth objects."""
    parents = [wl.gt[:0], wl.gt[:1], wl.gt[:2]]
    groups = []
    for p, parent in enumerate(parents):
        rem = sorted(set(_remaining(wl.mesh_multiset, parent)))
        h = synth.all_hypotheses(wl.grid, rem)
        groups.append((np.full(len(h), p, np.int32), h))
    hp = np.concatenate([g[0] for g in groups])
    hyps = np.concatenate([g[1] for g in groups])
    return parents, hp, hyps


def c3_batch(wl):
    """(parents, hyp_parent, hyps) of one expansion of the heavy-occlusion
    workload: the children of the first two ground-truth objects, i.e. every
    pose of the three remaining (uneven) meshes, 120k hypotheses."""
    parents = [wl.gt[:2]]
    rem = sorted(set(_remaining(wl.mesh_multiset, parents[0])))
    h = synth.all_hypotheses(wl.grid, rem)
    return parents, np.zeros(len(h), np.int32), h


def _remaining(multiset, parent):
    rem = list(multiset)
    for m in parent["mesh"]:
        rem.remove(int(m))
    return rem


def distinct_poses(hyps):
    """The distinct (mesh, ix, iy, iyaw) of a batch, as object records."""
    return np.unique(np.ascontiguousarray(hyps))


def algorithmic_ops(wl, poses, covered, n_new):
    """Lower bound of the arithmetic one evaluation step must do, split by
    kernel. Render (k_render, once per distinct pose): 40 ops per mesh vertex
    (pose + camera transform, projection, snap, reciprocal depth), 20 per
    triangle (edge setup, facing and extent tests, pixel box), 50 per covered
    pixel (3 edge functions, depth interpolation, z-buffer max, reciprocal,
    back-projection and the first delta probe of Eq. (1), which k_render
    decides once per pose). Cost (k_cost, per hypothesis): 10 per pixel of dR
    (parent compare, classification, the counts). Returns (render ops, cost
    ops)."""
    V = np.array([m.n_verts for m in wl.meshes], np.float64)
    T = np.array([m.n_tris for m in wl.meshes], np.float64)
    mi = poses["mesh"].astype(np.int64)
    render = float((40.0 * V[mi] + 20.0 * T[mi]).sum() + 50.0 * np.asarray(covered, np.float64).sum())
    return render, 10.0 * float(np.asarray(n_new, np.float64).sum())


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
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
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def whole_job(local_seconds: float, local_units: float):
    """(max over ranks of the timed seconds, whole-job rate = units of all
    ranks / that time). Every rank processes the same number of units (weak
    scaling); with one rank there is no collective."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return local_seconds, local_units / local_seconds
    ws = dist.get_world_size()
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([local_seconds], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total = float(t.item())
    dist.barrier()
    return total, ws * local_units / total


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def cpu_baseline(wl, parents, hp, hyps, target_s: float = 12.0, seed: int = 0, threads: int = 0):
    """The oracle as it stands on the host cores (threads = 0: all of them),
    on a bounded random sample of the same batch (sample grown until it
    takes about target_s)."""
    import oracle
    w = oracle.World.of(wl)
    threads = threads if threads > 0 else oracle.max_threads()
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(hyps))
    n = max(threads, 16)
    spent, done = 0.0, 0
    while True:
        idx = order[done:done + n]
        t0 = time.perf_counter()
        oracle.eval_batch(w, wl.depth, parents, hp[idx], hyps[idx], wl.K, threads)
        dt = time.perf_counter() - t0
        spent += dt
        done += len(idx)
        if spent >= target_s or done >= len(hyps):
            break
        rate = len(idx) / max(dt, 1e-6)
        n = int(min(max(n * 2, rate * (target_s - spent)), len(hyps) - done))
        n = max(n, 1)
    return {"value": done / spent, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{done} of the {len(hyps)} hypotheses of the batch (uniform random, seed {seed}), "
                      f"{spent:.1f} s on {threads} OpenMP threads"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    wl = synth.workload_c2()
    parents, hp, hyps = c2_batch(wl)
    import oracle
    w = oracle.World.of(wl)
    threads = oracle.max_threads()
    # bounded sample per step, large enough to keep every thread busy
    per = args.ref_sample if args.ref_sample > 0 else 128 * threads
    rng = np.random.default_rng(1)
    times = []
    for s in range(args.warmup + args.steps):
        idx = rng.choice(len(hyps), per, replace=False)
        t0 = time.perf_counter()
        oracle.eval_batch(w, wl.depth, parents, hp[idx], hyps[idx], wl.K, threads)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = per * len(times) / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "reference",
            "config": {"workload": "640x480 fx=525, 3 meshes ~10k triangles, 50x50x16 poses, delta 1 cm; "
                                   f"each step a random {per}-hypothesis sample of the 240k-hypothesis batch",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{per} hypotheses per step, {len(times)} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def c1_time_to_optimum(threads: int):
    """Time to the optimal scene on the 160x120 two-object workload, GPU
    search (warm, second run) beside the oracle's exact uniform-cost search
    on the host cores; both must return the same cost and scene."""
    try:
        import oracle
        from oracle import search
        from paper_1510_05613_gb300 import perch
        wl = synth.workload_c1()
        p = perch.Perch(0)
        p.setup(wl)
        p.perch_search(wl.mesh_multiset, batch_states=16)
        r = p.perch_search(wl.mesh_multiset, batch_states=16)
        p.close()
        w = oracle.World.of(wl)
        t0 = time.perf_counter()
        cost, key, expansions = search.uniform_cost_search(w, wl.depth, wl.grid, wl.mesh_multiset, threads=threads)
        oracle_s = time.perf_counter() - t0
        return {"gpu_s": r["seconds"], "oracle_s": oracle_s, "oracle_cores": threads,
                "cost": r["cost"], "proven_optimal": r["proven_optimal"],
                "same_cost_and_scene": (r["cost"], r["key"]) == (cost, key),
                "expansions": {"gpu": r["expansions"], "oracle": expansions},
                "workload": "160x120 fx=140, box + cylinder (1k/2k triangles), 10x10x8 poses, K=2, delta 1 cm"}
    except Exception as e:  # reported, never fatal to the headline line
        return {"error": f"{type(e).__name__}: {e}"}


def run_ours(args):
    import torch
    from paper_1510_05613_gb300 import perch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    # a dedicated stream: torch's default stream has the NULL handle, which the
    # library would read as "create your own stream"
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    wl = synth.workload_c3() if args.workload == "c3" else synth.workload_c2()
    parents, hp, hyps = c3_batch(wl) if args.workload == "c3" else c2_batch(wl)
    if args.max_hyps and args.max_hyps < len(hyps):  # reduced batch (profiling case)
        keep = np.linspace(0, len(hyps) - 1, args.max_hyps).astype(np.int64)
        hp, hyps = hp[keep], hyps[keep]
    n_hyp = len(hyps)
    p = perch.Perch(local, stream=stream.cuda_stream)
    p.setup(wl)

    P, plen, stride = perch.Perch.pack_parents(parents)
    tP = torch.from_numpy(P.view(np.int16).reshape(-1).copy()).to(dev)
    tplen = torch.from_numpy(plen).to(dev)
    thp = torch.from_numpy(hp).to(dev)
    th = torch.from_numpy(np.ascontiguousarray(hyps).view(np.int16).reshape(-1).copy()).to(dev)
    tout = torch.zeros(n_hyp * 7, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    if args.threads:
        p.perch_set_threads(args.threads)
        widths = [args.threads] * len(wl.meshes)
    else:
        widths = p.perch_autotune(args.tune_sample) if not args.no_autotune else None

    # the headline renders every hypothesis; the exact shortcut is measured after
    p.perch_set_shortcut(False)

    def step():  # the whole evaluation sequence as one CUDA-graph launch (or direct launches)
        if args.no_graph:
            p.perch_eval_successors_dev(tP, stride, tplen, thp, th, wl.K, tout)
        else:
            p.perch_eval_graph(tP, stride, tplen, thp, th, wl.K, tout)

    for _ in range(max(args.warmup, 3)):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    eval_ms, prep_ms = [], []
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            flush.fill_(k)
            evs[k][0].record(stream)
            step()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    # the same sequence without the graph, to time its phases with the
    # library's events on its stream (parent prep; grouping; the per-mesh
    # render launches; the per-mesh cost launches)
    phases, shared = [], False
    for k in range(max(3, args.steps // 2)):
        flush.fill_(k)
        p.perch_eval_successors_dev(tP, stride, tplen, thp, th, wl.K, tout)
        a, b = p.perch_last_timing()
        prep_ms.append(a)
        eval_ms.append(b)
        ph, shared = p.perch_last_phase_times()
        phases.append(ph)
    torch.cuda.synchronize()
    step_ms = [s.elapsed_time(e) for s, e in evs]
    total_s, value = whole_job(sum(step_ms) / 1e3, n_hyp * args.steps)
    phase_ms = np.mean(np.array(phases), 0)

    rec = tout.view(-1, 7).cpu().numpy()
    # pixels each distinct pose covers: its record against the empty parent
    poses = distinct_poses(hyps)
    covered = perch.records(p.perch_eval_successors([wl.gt[:0]], np.zeros(len(poses), np.int32), poses, wl.K))[:, 4]
    if not shared:  # one render per hypothesis (a batch of one parent): k_eval renders and costs each
        covered = covered[np.searchsorted(poses, np.ascontiguousarray(hyps))]
    render_ops, cost_ops = algorithmic_ops(wl, poses if shared else hyps, covered, rec[:, 4])
    if not shared:  # both in the one kernel, timed as the render phase
        render_ops, cost_ops = render_ops + cost_ops, 0.0
    peaks = _measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    peak_tops = n_sm * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
    eval_s = statistics.mean(eval_ms) / 1e3
    render_s = phase_ms[2] / 1e3
    achieved = render_ops / render_s / 1e12
    achieved_cost = cost_ops / max(phase_ms[3] / 1e3, 1e-9) / 1e12

    # end to end through the C ABI with host buffers (pinned)
    def pin(a):
        a = np.ascontiguousarray(a)
        t = torch.from_numpy(a.view(np.uint8).reshape(-1)).pin_memory()
        return t.numpy().view(a.dtype).reshape(a.shape)

    h_depth = pin(wl.depth)
    h_hyps, h_hp = pin(hyps), pin(hp)
    e2e_t = []
    for k in range(0 if args.no_e2e else 2 + max(2, args.steps // 2)):
        t0 = time.perf_counter()
        p.perch_set_observation(h_depth, wl.cam.fxfycxcy, wl.cam.T_wc, wl.delta)
        out = p.perch_eval_successors(parents, h_hp, h_hyps, wl.K)
        t1 = time.perf_counter()
        if k >= 2:
            e2e_t.append(t1 - t0)
    e2e_bytes_in = h_depth.nbytes + h_hyps.nbytes + h_hp.nbytes + P.nbytes + plen.nbytes
    if not e2e_t:
        out, e2e_t = np.zeros(n_hyp, perch.COST), [float("nan")]
    e2e = {"value": ws * n_hyp / statistics.mean(e2e_t), "unit": UNIT, "h2d_bytes_per_step": int(e2e_bytes_in),
           "d2h_bytes_per_step": int(out.nbytes),
           "includes": "perch_set_observation (depth upload, cloud + grid build) + perch_eval_successors "
                       "(batch upload, evaluation, record download)"}
    consistent = bool(np.array_equal(perch.records(out), rec.astype(np.int64)))

    # the same batch with the exact shortcut (records identical, checked)
    p.perch_set_shortcut(True)
    for _ in range(3):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    sc_ms = []
    for k in range(args.steps):
        flush.fill_(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        sc_ms.append(e0.elapsed_time(e1))
    p.perch_eval_successors_dev(tP, stride, tplen, thp, th, wl.K, tout)
    n_short, _ = p.perch_shortcut_stats()
    sc_same = bool(np.array_equal(tout.view(-1, 7).cpu().numpy(), rec))
    shortcut = {"value": ws * n_hyp / (statistics.mean(sc_ms) / 1e3), "unit": UNIT,
                "ms_per_step": statistics.mean(sc_ms), "fraction_shortcut": n_short / n_hyp,
                "records_identical": sc_same,
                "meaning": "exact shortcut on: hypotheses far from the observation and from the parent's render get "
                           "their record from a per-pose solo render table instead of being rasterised again"}

    # time to the optimal scene (uniform-cost search, exact; shortcut on),
    # over the full tree and over the tree with the meshes' rotational
    # symmetry (Sec. IV-E), with the pose accuracy of both (Sec. V-D)
    search = None
    if not args.no_search:
        from paper_1510_05613_gb300 import accuracy
        gt_key = tuple(sorted((int(o["mesh"]), int(o["ix"]), int(o["iy"]), int(o["iyaw"])) for o in wl.gt))

        def one_search(heur=0):
            r = p.perch_search(wl.mesh_multiset, batch_states=args.batch_states, time_limit_s=args.search_limit,
                               heuristics=heur)
            return {"seconds": r["seconds"], "proven_optimal": r["proven_optimal"], "cost": r["cost"],
                    "expansions": r["expansions"], "successors": r["successors"],
                    "found_ground_truth": r["key"] == gt_key, "batch_states": args.batch_states,
                    "pose_accuracy": accuracy.report([r], [wl], wl.meshes)}

        search = one_search()
        p.perch_set_symmetry(wl.meshes)
        search["symmetric"] = one_search()
        search["symmetric"]["symmetry_orders"] = [int(m.sym) for m in wl.meshes]
        p.perch_set_symmetry(None)
        # the same search keeping each pose's render across expansions (the
        # render cache: identical records, only poses not seen before rendered)
        p.perch_set_render_cache(True)
        search["render_cache"] = one_search()
        p.perch_set_symmetry(wl.meshes)
        search["render_cache_symmetric"] = one_search()
        p.perch_set_symmetry(None)
        # and with a greedy incumbent first (heuristics bit 4: the same optimum)
        search["render_cache_incumbent"] = one_search(16)
        p.perch_set_render_cache(False)

    base = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(wl, parents, hp, hyps, target_s=args.cpu_seconds)
        one = cpu_baseline(wl, parents, hp, hyps, target_s=args.cpu_seconds / 4, seed=1, threads=1)
        base["single_core"] = {"value": one["value"], "unit": one["unit"], "sample": one["sample"]}
        base["time_to_optimum_c1"] = c1_time_to_optimum(base["cores"])

    if rank == 0:
        cl = clocks.summary()
        # DRAM bytes per step of the dominant kernel (k_render with shared
        # renders, else k_eval), from the committed summary of its ncu capture
        traffic = (measured_traffic("perch_kernels.cu",
                                    f"{'k_render' if shared else 'k_eval'}_{args.workload}_launches.md")
                   if not args.max_hyps else None)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload],
                       "hypotheses_per_step": n_hyp, "l2": "flushed (256 MiB write) before every timed step",
                       "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "alu", "kernel": "k_render" if shared else "k_eval", "achieved": achieved,
                         "peak": peak_tops, "unit": "Tops/s", "frac": achieved / peak_tops,
                         "traffic": traffic,
                         "ops_per_step": render_ops, "render_ms": float(phase_ms[2]),
                         "distinct_poses": int(len(poses)),
                         "peak_from": f"{n_sm} SMs x {FP32_LANES_PER_SM} lanes x {sm_max:.0f} MHz "
                                      "(sm_max_mhz of MEASURED_PEAKS.json)",
                         "phases_ms": {"parent_prep": float(phase_ms[0]), "grouping": float(phase_ms[1]),
                                       "render": float(phase_ms[2]), "cost": float(phase_ms[3])},
                         "cost_kernel": {"kernel": "k_cost", "ops_per_step": cost_ops, "achieved": achieved_cost,
                                         "frac": achieved_cost / peak_tops},
                         "eval_ms": statistics.mean(eval_ms), "prep_ms": statistics.mean(prep_ms)},
            "hbm": hbm_fields(n_hyp / eval_s, traffic / n_hyp if traffic else None),
            "paper_context": PAPER_CONTEXT,
            "e2e": e2e, "e2e_matches_device_records": consistent,
            "gpu_launches": ((14 + 2 * len(wl.meshes)) if shared else (8 + len(wl.meshes))) * args.steps,
            "launch": {"graph": not args.no_graph, "persistent_per_mesh": True, "autotuned_threads": widths,
                       "config_in_use": dict(zip(("render_threads", "render_inline_pixels", "cost_threads"),
                                                 p.perch_launch_config()),
                                             render_bin_depth=p.perch_launch_bin_depths(),
                                             cost_stages=p.perch_launch_cost_stages()),
                       "shared_renders": shared},
            "clocks": cl,
            "time_to_optimum": search,
            "shortcut": shortcut,
            "cpu_baseline": base,
        }
        print(json.dumps(line), flush=True)
    p.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


class MemoryGuard:
    """Polls this process's resident memory; past `frac` of the host's RAM it
    prints an error line and exits, so a search that keeps too many states
    stops cleanly instead of exhausting the host. Records the peak."""

    def __init__(self, frac: float = 0.6):
        self.peak = 0
        self.limit = None
        try:
            with open("/proc/meminfo") as f:
                total_kb = int(next(l for l in f if l.startswith("MemTotal")).split()[1])
            self.limit = int(total_kb * 1024 * frac)
        except (OSError, StopIteration, ValueError):
            pass
        self.stop = threading.Event()

    def _rss(self):
        try:
            with open("/proc/self/statm") as f:
                return int(f.read().split()[1]) * os.sysconf("SC_PAGE_SIZE")
        except (OSError, ValueError):
            return 0

    def _run(self):
        while not self.stop.wait(0.5):
            r = self._rss()
            self.peak = max(self.peak, r)
            if self.limit and r > self.limit:
                print(json.dumps({"error": f"host memory {r / 2**30:.1f} GiB above the guard "
                                           f"{self.limit / 2**30:.1f} GiB; run stopped"}), flush=True)
                os._exit(3)

    def __enter__(self):
        threading.Thread(target=self._run, daemon=True).start()
        return self

    def __exit__(self, *a):
        self.stop.set()
        self.peak = max(self.peak, self._rss())


def run_c5(args):
    """Many scenes at once: one exact search per scene, all expansions packed
    into shared evaluation launches (perch_search_multi). Reports aggregate
    hypotheses/s over the whole run and per-scene time to the optimum."""
    import torch
    from paper_1510_05613_gb300 import accuracy, perch

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t0 = time.perf_counter()
    wls = synth.workloads_c5(args.scenes)
    gen_s = time.perf_counter() - t0
    p = perch.Perch(0)
    p.setup(wls[0])
    for s, wl in enumerate(wls[1:], 1):
        p.perch_set_scene(s, wl.depth)
    p.perch_autotune(args.tune_sample)
    if args.symmetric:
        p.perch_set_symmetry(wls[0].meshes)
    if args.render_cache:
        p.perch_set_render_cache(True)
    with ClockSampler(0) as clocks, MemoryGuard() as mem:
        t0 = time.perf_counter()
        res = p.perch_search_multi(list(range(len(wls))), [wl.mesh_multiset for wl in wls],
                                   batch_states=args.batch_states, max_hyps_per_launch=args.launch_hyps,
                                   time_limit_s=args.search_limit, w=args.w, heuristics=args.heuristics)
        wall = time.perf_counter() - t0
    succ = sum(r["successors"] for r in res)
    done = [r["seconds"] for r in res if r["cost"] >= 0 and r["seconds"] > 0]
    line = {"metric": METRIC, "value": succ / wall, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": 1e3 * wall, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{len(wls)} independent 640x480 scenes of 2-6 objects (8 procedural meshes of "
                                   "2k-50k triangles), 50x50x16 poses, sigma 3 mm, 5% dropout, delta 1 cm; exact "
                                   "search per scene, expansions of all scenes packed into shared launches",
                       "scenes": len(wls), "launch_hyps": args.launch_hyps, "batch_states": args.batch_states,
                       "time_limit_s": args.search_limit, "generation_s": gen_s},
            "search": {"w": args.w, "heuristics": args.heuristics, "symmetric": bool(args.symmetric),
                       "render_cache": bool(args.render_cache),
                       "meaning": ("cost <= w x optimum (Focal-MHA*, Theorem 2)" if args.w > 1 else "optimal") +
                                  (" of the tree with each mesh's symmetric yaws merged" if args.symmetric else "")},
            "scenes_finished": len(done),
            "ground_truth_found": sum(
                r["key"] == tuple(sorted((int(o["mesh"]), int(o["ix"]), int(o["iy"]), int(o["iyaw"])) for o in wl.gt))
                for r, wl in zip(res, wls)),
            "time_to_optimum_p50_s": float(np.percentile(done, 50)) if done else None,
            "time_to_optimum_p99_s": float(np.percentile(done, 99)) if done else None,
            "successors": succ, "wall_s": wall, "host_peak_rss_gib": mem.peak / 2**30,
            "search_seconds": dict(zip(("device_eval", "absorb_records", "select_states"), p.perch_search_times())),
            "pose_accuracy": accuracy.report(res, wls, wls[0].meshes),
            "hbm": hbm_fields(succ / wall, None), "paper_context": PAPER_CONTEXT, "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)
    p.close()
    return 0


# The paper's own timings (Sec. V-E), quoted with the hardware it states.
# They time whole searches (ICP refinement and MPI distribution included),
# not this benchmark's metric, so vs_baseline stays null.
PAPER_CONTEXT = {
    "source": "Sec. V-E (occlusion dataset, Sec. V-A)",
    "hardware": "2 x AWS m4.10xlarge (a 40-core virtual CPU each), MPI",
    "mean_planning_time_per_scene_s": 6.5 * 60,
    "mean_hypotheses_rendered_per_scene": 15564,
    "derived_hypotheses_per_s": 15564 / (6.5 * 60),
    "time_limit_per_scene_s": 15 * 60,
    "comparable": False,
}
ALG_BYTES_PER_HYP = 36  # 8-byte object in, 28-byte cost record out


def hbm_fields(hyps_per_s: float, traffic_per_hyp: float | None):
    """DRAM rate of the evaluation against the measured HBM copy peak:
    measured bytes per hypothesis when an ncu capture of the current kernel
    is committed, else the algorithmic 36 bytes."""
    peak = float(_measured_peaks().get("hbm_gbs", 6800.0))
    per = traffic_per_hyp if traffic_per_hyp is not None else float(ALG_BYTES_PER_HYP)
    gbs = hyps_per_s * per / 1e9
    return {"achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak, "bytes_per_hypothesis": per,
            "basis": "ncu DRAM bytes of k_eval" if traffic_per_hyp is not None else "algorithmic bytes",
            "meaning": "tables, observation index and parent z-buffers stay in L2; HBM carries the batch in and "
                       "the records out"}


CNN_TRAIN_FLOP_PER_CROP = 297.1e6  # forward 100.7 MFLOP + weight and data gradients (no data gradient of layer 1)
CNN_FWD_FLOP_PER_CROP = 100.7e6


def measured_traffic(kernel_file: str, summary: str):
    """DRAM bytes per step from a committed ncu summary, if it was taken on
    the current source of the kernel (its sha256 recorded there), else None."""
    import hashlib
    try:
        src = open(os.path.join(ROOT, "paper_1510_05613_gb300", "csrc", kernel_file), "rb").read()
        text = open(os.path.join(ROOT, "profiles", summary)).read()
    except OSError:
        return None
    h = hashlib.sha256(src).hexdigest()
    vals = dict(l.split(":", 1) for l in text.splitlines() if l.startswith(("source_sha256:", "dram_bytes_per_step:")))
    if vals.get("source_sha256", "").strip() != h:
        return None
    try:
        return float(vals["dram_bytes_per_step"])
    except (KeyError, ValueError):
        return None


def run_cnn(args):
    """The heuristic network alone: W warm-up and K timed training steps
    (forward, backward, Adam) of 256 seeded synthetic crops, then forward
    passes of 2048 crops; CUDA events on the network's stream, L2 flushed
    before every timed step. FLOPs per crop: forward 100.7 M, training 297.1 M
    (the network's GEMMs, algorithmic, without padding)."""
    import torch
    from paper_1510_05613_gb300 import heuristic as H
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    n_onehot = 8 * 16
    B = 256
    net = H.new_network(n_onehot, B, seed=3, stream=stream)
    u = synth.uniform(11, B * 64 * 64 * 2)
    crops = torch.from_numpy((u * 7.0 - 4.0).astype(np.float32)).reshape(B, 64, 64, 2).to(torch.bfloat16).cuda()
    onehot = torch.from_numpy((synth.uniform(12, B) * n_onehot).astype(np.int32)).cuda()
    target = torch.from_numpy((synth.uniform(13, B) * 5.0).astype(np.float32)).cuda()
    loss = torch.zeros(1, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            flush.fill_(1)
            net.perch_cnn_train_step(crops, onehot, target, 1e-4, loss)
    torch.cuda.synchronize()
    ms = []
    with ClockSampler(0) as clocks, torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            net.perch_cnn_train_step(crops, onehot, target, 1e-4, loss)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    step_ms = statistics.mean(ms)
    F = 2048
    big, oh = crops.repeat(F // B, 1, 1, 1).contiguous(), onehot.repeat(F // B).contiguous()
    pred = torch.empty(F, device="cuda")
    torch.cuda.synchronize()
    def time_forward():
        fwd = []
        with torch.cuda.stream(stream):
            for k in range(3 + args.steps):
                flush.fill_(k)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                net.lib.perch_cnn_forward(net.h, big.data_ptr(), oh.data_ptr(), F, pred.data_ptr())
                e1.record(stream)
                e1.synchronize()
                if k >= 3:
                    fwd.append(e0.elapsed_time(e1))
        return statistics.mean(fwd)

    fwd_ms = time_forward()
    ref_pred = pred.clone()
    net.perch_cnn_set_tensor_path(1)  # convolutions 2-4 on tcgen05
    tc_ms = time_forward()
    tc_status = net.perch_cnn_tensor_status()
    tc_dev = float((pred - ref_pred).abs().max())
    net.perch_cnn_set_tensor_path(0)
    peaks = _measured_peaks()
    peak = peaks.get("bf16_tflops") or 1900.0
    achieved = B * CNN_TRAIN_FLOP_PER_CROP / step_ms / 1e9
    line = {"metric": "heuristic network training crops/sec (BF16, 1 GB300)", "value": B / step_ms * 1e3,
            "unit": "crops/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "heuristic network, batch of 256 seeded synthetic 2x64x64 crops + one-hot of "
                                   "8 meshes x 16 yaws; one step = forward, backward, Adam",
                       "l2": "flushed (256 MiB write) before every timed step"},
            "roofline": {"bound": "tensor", "kernel": "training step (k_gemm and its helpers)",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": measured_traffic("perch_cnn.cu", "cnn_train_step_launches.md"),
                         "flop_per_crop": CNN_TRAIN_FLOP_PER_CROP,
                         "peak_from": "bf16_tflops (burst cuBLAS) of MEASURED_PEAKS.json"},
            "forward": {"batch": F, "ms": fwd_ms, "crops_per_s": F / fwd_ms * 1e3,
                        "tflops": F * CNN_FWD_FLOP_PER_CROP / fwd_ms / 1e9},
            "forward_tcgen05": {"batch": F, "ms": tc_ms, "crops_per_s": F / tc_ms * 1e3,
                                "tflops": F * CNN_FWD_FLOP_PER_CROP / tc_ms / 1e9,
                                "max_abs_diff_vs_mma_sync": tc_dev, "waits_gave_up": tc_status[1],
                                "meaning": "forward with convolutions 2-4 on tcgen05 (tensor-memory accumulator)"},
            "gpu_launches": None, "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_c4(args):
    """Learned heuristic: train the network on the GPU (its own kernels) on
    exact edge costs of seeded 2-5-object training scenes, then search
    held-out seeded 5-object scenes with plain uniform-cost search (w = 1),
    Focal-MHA* (h_depth, h_overlap) and Focal-MHA* with the learned queue.
    Every arm searches all scenes at once (perch_search_multi). Objects sit
    off the pose grid by up to half a step (--off-grid)."""
    import torch
    from paper_1510_05613_gb300 import accuracy
    from paper_1510_05613_gb300 import heuristic as H
    from paper_1510_05613_gb300 import perch

    torch.cuda.set_device(0)
    grid = synth.pose_grid(-0.49, 0.02, 50, 16) if args.c4_grid == 50 else synth.pose_grid(-0.48, 0.04, 25, 8)
    t0 = time.perf_counter()
    train_sc = H.training_scenes(args.train_scenes, grid=grid, off_grid=args.off_grid)
    test_sc = H.test_scenes(args.scenes, grid=grid, off_grid=args.off_grid)
    gen_s = time.perf_counter() - t0
    p = perch.Perch(0)
    tr = H.setup_scenes(p, train_sc)
    te = H.setup_scenes(p, test_sc, first_id=len(train_sc))
    p.perch_autotune(args.tune_sample)
    if args.symmetric:
        p.perch_set_symmetry(train_sc[0].meshes)
    if args.render_cache:
        p.perch_set_render_cache(True)
    stream = torch.cuda.Stream()
    n_onehot = len(train_sc[0].meshes) * grid.n_yaw
    data, dstats = H.make_dataset(p, train_sc, tr, per_parent=args.per_parent, seed=1)
    val, _ = H.make_dataset(p, test_sc[:min(32, len(test_sc))], te[:min(32, len(te))], per_parent=256, seed=2)
    net = H.new_network(n_onehot, 1024, seed=3, stream=stream)  # trains on 256, forwards the search's crops 1024 at a time
    with ClockSampler(0) as train_clocks:
        losses, train_s = H.train(net, data, epochs=args.epochs, batch=256, lr=1e-3, stream=stream)
    steps = len(losses)
    quality = H.evaluate(net, val)
    # forward throughput at the search's batch shape, CUDA events on the network's stream
    fwd_n = 2048
    crops, onehot = data[0][:fwd_n].contiguous(), data[1][:fwd_n].contiguous()
    pred = torch.empty(fwd_n, device="cuda")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(13):
        if k == 3:
            e0.record(stream)
        net.lib.perch_cnn_forward(net.h, crops.data_ptr(), onehot.data_ptr(), fwd_n, pred.data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / 10
    # the same network before training (same seeded initial weights): the
    # "_untrained" arms measure what training adds to the queue itself
    untrained = H.new_network(n_onehot, 1024, seed=3, stream=stream)
    peaks = _measured_peaks()
    # (name, w, heuristic bits): bit 0 h_depth, bit 1 h_overlap, bit 2 the
    # learned queue ordered by g + h_cnn across depths, bit 3 the learned
    # depth-first queue
    arms = [("plain", 1.0, 0), ("mha_depth", args.w, 1), ("mha_learned", args.w, 4),
            ("mha_learned_untrained", args.w, 4), ("mha_learned_dive", args.w, 8),
            ("mha_learned_dive_untrained", args.w, 8), ("mha", args.w, 3), ("mha_depth+learned", args.w, 5),
            ("mha_depth+learned_untrained", args.w, 5), ("mha+learned", args.w, 7)]
    if args.arms:
        arms = [a for a in arms if a[0] in args.arms.split(",")]
    out, learned_cost = {}, {}
    with ClockSampler(0) as clocks, MemoryGuard() as mem:
        for name, w, hb in arms:
            p.perch_set_heuristic_net(untrained if name.endswith("_untrained") else net, args.candidates)
            t1 = time.perf_counter()
            r = p.perch_search_multi(te, [wl.mesh_multiset for wl in test_sc], batch_states=args.batch_states,
                                     max_hyps_per_launch=args.launch_hyps, time_limit_s=args.search_limit, w=w,
                                     heuristics=hb)
            out[name] = (r, time.perf_counter() - t1)
            learned_cost[name] = p.perch_search_stats() + p.perch_search_times()
    plain = out["plain"][0] if "plain" in out else None

    def summary(name):
        r, wall = out[name]
        fin = [x for x in r if x["cost"] >= 0 and x["seconds"] > 0 and (x["proven_optimal"] or name != "plain")]
        both = [(a, b) for a, b in zip(r, plain) if a["cost"] >= 0 and b["proven_optimal"]] if plain else []
        return {"w": dict((n, w) for n, w, _ in arms)[name], "heuristics": dict((n, h) for n, _, h in arms)[name],
                "wall_s": wall, "finished": len(fin),
                "time_to_scene_p50_s": float(np.percentile([x["seconds"] for x in fin], 50)) if fin else None,
                "time_to_scene_mean_s": float(np.mean([x["seconds"] for x in fin])) if fin else None,
                "expansions_mean": float(np.mean([x["expansions"] for x in r])),
                "found_p50_s": float(np.percentile([x["found_seconds"] for x in r if x["cost"] >= 0], 50))
                if any(x["cost"] >= 0 for x in r) else None,
                "found_expansions_mean": float(np.mean([x["found_expansions"] for x in r])),
                "successors_mean": float(np.mean([x["successors"] for x in r])),
                "same_scene_as_plain": sum(a["key"] == b["key"] for a, b in both),
                "compared_with_plain": len(both),
                "cost_gap_mean": float(np.mean([a["cost"] - b["cost"] for a, b in both])) if both else None,
                "cost_gap_rel_max": float(max((a["cost"] - b["cost"]) / max(b["cost"], 1) for a, b in both))
                if both else None,
                "learned_queue_seconds": learned_cost[name][0], "learned_states_scored": learned_cost[name][1],
                "learned_crops": learned_cost[name][2],
                "search_eval_s": learned_cost[name][3], "search_absorb_s": learned_cost[name][4],
                "search_select_s": learned_cost[name][5],
                "pose_accuracy": accuracy.report(r, test_sc, test_sc[0].meshes),
                "per_scene": [{"cost": x["cost"], "expansions": x["expansions"], "seconds": round(x["seconds"], 3),
                               "found_expansions": x["found_expansions"], "found_s": round(x["found_seconds"], 3),
                               "proven": x["proven_optimal"]} for x in r]}

    head = next((n for n in ("mha_depth+learned", "mha_learned", "mha+learned", "mha_depth", "plain") if n in out),
                arms[0][0])
    learned = summary(head)
    train_tflops = steps * 256 * CNN_TRAIN_FLOP_PER_CROP / train_s / 1e12
    peak = peaks.get("bf16_tflops_sustained") or 1700.0
    line = {"metric": METRIC, "value": learned["time_to_scene_p50_s"], "unit": f"s (time to scene, p50, arm {head})",
            "n_gpus": 1, "steps": steps, "warmup": 0, "ms_per_step": 1e3 * train_s / steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"learned heuristic: {len(test_sc)} held-out 640x480 5-object scenes of the 8 "
                                   f"uneven meshes, {grid.nx}x{grid.ny}x{grid.n_yaw} poses, objects off the grid by up "
                                   f"to {args.off_grid / 2:g} step, sigma 3 mm, 5% dropout, delta 1 cm; network trained "
                                   f"on {dstats['pairs']} exact (crop, edge cost) pairs of {len(train_sc)} seeded "
                                   "2-5-object scenes",
                       "train_scenes": len(train_sc), "pairs": dstats["pairs"], "epochs": args.epochs, "batch": 256,
                       "symmetric": bool(args.symmetric), "render_cache": bool(args.render_cache),
                       "candidates": args.candidates, "time_limit_s": args.search_limit, "generation_s": gen_s,
                       "dataset_s": dstats["seconds"]},
            "training": {"seconds": train_s, "steps": steps, "crops_per_s": steps * 256 / train_s,
                         "loss_first": float(np.mean(losses[:50])), "loss_last": float(np.mean(losses[-50:])),
                         "heldout": quality},
            "inference": {"batch": fwd_n, "ms": fwd_ms, "crops_per_s": fwd_n / fwd_ms * 1e3,
                          "tflops": fwd_n * CNN_FWD_FLOP_PER_CROP / fwd_ms / 1e9},
            "roofline": {"bound": "tensor", "achieved": train_tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": train_tflops / peak, "traffic": None,
                         "note": "whole training step (algorithmic FLOPs / step time) against the sustained "
                                 "cuBLAS bf16 peak of MEASURED_PEAKS.json"},
            "arms": {n: summary(n) for n, _, _ in arms},
            "host_peak_rss_gib": mem.peak / 2**30, "clocks": clocks.summary(), "train_clocks": train_clocks.summary()}
    print(json.dumps(line), flush=True)
    p.close()
    return 0


ICP_RADIUS_M = 0.02  # Sec. V-B: correspondences within 2 cm
ICP_MAX_FITS = 20
ICP_OPS_PER_POINT_MATCH = 30  # back-projection (2), frame change (9), motion (6), cells (9), pair terms (4)


def run_icp(args):
    """ICP refinement of successors (Sec. IV-E-1) alone: every successor of
    the root expansion of the off-grid 640x480 scene (120k hypotheses) in
    one call, W warm-up and K timed steps with CUDA events on the library's
    stream and L2 flushed before each; then the same batch with no fit (the
    render and model set alone), the host API with host buffers (e2e), the
    oracle on a bounded sample, and the pose accuracy of refining the true
    scenes' objects (Sec. V-D criterion) against their grid poses."""
    import torch
    from paper_1510_05613_gb300 import accuracy, perch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    wl = synth.workload_c2_off_grid(0)
    p = perch.Perch(0, stream=stream.cuda_stream)
    p.setup(wl)
    hyps = synth.all_hypotheses(wl.grid, list(range(len(wl.meshes))))
    if args.max_hyps and args.max_hyps < len(hyps):  # reduced batch (profiling case)
        hyps = hyps[np.linspace(0, len(hyps) - 1, args.max_hyps).astype(np.int64)]
    n = len(hyps)
    hp = np.zeros(n, np.int32)
    P, plen, stride = perch.Perch.pack_parents([wl.gt[:0]])
    tP = torch.from_numpy(P.view(np.int16).reshape(-1).copy()).to(dev)
    tplen = torch.from_numpy(plen).to(dev)
    thp = torch.from_numpy(hp).to(dev)
    th = torch.from_numpy(np.ascontiguousarray(hyps).view(np.int16).reshape(-1).copy()).to(dev)
    tout = torch.zeros(n * perch.ICP.itemsize, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def timed(max_iter, steps, clocks=None):
        for _ in range(max(args.warmup, 3)):
            flush.fill_(1)
            p.perch_icp_refine_dev(tP, stride, tplen, thp, th, ICP_RADIUS_M, max_iter, tout)
        torch.cuda.synchronize()
        ms = []
        for k in range(steps):
            flush.fill_(k)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p.perch_icp_refine_dev(tP, stride, tplen, thp, th, ICP_RADIUS_M, max_iter, tout)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.mean(ms)

    with ClockSampler(0) as clocks:
        step_ms = timed(ICP_MAX_FITS, args.steps)
    rec = tout.cpu().numpy().view(perch.ICP).copy()
    render_ms = timed(0, max(3, args.steps // 2))
    # matchings per record: one per fit, plus the one that stopped the
    # iteration early (too few pairs, repeated sums, no turn)
    matchings = rec["iters"].astype(np.int64) + (rec["status"] != perch.PERCH_ICP_CAP)
    point_matches = float((rec["n_model"].astype(np.int64) * matchings).sum())
    poses = distinct_poses(hyps)
    render_ops, _ = algorithmic_ops(wl, poses, rec["n_model"], rec["n_model"])
    match_ops = ICP_OPS_PER_POINT_MATCH * point_matches
    peaks = _measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz") or 2070.0)
    peak = SM_COUNT_NOMINAL * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    achieved = (render_ops + match_ops) / (step_ms * 1e-3) / 1e12
    # end to end through the host API (host buffers, batch upload and record download)
    e2e_t = []
    for k in range(0 if args.no_e2e else 2 + max(2, args.steps // 2)):
        t0 = time.perf_counter()
        out = p.perch_icp_refine([wl.gt[:0]], hp, hyps, ICP_RADIUS_M, ICP_MAX_FITS)
        t1 = time.perf_counter()
        if k >= 2:
            e2e_t.append(t1 - t0)
    if not e2e_t:
        out, e2e_t = rec, [float("nan")]
    consistent = bool(np.array_equal(out.view(np.uint8), rec.view(np.uint8)))
    e2e = {"value": n / statistics.mean(e2e_t), "unit": "successors/s",
           "h2d_bytes_per_step": int(hyps.nbytes + hp.nbytes + P.nbytes + plen.nbytes),
           "d2h_bytes_per_step": int(out.nbytes),
           "includes": "perch_icp_refine (batch upload, parent render, ICP, record download)"}
    # pose accuracy (Sec. V-D): 8 off-grid scenes searched exactly on the
    # grid (uniform-cost search over the symmetric yaw classes, render cache,
    # incumbent), then the returned scene's objects refined against each
    # other; and the true objects' grid poses refined the same way
    syms = [int(getattr(m, "sym", 1)) for m in wl.meshes]
    p.perch_set_symmetry(wl.meshes)
    p.perch_set_render_cache(True)
    def acc(errs):
        c = accuracy.correct_counts(errs, dts=(0.002, 0.005, 0.01), dthetas=(2.0, 5.0, 180.0))
        return {"objects": len(errs), "correct": {f"{dt * 1000:g}mm/{d:g}deg": v for (dt, d), v in c.items()},
                "mean_position_error_mm": 1000 * float(np.mean([e for _, e, _ in errs])),
                "median_position_error_mm": 1000 * float(np.median([e for _, e, _ in errs])),
                "mean_yaw_error_deg_box": float(np.mean([a for m, _, a in errs if m == 0] or [float("nan")]))}

    accuracy_by_grid = {}
    # the headline's 2 cm grid, and the paper's own 4 cm x 22.5 degree grid
    # with pairs within 2 cm, half its step (Sec. V-B)
    for name, grid in (("2cm", synth.pose_grid(-0.49, 0.02, 50, 16)), ("4cm", synth.pose_grid(-0.48, 0.04, 25, 16))):
        p.perch_set_pose_grid(grid)
        found, found_icp, true_grid, true_icp, search_s = [], [], [], [], []
        for s in range(8):
            ws_ = synth.workload_c2_off_grid(s, grid=grid)
            p.perch_set_observation(ws_.depth, ws_.cam.fxfycxcy, ws_.cam.T_wc, ws_.delta)
            truth = accuracy.true_poses(ws_)
            # the paper's setting (Sec. V-B): Focal-MHA* with w = 3 and its two
            # heuristics, here with the greedy incumbent first; 10 s per scene
            r = p.perch_search(ws_.mesh_multiset, 3.0, 16, 10.0, 0, 1 | 2 | 16)
            search_s.append(r["seconds"])
            found += accuracy.pose_errors(r["objs"], truth, ws_.grid, syms)
            _, refined = p.perch_refine_scene(r["objs"], ICP_RADIUS_M, ICP_MAX_FITS)
            found_icp += accuracy.pose_errors_of(refined, truth, syms)
            true_grid += accuracy.pose_errors(ws_.gt, truth, ws_.grid, syms)
            _, refined = p.perch_refine_scene(ws_.gt, ICP_RADIUS_M, ICP_MAX_FITS)
            true_icp += accuracy.pose_errors_of(refined, truth, syms)
        accuracy_by_grid[name] = {"searched": acc(found), "searched_then_icp": acc(found_icp),
                                  "true_grid_pose": acc(true_grid), "true_grid_pose_then_icp": acc(true_icp),
                                  "search_seconds_p50": statistics.median(search_s)}

    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        w = oracle.World.of(wl)
        threads = oracle.max_threads()
        # evenly spaced samples, doubled until the oracle has run about
        # --cpu-seconds (the whole batch at most)
        m, dt = 256, 0.0
        while True:
            idx = np.linspace(0, n - 1, min(m, n)).astype(np.int64)
            t0 = time.perf_counter()
            ref = oracle.icp_refine(w, wl.depth, [wl.gt[:0]], hp[idx], hyps[idx], ICP_RADIUS_M, ICP_MAX_FITS,
                                    threads)
            dt = time.perf_counter() - t0
            if dt >= 0.4 * args.cpu_seconds or len(idx) >= n:
                break
            m = int(min(n, max(2 * m, m * 0.5 * args.cpu_seconds / max(dt, 1e-3))))
        same = all(np.array_equal(ref[f], rec[f][idx]) for f in ref.dtype.names)
        cpu = {"value": len(idx) / dt, "unit": "successors/s", "cores": threads, "kind": "oracle",
               "sample": f"{len(idx)} evenly spaced of the {n} successors, {dt:.1f} s on {threads} OpenMP threads",
               "records_identical_to_gpu": bool(same)}
    line = {"metric": "ICP-refined successors/sec at 640x480 (Sec. IV-E-1; 1 GB300)", "value": n / step_ms * 1e3,
            "unit": "successors/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS["icp"], "radius_m": ICP_RADIUS_M, "max_fits": ICP_MAX_FITS,
                       "l2": "flushed (256 MiB write) before every timed step"},
            "roofline": {"bound": "alu", "kernel": "k_icp (render, model set, matching, fits)",
                         "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                         "traffic": None, "algorithmic_ops_per_step": render_ops + match_ops,
                         "render_ops": render_ops, "match_ops": match_ops, "point_matchings": point_matches,
                         "peak_from": "152 SMs x 128 FP32 lanes x max SM clock of MEASURED_PEAKS.json"},
            "phases_ms": {"render_and_model_set": render_ms, "matching_and_fits": step_ms - render_ms},
            "records": {"refined (>= 3 pairs)": int((rec["n_corr"] >= 3).sum()),
                        "fits": int(rec["iters"].sum()),
                        "status_counts": {str(k): int(v) for k, v in zip(*np.unique(rec["status"], return_counts=True))}},
            "accuracy": {**accuracy_by_grid,
                         "criterion": "Sec. V-D: position error < dt and yaw difference (modulo symmetry) < dtheta; "
                                      "8 off-grid scenes per grid (2 cm and 4 cm steps, 16 yaws); searched = "
                                      "Focal-MHA* on the grid (w = 3, h_depth and h_overlap, symmetric yaw classes, "
                                      "render cache, incumbent, 10 s limit); ICP = each object of "
                                      "the scene refined against the others"},
            "e2e": e2e, "e2e_records_identical": consistent, "cpu_baseline": cpu,
            "gpu_launches": 3 * args.steps,  # per step: k_fill_u32, k_render_parents, k_icp
            "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch-states", type=int, default=16)
    ap.add_argument("--search-limit", type=float, default=60.0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-search", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--threads", type=int, default=0, help="fix the CTA width (128/256/512) instead of autotuning")
    ap.add_argument("--tune-sample", type=int, default=8192, help="hypotheses per mesh the autotuner times")
    ap.add_argument("--max-hyps", type=int, default=0, help="evenly subsample the batch (profiling case)")
    ap.add_argument("--ref-sample", type=int, default=0,
                    help="--impl reference: hypotheses per step (default 128 per host thread)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the evaluation directly instead of replaying its CUDA graph (same kernels)")
    ap.add_argument("--scenes", type=int, default=64, help="c5: number of scenes")
    ap.add_argument("--w", type=float, default=3.0, help="c5: suboptimality bound of Focal-MHA*")
    ap.add_argument("--heuristics", type=int, default=3,
                    help="c5: bit 0 h_depth, bit 1 h_overlap, bit 4 a greedy incumbent first")
    ap.add_argument("--launch-hyps", type=int, default=1 << 22, help="c5: hypotheses per shared launch")
    ap.add_argument("--train-scenes", type=int, default=256, help="c4: training scenes")
    ap.add_argument("--per-parent", type=int, default=1536, help="c4: labelled hypotheses per training parent")
    ap.add_argument("--epochs", type=int, default=2, help="c4: training epochs")
    ap.add_argument("--candidates", type=int, default=8, help="c4: placements per type the learned queue scores")
    ap.add_argument("--c4-grid", type=int, default=50, choices=[25, 50], help="c4: 50 = 2 cm x 16 yaws, 25 = 4 cm x 8")
    ap.add_argument("--off-grid", type=float, default=1.0, help="c4: off-grid offsets, in grid steps (0..1)")
    ap.add_argument("--arms", default="", help="c4: comma-separated subset of plain, mha_depth, mha_learned, "
                                               "mha_learned_untrained, mha_learned_dive, mha_learned_dive_untrained, "
                                               "mha, mha_depth+learned, mha_depth+learned_untrained, mha+learned "
                                               "(default: all)")
    ap.add_argument("--render-cache", action="store_true",
                    help="c4/c5: keep each pose's render across expansions (records unchanged)")
    ap.add_argument("--symmetric", action="store_true",
                    help="c4/c5: searches place each mesh only at yaws distinct modulo its rotational symmetry")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5", "cnn", "icp"],
                    help="c2: 640x480 three ~10k-triangle meshes (the headline); c3: heavy occlusion, 2k-50k "
                         "triangles; icp: ICP refinement of every root successor of an off-grid c2 scene")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c5":
        return run_c5(args)
    if args.workload == "c4":
        return run_c4(args)
    if args.workload == "cnn":
        return run_cnn(args)
    if args.workload == "icp":
        return run_icp(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
