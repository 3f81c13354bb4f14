"""Benchmark: ICP iterations per second on the ~226k-point depth scene.

One step = one ICP iteration of the dilation-based ICP hot path with the grid
rebuilt: voxel histogram, offset scan, CSR scatter, brick list, dilation,
localised NNS with the exact global fallback, the reduction of the
centroids and cross-covariance, and the rigid solve.  Steps cycle through the
scene's 30-iteration registration from the identity pose (the pose is reset
every 30 steps), so the average step is the average iteration of a
registration.  Inputs are resident in HBM before timing; L2 is flushed (a
256 MiB write) between timed steps, outside the timed events.  Exactly
`--steps` steps are timed; the same steps run untimed for half a second
before and after them, so that the nvidia-smi clock samples cover the timed
steps' conditions.

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank runs an
independent replica of the scene workload (no collective on the data path;
`value` = all ranks' iterations / the slowest rank's time), and the batched
workload's pairs are sharded across the ranks (each rank registers its share,
the poses are gathered once at the end).

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

The line also carries, besides the headline:
  * `precision`: the same step with the FP64 reduction and solve (the
    method's stated precision) beside the default double-float one, and each
    one's 30-iteration pose against the FP64 CPU oracle;
  * `workloads`: the 4k-point sphere+plane (30 iterations) and the 40k-point
    object (50 iterations): iterations/s, end to end, roofline, pose error
    against the oracle;
  * `batched`: 256 uneven pairs (4.6M points per side, 40 iterations) in
    pairs/s, end to end and device-timed, against the same pairs registered
    one at a time, in both precisions, with the pose error against the
    oracle on sampled pairs;
  * `differentiable`: forward + backward of the point-to-point loss over 64
    pairs of 20k points, and its values against the oracle's;
  * `sparse_grid`: the same step on the sparse (hashed) grid, and the peak
    device bytes of the dense, sparse and fixed-capacity layouts;
  * the fixed-capacity store and the histogram ablation;
  * `cpu_baseline`: the CPU oracle on all host cores (and on one).

`--impl reference` times the CPU oracle (the plain C restatement of the
paper) on this host's cores on the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ICP iters/s at 226k pts (grid rebuilt every iteration)"
UNIT = "iters/s"
L_LAYERS = 10
ITERS_PER_REGISTRATION = 30
FLUSH_BYTES = 256 << 20
CLOCK_WINDOW_S = 0.5
PRECISION_LABEL = {
    "double_float": "f32 coordinates, distances and dilation; centroid/cross-covariance sums and the rigid solve "
                    "in double-float (~48-bit) on the FP32 pipes; pose composition f64",
    "fp64": "f32 coordinates, distances and dilation; centroid/cross-covariance sums and the rigid solve in f64; "
            "pose composition f64",
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: str):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def _smi_id(dev) -> str:
    """nvidia-smi selector for a torch device (its UUID, robust to
    CUDA_VISIBLE_DEVICES renumbering)."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev.index or 0)


# ----------------------------------------------------------------------------
# distributed plumbing
# ----------------------------------------------------------------------------
def _dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch
    import torch.distributed as dist
    rank, local = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist.init_process_group("gloo")
    return rank, ws, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x: float, ws: int) -> float:
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# algorithmic bytes per launch
# ----------------------------------------------------------------------------
def algorithmic_bytes(kernel: str, w: dict) -> float:
    """Bytes a kernel must move at minimum for one launch, from the workload's
    sizes (V voxels, N target and M source points, occupied voxels, search
    counters)."""
    V, N, M, occ = w["V"], w["N"], w["M"], w["occupied"]
    if kernel == "histogram":      # points in, keys out, one count RMW per occupied voxel
        return 16 * N + 4 * N + 8 * occ
    if kernel == "scan":           # occupancy bits and occupied counts in; the offsets the searches read out
        return V / 8 + 4 * occ + 4 * (2 * occ + V / 32 + 1)
    if kernel == "scatter":        # keys, points, offsets in; ids, voxel- and brick-ordered points, brick boxes out; RMW
        return 4 * N + 16 * N + 4 * N + 4 * N + 16 * N + 16 * N + 8 * occ + 32 * w["nonempty_bricks"]
    if kernel == "brick_scan":     # brick counts in, brick offsets + list + ranges out
        return 4 * w["bricks"] + 4 * (w["bricks"] + 1) + 12 * w["nonempty_bricks"]
    if kernel == "dilate":         # occupancy bits in, root + ring out
        return V / 8 + 5 * V
    if kernel == "correspond":     # per query: point, root, offset pair, nn+d2; candidates 16 B each
        return 36 * w["queries"] + 16 * w["local_cand"] + 4 * w["fallbacks"]
    if kernel == "fallback":       # per fallback: point + list entry + result; candidates 16 B each
        return 28 * w["fallbacks"] + 16 * w["global_cand"]
    if kernel in ("reduce_solve", "reduce_solve_f64"):   # per point: source point, nn, gathered target point
        return 36 * M
    return 0.0


def _kernel_sha(kernel: str) -> str:
    src = {"histogram": ("vicp_grid.cu",), "scan": ("vicp_grid.cu",), "scatter": ("vicp_grid.cu",),
           "brick_scan": ("vicp_grid.cu",),
           "dilate": ("vicp_dilate.cu", "vicp_dilate.cuh"),
           "correspond": ("vicp_nns.cu", "vicp_search.cuh"), "fallback": ("vicp_nns.cu", "vicp_search.cuh"),
           "reduce_solve": ("vicp_solve.cu", "vicp_df.cuh"),
           "reduce_solve_f64": ("vicp_solve64.cu", "vicp_f64.cuh")}.get(kernel)
    if not src:
        return ""
    h = hashlib.sha256()
    for name in src + ("vicp_device.cuh",):
        with open(os.path.join(ROOT, "paper_2512_04996_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel: str, workload: str = "depth_scene_226k"):
    """DRAM bytes (read + write) per launch from the committed ncu capture of
    this kernel on this workload, if the kernel's source is unchanged since
    the capture."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        with open(path) as f:
            for ln in f:
                if ln.startswith("#") or not ln.strip():
                    continue
                parts = ln.split()
                name, rd, wr, _t, sha = parts[:5]
                wl = parts[5] if len(parts) > 5 else "depth_scene_226k"
                if name == kernel and wl == workload:
                    return float(rd) + float(wr) if sha == _kernel_sha(kernel) else None
    except Exception:
        return None
    return None


# ----------------------------------------------------------------------------
# shared measurement helpers
# ----------------------------------------------------------------------------
def _rot_err_rad(Ta, Tb) -> float:
    """Rotation angle between two poses from |Ra - Rb|_F = 2 sqrt(2) sin(a/2):
    full relative precision for small angles (the arccos of the trace
    resolves nothing below about 1e-8 rad)."""
    d = float(np.linalg.norm(np.asarray(Ta)[:3, :3] - np.asarray(Tb)[:3, :3]))
    return 2.0 * math.asin(min(1.0, d / (2.0 * math.sqrt(2.0))))


def _extent(pts) -> float:
    t = pts[:, :3]
    return float((t.max(0) - t.min(0)).max())


def _pose_err(T, R, extent) -> dict:
    """Pose difference: rotation angle (rad) and translation / extent."""
    return {"rot_rad": _rot_err_rad(T, R),
            "trans_rel_extent": float(np.linalg.norm(np.asarray(T)[:3, 3] - np.asarray(R)[:3, 3])) / extent}


def _oracle_threads() -> int:
    import oracle
    return oracle.use_threads(os.cpu_count() or 1)


def _oracle_register(pair, iters: int, eps: float = 0.0):
    """The FP64 CPU oracle's registration of a pair from the identity (all
    host cores; the threaded oracle gives bit-identical results)."""
    import oracle
    _oracle_threads()
    try:
        g = oracle.fit_grid(pair.target, pair.voxel_size, pair.grid_divisions)
        return oracle.register(g, L_LAYERS, pair.target, pair.source, np.eye(4), max_iters=iters, eps=eps)
    finally:
        oracle.use_threads(1)


def _timed_steps(one_step, n, flush, stream):
    """Device time (ms) of each of n steps, with L2 flushed before each one
    outside the timed events."""
    import torch
    ev = []
    for k in range(n):
        flush.fill_(k & 0xff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        one_step(k)
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def _kernel_table(ctx, one_step, steps, flush, w, peak):
    """Per-kernel event times over `steps` steps, with algorithmic bytes and
    GB/s; returns (table, name of the kernel with the largest total time)."""
    ctx.read_stats(reset=True)
    ctx.profile_enable(True)
    for k in range(steps):
        flush.fill_(k & 0xff)
        one_step(k)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    st = ctx.read_stats(reset=True)
    wl = dict(w)
    wl.update(queries=st["queries"] / steps, fallbacks=st["fallbacks"] / steps,
              local_cand=st["local_candidates"] / steps, global_cand=st["global_candidates"] / steps)
    table = {}
    for name, (n_l, ms) in prof.items():
        if n_l:
            avg_ms = ms / n_l
            b = algorithmic_bytes(name, wl)
            gbs = b / (avg_ms * 1e-3) / 1e9 if b else None
            table[name] = {"launches": n_l, "total_ms": round(ms, 4), "avg_us": round(1e3 * avg_ms, 3),
                           "alg_bytes": int(b), "gbs": round(gbs, 1) if gbs else None,
                           "frac_of_hbm": round(gbs / peak, 4) if gbs else None}
    dominant = max(table, key=lambda k: table[k]["total_ms"])
    return table, dominant, st


def _workload_sizes(ctx, view, N, M):
    mem = ctx.memory_report()
    nbt = int(math.ceil(view.dims[0] / 8) * math.ceil(view.dims[1] / 8) * math.ceil(view.dims[2] / 8))
    return dict(V=int(view.n_voxels), N=N, M=M, occupied=mem["occupied_voxels"], bricks=nbt,
                nonempty_bricks=mem["nonempty_bricks"]), mem


# ----------------------------------------------------------------------------
# single-pair workloads other than the headline: 4k sphere+plane, 40k object
# ----------------------------------------------------------------------------
def run_workload(dev, pair, flush, steps: int) -> dict:
    """ICP iterations/s of one pair with the grid rebuilt every iteration
    (device time, L2 flushed between steps), the dominant kernel's roofline,
    the full registration end to end from host buffers, and the registered
    pose against the oracle's."""
    import torch

    from paper_2512_04996_gb300 import vicp

    stream = torch.cuda.current_stream(dev)
    src = torch.from_numpy(pair.source).to(dev)
    tgt = torch.from_numpy(pair.target).to(dev)
    N, M, iters = tgt.shape[0], src.shape[0], pair.iters
    ctx = vicp.Context(voxel_size=pair.voxel_size, grid_divisions=pair.grid_divisions, dilation_layers=L_LAYERS,
                       max_iters=1, rmse_eps=0.0, flags=vicp.VICP_FLAG_KEEP_GRID)
    pose = torch.eye(4, dtype=torch.float64, device=dev).contiguous()
    eye = pose.clone()

    def one_step(k):
        if k % iters == 0:
            pose.copy_(eye)
        ctx.build_grid(tgt)
        ctx.dilate(L_LAYERS)
        ctx.step(src, pose)

    for k in range(5):
        one_step(k)
    if ctx.sync() != 0:
        raise RuntimeError("workload warm-up failed: " + ctx.last_error())
    view = ctx.grid_view()
    ms = _timed_steps(one_step, steps, flush, stream)
    value = steps / (sum(ms) / 1e3)
    w, mem = _workload_sizes(ctx, view, N, M)
    peak, peak_kind = _peaks()
    table, dom, _ = _kernel_table(ctx, one_step, min(steps, 200), flush, w, peak)
    # end to end: the full registration from pinned host buffers, pose read back
    # (the grid fitted at the first call is kept, so the calls replay their
    # captured CUDA graph from the second on)
    ctx_e = vicp.Context(voxel_size=pair.voxel_size, grid_divisions=pair.grid_divisions, dilation_layers=L_LAYERS,
                         max_iters=iters, rmse_eps=0.0, flags=vicp.VICP_FLAG_KEEP_GRID)
    src_h = torch.from_numpy(pair.source).pin_memory().numpy()
    tgt_h = torch.from_numpy(pair.target).pin_memory().numpy()
    for _ in range(3):
        ctx_e.register_host(src_h, tgt_h)
    reps = 20
    t0 = time.perf_counter()
    for _ in range(reps):
        st, T, it, rm = ctx_e.register_host(src_h, tgt_h)
    e2e_s = (time.perf_counter() - t0) / reps
    replayed = ctx_e.graph_replayed()
    # the pose against the oracle
    rst, R, rit, hist = _oracle_register(pair, iters)
    ext = _extent(pair.target)
    return {
        "workload": f"{pair.name}: {N} target / {M} source points, grid {list(view.dims[0:3])} "
                    f"({int(view.n_voxels)} voxels), L={L_LAYERS}, {iters}-iteration registrations from identity",
        "value": round(value, 1), "unit": UNIT, "ms_per_step": round(1e3 / value, 4),
        "what": "one ICP iteration with the grid rebuilt (device time, L2 flushed between steps)",
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": table[dom]["gbs"], "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": table[dom]["frac_of_hbm"],
                     "traffic": _ncu_traffic(dom, pair.name), "alg_bytes_per_launch": table[dom]["alg_bytes"]},
        "kernels": table,
        "e2e": {"value": round(iters / e2e_s, 1), "unit": UNIT, "registrations_per_s": round(1.0 / e2e_s, 1),
                "h2d_bytes_per_registration": int(16 * (N + M)), "d2h_bytes_per_registration": 16 * 8 + 24 + 4,
                "graph_replayed": replayed,
                "what": f"vicp_register_host, {iters} iterations per call: H2D of both clouds from pinned memory, "
                        "grid build, dilation, the iterations, pose read back (host wall clock; the grid of the "
                        "first call kept, each call replayed as one CUDA graph)"},
        "pose_err_vs_oracle": {**_pose_err(T, R, ext), "iters": it, "oracle_iters": rit,
                               "rmse_rel_diff": abs(rm - hist[-1]) / hist[-1]},
        "rot_err_vs_truth_deg": round(math.degrees(_rot_err_rad(T, pair.T_gt)), 5),
        "peak_device_bytes": mem["peak_bytes"],
    }


# ----------------------------------------------------------------------------
# batched registration (256 uneven pairs) against one pair at a time
# ----------------------------------------------------------------------------
BATCH_ITERS = 40


def run_batched(dev, flush, rank: int, ws: int, reps: int = 5, n_pairs: int = 256, oracle_sample: int = 8) -> dict:
    import torch

    from paper_2512_04996_gb300 import shard, synth, vicp

    ps_all = synth.batched_pairs(n_pairs=n_pairs)
    P_all = len(ps_all)
    work = [p.source.shape[0] + p.target.shape[0] for p in ps_all]
    mine = shard.partition_pairs(work, ws)[rank]
    ps = [ps_all[k] for k in mine]
    P = len(ps)
    stream = torch.cuda.current_stream(dev)
    tgt_np = np.ascontiguousarray(np.concatenate([p.target for p in ps]))
    src_np = np.ascontiguousarray(np.concatenate([p.source for p in ps]))
    n_tgt = np.array([p.target.shape[0] for p in ps], np.int32)
    n_src = np.array([p.source.shape[0] for p in ps], np.int32)
    vs = np.array([p.voxel_size for p in ps], np.float32)
    dv = np.array([p.grid_divisions for p in ps], np.int32)
    tgt = torch.from_numpy(tgt_np).to(dev)
    src = torch.from_numpy(src_np).to(dev)
    src_pin = torch.from_numpy(src_np).pin_memory().numpy()
    tgt_pin = torch.from_numpy(tgt_np).pin_memory().numpy()
    M, N = int(n_src.sum()), int(n_tgt.sum())

    def measure(flags):
        b = vicp.Batch(dilation_layers=L_LAYERS, max_iters=BATCH_ITERS, rmse_eps=0.0, flags=flags)
        b.build(tgt, n_tgt, vs, dv)
        shape, tune_ms = b.tune(src, n_src, iters=4, trials=2)
        for _ in range(2):   # warm-up: captures the iteration graph
            st, T, it, rm, pst = b.register(src, n_src)
            if st != 0:
                raise RuntimeError("batched warm-up failed: " + b._lib.vicp_batch_last_error(b.handle).decode())
        b.report(reset=True)
        reg_ms, launches0 = [], b.launch_count()
        _barrier(ws)
        for k in range(reps):
            flush.fill_(k & 0xff)
            e0, e1, r1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            b.build(tgt, n_tgt, vs, dv)
            e1.record(stream)
            st, T, it, rm, pst = b.register(src, n_src)
            r1.record(stream)
            torch.cuda.synchronize()
            if st != 0:
                raise RuntimeError("batched run failed")
            reg_ms.append((e0.elapsed_time(e1), e1.elapsed_time(r1)))
        graph = b.graph_replayed()
        launches = (b.launch_count() - launches0) // reps
        stats = b.report(reset=True)
        build_ms = statistics.median(x[0] for x in reg_ms)
        iter_ms = statistics.median(x[1] for x in reg_ms)
        total_s = _max_over_ranks((build_ms + iter_ms) / 1e3, ws)
        # end to end: host clouds in, poses out, through vicp_batch_register_host
        bh = vicp.Batch(dilation_layers=L_LAYERS, max_iters=BATCH_ITERS, rmse_eps=0.0, shape=shape, flags=flags)
        bh.register_host(src_pin, n_src, tgt_pin, n_tgt, vs, dv)
        torch.cuda.synchronize()
        _barrier(ws)
        t0 = time.perf_counter()
        for _ in range(reps):
            bh.register_host(src_pin, n_src, tgt_pin, n_tgt, vs, dv)
        e2e_s = _max_over_ranks((time.perf_counter() - t0) / reps, ws)
        rep = b.report()
        out = {"pairs_per_s": round(P_all / total_s, 1), "e2e_pairs_per_s": round(P_all / e2e_s, 1),
               "build_ms": round(build_ms, 3), "iterations_ms": round(iter_ms, 3),
               "graph_replayed": bool(graph == 1), "gpu_launches_per_batch": int(launches),
               "shape": {"index": shape, "tune_ms": [round(float(x), 3) for x in tune_ms]},
               "fallbacks_per_batch": stats["fallbacks"] // reps, "queries_per_batch": stats["queries"] // reps,
               "peak_device_bytes": rep["peak_bytes"]}
        return out, T, it

    res_df, T_df, it_df = measure(0)
    res_64, T_64, it_64 = measure(vicp.VICP_BATCH_FLAG_FP64)
    T_df_all, it_df_all = shard.gather_results(mine, T_df, it_df, P_all, ws)
    T_64_all, _ = shard.gather_results(mine, T_64, it_64, P_all, ws)
    out = {
        "metric": "batched pairs/s (256 pairs, 40 iterations each, grids built per batch)",
        "scaling": "strong" if ws > 1 else None, "ranks": ws, "pairs_on_rank0": len(mine),
        "workload": f"{P_all} pairs (even: sphere+plane, odd: bumpy object), sizes log-uniform in 2k..64k, "
                    f"{sum(p.source.shape[0] for p in ps_all)} source / {sum(p.target.shape[0] for p in ps_all)} "
                    f"target points, L={L_LAYERS}, {BATCH_ITERS} iterations from identity",
        "double_float": res_df, "fp64": res_64,
    }
    if rank == 0:
        # one pair at a time through the single-pair path (vicp_register), host wall clock
        src_t = [torch.from_numpy(p.source).to(dev) for p in ps_all]
        tgt_t = [torch.from_numpy(p.target).to(dev) for p in ps_all]
        dva = np.array([p.grid_divisions for p in ps_all], np.int32)
        nta = np.array([p.target.shape[0] for p in ps_all], np.int32)
        ctxs = {d: vicp.Context(dilation_layers=L_LAYERS, max_iters=BATCH_ITERS, rmse_eps=0.0, grid_divisions=int(d))
                for d in sorted(set(int(x) for x in dva))}
        for d, c in ctxs.items():   # size every context's buffers once
            k = int(np.flatnonzero(dva == d)[np.argmax(nta[dva == d])])
            c.register(src_t[k], tgt_t[k])
        torch.cuda.synchronize()
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plain = []
        for k, p in enumerate(ps_all):
            st, S, it1, rm1 = ctxs[int(dva[k])].register(src_t[k], tgt_t[k])
            plain.append(S)
        plain_pps = P_all / (time.perf_counter() - t0)
        ext = [_extent(p.target) for p in ps_all]
        # the oracle on pairs spread over the size range
        sizes = np.array([p.source.shape[0] for p in ps_all])
        order = np.argsort(sizes)
        sample = sorted(set(int(order[int(round(i))]) for i in np.linspace(0, P_all - 1, oracle_sample)))
        t_or = time.perf_counter()
        err_df, err_64 = [], []
        for k in sample:
            _, R, _, _ = _oracle_register(ps_all[k], BATCH_ITERS)
            err_df.append(_pose_err(T_df_all[k], R, ext[k]))
            err_64.append(_pose_err(T_64_all[k], R, ext[k]))
        t_or = time.perf_counter() - t_or

        def worst(errs):
            return {"rot_rad": max(e["rot_rad"] for e in errs),
                    "trans_rel_extent": max(e["trans_rel_extent"] for e in errs)}

        out.update({
            "value": res_df["e2e_pairs_per_s"], "unit": "pairs/s",
            "what": "end to end: vicp_batch_register_host (H2D of all pooled clouds from pinned memory, build, "
                    "40 iterations, poses read back), host wall clock -- against plain_one_at_a_time, also host "
                    "wall clock",
            "plain_one_at_a_time": {"value": round(plain_pps, 1), "unit": "pairs/s",
                                    "what": "the same 256 pairs through vicp_register one after another "
                                            "(device-resident clouds, each call synchronises; host wall clock)"},
            "speedup_e2e_vs_plain": round(res_df["e2e_pairs_per_s"] / plain_pps, 2),
            "speedup_device_vs_plain": round(res_df["pairs_per_s"] / plain_pps, 2),
            "accuracy": {
                "max_rot_diff_vs_plain_rad": max(_rot_err_rad(T_df_all[k], plain[k]) for k in range(P_all)),
                "max_trans_diff_vs_plain_rel_extent": max(
                    float(np.linalg.norm(T_df_all[k][:3, 3] - plain[k][:3, 3])) / ext[k] for k in range(P_all)),
                "max_rot_diff_fp64_vs_double_float_rad": max(_rot_err_rad(T_df_all[k], T_64_all[k])
                                                             for k in range(P_all)),
                "pose_err_vs_oracle_double_float": worst(err_df),
                "pose_err_vs_oracle_fp64": worst(err_64),
                "oracle_pairs": sample, "oracle_s": round(t_or, 1),
                "median_rot_err_vs_truth_deg": round(statistics.median(
                    math.degrees(_rot_err_rad(T_df_all[k], p.T_gt)) for k, p in enumerate(ps_all)), 6)},
        })
    return out


# ----------------------------------------------------------------------------
# the sparse (hashed) grid against the dense grid on the scene
# ----------------------------------------------------------------------------
def run_sparse(dev, pair, flush, steps: int, dense_pose, dense_mem) -> dict:
    import torch

    from paper_2512_04996_gb300 import vicp

    stream = torch.cuda.current_stream(dev)
    src = torch.from_numpy(pair.source).to(dev)
    tgt = torch.from_numpy(pair.target).to(dev)
    flags = vicp.VICP_FLAG_KEEP_GRID | vicp.VICP_FLAG_SPARSE_GRID
    ctx = vicp.Context(voxel_size=pair.voxel_size, dilation_layers=L_LAYERS, max_iters=1, rmse_eps=0.0, flags=flags)
    pose = torch.eye(4, dtype=torch.float64, device=dev).contiguous()
    eye = pose.clone()

    def one_step(k):
        if k % ITERS_PER_REGISTRATION == 0:
            pose.copy_(eye)
        ctx.build_grid(tgt)
        ctx.dilate(L_LAYERS)
        ctx.step(src, pose)

    for k in range(5):
        one_step(k)
    ms = _timed_steps(one_step, steps, flush, stream)
    ctx.profile_enable(True)
    for k in range(min(steps, 200)):
        flush.fill_(k & 0xff)
        one_step(k)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    ctx.build_grid(tgt)
    ctx.dilate(L_LAYERS)

    def step_only(k):
        if k % ITERS_PER_REGISTRATION == 0:
            pose.copy_(eye)
        ctx.step(src, pose)
    amort = _timed_steps(step_only, steps, flush, stream)
    mem = ctx.memory_report()
    ctx_r = vicp.Context(voxel_size=pair.voxel_size, dilation_layers=L_LAYERS, max_iters=ITERS_PER_REGISTRATION,
                         rmse_eps=0.0, flags=flags | vicp.VICP_FLAG_REBUILD_EACH_ITER)
    st, T, it, rm = ctx_r.register(src, tgt)
    ext = _extent(pair.target)
    return {
        "what": "the headline step on the sparse (hashed) grid: occupied voxels and labelled row segments "
                "in hash tables instead of per-voxel counts, offsets, root and ring (one host synchronisation "
                "per dilation to size the labelled-segment table)",
        "iters_per_s": round(len(ms) / (sum(ms) / 1e3), 1),
        "amortised_grid_built_once_iters_per_s": round(len(amort) / (sum(amort) / 1e3), 1),
        "kernels_us": {k: round(1e3 * v[1] / v[0], 2) for k, v in prof.items() if v[0]},
        "registration_30_vs_dense": {**_pose_err(T, dense_pose, ext), "status": st, "iters": it},
        "memory": {"peak_device_bytes": {"dense_csr": dense_mem["peak_bytes"], "sparse": mem["peak_bytes"]},
                   "per_voxel_arrays_bytes": {"dense_csr": dense_mem["csr_store_bytes"] - 4 * pair.target.shape[0],
                                              "sparse_tables": mem["csr_store_bytes"] - 4 * pair.target.shape[0]},
                   "fixed_capacity_bytes": mem["fixed_capacity_bytes"],
                   "paper_64KB_per_voxel_bytes": mem["paper_static_layout_bytes"],
                   "labelled_voxels": mem["labelled_voxels"], "occupied_voxels": mem["occupied_voxels"]},
    }


# ----------------------------------------------------------------------------
# fixed-capacity store (direct addressing) against the CSR store
# ----------------------------------------------------------------------------
def run_fixed(dev, pair, flush, reps: int = 100) -> dict:
    import torch

    from paper_2512_04996_gb300 import vicp

    stream = torch.cuda.current_stream(dev)
    src = torch.from_numpy(pair.source).to(dev)
    tgt = torch.from_numpy(pair.target).to(dev)
    ctx = vicp.Context(voxel_size=pair.voxel_size, dilation_layers=L_LAYERS, max_iters=1, rmse_eps=0.0)
    ctx.build_grid(tgt)
    ctx.dilate(L_LAYERS)
    mem = ctx.memory_report()
    C = int(mem["max_voxel_count"])
    view = ctx.grid_view()
    V, N = int(view.n_voxels), tgt.shape[0]
    over, nbytes = ctx.fixed_build(tgt, C)

    def timed(fn):
        ms = []
        for k in range(reps + 3):
            flush.fill_(k & 0xff)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            if k >= 3:
                ms.append(e0.elapsed_time(e1))
        return 1e3 * statistics.median(ms)

    ctx.profile_enable(True)
    for k in range(reps):
        flush.fill_(k & 0xff)
        ctx.build_grid(tgt)
    prof = ctx.profile_read()
    csr_build_us = sum(1e3 * prof[k][1] / max(1, prof[k][0]) for k in ("histogram", "scan", "scatter"))
    ctx.profile_enable(False)
    ctx.dilate(L_LAYERS)
    ctx.profile_enable(True)
    for k in range(reps):
        flush.fill_(k & 0xff)
        ctx.fixed_build(tgt, C)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    fixed_scatter_us = 1e3 * prof["fixed_scatter"][1] / max(1, prof["fixed_scatter"][0])
    reset = torch.empty(V, dtype=torch.int32, device=dev)   # the fill counts' reset, timed as a plain memset
    fixed_reset_us = timed(lambda: reset.zero_())
    del reset
    pose = torch.from_numpy(np.ascontiguousarray(pair.T_gt)).to(dev)
    nn = torch.empty(src.shape[0], dtype=torch.int32, device=dev)
    d2 = torch.empty(src.shape[0], dtype=torch.float32, device=dev)
    ctx.profile_enable(True)
    for k in range(reps):
        flush.fill_(k & 0xff)
        ctx.correspond(src, pose, nn, d2)
        flush.fill_(k & 0xff)
        ctx.fixed_correspond(src, pose, nn, d2)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    us = {k: 1e3 * prof[k][1] / max(1, prof[k][0]) for k in ("correspond", "fixed_correspond")}
    ctx.close()
    return {
        "capacity": C, "dropped_points": over,
        "store_bytes": {"fixed": nbytes, "csr_offsets_ids_points": 4 * (V + 1) + 4 * N + 16 * N},
        "build_us": {"csr_histogram_scan_scatter": round(csr_build_us, 2),
                     "fixed_scatter": round(fixed_scatter_us, 2), "fixed_count_reset": round(fixed_reset_us, 2),
                     "fixed_total": round(fixed_scatter_us + fixed_reset_us, 2)},
        "localised_search_us": {"csr": round(us["correspond"], 2), "fixed": round(us["fixed_correspond"], 2)},
        "workload": f"226k scene, {V} voxels, capacity = the largest voxel count (nothing dropped), "
                    f"search at the true pose; L2 flushed between launches",
    }


# ----------------------------------------------------------------------------
# histogram ablation: warp-aggregated vs the paper's shared-memory hash
# ----------------------------------------------------------------------------
def run_hist_ablation(dev, tgt, view, occupied: int, flush, reps: int = 200) -> dict:
    import torch

    from paper_2512_04996_gb300 import vicp

    stream = torch.cuda.current_stream(dev)
    N = tgt.shape[0]
    dims = [int(view.dims[a]) for a in range(3)]
    origin = [float(view.origin[a]) for a in range(3)]
    V = int(view.n_voxels)
    keys = torch.empty(N, dtype=torch.int32, device=dev)
    counts = torch.zeros(V, dtype=torch.int32, device=dev)
    alg = 16 * N + 4 * N + 8 * occupied
    out = {}
    for method, name in ((vicp.VICP_HIST_WARP_AGGREGATED, "warp_aggregated"),
                         (vicp.VICP_HIST_SHARED_HASH, "shared_hash")):
        ms = []
        for k in range(reps + 3):
            counts.zero_()
            flush.fill_(k & 0xff)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            vicp.vicp_voxel_histogram(tgt, origin, float(view.voxel_size), dims, method, keys, counts)
            e1.record(stream)
            e1.synchronize()
            if k >= 3:
                ms.append(e0.elapsed_time(e1))
        med = statistics.median(ms)
        out[name] = {"us": round(1e3 * med, 3), "gbs": round(alg / (med * 1e-3) / 1e9, 1)}
    out["workload"] = f"keys + counts of the {N}-point scene target on its {V}-voxel grid (L2 flushed)"
    return out


# ----------------------------------------------------------------------------
# differentiable loss: 64 pairs x 20k points, forward + backward
# ----------------------------------------------------------------------------
def run_loss(dev, flush, steps: int = 50, n_pairs: int = 64, oracle_sample: int = 4) -> dict:
    import torch

    from oracle import diff
    from paper_2512_04996_gb300 import synth, vicp

    ps = synth.loss_pairs(n_pairs=n_pairs, workers=max(1, min(16, os.cpu_count() or 1)))
    P = len(ps)
    stream = torch.cuda.current_stream(dev)
    tgt = torch.from_numpy(np.ascontiguousarray(np.concatenate([p.target for p in ps]))).to(dev)
    src = torch.from_numpy(np.ascontiguousarray(np.concatenate([p.source for p in ps]))).to(dev)
    n_tgt = np.array([p.target.shape[0] for p in ps], np.int32)
    n_src = np.array([p.source.shape[0] for p in ps], np.int32)
    b = vicp.Batch(dilation_layers=L_LAYERS)
    b.build(tgt, n_tgt, None, np.array([p.grid_divisions for p in ps], np.int32))
    T0 = torch.from_numpy(np.ascontiguousarray(np.stack([p.T_gt for p in ps]))).to(dev)
    src_g = src.clone().requires_grad_(True)

    def step(recompute=False):
        xi = torch.zeros((P, 6), dtype=torch.float32, device=dev, requires_grad=True)
        loss = vicp.point_to_point_loss(xi, src_g, b, n_src, T0, recompute)
        loss.sum().backward()
        return loss, xi

    out = {}
    for recompute in (False, True):
        for _ in range(3):
            step(recompute)
        torch.cuda.synchronize()
        l0 = b.launch_count()
        ms = []
        for k in range(steps):
            flush.fill_(k & 0xff)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            loss, xi = step(recompute)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            src_g.grad = None
        med = statistics.median(ms)
        out["recompute" if recompute else "stored"] = {
            "ms_per_forward_backward": round(med, 4), "pairs_per_s": round(P / (med / 1e3), 1),
            "points_per_s": round(int(n_src.sum()) / (med / 1e3), 1),
            # the batch context counts its own launches; Exp and the Jacobian transpose are two more
            "library_launches_per_step": int((b.launch_count() - l0) / steps) + 2}
    # the values at the evaluation poses against the FP64 oracle (sampled pairs)
    loss, xi = step(False)
    gx = xi.grad.detach().cpu().numpy().astype(np.float64)
    lv = loss.detach().cpu().numpy()
    nn, _ = b.correspond(src, n_src, T0)
    nn = np.split(nn.cpu().numpy(), np.cumsum(n_src)[:-1])
    T0n = T0.cpu().numpy()
    l_err, g_err = 0.0, 0.0
    for k in np.linspace(0, P - 1, oracle_sample).round().astype(int):
        p = ps[k]
        lr = diff.loss(p.target, p.source, T0n[k], nn[k])
        gr = diff.grad_left(p.target, p.source, T0n[k], nn[k])
        l_err = max(l_err, abs(lv[k] - lr) / lr)
        g_err = max(g_err, float(np.abs(gx[k] - gr).max() / np.abs(gr).max()))
    return {
        "workload": f"{P} pairs x {int(n_src[0])} points (bumpy-object generator, voxel = extent/128), "
                    "loss of Eq. 1 at the true poses, gradients in 6 float32 se(3) parameters per pair "
                    "and in every source point",
        "what": "one forward (Exp, batched NNS, loss) + backward (loss gradients, left-Jacobian transpose) "
                "through torch.autograd, CUDA events on the stream",
        **out,
        "vs_oracle": {"loss_rel_err": l_err, "grad_xi_rel_err": g_err,
                      "what": f"{oracle_sample} pairs: loss and pose gradient at the evaluation pose against the "
                              "FP64 oracle with the same correspondences (float32 se(3) parameters)"},
    }


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def run_ours(args, rank, ws, local):
    import torch

    from paper_2512_04996_gb300 import synth, vicp

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    pair = synth.depth_scene()
    src = torch.from_numpy(pair.source).to(dev)
    tgt = torch.from_numpy(pair.target).to(dev)
    N, M = tgt.shape[0], src.shape[0]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    peak, peak_kind = _peaks()

    def scene_stepper(prec_flags):
        ctx = vicp.Context(voxel_size=pair.voxel_size, dilation_layers=L_LAYERS, max_iters=1, rmse_eps=0.0,
                           flags=vicp.VICP_FLAG_KEEP_GRID | prec_flags)
        pose = torch.eye(4, dtype=torch.float64, device=dev).contiguous()
        eye = pose.clone()

        def one_step(k):
            if k % ITERS_PER_REGISTRATION == 0:
                pose.copy_(eye)
            ctx.build_grid(tgt)
            ctx.dilate(L_LAYERS)
            ctx.step(src, pose)
        return ctx, one_step

    ctx, one_step = scene_stepper(0)
    # warm-up (also fits the grid geometry once: KEEP_GRID)
    for k in range(args.warmup):
        one_step(k)
    if ctx.sync() != 0:
        raise RuntimeError("warm-up failed: " + ctx.last_error())
    view = ctx.grid_view()
    V = int(view.n_voxels)

    # ---- timed pass: exactly K steps, per-step CUDA events, L2 flushed -------
    # between steps; the same steps run untimed for CLOCK_WINDOW_S before and
    # after, so that the clock samples (every 100 ms) cover the timed steps
    ctx.read_stats(reset=True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(_smi_id(dev)) as clk:
        w0 = time.perf_counter()
        k = 0
        while time.perf_counter() - w0 < CLOCK_WINDOW_S:
            flush.fill_(k & 0xff)
            one_step(k)
            k += 1
            if k % 50 == 0:
                torch.cuda.synchronize()
        torch.cuda.synchronize()
        pre_roll = k
        ctx.read_stats(reset=True)
        launches0 = ctx.launch_count()
        _barrier(ws)
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(k & 0xff)
            starts[k].record(stream)
            one_step(k)
            ends[k].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        gpu_launches = ctx.launch_count() - launches0
        stats = ctx.read_stats(reset=True)
        w1 = time.perf_counter()
        k = 0
        while time.perf_counter() - w1 < CLOCK_WINDOW_S:
            flush.fill_(k & 0xff)
            one_step(k)
            k += 1
            if k % 50 == 0:
                torch.cuda.synchronize()
        torch.cuda.synchronize()
        post_roll = k
    _barrier(ws)
    if ctx.sync() != 0:
        raise RuntimeError("timed pass failed: " + ctx.last_error())
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s = _max_over_ranks(sum(step_ms) / 1e3, ws)
    value = ws * args.steps / total_s

    # ---- per-kernel times (the library's event timing) ------------------------
    w, mem = _workload_sizes(ctx, view, N, M)
    kernels, dominant, _ = _kernel_table(ctx, one_step, min(args.steps, 300), flush, w, peak)
    dk = kernels[dominant]
    achieved = dk["gbs"] if dk["gbs"] else 0.0

    # ---- grid built once (amortised over the registration) --------------------
    ctx.build_grid(tgt)
    ctx.dilate(L_LAYERS)
    pose_a = torch.eye(4, dtype=torch.float64, device=dev).contiguous()
    eye = pose_a.clone()

    def step_only(k):
        if k % ITERS_PER_REGISTRATION == 0:
            pose_a.copy_(eye)
        ctx.step(src, pose_a)
    amort_ms = _timed_steps(step_only, min(args.steps, 600), flush, stream)
    amortised = len(amort_ms) / (sum(amort_ms) / 1e3)

    # ---- end to end through the C ABI with host buffers -----------------------
    e2e_steps = min(args.steps, 200)
    ctx_e = vicp.Context(voxel_size=pair.voxel_size, dilation_layers=L_LAYERS, max_iters=1, rmse_eps=0.0,
                         flags=vicp.VICP_FLAG_KEEP_GRID)
    src_np = torch.from_numpy(pair.source).pin_memory().numpy()
    tgt_np = torch.from_numpy(pair.target).pin_memory().numpy()
    Pe = np.eye(4)
    for _ in range(3):
        ctx_e.register_host(src_np, tgt_np, Pe)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for k in range(e2e_steps):
        if k % ITERS_PER_REGISTRATION == 0:
            Pe = np.eye(4)
        st, Pe, it, rm = ctx_e.register_host(src_np, tgt_np, Pe)
        if st != 0:
            raise RuntimeError("e2e step failed: " + ctx_e.last_error())
    e2e_s = _max_over_ranks(time.perf_counter() - e0, ws)
    e2e_value = ws * e2e_steps / e2e_s
    e2e_replayed = ctx_e.graph_replayed()

    # ---- precision: the FP64 reduction + solve beside the double-float one ----
    ctx64, one_step64 = scene_stepper(vicp.VICP_FLAG_FP64_SOLVE)
    for k in range(5):
        one_step64(k)
    ms64 = _timed_steps(one_step64, min(args.steps, 600), flush, stream)
    ms_df = _timed_steps(one_step, min(args.steps, 600), flush, stream)   # the same count, same conditions
    ctx64.profile_enable(True)
    for k in range(min(args.steps, 300)):
        flush.fill_(k & 0xff)
        one_step64(k)
    prof64 = ctx64.profile_read()
    ctx64.profile_enable(False)
    # 30-iteration registrations (grid rebuilt each iteration, the timed
    # configuration) in both precisions against the oracle's
    ext = _extent(pair.target)
    t_or = time.perf_counter()
    rst, R, rit, hist = _oracle_register(pair, ITERS_PER_REGISTRATION) if rank == 0 else (0, np.eye(4), 0, [1.0])
    t_or = time.perf_counter() - t_or
    reg = {}
    for name, fl in (("double_float", 0), ("fp64", vicp.VICP_FLAG_FP64_SOLVE)):
        ctx_r = vicp.Context(voxel_size=pair.voxel_size, dilation_layers=L_LAYERS, max_iters=ITERS_PER_REGISTRATION,
                             rmse_eps=0.0, flags=vicp.VICP_FLAG_KEEP_GRID | vicp.VICP_FLAG_REBUILD_EACH_ITER | fl)
        st, T, it, rm = ctx_r.register(src, tgt)
        reg[name] = {"status": st, "iters": it, "rmse": rm, "pose": T.tolist(),
                     "pose_err_vs_oracle": {**_pose_err(T, R, ext), "oracle_iters": rit,
                                            "rmse_rel_diff": abs(rm - hist[-1]) / hist[-1]},
                     "rot_err_vs_truth_deg": round(math.degrees(_rot_err_rad(T, pair.T_gt)), 5),
                     "trans_err_vs_truth_m": float(np.linalg.norm(T[:3, 3] - pair.T_gt[:3, 3]))}
    rs64 = prof64.get("reduce_solve_f64", (0, 0.0))
    precision = {
        "double_float": {"label": PRECISION_LABEL["double_float"],
                         "iters_per_s": round(len(ms_df) / (sum(ms_df) / 1e3), 1),
                         "reduce_solve_us": kernels.get("reduce_solve", {}).get("avg_us"),
                         "registration_30": reg["double_float"]},
        "fp64": {"label": PRECISION_LABEL["fp64"],
                 "iters_per_s": round(len(ms64) / (sum(ms64) / 1e3), 1),
                 "reduce_solve_us": round(1e3 * rs64[1] / rs64[0], 3) if rs64[0] else None,
                 "registration_30": reg["fp64"]},
        "what": "the headline step (grid rebuilt, L2 flushed) with each reduction + solve, the same number of "
                "steps each, measured back to back; 30-iteration registrations against the FP64 CPU oracle "
                f"({t_or:.1f} s on {os.cpu_count()} threads)",
    }

    sections = set(args.sections.split(","))
    run_all = "all" in sections
    sparse = None
    if run_all or "sparse" in sections:
        dense_T = np.array(reg["double_float"]["pose"])
        sparse = run_sparse(dev, pair, flush, min(max(args.steps, 200), 600), dense_T, mem)
    workloads = None
    if run_all or "workloads" in sections:
        workloads = {p.name: run_workload(dev, p, flush, steps=min(max(args.steps, 200), 1000))
                     for p in (synth.sphere_plane(), synth.bumpy_object())}
    hist_ablation = run_hist_ablation(dev, tgt, view, mem["occupied_voxels"], flush) \
        if run_all or "hist" in sections else None
    fixed_capacity = run_fixed(dev, pair, flush) if run_all or "fixed" in sections else None
    batched = run_batched(dev, flush, rank, ws, n_pairs=32 if args.small else 256) \
        if run_all or "batched" in sections else None
    differentiable = run_loss(dev, flush, n_pairs=16 if args.small else 64) \
        if run_all or "loss" in sections else None

    result = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * total_s / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "depth_scene_226k: 640x480 synthetic depth image of planes and boxes, "
                               f"{N} target / {M} source points, 2 cm voxels, L={L_LAYERS}, "
                               f"{ITERS_PER_REGISTRATION}-iteration registrations from identity",
                   "grid": list(view.dims[0:3]), "voxels": V, "l2": "flushed between steps (256 MiB write)",
                   "precision": PRECISION_LABEL["double_float"],
                   "clock_window": f"{pre_roll} + {post_roll} identical untimed steps ({CLOCK_WINDOW_S} s each) "
                                   "around the timed steps, nvidia-smi sampled every 100 ms over all of them",
                   "parallelism": f"replicas x{ws}" + (", batched pairs sharded by pair" if ws > 1 else "")},
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": round(achieved, 1), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": _ncu_traffic(dominant), "alg_bytes_per_launch": dk["alg_bytes"]},
        "kernels": kernels,
        "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": int(16 * (N + M)),
                "d2h_bytes_per_step": 16 * 8 + 24 + 4, "graph_replayed": e2e_replayed,
                "what": "vicp_register_host with 1 iteration: H2D of both clouds from pinned memory, "
                        "grid build, dilation, one ICP step, pose + status read back (each call replayed "
                        "as one CUDA graph)"},
        "amortised_grid_built_once": {"value": round(amortised, 2), "unit": UNIT},
        "gpu_launches": int(gpu_launches),
        "clocks": clk.summary(),
        "wall_s_timed_loop": round(wall, 4),
        "pose_err_vs_oracle": reg["double_float"]["pose_err_vs_oracle"],
        "precision": precision,
        "search": {"fallbacks_per_iter": round(stats["fallbacks"] / args.steps, 1),
                   "local_candidates_per_iter": round(stats["local_candidates"] / args.steps, 1),
                   "global_candidates_per_iter": round(stats["global_candidates"] / args.steps, 1)},
        "memory": {"peak_device_bytes": mem["peak_bytes"], "csr_store_bytes": mem["csr_store_bytes"],
                   "static_bytes": mem["static_bytes"],
                   "fixed_capacity_bytes": mem["fixed_capacity_bytes"],
                   "paper_64KB_per_voxel_bytes": mem["paper_static_layout_bytes"],
                   "max_voxel_count": mem["max_voxel_count"], "occupied_voxels": mem["occupied_voxels"]},
        "sparse_grid": sparse,
        "workloads": workloads,
        "histogram_ablation": hist_ablation,
        "fixed_capacity_layout": fixed_capacity,
        "batched": batched,
        "differentiable": differentiable,
    }
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"], result["cpu_baseline_single_thread"] = cpu_baseline(pair)
    return result


# ----------------------------------------------------------------------------
# CPU oracle legs
# ----------------------------------------------------------------------------
def _oracle_iterations(pair, iters: int, threads: int):
    """`iters` full ICP iterations of the scene with the grid rebuilt each
    time, from the identity, on `threads` threads; returns (seconds, threads
    used)."""
    import oracle
    used = oracle.use_threads(threads)
    try:
        g = oracle.fit_grid(pair.target, pair.voxel_size, 0)
        T = np.eye(4)
        t0 = time.perf_counter()
        for _ in range(iters):
            b = oracle.build_grid(g, pair.target, L_LAYERS)
            st, T, *_ = oracle.iterate(g, b, pair.target, pair.source, T)
        return time.perf_counter() - t0, used
    finally:
        oracle.use_threads(1)


def cpu_baseline(pair):
    """The oracle as it stands on this host: full ICP iterations of the scene
    (grid rebuilt each), on all cores (the OpenMP build) and on one."""
    nproc = os.cpu_count() or 1
    dt, used = _oracle_iterations(pair, 4, nproc)
    all_cores = {"value": round(4 / dt, 4), "unit": UNIT, "cores": used, "kind": "oracle",
                 "sample": f"4 full ICP iterations of the 226k scene (grid rebuilt each), {dt:.1f} s "
                           f"on {used} threads (OpenMP build: parallel keys, dilation rounds and searches)"}
    dt1, _ = _oracle_iterations(pair, 2, 1)
    single = {"value": round(2 / dt1, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
              "sample": f"2 full ICP iterations of the 226k scene (grid rebuilt each), {dt1:.1f} s single-threaded"}
    return all_cores, single


def run_reference(args, rank, ws):
    """The oracle on the host cores: one step = one full ICP iteration of the
    scene with the grid rebuilt, on all cores.  When K + W such steps would
    not finish within about two minutes, each step searches a random sample
    of the source points instead and is scaled to a full iteration (the grid
    build is still timed in full every step)."""
    import oracle
    from paper_2512_04996_gb300 import synth
    if rank != 0:
        return None
    pair = synth.depth_scene()
    nproc = os.cpu_count() or 1
    used = oracle.use_threads(nproc)
    g = oracle.fit_grid(pair.target, pair.voxel_size, 0)
    M = pair.source.shape[0]
    # one untimed probe iteration decides between full and sampled steps
    t0 = time.perf_counter()
    b = oracle.build_grid(g, pair.target, L_LAYERS)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.iterate(g, b, pair.target, pair.source, np.eye(4))
    t_iter = time.perf_counter() - t0
    budget = 120.0
    full = (args.steps + args.warmup) * (t_build + t_iter) <= budget
    rng = np.random.default_rng(0)
    T = np.eye(4)
    steps_s = []
    for k in range(args.warmup + args.steps):
        if k % ITERS_PER_REGISTRATION == 0:
            T = np.eye(4)
        t0 = time.perf_counter()
        b = oracle.build_grid(g, pair.target, L_LAYERS)
        tb = time.perf_counter() - t0
        if full:
            t0 = time.perf_counter()
            st, T, *_ = oracle.iterate(g, b, pair.target, pair.source, T)
            step = tb + (time.perf_counter() - t0)
        else:
            per_step = budget / max(1, args.steps + args.warmup)
            m_s = int(max(256, min(M, (per_step - tb) / max(t_iter / M, 1e-9))))
            idx = np.sort(rng.choice(M, m_s, replace=False))
            sub = np.ascontiguousarray(pair.source[idx])
            t0 = time.perf_counter()
            oracle.iterate(g, b, pair.target, sub, T)
            step = tb + (time.perf_counter() - t0) * M / m_s
        if k >= args.warmup:
            steps_s.append(step)
    oracle.use_threads(1)
    total = sum(steps_s)
    value = args.steps / total
    sample = (f"full ICP iterations of the 226k scene, grid rebuilt every step, {used} threads" if full else
              f"grid build timed in full every step + the search, reduction and solve over a random sample of "
              f"source points scaled to all {M}, {used} threads")
    return {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "depth_scene_226k (same as ours), grid rebuilt every iteration, "
                                   "30-iteration registrations from identity",
                       "sampled": not full},
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sections", default="all",
                    help="extra measurements after the headline: all, or a comma list of sparse, workloads, hist, "
                         "fixed, batched, loss, none (for profiler captures)")
    ap.add_argument("--small", action="store_true",
                    help="batched and loss sections on 32 and 16 pairs (for profiler captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, ws, local = _dist_init()
    if args.impl == "reference":
        res = run_reference(args, rank, ws)
    else:
        res = run_ours(args, rank, ws, local)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
