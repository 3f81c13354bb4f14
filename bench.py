"""Benchmark: ICP iterations per second on the ~226k-point depth scene.

One step = one ICP iteration of the dilation-based ICP hot path with the grid
rebuilt: voxel histogram, offset scan, CSR scatter, brick list, dilation,
localised NNS with the exact global fallback, FP64 reduction and FP64 solve.
Steps cycle through the scene's 30-iteration registration from the identity
pose (the pose is reset every 30 steps), so the average step is the average
iteration of a registration.  Inputs are resident in HBM before timing; L2 is
flushed (a 256 MiB write) between timed steps, outside the timed events.

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank runs an
independent replica of the workload (no collective on the data path);
`value` = all ranks' iterations / the slowest rank's time.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

The line also carries `differentiable` (forward + backward of the
point-to-point loss over 64 pairs of 20k points) and `batched`: the 256-pair batched workload (sizes
log-uniform in 2k..64k points, 4.6M points per side, 40 iterations) in pairs/s
through the batched registration (one persistent launch per iteration,
replayed from a CUDA graph, kernel shape from the autotuner) against the same
256 pairs registered one at a time through the single-pair path, with the
pose agreement between the two.

`--impl reference` times the CPU oracle (the plain C restatement of the
paper) on this host's cores on a bounded sample of the same workload.
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

    def __init__(self, index: int):
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
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


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
# distributed plumbing (replicas only)
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
    if kernel == "reduce_solve":   # per point: source point, nn, gathered target point
        return 36 * M
    return 0.0


def _kernel_sha(kernel: str) -> str:
    src = {"histogram": ("vicp_grid.cu",), "scan": ("vicp_grid.cu",), "scatter": ("vicp_grid.cu",),
           "brick_scan": ("vicp_grid.cu",),
           "dilate": ("vicp_dilate.cu", "vicp_dilate.cuh"),
           "correspond": ("vicp_nns.cu", "vicp_search.cuh"), "fallback": ("vicp_nns.cu", "vicp_search.cuh"),
           "reduce_solve": ("vicp_solve.cu", "vicp_df.cuh")}.get(kernel)
    if not src:
        return ""
    h = hashlib.sha256()
    for name in src + ("vicp_device.cuh",):
        with open(os.path.join(ROOT, "paper_2512_04996_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel: str):
    """DRAM bytes (read + write) per launch from the committed ncu capture of
    this kernel, if the kernel's source is unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        with open(path) as f:
            for ln in f:
                if ln.startswith("#") or not ln.strip():
                    continue
                name, rd, wr, _t, sha = ln.split()
                if name == kernel:
                    return float(rd) + float(wr) if sha == _kernel_sha(kernel) else None
    except Exception:
        return None
    return None


# ----------------------------------------------------------------------------
# batched registration (256 uneven pairs) against one pair at a time
# ----------------------------------------------------------------------------
BATCH_ITERS = 40


def _rot_deg(Ta, Tb) -> float:
    E = Ta[:3, :3] @ Tb[:3, :3].T
    return math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(E) - 1.0) / 2.0))))


def run_batched(dev, flush, reps: int = 5, n_pairs: int = 256) -> dict:
    import torch

    from paper_2512_04996_gb300 import synth, vicp

    ps = synth.batched_pairs(n_pairs=n_pairs)
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
    b = vicp.Batch(dilation_layers=L_LAYERS, max_iters=BATCH_ITERS, rmse_eps=0.0)
    b.build(tgt, n_tgt, vs, dv)
    shape, tune_ms = b.tune(src, n_src, iters=4, trials=2)
    threads, ppt, blocks = vicp.vicp_batch_shape_info(shape)
    for _ in range(2):   # warm-up: captures the iteration graph
        st, T, it, rm, pst = b.register(src, n_src)
        if st != 0:
            raise RuntimeError("batched warm-up failed: " + b._lib.vicp_batch_last_error(b.handle).decode())
    b.report(reset=True)

    # build + 40 iterations of all pairs, per repetition (device time)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    reg_ms, launches0 = [], b.launch_count()
    for k in range(reps):
        flush.fill_(k & 0xff)
        e0, e1 = ev[k]
        e0.record(stream)
        b.build(tgt, n_tgt, vs, dv)
        e1.record(stream)
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        st, T, it, rm, pst = b.register(src, n_src)
        r1.record(stream)
        torch.cuda.synchronize()
        if st != 0:
            raise RuntimeError("batched run failed")
        reg_ms.append((e0.elapsed_time(e1), r0.elapsed_time(r1)))
    gpu_launches = b.launch_count() - launches0
    stats = b.report(reset=True)
    build_ms = statistics.median(x[0] for x in reg_ms)
    iter_ms = statistics.median(x[1] for x in reg_ms)
    batched_pps = P / ((build_ms + iter_ms) / 1e3)

    # the iteration kernel alone: one launch's average device time
    ctx_it = vicp.Batch(dilation_layers=L_LAYERS, max_iters=1, rmse_eps=0.0, shape=shape,
                        flags=vicp.VICP_BATCH_FLAG_NO_GRAPH)
    ctx_it.build(tgt, n_tgt, vs, dv)
    T_cur = np.ascontiguousarray(np.tile(np.eye(4), (P, 1, 1)))
    k_ms = []
    for k in range(BATCH_ITERS):
        flush.fill_(k & 0xff)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        st, T_cur, *_ = ctx_it.register(src, n_src, T_cur)
        a1.record(stream)
        torch.cuda.synchronize()
        k_ms.append(a0.elapsed_time(a1))
    it_stats = ctx_it.report(reset=True)

    # end to end: host clouds in, poses out, through vicp_batch_register_host
    bh = vicp.Batch(dilation_layers=L_LAYERS, max_iters=BATCH_ITERS, rmse_eps=0.0, shape=shape)
    src_pin = torch.from_numpy(src_np).pin_memory().numpy()
    tgt_pin = torch.from_numpy(tgt_np).pin_memory().numpy()
    bh.register_host(src_pin, n_src, tgt_pin, n_tgt, vs, dv)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        st, Th, *_ = bh.register_host(src_pin, n_src, tgt_pin, n_tgt, vs, dv)
    e2e_s = (time.perf_counter() - t0) / reps

    # one pair at a time through the single-pair path (vicp_register)
    src_t = [torch.from_numpy(p.source).to(dev) for p in ps]
    tgt_t = [torch.from_numpy(p.target).to(dev) for p in ps]
    ctxs = {d: vicp.Context(dilation_layers=L_LAYERS, max_iters=BATCH_ITERS, rmse_eps=0.0, grid_divisions=int(d))
            for d in sorted(set(int(x) for x in dv))}
    for d, c in ctxs.items():   # size every context's buffers once
        k = int(np.flatnonzero(dv == d)[np.argmax(n_tgt[dv == d])])
        c.register(src_t[k], tgt_t[k])
    torch.cuda.synchronize()
    flush.fill_(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = []
    for k, p in enumerate(ps):
        st, S, it1, rm1 = ctxs[int(dv[k])].register(src_t[k], tgt_t[k])
        plain.append(S)
    plain_s = time.perf_counter() - t0
    plain_pps = P / plain_s

    rot_diff = max(_rot_deg(T[k], plain[k]) for k in range(P))
    ext = [float((p.target[:, :3].max(0) - p.target[:, :3].min(0)).max()) for p in ps]
    tr_diff = max(float(np.linalg.norm(T[k][:3, 3] - plain[k][:3, 3])) / ext[k] for k in range(P))
    err_b = [_rot_deg(T[k], p.T_gt) for k, p in enumerate(ps)]
    err_p = [_rot_deg(plain[k], p.T_gt) for k, p in enumerate(ps)]
    rep = b.report()
    M, N = int(n_src.sum()), int(n_tgt.sum())
    return {
        "metric": "batched pairs/s (256 pairs, 40 iterations each, grids built per batch)",
        "value": round(batched_pps, 1), "unit": "pairs/s",
        "plain_one_at_a_time": {"value": round(plain_pps, 1), "unit": "pairs/s",
                                "what": "the same 256 pairs through vicp_register one after another "
                                        "(host wall clock, each call synchronises)"},
        "speedup_vs_plain": round(batched_pps / plain_pps, 2),
        "build_ms": round(build_ms, 3), "iterations_ms": round(iter_ms, 3),
        "iteration_kernel_us": round(1e3 * statistics.median(k_ms), 1),
        "e2e": {"value": round(P / e2e_s, 1), "unit": "pairs/s", "h2d_bytes_per_step": int(16 * (M + N)),
                "d2h_bytes_per_step": int(P * (16 * 8 + 48)),
                "what": "vicp_batch_register_host: H2D of all pooled clouds from pinned memory, build, "
                        "40 iterations, poses and states read back (host wall clock)"},
        "gpu_launches_per_batch": int(gpu_launches // reps),
        "shape": {"index": shape, "threads": threads, "points_per_thread": ppt, "resident_blocks": blocks,
                  "tune_ms": [round(float(x), 3) for x in tune_ms]},
        "accuracy": {"max_rot_diff_vs_plain_deg": rot_diff, "max_trans_diff_vs_plain_rel_extent": tr_diff,
                     "median_rot_err_vs_truth_deg": round(statistics.median(err_b), 6),
                     "median_rot_err_vs_truth_deg_plain": round(statistics.median(err_p), 6)},
        "search": {"fallbacks_per_batch": stats["fallbacks"] // reps,
                   "queries_per_batch": stats["queries"] // reps,
                   "iteration_kernel_fallbacks": it_stats["fallbacks"]},
        "workload": f"{P} pairs (even: sphere+plane, odd: bumpy object), sizes log-uniform in 2k..64k, "
                    f"{M} source / {N} target points, L={L_LAYERS}, {BATCH_ITERS} iterations from identity",
        "peak_device_bytes": rep["peak_bytes"],
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

    # builds: the CSR store's kernels (histogram, scan, scatter) by the
    # library's per-kernel timing; the fixed store's reset + scatter by events
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
    # searches at the true pose, each layout's localised search kernel alone
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
def run_loss(dev, flush, steps: int = 50, n_pairs: int = 64) -> dict:
    import torch

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
    return {
        "workload": f"{P} pairs x {int(n_src[0])} points (bumpy-object generator, voxel = extent/128), "
                    "loss of Eq. 1 at the true poses, gradients in 6 float32 se(3) parameters per pair "
                    "and in every source point",
        "what": "one forward (Exp, batched NNS, loss) + backward (loss gradients, left-Jacobian transpose) "
                "through torch.autograd, CUDA events on the stream",
        **out,
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
    flags = vicp.VICP_FLAG_KEEP_GRID
    ctx = vicp.Context(voxel_size=pair.voxel_size, dilation_layers=L_LAYERS, max_iters=1, rmse_eps=0.0,
                       flags=flags)
    pose = torch.eye(4, dtype=torch.float64, device=dev).contiguous()
    eye = torch.eye(4, dtype=torch.float64, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def one_step(k):
        if k % ITERS_PER_REGISTRATION == 0:
            pose.copy_(eye)
        ctx.build_grid(tgt)
        ctx.dilate(L_LAYERS)
        ctx.step(src, pose)

    # warm-up (also fits the grid geometry once: KEEP_GRID)
    for k in range(args.warmup):
        one_step(k)
    if ctx.sync() != 0:
        raise RuntimeError("warm-up failed: " + ctx.last_error())
    view = ctx.grid_view()
    V = int(view.n_voxels)

    # ---- timed pass: per-step CUDA events, L2 flushed between steps ----------
    ctx.read_stats(reset=True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = ctx.launch_count()
    _barrier(ws)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(_smi_id(dev)) as clk:
        for k in range(args.steps):
            flush.fill_(k & 0xff)
            starts[k].record(stream)
            one_step(k)
            ends[k].record(stream)
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    _barrier(ws)
    gpu_launches = ctx.launch_count() - launches0
    if ctx.sync() != 0:
        raise RuntimeError("timed pass failed: " + ctx.last_error())
    stats = ctx.read_stats(reset=True)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s = sum(step_ms) / 1e3
    total_s = _max_over_ranks(total_s, ws)
    value = ws * args.steps / total_s

    # ---- per-kernel times (the library's event timing) ------------------------
    prof_steps = min(args.steps, 300)
    ctx.profile_enable(True)
    for k in range(prof_steps):
        flush.fill_(k & 0xff)
        one_step(k)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    pstats = ctx.read_stats(reset=True)
    mem = ctx.memory_report()
    kernels = {}
    nbt = int(math.ceil(view.dims[0] / 8) * math.ceil(view.dims[1] / 8) * math.ceil(view.dims[2] / 8))
    w = dict(V=V, N=N, M=M, occupied=mem["occupied_voxels"], bricks=nbt, nonempty_bricks=mem["nonempty_bricks"])
    per_launch_w = dict(w)
    per_launch_w.update(queries=pstats["queries"] / prof_steps, fallbacks=pstats["fallbacks"] / prof_steps,
                        local_cand=pstats["local_candidates"] / prof_steps,
                        global_cand=pstats["global_candidates"] / prof_steps)
    for name, (n_l, ms) in prof.items():
        if n_l:
            avg_ms = ms / n_l
            b = algorithmic_bytes(name, per_launch_w)
            kernels[name] = {"launches": n_l, "total_ms": round(ms, 4), "avg_us": round(1e3 * avg_ms, 3),
                             "alg_bytes": int(b), "gbs": round(b / (avg_ms * 1e-3) / 1e9, 1) if b else None}
    dominant = max(kernels, key=lambda k: kernels[k]["total_ms"])
    peak, peak_kind = _peaks()
    dk = kernels[dominant]
    achieved = dk["gbs"] if dk["gbs"] else 0.0

    # ---- grid built once (amortised over the registration) --------------------
    amort_steps = min(args.steps, 600)
    ctx.build_grid(tgt)
    ctx.dilate(L_LAYERS)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    amort_ms = 0.0
    for k in range(amort_steps):
        if k % ITERS_PER_REGISTRATION == 0:
            pose.copy_(eye)
        flush.fill_(k & 0xff)
        a0.record(stream)
        ctx.step(src, pose)
        a1.record(stream)
        a1.synchronize()
        amort_ms += a0.elapsed_time(a1)
    amortised = amort_steps / (amort_ms / 1e3)

    # ---- end to end through the C ABI with host buffers -----------------------
    e2e_steps = min(args.steps, 200)
    ctx_e = vicp.Context(voxel_size=pair.voxel_size, dilation_layers=L_LAYERS, max_iters=1, rmse_eps=0.0,
                         flags=vicp.VICP_FLAG_KEEP_GRID)
    src_h = torch.from_numpy(pair.source).pin_memory()
    tgt_h = torch.from_numpy(pair.target).pin_memory()
    src_np, tgt_np = src_h.numpy(), tgt_h.numpy()
    P = np.eye(4)
    for _ in range(3):
        ctx_e.register_host(src_np, tgt_np, P)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for k in range(e2e_steps):
        if k % ITERS_PER_REGISTRATION == 0:
            P = np.eye(4)
        st, P, it, rm = ctx_e.register_host(src_np, tgt_np, P)
        if st != 0:
            raise RuntimeError("e2e step failed: " + ctx_e.last_error())
    e2e_s = _max_over_ranks(time.perf_counter() - e0, ws)
    e2e_value = ws * e2e_steps / e2e_s

    # ---- registration accuracy (30 iterations, grid built once) --------------
    ctx_r = vicp.Context(voxel_size=pair.voxel_size, dilation_layers=L_LAYERS,
                         max_iters=ITERS_PER_REGISTRATION, rmse_eps=0.0)
    st, T, it, rm = ctx_r.register(src, tgt)
    E = T @ np.linalg.inv(pair.T_gt)
    rot_err_deg = math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(E[:3, :3]) - 1) / 2))))

    sections = set(args.sections.split(","))
    run_all = "all" in sections
    hist_ablation = run_hist_ablation(dev, tgt, view, mem["occupied_voxels"], flush) \
        if run_all or "hist" in sections else None
    fixed_capacity = run_fixed(dev, pair, flush) if run_all or "fixed" in sections else None
    batched = run_batched(dev, flush, n_pairs=32 if args.small else 256) \
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
                   "precision": "f32 coordinates/distances, f64 reduction and solve",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": round(achieved, 1), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": _ncu_traffic(dominant), "alg_bytes_per_launch": dk["alg_bytes"]},
        "kernels": kernels,
        "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": int(16 * (N + M)),
                "d2h_bytes_per_step": 16 * 8 + 24 + 4,
                "what": "vicp_register_host with 1 iteration: H2D of both clouds from pinned memory, "
                        "grid build, dilation, one ICP step, pose + status read back"},
        "amortised_grid_built_once": {"value": round(amortised, 2), "unit": UNIT},
        "gpu_launches": int(gpu_launches),
        "clocks": clk.summary(),
        "wall_s_timed_loop": round(wall, 3),
        "search": {"fallbacks_per_iter": round(stats["fallbacks"] / args.steps, 1),
                   "local_candidates_per_iter": round(stats["local_candidates"] / args.steps, 1),
                   "global_candidates_per_iter": round(stats["global_candidates"] / args.steps, 1)},
        "memory": {"peak_device_bytes": mem["peak_bytes"], "csr_store_bytes": mem["csr_store_bytes"],
                   "static_bytes": mem["static_bytes"],
                   "fixed_capacity_bytes": mem["fixed_capacity_bytes"],
                   "paper_64KB_per_voxel_bytes": mem["paper_static_layout_bytes"],
                   "max_voxel_count": mem["max_voxel_count"], "occupied_voxels": mem["occupied_voxels"]},
        "registration": {"status": st, "iters": it, "rmse": rm, "rot_err_vs_truth_deg": round(rot_err_deg, 5),
                         "trans_err_vs_truth_m": float(np.linalg.norm(E[:3, 3]))},
        "histogram_ablation": hist_ablation,
        "fixed_capacity_layout": fixed_capacity,
        "batched": batched,
        "differentiable": differentiable,
    }
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(pair)
    return result


# ----------------------------------------------------------------------------
# CPU oracle legs
# ----------------------------------------------------------------------------
def cpu_baseline(pair, iters: int = 2) -> dict:
    """The oracle as it stands, single-threaded: `iters` ICP iterations of the
    scene, each with the grid rebuilt, from the identity pose."""
    import oracle
    g = oracle.fit_grid(pair.target, pair.voxel_size, 0)
    T = np.eye(4)
    t0 = time.perf_counter()
    for _ in range(iters):
        b = oracle.build_grid(g, pair.target, L_LAYERS)
        st, T, *_ = oracle.iterate(g, b, pair.target, pair.source, T)
    dt = time.perf_counter() - t0
    return {"value": round(iters / dt, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{iters} full ICP iterations of the 226k scene (grid rebuilt each), "
                      f"{dt:.1f} s single-threaded"}


def run_reference(args, rank, ws):
    """The oracle on the host cores: grid build timed once, then per step one
    search + reduction + solve over a random sample of the source points,
    scaled to a full iteration."""
    import oracle
    from paper_2512_04996_gb300 import synth
    if rank != 0:
        return None
    pair = synth.depth_scene()
    g = oracle.fit_grid(pair.target, pair.voxel_size, 0)
    t0 = time.perf_counter()
    b = oracle.build_grid(g, pair.target, L_LAYERS)
    t_build = time.perf_counter() - t0
    M = pair.source.shape[0]
    budget = 120.0 / max(1, args.steps + args.warmup)
    per_point = 4e-5
    rng = np.random.default_rng(0)
    steps_s = []
    for k in range(args.warmup + args.steps):
        m_s = int(max(256, min(M, budget / per_point)))
        idx = np.sort(rng.choice(M, m_s, replace=False))
        sub = np.ascontiguousarray(pair.source[idx])
        t0 = time.perf_counter()
        oracle.iterate(g, b, pair.target, sub, np.eye(4))
        dt = time.perf_counter() - t0
        per_point = dt / m_s
        if k >= args.warmup:
            steps_s.append(t_build + per_point * M)
    total = sum(steps_s)
    value = args.steps / total
    return {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "depth_scene_226k (same as ours)", "identity pose": True},
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"grid build timed once ({t_build:.2f} s) + per step the search, "
                                       f"reduction and solve over a random sample of source points "
                                       f"scaled to all {M}"},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sections", default="all",
                    help="extra measurements after the headline: all, or a comma list of hist, fixed, batched, "
                         "loss, none (for profiler captures)")
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
