"""Benchmark: segment x label cost volumes + winner-take-all depth for every reference view.

One step = one pass of the hot path over one synthetic frame of the 3840x2160 15-view convergent-arc
workload: pack the 15 views, build the 15 segment indexes, the 15 cost volumes (49432 segments x 400
labels, min over the 14 other views, 6.97e11 pixel x label x view evaluations, all references in one
launch of the cost kernel) and the 15 winner-take-all depth maps. --workload hd8 selects the 1920x1080
8-view workload instead.
`value` = evaluations / s with inputs resident in HBM; `e2e` = the same metric through the C ABI
with the inputs copied from pinned host memory and the depth labels read back inside the timed
region. The L2 is flushed (256 MB write) before every timed step.

--impl reference times the CPU oracle as it stands on a bounded sample of the same workload.
--part segmentation times the superpixel segmentation (Sec. IV-C) of every view of the workload instead;
--part centre the centre table (Eq. 4 at segment centres, Eq. 5's correspondence) and --part adjacency the
segment adjacency and beta (Eq. 2-3) of every reference.
Multi-GPU (torchrun): every rank runs an independent replica (the work shards by frames/jobs; there is
no exchange step), rank 0 prints the whole-job throughput from the slowest rank's time.
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
sys.path.insert(0, ROOT)

METRIC = "pixel·label·view evals/s"
UNIT = "evals/s"
WORKLOAD = "uhd15"


def reduce_max(value: float, device) -> float:
    """Largest value over the ranks of the default process group (the value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: float, slowest_seconds: float) -> float:
    """Whole-job throughput of `world` replicas that each processed units_per_rank units, timed by the
    slowest rank."""
    return world * units_per_rank / slowest_seconds


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _workload_desc(wl):
    S = wl.labels(wl.ref_views[0])[1]
    c = wl.cams[0]
    chroma = "4:4:4 (4:2:0 upsampled)" if wl.chroma420 else "4:4:4"
    return (f"{wl.name}: {wl.n_views} views {c.width}x{c.height} {wl.bit_depth}-bit {chroma}, "
            f"{S} segments/view, {wl.n_labels} labels, {len(wl.ref_views)} references, "
            f"{len(wl.neighbours(wl.ref_views[0]))} neighbours, min over views")


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _traffic_for_current_kernel(workload_key: str, table: str = "cost_kernel_traffic.txt",
                                source: str = "ftv_cost.cu", column: int = 2):
    """Bytes per launch of a kernel from the committed ncu summary table (column 2: DRAM read + write; columns
    3 and 4, where given: L2 and L1 bytes), if it was taken on the current source of that kernel (hash match);
    else None."""
    path = os.path.join(ROOT, "profiles", table)
    src = os.path.join(ROOT, "paper_1909_02294_gb300", "csrc", source)
    if not os.path.exists(path):
        return None
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    for line in open(path):
        parts = line.split("#")[0].split()
        if len(parts) > column and parts[0] == workload_key and parts[1] == h:
            return float(parts[column])
    return None


def algorithmic_bytes(wl, culled: int = 0) -> tuple[int, int]:
    """Per cost-volume launch: (evaluation bytes, compulsory bytes). One sampled evaluation reads one
    3-sample texel of the neighbour view (3 x sample_bytes); evaluations the kernel decided without
    sampling (a whole tile out of a neighbour's view, ftv_culled_evaluations) read nothing. Compulsory
    streams are every packed view read once, each reference pixel's index record and reference texel,
    and the int32 volume written once."""
    sb = wl.sample_bytes
    evals = wl.evaluations() - culled
    comp = 0
    for v in range(wl.n_views):
        c = wl.cams[v]
        comp += c.width * c.height * 4
    for r in wl.ref_views:
        c = wl.cams[r]
        S = wl.labels(r)[1]
        comp += c.width * c.height * 8 + S * wl.n_labels * 4
    return evals * 3 * sb, comp


# Issue slots the cost contract needs per pixel x label x neighbour evaluation at the least: 6 FMA
# (projection), 1 reciprocal, 2 multiplies, 2 adds (+0.5), 2 floor-converts, the in-view test, 1 address
# multiply-add, 1 gather, |dY|+|dCb|+|dCr| and 1 min over views, about 25 in all.
OPS_PER_EVAL = 25
# ... plus one add per pixel x label for the segment sum.
OPS_PER_PIXEL_LABEL = 1


def algorithmic_ops(wl, culled: int = 0) -> int:
    """Per cost-volume launch; a culled evaluation (decided without sampling) is not charged."""
    px_labels = sum(wl.cams[r].width * wl.cams[r].height * wl.n_labels for r in wl.ref_views)
    return (wl.evaluations() - culled) * OPS_PER_EVAL + px_labels * OPS_PER_PIXEL_LABEL


def _oracle_table(wl, r, nb, fp64: bool):
    import oracle
    table = oracle.homography_table_f64 if fp64 else oracle.homography_table
    return table(wl.cams, r, nb, wl.n_labels, wl.z_near, wl.z_far)


def cpu_baseline(wl, budget_s: float = 12.0, min_rows: int = 4, fp64: bool = False):
    """Time the oracle as it stands on the first k segments of reference 0 (whole label rows), k chosen
    so the run takes about budget_s seconds (FP64 projection mode with fp64). Returns (evals/s, sample
    description)."""
    import oracle
    r = wl.ref_views[0]
    lab, S = wl.labels(r)
    nb = wl.neighbours(r)
    H = _oracle_table(wl, r, nb, fp64)
    views = wl.views()
    sizes = np.bincount(lab.ravel(), minlength=S)
    out = np.zeros((S, wl.n_labels), np.int32)

    def run(k):
        lst = np.arange(k, dtype=np.int32)
        t = time.perf_counter()
        oracle.cost_volume(wl.cams, views, wl.sample_bytes, r, nb, H, wl.n_labels, lab, S, wl.oob_penalty,
                           wl.combine, seg_list=lst, out=out)
        dt = time.perf_counter() - t
        return int(sizes[:k].sum()) * wl.n_labels * len(nb), dt

    ev, dt = run(min_rows)
    k = int(min(S, max(min_rows, min_rows * budget_s / max(dt, 1e-3))))
    ev, dt = run(k)
    return ev / dt, f"oracle, 1 thread: cost rows of segments 0..{k - 1} of reference {r} ({ev:.3e} evaluations)", k


# Superpixel segmentation (Sec. IV-C). Operations the distance contract performs per (pixel, candidate
# cluster) pair of an assignment pass: 2 coordinate and 3 colour differences, 5 squares, 3 adds, the two
# weight products and their sum, 1 compare and 1 select.
SEG_OPS_PER_CANDIDATE = 18
SEG_COMPACTNESS, SEG_PASSES = 5, 10


def seg_candidates(W: int, H: int, S: int) -> int:
    """Exact (pixel, candidate cell) pairs of one assignment pass: the 3 x 3 neighbouring cells that exist."""
    def axis(n):
        cells = -(-n // S)
        ci = np.arange(n) // S
        return int(np.sum(np.minimum(ci + 1, cells - 1) - np.maximum(ci - 1, 0) + 1))
    return axis(W) * axis(H)


def seg_cpu_baseline(view, sb, bd, S, budget_s: float = 10.0):
    """The oracle's segmentation as it stands (one thread) on the first rows of one view, the row count
    chosen so the run takes about budget_s seconds. Returns (pixels/s, sample description)."""
    import oracle
    import synth

    def crop(rows):
        return synth.View(*(np.ascontiguousarray(np.asarray(a)[:rows]) for a in (view.Y, view.U, view.V)))

    W = np.asarray(view.Y).shape[1]
    rows = 2 * S
    t = time.perf_counter()
    oracle.superpixels(crop(rows), sb, bd, S, SEG_COMPACTNESS, SEG_PASSES)
    dt = time.perf_counter() - t
    rows = int(min(np.asarray(view.Y).shape[0], max(rows, rows * budget_s / max(dt, 1e-3))))
    t = time.perf_counter()
    oracle.superpixels(crop(rows), sb, bd, S, SEG_COMPACTNESS, SEG_PASSES)
    dt = time.perf_counter() - t
    return W * rows / dt, f"oracle, 1 thread: rows 0..{rows - 1} of view 0 ({W * rows} pixels, {SEG_PASSES} passes)"


def run_segmentation(args, rank, world, local):
    """One step = segmenting every view of the workload in one call (ftv_superpixels)."""
    import torch
    import torch.distributed as dist
    import paper_1909_02294_gb300 as ftv
    import synth

    wl = synth.make_workload(args.workload)
    dev = torch.device("cuda", local)
    S, sb, bd = wl.cell, wl.sample_bytes, wl.bit_depth
    views = wl.views()
    sizes = [(np.asarray(v.Y).shape[1], np.asarray(v.Y).shape[0]) for v in views]
    sg = ftv.Segmenter(sizes, sb, bd, S, SEG_COMPACTNESS, SEG_PASSES)
    segs = ftv.ftv_segmenter_segments(sg)
    host_planes = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (v.Y, v.U, v.V)] for v in views]
    planes = [[t.to(dev) for t in trip] for trip in host_planes]
    labels = [torch.empty((h, w), dtype=torch.int32, device=dev) for w, h in sizes]
    host_labels = [torch.empty((h, w), dtype=torch.int32).pin_memory() for w, h in sizes]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream(dev)

    def step():
        ftv.ftv_superpixels(sg, planes, labels)

    for _ in range(args.warmup):
        step()
    if ftv.ftv_segmenter_check(sg) != 0:
        raise RuntimeError("segmenter device status")
    ftv.ftv_segmenter_set_profiling(sg, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    assign_ms = []
    launches0 = ftv.ftv_segmenter_launch_count(sg)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            assign_ms.append(ftv.ftv_segmenter_kernel_ms(sg)[0])
        torch.cuda.synchronize()
    launches = ftv.ftv_segmenter_launch_count(sg) - launches0
    if world > 1:
        dist.barrier()
    total_s = reduce_max(sum(a.elapsed_time(b) for a, b in ev) / 1000.0, dev)
    pixels = sum(w * h for w, h in sizes)
    value = whole_job_rate(world, pixels * args.steps, total_s)
    if ftv.ftv_segmenter_check(sg) != 0:
        raise RuntimeError("segmenter device status")

    ftv.ftv_segmenter_set_profiling(sg, False)
    h2d = sum(t.numel() * t.element_size() for trip in host_planes for t in trip)
    d2h = sum(t.numel() * t.element_size() for t in host_labels)
    e2e_ev = []
    torch.cuda.synchronize()
    for k in range(max(3, args.steps // 2)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for trip_h, trip_d in zip(host_planes, planes):
            for th, td in zip(trip_h, trip_d):
                td.copy_(th, non_blocking=True)
        step()
        for th, td in zip(host_labels, labels):
            th.copy_(td, non_blocking=True)
        b.record(stream)
        e2e_ev.append((a, b))
    torch.cuda.synchronize()
    e2e_s = reduce_max(sum(a.elapsed_time(b) for a, b in e2e_ev) / 1000.0, dev)

    if rank == 0:
        peak, peak_kind = _peaks()
        clk = clocks.summary()
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        sm_mhz = clk["sm_mhz"] if clk else 2070.0
        alu_peak = n_sm * 128 * sm_mhz * 1e6 / 1e12
        ams = statistics.mean(assign_ms)
        ops = sum(seg_candidates(w, h, S) for w, h in sizes) * SEG_OPS_PER_CANDIDATE
        pass_bytes = pixels * (3 * sb + 4)
        c = wl.cams[0]
        line = {
            "metric": "segmented pixels/s", "value": value, "unit": "px/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "i32+i64", "data": "synthetic",
            "config": {"workload": f"superpixels of {wl.name}: {len(views)} views {c.width}x{c.height} {bd}-bit, "
                                   f"S = {S} ({segs[0]} segments/view), m = {SEG_COMPACTNESS}, {SEG_PASSES} passes",
                       "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "segmentations_per_s": whole_job_rate(world, len(views) * args.steps, total_s),
                       "assign_pass_ms": ams},
            "roofline": {"bound": "alu", "achieved": ops / (ams / 1000.0) / 1e12, "peak": alu_peak, "unit": "Tops/s",
                         "frac": ops / (ams / 1000.0) / 1e12 / alu_peak,
                         "traffic": _traffic_for_current_kernel(args.workload, "assign_kernel_traffic.txt",
                                                                "ftv_superpixels.cu"),
                         "peak_kind": f"{n_sm} SMs x 128 lanes x {sm_mhz:.0f} MHz (median sampled SM clock)",
                         "algorithmic_ops_per_launch": ops, "ops_per_candidate": SEG_OPS_PER_CANDIDATE,
                         "kernel": "assign_kernel (one assignment pass over every view)"},
            "hbm_roofline": {"bound": "hbm", "achieved": pass_bytes / (ams / 1000.0) / 1e9, "peak": peak,
                             "unit": "GB/s", "frac": pass_bytes / (ams / 1000.0) / 1e9 / peak,
                             "peak_kind": peak_kind, "algorithmic_bytes_per_launch": pass_bytes,
                             "definition": "three samples read and one int32 label written per pixel"},
            "e2e": {"value": whole_job_rate(world, pixels * len(e2e_ev), e2e_s), "unit": "px/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
        }
        if world == 1 and not args.no_cpu_baseline:
            rate, desc = seg_cpu_baseline(views[0], sb, bd, S)
            line["cpu_baseline"] = {"value": rate, "unit": "px/s", "cores": 1, "kind": "oracle", "sample": desc}
        print(json.dumps(line), flush=True)
    sg.close()


def cpu_baseline_all_cores(wl, k_single: int, budget_s: float = 10.0, fp64: bool = False):
    """The same oracle, unchanged, on every host core: threads compute disjoint segment rows of reference 0
    (the oracle keeps no global state and ctypes releases the GIL during the call). Each thread takes at
    most the row count one thread did in the single-thread baseline. Returns (evals/s, threads, sample)."""
    import concurrent.futures as cf
    import oracle
    r = wl.ref_views[0]
    lab, S = wl.labels(r)
    nb = wl.neighbours(r)
    views = wl.views()
    sizes = np.bincount(lab.ravel(), minlength=S)
    out = np.zeros((S, wl.n_labels), np.int32)
    H = _oracle_table(wl, r, nb, fp64)
    threads = max(1, os.cpu_count() or 1)
    per = max(1, min(k_single, S // threads))
    parts = [np.arange(t * per, (t + 1) * per, dtype=np.int32) for t in range(threads) if (t + 1) * per <= S]

    def run(lst):
        oracle.cost_volume(wl.cams, views, wl.sample_bytes, r, nb, H, wl.n_labels, lab, S, wl.oob_penalty,
                           wl.combine, seg_list=lst, out=out)

    t = time.perf_counter()
    with cf.ThreadPoolExecutor(len(parts)) as ex:
        list(ex.map(run, parts))
    dt = time.perf_counter() - t
    n = len(parts) * per
    ev = int(sizes[:n].sum()) * wl.n_labels * len(nb)
    return ev / dt, len(parts), (f"oracle on {len(parts)} threads: cost rows of segments 0..{n - 1} of reference {r} "
                                 f"({ev:.3e} evaluations)")


# Centre table (Eq. 4 literal at segment centres with the Eq. 5 correspondence): operations per (segment,
# label, neighbour) entry: the projection of the centre (6 FMA, 1 reciprocal, 2 multiplies, 2 adds, 2 floors,
# 5 compares) and per window pixel pair 2 gathers, 3 differences, 3 absolute values, 2 adds, 1 accumulate.
CENTRE_WINDOW = 3


def centre_ops_per_entry(window: int) -> int:
    return 18 + 11 * window * window


def _part_line(args, world, metric, unit, value, total_s, extra_config, roofline, e2e, launches, clocks, wl):
    c = wl.cams[0]
    return {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+i32", "data": "synthetic",
            "config": {"workload": f"{wl.name}: {wl.n_views} views {c.width}x{c.height} {wl.bit_depth}-bit, "
                                   f"{wl.labels(wl.ref_views[0])[1]} segments/view",
                       "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU", **extra_config},
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clocks}


# Temporal test thresholds for 10-bit samples: the paper's 8-bit T_P = 3, T_I = 1 scaled by 4.
TEMPORAL_T_P, TEMPORAL_T_I = 12, 4


def run_part(args, rank, world, local):
    """--part centre: one step = the centre table of every reference (ftv_centre_table, one call).
    --part adjacency: one step = adjacency and beta of every reference (ftv_adjacency per reference).
    --part temporal: one step = the temporal test of every reference (one ftv_temporal_mask_views call, luma
    mode) of the temporal workload's frame 1 against frame 0 as the previous P and the I frame.
    The roofline is taken over the whole call (pack, segment index and the part's kernels)."""
    import torch
    import torch.distributed as dist
    import paper_1909_02294_gb300 as ftv
    import synth
    import oracle

    wl = synth.make_workload("temporal" if args.part == "temporal" and args.workload == WORKLOAD else args.workload)
    dev = torch.device("cuda", local)
    R, L = len(wl.ref_views), wl.n_labels
    S = [wl.labels(r)[1] for r in wl.ref_views]
    ctx = ftv.ftv_depth_init(wl.cams, wl.ref_views, L, wl.z_near, wl.z_far, sample_bytes=wl.sample_bytes,
                             bit_depth=wl.bit_depth, oob_penalty=wl.oob_penalty, max_segments=max(S))
    views = wl.views()
    host_planes = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (v.Y, v.U, v.V)] for v in views]
    planes = [[t.to(dev) for t in trip] for trip in host_planes]
    host_labels = [torch.from_numpy(wl.labels(v)[0]).pin_memory() for v in range(wl.n_views)]
    labels = [t.to(dev) for t in host_labels]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    nbrs = [wl.neighbours(r) for r in wl.ref_views]
    if args.part == "centre":
        m_out = [torch.empty((S[i], L, len(nbrs[i])), dtype=torch.int32, device=dev) for i in range(R)]
        sp_out = [torch.empty_like(t) for t in m_out]
        host_out = [torch.empty(t.shape, dtype=torch.int32).pin_memory() for t in m_out]
        units = sum(S[i] * L * len(nbrs[i]) for i in range(R))

        def step():
            ftv.ftv_centre_table(ctx, planes, labels, S, CENTRE_WINDOW, m_out, sp_out)
        outs = m_out
    elif args.part == "temporal":
        # a step's new input is the current frame (the previous and I frames are resident from earlier
        # steps); luma mode reads one plane of each
        cur_host = [torch.from_numpy(np.ascontiguousarray(wl.view(r, 1).Y)).pin_memory() for r in wl.ref_views]
        cur = [t.to(dev) for t in cur_host]
        ref_prev = [planes[r][0] for r in wl.ref_views]  # frame 0
        masks = [torch.empty(S[i], dtype=torch.uint8, device=dev) for i in range(R)]
        changed = [torch.empty(S[i], dtype=torch.int32, device=dev) for i in range(R)]
        n_changed = [torch.zeros(1, dtype=torch.int32, device=dev) for _ in range(R)]
        host_out = [torch.empty(S[i], dtype=torch.uint8).pin_memory() for i in range(R)]
        units = sum(wl.cams[r].width * wl.cams[r].height for r in wl.ref_views)

        trips_cur = [(cur[i], None, None) for i in range(R)]
        trips_prev = [(ref_prev[i], None, None) for i in range(R)]
        ref_labels = [labels[r] for r in wl.ref_views]

        def step():
            # every reference of the frame in one ftv_temporal_mask_views call (one launch sequence)
            ftv.ftv_temporal_mask_views(ctx, list(range(R)), trips_cur, trips_prev, trips_prev, ref_labels, S,
                                        TEMPORAL_T_P, TEMPORAL_T_I, ftv.FTV_TM_Y_ONLY, masks, changed, n_changed)
        outs = masks
    else:
        cap = [8 * S[i] + 64 for i in range(R)]
        es = [torch.empty(c, dtype=torch.int32, device=dev) for c in cap]
        et = [torch.empty(c, dtype=torch.int32, device=dev) for c in cap]
        beta = [torch.empty(c, dtype=torch.float32, device=dev) for c in cap]
        ne = [torch.zeros(1, dtype=torch.int32, device=dev) for _ in range(R)]
        host_out = [torch.empty(c, dtype=torch.float32).pin_memory() for c in cap]
        units = sum(wl.cams[r].width * wl.cams[r].height for r in wl.ref_views)

        def step():
            for i, r in enumerate(wl.ref_views):
                ftv.ftv_adjacency(ctx, i, planes[r], labels[r], S[i], 4, 1.0, 1.0, es[i], et[i], beta[i], ne[i])
        outs = beta

    for _ in range(args.warmup):
        step()
    if ftv.ftv_check(ctx) != 0:
        raise RuntimeError("device status")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = ftv.ftv_launch_count(ctx)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    launches = ftv.ftv_launch_count(ctx) - launches0
    if world > 1:
        dist.barrier()
    step_s = [a.elapsed_time(b) / 1000.0 for a, b in ev]
    total_s = reduce_max(sum(step_s), dev)
    value = whole_job_rate(world, units * args.steps, total_s)
    if ftv.ftv_check(ctx) != 0:
        raise RuntimeError("device status")
    # end to end: the step's inputs up (planes and label maps; the temporal test: the current frame), the
    # part's result down, every step
    if args.part == "temporal":
        uploads = list(zip(cur_host, cur))
    else:
        uploads = [(th, td) for trip_h, trip_d in zip(host_planes, planes) for th, td in zip(trip_h, trip_d)]
        uploads += list(zip(host_labels, labels))
    h2d = sum(th.numel() * th.element_size() for th, _ in uploads)
    d2h = sum(t.numel() * t.element_size() for t in host_out)
    e2e_ev = []
    torch.cuda.synchronize()
    for k in range(max(3, args.steps // 2)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for th, td in uploads:
            td.copy_(th, non_blocking=True)
        step()
        for th, td in zip(host_out, outs):
            th.copy_(td, non_blocking=True)
        b.record(stream)
        e2e_ev.append((a, b))
    torch.cuda.synchronize()
    e2e_s = reduce_max(sum(a.elapsed_time(b) for a, b in e2e_ev) / 1000.0, dev)

    if rank == 0:
        clk = clocks.summary()
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        sm_mhz = clk["sm_mhz"] if clk else 2070.0
        mean_s = statistics.mean(step_s)
        if args.part == "centre":
            ops = units * centre_ops_per_entry(CENTRE_WINDOW)
            peak = n_sm * 128 * sm_mhz * 1e6 / 1e12
            roof = {"bound": "alu", "achieved": ops / mean_s / 1e12, "peak": peak, "unit": "Tops/s",
                    "frac": ops / mean_s / 1e12 / peak, "traffic": None,
                    "peak_kind": f"{n_sm} SMs x 128 lanes x {sm_mhz:.0f} MHz (median sampled SM clock)",
                    "algorithmic_ops_per_step": ops, "ops_per_entry": centre_ops_per_entry(CENTRE_WINDOW),
                    "kernel": "the whole ftv_centre_table call (pack, segment index, centroids, table)"}
            metric, unit = "centre-table entries/s", "entries/s"
            extra = {"window": CENTRE_WINDOW, "entries_per_step": units, "labels": L,
                     "neighbours": len(nbrs[0])}
        elif args.part == "temporal":
            peak, peak_kind = _peaks()
            byts = units * (3 * wl.sample_bytes + 4) + sum(S) * 5
            roof = {"bound": "hbm", "achieved": byts / mean_s / 1e9, "peak": peak, "unit": "GB/s",
                    "frac": byts / mean_s / 1e9 / peak, "traffic": None, "peak_kind": peak_kind,
                    "algorithmic_bytes_per_step": byts,
                    "definition": "per pixel its label and three luma samples (current, previous, I) read "
                                  "once, per segment its mask byte and list entry written",
                    "kernel": "the whole ftv_temporal_mask_views call (accumulate, decide and compact kernels)"}
            metric, unit = "temporal-test pixels/s", "px/s"
            extra = {"mode": "luma, previous P and I frame", "t_p": TEMPORAL_T_P, "t_i": TEMPORAL_T_I,
                     "changed_per_step": sum(int(t.item()) for t in n_changed)}
        else:
            peak, peak_kind = _peaks()
            n_edges = sum(int(t.item()) for t in ne)
            byts = units * (4 + 3 * wl.sample_bytes) + n_edges * 12
            roof = {"bound": "hbm", "achieved": byts / mean_s / 1e9, "peak": peak, "unit": "GB/s",
                    "frac": byts / mean_s / 1e9 / peak, "traffic": None, "peak_kind": peak_kind,
                    "algorithmic_bytes_per_step": byts,
                    "definition": "per pixel its label and three samples read once, per edge 12 bytes written",
                    "kernel": "the whole ftv_adjacency calls (segment index, neighbours, offsets, edges)"}
            metric, unit = "adjacency pixels/s", "px/s"
            extra = {"connectivity": 4, "edges_per_step": n_edges}
        line = _part_line(args, world, metric, unit, value, total_s, extra, roof,
                          {"value": whole_job_rate(world, units * len(e2e_ev), e2e_s), "unit": unit,
                           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}, launches, clk, wl)
        if world == 1 and not args.no_cpu_baseline:
            r0 = wl.ref_views[0]
            lab0, S0 = wl.labels(r0)
            if args.part == "centre":
                Lsub = 4
                H = oracle.homography_table(wl.cams, r0, nbrs[0], L, wl.z_near, wl.z_far)[:, :Lsub]
                labs_v = [wl.labels(v)[0] for v in range(wl.n_views)]
                t = time.perf_counter()
                oracle.centre_table(wl.cams, views, wl.sample_bytes, r0, nbrs[0], np.ascontiguousarray(H), Lsub,
                                    labs_v, S0, CENTRE_WINDOW, wl.oob_penalty)
                dt = time.perf_counter() - t
                n = S0 * Lsub * len(nbrs[0])
                line["cpu_baseline"] = {"value": n / dt, "unit": unit, "cores": 1, "kind": "oracle",
                                        "sample": f"oracle, 1 thread: the table of reference {r0} for labels "
                                                  f"0..{Lsub - 1} ({n} entries)"}
            elif args.part == "temporal":
                t = time.perf_counter()
                oracle.temporal_mask(lab0, S0, wl.view(r0, 1), wl.view(r0, 0), wl.view(r0, 0), wl.sample_bytes,
                                     TEMPORAL_T_P, TEMPORAL_T_I, 0)
                dt = time.perf_counter() - t
                n = lab0.size
                line["cpu_baseline"] = {"value": n / dt, "unit": unit, "cores": 1, "kind": "oracle",
                                        "sample": f"oracle, 1 thread: the temporal test of reference {r0} "
                                                  f"({n} pixels)"}
            else:
                t = time.perf_counter()
                oracle.adjacency(lab0, S0, views[r0], wl.sample_bytes, 4, 1.0, 1.0)
                dt = time.perf_counter() - t
                n = lab0.size
                line["cpu_baseline"] = {"value": n / dt, "unit": unit, "cores": 1, "kind": "oracle",
                                        "sample": f"oracle, 1 thread: adjacency and beta of reference {r0} "
                                                  f"({n} pixels)"}
        print(json.dumps(line), flush=True)
    ctx.close()


def run_reference(args, rank):
    if rank != 0:
        return
    import synth
    wl = synth.make_workload(args.workload)
    per_step = max(0.5, min(8.0, 90.0 / (args.steps + args.warmup)))  # whole run within a few minutes
    rate, desc, k = cpu_baseline(wl, budget_s=per_step)
    times, evals = [], 0
    import oracle
    lab_cache = {}
    for it in range(args.warmup + args.steps):
        r = wl.ref_views[it % len(wl.ref_views)]
        if r not in lab_cache:
            lab_cache[r] = wl.labels(r)
        lab, S = lab_cache[r]
        nb = wl.neighbours(r)
        H = oracle.homography_table(wl.cams, r, nb, wl.n_labels, wl.z_near, wl.z_far)
        lst = np.arange(min(k, S), dtype=np.int32)
        sizes = np.bincount(lab.ravel(), minlength=S)
        out = np.zeros((S, wl.n_labels), np.int32)
        t = time.perf_counter()
        oracle.cost_volume(wl.cams, wl.views(), wl.sample_bytes, r, nb, H, wl.n_labels, lab, S, wl.oob_penalty,
                           wl.combine, seg_list=lst, out=out)
        dt = time.perf_counter() - t
        if it >= args.warmup:
            times.append(dt)
            evals += int(sizes[: len(lst)].sum()) * wl.n_labels * len(nb)
    total = sum(times)
    value = evals / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+i32", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": _workload_desc(wl), "sample": f"cost rows of {len(lst)} segments per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"cost rows of the first {k} segments of one reference per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="synthetic workload (default: the 1920x1080 8-view configuration; others for profiling)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="sample positions of the depth part: the FP32 contract (default) or the FP64 projection")
    ap.add_argument("--part", default="depth", choices=["depth", "segmentation", "centre", "adjacency", "temporal"],
                    help="depth: the cost-volume hot path (default); segmentation: superpixels of every view; "
                         "centre: the centre table of every reference; adjacency: adjacency and beta; "
                         "temporal: the temporal test of every reference (temporal workload)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    if args.part != "depth":
        (run_segmentation if args.part == "segmentation" else run_part)(args, rank, world, local)
        if world > 1:
            dist.destroy_process_group()
        return

    import paper_1909_02294_gb300 as ftv
    import synth

    wl = synth.make_workload(args.workload)
    dev = torch.device("cuda", local)
    R, L = len(wl.ref_views), wl.n_labels
    S = [wl.labels(r)[1] for r in wl.ref_views]
    fp64 = args.precision == "fp64"
    ctx = ftv.ftv_depth_init(wl.cams, wl.ref_views, L, wl.z_near, wl.z_far, sample_bytes=wl.sample_bytes,
                             bit_depth=wl.bit_depth, oob_penalty=wl.oob_penalty, max_segments=max(S),
                             precision=ftv.FTV_PRECISION_FP64 if fp64 else ftv.FTV_PRECISION_FP32)
    host_views = wl.views()
    host_planes = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (v.Y, v.U, v.V)]
                   for v in host_views]
    host_labels = [torch.from_numpy(wl.labels(r)[0]).pin_memory() for r in wl.ref_views]
    planes = [[t.to(dev) for t in trip] for trip in host_planes]
    labels = [t.to(dev) for t in host_labels]
    costs = [torch.empty((s, L), dtype=torch.int32, device=dev) for s in S]
    wins = [torch.empty(s, dtype=torch.int16, device=dev) for s in S]
    host_wins = [torch.empty(s, dtype=torch.int16).pin_memory() for s in S]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream(dev)

    def step():
        ftv.ftv_cost_volume(ctx, planes, labels, S, costs)
        for i in range(R):
            ftv.ftv_wta_depth(ctx, i, costs[i], S[i], wins[i])

    # launch shape of the cost kernel: the autotuner's choice for this job class (cached per machine), chosen
    # before the untimed warm-up steps
    from paper_1909_02294_gb300 import tune
    key = tune.job_class(wl.cams, wl.ref_views, [len(wl.neighbours(r)) for r in wl.ref_views], L, wl.sample_bytes,
                         wl.bit_depth, ftv.FTV_COMBINE_MIN, ftv.FTV_PRECISION_FP64 if fp64 else ftv.FTV_PRECISION_FP32,
                         torch.cuda.get_device_name(dev))
    shape_rec = tune.apply_or_tune(ctx, key, planes, labels, S, costs, reps=2)
    shape_now = ftv.ftv_get_launch_shape(ctx)

    for _ in range(args.warmup):
        step()
    st = ftv.ftv_check(ctx)
    if st != 0:
        raise RuntimeError(f"device status {ftv.ftv_status_str(st)}")

    ftv.ftv_set_profiling(ctx, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kernel_ms = []
    launches0 = ftv.ftv_launch_count(ctx)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            kernel_ms.append(ftv.ftv_last_kernel_ms(ctx))
        torch.cuda.synchronize()
    launches = ftv.ftv_launch_count(ctx) - launches0
    culled = ftv.ftv_culled_evaluations(ctx)  # the same for every step (the last launch's count)
    recomputed = ftv.ftv_fp64_recomputed(ctx)
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = reduce_max(sum(step_ms) / 1000.0, dev)
    evals = wl.evaluations()
    value = whole_job_rate(world, evals * args.steps, total_s)
    st = ftv.ftv_check(ctx)
    if st != 0:
        raise RuntimeError(f"device status {ftv.ftv_status_str(st)}")

    # End to end through the C ABI: every step copies its planes and label maps from pinned host memory
    # and reads its depth labels back. Pipelined: step k + 1's inputs are copied on a second stream into
    # the other of two device input sets while step k computes; the timed region runs from the first
    # copy's start to the last read-back's end.
    ftv.ftv_set_profiling(ctx, False)
    h2d = sum(t.numel() * t.element_size() for trip in host_planes for t in trip)
    h2d += sum(t.numel() * t.element_size() for t in host_labels)
    d2h = sum(t.numel() * t.element_size() for t in host_wins)
    n_e2e = max(3, args.steps // 2)
    inputs = [(planes, labels), ([[torch.empty_like(t) for t in trip] for trip in planes],
                                 [torch.empty_like(t) for t in labels])]
    host_out = [host_wins, [torch.empty_like(t).pin_memory() for t in host_wins]]
    copy_stream = torch.cuda.Stream(dev)
    copied = [torch.cuda.Event() for _ in range(n_e2e)]
    computed = [torch.cuda.Event() for _ in range(n_e2e)]

    def upload(k):
        with torch.cuda.stream(copy_stream):
            if k >= 2:
                copy_stream.wait_event(computed[k - 2])  # that input set was step k - 2's
            pl, lb = inputs[k % 2]
            for trip_h, trip_d in zip(host_planes, pl):
                for th, td in zip(trip_h, trip_d):
                    td.copy_(th, non_blocking=True)
            for th, td in zip(host_labels, lb):
                td.copy_(th, non_blocking=True)
            copied[k].record(copy_stream)

    torch.cuda.synchronize()
    e2e_start, e2e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_start.record(copy_stream)
    upload(0)
    for k in range(n_e2e):
        if k + 1 < n_e2e:
            upload(k + 1)
        stream.wait_event(copied[k])
        flush.zero_()
        pl, lb = inputs[k % 2]
        ftv.ftv_cost_volume(ctx, pl, lb, S, costs)
        for i in range(R):
            ftv.ftv_wta_depth(ctx, i, costs[i], S[i], wins[i])
        for th, td in zip(host_out[k % 2], wins):
            th.copy_(td, non_blocking=True)
        computed[k].record(stream)
    e2e_end.record(stream)
    torch.cuda.synchronize()
    e2e_s = reduce_max(e2e_start.elapsed_time(e2e_end) / 1000.0, dev)
    e2e_value = whole_job_rate(world, evals * n_e2e, e2e_s)

    if rank == 0:
        peak, peak_kind = _peaks()
        ev_bytes, comp_bytes = algorithmic_bytes(wl, culled)
        kms = statistics.mean(kernel_ms)
        achieved = (ev_bytes + comp_bytes) / (kms / 1000.0) / 1e9
        traffic = _traffic_for_current_kernel(args.workload + ("_fp64" if fp64 else ""))
        l2_bytes = _traffic_for_current_kernel(args.workload + ("_fp64" if fp64 else ""), column=3)
        l1_bytes = _traffic_for_current_kernel(args.workload + ("_fp64" if fp64 else ""), column=4)
        clk = clocks.summary()
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        sm_mhz = clk["sm_mhz"] if clk else 2070.0
        alu_peak = n_sm * 128 * sm_mhz * 1e6 / 1e12  # lane operations per second, Tops/s
        alu_achieved = algorithmic_ops(wl, culled) / (kms / 1000.0) / 1e12
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+i32", "data": "synthetic",
            "config": {"workload": _workload_desc(wl), "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "depth_maps_per_s": whole_job_rate(world, R * args.steps, total_s),
                       "cost_kernel_ms": kms, "evaluations_per_step": evals,
                       "culled_evaluations_per_step": culled, "culled_fraction": culled / evals,
                       "precision": "FP64 projection" if fp64 else "FP32 contract",
                       "launch_shape": {"label_block": shape_now["label_block"],
                                        "ctas_per_sm": shape_now["ctas_per_sm"], "chosen_by": shape_rec["source"],
                                        "autotune_grid_ms": shape_rec.get("grid_ms")},
                       **({"fp64_recomputed_per_step": recomputed, "fp64_recomputed_fraction": recomputed / evals}
                          if fp64 else {})},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": ev_bytes + comp_bytes,
                         "definition": "one 3-sample texel (3 x sample bytes) per sampled evaluation (culled "
                                       "ones read nothing) + compulsory streams, over the cost kernel's "
                                       "event-timed duration",
                         "kernel": "cost_kernel<FMT_P10, MIN" + (", FP64 projection>" if fp64 else ">"),
                         "compulsory_bytes_per_launch": comp_bytes,
                         "compulsory_floor_ms": comp_bytes / (peak * 1e9) * 1e3,
                         "dram_fraction_of_algorithmic": (traffic / (ev_bytes + comp_bytes)) if traffic else None,
                         "ncu_dram_gbs": (traffic / (kms / 1000.0) / 1e9) if traffic else None,
                         "ncu_l2_gbs": (l2_bytes / (kms / 1000.0) / 1e9) if l2_bytes else None,
                         "ncu_l1_gbs": (l1_bytes / (kms / 1000.0) / 1e9) if l1_bytes else None,
                         "note": "a notional gather rate: most gathers hit L1/L2, and the DRAM traffic (traffic) "
                                 "is a small fraction of the algorithmic bytes; the kernel is issue/ALU-bound"},
            "alu_roofline": {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "Tops/s",
                             "frac": alu_achieved / alu_peak,
                             "peak_kind": f"{n_sm} SMs x 128 lanes x {sm_mhz:.0f} MHz (median sampled SM clock)",
                             "algorithmic_ops_per_launch": algorithmic_ops(wl, culled),
                             "ops_per_evaluation": OPS_PER_EVAL},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": n_e2e, "overlap": "step k+1's uploads on a second stream during step k (two input sets)"},
            "gpu_launches": launches,
            "clocks": clk,
        }
        if world == 1 and not args.no_cpu_baseline:
            rate, desc, k = cpu_baseline(wl, fp64=fp64)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
            rate_mt, threads, desc_mt = cpu_baseline_all_cores(wl, k, fp64=fp64)
            line["cpu_baseline_all_cores"] = {"value": rate_mt, "unit": UNIT, "cores": threads, "kind": "oracle",
                                              "sample": desc_mt}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
