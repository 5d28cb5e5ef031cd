"""Serving loop: continuous batching of depth jobs from many camera streams.

A thin host driver over the C ABI (all per-pixel work runs in the library's kernels). Each camera
stream is an ftv_ctx with resident temporal state (ftv_stream_init): its label maps, segment indexes,
previous-P and I frames and their per-segment labels stay on the device, so P frames only estimate
segments whose colour changed (Sec. III-E; 9 P frames between I frames as in the paper's experiments).

Served mode: up to `slots` batches are in flight on separate CUDA streams. Whenever a slot is free,
every request that has arrived, whose stream has no frame in flight (in-stream order is kept) and whose
footprint fits the HBM admission budget is admitted into one batch: its planes are copied from pinned
host memory on the slot's stream, the job is queued with ftv_batch_submit (one ticket per job) and the
batch is launched through its captured graph (ftv_batch_flush); each job completes when
ftv_batch_poll reports its ticket done, with that job's own status. Requests that arrive while others are
on the GPU join the next free slot. A job's footprint is ftv_job_footprint of its stream: the stream's
context, its resident state (frames, per-segment labels, cost rows) and one input frame.

Plain mode (the comparison): the same requests in arrival order, one job at a time, each launched on
its own (ftv_batch_launch of a single job, no graph) and completed before the next starts. Its GPU-busy
fraction (the jobs' launch sequences timed with CUDA events, summed, over the run's wall time) bounds
what any batching can gain over it: at most 1 / busy.

Both modes run the same kernels on the same stream states and produce bit-identical labels.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import ftv

T_P_10BIT, T_I_10BIT = 12, 4  # the paper's T_P = 3, T_I = 1 for 8-bit samples, scaled to 10 bits


@dataclass
class Request:
    rid: int
    sid: int
    seq: int          # position in its stream
    arrival: float    # seconds from the start of the run
    admitted: float = -1.0
    done: float = -1.0


class Stream:
    def __init__(self, wl, n_frames: int, gop: int, device, keep_labels: bool = False):
        self.wl = wl
        self.gop = gop
        self.S = [wl.labels(r)[1] for r in wl.ref_views]
        self.ctx = ftv.ftv_depth_init(wl.cams, wl.ref_views, wl.n_labels, wl.z_near, wl.z_far,
                                      sample_bytes=wl.sample_bytes, bit_depth=wl.bit_depth,
                                      oob_penalty=wl.oob_penalty, max_segments=max(self.S))
        labels = [torch.from_numpy(wl.labels(r)[0]).to(device) for r in wl.ref_views]
        ftv.ftv_stream_init(self.ctx, labels, self.S, T_P_10BIT, T_I_10BIT, ftv.FTV_TM_Y_ONLY)
        self.frames = []
        for k in range(n_frames):
            self.frames.append([[torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (v.Y, v.U, v.V)]
                                for v in wl.views(k)])
            wl.drop_frame(k)
        self.frame_bytes = sum(t.numel() * t.element_size() for trip in self.frames[0] for t in trip) \
            if self.frames else 0
        self.footprint = ftv.ftv_job_footprint(wl.cams, wl.ref_views, wl.n_labels, wl.z_near, wl.z_far, max(self.S),
                                               sample_bytes=wl.sample_bytes, bit_depth=wl.bit_depth,
                                               max_segments=max(self.S))
        self.out = [torch.zeros(s, dtype=torch.int16, device=device) for s in self.S]
        self.keep = keep_labels
        self.history = []
        self.busy = False
        self.n_refs = len(wl.ref_views)
        self.n_views = wl.n_views
        self.shape = (wl.cams[0].width, wl.cams[0].height, wl.n_views, wl.n_labels)
        self.heavy = wl.evaluations() >= HEAVY_EVALS

    def frame_type(self, seq: int) -> int:
        return ftv.FTV_FRAME_I if seq % self.gop == 0 else ftv.FTV_FRAME_P

    def upload(self, seq: int, stream):
        host = self.frames[seq % len(self.frames)]
        with torch.cuda.stream(stream):
            return [[t.to(stream.device, non_blocking=True) for t in trip] for trip in host]

    def job(self, seq: int, planes) -> dict:
        return {"ctx": self.ctx, "planes": planes, "frame_type": self.frame_type(seq), "label_out": self.out}

    def record(self):
        if self.keep:
            self.history.append([o.cpu().numpy().view(np.uint16).copy() for o in self.out])

    def close(self):
        self.ctx.close()


def poisson_trace(n_streams: int, n_jobs: int, rate: float, seed: int) -> list[Request]:
    """n_jobs requests, Poisson arrivals of total rate `rate` (jobs/s), stream chosen uniformly."""
    rng = np.random.default_rng(seed)
    t, reqs, seq = 0.0, [], [0] * n_streams
    for i in range(n_jobs):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        sid = int(rng.integers(n_streams))
        reqs.append(Request(i, sid, seq[sid], t))
        seq[sid] += 1
    return reqs


@dataclass
class Slot:
    batches: dict   # one ftv_batch per stream shape (each keeps its own captured graph)
    hi: object      # high-priority stream (batches of light shapes)
    lo: object      # low-priority stream (batches of heavy shapes)
    cur: object = None
    reqs: list = field(default_factory=list)
    tickets: list = field(default_factory=list)
    inputs: list = field(default_factory=list)
    bytes: int = 0
    heavy: bool = False


HEAVY_EVALS = 1e11  # a stream whose full frame is this many evaluations saturates the GPU by itself
HEAVY_CHUNKS = 16   # cost-kernel launches per heavy batch: light work can start between two of them


def run_served(streams: list[Stream], reqs: list[Request], slots: int = 3, budget_bytes: int = 16 << 30,
               max_jobs: int = 32, by_class: bool = True, heavy_exclusive: bool = True,
               heavy_chunks: int = HEAVY_CHUNKS) -> dict:
    """by_class: a batch only takes jobs of one stream shape (the shape of the earliest admissible
    request), so small jobs are not held until a large job in the same batch completes.
    heavy_exclusive: at most one batch of heavy streams (a full frame >= HEAVY_EVALS evaluations) is in
    flight; such a batch fills the GPU alone, and two of them running concurrently only contend for SMs
    and L2 (measured: 3 slots 131 vs 1 slot 147 depth maps/s on the full mix).
    heavy_chunks: a heavy batch runs its cost work in this many launches on a low-priority stream, light
    batches in one launch on a high-priority stream, so a light batch waits for at most about one chunk of
    a heavy one instead of all of it (ftv_batch_set_chunks)."""
    dev = torch.device("cuda")
    max_units = min(240, sum(s.n_refs for s in streams))
    max_views = sum(s.n_views for s in streams)
    low, high = torch.cuda.Stream.priority_range()  # e.g. (0, -5): a smaller number is a higher priority
    pool = [Slot({}, torch.cuda.Stream(dev, priority=high), torch.cuda.Stream(dev, priority=low))
            for _ in range(slots)]
    pending = list(reqs)  # arrival order
    inflight_bytes, done, batches, batch_sizes = 0, 0, 0, []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while done < len(reqs):
        now = time.perf_counter() - t0
        progressed = False
        for sl in pool:
            if not sl.reqs:
                continue
            polls = [ftv.ftv_batch_poll(sl.cur, t) for t in sl.tickets]
            if all(rc == 0 for rc, _ in polls):
                bad = [ftv.ftv_status_str(st) for _, st in polls if st != 0]
                if bad:
                    raise RuntimeError(f"job failed: {bad[0]}")
                t_done = time.perf_counter() - t0
                for r in sl.reqs:
                    r.done = t_done
                    streams[r.sid].busy = False
                    streams[r.sid].record()
                done += len(sl.reqs)
                inflight_bytes -= sl.bytes
                sl.reqs, sl.tickets, sl.inputs, sl.bytes = [], [], [], 0
                progressed = True
        free = [sl for sl in pool if not sl.reqs]
        heavy_busy = heavy_exclusive and any(sl.reqs and sl.heavy for sl in pool)
        if free:
            chosen, units, views, add_bytes, seen, cls = [], 0, 0, 0, set(), None
            for r in pending:
                if r.arrival > now:
                    break
                s = streams[r.sid]
                if r.sid in seen:
                    continue  # only a stream's earliest pending request may go (in-stream order)
                seen.add(r.sid)
                if s.busy:
                    continue
                if inflight_bytes + add_bytes + s.footprint > budget_bytes and (inflight_bytes or chosen):
                    continue  # admission by HBM footprint: wait until in-flight jobs free up (a job
                    # larger than the whole budget still runs, alone, when nothing else is in flight)
                if len(chosen) >= max_jobs or units + s.n_refs > max_units or views + s.n_views > max_views:
                    continue
                if by_class and cls is not None and s.shape != cls:
                    continue
                if heavy_busy and s.heavy:
                    continue
                cls = s.shape
                chosen.append(r)
                units += s.n_refs
                views += s.n_views
                add_bytes += s.footprint
            if chosen:
                sl = free[0]
                heavy = any(streams[r.sid].heavy for r in chosen)
                key = cls if by_class else None
                if key not in sl.batches:
                    b = ftv.ftv_batch_create(max_jobs, max_units, max_views)
                    ftv.ftv_batch_set_chunks(b, heavy_chunks if heavy and by_class else 1)
                    sl.batches[key] = b
                sl.cur = sl.batches[key]
                stream = sl.lo if heavy else sl.hi
                tickets = []
                for r in chosen:
                    s = streams[r.sid]
                    planes = s.upload(r.seq, stream)
                    sl.inputs.append(planes)
                    rc, t = ftv.ftv_batch_submit(sl.cur, s.job(r.seq, planes))
                    if rc != 0:
                        raise RuntimeError(f"submit failed: {ftv.ftv_status_str(rc)}")
                    tickets.append(t)
                    s.busy = True
                    r.admitted = now
                    pending.remove(r)
                rc = ftv.ftv_batch_flush(sl.cur, stream)
                if rc != 0:
                    raise RuntimeError(f"flush failed: {ftv.ftv_status_str(rc)}")
                sl.reqs, sl.tickets, sl.bytes = chosen, tickets, add_bytes
                sl.heavy = heavy
                inflight_bytes += add_bytes
                batches += 1
                batch_sizes.append(len(chosen))
                progressed = True
        if not progressed:
            time.sleep(20e-6)
    launches = sum(ftv.ftv_batch_launch_count(b) for sl in pool for b in sl.batches.values())
    for sl in pool:
        for b in sl.batches.values():
            b.close()
    out = _stats(streams, reqs)
    out.update({"mode": "served", "slots": slots, "batches": batches,
                "mean_batch_jobs": float(np.mean(batch_sizes)) if batch_sizes else 0.0, "gpu_launches": launches})
    return out


def run_plain(streams: list[Stream], reqs: list[Request]) -> dict:
    dev = torch.device("cuda")
    st = torch.cuda.Stream(dev)
    batch = ftv.ftv_batch_create(1, max(s.n_refs for s in streams), max(s.n_views for s in streams))
    per_job = []
    gpu_ms = 0.0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in reqs:
        while time.perf_counter() - t0 < r.arrival:
            time.sleep(20e-6)
        r.admitted = time.perf_counter() - t0
        s = streams[r.sid]
        planes = s.upload(r.seq, st)
        rc = ftv.ftv_batch_prepare(batch, [s.job(r.seq, planes)])
        if rc != 0:
            raise RuntimeError(f"prepare failed: {ftv.ftv_status_str(rc)}")
        ev0.record(st)
        ftv.ftv_batch_launch(batch, st)
        ev1.record(st)
        rc = ftv.ftv_batch_wait(batch)
        ev1.synchronize()
        gpu_ms += ev0.elapsed_time(ev1)
        if rc != 0:
            raise RuntimeError(f"batch failed: {ftv.ftv_status_str(rc)}")
        r.done = time.perf_counter() - t0
        s.record()
        per_job.append((f"{s.wl.cams[0].width}x{s.wl.cams[0].height}", "I" if s.frame_type(r.seq) == 0 else "P",
                        (r.done - r.admitted) * 1e3))
    launches = ftv.ftv_batch_launch_count(batch)
    batch.close()
    out = _stats(streams, reqs)
    service = {}
    for shape, ftype, ms in per_job:
        service.setdefault(f"{shape} {ftype}", []).append(ms)
    out.update({"mode": "plain", "gpu_launches": launches, "gpu_busy_ms": gpu_ms,
                "gpu_busy_fraction": gpu_ms / 1e3 / out["wall_s"],
                "service_ms_by_shape_and_type": {k: float(np.mean(v)) for k, v in sorted(service.items())}})
    return out


class _DeviceArray:
    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3}


def _device_int32(ptr: int):
    return torch.as_tensor(_DeviceArray(ptr, (1,), "<i4"), device="cuda")


def run_sequence(wl, n_frames: int, gop: int, replay: bool = True) -> dict:
    """One camera stream over n_frames consecutive frames (I frame every `gop` frames, P frames between):
    device-resident inputs, each frame timed with CUDA events on the launching stream. Reports depth
    maps/s over the sequence and the fraction of segments each P frame re-estimated."""
    dev = torch.device("cuda")
    s = Stream(wl, 0, gop, dev)
    frames = []
    for k in range(n_frames):
        frames.append([[torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (v.Y, v.U, v.V)]
                       for v in wl.views(k)])
        wl.drop_frame(k)
    batch = ftv.ftv_batch_create(1, s.n_refs, s.n_views)
    st = torch.cuda.current_stream(dev)
    counts = [ftv.ftv_stream_mask(s.ctx, i)[1] for i in range(s.n_refs)]
    ms, changed = [], []
    torch.cuda.synchronize()
    for k in range(n_frames):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        rc = ftv.ftv_batch_prepare(batch, [s.job(k, frames[k])])
        if rc != 0:
            raise RuntimeError(ftv.ftv_status_str(rc))
        a.record(st)
        (ftv.ftv_batch_replay if replay else ftv.ftv_batch_launch)(batch, st)
        b.record(st)
        if ftv.ftv_batch_wait(batch) != 0:
            raise RuntimeError("sequence frame failed")
        ms.append(a.elapsed_time(b))
        n = sum(int(_device_int32(p).item()) for p in counts)
        changed.append(n / sum(s.S))
    batch.close()
    s.close()
    p_idx = [k for k in range(n_frames) if k % gop]
    total_s = sum(ms) / 1e3
    return {"frames": n_frames, "gop": gop, "depth_maps": n_frames * s.n_refs,
            "depth_maps_per_s": n_frames * s.n_refs / total_s, "ms_per_frame": sum(ms) / n_frames,
            "ms_i_frame": float(np.mean([ms[k] for k in range(n_frames) if k % gop == 0])),
            "ms_p_frame": float(np.mean([ms[k] for k in p_idx])) if p_idx else None,
            "changed_fraction_p_frames": float(np.mean([changed[k] for k in p_idx])) if p_idx else None,
            "evaluations_i_frame": wl.evaluations()}


def _stats(streams, reqs) -> dict:
    lat = np.array([r.done - r.arrival for r in reqs]) * 1e3
    maps = sum(streams[r.sid].n_refs for r in reqs)
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    by_shape = {}
    for r in reqs:
        key = f"{streams[r.sid].wl.cams[0].width}x{streams[r.sid].wl.cams[0].height}"
        by_shape.setdefault(key, []).append((r.done - r.arrival) * 1e3)
    return {"jobs": len(reqs), "depth_maps": maps, "wall_s": span, "depth_maps_per_s": maps / span,
            "jobs_per_s": len(reqs) / span, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "p99_ms_by_shape": {k: float(np.percentile(v, 99)) for k, v in sorted(by_shape.items())}}


def tune_streams(streams: list[Stream], reps: int = 1) -> dict:
    """One autotuner run per stream shape (on its first stream's first frame, or the JSON cache of
    tune.py), the chosen launch shape applied to every stream of that shape. Returns {shape: record}."""
    from . import tune
    chosen = {}
    for st in streams:
        if st.shape not in chosen:
            wl = st.wl
            planes = st.upload(0, torch.cuda.current_stream())
            labels = [torch.from_numpy(wl.labels(r)[0]).cuda() for r in wl.ref_views]
            costs = [torch.empty((n, wl.n_labels), dtype=torch.int32, device="cuda") for n in st.S]
            key = tune.job_class(wl.cams, wl.ref_views, [len(wl.neighbours(r)) for r in wl.ref_views], wl.n_labels,
                                 wl.sample_bytes, wl.bit_depth, ftv.FTV_COMBINE_MIN, ftv.FTV_PRECISION_FP32,
                                 torch.cuda.get_device_name())
            chosen[st.shape] = tune.apply_or_tune(st.ctx, key, planes, labels, st.S, costs, reps=reps)
        rec = chosen[st.shape]
        ftv.ftv_set_launch_shape(st.ctx, rec["label_block"], rec["ctas_per_sm"])
    torch.cuda.synchronize()
    return {f"{k[0]}x{k[1]}/{k[2]}v/{k[3]}L": {"label_block": v["label_block"], "ctas_per_sm": v["ctas_per_sm"],
                                              "source": v["source"]} for k, v in chosen.items()}


def make_streams(per_shape: int, gop: int, n_frames: int, keep_labels: bool = False, shapes=None,
                 tune: bool = False):
    import synth.configs as configs
    wls = configs.serving_streams(per_shape)
    if shapes is not None:
        wls = [w for w in wls if any(w.name.startswith(p) for p in shapes)]
    dev = torch.device("cuda")
    streams = [Stream(w, n_frames if w.cams[0].width < 3840 else max(2, n_frames // 2), gop, dev, keep_labels)
               for w in wls]
    if tune:
        tune_streams(streams)
    return streams


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--jobs", type=int, default=2000)
    ap.add_argument("--per-shape", type=int, default=4, help="streams per shape (3 shapes)")
    ap.add_argument("--gop", type=int, default=10, help="frames per I frame (paper: 9 P frames between I frames)")
    ap.add_argument("--frames", type=int, default=4, help="distinct frames rendered per stream (cycled)")
    ap.add_argument("--slots", type=int, default=3)
    ap.add_argument("--budget-gb", type=float, default=16.0,
                    help="HBM admission budget: footprints (ftv_job_footprint) of the jobs in flight")
    ap.add_argument("--rate-frac", type=float, default=0.7, help="arrival rate as a fraction of measured capacity")
    ap.add_argument("--capacity-jobs", type=int, default=0, help="jobs of the saturated capacity run (0: --jobs)")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--shapes", default=None, help="comma-separated stream name prefixes (default: all)")
    ap.add_argument("--mixed-batches", action="store_true", help="let one batch mix stream shapes")
    ap.add_argument("--heavy-chunks", type=int, default=HEAVY_CHUNKS,
                    help="cost-kernel launches per heavy batch (1: one persistent launch)")
    ap.add_argument("--sequence", default=None, help="run one stream of this workload (e.g. temporal) over --frames")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch shapes (no autotuner run or cache lookup per stream shape)")
    ap.add_argument("--capacity-only", action="store_true", help="only the capacity runs (no Poisson arrivals)")
    args = ap.parse_args(argv)
    shapes = args.shapes.split(",") if args.shapes else None
    if args.sequence:
        import synth
        res = run_sequence(synth.make_workload(args.sequence), args.frames, args.gop)
        res["workload"] = args.sequence
        print(json.dumps(res), flush=True)
        return res

    def fresh():
        return make_streams(args.per_shape, args.gop, args.frames, shapes=shapes, tune=not args.no_tune)

    budget = int(args.budget_gb * (1 << 30))
    n_cap = args.capacity_jobs or args.jobs
    results = {}
    # capacity of each mode: every request present at t = 0
    for mode in ("served", "plain"):
        streams = fresh()
        trace = poisson_trace(len(streams), n_cap, 0.0, args.seed)
        res = run_served(streams, trace, args.slots, budget, by_class=not args.mixed_batches,
                         heavy_chunks=args.heavy_chunks) \
            if mode == "served" else run_plain(streams, trace)
        results[f"capacity_{mode}"] = res
        for s in streams:
            s.close()
    results["served_vs_plain_depth_maps_per_s"] = (results["capacity_served"]["depth_maps_per_s"] /
                                                   results["capacity_plain"]["depth_maps_per_s"])
    # latency under Poisson arrivals at rate_frac of each mode's own capacity
    for mode in (() if args.capacity_only else ("served", "plain")):
        rate = args.rate_frac * results[f"capacity_{mode}"]["jobs_per_s"]
        streams = fresh()
        trace = poisson_trace(len(streams), args.jobs, rate, args.seed + 7)
        res = run_served(streams, trace, args.slots, budget, by_class=not args.mixed_batches,
                         heavy_chunks=args.heavy_chunks) \
            if mode == "served" else run_plain(streams, trace)
        res["rate_jobs_per_s"] = rate
        results[f"poisson_{mode}"] = res
        for s in streams:
            s.close()
    results["config"] = {"streams": len(streams), "jobs": args.jobs, "class_batches": not args.mixed_batches,
                         "heavy_chunks": args.heavy_chunks,
                         "launch_shapes": "autotuned per stream shape (tune.py)" if not args.no_tune else "defaults",
                         "gop": args.gop, "slots": args.slots, "budget_gb": args.budget_gb,
                         "rate_frac": args.rate_frac, "shapes": "960x540/3v/64L, 1920x1080/8v/250L, 3840x2160/15v/400L"}
    print(json.dumps(results), flush=True)
    return results


if __name__ == "__main__":
    main()
