"""Launch-shape autotuning of the cost kernel, cached per job class in a JSON file.

A job class is what the kernel's speed depends on: the device, the view and reference sizes, the
neighbour counts, the label count, the sample format, the combination and the precision. For a class
seen before the cached (label block, CTAs per SM) is applied; otherwise ftv_autotune times the candidates
on the job's own inputs, keeps the fastest on the context and the result is written to the cache. The
volume is identical for every shape, so tuning changes speed only.
"""
from __future__ import annotations

import json
import os
import tempfile

from . import ftv

CACHE_ENV = "FTV_TUNE_CACHE"


def default_cache_path() -> str:
    """$FTV_TUNE_CACHE, else .tune_cache/tuned_shapes.json beside the package (a machine-local file)."""
    here = os.path.dirname(os.path.abspath(__file__))
    return os.environ.get(CACHE_ENV) or os.path.join(os.path.dirname(here), ".tune_cache", "tuned_shapes.json")


def job_class(cams, ref_views, nbr_counts, n_labels: int, sample_bytes: int, bit_depth: int, combine: int,
              precision: int, device: str) -> str:
    """Cache key of a job class (a canonical JSON string)."""
    key = {
        "device": device,
        "views": [[int(c.width), int(c.height)] for c in cams],
        "refs": [int(r) for r in ref_views],
        "nbrs": [int(n) for n in nbr_counts],
        "labels": int(n_labels),
        "sample_bytes": int(sample_bytes),
        "bit_depth": int(bit_depth),
        "combine": int(combine),
        "precision": int(precision),
    }
    return json.dumps(key, sort_keys=True, separators=(",", ":"))


def candidates(shape: dict) -> tuple[list[int], list[int]]:
    """Label blocks {max, max/2, 32, 16, 8} within the limit, and CTAs per SM {occ, occ-1, occ-2} >= 1."""
    m, occ = int(shape["max_label_block"]), int(shape["max_ctas_per_sm"])
    lbs = sorted({m, max(1, (m + 1) // 2), min(m, 32), min(m, 16), min(m, 8)}, reverse=True)
    cts = [c for c in (occ, occ - 1, occ - 2) if c >= 1]
    return lbs, cts


def load(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save(path: str, entries: dict) -> None:
    """Atomic write (a temporary file in the same directory, then a rename)."""
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".tune", suffix=".json")
    with os.fdopen(fd, "w") as f:
        json.dump(entries, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _fits(rec: dict, shape: dict) -> bool:
    return (1 <= int(rec.get("label_block", 0)) <= shape["max_label_block"]
            and 0 <= int(rec.get("ctas_per_sm", -1)) <= shape["max_ctas_per_sm"])


def apply_or_tune(ctx, key: str, planes, labels, n_segments, costs, cache_path: str | None = None,
                  tune: bool = True, reps: int = 3, write: bool = True) -> dict | None:
    """Apply the cached shape of job class `key` to ctx, or (tune=True) run the autotuner on these inputs,
    apply its choice and (write=True) store it. Returns the record used, with "source": "cache" or "tuned",
    or None when nothing was cached and tune is False."""
    path = cache_path or default_cache_path()
    entries = load(path)
    shape = ftv.ftv_get_launch_shape(ctx)
    rec = entries.get(key)
    if rec is not None and _fits(rec, shape):
        ftv.ftv_set_launch_shape(ctx, int(rec["label_block"]), int(rec["ctas_per_sm"]))
        return {**rec, "source": "cache"}
    if not tune:
        return None
    lbs, cts = candidates(shape)
    lb, ct, ms = ftv.ftv_autotune(ctx, planes, labels, n_segments, costs, lbs, cts, reps)
    rec = {"label_block": int(lb), "ctas_per_sm": int(ct), "ms": float(ms.min()),
           "grid_ms": {f"{a}x{b}": round(float(ms[i, j]), 4) for i, a in enumerate(lbs) for j, b in enumerate(cts)}}
    if write:
        entries = load(path)
        entries[key] = rec
        save(path, entries)
    return {**rec, "source": "tuned"}
