"""The checked build (FTV_CHECKED): every cost-kernel gather is tested against its view's texel count, and an
index outside would be reported as FTV_ERR_CHECKED instead of read. The kernel's unchecked paths (samples
proven in view for a whole tile, integer-shift columns, rectified rows) rely on exact arguments; this runs
them in the checked build on workloads that take every path (tiny, reduced 1080p, 4K arc, temporal and
serving shapes, FP32 and FP64 projection, the 4K arc at full size) and requires no such report and the
oracle's volumes. compute-sanitizer is not available on the GPU pool; this is its stand-in."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_finds_no_out_of_view_gather():
    sys.path.insert(0, os.path.join(ROOT, "paper_1909_02294_gb300"))
    import build
    lib = build.build(checked=True)
    env = dict(os.environ, FTV_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_runs.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "no out-of-view gather" in r.stdout
