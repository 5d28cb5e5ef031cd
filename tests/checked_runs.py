"""Runs the library's checked build (libftv_checked.so, loaded through FTV_LIBRARY) over workloads that take
every cost-kernel path, and exits non-zero if any launch reports FTV_ERR_CHECKED (a gather index outside its
view) or any volume differs from the oracle. Run as a separate process by tests/test_gpu_checked.py, because
a process loads one build of the library."""
from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import paper_1909_02294_gb300 as ftv  # noqa: E402
from synth.configs import make_workload  # noqa: E402
import oracle  # noqa: E402
import oracle_runs  # noqa: E402
from gpu_runs import Run, dev  # noqa: E402


def main() -> int:
    assert ftv.ftv.LIB_PATH.endswith("libftv_checked.so"), ftv.ftv.LIB_PATH
    failures = []
    for name, precision in (("tiny", 0), ("hd8", 0), ("uhd15", 0), ("temporal", 0), ("serving_small", 0),
                            ("tiny", 1), ("hd8", 1), ("uhd15", 1)):
        wl = make_workload(name, reduced=name not in ("tiny", "serving_small"))
        run = Run(wl, precision=precision)
        costs = run.volumes()
        st = run.check()
        if st != 0:
            failures.append(f"{name} precision {precision}: status {ftv.ftv_status_str(st)}")
        for i, r in enumerate(wl.ref_views):
            H = (oracle.homography_table_f64 if precision else oracle.homography_table)(
                wl.cams, r, wl.neighbours(r), wl.n_labels, wl.z_near, wl.z_far)
            want = oracle_runs.volume_all_cores(wl, r, table_=H)
            if not np.array_equal(costs[i].cpu().numpy(), want):
                failures.append(f"{name} precision {precision} ref {r}: volume differs from the oracle")
        run.close()
    # the 3840x2160 rig at full size (every path of the projective kernel at scale): status only
    wl = make_workload("uhd15")
    run = Run(wl)
    run.volumes()
    st = run.check()
    if st != 0:
        failures.append(f"uhd15 full size: status {ftv.ftv_status_str(st)}")
    run.close()
    print("\n".join(failures) if failures else "checked build: no out-of-view gather, volumes equal the oracle")
    return 1 if failures else 0


if __name__ == "__main__":
    sys.exit(main())
