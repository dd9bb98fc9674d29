"""Measures how far the SCHEDULED transform (critical subsampling with oversampling o) lies
from the EXACT one (every convolution at the full sampling rate, the definitions of Sec. 2,
Eq. 3): per-order relative L2 error over a few seeded signals of a workload.  Calls only this
package (test infrastructure, FP64).

Usage: python -m oracle.measure_schedule [workload] [signals] [o ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import synth_signals as SS  # noqa: E402
from oracle import jtfs_oracle as O  # noqa: E402


def measure(workload: int, n_signals: int, oversamplings):
    base = O.WORKLOADS[workload]
    x = SS.workload_signals(workload, n_signals, base.N).astype(np.float64)
    exact_plan = O.Plan(base)
    exact = O.Schedule(exact_plan, None)
    t0 = time.perf_counter()
    refs = [O.forward_one(x[b], exact_plan, exact) for b in range(n_signals)]
    t_exact = (time.perf_counter() - t0) / n_signals
    rows = {}
    for o in oversamplings:
        cfg = O.Config(**{**base.__dict__, "oversampling": o})
        p = O.Plan(cfg)
        s = O.Schedule(p, o)
        err = {"S0": 0.0, "S1": 0.0, "S2": 0.0}
        t0 = time.perf_counter()
        for b in range(n_signals):
            got = O.forward_one(x[b], p, s)
            for k in err:
                err[k] = max(err[k], O.relative_l2(got[k], refs[b][k]))
        sum_kl = int(sum((p.n1 - s.lam_min[a]) * s.L2[a] for a in range(p.n2) if not s.skip2[a]))
        rows[o] = dict(err, seconds_per_signal=(time.perf_counter() - t0) / n_signals,
                       u1_len=int(s.L1.sum()), sum_K_L=sum_kl, L1_max=int(s.L1.max()),
                       L2_max=int(max(s.L2[~s.skip2])))
    return {"workload": workload, "signals": n_signals, "exact_seconds_per_signal": t_exact,
            "oversampling": rows}


if __name__ == "__main__":
    w = int(sys.argv[1]) if len(sys.argv) > 1 else 2
    n = int(sys.argv[2]) if len(sys.argv) > 2 else 2
    os_ = [int(v) for v in sys.argv[3:]] or [0, 1, 2]
    print(json.dumps(measure(w, n, os_), indent=1))
