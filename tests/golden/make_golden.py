"""Writes the stored expected values of the oracle pins.  Calls only ``oracle/``.

Usage: python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import jtfs_oracle as O  # noqa: E402


def main():
    counts, bounds = {}, {}
    for w, cfg in O.WORKLOADS.items():
        p = O.Plan(cfg)
        s = O.Schedule(p, cfg.oversampling)
        counts[str(w)] = dict(p.shapes(), s1=[int(v) for v in s.s1], s2=[int(v) for v in s.s2],
                              lam_min=[int(v) for v in s.lam_min])
        lp1 = O.littlewood_paley(p, 1)
        om = O.grid_freqs(p.N)
        band = (om >= p.xi1.min()) & (om <= p.xi1.max())
        bounds[str(w)] = dict(c1=p.c1, c2=p.c2, c_fr=p.c_fr, A1=float(lp1[band].min()))
    with open(os.path.join(HERE, "counts.json"), "w") as f:
        json.dump(counts, f, indent=1)
    with open(os.path.join(HERE, "lp_bounds.json"), "w") as f:
        json.dump(bounds, f, indent=1)


if __name__ == "__main__":
    main()
