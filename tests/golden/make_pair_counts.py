"""Write tests/golden/pair_counts.json: the number of (target, sample) pairs
with d <= r (paper Eq. 1-2 support, Sect. 3.5) for the seeded benchmark
workloads, counted by the FP64 oracle's HEALPix-lookup gridder (oracle/ only).

Usage: python tests/golden/make_pair_counts.py [name ...]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402

OUT = os.path.join(HERE, "pair_counts.json")


def count(wl):
    k = oracle.gauss1d(wl.kernel["sigma"], wl.support) if wl.kernel["type"] == "gauss1d" else \
        oracle.gauss2d(wl.kernel["smaj"], wl.kernel["smin"], wl.kernel["pa"], wl.support)
    ns = oracle.nside_for_resolution(wl.hpx_maxres)
    ones = np.ones((wl.n_samples, 1))
    res = oracle.grid_lookup(ns, wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, ones, k)
    return int(res.npairs)


CASES = {
    "cube_scale1": lambda: workloads.cube(scale=1.0, n_channels=1),
    "cube_scale0.1": lambda: workloads.cube(scale=0.1, n_channels=1),
    "plain2d_scale1": lambda: workloads.plain2d(scale=1.0),
}

if __name__ == "__main__":
    names = sys.argv[1:] or list(CASES)
    table = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for nm in names:
        t0 = time.time()
        wl = CASES[nm]()
        table[nm] = {"pairs": count(wl), "n_samples": wl.n_samples, "n_targets": wl.n_targets,
                     "numpy": np.__version__}
        print(nm, table[nm], "%.1fs" % (time.time() - t0), flush=True)
        with open(OUT, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
