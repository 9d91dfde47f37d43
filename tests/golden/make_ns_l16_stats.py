"""Writes tests/golden/ns_L16_N1000_k500_s8.txt: whole nested-sampling runs of the FP64
oracle on the 16 x 16 broken-phase lattice (m2 = -4, lambda = 8, 1000 live points drawn
from N(0, I), 500 deleted per iteration, stop at 1e-3 of the evidence) with 8 slice
steps per new point, one line per seed 0..31: final log Z (live points included), its
error bar sqrt(H/N), the information H, the iterations and the abandoned slice steps.

Only the oracle runs here (the GPU's whole runs are compared with these values
statistically). The slice steps are cut from 3 D = 768 to 8 so that a run takes
minutes rather than hours on a CPU core; the runs are spread over worker processes.

Run from the repository root: python tests/golden/make_ns_l16_stats.py [--workers 6]
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
SETTINGS = dict(L=16, N=1000, m2=-4.0, lam=8.0, n_delete=500, slice_steps=8, stop_frac=1e-3)
SEEDS = range(32)
PATH = os.path.join(HERE, "ns_L16_N1000_k500_s8.txt")


def one(seed):
    sys.path.insert(0, ROOT)
    from oracle import ns as ons
    t0 = time.time()
    r = ons.NS(ons.NSConfig(seed=seed, **SETTINGS)).run()
    return seed, r["logz"], r["logz_err"], r["H"], r["n_iter"], r["capped"], time.time() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=6)
    a = ap.parse_args()
    with mp.get_context("spawn").Pool(a.workers) as pool:
        rows = sorted(pool.map(one, SEEDS, chunksize=1))
    with open(PATH, "w") as f:
        f.write("# FP64 oracle nested sampling, %s\n" % ", ".join("%s=%s" % kv for kv in SETTINGS.items()))
        f.write("# written by tests/golden/make_ns_l16_stats.py (oracle only)\n")
        f.write("# seed logz logz_err H iterations capped\n")
        for seed, lz, err, H, it, cap, _ in rows:
            f.write("%d %.10f %.6f %.6f %d %d\n" % (seed, lz, err, H, it, cap))
    print("wrote", PATH, "slowest run %.0f s" % max(r[-1] for r in rows))


if __name__ == "__main__":
    main()
