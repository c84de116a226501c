"""Writes the stored expected values under tests/golden/ for workloads too
large for a test to recompute.  Calls only the CPU oracle (oracle/) and the
seeded input generators -- never the GPU library.

    python tests/golden/make_golden.py [--threads N]
"""
import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2408_10743_gb300 import synth  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    t0 = time.time()
    g = synth.single_qc(0)
    r = oracle.bz(g, threads=args.threads)
    with open(os.path.join(HERE, "qc72_seed0.txt"), "w") as fh:
        fh.write("# Quasi-cyclic n = 72, K = 72 code: x and z parts are 6 x 6 arrays of 12 x 12\n")
        fh.write("# circulants (first-row weight uniform in {2..5}), seed seed_for(2, 0) of\n")
        fh.write("# paper_2408_10743_gb300.synth.single_qc.  Distance from the CPU oracle\n")
        fh.write("# (Algorithm 3, isometry + plain Brouwer-Zimmermann), written by make_golden.py.\n")
        fh.write("d %d\n" % r["d"])
        fh.write("k_eff %d\n" % r["k_eff"])
        fh.write("oracle_codewords %d\n" % r["codewords"])
        fh.write("oracle_seconds %.1f\n" % r["seconds"])
        fh.write("oracle_threads %d\n" % r["threads"])
    print("d =", r["d"], "in %.1f s" % (time.time() - t0))


if __name__ == "__main__":
    main()
