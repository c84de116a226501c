"""Command line: certified symplectic minimum distance of one code.

    python -m paper_2408_10743_gb300 --workload qc72 [--index 0] [--repeat 1]
    python -m paper_2408_10743_gb300 --matrix FILE [--field 2|4] [--n-stab S]
    python -m paper_2408_10743_gb300 --stabilizers FILE

FILE holds one generator row per line: 2n digits 0/1 (x | z) for field 2, or n
symbols 0-3 (a + 2b for a + alpha b) for field 4; blank lines and lines
starting with '#' are ignored.  With --stabilizers the rows generate the
stabilizer of a qubit code and the output is d(Q), the least weight of a
logical operator (the normalizer minus the stabilizer).
"""
import argparse
import json
import sys

import numpy as np

from . import binding
from . import synth


def read_matrix(path):
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([int(c) for c in line.replace(" ", "")])
    return np.array(rows, dtype=np.uint8)


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2408_10743_gb300")
    src = ap.add_mutually_exclusive_group(required=True)
    src.add_argument("--workload", choices=["qc72", "f2_24", "f4_40"])
    src.add_argument("--matrix")
    src.add_argument("--stabilizers", metavar="FILE",
                     help="stabilizer generators (x | z) of a qubit code: report d(Q)")
    src.add_argument("--random", nargs=2, type=int, metavar=("N", "K"),
                     help="random F2 code (i.i.d. bits, full rank), seeded by --index")
    src.add_argument("--batch", type=int, metavar="COUNT",
                     help="the first COUNT codes of the batched workload (n ~ U[16,56]), solved together")
    ap.add_argument("--index", type=int, default=0)
    ap.add_argument("--field", type=int, default=2, choices=[2, 4])
    ap.add_argument("--n-stab", type=int, default=0)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--time-limit", type=float, default=0.0)
    ap.add_argument("--isometry", action="store_true",
                    help="solve by the isometry method (Algorithm 3) instead of packages")
    args = ap.parse_args(argv)
    if args.batch:
        gens = synth.batch_codes(args.batch)
        codes = binding.Code.many(gens)
        with binding.Batch() as b:
            res = b.wait(b.submit(codes))
            st = b.stats()
        for c in codes:
            c.close()
        print(json.dumps({"codes": len(res), "ok": sum(r["status"] == 0 for r in res),
                          "codewords": int(sum(r["codewords"] for r in res)),
                          "gpu_seconds": st["gpu_seconds"], "launches": st["launches"],
                          "max_d": max(r["d"] for r in res)}))
        return 0
    field = args.field
    if args.workload == "qc72":
        g = synth.single_qc(args.index)
    elif args.workload == "f2_24":
        g = synth.single_f2(args.index)
    elif args.workload == "f4_40":
        g, field = synth.single_f4(args.index), 4
    elif args.stabilizers:
        with binding.Code.from_stabilizers(read_matrix(args.stabilizers)) as code:
            for _ in range(args.repeat):
                r = code.solve(time_limit_s=args.time_limit)
        out = {k: v for k, v in r.items() if k not in ("witness", "coeffs")}
        out["logical"] = "".join(str(int(v)) for v in r["witness"])
        print(json.dumps(out))
        return 0
    elif args.random:
        g = synth.random_f2_code(args.random[0], args.random[1],
                                 synth.Xoshiro256ss(synth.seed_for(5, args.index)))
    else:
        g = read_matrix(args.matrix)
    with binding.Code(g, field) as code:
        if args.n_stab:
            code.set_exclude(args.n_stab)
        for _ in range(args.repeat):
            r = code.solve_isometry() if args.isometry else code.solve(time_limit_s=args.time_limit)
    out = {k: v for k, v in r.items() if k not in ("witness", "coeffs")}
    out["witness"] = "".join(str(int(v)) for v in r["witness"])
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
