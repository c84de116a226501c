"""Writes the oracle's distances for the two many-code workloads, so that
tests and bench.py can check every GPU answer against them without running
the oracle on the spot.  Calls only the CPU oracle (oracle/) and the seeded
input generators -- never the GPU library.

* ``batch4096_oracle.txt``: the 4096 random F2 codes of
  ``synth.batch_codes(4096)`` (n ~ U[16,56], K ~ U[ceil(n/2), n]).  Every
  code is certified (the budget is large enough for all of them).
* ``stream_oracle.txt``: the first ``--stream-count`` requests of
  ``synth.request_stream`` (random F2 and quasi-cyclic codes, n ~ U[20,96]).
  A request's code depends only on its index, not on the arrival rate.  Each
  request gets the oracle for ``--stream-budget`` seconds (``--stream-budget2``
  more for n < ``--retry-below``); one the oracle cannot certify in that time
  is written as unchecked, with the oracle's bounds lower <= d <= upper.

Line format: ``index n K d`` for a certified d; ``index n K - lower upper``
for an unchecked one.  Header lines ``# generators sha256 <hex>`` and
``# first 1000 generators sha256 <hex>`` digest the generator matrices in
index order (all, and the first 1000), so that a reader can tell whether the
input generators still produce the same codes.

    python tests/golden/make_oracle_tables.py [--workers 8] [--only batch|stream]

Each code runs single-threaded; codes run in parallel in a process pool
(largest first).  Progress is kept in ``*.partial`` files next to the
outputs, so an interrupted run resumes where it stopped.
"""
import argparse
import hashlib
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def _batch_gen(i):
    from paper_2408_10743_gb300 import synth
    return synth.batch_code(i)


def _stream_gen(i):
    from paper_2408_10743_gb300 import synth
    return synth.stream_request(i)[1]


def _solve(job):
    kind, i, budget = job
    import oracle
    g = _batch_gen(i) if kind == "batch" else _stream_gen(i)
    r = oracle.bz(g, threads=1, time_budget=budget, allow_incomplete=True)
    return i, g.shape[1] // 2, g.shape[0], bool(r["complete"]), int(r["d"]), int(r["lower"]), r["seconds"]


def _digest(gens):
    h = hashlib.sha256()
    for g in gens:
        h.update(bytes([g.shape[0] & 255, g.shape[1] & 255]))
        h.update(g.tobytes())
    return h.hexdigest()


def _load_partial(path):
    done = {}
    if os.path.exists(path):
        for line in open(path):
            p = line.split()
            if len(p) >= 4 and not line.startswith("#"):
                done[int(p[0])] = p
    return done


def _run(kind, indices, budget, workers, partial, retry=None):
    """Runs the oracle on `indices` not yet certified in `partial` (a retry
    pass re-runs unchecked ones that `retry(n)` selects); appends lines."""
    done = _load_partial(partial)
    todo = []
    for i in indices:
        p = done.get(i)
        if p is None:
            todo.append(i)
        elif p[3] == "-" and retry is not None and retry(int(p[1])):
            todo.append(i)
    if not todo:
        return
    # largest first, so that the long ones do not form the tail
    sizes = {}
    for i in todo:
        g = _batch_gen(i) if kind == "batch" else _stream_gen(i)
        sizes[i] = g.shape[1] * g.shape[0]
    todo.sort(key=lambda i: -sizes[i])
    t0 = time.time()
    with mp.get_context("spawn").Pool(workers) as pool, open(partial, "a") as fh:
        for k, (i, n, K, ok, d, lo, secs) in enumerate(
                pool.imap_unordered(_solve, [(kind, i, budget) for i in todo], chunksize=1)):
            if ok:
                fh.write("%d %d %d %d\n" % (i, n, K, d))
            else:
                fh.write("%d %d %d - %d %d\n" % (i, n, K, lo, d))
            fh.flush()
            if (k + 1) % 200 == 0:
                print("%s: %d / %d in %.0f s" % (kind, k + 1, len(todo), time.time() - t0), flush=True)


def _finish(kind, indices, partial, out, header):
    done = _load_partial(partial)
    gens = [_batch_gen(i) if kind == "batch" else _stream_gen(i) for i in indices]
    with open(out, "w") as fh:
        for line in header:
            fh.write("# " + line + "\n")
        fh.write("# generators sha256 %s\n" % _digest(gens))
        fh.write("# first 1000 generators sha256 %s\n" % _digest(gens[:1000]))
        checked = 0
        for i in indices:
            p = done[i]
            if p[3] == "-":
                fh.write("%d %s %s - %s %s\n" % (i, p[1], p[2], p[4], p[5]))
            else:
                checked += 1
                fh.write("%d %s %s %s\n" % (i, p[1], p[2], p[3]))
    print("%s: %d of %d certified -> %s" % (kind, checked, len(indices), out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=max(1, os.cpu_count() or 1))
    ap.add_argument("--only", choices=["batch", "stream"], default=None)
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--batch-budget", type=float, default=86400.0)
    ap.add_argument("--stream-count", type=int, default=24000)
    ap.add_argument("--stream-budget", type=float, default=1.0)
    ap.add_argument("--stream-budget2", type=float, default=10.0)
    ap.add_argument("--retry-below", type=int, default=60)
    args = ap.parse_args()
    if args.only in (None, "batch"):
        idx = list(range(args.batch_count))
        part = os.path.join(HERE, "batch4096_oracle.txt.partial")
        _run("batch", idx, args.batch_budget, args.workers, part)
        _finish("batch", idx, part, os.path.join(HERE, "batch4096_oracle.txt"), [
            "Oracle distances of synth.batch_codes(%d): random F2 codes, n ~ U[16,56]," % args.batch_count,
            "K ~ U[ceil(n/2), n], item i seeded by seed_for(3, i).  Algorithm 3 (isometry +",
            "plain Brouwer-Zimmermann) on the CPU, written by make_oracle_tables.py.",
            "Columns: index n K d."])
    if args.only in (None, "stream"):
        idx = list(range(args.stream_count))
        part = os.path.join(HERE, "stream_oracle.txt.partial")
        _run("stream", idx, args.stream_budget, args.workers, part)
        _run("stream", idx, args.stream_budget2, args.workers, part,
             retry=lambda n: n < args.retry_below)
        _finish("stream", idx, part, os.path.join(HERE, "stream_oracle.txt"), [
            "Oracle distances of the first %d requests of synth.request_stream (random F2 and" % args.stream_count,
            "quasi-cyclic codes 50:50, n ~ U[20,96], K ~ U[ceil(n/2), n]; request i seeded by",
            "seed_for(4, i), independent of the arrival rate).  Algorithm 3 on the CPU with",
            "%.0f s per request (%.0f s more for n < %d); written by make_oracle_tables.py." % (
                args.stream_budget, args.stream_budget2, args.retry_below),
            "Columns: index n K d, or index n K - lower upper where the oracle did not",
            "certify d within its budget (its bounds: lower <= d <= upper)."])


if __name__ == "__main__":
    main()
