"""Benchmark: exact symplectic minimum distance on GB300.

Default workload: the quasi-cyclic n = 72, K = 72 code (x and z parts each a
6 x 6 array of 12 x 12 circulants of first-row weight 2..5), the single-code
measurement.  One step = one complete certified distance computation (all
rounds, all generator matrices, witness) through the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload qc72|f2_24|f4_40]

Multi-GPU: one process per GPU (torchrun); every rank solves the workload
code as an independent replica -- no collective on the data path ("scaling":
"weak").  Rank 0 prints one JSON line.

--impl reference times the CPU oracle (isometry + plain Brouwer-Zimmermann) on
the host cores, a bounded sample per step.
"""
import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "codewords/s"
PROFILE_JSON = os.path.join(ROOT, "profiles", "enum_kernel_qc72.json")


def workload(name, index):
    from paper_2408_10743_gb300 import synth
    if name == "qc72":
        return synth.single_qc(index), 2, {"workload": "qc72", "n": 72, "K": 72,
                                            "desc": "quasi-cyclic 6x6 blocks of 12x12 circulants"}
    if name == "f2_24":
        return synth.single_f2(index), 2, {"workload": "f2_24", "n": 24, "K": 24,
                                            "desc": "random F2 code"}
    if name == "f4_40":
        return synth.single_f4(index), 4, {"workload": "f4_40", "n": 40, "k": 20,
                                            "desc": "F4-linear [I_20|A]"}
    raise SystemExit("unknown workload " + name)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_digest():
    """Digest of the enumeration kernel's sources."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2408_10743_gb300", "csrc")
    for name in ("walk.cuh", "enum.cu", "dist_types.h"):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the enumeration kernel from the committed ncu
    summary, and a note saying why it applies or not: only while the kernel's
    sources are the ones the capture ran.  That the planner still hands the
    kernel the captured launch (tables, segments, parameters) is checked on
    the CPU by tests/test_hostwalk.py::test_launch_digest."""
    try:
        with open(PROFILE_JSON) as fh:
            p = json.load(fh)
    except (OSError, ValueError):
        return None, "no committed profile"
    if p.get("kernel_digest") != kernel_digest():
        return None, "kernel sources changed since the capture"
    return p.get("dram_bytes_per_launch"), "ncu capture in profiles/enum_kernel_qc72.json (kernel %s, launch %s)" % (
        p.get("kernel_digest"), p.get("launch_digest"))


def cpu_baseline(g, field, budget_s):
    import oracle
    r = oracle.bz(g, field=field, time_budget=budget_s, allow_incomplete=True)
    secs = max(r["seconds"], 1e-9)
    return {"value": r["codewords"] / secs, "unit": METRIC, "cores": r["threads"],
            "kind": "oracle",
            "sample": "isometry Brouwer-Zimmermann (Algorithm 3) on the same code, first %.0f s "
                      "of enumeration (%d codewords, rounds <= %d, %s)"
                      % (budget_s, r["codewords"], r["rounds"],
                         "complete" if r["complete"] else "stopped by the budget"),
            "complete": bool(r["complete"]), "seconds": r["seconds"],
            "time_to_d_s": r["seconds"] if r["complete"] else None,
            "one_core": one_core_rate(oracle, g, field, min(3.0, budget_s))}


def one_core_rate(oracle, g, field, budget_s):
    """The oracle on a single host thread, a bounded sample of the same code."""
    r = oracle.bz(g, field=field, threads=1, time_budget=budget_s, allow_incomplete=True)
    return {"value": r["codewords"] / max(r["seconds"], 1e-9), "unit": METRIC, "cores": 1,
            "sample": "first %.0f s of the same enumeration on one thread (%d codewords)" % (budget_s, r["codewords"])}


def hist10(ns):
    """Counts by decade of n, e.g. {"60-69": 12}."""
    out = {}
    for n in ns:
        k = "%d-%d" % (n // 10 * 10, n // 10 * 10 + 9)
        out[k] = out.get(k, 0) + 1
    return dict(sorted(out.items()))


def pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


def oracle_table(name):
    """The CPU oracle's stored distances of a many-code workload
    (tests/golden/<name>, written by tests/golden/make_oracle_tables.py):
    {index: (d or None, lower, upper)}; None if the table is absent."""
    path = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(path):
        return None
    out = {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            if p[3] == "-":
                out[int(p[0])] = (None, int(p[4]), int(p[5]))
            else:
                out[int(p[0])] = (int(p[3]), int(p[3]), int(p[3]))
    return out


def batch_measure(dist, count):
    """Workload 3: `count` random F2 codes (n ~ U[16,56], K ~ U[n/2,n]) solved
    (a) together by the batch engine (one multi-code launch unless a code
    needs more) and (b) one code per launch through dist_solve, on the same
    GPU, with the codes already initialised (tables resident).  Both arms
    receive every code at t = 0; a code's latency is measured at its own
    completion.  Every d is compared with the CPU oracle's stored value."""
    from paper_2408_10743_gb300 import synth
    gens = synth.batch_codes(count)
    t0 = time.perf_counter()
    codes = [dist.Code(g) for g in gens]
    t_init = time.perf_counter() - t0
    # the same codes initialised in one call (dist_init_many: planning on the
    # library's host threads, one device allocation)
    t0 = time.perf_counter()
    many = dist.Code.many(gens)
    t_init_many = time.perf_counter() - t0
    for c in many:
        c.close()
    with dist.Batch() as b:  # warm-up
        b.wait(b.submit(codes[:64]))
    # both arms read their results as raw dist_result records (no per-code
    # Python dictionaries inside the timed region)
    with dist.Batch() as b:
        t0 = time.perf_counter()
        res_b = b.wait_array(b.submit(codes))
        t_batch = time.perf_counter() - t0
        st = b.stats()
    for c in codes:  # warm the per-device solve caches
        dist.dist_solve(c._h)
    # one code per launch: a FIFO server with every code queued at t = 0
    res_p, lat_p = [], []
    t0 = time.perf_counter()
    for c in codes:
        res_p.append(dist.dist_solve(c._h))
        lat_p.append(time.perf_counter() - t0)
    t_plain = lat_p[-1] if lat_p else 0.0
    for c in codes:
        c.close()
    lat_b = [float(s) for s in res_b["seconds"]]
    table = oracle_table("batch4096_oracle.txt")
    checked = mism_b = mism_p = 0
    if table is not None:
        for i in range(count):
            if i in table and table[i][0] is not None:
                checked += 1
                mism_b += int(int(res_b["d"][i]) != table[i][0] or int(res_b["status"][i]) != 0)
                mism_p += int(res_p[i].d != table[i][0])
    return {"workload": "batch of %d random F2 codes, n ~ U[16,56], K ~ U[ceil(n/2), n]" % count,
            "codes": count,
            "oracle_checked": checked, "oracle_mismatches": mism_b,
            "oracle_mismatches_one_code_per_launch": mism_p,
            "oracle_source": "tests/golden/batch4096_oracle.txt (CPU oracle, Algorithm 3)",
            "batched": {"codes_per_s": count / t_batch, "wall_ms": 1e3 * t_batch,
                        "gpu_ms": 1e3 * st["gpu_seconds"], "launches": st["launches"],
                        "host_plan_ms": 1e3 * st["plan_seconds"], "host_post_ms": 1e3 * st["post_seconds"],
                        "codewords": int(res_b["codewords"].sum()),
                        "p50_ms": 1e3 * pct(lat_b, 50), "p99_ms": 1e3 * pct(lat_b, 99)},
            "one_code_per_launch": {"codes_per_s": count / t_plain, "wall_ms": 1e3 * t_plain,
                                    "gpu_ms": 1e3 * sum(r.gpu_seconds for r in res_p),
                                    "launches": int(sum(r.launches for r in res_p)),
                                    "codewords": int(sum(r.codewords for r in res_p)),
                                    "p50_ms": 1e3 * pct(lat_p, 50), "p99_ms": 1e3 * pct(lat_p, 99),
                                    "latency": "measured at each completion, all codes queued at t = 0"},
            "init_ms": 1e3 * t_init, "init_many_ms": 1e3 * t_init_many,
            "from_matrices": {"codes_per_s": count / (t_init_many + t_batch),
                              "wall_ms": 1e3 * (t_init_many + t_batch),
                              "note": "dist_init_many of the raw matrices, then the batched solve"}}


def small_k_measure(dist, stream, warmup, n=56, k=4, index=0, reps=3):
    """d(Q) of a random small-k stabilizer code (normalizer matrix, stabilizers
    excluded) with the planner's matrix-inclusion policy and with the first
    generator matrix only: rounds, codewords and time of each."""
    from paper_2408_10743_gb300 import synth
    N, n_stab = synth.small_k_code(index, n, k)
    info = dist.dist_plan_info_get(N, n_stab=n_stab)
    saved = dist.dist_get_gamma_limit()
    out = {"workload": "normalizer of a random [[%d, %d]] stabilizer code (K x N = %d x %d, K/N = %.3f), "
                       "stabilizers excluded" % (n, k, N.shape[0], N.shape[1], N.shape[0] / N.shape[1]),
           "free_rows": [int(info.f[j]) for j in range(info.n_gamma_built)]}
    try:
        for name, limit in (("policy", 0), ("first_matrix_only", 1)):
            dist.dist_set_gamma_limit(limit)
            with dist.Code(N) as c:
                c.set_exclude(n_stab)
                for _ in range(warmup):
                    c.solve(stream=stream)
                rs = [c.solve(stream=stream) for _ in range(reps)]
            best = min(rs, key=lambda r: r["gpu_seconds"])
            out[name] = {"matrices": best["n_gamma"], "d": best["d"], "rounds": best["rounds"],
                         "codewords": best["codewords"], "kernel_ms": 1e3 * best["gpu_seconds"],
                         "time_to_d_ms": 1e3 * min(r["seconds"] for r in rs),
                         "d_agrees": len({r["d"] for r in rs}) == 1}
    finally:
        dist.dist_set_gamma_limit(saved)
    a, b = out["policy"], out["first_matrix_only"]
    out["d_agrees"] = a["d"] == b["d"] and a["d_agrees"] and b["d_agrees"]
    out["codewords_saved"] = b["codewords"] - a["codewords"]
    out["time_ratio"] = b["time_to_d_ms"] / a["time_to_d_ms"] if a["time_to_d_ms"] else None
    return out


def _stream_code(i):
    from paper_2408_10743_gb300 import synth
    return synth.stream_request(i)


def stream_requests(rate, duration, workers=0):
    """The served stream's requests as (arrival_s, index, kind, generator),
    generated in a pool of spawned processes (the generator is pure Python)."""
    import multiprocessing as mp
    from paper_2408_10743_gb300 import synth
    times = synth.request_times(rate_hz=rate, duration_s=duration)
    workers = workers or min(16, os.cpu_count() or 1)
    if len(times) < 2000 or workers < 2:
        codes = [_stream_code(i) for i in range(len(times))]
    else:
        with mp.get_context("spawn").Pool(workers) as pool:
            codes = pool.map(_stream_code, range(len(times)), chunksize=64)
    return [(t, i, kind, g) for i, (t, (kind, g)) in enumerate(zip(times, codes))]


def serve_window(dist, requests, slice_ms, drain_s, time_limit_s):
    """Replays (arrival_s, index, kind, generator) requests against one batch
    engine in real time.  Each request is initialised and submitted at its
    arrival time; finished tickets are collected in completion order.  Returns
    per-request records (None = no answer by the end of the window plus
    drain)."""
    import threading
    batch = dist.Batch(slice_ms=slice_ms, time_limit_s=time_limit_s)
    recs = [None] * len(requests)
    by_ticket = {}
    lock = threading.Lock()
    t0 = time.perf_counter()
    codes = {}
    t_end = (requests[-1][0] if requests else 0.0) + drain_s

    def client():
        for i, (ta, _, kind, g) in enumerate(requests):
            now = time.perf_counter() - t0
            if now > t_end:
                return
            if ta > now:
                time.sleep(ta - now)
            code = dist.Code(g)
            with lock:
                t = batch.submit([code])
                by_ticket[t] = (i, time.perf_counter() - t0)
                codes[t] = code

    th = threading.Thread(target=client)
    th.start()
    answered = 0
    while answered < len(requests) and time.perf_counter() - t0 < t_end:
        t = batch.wait_any(timeout_s=0.05)
        if t is None:
            continue
        with lock:
            i, t_sub = by_ticket.pop(t)
            r = batch.poll(t)[0]
            codes.pop(t).close()  # collected: the batch no longer owns it
        ta = requests[i][0]
        recs[i] = {"d": r["d"], "lower": r["lower"], "status": r["status"],
                   "latency_s": (t_sub - ta) + r["seconds"], "codewords": r["codewords"],
                   "n": requests[i][3].shape[1] // 2, "kind": requests[i][2]}
        answered += 1
    th.join()
    wall = time.perf_counter() - t0
    st = batch.stats()
    batch.close()  # drops unanswered tickets; their codes are freed after it
    for c in codes.values():
        c.close()
    return recs, wall, st


def serve_one_per_launch(dist, requests, drain_s, time_limit_s):
    """The same requests served one code per launch: one server takes them in
    arrival order, waits for each arrival in real time, and answers each with
    dist_init + dist_solve_bounded (the same time limit) + dist_free before
    it takes the next.  Returns records as serve_window does."""
    recs = [None] * len(requests)
    t0 = time.perf_counter()
    t_end = (requests[-1][0] if requests else 0.0) + drain_s
    for i, (ta, _, kind, g) in enumerate(requests):
        now = time.perf_counter() - t0
        if now > t_end:
            break
        if ta > now:
            time.sleep(ta - now)
        with dist.Code(g) as c:
            r = c.solve(time_limit_s=time_limit_s)
        recs[i] = {"d": r["d"], "lower": r["lower"], "status": r["status"],
                   "latency_s": time.perf_counter() - t0 - ta, "codewords": r["codewords"],
                   "n": g.shape[1] // 2, "kind": kind}
    return recs, time.perf_counter() - t0


def serve_summary(requests, recs, wall, table):
    """Counts, latency percentiles and the oracle check of one served run."""
    from paper_2408_10743_gb300.binding import DIST_EINCOMPLETE
    cert = [r for r in recs if r is not None and r["status"] == 0]
    bounded = [r for r in recs if r is not None and r["status"] == DIST_EINCOMPLETE]
    answered = [r for r in recs if r is not None]
    lat_c = [r["latency_s"] for r in cert]
    lat_a = [r["latency_s"] for r in answered]
    # latency of every request, an unanswered one counted as waiting until the
    # run ended (a lower bound on its latency)
    lat_all = [r["latency_s"] if r is not None else wall - q[0] for q, r in zip(requests, recs)]
    checked = mismatched = consistent = inconsistent = 0
    unchecked = []
    for q, r in zip(requests, recs):
        if r is None or r["status"] != 0:
            continue
        ent = table.get(q[1]) if table is not None else None
        if ent is None:
            unchecked.append(r["n"])
        elif ent[0] is not None:
            checked += 1
            mismatched += int(ent[0] != r["d"])
        else:  # the oracle's bounds only
            unchecked.append(r["n"])
            ok = ent[1] <= r["d"] <= ent[2]
            consistent += int(ok)
            inconsistent += int(not ok)
    return {"requests": len(requests), "certified": len(cert), "bounded": len(bounded),
            "backlog": len(requests) - len(answered), "wall_s": wall,
            "certified_per_s": len(cert) / wall if wall > 0 else 0.0,
            "answers_per_s": len(answered) / wall if wall > 0 else 0.0,
            "p50_ms": 1e3 * pct(lat_c, 50) if lat_c else None,
            "p99_ms": 1e3 * pct(lat_c, 99) if lat_c else None,
            "answer_p50_ms": 1e3 * pct(lat_a, 50) if lat_a else None,
            "answer_p99_ms": 1e3 * pct(lat_a, 99) if lat_a else None,
            "all_p99_ms": 1e3 * pct(lat_all, 99) if lat_all else None,
            "certified_by_n": hist10(int(r["n"]) for r in cert),
            "bounded_by_n": hist10(int(r["n"]) for r in bounded),
            "bounds_valid": all(r["lower"] <= r["d"] for r in bounded),
            "codewords": int(sum(r["codewords"] for r in answered)),
            "oracle_checked": checked, "oracle_mismatches": mismatched,
            "unchecked_by_n": hist10(unchecked),
            "unchecked_within_oracle_bounds": consistent, "outside_oracle_bounds": inconsistent}


def serve_measure(dist, rate, duration, slice_ms, drain_s, time_limit_s, one_per_launch=True,
                  plain_drain_s=None):
    """Workload 4: Poisson requests (random F2 and quasi-cyclic codes,
    n ~ U[20,96]) at `rate` per second for `duration` seconds, each with a
    time limit (answers at the limit carry certified bounds lower <= d <= upper),
    through the continuous-batching engine and, on the same trace, one code
    per launch.  Certified answers are checked against the CPU oracle's
    stored values by request index."""
    t_gen = time.perf_counter()
    reqs = stream_requests(rate, duration)
    t_gen = time.perf_counter() - t_gen
    table = oracle_table("stream_oracle.txt")
    recs, wall, st = serve_window(dist, reqs, slice_ms, drain_s, time_limit_s)
    out = {"rate_hz": rate, "duration_s": duration, "time_limit_s": time_limit_s, "drain_s": drain_s,
           "generation_s": t_gen,
           "oracle_source": "tests/golden/stream_oracle.txt (CPU oracle, Algorithm 3; %s entries)" % (
               len(table) if table is not None else "no"),
           "served": serve_summary(reqs, recs, wall, table)}
    out["served"].update({"gpu_s": st["gpu_seconds"], "slices": st["slices"],
                          "host_plan_s": st["plan_seconds"], "host_post_s": st["post_seconds"]})
    if one_per_launch:
        prec, pwall = serve_one_per_launch(dist, reqs, drain_s if plain_drain_s is None else plain_drain_s,
                                           time_limit_s)
        out["one_code_per_launch"] = serve_summary(reqs, prec, pwall, table)
        a, b = out["served"], out["one_code_per_launch"]
        out["vs_one_per_launch"] = {
            "certified_per_s_ratio": a["certified_per_s"] / b["certified_per_s"] if b["certified_per_s"] else None,
            "all_p99_ratio": b["all_p99_ms"] / a["all_p99_ms"] if a["all_p99_ms"] else None}
    return out


def run_serve(args):
    import torch
    import paper_2408_10743_gb300 as dist
    torch.cuda.set_device(0)
    out = {"metric": "served codes/s and latency", "workload": "Poisson stream of distance queries",
           "config": {"workload": "served", "n": "U[20,96]", "K": "U[ceil(n/2), n]",
                      "kinds": "random F2 / quasi-cyclic 50:50", "slice_ms": args.slice_ms}}
    out["as_written"] = serve_measure(dist, args.rate, args.duration, args.slice_ms, args.drain,
                                      args.time_limit)
    sweep = []
    for rate in [float(x) for x in args.sweep.split(",") if x]:
        sweep.append(serve_measure(dist, rate, args.sweep_duration, args.slice_ms, args.drain,
                                   args.time_limit, one_per_launch=False))
    out["sweep"] = [dict(rate_hz=r["rate_hz"], **r["served"]) for r in sweep]
    # sustained: every request answered, answer p99 within the time limit plus one second
    ok = [r["rate_hz"] for r in sweep if r["served"]["backlog"] == 0 and r["served"]["oracle_mismatches"] == 0
          and r["served"]["answer_p99_ms"] is not None
          and r["served"]["answer_p99_ms"] <= 1e3 * (args.time_limit + 1.0)]
    out["highest_sustained_rate_hz"] = max(ok) if ok else None
    out["first_unsustained_rate_hz"] = min([r["rate_hz"] for r in sweep if r["rate_hz"] not in ok], default=None)
    print(json.dumps(out), flush=True)


def reduce_over_ranks(pg, seconds, codewords, device):
    """Whole-job figures of independent replicas: the slowest rank's time and
    the codewords of all ranks."""
    import torch
    t = torch.tensor([float(seconds)], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    c = torch.tensor([float(codewords)], device=device, dtype=torch.float64)
    pg.all_reduce(c, op=pg.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    g, field, cfg = workload(args.workload, 0)
    # each timed step may run long enough for the oracle to certify the
    # workload's d (about 8 s for qc72 on 16 Grace cores), so that the arm
    # reports a time to certified d; warm-up steps are short samples
    per_step = args.ref_step_budget
    import oracle
    for _ in range(args.warmup):
        oracle.bz(g, field=field, time_budget=1.0, allow_incomplete=True)
    cw = 0
    secs = 0.0
    threads = 0
    complete = []
    t0 = time.time()
    for _ in range(args.steps):
        r = oracle.bz(g, field=field, time_budget=per_step, allow_incomplete=True)
        cw += r["codewords"]
        secs += r["seconds"]
        threads = r["threads"]
        if r["complete"]:
            complete.append(r["seconds"])
    wall = time.time() - t0
    value = cw / max(secs, 1e-9)
    cfg = dict(cfg)
    cfg["l2"] = "n/a (CPU)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wall / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": threads, "kind": "oracle",
                             "sample": "isometry Brouwer-Zimmermann, at most %.1f s of enumeration per "
                                       "step; %d of %d steps certified d" % (per_step, len(complete), args.steps),
                             "time_to_d_s": statistics.mean(complete) if complete else None},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    import paper_2408_10743_gb300 as dist

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        pg = tdist
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    # every rank solves the same workload code (an independent replica of
    # identical size), so the per-GPU work is fixed as N grows
    g, field, cfg = workload(args.workload, 0)
    K = g.shape[0]

    code = dist.Code(g, field)
    # chunk granularity picked by the library's autotuner, timed on this
    # workload's code on this GPU (before the timed region)
    tuning = (dist.dist_autotune_codes([code], budget_s=args.autotune) if args.autotune > 0
              else dist.dist_get_tuning())
    # roofline denominator: the integer-issue microbenchmark on this GPU
    with torch.cuda.stream(stream):
        peak = dist.dist_intpeak(iters=20000, stream=stream)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)  # > L2 (129 MB)

    def one_step(timed, c=code):
        with torch.cuda.stream(stream):
            flush.fill_(7)  # evict L2 between steps (outside the timed events)
        # the flush has finished before the step starts, so that its last
        # writes do not run beside the step's launch
        stream.synchronize()
        with torch.cuda.stream(stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            raw = dist.dist_solve(c._h, stream=stream)  # the C-ABI call; its dict after the step
            e1.record(stream)
        e1.synchronize()
        return dist.result_dict(raw, c.n, c.K, c.field), e0.elapsed_time(e1) * 1e-3

    for _ in range(args.warmup):
        one_step(False)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    step_s, cws, kern_s, launches, ds, rounds = [], [], [], [], [], []
    for _ in range(args.steps):
        res, s = one_step(True)
        step_s.append(s)
        cws.append(res["codewords"])
        kern_s.append(res["gpu_seconds"])
        launches.append(res["launches"])
        ds.append(res["d"])
        rounds.append(res["rounds"])
    torch.cuda.synchronize()
    # The kernel's duration for the roofline from CUDA events on the launch
    # stream: the same steps again with the library's per-launch events on.
    # A timed event pair adds about 11 us to each launch, so the throughput
    # steps above run without them (their gpu_seconds is the kernel's own
    # %globaltimer span, reported beside).
    dist.dist_set_event_timing(1)
    try:
        ev_s, ev_cw = [], []
        for _ in range(args.steps):
            res, _s = one_step(True)
            ev_s.append(res["gpu_seconds"])
            ev_cw.append(res["codewords"])
    finally:
        dist.dist_set_event_timing(0)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_s = sum(step_s)
    total_cw = sum(cws)
    if pg:
        total_s, all_cw = reduce_over_ranks(pg, total_s, total_cw, dev)
    else:
        all_cw = float(total_cw)
    value = all_cw / total_s

    # end to end through the C-ABI calls with host buffers: dist_init (host
    # generator -> planner; the tables travel with the first solve's upload) +
    # dist_solve (uploads, launches, result read-back) + dist_free, every step
    e2e_s, e2e_cw, e2e_init, e2e_solve = [], [], [], []
    d_dev = ds[0]
    g_host = np.ascontiguousarray(g, dtype=np.uint8)
    n_e2e, K_e2e = (g_host.shape[1] // 2 if field == dist.DIST_F2 else g_host.shape[1]), g_host.shape[0]
    for _ in range(max(3, args.steps // 2)):
        with torch.cuda.stream(stream):
            flush.fill_(7)  # evict L2 between steps (outside the timed region)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2 = dist.dist_init(g_host, n_e2e, K_e2e, field)
        t1 = time.perf_counter()
        r2 = dist.dist_solve(h2, stream=stream)
        t2 = time.perf_counter()
        dist.dist_free(h2)
        e2e_s.append(time.perf_counter() - t0)
        e2e_init.append(t1 - t0)
        e2e_solve.append(t2 - t1)
        e2e_cw.append(r2.codewords)
        if r2.d != d_dev:
            raise RuntimeError(f"end-to-end solve gave d = {r2.d}, the device-resident one {d_dev}")
    e2e_value = sum(e2e_cw) / sum(e2e_s)
    # the same certified distance by the isometry method (Algorithm 3) on the
    # GPU: the work per certified d of the two algorithms, outside the timed
    # region
    iso_cmp = None
    if args.isometry:
        code.solve_isometry()
        its = [code.solve_isometry() for _ in range(3)]
        best = min(its, key=lambda r: r["gpu_seconds"])
        iso_cmp = {"algorithm": "isometry (a, b, a+b) + binary Brouwer-Zimmermann, one launch per step",
                   "d": best["d"], "d_agrees": all(r["d"] == ds[0] for r in its),
                   "codewords": best["codewords"], "matrices": best["n_gamma"], "rounds": best["rounds"],
                   "launches": best["launches"], "kernel_ms": 1e3 * best["gpu_seconds"],
                   "time_to_d_ms": 1e3 * best["seconds"],
                   "codewords_per_s": best["codewords"] / max(best["gpu_seconds"], 1e-12),
                   "work_vs_packages": best["codewords"] / (total_cw / args.steps),
                   "time_vs_packages": best["seconds"] / statistics.mean(step_s)}
        # the split walk's bound takes one popcount per codeword: its ceiling
        # is the measured popcount rate
        iso_cmp["popc_ceiling_Gcodewords_per_s"] = peak.popc_per_s / 1e9
        iso_cmp["frac_of_popc_ceiling"] = (iso_cmp["codewords_per_s"] / peak.popc_per_s
                                           if peak.popc_per_s else None)
    # the same code planned on the identity qubit order only (no
    # information-set search): a longer enumeration of the same kernel, the
    # single-code roofline on a launch long enough to fill the GPU
    greedy = None
    if args.greedy_plan:
        trials = dist.dist_get_plan_search()
        tuning_in_force = dist.dist_get_tuning()
        dist.dist_set_plan_search(0)
        dist.dist_set_event_timing(1)  # its frac, like the roofline's, from CUDA events
        try:
            with dist.Code(g, field) as cg:
                # this plan's launches are cut by the chunk setting too: tune
                # it on its own code, as the headline code was
                g_tuning = (dist.dist_autotune_codes([cg], budget_s=args.autotune) if args.autotune > 0
                            else tuning_in_force)
                for _ in range(args.warmup):
                    one_step(False, cg)
                gr = [one_step(True, cg) for _ in range(max(3, args.steps // 2))]
        finally:
            dist.dist_set_plan_search(trials)
            dist.dist_set_tuning(**tuning_in_force)
            dist.dist_set_event_timing(0)
        g_cw = sum(r["codewords"] for r, _ in gr)
        g_ks = sum(r["gpu_seconds"] for r, _ in gr)
        g_rate = g_cw / g_ks if g_ks > 0 else 0.0
        greedy = {"plan": "identity qubit order, greedy information sets (search trials 0)",
                  "d": gr[0][0]["d"], "d_agrees": all(r["d"] == ds[0] for r, _ in gr),
                  "rounds": gr[0][0]["rounds"], "codewords_per_step": g_cw / len(gr),
                  "value": g_cw / sum(s for _, s in gr), "unit": METRIC,
                  "time_to_d_ms": 1e3 * statistics.mean(s for _, s in gr),
                  "kernel_ms_per_step": 1e3 * g_ks / len(gr),
                  "kernel_Gcodewords_per_s": g_rate / 1e9,
                  "frac": g_rate / peak.mix_per_s if peak.mix_per_s else None,
                  "tuning": {k: g_tuning[k] for k in ("chunks_per_warp", "lane_cap_log2", "lane_floor_log2")}}
    code.close()
    # the second generator matrix on a small-k normalizer matrix (n = 56,
    # k = 4, K/N = 0.536, stabilizers excluded): the inclusion policy's
    # choice against the first matrix alone
    small_k = small_k_measure(dist, stream, args.warmup) if args.small_k else None

    kernel_s = sum(ev_s)
    achieved = sum(ev_cw) / kernel_s if kernel_s > 0 else 0.0
    traffic, traffic_note = profiled_traffic()
    roof = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak.mix_per_s / 1e9,
            "unit": "Gcodewords/s", "frac": achieved / peak.mix_per_s if peak.mix_per_s else None,
            "traffic": traffic,
            "traffic_source": traffic_note,
            "kernel": "dist::enum_kernel",
            "peak_source": "dist_intpeak mix (2 LOP3 + POPC + min per codeword), measured in this run",
            "popc_peak_Gops": peak.popc_per_s / 1e9, "lop3_peak_Gops": peak.lop3_per_s / 1e9,
            "intpeak_sm_mhz": peak.sm_mhz,
            "kernel_ms_per_step": 1e3 * kernel_s / len(ev_s),
            "kernel_time_source": "CUDA events around each launch on its stream (a second pass of the same "
                                  "steps with dist_set_event_timing(1))",
            "kernel_ms_per_step_globaltimer": 1e3 * sum(kern_s) / len(kern_s)}
    # the ceiling derived from unit counts and clocks: one POPC per codeword,
    # 16 POPC lanes per clock per SM, every SM, the maximum SM clock
    max_mhz = clk.get("sm_max_mhz") or 2070.0
    derived = 16.0 * float(peak.sms) * float(max_mhz) * 1e6
    roof["derived_peak"] = derived / 1e9
    roof["frac_of_derived"] = achieved / derived if derived > 0 else None
    roof["derived_peak_source"] = "POPC 16/clk/SM x %d SMs x %.0f MHz (one POPC per codeword)" % (peak.sms, max_mhz)
    # the same rate against a ceiling of W POPCs per codeword (every word of
    # both planes weighed); the kernel's exact word-0 bound weighs only word 0
    # of most codewords, so this fraction can exceed 1
    w_words = (int(cfg.get("n", 0)) + 31) // 32 or 1
    roof["frac_full_weight_count"] = achieved * w_words / peak.popc_per_s if peak.popc_per_s else None
    roof["frac_full_weight_count_note"] = ("achieved / (measured POPC rate / W), W = %d words per plane: "
                                           "the ceiling if every codeword were weighed on all W words" % w_words)

    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": dict(cfg, l2="flushed between steps (256 MB write)",
                           tuning={k: tuning[k] for k in ("chunks_per_warp", "lane_cap_log2",
                                                          "lane_floor_log2")},
                           parallelism="replicas: the same code solved independently on every GPU" if world > 1 else "1 GPU"),
            "time_to_d_ms": 1e3 * statistics.mean(step_s), "d": ds[0], "rounds": rounds[0],
            "codewords_per_step": total_cw / args.steps,
            "roofline": roof, "clocks": clk,
            "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": int(g.nbytes),
                    "d2h_bytes_per_step": int(ctypes.sizeof(dist.DistResult)),
                    "ms_per_step": 1e3 * statistics.mean(e2e_s),
                    # the time to certified d as a caller sees it: host
                    # generator -> planning (S1-S3) -> upload -> solve -> result
                    "time_to_d_ms": 1e3 * statistics.mean(e2e_s),
                    # dist_init (planning S1-S3 on the host, table upload) and
                    # the solve call, each as the caller sees it
                    "init_ms": 1e3 * statistics.mean(e2e_init),
                    "solve_ms": 1e3 * statistics.mean(e2e_solve)},
            "gpu_launches": int(sum(launches))}
    if greedy:
        line["greedy_plan"] = greedy
    if small_k:
        line["second_matrix"] = small_k
    if iso_cmp:
        line["isometry"] = iso_cmp
    if args.batch_codes > 0:
        line["batch"] = batch_measure(dist, args.batch_codes)
    if args.serve_window > 0 and rank == 0:
        # the served workload (Poisson stream, continuous batching) at its
        # written rate for a shorter window, and the same trace one code per
        # launch; --workload serve runs the full-length version and sweeps
        line["serve"] = serve_measure(dist, args.serve_rate, args.serve_window, args.slice_ms, args.drain,
                                      args.time_limit, plain_drain_s=args.plain_drain)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, field, args.cpu_budget)
        # like for like: the oracle's time to certified d over the library's
        # (the two count different codewords: binary isometry vs packages)
        if line["cpu_baseline"]["time_to_d_s"]:
            line["time_to_d_vs_cpu"] = {
                "oracle_s": line["cpu_baseline"]["time_to_d_s"],
                "e2e_ms": line["e2e"]["time_to_d_ms"], "device_ms": line["time_to_d_ms"],
                "ratio_e2e": line["cpu_baseline"]["time_to_d_s"] / (1e-3 * line["e2e"]["time_to_d_ms"]),
                "ratio_device": line["cpu_baseline"]["time_to_d_s"] / (1e-3 * line["time_to_d_ms"])}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="qc72", choices=["qc72", "f2_24", "f4_40", "serve"])
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: requests per second")
    ap.add_argument("--duration", type=float, default=2.0, help="serve: arrival window (s)")
    ap.add_argument("--drain", type=float, default=5.0, help="serve: time allowed after the window")
    ap.add_argument("--slice-ms", type=float, default=2.0, help="serve: launch time budget")
    ap.add_argument("--sweep", default="", help="serve: comma-separated rates to sweep")
    ap.add_argument("--sweep-duration", type=float, default=3.0)
    ap.add_argument("--time-limit", type=float, default=2.0,
                    help="serve: per-request time limit (s); answers at the limit carry bounds")
    ap.add_argument("--plain-drain", type=float, default=5.0,
                    help="serve: time the one-code-per-launch replay may run past the last arrival")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-step-budget", type=float, default=12.0,
                    help="reference arm: seconds of oracle enumeration allowed per timed step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", type=float, default=8.0,
                    help="seconds for the chunk-size autotuner before timing (0 = defaults)")
    ap.add_argument("--serve-window", type=float, default=10.0,
                    help="default run: seconds of served stream to report (0 = skip)")
    ap.add_argument("--serve-rate", type=float, default=2000.0,
                    help="default run: requests per second of that stream")
    ap.add_argument("--isometry", type=int, default=1,
                    help="also time the isometry method on the same code (0 = skip)")
    ap.add_argument("--greedy-plan", type=int, default=1,
                    help="also time the same code planned without the information-set search (0 = skip)")
    ap.add_argument("--small-k", type=int, default=1,
                    help="also compare the second generator matrix on a small-k normalizer (0 = skip)")
    ap.add_argument("--batch-codes", type=int, default=4096,
                    help="size of the batched-vs-one-per-launch comparison (0 = skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
