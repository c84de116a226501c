"""Batched and served solving (multi-code launches with continuous admission)
against the CPU oracle and against the single-code path."""
import time

import numpy as np
import pytest

import oracle
import paper_2408_10743_gb300 as dist
from paper_2408_10743_gb300 import synth
from paper_2408_10743_gb300.binding import DIST_EBUSY
from codes import load_oracle_table, sym_weight_bits, tiny_random_code, toric

pytestmark = pytest.mark.gpu


def valid(g, r, field=2):
    n = g.shape[1] // 2 if field == 2 else g.shape[1]
    assert r["status"] == 0
    if field == 2:
        assert sym_weight_bits(r["witness"], n) == r["d"]
        assert np.array_equal(np.bitwise_xor.reduce(g[r["coeffs"].astype(bool)], axis=0),
                              r["witness"])
    else:
        assert int(np.count_nonzero(r["witness"])) == r["d"]


def mixed_codes(count, seed):
    """Random F2 codes of the batched workload's shape (n ~ U[16, 56],
    K ~ U[n/2, n]) mixed with tiny codes of several kinds."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        if i % 3 == 0:
            n = int(rng.integers(1, 9))
            K = int(rng.integers(1, min(2 * n, 12) + 1))
            g = tiny_random_code(rng, n, K, ["iid", "css", "yheavy", "sparse"][i % 4])
            if not g.any():
                g[0, 0] = 1
        else:
            r = synth.Xoshiro256ss(synth.seed_for(3, 10_000 + seed * 1000 + i))
            n = 16 + r.below(25)
            K = (n + 1) // 2 + r.below(n - (n + 1) // 2 + 1)
            g = synth.random_f2_code(n, K, r)
        out.append(g)
    return out


def test_batch_vs_oracle():
    gens = mixed_codes(150, 1)
    codes = [dist.Code(g) for g in gens]
    with dist.Batch() as b:
        t = b.submit(codes)
        res = b.wait(t, timeout_s=120)
        st = b.stats()
    assert st["codes_done"] == len(gens)
    for g, r in zip(gens, res):
        assert r["d"] == oracle.bz(g)["d"]
        valid(g, r)
    for c in codes:
        c.close()


def test_batch_alone_equals_mix():
    """Every code's distance is the same when solved alone (one code per
    launch) and inside a mixed batch; witnesses are valid in both."""
    gens = mixed_codes(60, 2) + [synth.single_qc(0), synth.single_f2(1)]
    alone = [dist.distance(g) for g in gens]
    codes = [dist.Code(g) for g in gens]
    with dist.Batch(slice_ms=0.3) as b:
        t = b.submit(codes)
        mix = b.wait(t, timeout_s=120)
    for g, a, m in zip(gens, alone, mix):
        assert a["d"] == m["d"]
        valid(g, m)
    for c in codes:
        c.close()


def test_batch_f4_and_exclusion():
    g4 = [synth.single_f4(i) for i in range(3)]
    N, s = toric(3)
    N4, s4 = toric(4)
    codes = [dist.Code(g, field=4) for g in g4]
    ce = dist.Code(N)
    ce.set_exclude(s)
    ce4 = dist.Code(N4)
    ce4.set_exclude(s4)
    with dist.Batch() as b:
        t = b.submit(codes + [ce, ce4])
        res = b.wait(t, timeout_s=60)
    for g, r in zip(g4, res[:3]):
        assert r["d"] == oracle.bz(g, field=4)["d"]
        valid(g, r, field=4)
    assert res[3]["d"] == 3 and res[4]["d"] == 4


def test_served_requests_overlap_a_long_one():
    """Continuous batching: a long request is running when small requests
    arrive; they are admitted at the next slice, finish long before it, and
    give the same results as alone."""
    big = synth.random_f2_code(72, 72, synth.Xoshiro256ss(424242))  # d = 15, ~2.4e11 codewords
    smalls = mixed_codes(30, 3)
    with dist.Batch(slice_ms=1.0) as b:
        cb = dist.Code(big)
        tb = b.submit([cb])
        time.sleep(0.01)
        scs = [dist.Code(g) for g in smalls]
        ts = [b.submit([c]) for c in scs]
        small_res = [b.wait(t, timeout_s=60)[0] for t in ts]
        polled = b.poll(tb)  # None while the long one is still running
        big_res = polled[0] if polled is not None else b.wait(tb, timeout_s=120)[0]
        st = b.stats()
    assert big_res["d"] == 15
    valid(big, big_res)
    assert st["slices"] > 1
    for g, r in zip(smalls, small_res):
        assert r["d"] == dist.distance(g)["d"]
        valid(g, r)
    # the small requests did not wait for the long one
    assert max(r["seconds"] for r in small_res) < big_res["seconds"]


def test_admission_limits_and_ownership():
    gens = mixed_codes(40, 4)
    codes = [dist.Code(g) for g in gens]
    with dist.Batch(max_active=4, slice_ms=0.2) as b:
        t = b.submit(codes)
        with pytest.raises(dist.DistError) as e:
            codes[0].solve()  # owned by the batch until collected
        assert e.value.code == DIST_EBUSY
        with pytest.raises(dist.DistError):
            b.submit([codes[1]])
        res = b.wait(t, timeout_s=60)
        st = b.stats()
    assert st["slices"] >= 10  # at most four codes per slice
    for g, r in zip(gens, res):
        assert r["d"] == oracle.bz(g)["d"]
    assert codes[0].solve()["d"] == res[0]["d"]  # released after collection
    for c in codes:
        c.close()


def test_batch_workload_vs_oracle_table():
    """All 4096 codes of the batched workload (n ~ U[16,56], K ~ U[n/2,n]) in
    one batch, and each one solved alone, against the CPU oracle's stored
    distances (tests/golden/batch4096_oracle.txt): d equal element by element,
    every witness valid."""
    _, table = load_oracle_table("batch4096_oracle.txt")
    gens = synth.batch_codes(4096)
    codes = [dist.Code(g) for g in gens]
    with dist.Batch() as b:
        res = b.wait(b.submit(codes), timeout_s=300)
    bad = [(i, r["d"], table[i][2]) for i, r in enumerate(res) if r["d"] != table[i][2]]
    assert not bad, bad[:10]
    for g, r in zip(gens, res):
        valid(g, r)
    alone = [dist.dist_solve(c._h) for c in codes]
    bad = [(i, r.d, table[i][2]) for i, r in enumerate(alone) if r.d != table[i][2]]
    assert not bad, bad[:10]
    for c in codes:
        c.close()


def test_time_limit_bounds_and_wait_any():
    """A request that would take hours ends at its time limit with certified
    bounds lower <= d <= upper and a witness of weight upper; the small
    requests next to it are answered exactly, and wait_any reports every
    finished ticket once, in completion order."""
    from paper_2408_10743_gb300.binding import DIST_EINCOMPLETE
    big = synth.random_f2_code(96, 72, synth.Xoshiro256ss(synth.seed_for(5, 3)))
    smalls = mixed_codes(12, 5)
    with dist.Batch(slice_ms=1.0, time_limit_s=0.5) as b:
        cb = dist.Code(big)
        tb = b.submit([cb])
        scs = [dist.Code(g) for g in smalls]
        ts = [b.submit([c]) for c in scs]
        got = {}
        while len(got) < 1 + len(ts):
            t = b.wait_any(timeout_s=30)
            assert t is not None and t not in got
            got[t] = b.poll(t)[0]
    rb = got[tb]
    assert rb["status"] == DIST_EINCOMPLETE
    assert 1 <= rb["lower"] <= rb["d"]
    assert sym_weight_bits(rb["witness"], 96) == rb["d"]
    assert rb["seconds"] < 5
    for g, t in zip(smalls, ts):
        assert got[t]["status"] == 0
        assert got[t]["d"] == dist.distance(g)["d"]


def test_ten_thousand_tiny_codes_in_one_batch():
    """10^4 tiny codes (n <= 8, K <= 12; i.i.d., CSS-like, Y-heavy, sparse)
    solved together, against the oracle's brute force."""
    rng = np.random.default_rng(39)
    kinds = ["iid", "css", "yheavy", "sparse"]
    gens = []
    while len(gens) < 10000:
        n = int(rng.integers(1, 9))
        K = int(rng.integers(1, min(2 * n, 12) + 1))
        g = tiny_random_code(rng, n, K, kinds[len(gens) % 4])
        if g.any():
            gens.append(g)
    codes = [dist.Code(g) for g in gens]
    with dist.Batch() as b:
        res = b.wait(b.submit(codes), timeout_s=600)
    for g, r in zip(gens, res):
        assert r["status"] == 0
        assert r["d"] == oracle.bruteforce(g, threads=1)[0]
    for c in codes:
        c.close()


def test_wait_array_matches_wait():
    """The structured-array read-back carries the same results as the
    per-code dictionaries."""
    gens = mixed_codes(40, 6)
    codes = [dist.Code(g) for g in gens]
    with dist.Batch() as b:
        a = b.wait_array(b.submit(codes), timeout_s=60)
    with dist.Batch() as b:
        ref = b.wait(b.submit(codes), timeout_s=60)
    assert len(a) == len(ref)
    for g, row, r in zip(gens, a, ref):
        assert int(row["d"]) == r["d"] and int(row["status"]) == 0
        n = g.shape[1] // 2
        w = row["witness"][:2 * n]
        assert sym_weight_bits(w, n) == r["d"]
        assert np.array_equal(np.bitwise_xor.reduce(g[row["coeffs"][:g.shape[0]].astype(bool)], axis=0), w)
    for c in codes:
        c.close()


def test_slice_larger_than_the_initial_arena():
    """3000 codes of 80 qubits and 80 rows, each with a weight-1 row (d = 1),
    submitted together: their first slice stages about 45 MB of tables (two
    matrices of about 40 units, 15 KB per code), more than the batch's
    initial 32 MB arena, so the arena grows and the slice graph is captured
    again; every d is 1 with a valid witness."""
    rng = synth.Xoshiro256ss(4242)
    gens = []
    for i in range(3000):
        g = synth.random_f2_code(80, 80, rng)
        g[0, :] = 0
        g[0, i % 80] = 1  # x on one qubit
        gens.append(g)
    codes = [dist.Code(g) for g in gens]
    with dist.Batch() as b:
        res = b.wait_array(b.submit(codes), timeout_s=600)
    for g, row in zip(gens, res):
        assert int(row["status"]) == 0 and int(row["d"]) == 1
        w = row["witness"][:160]
        assert sym_weight_bits(w, 80) == 1
        assert np.array_equal(np.bitwise_xor.reduce(g[row["coeffs"][:80].astype(bool)], axis=0), w)
    for c in codes:
        c.close()


def test_init_many_vs_oracle_table():
    """dist_init_many: 1024 codes of the batched workload initialised in one
    call (planning on the host threads, one device allocation), solved
    together and one by one, against the CPU oracle's stored distances; the
    codes are freed in an interleaved order, the allocation with the last.
    Entries that dist_init rejects get its error and no handle, and the
    call's other codes are still initialised."""
    _, table = load_oracle_table("batch4096_oracle.txt")
    gens = synth.batch_codes(1024)
    codes = dist.Code.many(gens)
    with dist.Batch() as b:
        res = b.wait(b.submit(codes), timeout_s=300)
    bad = [(i, r["d"], table[i][2]) for i, r in enumerate(res) if r["d"] != table[i][2]]
    assert not bad, bad[:10]
    for g, r in zip(gens, res):
        valid(g, r)
    for i in range(0, 1024, 2):  # every other code freed first
        codes[i].close()
    for i in range(1, 1024, 64):
        r = dist.dist_solve(codes[i]._h)
        assert r.d == table[i][2], i
    for i in range(1, 1024, 2):
        codes[i].close()
    zero = np.zeros((3, 20), dtype=np.uint8)          # the zero code
    wide = np.ones((2, 2 * 129), dtype=np.uint8)      # 129 qubits
    handles, status = dist.dist_init_many([gens[0], zero, gens[1], wide])
    assert status[0] == 0 and status[2] == 0
    assert status[1] == dist.binding.DIST_EZERO and status[3] < 0
    assert handles[1] is None and handles[3] is None
    for i in (0, 2):
        r = dist.dist_solve(handles[i])
        assert r.d == table[i // 2][2]
        dist.dist_free(handles[i])
    assert dist.dist_init_many([]) == ([], [])
