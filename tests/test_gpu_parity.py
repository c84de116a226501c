"""GPU path vs the CPU oracle, through the C ABI.  Distances must be identical
(exact integers); witnesses must be codewords of weight d whose returned
coefficients rebuild them from the input rows."""
import os

import numpy as np
import pytest

import oracle
import paper_2408_10743_gb300 as dist
from paper_2408_10743_gb300 import synth
from codes import (GL2, f2_matmul, f2_rank, f4_linear_f2_view, f4_rows_to_f2, five_qubit,
                   hamming_743_xonly, load_fixture, local_clifford, permute_qubits,
                   py_bruteforce, random_invertible, steane, sym_weight_bits,
                   tiny_random_code, toric)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stream():
    import torch
    torch.cuda.set_device(0)
    return torch.cuda.Stream(device=0)


def gpu(g, field=2, n_stab=0, stream=None):
    with dist.Code(g, field) as c:
        if n_stab:
            c.set_exclude(n_stab)
        return c.solve(stream=stream)


def check_witness(g, res, field=2):
    n = g.shape[1] // 2 if field == 2 else g.shape[1]
    w, co = res["witness"], res["coeffs"]
    if field == 2:
        assert sym_weight_bits(w, n) == res["d"]
        assert np.array_equal(np.bitwise_xor.reduce(g[co.astype(bool)], axis=0), w)
    else:
        assert int(np.count_nonzero(w)) == res["d"]
        from codes import f4_mul
        acc = np.zeros(n, dtype=np.uint8)
        for i, lam in enumerate(co):
            if lam:
                acc ^= np.array([f4_mul(int(lam), int(s)) for s in g[i]], dtype=np.uint8)
        assert np.array_equal(acc, w)


def test_worked_examples(stream):
    fx = load_fixture("example1_alg1.txt")
    assert gpu(fx["matrices"]["A"], stream=stream)["d"] == fx["d"]
    fx = load_fixture("example2_f4.txt")
    assert gpu(f4_rows_to_f2(fx["matrices"]["A4"]), stream=stream)["d"] == fx["d"]
    assert gpu(f4_rows_to_f2(fx["matrices"]["B4"]), stream=stream)["d"] == fx["d"]


def test_known_codes(stream):
    assert gpu(hamming_743_xonly(), stream=stream)["d"] == 3
    N, s = five_qubit()
    assert gpu(N, stream=stream)["d"] == 3 and gpu(N, n_stab=s, stream=stream)["d"] == 3
    N, s = steane()
    assert gpu(N, stream=stream)["d"] == 3 and gpu(N, n_stab=s, stream=stream)["d"] == 3
    for L in (2, 3, 4, 5, 6):
        N, s = toric(L)
        r = gpu(N, stream=stream)
        assert r["d"] == min(L, 4)
        check_witness(N, r)
        r = gpu(N, n_stab=s, stream=stream)
        assert r["d"] == L
        check_witness(N, r)


@pytest.mark.parametrize("kind", ["iid", "css", "yheavy", "sparse"])
def test_tiny_random_vs_oracle(kind, stream):
    rng = np.random.default_rng({"iid": 41, "css": 42, "yheavy": 43, "sparse": 44}[kind])
    for _ in range(120):
        n = int(rng.integers(1, 9))
        K = int(rng.integers(1, min(2 * n, 12) + 1))
        g = tiny_random_code(rng, n, K, kind)
        if not g.any():
            continue
        r = gpu(g, stream=stream)
        assert r["d"] == oracle.bz(g)["d"]
        check_witness(g, r)


def test_exclusion_random_vs_python(stream):
    rng = np.random.default_rng(45)
    for t in range(80):
        n = int(rng.integers(2, 7))
        K = int(rng.integers(2, min(2 * n, 10) + 1))
        g = tiny_random_code(rng, n, K, ["iid", "css", "yheavy"][t % 3])
        s = int(rng.integers(1, K))
        ref = py_bruteforce(g, n, n_stab=s)
        if ref is None:
            with pytest.raises(dist.DistError):
                gpu(g, n_stab=s, stream=stream)
        else:
            assert gpu(g, n_stab=s, stream=stream)["d"] == ref


def test_medium_random_vs_oracle(stream):
    """n in [16, 64]: one and two words per plane, fast path, several tiles of
    chunks and a ragged last chunk."""
    for t in range(40):
        rng = synth.Xoshiro256ss(7000 + t)
        n = 16 + rng.below(49)
        K = (n + 1) // 2 + rng.below(n - (n + 1) // 2 + 1)
        g = synth.random_f2_code(n, K, rng)
        r = gpu(g, stream=stream)
        assert r["d"] == oracle.bz(g)["d"], (n, K)
        check_witness(g, r)


def test_workload0_f2_24(stream):
    g = synth.single_f2(0)
    d, _, _ = oracle.bruteforce(g)
    r = gpu(g, stream=stream)
    assert r["d"] == d
    check_witness(g, r)
    for i in range(1, 6):
        g = synth.single_f2(i)
        assert gpu(g, stream=stream)["d"] == oracle.bruteforce(g)[0]


def test_workload1_f4_40(stream):
    for i in range(3):
        g4 = synth.single_f4(i)
        d = oracle.bz(g4, field=4)["d"]
        r = gpu(g4, field=4, stream=stream)
        assert r["d"] == d
        check_witness(g4, r, field=4)
        # additive F2 view of the same code gives the same distance
        assert gpu(f4_linear_f2_view(g4), stream=stream)["d"] == d


def test_workload2_qc72(stream):
    path = os.path.join(os.path.dirname(__file__), "golden", "qc72_seed0.txt")
    want = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            want[k] = float(v)
    g = synth.single_qc(0)
    r = gpu(g, stream=stream)
    assert r["d"] == int(want["d"])
    check_witness(g, r)
    # quasi-cyclic symmetry: shifting every 12-qubit block by one maps the code
    # to itself, so the shifted witness is another codeword of weight d
    n = 72
    w = r["witness"]
    perm = np.array([(q // 12) * 12 + (q % 12 + 1) % 12 for q in range(n)])
    ws = np.zeros_like(w)
    ws[perm] = w[:n]
    ws[n + perm] = w[n:]
    assert f2_rank(np.vstack([g, ws])) == 72
    assert sym_weight_bits(ws, n) == r["d"]


def test_invariants(stream):
    rng = np.random.default_rng(46)
    for t in range(6):
        g = synth.random_f2_code(30, 26, synth.Xoshiro256ss(9000 + t))
        n, K = 30, 26
        d = gpu(g, stream=stream)["d"]
        assert gpu(permute_qubits(g, n, rng.permutation(n)), stream=stream)["d"] == d
        assert gpu(local_clifford(g, n, rng.integers(0, len(GL2), size=n)), stream=stream)["d"] == d
        assert gpu(f2_matmul(random_invertible(K, rng), g), stream=stream)["d"] == d


def test_edge_cases(stream):
    # one qubit, one row
    assert gpu(np.array([[1, 1]], dtype=np.uint8), stream=stream)["d"] == 1
    # the whole space F2^{2n} at the size limits
    n = 128
    full = np.eye(2 * n, dtype=np.uint8)
    assert gpu(full, stream=stream)["d"] == 1
    # rank-deficient input
    rng = np.random.default_rng(47)
    g = synth.random_f2_code(20, 10, synth.Xoshiro256ss(11))
    gd = np.vstack([g, g[:3] ^ g[3:6], g[:2]])
    r = gpu(gd, stream=stream)
    assert r["k_eff"] == 10 and r["d"] == gpu(g, stream=stream)["d"]
    check_witness(gd, r)
    # zero code and S = C
    with pytest.raises(dist.DistError) as e:
        gpu(np.zeros((3, 8), dtype=np.uint8), stream=stream)
    assert e.value.code == dist.binding.DIST_EZERO
    N, s = toric(2)
    with pytest.raises(dist.DistError):
        gpu(N, n_stab=N.shape[0], stream=stream)
    # malformed input
    with pytest.raises(dist.DistError):
        gpu(np.array([[3, 0]], dtype=np.uint8), stream=stream)


def test_repeat_and_streams(stream):
    import torch
    g = synth.single_f2(3)
    with dist.Code(g) as c:
        a = c.solve(stream=stream)
        b = c.solve()                       # library stream
        s2 = torch.cuda.Stream()
        cc = c.solve(stream=s2)
    assert a["d"] == b["d"] == cc["d"]
    # how much speculative work runs before U drops is timing dependent
    assert min(a["codewords"], b["codewords"], cc["codewords"]) > 0


def test_bounded_solve(stream):
    """Time-limited solves: a certified answer (status 0) is the unbounded
    solve's d; an answer at the limit brackets it, lower <= d <= upper.  The
    codes' first launches span several steps, and the short limits end them
    part way, when the upper bound may already have fallen."""
    g = synth.random_f2_code(96, 60, synth.Xoshiro256ss(12))
    with dist.Code(g) as c:
        r = c.solve(stream=stream, time_limit_s=0.05)
    assert r["status"] in (0, dist.binding.DIST_EINCOMPLETE)
    assert 1 <= r["lower"] <= r["d"]
    check_witness(g, r)
    early = 0
    for t, (n, K) in enumerate(((64, 56), (72, 72), (60, 44))):
        g = synth.random_f2_code(n, K, synth.Xoshiro256ss(7700 + t))
        with dist.Code(g) as c:
            d_ref = c.solve(stream=stream)["d"]
            for limit in (1e-4, 1e-3, 2e-3, 4e-3, 8e-3, 2e-2):
                r = c.solve(stream=stream, time_limit_s=limit)
                assert r["status"] in (0, dist.binding.DIST_EINCOMPLETE), (n, K, limit)
                if r["status"] == 0:
                    assert r["d"] == d_ref, (n, K, limit, r["d"], d_ref)
                else:
                    early += 1
                    assert r["lower"] <= d_ref <= r["d"], (n, K, limit)
                check_witness(g, r)
    assert early > 0


def test_tuning_changes_speed_not_results(stream):
    g = synth.random_f2_code(56, 50, synth.Xoshiro256ss(4321))
    saved = dist.dist_get_tuning()
    try:
        ds = set()
        for cpw, cap, fl in ((1, 10, 1), (6, 14, 10), (48, 20, 16)):
            dist.dist_set_tuning(cpw, cap, fl)
            ds.add(gpu(g, stream=stream)["d"])
        assert len(ds) == 1
        best = dist.dist_autotune(budget_s=3.0)
        assert best["codewords_per_s"] > 0
        assert dist.dist_get_tuning()["chunks_per_warp"] == best["chunks_per_warp"]
        assert gpu(g, stream=stream)["d"] in ds
        with dist.Code(g) as c:
            best = dist.dist_autotune_codes([c], budget_s=2.0)
            assert best["codewords_per_s"] > 0
            assert dist.dist_get_tuning() == {k: best[k] for k in ("chunks_per_warp", "lane_cap_log2",
                                                                   "lane_floor_log2")}
            assert c.solve(stream=stream)["d"] in ds
    finally:
        dist.dist_set_tuning(saved["chunks_per_warp"], saved["lane_cap_log2"],
                             saved["lane_floor_log2"])


def test_wide_codes_four_words(stream):
    """n = 100..128 (four words per plane: the two-word filter and pivots
    beyond word 1) with few rows, against the oracle's brute force."""
    for t, (n, K) in enumerate(((100, 16), (128, 18), (97, 20), (128, 24))):
        g = synth.random_f2_code(n, K, synth.Xoshiro256ss(8100 + t))
        r = gpu(g, stream=stream)
        assert r["d"] == oracle.bruteforce(g)[0], (n, K)
        check_witness(g, r)


def test_event_timing_changes_timing_not_results(stream):
    """gpu_seconds from the kernel's own %globaltimer stamps (default) and
    from CUDA events around each launch (dist_set_event_timing(1)) describe
    the same launches: the same d, codewords and launches, both nonzero and
    close to each other."""
    g = synth.single_qc(0)
    assert dist.dist_get_event_timing() == 0
    with dist.Code(g, dist.DIST_F2) as c:
        for _ in range(3):
            c.solve(stream=stream)
        a = c.solve(stream=stream)
        dist.dist_set_event_timing(1)
        try:
            assert dist.dist_get_event_timing() == 1
            c.solve(stream=stream)
            b = c.solve(stream=stream)
        finally:
            dist.dist_set_event_timing(0)
    assert a["d"] == b["d"] == 12
    assert a["codewords"] == b["codewords"] and a["launches"] == b["launches"]
    assert a["gpu_seconds"] > 0 and b["gpu_seconds"] > 0
    assert abs(a["gpu_seconds"] - b["gpu_seconds"]) < 0.5 * max(a["gpu_seconds"], b["gpu_seconds"])
