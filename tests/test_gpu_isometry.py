"""The isometry method (Algorithm 3) on the GPU against the CPU oracle (the
same algorithm written plainly, sharing no code) and against the package
method: identical distances, valid witnesses."""
import os

import numpy as np
import pytest

import oracle
import paper_2408_10743_gb300 as dist
from paper_2408_10743_gb300 import synth
from codes import f4_mul, sym_weight_bits, tiny_random_code, toric

pytestmark = pytest.mark.gpu


def iso(g, field=2, n_stab=0):
    with dist.Code(g, field) as c:
        if n_stab:
            c.set_exclude(n_stab)
        return c.solve_isometry()


def valid(g, r, field=2):
    n = g.shape[1] // 2 if field == 2 else g.shape[1]
    w, co = r["witness"], r["coeffs"]
    if field == 2:
        assert sym_weight_bits(w, n) == r["d"]
        assert np.array_equal(np.bitwise_xor.reduce(g[co.astype(bool)], axis=0), w)
    else:
        assert int(np.count_nonzero(w)) == r["d"]
        acc = np.zeros(n, dtype=np.uint8)
        for i, lam in enumerate(co):
            if lam:
                acc ^= np.array([f4_mul(int(lam), int(s)) for s in g[i]], dtype=np.uint8)
        assert np.array_equal(acc, w)


def test_tiny_random_vs_oracle():
    rng = np.random.default_rng(71)
    for t in range(200):
        n = int(rng.integers(1, 9))
        K = int(rng.integers(1, min(2 * n, 12) + 1))
        g = tiny_random_code(rng, n, K, ["iid", "css", "yheavy", "sparse"][t % 4])
        if not g.any():
            continue
        r = iso(g)
        assert r["d"] == oracle.bz(g)["d"]
        valid(g, r)


def test_medium_random_vs_oracle_and_packages():
    for t in range(20):
        rng = synth.Xoshiro256ss(7300 + t)
        n = 16 + rng.below(25)
        K = (n + 1) // 2 + rng.below(n - (n + 1) // 2 + 1)
        g = synth.random_f2_code(n, K, rng)
        r = iso(g)
        assert r["d"] == oracle.bz(g)["d"] == dist.distance(g)["d"], (n, K)
        valid(g, r)


def test_f4_and_exclusion():
    for i in range(2):
        g4 = synth.single_f4(i)
        r = iso(g4, field=4)
        assert r["d"] == oracle.bz(g4, field=4)["d"]
        valid(g4, r, field=4)
    for L in (3, 4, 5):
        N, s = toric(L)
        r = iso(N, n_stab=s)
        assert r["d"] == L
        valid(N, r)
        assert iso(N)["d"] == min(L, 4)


def test_qc72_and_work_comparison():
    """The n = 72 quasi-cyclic code: the stored oracle distance; the binary
    method evaluates about ten times the codewords of the package method."""
    path = os.path.join(os.path.dirname(__file__), "golden", "qc72_seed0.txt")
    want = {k: float(v) for k, v in (l.split() for l in open(path) if l.strip() and not l.startswith("#"))}
    g = synth.single_qc(0)
    with dist.Code(g) as c:
        ri = c.solve_isometry()
        rp = c.solve()
    assert ri["d"] == rp["d"] == int(want["d"])
    valid(g, ri)
    assert ri["codewords"] > 5 * rp["codewords"]


def test_batch_codes_vs_oracle_table():
    """The isometry method on 256 of the batch workload's random codes
    (n 16-56, so rounds up to 8 of matrices of up to 56 rows, through the
    split, pair and lane walks): every d equals the stored oracle value."""
    from codes import load_oracle_table
    _, table = load_oracle_table("batch4096_oracle.txt")
    gens = synth.batch_codes(256)
    for i, g in enumerate(gens):
        n, K, d, lo, hi = table[i]
        assert (n, K) == (g.shape[1] // 2, g.shape[0])
        r = iso(g)
        if d is not None:
            assert r["d"] == d, i
        else:
            assert lo <= r["d"] <= hi, i
        valid(g, r)


@pytest.mark.parametrize("mode", [1, 2])
def test_every_walk_vs_oracle(mode):
    """The split walk on every round r in [2, 8] (mode 1), and never (mode
    2): the same distances as the oracle and valid witnesses, on tiny codes
    (rounds up to the whole matrix, halves of one or two rows), medium
    codes, F4 inputs and exclusion."""
    dist.dist_set_iso_walk(mode)
    try:
        rng = np.random.default_rng(4100 + mode)
        for t in range(80):
            n = int(rng.integers(1, 9))
            K = int(rng.integers(1, min(2 * n, 12) + 1))
            g = tiny_random_code(rng, n, K, ["iid", "css", "yheavy", "sparse"][t % 4])
            if not g.any():
                continue
            r = iso(g)
            assert r["d"] == oracle.bz(g)["d"], (mode, t)
            valid(g, r)
        for t in range(8):
            rs = synth.Xoshiro256ss(8100 + t)
            n = 16 + rs.below(25)
            K = (n + 1) // 2 + rs.below(n - (n + 1) // 2 + 1)
            g = synth.random_f2_code(n, K, rs)
            r = iso(g)
            assert r["d"] == oracle.bz(g)["d"], (mode, n, K)
            valid(g, r)
        g4 = synth.single_f4(0)
        r = iso(g4, field=4)
        assert r["d"] == oracle.bz(g4, field=4)["d"]
        valid(g4, r, field=4)
        for L in (3, 4):
            N, s_ = toric(L)
            r = iso(N, n_stab=s_)
            assert r["d"] == L
            valid(N, r)
    finally:
        dist.dist_set_iso_walk(0)
    assert dist.dist_get_iso_walk() == 0


def test_iso_walk_setting():
    with pytest.raises(dist.DistError):
        dist.dist_set_iso_walk(3)
    assert dist.dist_get_iso_walk() == 0


def test_split_walk_on_240_rows():
    """An F4 [I_120 | A] code of length 128: its image has 240 rows, so the
    split walk's halves hold 120 rows each and its row indices run to 239;
    rounds 2-5 of two matrices, in the default walk and with the split walk
    on every round.  d as the oracle."""
    g4 = synth.f4_systematic(128, 120, synth.Xoshiro256ss(6))
    want = oracle.bz(g4, field=4)["d"]
    for mode in (0, 1):
        dist.dist_set_iso_walk(mode)
        try:
            r = iso(g4, field=4)
        finally:
            dist.dist_set_iso_walk(0)
        assert r["d"] == want, mode
        assert r["rounds"] >= 3
        valid(g4, r, field=4)
