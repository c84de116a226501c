"""Qubit stabilizer-code front end (Section 2): the normalizer matrix built by
the library (host only, no GPU) against textbook codes, an independent numpy
construction, and a brute force over all Pauli operators; d(Q) on the GPU
against the CPU oracle."""
import itertools

import numpy as np
import pytest

import oracle
import paper_2408_10743_gb300 as dist
from codes import f2_rank, five_qubit, normalizer, pauli, steane, sym_weight_bits, toric


def symp(u, v, n):
    return int((np.dot(u[:n], v[n:]) + np.dot(u[n:], v[:n])) % 2)


def random_stabilizers(rng, n, m):
    """m independent commuting generators, drawn greedily."""
    rows = []
    while len(rows) < m:
        v = rng.integers(0, 2, size=2 * n, dtype=np.uint8)
        if not v.any() or any(symp(v, r, n) for r in rows):
            continue
        if f2_rank(np.array(rows + [v])) == len(rows) + 1:
            rows.append(v)
    return np.array(rows, dtype=np.uint8)


def brute_dq(S, n):
    """d(Q) by its definition (Section 2): least symplectic weight over the
    Paulis that commute with S and are not in S (k > 0), or over S (k = 0)."""
    s = f2_rank(S)
    k = n - s
    best = None
    span = {tuple(np.bitwise_xor.reduce(S[list(c)], axis=0)) if c else tuple([0] * 2 * n)
            for t in range(len(S) + 1) for c in itertools.combinations(range(len(S)), t)}
    for bits in itertools.product((0, 1), repeat=2 * n):
        v = np.array(bits, dtype=np.uint8)
        if not v.any():
            continue
        if k > 0:
            if any(symp(v, r, n) for r in S) or tuple(v) in span:
                continue
        elif tuple(v) not in span:
            continue
        w = sym_weight_bits(v, n)
        best = w if best is None else min(best, w)
    return best


def check_structure(S, n, gen, n_stab):
    s = f2_rank(S)
    K = gen.shape[0]
    assert gen.shape[1] == 2 * n
    assert f2_rank(gen) == K
    if s < n:
        assert K == 2 * n - s and n_stab == s
        # the first n_stab rows span S; every row commutes with every generator
        assert f2_rank(np.vstack([S, gen[:n_stab]])) == s
        for r in gen:
            assert all(symp(r, q, n) == 0 for q in S)
    else:
        assert n_stab == 0 and K == s and f2_rank(np.vstack([S, gen])) == s


@pytest.mark.parametrize("name", ["five", "steane", "toric2", "toric3", "toric4"])
def test_known_codes(name):
    N, s = {"five": five_qubit, "steane": steane}.get(name, lambda: toric(int(name[-1])))()
    n = N.shape[1] // 2
    S = N[:s]
    gen, n_stab = dist.dist_normalizer(S)
    check_structure(S, n, gen, n_stab)
    want = {"five": 3, "steane": 3}.get(name, int(name[-1]) if name.startswith("toric") else None)
    assert oracle.bz(gen, n_stab=n_stab)["d"] == want
    # the same space as the independent numpy construction
    Nref, sref = normalizer(S, n)
    assert sref == n_stab and f2_rank(np.vstack([Nref, gen])) == gen.shape[0]


def test_random_codes_vs_pauli_bruteforce():
    rng = np.random.default_rng(61)
    for t in range(60):
        n = int(rng.integers(2, 6))
        m = int(rng.integers(1, n + 1))  # k = n - m, including k = 0
        S = random_stabilizers(rng, n, m)
        # redundant and reordered generators are fine
        S_in = np.vstack([S, S[:1] ^ S[-1:]])[rng.permutation(m + 1)]
        gen, n_stab = dist.dist_normalizer(S_in)
        check_structure(S, n, gen, n_stab)
        assert oracle.bz(gen, n_stab=n_stab)["d"] == brute_dq(S, n), (n, m)


def test_errors():
    with pytest.raises(dist.DistError) as e:
        dist.dist_normalizer(pauli(["XI", "ZI"]))  # anticommuting
    assert e.value.code == -1
    with pytest.raises(dist.DistError) as e:
        dist.dist_normalizer(np.zeros((2, 6), dtype=np.uint8))
    assert e.value.code == -6
    with pytest.raises(dist.DistError) as e:
        dist.dist_normalizer(np.array([[2, 0]], dtype=np.uint8))
    assert e.value.code == -1


@pytest.mark.gpu
def test_quantum_distance_gpu():
    for L in (3, 4, 5, 6):
        N, s = toric(L)
        r = dist.quantum_distance(N[:s])
        assert r["d"] == L
        w = r["witness"]
        n = N.shape[1] // 2
        assert sym_weight_bits(w, n) == L
        assert all(symp(w, q, n) == 0 for q in N[:s])     # a logical operator ...
        assert f2_rank(np.vstack([N[:s], w])) == f2_rank(N[:s]) + 1  # ... not in S
    rng = np.random.default_rng(62)
    for t in range(20):
        n = int(rng.integers(6, 14))
        S = random_stabilizers(rng, n, int(rng.integers(1, n + 1)))
        gen, n_stab = dist.dist_normalizer(S)
        assert dist.quantum_distance(S)["d"] == oracle.bz(gen, n_stab=n_stab)["d"]
