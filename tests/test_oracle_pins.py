"""Pins of the CPU oracle against facts that do not come from the oracle itself:
the paper's worked examples, textbook codes, closed forms, the MacWilliams
identity, invariants, and an independent pure-Python brute force."""
import math

import numpy as np
import pytest

import oracle
from codes import (GL2, f2_matmul, f2_rank, f4_linear_f2_view, f4_mul, f4_rows_to_f2,
                   five_qubit, hamming_743_xonly, load_fixture, local_clifford,
                   permute_qubits, py_bruteforce, py_f4_bruteforce, random_invertible,
                   steane, sym_weight_bits, symplectic_dual, tiny_random_code, toric)


# --- Worked examples (Sections 2.2 and 2.3) ---------------------------------

def test_example1_algorithm1():
    fx = load_fixture("example1_alg1.txt")
    A = fx["matrices"]["A"]
    assert oracle.bruteforce(A)[0] == fx["d"] == 1
    assert oracle.bz(A)["d"] == 1
    # B~ spans the same code (its extra row is row 1 + row 3 ... of the same span)
    Bt = fx["matrices"]["Btilde"]
    assert f2_rank(np.vstack([A, Bt])) == f2_rank(A)
    assert oracle.bz(Bt)["d"] == 1
    # naive enumeration of A's rows alone would stop at 2: the minimum row weight
    assert min(sym_weight_bits(r, 2) for r in A) == fx["naive_bz"]


def test_example2_additive_f4():
    fx = load_fixture("example2_f4.txt")
    A4 = fx["matrices"]["A4"]
    A2 = f4_rows_to_f2(A4)
    assert oracle.bruteforce(A2)[0] == fx["d"] == 2
    assert oracle.bz(A2)["d"] == 2
    assert py_bruteforce(A2, 4) == 2
    # Enumerating A_4 alone: every row and every sum of two rows weighs >= 3, so
    # the bounds meet at 3 after two rows; the sum of all three rows weighs 2.
    import itertools
    w12 = [int(np.count_nonzero(np.bitwise_xor.reduce(A4[list(c)], axis=0)))
           for t in (1, 2) for c in itertools.combinations(range(3), t)]
    assert min(w12) == fx["naive_bz"] == 3
    assert int(np.count_nonzero(A4[0] ^ A4[1] ^ A4[2])) == 2


def test_example2_layout_b2_d2():
    """The paper's F4 -> F2 images B_2, D_2 fix the bit-plane layout:
    row a + alpha b -> (a | b)."""
    fx = load_fixture("example2_f4.txt")
    assert np.array_equal(f4_rows_to_f2(fx["matrices"]["B4"]), fx["matrices"]["B2"])
    assert np.array_equal(f4_rows_to_f2(fx["matrices"]["D4"]), fx["matrices"]["D2"])
    # B_4's extra row is row1 + row2 (alpha^2 = 1 + alpha): a dependent row
    B4 = fx["matrices"]["B4"]
    assert np.array_equal(B4[3], B4[0] ^ B4[1])
    r = oracle.bz(f4_rows_to_f2(B4))
    assert r["k_eff"] == 3 and r["d"] == 2
    assert oracle.bruteforce(f4_rows_to_f2(B4))[0] == 2


# --- Closed forms and textbook codes -----------------------------------------

def test_isometry_weight_identity():
    rng = np.random.default_rng(1)
    for n in (1, 5, 31, 64, 65, 128):
        for _ in range(20):
            row = rng.integers(0, 2, size=2 * n, dtype=np.uint8)
            assert oracle.iso_weight(row, n) == 2 * sym_weight_bits(row, n)


def test_full_space_and_single_rows():
    n = 6
    full = np.eye(2 * n, dtype=np.uint8)
    assert oracle.bz(full)["d"] == 1
    assert oracle.bruteforce(full)[0] == 1
    rng = np.random.default_rng(2)
    for _ in range(20):
        row = rng.integers(0, 2, size=(1, 2 * n), dtype=np.uint8)
        if not row.any():
            continue
        w = sym_weight_bits(row[0], n)
        assert oracle.bz(row)["d"] == w
        assert oracle.bruteforce(row)[0] == w
    # the "repetition" vector Y...Y alone
    y = np.ones((1, 2 * n), dtype=np.uint8)
    assert oracle.bz(y)["d"] == n


def test_hamming_743():
    g = hamming_743_xonly()
    assert oracle.bz(g)["d"] == 3
    assert oracle.bruteforce(g)[0] == 3


def test_five_qubit_code():
    N, s = five_qubit()
    assert N.shape == (6, 10) and s == 4
    assert oracle.bz(N)["d"] == 3
    assert oracle.bz(N, n_stab=s)["d"] == 3
    assert oracle.bruteforce(N)[0] == 3
    assert oracle.bruteforce(N, n_stab=s)[0] == 3


def test_steane_code():
    N, s = steane()
    assert N.shape == (8, 14) and s == 6
    assert oracle.bz(N)["d"] == 3
    assert oracle.bz(N, n_stab=s)["d"] == 3
    assert oracle.bruteforce(N, n_stab=s)[0] == 3


@pytest.mark.parametrize("L", [2, 3, 4, 5])
def test_toric_codes(L):
    N, s = toric(L)
    n = 2 * L * L
    assert N.shape == (n + 2, 2 * n) and s == n - 2
    assert oracle.bz(N)["d"] == min(L, 4)
    assert oracle.bz(N, n_stab=s)["d"] == L
    if n + 2 <= 22:
        assert oracle.bruteforce(N)[0] == min(L, 4)
        assert oracle.bruteforce(N, n_stab=s)[0] == L


def test_macwilliams_identity():
    """W_{C^perp_s}(x, y) = W_C(x + 3y, x - y) / |C| for F2-linear C in F2^{2n}
    with the symplectic weight: pins the brute force's weight function and its
    enumeration of every codeword exactly once."""
    rng = np.random.default_rng(3)
    for n, K in ((4, 3), (5, 4), (6, 5), (5, 7)):
        for _ in range(5):
            while True:
                g = rng.integers(0, 2, size=(K, 2 * n), dtype=np.uint8)
                if f2_rank(g) == K:
                    break
            dual = symplectic_dual(g, n)
            _, _, A = oracle.bruteforce(g, want_wdist=True)
            _, _, B = oracle.bruteforce(dual, want_wdist=True)
            A = [int(a) for a in A]
            B = [int(b) for b in B]
            assert sum(A) == 2 ** K and sum(B) == 2 ** (2 * n - K)
            # coefficient of y^w in sum_j A_j (1 + 3y)^(n-j) (1 - y)^j
            pred = [0] * (n + 1)
            for j, aj in enumerate(A):
                if not aj:
                    continue
                for s in range(j + 1):
                    for t in range(n - j + 1):
                        pred[s + t] += aj * math.comb(j, s) * (-1) ** s * math.comb(n - j, t) * 3 ** t
            assert [p // 2 ** K for p in pred] == B
            assert all(p % 2 ** K == 0 for p in pred)


# --- Brute force on tiny random codes (independent Python implementation) ----

@pytest.mark.parametrize("kind", ["iid", "css", "yheavy", "sparse"])
def test_tiny_random_codes_vs_python(kind):
    rng = np.random.default_rng({"iid": 101, "css": 102, "yheavy": 103, "sparse": 104}[kind])
    for trial in range(60):
        n = int(rng.integers(1, 7))
        K = int(rng.integers(1, min(2 * n, 9) + 1))
        g = tiny_random_code(rng, n, K, kind)
        if not g.any():
            continue
        ref = py_bruteforce(g, n)
        assert oracle.bruteforce(g)[0] == ref, (kind, trial)
        r = oracle.bz(g, ltrace_cap=64)
        assert r["d"] == ref, (kind, trial, g)
        # the lower bound never passes the true distance (Hamming units: 2d)
        assert all(L <= 2 * ref for L in r["ltrace"][:-1])
        # Singleton-type bound for additive codes and the row-weight bound
        k = f2_rank(g)
        assert ref <= n - (k + 1) // 2 + 1
        assert ref <= min(sym_weight_bits(row, n) for row in g if row.any())


def test_exclusion_vs_python():
    rng = np.random.default_rng(11)
    checked = 0
    for trial in range(150):
        n = int(rng.integers(2, 6))
        K = int(rng.integers(2, min(2 * n, 8) + 1))
        g = tiny_random_code(rng, n, K, ["iid", "css", "yheavy"][trial % 3])
        s = int(rng.integers(1, K))
        ref = py_bruteforce(g, n, n_stab=s)
        if ref is None:
            with pytest.raises(oracle.OracleError):
                oracle.bz(g, n_stab=s)
            continue
        assert oracle.bruteforce(g, n_stab=s)[0] == ref
        assert oracle.bz(g, n_stab=s)["d"] == ref
        checked += 1
    assert checked > 100


# --- F4-linear codes ----------------------------------------------------------

def test_f4_linear_tiny_vs_python():
    rng = np.random.default_rng(5)
    for _ in range(25):
        n = int(rng.integers(2, 7))
        k = int(rng.integers(1, min(n, 4) + 1))
        g4 = rng.integers(0, 4, size=(k, n), dtype=np.uint8)
        if not g4.any():
            continue
        ref = py_f4_bruteforce(g4)
        assert oracle.bz(g4, field=4)["d"] == ref
        assert oracle.bruteforce(g4, field=4)[0] == ref
        # the same code handed over as its F2 view (rows g and alpha g)
        assert oracle.bz(f4_linear_f2_view(g4))["d"] == ref


def test_f4_monomial_equivalence():
    """Scaling coordinates by nonzero F4 scalars and permuting them keeps d."""
    rng = np.random.default_rng(6)
    for _ in range(10):
        n, k = 8, 4
        g4 = rng.integers(0, 4, size=(k, n), dtype=np.uint8)
        d = oracle.bz(g4, field=4)["d"]
        scale = rng.integers(1, 4, size=n)
        h = np.array([[f4_mul(int(scale[j]), int(g4[i, j])) for j in range(n)] for i in range(k)],
                     dtype=np.uint8)[:, rng.permutation(n)]
        assert oracle.bz(h, field=4)["d"] == d


# --- Invariants on larger codes --------------------------------------------------

def test_invariants_permutation_clifford_rowops():
    rng = np.random.default_rng(7)
    for _ in range(6):
        n, K = 14, 12
        while True:
            g = rng.integers(0, 2, size=(K, 2 * n), dtype=np.uint8)
            if f2_rank(g) == K:
                break
        d = oracle.bz(g)["d"]
        assert oracle.bruteforce(g)[0] == d
        assert oracle.bz(permute_qubits(g, n, rng.permutation(n)))["d"] == d
        assert oracle.bz(local_clifford(g, n, rng.integers(0, len(GL2), size=n)))["d"] == d
        assert oracle.bz(f2_matmul(random_invertible(K, rng), g))["d"] == d


def test_witness_is_a_codeword_of_weight_d():
    rng = np.random.default_rng(8)
    for _ in range(20):
        n, K = 10, 9
        g = rng.integers(0, 2, size=(K, 2 * n), dtype=np.uint8)
        if f2_rank(g) == 0:
            continue
        r = oracle.bz(g)
        w = r["witness"]
        assert sym_weight_bits(w, n) == r["d"]
        assert f2_rank(np.vstack([g, w])) == f2_rank(g)


def test_bruteforce_witness_is_a_codeword_of_weight_d():
    """The brute force's witness (decoded from the Gray-code index of the
    lightest codeword it met) is nonzero, lies in the span, weighs d, and in
    exclusion mode lies outside the span of the excluded rows; for an F4
    input it lies in the F4 span (the F2 span of v and alpha v)."""
    from codes import f4_linear_f2_view
    rng = np.random.default_rng(18)
    for trial in range(40):
        n = int(rng.integers(3, 11))
        K = int(rng.integers(1, min(2 * n, 14) + 1))
        g = tiny_random_code(rng, n, K, ["iid", "css", "yheavy", "sparse"][trial % 4])
        if f2_rank(g) == 0:
            continue
        d, w, _ = oracle.bruteforce(g)
        assert w.any() and sym_weight_bits(w, n) == d
        assert f2_rank(np.vstack([g, w])) == f2_rank(g)
        s = int(rng.integers(0, K))
        if s and f2_rank(g[:s]) < f2_rank(g):
            d2, w2, _ = oracle.bruteforce(g, n_stab=s)
            assert sym_weight_bits(w2, n) == d2 >= d
            assert f2_rank(np.vstack([g, w2])) == f2_rank(g)
            assert f2_rank(np.vstack([g[:s], w2])) == f2_rank(g[:s]) + 1
    for _ in range(10):
        n, k = int(rng.integers(3, 9)), int(rng.integers(1, 4))
        g4 = rng.integers(0, 4, size=(k, n), dtype=np.uint8)
        if not g4.any():
            continue
        d, w, _ = oracle.bruteforce(g4, field=4)
        view = f4_linear_f2_view(g4)
        assert sym_weight_bits(w, n) == d
        assert f2_rank(np.vstack([view, w])) == f2_rank(view)


def test_time_budget_returns_bounds():
    rng = np.random.default_rng(9)
    n, K = 60, 60
    g = rng.integers(0, 2, size=(K, 2 * n), dtype=np.uint8)
    r = oracle.bz(g, time_budget=0.2, allow_incomplete=True)
    assert r["status"] in (oracle.OK, oracle.EINCOMPLETE)
    assert r["lower"] <= r["d"]


def test_rejects_bad_input():
    with pytest.raises(oracle.OracleError):
        oracle.bz(np.array([[2, 0]], dtype=np.uint8))
    with pytest.raises(oracle.OracleError):
        oracle.bz(np.zeros((2, 4), dtype=np.uint8))
