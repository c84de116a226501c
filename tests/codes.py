"""Test-side helpers: textbook codes, F4 arithmetic, fixture parsing and a
pure-Python brute force.  Written independently of both the oracle (C) and the
GPU library; only tests import this module."""
from __future__ import annotations

import itertools
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# ---------------------------------------------------------------------------
# F4 = {0, 1, a, b}, a = alpha, b = alpha^2 = alpha + 1; symbol v = x + 2z
# stands for x + alpha z (x = coefficient of 1, z = coefficient of alpha).
# ---------------------------------------------------------------------------
SYM = {"0": 0, "1": 1, "a": 2, "b": 3}


def f4_mul(u: int, v: int) -> int:
    u0, u1 = u & 1, u >> 1
    v0, v1 = v & 1, v >> 1
    # (u0 + u1 a)(v0 + v1 a) with a^2 = a + 1
    c0 = (u0 & v0) ^ (u1 & v1)
    c1 = (u0 & v1) ^ (u1 & v0) ^ (u1 & v1)
    return c0 | (c1 << 1)


def f4_rows_to_f2(rows: np.ndarray) -> np.ndarray:
    """Row a + alpha b of F4^n -> (a | b) of F2^{2n}."""
    rows = np.asarray(rows, dtype=np.uint8)
    return np.concatenate([rows & 1, (rows >> 1) & 1], axis=1).astype(np.uint8)


def f4_linear_f2_view(rows: np.ndarray) -> np.ndarray:
    """F2 generators of the F4-span: each row g and alpha*g."""
    rows = np.asarray(rows, dtype=np.uint8)
    ag = np.vectorize(lambda s: f4_mul(2, int(s)))(rows).astype(np.uint8)
    out = np.empty((2 * rows.shape[0], rows.shape[1]), dtype=np.uint8)
    out[0::2] = rows
    out[1::2] = ag
    return f4_rows_to_f2(out)


# ---------------------------------------------------------------------------
# Fixture files.
# ---------------------------------------------------------------------------
def load_fixture(name: str) -> dict:
    out: dict = {"matrices": {}}
    cur = None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            if key == "matrix":
                cur = rest.strip()
                out["matrices"][cur] = []
            elif key in ("field", "n", "d", "naive_bz"):
                out[key] = rest.strip() if key == "field" else int(rest)
                cur = None
            else:
                assert cur is not None, line
                out["matrices"][cur].append([SYM[t] for t in line.split()])
    for k, v in out["matrices"].items():
        out["matrices"][k] = np.array(v, dtype=np.uint8)
    return out


# ---------------------------------------------------------------------------
# Symplectic vectors as (x, z) Python ints.
# ---------------------------------------------------------------------------
def to_ints(gen: np.ndarray, n: int):
    rows = []
    for r in np.asarray(gen, dtype=np.uint8):
        x = sum(int(r[i]) << i for i in range(n))
        z = sum(int(r[n + i]) << i for i in range(n))
        rows.append((x, z))
    return rows


def sym_weight_bits(row: np.ndarray, n: int) -> int:
    row = np.asarray(row, dtype=np.uint8)
    return int(np.count_nonzero(row[:n] | row[n:2 * n]))


def py_bruteforce(gen: np.ndarray, n: int, n_stab: int = 0) -> int:
    """min wt_s over the nonzero codewords of span(rows) minus span(first n_stab rows).
    Plain enumeration of all 2^K coefficient vectors (dependent rows allowed)."""
    rows = to_ints(gen, n)
    K = len(rows)
    stab = set()
    for coeffs in itertools.product((0, 1), repeat=n_stab):
        x = z = 0
        for c, (rx, rz) in zip(coeffs, rows[:n_stab]):
            if c:
                x ^= rx
                z ^= rz
        stab.add((x, z))
    best = None
    for coeffs in itertools.product((0, 1), repeat=K):
        x = z = 0
        for c, (rx, rz) in zip(coeffs, rows):
            if c:
                x ^= rx
                z ^= rz
        if x == 0 and z == 0:
            continue
        if (x, z) in stab:
            continue
        w = (x | z).bit_count()
        if best is None or w < best:
            best = w
    return best


def py_f4_bruteforce(gen4: np.ndarray) -> int:
    """min Hamming weight over the nonzero F4-linear combinations of F4 rows."""
    g = np.asarray(gen4, dtype=np.uint8)
    k, n = g.shape
    best = None
    for lam in itertools.product(range(4), repeat=k):
        v = np.zeros(n, dtype=np.uint8)
        for l, row in zip(lam, g):
            if l:
                v ^= np.array([f4_mul(l, int(s)) for s in row], dtype=np.uint8)
        w = int(np.count_nonzero(v))
        if w and (best is None or w < best):
            best = w
    return best


# ---------------------------------------------------------------------------
# F2 linear algebra for the tests' own constructions.
# ---------------------------------------------------------------------------
def f2_rref(M: np.ndarray):
    A = np.array(M, dtype=np.uint8) & 1
    rows, cols = A.shape
    piv = []
    r = 0
    for c in range(cols):
        p = next((i for i in range(r, rows) if A[i, c]), None)
        if p is None:
            continue
        A[[r, p]] = A[[p, r]]
        for i in range(rows):
            if i != r and A[i, c]:
                A[i] ^= A[r]
        piv.append(c)
        r += 1
        if r == rows:
            break
    return A[:r], piv


def f2_rank(M: np.ndarray) -> int:
    return len(f2_rref(M)[1])


def f2_nullspace(M: np.ndarray) -> np.ndarray:
    """Basis of {v : M v = 0} over F2."""
    M = np.asarray(M, dtype=np.uint8)
    cols = M.shape[1]
    R, piv = f2_rref(M)
    free = [c for c in range(cols) if c not in piv]
    basis = []
    for f in free:
        v = np.zeros(cols, dtype=np.uint8)
        v[f] = 1
        for i, p in enumerate(piv):
            v[p] = R[i, f]
        basis.append(v)
    return np.array(basis, dtype=np.uint8).reshape(len(basis), cols)


def symplectic_dual(gen: np.ndarray, n: int) -> np.ndarray:
    """{(a, b) : a.d + b.c = 0 for every row (c, d)} (Section 2, symplectic dual)."""
    g = np.asarray(gen, dtype=np.uint8)
    swapped = np.concatenate([g[:, n:], g[:, :n]], axis=1)
    return f2_nullspace(swapped)


def random_invertible(K: int, rng: np.random.Generator) -> np.ndarray:
    while True:
        M = rng.integers(0, 2, size=(K, K), dtype=np.uint8)
        if f2_rank(M) == K:
            return M


def f2_matmul(A, B):
    return (np.asarray(A, dtype=np.int64) @ np.asarray(B, dtype=np.int64) % 2).astype(np.uint8)


# ---------------------------------------------------------------------------
# Textbook stabilizer codes.  Pauli strings -> (x | z): X=(1,0) Z=(0,1) Y=(1,1).
# ---------------------------------------------------------------------------
def pauli(strings):
    n = len(strings[0])
    out = np.zeros((len(strings), 2 * n), dtype=np.uint8)
    for r, s in enumerate(strings):
        for i, ch in enumerate(s):
            if ch in "XY":
                out[r, i] = 1
            if ch in "ZY":
                out[r, n + i] = 1
    return out


def normalizer(stab: np.ndarray, n: int) -> np.ndarray:
    """Generator matrix of the normalizer N = S^{perp_s}: an independent set of
    stabilizer rows first, then rows completing a basis of N."""
    S = np.asarray(stab, dtype=np.uint8)
    keep = []
    for r in S:
        if f2_rank(np.array(keep + [r])) == len(keep) + 1:
            keep.append(r)
    N = symplectic_dual(np.array(keep), n)
    rows = list(keep)
    for v in N:
        if f2_rank(np.array(rows + [v])) == len(rows) + 1:
            rows.append(v)
    return np.array(rows, dtype=np.uint8), len(keep)


def five_qubit():
    s = pauli(["XZZXI", "IXZZX", "XIXZZ", "ZXIXZ"])
    return normalizer(s, 5)


def steane():
    H = ["0001111", "0110011", "1010101"]
    xs = ["".join("X" if c == "1" else "I" for c in h) for h in H]
    zs = ["".join("Z" if c == "1" else "I" for c in h) for h in H]
    return normalizer(pauli(xs + zs), 7)


def toric(L: int):
    """Kitaev's toric code on an L x L torus: 2L^2 edge qubits, vertex X-stars and
    face Z-plaquettes of weight 4."""
    n = 2 * L * L

    def h(i, j):
        return (i % L) * L + (j % L)

    def v(i, j):
        return L * L + (i % L) * L + (j % L)

    rows = []
    for i in range(L):
        for j in range(L):
            r = np.zeros(2 * n, dtype=np.uint8)
            for q in (h(i, j), h(i, j - 1), v(i, j), v(i - 1, j)):
                r[q] = 1                     # star: X on the four edges at vertex (i, j)
            rows.append(r)
    for i in range(L):
        for j in range(L):
            r = np.zeros(2 * n, dtype=np.uint8)
            for q in (h(i, j), h(i + 1, j), v(i, j), v(i, j + 1)):
                r[n + q] = 1                 # plaquette: Z on the four edges of face (i, j)
            rows.append(r)
    return normalizer(np.array(rows), n)


def hamming_743_xonly():
    G = np.array([[1, 0, 0, 0, 0, 1, 1],
                  [0, 1, 0, 0, 1, 0, 1],
                  [0, 0, 1, 0, 1, 1, 0],
                  [0, 0, 0, 1, 1, 1, 1]], dtype=np.uint8)
    return np.concatenate([G, np.zeros_like(G)], axis=1)


# Local Clifford action on one qubit: the six invertible 2x2 matrices over F2
# acting on (x_i, z_i).
GL2 = [np.array(m, dtype=np.uint8) for m in
       ([[1, 0], [0, 1]], [[0, 1], [1, 0]], [[1, 1], [0, 1]],
        [[1, 0], [1, 1]], [[0, 1], [1, 1]], [[1, 1], [1, 0]])]


def local_clifford(gen: np.ndarray, n: int, choice) -> np.ndarray:
    g = np.array(gen, dtype=np.uint8)
    out = g.copy()
    for i in range(n):
        m = GL2[choice[i]]
        xi, zi = g[:, i], g[:, n + i]
        out[:, i] = (m[0, 0] * xi + m[0, 1] * zi) % 2
        out[:, n + i] = (m[1, 0] * xi + m[1, 1] * zi) % 2
    return out


def permute_qubits(gen: np.ndarray, n: int, perm) -> np.ndarray:
    g = np.asarray(gen, dtype=np.uint8)
    perm = np.asarray(perm)
    return np.concatenate([g[:, :n][:, perm], g[:, n:][:, perm]], axis=1)


def tiny_random_code(rng: np.random.Generator, n: int, K: int, kind: str) -> np.ndarray:
    """Tiny random F2 codes of several shapes (not necessarily full rank)."""
    if kind == "iid":
        return rng.integers(0, 2, size=(K, 2 * n), dtype=np.uint8)
    if kind == "css":
        g = np.zeros((K, 2 * n), dtype=np.uint8)
        for r in range(K):
            if r % 2:
                g[r, n:] = rng.integers(0, 2, size=n)
            else:
                g[r, :n] = rng.integers(0, 2, size=n)
        return g
    if kind == "yheavy":
        # many qubits carry the same Pauli in every row -> rank-1 projections
        g = rng.integers(0, 2, size=(K, 2 * n), dtype=np.uint8)
        for i in range(n):
            if rng.random() < 0.6:
                t = rng.integers(1, 4)
                m = rng.integers(0, 2, size=K, dtype=np.uint8)
                g[:, i] = m * (t & 1)
                g[:, n + i] = m * ((t >> 1) & 1)
        return g
    if kind == "sparse":
        return (rng.random((K, 2 * n)) < 0.2).astype(np.uint8)
    raise ValueError(kind)


def generator_digest(gens):
    """The digest make_oracle_tables.py writes over generator matrices."""
    import hashlib
    h = hashlib.sha256()
    for g in gens:
        h.update(bytes([g.shape[0] & 255, g.shape[1] & 255]))
        h.update(np.ascontiguousarray(g, dtype=np.uint8).tobytes())
    return h.hexdigest()


def load_oracle_table(name):
    """Reads tests/golden/<name> (written by make_oracle_tables.py): returns
    (header digests {"all": hex, "first1000": hex}, {index: (n, K, d, lower,
    upper)}), d None where the oracle did not certify it (lower <= d <= upper)."""
    digests, rows = {}, {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.startswith("# generators sha256"):
                digests["all"] = line.split()[-1]
            elif line.startswith("# first 1000 generators sha256"):
                digests["first1000"] = line.split()[-1]
            elif line.strip() and not line.startswith("#"):
                p = line.split()
                i, n, K = int(p[0]), int(p[1]), int(p[2])
                if p[3] == "-":
                    rows[i] = (n, K, None, int(p[4]), int(p[5]))
                else:
                    d = int(p[3])
                    rows[i] = (n, K, d, d, d)
    return digests, rows
