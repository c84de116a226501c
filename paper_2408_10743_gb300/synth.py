"""Seeded synthetic codes for tests and benchmarks.

This module only draws random generator matrices.  It holds none of the
distance method's arithmetic, so both the GPU library's tests and the CPU
oracle's tests can use it.  The one piece of linear algebra here is a rank
test, used to resample a matrix until its rows are independent; it has its own
implementation and is not used by the library or the oracle.

Random numbers: SplitMix64 (to expand a seed) feeding xoshiro256** (Blackman
and Vigna, "Scrambled linear pseudorandom number generators", 2021).  A
workload item's seed is ``seed_for(config_id, index)``.

Workloads (the paper's matrices are not available; these stand in for them,
covering the K/N range of its random normalizer matrices, Section 3):

* ``random_f2_code``   -- K rows of F2^{2n} with i.i.d. uniform bits, resampled
  until rank K (n=24, K=24 is the small single-code case).
* ``f4_systematic``    -- [I_k | A] over F4 with A i.i.d. uniform, then a seeded
  column permutation (n=40, k=20).
* ``quasi_cyclic``     -- n=72, K=72: x and z parts each a 6x6 array of 12x12
  binary circulants whose first rows have weight uniform in {2..5} at uniform
  random positions; resampled until rank 72.
* ``batch_codes``      -- many random F2 codes, n ~ U[16,56], K ~ U[ceil(n/2), n].
* ``request_stream``   -- Poisson arrivals of random F2 and quasi-cyclic requests.
* ``small_k_code``     -- normalizer matrices of random stabilizer codes with
  few logical qubits (n + k rows, stabilizers first), K/N about 0.54.

Layouts match the library: F2 -> uint8 (K, 2n) bits x_0..x_{n-1} | z_0..z_{n-1};
F4 -> uint8 (k, n) symbols v = a + 2b standing for a + alpha*b.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> tuple[int, int]:
    """One SplitMix64 step: returns (new_state, output)."""
    x = (x + 0x9E3779B97F4A7C15) & MASK64
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return x, z ^ (z >> 31)


def _rotl(x: int, k: int) -> int:
    return ((x << k) | (x >> (64 - k))) & MASK64


class Xoshiro256ss:
    """xoshiro256** 1.0 seeded through SplitMix64."""

    def __init__(self, seed: int):
        st = seed & MASK64
        s = []
        for _ in range(4):
            st, out = splitmix64(st)
            s.append(out)
        self.s = s

    def next(self) -> int:
        s = self.s
        result = (_rotl((s[1] * 5) & MASK64, 7) * 9) & MASK64
        t = (s[1] << 17) & MASK64
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = _rotl(s[3], 45)
        return result

    def below(self, m: int) -> int:
        """Uniform integer in [0, m) (Lemire's multiply-shift with rejection)."""
        if m <= 0:
            raise ValueError("m must be positive")
        thresh = ((1 << 64) - m) % m
        while True:
            x = self.next()
            prod = x * m
            if (prod & MASK64) >= thresh:
                return prod >> 64

    def uniform(self) -> float:
        return (self.next() >> 11) * (1.0 / (1 << 53))

    def bits(self, count: int) -> np.ndarray:
        """count i.i.d. uniform bits as uint8."""
        words = (count + 63) // 64
        raw = np.array([self.next() for _ in range(words)], dtype=np.uint64)
        b = np.unpackbits(raw.view(np.uint8), bitorder="little")
        return b[:count].astype(np.uint8)

    def symbols4(self, count: int) -> np.ndarray:
        """count i.i.d. uniform values in {0,1,2,3}."""
        b = self.bits(2 * count).reshape(count, 2)
        return (b[:, 0] | (b[:, 1] << 1)).astype(np.uint8)

    def permutation(self, n: int) -> np.ndarray:
        p = np.arange(n)
        for i in range(n - 1, 0, -1):
            j = self.below(i + 1)
            p[i], p[j] = p[j], p[i]
        return p


def seed_for(config_id: int, index: int = 0) -> int:
    """Seed of item ``index`` of workload ``config_id``."""
    _, a = splitmix64(((config_id & 0xFFFFFFFF) << 32) ^ (index & 0xFFFFFFFF))
    _, b = splitmix64(a ^ 0xD1B54A32D192ED03)
    return b


def f2_rank(rows: np.ndarray) -> int:
    """Rank over F2 of a 0/1 matrix (rows as Python integers, plain elimination)."""
    basis: dict[int, int] = {}
    for r in rows:
        v = int.from_bytes(np.packbits(np.asarray(r, dtype=np.uint8), bitorder="little").tobytes(),
                           "little")
        while v:
            h = v.bit_length() - 1
            if h in basis:
                v ^= basis[h]
            else:
                basis[h] = v
                break
    return len(basis)


def random_f2_code(n: int, K: int, rng: Xoshiro256ss, max_tries: int = 1000) -> np.ndarray:
    """K x 2n i.i.d. uniform bits, redrawn from the same stream until rank K."""
    if K > 2 * n:
        raise ValueError("K must be <= 2n")
    for _ in range(max_tries):
        g = rng.bits(K * 2 * n).reshape(K, 2 * n)
        if f2_rank(g) == K:
            return g
    raise RuntimeError("no full-rank draw")


def f4_systematic(n: int, k: int, rng: Xoshiro256ss) -> np.ndarray:
    """[I_k | A] over F4 (A i.i.d. uniform k x (n-k)), columns permuted by the stream."""
    a = rng.symbols4(k * (n - k)).reshape(k, n - k)
    g = np.concatenate([np.eye(k, dtype=np.uint8), a], axis=1)
    perm = rng.permutation(n)
    return np.ascontiguousarray(g[:, perm])


def circulant(first_row: np.ndarray) -> np.ndarray:
    """b x b circulant whose row i is the first row shifted right by i:
    entry (i, j) is first_row[(j - i) mod b]."""
    fr = np.asarray(first_row, dtype=np.uint8)
    b = len(fr)
    idx = (np.arange(b)[None, :] - np.arange(b)[:, None]) % b
    return fr[idx]


def _qc_plane(rng: Xoshiro256ss, block_rows: int, block_cols: int, b: int,
              wmin: int, wmax: int) -> np.ndarray:
    out = np.zeros((block_rows * b, block_cols * b), dtype=np.uint8)
    for i in range(block_rows):
        for j in range(block_cols):
            w = wmin + rng.below(wmax - wmin + 1)
            pos = rng.permutation(b)[:w]
            fr = np.zeros(b, dtype=np.uint8)
            fr[pos] = 1
            out[i * b:(i + 1) * b, j * b:(j + 1) * b] = circulant(fr)
    return out


def quasi_cyclic(rng: Xoshiro256ss, n: int = 72, block_rows: int = 6, block_cols: int = 6,
                 wmin: int = 2, wmax: int = 5, max_tries: int = 1000) -> np.ndarray:
    """Quasi-cyclic F2 code: x and z parts drawn independently as block_rows x
    block_cols arrays of b x b circulants (b = n / block_cols), each first row of
    weight uniform in {wmin..min(wmax, b)}; redrawn until full rank."""
    if n % block_cols:
        raise ValueError("n must be a multiple of block_cols")
    b = n // block_cols
    K = block_rows * b
    wmax = min(wmax, b)
    for tries in range(1, max_tries + 1):
        x = _qc_plane(rng, block_rows, block_cols, b, wmin, wmax)
        z = _qc_plane(rng, block_rows, block_cols, b, wmin, wmax)
        g = np.concatenate([x, z], axis=1)
        if f2_rank(g) == K:
            quasi_cyclic.last_tries = tries
            return g
    raise RuntimeError("no full-rank quasi-cyclic draw")


quasi_cyclic.last_tries = 0


def random_symplectic_image(rows: np.ndarray, rng: Xoshiro256ss, steps: int) -> np.ndarray:
    """Applies `steps` symplectic transvections T_v(x) = x + <x, v> v with
    uniformly drawn nonzero v in F2^{2n} to each row (x | z) of `rows`; the
    form is <(a|b), (c|d)> = a.d + b.c.  Transvections generate the
    symplectic group, so the rows' commutation relations are kept."""
    out = np.array(rows, dtype=np.uint8, copy=True)
    n2 = out.shape[1]
    n = n2 // 2
    for _ in range(steps):
        v = rng.bits(n2)
        while not v.any():
            v = rng.bits(n2)
        sw = np.concatenate([v[n:], v[:n]])  # <x, v> = x . (v_z | v_x)
        form = (out.astype(np.int64) @ sw.astype(np.int64)) & 1
        out ^= (form[:, None] * v[None, :]).astype(np.uint8)
    return out


def small_k_normalizer(n: int, k: int, rng: Xoshiro256ss, steps: int | None = None):
    """Normalizer matrix of a random stabilizer code with n qubits and k
    logical qubits (small k): the standard code's stabilizers Z_1..Z_{n-k} and
    logicals X_j, Z_j (j > n-k) moved by a random symplectic map (a product of
    transvections).  Returns (N, n_stab): the n + k rows of N, stabilizers
    first (n_stab = n - k), each row x | z of 2n bits."""
    if not 0 <= k < n:
        raise ValueError("need 0 <= k < n")
    rows = np.zeros((n + k, 2 * n), dtype=np.uint8)
    for i in range(n - k):
        rows[i, n + i] = 1                     # Z_i
    for j in range(k):
        q = n - k + j
        rows[n - k + 2 * j, q] = 1             # X_q
        rows[n - k + 2 * j + 1, n + q] = 1     # Z_q
    return random_symplectic_image(rows, rng, 4 * n if steps is None else steps), n - k


# ---------------------------------------------------------------------------
# The named workloads.
# ---------------------------------------------------------------------------

def single_f2(index: int = 0, n: int = 24, K: int = 24) -> np.ndarray:
    """Random F2 code, n = 24 qubits, K = 24 generators (workload 0)."""
    return random_f2_code(n, K, Xoshiro256ss(seed_for(0, index)))


def single_f4(index: int = 0, n: int = 40, k: int = 20) -> np.ndarray:
    """F4-linear [I_20 | A] code of length 40 (workload 1)."""
    return f4_systematic(n, k, Xoshiro256ss(seed_for(1, index)))


def single_qc(index: int = 0) -> np.ndarray:
    """Quasi-cyclic n = 72, K = 72 code (workload 2)."""
    return quasi_cyclic(Xoshiro256ss(seed_for(2, index)))


def small_k_code(index: int = 0, n: int = 56, k: int | None = None):
    """A random small-k stabilizer code of n qubits (the paper's second-matrix
    dataset has K/N = (n+k)/2n of 0.538-0.545 and at most 9100 entries,
    i.e. n up to about 64): k = round(0.08 n) unless given.  Returns
    (N, n_stab)."""
    if k is None:
        k = max(1, int(round(0.08 * n)))
    return small_k_normalizer(n, k, Xoshiro256ss(seed_for(6, (n << 16) | (k << 8) | index)))


def batch_code(index: int, nmin: int = 16, nmax: int = 56, config_id: int = 3) -> np.ndarray:
    """Item ``index`` of the batched workload (workload 3): a random F2 code
    with n ~ U[nmin, nmax], K ~ U[ceil(n/2), n]."""
    rng = Xoshiro256ss(seed_for(config_id, index))
    n = nmin + rng.below(nmax - nmin + 1)
    kmin = (n + 1) // 2
    K = kmin + rng.below(n - kmin + 1)
    return random_f2_code(n, K, rng)


def batch_codes(count: int = 4096, nmin: int = 16, nmax: int = 56, config_id: int = 3):
    """Independent random F2 codes with n ~ U[nmin, nmax], K ~ U[ceil(n/2), n]
    (workload 3).  Returns a list of (K, 2n) uint8 arrays."""
    return [batch_code(i, nmin, nmax, config_id) for i in range(count)]


def stream_request(index: int, nmin: int = 20, nmax: int = 96, config_id: int = 4):
    """The code of request ``index`` of the served stream (workload 4), as
    (kind, generator): kind "f2" or "qc", drawn 50/50.  It depends only on the
    index, not on the arrival rate.  Quasi-cyclic sizes: n is snapped down to
    a multiple of 6 (>= 24), the x and z parts use 6 block-columns of b = n/6
    circulants, round(6K/n) in {3..6} block-rows (K = block_rows * b),
    circulant weights uniform in {2..min(5,b)}."""
    rng = Xoshiro256ss(seed_for(config_id, index))
    n = nmin + rng.below(nmax - nmin + 1)
    kmin = (n + 1) // 2
    K = kmin + rng.below(n - kmin + 1)
    if rng.below(2) == 0:
        return "f2", random_f2_code(n, K, rng)
    nq = max(24, (n // 6) * 6)
    br = min(6, max(3, int(round(6.0 * K / nq))))
    return "qc", quasi_cyclic(rng, n=nq, block_rows=br, block_cols=6, wmin=2, wmax=5)


def request_times(rate_hz: float = 2000.0, duration_s: float = 60.0, config_id: int = 4,
                  max_requests: int | None = None) -> list[float]:
    """Poisson arrival times (seconds) of the served stream: exponential gaps
    of mean 1/rate_hz from one seeded stream, up to duration_s."""
    master = Xoshiro256ss(seed_for(config_id, 0xFFFFFFFF))
    t = 0.0
    out = []
    while True:
        u = master.uniform()
        t += -math.log(1.0 - u) / rate_hz
        if t >= duration_s or (max_requests is not None and len(out) >= max_requests):
            return out
        out.append(t)


def request_stream(rate_hz: float = 2000.0, duration_s: float = 60.0, nmin: int = 20,
                   nmax: int = 96, config_id: int = 4, max_requests: int | None = None):
    """Poisson arrival stream of distance queries (workload 4).

    Yields (arrival_time_s, kind, generator); request i arrives at the i-th
    time of request_times and carries the code stream_request(i).
    """
    for i, t in enumerate(request_times(rate_hz, duration_s, config_id, max_requests)):
        kind, g = stream_request(i, nmin, nmax, config_id)
        yield t, kind, g
