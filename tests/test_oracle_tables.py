"""The stored oracle distances of the many-code workloads
(tests/golden/*_oracle.txt, written by tests/golden/make_oracle_tables.py from
the CPU oracle only): the tables still describe the codes the seeded
generators produce, and a sample of their entries agrees with the oracle run
afresh.  The GPU tests and bench.py compare the batched and served answers
with these tables."""
import os

import numpy as np
import pytest

import oracle
from paper_2408_10743_gb300 import synth
from codes import GOLDEN, generator_digest, load_oracle_table


def test_batch_table_matches_generators_and_oracle():
    dig, rows = load_oracle_table("batch4096_oracle.txt")
    gens = synth.batch_codes(4096)
    assert sorted(rows) == list(range(4096))
    assert generator_digest(gens) == dig["all"]
    assert generator_digest(gens[:1000]) == dig["first1000"]
    for i, g in enumerate(gens):
        n, K, d, lo, hi = rows[i]
        assert (n, K) == (g.shape[1] // 2, g.shape[0])
        assert d is not None and 1 <= d <= n - (K + 1) // 2 + 1  # Singleton-type bound
    # the oracle afresh on a seeded sample of the faster entries
    rng = np.random.default_rng(20260)
    small = [i for i in range(4096) if rows[i][0] <= 36]
    for i in rng.choice(small, size=60, replace=False):
        assert oracle.bz(gens[i])["d"] == rows[i][2], i


@pytest.mark.skipif(not os.path.exists(os.path.join(GOLDEN, "stream_oracle.txt")),
                    reason="stream table not written")
def test_stream_table_matches_generators_and_oracle():
    dig, rows = load_oracle_table("stream_oracle.txt")
    count = len(rows)
    assert sorted(rows) == list(range(count))
    first = [synth.stream_request(i)[1] for i in range(1000)]
    assert generator_digest(first) == dig["first1000"]
    for i, g in enumerate(first):
        n, K, d, lo, hi = rows[i]
        assert (n, K) == (g.shape[1] // 2, g.shape[0])
        assert 1 <= lo <= hi and (d is None or d == lo == hi)
    rng = np.random.default_rng(20261)
    small = [i for i in range(1000) if rows[i][0] <= 34]
    for i in rng.choice(small, size=40, replace=False):
        r = oracle.bz(first[i])
        assert r["d"] == rows[i][2], i
