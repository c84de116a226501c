"""Normalizer matrices of random stabilizer codes with few logical qubits
(n + k rows, stabilizers first, K/N about 0.54: the shape of the paper's
second-matrix dataset, Section 3) solved on the GPU with the stabilizers
excluded, d(Q) = min wt_s(N \\ S) (Section 2.1), against the CPU oracle; with
the second generator matrix enumerated (the inclusion policy's choice) and
with the first matrix only, which must give the same d."""
import numpy as np
import pytest

import oracle
import paper_2408_10743_gb300 as dist
from paper_2408_10743_gb300 import synth
from codes import f2_rank, sym_weight_bits

pytestmark = pytest.mark.gpu

# (n, k, index): k = 2..3 logical qubits, the second matrix has 2k or so free
# rows and the policy enumerates it on all but one of these
CASES = [(36, 2, 0), (40, 2, 0), (40, 2, 1), (44, 2, 0), (44, 3, 0), (44, 3, 1), (48, 3, 0)]


@pytest.mark.parametrize("n,k,index", CASES, ids=["n%d-k%d-%d" % c for c in CASES])
def test_small_k_normalizer_vs_oracle(n, k, index):
    N, n_stab = synth.small_k_code(index, n, k)
    want = oracle.bz(N, n_stab=n_stab)["d"]
    limit = dist.dist_get_gamma_limit()
    try:
        for m in (0, 1):
            dist.dist_set_gamma_limit(m)
            with dist.Code(N) as c:
                c.set_exclude(n_stab)
                r = c.solve()
            assert r["d"] == want, (n, index, m)
            w, co = r["witness"], r["coeffs"].astype(bool)
            assert sym_weight_bits(w, n) == want
            assert np.array_equal(np.bitwise_xor.reduce(N[co], axis=0), w)
            # the witness lies outside S = span of the first n_stab rows
            assert f2_rank(np.vstack([N[:n_stab], w[None, :]])) == n_stab + 1
    finally:
        dist.dist_set_gamma_limit(limit)


def test_second_matrix_is_planned_and_saves_work():
    """On these inputs the planner builds a second generator matrix with few
    free rows and the inclusion policy enumerates it; limiting J to the first
    matrix gives the same d with at least as many codewords."""
    N, n_stab = synth.small_k_code(1, 44, 3)
    limit = dist.dist_get_gamma_limit()
    try:
        info = dist.dist_plan_info_get(N, n_stab=n_stab)
        assert info.n_gamma_used >= 2
        res = {}
        for m in (0, 1):
            dist.dist_set_gamma_limit(m)
            with dist.Code(N) as c:
                c.set_exclude(n_stab)
                res[m] = c.solve()
        assert res[0]["d"] == res[1]["d"]
        assert res[0]["codewords"] <= res[1]["codewords"]
    finally:
        dist.dist_set_gamma_limit(limit)
