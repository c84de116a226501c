"""Host-side planner (steps S1-S3) checked on the CPU: the generator matrices
built by the package diagonalization (Sections 2.2-2.3) are checked here
with independent Python code, including the lemma behind the lower bound."""
import itertools

import numpy as np
import pytest

import paper_2408_10743_gb300 as dist
from paper_2408_10743_gb300 import synth
from codes import f2_rank, f4_mul, tiny_random_code, toric


def proj(v, n, q):
    return int(v[q]) | (int(v[n + q]) << 1)


def load_gammas(g, field=2):
    info = dist.dist_plan_info_get(g, field=field)
    n = g.shape[1] // 2 if field == 2 else g.shape[1]
    out = []
    for j in range(info.n_gamma_built):
        units = []
        for u in range(info.a[j] + info.b[j]):
            nrep = 3 if u < info.a[j] else 1
            reps = []
            q = kind = None
            for e in range(nrep):
                v, q, kind = dist.dist_plan_unit(g, j, u, e, field=field)
                reps.append(v)
            units.append({"reps": reps, "q": q, "kind": kind})
        out.append({"units": units, "a": info.a[j], "b": info.b[j], "f": info.f[j]})
    return info, n, out


def f2_image(g, field):
    if field == 2:
        return g
    from codes import f4_linear_f2_view
    return f4_linear_f2_view(g)


def check_structure(g, field=2):
    info, n, gammas = load_gammas(g, field)
    G2 = f2_image(g, field)
    rank = f2_rank(G2)
    used = set()
    for gm in gammas:
        reps_all = [r for u in gm["units"] for r in u["reps"]]
        # every representative is a codeword: together they add no rank
        assert f2_rank(np.vstack([G2] + reps_all)) == rank
        # the units' independent representatives form a basis of the code
        basis = []
        for u in gm["units"]:
            basis.append(u["reps"][0])
            if len(u["reps"]) == 3:
                basis.append(u["reps"][1])
                assert np.array_equal(u["reps"][0] ^ u["reps"][1], u["reps"][2])
        assert len(basis) == rank and f2_rank(np.array(basis)) == rank
        assert gm["f"] == sum(1 for u in gm["units"] if u["kind"] == 2)
        qs = [u["q"] for u in gm["units"] if u["q"] >= 0]
        assert len(qs) == len(set(qs))
        assert not (set(qs) & used)
        used |= set(qs)
        # package property: the unit's value at its pivot is never cancelled
        for t, u in enumerate(gm["units"]):
            if u["q"] < 0:
                continue
            q = u["q"]
            mine = {proj(r, n, q) for r in u["reps"]}
            assert 0 not in mine
            others = [proj(r, n, q) for s, v in enumerate(gm["units"]) if s != t for r in v["reps"]]
            span = {0}
            for o in others:
                span |= {x ^ o for x in span}
            assert not (mine & span), (t, q, mine, span)
    return info, gammas


@pytest.mark.parametrize("kind", ["iid", "css", "yheavy", "sparse"])
def test_package_structure_random(kind):
    rng = np.random.default_rng({"iid": 21, "css": 22, "yheavy": 23, "sparse": 24}[kind])
    for _ in range(25):
        n = int(rng.integers(2, 9))
        K = int(rng.integers(1, min(2 * n, 12) + 1))
        g = tiny_random_code(rng, n, K, kind)
        if not g.any():
            continue
        check_structure(g)


def test_package_structure_f4():
    rng = np.random.default_rng(25)
    for _ in range(15):
        n = int(rng.integers(3, 10))
        k = int(rng.integers(1, min(n, 5) + 1))
        g4 = rng.integers(0, 4, size=(k, n), dtype=np.uint8)
        if not g4.any():
            continue
        info, gammas = check_structure(g4, field=4)
        for gm in gammas:
            for u in gm["units"]:
                # representatives are g, alpha g, alpha^2 g
                r0, r1 = u["reps"][0], u["reps"][1]
                nn = len(r0) // 2
                sym0 = r0[:nn] | (r0[nn:] << 1)
                sym1 = r1[:nn] | (r1[nn:] << 1)
                assert all(f4_mul(2, int(a)) == int(b) for a, b in zip(sym0, sym1))


def test_structure_workloads():
    check_structure(synth.single_f2())
    info, _ = check_structure(synth.single_f4(), field=4)
    assert info.n_gamma_used >= 1


def test_qc72_plan_shape():
    info = dist.dist_plan_info_get(synth.single_qc())
    assert info.k_eff == 72 and info.n_gamma_built >= 2
    assert info.a[0] + info.b[0] <= 72
    assert info.f[0] == 0


def test_bound_lemma_bruteforce():
    """Every codeword, written in a generator matrix's units, weighs at least
    (number of units used) - (free rows used) on that matrix's pivot qubits."""
    rng = np.random.default_rng(26)
    for trial in range(40):
        n = int(rng.integers(2, 6))
        K = int(rng.integers(1, min(2 * n, 8) + 1))
        g = tiny_random_code(rng, n, K, ["iid", "css", "yheavy"][trial % 3])
        if not g.any():
            continue
        info, n, gammas = load_gammas(g)
        for gm in gammas:
            units = gm["units"]
            pivots = [u["q"] for u in units if u["q"] >= 0]
            choices = [[None] + list(range(len(u["reps"]))) for u in units]
            for pick in itertools.product(*choices):
                v = np.zeros(2 * n, dtype=np.uint8)
                used = free = 0
                for u, e in zip(units, pick):
                    if e is None:
                        continue
                    v ^= u["reps"][e]
                    used += 1
                    free += u["kind"] == 2
                if used == 0:
                    continue
                wpiv = sum(1 for q in pivots if v[q] | v[n + q])
                assert wpiv >= used - free
                assert v.any()  # distinct unit choices never cancel


def test_exclusion_rank():
    N, s = toric(3)
    info = dist.dist_plan_info_get(N, n_stab=s)
    assert info.s_rank == s
    with pytest.raises(dist.DistError) as e:
        dist.dist_plan_info_get(N, n_stab=N.shape[0])
    assert e.value.code == -6


def test_information_set_search():
    """The qubit-order search (reading C14) on the QC n = 72 code: the index
    order leaves the second matrix one free row, a searched order leaves none
    (so the bound gains one per matrix from the first round on); the estimate
    of d does not depend on the order, and the same code always gets the same
    plan."""
    g = synth.single_qc(0)
    prev = dist.dist_get_plan_search()
    try:
        dist.dist_set_plan_search(0)
        a = dist.dist_plan_info_get(g)
        dist.dist_set_plan_search(8)
        b = dist.dist_plan_info_get(g)
        c = dist.dist_plan_info_get(g)
    finally:
        dist.dist_set_plan_search(prev)
    fa = list(a.f[:a.n_gamma_built])
    fb = list(b.f[:b.n_gamma_built])
    assert sum(fa) > 0 and sum(fb) == 0
    assert a.d_est == b.d_est and b.u0 <= a.u0
    assert list(b.a[:b.n_gamma_built]) == list(c.a[:c.n_gamma_built])
    assert fb == list(c.f[:c.n_gamma_built]) and b.u0 == c.u0
    # a small code (little estimated work) is planned on the index order only
    s = synth.random_f2_code(16, 12, synth.Xoshiro256ss(3))
    dist.dist_set_plan_search(0)
    try:
        x = dist.dist_plan_info_get(s)
    finally:
        dist.dist_set_plan_search(prev)
    y = dist.dist_plan_info_get(s)
    assert list(x.a[:x.n_gamma_built]) == list(y.a[:y.n_gamma_built])
    assert list(x.f[:x.n_gamma_built]) == list(y.f[:y.n_gamma_built])


@pytest.mark.parametrize("case", ["f2_full", "f2_iid", "f2_css", "f4"])
def test_package_structure_max_sizes(case):
    """The largest inputs the planner takes: n = 128 qubits (four words per
    plane) and up to 256 rows (row sets of four words), dense, CSS-like and
    F4-linear."""
    rng = np.random.default_rng({"f2_full": 31, "f2_iid": 32, "f2_css": 33, "f4": 34}[case])
    n = 128
    if case == "f2_full":
        g = rng.integers(0, 2, size=(256, 2 * n), dtype=np.uint8)
    elif case == "f2_iid":
        g = rng.integers(0, 2, size=(200, 2 * n), dtype=np.uint8)
    elif case == "f2_css":
        g = np.zeros((240, 2 * n), dtype=np.uint8)
        for r in range(240):
            off = 0 if r % 2 == 0 else n
            g[r, off + rng.choice(n, size=6, replace=False)] = 1
    else:
        g = rng.integers(0, 4, size=(100, n), dtype=np.uint8)
    info, _ = check_structure(g, field=4 if case == "f4" else 2)
    assert info.k_eff == f2_rank(f2_image(g, 4 if case == "f4" else 2)) // (2 if case == "f4" else 1)


def test_small_k_normalizers_plan_a_second_matrix():
    """Normalizer matrices with few logical qubits (Section 2.3: the second
    matrix's bound term pays off when k is small): the planner builds a second
    matrix on the unused qubits with about 2k free rows, the inclusion policy
    enumerates it, and the inclusion limit of 1 keeps only the first."""
    import paper_2408_10743_gb300 as dist
    from paper_2408_10743_gb300 import synth
    limit = dist.dist_get_gamma_limit()
    try:
        for n, k, idx in ((40, 2, 0), (44, 3, 1), (48, 3, 0), (56, 4, 0)):
            N, n_stab = synth.small_k_code(idx, n, k)
            assert N.shape == (n + k, 2 * n) and n_stab == n - k
            dist.dist_set_gamma_limit(0)
            info = dist.dist_plan_info_get(N, n_stab=n_stab)
            assert info.n_gamma_built >= 2 and info.n_gamma_used == 2
            assert info.f[0] == 0 and 2 * k <= info.f[1] <= 2 * k + 2
            dist.dist_set_gamma_limit(1)
            assert dist.dist_plan_info_get(N, n_stab=n_stab).n_gamma_used == 1
        with pytest.raises(dist.DistError):
            dist.dist_set_gamma_limit(-1)
    finally:
        dist.dist_set_gamma_limit(limit)


def test_small_k_generator_is_a_normalizer():
    """synth.small_k_normalizer: the stabilizer rows commute with every row,
    the rows are independent, and a logical pair anticommutes."""
    from paper_2408_10743_gb300 import synth
    for n, k in ((12, 2), (30, 3), (56, 4)):
        N, s = synth.small_k_code(0, n, k)
        J = np.concatenate([N[:, n:], N[:, :n]], axis=1).astype(np.int64)
        G = (N.astype(np.int64) @ J.T) & 1
        assert not G[:s].any() and not G[:, :s].any()
        assert G[s, s + 1] == 1 and f2_rank(N) == n + k


def test_dependent_rows_fall_back_to_the_kept_basis():
    """Over F2 the planner first takes the input rows as independent and
    checks that on the first matrix's free rows; dependent inputs (a repeated
    row, a zero row, a sum of rows, anywhere in the input) end up with the
    rank and the package structure of the independent rows kept in input
    order."""
    rng = np.random.default_rng(41)
    for trial in range(30):
        n = int(rng.integers(6, 40))
        K = int(rng.integers(2, n + 1))
        g = rng.integers(0, 2, size=(K, 2 * n), dtype=np.uint8)
        where = int(rng.integers(0, K + 1))
        kind = trial % 3
        if kind == 0:
            extra = g[int(rng.integers(0, K))].copy()
        elif kind == 1:
            extra = np.zeros(2 * n, dtype=np.uint8)
        else:
            extra = g[0] ^ g[K - 1]
        gd = np.insert(g, where, extra, axis=0)
        info, _ = check_structure(gd)
        assert info.k_eff == f2_rank(gd)
        if f2_rank(g) == K:
            # the same code: the same rank and matrices as without the extra row
            # when the extra row comes last (earlier rows are kept first)
            if where == K:
                a = dist.dist_plan_info_get(g)
                assert list(a.a[:a.n_gamma_built]) == list(info.a[:info.n_gamma_built])
                assert list(a.f[:a.n_gamma_built]) == list(info.f[:info.n_gamma_built])


def test_planner_after_fork():
    """A child process made by fork() after the planner's helper thread has
    started (a 72-qubit plan uses it) plans on its own thread: the same plan,
    no wait on a thread the child does not have."""
    import os
    import time
    g = synth.single_qc(0)
    parent = dist.dist_plan_info_get(g)
    pid = os.fork()
    if pid == 0:  # child: plan again and report through the exit status
        ok = 0
        try:
            c = dist.dist_plan_info_get(g)
            ok = int(c.u0 == parent.u0 and c.d_est == parent.d_est
                     and list(c.f[:c.n_gamma_built]) == list(parent.f[:parent.n_gamma_built]))
        finally:
            os._exit(0 if ok else 3)
    t0 = time.time()
    status = None
    while time.time() - t0 < 60:
        done, status = os.waitpid(pid, os.WNOHANG)
        if done:
            break
        time.sleep(0.05)
    else:
        os.kill(pid, 9)
        os.waitpid(pid, 0)
        pytest.fail("the forked child did not finish planning")
    assert os.WIFEXITED(status) and os.WEXITSTATUS(status) == 0
