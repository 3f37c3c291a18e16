"""The no-allocation entry point (mce_enumerate_noalloc).

mce_enumerate_noalloc serves callers that cannot allocate device memory while
they enumerate; it keeps its working data in a fixed library-owned device
array.  It is compared here with mce_enumerate on two calls in a row, with
the CPU oracle directly (closed forms, the ER 2000 workload), and its input
checks and size limits are exercised (every rejected input is caught by a
check that runs before anything reads through it).  This file is collected
last so that, if it fails, a run stopping at the first failure has already
run every other test; it passes alone in a fresh process as well as after
the rest."""
import json
import os

import numpy as np
import pytest

import graphgen
import oracle as O

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _same(a, b):
    # integer outputs: the comparison is exact
    assert (a.count, a.hash, a.tree_nodes, list(a.hist)) == (b.count, b.hash, b.tree_nodes, list(b.hist))


def _moon_moser(k):
    parts = [list(range(3 * i, 3 * i + 3)) for i in range(k)]
    pairs = [(a, b) for i in range(k) for j in range(i + 1, k) for a in parts[i] for b in parts[j]]
    return 3 * k, np.array([a for a, b in pairs], np.int32), np.array([b for a, b in pairs], np.int32)


@pytest.mark.parametrize("case", ["er2000", "dense300", "moon_moser", "isolated"])
def test_noalloc_matches_enumerate_twice(gpu_lib, case):
    mce = gpu_lib
    if case == "er2000":
        w = graphgen.er_2000()
        n, u, v = w.n, w.u, w.v
    elif case == "dense300":
        n = 300
        u, v = graphgen.er(n, 0.3, 17)
    elif case == "moon_moser":
        n, u, v = _moon_moser(6)
    else:
        n = 50
        u = np.array(list(range(0, 20, 2)), np.int32)
        v = np.array(list(range(1, 21, 2)), np.int32)
    g = mce.Graph(n, _t(u), _t(v))
    for seed in (0, 99):
        ref = mce.enumerate_cliques(g, rank="degen", seed=seed)
        rank = mce.rank(g, rank="degen")
        first = mce.enumerate_noalloc(g, rank, seed=seed)
        second = mce.enumerate_noalloc(g, rank, seed=seed)
        _same(first, ref)
        _same(second, ref)
        assert first.complete and second.complete


def test_noalloc_er2000_against_oracle(gpu_lib):
    """The ER 2000 workload: summary equal to the oracle's stored one, tree
    nodes equal to the oracle's under the same (degeneracy) rank."""
    mce = gpu_lib
    with open(os.path.join(GOLDEN, "er_2000.json")) as f:
        gold = json.load(f)
    w = graphgen.er_2000()
    g = mce.Graph(w.n, _t(w.u), _t(w.v))
    r = mce.enumerate_noalloc(g, mce.rank(g, rank="degen"))
    assert (r.count, r.hash, list(r.hist)) == (gold["count"], int(gold["hash"]), gold["hist"])
    og = O.Graph(w.n, w.u, w.v)
    assert r.tree_nodes == O.parmce(og, O.rank(og, "degen")).nodes


@pytest.mark.parametrize("family", ["complete", "empty", "cycle", "moon_moser"])
def test_noalloc_closed_forms(gpu_lib, family):
    """Closed forms (Section 3 definitions): K_n has one maximal clique, the
    empty graph n singletons, C_n (n >= 4) n edges, Moon–Moser 3^k cliques of
    size k; tree nodes equal the oracle's."""
    mce = gpu_lib
    if family == "complete":
        n = 40
        pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
        expect = {n: 1}
    elif family == "empty":
        n, pairs, expect = 25, [], {1: 25}
    elif family == "cycle":
        n = 31
        pairs = [(i, (i + 1) % n) for i in range(n)]
        expect = {2: n}
    else:
        n, u, v = _moon_moser(7)
        pairs = list(zip(u.tolist(), v.tolist()))
        expect = {7: 3 ** 7}
    u = np.array([a for a, b in pairs], np.int32)
    v = np.array([b for a, b in pairs], np.int32)
    g = mce.Graph(n, _t(u), _t(v))
    r = mce.enumerate_noalloc(g, mce.rank(g, rank="degen"))
    hist = {s: int(c) for s, c in enumerate(r.hist) if c}
    assert hist == expect and r.count == sum(expect.values())
    og = O.Graph(n, u, v)
    ref = O.parmce(og, O.rank(og, "degen"))
    assert (r.hash, r.tree_nodes) == (ref.hash, ref.nodes)


def _csr(n, pairs):
    adj = [set() for _ in range(n)]
    for a, b in pairs:
        adj[a].add(b)
        adj[b].add(a)
    rows = [sorted(s) for s in adj]
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([x for r in rows for x in r], np.int32)
    return rp, col


@pytest.mark.parametrize("defect", ["asymmetric", "col_out_of_range", "negative_col", "unsorted_row",
                                    "repeated_id", "self_loop", "rank_duplicate", "rank_out_of_range",
                                    "row_ptr_end", "row_ptr_decreasing"])
def test_noalloc_rejects_bad_input(gpu_lib, defect):
    """Every defect is found by a check that reads only checked values, so no
    defect reaches the search; the call returns MCE_EINVAL and names it."""
    mce = gpu_lib
    n = 12
    rng = np.random.default_rng(5)
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < 0.4]
    rp, col = _csr(n, pairs)
    rank = np.arange(n, dtype=np.int32)[::-1].copy()
    want = {"asymmetric": "not symmetric", "col_out_of_range": "outside [0, n)", "negative_col": "outside [0, n)",
            "unsorted_row": "strictly increasing", "repeated_id": "strictly increasing", "self_loop": "self loop",
            "rank_duplicate": "not a permutation", "rank_out_of_range": "rank value", "row_ptr_end": "row_ptr[n]",
            "row_ptr_decreasing": "row_ptr decreases"}[defect]
    r0 = int(np.argmax(np.diff(rp)))   # a row with at least two entries
    a, b = rp[r0], rp[r0 + 1]
    assert b - a >= 2
    rp, col = rp.copy(), col.copy()
    if defect == "asymmetric":
        # row r0 loses its last entry x; row x still lists r0
        col = np.delete(col, b - 1)
        rp[r0 + 1:] -= 1
    elif defect == "col_out_of_range":
        col[b - 1] = n + 3
    elif defect == "negative_col":
        col[a] = -1
    elif defect == "unsorted_row":
        col[a], col[a + 1] = col[a + 1], col[a]
    elif defect == "repeated_id":
        col[a + 1] = col[a]
    elif defect == "self_loop":
        col[a] = r0
    elif defect == "rank_duplicate":
        rank[3] = rank[4]
    elif defect == "rank_out_of_range":
        rank[2] = n
    elif defect == "row_ptr_end":
        rp[n] += 5                       # row_ptr[n] != nnz
    elif defect == "row_ptr_decreasing":
        k = n // 2
        rp[k] = rp[k + 1] + 1            # row k ends before it starts
    with pytest.raises(mce.MceError) as e:
        mce.enumerate_noalloc_csr(_t(rp), _t(col), n, _t(rank))
    assert e.value.status == mce.MCE_EINVAL
    assert want in str(e.value), str(e.value)
    # the library stays usable
    g = mce.Graph(n, _t([p[0] for p in pairs]), _t([p[1] for p in pairs]))
    _same(mce.enumerate_noalloc(g, mce.rank(g, rank="degen")), mce.enumerate_cliques(g, rank="degen"))


def test_noalloc_rejects_oversized_graph(gpu_lib):
    mce = gpu_lib
    n = 5_000_000   # more vertices than the fixed scratch handles
    g = mce.Graph(n, _t(np.array([0], np.int32)), _t(np.array([1], np.int32)))
    rank = mce.rank(g, rank="degree")
    with pytest.raises(mce.MceError) as e:
        mce.enumerate_noalloc(g, rank)
    assert e.value.status == mce.MCE_EINVAL
    assert "more vertices" in str(e.value)


def test_noalloc_rejects_too_many_edges(gpu_lib):
    """K_6000 has 17,997,000 edges: its Γ+ lists alone need more than the
    fixed scratch, so the call stops before any kernel runs."""
    import torch
    mce = gpu_lib
    n = 6000
    iu = torch.triu_indices(n, n, 1, device="cuda").to(torch.int32)
    g = mce.Graph(n, iu[0].contiguous(), iu[1].contiguous())
    del iu
    with pytest.raises(mce.MceError) as e:
        mce.enumerate_noalloc(g, mce.rank(g, rank="degree"))
    assert e.value.status == mce.MCE_EINVAL
    assert "graph needs more than" in str(e.value)


def test_noalloc_rejects_large_search_workspace(gpu_lib):
    """K_400: one subproblem has 399 candidates, and the per-warp search
    workspaces of a whole launch would exceed the fixed scratch."""
    mce = gpu_lib
    n = 400
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    g = mce.Graph(n, _t([a for a, b in pairs]), _t([b for a, b in pairs]))
    with pytest.raises(mce.MceError) as e:
        mce.enumerate_noalloc(g, mce.rank(g, rank="degen"))
    assert e.value.status == mce.MCE_EINVAL
    assert "the search needs more than" in str(e.value)
