"""GPU parity of static MCE against the CPU oracle (through the C-ABI)."""
import itertools
import json
import os
import random

import numpy as np
import pytest

import graphgen
import oracle as O

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def gpu_graph(mce, n, u, v, device=True):
    return mce.Graph(n, _t(u), _t(v)) if device else mce.Graph(n, u, v)


def per_vertex_bufs(n):
    import torch
    return tuple(torch.zeros(max(n, 1), dtype=torch.int64, device="cuda") for _ in range(3))


def list_bufs(max_cliques, max_words):
    import torch
    return (torch.empty(max_cliques, dtype=torch.int64, device="cuda"),
            torch.empty(max_words, dtype=torch.int32, device="cuda"))


def u64(t):
    return t.cpu().numpy().view(np.uint64)


def assert_same_summary(r, o):
    assert r.count == o.count
    assert r.hash == o.hash
    assert list(r.hist) == list(o.hist)


def random_pairs(n, p, rng):
    return [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]


def rmat(scale, seed=5):
    u, v = graphgen.rmat(scale, 16 << scale, 0.57, 0.19, 0.19, seed)
    return 1 << scale, u, v


# ---------------------------------------------------------------- ingest and keys

@pytest.mark.parametrize("case", ["er", "rmat12", "messy", "empty", "isolated"])
def test_csr_matches_oracle(gpu_lib, case):
    mce = gpu_lib
    if case == "er":
        w = graphgen.er_2000()
        n, u, v = w.n, w.u, w.v
    elif case == "rmat12":
        n, u, v = rmat(12)
    elif case == "messy":
        rng = np.random.default_rng(1)
        n = 777
        u = rng.integers(0, n, 20000).astype(np.int32)
        v = rng.integers(0, n, 20000).astype(np.int32)
        u[:50] = v[:50]                                        # self loops
        u, v = np.concatenate([u, v]), np.concatenate([v, u])  # both directions and repeats
    elif case == "empty":
        n, u, v = 5, np.zeros(0, np.int32), np.zeros(0, np.int32)
    else:
        n, u, v = 1000, np.array([3, 4, 999], np.int32), np.array([4, 5, 0], np.int32)
    og = O.Graph(n, u, v)
    rp, col = og.csr()
    for dev in (True, False):
        g = gpu_graph(mce, n, u, v, device=dev)
        grp, gcol = g.csr()
        assert np.array_equal(grp.astype(np.int64), rp)
        assert np.array_equal(gcol, col)


def test_invalid_vertex_id(gpu_lib):
    mce = gpu_lib
    with pytest.raises(mce.MceError) as e:
        mce.Graph(10, np.array([1, 10], np.int32), np.array([2, 3], np.int32))
    assert e.value.status == mce.MCE_EINVAL


@pytest.mark.parametrize("case", ["er", "rmat13", "dense"])
def test_vertex_keys_and_ranks(gpu_lib, case):
    mce = gpu_lib
    if case == "er":
        w = graphgen.er_2000()
        n, u, v = w.n, w.u, w.v
    elif case == "rmat13":
        n, u, v = rmat(13)
    else:
        n = 300
        u, v = graphgen.er(n, 0.4, 3)
    og = O.Graph(n, u, v)
    g = gpu_graph(mce, n, u, v)
    assert np.array_equal(mce.vertex_key(g, "degree").cpu().numpy(), O.degree(og))
    assert np.array_equal(mce.vertex_key(g, "degen").cpu().numpy(), O.core_numbers(og).astype(np.int64))
    assert np.array_equal(mce.vertex_key(g, "triangle").cpu().numpy(), O.triangles(og))
    for kind in ("degree", "degen", "triangle"):
        assert np.array_equal(mce.rank(g, rank=kind).cpu().numpy(), O.rank(og, kind)), kind


# ---------------------------------------------------------------- enumeration: small exact cases

def _check_lists(mce, n, pairs, expect, **kw):
    u = np.array([a for a, b in pairs], np.int32)
    v = np.array([b for a, b in pairs], np.int32)
    g = mce.Graph(n, u, v)
    off, vtx = list_bufs(4096, 65536)
    r = mce.enumerate_cliques(g, list_buf=(off, vtx), **kw)
    got = mce.decode_list(off, vtx, r.list_cliques)
    assert got == expect
    assert r.count == len(expect)
    return r


@pytest.mark.parametrize("seed", range(10))
def test_small_random_vs_brute_force_oracle(gpu_lib, seed):
    rng = random.Random(500 + seed)
    n = rng.randint(1, 40)
    pairs = random_pairs(n, rng.choice([0.1, 0.3, 0.5, 0.8]), rng)
    og = O.Graph(n, np.array([a for a, b in pairs], np.int32), np.array([b for a, b in pairs], np.int32))
    expect = O.ttt_whole(og, want_list=True).cliques
    for kind in ("degree", "degen", "triangle"):
        _check_lists(gpu_lib, n, pairs, expect, rank=kind)


@pytest.mark.parametrize("shape", ["K1", "K2", "K33", "K64", "K70", "empty9", "C3", "C4", "C50", "mm4", "mm6"])
def test_closed_forms(gpu_lib, shape):
    mce = gpu_lib
    if shape.startswith("K"):
        n = int(shape[1:])
        pairs = list(itertools.combinations(range(n), 2))
        expect = [tuple(range(n))]
    elif shape.startswith("empty"):
        n = int(shape[5:])
        pairs = []
        expect = [(i,) for i in range(n)]
    elif shape.startswith("C"):
        n = int(shape[1:])
        pairs = [(i, (i + 1) % n) for i in range(n)]
        expect = [(0, 1, 2)] if n == 3 else sorted(tuple(sorted(p)) for p in pairs)
    else:
        k = int(shape[2:])
        parts = [list(range(3 * i, 3 * i + 3)) for i in range(k)]
        n = 3 * k
        pairs = [(a, b) for i in range(k) for j in range(i + 1, k) for a in parts[i] for b in parts[j]]
        expect = sorted(tuple(sorted(c)) for c in itertools.product(*parts))
    _check_lists(mce, n, pairs, expect)


def test_er_2000_full_list(gpu_lib):
    mce = gpu_lib
    w = graphgen.er_2000()
    og = O.Graph(w.n, w.u, w.v)
    expect = O.ttt_whole(og, want_list=True).cliques
    with open(os.path.join(GOLDEN, "er_2000.json")) as f:
        gold = json.load(f)
    assert len(expect) == gold["count"]
    g = gpu_graph(mce, w.n, w.u, w.v)
    off, vtx = list_bufs(40000, 200000)
    r = mce.enumerate_cliques(g, list_buf=(off, vtx))
    assert mce.decode_list(off, vtx, r.list_cliques) == expect
    assert r.count == gold["count"] and r.hash == int(gold["hash"]) and list(r.hist) == gold["hist"]


# ---------------------------------------------------------------- per-subproblem parity incl. tree nodes

@pytest.mark.parametrize("kind", ["degree", "degen", "triangle"])
@pytest.mark.parametrize("split", [False, True])
def test_rmat13_per_vertex_exact(gpu_lib, kind, split):
    """Each subproblem's count, hash and search-tree node count equal the
    oracle's under the same rank and pivot tie-break."""
    mce = gpu_lib
    n, u, v = rmat(13)
    og = O.Graph(n, u, v)
    rk = O.rank(og, kind)
    o = O.parmce(og, rk, per_vertex=True, threads=4)
    g = gpu_graph(mce, n, u, v)
    pv = per_vertex_bufs(n)
    r = mce.enumerate_cliques(g, rank=kind, per_vertex=pv, split=split)
    assert_same_summary(r, o)
    assert r.tree_nodes == o.nodes
    assert np.array_equal(u64(pv[0]), o.per_vertex["count"])
    assert np.array_equal(u64(pv[1]), o.per_vertex["hash"])
    assert np.array_equal(u64(pv[2]), o.per_vertex["nodes"])


@pytest.mark.parametrize("shape", [(2, 16), (3, 64), (4, 256)])
def test_handover_stress_keeps_every_subproblem(gpu_lib, shape):
    """Hand-overs every few nodes (ParTTT prefix rule, Algorithm 3) from wide
    frames, small mask frames and memory frames, under three launch shapes:
    per-subproblem counts, hashes and tree nodes still equal the oracle's, and
    the clique list equals the oracle's list."""
    mce = gpu_lib
    bps, split_nodes = shape
    n, u, v = rmat(12, seed=21)
    og = O.Graph(n, u, v)
    rk = O.rank(og, "degen")
    o = O.parmce(og, rk, per_vertex=True, threads=4)
    g = gpu_graph(mce, n, u, v)
    pv = per_vertex_bufs(n)
    r = mce.enumerate_cliques(g, rank="degen", per_vertex=pv, blocks_per_sm=bps, split_nodes=split_nodes)
    assert r.tasks_split > 0
    assert_same_summary(r, o)
    assert r.tree_nodes == o.nodes
    assert np.array_equal(u64(pv[0]), o.per_vertex["count"])
    assert np.array_equal(u64(pv[1]), o.per_vertex["hash"])
    assert np.array_equal(u64(pv[2]), o.per_vertex["nodes"])
    off, vtx = list_bufs(r.count + 16, r.count * 40 + 1024)
    r2 = mce.enumerate_cliques(g, rank="degen", list_buf=(off, vtx), blocks_per_sm=bps, split_nodes=split_nodes)
    assert mce.decode_list(off, vtx, r2.list_cliques) == O.ttt_whole(og, want_list=True).cliques


def test_user_rank_random_permutation(gpu_lib):
    mce = gpu_lib
    n, u, v = rmat(12, seed=9)
    og = O.Graph(n, u, v)
    perm = np.random.default_rng(4).permutation(n).astype(np.int32)
    o = O.parmce(og, perm, per_vertex=True, threads=4)
    g = gpu_graph(mce, n, u, v)
    pv = per_vertex_bufs(n)
    r = mce.enumerate_cliques(g, rank="user", user_rank=_t(perm), per_vertex=pv)
    assert_same_summary(r, o)
    assert np.array_equal(u64(pv[2]), o.per_vertex["nodes"])


def test_hash_seed(gpu_lib):
    mce = gpu_lib
    w = graphgen.er(500, 0.05, 12)
    og = O.Graph(500, *w)
    g = gpu_graph(mce, 500, *w)
    for seed in (0, 12345, 2 ** 63 + 7):
        assert mce.enumerate_cliques(g, seed=seed).hash == O.parmce(og, O.rank(og, "degen"), seed=seed).hash


# ---------------------------------------------------------------- statuses

def test_node_budget(gpu_lib):
    mce = gpu_lib
    n, u, v = rmat(13)
    g = gpu_graph(mce, n, u, v)
    r = mce.enumerate_cliques(g, node_budget=1000, allow=(mce.MCE_EBUDGET,))
    assert r.status == mce.MCE_EBUDGET and not r.complete


def test_list_overflow_keeps_summary(gpu_lib):
    mce = gpu_lib
    w = graphgen.er_2000()
    og = O.Graph(w.n, w.u, w.v)
    o = O.ttt_whole(og)
    g = gpu_graph(mce, w.n, w.u, w.v)
    off, vtx = list_bufs(100, 1000)
    r = mce.enumerate_cliques(g, list_buf=(off, vtx), allow=(mce.MCE_EOVERFLOW,))
    assert r.status == mce.MCE_EOVERFLOW
    assert_same_summary(r, o)


def test_subset_and_subproblem_budget(gpu_lib):
    """A subproblem is abandoned iff its search tree exceeds the budget; the
    completed ones are exact, and a subset run reproduces the oracle's
    restricted decomposition."""
    mce = gpu_lib
    n, u, v = rmat(12, seed=11)
    og = O.Graph(n, u, v)
    rk = O.rank(og, "degen")
    o = O.parmce(og, rk, per_vertex=True, threads=4)
    nodes = o.per_vertex["nodes"]
    budget = int(np.percentile(nodes[nodes > 1], 95))
    g = gpu_graph(mce, n, u, v)
    pv = per_vertex_bufs(n)
    r = mce.enumerate_cliques(g, per_vertex=pv, subproblem_budget=budget)
    ok = nodes <= budget
    assert r.incomplete == int((~ok).sum()) > 0
    assert np.array_equal(u64(pv[2])[ok], nodes[ok])
    assert np.array_equal(u64(pv[0])[ok], o.per_vertex["count"][ok])
    assert np.array_equal(u64(pv[1])[ok], o.per_vertex["hash"][ok])
    assert (u64(pv[2])[~ok] > budget).all()
    sub = np.nonzero(ok)[0].astype(np.int32)
    r2 = mce.enumerate_cliques(g, subset=_t(sub))
    o2 = O.parmce(og, rk, subset=sub, threads=4)
    assert_same_summary(r2, o2)
    assert r2.tree_nodes == o2.nodes and r2.incomplete == 0


@pytest.mark.parametrize("hub_degree", [1500, 2100, 5000])
def test_wide_candidate_sets(gpu_lib, hub_degree):
    """A rank that puts a hub lowest gives its subproblem every neighbour as a
    candidate (more than 1024 here, so frames in memory); the result must
    not depend on the rank."""
    mce = gpu_lib
    rng = np.random.default_rng(hub_degree)
    n = hub_degree + 1
    leaves = np.arange(1, n, dtype=np.int32)
    u = [np.zeros(hub_degree, np.int32)]
    v = [leaves]
    # sparse random structure among the leaves: triangles and small cliques through the hub
    a = rng.integers(1, n, 3 * hub_degree).astype(np.int32)
    b = rng.integers(1, n, 3 * hub_degree).astype(np.int32)
    u.append(a)
    v.append(b)
    u, v = np.concatenate(u), np.concatenate(v)
    og = O.Graph(n, u, v)
    rk = np.arange(n, dtype=np.int32)      # hub (vertex 0) ranked lowest
    o = O.parmce(og, rk, per_vertex=True, threads=4)
    g = gpu_graph(mce, n, u, v)
    pv = per_vertex_bufs(n)
    r = mce.enumerate_cliques(g, rank="user", user_rank=_t(rk), per_vertex=pv)
    assert_same_summary(r, o)
    assert r.tree_nodes == o.nodes
    assert np.array_equal(u64(pv[2]), o.per_vertex["nodes"])


def test_graph_from_csr_round_trip_and_validation(gpu_lib):
    """mce_graph_from_csr accepts exactly the simple undirected CSRs (Section 3)."""
    mce = gpu_lib
    u, v = graphgen.er(300, 0.05, 31)
    g = mce.Graph(300, u, v)
    row, col = g.csr()
    g2 = mce.Graph.from_csr(row, col)
    import torch
    g3 = mce.Graph.from_csr(torch.from_numpy(row).cuda(), torch.from_numpy(col).cuda())
    r1, r2, r3 = (mce.enumerate_cliques(x, rank="degen") for x in (g, g2, g3))
    assert (r1.count, r1.hash, r1.tree_nodes) == (r2.count, r2.hash, r2.tree_nodes) == (r3.count, r3.hash,
                                                                                        r3.tree_nodes)
    empty = mce.Graph.from_csr(np.zeros(6, np.int32), np.zeros(0, np.int32))
    assert mce.enumerate_cliques(empty).count == 5
    # path 0-1-2 as the reference CSR, then one defect at a time
    ok_row, ok_col = np.array([0, 1, 3, 4], np.int32), np.array([1, 0, 2, 1], np.int32)
    mce.Graph.from_csr(ok_row, ok_col)
    bad = {
        "row offsets": (np.array([0, 1, 3, 5], np.int32), ok_col),
        "row not strictly increasing": (ok_row, np.array([1, 2, 0, 1], np.int32)),
        "id outside": (ok_row, np.array([1, 0, 7, 1], np.int32)),
        "self loop": (np.array([0, 1, 4, 5], np.int32), np.array([1, 0, 1, 2, 1], np.int32)),
        "not symmetric": (np.array([0, 1, 3, 3], np.int32), np.array([1, 0, 2], np.int32)),
    }
    for what, (rp, cl) in bad.items():
        with pytest.raises(mce.MceError) as e:
            mce.Graph.from_csr(rp, cl)
        assert e.value.status == mce.MCE_EINVAL and what in str(e.value), what


# ---------------------------------------------------------------- whole-graph ParTTT (Algorithm 3)

@pytest.mark.parametrize("case", ["complete", "empty", "star", "cycle", "moon_moser", "traced", "er", "rmat12"])
def test_whole_graph_tree_equals_oracle(gpu_lib, case):
    """Algorithm 3 from K = ∅, cand = V on the GPU: the clique set and the
    search-tree node count equal the oracle's whole-graph TTT (pinned by the
    hand-derived closed forms and the traced example), with splitting on."""
    import json
    mce = gpu_lib
    if case == "complete":
        n = 30
        pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    elif case == "empty":
        n, pairs = 9, []
    elif case == "star":
        n, pairs = 12, [(0, i) for i in range(1, 12)]
    elif case == "cycle":
        n = 21
        pairs = [(i, (i + 1) % n) for i in range(n)]
    elif case == "moon_moser":
        k = 6
        parts = [list(range(3 * i, 3 * i + 3)) for i in range(k)]
        n = 3 * k
        pairs = [(a, b) for i in range(k) for j in range(i + 1, k) for a in parts[i] for b in parts[j]]
    elif case == "traced":
        with open(os.path.join(GOLDEN, "ttt_tree_trace.json")) as f:
            d = json.load(f)
        n, pairs = d["n"], [tuple(e) for e in d["edges"]]
    elif case == "er":
        n = 400
        u, v = graphgen.er(n, 0.05, 12)
        pairs = list(zip(u.tolist(), v.tolist()))
    else:
        n, u, v = rmat(12)
        pairs = list(zip(u.tolist(), v.tolist()))
    u = np.array([a for a, b in pairs], np.int32)
    v = np.array([b for a, b in pairs], np.int32)
    og = O.Graph(n, u, v)
    ref = O.ttt_whole(og)
    g = gpu_graph(mce, n, u, v)
    for split_nodes in (0, 64):
        r = mce.enumerate_cliques(g, whole_graph=True, split_nodes=split_nodes)
        assert (r.count, r.hash, list(r.hist), r.tree_nodes) == (ref.count, ref.hash, list(ref.hist), ref.nodes)


# ---------------------------------------------------------------- clique lists streamed to the host

@pytest.mark.parametrize("buf_words", [4096, 1 << 20])
def test_stream_er2000_full_list(gpu_lib, buf_words):
    """The ER 2000 workload's cliques streamed to the host through two small
    device buffers (many chunks, some split after overflowing): every clique
    arrives once and the list equals the oracle's."""
    mce = gpu_lib
    w = graphgen.er_2000()
    g = gpu_graph(mce, w.n, w.u, w.v)
    got = []
    chunks = []

    def sink(off, vtx):
        chunks.append(len(off))
        for p in off.tolist():
            k = int(vtx[p])
            got.append(tuple(sorted(int(x) for x in vtx[p + 1:p + 1 + k])))

    r = mce.enumerate_stream(g, sink, buf_words=buf_words, rank="degen")
    ref = O.parmce(O.Graph(w.n, w.u, w.v), O.rank(O.Graph(w.n, w.u, w.v), "degen"), want_list=True)
    assert sorted(got) == ref.cliques
    assert (r.count, r.hash, list(r.hist), r.tree_nodes) == (ref.count, ref.hash, list(ref.hist), ref.nodes)
    if buf_words == 4096:
        assert len(chunks) > 4


def test_stream_rmat12_summary(gpu_lib):
    mce = gpu_lib
    n, u, v = rmat(12)
    g = gpu_graph(mce, n, u, v)
    total = [0, 0]

    def sink(off, vtx):
        total[0] += len(off)
        total[1] += len(vtx)

    r = mce.enumerate_stream(g, sink, buf_words=1 << 24, rank="degree")
    ref = mce.enumerate_cliques(g, rank="degree")
    assert (r.count, r.hash, list(r.hist), r.tree_nodes) == (ref.count, ref.hash, list(ref.hist), ref.tree_nodes)
    assert total[0] == r.count and total[1] == r.count + sum(i * int(c) for i, c in enumerate(r.hist))


@pytest.mark.parametrize("rank", ["degen", "degree"])
def test_lane_search_equals_warp_search(gpu_lib, rank):
    """The lane-parallel small search (nodes taken by the lanes from a shared
    stack, closed forms for one- and two-candidate children) and the whole-warp small
    search visit the same trees: equal per-subproblem counts, hashes and node
    counts, and equal algorithmic word operations."""
    mce = gpu_lib
    n, u, v = rmat(13, seed=8)
    g = gpu_graph(mce, n, u, v)
    outs = []
    for warp in (False, True):
        pv = per_vertex_bufs(n)
        r = mce.enumerate_cliques(g, rank=rank, per_vertex=pv, warp_small_search=warp)
        outs.append((r, [u64(t) for t in pv]))
    (a, pa), (b, pb) = outs
    assert (a.count, a.hash, list(a.hist), a.tree_nodes, a.word_ops) == \
        (b.count, b.hash, list(b.hist), b.tree_nodes, b.word_ops)
    for x, y in zip(pa, pb):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("sms", [1, 19])
def test_sm_limit_keeps_results(gpu_lib, sms):
    """With only the blocks on the first 1 or 19 SMs taking work, every
    subproblem's count, hash and tree nodes equal the unrestricted run's and
    the oracle's totals."""
    mce = gpu_lib
    n, u, v = rmat(12, seed=3)
    g = gpu_graph(mce, n, u, v)
    og = O.Graph(n, u, v)
    ref = O.parmce(og, O.rank(og, "degen"))
    outs = []
    for lim in (0, sms):
        pv = per_vertex_bufs(n)
        r = mce.enumerate_cliques(g, rank="degen", per_vertex=pv, sm_limit=lim, split_nodes=256)
        outs.append((r, [u64(t) for t in pv]))
    (a, pa), (b, pb) = outs
    assert (b.count, b.hash, b.tree_nodes) == (ref.count, ref.hash, ref.nodes)
    assert (a.count, a.hash, list(a.hist), a.tree_nodes) == (b.count, b.hash, list(b.hist), b.tree_nodes)
    for x, y in zip(pa, pb):
        assert np.array_equal(x, y)
    assert b.stats[6] <= sms * 4 * 8       # warps that took part: at most those of sms SMs


def test_hold_policy_keeps_results(gpu_lib):
    """With small subtrees kept by the whole warp while any warp waits (the
    hold policy, off by default), and with hand-overs forced often, every
    subproblem's count, hash and tree nodes equal the default run's."""
    mce = gpu_lib
    n, u, v = rmat(13, seed=11)
    g = gpu_graph(mce, n, u, v)
    outs = []
    for hold in (0, 1):
        pv = per_vertex_bufs(n)
        r = mce.enumerate_cliques(g, rank="degen", per_vertex=pv, lane_hold_waiting=hold, split_nodes=512)
        outs.append((r, [u64(t) for t in pv]))
    (a, pa), (b, pb) = outs
    assert (a.count, a.hash, list(a.hist), a.tree_nodes, a.word_ops) == \
        (b.count, b.hash, list(b.hist), b.tree_nodes, b.word_ops)
    for x, y in zip(pa, pb):
        assert np.array_equal(x, y)
