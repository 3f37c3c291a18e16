"""Full-size parity on the benchmark workloads, in the configuration bench.py
times: every subproblem is enumerated on the GPU with per-subproblem outputs,
and the oracle recomputes a seeded sample of subproblems one by one."""
import numpy as np
import pytest

import graphgen
import oracle as O

pytestmark = pytest.mark.gpu

TREE_CAP = 1 << 24


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def u64(t):
    return t.cpu().numpy().view(np.uint64)


def cand_sizes(og, rk):
    rp, col = og.csr()
    d = np.diff(rp)
    src = np.repeat(np.arange(og.n), d)
    return np.bincount(src[rk[col] > rk[src]], minlength=og.n)


def test_rmat18_sampled_subproblems(gpu_lib):
    import torch
    mce = gpu_lib
    w = graphgen.rmat_18()
    og = O.Graph(w.n, w.u, w.v)
    rk = O.rank(og, "degen")
    g = mce.Graph(w.n, _t(w.u), _t(w.v))
    assert np.array_equal(mce.rank(g, rank="degen").cpu().numpy(), rk)
    pv = tuple(torch.zeros(w.n, dtype=torch.int64, device="cuda") for _ in range(3))
    r = mce.enumerate_cliques(g, per_vertex=pv, subproblem_budget=TREE_CAP)
    cnt, hsh, nodes = u64(pv[0]), u64(pv[1]), u64(pv[2])
    assert r.incomplete == int((nodes > TREE_CAP).sum())
    c = cand_sizes(og, rk)
    rng = np.random.default_rng(2024)
    light = rng.choice(np.nonzero((c >= 1) & (c <= 150))[0], 400, replace=False)
    mid = np.nonzero((nodes > 20000) & (nodes <= 400000))[0]
    mid = rng.choice(mid, min(40, len(mid)), replace=False)
    trivial = rng.choice(np.nonzero(c == 0)[0], 100, replace=False)
    sample = np.concatenate([light, mid, trivial]).astype(np.int32)
    o = O.parmce(og, rk, subset=sample, per_vertex=True, threads=8)
    assert np.array_equal(cnt[sample], o.per_vertex["count"])
    assert np.array_equal(hsh[sample], o.per_vertex["hash"])
    assert np.array_equal(nodes[sample], o.per_vertex["nodes"])
    # the capped set run as a subset gives the same totals as the per-subproblem sums
    keep = np.nonzero(nodes <= TREE_CAP)[0].astype(np.int32)
    r2 = mce.enumerate_cliques(g, subset=_t(keep))
    assert r2.count == int(cnt[keep].sum())
    assert r2.hash == int(hsh[keep].astype(object).sum()) % (1 << 64)
    assert r2.tree_nodes == int(nodes[keep].sum())
    assert r2.incomplete == 0 and r2.complete


def test_rmat18_every_subproblem_against_oracle(gpu_lib):
    """The whole R-MAT 18 benchmark set against the oracle's run of every
    subproblem (tests/golden/rmat_18_capped.json, written by
    tests/golden/make_golden.py from oracle.parmce with the 2^24-node cap):
    the same subproblems pass the cap, and every other subproblem's count,
    hash and tree nodes agree (SHA-256 of the per-subproblem arrays), as do
    the totals and the size histogram of the benchmark set."""
    import hashlib
    import json
    import os
    import torch
    mce = gpu_lib
    with open(os.path.join(os.path.dirname(__file__), "golden", "rmat_18_capped.json")) as f:
        gold = json.load(f)
    w = graphgen.rmat_18()
    g = mce.Graph(w.n, _t(w.u), _t(w.v))
    pv = tuple(torch.zeros(w.n, dtype=torch.int64, device="cuda") for _ in range(3))
    mce.enumerate_cliques(g, per_vertex=pv, subproblem_budget=TREE_CAP)
    cnt, hsh, nodes = u64(pv[0]), u64(pv[1]), u64(pv[2])
    over = nodes > TREE_CAP
    assert np.nonzero(over)[0].tolist() == gold["capped_vertices"]
    parts = []
    for a in (cnt, hsh, nodes):
        a = a.astype("<u8").copy()
        a[over] = 0
        parts.append(a.tobytes())
    assert hashlib.sha256(b"".join(parts)).hexdigest() == gold["per_vertex_sha256"]
    keep = np.nonzero(~over)[0].astype(np.int32)
    r = mce.enumerate_cliques(g, subset=_t(keep), blocks_per_sm=3, split_nodes=4096)
    assert (r.count, r.hash, r.tree_nodes, list(r.hist)) == \
        (gold["count"], int(gold["hash"]), gold["tree_nodes"], gold["hist"])


def test_chung_lu_planted_full_enumeration(gpu_lib):
    """The whole Chung-Lu graph (1.7M vertices, ~11M edges, 200 planted
    cliques): count, set hash and size histogram equal the oracle's stored
    summary (tests/golden/chung_lu_planted.json, written by make_golden.py
    from oracle.parmce), for every Section 4.2 rank."""
    import json
    import os
    mce = gpu_lib
    with open(os.path.join(os.path.dirname(__file__), "golden", "chung_lu_planted.json")) as f:
        gold = json.load(f)
    w = graphgen.chung_lu_planted()
    assert w.name == gold["workload"] and w.n == gold["n"]
    g = mce.Graph(w.n, _t(w.u), _t(w.v))
    assert g.nnz // 2 == gold["edges"]
    for kind in ("degen", "degree", "triangle"):
        r = mce.enumerate_cliques(g, rank=kind)
        assert r.count == gold["count"], kind
        assert r.hash == int(gold["hash"]), kind
        assert list(r.hist) == gold["hist"], kind


def test_batched_4096_sampled_graphs(gpu_lib):
    """The batched workload as the benchmark runs it (4,096 G(n, p) in one
    launch, a per-graph budget of 2^20 tree nodes): a seeded sample of the
    graphs finished within the budget is recomputed by the oracle, on global
    vertex ids, and compared graph by graph."""
    mce = gpu_lib
    w = graphgen.batched_er_4096()
    gptr = w.extra["graph_ptr"]
    g = mce.Graph(w.n, _t(w.u), _t(w.v))
    counts, hashes, status, tot = mce.enumerate_batched(g, gptr, node_budget=1 << 20)
    ok = np.nonzero(status == 0)[0]
    assert 0 < len(ok) < len(gptr) - 1 and not tot.complete
    assert (np.diff(w.u) >= 0).all()            # edges come graph by graph, in increasing u
    bounds = np.searchsorted(w.u, gptr)
    # stratified over the whole vertex range: up to 3 finished graphs from each
    # doubling of n (32-63, 64-127, ..., 1024-2048), so that the large sparse
    # graphs (wide candidate sets, many handed-over pieces) are compared too
    sizes = np.diff(gptr)
    rng = np.random.default_rng(77)
    sample = []
    for lo in (32, 64, 128, 256, 512, 1024):
        hi = 2 * lo if lo < 1024 else 2049
        pool = [i for i in ok if lo <= sizes[i] < hi]
        sample += list(rng.choice(pool, min(3, len(pool)), replace=False))
    assert max(sizes[sample]) >= 1024
    for i in sample:
        a, b = int(gptr[i]), int(gptr[i + 1])
        e0, e1 = int(bounds[i]), int(bounds[i + 1])
        og = O.Graph(b, w.u[e0:e1], w.v[e0:e1])      # vertices below a are isolated and left out
        sub = np.arange(a, b, dtype=np.int32)
        o = O.parmce(og, O.rank(og, "degen"), subset=sub, per_vertex=True, threads=8)
        assert int(counts[i]) == int(o.per_vertex["count"].sum()), i      # per-vertex arrays follow `sub`
        assert int(hashes[i]) == int(o.per_vertex["hash"].astype(object).sum()) % (1 << 64), i


def _delta_key(d):
    return (d.applied, d.new_count, d.new_hash, list(d.new_hist), d.sub_count, d.sub_hash, list(d.sub_hist), d.alive)


def test_chung_lu_stream_full(gpu_lib):
    """The dynamic workload at full size: the Chung-Lu base graph (n = 500,000,
    about 2M edges) and the whole stream of 10^6 new edges in its 45 batches.
    Every batch's (applied, Λnew and Λdel count, hash and histogram, alive
    cliques) equals the oracle's (Algorithms 6, 9 and 8), both through
    imce_add_edges and through the serving loop that the benchmark times."""
    mce = gpu_lib
    w = graphgen.chung_lu_stream()
    su, sv = w.extra["stream_u"], w.extra["stream_v"]
    sizes = w.extra["batch_sizes"]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    og = O.Graph(w.n, w.u, w.v)
    ost = O.Imce(og, threads=8)
    expect = []
    for i in range(len(sizes)):
        rho, onew, odel = ost.add(su[offs[i]:offs[i + 1]], sv[offs[i]:offs[i + 1]], want_list=False)
        expect.append((rho, onew.count, onew.hash, list(onew.hist), odel.count, odel.hash, list(odel.hist),
                       ost.alive))
    assert offs[-1] == 1_000_000 and len(sizes) == 45
    g = mce.Graph(w.n, _t(w.u), _t(w.v))
    st = mce.Imce(g)
    for i in range(len(sizes)):
        d = st.add_edges(_t(su[offs[i]:offs[i + 1]]), _t(sv[offs[i]:offs[i + 1]]))
        assert _delta_key(d) == expect[i], i
    st.close()
    # the serving loop: one tenant, every batch submitted at once, run in order
    srv = mce.Server(slots=4)
    t = srv.add_tenant(g)
    ids = [srv.submit(t, su[offs[i]:offs[i + 1]], sv[offs[i]:offs[i + 1]], arrival_ms=0.0)
           for i in range(len(sizes))]
    infos = [srv.wait(i) for i in ids]
    srv.close()
    for i, info in enumerate(infos):
        assert info.status == 0 and _delta_key(info.delta) == expect[i], i
