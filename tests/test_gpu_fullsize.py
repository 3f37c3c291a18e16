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
