"""Batched one-launch MCE over many small graphs, against the oracle."""
import numpy as np
import pytest

import graphgen
import oracle as O

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def oracle_per_graph(u, v, gptr, which):
    out = {}
    for g in which:
        a, b = gptr[g], gptr[g + 1]
        sel = (u >= a) & (u < b)
        og = O.Graph(b - a, u[sel] - a, v[sel] - a)
        # ids shifted: the hash is over global ids, so recompute with the cliques
        r = O.ttt_whole(og, want_list=True)
        h = sum(O.clique_hash([x + a for x in c]) for c in r.cliques) % (1 << 64)
        out[g] = (r.count, h)
    return out


def test_batched_small_graphs_exact(gpu_lib):
    mce = gpu_lib
    u, v, gptr, _ = graphgen.batched_er(200, 4, 60, 0.1, 0.6, 77)
    g = mce.Graph(int(gptr[-1]), _t(u), _t(v))
    counts, hashes, status, tot = mce.enumerate_batched(g, gptr)
    assert (status == 0).all()
    exp = oracle_per_graph(u, v, gptr, range(200))
    for i in range(200):
        assert (int(counts[i]), int(hashes[i])) == exp[i], i
    assert tot.count == sum(c for c, _ in exp.values())


def test_batched_budget_marks_large_graphs(gpu_lib):
    mce = gpu_lib
    u, v, gptr, probs = graphgen.batched_er(64, 16, 400, 0.1, 0.6, 78)
    g = mce.Graph(int(gptr[-1]), _t(u), _t(v))
    counts, hashes, status, tot = mce.enumerate_batched(g, gptr, node_budget=20000)
    ok = np.nonzero(status == 0)[0]
    over = np.nonzero(status == mce.MCE_EBUDGET)[0]
    assert len(over) > 0 and len(ok) > 0
    small = [i for i in ok if gptr[i + 1] - gptr[i] <= 200][:20]
    exp = oracle_per_graph(u, v, gptr, small)
    for i in small:
        assert (int(counts[i]), int(hashes[i])) == exp[i]
    assert not tot.complete
    # the budget is exact: a graph is over it iff its search trees are larger
    import torch
    pv = tuple(torch.zeros(g.n, dtype=torch.int64, device="cuda") for _ in range(3))
    mce.enumerate_cliques(g, rank="degen", per_vertex=pv)
    nodes = pv[2].cpu().numpy().view(np.uint64).astype(np.int64)
    tree = np.array([nodes[gptr[i]:gptr[i + 1]].sum() for i in range(64)])
    sizes = np.diff(gptr)
    assert (status[tree <= 20000] == 0).all()
    assert (status[tree > 20000 + sizes] == mce.MCE_EBUDGET).all()
    again = mce.enumerate_batched(g, gptr, node_budget=20000)
    assert np.array_equal(again[2], status)


def test_batched_rejects_crossing_edges(gpu_lib):
    mce = gpu_lib
    g = mce.Graph(6, np.array([0, 2], np.int32), np.array([1, 4], np.int32))
    with pytest.raises(mce.MceError):
        mce.enumerate_batched(g, np.array([0, 3, 6], np.int32))


def test_plan_replay_and_tune_keep_results(gpu_lib):
    """mce_batched_*: the captured run and its replays give the oracle's
    per-graph results; the tuner changes the launch shape, not the results."""
    mce = gpu_lib
    u, v, gptr, _ = graphgen.batched_er(300, 4, 120, 0.1, 0.6, 79)
    g = mce.Graph(int(gptr[-1]), _t(u), _t(v))
    plan = mce.BatchedPlan(g, gptr)
    exp = oracle_per_graph(u, v, gptr, range(300))
    before = mce.kernel_launches()
    seen = []
    for _ in range(3):
        plan.run()
        counts, hashes, status, tot = plan.read()
        assert (status == 0).all() and tot.complete
        for i in range(300):
            assert (int(counts[i]), int(hashes[i])) == exp[i], i
        seen.append((tot.count, tot.hash, tot.tree_nodes, list(tot.hist)))
    assert seen[0] == seen[1] == seen[2]
    assert mce.kernel_launches() - before == 9      # reset, search, status per run
    bps, split, warp_small = plan.tune(tune_budget=0, repeats=1)
    assert bps in (2, 3, 4) and split in (4096, 8192, 12288) and warp_small in (False, True)
    plan.run()
    counts, hashes, status, tot = plan.read()
    assert (tot.count, tot.hash, tot.tree_nodes, list(tot.hist)) == seen[0]
    ref = mce.enumerate_batched(g, gptr)
    assert np.array_equal(ref[0], counts) and np.array_equal(ref[1], hashes)
    plan.close()


def test_plan_budget_and_trivial_graphs(gpu_lib):
    """Per-graph budget in a plan; a batch of edgeless graphs (no search
    launch at all) still reports every isolated vertex."""
    mce = gpu_lib
    u, v, gptr, _ = graphgen.batched_er(64, 16, 400, 0.1, 0.6, 78)
    g = mce.Graph(int(gptr[-1]), _t(u), _t(v))
    plan = mce.BatchedPlan(g, gptr, node_budget=20000)
    plan.tune(tune_budget=5000, repeats=1)
    plan.run()
    counts, hashes, status, tot = plan.read()
    ref = mce.enumerate_batched(g, gptr, node_budget=20000)
    assert np.array_equal(status, ref[2])
    ok = status == 0
    assert np.array_equal(counts[ok], ref[0][ok]) and np.array_equal(hashes[ok], ref[1][ok])
    assert not tot.complete
    plan.close()
    e = np.zeros(0, np.int32)
    g0 = mce.Graph(10, e, e)
    plan0 = mce.BatchedPlan(g0, np.array([0, 3, 10], np.int32))
    plan0.run()
    counts, hashes, status, tot = plan0.read()
    assert list(counts) == [3, 7] and tot.count == 10 and tot.complete
    assert int(hashes[0]) == sum(O.clique_hash([x]) for x in range(3)) % (1 << 64)
    plan0.close()
