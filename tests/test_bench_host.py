"""Host-side helpers of the benchmark (no GPU)."""
import numpy as np

import bench
import graphgen
import oracle as O


def test_independent_sets_are_independent_and_disjoint():
    u, v = graphgen.er(800, 0.02, 17)
    row, col = O.Graph(800, u, v).csr()
    sets = bench.independent_sets(row, col, rounds=5, seed=3)
    seen = np.zeros(800, bool)
    for S in sets:
        assert len(S) > 0
        member = np.zeros(800, bool)
        member[S] = True
        for x in S:
            assert not member[col[row[x]:row[x + 1]]].any()      # no edge inside S
            assert row[x + 1] > row[x]                            # isolated vertices are skipped
        assert not seen[S].any()                                  # rounds are disjoint
        seen[S] = True
    # every vertex that is a local minimum of the first round's priorities joins it
    assert sum(len(S) for S in sets) > 800 // 10


def test_user_rank_puts_the_set_lowest():
    """The rank the label generator builds: S first (so every neighbour of a
    vertex of S ranks higher), a permutation of [0, n)."""
    u, v = graphgen.er(300, 0.05, 5)
    row, col = O.Graph(300, u, v).csr()
    S = bench.independent_sets(row, col, rounds=1, seed=1)[0]
    rank = bench.lowest_first_rank(300, S)
    assert sorted(rank.tolist()) == list(range(300))
    assert sorted(rank[S].tolist()) == list(range(len(S)))
    for x in S:
        assert (rank[col[row[x]:row[x + 1]]] > rank[x]).all()


def test_cpu_sample_is_a_plain_prefix():
    """The CPU baseline's sample: a seeded permutation of the benchmark set cut
    before the first subproblem that would pass the node budget, so a heavy
    subproblem ends the sample instead of being skipped."""
    rng = np.random.default_rng(0)
    subset = np.arange(5000, dtype=np.int32) * 2
    nodes = np.zeros(10000, np.uint64)
    nodes[subset] = rng.integers(1, 1000, len(subset)).astype(np.uint64)
    s1 = bench.sample_prefix(subset, nodes, 50_000, seed=7)
    assert np.array_equal(s1, bench.sample_prefix(subset, nodes, 50_000, seed=7))
    perm = np.random.default_rng(7).permutation(subset)
    k = len(s1)
    assert np.array_equal(np.sort(perm[:k]), s1)
    assert nodes[s1].sum() <= 50_000 < nodes[perm[:k + 1]].sum()


def test_latency_vs_change_fit():
    """The serving line's latency-against-change summary recovers a line."""
    x = np.array([1000, 5000, 20000, 80000])
    ms = 1.5 + 0.002 * x
    out = bench.latency_vs_change(x.tolist(), (2 * x).tolist(), ms.tolist())
    assert abs(out["per_edge"]["intercept_ms"] - 1.5) < 1e-9 and abs(out["per_edge"]["ms_per_1000"] - 2.0) < 1e-9
    assert abs(out["per_changed_clique"]["ms_per_1000"] - 1.0) < 1e-9
    assert out["per_edge"]["correlation"] > 0.999
