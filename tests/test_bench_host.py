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
