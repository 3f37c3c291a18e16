"""The no-allocation entry point (mce_enumerate_noalloc) against
mce_enumerate.

mce_enumerate_noalloc serves callers that cannot allocate device memory while
they enumerate; it keeps its working data in a fixed library-owned device
array.  This file is collected last so that, if it fails, a run stopping at
the first failure has already run every other test; it passes alone in a
fresh process as well as after the rest."""
import itertools

import numpy as np
import pytest

import graphgen

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _same(a, b):
    # integer outputs: the comparison is exact
    assert (a.count, a.hash, a.tree_nodes, list(a.hist)) == (b.count, b.hash, b.tree_nodes, list(b.hist))


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
        k = 6
        parts = [list(range(3 * i, 3 * i + 3)) for i in range(k)]
        pairs = [(a, b) for i in range(k) for j in range(i + 1, k) for a in parts[i] for b in parts[j]]
        n = 3 * k
        u = np.array([a for a, b in pairs], np.int32)
        v = np.array([b for a, b in pairs], np.int32)
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


def test_noalloc_rejects_oversized_graph(gpu_lib):
    mce = gpu_lib
    n = 5_000_000   # more vertices than the fixed scratch handles
    g = mce.Graph(n, _t(np.array([0], np.int32)), _t(np.array([1], np.int32)))
    rank = mce.rank(g, rank="degree")
    with pytest.raises(mce.MceError) as e:
        mce.enumerate_noalloc(g, rank)
    assert e.value.status == mce.MCE_EINVAL
