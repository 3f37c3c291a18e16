"""Failure detection in the forms this library supports, none of which faults,
traps or hangs the GPU:

  - a bounded device wait that runs out: the search's own time limit ends the
    launch with MCE_ETIMEOUT (complete = 0) and the library stays usable;
  - a device allocation that fails, injected on the host
    (mce_debug_fail_alloc): MCE_ENOMEM, and an incremental state is left
    exactly as it was (all or nothing per batch);
  - a task ring too small to take hand-overs: donors keep their work, and the
    results still equal the oracle's.
"""
import time

import numpy as np
import pytest

import graphgen
import oracle as O

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _rmat(scale, seed=5):
    u, v = graphgen.rmat(scale, 16 << scale, 0.57, 0.19, 0.19, seed)
    return 1 << scale, u, v


def test_time_limit_ends_search_with_timeout(gpu_lib):
    """R-MAT 16 has more than 10^10 maximal cliques (minutes of search); a
    20 ms limit ends the launch through the kernel's bounded checks."""
    mce = gpu_lib
    n, u, v = _rmat(16)
    g = mce.Graph(n, _t(u), _t(v))
    t0 = time.perf_counter()
    r = mce.enumerate_cliques(g, rank="degen", time_limit_ms=20, allow=(mce.MCE_ETIMEOUT,))
    wall = time.perf_counter() - t0
    assert r.status == mce.MCE_ETIMEOUT and not r.complete
    assert wall < 30.0
    assert r.tree_nodes > 0
    # the library (and the context) stay usable
    w = graphgen.er_2000()
    g2 = mce.Graph(w.n, _t(w.u), _t(w.v))
    og = O.Graph(w.n, w.u, w.v)
    ref = O.parmce(og, O.rank(og, "degen"))
    r2 = mce.enumerate_cliques(g2, rank="degen")
    assert (r2.count, r2.hash, r2.tree_nodes) == (ref.count, ref.hash, ref.nodes)


def _snapshot(st, nmax=1 << 16, wmax=1 << 20):
    row, col = st.graph().csr()
    return sorted(tuple(sorted(c)) for c in st.cliques(nmax, wmax)), row.copy(), col.copy()


def test_injected_allocation_failure_leaves_incremental_state_unchanged(gpu_lib):
    """Every device allocation of one imce_add_edges call is made to fail in
    turn; each failure returns MCE_ENOMEM with the graph and the clique index
    unchanged.  The batch then succeeds and equals the oracle's update."""
    mce = gpu_lib
    rng = np.random.default_rng(3)
    n = 120
    u, v = graphgen.er(n, 0.12, 41)
    bu = rng.integers(0, n, 300).astype(np.int32)
    bv = rng.integers(0, n, 300).astype(np.int32)
    g = mce.Graph(n, _t(u), _t(v))
    st = mce.Imce(g)
    before = _snapshot(st)
    failures = 0
    try:
        for after in range(0, 400):
            mce.debug_fail_alloc(after)
            try:
                d = st.add_edges(bu, bv)
            except mce.MceError as e:
                assert e.status == mce.MCE_ENOMEM, str(e)
                mce.debug_fail_alloc(-1)
                got = _snapshot(st)
                assert got[0] == before[0]
                assert np.array_equal(got[1], before[1]) and np.array_equal(got[2], before[2])
                failures += 1
                continue
            break
        else:
            pytest.fail("the batch never succeeded")
    finally:
        mce.debug_fail_alloc(-1)
    assert failures >= 10          # the batch allocates at many points; each one was tried
    og = O.Graph(n, u, v)
    om = O.Imce(og)
    rho, new, sub = om.add(bu, bv)
    assert (d.applied, d.new_count, d.new_hash, d.sub_count, d.sub_hash) == \
        (rho, new.count, new.hash, sub.count, sub.hash)
    after_cl = _snapshot(st)[0]
    assert after_cl == sorted(om.cliques().cliques)


def test_injected_allocation_failure_in_enumerate_and_open(gpu_lib):
    mce = gpu_lib
    w = graphgen.er_2000()
    g = mce.Graph(w.n, _t(w.u), _t(w.v))
    ref = mce.enumerate_cliques(g, rank="degen")
    for after in (0, 3, 7):
        mce.debug_fail_alloc(after)
        try:
            with pytest.raises(mce.MceError) as e:
                mce.enumerate_cliques(g, rank="degen")
            assert e.value.status == mce.MCE_ENOMEM
        finally:
            mce.debug_fail_alloc(-1)
        mce.debug_fail_alloc(after)
        try:
            with pytest.raises(mce.MceError) as e:
                mce.Imce(g)
            assert e.value.status == mce.MCE_ENOMEM
        finally:
            mce.debug_fail_alloc(-1)
    r = mce.enumerate_cliques(g, rank="degen")
    assert (r.count, r.hash, r.tree_nodes) == (ref.count, ref.hash, ref.tree_nodes)


@pytest.mark.parametrize("cap", [2, 3])
def test_tiny_task_ring_keeps_results(gpu_lib, cap):
    """A ring of 2 or 3 slots refuses most hand-overs; with hand-overs asked
    for every 256 nodes the per-subproblem results must still equal the
    oracle's (counts, hashes and tree nodes)."""
    import torch
    mce = gpu_lib
    n, u, v = _rmat(12)
    g = mce.Graph(n, _t(u), _t(v))
    pv = tuple(torch.zeros(n, dtype=torch.int64, device="cuda") for _ in range(3))
    r = mce.enumerate_cliques(g, rank="degen", per_vertex=pv, queue_capacity=cap, split_nodes=256)
    og = O.Graph(n, u, v)
    ref = O.parmce(og, O.rank(og, "degen"), per_vertex=True)
    assert (r.count, r.hash, r.tree_nodes) == (ref.count, ref.hash, ref.nodes)
    for k, name in enumerate(("count", "hash", "nodes")):
        assert np.array_equal(pv[k].cpu().numpy().view(np.uint64), ref.per_vertex[name])
