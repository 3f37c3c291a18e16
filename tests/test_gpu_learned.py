"""Learned cost model on the GPU against its CPU reference (oracle.mlp).

Labels are the per-subproblem search-tree node counts that the GPU search
records itself (they equal the oracle's exactly, see test_gpu_mce.py)."""
import numpy as np
import pytest

import graphgen
import oracle as O
from oracle import mlp

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _f(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def rmat(scale, seed=5):
    u, v = graphgen.rmat(scale, 16 << scale, 0.57, 0.19, 0.19, seed)
    return 1 << scale, u, v


def spearman(a, b):
    from scipy.stats import spearmanr
    return float(spearmanr(a, b).correlation)


@pytest.mark.parametrize("case", ["er2000", "rmat12"])
def test_features_match_reference(gpu_lib, case):
    mce = gpu_lib
    if case == "er2000":
        w = graphgen.er_2000()
        n, u, v = w.n, w.u, w.v
    else:
        n, u, v = rmat(12)
    F = mce.features(mce.Graph(n, _t(u), _t(v))).cpu().numpy()
    R = mlp.features(O.Graph(n, u, v))
    assert np.allclose(F, R, rtol=1e-4, atol=2e-3)


@pytest.mark.parametrize("case", ["er2000", "rmat12"])
def test_light_features_match_reference(gpu_lib, case):
    """The one-pass feature set (degrees only) against its float64 restatement."""
    mce = gpu_lib
    if case == "er2000":
        w = graphgen.er_2000()
        n, u, v = w.n, w.u, w.v
    else:
        n, u, v = rmat(12)
    F = mce.features(mce.Graph(n, _t(u), _t(v)), kind="light").cpu().numpy()
    R = mlp.features_light(O.Graph(n, u, v))
    assert np.allclose(F, R, rtol=1e-4, atol=2e-3)


def test_loss_and_gradient_match_reference(gpu_lib):
    """FP32 GPU gradient within 1e-4 of the float64 reference (relative to the
    largest gradient component)."""
    mce = gpu_lib
    n, u, v = rmat(11)
    X = mlp.features(O.Graph(n, u, v)).astype(np.float32)
    t = np.random.default_rng(3).normal(2.0, 1.0, n).astype(np.float32)
    m = mce.Model(64, seed=1)
    p = m.get().astype(np.float64)
    loss_g, grad_g = m.loss_grad(_f(X), _f(t))
    loss_r, grad_r = mlp.loss_grad(p, X.astype(np.float64), t.astype(np.float64), 64)
    assert loss_g == pytest.approx(loss_r, rel=1e-5)
    scale = np.abs(grad_r).max()
    assert np.abs(grad_g - grad_r).max() <= 1e-4 * scale


def test_prediction_fp32_and_bf16(gpu_lib):
    """BF16 inference: 8 significant bits per weight and activation; two
    64-term layers keep the error within a few percent of the output scale."""
    mce = gpu_lib
    n, u, v = rmat(11, seed=8)
    X = mlp.features(O.Graph(n, u, v)).astype(np.float32)
    m = mce.Model(64, seed=2)
    ref = mlp.forward(m.get().astype(np.float64), X.astype(np.float64), 64)
    y32 = m.predict(_f(X), bf16=False).cpu().numpy()
    y16 = m.predict(_f(X), bf16=True).cpu().numpy()
    assert np.allclose(y32, ref, rtol=1e-5, atol=1e-5)
    scale = np.abs(ref).max() + 1.0
    assert np.abs(y16 - ref).max() <= 0.03 * scale


def test_training_on_recorded_node_counts(gpu_lib):
    """Train on log(1 + tree nodes) recorded by the search (degeneracy rank).
    Gain over the method without the network: on held-out vertices the network
    predicts subproblem cost with a smaller squared error than the best affine
    function of any single Section 4.2 key (degree, core number, triangles)."""
    import torch
    mce = gpu_lib
    n, u, v = rmat(13)
    g = mce.Graph(n, _t(u), _t(v))
    pv = tuple(torch.zeros(n, dtype=torch.int64, device="cuda") for _ in range(3))
    mce.enumerate_cliques(g, rank="degen", per_vertex=pv)
    nodes = pv[2].cpu().numpy().view(np.uint64).astype(np.float64)
    label = np.log1p(nodes).astype(np.float32)
    feat = mce.features(g)
    F = feat.cpu().numpy()
    perm = np.random.default_rng(9).permutation(n)
    tr, te = perm[: int(0.8 * n)], perm[int(0.8 * n):]
    tri = torch.from_numpy(tr).cuda()
    m = mce.Model(64, seed=4)
    loss0, _ = m.loss_grad(feat[tri].contiguous(), _f(label[tr]))
    loss = m.train(feat[tri].contiguous(), _f(label[tr]), epochs=40, batch=1024, lr=3e-3, seed=5)
    assert loss < 0.5 * loss0
    pred = m.predict(feat, bf16=True).cpu().numpy()
    mse_model = float(np.mean((pred[te] - label[te]) ** 2))
    base = {}
    for name, col in (("degree", 0), ("core", 1), ("triangles", 2)):
        A = np.stack([F[tr, col], np.ones(len(tr))], 1)
        coef, *_ = np.linalg.lstsq(A, label[tr], rcond=None)
        base[name] = float(np.mean((F[te, col] * coef[0] + coef[1] - label[te]) ** 2))
    busy = nodes > 1
    print(f"held-out MSE: model {mse_model:.4f}, affine fits {base}; spearman(model) "
          f"{spearman(pred[busy], label[busy]):.3f}; train loss {loss0:.3f} -> {loss:.3f}")
    assert mse_model < min(base.values())


def test_learned_rank_and_order_keep_the_clique_set(gpu_lib):
    """Any total rank yields C(G) (Section 4.2); scheduling order changes nothing."""
    mce = gpu_lib
    n, u, v = rmat(12, seed=13)
    og = O.Graph(n, u, v)
    ref = O.parmce(og, O.rank(og, "degen"), threads=4)
    g = mce.Graph(n, _t(u), _t(v))
    m = mce.Model(64, seed=6)
    r1 = mce.enumerate_cliques(g, rank="learned", model=m)
    assert (r1.count, r1.hash, list(r1.hist)) == (ref.count, ref.hash, list(ref.hist))
    r2 = mce.enumerate_cliques(g, rank="degen", model=m, order_by_model=True)
    assert (r2.count, r2.hash, r2.tree_nodes) == (ref.count, ref.hash, ref.nodes)
    # the learned rank is the rank of the network's BF16 prediction
    pred = m.predict(mce.features(g), bf16=True).cpu().numpy().astype(np.float64)
    assert np.array_equal(mce.rank(g, rank="learned", model=m).cpu().numpy(), O.rank_from_key(pred))


def test_model_driven_splits_keep_results(gpu_lib):
    """Learned heavy-subtree splitting (a model's predicted tree sizes mark
    subproblems that hand over pieces every 64 nodes) changes the schedule
    only: clique set, tree-node total and every subproblem's count, hash and
    node count stay the oracle's."""
    import torch
    mce = gpu_lib
    n, u, v = rmat(13, seed=21)
    og = O.Graph(n, u, v)
    ref = O.parmce(og, O.rank(og, "degen"), per_vertex=True, threads=4)
    g = mce.Graph(n, _t(u), _t(v))
    m = mce.Model(64, seed=8, features="light")
    # a model that calls many subproblems heavy: predictions are around 0..1 before training
    pv = tuple(torch.zeros(n, dtype=torch.int64, device="cuda") for _ in range(3))
    r = mce.enumerate_cliques(g, rank="degen", split_model=m, heavy_nodes=1, heavy_split_nodes=64, per_vertex=pv)
    assert r.tasks_split > 0
    assert (r.count, r.hash, r.tree_nodes, list(r.hist)) == (ref.count, ref.hash, ref.nodes, list(ref.hist))
    for k, name in enumerate(("count", "hash", "nodes")):
        assert np.array_equal(pv[k].cpu().numpy().view(np.uint64), ref.per_vertex[name])
