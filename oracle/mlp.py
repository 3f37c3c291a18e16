"""CPU reference for the learned cost model — test infrastructure only.

Section 4.2 ranks vertices by an estimate of the cost of their subproblem
(higher cost -> higher rank, the load-balancing idea taken from PECO).  The
estimate here is an MLP 8 -> H -> H -> 1 with ReLU over per-vertex features,
trained with the mean squared error against log(1 + search-tree nodes).
This module restates the features and the network in float64 numpy, with the
gradient written out by the chain rule; tests pin the gradient against
central finite differences.

Parameter layout (row-major, y = W x + b): W1[H*8], b1[H], W2[H*H], b2[H],
w3[H], b3[1].
"""
from __future__ import annotations

import numpy as np

from . import Graph, core_numbers, degree, rank, triangles

N_FEAT = 8


def n_params(H: int) -> int:
    return 8 * H + H + H * H + H + H + 1


def unpack(p: np.ndarray, H: int):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + 8 * H].reshape(H, 8); o += 8 * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p, X, H: int):
    """Network output for rows X[N, 8]."""
    W1, b1, W2, b2, w3, b3 = unpack(p, H)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ w3 + b3


def loss_grad(p, X, t, H: int):
    """(mean squared error, its gradient w.r.t. the parameters)."""
    W1, b1, W2, b2, w3, b3 = unpack(p, H)
    X = np.asarray(X, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    N = X.shape[0]
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w3 + b3
    err = y - t
    loss = float(np.mean(err * err))
    dy = 2.0 * err / N                      # dL/dy
    gw3 = h2.T @ dy
    gb3 = dy.sum()
    dh2 = np.outer(dy, w3) * (a2 > 0)       # dL/da2
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (a1 > 0)             # dL/da1
    gW1 = dh1.T @ X
    gb1 = dh1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
    return loss, g


def features(g: Graph) -> np.ndarray:
    """Per-vertex features [n, 8]:
    0 log1p(degree), 1 core number, 2 log1p(triangles),
    3/4/5 mean / standard deviation / max of log1p(neighbour degree),
    6 log1p(number of neighbours of higher degree rank),
    7 local clustering 2 t / (d (d - 1)) (0 below degree 2)."""
    n = g.n
    rp, col = g.csr()
    d = degree(g).astype(np.float64)
    core = core_numbers(g).astype(np.float64)
    tri = triangles(g).astype(np.float64)
    drank = rank(g, "degree")
    F = np.zeros((n, N_FEAT), dtype=np.float64)
    F[:, 0] = np.log1p(d)
    F[:, 1] = core
    F[:, 2] = np.log1p(tri)
    ld = np.log1p(d)
    for v in range(n):
        nb = col[rp[v]:rp[v + 1]]
        if len(nb):
            x = ld[nb]
            F[v, 3] = x.mean()
            F[v, 4] = np.sqrt(max((x * x).mean() - x.mean() ** 2, 0.0))
            F[v, 5] = x.max()
            F[v, 6] = np.log1p(np.count_nonzero(drank[nb] > drank[v]))
    with np.errstate(divide="ignore", invalid="ignore"):
        F[:, 7] = np.where(d >= 2, 2.0 * tri / (d * (d - 1)), 0.0)
    return F


def features_light(g: Graph) -> np.ndarray:
    """One-pass per-vertex features [n, 8] (no core numbers, no triangles):
    0 log1p(degree d),
    1/2/3 mean / standard deviation / max of log1p(neighbour degree),
    4 log1p(number of neighbours of higher degree rank),
    5 log1p(sum over neighbours w of min(d, d(w)) / 2), a bound on the
      triangles through the vertex,
    6 fraction of neighbours of higher degree rank (0 without neighbours),
    7 log1p(sum of the neighbours' degrees)."""
    n = g.n
    rp, col = g.csr()
    d = degree(g).astype(np.float64)
    drank = rank(g, "degree")
    F = np.zeros((n, N_FEAT), dtype=np.float64)
    F[:, 0] = np.log1p(d)
    ld = np.log1p(d)
    for v in range(n):
        nb = col[rp[v]:rp[v + 1]]
        if len(nb):
            x = ld[nb]
            hi = np.count_nonzero(drank[nb] > drank[v])
            F[v, 1] = x.mean()
            F[v, 2] = np.sqrt(max((x * x).mean() - x.mean() ** 2, 0.0))
            F[v, 3] = x.max()
            F[v, 4] = np.log1p(hi)
            F[v, 5] = np.log1p(np.minimum(d[nb], d[v]).sum() / 2.0)
            F[v, 6] = hi / len(nb)
            F[v, 7] = np.log1p(d[nb].sum())
    return F
