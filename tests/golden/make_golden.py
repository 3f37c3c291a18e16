"""Write oracle-computed expected summaries for the synthetic workloads.

Calls only the CPU oracle (``oracle``) and the seeded input generators
(``graphgen``); no value here comes from the CUDA path.  Usage:

    python tests/golden/make_golden.py er_2000 [rmat_18 ...] [--threads N]
    python tests/golden/make_golden.py --rmat18-capped [--threads N]

Each workload's summary (maximal-clique count, 64-bit set hash with seed 0,
size histogram, vertex and edge counts) goes to tests/golden/<name>.json.
The clique set does not depend on the vertex rank (Section 4.2), so the
degeneracy rank is used for speed.

--rmat18-capped writes tests/golden/rmat_18_capped.json: the R-MAT scale-18
workload under the degeneracy rank, every subproblem (Algorithm 5) run with a
cap of 2^24 search-tree nodes.  It records which subproblems pass the cap,
the summary of all the others, and a SHA-256 digest of their per-subproblem
(count, hash, tree nodes) arrays (uint64, little endian, indexed by vertex,
entries of the capped subproblems set to 0, the three arrays concatenated).
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import graphgen  # noqa: E402
import oracle as O  # noqa: E402

WORKLOADS = {
    "er_2000": graphgen.er_2000,
    "rmat_18": graphgen.rmat_18,
    "chung_lu_planted": graphgen.chung_lu_planted,
}


TREE_CAP = 1 << 24


def per_vertex_digest(count, hsh, nodes, over):
    """SHA-256 of the per-subproblem arrays with the capped entries zeroed."""
    parts = []
    for a in (count, hsh, nodes):
        a = np.asarray(a, dtype="<u8").copy()
        a[over] = 0
        parts.append(a.tobytes())
    return hashlib.sha256(b"".join(parts)).hexdigest()


def rmat18_capped(threads):
    w = graphgen.rmat_18()
    g = O.Graph(w.n, w.u, w.v)
    t0 = time.time()
    r = O.parmce(g, O.rank(g, "degen"), threads=threads, per_vertex=True, node_cap=TREE_CAP)
    pv = r.per_vertex
    over = pv["over"]
    doc = {
        "workload": w.name,
        "generator": "graphgen.rmat_18()",
        "source": "oracle.parmce (Algorithm 5 with Algorithm 1), degeneracy rank, hash seed 0, "
                  f"node_cap {TREE_CAP} per subproblem",
        "n": w.n,
        "edges": g.nnz // 2,
        "tree_cap": TREE_CAP,
        "capped_vertices": [int(x) for x in np.nonzero(over)[0]],
        "count": r.count,
        "hash": str(r.hash),
        "hist": [int(x) for x in r.hist],
        "tree_nodes": r.nodes,
        "per_vertex_sha256": per_vertex_digest(pv["count"], pv["hash"], pv["nodes"], over),
        "oracle_seconds": round(time.time() - t0, 1),
        "oracle_threads": threads,
    }
    with open(os.path.join(HERE, "rmat_18_capped.json"), "w") as f:
        json.dump(doc, f, indent=1)
    print("rmat_18_capped", r.count, len(doc["capped_vertices"]), doc["oracle_seconds"], flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="*", choices=sorted(WORKLOADS))
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--rmat18-capped", action="store_true")
    a = ap.parse_args()
    if a.rmat18_capped:
        rmat18_capped(a.threads)
    for name in a.names:
        w = WORKLOADS[name]()
        g = O.Graph(w.n, w.u, w.v)
        t0 = time.time()
        r = O.parmce(g, O.rank(g, "degen"), threads=a.threads)
        doc = {
            "workload": w.name,
            "generator": f"graphgen.{WORKLOADS[name].__name__}()",
            "source": "oracle.parmce (Algorithm 5 with Algorithm 1), degeneracy rank, hash seed 0",
            "n": w.n,
            "edges": g.nnz // 2,
            "count": r.count,
            "hash": str(r.hash),
            "hist": [int(x) for x in r.hist],
            "oracle_seconds": round(time.time() - t0, 1),
            "oracle_threads": a.threads,
        }
        with open(os.path.join(HERE, f"{name}.json"), "w") as f:
            json.dump(doc, f, indent=1)
        print(name, r.count, doc["oracle_seconds"], flush=True)


if __name__ == "__main__":
    main()
