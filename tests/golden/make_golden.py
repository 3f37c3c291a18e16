"""Write oracle-computed expected summaries for the synthetic workloads.

Calls only the CPU oracle (``oracle``) and the seeded input generators
(``graphgen``); no value here comes from the CUDA path.  Usage:

    python tests/golden/make_golden.py er_2000 [rmat_18 ...] [--threads N]

Each workload's summary (maximal-clique count, 64-bit set hash with seed 0,
size histogram, vertex and edge counts) goes to tests/golden/<name>.json.
The clique set does not depend on the vertex rank (Section 4.2), so the
degeneracy rank is used for speed.
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import graphgen  # noqa: E402
import oracle as O  # noqa: E402

WORKLOADS = {
    "er_2000": graphgen.er_2000,
    "rmat_18": graphgen.rmat_18,
    "chung_lu_planted": graphgen.chung_lu_planted,
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="+", choices=sorted(WORKLOADS))
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
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
