"""Write tests/golden/counts.json: exact counts of the synthetic workloads,
computed by the CPU oracle only (never by the CUDA path).

Usage: python tests/golden/make_golden.py [--rmat-k 3,4] [--allk]
                                          [--rmat-small 16:6,7] [--skip-rmat20]
Entries already present are kept; only missing ones are computed.
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2104_13209_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "counts.json")


def load():
    if os.path.exists(OUT):
        with open(OUT) as f:
            return json.load(f)
    return {}


def save(d):
    with open(OUT + ".tmp", "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(OUT + ".tmp", OUT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rmat-k", default="3,4")
    ap.add_argument("--allk", action="store_true", help="also all-k counts of R-MAT 20 by the pivot oracle")
    ap.add_argument("--threads", type=int, default=O.default_threads())
    ap.add_argument("--rmat-small", default="",
                    help="scale:k,k;... exact counts of smaller R-MAT graphs (edge factor 16, seed 0)")
    ap.add_argument("--skip-rmat20", action="store_true")
    a = ap.parse_args()
    d = load()

    for spec in [x for x in a.rmat_small.split(";") if x]:
        scale, ks = spec.split(":")
        scale = int(scale)
        rec = d.setdefault(f"rmat{scale}_ef16_s0", {"graph": f"rmat({scale}, 16, a=.57, b=.19, c=.19, seed=0)",
                                                     "counts": {}})
        g = synth.rmat(scale, 16, seed=0)
        rec["num_edges"] = g.num_edges
        drp, dci, dmax, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
        rec["degeneracy_dmax"] = dmax
        for k in [int(x) for x in ks.split(",") if x]:
            if str(k) in rec["counts"]:
                continue
            t = time.time()
            rec["counts"][str(k)] = O.count_orient(drp, dci, k, threads=a.threads).total
            rec.setdefault("how", {})[str(k)] = f"oracle orientation route, degeneracy order, {a.threads} threads"
            print(f"R-MAT {scale} k={k}: {rec['counts'][str(k)]} ({time.time() - t:.1f}s)", flush=True)
            save(d)
    if a.skip_rmat20:
        return

    er = d.setdefault("er2000_p001_s0", {"graph": "erdos_renyi(2000, 0.01, seed=0)", "counts": {}})
    g = synth.erdos_renyi(2000, 0.01, 0)
    er["num_edges"] = g.num_edges
    res = O.count_all(g.row_ptr, g.col_idx, "degeneracy", threads=a.threads)
    er["counts"] = {str(j): c for j, c in enumerate(res.counts) if j >= 1 and (c or j <= 5)}
    er["omega"] = res.max_clique
    er["how"] = "oracle pivot route (all k), degeneracy order"
    save(d)

    rec = d.setdefault("rmat20_ef16_s0", {"graph": "rmat(20, 16, a=.57, b=.19, c=.19, seed=0)", "counts": {}})
    t = time.time()
    g = synth.rmat(20, 16, seed=0)
    print(f"generated R-MAT 20 in {time.time() - t:.1f}s", flush=True)
    rec["num_edges"] = g.num_edges
    drp, dci, dmax, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    rec["degeneracy_dmax"] = dmax
    for k in [int(x) for x in a.rmat_k.split(",") if x]:
        if str(k) in rec["counts"]:
            continue
        t = time.time()
        rec["counts"][str(k)] = O.count_orient(drp, dci, k, threads=a.threads).total
        rec.setdefault("how", {})[str(k)] = f"oracle orientation route, degeneracy order, {a.threads} threads"
        print(f"k={k}: {rec['counts'][str(k)]} ({time.time() - t:.1f}s)", flush=True)
        save(d)
    if a.allk and "allk" not in rec:
        t = time.time()
        res = O.count_pivot(g.row_ptr, g.col_idx, drp, dci, threads=a.threads)
        rec["allk"] = {str(j): c for j, c in enumerate(res.counts) if j >= 1 and c}
        rec["omega"] = res.max_clique
        rec.setdefault("how", {})["allk"] = "oracle pivot route (all k), degeneracy order"
        print(f"all-k in {time.time() - t:.1f}s", flush=True)
        save(d)


if __name__ == "__main__":
    main()
