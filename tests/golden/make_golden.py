"""Writes the stored expected values under tests/golden/ (oracle only).

    python tests/golden/make_golden.py fingerprints      # input fingerprints
    python tests/golden/make_golden.py er                # ER G(2000, 0.01) k=3..5
    python tests/golden/make_golden.py chunglu [k ...]   # Chung-Lu + planted, k=5..9 counts
    python tests/golden/make_golden.py rmat [k ...]      # R-MAT scale 22, count + checksum (default k=3,4)
    python tests/golden/make_golden.py rmatcount k ...   # R-MAT scale 22, count only
    python tests/golden/make_golden.py rmatscale S k ... # R-MAT scale S (config-3 parameters), count + checksum

Every expected value comes from ``oracle`` on inputs from the seeded
generator module; nothing here touches the CUDA path.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2502_00317_gb300 import graphgen as gg  # noqa: E402


def _update(name, key, value):
    path = os.path.join(HERE, name)
    d = json.load(open(path)) if os.path.exists(path) else {}
    d[key] = value
    with open(path, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
        f.write("\n")


def fingerprints():
    _update("graph_fingerprints.json", "er_2000_0.01_seed0", gg.config_er_small().fingerprint())
    _update("graph_fingerprints.json", "chung_lu_20000_40_seed1",
            gg.chung_lu_planted(n=20000, n_cliques=40, seed=1).fingerprint())
    _update("graph_fingerprints.json", "rmat_12_16_seed2", gg.rmat(scale=12, edge_factor=16, seed=2).fingerprint())
    _update("graph_fingerprints.json", "rgg_3000_25_seed3", gg.rgg_torus(3000, 25.0, seed=3).fingerprint())
    _update("graph_fingerprints.json", "er_gnm_5000_40000_seed4", gg.er_gnm(5000, 40000, seed=4).fingerprint())


def _record(name, key, og, g, ks, checksum):
    for k in ks:
        t = time.time()
        if checksum:
            c, s = og.checksum(k)
        else:
            c, s = og.count(k)[0], None
        dt = time.time() - t
        val = {"count": c, "checksum": s, "oracle_seconds": round(dt, 3), "fingerprint": g.fingerprint(),
               "m": og.m, "degeneracy": og.degeneracy}
        _update(name, f"{key}_k{k}", val)
        print(key, k, val, flush=True)


def er():
    g = gg.config_er_small()
    og = oracle.OracleGraph.from_graph(g)
    _record("config_results.json", "er_2000_0.01_seed0", og, g, [3, 4, 5], True)


def chunglu(ks):
    g = gg.config_chung_lu()
    og = oracle.OracleGraph.from_graph(g)
    _record("config_results.json", "chung_lu_1e6_2000cliques_seed1", og, g, ks, False)


def rmat(ks):
    # k = 6 has about 3.3e14 cliques on this graph: far beyond a CPU listing, so
    # the stored values stop at the sizes the oracle lists in minutes to hours
    g = gg.config_rmat()
    og = oracle.OracleGraph.from_graph(g)
    _record("config_results.json", "rmat_22_16_seed2", og, g, ks, True)


if __name__ == "__main__":
    what = sys.argv[1]
    if what == "fingerprints":
        fingerprints()
    elif what == "er":
        er()
    elif what == "chunglu":
        chunglu([int(x) for x in sys.argv[2:]] or [5, 6, 7, 8, 9])
    elif what == "rmat":
        rmat([int(x) for x in sys.argv[2:]] or [3, 4])
    elif what == "rmatscale":
        # config 3's generator at a scale the oracle lists in minutes (scale 14: about 1 min,
        # scale 16: about 11 min on 8 cores for k = 6)
        scale = int(sys.argv[2])
        g = gg.rmat(scale=scale, edge_factor=16, seed=2)
        _record("config_results.json", f"rmat_{scale}_16_seed2", oracle.OracleGraph.from_graph(g), g,
                [int(x) for x in sys.argv[3:]] or [6], True)
    elif what == "rmatcount":
        g = gg.config_rmat()
        _record("config_results.json", "rmat_22_16_seed2", oracle.OracleGraph.from_graph(g), g,
                [int(x) for x in sys.argv[2:]], False)
    else:
        raise SystemExit(__doc__)
