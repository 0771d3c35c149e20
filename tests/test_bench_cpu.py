"""The benchmark's reference arm (the oracle on the host cores) keeps its
JSON contract: one line with the metric, value, unit, a cpu_baseline record
and an end-to-end record with no host-device traffic."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--small", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    # the same workload description as the GPU arm's line (the same k sweep on the same graph)
    sys.path.insert(0, ROOT)
    import bench

    assert d["config"] == bench._config("chung_lu_n1e5_planted200_seed1", bench.KS, 1)
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT


def test_build_algorithmic_bytes_by_definition():
    """The build roofline's algorithmic bytes: for each k, 4 bytes for every
    DAG word a surviving root (out-degree >= k - 1) reads -- its own out-list
    and the out-list of each out-neighbour -- summed root by root."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench

    rng = np.random.default_rng(3)
    n = 60
    rows = [sorted(set(int(x) for x in rng.integers(u + 1, n, int(rng.integers(0, 12))))) if u < n - 1 else []
            for u in range(n)]
    orow = np.zeros(n + 1, dtype=np.uint64)
    orow[1:] = np.cumsum([len(r) for r in rows])
    ocol = np.array([v for r in rows for v in r], dtype=np.uint32)
    ks = (3, 5, 8)
    want = []
    for k in ks:
        b = 0
        for u in range(n):
            if len(rows[u]) >= k - 1:
                b += 4 * (len(rows[u]) + sum(len(rows[v]) for v in rows[u]))
        want.append(b)
    assert bench.build_algorithmic_bytes(orow, ocol, ks) == want
