"""Batched counting (kc_count_batched) against per-graph kc_count and the oracle.

Counts are exact integers: a batch must give, query by query, the same count
as kc_count on that graph alone and as the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2502_00317_gb300 import graphgen as gg
from paper_2502_00317_gb300 import kclique as kc

pytestmark = pytest.mark.gpu


def _mixed():
    return [
        (gg.er_gnp(300, 0.3, 1), 5),
        (gg.rgg_torus(3000, 40.0, seed=2), 6),
        (gg.complete(40), 7),
        (gg.chung_lu_planted(n=20000, n_cliques=40, seed=1), 8),
        (gg.er_gnp(400, 0.3, 12), 4),
        (gg.turan(30, 7), 5),
        (gg.csr_from_pairs(10, np.zeros(0), np.zeros(0)), 3),  # no edges
        (gg.complete(12), 1),
        (gg.complete(12), 2),
        (gg.complete(12), 13),  # k above the clique number
        (gg.rgg_torus(2000, 60.0, seed=3), 3),
    ]


@pytest.mark.parametrize("opts", [{}, {"no_memo": True}, {"split_threshold": 1}, {"no_prune": True}])
def test_batched_equals_separate_counts_and_oracle(opts):
    items = _mixed()
    with kc.Context(0, **opts) as c:
        hs = [c.upload_host(g.n, g.rowptr, g.col) for g, _ in items]
        # the same graph twice with two k, and every query in one batch
        graphs = hs + [hs[1], hs[3]]
        ks = [k for _, k in items] + [4, 6]
        got = c.count_batched(graphs, ks)
        alone = [c.count(h, k) for h, k in zip(graphs, ks)]
        assert got == alone
        og = {}
        for (g, _), h in zip(items, hs):
            og[h] = oracle.OracleGraph.from_graph(g)
        want = [og[h].count(k)[0] for h, k in zip(graphs, ks)]
        assert got == want
        # a second batch in a different order on the same context
        order = list(reversed(range(len(graphs))))
        got2 = c.count_batched([graphs[i] for i in order], [ks[i] for i in order])
        assert got2 == [want[i] for i in order]
        for h in hs:
            c.free(h)


def test_batched_config4_shape_sample():
    """A 64-graph sample of the config-4 mix (n <= 2,000): every query against kc_count."""
    batch = gg.config_batched(seed=5, count=64, nmax=2000)
    with kc.Context(0) as c:
        hs = [c.upload_host(g.n, g.rowptr, g.col) for g, _ in batch]
        ks = [k for _, k in batch]
        got = c.count_batched(hs, ks)
        assert got == [c.count(h, k) for h, k in zip(hs, ks)]
        for (g, k), h, v in list(zip(batch, hs, got))[:16]:
            assert v == oracle.OracleGraph.from_graph(g).count(k)[0]
        for h in hs:
            c.free(h)


def test_batched_errors():
    g = gg.complete(6)
    with kc.Context(0) as c:
        h = c.upload_host(g.n, g.rowptr, g.col)
        assert c.count_batched([], []) == []
        for bad_g, bad_k, code in (([h], [0], kc.KC_E_INVALID_ARG), ([h + 99], [3], kc.KC_E_NOT_FOUND),
                                   ([h], [kc.KC_MAX_K + 1], kc.KC_E_UNSUPPORTED)):
            with pytest.raises(kc.KcError) as e:
                c.count_batched(bad_g, bad_k)
            assert e.value.status == code
        assert c.count_batched([h, h], [3, 4]) == [20, 15]
        c.free(h)


def test_autotuner_choice_is_cached_and_changes_no_count(tmp_path):
    """kc_tune times the batch under candidate launch settings (warps per
    block, split threshold, memo budget) and applies the fastest: counts are
    unchanged.  With autotune on, the first batched call of a class probes
    and appends its choice to the cache file; a new context that reads the
    file uses the stored choice without probing (the file does not grow)."""
    batch = gg.config_batched(seed=6, count=48, nmax=3000)
    cache = tmp_path / "tune.txt"
    with kc.Context(0) as c:
        hs = [c.upload_host(g.n, g.rowptr, g.col) for g, _ in batch]
        ks = [k for _, k in batch]
        want = [c.count(h, k) for h, k in zip(hs, ks)]
        r = c.tune(hs, ks)
        assert r["probes"] >= 2 and r["ms_tuned"] <= r["ms_default"], r
        assert r["warps_small"] in (4, 8) and r["warps_large"] in (2, 4), r
        assert r["key"].startswith("NVIDIA") or "/" in r["key"], r
        assert c.count_batched(hs, ks) == want
        assert [c.count(h, k) for h, k in zip(hs, ks)] == want
        for h in hs:
            c.free(h)
    with kc.Context(0, autotune=True, tune_cache=str(cache)) as c:
        hs = [c.upload_host(g.n, g.rowptr, g.col) for g, _ in batch]
        assert c.count_batched(hs, ks) == want
        lines = cache.read_text().splitlines()
        assert len(lines) == 1 and len(lines[0].split()) == 5, lines
        for h in hs:
            c.free(h)
    with kc.Context(0, autotune=True, tune_cache=str(cache)) as c:
        hs = [c.upload_host(g.n, g.rowptr, g.col) for g, _ in batch]
        assert c.count_batched(hs, ks) == want
        assert cache.read_text().splitlines() == lines  # taken from the file, no new probe
        # a single graph in autotune mode: its class is probed once, on its dense core
        g, k = gg.chung_lu_planted(n=20000, n_cliques=40, seed=1), 7
        h = c.upload_host(g.n, g.rowptr, g.col)
        assert c.count(h, k) == oracle.OracleGraph.from_graph(g).count(k)[0]
        assert len(cache.read_text().splitlines()) == 2
        assert c.count(h, k) == oracle.OracleGraph.from_graph(g).count(k)[0]
        assert len(cache.read_text().splitlines()) == 2
        for hh in hs + [h]:
            c.free(hh)
