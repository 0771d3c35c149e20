"""Serving (kc_serve_*): continuous batching must not change any result.

Each request's count (and, for listing requests, checksum) must equal
kc_count / kc_list on the same graph alone, whatever mix of requests it was
batched with; the memory cap must hold, for what serving reserves and for
the device memory it really takes; a request too large for the cap fails
alone; stopping ends every request.  Counts and checksums are exact
integers, so "the same" is equality.
"""
import threading

import numpy as np
import pytest

import oracle
from paper_2502_00317_gb300 import graphgen as gg
from paper_2502_00317_gb300 import kclique as kc

pytestmark = pytest.mark.gpu


def _graphs():
    return [
        gg.er_gnp(300, 0.3, 1),
        gg.rgg_torus(3000, 40.0, seed=2),
        gg.complete(30),
        gg.chung_lu_planted(n=20000, n_cliques=40, seed=1),
        gg.er_gnp(400, 0.3, 12),
        gg.turan(30, 7),
        gg.rgg_torus(2000, 60.0, seed=3),
    ]


# Listing requests go up to this k: the planted-clique graph holds 1.7e10
# 8-cliques, whose listing (hashing every clique) takes far longer than the
# counts the rest of the mix asks for.
LIST_KMAX = 5


def _expected(c, hs, ks):
    """(count, checksum) of every (graph, k) alone: kc_count, and kc_list with
    cap 0 where the mix lists (checksum None elsewhere)."""
    table = {}
    for h in set(hs):
        for k in set(ks):
            count = c.count(h, k)
            checksum = None
            if k <= LIST_KMAX:
                _, total, checksum = c.list(h, k, None, 0)
                assert total == count
            table[(h, k)] = (count, checksum)
    return table


def test_results_same_alone_and_in_the_mix():
    graphs = _graphs()
    with kc.Context(0) as c:
        hs = [c.upload_host(g.n, g.rowptr, g.col) for g in graphs]
        ks = [1, 2, 3, 4, 5, 6, 7, 8, 31]
        want = _expected(c, hs, ks)
        kc.kc_serve_start(c.h, lanes=2, max_batch=64)
        rng = np.random.default_rng(0)
        n_req = 400
        modes = rng.integers(0, 2, n_req)
        reqs = [(int(hs[i]), int(ks[j]), int(md) if ks[j] <= LIST_KMAX else kc.KC_SERVE_COUNT) for i, j, md in
                zip(rng.integers(0, len(hs), n_req), rng.integers(0, len(ks), n_req), modes)]
        tickets = [None] * len(reqs)

        def submit(lo, hi):
            for i in range(lo, hi):
                tickets[i] = kc.kc_serve_submit(c.h, reqs[i][0], reqs[i][1], reqs[i][2])

        ths = [threading.Thread(target=submit, args=(i * 100, (i + 1) * 100)) for i in range(4)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        sizes = []
        for (h, k, mode), t in zip(reqs, tickets):
            r = kc.kc_serve_wait(c.h, t, 120000)
            assert r is not None and r["status"] == kc.KC_OK, r
            assert r["mode"] == mode
            assert r["count"] == want[(h, k)][0], (h, k, mode)
            assert r["checksum"] == (want[(h, k)][1] if mode == kc.KC_SERVE_LIST else 0), (h, k, mode)
            assert r["t_submit_ns"] <= r["t_start_ns"] <= r["t_done_ns"]
            sizes.append(r["batch_size"])
        assert max(sizes) > 1  # requests really were batched together
        st = kc.kc_serve_stats_get(c.h)
        assert st["submitted"] == st["completed"] == len(reqs) and st["failed"] == 0
        assert st["p50_ms"] <= st["p99_ms"]
        assert st["p50_enum_ms"] <= st["p99_enum_ms"]
        with pytest.raises(kc.KcError) as e:  # collected already
            kc.kc_serve_poll(c.h, tickets[0])
        assert e.value.status == kc.KC_E_NOT_FOUND
        kc.kc_serve_stop(c.h)
        for h in hs:
            c.free(h)


def test_inline_graphs_and_admission_cap():
    import threading as th

    import torch

    graphs = _graphs()
    cap = 256 << 20
    with kc.Context(0) as c:
        hs = [c.upload_host(g.n, g.rowptr, g.col) for g in graphs]
        # an inline graph whose upload alone needs more than half the cap fails alone
        huge = gg.er_gnm(2_000_000, 4_000_000, seed=1)
        raw = gg.rmat(scale=10, edge_factor=8, seed=4)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        low = [free0]
        stop = th.Event()

        def watch():  # device memory actually taken while serving
            while not stop.is_set():
                low[0] = min(low[0], torch.cuda.mem_get_info()[0])
                stop.wait(0.002)

        w = th.Thread(target=watch, daemon=True)
        w.start()
        try:
            _serve_inline(c, graphs, hs, huge, raw, cap)
        finally:
            stop.set()
            w.join()
            if kc.kc_serve_stats_get(c.h)["submitted"]:
                try:
                    kc.kc_serve_stop(c.h)
                except kc.KcError:
                    pass
        # what the device really lost while serving: the cap, plus the lanes' fixed
        # records (streams, events, accumulators) and the allocator's rounding
        assert free0 - low[0] <= cap + (32 << 20), (free0 - low[0], cap)
        for h in hs:
            c.free(h)


def _serve_inline(c, graphs, hs, huge, raw, cap):
    """Inline and resident requests, counted and listed, under a 256 MiB cap."""
    kc.kc_serve_start(c.h, lanes=2, max_batch=16, mem_cap_bytes=cap)
    jobs = []
    for i, g in enumerate(graphs):
        for k in (3, 5, 7):
            for mode in (kc.KC_SERVE_COUNT, kc.KC_SERVE_LIST) if k <= LIST_KMAX else (kc.KC_SERVE_COUNT,):
                jobs.append((kc.kc_serve_submit_csr(c.h, g.n, g.rowptr, g.col, k, mode=mode), g, k, mode))
                jobs.append((kc.kc_serve_submit(c.h, hs[i], k, mode), g, k, mode))
    # a raw CSR that the lane must canonicalise
    jobs.append((kc.kc_serve_submit_csr(c.h, raw.n, raw.rowptr, raw.col, 4, canonicalize=True), raw, 4, 0))
    jobs.append((kc.kc_serve_submit_csr(c.h, raw.n, raw.rowptr, raw.col, 4, canonicalize=True,
                                        mode=kc.KC_SERVE_LIST), raw, 4, 1))
    t_huge = kc.kc_serve_submit_csr(c.h, huge.n, huge.rowptr, huge.col, 3)
    oracles = {}
    for t, g, k, mode in jobs:
        r = kc.kc_serve_wait(c.h, t, 120000)
        assert r is not None and r["status"] == kc.KC_OK, (g.name, k, mode, r)
        og = oracles.setdefault(id(g), oracle.OracleGraph.from_graph(g))
        if mode == kc.KC_SERVE_LIST:
            assert (r["count"], r["checksum"]) == og.checksum(k), (g.name, k)
        else:
            assert (r["count"], r["checksum"]) == (og.count(k)[0], 0), (g.name, k)
    r = kc.kc_serve_wait(c.h, t_huge, 120000)
    assert r["status"] == kc.KC_E_OOM
    st = kc.kc_serve_stats_get(c.h)
    kc.kc_serve_stop(c.h)
    assert 0 < st["peak_reserved_bytes"] <= cap, (st, cap)


def test_stop_ends_every_request_and_errors():
    g = gg.rgg_torus(3000, 40.0, seed=2)
    with kc.Context(0) as c:
        h = c.upload_host(g.n, g.rowptr, g.col)
        want = c.count(h, 6)
        with pytest.raises(kc.KcError) as e:  # not serving yet
            kc.kc_serve_submit(c.h, h, 4)
        assert e.value.status == kc.KC_E_BUSY
        kc.kc_serve_start(c.h, lanes=1, max_batch=2)
        with pytest.raises(kc.KcError) as e:
            kc.kc_serve_start(c.h)
        assert e.value.status == kc.KC_E_BUSY
        for bad, code in (((h, 0), kc.KC_E_INVALID_ARG), ((h + 77, 4), kc.KC_E_NOT_FOUND),
                          ((h, kc.KC_MAX_K + 1), kc.KC_E_UNSUPPORTED), ((h, 4, 7), kc.KC_E_INVALID_ARG)):
            with pytest.raises(kc.KcError) as e:
                kc.kc_serve_submit(c.h, *bad)
            assert e.value.status == code
        tickets = [kc.kc_serve_submit(c.h, h, 6) for _ in range(200)]
        kc.kc_serve_stop(c.h)
        ok = busy = 0
        for t in tickets:
            r = kc.kc_serve_poll(c.h, t)
            assert r is not None  # every request ended
            if r["status"] == kc.KC_OK:
                assert r["count"] == want
                ok += 1
            else:
                assert r["status"] == kc.KC_E_BUSY
                busy += 1
        assert ok + busy == len(tickets)
        # serving again on the same context works
        kc.kc_serve_start(c.h, lanes=2)
        assert kc.kc_serve_wait(c.h, kc.kc_serve_submit(c.h, h, 6), 60000)["count"] == want
        kc.kc_serve_stop(c.h)
        c.free(h)
