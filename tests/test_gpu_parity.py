"""GPU parity: the CUDA path through the C ABI against the oracle.

Integer work, so the bar is bit-exact: counts, checksums, core numbers and
listed tuples must equal the oracle's.  Where several outputs are correct
(the DAG orientation, the order of listed tuples) the unique parts are
compared and the rest is checked for validity.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2502_00317_gb300 import graphgen as gg
from paper_2502_00317_gb300 import kclique as kc

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ctx():
    c = kc.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx_plain():
    c = kc.Context(0, no_memo=True, no_prune=True)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx_memo_only():
    c = kc.Context(0, no_prune=True, memo_min_k=3)
    yield c
    c.close()


def _torch():
    import torch
    return torch


def _list_all(c, g, k, total):
    torch = _torch()
    buf = torch.empty(max(total * k, 1), dtype=torch.int32, device="cuda")
    w, t, s = c.list(g, k, buf, total)
    torch.cuda.synchronize()
    arr = buf[: w * k].cpu().numpy().view(np.uint32).reshape(w, k)
    return arr, t, s


def _check_graph(c, g, og, ks, listing=True):
    h = c.upload_host(g.n, g.rowptr, g.col, canonicalize=not g.canonical)
    try:
        info = c.info(h)
        assert info["m"] == og.m
        assert info["degeneracy"] == og.degeneracy
        for k in ks:
            want_c, want_s = og.checksum(k)
            assert c.count(h, k) == want_c, ("count", g.name, k)
            if listing:
                arr, t, s = _list_all(c, h, k, want_c)
                assert t == want_c and s == want_s, ("list", g.name, k)
                assert arr.shape[0] == want_c
                if want_c and want_c <= 200000:
                    got = np.unique(arr, axis=0)
                    assert got.shape[0] == want_c  # no tuple twice
                    exp, _, _ = og.list(k)
                    assert np.array_equal(got, np.unique(exp, axis=0))
    finally:
        c.free(h)


def _fig2():
    d = json.load(open(os.path.join(GOLD, "fig2_dag.json")))
    out = {int(u): v for u, v in d["out"].items()}
    a = [u for u in out for v in out[u]]
    b = [v for u in out for v in out[u]]
    return d, gg.csr_from_pairs(d["n"], np.array(a), np.array(b))


# ------------------------------------------------------------ worked example
def test_fig2_dag(ctx):
    d, g = _fig2()
    og = oracle.OracleGraph.from_graph(g)
    h = ctx.upload_host(g.n, g.rowptr, g.col)
    assert ctx.count(h, 4) == d["k4_count"] == 14
    arr, t, s = _list_all(ctx, h, 4, 14)
    got = {tuple(r) for r in arr.tolist()}
    for cl in d["k4_first_cliques"]:
        assert tuple(cl) in got
    assert [ctx.count(h, k) for k in range(1, 7)] == [og.count(k)[0] for k in range(1, 7)]
    ctx.free(h)
    _check_graph(ctx, g, og, range(1, 7))


# ---------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [2, 5, 31, 32, 33, 64, 65, 100, 129, 200])
def test_complete_graphs(ctx, n):
    g = gg.complete(n)
    h = ctx.upload_host(g.n, g.rowptr, g.col)
    try:
        for k in sorted({1, 2, 3, 4, 5, 6, 9, min(n, 12), n, n + 1} - {0}):
            if k > kc.KC_MAX_K:
                continue
            if n >= 100 and 7 <= k < n - 3:
                continue  # C(n, k) too large to enumerate in a test
            assert ctx.count(h, k) == oracle.binom(n, k), (n, k)
    finally:
        ctx.free(h)


@pytest.mark.parametrize("n,r", [(10, 3), (17, 4), (24, 5), (30, 7), (40, 10), (70, 6)])
def test_turan_graphs(ctx, n, r):
    g = gg.turan(n, r)
    sizes = [len(range(i, n, r)) for i in range(r)]
    h = ctx.upload_host(g.n, g.rowptr, g.col)
    try:
        for k in range(1, r + 3):
            assert ctx.count(h, k) == oracle.elementary_symmetric(sizes, k), (n, r, k)
    finally:
        ctx.free(h)


def test_disjoint_cliques(ctx):
    sizes = [3, 7, 11, 20, 33, 47, 60, 1, 5]
    g = gg.disjoint_cliques(sizes)
    h = ctx.upload_host(g.n, g.rowptr, g.col)
    try:
        for k in range(1, 11):
            assert ctx.count(h, k) == sum(oracle.binom(s, k) for s in sizes)
    finally:
        ctx.free(h)


# ----------------------------------------------------- random vs oracle
@pytest.mark.parametrize("seed", range(10))
def test_tiny_random_vs_brute_force(ctx, seed):
    n = 8 + seed
    g = gg.er_gnp(n, [0.2, 0.4, 0.6, 0.8, 0.95][seed % 5], seed)
    adj = oracle.adjacency_sets(g.n, g.rowptr, g.col)
    h = ctx.upload_host(g.n, g.rowptr, g.col)
    try:
        for k in range(1, 9):
            bf = oracle.brute_force_cliques(g.n, adj, k)
            assert ctx.count(h, k) == len(bf)
            if bf:
                arr, t, s = _list_all(ctx, h, k, len(bf))
                assert sorted(map(tuple, arr.tolist())) == bf
                assert s == sum(oracle.clique_hash(c) for c in bf) % (1 << 64)
    finally:
        ctx.free(h)


@pytest.mark.parametrize("n,p,seed", [(300, 0.3, 1), (500, 0.12, 2), (1000, 0.05, 3), (150, 0.6, 4)])
def test_medium_random_vs_oracle(ctx, n, p, seed):
    g = gg.er_gnp(n, p, seed)
    og = oracle.OracleGraph.from_graph(g)
    _check_graph(ctx, g, og, [3, 4, 5, 6], listing=True)


def test_er_2000_config_vs_golden(ctx):
    """Erdos-Renyi G(2000, 0.01), seed 0: counts and checksums for k = 3, 4, 5."""
    gold = json.load(open(os.path.join(GOLD, "config_results.json")))
    g = gg.config_er_small()
    h = ctx.upload_host(g.n, g.rowptr, g.col)
    try:
        for k in (3, 4, 5):
            want = gold[f"er_2000_0.01_seed0_k{k}"]
            assert want["fingerprint"] == g.fingerprint()
            assert ctx.count(h, k) == want["count"]
            w, t, s = ctx.list(h, k, None, 0)
            assert (t, s) == (want["count"], want["checksum"])
    finally:
        ctx.free(h)


def test_chung_lu_small_tiers(ctx, ctx_plain, ctx_memo_only):
    """Power-law background + planted cliques: every width tier, memo and pruning on/off."""
    g = gg.chung_lu_planted(n=20000, n_cliques=40, seed=1)
    og = oracle.OracleGraph.from_graph(g)
    hs = [c.upload_host(g.n, g.rowptr, g.col) for c in (ctx, ctx_plain, ctx_memo_only)]
    try:
        for k in (3, 4, 5, 6, 7):
            want = og.count(k)[0]
            for c, h in zip((ctx, ctx_plain, ctx_memo_only), hs):
                assert c.count(h, k) == want, (k, c)
        for k in (4, 5):
            want_c, want_s = og.checksum(k)
            for c, h in zip((ctx, ctx_plain), hs[:2]):
                w, t, s = c.list(h, k, None, 0)
                assert (t, s) == (want_c, want_s)
    finally:
        for c, h in zip((ctx, ctx_plain, ctx_memo_only), hs):
            c.free(h)


@pytest.mark.parametrize("maker,ks,dense", [
    (lambda: gg.chung_lu_planted(n=4000, n_cliques=6, smin=20, smax=30, seed=3), (6, 7), True),
    (lambda: gg.complete(28), (6, 8), True),
    (lambda: gg.turan(36, 12), (6, 7), True),
    # neighbourhood density about 0.6: Eq. (1) never holds, the listing is plain
    (lambda: gg.rgg_torus(3000, 40.0, seed=2), (6,), False),
])
def test_listing_trie_replays_and_matches_oracle(ctx, ctx_plain, maker, ks, dense):
    """Listing with the device trie (Sec. IV, Algorithms 3-4): stored l-clique
    lists of dense prefix subgraphs are replayed under other prefixes.  The
    listed tuple set, total and checksum equal the oracle's with the memo on
    and off; with it on, the trie is used (hits) and fewer candidate words
    are intersected."""
    g = maker()
    og = oracle.OracleGraph.from_graph(g)
    hs = [c.upload_host(g.n, g.rowptr, g.col) for c in (ctx, ctx_plain)]
    try:
        for k in ks:
            want_c, want_s = og.checksum(k)
            got = []
            for c, h in zip((ctx, ctx_plain), hs):
                arr, t, s = _list_all(c, h, k, want_c)
                assert (t, s) == (want_c, want_s), (g.name, k)
                got.append((arr, c.stats()))
            if want_c <= 2_000_000:
                exp = np.unique(og.list(k)[0], axis=0)
                for arr, _ in got:
                    u = np.unique(arr, axis=0)
                    assert u.shape[0] == want_c  # no tuple twice
                    assert np.array_equal(u, exp)
            memo_st, plain_st = got[0][1], got[1][1]
            if want_c and dense:
                assert memo_st["memo_hits"] > 0, memo_st
                assert memo_st["word_ops"] < plain_st["word_ops"], (memo_st["word_ops"], plain_st["word_ops"])
    finally:
        for c, h in zip((ctx, ctx_plain), hs):
            c.free(h)


@pytest.mark.parametrize("maker,ks,plex", [
    (lambda: gg.planted_plexes(), range(3, 11), True),
    (lambda: gg.complete_minus(30, [(0, 1), (2, 3), (4, 5), (6, 7)]), range(3, 11), True),  # a 2-plex at the root
    (lambda: gg.complete_minus(30, [(0, 1), (1, 2)]), range(3, 11), False),  # vertex 1 misses two
    (lambda: gg.turan(24, 12), range(3, 11), True),  # K_24 minus a perfect matching
    (lambda: gg.complete_minus(70, [(3, 40), (41, 69)]), range(3, 6), True),  # three words
])
def test_two_plex_closed_form_matches_oracle(maker, ks, plex):
    """The 2-plex early termination (Sec. VII-A): a candidate set whose
    non-edges form a matching is counted by its closed form.  Counts equal
    the oracle's with it on and off, with the memo on and off; with it on,
    frames are counted that way."""
    g = maker()
    og = oracle.OracleGraph.from_graph(g)
    ctxs = [kc.Context(0), kc.Context(0, no_plex=True), kc.Context(0, no_memo=True),
            kc.Context(0, no_memo=True, no_prune=True, no_plex=True)]
    hs = [c.upload_host(g.n, g.rowptr, g.col) for c in ctxs]
    try:
        used = 0
        for k in ks:
            want = og.count(k)[0]
            for i, (c, h) in enumerate(zip(ctxs, hs)):
                assert c.count(h, k) == want, (g.name, k, i)
                st = c.stats()
                if i in (1, 3):
                    assert st["plex_frames"] == 0
                elif i == 0:
                    used += st["plex_frames"]
        assert (used > 0) or not plex, g.name
    finally:
        for c, h in zip(ctxs, hs):
            c.free(h)
            c.close()


@pytest.mark.parametrize("maker,splits", [
    (lambda: gg.chung_lu_planted(n=20000, n_cliques=40, seed=1), False),  # wide roots are dense: memo, no split
    (lambda: gg.rgg_torus(4000, 70.0, seed=6), True),
    (lambda: gg.er_gnp(400, 0.3, 12), True),
])
def test_split_path_matches_oracle(maker, splits):
    """Heavy-root split (one task per first-level branch, drained by a second
    launch): forced on every root of the split tiers, and switched off, in
    count mode with and without the memo and in list mode."""
    g = maker()
    og = oracle.OracleGraph.from_graph(g)
    ctxs = [kc.Context(0, split_threshold=1, memo_min_k=3), kc.Context(0, split_threshold=1, no_memo=True),
            kc.Context(0, split_threshold=0xFFFFFFFF)]
    try:
        hs = [c.upload_host(g.n, g.rowptr, g.col) for c in ctxs]
        heavy = 0
        for k in (5, 6, 7, 8):
            want = og.count(k)[0]
            for c, h in zip(ctxs, hs):
                assert c.count(h, k) == want, (k, c.stats())
            heavy += ctxs[0].stats()["roots_heavy"]
            assert ctxs[2].stats()["roots_heavy"] == 0
        if splits:  # wide sparse roots are split by the wedge test; others may be split by their run time
            assert heavy > 0
        for k in (5, 6):
            want = og.checksum(k)
            for c, h in zip(ctxs, hs):
                assert c.list(h, k, None, 0)[1:] == want, k
        if og.count(5)[0] <= 300000:
            arr, t, s = _list_all(ctxs[0], hs[0], 5, og.count(5)[0])
            assert np.array_equal(np.unique(arr, axis=0), np.unique(og.list(5)[0], axis=0))
    finally:
        for c in ctxs:
            c.close()


@pytest.mark.parametrize("maker", [
    lambda: gg.chung_lu_planted(n=20000, n_cliques=40, seed=1),
    lambda: gg.rgg_torus(4000, 70.0, seed=6),
    lambda: gg.er_gnp(400, 0.3, 12),
    lambda: gg.complete(70),
])
def test_edge_parallel_decomposition_matches_oracle(maker):
    """EdgeParallel as the whole decomposition (Sec. VII-D): every root's
    first-level branches (u, v) are separate tasks of the second launch, in
    every width tier; counts with and without the memo, checksums and the
    listed tuples equal the oracle's.  (A root whose G_u is a 2-plex is
    counted whole by its closed form, so the split invariant is checked with
    that off.)"""
    g = maker()
    og = oracle.OracleGraph.from_graph(g)
    ctxs = [kc.Context(0, decomposition=kc.KC_EDGE_PARALLEL, no_plex=True),
            kc.Context(0, decomposition=kc.KC_EDGE_PARALLEL, no_memo=True, no_plex=True),
            kc.Context(0, decomposition=kc.KC_EDGE_PARALLEL)]
    try:
        hs = [c.upload_host(g.n, g.rowptr, g.col) for c in ctxs]
        for k in (3, 4, 5, 6, 7):
            want = og.count(k)[0]
            for i, (c, h) in enumerate(zip(ctxs, hs)):
                assert c.count(h, k) == want, (k, c.stats())
                st = c.stats()
                if want and i < 2:  # every root that survives pruning was split into its branches
                    assert st["roots_heavy"] == st["roots_total"] - st["roots_pruned"] > 0, st
        for k in (3, 5):
            assert ctxs[0].list(hs[0], k, None, 0)[1:] == og.checksum(k), k
        want4 = og.count(4)[0]
        if want4 <= 300000:
            arr, t, s = _list_all(ctxs[0], hs[0], 4, want4)
            assert (t, s) == og.checksum(4)
            assert np.array_equal(np.unique(arr, axis=0), np.unique(og.list(4)[0], axis=0))
    finally:
        for c in ctxs:
            c.close()
    with pytest.raises(kc.KcError) as e:
        kc.Context(0, decomposition=7)
    assert e.value.status == kc.KC_E_INVALID_ARG


# ------------------------------------------------- peel / orient (a2, a3)
@pytest.mark.parametrize("maker", [
    lambda: gg.er_gnp(3000, 0.004, 7),
    lambda: gg.chung_lu_planted(n=20000, n_cliques=40, seed=1),
    lambda: gg.complete(70),
    lambda: gg.rgg_torus(5000, 30.0, seed=5),
    # two million low-degree vertices: every block's first wave outgrows shared memory and spills
    lambda: gg.er_gnm(2_000_000, 3_000_000, seed=9),
    # a perfect matching on two million vertices: the level-1 scan of every block spills
    lambda: gg.csr_from_pairs(2_000_000, np.arange(0, 2_000_000, 2), np.arange(1, 2_000_000, 2)),
    # a long path: one removal cascade of 50,000 waves
    lambda: gg.csr_from_pairs(100_000, np.arange(99_999), np.arange(1, 100_000)),
])
def test_core_numbers_and_dag(ctx, maker):
    g = maker()
    og = oracle.OracleGraph.from_graph(g)
    h = ctx.upload_host(g.n, g.rowptr, g.col)
    try:
        core, rank, orow, ocol = ctx.export_dag(h)
        info = ctx.info(h)
        # core numbers do not depend on tie-breaking: bit-exact
        assert np.array_equal(core, og.core_numbers())
        assert info["degeneracy"] == og.degeneracy
        # the order is a permutation and a degeneracy order: out-degree <= delta
        assert np.array_equal(np.sort(rank), np.arange(g.n, dtype=np.uint32))
        outdeg = np.diff(orow.astype(np.int64))
        assert outdeg.max(initial=0) == info["max_out_degree"] <= og.degeneracy
        # the DAG holds each undirected edge once, oriented to the higher rank, rows sorted
        assert int(orow[-1]) == og.m
        src = np.repeat(np.arange(g.n, dtype=np.int64), outdeg)
        dst = ocol.astype(np.int64)
        assert np.all(dst > src)
        if dst.size:
            same_row = src[1:] == src[:-1]
            assert np.all(dst[1:][same_row] > dst[:-1][same_row])
        vert = np.empty(g.n, dtype=np.int64)
        vert[rank.astype(np.int64)] = np.arange(g.n)
        a, b = vert[src], vert[dst]
        got = np.sort(np.minimum(a, b) * g.n + np.maximum(a, b))
        ea, eb = gg.edges_of(g)
        want = np.sort(ea.astype(np.int64) * g.n + eb)
        assert np.array_equal(got, want)
        # vertices of lower core come first in the order
        assert np.all(np.diff(core[vert].astype(np.int64)) >= 0)
    finally:
        ctx.free(h)


# -------------------------------------------------------- canonicalisation
def test_canonicalise_raw_rmat(ctx):
    g = gg.rmat(scale=12, edge_factor=16, seed=2)
    assert not g.canonical
    og = oracle.OracleGraph.from_graph(g)
    h = ctx.upload_host(g.n, g.rowptr, g.col, canonicalize=True)
    try:
        info = ctx.info(h)
        assert info["m"] == og.m and info["degeneracy"] == og.degeneracy
        core, rank, orow, ocol = ctx.export_dag(h)
        assert np.array_equal(core, og.core_numbers())
        for k in (3, 4, 5, 6):
            want_c, want_s = og.checksum(k)
            assert ctx.count(h, k) == want_c
            w, t, s = ctx.list(h, k, None, 0)
            assert (t, s) == (want_c, want_s)
    finally:
        ctx.free(h)


def test_canonicalise_hub_rows(ctx):
    """Rows longer than one shared-memory sort tile (4096 keys) with repeats."""
    rng = np.random.default_rng(3)
    n = 9000
    hub = np.zeros(30000, dtype=np.int64)
    other = rng.integers(0, n, 30000)
    extra_a = rng.integers(0, n, 20000)
    extra_b = rng.integers(0, n, 20000)
    g = gg.raw_csr_from_pairs(n, np.concatenate([hub, extra_a, other[:50]]),
                              np.concatenate([other, extra_b, hub[:50]]))
    og = oracle.OracleGraph.from_graph(g)
    h = ctx.upload_host(g.n, g.rowptr, g.col, canonicalize=True)
    try:
        assert ctx.info(h)["m"] == og.m
        core, _, _, _ = ctx.export_dag(h)
        assert np.array_equal(core, og.core_numbers())
        for k in (3, 4):
            assert ctx.list(h, k, None, 0)[1:] == og.checksum(k)
    finally:
        ctx.free(h)


def test_invalid_graphs_rejected(ctx):
    # asymmetric
    rowptr = np.array([0, 1, 1], dtype=np.uint64)
    col = np.array([1], dtype=np.uint32)
    with pytest.raises(kc.KcError) as e:
        ctx.upload_host(2, rowptr, col)
    assert e.value.status == kc.KC_E_INVALID_GRAPH
    # self-loop
    with pytest.raises(kc.KcError):
        ctx.upload_host(1, np.array([0, 1], dtype=np.uint64), np.array([0], dtype=np.uint32))
    # unsorted row
    with pytest.raises(kc.KcError):
        ctx.upload_host(3, np.array([0, 2, 3, 4], dtype=np.uint64), np.array([2, 1, 0, 0], dtype=np.uint32))
    # id out of range, also with canonicalisation
    with pytest.raises(kc.KcError):
        ctx.upload_host(2, np.array([0, 1, 1], dtype=np.uint64), np.array([7], dtype=np.uint32), canonicalize=True)
    # the context stays usable
    g = gg.complete(6)
    h = ctx.upload_host(g.n, g.rowptr, g.col)
    assert ctx.count(h, 3) == 20
    ctx.free(h)


# --------------------------------------------------------- list semantics
def test_list_capacity_and_ranges(ctx):
    g = gg.er_gnp(400, 0.15, 11)
    og = oracle.OracleGraph.from_graph(g)
    want_c, want_s = og.checksum(4)
    torch = _torch()
    h = ctx.upload_host(g.n, g.rowptr, g.col)
    try:
        cap = want_c // 3
        buf = torch.empty(cap * 4, dtype=torch.int32, device="cuda")
        w, t, s = ctx.list(h, 4, buf, cap, allow_capacity=True)
        assert (w, t, s) == (cap, want_c, want_s)
        arr = buf.cpu().numpy().view(np.uint32).reshape(cap, 4)
        full = {tuple(r) for r in og.list(4)[0].tolist()}
        assert len({tuple(r) for r in arr.tolist()}) == cap
        assert all(tuple(r) in full for r in arr.tolist())
        with pytest.raises(kc.KcError) as e:
            ctx.list(h, 4, buf, cap)
        assert e.value.status == kc.KC_E_CAPACITY
        cuts = [0, 1, 57, 200, 201, 399, 400]
        tot, chk = 0, 0
        for lo, hi in zip(cuts, cuts[1:]):
            _, t, s = ctx.list_range(h, 4, lo, hi)
            tot += t
            chk = (chk + s) % (1 << 64)
        assert (tot, chk) == (want_c, want_s)
    finally:
        ctx.free(h)


def test_edge_cases(ctx):
    g = gg.csr_from_pairs(5, np.zeros(0), np.zeros(0))
    h = ctx.upload_host(g.n, g.rowptr, g.col)
    assert [ctx.count(h, k) for k in (1, 2, 3)] == [5, 0, 0]
    assert ctx.list(h, 1, None, 0)[1] == 5
    ctx.free(h)
    g = gg.complete(7)
    h = ctx.upload_host(g.n, g.rowptr, g.col)
    assert ctx.count(h, 7) == 1 and ctx.count(h, 8) == 0
    for bad, code in ((0, kc.KC_E_INVALID_ARG), (kc.KC_MAX_K + 1, kc.KC_E_UNSUPPORTED)):
        with pytest.raises(kc.KcError) as e:
            ctx.count(h, bad)
        assert e.value.status == code
    k1 = ctx.list(h, 1, None, 0)
    assert k1[1] == 7 and k1[2] == sum(oracle.clique_hash([v]) for v in range(7)) % (1 << 64)
    ctx.free(h)
    with pytest.raises(kc.KcError) as e:
        ctx.count(12345, 3)
    assert e.value.status == kc.KC_E_NOT_FOUND


def test_device_pointer_upload(ctx):
    torch = _torch()
    g = gg.er_gnp(500, 0.1, 9)
    og = oracle.OracleGraph.from_graph(g)
    rp = torch.from_numpy(g.rowptr.view(np.int64)).cuda()
    cl = torch.from_numpy(g.col.view(np.int32)).cuda()
    h = ctx.upload_device(g.n, rp, cl)
    try:
        assert ctx.count(h, 4) == og.count(4)[0]
    finally:
        ctx.free(h)


# ------------------------------------------------------- full-size configs
def test_chung_lu_full_size_vs_golden(ctx):
    """Chung-Lu n = 1e6 + 2000 planted cliques: counts for every k the oracle has finished."""
    gold = json.load(open(os.path.join(GOLD, "config_results.json")))
    keys = sorted(k for k in gold if k.startswith("chung_lu_1e6_2000cliques_seed1_k"))
    assert keys
    g = gg.config_chung_lu()
    assert gold[keys[0]]["fingerprint"] == g.fingerprint()
    h = ctx.upload_host(g.n, g.rowptr, g.col)
    try:
        info = ctx.info(h)
        assert info["m"] == gold[keys[0]]["m"] and info["degeneracy"] == gold[keys[0]]["degeneracy"]
        for key in keys:
            k = int(key.rsplit("_k", 1)[1])
            assert ctx.count(h, k) == gold[key]["count"], k
    finally:
        ctx.free(h)


# ------------------------------------------------------ bounded device waits
def test_bounded_wait_gives_up_and_context_stays_usable():
    """A peel whose grid barrier may wait only 1 ns gives up, reports
    KC_E_DEVICE_TIMEOUT and leaves the context usable (no fault, no hang)."""
    g = gg.chung_lu_planted(n=20000, n_cliques=40, seed=1)
    small = gg.complete(9)  # fits one block: its barriers never wait
    with kc.Context(0, spin_limit=1) as c:
        with pytest.raises(kc.KcError) as e:
            c.upload_host(g.n, g.rowptr, g.col)
        assert e.value.status == kc.KC_E_DEVICE_TIMEOUT
        h = c.upload_host(small.n, small.rowptr, small.col)
        assert c.count(h, 4) == oracle.binom(9, 4)
        c.free(h)
    with kc.Context(0) as c:
        h = c.upload_host(g.n, g.rowptr, g.col)
        assert c.count(h, 5) == oracle.OracleGraph.from_graph(g).count(5)[0]
        c.free(h)


_RMAT22 = []


def _rmat22():
    """Config 3's graph, generated once per test session (about a minute)."""
    if not _RMAT22:
        _RMAT22.append(gg.config_rmat())
    return _RMAT22[0]


def test_rmat_scale22_full_size_vs_golden(ctx):
    """R-MAT scale 22 (raw pairs, canonicalised on the device): m, degeneracy,
    the k = 3 and 4 counts and checksums and the k = 5 count against the
    oracle's stored values; k = 4 also as a sum over a partition of root ranges."""
    gold = json.load(open(os.path.join(GOLD, "config_results.json")))
    g = _rmat22()
    assert gold["rmat_22_16_seed2_k3"]["fingerprint"] == g.fingerprint()
    h = ctx.upload_host(g.n, g.rowptr, g.col, canonicalize=True)
    try:
        info = ctx.info(h)
        assert info["m"] == gold["rmat_22_16_seed2_k3"]["m"]
        assert info["degeneracy"] == gold["rmat_22_16_seed2_k3"]["degeneracy"]
        for k in (3, 4):
            want = gold[f"rmat_22_16_seed2_k{k}"]
            assert ctx.count(h, k) == want["count"], k
            assert ctx.list(h, k, None, 0)[1:] == (want["count"], want["checksum"]), k
        # k = 5: 6.9e12 cliques, the oracle's count only (a CPU listing of each is out of reach)
        assert ctx.count(h, 5) == gold["rmat_22_16_seed2_k5"]["count"]
        cuts = [0, g.n // 2, g.n - 200000, g.n - 5000, g.n]
        tot, chk = 0, 0
        for lo, hi in zip(cuts, cuts[1:]):
            _, t, s = ctx.list_range(h, 4, lo, hi)
            tot += t
            chk = (chk + s) % (1 << 64)
        assert (tot, chk) == (gold["rmat_22_16_seed2_k4"]["count"], gold["rmat_22_16_seed2_k4"]["checksum"])
    finally:
        ctx.free(h)


@pytest.mark.parametrize("opts", [{}, {"no_memo": True}, {"no_prune": True}, {"split_threshold": 1},
                                  {"decomposition": kc.KC_EDGE_PARALLEL}, {"memo_min_k": 3}])
def test_rmat_k6_vs_oracle(opts):
    """Config 3's generator (R-MAT, edge factor 16, (0.57, 0.19, 0.19, 0.05),
    seed 2, raw pairs canonicalised on the device) at scale 14, where the
    oracle lists every 6-clique: count, total and checksum of the listing,
    and the listing split into root ranges whose totals add and checksums
    wrap-add to the whole; with the memo, pruning, heavy-root split and
    decomposition toggled.  At scale 16, the default settings: count and
    checksum against the oracle's."""
    gold = json.load(open(os.path.join(GOLD, "config_results.json")))
    c = kc.Context(0, **opts)
    try:
        for scale, list_it in ((14, True), (16, not opts)):
            key = f"rmat_{scale}_16_seed2_k6"
            if key not in gold:
                continue
            want = gold[key]
            g = gg.rmat(scale=scale, edge_factor=16, seed=2)
            assert want["fingerprint"] == g.fingerprint()
            h = c.upload_host(g.n, g.rowptr, g.col, canonicalize=True)
            try:
                assert c.info(h)["degeneracy"] == want["degeneracy"]
                assert c.count(h, 6) == want["count"], (scale, opts)
                if not list_it:
                    continue
                assert c.list(h, 6, None, 0)[1:] == (want["count"], want["checksum"]), (scale, opts)
                if scale == 14:
                    n = g.n
                    cuts = [0, n // 3, n - 3000, n - 800, n - 100, n]
                    tot, chk = 0, 0
                    for lo, hi in zip(cuts, cuts[1:]):
                        _, t, s = c.list_range(h, 6, lo, hi)
                        tot += t
                        chk = (chk + s) % (1 << 64)
                    assert (tot, chk) == (want["count"], want["checksum"]), opts
            finally:
                c.free(h)
    finally:
        c.close()


def _induced(n, rank, orow, ocol, ranks):
    """The subgraph induced by the vertices of the given ranks, in original ids
    (on all n ids; the others are isolated)."""
    vert = np.empty(n, dtype=np.int64)
    vert[rank.astype(np.int64)] = np.arange(n, dtype=np.int64)
    orow = orow.astype(np.int64)
    ranks = np.unique(np.asarray(ranks, dtype=np.int64))
    lens = orow[ranks + 1] - orow[ranks]
    rows = np.repeat(ranks, lens)
    first = np.repeat(orow[ranks] - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
    cols = ocol[first + np.arange(rows.size)].astype(np.int64)
    sel = np.isin(cols, ranks)
    return gg.csr_from_pairs(n, vert[rows[sel]], vert[cols[sel]])


def test_rmat_scale22_k6_dense_core():
    """Config 3 at full size, k = 6 (listing with checksum).  Listing all of its
    3.3e14 6-cliques costs as many hash chains, so the full-size check takes
    the innermost core: out-neighbours have higher ranks, so
    kc_list_range(n - X, n) lists exactly the 6-cliques of the subgraph that
    the top X ranks of the DAG's order induce.  That subgraph is listed by the
    oracle (total + checksum) and counted and listed in separate contexts with
    the memo, pruning, heavy-root split, 2-plex closed form and the
    decomposition toggled; the range also splits into sub-ranges whose totals
    add and checksums wrap-add."""
    g = _rmat22()
    k = 6
    c = kc.Context(0)
    try:
        h = c.upload_host(g.n, g.rowptr, g.col, canonicalize=True)
        n = c.info(h)["n"]
        _, rank, orow, ocol = c.export_dag(h)

        def top(x):
            return c.list_range(h, k, n - x, n)

        x = 16
        while x * 2 <= n and top(x * 2)[1] <= (1 << 24):
            x *= 2
        _, t_top, s_top = top(x)
        assert t_top > 0
        cuts = [n - x, n - x // 2, n - x // 8, n]
        tot, chk = 0, 0
        for lo, hi in zip(cuts, cuts[1:]):
            _, t, s = c.list_range(h, k, lo, hi)
            tot += t
            chk = (chk + s) % (1 << 64)
        assert (tot, chk) == (t_top, s_top)
        c.free(h)
    finally:
        c.close()
    print(f"config 3, k = 6: the top {x} ranks hold {t_top} cliques (checksum {s_top:#x})")
    core = _induced(n, rank, orow, ocol, np.arange(n - x, n))
    assert oracle.OracleGraph.from_graph(core).checksum(k) == (t_top, s_top)
    for opts in ({}, {"no_memo": True}, {"memo_min_k": 3}, {"no_prune": True}, {"split_threshold": 1},
                 {"no_plex": True}, {"decomposition": kc.KC_EDGE_PARALLEL}):
        cv = kc.Context(0, **opts)
        try:
            hv = cv.upload_host(core.n, core.rowptr, core.col)
            assert cv.count(hv, k) == t_top, opts
            assert cv.list(hv, k, None, 0)[1:] == (t_top, s_top), opts
            cv.free(hv)
        finally:
            cv.close()
