"""Pins for the oracle (CPU only).

The oracle is trusted only after it is tied to things other than itself:
values the paper prints for its worked example, closed forms, brute force on
tiny graphs and invariants.  Each group below names what it pins.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_2502_00317_gb300 import graphgen as gg

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _fig2():
    d = json.load(open(os.path.join(GOLD, "fig2_dag.json")))
    out = {int(u): set(v) for u, v in d["out"].items()}
    a = [u for u in out for v in out[u]]
    b = [v for u in out for v in out[u]]
    return d, out, gg.csr_from_pairs(d["n"], np.array(a), np.array(b))


# ------------------------------------------------- worked example (Fig. 2)
def test_fig2_four_cliques_match_paper():
    d, out, g = _fig2()
    og = oracle.OracleGraph.from_graph(g)
    assert og.m == 27
    assert og.count(4)[0] == d["k4_count"]
    cl, total, _ = og.list(4)
    assert total == d["k4_count"]
    got = {tuple(r) for r in cl.tolist()}
    for c in d["k4_first_cliques"]:
        assert tuple(c) in got


def test_fig2_counts_all_k_match_brute_force():
    d, out, g = _fig2()
    og = oracle.OracleGraph.from_graph(g)
    adj = oracle.adjacency_sets(g.n, g.rowptr, g.col)
    for k in range(1, 8):
        bf = oracle.brute_force_cliques(g.n, adj, k)
        assert og.count(k)[0] == len(bf), k
        c, s = og.checksum(k)
        assert c == len(bf)
        assert s == sum(oracle.clique_hash(t) for t in bf) % (1 << 64)


def test_fig2_example3_and_table2():
    """The rebuilt DAG reproduces Example 3 and every row of Table 2."""
    d, out, g = _fig2()
    adj = oracle.adjacency_sets(g.n, g.rowptr, g.col)
    sub = d["example3_subgraph"]
    tri = [t for t in itertools.combinations(sub, 3) if all(b in adj[a] for a, b in itertools.combinations(t, 2))]
    assert [list(t) for t in tri] == d["example3_three_cliques"]
    umin = min(sub)
    assert [list(t) for t in tri if umin in t] == d["example3_inclusive"]
    assert [list(t) for t in tri if umin not in t] == d["example3_exclusive"]
    for row in d["table2"]:
        for c in row["cliques"]:
            common = set(range(g.n))
            for u in c:
                common &= out[u]
            assert sorted(common, reverse=True) == row["string"], (c, row)
    # the trie (prefix tree) over the ten strings has 14 nodes, root included
    prefixes = {()}
    for row in d["table2"]:
        s = tuple(row["string"])
        for i in range(1, len(s) + 1):
            prefixes.add(s[:i])
    assert len(prefixes) == d["table2_trie_nodes"]


def test_fig2_order_is_a_degeneracy_order():
    d, out, g = _fig2()
    og = oracle.OracleGraph.from_graph(g)
    assert og.degeneracy == 5
    assert og.ranks().tolist() == list(range(9))


# ----------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [1, 2, 5, 12, 33, 40])
def test_complete_graph_binomial(n):
    og = oracle.OracleGraph.from_graph(gg.complete(n))
    for k in range(1, min(n, 8) + 2):
        assert og.count(k)[0] == oracle.binom(n, k), (n, k)
    assert og.degeneracy == max(n - 1, 0)


@pytest.mark.parametrize("n,r", [(10, 3), (17, 4), (24, 5), (30, 7), (12, 12)])
def test_turan_elementary_symmetric(n, r):
    og = oracle.OracleGraph.from_graph(gg.turan(n, r))
    sizes = [len(range(i, n, r)) for i in range(r)]
    for k in range(1, r + 3):
        assert og.count(k)[0] == oracle.elementary_symmetric(sizes, k), (n, r, k)


def test_turan_theorem_edge_bound():
    """T(n, r) is the largest graph with no (r+1)-clique (Turan, Sec. IV)."""
    for n, r in [(20, 3), (21, 4), (30, 6)]:
        og = oracle.OracleGraph.from_graph(gg.turan(n, r))
        assert og.count(r + 1)[0] == 0
        assert og.m <= (r - 1) / r * n * n / 2


def test_disjoint_cliques_sum_of_binomials():
    sizes = [3, 7, 11, 20, 1, 5]
    og = oracle.OracleGraph.from_graph(gg.disjoint_cliques(sizes))
    for k in range(1, 10):
        assert og.count(k)[0] == sum(oracle.binom(s, k) for s in sizes)


# ------------------------------------------------------------ brute force
@pytest.mark.parametrize("seed", range(12))
def test_random_tiny_graphs_brute_force(seed):
    n = 8 + seed
    p = [0.2, 0.4, 0.6, 0.8][seed % 4]
    g = gg.er_gnp(n, p, seed)
    og = oracle.OracleGraph.from_graph(g)
    adj = oracle.adjacency_sets(g.n, g.rowptr, g.col)
    for k in range(1, 8):
        bf = oracle.brute_force_cliques(g.n, adj, k)
        assert og.count(k)[0] == len(bf)
        c, s, pv = og.checksum(k, per_vertex=True)
        assert c == len(bf)
        assert s == sum(oracle.clique_hash(t) for t in bf) % (1 << 64)
        assert int(pv.sum()) == k * c
        expect_pv = np.zeros(n, dtype=np.int64)
        for t in bf:
            expect_pv[list(t)] += 1
        assert pv.astype(np.int64).tolist() == expect_pv.tolist()
        cl, total, s2 = og.list(k)
        assert sorted(map(tuple, cl.tolist())) == bf
        assert s2 == s


def test_checksum_sees_a_duplicate():
    g = gg.complete(6)
    og = oracle.OracleGraph.from_graph(g)
    c, s = og.checksum(3)
    h = oracle.clique_hash([0, 1, 2])
    assert (s + h) % (1 << 64) != s  # a repeated clique changes the sum


def test_order_invariance_under_relabelling():
    g = gg.er_gnp(60, 0.3, 5)
    og = oracle.OracleGraph.from_graph(g)
    perm = np.random.default_rng(0).permutation(g.n)
    src = np.repeat(np.arange(g.n), np.diff(g.rowptr).astype(np.int64))
    h = gg.csr_from_pairs(g.n, perm[src], perm[g.col.astype(np.int64)])
    oh = oracle.OracleGraph.from_graph(h)
    for k in range(3, 7):
        assert og.count(k)[0] == oh.count(k)[0]
        cl, _, _ = og.list(k)
        mapped = np.sort(perm[cl.astype(np.int64)], axis=1)
        want = sum(oracle.clique_hash(t) for t in mapped) % (1 << 64)
        assert oh.checksum(k)[1] == want


def test_canonicalisation_of_raw_input():
    """Self-loops, repeats and one-directional entries are cleaned (Sec. II-A: simple graphs)."""
    g = gg.er_gnp(40, 0.35, 7)
    src, dst = gg.edges_of(g)
    rng = np.random.default_rng(1)
    rs = np.concatenate([src, dst[:10], src[:30], np.arange(5)])
    rd = np.concatenate([dst, src[:10], dst[:30], np.arange(5)])
    raw = gg.raw_csr_from_pairs(g.n, rs, rd)
    og, orw = oracle.OracleGraph.from_graph(g), oracle.OracleGraph.from_graph(raw)
    assert og.m == orw.m
    for k in range(1, 7):
        assert og.checksum(k) == orw.checksum(k)


def test_bad_ids_rejected():
    rowptr = np.array([0, 1, 1], dtype=np.uint64)
    col = np.array([5], dtype=np.uint32)
    with pytest.raises(ValueError):
        oracle.OracleGraph(2, rowptr, col)


def test_edge_cases():
    g = gg.csr_from_pairs(5, np.zeros(0), np.zeros(0))
    og = oracle.OracleGraph.from_graph(g)
    assert og.count(1)[0] == 5 and og.count(2)[0] == 0 and og.count(3)[0] == 0
    og = oracle.OracleGraph.from_graph(gg.complete(7))
    assert og.count(8)[0] == 0
    assert og.count(7)[0] == 1


def test_root_ranges_partition_the_count():
    g = gg.er_gnp(200, 0.15, 3)
    og = oracle.OracleGraph.from_graph(g)
    total = og.checksum(4)
    cuts = [0, 17, 90, 91, 200]
    c = s = 0
    for lo, hi in zip(cuts, cuts[1:]):
        a, b = og.checksum(4, root_lo=lo, root_hi=hi)
        c += a
        s = (s + b) % (1 << 64)
    assert (c, s) == total


# ----------------------------------------------------- degeneracy / cores
def _cores_by_definition(n, adj):
    """core[v] = largest c such that v lies in a subgraph of minimum degree >= c."""
    core = [0] * n
    for c in range(1, n):
        alive = set(range(n))
        changed = True
        while changed:
            changed = False
            for v in list(alive):
                if len(adj[v] & alive) < c:
                    alive.discard(v)
                    changed = True
        if not alive:
            break
        for v in alive:
            core[v] = c
    return core


@pytest.mark.parametrize("seed", range(6))
def test_core_numbers_match_definition(seed):
    g = gg.er_gnp(40, 0.1 + 0.1 * seed, seed)
    og = oracle.OracleGraph.from_graph(g)
    adj = oracle.adjacency_sets(g.n, g.rowptr, g.col)
    assert og.core_numbers().tolist() == _cores_by_definition(g.n, adj)
    assert og.max_out_degree <= og.degeneracy


# ------------------------------------------------ Algorithm 5 (Sec. V)
def _is_soft_embedding(children, f, dag_out, pos):
    for v, ch in children.items():
        for c in ch:
            if f[c] not in dag_out.get(f[v], set()):
                return False
        for a in ch:
            for b in ch:
                if len(children[a]) < len(children[b]) and not pos[f[a]] > pos[f[b]]:
                    return False
    return True


def test_example5_soft_embeddings():
    d = json.load(open(os.path.join(GOLD, "example5_embeddings.json")))
    children = {int(k): v for k, v in d["tree_children"].items()}
    dag_out = {}
    for a, b in d["dag_edges"]:
        dag_out.setdefault(a, set()).add(b)
    verts = sorted({x for e in d["dag_edges"] for x in e})
    pos = {v: i for i, v in enumerate(verts)}
    for name in ("f", "g"):
        f = {int(k): v for k, v in d[name].items()}
        assert _is_soft_embedding(children, f, dag_out, pos), name
    img = sorted(set(d["f"].values()))
    assert img == d["f_image_is_4_clique"]
    out = {v: dag_out.get(v, set()) for v in verts}
    assert oracle.max_tree_embedding(verts, out, 1) >= 4
    assert oracle.soft_embedding_r(verts, out)[1] >= 4


def test_fig2_restricted_r_values():
    d, out, g = _fig2()
    order = list(range(9))
    r = [oracle.restricted_root_r(order, out, u) for u in order]
    # Lemma 1 + exactness on this DAG: r equals the largest clique with u as minimum
    adj = oracle.adjacency_sets(g.n, g.rowptr, g.col)
    best = []
    for u in order:
        b = 1
        for k in range(2, 7):
            if any(min(t) == u for t in oracle.brute_force_cliques(g.n, adj, k)):
                b = k
        best.append(b)
    assert r == best == [4, 4, 4, 4, 5, 4, 3, 2, 1]


def _random_dag(n, p, seed):
    rng = np.random.default_rng(seed)
    out = {u: set() for u in range(n)}
    for u in range(n):
        for v in range(u + 1, n):
            if rng.random() < p:
                out[u].add(v)
    return list(range(n)), out


@pytest.mark.parametrize("seed", range(25))
def test_theorem2_alg5_is_max_tree_embedding(seed):
    order, out = _random_dag(7 + seed % 5, [0.3, 0.5, 0.7, 0.9][seed % 4], seed)
    r = oracle.soft_embedding_r(order, out)
    for u in order:
        assert r[u] == oracle.max_tree_embedding(order, out, u), (seed, u)


@pytest.mark.parametrize("seed", range(12))
def test_lemma1_r_bounds_cliques(seed):
    order, out = _random_dag(9, [0.4, 0.6, 0.8][seed % 3], 100 + seed)
    adj = [set() for _ in order]
    for u in order:
        for v in out[u]:
            adj[u].add(v)
            adj[v].add(u)
    for u in order:
        ru = oracle.restricted_root_r(order, out, u)
        big = 1
        for k in range(2, 10):
            if any(min(t) == u for t in oracle.brute_force_cliques(len(order), adj, k)):
                big = k
        assert ru >= big


def test_alg5_complete_dag():
    """On K_n oriented by any order, the vertex with j out-neighbours has r = j + 1."""
    n = 9
    order = list(range(n))
    out = {u: set(range(u + 1, n)) for u in order}
    r = oracle.soft_embedding_r(order, out)
    for u in order:
        assert r[u] == (n - 1 - u) + 1


def test_alg5_plants_a_mistake():
    """A flipped comparison (r(u) < r(w) instead of <=) breaks the K_n pin."""
    n = 6
    order = list(range(n))
    out = {u: set(range(u + 1, n)) for u in order}
    r = {}
    for u in reversed(order):
        ru = 1
        for w in sorted(out[u], reverse=True):
            if ru < r[w]:
                ru += 1
        r[u] = ru
    assert any(r[u] != (n - 1 - u) + 1 for u in order)


# -------------------------------------------------------- input determinism
def test_generator_fingerprints():
    """The seeded generators give the same bytes on every host."""
    want = json.load(open(os.path.join(GOLD, "graph_fingerprints.json")))
    assert gg.config_er_small().fingerprint() == want["er_2000_0.01_seed0"]
    assert gg.chung_lu_planted(n=20000, n_cliques=40, seed=1).fingerprint() == want["chung_lu_20000_40_seed1"]
    assert gg.rmat(scale=12, edge_factor=16, seed=2).fingerprint() == want["rmat_12_16_seed2"]
    assert gg.rgg_torus(3000, 25.0, seed=3).fingerprint() == want["rgg_3000_25_seed3"]
    assert gg.er_gnm(5000, 40000, seed=4).fingerprint() == want["er_gnm_5000_40000_seed4"]
