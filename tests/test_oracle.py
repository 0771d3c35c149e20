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


@pytest.mark.parametrize("n,p", [(12, 3), (16, 8), (25, 5), (9, 0)])
def test_complete_minus_matching_closed_form(n, p):
    """K_n without a matching of p pairs (a 2-plex): a k-clique takes from
    each missing pair none or one of its two vertices, and any of the n - 2p
    others, so there are sum over j of C(p, j) 2^j C(n - 2p, k - j)."""
    from math import comb

    og = oracle.OracleGraph.from_graph(gg.complete_minus(n, [(2 * t, 2 * t + 1) for t in range(p)]))
    for k in range(1, n + 1):
        want = sum(comb(p, j) * 2 ** j * comb(n - 2 * p, k - j) for j in range(min(p, k) + 1))
        assert og.count(k)[0] == want, (n, p, k)


def _plex2_test(S, adj):
    """The device's 2-plex test on a vertex set S (ascending): p = non-edges;
    reject when 2p > |S|; each vertex v may miss at most one vertex above it
    (M_v); the vertices with a missing one and the missing ones together must
    number 2p (all endpoints distinct)."""
    m = len(S)
    e = sum(1 for i in range(m) for j in range(i + 1, m) if S[j] in adj[S[i]])
    p = m * (m - 1) // 2 - e
    if 2 * p > m:
        return False
    touched = set()
    for i, v in enumerate(S):
        miss = [w for w in S[i + 1:] if w not in adj[v]]
        if len(miss) > 1:
            return False
        if miss:
            touched.add(v)
            touched.add(miss[0])
    return len(touched) == 2 * p


@pytest.mark.parametrize("seed", range(4))
def test_plex2_test_accepts_exactly_matchings(seed):
    """The device counts a candidate set in closed form when its test accepts
    it; the test accepts exactly the sets whose non-edges form a matching
    (every vertex misses at most one other: a 2-plex), checked against that
    definition on near-complete random graphs and all their small subsets."""
    rng = np.random.default_rng(seed)
    n = 9
    for _ in range(30):
        miss = float(rng.choice([0.05, 0.15, 0.3]))
        adj = {v: set() for v in range(n)}
        for a in range(n):
            for b in range(a + 1, n):
                if rng.random() >= miss:
                    adj[a].add(b)
                    adj[b].add(a)
        for m in range(2, n + 1):
            for S in itertools.combinations(range(n), m):
                deg_miss = [sum(1 for w in S if w != v and w not in adj[v]) for v in S]
                assert _plex2_test(list(S), adj) == (max(deg_miss) <= 1), (S, deg_miss)


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


# Published SplitMix64 outputs (Steele, Lea & Flood, OOPSLA 2014; Vigna's
# public-domain splitmix64.c): the state x advances by 0x9E3779B97F4A7C15 and
# each output is the finaliser of the new state.  Seed 0 gives the sequence
# quoted with the generator; the other two are test vectors produced with
# the reference splitmix64.c for seeds 1234567 and 1477776061723855037.
SPLITMIX64_GAMMA = 0x9E3779B97F4A7C15
SPLITMIX64_PUBLISHED = {
    0: [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC, 0x1B39896A51A8749B],
    1234567: [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
              16408922859458223821],
    1477776061723855037: [1985237415132408290, 2979275885539914483, 13511426838097143398, 8488337342461049707,
                          15141737807933549159, 17093170987380407015],
}


def test_mix64_is_the_published_splitmix64_finaliser():
    """The checksum's mixer reproduces published SplitMix64 outputs (a wrong
    shift, constant or operator in the finaliser changes every one)."""
    for seed, outs in SPLITMIX64_PUBLISHED.items():
        x = seed
        for want in outs:
            x = (x + SPLITMIX64_GAMMA) % (1 << 64)
            assert oracle.mix64(x) == want, (seed, hex(want))


def test_clique_hash_worked_example():
    """The hash of one clique, worked step by step outside the oracle.

    The empty tuple (k = 0) hashes to mix(0x9E3779B97F4A7C15), the first
    SplitMix64 output for seed 0: 0xE220A8397B1DCDAF.

    The clique {1, 2} (k = 2): h0 = mix(0x9E3779B97F4A7C15 ^ 2), then
    h1 = mix(h0 ^ 1), then h2 = mix(h1 ^ 2), where mix(z) is
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
    z *= 0x94D049BB133111EB; z ^= z >> 31 (mod 2^64):

        mix(0x9E3779B97F4A7C17):  z ^ z>>30 = 0x9E3779BB07979AF2
                                  * c1      = 0xEE18B4F591B172E2
                                  ^ >>27    = 0xEE18B4E852A7EC50
                                  * c2      = 0x975835DF32273D70
                                  ^ >>31    = 0x975835DE1C9756CE = h0
        mix(h0 ^ 1 = 0x975835DE1C9756CF):   ... 0xF2826F98653E9E57 = h1
          (0x975835DC41F781B7, 0x3192C1B89DE1703F, 0x3192C1BEAFB9472C,
           0xF2826F99803A4164)
        mix(h1 ^ 2 = 0xF2826F98653E9E55):   ... 0x0C0266261F3A0C53 = h2
          (0xF2826F9BAF372034, 0x1E3222004CF4C994, 0x1E3222038AB0899D,
           0x0C026626073EC01F)
    """
    assert oracle.clique_hash([]) == 0xE220A8397B1DCDAF
    assert oracle.mix64(0x9E3779B97F4A7C17) == 0x975835DE1C9756CE
    assert oracle.mix64(0x975835DE1C9756CF) == 0xF2826F98653E9E57
    assert oracle.mix64(0xF2826F98653E9E55) == 0x0C0266261F3A0C53
    assert oracle.clique_hash([1, 2]) == 0x0C0266261F3A0C53
    # a graph with one k-clique has that clique's hash as its checksum
    og = oracle.OracleGraph.from_graph(gg.complete(3))
    assert og.checksum(3)[1] == oracle.clique_hash([0, 1, 2])
    # the single edge {1, 2} of a 3-vertex graph
    og2 = oracle.OracleGraph(3, np.array([0, 0, 1, 2], dtype=np.uint64), np.array([2, 1], dtype=np.uint32))
    assert og2.checksum(2) == (1, 0x0C0266261F3A0C53)


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


def _alg5_by_rounds(order, out, rcap):
    """Algorithm 5 in the round form the device uses: B_1 is every vertex;
    round t moves each vertex's increment point p to the largest out-neighbour
    in B_t below p, and the vertices that found one form B_{t+1}.  Returns r
    capped at rcap, and the capped r of a root adjacent to every vertex."""
    pos = {v: i for i, v in enumerate(order)}
    p = {u: len(order) for u in order}
    r = {u: 1 for u in order}
    b = set(order)
    q, root = len(order), 1
    for t in range(1, rcap):
        below = [pos[v] for v in b if pos[v] < q]
        q = max(below) if below else -1
        if q >= 0:
            root = t + 1
        nb = set()
        for u in order:
            c = [pos[w] for w in out[u] if w in b and pos[w] < p[u]]
            p[u] = max(c) if c else 0
            if c:
                r[u] = t + 1
                nb.add(u)
        b = nb
    return r, root


@pytest.mark.parametrize("seed", range(6))
def test_alg5_round_form_equals_vertex_order(seed):
    """The device computes Algorithm 5 by rounds over the sets B_t of
    vertices with r >= t (all rows at once) instead of vertex by vertex.  On
    random DAGs, for every cap, the two give the same capped r values, and the
    same r for a root adjacent to every vertex (the root's own test)."""
    rng = np.random.default_rng(seed)
    for _ in range(40):
        n = int(rng.integers(1, 40))
        dens = float(rng.random())
        order = [int(x) for x in rng.permutation(n)]
        out = {u: set() for u in order}
        for i in range(n):
            for j in range(i + 1, n):
                if rng.random() < dens:
                    out[order[i]].add(order[j])
        r = oracle.soft_embedding_r(order, out)
        apex = max(order) + 1  # a root before every vertex, adjacent to all
        r_root = oracle.soft_embedding_r([apex] + order, {**out, apex: set(order)})[apex]
        for rcap in (2, 3, 5, 9, 64):
            got, root = _alg5_by_rounds(order, out, rcap)
            assert got == {u: min(r[u], rcap) for u in order}
            assert root == min(r_root, rcap)


# -------------------------------------------------------- input determinism
def test_generator_fingerprints():
    """The seeded generators give the same bytes on every host."""
    want = json.load(open(os.path.join(GOLD, "graph_fingerprints.json")))
    assert gg.config_er_small().fingerprint() == want["er_2000_0.01_seed0"]
    assert gg.chung_lu_planted(n=20000, n_cliques=40, seed=1).fingerprint() == want["chung_lu_20000_40_seed1"]
    assert gg.rmat(scale=12, edge_factor=16, seed=2).fingerprint() == want["rmat_12_16_seed2"]
    assert gg.rgg_torus(3000, 25.0, seed=3).fingerprint() == want["rgg_3000_25_seed3"]
    assert gg.er_gnm(5000, 40000, seed=4).fingerprint() == want["er_gnm_5000_40000_seed4"]
