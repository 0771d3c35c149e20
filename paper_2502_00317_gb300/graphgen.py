"""Seeded synthetic graph generators (inputs only).

This module produces the graphs that both the CUDA path and the CPU oracle
consume.  It holds none of the k-clique method's arithmetic: no ordering, no
orientation, no intersection, no counting.  Every generator is a pure function
of its seed.

Cross-platform determinism.  The same seed must give the same graph on an
x86_64 host and on an aarch64 host with a different numpy build.  So:

* random bits come only from ``PCG64(SeedSequence([seed, tag])).random_raw``
  (the raw 64-bit PCG64 stream, which numpy keeps stable across versions and
  platforms); no ``Generator`` distribution method is used;
* bits are mapped to values with integer operations and single IEEE-754
  operations (+, -, *, floor, sqrt), all correctly rounded on every platform;
* no transcendental function (pow, log, exp) is evaluated per sample.  The two
  constants that need an 11th root are found by exact bisection over floats
  with ``fractions.Fraction``.

A graph is returned as CSR: ``rowptr`` uint64[n+1] and ``col`` uint32[nnz].
Generators of simple graphs return the canonical form (symmetric, no
self-loops, no duplicates, each row sorted ascending).  ``rmat`` returns the
raw sampled pairs (directed, with self-loops and duplicates) on purpose: the
consumer has to canonicalise them.
"""
from __future__ import annotations

import dataclasses
import hashlib
from fractions import Fraction

import numpy as np

U64 = np.uint64


@dataclasses.dataclass
class Graph:
    """A CSR graph. ``canonical`` is True when the CSR is simple and symmetric."""

    n: int
    rowptr: np.ndarray  # uint64 [n+1]
    col: np.ndarray  # uint32 [rowptr[n]]
    canonical: bool
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def fingerprint(self) -> str:
        """SHA-256 of (n, rowptr, col); used to check that two hosts generated the same input."""
        h = hashlib.sha256()
        h.update(np.uint64(self.n).tobytes())
        h.update(np.ascontiguousarray(self.rowptr, dtype=np.uint64).tobytes())
        h.update(np.ascontiguousarray(self.col, dtype=np.uint32).tobytes())
        return h.hexdigest()


# ---------------------------------------------------------------- random bits
def _stream(seed: int, tag: int) -> np.random.PCG64:
    return np.random.PCG64(np.random.SeedSequence([int(seed), int(tag)]))


def _raw(bg: np.random.PCG64, size: int) -> np.ndarray:
    return bg.random_raw(int(size)).astype(np.uint64, copy=False)


def _u01(raw: np.ndarray) -> np.ndarray:
    """Top 53 bits as a float64 in [0, 1); exact."""
    return (raw >> U64(11)).astype(np.float64) * (2.0 ** -53)


def _bounded(raw: np.ndarray, m: int) -> np.ndarray:
    """Integer in [0, m) from the top 32 bits (multiply-shift), m < 2**32."""
    assert 0 < m < 2 ** 32
    return (((raw >> U64(32)) * U64(m)) >> U64(32)).astype(np.int64)


def _random_permutation(seed: int, tag: int, n: int) -> np.ndarray:
    """A uniformly random permutation of range(n) (argsort of random keys)."""
    keys = _raw(_stream(seed, tag), n)
    return np.argsort(keys, kind="stable").astype(np.int64)


def _float_root(v: int, e: int) -> float:
    """Largest float y with y**e <= v, by exact bisection (platform independent)."""
    lo, hi = 0.0, float(max(2, v))
    target = Fraction(v)
    for _ in range(2000):
        mid = (lo + hi) / 2.0
        if mid == lo or mid == hi:
            break
        if Fraction(mid) ** e <= target:
            lo = mid
        else:
            hi = mid
    return lo


# ------------------------------------------------------------- CSR assembly
def csr_from_pairs(n: int, a: np.ndarray, b: np.ndarray) -> Graph:
    """Simple undirected CSR from an undirected pair list (input assembly).

    Drops pairs with a == b and repeated pairs, stores both directions and
    sorts each row.  This is how a generator states its output graph; the
    CUDA path and the oracle each canonicalise their input independently.
    """
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    keep = a != b
    a, b = a[keep], b[keep]
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    und = np.unique((lo << U64(32)) | hi)
    lo = und >> U64(32)
    hi = und & U64(0xFFFFFFFF)
    keys = np.concatenate([(lo << U64(32)) | hi, (hi << U64(32)) | lo])
    keys.sort(kind="stable")
    src = (keys >> U64(32)).astype(np.int64)
    col = (keys & U64(0xFFFFFFFF)).astype(np.uint32)
    counts = np.bincount(src, minlength=n).astype(np.uint64)
    rowptr = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(counts, out=rowptr[1:])
    return Graph(n=n, rowptr=rowptr, col=col, canonical=True)


def raw_csr_from_pairs(n: int, src: np.ndarray, dst: np.ndarray) -> Graph:
    """Directed CSR of sampled pairs, kept as drawn (self-loops, duplicates,
    no symmetry); rows are grouped by source, entries in draw order."""
    src = np.asarray(src, dtype=np.int64)
    order = np.argsort(src, kind="stable")
    col = np.asarray(dst, dtype=np.uint32)[order]
    counts = np.bincount(src, minlength=n).astype(np.uint64)
    rowptr = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(counts, out=rowptr[1:])
    return Graph(n=n, rowptr=rowptr, col=col, canonical=False)


def edges_of(g: Graph) -> tuple[np.ndarray, np.ndarray]:
    """Undirected edge list (u < v) of a canonical graph."""
    assert g.canonical
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr).astype(np.int64))
    dst = g.col.astype(np.int64)
    m = src < dst
    return src[m], dst[m]


# ----------------------------------------------------------------- families
def complete(n: int) -> Graph:
    i, j = np.triu_indices(n, 1)
    g = csr_from_pairs(n, i, j)
    g.name = f"K{n}"
    return g


def turan(n: int, r: int) -> Graph:
    """Turan graph T(n, r): r near-equal parts, every cross-part pair joined."""
    part = np.arange(n) % r
    i, j = np.triu_indices(n, 1)
    m = part[i] != part[j]
    g = csr_from_pairs(n, i[m], j[m])
    g.name = f"T({n},{r})"
    return g


def disjoint_cliques(sizes) -> Graph:
    sizes = [int(s) for s in sizes]
    a, b, base = [], [], 0
    for s in sizes:
        i, j = np.triu_indices(s, 1)
        a.append(i + base)
        b.append(j + base)
        base += s
    g = csr_from_pairs(base, np.concatenate(a) if a else np.zeros(0), np.concatenate(b) if b else np.zeros(0))
    g.name = f"cliques{sizes}"
    return g


def complete_minus(n: int, missing) -> Graph:
    """K_n without the listed vertex pairs (a matching of them makes a 2-plex)."""
    gone = {(min(a, b), max(a, b)) for a, b in missing}
    i, j = np.triu_indices(n, 1)
    keep = np.array([(int(x), int(y)) not in gone for x, y in zip(i, j)], dtype=bool)
    g = csr_from_pairs(n, i[keep], j[keep])
    g.name = f"K{n}-{sorted(gone)}"
    return g


def planted_plexes(n: int = 6000, p: float = 0.002, n_sets: int = 24, smin: int = 12, smax: int = 26,
                   seed: int = 9) -> Graph:
    """Sparse G(n, p) background plus planted near-cliques on random vertex
    sets: each is complete minus some vertex pairs.  Set i removes a random
    matching of up to s/2 pairs (a 2-plex) when i % 3 != 2, and otherwise a
    matching plus one extra pair that shares a vertex with it (not a 2-plex).
    Ids are randomly permuted."""
    bg = er_gnp(n, p, seed)
    a0, b0 = edges_of(bg)
    cg = _stream(seed, 11)
    pa, pb = [a0], [b0]
    for idx in range(n_sets):
        s = smin + int(_bounded(_raw(cg, 1), smax - smin + 1)[0])
        order = np.argsort(_raw(cg, n), kind="stable")[:s]
        mem = order.astype(np.int64)
        pairs = int(_bounded(_raw(cg, 1), s // 2 + 1)[0])
        gone = {(int(mem[2 * t]), int(mem[2 * t + 1])) for t in range(pairs)}
        if idx % 3 == 2 and s >= 3:
            gone.add((int(mem[0]), int(mem[2])))
        i, j = np.triu_indices(s, 1)
        keep = np.array([(int(mem[x]), int(mem[y])) not in gone and (int(mem[y]), int(mem[x])) not in gone
                         for x, y in zip(i, j)], dtype=bool)
        pa.append(mem[i][keep])
        pb.append(mem[j][keep])
    perm = _random_permutation(seed, 12, n)
    a = perm[np.concatenate(pa)]
    b = perm[np.concatenate(pb)]
    g = csr_from_pairs(n, a, b)
    g.name = f"plexes(n={n},sets={n_sets},seed={seed})"
    return g


def er_gnp(n: int, p: float, seed: int) -> Graph:
    """Erdos-Renyi G(n, p): each pair i < j drawn independently.

    One raw 64-bit draw per pair in row-major (i, j>i) order; the pair is an
    edge iff draw < floor(p * 2**64).  O(n^2) draws: meant for n up to ~10^4.
    """
    thr = U64(min(int(p * 2.0 ** 64), 2 ** 64 - 1))
    i, j = np.triu_indices(n, 1)
    raw = _raw(_stream(seed, 1), i.size)
    m = raw < thr
    g = csr_from_pairs(n, i[m], j[m])
    g.name = f"ER(n={n},p={p},seed={seed})"
    return g


def er_gnm(n: int, m: int, seed: int) -> Graph:
    """Erdos-Renyi G(n, M): M distinct pairs drawn uniformly (rejecting repeats)."""
    bg = _stream(seed, 2)
    have = np.zeros(0, dtype=np.uint64)
    while have.size < m:
        need = m - have.size
        raw = _raw(bg, 2 * need + 16)
        a = _bounded(raw[0::2], n).astype(np.uint64)
        b = _bounded(raw[1::2], n).astype(np.uint64)
        k = a != b
        lo, hi = np.minimum(a[k], b[k]), np.maximum(a[k], b[k])
        keys = (lo << U64(32)) | hi
        # keep first occurrences in draw order, then the first `need` new ones
        _, first = np.unique(keys, return_index=True)
        keys = keys[np.sort(first)]
        keys = keys[~np.isin(keys, have)][:need]
        have = np.concatenate([have, keys])
    g = csr_from_pairs(n, have >> U64(32), have & U64(0xFFFFFFFF))
    g.name = f"ER(n={n},M={m},seed={seed})"
    return g


# Chung-Lu (fast form): each of M = n*dbar/2 sampled edges picks both endpoints
# independently with P(index i) proportional to the integral of x^(-1/(gamma-1))
# over [x0+i, x0+i+1).  x0 = 390 puts the largest expected degree at
# sqrt(n*dbar) (the structural cutoff) for n=1e6, dbar=20, gamma=2.1.
CHUNG_LU_X0 = 390


def chung_lu_planted(
    n: int = 1_000_000,
    mean_deg: float = 20.0,
    n_cliques: int = 2000,
    smin: int = 20,
    smax: int = 60,
    seed: int = 1,
    x0: int = CHUNG_LU_X0,
) -> Graph:
    """Power-law (exponent 2.1) Chung-Lu graph plus planted cliques.

    Exponent 2.1 fixes the density exponent 1/(gamma-1) = 10/11, so endpoint
    indices are drawn by inverting the continuous CDF, which is linear in
    x^(1/11): y = a + U (b - a), x = y^11 (ten multiplications), i = floor(x) - x0.
    Then ``n_cliques`` cliques of size uniform in [smin, smax] are planted on
    uniformly random vertex sets (overlaps allowed) and vertex ids are randomly
    permuted.
    """
    m = int(round(n * mean_deg / 2))
    a = _float_root(x0, 11)
    b = _float_root(x0 + n, 11)
    bg = _stream(seed, 3)
    ends = []
    chunk = 1 << 22
    left = 2 * m
    while left > 0:
        c = min(chunk, left)
        u = _u01(_raw(bg, c))
        y = a + u * (b - a)
        y2 = y * y
        y4 = y2 * y2
        y8 = y4 * y4
        x = y8 * y2 * y
        idx = np.floor(x).astype(np.int64) - x0
        np.clip(idx, 0, n - 1, out=idx)
        ends.append(idx)
        left -= c
    ends = np.concatenate(ends)
    perm = _random_permutation(seed, 4, n)
    src = perm[ends[0::2]]
    dst = perm[ends[1::2]]
    # planted cliques
    cg = _stream(seed, 5)
    pa, pb = [src], [dst]
    planted = []
    for _ in range(n_cliques):
        s = smin + int(_bounded(_raw(cg, 1), smax - smin + 1)[0])
        members: list[int] = []
        seen = set()
        while len(members) < s:
            for v in _bounded(_raw(cg, s), n).tolist():
                if v not in seen and len(members) < s:
                    seen.add(v)
                    members.append(v)
        mem = np.array(members, dtype=np.int64)
        i, j = np.triu_indices(s, 1)
        pa.append(mem[i])
        pb.append(mem[j])
        planted.append(mem)
    g = csr_from_pairs(n, np.concatenate(pa), np.concatenate(pb))
    g.name = f"ChungLu(n={n},gamma=2.1,d={mean_deg})+{n_cliques}cliques[{smin},{smax}],seed={seed}"
    g.planted = planted  # type: ignore[attr-defined]
    return g


def rmat(scale: int = 22, edge_factor: int = 16, abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 2,
         permute: bool = True) -> Graph:
    """R-MAT pairs, returned RAW (directed, self-loops and duplicates kept).

    Each of edge_factor * 2^scale samples descends `scale` levels; at each level
    a 32-bit draw picks quadrant a/b/c/d by integer thresholds (no noise).
    Vertex ids are then randomly permuted.  Canonicalisation (symmetrise, drop
    self-loops and duplicates) is left to the consumer.
    """
    n = 1 << scale
    m = edge_factor * n
    a, b, c, _ = abcd
    t1 = U64(int(a * 2 ** 32))
    t2 = U64(int((a + b) * 2 ** 32))
    t3 = U64(int((a + b + c) * 2 ** 32))
    bg = _stream(seed, 6)
    perm = _random_permutation(seed, 7, n).astype(np.uint64) if permute else None
    srcs, dsts = [], []
    chunk = 1 << 22
    done = 0
    words = (scale + 1) // 2
    mask32 = U64(0xFFFFFFFF)
    while done < m:
        cnt = min(chunk, m - done)
        raw = _raw(bg, cnt * words).reshape(cnt, words)
        s = np.zeros(cnt, dtype=np.uint64)
        d = np.zeros(cnt, dtype=np.uint64)
        for lvl in range(scale):
            w = raw[:, lvl // 2]
            r = (w >> U64(32)) if (lvl & 1) == 0 else (w & mask32)
            q = (r >= t1).astype(np.uint64) + (r >= t2).astype(np.uint64) + (r >= t3).astype(np.uint64)
            s = (s << U64(1)) | (q >> U64(1))
            d = (d << U64(1)) | (q & U64(1))
        if perm is not None:
            s = perm[s.astype(np.int64)]
            d = perm[d.astype(np.int64)]
        srcs.append(s)
        dsts.append(d)
        done += cnt
    g = raw_csr_from_pairs(n, np.concatenate(srcs), np.concatenate(dsts))
    g.name = f"RMAT(scale={scale},ef={edge_factor},abcd={abcd},seed={seed},raw)"
    return g


def rgg_torus(n: int, mean_deg: float, seed: int, tag: int = 8) -> Graph:
    """2-D random geometric graph on the unit torus, r = sqrt(D / (pi (n-1)))."""
    bg = _stream(seed, tag)
    raw = _raw(bg, 2 * n)
    x = _u01(raw[0::2])
    y = _u01(raw[1::2])
    r = np.sqrt(mean_deg / (3.141592653589793 * (n - 1)))
    r2 = r * r
    gcells = max(1, int(np.floor(1.0 / r)))
    if gcells < 3:
        i, j = np.triu_indices(n, 1)
        cand_i, cand_j = i, j
    else:
        cx = np.minimum((x * gcells).astype(np.int64), gcells - 1)
        cy = np.minimum((y * gcells).astype(np.int64), gcells - 1)
        cell = cx * gcells + cy
        order = np.argsort(cell, kind="stable")
        cell_sorted = cell[order]
        start = np.searchsorted(cell_sorted, np.arange(gcells * gcells), side="left")
        end = np.searchsorted(cell_sorted, np.arange(gcells * gcells), side="right")
        ci, cj = [], []
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                nc = ((cx + dx) % gcells) * gcells + ((cy + dy) % gcells)
                cnt = end[nc] - start[nc]
                rep_i = np.repeat(np.arange(n), cnt)
                offs = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
                jj = order[np.repeat(start[nc], cnt) + offs]
                keep = rep_i < jj
                ci.append(rep_i[keep])
                cj.append(jj[keep])
        cand_i = np.concatenate(ci)
        cand_j = np.concatenate(cj)
    ddx = np.abs(x[cand_i] - x[cand_j])
    ddx = np.minimum(ddx, 1.0 - ddx)
    ddy = np.abs(y[cand_i] - y[cand_j])
    ddy = np.minimum(ddy, 1.0 - ddy)
    d2 = ddx * ddx + ddy * ddy
    m = d2 <= r2
    g = csr_from_pairs(n, cand_i[m], cand_j[m])
    g.name = f"RGG(n={n},D={mean_deg},seed={seed})"
    return g


# ------------------------------------------------------------- named configs
def config_er_small(seed: int = 0) -> Graph:
    """Erdos-Renyi G(n=2000, p=0.01), seed 0 (the small parity workload)."""
    return er_gnp(2000, 0.01, seed)


def config_chung_lu(seed: int = 1, n: int = 1_000_000, n_cliques: int = 2000) -> Graph:
    """Chung-Lu n=1e6, gamma 2.1, mean degree 20, 2000 planted cliques of size U[20,60]."""
    return chung_lu_planted(n=n, mean_deg=20.0, n_cliques=n_cliques, smin=20, smax=60, seed=seed)


def config_rmat(seed: int = 2, scale: int = 22) -> Graph:
    """R-MAT scale 22, edge factor 16, (0.57, 0.19, 0.19, 0.05), raw pairs."""
    return rmat(scale=scale, edge_factor=16, seed=seed)


def tiny_random(n: int, p: float, seed: int) -> Graph:
    return er_gnp(n, p, seed)


def config_batched(seed: int = 3, count: int = 4096, nmin: int = 50, nmax: int = 20000):
    """Config 4: `count` uneven graphs with a k each, as a list of (Graph, k).

    n is log-uniform in [nmin, nmax]: a 53-bit uniform u is compared with the
    table of thresholds log(n / nmin) / log(nmax / nmin), computed once for
    every integer n (no per-sample transcendental).  Even positions are
    Erdos-Renyi G(n, M) with M = round(n D / 2), D uniform in [8, 40]; odd
    positions are 2-D random geometric graphs on the unit torus with mean
    degree D uniform in [10, 60].  k is uniform in {4, ..., 8}.  Every graph
    has its own seed drawn from the batch's stream.
    """
    ns = np.arange(nmin, nmax + 1, dtype=np.float64)
    thr = np.log(ns / nmin) / np.log(nmax / nmin)  # thr[i]: smallest u giving n >= ns[i]
    bg = _stream(seed, 9)
    raw = _raw(bg, 4 * count).reshape(count, 4)
    u = _u01(raw[:, 0])
    n_of = nmin + np.searchsorted(thr, u, side="right") - 1
    dfrac = _u01(raw[:, 1])
    ks = 4 + _bounded(raw[:, 2], 5)
    seeds = (raw[:, 3] >> U64(33)).astype(np.int64)
    out = []
    for i in range(count):
        n = int(n_of[i])
        if i % 2 == 0:
            deg = 8.0 + 32.0 * float(dfrac[i])
            m = min(int(round(n * deg / 2.0)), n * (n - 1) // 2)
            g = er_gnm(n, m, int(seeds[i]))
        else:
            deg = 10.0 + 50.0 * float(dfrac[i])
            g = rgg_torus(n, min(deg, float(n - 1)), int(seeds[i]))
        out.append((g, int(ks[i])))
    return out
