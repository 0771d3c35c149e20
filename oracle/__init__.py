"""The oracle: plain CPU implementations used to check the CUDA path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_2502_00317_gb300``) and never imports it; the only
thing both sides share is the seeded input generator module.

Contents
--------
* ``OracleGraph`` -- ctypes front of ``kc_oracle.c``: canonicalise, degeneracy
  order, orient, list/count k-cliques with an order-independent checksum
  (Sec. II-A definitions; Algorithm 1).
* ``brute_force_cliques`` -- every k-subset tested pair by pair (clique
  definition, Sec. II-A); for n <= 20.
* ``soft_embedding_r`` -- Algorithm 5 (ComputeSoftEmbeddings), written from
  the Sec. V text, on a DAG given as out-neighbour lists.
* ``restricted_root_r`` -- Algorithm 5 applied to the DAG induced by
  N(u) ∪ {u}, the form used for pruning (Sec. V, after Theorem 2).
* ``max_tree_embedding`` -- the largest l such that a soft embedding of an
  l-tree is rooted at u, searched straight from the l-tree and soft-embedding
  definitions (Sec. V, Definitions of l-tree and soft embedding); used to pin
  Theorem 2 and Lemma 1.
* closed forms: C(n, k) for complete graphs, the elementary symmetric
  polynomial e_k of the part sizes for complete multipartite (Turan) graphs.
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os
import subprocess
from functools import lru_cache

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libkc_oracle.so")


def build(force: bool = False) -> str:
    """Compile kc_oracle.c into oracle/_build/libkc_oracle.so (gcc, -O2)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-pthread",
                               "-Wall", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


@lru_cache(maxsize=1)
def _lib():
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    u32, u64, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    lib.kco_build.restype = P
    lib.kco_build.argtypes = [u32, P, P, ctypes.POINTER(i32)]
    lib.kco_free.argtypes = [P]
    lib.kco_n.restype = u32
    lib.kco_n.argtypes = [P]
    lib.kco_m.restype = u64
    lib.kco_m.argtypes = [P]
    lib.kco_degeneracy.restype = u32
    lib.kco_degeneracy.argtypes = [P]
    lib.kco_max_out.restype = u32
    lib.kco_max_out.argtypes = [P]
    lib.kco_get_core.argtypes = [P, P]
    lib.kco_get_rank.argtypes = [P, P]
    lib.kco_get_adj.argtypes = [P, P, P]
    lib.kco_get_dag_edges.argtypes = [P, P, P]
    lib.kco_run.restype = i32
    lib.kco_run.argtypes = [P, u32, i32, u32, u32, i32, ctypes.POINTER(u64), ctypes.POINTER(u64), P,
                            ctypes.POINTER(i32)]
    lib.kco_list.restype = i32
    lib.kco_list.argtypes = [P, u32, P, u64, ctypes.POINTER(u64), ctypes.POINTER(u64)]
    lib.kco_clique_hash.restype = u64
    lib.kco_clique_hash.argtypes = [P, u32]
    lib.kco_mix64_value.restype = u64
    lib.kco_mix64_value.argtypes = [u64]
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleGraph:
    """The oracle's own copy of a graph: canonicalised, ordered and oriented on the CPU."""

    def __init__(self, n: int, rowptr: np.ndarray, col: np.ndarray):
        self._rowptr = np.ascontiguousarray(rowptr, dtype=np.uint64)
        self._col = np.ascontiguousarray(col, dtype=np.uint32)
        if self._col.size == 0:
            self._col = np.zeros(1, dtype=np.uint32)
        st = ctypes.c_int(0)
        self._h = _lib().kco_build(int(n), _ptr(self._rowptr), _ptr(self._col), ctypes.byref(st))
        if not self._h:
            raise ValueError(f"oracle rejected the graph (status {st.value})")

    @classmethod
    def from_graph(cls, g) -> "OracleGraph":
        return cls(g.n, g.rowptr, g.col)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib().kco_free(h)
            self._h = None

    @property
    def n(self) -> int:
        return int(_lib().kco_n(self._h))

    @property
    def m(self) -> int:
        return int(_lib().kco_m(self._h))

    @property
    def degeneracy(self) -> int:
        return int(_lib().kco_degeneracy(self._h))

    @property
    def max_out_degree(self) -> int:
        return int(_lib().kco_max_out(self._h))

    def core_numbers(self) -> np.ndarray:
        out = np.zeros(max(self.n, 1), dtype=np.uint32)
        _lib().kco_get_core(self._h, _ptr(out))
        return out[: self.n]

    def ranks(self) -> np.ndarray:
        out = np.zeros(max(self.n, 1), dtype=np.uint32)
        _lib().kco_get_rank(self._h, _ptr(out))
        return out[: self.n]

    def adjacency(self):
        """Canonical undirected CSR as the oracle sees it."""
        ptr = np.zeros(self.n + 1, dtype=np.uint64)
        adj = np.zeros(max(2 * self.m, 1), dtype=np.uint32)
        _lib().kco_get_adj(self._h, _ptr(ptr), _ptr(adj))
        return ptr, adj[: 2 * self.m]

    def dag_edges(self):
        src = np.zeros(max(self.m, 1), dtype=np.uint32)
        dst = np.zeros(max(self.m, 1), dtype=np.uint32)
        _lib().kco_get_dag_edges(self._h, _ptr(src), _ptr(dst))
        return src[: self.m], dst[: self.m]

    def count(self, k: int, threads: int = 0, root_lo: int = 0, root_hi: int | None = None):
        """Number of k-cliques (count mode); returns (count, threads_used)."""
        c = ctypes.c_uint64(0)
        s = ctypes.c_uint64(0)
        t = ctypes.c_int(0)
        hi = self.n if root_hi is None else int(root_hi)
        st = _lib().kco_run(self._h, int(k), 0, int(root_lo), hi, int(threads), ctypes.byref(c),
                            ctypes.byref(s), None, ctypes.byref(t))
        if st != 0:
            raise ValueError(f"oracle count failed ({st})")
        return int(c.value), int(t.value)

    def checksum(self, k: int, threads: int = 0, root_lo: int = 0, root_hi: int | None = None,
                 per_vertex: bool = False):
        """(count, checksum[, per_vertex counts]) visiting every k-clique."""
        c = ctypes.c_uint64(0)
        s = ctypes.c_uint64(0)
        t = ctypes.c_int(0)
        pv = np.zeros(max(self.n, 1), dtype=np.uint64) if per_vertex else None
        hi = self.n if root_hi is None else int(root_hi)
        st = _lib().kco_run(self._h, int(k), 1, int(root_lo), hi, int(threads), ctypes.byref(c),
                            ctypes.byref(s), _ptr(pv) if pv is not None else None, ctypes.byref(t))
        if st != 0:
            raise ValueError(f"oracle listing failed ({st})")
        if per_vertex:
            return int(c.value), int(s.value), pv[: self.n]
        return int(c.value), int(s.value)

    def list(self, k: int, cap: int | None = None):
        """All k-cliques as an (N, k) array of sorted original ids (single thread)."""
        total = ctypes.c_uint64(0)
        s = ctypes.c_uint64(0)
        if cap is None:
            _lib().kco_list(self._h, int(k), None, 0, ctypes.byref(total), ctypes.byref(s))
            cap = int(total.value)
        buf = np.zeros(max(cap * k, 1), dtype=np.uint32)
        _lib().kco_list(self._h, int(k), _ptr(buf), int(cap), ctypes.byref(total), ctypes.byref(s))
        got = min(cap, int(total.value))
        return buf[: got * k].reshape(got, k), int(total.value), int(s.value)


def mix64(z: int) -> int:
    """The SplitMix64 finaliser of the checksum (the oracle's C function)."""
    return int(_lib().kco_mix64_value(int(z) & 0xFFFFFFFFFFFFFFFF))


def clique_hash(ids_sorted) -> int:
    a = np.ascontiguousarray(ids_sorted, dtype=np.uint32)
    return int(_lib().kco_clique_hash(_ptr(a), int(a.size)))


# ------------------------------------------------------------ pure Python
def adjacency_sets(n: int, rowptr, col):
    """Undirected neighbour sets, symmetrised, self-loops dropped."""
    adj = [set() for _ in range(n)]
    rowptr = np.asarray(rowptr, dtype=np.int64)
    for u in range(n):
        for v in col[rowptr[u]:rowptr[u + 1]].tolist():
            if v != u:
                adj[u].add(int(v))
                adj[int(v)].add(u)
    return adj


def brute_force_cliques(n: int, adj, k: int):
    """Every k-subset of range(n) whose pairs are all adjacent (Sec. II-A)."""
    out = []
    for sub in itertools.combinations(range(n), k):
        if all(b in adj[a] for a, b in itertools.combinations(sub, 2)):
            out.append(sub)
    return out


def soft_embedding_r(order, out):
    """Algorithm 5: r(u) for every vertex of a DAG.

    ``order`` lists the vertices ascending in the DAG's total order; ``out[u]``
    is the set of out-neighbours of u (all later in the order).  Vertices are
    visited in descending order; r(u) starts at 1 and the out-neighbours are
    scanned from the largest to the smallest, adding one whenever the current
    r(u) is at most r of that neighbour (Sec. V).
    """
    pos = {v: i for i, v in enumerate(order)}
    r = {}
    for u in reversed(order):
        ru = 1
        for w in sorted(out[u], key=lambda x: pos[x], reverse=True):
            if ru <= r[w]:
                ru += 1
        r[u] = ru
    return r


def restricted_root_r(order, out, u):
    """r of u by Algorithm 5 on the DAG induced by N(u) ∪ {u} (Sec. V)."""
    keep = set(out[u]) | {u}
    sub_order = [v for v in order if v in keep]
    sub_out = {v: set(out[v]) & keep for v in sub_order}
    return soft_embedding_r(sub_order, sub_out)[u]


def max_tree_embedding(order, out, u, lmax=None):
    """Largest l with a soft embedding of an l-tree rooted at u, by search.

    Straight from the definitions (Sec. V): the root of an l-tree has l-1
    children whose subtrees are a 1-tree, ..., an (l-1)-tree; the child with
    the i-tree has out-degree i-1.  A soft embedding maps tree edges onto DAG
    edges and maps siblings of smaller out-degree to larger vertices.  So an
    l-tree embeds at u iff out-neighbours w_1 > w_2 > ... > w_{l-1} of u exist
    with an i-tree embedded at w_i for each i.  The chain is searched
    exhaustively (exponential: tiny DAGs only).
    """
    pos = {v: i for i, v in enumerate(order)}
    memo = {}

    def embeds(v, l):
        if l == 1:
            return True
        key = (v, l)
        if key in memo:
            return memo[key]
        nbrs = sorted(out[v], key=lambda x: pos[x], reverse=True)  # descending

        def chain(i, start):  # choose w_i among nbrs[start:], need w_i..w_{l-1}
            if i == l:
                return True
            for j in range(start, len(nbrs)):
                if embeds(nbrs[j], i) and chain(i + 1, j + 1):
                    return True
            return False

        memo[key] = chain(1, 0)
        return memo[key]

    top = (len(order) + 1) if lmax is None else lmax
    best = 1
    for l in range(2, top + 1):
        if embeds(u, l):
            best = l
        else:
            break
    return best


def binom(n: int, k: int) -> int:
    return math.comb(n, k) if 0 <= k <= n else 0


def elementary_symmetric(sizes, k: int) -> int:
    """e_k(sizes): k-cliques of the complete multipartite graph with these parts."""
    e = [1] + [0] * k
    for s in sizes:
        for j in range(k, 0, -1):
            e[j] += e[j - 1] * s
    return e[k]
