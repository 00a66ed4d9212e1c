"""Seeded synthetic workloads (input generators only).

This module draws the input facts of every workload used by the tests and the
benchmark.  It is shared by the CUDA engine and by the CPU oracle, and for that
reason it contains none of the method's arithmetic: no join, no semiring
operation, no fixpoint.  It only produces integer columns, f32 probabilities
and sample ids.

Randomness is one counter-based generator, SplitMix64 (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): draw ``i`` of
stream ``s`` is ``mix64(seed_s + (i + 1) * 0x9E3779B97F4A7C15)``.  Everything
is vectorised numpy so the full-size workloads generate in seconds.

The workloads stand in for the paper's datasets (SNAP graphs, CSPA inputs,
CLUTRR passages, Pathfinder images), none of which is available offline; each
generator states the shape it reproduces.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
PROJECT_SEED = 0x10B57E6B300  # project constant; workload seeds add an index


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= np.uint64(0xBF58476D1CE4E5B9)
    z ^= z >> np.uint64(27)
    z *= np.uint64(0x94D049BB133111EB)
    z ^= z >> np.uint64(31)
    return z


class Stream:
    """A counter-based SplitMix64 stream; ``take(n)`` returns the next n draws."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.pos = 0

    def take(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            idx = np.arange(self.pos + 1, self.pos + 1 + n, dtype=np.uint64)
            out = _mix64(self.seed + idx * GOLDEN)
        self.pos += n
        return out

    def below(self, n: int, bound) -> np.ndarray:
        """n integers uniform in [0, bound) (Lemire's multiply-shift, bound < 2^32)."""
        hi = self.take(n) >> np.uint64(32)
        return ((hi * np.asarray(bound, dtype=np.uint64)) >> np.uint64(32)).astype(np.uint32)

    def prob(self, n: int) -> np.ndarray:
        """n f32 values in (0, 1): odd multiples of 2^-24, all exactly representable."""
        k = self.take(n) >> np.uint64(41)
        return ((k * np.uint64(2) + np.uint64(1)).astype(np.float64) * 2.0 ** -24).astype(np.float32)

    def unit(self, n: int) -> np.ndarray:
        """n float64 values in [0, 1) with 53 random bits."""
        return (self.take(n) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53

    def normal(self, n: int) -> np.ndarray:
        """n standard normal float64 values (Box-Muller on two unit draws)."""
        u1 = 1.0 - self.unit(n)
        u2 = self.unit(n)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)

    def permutation(self, n: int) -> np.ndarray:
        """A uniformly random permutation of range(n) (sort by random keys)."""
        keys = self.take(n)
        return np.argsort(keys, kind="stable").astype(np.uint32)


def stream(workload_index: int, sub: int = 0) -> Stream:
    return Stream(PROJECT_SEED + 1000 * workload_index + sub)


# ----------------------------------------------------------------------------
# graphs
# ----------------------------------------------------------------------------

def _distinct_pairs(src: np.ndarray, dst: np.ndarray, n_nodes: int):
    """Drop self-loops and repeated pairs, keeping first occurrences in draw order."""
    keep = src != dst
    src, dst = src[keep], dst[keep]
    code = src.astype(np.uint64) * np.uint64(n_nodes) + dst.astype(np.uint64)
    _, first = np.unique(code, return_index=True)
    first.sort()
    return src[first], dst[first]


def erdos_renyi(n_nodes: int, n_edges: int, seed_index: int = 1):
    """Directed G(n, m): ``n_edges`` distinct uniform (src, dst) pairs, no self-loops."""
    s = stream(seed_index)
    draw = max(2 * n_edges, 64)
    while True:
        src = s.below(draw, n_nodes)
        dst = s.below(draw, n_nodes)
        a, b = _distinct_pairs(src, dst, n_nodes)
        if len(a) >= n_edges:
            return a[:n_edges].copy(), b[:n_edges].copy()
        draw *= 2
        s = stream(seed_index, sub=draw)


def random_tree(n_nodes: int, min_children: int = 1, max_children: int = 4, seed_index: int = 2,
                relabel: bool = True):
    """BFS-grown random tree: each node in BFS order gets U{min..max} children
    until ``n_nodes`` exist.  Returns parent(p, x) columns and each node's depth.
    Node ids are relabelled through a seeded permutation."""
    s = stream(seed_index)
    kids = (s.below(n_nodes, max_children - min_children + 1) + np.uint32(min_children)).astype(np.int64)
    # node j (BFS order) owns children ids [start_j, start_j + kids_j), truncated at n_nodes
    start = 1 + np.concatenate([[0], np.cumsum(kids)[:-1]])
    parent = np.empty(n_nodes - 1, dtype=np.uint32)
    depth = np.zeros(n_nodes, dtype=np.int64)
    for j in range(n_nodes):
        a = start[j]
        if a >= n_nodes:
            break
        b = min(a + kids[j], n_nodes)
        parent[a - 1:b - 1] = j
        depth[a:b] = depth[j] + 1
    child = np.arange(1, n_nodes, dtype=np.uint32)
    if relabel:
        perm = s.permutation(n_nodes)
        parent = perm[parent]
        child = perm[child]
        depth_l = np.empty_like(depth)
        depth_l[perm] = depth
        depth = depth_l
    return parent, child, depth


def perfect_tree(k: int, levels: int):
    """Perfect k-ary tree with ``levels`` levels below the root, BFS ids."""
    parent, child = [], []
    level = [0]
    nxt = 1
    for _ in range(levels):
        new = []
        for p in level:
            for _ in range(k):
                parent.append(p)
                child.append(nxt)
                new.append(nxt)
                nxt += 1
        level = new
    return np.array(parent, dtype=np.uint32), np.array(child, dtype=np.uint32)


def chung_lu_power_law(n_nodes: int, n_edges: int, gamma: float = 2.1, seed_index: int = 3):
    """Directed Chung-Lu graph with power-law expected degrees.

    Node i has weight (i + 1) ** (-1 / (gamma - 1)); sources and destinations are
    drawn independently proportional to weight, self-loops and duplicates are
    rejected until ``n_edges`` distinct edges exist, and ids are relabelled
    through a seeded permutation."""
    s = stream(seed_index)
    w = (np.arange(1, n_nodes + 1, dtype=np.float64)) ** (-1.0 / (gamma - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    src_all, dst_all = np.empty(0, np.uint32), np.empty(0, np.uint32)
    draw = 2 * n_edges
    while True:
        su = s.unit(draw)
        du = s.unit(draw)
        src_all = np.concatenate([src_all, np.minimum(np.searchsorted(cdf, su, side="right"), n_nodes - 1).astype(np.uint32)])
        dst_all = np.concatenate([dst_all, np.minimum(np.searchsorted(cdf, du, side="right"), n_nodes - 1).astype(np.uint32)])
        a, b = _distinct_pairs(src_all, dst_all, n_nodes)
        if len(a) >= n_edges:
            break
    a, b = a[:n_edges], b[:n_edges]
    perm = s.permutation(n_nodes)
    return perm[a].copy(), perm[b].copy()


def grid_edges(side: int):
    """Undirected 4-connected grid G_{side,side}: node id = row * side + col.
    Returns (u, v) for the 2 * side * (side - 1) undirected edges in a fixed
    order: all horizontal edges row by row, then all vertical edges."""
    r, c = np.meshgrid(np.arange(side), np.arange(side - 1), indexing="ij")
    hu = (r * side + c).ravel()
    hv = hu + 1
    r, c = np.meshgrid(np.arange(side - 1), np.arange(side), indexing="ij")
    vu = (r * side + c).ravel()
    vv = vu + side
    return (np.concatenate([hu, vu]).astype(np.uint32), np.concatenate([hv, vv]).astype(np.uint32))


def directed_from_undirected(u: np.ndarray, v: np.ndarray, p: np.ndarray):
    """Each undirected edge k becomes facts edge(u,v) (row 2k) and edge(v,u)
    (row 2k+1) sharing probability p[k]."""
    src = np.empty(2 * len(u), np.uint32)
    dst = np.empty(2 * len(u), np.uint32)
    src[0::2], dst[0::2] = u, v
    src[1::2], dst[1::2] = v, u
    return src, dst, np.repeat(p, 2).astype(np.float32)


def grid_reach_instance(side: int, seed_index: int = 4, sub: int = 0):
    """Probabilistic reachability on G_{side,side} (the Pathfinder shape): one
    f32 probability per undirected edge, two directed facts per edge, source 0."""
    u, v = grid_edges(side)
    p = stream(seed_index, sub).prob(len(u))
    src, dst, tags = directed_from_undirected(u, v, p)
    return {"edge": (src, dst, tags), "start": (np.array([0], np.uint32),), "p_undirected": p}


def ktree_chain(n: int):
    """Directed chain 0 -> 1 -> ... -> n-1."""
    a = np.arange(n - 1, dtype=np.uint32)
    return a, a + 1


def zipf_ranks(s: Stream, n: int, exponent: float, support: int) -> np.ndarray:
    """n draws of a Zipf(exponent) rank truncated to 1..support (inverse CDF)."""
    w = np.arange(1, support + 1, dtype=np.float64) ** (-exponent)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    return (np.minimum(np.searchsorted(cdf, s.unit(n), side="right"), support - 1) + 1).astype(np.int64)


def andersen_program(n_vars: int, n_stmts: int, exponent: float = 1.8, seed_index: int = 5):
    """Andersen-style points-to input: ``n_stmts`` statements of kinds
    address-of / assign / load / store in proportions 40/40/10/10 %, both
    operands truncated Zipf(exponent) ranks over 1..n_vars mapped through a
    seeded permutation.  Returns dict kind -> (lhs, rhs) raw columns (duplicates
    included; the engine and the oracle both merge them on load)."""
    s = stream(seed_index)
    kind = s.below(n_stmts, 10)  # 0-3 addr, 4-7 assign, 8 load, 9 store
    lhs = zipf_ranks(s, n_stmts, exponent, n_vars) - 1
    rhs = zipf_ranks(s, n_stmts, exponent, n_vars) - 1
    perm = s.permutation(n_vars)
    lhs = perm[lhs]
    rhs = perm[rhs]
    out = {}
    for name, sel in (("addr", kind < 4), ("assign", (kind >= 4) & (kind < 8)), ("load", kind == 8), ("store", kind == 9)):
        out[name] = (lhs[sel].astype(np.uint32).copy(), rhs[sel].astype(np.uint32).copy())
    return out


def kinship_instance(s: Stream, n_labels: int = 20, lo: int = 10, hi: int = 40):
    """One kinship sample: n ~ U{lo..hi} people, a random chain of n-1 labelled
    facts plus U{0..n} extra random facts (no self pairs), labels U{0..n_labels-1},
    f32 probabilities U(0,1)."""
    n = int(s.below(1, hi - lo + 1)[0]) + lo
    order = s.permutation(n)
    extra = int(s.below(1, n + 1)[0])
    a = np.concatenate([order[:-1], s.below(extra, n)])
    b = np.concatenate([order[1:], s.below(extra, n)])
    keep = a != b
    a, b = a[keep], b[keep]
    r = s.below(len(a), n_labels)
    p = s.prob(len(a))
    return n, r, a.astype(np.uint32), b.astype(np.uint32), p


def composition_table(n_labels: int = 20, seed_index: int = 6):
    """comp(r1, r2, r3): one r3 ~ U{0..n_labels-1} for every (r1, r2)."""
    s = stream(seed_index)
    r1, r2 = np.meshgrid(np.arange(n_labels), np.arange(n_labels), indexing="ij")
    r3 = s.below(n_labels * n_labels, n_labels)
    return r1.ravel().astype(np.uint32), r2.ravel().astype(np.uint32), r3


def batched_instance(n_samples: int = 512, side_lo: int = 8, side_hi: int = 48, n_labels: int = 20,
                     seed_index: int = 7):
    """Batched differentiable workload: per sample a grid of side U{side_lo..side_hi}
    with its own probabilities (reach from node 0), plus a kinship instance with
    the shared composition table replicated per sample.  Returns per-relation
    (cols..., tags, sample_ids) and per-sample metadata."""
    s = stream(seed_index)
    sides = (s.below(n_samples, side_hi - side_lo + 1) + np.uint32(side_lo)).astype(np.int64)
    c1, c2, c3 = composition_table(n_labels)
    edge_s, edge_d, edge_p, edge_sid = [], [], [], []
    start_x, start_sid = [], []
    fact_r, fact_a, fact_b, fact_p, fact_sid = [], [], [], [], []
    comp_cols = ([], [], [], [])
    for i in range(n_samples):
        g = grid_reach_instance(int(sides[i]), seed_index=seed_index, sub=1 + i)
        src, dst, tags = g["edge"]
        edge_s.append(src); edge_d.append(dst); edge_p.append(tags)
        edge_sid.append(np.full(len(src), i, np.uint32))
        start_x.append(np.array([0], np.uint32)); start_sid.append(np.array([i], np.uint32))
        ks = stream(seed_index, sub=100000 + i)
        _, r, a, b, p = kinship_instance(ks, n_labels)
        fact_r.append(r); fact_a.append(a); fact_b.append(b); fact_p.append(p)
        fact_sid.append(np.full(len(r), i, np.uint32))
        comp_cols[0].append(c1); comp_cols[1].append(c2); comp_cols[2].append(c3)
        comp_cols[3].append(np.full(len(c1), i, np.uint32))
    cat = np.concatenate
    return {
        "sides": sides,
        "edge": (cat(edge_s), cat(edge_d), cat(edge_p), cat(edge_sid)),
        "start": (cat(start_x), None, cat(start_sid)),
        "fact": (cat(fact_r), cat(fact_a), cat(fact_b), cat(fact_p), cat(fact_sid)),
        "comp": (cat(comp_cols[0]), cat(comp_cols[1]), cat(comp_cols[2]), None, cat(comp_cols[3])),
    }


# ----------------------------------------------------------------------------
# programs (Datalog text; the semantics live in the engine and the oracle)
# ----------------------------------------------------------------------------

TC_PROGRAM = "path(x,y) :- edge(x,y).\npath(x,z) :- path(x,y), edge(y,z).\n"
SG_PROGRAM = ("sg(x,y) :- parent(p,x), parent(p,y), x != y.\n"
              "sg(x,y) :- parent(a,x), sg(a,b), parent(b,y).\n")
REACH_PROGRAM = "reach(x) :- start(x).\nreach(y) :- reach(x), edge(x,y).\n"
KIN_PROGRAM = ("kin(r,x,y) :- fact(r,x,y).\n"
               "kin(r3,x,z) :- kin(r1,x,y), kin(r2,y,z), comp(r1,r2,r3), x != z.\n")
ANDERSEN_PROGRAM = ("pt(p,a) :- addr(p,a).\n"
                    "pt(p,o) :- assign(p,q), pt(q,o).\n"
                    "pt(p,o) :- load(p,q), pt(q,r), pt(r,o).\n"
                    "pt(r,o) :- store(p,q), pt(p,r), pt(q,o).\n")

# Programs of several strata (Sec. 3.1: a RAM program is a sequence of strata).
# LAYERED: the closure, then the nodes with a successor, then pairs two or more
# hops apart from such a node -- three strata, the last reading both below it.
LAYERED_PROGRAM = (TC_PROGRAM +
                   "src(x) :- path(x,y).\n"
                   "far(x,z) :- src(x), path(x,y), path(y,z), x != z.\n")
# ODD_EVEN: odd and even path lengths are mutually recursive (one stratum of two
# relations), and cnt reads even from the stratum above.
ODD_EVEN_PROGRAM = ("odd(x,y) :- edge(x,y).\n"
                    "odd(x,z) :- even(x,y), edge(y,z).\n"
                    "even(x,z) :- odd(x,y), edge(y,z).\n"
                    "cnt(x) :- even(x,y).\n")

SEMIRINGS = {"unit": 0, "max_min": 1, "add_mult": 2, "diff_max_min": 3, "diff_add_mult": 4}
