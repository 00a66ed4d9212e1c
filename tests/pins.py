"""Independent textbook computations that pin the oracle (and, through it, the
engine).  None of these share code with ``oracle/`` or with the engine; each is
a different algorithm for a quantity the semiring fixpoint must reproduce.
"""
from __future__ import annotations

import heapq
import itertools
from collections import defaultdict, deque

import numpy as np


def bfs_closure(src, dst, n_nodes=None):
    """Transitive closure as the set of (x, y) with y reachable from x by >= 1 edge,
    by one BFS per source."""
    adj = defaultdict(list)
    for a, b in zip(src.tolist(), dst.tolist()):
        adj[a].append(b)
    out = set()
    for s in list(adj):
        seen = set()
        q = deque(adj[s])
        while q:
            v = q.popleft()
            if v in seen:
                continue
            seen.add(v)
            q.extend(adj.get(v, ()))
        out.update((s, v) for v in seen)
    return out


def closure_count_scipy(src, dst, n_nodes):
    """|TC| via per-source BFS in scipy (for larger graphs)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import breadth_first_order
    g = sp.csr_matrix((np.ones(len(src)), (src, dst)), shape=(n_nodes, n_nodes))
    total = 0
    for s in range(n_nodes):
        if g.indptr[s + 1] == g.indptr[s]:
            continue
        order = breadth_first_order(g, s, directed=True, return_predecessors=False)
        reach = len(order) - 1
        # s itself is in the closure iff some successor reaches back to s
        nbrs = g.indices[g.indptr[s]:g.indptr[s + 1]]
        back = g[:, s].nonzero()[0]
        if len(back) and np.isin(back, order).any():
            reach += 1
        total += reach
    return total


def closure_keys_scipy(src, dst, n_nodes):
    """Transitive closure as sorted uint64 keys (x << 32 | y), one scipy BFS per
    source; (s, s) belongs to it when a successor of s reaches back to s."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import breadth_first_order
    g = sp.csr_matrix((np.ones(len(src)), (np.asarray(src, np.int64), np.asarray(dst, np.int64))),
                      shape=(n_nodes, n_nodes))
    gt = g.T.tocsr()
    parts = []
    for s in range(n_nodes):
        if g.indptr[s + 1] == g.indptr[s]:
            continue
        order = breadth_first_order(g, s, directed=True, return_predecessors=False)
        reach = order[1:].astype(np.uint64)
        back = gt.indices[gt.indptr[s]:gt.indptr[s + 1]]
        if np.isin(back, order).any():
            reach = np.append(reach, np.uint64(s))
        parts.append((np.uint64(s) << np.uint64(32)) | reach)
    return np.sort(np.concatenate(parts)) if parts else np.zeros(0, np.uint64)


def same_generation_closed_form(depth):
    """|sg| on a tree: ordered pairs of distinct nodes at equal depth >= 1."""
    nd = np.bincount(depth)
    nd = nd[1:].astype(np.int64)
    return int((nd * (nd - 1)).sum())


def same_generation_keys(depth):
    """The same-generation relation of a tree as sorted uint64 keys (x << 32 | y):
    every ordered pair of distinct nodes at equal depth >= 1 (siblings, or nodes
    whose parents are of the same generation, down from the root's children)."""
    depth = np.asarray(depth)
    parts = []
    for d in range(1, int(depth.max()) + 1 if len(depth) else 1):
        v = np.flatnonzero(depth == d).astype(np.uint64)
        if len(v) < 2:
            continue
        x = np.repeat(v, len(v))
        y = np.tile(v, len(v))
        keep = x != y
        parts.append((x[keep] << np.uint64(32)) | y[keep])
    return np.sort(np.concatenate(parts)) if parts else np.zeros(0, np.uint64)


def andersen_worklist(addr, assign, load, store):
    """Andersen's inclusion-based points-to analysis by a textbook worklist
    over points-to sets (no Datalog):
      p = &a      : a in pt(p)
      p = q       : pt(q) subset of pt(p)
      p = *q      : for r in pt(q): pt(r) subset of pt(p)
      *p = q      : for r in pt(p): pt(q) subset of pt(r)
    Note the store rule in Datalog form is pt(r,o) :- store(p,q), pt(p,r), pt(q,o)."""
    pt = defaultdict(set)
    succ = defaultdict(set)  # copy edges q -> p meaning pt(q) subset pt(p)
    loads = defaultdict(list)  # q -> [p] for p = *q
    stores = defaultdict(list)  # p -> [q] for *p = q
    for p, a in zip(*addr):
        pt[int(p)].add(int(a))
    for p, q in zip(*assign):
        succ[int(q)].add(int(p))
    for p, q in zip(*load):
        loads[int(q)].append(int(p))
    for p, q in zip(*store):
        stores[int(p)].append(int(q))
    work = deque(pt.keys())
    inq = set(work)
    while work:
        v = work.popleft()
        inq.discard(v)
        for r in list(pt[v]):
            for p in loads.get(v, ()):
                if p not in succ[r]:
                    succ[r].add(p)
                    if r not in inq:
                        work.append(r); inq.add(r)
            for q in stores.get(v, ()):
                if r not in succ[q]:
                    succ[q].add(r)
                    if q not in inq:
                        work.append(q); inq.add(q)
        for w in list(succ.get(v, ())):
            before = len(pt[w])
            pt[w] |= pt[v]
            if len(pt[w]) != before and w not in inq:
                work.append(w); inq.add(w)
    return {(p, o) for p, s in pt.items() for o in s}


def reach_set(edges, source):
    adj = defaultdict(list)
    for a, b in edges:
        adj[a].append(b)
    seen = {source}
    q = deque([source])
    while q:
        v = q.popleft()
        for w in adj[v]:
            if w not in seen:
                seen.add(w)
                q.append(w)
    return seen


def possible_worlds_maxmin_reach(src, dst, p, source, ids=None):
    """Max-min tag of reach(y) by enumerating every subset W of the edges:
    max over W with y reachable in W of min over W of (p, -id)  (min over the
    empty set = (1, +inf id)).  Returns {y: (value, id)}."""
    m = len(src)
    ids = list(range(m)) if ids is None else list(ids)
    best = {}
    for mask in range(1 << m):
        W = [i for i in range(m) if mask >> i & 1]
        if W:
            lo = min(W, key=lambda i: (p[i], -ids[i]))
            val = (float(p[lo]), -ids[lo])
        else:
            val = (1.0, -(2 ** 40))
        for y in reach_set([(int(src[i]), int(dst[i])) for i in W], source):
            if y not in best or val > best[y]:
                best[y] = val
    return {y: (v, -nid) for y, (v, nid) in best.items()}


def possible_worlds_probability(src, dst, p, source):
    """Exact probability that y is reachable from source when each edge is present
    independently with probability p (enumerating all 2^m worlds)."""
    m = len(src)
    prob = defaultdict(float)
    for mask in range(1 << m):
        w = 1.0
        W = []
        for i in range(m):
            if mask >> i & 1:
                w *= float(p[i]); W.append((int(src[i]), int(dst[i])))
            else:
                w *= 1.0 - float(p[i])
        for y in reach_set(W, source):
            prob[y] += w
    return dict(prob)


def widest_path(src, dst, p, source):
    """Max-min (bottleneck) path value from source by a Dijkstra-style search."""
    adj = defaultdict(list)
    for a, b, w in zip(src.tolist(), dst.tolist(), np.asarray(p, np.float64).tolist()):
        adj[a].append((b, w))
    best = {source: 1.0}
    heap = [(-1.0, source)]
    while heap:
        negv, v = heapq.heappop(heap)
        if -negv < best.get(v, -1):
            continue
        for w, pw in adj[v]:
            c = min(-negv, pw)
            if c > best.get(w, -1.0):
                best[w] = c
                heapq.heappush(heap, (-c, w))
    return best


def layered_reach_dp(src, dst, p, source):
    """Add-mult reach tags by BFS layers: t(source) = 1 and, for y at BFS distance
    d >= 1, t(y) = min(1, sum over edges x->y with dist(x) = d - 1 of t(x) * p_xy)."""
    adj = defaultdict(list)
    for a, b, w in zip(src.tolist(), dst.tolist(), np.asarray(p, np.float64).tolist()):
        adj[a].append((b, w))
    dist = {source: 0}
    order = [source]
    q = deque([source])
    while q:
        v = q.popleft()
        for w, _ in adj[v]:
            if w not in dist:
                dist[w] = dist[v] + 1
                order.append(w)
                q.append(w)
    t = {source: 1.0}
    acc = defaultdict(float)
    for v in order:
        if v != source:
            t[v] = min(1.0, acc[v])
        for w, pw in adj[v]:
            if dist[w] == dist[v] + 1:
                acc[w] += t[v] * pw
    return t, dist


def andersen_sparse(addr, assign, load, store, n_vars):
    """Andersen points-to as the least fixpoint of boolean sparse-matrix
    equations (pt as a vars x vars matrix P):
        P = Addr + Assign.P + Load.P.P + P^T.Store.P   (boolean),
    iterated from P = Addr until no entry changes."""
    import scipy.sparse as sp

    def mat(pq):
        p, q = pq
        m = sp.csr_matrix((np.ones(len(p), np.int64), (p.astype(np.int64), q.astype(np.int64))),
                          shape=(n_vars, n_vars))
        m.data[:] = 1
        m.sum_duplicates()
        m.data[:] = 1
        return m

    def boolify(m):
        m = m.tocsr()
        m.data = (m.data > 0).astype(np.int64)
        m.eliminate_zeros()
        return m

    Ad, As, Ld, St = mat(addr), mat(assign), mat(load), mat(store)
    P = boolify(Ad)
    while True:
        # products grouped so that the few-row statement matrices go first
        nxt = boolify(Ad + As @ P + boolify(Ld @ P) @ P + P.T @ boolify(St @ P))
        if nxt.nnz == P.nnz:
            return nxt
        P = nxt


def kinship_closure(r, a, b, comp):
    """Least fixpoint of kin(r,x,y) :- fact(r,x,y) and
    kin(r3,x,z) :- kin(r1,x,y), kin(r2,y,z), comp(r1,r2,r3), x != z
    by a worklist over facts: each new fact is composed with every known fact
    on either side (a different algorithm from naive iteration)."""
    c1, c2, c3 = comp
    table = defaultdict(list)
    for p, q, s in zip(c1.tolist(), c2.tolist(), c3.tolist()):
        table[(p, q)].append(s)
    known = set()
    by_src = defaultdict(set)  # x -> {(r, y)}
    by_dst = defaultdict(set)  # y -> {(r, x)}
    work = deque()

    def add(f):
        if f in known:
            return
        known.add(f)
        by_src[f[1]].add((f[0], f[2]))
        by_dst[f[2]].add((f[0], f[1]))
        work.append(f)

    for f in zip(r.tolist(), a.tolist(), b.tolist()):
        add(f)
    while work:
        r1, x, y = work.popleft()
        for r2, z in list(by_src[y]):  # (r1,x,y) then (r2,y,z)
            if x != z:
                for r3 in table[(r1, r2)]:
                    add((r3, x, z))
        for r0, w in list(by_dst[x]):  # (r0,w,x) then (r1,x,y)
            if w != y:
                for r3 in table[(r0, r1)]:
                    add((r3, w, y))
    return known


def possible_worlds_maxmin(facts, probs, closure):
    """Max-min tags by enumerating every subset W of the input facts: a key's
    tag is the max over W whose closure contains it of min over W of
    (p, -index) (the empty world's min is (1, -inf)).  Returns {key: (value, index)}."""
    m = len(facts)
    best = {}
    for mask in range(1 << m):
        W = [i for i in range(m) if mask >> i & 1]
        if W:
            lo = min(W, key=lambda i: (probs[i], -i))
            val = (float(probs[lo]), -lo)
        else:
            val = (1.0, -(2 ** 40))
        for k in closure([facts[i] for i in W]):
            if k not in best or val > best[k]:
                best[k] = val
    return {k: (v, -nid) for k, (v, nid) in best.items()}


def max_product_path(src, dst, p, source):
    """Most likely path from `source` to every reachable node (Dijkstra on the
    product of edge probabilities, all in [0, 1], so extending a path never
    makes it likelier): node -> (probability, edge indices of the path)."""
    adj = defaultdict(list)
    for e, (a, b, w) in enumerate(zip(src.tolist(), dst.tolist(), np.asarray(p, np.float64).tolist())):
        adj[a].append((b, w, e))
    best = {source: (1.0, [])}
    heap = [(-1.0, source)]
    done = set()
    while heap:
        negv, v = heapq.heappop(heap)
        if v in done:
            continue
        done.add(v)
        pv, path = best[v]
        for w, pw, e in adj[v]:
            c = pv * pw
            if w not in done and c > best.get(w, (-1.0, None))[0]:
                best[w] = (c, path + [e])
                heapq.heappush(heap, (-c, w))
    return best


def proof_is_path(src, dst, edge_ids, source, target):
    """The edges `edge_ids` form a simple path from source to target (in some order)."""
    out = {}
    for e in edge_ids:
        a = int(src[e])
        if a in out:
            return False
        out[a] = int(dst[e])
    v, seen = source, {source}
    for _ in range(len(edge_ids)):
        if v not in out:
            return False
        v = out[v]
        if v in seen:
            return False
        seen.add(v)
    return v == target
