"""Pins of the CPU oracle against facts fixed by the paper and by mathematics:
closed forms, textbook algorithms, brute-force possible worlds, finite
differences and invariants.  No expected value here comes from the engine."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2503_21937_gb300 import workloads as W
from tests import pins


def rel_set(rel):
    return set(map(tuple, rel.cols.T.tolist()))


# ----------------------------------------------------------------------------
# unit semiring: least fixpoint of the discrete program (Alg. 1; Sec. 3.1)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 5, 40])
def test_tc_chain_closed_form(n):
    a, b = W.ktree_chain(max(n, 2))
    a, b = a[: n - 1], b[: n - 1]
    if n == 1:
        a = b = np.zeros(0, np.uint32)
    r = oracle.run(W.TC_PROGRAM, {"edge": ((a, b),)})
    path = rel_set(r.relation("path"))
    assert len(path) == n * (n - 1) // 2
    assert path == {(i, j) for i in range(n) for j in range(i + 1, n)}


@pytest.mark.parametrize("n", [1, 3, 17])
def test_tc_cycle_and_complete_closed_form(n):
    a = np.arange(n, dtype=np.uint32)
    b = (a + 1) % n
    r = oracle.run(W.TC_PROGRAM, {"edge": ((a, b),)})
    assert len(rel_set(r.relation("path"))) == n * n
    x, y = np.meshgrid(np.arange(n), np.arange(n))
    keep = x != y
    r = oracle.run(W.TC_PROGRAM, {"edge": ((x[keep].astype(np.uint32), y[keep].astype(np.uint32)),)})
    # complete digraph without loops: every ordered pair, loops via 2-cycles (n >= 2)
    assert len(rel_set(r.relation("path"))) == (n * n if n >= 2 else 0)


def test_tc_matches_bfs_on_random_graphs():
    for n, m, seed in [(30, 60, 11), (200, 500, 12), (50, 400, 13)]:
        a, b = W.erdos_renyi(n, m, seed_index=seed)
        r = oracle.run(W.TC_PROGRAM, {"edge": ((a, b),)})
        assert rel_set(r.relation("path")) == pins.bfs_closure(a, b)


def test_scipy_closure_keys_equal_the_bfs_closure():
    """The vectorised closure the large engine checks use is the same set as
    the per-source BFS that pins the oracle."""
    for n, m, seed in [(30, 60, 14), (300, 700, 15), (100, 900, 16)]:
        a, b = W.erdos_renyi(n, m, seed_index=seed)
        keys = pins.closure_keys_scipy(a, b, n)
        assert np.all(keys[1:] > keys[:-1])
        want = pins.bfs_closure(a, b)
        assert {(int(k >> 32), int(k & 0xFFFFFFFF)) for k in keys} == want
    keys = pins.closure_keys_scipy(*W.ktree_chain(50), 50)
    assert len(keys) == 50 * 49 // 2


def test_sparse_matrix_andersen_matches_the_worklist_solver():
    """The boolean sparse-matrix fixpoint that checks the full-size Andersen
    run computes the same points-to set as the worklist solver pinned above."""
    for nv, ns, seed in [(3000, 8000, 31), (20000, 100000, 34)]:
        A = W.andersen_program(nv, ns, seed_index=seed)
        P = pins.andersen_sparse(A["addr"], A["assign"], A["load"], A["store"], nv).tocoo()
        got = set(zip(P.row.tolist(), P.col.tolist()))
        assert len(got) > 1000
        assert got == pins.andersen_worklist(A["addr"], A["assign"], A["load"], A["store"])


def test_sg_tree_depth_closed_form():
    parent, child, depth = W.random_tree(600, seed_index=21)
    r = oracle.run(W.SG_PROGRAM, {"parent": ((parent, child),)})
    sg = r.relation("sg")
    assert sg.cols.shape[1] == pins.same_generation_closed_form(depth)
    x, y = sg.cols
    assert np.all(depth[x] == depth[y]) and np.all(x != y) and np.all(depth[x] >= 1)
    keys = (x.astype(np.uint64) << np.uint64(32)) | y.astype(np.uint64)
    assert np.array_equal(keys, pins.same_generation_keys(depth))


@pytest.mark.parametrize("k,levels", [(2, 4), (3, 3)])
def test_sg_perfect_tree(k, levels):
    parent, child = W.perfect_tree(k, levels)
    r = oracle.run(W.SG_PROGRAM, {"parent": ((parent, child),)})
    expect = sum(k ** d * (k ** d - 1) for d in range(1, levels + 1))
    assert r.relation("sg").cols.shape[1] == expect


def test_andersen_matches_worklist_solver():
    A = W.andersen_program(3000, 8000, seed_index=31)
    inputs = {k: ((v[0], v[1]),) for k, v in A.items()}
    r = oracle.run(W.ANDERSEN_PROGRAM, inputs)
    expect = pins.andersen_worklist(A["addr"], A["assign"], A["load"], A["store"])
    got = rel_set(r.relation("pt"))
    assert len(expect) > 1000
    assert got == expect


def test_filters_constants_and_repeated_variables():
    edge = (np.array([0, 1, 1, 2, 3], np.uint32), np.array([1, 1, 2, 2, 0], np.uint32))
    prog = ("loop(x) :- edge(x,x).\n"
            "fromzero(y) :- edge(0,y).\n"
            "twohop(x,z) :- edge(x,y), edge(y,z), x != z.\n"
            "same(x) :- edge(x,y), x == 1.\n")
    r = oracle.run(prog, {"edge": (edge,)})
    assert rel_set(r.relation("loop")) == {(1,), (2,)}
    assert rel_set(r.relation("fromzero")) == {(1,)}
    E = set(zip(edge[0].tolist(), edge[1].tolist()))
    two = {(x, z) for (x, y) in E for (y2, z) in E if y == y2 and x != z}
    assert rel_set(r.relation("twohop")) == two
    assert rel_set(r.relation("same")) == {(1,)}


def test_duplicate_input_rows_are_merged():
    a = np.array([0, 0, 1], np.uint32)
    b = np.array([1, 1, 2], np.uint32)
    r = oracle.run(W.TC_PROGRAM, {"edge": ((a, b), np.array([0.2, 0.7, 0.5]))}, "max_min")
    p = r.relation("path")
    d = {tuple(c): t for c, t in zip(p.cols.T.tolist(), p.tags)}
    assert d[(0, 1)] == 0.7 and d[(0, 2)] == 0.5
    r = oracle.run(W.TC_PROGRAM, {"edge": ((a, b), np.array([0.2, 0.7, 0.5]))}, "add_mult")
    p = r.relation("path")
    d = {tuple(c): t for c, t in zip(p.cols.T.tolist(), p.tags)}
    assert d[(0, 1)] == pytest.approx(0.9) and d[(0, 2)] == pytest.approx(0.45)
    r = oracle.run(W.TC_PROGRAM, {"edge": ((a, b), np.array([0.6, 0.7, 0.5]))}, "add_mult")
    p = r.relation("path")
    d = {tuple(c): t for c, t in zip(p.cols.T.tolist(), p.tags)}
    assert d[(0, 1)] == 1.0  # clamped sum


# ----------------------------------------------------------------------------
# max-min-prob (semiring table of Sec. 3.1): possible worlds and widest paths
# ----------------------------------------------------------------------------

def small_graphs():
    out = []
    for m, seed in [(6, 41), (9, 42), (12, 43)]:
        s = W.stream(900 + seed)
        n = 5
        src = s.below(m, n)
        dst = s.below(m, n)
        p = s.prob(m).astype(np.float64)
        out.append((src, dst, p))
    # a graph with equal probabilities to exercise the id tie-break
    out.append((np.array([0, 0, 1, 2], np.uint32), np.array([1, 2, 3, 3], np.uint32), np.array([0.5] * 4)))
    return out


@pytest.mark.parametrize("g", range(4))
def test_maxmin_possible_worlds(g):
    src, dst, p = small_graphs()[g]
    inputs = {"edge": ((src, dst), p), "start": ((np.array([0], np.uint32),),)}
    truth = pins.possible_worlds_maxmin_reach(src, dst, p, 0)
    for sr in ("max_min", "diff_max_min"):
        r = oracle.run(W.REACH_PROGRAM, inputs, sr)
        rel = r.relation("reach")
        got = {int(c): t for c, t in zip(rel.cols[0], rel.tags)}
        assert set(got) == set(truth)
        for y, (v, _) in truth.items():
            assert got[y] == v
        if sr == "diff_max_min":
            ids = r.ids("reach")
            for c, i in zip(rel.cols[0], ids):
                want = truth[int(c)][1]
                # ids index the loaded rows in load order: edge rows first
                assert (i if i != 0xFFFFFFFF else 2 ** 40) == want


def test_maxmin_matches_widest_path_on_grid():
    g = W.grid_reach_instance(12, sub=5)
    src, dst, p = g["edge"]
    r = oracle.run(W.REACH_PROGRAM, {"edge": ((src, dst), p), "start": (g["start"],)}, "max_min")
    rel = r.relation("reach")
    best = pins.widest_path(src, dst, p, 0)
    got = {int(c): t for c, t in zip(rel.cols[0], rel.tags)}
    assert set(got) == set(best)
    for y in best:
        assert got[y] == pytest.approx(best[y], abs=0)
    vals = set(np.asarray(p, np.float64).tolist()) | {1.0}
    assert set(got.values()) <= vals


def test_maxmin_chain_is_min_of_edges():
    n = 9
    a, b = W.ktree_chain(n)
    p = W.stream(77).prob(n - 1).astype(np.float64)
    r = oracle.run(W.TC_PROGRAM, {"edge": ((a, b), p)}, "max_min")
    rel = r.relation("path")
    for (x, y), t in zip(rel.cols.T.tolist(), rel.tags):
        assert t == p[x:y].min()


# ----------------------------------------------------------------------------
# add-mult-prob: layered DP, lattice-path closed form, exact probability on trees
# ----------------------------------------------------------------------------

def test_addmult_reach_equals_layered_dp():
    for side, sub in [(7, 1), (16, 2)]:
        g = W.grid_reach_instance(side, sub=sub)
        src, dst, p = g["edge"]
        r = oracle.run(W.REACH_PROGRAM, {"edge": ((src, dst), p), "start": (g["start"],)}, "add_mult")
        rel = r.relation("reach")
        t, dist = pins.layered_reach_dp(src, dst, p, 0)
        got = {int(c): v for c, v in zip(rel.cols[0], rel.tags)}
        assert set(got) == set(t)
        for y in t:
            assert got[y] == pytest.approx(t[y], rel=1e-12)
        assert r.iterations == max(dist.values()) + 2  # one per layer, the source's rule, one empty


def test_addmult_grid_lattice_paths_closed_form():
    side = 6
    u, v = W.grid_edges(side)
    src, dst, tags = W.directed_from_undirected(u, v, np.full(len(u), 0.5, np.float32))
    r = oracle.run(W.REACH_PROGRAM, {"edge": ((src, dst), tags.astype(np.float64)),
                                     "start": ((np.array([0], np.uint32),),)}, "add_mult")
    rel = r.relation("reach")
    for c, t in zip(rel.cols[0], rel.tags):
        dx, dy = int(c) % side, int(c) // side
        assert t == pytest.approx(math.comb(dx + dy, dx) * 0.5 ** (dx + dy), rel=1e-14)


def test_addmult_tree_equals_possible_worlds_probability():
    # directed tree: one derivation per fact, so the tag is the exact probability
    parent, child = W.perfect_tree(2, 3)
    p = W.stream(78).prob(len(parent)).astype(np.float64)
    r = oracle.run(W.REACH_PROGRAM, {"edge": ((parent, child), p), "start": ((np.array([0], np.uint32),),)},
                   "add_mult")
    exact = pins.possible_worlds_probability(parent, child, p, 0)
    rel = r.relation("reach")
    got = {int(c): t for c, t in zip(rel.cols[0], rel.tags)}
    assert set(got) == set(exact)
    for y in exact:
        assert got[y] == pytest.approx(exact[y], rel=1e-12)


def test_addmult_counts_each_grounding_once_in_nonlinear_rule():
    # chain 0-1-2-3, every label 0, comp(0,0,0), p = 0.3: kin(0,0,2) first appears
    # at iteration 2 with one grounding (0.09); kin(0,0,3) first appears at
    # iteration 3 with two groundings, kin(0,0,1)+kin(0,1,3) and kin(0,0,2)+kin(0,2,3),
    # each 0.3 * 0.09, so its tag is their sum 0.054 (no clamp)
    fact = (np.zeros(3, np.uint32), np.array([0, 1, 2], np.uint32), np.array([1, 2, 3], np.uint32))
    comp = (np.zeros(1, np.uint32), np.zeros(1, np.uint32), np.zeros(1, np.uint32))
    r = oracle.run(W.KIN_PROGRAM, {"fact": (fact, np.full(3, 0.3)), "comp": (comp,)}, "add_mult")
    rel = r.relation("kin")
    d = {tuple(c): t for c, t in zip(rel.cols.T.tolist(), rel.tags)}
    assert d[(0, 0, 2)] == pytest.approx(0.09)
    # kin(0,0,3) appears at iteration 3 only via (0,2)+(2,3) and (0,1)+(1,3): 2 * 0.027
    assert d[(0, 0, 3)] == pytest.approx(2 * 0.027)


# ----------------------------------------------------------------------------
# invariants across semirings
# ----------------------------------------------------------------------------

def test_key_sets_agree_across_semirings_and_tag_ranges():
    g = W.grid_reach_instance(9, sub=3)
    src, dst, p = g["edge"]
    inputs = {"edge": ((src, dst), p), "start": (g["start"],)}
    keys = None
    for sr in ("unit", "max_min", "add_mult", "diff_max_min", "diff_add_mult"):
        rel = oracle.run(W.REACH_PROGRAM, inputs, sr).relation("reach")
        k = rel_set(rel)
        keys = k if keys is None else keys
        assert k == keys
        assert np.all(rel.tags >= 0) and np.all(rel.tags <= 1)
    assert len(keys) == 81


def test_batched_equals_per_sample():
    B = W.batched_instance(4)
    e = B["edge"]
    inputs = {"edge": ((e[0], e[1]), e[2], e[3]), "start": ((B["start"][0],), None, B["start"][2])}
    both = oracle.run(W.REACH_PROGRAM, inputs, "add_mult").relation("reach")
    for i in range(4):
        sel = e[3] == i
        one = oracle.run(W.REACH_PROGRAM, {"edge": ((e[0][sel], e[1][sel]), e[2][sel]),
                                           "start": ((np.array([0], np.uint32),),)}, "add_mult").relation("reach")
        m = both.samples == i
        assert np.array_equal(both.cols[:, m], one.cols)
        assert np.array_equal(both.tags[m], one.tags)


# ----------------------------------------------------------------------------
# gradients: forward-mode duals vs FP64 central finite differences
# ----------------------------------------------------------------------------

def _fd_check(program, inputs, rel_name, sr, gout, which, h=1e-6, tol=1e-4, skip=None):
    res = oracle.run(program, inputs, sr)
    grads = res.vjp({rel_name: gout})["edge"]
    base_rel = res.relation(rel_name)
    for e in which:
        if skip is not None and skip(e):
            continue
        vals = []
        for sign in (+1, -1):
            cols, p = inputs["edge"][0], np.array(inputs["edge"][1], np.float64)
            p[e] += sign * h
            inp = dict(inputs)
            inp["edge"] = (cols, p)
            rel = oracle.run(program, inp, sr.replace("diff_", "")).relation(rel_name)
            assert np.array_equal(rel.cols, base_rel.cols)
            vals.append(float(np.dot(rel.tags, gout)))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert grads[e] == pytest.approx(fd, abs=tol, rel=tol), (e, grads[e], fd)


def test_addmult_gradient_matches_finite_differences():
    side = 8
    g = W.grid_reach_instance(side, sub=9)
    src, dst, p = g["edge"]
    p = p.astype(np.float64) * 0.5  # keep sums away from the clamp
    inputs = {"edge": ((src, dst), p), "start": (g["start"],)}
    n_out = oracle.run(W.REACH_PROGRAM, inputs, "add_mult").relation("reach").cols.shape[1]
    gout = W.stream(55).normal(n_out)
    _fd_check(W.REACH_PROGRAM, inputs, "reach", "diff_add_mult", gout, range(len(src)))


def test_maxmin_gradient_matches_finite_differences():
    # one independent probability per directed fact, so each fact is its own input
    side = 6
    u, v = W.grid_edges(side)
    src, dst, _ = W.directed_from_undirected(u, v, np.zeros(len(u), np.float32))
    p = W.stream(57).prob(len(src)).astype(np.float64)
    inputs = {"edge": ((src, dst), p), "start": ((np.array([0], np.uint32),),)}
    n_out = oracle.run(W.REACH_PROGRAM, inputs, "max_min").relation("reach").cols.shape[1]
    gout = W.stream(56).normal(n_out)

    def near_tie(e):
        d = np.abs(p - p[e])
        d[e] = np.inf
        return d.min() < 2e-6

    _fd_check(W.REACH_PROGRAM, inputs, "reach", "diff_max_min", gout, range(len(src)), skip=near_tie)


def test_addmult_gradient_is_zero_through_a_clamped_sum():
    """(+) = min(1, a + b): an output whose summed derivations exceed 1 strictly
    is flat in every input, so its FP64 central differences are 0, while the
    unclamped outputs keep theirs.  Source 0 -> k middle nodes -> target, every
    edge probability 0.9: the target sums k * 0.81 > 1 for k >= 2."""
    k = 4
    mid = np.arange(1, k + 1, dtype=np.uint32)
    src = np.concatenate([np.zeros(k, np.uint32), mid])
    dst = np.concatenate([mid, np.full(k, k + 1, np.uint32)])
    p = np.full(2 * k, 0.9)
    inputs = {"edge": ((src, dst), p), "start": ((np.array([0], np.uint32),),)}
    res = oracle.run(W.REACH_PROGRAM, inputs, "add_mult")
    reach = res.relation("reach")
    assert reach.tags[list(reach.cols[0]).index(k + 1)] == 1.0  # clamped
    n_out = reach.cols.shape[1]
    target_only = np.zeros(n_out)
    target_only[list(reach.cols[0]).index(k + 1)] = 1.0
    _fd_check(W.REACH_PROGRAM, inputs, "reach", "diff_add_mult", target_only, range(len(src)))
    grads = oracle.run(W.REACH_PROGRAM, inputs, "diff_add_mult").vjp({"reach": target_only})["edge"]
    assert np.all(grads == 0.0)
    # a middle node is unclamped: d t(m) / d p(0 -> m) = 1
    middle_only = np.zeros(n_out)
    middle_only[list(reach.cols[0]).index(1)] = 1.0
    _fd_check(W.REACH_PROGRAM, inputs, "reach", "diff_add_mult", middle_only, range(len(src)))


# ----------------------------------------------------------------------------
# the paper's printed example and semiring table (tests/golden/, cited there)
# ----------------------------------------------------------------------------

def test_pathfinder_example_from_the_paper():
    from tests.golden.load import pathfinder_example, provenance_semirings
    program, inputs = pathfinder_example()
    table = provenance_semirings()
    chain = [0.9, 0.8, 0.95, 0.85]
    # Bool: the discrete result; 5 cannot reach 1, and x != y drops (x, x)
    r = oracle.run(program, inputs, "unit")
    assert rel_set(r.relation("connected")) == {(1, 5)}
    assert (0, 1) in rel_set(r.relation("path")) and (1, 5) in rel_set(r.relation("path"))
    # Max-Min-Prob: (x) = min along the single proof, (+) = max; endpoint facts
    # carry the semiring's 1, the identity of min
    assert table["max_min"]["otimes"] == "min" and table["max_min"]["one"] == 1.0
    r = oracle.run(program, inputs, "max_min")
    path = r.relation("path")
    tag = dict(zip(map(tuple, path.cols.T.tolist()), path.tags.tolist()))
    assert tag[(0, 1)] == 0.97  # the printed fact 0.97::edge(0, 1)
    assert tag[(0, 5)] == min([0.97] + chain)
    conn = r.relation("connected")
    assert conn.tags.tolist() == [min(chain)]
    # add-mult: the single proof's probability is the product of its facts
    r = oracle.run(program, inputs, "add_mult")
    assert r.relation("connected").tags[0] == pytest.approx(math.prod(chain), rel=1e-12)


# ----------------------------------------------------------------------------
# kinship composition (the batched workload's non-linear program)
# ----------------------------------------------------------------------------

def test_kinship_unit_matches_worklist_closure():
    for seed in (140, 141, 142):
        n, r, a, b, p = W.kinship_instance(W.stream(seed))
        comp = W.composition_table()
        res = oracle.run(W.KIN_PROGRAM, {"fact": ((r, a, b),), "comp": (comp,)})
        assert rel_set(res.relation("kin")) == pins.kinship_closure(r, a, b, comp)


def test_kinship_maxmin_possible_worlds():
    s = W.stream(143)
    labels = 3
    r = s.below(9, labels).astype(np.uint32)
    a = s.below(9, 5).astype(np.uint32)
    b = ((a + 1 + s.below(9, 4)) % 5).astype(np.uint32)  # no self pairs
    p = s.prob(9).astype(np.float64)
    comp = tuple(np.asarray(c, np.uint32) for c in zip(*[(i, j, (i + 2 * j + 1) % labels)
                                                           for i in range(labels) for j in range(labels)]))
    facts = list(zip(r.tolist(), a.tolist(), b.tolist()))
    if len(set(facts)) != len(facts):  # the enumeration treats facts as distinct inputs
        pytest.skip("duplicate facts in this draw")
    res = oracle.run(W.KIN_PROGRAM, {"fact": ((r, a, b), p), "comp": (comp,)}, "diff_max_min")
    kin = res.relation("kin")
    ids = res.ids("kin")
    want = pins.possible_worlds_maxmin(facts, p, lambda fs: pins.kinship_closure(
        np.array([f[0] for f in fs], np.int64), np.array([f[1] for f in fs], np.int64),
        np.array([f[2] for f in fs], np.int64), comp) if fs else set())
    got = {tuple(k): (float(v), int(i)) for k, v, i in zip(kin.cols.T.tolist(), kin.tags, ids)}
    assert set(got) == set(want)
    for k, (v, i) in want.items():
        assert got[k][0] == v, k
        assert got[k][1] == i, k


# ----------------------------------------------------------------------------
# top-1-proofs (Sec. 5.3 "Limitations"; Sec. 3.4): one proof per fact, (x) =
# union of proofs, (+) = the more likely proof
# ----------------------------------------------------------------------------

def _f32(x):
    return float(np.float32(x))


@pytest.mark.parametrize("g", range(3))
def test_top1_reach_is_the_most_likely_path(g):
    """On reachability every kept proof is a simple path, so the tag of reach(y)
    is the probability of the most likely path (Dijkstra on products)."""
    src, dst, p = small_graphs()[g]
    inputs = {"edge": ((src, dst), p), "start": ((np.array([0], np.uint32),),)}
    best = pins.max_product_path(src, dst, p, 0)
    for sr in ("top1_proofs", "diff_top1_proofs"):
        r = oracle.run(W.REACH_PROGRAM, inputs, sr)
        assert r.ties == 0
        rel = r.relation("reach")
        proofs = r.proofs("reach")
        assert set(rel.cols[0].tolist()) == set(best)
        for y, t, pr in zip(rel.cols[0].tolist(), rel.tags.tolist(), proofs):
            assert t == pytest.approx(best[y][0], rel=1e-6)
            assert sorted(pr.tolist()) == sorted(best[y][1])  # edge rows come first in load order
            assert pins.proof_is_path(src, dst, pr.tolist(), 0, y)
            assert t == _f32(math.prod(np.asarray(p, np.float64)[pr].tolist()))


def test_top1_grid_paths_against_dijkstra():
    g = W.grid_reach_instance(10, sub=3)
    src, dst, p = g["edge"]
    r = oracle.run(W.REACH_PROGRAM, {"edge": ((src, dst), p), "start": (g["start"],)}, "top1_proofs")
    best = pins.max_product_path(src, dst, p, 0)
    rel = r.relation("reach")
    proofs = r.proofs("reach")
    assert len(rel.cols[0]) == len(best) == 100
    for y, t, pr in zip(rel.cols[0].tolist(), rel.tags.tolist(), proofs):
        assert t == pytest.approx(best[y][0], rel=1e-6)
        assert pins.proof_is_path(src, dst, pr.tolist(), 0, y)


def test_top1_a_fact_used_twice_counts_once():
    """(x) is the union of proofs: a(x), a(x) has the probability of a(x)."""
    pa = np.array([0.5, 0.25, 0.8])
    pb = np.array([0.4, 0.9, 0.3])
    x = np.array([0, 1, 2], np.uint32)
    prog = "q(x) :- a(x), a(x).\nr(x) :- a(x), b(x), a(x).\n"
    r = oracle.run(prog, {"a": ((x,), pa), "b": ((x,), pb)}, "top1_proofs")
    q, rr = r.relation("q"), r.relation("r")
    assert q.tags.tolist() == [_f32(v) for v in pa]
    assert [p.tolist() for p in r.proofs("q")] == [[0], [1], [2]]
    assert rr.tags.tolist() == [_f32(a * b) for a, b in zip(pa, pb)]
    assert [p.tolist() for p in r.proofs("r")] == [[0, 3], [1, 4], [2, 5]]


def test_top1_two_hop_is_the_best_middle_vertex():
    """t(x,z) :- e(x,y), f(y,z): the most likely grounding over y (brute force)."""
    s = W.stream(4242)
    n, m = 6, 30
    e = (s.below(m, n), s.below(m, n))
    f = (s.below(m, n), s.below(m, n))
    pe, pf = s.prob(m).astype(np.float64), s.prob(m).astype(np.float64)
    r = oracle.run("t(x,z) :- e(x,y), f(y,z).\n", {"e": (e, pe), "f": (f, pf)}, "top1_proofs")
    # distinct input rows (duplicates keep the likelier row)
    def best_rows(cols, p):
        d = {}
        for i, k in enumerate(zip(*[c.tolist() for c in cols])):
            if k not in d or p[i] > p[d[k]]:
                d[k] = i
        return d
    de, df = best_rows(e, pe), best_rows(f, pf)
    want = {}
    for (x, y), i in de.items():
        for (y2, z), j in df.items():
            if y2 != y:
                continue
            v = _f32(pe[i] * pf[j])
            if (x, z) not in want or v > want[(x, z)][0]:
                want[(x, z)] = (v, [i, m + j])
    assert r.ties == 0
    rel = r.relation("t")
    got = {k: (t, pr.tolist()) for k, t, pr in zip(map(tuple, rel.cols.T.tolist()), rel.tags.tolist(), r.proofs("t"))}
    assert got == want


def test_top1_pathfinder_example_proof_from_the_paper():
    """The proof of connected(1,5) is the chain edge(1,2), ..., edge(4,5) that the
    paper's Sec. 2 example prints; the endpoint facts carry no probability and
    join the proof as the empty conjunction."""
    from tests.golden.load import pathfinder_example
    program, inputs = pathfinder_example()
    chain = [0.9, 0.8, 0.95, 0.85]
    r = oracle.run(program, inputs, "top1_proofs")
    conn = r.relation("connected")
    assert rel_set(conn) == {(1, 5)}
    assert [p.tolist() for p in r.proofs("connected")] == [[1, 2, 3, 4]]  # edge rows 1..4 of the fixture
    assert conn.tags.tolist() == [_f32(math.prod(chain))]
    path = r.relation("path")
    tag = dict(zip(map(tuple, path.cols.T.tolist()), path.tags.tolist()))
    assert tag[(0, 1)] == _f32(0.97)


def test_top1_proof_cap_is_enforced():
    n = 9
    a, b = W.ktree_chain(n)
    p = np.full(n - 1, 0.5)
    inputs = {"edge": ((a, b), p), "start": ((np.array([0], np.uint32),),)}
    with pytest.raises(oracle.OracleError) as ei:
        oracle.run(W.REACH_PROGRAM, inputs, "top1_proofs", proof_cap=5)
    assert ei.value.code == -5
    r = oracle.run(W.REACH_PROGRAM, inputs, "top1_proofs", proof_cap=8)
    pr = r.proofs("reach")
    assert [len(x) for x in pr] == list(range(n))
    assert r.relation("reach").tags[-1] == 0.5 ** 8


def test_top1_proofs_are_valid_derivations_on_kinship():
    """Every kept proof derives its fact on its own (the unit fixpoint over the
    proof's facts plus the facts without a probability contains it), and the tag
    is the product of the proof's probabilities."""
    n, rr, a, b, p = W.kinship_instance(W.stream(143))
    comp = W.composition_table()
    inputs = {"fact": ((rr, a, b), p), "comp": (comp,)}
    r = oracle.run(W.KIN_PROGRAM, inputs, "top1_proofs")
    kin = r.relation("kin")
    proofs = r.proofs("kin")
    s = W.stream(99)
    picks = s.below(min(40, len(proofs)), len(proofs)).tolist()
    for i in picks:
        pr = proofs[i]
        assert kin.tags[i] == _f32(math.prod(p.astype(np.float64)[pr].tolist()))
        sub = {"fact": ((rr[pr], a[pr], b[pr]),), "comp": (comp,)}
        got = rel_set(oracle.run(W.KIN_PROGRAM, sub, "unit").relation("kin"))
        assert tuple(kin.cols[:, i].tolist()) in got


def test_top1_gradient_matches_finite_differences():
    src, dst, p = small_graphs()[2]
    inputs = {"edge": ((src, dst), p), "start": ((np.array([0], np.uint32),),)}
    n_out = oracle.run(W.REACH_PROGRAM, inputs, "top1_proofs").relation("reach").cols.shape[1]
    gout = W.stream(56).normal(n_out)
    # the tags are products rounded to f32: a wide step keeps the rounding
    # error small, and a product is linear in each factor, so the central
    # difference has no truncation error
    _fd_check(W.REACH_PROGRAM, inputs, "reach", "diff_top1_proofs", gout, range(len(src)), h=1e-3)


# ----------------------------------------------------------------------------
# computed projections and selections (Sec. 5.2): u32 arithmetic in head
# arguments, comparisons in filters
# ----------------------------------------------------------------------------

def test_bounded_walk_lengths_match_boolean_matrix_powers():
    """walk(y, d+1) :- walk(x, d), edge(x, y), d < L: walk(y, k) holds iff some
    walk of exactly k <= L edges leads from node 0 to y (powers of the
    adjacency matrix)."""
    s = W.stream(4343)
    n, m, L = 9, 20, 6
    src, dst = s.below(m, n), s.below(m, n)
    prog = ("walk(x, 0) :- start(x).\n"
            "walk(y, d + 1) :- walk(x, d), edge(x, y), d < %d.\n" % L)
    r = oracle.run(prog, {"edge": ((src, dst),), "start": ((np.array([0], np.uint32),),)})
    A = np.zeros((n, n), bool)
    A[src, dst] = True
    want, v = set(), np.zeros(n, bool)
    v[0] = True
    for k in range(L + 1):
        want |= {(int(y), k) for y in np.nonzero(v)[0]}
        v = (v[:, None] & A).any(axis=0)
    assert rel_set(r.relation("walk")) == want


def test_arithmetic_wraps_and_drops():
    x = np.array([0, 1, 5, 7, 4000000000, 3], np.uint32)
    y = np.array([0, 3, 5, 2, 3000000000, 0], np.uint32)
    prog = ("diff(x, y - x) :- p(x, y), x <= y.\n"
            "quot(x, x / y) :- p(x, y).\n"
            "prod(x, x * y + 1) :- p(x, y).\n"
            "pred(x - 1) :- p(x, y).\n"
            "big(x) :- p(x, y), x + y > y * 2, (x - y) / 2 >= 1.\n")
    r = oracle.run(prog, {"p": ((x, y),)})
    pairs = list(zip(x.tolist(), y.tolist()))
    M = 1 << 32
    assert rel_set(r.relation("diff")) == {(a, b - a) for a, b in pairs if a <= b}
    assert rel_set(r.relation("quot")) == {(a, a // b) for a, b in pairs if b}  # a zero divisor drops the row
    assert rel_set(r.relation("prod")) == {(a, (a * b + 1) % M) for a, b in pairs}
    assert rel_set(r.relation("pred")) == {((a - 1) % M,) for a, b in pairs if a != 0}  # 2^32-1 is reserved
    assert rel_set(r.relation("big")) == {(a,) for a, b in pairs
                                          if (a + b) % M > (b * 2) % M and ((a - b) % M) // 2 >= 1}


# ----------------------------------------------------------------------------
# strata (Sec. 3.1; Algorithm 1's loop over the strata of a program): each
# stratum runs to its fixpoint before the next one reads its relations
# ----------------------------------------------------------------------------

def _chain(n, seed):
    """Chain 0 -> 1 -> ... -> n-1 with probabilities below 1/2, so that sums of
    path products stay below 1 (no clamp), and its path products P[x][y]."""
    a = np.arange(n - 1, dtype=np.uint32)
    p = W.stream(seed).prob(n - 1).astype(np.float64) * 0.5
    P = {}
    for x in range(n):
        v = 1.0
        for y in range(x + 1, n):
            v *= p[y - 1]
            P[x, y] = v
    return (a, a + 1), p, P


@pytest.mark.parametrize("reverse", [False, True])
def test_strata_projection_sums_every_path_of_the_closure(reverse):
    """out(x) :- path(x,y) in the stratum above the closure: on a chain every
    path fact has one derivation (the product of its edges), and out(x) sums
    all of them -- min(1, sum_{y > x} P[x][y]) -- because the closure is complete
    before out is derived.  Rules written above the rules they read must give
    the same result."""
    n = 9
    cols, p, P = _chain(n, 6100)
    rules = [W.TC_PROGRAM, "out(x) :- path(x,y).\n"]
    prog = "".join(reversed(rules) if reverse else rules)
    r = oracle.run(prog, {"edge": (cols, p)}, "add_mult")
    path = {tuple(c): t for c, t in zip(r.relation("path").cols.T.tolist(), r.relation("path").tags)}
    assert set(path) == set(P)
    for k in P:
        assert path[k] == pytest.approx(P[k], rel=1e-12)
    out = {int(c): t for c, t in zip(r.relation("out").cols[0], r.relation("out").tags)}
    assert set(out) == set(range(n - 1))
    for x in range(n - 1):
        want = min(1.0, sum(P[x, y] for y in range(x + 1, n)))
        assert out[x] == pytest.approx(want, rel=1e-12)


def test_strata_mutually_recursive_relations_share_one_stratum():
    """odd/even path lengths depend on each other, so they are evaluated
    together; cnt(x) :- even(x,y) above them sums every even-length path of
    the chain: min(1, sum over y - x even >= 2 of P[x][y])."""
    n = 10
    cols, p, P = _chain(n, 6200)
    r = oracle.run(W.ODD_EVEN_PROGRAM, {"edge": (cols, p)}, "add_mult")
    odd = {tuple(c): t for c, t in zip(r.relation("odd").cols.T.tolist(), r.relation("odd").tags)}
    even = {tuple(c): t for c, t in zip(r.relation("even").cols.T.tolist(), r.relation("even").tags)}
    assert set(odd) == {k for k in P if (k[1] - k[0]) % 2 == 1}
    assert set(even) == {k for k in P if (k[1] - k[0]) % 2 == 0}
    for k, t in list(odd.items()) + list(even.items()):
        assert t == pytest.approx(P[k], rel=1e-12)
    cnt = {int(c): t for c, t in zip(r.relation("cnt").cols[0], r.relation("cnt").tags)}
    assert set(cnt) == set(range(n - 2))
    for x in range(n - 2):
        want = min(1.0, sum(P[x, y] for y in range(x + 2, n, 2)))
        assert cnt[x] == pytest.approx(want, rel=1e-12)


def test_strata_three_layers_sum_over_middle_vertices():
    """LAYERED on a chain: src(x) = sum_y P[x][y]; far(x,z) sums, over the middle
    vertices x < y < z, src(x) * P[x][y] * P[y][z] = src(x) * (z - x - 1) *
    P[x][z], clamped to 1."""
    n = 8
    cols, p, P = _chain(n, 6300)
    r = oracle.run(W.LAYERED_PROGRAM, {"edge": (cols, p)}, "add_mult")
    src = {x: min(1.0, sum(P[x, y] for y in range(x + 1, n))) for x in range(n - 1)}
    far = {tuple(c): t for c, t in zip(r.relation("far").cols.T.tolist(), r.relation("far").tags)}
    want = {(x, z): min(1.0, src[x] * (z - x - 1) * P[x, z]) for x in range(n) for z in range(x + 2, n)}
    assert set(far) == set(want)
    for k in want:
        assert far[k] == pytest.approx(want[k], rel=1e-12)


def test_strata_maxmin_reads_the_widest_paths():
    """max-min: q(x,z) :- path(x,y), hop(y,z) above the closure is
    max_y min(W[x][y], hop(y,z)) with W the widest-path (max over paths of the
    smallest edge) matrix from Floyd-Warshall."""
    s = W.stream(6400)
    n, m = 8, 18
    a, b = W.erdos_renyi(n, m, seed_index=6401)
    pe = s.prob(len(a)).astype(np.float32).astype(np.float64)
    ha, hb = s.below(6, n), s.below(6, n)
    keep = np.unique(np.stack([ha, hb]), axis=1)
    ha, hb = keep[0].astype(np.uint32), keep[1].astype(np.uint32)
    ph = s.prob(len(ha)).astype(np.float32).astype(np.float64)
    Wm = np.zeros((n, n))
    for x, y, t in zip(a, b, pe):
        Wm[x, y] = max(Wm[x, y], t)
    for k in range(n):
        Wm = np.maximum(Wm, np.minimum(Wm[:, k:k + 1], Wm[k:k + 1, :]))
    prog = W.TC_PROGRAM + "q(x,z) :- path(x,y), hop(y,z).\n"
    r = oracle.run(prog, {"edge": ((a, b), pe), "hop": ((ha, hb), ph)}, "max_min")
    want = {}
    for x in range(n):
        for y, z, t in zip(ha, hb, ph):
            if Wm[x, y] > 0:
                want[x, int(z)] = max(want.get((x, int(z)), 0.0), min(Wm[x, y], t))
    got = {tuple(c): t for c, t in zip(r.relation("q").cols.T.tolist(), r.relation("q").tags)}
    assert want and got == want


def test_strata_gradient_matches_finite_differences():
    a, b = W.erdos_renyi(12, 26, seed_index=6500)
    p = W.stream(6501).prob(len(a)).astype(np.float64) * 0.3
    inputs = {"edge": ((a, b), p)}
    n_out = oracle.run(W.LAYERED_PROGRAM, inputs, "add_mult").relation("far").cols.shape[1]
    assert n_out > 10
    gout = W.stream(6502).normal(n_out)
    _fd_check(W.LAYERED_PROGRAM, inputs, "far", "diff_add_mult", gout, range(len(a)))


def test_top1_strata_read_the_finished_proofs_of_the_stratum_below():
    """top-1-proofs under strata: h(y) :- r(y), s(y) sits above r and s, so it
    reads their final proofs.  r(2) first gets the proof {e(0,2)} (0.5), then the
    likelier {e(0,1), e(1,2)} (0.81); s(2) has {e(0,2)}.  Run after r and s are
    complete, h(2) = their union {e(0,1), e(1,2), e(0,2)} = 0.9 * 0.9 * 0.5;
    h(1) = {e(0,1)} = 0.9.  (One loop over every rule would have kept the union
    with r(2)'s first proof, {e(0,2)} = 0.5.)"""
    prog = ("r(x) :- start(x).\n"
            "r(y) :- r(x), e(x,y).\n"
            "s(y) :- e(0,y).\n"
            "h(y) :- r(y), s(y).\n")
    e = (np.array([0, 1, 0], np.uint32), np.array([1, 2, 2], np.uint32))
    p = np.array([0.9, 0.9, 0.5])
    r = oracle.run(prog, {"e": (e, p), "start": ((np.array([0], np.uint32),),)}, "top1_proofs")
    assert r.ties == 0
    rel = r.relation("h")
    got = {int(c): (t, pr.tolist()) for c, t, pr in zip(rel.cols[0], rel.tags.tolist(), r.proofs("h"))}
    assert got == {1: (_f32(0.9), [0]), 2: (_f32(0.9 * 0.9 * 0.5), [0, 1, 2])}


def test_strata_keep_loaded_facts_of_a_derived_relation():
    """add-mult, out(x) :- path(x,y) above the closure of a chain, with out(0)
    also loaded (tag 0.25): a loaded key keeps its tag (first appearance), the
    other keys sum every path of the closure, and a sample of its own runs its
    own strata (the same program on a second, shorter chain)."""
    n = 7
    cols, p, P = _chain(n, 6600)
    prog = W.TC_PROGRAM + "out(x) :- path(x,y).\n"
    a, b = cols
    m = 4  # sample 1: the chain's first m nodes
    edge = ((np.concatenate([a, a[:m - 1]]), np.concatenate([b, b[:m - 1]])),
            np.concatenate([p, p[:m - 1]]), np.concatenate([np.zeros(n - 1, np.uint32), np.ones(m - 1, np.uint32)]))
    out_in = ((np.array([0], np.uint32),), np.array([0.25]), np.array([0], np.uint32))
    r = oracle.run(prog, {"edge": edge, "out": out_in}, "add_mult")
    rel = r.relation("out")
    got = {(int(s), int(c)): t for s, c, t in zip(rel.samples, rel.cols[0], rel.tags)}
    want = {(0, 0): 0.25}
    want.update({(0, x): min(1.0, sum(P[x, y] for y in range(x + 1, n))) for x in range(1, n - 1)})
    want.update({(1, x): min(1.0, sum(P[x, y] for y in range(x + 1, m))) for x in range(m - 1)})
    assert set(got) == set(want)
    for k in want:
        assert got[k] == pytest.approx(want[k], rel=1e-12), k


def test_strata_diamond_written_bottom_up():
    """A diamond of strata, rules written with the top first: path (the chain's
    closure), then b(x) = sum over successors and c(y) = sum over predecessors,
    then d(x) :- b(x), c(x) with one grounding per x: d(x) = b(x) * c(x)."""
    n = 8
    cols, p, P = _chain(n, 6700)
    prog = ("d(x) :- b(x), c(x).\n"
            "c(y) :- path(x,y).\n"
            "b(x) :- path(x,y).\n" + W.TC_PROGRAM)
    r = oracle.run(prog, {"edge": (cols, p)}, "add_mult")
    b = {x: min(1.0, sum(P[x, y] for y in range(x + 1, n))) for x in range(n - 1)}
    c = {y: min(1.0, sum(P[x, y] for x in range(y))) for y in range(1, n)}
    rel = r.relation("d")
    got = {int(x): t for x, t in zip(rel.cols[0], rel.tags)}
    assert set(got) == set(range(1, n - 1))
    for x in got:
        assert got[x] == pytest.approx(min(1.0, b[x] * c[x]), rel=1e-12), x
