"""The synthetic inputs follow the recipe the design states (seeded, with the
sizes, distributions and structure of the paper's workloads): deterministic
per seed, distinct edges, the tree's branching and relabelling, the grid's
shape, power-law skew, statement mix and batching."""
import numpy as np

from paper_2503_21937_gb300 import workloads as W


def test_streams_are_deterministic_and_independent():
    a = W.stream(3, 1).below(1000, 10**6)
    b = W.stream(3, 1).below(1000, 10**6)
    c = W.stream(3, 2).below(1000, 10**6)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    p = W.stream(4).prob(10000)
    assert p.dtype == np.float32 and p.min() > 0 and p.max() < 1


def test_erdos_renyi_distinct_edges_no_loops():
    s, d = W.erdos_renyi(1000, 3000)
    assert len(s) == 3000 and np.all(s != d)
    assert len(set(zip(s.tolist(), d.tolist()))) == 3000
    assert s.max() < 1000 and d.max() < 1000


def test_random_tree_branching_and_levels():
    parent, child, depth = W.random_tree(50_000)
    assert len(child) == 49_999 and len(np.unique(child)) == 49_999  # every non-root node once
    kids = np.bincount(parent, minlength=50_000)
    internal = kids[kids > 0]
    assert internal.min() >= 1 and internal.max() <= 4  # U{1..4} children per expanded node
    assert depth.max() == 11 and (depth == 0).sum() == 1  # 12 levels
    assert np.all(depth[child] == depth[parent] + 1)
    assert not np.array_equal(np.sort(child), np.arange(1, 50_000))  # ids relabelled


def test_chung_lu_power_law_skew():
    s, d = W.chung_lu_power_law(20_000, 100_000)
    assert len(s) == 100_000 and np.all(s != d)
    assert len(set(zip(s.tolist(), d.tolist()))) == 100_000
    out = np.bincount(s, minlength=20_000)
    # heavy tail: the top 1 % of sources hold far more than 1 % of the edges
    top = np.sort(out)[::-1][:200].sum()
    assert top > 0.15 * 100_000 and out.max() > 50 * out.mean()


def test_grid_reach_shape():
    g = W.grid_reach_instance(64)
    src, dst, p = g["edge"]
    assert len(src) == 2 * 2 * 64 * 63  # undirected edges, both directions
    assert len(g["p_undirected"]) == 2 * 64 * 63
    diff = np.abs(src.astype(np.int64) - dst.astype(np.int64))
    assert set(np.unique(diff).tolist()) == {1, 64}


def test_andersen_statement_mix():
    A = W.andersen_program(200_000, 1_000_000)
    n = {k: len(v[0]) for k, v in A.items()}
    assert set(n) == {"addr", "assign", "load", "store"}
    assert sum(n.values()) <= 1_000_000  # distinct statements after dedup
    for k, v in A.items():
        assert v[0].max() < 200_000 and v[1].max() < 200_000


def test_batched_instance_sample_ids():
    B = W.batched_instance(16)
    e, f = B["edge"], B["fact"]
    assert set(np.unique(e[3]).tolist()) == set(range(16))
    assert set(np.unique(f[4]).tolist()) <= set(range(16))
    assert e[2].dtype == np.float32
