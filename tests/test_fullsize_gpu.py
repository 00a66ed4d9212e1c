"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (default engine options).  Where the naive oracle cannot finish, the
outputs are checked on samples against textbook computations pinned to the
oracle (tests/pins.py) and against properties that hold at any size."""
import numpy as np
import pytest

from paper_2503_21937_gb300 import workloads as W
from tests import pins
from tests.common import oracle_run

pytestmark = pytest.mark.gpu


def _engine(program, inputs, semiring="unit"):
    import torch
    from paper_2503_21937_gb300 import Engine, build
    build.build()
    e = Engine()
    e.program(program)
    for name, spec in inputs.items():
        if isinstance(spec, np.ndarray):
            spec = (spec,)
        cols, tags, samples = (list(spec) + [None, None])[:3]
        e.load(name, torch.from_numpy(np.asarray(cols).astype(np.int32)).cuda(),
               None if tags is None else torch.from_numpy(np.asarray(tags, np.float32)).cuda(),
               None if samples is None else torch.from_numpy(np.asarray(samples).astype(np.int32)).cuda())
    st = e.run(semiring)
    return e, st


def _strictly_sorted_pairs(cols):
    import torch
    k = (cols[0].to(torch.int64) << 32) | cols[1].to(torch.int64)
    return bool(torch.all(k[1:] > k[:-1]).item())


def test_same_generation_50k_tree():
    parent, child, depth = W.random_tree(50_000)
    e, st = _engine(W.SG_PROGRAM, {"parent": np.stack([parent, child])})
    rel = e.read("sg", device=True)
    n = rel.cols.shape[1]
    assert n == pins.same_generation_closed_form(depth) == st["derived"]
    assert _strictly_sorted_pairs(rel.cols)  # distinct facts, read order
    idx = np.unique(W.stream(990).below(1_000_000, n))
    import torch
    x = rel.cols[0][torch.from_numpy(idx.astype(np.int64)).cuda()].cpu().numpy()
    y = rel.cols[1][torch.from_numpy(idx.astype(np.int64)).cuda()].cpu().numpy()
    assert np.all(depth[x] == depth[y]) and np.all(depth[x] >= 1) and np.all(x != y)
    e.close()


def test_transitive_closure_power_law_20k():
    import torch
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import breadth_first_order
    s, d = W.chung_lu_power_law(20_000, 100_000)
    e, st = _engine(W.TC_PROGRAM, {"edge": np.stack([s, d])})
    rel = e.read("path", device=True)
    assert _strictly_sorted_pairs(rel.cols)
    x = rel.cols[0].cpu().numpy()
    y = rel.cols[1].cpu().numpy()
    g = csr_matrix((np.ones(len(s)), (s, d)), shape=(20_000, 20_000))
    gt = g.T.tocsr()
    starts = np.searchsorted(x, np.arange(20_001))
    for src in np.unique(W.stream(991).below(64, 20_000)).tolist() + [int(np.argmax(np.bincount(s)))]:
        order = breadth_first_order(g, src, directed=True, return_predecessors=False)
        reach = set(order[1:].tolist())
        preds = gt.indices[gt.indptr[src]:gt.indptr[src + 1]]
        if np.isin(preds, order).any():  # a cycle leads back to src
            reach.add(src)
        got = y[starts[src]:starts[src + 1]]
        assert np.array_equal(got, np.array(sorted(reach), np.uint32)), src
    e.close()


@pytest.mark.parametrize("semiring", ["diff_add_mult", "diff_max_min"])
def test_grid_64_forward_and_gradients(semiring):
    g = W.grid_reach_instance(64)
    src, dst, p = g["edge"]
    inputs = {"edge": ((src, dst), p), "start": (g["start"],)}
    res = oracle_run(W.REACH_PROGRAM, inputs, semiring)
    want = res.relation("reach")
    e, st = _engine(W.REACH_PROGRAM, {"edge": (np.stack([src, dst]), p), "start": (np.zeros((1, 1), np.uint32),)},
                    semiring)
    got = e.read("reach")
    assert np.array_equal(got.cols, want.cols)
    if semiring == "diff_max_min":
        assert np.array_equal(got.tags, want.tags.astype(np.float32))
    else:
        np.testing.assert_allclose(got.tags, want.tags, rtol=1e-5, atol=0)
    gout = W.stream(992).normal(want.cols.shape[1])
    gw = res.vjp({"reach": gout})["edge"]
    gin = {"edge": np.zeros(len(src), np.float32)}
    e.backward("reach", gout.astype(np.float32), gin)
    np.testing.assert_allclose(gin["edge"], gw, rtol=1e-4, atol=1e-4)
    e.close()


def test_andersen_200k_vars_1m_statements():
    A = W.andersen_program(200_000, 1_000_000)
    e, st = _engine(W.ANDERSEN_PROGRAM, {k: np.stack([v[0], v[1]]) for k, v in A.items()})
    rel = e.read("pt")
    P = pins.andersen_sparse(A["addr"], A["assign"], A["load"], A["store"], 200_000).tocsr()
    P.sort_indices()
    r = np.repeat(np.arange(200_000), np.diff(P.indptr))
    assert rel.cols.shape[1] == P.nnz
    assert np.array_equal(rel.cols[0], r.astype(np.uint32))
    assert np.array_equal(rel.cols[1], P.indices.astype(np.uint32))
    e.close()


def _spread_samples(sides, k=8):
    """k sample ids spread over the side range, the smallest and largest side included."""
    order = np.argsort(sides, kind="stable")
    pick = np.unique(np.linspace(0, len(order) - 1, k).round().astype(int))
    return sorted(int(order[i]) for i in pick)


@pytest.mark.parametrize("semiring", ["diff_add_mult", "diff_max_min"])
def test_batched_512_samples_sampled_against_oracle(semiring):
    """One launch over all 512 samples (grid reachability + kinship composition),
    forward and backward from both outputs.  Eight samples spread over the side
    range are checked against the oracle run on that sample alone (a batched
    run restricted to sample i equals the single run of sample i): tags of
    reach and kin (bitwise for max-min, 1e-5 relative for add-mult) and the
    gradients of both inputs (1e-4).  For max-min the gradient of an output
    lands on the input fact that bounds its tag, so matching gradients under a
    random upstream gradient also check those input ids."""
    B = W.batched_instance(512)
    program = W.REACH_PROGRAM + W.KIN_PROGRAM
    e_, f, c, st = B["edge"], B["fact"], B["comp"], B["start"]
    inputs = {"edge": (np.stack([e_[0], e_[1]]), e_[2], e_[3]), "start": (st[0][None, :], None, st[2]),
              "fact": (np.stack([f[0], f[1], f[2]]), f[3], f[4]), "comp": (np.stack([c[0], c[1], c[2]]), None, c[4])}
    e, stats = _engine(program, inputs, semiring)
    reach = e.read("reach")
    kin = e.read("kin")
    g_reach = W.stream(993).normal(reach.cols.shape[1]).astype(np.float32)
    g_kin = W.stream(994).normal(kin.cols.shape[1]).astype(np.float32)
    gin = {"edge": np.zeros(len(e_[0]), np.float32), "fact": np.zeros(len(f[0]), np.float32)}
    e.backward("reach", g_reach, gin)
    e.backward("kin", g_kin, gin)
    e.close()
    samples = _spread_samples(B["sides"])
    assert B["sides"][samples].min() == 8 and B["sides"][samples].max() == 48
    exact = semiring == "diff_max_min"
    # the chosen samples in one oracle call: the oracle runs every sample as its
    # own fixpoint (pinned by test_batched_equals_per_sample), and its results
    # come sorted by sample, then tuple, as the engine reads them
    me, mf, ms, mc = (np.isin(x, samples) for x in (e_[3], f[4], st[2], c[4]))
    res = oracle_run(W.REACH_PROGRAM, {"edge": ((e_[0][me], e_[1][me]), e_[2][me], e_[3][me]),
                                       "start": ((st[0][ms],), None, st[2][ms])}, semiring)
    resk = oracle_run(W.KIN_PROGRAM, {"fact": ((f[0][mf], f[1][mf], f[2][mf]), f[3][mf], f[4][mf]),
                                      "comp": ((c[0][mc], c[1][mc], c[2][mc]), None, c[4][mc])}, semiring)
    for out, res_, rel, g_out, inp, m_in in (("reach", res, reach, g_reach, "edge", me), ("kin", resk, kin, g_kin, "fact", mf)):
        want = res_.relation(out)
        assert sorted(set(want.samples.tolist())) == samples, out
        m = np.isin(rel.samples, samples)
        assert np.array_equal(rel.samples[m], want.samples), out
        assert np.array_equal(rel.cols[:, m], want.cols), out
        if exact:
            assert np.array_equal(rel.tags[m], want.tags.astype(np.float32)), out
        else:
            np.testing.assert_allclose(rel.tags[m], want.tags, rtol=1e-5, atol=0, err_msg=out)
        gw = res_.vjp({out: g_out[m].astype(np.float64)})[inp]
        np.testing.assert_allclose(gin[inp][m_in], gw, rtol=1e-4, atol=1e-4, err_msg=out)
