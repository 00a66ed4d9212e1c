"""top-1-proofs and diff-top-1-proofs on the GPU (Sec. 5.3 "Limitations";
Sec. 3.4): every fact keeps one proof, the union of its derivation's proofs,
and the likelier proof wins.  Parity with the oracle is on the probabilities
(bitwise f32) and on the proofs themselves (the same input-fact ids), on
instances where the oracle met no two equally likely proofs."""
import numpy as np
import pytest

from paper_2503_21937_gb300 import workloads as W
from tests.common import compare, engine_run, oracle_run

pytestmark = pytest.mark.gpu
SEMIRINGS = ["top1_proofs", "diff_top1_proofs"]


def _reach_inputs(n, m, seed):
    s = W.stream(seed)
    src, dst = s.below(m, n), s.below(m, n)
    p = s.prob(m)
    return {"edge": ((src, dst), p), "start": ((np.array([0], np.uint32),),)}


@pytest.mark.parametrize("sr", SEMIRINGS)
@pytest.mark.parametrize("n,m,seed", [(6, 12, 1), (200, 900, 2), (3000, 12000, 3)])
def test_reach_random_graphs(sr, n, m, seed):
    compare(W.REACH_PROGRAM, _reach_inputs(n, m, seed), sr)


@pytest.mark.parametrize("sr", SEMIRINGS)
def test_tc_nonlinear_and_linear(sr):
    s = W.stream(31)
    n, m = 60, 150
    src, dst, p = s.below(m, n), s.below(m, n), s.prob(m)
    compare(W.TC_PROGRAM, {"edge": ((src, dst), p)}, sr)
    nonlinear = "path(x,y) :- edge(x,y).\npath(x,z) :- path(x,y), path(y,z).\n"
    compare(nonlinear, {"edge": ((src, dst), p)}, sr)


def test_same_generation_three_atom_rule():
    parent, child, _ = W.random_tree(300, seed_index=5)
    p = W.stream(32).prob(len(parent))
    compare(W.SG_PROGRAM, {"parent": ((parent, child), p)}, "top1_proofs")


def test_batched_kinship():
    """Three kinship samples (sample ids in the keys) with the untagged
    composition table replicated per sample: comp facts join proofs as the
    empty conjunction."""
    c1, c2, c3 = W.composition_table()
    cols, sids = [[], [], [], []], []
    for i in range(3):
        _, r, a, b, p = W.kinship_instance(W.stream(500 + i), lo=10, hi=14)
        for q, x in enumerate((r, a, b, p)):
            cols[q].append(x)
        sids.append(np.full(len(r), i, np.uint32))
    cat = np.concatenate
    k = len(c1)
    inputs = {"fact": ((cat(cols[0]), cat(cols[1]), cat(cols[2])), cat(cols[3]), cat(sids)),
              "comp": ((np.tile(c1, 3), np.tile(c2, 3), np.tile(c3, 3)), None, np.repeat(np.arange(3, dtype=np.uint32), k))}
    compare(W.KIN_PROGRAM, inputs, "diff_top1_proofs", rels=["kin"])


def test_grid_grows_the_proof_arena():
    """A 48 x 48 grid (paths of up to ~100 edges, improved many times) with an
    arena of 1,024 free words: it has to grow many times, each growth running
    the overflowing step again, and the results stay exact."""
    g = W.grid_reach_instance(48)
    src, dst, p = g["edge"]
    inputs = {"edge": ((src, dst), p), "start": (g["start"],)}
    st, _ = compare(W.REACH_PROGRAM, inputs, "top1_proofs", options={"proof_arena_words": 1024})
    assert st["proof_words"] > 2 * len(src) + 1 + (1 << 20)


def test_paper_example_proof():
    from tests.golden.load import pathfinder_example
    program, inputs = pathfinder_example()
    from tests.common import _fact_names
    e, st, got = engine_run(program, inputs, "top1_proofs")
    rows = {k: len(v[0][0]) for k, v in inputs.items()}
    order = sorted(e.ids, key=lambda k: e.ids[k])
    # edge(1,2) .. edge(4,5): rows 1..4 of the fixture's edge facts
    assert [_fact_names(p, order, rows) for p in e.proofs("connected")] == [[("edge", q) for q in range(1, 5)]]
    assert got["connected"].tags.tolist() == [np.float32(0.9 * 0.8 * 0.95 * 0.85)]
    e.close()
    compare(program, inputs, "top1_proofs")


def test_proof_cap_is_an_error():
    from paper_2503_21937_gb300 import LobsterError
    n = 9
    a, b = W.ktree_chain(n)
    inputs = {"edge": ((a, b), np.full(n - 1, 0.5, np.float32)), "start": ((np.array([0], np.uint32),),)}
    with pytest.raises(LobsterError) as ei:
        engine_run(W.REACH_PROGRAM, inputs, "top1_proofs", options={"proof_cap": 5})
    assert ei.value.code == -9  # LOB_E_CAPACITY
    e, st, got = engine_run(W.REACH_PROGRAM, inputs, "top1_proofs", options={"proof_cap": 8})
    assert [len(x) for x in e.proofs("reach")] == list(range(n))
    e.close()


def test_gradient_matches_oracle():
    inputs = _reach_inputs(150, 600, 7)
    res = oracle_run(W.REACH_PROGRAM, inputs, "diff_top1_proofs")
    assert res.ties == 0
    e, st, got = engine_run(W.REACH_PROGRAM, inputs, "diff_top1_proofs")
    n_out = got["reach"].cols.shape[1]
    g = W.stream(8).normal(n_out).astype(np.float32)
    gin = np.zeros(len(inputs["edge"][1]), np.float32)
    e.backward("reach", g, {"edge": gin})
    want = res.vjp({"reach": g.astype(np.float64)})["edge"]
    np.testing.assert_allclose(gin, want, rtol=1e-4, atol=1e-5)
    e.close()


def test_pathfinder_training_step_with_top1():
    """The training pipeline of Sec. 2 with the paper's semiring for it."""
    from paper_2503_21937_gb300 import pathfinder as PF
    out = PF.train(side=6, batch=16, steps=3, semiring="diff_top1_proofs", seed=2)
    assert len(out["history"]) == 3 and all(np.isfinite(h[0]) for h in out["history"])
