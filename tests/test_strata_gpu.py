"""Programs of several strata (Sec. 3.1: a RAM program is a sequence of
strata; Algorithm 1 runs each to its fixpoint before the next), engine vs
oracle on seeded random graphs, in every semiring family, with gradients and
batched samples.  Under add-mult and top-1-proofs the engine runs the strata
one after another; under the lattice semirings one loop reaches the same
least fixpoint as the oracle's strata."""
import numpy as np
import pytest

from paper_2503_21937_gb300 import workloads as W
from tests.common import compare, engine_run, oracle_run

pytestmark = pytest.mark.gpu

ALL = ["unit", "max_min", "add_mult", "diff_max_min", "diff_add_mult", "top1_proofs", "diff_top1_proofs"]
SPLIT = ("add_mult", "diff_add_mult", "top1_proofs", "diff_top1_proofs")


def _graph(n, m, seed, scale=1.0):
    a, b = W.erdos_renyi(n, m, seed_index=seed)
    return a, b, (W.stream(seed + 1).prob(len(a)) * scale).astype(np.float32)


@pytest.mark.parametrize("sr", ALL)
def test_layered_three_strata(sr):
    a, b, p = _graph(60, 150, 7100)
    st, _ = compare(W.LAYERED_PROGRAM, {"edge": ((a, b), p)}, sr)
    assert st["strata"] == (3 if sr in SPLIT else 1)
    assert st["derived"] > 1000


@pytest.mark.parametrize("sr", ALL)
def test_mutually_recursive_stratum_below_a_projection(sr):
    a, b, p = _graph(80, 130, 7200)
    st, _ = compare(W.ODD_EVEN_PROGRAM, {"edge": ((a, b), p)}, sr)
    assert st["strata"] == (2 if sr in SPLIT else 1)


def test_rules_written_above_the_rules_they_read():
    a, b, p = _graph(50, 110, 7300)
    prog = "far(x,z) :- src(x), path(x,y), path(y,z), x != z.\nsrc(x) :- path(x,y).\n" + W.TC_PROGRAM
    st, _ = compare(prog, {"edge": ((a, b), p)}, "add_mult")
    assert st["strata"] == 3


@pytest.mark.parametrize("packed", [1, 0])
def test_gradients_through_three_strata(packed):
    """The backward replay of a stratum's first iteration takes every fact
    derived before it as that iteration's recent set."""
    a, b, p = _graph(40, 70, 7400, scale=0.3)  # sums stay below the clamp
    inputs = {"edge": ((a, b), p)}
    res = oracle_run(W.LAYERED_PROGRAM, inputs, "diff_add_mult")
    for out in ("far", "src", "path"):
        rel = res.relation(out)
        gout = W.stream(7401).normal(rel.cols.shape[1])
        want = res.vjp({out: gout})["edge"]
        e, st, got = engine_run(W.LAYERED_PROGRAM, inputs, "diff_add_mult", read=[out],
                                options={"packed_backward": packed})
        assert st["strata"] == 3
        assert np.array_equal(got[out].cols, rel.cols)
        gin = {"edge": np.zeros(len(a), np.float32)}
        e.backward(out, gout.astype(np.float32), gin)
        e.close()
        assert np.abs(want).max() > 0
        np.testing.assert_allclose(gin["edge"], want, rtol=1e-4, atol=1e-4, err_msg=out)


def test_batched_samples_keep_their_strata_apart():
    parts = [_graph(30, 60, 7500 + 10 * i) for i in range(3)]
    a = np.concatenate([q[0] for q in parts])
    b = np.concatenate([q[1] for q in parts])
    p = np.concatenate([q[2] for q in parts])
    s = np.concatenate([np.full(len(q[0]), i, np.uint32) for i, q in enumerate(parts)])
    compare(W.LAYERED_PROGRAM, {"edge": ((a, b), p, s)}, "add_mult")
    compare(W.ODD_EVEN_PROGRAM, {"edge": ((a, b), p, s)}, "diff_add_mult")
