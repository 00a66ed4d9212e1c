"""Computed head arguments and comparison filters (Sec. 5.2: projections and
selections that compute run as bytecode on a per-thread stack machine),
engine vs oracle on the same seeded inputs, in every semiring family."""
import numpy as np
import pytest

from paper_2503_21937_gb300 import workloads as W
from tests.common import compare, engine_run

pytestmark = pytest.mark.gpu

WALK = ("walk(x, 0) :- start(x).\n"
        "walk(y, d + 1) :- walk(x, d), edge(x, y), d < 12.\n")


def _graph(n, m, seed):
    s = W.stream(seed)
    return s.below(m, n), s.below(m, n), s.prob(m)


@pytest.mark.parametrize("sr", ["unit", "max_min", "add_mult", "diff_max_min", "diff_add_mult", "top1_proofs"])
def test_bounded_walk_lengths(sr):
    src, dst, p = _graph(300, 1200, 61)
    inputs = {"edge": ((src, dst), p), "start": ((np.array([0], np.uint32),),)}
    compare(WALK, inputs, sr)


def test_arithmetic_and_comparisons_over_several_tiles():
    """Wrap-around, division (a zero divisor drops the row), the reserved value
    2^32 - 1, order comparisons and nested expressions on 20,000 rows."""
    s = W.stream(62)
    n = 20000
    x = s.below(n, 1 << 31).astype(np.uint32) * np.uint32(2) + (s.below(n, 2)).astype(np.uint32)
    y = s.below(n, 1000).astype(np.uint32)
    y[:50] = 0
    x[:7] = 0
    x[100:1100] = s.below(1000, 1500)  # rows where x <= y holds
    prog = ("diff(x, y - x) :- p(x, y), x <= y.\n"
            "quot(x, x / y) :- p(x, y).\n"
            "prod(x, x * y + 1) :- p(x, y).\n"
            "pred(x - 1) :- p(x, y).\n"
            "big(x) :- p(x, y), x + y > y * 2, (x - y) / 2 >= 1.\n"
            "pair(x, z) :- p(x, y), p(z, w), y == w + 1, x < z.\n")
    inputs = {"p": ((x[:2000], y[:2000]),)}
    compare(prog, inputs, "unit")
    compare("quot(x, x / y) :- p(x, y).\nprod(x, x * y + 1) :- p(x, y).\n", {"p": ((x, y),)}, "unit")


def test_join_on_a_computed_column():
    """A computed column is joined on by a later rule (its 32-bit field probes
    the narrower fields of the loaded relation)."""
    src, dst, p = _graph(500, 2000, 63)
    prog = ("shift(x + 1, y) :- edge(x, y).\n"
            "hit(x, y) :- shift(x, y), edge(x, y).\n")
    compare(prog, {"edge": ((src, dst), p)}, "max_min")


def test_batched_samples_with_arithmetic():
    src, dst, p = _graph(80, 300, 64)
    n = len(src)
    sid = (np.arange(n) % 3).astype(np.uint32)
    start = ((np.zeros(3, np.uint32),), None, np.arange(3, dtype=np.uint32))
    compare(WALK, {"edge": ((src, dst), p, sid), "start": start}, "diff_max_min")


def test_gradient_through_computed_rules():
    import oracle as O
    from tests.common import oracle_run
    src, dst, p = _graph(60, 200, 65)
    inputs = {"edge": ((src, dst), p), "start": ((np.array([0], np.uint32),),)}
    for sr in ("diff_add_mult", "diff_max_min"):
        res = oracle_run(WALK, inputs, sr)
        e, st, got = engine_run(WALK, inputs, sr)
        g = W.stream(66).normal(got["walk"].cols.shape[1]).astype(np.float32)
        gin = np.zeros(len(p), np.float32)
        e.backward("walk", g, {"edge": gin})
        want = res.vjp({"walk": g.astype(np.float64)})["edge"]
        np.testing.assert_allclose(gin, want, rtol=1e-4, atol=1e-5)
        e.close()


def test_parse_errors_and_unsafe_expressions():
    from paper_2503_21937_gb300 import Engine, LobsterError
    e = Engine()
    e.declare("p", 2)
    e.declare("q", 1)
    for bad, code in [("q(x + z) :- p(x, y).", -4),      # z unbound
                      ("q(x) :- p(x, y), x < z.", -4),    # z unbound in a filter
                      ("q(x) :- p(x, y), x + y.", -2),    # no comparison
                      ("q(x) :- p(x, y), x < .", -2)]:
        with pytest.raises(LobsterError) as ei:
            e.add_rule(bad)
        assert ei.value.code == code, bad
    deep = "q(" + "x + (" * 9 + "y" + ")" * 9 + ") :- p(x, y)."  # needs a stack of 10
    with pytest.raises(LobsterError):
        e.add_rule(deep)
    e.close()
