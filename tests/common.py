"""Helpers shared by the engine tests: run the CUDA engine and the CPU oracle on
the same seeded inputs and compare."""
from __future__ import annotations

import hashlib

import numpy as np

import oracle

_ORACLE_CACHE: dict = {}


def _digest(program: str, inputs: dict, semiring: str) -> str:
    h = hashlib.sha256(program.encode() + semiring.encode())
    for k in sorted(inputs):
        h.update(k.encode())
        for part in inputs[k]:
            if part is None:
                h.update(b"none")
                continue
            for a in (part if isinstance(part, (tuple, list)) else (part,)):
                a = np.ascontiguousarray(a)
                h.update(str(a.dtype).encode() + str(a.shape).encode() + a.tobytes())
    return h.hexdigest()


def engine_run(program: str, inputs: dict, semiring: str = "unit", max_iters: int = 1 << 30, options=None,
               read=None, allocator=None):
    """Run the CUDA engine.  inputs: name -> (cols, tags, samples); allocator:
    optional (alloc, release) pair handed to lob_create.
    Returns (engine, stats, {relation: Relation})."""
    from paper_2503_21937_gb300 import Engine
    e = Engine(allocator=allocator)
    e.program(program)
    for k, v in (options or {}).items():
        e.set_option(k, v)
    for name, spec in inputs.items():
        cols, tags, samples = (list(spec) + [None, None])[:3]
        if name not in e.ids:
            e.declare(name, len(cols))
        e.load(name, cols, None if tags is None else np.asarray(tags, np.float32), samples)
    st = e.run(semiring, max_iters)
    names = read if read is not None else list(e.ids)
    return e, st, {n: e.read(n) for n in names}


def oracle_run(program: str, inputs: dict, semiring: str = "unit"):
    """The oracle's result, memoised per process on (program, inputs, semiring)
    so parametrised engine tests of one instance run the oracle once."""
    key = _digest(program, inputs, semiring)
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = _oracle_run(program, inputs, semiring)
    return _ORACLE_CACHE[key]


def _oracle_run(program: str, inputs: dict, semiring: str = "unit"):
    return oracle.run(program, {k: (v[0], None if (len(v) < 2 or v[1] is None) else np.asarray(v[1], np.float32)
                                    .astype(np.float64), v[2] if len(v) > 2 else None)
                                for k, v in inputs.items()}, semiring)


def _fact_names(ids, order, rows):
    """Input-fact ids -> sorted (relation, row) pairs, ids counting rows over
    the relations in `order` (relations without loaded rows count 0)."""
    bases, b = [], 0
    for k in order:
        bases.append((b, k))
        b += rows.get(k, 0)
    out = []
    for i in np.asarray(ids).tolist():
        base, k = max((bb, kk) for bb, kk in bases if bb <= i and i < bb + rows.get(kk, 0))
        out.append((k, i - base))
    return sorted(out)


def compare(program: str, inputs: dict, semiring: str = "unit", rels=None, rtol=1e-5, options=None, allocator=None):
    """Engine vs oracle: key sets bit-exact, tags per semiring tolerance.
    Returns (engine stats, oracle result)."""
    res = oracle_run(program, inputs, semiring)
    e, st, got = engine_run(program, inputs, semiring, options=options, read=rels, allocator=allocator)
    for name, rel in got.items():
        want = res.relation(name)
        assert rel.cols.shape == want.cols.shape, (name, rel.cols.shape, want.cols.shape)
        assert np.array_equal(rel.samples, want.samples), name
        assert np.array_equal(rel.cols, want.cols), name
        if semiring in ("max_min", "diff_max_min"):
            # min / max are exact: the f32 tag equals the oracle's value bitwise
            assert np.array_equal(rel.tags, want.tags.astype(np.float32)), name
        elif semiring in ("add_mult", "diff_add_mult"):
            np.testing.assert_allclose(rel.tags, want.tags, rtol=rtol, atol=0, err_msg=name)
        elif semiring in ("top1_proofs", "diff_top1_proofs"):
            # with no equally likely proofs met, the kept proof of every key is
            # unique: the same ids and the same f32 product on both sides
            assert res.ties == 0, "instance has ties: proofs are not unique"
            assert np.array_equal(rel.tags, want.tags.astype(np.float32)), name
            # both number input facts by row over the relations, but in
            # different relation orders: compare (relation, row) pairs
            rows = {k: len(np.asarray(v[0][0])) for k, v in inputs.items()}
            eng_order = sorted(e.ids, key=lambda k: e.ids[k])
            got_p = [_fact_names(p, eng_order, rows) for p in e.proofs(name)]
            want_p = [_fact_names(p, list(inputs), rows) for p in res.proofs(name)]
            assert len(got_p) == len(want_p), name
            for i, (a, b) in enumerate(zip(got_p, want_p)):
                assert a == b, (name, i, a, b)
        else:
            assert np.all(rel.tags == 1.0)
    e.close()
    return st, res
