"""torch.autograd binding of the fixpoint engine (Sec. 3.4 differentiable
semirings; the PyTorch side of the neurosymbolic pipeline).

``fixpoint(program, inputs, semiring, outputs)`` runs the engine on CUDA
tensors and returns, per output relation, its columns and its tags; the tags
are differentiable with respect to the probability tensors of the inputs.  The
backward pass is the engine's own (``lob_backward``): the binding only moves
tensors.
"""
from __future__ import annotations

import torch

from .lobster import Engine, relation_arities

_DIFF = {"diff_max_min", "diff_add_mult", "diff_top1_proofs"}

# Idle engines per (program, relations, stream, device, input-size class).  An
# engine is taken for one forward (+ backward) and returned afterwards, so a
# training loop reuses its device buffers and the sizes it recorded (the
# device-driven iteration loop plans from them), and calls of very different
# sizes do not share capacity plans.
_IDLE: dict = {}
_MAX_IDLE = 4


def _engine_key(program, names, cols, options):
    rows = sum(int(c.shape[1]) for c in cols)
    stream = torch.cuda.current_stream().cuda_stream
    return (program, tuple(names), tuple(int(c.shape[0]) for c in cols), stream, torch.cuda.current_device(),
            max(rows, 1).bit_length(), tuple(sorted(options.items())))


def _take_engine(key, program, options):
    idle = _IDLE.get(key)
    if idle:
        e = idle.pop()
        e.reset()
        return e
    e = Engine()
    e.program(program)
    for k, v in options.items():
        e.set_option(k, v)
    return e


def _give_back(key, e):
    idle = _IDLE.setdefault(key, [])
    if len(idle) < _MAX_IDLE:
        idle.append(e)
    else:
        e.close()


class _FixpointFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, spec, *probs):
        program, names, cols, samples, semiring, outputs, options = spec
        key = _engine_key(program, names, cols, options)
        e = _take_engine(key, program, options)
        ctx.stats = None
        for name, c, p, s in zip(names, cols, probs, samples):
            if name not in e.ids:
                e.declare(name, c.shape[0])
            e.load(name, c, p.detach() if p is not None else None, s)
        ctx.stats = e.run(semiring)
        LAST_STATS.clear()
        LAST_STATS.update(ctx.stats)
        rels = [e.read(o, device=True) for o in outputs]
        ctx.engine = e
        ctx.key = key
        ctx.spec = spec
        ctx.sizes = [c.shape[1] for c in cols]
        ctx.has_prob = [p is not None for p in probs]
        tags = [r.tags.clone() for r in rels]
        out_cols = [r.cols.clone() for r in rels]
        out_smp = [r.samples.clone() for r in rels]
        ctx.mark_non_differentiable(*out_cols, *out_smp)
        if semiring not in _DIFF:  # no backward will need this engine's state
            ctx.engine = None
            _give_back(key, e)
        return (*tags, *out_cols, *out_smp)

    @staticmethod
    def backward(ctx, *grads):
        program, names, cols, samples, semiring, outputs, options = ctx.spec
        e = ctx.engine
        if semiring not in _DIFF or e is None:
            raise RuntimeError("gradients need a diff_* semiring")
        gin = {n: torch.zeros(sz, dtype=torch.float32, device="cuda")
               for n, sz, hp in zip(names, ctx.sizes, ctx.has_prob) if hp}
        for o, g in zip(outputs, grads[:len(outputs)]):
            if g is not None:
                e.backward(o, g.contiguous().to(torch.float32), gin)
        torch.cuda.synchronize()
        ctx.engine = None
        _give_back(ctx.key, e)
        return (None, *[gin.get(n) if hp else None for n, hp in zip(names, ctx.has_prob)])


# statistics (lob_stats) of the most recent forward run, for benchmarks
LAST_STATS: dict = {}


def fixpoint(program: str, inputs: dict, semiring: str = "diff_add_mult", outputs=None, options=None):
    """inputs: name -> (cols (arity, n) int tensor, probs (n,) float tensor or None,
    sample ids (n,) int tensor or None), all on CUDA.  Returns name -> (cols,
    tags, sample ids) for each output relation (default: every rule head).
    options: engine options (lob_set_option keys) for the engines that run it."""
    if outputs is None:
        heads = []
        for line in program.split("."):
            if ":-" in line:
                h = line.split(":-")[0].strip()
                h = h[: h.index("(")].strip()
                if h not in heads:
                    heads.append(h)
        outputs = heads
    names = list(inputs)
    cols = [inputs[n][0] for n in names]
    probs = [inputs[n][1] if len(inputs[n]) > 1 else None for n in names]
    samples = [inputs[n][2] if len(inputs[n]) > 2 else None for n in names]
    spec = (program, names, cols, samples, semiring, list(outputs), dict(options or {}))
    res = _FixpointFn.apply(spec, *probs)
    m = len(outputs)
    return {o: (res[m + i], res[i], res[2 * m + i]) for i, o in enumerate(outputs)}


__all__ = ["fixpoint", "relation_arities"]
