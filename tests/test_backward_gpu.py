"""Gradients of the differentiable semirings: engine reverse mode (lob_backward)
vs the oracle's forward-mode gradient (itself pinned to FP64 central
differences in test_oracle_pins.py), within 1e-4."""
import numpy as np
import pytest

from paper_2503_21937_gb300 import workloads as W
from tests.common import engine_run, oracle_run

pytestmark = pytest.mark.gpu


def _grads(program, inputs, semiring, out, gout):
    e, st, got = engine_run(program, inputs, semiring, read=[out])
    gin = {k: np.zeros(len(v[0][0]) if not hasattr(v[0], "shape") else v[0].shape[-1], np.float32)
           for k, v in inputs.items() if len(v) > 1 and v[1] is not None}
    e.backward(out, gout.astype(np.float32), gin)
    e.close()
    return got[out], gin


def _check(program, inputs, semiring, out, seed, tol=1e-4):
    res = oracle_run(program, inputs, semiring)
    rel = res.relation(out)
    gout = W.stream(seed).normal(rel.cols.shape[1])
    want = res.vjp({out: gout})
    got_rel, got = _grads(program, inputs, semiring, out, gout)
    assert np.array_equal(got_rel.cols, rel.cols)
    for k, g in got.items():
        np.testing.assert_allclose(g, want[k], rtol=tol, atol=tol, err_msg=k)
    return want


@pytest.mark.parametrize("side", [4, 8, 24])
def test_grid_add_mult_gradient_unclamped(side):
    g = W.grid_reach_instance(side, sub=40 + side)
    src, dst, p = g["edge"]
    p = (p * 0.5).astype(np.float32)  # path sums stay below the clamp
    want = _check(W.REACH_PROGRAM, {"edge": ((src, dst), p), "start": (g["start"],)}, "diff_add_mult", "reach", 60)
    assert np.abs(want["edge"]).max() > 0


def test_grid_add_mult_gradient_with_clamping():
    g = W.grid_reach_instance(12, sub=77)
    src, dst, p = g["edge"]
    _check(W.REACH_PROGRAM, {"edge": ((src, dst), p), "start": (g["start"],)}, "diff_add_mult", "reach", 61)


@pytest.mark.parametrize("side", [6, 32])
def test_grid_max_min_gradient(side):
    g = W.grid_reach_instance(side, sub=50 + side)
    src, dst, p = g["edge"]
    _check(W.REACH_PROGRAM, {"edge": ((src, dst), p), "start": (g["start"],)}, "diff_max_min", "reach", 62, tol=1e-5)


@pytest.mark.parametrize("semiring", ["diff_add_mult", "diff_max_min"])
def test_kinship_gradient_nonlinear(semiring):
    s = W.stream(131)
    n, r, a, b, p = W.kinship_instance(s)
    p = (p * 0.6).astype(np.float32)
    c1, c2, c3 = W.composition_table()
    _check(W.KIN_PROGRAM, {"fact": ((r, a, b), p), "comp": ((c1, c2, c3),)}, semiring, "kin", 63)


def test_tc_gradient_duplicate_inputs():
    a = np.array([0, 0, 1, 2, 2, 3], np.uint32)
    b = np.array([1, 1, 2, 3, 3, 4], np.uint32)
    p = np.array([0.2, 0.3, 0.5, 0.1, 0.6, 0.9], np.float32)
    for sr in ("diff_add_mult", "diff_max_min"):
        _check(W.TC_PROGRAM, {"edge": ((a, b), p)}, sr, "path", 64)


def test_batched_gradient_matches_oracle():
    B = W.batched_instance(6)
    e = B["edge"]
    inputs = {"edge": ((e[0], e[1]), (e[2] * 0.5).astype(np.float32), e[3]),
              "start": ((B["start"][0],), None, B["start"][2])}
    _check(W.REACH_PROGRAM, inputs, "diff_add_mult", "reach", 65)
    f, c = B["fact"], B["comp"]
    inputs = {"fact": ((f[0], f[1], f[2]), (f[3] * 0.6).astype(np.float32), f[4]),
              "comp": ((c[0], c[1], c[2]), None, c[4])}
    _check(W.KIN_PROGRAM, inputs, "diff_add_mult", "kin", 66)


def test_autograd_function():
    import torch
    from paper_2503_21937_gb300.autograd import fixpoint
    g = W.grid_reach_instance(10, sub=90)
    src, dst, p = g["edge"]
    p = (p * 0.5).astype(np.float32)
    cols = torch.from_numpy(np.stack([src, dst]).astype(np.int32)).cuda()
    probs = torch.from_numpy(p).cuda().requires_grad_(True)
    start = torch.zeros((1, 1), dtype=torch.int32, device="cuda")
    out = fixpoint(W.REACH_PROGRAM, {"edge": (cols, probs), "start": (start, None)}, "diff_add_mult")
    tags = out["reach"][1]
    gout = torch.from_numpy(W.stream(91).normal(tags.numel()).astype(np.float32)).cuda()
    (tags * gout).sum().backward()
    res = oracle_run(W.REACH_PROGRAM, {"edge": ((src, dst), p), "start": (g["start"],)}, "diff_add_mult")
    want = res.vjp({"reach": gout.cpu().numpy().astype(np.float64)})["edge"]
    np.testing.assert_allclose(probs.grad.cpu().numpy(), want, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("packed", [1, 0])
def test_packed_and_general_backward_replays(packed):
    """The diff-add-mult backward on the packed kernels (binding words plus the
    rows of the facts matched so far) and on the general kernels, each against
    the oracle: a linear rule (grid reachability) and the three-atom kinship
    rule with a filter, batched."""
    def grads(program, inputs, out, seed):
        res = oracle_run(program, inputs, "diff_add_mult")
        rel = res.relation(out)
        gout = W.stream(seed).normal(rel.cols.shape[1])
        want = res.vjp({out: gout})
        e, st, got = engine_run(program, inputs, "diff_add_mult", read=[out], options={"packed_backward": packed})
        gin = {k: np.zeros(len(v[1]), np.float32) for k, v in inputs.items() if len(v) > 1 and v[1] is not None}
        e.backward(out, gout.astype(np.float32), gin)
        e.close()
        assert np.array_equal(got[out].cols, rel.cols)
        for k, g in gin.items():
            np.testing.assert_allclose(g, want[k], rtol=1e-4, atol=1e-4, err_msg=k)
    g = W.grid_reach_instance(14, sub=95)
    src, dst, p = g["edge"]
    grads(W.REACH_PROGRAM, {"edge": ((src, dst), (p * 0.5).astype(np.float32)), "start": (g["start"],)}, "reach", 96)
    B = W.batched_instance(5)
    f, c = B["fact"], B["comp"]
    inputs = {"fact": ((f[0], f[1], f[2]), (f[3] * 0.6).astype(np.float32), f[4]),
              "comp": ((c[0], c[1], c[2]), None, c[4])}
    grads(W.KIN_PROGRAM, inputs, "kin", 97)
