"""The allocation-free entry point lob_unique_rows_noalloc, checked against the
engine's own load-time deduplication (a relation without rules read back after
lob_run_to_fixpoint).  Kept in a file that pytest collects last."""
import numpy as np
import pytest

from paper_2503_21937_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _rows(arity, n, bound, seed):
    s = W.stream(5000 + seed)
    return np.stack([s.below(n, bound) for _ in range(arity)])


def _engine_unique(rows):
    from paper_2503_21937_gb300 import Engine
    e = Engine()
    e.declare("r", rows.shape[0])
    e.load("r", rows)
    e.run("unit")
    out = e.read("r").cols
    e.close()
    return out


@pytest.mark.parametrize("arity", [1, 2])
def test_noalloc_matches_engine_on_two_calls_in_a_row(arity):
    import torch
    from paper_2503_21937_gb300 import build, lobster
    build.build()
    # two calls in a row on different inputs: the second must not see the first's leftovers
    for call, (n, bound) in enumerate([(150_000, 3000), (70_001, 900)]):
        rows = _rows(arity, n, bound, seed=10 * arity + call)
        cols = torch.from_numpy(rows.astype(np.int32)).cuda()
        out = torch.full((arity, n), -1, dtype=torch.int32, device="cuda")
        n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
        assert lobster.unique_rows_noalloc(cols, out, n_out) == 0
        torch.cuda.synchronize()
        m = int(n_out.item())
        got = out[:, :m].cpu().numpy().astype(np.uint32)
        want = _engine_unique(rows)
        assert got.shape == want.shape
        assert np.array_equal(got, want)


def test_noalloc_rejects_too_many_rows():
    import torch
    from paper_2503_21937_gb300 import build, lobster
    build.build()
    n = lobster.NOALLOC_MAX_ROWS + 1
    cols = torch.zeros((1, n), dtype=torch.int32, device="cuda")
    out = torch.zeros((1, n), dtype=torch.int32, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert lobster.unique_rows_noalloc(cols, out, n_out) == -9  # LOB_E_CAPACITY
    assert lobster.unique_rows_noalloc(cols[:, :10], out, n_out, ) == 0
    torch.cuda.synchronize()
    assert int(n_out.item()) == 1
