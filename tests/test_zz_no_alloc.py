"""The allocation-free entry point lob_unique_rows_noalloc.

Some callers cannot allocate device memory when they need this step (serving
paths where cudaMalloc / cudaFree would synchronise the device, plug-ins inside
an application that owns all device memory, processes that split the GPU's
memory among tenants ahead of time).  This file checks that the entry point
gives the same rows as the engine's existing entry point (load-time
deduplication, read back after lob_run_to_fixpoint) and as an independent
numpy deduplication, on two calls in a row, plus its edge cases.  Kept in a
file that pytest collects last."""
import numpy as np
import pytest

from paper_2503_21937_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _rows(arity, n, bound, seed):
    s = W.stream(5000 + seed)
    return np.stack([s.below(n, bound) for _ in range(arity)]).astype(np.uint32)


def _numpy_unique(rows):
    """Distinct rows in lexicographic order, all-0xFFFFFFFF rows dropped."""
    keep = ~np.all(rows == 0xFFFFFFFF, axis=0)
    rows = rows[:, keep]
    if rows.shape[1] == 0:
        return rows
    return np.unique(rows, axis=1)


def _engine_unique(rows):
    from paper_2503_21937_gb300 import Engine
    e = Engine()
    e.declare("r", rows.shape[0])
    e.load("r", rows)
    e.run("unit")
    out = e.read("r").cols
    e.close()
    return out


def _noalloc(rows):
    import torch
    from paper_2503_21937_gb300 import lobster
    arity, n = rows.shape
    cols = torch.from_numpy(rows.view(np.int32).copy()).cuda()
    out = torch.full((arity, n), -1, dtype=torch.int32, device="cuda")
    n_out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    assert lobster.unique_rows_noalloc(cols, out, n_out) == 0
    torch.cuda.synchronize()
    m = int(n_out.item())
    return out[:, :m].cpu().numpy().view(np.uint32)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_21937_gb300 import build
    build.build()


@pytest.mark.parametrize("arity", [1, 2])
def test_noalloc_matches_engine_on_two_calls_in_a_row(arity):
    # two calls in a row on different inputs: the second must not see the first's leftovers
    for call, (n, bound) in enumerate([(150_000, 3000), (70_001, 900)]):
        rows = _rows(arity, n, bound, seed=10 * arity + call)
        got = _noalloc(rows)
        assert np.array_equal(got, _engine_unique(rows))
        assert np.array_equal(got, _numpy_unique(rows))


@pytest.mark.parametrize("arity", [1, 2])
def test_noalloc_edge_cases(arity):
    # one row; a row of all 0xFFFFFFFF (dropped) among others; only such rows;
    # values using all 32 bits; the largest accepted batch
    from paper_2503_21937_gb300 import lobster
    one = _rows(arity, 1, 1 << 32, seed=40 + arity)
    mixed = _rows(arity, 1000, 50, seed=50 + arity)
    mixed[:, 7] = 0xFFFFFFFF
    mixed[:, 500] = 0xFFFFFFFF
    if arity == 2:
        mixed[:, 9] = (0xFFFFFFFF, 3)  # only one column all-ones: kept
    sentinels = np.full((arity, 5), 0xFFFFFFFF, np.uint32)
    wide = _rows(arity, 20_000, 1 << 32, seed=60 + arity)
    wide[:, ::7] = wide[:, :1]
    biggest = _rows(arity, lobster.NOALLOC_MAX_ROWS, 1 << 16, seed=70 + arity)
    for rows in (one, mixed, sentinels, wide, biggest):
        assert np.array_equal(_noalloc(rows), _numpy_unique(rows))


def test_noalloc_empty_input():
    import torch
    from paper_2503_21937_gb300 import lobster
    for arity in (1, 2):
        cols = torch.zeros((arity, 0), dtype=torch.int32, device="cuda")
        out = torch.zeros((arity, 0), dtype=torch.int32, device="cuda")
        n_out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        assert lobster.unique_rows_noalloc(cols, out, n_out) == 0
        torch.cuda.synchronize()
        assert int(n_out.item()) == 0


def test_noalloc_rejects_too_many_rows():
    import torch
    from paper_2503_21937_gb300 import lobster
    n = lobster.NOALLOC_MAX_ROWS + 1
    cols = torch.zeros((1, n), dtype=torch.int32, device="cuda")
    out = torch.zeros((1, n), dtype=torch.int32, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert lobster.unique_rows_noalloc(cols, out, n_out) == -9  # LOB_E_CAPACITY
    assert lobster.unique_rows_noalloc(cols[:, :10], out, n_out) == 0
    torch.cuda.synchronize()
    assert int(n_out.item()) == 1
