"""Engine vs oracle parity on the GPU (through the C ABI)."""
import numpy as np
import pytest

from paper_2503_21937_gb300 import workloads as W
from tests import pins
from tests.common import compare, engine_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_21937_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


# ---------------------------------------------------------------------------
# unit semiring
# ---------------------------------------------------------------------------

def _closure_against_bfs(a, b, n_nodes, options=None):
    """Unit TC where the naive oracle would take a minute or more: the engine's
    path relation, element by element, against the per-source BFS closure (the
    textbook computation the oracle is pinned to)."""
    e, st, got = engine_run(W.TC_PROGRAM, {"edge": ((a, b),)}, read=["path"], options=options)
    e.close()
    x, y = got["path"].cols.astype(np.uint64)
    keys = (x << np.uint64(32)) | y
    assert np.all(keys[1:] > keys[:-1])  # sorted distinct facts, read order
    assert np.array_equal(keys, pins.closure_keys_scipy(a, b, n_nodes))
    return st


@pytest.mark.parametrize("n", [2, 3, 65])
def test_tc_chain(n):
    a, b = W.ktree_chain(n)
    st, _ = compare(W.TC_PROGRAM, {"edge": ((a, b),)})
    assert st["derived"] == n * (n - 1) // 2


def test_tc_long_chain():
    """700 iterations, one new fact per source and iteration."""
    st = _closure_against_bfs(*W.ktree_chain(700), 700)
    assert st["derived"] == 700 * 699 // 2


@pytest.mark.parametrize("n,m,seed", [(40, 80, 1), (300, 900, 2)])
def test_tc_random(n, m, seed):
    a, b = W.erdos_renyi(n, m, seed_index=100 + seed)
    compare(W.TC_PROGRAM, {"edge": ((a, b),)})


def test_tc_random_2000_nodes():
    a, b = W.erdos_renyi(2000, 5000, seed_index=103)
    _closure_against_bfs(a, b, 2000)


def test_tc_config1_full_size():
    a, b = W.erdos_renyi(1000, 3000)
    st, res = compare(W.TC_PROGRAM, {"edge": ((a, b),)})
    assert st["derived"] == res.relation("path").cols.shape[1]


def test_sg_random_tree():
    parent, child, depth = W.random_tree(3000, seed_index=22)
    st, _ = compare(W.SG_PROGRAM, {"parent": ((parent, child),)})


def test_tc_power_law_small():
    s, d = W.chung_lu_power_law(1500, 6000, seed_index=23)
    _closure_against_bfs(s, d, 1500)


def test_andersen_small():
    A = W.andersen_program(4000, 12000, seed_index=33)
    compare(W.ANDERSEN_PROGRAM, {k: ((v[0], v[1]),) for k, v in A.items()}, rels=["pt"])


def test_filters_constants_repeats():
    edge = (np.array([0, 1, 1, 2, 3, 5, 5], np.uint32), np.array([1, 1, 2, 2, 0, 5, 6], np.uint32))
    prog = ("loop(x) :- edge(x,x).\n"
            "fromzero(y) :- edge(0,y).\n"
            "twohop(x,z) :- edge(x,y), edge(y,z), x != z.\n"
            "same(x) :- edge(x,y), x == 1.\n"
            "tagged(x,7) :- edge(x,y), edge(y,x).\n")
    compare(prog, {"edge": (edge,)})


def test_duplicate_inputs_and_empty_relation():
    a = np.array([0, 0, 1, 1, 2], np.uint32)
    b = np.array([1, 1, 2, 2, 3], np.uint32)
    prog = W.TC_PROGRAM + "other(x) :- nothing(x).\n"
    compare(prog, {"edge": ((a, b),), "nothing": ((np.zeros(0, np.uint32),),)})


# ---------------------------------------------------------------------------
# probabilistic semirings
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("semiring", ["max_min", "add_mult", "diff_max_min", "diff_add_mult"])
@pytest.mark.parametrize("side", [5, 24])
def test_grid_reach(semiring, side):
    g = W.grid_reach_instance(side, sub=side)
    src, dst, p = g["edge"]
    compare(W.REACH_PROGRAM, {"edge": ((src, dst), p), "start": (g["start"],)}, semiring)


@pytest.mark.parametrize("semiring", ["max_min", "add_mult"])
def test_tc_probabilistic_random(semiring):
    a, b = W.erdos_renyi(60, 150, seed_index=120)
    p = W.stream(121).prob(len(a))
    compare(W.TC_PROGRAM, {"edge": ((a, b), p)}, semiring)


@pytest.mark.parametrize("semiring", ["unit", "max_min", "add_mult"])
def test_kinship_nonlinear(semiring):
    s = W.stream(130)
    n, r, a, b, p = W.kinship_instance(s)
    c1, c2, c3 = W.composition_table()
    compare(W.KIN_PROGRAM, {"fact": ((r, a, b), p), "comp": ((c1, c2, c3),)}, semiring, rels=["kin"])


def test_batched_reach_matches_oracle():
    B = W.batched_instance(12)
    e = B["edge"]
    inputs = {"edge": ((e[0], e[1]), e[2], e[3]), "start": ((B["start"][0],), None, B["start"][2])}
    for sr in ("unit", "max_min", "add_mult"):
        compare(W.REACH_PROGRAM, inputs, sr, rels=["reach"])


def test_batched_kinship_matches_oracle():
    B = W.batched_instance(10)
    f = B["fact"]
    c = B["comp"]
    inputs = {"fact": ((f[0], f[1], f[2]), f[3], f[4]), "comp": ((c[0], c[1], c[2]), None, c[4])}
    compare(W.KIN_PROGRAM, inputs, "add_mult", rels=["kin"])


# ---------------------------------------------------------------------------
# candidate sets larger than one sort: chunked sort + unique + (+)-accumulation
# ---------------------------------------------------------------------------

# sorted candidates in chunks: the dense (+)-accumulation (which needs no
# candidate sort) is switched off so the tagged runs take the chunked path
CHUNK = {"max_candidates": 4096, "acc_dense": 0}


def test_chunked_tc_unit():
    a, b = W.erdos_renyi(300, 1500, seed_index=140)
    st, _ = compare(W.TC_PROGRAM, {"edge": ((a, b),)}, options=CHUNK)
    assert st["candidates"] > 10 * 4096


@pytest.mark.parametrize("semiring", ["max_min", "add_mult", "diff_max_min"])
def test_chunked_grid(semiring):
    g = W.grid_reach_instance(40, sub=141)
    src, dst, p = g["edge"]
    compare(W.REACH_PROGRAM, {"edge": ((src, dst), p), "start": (g["start"],)}, semiring, options=CHUNK)


def test_chunked_batched_kinship_add_mult():
    B = W.batched_instance(4)
    f, c = B["fact"], B["comp"]
    inputs = {"fact": ((f[0], f[1], f[2]), f[3], f[4]), "comp": ((c[0], c[1], c[2]), None, c[4])}
    st, _ = compare(W.KIN_PROGRAM, inputs, "add_mult", rels=["kin"], options=CHUNK)
    assert st["candidates"] > 10 * 4096


# ---------------------------------------------------------------------------
# membership filter at emission (unit semiring), forced on from iteration 1
# ---------------------------------------------------------------------------

FILTER = {"emit_filter": 2}


# ---------------------------------------------------------------------------
# dense (+)-accumulation of tagged candidates vs sorted candidates
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("semiring", ["max_min", "add_mult", "diff_max_min", "diff_add_mult"])
@pytest.mark.parametrize("opts", [{"acc_dense": 1}, {"acc_dense": 1, "packed_join": 0}, {"acc_dense": 0},
                                  {"acc_dense": 1, "acc_bits": 12}])
def test_dense_accumulation(semiring, opts):
    """Dense accumulation from the packed emission (atomics) and from folded
    candidates of the general join steps, the sorted path, and a key-width
    limit that leaves kin (26 bits) sorted while reach (12 bits) is dense;
    every variant against the oracle, on a linear and a non-linear program
    with a filter, samples and duplicate derivations."""
    g = W.grid_reach_instance(16, sub=77)
    src, dst, p = g["edge"]
    compare(W.REACH_PROGRAM, {"edge": ((src, dst), p), "start": (g["start"],)}, semiring, options=opts)
    B = W.batched_instance(6)
    f, c = B["fact"], B["comp"]
    inputs = {"fact": ((f[0], f[1], f[2]), f[3], f[4]), "comp": ((c[0], c[1], c[2]), None, c[4])}
    compare(W.KIN_PROGRAM, inputs, semiring, rels=["kin"], options=opts)


def test_filter_tc_and_sg():
    a, b = W.erdos_renyi(300, 1500, seed_index=150)
    compare(W.TC_PROGRAM, {"edge": ((a, b),)}, options=FILTER)
    parent, child, _ = W.random_tree(2000, seed_index=151)
    compare(W.SG_PROGRAM, {"parent": ((parent, child),)}, options=FILTER)


def test_filter_andersen_with_secondary_views():
    A = W.andersen_program(4000, 12000, seed_index=152)
    compare(W.ANDERSEN_PROGRAM, {k: ((v[0], v[1]),) for k, v in A.items()}, rels=["pt"], options=FILTER)


def test_filter_with_chunking():
    a, b = W.erdos_renyi(300, 1500, seed_index=153)
    compare(W.TC_PROGRAM, {"edge": ((a, b),)}, options={"emit_filter": 2, "max_candidates": 4096})


# ---------------------------------------------------------------------------
# errors
# ---------------------------------------------------------------------------

def test_max_iters_error_keeps_state():
    from paper_2503_21937_gb300 import LobsterError
    a, b = W.ktree_chain(50)
    with pytest.raises(LobsterError) as ei:
        engine_run(W.TC_PROGRAM, {"edge": ((a, b),)}, max_iters=3)
    assert "MAXITER" in str(ei.value)


def test_parse_and_unknown_relation_errors():
    from paper_2503_21937_gb300 import Engine, LobsterError
    e = Engine()
    e.declare("edge", 2)
    e.declare("path", 2)
    with pytest.raises(LobsterError, match="PARSE"):
        e.add_rule("path(x,y) :- edge(x,y)")
    with pytest.raises(LobsterError, match="UNKNOWN_REL"):
        e.add_rule("path(x,y) :- edgez(x,y).")
    with pytest.raises(LobsterError, match="UNSAFE"):
        e.add_rule("path(x,w) :- edge(x,y).")
    with pytest.raises(LobsterError, match="E_ARG"):
        e.add_rule("path(x,y) :- edge(x,y,z).")
    e.close()


# ---------------------------------------------------------------------------
# join steps: packed-word kernels (block-local offsets) vs the general kernels,
# on skewed fan-out, ragged row counts, sub-range emission and the filter
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("packed_join", [0, 1])
def test_emission_paths(packed_join):
    opts = {"packed_join": packed_join}
    parent, child, _ = W.random_tree(2500, seed_index=160)
    compare(W.SG_PROGRAM, {"parent": ((parent, child),)}, options=opts)
    compare(W.SG_PROGRAM, {"parent": ((parent, child),)}, options=dict(opts, emit_filter=2))
    a, b = W.ktree_chain(300)
    compare(W.TC_PROGRAM, {"edge": ((a, b),)}, options=dict(opts, max_candidates=4096))
    s, d = W.chung_lu_power_law(3000, 15000, seed_index=162)  # skewed fan-out: rows with thousands of matches
    _closure_against_bfs(s, d, 3000, options=opts)
    _closure_against_bfs(s, d, 3000, options=dict(opts, emit_filter=2, max_candidates=50000))
    A = W.andersen_program(3000, 9000, seed_index=163)
    compare(W.ANDERSEN_PROGRAM, {k: ((v[0], v[1]),) for k, v in A.items()}, rels=["pt"], options=opts)
    g = W.grid_reach_instance(20, sub=161)
    src, dst, p = g["edge"]
    for sr in ("max_min", "diff_add_mult"):
        compare(W.REACH_PROGRAM, {"edge": ((src, dst), p), "start": (g["start"],)}, sr, options=opts)


# ---------------------------------------------------------------------------
# bitmap delta mode: new facts read out of the membership bitmaps
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [0, 1, 2])
def test_bitmap_delta(mode):
    opts = {"bitmap_delta": mode, "emit_filter": 2}
    parent, child, _ = W.random_tree(2500, seed_index=170)
    compare(W.SG_PROGRAM, {"parent": ((parent, child),)}, options=opts)
    a, b = W.erdos_renyi(300, 1500, seed_index=171)
    compare(W.TC_PROGRAM, {"edge": ((a, b),)}, options=opts)
    # chunked candidate sets from the general kernels and projections
    compare(W.TC_PROGRAM, {"edge": ((a, b),)}, options=dict(opts, max_candidates=4096, packed_join=0))
    # the full relation is probed after iteration 1 (non-linear rule): merged every iteration
    nonlinear = "path(x,y) :- edge(x,y).\npath(x,z) :- path(x,y), path(y,z).\n"
    compare(nonlinear, {"edge": ((a, b),)}, options=opts)
    A = W.andersen_program(3000, 9000, seed_index=172)
    compare(W.ANDERSEN_PROGRAM, {k: ((v[0], v[1]),) for k, v in A.items()}, rels=["pt"], options=opts)
    # 34-bit keys (u64 words, 2 GB bitmaps)
    s, d = W.erdos_renyi(70000, 140000, seed_index=173)
    compare(W.TC_PROGRAM, {"edge": ((s[:3000], d[:3000]),)}, options=opts)
    # batched: the sample id is the key's top field, so one bitmap spans all samples
    B = W.batched_instance(6)
    e = B["edge"]
    compare(W.REACH_PROGRAM, {"edge": ((e[0], e[1]), None, e[3]), "start": ((B["start"][0],), None, B["start"][2])},
            rels=["reach"], options=opts)


# ---------------------------------------------------------------------------
# warp-balanced join steps (unit semiring) with and without the bitmap delta
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("warp_join", [0, 1])
@pytest.mark.parametrize("bitmap_delta", [0, 2])
def test_warp_join(warp_join, bitmap_delta):
    opts = {"warp_join": warp_join, "bitmap_delta": bitmap_delta}
    parent, child, _ = W.random_tree(3000, seed_index=180)
    compare(W.SG_PROGRAM, {"parent": ((parent, child),)}, options=opts)
    s, d = W.chung_lu_power_law(3000, 15000, seed_index=181)  # hub rows with thousands of matches
    _closure_against_bfs(s, d, 3000, options=opts)
    A = W.andersen_program(3000, 9000, seed_index=182)
    compare(W.ANDERSEN_PROGRAM, {k: ((v[0], v[1]),) for k, v in A.items()}, rels=["pt"], options=opts)
    n, r, a, b, p = W.kinship_instance(W.stream(183))
    c1, c2, c3 = W.composition_table()
    compare(W.KIN_PROGRAM, {"fact": ((r, a, b),), "comp": ((c1, c2, c3),)}, rels=["kin"], options=opts)


# ---------------------------------------------------------------------------
# autotuner: timed trials, then a normal run with the chosen options
# ---------------------------------------------------------------------------

def test_autotune_then_run_matches_oracle():
    from paper_2503_21937_gb300 import Engine, LobsterError
    from tests.common import oracle_run
    s, d = W.chung_lu_power_law(1500, 6000, seed_index=190)
    e = Engine()
    e.program(W.TC_PROGRAM)
    e.load("edge", (s, d))
    rep = e.autotune("unit", repeats=1)
    # the first setting + every alternative of 7 knobs (join_index: offset table, 30-bit table, search, hash;
    # the hash table's size only when the hash index was kept)
    assert rep["trials"] >= 1 + 1 + 3 + 1 + 2 + 2 + 2 + 1 + (1 if rep["join_index"] == 3 else 0)
    assert rep["join_index"] in (0, 1, 2, 3) and rep["cross_join"] in (0, 1)
    assert 0 < rep["best_ms"] <= rep["first_ms"]
    assert rep["warp_join"] in (0, 1, 2) and rep["bitmap_delta"] in (0, 1, 2) and rep["radix_bits"] in (6, 8)
    e.run("unit")
    want = oracle_run(W.TC_PROGRAM, {"edge": ((s, d),)}).relation("path")
    assert np.array_equal(e.read("path").cols, want.cols)
    with pytest.raises(LobsterError, match="STATE"):
        e.autotune("unit")
    e.close()
    g = W.grid_reach_instance(16, sub=191)
    src, dst, p = g["edge"]
    inputs = {"edge": ((src, dst), p), "start": (g["start"],)}
    e = Engine()
    e.program(W.REACH_PROGRAM)
    e.load("edge", (src, dst), np.asarray(p, np.float32))
    e.load("start", g["start"])
    rep = e.autotune("max_min", repeats=1)
    # semirings with tags tune packed_join, join_index, radix_bits and acc_dense,
    # and the hash table's size when the hash index was kept
    assert rep["trials"] == 1 + 1 + 3 + 1 + 1 + (1 if rep["join_index"] == 3 else 0)
    assert rep["hash_slots"] in (2, 4)
    e.run("max_min")
    want = oracle_run(W.REACH_PROGRAM, inputs, "max_min").relation("reach")
    got = e.read("reach")
    assert np.array_equal(got.cols, want.cols) and np.array_equal(got.tags, want.tags.astype(np.float32))
    e.close()


# ---------------------------------------------------------------------------
# the paper's Pathfinder example (tests/golden/pathfinder_example.txt)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("semiring", ["unit", "max_min", "add_mult", "diff_max_min", "diff_add_mult"])
def test_pathfinder_example(semiring):
    from tests.golden.load import pathfinder_example
    program, inputs = pathfinder_example()
    compare(program, inputs, semiring)


# ---------------------------------------------------------------------------
# failure handling on the host side (no GPU fault): allocator refusal,
# too-small read buffers; and run-to-run determinism despite atomics
# ---------------------------------------------------------------------------

def test_allocator_refusal_reports_oom_and_engine_stays_usable():
    import torch
    from paper_2503_21937_gb300 import Engine, LobsterError
    from tests.common import oracle_run
    budget = {"left": 1 << 16}
    live = {}

    def alloc(nbytes, stream):
        if nbytes > budget["left"]:
            return 0
        p = torch.cuda.caching_allocator_alloc(nbytes, stream=stream)
        budget["left"] -= nbytes
        live[p] = nbytes
        return p

    def release(p, nbytes, stream):
        torch.cuda.caching_allocator_delete(p)
        budget["left"] += live.pop(p)

    a, b = W.erdos_renyi(300, 1500, seed_index=200)
    e = Engine(allocator=(alloc, release))
    e.program(W.TC_PROGRAM)
    e.load("edge", (a, b))
    with pytest.raises(LobsterError, match="OOM"):
        e.run("unit")
    budget["left"] += 1 << 32
    e.reset()
    e.load("edge", (a, b))
    e.run("unit")
    want = oracle_run(W.TC_PROGRAM, {"edge": ((a, b),)}).relation("path")
    assert np.array_equal(e.read("path").cols, want.cols)
    e.close()
    torch.cuda.synchronize()
    assert not live  # every allocation was returned


def _poisoned_allocator(live):
    """An allocator whose every block starts as 0xFF bytes (a torch tensor kept
    alive until the engine releases it), so that no status word or counter of
    the engine can rely on memory an allocator happens to hand out zeroed."""
    import torch

    def alloc(nbytes, stream):
        t = torch.full((nbytes,), 0xFF, dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    def release(p, nbytes, stream):
        live.pop(p)

    return alloc, release


@pytest.mark.parametrize("semiring", ["unit", "max_min", "add_mult", "diff_max_min", "diff_add_mult"])
def test_status_words_do_not_depend_on_allocator_contents(semiring):
    """Runs through every flag-reporting step -- the difference+merge, the
    merge into a secondary view (the kinship program's kin(r1,x,y) probe by
    (r1, y)), the (+)-combination of candidate chunks -- with all-ones device
    memory from the allocator, against the oracle."""
    import torch
    live = {}
    alloc = _poisoned_allocator(live)
    g = W.grid_reach_instance(12, sub=12)
    src, dst, p = g["edge"]
    compare(W.REACH_PROGRAM, {"edge": ((src, dst), p), "start": (g["start"],)}, semiring, allocator=alloc)
    s = W.stream(130)
    n, r, a, b, pk = W.kinship_instance(s)
    c1, c2, c3 = W.composition_table()
    compare(W.KIN_PROGRAM, {"fact": ((r, a, b), pk), "comp": ((c1, c2, c3),)}, semiring, rels=["kin"],
            allocator=alloc)
    g = W.grid_reach_instance(40, sub=141)
    src, dst, p = g["edge"]
    compare(W.REACH_PROGRAM, {"edge": ((src, dst), p), "start": (g["start"],)}, semiring, options=CHUNK,
            allocator=alloc)
    torch.cuda.synchronize()
    assert not live  # every allocation was returned


def test_prim_diff_merge_with_poisoned_allocator():
    import torch
    from paper_2503_21937_gb300 import Engine
    live = {}
    e = Engine(allocator=_poisoned_allocator(live))
    s = W.stream(960)
    for call in range(2):  # the second call must not see the first one's flags
        F = np.unique(s.below(40_000, 1 << 24)).astype(np.uint32)
        U = np.unique(np.concatenate([F[::5], s.below(30_000, 1 << 24)])).astype(np.uint32)
        dev = lambda x: torch.from_numpy(x.astype(np.int32)).cuda()
        ok = torch.zeros(len(F) + len(U), dtype=torch.int32, device="cuda")
        rk = torch.zeros(len(U), dtype=torch.int32, device="cuda")
        no, nr = e.prim_diff_merge("unit", dev(F), None, dev(U), None, ok, None, rk, None)
        want_new = np.setdiff1d(U, F)
        assert nr == len(want_new)
        assert np.array_equal(rk.cpu().numpy().astype(np.uint32)[:nr], want_new)
        assert np.array_equal(ok.cpu().numpy().astype(np.uint32)[:no], np.union1d(F, U))
    e.close()
    torch.cuda.synchronize()
    assert not live


def test_read_capacity_error_reports_the_size():
    import ctypes
    from paper_2503_21937_gb300 import lobster
    a, b = W.ktree_chain(40)
    e, st, _ = engine_run(W.TC_PROGRAM, {"edge": ((a, b),)}, read=[])
    n = ctypes.c_uint64()
    cols = np.zeros((2, 5), np.uint32)
    rc = e.lib.lob_read_relation(e.h, e.ids["path"], cols.ctypes.data, None, None, 5, ctypes.byref(n),
                                 lobster.MEM_HOST)
    assert lobster.ERRORS[rc] == "LOB_E_CAPACITY"
    assert n.value == 40 * 39 // 2
    e.close()


def test_runs_are_bitwise_repeatable():
    parent, child, _ = W.random_tree(4000, seed_index=201)
    s, d = W.chung_lu_power_law(2000, 9000, seed_index=202)
    for program, inputs, rel, sr in [(W.SG_PROGRAM, {"parent": ((parent, child),)}, "sg", "unit"),
                                     (W.TC_PROGRAM, {"edge": ((s, d),)}, "path", "unit"),
                                     (W.TC_PROGRAM, {"edge": ((s, d), W.stream(203).prob(len(s)))}, "path", "max_min")]:
        outs = []
        for _ in range(2):
            e, st, got = engine_run(program, inputs, sr, read=[rel])
            outs.append(got[rel])
            e.close()
        assert np.array_equal(outs[0].cols, outs[1].cols)
        assert np.array_equal(outs[0].tags, outs[1].tags)


# ---------------------------------------------------------------------------
# device-driven iteration loop (a CUDA graph after the first iteration) vs the
# host-driven loop and the oracle
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("semiring", ["max_min", "add_mult", "diff_max_min", "diff_add_mult"])
@pytest.mark.parametrize("opts", [{"driver": 2}, {"driver": 2, "loop_cap_floor": 256}, {"driver": 0}])
def test_device_loop_matches_oracle(semiring, opts):
    """Linear (grid reachability) and non-linear, filtered, batched (kinship)
    programs; with a capacity floor of 256 rows the loop's buffers overflow and
    grow several times mid-run, each time resuming from the last committed
    iteration."""
    g = W.grid_reach_instance(20, sub=78)
    src, dst, p = g["edge"]
    st, _ = compare(W.REACH_PROGRAM, {"edge": ((src, dst), p), "start": (g["start"],)}, semiring, options=opts)
    if opts["driver"]:
        assert st["device_iterations"] > 0 and st["iterations"] > 30
        if "loop_cap_floor" not in opts:
            assert st["graph_launches"] == 1
    B = W.batched_instance(8)
    f, c = B["fact"], B["comp"]
    inputs = {"fact": ((f[0], f[1], f[2]), f[3], f[4]), "comp": ((c[0], c[1], c[2]), None, c[4])}
    st, _ = compare(W.KIN_PROGRAM, inputs, semiring, rels=["kin"], options=opts)
    if opts["driver"]:
        assert st["device_iterations"] > 0
        if "loop_cap_floor" in opts:
            assert st["graph_launches"] > 1


@pytest.mark.parametrize("semiring", ["max_min", "add_mult"])
def test_device_loop_max_iters(semiring):
    """LOB_E_MAXITER inside the device loop leaves the same state as the host loop."""
    from paper_2503_21937_gb300 import LobsterError
    g = W.grid_reach_instance(16, sub=79)
    src, dst, p = g["edge"]
    inputs = {"edge": ((src, dst), p), "start": (g["start"],)}
    got = []
    for driver in (2, 0):
        from paper_2503_21937_gb300 import Engine
        e = Engine()
        e.program(W.REACH_PROGRAM)
        e.set_option("driver", driver)
        e.load("edge", (src, dst), p)
        e.load("start", g["start"])
        with pytest.raises(LobsterError, match="MAXITER"):
            e.run(semiring, max_iters=9)
        got.append(e.read("reach"))
        e.close()
    assert np.array_equal(got[0].cols, got[1].cols)
    assert np.array_equal(got[0].tags, got[1].tags)


def test_device_loop_gradients_match_host_loop():
    """Backward after a device-driven forward uses the iteration records the
    loop kept on the device: gradients equal the host loop's."""
    B = W.batched_instance(6)
    e_ = B["edge"]
    inputs = {"edge": ((e_[0], e_[1]), e_[2], e_[3]), "start": ((B["start"][0],), None, B["start"][2])}
    grads = []
    for driver in (2, 0):
        e, st, got = engine_run(W.REACH_PROGRAM, inputs, "diff_add_mult", options={"driver": driver}, read=["reach"])
        gin = {"edge": np.zeros(len(e_[0]), np.float32)}
        e.backward("reach", np.linspace(-1, 1, got["reach"].cols.shape[1]).astype(np.float32), gin)
        grads.append(gin["edge"])
        e.close()
    np.testing.assert_allclose(grads[0], grads[1], rtol=1e-5, atol=1e-6)


def test_device_loop_takes_over_after_a_recorded_run():
    """Default option (driver 1): the first run of an engine is host-driven and
    records the sizes; a second run on the same engine plans the graph from
    them, launches it once, and waits for the host a few times per run, not
    per iteration; both runs match the oracle."""
    from paper_2503_21937_gb300 import Engine
    g = W.grid_reach_instance(24, sub=80)
    src, dst, p = g["edge"]
    want = compare(W.REACH_PROGRAM, {"edge": ((src, dst), p), "start": (g["start"],)}, "max_min")[1].relation("reach")
    e = Engine()
    e.program(W.REACH_PROGRAM)
    stats = []
    for _ in range(2):
        e.reset()
        e.load("edge", (src, dst), p)
        e.load("start", g["start"])
        stats.append(e.run("max_min"))
        got = e.read("reach")
        assert np.array_equal(got.cols, want.cols)
        assert np.array_equal(got.tags, want.tags.astype(np.float32))
    e.close()
    assert stats[0]["device_iterations"] == 0 and stats[1]["device_iterations"] == stats[1]["iterations"] - 1
    assert stats[1]["graph_launches"] == 1
    assert stats[1]["host_syncs"] < stats[0]["host_syncs"] / 5


@pytest.mark.parametrize("cross", [1, 0])
def test_cross_product_step(cross):
    """Same generation, whose recursive rule probes parent twice with keys from
    the delta row alone: the fused cross-product step (children(a) x
    children(b) straight into the membership bitmap) and the two-step
    pipeline, against the same-generation pairs by depth; also on a batched
    (sample-id) instance."""
    parent, child, depth = W.random_tree(5000, seed_index=31)
    opts = {"cross_join": cross, "bitmap_delta": 2}
    # element by element against the same-generation pairs by depth (which pin
    # the oracle; its naive run on these trees takes most of a minute)
    e, st, got = engine_run(W.SG_PROGRAM, {"parent": ((parent, child),)}, read=["sg"], options=opts)
    e.close()
    x, y = got["sg"].cols.astype(np.uint64)
    assert np.array_equal((x << np.uint64(32)) | y, pins.same_generation_keys(depth))
    assert st["derived"] == pins.same_generation_closed_form(depth)
    p2, c2, depth2 = W.random_tree(800, seed_index=32)
    samples = np.concatenate([np.zeros(len(parent), np.uint32), np.ones(len(p2), np.uint32)])
    e, st, got = engine_run(W.SG_PROGRAM, {"parent": ((np.concatenate([parent, p2]), np.concatenate([child, c2])),
                                                     None, samples)}, read=["sg"], options=opts)
    e.close()
    rel = got["sg"]
    for smp, d in ((0, depth), (1, depth2)):
        m = rel.samples == smp
        x, y = rel.cols[:, m].astype(np.uint64)
        assert np.array_equal((x << np.uint64(32)) | y, pins.same_generation_keys(d)), smp


# ---------------------------------------------------------------------------
# hash index of join prefixes (join_index = 3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("packed", [1, 0])
def test_hash_index_join(packed):
    """Join probes through the open-addressing hash index of each view's
    distinct prefixes, on the packed and the general kernels: transitive
    closure, same generation, Andersen (four rules, secondary views),
    batched kinship in a tagged semiring, and the backward pass."""
    opts = {"join_index": 3, "packed_join": packed}
    a, b = W.erdos_renyi(400, 1400, seed_index=150)
    compare(W.TC_PROGRAM, {"edge": ((a, b),)}, options=opts)
    parent, child, _ = W.random_tree(3000, seed_index=151)
    compare(W.SG_PROGRAM, {"parent": ((parent, child),)}, options=opts)
    A = W.andersen_program(3000, 9000, seed_index=152)
    compare(W.ANDERSEN_PROGRAM, {k: ((v[0], v[1]),) for k, v in A.items()}, rels=["pt"], options=opts)
    B = W.batched_instance(5)
    f, c = B["fact"], B["comp"]
    inputs = {"fact": ((f[0], f[1], f[2]), f[3], f[4]), "comp": ((c[0], c[1], c[2]), None, c[4])}
    compare(W.KIN_PROGRAM, inputs, "max_min", rels=["kin"], options=opts)
    g = W.grid_reach_instance(12, sub=153)
    src, dst, p = g["edge"]
    p = (p * 0.5).astype(np.float32)
    ins = {"edge": ((src, dst), p), "start": (g["start"],)}
    res = oracle_run(W.REACH_PROGRAM, ins, "diff_add_mult")
    gout = W.stream(154).normal(res.relation("reach").cols.shape[1])
    e, st, got = engine_run(W.REACH_PROGRAM, ins, "diff_add_mult", options=opts, read=["reach"])
    gin = {"edge": np.zeros(len(src), np.float32)}
    e.backward("reach", gout.astype(np.float32), gin)
    e.close()
    np.testing.assert_allclose(gin["edge"], res.vjp({"reach": gout})["edge"], rtol=1e-4, atol=1e-4)


def test_read_into_pinned_host_buffers_matches_pageable():
    """lob_read_relation writes page-locked, mapped host buffers directly from
    the read-out kernel; the rows equal those read through the staging copy,
    and a pageable or partly too small buffer still takes the staging path."""
    import torch
    from tests.common import engine_run
    s = W.stream(4711)
    src, dst, p = s.below(3000, 400), s.below(3000, 400), s.prob(3000)
    e, st, got = engine_run(W.TC_PROGRAM, {"edge": ((src, dst), p)}, "max_min", read=["path"])
    n = e.size("path")
    cols = torch.zeros((2, n + 5), dtype=torch.int32).pin_memory().numpy()
    tags = torch.zeros(n + 5, dtype=torch.float32).pin_memory().numpy()
    smp = torch.zeros(n + 5, dtype=torch.int32).pin_memory().numpy()
    assert e.read_into("path", cols, tags, smp) == n
    ref = got["path"]
    assert np.array_equal(cols[:, :n].view(np.uint32), ref.cols)
    assert np.array_equal(tags[:n], ref.tags)
    assert np.array_equal(smp[:n].view(np.uint32), ref.samples)
    # pinned columns with pageable tags: the staging path, same rows
    tags2 = np.zeros(n + 5, np.float32)
    cols[:] = 0
    assert e.read_into("path", cols, tags2, None) == n
    assert np.array_equal(cols[:, :n].view(np.uint32), ref.cols) and np.array_equal(tags2[:n], ref.tags)
    e.close()
