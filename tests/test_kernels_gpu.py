"""Kernel-level tests of the sort / scan / unique / difference-merge primitives
(through the C ABI) against plain numpy definitions, including adversarial
inputs: empty, single element, tile boundaries, all-equal keys, every key bit
used, maximal skew."""
import numpy as np
import pytest

from paper_2503_21937_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    from paper_2503_21937_gb300 import Engine, build
    build.build()
    e = Engine()
    yield e
    e.close()
    torch.cuda.synchronize()


def _dev(a):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).cuda()
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).cuda()
    return torch.from_numpy(a).cuda()


def _host(t, dtype):
    return t.cpu().numpy().view(dtype)


SORT_CASES = [(0, 32), (1, 32), (2, 8), (4095, 20), (4096, 30), (4097, 32), (100_003, 30), (1_000_000, 17),
              (262_145, 32)]


@pytest.mark.parametrize("n,bits", SORT_CASES)
def test_sort_u32_with_payload_is_stable(eng, n, bits):
    s = W.stream(300 + n % 97)
    keys = (s.take(n) & np.uint64((1 << bits) - 1)).astype(np.uint32)
    pay = np.arange(n, dtype=np.uint32)
    k, p = _dev(keys), _dev(pay)
    eng.prim_sort(k, p, key_bits=bits)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(_host(k, np.uint32), keys[order])
    assert np.array_equal(_host(p, np.uint32), pay[order])


@pytest.mark.parametrize("bits", [36, 64])
def test_sort_u64_keys_every_bit(eng, bits):
    n = 300_001
    s = W.stream(400 + bits)
    mask = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    keys = s.take(n) & mask
    keys[:10] = mask  # all bits set
    keys[10:20] = 0
    pay = s.take(n)
    k, p = _dev(keys), _dev(pay)
    eng.prim_sort(k, p, key_bits=bits)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(_host(k, np.uint64), keys[order])
    assert np.array_equal(_host(p, np.uint64), pay[order])


@pytest.mark.parametrize("pattern", ["equal", "sorted", "reversed", "two_values"])
def test_sort_adversarial(eng, pattern):
    n = 70_000
    if pattern == "equal":
        keys = np.full(n, 12345, np.uint32)
    elif pattern == "sorted":
        keys = np.arange(n, dtype=np.uint32) * 7
    elif pattern == "reversed":
        keys = (np.arange(n, dtype=np.uint32) * 7)[::-1].copy()
    else:
        keys = (np.arange(n) % 2).astype(np.uint32) * 0xFFFFFF00
    pay = np.arange(n, dtype=np.uint32)
    k, p = _dev(keys), _dev(pay)
    eng.prim_sort(k, p, key_bits=32)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(_host(k, np.uint32), keys[order])
    assert np.array_equal(_host(p, np.uint32), pay[order])


@pytest.mark.parametrize("n,bits,pay", [(1, 30, 4), (4097, 30, 4), (1_000_003, 30, 0), (300_001, 36, 8), (70_000, 32, 4)])
def test_sort_lookback_variant(eng, n, bits, pay):
    eng.set_option("sort_algo", 1)
    try:
        s = W.stream(520 + n % 11)
        mask = np.uint64((1 << bits) - 1)
        keys = s.take(n) & mask
        keys = keys.astype(np.uint32) if bits <= 32 else keys
        if n > 100:
            keys[:50] = keys[0]  # a run of equal keys
        p = np.arange(n, dtype=np.uint32) if pay == 4 else (s.take(n) if pay == 8 else None)
        k = _dev(keys)
        pd = _dev(p) if p is not None else None
        eng.prim_sort(k, pd, key_bits=bits)
        order = np.argsort(keys, kind="stable")
        assert np.array_equal(_host(k, keys.dtype), keys[order])
        if p is not None:
            assert np.array_equal(_host(pd, p.dtype), p[order])
    finally:
        eng.set_option("sort_algo", 0)


def test_sort_keys_only(eng):
    n = 500_000
    keys = W.stream(501).below(n, 1 << 30)
    k = _dev(keys)
    eng.prim_sort(k, None, key_bits=30)
    assert np.array_equal(_host(k, np.uint32), np.sort(keys))


@pytest.mark.parametrize("n", [0, 1, 2047, 2048, 2049, 5_000_000])
def test_exclusive_scan(eng, n):
    import torch
    x = W.stream(600).below(n, 1000)
    out = torch.zeros(max(n, 1), dtype=torch.int64, device="cuda")
    tot = eng.prim_scan(_dev(x), out)
    ref = np.concatenate([[0], np.cumsum(x.astype(np.uint64))[:-1]]) if n else np.zeros(0)
    assert tot == int(x.astype(np.uint64).sum())
    assert np.array_equal(out.cpu().numpy()[:n].astype(np.uint64), ref.astype(np.uint64))


def _runs(n, nkeys, seed, with_invalid=True):
    s = W.stream(700 + seed)
    keys = np.sort(s.below(n, nkeys))
    if with_invalid and n > 10:
        keys[-5:] = 0xFFFFFFFF
    return keys


@pytest.mark.parametrize("n,nkeys", [(1, 10), (5000, 10), (100_000, 90_000), (300_000, 3), (4096 * 3, 1)])
def test_unique_unit_and_maxmin(eng, n, nkeys):
    import torch
    keys = _runs(n, nkeys, n % 13)
    valid = keys != 0xFFFFFFFF
    want = np.unique(keys[valid])
    ok = torch.zeros(n, dtype=torch.int32, device="cuda")
    m = eng.prim_unique("unit", _dev(keys), None, ok, None)
    assert m == len(want)
    assert np.array_equal(_host(ok, np.uint32)[:m], want)
    tags = W.stream(800).prob(n)
    ot = torch.zeros(n, dtype=torch.float32, device="cuda")
    m = eng.prim_unique("max_min", _dev(keys), _dev(tags), ok, ot)
    ref = {}
    for k, t in zip(keys[valid].tolist(), tags[valid].tolist()):
        ref[k] = max(ref.get(k, 0.0), t)
    assert np.array_equal(_host(ot, np.float32)[:m], np.array([ref[k] for k in want], np.float32))


def test_unique_addmult_sums_runs_in_fp64(eng):
    import torch
    n = 200_000
    keys = _runs(n, 20_000, 5)
    tags = W.stream(801).unit(n)
    ok = torch.zeros(n, dtype=torch.int32, device="cuda")
    ot = torch.zeros(n, dtype=torch.float64, device="cuda")
    m = eng.prim_unique("add_mult", _dev(keys), _dev(tags), ok, ot)
    valid = keys != 0xFFFFFFFF
    want_k, inv = np.unique(keys[valid], return_inverse=True)
    want_t = np.zeros(len(want_k))
    np.add.at(want_t, inv, tags[valid])
    assert m == len(want_k)
    np.testing.assert_allclose(ot.cpu().numpy()[:m], want_t, rtol=1e-12)


@pytest.mark.parametrize("nf,nu,overlap", [(0, 1000, 0.0), (1000, 0, 0.0), (100_000, 50_000, 0.5), (3000, 300_000, 0.01),
                                           (200_000, 200_000, 1.0), (1, 1, 1.0)])
def test_diff_merge_unit(eng, nf, nu, overlap):
    import torch
    s = W.stream(900 + nf % 7 + nu % 11)
    F = np.unique(s.below(nf * 2 + 1, 1 << 28))[:nf]
    n_ov = int(overlap * min(nu, len(F)))
    U = np.unique(np.concatenate([F[:n_ov], s.below(max(nu - n_ov, 0), 1 << 28)]))[:nu] if nu else np.zeros(0, np.uint32)
    F = F.astype(np.uint32)
    U = np.sort(U).astype(np.uint32)
    cap = len(F) + len(U) + 1
    ok = torch.zeros(cap, dtype=torch.int32, device="cuda")
    rk = torch.zeros(max(len(U), 1), dtype=torch.int32, device="cuda")
    no, nr = eng.prim_diff_merge("unit", _dev(F), None, _dev(U), None, ok, None, rk, None)
    want_new = np.setdiff1d(U, F)
    assert nr == len(want_new)
    assert np.array_equal(_host(rk, np.uint32)[:nr], want_new)
    assert np.array_equal(_host(ok, np.uint32)[:no], np.union1d(F, U))


def test_diff_merge_maxmin_improvement(eng):
    import torch
    s = W.stream(950)
    F = np.unique(s.below(50_000, 1 << 20)).astype(np.uint32)
    U = np.unique(np.concatenate([F[::3], s.below(20_000, 1 << 20)])).astype(np.uint32)
    ft = s.prob(len(F))
    ut = s.prob(len(U))
    ok = torch.zeros(len(F) + len(U), dtype=torch.int32, device="cuda")
    ot = torch.zeros(len(F) + len(U), dtype=torch.float32, device="cuda")
    rk = torch.zeros(len(U), dtype=torch.int32, device="cuda")
    rt = torch.zeros(len(U), dtype=torch.float32, device="cuda")
    no, nr = eng.prim_diff_merge("max_min", _dev(F), _dev(ft), _dev(U), _dev(ut), ok, ot, rk, rt)
    fmap = dict(zip(F.tolist(), ft.tolist()))
    merged = dict(fmap)
    recent = {}
    for k, t in zip(U.tolist(), ut.tolist()):
        if k not in fmap or t > fmap[k]:
            recent[k] = t
            merged[k] = t
    mk = np.array(sorted(merged), np.uint32)
    assert no == len(mk) and nr == len(recent)
    assert np.array_equal(_host(ok, np.uint32)[:no], mk)
    assert np.array_equal(_host(ot, np.float32)[:no], np.array([merged[k] for k in mk.tolist()], np.float32))
    rkk = np.array(sorted(recent), np.uint32)
    assert np.array_equal(_host(rk, np.uint32)[:nr], rkk)
    assert np.array_equal(_host(rt, np.float32)[:nr], np.array([recent[k] for k in rkk.tolist()], np.float32))
