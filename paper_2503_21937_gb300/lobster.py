"""Python binding of the engine's C ABI (``include/lobster.h``).

Argument marshalling only: every step of the fixpoint runs in the CUDA
library ``liblobster.so``.  There is no CPU fallback; if the library is missing
or no GPU is present the calls raise.

Inputs may be numpy arrays (host memory) or CUDA torch tensors (device
memory, used in place on the current torch stream).
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblobster.so")

LOB_OK = 0
ERRORS = {-1: "LOB_E_ARG", -2: "LOB_E_PARSE", -3: "LOB_E_UNKNOWN_REL", -4: "LOB_E_UNSAFE_RULE", -5: "LOB_E_OOM",
          -6: "LOB_E_MAXITER", -7: "LOB_E_TIMEOUT", -8: "LOB_E_CUDA", -9: "LOB_E_CAPACITY", -10: "LOB_E_STATE",
          -11: "LOB_E_KEY_WIDTH"}
SEMIRINGS = {"unit": 0, "max_min": 1, "add_mult": 2, "diff_max_min": 3, "diff_add_mult": 4,
             "top1_proofs": 5, "diff_top1_proofs": 6}
MEM_HOST, MEM_DEVICE = 0, 1

# every symbol declared in include/lobster.h (checked by the tests)
EXPORTS = ["lob_create", "lob_destroy", "lob_last_error", "lob_declare_relation", "lob_relation_id",
           "lob_load_relation", "lob_add_rule", "lob_run_to_fixpoint", "lob_relation_size", "lob_read_relation",
           "lob_backward", "lob_reset", "lob_set_option", "lob_profile_count", "lob_profile_entry",
           "lob_profile_reset", "lob_prim_sort", "lob_prim_exclusive_scan", "lob_prim_unique",
           "lob_prim_diff_merge", "lob_unique_rows_noalloc", "lob_autotune", "lob_read_proofs"]
NOALLOC_MAX_ROWS = 262144

_lib = None


class LobsterError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_uint32), ("semiring", ctypes.c_uint32), ("derived", ctypes.c_uint64),
                ("candidates", ctypes.c_uint64), ("new_facts", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64),
                ("ms", ctypes.c_double), ("kernel_launches", ctypes.c_uint64), ("host_syncs", ctypes.c_uint64),
                ("device_iterations", ctypes.c_uint32), ("graph_launches", ctypes.c_uint32),
                ("proof_words", ctypes.c_uint64), ("strata", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class LobAlloc(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("release", _RELEASE_FN), ("ctx", ctypes.c_void_p)]


class TuneReport(ctypes.Structure):
    _fields_ = [("packed_join", ctypes.c_int32), ("warp_join", ctypes.c_int32), ("bitmap_delta", ctypes.c_int32),
                ("join_index", ctypes.c_int32), ("radix_bits", ctypes.c_int32), ("emit_filter", ctypes.c_int32),
                ("trials", ctypes.c_uint32), ("first_ms", ctypes.c_double), ("best_ms", ctypes.c_double),
                ("acc_dense", ctypes.c_int32), ("cross_join", ctypes.c_int32), ("hash_slots", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def load_library(path: str = LIB_PATH):
    """Load liblobster.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2503_21937_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, vp, u32, u64 = ctypes.POINTER, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    lib.lob_create.argtypes = [P(vp), vp, vp]
    lib.lob_destroy.argtypes = [vp]
    lib.lob_destroy.restype = None
    lib.lob_last_error.argtypes = [vp]
    lib.lob_last_error.restype = ctypes.c_char_p
    lib.lob_declare_relation.argtypes = [vp, ctypes.c_char_p, u32, P(u32)]
    lib.lob_relation_id.argtypes = [vp, ctypes.c_char_p, P(u32)]
    lib.lob_load_relation.argtypes = [vp, u32, vp, vp, vp, u64, ctypes.c_int]
    lib.lob_add_rule.argtypes = [vp, ctypes.c_char_p]
    lib.lob_run_to_fixpoint.argtypes = [vp, ctypes.c_int, u32, P(Stats)]
    lib.lob_autotune.argtypes = [vp, ctypes.c_int, u32, u32, P(TuneReport)]
    lib.lob_relation_size.argtypes = [vp, u32, P(u64)]
    lib.lob_read_relation.argtypes = [vp, u32, vp, vp, vp, u64, P(u64), ctypes.c_int]
    lib.lob_backward.argtypes = [vp, u32, vp, vp, ctypes.c_int]
    lib.lob_read_proofs.argtypes = [vp, u32, vp, vp, u64, P(u64), ctypes.c_int]
    lib.lob_reset.argtypes = [vp]
    lib.lob_set_option.argtypes = [vp, ctypes.c_char_p, ctypes.c_int64]
    lib.lob_profile_count.argtypes = [vp, P(u32)]
    lib.lob_profile_entry.argtypes = [vp, u32, ctypes.c_char_p, ctypes.c_size_t, P(u64), P(ctypes.c_double),
                                      P(ctypes.c_double)]
    lib.lob_profile_reset.argtypes = [vp]
    lib.lob_unique_rows_noalloc.argtypes = [vp, u32, u64, vp, vp, vp]
    lib.lob_prim_sort.argtypes = [vp, vp, vp, u64, u32, u32, u32]
    lib.lob_prim_exclusive_scan.argtypes = [vp, vp, vp, u64, P(u64)]
    lib.lob_prim_unique.argtypes = [vp, ctypes.c_int, vp, vp, u64, u32, vp, vp, P(u64)]
    lib.lob_prim_diff_merge.argtypes = [vp, ctypes.c_int, vp, vp, u64, vp, vp, u64, u32, vp, vp, vp, vp, P(u64),
                                        P(u64)]
    _lib = lib
    return lib


_ATOM = re.compile(r"([A-Za-z_][A-Za-z0-9_]*)\s*\(([^()]*)\)")


def relation_arities(program: str) -> dict:
    """Relation name -> arity for every atom in the program text."""
    out = {}
    for line in program.splitlines():
        line = re.split(r"//|#|%", line)[0]
        for name, args in _ATOM.findall(line):
            out[name] = len([a for a in args.split(",") if a.strip()])
    return out


def split_rules(program: str) -> list:
    text = "\n".join(re.split(r"//|#|%", l)[0] for l in program.splitlines())
    return [r.strip() + "." for r in text.split(".") if r.strip()]


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _torch_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def unique_rows_noalloc(cols, out_cols, n_out, stream=None) -> int:
    """Distinct rows of a (arity, n) int32 CUDA tensor, sorted, written into the
    caller's out_cols ((arity, n) int32 CUDA tensor) and n_out (one int64 CUDA
    element), without any device allocation by the library.  Returns the status
    code of lob_unique_rows_noalloc (0 on success)."""
    lib = load_library()
    arity, n = cols.shape
    stream = _torch_stream() if stream is None else stream
    return lib.lob_unique_rows_noalloc(cols.data_ptr(), arity, n, out_cols.data_ptr(), n_out.data_ptr(),
                                       ctypes.c_void_p(stream) if stream else None)


@dataclass
class Relation:
    cols: object   # (arity, n) uint32 numpy array or torch int32 tensor
    tags: object   # (n,) float32
    samples: object


class Engine:
    """One fixpoint engine on the current CUDA device."""

    def __init__(self, stream=None, allocator=None):
        """allocator: optional (alloc(nbytes, stream) -> device pointer or 0,
        release(ptr, nbytes, stream)) pair passed to lob_create as lob_alloc."""
        self.lib = load_library()
        self.h = ctypes.c_void_p()
        stream = _torch_stream() if stream is None else stream
        alloc = None
        if allocator is not None:
            fa, fr = allocator
            self._alloc_cbs = (_ALLOC_FN(lambda n, st, ctx: fa(n, st or 0) or None),
                               _RELEASE_FN(lambda p, n, st, ctx: fr(p, n, st or 0)))
            self._alloc_struct = LobAlloc(self._alloc_cbs[0], self._alloc_cbs[1], None)
            alloc = ctypes.cast(ctypes.pointer(self._alloc_struct), ctypes.c_void_p)
        rc = self.lib.lob_create(ctypes.byref(self.h), alloc, ctypes.c_void_p(stream) if stream else None)
        if rc != LOB_OK:
            raise LobsterError(rc, self.lib.lob_last_error(None).decode())
        self.ids = {}
        self.arity = {}

    def close(self):
        if self.h:
            self.lib.lob_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _chk(self, rc):
        if rc != LOB_OK:
            raise LobsterError(rc, self.lib.lob_last_error(self.h).decode())
        return rc

    def declare(self, name: str, arity: int) -> int:
        rid = ctypes.c_uint32()
        self._chk(self.lib.lob_declare_relation(self.h, name.encode(), arity, ctypes.byref(rid)))
        self.ids[name] = rid.value
        self.arity[name] = arity
        return rid.value

    def program(self, text: str):
        """Declare every relation the program mentions (arity from its atoms) and add its rules."""
        for name, ar in relation_arities(text).items():
            if name not in self.ids:
                self.declare(name, ar)
        for r in split_rules(text):
            self.add_rule(r)

    def add_rule(self, text: str):
        self._chk(self.lib.lob_add_rule(self.h, text.encode()))

    def set_option(self, key: str, value: int):
        self._chk(self.lib.lob_set_option(self.h, key.encode(), int(value)))

    def load(self, name: str, cols, tags=None, samples=None):
        """cols: (arity, n) array/tensor or a sequence of n-long columns."""
        rid = self.ids[name]
        if _is_torch(cols) or (isinstance(cols, (list, tuple)) and cols and _is_torch(cols[0])):
            import torch
            c = cols if _is_torch(cols) else torch.stack(list(cols))
            c = c.to(torch.int32).contiguous()
            n = c.shape[1]
            t = tags.to(torch.float32).contiguous() if tags is not None else None
            s = samples.to(torch.int32).contiguous() if samples is not None else None
            self._chk(self.lib.lob_load_relation(self.h, rid, c.data_ptr(), t.data_ptr() if t is not None else None,
                                                 s.data_ptr() if s is not None else None, n, MEM_DEVICE))
            return
        c = np.ascontiguousarray(np.asarray(cols, dtype=np.uint32).reshape(len(cols), -1))
        n = c.shape[1]
        t = np.ascontiguousarray(np.asarray(tags, np.float32)) if tags is not None else None
        s = np.ascontiguousarray(np.asarray(samples, np.uint32)) if samples is not None else None
        self._chk(self.lib.lob_load_relation(self.h, rid, c.ctypes.data, t.ctypes.data if t is not None else None,
                                             s.ctypes.data if s is not None else None, n, MEM_HOST))

    def run(self, semiring="unit", max_iters: int = 1 << 30) -> dict:
        sr = SEMIRINGS[semiring] if isinstance(semiring, str) else int(semiring)
        st = Stats()
        self._chk(self.lib.lob_run_to_fixpoint(self.h, sr, max_iters, ctypes.byref(st)))
        return st.as_dict()

    def autotune(self, semiring="unit", max_iters: int = 1 << 30, repeats: int = 3) -> dict:
        """lob_autotune: choose strategy options for the loaded program by timed
        fixpoint runs; the inputs stay loaded and run() comes next."""
        sr = SEMIRINGS[semiring] if isinstance(semiring, str) else int(semiring)
        rep = TuneReport()
        self._chk(self.lib.lob_autotune(self.h, sr, max_iters, repeats, ctypes.byref(rep)))
        return rep.as_dict()

    def size(self, name: str) -> int:
        n = ctypes.c_uint64()
        self._chk(self.lib.lob_relation_size(self.h, self.ids[name], ctypes.byref(n)))
        return n.value

    def read(self, name: str, device: bool = False) -> Relation:
        n = self.size(name)
        ar = self.arity[name]
        if device:
            import torch
            cols = torch.empty((ar, max(n, 1)), dtype=torch.int32, device="cuda")
            tags = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
            smp = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
            got = ctypes.c_uint64()
            self._chk(self.lib.lob_read_relation(self.h, self.ids[name], cols.data_ptr(), tags.data_ptr(),
                                                 smp.data_ptr(), max(n, 1), ctypes.byref(got), MEM_DEVICE))
            return Relation(cols[:, :n], tags[:n], smp[:n])
        cols = np.zeros((ar, max(n, 1)), np.uint32)
        tags = np.zeros(max(n, 1), np.float32)
        smp = np.zeros(max(n, 1), np.uint32)
        got = ctypes.c_uint64()
        self._chk(self.lib.lob_read_relation(self.h, self.ids[name], cols.ctypes.data, tags.ctypes.data,
                                             smp.ctypes.data, max(n, 1), ctypes.byref(got), MEM_HOST))
        return Relation(cols[:, :n], tags[:n], smp[:n])

    def read_into(self, name: str, cols, tags=None, samples=None) -> int:
        """Read into preallocated host arrays: cols (arity, capacity) uint32/int32
        C-contiguous, tags/samples (capacity,) or None.  Returns the row count."""
        cap = cols.shape[1]
        got = ctypes.c_uint64()
        self._chk(self.lib.lob_read_relation(self.h, self.ids[name], cols.ctypes.data,
                                             tags.ctypes.data if tags is not None else None,
                                             samples.ctypes.data if samples is not None else None, cap,
                                             ctypes.byref(got), MEM_HOST))
        return got.value

    def proofs(self, name: str) -> list:
        """top-1-proofs: per fact of ``read(name)`` (same order) its proof, an
        ascending uint32 array of input-fact ids (row q of relation k has id q
        plus the rows loaded into the relations declared before k)."""
        n = self.size(name)
        lens = np.zeros(max(n, 1), np.uint32)
        total = ctypes.c_uint64()
        self._chk(self.lib.lob_read_proofs(self.h, self.ids[name], lens.ctypes.data, None, 0, ctypes.byref(total),
                                           MEM_HOST))
        ids = np.zeros(max(total.value, 1), np.uint32)
        self._chk(self.lib.lob_read_proofs(self.h, self.ids[name], None, ids.ctypes.data, total.value,
                                           ctypes.byref(total), MEM_HOST))
        if n == 0:
            return []
        return np.split(ids[:total.value], np.cumsum(lens[:n].astype(np.int64))[:-1])

    def backward(self, out_name: str, grad, grad_inputs: dict):
        """grad: gradient per fact of out_name (read order).  grad_inputs: name ->
        float32 array (host) or tensor (device) of the relation's loaded-row count;
        gradients are added into them."""
        device = _is_torch(grad)
        nrel = max(self.ids.values()) + 1
        ptrs = (ctypes.c_void_p * nrel)()
        keep = []
        if device:
            g = grad.to(dtype=__import__("torch").float32).contiguous()
            for k, v in grad_inputs.items():
                ptrs[self.ids[k]] = v.data_ptr()
            gp = g.data_ptr()
        else:
            g = np.ascontiguousarray(np.asarray(grad, np.float32))
            for k, v in grad_inputs.items():
                assert v.dtype == np.float32 and v.flags["C_CONTIGUOUS"]
                ptrs[self.ids[k]] = v.ctypes.data
            gp = g.ctypes.data
        keep.append(g)
        self._chk(self.lib.lob_backward(self.h, self.ids[out_name], gp, ptrs, MEM_DEVICE if device else MEM_HOST))

    def reset(self):
        self._chk(self.lib.lob_reset(self.h))

    # kernel-level primitives on CUDA tensors (used by the kernel tests)
    def prim_sort(self, keys, payload=None, key_bits=None):
        kb = keys.element_size()
        pb = payload.element_size() if payload is not None else 0
        bits = kb * 8 if key_bits is None else key_bits
        self._chk(self.lib.lob_prim_sort(self.h, keys.data_ptr(), payload.data_ptr() if payload is not None else None,
                                         keys.numel(), bits, kb, pb))

    def prim_scan(self, x, out):
        tot = ctypes.c_uint64()
        self._chk(self.lib.lob_prim_exclusive_scan(self.h, x.data_ptr(), out.data_ptr(), x.numel(), ctypes.byref(tot)))
        return tot.value

    def prim_unique(self, semiring, keys, tags, out_keys, out_tags):
        n = ctypes.c_uint64()
        sr = SEMIRINGS[semiring] if isinstance(semiring, str) else semiring
        self._chk(self.lib.lob_prim_unique(self.h, sr, keys.data_ptr(), tags.data_ptr() if tags is not None else None,
                                           keys.numel(), keys.element_size(), out_keys.data_ptr(),
                                           out_tags.data_ptr() if out_tags is not None else None, ctypes.byref(n)))
        return n.value

    def prim_diff_merge(self, semiring, fk, ft, uk, ut, ok, ot, rk, rt):
        no, nr = ctypes.c_uint64(), ctypes.c_uint64()
        sr = SEMIRINGS[semiring] if isinstance(semiring, str) else semiring
        p = lambda t: t.data_ptr() if t is not None else None
        self._chk(self.lib.lob_prim_diff_merge(self.h, sr, p(fk), p(ft), fk.numel(), p(uk), p(ut), uk.numel(),
                                               fk.element_size(), p(ok), p(ot), p(rk), p(rt), ctypes.byref(no),
                                               ctypes.byref(nr)))
        return no.value, nr.value

    def profile(self) -> dict:
        """kernel name -> {launches, ms, bytes} accumulated since the last profile_reset."""
        n = ctypes.c_uint32()
        self._chk(self.lib.lob_profile_count(self.h, ctypes.byref(n)))
        out = {}
        buf = ctypes.create_string_buffer(128)
        for i in range(n.value):
            la, ms, by = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_double()
            self._chk(self.lib.lob_profile_entry(self.h, i, buf, 128, ctypes.byref(la), ctypes.byref(ms),
                                                 ctypes.byref(by)))
            out[buf.value.decode()] = {"launches": la.value, "ms": ms.value, "bytes": by.value}
        return out

    def profile_reset(self):
        self._chk(self.lib.lob_profile_reset(self.h))
