"""CPU oracle for the semiring Datalog fixpoint -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA engine in
``paper_2503_21937_gb300``) never calls it and shares no code with it.

The arithmetic lives in ``oracle.cpp`` (naive Kleene iteration over
``std::map`` relations with FP64 tags; see its header for the definitions and
the paper passages they follow).  This module compiles it with g++ on first
use and wraps its C interface with ctypes.

Parity status per function (pins are in ``tests/test_oracle_pins.py``):
  * unit semiring fixpoint        -- pinned (closed forms, BFS, tree depths, worklist Andersen)
  * max-min-prob / diff-max-min   -- pinned (possible worlds, widest path, chains)
  * add-mult-prob / diff-add-mult -- pinned (layered DP, lattice-path closed form, trees)
  * forward-mode gradients        -- pinned (FP64 central finite differences)
  * batching by sample id         -- pinned (per-sample runs)
  * top-1-proofs / diff-top-1     -- pinned (max-product paths by Dijkstra, the
                                     paper's printed proof, union of shared
                                     facts, brute-force two-hop maxima, the cap,
                                     finite differences)
  * computed heads and filters    -- pinned (bounded walk lengths by boolean
                                     matrix powers; wrap-around, division,
                                     reserved value by direct u32 arithmetic)
  * strata run one after another  -- pinned (sums over every path of a chain's
                                     closure, mutually recursive odd/even
                                     lengths, widest paths by Floyd-Warshall,
                                     rules written in reverse order, finite
                                     differences, a top-1 proof that reads
                                     the stratum below when it is finished)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
# ORACLE_MUTANT=k (k > 0) selects a library with one deliberate mistake compiled
# in (oracle.cpp lists them); only tests/test_oracle_mutants.py sets it, to show
# that the pins catch each mistake.  Unset: the oracle itself.
_MUTANT = int(os.environ.get("ORACLE_MUTANT", "0"))
_LIB = os.path.join(_HERE, "liboracle.so" if _MUTANT == 0 else f"liboracle_mutant{_MUTANT}.so")
_lock = threading.Lock()
_lib = None

SEMIRINGS = {"unit": 0, "max_min": 1, "add_mult": 2, "diff_max_min": 3, "diff_add_mult": 4,
             "top1_proofs": 5, "diff_top1_proofs": 6}


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (g++, no GPU code)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-shared", "-fPIC", f"-DORACLE_MUTANT={_MUTANT}", "-o", tmp, _SRC],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            lib.orc_run.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_int, P(ctypes.c_char_p),
                                    P(ctypes.c_uint32), P(ctypes.c_uint64), P(ctypes.c_void_p),
                                    P(ctypes.c_void_p), P(ctypes.c_void_p), ctypes.c_uint32,
                                    P(ctypes.c_void_p)]
            lib.orc_run.restype = ctypes.c_int
            lib.orc_error.restype = ctypes.c_char_p
            lib.orc_iterations.argtypes = [ctypes.c_void_p]
            lib.orc_size.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
            lib.orc_size.restype = ctypes.c_int64
            lib.orc_arity.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
            lib.orc_read.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]
            lib.orc_read_ids.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_void_p]
            lib.orc_vjp.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_void_p, P(ctypes.c_void_p)]
            lib.orc_free.argtypes = [ctypes.c_void_p]
            lib.orc_set_proof_cap.argtypes = [ctypes.c_uint32]
            lib.orc_ties.argtypes = [ctypes.c_void_p]
            lib.orc_ties.restype = ctypes.c_uint64
            lib.orc_read_proofs.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_read_proofs.restype = ctypes.c_int64
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"oracle error {code}: {msg}")
        self.code = code


@dataclass
class Relation:
    cols: np.ndarray      # (arity, n) uint32, sorted by (sample, cols)
    tags: np.ndarray      # (n,) float64
    samples: np.ndarray   # (n,) uint32


class Result:
    """Outcome of one oracle run; owns the C result handle."""

    def __init__(self, handle, input_names, input_sizes, semiring):
        self._h = handle
        self.input_names = input_names
        self.input_sizes = input_sizes
        self.semiring = semiring

    def __del__(self):
        if getattr(self, "_h", None):
            _load().orc_free(self._h)
            self._h = None

    @property
    def iterations(self) -> int:
        return _load().orc_iterations(self._h)

    def relation(self, name: str) -> Relation:
        lib = _load()
        n = lib.orc_size(self._h, name.encode())
        if n < 0:
            raise KeyError(name)
        ar = lib.orc_arity(self._h, name.encode())
        cols = np.zeros((ar, n), np.uint32)
        tags = np.zeros(n, np.float64)
        smp = np.zeros(n, np.uint32)
        lib.orc_read(self._h, name.encode(), cols.ctypes.data, tags.ctypes.data, smp.ctypes.data)
        return Relation(cols, tags, smp)

    def ids(self, name: str) -> np.ndarray:
        n = _load().orc_size(self._h, name.encode())
        out = np.zeros(max(n, 0), np.uint32)
        _load().orc_read_ids(self._h, name.encode(), out.ctypes.data)
        return out

    @property
    def ties(self) -> int:
        """top-1-proofs: how often (+) met two different, equally likely proofs."""
        return int(_load().orc_ties(self._h))

    def proofs(self, name: str) -> list:
        """top-1-proofs: per fact of ``relation(name)`` (same order) its proof,
        an ascending array of input-fact ids (global row index over the inputs
        in load order)."""
        lib = _load()
        n = lib.orc_size(self._h, name.encode())
        total = lib.orc_read_proofs(self._h, name.encode(), None, None)
        lens = np.zeros(max(n, 0), np.uint32)
        ids = np.zeros(max(total, 0), np.uint32)
        lib.orc_read_proofs(self._h, name.encode(), lens.ctypes.data, ids.ctypes.data)
        return np.split(ids, np.cumsum(lens.astype(np.int64))[:-1]) if n > 0 else []

    def vjp(self, grads: dict) -> dict:
        """grads: relation -> upstream gradient aligned with ``relation(name)``.
        Returns input relation -> gradient aligned with its loaded rows."""
        lib = _load()
        outs = {k: np.zeros(n, np.float64) for k, n in zip(self.input_names, self.input_sizes)}
        ptrs = (ctypes.c_void_p * len(outs))(*[outs[k].ctypes.data for k in self.input_names])
        for name, g in grads.items():
            g = np.ascontiguousarray(g, np.float64)
            rc = lib.orc_vjp(self._h, name.encode(), g.ctypes.data, ptrs)
            if rc != 0:
                raise OracleError(rc, "vjp needs a diff semiring")
        return outs


def run(program: str, inputs: dict, semiring="unit", max_iters: int = 100000, proof_cap: int = 300) -> Result:
    """Run the naive fixpoint.  ``proof_cap`` bounds the proofs of the
    top-1-proofs semirings (a longer union is an error).

    inputs: name -> (cols, tags, samples) with cols an (arity, n) array (or a
    sequence of n-long columns), tags a length-n float array or None (tag 1,
    not differentiable) and samples a length-n uint32 array or None."""
    lib = _load()
    sr = SEMIRINGS[semiring] if isinstance(semiring, str) else int(semiring)
    names, arities, sizes, keep = [], [], [], []
    col_ptrs, tag_ptrs, smp_ptrs = [], [], []
    for name, spec in inputs.items():
        cols, tags, samples = (list(spec) + [None, None])[:3]
        cols = np.ascontiguousarray(np.asarray(cols, dtype=np.uint32).reshape(len(cols), -1))
        n = cols.shape[1]
        names.append(name)
        arities.append(cols.shape[0])
        sizes.append(n)
        keep.append(cols)
        col_ptrs.append(cols.ctypes.data)
        if tags is not None:
            t = np.ascontiguousarray(np.asarray(tags, dtype=np.float64))
            keep.append(t)
            tag_ptrs.append(t.ctypes.data)
        else:
            tag_ptrs.append(None)
        if samples is not None:
            s = np.ascontiguousarray(np.asarray(samples, dtype=np.uint32))
            keep.append(s)
            smp_ptrs.append(s.ctypes.data)
        else:
            smp_ptrs.append(None)
    k = len(names)
    c_names = (ctypes.c_char_p * k)(*[n.encode() for n in names])
    c_ar = (ctypes.c_uint32 * k)(*arities)
    c_n = (ctypes.c_uint64 * k)(*sizes)
    c_cols = (ctypes.c_void_p * k)(*col_ptrs)
    c_tags = (ctypes.c_void_p * k)(*tag_ptrs)
    c_smp = (ctypes.c_void_p * k)(*smp_ptrs)
    h = ctypes.c_void_p()
    lib.orc_set_proof_cap(int(proof_cap))
    rc = lib.orc_run(program.encode(), sr, k, c_names, c_ar, c_n, c_cols, c_tags, c_smp, max_iters,
                     ctypes.byref(h))
    if rc != 0:
        raise OracleError(rc, lib.orc_error().decode())
    return Result(h, names, sizes, sr)
