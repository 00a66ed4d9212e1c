"""CPU-side checks of the C-ABI library: it builds, loads, and exports every
symbol include/lobster.h declares (no compute call: there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    out = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            out.update(re.findall(r"\b(lob_[a-z0-9_]+)\s*\(", text))
    return out


def test_library_builds_and_exports_all_declared_symbols():
    from paper_2503_21937_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert {"lob_create", "lob_run_to_fixpoint", "lob_backward"} <= syms
    for s in sorted(syms):
        assert hasattr(lib, s), s


def test_binding_lists_every_export():
    from paper_2503_21937_gb300 import lobster
    assert declared_symbols() == set(lobster.EXPORTS)


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2503_21937_gb300 import Engine, LobsterError
    with pytest.raises(LobsterError):
        Engine()


def test_relation_arity_scan():
    from paper_2503_21937_gb300 import lobster, workloads as W
    assert lobster.relation_arities(W.ANDERSEN_PROGRAM) == {"pt": 2, "addr": 2, "assign": 2, "load": 2, "store": 2}
    assert lobster.relation_arities(W.KIN_PROGRAM) == {"kin": 3, "fact": 3, "comp": 3}
    assert len(lobster.split_rules(W.SG_PROGRAM)) == 2


def test_every_engine_option_is_documented_in_the_header():
    src = open(os.path.join(ROOT, "paper_2503_21937_gb300", "csrc", "engine.cu")).read()
    body = src[src.index("int lob_set_option("):]
    body = body[: body.index("\n}\n")]
    keys = set(re.findall(r'k == "([a-z_]+)"', body))
    header = open(os.path.join(ROOT, "include", "lobster.h")).read()
    doc = header[header.index("Engine options (key, value)"): header.index("int lob_set_option(")]
    assert keys and keys == set(re.findall(r'"([a-z_]+)"', doc)), (keys, doc)
