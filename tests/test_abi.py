"""The C-ABI library builds, loads and exports every function include/esg.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

import paper_2504_04018_gb300 as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "esg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(esg_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["esg_build", "esg_search_batch", "esg_bruteforce_filtered_knn",
                     "esg_decompose_batch", "esg_index_import", "esg_free"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = E.load_library()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(E.EXPORTED) <= set(_declared())


def test_defaults_and_status_strings():
    lib = E.load_library()
    b = lib.esg_build_params_default()
    assert (b.M, b.leaf_size, b.n_entries) == (16, 256, 16)
    s = lib.esg_search_params_default()
    assert s.ef == 64 and s.use_learned == 0
    assert (s.post_root, s.max_registers) == (0, 0)
    t = lib.esg_train_params_default()
    # the last fields: a mismatch of layout between header and binding would garble them
    assert (t.ef_lo, t.ef_hi, t.per_k_class, t.seed) == (8, 128, 0, 4005)
    assert lib.esg_status_str(0) == b"ok"
    assert lib.esg_status_str(7) == b"unsupported"


def test_invalid_arguments_rejected_on_host():
    lib = E.load_library()
    h = ctypes.c_void_p()
    assert lib.esg_build(None, 10, 16, None, None, ctypes.byref(h)) == 1
    assert b"esg_build" in lib.esg_last_error()
    # d not a multiple of 8
    import numpy as np
    v = np.zeros((4, 12), np.float32)
    assert lib.esg_build(v.ctypes.data_as(ctypes.c_void_p), 4, 12, None, None, ctypes.byref(h)) == 1
    assert lib.esg_decompose_batch(0, 16, 0, 2, 0, None, None, 1, None, None, None) == 1
    assert lib.esg_decompose_batch(100, 16, 0, 17, 0, None, None, 0, None, None, None) == 1   # fanout > 16
    assert lib.esg_decompose_batch(100, 16, 2, 2, 0, None, None, 0, None, None, None) == 1    # no such layout
    # build parameters: fanout outside 2..16, unknown layout
    v16 = np.zeros((40, 16), np.float32)
    p = lib.esg_build_params_default()
    assert p.fanout == 2 and p.layout == 0
    p.fanout = 17
    assert lib.esg_build(v16.ctypes.data_as(ctypes.c_void_p), 40, 16, None, ctypes.byref(p), ctypes.byref(h)) == 1
    p.fanout, p.layout = 4, 3
    assert lib.esg_build(v16.ctypes.data_as(ctypes.c_void_p), 40, 16, None, ctypes.byref(p), ctypes.byref(h)) == 1
    assert lib.esg_search_batch(None, None, 1, None, None, None, 10, None, None, None, None, None,
                                None, None) == 1
    assert lib.esg_bruteforce_filtered_knn(None, 10, 16, 0, None, 1, None, None, 0, None, None,
                                           None, None) == 1


def test_load_missing_and_corrupt_files(tmp_path):
    lib = E.load_library()
    h = ctypes.c_void_p()
    assert lib.esg_load(str(tmp_path / "nope.esg").encode(), ctypes.byref(h)) == 4   # IO
    bad = tmp_path / "bad.esg"
    bad.write_bytes(b"\x00" * 64)
    assert lib.esg_load(str(bad).encode(), ctypes.byref(h)) == 5                     # CORRUPT


def test_binding_structs_follow_the_header():
    """The ctypes records of the binding list the header's struct fields in
    the header's order (names, and 32/64-bit widths)."""
    hdr = open(os.path.join(ROOT, "include", "esg.h")).read()
    for cname, pyname in (("esg_build_params", "_BuildParams"), ("esg_search_params", "_SearchParams"),
                          ("esg_train_params", "_TrainParams")):
        body = re.search(r"typedef struct \{([^}]*)\}\s*" + cname + r";", hdr).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            typ, names = decl.split(None, 1)
            for nm in names.split(","):
                fields.append((nm.strip(), 8 if typ in ("uint64_t", "int64_t", "double") else 4))
        py = getattr(E, pyname)._fields_
        assert [f for f, _ in py] == [f for f, _ in fields], cname
        assert [ctypes.sizeof(t) for _, t in py] == [w for _, w in fields], cname
