"""The C-ABI library builds, loads, and exports every symbol pndf.h declares.

No compute call is made here (no GPU needed): only argument validation paths
that return before touching the device.
"""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_08985_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(pndf_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pndf_build_hierarchy", "pndf_eval_batch", "pndf_diffuse_projected_area",
                     "pndf_free_hierarchy", "pndf_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_status_strings(lib):
    lib.pndf_status_string.restype = ctypes.c_char_p
    lib.pndf_status_string.argtypes = [ctypes.c_int]
    assert lib.pndf_status_string(0) == b"ok"
    assert lib.pndf_status_string(1) == b"invalid argument"
    assert lib.pndf_status_string(99) == b"unknown status"
    assert lib.pndf_version() >= 100


def test_argument_errors_without_device(lib):
    vp = ctypes.c_void_p
    lib.pndf_build_hierarchy.argtypes = [vp, vp, vp, ctypes.POINTER(vp)]
    out = vp(1234)
    assert lib.pndf_build_hierarchy(None, None, None, ctypes.byref(out)) == 1
    assert out.value is None  # cleared on error
    assert lib.pndf_build_hierarchy(None, None, None, None) == 1
    lib.pndf_eval_batch.argtypes = [vp, vp, ctypes.c_int64, vp, vp, vp, vp]
    assert lib.pndf_eval_batch(None, None, 0, None, None, None, None) == 1
    lib.pndf_diffuse_projected_area.argtypes = [vp, vp, vp, ctypes.c_int64, vp, vp]
    assert lib.pndf_diffuse_projected_area(None, None, None, 0, None, None) == 1
    lib.pndf_free_hierarchy.argtypes = [vp]
    lib.pndf_free_hierarchy(None)  # no-op
    lib.pndf_hierarchy_bytes.restype = ctypes.c_size_t
    lib.pndf_hierarchy_bytes.argtypes = [vp]
    assert lib.pndf_hierarchy_bytes(None) == 0


def test_build_params_invalid_n(lib):
    class P(ctypes.Structure):
        _fields_ = [("n", ctypes.c_int32), ("texel_fmt", ctypes.c_int32), ("bounds_fmt", ctypes.c_int32),
                    ("leaf_level", ctypes.c_int32), ("clusters", ctypes.c_int32)]

    vp = ctypes.c_void_p
    lib.pndf_build_hierarchy.argtypes = [vp, ctypes.POINTER(P), vp, ctypes.POINTER(vp)]
    out = vp()
    dummy = ctypes.c_void_p(256)  # never dereferenced: validation fails first
    for bad in (P(1, 0, 0, 0, 0), P(16385, 0, 0, 0, 0), P(64, 7, 0, 0, 0), P(64, 0, 9, 0, 0), P(64, 0, 0, 0, 2)):
        assert lib.pndf_build_hierarchy(dummy, ctypes.byref(bad), None, ctypes.byref(out)) == 1
    assert lib.pndf_build_hierarchy(dummy, ctypes.byref(P(64, 0, 0, 3, 0)), None, ctypes.byref(out)) == 6


def header_struct_fields(name):
    """(field name, C type) in declaration order of `typedef struct name {...}` in pndf.h."""
    src = open(os.path.join(ROOT, "include", "pndf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), src, flags=re.S).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        m = re.match(r"(.*?)([A-Za-z_]\w*)$", decl.replace("\n", " "))
        ctype, names = m.group(1).strip(), [m.group(2)]
        if "," in decl:  # float x, y, ...
            first = re.match(r"([A-Za-z_][\w ]*?)\s+([A-Za-z_]\w*)\s*,", decl)
            ctype = first.group(1)
            names = [n.strip() for n in decl[len(first.group(1)):].split(",")]
        fields += [(n, ctype) for n in names]
    return fields


@pytest.mark.parametrize("cname,pyname", [("pndf_build_params", "_BuildParams"), ("pndf_eval_config", "_EvalConfig"),
                                          ("pndf_segment", "_Segment"), ("pndf_server_config", "_ServerConfig")])
def test_binding_structs_match_header(lib, cname, pyname):
    """The binding's ctypes mirrors of the ABI structs have the header's fields,
    in order, with matching kinds (32-bit int, float, pointer)."""
    from paper_2505_08985_gb300 import pndf
    ours = getattr(pndf, pyname)._fields_
    theirs = header_struct_fields(cname)
    assert [n for n, _ in ours] == [n for n, _ in theirs], (cname, ours, theirs)
    for (n, t), (_, ct) in zip(ours, theirs):
        if "*" in ct:
            assert t is ctypes.c_void_p, (cname, n)
        elif ct == "float":
            assert t is ctypes.c_float, (cname, n)
        else:
            assert t is ctypes.c_int32, (cname, n, ct)


def test_query_record_layout():
    fields = header_struct_fields("pndf_query")
    assert [n for n, _ in fields] == ["x", "y", "sxx", "sxy", "syy", "ms", "mt", "pad"]
    assert all(t == "float" for _, t in fields)  # 32 bytes, the (nq, 8) float32 tensor of the binding


def test_binding_refuses_pageable_texels(lib):
    """Texels must be a CUDA tensor or page-locked: a plain CPU tensor is refused
    before the library is called."""
    import torch
    from paper_2505_08985_gb300 import pndf
    with pytest.raises(ValueError):
        pndf.pndf_build_hierarchy(torch.zeros(8, 8, 2))


def test_stats_names_match_header(lib):
    from paper_2505_08985_gb300 import pndf
    fields = header_struct_fields("pndf_query_stats")
    assert list(pndf.STATS_NAMES) == [n for n, _ in fields] and pndf.STATS_FIELDS == len(fields)
    assert all(t == "uint32_t" for _, t in fields)


def test_binding_refuses_short_or_misplaced_buffers():
    """The binding checks every buffer's size and device before the call: the
    C ABI takes bare pointers, so a short output would be written past its end.
    Shapes are checked before placement, so this runs without a GPU."""
    import torch

    from paper_2505_08985_gb300 import pndf

    need = pndf._need
    cuda0 = torch.device("cuda", 0)
    with pytest.raises(ValueError, match="4 elements"):
        need(torch.empty(3), "out", dtype=torch.float32, numel=4, on=cuda0)
    with pytest.raises(ValueError, match="4 elements"):
        need(torch.empty(5, dtype=torch.int32), "flags", dtype=torch.int32, numel=4, on=cuda0)
    with pytest.raises(ValueError, match="4 rows"):
        need(torch.empty(3, pndf.STATS_FIELDS, dtype=torch.int32), "stats", dtype=torch.int32,
             shape_last=pndf.STATS_FIELDS, rows=4, on=cuda0)
    with pytest.raises(ValueError, match="last dimension 3"):
        need(torch.empty(4, 2), "omega", dtype=torch.float32, shape_last=3, rows=4, on=cuda0)
    with pytest.raises(ValueError, match="float32"):
        need(torch.empty(4, dtype=torch.float64), "out", dtype=torch.float32, numel=4)
    with pytest.raises(ValueError, match="contiguous"):
        need(torch.empty(4, 2).t(), "out", dtype=torch.float32)
    # right shape, wrong place: a CPU tensor where a device buffer is expected
    with pytest.raises(ValueError, match="CUDA tensor"):
        need(torch.empty(4), "out", dtype=torch.float32, numel=4, on=cuda0)
    # the host variant refuses a short result buffer before copying anything
    q = torch.zeros(4, 8)
    with pytest.raises(ValueError, match="4 elements"):
        pndf.pndf_eval_batch_host(None, q, out_host=torch.empty(3))
