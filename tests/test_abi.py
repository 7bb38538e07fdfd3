"""CPU-only checks of the C ABI: the library builds/loads, exports every symbol declared in
include/tocab.h, and its host-only logic (default block width) follows the paper."""
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(tc_[a-z0-9_]+)\s*\(", txt):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1904_02241_gb300 import build
    build.build()
    import paper_1904_02241_gb300 as T
    return T.lib()


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert {"tc_graph_load_csr", "tc_tocab_partition", "tc_pagerank_pull", "tc_pagerank_push",
            "tc_bfs_pull"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_1904_02241_gb300 import _lib
    assert _declared_functions() <= set(_lib.SIGNATURES)


def test_status_strings(lib):
    assert lib.tc_status_string(0) == b"TC_OK"
    assert lib.tc_status_string(-2) == b"TC_ERR_INVALID_GRAPH"
    assert lib.tc_status_string(-6) == b"TC_ERR_UNSUPPORTED"


def test_default_block_width_is_paper_choice_on_paper_l2(lib):
    """2.75 MB L2 (Sec. 4) -> 256 Ki vertices per subgraph (Sec. 4.3), which reproduces
    every subgraph count of Table 3 within the rounding of the printed vertex counts."""
    l2 = int(2.75 * 1024 * 1024)
    W = lib.tc_default_block_width(1 << 30, l2, 0.0)
    assert W == 262144
    path = os.path.join(ROOT, "tests", "golden", "table3_subgraphs.txt")
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        name, vp, unit, cnt = line.split()
        lo, hi = float(vp) - float(unit) / 2, float(vp) + float(unit) / 2
        counts = {math.ceil(v / W) for v in (lo, float(vp), hi)}
        assert int(cnt) in set(range(min(counts), max(counts) + 1)), name


def test_default_block_width_scales_with_l2_and_clamps(lib):
    gb300_l2 = 135528448
    W = lib.tc_default_block_width(1 << 24, gb300_l2, 0.0)
    assert W == gb300_l2 // 11
    assert lib.tc_default_block_width(1000, gb300_l2, 0.0) == 1000     # never wider than V
    assert lib.tc_default_block_width(1 << 24, 4096, 0.0) == 372
    assert lib.tc_default_block_width(1 << 24, 64, 0.0) == 32                    # floor of 32
    assert lib.tc_default_block_width(1 << 26, gb300_l2, 0.5) == int(0.5 * gb300_l2 / 4)


def test_memory_cap_arguments(lib):
    """The cap is host state: a negative byte count is refused, 0 clears it (no device needed)."""
    assert lib.tc_set_device_memory_limit(-1) == -1
    assert lib.tc_set_device_memory_limit(0) == 0
    assert lib.tc_device_memory_held() >= 0


def _header_structs():
    """Field names of every `typedef struct X { ... } X;` in include/tocab.h, in order."""
    txt = open(os.path.join(ROOT, "include", "tocab.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for m in re.finditer(r"typedef struct (tc_[a-z_]+)\s*\{(.*?)\}\s*\1\s*;", txt, flags=re.S):
        fields = []
        for decl in m.group(2).split(";"):
            decl = decl.strip()
            if not decl:
                continue
            for part in decl.split(","):  # "int32_t a, b" declares two fields
                part = part.split("[")[0]  # "float x[N]": the name is before the bound
                fields.append(re.findall(r"[A-Za-z_][A-Za-z0-9_]*", part)[-1])
        out[m.group(1)] = fields
    return out


def test_ctypes_structs_mirror_the_header():
    """Every struct the binding passes by pointer has the header's fields in the header's order
    (a field missing or out of place would shift every later one)."""
    from paper_1904_02241_gb300 import _lib as L
    hdr = _header_structs()
    mirrored = [n for n in dir(L) if n.startswith("tc_") and isinstance(getattr(L, n), type)
                and issubclass(getattr(L, n), L.C.Structure)]
    assert {"tc_pr_params", "tc_part_params", "tc_bfs_params", "tc_multi_params"} <= set(mirrored)
    for name in mirrored:
        assert name in hdr, name
        assert [f[0] for f in getattr(L, name)._fields_] == hdr[name], name


def test_missing_library_fails_loudly():
    """Without the built library the binding raises: there is no CPU fallback to land on."""
    from paper_1904_02241_gb300 import _lib as L
    absent = os.path.join(ROOT, "paper_1904_02241_gb300", "no_such_dir", "libtocab.so")
    saved = L._lib
    L._lib = None
    try:
        with pytest.raises(ImportError, match="missing"):
            L.load(absent)
    finally:
        L._lib = saved
