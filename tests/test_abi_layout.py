"""The ctypes mirrors of the C ABI's structs (paper_1712_09407_gb300/tracker.py) against the
declarations in include/tpcca.h: same fields in the same order, each with the size its C type
has, and the same total size.  A mismatch would shift every later field of a struct passed
across the boundary."""
import ctypes
import os
import re

import pytest

from paper_1712_09407_gb300 import tracker

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "tpcca.h")

C_SIZES = {"float": 4, "double": 8, "int": 4, "int32_t": 4, "uint32_t": 4, "int64_t": 8, "uint64_t": 8,
           "size_t": 8, "uint8_t": 1}


def _header_structs():
    """{name: [(field, bytes), ...]} for every `typedef struct { ... } name;` in the header."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    out = {}
    for body, name in re.findall(r"typedef\s+struct\s*\{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"((?:const\s+)?\w+)\s+(.*)$", decl)
            ctype, rest = m.group(1).replace("const ", ""), m.group(2)
            for item in rest.split(","):
                item = item.strip()
                ptr = item.startswith("*")
                item = item.lstrip("*").strip()
                am = re.match(r"(\w+)(?:\[(\d+)\])?$", item)
                fname, count = am.group(1), int(am.group(2) or 1)
                size = 8 if ptr else C_SIZES[ctype]
                fields.append((fname, size * count))
        out[name] = fields
    return out


STRUCTS = ["tpc_geometry", "tpc_params", "tpc_tuning", "tpc_track_view", "tpc_debug_view", "tpc_call_stats",
           "tpc_server_config", "tpc_server_result"]


def test_every_header_struct_has_a_mirror():
    assert set(_header_structs()) == set(STRUCTS)


@pytest.mark.parametrize("name", STRUCTS)
def test_struct_mirror_matches_header(name):
    c_fields = _header_structs()[name]
    py = getattr(tracker, name)
    py_fields = [(f[0], ctypes.sizeof(f[1])) for f in py._fields_]
    assert [f for f, _ in py_fields] == [f for f, _ in c_fields], name
    assert py_fields == c_fields, name
    # same total size: the C compiler pads like ctypes does for these plain layouts
    offset, align = 0, 1
    for (_, size), (_, t) in zip(c_fields, py._fields_):
        a = ctypes.alignment(t)
        offset = (offset + a - 1) // a * a + size
        align = max(align, a)
    assert ctypes.sizeof(py) == (offset + align - 1) // align * align
