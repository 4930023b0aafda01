"""The ctypes mirrors of the public structs have the C layout (no GPU): a C
program compiled against include/epic_interp.h prints every field's offset
and size and each struct's size, and the binding's structures must agree.
A field added, removed, reordered or retyped on one side fails here instead
of corrupting memory at the ABI."""

import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_1501_02565_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")
HEADER = os.path.join(INCLUDE, "epic_interp.h")

MIRRORS = {
    "epic_config_t": native.epic_config_t,
    "epic_pair_desc_t": native.epic_pair_desc_t,
    "epic_tile_rule_t": native.epic_tile_rule_t,
    "epic_refine_params_t": native.epic_refine_params_t,
}


def header_fields(struct_name):
    """Field names of `typedef struct { ... } struct_name;` in declaration order."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    m = re.search(r"typedef\s+struct\s*\{([^{}]*)\}\s*%s\s*;" % struct_name, text)
    assert m, struct_name
    names = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        # "const float *cost_map" / "int H, W, N, K" / "long long max_pixels"
        first, *rest = [p.strip() for p in decl.split(",")]
        names.append(re.findall(r"\w+", first)[-1])
        names += [re.findall(r"\w+", r)[-1] for r in rest]
    return names


def test_field_names_and_order_match_the_header():
    for name, cls in MIRRORS.items():
        assert [f[0] for f in cls._fields_] == header_fields(name), name


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "epic_interp.h"',
             "int main(void) {"]
    for name in MIRRORS:
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for f in header_fields(name):
            lines.append('printf("%s.%s %%zu %%zu\\n", offsetof(%s, %s), sizeof(((%s *)0)->%s));'
                         % (name, f, name, f, name, f))
    lines += ["return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c99", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        key, *vals = line.split()
        layout[key] = tuple(int(v) for v in vals if v.isdigit())
    return layout


def test_offsets_sizes_and_struct_sizes_match_c(c_layout):
    for name, cls in MIRRORS.items():
        assert ctypes.sizeof(cls) == c_layout[f"{name}"][0], name
        for fname, ftype in cls._fields_:
            off, size = c_layout[f"{name}.{fname}"]
            assert getattr(cls, fname).offset == off, (name, fname)
            assert ctypes.sizeof(ftype) == size, (name, fname)
