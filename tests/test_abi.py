"""The C-ABI library builds, loads without a GPU and exports every function
that include/rwpc.h declares (no compute calls here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rwpc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"typedef[^;]*;", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(n for n in names if not n.startswith("RW")))


@pytest.fixture(scope="module")
def lib_path():
    from paper_math_0609672_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rw_build_factor", "pcg_solve", "rw_context_create", "rw_factor_view"):
        assert required in names


def test_library_exports_every_declared_function(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_without_gpu(lib_path):
    import paper_math_0609672_gb300 as P
    lib = P.load()
    assert P.rw_status_string(-2).startswith("matrix is not")
    o = P.rw_options_default()
    assert o.max_steps == 1 << 24 and o.store_fp32 == 1 and o.refine_every == 50


def test_product_path_has_no_cpu_fallback():
    # the package must not import the oracle anywhere
    pkg = os.path.join(ROOT, "paper_math_0609672_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "rw_oracle" not in txt, f


def test_sha256_matches_hashlib():
    """The factor-file digest (host code of the library) against hashlib on
    the FIPS 180-4 example and random buffers spanning the padding cases."""
    import hashlib
    import numpy as np
    import paper_math_0609672_gb300 as P
    P.load()
    assert P.rw_sha256(b"abc") == hashlib.sha256(b"abc").digest()
    rng = np.random.default_rng(0)
    for size in (0, 1, 55, 56, 63, 64, 65, 119, 120, 1000, 100000):
        data = rng.integers(0, 256, size, dtype=np.uint8).tobytes()
        assert P.rw_sha256(data) == hashlib.sha256(data).digest(), size


def documented_option_defaults():
    """(field, default) for every rw_options field whose comment in
    include/rwpc.h states its default."""
    src = open(os.path.join(ROOT, "include", "rwpc.h")).read()
    body = src[src.index("typedef struct {\n    uint64_t max_steps;"):src.index("} rw_options;")]
    fields = re.split(r"\n(?=    (?:int32_t|uint64_t) )", body)
    out = {}
    for f in fields:
        m = re.match(r"\s*(?:int32_t|uint64_t)\s+(\w+);(.*)", f, flags=re.S)
        if not m:
            continue
        name, comment = m.group(1), " ".join(m.group(2).split())
        d = re.search(r"default (-?\d+)(?: << (\d+))?", comment)
        if d:
            out[name] = int(d.group(1)) << int(d.group(2) or 0)
            continue
        d = re.search(r"(-?\d+) = [^()]*\(default\)", comment)
        if d:
            out[name] = int(d.group(1))
    return out


def test_option_defaults_match_the_header(lib_path):
    import paper_math_0609672_gb300 as P
    P.load()
    doc = documented_option_defaults()
    assert len(doc) >= 15, sorted(doc)
    o = P.rw_options_default()
    got = {k: getattr(o, k) for k in doc}
    assert got == doc


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the C struct's size and each
    field's offset (a C program built from include/rwpc.h prints them)."""
    import ctypes
    import shutil
    import paper_math_0609672_gb300 as P
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [("rw_csr", P.rw_csr_t), ("rw_options", P.rw_options_t), ("rw_factor_desc", P.rw_factor_desc_t),
             ("rw_pcg_stats", P.rw_pcg_stats_t)]
    lines = ['#include <stdio.h>', '#include "rwpc.h"', "int main(void) {"]
    for cname, py in pairs:
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'    printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    for cname, py in pairs:
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])
