"""CPU checks of the C ABI: the library builds, loads, and exports every declared entry point."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1603_00937_gb300 import build
    build.build()
    import paper_1603_00937_gb300 as gbe
    return gbe.load_library()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(gbe_\w+)\s*\(", text, re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    import paper_1603_00937_gb300 as gbe
    decl = declared_symbols()
    assert len(decl) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", gbe.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(gbe_\w+)\b", out))
    assert decl <= exported, decl - exported
    assert set(gbe.EXPORTS) <= decl
    for name in decl:
        getattr(lib, name)


def test_strerror_names_codes(lib):
    import paper_1603_00937_gb300 as gbe
    assert lib.gbe_strerror(gbe.GBE_ETIMEOUT).decode() == "device wait timed out"
    assert lib.gbe_strerror(0).decode() == "ok"
    # every code the header defines has its own name, and the binding's constants agree
    with open(os.path.join(ROOT, "include", "gbe.h")) as f:
        codes = dict(re.findall(r"#define\s+(GBE_(?:OK|E[A-Z]+))\s+(-?\d+)", f.read()))
    assert len(codes) >= 9
    names = set()
    for name, val in codes.items():
        assert getattr(gbe, name) == int(val), name
        msg = lib.gbe_strerror(int(val)).decode()
        assert msg != "unknown error", name
        names.add(msg)
    assert len(names) == len(codes)
    assert lib.gbe_strerror(-99).decode() == "unknown error"


def test_create_without_gpu_fails_loudly(lib):
    import torch
    import paper_1603_00937_gb300 as gbe
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(gbe.GbeError) as e:
        gbe.Context(0)
    assert e.value.code == gbe.GBE_ENODEV


def declared_prototypes():
    """name -> (return type, [argument types]) of every gbe_* prototype in include/*.h."""
    protos = {}
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        for m in re.finditer(r"^\s*((?:const\s+)?\w+\s*\*?)\s*(gbe_\w+)\s*\(([^)]*)\)\s*;", text, re.M):
            args = [a.strip() for a in m.group(3).split(",") if a.strip() and a.strip() != "void"]
            protos[m.group(2)] = (m.group(1).strip(), args)
    return protos


def _ctype_of(decl):
    """The ctypes type a C parameter or return type needs (pointer, int32, int64, double, float)."""
    import ctypes
    if "*" in decl:
        return ctypes.c_char_p if re.match(r"^const\s+char\s*\*", decl) else ctypes.c_void_p
    t = decl.replace("const", "").split()[0]
    return {"int": ctypes.c_int, "int32_t": ctypes.c_int, "int64_t": ctypes.c_int64, "double": ctypes.c_double,
            "float": ctypes.c_float, "uint8_t": ctypes.c_ubyte}[t]


def test_binding_signatures_match_header(lib):
    """Every ctypes signature the binding installs has the header's argument count and types:
    a mismatch (an int64_t passed as int, a float as double) corrupts arguments silently."""
    import ctypes
    protos = declared_prototypes()
    checked = 0
    for name, (ret, args) in protos.items():
        f = getattr(lib, name)
        if f.argtypes is None:
            continue
        want = [_ctype_of(a) for a in args]
        got = list(f.argtypes)
        assert len(got) == len(want), (name, got, want)
        for g, w in zip(got, want):
            if w is ctypes.c_char_p:
                assert g in (ctypes.c_char_p, ctypes.c_void_p), (name, g, w)
            else:
                assert g is w, (name, args, got)
        if ret != "void":
            assert f.restype is _ctype_of(ret) or (_ctype_of(ret) is ctypes.c_char_p and f.restype is ctypes.c_char_p), \
                (name, ret, f.restype)
        checked += 1
    assert checked >= 40, checked


STRUCTS = {"Csr": "gbe_csr", "Ell": "gbe_ell", "Sites": "gbe_sites", "TbModel": "gbe_tb_model",
           "GraphParams": "gbe_graph_params", "PartitionParams": "gbe_partition_params",
           "Sp2Params": "gbe_sp2_params", "Sp2Report": "gbe_sp2_report", "FoeParams": "gbe_foe_params",
           "FoeReport": "gbe_foe_report", "TcConfig": "gbe_tc_config", "TuneReport": "gbe_tune_report"}


def test_binding_structs_match_header(tmp_path):
    """Every struct the binding passes by pointer has the header's size and field offsets
    (a smaller ctypes struct would be overrun by the library's writes)."""
    import ctypes
    import shutil
    import paper_1603_00937_gb300 as gbe
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "gbe.h"', "int main(void) {"]
    for py, c in STRUCTS.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (py, c))
        for f in getattr(gbe, py)._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (py, f[0], c, f[0]))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.rsplit(" ", 1) for line in out if line)
    for py in STRUCTS:
        S = getattr(gbe, py)
        assert int(got["%s size" % py]) == ctypes.sizeof(S), py
        for f in S._fields_:
            assert int(got["%s.%s" % (py, f[0])]) == getattr(S, f[0]).offset, (py, f[0])


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_1603_00937_gb300 as gbe
    monkeypatch.setattr(gbe, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        gbe.load_library(str(tmp_path / "libgbe.so"))


def test_product_path_never_touches_the_oracle():
    """The package neither imports nor names the CPU oracle: importing it loads no oracle
    module, and no source file of the package or the C headers refers to it."""
    import sys
    code = ("import sys; import paper_1603_00937_gb300 as g; g.load_library(); "
            "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]; "
            "assert not bad, bad")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    pkg = os.path.join(ROOT, "paper_1603_00937_gb300")
    files = [os.path.join(d, f) for d, _, fs in os.walk(pkg) if "_build" not in d and "__pycache__" not in d
             for f in fs if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp"))]
    files += [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))]
    assert len(files) >= 10
    for fn in files:
        text = open(fn).read()
        assert not re.search(r"^\s*(from|import)\s+oracle\b", text, re.M), fn
        assert "oracle/" not in text and '"oracle"' not in text, fn


def test_oracle_and_inputs_never_touch_the_package():
    """The converse: the oracle and the shared seeded-input module import neither the
    package nor its library, and the input module imports nothing of the oracle."""
    for sub in ("oracle", "synth"):
        d = os.path.join(ROOT, sub)
        for fn in os.listdir(d):
            if not fn.endswith(".py"):
                continue
            text = open(os.path.join(d, fn)).read()
            assert "paper_1603_00937_gb300" not in text and "libgbe" not in text and "ctypes" not in text, fn
            if sub == "synth":
                assert not re.search(r"^\s*(from|import)\s+(oracle|\.)", text, re.M), fn


def test_docstring_example_uses_the_binding():
    """The package docstring's usage example parses and every gbe.* name it uses exists in
    the binding (it runs only on a GPU; its calls are the ones the full-size parity test
    makes)."""
    import ast
    import textwrap
    import paper_1603_00937_gb300 as gbe
    doc = gbe.__doc__
    start = doc.index("::\n") + 3
    block = textwrap.dedent(doc[start:])
    names = set()
    for node in ast.walk(ast.parse(block)):
        if isinstance(node, ast.Attribute) and isinstance(node.value, ast.Name) and node.value.id == "gbe":
            names.add(node.attr)
    assert {"Context", "build_graph", "partition", "sp2_submatrices", "assemble_D"} <= names
    missing = sorted(n for n in names if not hasattr(gbe, n))
    assert not missing, missing
