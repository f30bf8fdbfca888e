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


def test_create_without_gpu_fails_loudly(lib):
    import torch
    import paper_1603_00937_gb300 as gbe
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(gbe.GbeError) as e:
        gbe.Context(0)
    assert e.value.code == gbe.GBE_ENODEV
