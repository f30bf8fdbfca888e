"""Every function and class of the CPU oracle says which passage it follows (CPU): its
docstring names a section, equation, figure or observation of the paper, or says that it
is the workload model, a test helper or not in the paper (the learned proposal)."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("Eq", "Sec.", "Fig.", "obs.", "not in the paper", "module docstring", "test helper", "published")


def test_every_oracle_function_cites_a_passage():
    d = os.path.join(ROOT, "oracle")
    missing, n = [], 0
    for fn in sorted(os.listdir(d)):
        if not fn.endswith(".py") or fn == "__init__.py":
            continue
        tree = ast.parse(open(os.path.join(d, fn)).read())
        assert any(k in (ast.get_docstring(tree) or "") for k in KEYS), fn
        for node in tree.body:
            if isinstance(node, (ast.FunctionDef, ast.ClassDef)):
                n += 1
                doc = ast.get_docstring(node) or ""
                if not any(k in doc for k in KEYS):
                    missing.append("%s:%s" % (fn, node.name))
    assert n >= 50
    assert not missing, missing


def test_every_header_entry_point_cites_a_passage():
    """Each gbe_* prototype in include/*.h sits under a comment that names the passage of the
    paper it follows, or says that it has no counterpart there."""
    import re
    keys = KEYS + ("no counterpart", "paper")
    bad, n = [], 0
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        lines = open(os.path.join(ROOT, "include", fn)).read().split("\n")
        for i, line in enumerate(lines):
            m = re.match(r"^\s*(?:const\s+)?\w+\*?\s+\*?(gbe_\w+)\s*\(", line)
            if not m:
                continue
            n += 1
            j = i - 1          # up to the nearest comment, across the prototypes of its group
            while j >= 0 and not lines[j].strip().endswith("*/") and lines[j].strip():
                j -= 1
            block = []
            if j >= 0 and lines[j].strip().endswith("*/"):
                k = j
                while k >= 0 and "/*" not in lines[k]:
                    k -= 1
                block = lines[k:j + 1]
            if not any(key in " ".join(block) for key in keys):
                bad.append(m.group(1))
    assert n >= 40
    assert not bad, bad


def test_golden_values_carry_their_citation():
    """Each stored value of tests/golden/ is the paper's, with the passage it comes from in
    the comment lines right above it (no value there comes from the CUDA path)."""
    gdir = os.path.join(ROOT, "tests", "golden")
    n = 0
    for fn in sorted(os.listdir(gdir)):
        comment, after_value = "", False   # a comment block covers the values that follow it
        for line in open(os.path.join(gdir, fn)):
            line = line.strip()
            if line.startswith("#"):
                comment = (line if after_value else comment + " " + line)
                after_value = False
                continue
            if not line:
                continue
            name, *vals = line.split()
            assert vals and all(float(v) == float(v) for v in vals), (fn, line)
            assert any(k in comment for k in ("Sec.", "Eq", "Fig.", "Table")), (fn, name)
            n += 1
            after_value = True
    assert n >= 3
