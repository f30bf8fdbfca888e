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
