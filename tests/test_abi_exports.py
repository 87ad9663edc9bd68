"""The C-ABI library builds, loads and exports every function include/*.h
declares; the binding declares the same names (no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(ht_\w+)\s*\(", txt, flags=re.M)
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1505_00383_gb300 import _build
    return _build.build()


def test_headers_declare_entry_points():
    names = _declared()
    for n in ("ht_create_system", "ht_destroy_system", "ht_eval_diff", "ht_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (ht_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_matches_header(libpath):
    from paper_1505_00383_gb300 import ht
    declared = set(_declared())
    assert set(ht.SIGNATURES) <= declared
    public = {n for n in declared if not n.startswith("ht_bench_")}
    assert public <= set(ht.SIGNATURES), public - set(ht.SIGNATURES)
    L = ht.lib()  # loads without a GPU
    for n in declared:
        assert hasattr(L, n)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1505_00383_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "ht_oracle" not in txt, f


def test_binding_constants_equal_the_header():
    """The binding's copies of the header's size constants (the no-alloc
    scratch limit, the network's shape) cannot drift from include/ht.h."""
    from paper_1505_00383_gb300 import ht
    txt = open(os.path.join(ROOT, "include", "ht.h")).read()
    defs = dict(re.findall(r"^#define\s+(HT_\w+)\s+(.+?)\s*$", txt, flags=re.M))
    for name in ("HT_NOALLOC_MAX_PATHS", "HT_MLP_IN", "HT_MLP_OUT", "HT_MLP_NPARAM"):
        expr = defs[name]
        assert re.fullmatch(r"[0-9()<\s]+", expr), expr
        assert getattr(ht, name) == eval(expr), name
