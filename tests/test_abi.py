"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function that include/rewl.h declares.  No compute call is made here."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(rewl_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1407_5140_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert {"rewl_create", "rewl_run", "rewl_exchange", "rewl_get_dos", "rewl_destroy"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_the_same_calls():
    from paper_1407_5140_gb300 import rewl
    src = open(rewl.__file__).read()
    for n in _declared():
        assert n in src, n
