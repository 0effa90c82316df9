"""The C-ABI library builds for sm_103a, loads, and exports every entry point that include/*.h
declares (no GPU needed: symbols are looked up, nothing is called)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(se_[a-z0-9_]+)\s*\(",
                            src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    path = __graft_entry__._load_builder().build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2110_07663_gb300 import se
    assert set(names) <= set(se.EXPORTED), set(names) - set(se.EXPORTED)
