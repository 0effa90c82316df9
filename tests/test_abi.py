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


def test_autotune_space_is_table_4():
    """The default preconditioner space (host only, no GPU call): Sec. 5, Table 5 without
    SEMFEM for p = 7 and p = 9, and the same rule for other orders."""
    from paper_2110_07663_gb300 import se
    want = {
        7: [(se.SE_SMOOTH_ASM, [7, 3, 1]), (se.SE_SMOOTH_RAS, [7, 3, 1]),
            (se.SE_SMOOTH_JACOBI, [7, 5, 3, 1])],
        9: [(se.SE_SMOOTH_ASM, [9, 5, 1]), (se.SE_SMOOTH_RAS, [9, 5, 1]),
            (se.SE_SMOOTH_JACOBI, [9, 7, 5, 1])],
        3: [(se.SE_SMOOTH_ASM, [3, 1]), (se.SE_SMOOTH_RAS, [3, 1]),
            (se.SE_SMOOTH_JACOBI, [3, 1])],
        5: [(se.SE_SMOOTH_ASM, [5, 3, 1]), (se.SE_SMOOTH_RAS, [5, 3, 1]),
            (se.SE_SMOOTH_JACOBI, [5, 3, 1])],
    }
    for p, rows in want.items():
        got = se.se_pmg_autotune_space(p, se.SE_FP32)
        assert [(c.pmg.smoother, list(c.pmg.schedule[:c.pmg.nlev])) for c in got] == rows, p
        for c in got:
            assert c.pmg.precision == se.SE_FP32
            assert list(c.pmg.cheb_order[:c.pmg.nlev]) == [2] * c.pmg.nlev
            assert (c.pmg.eig_lo, c.pmg.eig_hi, c.pmg.arnoldi_steps) == (0.1, 1.1, 10)
    import pytest
    with pytest.raises(se.SeError):
        se.se_pmg_autotune_space(1, se.SE_FP64)
