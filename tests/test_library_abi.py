"""The C-ABI library builds, loads without a GPU and exports every entry point include/*.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    import glob
    src = "".join(open(h).read() for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(trals_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    import paper_2210_11362_gb300 as P
    if not os.path.exists(P.LIB_PATH):
        from paper_2210_11362_gb300 import build
        build.build()
    return P.LIB_PATH


def test_header_declares_entry_points():
    names = _declared()
    for must in ["trals_create", "trals_destroy", "trals_decompose", "trals_last_error", "trals_plan_create",
                 "trals_mttsp", "trals_gamma", "trals_coef_matrix", "trals_solve_chol"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_exports(libpath):
    import paper_2210_11362_gb300 as P
    for n in _declared():
        assert n in P.EXPORTED, n
        assert hasattr(P, n), n


def test_version_and_no_gpu_error(libpath):
    import paper_2210_11362_gb300 as P
    assert "sm_103a" in P.trals_version()
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        with pytest.raises(P.TralsError):
            P.trals_create(0)
