"""The C ABI library builds, loads without a GPU and exports every function include/kep.h declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "kep.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kep_[a-z_]+)\s*\(", src)))


def test_header_declares_binding_list():
    import paper_1710_05134_gb300.kep as k
    assert _declared() == sorted(k.EXPORTED)


def test_library_loads_and_exports_all_symbols():
    import paper_1710_05134_gb300 as k
    L = k.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert k.status_str(k.KEP_ERR_SINGULAR).startswith("exact zero pivot")


def test_invalid_arguments_rejected_without_gpu():
    """Pattern validation happens on the host before any device call."""
    import numpy as np
    import paper_1710_05134_gb300 as k
    with pytest.raises(k.KepError) as e:
        k.Problem(2, np.array([0, 1, 2]), np.array([0, 5]), np.ones(2), np.ones(2))
    assert e.value.code == 1
    with pytest.raises(k.KepError):       # duplicate column in a row
        k.Problem(2, np.array([0, 2, 3]), np.array([0, 0, 1]), np.ones(3), np.ones(3))
    with pytest.raises(k.KepError):       # lower pattern with an upper entry
        k.Problem(2, np.array([0, 2, 3]), np.array([0, 1, 1]), np.ones(3), np.ones(3), lower=True)
