"""The C ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/apo.h declares (no compute calls are made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "apo.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\s*(?:apo_status|void|int|const char\*)\s+(apo_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2510_14982_gb300 import build
    return build.build()


def test_header_declares_the_documented_entry_points():
    names = _declared()
    for want in ("apo_problem_create", "apo_run", "apo_run_batch", "apo_step", "apo_histogram_u8"):
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_2510_14982_gb300 import apo
    assert sorted(apo.EXPORTS) == _declared()


def test_status_strings_without_gpu(libpath):
    from paper_2510_14982_gb300 import apo
    assert apo.apo_status_string(0) == "ok"
    assert "timed out" in apo.apo_status_string(apo.APO_ERR_TIMEOUT)


def test_argument_validation_without_gpu(libpath):
    """Rejected arguments return an error code before any device work."""
    from paper_2510_14982_gb300 import apo
    import numpy as np
    with pytest.raises(apo.ApoError) as e:
        apo.apo_problem_create(0, [], [], apo.APO_OBJ_SPHERE)
    assert e.value.status == apo.APO_ERR_INVALID_ARG
    with pytest.raises(apo.ApoError) as e:
        apo.apo_problem_create(3, np.zeros(3), np.zeros(3), apo.APO_OBJ_SPHERE)   # lb == ub
    assert e.value.status == apo.APO_ERR_INVALID_ARG
    with pytest.raises(apo.ApoError) as e:
        apo.apo_problem_create(4, -np.ones(4), np.ones(4), apo.APO_OBJ_HYBRID, perm=np.array([0, 0, 1, 2]))
    assert e.value.status == apo.APO_ERR_INVALID_ARG
    with pytest.raises(apo.ApoError) as e:
        apo.apo_problem_create(1025, -np.ones(1025), np.ones(1025), apo.APO_OBJ_SPHERE)
    assert e.value.status == apo.APO_ERR_UNSUPPORTED
