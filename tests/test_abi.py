"""The C-ABI library builds, loads and exports every function include/mgcccs.h declares
(no compute calls: this runs without a GPU)."""
import ctypes

import pytest

from paper_1412_1953_gb300 import build, mgcccs


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    names = mgcccs.header_functions()
    assert "mgcccs_setup" in names and "mgcccs_solve" in names
    L = ctypes.CDLL(libpath)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(names) == set(mgcccs._SIGS)


def test_host_only_entry_points(libpath):
    p = mgcccs.make_params(128, 128, 30.0, 30.0, 20.0, 20.0, 0.5, 0.5, levels=5, n_b=3)
    n = mgcccs.mgcccs_workspace_size(p)
    assert n > 16 * 127 * 127 * 4
    bad = mgcccs.make_params(100, 100, 30.0, 30.0, 20.0, 20.0, 0.5, 0.5, levels=5)   # 100 not divisible by 16
    assert mgcccs.mgcccs_workspace_size(bad) == 0
    # a coarsest grid beyond 1024 nodes takes block cyclic reduction: rows of at most 64 nodes
    rows63 = mgcccs.make_params(128, 128, 30.0, 30.0, 20.0, 20.0, 0.5, 0.5, levels=2)      # 63 x 63
    assert 16 * 13 * 63 ** 3 < mgcccs.mgcccs_workspace_size(rows63) < 16 * 63 ** 4   # factors, not an inverse
    too_coarse = mgcccs.make_params(256, 128, 30.0, 30.0, 20.0, 20.0, 0.5, 0.5, levels=2)  # 127 x 63
    assert mgcccs.mgcccs_workspace_size(too_coarse) == 0
    assert mgcccs.mgcccs_strerror(mgcccs.ENOTCONV).startswith("max_iter")
    assert mgcccs.lib().mgcccs_setup(None, None, None, None, None, None, 0, None) == mgcccs.EINVAL
