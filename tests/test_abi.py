"""The C-ABI library loads, exports every symbol include/pd.h declares, and
rejects bad inputs before touching the GPU (no compute calls here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2405_12484_gb300 import build, _lib
    build.build()
    return _lib.load()


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", hdr)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"\b(pd_[a-z_0-9]+)\s*\(", txt)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "pd_step" in names and "pd_prefactor" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2405_12484_gb300 import _lib
    bound = {n for n, _, _ in _lib.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_status_strings(lib):
    assert lib.pd_status_string(0) == b"ok"
    assert lib.pd_status_string(-5).startswith(b"matrix not positive")
    assert lib.pd_phase_name(1) == b"local"


def _create(lib, rest, tets, **kw):
    h = C.c_void_p()
    rest = np.ascontiguousarray(rest, np.float64)
    tets = np.ascontiguousarray(tets, np.int32)
    n_dom = kw.get("n_domains", 1)
    st = lib.pd_create_mesh(rest.ctypes.data, rest.shape[0], tets.ctypes.data, tets.shape[0], None, 300.0, None,
                            n_dom, None, None, C.byref(h))
    return st, h


def test_bad_inputs_are_rejected_before_any_cuda_call(lib):
    from paper_2405_12484_gb300 import _lib
    rest = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    st, h = _create(lib, rest, [[0, 1, 2, 4]])
    assert st == _lib.PD_ERR_BAD_MESH and not h.value
    st, h = _create(lib, rest, [[0, 1, 1, 2]])
    assert st == _lib.PD_ERR_BAD_MESH
    flat = rest.copy()
    flat[3] = [1, 1, 0]
    st, h = _create(lib, flat, [[0, 1, 2, 3]])
    assert st == _lib.PD_ERR_BAD_MESH
    st, h = _create(lib, rest, [[0, 1, 2, 3]], n_domains=0)
    assert st == _lib.PD_ERR_INVALID_ARG
    assert b"range" in lib.pd_last_error() or len(lib.pd_last_error()) > 0
    # null outputs and handles
    assert lib.pd_step(None, None, None, 1, None) == _lib.PD_ERR_INVALID_ARG
    assert lib.pd_prefactor(None, 0.01, None) == _lib.PD_ERR_INVALID_ARG
    assert lib.pd_sync(None) == _lib.PD_ERR_INVALID_ARG


def test_fitting_entry_points_reject_bad_arguments_before_any_cuda_call(lib):
    from paper_2405_12484_gb300 import _lib
    E = _lib.PD_ERR_INVALID_ARG
    # null mesh / workspace
    assert lib.pd_pose_misfit(None, None, None, None, None) == E
    assert lib.pd_gn_product(None, None, None, None, None, 2.0, None) == E
    assert lib.pd_gn_direction(None, None, None, None, None, 1e-2, 2.0, 10, None, None) == E
    opts = _lib.pd_fit_opts(1, 1, 0.01, 1.0, 1e-2, 1e-3, 12, 8, 30, 4, 20, 1.0 / 150, None)
    rep = _lib.pd_fit_report()
    assert lib.pd_fit_pose(None, None, C.byref(opts), None, None, None, None, None, None, None, C.byref(rep)) == E
    assert lib.pd_fit_pose_reduced(None, None, C.byref(opts), None, 1, None, None, None, None, None, None, None,
                                   C.byref(rep)) == E
    assert lib.pd_harmonic_basis(None, 4, None, None, None) == E
    assert lib.pd_test_inflate_copy(None, 16) == E
    assert lib.pd_server_run(None, 10, None) == E
    assert len(lib.pd_last_error()) > 0
