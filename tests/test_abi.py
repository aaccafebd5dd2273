"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/sgn.h declares.

No compute call is made here (no GPU is needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sgn.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(sgn_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_16045_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sgn_apply_operator", "sgn_precond_solve", "sgn_pcg", "sgn_step_rk4",
                 "sgn_step_abk", "sgn_step_linimp", "sgn_precond_coeffs", "sgn_rhs",
                 "sgn_spectral_grad", "sgn_gmres", "sgn_step_rk4_nc", "sgn_state_set_dealias",
                 "sgn_state_set_forcing", "sgn_layout_set_forms", "sgn_state_autotune",
                 "sgn_server_create", "sgn_batch_submit", "sgn_batch_poll",
                 "sgn_pcg1d_noalloc", "sgn_pcg_async"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_the_header(lib):
    from paper_2506_16045_gb300 import sgn
    bound = {s[0] for s in sgn.SIGNATURES}
    assert set(declared_functions()) <= bound | {"sgn_batch_submit", "sgn_batch_poll",
                                                 "sgn_result_release"}


def test_status_strings_without_gpu(lib):
    from paper_2506_16045_gb300 import sgn
    L = sgn.load()
    assert L.sgn_status_string(0) == b"ok"
    assert L.sgn_status_string(7) == b"non-positive depth"
