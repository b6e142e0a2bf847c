"""The C-ABI library builds, loads and exports every symbol include/ges.h declares (CPU only:
no compute calls)."""
import ctypes
import os
import re

import numpy as np
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


def test_training_struct_layouts_and_defaults(lib):
    from paper_2402_10128_gb300 import ges
    assert ctypes.sizeof(ges.ges_train_set) == 8 + 8 + 18 * 8
    assert ctypes.sizeof(ges.ges_scene_out) == 6 * 8
    assert ctypes.sizeof(ges.ges_adam_params) == 4 * 10
    assert ctypes.sizeof(ges.ges_density_params) == 4 * 6
    hp = ges.adam_params_default()   # App. B.2 (SH rest as in Gaussian splatting)
    assert list(np.float32(hp.lr)) == list(np.float32([1.6e-4, 0.005, 0.001, 0.001, 0.05, 0.0025]))
    assert np.float32(hp.lr_sh_rest) == np.float32(0.0025 / 20) and hp.beta1 == np.float32(0.9)
    assert hp.beta2 == np.float32(0.999) and hp.eps == np.float32(1e-15)
    dp = ges.density_params_default()
    assert dp.grad_threshold == np.float32(0.0003) and dp.percent_dense == np.float32(0.01)
    assert dp.min_opacity == np.float32(0.005)


def test_position_lr_matches_the_oracle_schedule(lib):
    """ges_position_lr is host-only; compared with the oracle's schedule (pinned by its closed forms)."""
    from oracle import train as ot
    from paper_2402_10128_gb300 import ges
    for step in (0, 1, 500, 7500, 15000, 29999, 30000, 45000):
        for delay in (0, 1000):
            got = ges.ges_position_lr(step, delay_steps=delay)
            assert got == pytest.approx(ot.position_lr(step, delay_steps=delay), rel=1e-6)
    with pytest.raises(ges.GesError):
        ges.ges_position_lr(10, max_steps=0)


def test_training_calls_validate_on_the_host(lib):
    """NULL and misaligned pointers are refused before any device work."""
    from paper_2402_10128_gb300 import ges
    lib = ges._lib   # the binding's handle, whose functions carry their argument types
    fake = ctypes.create_string_buffer(64)           # never dereferenced: validation fails first
    buf = ctypes.create_string_buffer(4096)
    base = (ctypes.addressof(buf) + 15) & ~15
    arrs = [base + 256 * k for k in range(6)]
    ts = ges.make_train_set(10, 0, arrs, arrs, [a + 4 for a in arrs])   # v misaligned
    ph = ges.make_scene_out(*arrs)
    gr = ges.ges_grads(*arrs)
    hp = ges.adam_params_default()
    st = lib.ges_adam_step(ctypes.addressof(fake), ctypes.byref(ts), ctypes.byref(gr), ctypes.byref(ph),
                           ctypes.byref(hp), 1, None)
    assert st == ges.GES_ERR_INVALID_ARG and "aligned" in ges.last_error()
    ts = ges.make_train_set(10, 0, arrs, arrs, arrs)
    st = lib.ges_adam_step(ctypes.addressof(fake), ctypes.byref(ts), ctypes.byref(gr), ctypes.byref(ph),
                           ctypes.byref(hp), 0, None)
    assert st == ges.GES_ERR_INVALID_ARG and "step" in ges.last_error()
    ts = ges.make_train_set(10, 4, arrs, arrs, arrs)
    st = lib.ges_activate(ctypes.addressof(fake), ctypes.byref(ts), ctypes.byref(ph), None)
    assert st == ges.GES_ERR_INVALID_ARG and "sh_degree" in ges.last_error()
    assert lib.ges_reset_opacity(ctypes.addressof(fake), ctypes.byref(ts), ctypes.c_float(1.5), None) == \
        ges.GES_ERR_INVALID_ARG
    dp = ges.density_params_default(scene_extent=0.0)
    n_out = ctypes.c_int64()
    ts = ges.make_train_set(10, 0, arrs, arrs, arrs)
    st = lib.ges_density_control(ctypes.addressof(fake), ctypes.byref(ts), arrs[0], arrs[0], arrs[0],
                                 ctypes.byref(dp), ctypes.byref(ts), ctypes.byref(n_out), None)
    assert st == ges.GES_ERR_INVALID_ARG


def test_fit1d_calls_validate_on_the_host(lib):
    """Out-of-range sizes and constants of the 1D fits are refused before any device work."""
    from paper_2402_10128_gb300 import ges
    lib = ges._lib   # the binding's handle, whose functions carry their argument types
    fake = ctypes.create_string_buffer(64)
    buf = ctypes.create_string_buffer(4096)
    a = ctypes.addressof(buf)
    p = ges.fit1d_params_default()
    assert p.model == ges.GES_MIX_GEF and p.n_components == 5 and p.epochs == 1000 and p.precision == 32
    assert p.lr == 0.01 and p.beta1 == 0.9 and p.beta2 == 0.999 and p.adam_eps == 1e-8 and p.nu == 4.0
    cases = [dict(n_components=0), dict(n_components=129), dict(model=7), dict(precision=16), dict(epochs=-1),
             dict(lr=0.0), dict(beta1=1.0), dict(nu=0.0)]
    for kw in cases:
        q = ges.fit1d_params_default(**kw)
        st = lib.ges_fit1d(ctypes.addressof(fake), ctypes.byref(q), 4, 100, a, a, 0, a, None, a, None, None)
        assert st == ges.GES_ERR_INVALID_ARG, kw
    st = lib.ges_fit1d(ctypes.addressof(fake), ctypes.byref(p), 4, 5000, a, a, 0, a, None, a, None, None)
    assert st == ges.GES_ERR_INVALID_ARG and "n_points" in ges.last_error()
    st = lib.ges_fit1d(ctypes.addressof(fake), ctypes.byref(p), 4, 100, a, a, 0, None, None, a, None, None)
    assert st == ges.GES_ERR_INVALID_ARG
    assert lib.ges_signal1d(ctypes.addressof(fake), 9, 1.0, 10, -1.0, 1.0, 32, a, a, None) == ges.GES_ERR_INVALID_ARG
    assert lib.ges_signal1d(ctypes.addressof(fake), 0, 0.0, 10, -1.0, 1.0, 32, a, a, None) == ges.GES_ERR_INVALID_ARG
    assert lib.ges_signal1d(ctypes.addressof(fake), 0, 1.0, 10, -1.0, 1.0, 8, a, a, None) == ges.GES_ERR_INVALID_ARG
