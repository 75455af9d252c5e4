"""The C-ABI library loads and exports every symbol include/wskpn.h
declares; argument validation that needs no GPU.  CPU only."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2202_05977_b300 as wk
from paper_2202_05977_b300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(wskpn_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    # and the binding declares exactly the header's functions
    assert sorted(_lib.SIGNATURES) == names


def test_default_config_and_weight_count():
    c = wk.default_config()
    assert c.n_layers == 4 and list(c.widths[:5]) == [10, 32, 48, 64, 12]
    assert c.conv_ks == 5 and c.n_kernels == 6 and list(c.ksizes[:6]) == [3, 5, 7, 9, 11, 13]
    assert wk.n_weights(c) == 142556          # 25 * (10*32 + 32*48 + 48*64 + 64*12) + 156
    assert wk.n_weights(wk.default_config(conv_ks=3)) == 51420
    assert _lib.load().wskpn_version().startswith(b"wskpn")


@pytest.mark.parametrize("field,value", [("conv_ks", 4), ("n_kernels", 0), ("albedo_eps", 0.0),
                                         ("max_batch", 0), ("n_layers", 9)])
def test_invalid_config_is_rejected_without_touching_the_gpu(field, value):
    lib = _lib.load()
    c = wk.default_config()
    setattr(c, field, value)
    assert lib.wskpn_n_weights(ctypes.byref(c)) == 0
    h = ctypes.c_void_p()
    w = np.zeros(142556, np.float32)
    s = lib.wskpn_create(ctypes.byref(c), w.ctypes.data, w.size, ctypes.byref(h))
    assert s == _lib.EINVAL and not h.value
    assert lib.wskpn_last_error(None)


def test_even_kernel_size_rejected():
    lib = _lib.load()
    ks = (ctypes.c_int * 2)(3, 4)
    s = lib.wskpn_decode_fuse_fwd(ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), 1, 4, 4, 2,
                                  ks, 0.01, ctypes.c_void_p(16), None, None)
    assert s == _lib.EINVAL
    assert b"odd" in lib.wskpn_last_error(None)


def test_backward_scratch_size():
    # planes per frame: Lp_i and d_i of every size, then g_0, g_1, g_2
    lib = _lib.load()
    assert lib.wskpn_decode_fuse_bwd_scratch_floats(2, 3, 5, 6) == (2 * 6 + 3) * 2 * 3 * 5
    assert lib.wskpn_decode_fuse_bwd_scratch_floats(1, 1, 1, 1) == 5
    assert lib.wskpn_decode_fuse_bwd_scratch_floats(1, 4, 4, 0) == 0
    assert lib.wskpn_decode_fuse_bwd_scratch_floats(1, 4, 4, 9) == 0


def test_null_arguments_rejected():
    lib = _lib.load()
    assert lib.wskpn_denoise(None, None, 1, 4, 4, None, None) == _lib.EINVAL
    assert lib.wskpn_create(None, None, 0, None) == _lib.EINVAL
    lib.wskpn_destroy(None)


def test_temporal_arguments_rejected_without_touching_the_gpu():
    lib = _lib.load()
    out = ctypes.c_void_p()
    assert lib.wskpn_temporal_create(None, 0, 16, ctypes.byref(out)) == _lib.EINVAL
    cfg = _lib.TemporalConfig()
    lib.wskpn_temporal_config_default(ctypes.byref(cfg))
    assert (cfg.alpha_min, cfg.tau_normal) == (pytest.approx(0.2), pytest.approx(0.9))
    cfg.alpha_min = 0.0
    assert lib.wskpn_temporal_create(ctypes.byref(cfg), 8, 8, ctypes.byref(out)) == _lib.EINVAL
    assert b"alpha_min" in lib.wskpn_last_error(None)
    assert lib.wskpn_temporal_step(None, None, None, None, None, None, None) == _lib.EINVAL
    lib.wskpn_temporal_destroy(None)


def test_multires_arguments_rejected_without_touching_the_gpu():
    lib = _lib.load()
    out = ctypes.c_void_p()
    w = np.zeros(10, np.float32)
    assert lib.wskpn_mr_create(None, w.ctypes.data, w.size, ctypes.byref(out)) == _lib.EINVAL
    assert b"weights" in lib.wskpn_last_error(None)
    cfg = _lib.MrConfig()
    lib.wskpn_mr_config_default(ctypes.byref(cfg))
    assert (cfg.max_h, cfg.max_w) == (1080, 1920)
    cfg.max_h = 0
    assert lib.wskpn_mr_create(ctypes.byref(cfg), w.ctypes.data, w.size, ctypes.byref(out)) == _lib.EINVAL
    assert lib.wskpn_mr_n_weights() == 188_878
    lib.wskpn_mr_destroy(None)


def test_header_compiles_as_c(tmp_path):
    """include/wskpn.h is a plain C header: a C99 translation unit that
    includes it compiles without warnings (no C++ or CUDA types in the
    signatures)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = tmp_path / "use_header.c"
    src.write_text('#include "wskpn.h"\nint main(void) { return 0; }\n')
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I", inc, str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
