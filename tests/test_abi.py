"""The C-ABI library builds, loads and exports every entry point include/coded_qr.h declares
(CPU only: no compute call is made)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2311_11943_gb300 import build
    return build.build()


def _declared():
    with open(os.path.join(ROOT, "include", "coded_qr.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"\b(coded_qr_\w+)\s*\(", text)))


def test_header_declares_the_hot_path():
    names = _declared()
    for verb in ("create", "destroy", "encode", "factor", "inject_erasure", "recover",
                 "post_orth", "solve", "run", "get_generator", "get_decode_sets",
                 "sync_status", "errstr"):
        assert "coded_qr_" + verb in names


def test_library_exports_every_declared_symbol(libpath):
    lib = C.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert missing == []


def test_binding_names_match_header(libpath):
    from paper_2311_11943_gb300 import binding
    assert sorted(binding.EXPORTS) == _declared()
    binding.lib()


def test_config_struct_layout(libpath):
    from paper_2311_11943_gb300 import binding
    assert C.sizeof(binding.Config) == 88
    assert binding.Config.panel.offset == 56 and binding.Config.in_node.offset == 60
    assert binding.Config.seed.offset == 64 and binding.Config.stream.offset == 80


def test_errstr_and_argument_validation_without_gpu(libpath):
    from paper_2311_11943_gb300 import binding as B
    assert B.errstr(B.CQR_EUNRECOVERABLE) == "erasure pattern not recoverable"
    cfg = B.Config()
    cfg.m, cfg.n, cfg.p_r, cfg.p_c, cfg.f, cfg.b = 64, 60, 4, 8, 1, 8   # p_c does not divide n
    n = C.c_size_t(0)
    assert B.lib().coded_qr_workspace_size(C.byref(cfg), C.byref(n)) == B.CQR_EINVAL
    cfg.n, cfg.f = 64, 3                                                # 2f > p_r
    assert B.lib().coded_qr_workspace_size(C.byref(cfg), C.byref(n)) == B.CQR_EINVAL
    cfg.f, cfg.dtype, cfg.mma = 1, B.CQR_F64, B.CQR_MMA_TF32            # tensor cores need F32
    assert B.lib().coded_qr_workspace_size(C.byref(cfg), C.byref(n)) == B.CQR_ENOTSUP
    h = C.c_void_p()
    assert B.lib().coded_qr_create(None, C.byref(h)) == B.CQR_EINVAL
    assert B.lib().coded_qr_factor(None, 0, -1) == B.CQR_EINVAL
