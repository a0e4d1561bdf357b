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
                 "post_orth", "solve", "solve_ls", "run", "get_generator", "get_decode_sets",
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


def test_binding_flag_values_match_header():
    """Every CQR_BATCH_* / CQR_RUN_* flag the binding passes has the header's value."""
    with open(os.path.join(ROOT, "include", "coded_qr.h")) as fh:
        text = fh.read()
    vals = {k: int(v) for k, v in re.findall(r"\b(CQR_BATCH_\w+)\s*=\s*(\d+)", text)}
    vals.update({k: int(v) for k, v in re.findall(r"#define\s+(CQR_RUN_\w+)\s+(\d+)u?", text)})
    from paper_2311_11943_gb300 import binding
    for name in ("CQR_BATCH_GRAPH", "CQR_BATCH_POST_ORTH", "CQR_BATCH_HOST_BUFFERS",
                 "CQR_RUN_HOST_BUFFERS"):
        assert getattr(binding, name) == vals[name], name


def test_solve_ls_validates_like_solve_without_gpu(libpath):
    # the least-squares verb under the problem statement's name takes the same arguments and
    # rejects the same null handle before touching the device
    from paper_2311_11943_gb300 import binding as B
    assert B.coded_qr_solve_ls(None, 0, 1, 0, 1, 1) == B.CQR_EINVAL
    assert B.coded_qr_solve(None, 0, 1, 0, 1, 1) == B.CQR_EINVAL
    assert B.lib().coded_qr_set_wait_limit(None, 100) == B.CQR_EINVAL


def test_config_struct_layout(libpath):
    from paper_2311_11943_gb300 import binding
    assert C.sizeof(binding.Config) == 96
    assert binding.Config.panel.offset == 56 and binding.Config.in_node.offset == 60
    assert binding.Config.post_orth.offset == 64 and binding.Config.reserved.offset == 68
    assert binding.Config.seed.offset == 72 and binding.Config.stream.offset == 88


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


def _cfg(B, **kw):
    cfg = B.Config()
    base = dict(m=64, n=64, p_r=4, p_c=4, f=1, b=8, dtype=B.CQR_F64, mma=B.CQR_MMA_SIMT,
                protect_r=1, gdist=B.CQR_G_UNIF01, nrhs_max=1, reorth_block=0, panel=0,
                in_node=0, seed=1, tau=0.0)
    base.update(kw)
    for k, v in base.items():
        setattr(cfg, k, v)
    return cfg


# each configuration rule of coded_qr_create (header: argument errors return synchronously,
# before any device call) with the status it must give
RULES = [
    (dict(m=0), "EINVAL"), (dict(n=0), "EINVAL"), (dict(m=32, n=64), "EINVAL"),   # m >= n >= 1
    (dict(p_r=0), "EINVAL"), (dict(p_c=0), "EINVAL"), (dict(b=0), "EINVAL"),
    (dict(f=-1), "EINVAL"), (dict(n=62), "EINVAL"),                             # p_c | n
    (dict(f=3), "EINVAL"),                                                      # 2f <= p_r
    (dict(p_r=8, f=3), "EINVAL"),                                               # 2f <= p_c (R protected)
    (dict(m=4096, n=4096, p_r=64, p_c=64, f=17), "ENOTSUP"),                    # f <= 16
    (dict(m=8192, n=8192, p_r=128, p_c=128, f=1), "ENOTSUP"),                   # p + f <= 128
    (dict(m=6, n=4, p_r=8, p_c=4), "EINVAL"),                                   # p_r <= m
    (dict(dtype=7), "EINVAL"), (dict(mma=9), "EINVAL"),
    (dict(mma=1), "ENOTSUP"),                                                   # tensor cores need FP32
    (dict(gdist=5), "EINVAL"), (dict(nrhs_max=-1), "EINVAL"), (dict(panel=4), "EINVAL"),
    (dict(in_node=2), "EINVAL"), (dict(in_node=1, f=4), "EINVAL"),              # in-node: f < p_r
    (dict(in_node=1, p_c=2, n=64), "ENOTSUP"),                                  # in-node R: p_c = p_r
]


@pytest.mark.parametrize("kw,status", RULES)
def test_configuration_rules(libpath, kw, status):
    from paper_2311_11943_gb300 import binding as B
    n = C.c_size_t(0)
    cfg = _cfg(B, **kw)
    want = getattr(B, "CQR_" + status)
    assert B.lib().coded_qr_workspace_size(C.byref(cfg), C.byref(n)) == want
    h = C.c_void_p()
    assert B.lib().coded_qr_create(C.byref(cfg), C.byref(h)) == want
    assert not h.value


def test_valid_configuration_without_a_device_is_a_cuda_error(libpath):
    # no CPU fallback: a valid configuration on a machine without a GPU fails with CQR_ECUDA
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2311_11943_gb300 import binding as B
    cfg = _cfg(B)
    n = C.c_size_t(0)
    assert B.lib().coded_qr_workspace_size(C.byref(cfg), C.byref(n)) == B.CQR_ECUDA
    h = C.c_void_p()
    assert B.lib().coded_qr_create(C.byref(cfg), C.byref(h)) == B.CQR_ECUDA


BATCH_RULES = [
    (dict(), [(256, 32), (512, 64)], 0, "EINVAL"),                     # count >= 1
    (dict(dtype=0), [(256, 32)], 1, "ENOTSUP"),                        # FP32 only
    (dict(mma=2), [(256, 32)], 1, "ENOTSUP"),                          # CUDA-core products
    (dict(b=-1), [(256, 32)], 1, "EINVAL"), (dict(b=65), [(256, 32)], 1, "ENOTSUP"),
    (dict(reorth_block=1), [(256, 32)], 1, "ENOTSUP"),
    (dict(), [(256, 32), (16, 32)], 2, "EINVAL"),                      # an instance with m < n
    (dict(), [(256, 32), (256, 30)], 2, "EINVAL"),                     # p_c does not divide n
]


@pytest.mark.parametrize("kw,shapes,count,status", BATCH_RULES)
def test_batched_configuration_rules(libpath, kw, shapes, count, status):
    from paper_2311_11943_gb300 import binding as B
    args = dict(dtype=B.CQR_F32, p_r=8, p_c=4, f=2, b=0)
    args.update(kw)
    cfg = _cfg(B, **args)
    ms = (C.c_int64 * len(shapes))(*[s[0] for s in shapes])
    ns = (C.c_int64 * len(shapes))(*[s[1] for s in shapes])
    h = C.c_void_p()
    assert B.lib().coded_qr_batched_create(C.byref(cfg), ms, ns, count, C.byref(h)) == \
        getattr(B, "CQR_" + status)
    assert not h.value
