"""Thin Python binding of the coded-QR C ABI (include/coded_qr.h).

Argument marshalling only: every step of the computation runs in the CUDA library.  The
functions `coded_qr_*` keep the C names and signatures (plain ints for pointers); the class
`CodedQR` wraps a handle for callers that hold their matrices in torch tensors (column-major
views: shape (rows, cols), stride (1, ld)).  There is no fallback: if the shared library is
missing this module raises on first use.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# CQR_LIBRARY=debug loads the bounds-checked build (build.build(debug_bounds=True)) instead
LIB_PATH = (os.path.join(_HERE, "_build_debug", "libcoded_qr_debug.so")
            if os.environ.get("CQR_LIBRARY") == "debug"
            else os.path.join(_HERE, "_build", "libcoded_qr.so"))

CQR_OK, CQR_EINVAL, CQR_ENOMEM, CQR_ECUDA, CQR_ESTATE = 0, 1, 2, 3, 4
CQR_EUNRECOVERABLE, CQR_EBREAKDOWN, CQR_ETIMEOUT, CQR_ENOTSUP, CQR_EBOUNDS = 5, 6, 7, 8, 9
CQR_F64, CQR_F32 = 0, 1
CQR_MMA_SIMT, CQR_MMA_TF32, CQR_MMA_3XTF32, CQR_MMA_BF16, CQR_MMA_BF16X3 = 0, 1, 2, 3, 4
MMA_NAMES = {"simt": CQR_MMA_SIMT, "tf32": CQR_MMA_TF32, "3xtf32": CQR_MMA_3XTF32,
             "bf16": CQR_MMA_BF16, "bf16x3": CQR_MMA_BF16X3}
CQR_G_UNIF01, CQR_G_NORMAL = 0, 1
PANEL_NAMES = {"icgs": 0, "mgs": 1, "cgs1": 2, "cgs2": 3}
POST_ORTH_NAMES = {"auto": 0, "g0": 1, "projected": 2}
CQR_RUN_HOST_BUFFERS = 1
GEO_FIELDS = ["m", "n", "mb", "nb", "m_pad", "c", "d", "M", "N", "ldq", "ldr", "grid_rows",
              "grid_cols", "panels", "code_blocks"]

EXPORTS = ["coded_qr_workspace_size", "coded_qr_create", "coded_qr_create_in", "coded_qr_destroy",
           "coded_qr_geometry", "coded_qr_encode", "coded_qr_factor", "coded_qr_inject_erasure",
           "coded_qr_recover", "coded_qr_post_orth", "coded_qr_solve", "coded_qr_solve_ls",
           "coded_qr_run",
           "coded_qr_get_factors", "coded_qr_get_generator", "coded_qr_get_decode_sets",
           "coded_qr_stats", "coded_qr_sync_status", "coded_qr_errstr", "coded_qr_profile",
           "coded_qr_profile_read", "coded_qr_profile_name", "coded_qr_panel_icgs_noalloc",
           "coded_qr_batched_create", "coded_qr_batched_destroy", "coded_qr_batched_geometry",
           "coded_qr_batched_encode", "coded_qr_batched_factor",
           "coded_qr_batched_inject_erasure", "coded_qr_batched_recover",
           "coded_qr_batched_post_orth", "coded_qr_batched_run", "coded_qr_batched_autotune",
           "coded_qr_batched_set_tuning", "coded_qr_batched_get_tuning",
           "coded_qr_batched_get_factors", "coded_qr_batched_get_decode_sets",
           "coded_qr_batched_sync_status", "coded_qr_batched_last_error",
           "coded_qr_batched_profile", "coded_qr_batched_phases",
           "coded_qr_adjoint_qr", "coded_qr_adjoint_lstsq", "coded_qr_mds_stats",
           "coded_qr_inject_node_failure", "coded_qr_set_wait_limit", "coded_qr_debug_bounds",
           "coded_qr_debug_bounds_selftest", "coded_qr_probe_exchange"]
CQR_BATCH_GRAPH, CQR_BATCH_POST_ORTH, CQR_BATCH_HOST_BUFFERS = 1, 2, 4
PROF_CLASSES = 17


class Config(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("p_r", C.c_int32), ("p_c", C.c_int32),
                ("f", C.c_int32), ("b", C.c_int32), ("dtype", C.c_int32), ("mma", C.c_int32),
                ("protect_r", C.c_int32), ("gdist", C.c_int32), ("nrhs_max", C.c_int32),
                ("reorth_block", C.c_int32), ("panel", C.c_int32), ("in_node", C.c_int32),
                ("post_orth", C.c_int32), ("reserved", C.c_int32),
                ("seed", C.c_uint64), ("tau", C.c_double),
                ("stream", C.c_void_p)]


class CodedQRError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, errstr(status), status))


_lib = None


def lib():
    """Load the CUDA library (no fallback: raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("coded-QR CUDA library not built (%s); run "
                               "__graft_entry__.build() or paper_2311_11943_gb300/build.py"
                               % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32
        pcfg = C.POINTER(Config)
        sig = {
            "coded_qr_workspace_size": [pcfg, C.POINTER(C.c_size_t)],
            "coded_qr_create": [pcfg, C.POINTER(vp)],
            "coded_qr_create_in": [pcfg, vp, C.c_size_t, C.POINTER(vp)],
            "coded_qr_destroy": [vp],
            "coded_qr_geometry": [vp, C.POINTER(i64)],
            "coded_qr_encode": [vp, vp, i64],
            "coded_qr_factor": [vp, i32, i32],
            "coded_qr_inject_erasure": [vp, C.POINTER(i32), i32],
            "coded_qr_inject_node_failure": [vp, C.POINTER(i32), i32],
            "coded_qr_recover": [vp, C.POINTER(i32)],
            "coded_qr_post_orth": [vp, vp, i64, vp, i64, vp, i64, i32],
            "coded_qr_solve": [vp, vp, i64, vp, i64, i32],
            "coded_qr_solve_ls": [vp, vp, i64, vp, i64, i32],
            "coded_qr_run": [vp, vp, i64, vp, i64, vp, i64, i32, C.POINTER(i32), i32, u32],
            "coded_qr_get_factors": [vp, C.POINTER(vp), C.POINTER(i64), C.POINTER(vp),
                                     C.POINTER(i64)],
            "coded_qr_get_generator": [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)],
            "coded_qr_get_decode_sets": [vp, C.POINTER(i32), i32, C.POINTER(i32)],
            "coded_qr_stats": [vp, C.POINTER(i64)],
            "coded_qr_sync_status": [vp],
            "coded_qr_set_wait_limit": [vp, i64],
            "coded_qr_debug_bounds": [C.POINTER(i32)],
            "coded_qr_debug_bounds_selftest": [vp],
            "coded_qr_probe_exchange": [i32, i64, i32, i32, C.POINTER(C.c_double), vp],
            "coded_qr_profile": [vp, i32],
            "coded_qr_profile_read": [vp, C.POINTER(C.c_double), C.POINTER(i64), i32, i32],
            "coded_qr_panel_icgs_noalloc": [i32, i64, i32, vp, i64, vp, i64, C.c_double, vp, vp],
            "coded_qr_adjoint_qr": [vp, vp, i64, vp, i64, vp, i64, vp, i64],
            "coded_qr_mds_stats": [C.POINTER(C.c_double), i32, i32, C.POINTER(C.c_double),
                                   C.POINTER(C.c_double), C.POINTER(i64), vp],
            "coded_qr_adjoint_lstsq": [vp, vp, i64, vp, i64, vp, i64, vp, i64, i32, vp, i64, vp,
                                       i64],
            "coded_qr_batched_create": [pcfg, C.POINTER(i64), C.POINTER(i64), i32, C.POINTER(vp)],
            "coded_qr_batched_destroy": [vp],
            "coded_qr_batched_geometry": [vp, i32, C.POINTER(i64)],
            "coded_qr_batched_encode": [vp, C.POINTER(vp), C.POINTER(i64)],
            "coded_qr_batched_factor": [vp, C.POINTER(i32)],
            "coded_qr_batched_inject_erasure": [vp, C.POINTER(i32), i32],
            "coded_qr_batched_recover": [vp, C.POINTER(i32)],
            "coded_qr_batched_post_orth": [vp],
            "coded_qr_batched_run": [vp, C.POINTER(vp), C.POINTER(i64), C.POINTER(i32), i32, i32],
            "coded_qr_batched_autotune": [vp, C.POINTER(vp), C.POINTER(i64), C.POINTER(i32), i32,
                                          i32, C.POINTER(i32)],
            "coded_qr_batched_set_tuning": [vp, i32, C.POINTER(i32)],
            "coded_qr_batched_get_tuning": [vp, C.POINTER(i32), C.POINTER(i32)],
            "coded_qr_batched_get_factors": [vp, i32, C.POINTER(vp), C.POINTER(i64),
                                             C.POINTER(vp), C.POINTER(i64)],
            "coded_qr_batched_get_decode_sets": [vp, i32, C.POINTER(i32), i32, C.POINTER(i32)],
            "coded_qr_batched_sync_status": [vp, C.POINTER(i32), C.POINTER(i64)],
            "coded_qr_batched_profile": [vp, i32],
            "coded_qr_batched_phases": [vp, C.POINTER(i64), i32],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.coded_qr_errstr.argtypes = [C.c_int]
        L.coded_qr_errstr.restype = C.c_char_p
        L.coded_qr_batched_last_error.argtypes = []
        L.coded_qr_batched_last_error.restype = C.c_char_p
        L.coded_qr_profile_name.argtypes = [C.c_int32]
        L.coded_qr_profile_name.restype = C.c_char_p
        _lib = L
    return _lib


def errstr(status):
    return lib().coded_qr_errstr(int(status)).decode()


def check(status, where):
    if status != CQR_OK:
        raise CodedQRError(status, where)


# ------------------------------------------------------------------ C-named entry points
def coded_qr_workspace_size(cfg):
    n = C.c_size_t(0)
    check(lib().coded_qr_workspace_size(C.byref(cfg), C.byref(n)), "coded_qr_workspace_size")
    return n.value


def coded_qr_create(cfg):
    h = C.c_void_p()
    check(lib().coded_qr_create(C.byref(cfg), C.byref(h)), "coded_qr_create")
    return h


def coded_qr_create_in(cfg, workspace_ptr, nbytes):
    h = C.c_void_p()
    check(lib().coded_qr_create_in(C.byref(cfg), C.c_void_p(workspace_ptr), nbytes, C.byref(h)),
          "coded_qr_create_in")
    return h


def coded_qr_destroy(h):
    return lib().coded_qr_destroy(h)


def coded_qr_geometry(h):
    d = (C.c_int64 * len(GEO_FIELDS))()
    check(lib().coded_qr_geometry(h, d), "coded_qr_geometry")
    return dict(zip(GEO_FIELDS, [int(v) for v in d]))


def coded_qr_encode(h, A_ptr, lda):
    return lib().coded_qr_encode(h, C.c_void_p(A_ptr), lda)


def coded_qr_factor(h, t0, t1=-1):
    return lib().coded_qr_factor(h, t0, t1)


def coded_qr_inject_erasure(h, tiles):
    flat = (C.c_int32 * max(1, 2 * len(tiles)))(*[int(v) for t in tiles for v in t])
    return lib().coded_qr_inject_erasure(h, flat, len(tiles))


def coded_qr_inject_node_failure(h, nodes):
    flat = (C.c_int32 * max(1, 2 * len(nodes)))(*[v for t in nodes for v in t])
    return lib().coded_qr_inject_node_failure(h, flat, len(nodes))


def coded_qr_recover(h):
    n = C.c_int32(0)
    st = lib().coded_qr_recover(h, C.byref(n))
    return st, n.value


def coded_qr_post_orth(h, Q_ptr, ldq, y_ptr, ldy, yo_ptr, ldyo, nrhs):
    return lib().coded_qr_post_orth(h, C.c_void_p(Q_ptr or None), ldq, C.c_void_p(y_ptr or None),
                                    ldy, C.c_void_p(yo_ptr or None), ldyo, nrhs)


def coded_qr_solve(h, y_ptr, ldy, x_ptr, ldx, nrhs):
    return lib().coded_qr_solve(h, C.c_void_p(y_ptr), ldy, C.c_void_p(x_ptr), ldx, nrhs)


def coded_qr_solve_ls(h, y_ptr, ldy, x_ptr, ldx, nrhs):
    return lib().coded_qr_solve_ls(h, C.c_void_p(y_ptr), ldy, C.c_void_p(x_ptr), ldx, nrhs)


def coded_qr_run(h, A_ptr, lda, y_ptr, ldy, x_ptr, ldx, nrhs, plan, flags=0):
    flat = (C.c_int32 * max(1, 3 * len(plan)))(*[int(v) for p in plan for v in p])
    return lib().coded_qr_run(h, C.c_void_p(A_ptr), lda, C.c_void_p(y_ptr or None), ldy,
                              C.c_void_p(x_ptr or None), ldx, nrhs, flat, len(plan), flags)


def coded_qr_get_factors(h):
    q, r = C.c_void_p(), C.c_void_p()
    lq, lr = C.c_int64(), C.c_int64()
    check(lib().coded_qr_get_factors(h, C.byref(q), C.byref(lq), C.byref(r), C.byref(lr)),
          "coded_qr_get_factors")
    return q.value, lq.value, r.value, lr.value


def coded_qr_get_generator(h, f, p_r, p_c):
    Gt = np.zeros(max(1, f * p_r))
    Gh = np.zeros(max(1, f * p_c))
    check(lib().coded_qr_get_generator(h, Gt.ctypes.data_as(C.POINTER(C.c_double)),
                                       Gh.ctypes.data_as(C.POINTER(C.c_double))),
          "coded_qr_get_generator")
    return Gt[: f * p_r].reshape(f, p_r), Gh[: f * p_c].reshape(p_c, f)


def coded_qr_get_decode_sets(h):
    n = C.c_int32(0)
    check(lib().coded_qr_get_decode_sets(h, None, 0, C.byref(n)), "coded_qr_get_decode_sets")
    buf = (C.c_int32 * max(1, n.value))()
    check(lib().coded_qr_get_decode_sets(h, buf, n.value, C.byref(n)), "coded_qr_get_decode_sets")
    return [int(buf[i]) for i in range(n.value)]


def coded_qr_stats(h):
    out = (C.c_int64 * 4)()
    check(lib().coded_qr_stats(h, out), "coded_qr_stats")
    return dict(n_reorth=out[0], n_recovered=out[1], panels_run=out[2], n_injected=out[3])


def coded_qr_sync_status(h):
    return lib().coded_qr_sync_status(h)


def coded_qr_profile(h, enable):
    return lib().coded_qr_profile(h, int(bool(enable)))


def coded_qr_profile_read(h, reset=True):
    ms = (C.c_double * PROF_CLASSES)()
    ln = (C.c_int64 * PROF_CLASSES)()
    check(lib().coded_qr_profile_read(h, ms, ln, PROF_CLASSES, int(bool(reset))),
          "coded_qr_profile_read")
    return {coded_qr_profile_name(k): (ms[k], ln[k]) for k in range(PROF_CLASSES)}


def coded_qr_panel_icgs_noalloc(dtype, M, bk, Q_ptr, ldq, R_ptr, ldr, tau=0.0, status_ptr=0,
                                stream=0):
    return lib().coded_qr_panel_icgs_noalloc(dtype, M, bk, C.c_void_p(Q_ptr), ldq, C.c_void_p(R_ptr),
                                             ldr, tau, C.c_void_p(status_ptr or None),
                                             C.c_void_p(stream or None))


def coded_qr_adjoint_qr(h, Q_ptr, ldq, Qbar_ptr, ldqb, Rbar_ptr, ldrb, Abar_ptr, ldab):
    return lib().coded_qr_adjoint_qr(h, Q_ptr, ldq, Qbar_ptr or None, ldqb, Rbar_ptr or None, ldrb,
                                     Abar_ptr, ldab)


def coded_qr_adjoint_lstsq(h, A_ptr, lda, y_ptr, ldy, x_ptr, ldx, xbar_ptr, ldxb, nrhs, Abar_ptr,
                           ldab, ybar_ptr, ldyb):
    return lib().coded_qr_adjoint_lstsq(h, A_ptr, lda, y_ptr, ldy, x_ptr, ldx, xbar_ptr, ldxb, nrhs,
                                        Abar_ptr or None, ldab, ybar_ptr or None, ldyb)


def coded_qr_mds_stats(G, stream=0):
    """(min |det| per size, max condition number per size, count) over every square
    submatrix of G (f x p_r); index 0 of each list is the value over all sizes."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    f, p = G.shape
    md = (C.c_double * (f + 1))()
    mc = (C.c_double * (f + 1))()
    cnt = C.c_int64(0)
    check(lib().coded_qr_mds_stats(G.ctypes.data_as(C.POINTER(C.c_double)), f, p, md, mc,
                                   C.byref(cnt), C.c_void_p(stream)), "coded_qr_mds_stats")
    return list(md), list(mc), cnt.value


def coded_qr_profile_name(k):
    v = lib().coded_qr_profile_name(k)
    return v.decode() if v else None


# ------------------------------------------------------------------ torch convenience layer
def _i64s(vals):
    return (C.c_int64 * len(vals))(*[int(v) for v in vals])


def _i32s(vals):
    vals = list(vals)
    return (C.c_int32 * max(1, len(vals)))(*[int(v) for v in vals])


def _ptrs(vals):
    return (C.c_void_p * len(vals))(*[int(v) for v in vals])


def coded_qr_batched_last_error():
    return lib().coded_qr_batched_last_error().decode()


def _bcheck(status, where):
    if status == CQR_ECUDA:
        where = "%s [%s]" % (where, coded_qr_batched_last_error())
    check(status, where)


def coded_qr_batched_create(cfg, m, n):
    bh = C.c_void_p()
    _bcheck(lib().coded_qr_batched_create(C.byref(cfg), _i64s(m), _i64s(n), len(m), C.byref(bh)),
          "coded_qr_batched_create")
    return bh


def coded_qr_batched_destroy(bh):
    return lib().coded_qr_batched_destroy(bh)


def coded_qr_batched_geometry(bh, i):
    d = (C.c_int64 * len(GEO_FIELDS))()
    _bcheck(lib().coded_qr_batched_geometry(bh, i, d), "coded_qr_batched_geometry")
    return dict(zip(GEO_FIELDS, [int(v) for v in d]))


def coded_qr_batched_encode(bh, A_ptrs, ldas):
    return lib().coded_qr_batched_encode(bh, _ptrs(A_ptrs), _i64s(ldas))


def coded_qr_batched_factor(bh, panel_end=None):
    return lib().coded_qr_batched_factor(bh, _i32s(panel_end) if panel_end is not None else None)


def coded_qr_batched_inject_erasure(bh, triples):
    flat = [v for t in triples for v in t]
    return lib().coded_qr_batched_inject_erasure(bh, _i32s(flat), len(triples))


def coded_qr_batched_recover(bh):
    n = C.c_int32(0)
    st = lib().coded_qr_batched_recover(bh, C.byref(n))
    return st, n.value


def coded_qr_batched_post_orth(bh):
    return lib().coded_qr_batched_post_orth(bh)


def coded_qr_batched_run(bh, A_ptrs, ldas, erasures, flags):
    flat = [v for e in erasures for v in e]
    return lib().coded_qr_batched_run(bh, _ptrs(A_ptrs), _i64s(ldas), _i32s(flat), len(erasures),
                                      flags)


def coded_qr_batched_autotune(bh, A_ptrs, ldas, erasures, reps):
    g = C.c_int32(0)
    flat = [v for e in erasures for v in e]
    st = lib().coded_qr_batched_autotune(bh, _ptrs(A_ptrs), _i64s(ldas), _i32s(flat),
                                         len(erasures), reps, C.byref(g))
    return st, g.value


def coded_qr_batched_set_tuning(bh, cluster, b=None):
    return lib().coded_qr_batched_set_tuning(bh, cluster, _i32s(b) if b is not None else None)


def coded_qr_batched_get_tuning(bh, count):
    g = C.c_int32(0)
    b = (C.c_int32 * count)()
    _bcheck(lib().coded_qr_batched_get_tuning(bh, C.byref(g), b), "coded_qr_batched_get_tuning")
    return g.value, [int(v) for v in b]


def coded_qr_batched_get_factors(bh, i):
    q, r = C.c_void_p(), C.c_void_p()
    ldq, ldr = C.c_int64(0), C.c_int64(0)
    _bcheck(lib().coded_qr_batched_get_factors(bh, i, C.byref(q), C.byref(ldq), C.byref(r),
                                             C.byref(ldr)), "coded_qr_batched_get_factors")
    return q.value, ldq.value, r.value, ldr.value


def coded_qr_batched_get_decode_sets(bh, i):
    n = C.c_int32(0)
    _bcheck(lib().coded_qr_batched_get_decode_sets(bh, i, None, 0, C.byref(n)),
          "coded_qr_batched_get_decode_sets")
    buf = (C.c_int32 * max(1, n.value))()
    _bcheck(lib().coded_qr_batched_get_decode_sets(bh, i, buf, n.value, C.byref(n)),
          "coded_qr_batched_get_decode_sets")
    return [int(v) for v in buf[: n.value]]


def coded_qr_batched_sync_status(bh):
    bad = C.c_int32(-1)
    nre = C.c_int64(0)
    st = lib().coded_qr_batched_sync_status(bh, C.byref(bad), C.byref(nre))
    return st, bad.value, nre.value


class _DevView:
    """__cuda_array_interface__ over memory owned by the library (borrowed)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def colmajor_empty(rows, cols, dtype, device="cuda", ld=None):
    """A (rows x cols) column-major torch tensor (stride (1, ld))."""
    import torch
    ld = ld or rows
    return torch.empty((cols, ld), dtype=dtype, device=device).t()[:rows, :]


def _ld(t):
    if t.dim() == 1:
        return t.shape[0]
    assert t.stride(0) == 1, "column-major tensor expected (stride (1, ld))"
    return t.stride(1) if t.shape[1] > 1 else max(t.shape[0], 1)


class CodedQR:
    """One coded QR problem on the current CUDA device (handle wrapper)."""

    def __init__(self, m, n, p_r, p_c, f, b, dtype="f64", mma="simt", protect_r=True,
                 gdist=CQR_G_UNIF01, nrhs_max=1, seed=1, tau=0.0, stream=None, workspace=None,
                 reorth_block=False, panel="icgs", in_node=False, post_orth="auto"):
        import torch
        self.torch = torch
        self.tdtype = torch.float64 if dtype in ("f64", "float64") else torch.float32
        cfg = Config()
        cfg.m, cfg.n, cfg.p_r, cfg.p_c, cfg.f, cfg.b = m, n, p_r, p_c, f, b
        cfg.dtype = CQR_F64 if self.tdtype == torch.float64 else CQR_F32
        cfg.mma = MMA_NAMES[mma]
        cfg.protect_r = int(bool(protect_r))
        cfg.gdist = gdist
        cfg.nrhs_max = nrhs_max
        cfg.reorth_block = int(bool(reorth_block))
        cfg.panel = PANEL_NAMES[panel]
        cfg.in_node = int(bool(in_node))
        cfg.post_orth = POST_ORTH_NAMES[post_orth]
        cfg.seed = seed
        cfg.tau = tau
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        cfg.stream = C.c_void_p(stream.cuda_stream)
        self.cfg = cfg
        self._ws = None
        if workspace == "torch":
            nbytes = coded_qr_workspace_size(cfg)
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = (self._ws.data_ptr() + 255) // 256 * 256
            self.h = coded_qr_create_in(cfg, base, nbytes)
        else:
            self.h = coded_qr_create(cfg)
        self.geo = coded_qr_geometry(self.h)

    def close(self):
        if getattr(self, "h", None):
            coded_qr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- hot-path verbs
    def encode(self, A):
        check(coded_qr_encode(self.h, A.data_ptr(), _ld(A)), "coded_qr_encode")

    def factor(self, t0=0, t1=-1):
        check(coded_qr_factor(self.h, t0, t1), "coded_qr_factor")

    def inject(self, tiles):
        check(coded_qr_inject_erasure(self.h, tiles), "coded_qr_inject_erasure")

    def fail_nodes(self, nodes):
        check(coded_qr_inject_node_failure(self.h, nodes), "coded_qr_inject_node_failure")

    def recover(self):
        st, n = coded_qr_recover(self.h)
        check(st, "coded_qr_recover")
        return n

    def post_orth(self, Q=None, y=None, yo=None):
        nrhs = 0 if y is None else (1 if y.dim() == 1 else y.shape[1])
        check(coded_qr_post_orth(self.h, Q.data_ptr() if Q is not None else 0,
                                 _ld(Q) if Q is not None else 0,
                                 y.data_ptr() if y is not None else 0,
                                 _ld(y) if y is not None else 0,
                                 yo.data_ptr() if yo is not None else 0,
                                 _ld(yo) if yo is not None else 0, nrhs), "coded_qr_post_orth")

    def solve(self, y, x):
        nrhs = 1 if y.dim() == 1 else y.shape[1]
        check(coded_qr_solve(self.h, y.data_ptr(), _ld(y), x.data_ptr(), _ld(x), nrhs),
              "coded_qr_solve")

    def solve_ls(self, y, x):
        """min |A x - y| through the coded factors (coded_qr_solve_ls)."""
        nrhs = 1 if y.dim() == 1 else y.shape[1]
        check(coded_qr_solve_ls(self.h, y.data_ptr(), _ld(y), x.data_ptr(), _ld(x), nrhs),
              "coded_qr_solve_ls")

    def run(self, A, y=None, x=None, plan=(), host=False):
        nrhs = 0 if y is None else (1 if y.ndim == 1 else y.shape[1])
        if host:
            import numpy as _np
            A_ptr = A.ctypes.data
            lda = A.shape[0] if A.flags.f_contiguous else None
            assert lda is not None, "host A must be Fortran-ordered"
            y_ptr = y.ctypes.data if y is not None else 0
            x_ptr = x.ctypes.data if x is not None else 0
            ldy = y.shape[0] if y is not None else 0
            ldx = x.shape[0] if x is not None else 0
            st = coded_qr_run(self.h, A_ptr, lda, y_ptr, ldy, x_ptr, ldx, nrhs, list(plan),
                              CQR_RUN_HOST_BUFFERS)
        else:
            st = coded_qr_run(self.h, A.data_ptr(), _ld(A), y.data_ptr() if y is not None else 0,
                              _ld(y) if y is not None else 0,
                              x.data_ptr() if x is not None else 0,
                              _ld(x) if x is not None else 0, nrhs, list(plan), 0)
        check(st, "coded_qr_run")

    # -- inspection
    def factors(self):
        """Borrowed torch views (column-major) of the coded Q (M x N) and R (N x N)."""
        q, ldq, r, ldr = coded_qr_get_factors(self.h)
        g = self.geo
        ts = "<f8" if self.tdtype == self.torch.float64 else "<f4"
        Qv = self.torch.as_tensor(_DevView(q, (g["N"], ldq), ts), device="cuda").t()[: g["M"], :]
        Rv = self.torch.as_tensor(_DevView(r, (g["N"], ldr), ts), device="cuda").t()[: g["N"], :]
        return Qv, Rv

    def generator(self):
        return coded_qr_get_generator(self.h, self.cfg.f, self.cfg.p_r, self.cfg.p_c)

    def decode_sets(self):
        return coded_qr_get_decode_sets(self.h)

    def stats(self):
        return coded_qr_stats(self.h)

    def sync_status(self):
        return coded_qr_sync_status(self.h)

    def set_wait_limit(self, cycles):
        """Bound (SM cycles) of the panel's waits between CTAs; 0 restores the default."""
        check(lib().coded_qr_set_wait_limit(self.h, int(cycles)), "coded_qr_set_wait_limit")

    def profile(self, enable=True):
        check(coded_qr_profile(self.h, enable), "coded_qr_profile")

    def profile_read(self, reset=True):
        return coded_qr_profile_read(self.h, reset)

    # -- reverse mode (accumulating into Abar / ybar)
    def adjoint_qr(self, Q, Qbar, Rbar, Abar):
        check(coded_qr_adjoint_qr(self.h, Q.data_ptr(), _ld(Q),
                                  Qbar.data_ptr() if Qbar is not None else 0,
                                  _ld(Qbar) if Qbar is not None else 0,
                                  Rbar.data_ptr() if Rbar is not None else 0,
                                  _ld(Rbar) if Rbar is not None else 0,
                                  Abar.data_ptr(), _ld(Abar)), "coded_qr_adjoint_qr")

    def adjoint_lstsq(self, A, y, x, xbar, Abar, ybar):
        nrhs = 1 if x.dim() == 1 else x.shape[1]
        check(coded_qr_adjoint_lstsq(self.h, A.data_ptr(), _ld(A), y.data_ptr(), _ld(y),
                                     x.data_ptr(), _ld(x), xbar.data_ptr(), _ld(xbar), nrhs,
                                     Abar.data_ptr() if Abar is not None else 0,
                                     _ld(Abar) if Abar is not None else 0,
                                     ybar.data_ptr() if ybar is not None else 0,
                                     _ld(ybar) if ybar is not None else 0),
              "coded_qr_adjoint_lstsq")


class CodedQRBatch:
    """A batch of independent FP32 coded QRs of shapes (m_i, n_i) (batch handle wrapper).
    Inputs are lists of column-major torch tensors on the current CUDA device."""

    def __init__(self, shapes, p_r, p_c, f, b=0, protect_r=True, gdist=CQR_G_UNIF01, seed=1,
                 tau=0.0, stream=None):
        import torch
        self.torch = torch
        cfg = Config()
        cfg.m, cfg.n = 0, 0
        cfg.p_r, cfg.p_c, cfg.f, cfg.b = p_r, p_c, f, b
        cfg.dtype, cfg.mma = CQR_F32, CQR_MMA_SIMT
        cfg.protect_r = int(bool(protect_r))
        cfg.gdist = gdist
        cfg.nrhs_max = 1
        cfg.seed = seed
        cfg.tau = tau
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        cfg.stream = C.c_void_p(stream.cuda_stream)
        self.cfg = cfg
        self.shapes = [(int(m), int(n)) for m, n in shapes]
        self.count = len(self.shapes)
        self.h = coded_qr_batched_create(cfg, [m for m, _ in self.shapes],
                                         [n for _, n in self.shapes])
        self.geo = [coded_qr_batched_geometry(self.h, i) for i in range(self.count)]

    def close(self):
        if getattr(self, "h", None):
            coded_qr_batched_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _args(As):
        return [a.data_ptr() for a in As], [_ld(a) for a in As]

    def encode(self, As):
        _bcheck(coded_qr_batched_encode(self.h, *self._args(As)), "coded_qr_batched_encode")

    def factor(self, panel_end=None):
        _bcheck(coded_qr_batched_factor(self.h, panel_end), "coded_qr_batched_factor")

    def inject(self, triples):
        _bcheck(coded_qr_batched_inject_erasure(self.h, triples), "coded_qr_batched_inject_erasure")

    def recover(self):
        st, n = coded_qr_batched_recover(self.h)
        _bcheck(st, "coded_qr_batched_recover")
        return n

    def post_orth(self):
        _bcheck(coded_qr_batched_post_orth(self.h), "coded_qr_batched_post_orth")

    def run(self, As, erasures=(), graph=True, post_orth=False, host=False):
        """The whole sequence; with host=True, As are Fortran-ordered host arrays (numpy
        views of pinned memory copy at full speed), copied by the library on its stream."""
        flags = (CQR_BATCH_GRAPH if graph else 0) | (CQR_BATCH_POST_ORTH if post_orth else 0)
        if host:
            for a in As:
                assert a.flags.f_contiguous, "host A must be Fortran-ordered"
            args = ([a.ctypes.data for a in As], [a.shape[0] for a in As])
            flags |= CQR_BATCH_HOST_BUFFERS
        else:
            args = self._args(As)
        _bcheck(coded_qr_batched_run(self.h, *args, list(erasures), flags),
              "coded_qr_batched_run")

    def autotune(self, As, erasures=(), reps=2):
        st, g = coded_qr_batched_autotune(self.h, *self._args(As), list(erasures), reps)
        _bcheck(st, "coded_qr_batched_autotune")
        self.geo = [coded_qr_batched_geometry(self.h, i) for i in range(self.count)]
        return g

    def set_tuning(self, cluster, b=None):
        _bcheck(coded_qr_batched_set_tuning(self.h, cluster, b), "coded_qr_batched_set_tuning")
        self.geo = [coded_qr_batched_geometry(self.h, i) for i in range(self.count)]

    def tuning(self):
        return coded_qr_batched_get_tuning(self.h, self.count)

    def factors(self, i):
        """Borrowed column-major views of instance i's coded Q (M x N) and R (N x N)."""
        q, ldq, r, ldr = coded_qr_batched_get_factors(self.h, i)
        g = self.geo[i]
        Qv = self.torch.as_tensor(_DevView(q, (g["N"], ldq), "<f4"), device="cuda").t()[: g["M"], :]
        Rv = self.torch.as_tensor(_DevView(r, (g["N"], ldr), "<f4"), device="cuda").t()[: g["N"], :]
        return Qv, Rv

    def decode_sets(self, i):
        return coded_qr_batched_get_decode_sets(self.h, i)

    def sync_status(self):
        return coded_qr_batched_sync_status(self.h)

    BATCH_PHASES = ("recover", "panel", "s_product", "rbar_reduce", "update", "other",
                    "s_product_wait", "update_wait")

    def profile(self, on=True):
        """Phase clocks of the later factor launches (coded_qr_batched_profile)."""
        _bcheck(lib().coded_qr_batched_profile(self.h, 1 if on else 0), "coded_qr_batched_profile")

    def phases(self, reset=True):
        """SM cycles per phase summed over the CTAs, and the number of CTAs."""
        n = len(self.BATCH_PHASES)
        buf = (C.c_int64 * (n + 1))()
        _bcheck(lib().coded_qr_batched_phases(self.h, buf, 1 if reset else 0),
                "coded_qr_batched_phases")
        return dict(zip(self.BATCH_PHASES, buf[:n])), buf[n]


def debug_bounds():
    """(status, site) of the bounds-checked build's index checks since the last call
    (coded_qr_debug_bounds; CQR_ENOTSUP from the normal build)."""
    site = C.c_int32(0)
    st = lib().coded_qr_debug_bounds(C.byref(site))
    return st, site.value


def probe_exchange(kind, M, bk, reps=8, stream=None):
    """Mean device time per panel column (microseconds) of the per-column reductions alone, for
    an M x bk FP32 panel: kind 0 the register panel, 1 the shared-memory panel
    (coded_qr_probe_exchange)."""
    us = C.c_double(0.0)
    check(lib().coded_qr_probe_exchange(kind, M, bk, reps, C.byref(us), C.c_void_p(stream)),
          "coded_qr_probe_exchange")
    return us.value


def debug_bounds_selftest(stream=None):
    """Enqueue the bounds-checked build's self-test (one guarded write out of range)."""
    return lib().coded_qr_debug_bounds_selftest(C.c_void_p(stream))
