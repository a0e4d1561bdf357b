"""ctypes front end of the FP64 CPU oracle (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this module.
Every function forwards to a routine of cqr_oracle.c, which cites the passage of the
paper (arXiv 2311.11943) it follows.  Arrays are numpy float64, Fortran (column-major)
order.  Nothing here imports the CUDA package.
"""
import contextlib
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

EBREAKDOWN = 6
EUNRECOVERABLE = 5


class Geom(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("p_r", C.c_int32), ("p_c", C.c_int32),
                ("f", C.c_int32), ("protect_r", C.c_int32), ("mb", C.c_int64),
                ("nb", C.c_int64), ("m_pad", C.c_int64), ("c", C.c_int64), ("d", C.c_int64),
                ("M", C.c_int64), ("N", C.c_int64), ("grid_rows", C.c_int32),
                ("grid_cols", C.c_int32)]


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(C.CDLL(_build.build()))
    return _lib


@contextlib.contextmanager
def library(path):
    """Run the oracle from another build of cqr_oracle.c for the duration of the block (the
    tests plant mistakes in copies of the source to show that the pins catch them)."""
    global _lib
    saved = _lib
    _lib = _bind(C.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _bind(L):
    d = C.POINTER(C.c_double)
    i64 = C.c_int64
    L.cqro_geom_init.argtypes = [C.POINTER(Geom), i64, i64, C.c_int, C.c_int, C.c_int, C.c_int]
    L.cqro_generator.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int, C.c_int, d, d]
    L.cqro_splitmix64.argtypes = [C.c_uint64, C.c_int, C.POINTER(C.c_uint64)]
    L.cqro_encode.argtypes = [C.POINTER(Geom), d, d, d, i64, d, i64]
    L.cqro_icgs_panel.argtypes = [i64, i64, i64, C.c_double, d, i64, d, i64, C.POINTER(i64)]
    L.cqro_factor.argtypes = [i64, i64, i64, i64, C.c_int, C.c_int, C.c_double, d, i64, d,
                              i64, C.POINTER(i64)]
    L.cqro_factor2.argtypes = [i64, i64, i64, i64, C.c_int, C.c_int, C.c_double, C.c_int, d,
                               i64, d, i64, C.POINTER(i64)]
    L.cqro_factor3.argtypes = [i64, i64, i64, i64, C.c_int, C.c_int, C.c_double, C.c_int,
                               C.c_int, d, i64, d, i64, C.POINTER(i64)]
    L.cqro_cgs_panel.argtypes = [i64, i64, i64, C.c_int, d, i64, d, i64]
    L.cqro_inject.argtypes = [C.POINTER(Geom), C.POINTER(C.c_int), C.c_int,
                              C.POINTER(C.c_uint8), d, i64, d, i64]
    L.cqro_invert_small.argtypes = [C.c_int, d, d]
    L.cqro_recover.argtypes = [C.POINTER(Geom), d, d, C.POINTER(C.c_uint8), d, i64, d, i64,
                               C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int),
                               C.POINTER(C.c_int)]
    L.cqro_build_G0.argtypes = [C.POINTER(Geom), d, d, i64]
    L.cqro_post_orth_dense.argtypes = [C.POINTER(Geom), d, d, i64, i64, d, i64]
    L.cqro_post_orth_block.argtypes = [C.POINTER(Geom), d, d, i64, i64, d, i64]
    L.cqro_back_substitute.argtypes = [i64, d, i64, d, i64, i64]
    L.cqro_solve_square.argtypes = [i64, i64, d, i64, d, i64, d, i64, i64, d, i64]
    L.cqro_solve_ls.argtypes = [i64, i64, d, i64, d, i64, d, i64, i64, d, i64]
    return L


def _p(a):
    assert a.dtype == np.float64 and (a.flags.f_contiguous or a.ndim == 1)
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ld(a):
    return a.shape[0]


class OracleError(RuntimeError):
    def __init__(self, rc, what):
        super().__init__("%s failed with status %d" % (what, rc))
        self.rc = rc


def _chk(rc, what):
    if rc != 0:
        raise OracleError(rc, what)


def geom(m, n, p_r, p_c, f, protect_r=True):
    g = Geom()
    _chk(lib().cqro_geom_init(C.byref(g), m, n, p_r, p_c, f, int(bool(protect_r))), "geom")
    return g


def splitmix64(seed, count):
    out = (C.c_uint64 * count)()
    lib().cqro_splitmix64(seed, count, out)
    return [int(v) for v in out]


def generator(f, p_r, p_c, seed, gdist=0, gh_ones=False):
    """a1: (G~ f x p_r, G~_h p_c x f), both returned as 2-D float64 arrays."""
    Gt = np.zeros(max(f * p_r, 1))
    Gh = np.zeros(max(p_c * f, 1))
    _chk(lib().cqro_generator(f, p_r, p_c, seed, gdist, int(gh_ones), _p(Gt), _p(Gh)), "generator")
    return Gt[: f * p_r].reshape(f, p_r).copy(), Gh[: p_c * f].reshape(p_c, f).copy()


def _rowmajor(G):
    G = np.ascontiguousarray(G, dtype=np.float64).ravel()
    return G if G.size else np.zeros(1)


def encode(g, Gt, Gh, A):
    """a2: the encoded matrix At (M x N) from A (m x n)."""
    A = np.asfortranarray(A, dtype=np.float64)
    At = np.zeros((g.M, g.N), order="F")
    _chk(lib().cqro_encode(C.byref(g), _p(_rowmajor(Gt)), _p(_rowmajor(Gh)), _p(A), _ld(A),
                           _p(At), _ld(At)), "encode")
    return At


def icgs_panel(Q, R, kb, bk, tau=0.7071067811865476):
    nre = C.c_int64(0)
    rc = lib().cqro_icgs_panel(Q.shape[0], kb, bk, tau, _p(Q), _ld(Q), _p(R), _ld(R), C.byref(nre))
    _chk(rc, "icgs_panel")
    return nre.value


PANELS = {"icgs": 0, "mgs": 1, "cgs1": 2, "cgs2": 3}


def cgs_panel(Q, R, kb, bk, passes):
    """Left-looking classical Gram-Schmidt on columns kb..kb+bk-1 (passes 1 or 2)."""
    _chk(lib().cqro_cgs_panel(Q.shape[0], kb, bk, passes, _p(Q), _ld(Q), _p(R), _ld(R)),
         "cgs_panel")


def factor(Q, R, n, b, t0=0, t1=-1, tau=0.7071067811865476, reorth_block=False, panel="icgs"):
    """a3-a5: PBMGS panels t0..t1-1 in place on Q (M x N) and R (N x N). Returns #reorth.
    reorth_block: project each panel once more on all computed columns before its ICGS.
    panel: "icgs" (the paper's), "mgs" (no reorthogonalisation test), "cgs1" / "cgs2"
    (left-looking classical Gram-Schmidt, one / two passes)."""
    nre = C.c_int64(0)
    rc = lib().cqro_factor3(Q.shape[0], Q.shape[1], n, b, t0, t1, tau, int(bool(reorth_block)),
                            PANELS[panel], _p(Q), _ld(Q), _p(R), _ld(R), C.byref(nre))
    _chk(rc, "factor")
    return nre.value


def inject(g, tiles, mask, Q, R):
    """a6: erase node tiles (list of (i, j)); mask is a uint8 (grid_rows x grid_cols) array."""
    flat = (C.c_int * max(2 * len(tiles), 1))(*[v for t in tiles for v in t])
    _chk(lib().cqro_inject(C.byref(g), flat, len(tiles),
                           mask.ctypes.data_as(C.POINTER(C.c_uint8)), _p(Q), _ld(Q), _p(R),
                           _ld(R)), "inject")


def recover(g, Gt, Gh, mask, Q, R, cap=4096):
    """a7: decode every erased tile; returns (decode-set list, #tiles recovered)."""
    sets = (C.c_int * cap)()
    ln = C.c_int(0)
    nrec = C.c_int(0)
    rc = lib().cqro_recover(C.byref(g), _p(_rowmajor(Gt)), _p(_rowmajor(Gh)),
                            mask.ctypes.data_as(C.POINTER(C.c_uint8)), _p(Q), _ld(Q), _p(R),
                            _ld(R), sets, cap, C.byref(ln), C.byref(nrec))
    _chk(rc, "recover")
    return [int(sets[i]) for i in range(ln.value)], nrec.value


def invert_small(G):
    G = np.ascontiguousarray(G, dtype=np.float64)
    k = G.shape[0]
    out = np.zeros_like(G)
    _chk(lib().cqro_invert_small(k, _p(G.ravel()), out.ctypes.data_as(C.POINTER(C.c_double))),
         "invert")
    return out


def build_G0(g, Gt):
    G0 = np.zeros((g.m_pad, g.m_pad), order="F")
    lib().cqro_build_G0(C.byref(g), _p(_rowmajor(Gt)), _p(G0), _ld(G0))
    return G0


def post_orth(g, Gt, Z, dense=False):
    """a8: W = G_0 Z for Z m_pad x k (dense: explicit G_0; else the block formula)."""
    Z = np.asfortranarray(Z, dtype=np.float64)
    if Z.ndim == 1:
        Z = Z.reshape(-1, 1, order="F")
    W = np.zeros_like(Z, order="F")
    fn = lib().cqro_post_orth_dense if dense else lib().cqro_post_orth_block
    _chk(fn(C.byref(g), _p(_rowmajor(Gt)), _p(Z), _ld(Z), Z.shape[1], _p(W), _ld(W)), "post_orth")
    return W


def post_orth_projected(g, Gt, Q1, Q2):
    """a8, drift-robust reading: W = G_0^{-1} (Q_1 + G^T Q_2), G = G~ (x) I_mb.  With
    G_0^2 = I + G^T G (G_0 symmetric, Theorem G_0) this is G_0 applied to the orthogonal
    projection of [Q_1; Q_2] onto the range {[x; G x]} of the encoding, so it equals G_0 Q_1
    whenever Q_2 = G Q_1 (the checksum-preservation Lemma); in floating point, where Q_2
    drifts from G Q_1 by delta, its loss of orthogonality is of order delta^2 instead of
    delta.  Plain definition: the dense G_0 and a library solve.  Q1 m_pad x k, Q2 c x k."""
    G0 = build_G0(g, Gt)
    G = np.kron(np.asarray(Gt, dtype=np.float64), np.eye(g.mb))
    return np.asfortranarray(np.linalg.solve(G0, np.asarray(Q1) + G.T @ np.asarray(Q2)))


def back_substitute(R, rhs):
    x = np.asfortranarray(rhs, dtype=np.float64).copy(order="F")
    if x.ndim == 1:
        x = x.reshape(-1, 1, order="F")
    R = np.asfortranarray(R)
    lib().cqro_back_substitute(x.shape[0], _p(R), _ld(R), _p(x), _ld(x), x.shape[1])
    return x


def solve_square(Qo, R, yo):
    """a9 (square): x from R x = Qo^T yo, Qo = G_0 Q_1, yo = G_0 y."""
    Qo = np.asfortranarray(Qo)
    yo = np.asfortranarray(yo if yo.ndim == 2 else yo.reshape(-1, 1), dtype=np.float64)
    n = Qo.shape[1]
    R = np.asfortranarray(R)
    x = np.zeros((n, yo.shape[1]), order="F")
    _chk(lib().cqro_solve_square(Qo.shape[0], n, _p(Qo), _ld(Qo), _p(R), _ld(R), _p(yo),
                                 _ld(yo), yo.shape[1], _p(x), _ld(x)), "solve_square")
    return x


def solve_ls(Q1, R, y):
    """a9 (tall): least squares through A = Q_1 R."""
    Q1 = np.asfortranarray(Q1)
    y = np.asfortranarray(y if y.ndim == 2 else y.reshape(-1, 1), dtype=np.float64)
    n = Q1.shape[1]
    R = np.asfortranarray(R)
    x = np.zeros((n, y.shape[1]), order="F")
    _chk(lib().cqro_solve_ls(Q1.shape[0], n, _p(Q1), _ld(Q1), _p(R), _ld(R), _p(y), _ld(y),
                             y.shape[1], _p(x), _ld(x)), "solve_ls")
    return x


def run(A, p_r, p_c, f, b, seed=1, erasures=None, protect_r=True, gdist=0, tau=0.7071067811865476,
        y=None, Gt=None, Gh=None, keep_states=False, reorth_block=False, panel="icgs"):
    """The whole hot path on the CPU: generator, encode, PBMGS with erasures injected at the
    start of the listed panels (dict panel -> list of (i, j)) and recovered, post-orth, solve.

    Returns a dict with the generator, the encoded matrix, the final coded Q and R, the
    post-orthogonalised Q, the decode sets, the reorth count and, when y is given, x.
    """
    A = np.asfortranarray(A, dtype=np.float64)
    m, n = A.shape
    g = geom(m, n, p_r, p_c, f, protect_r)
    if Gt is None:
        Gt, Gh = generator(f, p_r, p_c, seed, gdist)
    At = encode(g, Gt, Gh, A)
    Q = At.copy(order="F")
    R = np.zeros((g.N, g.N), order="F")
    T = (n + b - 1) // b
    mask = np.zeros((g.grid_rows, g.grid_cols), dtype=np.uint8)
    sets = []
    nrec = 0
    nre = 0
    states = []
    erasures = erasures or {}
    for t in range(T):
        if t in erasures and erasures[t]:
            inject(g, erasures[t], mask, Q, R)
            s, k = recover(g, Gt, Gh, mask, Q, R)
            sets += s
            nrec += k
        nre += factor(Q, R, n, b, t, t + 1, tau, reorth_block, panel)
        if keep_states:
            states.append((Q.copy(order="F"), R.copy(order="F")))
    out = dict(geom=g, Gt=Gt, Gh=Gh, At=At, Q=Q, R=R, sets=sets, n_recovered=nrec,
               n_reorth=nre, states=states)
    if f > 0:
        Qo = post_orth(g, Gt, Q[: g.m_pad, :n])
    else:
        Qo = Q[: g.m_pad, :n].copy(order="F")
    out["Qo"] = Qo
    if y is not None:
        y = np.asarray(y, dtype=np.float64)
        y2 = y.reshape(m, -1)
        yp = np.zeros((g.m_pad, y2.shape[1]), order="F")
        yp[:m] = y2
        if m == n and g.m_pad == m:
            yo = post_orth(g, Gt, yp) if f > 0 else yp
            out["yo"] = yo
            out["x"] = solve_square(Qo, R[:n, :n], yo)
        else:
            out["x"] = solve_ls(Q[: g.m_pad, :n], R[:n, :n], yp)
    return out


def mds_stats(G):
    """E1 (Theorem prob_det and the comparison after it, Section 4.2): the least |det S| and
    the largest 2-norm condition number over every square submatrix S of G, per size k
    (index k) and overall (index 0).  Brute force over all row and column k-subsets with
    numpy's LU determinant and SVD singular values; a condition number of 1/eps or more
    (eps = 2^-52) is reported as +inf.  Small sizes only."""
    import itertools
    G = np.asarray(G, dtype=np.float64)
    f, p = G.shape
    mind = [np.inf] * (f + 1)
    maxc = [0.0] * (f + 1)
    for k in range(1, f + 1):
        for rows in itertools.combinations(range(f), k):
            sub = G[list(rows), :]
            for cols in itertools.combinations(range(p), k):
                S = sub[:, list(cols)]
                d = abs(np.linalg.det(S))
                sv = np.linalg.svd(S, compute_uv=False)
                # numerically singular (sigma_min <= eps sigma_max, eps = 2^-52): +inf
                c = np.inf if sv[-1] <= np.finfo(np.float64).eps * sv[0] else sv[0] / sv[-1]
                mind[k] = min(mind[k], d)
                maxc[k] = max(maxc[k], c)
    mind[0] = min(mind[1:])
    maxc[0] = max(maxc[1:])
    return mind, maxc


# ------------------------------------------------------------------ in-node checksum storage
def in_node_checks(P, L, f):
    """Theorem in_node_opt with equality: K = f L / P + f ceil(f L / ((P - f) P)) checksum blocks
    (P nodes, L data blocks, P | L)."""
    return f * L // P + f * (-(-(f * L) // ((P - f) * P)))


def in_node_hosts(K, P):
    """Load-balanced in-node checksum distribution (Definition innode_distr): checksum block k
    goes to node (k P) // K when K <= P (spread over the nodes), else to node k mod P; either
    way K - P floor(K/P) nodes host ceil(K/P) blocks and the others floor(K/P)."""
    return [(k * P) // K if K <= P else k % P for k in range(K)]


def node_tiles(p_r, p_c, K, protect_r, i, j):
    """Every tile (I, J) of the encoded grid hosted by node (i, j) of the p_r x p_c node grid:
    data tile (i, j), the vertical checksum tiles of column j hosted by row node i, the
    horizontal checksum tiles of row i hosted by column node j, and the checksum-of-checksum
    tiles hosted by (i, j)."""
    hv = in_node_hosts(K, p_r)
    hh = in_node_hosts(K, p_c) if protect_r else []
    rows = [i] + [p_r + k for k in range(K) if hv[k] == i]
    cols = [j] + [p_c + l for l in range(len(hh)) if hh[l] == j]
    return [(I, J) for I in rows for J in cols]


def run_in_node(A, p, f, b, seed=1, node_failures=None, protect_r=True, tau=0.7071067811865476,
                y=None):
    """The coded QR with in-node checksum storage (Section 5, Construction in_node and
    Remark alt_in_node; the Q generator of Construction in_node_qr): K checksum blocks per code
    on a p x p node grid, the structured K x p generator, node failures {panel t: [(i, j)]}
    erasing every tile their node hosts.  Returns oracle.run's dict plus K."""
    K = in_node_checks(p, p, f)
    er = {}
    for t, nodes in (node_failures or {}).items():
        tiles = []
        for (i, j) in nodes:
            tiles += node_tiles(p, p, K, protect_r, i, j)
        er[t] = tiles
    out = run(A, p, p, K, b, seed=seed, erasures=er, protect_r=protect_r, tau=tau, y=y)
    out["K"] = K
    return out
