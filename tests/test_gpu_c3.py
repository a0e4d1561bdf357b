"""The largest single-GPU workload at full size against the FP64 oracle, through the C ABI
(needs a GB300): A 16384 x 16384 = U diag(sigma) V^T with kappa 1e4, grid 16 x 16, f = 4,
b = 256 (coded 20480 x 20480), four simultaneous erasures, FP32 storage with tensor-core
trailing updates and block reorthogonalisation.

The oracle runs encode, panel 0, the loss and recovery of the four tiles, and panel 1 (about
half a minute on the host cores); the whole factorisation (64 panels) would take it about
twenty minutes.  So:
  - the timed step itself (erasures at panel 50, as bench.py runs it) is compared with the
    oracle on panel 0's Q columns and R rows, bit for bit on the decode index sets, and on
    the properties that hold at any size (backward error, orthogonality before and after
    post-orthogonalisation, checksum drift, solve residual);
  - the same four tiles lost at the start of panel 1 are compared on the whole coded Q and
    on R's first two panels of rows, for every tensor-core precision.

Tolerances (column j of the coded matrix, a_j its encoded column, u_p the unit roundoff of
the products of the precision, u the FP32 unit roundoff, M = 20480 rows, b = 256):
  - a trailing update adds to column j at most 2 u_p |Qbar|_F |Rbar_j| <= 2 sqrt(b) u_p |a_j|
    (both operands rounded to the product type), and its FP32 accumulation over K terms about
    sqrt(K) u |a_j|; two updates and one block reorthogonalisation reach the columns right
    of panel 1, so their 2-norm error is below (6 sqrt(b) u_p + 4 sqrt(M) u) |a_j|;
  - a normalised column of panels 0 and 1 carries that error divided by r_jj, i.e. times
    rho_j = |a_j| / r_jj, plus the panel's own FP32 rounding (b u relative, 4 b u in 2-norm);
  - an entry R_kj of the first 512 rows carries at most (4 u_p + 4 sqrt(M) u) |a_j|.
"""
import numpy as np
import pytest

import bench
from oracle import oracle as O
from paper_2311_11943_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2311_11943_gb300 import binding as B  # noqa: E402

U32 = np.finfo(np.float32).eps / 2
U3X = 8 * U32
U_PROD = {"3xtf32": U3X, "tf32": 2.0 ** -11, "bf16": 2.0 ** -8, "bf16x3": 2.0 ** -16}
CFG = bench.CONFIGS["c3"]


@pytest.fixture(scope="module")
def c3():
    """The seeded input (device FP32 and its FP64 host copy), and the oracle's state after
    panel 0 and after the early-recovery schedule (tiles lost at the start of panel 1)."""
    m, n, p, f, b = (CFG[k] for k in ("m", "n", "p_r", "f", "b"))
    A32 = synth.kappa_matrix_torch(m, n, CFG["kappa"], CFG["seed"])
    A_np = A32.double().cpu().numpy()
    g = O.geom(m, n, p, p, f)
    Gt, Gh = O.generator(f, p, p, CFG["seed"])
    Q = O.encode(g, Gt, Gh, A_np)
    anorm = np.linalg.norm(Q, axis=0)
    R = np.zeros((g.N, g.N), order="F")
    O.factor(Q, R, n, b, 0, 1, reorth_block=True)
    snap0 = (Q[:, :b].copy(), R[:b, :].copy())
    tiles = [(i, j) for (_, i, j) in bench.erasure_plan(CFG)]
    mask = np.zeros((g.grid_rows, g.grid_cols), np.uint8)
    O.inject(g, tiles, mask, Q, R)
    sets, nrec = O.recover(g, Gt, Gh, mask, Q, R)
    O.factor(Q, R, n, b, 1, 2, reorth_block=True)
    dev = torch.device("cuda")
    out = dict(A32=A32, A_np=A_np, g=g, Gt=Gt, Gh=Gh, anorm=anorm, snap0=snap0, tiles=tiles,
               sets=sets, nrec=nrec, Q2p=torch.from_numpy(Q).to(dev), R2p=R[:2 * b, :].copy())
    del Q, R
    return out


def _col_err(Qg, Qo):
    """2-norm of each column of Qg - Qo on the device (both M x k, Qg FP32, Qo FP64)."""
    return torch.linalg.norm(Qg.double() - Qo, dim=0).cpu().numpy()


@pytest.mark.parametrize("mode", ["3xtf32", "tf32", "bf16", "bf16x3"])
def test_c3_four_tiles_recovered_at_panel_1_full_size(c3, mode):
    m, n, p, f, b = (CFG[k] for k in ("m", "n", "p_r", "f", "b"))
    g = c3["g"]
    q = B.CodedQR(m, n, p, p, f, b, dtype="f32", mma=mode, seed=CFG["seed"], reorth_block=True,
                  stream=torch.cuda.current_stream())
    q.encode(c3["A32"])
    q.factor(0, 1)
    q.inject(c3["tiles"])
    assert q.recover() == c3["nrec"]
    q.factor(1, 2)
    torch.cuda.synchronize()
    assert q.sync_status() == 0
    assert q.decode_sets() == c3["sets"]          # bit for bit, at full size
    Gt, Gh = q.generator()
    assert np.array_equal(Gt, c3["Gt"]) and np.array_equal(Gh, c3["Gh"])
    Qc, Rc = q.factors()
    err = _col_err(Qc, c3["Q2p"])
    Rg = Rc[:2 * b, :].double().cpu().numpy()
    q.close()

    up = U_PROD[mode]
    an = c3["anorm"]
    Ro = c3["R2p"]
    rho = an[:2 * b] / np.abs(np.diag(Ro[:, :2 * b]))
    upd = 6 * np.sqrt(b) * up + 4 * np.sqrt(g.M) * U32
    tol_cols = np.empty(g.N)
    tol_cols[:2 * b] = upd * an[:2 * b] * rho + 4 * b * U32
    tol_cols[2 * b:] = upd * an[2 * b:]
    worst = np.argmax(err / tol_cols)
    assert (err < tol_cols).all(), (mode, int(worst), err[worst], tol_cols[worst])
    tol_r = (4 * up + 4 * np.sqrt(g.M) * U32) * an[None, :]
    dr = np.abs(Rg - Ro)
    assert (dr <= tol_r).all(), (mode, dr.max(), np.unravel_index(np.argmax(dr / tol_r), dr.shape))
    print("c3 early recovery %s: max col err %.3g (tol %.3g), max R err %.3g"
          % (mode, err.max(), tol_cols[np.argmax(err)], dr.max()))


def test_c3_bench_step_full_size(c3):
    # the timed step exactly as bench.py runs it on the current stream: 3xTF32, block
    # reorthogonalisation, the factor segments around the four-tile erasure at panel 50, the
    # in-handle post-orthogonalisation (projected form, the FP32 default) and the solve
    m, n, p, f, b, kap = (CFG[k] for k in ("m", "n", "p_r", "f", "b", "kappa"))
    g = c3["g"]
    M = g.M
    plan = bench.erasure_plan(CFG)
    y = synth.rhs(m, 1, CFG["seed"])
    q = B.CodedQR(m, n, p, p, f, b, dtype="f32", mma="3xtf32", seed=CFG["seed"],
                  stream=torch.cuda.current_stream(), reorth_block=True)
    Ad = c3["A32"]
    yd = B.colmajor_empty(m, 1, torch.float32)
    yd.copy_(torch.from_numpy(y))
    xd = B.colmajor_empty(n, 1, torch.float32)
    bench.coded_factor(q, Ad, plan)
    Qc, Rc = q.factors()
    dev = Qc.device
    Qp = Qc[:, :b].double().cpu().numpy()
    Rp = Rc[:b, :].double().cpu().numpy()
    # properties at full size, in FP64 on the device, before post-orthogonalisation
    A64 = torch.from_numpy(c3["A_np"]).to(dev)
    back = (torch.linalg.norm(A64 - Qc[:m, :n].double() @ Rc[:n, :n].double()) /
            torch.linalg.norm(A64)).item()
    Qt = Qc[:M, :n].double()
    eye = torch.eye(n, dtype=torch.float64, device=dev)
    orth_coded = (Qt.T @ Qt - eye).abs().max().item()
    Gv = torch.kron(torch.from_numpy(c3["Gt"]), torch.eye(g.mb, dtype=torch.float64)).to(dev)
    drift = (Qt[m:M] - Gv @ Qt[:m]).abs().max().item()
    del Qt, Gv
    q.post_orth()
    q.solve(yd, xd)
    Qo = Qc[:m, :n].double()              # the post-orthogonalised Q_1, written in place
    orth = (Qo.T @ Qo - eye).abs().max().item()
    del Qo
    torch.cuda.synchronize()
    assert q.sync_status() == 0
    sets = q.decode_sets()
    q.close()
    x = xd.double()
    resid = (torch.linalg.norm(A64 @ x - torch.from_numpy(y).to(dev)) /
             np.linalg.norm(y)).item()
    del A64
    print("c3 step: back %.3g orth_coded %.3g orth %.3g drift %.3g resid %.3g"
          % (back, orth_coded, orth, drift, resid))
    # the FP32 targets at kappa <= 1e4
    assert back <= 1e-5 and orth_coded <= 1e-5 and orth <= 1e-5, (back, orth_coded, orth)
    # the drift of Q_2 from G_v Q_1: the updates of systematic and checksum rows round
    # independently (3xTF32 products), and normalising by r_jj >= sigma_min magnifies that
    # by at most |a_j| / sigma_min <= kappa max_j |a_j| (|A|_2 = 1)
    assert drift < 10 * U3X * kap * c3["anorm"].max(), drift
    assert resid <= 1e-5 * kap, resid

    # decode index sets: the oracle's plan logic on a grid of the same shape (any tile size)
    er = {}
    for (t, i, j) in plan:
        er.setdefault(t, []).append((i, j))
    gs = O.geom(2 * p, p, p, p, f)
    Qs = O.encode(gs, c3["Gt"], c3["Gh"], synth.gaussian(2 * p, p, 1))
    Rs = np.zeros((gs.N, gs.N), order="F")
    ref_sets = []
    for t in sorted(er):
        mask = np.zeros((gs.grid_rows, gs.grid_cols), np.uint8)
        O.inject(gs, er[t], mask, Qs, Rs)
        ref_sets += O.recover(gs, c3["Gt"], c3["Gh"], mask, Qs, Rs)[0]
    assert sets == ref_sets

    # panel 0 element by element: FP32 rounding of the panel alone (no product reaches it);
    # R's first rows also receive the later block reorthogonalisations' corrections, of the
    # size of the 3xTF32 rounding of the columns they touch
    Q0, R0 = c3["snap0"]
    assert np.abs(Qp - Q0).max() < 64 * U3X
    tol_r = (4 * U3X + 4 * np.sqrt(M) * U32) * c3["anorm"][None, :] * 8
    keep = np.ones(g.N, bool)
    for (_, i, j) in plan:
        if i == 0:
            keep[j * g.nb:(j + 1) * g.nb] = False
    assert (np.abs(Rp - R0)[:, keep] <= tol_r[:, keep]).all()
