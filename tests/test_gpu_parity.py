"""GPU path vs the FP64 oracle, element by element, through the C ABI (needs a GB300).

Tolerances: Gram-Schmidt factors carry a forward error of order n u kappa(A), u the unit
roundoff of the storage precision (8 u for 3xTF32 products, whose hi/lo split leaves about
2^-21 per product); the decode adds kappa(G^) u per recovered tile.  Integer results (decode index sets) and the FP64 generator
(computed with explicitly rounded operations on both sides) are compared bit for bit.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_11943_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2311_11943_gb300 import binding as B  # noqa: E402

U64 = np.finfo(np.float64).eps / 2
U32 = np.finfo(np.float32).eps / 2


def to_dev(A, tdtype):
    A = np.asarray(A)
    if A.ndim == 1:
        A = A.reshape(-1, 1)
    d = B.colmajor_empty(A.shape[0], A.shape[1], tdtype)
    d.copy_(torch.from_numpy(np.ascontiguousarray(A)))
    return d


def to_np(t):
    return np.asfortranarray(t.detach().double().cpu().numpy())


def gpu_run(A, p_r, p_c, f, b, seed, erasures=None, y=None, dtype="f64", mma="simt",
            protect_r=True, tau=0.0, workspace=None):
    m, n = A.shape
    td = torch.float64 if dtype == "f64" else torch.float32
    k = 1 if y is None else y.shape[1]
    q = B.CodedQR(m, n, p_r, p_c, f, b, dtype=dtype, mma=mma, protect_r=protect_r, seed=seed,
                  nrhs_max=k, tau=tau, workspace=workspace)
    Ad = to_dev(A, td)
    q.encode(Ad)
    erasures = erasures or {}
    T = q.geo["panels"]
    for t in range(T):
        if erasures.get(t):
            q.inject(erasures[t])
            q.recover()
        q.factor(t, t + 1)
    Qc, Rc = q.factors()
    out = dict(Q=to_np(Qc), R=to_np(Rc), sets=q.decode_sets(), geo=q.geo)
    Qo = B.colmajor_empty(q.geo["m_pad"], n, td)
    q.post_orth(Qo)
    out["Qo"] = to_np(Qo)
    if y is not None and m == n and q.geo["m_pad"] == m:
        x = B.colmajor_empty(n, k, td)
        q.solve(to_dev(y, td), x)
        out["x"] = to_np(x)
    torch.cuda.synchronize()
    out["status"] = q.sync_status()
    out["stats"] = q.stats()
    out["Gt"], out["Gh"] = q.generator()
    q.close()
    return out


def rel(a, b):
    return np.abs(a - b).max() / max(1.0, np.abs(b).max())


# ----------------------------------------------------------------- a1 / a2
@pytest.mark.parametrize("f,p_r,p_c,gdist", [(1, 4, 4, 0), (2, 8, 8, 0), (4, 16, 16, 0),
                                             (3, 6, 8, 1), (6, 12, 12, 0)])
def test_generator_and_encode(f, p_r, p_c, gdist):
    # f = 6: the encode kernels' generic path (checksum counts above 4)
    m, n = 4 * p_r + 3, 2 * p_c
    A = synth.gaussian(m, n, 11)
    q = B.CodedQR(m, n, p_r, p_c, f, 4, dtype="f64", gdist=gdist, seed=1234 + f)
    q.encode(to_dev(A, torch.float64))
    Gt, Gh = q.generator()
    Gt_o, Gh_o = O.generator(f, p_r, p_c, 1234 + f, gdist)
    if gdist == 0:
        assert np.array_equal(Gt, Gt_o) and np.array_equal(Gh, Gh_o)  # bit-exact
    else:
        assert np.abs(Gt - Gt_o).max() < 1e-13 and np.abs(Gh - Gh_o).max() < 1e-13
    Qc, _ = q.factors()
    g = O.geom(m, n, p_r, p_c, f)
    At = O.encode(g, Gt_o, Gh_o, A)
    assert rel(to_np(Qc), At) < 8 * p_r * U64
    q.close()


# ----------------------------------------------------------------- the whole path, C1 shape
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_c1_full_path_parity(dtype):
    # 256 x 256 N(0,1), grid 4 x 4, f = 1, b = 32, one node erased at the start of panel 3
    A = synth.gaussian(256, 256, 1)
    y = synth.rhs(256, 2, 1)
    er = {3: synth.random_erasures(5, 5, 1, 1, seed=1)}
    ref = O.run(A, 4, 4, 1, 32, seed=1, erasures=er, y=y)
    got = gpu_run(A, 4, 4, 1, 32, seed=1, erasures=er, y=y, dtype=dtype)
    assert got["status"] == 0
    assert got["sets"] == ref["sets"]
    assert got["stats"]["n_recovered"] == ref["n_recovered"]
    u = U64 if dtype == "f64" else U32
    kappa = np.linalg.cond(A)
    n = 256
    tol = n * u * kappa
    g = ref["geom"]
    assert rel(got["Q"][: g.M, :n], ref["Q"][:, :n]) < tol
    assert rel(got["R"], ref["R"]) < tol
    assert rel(got["Qo"], ref["Qo"]) < tol
    # x is kappa times more sensitive than the factors, but both sides solve with the same
    # (nearly equal) R, so their difference stays within the factors' tolerance
    assert rel(got["x"], ref["x"]) < tol
    Qo = got["Qo"]
    assert np.abs(Qo.T @ Qo - np.eye(n)).max() < 8 * n * u * kappa


def test_reorth_count_matches_oracle():
    A = synth.gaussian(128, 128, 5)
    ref = O.run(A, 4, 4, 1, 32, seed=3)
    got = gpu_run(A, 4, 4, 1, 32, seed=3)
    # the criterion v_j < tau^2 eta_j is met at the same columns unless a value sits within
    # rounding of the threshold; allow a one-column difference
    assert abs(got["stats"]["n_reorth"] - ref["n_reorth"]) <= 1


def test_ragged_tall_shapes_and_every_grid_column():
    # m not a multiple of p_r (zero padding), last panel narrower than b, erasures in
    # systematic, checksum-row, checksum-column and corner tiles
    A = synth.gaussian(203, 96, 7)
    er = {1: [(0, 0), (9, 1)], 3: [(8, 5), (2, 4)]}
    ref = O.run(A, 8, 4, 2, 20, seed=9, erasures=er)
    got = gpu_run(A, 8, 4, 2, 20, seed=9, erasures=er)
    assert got["status"] == 0
    assert got["sets"] == ref["sets"]
    g = ref["geom"]
    tol = 96 * U64 * np.linalg.cond(A) * 10
    assert rel(got["Q"][: g.M, :96], ref["Q"][:, :96]) < tol
    assert rel(got["R"], ref["R"]) < tol
    assert rel(got["Qo"], ref["Qo"]) < tol
    Q1 = got["Q"][:203, :96]
    assert np.abs(A - Q1 @ got["R"][:96, :96]).max() < tol * np.abs(A).max()


def test_uncoded_f0_is_plain_bmgs():
    A = synth.gaussian(96, 64, 2)
    ref = O.run(A, 4, 4, 0, 16, seed=1)
    got = gpu_run(A, 4, 4, 0, 16, seed=1)
    assert rel(got["R"], ref["R"]) < 64 * U64 * np.linalg.cond(A)
    Qh, Rh = np.linalg.qr(A)
    assert rel(np.abs(got["R"][:64, :64]), np.abs(Rh)) < 1e-12


def test_recovered_gpu_run_equals_fault_free_gpu_run():
    A = synth.gaussian(192, 192, 4)
    y = synth.rhs(192, 1, 4)
    er = {t: synth.reverse_diagonal(6, 2, shift=t) for t in range(1, 6)}
    clean = gpu_run(A, 6, 6, 2, 32, seed=2, y=y)
    hit = gpu_run(A, 6, 6, 2, 32, seed=2, y=y, erasures=er)
    assert hit["stats"]["n_recovered"] >= 5 * 12
    tol = 1e-9
    for k in ("R", "Qo", "x"):
        assert rel(hit[k], clean[k]) < tol


def test_unrecoverable_pattern_leaves_state_untouched():
    A = synth.gaussian(64, 64, 1)
    q = B.CodedQR(64, 64, 4, 4, 1, 16, dtype="f64", seed=1)
    q.encode(to_dev(A, torch.float64))
    q.factor(0, 2)
    q.inject([(0, 1), (2, 1)])
    st, n = B.coded_qr_recover(q.h)
    assert st == B.CQR_EUNRECOVERABLE and n == 0
    assert B.coded_qr_factor(q.h, 2, -1) == B.CQR_ESTATE     # erasures still pending
    assert q.decode_sets() == []
    q.close()


def test_state_machine_errors():
    q = B.CodedQR(64, 64, 4, 4, 1, 16, dtype="f64", seed=1)
    assert B.coded_qr_factor(q.h, 0, -1) == B.CQR_ESTATE          # before encode
    q.encode(to_dev(synth.gaussian(64, 64, 1), torch.float64))
    assert B.coded_qr_factor(q.h, 1, 2) == B.CQR_ESTATE           # must resume at panel 0
    assert B.coded_qr_post_orth(q.h, 0, 0, 0, 0, 0, 0, 0) == B.CQR_ESTATE  # not factored
    assert B.coded_qr_inject_erasure(q.h, [(9, 0)]) == B.CQR_EINVAL       # outside the grid
    q.factor()
    assert q.sync_status() == 0
    q.close()


def test_breakdown_is_reported_on_the_device():
    A = synth.gaussian(64, 64, 3)
    A[:, 10] = 0.0
    q = B.CodedQR(64, 64, 4, 4, 1, 16, dtype="f64", seed=1)
    q.encode(to_dev(A, torch.float64))
    q.factor()
    assert q.sync_status() == B.CQR_EBREAKDOWN
    q.close()


def test_run_with_host_buffers_matches_device_path_bitwise():
    A = synth.gaussian(256, 256, 8)
    y = synth.rhs(256, 1, 8)
    plan = [(2, 1, 1), (5, 4, 0)]
    q = B.CodedQR(256, 256, 4, 4, 1, 32, dtype="f64", seed=5)
    x_host = np.zeros((256, 1), order="F")
    q.run(np.asfortranarray(A), np.asfortranarray(y), x_host, plan=plan, host=True)
    Ad, yd = to_dev(A, torch.float64), to_dev(y, torch.float64)
    xd = B.colmajor_empty(256, 1, torch.float64)
    q.run(Ad, yd, xd, plan=plan)
    assert np.array_equal(x_host, to_np(xd))
    ref = O.run(A, 4, 4, 1, 32, seed=5, y=y, erasures={2: [(1, 1)], 5: [(4, 0)]})
    assert rel(x_host, ref["x"]) < 256 * U64 * np.linalg.cond(A) ** 2
    q.close()


def test_caller_workspace_gives_identical_results():
    A = synth.gaussian(128, 128, 6)
    a = gpu_run(A, 4, 4, 1, 16, seed=4)
    b = gpu_run(A, 4, 4, 1, 16, seed=4, workspace="torch")
    assert np.array_equal(a["R"], b["R"]) and np.array_equal(a["Qo"], b["Qo"])


# ----------------------------------------------------------------- C2 shape at full size
def test_c2_fp64_full_size_sampled():
    # 4096 x 4096, kappa = 1e2, grid 8 x 8, f = 2, b = 128, two nodes erased at two panels.
    n, p, f, b = 4096, 8, 2, 128
    A = synth.kappa_matrix(n, n, 1e2, seed=2)
    T = n // b
    ts = synth.random_panels(T, 2, seed=2)
    er = {t: synth.random_erasures(p + f, p + f, f, 1, seed=2 + t) for t in ts}
    got = gpu_run(A, p, p, f, b, seed=2, erasures=er)
    assert got["status"] == 0
    g = O.geom(n, n, p, p, f)
    # sampled outputs the oracle computes exactly: the first panel's R rows and Q columns
    Gt, Gh = O.generator(f, p, p, 2)
    assert np.array_equal(Gt, got["Gt"])
    Q = O.encode(g, Gt, Gh, A)
    R = np.zeros((g.N, g.N), order="F")
    O.factor(Q, R, n, b, 0, 1)
    tol = n * U64 * 1e2
    assert rel(got["R"][:b, :], R[:b, :]) < tol
    assert rel(got["Q"][: g.M, :b], Q[:, :b]) < tol
    # decode index sets: the oracle's plan logic on the same grid (any tile size)
    gs = O.geom(2 * p, p, p, p, f)
    Gs, Ghs = O.generator(f, p, p, 2)
    Qs = O.encode(gs, Gs, Ghs, synth.gaussian(2 * p, p, 1))
    Rs = np.zeros((gs.N, gs.N), order="F")
    sets = []
    for t in ts:
        mask = np.zeros((gs.grid_rows, gs.grid_cols), np.uint8)
        O.inject(gs, er[t], mask, Qs, Rs)
        sets += O.recover(gs, Gs, Ghs, mask, Qs, Rs)[0]
    assert got["sets"] == sets
    # properties that hold at any size
    Q1, R1 = got["Q"][:n, :n], got["R"][:n, :n]
    assert np.linalg.norm(A - Q1 @ R1) / np.linalg.norm(A) < 1e-12
    Qo = got["Qo"]
    assert np.abs(Qo.T @ Qo - np.eye(n)).max() < 1e-12
    Gv = np.kron(got["Gt"], np.eye(g.mb))
    assert np.abs(got["Q"][n: g.M, :n] - Gv @ Q1).max() < 1e-12
    Ghk = np.kron(got["Gh"], np.eye(g.nb))
    assert np.abs(got["R"][:n, n:] - R1 @ Ghk).max() < 1e-12 * np.abs(R1).max()


# ----------------------------------------------------------------- the timed C2 step at full size
def test_c2_bench_step_full_size():
    # The C2 step exactly as bench.py times it: 4096 x 4096 U diag(sigma) V^T with kappa 1e2,
    # grid 8 x 8, f = 2, b = 128, FP32 storage, 3xTF32 trailing updates, block
    # reorthogonalisation, factor segments between the two seeded erasure panels, Q_1
    # post-orthogonalised inside the handle, then the solve; on the current stream.
    import bench
    cfg = bench.CONFIGS["c2"]
    m, n, p, f, b, kap = (cfg[k] for k in ("m", "n", "p_r", "f", "b", "kappa"))
    A, y = bench.make_inputs(cfg)
    plan = bench.erasure_plan(cfg)
    q = B.CodedQR(m, n, p, p, f, b, dtype="f32", mma="3xtf32", seed=cfg["seed"],
                  stream=torch.cuda.current_stream(), reorth_block=True)
    Ad, yd = to_dev(A, torch.float32), to_dev(y, torch.float32)
    xd = B.colmajor_empty(n, 1, torch.float32)
    bench.coded_factor(q, Ad, plan)
    Qc, Rc = q.factors()
    Qt, R = Qc.double(), Rc.double()      # the coded factors before post-orthogonalisation
    q.post_orth()
    q.solve(yd, xd)
    Qo = Qc[:m, :n].double()              # G_0 Q_1, written over Q_1 by the step
    x = to_np(xd)
    torch.cuda.synchronize()
    assert q.sync_status() == 0
    sets = q.decode_sets()
    Gt, Gh = q.generator()
    q.close()
    g = O.geom(m, n, p, p, f)
    M = g.M

    # the FP32 accuracy target (kappa <= 1e4): backward error and orthogonality at most 1e-5
    dev = Qt.device
    A64 = torch.from_numpy(A).to(dev)
    eye = torch.eye(n, dtype=torch.float64, device=dev)
    back = (torch.linalg.norm(A64 - Qt[:m, :n] @ R[:n, :n]) / torch.linalg.norm(A64)).item()
    orth_coded = (Qt[:, :n].T @ Qt[:, :n] - eye).abs().max().item()
    orth = (Qo.T @ Qo - eye).abs().max().item()
    assert back <= 1e-5 and orth_coded <= 1e-5 and orth <= 1e-5, (back, orth_coded, orth)

    # generator bit for bit; decode index sets from the oracle's plan logic (any tile size)
    Gto, Gho = O.generator(f, p, p, cfg["seed"])
    assert np.array_equal(Gt, Gto) and np.array_equal(Gh, Gho)
    er = {}
    for (t, i, j) in plan:
        er.setdefault(t, []).append((i, j))
    gs = O.geom(2 * p, p, p, p, f)
    Qs = O.encode(gs, Gto, Gho, synth.gaussian(2 * p, p, 1))
    Rs = np.zeros((gs.N, gs.N), order="F")
    ref_sets = []
    for t in sorted(er):
        mask = np.zeros((gs.grid_rows, gs.grid_cols), np.uint8)
        O.inject(gs, er[t], mask, Qs, Rs)
        ref_sets += O.recover(gs, Gto, Gho, mask, Qs, Rs)[0]
    assert sets == ref_sets

    # the whole oracle run with the same erasure plan (about ten seconds on the host cores),
    # compared column by column.  A trailing update adds to column j at most
    # 2 sqrt(b) u3x |a_j| (both operands rounded, three products) plus its FP32 accumulation,
    # about sqrt(M) u |a_j|; column j of panel t has been through t + 1 updates and block
    # projections, and normalising by r_jj multiplies its error by rho_j = |a_j| / r_jj.
    # Errors of earlier columns reach later ones through those same projections, which the
    # factor 4 covers; the tiles rebuilt by recovery add kappa(G^) u, far below that.
    A32 = A.astype(np.float32).astype(np.float64)      # the bytes the FP32 path factors
    y32 = y.astype(np.float32).astype(np.float64)
    ref = O.run(A32, p, p, f, b, seed=cfg["seed"], erasures=er, y=y32, reorth_block=True)
    assert ref["sets"] == sets
    an = np.linalg.norm(ref["At"], axis=0)
    upd = 2 * np.sqrt(b) * U3X + np.sqrt(M) * U32
    t_of = np.minimum(np.arange(g.N) // b, n // b)
    rho = np.ones(g.N)
    rho[:n] = an[:n] / np.abs(np.diag(ref["R"])[:n])
    tol_col = 4 * (t_of + 1) * upd * an * rho + 4 * b * U32
    err_q = torch.linalg.norm(Qt - torch.from_numpy(ref["Q"]).to(dev), dim=0).cpu().numpy()
    worst = int(np.argmax(err_q / tol_col))
    assert (err_q < tol_col).all(), (worst, err_q[worst], tol_col[worst])
    err_r = np.abs(R.cpu().numpy() - ref["R"])
    tol_r = 4 * (t_of[None, :] + 1) * upd * an[None, :]
    assert (err_r <= tol_r).all(), np.unravel_index(np.argmax(err_r / tol_r), err_r.shape)
    # post-orthogonalisation (the projected form, the FP32 default) against the oracle's
    # G_0 Q_1: the same matrix in exact arithmetic; |G_0|_2 <= sqrt(1 + |G~|_2^2) bounds how
    # much it magnifies the column errors of Q_1
    g0n = np.sqrt(1 + np.linalg.norm(Gto, 2) ** 2)
    err_o = torch.linalg.norm(Qo - torch.from_numpy(ref["Qo"]).to(dev), dim=0).cpu().numpy()
    assert (err_o < g0n * tol_col[:n]).all(), (err_o.max(), int(np.argmax(err_o / tol_col[:n])))
    # the solve: the forward error of x is kappa times the backward error of the factors
    assert rel(x, ref["x"]) < 1e-4 * kap, rel(x, ref["x"])

    # properties at any size: the checksum rows follow the systematic rows (drift of the
    # FP32 updates, u kappa scale); the solve's residual is within kappa times the 1e-5
    # backward-error target
    Gv = torch.kron(torch.from_numpy(Gto), torch.eye(g.mb, dtype=torch.float64)).to(dev)
    drift = (Qt[m:M, :n] - Gv @ Qt[:m, :n]).abs().max().item()
    assert drift < 100 * U3X * kap, drift
    resid = np.linalg.norm(A @ x - y) / np.linalg.norm(y)
    assert resid <= 1e-5 * kap, resid
    print("c2 step: back %.3g orth_coded %.3g orth %.3g drift %.3g resid %.3g"
          % (back, orth_coded, orth, drift, resid))


# ----------------------------------------------------------------- tensor-core trailing update
# 3xTF32 splits each FP32 operand into a TF32 head and tail (three tcgen05 products); its
# products carry a relative error of about 2^-21 (8 u32).  Plain TF32 has unit roundoff 2^-11.
U3X = 8 * U32
UTF32 = 2.0 ** -11


@pytest.mark.parametrize("shape", [(256, 256, 4, 4, 1, 32), (203, 96, 8, 4, 2, 20),
                                   (640, 640, 8, 8, 2, 128), (1024, 512, 8, 4, 2, 256)])
def test_3xtf32_path_parity(shape):
    m, n, p_r, p_c, f, b = shape
    A = synth.kappa_matrix(m, n, 1e2, seed=3)
    y = synth.rhs(m, 1, 3)
    T = -(-n // b)
    er = {T // 2: synth.random_erasures(p_r + f, p_c + f, f, 2, seed=5)}
    ref = O.run(A, p_r, p_c, f, b, seed=4, erasures=er, y=y)
    got = gpu_run(A, p_r, p_c, f, b, seed=4, erasures=er, y=y, dtype="f32", mma="3xtf32")
    assert got["status"] == 0
    assert got["sets"] == ref["sets"]
    g = ref["geom"]
    tol = n * U3X * 1e2
    assert rel(got["Q"][: g.M, :n], ref["Q"][:, :n]) < tol
    assert rel(got["R"], ref["R"]) < tol
    assert rel(got["Qo"], ref["Qo"]) < tol
    if "x" in got:
        assert rel(got["x"], ref["x"]) < tol * 1e2
    Q1, R1 = got["Q"][:m, :n], got["R"][:n, :n]
    assert np.linalg.norm(A - Q1 @ R1) / np.linalg.norm(A) < 1e-5


def test_tf32_path_well_conditioned():
    m = n = 512
    A = synth.kappa_matrix(m, n, 4.0, seed=8)
    ref = O.run(A, 8, 8, 2, 128, seed=1)
    got = gpu_run(A, 8, 8, 2, 128, seed=1, dtype="f32", mma="tf32")
    assert got["status"] == 0
    Q1, R1 = got["Q"][:m, :n], got["R"][:n, :n]
    assert np.linalg.norm(A - Q1 @ R1) / np.linalg.norm(A) < 8 * UTF32
    assert rel(got["R"], ref["R"]) < n * UTF32 * 4.0
    Qo = got["Qo"]
    assert np.abs(Qo.T @ Qo - np.eye(n)).max() < n * UTF32


def test_tc_matches_simt_fp32_closely():
    # same FP32 storage, trailing updates on tensor cores (3xTF32) vs CUDA cores (FP32 FMA)
    A = synth.kappa_matrix(384, 384, 10.0, seed=9)
    a = gpu_run(A, 4, 4, 1, 64, seed=2, dtype="f32", mma="simt")
    b = gpu_run(A, 4, 4, 1, 64, seed=2, dtype="f32", mma="3xtf32")
    assert rel(b["R"], a["R"]) < 384 * U3X * 10.0


@pytest.mark.parametrize("shape", [(256, 256, 4, 1, 32), (640, 640, 8, 2, 128), (4096, 512, 8, 2, 64)])
def test_register_and_shared_memory_panels_agree(shape, monkeypatch):
    # the FP32 panel runs register-resident in one cluster when it fits, else from shared
    # memory; both follow the same column recurrence (reorthogonalisation included)
    m, n, p, f, b = shape
    A = synth.gaussian(m, n, 12)
    A[:, 1::7] = A[:, 0::7][:, : A[:, 1::7].shape[1]] + 1e-4 * A[:, 1::7]  # force reorth
    a = gpu_run(A, p, p if n % p == 0 else 4, f, b, seed=3, dtype="f32", mma="3xtf32")
    monkeypatch.setenv("CQR_PANEL_REG", "0")
    bb = gpu_run(A, p, p if n % p == 0 else 4, f, b, seed=3, dtype="f32", mma="3xtf32")
    assert a["status"] == 0 and bb["status"] == 0
    assert a["stats"]["n_reorth"] > 0
    assert abs(a["stats"]["n_reorth"] - bb["stats"]["n_reorth"]) <= 2
    kap = np.linalg.cond(A)
    assert rel(a["R"], bb["R"]) < n * U3X * kap
    ref = O.run(A, p, p if n % p == 0 else 4, f, b, seed=3)
    assert rel(a["R"], ref["R"]) < n * U3X * kap


@pytest.mark.parametrize("env", [{"CQR_LOOKAHEAD": "0"}, {"CQR_PDL": "0"}])
def test_lookahead_and_pdl_change_rounding_only(env, monkeypatch):
    # the look-ahead (narrow and wide trailing updates on two streams) and programmatic
    # dependent launch are schedules of the same panels: the factors match the sequential
    # schedule to rounding (the split-K factors of the two updates differ), with the same
    # decode sets, erasures injected at a panel start
    m, n, p_r, p_c, f, b = 1280, 1024, 8, 8, 2, 128
    A = synth.kappa_matrix(m, n, 1e2, seed=41)
    er = {3: synth.random_erasures(p_r + f, p_c + f, f, 2, seed=9)}
    a = gpu_run(A, p_r, p_c, f, b, seed=6, erasures=er, dtype="f32", mma="3xtf32")
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    c = gpu_run(A, p_r, p_c, f, b, seed=6, erasures=er, dtype="f32", mma="3xtf32")
    assert a["status"] == 0 and c["status"] == 0
    assert a["sets"] == c["sets"]
    tol = n * U3X * 1e2
    assert rel(a["R"], c["R"]) < tol
    assert rel(a["Qo"], c["Qo"]) < tol
    ref = O.run(A, p_r, p_c, f, b, seed=6, erasures=er)
    assert rel(c["R"], ref["R"]) < tol


# BF16 operands (tcgen05 kind::f16): one product carries the BF16 rounding 2^-9; the hi/lo
# split with three products leaves the lo rounding and the dropped lo*lo term, about 2^-17.
UBF16 = 2.0 ** -8
UBF3 = 2.0 ** -16


@pytest.mark.parametrize("shape", [(256, 256, 4, 4, 1, 32), (203, 96, 8, 4, 2, 20),
                                   (640, 640, 8, 8, 2, 128)])
def test_bf16x3_path_parity(shape):
    m, n, p_r, p_c, f, b = shape
    A = synth.kappa_matrix(m, n, 1e2, seed=3)
    y = synth.rhs(m, 1, 3)
    T = -(-n // b)
    er = {T // 2: synth.random_erasures(p_r + f, p_c + f, f, 2, seed=5)}
    ref = O.run(A, p_r, p_c, f, b, seed=4, erasures=er, y=y)
    got = gpu_run(A, p_r, p_c, f, b, seed=4, erasures=er, y=y, dtype="f32", mma="bf16x3")
    assert got["status"] == 0
    assert got["sets"] == ref["sets"]
    g = ref["geom"]
    tol = n * UBF3 * 1e2
    assert rel(got["Q"][: g.M, :n], ref["Q"][:, :n]) < tol
    assert rel(got["R"], ref["R"]) < tol
    assert rel(got["Qo"], ref["Qo"]) < tol
    Q1, R1 = got["Q"][:m, :n], got["R"][:n, :n]
    assert np.linalg.norm(A - Q1 @ R1) / np.linalg.norm(A) < 64 * UBF3


def test_bf16_path_well_conditioned():
    m = n = 512
    A = synth.kappa_matrix(m, n, 4.0, seed=8)
    ref = O.run(A, 8, 8, 2, 128, seed=1)
    got = gpu_run(A, 8, 8, 2, 128, seed=1, dtype="f32", mma="bf16")
    assert got["status"] == 0
    Q1, R1 = got["Q"][:m, :n], got["R"][:n, :n]
    assert np.linalg.norm(A - Q1 @ R1) / np.linalg.norm(A) < 8 * UBF16
    assert rel(got["R"], ref["R"]) < n * UBF16 * 4.0


def test_bf16x3_with_block_reorth_matches_3xtf32():
    # the same factorisation through both split modes, block reorthogonalisation on
    m = n = 512
    A = synth.kappa_matrix(m, n, 1e3, seed=17)
    res = {}
    for mma in ("3xtf32", "bf16x3"):
        q = B.CodedQR(m, n, 8, 8, 2, 64, dtype="f32", mma=mma, seed=6, reorth_block=True)
        q.encode(to_dev(A, torch.float32))
        q.factor(0, -1)
        torch.cuda.synchronize()
        assert q.sync_status() == 0
        Qc, Rc = q.factors()
        res[mma] = (to_np(Qc), to_np(Rc))
        q.close()
    Q, R = res["bf16x3"]
    g = q.geo
    Qt = Q[: g["M"], :n]
    assert np.abs(Qt.T @ Qt - np.eye(n)).max() < 1e-4
    assert rel(R, res["3xtf32"][1]) < n * UBF3 * 1e3


# ----------------------------------------------------------------- block reorthogonalisation
@pytest.mark.parametrize("dtype,mma,kappa", [("f64", "simt", 1e8), ("f32", "3xtf32", 1e4),
                                             ("f32", "simt", 1e4)])
def test_block_reorth_parity_and_orthogonality(dtype, mma, kappa):
    m = n = 512
    p, f, b = 8, 2, 64
    A = synth.kappa_matrix(m, n, kappa, seed=13)
    er = {3: synth.random_erasures(p + f, p + f, f, 2, seed=3), 6: [(1, 1)]}
    ref = O.run(A, p, p, f, b, seed=6, erasures=er, reorth_block=True)
    q = B.CodedQR(m, n, p, p, f, b, dtype=dtype, mma=mma, seed=6, reorth_block=True)
    td = torch.float64 if dtype == "f64" else torch.float32
    q.encode(to_dev(A, td))
    for t in range(q.geo["panels"]):
        if er.get(t):
            q.inject(er[t])
            q.recover()
        q.factor(t, t + 1)
    Qc, Rc = q.factors()
    Q, R = to_np(Qc), to_np(Rc)
    Qo = B.colmajor_empty(q.geo["m_pad"], n, td)
    q.post_orth(Qo)
    torch.cuda.synchronize()
    assert q.sync_status() == 0
    assert q.decode_sets() == ref["sets"]
    q.close()
    u = U64 if dtype == "f64" else (U3X if mma == "3xtf32" else U32)
    g = ref["geom"]
    tol = n * u * kappa
    assert rel(R, ref["R"]) < tol
    Qo = to_np(Qo)
    orth = np.abs(Qo.T @ Qo - np.eye(n)).max()
    back = np.linalg.norm(A - Q[:m, :n] @ R[:n, :n]) / np.linalg.norm(A)
    # the coded factor itself is orthogonal to working precision after the extra pass; the
    # post-orthogonalised G_0 Q_1 inherits the drift of Q_2 = G_v Q_1, which the pivots
    # amplify like u kappa (the oracle shows the same)
    Qt = Q[: g.M, :n]
    orth_coded = np.abs(Qt.T @ Qt - np.eye(n)).max()
    orth_ref = np.abs(ref["Qo"].T @ ref["Qo"] - np.eye(n)).max()
    drift = np.abs(Q[g.m_pad: g.M, :n] - np.kron(ref["Gt"], np.eye(g.mb)) @ Q[: g.m_pad, :n]).max()
    assert orth <= 4 * drift + 64 * n * u, (orth, drift)   # post-orth limited by the drift
    if dtype == "f32":
        # FP32 accuracy target on the coded factor and the backward error
        assert orth_coded < 1e-5 and back < 1e-5, (orth_coded, back)
        assert drift < 100 * u * kappa
    else:
        assert orth_coded < 64 * n * u
        assert back < 1e-12 and orth < max(1e-12, 10 * orth_ref), (orth, orth_ref, back)


# ----------------------------------------------------------------- vertical code alone
@pytest.mark.parametrize("dtype,mma", [("f64", "simt"), ("f32", "3xtf32")])
def test_vertical_only_code_parity(dtype, mma):
    # R protection off (vertical code alone, d = 0): no checksum columns; only Q tiles are
    # erased and rebuilt.  Q, R, G_0 Q_1 and x against the oracle, decode sets bit for bit.
    m = n = 640
    p, f, b = 8, 2, 64
    A = synth.kappa_matrix(m, n, 1e2, seed=23)
    y = synth.rhs(m, 1, 23)
    er = {3: synth.random_erasures(p + f, p, f, 2, seed=11),
          7: synth.random_erasures(p + f, p, f, 1, seed=12)}
    ref = O.run(A, p, p, f, b, seed=5, erasures=er, y=y, protect_r=False)
    got = gpu_run(A, p, p, f, b, seed=5, erasures=er, y=y, dtype=dtype, mma=mma,
                  protect_r=False)
    assert got["status"] == 0
    assert got["geo"]["N"] == n
    assert got["sets"] == ref["sets"]
    g = ref["geom"]
    tol = n * (U64 if dtype == "f64" else U3X) * 1e2
    assert rel(got["Q"][: g.M, :n], ref["Q"][:, :n]) < tol
    assert rel(got["R"], ref["R"]) < tol
    assert rel(got["Qo"], ref["Qo"]) < tol
    assert rel(got["x"], ref["x"]) < tol * 1e2


# ----------------------------------------------------------------- square solve (a9)
@pytest.mark.parametrize("dtype,mma", [("f64", "simt"), ("f32", "3xtf32")])
def test_square_solve_ragged_block_count(dtype, mma):
    # n = 1096: 18 row blocks of the back substitution (the last one 8 rows), more than the
    # 16 CTAs of its cluster, so some CTAs own two blocks; three right-hand sides
    n = 1096
    A = synth.kappa_matrix(n, n, 1e2, seed=23)
    y = synth.rhs(n, 3, 23)
    er = {2: [(5, 3)]}
    ref = O.run(A, 8, 8, 1, 64, seed=4, erasures=er, y=y)
    got = gpu_run(A, 8, 8, 1, 64, seed=4, erasures=er, y=y, dtype=dtype, mma=mma)
    assert got["status"] == 0
    u = U64 if dtype == "f64" else U3X
    tol = n * u * 1e2 * 10
    assert rel(got["x"], ref["x"]) < tol * max(1.0, np.abs(ref["x"]).max())
    # the residual of the computed x against A itself
    res = np.linalg.norm(A @ got["x"] - y) / (np.linalg.norm(A) * np.linalg.norm(got["x"]))
    assert res < 10 * n * u


# ----------------------------------------------------------------- tall least squares (a9)
@pytest.mark.parametrize("dtype,mma,shape", [("f64", "simt", (1024, 256, 8, 4, 2, 64)),
                                             ("f64", "simt", (1003, 192, 8, 4, 1, 48)),
                                             ("f32", "3xtf32", (2048, 256, 8, 4, 2, 128))])
def test_tall_least_squares(dtype, mma, shape):
    m, n, p_r, p_c, f, b = shape
    A = synth.kappa_matrix(m, n, 1e3, seed=17)
    y = synth.rhs(m, 2, 17)
    er = {1: [(2, 1)]}
    ref = O.run(A, p_r, p_c, f, b, seed=7, y=y, erasures=er)
    td = torch.float64 if dtype == "f64" else torch.float32
    q = B.CodedQR(m, n, p_r, p_c, f, b, dtype=dtype, mma=mma, seed=7, nrhs_max=2)
    q.encode(to_dev(A, td))
    for t in range(q.geo["panels"]):
        if er.get(t):
            q.inject(er[t])
            q.recover()
        q.factor(t, t + 1)
    x = B.colmajor_empty(n, 2, td)
    yd = to_dev(y, td)
    q.solve(yd, x)
    # the same verb under the problem statement's name gives the same x bit for bit
    x_ls = B.colmajor_empty(n, 2, td)
    q.solve_ls(yd, x_ls)
    torch.cuda.synchronize()
    assert q.sync_status() == 0
    assert torch.equal(x, x_ls)
    q.close()
    x = to_np(x)
    xl, *_ = np.linalg.lstsq(A, y, rcond=None)
    u = U64 if dtype == "f64" else U3X
    tol = n * u * 1e3 * 10
    assert rel(x, ref["x"]) < tol * max(1.0, np.abs(ref["x"]).max())
    assert rel(x, xl) < tol * max(1.0, np.abs(xl).max())
