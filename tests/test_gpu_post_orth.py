"""Post-orthogonalisation (a8) on the GPU against the oracle, element by element, through the
C ABI (needs a GB300).

Both forms are fed the same coded Q: the oracle's own factorisation rounded to the storage
precision, written into the handle through its borrowed factor view, with a seeded drift
planted in the checksum rows.  The paper's form is Qo = G_0 Q_1 (Theorem G_0); the projected
form is Qo = G_0^{-1} (Q_1 + G^T Q_2) (coded_qr.h, CQR_POST_ORTH_PROJECTED), which equals
G_0 Q_1 when Q_2 = G Q_1 and loses orthogonality only to second order in the drift.

Tolerance: every output is a fixed linear combination of the p_r + f entries of one tile
position; the kernel forms it in the storage precision through five dependent stages (h, Y,
U, Z, G_0 Z), each a sum of at most p_r + f products with coefficients below
g = max(1, max |G~|, max |K|) in magnitude.  Its rounding is therefore below
5 (p_r + f) g^2 u max|Q| (u the unit roundoff of the storage type).
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

U = {"f64": np.finfo(np.float64).eps / 2, "f32": np.finfo(np.float32).eps / 2}


def _load_into_handle(q, Q_np, td):
    """Overwrite the handle's coded Q (M x N) with Q_np (already in the storage precision)."""
    Qc, _ = q.factors()
    Qc.copy_(torch.from_numpy(np.ascontiguousarray(Q_np)).to(td))
    torch.cuda.synchronize()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("shape", [(256, 256, 4, 4, 1, 32), (640, 512, 8, 8, 2, 64),
                                   (512, 256, 16, 8, 4, 32), (384, 384, 12, 12, 6, 32),
                                   (1280, 128, 40, 8, 2, 32)])
def test_both_forms_match_the_oracle_on_the_same_coded_q(dtype, shape):
    # (12, 6): the generic checksum count; (40, 2): p_r > 32, the two-pass form
    m, n, p_r, p_c, f, b = shape
    td = torch.float64 if dtype == "f64" else torch.float32
    npt = np.float64 if dtype == "f64" else np.float32
    A = synth.kappa_matrix(m, n, 1e2, seed=31)
    ref = O.run(A, p_r, p_c, f, b, seed=5)
    g = ref["geom"]
    # an orthonormal coded factor whose checksum rows drifted from G Q_1: the oracle's Q with
    # a seeded perturbation of Q_2, orthonormalised again as a whole (numpy QR)
    delta = 1e-3
    Qd = ref["Q"][:, :n].copy()
    Qd[g.m_pad:g.M] += delta * synth.gaussian(g.c, n, 77) / np.sqrt(g.M)
    Qd, _ = np.linalg.qr(Qd)
    Qs = np.asfortranarray(ref["Q"].astype(npt))
    Qs[:g.M, :n] = Qd.astype(npt)
    Q64 = Qs.astype(np.float64)
    Q1, Q2 = Q64[:g.m_pad, :n], Q64[g.m_pad:g.M, :n]
    want_proj = O.post_orth_projected(g, ref["Gt"], Q1, Q2)
    want_g0 = O.post_orth(g, ref["Gt"], Q1)

    got = {}
    for form in ("g0", "projected"):
        q = B.CodedQR(m, n, p_r, p_c, f, b, dtype=dtype, mma="simt", seed=5, post_orth=form)
        Ad = B.colmajor_empty(m, n, td)
        Ad.copy_(torch.from_numpy(A))
        q.encode(Ad)
        q.factor(0, -1)
        Gt, _ = q.generator()
        assert np.array_equal(Gt, ref["Gt"])
        _load_into_handle(q, Qs, td)
        Qo = B.colmajor_empty(g.m_pad, n, td)
        q.post_orth(Qo)
        torch.cuda.synchronize()
        assert q.sync_status() == 0
        got[form] = Qo.double().cpu().numpy()
        q.close()

    Gt = ref["Gt"]
    K = np.linalg.inv(np.eye(f) + Gt @ Gt.T)
    gmax = max(1.0, np.abs(Gt).max(), np.abs(K).max())
    tol = 5 * (p_r + f) * gmax ** 2 * U[dtype] * np.abs(Qs).max()
    assert np.abs(got["projected"] - want_proj).max() < tol
    assert np.abs(got["g0"] - want_g0).max() < tol

    # the planted drift: the paper's form loses orthogonality to first order in it, the
    # projected form to second order (the oracle pins the same scaling), down to the
    # rounding of the storage type
    eye = np.eye(n)
    drift = np.abs(Q2 - np.kron(Gt, np.eye(g.mb)) @ Q1).max()
    loss_g0 = np.abs(got["g0"].T @ got["g0"] - eye).max()
    loss_proj = np.abs(got["projected"].T @ got["projected"] - eye).max()
    assert loss_g0 > 0.1 * drift
    assert loss_proj < n * drift ** 2 + 10 * gmax * U[dtype] * np.sqrt(g.M)
    assert loss_proj < 0.1 * loss_g0


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_projected_form_in_place_and_through_the_solve(dtype):
    # no planted drift: on the handle's own factors the projected form equals the paper's to
    # the drift of the computation, in place (Q_1 overwritten, as the square solve does) as
    # well as out of place, and the square solve with it matches the oracle's x
    n, p, f, b = 512, 8, 2, 64
    td = torch.float64 if dtype == "f64" else torch.float32
    A = synth.kappa_matrix(n, n, 1e2, seed=12)
    y = synth.rhs(n, 1, 12)
    ref = O.run(A, p, p, f, b, seed=9, y=y, erasures={3: [(2, 5)]})
    outs = {}
    for form in ("g0", "projected"):
        q = B.CodedQR(n, n, p, p, f, b, dtype=dtype, mma="simt", seed=9, post_orth=form)
        Ad = B.colmajor_empty(n, n, td)
        Ad.copy_(torch.from_numpy(A))
        q.encode(Ad)
        q.factor(0, 3)
        q.inject([(2, 5)])
        q.recover()
        q.factor(3, -1)
        Qo = B.colmajor_empty(n, n, td)
        q.post_orth(Qo)
        Qc, _ = q.factors()
        Q1_before = Qc[:n, :n].clone()
        q.post_orth()                       # in place
        yd = B.colmajor_empty(n, 1, td)
        yd.copy_(torch.from_numpy(y))
        x = B.colmajor_empty(n, 1, td)
        q.solve(yd, x)
        torch.cuda.synchronize()
        assert q.sync_status() == 0
        assert torch.equal(Qc[:n, :n], Qo)  # in place gives the same bits as out of place
        assert not torch.equal(Q1_before, Qo)
        outs[form] = (Qo.double().cpu().numpy(), x.double().cpu().numpy())
        q.close()
    u = U[dtype]
    tol = n * u * 1e2 * 10
    for form in ("g0", "projected"):
        Qo, x = outs[form]
        assert np.abs(Qo - ref["Qo"]).max() < tol
        assert np.abs(x - ref["x"]).max() < tol * np.abs(ref["x"]).max()
