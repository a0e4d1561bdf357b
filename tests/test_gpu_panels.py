"""Panel variants on the GPU (NEXT f3) against the same variants in the oracle: the paper's
ICGS, MGS (no reorthogonalisation test), left-looking CGS with one reduction per column
(CGS1) and CGS2.  Tolerances: n u kappa for the stable variants, n u kappa^2 for CGS1 (its
orthogonality loss)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_11943_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2311_11943_gb300 import binding as B  # noqa: E402


def _dev(A, td):
    d = B.colmajor_empty(A.shape[0], A.shape[1], td)
    d.copy_(torch.from_numpy(np.ascontiguousarray(A)))
    return d


def rel(a, b):
    return np.abs(a - b).max() / max(1.0, np.abs(b).max())


@pytest.mark.parametrize("panel", ["mgs", "cgs1", "cgs2"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_panel_variant_matches_oracle(panel, dtype):
    m, n, p, f, b, kappa = 640, 320, 8, 2, 64, 10.0
    A = synth.kappa_matrix(m, n, kappa, seed=23)
    er = {2: synth.random_erasures(p + f, 4 + f, f, 2, seed=4)}
    ref = O.run(A, p, 4, f, b, seed=8, erasures=er, panel=panel)
    td = torch.float64 if dtype == "f64" else torch.float32
    q = B.CodedQR(m, n, p, 4, f, b, dtype=dtype, seed=8, panel=panel)
    q.encode(_dev(A, td))
    for t in range(q.geo["panels"]):
        if er.get(t):
            q.inject(er[t])
            q.recover()
        q.factor(t, t + 1)
    Qc, Rc = q.factors()
    torch.cuda.synchronize()
    assert q.sync_status() == 0
    assert q.decode_sets() == ref["sets"]
    Q = Qc.double().cpu().numpy()
    R = Rc.double().cpu().numpy()
    q.close()
    u = (np.finfo(np.float64).eps if dtype == "f64" else np.finfo(np.float32).eps) / 2
    tol = n * u * (kappa ** 2 if panel == "cgs1" else kappa) * 10
    g = ref["geom"]
    assert rel(Q[: g.M, :n], ref["Q"][:, :n]) < tol
    assert rel(R, ref["R"]) < tol


SCHEDULES = {"sub-panels": {"CQR_PANEL_SUB": "1"}, "two-level": {},
             "flat grid": {"CQR_PANEL_HIER": "0"}}


@pytest.mark.parametrize("mma", ["3xtf32", "simt"])
def test_tall_panel_schedules_match_oracle_and_each_other(mma, monkeypatch):
    # The panel of the 16384^2 workload's shape (20480 x 256, FP32) needs more CTAs than one
    # cluster holds.  Three schedules factor it: the two-level exchange (clusters of 8 whose
    # leaders publish tagged sums; the default); 32-column sub-panels that each fit one
    # cluster, with the panel's remaining columns projected on each (on request); the flat
    # grid barrier.  A 16384 x 1024 problem on that grid (16 x 8, f = 4, b = 256) has the same
    # panel; each schedule is compared with the oracle (n u kappa, with u = 8 u32 for 3xTF32
    # products) and with the others (the same arithmetic in another order, n u kappa).
    m, n, p_r, p_c, f, b, kappa = 16384, 1024, 16, 8, 4, 256, 10.0
    A = synth.kappa_matrix(m, n, kappa, seed=61)
    er = {2: [(3, 5), (17, 2)]}
    ref = O.run(A, p_r, p_c, f, b, seed=4, erasures=er)
    out = {}
    for name, env in SCHEDULES.items():
        for k in ("CQR_PANEL_SUB", "CQR_PANEL_HIER"):
            monkeypatch.delenv(k, raising=False)
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        q = B.CodedQR(m, n, p_r, p_c, f, b, dtype="f32", mma=mma, seed=4)
        q.encode(_dev(A, torch.float32))
        for t in range(q.geo["panels"]):
            if er.get(t):
                q.inject(er[t])
                q.recover()
            q.factor(t, t + 1)
        Qc, Rc = q.factors()
        torch.cuda.synchronize()
        assert q.sync_status() == 0
        assert q.decode_sets() == ref["sets"]
        out[name] = (Qc.double().cpu().numpy(), Rc.double().cpu().numpy())
        q.close()
    u = np.finfo(np.float32).eps / 2 * (8 if mma == "3xtf32" else 1)
    tol = n * u * kappa
    for name in SCHEDULES:
        Q, R = out[name]
        assert rel(Q, ref["Q"]) < tol and rel(R, ref["R"]) < tol, name
    for x, y in (("sub-panels", "two-level"), ("two-level", "flat grid")):
        assert rel(out[x][0], out[y][0]) < tol and rel(out[x][1], out[y][1]) < tol, (x, y)
