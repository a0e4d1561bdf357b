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
