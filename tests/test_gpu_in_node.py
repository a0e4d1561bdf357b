"""In-node checksum storage (NEXT f2) on the GPU against the oracle: K checksum blocks per
code hosted by the data nodes, node failures erasing every tile their node hosts, recovery
through the same decode.  Decode index sets bit for bit, factors within n u kappa."""
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


@pytest.mark.parametrize("p,f,dtype,mma,nodes", [
    (4, 1, "f64", "simt", [(2, 1)]),
    (8, 2, "f64", "simt", [(0, 3), (5, 3)]),
    (8, 2, "f32", "3xtf32", [(1, 1), (6, 4)]),
])
def test_in_node_node_failures_match_oracle(p, f, dtype, mma, nodes):
    m = n = 32 * p
    b = 16
    A = synth.kappa_matrix(m, n, 1e2, seed=41)
    t_fail = 3
    ref = O.run_in_node(A, p, f, b, seed=9, node_failures={t_fail: nodes})
    td = torch.float64 if dtype == "f64" else torch.float32
    q = B.CodedQR(m, n, p, p, f, b, dtype=dtype, mma=mma, seed=9, in_node=True)
    assert q.geo["code_blocks"] == ref["K"]
    assert q.geo["grid_rows"] == p + ref["K"]
    q.encode(_dev(A, td))
    for t in range(q.geo["panels"]):
        if t == t_fail:
            q.fail_nodes(nodes)
            q.recover()
        q.factor(t, t + 1)
    Qc, Rc = q.factors()
    torch.cuda.synchronize()
    assert q.sync_status() == 0
    assert q.decode_sets() == ref["sets"]
    Q = Qc.double().cpu().numpy()
    R = Rc.double().cpu().numpy()
    q.close()
    u = (np.finfo(np.float64).eps / 2) if dtype == "f64" else 8 * np.finfo(np.float32).eps / 2
    tol = n * u * 1e2 * 10
    g = ref["geom"]
    assert rel(Q[: g.M, :n], ref["Q"][:, :n]) < tol
    assert rel(R, ref["R"]) < tol


def test_in_node_run_plan_uses_node_coordinates():
    p, f, b = 8, 2, 32
    m = n = 256
    A = synth.kappa_matrix(m, n, 1e2, seed=43)
    plan = [(2, 4, 4), (5, 0, 7)]
    ref = O.run_in_node(A, p, f, b, seed=3, node_failures={2: [(4, 4)], 5: [(0, 7)]})
    q = B.CodedQR(m, n, p, p, f, b, dtype="f64", seed=3, in_node=True)
    q.run(_dev(A, torch.float64), plan=plan)
    torch.cuda.synchronize()
    assert q.sync_status() == 0
    assert q.decode_sets() == ref["sets"]
    _, Rc = q.factors()
    assert rel(Rc.cpu().numpy(), ref["R"]) < n * 1.1e-16 * 1e3
    q.close()


def test_in_node_rejects_codes_the_generator_cannot_carry():
    # p = 6, f = 2: K = 2 + 2 ceil(2/4) = 4 and 2K > p_r
    with pytest.raises(B.CodedQRError) as e:
        B.CodedQR(96, 96, 6, 6, 2, 16, dtype="f64", in_node=True)
    assert e.value.status == B.CQR_EINVAL
