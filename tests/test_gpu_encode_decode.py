"""The FP32 encode (both codes in one pass) and the four-row FP32 decode against the FP64
oracle on awkward shapes (needs a GB300).

Shapes: tile heights that are not a multiple of the 32-row thread blocks, ragged last tile
rows, tile-column counts that leave some of the encode's four column groups empty or uneven,
one to four checksums; decodes of several grid columns and R block rows at once, a
checksum tile lost together with a systematic one, and two lost tiles in one grid column.
The encoded matrix is compared element by element; decode index sets bit for bit.
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

U32 = np.finfo(np.float32).eps / 2


def dev_a(A, ld):
    d = B.colmajor_empty(A.shape[0], A.shape[1], torch.float32, ld=ld)
    d.copy_(torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)))
    return d


# (m, n, p_r, p_c, f, lda): tile heights mb = 260, 128, 100, 200, 52 and 1024; ragged last
# tile rows; p_c = 5, 6 and 3 leave column groups uneven or empty
ENCODE_CASES = [
    (2077, 64, 8, 16, 4, 2080),
    (2048, 2048, 16, 16, 4, 2048),
    (600, 30, 6, 5, 2, 600),
    (1197, 36, 6, 6, 3, 1200),
    (103, 12, 2, 3, 1, 104),
    (4093, 256, 4, 8, 2, 4096),
]


@pytest.mark.parametrize("m,n,p_r,p_c,f,lda", ENCODE_CASES)
def test_fp32_encode_matches_oracle(m, n, p_r, p_c, f, lda):
    A = synth.gaussian(m, n, 5 + m)
    q = B.CodedQR(m, n, p_r, p_c, f, 4, dtype="f32", seed=77)
    q.encode(dev_a(A, lda))
    Qc, _ = q.factors()
    torch.cuda.synchronize()
    assert q.sync_status() == 0
    Gt, Gh = q.generator()
    M, N = q.geo["M"], q.geo["N"]
    Qs = Qc.double().cpu().numpy()[:M, :N]
    q.close()
    g = O.geom(m, n, p_r, p_c, f)
    At = O.encode(g, Gt, Gh, A.astype(np.float32).astype(np.float64))
    # the copy is exact; each checksum sums at most p_r p_c FP32 products of O(1) terms
    assert np.array_equal(Qs[:m, :n], At[:m, :n])
    assert np.abs(Qs - At).max() / np.abs(At).max() < 4 * (p_r + p_c) * U32


# (m, n, p_r, p_c, f, b, {panel: tiles}): two grid columns and two R block rows at once; a
# checksum-row tile (row p_r) with a systematic one of the same grid column; mb = 260 and 128;
# the 16 x 16 grid with four checksums and four lost tiles, two of them in one grid column
DECODE_CASES = [
    (1040, 512, 4, 4, 2, 64, {2: [(1, 1), (3, 2)]}),
    (1040, 512, 4, 4, 2, 64, {1: [(0, 3), (4, 3)]}),
    (2048, 2048, 16, 16, 4, 128, {3: [(2, 5), (7, 9), (11, 9), (15, 14)]}),
]


@pytest.mark.parametrize("m,n,p_r,p_c,f,b,plan", DECODE_CASES)
def test_fp32_decode_matches_oracle(m, n, p_r, p_c, f, b, plan):
    A = synth.kappa_matrix(m, n, 10.0, seed=m + 3)
    q = B.CodedQR(m, n, p_r, p_c, f, b, dtype="f32", mma="3xtf32", seed=9)
    q.encode(dev_a(A, m))
    for t in range(q.geo["panels"]):
        if plan.get(t):
            q.inject(plan[t])
            q.recover()
        q.factor(t, t + 1)
    Qc, Rc = q.factors()
    torch.cuda.synchronize()
    st, sets = q.sync_status(), q.decode_sets()
    Q, R = Qc.double().cpu().numpy(), Rc.double().cpu().numpy()
    q.close()
    assert st == 0
    ref = O.run(A, p_r, p_c, f, b, seed=9, erasures=plan)
    assert sets == ref["sets"]
    g = ref["geom"]
    tol = n * 8 * U32 * 10.0  # n u kappa with the 3xTF32 unit roundoff (8 u) and kappa = 10
    assert np.abs(R - ref["R"]).max() / np.abs(ref["R"]).max() < tol
    assert np.abs(Q[: g.M, :n] - ref["Q"][:, :n]).max() < tol
