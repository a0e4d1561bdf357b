"""The TMA-streamed FP32 encode and decode (needs a GB300).

Both stream their inputs through shared memory but keep the register kernels' arithmetic in
the same order, so with CQR_NO_TMA_STREAM=1 (the register kernels) the encoded matrix and the
recovered tiles must agree bit for bit; both are also compared with the FP64 oracle.  The
shapes cover tile heights that are not a multiple of the 128-row box, ragged last tile rows
(A's rows padded to a multiple of four in its leading dimension), tile-column counts that do
not split evenly over the four column groups, one to four checksums, several grid columns and
R block rows rebuilt at once, and a checksum tile lost together with a systematic one.
"""
import os

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


class register_kernels:
    """CQR_NO_TMA_STREAM=1 inside the block when on, the environment as it was afterwards."""

    def __init__(self, on):
        self.on = on

    def __enter__(self):
        self.old = os.environ.pop("CQR_NO_TMA_STREAM", None)
        if self.on:
            os.environ["CQR_NO_TMA_STREAM"] = "1"

    def __exit__(self, *exc):
        os.environ.pop("CQR_NO_TMA_STREAM", None)
        if self.old is not None:
            os.environ["CQR_NO_TMA_STREAM"] = self.old


def encode_once(A, p_r, p_c, f, ld, stream):
    m, n = A.shape
    with register_kernels(not stream):
        q = B.CodedQR(m, n, p_r, p_c, f, 4, dtype="f32", seed=77)
        q.encode(dev_a(A, ld))
        Qc, _ = q.factors()
        torch.cuda.synchronize()
        out = Qc.clone().cpu().numpy(), q.geo, q.generator()
        assert q.sync_status() == 0
        q.close()
    return out


# (m, n, p_r, p_c, f, lda): tile heights mb = 260 (two full boxes and a partial one), 128, 100,
# 200, 52 and 1024; ragged last tile rows; p_c = 5, 6 and 3 leave column groups uneven or empty
ENCODE_CASES = [
    (2077, 64, 8, 16, 4, 2080),
    (2048, 2048, 16, 16, 4, 2048),
    (600, 30, 6, 5, 2, 600),
    (1197, 36, 6, 6, 3, 1200),
    (103, 12, 2, 3, 1, 104),
    (4093, 256, 4, 8, 2, 4096),
]


@pytest.mark.parametrize("m,n,p_r,p_c,f,lda", ENCODE_CASES)
def test_streamed_encode_bits_and_oracle(m, n, p_r, p_c, f, lda):
    A = synth.gaussian(m, n, 5 + m)
    Qs, geo, (Gt, Gh) = encode_once(A, p_r, p_c, f, lda, True)
    Qr, _, _ = encode_once(A, p_r, p_c, f, lda, False)
    M, N = geo["M"], geo["N"]
    assert np.array_equal(Qs[:M, :N], Qr[:M, :N])
    g = O.geom(m, n, p_r, p_c, f)
    At = O.encode(g, Gt, Gh, A.astype(np.float32).astype(np.float64))
    # each checksum is a sum of at most p_r p_c FP32 products of O(1) terms
    err = np.abs(Qs[:M, :N].astype(np.float64) - At).max() / np.abs(At).max()
    assert err < 4 * (p_r + p_c) * U32


def factor_and_recover(A, p_r, p_c, f, b, plan, stream):
    m, n = A.shape
    with register_kernels(not stream):
        q = B.CodedQR(m, n, p_r, p_c, f, b, dtype="f32", mma="3xtf32", seed=9)
        q.encode(dev_a(A, m))
        for t in range(q.geo["panels"]):
            if plan.get(t):
                q.inject(plan[t])
                q.recover()
            q.factor(t, t + 1)
        Qc, Rc = q.factors()
        torch.cuda.synchronize()
        out = dict(Q=Qc.clone().cpu().numpy(), R=Rc.clone().cpu().numpy(), sets=q.decode_sets(),
                   status=q.sync_status())
        q.close()
    return out


# (m, n, p_r, p_c, f, b, {panel: tiles}): two grid columns and two R block rows at once; a
# checksum-row tile (row p_r) with a systematic one of the same grid column; mb = 260 and 128;
# the 16 x 16 grid with four checksums and four lost tiles, two of them in one grid column
DECODE_CASES = [
    (1040, 512, 4, 4, 2, 64, {2: [(1, 1), (3, 2)]}),
    (1040, 512, 4, 4, 2, 64, {1: [(0, 3), (4, 3)]}),
    (2048, 2048, 16, 16, 4, 128, {3: [(2, 5), (7, 9), (11, 9), (15, 14)]}),
]


@pytest.mark.parametrize("m,n,p_r,p_c,f,b,plan", DECODE_CASES)
def test_streamed_decode_bits_and_oracle(m, n, p_r, p_c, f, b, plan):
    A = synth.kappa_matrix(m, n, 10.0, seed=m + 3)
    s = factor_and_recover(A, p_r, p_c, f, b, plan, True)
    r = factor_and_recover(A, p_r, p_c, f, b, plan, False)
    assert s["status"] == 0 and r["status"] == 0
    assert s["sets"] == r["sets"]
    assert np.array_equal(s["Q"], r["Q"]) and np.array_equal(s["R"], r["R"])
    ref = O.run(A, p_r, p_c, f, b, seed=9, erasures=plan)
    assert s["sets"] == ref["sets"]
    g = ref["geom"]
    tol = n * 8 * U32 * 10.0  # n u kappa with the 3xTF32 unit roundoff (8 u) and kappa = 10
    assert np.abs(s["R"] - ref["R"]).max() / np.abs(ref["R"]).max() < tol
    assert np.abs(s["Q"][: g.M, :n] - ref["Q"][:, :n]).max() < tol
