"""Bounded waits leave the kernel and report CQR_ETIMEOUT (needs a GB300; through the C ABI).

Nothing here faults or hangs a GPU: the panel launches are correct, only the bound of their
waits between CTAs is set to a few hundred SM cycles (coded_qr_set_wait_limit), so every
exchange runs out before its peers' partial sums arrive.  Each CTA then records
CQR_ETIMEOUT, every CTA of the launch leaves at its next wait, and the later launches of the
factorisation see the recorded error and leave too.  The status must come back within a
second; with the default bound restored and the matrix encoded again, the same handle
factors correctly.
"""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_11943_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2311_11943_gb300 import binding as B  # noqa: E402


# (m, n, p_r, p_c, f, b, dtype, mma): the register-resident cluster panel (FP32, its exchange
# of partial vectors by st.async into every CTA, bounded mbarrier waits), the cooperative
# grid-barrier panel (FP64, 10240 rows: too tall for one cluster's shared memory) and the
# two-level exchange (FP32, 20480 x 256 with the sub-panel schedule off: clusters of 8 whose
# leaders publish tagged sums that every CTA polls)
CASES = [(1024, 1024, 8, 8, 2, 64, "f32", "3xtf32"), (8192, 256, 8, 4, 2, 64, "f64", "simt"),
         (16384, 1024, 16, 8, 4, 256, "f32", "3xtf32")]


@pytest.mark.parametrize("case", CASES)
def test_expired_waits_leave_and_report_timeout(case, monkeypatch):
    m, n, p_r, p_c, f, b, dtype, mma = case
    monkeypatch.setenv("CQR_PANEL_SUB", "0")
    td = torch.float64 if dtype == "f64" else torch.float32
    A = synth.kappa_matrix(m, n, 1e2, seed=41)
    Ad = B.colmajor_empty(m, n, td)
    Ad.copy_(torch.from_numpy(A))
    q = B.CodedQR(m, n, p_r, p_c, f, b, dtype=dtype, mma=mma, seed=6)
    q.encode(Ad)
    torch.cuda.synchronize()
    q.set_wait_limit(200)
    t0 = time.perf_counter()
    q.factor(0, -1)
    st = q.sync_status()
    dt = time.perf_counter() - t0
    assert st == B.CQR_ETIMEOUT, B.errstr(st)
    assert dt < 1.0, dt
    # the default bound again: a new encode clears the status and the factors are right
    q.set_wait_limit(0)
    q.encode(Ad)
    q.factor(0, -1)
    torch.cuda.synchronize()
    assert q.sync_status() == 0
    _, Rc = q.factors()
    R = Rc.double().cpu().numpy()
    q.close()
    ref = O.run(A, p_r, p_c, f, b, seed=6)
    u = np.finfo(np.float64 if dtype == "f64" else np.float32).eps / 2
    if mma == "3xtf32":
        u *= 8
    assert np.abs(R - ref["R"]).max() < n * u * 1e2 * np.abs(ref["R"]).max()


def test_wait_limit_rejects_a_negative_bound():
    q = B.CodedQR(256, 256, 4, 4, 1, 32, dtype="f64", seed=1)
    with pytest.raises(B.CodedQRError):
        q.set_wait_limit(-1)
    q.close()
