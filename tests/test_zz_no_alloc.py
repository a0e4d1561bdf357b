"""coded_qr_panel_icgs_noalloc: the panel factorisation for callers that cannot allocate device
memory (caching allocators that must not be re-entered, hosts that gave all device memory to
another framework, latency-critical paths that must not take the allocation lock).  Its
scratch is a fixed array inside the library, so these tests check that two calls in a row --
the second one seeing the array as the first left it -- give the same panel as the allocating
path (coded_qr_factor's first panel step), within the parity tolerance of the other GPU tests,
and that the largest panel it accepts is one 1024-row slice per co-resident CTA,
min(160, #SMs) of them.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2311_11943_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2311_11943_gb300 import binding as B  # noqa: E402


def _colmajor(X, td):
    d = B.colmajor_empty(X.shape[0], X.shape[1], td)
    d.copy_(X if torch.is_tensor(X) else torch.from_numpy(np.ascontiguousarray(X)))
    return d


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_panel_matches_factor_panel_twice(dtype):
    td = torch.float64 if dtype == "f64" else torch.float32
    u = (np.finfo(np.float64).eps if dtype == "f64" else np.finfo(np.float32).eps) / 2
    m = n = 1024
    p, f, b = 8, 2, 128
    A = synth.kappa_matrix(m, n, 1e2, seed=21)
    q = B.CodedQR(m, n, p, p, f, b, dtype=dtype, seed=5)
    q.encode(_colmajor(A, td))
    Qc, Rc = q.factors()
    M = q.geo["M"]
    panel0 = Qc[:M, :b].clone()           # encoded panel before factorisation
    q.factor(0, 1)                        # allocating path: the handle's panel step
    torch.cuda.synchronize()
    assert q.sync_status() == 0
    Q_ref = Qc[:M, :b].double().cpu().numpy()
    R_ref = Rc[:b, :b].double().cpu().numpy()
    kappa = np.linalg.cond(panel0.double().cpu().numpy())
    tol = b * u * kappa * 10
    dt = B.CQR_F64 if dtype == "f64" else B.CQR_F32
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        Qp = _colmajor(panel0, td)
        Rp = torch.zeros((b, b), dtype=td, device="cuda").t()   # column-major b x b
        status = torch.full((4,), -1, dtype=torch.int32, device="cuda")
        st = B.coded_qr_panel_icgs_noalloc(dt, M, b, Qp.data_ptr(), Qp.stride(1), Rp.data_ptr(),
                                           Rp.stride(1), 0.0, status.data_ptr(), stream)
        assert st == B.CQR_OK, B.errstr(st)
        torch.cuda.synchronize()
        assert int(status[0].item()) == 0, call
        Qn = Qp.double().cpu().numpy()
        Rn = Rp.double().cpu().numpy()
        assert np.abs(Qn - Q_ref).max() < tol, (call, np.abs(Qn - Q_ref).max(), tol)
        assert np.abs(Rn - R_ref).max() / np.abs(R_ref).max() < tol, call
        assert np.abs(np.tril(Rn, -1)).max() == 0.0
    q.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    x = torch.zeros(8, device="cuda")
    assert B.coded_qr_panel_icgs_noalloc(B.CQR_F32, 1024, 257, x.data_ptr(), 1024, x.data_ptr(),
                                         257) == B.CQR_EINVAL
    assert B.coded_qr_panel_icgs_noalloc(B.CQR_F64, 10_000_000, 64, x.data_ptr(), 10_000_000,
                                         x.data_ptr(), 64) == B.CQR_EINVAL
    assert B.coded_qr_panel_icgs_noalloc(7, 64, 8, x.data_ptr(), 64, x.data_ptr(), 8) == B.CQR_EINVAL


def test_noalloc_row_limit_is_one_slice_per_resident_cta():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    lim = min(160, sms) * 1024
    bk = 8
    Q = B.colmajor_empty(lim + 1, bk, torch.float32)
    Q.copy_(torch.randn(bk, lim + 1, device="cuda", generator=torch.Generator("cuda").manual_seed(5)).t())
    R = B.colmajor_empty(bk, bk, torch.float32)
    R.zero_()
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    # at the limit: accepted and factored (an orthonormal panel)
    assert B.coded_qr_panel_icgs_noalloc(B.CQR_F32, lim, bk, Q.data_ptr(), lim + 1, R.data_ptr(), bk,
                                         0.0, st.data_ptr()) == B.CQR_OK
    torch.cuda.synchronize()
    assert int(st[0].item()) == 0
    Qd = Q[:lim].double()
    assert (Qd.t() @ Qd - torch.eye(bk, dtype=torch.float64, device="cuda")).abs().max().item() < 1e-4
    # one row more: rejected without a launch
    assert B.coded_qr_panel_icgs_noalloc(B.CQR_F32, lim + 1, bk, Q.data_ptr(), lim + 1, R.data_ptr(),
                                         bk, 0.0, st.data_ptr()) == B.CQR_EINVAL
