"""coded_qr_probe_exchange: the panel's per-column reductions alone (needs a GB300).

The probe runs the reductions of one panel through the panel kernels' own exchange code with
no column arithmetic; every CTA contributes a + 1 to entry a, so each reduced entry must come
back as exactly G (a + 1) -- the call returns CQR_ECUDA otherwise.  Covered: the register
panel's cluster exchange, the shared-memory panel in one cluster and with the two-level
exchange (the 16384^2 workload's 20480 x 256 panel), and the rejection of a panel that the
chosen kind cannot hold.
"""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2311_11943_gb300 import binding as B  # noqa: E402


@pytest.mark.parametrize("kind,M,bk", [(0, 5120, 128), (0, 1280, 32), (1, 2048, 64),
                                       (1, 20480, 256)])
def test_probe_sums_are_exact_and_time_is_positive(kind, M, bk):
    us = B.probe_exchange(kind, M, bk, reps=2)
    # a reduction takes at least a shared-memory round trip and well under a millisecond
    assert 0.05 < us < 1000.0


def test_probe_rejects_a_panel_the_kind_cannot_hold():
    with pytest.raises(B.CodedQRError) as e:
        B.probe_exchange(0, 5120, 200)  # the register panel holds at most 128 columns
    assert e.value.status == B.CQR_EINVAL
