"""E1 MDS statistics on the GPU (one thread per square submatrix) against the oracle's
brute force, for the structured generator of the construction and a completely random one."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_11943_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2311_11943_gb300 import binding as B  # noqa: E402


def _gens(f, p_r, seed):
    Gt, _ = O.generator(f, p_r, 4, seed)
    Gr = Gt.copy()
    Gr[:, :f] = synth.unif01(f, f, seed)            # G~_1' i.i.d. Unif(0,1), same V~
    return Gt, Gr


@pytest.mark.parametrize("f,p_r", [(2, 16), (3, 12), (4, 24)])
def test_mds_stats_match_the_oracle(f, p_r):
    for G in _gens(f, p_r, 7):
        md, mc, cnt = B.coded_qr_mds_stats(G)
        rd, rc = O.mds_stats(G)
        assert cnt == sum(int(np.prod([f - i for i in range(k)]) / np.prod(range(1, k + 1))) *
                          int(np.prod([p_r - i for i in range(k)]) / np.prod(range(1, k + 1)))
                          for k in range(1, f + 1))
        assert md[1] == np.abs(G).min() and mc[1] == 1.0   # 1 x 1: exact on the GPU
        for k in range(0, f + 1):
            assert md[k] == pytest.approx(rd[k], rel=1e-10)
            assert mc[k] == pytest.approx(rc[k], rel=1e-8)


def test_mds_stats_singular_minor():
    G = np.array([[1.0, 2.0, 2.0, 5.0], [3.0, 1.0, 1.0, 7.0]])
    md, mc, _ = B.coded_qr_mds_stats(G)
    assert md[2] == 0.0 and mc[2] == np.inf


def test_mds_stats_full_size_f6_p64():
    Gt, _ = _gens(6, 64, 3)
    md, mc, cnt = B.coded_qr_mds_stats(Gt)
    assert cnt == 6 * 64 + 15 * 2016 + 20 * 41664 + 15 * 635376 + 6 * 7624512 + 74974368
    assert md[1] == np.abs(Gt).min()
    assert md[0] > 0.0 and np.isfinite(mc[0]) and mc[0] >= 1.0
