"""Batches of uneven tall-skinny coded QRs (one persistent factor launch, optionally recorded
into a CUDA graph) against the FP64 oracle run per instance.

Every instance is the single-instance method on its own matrix, so each one is compared with
oracle.run on the same A, generator seed, panel width and erasures: coded Q and R element by
element within the FP32 forward-error bound n u kappa(A) (times a small constant for the
decode of recovered tiles), decode index sets bit for bit.  Runs are deterministic (fixed
reduction orders), so a replayed graph and the step-by-step verbs reproduce a run exactly.
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
P_R, P_C, F, SEED = 8, 4, 2, 4


def to_dev(A):
    d = B.colmajor_empty(A.shape[0], A.shape[1], torch.float32)
    d.copy_(torch.from_numpy(np.ascontiguousarray(A.astype(np.float32))))
    return d


def rel(a, b):
    return np.abs(a - b).max() / max(1.0, np.abs(b).max())


def make_batch(count, seed, m_hi=1200, n_hi=96, n_lo=8, m_lo=128):
    shapes = synth.batched_shapes(count, seed, p_r=P_R, p_c=P_C, m_lo=m_lo, m_hi=m_hi, n_lo=n_lo,
                                  n_hi=n_hi)
    As = [synth.gaussian(m, n, seed * 1000 + i) for i, (m, n) in enumerate(shapes)]
    return shapes, As


def erasure_plan(bt, seed, count=None):
    """At most two random tiles (<= f per grid row / column) per instance, at one random panel."""
    rng = np.random.default_rng(seed)
    quads = []
    for i in range(bt.count if count is None else count):
        g = bt.geo[i]
        k = int(rng.integers(0, 3))
        if k == 0:
            continue
        t = int(rng.integers(0, g["panels"]))
        for (r, c) in synth.random_erasures(g["grid_rows"], g["grid_cols"], F, k, seed + 7 * i):
            quads.append((i, t, r, c))
    return quads


def oracle_instance(A, b, quads, i):
    er = {}
    for (k, t, r, c) in quads:
        if k == i:
            er.setdefault(t, []).append((r, c))
    return O.run(A.astype(np.float32).astype(np.float64), P_R, P_C, F, b, seed=SEED, erasures=er)


def check_instance(bt, i, A, quads, factor=50.0, post_orth=False):
    _, b = bt.tuning()
    ref = oracle_instance(A, b[i], quads, i)
    Qc, Rc = bt.factors(i)
    g = ref["geom"]
    Q = Qc.double().cpu().numpy()
    R = Rc.double().cpu().numpy()
    n = A.shape[1]
    tol = factor * n * U32 * np.linalg.cond(A)
    if post_orth:
        assert rel(Q[: g.m_pad, :n], ref["Qo"]) < tol, i
    else:
        assert rel(Q[: g.M, :], ref["Q"]) < tol, i
    assert rel(R, ref["R"]) < tol, i
    assert bt.decode_sets(i) == ref["sets"], i
    return ref


@pytest.fixture(scope="module")
def small_batch():
    shapes, As = make_batch(12, seed=41)
    bt = B.CodedQRBatch(shapes, P_R, P_C, F, b=0, seed=SEED)
    Ad = [to_dev(A) for A in As]
    yield bt, As, Ad
    bt.close()


@pytest.mark.parametrize("graph", [False, True])
def test_batched_run_matches_oracle_per_instance(small_batch, graph):
    bt, As, Ad = small_batch
    quads = erasure_plan(bt, 5)
    assert len(quads) > 0
    bt.run(Ad, quads, graph=graph)
    torch.cuda.synchronize()
    st, bad, _ = bt.sync_status()
    assert st == 0 and bad == -1
    for i, A in enumerate(As):
        check_instance(bt, i, A, quads)


def test_graph_replay_and_stepwise_verbs_reproduce_the_run_bitwise(small_batch):
    bt, As, Ad = small_batch
    quads = erasure_plan(bt, 6)
    bt.run(Ad, quads, graph=True)
    first = [tuple(t.clone() for t in bt.factors(i)) for i in range(bt.count)]
    bt.run(Ad, quads, graph=True)           # replay of the recorded graph
    for i in range(bt.count):
        Q, R = bt.factors(i)
        assert torch.equal(Q, first[i][0]) and torch.equal(R, first[i][1])
    bt.run(Ad, quads, graph=False)          # the same launches, not recorded
    for i in range(bt.count):
        Q, R = bt.factors(i)
        assert torch.equal(Q, first[i][0]) and torch.equal(R, first[i][1])
    # step by step: encode, factor up to each erasure panel, erase, recover, factor to the end
    t_of = {k: t for (k, t, _, _) in quads}
    bt.encode(Ad)
    bt.factor([t_of.get(i, bt.geo[i]["panels"]) for i in range(bt.count)])
    bt.inject([(k, r, c) for (k, _, r, c) in quads])
    assert bt.recover() > 0
    bt.factor()
    torch.cuda.synchronize()
    for i in range(bt.count):
        Q, R = bt.factors(i)
        assert torch.equal(Q, first[i][0]) and torch.equal(R, first[i][1])


@pytest.mark.parametrize("graph", [False, True])
def test_host_buffer_run_reproduces_the_device_run_bitwise(small_batch, graph):
    """CQR_BATCH_HOST_BUFFERS: the library copies every A from host memory into the systematic
    block of its encoded matrix and encodes in place there; the factors are those of the run
    on device buffers, bit for bit, for pinned and for pageable host arrays, and when the
    recorded graph is replayed with other host arrays."""
    bt, As, Ad = small_batch
    quads = erasure_plan(bt, 8)
    bt.run(Ad, quads, graph=graph)
    torch.cuda.synchronize()
    first = [tuple(t.clone() for t in bt.factors(i)) for i in range(bt.count)]

    def same():
        st, bad, _ = bt.sync_status()
        assert st == 0 and bad == -1
        for i in range(bt.count):
            Q, R = bt.factors(i)
            assert torch.equal(Q, first[i][0]) and torch.equal(R, first[i][1]), i

    pinned = []
    for A in As:
        h = torch.empty((A.shape[1], A.shape[0]), dtype=torch.float32, pin_memory=True)
        h.copy_(torch.from_numpy(np.ascontiguousarray(A.T.astype(np.float32))))
        pinned.append(h)
    for _ in range(2):
        bt.run([h.numpy().T for h in pinned], quads, graph=graph, host=True)
        same()
    plain = [np.asfortranarray(A.astype(np.float32)) for A in As]
    bt.run(plain, quads, graph=graph, host=True)
    same()
    with pytest.raises(AssertionError):
        bt.run([np.ascontiguousarray(a) for a in plain], quads, graph=graph, host=True)


def test_phase_clocks_count_every_cta_and_leave_the_factors_unchanged(small_batch):
    """coded_qr_batched_profile: every CTA of the launch adds its cycles per phase once; the
    run with the clocks on gives the same factors bit for bit."""
    bt, As, Ad = small_batch
    quads = erasure_plan(bt, 9)
    assert len(quads) > 0
    bt.run(Ad, quads, graph=False)
    torch.cuda.synchronize()
    first = [tuple(t.clone() for t in bt.factors(i)) for i in range(bt.count)]
    bt.profile(True)
    try:
        bt.phases(reset=True)
        for graph in (False, True):
            bt.run(Ad, quads, graph=graph)
            ph, ctas = bt.phases(reset=True)
            assert ctas > 0
            for k in ("panel", "s_product", "rbar_reduce", "update", "recover"):
                assert ph[k] > 0, (graph, k, ph)
            assert all(v >= 0 for v in ph.values())
            for i in range(bt.count):
                Q, R = bt.factors(i)
                assert torch.equal(Q, first[i][0]) and torch.equal(R, first[i][1]), i
        ph, ctas = bt.phases(reset=False)
        assert ctas == 0 and sum(ph.values()) == 0
    finally:
        bt.profile(False)
    bt.run(Ad, quads, graph=True)   # clocks off again: a new recording without them
    bt.sync_status()
    ph, ctas = bt.phases(reset=False)
    assert ctas == 0


@pytest.mark.parametrize("G", [1, 2, 4, 8])
@pytest.mark.parametrize("width", [16, 32, 64])
def test_every_cluster_size_and_width(small_batch, G, width):
    bt, As, Ad = small_batch
    bt.set_tuning(G, [width] * bt.count)
    quads = erasure_plan(bt, 7)
    bt.run(Ad, quads, graph=False)
    torch.cuda.synchronize()
    assert bt.sync_status()[0] == 0
    for i in (0, bt.count // 2, bt.count - 1):
        check_instance(bt, i, As[i], quads)
    bt.set_tuning(2)


def test_post_orth_in_place(small_batch):
    bt, As, Ad = small_batch
    quads = erasure_plan(bt, 8)
    bt.run(Ad, quads, graph=True, post_orth=True)
    torch.cuda.synchronize()
    for i in range(0, bt.count, 3):
        check_instance(bt, i, As[i], quads, post_orth=True)


def test_panel_worked_on_in_l2_when_it_does_not_fit_shared_memory():
    # 6400 encoded rows in one CTA with b = 64: the panel slice exceeds the shared-memory pool
    # and is factorised in place in global memory
    shapes = [(5120, 64), (600, 40)]
    As = [synth.gaussian(m, n, 90 + i) for i, (m, n) in enumerate(shapes)]
    bt = B.CodedQRBatch(shapes, P_R, P_C, F, b=64, seed=SEED)
    bt.set_tuning(1, [64, 64])
    Ad = [to_dev(A) for A in As]
    quads = [(0, 0, 3, 1), (1, 0, 9, 2)]
    bt.run(Ad, quads, graph=False)
    torch.cuda.synchronize()
    assert bt.sync_status()[0] == 0
    for i in range(2):
        check_instance(bt, i, As[i], quads)
    bt.close()


def test_autotune_keeps_results_within_parity(small_batch):
    bt, As, Ad = small_batch
    G = bt.autotune(Ad, erasure_plan(bt, 11), reps=1)
    assert G in (1, 2, 4, 8)
    cl, widths = bt.tuning()
    assert cl == G and all(w in (16, 32, 64) for w in widths)
    torch.cuda.synchronize()
    for i in (0, bt.count - 1):
        check_instance(bt, i, As[i], [])


def test_unrecoverable_pattern_launches_nothing(small_batch):
    bt, As, Ad = small_batch
    g = bt.geo[0]
    # three tiles of one grid column with f = 2
    quads = [(0, 0, r, 1) for r in range(3)]
    with pytest.raises(B.CodedQRError) as e:
        bt.run(Ad, quads, graph=False)
    assert e.value.status == B.CQR_EUNRECOVERABLE
    assert g["grid_rows"] >= 3


def test_breakdown_is_reported_for_its_instance_only():
    shapes = [(256, 32), (256, 32), (320, 48)]
    As = [synth.gaussian(m, n, 70 + i) for i, (m, n) in enumerate(shapes)]
    As[1][:, 5] = 0.0                           # a zero column: r_55 = 0
    bt = B.CodedQRBatch(shapes, P_R, P_C, F, b=16, seed=SEED)
    Ad = [to_dev(A) for A in As]
    bt.run(Ad, [], graph=False)
    torch.cuda.synchronize()
    st, bad, _ = bt.sync_status()
    assert st == B.CQR_EBREAKDOWN and bad == 1
    for i in (0, 2):
        check_instance(bt, i, As[i], [])
    bt.close()


def test_full_size_batch_sampled_instances():
    # 512 instances, m in [256, 8192], n in [32, 256] (m >= 4 n), f = 2 per instance and up to
    # two erased tiles each; the smallest, a middle and the largest instance vs the oracle
    shapes = synth.batched_shapes(512, 4)
    bt = B.CodedQRBatch(shapes, P_R, P_C, F, b=0, seed=SEED)
    cost = [m * n * n for (m, n) in shapes]
    order = np.argsort(cost)
    pick = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    As, Ad = {}, []
    for i, (m, n) in enumerate(shapes):
        A = synth.gaussian(m, n, 4000 + i, dtype=np.float32)
        if i in pick:
            As[i] = A
        Ad.append(to_dev(A))
    quads = erasure_plan(bt, 9)
    bt.run(Ad, quads, graph=True)
    torch.cuda.synchronize()
    st, bad, _ = bt.sync_status()
    assert st == 0 and bad == -1
    for i in pick:
        check_instance(bt, i, As[i], quads)
    bt.close()
