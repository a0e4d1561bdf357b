"""Reverse mode through the coded least-squares path (hand-written adjoint kernels behind
torch.autograd.Function) against
  * FP64 central finite differences of the GPU forward itself, and
  * a CPU FP64 reference gradient: plain torch autograd through the defining formulas
    (Q R = G_0 A by torch.linalg.qr with positive diagonal, x from the normal equations),
    with G_0 built densely by the oracle.
The loss is L = <W_Q, Q> + <W_R, triu R> + <W_x, x> with fixed random weights.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_11943_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2311_11943_gb300.autograd import coded_lstsq  # noqa: E402


def weights(m, n, k, seed, batch=1):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((batch, m, n)), rng.standard_normal((batch, n, n)),
            rng.standard_normal((batch, n, k)))


def loss_gpu(A, y, W, opts):
    Q, R, x = coded_lstsq(A, y, **opts)
    WQ, WR, Wx = (torch.as_tensor(w, dtype=A.dtype, device="cuda") for w in W)
    return (WQ * Q).sum() + (WR * torch.triu(R)).sum() + (Wx * x).sum()


def reference_grad(A, y, W, p_r, p_c, f, seed):
    """CPU FP64 plain-torch gradient of the same loss (batch of problems)."""
    batch, m, n = A.shape
    g = O.geom(m, n, p_r, p_c, f, True)
    Gt, _ = O.generator(f, p_r, p_c, seed)
    G0 = torch.tensor(O.build_G0(g, Gt), dtype=torch.float64)
    At = torch.tensor(A, dtype=torch.float64, requires_grad=True)
    yt = torch.tensor(y, dtype=torch.float64, requires_grad=True)
    WQ, WR, Wx = (torch.tensor(w, dtype=torch.float64) for w in W)
    L = 0.0
    for i in range(batch):
        Ap = torch.cat([At[i], torch.zeros(g.m_pad - m, n, dtype=torch.float64)])
        Qr, Rr = torch.linalg.qr(G0 @ Ap)
        d = torch.sign(torch.diagonal(Rr))
        Qr = Qr * d
        Rr = d[:, None] * Rr
        x = torch.linalg.solve(At[i].T @ At[i], At[i].T @ yt[i])
        L = L + (WQ[i] * Qr[:m]).sum() + (WR[i] * torch.triu(Rr)).sum() + (Wx[i] * x).sum()
    L.backward()
    return At.grad.numpy(), yt.grad.numpy()


def small_problem(batch, m, n, k, kappa, seed):
    A = np.stack([synth.kappa_matrix(m, n, kappa, seed + i) for i in range(batch)])
    y = np.stack([synth.rhs(m, k, seed + 50 + i) for i in range(batch)])
    return A, y


@pytest.mark.parametrize("erasure", [False, True])
def test_adjoint_matches_fp64_finite_differences(erasure):
    m, n, k = 192, 32, 2
    opts = dict(p_r=4, p_c=4, f=1, b=8, seed=3,
                erasures={2: [(1, 2)]} if erasure else None)
    A, y = small_problem(1, m, n, k, 10.0, 11)
    W = weights(m, n, k, 5)
    Ad = torch.tensor(A, dtype=torch.float64, device="cuda", requires_grad=True)
    yd = torch.tensor(y, dtype=torch.float64, device="cuda", requires_grad=True)
    L = loss_gpu(Ad, yd, W, opts)
    L.backward()
    gA, gy = Ad.grad.detach().cpu().numpy(), yd.grad.detach().cpu().numpy()
    rng = np.random.default_rng(7)
    eps = 1e-6
    for _ in range(3):
        EA = rng.standard_normal(A.shape)
        Ey = rng.standard_normal(y.shape)
        with torch.no_grad():
            lp = loss_gpu(torch.tensor(A + eps * EA, device="cuda"),
                          torch.tensor(y + eps * Ey, device="cuda"), W, opts).item()
            lm = loss_gpu(torch.tensor(A - eps * EA, device="cuda"),
                          torch.tensor(y - eps * Ey, device="cuda"), W, opts).item()
        fd = (lp - lm) / (2 * eps)
        an = float((gA * EA).sum() + (gy * Ey).sum())
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_adjoint_matches_cpu_fp64_reference_gradient():
    m, n, k, batch = 256, 48, 1, 2
    p_r, p_c, f, seed = 4, 4, 2, 9
    A, y = small_problem(batch, m, n, k, 30.0, 21)
    W = weights(m, n, k, 8, batch)
    Ad = torch.tensor(A, dtype=torch.float64, device="cuda", requires_grad=True)
    yd = torch.tensor(y, dtype=torch.float64, device="cuda", requires_grad=True)
    L = loss_gpu(Ad, yd, W, dict(p_r=p_r, p_c=p_c, f=f, b=16, seed=seed,
                                  erasures={1: [(0, 3), (5, 1)]}))
    L.backward()
    gA_ref, gy_ref = reference_grad(A, y, W, p_r, p_c, f, seed)
    gA = Ad.grad.cpu().numpy()
    gy = yd.grad.cpu().numpy()
    assert np.abs(gA - gA_ref).max() <= 1e-9 * np.abs(gA_ref).max()
    assert np.abs(gy - gy_ref).max() <= 1e-9 * np.abs(gy_ref).max()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_c5_shape_against_cpu_fp64_reference(dtype):
    # A 8192 x 1024, kappa 1e3, y ~ N(0,1); grid 8 x 8, f = 1, b = 128, one node erased at the
    # start of the middle panel and recovered (FP32: 3xTF32 tensor-core trailing updates)
    m, n, k, batch = 8192, 1024, 1, 1
    p_r = p_c = 8
    f, b, seed, kappa = 1, 128, 5, 1e3
    A, y = small_problem(batch, m, n, k, kappa, 31)
    W = weights(m, n, k, 12, batch)
    td = torch.float64 if dtype == "f64" else torch.float32
    Ad = torch.tensor(A, dtype=td, device="cuda", requires_grad=True)
    yd = torch.tensor(y, dtype=td, device="cuda", requires_grad=True)
    L = loss_gpu(Ad, yd, W, dict(p_r=p_r, p_c=p_c, f=f, b=b, seed=seed,
                                  erasures={4: [(3, 6)]}))
    L.backward()
    gA_ref, gy_ref = reference_grad(A, y, W, p_r, p_c, f, seed)
    gA = Ad.grad.double().cpu().numpy()
    gy = yd.grad.double().cpu().numpy()
    # Tolerance from the gradient's own sensitivity: the path's backward-error target eps
    # (1e-12 in FP64, 1e-5 in FP32 storage) is a relative perturbation of the inputs, so the
    # reference gradient at a seeded perturbation of that size shows how far a gradient of a
    # computation meeting the target may move (linearly in eps; about 6e-4 for A and 2e-3 for
    # y at 1e-5 here, where the kappa^2 worst case would allow 1e-1); twice that is the bound,
    # and it stays below 1%, so a gradient wrong by 1% fails
    eps = 1e-12 if dtype == "f64" else 1e-5
    E = synth.gaussian(m, n, 99)[None]
    E *= eps * np.linalg.norm(A) / np.linalg.norm(E)
    e = synth.rhs(m, k, 98)[None]
    e *= eps * np.linalg.norm(y) / np.linalg.norm(e)
    gA_p, gy_p = reference_grad(A + E, y + e, W, p_r, p_c, f, seed)
    tolA = 2 * np.linalg.norm(gA_p - gA_ref) / np.linalg.norm(gA_ref)
    toly = 2 * np.linalg.norm(gy_p - gy_ref) / np.linalg.norm(gy_ref)
    assert tolA < 1e-2 and toly < 1e-2
    relA = np.linalg.norm(gA - gA_ref) / np.linalg.norm(gA_ref)
    rely = np.linalg.norm(gy - gy_ref) / np.linalg.norm(gy_ref)
    assert relA < tolA and rely < toly, (relA, rely, tolA, toly)
