"""The seeded input generators produce what the input recipe states (CPU only)."""
import numpy as np
import pytest

from paper_2311_11943_gb300 import synth


@pytest.mark.parametrize("m,n,kappa", [(96, 64, 1e2), (64, 64, 1e6), (200, 40, 1e3)])
def test_kappa_matrix_has_the_stated_singular_values(m, n, kappa):
    A = synth.kappa_matrix(m, n, kappa, seed=3)
    assert A.shape == (m, n) and A.flags.f_contiguous
    s = np.linalg.svd(A, compute_uv=False)
    want = kappa ** (-np.arange(n) / (n - 1))
    assert np.abs(s - want).max() < 1e-12 * max(1.0, kappa * 1e-6)
    assert abs(s[0] / s[-1] / kappa - 1) < 1e-8
    assert np.array_equal(A, synth.kappa_matrix(m, n, kappa, seed=3))
    assert not np.array_equal(A, synth.kappa_matrix(m, n, kappa, seed=4))


@pytest.mark.parametrize("m,n,kappa", [(96, 64, 1e2), (300, 200, 1e4)])
def test_device_kappa_matrix_has_the_stated_singular_values(m, n, kappa):
    # the FP32 torch form of the recipe (used where the host construction takes minutes),
    # run here on the CPU: column-major FP32, singular values kappa^(-(i-1)/(n-1)) to the FP32
    # orthogonality of the factors (multiplicative, about 1e-6) plus the rounding of A (u |A|)
    torch = pytest.importorskip("torch")
    A = synth.kappa_matrix_torch(m, n, kappa, seed=3, device="cpu")
    assert A.shape == (m, n) and A.stride() == (1, m) and A.dtype == torch.float32
    s = np.linalg.svd(A.double().numpy(), compute_uv=False)
    want = kappa ** (-np.arange(n) / (n - 1))
    # Weyl: the rounding E of A moves each singular value by at most |E|_2 <= u |A|_F
    u = 2.0 ** -24
    assert (np.abs(s - want) <= 1e-5 * want + u * np.linalg.norm(want)).all()
    assert abs(s[0] / s[-1] / kappa - 1) < 1e-3
    assert torch.equal(A, synth.kappa_matrix_torch(m, n, kappa, seed=3, device="cpu"))
    assert not torch.equal(A, synth.kappa_matrix_torch(m, n, kappa, seed=4, device="cpu"))


def test_haar_orthogonal_is_orthogonal_and_sign_normalised():
    rng = np.random.default_rng(1)
    Q = synth.haar_orthogonal(50, rng)
    assert np.abs(Q.T @ Q - np.eye(50)).max() < 1e-13
    # folding the signs of R's diagonal into Q makes the distribution Haar, so every entry is
    # symmetric about zero across draws
    firsts = [synth.haar_orthogonal(8, np.random.default_rng(s))[0, 0] for s in range(400)]
    assert abs(np.mean(firsts)) < 0.05


def test_gaussian_and_rhs_are_seeded_standard_normal():
    A = synth.gaussian(400, 300, 7)
    assert A.flags.f_contiguous and np.array_equal(A, synth.gaussian(400, 300, 7))
    assert abs(A.mean()) < 0.01 and abs(A.std() - 1) < 0.01
    y = synth.rhs(400, 2, 7)
    assert y.shape == (400, 2) and not np.array_equal(y[:, 0], A[:, 0])   # its own stream
    assert abs(y.mean()) < 0.1 and abs(y.std() - 1) < 0.1


@pytest.mark.parametrize("rows,cols,f,count", [(10, 10, 2, 2), (10, 10, 2, 20), (20, 20, 4, 4),
                                               (5, 4, 1, 4)])
def test_random_erasures_respect_the_per_row_and_column_limit(rows, cols, f, count):
    tiles = synth.random_erasures(rows, cols, f, count, seed=11)
    assert tiles == synth.random_erasures(rows, cols, f, count, seed=11)
    assert len(tiles) == count and len(set(tiles)) == count
    assert all(0 <= i < rows and 0 <= j < cols for i, j in tiles)
    assert max(np.bincount([i for i, _ in tiles])) <= f
    assert max(np.bincount([j for _, j in tiles])) <= f


@pytest.mark.parametrize("p,f,shift", [(4, 1, 0), (8, 2, 3), (6, 3, 5)])
def test_reverse_diagonal_has_f_failures_per_row_and_column(p, f, shift):
    tiles = synth.reverse_diagonal(p, f, shift)
    assert len(set(tiles)) == p * f
    assert list(np.bincount([i for i, _ in tiles], minlength=p)) == [f] * p
    assert list(np.bincount([j for _, j in tiles], minlength=p)) == [f] * p
    # anti-diagonals: i + j is constant modulo p for each k
    for k in range(f):
        assert {(i + j) % p for (i, j) in tiles[k::f]} == {(p - 1 - k - shift) % p}


def test_random_panels_are_distinct_sorted_and_skip_panel_zero():
    ts = synth.random_panels(32, 5, seed=2)
    assert ts == sorted(set(ts)) and len(ts) == 5 and all(1 <= t < 32 for t in ts)


def test_batched_shapes_follow_the_recipe():
    shapes = synth.batched_shapes(512, 4)
    assert len(shapes) == 512 and shapes == synth.batched_shapes(512, 4)
    ms = np.array([s[0] for s in shapes])
    ns = np.array([s[1] for s in shapes])
    assert ms.min() >= 256 and ms.max() <= 8192
    assert ns.min() >= 32 and ns.max() <= 256 and np.all(ns % 4 == 0)
    assert np.all(ms >= 4 * ns)
    # both ends of the ranges are reached by a batch of this size
    assert ms.min() < 600 and ms.max() > 7500 and ns.min() <= 40 and ns.max() >= 248
