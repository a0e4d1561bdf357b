"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

Holds none of the method's arithmetic: only random matrices, right-hand sides and
erasure patterns.  The paper's only workload is a random dense matrix (Section 6,
n = 24000); these generators stand in for it with the shapes of the benchmark configs.
"""
import numpy as np


def gaussian(m, n, seed, dtype=np.float64):
    """i.i.d. N(0,1) entries, column-major."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((m, n)).astype(dtype))


def haar_orthogonal(n, rng):
    """Haar-distributed orthogonal matrix: QR of a Gaussian matrix with the signs of R's
    diagonal folded into Q (Mezzadri, Notices AMS 2007)."""
    Z = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    return Q * np.sign(np.diag(R))[None, :]


def kappa_matrix(m, n, kappa, seed, dtype=np.float64):
    """A = U diag(sigma) V^T with U (m x n, orthonormal columns of a Haar matrix), V Haar,
    sigma_i = kappa^(-(i-1)/(n-1)): 2-norm condition number kappa."""
    rng = np.random.default_rng(seed)
    U = haar_orthogonal(m, rng)[:, :n]
    V = haar_orthogonal(n, rng)
    sig = kappa ** (-np.arange(n) / max(n - 1, 1))
    return np.asfortranarray(((U * sig[None, :]) @ V.T).astype(dtype))


def kappa_matrix_torch(m, n, kappa, seed, device="cuda"):
    """The recipe of kappa_matrix drawn with torch on `device` in FP32, for sizes where the
    host construction takes minutes (16384^2: QR of two Gaussian matrices).  U (m x n,
    orthonormal columns) and V (n x n) come from torch.linalg.qr of N(0,1) matrices drawn by
    a torch.Generator seeded with `seed`, with the signs of R's diagonal folded in (Haar,
    Mezzadri 2007); A = U diag(sigma) V^T with sigma_i = kappa^(-(i-1)/(n-1)), formed in full
    FP32 (TF32 off).  The FP32 factors are orthogonal to about 1e-6, which perturbs sigma
    multiplicatively by that much, so the 2-norm condition number stays kappa to about 1e-6
    relative before the final FP32 rounding of A.  Returns a column-major FP32 tensor
    (stride (1, m)) on `device`.  The same seed on the same device and library versions gives
    the same bytes; the tests hand exactly those bytes to both the CUDA path and the oracle."""
    import torch
    gen = torch.Generator(device=device).manual_seed(int(seed))
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        Z = torch.randn(m, n, generator=gen, device=device, dtype=torch.float32)
        U, Ru = torch.linalg.qr(Z)
        U *= torch.sign(torch.diagonal(Ru))[None, :]
        del Z, Ru
        Z = torch.randn(n, n, generator=gen, device=device, dtype=torch.float32)
        V, Rv = torch.linalg.qr(Z)
        V *= torch.sign(torch.diagonal(Rv))[None, :]
        del Z, Rv
        sig = (kappa ** (-torch.arange(n, device=device, dtype=torch.float64)
                         / max(n - 1, 1))).to(torch.float32)
        U *= sig[None, :]
        # column-major m x n: store A^T row-major, A = (U Sigma) V^T  <=>  A^T = V (U Sigma)^T
        At = torch.matmul(V, U.t())
        del U, V
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return At.t()


def rhs(m, k, seed, dtype=np.float64):
    rng = np.random.default_rng(seed + 7919)
    y = rng.standard_normal((m, k)).astype(dtype)
    return np.asfortranarray(y)


def random_erasures(grid_rows, grid_cols, f, count, seed):
    """`count` distinct node tiles (i, j) with at most f per grid row and per grid column."""
    rng = np.random.default_rng(seed + 104729)
    for _ in range(10000):
        cells = rng.permutation(grid_rows * grid_cols)
        rows = np.zeros(grid_rows, int)
        cols = np.zeros(grid_cols, int)
        out = []
        for cell in cells:
            i, j = divmod(int(cell), grid_cols)
            if rows[i] < f and cols[j] < f:
                out.append((i, j))
                rows[i] += 1
                cols[j] += 1
                if len(out) == count:
                    return out
    raise ValueError("no pattern found")


def reverse_diagonal(p, f, shift=0):
    """Reverse-diagonal failure pattern of the experiments (Section 6): systematic nodes
    (i, (p-1-i-k-shift) mod p) for k < f; f failures per grid row and column."""
    return [(i, (p - 1 - i - k - shift) % p) for i in range(p) for k in range(f)]


def random_panels(T, count, seed):
    rng = np.random.default_rng(seed + 1299709)
    return sorted(int(t) for t in rng.choice(np.arange(1, T), size=count, replace=False))


def batched_shapes(count, seed, p_r=8, p_c=4, m_lo=256, m_hi=8192, n_lo=32, n_hi=256):
    """Shapes of independent tall-skinny problems: m ~ U[m_lo, m_hi], n ~ U[n_lo, n_hi]
    restricted to multiples of p_c, resampled until m >= 4 n."""
    rng = np.random.default_rng(seed)
    shapes = []
    while len(shapes) < count:
        m = int(rng.integers(m_lo, m_hi + 1))
        n = int(rng.integers(n_lo // p_c, n_hi // p_c + 1)) * p_c
        if m >= 4 * n:
            shapes.append((m, n))
    return shapes


def unif01(m, n, seed):
    """i.i.d. Unif(0,1) entries (the completely random generator block of the MDS comparison)."""
    rng = np.random.default_rng(seed + 15485863)
    return rng.random((m, n))
