"""A seeded sweep of small random configurations through the oracle (CPU): shapes with
ragged m, grids, checksum counts, panel widths, R protection, block reorthogonalisation and
random erasure schedules.  Every case must satisfy what the paper and the mathematics fix:
R is the Householder R of the encoded matrix, the checksum relation Q_2 = G_v Q_1 holds at
the end, a run with erasures recovers the fault-free run, G_0 Q_1 is orthogonal, and the
square solve matches numpy."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_11943_gb300 import synth


def _cases(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        p_r = int(rng.integers(2, 9))
        p_c = int(rng.integers(2, 9))
        f = int(rng.integers(0, 1 + min(p_r, p_c) // 2))
        protect_r = bool(rng.integers(0, 2))
        n = p_c * int(rng.integers(2, 9))
        m = n if rng.integers(0, 3) == 0 else n + int(rng.integers(1, 3 * n))
        if m < p_r:
            continue
        b = int(rng.integers(1, n + 1))
        T = -(-n // b)
        erasures = {}
        if f > 0:
            gr, gc = p_r + f, p_c + (f if protect_r else 0)
            for t in rng.choice(T, size=min(T, int(rng.integers(1, 4))), replace=False):
                cnt = int(rng.integers(1, f + 1))
                erasures[int(t)] = synth.random_erasures(gr, gc, f, cnt, int(rng.integers(1 << 30)))
        out.append(dict(m=m, n=n, p_r=p_r, p_c=p_c, f=f, b=b, protect_r=protect_r,
                        rb=bool(rng.integers(0, 2)), erasures=erasures,
                        seed=int(rng.integers(1 << 30))))
    return out


CASES = _cases(40, 20231120)


@pytest.mark.parametrize("c", CASES, ids=["m%(m)d n%(n)d p%(p_r)dx%(p_c)d f%(f)d b%(b)d" % c
                                          for c in CASES])
def test_random_configuration_invariants(c):
    m, n = c["m"], c["n"]
    A = synth.kappa_matrix(m, n, 1e2, c["seed"])
    y = synth.rhs(m, 1, c["seed"]) if m == n else None
    kw = dict(seed=c["seed"] % 1000 + 1, protect_r=c["protect_r"], reorth_block=c["rb"])
    ref = O.run(A, c["p_r"], c["p_c"], c["f"], c["b"], y=y, **kw)
    g, Q, R, At = ref["geom"], ref["Q"], ref["R"], ref["At"]
    # R is the sign-normalised Householder R of the encoded matrix; Q~ is orthonormal
    Qh, Rh = np.linalg.qr(At[:, :n])
    Rh = Rh * np.sign(np.diag(Rh))[:, None]
    assert np.abs(R[:n, :n] - Rh).max() < 1e-11 * np.abs(Rh).max()
    assert np.abs(Q[:, :n].T @ Q[:, :n] - np.eye(n)).max() < 1e-11
    # the final form: Q_2 = G_v Q_1 and A = Q_1 R_1 (the padded rows of Q_1 are zero)
    if g.f > 0:
        Gv = np.kron(ref["Gt"], np.eye(g.mb))
        assert np.abs(Q[g.m_pad:, :n] - Gv @ Q[: g.m_pad, :n]).max() < 1e-10
    assert np.abs(A - Q[:m, :n] @ R[:n, :n]).max() < 1e-12 * np.abs(A).max() * n
    # post-orthogonalisation (Theorem G_0): orthonormal
    Qo = ref["Qo"]
    assert np.abs(Qo.T @ Qo - np.eye(n)).max() < 1e-10
    if y is not None:
        x = np.linalg.solve(A, y)
        assert np.abs(ref["x"] - x).max() < 1e-9 * np.abs(x).max()
    # erasures at the start of seeded panels, recovered before they run: same results
    if c["erasures"]:
        rec = O.run(A, c["p_r"], c["p_c"], c["f"], c["b"], y=y, erasures=c["erasures"], **kw)
        assert rec["n_recovered"] >= sum(len(v) for v in c["erasures"].values())
        for k in ("Q", "R", "Qo") + (("x",) if y is not None else ()):
            assert np.abs(rec[k] - ref[k]).max() < 1e-9 * max(1.0, np.abs(ref[k]).max()), k
