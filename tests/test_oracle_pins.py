"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test names the passage it checks.  None of them re-types an oracle formula: they use
worked-example values, identities the paper proves, independent library routines
(LAPACK Householder QR, dense Kronecker products, numpy solvers) and brute force.
"""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_11943_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
TAU = 1.0 / np.sqrt(2.0)


def _gold(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


# --------------------------------------------------------------------------- a1 generator
def test_splitmix64_published_outputs():
    g = _gold("splitmix64_seed0.json")
    assert [v for v in O.splitmix64(g["seed"], 4)] == [int(h, 16) for h in g["outputs_hex"]]


def test_generator_draws_unif01():
    # Construction 'Q-factor checksum-generator matrix': V~ entries i.i.d. Unif(0,1)
    vals = []
    for seed in range(200):
        Gt, Gh = O.generator(4, 16, 16, seed)
        vals.append(Gt[:, 4:].ravel())
        vals.append(Gh.ravel())
    v = np.concatenate(vals)
    assert v.min() > 0.0 and v.max() < 1.0
    assert abs(v.mean() - 0.5) < 0.01 and abs(v.var() - 1.0 / 12.0) < 0.005


@pytest.mark.parametrize("f,p_r,gdist", [(1, 2, 0), (2, 8, 0), (4, 16, 0), (3, 6, 1)])
def test_G0_observation_identity(f, p_r, gdist):
    # Observation in the proof of Theorem 'G_0': G_1 = -1/2 V V^T  =>  G_0^T G_0 = I + G^T G,
    # with G = G~ (x) I (Eq. (generator_mat1)) built here by numpy.kron, G_0 by the oracle.
    Gt, _ = O.generator(f, p_r, p_r, seed=11, gdist=gdist)
    mb = 3
    g = O.geom(p_r * mb, p_r, p_r, p_r, f)
    G = np.kron(Gt, np.eye(mb))
    G0 = O.build_G0(g, Gt)
    lhs = G0.T @ G0
    rhs = np.eye(g.m_pad) + G.T @ G
    assert np.abs(lhs - rhs).max() < 1e-13


def test_G0_identity_fails_for_planted_wrong_generator():
    # planted mistake: +1/2 instead of -1/2 in G~_1 breaks the identity (sensitivity of the pin)
    Gt, _ = O.generator(2, 8, 8, seed=3)
    V = Gt[:, 2:]
    Gbad = Gt.copy()
    Gbad[:, :2] = +0.5 * V @ V.T
    g = O.geom(8 * 2, 8, 8, 8, 2)
    G0 = O.build_G0(g, Gbad)
    G = np.kron(Gbad, np.eye(2))
    assert np.abs(G0.T @ G0 - (np.eye(16) + G.T @ G)).max() > 1e-2


@pytest.mark.parametrize("f,p_r,mb", [(1, 4, 2), (2, 8, 3), (3, 6, 2)])
def test_det_G0(f, p_r, mb):
    # Proof of Theorem 'G_0', claim 2: det(G_0) = (-1)^(m-c) det(I + 1/2 V V^T) != 0
    Gt, _ = O.generator(f, p_r, p_r, seed=5)
    g = O.geom(p_r * mb, p_r, p_r, p_r, f)
    G0 = O.build_G0(g, Gt)
    V = np.kron(Gt[:, f:], np.eye(mb))
    s1, l1 = np.linalg.slogdet(G0)
    s2, l2 = np.linalg.slogdet(np.eye(g.c) + 0.5 * V @ V.T)
    assert s2 > 0
    assert s1 == (-1) ** (g.m_pad - g.c) * s2
    assert abs(l1 - l2) < 1e-10


@pytest.mark.parametrize("f,p_r", [(1, 2), (2, 4), (2, 6), (3, 6), (4, 8)])
def test_mds_every_square_submatrix_nonsingular(f, p_r):
    # Theorem 'prob_det' (MDS w.p. 1 when 2f <= p_r): brute force over all square submatrices
    for seed in range(5):
        Gt, Gh = O.generator(f, p_r, p_r, seed)
        for G in (Gt, Gh.T):
            for k in range(1, f + 1):
                for rows in itertools.combinations(range(G.shape[0]), k):
                    for cols in itertools.combinations(range(G.shape[1]), k):
                        sub = G[np.ix_(rows, cols)]
                        assert abs(np.linalg.det(sub)) > 1e-12


def test_invert_small_matches_numpy():
    rng = np.random.default_rng(0)
    for k in (1, 2, 3, 5, 8):
        G = rng.uniform(size=(k, k)) + k * np.eye(k) * 0.1
        assert np.allclose(O.invert_small(G), np.linalg.inv(G), rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------- a2 encode
@pytest.mark.parametrize("m,n,p_r,p_c,f,pr", [(24, 16, 4, 4, 1, True), (30, 24, 6, 4, 2, True),
                                              (35, 18, 6, 6, 3, True), (32, 16, 4, 4, 2, False)])
def test_encode_equals_kronecker_definition(m, n, p_r, p_c, f, pr):
    # Eq. (encoding) with G_v = G~ (x) I, G_h = G~_h (x) I (Eq. (tildeG_eq)), A zero-padded
    A = synth.gaussian(m, n, 3)
    g = O.geom(m, n, p_r, p_c, f, pr)
    Gt, Gh = O.generator(f, p_r, p_c, 9)
    At = O.encode(g, Gt, Gh, A)
    Ap = np.zeros((g.m_pad, n))
    Ap[:m] = A
    Gv = np.kron(Gt, np.eye(g.mb))
    top = Ap
    bot = Gv @ Ap
    if pr:
        Ghk = np.kron(Gh, np.eye(g.nb))
        ref = np.block([[top, top @ Ghk], [bot, bot @ Ghk]])
    else:
        ref = np.vstack([top, bot])
    assert At.shape == ref.shape
    assert np.abs(At - ref).max() < 1e-13 * max(1.0, np.abs(ref).max())


def test_worked_example_encode_and_G0():
    ex = _gold("worked_example_f1_p2.json")
    A = np.array(ex["A"])
    v = ex["v"]
    Gt = np.array([[ex["g1"], v]])
    Gh = np.array(ex["Gh"])
    g = O.geom(2, 2, 2, 2, 1)
    At = O.encode(g, Gt, Gh, A)
    assert np.array_equal(At, np.array(ex["At_expected"]))
    G0 = O.build_G0(g, Gt)
    assert np.array_equal(G0, np.array(ex["G0_expected"]))
    assert np.allclose(G0.T @ G0, np.array(ex["G0tG0_expected"]), atol=0, rtol=1e-15)


def test_worked_example_recovery_formulas():
    # After the first MGS iteration node (1,1) fails: Q11 = (Q31 - v Q21)/g1, R11 = R13 - R12
    ex = _gold("worked_example_f1_p2.json")
    A = np.array(ex["A"])
    v, g1 = ex["v"], ex["g1"]
    Gt = np.array([[g1, v]])
    Gh = np.array(ex["Gh"])
    g = O.geom(2, 2, 2, 2, 1)
    Q = O.encode(g, Gt, Gh, A)
    R = np.zeros((3, 3), order="F")
    O.factor(Q, R, 2, 1, 0, 1)
    Q0, R0 = Q.copy(order="F"), R.copy(order="F")
    q11 = (Q0[2, 0] - v * Q0[1, 0]) / g1
    r11 = R0[0, 2] - R0[0, 1]
    mask = np.zeros((3, 3), np.uint8)
    O.inject(g, [(0, 0)], mask, Q, R)
    assert np.isnan(Q[0, 0]) and np.isnan(R[0, 0])
    sets, nrec = O.recover(g, Gt, Gh, mask, Q, R)
    assert nrec == 1
    tol = 4 * np.finfo(float).eps
    assert abs(Q[0, 0] - q11) <= tol * abs(q11) and abs(Q[0, 0] - Q0[0, 0]) <= tol * abs(q11)
    assert abs(R[0, 0] - r11) <= tol * abs(r11) and abs(R[0, 0] - R0[0, 0]) <= tol * abs(r11)


# --------------------------------------------------------------------------- a3-a5 factor
def _signfix(Q, R):
    s = np.sign(np.diag(R))
    s[s == 0] = 1
    return Q * s[None, :], R * s[:, None]


@pytest.mark.parametrize("m,n,p,f,b", [(64, 64, 4, 1, 8), (96, 64, 4, 2, 16), (50, 40, 5, 2, 7),
                                       (64, 64, 4, 0, 16)])
def test_factor_matches_householder_of_encoded(m, n, p, f, b):
    # R equals the (sign-normalised) Householder R of the encoded matrix At (not of A):
    # Section 2.3 (QR of At) with LAPACK's Householder QR as the independent routine.
    A = synth.gaussian(m, n, 1)
    out = O.run(A, p, p, f, b, seed=2)
    g, Q, R, At = out["geom"], out["Q"], out["R"], out["At"]
    Qh, Rh = np.linalg.qr(At[:, :n])
    Qh, Rh = _signfix(Qh, Rh)
    assert np.abs(R[:n, :n] - Rh).max() < 1e-12 * np.abs(Rh).max()
    assert np.abs(Q[:, :n] - Qh).max() < 1e-11
    if f > 0:
        # checksum columns of R: R_2 = Q_H^T At[:, n:] (Householder Q restricted to rank n)
        assert np.abs(R[:n, n:] - Qh.T @ At[:, n:]).max() < 1e-11 * np.abs(At).max()
    assert np.all(np.diag(R[:n, :n]) > 0)
    assert np.abs(np.tril(R[:n, :n], -1)).max() == 0.0


@pytest.mark.parametrize("f", [1, 2])
def test_corollary_final_form_and_checksums_every_iteration(f):
    # Lemma 'checksum preservation' (Q_2 = G_v Q_1, R_2 = R_1 G_h at every iteration) and
    # Corollary 'final form' (At = [Q_1; G_v Q_1][R_1, R_1 G_h], A = Q_1 R_1).
    m = n = 48
    p, b = 4, 6
    A = synth.gaussian(m, n, 4)
    out = O.run(A, p, p, f, b, seed=6, keep_states=True)
    g, Gt, Gh = out["geom"], out["Gt"], out["Gh"]
    Gv = np.kron(Gt, np.eye(g.mb))
    Ghk = np.kron(Gh, np.eye(g.nb))
    for Q, R in out["states"]:
        assert np.abs(Q[g.m_pad:] - Gv @ Q[: g.m_pad]).max() < 1e-12
        assert np.abs(R[:, n:] - R[:, :n] @ Ghk).max() < 1e-12
    Q, R = out["Q"], out["R"]
    assert np.abs(out["At"] - Q @ R).max() < 1e-12
    assert np.abs(A - Q[:m, :n] @ R[:n, :n]).max() < 1e-12
    assert np.abs(Q[:, :n].T @ Q[:, :n] - np.eye(n)).max() < 1e-12
    assert np.abs(R[n:]).max() == 0.0  # checksum columns are never pivots
    assert np.abs(Q[:, n:]).max() < 1e-12  # their residual vanishes


def test_block_width_invariance():
    # BMGS gives the same factors for any panel width (exact arithmetic); b=1 is column MGS.
    A = synth.gaussian(40, 40, 8)
    ref = O.run(A, 4, 4, 1, 40, seed=1)
    for b in (1, 3, 8, 10):
        out = O.run(A, 4, 4, 1, b, seed=1)
        assert np.abs(out["R"] - ref["R"]).max() < 1e-12
        assert np.abs(out["Q"][:, :40] - ref["Q"][:, :40]).max() < 1e-12


def test_reorth_criterion_restores_orthogonality():
    # ICGS: the reorthogonalisation pass removes the loss of orthogonality of one CGS pass
    # on nearly dependent panel columns (Appendix A, ICGS paragraph).
    rng = np.random.default_rng(0)
    M, b = 200, 16
    base = rng.standard_normal((M, 1))
    P = base + 1e-7 * rng.standard_normal((M, b))
    Q1 = np.asfortranarray(P.copy())
    R1 = np.zeros((b, b), order="F")
    n1 = O.icgs_panel(Q1, R1, 0, b, tau=TAU)
    Q0 = np.asfortranarray(P.copy())
    R0 = np.zeros((b, b), order="F")
    n0 = O.icgs_panel(Q0, R0, 0, b, tau=0.0)
    e1 = np.abs(Q1.T @ Q1 - np.eye(b)).max()
    e0 = np.abs(Q0.T @ Q0 - np.eye(b)).max()
    assert n1 > 0 and n0 == 0
    assert e1 < 1e-14 and e0 > 1e3 * e1
    assert np.abs(Q1 @ R1 - P).max() < 1e-14


def test_breakdown_reported():
    # a zero column of A gives a zero column of At (G_v A and A G_h are linear): the pivot
    # r_jj is exactly zero and the factorisation reports breakdown instead of dividing by 0.
    A = synth.gaussian(32, 32, 1)
    A[:, 5] = 0.0
    g = O.geom(32, 32, 4, 4, 1)
    Gt, Gh = O.generator(1, 4, 4, 1)
    Q = O.encode(g, Gt, Gh, A)
    R = np.zeros((g.N, g.N), order="F")
    with pytest.raises(O.OracleError) as e:
        O.factor(Q, R, 32, 4)
    assert e.value.rc == O.EBREAKDOWN


# --------------------------------------------------------------------------- a6-a7 recovery
def _erasure_sets(g, f, max_size):
    nodes = [(i, j) for i in range(g.grid_rows) for j in range(g.grid_cols)]
    for k in range(1, max_size + 1):
        for sub in itertools.combinations(nodes, k):
            yield list(sub)


def _ok_pattern(g, f, tiles):
    rows, cols = {}, {}
    for i, j in tiles:
        rows[i] = rows.get(i, 0) + 1
        cols[j] = cols.get(j, 0) + 1
    return max(rows.values()) <= f and max(cols.values()) <= f


@pytest.mark.parametrize("p,f,max_size", [(2, 1, 3), (4, 1, 2), (4, 2, 2), (6, 3, 2)])
def test_recover_bruteforce_every_pattern(p, f, max_size):
    # MDS decodability (Theorem 'prob_det' + recovery Lemma): every pattern with <= f erasures
    # per grid row and column, at a mid-factorisation iteration, restores the pre-erasure state.
    n = 4 * p
    b = 2
    A = synth.gaussian(n, n, 5)
    g = O.geom(n, n, p, p, f)
    Gt, Gh = O.generator(f, p, p, 13)
    Q = O.encode(g, Gt, Gh, A)
    R = np.zeros((g.N, g.N), order="F")
    O.factor(Q, R, n, b, 0, 3)
    count = 0
    for tiles in _erasure_sets(g, f, max_size):
        if not _ok_pattern(g, f, tiles):
            continue
        Qe, Re = Q.copy(order="F"), R.copy(order="F")
        mask = np.zeros((g.grid_rows, g.grid_cols), np.uint8)
        O.inject(g, tiles, mask, Qe, Re)
        O.recover(g, Gt, Gh, mask, Qe, Re)
        assert np.abs(Qe - Q).max() < 1e-11, tiles
        assert np.abs(Re - R).max() < 1e-11, tiles
        count += 1
    assert count > 0


@pytest.mark.parametrize("p,f", [(4, 1), (4, 2), (6, 3), (8, 4)])
def test_recover_reverse_diagonal_pattern(p, f):
    # Section 6 failure model: reverse-diagonal pattern, f failures per grid row and column
    n = 4 * p
    A = synth.gaussian(n, n, 2)
    out0 = O.run(A, p, p, f, 4, seed=3)
    er = {t: synth.reverse_diagonal(p, f, shift=t) for t in range(1, n // 4)}
    out1 = O.run(A, p, p, f, 4, seed=3, erasures=er)
    assert out1["n_recovered"] >= p * f
    # decode rounding is bounded by kappa(G^) u |Q| per recovery and compounds over the
    # recovered iterations: tolerance 10 * kappa_max * u * (#iterations with erasures)
    Gt = out0["Gt"]
    kmax = max(np.linalg.cond(Gt[np.ix_(r, c)])
               for k in range(1, f + 1)
               for r in itertools.combinations(range(f), k)
               for c in itertools.combinations(range(p), k))
    tol = 10 * kmax * np.finfo(float).eps * len(er)
    assert np.abs(out1["Q"] - out0["Q"]).max() < tol
    assert np.abs(out1["R"] - out0["R"]).max() < tol * np.abs(out0["R"]).max()


def test_unrecoverable_pattern_rejected_and_untouched():
    g = O.geom(16, 16, 4, 4, 1)
    Gt, Gh = O.generator(1, 4, 4, 1)
    Q = O.encode(g, Gt, Gh, synth.gaussian(16, 16, 1))
    R = np.zeros((g.N, g.N), order="F")
    mask = np.zeros((g.grid_rows, g.grid_cols), np.uint8)
    O.inject(g, [(0, 1), (2, 1)], mask, Q, R)  # two erasures in one grid column, f = 1
    Qs = Q.copy()
    with pytest.raises(O.OracleError) as e:
        O.recover(g, Gt, Gh, mask, Q, R)
    assert e.value.rc == O.EUNRECOVERABLE
    assert np.array_equal(np.isnan(Q), np.isnan(Qs))
    assert mask.sum() == 2


def test_decode_sets_lowest_surviving_checksums():
    # Reading: with more surviving checksum rows than needed, the lowest-index ones are used.
    g = O.geom(24, 24, 6, 6, 3)
    Gt, Gh = O.generator(3, 6, 6, 1)
    Q = O.encode(g, Gt, Gh, synth.gaussian(24, 24, 1))
    R = np.zeros((g.N, g.N), order="F")
    mask = np.zeros((g.grid_rows, g.grid_cols), np.uint8)
    O.inject(g, [(1, 2), (6, 2), (4, 0)], mask, Q, R)
    sets, nrec = O.recover(g, Gt, Gh, mask, Q, R)
    # Hand-derived records (kind, index, f1, f2, A_fail, C_fail, C_use):
    #  Q grid column 0: systematic row 4 lost -> checksum row 0 used
    #  Q grid column 2: systematic row 1 and checksum row 0 lost -> checksum row 1 used
    #  R block rows 1, 4, 6 (all < p_c + f = 9): one systematic tile each, checksum col 0 used
    assert sets == [0, 0, 1, 0, 4, 0,
                    0, 2, 1, 1, 1, 0, 1,
                    1, 1, 1, 0, 2, 0,
                    1, 4, 1, 0, 0, 0,
                    1, 6, 1, 0, 2, 0]
    assert nrec == 3


def test_recovered_run_equals_fault_free_run():
    # c.f. Section 6: the framework recovers the failed nodes and proceeds; results match.
    A = synth.gaussian(64, 64, 9)
    y = synth.rhs(64, 1, 9)
    ref = O.run(A, 4, 4, 1, 8, seed=1, y=y)
    out = O.run(A, 4, 4, 1, 8, seed=1, y=y, erasures={3: [(1, 2)], 5: [(4, 0), (0, 4)]})
    assert out["n_recovered"] == 3
    for k in ("Q", "R", "Qo", "x"):
        assert np.abs(out[k] - ref[k]).max() < 1e-10 * max(1, np.abs(ref[k]).max())


def test_vertical_only_code():
    # R protection off (Section 4.2 with the vertical code alone, d = 0): At = [A; G_v A], R is
    # the sign-normalised Householder R of At, Q_2 = G_v Q_1 at the end, and a run whose Q
    # tiles (systematic and checksum) are erased and recovered equals the fault-free run.
    m, n, p, f, b = 48, 36, 4, 1, 6
    A = synth.gaussian(m, n, 3)
    ref = O.run(A, p, p, f, b, seed=2, protect_r=False)
    g, At, Q, R = ref["geom"], ref["At"], ref["Q"], ref["R"]
    assert g.d == 0 and g.N == n and g.grid_cols == p
    Gv = np.kron(ref["Gt"], np.eye(g.mb))
    assert np.array_equal(At[:m], A)
    assert np.abs(At[m:] - Gv @ A).max() < 1e-14 * np.abs(Gv @ A).max()
    Qh, Rh = _signfix(*np.linalg.qr(At))
    assert np.abs(R - Rh).max() < 1e-12 * np.abs(Rh).max()
    assert np.abs(Q - Qh).max() < 1e-11
    assert np.abs(Q[m:] - Gv @ Q[:m]).max() < 1e-12
    out = O.run(A, p, p, f, b, seed=2, protect_r=False, erasures={2: [(0, 1), (4, 2)], 4: [(3, 0)]})
    assert out["n_recovered"] == 3
    for k in ("Q", "R", "Qo"):
        assert np.abs(out[k] - ref[k]).max() < 1e-10 * max(1, np.abs(ref[k]).max())


# --------------------------------------------------------------------------- a8-a9
@pytest.mark.parametrize("m,p,f", [(32, 4, 1), (48, 6, 3), (45, 5, 2)])
def test_post_orth_block_equals_dense_and_is_orthogonal(m, p, f):
    # Theorem 'G_0' claim 1: (G_0 Q_1)^T (G_0 Q_1) = I; the sparse block pipeline of the
    # overhead proof equals the dense G_0 product.
    n = 24
    A = synth.gaussian(m, n, 1)
    n_eff = n
    pc = max(4, 2 * f)
    out = O.run(A, p, pc, f, 5, seed=4)
    g = out["geom"]
    Q1 = out["Q"][: g.m_pad, :n_eff]
    W = O.post_orth(g, out["Gt"], Q1)
    Wd = O.post_orth(g, out["Gt"], Q1, dense=True)
    assert np.abs(W - Wd).max() < 1e-14
    assert np.abs(W.T @ W - np.eye(n_eff)).max() < 1e-13
    assert np.abs(Q1.T @ Q1 - np.eye(n_eff)).max() > 1e-3  # Q_1 alone is not orthogonal


def test_projected_post_orth_equals_G0_Q1_on_consistent_checksums():
    # when Q_2 = G Q_1 exactly, G_0^{-1} (Q_1 + G^T Q_2) = G_0^{-1} (I + G^T G) Q_1 = G_0 Q_1
    m, p, f = 48, 6, 2
    g = O.geom(m, 12, p, p, f)
    Gt, _ = O.generator(f, p, p, 3)
    Q1 = synth.gaussian(m, 12, 4)
    Q2 = np.kron(Gt, np.eye(g.mb)) @ Q1
    W = O.post_orth_projected(g, Gt, Q1, Q2)
    assert np.abs(W - O.post_orth(g, Gt, Q1, dense=True)).max() < 1e-12 * np.abs(W).max()


@pytest.mark.parametrize("delta", [1e-5, 1e-3])
def test_projected_post_orth_loses_orthogonality_to_second_order(delta):
    # an orthonormal coded factor whose checksum rows drifted by delta from G Q_1: G_0 Q_1
    # loses orthogonality to first order in the drift, the projected form to second order
    m = n = 64
    p, f, b = 4, 1, 8
    ref = O.run(synth.gaussian(m, n, 6), p, p, f, b, seed=2)
    g, Gt = ref["geom"], ref["Gt"]
    Q = ref["Q"][:, :n].copy()
    Q[m:] += delta * synth.gaussian(g.c, n, 7) / np.sqrt(m)
    Q, _ = np.linalg.qr(Q)
    Q1, Q2 = Q[:m], Q[m:]
    drift = np.abs(Q2 - np.kron(Gt, np.eye(g.mb)) @ Q1).max()
    W0 = O.post_orth(g, Gt, Q1)
    W1 = O.post_orth_projected(g, Gt, Q1, Q2)
    e0 = np.abs(W0.T @ W0 - np.eye(n)).max()
    e1 = np.abs(W1.T @ W1 - np.eye(n)).max()
    assert e0 > 0.1 * drift
    assert e1 < n * drift ** 2 + 1e-13


@pytest.mark.parametrize("n,p,f,b", [(32, 4, 1, 8), (60, 6, 2, 10), (64, 4, 2, 16)])
def test_solve_square_matches_numpy(n, p, f, b):
    # Eqs. (linearsolve1)-(linearsolve3): R x = (G_0 Q_1)^T (G_0 y)
    A = synth.gaussian(n, n, 3)
    y = synth.rhs(n, 2, 3)
    out = O.run(A, p, p, f, b, seed=8, y=y)
    x = np.linalg.solve(A, y)
    assert np.abs(out["x"] - x).max() < 1e-10 * max(1, np.abs(x).max())


def test_solve_ls_tall_matches_lstsq():
    A = synth.gaussian(96, 24, 3)
    y = synth.rhs(96, 2, 3)
    out = O.run(A, 8, 4, 2, 8, seed=8, y=y)
    x, *_ = np.linalg.lstsq(A, y, rcond=None)
    assert np.abs(out["x"] - x).max() < 1e-11


def test_tall_ragged_rows_padding():
    # m not divisible by p_r: zero padding rows stay zero, A = Q_1 R still holds
    A = synth.gaussian(70, 16, 2)
    out = O.run(A, 8, 4, 2, 4, seed=1)
    g = out["geom"]
    assert g.m_pad == 72
    Q, R = out["Q"], out["R"]
    assert np.abs(Q[70:72, :16]).max() == 0.0
    assert np.abs(A - Q[:70, :16] @ R[:16, :16]).max() < 1e-13


# --------------------------------------------------------------------------- block reorth
def test_block_reorth_keeps_factorisation_and_restores_orthogonality():
    # Block MGS loses orthogonality like u kappa(A); projecting each panel once more on all
    # computed columns (block "twice is enough") brings it back to O(u), keeps At = Q R,
    # R equal to the Householder R of At, and the checksum relations (column operations).
    n, p, f, b = 96, 4, 1, 8
    kappa = 1e8
    A = synth.kappa_matrix(n, n, kappa, seed=4)
    one = O.run(A, p, p, f, b, seed=2)
    two = O.run(A, p, p, f, b, seed=2, reorth_block=True)
    g = two["geom"]
    o1 = np.abs(one["Q"][:, :n].T @ one["Q"][:, :n] - np.eye(n)).max()
    o2 = np.abs(two["Q"][:, :n].T @ two["Q"][:, :n] - np.eye(n)).max()
    assert o2 < 1e-13 and o1 > 1e3 * o2
    At = two["At"]
    assert np.abs(At[:, :n] - two["Q"][:, :n] @ two["R"][:n, :n]).max() < 1e-13 * np.abs(At).max()
    # rounding drift of Q_2 - G_v Q_1 is amplified by the pivots like u kappa, with or without
    # the reorthogonalisation (which is a column operation)
    Gv = np.kron(two["Gt"], np.eye(g.mb))
    u = np.finfo(float).eps / 2
    assert np.abs(two["Q"][g.m_pad:] - Gv @ two["Q"][: g.m_pad]).max() < 100 * u * kappa
    Qh, Rh = np.linalg.qr(At[:, :n])
    Rh = Rh * np.sign(np.diag(Rh))[:, None]
    assert np.abs(two["R"][:n, :n] - Rh).max() < 100 * u * kappa * np.abs(Rh).max()


def test_G0_is_symmetric():
    # G_0 = [[I + G~_1, V~], [V~^T, -I]] (x) I_mb with G~_1 = -V~ V~^T / 2 symmetric, so
    # G_0^T = G_0: the reverse pass applies G_0^T with the post-orthogonalisation pipeline
    for (p_r, f, gdist) in [(4, 1, 0), (8, 2, 0), (6, 3, 1)]:
        g = O.geom(5 * p_r, 8, p_r, 8, f, True)
        Gt, _ = O.generator(f, p_r, 8, 17, gdist)
        G0 = O.build_G0(g, Gt)
        assert np.array_equal(G0, G0.T)


# ----------------------------------------------------------------- E1 MDS statistics
def test_mds_stats_closed_forms():
    G = np.array([[1.0, 2.0, 3.0], [4.0, -5.0, 6.0]])
    mind, maxc = O.mds_stats(G)
    # 1 x 1 submatrices: |det| = |entry|, condition number 1
    assert mind[1] == 1.0 and maxc[1] == 1.0
    # 2 x 2 minors, by hand: |1*-5 - 2*4| = 13, |1*6 - 3*4| = 6, |2*6 - 3*-5| = 27
    assert mind[2] == pytest.approx(6.0, rel=1e-14)

    def cond2x2(S):  # sigma^2 = (T +- sqrt(T^2 - 4 D^2)) / 2, T = |S|_F^2, D = det S
        T = (S ** 2).sum()
        D = S[0, 0] * S[1, 1] - S[0, 1] * S[1, 0]
        disc = np.sqrt(T * T - 4 * D * D)
        return np.sqrt((T + disc) / (T - disc))

    worst = max(cond2x2(G[:, [a, b]]) for a, b in [(0, 1), (0, 2), (1, 2)])
    assert maxc[2] == pytest.approx(worst, rel=1e-12)
    assert mind[0] == 1.0 and maxc[0] == pytest.approx(worst, rel=1e-12)


def test_mds_stats_detects_a_singular_minor():
    G = np.array([[1.0, 2.0, 2.0, 5.0], [3.0, 1.0, 1.0, 7.0]])   # columns 1 and 2 equal
    mind, maxc = O.mds_stats(G)
    assert mind[2] == 0.0 and maxc[2] == np.inf


def test_structured_generator_has_no_singular_minor():
    for (f, p_r, seed) in [(2, 8, 1), (3, 10, 2), (4, 12, 3)]:
        Gt, _ = O.generator(f, p_r, 4, seed)
        mind, maxc = O.mds_stats(Gt)
        assert mind[0] > 0.0 and np.isfinite(maxc[0])


# ----------------------------------------------------------------- panel variants (NEXT f3)
def _orth(Q):
    return np.abs(Q.T @ Q - np.eye(Q.shape[1])).max()


def test_panel_variants_follow_their_known_orthogonality_scaling():
    # one panel over a whole 600 x 80 matrix with kappa 1e5: CGS2 and ICGS orthogonal to O(u),
    # MGS loses like u kappa, CGS1 (Pythagorean norm) like u kappa^2 (Bjorck 1994; Giraud,
    # Langou & Rozloznik 2005; Smoktunowicz, Barlow & Langou 2006)
    m, n, kappa = 600, 80, 1e5
    u = np.finfo(np.float64).eps / 2
    A = synth.kappa_matrix(m, n, kappa, 7)
    orth = {}
    for panel in ("icgs", "mgs", "cgs1", "cgs2"):
        Q = np.asfortranarray(A.copy())
        R = np.zeros((n, n), order="F")
        O.factor(Q, R, n, n, panel=panel)
        assert np.linalg.norm(A - Q @ R) / np.linalg.norm(A) < 50 * n * u, panel
        assert np.allclose(np.tril(R, -1), 0.0), panel
        orth[panel] = _orth(Q)
    assert orth["cgs2"] < 100 * n * u and orth["icgs"] < 100 * n * u
    assert 10 * u * kappa * 1e-3 < orth["mgs"] < 10 * n * u * kappa
    assert orth["mgs"] < orth["cgs1"] < 10 * n * u * kappa ** 2


def test_panel_variants_agree_with_householder_r():
    m, n = 300, 40
    A = synth.kappa_matrix(m, n, 1e2, 3)
    Rh = np.linalg.qr(A, mode="r")
    Rh = np.diag(np.sign(np.diag(Rh))) @ Rh
    for panel in ("mgs", "cgs1", "cgs2"):
        Q = np.asfortranarray(A.copy())
        R = np.zeros((n, n), order="F")
        O.factor(Q, R, n, 16, panel=panel)
        assert np.abs(R - Rh).max() / np.abs(Rh).max() < 1e-12, panel


# ----------------------------------------------------------------- in-node storage (NEXT f2)
def _min_k_brute(P, f):
    """Smallest K for which the load-balanced distribution leaves at least f surviving checksum
    blocks (the f lost data blocks, L = P) for every set of f failed nodes."""
    for K in range(1, 4 * P):
        hosts = O.in_node_hosts(K, P)
        load = [hosts.count(q) for q in range(P)]
        worst = max(sum(load[q] for q in S) for S in itertools.combinations(range(P), f))
        if K - worst >= f:
            return K
    return None


def test_in_node_k_bound_is_tight_by_brute_force():
    for P in range(3, 11):
        for f in range(1, P // 2 + 1):
            assert _min_k_brute(P, f) == O.in_node_checks(P, P, f), (P, f)


def test_in_node_distribution_is_load_balanced():
    for (K, P) in [(4, 8), (3, 8), (8, 16), (10, 4), (7, 3)]:
        hosts = O.in_node_hosts(K, P)
        load = sorted(hosts.count(q) for q in range(P))
        a_bar = K - P * (K // P)
        assert load == [K // P] * (P - a_bar) + [-(-K // P)] * a_bar


@pytest.mark.parametrize("p,f", [(4, 1), (8, 2)])
def test_in_node_every_node_failure_pattern_recovers(p, f):
    # every set of at most f failed nodes with at most f per node row and column, at the
    # start of a middle panel, recovers the fault-free factorisation
    m = n = 8 * p
    A = synth.gaussian(m, n, 31)
    clean = O.run_in_node(A, p, f, b=8, seed=5)
    K = clean["K"]
    assert 2 * K <= p
    nodes = [(i, j) for i in range(p) for j in range(p)]
    pats = [c for r in range(1, f + 1) for c in itertools.combinations(nodes, r)
            if max(sum(1 for (i, _) in c if i == q) for q in range(p)) <= f
            and max(sum(1 for (_, j) in c if j == q) for q in range(p)) <= f]
    if len(pats) > 400:
        pats = [pats[k] for k in np.random.default_rng(3).choice(len(pats), 400, replace=False)]
    for pat in pats:
        hit = O.run_in_node(A, p, f, b=8, seed=5, node_failures={3: list(pat)})
        assert np.abs(hit["Q"] - clean["Q"]).max() < 1e-9, pat
        assert np.abs(hit["R"] - clean["R"]).max() < 1e-9, pat
