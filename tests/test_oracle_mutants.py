"""The oracle's pins discriminate: each plausible mistake planted in a copy of the oracle's
source (a dropped term, a wrong sign, a transposed index, the wrong decode rows, a changed
RNG constant) makes at least one pin of tests/test_oracle_pins.py fail.  CPU only; the
copies are compiled into a temporary directory with the oracle's own flags, and every
planted mistake keeps all memory accesses in bounds.

Not listed, because they are equivalent up to rounding: dropping the coefficients that the
ICGS reorthogonalisation or the block reorthogonalisation add to R.  Those coefficients
correct the rounding of the first projection and are of size u ||a||: leaving them out
moves R by about 1e-15 relative (measured on the pins' cases), inside every tolerance."""
import os

import pytest

import test_oracle_pins as P
from oracle import build as OB
from oracle import oracle as O

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "cqr_oracle.c")

# (what the mistake is, source text, replacement)
MUTANTS = [
    ("generator: G~_1 = +1/2 V V^T",
     "Gt[i * p_r + l] = -0.5 * acc;", "Gt[i * p_r + l] = 0.5 * acc;"),
    ("generator: G~_1 from the products of row i with itself only",
     "acc += Gt[i * p_r + f + t] * Gt[l * p_r + f + t];",
     "acc += Gt[i * p_r + f + t] * Gt[i * p_r + f + t];"),
    ("SplitMix64: second shift 31 instead of 30",
     "z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;", "z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ULL;"),
    ("Unif(0,1): 52 bits scaled by 2^-53",
     "uint64_t x = sm64_next(s) >> 11;", "uint64_t x = sm64_next(s) >> 12;"),
    ("encode: generator read as p_r x f",
     "acc += Gt[i * g->p_r + t] * At[t * mb + r + col * ldat];",
     "acc += Gt[t * g->f + i] * At[t * mb + r + col * ldat];"),
    ("encode: horizontal checksums of the systematic rows only (no corner)",
     "for (int64_t row = 0; row < g->M; ++row) {", "for (int64_t row = 0; row < g->m_pad; ++row) {"),
    ("ICGS: criterion inverted",
     "v[0] < tau * tau * eta[j]", "v[0] > tau * tau * eta[j]"),
    ("ICGS: rank-1 update with the wrong sign",
     "for (int64_t r = 0; r < M; ++r) qa[r] -= qc[r] * rca;",
     "for (int64_t r = 0; r < M; ++r) qa[r] += qc[r] * rca;"),
    ("trailing update with the wrong sign",
     "for (int64_t a = 0; a < bk; ++a) acc -= Q[r + (kb + a) * ldq] * R[(kb + a) + j * ldr];",
     "for (int64_t a = 0; a < bk; ++a) acc += Q[r + (kb + a) * ldq] * R[(kb + a) + j * ldr];"),
    ("decode: highest-index surviving checksum rows",
     "for (int i = 0; i < nchk && cu < a; ++i) if (!lost_chk[i]) C_use[cu++] = i;",
     "for (int i = nchk - 1; i >= 0 && cu < a; --i) if (!lost_chk[i]) C_use[cu++] = i;"),
    ("decode of Q: surviving systematic tiles not subtracted",
     "if (!ls[l]) acc -= Gt[i * p_r + l] * Q[l * mb + r + col * ldq];", "(void)ls;"),
    ("decode of R: surviving tiles not subtracted",
     "if (!ls[j]) acc -= Gh[j * f + l] * R[r + (j * nb + s) * ldr];", "(void)ls;"),
    ("decode: G^ transposed",
     "Ghat[a * f1 + bb] = Gt[C_use[a] * p_r + A_fail[bb]];",
     "Ghat[bb * f1 + a] = Gt[C_use[a] * p_r + A_fail[bb]];"),
    ("post-orthogonalisation (block form): -I block as +I",
     "acc -= Z[i * mb + s + col * ldz];", "acc += Z[i * mb + s + col * ldz];"),
    ("G_0 (dense form): -I block as +I",
     "for (int64_t r = c; r < mp; ++r) G0[r + r * ldg] = -1.0;",
     "for (int64_t r = c; r < mp; ++r) G0[r + r * ldg] = 1.0;"),
    ("back substitution with R transposed",
     "for (int64_t j = i + 1; j < n; ++j) acc -= R[i + j * ldr] * x[j + col * ldx];",
     "for (int64_t j = i + 1; j < n; ++j) acc -= R[j + i * ldr] * x[j + col * ldx];"),
    ("least squares: Cholesky column not divided by its pivot",
     "Gm[i + j * n] = a2 / ljj;", "Gm[i + j * n] = a2;"),
]

# the pins, with one parameter set each
BATTERY = [
    (P.test_splitmix64_published_outputs, ()),
    (P.test_generator_draws_unif01, ()),
    (P.test_G0_observation_identity, (2, 8, 0)),
    (P.test_G0_observation_identity, (3, 6, 1)),
    (P.test_det_G0, (2, 8, 3)),
    (P.test_invert_small_matches_numpy, ()),
    (P.test_encode_equals_kronecker_definition, (30, 24, 6, 4, 2, True)),
    (P.test_worked_example_encode_and_G0, ()),
    (P.test_worked_example_recovery_formulas, ()),
    (P.test_factor_matches_householder_of_encoded, (96, 64, 4, 2, 16)),
    (P.test_corollary_final_form_and_checksums_every_iteration, (2,)),
    (P.test_reorth_criterion_restores_orthogonality, ()),
    (P.test_recover_bruteforce_every_pattern, (4, 2, 2)),
    (P.test_decode_sets_lowest_surviving_checksums, ()),
    (P.test_recovered_run_equals_fault_free_run, ()),
    (P.test_vertical_only_code, ()),
    (P.test_post_orth_block_equals_dense_and_is_orthogonal, (48, 6, 3)),
    (P.test_solve_square_matches_numpy, (60, 6, 2, 10)),
    (P.test_solve_ls_tall_matches_lstsq, ()),
    (P.test_block_reorth_keeps_factorisation_and_restores_orthogonality, ()),
    (P.test_G0_is_symmetric, ()),
]


def _failing_pins():
    failed = []
    for fn, args in BATTERY:
        try:
            fn(*args)
        except Exception:  # an assertion, or an oracle status the pin did not expect
            failed.append(fn.__name__)
    return failed


def test_every_pin_of_the_battery_passes_on_the_oracle():
    assert _failing_pins() == []


@pytest.mark.parametrize("what,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_a_planted_mistake(what, old, new, tmp_path):
    with open(SRC) as fh:
        src = fh.read()
    assert src.count(old) == 1, what
    path = OB.build_from_source(src.replace(old, new), str(tmp_path))
    with O.library(path):
        failed = _failing_pins()
    assert failed, "no pin catches: " + what
