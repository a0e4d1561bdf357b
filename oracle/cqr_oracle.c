/*
 * cqr_oracle.c -- plain FP64 CPU oracle for coded block Gram-Schmidt QR
 * (Coded Computing for Fault-Tolerant Parallel QR Decomposition, arXiv 2311.11943).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct restatement of
 * the method that the CUDA library is checked against.  Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the product path never
 * does.  It shares no code, header, table or helper with the CUDA library.
 *
 * Every routine follows one passage of the paper, cited by section / equation /
 * algorithm.  No blocking, fusion or reordering beyond what the cited definition
 * states.  Storage is column-major throughout; all pointers are host pointers.
 * Built with -ffp-contract=off so that x86-64 and aarch64 hosts give identical bits.
 *
 * Geometry (Section 2 "Distributed computing model", Eq. (encoding), Eq. (tildeG_eq)):
 *   A is m x n.  Virtual node grid p_r x p_c.  Tile height mb = ceil(m/p_r); A is
 *   zero-padded to m_pad = p_r*mb rows (padded rows stay zero under Gram-Schmidt).
 *   Tile width nb = n/p_c (p_c must divide n).  c = f*mb checksum rows, d = f*nb
 *   checksum columns (d = 0 when R-protection is off).  The encoded matrix
 *   At = [[A, A G_h], [G_v A, G_v A G_h]] is M x N with M = m_pad + c, N = n + d.
 *   Node (i,j), i < p_r+f, j < p_c+f (checksum columns only when R-protected), owns
 *   Q tile (i,j) = rows [i*mb,(i+1)*mb) x cols [j*nb,(j+1)*nb) and, for i < p_c+f,
 *   R tile (i,j) = rows [i*nb,(i+1)*nb) x cols [j*nb,(j+1)*nb).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CQRO_OK 0
#define CQRO_EINVAL 1
#define CQRO_EUNRECOVERABLE 5
#define CQRO_EBREAKDOWN 6

typedef struct {
  int64_t m, n;
  int32_t p_r, p_c, f, protect_r;
  int64_t mb, nb, m_pad, c, d, M, N;
  int32_t grid_rows, grid_cols;
} cqro_geom;

int cqro_version(void) { return 1; }

/* Geometry from (m, n, p_r, p_c, f, protect_r); Section 2 and Eq. (tildeG_eq). */
int cqro_geom_init(cqro_geom* g, int64_t m, int64_t n, int p_r, int p_c, int f,
                   int protect_r) {
  if (m <= 0 || n <= 0 || p_r <= 0 || p_c <= 0 || f < 0) return CQRO_EINVAL;
  if (n % p_c != 0) return CQRO_EINVAL;
  if (2 * f > p_r || (protect_r && 2 * f > p_c)) return CQRO_EINVAL; /* f <= min(p_r,p_c)/2 */
  g->m = m; g->n = n; g->p_r = p_r; g->p_c = p_c; g->f = f; g->protect_r = protect_r ? 1 : 0;
  g->mb = (m + p_r - 1) / p_r;
  g->nb = n / p_c;
  g->m_pad = g->mb * p_r;
  g->c = (int64_t)f * g->mb;
  g->d = g->protect_r ? (int64_t)f * g->nb : 0;
  g->M = g->m_pad + g->c;
  g->N = n + g->d;
  g->grid_rows = p_r + f;
  g->grid_cols = p_c + (g->protect_r ? f : 0);
  return CQRO_OK;
}

/* ---------------------------------------------------------------------------------
 * a1. Generator (Construction "Q-factor checksum-generator matrix", Section 4.2):
 * V~ is f x (p_r - f) with i.i.d. Unif(0,1) entries, G~_1 = -1/2 V~ V~^T, and
 * G~ = [G~_1  V~] (f x p_r, first f columns = G~_1).  The horizontal generator G~_h
 * (p_c x f) may be any MDS matrix; here i.i.d. draws from the same distribution
 * (every square submatrix nonsingular with probability 1).
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), state advanced by the
 * golden gamma 0x9E3779B97F4A7C15 and finalised by the published mix13 variant.
 * Unif(0,1): top 53 bits times 2^-53, zero rejected.  Normal: Box-Muller, cosine branch.
 * Draw order: V~ row-major, then G~_h row-major, one stream seeded with `seed`.
 * --------------------------------------------------------------------------------- */
static uint64_t sm64_next(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static double sm64_unif01(uint64_t* s) {
  for (;;) {
    uint64_t x = sm64_next(s) >> 11;
    if (x != 0) return (double)x * 0x1.0p-53;
  }
}

static double draw(uint64_t* s, int gdist) {
  if (gdist == 0) return sm64_unif01(s);
  double u1 = sm64_unif01(s), u2 = sm64_unif01(s);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
}

void cqro_splitmix64(uint64_t seed, int count, uint64_t* out) {
  uint64_t s = seed;
  for (int i = 0; i < count; ++i) out[i] = sm64_next(&s);
}

/* Gt: f x p_r row-major (Gt[i*p_r + t] = g~_{i,t}); Gh: p_c x f row-major
 * (Gh[j*f + l] = g~h_{j,l}).  gh_ones = 1 selects G~_h = all ones (the f = 1 worked
 * example of Appendix "Example for code construction"). */
int cqro_generator(int f, int p_r, int p_c, uint64_t seed, int gdist, int gh_ones,
                   double* Gt, double* Gh) {
  if (f < 0 || f > p_r) return CQRO_EINVAL;
  uint64_t s = seed;
  int nv = p_r - f;
  for (int i = 0; i < f; ++i)
    for (int t = 0; t < nv; ++t) Gt[i * p_r + f + t] = draw(&s, gdist);
  for (int i = 0; i < f; ++i)
    for (int l = 0; l < f; ++l) {
      double acc = 0.0;
      for (int t = 0; t < nv; ++t) acc += Gt[i * p_r + f + t] * Gt[l * p_r + f + t];
      Gt[i * p_r + l] = -0.5 * acc;
    }
  if (Gh != NULL)
    for (int j = 0; j < p_c; ++j)
      for (int l = 0; l < f; ++l) Gh[j * f + l] = gh_ones ? 1.0 : draw(&s, gdist);
  return CQRO_OK;
}

/* ---------------------------------------------------------------------------------
 * a2. Encode (Eq. (encoding) and the checksum tile formula C_{i,j} = sum_t g~_{i,t}
 * A_{t,j} of Section 4.2).  Vertical checksums for every column of A; horizontal
 * checksums (A G_h, and the corner (G_v A) G_h) for every row of At when protected.
 * --------------------------------------------------------------------------------- */
int cqro_encode(const cqro_geom* g, const double* Gt, const double* Gh, const double* A,
                int64_t lda, double* At, int64_t ldat) {
  const int64_t mb = g->mb, nb = g->nb;
#pragma omp parallel for schedule(static)
  for (int64_t col = 0; col < g->n; ++col) {
    for (int64_t r = 0; r < g->m_pad; ++r)
      At[r + col * ldat] = (r < g->m) ? A[r + col * lda] : 0.0;
    for (int i = 0; i < g->f; ++i)
      for (int64_t r = 0; r < mb; ++r) {
        double acc = 0.0;
        for (int t = 0; t < g->p_r; ++t) acc += Gt[i * g->p_r + t] * At[t * mb + r + col * ldat];
        At[g->m_pad + i * mb + r + col * ldat] = acc;
      }
  }
  if (g->protect_r) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < g->d; ++k) {
      int64_t l = k / nb, s = k % nb;
      for (int64_t row = 0; row < g->M; ++row) {
        double acc = 0.0;
        for (int j = 0; j < g->p_c; ++j) acc += Gh[j * g->f + l] * At[row + (j * nb + s) * ldat];
        At[row + (g->n + k) * ldat] = acc;
      }
    }
  }
  return CQRO_OK;
}

/* ---------------------------------------------------------------------------------
 * a3. ICGS panel (Appendix A, Algorithm CGS, with the reorthogonalisation of ICGS).
 * The listing computes, per column i, the single reduction v = Q[:, i:b]^T Q[:, i],
 * normalises q = Q[:, i] / sqrt(v_1), writes row i of R, and removes q from the
 * remaining panel columns.  Reading of the listing: the R row and the rank-1 update
 * use v / sqrt(v_1) (the listing omits this scaling).  ICGS reorthogonalises column i
 * once more when its norm has dropped below tau times its norm at the panel start
 * (Kahan-Parlett criterion, tau = 1/sqrt(2)); the extra pass projects column i on the
 * already computed panel columns, adds the coefficients to R, and recomputes v.
 * tau <= 0 disables reorthogonalisation.  Inner products run over all M rows.
 * --------------------------------------------------------------------------------- */
static int icgs_panel(int64_t M, int64_t kb, int64_t bk, double tau, double* Q, int64_t ldq,
                      double* R, int64_t ldr, int64_t* n_reorth) {
  double* eta = (double*)malloc(sizeof(double) * (size_t)bk);
  double* v = (double*)malloc(sizeof(double) * (size_t)bk);
  double* s = (double*)malloc(sizeof(double) * (size_t)bk);
  int rc = CQRO_OK;
  for (int64_t j = 0; j < bk; ++j) {
    const double* qj = Q + (kb + j) * ldq;
    double acc = 0.0;
    for (int64_t r = 0; r < M; ++r) acc += qj[r] * qj[r];
    eta[j] = acc;
  }
  for (int64_t j = 0; j < bk && rc == CQRO_OK; ++j) {
    const int64_t c = kb + j;
    double* qc = Q + c * ldq;
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < bk - j; ++a) {
      const double* qa = Q + (c + a) * ldq;
      double acc = 0.0;
      for (int64_t r = 0; r < M; ++r) acc += qa[r] * qc[r];
      v[a] = acc;
    }
    if (j > 0 && tau > 0.0 && v[0] < tau * tau * eta[j]) {
      /* reorthogonalisation pass against the panel's computed columns kb..c-1 */
#pragma omp parallel for schedule(static)
      for (int64_t a = 0; a < j; ++a) {
        const double* qa = Q + (kb + a) * ldq;
        double acc = 0.0;
        for (int64_t r = 0; r < M; ++r) acc += qa[r] * qc[r];
        s[a] = acc;
      }
#pragma omp parallel for schedule(static)
      for (int64_t r = 0; r < M; ++r) {
        double acc = qc[r];
        for (int64_t a = 0; a < j; ++a) acc -= Q[r + (kb + a) * ldq] * s[a];
        qc[r] = acc;
      }
      for (int64_t a = 0; a < j; ++a) R[(kb + a) + c * ldr] += s[a];
      if (n_reorth) ++*n_reorth;
#pragma omp parallel for schedule(static)
      for (int64_t a = 0; a < bk - j; ++a) {
        const double* qa = Q + (c + a) * ldq;
        double acc = 0.0;
        for (int64_t r = 0; r < M; ++r) acc += qa[r] * qc[r];
        v[a] = acc;
      }
    }
    if (!(v[0] > 0.0) || !isfinite(v[0])) { rc = CQRO_EBREAKDOWN; break; }
    const double rcc = sqrt(v[0]);
    R[c + c * ldr] = rcc;
    for (int64_t r = 0; r < M; ++r) qc[r] = qc[r] / rcc;
    for (int64_t a = 1; a < bk - j; ++a) R[c + (c + a) * ldr] = v[a] / rcc;
#pragma omp parallel for schedule(static)
    for (int64_t a = 1; a < bk - j; ++a) {
      double* qa = Q + (c + a) * ldq;
      const double rca = R[c + (c + a) * ldr];
      for (int64_t r = 0; r < M; ++r) qa[r] -= qc[r] * rca;
    }
  }
  free(eta); free(v); free(s);
  return rc;
}

/* Stand-alone panel routine (same arithmetic as inside cqro_factor). */
/* Panel variants for the comparison of NEXT f3 (left-looking classical Gram-Schmidt,
 * Bjorck, "Numerics of Gram-Schmidt orthogonalization", 1994):
 *   passes = 1 ("CGS1", one reduction per column): s = Q_{:,0:j}^T p_j and |p_j|^2 from the
 *     original p_j; p_j -= Q_{:,0:j} s; r_jj^2 = |p_j|^2 - |s|^2 (Pythagorean identity, Smoktunowicz,
 *     Barlow & Langou 2006); loses orthogonality like u kappa^2.
 *   passes = 2 ("CGS2", twice is enough): the projection repeated once on the result, R gets
 *     s + s', r_jj^2 = |p'|^2 - |s'|^2; orthogonal to O(u).
 * Columns kb .. kb+bk-1 of Q (M rows); R rows / columns kb.. receive the panel's block. */
static int cgs_panel(int64_t M, int64_t kb, int64_t bk, int passes, double* Q, int64_t ldq,
                     double* R, int64_t ldr) {
  double* s = (double*)malloc(sizeof(double) * (size_t)(bk + 1));
  int rc = CQRO_OK;
  for (int64_t j = 0; j < bk && rc == CQRO_OK; ++j) {
    const int64_t c = kb + j;
    double* qc = Q + c * ldq;
    double r2 = 0.0;
    for (int pass = 0; pass < passes; ++pass) {
#pragma omp parallel for schedule(static)
      for (int64_t a = 0; a <= j; ++a) {  /* s_a = q_a^T p (a < j), s_j = p^T p */
        const double* qa = Q + (kb + a) * ldq;
        double acc = 0.0;
        for (int64_t r = 0; r < M; ++r) acc += qa[r] * qc[r];
        s[a] = acc;
      }
#pragma omp parallel for schedule(static)
      for (int64_t r = 0; r < M; ++r) {
        double acc = qc[r];
        for (int64_t a = 0; a < j; ++a) acc -= Q[r + (kb + a) * ldq] * s[a];
        qc[r] = acc;
      }
      double ss = 0.0;
      for (int64_t a = 0; a < j; ++a) {
        R[(kb + a) + c * ldr] += s[a];
        ss += s[a] * s[a];
      }
      r2 = s[j] - ss;
    }
    if (!(r2 > 0.0) || !isfinite(r2)) { rc = CQRO_EBREAKDOWN; break; }
    const double rcc = sqrt(r2);
    R[c + c * ldr] = rcc;
    for (int64_t r = 0; r < M; ++r) qc[r] = qc[r] / rcc;
  }
  free(s);
  return rc;
}

int cqro_cgs_panel(int64_t M, int64_t kb, int64_t bk, int passes, double* Q, int64_t ldq,
                   double* R, int64_t ldr) {
  if (passes != 1 && passes != 2) return CQRO_EINVAL;
  return cgs_panel(M, kb, bk, passes, Q, ldq, R, ldr);
}

int cqro_icgs_panel(int64_t M, int64_t kb, int64_t bk, double tau, double* Q, int64_t ldq,
                    double* R, int64_t ldr, int64_t* n_reorth) {
  return icgs_panel(M, kb, bk, tau, Q, ldq, R, ldr, n_reorth);
}

/* ---------------------------------------------------------------------------------
 * a3-a5. PBMGS (Appendix A, Algorithm PBMGS; sequential form BMGS, Appendix B): for
 * each panel of b columns among the first n: ICGS on the panel, then
 * Rbar = Qbar^T Q[:, i+b : N] and Q[:, i+b : N] -= Qbar Rbar, Rbar stored in
 * R[i : i+b, i+b : N] (reading of the listing: the off-diagonal block, as in BMGS).
 * The d checksum columns are trailing columns of every update and are never
 * normalised.  Panels t0 .. t1-1 are run (resumable); the last panel may be narrower.
 * --------------------------------------------------------------------------------- */
/* Block reorthogonalisation of panel columns kb .. kb+bk-1 against the computed columns
 * 0 .. kb-1 (the block form of "twice is enough"; an addition to the paper's PBMGS, used
 * when reorth_block != 0):  S = Q[:, :kb]^T Qbar,  Qbar -= Q[:, :kb] S,  R[:kb, panel] += S.
 * A column operation on the encoded matrix, so Q_2 = G_v Q_1 is preserved. */
static void block_reorth(int64_t M, int64_t kb, int64_t bk, double* Q, int64_t ldq, double* R,
                         int64_t ldr) {
  double* S = (double*)malloc(sizeof(double) * (size_t)(kb * bk));
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < bk; ++i)
    for (int64_t a = 0; a < kb; ++a) {
      const double* qa = Q + a * ldq;
      const double* qi = Q + (kb + i) * ldq;
      double acc = 0.0;
      for (int64_t r = 0; r < M; ++r) acc += qa[r] * qi[r];
      S[a + i * kb] = acc;
    }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < bk; ++i) {
    double* qi = Q + (kb + i) * ldq;
    for (int64_t r = 0; r < M; ++r) {
      double acc = qi[r];
      for (int64_t a = 0; a < kb; ++a) acc -= Q[r + a * ldq] * S[a + i * kb];
      qi[r] = acc;
    }
    for (int64_t a = 0; a < kb; ++a) R[a + (kb + i) * ldr] += S[a + i * kb];
  }
  free(S);
}

/* panel: 0 ICGS (the paper's listing with the reorthogonalisation test), 1 MGS (the same
 * right-looking column loop without it), 2 CGS1, 3 CGS2 (see cgs_panel). */
int cqro_factor3(int64_t M, int64_t N, int64_t n, int64_t b, int t0, int t1, double tau,
                 int reorth_block, int panel, double* Q, int64_t ldq, double* R, int64_t ldr,
                 int64_t* n_reorth) {
  if (b <= 0 || M <= 0 || n <= 0 || N < n) return CQRO_EINVAL;
  const int T = (int)((n + b - 1) / b);
  if (t1 < 0 || t1 > T) t1 = T;
  for (int t = t0; t < t1; ++t) {
    const int64_t kb = (int64_t)t * b;
    const int64_t bk = (kb + b <= n) ? b : n - kb;
    if (reorth_block && kb > 0) block_reorth(M, kb, bk, Q, ldq, R, ldr);
    int rc;
    if (panel == 2 || panel == 3)
      rc = cgs_panel(M, kb, bk, panel - 1, Q, ldq, R, ldr);
    else
      rc = icgs_panel(M, kb, bk, panel == 1 ? -1.0 : tau, Q, ldq, R, ldr, n_reorth);
    if (rc != CQRO_OK) return rc;
    const int64_t j0 = kb + bk;
    if (j0 >= N) continue;
#pragma omp parallel for schedule(static)
    for (int64_t j = j0; j < N; ++j) {
      double* qj = Q + j * ldq;
      for (int64_t a = 0; a < bk; ++a) {
        const double* qa = Q + (kb + a) * ldq;
        double acc = 0.0;
        for (int64_t r = 0; r < M; ++r) acc += qa[r] * qj[r];
        R[(kb + a) + j * ldr] = acc;
      }
      for (int64_t r = 0; r < M; ++r) {
        double acc = qj[r];
        for (int64_t a = 0; a < bk; ++a) acc -= Q[r + (kb + a) * ldq] * R[(kb + a) + j * ldr];
        qj[r] = acc;
      }
    }
  }
  return CQRO_OK;
}

int cqro_factor2(int64_t M, int64_t N, int64_t n, int64_t b, int t0, int t1, double tau,
                 int reorth_block, double* Q, int64_t ldq, double* R, int64_t ldr,
                 int64_t* n_reorth) {
  return cqro_factor3(M, N, n, b, t0, t1, tau, reorth_block, 0, Q, ldq, R, ldr, n_reorth);
}

int cqro_factor(int64_t M, int64_t N, int64_t n, int64_t b, int t0, int t1, double tau,
                double* Q, int64_t ldq, double* R, int64_t ldr, int64_t* n_reorth) {
  return cqro_factor2(M, N, n, b, t0, t1, tau, 0, Q, ldq, R, ldr, n_reorth);
}

/* ---------------------------------------------------------------------------------
 * a6. Erasure (Section 2 "Failure model": fail-stop, the node loses all its data).
 * tiles: `count` (i, j) pairs.  The node's Q tile is poisoned with NaN and, when R is
 * protected and i < p_c+f, its R tile too.  mask is (grid_rows x grid_cols) row-major.
 * --------------------------------------------------------------------------------- */
int cqro_inject(const cqro_geom* g, const int* tiles, int count, uint8_t* mask, double* Q,
                int64_t ldq, double* R, int64_t ldr) {
  for (int e = 0; e < count; ++e) {
    int i = tiles[2 * e], j = tiles[2 * e + 1];
    if (i < 0 || i >= g->grid_rows || j < 0 || j >= g->grid_cols) return CQRO_EINVAL;
  }
  for (int e = 0; e < count; ++e) {
    int i = tiles[2 * e], j = tiles[2 * e + 1];
    mask[i * g->grid_cols + j] = 1;
    for (int64_t col = j * g->nb; col < (j + 1) * g->nb; ++col)
      for (int64_t r = i * g->mb; r < (i + 1) * g->mb; ++r) Q[r + col * ldq] = NAN;
    if (g->protect_r && i < g->p_c + g->f)
      for (int64_t col = j * g->nb; col < (j + 1) * g->nb; ++col)
        for (int64_t r = i * g->nb; r < (i + 1) * g->nb; ++r) R[r + col * ldr] = NAN;
  }
  return CQRO_OK;
}

/* Gauss-Jordan inverse with partial pivoting (Golub & Van Loan, Sec. 3.4); k <= 64. */
static int invert_small(int k, const double* Gin, double* Ginv) {
  double a[64 * 128];
  if (k > 64) return CQRO_EINVAL;
  for (int r = 0; r < k; ++r)
    for (int c = 0; c < 2 * k; ++c)
      a[r * 2 * k + c] = (c < k) ? Gin[r * k + c] : (c - k == r ? 1.0 : 0.0);
  for (int col = 0; col < k; ++col) {
    int piv = col;
    for (int r = col + 1; r < k; ++r)
      if (fabs(a[r * 2 * k + col]) > fabs(a[piv * 2 * k + col])) piv = r;
    if (!(fabs(a[piv * 2 * k + col]) > 0.0)) return CQRO_EUNRECOVERABLE;
    if (piv != col)
      for (int c = 0; c < 2 * k; ++c) {
        double t = a[col * 2 * k + c]; a[col * 2 * k + c] = a[piv * 2 * k + c]; a[piv * 2 * k + c] = t;
      }
    double p = a[col * 2 * k + col];
    for (int c = 0; c < 2 * k; ++c) a[col * 2 * k + c] = a[col * 2 * k + c] / p;
    for (int r = 0; r < k; ++r) {
      if (r == col) continue;
      double fct = a[r * 2 * k + col];
      if (fct != 0.0)
        for (int c = 0; c < 2 * k; ++c) a[r * 2 * k + c] -= fct * a[col * 2 * k + c];
    }
  }
  for (int r = 0; r < k; ++r)
    for (int c = 0; c < k; ++c) Ginv[r * k + c] = a[r * 2 * k + k + c];
  return CQRO_OK;
}

int cqro_invert_small(int k, const double* G, double* Ginv) { return invert_small(k, G, Ginv); }

/* ---------------------------------------------------------------------------------
 * a7. Recovery (Appendix "Proof of Theorem overhead", Lemma on the recovery overhead):
 * per grid column j, A_fail / C_fail are the erased systematic / checksum row tiles.
 * With G^ = [g~_{i,t}], i in the f1 lowest-index surviving checksum rows, t in A_fail,
 *   A_{t,j} = sum_i g^-1_{t,i} (C_{i,j} - sum_{l in A_succ} g~_{i,l} A_{l,j})
 * (reading of the garbled index: the inner coefficient is g~_{i,l}); erased checksum
 * tiles are then re-encoded.  Valid at any iteration because Q_2 = G_v Q_1 holds
 * throughout (Lemma "checksum preservation").  R tiles are recovered row-block-wise
 * from R_2 = R_1 G_h with the horizontal generator, the same way.
 *
 * sets (optional, capacity cap ints) receives the decode index sets, one record per
 * decoded grid column (kind 0) then per decoded R row block (kind 1):
 *   kind, index, f1, f2, A_fail[f1], C_fail[f2], C_use[f1]
 * *sets_len gets the number of ints written.  The mask is cleared on success.
 * Nothing is modified when some column or row is unrecoverable.
 * --------------------------------------------------------------------------------- */
static int decode_plan(int nsys, int nchk, const uint8_t* lost_sys, const uint8_t* lost_chk,
                       int f, int* A_fail, int* f1, int* C_fail, int* f2, int* C_use) {
  int a = 0, cf = 0, cu = 0;
  for (int t = 0; t < nsys; ++t) if (lost_sys[t]) A_fail[a++] = t;
  for (int i = 0; i < nchk; ++i) if (lost_chk[i]) C_fail[cf++] = i;
  *f1 = a; *f2 = cf;
  if (a + cf > f) return CQRO_EUNRECOVERABLE;
  for (int i = 0; i < nchk && cu < a; ++i) if (!lost_chk[i]) C_use[cu++] = i;
  if (cu < a) return CQRO_EUNRECOVERABLE;
  return CQRO_OK;
}

int cqro_recover(const cqro_geom* g, const double* Gt, const double* Gh, uint8_t* mask,
                 double* Q, int64_t ldq, double* R, int64_t ldr, int* sets, int cap,
                 int* sets_len, int* n_recovered) {
  const int f = g->f, p_r = g->p_r, p_c = g->p_c, gc = g->grid_cols;
  const int64_t mb = g->mb, nb = g->nb;
  uint8_t ls[256], lc[256];
  int A_fail[128], C_fail[128], C_use[128], f1, f2;
  if (p_r > 256 || p_c > 256 || f > 64) return CQRO_EINVAL;
  /* feasibility check first: nothing is modified when a pattern is unrecoverable */
  for (int j = 0; j < gc; ++j) {
    for (int t = 0; t < p_r; ++t) ls[t] = mask[t * gc + j];
    for (int i = 0; i < f; ++i) lc[i] = mask[(p_r + i) * gc + j];
    if (decode_plan(p_r, f, ls, lc, f, A_fail, &f1, C_fail, &f2, C_use)) return CQRO_EUNRECOVERABLE;
  }
  if (g->protect_r)
    for (int i = 0; i < p_c + f && i < g->grid_rows; ++i) {
      for (int j = 0; j < p_c; ++j) ls[j] = mask[i * gc + j];
      for (int l = 0; l < f; ++l) lc[l] = mask[i * gc + p_c + l];
      if (decode_plan(p_c, f, ls, lc, f, A_fail, &f1, C_fail, &f2, C_use)) return CQRO_EUNRECOVERABLE;
    }
  int pos = 0, nrec = 0;
  double Ghat[64 * 64], Ginv[64 * 64];
  /* Q tiles, per grid column, vertical code */
  for (int j = 0; j < gc; ++j) {
    for (int t = 0; t < p_r; ++t) ls[t] = mask[t * gc + j];
    for (int i = 0; i < f; ++i) lc[i] = mask[(p_r + i) * gc + j];
    decode_plan(p_r, f, ls, lc, f, A_fail, &f1, C_fail, &f2, C_use);
    if (f1 + f2 == 0) continue;
    if (f1 > 0) {
      for (int a = 0; a < f1; ++a)
        for (int bb = 0; bb < f1; ++bb) Ghat[a * f1 + bb] = Gt[C_use[a] * p_r + A_fail[bb]];
      if (invert_small(f1, Ghat, Ginv)) return CQRO_EUNRECOVERABLE;
      for (int64_t col = j * nb; col < (j + 1) * nb; ++col)
        for (int64_t r = 0; r < mb; ++r) {
          double rhs[64];
          for (int a = 0; a < f1; ++a) {
            const int i = C_use[a];
            double acc = Q[g->m_pad + i * mb + r + col * ldq];
            for (int l = 0; l < p_r; ++l)
              if (!ls[l]) acc -= Gt[i * p_r + l] * Q[l * mb + r + col * ldq];
            rhs[a] = acc;
          }
          for (int bb = 0; bb < f1; ++bb) {
            double acc = 0.0;
            for (int a = 0; a < f1; ++a) acc += Ginv[bb * f1 + a] * rhs[a];
            Q[A_fail[bb] * mb + r + col * ldq] = acc;
          }
        }
    }
    for (int e = 0; e < f2; ++e) {
      const int i = C_fail[e];
      for (int64_t col = j * nb; col < (j + 1) * nb; ++col)
        for (int64_t r = 0; r < mb; ++r) {
          double acc = 0.0;
          for (int t = 0; t < p_r; ++t) acc += Gt[i * p_r + t] * Q[t * mb + r + col * ldq];
          Q[g->m_pad + i * mb + r + col * ldq] = acc;
        }
    }
    nrec += f1 + f2;
    int need = 4 + 2 * f1 + f2;
    if (sets && pos + need <= cap) {
      sets[pos++] = 0; sets[pos++] = j; sets[pos++] = f1; sets[pos++] = f2;
      for (int a = 0; a < f1; ++a) sets[pos++] = A_fail[a];
      for (int e = 0; e < f2; ++e) sets[pos++] = C_fail[e];
      for (int a = 0; a < f1; ++a) sets[pos++] = C_use[a];
    }
  }
  /* R tiles, per R block row, horizontal code R_2 = R_1 G_h */
  if (g->protect_r)
    for (int i = 0; i < p_c + f && i < g->grid_rows; ++i) {
      for (int j = 0; j < p_c; ++j) ls[j] = mask[i * gc + j];
      for (int l = 0; l < f; ++l) lc[l] = mask[i * gc + p_c + l];
      decode_plan(p_c, f, ls, lc, f, A_fail, &f1, C_fail, &f2, C_use);
      if (f1 + f2 == 0) continue;
      if (f1 > 0) {
        for (int a = 0; a < f1; ++a)
          for (int bb = 0; bb < f1; ++bb) Ghat[a * f1 + bb] = Gh[A_fail[bb] * f + C_use[a]];
        if (invert_small(f1, Ghat, Ginv)) return CQRO_EUNRECOVERABLE;
        for (int64_t s = 0; s < nb; ++s)
          for (int64_t r = i * nb; r < (i + 1) * nb; ++r) {
            double rhs[64];
            for (int a = 0; a < f1; ++a) {
              const int l = C_use[a];
              double acc = R[r + (g->n + l * nb + s) * ldr];
              for (int j = 0; j < p_c; ++j)
                if (!ls[j]) acc -= Gh[j * f + l] * R[r + (j * nb + s) * ldr];
              rhs[a] = acc;
            }
            for (int bb = 0; bb < f1; ++bb) {
              double acc = 0.0;
              for (int a = 0; a < f1; ++a) acc += Ginv[bb * f1 + a] * rhs[a];
              R[r + (A_fail[bb] * nb + s) * ldr] = acc;
            }
          }
      }
      for (int e = 0; e < f2; ++e) {
        const int l = C_fail[e];
        for (int64_t s = 0; s < nb; ++s)
          for (int64_t r = i * nb; r < (i + 1) * nb; ++r) {
            double acc = 0.0;
            for (int j = 0; j < p_c; ++j) acc += Gh[j * f + l] * R[r + (j * nb + s) * ldr];
            R[r + (g->n + l * nb + s) * ldr] = acc;
          }
      }
      int need = 4 + 2 * f1 + f2;
      if (sets && pos + need <= cap) {
        sets[pos++] = 1; sets[pos++] = i; sets[pos++] = f1; sets[pos++] = f2;
        for (int a = 0; a < f1; ++a) sets[pos++] = A_fail[a];
        for (int e = 0; e < f2; ++e) sets[pos++] = C_fail[e];
        for (int a = 0; a < f1; ++a) sets[pos++] = C_use[a];
      }
    }
  memset(mask, 0, (size_t)g->grid_rows * (size_t)g->grid_cols);
  if (sets_len) *sets_len = pos;
  if (n_recovered) *n_recovered = nrec;
  return CQRO_OK;
}

/* ---------------------------------------------------------------------------------
 * a8. Post-orthogonalisation (Theorem "G_0", Eq. (G0_formula1)):
 *   G_0 = [[I_c + G_1, V], [V^T, -I_{m-c}]],  G = [G_1 V] = G~ (x) I_mb.
 * Dense form: G_0 built explicitly (m_pad x m_pad) and multiplied -- the definition.
 * Z is m_pad x k (column-major), W = G_0 Z.
 * --------------------------------------------------------------------------------- */
int cqro_build_G0(const cqro_geom* g, const double* Gt, double* G0, int64_t ldg) {
  const int64_t mp = g->m_pad, c = g->c, mb = g->mb;
  for (int64_t col = 0; col < mp; ++col)
    for (int64_t r = 0; r < mp; ++r) G0[r + col * ldg] = 0.0;
  /* G = G~ (x) I_mb : G[i*mb + s, t*mb + s] = g~_{i,t} */
  for (int i = 0; i < g->f; ++i)
    for (int t = 0; t < g->p_r; ++t)
      for (int64_t s = 0; s < mb; ++s) {
        const int64_t gr = i * mb + s, gcol = t * mb + s;
        const double val = Gt[i * g->p_r + t];
        if (gcol < c) G0[gr + gcol * ldg] = val;         /* G_1 block */
        else {
          G0[gr + gcol * ldg] = val;                      /* V block, top right */
          G0[gcol + gr * ldg] = val;                      /* V^T block, bottom left */
        }
      }
  for (int64_t r = 0; r < c; ++r) G0[r + r * ldg] += 1.0; /* I_c + G_1 */
  for (int64_t r = c; r < mp; ++r) G0[r + r * ldg] = -1.0; /* -I_{m-c} */
  return CQRO_OK;
}

int cqro_post_orth_dense(const cqro_geom* g, const double* Gt, const double* Z, int64_t ldz,
                         int64_t k, double* W, int64_t ldw) {
  const int64_t mp = g->m_pad;
  double* G0 = (double*)malloc(sizeof(double) * (size_t)(mp * mp));
  if (!G0) return CQRO_EINVAL;
  cqro_build_G0(g, Gt, G0, mp);
#pragma omp parallel for schedule(static)
  for (int64_t col = 0; col < k; ++col)
    for (int64_t r = 0; r < mp; ++r) {
      double acc = 0.0;
      for (int64_t q = 0; q < mp; ++q) acc += G0[r + q * mp] * Z[q + col * ldz];
      W[r + col * ldw] = acc;
    }
  free(G0);
  return CQRO_OK;
}

/* Block form of G_0 Z (Appendix "Proof of Theorem overhead", post-processing pipeline):
 * with H = I_f + G~_1 and Z_t the t-th block row (mb rows),
 *   W_i = sum_{l<f} h_{i,l} Z_l + sum_{t>=f} g~_{i,t} Z_t          (i < f)
 *   W_i = sum_{l<f} g~_{l,i} Z_l - Z_i                             (i >= f)
 * (the garbled v~ indices read as the G~-indexed entries g~_{i,t}, g~_{l,i}). */
int cqro_post_orth_block(const cqro_geom* g, const double* Gt, const double* Z, int64_t ldz,
                         int64_t k, double* W, int64_t ldw) {
  const int f = g->f, p_r = g->p_r;
  const int64_t mb = g->mb;
#pragma omp parallel for schedule(static)
  for (int64_t col = 0; col < k; ++col)
    for (int i = 0; i < p_r; ++i)
      for (int64_t s = 0; s < mb; ++s) {
        double acc = 0.0;
        if (i < f) {
          for (int l = 0; l < f; ++l) {
            const double h = (l == i ? 1.0 : 0.0) + Gt[i * p_r + l];
            acc += h * Z[l * mb + s + col * ldz];
          }
          for (int t = f; t < p_r; ++t) acc += Gt[i * p_r + t] * Z[t * mb + s + col * ldz];
        } else {
          for (int l = 0; l < f; ++l) acc += Gt[l * p_r + i] * Z[l * mb + s + col * ldz];
          acc -= Z[i * mb + s + col * ldz];
        }
        W[i * mb + s + col * ldw] = acc;
      }
  return CQRO_OK;
}

/* ---------------------------------------------------------------------------------
 * a9. Solve (Section 4.1, Eqs. (linearsolve1)-(linearsolve3)): R x = (G_0 Q_1)^T (G_0 y),
 * then back substitution with the n x n upper-triangular R.  Qo = G_0 Q_1 (m_pad x n),
 * yo = G_0 y (m_pad x k).  x is n x k.
 * --------------------------------------------------------------------------------- */
int cqro_back_substitute(int64_t n, const double* R, int64_t ldr, double* x, int64_t ldx,
                         int64_t k) {
  for (int64_t col = 0; col < k; ++col)
    for (int64_t i = n - 1; i >= 0; --i) {
      double acc = x[i + col * ldx];
      for (int64_t j = i + 1; j < n; ++j) acc -= R[i + j * ldr] * x[j + col * ldx];
      x[i + col * ldx] = acc / R[i + i * ldr];
    }
  return CQRO_OK;
}

int cqro_solve_square(int64_t mp, int64_t n, const double* Qo, int64_t ldq, const double* R,
                      int64_t ldr, const double* yo, int64_t ldy, int64_t k, double* x,
                      int64_t ldx) {
#pragma omp parallel for schedule(static)
  for (int64_t col = 0; col < k; ++col)
    for (int64_t j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int64_t r = 0; r < mp; ++r) acc += Qo[r + j * ldq] * yo[r + col * ldy];
      x[j + col * ldx] = acc;
    }
  return cqro_back_substitute(n, R, ldr, x, ldx, k);
}

/* Least squares for tall A through the coded factors (reading for m > n): A = Q_1 R
 * (Corollary "final form"), so the normal equations give
 *   R x = (Q_1^T Q_1)^{-1} Q_1^T y,
 * solved here by the plain definition: the n x n Gram matrix Q_1^T Q_1, a Cholesky
 * factorisation (Golub & Van Loan Alg. 4.2.1), two triangular solves, then R.
 * Q1 is the top m_pad rows of the coded Q (first n columns); y is m_pad x k. */
int cqro_solve_ls(int64_t mp, int64_t n, const double* Q1, int64_t ldq, const double* R,
                  int64_t ldr, const double* y, int64_t ldy, int64_t k, double* x, int64_t ldx) {
  double* Gm = (double*)malloc(sizeof(double) * (size_t)(n * n));
  if (!Gm) return CQRO_EINVAL;
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      double acc = 0.0;
      for (int64_t r = 0; r < mp; ++r) acc += Q1[r + i * ldq] * Q1[r + j * ldq];
      Gm[i + j * n] = acc;
    }
  /* Cholesky Gm = L L^T, L stored in the lower triangle */
  for (int64_t j = 0; j < n; ++j) {
    double acc = Gm[j + j * n];
    for (int64_t p = 0; p < j; ++p) acc -= Gm[j + p * n] * Gm[j + p * n];
    if (!(acc > 0.0)) { free(Gm); return CQRO_EBREAKDOWN; }
    const double ljj = sqrt(acc);
    Gm[j + j * n] = ljj;
    for (int64_t i = j + 1; i < n; ++i) {
      double a2 = Gm[i + j * n];
      for (int64_t p = 0; p < j; ++p) a2 -= Gm[i + p * n] * Gm[j + p * n];
      Gm[i + j * n] = a2 / ljj;
    }
  }
  for (int64_t col = 0; col < k; ++col) {
    double* xc = x + col * ldx;
    for (int64_t j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int64_t r = 0; r < mp; ++r) acc += Q1[r + j * ldq] * y[r + col * ldy];
      xc[j] = acc;
    }
    for (int64_t i = 0; i < n; ++i) { /* L z = rhs */
      double acc = xc[i];
      for (int64_t p = 0; p < i; ++p) acc -= Gm[i + p * n] * xc[p];
      xc[i] = acc / Gm[i + i * n];
    }
    for (int64_t i = n - 1; i >= 0; --i) { /* L^T w = z */
      double acc = xc[i];
      for (int64_t p = i + 1; p < n; ++p) acc -= Gm[p + i * n] * xc[p];
      xc[i] = acc / Gm[i + i * n];
    }
  }
  free(Gm);
  return cqro_back_substitute(n, R, ldr, x, ldx, k);
}
