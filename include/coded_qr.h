/*
 * coded_qr.h -- C ABI of the GB300 coded block Gram-Schmidt QR library.
 *
 * The library computes the fault-tolerant QR of "Coded Computing for Fault-Tolerant
 * Parallel QR Decomposition" (arXiv 2311.11943) on one GPU.  The paper's p_r x p_c
 * processor grid becomes virtual nodes: tiles of one matrix in device memory; a node
 * failure becomes an injected erasure of that node's tiles.
 *
 * Conventions shared by every entry point
 *  - Matrices are column-major.  `ld*` arguments are leading dimensions in elements.
 *  - Element type: double when cfg.dtype == CQR_F64, float when CQR_F32.  The generator
 *    arrays of coded_qr_get_generator are always double.
 *  - Pointers are DEVICE pointers unless the argument is marked "host".
 *  - Ownership: the caller owns A, y, x, Q, R and every output buffer it passes.  The
 *    handle owns the encoded matrix, the coded R, the generator, the erasure mask and its
 *    workspace (allocated by coded_qr_create, or carved from caller memory by
 *    coded_qr_create_in, in which case the caller keeps ownership of that memory and must
 *    keep it alive until coded_qr_destroy).
 *  - Ordering: all GPU work is enqueued on cfg.stream (NULL = the legacy default stream)
 *    in call order.  Argument and state errors are returned synchronously and nothing is
 *    enqueued.  Errors detected on the device (pivot breakdown, a barrier wait that ran
 *    out) are recorded in a device status word and returned by coded_qr_sync_status and
 *    by coded_qr_run, which synchronise the stream.
 *  - Threads: a handle is not internally locked.  Calls on one handle must come from one
 *    host thread at a time (or be serialised by the caller); distinct handles are
 *    independent and may be driven from different threads and streams.
 *  - State machine: create -> encode -> factor* -> [inject_erasure -> recover]* ->
 *    post_orth / solve.  factor runs panels in order and may be split into ranges
 *    (resume from any panel boundary).  Calls out of order return CQR_ESTATE.
 *  - Geometry (Section 2 "Distributed computing model", Eq. (tildeG_eq)): tile height
 *    mb = ceil(m / p_r) (A is zero-padded to m_pad = p_r * mb rows), tile width
 *    nb = n / p_c (p_c must divide n), c = f * mb checksum rows, d = f * nb checksum
 *    columns (0 without R protection), encoded matrix M x N = (m_pad + c) x (n + d).
 *    Node (i, j), i < p_r + f, j < p_c + f (checksum grid columns only with R protection),
 *    owns Q tile (i, j) = rows [i mb, (i+1) mb) x columns [j nb, (j+1) nb) of the coded Q
 *    and, when i < p_c + f, R tile (i, j) = rows [i nb, (i+1) nb) x columns
 *    [j nb, (j+1) nb) of the coded R.  f <= min(p_r, p_c) / 2 (Section 2 "Failure model").
 */
#ifndef CODED_QR_H
#define CODED_QR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cqr_handle_s* cqr_handle;

typedef enum {
  CQR_OK = 0,
  CQR_EINVAL = 1,          /* bad argument or geometry */
  CQR_ENOMEM = 2,          /* device or pinned host allocation failed, or workspace too small */
  CQR_ECUDA = 3,           /* a CUDA runtime call failed (launch, copy, missing device) */
  CQR_ESTATE = 4,          /* call out of order, or erasures pending */
  CQR_EUNRECOVERABLE = 5,  /* more than f erasures in a grid row/column, or singular G^ */
  CQR_EBREAKDOWN = 6,      /* zero or non-finite pivot r_jj in the panel factorisation */
  CQR_ETIMEOUT = 7,        /* a device-side wait exceeded its limit; the kernel gave up */
  CQR_ENOTSUP = 8,         /* configuration not supported by this build */
  CQR_EBOUNDS = 9          /* bounds-checked build only: a kernel found an index outside the
                              extent it was given, recorded it and returned without the access */
} cqr_status;

enum { CQR_F64 = 0, CQR_F32 = 1 };

/* Arithmetic of the trailing-update GEMMs (Algorithm PBMGS, Rbar and Q -= Qbar Rbar). */
enum {
  CQR_MMA_SIMT = 0,   /* CUDA-core FMA in the storage precision (the only choice for F64) */
  CQR_MMA_TF32 = 1,   /* F32 storage: tcgen05 kind::tf32 tensor cores, FP32 accumulation */
  CQR_MMA_3XTF32 = 2, /* F32 storage: split operands hi + lo, three tcgen05 tf32 products */
  CQR_MMA_BF16 = 3,   /* F32 storage: operands rounded to BF16, tcgen05 kind::f16, FP32
                         accumulation */
  CQR_MMA_BF16X3 = 4  /* F32 storage: BF16 hi + lo splits, three tcgen05 BF16 products */
};

enum { CQR_G_UNIF01 = 0, CQR_G_NORMAL = 1 };

typedef struct {
  int64_t m, n;        /* A is m x n, m >= n */
  int32_t p_r, p_c;    /* virtual node grid */
  int32_t f;           /* tolerated failures per grid row and column; 0 = uncoded QR */
  int32_t b;           /* PBMGS panel width (columns per iteration) */
  int32_t dtype;       /* CQR_F64 | CQR_F32 */
  int32_t mma;         /* CQR_MMA_* */
  int32_t protect_r;   /* 1: horizontal checksums protect R (Eq. (encoding)); 0: Q only */
  int32_t gdist;       /* distribution of V~ and G~_h: CQR_G_UNIF01 (paper) | CQR_G_NORMAL */
  int32_t nrhs_max;    /* largest right-hand-side count for post_orth / solve (>= 1) */
  int32_t reorth_block; /* 1: before each panel's ICGS, project the panel once more on all
                           computed columns (block "twice is enough"; an addition to the
                           paper's PBMGS that keeps Q_2 = G_v Q_1); 0: off */
  int32_t panel;       /* CQR_PANEL_*: the panel factorisation (the paper's ICGS by default) */
  int32_t in_node;     /* 0: out-of-node checksum storage (f checksum node rows / columns, the
                          paper's main setting); 1: in-node storage (Section 5): K = f + f
                          ceil(f / (p_r - f)) checksum blocks per code hosted by the data nodes
                          with the load-balanced distribution (Definition innode_distr); the
                          vertical generator is the K x p_r structured matrix of Construction
                          in_node_qr, encoded conventionally (Remark alt_in_node); needs
                          2 K <= p_r and, with protect_r, p_c = p_r */
  int32_t post_orth;   /* CQR_POST_ORTH_*: which form of the post-orthogonalisation (a8) the
                          single-problem verbs apply */
  int32_t reserved;    /* must be 0 */
  uint64_t seed;       /* seed of the generator's SplitMix64 stream */
  double tau;          /* ICGS criterion: reorthogonalise column j when its norm fell below
                          tau times its norm at the panel start.  0 selects 1/sqrt(2);
                          a negative value disables reorthogonalisation. */
  void* stream;        /* cudaStream_t */
} cqr_config;

/* Panel factorisation variants (a3).  ICGS is the paper's (Algorithm CGS with the
 * reorthogonalisation of ICGS, right-looking, one reduction per column).  The others serve
 * the latency / orthogonality comparison: MGS is the same column loop without the
 * reorthogonalisation test; CGS1 is left-looking classical Gram-Schmidt with one reduction per
 * column (projections and norm together, Pythagorean norm); CGS2 repeats its projection
 * once ("twice is enough").  The variants other than ICGS run on the shared-memory panel
 * kernels (not the register-resident FP32 one). */
enum {
  CQR_PANEL_ICGS = 0,
  CQR_PANEL_MGS = 1,
  CQR_PANEL_CGS1 = 2,
  CQR_PANEL_CGS2 = 3
};

/* Post-orthogonalisation forms (a8).  G0 is the paper's Qo = G_0 Q_1 (Theorem "G_0", the
 * sparse block pipeline of the overhead proof).  PROJECTED is Qo = G_0^{-1} (Q_1 + G^T Q_2),
 * G = G~ (x) I_mb: G_0 applied to the orthogonal projection of the coded Q's columns onto the
 * range {[x; G x]} of the encoding (G_0^2 = I + G^T G, G_0 symmetric).  It equals G_0 Q_1
 * whenever the checksum rows satisfy Q_2 = G Q_1 (Lemma "2way_checksum"), so in exact
 * arithmetic it is the paper's matrix; in floating point, where Q_2 drifts from G Q_1 by
 * delta (about u kappa(A) in the storage precision), its loss of orthogonality is of order
 * delta^2 instead of delta.  With the drift D = Q_2 - G Q_1 it equals
 * G_0 (Q_1 + G^T K D), K = (I_f + G~ G~^T)^{-1} acting on block rows (an f x f Cholesky
 * inverse in FP64 on the device), and is computed in that form per tile position, reading
 * Q_1 and Q_2 once: the correction comes from the drift itself, so no large terms cancel.  AUTO picks PROJECTED for CQR_F32 and G0
 * for CQR_F64.  The right-hand side is always transformed as G_0 y, and the square solve
 * uses the selected Qo: Qo^T (G_0 y) = (Q_1 + G^T Q_2)^T y for PROJECTED.  Batches always
 * apply G0. */
enum { CQR_POST_ORTH_AUTO = 0, CQR_POST_ORTH_G0 = 1, CQR_POST_ORTH_PROJECTED = 2 };

/* Geometry record filled by coded_qr_geometry (all int64). */
enum {
  CQR_GEO_M = 0, CQR_GEO_N, CQR_GEO_MB, CQR_GEO_NB, CQR_GEO_MPAD, CQR_GEO_C, CQR_GEO_D,
  CQR_GEO_MROWS, CQR_GEO_NCOLS, CQR_GEO_LDQ, CQR_GEO_LDR, CQR_GEO_GRID_ROWS,
  CQR_GEO_GRID_COLS, CQR_GEO_PANELS, CQR_GEO_CODE_BLOCKS, CQR_GEO_COUNT
};

/* Bytes of device workspace a handle with this configuration needs (for coded_qr_create_in). */
cqr_status coded_qr_workspace_size(const cqr_config* cfg, size_t* bytes);

/* Create a handle; allocates the encoded matrix, the coded R and the workspace with
 * cudaMalloc on the current device.  *out receives the handle. */
cqr_status coded_qr_create(const cqr_config* cfg, cqr_handle* out);

/* Same, but every device buffer is carved from `workspace` (device memory of at least
 * coded_qr_workspace_size bytes, 256-byte aligned, owned by the caller). */
cqr_status coded_qr_create_in(const cqr_config* cfg, void* workspace, size_t bytes,
                              cqr_handle* out);

/* Release the handle (synchronises its stream first).  NULL is accepted. */
cqr_status coded_qr_destroy(cqr_handle h);

/* Fill dims[CQR_GEO_COUNT] (host) with the handle's geometry. */
cqr_status coded_qr_geometry(cqr_handle h, int64_t* dims);

/* a1 + a2.  Generator (Construction "Q-factor checksum-generator matrix", Section 4.2:
 * V~ i.i.d. Unif(0,1) from SplitMix64(seed), G~_1 = -1/2 V~ V~^T, G~ = [G~_1 V~]; G~_h
 * p_c x f from the same stream) computed on the device, then the checksum encode
 * At = [[A, A G_h], [G_v A, G_v A G_h]] (Eq. (encoding)), each checksum tile
 * C_{i,j} = sum_t g~_{i,t} A_{t,j} (Section 4.2).  A: m x n, lda >= m.  Resets the
 * factorisation (next panel = 0, R = 0, no pending erasures). */
cqr_status coded_qr_encode(cqr_handle h, const void* A, int64_t lda);

/* a3-a5.  PBMGS (Appendix A, Algorithm PBMGS) panels [panel_begin, panel_end) on the
 * encoded matrix: ICGS on each panel (Algorithm CGS plus the reorthogonalisation of ICGS),
 * Rbar = Qbar^T Q[:, i+b : N], Q[:, i+b : N] -= Qbar Rbar, Rbar stored into R.
 * panel_begin must equal the next unfactored panel; panel_end = -1 means the last panel.
 * Returns CQR_ESTATE while erasures are pending (erased tiles hold NaN).
 *
 * Scheduling (FP32 tensor-core handles whose panel runs on one thread-block cluster): the
 * trailing update of each panel is split into the next panel's columns, on an internal
 * stream of the highest priority, and the rest, on an internal stream of the lowest
 * priority that overlaps the next panel's factorisation; kernels on the first stream use
 * programmatic dependent launch.  Both streams fork from and join into cfg.stream inside the
 * call.  Environment switches, for comparisons only: CQR_LOOKAHEAD=0 (one stream, no
 * split), CQR_PDL=0 (no programmatic dependent launch), CQR_PANEL_REG=0 (no register-
 * resident panel kernel), CQR_PANEL_CLUSTER=0 (no single-cluster panel kernels),
 * CQR_PANEL_RPL=r (rows per lane of the shared-memory / grid panel kernels). */
cqr_status coded_qr_factor(cqr_handle h, int32_t panel_begin, int32_t panel_end);

/* a6.  Fail-stop erasure of nodes (Section 2 "Failure model"): tiles (host) holds `count`
 * (i, j) pairs; each node's Q tile and, with R protection and i < p_c + f, its R tile are
 * overwritten with NaN and marked lost.  Allowed any time after encode. */
cqr_status coded_qr_inject_erasure(cqr_handle h, const int32_t* tiles, int32_t count);

/* a7.  Recovery (Appendix, Lemma on the recovery overhead, Eq. (A_recov)): per grid column,
 * G^ = G~[C_use, A_fail] (C_use = the f1 lowest-index surviving checksum rows) is inverted
 * in FP64 on the device, the lost systematic tiles are rebuilt from the surviving tiles and
 * checksums, and lost checksum tiles are re-encoded; R tiles are rebuilt the same way from
 * R_2 = R_1 G_h.  Valid at every iteration by the checksum-preservation Lemma.
 * *n_recovered (host, may be NULL) receives the number of Q tiles rebuilt.  On
 * CQR_EUNRECOVERABLE nothing is modified and the erasures stay pending. */
cqr_status coded_qr_recover(cqr_handle h, int32_t* n_recovered);

/* a6 by node: nodes holds count pairs (node row, node column).  Out-of-node storage: nodes of
 * the extended (p_r + f) x (p_c + f) grid, each holding one tile (same as
 * coded_qr_inject_erasure).  In-node storage: nodes of the p_r x p_c grid; a failed node loses
 * its data tile and every checksum tile it hosts.  coded_qr_run's plan uses the same node
 * coordinates. */
cqr_status coded_qr_inject_node_failure(cqr_handle h, const int32_t* nodes, int32_t count);

/* a8.  Post-orthogonalisation (Theorem "G_0", Eq. (G0_formula1); sparse block pipeline of
 * the overhead proof): Qo = G_0 Q_1 (m_pad x n) with G_0 = [[I + G_1, V], [V^T, -I]].
 * Q == NULL overwrites Q_1 inside the handle (then solve uses it directly).
 * y (m x nrhs, may be NULL) is transformed too: yo = G_0 [y; 0] (m_pad x nrhs) into yo,
 * or into the handle's workspace when yo == NULL.  Requires a finished factorisation. */
cqr_status coded_qr_post_orth(cqr_handle h, void* Q, int64_t ldq, const void* y, int64_t ldy,
                              void* yo, int64_t ldyo, int32_t nrhs);

/* a9.  Solve (Section 4.1, Eqs. (linearsolve1)-(linearsolve3)): for square A,
 * R x = (G_0 Q_1)^T (G_0 y) and a triangular solve with the n x n R.  For m > n (and
 * whenever m is not a multiple of p_r) least squares through A = Q_1 R (Corollary "final
 * form"): R x = (Q_1^T Q_1)^{-1} Q_1^T y with Q_1^T Q_1 = I - Q_2^T Q_2 (orthonormality of
 * the coded Q), formed and Cholesky-factored in FP64 on the device (n x n).
 * y: m x nrhs, x: n x nrhs. */
cqr_status coded_qr_solve(cqr_handle h, const void* y, int64_t ldy, void* x, int64_t ldx,
                          int32_t nrhs);

/* a9 under the name of the method's problem statement, min |A x - y| (Section 4.1 for square
 * A; for tall A the least-squares reading through A = Q_1 R of Corollary "final form").  The
 * same call as coded_qr_solve: the same arguments, layout, ownership and errors, and the same
 * result bit for bit. */
cqr_status coded_qr_solve_ls(cqr_handle h, const void* y, int64_t ldy, void* x, int64_t ldx,
                             int32_t nrhs);

/* The whole hot path in one call: encode, factor with the erasure plan applied, post_orth
 * (in place) and solve.  plan (host) holds plan_len triples (panel, i, j): node (i, j) is
 * erased at the start of that panel and recovered before it runs.  With
 * flags & CQR_RUN_HOST_BUFFERS, A, y and x are HOST pointers and the library copies them
 * to and from the device inside the call.  Synchronises cfg.stream and returns the device
 * status. */
#define CQR_RUN_HOST_BUFFERS 1u
cqr_status coded_qr_run(cqr_handle h, const void* A, int64_t lda, const void* y, int64_t ldy,
                        void* x, int64_t ldx, int32_t nrhs, const int32_t* plan,
                        int32_t plan_len, uint32_t flags);

/* Borrow the coded factors: *Q (M x N, leading dimension *ldq) and *R (N x N, *ldr) stay
 * owned by the handle and valid until the next encode or destroy. */
cqr_status coded_qr_get_factors(cqr_handle h, void** Q, int64_t* ldq, void** R, int64_t* ldr);

/* Copy the generator to the host: Gt f x p_r row-major, Gh p_c x f row-major (either may be
 * NULL).  Synchronises the stream. */
cqr_status coded_qr_get_generator(cqr_handle h, double* Gt, double* Gh);

/* Decode index sets of every recover call since encode, one record per decoded grid column
 * (kind 0) then per decoded R block row (kind 1): kind, index, f1, f2, A_fail[f1],
 * C_fail[f2], C_use[f1].  buf (host) receives up to cap ints; *len the full length. */
cqr_status coded_qr_get_decode_sets(cqr_handle h, int32_t* buf, int32_t cap, int32_t* len);

/* Counters since encode (host, out[4]): reorthogonalisations, recovered Q tiles, panels run,
 * erasures injected.  Synchronises the stream. */
cqr_status coded_qr_stats(cqr_handle h, int64_t* out);

/* Synchronise the stream and return the first device-side error since encode (CQR_OK when
 * none), clearing it. */
cqr_status coded_qr_sync_status(cqr_handle h);

/* Bound of the waits between the CTAs of one panel factorisation (instrumentation, no
 * counterpart in the paper; the paper assumes fail-stop nodes and an external failure
 * detector).  Every such wait -- the partial-vector exchange of the cluster panel, the
 * grid barrier of the cooperative panel -- gives up after `cycles` SM clock cycles
 * (0 restores the default, about one second): the CTA records CQR_ETIMEOUT in the device
 * status word, every CTA of the launch leaves at its next wait, and coded_qr_sync_status
 * returns CQR_ETIMEOUT.  The factors computed after that are not meaningful; a new encode
 * clears the status.  The tensor-core GEMMs keep their own fixed bound.  A deployment may
 * shorten the bound to detect a stalled launch sooner; the tests set it to a few cycles so
 * that every exchange of a correct launch runs out.  Takes effect for the next launches. */
cqr_status coded_qr_set_wait_limit(cqr_handle h, int64_t cycles);

/* Bounds-checked build (instrumentation, no counterpart in the paper; the stand-in for a
 * memory checker on GPUs where none can run).  The library built with -DCQR_DEBUG_BOUNDS
 * (libcoded_qr_debug.so) checks, in each kernel of the hot path, that the indices it is about to
 * use stay inside the extents it was given (leading dimensions against row counts, tile and
 * plan indices against the grid, slices against the panel).  A failed check records
 * CQR_EBOUNDS and the check's site number in a device word of its source file and returns
 * without the access: it never traps.  coded_qr_debug_bounds synchronises the device, collects
 * and clears those words and returns CQR_EBOUNDS with *site (host, may be NULL) set to the
 * first failed site, else CQR_OK; coded_qr_debug_bounds_selftest enqueues on `stream` one
 * guarded write past a four-element array (site 199), which the check must catch.  In the
 * normal build both return CQR_ENOTSUP and launch nothing. */
cqr_status coded_qr_debug_bounds(int32_t* site);
cqr_status coded_qr_debug_bounds_selftest(void* stream);

/* Exchange-latency probe (a measurement aid: the paper has no counterpart).  The panel of
 * Appendix A's Algorithm CGS (right-looking, with the ICGS criterion) performs one reduction
 * across its CTAs per column; with everything else on chip, those reductions bound how fast a
 * column can go.  This call runs the reductions of one M x bk FP32 panel -- a first one of
 * 2 bk entries, then bk - 1 - j entries for column j -- with the panel kernel's own exchange
 * code, launch shape and shared-memory footprint but no column arithmetic, `reps` times in one
 * launch after a one-launch warm-up, and stores the mean device time per panel column in
 * microseconds (CUDA events on `stream`; the call synchronises the stream).
 *   kind 0: the register panel (one cluster; bk <= 128 and M within its registers);
 *   kind 1: the shared-memory panel as the handle plans it for M rows (one cluster of up to
 *           16 CTAs, the two-level exchange over clusters of 16 or 8, or the grid barrier).
 * It allocates its scratch with cudaMalloc and frees it.  Returns CQR_EINVAL when the panel does
 * not fit the chosen kind (or its slices would not be in shared memory), the device status
 * (CQR_ETIMEOUT) when an exchange wait ran out, CQR_ECUDA when a sum came back wrong or a CUDA
 * call failed. */
cqr_status coded_qr_probe_exchange(int32_t kind, int64_t M, int32_t bk, int32_t reps,
                                   double* us_per_column, void* stream);

/* Profile of the library's own kernels (instrumentation, no counterpart in the paper).
 * Launch counts per kernel class are always kept; with enable != 0 every launch site is
 * also bracketed by a pair of CUDA events on the stream its launches go to (cfg.stream, or
 * one of the two internal streams of the look-ahead; classes on different streams overlap).  coded_qr_profile_read
 * synchronises the stream and fills (host) ms[k] (device milliseconds) and launches[k]
 * for the first cap classes (CQR_PROF_CLASSES in total) since the last reset; reset != 0
 * clears the accumulators.  coded_qr_profile_name gives the class name (NULL past the end). */
#define CQR_PROF_CLASSES 17
cqr_status coded_qr_profile(cqr_handle h, int32_t enable);
cqr_status coded_qr_profile_read(cqr_handle h, double* ms, int64_t* launches, int32_t cap,
                                 int32_t reset);
const char* coded_qr_profile_name(int32_t cls);

/* Allocation-free panel factorisation (the paper has no counterpart: this is a deployment
 * aid).  Some callers cannot call cudaMalloc where they need a panel factored: a caching
 * allocator that must not be re-entered from inside its own callbacks, a host that has handed
 * every byte of device memory to another framework, or a latency-critical path that must not
 * take the driver's allocation lock (cudaMalloc can synchronise the device).  This call runs
 * the same ICGS algorithm as coded_qr_factor's panel step (one reduction per column, the same
 * reorthogonalisation criterion) on the grid-barrier panel kernel; the handle's panel step
 * may pick a register or cluster kernel that sums in another order, so the two agree to
 * rounding, not bit for bit.  Its scratch (partial sums, barrier counter, status word) lives
 * in a fixed device array of 1,311,232 bytes inside the library, which every GPU that loads
 * the library holds until the process exits; nothing is allocated.
 *   Q:  M x bk panel (device, column-major, ld ldq >= M), orthonormalised in place;
 *   R:  bk x bk (device, ld ldr >= bk): receives the upper triangle (caller zeroes it first);
 *   tau: reorthogonalisation criterion as cqr_config.tau; status: optional device int[4]
 *   that receives the device-side status word (CQR_EBREAKDOWN, CQR_ETIMEOUT), else NULL.
 * Limits: bk <= 256 and M <= min(160, number of SMs) x 1024 rows (the panel must fit that
 * many co-resident CTAs: 155,648 rows on a 152-SM GPU); larger sizes return CQR_EINVAL
 * without launching anything.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current) and caches it for the life of the
 * process, so make that first call before any stream capture; after cudaDeviceReset the
 * cached address is stale and further calls in that process are not supported.  All calls
 * share the one array, and the array keeps the previous call's contents (the call clears the
 * barrier counter and the status word itself): calls whose work overlaps on the GPU
 * (different streams, or several host threads) race and must be serialised by the caller. */
cqr_status coded_qr_panel_icgs_noalloc(int32_t dtype, int64_t M, int32_t bk, void* Q, int64_t ldq,
                                       void* R, int64_t ldr, double tau, int32_t* status,
                                       void* stream);

/* ---------------------------------------------------------------------------------------
 * Batches.  `count` independent instances of the coded method (Section 4 applied to each
 * m_i x n_i matrix; tall-skinny shapes), FP32 on the CUDA cores, sharing p_r, p_c, f, protect_r,
 * gdist, tau, seed (one generator for every instance) and the stream of the configuration.
 * cfg->m and cfg->n are ignored; cfg->dtype must be CQR_F32 and cfg->mma CQR_MMA_SIMT
 * (CQR_ENOTSUP otherwise), cfg->reorth_block must be 0.  cfg->b in 1..64 fixes every panel
 * width; cfg->b == 0 picks each width from the instance's shape (32 for n_i >= 96, else 16),
 * which coded_qr_batched_autotune can then refine.
 * Every instance is factorised by one thread-block cluster of the persistent factor launch;
 * the results are those of the single-instance verbs up to rounding order.  Each instance
 * owns its encoded matrix Q (M_i x N_i) and R (N_i x N_i) inside the batch's device memory.
 * Per-instance arrays (m, n, A, lda, panel_end) are host arrays of length count. */
typedef struct cqr_batched_s* cqr_batched;

enum { CQR_BATCH_GRAPH = 1, CQR_BATCH_POST_ORTH = 2, CQR_BATCH_HOST_BUFFERS = 4 };

/* Allocate the batch (cudaMalloc on the current device) and compute the shared generator.
 * Every instance must satisfy the single-instance rules (m_i >= n_i, p_c | n_i, ...). */
cqr_status coded_qr_batched_create(const cqr_config* cfg, const int64_t* m, const int64_t* n,
                                   int32_t count, cqr_batched* out);
cqr_status coded_qr_batched_destroy(cqr_batched bh);
/* Geometry of instance i, as coded_qr_geometry. */
cqr_status coded_qr_batched_geometry(cqr_batched bh, int32_t i, int64_t* dims);
/* a2 for every instance: A[i] (device pointer, m_i x n_i column-major, lda[i] >= m_i). */
cqr_status coded_qr_batched_encode(cqr_batched bh, const void* const* A, const int64_t* lda);
/* a3-a5: instance i runs its panels from where it stopped up to panel_end[i] (NULL: to the
 * last panel), all instances in one persistent launch. */
cqr_status coded_qr_batched_factor(cqr_batched bh, const int32_t* panel_end);
/* a6: tiles holds count triples (instance, grid row, grid column), as
 * coded_qr_inject_erasure per instance. */
cqr_status coded_qr_batched_inject_erasure(cqr_batched bh, const int32_t* tiles, int32_t count);
/* a7 for every instance with pending erasures, one launch; CQR_EUNRECOVERABLE (nothing
 * launched) when an instance lost more than f tiles of one code. */
cqr_status coded_qr_batched_recover(cqr_batched bh, int32_t* n_recovered);
/* a8: Q_1 <- G_0 Q_1 in place for every instance (after the last panel). */
cqr_status coded_qr_batched_post_orth(cqr_batched bh);
/* The whole sequence: encode, factor up to each instance's erasure panel, erase, recover,
 * factor to the end, and with CQR_BATCH_POST_ORTH the post-orthogonalisation.  erasures
 * holds count quadruples (instance, panel t, grid row, grid column): the tiles are lost at
 * the start of panel t (every tile of one instance at the same t, CQR_ENOTSUP otherwise).
 * With CQR_BATCH_GRAPH the launches are recorded into a CUDA graph on the first call and the
 * graph is replayed while the erasure list, the inputs and the tuning stay the same.
 * With CQR_BATCH_HOST_BUFFERS, A[i] are host pointers (pinned memory gives full copy speed):
 * each instance's A is copied on the batch's stream (one 2-D copy per instance) straight into
 * the systematic block of its own encoded matrix, and the encode then runs in place there.
 * The call returns once everything is enqueued, so the host arrays must stay untouched until
 * the stream has passed the copies (coded_qr_batched_sync_status synchronises it).  The
 * recorded graph does not depend on the host pointers. */
cqr_status coded_qr_batched_run(cqr_batched bh, const void* const* A, const int64_t* lda,
                                const int32_t* erasures, int32_t count, int32_t flags);
/* Autotuner: times coded_qr_batched_run on A with the given erasure list (CUDA events, best
 * of reps after one untimed run) over the cluster sizes 1/2/4/8 and the width rules
 * 16/32/64/shape, then refines the width per class of encoded height (< 1024, < 4096,
 * >= 4096 rows); keeps the fastest and leaves the batch encoded and factorised (without
 * erasures) with it.  The erasure panels refer to the current widths; for other widths each
 * event keeps its column position.  *cluster (host, optional) receives the cluster size. */
cqr_status coded_qr_batched_autotune(cqr_batched bh, const void* const* A, const int64_t* lda,
                                     const int32_t* erasures, int32_t count, int32_t reps,
                                     int32_t* cluster);
/* Set / read the tuning: cluster size (1, 2, 4, 8) and the panel widths b[count] (host; NULL
 * on set: the shape rule).  Setting it requires a new encode. */
cqr_status coded_qr_batched_set_tuning(cqr_batched bh, int32_t cluster, const int32_t* b);
cqr_status coded_qr_batched_get_tuning(cqr_batched bh, int32_t* cluster, int32_t* b);
/* Borrow instance i's coded factors (device, owned by the batch). */
cqr_status coded_qr_batched_get_factors(cqr_batched bh, int32_t i, void** Q, int64_t* ldq,
                                        void** R, int64_t* ldr);
/* Decode index sets of instance i since the last encode/run (format of
 * coded_qr_get_decode_sets). */
cqr_status coded_qr_batched_get_decode_sets(cqr_batched bh, int32_t i, int32_t* buf, int32_t cap,
                                            int32_t* len);
/* Synchronise; the status of the first instance whose device status word is set (CQR_OK if
 * none), *first_bad its index or -1, *reorth the reorthogonalisations of all instances. */
cqr_status coded_qr_batched_sync_status(cqr_batched bh, int32_t* first_bad, int64_t* reorth);

/* Phase clocks of the persistent factor launch (instrumentation, no counterpart in the paper).
 * With enable != 0 every later factor launch of the batch (direct, or recorded into a new
 * graph) adds, for each CTA, the SM clock cycles it spent in each phase to counters of the
 * batch (allocated on the first enable): in-launch recovery, panel, the product Qbar^T B,
 * its reduction into Rbar, the update B -= Qbar Rbar, the rest (work queue, the wait at the
 * end), and the parts of the two products spent at the top of each pipeline stage waiting for
 * its copies and the CTA barrier.  Thread 0 of the CTA reads the clock at the phase
 * boundaries, so the cost when on is a few instructions per pipeline stage; when off, one
 * test per boundary.  coded_qr_batched_phases synchronises the stream and writes
 * cycles[0..7] (host, summed over the CTAs, in the order above) and cycles[8] (the number of
 * CTAs that added theirs); with reset != 0 it then zeroes the counters.  CQR_ESTATE if the
 * clocks were never enabled. */
cqr_status coded_qr_batched_profile(cqr_batched bh, int32_t enable);
cqr_status coded_qr_batched_phases(cqr_batched bh, int64_t* cycles, int32_t reset);

/* Name of the last CUDA error behind a CQR_ECUDA of a batch entry point on this host thread. */
const char* coded_qr_batched_last_error(void);

/* Reverse mode (no counterpart in the paper, which has no differentiation): gradients of a
 * loss through the outputs of the coded method.  Both verbs need the handle after the last
 * panel with no pending erasure; they ACCUMULATE into Abar (m x n, ld ldab) and ybar, use
 * the handle's stream, and allocate scratch device memory on first use (kept until destroy).
 *
 * coded_qr_adjoint_qr: outputs Q = G_0 Q_1 (m_pad x n, as written by coded_qr_post_orth into
 * a caller buffer) and the coded R (n x n) satisfy G_0 A = Q R with Q^T Q = I (Theorem on
 * post-orthogonalisation, Section 4.3), so the thin-QR reverse rule applies to G_0 A:
 *   M = R Rbar^T - Qbar^T Q,  Bbar = (Qbar + Q copyltu(M)) R^{-T},  Abar += G_0^T Bbar
 * (copyltu(M) = tril(M) + tril(M,-1)^T; G_0 is symmetric).  Qbar (m_pad x n) or Rbar (n x n,
 * only its upper triangle is meaningful) may be NULL, not both. */
cqr_status coded_qr_adjoint_qr(cqr_handle h, const void* Q, int64_t ldq, const void* Qbar,
                               int64_t ldqb, const void* Rbar, int64_t ldrb, void* Abar,
                               int64_t ldab);
/* coded_qr_adjoint_lstsq: x = argmin |A x - y| (x n x nrhs from coded_qr_solve on this handle,
 * A m x n with full column rank, y m x nrhs).  With z = (A^T A)^{-1} xbar evaluated through the
 * coded factors as R^{-1} (I - Q_2^T Q_2)^{-1} R^{-T} xbar (FP64 conjugate gradients for the
 * middle factor) and r = y - A x:  Abar += r z^T - (A z) x^T,  ybar += A z.  Abar or ybar may
 * be NULL.  Needs Q_1 in the handle (CQR_ESTATE after an in-place post-orthogonalisation). */
cqr_status coded_qr_adjoint_lstsq(cqr_handle h, const void* A, int64_t lda, const void* y,
                                  int64_t ldy, const void* x, int64_t ldx, const void* xbar,
                                  int64_t ldxb, int32_t nrhs, void* Abar, int64_t ldab,
                                  void* ybar, int64_t ldyb);

/* E1 MDS statistics (Theorem prob_det, Section 4.2, and the comparison of the structured
 * generator with a completely random one that follows it): over every square submatrix S of
 * the f x p_r matrix G (host, row-major, FP64), the least |det S| and the largest 2-norm
 * condition number (+inf when sigma_min <= 2^-52 sigma_max).  min_det[k], max_cond[k] (host, f + 1 entries) hold
 * the values over the k x k submatrices, k = 1..f, and entry 0 those over all of them;
 * *count (optional) receives the number of submatrices.  One GPU thread per submatrix:
 * |det| by LU with partial pivoting, singular values by one-sided Jacobi, FP64.
 * 1 <= f <= 6, f <= p_r <= 64.  Allocates and frees a small device buffer; synchronises
 * `stream` (cudaStream_t). */
cqr_status coded_qr_mds_stats(const double* G, int32_t f, int32_t p_r, double* min_det,
                              double* max_cond, int64_t* count, void* stream);

/* Static description of a status code. */
const char* coded_qr_errstr(cqr_status s);

#ifdef __cplusplus
}
#endif
#endif /* CODED_QR_H */
