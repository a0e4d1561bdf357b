// cqr_kernels.cuh -- launchers of the coded-QR kernels (host-callable, stream-ordered).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cqr {

// Geometry of one coded problem (see coded_qr.h, "Geometry").
struct Geo {
  int64_t m, n, mb, nb, m_pad, c, d, M, N, ldq, ldr;
  int p_r, p_c, f, protect_r, grid_rows, grid_cols, panels, b;
};

// Decode plan of one grid column (Q, vertical code) or one R block row (horizontal code).
constexpr int kMaxF = 16;
constexpr int kMaxCode = 128;  // p_r + f (Q) or p_c + f (R)
struct DecodePlan {
  int kind;       // 0: Q grid column `idx`; 1: R block row `idx`
  int idx;
  int f1, f2;     // lost systematic / lost checksum tiles
  int nsys;       // systematic tiles in the code (p_r for Q, p_c for R)
  int pad_;
  int A_fail[kMaxF];
  int C_fail[kMaxF];
  int C_use[kMaxF];
};

// Panel factorisation launch plan.
struct PanelPlan {
  int G;          // CTAs (cooperative)
  int rpc;        // rows per CTA
  int rpc_pad;    // shared-memory column stride
  int smem;       // 1: panel slice resident in shared memory
  int cluster;    // 1: one thread-block cluster (distributed shared memory reductions)
  int hier;       // 1: grid of clusters with the two-level exchange (FP32, shared-memory slices)
  int hcs;        // two-level: CTAs per cluster (8, or 16 with CQR_HIER_CS=16)
  size_t smem_bytes;
};

template <typename T>
cudaError_t launch_generator(int f, int p_r, int p_c, uint64_t seed, int gdist, double* Gt,
                             double* Gh, T* Gt_t, T* Gh_t, cudaStream_t st);

// status: the device status word (unused by the current encode kernels, which do not wait).
template <typename T>
cudaError_t launch_encode(const Geo& g, const T* A, int64_t lda, const T* Gt, const T* Gh, T* Q,
                          int* status, cudaStream_t st);


// allow_hier: a grid of more than 48 FP32 CTAs may use the two-level exchange, in clusters of
// hier_cs (16, or 8) CTAs
PanelPlan plan_panel(int64_t M, int bk, size_t elem, int num_sms, bool allow_cluster,
                     bool allow_hier = true, int hier_cs = 16);
template <typename T>
bool panel_cluster_fits(const PanelPlan& pp);
// Whether every cluster of a two-level plan can be resident at once.
template <typename T>
bool panel_hier_fits(const PanelPlan& pp);
size_t panel_partial_bytes(int bk, size_t elem, int num_sms);

// Bounds words of the bounds-checked build (-DCQR_DEBUG_BOUNDS), one per source file: read and
// cleared; (0, 0) in the normal build.
cudaError_t bounds_take_kernels(int* code, int* site);
cudaError_t bounds_take_panel(int* code, int* site);
cudaError_t bounds_take_panel_reg(int* code, int* site);
cudaError_t bounds_take_tc(int* code, int* site);
// A guarded write past a four-element array (the bounds-checked build's self-test).
cudaError_t launch_bounds_selftest(int idx, cudaStream_t st);

// Register-resident FP32 panel in one cluster (cqr_panel_reg.cu).
bool plan_panel_reg(int64_t M, int bk, int* rpl, int* cpw, int* G);
bool panel_reg_cluster_fits(int rpl, int cpw, int G);
// pdl: launch with programmatic stream serialization (the kernel waits for its predecessor).
// wait_limit: bound of each exchange wait in SM cycles (<= 0: kWaitLimitCycles).
cudaError_t launch_panel_reg(int rpl, int cpw, int G, float* Q, int64_t ldq, float* R, int64_t ldr,
                             int64_t M, int bk, double tau, int* status, int col0, cudaStream_t st,
                             bool pdl = false, long long wait_limit = 0);

// variant: 0 the paper's ICGS panel (MGS order; no reorthogonalisation when tau <= 0),
// 1 left-looking CGS with one reduction per column, 2 CGS2.
template <typename T>
cudaError_t launch_panel(const PanelPlan& pp, T* Q, int64_t ldq, T* R, int64_t ldr, int64_t M,
                         int bk, double tau, T* part, unsigned* bar, int* status, int col0,
                         cudaStream_t st, int variant = 0, long long wait_limit = 0);

// Exchange probes (measurement aids): `reps` times the per-column reductions of a panel of
// bk FP32 columns, without the column arithmetic, with the exchange code, launch shape and
// shared memory of the shared-memory panel on plan pp (cqr_panel.cu) or of the register panel
// for M rows (cqr_panel_reg.cu); *bad counts sums that came back wrong.  part, bar: the
// panel's partial buffer (panel_partial_bytes) and barrier counter.
cudaError_t launch_exchange_probe(const PanelPlan& pp, int bk, int reps, float* part,
                                  unsigned* bar, int* status, int* bad, cudaStream_t st);
cudaError_t launch_exchange_probe_reg(int64_t M, int bk, int reps, int* status, int* bad,
                                      cudaStream_t st);

// Rbar partials: P[s] (bk x w, col-major) = Qbar^T Qtrail over K-split s.
template <typename T>
cudaError_t launch_gemm_tn_splitk(const T* A, int64_t lda, const T* B, int64_t ldb, int64_t K,
                                  int bk, int64_t w, int splits, T* P, cudaStream_t st);
// Sum the split partials into R (store, or add when accumulate) and the compact Rbar (ld = bk).
template <typename T>
cudaError_t launch_splitk_reduce(const T* P, int splits, int bk, int64_t w, T* R, int64_t ldr,
                                 T* Rb, cudaStream_t st, int accumulate = 0);
// C (M x w) -= A (M x bk) * B (bk x w).
template <typename T>
cudaError_t launch_gemm_nn_sub(const T* A, int64_t lda, const T* B, int64_t ldb, T* C,
                               int64_t ldc, int64_t M, int bk, int64_t w, cudaStream_t st);

template <typename T>
cudaError_t launch_poison(const Geo& g, const int* tiles, int count, T* Q, T* R,
                          cudaStream_t st);

template <typename T>
cudaError_t launch_decode(const Geo& g, const DecodePlan* plans_dev, int nplans, int max_h,
                          const double* Gt, const double* Gh, T* Q, T* R, int* status,
                          cudaStream_t st);

// W = G_0 Z for Z (m_pad x k, rows >= zrows read as 0); W may alias Z.
template <typename T>
cudaError_t launch_post_orth(const Geo& g, const T* Gt_t, const T* Z, int64_t ldz,
                             int64_t zrows, int64_t k, T* W, int64_t ldw, cudaStream_t st);

// Drift-robust post-orthogonalisation W = G_0^{-1} (Q_1 + G^T Q_2) (coded_qr.h,
// CQR_POST_ORTH_PROJECTED) of the first k columns of the coded Q (Q_1 rows 0 .. m_pad-1, Q_2
// rows m_pad .. m_pad+c-1, ld ldq) into W (m_pad x k; W may alias Q_1).  Two launches: the
// f x f FP64 inverse K = (I_f + G~ G~^T)^{-1} from the FP64 generator Gt into K64 and its
// storage-type copy Kt (kMaxF^2 entries each), then the tile pipeline.
template <typename T>
cudaError_t launch_post_orth_projected(const Geo& g, const double* Gt, const T* Gt_t, double* K64,
                                       T* Kt, const T* Q, int64_t ldq, int64_t k, T* W, int64_t ldw,
                                       cudaStream_t st);

// z (n x k) = Qo^T yo, Qo rows x n.
template <typename T>
cudaError_t launch_gemv_t(const T* Qo, int64_t ldq, int64_t rows, int64_t n, const T* y,
                          int64_t ldy, int64_t k, T* z, int64_t ldz, cudaStream_t st);

// In-place back substitution R x = z (R n x n upper, k right-hand sides) on one thread-block
// cluster; cudaErrorInvalidValue when the x blocks do not fit one cluster's shared memory
// (n above about 300,000 in FP64, 700,000 in FP32).
template <typename T>
cudaError_t launch_trsv_upper(const T* R, int64_t ldr, int64_t n, T* x, int64_t ldx, int64_t k,
                              cudaStream_t st);

// Tall least squares through the coded factors: x (n, one column) = (I - Q_2^T Q_2)^{-1} Q_1^T y
// by conjugate gradients in FP64 (cooperative launch); ws holds 7 n + c + 2 #SMs doubles.
// With u non-null the right-hand side is u (n entries) instead of Q_1^T y.
template <typename T>
cudaError_t launch_ls_cg(const T* Q, int64_t ldq, int64_t m, int64_t m_pad, int64_t c, int64_t n,
                         const T* y, T* x, double* ws, unsigned* bar, int* status, int num_sms,
                         cudaStream_t st, const T* u = nullptr);

// ---------------------------------------------------------------- adjoint building blocks
// C (M x N) = alpha op(A) op(B) + beta C (op = transpose when ta / tb); beta == 0 ignores C.
template <typename T>
cudaError_t launch_gemm_general(int ta, int tb, int64_t M, int64_t N, int64_t K, T alpha,
                                const T* A, int64_t lda, const T* B, int64_t ldb, T beta, T* C,
                                int64_t ldc, cudaStream_t st);
// S = tril(M) + tril(M, -1)^T (n x n, ld n).
template <typename T>
cudaError_t launch_copyltu(const T* Mm, int64_t n, T* S, cudaStream_t st);
// Y += alpha X (or Y = alpha X when overwrite); element (i, j) at i rs + j cs.
template <typename T>
cudaError_t launch_axpy2d(int64_t rows, int64_t cols, T alpha, const T* X, int64_t xrs, int64_t xcs,
                          T* Y, int64_t yrs, int64_t ycs, bool overwrite, cudaStream_t st);
// X op(R) = B in place, R n x n upper; trans = 1: X R^T = B; trans = 0: X R = B.
template <typename T>
cudaError_t launch_trsm_right(int trans, const T* R, int64_t ldr, int64_t n, T* B, int64_t rs,
                              int64_t cs, int64_t m, cudaStream_t st);

// ---------------------------------------------------------------- batches of instances
// One instance of a batch of independent coded QRs (device copy).  Every batched launch maps
// a flat list of "virtual blocks" onto the instances: off[i] .. off[i+1]-1 belong to
// instance i (prefix sums over the per-instance block counts of the single-instance grid).
template <typename T>
struct BatchInst {
  Geo g;
  T* Q;             // encoded matrix, M x N, ld g.ldq
  T* R;             // N x N, ld g.ldr
  const T* A;       // input (encode), m x n, ld lda
  int64_t lda;
  int* status;      // this instance's status words
  int b;            // panel width
  // recovery inside the batched factor launch: at the start of panel rec_at - 1 (0: none),
  // the tiles [tile0, tile0 + ntiles) of the poisoned-tile list are poisoned and the codes
  // [plan0, plan0 + nplans) of the decode-plan list decoded
  int rec_at;
  int tile0, ntiles;
  int plan0, nplans;
};

struct BatchPlan {
  int inst;
  int pad_;
  DecodePlan p;
};

struct BatchTile {  // one poisoned tile
  int inst, i, j, isR;
};

// Virtual blocks of the single-instance encode / post-orth grids (32 x 8 threads per block).
int64_t batch_encode_blocks(const Geo& g, bool horizontal);
int64_t batch_post_orth_blocks(const Geo& g);
int64_t batch_decode_blocks(const Geo& g, const DecodePlan& p);

template <typename T>
cudaError_t launch_b_encode(const BatchInst<T>* inst, int count, const int64_t* off_v,
                            int64_t total_v, const int64_t* off_h, int64_t total_h,
                            const T* Gt_t, const T* Gh_t, int f, cudaStream_t st);
template <typename T>
cudaError_t launch_b_poison(const BatchInst<T>* inst, const BatchTile* tiles, int count,
                            int64_t max_elems, int num_sms, cudaStream_t st);
template <typename T>
cudaError_t launch_b_decode(const BatchInst<T>* inst, const BatchPlan* plans, int nplans,
                            const int64_t* off, int64_t total, const double* Gt, const double* Gh,
                            int num_sms, cudaStream_t st);
// Q_1 <- G_0 Q_1 in place for every instance.
template <typename T>
cudaError_t launch_b_post_orth(const BatchInst<T>* inst, int count, const int64_t* off,
                               int64_t total, const T* Gt_t, int num_sms, cudaStream_t st);

}  // namespace cqr
