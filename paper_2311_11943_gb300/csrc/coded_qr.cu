// coded_qr.cu -- C-ABI entry points of the coded-QR library: handle, device workspace,
// state machine, erasure bookkeeping (host-side index sets) and the launch sequence of the
// hot path.  Every arithmetic step runs in the kernels of cqr_kernels.cu / cqr_tc_gemm.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "coded_qr.h"
#include "cqr_kernels.cuh"
#include "cqr_tc_gemm.cuh"

using namespace cqr;

namespace {

enum State { ST_CREATED = 0, ST_ENCODED = 1, ST_FACTORED = 2 };

constexpr int kMaxSplits = 8;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

struct Layout {
  size_t Q, R, Gt, Gh, Gt_t, Gh_t, Kpo, part, bar, status, P, Rb, Pt, yw, xw, plans, cg, tc, total;
};

struct Buffers {
  void* Q;
  void* R;
  double* Gt;
  double* Gh;
  void* Gt_t;
  void* Gh_t;
  void* Kpo;  // (I_f + G~ G~^T)^{-1}: f x f doubles, then f x f in the storage type
  void* part;
  unsigned* bar;
  int* status;
  void* P;
  void* Rb;
  void* Pt;
  void* yw;
  void* xw;
  DecodePlan* plans;
  double* cg;
  void* tc;
};

// Checksum blocks per code.  Out-of-node storage: f (one per tolerated failure, on f extra
// nodes).  In-node storage (Section 5): K = f + f ceil(f / (P - f)) with P = p_r nodes per code
// and L = P data blocks, the equality case of Theorem in_node_opt.
// Sub-panel width of panels too tall for one thread-block cluster (FP32): a 20480-row panel
// of 32 columns takes 1280-row slices on 16 CTAs.
constexpr int kSubPanel = 32;

int code_blocks(const cqr_config* c) {
  if (!c->in_node || c->f == 0) return c->f;
  return c->f + c->f * ((c->f + (c->p_r - c->f) - 1) / (c->p_r - c->f));
}

cqr_status validate(const cqr_config* c) {
  if (!c) return CQR_EINVAL;
  if (c->m < 1 || c->n < 1 || c->m < c->n) return CQR_EINVAL;
  if (c->p_r < 1 || c->p_c < 1 || c->b < 1 || c->f < 0) return CQR_EINVAL;
  if (c->n % c->p_c != 0) return CQR_EINVAL;
  if (c->in_node != 0 && c->in_node != 1) return CQR_EINVAL;
  if (c->in_node && c->f >= c->p_r) return CQR_EINVAL;
  if (c->in_node && c->protect_r && c->p_c != c->p_r) return CQR_ENOTSUP;  // one K for both codes
  const int K = code_blocks(c);
  if (2 * K > c->p_r) return CQR_EINVAL;
  if (c->protect_r && 2 * K > c->p_c) return CQR_EINVAL;
  if (K > kMaxF || c->p_r + K > kMaxCode || c->p_c + K > kMaxCode) return CQR_ENOTSUP;
  if (c->p_r > (int64_t)c->m) return CQR_EINVAL;
  if (c->dtype != CQR_F64 && c->dtype != CQR_F32) return CQR_EINVAL;
  if (c->mma < CQR_MMA_SIMT || c->mma > CQR_MMA_BF16X3) return CQR_EINVAL;
  if (c->dtype == CQR_F64 && c->mma != CQR_MMA_SIMT) return CQR_ENOTSUP;
  if (c->mma != CQR_MMA_SIMT && !tc_available()) return CQR_ENOTSUP;
  if (c->gdist != CQR_G_UNIF01 && c->gdist != CQR_G_NORMAL) return CQR_EINVAL;
  if (c->nrhs_max < 0) return CQR_EINVAL;
  if (c->panel < CQR_PANEL_ICGS || c->panel > CQR_PANEL_CGS2) return CQR_EINVAL;
  if (c->post_orth < CQR_POST_ORTH_AUTO || c->post_orth > CQR_POST_ORTH_PROJECTED) return CQR_EINVAL;
  if (c->reserved != 0) return CQR_EINVAL;
  return CQR_OK;
}

Geo make_geo(const cqr_config* c) {
  Geo g{};
  g.m = c->m;
  g.n = c->n;
  g.p_r = c->p_r;
  g.p_c = c->p_c;
  const int K = code_blocks(c);
  g.f = K;  // checksum blocks of each code (= f out of node)
  g.protect_r = (c->protect_r && K > 0) ? 1 : 0;
  g.mb = (c->m + c->p_r - 1) / c->p_r;
  g.nb = c->n / c->p_c;
  g.m_pad = g.mb * c->p_r;
  g.c = (int64_t)K * g.mb;
  g.d = g.protect_r ? (int64_t)K * g.nb : 0;
  g.M = g.m_pad + g.c;
  g.N = g.n + g.d;
  g.ldq = round_up(g.M, 32);
  g.ldr = round_up(g.N, 32);
  g.grid_rows = c->p_r + K;
  g.grid_cols = c->p_c + (g.protect_r ? K : 0);
  g.b = c->b;
  g.panels = (int)((c->n + c->b - 1) / c->b);
  return g;
}

Layout make_layout(const cqr_config* c, const Geo& g, int num_sms) {
  const size_t s = c->dtype == CQR_F64 ? 8 : 4;
  const int bmax = c->b < g.n ? c->b : (int)g.n;
  const int nrhs = c->nrhs_max > 0 ? c->nrhs_max : 1;
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t at = off; off += align256(bytes ? bytes : 1); return at; };
  L.Q = take((size_t)g.ldq * g.N * s);
  L.R = take((size_t)g.ldr * g.N * s);
  L.Gt = take((size_t)(g.f * c->p_r + 1) * 8);
  L.Gh = take((size_t)(g.f * c->p_c + 1) * 8);
  L.Gt_t = take((size_t)(g.f * c->p_r + 1) * s);
  L.Gh_t = take((size_t)(g.f * c->p_c + 1) * s);
  L.Kpo = take((size_t)kMaxF * kMaxF * (8 + s));
  L.part = take(panel_partial_bytes(bmax, s, num_sms));
  L.bar = take(256);
  L.status = take(256);
  L.P = take((size_t)kMaxSplits * bmax * g.N * s);
  L.Rb = take((size_t)bmax * g.N * s);
  L.Pt = take(c->dtype == CQR_F32 && c->mma != CQR_MMA_SIMT ? tc_panel_bytes(g.M, bmax) : 0);
  L.yw = take((size_t)g.m_pad * nrhs * s);
  L.xw = take((size_t)(g.m + g.N) * nrhs * s);
  L.plans = take(sizeof(DecodePlan) * (size_t)(g.grid_cols + g.p_c + g.f + 2));
  L.cg = take(sizeof(double) * (size_t)(7 * g.n + g.c + 2 * (num_sms + 1)));
  L.tc = take(c->dtype == CQR_F32 && c->mma != CQR_MMA_SIMT
                  ? tc_workspace_bytes(c->mma, g.M, g.N, g.n, bmax, c->reorth_block != 0)
                  : 0);
  L.total = off;
  return L;
}

}  // namespace

// Kernel classes of the per-launch-site profile (coded_qr_profile_read).
enum KClass {
  K_GENERATOR = 0, K_ENCODE, K_PANEL, K_GEMM_RBAR, K_SPLITK_REDUCE, K_GEMM_UPDATE, K_POISON,
  K_DECODE, K_POST_ORTH, K_SOLVE_GEMV, K_TRSV, K_TC_RBAR, K_TC_UPDATE, K_TC_SPLIT,
  K_BLOCK_REORTH, K_TC_NARROW, K_PANEL_SUB_UPDATE, K_COUNT
};
static const char* kClassNames[K_COUNT] = {
    "generator", "encode", "panel_icgs", "gemm_rbar_simt", "splitk_reduce", "gemm_update_simt",
    "erasure_poison", "decode", "post_orth", "solve_gemv", "trsv", "tc_rbar", "tc_update",
    "tc_split_panel", "block_reorth", "tc_narrow_update", "panel_sub_update"};

struct ProfRec {
  int cls;
  cudaEvent_t a, b;
};

struct cqr_handle_s {
  cqr_config cfg;
  Geo g;
  Layout L;
  Buffers B;
  int dev = 0, num_sms = 0;
  bool owns_ws = false;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t st = nullptr;
  DecodePlan* plans_host = nullptr;  // pinned
  int* status_host = nullptr;        // pinned
  cudaEvent_t plans_ev = nullptr;
  std::vector<uint8_t> mask;
  std::vector<int32_t> sets;
  bool pending = false;
  bool postorth_inplace = false;
  int state = ST_CREATED;
  int next_panel = 0;
  int64_t n_recovered = 0, panels_run = 0, n_injected = 0;
  size_t esz = 8;
  double tau = 0.7071067811865476;
  TcGemm* tc = nullptr;
  PanelPlan plan{};
  int plan_bk = -1;
  bool reg_ok = false;
  // sub-panel schedule of panels too tall for one cluster (FP32): width and cluster plan
  int sub_bs = 0;
  PanelPlan sub_plan{};
  int reg_rpl = 0, reg_cpw = 0, reg_G = 0;
  // profile: launch counts always, event-pair device times when enabled
  bool prof_on = false;
  std::vector<ProfRec> prof_recs;
  std::vector<cudaEvent_t> prof_pool;
  double prof_ms[K_COUNT] = {0};
  int64_t prof_launches[K_COUNT] = {0};
  // adjoint scratch (allocated by the first adjoint call)
  void* adj = nullptr;
  size_t adj_bytes = 0;
  // look-ahead of the tensor-core path: the critical stream (highest priority) and the stream
  // of the wide trailing updates (lowest priority), created on first use; events fork, a, w
  cudaStream_t la_st[2] = {nullptr, nullptr};
  cudaEvent_t la_ev[3] = {nullptr, nullptr, nullptr};
  bool la_pdl = false;  // programmatic dependent launch on the critical stream
  long long wait_limit = 0;  // panel exchange / grid-barrier wait bound (0: the default)
};

namespace {

cudaEvent_t prof_event(cqr_handle h) {
  if (!h->prof_pool.empty()) {
    cudaEvent_t e = h->prof_pool.back();
    h->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets the launches of one kernel class at one call site, on the stream they go to.
struct ProfScope {
  cqr_handle h;
  int cls;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  ProfScope(cqr_handle h_, int cls_, int nlaunch, cudaStream_t s = nullptr)
      : h(h_), cls(cls_), st(s ? s : h_->st) {
    h->prof_launches[cls] += nlaunch;
    if (h->prof_on) {
      a = prof_event(h);
      cudaEventRecord(a, st);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = prof_event(h);
      cudaEventRecord(b, st);
      h->prof_recs.push_back(ProfRec{cls, a, b});
    }
  }
};

}  // namespace

// A failed runtime call returns CQR_ECUDA; the runtime's last-error slot is cleared so that a
// later, unrelated launch check does not report it again (sticky errors stay sticky).
#define CK(x)                                          \
  do {                                                 \
    cudaError_t e_ = (x);                              \
    if (e_ != cudaSuccess) {                           \
      cudaGetLastError();                              \
      return CQR_ECUDA;                                \
    }                                                  \
  } while (0)

namespace {

template <typename T>
T* ptr(void* p) { return reinterpret_cast<T*>(p); }

cqr_status setup(cqr_handle h) {
  char* base = reinterpret_cast<char*>(h->ws);
  const Layout& L = h->L;
  h->B.Q = base + L.Q;
  h->B.R = base + L.R;
  h->B.Gt = reinterpret_cast<double*>(base + L.Gt);
  h->B.Gh = reinterpret_cast<double*>(base + L.Gh);
  h->B.Gt_t = base + L.Gt_t;
  h->B.Gh_t = base + L.Gh_t;
  h->B.Kpo = base + L.Kpo;
  h->B.part = base + L.part;
  h->B.bar = reinterpret_cast<unsigned*>(base + L.bar);
  h->B.status = reinterpret_cast<int*>(base + L.status);
  h->B.P = base + L.P;
  h->B.Rb = base + L.Rb;
  h->B.Pt = base + L.Pt;
  h->B.yw = base + L.yw;
  h->B.xw = base + L.xw;
  h->B.plans = reinterpret_cast<DecodePlan*>(base + L.plans);
  h->B.cg = reinterpret_cast<double*>(base + L.cg);
  h->B.tc = base + L.tc;
  h->mask.assign((size_t)h->g.grid_rows * h->g.grid_cols, 0);
  CK(cudaMallocHost(&h->plans_host, sizeof(DecodePlan) * (size_t)(h->g.grid_cols + h->g.p_c + h->g.f + 2)));
  CK(cudaMallocHost(&h->status_host, 4 * sizeof(int)));
  CK(cudaEventCreateWithFlags(&h->plans_ev, cudaEventDisableTiming));
  CK(cudaMemsetAsync(h->B.part, 0, h->L.bar - h->L.part, h->st));
  CK(cudaMemsetAsync(h->B.status, 0, 256, h->st));
  if (h->cfg.dtype == CQR_F32 && h->cfg.mma != CQR_MMA_SIMT) {
    h->tc = tc_create(h->cfg.mma, h->g.M, h->g.N, h->g.n, std::min<int64_t>(h->cfg.b, h->g.n),
                      ptr<float>(h->B.Q), h->g.ldq, h->B.tc, h->num_sms, h->cfg.reorth_block != 0,
                      h->st);
    if (!h->tc) return CQR_ECUDA;
    tc_set_status(h->tc, h->B.status);
  }
  return CQR_OK;
}

cqr_status create_common(const cqr_config* cfg, void* ws, size_t bytes, bool own, cqr_handle* out) {
  if (!out) return CQR_EINVAL;
  *out = nullptr;
  cqr_status v = validate(cfg);
  if (v != CQR_OK) return v;
  cqr_handle h = new (std::nothrow) cqr_handle_s();
  if (!h) return CQR_ENOMEM;
  h->cfg = *cfg;
  if (h->cfg.nrhs_max <= 0) h->cfg.nrhs_max = 1;
  h->g = make_geo(&h->cfg);
  h->esz = cfg->dtype == CQR_F64 ? 8 : 4;
  h->tau = cfg->tau == 0.0 ? 0.7071067811865476 : cfg->tau;
  if (cfg->panel == CQR_PANEL_MGS) h->tau = -1.0;  // the same column loop, no reorthogonalisation
  h->st = reinterpret_cast<cudaStream_t>(cfg->stream);
  if (cudaGetDevice(&h->dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->dev) != cudaSuccess) {
    delete h;
    return CQR_ECUDA;
  }
  h->L = make_layout(&h->cfg, h->g, h->num_sms);
  if (own) {
    if (cudaMalloc(&h->ws, h->L.total) != cudaSuccess) {
      delete h;
      return CQR_ENOMEM;
    }
    h->owns_ws = true;
  } else {
    if (!ws || bytes < h->L.total || (reinterpret_cast<uintptr_t>(ws) & 255)) {
      delete h;
      return ws && bytes < h->L.total ? CQR_ENOMEM : CQR_EINVAL;
    }
    h->ws = ws;
  }
  h->ws_bytes = h->L.total;
  cqr_status s = setup(h);
  if (s != CQR_OK) {
    coded_qr_destroy(h);
    return s;
  }
  *out = h;
  return CQR_OK;
}

// ------------------------------------------------------------------------------- encode
template <typename T>
cqr_status encode_t(cqr_handle h, const T* A, int64_t lda) {
  const Geo& g = h->g;
  CK(cudaMemsetAsync(h->B.status, 0, 4 * sizeof(int), h->st));
  if (g.f > 0) {
    ProfScope ps(h, K_GENERATOR, 1);
    CK(launch_generator<T>(g.f, g.p_r, g.p_c, h->cfg.seed, h->cfg.gdist, h->B.Gt, h->B.Gh,
                           ptr<T>(h->B.Gt_t), ptr<T>(h->B.Gh_t), h->st));
  }
  {
    ProfScope ps(h, K_ENCODE, (g.protect_r && g.f > 0) ? 2 : 1);
    CK(launch_encode<T>(g, A, lda, ptr<T>(h->B.Gt_t), ptr<T>(h->B.Gh_t), ptr<T>(h->B.Q),
                      h->B.status, h->st));
  }
  CK(cudaMemsetAsync(h->B.R, 0, (size_t)g.ldr * g.N * sizeof(T), h->st));
  return CQR_OK;
}

// ------------------------------------------------------------------------------- factor
int choose_splits(int bk, int64_t w, int64_t K, int num_sms) {
  const int64_t tiles = ((bk + 63) / 64) * ((w + 63) / 64);
  int s = (int)((2 * num_sms + tiles - 1) / tiles);
  if (s > kMaxSplits) s = kMaxSplits;
  if (s < 1) s = 1;
  while (s > 1 && K / s < 256) --s;
  return s;
}

template <typename T>
void ensure_panel_plan(cqr_handle h, int bk) {
  if (bk == h->plan_bk) return;
  const Geo& g = h->g;
  h->plan = plan_panel(g.M, bk, sizeof(T), h->num_sms, true);
  if (h->plan.cluster && !panel_cluster_fits<T>(h->plan))
    h->plan = plan_panel(g.M, bk, sizeof(T), h->num_sms, false);
  // two-level plans: clusters of 16, else of 8, else the flat grid, whichever can have all
  // its clusters resident at once
  if (h->plan.hier && !panel_hier_fits<T>(h->plan))
    h->plan = plan_panel(g.M, bk, sizeof(T), h->num_sms, h->plan.cluster != 0, true, 8);
  if (h->plan.hier && !panel_hier_fits<T>(h->plan))
    h->plan = plan_panel(g.M, bk, sizeof(T), h->num_sms, h->plan.cluster != 0, false);
  h->reg_ok = false;
  const char* env = getenv("CQR_PANEL_REG");
  const bool left_looking = h->cfg.panel == CQR_PANEL_CGS1 || h->cfg.panel == CQR_PANEL_CGS2;
  if (sizeof(T) == 4 && !(env && env[0] == '0') && !left_looking &&
      plan_panel_reg(g.M, bk, &h->reg_rpl, &h->reg_cpw, &h->reg_G))
    h->reg_ok = panel_reg_cluster_fits(h->reg_rpl, h->reg_cpw, h->reg_G);
  // on request (CQR_PANEL_SUB=1), an FP32 panel too tall for one cluster is factored as
  // sub-panels of kSubPanel columns that each fit one cluster (measured slower than the
  // two-level exchange at 20480 x 256: its in-panel updates are skinny CUDA-core products)
  h->sub_bs = 0;
  const char* se = getenv("CQR_PANEL_SUB");
  if (sizeof(T) == 4 && !h->reg_ok && !h->plan.cluster && !left_looking && bk > kSubPanel &&
      se && se[0] == '1') {
    const PanelPlan sp = plan_panel(g.M, kSubPanel, sizeof(T), h->num_sms, true, false);
    if (sp.cluster && panel_cluster_fits<T>(sp)) {
      h->sub_bs = kSubPanel;
      h->sub_plan = sp;
    }
  }
  h->plan_bk = bk;
}

// The panel of columns kb .. kb+bk-1 as sub-panels of sub_bs columns (the blocked schedule of
// the same Gram-Schmidt: reading "sub-panels" of the design notes).  Each sub-panel runs the
// panel kernel (ICGS, the criterion within the sub-panel) on one thread-block cluster; the
// panel's columns to its right are then projected once on it, R[sub rows, right] = Qs^T P and
// P -= Qs R, by the split-K CUDA-core kernels in the storage precision.
template <typename T>
cqr_status sub_panel_step(cqr_handle h, int64_t kb, int bk, cudaStream_t st) {
  const Geo& g = h->g;
  T* Q = ptr<T>(h->B.Q);
  T* R = ptr<T>(h->B.R);
  const int bs = h->sub_bs;
  for (int s0 = 0; s0 < bk; s0 += bs) {
    const int w0 = std::min(bs, bk - s0);
    const int64_t ks = kb + s0;
    {
      ProfScope ps(h, K_PANEL, 1, st);
      CK(launch_panel<T>(h->sub_plan, Q + ks * g.ldq, g.ldq, R + ks + ks * g.ldr, g.ldr, g.M, w0,
                         h->tau, ptr<T>(h->B.part), h->B.bar, h->B.status, (int)ks, st, 0,
                         h->wait_limit));
    }
    const int64_t j0 = ks + w0;
    const int64_t w = kb + bk - j0;
    if (w <= 0) break;
    ProfScope ps(h, K_PANEL_SUB_UPDATE, 3, st);
    const int splits = choose_splits(w0, w, g.M, h->num_sms);
    CK(launch_gemm_tn_splitk<T>(Q + ks * g.ldq, g.ldq, Q + j0 * g.ldq, g.ldq, g.M, w0, w, splits,
                                ptr<T>(h->B.P), st));
    CK(launch_splitk_reduce<T>(ptr<T>(h->B.P), splits, w0, w, R + ks + j0 * g.ldr, g.ldr,
                               ptr<T>(h->B.Rb), st));
    CK(launch_gemm_nn_sub<T>(Q + ks * g.ldq, g.ldq, ptr<T>(h->B.Rb), w0, Q + j0 * g.ldq, g.ldq,
                             g.M, w0, w, st));
  }
  return CQR_OK;
}

// Block reorthogonalisation of panel columns kb .. kb+bk-1 against columns 0 .. kb-1:
// S = Q[:, :kb]^T Qbar, Qbar -= Q[:, :kb] S, R[:kb, panel] += S.
template <typename T>
cqr_status reorth_block_step(cqr_handle h, int64_t kb, int bk, int buf, cudaStream_t st) {
  if (!h->cfg.reorth_block || kb <= 0) return CQR_OK;
  const Geo& g = h->g;
  T* Q = ptr<T>(h->B.Q);
  T* R = ptr<T>(h->B.R);
  if (h->tc) {
    ProfScope ps(h, K_BLOCK_REORTH, 0, st);
    int nl = 0;
    const cudaError_t e = tc_block_reorth(h->tc, kb, bk, ptr<float>(h->B.R), g.ldr, buf, st, &nl);
    h->prof_launches[K_BLOCK_REORTH] += nl;
    CK(e);
    return CQR_OK;
  }
  ProfScope ps(h, K_BLOCK_REORTH, 3, st);
  const int sp = choose_splits((int)kb, bk, g.M, h->num_sms);
  CK(launch_gemm_tn_splitk<T>(Q, g.ldq, Q + kb * g.ldq, g.ldq, g.M, (int)kb, bk, sp,
                              ptr<T>(h->B.P), st));
  CK(launch_splitk_reduce<T>(ptr<T>(h->B.P), sp, (int)kb, bk, R + kb * g.ldr, g.ldr,
                             ptr<T>(h->B.Rb), st, 1));
  CK(launch_gemm_nn_sub<T>(Q, g.ldq, ptr<T>(h->B.Rb), kb, Q + kb * g.ldq, g.ldq, g.M, (int)kb,
                           bk, st));
  return CQR_OK;
}

// The panel factorisation (ICGS, or the chosen variant) of columns kb .. kb+bk-1.
template <typename T>
cqr_status panel_kernel_step(cqr_handle h, int64_t kb, int bk, cudaStream_t st) {
  const Geo& g = h->g;
  T* Q = ptr<T>(h->B.Q);
  T* R = ptr<T>(h->B.R);
  ensure_panel_plan<T>(h, bk);
  if (h->sub_bs > 0) return sub_panel_step<T>(h, kb, bk, st);
  ProfScope ps(h, K_PANEL, 1, st);
  if (sizeof(T) == 4 && h->reg_ok) {
    CK(launch_panel_reg(h->reg_rpl, h->reg_cpw, h->reg_G, reinterpret_cast<float*>(Q + kb * g.ldq),
                        g.ldq, reinterpret_cast<float*>(R + kb + kb * g.ldr), g.ldr, g.M, bk, h->tau,
                        h->B.status, (int)kb, st, h->la_pdl && st == h->la_st[0], h->wait_limit));
  } else {
    const int variant = h->cfg.panel == CQR_PANEL_CGS1 ? 1 : (h->cfg.panel == CQR_PANEL_CGS2 ? 2 : 0);
    CK(launch_panel<T>(h->plan, Q + kb * g.ldq, g.ldq, R + kb + kb * g.ldr, g.ldr, g.M, bk, h->tau,
                       ptr<T>(h->B.part), h->B.bar, h->B.status, (int)kb, st, variant,
                       h->wait_limit));
  }
  return CQR_OK;
}

// Tensor-core trailing update of columns j0 .. j0+w-1 by the panel kb .. kb+bk-1 (its operand
// planes in buffer buf), partials and Rbar planes of context ctx, at most max_ctas CTAs.
cqr_status tc_update_cols(cqr_handle h, int64_t kb, int bk, int64_t j0, int64_t w, int buf, int ctx,
                          int max_ctas, cudaStream_t st) {
  if (w <= 0) return CQR_OK;
  {
    ProfScope ps(h, K_TC_RBAR, 1, st);
    CK(tc_gemm_rbar(h->tc, bk, j0, w, buf, ctx, max_ctas, st));
  }
  {
    ProfScope ps(h, K_SPLITK_REDUCE, 1, st);
    CK(tc_reduce(h->tc, kb, bk, j0, w, ptr<float>(h->B.R), h->g.ldr, ctx, max_ctas, st));
  }
  {
    ProfScope ps(h, K_TC_UPDATE, 1, st);
    CK(tc_gemm_update(h->tc, bk, j0, w, buf, ctx, max_ctas, st));
  }
  return CQR_OK;
}

// One panel in stream order: block reorthogonalisation, panel, trailing update of every
// column to the right.
template <typename T>
cqr_status panel_step(cqr_handle h, int t) {
  const Geo& g = h->g;
  const int64_t kb = (int64_t)t * g.b;
  const int bk = (int)std::min<int64_t>(g.b, g.n - kb);
  T* Q = ptr<T>(h->B.Q);
  T* R = ptr<T>(h->B.R);
  const int buf = t & 1;
  cqr_status s = reorth_block_step<T>(h, kb, bk, buf, h->st);
  if (s != CQR_OK) return s;
  s = panel_kernel_step<T>(h, kb, bk, h->st);
  if (s != CQR_OK) return s;
  const int64_t j0 = kb + bk;
  if (j0 >= g.N) return CQR_OK;
  const int64_t w = g.N - j0;
  if (h->tc) {
    {
      ProfScope ps(h, K_TC_SPLIT, 1);
      CK(tc_split_panel(h->tc, kb, bk, true, buf, h->st));
    }
    return tc_update_cols(h, kb, bk, j0, w, buf, 0, 0, h->st);
  }
  const int splits = choose_splits(bk, w, g.M, h->num_sms);
  {
    ProfScope ps(h, K_GEMM_RBAR, 1);
    CK(launch_gemm_tn_splitk<T>(Q + kb * g.ldq, g.ldq, Q + j0 * g.ldq, g.ldq, g.M, bk, w, splits,
                                ptr<T>(h->B.P), h->st));
  }
  {
    ProfScope ps(h, K_SPLITK_REDUCE, 1);
    CK(launch_splitk_reduce<T>(ptr<T>(h->B.P), splits, bk, w, R + kb + j0 * g.ldr, g.ldr,
                               ptr<T>(h->B.Rb), h->st));
  }
  {
    ProfScope ps(h, K_GEMM_UPDATE, 1);
    CK(launch_gemm_nn_sub<T>(Q + kb * g.ldq, g.ldq, ptr<T>(h->B.Rb), bk, Q + j0 * g.ldq, g.ldq,
                             g.M, bk, w, h->st));
  }
  return CQR_OK;
}

// Look-ahead (tensor-core path, panel on one thread-block cluster): the trailing update of
// panel t is split into the next panel's columns (narrow, on the critical stream A) and the
// rest (wide, on stream B, at most num_sms - panel CTAs CTAs), so that the wide update runs
// while panel t+1 is factorised.  Per panel t on A: block reorthogonalisation of panel t;
// event a (B waits on it, then issues the wide update of panel t-1 and records event w); the
// panel; the operand split (buffer t mod 2); A waits on w (the wide update of panel t-1 wrote
// panel t+1's columns); the narrow update.  Both streams fork from and join into the
// handle's stream, so the result of the call is stream-ordered like the sequential form.
// The arithmetic of every panel (the column ranges of its two updates, their split-K
// factors) does not depend on where factor calls start and end.
bool lookahead_eligible(cqr_handle h) {
  if (!h->tc) return false;
  const char* env = getenv("CQR_LOOKAHEAD");
  if (env && env[0] == '0') return false;
  ensure_panel_plan<float>(h, (int)std::min<int64_t>(h->g.b, h->g.n));
  // a cooperative (grid-barrier) panel must not wait for CTAs of a concurrent GEMM
  return h->reg_ok || h->plan.cluster;
}

cqr_status lookahead_setup(cqr_handle h) {
  if (h->la_st[0]) return CQR_OK;
  int least = 0, greatest = 0;
  CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  CK(cudaStreamCreateWithPriority(&h->la_st[0], cudaStreamNonBlocking, greatest));
  CK(cudaStreamCreateWithPriority(&h->la_st[1], cudaStreamNonBlocking, least));
  for (auto& e : h->la_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return CQR_OK;
}

cqr_status factor_lookahead(cqr_handle h, int t0, int t1) {
  cqr_status s = lookahead_setup(h);
  if (s != CQR_OK) return s;
  const Geo& g = h->g;
  cudaStream_t A = h->la_st[0], Bst = h->la_st[1];
  // programmatic dependent launch along the critical stream (CQR_PDL=0 turns it off)
  const char* pe = getenv("CQR_PDL");
  h->la_pdl = !(pe && pe[0] == '0');
  tc_set_pdl_stream(h->tc, h->la_pdl ? A : nullptr);
  cudaEvent_t ev_fork = h->la_ev[0], ev_a = h->la_ev[1], ev_w = h->la_ev[2];
  CK(cudaEventRecord(ev_fork, h->st));
  CK(cudaStreamWaitEvent(A, ev_fork, 0));  // B joins through A's events (only if it gets work)
  // the wide update waiting to be issued: panel (kb, bk), columns j0 .. j0+w-1, buffer
  struct Wide { int64_t kb, j0, w; int bk, buf; } wide{0, 0, 0, 0, 0};
  bool wide_due = false, w_pending = false;
  auto issue_wide = [&]() -> cqr_status {
    CK(cudaEventRecord(ev_a, A));
    CK(cudaStreamWaitEvent(Bst, ev_a, 0));
    const int pc = h->reg_ok ? h->reg_G : h->plan.G;
    cqr_status r = tc_update_cols(h, wide.kb, wide.bk, wide.j0, wide.w, wide.buf, 1,
                                  std::max(1, h->num_sms - pc), Bst);
    if (r != CQR_OK) return r;
    CK(cudaEventRecord(ev_w, Bst));
    wide_due = false;
    w_pending = true;
    return CQR_OK;
  };
  for (int t = t0; t < t1; ++t) {
    const int64_t kb = (int64_t)t * g.b;
    const int bk = (int)std::min<int64_t>(g.b, g.n - kb);
    const int buf = t & 1;
    s = reorth_block_step<float>(h, kb, bk, buf, A);
    if (s != CQR_OK) return s;
    if (wide_due && (s = issue_wide()) != CQR_OK) return s;
    s = panel_kernel_step<float>(h, kb, bk, A);
    if (s != CQR_OK) return s;
    const int64_t j0 = kb + bk;
    if (j0 >= g.N) continue;
    {
      ProfScope ps(h, K_TC_SPLIT, 1, A);
      CK(tc_split_panel(h->tc, kb, bk, true, buf, A));
    }
    const int64_t wn = j0 < g.n ? std::min<int64_t>(g.b, g.n - j0) : g.N - j0;
    if (w_pending) {
      CK(cudaStreamWaitEvent(A, ev_w, 0));
      w_pending = false;
    }
    {
      // the look-ahead's narrow update as a whole (its three launches are also counted in
      // their own classes)
      ProfScope ps(h, K_TC_NARROW, 0, A);
      s = tc_update_cols(h, kb, bk, j0, wn, buf, 0, 0, A);
    }
    if (s != CQR_OK) return s;
    if (j0 + wn < g.N) {
      wide = Wide{kb, j0 + wn, g.N - j0 - wn, bk, buf};
      wide_due = true;
    }
  }
  if (wide_due && (s = issue_wide()) != CQR_OK) return s;
  if (w_pending) CK(cudaStreamWaitEvent(A, ev_w, 0));
  CK(cudaEventRecord(ev_a, A));
  CK(cudaStreamWaitEvent(h->st, ev_a, 0));
  return CQR_OK;
}

// ------------------------------------------------------------------------------- recover
// Decode plan of one code (reading of the recovery Lemma: the f1 lowest-index surviving
// checksum rows are used).  Returns false when f1 + f2 > f.
bool make_plan(int nsys, int f, const uint8_t* lost_sys, const uint8_t* lost_chk, DecodePlan* p) {
  p->f1 = p->f2 = 0;
  p->nsys = nsys;
  for (int t = 0; t < nsys; ++t)
    if (lost_sys[t]) p->A_fail[p->f1++] = t;
  for (int i = 0; i < f; ++i)
    if (lost_chk[i]) p->C_fail[p->f2++] = i;
  if (p->f1 + p->f2 > f) return false;
  int u = 0;
  for (int i = 0; i < f && u < p->f1; ++i)
    if (!lost_chk[i]) p->C_use[u++] = i;
  return u == p->f1;
}

template <typename T>
cqr_status recover_t(cqr_handle h, int32_t* n_recovered) {
  const Geo& g = h->g;
  const int gc = g.grid_cols, f = g.f;
  std::vector<DecodePlan> plans;
  std::vector<uint8_t> ls(kMaxCode), lc(kMaxCode);
  int nrec = 0;
  for (int j = 0; j < gc; ++j) {
    DecodePlan p{};
    p.kind = 0;
    p.idx = j;
    for (int t = 0; t < g.p_r; ++t) ls[t] = h->mask[(size_t)t * gc + j];
    for (int i = 0; i < f; ++i) lc[i] = h->mask[(size_t)(g.p_r + i) * gc + j];
    if (!make_plan(g.p_r, f, ls.data(), lc.data(), &p)) return CQR_EUNRECOVERABLE;
    if (p.f1 + p.f2 == 0) continue;
    nrec += p.f1 + p.f2;
    plans.push_back(p);
  }
  size_t nq = plans.size();
  if (g.protect_r) {
    for (int i = 0; i < g.p_c + f && i < g.grid_rows; ++i) {
      DecodePlan p{};
      p.kind = 1;
      p.idx = i;
      for (int j = 0; j < g.p_c; ++j) ls[j] = h->mask[(size_t)i * gc + j];
      for (int l = 0; l < f; ++l) lc[l] = h->mask[(size_t)i * gc + g.p_c + l];
      if (!make_plan(g.p_c, f, ls.data(), lc.data(), &p)) return CQR_EUNRECOVERABLE;
      if (p.f1 + p.f2 == 0) continue;
      plans.push_back(p);
    }
  }
  if (!plans.empty()) {
    CK(cudaEventSynchronize(h->plans_ev));
    memcpy(h->plans_host, plans.data(), sizeof(DecodePlan) * plans.size());
    CK(cudaMemcpyAsync(h->B.plans, h->plans_host, sizeof(DecodePlan) * plans.size(),
                       cudaMemcpyHostToDevice, h->st));
    CK(cudaEventRecord(h->plans_ev, h->st));
    const int max_h = (int)std::max(g.mb, g.nb);
    ProfScope ps(h, K_DECODE, 1);
    CK(launch_decode<T>(g, h->B.plans, (int)plans.size(), max_h, h->B.Gt, h->B.Gh,
                        ptr<T>(h->B.Q), ptr<T>(h->B.R), h->B.status, h->st));
  }
  for (size_t k = 0; k < plans.size(); ++k) {
    const DecodePlan& p = plans[k];
    h->sets.push_back(p.kind);
    h->sets.push_back(p.idx);
    h->sets.push_back(p.f1);
    h->sets.push_back(p.f2);
    for (int a = 0; a < p.f1; ++a) h->sets.push_back(p.A_fail[a]);
    for (int e = 0; e < p.f2; ++e) h->sets.push_back(p.C_fail[e]);
    for (int a = 0; a < p.f1; ++a) h->sets.push_back(p.C_use[a]);
  }
  (void)nq;
  if (h->tc && tc_has_block_reorth(h->tc) && !plans.empty()) {
    // the row-major copy of the computed columns is part of the nodes' state: rebuild the
    // recovered Q tiles of it (tile (i, j) holds rows i mb .., columns j nb ..)
    const int64_t ncols = std::min<int64_t>((int64_t)h->next_panel * g.b, g.n);
    for (int i = 0; i < g.grid_rows; ++i)
      for (int j = 0; j < g.grid_cols; ++j) {
        if (!h->mask[(size_t)i * g.grid_cols + j]) continue;
        const int64_t c0 = (int64_t)j * g.nb;
        if (c0 >= ncols) continue;
        CK(tc_refresh_rect(h->tc, (int64_t)i * g.mb, g.mb, c0, std::min<int64_t>(g.nb, ncols - c0), h->st));
      }
  }
  std::fill(h->mask.begin(), h->mask.end(), 0);
  h->pending = false;
  h->n_recovered += nrec;
  if (n_recovered) *n_recovered = nrec;
  return CQR_OK;
}

// ------------------------------------------------------------------------------- post-orth
template <typename T>
cqr_status copy_pad(cqr_handle h, const T* src, int64_t lds, int64_t rows, int64_t rows_pad,
                    int64_t cols, T* dst, int64_t ldd) {
  if (rows_pad > rows) CK(cudaMemset2DAsync(dst + rows, ldd * sizeof(T), 0, (rows_pad - rows) * sizeof(T), cols, h->st));
  if (dst != src)
    CK(cudaMemcpy2DAsync(dst, ldd * sizeof(T), src, lds * sizeof(T), rows * sizeof(T), cols,
                         cudaMemcpyDeviceToDevice, h->st));
  return CQR_OK;
}

template <typename T>
cqr_status post_orth_q(cqr_handle h, T* Qout, int64_t ldqo) {
  const Geo& g = h->g;
  T* Q = ptr<T>(h->B.Q);
  T* dst = Qout ? Qout : Q;
  const int64_t ldd = Qout ? ldqo : g.ldq;
  if (h->postorth_inplace) {  // Q_1 already transformed
    if (Qout) return copy_pad<T>(h, Q, g.ldq, g.m_pad, g.m_pad, g.n, Qout, ldqo);
    return CQR_OK;
  }
  const bool projected = h->cfg.post_orth == CQR_POST_ORTH_PROJECTED ||
                         (h->cfg.post_orth == CQR_POST_ORTH_AUTO && h->esz == 4);
  if (g.f == 0) {
    if (Qout) return copy_pad<T>(h, Q, g.ldq, g.m_pad, g.m_pad, g.n, Qout, ldqo);
  } else if (projected) {
    ProfScope ps(h, K_POST_ORTH, 2);
    double* K64 = reinterpret_cast<double*>(h->B.Kpo);
    T* Kt = reinterpret_cast<T*>(K64 + kMaxF * kMaxF);
    CK(launch_post_orth_projected<T>(g, h->B.Gt, ptr<T>(h->B.Gt_t), K64, Kt, Q, g.ldq, g.n, dst,
                                     ldd, h->st));
  } else {
    ProfScope ps(h, K_POST_ORTH, 1);
    CK(launch_post_orth<T>(g, ptr<T>(h->B.Gt_t), Q, g.ldq, g.m_pad, g.n, dst, ldd, h->st));
  }
  if (!Qout) h->postorth_inplace = true;
  return CQR_OK;
}

template <typename T>
cqr_status post_orth_y(cqr_handle h, const T* y, int64_t ldy, int32_t nrhs, T* yo, int64_t ldyo) {
  const Geo& g = h->g;
  if (g.f == 0) return copy_pad<T>(h, y, ldy, g.m, g.m_pad, nrhs, yo, ldyo);
  ProfScope ps(h, K_POST_ORTH, 1);
  CK(launch_post_orth<T>(g, ptr<T>(h->B.Gt_t), y, ldy, g.m, nrhs, yo, ldyo, h->st));
  return CQR_OK;
}

// ------------------------------------------------------------------------------- solve
template <typename T>
cqr_status solve_t(cqr_handle h, const T* y, int64_t ldy, T* x, int64_t ldx, int32_t nrhs) {
  const Geo& g = h->g;
  const bool square = (g.m == g.n && g.m_pad == g.m);
  if (!square) {
    // least squares through A = Q_1 R: CG in FP64 on (I - Q_2^T Q_2) w = Q_1^T y, then R x = w
    if (h->postorth_inplace) return CQR_ESTATE;  // Q_1 was overwritten by G_0 Q_1
    for (int32_t k = 0; k < nrhs; ++k) {
      {
        ProfScope ps(h, K_SOLVE_GEMV, 1);
        CK(launch_ls_cg<T>(ptr<T>(h->B.Q), g.ldq, g.m, g.m_pad, g.c, g.n, y + (int64_t)k * ldy,
                           x + (int64_t)k * ldx, h->B.cg, h->B.bar, h->B.status, h->num_sms, h->st));
      }
    }
    ProfScope ps(h, K_TRSV, nrhs);
    CK(launch_trsv_upper<T>(ptr<T>(h->B.R), g.ldr, g.n, x, ldx, nrhs, h->st));
    return CQR_OK;
  }
  cqr_status s = post_orth_q<T>(h, nullptr, 0);
  if (s != CQR_OK) return s;
  T* yo = ptr<T>(h->B.yw);
  s = post_orth_y<T>(h, y, ldy, nrhs, yo, g.m_pad);
  if (s != CQR_OK) return s;
  {
    ProfScope ps(h, K_SOLVE_GEMV, 1);
    CK(launch_gemv_t<T>(ptr<T>(h->B.Q), g.ldq, g.m_pad, g.n, yo, g.m_pad, nrhs, x, ldx, h->st));
  }
  {
    ProfScope ps(h, K_TRSV, 1);
    CK(launch_trsv_upper<T>(ptr<T>(h->B.R), g.ldr, g.n, x, ldx, nrhs, h->st));
  }
  return CQR_OK;
}

cqr_status read_status(cqr_handle h, bool clear) {
  CK(cudaMemcpyAsync(h->status_host, h->B.status, 4 * sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  const int code = h->status_host[0];
  if (clear && code != 0) CK(cudaMemsetAsync(h->B.status, 0, sizeof(int), h->st));
  return (cqr_status)code;
}

}  // namespace

// =================================================================== exported entry points
extern "C" {

cqr_status coded_qr_workspace_size(const cqr_config* cfg, size_t* bytes) {
  if (!bytes) return CQR_EINVAL;
  cqr_status v = validate(cfg);
  if (v != CQR_OK) return v;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CQR_ECUDA;
  cqr_config c = *cfg;
  if (c.nrhs_max <= 0) c.nrhs_max = 1;
  Geo g = make_geo(&c);
  *bytes = make_layout(&c, g, sms).total;
  return CQR_OK;
}

cqr_status coded_qr_create(const cqr_config* cfg, cqr_handle* out) {
  return create_common(cfg, nullptr, 0, true, out);
}

cqr_status coded_qr_create_in(const cqr_config* cfg, void* workspace, size_t bytes,
                              cqr_handle* out) {
  return create_common(cfg, workspace, bytes, false, out);
}

cqr_status coded_qr_destroy(cqr_handle h) {
  if (!h) return CQR_OK;
  if (h->st || true) cudaStreamSynchronize(h->st);
  if (h->tc) tc_destroy(h->tc);
  for (auto e : h->la_ev)
    if (e) cudaEventDestroy(e);
  for (auto q : h->la_st)
    if (q) cudaStreamDestroy(q);
  for (auto& r : h->prof_recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : h->prof_pool) cudaEventDestroy(e);
  if (h->plans_ev) cudaEventDestroy(h->plans_ev);
  if (h->plans_host) cudaFreeHost(h->plans_host);
  if (h->status_host) cudaFreeHost(h->status_host);
  if (h->owns_ws && h->ws) cudaFree(h->ws);
  if (h->adj) cudaFree(h->adj);
  delete h;
  return CQR_OK;
}

cqr_status coded_qr_geometry(cqr_handle h, int64_t* d) {
  if (!h || !d) return CQR_EINVAL;
  const Geo& g = h->g;
  d[CQR_GEO_M] = g.m;
  d[CQR_GEO_N] = g.n;
  d[CQR_GEO_MB] = g.mb;
  d[CQR_GEO_NB] = g.nb;
  d[CQR_GEO_MPAD] = g.m_pad;
  d[CQR_GEO_C] = g.c;
  d[CQR_GEO_D] = g.d;
  d[CQR_GEO_MROWS] = g.M;
  d[CQR_GEO_NCOLS] = g.N;
  d[CQR_GEO_LDQ] = g.ldq;
  d[CQR_GEO_LDR] = g.ldr;
  d[CQR_GEO_GRID_ROWS] = g.grid_rows;
  d[CQR_GEO_GRID_COLS] = g.grid_cols;
  d[CQR_GEO_PANELS] = g.panels;
  d[CQR_GEO_CODE_BLOCKS] = g.f;
  return CQR_OK;
}

cqr_status coded_qr_encode(cqr_handle h, const void* A, int64_t lda) {
  if (!h || !A || lda < h->g.m) return CQR_EINVAL;
  cqr_status s = h->esz == 8 ? encode_t<double>(h, (const double*)A, lda)
                             : encode_t<float>(h, (const float*)A, lda);
  if (s != CQR_OK) return s;
  std::fill(h->mask.begin(), h->mask.end(), 0);
  h->sets.clear();
  h->pending = false;
  h->postorth_inplace = false;
  h->next_panel = 0;
  h->n_recovered = h->panels_run = h->n_injected = 0;
  h->state = ST_ENCODED;
  return CQR_OK;
}

cqr_status coded_qr_factor(cqr_handle h, int32_t t0, int32_t t1) {
  if (!h) return CQR_EINVAL;
  if (h->state == ST_CREATED || h->pending || h->postorth_inplace) return CQR_ESTATE;
  if (t1 < 0) t1 = h->g.panels;
  if (t0 != h->next_panel || t1 < t0 || t1 > h->g.panels) return CQR_ESTATE;
  if (t1 > t0 && h->esz == 4 && lookahead_eligible(h)) {
    cqr_status s = factor_lookahead(h, t0, t1);
    if (s != CQR_OK) return s;
    h->panels_run += t1 - t0;
  } else {
    for (int t = t0; t < t1; ++t) {
      cqr_status s = h->esz == 8 ? panel_step<double>(h, t) : panel_step<float>(h, t);
      if (s != CQR_OK) return s;
      ++h->panels_run;
    }
  }
  h->next_panel = t1;
  h->state = (t1 == h->g.panels) ? ST_FACTORED : ST_ENCODED;
  return CQR_OK;
}

cqr_status coded_qr_inject_erasure(cqr_handle h, const int32_t* tiles, int32_t count) {
  if (!h || count < 0 || (count > 0 && !tiles)) return CQR_EINVAL;
  if (h->state == ST_CREATED || h->postorth_inplace) return CQR_ESTATE;
  const Geo& g = h->g;
  for (int e = 0; e < count; ++e) {
    const int i = tiles[2 * e], j = tiles[2 * e + 1];
    if (i < 0 || i >= g.grid_rows || j < 0 || j >= g.grid_cols) return CQR_EINVAL;
  }
  if (count == 0) return CQR_OK;
  for (int e = 0; e < count; ++e) h->mask[(size_t)tiles[2 * e] * g.grid_cols + tiles[2 * e + 1]] = 1;
  int nr_tiles = 0;
  for (int e = 0; e < count; ++e) nr_tiles += (g.protect_r && tiles[2 * e] < g.p_c + g.f) ? 1 : 0;
  ProfScope ps(h, K_POISON, (count + 63) / 64 + (nr_tiles + 63) / 64);
  cudaError_t err = h->esz == 8
      ? launch_poison<double>(g, tiles, count, ptr<double>(h->B.Q), ptr<double>(h->B.R), h->st)
      : launch_poison<float>(g, tiles, count, ptr<float>(h->B.Q), ptr<float>(h->B.R), h->st);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return CQR_ECUDA;
  }
  h->pending = true;
  h->n_injected += count;
  return CQR_OK;
}

namespace {

// Checksum block k of a code of K blocks over P nodes goes to node (k P) / K when K <= P,
// else to node k mod P: the load-balanced in-node distribution (Definition innode_distr).
int in_node_host(int k, int K, int P) { return K <= P ? (int)((int64_t)k * P / K) : k % P; }

// Tiles of the encoded grid lost when node (i, j) fails (as (row, col) pairs).  In-node:
// the node's data tile and every checksum tile it hosts (vertical checksums of column j hosted
// by row node i, horizontal checksums of row i hosted by column node j, and their corner
// tiles).  Out of node: node (i, j) of the extended grid holds tile (i, j).
void node_tiles(const cqr_handle h, int i, int j, std::vector<int32_t>* out) {
  const Geo& g = h->g;
  if (!h->cfg.in_node) {
    out->push_back(i);
    out->push_back(j);
    return;
  }
  std::vector<int> rows{i}, cols{j};
  for (int k = 0; k < g.f; ++k)
    if (in_node_host(k, g.f, g.p_r) == i) rows.push_back(g.p_r + k);
  if (g.protect_r)
    for (int l = 0; l < g.f; ++l)
      if (in_node_host(l, g.f, g.p_c) == j) cols.push_back(g.p_c + l);
  for (int I : rows)
    for (int J : cols) {
      out->push_back(I);
      out->push_back(J);
    }
}

bool node_in_range(const cqr_handle h, int i, int j) {
  const Geo& g = h->g;
  if (h->cfg.in_node) return i >= 0 && i < g.p_r && j >= 0 && j < g.p_c;
  return i >= 0 && i < g.grid_rows && j >= 0 && j < g.grid_cols;
}

}  // namespace

cqr_status coded_qr_inject_node_failure(cqr_handle h, const int32_t* nodes, int32_t count) {
  if (!h || count < 0 || (count > 0 && !nodes)) return CQR_EINVAL;
  for (int e = 0; e < count; ++e)
    if (!node_in_range(h, nodes[2 * e], nodes[2 * e + 1])) return CQR_EINVAL;
  std::vector<int32_t> tiles;
  for (int e = 0; e < count; ++e) node_tiles(h, nodes[2 * e], nodes[2 * e + 1], &tiles);
  return coded_qr_inject_erasure(h, tiles.data(), (int32_t)(tiles.size() / 2));
}

cqr_status coded_qr_recover(cqr_handle h, int32_t* n_recovered) {
  if (!h) return CQR_EINVAL;
  if (h->state == ST_CREATED) return CQR_ESTATE;
  if (n_recovered) *n_recovered = 0;
  if (!h->pending) return CQR_OK;
  if (h->g.f == 0) return CQR_EUNRECOVERABLE;
  return h->esz == 8 ? recover_t<double>(h, n_recovered) : recover_t<float>(h, n_recovered);
}

cqr_status coded_qr_post_orth(cqr_handle h, void* Q, int64_t ldq, const void* y, int64_t ldy,
                              void* yo, int64_t ldyo, int32_t nrhs) {
  if (!h) return CQR_EINVAL;
  if (h->state != ST_FACTORED || h->pending) return CQR_ESTATE;
  if (Q && ldq < h->g.m_pad) return CQR_EINVAL;
  if (y && (nrhs < 1 || ldy < h->g.m)) return CQR_EINVAL;
  if (y && !yo && nrhs > h->cfg.nrhs_max) return CQR_EINVAL;
  if (y && yo && ldyo < h->g.m_pad) return CQR_EINVAL;
  cqr_status s;
  if (h->esz == 8) {
    s = post_orth_q<double>(h, (double*)Q, ldq);
    if (s == CQR_OK && y)
      s = post_orth_y<double>(h, (const double*)y, ldy, nrhs, yo ? (double*)yo : ptr<double>(h->B.yw),
                              yo ? ldyo : h->g.m_pad);
  } else {
    s = post_orth_q<float>(h, (float*)Q, ldq);
    if (s == CQR_OK && y)
      s = post_orth_y<float>(h, (const float*)y, ldy, nrhs, yo ? (float*)yo : ptr<float>(h->B.yw),
                             yo ? ldyo : h->g.m_pad);
  }
  return s;
}

cqr_status coded_qr_solve(cqr_handle h, const void* y, int64_t ldy, void* x, int64_t ldx,
                          int32_t nrhs) {
  if (!h || !y || !x) return CQR_EINVAL;
  if (h->state != ST_FACTORED || h->pending) return CQR_ESTATE;
  if (nrhs < 1 || nrhs > h->cfg.nrhs_max || ldy < h->g.m || ldx < h->g.n) return CQR_EINVAL;
  return h->esz == 8 ? solve_t<double>(h, (const double*)y, ldy, (double*)x, ldx, nrhs)
                     : solve_t<float>(h, (const float*)y, ldy, (float*)x, ldx, nrhs);
}

cqr_status coded_qr_solve_ls(cqr_handle h, const void* y, int64_t ldy, void* x, int64_t ldx,
                             int32_t nrhs) {
  return coded_qr_solve(h, y, ldy, x, ldx, nrhs);
}

cqr_status coded_qr_run(cqr_handle h, const void* A, int64_t lda, const void* y, int64_t ldy,
                        void* x, int64_t ldx, int32_t nrhs, const int32_t* plan,
                        int32_t plan_len, uint32_t flags) {
  if (!h || !A || lda < h->g.m || plan_len < 0 || (plan_len > 0 && !plan)) return CQR_EINVAL;
  if ((y == nullptr) != (x == nullptr)) return CQR_EINVAL;
  if (y && (nrhs < 1 || nrhs > h->cfg.nrhs_max || ldy < h->g.m || ldx < h->g.n)) return CQR_EINVAL;
  for (int e = 0; e < plan_len; ++e) {
    const int t = plan[3 * e], i = plan[3 * e + 1], j = plan[3 * e + 2];
    if (t < 0 || t >= h->g.panels || !node_in_range(h, i, j)) return CQR_EINVAL;
  }
  const bool host = (flags & CQR_RUN_HOST_BUFFERS) != 0;
  const size_t es = h->esz;
  const Geo& g = h->g;
  const void* Ad = A;
  int64_t ldad = lda;
  const void* yd = y;
  int64_t ldyd = ldy;
  void* xd = x;
  int64_t ldxd = ldx;
  if (host) {
    // host -> device: A as one contiguous copy into the R buffer when it fits there (encode
    // reads it before it clears R; one large copy instead of n rows of a pitched copy), else
    // pitched straight into the systematic block of the encoded matrix (encode then runs in
    // place); y into the handle's workspace; x comes back from the workspace.
    const size_t a_bytes = (size_t)lda * (size_t)(g.n - 1) * es + (size_t)g.m * es;
    if (a_bytes <= (size_t)g.ldr * (size_t)g.N * es) {
      CK(cudaMemcpyAsync(h->B.R, A, a_bytes, cudaMemcpyHostToDevice, h->st));
      Ad = h->B.R;
      ldad = lda;
    } else {
      CK(cudaMemcpy2DAsync(h->B.Q, g.ldq * es, A, lda * es, g.m * es, g.n, cudaMemcpyHostToDevice,
                           h->st));
      Ad = h->B.Q;
      ldad = g.ldq;
    }
    if (y) {
      CK(cudaMemcpy2DAsync(h->B.xw, g.m * es, y, ldy * es, g.m * es, nrhs, cudaMemcpyHostToDevice, h->st));
      yd = h->B.xw;
      ldyd = g.m;
      xd = static_cast<char*>(h->B.xw) + (size_t)g.m * nrhs * es;
      ldxd = g.n;
    }
  }
  cqr_status s = coded_qr_encode(h, Ad, ldad);
  if (s != CQR_OK) return s;
  std::vector<int32_t> tiles;
  int t = 0;
  while (t < g.panels) {
    tiles.clear();
    for (int e = 0; e < plan_len; ++e)
      if (plan[3 * e] == t) node_tiles(h, plan[3 * e + 1], plan[3 * e + 2], &tiles);
    if (!tiles.empty()) {
      s = coded_qr_inject_erasure(h, tiles.data(), (int32_t)(tiles.size() / 2));
      if (s == CQR_OK) s = coded_qr_recover(h, nullptr);
      if (s != CQR_OK) return s;
    }
    int t_next = t + 1;
    while (t_next < g.panels) {
      bool hit = false;
      for (int e = 0; e < plan_len; ++e) hit |= (plan[3 * e] == t_next);
      if (hit) break;
      ++t_next;
    }
    s = coded_qr_factor(h, t, t_next);
    if (s != CQR_OK) return s;
    t = t_next;
  }
  if (g.m == g.n && g.m_pad == g.m) {
    s = coded_qr_post_orth(h, nullptr, 0, nullptr, 0, nullptr, 0, 0);
    if (s != CQR_OK) return s;
  }
  if (y) {
    s = coded_qr_solve(h, yd, ldyd, xd, ldxd, nrhs);
    if (s != CQR_OK) return s;
    if (host)
      CK(cudaMemcpy2DAsync(x, ldx * es, xd, ldxd * es, g.n * es, nrhs, cudaMemcpyDeviceToHost, h->st));
  }
  return read_status(h, false);
}

cqr_status coded_qr_get_factors(cqr_handle h, void** Q, int64_t* ldq, void** R, int64_t* ldr) {
  if (!h) return CQR_EINVAL;
  if (Q) *Q = h->B.Q;
  if (ldq) *ldq = h->g.ldq;
  if (R) *R = h->B.R;
  if (ldr) *ldr = h->g.ldr;
  return CQR_OK;
}

cqr_status coded_qr_get_generator(cqr_handle h, double* Gt, double* Gh) {
  if (!h) return CQR_EINVAL;
  if (h->state == ST_CREATED) return CQR_ESTATE;
  const Geo& g = h->g;
  if (g.f == 0) return CQR_OK;
  if (Gt) CK(cudaMemcpyAsync(Gt, h->B.Gt, sizeof(double) * g.f * g.p_r, cudaMemcpyDeviceToHost, h->st));
  if (Gh) CK(cudaMemcpyAsync(Gh, h->B.Gh, sizeof(double) * g.f * g.p_c, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return CQR_OK;
}

cqr_status coded_qr_get_decode_sets(cqr_handle h, int32_t* buf, int32_t cap, int32_t* len) {
  if (!h || cap < 0 || (cap > 0 && !buf)) return CQR_EINVAL;
  const int32_t n = (int32_t)h->sets.size();
  for (int32_t i = 0; i < n && i < cap; ++i) buf[i] = h->sets[i];
  if (len) *len = n;
  return CQR_OK;
}

cqr_status coded_qr_stats(cqr_handle h, int64_t* out) {
  if (!h || !out) return CQR_EINVAL;
  CK(cudaMemcpyAsync(h->status_host, h->B.status, 4 * sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  out[0] = h->status_host[1];
  out[1] = h->n_recovered;
  out[2] = h->panels_run;
  out[3] = h->n_injected;
  return CQR_OK;
}

cqr_status coded_qr_debug_bounds(int32_t* site) {
  if (site) *site = 0;
#ifndef CQR_DEBUG_BOUNDS
  return CQR_ENOTSUP;
#else
  cudaError_t (*const takes[])(int*, int*) = {bounds_take_kernels, bounds_take_panel,
                                              bounds_take_panel_reg, bounds_take_tc};
  cqr_status out = CQR_OK;
  for (auto take : takes) {
    int code = 0, where = 0;
    CK(take(&code, &where));
    if (code != 0 && out == CQR_OK) {
      out = CQR_EBOUNDS;
      if (site) *site = where;
    }
  }
  return out;
#endif
}

cqr_status coded_qr_debug_bounds_selftest(void* stream) {
#ifndef CQR_DEBUG_BOUNDS
  (void)stream;
  return CQR_ENOTSUP;
#else
  CK(launch_bounds_selftest(4, reinterpret_cast<cudaStream_t>(stream)));
  return CQR_OK;
#endif
}

cqr_status coded_qr_probe_exchange(int32_t kind, int64_t M, int32_t bk, int32_t reps,
                                   double* us_per_column, void* stream) {
  if (!us_per_column || M < 1 || bk < 1 || bk > 256 || reps < 1 || (kind != 0 && kind != 1))
    return CQR_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PanelPlan pp{};
  if (kind == 0) {
    int rpl = 0, cpw = 0, G = 0;
    if (!plan_panel_reg(M, bk, &rpl, &cpw, &G) || !panel_reg_cluster_fits(rpl, cpw, G))
      return CQR_EINVAL;
  } else {
    // the plan the handle's panel step takes for an FP32 panel of M rows (ensure_panel_plan)
    pp = plan_panel(M, bk, sizeof(float), sms, true);
    if (pp.cluster && !panel_cluster_fits<float>(pp)) pp = plan_panel(M, bk, sizeof(float), sms, false);
    if (pp.hier && !panel_hier_fits<float>(pp))
      pp = plan_panel(M, bk, sizeof(float), sms, pp.cluster != 0, true, 8);
    if (pp.hier && !panel_hier_fits<float>(pp))
      pp = plan_panel(M, bk, sizeof(float), sms, pp.cluster != 0, false);
    if (!pp.smem) return CQR_EINVAL;  // slices in global memory: no exchange-only floor
  }
  const size_t part_bytes = align256(panel_partial_bytes(bk, sizeof(float), sms));
  unsigned char* ws = nullptr;
  CK(cudaMalloc(&ws, part_bytes + 256));
  float* part = reinterpret_cast<float*>(ws);
  unsigned* bar = reinterpret_cast<unsigned*>(ws + part_bytes);
  int* status = reinterpret_cast<int*>(ws + part_bytes + 64);
  int* bad = reinterpret_cast<int*>(ws + part_bytes + 128);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMemsetAsync(ws, 0, part_bytes + 256, st);
  auto launch = [&](int r) {
    return kind == 0 ? launch_exchange_probe_reg(M, bk, r, status, bad, st)
                     : launch_exchange_probe(pp, bk, r, part, bar, status, bad, st);
  };
  if (e == cudaSuccess) e = launch(1);  // warm-up
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) e = launch(reps);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  int hs[4] = {0, 0, 0, 0}, hbad = 0;
  if (e == cudaSuccess) e = cudaMemcpy(hs, status, sizeof(hs), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(ws);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CQR_ECUDA;
  }
  if (hs[0] != 0) return (cqr_status)hs[0];
  if (hbad != 0) return CQR_ECUDA;
  *us_per_column = 1000.0 * ms / ((double)reps * bk);
  return CQR_OK;
}

cqr_status coded_qr_set_wait_limit(cqr_handle h, int64_t cycles) {
  if (!h || cycles < 0) return CQR_EINVAL;
  h->wait_limit = (long long)cycles;
  return CQR_OK;
}

cqr_status coded_qr_sync_status(cqr_handle h) {
  if (!h) return CQR_EINVAL;
  return read_status(h, true);
}

cqr_status coded_qr_profile(cqr_handle h, int32_t enable) {
  if (!h) return CQR_EINVAL;
  h->prof_on = enable != 0;
  return CQR_OK;
}

cqr_status coded_qr_profile_read(cqr_handle h, double* ms, int64_t* launches, int32_t cap,
                                 int32_t reset) {
  if (!h || cap < 0) return CQR_EINVAL;
  CK(cudaStreamSynchronize(h->st));
  for (auto& r : h->prof_recs) {
    float dt = 0.f;
    if (cudaEventElapsedTime(&dt, r.a, r.b) == cudaSuccess) h->prof_ms[r.cls] += dt;
    h->prof_pool.push_back(r.a);
    h->prof_pool.push_back(r.b);
  }
  h->prof_recs.clear();
  for (int k = 0; k < K_COUNT && k < cap; ++k) {
    if (ms) ms[k] = h->prof_ms[k];
    if (launches) launches[k] = h->prof_launches[k];
  }
  if (reset)
    for (int k = 0; k < K_COUNT; ++k) { h->prof_ms[k] = 0.0; h->prof_launches[k] = 0; }
  return CQR_OK;
}

const char* coded_qr_profile_name(int32_t cls) {
  return (cls >= 0 && cls < K_COUNT) ? kClassNames[cls] : nullptr;
}

const char* coded_qr_errstr(cqr_status s) {
  switch (s) {
    case CQR_OK: return "ok";
    case CQR_EINVAL: return "invalid argument";
    case CQR_ENOMEM: return "out of memory";
    case CQR_ECUDA: return "CUDA error";
    case CQR_ESTATE: return "call out of order or erasures pending";
    case CQR_EUNRECOVERABLE: return "erasure pattern not recoverable";
    case CQR_EBREAKDOWN: return "Gram-Schmidt breakdown (zero or non-finite pivot)";
    case CQR_ETIMEOUT: return "device wait timed out";
    case CQR_ENOTSUP: return "not supported";
    case CQR_EBOUNDS: return "index check failed on the device (bounds-checked build)";
  }
  return "unknown status";
}

}  // extern "C"

// ------------------------------------------------------------------------------- adjoints
namespace {

cqr_status adj_scratch(cqr_handle h, size_t bytes) {
  if (h->adj_bytes >= bytes) return CQR_OK;
  CK(cudaStreamSynchronize(h->st));
  if (h->adj) cudaFree(h->adj);
  h->adj = nullptr;
  h->adj_bytes = 0;
  if (cudaMalloc(&h->adj, bytes) != cudaSuccess) {
    cudaGetLastError();
    return CQR_ENOMEM;
  }
  h->adj_bytes = bytes;
  return CQR_OK;
}

template <typename T>
cqr_status adjoint_qr_t(cqr_handle h, const T* Q, int64_t ldq, const T* Qbar, int64_t ldqb,
                        const T* Rbar, int64_t ldrb, T* Abar, int64_t ldab) {
  const Geo& g = h->g;
  const int64_t n = g.n, mp = g.m_pad;
  const size_t nn = (size_t)n * n;
  // FP32 handles with tensor cores take the two large products (n x n x m_pad and m_pad x n
  // x n) in 3xTF32 through the operand planes; the rest, and FP64, on the CUDA cores
  bool tcq = false;
  if constexpr (sizeof(T) == 4) tcq = h->tc != nullptr;
  const size_t base_el = (2 * nn + (size_t)mp * n + 63) / 64 * 64;
  const size_t plane_el = tcq ? std::max(tc_gemm_sub_planes(true, n, mp), tc_gemm_sub_planes(false, mp, n)) : 0;
  cqr_status s = adj_scratch(h, sizeof(T) * (base_el + plane_el));
  if (s != CQR_OK) return s;
  T* Mm = static_cast<T*>(h->adj);
  T* S = Mm + nn;
  T* Bb = S + nn;
  float* planes = reinterpret_cast<float*>(Mm + base_el);
  const T* R = ptr<T>(h->B.R);
  // C -= op(A) B on the tensor cores; false when the operands break a tensor-map rule
  auto tc_sub = [&](bool a_trans, const T* A_, int64_t lda_, const T* B_, int64_t ldb_, T* C_,
                    int64_t ldc_, int64_t M_, int64_t N_, int64_t K_) -> int {
    if (!tcq) return 0;
    const cudaError_t e = tc_gemm_sub3(a_trans, reinterpret_cast<const float*>(A_), lda_,
                                       reinterpret_cast<const float*>(B_), ldb_,
                                       reinterpret_cast<float*>(C_), ldc_, M_, N_, K_, planes,
                                       h->num_sms, h->B.status, h->st);
    if (e == cudaSuccess) return 1;
    cudaGetLastError();
    return e == cudaErrorInvalidValue ? 0 : -1;
  };
  // M = R Rbar^T - Qbar^T Q
  if (Rbar)
    CK(launch_gemm_general<T>(0, 1, n, n, n, T(1), R, g.ldr, Rbar, ldrb, T(0), Mm, n, h->st));
  else
    CK(cudaMemsetAsync(Mm, 0, sizeof(T) * nn, h->st));
  if (Qbar) {
    const int r = tc_sub(true, Qbar, ldqb, Q, ldq, Mm, n, n, n, mp);
    if (r < 0) return CQR_ECUDA;
    if (r == 0)
      CK(launch_gemm_general<T>(1, 0, n, n, mp, T(-1), Qbar, ldqb, Q, ldq, T(1), Mm, n, h->st));
  }
  CK(launch_copyltu<T>(Mm, n, S, h->st));
  // Bbar = Qbar + Q copyltu(M), then Bbar R^{-T}
  if (Qbar)
    CK(launch_axpy2d<T>(mp, n, T(1), Qbar, 1, ldqb, Bb, 1, mp, true, h->st));
  else
    CK(cudaMemsetAsync(Bb, 0, sizeof(T) * (size_t)mp * n, h->st));
  int r3 = 0;
  if (tcq) {
    // Bbar -= Q (-S)
    CK(launch_axpy2d<T>(n, n, T(-1), S, 1, n, S, 1, n, true, h->st));
    r3 = tc_sub(false, Q, ldq, S, n, Bb, mp, mp, n, n);
    if (r3 < 0) return CQR_ECUDA;
    if (r3 == 0) CK(launch_axpy2d<T>(n, n, T(-1), S, 1, n, S, 1, n, true, h->st));  // S back
  }
  if (r3 == 0)
    CK(launch_gemm_general<T>(0, 0, mp, n, n, T(1), Q, ldq, S, n, T(1), Bb, mp, h->st));
  CK(launch_trsm_right<T>(1, R, g.ldr, n, Bb, 1, mp, mp, h->st));
  // Abar += G_0^T Bbar (G_0 is symmetric: its leading block I - V V^T / 2 is), rows < m
  if (g.f > 0) CK(launch_post_orth<T>(g, ptr<T>(h->B.Gt_t), Bb, mp, mp, n, Bb, mp, h->st));
  CK(launch_axpy2d<T>(g.m, n, T(1), Bb, 1, mp, Abar, 1, ldab, false, h->st));
  return CQR_OK;
}

template <typename T>
cqr_status adjoint_lstsq_t(cqr_handle h, const T* A, int64_t lda, const T* y, int64_t ldy,
                           const T* x, int64_t ldx, const T* xbar, int64_t ldxb, int32_t k,
                           T* Abar, int64_t ldab, T* ybar, int64_t ldyb) {
  const Geo& g = h->g;
  const int64_t m = g.m, n = g.n;
  cqr_status s = adj_scratch(h, sizeof(T) * ((size_t)2 * n * k + (size_t)2 * m * k));
  if (s != CQR_OK) return s;
  T* u = static_cast<T*>(h->adj);  // n x k: R^{-T} xbar, then z
  T* w = u + (size_t)n * k;        // n x k
  T* Az = w + (size_t)n * k;       // m x k
  T* r = Az + (size_t)m * k;       // m x k
  const T* R = ptr<T>(h->B.R);
  // u = R^{-T} xbar: rows of the (k x n) view solve u^T R = xbar^T
  CK(launch_axpy2d<T>(n, k, T(1), xbar, 1, ldxb, u, 1, n, true, h->st));
  for (int32_t j = 0; j < k; ++j)  // each right-hand side is one contiguous row
    CK(launch_trsm_right<T>(0, R, g.ldr, n, u + (size_t)j * n, 1, 1, 1, h->st));
  // w = (I - Q_2^T Q_2)^{-1} u (FP64 conjugate gradients), z = R^{-1} w
  for (int32_t j = 0; j < k; ++j)
    CK(launch_ls_cg<T>(ptr<T>(h->B.Q), g.ldq, g.m, g.m_pad, g.c, n, nullptr, w + (size_t)j * n,
                       h->B.cg, h->B.bar, h->B.status, h->num_sms, h->st, u + (size_t)j * n));
  for (int32_t j = 0; j < k; ++j)
    CK(launch_trsm_right<T>(1, R, g.ldr, n, w + (size_t)j * n, 1, 1, 1, h->st));
  const T* z = w;
  // Az, r = y - A x
  CK(launch_gemm_general<T>(0, 0, m, k, n, T(1), A, lda, z, n, T(0), Az, m, h->st));
  CK(launch_axpy2d<T>(m, k, T(1), y, 1, ldy, r, 1, m, true, h->st));
  CK(launch_gemm_general<T>(0, 0, m, k, n, T(-1), A, lda, x, ldx, T(1), r, m, h->st));
  // Abar += r z^T - (A z) x^T;  ybar += A z
  if (Abar) {
    CK(launch_gemm_general<T>(0, 1, m, n, k, T(1), r, m, z, n, T(1), Abar, ldab, h->st));
    CK(launch_gemm_general<T>(0, 1, m, n, k, T(-1), Az, m, x, ldx, T(1), Abar, ldab, h->st));
  }
  if (ybar) CK(launch_axpy2d<T>(m, k, T(1), Az, 1, m, ybar, 1, ldyb, false, h->st));
  return CQR_OK;
}

}  // namespace

cqr_status coded_qr_adjoint_qr(cqr_handle h, const void* Q, int64_t ldq, const void* Qbar,
                               int64_t ldqb, const void* Rbar, int64_t ldrb, void* Abar,
                               int64_t ldab) {
  if (!h || !Q || !Abar || (!Qbar && !Rbar)) return CQR_EINVAL;
  if (h->state != ST_FACTORED || h->pending || h->next_panel < h->g.panels) return CQR_ESTATE;
  if (ldq < h->g.m_pad || (Qbar && ldqb < h->g.m_pad) || (Rbar && ldrb < h->g.n) ||
      ldab < h->g.m)
    return CQR_EINVAL;
  return h->esz == 8
             ? adjoint_qr_t<double>(h, (const double*)Q, ldq, (const double*)Qbar, ldqb,
                                    (const double*)Rbar, ldrb, (double*)Abar, ldab)
             : adjoint_qr_t<float>(h, (const float*)Q, ldq, (const float*)Qbar, ldqb,
                                   (const float*)Rbar, ldrb, (float*)Abar, ldab);
}

cqr_status coded_qr_adjoint_lstsq(cqr_handle h, const void* A, int64_t lda, const void* y,
                                  int64_t ldy, const void* x, int64_t ldx, const void* xbar,
                                  int64_t ldxb, int32_t nrhs, void* Abar, int64_t ldab,
                                  void* ybar, int64_t ldyb) {
  if (!h || !A || !y || !x || !xbar || nrhs < 1 || (!Abar && !ybar)) return CQR_EINVAL;
  if (h->state != ST_FACTORED || h->pending || h->next_panel < h->g.panels) return CQR_ESTATE;
  if (h->postorth_inplace) return CQR_ESTATE;  // Q_1 was overwritten by G_0 Q_1
  const Geo& g = h->g;
  if (lda < g.m || ldy < g.m || ldx < g.n || ldxb < g.n || (Abar && ldab < g.m) ||
      (ybar && ldyb < g.m))
    return CQR_EINVAL;
  return h->esz == 8
             ? adjoint_lstsq_t<double>(h, (const double*)A, lda, (const double*)y, ldy,
                                       (const double*)x, ldx, (const double*)xbar, ldxb, nrhs,
                                       (double*)Abar, ldab, (double*)ybar, ldyb)
             : adjoint_lstsq_t<float>(h, (const float*)A, lda, (const float*)y, ldy,
                                      (const float*)x, ldx, (const float*)xbar, ldxb, nrhs,
                                      (float*)Abar, ldab, (float*)ybar, ldyb);
}

// Host helpers shared with the batched entry points (coded_qr_batched.cu).
namespace cqr {
cqr_status host_validate(const cqr_config* c) { return validate(c); }
Geo host_geo(const cqr_config* c) { return make_geo(c); }
bool host_make_plan(int nsys, int f, const uint8_t* lost_sys, const uint8_t* lost_chk,
                    DecodePlan* p) {
  return make_plan(nsys, f, lost_sys, lost_chk, p);
}
}  // namespace cqr
