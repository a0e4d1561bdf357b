// coded_qr_batched.cu -- C-ABI entry points for a batch of independent coded QRs: device
// memory of all instances, erasure bookkeeping (host-side index sets per instance), the
// autotuner of the panel widths and the cluster size, and the launch sequence, optionally
// recorded once into a CUDA graph and replayed.  Every arithmetic step runs in the kernels of
// cqr_batched.cu and cqr_kernels.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "coded_qr.h"
#include "cqr_batched.cuh"
#include "cqr_host.h"

using namespace cqr;

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Last CUDA error seen by a batch entry point on this host thread (coded_qr_batched_last_error).
thread_local cudaError_t g_last_cuda = cudaSuccess;

#define BK(x)                 \
  do {                        \
    cudaError_t e_ = (x);     \
    if (e_ != cudaSuccess) {  \
      g_last_cuda = e_;       \
      cudaGetLastError();     \
      return CQR_ECUDA;       \
    }                         \
  } while (0)

}  // namespace

struct cqr_batched_s {
  cqr_config cfg{};
  int count = 0;
  int num_sms = 0;
  cudaStream_t st = nullptr;
  cudaStream_t cap_st = nullptr;  // recording stream (the caller's may be the legacy stream)
  double tau2 = 0.5;
  std::vector<Geo> geo;
  std::vector<int> b;            // panel width per instance
  std::vector<int> next_panel;   // first panel not yet factorised
  std::vector<uint8_t> mask;     // pending erasures, grid_rows x grid_cols per instance
  std::vector<size_t> mask_off;
  std::vector<std::vector<int32_t>> sets;  // decode index sets since encode, per instance
  std::vector<int> order;        // scheduling order (decreasing cost)
  int G = 1;                     // CTAs per instance
  int grid = 0;                  // CTAs of the factor launch
  int panel_cap = 0;
  bool encoded = false, pending = false, post_orthed = false;
  int64_t n_injected = 0, n_recovered = 0;
  // device memory
  void* mem = nullptr;
  BatchInst<float>* d_inst = nullptr;
  std::vector<BatchInst<float>> h_inst;
  int64_t* d_off_v = nullptr;
  int64_t* d_off_h = nullptr;
  int64_t* d_off_p = nullptr;
  int64_t tot_v = 0, tot_h = 0, tot_p = 0;
  int* d_order = nullptr;
  int* d_order_ab = nullptr;   // [2][count]: the two factor phases of a run, each by its own work
  int* d_queue = nullptr;      // two counters
  int* d_range_a = nullptr;
  int* d_range_b = nullptr;
  int* d_status = nullptr;     // 4 ints per instance
  double* d_Gt = nullptr;
  double* d_Gh = nullptr;
  float* d_Gt_t = nullptr;
  float* d_Gh_t = nullptr;
  float* d_R0 = nullptr;       // first R (all R blocks are contiguous)
  size_t r_bytes = 0;
  BatchPlan* d_plans = nullptr;
  int64_t* d_plan_off = nullptr;
  int plan_cap = 0;
  BatchTile* d_tiles = nullptr;
  int tile_cap = 0;
  int64_t max_tile_elems = 0;
  // phase clocks of the factor launch (instrumentation)
  unsigned long long* d_prof = nullptr;
  bool prof_on = false;
  // recorded sequence
  cudaGraphExec_t gexec = nullptr;
  std::vector<int64_t> gkey;
};

namespace {

cqr_status upload(cqr_batched bh, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return CQR_OK;
  // pageable source: the call returns once the bytes are staged, so src may be reused
  BK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, bh->st));
  return CQR_OK;
}

// Panel width from the shape: 32 (fewer passes over the trailing columns) unless the
// instance is narrow, where the ICGS column steps of a wide panel dominate.
int fit_width(const Geo& g, int G, int cap) {
  (void)G;
  (void)cap;
  return g.n >= 96 ? 32 : 16;
}

cqr_status set_cluster(cqr_batched bh, int G) {
  const int cap = b_panel_cap_floats(G);
  const int nc = b_max_clusters(G, cap);
  if (nc <= 0) return CQR_ENOTSUP;
  bh->G = G;
  bh->panel_cap = cap;
  bh->grid = nc * G;
  return CQR_OK;
}

cqr_status push_widths(cqr_batched bh) {
  for (int i = 0; i < bh->count; ++i) {
    bh->h_inst[i].b = bh->b[i];
    bh->geo[i].b = bh->b[i];
    bh->geo[i].panels = (int)((bh->geo[i].n + bh->b[i] - 1) / bh->b[i]);
    bh->h_inst[i].g = bh->geo[i];
  }
  bh->gkey.clear();
  return upload(bh, bh->d_inst, bh->h_inst.data(), sizeof(BatchInst<float>) * bh->count);
}

cqr_status enqueue_encode(cqr_batched bh) {
  BK(cudaMemsetAsync(bh->d_R0, 0, bh->r_bytes, bh->st));
  BK(cudaMemsetAsync(bh->d_status, 0, sizeof(int) * 4 * bh->count, bh->st));
  BK(launch_b_encode<float>(bh->d_inst, bh->count, bh->d_off_v, bh->tot_v, bh->d_off_h, bh->tot_h,
                            bh->d_Gt_t, bh->d_Gh_t, bh->cfg.f, bh->st));
  return CQR_OK;
}

cqr_status enqueue_factor(cqr_batched bh, const int* d_range, int queue_slot,
                          const int* d_order = nullptr) {
  BK(cudaMemsetAsync(bh->d_queue + queue_slot, 0, sizeof(int), bh->st));
  BFactorLaunch L;
  L.G = bh->G;
  L.grid = bh->grid;
  L.inst = bh->d_inst;
  L.count = bh->count;
  L.order = d_order ? d_order : bh->d_order;
  L.range = d_range;
  L.queue = bh->d_queue + queue_slot;
  L.tau2 = bh->tau2;
  L.panel_cap = bh->panel_cap;
  L.tiles = bh->d_tiles;
  L.plans = bh->d_plans;
  L.Gt = bh->d_Gt;
  L.Gh = bh->d_Gh;
  L.prof = bh->prof_on ? bh->d_prof : nullptr;
  BK(launch_b_factor(L, bh->st));
  return CQR_OK;
}

// Tiles poisoned by one erasure event (Q tile, and the R tile of a protected block row).
void tiles_of(const Geo& g, int inst, int i, int j, std::vector<BatchTile>* out) {
  out->push_back(BatchTile{inst, i, j, 0});
  if (g.protect_r && i < g.p_c + g.f) out->push_back(BatchTile{inst, i, j, 1});
}

// Decode plans of instance `inst` from its mask; appends to plans and to the index sets.
cqr_status plan_instance(cqr_batched bh, int inst, std::vector<BatchPlan>* plans, int* nrec) {
  const Geo& g = bh->geo[inst];
  const uint8_t* mk = bh->mask.data() + bh->mask_off[inst];
  const int gc = g.grid_cols, f = g.f;
  std::vector<uint8_t> ls(kMaxCode), lc(kMaxCode);
  std::vector<BatchPlan> mine;
  for (int j = 0; j < gc; ++j) {
    BatchPlan bp{};
    bp.inst = inst;
    bp.p.kind = 0;
    bp.p.idx = j;
    for (int t = 0; t < g.p_r; ++t) ls[t] = mk[(size_t)t * gc + j];
    for (int i = 0; i < f; ++i) lc[i] = mk[(size_t)(g.p_r + i) * gc + j];
    if (!host_make_plan(g.p_r, f, ls.data(), lc.data(), &bp.p)) return CQR_EUNRECOVERABLE;
    if (bp.p.f1 + bp.p.f2 == 0) continue;
    *nrec += bp.p.f1 + bp.p.f2;
    mine.push_back(bp);
  }
  if (g.protect_r) {
    for (int i = 0; i < g.p_c + f && i < g.grid_rows; ++i) {
      BatchPlan bp{};
      bp.inst = inst;
      bp.p.kind = 1;
      bp.p.idx = i;
      for (int j = 0; j < g.p_c; ++j) ls[j] = mk[(size_t)i * gc + j];
      for (int l = 0; l < f; ++l) lc[l] = mk[(size_t)i * gc + g.p_c + l];
      if (!host_make_plan(g.p_c, f, ls.data(), lc.data(), &bp.p)) return CQR_EUNRECOVERABLE;
      if (bp.p.f1 + bp.p.f2 == 0) continue;
      mine.push_back(bp);
    }
  }
  for (const BatchPlan& bp : mine) {
    const DecodePlan& p = bp.p;
    std::vector<int32_t>& s = bh->sets[inst];
    s.push_back(p.kind);
    s.push_back(p.idx);
    s.push_back(p.f1);
    s.push_back(p.f2);
    for (int a = 0; a < p.f1; ++a) s.push_back(p.A_fail[a]);
    for (int e = 0; e < p.f2; ++e) s.push_back(p.C_fail[e]);
    for (int a = 0; a < p.f1; ++a) s.push_back(p.C_use[a]);
    plans->push_back(bp);
  }
  return CQR_OK;
}

cqr_status upload_plans(cqr_batched bh, const std::vector<BatchPlan>& plans, int64_t* total) {
  if ((int)plans.size() > bh->plan_cap) return CQR_EINVAL;
  std::vector<int64_t> off(plans.size() + 1, 0);
  for (size_t k = 0; k < plans.size(); ++k)
    off[k + 1] = off[k] + batch_decode_blocks(bh->geo[plans[k].inst], plans[k].p);
  *total = off.back();
  cqr_status s = upload(bh, bh->d_plans, plans.data(), sizeof(BatchPlan) * plans.size());
  if (s != CQR_OK) return s;
  return upload(bh, bh->d_plan_off, off.data(), sizeof(int64_t) * off.size());
}

cqr_status check_inputs(cqr_batched bh, const void* const* A, const int64_t* lda) {
  if (!A || !lda) return CQR_EINVAL;
  for (int i = 0; i < bh->count; ++i)
    if (!A[i] || lda[i] < bh->geo[i].m) return CQR_EINVAL;
  for (int i = 0; i < bh->count; ++i) {
    bh->h_inst[i].A = static_cast<const float*>(A[i]);
    bh->h_inst[i].lda = lda[i];
    bh->h_inst[i].rec_at = 0;  // no recovery inside a factor launch unless a run plans one
  }
  return upload(bh, bh->d_inst, bh->h_inst.data(), sizeof(BatchInst<float>) * bh->count);
}

void reset_state(cqr_batched bh) {
  std::fill(bh->next_panel.begin(), bh->next_panel.end(), 0);
  std::fill(bh->mask.begin(), bh->mask.end(), 0);
  for (auto& s : bh->sets) s.clear();
  bh->pending = false;
  bh->post_orthed = false;
  bh->n_injected = bh->n_recovered = 0;
  bh->encoded = true;
}

}  // namespace

extern "C" {

cqr_status coded_qr_batched_create(const cqr_config* cfg, const int64_t* m, const int64_t* n,
                                   int32_t count, cqr_batched* out) {
  if (!cfg || !m || !n || !out || count < 1) return CQR_EINVAL;
  *out = nullptr;
  if (cfg->dtype != CQR_F32) return CQR_ENOTSUP;
  if (cfg->mma != CQR_MMA_SIMT) return CQR_ENOTSUP;
  if (cfg->b < 0 || cfg->b > kBMax) return cfg->b < 0 ? CQR_EINVAL : CQR_ENOTSUP;
  if (cfg->reorth_block || cfg->in_node || cfg->panel != CQR_PANEL_ICGS) return CQR_ENOTSUP;
  std::vector<Geo> geo(count);
  for (int i = 0; i < count; ++i) {
    cqr_config c = *cfg;
    c.m = m[i];
    c.n = n[i];
    c.b = cfg->b > 0 ? cfg->b : 16;
    c.mma = CQR_MMA_SIMT;
    const cqr_status v = host_validate(&c);
    if (v != CQR_OK) return v;
    geo[i] = host_geo(&c);
  }
  cqr_batched bh = new (std::nothrow) cqr_batched_s();
  if (!bh) return CQR_ENOMEM;
  bh->cfg = *cfg;
  bh->count = count;
  bh->st = static_cast<cudaStream_t>(cfg->stream);
  bh->tau2 = cfg->tau == 0.0 ? 0.5 : (cfg->tau > 0.0 ? cfg->tau * cfg->tau : -1.0);
  bh->geo = geo;
  bh->b.assign(count, cfg->b > 0 ? cfg->b : 16);
  bh->next_panel.assign(count, 0);
  bh->sets.resize(count);
  bh->mask_off.resize(count + 1, 0);
  for (int i = 0; i < count; ++i)
    bh->mask_off[i + 1] = bh->mask_off[i] + (size_t)geo[i].grid_rows * geo[i].grid_cols;
  bh->mask.assign(bh->mask_off[count], 0);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&bh->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaStreamCreateWithFlags(&bh->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete bh;
    return CQR_ECUDA;
  }
  // default cluster size: the smallest that keeps most panel slices in shared memory
  cqr_status s = CQR_ENOTSUP;
  for (int G : {2, 1, 4, 8})
    if ((s = set_cluster(bh, G)) == CQR_OK) break;
  if (s != CQR_OK) {
    cudaStreamDestroy(bh->cap_st);
    delete bh;
    return s;
  }
  if (cfg->b == 0)
    for (int i = 0; i < count; ++i) bh->b[i] = fit_width(geo[i], bh->G, bh->panel_cap);
  // device memory: all Q blocks, all R blocks (contiguous), then the small arrays
  size_t off = 0;
  std::vector<size_t> qoff(count), roff(count);
  for (int i = 0; i < count; ++i) {
    qoff[i] = off;
    off += al256((size_t)geo[i].ldq * geo[i].N * sizeof(float));
  }
  const size_t r0 = off;
  for (int i = 0; i < count; ++i) {
    roff[i] = off;
    off += al256((size_t)geo[i].ldr * geo[i].N * sizeof(float));
  }
  bh->r_bytes = off - r0;
  int plan_cap = 0, tile_cap = 0;
  int64_t max_elems = 0;
  for (int i = 0; i < count; ++i) {
    plan_cap += geo[i].grid_cols + geo[i].p_c + geo[i].f;
    tile_cap += 2 * geo[i].grid_rows * geo[i].grid_cols;
    max_elems = std::max<int64_t>(max_elems, std::max(geo[i].mb, geo[i].nb) * geo[i].nb);
  }
  bh->plan_cap = plan_cap;
  bh->tile_cap = tile_cap;
  bh->max_tile_elems = max_elems;
  auto take = [&](size_t bytes) { size_t o = off; off += al256(bytes); return o; };
  const size_t o_inst = take(sizeof(BatchInst<float>) * count);
  const size_t o_offv = take(sizeof(int64_t) * (count + 1));
  const size_t o_offh = take(sizeof(int64_t) * (count + 1));
  const size_t o_offp = take(sizeof(int64_t) * (count + 1));
  const size_t o_order = take(sizeof(int) * count);
  const size_t o_order_ab = take(sizeof(int) * 2 * count);
  const size_t o_queue = take(sizeof(int) * 2);
  const size_t o_ra = take(sizeof(int) * 2 * count);
  const size_t o_rb = take(sizeof(int) * 2 * count);
  const size_t o_status = take(sizeof(int) * 4 * count);
  const int f = cfg->f, p_r = cfg->p_r, p_c = cfg->p_c;
  const size_t o_gt = take(sizeof(double) * std::max(1, f * p_r));
  const size_t o_gh = take(sizeof(double) * std::max(1, p_c * f));
  const size_t o_gtt = take(sizeof(float) * std::max(1, f * p_r));
  const size_t o_ght = take(sizeof(float) * std::max(1, p_c * f));
  const size_t o_plans = take(sizeof(BatchPlan) * std::max(1, plan_cap));
  const size_t o_planoff = take(sizeof(int64_t) * (plan_cap + 1));
  const size_t o_tiles = take(sizeof(BatchTile) * std::max(1, tile_cap));
  if (cudaMalloc(&bh->mem, off) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamDestroy(bh->cap_st);
    delete bh;
    return CQR_ENOMEM;
  }
  char* base = static_cast<char*>(bh->mem);
  bh->d_R0 = reinterpret_cast<float*>(base + r0);
  bh->d_inst = reinterpret_cast<BatchInst<float>*>(base + o_inst);
  bh->d_off_v = reinterpret_cast<int64_t*>(base + o_offv);
  bh->d_off_h = reinterpret_cast<int64_t*>(base + o_offh);
  bh->d_off_p = reinterpret_cast<int64_t*>(base + o_offp);
  bh->d_order = reinterpret_cast<int*>(base + o_order);
  bh->d_order_ab = reinterpret_cast<int*>(base + o_order_ab);
  bh->d_queue = reinterpret_cast<int*>(base + o_queue);
  bh->d_range_a = reinterpret_cast<int*>(base + o_ra);
  bh->d_range_b = reinterpret_cast<int*>(base + o_rb);
  bh->d_status = reinterpret_cast<int*>(base + o_status);
  bh->d_Gt = reinterpret_cast<double*>(base + o_gt);
  bh->d_Gh = reinterpret_cast<double*>(base + o_gh);
  bh->d_Gt_t = reinterpret_cast<float*>(base + o_gtt);
  bh->d_Gh_t = reinterpret_cast<float*>(base + o_ght);
  bh->d_plans = reinterpret_cast<BatchPlan*>(base + o_plans);
  bh->d_plan_off = reinterpret_cast<int64_t*>(base + o_planoff);
  bh->d_tiles = reinterpret_cast<BatchTile*>(base + o_tiles);
  bh->h_inst.resize(count);
  for (int i = 0; i < count; ++i) {
    BatchInst<float>& I = bh->h_inst[i];
    I = BatchInst<float>{};
    I.g = geo[i];
    I.Q = reinterpret_cast<float*>(base + qoff[i]);
    I.R = reinterpret_cast<float*>(base + roff[i]);
    I.status = bh->d_status + 4 * i;
  }
  // scheduling order: decreasing flops 2 M n (n + 2 d), ties by index
  std::vector<double> cost(count);
  for (int i = 0; i < count; ++i)
    cost[i] = 2.0 * geo[i].M * geo[i].n * (double)(geo[i].n + 2 * geo[i].d);
  bh->order.resize(count);
  std::iota(bh->order.begin(), bh->order.end(), 0);
  std::stable_sort(bh->order.begin(), bh->order.end(),
                   [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<int64_t> ov(count + 1, 0), oh(count + 1, 0), op(count + 1, 0);
  for (int i = 0; i < count; ++i) {
    ov[i + 1] = ov[i] + batch_encode_blocks(geo[i], false);
    oh[i + 1] = oh[i] + batch_encode_blocks(geo[i], true);
    op[i + 1] = op[i] + batch_post_orth_blocks(geo[i]);
  }
  bh->tot_v = ov[count];
  bh->tot_h = oh[count];
  bh->tot_p = op[count];
  s = CQR_OK;
  if (s == CQR_OK) s = push_widths(bh);
  if (s == CQR_OK) s = upload(bh, bh->d_off_v, ov.data(), sizeof(int64_t) * ov.size());
  if (s == CQR_OK) s = upload(bh, bh->d_off_h, oh.data(), sizeof(int64_t) * oh.size());
  if (s == CQR_OK) s = upload(bh, bh->d_off_p, op.data(), sizeof(int64_t) * op.size());
  if (s == CQR_OK) s = upload(bh, bh->d_order, bh->order.data(), sizeof(int) * count);
  if (s == CQR_OK && cudaMemsetAsync(bh->d_status, 0, sizeof(int) * 4 * count, bh->st) != cudaSuccess)
    s = CQR_ECUDA;
  if (s == CQR_OK && launch_generator<float>(f, p_r, p_c, cfg->seed, cfg->gdist, bh->d_Gt, bh->d_Gh,
                                             bh->d_Gt_t, bh->d_Gh_t, bh->st) != cudaSuccess)
    s = CQR_ECUDA;
  if (s == CQR_OK && cudaStreamSynchronize(bh->st) != cudaSuccess) s = CQR_ECUDA;
  if (s != CQR_OK) {
    cudaGetLastError();
    cudaFree(bh->mem);
    cudaStreamDestroy(bh->cap_st);
    delete bh;
    return s;
  }
  *out = bh;
  return CQR_OK;
}

cqr_status coded_qr_batched_destroy(cqr_batched bh) {
  if (!bh) return CQR_EINVAL;
  cudaStreamSynchronize(bh->st);
  if (bh->gexec) cudaGraphExecDestroy(bh->gexec);
  if (bh->mem) cudaFree(bh->mem);
  if (bh->d_prof) cudaFree(bh->d_prof);
  if (bh->cap_st) cudaStreamDestroy(bh->cap_st);
  cudaGetLastError();
  delete bh;
  return CQR_OK;
}

cqr_status coded_qr_batched_geometry(cqr_batched bh, int32_t i, int64_t* d) {
  if (!bh || !d || i < 0 || i >= bh->count) return CQR_EINVAL;
  const Geo& g = bh->geo[i];
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

cqr_status coded_qr_batched_encode(cqr_batched bh, const void* const* A, const int64_t* lda) {
  if (!bh) return CQR_EINVAL;
  cqr_status s = check_inputs(bh, A, lda);
  if (s != CQR_OK) return s;
  s = enqueue_encode(bh);
  if (s != CQR_OK) return s;
  reset_state(bh);
  return CQR_OK;
}

cqr_status coded_qr_batched_factor(cqr_batched bh, const int32_t* panel_end) {
  if (!bh) return CQR_EINVAL;
  if (!bh->encoded || bh->pending || bh->post_orthed) return CQR_ESTATE;
  std::vector<int> r(2 * bh->count);
  for (int i = 0; i < bh->count; ++i) {
    const int pe = panel_end ? panel_end[i] : bh->geo[i].panels;
    if (pe < bh->next_panel[i] || pe > bh->geo[i].panels) return CQR_EINVAL;
    r[2 * i] = bh->next_panel[i];
    r[2 * i + 1] = pe;
  }
  bh->gkey.clear();  // the recorded sequence reads d_range_a
  cqr_status s = upload(bh, bh->d_range_a, r.data(), sizeof(int) * r.size());
  if (s != CQR_OK) return s;
  s = enqueue_factor(bh, bh->d_range_a, 0);
  if (s != CQR_OK) return s;
  for (int i = 0; i < bh->count; ++i) bh->next_panel[i] = r[2 * i + 1];
  return CQR_OK;
}

cqr_status coded_qr_batched_inject_erasure(cqr_batched bh, const int32_t* tiles, int32_t count) {
  if (!bh || count < 0 || (count > 0 && !tiles)) return CQR_EINVAL;
  if (!bh->encoded || bh->post_orthed) return CQR_ESTATE;
  for (int e = 0; e < count; ++e) {
    const int k = tiles[3 * e], i = tiles[3 * e + 1], j = tiles[3 * e + 2];
    if (k < 0 || k >= bh->count) return CQR_EINVAL;
    if (i < 0 || i >= bh->geo[k].grid_rows || j < 0 || j >= bh->geo[k].grid_cols) return CQR_EINVAL;
  }
  if (count == 0) return CQR_OK;
  std::vector<BatchTile> list;
  for (int e = 0; e < count; ++e) {
    const int k = tiles[3 * e], i = tiles[3 * e + 1], j = tiles[3 * e + 2];
    bh->mask[bh->mask_off[k] + (size_t)i * bh->geo[k].grid_cols + j] = 1;
    tiles_of(bh->geo[k], k, i, j, &list);
  }
  if ((int)list.size() > bh->tile_cap) return CQR_EINVAL;
  bh->gkey.clear();  // the recorded sequence reads d_tiles
  cqr_status s = upload(bh, bh->d_tiles, list.data(), sizeof(BatchTile) * list.size());
  if (s != CQR_OK) return s;
  BK(launch_b_poison<float>(bh->d_inst, bh->d_tiles, (int)list.size(), bh->max_tile_elems,
                            bh->num_sms, bh->st));
  bh->pending = true;
  bh->n_injected += count;
  return CQR_OK;
}

cqr_status coded_qr_batched_recover(cqr_batched bh, int32_t* n_recovered) {
  if (!bh) return CQR_EINVAL;
  if (n_recovered) *n_recovered = 0;
  if (!bh->encoded) return CQR_ESTATE;
  if (!bh->pending) return CQR_OK;
  if (bh->cfg.f == 0) return CQR_EUNRECOVERABLE;
  std::vector<BatchPlan> plans;
  int nrec = 0;
  for (int k = 0; k < bh->count; ++k) {
    const cqr_status s = plan_instance(bh, k, &plans, &nrec);
    if (s != CQR_OK) return s;
  }
  int64_t total = 0;
  bh->gkey.clear();  // the recorded sequence reads d_plans
  cqr_status s = upload_plans(bh, plans, &total);
  if (s != CQR_OK) return s;
  BK(launch_b_decode<float>(bh->d_inst, bh->d_plans, (int)plans.size(), bh->d_plan_off, total,
                            bh->d_Gt, bh->d_Gh, bh->num_sms, bh->st));
  std::fill(bh->mask.begin(), bh->mask.end(), 0);
  bh->pending = false;
  bh->n_recovered += nrec;
  if (n_recovered) *n_recovered = nrec;
  return CQR_OK;
}

cqr_status coded_qr_batched_post_orth(cqr_batched bh) {
  if (!bh) return CQR_EINVAL;
  if (!bh->encoded || bh->pending || bh->post_orthed) return CQR_ESTATE;
  for (int i = 0; i < bh->count; ++i)
    if (bh->next_panel[i] != bh->geo[i].panels) return CQR_ESTATE;
  BK(launch_b_post_orth<float>(bh->d_inst, bh->count, bh->d_off_p, bh->tot_p, bh->d_Gt_t,
                               bh->num_sms, bh->st));
  bh->post_orthed = true;
  return CQR_OK;
}

cqr_status coded_qr_batched_run(cqr_batched bh, const void* const* A, const int64_t* lda,
                                const int32_t* erasures, int32_t count, int32_t flags) {
  if (!bh || count < 0 || (count > 0 && !erasures)) return CQR_EINVAL;
  if (flags & ~(CQR_BATCH_GRAPH | CQR_BATCH_POST_ORTH | CQR_BATCH_HOST_BUFFERS)) return CQR_EINVAL;
  // one erasure event per instance: every tile of instance k is lost at the same panel
  std::vector<int> t_of(bh->count, -1);
  for (int e = 0; e < count; ++e) {
    const int k = erasures[4 * e], t = erasures[4 * e + 1];
    const int i = erasures[4 * e + 2], j = erasures[4 * e + 3];
    if (k < 0 || k >= bh->count) return CQR_EINVAL;
    const Geo& g = bh->geo[k];
    if (t < 0 || t >= g.panels || i < 0 || i >= g.grid_rows || j < 0 || j >= g.grid_cols)
      return CQR_EINVAL;
    if (t_of[k] >= 0 && t_of[k] != t) return CQR_ENOTSUP;
    t_of[k] = t;
  }
  // host buffers: the encode reads each A from the systematic block of the instance's own
  // encoded matrix, where copy_in puts it (in place: every position is read and rewritten
  // with the same value by one thread); the device addresses also key the recorded graph
  const bool host = (flags & CQR_BATCH_HOST_BUFFERS) != 0;
  std::vector<const void*> a_dev;
  std::vector<int64_t> ld_dev;
  if (host) {
    if (!A || !lda) return CQR_EINVAL;
    for (int k = 0; k < bh->count; ++k) {
      if (!A[k] || lda[k] < bh->geo[k].m) return CQR_EINVAL;
      a_dev.push_back(bh->h_inst[k].Q);
      ld_dev.push_back(bh->geo[k].ldq);
    }
  }
  const void* const* Ause = host ? a_dev.data() : A;
  const int64_t* lduse = host ? ld_dev.data() : lda;
  cqr_status s = check_inputs(bh, Ause, lduse);
  if (s != CQR_OK) return s;
  reset_state(bh);
  auto copy_in = [&]() -> cqr_status {
    if (!host) return CQR_OK;
    for (int k = 0; k < bh->count; ++k) {
      const Geo& g = bh->geo[k];
      BK(cudaMemcpy2DAsync(bh->h_inst[k].Q, (size_t)g.ldq * sizeof(float), A[k],
                           (size_t)lda[k] * sizeof(float), (size_t)g.m * sizeof(float),
                           (size_t)g.n, cudaMemcpyHostToDevice, bh->st));
    }
    return CQR_OK;
  };
  // host planning (before anything is enqueued, so that an unrecoverable pattern launches
  // nothing): panel ranges of the two factor phases, poisoned tiles, decode plans
  std::vector<int> ra(2 * bh->count), rb(2 * bh->count);
  for (int k = 0; k < bh->count; ++k) {
    const int P = bh->geo[k].panels, t = t_of[k] >= 0 ? t_of[k] : P;
    ra[2 * k] = 0;
    ra[2 * k + 1] = t;
    rb[2 * k] = t;
    rb[2 * k + 1] = P;
  }
  std::vector<BatchTile> list;
  for (int e = 0; e < count; ++e) {
    const int k = erasures[4 * e], i = erasures[4 * e + 2], j = erasures[4 * e + 3];
    bh->mask[bh->mask_off[k] + (size_t)i * bh->geo[k].grid_cols + j] = 1;
    tiles_of(bh->geo[k], k, i, j, &list);
  }
  if ((int)list.size() > bh->tile_cap) return CQR_EINVAL;
  std::vector<BatchPlan> plans;
  int nrec = 0;
  if (count > 0) {
    if (bh->cfg.f == 0) s = CQR_EUNRECOVERABLE;
    for (int k = 0; k < bh->count && s == CQR_OK; ++k) s = plan_instance(bh, k, &plans, &nrec);
    if (s != CQR_OK) {
      bh->encoded = false;
      std::fill(bh->mask.begin(), bh->mask.end(), 0);
      return s;
    }
  }
  // Recovery inside the factor launch when the coefficient tables fit the panel pool: every
  // instance runs all its panels in one launch and its cluster poisons and decodes its own
  // tiles at the start of its erasure panel (no second launch waiting for the slowest
  // instance of the first).  Tiles and plans are grouped by instance.
  const bool fused = !list.empty() && bh->panel_cap >= b_recover_floats();
  if (fused) {
    std::stable_sort(list.begin(), list.end(),
                     [](const BatchTile& x, const BatchTile& y) { return x.inst < y.inst; });
    for (int k = 0; k < bh->count; ++k) {
      BatchInst<float>& I = bh->h_inst[k];
      I.rec_at = 0;
      I.tile0 = I.ntiles = I.plan0 = I.nplans = 0;
    }
    for (int e = 0; e < (int)list.size(); ++e) {
      BatchInst<float>& I = bh->h_inst[list[e].inst];
      if (I.ntiles == 0) I.tile0 = e;
      ++I.ntiles;
    }
    for (int e = 0; e < (int)plans.size(); ++e) {
      BatchInst<float>& I = bh->h_inst[plans[e].inst];
      if (I.nplans == 0) I.plan0 = e;
      ++I.nplans;
    }
    for (int k = 0; k < bh->count; ++k) {
      BatchInst<float>& I = bh->h_inst[k];
      if (t_of[k] >= 0 && (I.ntiles > 0 || I.nplans > 0)) I.rec_at = t_of[k] + 1;
      ra[2 * k] = 0;
      ra[2 * k + 1] = bh->geo[k].panels;
    }
    s = upload(bh, bh->d_inst, bh->h_inst.data(), sizeof(BatchInst<float>) * bh->count);
    if (s != CQR_OK) return s;
  }
  // work order of each factor phase: decreasing work of that phase (longest first), the work
  // of panel t being M bk (N - t b) (its panel and its trailing update)
  std::vector<int> ord(2 * bh->count);
  for (int ph = 0; ph < 2; ++ph) {
    const std::vector<int>& rg = ph == 0 ? ra : rb;
    std::vector<double> w(bh->count, 0.0);
    for (int k = 0; k < bh->count; ++k) {
      const Geo& g = bh->geo[k];
      const int b = bh->h_inst[k].b;
      for (int t = rg[2 * k]; t < rg[2 * k + 1]; ++t) {
        const int64_t kb = (int64_t)t * b;
        w[k] += (double)g.M * (double)std::min<int64_t>(b, g.n - kb) * (double)(g.N - kb);
      }
    }
    int* o = ord.data() + ph * bh->count;
    std::iota(o, o + bh->count, 0);
    std::stable_sort(o, o + bh->count, [&](int x, int y) { return w[x] > w[y]; });
  }
  std::vector<int64_t> key;
  key.push_back(flags);
  key.push_back(fused ? 1 : 0);
  key.push_back(bh->prof_on ? 1 : 0);
  for (int e = 0; e < 4 * count; ++e) key.push_back(erasures[e]);
  for (int k = 0; k < bh->count; ++k) {
    key.push_back(reinterpret_cast<int64_t>(Ause[k]));
    key.push_back(lduse[k]);
  }
  const bool replay = (flags & CQR_BATCH_GRAPH) && bh->gexec && key == bh->gkey;
  int64_t dec_total = 0;
  if (!replay) {
    s = upload(bh, bh->d_range_a, ra.data(), sizeof(int) * ra.size());
    if (s == CQR_OK) s = upload(bh, bh->d_range_b, rb.data(), sizeof(int) * rb.size());
    if (s == CQR_OK) s = upload(bh, bh->d_order_ab, ord.data(), sizeof(int) * ord.size());
    if (s == CQR_OK) s = upload(bh, bh->d_tiles, list.data(), sizeof(BatchTile) * list.size());
    if (s == CQR_OK) s = upload_plans(bh, plans, &dec_total);
    if (s != CQR_OK) return s;
  }
  auto sequence = [&]() -> cqr_status {
    cqr_status r = enqueue_encode(bh);
    if (fused) {
      if (r == CQR_OK) r = enqueue_factor(bh, bh->d_range_a, 0, bh->d_order);
      if (r == CQR_OK && (flags & CQR_BATCH_POST_ORTH))
        BK(launch_b_post_orth<float>(bh->d_inst, bh->count, bh->d_off_p, bh->tot_p, bh->d_Gt_t,
                                     bh->num_sms, bh->st));
      return r;
    }
    if (r == CQR_OK) r = enqueue_factor(bh, bh->d_range_a, 0, bh->d_order_ab);
    if (r == CQR_OK && !list.empty()) {
      BK(launch_b_poison<float>(bh->d_inst, bh->d_tiles, (int)list.size(), bh->max_tile_elems,
                                bh->num_sms, bh->st));
      BK(launch_b_decode<float>(bh->d_inst, bh->d_plans, (int)plans.size(), bh->d_plan_off,
                                dec_total, bh->d_Gt, bh->d_Gh, bh->num_sms, bh->st));
    }
    if (r == CQR_OK && !list.empty()) r = enqueue_factor(bh, bh->d_range_b, 1, bh->d_order_ab + bh->count);
    if (r == CQR_OK && (flags & CQR_BATCH_POST_ORTH))
      BK(launch_b_post_orth<float>(bh->d_inst, bh->count, bh->d_off_p, bh->tot_p, bh->d_Gt_t,
                                   bh->num_sms, bh->st));
    return r;
  };
  if (flags & CQR_BATCH_GRAPH) {
    if (!replay) {
      if (bh->gexec) {
        cudaGraphExecDestroy(bh->gexec);
        bh->gexec = nullptr;
      }
      bh->gkey.clear();
      // record on the batch's own stream; the graph is then launched on the caller's
      cudaStream_t user = bh->st;
      BK(cudaStreamBeginCapture(bh->cap_st, cudaStreamCaptureModeThreadLocal));
      bh->st = bh->cap_st;
      const cqr_status r = sequence();
      bh->st = user;
      cudaGraph_t graph = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(bh->cap_st, &graph);
      if (r != CQR_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return r != CQR_OK ? r : CQR_ECUDA;
      }
      const cudaError_t ie = cudaGraphInstantiate(&bh->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) {
        bh->gexec = nullptr;
        cudaGetLastError();
        return CQR_ECUDA;
      }
      bh->gkey = key;
    }
    s = copy_in();
    if (s != CQR_OK) return s;
    BK(cudaGraphLaunch(bh->gexec, bh->st));
  } else {
    s = copy_in();
    if (s == CQR_OK) s = sequence();
    if (s != CQR_OK) return s;
  }
  for (int k = 0; k < bh->count; ++k) bh->next_panel[k] = bh->geo[k].panels;
  std::fill(bh->mask.begin(), bh->mask.end(), 0);
  bh->n_injected += count;
  bh->n_recovered += nrec;
  bh->post_orthed = (flags & CQR_BATCH_POST_ORTH) != 0;
  return CQR_OK;
}

cqr_status coded_qr_batched_set_tuning(cqr_batched bh, int32_t cluster, const int32_t* b) {
  if (!bh) return CQR_EINVAL;
  if (cluster != 1 && cluster != 2 && cluster != 4 && cluster != 8) return CQR_EINVAL;
  if (b)
    for (int i = 0; i < bh->count; ++i)
      if (b[i] < 1 || b[i] > kBMax) return CQR_EINVAL;
  BK(cudaStreamSynchronize(bh->st));
  const cqr_status s = set_cluster(bh, cluster);
  if (s != CQR_OK) return s;
  for (int i = 0; i < bh->count; ++i)
    bh->b[i] = b ? b[i] : fit_width(bh->geo[i], bh->G, bh->panel_cap);
  bh->encoded = false;  // panel boundaries changed: encode again before factorising
  return push_widths(bh);
}

cqr_status coded_qr_batched_get_tuning(cqr_batched bh, int32_t* cluster, int32_t* b) {
  if (!bh) return CQR_EINVAL;
  if (cluster) *cluster = bh->G;
  if (b)
    for (int i = 0; i < bh->count; ++i) b[i] = bh->b[i];
  return CQR_OK;
}

cqr_status coded_qr_batched_autotune(cqr_batched bh, const void* const* A, const int64_t* lda,
                                     const int32_t* erasures, int32_t count, int32_t reps,
                                     int32_t* cluster_out) {
  if (!bh || reps < 1 || count < 0 || (count > 0 && !erasures)) return CQR_EINVAL;
  cqr_status s = check_inputs(bh, A, lda);
  if (s != CQR_OK) return s;
  // the erasure panels are given for the shape rule's widths; a candidate with other widths
  // keeps each event at the same column position (panel index rescaled, clamped)
  std::vector<int> t_col(count);
  for (int e = 0; e < count; ++e) {
    const int k = erasures[4 * e];
    if (k < 0 || k >= bh->count) return CQR_EINVAL;
    t_col[e] = erasures[4 * e + 1] * bh->b[k];
  }
  cudaEvent_t e0, e1;
  BK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return CQR_ECUDA;
  }
  // time of the whole sequence of coded_qr_batched_run (encode, factor, erase, recover,
  // factor) under (G, widths): the best of `reps` runs, after one untimed run
  std::vector<int32_t> er(erasures ? erasures : (const int32_t*)nullptr,
                          erasures ? erasures + 4 * count : (const int32_t*)nullptr);
  auto measure = [&](int G, const std::vector<int>& w, float* ms) -> cqr_status {
    cqr_status r = coded_qr_batched_set_tuning(bh, G, w.data());
    if (r != CQR_OK) return r;
    for (int e = 0; e < count; ++e) {
      const int k = er[4 * e];
      er[4 * e + 1] = std::min(t_col[e] / bh->b[k], bh->geo[k].panels - 1);
    }
    float best = 1e30f;
    for (int k = -1; k < reps; ++k) {
      BK(cudaEventRecord(e0, bh->st));
      r = coded_qr_batched_run(bh, A, lda, er.data(), count, 0);
      if (r != CQR_OK) return r;
      BK(cudaEventRecord(e1, bh->st));
      BK(cudaEventSynchronize(e1));
      float t = 0.f;
      BK(cudaEventElapsedTime(&t, e0, e1));
      if (k >= 0) best = std::min(best, t);
    }
    *ms = best;
    return CQR_OK;
  };
  int bestG = bh->G;
  std::vector<int> bestw = bh->b;
  float best_ms = 1e30f;
  // 1. cluster size x uniform width rule (16, 32, 64, or the shape-fit rule)
  for (int G : {1, 2, 4, 8}) {
    const int cap = b_panel_cap_floats(G);
    if (b_max_clusters(G, cap) <= 0) continue;
    for (int rule : {0, 16, 32, 64}) {
      std::vector<int> w(bh->count);
      for (int i = 0; i < bh->count; ++i) w[i] = rule ? rule : fit_width(bh->geo[i], G, cap);
      float ms = 0.f;
      s = measure(G, w, &ms);
      if (s != CQR_OK) break;
      if (ms < best_ms) {
        best_ms = ms;
        bestG = G;
        bestw = w;
      }
    }
    if (s != CQR_OK) break;
  }
  // 2. per size class of the encoded height (M < 1024, < 4096, >= 4096): try each width
  //    for that class alone, keep it when the whole batch gets faster
  if (s == CQR_OK) {
    for (int cls = 0; cls < 3 && s == CQR_OK; ++cls) {
      auto in_cls = [&](int i) {
        const int64_t M = bh->geo[i].M;
        return cls == 0 ? M < 1024 : (cls == 1 ? (M >= 1024 && M < 4096) : M >= 4096);
      };
      bool any = false;
      for (int i = 0; i < bh->count; ++i) any |= in_cls(i);
      if (!any) continue;
      for (int wv : {16, 32, 64}) {
        std::vector<int> w = bestw;
        for (int i = 0; i < bh->count; ++i)
          if (in_cls(i)) w[i] = wv;
        if (w == bestw) continue;
        float ms = 0.f;
        s = measure(bestG, w, &ms);
        if (s != CQR_OK) break;
        if (ms < best_ms) {
          best_ms = ms;
          bestw = w;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != CQR_OK) return s;
  // leave the batch encoded and factorised (no erasures) under the chosen tuning
  s = coded_qr_batched_set_tuning(bh, bestG, bestw.data());
  if (s == CQR_OK) s = coded_qr_batched_encode(bh, A, lda);
  if (s == CQR_OK) s = coded_qr_batched_factor(bh, nullptr);
  if (s == CQR_OK && cluster_out) *cluster_out = bestG;
  return s;
}

cqr_status coded_qr_batched_get_factors(cqr_batched bh, int32_t i, void** Q, int64_t* ldq,
                                        void** R, int64_t* ldr) {
  if (!bh || i < 0 || i >= bh->count) return CQR_EINVAL;
  if (Q) *Q = bh->h_inst[i].Q;
  if (ldq) *ldq = bh->geo[i].ldq;
  if (R) *R = bh->h_inst[i].R;
  if (ldr) *ldr = bh->geo[i].ldr;
  return CQR_OK;
}

cqr_status coded_qr_batched_get_decode_sets(cqr_batched bh, int32_t i, int32_t* buf, int32_t cap,
                                            int32_t* len) {
  if (!bh || i < 0 || i >= bh->count || cap < 0) return CQR_EINVAL;
  const std::vector<int32_t>& s = bh->sets[i];
  if (len) *len = (int32_t)s.size();
  if (buf)
    for (int32_t k = 0; k < cap && k < (int32_t)s.size(); ++k) buf[k] = s[k];
  return CQR_OK;
}

cqr_status coded_qr_batched_sync_status(cqr_batched bh, int32_t* first_bad, int64_t* reorth) {
  if (!bh) return CQR_EINVAL;
  BK(cudaStreamSynchronize(bh->st));
  std::vector<int> st(4 * (size_t)bh->count);
  BK(cudaMemcpy(st.data(), bh->d_status, sizeof(int) * st.size(), cudaMemcpyDeviceToHost));
  int64_t nre = 0;
  int bad = -1;
  for (int i = 0; i < bh->count; ++i) {
    nre += st[4 * i + 1];
    if (bad < 0 && st[4 * i] != 0) bad = i;
  }
  if (first_bad) *first_bad = bad;
  if (reorth) *reorth = nre;
  return bad < 0 ? CQR_OK : (cqr_status)st[4 * bad];
}

cqr_status coded_qr_batched_profile(cqr_batched bh, int32_t enable) {
  if (!bh) return CQR_EINVAL;
  if (enable && !bh->d_prof) {
    BK(cudaMalloc(&bh->d_prof, sizeof(unsigned long long) * (kPhases + 1)));
    BK(cudaMemsetAsync(bh->d_prof, 0, sizeof(unsigned long long) * (kPhases + 1), bh->st));
  }
  bh->prof_on = enable != 0;
  return CQR_OK;
}

cqr_status coded_qr_batched_phases(cqr_batched bh, int64_t* cycles, int32_t reset) {
  if (!bh || !cycles) return CQR_EINVAL;
  if (!bh->d_prof) return CQR_ESTATE;
  unsigned long long h[kPhases + 1];
  BK(cudaStreamSynchronize(bh->st));
  BK(cudaMemcpy(h, bh->d_prof, sizeof(h), cudaMemcpyDeviceToHost));
  for (int k = 0; k <= kPhases; ++k) cycles[k] = (int64_t)h[k];
  if (reset) {
    BK(cudaMemsetAsync(bh->d_prof, 0, sizeof(h), bh->st));
    BK(cudaStreamSynchronize(bh->st));
  }
  return CQR_OK;
}

const char* coded_qr_batched_last_error(void) { return cudaGetErrorString(g_last_cuda); }

}  // extern "C"
