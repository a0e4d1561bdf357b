// cqr_batched.cu -- many independent coded QRs (uneven tall-skinny shapes) factorised by one
// persistent launch.
//
// Each instance is the method of Section 4 on its own encoded matrix: PBMGS (Section 2.2,
// Algorithm PBMGS) whose panels are factorised by CGS with the ICGS reorthogonalisation test
// (Appendix A, Algorithm CGS / ICGS), followed by the trailing update
//   Rbar = Qbar^T Q[:, kb+bk : N],   Q[:, kb+bk : N] -= Qbar Rbar,   R[kb:kb+bk, kb+bk:] = Rbar.
// The trailing block includes the d horizontal checksum columns, so the checksum relations
// Q_2 = G_v Q_1 and R_2 = R_1 G_h are carried along exactly as in the single-instance path.
//
// Schedule: the grid is persistent (as many clusters as fit at one CTA per SM).  A cluster of
// G CTAs takes the next instance from an atomic queue (instances sorted by decreasing cost,
// so the long ones start first) and factorises its panel range; CTA g of the cluster owns
// the contiguous row slice [g rpc, (g+1) rpc) of that instance for the whole factorisation.
// Column sums over rows are reduced within a CTA (warp shuffles, then a fixed-order sum of the
// warp partials) and across the cluster through distributed shared memory after a hardware
// cluster barrier (fixed order over the G CTAs): every reduction is deterministic.
// The panel slice lives in shared memory when it fits, otherwise it is worked on in place in
// global memory (L2).  The trailing update runs in chunks of 64 columns with FP32 FMAs.
// There are no spin-waits: only CTA and cluster barriers.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "cqr_batched.cuh"
#include "cqr_decode.cuh"
#include "cqr_device.cuh"

namespace cqr {

namespace {

constexpr int kBT = 512;        // threads per CTA
constexpr int kBW = kBT / 32;   // warps per CTA

__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}
__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t s_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ float ld_cl(uint32_t local_addr, uint32_t rank) {
  uint32_t a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(local_addr), "r"(rank));
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ int ld_cl_i32(uint32_t local_addr, uint32_t rank) {
  uint32_t a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(local_addr), "r"(rank));
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}

// Phase clocks (instrumentation, off unless the launch is given a counter array): thread 0 of
// each CTA adds the SM cycles between consecutive marks to the phase that just ended, in
// shared memory, and adds its totals to the launch's array when the CTA leaves.  The slots
// live in shared memory so that the other threads carry no extra registers.
//   slots [0, kPhases): cycles per phase; [kPhases]: last mark; [kPhases + 1]: the array
__device__ __forceinline__ long long* ph_slots() {
  __shared__ long long s_ph[kPhases + 2];
  return s_ph;
}
__device__ __forceinline__ void ph_begin(unsigned long long* prof) {
  if (threadIdx.x == 0) {
    long long* s = ph_slots();
    for (int k = 0; k < kPhases; ++k) s[k] = 0;
    s[kPhases] = clock64();
    s[kPhases + 1] = (long long)reinterpret_cast<uintptr_t>(prof);
  }
}
__device__ __forceinline__ void ph_mark(int phase) {
  if (threadIdx.x == 0) {
    long long* s = ph_slots();
    if (s[kPhases + 1] != 0) {
      const long long now = clock64();
      s[phase] += now - s[kPhases];
      s[kPhases] = now;
    }
  }
}
__device__ __forceinline__ void ph_end() {
  if (threadIdx.x == 0) {
    long long* s = ph_slots();
    unsigned long long* prof = reinterpret_cast<unsigned long long*>((uintptr_t)s[kPhases + 1]);
    if (prof) {
      ph_mark(PH_OTHER);
      for (int k = 0; k < kPhases; ++k) atomicAdd(prof + k, (unsigned long long)s[k]);
      atomicAdd(prof + kPhases, 1ull);
    }
  }
}

// Shared-memory layout (in floats), the same for every CTA of a launch.
//   small : v, eta, sv [kBMax each], warp partials [256]
//   cpart : cluster partials, two buffers of kBMax * kWC (G > 1)
//   rbar  : the summed Rbar chunk [kBMax][kWC]
//   pool  : the stages of the trailing-update pipeline (B rows and Qbar rows, see b_update);
//           after a K loop it holds the K-split partial sums (<= 8192 floats); during the
//           panel it is scratch for per-CTA sums
constexpr int kKT = 64;        // rows per pipeline stage
constexpr int kLDS = kKT + 4;  // row stride of a staged column (16-byte aligned)
constexpr int kMaxStages = 8;
constexpr int kPanelScratch = 8192 + kBW * 2 * kBMax;  // per-CTA sums and warp partials

struct BLayout {
  int small, wpart, cpart, rbar, pool, total;
};

__host__ __device__ inline BLayout b_layout(int G) {
  BLayout L;
  L.small = 0;
  L.wpart = 3 * kBMax;
  L.cpart = L.wpart + 256;
  L.rbar = L.cpart + (G > 1 ? 2 * kBMax * kWC : 0);
  L.pool = L.rbar + kBMax * kWC;
  L.total = L.pool;
  return L;
}

// Floats of one pipeline stage for a panel of width bk: kWC columns of B and bk (rounded up
// to 4) columns of Qbar, kKT rows each.
__host__ __device__ inline int stage_floats(int bk) { return (kWC + (bk + 3) / 4 * 4) * kLDS; }

template <int G>
struct BCtx {
  float* sm;
  BLayout L;
  int tid, lane, warp;
  uint32_t rank;
  unsigned step;  // reduction counter (same sequence on every CTA of the cluster)
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Wait until at most n committed groups are pending (n is rounded down to 0 .. 6).
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_wait_dyn(int n) {
  switch (n) {
    case 6: cp_wait<6>(); break;
    case 5: cp_wait<5>(); break;
    case 4: cp_wait<4>(); break;
    case 3: cp_wait<3>(); break;
    case 2: cp_wait<2>(); break;
    case 1: cp_wait<1>(); break;
    default: cp_wait<0>(); break;
  }
}

// Sum over the cluster of this CTA's values loc[0 .. n) (already summed over the CTA) into
// out[0 .. n).  The partials go to the cpart buffer of parity `step`; a buffer is rewritten
// two reductions later, after every peer has passed the barrier of the reduction in between.
template <int G>
__device__ __forceinline__ void cluster_sum(BCtx<G>& c, const float* loc, int n, float* out) {
  if (G == 1) {
    __syncthreads();
    for (int a = c.tid; a < n; a += kBT) out[a] = loc[a];
    __syncthreads();
    return;
  }
  float* mine = c.sm + c.L.cpart + (c.step & 1) * (kBMax * kWC);
  __syncthreads();
  for (int a = c.tid; a < n; a += kBT) mine[a] = loc[a];
  cl_sync();
  const uint32_t base = s_addr(mine);
  for (int a = c.tid; a < n; a += kBT) {
    float s = 0.f;
#pragma unroll
    for (int g = 0; g < G; ++g) s += ld_cl(base + 4u * (uint32_t)a, (uint32_t)g);
    out[a] = s;
  }
  ++c.step;
  __syncthreads();
}

// Warps form a (column group) x (row group) grid that depends on nv only: cg column groups
// (a power of two <= min(nv, 16)), 16 / cg row groups; row group q covers rows
// q*32 + lane + k*32*(16/cg).
struct ColGrid {
  int cg, rg, cgi, rgi;
  __device__ ColGrid(int nv, int warp) {
    cg = 1;
    while (cg * 2 <= nv && cg * 2 <= kBW) cg *= 2;
    rg = kBW / cg;
    cgi = warp % cg;
    rgi = warp / cg;
  }
};

// Per-CTA column sums of a load-only summand val(a, r) for a in [0, nv), over rows [0, nr).
// Four independent partial sums per lane keep several loads in flight; the combination order
// is fixed.  Result in loc[0 .. nv) (after the CTA barrier inside).
template <int G, typename F>
__device__ __forceinline__ void cta_colsums(BCtx<G>& c, int nv, int nr, float* loc, F val) {
  const ColGrid cg(nv, c.warp);
  float* wp = c.sm + c.L.wpart;  // [rg][nv], rg * nv <= 256
  const int step = 32 * cg.rg;
  for (int a = cg.cgi; a < nv; a += cg.cg) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int r = cg.rgi * 32 + c.lane;
    for (; r + 3 * step < nr; r += 4 * step) {
      s0 += val(a, r);
      s1 += val(a, r + step);
      s2 += val(a, r + 2 * step);
      s3 += val(a, r + 3 * step);
    }
    for (; r < nr; r += step) s0 += val(a, r);
    const float s = warp_sum((s0 + s1) + (s2 + s3));
    if (c.lane == 0) wp[cg.rgi * nv + a] = s;
  }
  __syncthreads();
  for (int a = c.tid; a < nv; a += kBT) {
    float s = 0.f;
    for (int q = 0; q < cg.rg; ++q) s += wp[q * nv + a];
    loc[a] = s;
  }
}

// Rows of the slice per thread and block: thread t owns rows blk*RPT*kBT + t + k*kBT, k < RPT
// (RPT = 4, 8 or 10 by the slice height, so that short slices run short loops).

// Sum of one value per thread over the CTA for each of nv columns: warp shuffles, then a
// fixed-order sum over the warps (wp: [kBW][nv] scratch) into loc (accumulate when add).
__device__ __forceinline__ void warp_part(float s, int a, int nv, float* wp, int warp, int lane) {
  s = warp_sum(s);
  if (lane == 0) wp[warp * nv + a] = s;
}

// Columns a = j + 1 + a1 + u (u < CW) of the fused column step: every load of the CW columns
// first, then per column the update p_a -= q (v_a / r_jj), its store and the warp's part of
// p_a^T p'.  The arithmetic of each column is that of a group of one.
template <int kRPT, int CW>
__device__ __forceinline__ void update_cols(float* P, int64_t cs, int nr, int rb, int j, int a1,
                                            int nv, float inv, const float* v,
                                            const float (&q)[kRPT], const float (&p1)[kRPT],
                                            float* wp, int warp, int lane) {
  float x[CW][kRPT];
#pragma unroll
  for (int u = 0; u < CW; ++u) {
    const float* pa = P + (j + 1 + a1 + u) * cs;
#pragma unroll
    for (int k = 0; k < kRPT; ++k) {
      const int r = rb + k * kBT;
      x[u][k] = (r < nr) ? pa[r] : 0.f;
    }
  }
#pragma unroll
  for (int u = 0; u < CW; ++u) {
    float* pa = P + (j + 1 + a1 + u) * cs;
    const float ca = v[j + 1 + a1 + u] * inv;
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kRPT; ++k) {
      const int r = rb + k * kBT;
      x[u][k] = fmaf(-q[k], ca, x[u][k]);
      if (r < nr) pa[r] = x[u][k];
      s = fmaf(x[u][k], p1[k], s);
    }
    warp_part(s, a1 + u, nv, wp, warp, lane);
  }
}

// The fused column step of the panel, row-split: with q = p_j / r_jj and p' = p_{j+1} - q c1
// (kept in registers for the thread's own rows and written back at once, since no other
// thread reads these rows during the step),
//   p_a -= q (v_a / r_jj) for a >= j+2, and per-CTA sums v'_a = p_a^T p' for a >= j+1
//   (a = j+1 giving |p'|^2), into loc[0 .. bk-j-1).
template <int G, int kRPT>
__device__ __forceinline__ void cta_update_sums(BCtx<G>& c, float* P, int64_t cs, int nr, int bk,
                                                int j, float inv, float c1, const float* v,
                                                float* loc) {
  constexpr int kRB = kRPT * kBT;
  const int nv = bk - j - 1;
  float* wp = c.sm + c.L.pool + 8192;  // [kBW][nv] (the pool is idle during the panel)
  float* pj = P + j * cs;
  float* pj1 = P + (j + 1) * cs;
  for (int a = c.tid; a < nv; a += kBT) loc[a] = 0.f;
  for (int blk = 0; blk * kRB < nr; ++blk) {
    const int rb = blk * kRB + c.tid;
    float q[kRPT], p1[kRPT];
#pragma unroll
    for (int k = 0; k < kRPT; ++k) {
      const int r = rb + k * kBT;
      q[k] = 0.f;
      p1[k] = 0.f;
      if (r < nr) {
        q[k] = pj[r] * inv;
        p1[k] = fmaf(-q[k], c1, pj1[r]);
      }
    }
#pragma unroll
    for (int k = 0; k < kRPT; ++k) {
      const int r = rb + k * kBT;
      if (r < nr) {
        pj[r] = q[k];
        pj1[r] = p1[k];
      }
    }
    {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < kRPT; ++k) s = fmaf(p1[k], p1[k], s);
      warp_part(s, 0, nv, wp, c.warp, c.lane);
    }
    // columns in groups of kCW: with the slice in L2 every group costs one round trip, since
    // the loads of a column cannot move above the stores of the one before it
    constexpr int kCW = 4;
    int a1 = 1;
    for (; a1 + kCW <= nv; a1 += kCW)
      update_cols<kRPT, kCW>(P, cs, nr, rb, j, a1, nv, inv, v, q, p1, wp, c.warp, c.lane);
    for (; a1 < nv; ++a1)
      update_cols<kRPT, 1>(P, cs, nr, rb, j, a1, nv, inv, v, q, p1, wp, c.warp, c.lane);
    __syncthreads();
    for (int a = c.tid; a < nv; a += kBT) {
      float t = 0.f;
      for (int w = 0; w < kBW; ++w) t += wp[w * nv + a];
      loc[a] += t;
    }
    __syncthreads();
  }
}

// Step 0 of the panel, row-split: per-CTA v_a = p_a^T p_0 (loc[a]) and eta_a = p_a^T p_a
// (loc[bk + a]).
template <int G, int kRPT>
__device__ __forceinline__ void cta_start_sums(BCtx<G>& c, const float* P, int64_t cs, int nr,
                                               int bk, float* loc) {
  constexpr int kRB = kRPT * kBT;
  float* wp = c.sm + c.L.pool + 8192;  // [kBW][2 bk]
  for (int a = c.tid; a < 2 * bk; a += kBT) loc[a] = 0.f;
  for (int blk = 0; blk * kRB < nr; ++blk) {
    const int rb = blk * kRB + c.tid;
    float p0[kRPT];
#pragma unroll
    for (int k = 0; k < kRPT; ++k) {
      const int r = rb + k * kBT;
      p0[k] = (r < nr) ? P[r] : 0.f;
    }
    // columns in groups of four: the loads of a group go out together (the shared-memory
    // stores of the warp partials keep later loads from moving above them)
    int a = 0;
    for (; a + 4 <= bk; a += 4) {
      float x[4][kRPT];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int k = 0; k < kRPT; ++k) {
          const int r = rb + k * kBT;
          x[u][k] = (r < nr) ? P[(a + u) * cs + r] : 0.f;
        }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int k = 0; k < kRPT; ++k) {
          s0 = fmaf(x[u][k], p0[k], s0);
          s1 = fmaf(x[u][k], x[u][k], s1);
        }
        warp_part(s0, a + u, 2 * bk, wp, c.warp, c.lane);
        warp_part(s1, bk + a + u, 2 * bk, wp, c.warp, c.lane);
      }
    }
    for (; a < bk; ++a) {
      const float* pa = P + a * cs;
      float x[kRPT];
#pragma unroll
      for (int k = 0; k < kRPT; ++k) {
        const int r = rb + k * kBT;
        x[k] = (r < nr) ? pa[r] : 0.f;
      }
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int k = 0; k < kRPT; ++k) {
        s0 = fmaf(x[k], p0[k], s0);
        s1 = fmaf(x[k], x[k], s1);
      }
      warp_part(s0, a, 2 * bk, wp, c.warp, c.lane);
      warp_part(s1, bk + a, 2 * bk, wp, c.warp, c.lane);
    }
    __syncthreads();
    for (int a = c.tid; a < 2 * bk; a += kBT) {
      float t = 0.f;
      for (int w = 0; w < kBW; ++w) t += wp[w * 2 * bk + a];
      loc[a] += t;
    }
    __syncthreads();
  }
}

// One panel: columns kb .. kb+bk-1 of the instance, this CTA's rows [0, nr) of the slice at
// P (column stride cs).  Writes R's diagonal block (rank 0).  Returns false on breakdown.
template <int G, int RPT>
__device__ bool b_panel(BCtx<G>& c, float* P, int64_t cs, int nr, int bk, float* R, int64_t ldr,
                        int kb, double tau2, int* status) {
  float* v = c.sm + c.L.small;
  float* eta = v + kBMax;
  float* sv = eta + kBMax;
  float* loc = c.sm + c.L.pool;  // per-CTA sums (the pipeline stages are idle during the panel)
  float* tmp = c.sm + c.L.rbar;  // cluster sums
  // step 0: v_a = p_a^T p_0 and eta_a = p_a^T p_a
  cta_start_sums<G, RPT>(c, P, cs, nr, bk, loc);
  cluster_sum<G>(c, loc, 2 * bk, tmp);
  // eta_a is kept as the ICGS threshold: the FP64 product tau^2 eta_a rounded up to FP32, so
  // that the FP32 test v_j < eta_j decides exactly as the FP64 one, with one FP64 product per
  // column instead of one per thread and column
  const bool icgs = tau2 > 0.0;
  for (int a = c.tid; a < bk; a += kBT) {
    v[a] = tmp[a];
    eta[a] = icgs ? __double2float_ru(tau2 * (double)tmp[bk + a]) : tmp[bk + a];
  }
  __syncthreads();
  for (int j = 0; j < bk; ++j) {
    if (j > 0 && icgs && v[j] < eta[j]) {
      // ICGS: project p_j once more on q_0 .. q_{j-1}
      cta_colsums<G>(c, j, nr, loc, [&](int a, int r) { return P[r + a * cs] * P[r + j * cs]; });
      cluster_sum<G>(c, loc, j, sv);
      for (int r = c.tid; r < nr; r += kBT) {
        float acc = P[r + j * cs];
        for (int a = 0; a < j; ++a) acc -= P[r + a * cs] * sv[a];
        P[r + j * cs] = acc;
      }
      if (c.rank == 0) {
        for (int a = c.tid; a < j; a += kBT) R[(kb + a) + (int64_t)(kb + j) * ldr] += sv[a];
        if (c.tid == 0) atomicAdd(status + ST_REORTH, 1);
      }
      __syncthreads();
      cta_colsums<G>(c, bk - j, nr, loc,
                     [&](int a, int r) { return P[r + (j + a) * cs] * P[r + j * cs]; });
      cluster_sum<G>(c, loc, bk - j, tmp);
      for (int a = c.tid; a < bk - j; a += kBT) v[j + a] = tmp[a];
      __syncthreads();
    }
    const float v0 = v[j];
    if (!(v0 > 0.f) || !isfinite(v0)) {
      if (c.rank == 0 && c.tid == 0) set_status(status, CQR_EBREAKDOWN, kb + j);
      return false;
    }
    const float rjj = sqrtf(v0);
    const float inv = 1.f / rjj;
    if (c.rank == 0) {
      for (int a = j + c.tid; a < bk; a += kBT)
        R[(kb + j) + (int64_t)(kb + a) * ldr] = (a == j) ? rjj : v[a] * inv;
    }
    if (j + 1 == bk) {
      for (int r = c.tid; r < nr; r += kBT) P[r + j * cs] *= inv;
      __syncthreads();
      break;
    }
    const float c1 = v[j + 1] * inv;
    cta_update_sums<G, RPT>(c, P, cs, nr, bk, j, inv, c1, v, loc);
    cluster_sum<G>(c, loc, bk - j - 1, tmp);
    for (int a = c.tid; a < bk - j - 1; a += kBT) v[j + 1 + a] = tmp[a];
    __syncthreads();
  }
  return true;
}

// Trailing update of one panel on this CTA's rows, in chunks of kWC columns:
//   S = Qbar^T B over this CTA's rows: stages of kKT rows of B and of Qbar stream in through
//       a cp.async pipeline as deep as the shared-memory pool allows (up to kMaxStages),
//       two stages per CTA barrier; each thread accumulates a 4 x 4 tile of S over a K-split
//       share of four-row groups;
//   Rbar = cluster sum of S (fixed order);  R[kb.., col] = Rbar (rank 0);
//   B -= Qbar Rbar: the same stages stream in again, each thread updates four rows x two
//       columns and stores them straight to global memory.
// Qbar: P (global, rows [0, nr) of the slice, stride cs); B: Qs + col * ldq.
template <int G>
__device__ void b_update(BCtx<G>& c, const float* P, int64_t cs, int nr, int bk, float* Qs,
                         int64_t ldq, int64_t col_begin, int64_t col_end, float* R, int64_t ldr,
                         int kb, int pool_floats) {
  float* pool = c.sm + c.L.pool;
  float* spart = pool;             // K-split partials after the K loop
  float* rbar = c.sm + c.L.rbar;   // [bk][kWC]
  const int sf = stage_floats(bk);
  int nst = pool_floats / sf;
  if (nst > kMaxStages) nst = kMaxStages;
  // two stages per CTA barrier when at least four fit (one otherwise); `depth` stages are in
  // flight ahead of the ones being consumed
  const int spb = nst >= 4 ? 2 : 1;
  const int depth = nst - spb;
  const int bkq = (bk + 3) / 4;
  const int tiles = bkq * (kWC / 4);
  int ks_n = kBT / tiles;
  if (ks_n > 8) ks_n = 8;
  if (ks_n < 1) ks_n = 1;
  const int t_id = c.tid % tiles, ks = c.tid / tiles;
  const bool active = c.tid < tiles * ks_n;
  // a thread's S tile: columns ai + x bkq of Qbar and ji + 16 y of B (x, y < 4); neighbouring
  // lanes read neighbouring staged columns, so the 16-byte shared loads do not conflict
  const int ai = t_id % bkq, ji = t_id / bkq;
  const int nkt = (nr + kKT - 1) / kKT;
  const uint32_t pool_u = s_addr(pool);
  // GEMM2 thread layout: rows 4*rq4 .. +3 of a stage, columns 2*cp, 2*cp+1
  const int rq4 = c.tid % (kKT / 4), cp = c.tid / (kKT / 4);
  for (int64_t c0 = col_begin; c0 < col_end; c0 += kWC) {
    const int wc = (int)((col_end - c0) < kWC ? (col_end - c0) : kWC);
    // stage t: B rows [r0, r0 + kKT) x columns [c0, c0 + kWC), then Qbar rows [r0, r0 + kKT) x
    // columns [0, bk), as 16-byte pieces (four rows of one column); rows >= nr and columns
    // beyond the block are zero-filled.  One commit group per stage (empty past the end).
    auto issue = [&](int t) {
      if (t < nkt) {
        const uint32_t base = pool_u + 4u * (uint32_t)((t % nst) * sf);
        const int r0 = t * kKT;
        for (int e = c.tid; e < (kWC + bkq * 4) * (kKT / 4); e += kBT) {
          const int q4 = e % (kKT / 4), j = e / (kKT / 4);
          const int r = r0 + 4 * q4;
          const bool isB = j < kWC;
          const int col = isB ? j : j - kWC;
          const bool ok = (isB ? col < wc : col < bk) && r < nr;
          const int nb = ok ? ((nr - r) >= 4 ? 16 : 4 * (nr - r)) : 0;
          const float* src = isB ? Qs + (ok ? r : 0) + (c0 + (ok ? col : 0)) * ldq
                                 : P + (ok ? r : 0) + (ok ? col : 0) * cs;
          cp_async16(base + 4u * (uint32_t)(j * kLDS + 4 * q4), src, nb);
        }
      }
      cp_commit();
    };
    auto stage = [&](int t) { return pool + (t % nst) * sf; };
    // ---------------------------------------------------------------- S = Qbar^T B
    float acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
    __syncthreads();  // the previous readers of the pool are done
    // one stage of S: this thread's 4 x 4 tile over its K-split share of the four-row groups
    auto s_stage = [&](int t) {
      const int r0 = t * kKT;
      const int kr = (nr - r0) < kKT ? (nr - r0) : kKT;
      const int ng = (kr + 3) / 4;
      if (active) {
        const float* Bt = stage(t);
        const float* At = Bt + kWC * kLDS;
        for (int g4 = ks; g4 < ng; g4 += ks_n) {
          const int rr = 4 * g4;
          float4 qv[4], bv[4];
#pragma unroll
          for (int x = 0; x < 4; ++x)
            qv[x] = (ai + x * bkq < bk) ? *reinterpret_cast<const float4*>(At + (ai + x * bkq) * kLDS + rr)
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int y = 0; y < 4; ++y)
            bv[y] = *reinterpret_cast<const float4*>(Bt + (ji + 16 * y) * kLDS + rr);
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) {
              float a = acc[x][y];
              a = fmaf(qv[x].x, bv[y].x, a);
              a = fmaf(qv[x].y, bv[y].y, a);
              a = fmaf(qv[x].z, bv[y].z, a);
              a = fmaf(qv[x].w, bv[y].w, a);
              acc[x][y] = a;
            }
        }
      }
    };
    for (int t = 0; t < depth; ++t) issue(t);
    for (int t = 0; t < nkt; t += spb) {
      ph_mark(PH_SPROD);
      cp_wait_dyn(depth - spb);
      __syncthreads();
      ph_mark(PH_SPROD_WAIT);
      for (int u = 0; u < spb; ++u) issue(t + depth + u);
      for (int u = 0; u < spb; ++u)
        if (t + u < nkt) s_stage(t + u);
    }
    cp_wait<0>();
    __syncthreads();
    ph_mark(PH_SPROD);
    // K-split partials -> spart[ks][a][j] (ld kWC), then a fixed-order sum
    if (active)
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y)
          if (ai + x * bkq < bk) spart[ks * (bkq * 4 * kWC) + (ai + x * bkq) * kWC + ji + 16 * y] = acc[x][y];
    __syncthreads();
    if (G == 1) {
      for (int e = c.tid; e < bk * kWC; e += kBT) {
        float sum = 0.f;
        for (int q = 0; q < ks_n; ++q) sum += spart[q * (bkq * 4 * kWC) + e];
        rbar[e] = sum;
      }
      __syncthreads();
    } else {
      float* mine = c.sm + c.L.cpart + (c.step & 1) * (kBMax * kWC);
      for (int e = c.tid; e < bk * kWC; e += kBT) {
        float sum = 0.f;
        for (int q = 0; q < ks_n; ++q) sum += spart[q * (bkq * 4 * kWC) + e];
        mine[e] = sum;
      }
      cl_sync();
      const uint32_t base = s_addr(mine);
      for (int e = c.tid; e < bk * kWC; e += kBT) {
        float sum = 0.f;
#pragma unroll
        for (int g = 0; g < G; ++g) sum += ld_cl(base + 4u * (uint32_t)e, (uint32_t)g);
        rbar[e] = sum;
      }
      ++c.step;
      __syncthreads();
    }
    if (c.rank == 0)
      for (int e = c.tid; e < bk * wc; e += kBT) {
        const int a = e / wc, j = e % wc;
        R[(kb + a) + (c0 + j) * ldr] = rbar[a * kWC + j];
      }
    ph_mark(PH_RBAR);
    // ---------------------------------------------------------------- B -= Qbar Rbar
    // one stage of the update: four rows x two columns of B per thread, stored to global
    auto u_stage = [&](int t) {
      const int r = t * kKT + 4 * rq4;
      const int j = 2 * cp;
      if (r < nr && j < wc) {
        const float* Bt = stage(t);
        const float* At = Bt + kWC * kLDS;
        float o[4][2];
#pragma unroll
        for (int x = 0; x < 4; ++x) o[x][0] = o[x][1] = 0.f;
        for (int a = 0; a < bk; ++a) {
          const float4 q = *reinterpret_cast<const float4*>(At + a * kLDS + 4 * rq4);
          const float2 rv = *reinterpret_cast<const float2*>(rbar + a * kWC + j);
          o[0][0] = fmaf(q.x, rv.x, o[0][0]); o[0][1] = fmaf(q.x, rv.y, o[0][1]);
          o[1][0] = fmaf(q.y, rv.x, o[1][0]); o[1][1] = fmaf(q.y, rv.y, o[1][1]);
          o[2][0] = fmaf(q.z, rv.x, o[2][0]); o[2][1] = fmaf(q.z, rv.y, o[2][1]);
          o[3][0] = fmaf(q.w, rv.x, o[3][0]); o[3][1] = fmaf(q.w, rv.y, o[3][1]);
        }
#pragma unroll
        for (int y = 0; y < 2; ++y) {
          if (j + y >= wc) break;
          const float4 b4 = *reinterpret_cast<const float4*>(Bt + (j + y) * kLDS + 4 * rq4);
          float* dst = Qs + r + (c0 + j + y) * ldq;
          if (r + 4 <= nr) {
            *reinterpret_cast<float4*>(dst) =
                make_float4(b4.x - o[0][y], b4.y - o[1][y], b4.z - o[2][y], b4.w - o[3][y]);
          } else {
            const float bb[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int x = 0; x < 4; ++x)
              if (r + x < nr) dst[x] = bb[x] - o[x][y];
          }
        }
      }
    };
    for (int t = 0; t < depth; ++t) issue(t);
    for (int t = 0; t < nkt; t += spb) {
      ph_mark(PH_UPDATE);
      cp_wait_dyn(depth - spb);
      __syncthreads();
      ph_mark(PH_UPDATE_WAIT);
      for (int u = 0; u < spb; ++u) issue(t + depth + u);
      for (int u = 0; u < spb; ++u)
        if (t + u < nkt) u_stage(t + u);
    }
    cp_wait<0>();
    ph_mark(PH_UPDATE);
  }
  __syncthreads();
}

// In-launch recovery of one instance (a6 + a7) by its cluster, at the start of its erasure
// panel: the listed tiles are poisoned (NaN), then every code with lost tiles is decoded.  The
// coefficient tables go in the panel pool, which is free between panels.  Cluster barriers
// order the poisoning before the decode and the decode before the next panel.
template <int G>
__device__ void b_recover(BCtx<G>& c, const BatchInst<float>& I, const BatchTile* __restrict__ tiles,
                          const BatchPlan* __restrict__ plans, const double* __restrict__ Gt,
                          const double* __restrict__ Gh) {
  const Geo& g = I.g;
  for (int e = I.tile0; e < I.tile0 + I.ntiles; ++e) {
    const BatchTile t = tiles[e];
    float* X = t.isR ? I.R : I.Q;
    const int64_t ld = t.isR ? g.ldr : g.ldq;
    const int64_t th = t.isR ? g.nb : g.mb, tw = g.nb;
    for (int64_t idx = (int64_t)c.rank * kBT + c.tid; idx < th * tw; idx += (int64_t)G * kBT) {
      const int64_t r = idx % th, s = idx / th;
      X[(int64_t)t.i * th + r + ((int64_t)t.j * tw + s) * ld] = nan_value<float>();
    }
  }
  if (G > 1) cl_sync(); else __syncthreads();
  DecodeScratch<float>& sh = *reinterpret_cast<DecodeScratch<float>*>(c.sm + ((c.L.pool + 3) & ~3));
  for (int pi = I.plan0; pi < I.plan0 + I.nplans; ++pi) {
    const DecodePlan& p = plans[pi].p;
    if (decode_setup<float>(g, p, Gt, Gh, sh, c.tid, kBT, I.status, c.rank == 0)) {
      const int64_t h = p.kind == 0 ? g.mb : g.nb;
      for (int64_t e = (int64_t)c.rank * kBT + c.tid; e < h * g.nb; e += (int64_t)G * kBT)
        decode_apply<float>(g, p, sh, I.Q, I.R, e % h, e / h);
    }
    __syncthreads();  // the next code's setup overwrites the tables
  }
  if (G > 1) cl_sync(); else __syncthreads();
}

template <int G>
__global__ void __launch_bounds__(kBT, 1) k_b_factor(BatchInst<float>* __restrict__ inst, int count,
                                                     const int* __restrict__ order,
                                                     const int* __restrict__ range, int* queue,
                                                     double tau2, int panel_cap,
                                                     const BatchTile* __restrict__ tiles,
                                                     const BatchPlan* __restrict__ plans,
                                                     const double* __restrict__ Gt,
                                                     const double* __restrict__ Gh,
                                                     unsigned long long* prof) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int s_item;
  BCtx<G> c;
  c.sm = smem;
  c.L = b_layout(G);
  c.tid = threadIdx.x;
  c.lane = threadIdx.x & 31;
  c.warp = threadIdx.x >> 5;
  c.rank = (G > 1) ? cl_rank() : 0;
  c.step = 0;
  ph_begin(prof);
  for (;;) {
    if (c.rank == 0 && c.tid == 0) s_item = atomicAdd(queue, 1);
    int item;
    if (G > 1) {
      cl_sync();
      item = ld_cl_i32(s_addr(&s_item), 0);
      cl_sync();  // rank 0 rewrites s_item only after every CTA has read it
    } else {
      __syncthreads();
      item = s_item;
      __syncthreads();
    }
    ph_mark(PH_OTHER);
    if (item >= count) break;
    const int idx = order[item];
    BatchInst<float>& I = inst[idx];
    const Geo g = I.g;
    const int pb = range[2 * idx], pe = range[2 * idx + 1];
    if (pb >= pe) continue;
    const int64_t rpc = ((g.M + G - 1) / G + 3) / 4 * 4;
    const int64_t row0 = (int64_t)c.rank * rpc;
    const int nr = (int)std::max<int64_t>(0, std::min<int64_t>(rpc, g.M - row0));
    float* Qs = I.Q + row0;
    bool ok = true;
    for (int k = pb; k < pe && ok; ++k) {
      if (k == I.rec_at - 1) {
        b_recover<G>(c, I, tiles, plans, Gt, Gh);
        ph_mark(PH_RECOVER);
      }
      const int kb = k * I.b;
      const int bk = (int)std::min<int64_t>(I.b, g.n - kb);
      // ICGS on the panel slice: in the shared-memory pool (after the panel's scratch) when it
      // fits, else in place in global memory (L2); the update then streams it from global
      float* Pg = Qs + (int64_t)kb * g.ldq;
      const int rpad = (nr + 3) / 4 * 4;
      const bool in_smem = rpad * bk <= panel_cap - kPanelScratch;
      float* P = in_smem ? smem + c.L.pool + kPanelScratch : Pg;
      const int64_t cs = in_smem ? rpad : g.ldq;
      if (in_smem) {
        for (int e = c.tid; e < rpad * bk; e += kBT) {
          const int r = e % rpad, a = e / rpad;
          P[e] = (r < nr) ? Pg[r + (int64_t)a * g.ldq] : 0.f;
        }
        __syncthreads();
      }
      if (nr <= 4 * kBT)
        ok = b_panel<G, 4>(c, P, cs, nr, bk, I.R, g.ldr, kb, tau2, I.status);
      else if (nr <= 8 * kBT)
        ok = b_panel<G, 8>(c, P, cs, nr, bk, I.R, g.ldr, kb, tau2, I.status);
      else
        ok = b_panel<G, 10>(c, P, cs, nr, bk, I.R, g.ldr, kb, tau2, I.status);
      if (!ok) break;
      if (in_smem)
        for (int e = c.tid; e < rpad * bk; e += kBT) {
          const int r = e % rpad, a = e / rpad;
          if (r < nr) Pg[r + (int64_t)a * g.ldq] = P[e];
        }
      __syncthreads();
      ph_mark(PH_PANEL);
      b_update<G>(c, Pg, g.ldq, nr, bk, Qs, g.ldq, kb + bk, g.N, I.R, g.ldr, kb, panel_cap);
    }
  }
  if (G > 1) cl_sync();  // peers may still read this CTA's shared memory
  ph_end();
}

template <int G>
cudaError_t launch_g(const BFactorLaunch& L, cudaStream_t st) {
  auto fn = k_b_factor<G>;
  const BLayout lay = b_layout(G);
  const size_t smem = ((size_t)lay.total + (size_t)L.panel_cap) * sizeof(float);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)L.grid);
  cfg.blockDim = dim3(kBT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = G;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = G > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, fn, L.inst, L.count, L.order, L.range, L.queue, L.tau2,
                            L.panel_cap, L.tiles, L.plans, L.Gt, L.Gh, L.prof);
}

template <int G>
int max_clusters_g(int panel_cap) {
  auto fn = k_b_factor<G>;
  const BLayout lay = b_layout(G);
  const size_t smem = ((size_t)lay.total + (size_t)panel_cap) * sizeof(float);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kBT);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = G;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace

int b_recover_floats() { return (int)((sizeof(DecodeScratch<float>) + sizeof(float) - 1) / sizeof(float)) + 4; }

int b_panel_cap_floats(int G) {
  const size_t cap = 227 * 1024 / sizeof(float) - 64;  // static shared and alignment slack
  return (int)(cap - (size_t)b_layout(G).total);
}

int b_max_clusters(int G, int panel_cap) {
  switch (G) {
    case 1: return max_clusters_g<1>(panel_cap);
    case 2: return max_clusters_g<2>(panel_cap);
    case 4: return max_clusters_g<4>(panel_cap);
    case 8: return max_clusters_g<8>(panel_cap);
    default: return 0;
  }
}

cudaError_t launch_b_factor(const BFactorLaunch& L, cudaStream_t st) {
  switch (L.G) {
    case 1: return launch_g<1>(L, st);
    case 2: return launch_g<2>(L, st);
    case 4: return launch_g<4>(L, st);
    case 8: return launch_g<8>(L, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cqr
