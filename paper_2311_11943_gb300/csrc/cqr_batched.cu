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
#include "cqr_device.cuh"

namespace cqr {

namespace {

constexpr int kBT = 512;        // threads per CTA
constexpr int kBW = kBT / 32;   // warps per CTA
constexpr int kKT = 32;         // rows per staged tile of the Rbar product

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

// Shared-memory layout (in floats), the same for every CTA of a launch.
struct BLayout {
  int small;   // v [kBMax], eta [kBMax], sv [kBMax]
  int wpart;   // panel: warp partials [kBW][2 kBMax]; GEMM: K-split partials [8192]
  int stage;   // GEMM staging: As [kKT][kBMax + 4], Bs [kKT][kWC + 4]
  int cpart;   // cluster partials [2][kBMax kWC] (G > 1)
  int rbar;    // Rbar chunk [kBMax][kWC]
  int panel;   // panel slice
  int total;   // floats before the panel slice
};

__host__ __device__ inline BLayout b_layout(int G) {
  BLayout L;
  L.small = 0;
  L.wpart = 3 * kBMax;
  L.stage = L.wpart + 8192;
  L.cpart = L.stage + kKT * (kBMax + 4) + kKT * (kWC + 4);
  L.rbar = L.cpart + (G > 1 ? 2 * kBMax * kWC : 0);
  L.panel = L.rbar + kBMax * kWC;
  L.total = L.panel;
  return L;
}

template <int G>
struct BCtx {
  float* sm;
  BLayout L;
  int tid, lane, warp;
  uint32_t rank;
  unsigned step;  // reduction counter (same sequence on every CTA of the cluster)
};

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

// Column sums over the rows of this CTA's slice.  Values a in [0, nv): val(a, r) is the
// summand of row r.  Warps form a (column group) x (row group) grid that depends on nv only.
// The per-CTA result (warp partials summed in a fixed order) lands in loc[0 .. nv).
template <int G, typename F>
__device__ __forceinline__ void cta_colsums(BCtx<G>& c, int nv, int nr, float* loc, F val) {
  int cg = 1;
  while (cg * 2 <= nv && cg * 2 <= kBW) cg *= 2;
  const int rg = kBW / cg;
  const int cgi = c.warp % cg, rgi = c.warp / cg;
  float* wp = c.sm + c.L.wpart;  // [rg][nv]
  for (int a = cgi; a < nv; a += cg) {
    float s = 0.f;
    for (int r = rgi * 32 + c.lane; r < nr; r += 32 * rg) s += val(a, r);
    s = warp_sum(s);
    if (c.lane == 0) wp[rgi * nv + a] = s;
  }
  __syncthreads();
  for (int a = c.tid; a < nv; a += kBT) {
    float s = 0.f;
    for (int q = 0; q < rg; ++q) s += wp[q * nv + a];
    loc[a] = s;
  }
}

// One panel: columns kb .. kb+bk-1 of the instance, this CTA's rows [0, nr) of the slice at
// P (column stride cs).  Writes R's diagonal block (rank 0).  Returns false on breakdown.
template <int G>
__device__ bool b_panel(BCtx<G>& c, float* P, int64_t cs, int nr, int bk, float* R, int64_t ldr,
                        int kb, double tau2, int* status) {
  float* v = c.sm + c.L.small;
  float* eta = v + kBMax;
  float* sv = eta + kBMax;
  float* loc = c.sm + c.L.stage;  // scratch for per-CTA sums (the GEMM staging is idle here)
  // step 0: v_a = p_a^T p_0 and eta_a = p_a^T p_a
  cta_colsums<G>(c, 2 * bk, nr, loc, [&](int a, int r) {
    if (a < bk) return P[r + a * cs] * P[r];
    const float x = P[r + (a - bk) * cs];
    return x * x;
  });
  {
    float* tmp = c.sm + c.L.rbar;
    cluster_sum<G>(c, loc, 2 * bk, tmp);
    for (int a = c.tid; a < bk; a += kBT) {
      v[a] = tmp[a];
      eta[a] = tmp[bk + a];
    }
    __syncthreads();
  }
  for (int j = 0; j < bk; ++j) {
    if (j > 0 && tau2 > 0.0 && (double)v[j] < tau2 * (double)eta[j]) {
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
      float* tmp = c.sm + c.L.rbar;
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
    // p_a -= q_j R[j, a] for a >= j+2 (stored) and v'_a = p_a^T p'_{j+1} for a >= j+1, with
    // q_j = p_j / r_jj and p'_{j+1} = p_{j+1} - q_j R[j, j+1] formed on the fly
    cta_colsums<G>(c, bk - j - 1, nr, loc, [&](int a1, int r) {
      const float q = P[r + j * cs] * inv;
      const float p1 = fmaf(-q, c1, P[r + (j + 1) * cs]);
      if (a1 == 0) return p1 * p1;
      const int a = j + 1 + a1;
      const float x = fmaf(-q, v[a] * inv, P[r + a * cs]);
      P[r + a * cs] = x;
      return x * p1;
    });
    // every read of columns j, j+1 is done: publish q_j and p'_{j+1}
    for (int r = c.tid; r < nr; r += kBT) {
      const float q = P[r + j * cs] * inv;
      P[r + j * cs] = q;
      P[r + (j + 1) * cs] = fmaf(-q, c1, P[r + (j + 1) * cs]);
    }
    {
      float* tmp = c.sm + c.L.rbar;
      cluster_sum<G>(c, loc, bk - j - 1, tmp);
      for (int a = c.tid; a < bk - j - 1; a += kBT) v[j + 1 + a] = tmp[a];
      __syncthreads();
    }
  }
  return true;
}

// Trailing update of one panel on this CTA's rows, in chunks of kWC columns:
//   S = Qbar^T B (per CTA, K-split over 4x4 register tiles), Rbar = cluster sum of S,
//   R[kb.., col] = Rbar (rank 0), B -= Qbar Rbar.
// Qbar: P (rows [0, nr), stride cs); B: Qs + col * ldq (rows [0, nr) of the slice).
template <int G>
__device__ void b_update(BCtx<G>& c, const float* P, int64_t cs, int nr, int bk, float* Qs,
                         int64_t ldq, int64_t col_begin, int64_t col_end, float* R, int64_t ldr,
                         int kb) {
  float* spart = c.sm + c.L.wpart;
  float* As = c.sm + c.L.stage;              // [kKT][kBMax + 4]
  float* Bs = As + kKT * (kBMax + 4);        // [kKT][kWC + 4]
  float* rbar = c.sm + c.L.rbar;             // [bk][kWC]
  float* loc = spart;                        // per-CTA S after the K-split sum (first bk*kWC)
  const int bkq = (bk + 3) / 4;              // row quads of S
  const int tiles = bkq * (kWC / 4);
  const int ks_n = kBT / tiles >= 1 ? (kBT / tiles > 8 ? 8 : kBT / tiles) : 1;
  for (int64_t c0 = col_begin; c0 < col_end; c0 += kWC) {
    const int wc = (int)std::min<int64_t>(kWC, col_end - c0);
    // --- S = Qbar^T B over this CTA's rows
    const int t = c.tid % tiles, ks = c.tid / tiles;
    const bool active = ks < ks_n && c.tid < tiles * ks_n;
    const int a0 = (t % bkq) * 4, j0 = (t / bkq) * 4;
    float acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
    for (int r0 = 0; r0 < nr; r0 += kKT) {
      const int kr = (nr - r0) < kKT ? (nr - r0) : kKT;
      __syncthreads();
      for (int e = c.tid; e < kKT * kBMax; e += kBT) {
        const int rr = e % kKT, a = e / kKT;
        As[rr * (kBMax + 4) + a] = (rr < kr && a < bk) ? P[(r0 + rr) + a * cs] : 0.f;
      }
      for (int e = c.tid; e < kKT * kWC; e += kBT) {
        const int rr = e % kKT, j = e / kKT;
        Bs[rr * (kWC + 4) + j] = (rr < kr && j < wc) ? Qs[(r0 + rr) + (c0 + j) * ldq] : 0.f;
      }
      __syncthreads();
      if (active) {
        for (int rr = ks; rr < kr; rr += ks_n) {
          const float4 av = *reinterpret_cast<const float4*>(As + rr * (kBMax + 4) + a0);
          const float4 bv = *reinterpret_cast<const float4*>(Bs + rr * (kWC + 4) + j0);
          const float ax[4] = {av.x, av.y, av.z, av.w};
          const float bx[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(ax[x], bx[y], acc[x][y]);
        }
      }
    }
    __syncthreads();
    // K-split partials -> spart[ks][a][j] (ld kWC), then a fixed-order sum into loc
    if (active)
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) spart[ks * (bkq * 4 * kWC) + (a0 + x) * kWC + j0 + y] = acc[x][y];
    __syncthreads();
    float sum_local[8];
    int nloc = 0;
    for (int e = c.tid; e < bk * kWC; e += kBT) {
      float s = 0.f;
      for (int q = 0; q < ks_n; ++q) s += spart[q * (bkq * 4 * kWC) + e];
      sum_local[nloc++] = s;
    }
    __syncthreads();
    nloc = 0;
    for (int e = c.tid; e < bk * kWC; e += kBT) loc[e] = sum_local[nloc++];
    cluster_sum<G>(c, loc, bk * kWC, rbar);
    if (c.rank == 0)
      for (int e = c.tid; e < bk * wc; e += kBT) {
        const int a = e / wc, j = e % wc;
        R[(kb + a) + (c0 + j) * ldr] = rbar[a * kWC + j];
      }
    // --- B -= Qbar Rbar on this CTA's rows (4 rows x 4 columns per thread and step)
    const int rq = (nr + 3) / 4;
    for (int e = c.tid; e < rq * (kWC / 4); e += kBT) {
      const int r = (e % rq) * 4, j = (e / rq) * 4;
      if (j >= wc) continue;
      float o[4][4];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) o[x][y] = 0.f;
      for (int a = 0; a < bk; ++a) {
        float q[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) q[x] = (r + x < nr) ? P[(r + x) + a * cs] : 0.f;
        const float4 rv = *reinterpret_cast<const float4*>(rbar + a * kWC + j);
        const float rr4[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) o[x][y] = fmaf(q[x], rr4[y], o[x][y]);
      }
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        if (j + y >= wc) break;
        float* bc = Qs + (c0 + j + y) * ldq;
#pragma unroll
        for (int x = 0; x < 4; ++x)
          if (r + x < nr) bc[r + x] -= o[x][y];
      }
    }
  }
  __syncthreads();
}

template <int G>
__global__ void __launch_bounds__(kBT, 1) k_b_factor(BatchInst<float>* __restrict__ inst, int count,
                                                     const int* __restrict__ order,
                                                     const int* __restrict__ range, int* queue,
                                                     double tau2, int panel_cap) {
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
    if (item >= count) break;
    const int idx = order[item];
    BatchInst<float>& I = inst[idx];
    const Geo g = I.g;
    const int pb = range[2 * idx], pe = range[2 * idx + 1];
    if (pb >= pe) continue;
    const int64_t rpc = ((g.M + G - 1) / G + 3) / 4 * 4;
    const int64_t row0 = (int64_t)c.rank * rpc;
    const int nr = (int)std::max<int64_t>(0, std::min<int64_t>(rpc, g.M - row0));
    const int rpad = (nr + 3) / 4 * 4;
    float* Qs = I.Q + row0;
    bool ok = true;
    for (int k = pb; k < pe && ok; ++k) {
      const int kb = k * I.b;
      const int bk = (int)std::min<int64_t>(I.b, g.n - kb);
      const bool in_smem = (int64_t)rpad * bk <= panel_cap;
      float* P;
      int64_t cs;
      if (in_smem) {
        P = smem + c.L.panel;
        cs = rpad;
        for (int e = c.tid; e < rpad * bk; e += kBT) {
          const int r = e % rpad, a = e / rpad;
          P[e] = (r < nr) ? Qs[r + (int64_t)(kb + a) * g.ldq] : 0.f;
        }
        __syncthreads();
      } else {
        P = Qs + (int64_t)kb * g.ldq;
        cs = g.ldq;
      }
      ok = b_panel<G>(c, P, cs, nr, bk, I.R, g.ldr, kb, tau2, I.status);
      if (!ok) break;
      if (in_smem) {
        for (int e = c.tid; e < rpad * bk; e += kBT) {
          const int r = e % rpad, a = e / rpad;
          if (r < nr) Qs[r + (int64_t)(kb + a) * g.ldq] = P[e];
        }
      }
      __syncthreads();
      b_update<G>(c, P, cs, nr, bk, Qs, g.ldq, kb + bk, g.N, I.R, g.ldr, kb);
    }
  }
  if (G > 1) cl_sync();  // peers may still read this CTA's shared memory
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
                            L.panel_cap);
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
