// cqr_panel.cu -- panel factorisation of PBMGS (a3): ICGS on one block column of the
// encoded matrix, all M = m_pad + c rows, on G CTAs that each own a contiguous slice of rows.
//
// Appendix A, Algorithm CGS (one reduction per column, right-looking) with the ICGS
// reorthogonalisation.  Per column j, with v_a = p_a^T p_j (a >= j) already reduced:
//   if j > 0 and v_j < tau^2 eta_j:   reorthogonalise p_j against columns < j (two more
//                                      reductions), add the coefficients to R, recompute v
//   r_jj = sqrt(v_j), q_j = p_j / r_jj, R[j, a] = v_a / r_jj,
//   p_a -= q_j R[j, a] for a > j                  -- fused with the next column's products
//   v'_a = p_a^T p_{j+1} for a > j                  (p_{j+1} updated first, in registers)
// eta_j are the squared column norms at the panel start (reduced together with v for j = 0).
//
// Reductions are deterministic: every CTA sums the G per-CTA partials in the same order.
// Two synchronisation variants:
//   cluster: G <= 16 CTAs form one thread-block cluster; partials live in shared memory and
//            are read through distributed shared memory after a hardware cluster barrier;
//   grid:    G <= #SMs CTAs in a cooperative launch; partials go through global memory
//            (L2) and a release/acquire counter barrier with a bounded wait.
#include <math.h>
#include <stdlib.h>

#include "cqr_device.cuh"
#include "cqr_kernels.cuh"

namespace cqr {

namespace {

constexpr int kNT = 512;
constexpr int kNW = kNT / 32;
constexpr size_t kSmemCap = 227 * 1024;
constexpr int kMaxCluster = 16;
// Two-level exchange of the grid variant: clusters of kHierCS (or kHierCSWide) CTAs, used for
// FP32 panels
// that need more than kHierMinG CTAs.
constexpr int kHierCS = 8;
constexpr int kHierCSWide = 16;  // non-portable cluster size
constexpr int kHierMinG = 48;

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t map_peer(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ float ld_peer(uint32_t addr, float) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ double ld_peer(uint32_t addr, double) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}

// Release/acquire grid barrier for a cooperative launch.  bar is zeroed before the launch.
// Thread 0 arrives with a release add (ordered after the CTA barrier, hence after every
// thread's prior writes) and polls with acquire loads; the wait is bounded.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned& target,
                                             int* status, int site, long long limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    target += nblocks;
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(bar), "r"(1u) : "memory");
    int ok = 1;
    const long long t0 = clock64();
    while (ld_acquire_u32(bar) < target) {
      if (ld_relaxed_i32(status + ST_CODE) == CQR_ETIMEOUT) { ok = 0; break; }
      if (clock64() - t0 > limit) {
        set_status(status, CQR_ETIMEOUT, site);
        status[ST_SITE] = site;
        ok = 0;
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// t rounded towards +infinity to T (the FP32 threshold of the ICGS test; exact for double)
template <typename T>
__device__ __forceinline__ T round_up_to(double t);
template <>
__device__ __forceinline__ float round_up_to<float>(double t) { return __double2float_ru(t); }
template <>
__device__ __forceinline__ double round_up_to<double>(double t) { return t; }

template <typename T>
struct Ctx {
  T* base;       // slice, column 0, first row of this CTA
  int64_t cs;    // column stride of the slice
  int nr;        // rows owned
  int pld;       // padded panel width
  T* gpart;      // grid variant: [2][G][2*pld]; two-level: [G][2*pld] (first reduction) then
                 // [2][clusters][2*pld] cluster sums
  T* lpart;      // cluster and two-level variants: this CTA's [2][2*pld] in shared memory
  T* red;        // grid variant: shared [8][2*pld] scratch
  T* rbuf;       // two-level, cluster leader: receive buffer [hcs][pld] (one buffer: a CTA
                 // sends step s + 1 only after it has read its leader's sums of step s, which
                 // the leader writes after reading the buffer)
  uint64_t* mbar;  // two-level: [2] mbarriers of rbuf (used in the leader)
  unsigned* bar;
  int* status;
  unsigned target;
  unsigned phases;   // two-level: bit p = phase parity of mbar[p]
  int crank, cl, ncl;  // two-level: rank in the cluster, cluster index, clusters
  int hcs;             // two-level: CTAs per cluster
  long long wait_limit;  // bound of each wait on other CTAs, SM cycles
};

// SMP: the partial vectors live in shared memory (cluster and two-level variants)
template <typename T, bool SMP>
__device__ __forceinline__ void put_partial(const Ctx<T>& c, int idx, T val, int step) {
  if (SMP)
    c.lpart[(step & 1) * 2 * c.pld + idx] = val;
  else
    c.gpart[((size_t)(step & 1) * gridDim.x + blockIdx.x) * 2 * c.pld + idx] = val;
}

// out[a] = sum over r < rows of P[r * stride + a] for lo <= a < hi, with P in global memory
// (L2).  Each entry is summed by gr adjacent lanes (rows gr apart, four loads in flight) and
// combined by a butterfly over those lanes: a fixed order, the same in every CTA.  Every
// thread of the CTA must call it.
template <typename T>
__device__ __forceinline__ void reduce_rows(const T* P, int rows, size_t stride, int lo, int hi,
                                            T* out) {
  const int n = hi - lo, tid = threadIdx.x;
  if (n <= 0) return;
  int gr = 1;
  while (gr < 8 && gr * 2 * n <= kNT && gr * 2 <= rows) gr *= 2;
  const int total = n * gr;
  for (int base = 0; base < total; base += kNT) {
    const int idx = base + tid;
    const int e = idx / gr, m = idx - e * gr;
    T acc = T(0);
    if (idx < total) {
      const int a = lo + e;
      int r = m;
      for (; r + 3 * gr < rows; r += 4 * gr) {
        const T x0 = __ldcg(P + (size_t)r * stride + a);
        const T x1 = __ldcg(P + (size_t)(r + gr) * stride + a);
        const T x2 = __ldcg(P + (size_t)(r + 2 * gr) * stride + a);
        const T x3 = __ldcg(P + (size_t)(r + 3 * gr) * stride + a);
        acc += x0; acc += x1; acc += x2; acc += x3;
      }
      for (; r < rows; r += gr) acc += __ldcg(P + (size_t)r * stride + a);
    }
    for (int o = 1; o < gr; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (idx < total && m == 0) out[lo + e] = acc;
  }
}

struct NoHook {
  __device__ void operator()() const {}
};

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// out[a] = sum over r < rows of the FP32 values of tagged words P[r * stride + a] (value in the
// low half, `tag` in the high half) for lo <= a < hi, each word polled (bounded) until it
// carries the tag: a word is written whole by one aligned 64-bit store, so a matching tag
// certifies its value, and no separate flag or barrier is needed.  Summation as in
// reduce_rows (gr adjacent lanes, rows gr apart, then a butterfly): a fixed order.  Every
// thread of the CTA must call it; returns false (the same in every thread) when a wait ran
// out or another CTA recorded an error.
__device__ __forceinline__ bool reduce_tagged(const unsigned long long* P, int rows, size_t stride,
                                              int lo, int hi, unsigned tag, float* out, int* status,
                                              int site, long long limit) {
  const int n = hi - lo, tid = threadIdx.x;
  bool ok = true;
  if (n > 0) {
    int gr = 1;
    while (gr < 8 && gr * 2 * n <= kNT && gr * 2 <= rows) gr *= 2;
    const int total = n * gr;
    for (int base = 0; base < total; base += kNT) {
      const int idx = base + tid;
      const int e = idx / gr, m = idx - e * gr;
      float acc = 0.f;
      if (idx < total && ok) {
        const int a = lo + e;
        for (int r0 = m; r0 < rows && ok; r0 += 4 * gr) {
          unsigned long long x[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = r0 + u * gr;
            x[u] = r < rows ? ld_relaxed_u64(P + (size_t)r * stride + a) : 0ull;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = r0 + u * gr;
            if (r >= rows || !ok) continue;
            if ((unsigned)(x[u] >> 32) != tag) {
              const long long t0 = clock64();
              unsigned spins = 0u;
              do {
                x[u] = ld_relaxed_u64(P + (size_t)r * stride + a);
                const long long el = clock64() - t0;
                if (el > limit) {
                  set_status(status, CQR_ETIMEOUT, site);
                  ok = false;
                  break;
                }
                if (el > kPollAfterCycles && (++spins & 63u) == 0u &&
                    ld_relaxed_i32(status + ST_CODE) != 0) {
                  ok = false;
                  break;
                }
              } while ((unsigned)(x[u] >> 32) != tag);
            }
            if (ok) acc += __uint_as_float((unsigned)x[u]);
          }
        }
      }
      for (int o = 1; o < gr; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (idx < total && m == 0) out[lo + e] = acc;
    }
  }
  return __syncthreads_and(ok) != 0;
}

// Synchronise and reduce entries [lo, hi) of the partial vectors into out[].  `hook` runs
// right after the barrier, when every thread of this CTA has finished the step's reads.
// HIER (two-level, FP32): the CTAs of each cluster push their partials (16-byte st.async) into
// the leader's receive buffer; the leader sums them in rank order and writes the cluster sum
// to global memory as tagged words; every CTA polls the words of all clusters and sums them
// in cluster order.  The first reduction (v and eta, wider than one buffer row)
// goes through global memory from every CTA, as in the grid variant.
template <typename T, bool CL, bool HIER = false, typename Hook = NoHook>
__device__ __forceinline__ bool sync_reduce(Ctx<T>& c, int lo, int hi, T* out, int step, int site,
                                            Hook hook = Hook()) {
  const int G = gridDim.x, tid = threadIdx.x;
  if constexpr (HIER) {
    const int par = step & 1;
    if (hi <= c.pld) {
      const int c0 = lo / 4, c1 = (hi + 3) / 4;
      __syncthreads();  // this CTA's partials are complete; no thread reads the step's columns
      hook();
      const uint32_t lead_buf =
          map_peer(smem_addr(c.rbuf + (size_t)c.crank * c.pld), 0);
      const uint32_t lead_bar = map_peer(smem_addr(c.mbar + par), 0);
      if (c.crank == 0 && tid == 0) mbar_expect(c.mbar + par, (unsigned)(c.hcs * (c1 - c0) * 16));
      for (int ch = c0 + tid; ch < c1; ch += kNT)
        st_async4(lead_buf + 16u * ch,
                  *reinterpret_cast<const float4*>(c.lpart + par * 2 * c.pld + 4 * ch), lead_bar);
      if (c.crank == 0) {
        const bool ok = mbar_wait_bounded(c.mbar + par, (c.phases >> par) & 1u, c.wait_limit,
                                          c.status, site);
        c.phases ^= 1u << par;
        if (!__syncthreads_and(ok)) return false;
        // cluster sums as tagged words (value, step + 1): rows G + par ncl + cl of the partial
        // buffer, each row 2 pld floats = pld words (rows below G hold the first reduction's
        // per-CTA partials, which slower CTAs may still be reading); cleared before the launch
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(
            c.gpart + ((size_t)G + par * c.ncl + c.cl) * 2 * c.pld);
        const unsigned long long tag = (unsigned long long)(step + 1) << 32;
        for (int a = lo + tid; a < hi; a += kNT) {
          float sum = 0.f;
#pragma unroll
          for (int k = 0; k < c.hcs; ++k) sum += (float)c.rbuf[(size_t)k * c.pld + a];
          st_relaxed_u64(dst + a, tag | __float_as_uint(sum));
        }
      }
      const bool ok = reduce_tagged(
          reinterpret_cast<const unsigned long long*>(c.gpart + ((size_t)G + par * c.ncl) * 2 * c.pld),
          c.ncl, (size_t)c.pld, lo, hi, (unsigned)(step + 1), reinterpret_cast<float*>(out),
          c.status, site, c.wait_limit);
      return ok;
    }
    __syncthreads();
    T* dst = c.gpart + ((size_t)par * G + blockIdx.x) * 2 * c.pld;
    for (int a = lo + tid; a < hi; a += kNT) dst[a] = c.lpart[par * 2 * c.pld + a];
    if (!grid_barrier(c.bar, G, c.target, c.status, site, c.wait_limit)) return false;
    hook();
    reduce_rows(c.gpart + (size_t)par * G * 2 * c.pld, G, (size_t)2 * c.pld, lo, hi, out);
    __syncthreads();
    return true;
  }
  if (CL) {
    cluster_sync_all();
    hook();
    const uint32_t base = smem_addr(c.lpart + (step & 1) * 2 * c.pld);
    for (int a = lo + tid; a < hi; a += kNT) {
      T x[kMaxCluster];
#pragma unroll
      for (int g = 0; g < kMaxCluster; ++g)
        x[g] = (g < G) ? ld_peer(map_peer(base + a * (uint32_t)sizeof(T), g), T(0)) : T(0);
      T s = T(0);
#pragma unroll
      for (int g = 0; g < kMaxCluster; ++g) s += x[g];
      out[a] = s;
    }
    __syncthreads();
    return true;
  }
  if (!grid_barrier(c.bar, G, c.target, c.status, site, c.wait_limit)) return false;
  hook();
  const T* P = c.gpart + (size_t)(step & 1) * G * 2 * c.pld;
  const int n = hi - lo;
  if (n <= 0) {
    __syncthreads();
    return true;
  }
  // `groups` threads share one entry; group k sums partial rows k, k+groups, ...
  int groups = kNT / n;
  if (groups > 8) groups = 8;
  if (groups > G) groups = G;
  if (groups < 1) groups = 1;
  for (int idx = tid; idx < n * groups; idx += kNT) {
    const int grp = idx / n, a = lo + idx - grp * n;
    T acc = T(0);
    int g = grp;
    for (; g + 3 * groups < G; g += 4 * groups) {
      const T x0 = __ldcg(P + (size_t)g * 2 * c.pld + a);
      const T x1 = __ldcg(P + (size_t)(g + groups) * 2 * c.pld + a);
      const T x2 = __ldcg(P + (size_t)(g + 2 * groups) * 2 * c.pld + a);
      const T x3 = __ldcg(P + (size_t)(g + 3 * groups) * 2 * c.pld + a);
      acc += x0; acc += x1; acc += x2; acc += x3;
    }
    for (; g < G; g += groups) acc += __ldcg(P + (size_t)g * 2 * c.pld + a);
    c.red[grp * 2 * c.pld + a] = acc;
  }
  __syncthreads();
  for (int k = lo + tid; k < hi; k += kNT) {
    T s = T(0);
    for (int q = 0; q < groups; ++q) s += c.red[q * 2 * c.pld + k];
    out[k] = s;
  }
  __syncthreads();
  return true;
}

// Lane-local access to the slice.  VW = 2 (FP32 in shared memory): a lane owns row pairs
// r = 64 i + 2 lane + {0, 1} and works on them with 64-bit loads and packed f32x2 FMAs;
// VW = 1: rows r = 32 i + lane.  With the slice in shared memory the CTA's rows are padded
// with zeros to exactly 32 RPL, so no row guard is needed.
// Packed FP32 pair held in one 64-bit register (low half = even row).
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

template <typename T, int VW>
struct LaneOps;

template <>
struct LaneOps<float, 2> {
  using V = uint64_t;
  __device__ static int row(int i, int lane) { return 64 * i + 2 * lane; }
  __device__ static V ld(const float* p) { return *reinterpret_cast<const unsigned long long*>(p); }
  __device__ static void st(float* p, V v) { *reinterpret_cast<unsigned long long*>(p) = v; }
  __device__ static V fma(V a, V b, V c) { return ffma2(a, b, c); }
  __device__ static V splat(float s) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(s));
    return r;
  }
  __device__ static V zero() { return 0ull; }
  __device__ static V scale(V a, float s) { return ffma2(a, splat(s), 0ull); }
  __device__ static float sum(V v) {
    float x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
    return x + y;
  }
};

template <typename T>
struct LaneOps<T, 1> {
  using V = T;
  __device__ static int row(int i, int lane) { return 32 * i + lane; }
  __device__ static V ld(const T* p) { return *p; }
  __device__ static void st(T* p, V v) { *p = v; }
  __device__ static V fma(V a, V b, V c) { return a * b + c; }
  __device__ static V splat(T s) { return s; }
  __device__ static V zero() { return T(0); }
  __device__ static V scale(V a, T s) { return a * s; }
  __device__ static T sum(V v) { return v; }
};

template <typename T, int RPL, bool CL, bool SMEM, bool HIER>
__global__ void __launch_bounds__(kNT, 1) k_panel(T* __restrict__ Q, int64_t ldq, T* __restrict__ R,
                                                   int64_t ldr, int64_t M, int bk, int rpc,
                                                   int rpc_pad, double tau2, T* gpart,
                                                   unsigned* bar, int* status, int col0,
                                                   long long wait_limit) {
  constexpr int VW = (SMEM && sizeof(T) == 4 && RPL % 2 == 0) ? 2 : 1;
  constexpr int NV = RPL / VW;  // vectors per lane
  using L = LaneOps<T, VW>;
  using V = typename L::V;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int g = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  // the slices and R rows stay inside their buffers (the same for every CTA: before any
  // barrier)
  CQR_CHECK(ldq >= M && ldr >= bk && rpc == 32 * RPL && rpc_pad >= rpc &&
                (int64_t)gridDim.x * rpc >= M, 201);
  const int pld = (bk + 3) / 4 * 4;
  const int64_t row0 = (int64_t)g * rpc;
  const int nr = (int)((M - row0) < rpc ? (M - row0) : rpc);
  T* sm = reinterpret_cast<T*>(smraw);
  T* small = sm + (SMEM ? (size_t)bk * rpc_pad : 0);
  T* v = small;          // [2 pld]: v, and eta in the second half (first reduction)
  T* eta = v + pld;
  T* sv = v + 2 * pld;
  Ctx<T> c;
  c.base = SMEM ? sm : Q + row0;
  c.cs = SMEM ? rpc_pad : ldq;
  c.nr = nr;
  c.pld = pld;
  c.gpart = gpart;
  c.red = sv + 2 * pld;
  c.lpart = c.red + (CL ? 0 : 8 * 2 * pld);
  c.rbuf = c.red;
  c.mbar = reinterpret_cast<uint64_t*>(c.lpart + 4 * pld);
  c.bar = bar;
  c.status = status;
  c.target = 0;
  c.phases = 0u;
  c.hcs = kHierCS;
  if (HIER) {
    unsigned ncta;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(ncta));
    c.hcs = (int)ncta;
  }
  c.crank = g % c.hcs;
  c.cl = g / c.hcs;
  c.ncl = gridDim.x / c.hcs;
  c.wait_limit = wait_limit;
  int step = 0;
  auto ok_row = [&](int r) { return SMEM ? true : (r < nr); };
  // leaving after an abandoned exchange: the two-level variant first meets the rest of its
  // cluster (whose stores into the leader's shared memory were all issued before it arrived)
  // and leaves them time to land
  auto leave = [&]() {
    if (HIER) {
      cluster_sync_all();
      const long long t0 = clock64();
      while (clock64() - t0 < kDrainCycles) {
      }
    }
  };
  if (HIER) {
    // the exchange addresses rank 0 of a cluster of 8 or 16 CTAs: a launch of any other shape
    // (the same for every CTA) records an error and leaves before touching another CTA
    unsigned ncta;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(ncta));
    if ((ncta != (unsigned)kHierCS && ncta != (unsigned)kHierCSWide) || gridDim.x % ncta != 0) {
      if (g == 0 && tid == 0) set_status(status, CQR_ECUDA, 50);
      return;
    }
    if (tid == 0) {
      mbar_init(c.mbar, 1);
      mbar_init(c.mbar + 1, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cluster_sync_all();  // the leader's mbarriers are initialised before any CTA sends
  }

  if (SMEM)
    for (int a = 0; a < bk; ++a)
      for (int r = tid; r < rpc; r += kNT)
        sm[(size_t)a * rpc_pad + r] = (r < nr) ? Q[row0 + r + a * ldq] : T(0);
  __syncthreads();

  V q[NV], pn[NV];
  // step 0: v_a = p_a^T p_0 and eta_a = p_a^T p_a
  {
    const T* p0 = c.base;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const int r = L::row(i, lane);
      pn[i] = ok_row(r) ? L::ld(p0 + r) : L::zero();
    }
    for (int a = warp; a < bk; a += kNW) {
      const T* pa = c.base + a * c.cs;
      V d0 = L::zero(), d1 = L::zero();
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const int r = L::row(i, lane);
        if (ok_row(r)) {
          const V x = L::ld(pa + r);
          d0 = L::fma(x, pn[i], d0);
          d1 = L::fma(x, x, d1);
        }
      }
      T s0 = warp_sum(L::sum(d0)), s1 = warp_sum(L::sum(d1));
      if (lane == 0) {
        put_partial<T, CL || HIER>(c, a, s0, step);
        put_partial<T, CL || HIER>(c, pld + a, s1, step);
      }
    }
    if (!sync_reduce<T, CL, HIER>(c, 0, 2 * pld, v, step++, 1)) { leave(); return; }
  }
  // The ICGS test of column j, v_j < tau^2 eta_j with the product in FP64, is taken in T
  // against eta_j replaced by the FP64 product rounded up to T: for a T value v and a double
  // t, (double)v < t exactly when v < t rounded up to T, so the decision is the same, with
  // one FP64 product per column and CTA instead of one per thread and column.  The first
  // use (j = 1) comes after the next reduction's barriers.
  const bool icgs = tau2 > 0.0;
  if (icgs)
    for (int a = tid; a < bk; a += kNT) eta[a] = round_up_to<T>(tau2 * (double)eta[a]);

  for (int j = 0; j < bk; ++j) {
    if (j > 0 && icgs && v[j] < eta[j]) {
      // ICGS: one more projection of p_j on the computed columns 0 .. j-1
      const T* pj = c.base + j * c.cs;
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const int r = L::row(i, lane);
        pn[i] = ok_row(r) ? L::ld(pj + r) : L::zero();
      }
      for (int a = warp; a < j; a += kNW) {
        const T* pa = c.base + a * c.cs;
        V d = L::zero();
#pragma unroll
        for (int i = 0; i < NV; ++i) {
          const int r = L::row(i, lane);
          if (ok_row(r)) d = L::fma(L::ld(pa + r), pn[i], d);
        }
        const T s0 = warp_sum(L::sum(d));
        if (lane == 0) put_partial<T, CL || HIER>(c, a, s0, step);
      }
      if (!sync_reduce<T, CL, HIER>(c, 0, j, sv, step++, 3)) { leave(); return; }
      T* pjw = c.base + j * c.cs;
      for (int r = tid; r < (SMEM ? rpc : nr); r += kNT) {
        T acc = pjw[r];
        for (int a = 0; a < j; ++a) acc -= c.base[a * c.cs + r] * sv[a];
        pjw[r] = acc;
      }
      if (g == 0) {
        for (int a = tid; a < j; a += kNT) R[a + j * ldr] += sv[a];
        if (tid == 0) atomicAdd(status + ST_REORTH, 1);
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const int r = L::row(i, lane);
        pn[i] = ok_row(r) ? L::ld(pjw + r) : L::zero();
      }
      for (int a = j + warp; a < bk; a += kNW) {
        const T* pa = c.base + a * c.cs;
        V d = L::zero();
#pragma unroll
        for (int i = 0; i < NV; ++i) {
          const int r = L::row(i, lane);
          if (ok_row(r)) d = L::fma(L::ld(pa + r), pn[i], d);
        }
        const T s0 = warp_sum(L::sum(d));
        if (lane == 0) put_partial<T, CL || HIER>(c, a, s0, step);
      }
      if (!sync_reduce<T, CL, HIER>(c, j, bk, v, step++, 4)) { leave(); return; }
    }
    const T v0 = v[j];
    if (!(v0 > T(0)) || !isfinite(v0)) {
      if (g == 0 && tid == 0) set_status(status, CQR_EBREAKDOWN, col0 + j);
      if (CL || HIER) cluster_sync_all();
      return;
    }
    const T rjj = sqrt(v0);
    const T inv = T(1) / rjj;
    const bool nxt = (j + 1 < bk);
    const T cn = nxt ? v[j + 1] * inv : T(0);
    if (g == 0 && tid == 0) R[j + j * ldr] = rjj;
    // q_j and the updated p_{j+1} live in registers; warp 0 stores both to shared memory
    // right after the next barrier, when no warp of this CTA still reads columns j, j+1
    const T* pj = c.base + j * c.cs;
    const T* pj1 = c.base + (j + 1) * c.cs;
    const V ncn = L::splat(-cn);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const int r = L::row(i, lane);
      const bool ok = ok_row(r);
      q[i] = ok ? L::scale(L::ld(pj + r), inv) : L::zero();
      pn[i] = (nxt && ok) ? L::fma(q[i], ncn, L::ld(pj1 + r)) : L::zero();
    }
    // update columns a >= j+2 and form p_a^T p_{j+1}; column j+1 contributes its norm
    int a = j + 1 + warp;
    for (; a + kNW < bk; a += 2 * kNW) {
      const int b2 = a + kNW;
      const T ca = v[a] * inv, cb = v[b2] * inv;
      if (g == 0 && lane == 0) {
        R[j + a * ldr] = ca;
        R[j + b2 * ldr] = cb;
      }
      T* pa = c.base + a * c.cs;
      T* pb = c.base + b2 * c.cs;
      const V nca = L::splat(-ca), ncb = L::splat(-cb);
      V da = L::zero(), db = L::zero();
      const bool first = (a == j + 1);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const int r = L::row(i, lane);
        if (ok_row(r)) {
          if (first) {
            da = L::fma(pn[i], pn[i], da);
          } else {
            const V xa = L::fma(q[i], nca, L::ld(pa + r));
            L::st(pa + r, xa);
            da = L::fma(xa, pn[i], da);
          }
          const V xb = L::fma(q[i], ncb, L::ld(pb + r));
          L::st(pb + r, xb);
          db = L::fma(xb, pn[i], db);
        }
      }
      T sa = L::sum(da), sb = L::sum(db);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
      }
      if (lane == 0) {
        put_partial<T, CL || HIER>(c, a, sa, step);
        put_partial<T, CL || HIER>(c, b2, sb, step);
      }
    }
    if (a < bk) {
      const T ca = v[a] * inv;
      if (g == 0 && lane == 0) R[j + a * ldr] = ca;
      T* pa = c.base + a * c.cs;
      const V nca = L::splat(-ca);
      V da = L::zero();
      const bool first = (a == j + 1);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const int r = L::row(i, lane);
        if (ok_row(r)) {
          if (first) {
            da = L::fma(pn[i], pn[i], da);
          } else {
            const V xa = L::fma(q[i], nca, L::ld(pa + r));
            L::st(pa + r, xa);
            da = L::fma(xa, pn[i], da);
          }
        }
      }
      const T sa = warp_sum(L::sum(da));
      if (lane == 0) put_partial<T, CL || HIER>(c, a, sa, step);
    }
    T* pjw = c.base + j * c.cs;
    T* pj1w = c.base + (j + 1) * c.cs;
    if (!nxt) {
      __syncthreads();
      if (warp == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) {
          const int r = L::row(i, lane);
          if (ok_row(r)) L::st(pjw + r, q[i]);
        }
      break;
    }
    auto publish = [&]() {
      if (warp == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) {
          const int r = L::row(i, lane);
          if (ok_row(r)) {
            L::st(pjw + r, q[i]);
            L::st(pj1w + r, pn[i]);
          }
        }
    };
    if (!sync_reduce<T, CL, HIER>(c, j + 1, bk, v, step++, 2, publish)) { leave(); return; }
  }
  __syncthreads();
  if (SMEM)
    for (int a = 0; a < bk; ++a)
      for (int r = tid; r < nr; r += kNT) Q[row0 + r + a * ldq] = sm[(size_t)a * rpc_pad + r];
  if (CL || HIER) cluster_sync_all();  // peers may still read this CTA's partials
}

// Left-looking classical Gram-Schmidt on the panel (the variants compared in NEXT f3):
// per column j and pass, one reduction gives s_a = q_a^T p_j (a < j) and |p_j|^2 from the
// current p_j; then p_j -= Q_{:,0:j} s, R[0:j, j] += s, r_jj^2 = |p_j|^2 - |s|^2 (Pythagorean).
// PASSES = 1: one reduction per column (orthogonality ~ u kappa^2); PASSES = 2: CGS2.
// Same slices, reductions and synchronisation variants as k_panel.
template <typename T, int RPL, bool CL, bool SMEM, int PASSES>
__global__ void __launch_bounds__(kNT, 1) k_panel_cgs(T* __restrict__ Q, int64_t ldq, T* __restrict__ R,
                                                       int64_t ldr, int64_t M, int bk, int rpc,
                                                       int rpc_pad, double tau2, T* gpart,
                                                       unsigned* bar, int* status, int col0,
                                                   long long wait_limit) {
  constexpr int VW = (SMEM && sizeof(T) == 4 && RPL % 2 == 0) ? 2 : 1;
  constexpr int NV = RPL / VW;
  using L = LaneOps<T, VW>;
  using V = typename L::V;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int g = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int pld = (bk + 3) / 4 * 4;
  const int64_t row0 = (int64_t)g * rpc;
  const int nr = (int)((M - row0) < rpc ? (M - row0) : rpc);
  T* sm = reinterpret_cast<T*>(smraw);
  T* small = sm + (SMEM ? (size_t)bk * rpc_pad : 0);
  T* sv = small + 2 * pld;
  Ctx<T> c;
  c.base = SMEM ? sm : Q + row0;
  c.cs = SMEM ? rpc_pad : ldq;
  c.nr = nr;
  c.pld = pld;
  c.gpart = gpart;
  c.red = sv + 2 * pld;
  c.lpart = c.red + (CL ? 0 : 8 * 2 * pld);
  c.bar = bar;
  c.status = status;
  c.target = 0;
  c.wait_limit = wait_limit;
  (void)tau2;
  int step = 0;
  auto ok_row = [&](int r) { return SMEM ? true : (r < nr); };
  const int nrows = SMEM ? rpc : nr;
  if (SMEM)
    for (int a = 0; a < bk; ++a)
      for (int r = tid; r < rpc; r += kNT)
        sm[(size_t)a * rpc_pad + r] = (r < nr) ? Q[row0 + r + a * ldq] : T(0);
  __syncthreads();
  for (int j = 0; j < bk; ++j) {
    T* pj = c.base + j * c.cs;
    T r2 = T(0);
    for (int pass = 0; pass < PASSES; ++pass) {
      V pv[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const int r = L::row(i, lane);
        pv[i] = ok_row(r) ? L::ld(pj + r) : L::zero();
      }
      for (int a = warp; a <= j; a += kNW) {
        const T* pa = c.base + a * c.cs;
        V d = L::zero();
#pragma unroll
        for (int i = 0; i < NV; ++i) {
          const int r = L::row(i, lane);
          if (ok_row(r)) d = L::fma(L::ld(pa + r), pv[i], d);
        }
        const T s0 = warp_sum(L::sum(d));
        if (lane == 0) put_partial<T, CL>(c, a, s0, step);
      }
      if (!sync_reduce<T, CL>(c, 0, j + 1, sv, step++, 5)) return;
      for (int r = tid; r < nrows; r += kNT) {
        T acc = pj[r];
        for (int a = 0; a < j; ++a) acc -= c.base[a * c.cs + r] * sv[a];
        pj[r] = acc;
      }
      T ss = T(0);
      for (int a = 0; a < j; ++a) ss += sv[a] * sv[a];
      r2 = sv[j] - ss;
      if (g == 0)
        for (int a = tid; a < j; a += kNT) R[a + j * ldr] += sv[a];
      __syncthreads();
    }
    if (!(r2 > T(0)) || !isfinite(r2)) {
      if (g == 0 && tid == 0) set_status(status, CQR_EBREAKDOWN, col0 + j);
      if (CL) cluster_sync_all();
      return;
    }
    const T rjj = sqrt(r2);
    const T inv = T(1) / rjj;
    if (g == 0 && tid == 0) R[j + j * ldr] = rjj;
    for (int r = tid; r < nrows; r += kNT) pj[r] *= inv;
    __syncthreads();
  }
  if (SMEM)
    for (int a = 0; a < bk; ++a)
      for (int r = tid; r < nr; r += kNT) Q[row0 + r + a * ldq] = sm[(size_t)a * rpc_pad + r];
  if (CL) cluster_sync_all();  // peers may still read this CTA's partials
}

// Latency floor of k_panel's per-column exchange (a measurement aid; the paper has no
// counterpart): the reductions one panel of bk FP32 columns performs -- the first one of 2 pld
// entries, then entries j+1 .. bk-1 for j = 0 .. bk-2 -- `reps` times, through the same
// sync_reduce with the same launch shape and shared-memory footprint, and no column
// arithmetic around them.  Each CTA's partial of entry a is a + 1, so every sum must come
// back as G (a + 1) exactly; *bad counts the entries that did not.
template <bool CL, bool HIER>
__global__ void __launch_bounds__(kNT, 1) k_exchange_probe(int bk, int reps, float* gpart,
                                                           unsigned* bar, int* status, int* bad,
                                                           long long wait_limit) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int g = blockIdx.x, tid = threadIdx.x;
  const int pld = (bk + 3) / 4 * 4;
  float* v = reinterpret_cast<float*>(smraw);
  float* sv = v + 2 * pld;
  Ctx<float> c;
  c.base = nullptr;
  c.cs = 0;
  c.nr = 0;
  c.pld = pld;
  c.gpart = gpart;
  c.red = sv + 2 * pld;
  c.lpart = c.red + (CL ? 0 : 8 * 2 * pld);
  c.rbuf = c.red;
  c.mbar = reinterpret_cast<uint64_t*>(c.lpart + 4 * pld);
  c.bar = bar;
  c.status = status;
  c.target = 0;
  c.phases = 0u;
  c.hcs = kHierCS;
  if (HIER) {
    unsigned ncta;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(ncta));
    c.hcs = (int)ncta;
  }
  c.crank = g % c.hcs;
  c.cl = g / c.hcs;
  c.ncl = gridDim.x / c.hcs;
  c.wait_limit = wait_limit;
  if (HIER) {
    unsigned ncta;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(ncta));
    if ((ncta != (unsigned)kHierCS && ncta != (unsigned)kHierCSWide) || gridDim.x % ncta != 0) {
      if (g == 0 && tid == 0) set_status(status, CQR_ECUDA, 51);
      return;
    }
    if (tid == 0) {
      mbar_init(c.mbar, 1);
      mbar_init(c.mbar + 1, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cluster_sync_all();
  }
  const float G = (float)gridDim.x;
  int wrong = 0, step = 0;
  bool ok = true;
  for (int rep = 0; rep < reps && ok; ++rep)
    for (int j = -1; j < bk - 1 && ok; ++j) {
      const int lo = j < 0 ? 0 : j + 1, hi = j < 0 ? 2 * pld : bk;
      for (int a = lo + tid; a < hi; a += kNT)
        put_partial<float, CL || HIER>(c, a, (float)(a + 1), step);
      ok = sync_reduce<float, CL, HIER>(c, lo, hi, v, step++, 70);
      if (ok)
        for (int a = lo + tid; a < hi; a += kNT) wrong += v[a] != G * (float)(a + 1);
      __syncthreads();  // v is read before the next step overwrites it
    }
  if (wrong) atomicAdd(bad, wrong);
  if (CL || HIER) {
    cluster_sync_all();  // peers may still read this CTA's partials or push into it
    if (!ok) {
      const long long t0 = clock64();
      while (clock64() - t0 < kDrainCycles) {
      }
    }
  }
}

size_t small_bytes(int bk, size_t elem, bool cl, bool hier = false) {
  const int pld = (bk + 3) / 4 * 4;
  // v (2 pld, includes eta), sv (2 pld), then either red [8][2 pld] or lpart [2][2 pld];
  // two-level: red (the leader's receive buffer), lpart and two mbarriers
  if (hier) return (size_t)(2 * pld + 2 * pld + 16 * pld + 4 * pld) * elem + 16 + 256;
  return (size_t)(2 * pld + 2 * pld + (cl ? 4 * pld : 16 * pld)) * elem + 256;
}

int env_int(const char* name, int dflt) {
  const char* s = getenv(name);
  return s ? atoi(s) : dflt;
}

template <typename T, int RPL, int PASSES>
const void* cgs_of(bool cl, bool smem) {
  if (cl) return (const void*)k_panel_cgs<T, RPL, true, true, PASSES>;
  if (smem) return (const void*)k_panel_cgs<T, RPL, false, true, PASSES>;
  return (const void*)k_panel_cgs<T, RPL, false, false, PASSES>;
}

// variant: 0 the paper's ICGS (MGS when tau2 <= 0), 1 CGS1, 2 CGS2
template <typename T, int RPL>
const void* kernel_of(bool cl, bool smem, int variant) {
  if (variant == 1) return cgs_of<T, RPL, 1>(cl, smem);
  if (variant == 2) return cgs_of<T, RPL, 2>(cl, smem);
  if (cl) return (const void*)k_panel<T, RPL, true, true, false>;
  if (smem) return (const void*)k_panel<T, RPL, false, true, false>;
  return (const void*)k_panel<T, RPL, false, false, false>;
}

template <typename T, int RPL>
const void* hier_of() {
  if constexpr (sizeof(T) == 4) return (const void*)k_panel<T, RPL, false, true, true>;
  return nullptr;
}

template <typename T>
const void* pick_hier(int rpl) {
  switch (rpl) {
    case 4: return hier_of<T, 4>();
    case 6: return hier_of<T, 6>();
    case 8: return hier_of<T, 8>();
    case 12: return hier_of<T, 12>();
    case 16: return hier_of<T, 16>();
    case 24: return hier_of<T, 24>();
    default: return hier_of<T, 32>();
  }
}

template <typename T>
const void* pick_kernel(int rpl, bool cl, bool smem, int variant = 0) {
  switch (rpl) {
    case 4: return kernel_of<T, 4>(cl, smem, variant);
    case 6: return kernel_of<T, 6>(cl, smem, variant);
    case 8: return kernel_of<T, 8>(cl, smem, variant);
    case 12: return kernel_of<T, 12>(cl, smem, variant);
    case 16: return kernel_of<T, 16>(cl, smem, variant);
    case 24: return kernel_of<T, 24>(cl, smem, variant);
    case 40: return kernel_of<T, 40>(cl, smem, variant);
    default: return kernel_of<T, 32>(cl, smem, variant);
  }
}

constexpr int kRpl[] = {4, 6, 8, 12, 16, 24, 32};
// one cluster of 16 CTAs may also take 1280-row slices (a 20480-row panel of 32 FP32 columns)
constexpr int kRplCluster[] = {4, 6, 8, 12, 16, 24, 32, 40};

int rpl_for_rows(int rpc) {
  for (int r : kRpl)
    if (32 * r >= rpc) return r;
  return 32;
}

}  // namespace

// Launch plan.  A CTA's slice has rpc = 32 RPL rows (RPL rows per lane).  Preferred: the
// smallest RPL whose slices fit shared memory and give G <= 16 CTAs (one cluster); otherwise
// the smallest RPL that fits shared memory with G <= #SMs (grid barrier); otherwise slices in
// global memory.  CQR_PANEL_RPL / CQR_PANEL_CLUSTER override the choice (tuning).
PanelPlan plan_panel(int64_t M, int bk, size_t elem, int num_sms, bool allow_cluster,
                     bool allow_hier, int hier_cs) {
  PanelPlan p{};
  const int rpl_env = env_int("CQR_PANEL_RPL", 0);
  const int cl_env = env_int("CQR_PANEL_CLUSTER", -1);
  auto fits = [&](int rpl, bool cl) {
    const int rpc = 32 * rpl;
    return (size_t)bk * rpc * elem + small_bytes(bk, elem, cl) + 1024 <= kSmemCap;
  };
  int best = -1;
  bool best_cl = false;
  if (allow_cluster && cl_env != 0)
    for (int r : kRplCluster)
      if ((rpl_env == 0 || r == rpl_env) && fits(r, true) && (M + 32 * r - 1) / (32 * r) <= kMaxCluster) {
        best = r;
        best_cl = true;
        break;
      }
  // grid of CTAs with shared-memory slices: the largest slices that fit, so the fewest CTAs
  // (a cheaper grid barrier, and more independent panels resident at once; at 9216 x 128 the
  // per-column time is flat in the slice height while 16 concurrent problems run 3x faster
  // with 24 CTAs each than with 72)
  if (best < 0)
    for (int q = (int)(sizeof(kRpl) / sizeof(kRpl[0])) - 1; q >= 0; --q) {
      const int r = kRpl[q];
      if ((rpl_env == 0 || r == rpl_env) && fits(r, false) && (M + 32 * r - 1) / (32 * r) <= num_sms) {
        best = r;
        break;
      }
    }
  if (best > 0) {
    p.smem = 1;
    p.cluster = best_cl ? 1 : 0;
    p.rpc = 32 * best;
    p.G = (int)((M + p.rpc - 1) / p.rpc);
    p.rpc_pad = p.rpc;
    p.smem_bytes = (size_t)bk * p.rpc_pad * elem + small_bytes(bk, elem, best_cl);
    // many CTAs (FP32): the two-level exchange, the grid padded to whole clusters (the extra
    // CTAs own no rows)
    if (!best_cl && allow_hier && elem == 4 && p.G > kHierMinG && env_int("CQR_PANEL_HIER", 1) != 0) {
      // clusters of 16 (non-portable) unless the caller or CQR_HIER_CS asks for 8: half as
      // many cluster sums for every CTA to poll (20480 x 256, FP32: 73.5 against 78.3 ms per
      // 64 panels)
      const int req = env_int("CQR_HIER_CS", hier_cs);
      const int hcs = req == kHierCS ? kHierCS : kHierCSWide;
      const int Gh = (p.G + hcs - 1) / hcs * hcs;
      const size_t sb = (size_t)bk * p.rpc_pad * elem + small_bytes(bk, elem, false, true);
      if (Gh <= num_sms && sb + 1024 <= kSmemCap) {
        p.hier = 1;
        p.hcs = hcs;
        p.G = Gh;
        p.smem_bytes = sb;
      }
    }
    return p;
  }
  // slices stay in global memory (L2): at most 32 rows per lane
  int rpl = (int)((M + 32LL * num_sms - 1) / (32LL * num_sms));
  rpl = rpl_for_rows(32 * rpl);
  if (rpl_env > rpl) rpl = rpl_for_rows(32 * rpl_env);  // never more CTAs than SMs
  p.smem = 0;
  p.cluster = 0;
  p.rpc = 32 * rpl;
  p.G = (int)((M + p.rpc - 1) / p.rpc);
  p.rpc_pad = p.rpc;
  p.smem_bytes = small_bytes(bk, elem, false);
  return p;
}

// Launch configuration of the two-level variant: clusters of pp.hcs CTAs over the whole
// grid.  Its leaders wait for one another, so every cluster must be resident at once: the
// plan is taken only when the occupancy query says they all fit (panel_hier_fits), and the
// variant is used only on the sequential schedule, where the panel is the only work on the
// GPU when it runs.
void hier_config(const PanelPlan& pp, cudaStream_t st, cudaLaunchConfig_t* cfg,
                 cudaLaunchAttribute* attr) {
  *cfg = cudaLaunchConfig_t{};
  cfg->gridDim = dim3(pp.G);
  cfg->blockDim = dim3(kNT);
  cfg->dynamicSmemBytes = pp.smem_bytes;
  cfg->stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = pp.hcs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg->attrs = attr;
  cfg->numAttrs = 1;
}

template <typename T>
cudaError_t launch_hier(const PanelPlan& pp, int rpl, void** args, cudaStream_t st) {
  const void* fn = pick_hier<T>(rpl);
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)pp.smem_bytes);
  if (e == cudaSuccess && pp.hcs > 8)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  hier_config(pp, st, &cfg, attr);
  return cudaLaunchKernelExC(&cfg, fn, args);
}

template <typename T>
cudaError_t launch_panel(const PanelPlan& pp, T* Q, int64_t ldq, T* R, int64_t ldr, int64_t M,
                         int bk, double tau, T* part, unsigned* bar, int* status, int col0,
                         cudaStream_t st, int variant, long long wait_limit) {
  if (pp.G > 1 && !pp.cluster) {
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
  }
  const int rpl = (pp.rpc / 32);
  double tau2 = tau > 0.0 ? tau * tau : -1.0;
  int rpc = pp.rpc, rpc_pad = pp.rpc_pad;
  long long wl = wait_limit > 0 ? wait_limit : kWaitLimitCycles;
  void* args[] = {&Q, &ldq, &R, &ldr, &M, &bk, &rpc, &rpc_pad, &tau2, &part, &bar, &status, &col0,
                  &wl};
  if (pp.hier && variant == 0) {
    // the tagged cluster-sum rows (G .. G + 2 clusters) start cleared: no tag of an earlier
    // launch can match
    const int pld = (bk + 3) / 4 * 4;
    const size_t row = (size_t)2 * pld * sizeof(T);
    cudaError_t e = cudaMemsetAsync(reinterpret_cast<char*>(part) + (size_t)pp.G * row, 0,
                                    (size_t)2 * (pp.G / pp.hcs) * row, st);
    if (e != cudaSuccess) return e;
    return launch_hier<T>(pp, rpl, args, st);
  }
  const void* fn = pick_kernel<T>(rpl, pp.cluster != 0, pp.smem != 0, variant);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)pp.smem_bytes);
  if (e != cudaSuccess) return e;
  if (pp.cluster) {
    if (pp.G > 8) {
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pp.G);
    cfg.blockDim = dim3(kNT);
    cfg.dynamicSmemBytes = pp.smem_bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = pp.G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
  }
  return cudaLaunchCooperativeKernel(fn, dim3(pp.G), dim3(kNT), args, pp.smem_bytes, st);
}

// Whether a cluster of pp.G CTAs with this shared-memory footprint can be scheduled.
template <typename T>
bool panel_cluster_fits(const PanelPlan& pp) {
  const void* fn = pick_kernel<T>((pp.rpc / 32), true, true);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pp.smem_bytes) !=
      cudaSuccess)
    return false;
  if (pp.G > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                      cudaSuccess)
    return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pp.G);
  cfg.blockDim = dim3(kNT);
  cfg.dynamicSmemBytes = pp.smem_bytes;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = pp.G;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n >= 1;
}

template <typename T>
bool panel_hier_fits(const PanelPlan& pp) {
  if (!pp.hier) return false;
  const void* fn = pick_hier<T>((pp.rpc / 32));
  if (!fn) return false;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pp.smem_bytes) !=
          cudaSuccess ||
      (pp.hcs > 8 &&
       cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  hier_config(pp, nullptr, &cfg, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n >= pp.G / pp.hcs;
}

size_t panel_partial_bytes(int bk, size_t elem, int num_sms) {
  const int pld = (bk + 3) / 4 * 4;
  return (size_t)2 * (num_sms + 1) * 2 * pld * elem;
}

template cudaError_t launch_panel<float>(const PanelPlan&, float*, int64_t, float*, int64_t, int64_t,
                                         int, double, float*, unsigned*, int*, int, cudaStream_t,
                                         int, long long);
template cudaError_t launch_panel<double>(const PanelPlan&, double*, int64_t, double*, int64_t,
                                          int64_t, int, double, double*, unsigned*, int*, int,
                                          cudaStream_t, int, long long);
template bool panel_cluster_fits<float>(const PanelPlan&);
template bool panel_cluster_fits<double>(const PanelPlan&);
template bool panel_hier_fits<float>(const PanelPlan&);
template bool panel_hier_fits<double>(const PanelPlan&);

// One launch of the exchange probe on the plan of a panel (the same grid, clusters and dynamic
// shared memory as launch_panel; the tagged rows and the barrier counter cleared first).
cudaError_t launch_exchange_probe(const PanelPlan& pp, int bk, int reps, float* part,
                                  unsigned* bar, int* status, int* bad, cudaStream_t st) {
  const void* fn = pp.hier      ? (const void*)k_exchange_probe<false, true>
                   : pp.cluster ? (const void*)k_exchange_probe<true, false>
                                : (const void*)k_exchange_probe<false, false>;
  const int pld = (bk + 3) / 4 * 4;
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), st);
  if (e == cudaSuccess && pp.hier) {
    const size_t row = (size_t)2 * pld * sizeof(float);
    e = cudaMemsetAsync(reinterpret_cast<char*>(part) + (size_t)pp.G * row, 0,
                        (size_t)2 * (pp.G / pp.hcs) * row, st);
  }
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pp.smem_bytes);
  if (e == cudaSuccess && ((pp.cluster && pp.G > 8) || (pp.hier && pp.hcs > 8)))
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  long long wl = kWaitLimitCycles;
  void* args[] = {&bk, &reps, &part, &bar, &status, &bad, &wl};
  if (pp.hier || pp.cluster) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pp.G);
    cfg.blockDim = dim3(kNT);
    cfg.dynamicSmemBytes = pp.smem_bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = pp.hier ? pp.hcs : pp.G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
  }
  return cudaLaunchCooperativeKernel(fn, dim3(pp.G), dim3(kNT), args, pp.smem_bytes, st);
}

cudaError_t bounds_take_panel(int* code, int* site) { return bounds_take_here(code, site); }

}  // namespace cqr

// =========================================================================================
// Allocation-free panel factorisation (coded_qr_panel_icgs_noalloc in coded_qr.h).
//
// Some callers cannot allocate device memory at the point where they need one panel
// factored: a caching allocator that must not be re-entered from its own callbacks, a host
// that has handed all device memory to another framework, or a latency-critical path that
// must not take the driver's allocation lock.  For them
// the grid-barrier panel kernel above runs with its scratch (per-CTA partial sums, the
// barrier counter and the status word) in the file-scope device array below instead of a
// handle's workspace.  Every GPU that loads the library keeps this array until exit.
// =========================================================================================
namespace cqr {
namespace {

constexpr int kNoallocMaxBk = 256;
constexpr int kNoallocMaxG = 160;
constexpr size_t kNoallocPartBytes =
    (size_t)2 * kNoallocMaxG * 2 * kNoallocMaxBk * sizeof(double);   // 1,310,720 bytes
constexpr size_t kNoallocBytes = kNoallocPartBytes + 512;            // + barrier + status

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device; looked up once per device
// (cudaGetSymbolAddress, with that device current) and cached.
cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  void* p = __atomic_load_n(&g_noalloc_ptr[dev], __ATOMIC_ACQUIRE);
  if (!p) {
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    __atomic_store_n(&g_noalloc_ptr[dev], p, __ATOMIC_RELEASE);
  }
  *out = p;
  return cudaSuccess;
}

template <typename T>
cqr_status noalloc_run(int64_t M, int bk, T* Q, int64_t ldq, T* R, int64_t ldr, double tau,
                       int* status_out, cudaStream_t st) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return CQR_ECUDA;
  }
  PanelPlan pp = plan_panel(M, bk, sizeof(T), sms, false, false);
  if (pp.G > kNoallocMaxG || pp.G > sms) return CQR_EINVAL;
  void* base = nullptr;
  if (noalloc_scratch(&base) != cudaSuccess) {
    cudaGetLastError();
    return CQR_ECUDA;
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  T* part = reinterpret_cast<T*>(b);
  unsigned* bar = reinterpret_cast<unsigned*>(b + kNoallocPartBytes);
  int* status = status_out ? status_out : reinterpret_cast<int*>(b + kNoallocPartBytes + 256);
  // the array keeps the previous call's contents: the status word must start at zero (the
  // barrier counter is zeroed by launch_panel)
  cudaError_t e = cudaMemsetAsync(status, 0, 4 * sizeof(int), st);
  if (e == cudaSuccess) e = launch_panel<T>(pp, Q, ldq, R, ldr, M, bk, tau, part, bar, status, 0, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CQR_ECUDA;
  }
  return CQR_OK;
}

}  // namespace

}  // namespace cqr

extern "C" cqr_status coded_qr_panel_icgs_noalloc(int32_t dtype, int64_t M, int32_t bk, void* Q,
                                                  int64_t ldq, void* R, int64_t ldr, double tau,
                                                  int32_t* status, void* stream) {
  using namespace cqr;
  if (!Q || !R || M < 1 || bk < 1 || ldq < M || ldr < bk) return CQR_EINVAL;
  if (dtype != CQR_F64 && dtype != CQR_F32) return CQR_EINVAL;
  if (bk > kNoallocMaxBk) return CQR_EINVAL;  // beyond the static scratch's capacity
  const double t = tau == 0.0 ? 0.7071067811865476 : tau;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return dtype == CQR_F64
             ? noalloc_run<double>(M, bk, (double*)Q, ldq, (double*)R, ldr, t, status, st)
             : noalloc_run<float>(M, bk, (float*)Q, ldq, (float*)R, ldr, t, status, st);
}
