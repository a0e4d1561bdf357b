// cqr_panel_reg.cu -- register-resident panel ICGS (a3) for FP32 panels that fit one
// thread-block cluster: same algorithm and arithmetic order as cqr_panel.cu (Appendix A,
// Algorithm CGS with the ICGS reorthogonalisation, one reduction per column), but the slice
// of the panel owned by a CTA lives in registers instead of shared memory.
//
// Layout: G <= 16 CTAs (one cluster), CTA g owns rows [g rpc, (g+1) rpc), rpc = 32 RPL.
// Warp w owns panel columns a = w + 8 k (k < CPW); lane l owns row pairs
// 64 i + 2 l + {0, 1} (i < RPL / 2), packed in 64-bit registers for f32x2 FMAs.
// Per column j (v_a = p_a^T p_j already reduced, identical in every CTA):
//   q_j = p_j / r_jj and the updated p_{j+1} are formed by every warp from a shared staging
//   copy of columns j, j+1 (double-buffered by column parity); each warp updates its own
//   columns a > j in registers and forms p_a^T p_{j+1}; the per-lane partials of a warp's
//   columns are combined by a butterfly over the lanes into this CTA's partial vector in
//   shared memory; every CTA then stores its partial vector into every CTA's receive buffer
//   (16-byte asynchronous distributed-shared-memory stores that count their bytes on the
//   receiver's mbarrier), waits on its own mbarrier for the G vectors and sums them in the
//   same fixed order.  The owners of columns j+1 and j+2 write them to the other staging
//   buffer before the exchange.  Receive buffers and mbarriers alternate by reduction parity:
//   a CTA sends reduction k+2 only after it has received reduction k+1 from every CTA, each
//   of which sent it after finishing with its own buffer of reduction k.
#include <math.h>

#include "cqr_device.cuh"
#include "cqr_kernels.cuh"

namespace cqr {

namespace {

constexpr int kNT = 256;
constexpr int kNW = kNT / 32;   // 8 warps
constexpr int kMaxG = 16;

__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}

__device__ __forceinline__ uint64_t f2fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t f2splat(float s) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(s));
  return r;
}
__device__ __forceinline__ float f2sum(uint64_t v) {
  float x, y;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
  return x + y;
}

// Butterfly over the 32 lanes of CPW per-lane values (one per owned column slot).  After it,
// lane l holds the full 32-lane sum of slot slot_of(l).
template <int CPW>
__device__ __forceinline__ float butterfly(float (&x)[CPW], int lane) {
  float y[CPW];
#pragma unroll
  for (int k = 0; k < CPW; ++k) y[k] = x[k];
  int n = CPW;
  int off = 16;
#pragma unroll
  for (int round = 0; round < 4; ++round) {
    if ((CPW >> round) > 1) {
      const int h = (CPW >> round) / 2;
      const bool upper = (lane & off) != 0;
#pragma unroll
      for (int k = 0; k < CPW / 2; ++k) {
        if (k < h) {
          const float mine = upper ? y[k + h] : y[k];
          const float other = upper ? y[k] : y[k + h];
          y[k] = mine + __shfl_xor_sync(0xffffffffu, other, off);
        }
      }
      n = h;
      off >>= 1;
    }
  }
  (void)n;
  float s = y[0];
  for (; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

template <int CPW>
__device__ __forceinline__ int slot_of(int lane) {
  // bit 4 of the lane picks the upper half of the slots in the first round, bit 3 in the
  // second, and so on (as many rounds as log2 CPW)
  int s = 0, h = CPW, off = 16;
#pragma unroll
  for (int round = 0; round < 4; ++round) {
    if ((CPW >> round) > 1) {
      h >>= 1;
      if (lane & off) s += h;
      off >>= 1;
    }
  }
  return s;
}

template <int CPW>
__device__ __forceinline__ int lanes_per_slot() {
  return 32 / CPW;
}

// The cluster exchange of the partial vectors, shared by k_panel_reg and the exchange probe.
// Entries lo .. hi-1 (whole 4-entry chunks) of this CTA's partial vector lpart[par] go into
// receive buffer [par][g] of every CTA of the cluster (16-byte st.async that count their bytes
// on the receiver's mbarrier); then the wait for all G vectors.  The wait is bounded by
// wait_limit cycles; when it runs out, the CTA records CQR_ETIMEOUT and returns false, and a
// CTA whose wait is long overdue also gives up once any CTA has recorded an error.  The result
// is the same in every thread of the CTA.  phases: bit p is the phase parity of mbarrier p.
__device__ __forceinline__ bool reg_exchange(const float* lpart, float* rbuf, uint64_t* mbar,
                                             unsigned& phases, int par, int lo, int hi,
                                             long long wait_limit, int* status) {
  const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, warp = tid >> 5;
  const int c0 = lo / 4, nch = (hi + 3) / 4 - c0;
  __syncthreads();  // this CTA's partials are complete
  if (tid == 0) mbar_expect(mbar + par, (unsigned)(G * nch * 16));
  const uint32_t dst0 = saddr(rbuf + ((size_t)par * kMaxG + g) * 512);
  const uint32_t bar0 = saddr(mbar + par);
  if (nch <= 32) {
    // lane l sends chunk c0 + l to the peers warp, warp + 8 (one float4 read, G <= 16)
    const int l = tid & 31;
    if (l < nch) {
      const float4 x = *reinterpret_cast<const float4*>(lpart + par * 512 + 4 * (c0 + l));
      for (int peer = warp; peer < G; peer += kNW)
        st_async4(peer_addr(dst0, peer) + 16u * (c0 + l), x, peer_addr(bar0, peer));
    }
  } else {
    for (int it = tid; it < G * nch; it += kNT) {
      const int peer = it / nch, ch = c0 + it % nch;
      const float4 x = *reinterpret_cast<const float4*>(lpart + par * 512 + 4 * ch);
      st_async4(peer_addr(dst0, peer) + 16u * ch, x, peer_addr(bar0, peer));
    }
  }
  const bool ok = mbar_wait_bounded(mbar + par, (phases >> par) & 1u, wait_limit, status, 40);
  phases ^= 1u << par;
  return __syncthreads_and(ok) != 0;
}

// out[a] (lo <= a < hi) = sum over the G CTAs of their partial vectors in receive buffer par,
// a fixed-shape tree over kMaxG senders (absent ones add zero): the same order in every CTA.
__device__ __forceinline__ void reg_gather(const float* rbuf, int par, int lo, int hi, float* out) {
  const int G = gridDim.x;
  const float* rb = rbuf + (size_t)par * kMaxG * 512;
  for (int a = lo + (int)threadIdx.x; a < hi; a += kNT) {
    float x[kMaxG];
#pragma unroll
    for (int q = 0; q < kMaxG; ++q) x[q] = q < G ? rb[q * 512 + a] : 0.f;
#pragma unroll
    for (int w = kMaxG / 2; w > 0; w /= 2)
#pragma unroll
      for (int q = 0; q < w; ++q) x[q] += x[q + w];
    out[a] = x[0];
  }
}

template <int RPL, int CPW>
__global__ void __launch_bounds__(kNT, 1) k_panel_reg(float* __restrict__ Q, int64_t ldq,
                                                       float* __restrict__ R, int64_t ldr,
                                                       int64_t M, int bk, double tau2, int* status,
                                                       int col0, long long wait_limit) {
  constexpr int NP = RPL / 2;            // row pairs per lane
  constexpr int RPC = 32 * RPL;          // rows per CTA
  extern __shared__ __align__(16) unsigned char smraw[];
  float* stage = reinterpret_cast<float*>(smraw);       // [2 parity][2 columns][RPC]
  float* lpart = stage + 4 * RPC;                        // [2 parity][512] own partials
  float* rbuf = lpart + 2 * 512;                         // [2 parity][kMaxG senders][512]
  float* v = rbuf + 2 * kMaxG * 512;                     // [512]: v, eta in [256..)
  float* sv = v + 512;                                   // [256]
  float* racc = sv + 256;                                // [kNW][RPC] reorth contributions
  uint64_t* mbar = reinterpret_cast<uint64_t*>(racc + kNW * RPC);  // [2 parity]
  const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  // the panel's columns fit the owned slots and its rows the cluster's slices (uniform:
  // before any barrier)
  CQR_CHECK(ldq >= M && ldr >= bk && bk <= kNW * CPW && bk <= 256 && G <= kMaxG &&
                (int64_t)G * RPC >= M, 301);
  const int64_t row0 = (int64_t)g * RPC;
  const int nr = (int)((M - row0) < RPC ? (M - row0) : RPC);
  float* eta = v + 256;
  constexpr int GS = CPW < 8 ? CPW : 8;  // slots reduced per butterfly
  constexpr int NG = CPW / GS;
  const int slot = slot_of<GS>(lane);
  const int lps = lanes_per_slot<GS>();
  const int sub = lane % lps;            // which subset of peers this lane pushes to

  if (tid == 0) {
    mbar_init(mbar, 1);
    mbar_init(mbar + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  cl_sync();  // every CTA's mbarriers are initialised before any peer stores into it
  // launched with programmatic stream serialization, the kernel may start while its
  // predecessor finishes: wait for it before reading the panel (no early trigger of the
  // successor, whose waiting CTAs would take SMs from concurrent work)
  asm volatile("griddepcontrol.wait;" ::: "memory");

  uint64_t P[CPW][NP];
  // load the slice (zero rows past M)
#pragma unroll
  for (int k = 0; k < CPW; ++k) {
    const int a = warp + kNW * k;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const int r = 64 * i + 2 * lane;
      float x0 = 0.f, x1 = 0.f;
      if (a < bk) {
        if (r < nr) x0 = Q[row0 + r + a * ldq];
        if (r + 1 < nr) x1 = Q[row0 + r + 1 + a * ldq];
      }
      asm("mov.b64 %0, {%1, %2};" : "=l"(P[k][i]) : "f"(x0), "f"(x1));
    }
  }
  auto owner_write = [&](int col, float* dst) {  // owner warp of `col` stores it to dst[RPC]
    if (col < bk && warp == (col % kNW)) {
      const int k = col / kNW;
#pragma unroll
      for (int kk = 0; kk < CPW; ++kk)
        if (kk == k)
#pragma unroll
          for (int i = 0; i < NP; ++i)
            *reinterpret_cast<uint64_t*>(dst + 64 * i + 2 * lane) = P[kk][i];
    }
  };
  // the warp's per-slot sums (after the butterfly) into this CTA's partial vector
  auto push = [&](float s, int par, int base, bool active_slot, int a) {
    if (active_slot && sub == 0) lpart[par * 512 + base + a] = s;
  };
  // exchange and gather (reg_exchange, reg_gather): when an exchange gives up, every CTA
  // leaves the column loop (the decision is uniform within a CTA) and meets the others at the
  // kernel's final cluster barrier
  unsigned phases = 0u;  // bit p: the phase parity of mbarrier p
  auto exchange = [&](int par, int lo, int hi) -> bool {
    return reg_exchange(lpart, rbuf, mbar, phases, par, lo, hi, wait_limit, status);
  };
  auto gather = [&](int par, int lo, int hi, float* out) { reg_gather(rbuf, par, lo, hi, out); };

  int par = 0;
  // ---- step 0: v_a = p_a^T p_0, eta_a = p_a^T p_a
  owner_write(0, stage);
  __syncthreads();
  {
    uint64_t p0[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) p0[i] = *reinterpret_cast<const uint64_t*>(stage + 64 * i + 2 * lane);
#pragma unroll
    for (int gr = 0; gr < NG; ++gr) {
      float d0[GS], d1[GS];
#pragma unroll
      for (int kk = 0; kk < GS; ++kk) {
        const int k = gr * GS + kk;
        uint64_t s0 = 0ull, s1 = 0ull;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          s0 = f2fma(P[k][i], p0[i], s0);
          s1 = f2fma(P[k][i], P[k][i], s1);
        }
        d0[kk] = f2sum(s0);
        d1[kk] = f2sum(s1);
      }
      const float e0 = butterfly<GS>(d0, lane), e1 = butterfly<GS>(d1, lane);
      const int a = warp + kNW * (gr * GS + slot);
      push(e0, par, 0, a < bk, a);
      push(e1, par, 256, a < bk, a);
    }
  }
  // columns 0 and 1 go to staging buffer 0 (column 0 is still there)
  owner_write(1, stage + RPC);
  bool aborted = !exchange(par, 0, 256 + bk);
  gather(par, 0, bk, v);
  gather(par, 256, 256 + bk, v);
  __syncthreads();
  par ^= 1;
  // The ICGS test v_j < tau^2 eta_j (product in FP64) in FP32 against the FP64 product
  // rounded up to FP32: the same decision for every FP32 v, with one FP64 product per column
  // and CTA instead of one per thread and column.  First used at j = 1, after the next
  // exchange's barriers.
  const bool icgs = tau2 > 0.0;
  if (icgs)
    for (int a = tid; a < bk; a += kNT) eta[a] = __double2float_ru(tau2 * (double)eta[a]);

  for (int j = 0; j < bk && !aborted; ++j) {
    float* st_cur = stage + (size_t)(j & 1) * 2 * RPC;   // p_j, p_{j+1}
    float* st_nxt = stage + (size_t)((j + 1) & 1) * 2 * RPC;
    if (j > 0 && icgs && v[j] < eta[j]) {
      // ICGS reorthogonalisation of p_j against columns 0 .. j-1 (held by their owners)
      uint64_t pj[NP];
#pragma unroll
      for (int i = 0; i < NP; ++i) pj[i] = *reinterpret_cast<const uint64_t*>(st_cur + 64 * i + 2 * lane);
#pragma unroll
      for (int gr = 0; gr < NG; ++gr) {
        float d[GS];
#pragma unroll
        for (int kk = 0; kk < GS; ++kk) {
          uint64_t s = 0ull;
#pragma unroll
          for (int i = 0; i < NP; ++i) s = f2fma(P[gr * GS + kk][i], pj[i], s);
          d[kk] = f2sum(s);
        }
        const float e = butterfly<GS>(d, lane);
        const int a = warp + kNW * (gr * GS + slot);
        push(e, par, 0, a < j, a);
      }
      if (!exchange(par, 0, j)) {
        aborted = true;
        break;
      }
      gather(par, 0, j, sv);
      __syncthreads();
      par ^= 1;
      // each warp's contribution sum_{a < j, owned} q_a s_a for its rows, then the owner sums
      uint64_t cacc[NP];
#pragma unroll
      for (int i = 0; i < NP; ++i) cacc[i] = 0ull;
#pragma unroll
      for (int k = 0; k < CPW; ++k) {
        const int a = warp + kNW * k;
        if (a < j) {
          const uint64_t sa = f2splat(sv[a]);
#pragma unroll
          for (int i = 0; i < NP; ++i) cacc[i] = f2fma(P[k][i], sa, cacc[i]);
        }
      }
#pragma unroll
      for (int i = 0; i < NP; ++i)
        *reinterpret_cast<uint64_t*>(racc + (size_t)warp * RPC + 64 * i + 2 * lane) = cacc[i];
      __syncthreads();
      if (warp == (j % kNW)) {
        const int kj = j / kNW;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          float t0 = 0.f, t1 = 0.f;
          for (int w = 0; w < kNW; ++w) {
            const float2 c2 = *reinterpret_cast<const float2*>(racc + (size_t)w * RPC + 64 * i + 2 * lane);
            t0 += c2.x;
            t1 += c2.y;
          }
          uint64_t tt;
          asm("mov.b64 %0, {%1, %2};" : "=l"(tt) : "f"(-t0), "f"(-t1));
#pragma unroll
          for (int kk = 0; kk < CPW; ++kk)
            if (kk == kj) {
              P[kk][i] = f2fma(tt, f2splat(1.f), P[kk][i]);
              *reinterpret_cast<uint64_t*>(st_cur + 64 * i + 2 * lane) = P[kk][i];
            }
        }
      }
      if (g == 0) {
        for (int a = tid; a < j; a += kNT) R[a + j * ldr] += sv[a];
        if (tid == 0) atomicAdd(status + ST_REORTH, 1);
      }
      __syncthreads();
      // v_a = p_a^T p_j for a >= j with the new p_j
#pragma unroll
      for (int i = 0; i < NP; ++i) pj[i] = *reinterpret_cast<const uint64_t*>(st_cur + 64 * i + 2 * lane);
#pragma unroll
      for (int gr = 0; gr < NG; ++gr) {
        float d[GS];
#pragma unroll
        for (int kk = 0; kk < GS; ++kk) {
          uint64_t s = 0ull;
#pragma unroll
          for (int i = 0; i < NP; ++i) s = f2fma(P[gr * GS + kk][i], pj[i], s);
          d[kk] = f2sum(s);
        }
        const float e = butterfly<GS>(d, lane);
        const int a = warp + kNW * (gr * GS + slot);
        push(e, par, 0, a >= j && a < bk, a);
      }
      if (!exchange(par, j, bk)) {
        aborted = true;
        break;
      }
      gather(par, j, bk, v);
      __syncthreads();
      par ^= 1;
    }
    const float v0 = v[j];
    if (!(v0 > 0.f) || !isfinite(v0)) {
      if (g == 0 && tid == 0) set_status(status, CQR_EBREAKDOWN, col0 + j);
      cl_sync();  // uniform exit (every CTA sees the same v)
      return;
    }
    const float rjj = sqrtf(v0);
    const float inv = 1.f / rjj;
    const bool nxt = j + 1 < bk;
    const float cn = nxt ? v[j + 1] * inv : 0.f;
    if (g == 0) {  // row j of R: r_jj and r_ja = v_a / r_jj (a > j)
      if (tid == 0) R[j + j * ldr] = rjj;
      for (int a = j + 1 + tid; a < bk; a += kNT) R[j + a * ldr] = v[a] * inv;
    }
    uint64_t q[NP], pn[NP];
    const uint64_t sinv = f2splat(inv), ncn = f2splat(-cn);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      q[i] = f2fma(*reinterpret_cast<const uint64_t*>(st_cur + 64 * i + 2 * lane), sinv, 0ull);
      pn[i] = nxt ? f2fma(q[i], ncn, *reinterpret_cast<const uint64_t*>(st_cur + RPC + 64 * i + 2 * lane))
                  : 0ull;
    }
    // Straight-line update of the owned columns of a group of GS (no branch between columns,
    // so the compiler interleaves their independent chains): a column that is not active
    // (a <= j or past the panel) is updated with the coefficient 0, which leaves it exactly
    // unchanged, and its product is not pushed; column j then takes q_j.
#pragma unroll
    for (int gr = 0; gr < NG; ++gr) {
      // a group whose columns are all finished (a <= j) has nothing to update or push
      if (warp + kNW * (gr * GS + GS - 1) <= j) continue;
      float d[GS];
#pragma unroll
      for (int kk = 0; kk < GS; ++kk) {
        const int k = gr * GS + kk;
        const int a = warp + kNW * k;
        const bool act = a > j && a < bk;
        const uint64_t nca = f2splat(act ? -(v[a] * inv) : 0.f);
        uint64_t s = 0ull;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          const uint64_t x = f2fma(q[i], nca, P[k][i]);
          P[k][i] = x;
          s = f2fma(x, pn[i], s);
        }
        d[kk] = f2sum(s);
      }
      if (nxt) {
        const float e = butterfly<GS>(d, lane);
        const int a = warp + kNW * (gr * GS + slot);
        push(e, par, 0, a > j && a < bk, a);
      }
    }
    if (warp == (j % kNW)) {
      const int kj = j / kNW;
#pragma unroll
      for (int k = 0; k < CPW; ++k)
        if (k == kj)
#pragma unroll
          for (int i = 0; i < NP; ++i) P[k][i] = q[i];
    }
    if (!nxt) break;
    owner_write(j + 1, st_nxt);
    owner_write(j + 2, st_nxt + RPC);
    if (!exchange(par, j + 1, bk)) {
      aborted = true;
      break;
    }
    gather(par, j + 1, bk, v);
    __syncthreads();
    par ^= 1;
  }
  cl_sync();  // uniform end
  if (aborted) {
    // every CTA issued its last partial-vector stores before it arrived at the barrier above;
    // leave them time to land in this CTA's shared memory before it is released
    const long long t0 = clock64();
    while (clock64() - t0 < kDrainCycles) {
    }
    return;
  }
  // write the finished slice back
#pragma unroll
  for (int k = 0; k < CPW; ++k) {
    const int a = warp + kNW * k;
    if (a < bk)
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const int r = 64 * i + 2 * lane;
        float x0, x1;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(x0), "=f"(x1) : "l"(P[k][i]));
        if (r < nr) Q[row0 + r + a * ldq] = x0;
        if (r + 1 < nr) Q[row0 + r + 1 + a * ldq] = x1;
      }
  }
}

// Latency floor of k_panel_reg's per-column exchange (a measurement aid; the paper has no
// counterpart): the exchanges one panel of bk columns performs -- the first one of 256 + bk
// entries, then entries j+1 .. bk-1 for j = 0 .. bk-2 -- `reps` times, through the same
// reg_exchange and reg_gather with the panel's launch shape and shared-memory footprint, and
// no column arithmetic.  Each CTA's partial of entry a is a + 1, so every sum must come back
// as G (a + 1) exactly; *bad counts the entries that did not.
__global__ void __launch_bounds__(kNT, 1) k_exchange_probe_reg(int bk, int reps, int rpc,
                                                               int* status, int* bad,
                                                               long long wait_limit) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* lpart = reinterpret_cast<float*>(smraw) + 4 * (size_t)rpc;  // the panel's layout
  float* rbuf = lpart + 2 * 512;
  float* v = rbuf + 2 * kMaxG * 512;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(v + 512 + 256 + (size_t)kNW * rpc);
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(mbar, 1);
    mbar_init(mbar + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  cl_sync();
  const float G = (float)gridDim.x;
  unsigned phases = 0u;
  int par = 0, wrong = 0;
  bool ok = true;
  for (int rep = 0; rep < reps && ok; ++rep)
    for (int j = -1; j < bk - 1 && ok; ++j) {
      const int lo = j < 0 ? 0 : j + 1, hi = j < 0 ? 256 + bk : bk;
      for (int a = lo + tid; a < hi; a += kNT) lpart[par * 512 + a] = (float)(a + 1);
      ok = reg_exchange(lpart, rbuf, mbar, phases, par, lo, hi, wait_limit, status);
      if (ok) {
        reg_gather(rbuf, par, lo, hi, v);
        __syncthreads();
        for (int a = lo + tid; a < hi; a += kNT) wrong += v[a] != G * (float)(a + 1);
      }
      __syncthreads();
      par ^= 1;
    }
  if (wrong) atomicAdd(bad, wrong);
  cl_sync();  // uniform end
  if (!ok) {
    const long long t0 = clock64();
    while (clock64() - t0 < kDrainCycles) {
    }
  }
}

size_t reg_smem_bytes(int rpl) {
  const size_t rpc = 32 * (size_t)rpl;
  return (4 * rpc + 2 * 512 + 2 * (size_t)kMaxG * 512 + 512 + 256 + (size_t)kNW * rpc) * sizeof(float) +
         2 * sizeof(uint64_t) + 256;
}

template <int RPL, int CPW>
const void* reg_fn() { return (const void*)k_panel_reg<RPL, CPW>; }

const void* pick_reg(int rpl, int cpw) {
#define CQR_REG_CASE(R_, C_) \
  if (rpl == R_ && cpw == C_) return reg_fn<R_, C_>();
  CQR_REG_CASE(4, 4) CQR_REG_CASE(4, 8) CQR_REG_CASE(4, 16)
  CQR_REG_CASE(6, 4) CQR_REG_CASE(6, 8) CQR_REG_CASE(6, 16)
  CQR_REG_CASE(8, 4) CQR_REG_CASE(8, 8) CQR_REG_CASE(8, 16)
  CQR_REG_CASE(10, 4) CQR_REG_CASE(10, 8) CQR_REG_CASE(10, 16)
  CQR_REG_CASE(12, 4) CQR_REG_CASE(12, 8)
#undef CQR_REG_CASE
  return nullptr;
}

}  // namespace

// Register plan for an FP32 panel of M rows and bk columns: rows per lane (even) and columns
// per warp; false when the slice does not fit one cluster's registers.
bool plan_panel_reg(int64_t M, int bk, int* rpl_out, int* cpw_out, int* G_out) {
  if (bk > 128) return false;
  const int cpw = bk <= 32 ? 4 : bk <= 64 ? 8 : 16;
  for (int rpl : {4, 6, 8, 10, 12}) {
    if (cpw == 16 && rpl > 10) break;
    const int64_t G = (M + 32LL * rpl - 1) / (32LL * rpl);
    if (G <= kMaxG) {
      *rpl_out = rpl;
      *cpw_out = cpw;
      *G_out = (int)G;
      return pick_reg(rpl, cpw) != nullptr;
    }
  }
  return false;
}

cudaError_t launch_panel_reg(int rpl, int cpw, int G, float* Q, int64_t ldq, float* R, int64_t ldr,
                             int64_t M, int bk, double tau, int* status, int col0, cudaStream_t st,
                             bool pdl, long long wait_limit) {
  const void* fn = pick_reg(rpl, cpw);
  if (!fn) return cudaErrorInvalidValue;
  const size_t smem = reg_smem_bytes(rpl);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (G > 8) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  double tau2 = tau > 0.0 ? tau * tau : -1.0;
  long long wl = wait_limit > 0 ? wait_limit : kWaitLimitCycles;
  void* args[] = {&Q, &ldq, &R, &ldr, &M, &bk, &tau2, &status, &col0, &wl};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kNT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = G;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 2 : 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

bool panel_reg_cluster_fits(int rpl, int cpw, int G) {
  const void* fn = pick_reg(rpl, cpw);
  if (!fn) return false;
  const size_t smem = reg_smem_bytes(rpl);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return false;
  if (G > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kNT);
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
    return false;
  }
  return n >= 1;
}

// One launch of the register-panel exchange probe for a panel of M rows and bk columns (the
// register panel's plan: its cluster of G CTAs and its shared-memory footprint).
cudaError_t launch_exchange_probe_reg(int64_t M, int bk, int reps, int* status, int* bad,
                                      cudaStream_t st) {
  int rpl = 0, cpw = 0, G = 0;
  if (!plan_panel_reg(M, bk, &rpl, &cpw, &G) || !panel_reg_cluster_fits(rpl, cpw, G))
    return cudaErrorInvalidValue;
  const void* fn = (const void*)k_exchange_probe_reg;
  const size_t smem = reg_smem_bytes(rpl);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && G > 8)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  int rpc = 32 * rpl;
  long long wl = kWaitLimitCycles;
  void* args[] = {&bk, &reps, &rpc, &status, &bad, &wl};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kNT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = G;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t bounds_take_panel_reg(int* code, int* site) { return bounds_take_here(code, site); }

}  // namespace cqr
