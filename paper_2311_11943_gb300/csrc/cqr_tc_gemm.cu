// cqr_tc_gemm.cu -- tensor-core trailing update of PBMGS for FP32 storage (sm_103a):
//   GEMM1  Rbar = Qbar^T Q[:, j0:j0+w]        (M_mma = panel columns, K = all M rows, split-K)
//   GEMM2  Q[:, j0:j0+w] -= Qbar Rbar          (M_mma = rows, K = panel width)
// (Appendix A, Algorithm PBMGS, the All-reduce product and the trailing update.)
//
// One persistent, warp-specialised kernel computes D = sum_p A_p B_p^T for up to three
// (A_p, B_p) operand pairs, every operand K-major, with tcgen05.mma kind::tf32 (M = 128,
// N = 128, K = 8 per instruction) accumulating in tensor memory (TMEM, FP32):
//   warp 0      TMA producer: cp.async.bulk.tensor tiles (128-byte swizzle) into a ring of
//               shared-memory stages, completion counted on an mbarrier per stage
//   warp 1      allocates TMEM; one thread issues the MMAs and tcgen05.commit's each stage
//               back to the producer and each finished tile to the epilogue
//   warps 2-3   3xTF32 only: split the streamed B tile in shared memory into hi = rna_tf32(x)
//               (in place) and lo = x - hi (second buffer)
//   warps 4-7   epilogue: tcgen05.ld 32 lanes x 32 columns per warp, then either store the
//               FP32 partial (GEMM1) or subtract it from Q in place (GEMM2)
// 3xTF32 (hi*hi + hi*lo + lo*hi) recovers about FP32 accuracy from TF32 products.  The small
// operands (panel and Rbar) are split into hi/lo planes in global memory by helper kernels.
// Every mbarrier wait is bounded: on expiry the kernel records CQR_ETIMEOUT, stops issuing,
// waits (bounded) for its own copies, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "coded_qr.h"
#include "cqr_device.cuh"
#include "cqr_tc_gemm.cuh"

namespace cqr {

namespace {

constexpr int BM = 128;       // UMMA M (TMEM lanes)
constexpr int BN = 128;       // UMMA N (TMEM columns)
constexpr int kTmemCols = 2 * BN;  // two accumulator buffers (power of two, <= 512)
constexpr int BK = 32;        // K per stage: 32 FP32 = 128 bytes = one swizzle row
constexpr int UMMA_K = 8;     // K per tcgen05.mma kind::tf32
constexpr int kThreads = 256;
constexpr int kMaxSplits = 16;
constexpr uint32_t kTileBytesA = BM * BK * 4;  // 16 KB
constexpr uint32_t kTileBytesB = BN * BK * 4;  // 16 KB

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of barrier b.  Returns false (and raises the CTA's abort
// flag) when the limit is reached or another role already aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
  if (mbar_test(b, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(b, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitLimitCycles) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* tm) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tm)) : "memory");
}

// tcgen05 shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused with this swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // version
  d |= (uint64_t)2 << 61;             // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::tf32: D FP32, A/B TF32, both K-major, N and M encoded.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem_d), "l"(a), "l"(b), "r"(kIdesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   su32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// ------------------------------------------------------------------ the GEMM kernel
struct TcMaps {
  CUtensorMap a[2];  // A hi / lo (lo unused for one product)
  CUtensorMap b[2];  // B hi / lo; with an in-smem split only b[0] (raw FP32) is loaded
};

struct TcJob {
  int nprod;          // 1 (TF32) or 3 (3xTF32)
  int split_b_smem;   // 1: B arrives raw and is split in shared memory
  int epi;            // 0: store partial P[s] ; 1: C -= D
  int m_tiles, n_tiles, splits;
  int64_t a_row0;     // A tile y coordinate offset (rows of the MMA M dimension)
  int64_t b_row0;     // B tile y coordinate offset
  int64_t k0;         // K start
  int64_t kchunk;     // K per split (multiple of BK)
  int64_t K;          // K end (exclusive)
  int64_t mrows;      // valid D rows (M dimension)
  int64_t ncols;      // valid D columns (N dimension)
  float* out;         // epi 0: P base; epi 1: C base (already offset to column j0)
  int64_t ldo;        // leading dimension of out
  int64_t split_stride;  // epi 0: elements between split partials
  int* status;
};

template <int STAGES, int NA, int NB>
struct Smem {
  // per stage: NA A tiles then NB B tiles (each 1024-byte aligned, 16 KB)
  static constexpr uint32_t kStageBytes = NA * kTileBytesA + NB * kTileBytesB;
  static constexpr uint32_t kTiles = STAGES * kStageBytes;
  static constexpr uint32_t kTotal = kTiles + 1024 /*alignment*/ + 256 /*barriers*/;
  // full/ready/empty per stage, acc_full[2], acc_empty[2], TMEM slot, abort flag
  static_assert(STAGES * 3 * 8 + 4 * 8 + 8 <= 256, "barrier region too small");
};

template <int STAGES, int NA, int NB>
__global__ void __launch_bounds__(kThreads, 1) k_tc_gemm(const __grid_constant__ TcMaps maps,
                                                          const TcJob job) {
  using S = Smem<STAGES, NA, NB>;
  extern __shared__ __align__(1024) unsigned char smraw[];
  const uint32_t base_u = su32(smraw);
  const uint32_t tiles_u = (base_u + 1023u) & ~1023u;
  unsigned char* tiles = smraw + (tiles_u - base_u);
  uint64_t* full = reinterpret_cast<uint64_t*>(tiles + S::kTiles);
  uint64_t* ready = full + STAGES;     // B split done (3xTF32 in-smem split)
  uint64_t* empty = ready + STAGES;
  uint64_t* acc_full = empty + STAGES;  // [2]: one per TMEM accumulator buffer
  uint64_t* acc_empty = acc_full + 2;   // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int total_tiles = job.m_tiles * job.n_tiles * job.splits;
  const int nkb_full = (int)(job.kchunk / BK);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&ready[s], 64);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    prefetch_tmap(&maps.a[0]);
    prefetch_tmap(&maps.b[0]);
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_slot)),
                 "r"((uint32_t)kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // K blocks of tile t
  auto kblocks = [&](int split) -> int {
    const int64_t k0 = job.k0 + (int64_t)split * job.kchunk;
    int64_t k1 = k0 + job.kchunk;
    if (k1 > job.K) k1 = job.K;
    const int64_t n = k1 > k0 ? (k1 - k0 + BK - 1) / BK : 0;
    return (int)(n < nkb_full ? n : nkb_full);
  };

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      for (int t = blockIdx.x; t < total_tiles && !*abort_flag; t += gridDim.x) {
        const int split = t % job.splits;
        const int mn = t / job.splits;
        const int mt = mn % job.m_tiles, nt = mn / job.m_tiles;
        const int nk = kblocks(split);
        const int64_t kbase = job.k0 + (int64_t)split * job.kchunk;
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % STAGES;
          if (!mbar_wait(&empty[s], ((it / STAGES) & 1) ^ 1, abort_flag)) break;
          const uint32_t st = tiles_u + s * S::kStageBytes;
          const int x = (int)(kbase + (int64_t)kb * BK);
          const int ya = (int)(job.a_row0 + (int64_t)mt * BM);
          const int yb = (int)(job.b_row0 + (int64_t)nt * BN);
          const int nb_load = job.split_b_smem ? 1 : NB;
          mbar_expect_tx(&full[s], NA * kTileBytesA + nb_load * kTileBytesB);
          for (int p = 0; p < NA; ++p) tma_load_2d(st + p * kTileBytesA, &maps.a[p], x, ya, &full[s]);
          for (int p = 0; p < nb_load; ++p)
            tma_load_2d(st + NA * kTileBytesA + p * kTileBytesB, &maps.b[p], x, yb, &full[s]);
        }
      }
      // the last load issued into each stage has landed before the CTA may exit (bounded)
      for (int i = (it > STAGES ? it - STAGES : 0); i < it; ++i) {
        const long long t0 = clock64();
        while (!mbar_test(&full[i % STAGES], (i / STAGES) & 1) && clock64() - t0 < kWaitLimitCycles) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int it = 0, tl = 0;
      for (int t = blockIdx.x; t < total_tiles && !*abort_flag; t += gridDim.x, ++tl) {
        const int split = t % job.splits;
        const int nk = kblocks(split);
        // two accumulators: the epilogue drains tile tl-1 while tile tl accumulates
        const int buf = tl & 1;
        const uint32_t acc = tmem + (uint32_t)(buf * BN);
        if (!mbar_wait(&acc_empty[buf], ((tl >> 1) & 1) ^ 1, abort_flag)) break;
        tc_fence_after();
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % STAGES;
          uint64_t* gate = job.split_b_smem ? &ready[s] : &full[s];
          if (!mbar_wait(gate, (it / STAGES) & 1, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t st = tiles_u + s * S::kStageBytes;
          const uint32_t a_hi = st, a_lo = st + kTileBytesA;
          const uint32_t b_hi = st + NA * kTileBytesA, b_lo = b_hi + kTileBytesB;
#pragma unroll
          for (int ks = 0; ks < BK / UMMA_K; ++ks) {
            const uint32_t off = ks * UMMA_K * 4;
            const uint32_t acc0 = (kb > 0 || ks > 0) ? 1u : 0u;
            mma_tf32(acc, sdesc(a_hi + off), sdesc(b_hi + off), acc0);
            if (job.nprod == 3) {
              mma_tf32(acc, sdesc(a_hi + off), sdesc(b_lo + off), 1u);
              mma_tf32(acc, sdesc(a_lo + off), sdesc(b_hi + off), 1u);
            }
          }
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&acc_full[buf]);
      }
    }
  } else if (warp == 2 || warp == 3) {
    if (job.split_b_smem) {
      const int tt = threadIdx.x - 64;  // 0..63
      int it = 0;
      for (int t = blockIdx.x; t < total_tiles && !*abort_flag; t += gridDim.x) {
        const int split = t % job.splits;
        const int nk = kblocks(split);
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % STAGES;
          if (!mbar_wait(&full[s], (it / STAGES) & 1, abort_flag)) { ok = false; break; }
          float4* raw = reinterpret_cast<float4*>(tiles + s * S::kStageBytes + NA * kTileBytesA);
          float4* lo = raw + kTileBytesB / 16;
          for (int e = tt; e < (int)(kTileBytesB / 16); e += 64) {
            const float4 x = raw[e];
            float4 h, l;
            h.x = tf32_hi(x.x); l.x = x.x - h.x;
            h.y = tf32_hi(x.y); l.y = x.y - h.y;
            h.z = tf32_hi(x.z); l.z = x.z - h.z;
            h.w = tf32_hi(x.w); l.w = x.w - h.w;
            raw[e] = h;
            lo[e] = l;
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive(&ready[s]);
        }
        if (!ok) break;
      }
    }
  } else {
    // epilogue warps 4..7: TMEM lanes 32 (warp % 4) .. +32
    const int ew = warp & 3;
    int tl = 0;
    for (int t = blockIdx.x; t < total_tiles && !*abort_flag; t += gridDim.x, ++tl) {
      const int split = t % job.splits;
      const int mn = t / job.splits;
      const int mt = mn % job.m_tiles, nt = mn / job.m_tiles;
      const int buf = tl & 1;
      if (!mbar_wait(&acc_full[buf], (tl >> 1) & 1, abort_flag)) break;
      tc_fence_after();
      const int64_t row = (int64_t)mt * BM + ew * 32 + lane;
      const bool row_ok = row < job.mrows;
      const bool has_k = kblocks(split) > 0;
#pragma unroll 1
      for (int c = 0; c < BN / 32; ++c) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(buf * BN + c * 32), v);
        if (!has_k)
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = 0.f;
        const int64_t col0 = (int64_t)nt * BN + c * 32;
        if (job.epi == 0) {
          float* o = job.out + (int64_t)split * job.split_stride;
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int64_t col = col0 + i;
            if (row_ok && col < job.ncols) o[row + col * job.ldo] = v[i];
          }
        } else {
          float old[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int64_t col = col0 + i;
            old[i] = (row_ok && col < job.ncols) ? job.out[row + col * job.ldo] : 0.f;
          }
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int64_t col = col0 + i;
            if (row_ok && col < job.ncols) job.out[row + col * job.ldo] = old[i] - v[i];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
  }

  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) set_status(job.status, CQR_ETIMEOUT, 20);
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)kTmemCols)
                 : "memory");
  }
}

// ------------------------------------------------------------------ helper kernels
// Panel split: Qbar = Q[:, kb : kb+bk] (M x bk) -> for GEMM1's A (column-major, ld ldk):
// Ak_hi / Ak_lo; for GEMM2's A (row-major, row stride bkp): At_hi / At_lo; columns k >= bk
// zero-filled up to bkp (and up to 128 columns for GEMM1's M tile).  With Qr != nullptr the
// finished panel is also copied into the row-major planes of all computed columns
// (Qr[r * ldrow + kb + k]), the K-major operand of the block reorthogonalisation.
__global__ void k_split_panel(const float* __restrict__ Q, int64_t ldq, int64_t M, int bk, int bkp,
                              int ak_cols, int nplanes, float* __restrict__ Ak_hi,
                              float* __restrict__ Ak_lo, int64_t ldk, float* __restrict__ At_hi,
                              float* __restrict__ At_lo, float* __restrict__ Qr_hi,
                              float* __restrict__ Qr_lo, int64_t ldrow, int64_t kb) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (r >= M) return;
  const float x = (k < bk) ? Q[r + (int64_t)k * ldq] : 0.f;
  const float h = nplanes == 2 ? tf32_hi(x) : x;
  const float l = x - h;
  if (k < ak_cols) {
    if (Ak_hi) Ak_hi[r + (int64_t)k * ldk] = h;
    if (Ak_lo && nplanes == 2) Ak_lo[r + (int64_t)k * ldk] = l;
  }
  if (k < bkp) {
    At_hi[r * bkp + k] = h;
    if (nplanes == 2) At_lo[r * bkp + k] = l;
  }
  if (Qr_hi && k < bk) {
    Qr_hi[r * ldrow + kb + k] = h;
    if (nplanes == 2) Qr_lo[r * ldrow + kb + k] = l;
  }
}

// C -= sum_s P[s] in a fixed order of s (split-K partials of a C -= A B update; P[s] is
// mrows x ncols column-major with leading dimension mrows).
__global__ void k_tc_sub_partials(const float* __restrict__ P, int splits, int64_t mrows,
                                  int64_t ncols, float* __restrict__ C, int64_t ldc) {
  const int64_t total = mrows * ncols;
  const int64_t stride = total;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx % mrows, c = idx / mrows;
    float s = 0.f;
    for (int sp = 0; sp < splits; ++sp) s += __ldcs(P + sp * stride + idx);
    C[r + c * ldc] -= s;
  }
}

// Row-major planes of the computed columns 0 .. ncols-1 from Q (after a recovery).
__global__ void k_refresh_rows(const float* __restrict__ Q, int64_t ldq, int64_t M, int64_t ncols,
                               int nplanes, float* __restrict__ Qr_hi, float* __restrict__ Qr_lo,
                               int64_t ldrow) {
  const int64_t total = M * ncols;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx % M, c = idx / M;
    const float x = Q[r + c * ldq];
    const float h = nplanes == 2 ? tf32_hi(x) : x;
    Qr_hi[r * ldrow + c] = h;
    if (nplanes == 2) Qr_lo[r * ldrow + c] = x - h;
  }
}

// Block reorthogonalisation, reduce: the GEMM1 partials hold S^T = Qbar^T Q[:, 0:kb]
// (P[s][i + j bkp]); R[j, kb+i] += S[j][i] and S (column-major, ld ldrow, rows >= kb zero)
// goes into the B planes of the second product.
__global__ void k_tc_reduce_t(const float* __restrict__ P, int splits, int64_t split_stride,
                              int64_t ldp, int bk, int64_t kb, int64_t kbp, float* __restrict__ R,
                              int64_t ldr, int nplanes, float* __restrict__ Sh,
                              float* __restrict__ Sl, int64_t ldrow) {
  const int64_t total = kbp * bk;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx % kbp, i = idx / kbp;
    float s = 0.f;
    if (j < kb) {
      for (int sp = 0; sp < splits; ++sp) s += P[sp * split_stride + i + j * ldp];
      R[j + (kb + i) * ldr] += s;
    }
    const float h = nplanes == 2 ? tf32_hi(s) : s;
    Sh[j + i * ldrow] = h;
    if (nplanes == 2) Sl[j + i * ldrow] = s - h;
  }
}

// Split-K reduction of GEMM1: Rbar = sum_s P[s] (fixed order) into R (rows kb.., columns
// j0..) and into GEMM2's B operand planes (column-major, ld bkp, rows >= bk zero).
__global__ void k_tc_reduce(const float* __restrict__ P, int splits, int64_t split_stride, int64_t ldp,
                            int bk, int bkp, int64_t w, float* __restrict__ R, int64_t ldr,
                            int nplanes, float* __restrict__ Bh, float* __restrict__ Bl) {
  const int64_t total = (int64_t)bkp * w;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % bkp, j = idx / bkp;
    float s = 0.f;
    if (i < bk) {
      for (int sp = 0; sp < splits; ++sp) s += P[sp * split_stride + i + j * ldp];
      R[i + j * ldr] = s;
    }
    const float h = nplanes == 2 ? tf32_hi(s) : s;
    Bh[idx] = h;
    if (nplanes == 2) Bl[idx] = s - h;
  }
}

}  // namespace

// ------------------------------------------------------------------ host side
struct TcGemm {
  int mode;           // CQR_MMA_TF32 | CQR_MMA_3XTF32
  int nplanes;        // 1 or 2
  int64_t M, N, b, bkp, ldq, ldk;
  float* Q;
  float *Ak_hi, *Ak_lo, *At_hi, *At_lo, *Bh, *Bl, *P;
  float *Qr_hi, *Qr_lo, *Sh, *Sl;   // block reorthogonalisation operands
  int64_t n, ldrow;
  int num_sms;
  int* status;
  CUtensorMap tm_q_b;     // Q as GEMM1's B (box 32 x BN)
  CUtensorMap tm_ak[2];   // panel, column-major (box 32 x BM)
  CUtensorMap tm_at[2];   // panel, row-major (box 32 x BM)
  CUtensorMap tm_bh[2];   // Rbar planes (box 32 x BN)
  CUtensorMap tm_qr[2];   // computed columns, row-major (box 32 x BM)
  CUtensorMap tm_s[2];    // S planes, column-major ld ldrow (box 32 x BN)
};

namespace {

// The driver's tensor-map encoder, resolved through the runtime (the library does not link
// the driver library, so it loads on machines without a GPU driver).
PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool encode_2d(CUtensorMap* tm, void* base, uint64_t inner, uint64_t outer, uint64_t row_bytes,
               uint32_t box_inner, uint32_t box_outer) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es,
                                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

template <int STAGES, int NA, int NB>
cudaError_t launch_gemm(const TcMaps& maps, const TcJob& job, int num_sms, cudaStream_t st) {
  using S = Smem<STAGES, NA, NB>;
  const void* fn = (const void*)k_tc_gemm<STAGES, NA, NB>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kTotal);
  if (e != cudaSuccess) return e;
  const int tiles = job.m_tiles * job.n_tiles * job.splits;
  const int grid = std::max(1, std::min(tiles, num_sms));
  k_tc_gemm<STAGES, NA, NB><<<grid, kThreads, S::kTotal, st>>>(maps, job);
  return cudaGetLastError();
}

}  // namespace

bool tc_available() { return true; }

size_t tc_panel_bytes(int64_t, int) { return 0; }

size_t tc_workspace_bytes(int64_t M, int64_t N, int64_t n, int b, int reorth_block) {
  const int64_t bkp = (b + BK - 1) / BK * BK;
  const int64_t ldk = (M + 31) / 32 * 32;
  const int64_t akc = std::max<int64_t>(bkp, (b + BM - 1) / BM * BM);
  const int64_t ldrow = (n + 31) / 32 * 32;
  size_t s = 0;
  s += 2 * al256((size_t)ldk * akc * 4);        // Ak hi/lo
  s += 2 * al256((size_t)M * bkp * 4);          // At hi/lo
  s += 2 * al256((size_t)bkp * N * 4);          // Rbar planes
  s += al256((size_t)kMaxSplits * bkp * N * 4);  // split-K partials
  if (reorth_block) {
    s += 2 * al256((size_t)M * ldrow * 4);      // row-major computed columns hi/lo
    s += 2 * al256((size_t)ldrow * akc * 4);    // S planes
  }
  return s;
}

TcGemm* tc_create(int mode, int64_t M, int64_t N, int64_t n, int64_t b, float* Q, int64_t ldq,
                  void* ws, int num_sms, int reorth_block, cudaStream_t st) {
  TcGemm* t = new (std::nothrow) TcGemm();
  if (!t) return nullptr;
  t->mode = mode;
  t->nplanes = mode == CQR_MMA_3XTF32 ? 2 : 1;
  t->M = M;
  t->N = N;
  t->b = b;
  t->bkp = (b + BK - 1) / BK * BK;
  t->ldq = ldq;
  t->ldk = (M + 31) / 32 * 32;
  t->Q = Q;
  t->num_sms = num_sms;
  const int64_t akc = std::max<int64_t>(t->bkp, (b + BM - 1) / BM * BM);
  char* p = static_cast<char*>(ws);
  auto take = [&](size_t bytes) { char* r = p; p += al256(bytes); return reinterpret_cast<float*>(r); };
  t->Ak_hi = take((size_t)t->ldk * akc * 4);
  t->Ak_lo = take((size_t)t->ldk * akc * 4);
  t->At_hi = take((size_t)M * t->bkp * 4);
  t->At_lo = take((size_t)M * t->bkp * 4);
  t->Bh = take((size_t)t->bkp * N * 4);
  t->Bl = take((size_t)t->bkp * N * 4);
  t->P = take((size_t)kMaxSplits * t->bkp * N * 4);
  t->n = n;
  t->ldrow = (n + 31) / 32 * 32;
  t->Qr_hi = t->Qr_lo = t->Sh = t->Sl = nullptr;
  if (reorth_block) {
    t->Qr_hi = take((size_t)M * t->ldrow * 4);
    t->Qr_lo = take((size_t)M * t->ldrow * 4);
    t->Sh = take((size_t)t->ldrow * akc * 4);
    t->Sl = take((size_t)t->ldrow * akc * 4);
    // columns not yet computed are read (times zero rows of S) when kb is not a multiple of
    // 32: keep them finite
    if (cudaMemsetAsync(t->Qr_hi, 0, (size_t)M * t->ldrow * 4, st) != cudaSuccess ||
        cudaMemsetAsync(t->Qr_lo, 0, (size_t)M * t->ldrow * 4, st) != cudaSuccess) {
      delete t;
      return nullptr;
    }
  }
  bool ok = true;
  ok &= encode_2d(&t->tm_q_b, Q, (uint64_t)M, (uint64_t)N, (uint64_t)ldq * 4, BK, BN);
  ok &= encode_2d(&t->tm_ak[0], t->Ak_hi, (uint64_t)M, (uint64_t)akc, (uint64_t)t->ldk * 4, BK, BM);
  ok &= encode_2d(&t->tm_ak[1], t->Ak_lo, (uint64_t)M, (uint64_t)akc, (uint64_t)t->ldk * 4, BK, BM);
  ok &= encode_2d(&t->tm_at[0], t->At_hi, (uint64_t)t->bkp, (uint64_t)M, (uint64_t)t->bkp * 4, BK, BM);
  ok &= encode_2d(&t->tm_at[1], t->At_lo, (uint64_t)t->bkp, (uint64_t)M, (uint64_t)t->bkp * 4, BK, BM);
  ok &= encode_2d(&t->tm_bh[0], t->Bh, (uint64_t)t->bkp, (uint64_t)N, (uint64_t)t->bkp * 4, BK, BN);
  ok &= encode_2d(&t->tm_bh[1], t->Bl, (uint64_t)t->bkp, (uint64_t)N, (uint64_t)t->bkp * 4, BK, BN);
  if (reorth_block) {
    ok &= encode_2d(&t->tm_qr[0], t->Qr_hi, (uint64_t)t->ldrow, (uint64_t)M, (uint64_t)t->ldrow * 4, BK, BM);
    ok &= encode_2d(&t->tm_qr[1], t->Qr_lo, (uint64_t)t->ldrow, (uint64_t)M, (uint64_t)t->ldrow * 4, BK, BM);
    ok &= encode_2d(&t->tm_s[0], t->Sh, (uint64_t)t->ldrow, (uint64_t)akc, (uint64_t)t->ldrow * 4, BK, BN);
    ok &= encode_2d(&t->tm_s[1], t->Sl, (uint64_t)t->ldrow, (uint64_t)akc, (uint64_t)t->ldrow * 4, BK, BN);
  }
  if (!ok) {
    delete t;
    return nullptr;
  }
  return t;
}

void tc_destroy(TcGemm* t) { delete t; }

void tc_set_status(TcGemm* t, int* status) { t->status = status; }

namespace {
int tc_splits(const TcGemm* t, int m1, int n1, int64_t* kchunk) {
  int splits = (int)std::max<int64_t>(1, std::min<int64_t>(kMaxSplits, (t->num_sms + m1 * n1 - 1) / (m1 * n1)));
  const int64_t kblocks = (t->M + BK - 1) / BK;
  if (splits > kblocks) splits = (int)kblocks;
  *kchunk = (kblocks + splits - 1) / splits * BK;
  return (int)((t->M + *kchunk - 1) / *kchunk);
}
}  // namespace

// 1. split the panel Q[:, kb : kb+bk] into the operand planes of both GEMMs (and, for a
//    finished panel with block reorthogonalisation on, into the row-major computed columns)
cudaError_t tc_split_panel(TcGemm* t, int64_t kb, int bk, bool finished, cudaStream_t st) {
  const int bkp = (int)((bk + BK - 1) / BK * BK);
  const int m1 = (bk + BM - 1) / BM;
  dim3 grd((unsigned)((t->M + 255) / 256), (unsigned)std::max(bkp, m1 * BM));
  float* qh = finished ? t->Qr_hi : nullptr;
  k_split_panel<<<grd, 256, 0, st>>>(t->Q + kb * t->ldq, t->ldq, t->M, bk, bkp, m1 * BM, t->nplanes,
                                     t->Ak_hi, t->Ak_lo, t->ldk, t->At_hi, t->At_lo, qh, t->Qr_lo,
                                     t->ldrow, kb);
  return cudaGetLastError();
}

bool tc_has_block_reorth(const TcGemm* t) { return t->Qr_hi != nullptr; }

// Row-major planes of columns 0 .. ncols-1 rebuilt from Q (after a recovery changed tiles).
cudaError_t tc_refresh_rows(TcGemm* t, int64_t ncols, cudaStream_t st) {
  if (!t->Qr_hi || ncols <= 0) return cudaSuccess;
  const int64_t total = t->M * ncols;
  const int blocks = (int)std::min<int64_t>(8192, (total + 255) / 256);
  k_refresh_rows<<<blocks, 256, 0, st>>>(t->Q, t->ldq, t->M, ncols, t->nplanes, t->Qr_hi, t->Qr_lo,
                                         t->ldrow);
  return cudaGetLastError();
}

// 2. GEMM1, split-K over the M rows: partials P[s] = Qbar^T Q[:, j0 : j0+w]
cudaError_t tc_gemm_rbar(TcGemm* t, int bk, int64_t j0, int64_t w, cudaStream_t st) {
  const int three = t->nplanes == 2;
  const int bkp = (int)((bk + BK - 1) / BK * BK);
  const int m1 = (bk + BM - 1) / BM;
  const int n1 = (int)((w + BN - 1) / BN);
  int64_t kchunk = 0;
  const int splits = tc_splits(t, m1, n1, &kchunk);
  TcMaps maps;
  maps.a[0] = t->tm_ak[0];
  maps.a[1] = t->tm_ak[1];
  maps.b[0] = t->tm_q_b;
  maps.b[1] = t->tm_q_b;
  TcJob job{};
  job.nprod = three ? 3 : 1;
  job.split_b_smem = three;
  job.epi = 0;
  job.m_tiles = m1;
  job.n_tiles = n1;
  job.splits = splits;
  job.a_row0 = 0;
  job.b_row0 = j0;
  job.k0 = 0;
  job.kchunk = kchunk;
  job.K = t->M;
  job.mrows = bk;
  job.ncols = w;
  job.out = t->P;
  job.ldo = bkp;
  job.split_stride = (int64_t)bkp * w;
  job.status = t->status;
  return three ? launch_gemm<3, 2, 2>(maps, job, t->num_sms, st)
               : launch_gemm<6, 1, 1>(maps, job, t->num_sms, st);
}

// 3. reduce the partials into R[kb.., j0..] and GEMM2's B planes
cudaError_t tc_reduce(TcGemm* t, int64_t kb, int bk, int64_t j0, int64_t w, float* R, int64_t ldr,
                      cudaStream_t st) {
  const int bkp = (int)((bk + BK - 1) / BK * BK);
  const int m1 = (bk + BM - 1) / BM;
  const int n1 = (int)((w + BN - 1) / BN);
  int64_t kchunk = 0;
  const int splits = tc_splits(t, m1, n1, &kchunk);
  const int64_t total = (int64_t)bkp * w;
  const int blocks = (int)std::min<int64_t>(4096, (total + 255) / 256);
  k_tc_reduce<<<blocks, 256, 0, st>>>(t->P, splits, (int64_t)bkp * w, bkp, bk, bkp, w,
                                      R + kb + j0 * ldr, ldr, t->nplanes, t->Bh, t->Bl);
  return cudaGetLastError();
}

// 4. GEMM2: Q[:, j0 : j0+w] -= Qbar Rbar (M tiles over rows, N tiles over trailing columns)
cudaError_t tc_gemm_update(TcGemm* t, int bk, int64_t j0, int64_t w, cudaStream_t st) {
  const int three = t->nplanes == 2;
  const int bkp = (int)((bk + BK - 1) / BK * BK);
  TcMaps maps;
  maps.a[0] = t->tm_at[0];
  maps.a[1] = t->tm_at[1];
  maps.b[0] = t->tm_bh[0];
  maps.b[1] = t->tm_bh[1];
  TcJob job{};
  job.nprod = three ? 3 : 1;
  job.split_b_smem = 0;
  job.epi = 1;
  job.m_tiles = (int)((t->M + BM - 1) / BM);
  job.n_tiles = (int)((w + BN - 1) / BN);
  job.splits = 1;
  job.a_row0 = 0;
  job.b_row0 = 0;
  job.k0 = 0;
  job.kchunk = bkp;
  job.K = bkp;
  job.mrows = t->M;
  job.ncols = w;
  job.out = t->Q + j0 * t->ldq;
  job.ldo = t->ldq;
  job.split_stride = 0;
  job.status = t->status;
  return three ? launch_gemm<3, 2, 2>(maps, job, t->num_sms, st)
               : launch_gemm<6, 1, 1>(maps, job, t->num_sms, st);
}

// Block reorthogonalisation of panel kb .. kb+bk-1 against columns 0 .. kb-1 (four
// launches: split the panel, S^T = Qbar^T Q[:, 0:kb] split-K on the tensor cores, reduce
// into R and S, Qbar -= Qrows S on the tensor cores).
cudaError_t tc_block_reorth(TcGemm* t, int64_t kb, int bk, float* R, int64_t ldr, cudaStream_t st,
                            int* launches) {
  *launches = 0;
  if (!t->Qr_hi || kb <= 0) return cudaSuccess;
  *launches = 4;
  cudaError_t e = tc_split_panel(t, kb, bk, false, st);
  if (e != cudaSuccess) return e;
  e = tc_gemm_rbar(t, bk, 0, kb, st);  // partials of S^T (bk x kb)
  if (e != cudaSuccess) return e;
  const int three = t->nplanes == 2;
  const int bkp = (int)((bk + BK - 1) / BK * BK);
  const int m1 = (bk + BM - 1) / BM;
  const int n1 = (int)((kb + BN - 1) / BN);
  int64_t kchunk = 0;
  const int splits = tc_splits(t, m1, n1, &kchunk);
  const int64_t kbp = (kb + BK - 1) / BK * BK;
  {
    const int64_t total = kbp * bk;
    const int blocks = (int)std::min<int64_t>(4096, (total + 255) / 256);
    k_tc_reduce_t<<<blocks, 256, 0, st>>>(t->P, splits, (int64_t)bkp * kb, bkp, bk, kb, kbp, R, ldr,
                                          t->nplanes, t->Sh, t->Sl, t->ldrow);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  TcMaps maps;
  maps.a[0] = t->tm_qr[0];
  maps.a[1] = t->tm_qr[1];
  maps.b[0] = t->tm_s[0];
  maps.b[1] = t->tm_s[1];
  TcJob job{};
  job.nprod = three ? 3 : 1;
  job.split_b_smem = 0;
  job.epi = 1;
  job.m_tiles = (int)((t->M + BM - 1) / BM);
  job.n_tiles = (bk + BN - 1) / BN;
  // Split K (the kb computed columns) when the M x bk output has too few tiles to fill the
  // SMs; the partials go to P (capacity kMaxSplits * bkp * N floats) and are subtracted in
  // a fixed order, so the result does not depend on the schedule.
  const int64_t kblk = kbp / BK;
  const int tiles2 = job.m_tiles * job.n_tiles;
  int64_t want = std::min<int64_t>(std::min<int64_t>(kMaxSplits, kblk), t->num_sms / std::max(1, tiles2));
  const int64_t cap = (int64_t)kMaxSplits * t->bkp * t->N / (t->M * (int64_t)bk);
  want = std::min<int64_t>(want, cap);
  int64_t kchunk2 = kbp;
  if (want > 1) kchunk2 = (kblk + want - 1) / want * BK;
  const int splits2 = (int)((kbp + kchunk2 - 1) / kchunk2);
  job.splits = splits2;
  job.a_row0 = 0;
  job.b_row0 = 0;
  job.k0 = 0;
  job.kchunk = kchunk2;
  job.K = kbp;
  job.mrows = t->M;
  job.ncols = bk;
  job.status = t->status;
  if (splits2 == 1) {
    job.epi = 1;
    job.out = t->Q + kb * t->ldq;
    job.ldo = t->ldq;
    job.split_stride = 0;
  } else {
    job.epi = 0;
    job.out = t->P;
    job.ldo = t->M;
    job.split_stride = t->M * (int64_t)bk;
  }
  e = three ? launch_gemm<3, 2, 2>(maps, job, t->num_sms, st)
            : launch_gemm<6, 1, 1>(maps, job, t->num_sms, st);
  if (e != cudaSuccess || splits2 == 1) return e;
  *launches = 5;
  const int64_t total = t->M * (int64_t)bk;
  const int blocks = (int)std::min<int64_t>((int64_t)t->num_sms * 8, (total + 255) / 256);
  k_tc_sub_partials<<<blocks, 256, 0, st>>>(t->P, splits2, t->M, bk, t->Q + kb * t->ldq, t->ldq);
  return cudaGetLastError();
}

}  // namespace cqr
