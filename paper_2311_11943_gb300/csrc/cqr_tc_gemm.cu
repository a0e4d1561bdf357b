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
//   warps 4-11  epilogue, two warps per quarter of the TMEM lanes: tcgen05.ld 32 lanes x 32
//               columns per warp (alternate column chunks), then either store the FP32
//               partial (GEMM1) or subtract it from Q in place (GEMM2)
// A work unit is one 128 x 128 output tile, or, for GEMM1 in 3xTF32 with a 256-column panel,
// the two vertically adjacent tiles of one B tile (two accumulators; B is loaded and split
// once for both).
// 3xTF32 (hi*hi + hi*lo + lo*hi) recovers about FP32 accuracy from TF32 products.  The small
// operands (panel and Rbar) are split into hi/lo planes in global memory by helper kernels.
// Every mbarrier wait is bounded: on expiry the kernel records CQR_ETIMEOUT, stops issuing,
// waits (bounded) for its own copies, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
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
// TMEM columns: two accumulator buffers of U 128 x 128 accumulators (a power of two, <= 512)
template <int U>
constexpr int tmem_cols() { return 2 * U * BN; }
constexpr int kEpiWarps = 8;  // two per TMEM lane quarter, each draining half the columns
constexpr int kThreads = 32 * (4 + kEpiWarps);
constexpr int kMaxSplits = 16;
constexpr uint32_t kTileBytesA = BM * 128;  // 16 KB: 128 rows of one 128-byte swizzle row
constexpr uint32_t kTileBytesB = BN * 128;  // 16 KB

// Operand type of the MMAs: TF32 (kind::tf32) or BF16 (kind::f16 with BF16 inputs).  One stage
// of K is one 128-byte swizzle row of the operand type, 32 TF32 or 64 BF16 elements; each
// tcgen05.mma consumes 32 bytes of it (8 TF32 or 16 BF16 elements).
template <bool BF>
struct Op {
  static constexpr int KE = BF ? 64 : 32;
  static constexpr int UK = BF ? 16 : 8;
};

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

// L2 prefetch of one tensor-map box (no shared memory, no completion to wait for)
__device__ __forceinline__ void tma_prefetch_l2(const CUtensorMap* tm, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];"
               ::"l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y)
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

// Instruction descriptor: D FP32, both operands K-major, N and M encoded; A/B format TF32
// (kind::tf32) or BF16 (kind::f16, A and B of the same type).
template <bool BF>
constexpr uint32_t idesc() {
  return (1u << 4) | ((BF ? 1u : 2u) << 7) | ((BF ? 1u : 2u) << 10) |
         ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <bool BF>
__device__ __forceinline__ void mma_op(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accum) {
  if (BF)
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc<true>()), "r"(accum)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc<false>()), "r"(accum)
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
  CUtensorMap c;     // subtract epilogue: the FP32 output (Q), boxes of 32 rows x BN columns
};

struct TcJob {
  int nprod;          // 1 (TF32) or 3 (3xTF32)
  int split_b_smem;   // 1: B arrives raw and is split in shared memory
  int epi;            // 0: store partial P[s] ; 1: C -= D
  int prefetch_c;     // epi 1: prefetch each output tile into L2 when its loads start
  int pair_n;         // B from planes: work units of two N tiles when n_tiles is even
  int64_t c_col0;     // epi 1: column of `out` in the tensor map of C
  int m_tiles, n_tiles, splits;
  int64_t a_row0;     // A tile y coordinate offset (rows of the MMA M dimension)
  int64_t b_row0;     // B tile y coordinate offset
  int64_t k0;         // K start
  int64_t kchunk;     // K per split (multiple of the stage K)
  int64_t K;          // K end (exclusive)
  int64_t mrows;      // valid D rows (M dimension)
  int64_t ncols;      // valid D columns (N dimension)
  float* out;         // epi 0: P base; epi 1: C base (already offset to column j0)
  int64_t ldo;        // leading dimension of out
  int64_t split_stride;  // epi 0: elements between split partials
  int* status;
};

template <int STAGES, int NA, int NB, int MP = 1, int NP = 1>
struct Smem {
  // per stage: NA A tiles for each of the MP M tiles, then NB B tiles for each of the NP N
  // tiles (each 1024-byte aligned, 16 KB)
  static constexpr uint32_t kStageBytes = MP * NA * kTileBytesA + NP * NB * kTileBytesB;
  static constexpr uint32_t kTiles = STAGES * kStageBytes;
  static constexpr uint32_t kTotal = kTiles + 1024 /*alignment*/ + 256 /*barriers*/;
  // full/ready/empty per stage, acc_full[2], acc_empty[2], TMEM slot, abort flag
  static_assert(STAGES * 3 * 8 + 4 * 8 + 8 <= 256, "barrier region too small");
};

// Programmatic dependent launch: a kernel launched with programmatic stream serialization may
// start while its predecessor in the stream finishes.  Every kernel here waits for the
// predecessor's completion (and memory) before touching any data, and only then lets its own
// successor launch, so at most one kernel ahead is resident and waiting.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// MP = 2: a work unit is a pair of vertically adjacent M tiles on the same N tile (m_tiles
// even): the B tile is loaded (and split) once for both, and two accumulators are formed.
// NP = 2: a pair of adjacent N tiles on the same M tile (n_tiles even, B from planes): the A
// tiles are loaded once for both.  MP NP <= 2.
template <bool BF, int STAGES, int NA, int NB, int MP, int NP>
__global__ void __launch_bounds__(kThreads, 1) k_tc_gemm(const __grid_constant__ TcMaps maps,
                                                          const TcJob job) {
  static_assert(MP * NP <= 2, "at most two accumulators per buffer");
  using S = Smem<STAGES, NA, NB, MP, NP>;
  constexpr int kAcc = MP * NP;  // accumulators per work unit
  constexpr int kTmemCols = tmem_cols<kAcc>();
  constexpr int BK = Op<BF>::KE;
  constexpr int UMMA_K = Op<BF>::UK;
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
  // the output tiles stay inside `out` (uniform over the launch: before any barrier or TMEM
  // allocation)
  CQR_CHECK(job.ldo >= job.mrows && (int64_t)job.m_tiles * BM >= job.mrows &&
                (int64_t)job.n_tiles * BN >= job.ncols && job.m_tiles % MP == 0 &&
                job.n_tiles % NP == 0 && (NP == 1 || !job.split_b_smem), 401);
  const int mu = job.m_tiles / MP;  // work units along M
  const int total_tiles = mu * (job.n_tiles / NP) * job.splits;
  const int nkb_full = (int)(job.kchunk / BK);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&ready[s], 64);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kEpiWarps);
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
  pdl_wait();
  pdl_trigger();

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
        const int mt = (mn % mu) * MP, nt = (mn / mu) * NP;  // first M and N tiles of the unit
        const int nk = kblocks(split);
        const int64_t kbase = job.k0 + (int64_t)split * job.kchunk;
        if (job.prefetch_c) {
          // the output tiles (BM rows x BN columns of C) are read by the epilogue once this
          // unit's products are done: start bringing them into L2 now
          for (int n = 0; n < NP; ++n) {
            const int y = (int)(job.c_col0 + (int64_t)(nt + n) * BN);
            for (int r = 0; r < BM; r += 32) tma_prefetch_l2(&maps.c, mt * BM + r, y);
          }
        }
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % STAGES;
          if (!mbar_wait(&empty[s], ((it / STAGES) & 1) ^ 1, abort_flag)) break;
          const uint32_t st = tiles_u + s * S::kStageBytes;
          const int x = (int)(kbase + (int64_t)kb * BK);
          const int ya = (int)(job.a_row0 + (int64_t)mt * BM);
          const int yb = (int)(job.b_row0 + (int64_t)nt * BN);
          // raw FP32 B for the in-smem split: one 32-element box (TF32) or two (BF16: 64
          // elements of K, split in place into the BF16 hi and lo tiles)
          const int nb_load = job.split_b_smem ? (BF ? 2 : 1) : NB;
          mbar_expect_tx(&full[s], MP * NA * kTileBytesA + NP * nb_load * kTileBytesB);
#pragma unroll
          for (int m = 0; m < MP; ++m)
            for (int p = 0; p < NA; ++p)
              tma_load_2d(st + (m * NA + p) * kTileBytesA, &maps.a[p], x, ya + m * BM, &full[s]);
#pragma unroll
          for (int n = 0; n < NP; ++n)
            for (int p = 0; p < nb_load; ++p) {
              const bool raw = job.split_b_smem;
              tma_load_2d(st + MP * NA * kTileBytesA + (n * NB + p) * kTileBytesB,
                          raw ? &maps.b[0] : &maps.b[p], raw ? x + 32 * p : x, yb + n * BN,
                          &full[s]);
            }
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
        // two accumulator buffers: the epilogue drains unit tl-1 while unit tl accumulates;
        // a buffer holds MP accumulators of BN columns
        const int buf = tl & 1;
        const uint32_t acc = tmem + (uint32_t)(buf * kAcc * BN);
        if (!mbar_wait(&acc_empty[buf], ((tl >> 1) & 1) ^ 1, abort_flag)) break;
        tc_fence_after();
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % STAGES;
          uint64_t* gate = job.split_b_smem ? &ready[s] : &full[s];
          if (!mbar_wait(gate, (it / STAGES) & 1, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t st = tiles_u + s * S::kStageBytes;
#pragma unroll
          for (int ks = 0; ks < BK / UMMA_K; ++ks) {
            const uint32_t off = ks * 32;  // 32 bytes of K per instruction
            const uint32_t acc0 = (kb > 0 || ks > 0) ? 1u : 0u;
#pragma unroll
            for (int m = 0; m < MP; ++m)
#pragma unroll
              for (int n = 0; n < NP; ++n) {
                const uint32_t am = acc + (uint32_t)((m * NP + n) * BN);
                const uint32_t a_hi = st + m * NA * kTileBytesA, a_lo = a_hi + kTileBytesA;
                const uint32_t b_hi = st + MP * NA * kTileBytesA + n * NB * kTileBytesB;
                const uint32_t b_lo = b_hi + kTileBytesB;
                mma_op<BF>(am, sdesc(a_hi + off), sdesc(b_hi + off), acc0);
                if (job.nprod == 3) {
                  mma_op<BF>(am, sdesc(a_hi + off), sdesc(b_lo + off), 1u);
                  mma_op<BF>(am, sdesc(a_lo + off), sdesc(b_hi + off), 1u);
                }
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
          float4* raw = reinterpret_cast<float4*>(tiles + s * S::kStageBytes + MP * NA * kTileBytesA);
          float4* lo = raw + kTileBytesB / 16;
          if (!BF) {
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
          } else {
            // row r of the two raw FP32 tiles (K 0..31 and 32..63, 16-byte chunks swizzled by
            // r % 8) becomes row r of the BF16 hi tile (first 16 KB) and lo tile (second):
            // a thread reads both raw rows before writing, and no other thread touches row r
            for (int r = tt; r < BN; r += 64) {
              float v[64];
#pragma unroll
              for (int c = 0; c < 16; ++c) {
                const int tile = c >> 3, lc = c & 7;
                const float4 x = raw[tile * (kTileBytesB / 16) + r * 8 + (lc ^ (r & 7))];
                v[4 * c] = x.x; v[4 * c + 1] = x.y; v[4 * c + 2] = x.z; v[4 * c + 3] = x.w;
              }
#pragma unroll
              for (int c = 0; c < 8; ++c) {
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                  const float a0 = v[8 * c + 2 * q], a1 = v[8 * c + 2 * q + 1];
                  const __nv_bfloat16 h0 = __float2bfloat16_rn(a0), h1 = __float2bfloat16_rn(a1);
                  const __nv_bfloat16 l0 = __float2bfloat16_rn(a0 - __bfloat162float(h0));
                  const __nv_bfloat16 l1 = __float2bfloat16_rn(a1 - __bfloat162float(h1));
                  hw[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                  lw[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                }
                const int pc = r * 8 + (c ^ (r & 7));
                reinterpret_cast<uint4*>(raw)[pc] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                if (job.nprod == 3) reinterpret_cast<uint4*>(lo)[pc] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
              }
            }
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive(&ready[s]);
        }
        if (!ok) break;
      }
    }
  } else {
    // epilogue warps 4 .. 4+kEpiWarps-1: TMEM lanes 32 (warp % 4) .. +32 (a warp may only
    // read its own quarter of the lanes); the two warps of a quarter take alternate 32-column
    // chunks (of each of the unit's MP accumulators), so twice as many loads of the output
    // tile are in flight
    const int ew = warp & 3;
    const int half = (warp - 4) >> 2;
    constexpr int kChunks = BN / 32;
    int tl = 0;
    for (int t = blockIdx.x; t < total_tiles && !*abort_flag; t += gridDim.x, ++tl) {
      const int split = t % job.splits;
      const int mn = t / job.splits;
      const int mt = (mn % mu) * MP, nt = (mn / mu) * NP;
      const int buf = tl & 1;
      if (!mbar_wait(&acc_full[buf], (tl >> 1) & 1, abort_flag)) break;
      tc_fence_after();
      const bool has_k = kblocks(split) > 0;
#pragma unroll 1
      for (int q = half; q < kAcc * kChunks; q += kEpiWarps / 4) {
        const int a = q / kChunks, c = q % kChunks;  // accumulator a = m NP + n
        const int m = a / NP, n = a % NP;
        const int64_t row = (int64_t)(mt + m) * BM + ew * 32 + lane;
        const bool row_ok = row < job.mrows;
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)((buf * kAcc + a) * BN + c * 32), v);
        if (!has_k)
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = 0.f;
        const int64_t col0 = (int64_t)(nt + n) * BN + c * 32;
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
// Operand planes: x = hi + lo with hi = rna_tf32(x) (TF32; hi = x with one product, the MMA
// reads TF32 from the FP32 word) or hi = bf16_rn(x), lo = bf16_rn(x - hi) (BF16).
__device__ __forceinline__ void hilo(float x, int nplanes, float& h, float& l) {
  h = nplanes == 2 ? tf32_hi(x) : x;
  l = x - h;
}
__device__ __forceinline__ void hilo(float x, int, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  l = __float2bfloat16_rn(x - __bfloat162float(h));
}

// One 32-row x 32-column tile per CTA: Q is read and Ak written along the rows (coalesced);
// the row-major planes (At, Qr) are written from a shared-memory transpose of the tile, so
// that consecutive threads write consecutive columns of a row.
template <typename P>
__global__ void __launch_bounds__(256) k_split_panel(const float* __restrict__ Q, int64_t ldq,
                                                     int64_t M, int bk, int bkp, int ak_cols,
                                                     int nplanes, P* __restrict__ Ak_hi,
                                                     P* __restrict__ Ak_lo, int64_t ldk,
                                                     P* __restrict__ At_hi, P* __restrict__ At_lo,
                                                     P* __restrict__ Qr_hi, P* __restrict__ Qr_lo,
                                                     int64_t ldrow, int64_t kb) {
  __shared__ P sh[32][33], sl[32][33];
  pdl_wait();
  pdl_trigger();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int k0 = blockIdx.y * 32;
  const int64_t r = r0 + tx;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = k0 + ty + 8 * i;
    const float x = (r < M && k < bk) ? Q[r + (int64_t)k * ldq] : 0.f;
    P h, l;
    hilo(x, nplanes, h, l);
    if (r < M && k < ak_cols) {
      if (Ak_hi) Ak_hi[r + (int64_t)k * ldk] = h;
      if (Ak_lo && nplanes == 2) Ak_lo[r + (int64_t)k * ldk] = l;
    }
    sh[ty + 8 * i][tx] = h;
    sl[ty + 8 * i][tx] = l;
  }
  __syncthreads();
  const int k = k0 + tx;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t rr = r0 + ty + 8 * i;
    if (rr >= M) continue;
    const P h = sh[tx][ty + 8 * i], l = sl[tx][ty + 8 * i];
    if (At_hi && k < bkp) {
      At_hi[rr * bkp + k] = h;
      if (nplanes == 2) At_lo[rr * bkp + k] = l;
    }
    if (Qr_hi && k < bk) {
      Qr_hi[rr * ldrow + kb + k] = h;
      if (nplanes == 2) Qr_lo[rr * ldrow + kb + k] = l;
    }
  }
}

// C -= sum_s P[s] in a fixed order of s (split-K partials of a C -= A B update; P[s] is
// mrows x ncols column-major with leading dimension mrows).
__global__ void k_tc_sub_partials(const float* __restrict__ P, int splits, int64_t mrows,
                                  int64_t ncols, float* __restrict__ C, int64_t ldc) {
  pdl_wait();
  pdl_trigger();
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

// Row-major planes of the rectangle rows [r0, r0 + nr) x columns [c0, c0 + nc) from Q (after a
// recovery rebuilt those tiles): 32 x 32 tiles through shared memory, coalesced both ways.
template <typename P>
__global__ void __launch_bounds__(256) k_refresh_rect(const float* __restrict__ Q, int64_t ldq,
                                                      int64_t r0, int nr, int64_t c0, int nc,
                                                      int nplanes, P* __restrict__ Qr_hi,
                                                      P* __restrict__ Qr_lo, int64_t ldrow) {
  __shared__ P sh[32][33], sl[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int rb = blockIdx.x * 32, cb = blockIdx.y * 32;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int r = rb + tx, c = cb + ty + 8 * u;
    P h, l;
    hilo((r < nr && c < nc) ? Q[r0 + r + (c0 + c) * ldq] : 0.f, nplanes, h, l);
    sh[ty + 8 * u][tx] = h;
    sl[ty + 8 * u][tx] = l;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int r = rb + ty + 8 * u, c = cb + tx;
    if (r >= nr || c >= nc) continue;
    Qr_hi[(r0 + r) * ldrow + c0 + c] = sh[tx][ty + 8 * u];
    if (nplanes == 2) Qr_lo[(r0 + r) * ldrow + c0 + c] = sl[tx][ty + 8 * u];
  }
}

// Block reorthogonalisation, reduce: the GEMM1 partials hold S^T = Qbar^T Q[:, 0:kb]
// (P[s][i + j bkp]); R[j, kb+i] += S[j][i] and S (column-major, ld ldrow, rows >= kb zero)
// goes into the B planes of the second product.  One 32 x 32 tile (i, j) per CTA: the
// partials are read along i and the sums go through shared memory, so R and S are written
// along j (both coalesced).
template <typename PT>
__global__ void __launch_bounds__(256) k_tc_reduce_t(const float* __restrict__ P, int splits,
                                                     int64_t split_stride, int64_t ldp, int bk,
                                                     int64_t kb, int64_t kbp, float* __restrict__ R,
                                                     int64_t ldr, int nplanes, PT* __restrict__ Sh,
                                                     PT* __restrict__ Sl, int64_t ldrow) {
  __shared__ float tile[32][33];
  pdl_wait();
  pdl_trigger();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i0 = blockIdx.x * 32;
  const int64_t j0 = (int64_t)blockIdx.y * 32;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + tx;
    const int64_t j = j0 + ty + 8 * u;
    float s = 0.f;
    if (i < bk && j < kb)
      for (int sp = 0; sp < splits; ++sp) s += P[sp * split_stride + i + j * ldp];
    tile[ty + 8 * u][tx] = s;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + ty + 8 * u;
    const int64_t j = j0 + tx;
    if (i >= bk || j >= kbp) continue;
    const float s = tile[tx][ty + 8 * u];
    if (j < kb) R[j + (kb + i) * ldr] += s;
    PT h, l;
    hilo(s, nplanes, h, l);
    Sh[j + i * ldrow] = h;
    if (nplanes == 2) Sl[j + i * ldrow] = l;
  }
}

// Split-K reduction of GEMM1: Rbar = sum_s P[s] (fixed order) into R (rows kb.., columns
// j0..) and into GEMM2's B operand planes (column-major, ld bkp, rows >= bk zero).
template <typename PT>
__global__ void k_tc_reduce(const float* __restrict__ P, int splits, int64_t split_stride, int64_t ldp,
                            int bk, int bkp, int64_t w, float* __restrict__ R, int64_t ldr,
                            int nplanes, PT* __restrict__ Bh, PT* __restrict__ Bl) {
  pdl_wait();
  pdl_trigger();
  const int64_t total = (int64_t)bkp * w;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % bkp, j = idx / bkp;
    float s = 0.f;
    if (i < bk) {
      for (int sp = 0; sp < splits; ++sp) s += P[sp * split_stride + i + j * ldp];
      R[i + j * ldr] = s;
    }
    PT h, l;
    hilo(s, nplanes, h, l);
    Bh[idx] = h;
    if (nplanes == 2) Bl[idx] = l;
  }
}

}  // namespace

// ------------------------------------------------------------------ host side
struct TcGemm {
  int mode;           // CQR_MMA_TF32 | _3XTF32 | _BF16 | _BF16X3
  int nplanes;        // 1 or 2
  bool bf;            // operand planes in BF16 (kind::f16) rather than TF32-in-FP32
  int KE;             // K elements per stage (32 TF32, 64 BF16)
  size_t pe;          // bytes per plane element
  int64_t M, N, b, bkp, ldq, ldk;
  float* Q;
  // panel operand planes, two buffers (panels of alternating parity), and the Rbar planes and
  // split-K partials of two update contexts (the look-ahead runs two updates concurrently)
  void *Ak_hi[2], *Ak_lo[2], *At_hi[2], *At_lo[2], *Bh[2], *Bl[2];
  float* P[2];
  void *Qr_hi, *Qr_lo, *Sh, *Sl;   // block reorthogonalisation operands
  int64_t n, ldrow;
  int num_sms;
  int* status;
  cudaStream_t pdl_st = nullptr;  // launches on this stream use programmatic dependent launch
  CUtensorMap tm_q_b;        // Q (FP32) as GEMM1's raw B (box 32 x BN)
  CUtensorMap tm_ak[2][2];   // [buffer][plane] panel, column-major (box KE x BM)
  CUtensorMap tm_at[2][2];   // [buffer][plane] panel, row-major (box KE x BM)
  CUtensorMap tm_bh[2][2];   // [context][plane] Rbar planes (box KE x BN)
  CUtensorMap tm_qr[2];      // computed columns, row-major (box KE x BM)
  CUtensorMap tm_s[2];       // S planes, column-major ld ldrow (box KE x BN)
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

bool encode_2d(CUtensorMap* tm, void* base, bool bf, uint64_t inner, uint64_t outer,
               uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(tm, bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                   base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Kernel launch, with programmatic stream serialization when pdl is set.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     bool pdl, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? at : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <bool BF, int STAGES, int NA, int NB, int MP = 1, int NP = 1>
cudaError_t launch_gemm(const TcMaps& maps, const TcJob& job, int max_ctas, cudaStream_t st, bool pdl) {
  using S = Smem<STAGES, NA, NB, MP, NP>;
  const void* fn = (const void*)k_tc_gemm<BF, STAGES, NA, NB, MP, NP>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kTotal);
  if (e != cudaSuccess) return e;
  const int tiles = job.m_tiles / MP * (job.n_tiles / NP) * job.splits;
  const int grid = std::max(1, std::min(tiles, max_ctas));
  return launch_k(k_tc_gemm<BF, STAGES, NA, NB, MP, NP>, dim3(grid), dim3(kThreads), S::kTotal, st,
                  pdl, maps, job);
}

// GEMM1-shaped launches (B raw and split in shared memory, 3xTF32) take pairs of M tiles when
// the panel spans an even number of them (b = 256): the B tile is then loaded and split once
// for both halves of the panel, which halves the B traffic into shared memory per flop.
// CQR_GEMM_PAIR=0 keeps one M tile per work unit.
bool pair_m_tiles(bool three, bool bf, bool split, int m_tiles) {
  static const int env = [] {
    const char* e = getenv("CQR_GEMM_PAIR");
    return e ? atoi(e) : 1;
  }();
  return env != 0 && three && !bf && split && m_tiles % 2 == 0;
}

// Launches whose B comes from planes (GEMM2 and the block pass's second product) take pairs of
// N tiles when the job asks for it (TcJob::pair_n) and n_tiles is even: the A tiles are then
// loaded once for both.  CQR_GEMM_NPAIR: 0 never, 1 the block pass's second product only
// (the default), 2 also GEMM2.
int npair_level() {
  static const int env = [] {
    const char* e = getenv("CQR_GEMM_NPAIR");
    return e ? atoi(e) : 1;
  }();
  return env;
}
bool pair_n_tiles(bool three, bool bf, bool split, const TcJob& job) {
  return job.pair_n && three && !bf && !split && job.n_tiles % 2 == 0;
}

// One launch of the tensor-core kernel in the variant of the handle's mode.  split: B arrives
// as raw FP32 and is split in shared memory (GEMM1 and the first block-reorthogonalisation
// product); otherwise B comes from planes.  Stages: 3 x 64 KB (two products), 2 x 96 KB (two
// products on pairs of M tiles), 6 x 32 KB (one product), 4 x 48 KB (BF16, one product, raw
// FP32 B of 64 K elements).
cudaError_t launch_mode(const TcGemm* t, bool split, const TcMaps& maps, const TcJob& job,
                        cudaStream_t st, int max_ctas = 0) {
  const bool three = t->nplanes == 2;
  const int mc = max_ctas > 0 ? std::min(max_ctas, t->num_sms) : t->num_sms;
  const bool pdl = st == t->pdl_st && st != nullptr;
  if (!t->bf) {
    if (pair_m_tiles(three, false, split, job.m_tiles))
      return launch_gemm<false, 2, 2, 2, 2>(maps, job, mc, st, pdl);
    if (pair_n_tiles(three, false, split, job))
      return launch_gemm<false, 2, 2, 2, 1, 2>(maps, job, mc, st, pdl);
    return three ? launch_gemm<false, 3, 2, 2>(maps, job, mc, st, pdl)
                 : launch_gemm<false, 6, 1, 1>(maps, job, mc, st, pdl);
  }
  if (three) return launch_gemm<true, 3, 2, 2>(maps, job, mc, st, pdl);
  return split ? launch_gemm<true, 4, 1, 2>(maps, job, mc, st, pdl)
               : launch_gemm<true, 6, 1, 1>(maps, job, mc, st, pdl);
}

template <typename P>
P* pl(void* p) { return static_cast<P*>(p); }

int64_t round_to(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

}  // namespace


bool tc_available() { return true; }

size_t tc_panel_bytes(int64_t, int) { return 0; }

size_t tc_workspace_bytes(int mode, int64_t M, int64_t N, int64_t n, int b, int reorth_block) {
  const bool bf = mode == CQR_MMA_BF16 || mode == CQR_MMA_BF16X3;
  const size_t pe = bf ? 2 : 4;
  const int64_t KE = bf ? 64 : 32;
  const int64_t bkp = round_to(b, KE);
  const int64_t ldk = round_to(M, 32);
  const int64_t akc = std::max<int64_t>(bkp, round_to(b, BM));
  const int64_t ldrow = round_to(n, 64);
  size_t s = 0;
  s += 4 * al256((size_t)ldk * akc * pe);            // Ak hi/lo, two buffers
  s += 4 * al256((size_t)M * bkp * pe);              // At hi/lo, two buffers
  s += 4 * al256((size_t)bkp * N * pe);              // Rbar planes, two contexts
  s += 2 * al256((size_t)kMaxSplits * bkp * N * 4);  // split-K partials (FP32), two contexts
  if (reorth_block) {
    s += 2 * al256((size_t)M * ldrow * pe);      // row-major computed columns hi/lo
    s += 2 * al256((size_t)ldrow * akc * pe);    // S planes
  }
  return s;
}

TcGemm* tc_create(int mode, int64_t M, int64_t N, int64_t n, int64_t b, float* Q, int64_t ldq,
                  void* ws, int num_sms, int reorth_block, cudaStream_t st) {
  TcGemm* t = new (std::nothrow) TcGemm();
  if (!t) return nullptr;
  t->mode = mode;
  t->bf = mode == CQR_MMA_BF16 || mode == CQR_MMA_BF16X3;
  t->nplanes = (mode == CQR_MMA_3XTF32 || mode == CQR_MMA_BF16X3) ? 2 : 1;
  t->KE = t->bf ? 64 : 32;
  t->pe = t->bf ? 2 : 4;
  t->M = M;
  t->N = N;
  t->b = b;
  t->bkp = round_to(b, t->KE);
  t->ldq = ldq;
  t->ldk = round_to(M, 32);
  t->Q = Q;
  t->num_sms = num_sms;
  const int64_t akc = std::max<int64_t>(t->bkp, round_to(b, BM));
  const size_t pe = t->pe;
  char* p = static_cast<char*>(ws);
  auto take = [&](size_t bytes) { char* r = p; p += al256(bytes); return static_cast<void*>(r); };
  for (int u = 0; u < 2; ++u) {
    t->Ak_hi[u] = take((size_t)t->ldk * akc * pe);
    t->Ak_lo[u] = take((size_t)t->ldk * akc * pe);
    t->At_hi[u] = take((size_t)M * t->bkp * pe);
    t->At_lo[u] = take((size_t)M * t->bkp * pe);
    t->Bh[u] = take((size_t)t->bkp * N * pe);
    t->Bl[u] = take((size_t)t->bkp * N * pe);
    t->P[u] = static_cast<float*>(take((size_t)kMaxSplits * t->bkp * N * 4));
  }
  t->n = n;
  t->ldrow = round_to(n, 64);
  t->Qr_hi = t->Qr_lo = t->Sh = t->Sl = nullptr;
  if (reorth_block) {
    t->Qr_hi = take((size_t)M * t->ldrow * pe);
    t->Qr_lo = take((size_t)M * t->ldrow * pe);
    t->Sh = take((size_t)t->ldrow * akc * pe);
    t->Sl = take((size_t)t->ldrow * akc * pe);
    // columns not yet computed are read (times zero rows of S) when kb is not a multiple of
    // the stage K: keep them finite
    if (cudaMemsetAsync(t->Qr_hi, 0, (size_t)M * t->ldrow * pe, st) != cudaSuccess ||
        cudaMemsetAsync(t->Qr_lo, 0, (size_t)M * t->ldrow * pe, st) != cudaSuccess) {
      delete t;
      return nullptr;
    }
  }
  const bool bf = t->bf;
  const uint32_t KE = (uint32_t)t->KE;
  bool ok = true;
  ok &= encode_2d(&t->tm_q_b, Q, false, (uint64_t)M, (uint64_t)N, (uint64_t)ldq * 4, 32, BN);
  for (int u = 0; u < 2; ++u) {
    ok &= encode_2d(&t->tm_ak[u][0], t->Ak_hi[u], bf, (uint64_t)M, (uint64_t)akc, (uint64_t)t->ldk * pe, KE, BM);
    ok &= encode_2d(&t->tm_ak[u][1], t->Ak_lo[u], bf, (uint64_t)M, (uint64_t)akc, (uint64_t)t->ldk * pe, KE, BM);
    ok &= encode_2d(&t->tm_at[u][0], t->At_hi[u], bf, (uint64_t)t->bkp, (uint64_t)M, (uint64_t)t->bkp * pe, KE, BM);
    ok &= encode_2d(&t->tm_at[u][1], t->At_lo[u], bf, (uint64_t)t->bkp, (uint64_t)M, (uint64_t)t->bkp * pe, KE, BM);
    ok &= encode_2d(&t->tm_bh[u][0], t->Bh[u], bf, (uint64_t)t->bkp, (uint64_t)N, (uint64_t)t->bkp * pe, KE, BN);
    ok &= encode_2d(&t->tm_bh[u][1], t->Bl[u], bf, (uint64_t)t->bkp, (uint64_t)N, (uint64_t)t->bkp * pe, KE, BN);
  }
  if (reorth_block) {
    ok &= encode_2d(&t->tm_qr[0], t->Qr_hi, bf, (uint64_t)t->ldrow, (uint64_t)M, (uint64_t)t->ldrow * pe, KE, BM);
    ok &= encode_2d(&t->tm_qr[1], t->Qr_lo, bf, (uint64_t)t->ldrow, (uint64_t)M, (uint64_t)t->ldrow * pe, KE, BM);
    ok &= encode_2d(&t->tm_s[0], t->Sh, bf, (uint64_t)t->ldrow, (uint64_t)akc, (uint64_t)t->ldrow * pe, KE, BN);
    ok &= encode_2d(&t->tm_s[1], t->Sl, bf, (uint64_t)t->ldrow, (uint64_t)akc, (uint64_t)t->ldrow * pe, KE, BN);
  }
  if (!ok) {
    delete t;
    return nullptr;
  }
  return t;
}

void tc_destroy(TcGemm* t) { delete t; }

void tc_set_status(TcGemm* t, int* status) { t->status = status; }

void tc_set_pdl_stream(TcGemm* t, cudaStream_t st) { t->pdl_st = st; }

namespace {
// Split-K factor of a product with m1 x n1 output tiles and K = M rows: the count s whose
// launch finishes first on `ctas` persistent CTAs, i.e. the least (waves of work units) x
// (K blocks per unit), each unit one tile and one K chunk; a split adds partial-sum traffic,
// so each split costs 2% more and ties go to fewer splits.
// K blocks per work unit for `tiles` output tiles and `kblocks` K blocks on `ctas` CTAs, at
// most max_splits chunks (see tc_splits).
int64_t best_kchunk(int64_t tiles, int64_t kblocks, int ctas, int max_splits) {
  int64_t best_kc = kblocks;
  double best = -1.0;
  for (int s = 1; s <= max_splits && s <= kblocks; ++s) {
    const int64_t kc = (kblocks + s - 1) / s;
    const int64_t units = tiles * ((kblocks + kc - 1) / kc);
    const int64_t waves = (units + ctas - 1) / ctas;
    const double cost = (double)waves * (double)kc * (1.0 + 0.02 * s);
    if (best < 0.0 || cost < best) {
      best = cost;
      best_kc = kc;
    }
  }
  return best_kc;
}

int tc_splits(const TcGemm* t, int m1, int n1, int64_t* kchunk, int max_ctas = 0) {
  const int ctas = max_ctas > 0 ? std::min(max_ctas, t->num_sms) : t->num_sms;
  const int64_t kblocks = (t->M + t->KE - 1) / t->KE;
  // work units of the GEMM1-shaped launch (pairs of M tiles where launch_mode pairs them)
  const bool three = t->nplanes == 2;
  const int units_m = pair_m_tiles(three, t->bf, three || t->bf, m1) ? m1 / 2 : m1;
  *kchunk = best_kchunk((int64_t)units_m * n1, kblocks, ctas, kMaxSplits) * t->KE;
  return (int)((t->M + *kchunk - 1) / *kchunk);
}
}  // namespace

// 1. split the panel Q[:, kb : kb+bk] into the operand planes of both GEMMs (and, for a
//    finished panel with block reorthogonalisation on, into the row-major computed columns)
cudaError_t tc_split_panel(TcGemm* t, int64_t kb, int bk, bool finished, int buf, cudaStream_t st) {
  const int bkp = (int)round_to(bk, t->KE);
  const int m1 = (bk + BM - 1) / BM;
  dim3 grd((unsigned)((t->M + 31) / 32), (unsigned)((std::max(bkp, m1 * BM) + 31) / 32));
  void* qh = finished ? t->Qr_hi : nullptr;
  const bool pdl = st == t->pdl_st && st != nullptr;
  const float* q0 = t->Q + kb * t->ldq;
  if (t->bf) {
    using B16 = __nv_bfloat16;
    return launch_k(k_split_panel<B16>, grd, dim3(256), 0, st, pdl, q0, t->ldq, t->M, bk, bkp,
                    (int)(m1 * BM), t->nplanes, pl<B16>(t->Ak_hi[buf]), pl<B16>(t->Ak_lo[buf]), t->ldk,
                    pl<B16>(t->At_hi[buf]), pl<B16>(t->At_lo[buf]), pl<B16>(qh), pl<B16>(t->Qr_lo),
                    t->ldrow, kb);
  }
  return launch_k(k_split_panel<float>, grd, dim3(256), 0, st, pdl, q0, t->ldq, t->M, bk, bkp,
                  (int)(m1 * BM), t->nplanes, pl<float>(t->Ak_hi[buf]), pl<float>(t->Ak_lo[buf]), t->ldk,
                  pl<float>(t->At_hi[buf]), pl<float>(t->At_lo[buf]), pl<float>(qh), pl<float>(t->Qr_lo),
                  t->ldrow, kb);
}

bool tc_has_block_reorth(const TcGemm* t) { return t->Qr_hi != nullptr; }

// Row-major planes of one rectangle of Q (rows r0.., columns c0.. below the computed-column
// count) rebuilt after a recovery changed it.
cudaError_t tc_refresh_rect(TcGemm* t, int64_t r0, int64_t nr, int64_t c0, int64_t nc, cudaStream_t st) {
  if (!t->Qr_hi || nr <= 0 || nc <= 0) return cudaSuccess;
  const dim3 grd((unsigned)((nr + 31) / 32), (unsigned)((nc + 31) / 32));
  if (t->bf)
    k_refresh_rect<__nv_bfloat16><<<grd, 256, 0, st>>>(t->Q, t->ldq, r0, (int)nr, c0, (int)nc, t->nplanes,
                                                      pl<__nv_bfloat16>(t->Qr_hi),
                                                      pl<__nv_bfloat16>(t->Qr_lo), t->ldrow);
  else
    k_refresh_rect<float><<<grd, 256, 0, st>>>(t->Q, t->ldq, r0, (int)nr, c0, (int)nc, t->nplanes,
                                              pl<float>(t->Qr_hi), pl<float>(t->Qr_lo), t->ldrow);
  return cudaGetLastError();
}

// 2. GEMM1, split-K over the M rows: partials P[s] = Qbar^T Q[:, j0 : j0+w]
cudaError_t tc_gemm_rbar(TcGemm* t, int bk, int64_t j0, int64_t w, int buf, int ctx, int max_ctas,
                         cudaStream_t st) {
  const int three = t->nplanes == 2;
  const int bkp = (int)round_to(bk, t->KE);
  const int m1 = (bk + BM - 1) / BM;
  const int n1 = (int)((w + BN - 1) / BN);
  int64_t kchunk = 0;
  const int splits = tc_splits(t, m1, n1, &kchunk, max_ctas);
  TcMaps maps;
  maps.a[0] = t->tm_ak[buf][0];
  maps.a[1] = t->tm_ak[buf][1];
  maps.b[0] = t->tm_q_b;
  maps.b[1] = t->tm_q_b;
  TcJob job{};
  job.nprod = three ? 3 : 1;
  // TF32 reads the raw FP32 words directly with one product; every other mode splits B
  const bool split = three || t->bf;
  job.split_b_smem = split ? 1 : 0;
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
  job.out = t->P[ctx];
  job.ldo = bkp;
  job.split_stride = (int64_t)bkp * w;
  job.status = t->status;
  return launch_mode(t, split, maps, job, st, max_ctas);
}

// 3. reduce the partials into R[kb.., j0..] and GEMM2's B planes
cudaError_t tc_reduce(TcGemm* t, int64_t kb, int bk, int64_t j0, int64_t w, float* R, int64_t ldr,
                      int ctx, int max_ctas, cudaStream_t st) {
  const int bkp = (int)round_to(bk, t->KE);
  const int m1 = (bk + BM - 1) / BM;
  const int n1 = (int)((w + BN - 1) / BN);
  int64_t kchunk = 0;
  const int splits = tc_splits(t, m1, n1, &kchunk, max_ctas);
  const int64_t total = (int64_t)bkp * w;
  const int blocks = (int)std::min<int64_t>(4096, (total + 255) / 256);
  const bool pdl = st == t->pdl_st && st != nullptr;
  const float* P = t->P[ctx];
  float* Rd = R + kb + j0 * ldr;
  if (t->bf)
    return launch_k(k_tc_reduce<__nv_bfloat16>, dim3(blocks), dim3(256), 0, st, pdl, P, splits,
                    (int64_t)bkp * w, (int64_t)bkp, bk, bkp, w, Rd, ldr, t->nplanes,
                    pl<__nv_bfloat16>(t->Bh[ctx]), pl<__nv_bfloat16>(t->Bl[ctx]));
  return launch_k(k_tc_reduce<float>, dim3(blocks), dim3(256), 0, st, pdl, P, splits, (int64_t)bkp * w,
                  (int64_t)bkp, bk, bkp, w, Rd, ldr, t->nplanes, pl<float>(t->Bh[ctx]),
                  pl<float>(t->Bl[ctx]));
}

// 4. GEMM2: Q[:, j0 : j0+w] -= Qbar Rbar (M tiles over rows, N tiles over trailing columns)
cudaError_t tc_gemm_update(TcGemm* t, int bk, int64_t j0, int64_t w, int buf, int ctx, int max_ctas,
                           cudaStream_t st) {
  const int three = t->nplanes == 2;
  const int bkp = (int)round_to(bk, t->KE);
  TcMaps maps;
  maps.a[0] = t->tm_at[buf][0];
  maps.a[1] = t->tm_at[buf][1];
  maps.b[0] = t->tm_bh[ctx][0];
  maps.b[1] = t->tm_bh[ctx][1];
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
  maps.c = t->tm_q_b;
  job.prefetch_c = 1;
  job.c_col0 = j0;
  job.pair_n = npair_level() >= 2 ? 1 : 0;
  return launch_mode(t, false, maps, job, st, max_ctas);
}

// Block reorthogonalisation of panel kb .. kb+bk-1 against columns 0 .. kb-1 (four
// launches: split the panel, S^T = Qbar^T Q[:, 0:kb] split-K on the tensor cores, reduce
// into R and S, Qbar -= Qrows S on the tensor cores).
cudaError_t tc_block_reorth(TcGemm* t, int64_t kb, int bk, float* R, int64_t ldr, int buf,
                            cudaStream_t st, int* launches) {
  *launches = 0;
  if (!t->Qr_hi || kb <= 0) return cudaSuccess;
  *launches = 4;
  cudaError_t e = tc_split_panel(t, kb, bk, false, buf, st);
  if (e != cudaSuccess) return e;
  e = tc_gemm_rbar(t, bk, 0, kb, buf, 0, 0, st);  // partials of S^T (bk x kb), context 0
  if (e != cudaSuccess) return e;
  const int KE = t->KE;
  const int bkp = (int)round_to(bk, KE);
  const int m1 = (bk + BM - 1) / BM;
  const int n1 = (int)((kb + BN - 1) / BN);
  int64_t kchunk = 0;
  const int splits = tc_splits(t, m1, n1, &kchunk);
  const int64_t kbp = round_to(kb, KE);
  {
    const dim3 blocks((unsigned)((bk + 31) / 32), (unsigned)((kbp + 31) / 32));
    const bool pdl = st == t->pdl_st && st != nullptr;
    const float* P0 = t->P[0];
    if (t->bf)
      e = launch_k(k_tc_reduce_t<__nv_bfloat16>, blocks, dim3(256), 0, st, pdl, P0, splits,
                   (int64_t)bkp * kb, (int64_t)bkp, bk, kb, kbp, R, ldr, t->nplanes,
                   pl<__nv_bfloat16>(t->Sh), pl<__nv_bfloat16>(t->Sl), t->ldrow);
    else
      e = launch_k(k_tc_reduce_t<float>, blocks, dim3(256), 0, st, pdl, P0, splits,
                   (int64_t)bkp * kb, (int64_t)bkp, bk, kb, kbp, R, ldr, t->nplanes,
                   pl<float>(t->Sh), pl<float>(t->Sl), t->ldrow);
    if (e != cudaSuccess) return e;
  }
  TcMaps maps;
  maps.a[0] = t->tm_qr[0];
  maps.a[1] = t->tm_qr[1];
  maps.b[0] = t->tm_s[0];
  maps.b[1] = t->tm_s[1];
  TcJob job{};
  job.nprod = t->nplanes == 2 ? 3 : 1;
  job.split_b_smem = 0;
  job.epi = 1;
  job.m_tiles = (int)((t->M + BM - 1) / BM);
  job.n_tiles = (bk + BN - 1) / BN;
  // Split K (the kb computed columns) when that makes the launch finish sooner on the SMs
  // (too few M x bk output tiles, or a last wave mostly idle); the partials go to P (capacity
  // kMaxSplits * bkp * N floats) and are subtracted in a fixed order, so the result does not
  // depend on the schedule.
  const int64_t kblk = kbp / KE;
  job.pair_n = npair_level() >= 1 ? 1 : 0;
  const bool np2 = pair_n_tiles(t->nplanes == 2, t->bf, false, job);
  const int tiles2 = job.m_tiles * (job.n_tiles / (np2 ? 2 : 1));
  const int64_t cap = std::min<int64_t>(kMaxSplits, (int64_t)kMaxSplits * t->bkp * t->N /
                                                        (t->M * (int64_t)bk));
  const int64_t kchunk2 = best_kchunk(tiles2, kblk, t->num_sms, (int)std::max<int64_t>(1, cap)) * KE;
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
    job.out = t->P[0];
    job.ldo = t->M;
    job.split_stride = t->M * (int64_t)bk;
  }
  e = launch_mode(t, false, maps, job, st);
  if (e != cudaSuccess || splits2 == 1) return e;
  *launches = 5;
  const int64_t total = t->M * (int64_t)bk;
  const int blocks = (int)std::min<int64_t>((int64_t)t->num_sms * 8, (total + 255) / 256);
  const bool pdl = st == t->pdl_st && st != nullptr;
  return launch_k(k_tc_sub_partials, dim3(blocks), dim3(256), 0, st, pdl, (const float*)t->P[0], splits2,
                  t->M, (int64_t)bk, t->Q + kb * t->ldq, t->ldq);
}

// General C -= op(A) B in 3xTF32 on the tensor cores (the large products of the reverse mode).
// op(A) is A^T (A: K x M column-major) when a_trans, else A (M x K column-major); B is K x N
// column-major, C is M x N column-major.  A goes through the operand split into hi / lo
// planes (K-major: column-major for A^T, row-major for A); B is loaded raw and split in shared
// memory.  One CTA per 128 x 128 output tile (at most the SMs, persistent), no split over K.
// Returns cudaErrorInvalidValue (nothing launched) when a tensor-map rule is not met: B and C
// 16-byte aligned, ldb a multiple of 4.
size_t tc_gemm_sub_planes(bool a_trans, int64_t M, int64_t K) {
  return a_trans ? 2 * (size_t)round_to(K, 32) * (size_t)M : 2 * (size_t)M * (size_t)round_to(K, 32);
}

cudaError_t tc_gemm_sub3(bool a_trans, const float* A, int64_t lda, const float* B, int64_t ldb,
                         float* C, int64_t ldc, int64_t M, int64_t N, int64_t K, float* planes,
                         int num_sms, int* status, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  if ((reinterpret_cast<uintptr_t>(B) & 15) || (ldb % 4) || (reinterpret_cast<uintptr_t>(planes) & 15))
    return cudaErrorInvalidValue;
  const int64_t kp = round_to(K, 32);
  float* hi = planes;
  TcMaps maps;
  bool ok = true;
  if (a_trans) {
    // planes of A (K x M): column-major, ld kp; rows of op(A) are columns of A
    float* lo = hi + kp * M;
    const dim3 grd((unsigned)((K + 31) / 32), (unsigned)((M + 31) / 32));
    k_split_panel<float><<<grd, 256, 0, st>>>(A, lda, K, (int)M, 0, (int)M, 2, hi, lo, kp, nullptr,
                                              nullptr, nullptr, nullptr, 0, 0);
    ok &= encode_2d(&maps.a[0], hi, false, (uint64_t)K, (uint64_t)M, (uint64_t)kp * 4, 32, BM);
    ok &= encode_2d(&maps.a[1], lo, false, (uint64_t)K, (uint64_t)M, (uint64_t)kp * 4, 32, BM);
  } else {
    // planes of A (M x K): row-major, row stride kp
    float* lo = hi + M * kp;
    const dim3 grd((unsigned)((M + 31) / 32), (unsigned)((kp + 31) / 32));
    k_split_panel<float><<<grd, 256, 0, st>>>(A, lda, M, (int)K, (int)kp, 0, 2, nullptr, nullptr, 0, hi,
                                              lo, nullptr, nullptr, 0, 0);
    ok &= encode_2d(&maps.a[0], hi, false, (uint64_t)kp, (uint64_t)M, (uint64_t)kp * 4, 32, BM);
    ok &= encode_2d(&maps.a[1], lo, false, (uint64_t)kp, (uint64_t)M, (uint64_t)kp * 4, 32, BM);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ok &= encode_2d(&maps.b[0], const_cast<float*>(B), false, (uint64_t)K, (uint64_t)N, (uint64_t)ldb * 4, 32, BN);
  maps.b[1] = maps.b[0];
  if (!ok) return cudaErrorInvalidValue;
  TcJob job{};
  job.nprod = 3;
  job.split_b_smem = 1;
  job.epi = 1;
  job.m_tiles = (int)((M + BM - 1) / BM);
  job.n_tiles = (int)((N + BN - 1) / BN);
  job.splits = 1;
  job.a_row0 = 0;
  job.b_row0 = 0;
  job.k0 = 0;
  job.kchunk = kp;
  job.K = K;
  job.mrows = M;
  job.ncols = N;
  job.out = C;
  job.ldo = ldc;
  job.split_stride = 0;
  job.status = status;
  return launch_gemm<false, 3, 2, 2>(maps, job, num_sms, st, false);
}

cudaError_t bounds_take_tc(int* code, int* site) { return bounds_take_here(code, site); }

}  // namespace cqr
