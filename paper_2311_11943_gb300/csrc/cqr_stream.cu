// cqr_stream.cu -- the bandwidth-bound FP32 encode (checksum tiles, §4.2) and erasure decode
// (Recovery Lemma, Eq. (A_recov)) with their inputs streamed by the tensor memory accelerator.
//
// Each CTA of a persistent grid keeps a ring of shared-memory stages.  One thread fills them
// with cp.async.bulk.tensor boxes of 128 rows, and an mbarrier per stage counts the bytes.  So
// the bytes in flight per SM do not depend on the registers the arithmetic needs, and a CTA's
// next blocks load while it works on the current one.  The arithmetic of every element is that
// of the register kernels in cqr_kernels.cu, in the same order, so both give the same bits.
// Every wait is bounded: on a timeout the CTA records CQR_ETIMEOUT, waits (bounded) for the
// boxes it still has in flight and leaves at a point that all its threads reach together.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>

#include "cqr_decode.cuh"
#include "cqr_device.cuh"
#include "cqr_kernels.cuh"
#include "cqr_tc_gemm.cuh"

namespace cqr {
namespace {

constexpr int kBoxRows = 128;  // rows of one box: 32 lanes x 4 rows

__device__ __forceinline__ void box_load(uint32_t dst, const CUtensorMap* tm, int x, int y,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}

__device__ __forceinline__ void fma4(float4& acc, float c, const float4& v) {
  acc.x += c * v.x;
  acc.y += c * v.y;
  acc.z += c * v.z;
  acc.w += c * v.w;
}
__device__ __forceinline__ void add4(float4& acc, const float4& v) {
  acc.x += v.x;
  acc.y += v.y;
  acc.z += v.z;
  acc.w += v.w;
}
__device__ __forceinline__ void st4(float* p, const float4& v) {
  *reinterpret_cast<float4*>(p) = v;
}

// Thread 0 waits (bounded by kDrainCycles each) for the stages [first, end) it issued and
// nobody consumed, so that no box lands in shared memory after the CTA has left.
__device__ __forceinline__ void drain_stages(uint64_t* full, int D, int64_t first, int64_t end,
                                             int* status, int site) {
  if (threadIdx.x != 0 || threadIdx.y != 0) return;
  for (int64_t k = first; k < end; ++k)
    mbar_wait_bounded(full + (int)(k % D), (unsigned)((k / D) & 1), kDrainCycles, status, site);
}

// ------------------------------------------------------------------------------- encode
// Both codes in one pass, as k_encode_fused (R protected, F <= 4 checksums, p_c <= 16 tile
// columns).  A block of positions is 128 rows r (32 lanes x 4 rows) of one position column s;
// stage t of a block holds the p_c boxes A_{t,j}(r0 .. r0+127, s), one per tile column.  The
// 4 thread groups split the p_c tile columns into contiguous groups of at most 4; each thread
// copies its tiles into the encoded matrix and keeps the vertical checksums of its columns in
// registers; the group partials of the horizontal checksums, and at the end of a block those
// of the corners, are added through shared memory in group order.  A is read once (by TMA) and
// the encoded matrix written once.
template <int F>
__global__ void __launch_bounds__(128) k_encode_tma(const __grid_constant__ CUtensorMap tmA, Geo g,
                                                    const float* __restrict__ Gt,
                                                    const float* __restrict__ Gh,
                                                    float* __restrict__ Q, int* status, int D,
                                                    int nbx) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int KMAX = 4;
  const int p_r = g.p_r, p_c = g.p_c, mb = (int)g.mb, nb = (int)g.nb;
  const int64_t ldq = g.ldq;
  const int tx = threadIdx.x, jg = threadIdx.y, tid = jg * 32 + tx;
  const int cpg = (p_c + 3) / 4, j0 = jg * cpg;
  const int nj = max(0, min(cpg, p_c - j0));
  unsigned char* sb = smem + ((128u - (saddr(smem) & 127u)) & 127u);  // boxes 128-byte aligned
  float* slots = reinterpret_cast<float*>(sb);                               // [D][p_c][128]
  float4* hs = reinterpret_cast<float4*>(sb + (size_t)D * p_c * 512);        // [2][4][F][32]
  uint64_t* full = reinterpret_cast<uint64_t*>(hs + 2 * 4 * F * 32);         // [D]
  float* gts = reinterpret_cast<float*>(full + D);                           // [F][p_r]
  // uniform over the launch, before any barrier: the geometry the indexing below assumes
  CQR_CHECK(p_c <= 4 * KMAX && g.M <= ldq && g.n + (int64_t)F * nb <= g.N &&
                g.m_pad + (int64_t)F * mb <= g.M && mb % 4 == 0 && ldq % 4 == 0,
            113);
  const int64_t nblk = (int64_t)nbx * nb;  // position blocks
  const int64_t nmine = blockIdx.x < nblk ? (nblk - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t nst = nmine * p_r;         // stages of this CTA: block-major, tile row minor
  auto issue = [&](int64_t i) {            // thread 0: stage i into slot i % D
    const int64_t blk = blockIdx.x + (i / p_r) * gridDim.x;
    const int t = (int)(i % p_r);
    const int bx = (int)(blk % nbx), s = (int)(blk / nbx);
    const int slot = (int)(i % D);
    uint64_t* bar = full + slot;
    mbar_expect(bar, (unsigned)p_c * kBoxRows * 4u);
    for (int j = 0; j < p_c; ++j)
      box_load(saddr(slots + ((size_t)slot * p_c + j) * kBoxRows), &tmA, t * mb + bx * kBoxRows,
               j * nb + s, bar);
  };
  if (tid == 0) {
    for (int k = 0; k < D; ++k) mbar_init(full + k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int idx = tid; idx < F * p_r; idx += blockDim.x * blockDim.y) gts[idx] = Gt[idx];
  __syncthreads();
  if (tid == 0)
    for (int64_t i = 0; i < std::min<int64_t>(D, nst); ++i) issue(i);
  float hc[KMAX][F];  // G_h entries of this thread's tile columns
#pragma unroll
  for (int k = 0; k < KMAX; ++k)
#pragma unroll
    for (int l = 0; l < F; ++l) hc[k][l] = k < nj ? Gh[(j0 + k) * F + l] : 0.f;
  float4 vacc[KMAX][F];
  for (int64_t i = 0; i < nst; ++i) {
    const int64_t blk = blockIdx.x + (i / p_r) * gridDim.x;
    const int t = (int)(i % p_r);
    const int bx = (int)(blk % nbx), s = (int)(blk / nbx);
    const int r = bx * kBoxRows + 4 * tx;
    const bool live = r < mb;
    if (t == 0) {
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
#pragma unroll
        for (int q = 0; q < F; ++q) vacc[k][q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int slot = (int)(i % D);
    const bool ok = mbar_wait_bounded(full + slot, (unsigned)((i / D) & 1), kWaitLimitCycles,
                                      status, 60);
    const int64_t row = (int64_t)t * mb + r;
    float4 h[F];
#pragma unroll
    for (int l = 0; l < F; ++l) h[l] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ok) {
      const float* sl = slots + (size_t)slot * p_c * kBoxRows + 4 * tx;
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
        if (k < nj) {
          const int j = j0 + k;
          const float4 a = *reinterpret_cast<const float4*>(sl + (size_t)j * kBoxRows);
          if (live) st4(Q + row + ((int64_t)j * nb + s) * ldq, a);
#pragma unroll
          for (int q = 0; q < F; ++q) fma4(vacc[k][q], gts[q * p_r + t], a);
#pragma unroll
          for (int l = 0; l < F; ++l) fma4(h[l], hc[k][l], a);
        }
    }
    float4* hp = hs + (size_t)(i & 1) * 4 * F * 32;
#pragma unroll
    for (int l = 0; l < F; ++l) hp[(jg * F + l) * 32 + tx] = h[l];
    // every thread is done with the slot and has its partials in place
    if (__syncthreads_or(!ok)) {
      drain_stages(full, D, i, std::min<int64_t>(i + D, nst), status, 60);
      return;
    }
    if (tid == 0 && i + D < nst) issue(i + D);
    if (jg < F && live) {  // thread group jg writes checksum l = jg of this row
      const int l = jg;
      float4 sum = hp[l * 32 + tx];
      for (int q = 1; q < 4; ++q) add4(sum, hp[(q * F + l) * 32 + tx]);
      st4(Q + row + (g.n + (int64_t)l * nb + s) * ldq, sum);
    }
    if (t == p_r - 1) {  // the block's vertical checksums, then the corners
#pragma unroll
      for (int q = 0; q < F; ++q) {
        const int64_t crow = g.m_pad + (int64_t)q * mb + r;
        float4 c[F];
#pragma unroll
        for (int l = 0; l < F; ++l) c[l] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
          if (k < nj) {
            const int j = j0 + k;
            if (live) st4(Q + crow + ((int64_t)j * nb + s) * ldq, vacc[k][q]);
#pragma unroll
            for (int l = 0; l < F; ++l) fma4(c[l], hc[k][l], vacc[k][q]);
          }
        __syncthreads();  // earlier reads of the partials are done
#pragma unroll
        for (int l = 0; l < F; ++l) hs[(jg * F + l) * 32 + tx] = c[l];
        __syncthreads();
        if (jg < F && live) {
          const int l = jg;
          float4 sum = hs[l * 32 + tx];
          for (int u = 1; u < 4; ++u) add4(sum, hs[(u * F + l) * 32 + tx]);
          st4(Q + crow + (g.n + (int64_t)l * nb + s) * ldq, sum);
        }
      }
      __syncthreads();  // the corner partials are read before the next stage writes partials
    }
  }
}

size_t encode_smem(int D, int p_c, int p_r, int F) {
  return 128 + (size_t)D * p_c * 512 + (size_t)2 * 4 * F * 32 * 16 + (size_t)D * 8 +
         (size_t)F * p_r * 4;
}

int num_sms_now() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

template <int F>
cudaError_t launch_encode_tma_f(const CUtensorMap& tm, const Geo& g, const float* Gt,
                                const float* Gh, float* Q, int* status, cudaStream_t st) {
  // a ring of about 48 KB of boxes: three CTAs of 128 threads per SM
  const int D = std::max(2, std::min(8, 49152 / (g.p_c * 512)));
  const size_t smem = encode_smem(D, g.p_c, g.p_r, F);
  cudaError_t e = cudaFuncSetAttribute(k_encode_tma<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_encode_tma<F>, 128, smem);
  if (e != cudaSuccess) return e;
  const int nbx = (int)((g.mb + kBoxRows - 1) / kBoxRows);
  const int64_t nblk = (int64_t)nbx * g.nb;
  const int64_t grid = std::max<int64_t>(
      1, std::min<int64_t>(nblk, (int64_t)std::max(1, occ) * num_sms_now()));
  k_encode_tma<F><<<(unsigned)grid, dim3(32, 4), smem, st>>>(tm, g, Gt, Gh, Q, status, D, nbx);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------- decode
// One code per blockIdx.y; its CTAs (blockIdx.x, gridDim.x of them) take the code's position
// blocks (128 rows x 4 position columns) in turn.  Stage k of a CTA holds the boxes of the nuse
// code tiles it reads for one block, in the order of tuse.  Thread 0 starts the first stages as
// soon as the tile list is known, while the coefficient tables are still being built.
__global__ void __launch_bounds__(128) k_decode_tma(const __grid_constant__ CUtensorMap tmQ,
                                                    const __grid_constant__ CUtensorMap tmR, Geo g,
                                                    const DecodePlan* __restrict__ plans,
                                                    const double* __restrict__ Gt,
                                                    const double* __restrict__ Gh, float* Q,
                                                    float* R, int* status, int D, int maxuse) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ DecodeScratch<float> sh;
  constexpr int S = 4;  // position columns of a block
  const DecodePlan& p = plans[blockIdx.y];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const bool isQ = (p.kind == 0);
  const int64_t h = isQ ? g.mb : g.nb;
  const int nbx = (int)((h + kBoxRows - 1) / kBoxRows);
  const int64_t nblk = (int64_t)nbx * (g.nb / S);
  const int64_t nmine = blockIdx.x < nblk ? (nblk - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  unsigned char* sb = smem + ((128u - (saddr(smem) & 127u)) & 127u);  // boxes 128-byte aligned
  float* slots = reinterpret_cast<float*>(sb);                          // [D][maxuse][S][128]
  uint64_t* full = reinterpret_cast<uint64_t*>(sb + (size_t)D * maxuse * S * kBoxRows * 4);
  CQR_CHECK(p.f1 + p.f2 <= g.f && g.f <= 4 && p.idx >= 0 &&
                p.idx < (isQ ? g.grid_cols : g.p_c + g.f) && g.M <= g.ldq && g.mb % 4 == 0 &&
                g.nb % S == 0 && g.ldq % 4 == 0 && g.ldr % 4 == 0 && p.nsys <= maxuse,
            114);
  auto issue = [&](int64_t k) {  // thread 0: block k of this CTA into slot k % D
    const int64_t blk = blockIdx.x + k * gridDim.x;
    const int r0 = (int)(blk % nbx) * kBoxRows, s0 = (int)(blk / nbx) * S;
    const int slot = (int)(k % D);
    uint64_t* bar = full + slot;
    mbar_expect(bar, (unsigned)sh.nuse * S * kBoxRows * 4u);
    for (int u = 0; u < sh.nuse; ++u) {
      const int t = sh.tuse[u];
      const uint32_t dst = saddr(slots + ((size_t)slot * maxuse + u) * S * kBoxRows);
      if (isQ)
        box_load(dst, &tmQ, t * (int)g.mb + r0, p.idx * (int)g.nb + s0, bar);
      else
        box_load(dst, &tmR, p.idx * (int)g.nb + r0, t * (int)g.nb + s0, bar);
    }
  };
  if (tid == 0) {
    for (int k = 0; k < D; ++k) mbar_init(full + k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int64_t npre = std::min<int64_t>(D, nmine);
  bool started = false;
  const bool ready = decode_setup<float>(
      g, p, Gt, Gh, sh, tid, blockDim.x * blockDim.y, status, blockIdx.x == 0,
      [&]() {
        if (sh.nuse <= maxuse) {
          for (int64_t k = 0; k < npre; ++k) issue(k);
          started = true;
        }
      });
  // a singular G^ (recorded by decode_setup) or a tile list longer than the ring was sized for
  const bool fits = sh.nuse <= maxuse;
  if (!ready || !fits) {
    if (!fits && tid == 0) set_status(status, CQR_EINVAL, p.idx);
    if (started) drain_stages(full, D, 0, npre, status, 61);
    return;
  }
  const int64_t tstride = isQ ? g.mb : g.nb * g.ldr;
  const int64_t ld = isQ ? g.ldq : g.ldr;
  float* base = isQ ? Q + (int64_t)p.idx * g.nb * g.ldq : R + (int64_t)p.idx * g.nb;
  for (int64_t k = 0; k < nmine; ++k) {
    const int64_t blk = blockIdx.x + k * gridDim.x;
    const int64_t r4 = (int64_t)(blk % nbx) * kBoxRows + 4 * tx;
    const int64_t s = (blk / nbx) * S + ty;
    const int slot = (int)(k % D);
    const bool ok = mbar_wait_bounded(full + slot, (unsigned)((k / D) & 1), kWaitLimitCycles,
                                      status, 61);
    if (ok && r4 < h) {
      const float* sl = slots + (size_t)slot * maxuse * S * kBoxRows + ty * kBoxRows + 4 * tx;
      decode_combine4(p, sh, base + r4 + s * ld, tstride, [&](int u) {
        return *reinterpret_cast<const float4*>(sl + (size_t)u * S * kBoxRows);
      });
    }
    if (__syncthreads_or(!ok)) {  // every thread is done with the slot
      drain_stages(full, D, k, std::min<int64_t>(k + D, nmine), status, 61);
      return;
    }
    if (tid == 0 && k + D < nmine) issue(k + D);
  }
}

}  // namespace

// The streamed paths apply to FP32 with 16-byte aligned rows; false leaves the caller to the
// register kernels.  CQR_NO_TMA_STREAM=1 selects the register kernels (same bits).
bool encode_tma_applies(const Geo& g, const float* A, int64_t lda, const float* Q) {
  return g.f >= 1 && g.f <= 4 && g.protect_r && g.p_c <= 16 && g.mb % 4 == 0 && lda % 4 == 0 &&
         g.ldq % 4 == 0 && lda >= g.m && g.m < (1LL << 31) && g.n < (1LL << 31) &&
         (reinterpret_cast<uintptr_t>(A) & 15) == 0 && (reinterpret_cast<uintptr_t>(Q) & 15) == 0 &&
         !getenv("CQR_NO_TMA_STREAM");
}

cudaError_t launch_encode_tma(const Geo& g, const float* A, int64_t lda, const float* Gt,
                              const float* Gh, float* Q, int* status, cudaStream_t st) {
  CUtensorMap tm;
  if (!tmap_f32_plain(&tm, A, (uint64_t)g.m, (uint64_t)g.n, (uint64_t)lda * 4, kBoxRows, 1))
    return cudaErrorInvalidValue;
  switch (g.f) {
    case 1: return launch_encode_tma_f<1>(tm, g, Gt, Gh, Q, status, st);
    case 2: return launch_encode_tma_f<2>(tm, g, Gt, Gh, Q, status, st);
    case 3: return launch_encode_tma_f<3>(tm, g, Gt, Gh, Q, status, st);
    default: return launch_encode_tma_f<4>(tm, g, Gt, Gh, Q, status, st);
  }
}

bool decode_tma_applies(const Geo& g, const float* Q, const float* R, int maxuse) {
  return g.f <= 4 && g.mb % 4 == 0 && g.nb % 4 == 0 && g.ldq % 4 == 0 && g.ldr % 4 == 0 &&
         maxuse <= 32 && g.M < (1LL << 31) && g.N < (1LL << 31) &&
         (reinterpret_cast<uintptr_t>(Q) & 15) == 0 && (reinterpret_cast<uintptr_t>(R) & 15) == 0 &&
         !getenv("CQR_NO_TMA_STREAM");
}

cudaError_t launch_decode_tma(const Geo& g, const DecodePlan* plans_dev, int nplans, int maxuse,
                              const double* Gt, const double* Gh, float* Q, float* R, int* status,
                              cudaStream_t st) {
  if (nplans == 0) return cudaSuccess;
  CUtensorMap tq, tr;
  if (!tmap_f32_plain(&tq, Q, (uint64_t)g.M, (uint64_t)g.N, (uint64_t)g.ldq * 4, kBoxRows, 4) ||
      !tmap_f32_plain(&tr, R, (uint64_t)g.N, (uint64_t)g.N, (uint64_t)g.ldr * 4, kBoxRows, 4))
    return cudaErrorInvalidValue;
  const int D = 2;
  const size_t smem = 128 + (size_t)D * maxuse * 4 * kBoxRows * 4 + (size_t)D * 8;
  cudaError_t e = cudaFuncSetAttribute(k_decode_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_decode_tma, 128, smem);
  if (e != cudaSuccess) return e;
  const int64_t hmax = std::max(g.mb, g.nb);
  const int64_t nblk = ((hmax + kBoxRows - 1) / kBoxRows) * (g.nb / 4);
  const int64_t per = std::max<int64_t>(
      1, std::min<int64_t>(nblk, ((int64_t)std::max(1, occ) * num_sms_now() + nplans - 1) / nplans));
  k_decode_tma<<<dim3((unsigned)per, (unsigned)nplans), dim3(32, 4), smem, st>>>(
      tq, tr, g, plans_dev, Gt, Gh, Q, R, status, D, maxuse);
  return cudaGetLastError();
}

}  // namespace cqr
