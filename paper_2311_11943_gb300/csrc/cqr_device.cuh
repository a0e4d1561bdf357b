// cqr_device.cuh -- device-side primitives shared by the coded-QR kernels: the device
// status word, a bounded grid-wide barrier for cooperative launches, warp reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "coded_qr.h"

namespace cqr {

// Device status word layout (int[4]): [0] first error code (CQR_*), [1] reorthogonalisation
// count, [2] detail of the first error (e.g. the global column of a breakdown), [3] the
// barrier site that timed out.
enum { ST_CODE = 0, ST_REORTH = 1, ST_DETAIL = 2, ST_SITE = 3 };

__device__ __forceinline__ void set_status(int* st, int code, int detail) {
  if (atomicCAS(st + ST_CODE, 0, code) == 0) st[ST_DETAIL] = detail;
}

// Index checks of the bounds-checked build (compiled with -DCQR_DEBUG_BOUNDS; nothing in the
// normal build).  CQR_CHECK(cond, site): when cond is false the thread records CQR_EBOUNDS with
// the site number in this file's bounds word and returns from the kernel before the access the
// condition guards; it never traps.  CQR_CHECK_OK(cond, site) records the same and yields false
// (for accesses that are skipped instead, where a return would strand other threads at a
// barrier).  Each source file has its own word; coded_qr_debug_bounds collects them.
#ifdef CQR_DEBUG_BOUNDS
static __device__ int g_bounds[2];  // [0] CQR_EBOUNDS once a check failed, [1] its site
__device__ __forceinline__ bool bounds_fail(int site) {
  if (atomicCAS(&g_bounds[0], 0, CQR_EBOUNDS) == 0) g_bounds[1] = site;
  return false;
}
#define CQR_CHECK(cond, site) \
  do {                        \
    if (!(cond)) {            \
      ::cqr::bounds_fail(site); \
      return;                 \
    }                         \
  } while (0)
#define CQR_CHECK_OK(cond, site) ((cond) ? true : ::cqr::bounds_fail(site))
// This file's bounds word (code, site), cleared after the read.
static inline cudaError_t bounds_take_here(int* code, int* site) {
  int v[2] = {0, 0};
  cudaError_t e = cudaMemcpyFromSymbol(v, g_bounds, sizeof(v));
  if (e != cudaSuccess) return e;
  const int z[2] = {0, 0};
  e = cudaMemcpyToSymbol(g_bounds, z, sizeof(z));
  *code = v[0];
  *site = v[1];
  return e;
}
#else
#define CQR_CHECK(cond, site) \
  do {                        \
  } while (0)
#define CQR_CHECK_OK(cond, site) true
static inline cudaError_t bounds_take_here(int* code, int* site) {
  *code = 0;
  *site = 0;
  return cudaSuccess;
}
#endif

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Upper bound of one barrier wait, in SM clock cycles (about one second at 2 GHz).  A wait
// that runs out records CQR_ETIMEOUT and returns false; every CTA then leaves the kernel.
constexpr long long kWaitLimitCycles = 2000000000LL;
// A CTA whose wait on its peers has lasted this long also polls the status word and leaves
// once any CTA has recorded an error (so that one expired wait ends the whole launch soon).
constexpr long long kPollAfterCycles = 20000LL;
// After an abandoned exchange of distributed-shared-memory stores, the pause before a CTA
// releases its shared memory (every peer has issued its last store by then).
constexpr long long kDrainCycles = 20000LL;

// Grid-wide barrier for a cooperative launch of `nblocks` CTAs.  `bar` is a global counter
// zeroed before the launch; `target` is a per-CTA running target (start at 0).  Ordering:
// CTA barrier, then thread 0 arrives with a release add (cumulative over the CTA's writes
// ordered before it by the CTA barrier) and polls with acquire loads; a CTA barrier then
// extends the acquire to every thread.
// Returns false when this CTA must abandon the kernel (own wait ran out, or another CTA
// already recorded an error).
__device__ __forceinline__ bool grid_sync(unsigned* bar, unsigned nblocks, unsigned& target,
                                          int* status, int site) {
  __shared__ int s_ok;
  __syncthreads();
  if (nblocks == 1) return true;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    target += nblocks;
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(bar), "r"(1u) : "memory");
    int ok = 1;
    const long long t0 = clock64();
    while (ld_acquire_u32(bar) < target) {
      if (ld_relaxed_i32(status + ST_CODE) == CQR_ETIMEOUT) { ok = 0; break; }
      if (clock64() - t0 > kWaitLimitCycles) {
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

// ---- distributed shared memory exchanges within a thread-block cluster
__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t peer_addr(uint32_t local_addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_addr), "r"(rank));
  return r;
}
// 16 bytes into a peer's shared memory, completing 16 transaction bytes on its mbarrier
__device__ __forceinline__ void st_async4(uint32_t dst, float4 v, uint32_t mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
               ::"r"(dst), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
               ::"r"(saddr(bar)), "r"(bytes) : "memory");
}
// non-blocking probe of the phase (the waits below use it when a bound shorter than the
// hardware's own suspend interval of try_wait is set)
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\t"
               "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
               "selp.u32 %0, 1, 0, p;\n\t}"
               : "=r"(ok) : "r"(saddr(bar)), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\t"
               "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
               "selp.u32 %0, 1, 0, p;\n\t}"
               : "=r"(ok) : "r"(saddr(bar)), "r"(parity) : "memory");
  return ok != 0;
}


// Bounded wait for phase `parity` of a shared-memory mbarrier completed by peers' st.async
// transactions.  Returns false after recording CQR_ETIMEOUT (detail `site`) when `limit`
// cycles pass, or once any CTA has recorded an error while this wait is long overdue
// (kPollAfterCycles).  try_wait may suspend the thread for the hardware's own interval before
// it returns, so a bound shorter than kPollAfterCycles (set by coded_qr_set_wait_limit) polls
// with test_wait instead.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long limit,
                                                  int* status, int site) {
  const long long t0 = clock64();
  unsigned spins = 0u;
  const bool short_bound = limit < kPollAfterCycles;
  while (!(short_bound ? mbar_test_wait(bar, parity) : mbar_try_wait(bar, parity))) {
    const long long el = clock64() - t0;
    if (el > limit) {
      set_status(status, CQR_ETIMEOUT, site);
      return false;
    }
    if (el > kPollAfterCycles && (++spins & 63u) == 0u && ld_relaxed_i32(status + ST_CODE) != 0)
      return false;
  }
  return true;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T nan_value();
template <>
__device__ __forceinline__ float nan_value<float>() { return __int_as_float(0x7fc00000); }
template <>
__device__ __forceinline__ double nan_value<double>() {
  return __longlong_as_double(0x7ff8000000000000LL);
}

}  // namespace cqr
