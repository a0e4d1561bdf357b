// cqr_kernels.cu -- CUDA-core kernels of the coded QR hot path (sm_103a):
// generator (a1), encode (a2), panel ICGS (a3), SIMT trailing-update GEMMs (a4, a5; the
// FP64 path and the FP32 reference path), erasure poisoning (a6), decode (a7),
// post-orthogonalisation (a8) and the solve (a9).  Templated on the storage type.
#include <math.h>

#include <algorithm>

#include "cqr_decode.cuh"
#include "cqr_device.cuh"
#include "cqr_kernels.cuh"

namespace cqr {

// ===================================================================== a1 generator
// Construction "Q-factor checksum-generator matrix" (Section 4.2): V~ i.i.d. Unif(0,1),
// G~_1 = -1/2 V~ V~^T; G~_h from the same stream.  SplitMix64 (Steele, Lea & Flood 2014);
// G~_1 accumulated with explicitly rounded products and sums (t ascending) so the FP64
// generator is bit-reproducible on any host.
__device__ __forceinline__ uint64_t splitmix64_next(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ double draw_unif01(uint64_t& s) {
  for (;;) {
    const uint64_t x = splitmix64_next(s) >> 11;
    if (x != 0) return __dmul_rn(__ull2double_rn(x), 0x1.0p-53);
  }
}

__device__ double draw_value(uint64_t& s, int gdist) {
  if (gdist == 0) return draw_unif01(s);
  const double u1 = draw_unif01(s), u2 = draw_unif01(s);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);  // Box-Muller
}

template <typename T>
__global__ void k_generator(int f, int p_r, int p_c, uint64_t seed, int gdist, double* Gt,
                            double* Gh, T* Gt_t, T* Gh_t) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint64_t s = seed;
  const int nv = p_r - f;
  for (int i = 0; i < f; ++i)
    for (int t = 0; t < nv; ++t) Gt[i * p_r + f + t] = draw_value(s, gdist);
  for (int i = 0; i < f; ++i)
    for (int l = 0; l < f; ++l) {
      double acc = 0.0;
      for (int t = 0; t < nv; ++t)
        acc = __dadd_rn(acc, __dmul_rn(Gt[i * p_r + f + t], Gt[l * p_r + f + t]));
      Gt[i * p_r + l] = __dmul_rn(-0.5, acc);
    }
  for (int j = 0; j < p_c; ++j)
    for (int l = 0; l < f; ++l) Gh[j * f + l] = draw_value(s, gdist);
  for (int e = 0; e < f * p_r; ++e) Gt_t[e] = (T)Gt[e];
  for (int e = 0; e < f * p_c; ++e) Gh_t[e] = (T)Gh[e];
}

template <typename T>
cudaError_t launch_generator(int f, int p_r, int p_c, uint64_t seed, int gdist, double* Gt,
                             double* Gh, T* Gt_t, T* Gh_t, cudaStream_t st) {
  k_generator<T><<<1, 32, 0, st>>>(f, p_r, p_c, seed, gdist, Gt, Gh, Gt_t, Gh_t);
  return cudaGetLastError();
}

// ===================================================================== a2 encode
// Eq. (encoding), checksum tile formula C_{i,j} = sum_t g~_{i,t} A_{t,j} (Section 4.2).
// Pass 1 (grid z = tile column j): one thread per local position (r, s) reads the p_r tiles
// A_{t,j}(r, s) once, writes them into the encoded matrix (zero-padded rows) and writes the f
// vertical checksums.  Pass 2 (grid z = tile row t, protected R only): reads the p_c tiles of
// row t (systematic or checksum) and writes the f horizontal checksums; the corner block is
// (G_v A) G_h.  Sums run in the oracle's order (t, resp. j, ascending).
// The bodies take their block coordinates as arguments so that the batched kernels can map
// a flat list of blocks over many instances onto them.
// F checksums known at compile time (F <= 8; larger f takes the generic loop, F = -1): the
// geometry in registers, per-column base pointers, eight tile loads in flight per chunk.
template <typename T, int F>
__device__ __forceinline__ void encode_vertical_f(const Geo& g, const T* __restrict__ A, int64_t lda,
                                                  const T* __restrict__ Gt, T* __restrict__ Q,
                                                  int bx, int by, int j) {
  const int mb = (int)g.mb, nb = (int)g.nb, p_r = g.p_r;
  const int f = F >= 0 ? F : g.f;
  constexpr int NA = F > 0 ? F : (F == 0 ? 1 : kMaxF);
  const int64_t m = g.m;
  const int r = bx * 32 + threadIdx.x;
  const int s = by * 8 + threadIdx.y;
  if (r >= mb || s >= nb) return;
  const int64_t col = (int64_t)j * nb + s;
  // A: m rows below lda; the encoded column: m_pad + f mb rows below ldq
  CQR_CHECK(col < g.n && lda >= m && g.m_pad + (int64_t)f * mb <= g.ldq, 101);
  const T* Ac = A + col * lda;
  T* Qc = Q + col * g.ldq;
  T acc[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) acc[i] = T(0);
  for (int t0 = 0; t0 < p_r; t0 += 8) {
    T a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t row = (int64_t)(t0 + u) * mb + r;
      a[u] = (t0 + u < p_r && row < m) ? Ac[row] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t0 + u;
      if (t >= p_r) break;
      Qc[(int64_t)t * mb + r] = a[u];
#pragma unroll
      for (int i = 0; i < NA; ++i)
        if (i < f) acc[i] += Gt[i * p_r + t] * a[u];
    }
  }
#pragma unroll
  for (int i = 0; i < NA; ++i)
    if (i < f) Qc[g.m_pad + (int64_t)i * mb + r] = acc[i];
}

// F bucket of a checksum count: the count itself up to 4, else -1 (generic)
inline int f_bucket(int f) { return f <= 4 ? f : -1; }

template <typename T, int F>
__global__ void __launch_bounds__(256, 4) k_encode_vertical(Geo g, const T* __restrict__ A, int64_t lda,
                                                          const T* __restrict__ Gt, T* __restrict__ Q) {
  encode_vertical_f<T, F>(g, A, lda, Gt, Q, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <typename T, int F>
__device__ __forceinline__ void encode_horizontal_f(const Geo& g, const T* __restrict__ Gh,
                                                    T* __restrict__ Q, int bx, int by, int t) {
  const int mb = (int)g.mb, nb = (int)g.nb, p_c = g.p_c;
  const int f = F >= 0 ? F : g.f;
  constexpr int NA = F > 0 ? F : (F == 0 ? 1 : kMaxF);
  const int r = bx * 32 + threadIdx.x;
  const int s = by * 8 + threadIdx.y;
  if (r >= mb || s >= nb) return;
  const int64_t ldq = g.ldq;
  // row (t, r) inside the encoded matrix; the checksum columns n + l nb + s inside N
  CQR_CHECK((int64_t)t * mb + r < g.M && g.M <= ldq && g.n + (int64_t)f * nb <= g.N, 102);
  T* Qr = Q + (int64_t)t * mb + r + (int64_t)s * ldq;  // row (t, r), column s of tile column 0
  const int64_t tcs = (int64_t)nb * ldq;                 // one tile column
  T acc[NA];
#pragma unroll
  for (int l = 0; l < NA; ++l) acc[l] = T(0);
  for (int j0 = 0; j0 < p_c; j0 += 8) {
    T a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = (j0 + u < p_c) ? Qr[(int64_t)(j0 + u) * tcs] : T(0);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = j0 + u;
      if (j >= p_c) break;
#pragma unroll
      for (int l = 0; l < NA; ++l)
        if (l < f) acc[l] += Gh[j * f + l] * a[u];
    }
  }
  T* Qd = Q + (int64_t)t * mb + r + (g.n + (int64_t)s) * ldq;
#pragma unroll
  for (int l = 0; l < NA; ++l)
    if (l < f) Qd[(int64_t)l * tcs] = acc[l];
}

template <typename T, int F>
__global__ void __launch_bounds__(256, 4) k_encode_horizontal(Geo g, const T* __restrict__ Gh, T* __restrict__ Q) {
  encode_horizontal_f<T, F>(g, Gh, Q, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Both codes in one pass (R protected, F <= 4 checksums, p_c <= 16 tile columns).  A block of
// 32 x 4 x 2 threads covers 32 rows r and 2 columns s of a tile position; the four threads of
// a position (r, s) split the p_c tile columns into four contiguous groups of at most four.
// Each walks its tiles A_{t,j}(r, s) once, tile row by tile row (two rows' loads in flight),
// writes them into the encoded matrix and keeps the vertical checksums of its columns in
// registers; the four partial horizontal checksums of a row, and at the end the four partial
// corners (G_h applied to the vertical checksums), are added through shared memory in group
// order.  A is read once and the encoded matrix written once.  Vertical sums run over t
// ascending, as in the oracle; horizontal sums over j ascending within a group, groups in order.
template <typename T, int F>
__global__ void __launch_bounds__(256) k_encode_fused(Geo g, const T* __restrict__ A, int64_t lda,
                                                     const T* __restrict__ Gt,
                                                     const T* __restrict__ Gh, T* __restrict__ Q) {
  constexpr int KMAX = 4;  // tile columns per thread
  __shared__ T hs[2][2][4][F][32];  // [row parity][s][group][l][r]
  const int mb = (int)g.mb, nb = (int)g.nb, p_r = g.p_r, p_c = g.p_c;
  const int64_t m = g.m, ldq = g.ldq;
  const int tx = threadIdx.x, jg = threadIdx.y, sz = threadIdx.z;
  const int r = blockIdx.x * 32 + tx;
  const int s = blockIdx.y * 2 + sz;
  const bool live = r < mb && s < nb;
  const int cpg = (p_c + 3) / 4;
  const int j0 = jg * cpg;
  const int nj = max(0, min(cpg, p_c - j0));
  // uniform over the launch, before the barriers: the geometry the indexing below assumes
  CQR_CHECK(p_c <= 4 * KMAX && lda >= m && g.M <= ldq && g.n + (int64_t)F * nb <= g.N &&
                g.m_pad + (int64_t)F * mb <= g.M, 112);
  T vacc[KMAX][F];
#pragma unroll
  for (int k = 0; k < KMAX; ++k)
#pragma unroll
    for (int i = 0; i < F; ++i) vacc[k][i] = T(0);
  for (int t0 = 0; t0 < p_r; t0 += 2) {
    T a[2][KMAX];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const int64_t row = (int64_t)(t0 + d) * mb + r;
      const bool in = live && t0 + d < p_r && row < m;
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
        a[d][k] = (in && k < nj) ? A[row + ((int64_t)(j0 + k) * nb + s) * lda] : T(0);
    }
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const int t = t0 + d;
      if (t >= p_r) break;
      const int64_t row = (int64_t)t * mb + r;
      T h[F];
#pragma unroll
      for (int l = 0; l < F; ++l) h[l] = T(0);
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
        if (k < nj) {
          const int j = j0 + k;
          if (live) Q[row + ((int64_t)j * nb + s) * ldq] = a[d][k];
#pragma unroll
          for (int i = 0; i < F; ++i) vacc[k][i] += Gt[i * p_r + t] * a[d][k];
#pragma unroll
          for (int l = 0; l < F; ++l) h[l] += Gh[j * F + l] * a[d][k];
        }
#pragma unroll
      for (int l = 0; l < F; ++l) hs[t & 1][sz][jg][l][tx] = h[l];
      __syncthreads();
      if (jg < F && live) {  // thread group jg writes checksum l = jg of this row
        const int l = jg;
        T sum = hs[t & 1][sz][0][l][tx];
        for (int q = 1; q < 4; ++q) sum += hs[t & 1][sz][q][l][tx];
        Q[row + (g.n + (int64_t)l * nb + s) * ldq] = sum;
      }
    }
  }
  // vertical checksums of this thread's columns, then the corner through shared memory
#pragma unroll
  for (int i = 0; i < F; ++i) {
    const int64_t row = g.m_pad + (int64_t)i * mb + r;
    T c[F];
#pragma unroll
    for (int l = 0; l < F; ++l) c[l] = T(0);
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
      if (k < nj) {
        const int j = j0 + k;
        if (live) Q[row + ((int64_t)j * nb + s) * ldq] = vacc[k][i];
#pragma unroll
        for (int l = 0; l < F; ++l) c[l] += Gh[j * F + l] * vacc[k][i];
      }
    __syncthreads();  // the previous round's reads of hs are done
#pragma unroll
    for (int l = 0; l < F; ++l) hs[0][sz][jg][l][tx] = c[l];
    __syncthreads();
    if (jg < F && live) {
      const int l = jg;
      T sum = hs[0][sz][0][l][tx];
      for (int q = 1; q < 4; ++q) sum += hs[0][sz][q][l][tx];
      Q[row + (g.n + (int64_t)l * nb + s) * ldq] = sum;
    }
  }
}

template <typename T, int F>
cudaError_t launch_encode_f(const Geo& g, const T* A, int64_t lda, const T* Gt, const T* Gh, T* Q,
                            cudaStream_t st) {
  if constexpr (F > 0) {
    if (g.protect_r && g.p_c <= 16) {
      dim3 grd((unsigned)((g.mb + 31) / 32), (unsigned)((g.nb + 1) / 2));
      dim3 blk(32, 4, 2);
      k_encode_fused<T, F><<<grd, blk, 0, st>>>(g, A, lda, Gt, Gh, Q);
      return cudaGetLastError();
    }
  }
  dim3 blk(32, 8);
  dim3 grd((unsigned)((g.mb + 31) / 32), (unsigned)((g.nb + 7) / 8), (unsigned)g.p_c);
  k_encode_vertical<T, F><<<grd, blk, 0, st>>>(g, A, lda, Gt, Q);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !g.protect_r || g.f == 0) return e;
  grd.z = (unsigned)(g.p_r + g.f);
  k_encode_horizontal<T, F><<<grd, blk, 0, st>>>(g, Gh, Q);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_encode(const Geo& g, const T* A, int64_t lda, const T* Gt, const T* Gh, T* Q,
                          int* status, cudaStream_t st) {
  (void)status;
  switch (f_bucket(g.f)) {
    case 0: return launch_encode_f<T, 0>(g, A, lda, Gt, Gh, Q, st);
    case 1: return launch_encode_f<T, 1>(g, A, lda, Gt, Gh, Q, st);
    case 2: return launch_encode_f<T, 2>(g, A, lda, Gt, Gh, Q, st);
    case 3: return launch_encode_f<T, 3>(g, A, lda, Gt, Gh, Q, st);
    case 4: return launch_encode_f<T, 4>(g, A, lda, Gt, Gh, Q, st);
    default: return launch_encode_f<T, -1>(g, A, lda, Gt, Gh, Q, st);
  }
}

// ===================================================================== a4/a5 SIMT GEMMs
// Rbar = Qbar^T Qtrail (split over K) and Qtrail -= Qbar Rbar on CUDA cores: the FP64 path
// and the FP32 reference path.  64 x 64 output tiles, 256 threads, 4 x 4 per thread with a
// stride-16 micro-tile so that each half-warp touches 16 consecutive rows.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm_tn_splitk(const T* __restrict__ A, int64_t lda,
                                                         const T* __restrict__ B, int64_t ldb,
                                                         int64_t K, int bk, int64_t w,
                                                         int64_t kchunk, T* __restrict__ P) {
  __shared__ T As[32][65];
  __shared__ T Bs[32][65];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  CQR_CHECK(lda >= K && ldb >= K, 103);  // uniform over the launch: before any barrier
  const int i0 = blockIdx.x * 64;
  const int64_t j0 = (int64_t)blockIdx.y * 64;
  const int64_t k0 = (int64_t)blockIdx.z * kchunk;
  const int64_t k1 = (k0 + kchunk < K) ? k0 + kchunk : K;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int64_t kb = k0; kb < k1; kb += 32) {
    const int kk = tid & 31;
    const int64_t k = kb + kk;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int ii = (tid >> 5) + 8 * e;
      const int i = i0 + ii;
      As[kk][ii] = (k < k1 && i < bk) ? A[k + (int64_t)i * lda] : T(0);
      const int64_t j = j0 + ii;
      Bs[kk][ii] = (k < k1 && j < w) ? B[k + j * ldb] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < 32; ++q) {
      T a[4], b[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) { a[e] = As[q][tx + 16 * e]; b[e] = Bs[q][ty + 16 * e]; }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * b[y];
    }
    __syncthreads();
  }
  T* Ps = P + (size_t)blockIdx.z * (size_t)bk * (size_t)w;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int i = i0 + tx + 16 * x;
      const int64_t j = j0 + ty + 16 * y;
      if (i < bk && j < w) Ps[i + j * bk] = acc[x][y];
    }
}

template <typename T>
cudaError_t launch_gemm_tn_splitk(const T* A, int64_t lda, const T* B, int64_t ldb, int64_t K,
                                  int bk, int64_t w, int splits, T* P, cudaStream_t st) {
  int64_t kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + 31) / 32 * 32;
  dim3 grd((unsigned)((bk + 63) / 64), (unsigned)((w + 63) / 64), (unsigned)splits);
  k_gemm_tn_splitk<T><<<grd, 256, 0, st>>>(A, lda, B, ldb, K, bk, w, kchunk, P);
  return cudaGetLastError();
}

// Sum the split partials in a fixed order; store (accumulate = 0) or add (accumulate = 1)
// into R, and store into the compact operand Rb.
template <typename T>
__global__ void k_splitk_reduce(const T* __restrict__ P, int splits, int bk, int64_t w,
                                T* __restrict__ R, int64_t ldr, T* __restrict__ Rb, int accumulate) {
  CQR_CHECK(ldr >= bk, 104);
  const int64_t total = (int64_t)bk * w;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    T s = T(0);
    for (int sp = 0; sp < splits; ++sp) s += P[(size_t)sp * total + idx];
    const int64_t i = idx % bk, j = idx / bk;
    if (accumulate)
      R[i + j * ldr] += s;
    else
      R[i + j * ldr] = s;
    Rb[idx] = s;
  }
}

template <typename T>
cudaError_t launch_splitk_reduce(const T* P, int splits, int bk, int64_t w, T* R, int64_t ldr,
                                 T* Rb, cudaStream_t st, int accumulate) {
  const int64_t total = (int64_t)bk * w;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_splitk_reduce<T><<<blocks, 256, 0, st>>>(P, splits, bk, w, R, ldr, Rb, accumulate);
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_nn_sub(const T* __restrict__ A, int64_t lda,
                                                      const T* __restrict__ B, int64_t ldb,
                                                      T* __restrict__ C, int64_t ldc, int64_t M,
                                                      int bk, int64_t w) {
  __shared__ T As[32][65];
  __shared__ T Bs[32][65];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  CQR_CHECK(lda >= M && ldc >= M && ldb >= bk, 105);  // uniform: before any barrier
  const int64_t i0 = (int64_t)blockIdx.x * 64;
  const int64_t j0 = (int64_t)blockIdx.y * 64;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int kb = 0; kb < bk; kb += 32) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int ii = tid & 63, kk = (tid >> 6) + 4 * e;
      const int64_t i = i0 + ii;
      const int k = kb + kk;
      As[kk][ii] = (i < M && k < bk) ? A[i + (int64_t)k * lda] : T(0);
      const int kk2 = tid & 31, jj = (tid >> 5) + 8 * e;
      const int64_t j = j0 + jj;
      const int k2 = kb + kk2;
      Bs[kk2][jj] = (j < w && k2 < bk) ? B[k2 + j * ldb] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < 32; ++q) {
      T a[4], b[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) { a[e] = As[q][tx + 16 * e]; b[e] = Bs[q][ty + 16 * e]; }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * b[y];
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t i = i0 + tx + 16 * x;
      const int64_t j = j0 + ty + 16 * y;
      if (i < M && j < w) C[i + j * ldc] -= acc[x][y];
    }
}

template <typename T>
cudaError_t launch_gemm_nn_sub(const T* A, int64_t lda, const T* B, int64_t ldb, T* C,
                               int64_t ldc, int64_t M, int bk, int64_t w, cudaStream_t st) {
  dim3 grd((unsigned)((M + 63) / 64), (unsigned)((w + 63) / 64));
  k_gemm_nn_sub<T><<<grd, 256, 0, st>>>(A, lda, B, ldb, C, ldc, M, bk, w);
  return cudaGetLastError();
}

// ===================================================================== a6 erasure
// Section 2 "Failure model": a failed node loses its data -- its tiles are overwritten with
// NaN so that any later read of an erased value propagates into the results.
struct TileList {
  int count;
  int ij[2 * 64];
};

template <typename T>
__global__ void k_poison(T* __restrict__ X, int64_t ld, int64_t th, int64_t tw, TileList tl) {
  const int e = blockIdx.y;
  const int i = tl.ij[2 * e], j = tl.ij[2 * e + 1];
  CQR_CHECK(e < tl.count && i >= 0 && j >= 0 && (int64_t)(i + 1) * th <= ld, 106);
  const int64_t total = th * tw;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx % th, s = idx / th;
    X[(int64_t)i * th + r + ((int64_t)j * tw + s) * ld] = nan_value<T>();
  }
}

template <typename T>
cudaError_t launch_poison(const Geo& g, const int* tiles, int count, T* Q, T* R,
                          cudaStream_t st) {
  for (int base = 0; base < count; base += 64) {
    TileList q{}, rl{};
    const int n = (count - base) < 64 ? (count - base) : 64;
    for (int e = 0; e < n; ++e) {
      const int i = tiles[2 * (base + e)], j = tiles[2 * (base + e) + 1];
      q.ij[2 * q.count] = i;
      q.ij[2 * q.count + 1] = j;
      ++q.count;
      if (g.protect_r && i < g.p_c + g.f) {
        rl.ij[2 * rl.count] = i;
        rl.ij[2 * rl.count + 1] = j;
        ++rl.count;
      }
    }
    int bx = (int)((g.mb * g.nb + 255) / 256);
    if (bx > 1024) bx = 1024;
    k_poison<T><<<dim3(bx, q.count), 256, 0, st>>>(Q, g.ldq, g.mb, g.nb, q);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (rl.count > 0) {
      int by = (int)((g.nb * g.nb + 255) / 256);
      if (by > 1024) by = 1024;
      k_poison<T><<<dim3(by, rl.count), 256, 0, st>>>(R, g.ldr, g.nb, g.nb, rl);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// ===================================================================== a7 decode
// The decode itself (setup of a code's coefficient tables, recovery of one position) is in
// cqr_decode.cuh; here one CTA of 32 x 8 threads builds the code's tables once and recovers
// rows 32 bx .. 32 bx + 31 of the 8-column group by of one code, and with Strided also of the
// groups by + sy, by + 2 sy, ...
template <typename T, bool Strided>
__device__ __forceinline__ void decode_body(const Geo& g, const DecodePlan& p,
                                            const double* __restrict__ Gt,
                                            const double* __restrict__ Gh, T* Q, T* R,
                                            int* status, int bx, int by, int sy) {
  __shared__ DecodeScratch<T> sh;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  // the plan names a code of the grid and at most f lost tiles (uniform over the CTA)
  CQR_CHECK(p.f1 + p.f2 <= g.f && p.idx >= 0 &&
                p.idx < (p.kind == 0 ? g.grid_cols : g.p_c + g.f) && g.M <= g.ldq, 107);
  if (!decode_setup<T>(g, p, Gt, Gh, sh, tid, blockDim.x * blockDim.y, status, bx == 0 && by == 0))
    return;
  const int64_t h = p.kind == 0 ? g.mb : g.nb;
  const int64_t r = (int64_t)bx * blockDim.x + threadIdx.x;
  if (r >= h) return;
  if constexpr (Strided) {
    for (int64_t s = (int64_t)by * blockDim.y + threadIdx.y; s < g.nb;
         s += (int64_t)sy * blockDim.y)
      decode_apply<T, 4>(g, p, sh, Q, R, r, s);
  } else {
    (void)sy;
    const int64_t s = (int64_t)by * blockDim.y + threadIdx.y;
    if (s < g.nb) decode_apply<T, 4>(g, p, sh, Q, R, r, s);
  }
}

// Four rows per thread (FP32, f <= 4, tile heights and leading dimensions multiples of four):
// a 32 x 8 block covers 128 rows of 8 position columns, strided over the grid's y.
__global__ void __launch_bounds__(256) k_decode4(Geo g, const DecodePlan* __restrict__ plans,
                                                  const double* __restrict__ Gt,
                                                  const double* __restrict__ Gh, float* Q,
                                                  float* R, int* status) {
  __shared__ DecodeScratch<float> sh;
  const DecodePlan& p = plans[blockIdx.z];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  CQR_CHECK(p.f1 + p.f2 <= g.f && g.f <= 4 && p.idx >= 0 &&
                p.idx < (p.kind == 0 ? g.grid_cols : g.p_c + g.f) && g.M <= g.ldq &&
                g.mb % 4 == 0 && g.nb % 4 == 0 && g.ldq % 4 == 0 && g.ldr % 4 == 0, 111);
  if (!decode_setup<float>(g, p, Gt, Gh, sh, tid, blockDim.x * blockDim.y, status,
                           blockIdx.x == 0 && blockIdx.y == 0))
    return;
  const int64_t h = p.kind == 0 ? g.mb : g.nb;
  const int64_t r4 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (r4 >= h) return;
  for (int64_t s = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; s < g.nb;
       s += (int64_t)gridDim.y * blockDim.y)
    decode_apply4(g, p, sh, Q, R, r4, s);
}

template <typename T>
__global__ void __launch_bounds__(256) k_decode(Geo g, const DecodePlan* __restrict__ plans,
                                                 const double* __restrict__ Gt,
                                                 const double* __restrict__ Gh, T* Q, T* R,
                                                 int* status) {
  decode_body<T, true>(g, plans[blockIdx.z], Gt, Gh, Q, R, status, blockIdx.x, blockIdx.y,
                       gridDim.y);
}

template <typename T>
cudaError_t launch_decode(const Geo& g, const DecodePlan* plans_dev, int nplans, int max_h,
                          const double* Gt, const double* Gh, T* Q, T* R, int* status,
                          cudaStream_t st) {
  if (nplans == 0) return cudaSuccess;
  // about one wave (768 CTAs over all codes), so that each CTA's table setup is amortised
  // over several 8-column groups
  dim3 blk(32, 8);
  const int64_t nby = (g.nb + 7) / 8;
  if (sizeof(T) == 4 && g.f <= 4 && g.mb % 4 == 0 && g.nb % 4 == 0 && g.ldq % 4 == 0 &&
      g.ldr % 4 == 0) {
    // 16-byte accesses, four rows per thread: a block covers 128 rows
    const int64_t nbx = (max_h + 127) / 128;
    // one wave of resident CTAs over all codes, so that each CTA builds its tables once and
    // then streams several 8-column groups
    int occ = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_decode4, 256, 0) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      occ = 4;
      sms = 152;
    }
    const int64_t resident = (int64_t)std::max(1, occ) * std::max(1, sms);
    const int64_t gy = std::max<int64_t>(
        1, std::min<int64_t>(nby, resident / std::max<int64_t>(1, nbx * nplans)));
    dim3 grd((unsigned)nbx, (unsigned)gy, (unsigned)nplans);
    k_decode4<<<grd, blk, 0, st>>>(g, plans_dev, Gt, Gh, reinterpret_cast<float*>(Q),
                                   reinterpret_cast<float*>(R), status);
    return cudaGetLastError();
  }
  const int64_t nbx = (max_h + 31) / 32;
  const int64_t gy = std::max<int64_t>(1, std::min<int64_t>(nby, 768 / std::max<int64_t>(1, nbx * nplans)));
  dim3 grd((unsigned)nbx, (unsigned)gy, (unsigned)nplans);
  k_decode<T><<<grd, blk, 0, st>>>(g, plans_dev, Gt, Gh, Q, R, status);
  return cudaGetLastError();
}

// ===================================================================== a8 post-orth
// Sparse block pipeline of G_0 Z (Appendix, proof of the overhead theorem): with
// H = I + G~_1 and Z_t the t-th block row,
//   W_i = sum_{l<f} h_{i,l} Z_l + sum_{t>=f} g~_{i,t} Z_t   (i < f)
//   W_i = sum_{l<f} g~_{l,i} Z_l - Z_i                      (i >= f)
// One thread per (local row, column): reads each Z_t once, writes each W_i once (in place
// is safe: every thread owns one position across all block rows).
// F checksums known at compile time (F <= 4; -1: generic up to kMaxF), eight tile loads in
// flight per chunk of the t loop; the order of every sum is unchanged.  W may alias Z: each
// position is read before it is written.
template <typename T, int F>
__device__ __forceinline__ void post_orth_f(const Geo& g, const T* __restrict__ Gt, const T* Z,
                                            int64_t ldz, int64_t zrows, int64_t k, T* W,
                                            int64_t ldw, int bx, int by) {
  constexpr int NA = F > 0 ? F : (F == 0 ? 1 : kMaxF);
  const int64_t s = (int64_t)bx * 32 + threadIdx.x;
  const int64_t col = (int64_t)by * 8 + threadIdx.y;
  const int64_t mb = g.mb;
  if (s >= mb || col >= k) return;
  const int f = F >= 0 ? F : g.f, p_r = g.p_r;
  // every block row t < p_r of W lies below ldw; Z is read below zrows <= ldz
  CQR_CHECK((int64_t)p_r * mb <= ldw && zrows <= ldz, 108);
  const T* zc = Z + col * ldz;
  T* wc = W + col * ldw;
  T zl[NA], acc[NA];
#pragma unroll
  for (int l = 0; l < NA; ++l) {
    const int64_t row = (int64_t)l * mb + s;
    zl[l] = (l < f && row < zrows) ? zc[row] : T(0);
  }
#pragma unroll
  for (int i = 0; i < NA; ++i) {
    T a = T(0);
    if (i < f) {
#pragma unroll
      for (int l = 0; l < NA; ++l)
        if (l < f) a += ((l == i ? T(1) : T(0)) + Gt[i * p_r + l]) * zl[l];
    }
    acc[i] = a;
  }
  for (int t0 = f; t0 < p_r; t0 += 8) {
    T z[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t row = (int64_t)(t0 + u) * mb + s;
      z[u] = (t0 + u < p_r && row < zrows) ? zc[row] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t0 + u;
      if (t >= p_r) break;
#pragma unroll
      for (int i = 0; i < NA; ++i)
        if (i < f) acc[i] += Gt[i * p_r + t] * z[u];
      T wv = T(0);
#pragma unroll
      for (int l = 0; l < NA; ++l)
        if (l < f) wv += Gt[l * p_r + t] * zl[l];
      wc[(int64_t)t * mb + s] = wv - z[u];
    }
  }
#pragma unroll
  for (int i = 0; i < NA; ++i)
    if (i < f) wc[(int64_t)i * mb + s] = acc[i];
}

template <typename T, int F>
__global__ void __launch_bounds__(256, 4) k_post_orth(Geo g, const T* __restrict__ Gt, const T* Z,
                                                       int64_t ldz, int64_t zrows, int64_t k, T* W,
                                                       int64_t ldw) {
  post_orth_f<T, F>(g, Gt, Z, ldz, zrows, k, W, ldw, blockIdx.x, blockIdx.y);
}

template <typename T>
cudaError_t launch_post_orth(const Geo& g, const T* Gt_t, const T* Z, int64_t ldz,
                             int64_t zrows, int64_t k, T* W, int64_t ldw, cudaStream_t st) {
  dim3 blk(32, 8);
  dim3 grd((unsigned)((g.mb + 31) / 32), (unsigned)((k + 7) / 8));
  switch (f_bucket(g.f)) {
    case 0: k_post_orth<T, 0><<<grd, blk, 0, st>>>(g, Gt_t, Z, ldz, zrows, k, W, ldw); break;
    case 1: k_post_orth<T, 1><<<grd, blk, 0, st>>>(g, Gt_t, Z, ldz, zrows, k, W, ldw); break;
    case 2: k_post_orth<T, 2><<<grd, blk, 0, st>>>(g, Gt_t, Z, ldz, zrows, k, W, ldw); break;
    case 3: k_post_orth<T, 3><<<grd, blk, 0, st>>>(g, Gt_t, Z, ldz, zrows, k, W, ldw); break;
    case 4: k_post_orth<T, 4><<<grd, blk, 0, st>>>(g, Gt_t, Z, ldz, zrows, k, W, ldw); break;
    default: k_post_orth<T, -1><<<grd, blk, 0, st>>>(g, Gt_t, Z, ldz, zrows, k, W, ldw); break;
  }
  return cudaGetLastError();
}

// ===================================================================== a8, drift-robust form
// W = G_0^{-1} (Q_1 + G^T Q_2) with G = G~ (x) I_mb (reading of Theorem G_0 for checksum rows
// that drift from G Q_1 in floating point).  Write Q_2 = G Q_1 + D (D the drift).  Since
// G_0^2 = I + G^T G (G_0 symmetric), G_0^{-1}(I + G^T G) = G_0, and by the push-through
// identity (I + G~^T G~)^{-1} G~^T = G~^T K with K = (I_f + G~ G~^T)^{-1}:
//   W = G_0 Q_1 + G_0^{-1} G^T D = G_0 (Q_1 + G^T K D)   (K acting on block rows).
// Per tile position s and column j, with z_t the entry of block row t of Q_1 and c_i that of
// block row i of Q_2:
//   d = c - G~ z,   e = K d,   Z = z + G~^T e,   W = G_0 Z   (the block pipeline of post_orth_f:
//   W_i = Z_i + (G~ Z)_i for i < f, W_t = sum_{l<f} g~_{l,t} Z_l - Z_t for t >= f).
// The correction is formed from the drift itself, so the coefficients' rounding in the
// storage type perturbs W only by that rounding times |G~^T K| <= 1/2 (no cancellation of
// the large (I + G~^T G~) z against G~^T G~ z); with D = 0, W is G_0 Q_1 computed as the
// paper's pipeline.

// K from the FP64 generator: Cholesky L L^T = I_f + G~ G~^T (Golub and Van Loan, the outer
// product form), then K = L^{-T} L^{-1} column by column; one thread.  F > 0: f = F known at
// compile time, every loop unrolled and the f x f work in registers (F = -1: generic f <=
// kMaxF).
template <typename T, int F>
__global__ void k_post_orth_coef(int f_rt, int p_r, const double* __restrict__ Gt, double* K64,
                                 T* Kt) {
  constexpr int NF = F > 0 ? F : kMaxF;
  const int f = F > 0 ? F : f_rt;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double A[NF][NF];
#pragma unroll
  for (int i = 0; i < NF; ++i)
#pragma unroll
    for (int l = 0; l < NF; ++l) {
      if (i >= f || l > i) continue;
      double a = (i == l) ? 1.0 : 0.0;
      for (int t = 0; t < p_r; ++t) a += Gt[i * p_r + t] * Gt[l * p_r + t];
      A[i][l] = a;
    }
  // lower triangle of A overwritten by L
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    if (j >= f) continue;
    double d = A[j][j];
#pragma unroll
    for (int k = 0; k < NF; ++k)
      if (k < j) d -= A[j][k] * A[j][k];
    d = sqrt(d);
    A[j][j] = d;
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      if (i <= j || i >= f) continue;
      double v = A[i][j];
#pragma unroll
      for (int k = 0; k < NF; ++k)
        if (k < j) v -= A[i][k] * A[j][k];
      A[i][j] = v / d;
    }
  }
#pragma unroll
  for (int col = 0; col < NF; ++col) {
    if (col >= f) continue;
    double x[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) {          // L x = e_col
      if (i >= f) continue;
      double v = (i == col) ? 1.0 : 0.0;
#pragma unroll
      for (int k = 0; k < NF; ++k)
        if (k < i) v -= A[i][k] * x[k];
      x[i] = v / A[i][i];
    }
#pragma unroll
    for (int i = NF - 1; i >= 0; --i) {     // L^T x = x
      if (i >= f) continue;
      double v = x[i];
#pragma unroll
      for (int k = 0; k < NF; ++k)
        if (k > i && k < f) v -= A[k][i] * x[k];
      x[i] = v / A[i][i];
    }
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      if (i >= f) continue;
      K64[i * f + col] = x[i];
      Kt[i * f + col] = (T)x[i];
    }
  }
}

// One thread per (position s, column j), 32 x 8 threads per CTA.  ONE: every block row of the
// position in registers (p_r <= 32), Q_1 and Q_2 read once; otherwise two passes over Q_1
// (d first, then Z, G~ Z and the rows t >= f of W), the f values Z_0 .. Z_{f-1} kept between
// them.  Coefficients in shared memory.  W may alias Q_1: each thread reads its own position
// before writing it.
template <typename T, int F, bool ONE>
__global__ void __launch_bounds__(256) k_post_orth_proj(Geo g, const T* __restrict__ Gt,
                                                        const T* __restrict__ Kt, const T* Q,
                                                        int64_t ldq, int64_t k, T* W,
                                                        int64_t ldw) {
  constexpr int NF = F > 0 ? F : kMaxF;
  constexpr int PR = 32;
  __shared__ T sG[kMaxF * kMaxCode];
  __shared__ T sK[kMaxF * kMaxF];
  const int f = F > 0 ? F : g.f, p_r = g.p_r;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int e = tid; e < f * p_r; e += 256) sG[e] = Gt[e];
  for (int e = tid; e < f * f; e += 256) sK[e] = Kt[e];
  __syncthreads();
  const int64_t s = (int64_t)blockIdx.x * 32 + threadIdx.x;
  const int64_t col = (int64_t)blockIdx.y * 8 + threadIdx.y;
  const int64_t mb = g.mb;
  if (s >= mb || col >= k) return;
  // Q_1 and Q_2 (m_pad + f mb rows) below ldq; W's m_pad rows below ldw
  CQR_CHECK(g.m_pad + (int64_t)f * mb <= ldq && g.m_pad <= ldw && p_r * mb == g.m_pad, 109);
  const T* qc = Q + col * ldq;
  T* wc = W + col * ldw;
  T d[NF], e[NF], a[NF];
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    d[i] = (i < f) ? qc[g.m_pad + (int64_t)i * mb + s] : T(0);
    a[i] = T(0);
  }
  if constexpr (ONE) {
    T z[PR];
#pragma unroll
    for (int t = 0; t < PR; ++t) z[t] = (t < p_r) ? qc[(int64_t)t * mb + s] : T(0);
    // d = c - G~ z
#pragma unroll
    for (int t = 0; t < PR; ++t)
      if (t < p_r)
#pragma unroll
        for (int i = 0; i < NF; ++i)
          if (i < f) d[i] -= sG[i * p_r + t] * z[t];
    // e = K d
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      T u = T(0);
#pragma unroll
      for (int l = 0; l < NF; ++l)
        if (l < f) u += sK[i * f + l] * d[l];
      e[i] = u;
    }
    // Z = z + G~^T e, a = G~ Z
#pragma unroll
    for (int t = 0; t < PR; ++t) {
      if (t < p_r) {
        T zt = z[t];
#pragma unroll
        for (int i = 0; i < NF; ++i)
          if (i < f) zt += sG[i * p_r + t] * e[i];
        z[t] = zt;
#pragma unroll
        for (int i = 0; i < NF; ++i)
          if (i < f) a[i] += sG[i * p_r + t] * zt;
      }
    }
    // W = G_0 Z
#pragma unroll
    for (int t = 0; t < PR; ++t) {
      if (t < p_r) {
        T w;
        if (t < f) {
          w = z[t] + a[t < NF ? t : 0];
        } else {
          w = T(0);
#pragma unroll
          for (int l = 0; l < NF; ++l)
            if (l < f) w += sG[l * p_r + t] * z[l];
          w -= z[t];
        }
        wc[(int64_t)t * mb + s] = w;
      }
    }
  } else {
    // pass 1: d = c - G~ z over every block row
    for (int t0 = 0; t0 < p_r; t0 += 8) {
      T z[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) z[u] = (t0 + u < p_r) ? qc[(int64_t)(t0 + u) * mb + s] : T(0);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (t0 + u < p_r)
#pragma unroll
          for (int i = 0; i < NF; ++i)
            if (i < f) d[i] -= sG[i * p_r + t0 + u] * z[u];
    }
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      T u = T(0);
#pragma unroll
      for (int l = 0; l < NF; ++l)
        if (l < f) u += sK[i * f + l] * d[l];
      e[i] = u;
    }
    // pass 2: Z, a = G~ Z, and the rows t >= f of W (Z_0 .. Z_{f-1} come first)
    T zf[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) zf[i] = T(0);
    for (int t0 = 0; t0 < p_r; t0 += 8) {
      T z[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) z[u] = (t0 + u < p_r) ? qc[(int64_t)(t0 + u) * mb + s] : T(0);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t = t0 + u;
        if (t < p_r) {
          T zt = z[u];
#pragma unroll
          for (int i = 0; i < NF; ++i)
            if (i < f) zt += sG[i * p_r + t] * e[i];
#pragma unroll
          for (int i = 0; i < NF; ++i)
            if (i < f) a[i] += sG[i * p_r + t] * zt;
          if (t < f) {
#pragma unroll
            for (int i = 0; i < NF; ++i)
              if (i == t) zf[i] = zt;
          } else {
            T w = T(0);
#pragma unroll
            for (int l = 0; l < NF; ++l)
              if (l < f) w += sG[l * p_r + t] * zf[l];
            wc[(int64_t)t * mb + s] = w - zt;
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NF; ++i)
      if (i < f) wc[(int64_t)i * mb + s] = zf[i] + a[i];
  }
}

template <typename T>
cudaError_t launch_post_orth_projected(const Geo& g, const double* Gt, const T* Gt_t, double* K64,
                                       T* Kt, const T* Q, int64_t ldq, int64_t k, T* W, int64_t ldw,
                                       cudaStream_t st) {
  if (g.f < 1 || g.f > kMaxF || g.p_r + g.f > kMaxCode) return cudaErrorInvalidValue;
  switch (f_bucket(g.f)) {
    case 1: k_post_orth_coef<T, 1><<<1, 32, 0, st>>>(g.f, g.p_r, Gt, K64, Kt); break;
    case 2: k_post_orth_coef<T, 2><<<1, 32, 0, st>>>(g.f, g.p_r, Gt, K64, Kt); break;
    case 3: k_post_orth_coef<T, 3><<<1, 32, 0, st>>>(g.f, g.p_r, Gt, K64, Kt); break;
    case 4: k_post_orth_coef<T, 4><<<1, 32, 0, st>>>(g.f, g.p_r, Gt, K64, Kt); break;
    default: k_post_orth_coef<T, -1><<<1, 32, 0, st>>>(g.f, g.p_r, Gt, K64, Kt); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 blk(32, 8);
  dim3 grd((unsigned)((g.mb + 31) / 32), (unsigned)((k + 7) / 8));
  const bool one = g.p_r <= 32;
#define CQR_PO_PROJ(FF)                                                                         \
  if (one) k_post_orth_proj<T, FF, true><<<grd, blk, 0, st>>>(g, Gt_t, Kt, Q, ldq, k, W, ldw);  \
  else k_post_orth_proj<T, FF, false><<<grd, blk, 0, st>>>(g, Gt_t, Kt, Q, ldq, k, W, ldw);
  switch (f_bucket(g.f)) {
    case 1: CQR_PO_PROJ(1) break;
    case 2: CQR_PO_PROJ(2) break;
    case 3: CQR_PO_PROJ(3) break;
    case 4: CQR_PO_PROJ(4) break;
    default: CQR_PO_PROJ(-1) break;
  }
#undef CQR_PO_PROJ
  return cudaGetLastError();
}

// ===================================================================== a9 solve
// z = Qo^T yo (Eq. (linearsolve3)), one warp per output entry.
template <typename T>
__global__ void __launch_bounds__(256) k_gemv_t(const T* __restrict__ Qo, int64_t ldq, int64_t rows,
                                                 int64_t n, const T* __restrict__ y, int64_t ldy,
                                                 int64_t k, T* __restrict__ z, int64_t ldz) {
  const int lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int64_t col = blockIdx.y;
  if (j >= n) return;
  CQR_CHECK(rows <= ldq && rows <= ldy && n <= ldz, 110);
  const T* q = Qo + j * ldq;
  const T* yy = y + col * ldy;
  T acc = T(0);
  for (int64_t r = lane; r < rows; r += 32) acc += q[r] * yy[r];
  acc = warp_sum(acc);
  if (lane == 0) z[j + col * ldz] = acc;
}

template <typename T>
cudaError_t launch_gemv_t(const T* Qo, int64_t ldq, int64_t rows, int64_t n, const T* y,
                          int64_t ldy, int64_t k, T* z, int64_t ldz, cudaStream_t st) {
  dim3 grd((unsigned)((n + 7) / 8), (unsigned)k);
  k_gemv_t<T><<<grd, 256, 0, st>>>(Qo, ldq, rows, n, y, ldy, k, z, ldz);
  return cudaGetLastError();
}

// Blocked back substitution (Golub & Van Loan, Alg. 3.1.4, column version) on one thread-block
// cluster of C CTAs.  The 64-row blocks of x are owned cyclically (block p by CTA p % C) and
// live in the owner's shared memory from start to end.  Phase p (p = nblk-1 .. 0):
//   * the owner of block p applies the just-solved x_{p+1} to it (the R[p, p+1] tile is
//     already in shared memory), solves the 64 x 64 diagonal system in one warp and stores
//     x_p into every CTA's shared memory (distributed shared memory, buffer p mod 3);
//   * every CTA arrives at the cluster barrier (release), then, off the critical path, applies
//     x_{p+1} to its other blocks below p from tiles R[i, p+1] that cp.async brought into
//     shared memory during the previous phase, starts the copies of the tiles R[i, p] that
//     the next phase needs (and of its next diagonal block), then waits (acquire).
// The diagonal solve goes by 8-row sub-blocks: the warp gathers the sub-block's 8 right-hand
// sides by shuffle, every lane solves the 8 x 8 triangle (reciprocals of the diagonal
// precomputed), and the lanes owning rows above the sub-block apply it.  Every update of b_i
// by x_j (i < j) happens once: by i's owner, in phase j-1.  Three x buffers suffice: when
// the owner of p writes buffer p mod 3, every CTA has arrived at phase p+1's barrier, so none
// still reads x_{p+3}.  Tiles are column-major with a padded column stride (16-byte aligned).
template <typename T>
__device__ __forceinline__ void st_dsmem(T* local, uint32_t rank, T v);
template <>
__device__ __forceinline__ void st_dsmem<float>(float* local, uint32_t rank, float v) {
  uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(local)), r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(r), "f"(v) : "memory");
}
template <>
__device__ __forceinline__ void st_dsmem<double>(double* local, uint32_t rank, double v) {
  uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(local)), r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(r), "d"(v) : "memory");
}
__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// asynchronous global -> shared copy of `bytes` (16, 8 or 4) with the tail past `valid` zeroed
__device__ __forceinline__ void cp_async_n(void* dst, const void* src, int bytes, int valid) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid) : "memory");
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

constexpr int kTrsvBS = 64;
template <typename T>
constexpr int trsv_ldc() { return sizeof(T) == 4 ? 68 : 66; }  // 16-byte aligned columns

template <typename T>
size_t trsv_smem_bytes(int64_t n, int C, int npf) {
  const int64_t nblk = (n + kTrsvBS - 1) / kTrsvBS;
  const int64_t nloc = (nblk + C - 1) / C;
  return sizeof(T) * (size_t)((2 + npf) * kTrsvBS * trsv_ldc<T>() + 8 * kTrsvBS + nloc * kTrsvBS);
}

template <typename T>
__global__ void __launch_bounds__(256, 1) k_trsv_upper(const T* __restrict__ R, int64_t ldr,
                                                        int64_t n, T* x, int64_t ldx, int64_t k,
                                                        int npf, int vec) {
  constexpr int BS = kTrsvBS, LDC = trsv_ldc<T>();
  constexpr int VE = 16 / (int)sizeof(T);  // elements per 16-byte copy
  extern __shared__ __align__(16) unsigned char trsv_raw[];
  T* Rd = reinterpret_cast<T*>(trsv_raw);  // [BS columns][LDC] diagonal tile of the next own block
  T* Ro = Rd + BS * LDC;                    // its tile right of the diagonal
  T* tiles = Ro + BS * LDC;                 // [npf][BS][LDC] tiles of the bulk updates
  T* rinv = tiles + (size_t)npf * BS * LDC; // [BS]
  T* xs = rinv + BS;                        // [3][BS] x_p in buffer p mod 3
  T* red = xs + 3 * BS;                     // [4][BS]
  T* xb = red + 4 * BS;                     // [nloc][BS] own blocks: b, then x
  const int C = gridDim.x, c = blockIdx.x, tid = threadIdx.x;
  const int64_t nblk = (n + BS - 1) / BS;
  const int r64 = tid & (BS - 1), q4 = tid >> 6;  // row of a tile, quarter of its columns

  // column-major tile of R at (i0, k0) into t; zero outside R
  auto tile_async = [&](T* t, int64_t i0, int64_t k0) {
    if (vec) {
      for (int e = tid; e < BS * BS / VE; e += blockDim.x) {
        const int rv = (e % (BS / VE)) * VE, cc = e / (BS / VE);
        const int64_t gi = i0 + rv, gc = k0 + cc, rows = n - gi;
        const int valid = (gc < n && rows > 0) ? (int)(sizeof(T) * (rows < VE ? rows : VE)) : 0;
        cp_async_n(t + cc * LDC + rv, valid ? (const void*)(R + gi + gc * ldr) : (const void*)R, 16, valid);
      }
    } else {
      for (int e = tid; e < BS * BS; e += blockDim.x) {
        const int r = e & (BS - 1), cc = e >> 6;
        const int64_t gi = i0 + r, gc = k0 + cc;
        const int valid = (gc < n && gi < n) ? (int)sizeof(T) : 0;
        cp_async_n(t + cc * LDC + r, valid ? (const void*)(R + gi + gc * ldr) : (const void*)R,
                   (int)sizeof(T), valid);
      }
    }
  };
  auto issue_diag = [&](int64_t p) {
    tile_async(Rd, p * BS, p * BS);
    tile_async(Ro, p * BS, p * BS + BS);
  };
  auto fix_diag = [&](int64_t p) {  // identity on the padded diagonal, reciprocals
    if (tid < BS) {
      if (p * BS + tid >= n) Rd[tid * LDC + tid] = T(1);
      rinv[tid] = T(1) / Rd[tid * LDC + tid];
    }
  };
  auto issue_bulk = [&](int64_t q) {  // R[i, q] for the first npf own blocks i < q - 1
    int u = 0;
    for (int64_t i = c; i < q - 1 && u < npf; i += C, ++u) tile_async(tiles + (size_t)u * BS * LDC, i * BS, q * BS);
  };

  for (int64_t col = 0; col < k; ++col) {
    T* xc = x + col * ldx;
    for (int64_t l = 0, p = c; p < nblk; ++l, p += C)
      if (tid < BS) xb[l * BS + tid] = (p * BS + tid < n) ? xc[p * BS + tid] : T(0);
    int64_t mine = -1;  // highest own block
    for (int64_t p = c; p < nblk; p += C) mine = p;
    if (mine >= 0) issue_diag(mine);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    if (mine >= 0) fix_diag(mine);
    int64_t pend = -1;  // own diagonal block whose tiles are in flight
    __syncthreads();

    for (int64_t p = nblk - 1; p >= 0; --p) {
      const bool own = (p % C) == c;
      const T* xnext = xs + ((p + 1) % 3) * BS;  // x_{p+1}
      if (own) {
        T* bp = xb + (p / C) * BS;
        if (p + 1 < nblk) {
          T s = T(0);
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) s += Ro[(q4 * 16 + cc) * LDC + r64] * xnext[q4 * 16 + cc];
          red[q4 * BS + r64] = s;
          __syncthreads();
          if (tid < BS) bp[tid] -= ((red[tid] + red[BS + tid]) + (red[2 * BS + tid] + red[3 * BS + tid]));
          __syncthreads();
        }
        if (tid < 32) {
          const int lane = tid;
          T b0 = bp[lane], b1 = bp[lane + 32];  // rows lane and lane + 32
#pragma unroll
          for (int sb = 7; sb >= 0; --sb) {
            const int base = sb * 8;
            T v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = __shfl_sync(0xffffffffu, sb >= 4 ? b1 : b0, (base + q) & 31);
#pragma unroll
            for (int q = 7; q >= 0; --q) {
              v[q] *= rinv[base + q];
#pragma unroll
              for (int qq = 0; qq < q; ++qq) v[qq] -= Rd[(base + q) * LDC + base + qq] * v[q];
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              if (sb >= 4) {
                if (lane == ((base + q) & 31)) b1 = v[q];
              } else if (lane == base + q) {
                b0 = v[q];
              }
            }
            T a0 = T(0), a1 = T(0);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              a0 += Rd[(base + q) * LDC + lane] * v[q];
              a1 += Rd[(base + q) * LDC + lane + 32] * v[q];
            }
            if (lane < base) b0 -= a0;
            if (lane + 32 < base) b1 -= a1;
          }
          bp[lane] = b0;
          bp[lane + 32] = b1;
        }
        __syncthreads();
        // x_p into buffer p mod 3 of every CTA of the cluster (this one included)
        T* dst = xs + (p % 3) * BS;
        for (int e = tid; e < BS * C; e += blockDim.x)
          st_dsmem<T>(dst + (e & (BS - 1)), (uint32_t)(e >> 6), bp[e & (BS - 1)]);
      }
      cluster_arrive_release();
      // this phase's bulk tiles (started one phase ago) and any diagonal prefetch have landed
      cp_async_wait_all();
      __syncthreads();
      if (pend >= 0) {
        fix_diag(pend);
        pend = -1;
      }
      if (p + 1 < nblk) {
        const int64_t k0 = (p + 1) * BS;
        int u = 0;
        for (int64_t l = 0, i = c; i < p; ++l, i += C, ++u) {
          T s = T(0);
          if (u < npf) {
            const T* t = tiles + (size_t)u * BS * LDC;
#pragma unroll
            for (int cc = 0; cc < 16; ++cc) s += t[(q4 * 16 + cc) * LDC + r64] * xnext[q4 * 16 + cc];
          } else {
#pragma unroll 16
            for (int cc = 0; cc < 16; ++cc) {
              const int64_t gc = k0 + q4 * 16 + cc;
              if (gc < n) s += R[i * BS + r64 + gc * ldr] * xnext[q4 * 16 + cc];
            }
          }
          red[q4 * BS + r64] = s;
          __syncthreads();
          if (tid < BS) xb[l * BS + tid] -= ((red[tid] + red[BS + tid]) + (red[2 * BS + tid] + red[3 * BS + tid]));
          __syncthreads();
        }
      }
      // refill: the next phase's bulk tiles, the next own diagonal block
      if (p >= 1) issue_bulk(p);
      if (own && p - C >= 0) {
        issue_diag(p - C);
        pend = p - C;
      }
      cp_async_commit();
      cluster_wait_acquire();
    }
    cp_async_wait_all();
    for (int64_t l = 0, p = c; p < nblk; ++l, p += C)
      if (tid < BS && p * BS + tid < n) xc[p * BS + tid] = xb[l * BS + tid];
    // no CTA may overwrite its blocks or buffers for the next column while a peer could
    // still write into them or read them
    cluster_arrive_release();
    cluster_wait_acquire();
  }
}

template <typename T>
bool trsv_cluster_fits(int C, size_t smem) {
  const void* fn = (const void*)k_trsv_upper<T>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      (C > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return nc >= 1;
}

template <typename T>
cudaError_t launch_trsv_upper(const T* R, int64_t ldr, int64_t n, T* x, int64_t ldx, int64_t k,
                              cudaStream_t st) {
  if (n <= 0 || k <= 0) return cudaSuccess;
  constexpr size_t kSmemMax = 227 * 1024;
  const int64_t nblk = (n + kTrsvBS - 1) / kTrsvBS;
  const size_t tile = sizeof(T) * kTrsvBS * trsv_ldc<T>();
  int C = 0, npf = 0;
  size_t smem = 0;
  for (int Ct : {16, 8}) {
    const int Cc = (int)std::min<int64_t>(Ct, nblk);
    const size_t base = trsv_smem_bytes<T>(n, Cc, 0);
    if (base > kSmemMax) continue;
    const int64_t below = (nblk + Cc - 1) / Cc;  // own blocks of a CTA, the upper bound of a phase's bulk
    const int np = (int)std::min<int64_t>(std::min<int64_t>(8, below), (int64_t)((kSmemMax - base) / tile));
    const size_t sm = trsv_smem_bytes<T>(n, Cc, np);
    if (trsv_cluster_fits<T>(Cc, sm)) {
      C = Cc;
      npf = np;
      smem = sm;
      break;
    }
  }
  if (C == 0) return cudaErrorInvalidValue;
  const int vec = ((reinterpret_cast<uintptr_t>(R) & 15) == 0 && (ldr * (int64_t)sizeof(T)) % 16 == 0) ? 1 : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_trsv_upper<T>, R, ldr, n, x, ldx, k, npf, vec);
}

// Least squares for tall A (reading: A = Q_1 R, so R x = (Q_1^T Q_1)^{-1} Q_1^T y with
// Q_1^T Q_1 = I - Q_2^T Q_2 by the orthonormality of the coded Q).  One cooperative kernel,
// FP64 vectors: z = Q_1^T y, then conjugate gradients on (I - Q_2^T Q_2) w = z.  The matrix
// is SPD with condition number <= 1 + ||G~||^2 (Q_1^T (I + G_v^T G_v) Q_1 = I), a property
// of the code, so a few dozen iterations reach FP64 accuracy.  w goes to x (n entries), the
// back substitution with R follows.  Work vectors: ws[6 n + c + 2 G] doubles.
template <typename T>
__global__ void __launch_bounds__(256) k_ls_cg(const T* __restrict__ Q, int64_t ldq, int64_t m,
                                                int64_t m_pad, int64_t c, int64_t n,
                                                const T* __restrict__ y, const T* __restrict__ u,
                                                T* __restrict__ x, double* ws, int maxit,
                                                unsigned* bar, int* status) {
  const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int64_t gw = (int64_t)g * 8 + warp, nw = (int64_t)G * 8;  // global warp index
  double* z = ws;
  double* w = z + n;
  double* r = w + n;
  double* p = r + n;
  double* sp = p + n;
  double* tv = sp + n + n;  // c entries
  double* part = tv + c;    // [2][G]
  unsigned target = 0;
  __shared__ double red[8];
  __shared__ double tpart[8][33];
  const T* Q2 = Q + m_pad;
  auto block_sum = [&](double v) -> double {  // sum over the CTA, result in every thread
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[k];
    return t;
  };
  auto grid_sum = [&](double v, int slot, int site, double* out) -> bool {
    const double s = block_sum(v);
    if (tid == 0) part[slot * G + g] = s;
    if (!grid_sync(bar, G, target, status, site)) return false;
    double t = 0.0;
    for (int k = 0; k < G; ++k) t += __ldcg(part + slot * G + k);
    *out = t;
    return true;
  };
  // z = Q_1^T y (warp per column), or z = u when the right-hand side is given; w = 0, r = p = z
  double zz_loc = 0.0;
  for (int64_t j = gw; j < n; j += nw) {
    double acc = 0.0;
    if (u) {
      acc = (double)u[j];
    } else {
      const T* qj = Q + j * ldq;
      for (int64_t i = lane; i < m; i += 32) acc += (double)qj[i] * (double)y[i];
      acc = warp_sum(acc);
    }
    if (lane == 0) {
      z[j] = acc; w[j] = 0.0; r[j] = acc; p[j] = acc;
      zz_loc += acc * acc;
    }
  }
  double rr;
  if (!grid_sum(lane == 0 ? zz_loc : 0.0, 0, 30, &rr)) return;
  const double stop = rr * 1e-30;  // |r| <= 1e-15 |z|
  int slot = 1;
  for (int it = 0; it < maxit && c > 0 && rr > stop; ++it) {
    // t = Q_2 p: tiles of 32 rows per CTA, lanes on rows (coalesced), the 8 warps on
    // interleaved columns, partial sums combined in a fixed order
    for (int64_t i0 = (int64_t)g * 32; i0 < c; i0 += (int64_t)G * 32) {
      const int64_t i = i0 + lane;
      double acc = 0.0;
      if (i < c)
        for (int64_t j = warp; j < n; j += 8) acc += (double)Q2[i + j * ldq] * __ldcg(p + j);
      tpart[warp][lane] = acc;
      __syncthreads();
      if (warp == 0 && i < c) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += tpart[k][lane];
        tv[i] = t;
      }
      __syncthreads();
    }
    if (!grid_sync(bar, G, target, status, 31)) return;
    // sp = p - Q_2^T t (warp per column), partial p . sp
    double psp_loc = 0.0;
    for (int64_t j = gw; j < n; j += nw) {
      const T* qj = Q2 + j * ldq;
      double acc = 0.0;
      for (int64_t i = lane; i < c; i += 32) acc += (double)qj[i] * __ldcg(tv + i);
      acc = warp_sum(acc);
      if (lane == 0) {
        const double pj = __ldcg(p + j);
        const double v = pj - acc;
        sp[j] = v;
        psp_loc += pj * v;
      }
    }
    double psp;
    if (!grid_sum(lane == 0 ? psp_loc : 0.0, slot, 32, &psp)) return;
    slot ^= 1;
    const double alpha = rr / psp;
    double rr_loc = 0.0;
    for (int64_t j = (int64_t)g * blockDim.x + tid; j < n; j += (int64_t)G * blockDim.x) {
      w[j] += alpha * __ldcg(p + j);
      const double rj = __ldcg(r + j) - alpha * __ldcg(sp + j);
      r[j] = rj;
      rr_loc += rj * rj;
    }
    double rr_new;
    if (!grid_sum(rr_loc, slot, 33, &rr_new)) return;
    slot ^= 1;
    const double beta = rr_new / rr;
    rr = rr_new;
    for (int64_t j = (int64_t)g * blockDim.x + tid; j < n; j += (int64_t)G * blockDim.x)
      p[j] = __ldcg(r + j) + beta * __ldcg(p + j);
    if (!grid_sync(bar, G, target, status, 34)) return;
  }
  for (int64_t j = (int64_t)g * blockDim.x + tid; j < n; j += (int64_t)G * blockDim.x)
    x[j] = (T)(c > 0 ? __ldcg(w + j) : __ldcg(z + j));
}

template <typename T>
cudaError_t launch_ls_cg(const T* Q, int64_t ldq, int64_t m, int64_t m_pad, int64_t c, int64_t n,
                         const T* y, T* x, double* ws, unsigned* bar, int* status, int num_sms,
                         cudaStream_t st, const T* u) {
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  // enough CTAs to spread the two products with Q_2 (c x n) per iteration, few enough that a
  // grid barrier stays near a microsecond
  int64_t want = std::max<int64_t>((c + 31) / 32, (n + 7) / 8);
  int G = (int)std::min<int64_t>(want, 32);
  if (G > num_sms) G = num_sms;
  if (G < 1) G = 1;
  int maxit = 200;
  void* args[] = {(void*)&Q, &ldq, &m, &m_pad, &c, &n, (void*)&y, (void*)&u, &x, &ws, &maxit,
                  &bar, &status};
  return cudaLaunchCooperativeKernel((const void*)k_ls_cg<T>, dim3(G), dim3(256), args, 0, st);
}

// ===================================================================== instantiations
// ===================================================================== batches
// Each batched kernel walks a flat list of virtual blocks; block v belongs to the instance i
// with off[i] <= v < off[i+1] and plays block `v - off[i]` of that instance's own grid.
__device__ __forceinline__ int find_instance(const int64_t* __restrict__ off, int count, int64_t v) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

int64_t batch_encode_blocks(const Geo& g, bool horizontal) {
  if (horizontal && (!g.protect_r || g.f == 0)) return 0;
  return ((g.mb + 31) / 32) * ((g.nb + 7) / 8) * (horizontal ? (g.p_r + g.f) : g.p_c);
}
int64_t batch_post_orth_blocks(const Geo& g) {
  if (g.f == 0) return 0;
  return ((g.mb + 31) / 32) * ((g.n + 7) / 8);
}
int64_t batch_decode_blocks(const Geo& g, const DecodePlan& p) {
  const int64_t h = p.kind == 0 ? g.mb : g.nb;
  return ((h + 31) / 32) * ((g.nb + 7) / 8);
}

// Batched encode: grid.y strides over the instances, grid.x blocks over one instance's blocks
// (no search of a flat block index, 32-bit block coordinates).
constexpr int kBEncX = 32;

template <typename T, int F>
__global__ void __launch_bounds__(256, 4) k_b_encode_vertical(const BatchInst<T>* __restrict__ inst,
                                                            int count, const T* __restrict__ Gt) {
  for (int i = blockIdx.y; i < count; i += gridDim.y) {
    const BatchInst<T>& I = inst[i];
    const int nbx = (int)((I.g.mb + 31) / 32), nby = (int)((I.g.nb + 7) / 8);
    const int total = nbx * nby * I.g.p_c;
    for (int v = blockIdx.x; v < total; v += gridDim.x) {
      const int bx = v % nbx, rest = v / nbx;
      encode_vertical_f<T, F>(I.g, I.A, I.lda, Gt, I.Q, bx, rest % nby, rest / nby);
    }
  }
}

template <typename T, int F>
__global__ void __launch_bounds__(256, 4) k_b_encode_horizontal(const BatchInst<T>* __restrict__ inst,
                                                              int count, const T* __restrict__ Gh) {
  for (int i = blockIdx.y; i < count; i += gridDim.y) {
    const BatchInst<T>& I = inst[i];
    if (!I.g.protect_r || I.g.f == 0) continue;
    const int nbx = (int)((I.g.mb + 31) / 32), nby = (int)((I.g.nb + 7) / 8);
    const int total = nbx * nby * (I.g.p_r + I.g.f);
    for (int v = blockIdx.x; v < total; v += gridDim.x) {
      const int bx = v % nbx, rest = v / nbx;
      encode_horizontal_f<T, F>(I.g, Gh, I.Q, bx, rest % nby, rest / nby);
    }
  }
}

template <typename T, int F>
cudaError_t launch_b_encode_f(const BatchInst<T>* inst, int count, int64_t total_v, int64_t total_h,
                              const T* Gt_t, const T* Gh_t, cudaStream_t st) {
  const dim3 blk(32, 8);
  const dim3 grd(kBEncX, (unsigned)std::min(count, 65535));
  if (total_v > 0 && count > 0) {
    k_b_encode_vertical<T, F><<<grd, blk, 0, st>>>(inst, count, Gt_t);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (total_h > 0 && count > 0) {
    k_b_encode_horizontal<T, F><<<grd, blk, 0, st>>>(inst, count, Gh_t);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

// f: the checksum count shared by every instance of the batch
template <typename T>
cudaError_t launch_b_encode(const BatchInst<T>* inst, int count, const int64_t* /*off_v*/,
                            int64_t total_v, const int64_t* /*off_h*/, int64_t total_h,
                            const T* Gt_t, const T* Gh_t, int f, cudaStream_t st) {
  switch (f_bucket(f)) {
    case 0: return launch_b_encode_f<T, 0>(inst, count, total_v, total_h, Gt_t, Gh_t, st);
    case 1: return launch_b_encode_f<T, 1>(inst, count, total_v, total_h, Gt_t, Gh_t, st);
    case 2: return launch_b_encode_f<T, 2>(inst, count, total_v, total_h, Gt_t, Gh_t, st);
    case 3: return launch_b_encode_f<T, 3>(inst, count, total_v, total_h, Gt_t, Gh_t, st);
    case 4: return launch_b_encode_f<T, 4>(inst, count, total_v, total_h, Gt_t, Gh_t, st);
    default: return launch_b_encode_f<T, -1>(inst, count, total_v, total_h, Gt_t, Gh_t, st);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_b_poison(const BatchInst<T>* __restrict__ inst,
                                                   const BatchTile* __restrict__ tiles) {
  const BatchTile t = tiles[blockIdx.y];
  const Geo& g = inst[t.inst].g;
  T* X = t.isR ? inst[t.inst].R : inst[t.inst].Q;
  const int64_t ld = t.isR ? g.ldr : g.ldq;
  const int64_t th = t.isR ? g.nb : g.mb, tw = g.nb;
  const int64_t total = th * tw;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx % th, s = idx / th;
    X[(int64_t)t.i * th + r + ((int64_t)t.j * tw + s) * ld] = nan_value<T>();
  }
}

template <typename T>
cudaError_t launch_b_poison(const BatchInst<T>* inst, const BatchTile* tiles, int count,
                            int64_t max_elems, int num_sms, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  for (int base = 0; base < count; base += 65535) {
    const int n = std::min(count - base, 65535);
    const unsigned bx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(64, (max_elems + 255) / 256));
    k_b_poison<T><<<dim3(bx, (unsigned)n), 256, 0, st>>>(inst, tiles + base);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  (void)num_sms;
  return cudaSuccess;
}

template <typename T>
__global__ void __launch_bounds__(256) k_b_decode(const BatchInst<T>* __restrict__ inst,
                                                   const BatchPlan* __restrict__ plans, int nplans,
                                                   const int64_t* __restrict__ off,
                                                   const double* __restrict__ Gt,
                                                   const double* __restrict__ Gh) {
  const int64_t total = off[nplans];
  for (int64_t v = blockIdx.x; v < total; v += gridDim.x) {
    __syncthreads();  // the previous block's readers of the shared tableau are done
    const int k = find_instance(off, nplans, v);
    const BatchPlan& bp = plans[k];
    const BatchInst<T>& I = inst[bp.inst];
    const int64_t h = bp.p.kind == 0 ? I.g.mb : I.g.nb;
    const int64_t nbx = (h + 31) / 32;
    const int64_t loc = v - off[k];
    decode_body<T, false>(I.g, bp.p, Gt, Gh, I.Q, I.R, I.status, (int)(loc % nbx),
                          (int)(loc / nbx), 1);
  }
}

template <typename T>
cudaError_t launch_b_decode(const BatchInst<T>* inst, const BatchPlan* plans, int nplans,
                            const int64_t* off, int64_t total, const double* Gt, const double* Gh,
                            int num_sms, cudaStream_t st) {
  if (nplans == 0 || total == 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>(total, (int64_t)num_sms * 8);
  k_b_decode<T><<<grid, dim3(32, 8), 0, st>>>(inst, plans, nplans, off, Gt, Gh);
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(256) k_b_post_orth(const BatchInst<T>* __restrict__ inst,
                                                      int count, const int64_t* __restrict__ off,
                                                      const T* __restrict__ Gt) {
  const int64_t total = off[count];
  for (int64_t v = blockIdx.x; v < total; v += gridDim.x) {
    const int i = find_instance(off, count, v);
    const BatchInst<T>& I = inst[i];
    const int64_t nbx = (I.g.mb + 31) / 32;
    const int64_t loc = v - off[i];
    post_orth_f<T, -1>(I.g, Gt, I.Q, I.g.ldq, I.g.m_pad, I.g.n, I.Q, I.g.ldq, (int)(loc % nbx),
                       (int)(loc / nbx));
  }
}

template <typename T>
cudaError_t launch_b_post_orth(const BatchInst<T>* inst, int count, const int64_t* off,
                               int64_t total, const T* Gt_t, int num_sms, cudaStream_t st) {
  if (total == 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>(total, (int64_t)num_sms * 16);
  k_b_post_orth<T><<<grid, dim3(32, 8), 0, st>>>(inst, count, off, Gt_t);
  return cudaGetLastError();
}

// Self-test of the bounds-checked build: a write to element idx of a four-element array,
// guarded by its index check (site 199); with idx >= 4 the check records CQR_EBOUNDS and the
// thread returns without the write.  Launched only by the bounds-checked build.
static __device__ float g_selftest[4];
__global__ void k_bounds_selftest(int idx) {
  CQR_CHECK(idx >= 0 && idx < 4, 199);
  g_selftest[idx] = 1.f;
}

cudaError_t launch_bounds_selftest(int idx, cudaStream_t st) {
  k_bounds_selftest<<<1, 1, 0, st>>>(idx);
  return cudaGetLastError();
}

cudaError_t bounds_take_kernels(int* code, int* site) { return bounds_take_here(code, site); }

#define CQR_INSTANTIATE(T)                                                                        \
  template cudaError_t launch_generator<T>(int, int, int, uint64_t, int, double*, double*, T*,   \
                                           T*, cudaStream_t);                                     \
  template cudaError_t launch_encode<T>(const Geo&, const T*, int64_t, const T*, const T*, T*,   \
                                        int*, cudaStream_t);                                      \
  template cudaError_t launch_gemm_tn_splitk<T>(const T*, int64_t, const T*, int64_t, int64_t,   \
                                                int, int64_t, int, T*, cudaStream_t);             \
  template cudaError_t launch_splitk_reduce<T>(const T*, int, int, int64_t, T*, int64_t, T*,     \
                                               cudaStream_t, int);                                \
  template cudaError_t launch_gemm_nn_sub<T>(const T*, int64_t, const T*, int64_t, T*, int64_t,  \
                                             int64_t, int, int64_t, cudaStream_t);                \
  template cudaError_t launch_poison<T>(const Geo&, const int*, int, T*, T*, cudaStream_t);      \
  template cudaError_t launch_decode<T>(const Geo&, const DecodePlan*, int, int, const double*,  \
                                        const double*, T*, T*, int*, cudaStream_t);               \
  template cudaError_t launch_post_orth<T>(const Geo&, const T*, const T*, int64_t, int64_t,     \
                                           int64_t, T*, int64_t, cudaStream_t);                   \
  template cudaError_t launch_post_orth_projected<T>(const Geo&, const double*, const T*,        \
                                                     double*, T*, const T*, int64_t, int64_t, T*, \
                                                     int64_t, cudaStream_t);                      \
  template cudaError_t launch_gemv_t<T>(const T*, int64_t, int64_t, int64_t, const T*, int64_t,  \
                                        int64_t, T*, int64_t, cudaStream_t);                      \
  template cudaError_t launch_trsv_upper<T>(const T*, int64_t, int64_t, T*, int64_t, int64_t,    \
                                            cudaStream_t);                                         \
  template cudaError_t launch_ls_cg<T>(const T*, int64_t, int64_t, int64_t, int64_t, int64_t,     \
                                       const T*, T*, double*, unsigned*, int*, int, cudaStream_t,  \
                                       const T*);

CQR_INSTANTIATE(float)
template cudaError_t launch_b_encode<float>(const BatchInst<float>*, int, const int64_t*, int64_t,
                                            const int64_t*, int64_t, const float*, const float*,
                                            int, cudaStream_t);
template cudaError_t launch_b_poison<float>(const BatchInst<float>*, const BatchTile*, int, int64_t,
                                            int, cudaStream_t);
template cudaError_t launch_b_decode<float>(const BatchInst<float>*, const BatchPlan*, int,
                                            const int64_t*, int64_t, const double*, const double*,
                                            int, cudaStream_t);
template cudaError_t launch_b_post_orth<float>(const BatchInst<float>*, int, const int64_t*,
                                               int64_t, const float*, int, cudaStream_t);
CQR_INSTANTIATE(double)

}  // namespace cqr
