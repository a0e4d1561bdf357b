// cqr_mds.cu -- E1: MDS statistics of a checksum generator (Section 4.2, Theorem prob_det and
// the empirical comparison after it): over every square submatrix S of an f x p_r matrix G,
// the least |det S| and the largest 2-norm condition number, per size k and overall.
//
// One thread per submatrix.  The k rows and k columns of submatrix `idx` are the idx-th
// k-subsets of {0..f-1} and {0..p_r-1} in lexicographic order (combinatorial number system,
// unranked with a binomial table).  |det S| from LU with partial pivoting; the singular
// values from one-sided Jacobi (Hestenes) on the columns, all in FP64.  Minima and maxima of
// non-negative doubles are reduced through atomicMin / atomicMax on their bit patterns,
// which order like the values, so the result does not depend on the schedule.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "coded_qr.h"

namespace cqr {

namespace {

constexpr int kMdsMaxF = 6;
constexpr int kMdsMaxP = 64;

__constant__ unsigned long long c_binom[kMdsMaxP + 1][kMdsMaxF + 1];

// the rank-th k-subset of {0..n-1} in lexicographic order
__device__ void unrank(unsigned long long rank, int n, int k, int* out) {
  int x = 0;
  for (int i = 0; i < k; ++i) {
    // smallest element x such that the subsets starting with x cover `rank`
    for (;; ++x) {
      const unsigned long long cnt = c_binom[n - x - 1][k - i - 1];
      if (rank < cnt) break;
      rank -= cnt;
    }
    out[i] = x++;
  }
}

__device__ double abs_det(double (*a)[kMdsMaxF], int k) {
  double det = 1.0;
  for (int c = 0; c < k; ++c) {
    int piv = c;
    for (int r = c + 1; r < k; ++r)
      if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
    if (a[piv][c] == 0.0) return 0.0;
    if (piv != c)
      for (int q = 0; q < k; ++q) { const double t = a[c][q]; a[c][q] = a[piv][q]; a[piv][q] = t; }
    det *= a[c][c];
    for (int r = c + 1; r < k; ++r) {
      const double l = a[r][c] / a[c][c];
      for (int q = c; q < k; ++q) a[r][q] -= l * a[c][q];
    }
  }
  return fabs(det);
}

// 2-norm condition number from the singular values of one-sided Jacobi rotations on the
// columns of a (k x k, row index first); +inf when sigma_min <= 2^-52 sigma_max.
__device__ double cond2(double (*a)[kMdsMaxF], int k) {
  for (int sweep = 0; sweep < 40; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < k - 1; ++p)
      for (int q = p + 1; q < k; ++q) {
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int r = 0; r < k; ++r) {
          alpha += a[r][p] * a[r][p];
          beta += a[r][q] * a[r][q];
          gamma += a[r][p] * a[r][q];
        }
        if (gamma == 0.0 || fabs(gamma) <= 1e-15 * sqrt(alpha * beta)) continue;
        rotated = true;
        const double zeta = (beta - alpha) / (2.0 * gamma);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        for (int r = 0; r < k; ++r) {
          const double x = a[r][p], y = a[r][q];
          a[r][p] = c * x - s * y;
          a[r][q] = s * x + c * y;
        }
      }
    if (!rotated) break;
  }
  double smax = 0.0, smin = INFINITY;
  for (int q = 0; q < k; ++q) {
    double n2 = 0.0;
    for (int r = 0; r < k; ++r) n2 += a[r][q] * a[r][q];
    const double sv = sqrt(n2);
    smax = fmax(smax, sv);
    smin = fmin(smin, sv);
  }
  // numerically singular (sigma_min <= eps sigma_max, eps = 2^-52): +inf
  return smin > 2.220446049250313e-16 * smax ? smax / smin : INFINITY;
}

__device__ __forceinline__ void atomic_min_pos(unsigned long long* p, double v) {
  atomicMin(p, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_max_pos(unsigned long long* p, double v) {
  atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

// res: [0 .. f] least |det| (0 = overall), [f+1 .. 2f+1] largest condition number
__global__ void __launch_bounds__(256) k_mds(const double* __restrict__ G, int f, int p,
                                             const unsigned long long* __restrict__ off,
                                             unsigned long long* res) {
  __shared__ unsigned long long s_res[2 * (kMdsMaxF + 1)];
  for (int i = threadIdx.x; i < 2 * (f + 1); i += blockDim.x)
    s_res[i] = i <= f ? 0x7FF0000000000000ull : 0ull;  // +inf for minima, +0 for maxima
  __syncthreads();
  const unsigned long long total = off[f];
  for (unsigned long long idx = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
       idx < total; idx += (unsigned long long)gridDim.x * blockDim.x) {
    int k = 1;
    while (idx >= off[k]) ++k;
    const unsigned long long loc = idx - off[k - 1];
    const unsigned long long ncol = c_binom[p][k];
    int rows[kMdsMaxF], cols[kMdsMaxF];
    unrank(loc / ncol, f, k, rows);
    unrank(loc % ncol, p, k, cols);
    double a[kMdsMaxF][kMdsMaxF];
    for (int r = 0; r < k; ++r)
      for (int q = 0; q < k; ++q) a[r][q] = G[rows[r] * p + cols[q]];
    double b[kMdsMaxF][kMdsMaxF];
    for (int r = 0; r < k; ++r)
      for (int q = 0; q < k; ++q) b[r][q] = a[r][q];
    const double det = abs_det(a, k);
    const double cn = cond2(b, k);
    atomic_min_pos(&s_res[k], det);
    atomic_max_pos(&s_res[f + 1 + k], cn);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * (f + 1); i += blockDim.x) {
    if (i == 0 || i == f + 1) continue;
    if (i <= f)
      atomicMin(&res[i], s_res[i]);
    else
      atomicMax(&res[i], s_res[i]);
  }
}

unsigned long long binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  unsigned long long r = 1;
  for (int i = 1; i <= k; ++i) r = r * (unsigned long long)(n - k + i) / (unsigned long long)i;
  return r;
}

}  // namespace

}  // namespace cqr

using namespace cqr;

extern "C" cqr_status coded_qr_mds_stats(const double* G, int32_t f, int32_t p_r, double* min_det,
                                         double* max_cond, int64_t* count, void* stream) {
  if (!G || !min_det || !max_cond || f < 1 || f > kMdsMaxF || p_r < f || p_r > kMdsMaxP)
    return CQR_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned long long tab[kMdsMaxP + 1][kMdsMaxF + 1];
  for (int n = 0; n <= kMdsMaxP; ++n)
    for (int k = 0; k <= kMdsMaxF; ++k) tab[n][k] = binom(n, k);
  unsigned long long off[kMdsMaxF + 1];
  off[0] = 0;
  for (int k = 1; k <= f; ++k) off[k] = off[k - 1] + binom(f, k) * binom(p_r, k);
  unsigned long long init[2 * (kMdsMaxF + 1)];
  for (int i = 0; i < 2 * (f + 1); ++i) init[i] = i <= f ? 0x7FF0000000000000ull : 0ull;
  void* mem = nullptr;
  const size_t gbytes = sizeof(double) * (size_t)f * p_r;
  const size_t bytes = 256 + gbytes + sizeof(off) + sizeof(init);
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return CQR_ENOMEM;
  }
  char* base = static_cast<char*>(mem);
  double* dG = reinterpret_cast<double*>(base);
  unsigned long long* doff = reinterpret_cast<unsigned long long*>(base + ((gbytes + 255) & ~(size_t)255));
  unsigned long long* dres = doff + (kMdsMaxF + 1);
  cqr_status s = CQR_OK;
  unsigned long long res[2 * (kMdsMaxF + 1)];
  if (cudaMemcpyToSymbolAsync(c_binom, tab, sizeof(tab), 0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dG, G, gbytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(doff, off, sizeof(off), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dres, init, sizeof(init), cudaMemcpyHostToDevice, st) != cudaSuccess) {
    s = CQR_ECUDA;
  }
  if (s == CQR_OK) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned long long total = off[f];
    const unsigned grid = (unsigned)std::min<unsigned long long>((total + 255) / 256, (unsigned long long)sms * 32);
    k_mds<<<grid, 256, 0, st>>>(dG, f, p_r, doff, dres);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(res, dres, sizeof(init), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      s = CQR_ECUDA;
  }
  cudaFree(mem);
  if (s != CQR_OK) {
    cudaGetLastError();
    return s;
  }
  double mn = INFINITY, mx = 0.0;
  for (int k = 1; k <= f; ++k) {
    double d, c;
    memcpy(&d, &res[k], 8);
    memcpy(&c, &res[f + 1 + k], 8);
    min_det[k] = d;
    max_cond[k] = c;
    mn = std::min(mn, d);
    mx = std::max(mx, c);
  }
  min_det[0] = mn;
  max_cond[0] = mx;
  if (count) *count = (int64_t)off[f];
  return CQR_OK;
}
