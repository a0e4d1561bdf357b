// cqr_adjoint.cu -- kernels of the reverse-mode (adjoint) pass through the coded QR and the
// least-squares solve.
//
// QR adjoint (the coded method's outputs Q = G_0 Q_1, R with G_0 A = Q R, Q^T Q = I): for a
// loss with gradients Qbar, Rbar,
//   M = R Rbar^T - Qbar^T Q,   Bbar = (Qbar + Q copyltu(M)) R^{-T},   Abar = G_0^T Bbar,
// copyltu(M) = tril(M) + tril(M, -1)^T.  This is the standard reverse rule of a thin QR with
// positive diagonal (e.g. Walter & Lehmann 2018, Seeger et al. 2017) applied to G_0 A,
// followed by the chain rule through the linear map A -> G_0 A.
// Least-squares adjoint (x = argmin |A x - y|, A of full column rank): with g = xbar,
//   z = (A^T A)^{-1} g,   r = y - A x,   Abar = r z^T - (A z) x^T,   ybar = A z,
// where A^T A = R^T (Q_1^T Q_1) R and Q_1^T Q_1 = I - Q_2^T Q_2 (coded factors), so
// z = R^{-1} (I - Q_2^T Q_2)^{-1} R^{-T} g.
//
// The building blocks here: a tiled FP32/FP64 GEMM with transposes, copyltu, and a
// triangular solve from the right, X op(R) = B, row blocks in shared memory.
#include <math.h>

#include <algorithm>

#include "cqr_device.cuh"
#include "cqr_kernels.cuh"

namespace cqr {

namespace {

constexpr int kGT = 64;  // GEMM tile (rows and columns of C)
constexpr int kGK = 16;  // GEMM K step

// C (M x N) = alpha op(A) op(B) + beta C; op(A) M x K, op(B) K x N; column-major operands.
// 256 threads; thread (tx, ty) owns rows ty + 16 a and columns tx + 16 b (a, b < 4) of the tile.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm(int ta, int tb, int64_t M, int64_t N, int64_t K,
                                              T alpha, const T* __restrict__ A, int64_t lda,
                                              const T* __restrict__ B, int64_t ldb, T beta,
                                              T* __restrict__ C, int64_t ldc) {
  __shared__ T As[kGK][kGT + 1];  // As[k][i] = op(A)[i0 + i][k0 + k]
  __shared__ T Bs[kGK][kGT + 1];  // Bs[k][j] = op(B)[k0 + k][j0 + j]
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t i0 = (int64_t)blockIdx.x * kGT, j0 = (int64_t)blockIdx.y * kGT;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int64_t k0 = 0; k0 < K; k0 += kGK) {
    for (int e = tid; e < kGT * kGK; e += 256) {
      // consecutive threads walk the contiguous index of the stored operand
      int i, k;
      if (!ta) { i = e % kGT; k = e / kGT; } else { k = e % kGK; i = e / kGK; }
      const int64_t gi = i0 + i, gk = k0 + k;
      T v = T(0);
      if (gi < M && gk < K) v = ta ? A[gk + gi * lda] : A[gi + gk * lda];
      As[k][i] = v;
      int j;
      if (!tb) { k = e % kGK; j = e / kGK; } else { j = e % kGT; k = e / kGT; }
      const int64_t gj = j0 + j, gk2 = k0 + k;
      T w = T(0);
      if (gj < N && gk2 < K) w = tb ? B[gj + gk2 * ldb] : B[gk2 + gj * ldb];
      Bs[k][j] = w;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kGK; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[k][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t gi = i0 + ty + 16 * a, gj = j0 + tx + 16 * b;
      if (gi < M && gj < N) {
        T* cp = C + gi + gj * ldc;
        *cp = alpha * acc[a][b] + (beta == T(0) ? T(0) : beta * *cp);
      }
    }
}

// S = copyltu(M): S[i][j] = M[i][j] for i >= j, M[j][i] for i < j (n x n, ld n for both).
template <typename T>
__global__ void k_copyltu(const T* __restrict__ Mm, int64_t n, T* __restrict__ S) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    S[e] = i >= j ? Mm[i + j * n] : Mm[j + i * n];
  }
}

// Y (rows x cols, strides rs / cs) += alpha X (same shape, strides xrs / xcs).
template <typename T>
__global__ void k_axpy2d(int64_t rows, int64_t cols, T alpha, const T* __restrict__ X, int64_t xrs,
                         int64_t xcs, T* __restrict__ Y, int64_t yrs, int64_t ycs, int overwrite) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    T* y = Y + i * yrs + j * ycs;
    const T v = alpha * X[i * xrs + j * xcs];
    *y = overwrite ? v : *y + v;
  }
}

// X op(R) = B in place (X overwrites B), R upper triangular n x n (ld ldr), B m x n with
// element (i, j) at B[i rs + j cs].  trans = 1: X R^T = B, columns solved from the last
// (X[:, j] = (B[:, j] - sum_{k>j} X[:, k] R[j, k]) / R[j, j]); trans = 0: X R = B, columns
// solved from the first (X[:, j] = (B[:, j] - sum_{k<j} X[:, k] R[k, j]) / R[j, j]).
// One CTA per block of rb <= 32 rows, held in shared memory [rb][n + 1]; right-looking: once
// column j is final, its contribution leaves every column still to be solved.  Thread t works
// on row t % 32 and the columns congruent to t / 32 modulo 8 (all lanes of a warp read the
// same coefficient of R).  Used for diagonal blocks and for a few right-hand sides.
template <typename T>
__global__ void __launch_bounds__(256) k_trsm_right(int trans, const T* __restrict__ R, int64_t ldr,
                                                    int n, T* __restrict__ B, int64_t rs,
                                                    int64_t cs, int64_t m, int rb) {
  extern __shared__ __align__(16) unsigned char trsm_raw[];
  T* X = reinterpret_cast<T*>(trsm_raw);  // [rb][n + 1]
  const int tid = threadIdx.x, ld = n + 1;
  const int64_t r0 = (int64_t)blockIdx.x * rb;
  const int nrow = (int)((m - r0) < rb ? (m - r0) : rb);
  for (int e = tid; e < nrow * n; e += 256) {
    const int j = e / nrow, r = e % nrow;
    X[r * ld + j] = B[(r0 + r) * rs + (int64_t)j * cs];
  }
  __syncthreads();
  const int r = tid & 31, grp = tid >> 5;
  for (int s = 0; s < n; ++s) {
    const int j = trans ? n - 1 - s : s;
    if (tid < nrow) X[tid * ld + j] /= R[j + (int64_t)j * ldr];
    __syncthreads();
    if (r < nrow) {
      const T xj = X[r * ld + j];
      if (trans) {
        for (int k = grp; k < j; k += 8) X[r * ld + k] -= xj * R[k + (int64_t)j * ldr];
      } else {
        for (int k = j + 1 + grp; k < n; k += 8) X[r * ld + k] -= xj * R[j + (int64_t)k * ldr];
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < nrow * n; e += 256) {
    const int j = e / nrow, r2 = e % nrow;
    B[(r0 + r2) * rs + (int64_t)j * cs] = X[r2 * ld + j];
  }
}

template <typename T>
cudaError_t trsm_unblocked(int trans, const T* R, int64_t ldr, int n, T* B, int64_t rs, int64_t cs,
                           int64_t m, cudaStream_t st) {
  const size_t cap = 200 * 1024;
  int rb = (int)std::min<int64_t>(32, (int64_t)(cap / ((size_t)(n + 1) * sizeof(T))));
  if (rb < 1) return cudaErrorInvalidValue;  // n too large for one row in shared memory
  const size_t smem = (size_t)rb * (n + 1) * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(k_trsm_right<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((m + rb - 1) / rb);
  k_trsm_right<T><<<grid, 256, smem, st>>>(trans, R, ldr, n, B, rs, cs, m, rb);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_gemm_general(int ta, int tb, int64_t M, int64_t N, int64_t K, T alpha,
                                const T* A, int64_t lda, const T* B, int64_t ldb, T beta, T* C,
                                int64_t ldc, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((M + kGT - 1) / kGT), (unsigned)((N + kGT - 1) / kGT));
  k_gemm<T><<<grid, 256, 0, st>>>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_copyltu(const T* Mm, int64_t n, T* S, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>(1024, (n * n + 255) / 256);
  k_copyltu<T><<<blocks, 256, 0, st>>>(Mm, n, S);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_axpy2d(int64_t rows, int64_t cols, T alpha, const T* X, int64_t xrs, int64_t xcs,
                          T* Y, int64_t yrs, int64_t ycs, bool overwrite, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>(2048, (rows * cols + 255) / 256);
  k_axpy2d<T><<<blocks, 256, 0, st>>>(rows, cols, alpha, X, xrs, xcs, Y, yrs, ycs, overwrite ? 1 : 0);
  return cudaGetLastError();
}

// Blocked for a column-major B (rs == 1) with many rows: diagonal blocks of kTB columns are
// solved by the row-block kernel, the rest of each step is one GEMM update
//   trans = 1 (blocks from the last):  B[:, K] -= X[:, J] R[K, J]^T  for the blocks K < J
//   trans = 0 (blocks from the first): B[:, K] -= X[:, J] R[J, K]    for the blocks K > J.
template <typename T>
cudaError_t launch_trsm_right(int trans, const T* R, int64_t ldr, int64_t n, T* B, int64_t rs,
                              int64_t cs, int64_t m, cudaStream_t st) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  constexpr int kTB = 64;
  // blocked when B is column-major (or a single contiguous row, cs == 1)
  const bool colmajor = (rs == 1) || (m == 1);
  if (!colmajor || n <= kTB) return trsm_unblocked<T>(trans, R, ldr, (int)n, B, rs, cs, m, st);
  const int64_t nblk = (n + kTB - 1) / kTB;
  for (int64_t s = 0; s < nblk; ++s) {
    const int64_t J = trans ? nblk - 1 - s : s;
    const int64_t j0 = J * kTB, jb = std::min<int64_t>(kTB, n - j0);
    cudaError_t e = trsm_unblocked<T>(trans, R + j0 + j0 * ldr, ldr, (int)jb, B + j0 * cs, 1, cs, m, st);
    if (e != cudaSuccess) return e;
    if (trans && j0 > 0) {
      e = launch_gemm_general<T>(0, 1, m, j0, jb, T(-1), B + j0 * cs, cs, R + j0 * ldr, ldr, T(1),
                                 B, cs, st);
    } else if (!trans && j0 + jb < n) {
      e = launch_gemm_general<T>(0, 0, m, n - j0 - jb, jb, T(-1), B + j0 * cs, cs,
                                 R + j0 + (j0 + jb) * ldr, ldr, T(1), B + (j0 + jb) * cs, cs, st);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

#define CQR_ADJ_INSTANTIATE(T)                                                                   \
  template cudaError_t launch_gemm_general<T>(int, int, int64_t, int64_t, int64_t, T, const T*,  \
                                              int64_t, const T*, int64_t, T, T*, int64_t,        \
                                              cudaStream_t);                                     \
  template cudaError_t launch_copyltu<T>(const T*, int64_t, T*, cudaStream_t);                   \
  template cudaError_t launch_axpy2d<T>(int64_t, int64_t, T, const T*, int64_t, int64_t, T*,     \
                                        int64_t, int64_t, bool, cudaStream_t);                   \
  template cudaError_t launch_trsm_right<T>(int, const T*, int64_t, int64_t, T*, int64_t,        \
                                            int64_t, int64_t, cudaStream_t);

CQR_ADJ_INSTANTIATE(float)
CQR_ADJ_INSTANTIATE(double)

}  // namespace cqr
