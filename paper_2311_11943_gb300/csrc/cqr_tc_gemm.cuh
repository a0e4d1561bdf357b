// cqr_tc_gemm.cuh -- tensor-core (tcgen05, sm_103a) trailing update of PBMGS for FP32 storage:
// TF32 or BF16 operands (one product, or hi/lo splits with three products), FP32 accumulation.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace cqr {

struct TcGemm;

bool tc_available();
size_t tc_panel_bytes(int64_t M, int b);
size_t tc_workspace_bytes(int mode, int64_t M, int64_t N, int64_t n, int b, int reorth_block);
TcGemm* tc_create(int mode, int64_t M, int64_t N, int64_t n, int64_t b, float* Q, int64_t ldq,
                  void* ws, int num_sms, int reorth_block, cudaStream_t st);
void tc_destroy(TcGemm* t);
void tc_set_status(TcGemm* t, int* status);
// Launches on stream st (and only there) use programmatic dependent launch: each kernel waits
// for its predecessor's completion before touching data, then lets its successor launch.
void tc_set_pdl_stream(TcGemm* t, cudaStream_t st);
// The trailing update of one panel, in four stream-ordered launches:
//   split the panel into operand planes; Rbar partials = Qbar^T Q[:, j0:j0+w] (split-K);
//   reduce into R[kb:kb+bk, j0:j0+w] and GEMM2's operand; Q[:, j0:j0+w] -= Qbar Rbar.
// buf (0/1) selects the panel's operand planes (panels of alternating parity use different
// buffers), ctx (0/1) the partials and Rbar planes of an update, so that two updates of
// disjoint column ranges can run concurrently on two streams; max_ctas (0: all SMs) caps the
// CTAs of a GEMM launch and its split-K factor (the same cap for rbar and reduce).
cudaError_t tc_split_panel(TcGemm* t, int64_t kb, int bk, bool finished, int buf, cudaStream_t st);
cudaError_t tc_gemm_rbar(TcGemm* t, int bk, int64_t j0, int64_t w, int buf, int ctx, int max_ctas,
                         cudaStream_t st);
cudaError_t tc_reduce(TcGemm* t, int64_t kb, int bk, int64_t j0, int64_t w, float* R, int64_t ldr,
                      int ctx, int max_ctas, cudaStream_t st);
cudaError_t tc_gemm_update(TcGemm* t, int bk, int64_t j0, int64_t w, int buf, int ctx, int max_ctas,
                           cudaStream_t st);

// Block reorthogonalisation of panel columns kb .. kb+bk-1 against columns 0 .. kb-1:
// S = Q[:, 0:kb]^T Qbar, Qbar -= Q[:, 0:kb] S, R[0:kb, kb:kb+bk] += S (four launches, five
// when the second product is split over K); *launches receives the count.
bool tc_has_block_reorth(const TcGemm* t);
cudaError_t tc_block_reorth(TcGemm* t, int64_t kb, int bk, float* R, int64_t ldr, int buf,
                            cudaStream_t st, int* launches);
// Row-major planes of one rectangle of Q (rows r0 .. r0+nr-1, columns c0 .. c0+nc-1) rebuilt
// after a recovery changed it.
cudaError_t tc_refresh_rect(TcGemm* t, int64_t r0, int64_t nr, int64_t c0, int64_t nc, cudaStream_t st);

// General C -= op(A) B in 3xTF32 (op(A) = A^T for a_trans with A K x M, else A M x K; B K x N;
// all column-major).  planes: tc_gemm_sub_planes(a_trans, M, K) floats of scratch, 16-byte
// aligned.  cudaErrorInvalidValue, with nothing launched, when B is not 16-byte aligned or
// ldb is not a multiple of 4 (the tensor-map rules).
size_t tc_gemm_sub_planes(bool a_trans, int64_t M, int64_t K);
cudaError_t tc_gemm_sub3(bool a_trans, const float* A, int64_t lda, const float* B, int64_t ldb,
                         float* C, int64_t ldc, int64_t M, int64_t N, int64_t K, float* planes,
                         int num_sms, int* status, cudaStream_t st);

}  // namespace cqr
