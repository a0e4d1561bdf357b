// cqr_tc_gemm.cu -- tensor-core trailing update (tcgen05 + TMA + TMEM), FP32 storage.
#include "cqr_tc_gemm.cuh"

namespace cqr {

struct TcGemm {
  int mode;
};

bool tc_available() { return false; }
size_t tc_panel_bytes(int64_t, int) { return 0; }
size_t tc_workspace_bytes(int64_t, int64_t, int) { return 0; }
TcGemm* tc_create(int, int64_t, int64_t, int64_t, float*, int64_t, void*, void*, int) { return nullptr; }
void tc_destroy(TcGemm* t) { delete t; }
int tc_launches_per_update(const TcGemm*) { return 0; }
cudaError_t tc_trailing_update(TcGemm*, int64_t, int, int64_t, int64_t, float*, int64_t, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace cqr
