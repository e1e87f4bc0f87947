// Instantiates the order-2 symmetric MTTKRP kernels.
#include "mttkrp.cuh"

namespace symgpu {
template <>
sym_status launch_mttkrp_order<2>(const sym_tensor_s* X, const void* B, bool bf16, int R, int64_t ldb, float* M,
                                  int64_t ldm, const sym_mttkrp_cfg& cfg, cudaStream_t s) {
    return launch_mttkrp_impl<2>(X, B, bf16, R, ldb, M, ldm, cfg, s);
}
}  // namespace symgpu
