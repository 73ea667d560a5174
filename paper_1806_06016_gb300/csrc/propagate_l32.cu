// propagate_l32.cu -- propagate kernels for 32 lanes per replica.
#include "propagate_impl.cuh"

namespace pamd {
cudaError_t propagate_l32(const PropParams* p, int per_lane, int warps, int grid, size_t smem,
                         cudaStream_t s, int* blocks_per_sm) {
    return propagate_dispatch<32>(p, per_lane, warps, grid, smem, s, blocks_per_sm);
}
}  // namespace pamd
