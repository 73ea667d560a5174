// Packed-pair propagate kernels for 6, 7 and 8 atoms per lane.
#include "propagate_x2_impl.cuh"

namespace pamd {

cudaError_t propagate_x2_b678(int B, const PropParams* p, int warps, int grid, size_t smem,
                              cudaStream_t s, int* blocks_per_sm) {
    switch (B) {
        case 6: return propagate_x2_launch<6>(p, warps, grid, smem, s, blocks_per_sm);
        case 7: return propagate_x2_launch<7>(p, warps, grid, smem, s, blocks_per_sm);
        case 8: return propagate_x2_launch<8>(p, warps, grid, smem, s, blocks_per_sm);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pamd
