// Packed-pair propagate kernels for 3, 4 and 5 atoms per lane, and the
// dispatcher over every instantiated count (6..8 live in propagate_x2_b678.cu).
#include "propagate_x2_impl.cuh"

namespace pamd {

cudaError_t propagate_x2_b678(int B, const PropParams* p, int warps, int grid, size_t smem,
                              cudaStream_t s, int* blocks_per_sm);

cudaError_t propagate_x2_dispatch(int B, const PropParams* p, int warps, int grid, size_t smem,
                                  cudaStream_t s, int* blocks_per_sm) {
    switch (B) {
        case 3: return propagate_x2_launch<3>(p, warps, grid, smem, s, blocks_per_sm);
        case 4: return propagate_x2_launch<4>(p, warps, grid, smem, s, blocks_per_sm);
        case 5: return propagate_x2_launch<5>(p, warps, grid, smem, s, blocks_per_sm);
        default: return propagate_x2_b678(B, p, warps, grid, smem, s, blocks_per_sm);
    }
}

}  // namespace pamd
