// propagate_b78.cu -- propagate kernels for 7 and 8 atoms per lane.
#include "propagate_impl.cuh"

namespace pamd {
cudaError_t propagate_b7(const PropParams* p, bool chain, bool table, int warps, int grid,
                         size_t smem, cudaStream_t s, int* blocks_per_sm) {
    return propagate_dispatch_b<7>(p, chain, table, warps, grid, smem, s, blocks_per_sm);
}
cudaError_t propagate_b8(const PropParams* p, bool chain, bool table, int warps, int grid,
                         size_t smem, cudaStream_t s, int* blocks_per_sm) {
    return propagate_dispatch_b<8>(p, chain, table, warps, grid, smem, s, blocks_per_sm);
}
}  // namespace pamd
