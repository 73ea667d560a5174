// propagate_b12.cu -- propagate kernels for 1 and 2 atoms per lane.
#include "propagate_impl.cuh"

namespace pamd {
cudaError_t propagate_b1(const PropParams* p, bool chain, bool table, int warps, int grid,
                         size_t smem, cudaStream_t s, int* blocks_per_sm) {
    return propagate_dispatch_b<1>(p, chain, table, warps, grid, smem, s, blocks_per_sm);
}
cudaError_t propagate_b2(const PropParams* p, bool chain, bool table, int warps, int grid,
                         size_t smem, cudaStream_t s, int* blocks_per_sm) {
    return propagate_dispatch_b<2>(p, chain, table, warps, grid, smem, s, blocks_per_sm);
}
}  // namespace pamd
