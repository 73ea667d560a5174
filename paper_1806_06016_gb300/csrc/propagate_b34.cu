// propagate_b34.cu -- propagate kernels for 3 and 4 atoms per lane.
#include "propagate_impl.cuh"

namespace pamd {
cudaError_t propagate_b3(const PropParams* p, bool chain, bool table, int warps, int grid,
                         size_t smem, cudaStream_t s, int* blocks_per_sm) {
    return propagate_dispatch_b<3>(p, chain, table, warps, grid, smem, s, blocks_per_sm);
}
cudaError_t propagate_b4(const PropParams* p, bool chain, bool table, int warps, int grid,
                         size_t smem, cudaStream_t s, int* blocks_per_sm) {
    return propagate_dispatch_b<4>(p, chain, table, warps, grid, smem, s, blocks_per_sm);
}
}  // namespace pamd
