// propagate_b56.cu -- propagate kernels for 5 and 6 atoms per lane.
#include "propagate_impl.cuh"

namespace pamd {
cudaError_t propagate_b5(const PropParams* p, bool chain, bool table, int warps, int grid,
                         size_t smem, cudaStream_t s, int* blocks_per_sm) {
    return propagate_dispatch_b<5>(p, chain, table, warps, grid, smem, s, blocks_per_sm);
}
cudaError_t propagate_b6(const PropParams* p, bool chain, bool table, int warps, int grid,
                         size_t smem, cudaStream_t s, int* blocks_per_sm) {
    return propagate_dispatch_b<6>(p, chain, table, warps, grid, smem, s, blocks_per_sm);
}
}  // namespace pamd
