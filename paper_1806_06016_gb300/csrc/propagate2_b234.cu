// propagate2_b234.cu -- paired (two replicas per lane) propagate kernels for
// 2, 3 and 4 atoms per lane.
#include "propagate2_impl.cuh"

namespace pamd {
cudaError_t propagate2_b2(const PropParams* p, bool chain, int warps, int grid, size_t smem,
                          cudaStream_t s, int* blocks_per_sm) {
    return propagate2_dispatch_b<2>(p, chain, warps, grid, smem, s, blocks_per_sm);
}
cudaError_t propagate2_b3(const PropParams* p, bool chain, int warps, int grid, size_t smem,
                          cudaStream_t s, int* blocks_per_sm) {
    return propagate2_dispatch_b<3>(p, chain, warps, grid, smem, s, blocks_per_sm);
}
cudaError_t propagate2_b4(const PropParams* p, bool chain, int warps, int grid, size_t smem,
                          cudaStream_t s, int* blocks_per_sm) {
    return propagate2_dispatch_b<4>(p, chain, warps, grid, smem, s, blocks_per_sm);
}
}  // namespace pamd
