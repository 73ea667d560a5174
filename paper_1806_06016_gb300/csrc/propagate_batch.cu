// propagate_batch.cu -- persistent launches for many molecules of uneven
// size (batched independent anneals).
//
// Each molecule m has its own population, topology table and launch shape
// (L_m lanes per replica, B_m atoms per lane, 3 <= B_m <= 7).  Molecules are
// grouped by B; each group is one launch of a kernel compiled for that B, so
// the register allocation fits the group instead of the largest shape.  The
// host cuts every population into work items of one CTA's worth of replicas
// and sorts a group's items by cost (N_m^2 per replica, largest first).  CTAs
// take items from the group's device counter (atomicAdd; no CTA ever waits on
// another) until the list is exhausted.  When a CTA moves to an item of
// another molecule it reloads that molecule's table into shared memory; items
// of one molecule are contiguous in the list, so that happens about once per
// molecule per CTA.
#include "propagate_impl.cuh"

namespace pamd {

namespace {

// blocks of kBatchThreads per SM the compiler is asked to fit: 128 registers
// for B = 3 (no spills there), otherwise what the shape needs
template <int B>
struct BatchCfg {
    static constexpr int MIN_BLOCKS = (B <= 3) ? 4 : 2;
};

template <int B>
__global__ void __launch_bounds__(kBatchThreads, BatchCfg<B>::MIN_BLOCKS)
    propagate_batch_kernel(const __grid_constant__ BatchParams bp) {
    extern __shared__ float4 smem4[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(smem4);
    __shared__ int s_item;
    __shared__ int s_mol;
    if (threadIdx.x == 0) s_mol = -1;
    const int lane = threadIdx.x & 31;
    for (;;) {
        __syncthreads();  // the previous item (and table) is no longer in use
        if (threadIdx.x == 0) s_item = atomicAdd(bp.queue, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= bp.n_items) break;
        const int4 w = bp.items[it];
        const PropParams& p = bp.mol[w.x];
        const TopoLayout& lay = p.lay;
        if (w.x != s_mol) {  // uniform across the block
            const float4* src = reinterpret_cast<const float4*>(p.topo);
            for (int i = threadIdx.x; i < lay.bytes / 16; i += blockDim.x) smem4[i] = src[i];
            __syncthreads();
            if (threadIdx.x == 0) s_mol = w.x;
        }
        const float4* prm = reinterpret_cast<const float4*>(sm + lay.off_params);
        const unsigned long long* masks =
            reinterpret_cast<const unsigned long long*>(sm + lay.off_masks);
        float4* slots = smem4 + lay.bytes / 16;
        const int L = lay.lanes;
        const int G = 32 / L;
        const int grp = lane / L;
        if (grp < G) {
            const int g = lane - grp * L;
            const int base = grp * L;
            const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << base);
            const int slot_local = (threadIdx.x >> 5) * G + grp;
            float4* pos = slots + slot_local * (2 * lay.nk + 1);
            float4* frc = pos + lay.nk;
            const long long k = (long long)w.y + slot_local;
            if (k < w.z) {
                if (lay.chain && lay.ptab)
                    advance_replica<B, true, true>(p, sm, prm, masks, pos, frc, k, L, g, base, gmask);
                else if (lay.chain)
                    advance_replica<B, true, false>(p, sm, prm, masks, pos, frc, k, L, g, base, gmask);
                else
                    advance_replica<B, false, false>(p, sm, prm, masks, pos, frc, k, L, g, base, gmask);
            }
        }
    }
}

template <int B>
cudaError_t launch_b(const BatchParams& bp, int grid, size_t smem, cudaStream_t s, int* blocks_per_sm) {
    const cudaError_t e = ensure_dyn_smem((const void*)propagate_batch_kernel<B>, smem);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, propagate_batch_kernel<B>,
                                                             kBatchThreads, smem);
    propagate_batch_kernel<B><<<grid, kBatchThreads, smem, s>>>(bp);
    return cudaGetLastError();
}

cudaError_t dispatch_b(int B, const BatchParams* bp, int grid, size_t smem, cudaStream_t s,
                       int* blocks_per_sm) {
    static const BatchParams empty{};
    const BatchParams& q = bp ? *bp : empty;
    switch (B) {
        case 3: return launch_b<3>(q, grid, smem, s, blocks_per_sm);
        case 4: return launch_b<4>(q, grid, smem, s, blocks_per_sm);
        case 5: return launch_b<5>(q, grid, smem, s, blocks_per_sm);
        case 6: return launch_b<6>(q, grid, smem, s, blocks_per_sm);
        case 7: return launch_b<7>(q, grid, smem, s, blocks_per_sm);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_propagate_batch(const BatchParams& bp, int B, int grid, size_t smem, cudaStream_t s) {
    return dispatch_b(B, &bp, grid, smem, s, nullptr);
}

cudaError_t propagate_batch_occupancy(int B, size_t smem, int* blocks_per_sm) {
    return dispatch_b(B, nullptr, 0, smem, nullptr, blocks_per_sm);
}

}  // namespace pamd
