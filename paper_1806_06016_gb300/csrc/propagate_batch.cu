// propagate_batch.cu -- one persistent launch for many molecules of uneven
// size (batched independent anneals).
//
// Each molecule m has its own population, topology table and launch shape
// (L_m lanes per replica, B_m atoms per lane, 3 <= B_m <= 7).  The host cuts
// every population into work items of one CTA's worth of replicas and sorts
// them by cost (N_m^2 per replica, largest first).  CTAs take items from a
// device counter (atomicAdd; no CTA ever waits on another) until the list is
// exhausted.  When a CTA moves to an item of another molecule it reloads that
// molecule's table into shared memory; items of one molecule are contiguous in
// the list, so that happens about once per molecule per CTA.
#include "propagate_impl.cuh"

namespace pamd {

namespace {

template <bool CHAIN>
__device__ __forceinline__ void advance_any(int B, const PropParams& p, const unsigned char* sm,
                                            const float4* prm, const unsigned long long* masks,
                                            float4* pos, float4* frc, long long k, int L, int g,
                                            int base, unsigned gmask) {
    switch (B) {
        case 3: advance_replica<3, CHAIN>(p, sm, prm, masks, pos, frc, k, L, g, base, gmask); break;
        case 4: advance_replica<4, CHAIN>(p, sm, prm, masks, pos, frc, k, L, g, base, gmask); break;
        case 5: advance_replica<5, CHAIN>(p, sm, prm, masks, pos, frc, k, L, g, base, gmask); break;
        case 6: advance_replica<6, CHAIN>(p, sm, prm, masks, pos, frc, k, L, g, base, gmask); break;
        case 7: advance_replica<7, CHAIN>(p, sm, prm, masks, pos, frc, k, L, g, base, gmask); break;
        default: break;
    }
}

__global__ void __launch_bounds__(kBatchThreads, 1) propagate_batch_kernel(const __grid_constant__ BatchParams bp) {
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
                if (lay.chain)
                    advance_any<true>(lay.per_lane, p, sm, prm, masks, pos, frc, k, L, g, base, gmask);
                else
                    advance_any<false>(lay.per_lane, p, sm, prm, masks, pos, frc, k, L, g, base, gmask);
            }
        }
    }
}

}  // namespace

cudaError_t launch_propagate_batch(const BatchParams& bp, int grid, size_t smem, cudaStream_t s) {
    static size_t configured = 0;
    if (smem > configured) {
        const cudaError_t e = cudaFuncSetAttribute(
            propagate_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    propagate_batch_kernel<<<grid, kBatchThreads, smem, s>>>(bp);
    return cudaGetLastError();
}

cudaError_t propagate_batch_occupancy(size_t smem, int* blocks_per_sm) {
    const cudaError_t e = cudaFuncSetAttribute(
        propagate_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, propagate_batch_kernel,
                                                         kBatchThreads, smem);
}

}  // namespace pamd
