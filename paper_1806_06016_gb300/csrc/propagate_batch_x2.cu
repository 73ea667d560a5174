// propagate_batch_x2.cu -- the batched persistent launch (many molecules of
// uneven size, see propagate_batch.cu) for molecules whose chain layout takes
// the packed FP32x2 pair arithmetic of propagate_x2_impl.cuh.
//
// Same work queue as the scalar batched kernel: the host cuts every
// population into work items of one CTA's worth of replicas, a group's items
// are sorted by cost, CTAs take items from the group's device counter
// (atomicAdd; no CTA ever waits on another).  When a CTA moves to an item of
// another molecule it reloads that molecule's topology table and rebuilds the
// packed kernel's per-atom tables (duplicated mixing parameters, and the
// half-kick and noise scales of the molecule's launch parameters) in shared
// memory; the replica slots follow them, as in the single-molecule kernel.
#include "propagate_x2_impl.cuh"

namespace pamd {

namespace {

template <int B>
__global__ void __launch_bounds__(kBatchThreads, X2Cfg<B>::MIN_BLOCKS)
    propagate_batch_x2_kernel(const __grid_constant__ BatchParams bp) {
    static_assert(kBatchThreads <= kPackedMaxThreads, "batched blocks must fit the packed kernel");
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
        const int tb = x2_topo_bytes(lay);
        const float4* prm = reinterpret_cast<const float4*>(sm + lay.off_params);
        float4* dprm = smem4 + tb / 16;
        float2* aux = reinterpret_cast<float2*>(dprm + lay.nk);
        if (w.x != s_mol) {  // uniform across the block
            const float4* src = reinterpret_cast<const float4*>(p.topo);
            for (int i = threadIdx.x; i < tb / 16; i += blockDim.x) smem4[i] = src[i];
            __syncthreads();
            for (int i = threadIdx.x; i < lay.nk; i += blockDim.x) {
                const float4 c = prm[i];
                dprm[i] = make_float4(c.x, c.x, c.y, c.y);
                aux[i] = make_float2(p.hdt * c.w, p.c2kT * sqrtf(c.w));
            }
            __syncthreads();
            if (threadIdx.x == 0) s_mol = w.x;
        }
        const unsigned long long* masks = reinterpret_cast<const unsigned long long*>(sm + lay.off_masks);
        float4* slots = dprm + lay.nk + (lay.nk + 1) / 2;
        const int L = lay.lanes;
        const int G = 32 / L;
        const int grp = lane / L;
        if (grp < G) {
            const int g = lane - grp * L;
            const int base = grp * L;
            const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << base);
            const int slot_local = (threadIdx.x >> 5) * G + grp;
            float4* posA = slots + slot_local * x2_slot_f4(lay);
            float4* posB = posA + lay.nk;
            float4* vel = posB + lay.nk;
            const long long k = (long long)w.y + slot_local;
            if (k < w.z) advance_replica_x2<B>(p, sm, prm, dprm, aux, masks, posA, posB, vel, k, L, g, base, gmask);
        }
    }
}

template <int B>
cudaError_t launch_b(const BatchParams& bp, int grid, size_t smem, cudaStream_t s, int* blocks_per_sm) {
    const cudaError_t e = ensure_dyn_smem((const void*)propagate_batch_x2_kernel<B>, smem);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, propagate_batch_x2_kernel<B>,
                                                             kBatchThreads, smem);
    propagate_batch_x2_kernel<B><<<grid, kBatchThreads, smem, s>>>(bp);
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

cudaError_t launch_propagate_batch_x2(const BatchParams& bp, int B, int grid, size_t smem, cudaStream_t s) {
    return dispatch_b(B, &bp, grid, smem, s, nullptr);
}

cudaError_t propagate_batch_x2_occupancy(int B, size_t smem, int* blocks_per_sm) {
    return dispatch_b(B, nullptr, 0, smem, nullptr, blocks_per_sm);
}

}  // namespace pamd
