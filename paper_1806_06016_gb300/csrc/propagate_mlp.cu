// propagate_mlp.cu -- BAOAB Langevin steps of a population whose forces and
// energies come from the MLP energy surrogate.
//
// The exact-force propagate kernel keeps each replica in shared memory for
// all theta steps; here every force evaluation is a batch of tensor-core
// GEMMs over the whole population, so the state stays in global memory and
// one step is five launches: this kernel (finish the previous step with its
// closing half kick, then B A O A of the next one and the features of the new
// positions) and the four GEMMs.  Inside a graph capture (pamd_anneal) the
// theta steps become one WHILE node whose body is those five launches and a
// one-thread counter kernel.  The update arithmetic and the Philox noise
// stream are those of the exact propagate kernel (same key, counter and
// purpose), so that the two force fields can be compared on identical noise.
#include <map>
#include <mutex>
#include <tuple>

#include "mlp_device.cuh"
#include "pamd_device.cuh"

namespace pamd {

namespace {

constexpr int kStepThreads = 256;
static_assert(PAMD_MAX_ATOMS <= kStepThreads, "one atom per thread in the update");
// Molecules with gamma_matrix(N) split each atom's force sum over up to this
// many threads (consecutive thirds of the row, added in order afterwards).
constexpr int kForceSplit = 3;

__host__ __device__ __forceinline__ int force_split(int N) {
    if (!gamma_matrix(N)) return 1;
    return N * kForceSplit <= kStepThreads ? kForceSplit : (2 * N <= kStepThreads ? 2 : 1);
}
// The per-pair tables and the double buffers live in shared memory when the
// whole layout fits in this many bytes (two blocks per SM at least).
constexpr size_t kFastSmemMax = 113 * 1024;

// Byte offsets of the step kernel's dynamic shared memory.  Always: the
// positions (float4 per atom), the force table of load_gamma and the partial
// force sums (float4 per atom and part).  With
// `fast`: the pair table, the feature means and inverse SDs, and two buffers
// of one replica's state [6][Np] and de/da row [Pp], filled ahead by
// cp.async.
struct StepSmem {
    size_t pos, gam, fpart, pij, mu, isd, gbuf, sbuf, total;
    bool fast;
};

__host__ __device__ __forceinline__ size_t up16(size_t b) { return (b + 15) & ~size_t(15); }

__host__ __device__ __forceinline__ StepSmem step_smem_layout(int N, int Np, int Pp) {
    StepSmem L{};
    L.pos = 0;
    L.gam = L.pos + up16(step_pos_bytes(N));
    L.fpart = L.gam + up16(4 * (size_t)gamma_floats(N, Pp));
    L.pij = L.fpart + up16(16 * (size_t)kForceSplit * N);
    L.mu = L.pij + up16(4 * (size_t)Pp);
    L.isd = L.mu + up16(4 * (size_t)Pp);
    L.gbuf = L.isd + up16(4 * (size_t)Pp);
    L.sbuf = L.gbuf + up16(2 * 2 * (size_t)Pp);
    const size_t end = L.sbuf + up16(2 * 4 * 6 * (size_t)Np);
    L.fast = end <= kFastSmemMax;
    L.total = L.fast ? end : L.pij;
    return L;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Queue the copies of replica k's state (and de/da row) into buffer b; one
// commit group per call, empty when k >= R, so that "all but the newest
// group" always means "the buffer of the current replica".  Rows are 16-byte
// multiples: 6 Np floats with Np a multiple of 4, Pp BF16 values with Pp a
// multiple of 8.
__device__ __forceinline__ void prefetch_replica(const MlpStepParams& p, long long k, int b,
                                                 unsigned char* sm, const StepSmem& L, bool need_ga) {
    if (k < p.R) {
        const int ns = 6 * p.Np / 4, ng = p.Pp / 8;
        const int4* src = reinterpret_cast<const int4*>(p.state + (size_t)k * 6 * p.Np);
        int4* dst = reinterpret_cast<int4*>(sm + L.sbuf) + (size_t)b * ns;
        for (int t = threadIdx.x; t < ns; t += blockDim.x) cp_async16(dst + t, src + t);
        if (need_ga) {
            const int4* gsrc = reinterpret_cast<const int4*>(p.ga + (size_t)k * p.Pp);
            int4* gdst = reinterpret_cast<int4*>(sm + L.gbuf) + (size_t)b * ng;
            for (int t = threadIdx.x; t < ng; t += blockDim.x) cp_async16(gdst + t, gsrc + t);
        }
    }
    cp_async_commit();
}

template <bool FAST>
__global__ void __launch_bounds__(kStepThreads) mlp_step_kernel(const MlpStepParams p) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double red[32];
    const int N = p.N, Np = p.Np;
    const StepSmem L = step_smem_layout(N, Np, p.Pp);
    float4* xs4 = reinterpret_cast<float4*>(sm + L.pos);
    float* gam = reinterpret_cast<float*>(sm + L.gam);
    float4* fpart = reinterpret_cast<float4*>(sm + L.fpart);
    const int nsplit = force_split(N);
    const ushort2* pij = p.pairs;
    const float* mu_t = p.mu;
    const float* isd_t = p.inv_sd;
    const int step_index = p.step_index_dev ? *p.step_index_dev : p.step_index;
    const uint32_t step = (p.dev_counters ? p.dev_counters[0] : 0u) + p.step0 + (uint32_t)step_index;
    const float sE = (float)p.sigma_E;
    const bool need_ga = p.mode != 0;
    init_gamma(N, gam);
    if (FAST) {
        ushort2* ps = reinterpret_cast<ushort2*>(sm + L.pij);
        float* ms = reinterpret_cast<float*>(sm + L.mu);
        float* is = reinterpret_cast<float*>(sm + L.isd);
        for (int t = threadIdx.x; t < p.Pp; t += blockDim.x) {
            ps[t] = p.pairs[t];
            ms[t] = p.mu[t];
            is[t] = p.inv_sd[t];
        }
        pij = ps;
        mu_t = ms;
        isd_t = is;
        prefetch_replica(p, blockIdx.x, 0, sm, L, need_ga);
    }
    int b = 0;
    for (long long k = blockIdx.x; k < p.R; k += gridDim.x, b ^= 1) {
        float* st = p.state + (size_t)k * 6 * Np;
        const float* ss = st;
        const __nv_bfloat16* gs = p.ga + (size_t)k * p.Pp;
        __syncthreads();  // the previous replica is done with every buffer
        if (FAST) {
            prefetch_replica(p, k + gridDim.x, b ^ 1, sm, L, need_ga);
            cp_async_wait_prev();
            __syncthreads();  // every thread's copies of this replica have landed
            ss = reinterpret_cast<const float*>(sm + L.sbuf) + (size_t)b * 6 * Np;
            gs = reinterpret_cast<const __nv_bfloat16*>(sm + L.gbuf) + (size_t)b * p.Pp;
        }
        load_pos4(ss, N, Np, xs4);
        __syncthreads();
        if (p.mode == 0) {
            pass_features(xs4, pij, p.P, p.Pp, mu_t, isd_t, p.a + (size_t)k * p.Pp);
            continue;
        }
        pass_gamma(xs4, pij, p.P, N, gs, isd_t, gam);
        __syncthreads();
        // forces of the current positions, F = -dE/dx (thread i: atom i)
        const int i = threadIdx.x;
        float3 f = make_float3(0.0f, 0.0f, 0.0f);
        if (nsplit == 1) {
            if (i < N) f = atom_force4(i, xs4, gam, N);
        } else {
            const int h = threadIdx.x / N, kk = threadIdx.x - h * N, len = (N + nsplit - 1) / nsplit;
            if (h < nsplit) {
                const int j0 = h * len, j1 = min(N, j0 + len);
                const float3 fp = atom_force4_range(kk, xs4, gam, N, j0, j1);
                fpart[h * N + kk] = make_float4(fp.x, fp.y, fp.z, 0.0f);
            }
            __syncthreads();
            if (i < N) {
                for (int hh = 0; hh < nsplit; ++hh) {
                    const float4 fp = fpart[hh * N + i];
                    f.x += fp.x;
                    f.y += fp.y;
                    f.z += fp.z;
                }
            }
        }
        f = make_float3(sE * f.x, sE * f.y, sE * f.z);
        __syncthreads();  // every force sum has read xs4
        double ek = 0.0;
        if (i < N) {
            const float im = 1.0f / p.masses[i];
            const float4 x4 = xs4[i];
            float x = x4.x, y = x4.y, z = x4.z;
            float vx = ss[3 * Np + i], vy = ss[4 * Np + i], vz = ss[5 * Np + i];
            if (p.mode == 1) {
                if (step_index > 0) {  // closing B of the previous step
                    vx = fmaf(p.hdt * im, f.x, vx);
                    vy = fmaf(p.hdt * im, f.y, vy);
                    vz = fmaf(p.hdt * im, f.z, vz);
                }
                vx = fmaf(p.hdt * im, f.x, vx);  // B
                vy = fmaf(p.hdt * im, f.y, vy);
                vz = fmaf(p.hdt * im, f.z, vz);
                x = fmaf(p.hdt, vx, x);  // A
                y = fmaf(p.hdt, vy, y);
                z = fmaf(p.hdt, vz, z);
                const float sd = p.c2kT * sqrtf(im);  // O
                const float3 n = normal3_fast(p.seed, (uint32_t)i, (uint32_t)k, step, p.purpose_mol);
                vx = fmaf(p.c1, vx, sd * n.x);
                vy = fmaf(p.c1, vy, sd * n.y);
                vz = fmaf(p.c1, vz, sd * n.z);
                x = fmaf(p.hdt, vx, x);  // A
                y = fmaf(p.hdt, vy, y);
                z = fmaf(p.hdt, vz, z);
                xs4[i] = make_float4(x, y, z, 0.0f);
                st[i] = x;
                st[Np + i] = y;
                st[2 * Np + i] = z;
            } else {
                if (p.theta > 0) {  // closing B of the last step
                    vx = fmaf(p.hdt * im, f.x, vx);
                    vy = fmaf(p.hdt * im, f.y, vy);
                    vz = fmaf(p.hdt * im, f.z, vz);
                }
                if (p.fout) {
                    float* fo = p.fout + (size_t)k * 3 * Np;
                    fo[i] = f.x;
                    fo[Np + i] = f.y;
                    fo[2 * Np + i] = f.z;
                }
                const double ms = (double)p.masses[i];
                ek += 0.5 * ms * ((double)vx * vx + (double)vy * vy + (double)vz * vz);
            }
            if (p.mode == 1 || p.theta > 0) {
                st[3 * Np + i] = vx;
                st[4 * Np + i] = vy;
                st[5 * Np + i] = vz;
            }
        }
        __syncthreads();  // new positions complete in xs4
        if (p.mode == 1) {
            pass_features(xs4, pij, p.P, p.Pp, mu_t, isd_t, p.a + (size_t)k * p.Pp);
            continue;
        }
        // mode 2: per-replica energy, kinetic energy and radius of gyration
        ek = block_sum(ek, red);
        double c[3];
        for (int d = 0; d < 3; ++d) {
            double s = 0.0;
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                const float4 x4 = xs4[i];
                s += d == 0 ? x4.x : (d == 1 ? x4.y : x4.z);
            }
            c[d] = block_sum(s, red) / N;
        }
        double r2 = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const float4 x4 = xs4[i];
            const double dx = x4.x - c[0], dy = x4.y - c[1], dz = x4.z - c[2];
            r2 += dx * dx + dy * dy + dz * dz;
        }
        r2 = block_sum(r2, red);
        if (threadIdx.x == 0) {
            const double E = p.sigma_E * head_energy(p.part, p.nparts, (int)k, p.b3) + p.mu_E;
            p.E[k] = E;
            p.ke[k] = ek;
            p.rg[k] = sqrt(r2 / N);
            if (!isfinite(E) && atomicCAS(&p.status[0], 0, PAMD_ENONFINITE) == 0) p.status[1] = (int)k;
        }
    }
    if (FAST) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Last node of a captured MD loop's body: advance the step index and keep the
// WHILE node looping until theta steps have run.
__global__ void mlp_loop_next_kernel(cudaGraphConditionalHandle h, int* ctr, int theta) {
    const int c = *ctr + 1;
    *ctr = c;
    cudaGraphSetConditional(h, c < theta ? 1u : 0u);
}

}  // namespace

size_t mlp_step_smem(int N, int Np, int Pp) { return step_smem_layout(N, Np, Pp).total; }

cudaError_t launch_mlp_step(const MlpStepParams& p, cudaStream_t s) {
    // the resident grid for this shared-memory size on the current device
    // (one block per resident slot; each block walks the replicas with
    // stride gridDim.x), looked up once per device, variant and size
    static std::mutex mu;
    static std::map<std::tuple<int, bool, size_t>, int> resident;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const StepSmem L = step_smem_layout(p.N, p.Np, p.Pp);
    const void* fn = L.fast ? (const void*)mlp_step_kernel<true> : (const void*)mlp_step_kernel<false>;
    e = ensure_dyn_smem(fn, L.total);
    if (e != cudaSuccess) return e;
    int grid_max = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        int& r = resident[std::make_tuple(dev, L.fast, L.total)];
        if (r == 0) {
            int per_sm = 0, sms = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kStepThreads, L.total);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
            if (per_sm < 1) return cudaErrorInvalidConfiguration;
            r = per_sm * sms;
        }
        grid_max = r;
    }
    const long long g = p.R < grid_max ? p.R : grid_max;
    if (L.fast)
        mlp_step_kernel<true><<<(int)g, kStepThreads, L.total, s>>>(p);
    else
        mlp_step_kernel<false><<<(int)g, kStepThreads, L.total, s>>>(p);
    return cudaGetLastError();
}

int mlp_propagate(pamd_mlp* m, float* state, double* E, double* ke, double* rg, float* fout,
                  const float* masses, int* status, const uint32_t* dev_counters, long long R,
                  int Np, int theta, double dt, double T, double gamma, unsigned long long seed,
                  uint32_t step0, uint32_t purpose_mol, cudaStream_t s, long long* launches) {
    if (m->broken) {
        set_last_error("force model unusable after an earlier CUDA error");
        return PAMD_ESTATE;
    }
    if (R > m->w.cap) {
        set_last_error("force model workspace smaller than the population");
        return PAMD_ESTATE;
    }
    MlpStepParams p{};
    p.state = state;
    p.E = E;
    p.ke = ke;
    p.rg = rg;
    p.fout = fout;
    p.masses = masses;
    p.status = status;
    p.dev_counters = dev_counters;
    p.R = R;
    p.N = m->N;
    p.Np = Np;
    p.P = m->P;
    p.Pp = m->Pp;
    p.nparts = m->nparts;
    p.theta = theta;
    p.ga = m->w.ga;
    p.part = m->w.part;
    p.mu = m->mu;
    p.inv_sd = m->inv_sd;
    p.pairs = m->pairs;
    p.a = m->w.a;
    p.b3 = m->params + m->ob3;
    p.sigma_E = m->sigma_E;
    p.mu_E = m->mu_E;
    p.hdt = (float)(0.5 * dt);
    const double c1 = std::exp(-gamma * dt);
    p.c1 = (float)c1;
    p.c2kT = (float)std::sqrt((1.0 - c1 * c1) * kBoltzmann * T);
    p.seed = seed;
    p.step0 = step0;
    p.purpose_mol = purpose_mol;
    const long long before = m->launches;
    int rc = PAMD_OK;
    auto step_launch = [&](int mode, int idx) {
        p.mode = mode;
        p.step_index = idx;
        const cudaError_t e = launch_mlp_step(p, s);
        m->launches += 1;
        if (e != cudaSuccess) {
            m->broken = true;
            set_last_error(std::string("surrogate step launch: ") + cudaGetErrorString(e));
            return PAMD_ECUDA;
        }
        return PAMD_OK;
    };
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &cs);
    if (ce != cudaSuccess) {
        m->broken = true;
        set_last_error(std::string("surrogate propagate: ") + cudaGetErrorString(ce));
        return PAMD_ECUDA;
    }
    rc = step_launch(0, 0);
    if (!rc) rc = mlp_gemms(m, (int)R, true, s, status);
    if (cs == cudaStreamCaptureStatusActive && theta > 0) {
        // In a graph the theta steps are one WHILE node whose body (step
        // kernel, four GEMMs, loop counter) runs theta times; the step index
        // lives in device memory.
        const long long b0 = m->launches;
        if (!rc) rc = mlp_loop_captured(m, p, theta, (int)R, s, status);
        if (!rc) m->launches += (long long)(theta - 1) * (m->launches - b0);
    } else {
        for (int i = 0; i < theta && !rc; ++i) {
            rc = step_launch(1, i);
            if (!rc) rc = mlp_gemms(m, (int)R, true, s, status);
        }
    }
    if (!rc) rc = step_launch(2, 0);
    if (launches) *launches += m->launches - before;
    return rc;
}

int mlp_loop_captured(pamd_mlp* m, MlpStepParams p, int theta, int M, cudaStream_t s, int* status) {
    if (!m->loop_ctr || !m->body_stream) {
        set_last_error("surrogate loop captured without mlp_prepare_capture");
        return PAMD_ESTATE;
    }
    auto bad = [&](cudaError_t e, const char* what) {
        m->broken = true;
        set_last_error(std::string("surrogate loop capture (") + what + "): " + cudaGetErrorString(e));
        return PAMD_ECUDA;
    };
    cudaError_t e = cudaMemsetAsync(m->loop_ctr, 0, sizeof(int), s);
    if (e != cudaSuccess) return bad(e, "counter reset");
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd);
    if (e != cudaSuccess) return bad(e, "capture info");
    cudaGraphConditionalHandle h{};
    e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return bad(e, "conditional handle");
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp);
    if (e != cudaSuccess) return bad(e, "WHILE node");
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) return bad(e, "capture dependencies");
    cudaStream_t bs = m->body_stream;
    e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bad(e, "body capture");
    p.mode = 1;
    p.step_index = 0;
    p.step_index_dev = m->loop_ctr;
    int rc = PAMD_OK;
    e = launch_mlp_step(p, bs);
    m->launches += 1;
    if (e != cudaSuccess) rc = bad(e, "step kernel");
    if (!rc) rc = mlp_gemms(m, M, true, bs, status);
    if (!rc) {
        mlp_loop_next_kernel<<<1, 1, 0, bs>>>(h, m->loop_ctr, theta);
        m->launches += 1;
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = bad(e, "loop counter kernel");
    }
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(bs, &out);
    if (!rc && e != cudaSuccess) rc = bad(e, "end of body capture");
    return rc;
}

}  // namespace pamd
