// propagate_mlp.cu -- BAOAB Langevin steps of a population whose forces and
// energies come from the MLP energy surrogate.
//
// The exact-force propagate kernel keeps each replica in shared memory for
// all theta steps; here every force evaluation is a batch of tensor-core
// GEMMs over the whole population, so the state stays in global memory and
// one step is five launches: this kernel (finish the previous step with its
// closing half kick, then B A O A of the next one and the features of the new
// positions) and the four GEMMs.  The update arithmetic and the Philox noise
// stream are those of the exact propagate kernel (same key, counter and
// purpose), so that the two force fields can be compared on identical noise.
#include "mlp_device.cuh"
#include "pamd_device.cuh"

namespace pamd {

namespace {

constexpr int kAtomsPerThread = (PAMD_MAX_ATOMS + kMlpThreads - 1) / kMlpThreads;

__global__ void __launch_bounds__(kMlpThreads) mlp_step_kernel(const MlpStepParams p) {
    extern __shared__ float ssm[];
    __shared__ double red[32];
    float* xs = ssm;             // [3][kXs]
    float* gam = ssm + 3 * kXs;  // gamma_floats(N, Pp)
    const int N = p.N, Np = p.Np;
    const uint32_t step = (p.dev_counters ? p.dev_counters[0] : 0u) + p.step0 + (uint32_t)p.step_index;
    const float sE = (float)p.sigma_E;
    init_gamma(N, gam);
    for (long long k = blockIdx.x; k < p.R; k += gridDim.x) {
        float* st = p.state + (size_t)k * 6 * Np;
        __syncthreads();
        for (int t = threadIdx.x; t < 3 * N; t += blockDim.x) {
            const int c = t / N, i = t - c * N;
            xs[c * kXs + i] = st[c * Np + i];
        }
        __syncthreads();
        if (p.mode == 0) {
            block_features(xs, p.pairs, p.mu, p.inv_sd, p.P, p.Pp, p.a + (size_t)k * p.Pp, nullptr, 0, 0);
            continue;
        }
        load_gamma(xs, p.ga + (size_t)k * p.Pp, p.inv_sd, p.pairs, p.P, N, gam);
        __syncthreads();
        // forces of the current positions, F = -dE/dx
        float fx[kAtomsPerThread], fy[kAtomsPerThread], fz[kAtomsPerThread];
#pragma unroll
        for (int q = 0; q < kAtomsPerThread; ++q) {
            const int i = threadIdx.x + q * kMlpThreads;
            fx[q] = fy[q] = fz[q] = 0.0f;
            if (i < N) {
                const float3 f = atom_force_any(i, xs, gam, N);
                fx[q] = sE * f.x;
                fy[q] = sE * f.y;
                fz[q] = sE * f.z;
            }
        }
        __syncthreads();  // every force sum has read xs
        double ek = 0.0;
#pragma unroll
        for (int q = 0; q < kAtomsPerThread; ++q) {
            const int i = threadIdx.x + q * kMlpThreads;
            if (i >= N) continue;
            const float im = 1.0f / p.masses[i];
            float x = xs[i], y = xs[kXs + i], z = xs[2 * kXs + i];
            float vx = st[3 * Np + i], vy = st[4 * Np + i], vz = st[5 * Np + i];
            if (p.mode == 1) {
                if (p.step_index > 0) {  // closing B of the previous step
                    vx = fmaf(p.hdt * im, fx[q], vx);
                    vy = fmaf(p.hdt * im, fy[q], vy);
                    vz = fmaf(p.hdt * im, fz[q], vz);
                }
                vx = fmaf(p.hdt * im, fx[q], vx);  // B
                vy = fmaf(p.hdt * im, fy[q], vy);
                vz = fmaf(p.hdt * im, fz[q], vz);
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
                xs[i] = x;
                xs[kXs + i] = y;
                xs[2 * kXs + i] = z;
                st[i] = x;
                st[Np + i] = y;
                st[2 * Np + i] = z;
            } else {
                if (p.theta > 0) {  // closing B of the last step
                    vx = fmaf(p.hdt * im, fx[q], vx);
                    vy = fmaf(p.hdt * im, fy[q], vy);
                    vz = fmaf(p.hdt * im, fz[q], vz);
                }
                if (p.fout) {
                    float* fo = p.fout + (size_t)k * 3 * Np;
                    fo[i] = fx[q];
                    fo[Np + i] = fy[q];
                    fo[2 * Np + i] = fz[q];
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
        __syncthreads();  // new positions complete in xs
        if (p.mode == 1) {
            block_features(xs, p.pairs, p.mu, p.inv_sd, p.P, p.Pp, p.a + (size_t)k * p.Pp, nullptr, 0, 0);
            continue;
        }
        // mode 2: per-replica energy, kinetic energy and radius of gyration
        ek = block_sum(ek, red);
        double c[3];
        for (int d = 0; d < 3; ++d) {
            double s = 0.0;
            for (int i = threadIdx.x; i < N; i += blockDim.x) s += xs[d * kXs + i];
            c[d] = block_sum(s, red) / N;
        }
        double r2 = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const double dx = xs[i] - c[0], dy = xs[kXs + i] - c[1], dz = xs[2 * kXs + i] - c[2];
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
}

}  // namespace

size_t mlp_step_smem(int N, int Pp) {
    return sizeof(float) * (3 * (size_t)kXs + (size_t)gamma_floats(N, Pp));
}

cudaError_t launch_mlp_step(const MlpStepParams& p, cudaStream_t s) {
    static size_t configured = 0;
    const size_t smem = mlp_step_smem(p.N, p.Pp);
    if (smem > configured) {
        const cudaError_t e =
            cudaFuncSetAttribute(mlp_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    const long long g = p.R < 152LL * 16 ? p.R : 152LL * 16;
    mlp_step_kernel<<<(int)g, kMlpThreads, smem, s>>>(p);
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
    rc = step_launch(0, 0);
    if (!rc) rc = mlp_gemms(m, (int)R, true, s, status);
    for (int i = 0; i < theta && !rc; ++i) {
        rc = step_launch(1, i);
        if (!rc) rc = mlp_gemms(m, (int)R, true, s, status);
    }
    if (!rc) rc = step_launch(2, 0);
    if (launches) *launches += m->launches - before;
    return rc;
}

}  // namespace pamd
