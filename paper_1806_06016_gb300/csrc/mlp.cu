// mlp.cu -- the MLP energy surrogate: parameters, features, forces, the
// force-matching loss and its gradient, Adam, and the C-ABI of pamd_mlp.h.
//
// Dense layers are BF16 tensor-core GEMMs (mlp_gemm.cu) whose epilogues apply
// the bias, the SiLU and its derivative and write the BF16 operands of the
// next product (row-major, and transposed where a weight gradient needs them).
// Everything between the products (features, the pair Jacobian and its
// transpose, second-derivative terms, column sums) is FP32 here; energies and
// loss sums are FP64.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "mlp_device.cuh"
#include "pamd_device.cuh"

namespace pamd {

constexpr uint32_t kPurposeMlpInit = 3u;

namespace {

int mfail(int code, const std::string& msg) {
    set_last_error(msg);
    return code;
}

int mcuda(pamd_mlp* m, cudaError_t e, const char* what) {
    if (m) m->broken = true;
    return mfail(PAMD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define MLP_CU(m, call)                                       \
    do {                                                      \
        const cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return mcuda((m), e_, #call);  \
    } while (0)

int grid_for(long long n, int threads, int cap = 152 * 16) {
    long long g = (n + threads - 1) / threads;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

__device__ __forceinline__ float sig(float z) { return 1.0f / (1.0f + __expf(-z)); }
// second derivative of silu(z) = z s(z): s (1 - s) (2 + z (1 - 2 s))
__device__ __forceinline__ float d2silu(float z) {
    const float s = sig(z);
    return s * (1.0f - s) * (2.0f + z * (1.0f - 2.0f * s));
}

// ---------------------------------------------------------------- parameters

__global__ void mlp_init_kernel(float* params, size_t oW1, size_t oW2, size_t ow3, int H, int P,
                                int Pp, unsigned long long seed) {
    const long long n1 = (long long)H * Pp, n2 = (long long)H * H, n3 = H;
    const long long n = n1 + n2 + n3;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        uint32_t region;
        long long local;
        size_t dst;
        float scale;
        bool zero = false;
        if (e < n1) {
            region = 1;
            local = e;
            zero = (int)(e % Pp) >= P;
            scale = rsqrtf((float)P);
            dst = oW1 + (size_t)local;
        } else if (e < n1 + n2) {
            region = 2;
            local = e - n1;
            scale = rsqrtf((float)H);
            dst = oW2 + (size_t)local;
        } else {
            region = 3;
            local = e - n1 - n2;
            scale = rsqrtf((float)H);
            dst = ow3 + (size_t)local;
        }
        float v = 0.0f;
        if (!zero) {
            const uint4 o = philox4x32_10(
                make_uint4((uint32_t)local, (uint32_t)(local >> 32), region, kPurposeMlpInit),
                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
            const float u0 = ((float)(o.x >> 9) + 0.5f) * 1.1920928955078125e-07f;
            const float u1 = ((float)(o.y >> 9) + 0.5f) * 1.1920928955078125e-07f;
            v = sqrtf(-2.0f * logf(u0)) * cospif(2.0f * u1) * scale;  // Box-Muller
        }
        params[dst] = v;
    }
}

// BF16 copies of W1 and W2, row-major and transposed
__global__ void mlp_pack_kernel(const float* __restrict__ params, size_t oW1, size_t oW2, int H,
                                int Pp, __nv_bfloat16* W1b, __nv_bfloat16* W1Tb,
                                __nv_bfloat16* W2b, __nv_bfloat16* W2Tb) {
    const long long n1 = (long long)H * Pp, n2 = (long long)H * H;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n1 + n2;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < n1) {
            const int h = (int)(e / Pp), p = (int)(e % Pp);
            const __nv_bfloat16 b = __float2bfloat16(params[oW1 + e]);
            W1b[e] = b;
            W1Tb[(size_t)p * H + h] = b;
        } else {
            const long long l = e - n1;
            const int h = (int)(l / H), k = (int)(l % H);
            const __nv_bfloat16 b = __float2bfloat16(params[oW2 + l]);
            W2b[l] = b;
            W2Tb[(size_t)k * H + h] = b;
        }
    }
}

__global__ void mlp_adam_kernel(float* p, const float* __restrict__ g, float* m, float* v,
                                long long n, float lr, float b1, float b2, float eps, float bc1,
                                float bc2) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const float gi = g[e];
        const float mi = b1 * m[e] + (1.0f - b1) * gi;
        const float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
        m[e] = mi;
        v[e] = vi;
        p[e] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

// ------------------------------------------------------------- normalisation

__global__ void mlp_feature_stats_kernel(ConfigView cv, long long n, int N, int P,
                                         const ushort2* __restrict__ pairs, float* mu, float* sd,
                                         float* inv_sd) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const ushort2 ij = pairs[p];
    auto g_of = [&](long long m) {
        const float* x = cv.x + m * cv.s_cfg;
        const double dx = (double)x[ij.x * cv.s_atom] - x[ij.y * cv.s_atom];
        const double dy = (double)x[ij.x * cv.s_atom + cv.s_coord] - x[ij.y * cv.s_atom + cv.s_coord];
        const double dz = (double)x[ij.x * cv.s_atom + 2 * cv.s_coord] - x[ij.y * cv.s_atom + 2 * cv.s_coord];
        return 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
    };
    double s = 0.0;
    for (long long m = 0; m < n; ++m) s += g_of(m);
    const double mean = s / (double)n;
    double q = 0.0;
    for (long long m = 0; m < n; ++m) {
        const double d = g_of(m) - mean;
        q += d * d;
    }
    double dev = sqrt(q / (double)n);
    if (!(dev > 0.0)) dev = 1.0;
    mu[p] = (float)mean;
    sd[p] = (float)dev;
    inv_sd[p] = (float)(1.0 / dev);
}

__global__ void mlp_energy_stats_kernel(const double* __restrict__ E, long long n, double* out) {
    __shared__ double red[32];
    double s = 0.0;
    for (long long m = threadIdx.x; m < n; m += blockDim.x) s += E[m];
    const double mean = block_sum(s, red) / (double)n;
    double q = 0.0;
    for (long long m = threadIdx.x; m < n; m += blockDim.x) {
        const double d = E[m] - mean;
        q += d * d;
    }
    q = block_sum(q, red);
    if (threadIdx.x == 0) {
        out[0] = mean;
        out[1] = sqrt(q / (double)n);
    }
}

// ------------------------------------------------------- features and forces

__global__ void __launch_bounds__(kMlpThreads) mlp_features_kernel(const FeatArgs f) {
    __shared__ float xs[3 * kXs];
    for (int m = blockIdx.x; m < f.M; m += gridDim.x) {
        __syncthreads();
        load_config(f.cv, m, f.N, xs);
        __syncthreads();
        block_features(xs, f.pairs, f.mu, f.inv_sd, f.P, f.Pp, f.a + (size_t)m * f.Pp, f.aT,
                       f.ldt, m);
    }
}

__global__ void __launch_bounds__(kMlpThreads) mlp_forces_kernel(const ForceArgs f) {
    extern __shared__ float fsm[];
    float* xs = fsm;
    float* gam = fsm + 3 * kXs;
    init_gamma(f.N, gam);
    for (int m = blockIdx.x; m < f.M; m += gridDim.x) {
        __syncthreads();
        load_config(f.cv, m, f.N, xs);
        __syncthreads();
        if (f.F) load_gamma(xs, f.ga + (size_t)m * f.Pp, f.inv_sd, f.pairs, f.P, f.N, gam);
        __syncthreads();
        if (f.F) {
            const float sE = (float)f.sigma_E;
            float* Fo = f.F + (size_t)m * 3 * f.N;
            for (int k = threadIdx.x; k < f.N; k += blockDim.x) {
                const float3 a = atom_force_any(k, xs, gam, f.N);
                Fo[3 * k] = sE * a.x;
                Fo[3 * k + 1] = sE * a.y;
                Fo[3 * k + 2] = sE * a.z;
            }
        }
        if (f.E && threadIdx.x == 0)
            f.E[m] = f.sigma_E * head_energy(f.part, f.nparts, m, f.b3) + f.mu_E;
    }
}

// Force-matching loss of one sample and the direction of the tangent pass:
// f = sum_p gam_p dg_p/dx (normalised forces), u = dL/df, and
// nu_a = dL/d(de/da) = (J u) / sd with (J u)_p = (x_i - x_j).(u_i - u_j) / r^3.
__global__ void __launch_bounds__(kMlpThreads) mlp_loss_kernel(const LossArgs L) {
    extern __shared__ float lsm[];
    __shared__ double red[32];
    float* xs = lsm;
    float* us = lsm + 3 * kXs;
    float* gam = lsm + 6 * kXs;
    const double inv_sE = 1.0 / L.sigma_E;
    const float cu = (float)(2.0 * L.lam / (3.0 * L.N * (double)L.M));
    init_gamma(L.N, gam);
    for (int m = blockIdx.x; m < L.M; m += gridDim.x) {
        __syncthreads();
        load_config(L.cv, m, L.N, xs);
        __syncthreads();
        load_gamma(xs, L.ga + (size_t)m * L.Pp, L.inv_sd, L.pairs, L.P, L.N, gam);
        __syncthreads();
        const long long src = config_index(L.cv, m);
        const float* Fr = L.F_ref + src * 3 * L.N;
        double sq = 0.0;
        for (int k = threadIdx.x; k < L.N; k += blockDim.x) {
            const float3 a = atom_force_any(k, xs, gam, L.N);
            const float dfx = a.x - (float)(Fr[3 * k] * inv_sE);
            const float dfy = a.y - (float)(Fr[3 * k + 1] * inv_sE);
            const float dfz = a.z - (float)(Fr[3 * k + 2] * inv_sE);
            us[k] = cu * dfx;
            us[kXs + k] = cu * dfy;
            us[2 * kXs + k] = cu * dfz;
            sq += (double)dfx * dfx + (double)dfy * dfy + (double)dfz * dfz;
        }
        sq = block_sum(sq, red);  // also orders the writes of us before the reads below
        __nv_bfloat16* nrow = L.nu_a + (size_t)m * L.Pp;
        for (int p = threadIdx.x; p < L.Pp; p += blockDim.x) {
            float v = 0.0f;
            if (p < L.P) {
                const ushort2 ij = L.pairs[p];
                const int i = ij.x, j = ij.y;
                const float dx = xs[i] - xs[j], dy = xs[kXs + i] - xs[kXs + j],
                            dz = xs[2 * kXs + i] - xs[2 * kXs + j];
                const float ir = rsqrtf(dx * dx + dy * dy + dz * dz);
                const float jn = (dx * (us[i] - us[j]) + dy * (us[kXs + i] - us[kXs + j]) +
                                  dz * (us[2 * kXs + i] - us[2 * kXs + j])) *
                                 ir * ir * ir;
                v = jn * L.inv_sd[p];
            }
            const __nv_bfloat16 b = __float2bfloat16(v);
            nrow[p] = b;
            L.nu_aT[(size_t)p * L.ldt + m] = b;
        }
        if (threadIdx.x == 0) {
            const double e = head_energy(L.part, L.nparts, m, L.b3);
            const double de = e - (L.E_ref[src] - L.mu_E) * inv_sE;
            L.ebar[m] = (float)(2.0 * de / (double)L.M);
            L.loss_part[m] = de * de + L.lam / (3.0 * L.N) * sq;
        }
    }
}

// dL/dz2 = ebar d2 + w3 zd2 silu''(z2), with d2 = w3 silu'(z2); also the
// per-sample terms of the b2 and w3 gradients
__global__ void mlp_z2bar_kernel(int M, int H, const float* __restrict__ ebar,
                                 const float* __restrict__ z2, const float* __restrict__ s2,
                                 const float* __restrict__ zd2, const float* __restrict__ w3,
                                 __nv_bfloat16* z2b, __nv_bfloat16* A2T, int ldt, float* t_b2,
                                 float* t_w3) {
    const long long n = (long long)M * H;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(e / H), h = (int)(e % H);
        const float z = z2[e], ds = s2[e], td = zd2[e];
        const float zb = ebar[m] * (w3[h] * ds) + w3[h] * td * d2silu(z);
        const __nv_bfloat16 b = __float2bfloat16(zb);
        z2b[e] = b;
        A2T[(size_t)h * ldt + m] = b;
        t_b2[e] = zb;
        t_w3[e] = ebar[m] * (z * sig(z)) + td * ds;
    }
}

// dL/dz1 = h1_bar silu'(z1) + (W2^T d2) zd1 silu''(z1)
__global__ void mlp_z1bar_kernel(int M, int H, const float* __restrict__ h1b,
                                 const float* __restrict__ z1, const float* __restrict__ s1,
                                 const float* __restrict__ zd1, const float* __restrict__ w2d2,
                                 __nv_bfloat16* A1T, int ldt, float* t_b1) {
    const long long n = (long long)M * H;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(e / H), h = (int)(e % H);
        const float zb = h1b[e] * s1[e] + w2d2[e] * zd1[e] * d2silu(z1[e]);
        A1T[(size_t)h * ldt + m] = __float2bfloat16(zb);
        t_b1[e] = zb;
    }
}

// out[c] = sum over m of X[m * ld + c] (FP64 accumulation)
__global__ void mlp_colsum_kernel(const float* __restrict__ X, int M, int ncols, int ld, float* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    double s = 0.0;
    for (int m = 0; m < M; ++m) s += (double)X[(size_t)m * ld + c];
    out[c] = (float)s;
}

__global__ void mlp_loss_reduce_kernel(const double* __restrict__ part, int M, double* out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int m = threadIdx.x; m < M; m += blockDim.x) s += part[m];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[0] = s / (double)M;
}

// ------------------------------------------------------------------ helpers

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

int launch_check(pamd_mlp* m, const char* what) {
    m->launches += 1;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mcuda(m, e, what);
    return PAMD_OK;
}

int gemm(pamd_mlp* m, GemmArgs g, cudaStream_t s, int* status = nullptr) {
    g.status = status ? status : m->status;
    const cudaError_t e = launch_gemm_bf16(g, s);
    m->launches += 1;
    if (e != cudaSuccess) return mcuda(m, e, "tensor-core GEMM launch");
    return PAMD_OK;
}

int check_model(pamd_mlp* m) {
    if (!m) return mfail(PAMD_EINVAL, "null model");
    if (m->broken) return mfail(PAMD_ESTATE, "model unusable after an earlier CUDA error");
    return PAMD_OK;
}

int read_model_status(pamd_mlp* m) {
    int st = 0;
    MLP_CU(m, cudaMemcpyAsync(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    MLP_CU(m, cudaStreamSynchronize(m->stream));
    if (st) {
        m->broken = true;
        return mfail(st, "tensor-core pipeline timed out");
    }
    return PAMD_OK;
}

int pack(pamd_mlp* m) {
    const long long n = (long long)m->H * m->Pp + (long long)m->H * m->H;
    mlp_pack_kernel<<<grid_for(n, 256), 256, 0, m->stream>>>(m->params, m->oW1, m->oW2, m->H, m->Pp,
                                                             m->W1b, m->W1Tb, m->W2b, m->W2Tb);
    return launch_check(m, "weight pack");
}

size_t forces_smem(const pamd_mlp* m) { return sizeof(float) * (3 * kXs + (size_t)gamma_floats(m->N, m->Pp)); }
size_t loss_smem(const pamd_mlp* m) { return sizeof(float) * (6 * kXs + (size_t)gamma_floats(m->N, m->Pp)); }

// The dynamic shared-memory limits of the force and loss kernels on the
// current device, raised to what this model needs.
int set_smem_attrs(const pamd_mlp* m) {
    cudaError_t e = ensure_dyn_smem((const void*)mlp_forces_kernel, forces_smem(m));
    if (e == cudaSuccess) e = ensure_dyn_smem((const void*)mlp_loss_kernel, loss_smem(m));
    return e == cudaSuccess ? PAMD_OK : mfail(PAMD_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
}

int features(pamd_mlp* m, const ConfigView& cv, int M, __nv_bfloat16* aT, int ldt) {
    FeatArgs f{};
    f.cv = cv;
    f.M = M;
    f.N = m->N;
    f.P = m->P;
    f.Pp = m->Pp;
    f.pairs = m->pairs;
    f.mu = m->mu;
    f.inv_sd = m->inv_sd;
    f.a = m->w.a;
    f.aT = aT;
    f.ldt = ldt;
    mlp_features_kernel<<<grid_for((long long)M * kMlpThreads, kMlpThreads, 152 * 16), kMlpThreads, 0,
                          m->stream>>>(f);
    return launch_check(m, "features");
}

}  // namespace

// Workspace of cap >= M configurations (grows only; training buffers once
// requested stay).
int mlp_ensure_work(pamd_mlp* m, long long M, bool train) {
    MlpWork& w = m->w;
    if (M <= w.cap && (!train || w.train)) return PAMD_OK;
    const long long cap = M > w.cap ? ((M + 127) / 128) * 128 : w.cap;
    const bool tr = train || w.train;
    const size_t H = (size_t)m->H, Pp = (size_t)m->Pp, C = (size_t)cap;
    std::vector<size_t> sizes;
    // order: a h1 d2 d1 s1 ga part | z1 z2 s2 w2d2 zd1 zd2 h1b t0 t1 t2 nu_a hd1 z2b A1T B1T A2T B2T ebar loss
    sizes = {2 * C * Pp, 2 * C * H, 2 * C * H, 2 * C * H, 4 * C * H, 2 * C * Pp, 4 * C * (size_t)m->nparts};
    if (tr) {
        for (int i = 0; i < 10; ++i) sizes.push_back(4 * C * H);
        sizes.push_back(2 * C * Pp);
        sizes.push_back(2 * C * H);
        sizes.push_back(2 * C * H);
        sizes.push_back(2 * H * 2 * C);
        sizes.push_back(2 * Pp * 2 * C);
        sizes.push_back(2 * H * 2 * C);
        sizes.push_back(2 * H * 2 * C);
        sizes.push_back(4 * C);
        sizes.push_back(8 * C);
    }
    size_t total = 0;
    for (size_t s : sizes) total += align256(s);
    void* base = nullptr;
    if (cudaMalloc(&base, total) != cudaSuccess) {
        cudaGetLastError();
        return mfail(PAMD_ENOMEM, "surrogate workspace: cudaMalloc failed");
    }
    if (w.base) {
        cudaStreamSynchronize(m->stream);
        cudaFree(w.base);
    }
    m->work_gen += 1;  // graphs captured over the old workspace are stale
    MlpWork nw;
    nw.cap = cap;
    nw.train = tr;
    nw.base = base;
    char* p = static_cast<char*>(base);
    size_t k = 0;
    auto take = [&]() {
        char* r = p;
        p += align256(sizes[k++]);
        return r;
    };
    nw.a = reinterpret_cast<__nv_bfloat16*>(take());
    nw.h1 = reinterpret_cast<__nv_bfloat16*>(take());
    nw.d2 = reinterpret_cast<__nv_bfloat16*>(take());
    nw.d1 = reinterpret_cast<__nv_bfloat16*>(take());
    nw.s1 = reinterpret_cast<float*>(take());
    nw.ga = reinterpret_cast<__nv_bfloat16*>(take());
    nw.part = reinterpret_cast<float*>(take());
    if (tr) {
        float** f32[10] = {&nw.z1, &nw.z2, &nw.s2, &nw.w2d2, &nw.zd1, &nw.zd2, &nw.h1b, &nw.t0, &nw.t1, &nw.t2};
        for (auto q : f32) *q = reinterpret_cast<float*>(take());
        nw.nu_a = reinterpret_cast<__nv_bfloat16*>(take());
        nw.hd1 = reinterpret_cast<__nv_bfloat16*>(take());
        nw.z2b = reinterpret_cast<__nv_bfloat16*>(take());
        nw.A1T = reinterpret_cast<__nv_bfloat16*>(take());
        nw.B1T = reinterpret_cast<__nv_bfloat16*>(take());
        nw.A2T = reinterpret_cast<__nv_bfloat16*>(take());
        nw.B2T = reinterpret_cast<__nv_bfloat16*>(take());
        nw.ebar = reinterpret_cast<float*>(take());
        nw.loss_part = reinterpret_cast<double*>(take());
        // the transposed operands are read over K = 2M columns: clear them so
        // that no column is ever uninitialised memory
        if (cudaMemsetAsync(nw.A1T, 0, (size_t)(p - reinterpret_cast<char*>(nw.A1T)), m->stream) != cudaSuccess)
            return mcuda(m, cudaGetLastError(), "workspace clear");
    }
    w = nw;
    return PAMD_OK;
}

int mlp_prepare_capture(pamd_mlp* m) {
    if (!m->loop_ctr && cudaMalloc(&m->loop_ctr, sizeof(int)) != cudaSuccess) {
        m->loop_ctr = nullptr;
        cudaGetLastError();
        return mfail(PAMD_ENOMEM, "surrogate loop counter");
    }
    if (!m->body_stream && cudaStreamCreateWithFlags(&m->body_stream, cudaStreamNonBlocking) != cudaSuccess) {
        m->body_stream = nullptr;
        cudaGetLastError();
        return mfail(PAMD_ECUDA, "surrogate capture stream");
    }
    const cudaError_t e = gemm_prepare_device();
    if (e != cudaSuccess) return mcuda(m, e, "tensor-core GEMM set-up");
    return PAMD_OK;
}

int mlp_gemms(pamd_mlp* m, int M, bool forces, cudaStream_t s, int* status) {
    const MlpWork& w = m->w;
    const int H = m->H, Pp = m->Pp;
    int rc;
    GemmArgs g{};
    // layer 1: h1 = silu(a W1^T + b1), s1 = silu'(.)
    g.A = w.a; g.B = m->W1b; g.M = M; g.N = H; g.K = Pp; g.lda = Pp; g.ldb = Pp;
    g.bias = m->params + m->ob1; g.epi = kEpiSilu;
    g.Cs = w.s1; g.ldc = H; g.Cb = w.h1; g.ldcb = H;
    if ((rc = gemm(m, g, s, status))) return rc;
    // layer 2 and head: d2 = w3 silu'(z2), partial sums of w3 . silu(z2)
    g = GemmArgs{};
    g.A = w.h1; g.B = m->W2b; g.M = M; g.N = H; g.K = H; g.lda = H; g.ldb = H;
    g.bias = m->params + m->ob2; g.epi = kEpiHead; g.vec = m->params + m->ow3;
    g.Cb = w.d2; g.ldcb = H; g.ldc = H; g.part = w.part;
    if ((rc = gemm(m, g, s, status))) return rc;
    if (!forces) return PAMD_OK;
    // d1 = (d2 W2) * s1
    g = GemmArgs{};
    g.A = w.d2; g.B = m->W2Tb; g.M = M; g.N = H; g.K = H; g.lda = H; g.ldb = H;
    g.epi = kEpiMul; g.mul = w.s1; g.ldc = H; g.Cb = w.d1; g.ldcb = H;
    if ((rc = gemm(m, g, s, status))) return rc;
    // de/da = d1 W1
    g = GemmArgs{};
    g.A = w.d1; g.B = m->W1Tb; g.M = M; g.N = Pp; g.K = H; g.lda = H; g.ldb = H;
    g.epi = kEpiStore; g.Cb = w.ga; g.ldcb = Pp; g.ldc = Pp;
    return gemm(m, g, s, status);
}

}  // namespace pamd

using namespace pamd;

extern "C" {

int pamd_mlp_create(pamd_mlp** out, int32_t n_atoms, int32_t hidden, uint64_t seed, void* stream) {
    if (!out) return mfail(PAMD_EINVAL, "pamd_mlp_create: null output");
    *out = nullptr;
    if (n_atoms < 2 || n_atoms > PAMD_MAX_ATOMS)
        return mfail(PAMD_EINVAL, "pamd_mlp_create: n_atoms must be in 2.." + std::to_string(PAMD_MAX_ATOMS));
    if (hidden < 32 || hidden > 1024 || hidden % 32)
        return mfail(PAMD_EINVAL, "pamd_mlp_create: hidden must be 32..1024, a multiple of 32");
    pamd_mlp* m = new pamd_mlp;
    m->N = n_atoms;
    m->P = n_atoms * (n_atoms - 1) / 2;
    m->Pp = (m->P + 7) / 8 * 8;
    m->H = hidden;
    m->nparts = kGemmHeadParts * ((hidden + kGemmTileN - 1) / kGemmTileN);
    const size_t H = (size_t)hidden, Pp = (size_t)m->Pp;
    m->oW1 = 0;
    m->ob1 = H * Pp;
    m->oW2 = m->ob1 + H;
    m->ob2 = m->oW2 + H * H;
    m->ow3 = m->ob2 + H;
    m->ob3 = m->ow3 + H;
    m->n_params = m->ob3 + 4;
    const size_t pbytes = align256(4 * m->n_params);
    const size_t sizes[] = {pbytes, pbytes, pbytes, pbytes, align256(4 * Pp), align256(4 * Pp),
                            align256(4 * Pp), align256(2 * H * Pp), align256(2 * H * Pp),
                            align256(2 * H * H), align256(2 * H * H), align256(4 * Pp),
                            align256(sizeof(int)), align256(8 * 4)};
    size_t total = 0;
    for (size_t s : sizes) total += s;
    if (stream) {
        m->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete m;
            return mfail(PAMD_ECUDA, "pamd_mlp_create: stream creation failed");
        }
        m->own_stream = true;
    }
    if (cudaMalloc(&m->base, total) != cudaSuccess) {
        cudaGetLastError();
        pamd_mlp_destroy(m);
        return mfail(PAMD_ENOMEM, "pamd_mlp_create: cudaMalloc failed");
    }
    char* p = static_cast<char*>(m->base);
    int k = 0;
    auto take = [&]() {
        char* r = p;
        p += sizes[k++];
        return r;
    };
    m->params = reinterpret_cast<float*>(take());
    m->grads = reinterpret_cast<float*>(take());
    m->adam_m = reinterpret_cast<float*>(take());
    m->adam_v = reinterpret_cast<float*>(take());
    m->mu = reinterpret_cast<float*>(take());
    m->sd = reinterpret_cast<float*>(take());
    m->inv_sd = reinterpret_cast<float*>(take());
    m->W1b = reinterpret_cast<__nv_bfloat16*>(take());
    m->W1Tb = reinterpret_cast<__nv_bfloat16*>(take());
    m->W2b = reinterpret_cast<__nv_bfloat16*>(take());
    m->W2Tb = reinterpret_cast<__nv_bfloat16*>(take());
    m->pairs = reinterpret_cast<ushort2*>(take());
    m->status = reinterpret_cast<int*>(take());
    m->scratch = reinterpret_cast<double*>(take());
    // pair table, identity normalisation, zero moments
    std::vector<ushort2> pr(Pp, make_ushort2(0, 0));
    for (int i = 0, q = 0; i < n_atoms; ++i)
        for (int j = i + 1; j < n_atoms; ++j, ++q) pr[q] = make_ushort2((unsigned short)i, (unsigned short)j);
    std::vector<float> zeros(Pp, 0.0f), ones(Pp, 1.0f);
    cudaStream_t s = m->stream;
    int rc = PAMD_OK;
    if (cudaMemcpyAsync(m->pairs, pr.data(), 4 * Pp, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(m->mu, zeros.data(), 4 * Pp, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(m->sd, ones.data(), 4 * Pp, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(m->inv_sd, ones.data(), 4 * Pp, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(m->params, 0, 4 * pbytes, s) != cudaSuccess ||
        cudaMemsetAsync(m->status, 0, sizeof(int), s) != cudaSuccess)
        rc = mcuda(m, cudaGetLastError(), "pamd_mlp_create: initial copies");
    if (!rc) {
        const long long n = (long long)H * Pp + (long long)H * H + (long long)H;
        mlp_init_kernel<<<grid_for(n, 256), 256, 0, s>>>(m->params, m->oW1, m->oW2, m->ow3, m->H,
                                                         m->P, m->Pp, seed);
        rc = launch_check(m, "weight init");
    }
    if (!rc) rc = pack(m);
    if (!rc) rc = set_smem_attrs(m);
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = mcuda(m, cudaGetLastError(), "pamd_mlp_create");
    if (rc) {
        const std::string msg = pamd_last_error();
        pamd_mlp_destroy(m);
        return mfail(rc, msg);
    }
    *out = m;
    return PAMD_OK;
}

int pamd_mlp_info(pamd_mlp* m, int32_t* n_atoms, int32_t* n_pairs, int32_t* hidden) {
    if (!m) return mfail(PAMD_EINVAL, "null model");
    if (n_atoms) *n_atoms = m->N;
    if (n_pairs) *n_pairs = m->P;
    if (hidden) *hidden = m->H;
    return PAMD_OK;
}

int pamd_mlp_set_params(pamd_mlp* m, const pamd_mlp_params* hp) {
    int rc = check_model(m);
    if (rc) return rc;
    if (!hp) return mfail(PAMD_EINVAL, "pamd_mlp_set_params: null parameters");
    if (hp->sd)
        for (int p = 0; p < m->P; ++p)
            if (!(hp->sd[p] > 0.0f) || !std::isfinite(hp->sd[p]))
                return mfail(PAMD_EINVAL, "pamd_mlp_set_params: sd must be positive and finite");
    if (!(hp->sigma_E > 0.0) || !std::isfinite(hp->sigma_E) || !std::isfinite(hp->mu_E) ||
        !std::isfinite(hp->b3))
        return mfail(PAMD_EINVAL, "pamd_mlp_set_params: sigma_E > 0, mu_E and b3 finite");
    const int H = m->H, P = m->P, Pp = m->Pp;
    std::vector<float> buf((size_t)m->n_params);
    MLP_CU(m, cudaMemcpy(buf.data(), m->params, 4 * m->n_params, cudaMemcpyDeviceToHost));
    if (hp->W1)
        for (int h = 0; h < H; ++h)
            std::memcpy(&buf[m->oW1 + (size_t)h * Pp], hp->W1 + (size_t)h * P, 4 * (size_t)P);
    if (hp->b1) std::memcpy(&buf[m->ob1], hp->b1, 4 * (size_t)H);
    if (hp->W2) std::memcpy(&buf[m->oW2], hp->W2, 4 * (size_t)H * H);
    if (hp->b2) std::memcpy(&buf[m->ob2], hp->b2, 4 * (size_t)H);
    if (hp->w3) std::memcpy(&buf[m->ow3], hp->w3, 4 * (size_t)H);
    buf[m->ob3] = (float)hp->b3;
    MLP_CU(m, cudaMemcpy(m->params, buf.data(), 4 * m->n_params, cudaMemcpyHostToDevice));
    if (hp->mu || hp->sd) {
        std::vector<float> mu(Pp, 0.0f), sd(Pp, 1.0f), isd(Pp, 1.0f);
        MLP_CU(m, cudaMemcpy(mu.data(), m->mu, 4 * (size_t)Pp, cudaMemcpyDeviceToHost));
        MLP_CU(m, cudaMemcpy(sd.data(), m->sd, 4 * (size_t)Pp, cudaMemcpyDeviceToHost));
        if (hp->mu) std::memcpy(mu.data(), hp->mu, 4 * (size_t)P);
        if (hp->sd) std::memcpy(sd.data(), hp->sd, 4 * (size_t)P);
        for (int p = 0; p < Pp; ++p) isd[p] = (float)(1.0 / (double)sd[p]);
        MLP_CU(m, cudaMemcpy(m->mu, mu.data(), 4 * (size_t)Pp, cudaMemcpyHostToDevice));
        MLP_CU(m, cudaMemcpy(m->sd, sd.data(), 4 * (size_t)Pp, cudaMemcpyHostToDevice));
        MLP_CU(m, cudaMemcpy(m->inv_sd, isd.data(), 4 * (size_t)Pp, cudaMemcpyHostToDevice));
    }
    m->mu_E = hp->mu_E;
    m->sigma_E = hp->sigma_E;
    MLP_CU(m, cudaMemsetAsync(m->adam_m, 0, 4 * m->n_params, m->stream));
    MLP_CU(m, cudaMemsetAsync(m->adam_v, 0, 4 * m->n_params, m->stream));
    m->adam_t = 0;
    if ((rc = pack(m))) return rc;
    MLP_CU(m, cudaStreamSynchronize(m->stream));
    return PAMD_OK;
}

static int copy_out(pamd_mlp* m, const float* src, pamd_mlp_params* hp, bool with_norm) {
    const int H = m->H, P = m->P, Pp = m->Pp;
    std::vector<float> buf((size_t)m->n_params);
    MLP_CU(m, cudaStreamSynchronize(m->stream));
    MLP_CU(m, cudaMemcpy(buf.data(), src, 4 * m->n_params, cudaMemcpyDeviceToHost));
    if (hp->W1)
        for (int h = 0; h < H; ++h)
            std::memcpy(hp->W1 + (size_t)h * P, &buf[m->oW1 + (size_t)h * Pp], 4 * (size_t)P);
    if (hp->b1) std::memcpy(hp->b1, &buf[m->ob1], 4 * (size_t)H);
    if (hp->W2) std::memcpy(hp->W2, &buf[m->oW2], 4 * (size_t)H * H);
    if (hp->b2) std::memcpy(hp->b2, &buf[m->ob2], 4 * (size_t)H);
    if (hp->w3) std::memcpy(hp->w3, &buf[m->ow3], 4 * (size_t)H);
    hp->b3 = buf[m->ob3];
    if (with_norm) {
        if (hp->mu) MLP_CU(m, cudaMemcpy(hp->mu, m->mu, 4 * (size_t)P, cudaMemcpyDeviceToHost));
        if (hp->sd) MLP_CU(m, cudaMemcpy(hp->sd, m->sd, 4 * (size_t)P, cudaMemcpyDeviceToHost));
        hp->mu_E = m->mu_E;
        hp->sigma_E = m->sigma_E;
    }
    return PAMD_OK;
}

int pamd_mlp_get_params(pamd_mlp* m, pamd_mlp_params* hp) {
    int rc = check_model(m);
    if (rc) return rc;
    if (!hp) return mfail(PAMD_EINVAL, "pamd_mlp_get_params: null output");
    return copy_out(m, m->params, hp, true);
}

int pamd_mlp_get_grads(pamd_mlp* m, pamd_mlp_params* hp) {
    int rc = check_model(m);
    if (rc) return rc;
    if (!hp) return mfail(PAMD_EINVAL, "pamd_mlp_get_grads: null output");
    if ((rc = read_model_status(m))) return rc;
    return copy_out(m, m->grads, hp, false);
}

int pamd_mlp_fit_normalization(pamd_mlp* m, const float* x_dev, const double* E_dev, int64_t n) {
    int rc = check_model(m);
    if (rc) return rc;
    if (!x_dev || !E_dev || n < 2) return mfail(PAMD_EINVAL, "pamd_mlp_fit_normalization: null pointer or n < 2");
    ConfigView cv{x_dev, 3LL * m->N, 3, 1, nullptr};
    mlp_feature_stats_kernel<<<(m->P + 127) / 128, 128, 0, m->stream>>>(cv, n, m->N, m->P, m->pairs,
                                                                         m->mu, m->sd, m->inv_sd);
    if ((rc = launch_check(m, "feature statistics"))) return rc;
    mlp_energy_stats_kernel<<<1, 1024, 0, m->stream>>>(E_dev, n, m->scratch);
    if ((rc = launch_check(m, "energy statistics"))) return rc;
    double st[2];
    MLP_CU(m, cudaMemcpyAsync(st, m->scratch, sizeof(st), cudaMemcpyDeviceToHost, m->stream));
    MLP_CU(m, cudaStreamSynchronize(m->stream));
    if (!std::isfinite(st[0]) || !std::isfinite(st[1]))
        return mfail(PAMD_EINVAL, "pamd_mlp_fit_normalization: non-finite energies");
    m->mu_E = st[0];
    m->sigma_E = st[1] > 0.0 ? st[1] : 1.0;
    return PAMD_OK;
}

int pamd_mlp_energy_forces(pamd_mlp* m, const float* x_dev, int64_t M, double* E_dev, float* F_dev) {
    int rc = check_model(m);
    if (rc) return rc;
    if (!x_dev || M < 1 || M > (1LL << 24)) return mfail(PAMD_EINVAL, "pamd_mlp_energy_forces: null x or M");
    if (!E_dev && !F_dev) return PAMD_OK;
    if ((rc = mlp_ensure_work(m, M, false))) return rc;
    const ConfigView cv{x_dev, 3LL * m->N, 3, 1, nullptr};
    if ((rc = features(m, cv, (int)M, nullptr, 0))) return rc;
    if ((rc = mlp_gemms(m, (int)M, F_dev != nullptr, m->stream, m->status))) return rc;
    ForceArgs f{};
    f.cv = cv;
    f.M = (int)M;
    f.N = m->N;
    f.P = m->P;
    f.Pp = m->Pp;
    f.nparts = m->nparts;
    f.ga = m->w.ga;
    f.pairs = m->pairs;
    f.part = m->w.part;
    f.inv_sd = m->inv_sd;
    f.b3 = m->params + m->ob3;
    f.sigma_E = m->sigma_E;
    f.mu_E = m->mu_E;
    f.E = E_dev;
    f.F = F_dev;
    mlp_forces_kernel<<<grid_for(M * kMlpThreads, kMlpThreads, 152 * 16), kMlpThreads,
                        forces_smem(m), m->stream>>>(f);
    return launch_check(m, "surrogate forces");
}

int pamd_mlp_loss_grads(pamd_mlp* m, const float* x_dev, const double* E_dev, const float* F_dev,
                        const int32_t* idx_dev, int64_t M, double lam, double* loss) {
    int rc = check_model(m);
    if (rc) return rc;
    if (!x_dev || !E_dev || !F_dev) return mfail(PAMD_EINVAL, "pamd_mlp_loss_grads: null data pointer");
    if (M < 4 || M > 65536 || M % 4) return mfail(PAMD_EINVAL, "pamd_mlp_loss_grads: M must be 4..65536, a multiple of 4");
    if (!(lam >= 0.0) || !std::isfinite(lam)) return mfail(PAMD_EINVAL, "pamd_mlp_loss_grads: lam must be >= 0");
    if ((rc = mlp_ensure_work(m, M, true))) return rc;
    const MlpWork& w = m->w;
    const int H = m->H, Pp = m->Pp, Mi = (int)M, ldt = 2 * Mi;
    cudaStream_t s = m->stream;
    const ConfigView cv{x_dev, 3LL * m->N, 3, 1, idx_dev};
    // forward, keeping what the gradient needs
    if ((rc = features(m, cv, Mi, w.B1T, ldt))) return rc;
    GemmArgs g{};
    g.A = w.a; g.B = m->W1b; g.M = Mi; g.N = H; g.K = Pp; g.lda = Pp; g.ldb = Pp;
    g.bias = m->params + m->ob1; g.epi = kEpiSilu;
    g.C = w.z1; g.Cs = w.s1; g.ldc = H; g.Cb = w.h1; g.ldcb = H; g.CbT = w.B2T; g.ldt = ldt;
    if ((rc = gemm(m, g, s))) return rc;
    g = GemmArgs{};
    g.A = w.h1; g.B = m->W2b; g.M = Mi; g.N = H; g.K = H; g.lda = H; g.ldb = H;
    g.bias = m->params + m->ob2; g.epi = kEpiHead; g.vec = m->params + m->ow3;
    g.C = w.z2; g.Cs = w.s2; g.ldc = H; g.Cb = w.d2; g.ldcb = H; g.CbT = w.A2T + Mi; g.ldt = ldt;
    g.part = w.part;
    if ((rc = gemm(m, g, s))) return rc;
    g = GemmArgs{};
    g.A = w.d2; g.B = m->W2Tb; g.M = Mi; g.N = H; g.K = H; g.lda = H; g.ldb = H;
    g.epi = kEpiMul; g.mul = w.s1; g.C = w.w2d2; g.ldc = H; g.Cb = w.d1; g.ldcb = H;
    g.CbT = w.A1T + Mi; g.ldt = ldt;
    if ((rc = gemm(m, g, s))) return rc;
    g = GemmArgs{};
    g.A = w.d1; g.B = m->W1Tb; g.M = Mi; g.N = Pp; g.K = H; g.lda = H; g.ldb = H;
    g.epi = kEpiStore; g.Cb = w.ga; g.ldcb = Pp; g.ldc = Pp;
    if ((rc = gemm(m, g, s))) return rc;
    // loss, energy cotangent and the tangent direction nu_a
    LossArgs L{};
    L.cv = cv;
    L.E_ref = E_dev;
    L.F_ref = F_dev;
    L.M = Mi;
    L.N = m->N;
    L.P = m->P;
    L.Pp = Pp;
    L.nparts = m->nparts;
    L.pairs = m->pairs;
    L.ga = w.ga;
    L.part = w.part;
    L.inv_sd = m->inv_sd;
    L.b3 = m->params + m->ob3;
    L.mu_E = m->mu_E;
    L.sigma_E = m->sigma_E;
    L.lam = lam;
    L.nu_a = w.nu_a;
    L.nu_aT = w.B1T + Mi;
    L.ldt = ldt;
    L.ebar = w.ebar;
    L.loss_part = w.loss_part;
    mlp_loss_kernel<<<grid_for(M * kMlpThreads, kMlpThreads, 152 * 16), kMlpThreads, loss_smem(m), s>>>(L);
    if ((rc = launch_check(m, "loss"))) return rc;
    // tangent pass: zd1 = W1 nu_a, hd1 = zd1 s1, zd2 = W2 hd1
    g = GemmArgs{};
    g.A = w.nu_a; g.B = m->W1b; g.M = Mi; g.N = H; g.K = Pp; g.lda = Pp; g.ldb = Pp;
    g.epi = kEpiMul; g.mul = w.s1; g.C = w.zd1; g.ldc = H; g.Cb = w.hd1; g.ldcb = H;
    g.CbT = w.B2T + Mi; g.ldt = ldt;
    if ((rc = gemm(m, g, s))) return rc;
    g = GemmArgs{};
    g.A = w.hd1; g.B = m->W2b; g.M = Mi; g.N = H; g.K = H; g.lda = H; g.ldb = H;
    g.epi = kEpiStore; g.C = w.zd2; g.ldc = H;
    if ((rc = gemm(m, g, s))) return rc;
    // reverse: z2_bar, h1_bar = z2_bar W2, z1_bar
    const long long nMH = (long long)Mi * H;
    mlp_z2bar_kernel<<<grid_for(nMH, 256), 256, 0, s>>>(Mi, H, w.ebar, w.z2, w.s2, w.zd2,
                                                        m->params + m->ow3, w.z2b, w.A2T, ldt,
                                                        w.t0, w.t1);
    if ((rc = launch_check(m, "z2 cotangent"))) return rc;
    g = GemmArgs{};
    g.A = w.z2b; g.B = m->W2Tb; g.M = Mi; g.N = H; g.K = H; g.lda = H; g.ldb = H;
    g.epi = kEpiStore; g.C = w.h1b; g.ldc = H;
    if ((rc = gemm(m, g, s))) return rc;
    mlp_z1bar_kernel<<<grid_for(nMH, 256), 256, 0, s>>>(Mi, H, w.h1b, w.z1, w.s1, w.zd1, w.w2d2,
                                                        w.A1T, ldt, w.t2);
    if ((rc = launch_check(m, "z1 cotangent"))) return rc;
    // weight gradients: contractions over the 2M columns of the transposed operands
    g = GemmArgs{};
    g.A = w.A1T; g.B = w.B1T; g.M = H; g.N = Pp; g.K = ldt; g.lda = ldt; g.ldb = ldt;
    g.epi = kEpiStore; g.C = m->grads + m->oW1; g.ldc = Pp;
    if ((rc = gemm(m, g, s))) return rc;
    g = GemmArgs{};
    g.A = w.A2T; g.B = w.B2T; g.M = H; g.N = H; g.K = ldt; g.lda = ldt; g.ldb = ldt;
    g.epi = kEpiStore; g.C = m->grads + m->oW2; g.ldc = H;
    if ((rc = gemm(m, g, s))) return rc;
    const int cg = (H + 127) / 128;
    mlp_colsum_kernel<<<cg, 128, 0, s>>>(w.t2, Mi, H, H, m->grads + m->ob1);
    if ((rc = launch_check(m, "b1 gradient"))) return rc;
    mlp_colsum_kernel<<<cg, 128, 0, s>>>(w.t0, Mi, H, H, m->grads + m->ob2);
    if ((rc = launch_check(m, "b2 gradient"))) return rc;
    mlp_colsum_kernel<<<cg, 128, 0, s>>>(w.t1, Mi, H, H, m->grads + m->ow3);
    if ((rc = launch_check(m, "w3 gradient"))) return rc;
    mlp_colsum_kernel<<<1, 128, 0, s>>>(w.ebar, Mi, 1, 1, m->grads + m->ob3);
    if ((rc = launch_check(m, "b3 gradient"))) return rc;
    mlp_loss_reduce_kernel<<<1, 256, 0, s>>>(w.loss_part, Mi, m->scratch);
    if ((rc = launch_check(m, "loss sum"))) return rc;
    if (loss) {
        MLP_CU(m, cudaMemcpyAsync(loss, m->scratch, sizeof(double), cudaMemcpyDeviceToHost, s));
        if ((rc = read_model_status(m))) return rc;
    }
    return PAMD_OK;
}

int pamd_mlp_adam_step(pamd_mlp* m, double lr, double beta1, double beta2, double eps) {
    int rc = check_model(m);
    if (rc) return rc;
    if (!(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
        return mfail(PAMD_EINVAL, "pamd_mlp_adam_step: lr > 0, 0 <= beta < 1, eps > 0");
    m->adam_t += 1;
    const float bc1 = (float)(1.0 - std::pow(beta1, (double)m->adam_t));
    const float bc2 = (float)(1.0 - std::pow(beta2, (double)m->adam_t));
    const long long n = (long long)m->ob3 + 1;
    mlp_adam_kernel<<<grid_for(n, 256), 256, 0, m->stream>>>(m->params, m->grads, m->adam_m, m->adam_v, n,
                                                             (float)lr, (float)beta1, (float)beta2,
                                                             (float)eps, bc1, bc2);
    if ((rc = launch_check(m, "Adam"))) return rc;
    return pack(m);
}

// Model file: magic, {N, H}, the FP32 parameter block (W1 padded to Pp
// columns), mu and sd [Pp], mu_E, sigma_E, FNV-1a 64 checksum of all before.
static const char kMlpMagic[8] = {'P', 'A', 'M', 'D', 'M', 'L', 'P', '1'};

static uint64_t mlp_fnv(const void* d, size_t n, uint64_t h) {
    const unsigned char* b = static_cast<const unsigned char*>(d);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

int pamd_mlp_save(pamd_mlp* m, const char* path) {
    int rc = check_model(m);
    if (rc) return rc;
    if (!path) return mfail(PAMD_EINVAL, "pamd_mlp_save: null path");
    std::vector<float> prm(m->n_params), mu(m->Pp), sd(m->Pp);
    MLP_CU(m, cudaStreamSynchronize(m->stream));
    MLP_CU(m, cudaMemcpy(prm.data(), m->params, 4 * prm.size(), cudaMemcpyDeviceToHost));
    MLP_CU(m, cudaMemcpy(mu.data(), m->mu, 4 * mu.size(), cudaMemcpyDeviceToHost));
    MLP_CU(m, cudaMemcpy(sd.data(), m->sd, 4 * sd.size(), cudaMemcpyDeviceToHost));
    const int32_t shape[2] = {m->N, m->H};
    const double norm[2] = {m->mu_E, m->sigma_E};
    uint64_t h = mlp_fnv(kMlpMagic, 8, 1469598103934665603ull);
    h = mlp_fnv(shape, sizeof(shape), h);
    h = mlp_fnv(prm.data(), 4 * prm.size(), h);
    h = mlp_fnv(mu.data(), 4 * mu.size(), h);
    h = mlp_fnv(sd.data(), 4 * sd.size(), h);
    h = mlp_fnv(norm, sizeof(norm), h);
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return mfail(PAMD_EINVAL, std::string("pamd_mlp_save: cannot write ") + tmp);
    bool ok = std::fwrite(kMlpMagic, 1, 8, f) == 8 && std::fwrite(shape, sizeof(shape), 1, f) == 1 &&
              std::fwrite(prm.data(), 4, prm.size(), f) == prm.size() &&
              std::fwrite(mu.data(), 4, mu.size(), f) == mu.size() &&
              std::fwrite(sd.data(), 4, sd.size(), f) == sd.size() &&
              std::fwrite(norm, sizeof(norm), 1, f) == 1 && std::fwrite(&h, sizeof(h), 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return mfail(PAMD_EINVAL, std::string("pamd_mlp_save: cannot write ") + path);
    }
    return PAMD_OK;
}

int pamd_mlp_load(pamd_mlp** out, const char* path, void* stream) {
    if (!out || !path) return mfail(PAMD_EINVAL, "pamd_mlp_load: null output or path");
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return mfail(PAMD_EINVAL, std::string("pamd_mlp_load: cannot read ") + path);
    char magic[8];
    int32_t shape[2] = {0, 0};
    if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kMlpMagic, 8) != 0 ||
        std::fread(shape, sizeof(shape), 1, f) != 1) {
        std::fclose(f);
        return mfail(PAMD_EINVAL, std::string("pamd_mlp_load: ") + path + " is not a model file");
    }
    pamd_mlp* m = nullptr;
    int rc = pamd_mlp_create(&m, shape[0], shape[1], 0, stream);
    if (rc) {
        std::fclose(f);
        return rc;
    }
    std::vector<float> prm(m->n_params), mu(m->Pp), sd(m->Pp);
    double norm[2] = {0.0, 1.0};
    uint64_t h_file = 0;
    bool ok = std::fread(prm.data(), 4, prm.size(), f) == prm.size() &&
              std::fread(mu.data(), 4, mu.size(), f) == mu.size() &&
              std::fread(sd.data(), 4, sd.size(), f) == sd.size() &&
              std::fread(norm, sizeof(norm), 1, f) == 1 && std::fread(&h_file, sizeof(h_file), 1, f) == 1;
    std::fclose(f);
    uint64_t h = mlp_fnv(kMlpMagic, 8, 1469598103934665603ull);
    h = mlp_fnv(shape, sizeof(shape), h);
    h = mlp_fnv(prm.data(), 4 * prm.size(), h);
    h = mlp_fnv(mu.data(), 4 * mu.size(), h);
    h = mlp_fnv(sd.data(), 4 * sd.size(), h);
    h = mlp_fnv(norm, sizeof(norm), h);
    bool sane = ok && h == h_file && norm[1] > 0.0 && std::isfinite(norm[0]) && std::isfinite(norm[1]);
    for (size_t p = 0; sane && p < sd.size(); ++p) sane = sd[p] > 0.0f && std::isfinite(sd[p]);
    if (!sane) {
        pamd_mlp_destroy(m);
        return mfail(PAMD_EINVAL, std::string("pamd_mlp_load: ") + path + " is truncated or corrupt");
    }
    std::vector<float> isd(m->Pp);
    for (int p = 0; p < m->Pp; ++p) isd[p] = (float)(1.0 / (double)sd[p]);
    m->mu_E = norm[0];
    m->sigma_E = norm[1];
    cudaError_t e = cudaMemcpy(m->params, prm.data(), 4 * prm.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->mu, mu.data(), 4 * mu.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->sd, sd.data(), 4 * sd.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->inv_sd, isd.data(), 4 * isd.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        pamd_mlp_destroy(m);
        return mfail(PAMD_ECUDA, std::string("pamd_mlp_load: ") + cudaGetErrorString(e));
    }
    if ((rc = pack(m)) || (rc = read_model_status(m))) {
        pamd_mlp_destroy(m);
        return rc;
    }
    *out = m;
    return PAMD_OK;
}

int pamd_mlp_sync(pamd_mlp* m) {
    int rc = check_model(m);
    if (rc) return rc;
    return read_model_status(m);
}

int64_t pamd_mlp_launch_count(pamd_mlp* m) { return m ? m->launches : 0; }

void pamd_mlp_destroy(pamd_mlp* m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    if (m->loop_ctr) cudaFree(m->loop_ctr);
    if (m->body_stream) cudaStreamDestroy(m->body_stream);
    if (m->w.base) cudaFree(m->w.base);
    if (m->base) cudaFree(m->base);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

}  // extern "C"
