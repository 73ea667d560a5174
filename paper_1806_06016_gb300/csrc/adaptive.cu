// adaptive.cu -- the next temperature of an anneal from an overlap condition
// on the population's energy distribution (temperature-choice sentence of the
// PAMD scheme; the overlap estimate of Barash et al. 2017).
//
// For energies E_j at beta = 1/(k_B T_prev) and dbeta = 1/(k_B T) - beta:
//   tau_j = R exp(-dbeta E_j) / sum_k exp(-dbeta E_k),
//   alpha(dbeta) = (1/R) sum_j min(1, tau_j),
// and the next temperature is T_final if alpha(dbeta_final) >= alpha*, else
// the T with alpha = alpha*.  The search is a multisection: pass 0 tries
// dbeta_final alone, each later pass evaluates kG equally spaced candidates
// inside the current bracket (one block per candidate) and keeps the pair
// that straddles alpha*, shrinking the bracket by kG + 1; after kPasses the
// bracket is below 1e-6 of dbeta_final, about the resolution of the FP32
// candidate values.  The exponentials are FP32 on x_j = E_j - min E (FP64
// difference, rounded once); partial sums of up to kChunk FP32 terms go into
// FP64 accumulators and blocks reduce in a fixed order, so the result is
// deterministic.  Launches per step: 2 (min and x), then 2 per pass.
#include <cmath>
#include <string>

#include "../../include/pamd_adaptive.h"
#include "pamd_internal.h"

namespace pamd {
namespace {

constexpr int kT = 256;
constexpr int kG = 128;      // candidates per pass
constexpr int kPasses = 3;   // after pass 0
constexpr int kChunk = 32;   // FP32 terms per FP64 partial sum
constexpr int kMinBlocks = 1024;

struct OvState {
    double lo, hi, alpha_lo, emin;
    int done, at_final, pass, n_cand, bad, pad_[3];
    double cand[kG];
    double alpha[kG];
};

__device__ double blk_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kT / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] = __dadd_rn(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__device__ double blk_min(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kT / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// per-block minimum of E; NaN marks a block that saw a non-finite energy
__global__ void __launch_bounds__(kT) ov_min_kernel(const double* E, long long R, double* part) {
    __shared__ double sh[kT];
    double m = INFINITY;
    int bad = 0;
    for (long long j = (long long)blockIdx.x * kT + threadIdx.x; j < R; j += (long long)gridDim.x * kT) {
        const double e = E[j];
        if (!isfinite(e)) bad = 1;
        m = fmin(m, e);
    }
    bad = __syncthreads_or(bad);
    m = blk_min(m, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = bad ? NAN : m;
}

// x_j = E_j - min E in FP32; block 0 also sets up the search (pass 0: the
// final temperature alone)
__global__ void __launch_bounds__(kT) ov_x_kernel(const double* E, long long R, const double* part, int nparts,
                                                  double d_final, float* x, OvState* st) {
    __shared__ double sh[kT];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    double m = INFINITY;
    for (int i = threadIdx.x; i < nparts; i += kT) {
        const double p = part[i];
        if (isnan(p)) sbad = 1;
        m = fmin(m, p);
    }
    m = blk_min(m, sh);
    const int bad = sbad;
    for (long long j = (long long)blockIdx.x * kT + threadIdx.x; j < R; j += (long long)gridDim.x * kT)
        x[j] = __double2float_rn(__dsub_rn(E[j], m));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->lo = 0.0;
        st->hi = d_final;
        st->alpha_lo = 1.0;
        st->emin = m;
        st->done = bad;
        st->at_final = 0;
        st->pass = 0;
        st->n_cand = 1;
        st->bad = bad;
        st->cand[0] = d_final;
    }
}

// block g: alpha at candidate g
__global__ void __launch_bounds__(kT) ov_eval_kernel(const float* x, long long R, OvState* st) {
    __shared__ double sh[kT];
    if (st->done || (int)blockIdx.x >= st->n_cand) return;
    const float d = __double2float_rn(st->cand[blockIdx.x]);
    double S = 0.0;
    for (long long j0 = (long long)threadIdx.x; j0 < R; j0 += (long long)kT * kChunk) {
        float s = 0.0f;
        for (int c = 0; c < kChunk; ++c) {
            const long long j = j0 + (long long)c * kT;
            if (j < R) s += expf(-d * x[j]);
        }
        S += (double)s;
    }
    S = blk_sum(S, sh);
    const float r = (float)((double)R / S);
    double A = 0.0;
    for (long long j0 = (long long)threadIdx.x; j0 < R; j0 += (long long)kT * kChunk) {
        float s = 0.0f;
        for (int c = 0; c < kChunk; ++c) {
            const long long j = j0 + (long long)c * kT;
            if (j < R) s += fminf(1.0f, expf(-d * x[j]) * r);
        }
        A += (double)s;
    }
    A = blk_sum(A, sh);
    if (threadIdx.x == 0) st->alpha[blockIdx.x] = A / (double)R;
}

// keep the candidates that straddle alpha*, then lay out the next pass
__global__ void ov_pick_kernel(OvState* st, double target) {
    if (threadIdx.x != 0 || st->done) return;
    const int n = st->n_cand;
    if (st->pass == 0) {
        if (st->alpha[0] >= target) {
            st->lo = st->cand[0];
            st->alpha_lo = st->alpha[0];
            st->at_final = 1;
            st->done = 1;
            return;
        }
    } else {
        int g = 0;
        while (g < n && st->alpha[g] >= target) ++g;  // first candidate below the target
        if (g > 0) {
            st->lo = st->cand[g - 1];
            st->alpha_lo = st->alpha[g - 1];
        }
        if (g < n) st->hi = st->cand[g];
    }
    st->pass += 1;
    const double lo = st->lo, w = (st->hi - st->lo) / (double)(kG + 1);
    for (int g = 0; g < kG; ++g) st->cand[g] = lo + (double)(g + 1) * w;
    st->n_cand = kG;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

size_t overlap_work_bytes(long long R) {
    const int nparts = (int)std::min<long long>((R + kT - 1) / kT, kMinBlocks);
    return align256(sizeof(float) * (size_t)R) + align256(sizeof(double) * nparts) + align256(sizeof(OvState));
}

int overlap_step(cudaStream_t s, const double* E, long long R, double T_prev, double T_final,
                 double alpha_target, void* work, int num_sms, double* T_next, double* alpha_out,
                 long long* launches) {
    const int nparts = (int)std::min<long long>((R + kT - 1) / kT, kMinBlocks);
    unsigned char* base = static_cast<unsigned char*>(work);
    float* x = reinterpret_cast<float*>(base);
    double* part = reinterpret_cast<double*>(base + align256(sizeof(float) * (size_t)R));
    OvState* st = reinterpret_cast<OvState*>(base + align256(sizeof(float) * (size_t)R) +
                                             align256(sizeof(double) * nparts));
    const double beta = 1.0 / (kBoltzmann * T_prev);
    const double d_final = 1.0 / (kBoltzmann * T_final) - beta;
    const int gx = (int)std::min<long long>((R + kT - 1) / kT, 8LL * num_sms);
    ov_min_kernel<<<nparts, kT, 0, s>>>(E, R, part);
    ov_x_kernel<<<gx, kT, 0, s>>>(E, R, part, nparts, d_final, x, st);
    for (int r = 0; r <= kPasses; ++r) {
        ov_eval_kernel<<<r == 0 ? 1 : kG, kT, 0, s>>>(x, R, st);
        ov_pick_kernel<<<1, 32, 0, s>>>(st, alpha_target);
    }
    if (launches) *launches += 2 + 2 * (kPasses + 1);
    cudaError_t e = cudaGetLastError();
    OvState h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, st, sizeof(OvState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_last_error(std::string("overlap step: ") + cudaGetErrorString(e));
        return PAMD_ECUDA;
    }
    if (h.bad) {
        set_last_error("overlap step: a replica energy is not finite");
        return PAMD_ENONFINITE;
    }
    *T_next = h.at_final ? T_final : 1.0 / (kBoltzmann * (beta + h.lo));
    if (alpha_out) *alpha_out = h.alpha_lo;
    return PAMD_OK;
}

int overlap_check_args(long long R, double T_prev, double T_final, double alpha_target) {
    if (R < 1) {
        set_last_error("overlap step: R must be >= 1");
        return PAMD_EINVAL;
    }
    if (!(T_prev > 0) || !std::isfinite(T_prev) || !(T_final > 0) || !(T_final < T_prev)) {
        set_last_error("overlap step: temperatures must satisfy 0 < T_final < T_prev");
        return PAMD_EINVAL;
    }
    if (!(alpha_target > 0) || !(alpha_target < 1)) {
        set_last_error("overlap step: alpha_target must be in (0, 1)");
        return PAMD_EINVAL;
    }
    return PAMD_OK;
}

}  // namespace pamd

using namespace pamd;

extern "C" int pamd_overlap_temperature(const double* E_dev, int64_t R, double T_prev, double T_final,
                                        double alpha_target, double* T_next_out, double* alpha_out,
                                        void* stream) {
    if (!E_dev || !T_next_out) {
        set_last_error("overlap step: E_dev and T_next_out are required");
        return PAMD_EINVAL;
    }
    int rc = overlap_check_args(R, T_prev, T_final, alpha_target);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void* work = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync(&work, overlap_work_bytes(R), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_last_error(std::string("overlap step: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? PAMD_ENOMEM : PAMD_ECUDA;
    }
    rc = overlap_step(s, E_dev, R, T_prev, T_final, alpha_target, work, sms, T_next_out, alpha_out, nullptr);
    e = cudaFreeAsync(work, s);
    if (!rc && e != cudaSuccess) {
        set_last_error(std::string("overlap step: ") + cudaGetErrorString(e));
        return PAMD_ECUDA;
    }
    return rc;
}
