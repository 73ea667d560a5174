// wham.cu -- multiple-histogram reweighting (WHAM) of sampled potential
// energies on the GPU: histograms of every temperature's samples, the FP64
// self-consistency sweeps of Ferrenberg & Swendsen (1989) / Kumar et al.
// (1992) seeded by the running sum of ln Q (free-energy paragraph of the PAMD
// paper), and reweighted averages at any temperature.  Definitions in
// include/pamd_wham.h.
//
// Kernels:
//   range_kernel / range_final_kernel  min and max of the finite samples
//   hist_edges_kernel / hist_kernel   one grid row per temperature; integer
//                   counters in shared memory merged into global memory with
//                   integer atomics, so the counts are exact and independent
//                   of scheduling.  Up to kEdgeBins bins the bin comes from
//                   exact key-space edges (no FP64 work per sample: GB300's
//                   FP64 rate would bound the pass), above that from the FP64
//                   definition directly.
//   rowsum_kernel / colsum_kernel      N_i and ln H(b)
//   dos_kernel      one thread per bin: ln g_b from the current ln Z_i
//   lnz_kernel      one block per temperature: ln Z_i = ln sum_b g_b e^(-beta_i E_b)
//   gauge_kernel    ln Z_i -= ln Z_0, largest change, convergence flag
//   reweight_kernel one block per evaluation temperature
// A sweep is the last four launches; every sweep kernel returns at once once
// the flag is set, so the host checks it only every kCheckEvery sweeps.
// Sums of exponentials are max + ln sum exp(x - max), each sum taken in a
// fixed order (thread-strided partial sums, then a fixed tree).
#include <cmath>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "../../include/pamd_wham.h"
#include "pamd_internal.h"

namespace pamd {
namespace {

constexpr int kT = 256;             // threads of every block
constexpr int kSmemBins = 12288;    // shared-memory histogram limit (48 KiB)
constexpr int kMaxBins = 65536;
constexpr int kCheckEvery = 32;

__device__ __forceinline__ double centre(double e_min, double w, int b) {
    return __dadd_rn(e_min, __dmul_rn((double)b + 0.5, w));
}

// Block-wide max / sum of one value per thread, fixed tree order; result in
// every thread.
__device__ double block_max(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kT / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__device__ double block_sum(double v, double* sh) {
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

// Samples are read kUnroll per thread per step (coalesced across the block,
// independent loads in flight) so that the HBM-bound passes keep enough
// bytes in flight.
constexpr int kUnroll = 8;

// Order-preserving map of a double's bits to a signed 64-bit key: for
// doubles a < b (neither NaN), key(a) < key(b), and -0 and +0 both map to 0,
// so key comparisons agree with IEEE comparisons.  Range tests and min / max
// then run on the integer pipes, which GB300 has in far greater number than
// FP64 units.  NaNs map beyond the keys of +-inf.  The map is its own inverse
// on every key except 0, which goes back to +0.
__host__ __device__ __forceinline__ long long order_key(long long bits) {
    if (bits >= 0) return bits;
    return bits == (long long)0x8000000000000000ULL ? 0 : (bits ^ 0x7fffffffffffffffLL);
}
constexpr long long kKeyPosInf = 0x7ff0000000000000LL;
constexpr long long kKeyNegInf = -0x7ff0000000000001LL;  // order_key of -inf

__global__ void __launch_bounds__(kT) range_kernel(const double* E, long long n, double* bmin,
                                                   double* bmax) {
    __shared__ double sh[kT];
    const long long* Eb = reinterpret_cast<const long long*>(E);
    long long klo = kKeyPosInf, khi = kKeyNegInf;  // finite keys lie strictly between
    const long long stride = (long long)gridDim.x * kT;
    for (long long i0 = (long long)blockIdx.x * kT + threadIdx.x; i0 < n; i0 += stride * kUnroll) {
        long long v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const long long i = i0 + u * stride;
            v[u] = i < n ? order_key(Eb[i]) : kKeyPosInf;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (v[u] > kKeyNegInf && v[u] < kKeyPosInf) {  // finite
                klo = min(klo, v[u]);
                khi = max(khi, v[u]);
            }
        }
    }
    // back to doubles for the block reduction (exact: min and max pick values)
    const double lo = klo < kKeyPosInf ? __longlong_as_double(order_key(klo)) : INFINITY;
    const double hi = khi > kKeyNegInf ? __longlong_as_double(order_key(khi)) : -INFINITY;
    const double rhi = block_max(hi, sh);
    const double rlo = -block_max(-lo, sh);
    if (threadIdx.x == 0) {
        bmin[blockIdx.x] = rlo;
        bmax[blockIdx.x] = rhi;
    }
}

__global__ void __launch_bounds__(kT) range_final_kernel(const double* bmin, const double* bmax, int nb,
                                                         double* out) {
    __shared__ double sh[kT];
    double lo = INFINITY, hi = -INFINITY;
    for (int i = threadIdx.x; i < nb; i += kT) {
        lo = fmin(lo, bmin[i]);
        hi = fmax(hi, bmax[i]);
    }
    hi = block_max(hi, sh);
    lo = -block_max(-lo, sh);
    if (threadIdx.x == 0) {
        out[0] = lo;
        out[1] = hi;
    }
}

// Row blockIdx.y of E (the samples of one temperature) into hist[row][:].
// The range test runs on the order keys (kmin = key(e_min), kmax =
// key(e_max)); the bin is floor((e - e_min) * inv) in FP64 as the definition
// states, taken with one round-down conversion.
__global__ void __launch_bounds__(kT) hist_kernel(const double* E, long long R, int nbins, double e_min,
                                                  long long kmin, long long kmax, double inv, unsigned* hist,
                                                  int smem_bins) {
    extern __shared__ unsigned sh_hist[];
    const double* row = E + (size_t)blockIdx.y * (size_t)R;
    unsigned* gh = hist + (size_t)blockIdx.y * (size_t)nbins;
    if (smem_bins) {
        for (int b = threadIdx.x; b < nbins; b += kT) sh_hist[b] = 0u;
        __syncthreads();
    }
    const long long* rowb = reinterpret_cast<const long long*>(row);
    const long long stride = (long long)gridDim.x * kT;
    for (long long k0 = (long long)blockIdx.x * kT + threadIdx.x; k0 < R; k0 += stride * kUnroll) {
        long long v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const long long k = k0 + u * stride;
            v[u] = k < R ? rowb[k] : 0x7fffffffffffffffLL;  // a NaN: dropped below
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const long long key = order_key(v[u]);
            if (key < kmin || key > kmax) continue;  // NaN and out-of-range samples are dropped
            const double e = __longlong_as_double(v[u]);
            long long b = __double2ll_rd(__dmul_rn(__dsub_rn(e, e_min), inv));
            b = b < 0 ? 0 : (b > nbins - 1 ? nbins - 1 : b);
            if (smem_bins)
                atomicAdd(&sh_hist[b], 1u);
            else
                atomicAdd(&gh[b], 1u);
        }
    }
    if (smem_bins) {
        __syncthreads();
        for (int b = threadIdx.x; b < nbins; b += kT)
            if (sh_hist[b]) atomicAdd(&gh[b], sh_hist[b]);
    }
}

// The same histogram without FP64 arithmetic per sample (up to kEdgeBins
// bins): the host has found, for every bin b >= 1, the smallest order key
// edges[b - 1] whose value the definition puts in bin b or above (the bin is
// a non-decreasing function of the key).  A sample's bin is estimated in FP32
// and then moved to the one with edges[b - 1] <= key < edges[b], so the count
// is exactly the definition's.  Edges and counters live in shared memory.
constexpr int kEdgeBins = 4096;

// edges[b - 1] for b = 1 .. nbins - 1: the smallest key in [kmin, kmax] whose
// value the definition puts in bin b or above (kmax + 1 if none), by
// bisection over keys, one thread per edge.
__global__ void edges_kernel(int nbins, double e_min, double inv, long long kmin, long long kmax,
                             long long* edges) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x + 1;
    if (b >= nbins) return;
    long long lo = kmin, hi = kmax + 1;
    while (lo < hi) {
        // keys of a range across zero span nearly 2^64: halve the unsigned gap
        const long long mid = lo + (long long)(((unsigned long long)hi - (unsigned long long)lo) / 2ull);
        const double e = __longlong_as_double(mid >= 0 ? mid : (mid ^ 0x7fffffffffffffffLL));
        const long long bin = __double2ll_rd(__dmul_rn(__dsub_rn(e, e_min), inv));
        if (bin >= b) hi = mid;
        else lo = mid + 1;
    }
    edges[b - 1] = lo;
}

__global__ void __launch_bounds__(kT) hist_edges_kernel(const double* E, long long R, int nbins,
                                                        float e_min_f, float inv_f, long long kmin,
                                                        long long kmax, const long long* edges_g,
                                                        unsigned* hist) {
    extern __shared__ long long sh_edges[];                   // [nbins - 1]
    unsigned* sh_hist = reinterpret_cast<unsigned*>(sh_edges + (nbins - 1));  // [nbins]
    const long long* rowb = reinterpret_cast<const long long*>(E + (size_t)blockIdx.y * (size_t)R);
    unsigned* gh = hist + (size_t)blockIdx.y * (size_t)nbins;
    for (int b = threadIdx.x; b < nbins - 1; b += kT) sh_edges[b] = edges_g[b];
    for (int b = threadIdx.x; b < nbins; b += kT) sh_hist[b] = 0u;
    __syncthreads();
    const long long stride = (long long)gridDim.x * kT;
    for (long long k0 = (long long)blockIdx.x * kT + threadIdx.x; k0 < R; k0 += stride * kUnroll) {
        long long v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const long long k = k0 + u * stride;
            v[u] = k < R ? rowb[k] : 0x7fffffffffffffffLL;  // a NaN: dropped below
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const long long key = order_key(v[u]);
            if (key < kmin || key > kmax) continue;  // NaN and out-of-range samples are dropped
            const float t = (__double2float_rn(__longlong_as_double(v[u])) - e_min_f) * inv_f;
            int b = t > 0.0f ? (t < (float)(nbins - 1) ? (int)t : nbins - 1) : 0;
            while (b > 0 && key < sh_edges[b - 1]) --b;
            while (b < nbins - 1 && key >= sh_edges[b]) ++b;
            atomicAdd(&sh_hist[b], 1u);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += kT)
        if (sh_hist[b]) atomicAdd(&gh[b], sh_hist[b]);
}

// N_i = sum_b H_i(b) (exact, 64-bit) and ln N_i (-inf for an empty row).
__global__ void __launch_bounds__(kT) rowsum_kernel(const unsigned* hist, int nbins, double* lnN,
                                                    unsigned long long* N) {
    __shared__ unsigned long long sh[kT];
    const unsigned* h = hist + (size_t)blockIdx.x * (size_t)nbins;
    unsigned long long s = 0;
    for (int b = threadIdx.x; b < nbins; b += kT) s += h[b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int st = kT / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        N[blockIdx.x] = sh[0];
        lnN[blockIdx.x] = sh[0] ? log((double)sh[0]) : -INFINITY;
    }
}

// ln H(b), H(b) = sum_i H_i(b) (-inf for an empty bin).
__global__ void __launch_bounds__(kT) colsum_kernel(const unsigned* hist, int n_temps, int nbins,
                                                    double* lnH) {
    const int b = blockIdx.x * kT + threadIdx.x;
    if (b >= nbins) return;
    unsigned long long s = 0;
    for (int i = 0; i < n_temps; ++i) s += hist[(size_t)i * nbins + b];
    lnH[b] = s ? log((double)s) : -INFINITY;
}

struct SweepState {
    int done;
    int sweeps;
    double delta;
};

// ln g_b = ln H(b) - ln sum_i N_i exp(-beta_i E_b - ln Z_i)
__global__ void __launch_bounds__(kT) dos_kernel(const double* lnH, const double* lnN, const double* beta,
                                                 const double* lnZ, int n_temps, int nbins, double e_min,
                                                 double w, double* ln_g, const SweepState* st, int force) {
    if (!force && st->done) return;
    const int b = blockIdx.x * kT + threadIdx.x;
    if (b >= nbins) return;
    const double lh = lnH[b];
    if (!(lh > -INFINITY)) {
        ln_g[b] = -INFINITY;
        return;
    }
    const double Eb = centre(e_min, w, b);
    double m = -INFINITY;
    for (int i = 0; i < n_temps; ++i) {
        const double x = __dsub_rn(__dsub_rn(lnN[i], __dmul_rn(Eb, beta[i])), lnZ[i]);
        m = fmax(m, x);
    }
    double s = 0.0;
    for (int i = 0; i < n_temps; ++i) {
        const double x = __dsub_rn(__dsub_rn(lnN[i], __dmul_rn(Eb, beta[i])), lnZ[i]);
        s = __dadd_rn(s, exp(__dsub_rn(x, m)));
    }
    ln_g[b] = __dsub_rn(lh, __dadd_rn(log(s), m));
}

// block i: ln Z_i = ln sum_b g_b exp(-beta_i E_b)
__global__ void __launch_bounds__(kT) lnz_kernel(const double* ln_g, const double* beta, int nbins,
                                                 double e_min, double w, double* lnZ_new,
                                                 const SweepState* st) {
    __shared__ double sh[kT];
    if (st->done) return;
    const double bi = beta[blockIdx.x];
    double m = -INFINITY;
    for (int b = threadIdx.x; b < nbins; b += kT)
        m = fmax(m, __dsub_rn(ln_g[b], __dmul_rn(bi, centre(e_min, w, b))));
    m = block_max(m, sh);
    double s = 0.0;
    for (int b = threadIdx.x; b < nbins; b += kT) {
        const double x = __dsub_rn(ln_g[b], __dmul_rn(bi, centre(e_min, w, b)));
        s = __dadd_rn(s, exp(__dsub_rn(x, m)));
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) lnZ_new[blockIdx.x] = __dadd_rn(log(s), m);
}

// ln Z_i <- ln Z_new_i - ln Z_new_0; largest change; stop flag
__global__ void __launch_bounds__(kT) gauge_kernel(const double* lnZ_new, double* lnZ, int n_temps,
                                                   double tol, SweepState* st) {
    __shared__ double sh[kT];
    if (st->done) return;
    const double z0 = lnZ_new[0];
    double d = 0.0;
    for (int i = threadIdx.x; i < n_temps; i += kT) {
        const double v = __dsub_rn(lnZ_new[i], z0);
        d = fmax(d, fabs(__dsub_rn(v, lnZ[i])));
        lnZ[i] = v;
    }
    d = block_max(d, sh);
    if (threadIdx.x == 0) {
        st->sweeps += 1;
        st->delta = d;
        if (d < tol) st->done = 1;
    }
}

// block j: ln Z, <E> and var E at inverse temperature beta_eval[j]
__global__ void __launch_bounds__(kT) reweight_kernel(const double* ln_g, int nbins, double e_min, double w,
                                                      const double* beta_eval, double* out) {
    __shared__ double sh[kT];
    const double bj = beta_eval[blockIdx.x];
    double m = -INFINITY;
    for (int b = threadIdx.x; b < nbins; b += kT)
        m = fmax(m, __dsub_rn(ln_g[b], __dmul_rn(bj, centre(e_min, w, b))));
    m = block_max(m, sh);
    double s = 0.0;
    for (int b = threadIdx.x; b < nbins; b += kT)
        s = __dadd_rn(s, exp(__dsub_rn(__dsub_rn(ln_g[b], __dmul_rn(bj, centre(e_min, w, b))), m)));
    const double lz = __dadd_rn(log(block_sum(s, sh)), m);
    double mean = 0.0;
    for (int b = threadIdx.x; b < nbins; b += kT) {
        const double Eb = centre(e_min, w, b);
        const double p = exp(__dsub_rn(__dsub_rn(ln_g[b], __dmul_rn(bj, Eb)), lz));
        mean = __dadd_rn(mean, __dmul_rn(Eb, p));
    }
    mean = block_sum(mean, sh);
    double var = 0.0;
    for (int b = threadIdx.x; b < nbins; b += kT) {
        const double Eb = centre(e_min, w, b);
        const double p = exp(__dsub_rn(__dsub_rn(ln_g[b], __dmul_rn(bj, Eb)), lz));
        const double d = __dsub_rn(Eb, mean);
        var = __dadd_rn(var, __dmul_rn(__dmul_rn(d, d), p));
    }
    var = block_sum(var, sh);
    if (threadIdx.x == 0) {
        out[3 * blockIdx.x] = lz;
        out[3 * blockIdx.x + 1] = mean;
        out[3 * blockIdx.x + 2] = var;
    }
}

// Device workspace of one call, carved from one allocation.
struct Work {
    void* base = nullptr;
    unsigned* hist = nullptr;
    double *lnH = nullptr, *lnN = nullptr, *beta = nullptr, *lnZ = nullptr, *lnZ_new = nullptr;
    double *ln_g = nullptr, *beta_eval = nullptr, *eval = nullptr, *bmin = nullptr, *bmax = nullptr;
    double* range = nullptr;
    unsigned long long* N = nullptr;
    long long* edges = nullptr;
    SweepState* st = nullptr;
    ~Work() {
        if (base) cudaFree(base);
    }
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int cuda_err(cudaError_t e, const char* what) {
    set_last_error(std::string("pamd_wham: ") + what + ": " + cudaGetErrorString(e));
    return PAMD_ECUDA;
}

}  // namespace
}  // namespace pamd

using namespace pamd;

extern "C" int pamd_wham(const pamd_wham_args* a, pamd_wham_result* r) {
    if (!a || !r || !a->E || !a->T || !r->lnZ) {
        set_last_error("pamd_wham: args, result, E, T and result->lnZ are required");
        return PAMD_EINVAL;
    }
    const int nT = a->n_temps, nb = a->n_bins, ne = a->n_eval;
    const long long R = a->R;
    if (nT < 1 || nT > 65535 || R < 1 || R > 0xffffffffLL || nb < 1 || nb > kMaxBins || a->max_iter < 0 ||
        ne < 0 || (ne > 0 && !a->T_eval) || !(a->tol >= 0)) {
        set_last_error("pamd_wham: n_temps 1..65535, R 1..2^32-1 (32-bit counters), n_bins 1..65536, "
                       "max_iter >= 0, n_eval >= 0 with T_eval, tol >= 0");
        return PAMD_EINVAL;
    }
    const bool given_range = a->e_max > a->e_min;
    if (given_range && !(std::isfinite(a->e_min) && std::isfinite(a->e_max))) {
        set_last_error("pamd_wham: the energy range must be finite");
        return PAMD_EINVAL;
    }
    std::vector<double> beta(nT), beta_eval(ne > 0 ? ne : 1), lnZ0(nT, 0.0);
    for (int i = 0; i < nT; ++i) {
        if (!(a->T[i] > 0) || !std::isfinite(a->T[i])) {
            set_last_error("pamd_wham: temperatures must be > 0");
            return PAMD_EINVAL;
        }
        beta[i] = 1.0 / (kBoltzmann * a->T[i]);
    }
    for (int j = 0; j < ne; ++j) {
        if (!(a->T_eval[j] > 0) || !std::isfinite(a->T_eval[j])) {
            set_last_error("pamd_wham: evaluation temperatures must be > 0");
            return PAMD_EINVAL;
        }
        beta_eval[j] = 1.0 / (kBoltzmann * a->T_eval[j]);
    }
    if (a->lnZ_init) {
        for (int i = 0; i < nT; ++i) {
            if (!std::isfinite(a->lnZ_init[i])) {
                set_last_error("pamd_wham: lnZ_init must be finite");
                return PAMD_EINVAL;
            }
            lnZ0[i] = a->lnZ_init[i] - a->lnZ_init[0];
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(a->stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_err(e, "device query");

    const long long n_all = (long long)nT * R;
    const int range_blocks = (int)std::min<long long>((n_all + kT * kUnroll - 1) / (kT * kUnroll), 16LL * sms);
    // workspace layout
    Work wk;
    size_t off = 0;
    const size_t o_hist = off; off += align256(sizeof(unsigned) * (size_t)nT * nb);
    const size_t o_lnH = off; off += align256(sizeof(double) * nb);
    const size_t o_lng = off; off += align256(sizeof(double) * nb);
    const size_t o_lnN = off; off += align256(sizeof(double) * nT);
    const size_t o_beta = off; off += align256(sizeof(double) * nT);
    const size_t o_lnZ = off; off += align256(sizeof(double) * nT);
    const size_t o_lnZn = off; off += align256(sizeof(double) * nT);
    const size_t o_N = off; off += align256(sizeof(unsigned long long) * nT);
    const size_t o_be = off; off += align256(sizeof(double) * beta_eval.size());
    const size_t o_ev = off; off += align256(sizeof(double) * 3 * beta_eval.size());
    const size_t o_bmin = off; off += align256(sizeof(double) * range_blocks);
    const size_t o_bmax = off; off += align256(sizeof(double) * range_blocks);
    const size_t o_rng = off; off += align256(sizeof(double) * 2);
    const size_t o_st = off; off += align256(sizeof(SweepState));
    const size_t o_edges = off; off += align256(sizeof(long long) * (size_t)std::min(nb, kEdgeBins));
    e = cudaMalloc(&wk.base, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        wk.base = nullptr;
        set_last_error("pamd_wham: workspace allocation failed");
        return PAMD_ENOMEM;
    }
    unsigned char* base = static_cast<unsigned char*>(wk.base);
    wk.hist = reinterpret_cast<unsigned*>(base + o_hist);
    wk.lnH = reinterpret_cast<double*>(base + o_lnH);
    wk.ln_g = reinterpret_cast<double*>(base + o_lng);
    wk.lnN = reinterpret_cast<double*>(base + o_lnN);
    wk.beta = reinterpret_cast<double*>(base + o_beta);
    wk.lnZ = reinterpret_cast<double*>(base + o_lnZ);
    wk.lnZ_new = reinterpret_cast<double*>(base + o_lnZn);
    wk.N = reinterpret_cast<unsigned long long*>(base + o_N);
    wk.beta_eval = reinterpret_cast<double*>(base + o_be);
    wk.eval = reinterpret_cast<double*>(base + o_ev);
    wk.bmin = reinterpret_cast<double*>(base + o_bmin);
    wk.bmax = reinterpret_cast<double*>(base + o_bmax);
    wk.range = reinterpret_cast<double*>(base + o_rng);
    wk.st = reinterpret_cast<SweepState*>(base + o_st);
    wk.edges = reinterpret_cast<long long*>(base + o_edges);

    // energy range
    double e_min = a->e_min, e_max = a->e_max;
    if (!given_range) {
        range_kernel<<<range_blocks, kT, 0, s>>>(a->E, n_all, wk.bmin, wk.bmax);
        range_final_kernel<<<1, kT, 0, s>>>(wk.bmin, wk.bmax, range_blocks, wk.range);
        double rg[2];
        if ((e = cudaMemcpyAsync(rg, wk.range, sizeof(rg), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_err(e, "energy range");
        if (!std::isfinite(rg[0]) || !std::isfinite(rg[1])) {
            set_last_error("pamd_wham: no finite energy");
            return PAMD_EINVAL;
        }
        e_min = rg[0];
        e_max = rg[1] > rg[0] ? rg[1] : rg[0] + 1.0;
    }
    const double inv = (double)nb / (e_max - e_min);
    const double w = (e_max - e_min) / (double)nb;

    // histograms
    if ((e = cudaMemsetAsync(wk.hist, 0, sizeof(unsigned) * (size_t)nT * nb, s)) != cudaSuccess)
        return cuda_err(e, "clear histograms");
    const int smem_bins = nb <= kSmemBins ? 1 : 0;
    long long bx = (R + (long long)kT * kUnroll - 1) / ((long long)kT * kUnroll);
    const long long want = (16LL * sms + nT - 1) / nT;
    if (bx > want) bx = want;
    if (bx < 1) bx = 1;
    long long bmin_bits, bmax_bits;
    std::memcpy(&bmin_bits, &e_min, 8);
    std::memcpy(&bmax_bits, &e_max, 8);
    const long long kmin = order_key(bmin_bits), kmax = order_key(bmax_bits);
    if (nb <= kEdgeBins) {
        if (nb > 1) edges_kernel<<<(nb - 1 + 63) / 64, 64, 0, s>>>(nb, e_min, inv, kmin, kmax, wk.edges);
        const size_t smem = sizeof(long long) * (size_t)(nb - 1) + sizeof(unsigned) * (size_t)nb;
        hist_edges_kernel<<<dim3((unsigned)bx, (unsigned)nT), kT, smem, s>>>(
            a->E, R, nb, (float)e_min, (float)inv, kmin, kmax, wk.edges, wk.hist);
    } else {
        hist_kernel<<<dim3((unsigned)bx, (unsigned)nT), kT, smem_bins ? sizeof(unsigned) * nb : 0, s>>>(
            a->E, R, nb, e_min, kmin, kmax, inv, wk.hist, smem_bins);
    }
    rowsum_kernel<<<nT, kT, 0, s>>>(wk.hist, nb, wk.lnN, wk.N);
    colsum_kernel<<<(nb + kT - 1) / kT, kT, 0, s>>>(wk.hist, nT, nb, wk.lnH);
    std::vector<unsigned long long> N(nT);
    if ((e = cudaMemcpyAsync(N.data(), wk.N, sizeof(unsigned long long) * nT, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(wk.beta, beta.data(), sizeof(double) * nT, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(wk.lnZ, lnZ0.data(), sizeof(double) * nT, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaMemsetAsync(wk.st, 0, sizeof(SweepState), s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_err(e, "histograms");
    unsigned long long total = 0;
    for (unsigned long long n : N) total += n;
    if (total == 0) {
        set_last_error("pamd_wham: no sample inside the energy range");
        return PAMD_EINVAL;
    }

    // self-consistency sweeps
    const int gb = (nb + kT - 1) / kT;
    for (int it = 0; it < a->max_iter;) {
        const int chunk = std::min(kCheckEvery, a->max_iter - it);
        for (int c = 0; c < chunk; ++c) {
            dos_kernel<<<gb, kT, 0, s>>>(wk.lnH, wk.lnN, wk.beta, wk.lnZ, nT, nb, e_min, w, wk.ln_g, wk.st, 0);
            lnz_kernel<<<nT, kT, 0, s>>>(wk.ln_g, wk.beta, nb, e_min, w, wk.lnZ_new, wk.st);
            gauge_kernel<<<1, kT, 0, s>>>(wk.lnZ_new, wk.lnZ, nT, a->tol, wk.st);
        }
        it += chunk;
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "sweep launch");
        if (a->tol > 0 && it < a->max_iter) {
            SweepState h{};
            if ((e = cudaMemcpyAsync(&h, wk.st, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
                (e = cudaStreamSynchronize(s)) != cudaSuccess)
                return cuda_err(e, "convergence flag");
            if (h.done) break;
        }
    }
    // density of states of the final ln Z, and reweighting
    dos_kernel<<<gb, kT, 0, s>>>(wk.lnH, wk.lnN, wk.beta, wk.lnZ, nT, nb, e_min, w, wk.ln_g, wk.st, 1);
    if (ne > 0) {
        if ((e = cudaMemcpyAsync(wk.beta_eval, beta_eval.data(), sizeof(double) * ne, cudaMemcpyHostToDevice,
                                 s)) != cudaSuccess)
            return cuda_err(e, "evaluation temperatures");
        reweight_kernel<<<ne, kT, 0, s>>>(wk.ln_g, nb, e_min, w, wk.beta_eval, wk.eval);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "launch");
    SweepState h{};
    std::vector<double> ev(3 * (size_t)std::max(ne, 1));
    if ((e = cudaMemcpyAsync(&h, wk.st, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(r->lnZ, wk.lnZ, sizeof(double) * nT, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (r->ln_g &&
         (e = cudaMemcpyAsync(r->ln_g, wk.ln_g, sizeof(double) * nb, cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
        (r->hist && (e = cudaMemcpyAsync(r->hist, wk.hist, sizeof(unsigned) * (size_t)nT * nb,
                                         cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
        (ne > 0 && (e = cudaMemcpyAsync(ev.data(), wk.eval, sizeof(double) * 3 * ne, cudaMemcpyDeviceToHost,
                                        s)) != cudaSuccess) ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_err(e, "results");
    for (int j = 0; j < ne; ++j) {
        if (r->lnZ_eval) r->lnZ_eval[j] = ev[3 * j];
        if (r->e_mean_eval) r->e_mean_eval[j] = ev[3 * j + 1];
        if (r->e_var_eval) r->e_var_eval[j] = ev[3 * j + 2];
    }
    r->e_min = e_min;
    r->bin_width = w;
    r->iterations = h.sweeps;
    r->max_delta = h.sweeps > 0 ? h.delta : std::numeric_limits<double>::infinity();
    return PAMD_OK;
}
