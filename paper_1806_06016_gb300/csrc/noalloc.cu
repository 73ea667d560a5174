// noalloc.cu -- resampling copy counts without any device allocation.
//
// Some callers cannot allocate device memory: code that runs under a
// framework which owns the whole device pool (a custom operator whose memory
// must all come from the host framework), code that must not trigger the
// implicit device-wide synchronisation that cudaFree can cause, and loops
// with a fixed, pre-reserved memory budget.  pamd_resample_counts_noalloc
// serves them: the caller passes device inputs and outputs, and the scratch
// the resampling needs (weights and their prefix sums, per-block partial sums,
// a few scalars) lives in one file-scope device array of fixed size that every
// GPU loading this library holds until the process exits.
#include <cmath>
#include <mutex>
#include <string>

#include "pamd_device.cuh"
#include "pamd_internal.h"

namespace pamd {

__global__ void weights_kernel(const double* E, long long R, double dbeta, double two_s,
                               DevScalars* s, ExpCoef cf, unsigned long long* W,
                               unsigned long long* blk_w, double* blk_e, const uint32_t* live);

namespace {

constexpr long long kNoAllocMaxR = 1LL << 18;            // replicas per call at most
constexpr int kNoAllocBlocks = (int)(kNoAllocMaxR / 1024);  // 1024-element scan blocks
// Byte layout of the scratch array (all parts 256-byte aligned).
constexpr size_t kOffC = 0;                                    // u64 [kNoAllocMaxR]
constexpr size_t kOffBlkW = kOffC + 8 * kNoAllocMaxR;           // u64 [kNoAllocBlocks]
constexpr size_t kOffBlkE = kOffBlkW + 8 * kNoAllocBlocks;      // double [kNoAllocBlocks]
constexpr size_t kOffScal = kOffBlkE + 8 * kNoAllocBlocks;      // DevScalars
constexpr size_t kScratchBytes = kOffScal + 256;               // 2.1 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (the array's
// name in host code is only a stand-in).  Looked up again on every call made
// outside stream capture, so that a device reset, which may reload the module
// at another address, leaves no stale pointer behind; a call whose stream is
// being captured uses the address of the device's last uncaptured call.
int scratch_address(cudaStream_t s, unsigned char** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_last_error("no usable CUDA device");
        return PAMD_ECUDA;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        set_last_error("cudaStreamIsCapturing failed");
        return PAMD_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return PAMD_ECUDA;
        }
        g_scratch_ptr[dev] = p;
    } else if (!g_scratch_ptr[dev]) {
        set_last_error("the first call on a device must come before any stream capture");
        return PAMD_ECUDA;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return PAMD_OK;
}

ExpCoef inverse_factorials() {
    ExpCoef cf;
    double f = 1.0;
    for (int n = 0; n < 14; ++n) {
        if (n > 0) f *= (double)n;
        cf.c[n] = 1.0 / f;
    }
    return cf;
}

}  // namespace
}  // namespace pamd

using namespace pamd;

extern "C" int pamd_resample_counts_noalloc(const double* E_dev, int64_t R, double T_prev,
                                            double T_next, uint64_t seed, uint32_t resample_index,
                                            int32_t mol_id, int32_t* counts_dev, double* lnQ_dev,
                                            int32_t* status_dev, void* stream) {
    if (!E_dev || !counts_dev) {
        set_last_error("E_dev and counts_dev are required");
        return PAMD_EINVAL;
    }
    if (R < 1 || R > kNoAllocMaxR) {
        set_last_error("R must be in 1 .. 262144 (the size of the fixed scratch array)");
        return PAMD_EINVAL;
    }
    if (!(T_prev > 0) || !(T_next > 0) || !std::isfinite(T_prev) || !std::isfinite(T_next)) {
        set_last_error("temperatures must be > 0");
        return PAMD_EINVAL;
    }
    if (mol_id < 0 || mol_id > 0xffffff) {
        set_last_error("mol_id must be 0..2^24-1");
        return PAMD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* base = nullptr;
    int rc = scratch_address(s, &base);
    if (rc) return rc;
    unsigned long long* C = reinterpret_cast<unsigned long long*>(base + kOffC);
    unsigned long long* blk_w = reinterpret_cast<unsigned long long*>(base + kOffBlkW);
    double* blk_e = reinterpret_cast<double*>(base + kOffBlkE);
    DevScalars* scal = reinterpret_cast<DevScalars*>(base + kOffScal);

    const int nblk = (int)((R + 1023) / 1024);
    const double dbeta = 1.0 / (kBoltzmann * T_next) - 1.0 / (kBoltzmann * T_prev);
    int bits = 0;
    while ((1LL << bits) < R) ++bits;
    const double two_s = ldexp(1.0, 63 - bits);
    static const ExpCoef cf = inverse_factorials();
    int grid = (int)((R + 255) / 256);

    // the scratch keeps the previous call's contents: the scalars (running
    // sums among them) and the output counts must start from zero
    reset_scalars_kernel<<<1, 1, 0, s>>>(scal);
    cudaError_t e = cudaMemsetAsync(counts_dev, 0, sizeof(int32_t) * (size_t)R, s);
    if (e != cudaSuccess) {
        set_last_error(std::string("clearing counts: ") + cudaGetErrorString(e));
        return PAMD_ECUDA;
    }
    amax_kernel<<<nblk, 256, 0, s>>>(E_dev, R, dbeta, blk_e, nullptr);
    max_top_kernel<<<1, 1024, 0, s>>>(blk_e, nblk, scal);
    // W is written into C and scanned in place, block by block
    weights_kernel<<<nblk, 256, 0, s>>>(E_dev, R, dbeta, two_s, scal, cf, C, blk_w, blk_e, nullptr);
    weights_top_kernel<<<1, 256, 0, s>>>(blk_w, blk_e, nblk, R, scal, nullptr);
    scan_local_u64_kernel<<<nblk, 256, 0, s>>>(C, R, blk_w, C, nullptr);
    counts_kernel<<<grid, 256, 0, s>>>(C, R, scal, seed, nullptr, resample_index,
                                       kPurposeResample | ((uint32_t)mol_id << 8), 1, counts_dev,
                                       nullptr);
    if (lnQ_dev) {
        e = cudaMemcpyAsync(lnQ_dev, &scal->lnQ, sizeof(double), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) {
            set_last_error(std::string("ln Q copy: ") + cudaGetErrorString(e));
            return PAMD_ECUDA;
        }
    }
    if (status_dev) {  // 0, or PAMD_ENONFINITE when an energy was NaN or infinite
        e = cudaMemcpyAsync(status_dev, &scal->status, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) {
            set_last_error(std::string("status copy: ") + cudaGetErrorString(e));
            return PAMD_ECUDA;
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("launch: ") + cudaGetErrorString(e));
        return PAMD_ECUDA;
    }
    return PAMD_OK;
}
