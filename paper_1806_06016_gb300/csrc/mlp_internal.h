// mlp_internal.h -- the MLP energy surrogate's host object and the parameter
// blocks of its kernels (mlp.cu, propagate_mlp.cu, mlp_gemm.cu).
#pragma once

#include <cuda_bf16.h>

#include "../../include/pamd_mlp.h"
#include "pamd_internal.h"

namespace pamd {

constexpr int kMlpThreads = 128;

// Activations and workspace of one batch of up to `cap` configurations.
struct MlpWork {
    long long cap = 0;
    bool train = false;
    void* base = nullptr;        // one allocation holding everything below
    __nv_bfloat16* a = nullptr;  // [cap][Pp] normalised features
    __nv_bfloat16* h1 = nullptr; // [cap][H]
    __nv_bfloat16* d2 = nullptr; // [cap][H] w3 * silu'(z2)
    __nv_bfloat16* d1 = nullptr; // [cap][H] (W2^T d2) * silu'(z1)
    float* s1 = nullptr;         // [cap][H] silu'(z1)
    __nv_bfloat16* ga = nullptr; // [cap][Pp] de/da (BF16: it feeds an FP32 sum of per-pair terms)
    float* part = nullptr;       // [cap][nparts] partial sums of w3 . h2
    // training only
    float* z1 = nullptr;         // [cap][H]
    float* z2 = nullptr;
    float* s2 = nullptr;
    float* w2d2 = nullptr;       // W2^T d2
    float* zd1 = nullptr;        // tangent pass
    float* zd2 = nullptr;
    float* h1b = nullptr;        // dL/dh1
    float* t0 = nullptr;         // per-sample contributions to the bias / w3 gradients
    float* t1 = nullptr;
    float* t2 = nullptr;
    __nv_bfloat16* nu_a = nullptr;  // [cap][Pp]
    __nv_bfloat16* hd1 = nullptr;   // [cap][H]
    __nv_bfloat16* z2b = nullptr;   // [cap][H]
    __nv_bfloat16* A1T = nullptr;   // [H][2cap]  (z1_bar^T | d1^T)
    __nv_bfloat16* B1T = nullptr;   // [Pp][2cap] (a^T | nu_a^T)
    __nv_bfloat16* A2T = nullptr;   // [H][2cap]  (z2_bar^T | d2^T)
    __nv_bfloat16* B2T = nullptr;   // [H][2cap]  (h1^T | hd1^T)
    float* ebar = nullptr;          // [cap]
    double* loss_part = nullptr;    // [cap]
};

// Configurations read with strides: element (m, atom i, coordinate c) at
// x[m * s_cfg + i * s_atom + c * s_coord], sample m taken as idx[m] if idx.
struct ConfigView {
    const float* x;
    long long s_cfg;
    int s_atom, s_coord;
    const int32_t* idx;
};

struct FeatArgs {
    ConfigView cv;
    int M, N, P, Pp;
    const ushort2* pairs;    // [Pp] (i, j)
    const float* mu;         // [Pp]
    const float* inv_sd;     // [Pp]
    __nv_bfloat16* a;        // [M][Pp]
    __nv_bfloat16* aT;       // [Pp][ldt] or null
    int ldt;
};

struct ForceArgs {
    ConfigView cv;
    int M, N, P, Pp, nparts;
    const ushort2* pairs;    // [Pp] (i, j)
    const __nv_bfloat16* ga; // [M][Pp]
    const float* part;       // [M][nparts]
    const float* inv_sd;
    const float* b3;         // device scalar
    double sigma_E, mu_E;
    double* E;               // [M] or null
    float* F;                // [M][N][3] or null
};

struct LossArgs {
    ConfigView cv;
    const double* E_ref;     // [n] (indexed like x)
    const float* F_ref;      // [n][N][3]
    int M, N, P, Pp, nparts;
    const ushort2* pairs;    // [Pp] (i, j)
    const __nv_bfloat16* ga;
    const float* part;
    const float* inv_sd;
    const float* b3;         // device scalar
    double mu_E, sigma_E, lam;
    __nv_bfloat16* nu_a;     // [M][Pp]
    __nv_bfloat16* nu_aT;    // [Pp][ldt], column offset included
    int ldt;
    float* ebar;             // [M]
    double* loss_part;       // [M]
};

// Surrogate BAOAB kernel (propagate_mlp.cu).  mode 0: features of the
// incoming state; 1: one step (closing half kick of the previous step when
// step_index > 0, then B A O A, then the features of the new positions);
// 2: closing half kick (theta > 0), energy, kinetic energy, R_g, forces.
struct MlpStepParams {
    float* state;            // [R][6][Np]
    double* E;
    double* ke;
    double* rg;
    float* fout;             // [R][3][Np] or null
    const float* masses;     // [Np]
    int* status;
    const uint32_t* dev_counters;
    long long R;
    int N, Np, P, Pp, nparts;
    int mode, step_index, theta;
    const int* step_index_dev;  // mode 1 inside a captured loop: the step index in device memory
    const __nv_bfloat16* ga;
    const float* part;
    const float* mu;
    const float* inv_sd;
    const ushort2* pairs;
    __nv_bfloat16* a;
    const float* b3;         // device scalar
    double sigma_E, mu_E;
    float hdt, c1, c2kT;
    unsigned long long seed;
    uint32_t step0;
    uint32_t purpose_mol;
};
cudaError_t launch_mlp_step(const MlpStepParams& p, cudaStream_t s);
size_t mlp_step_smem(int N, int Np, int Pp);

}  // namespace pamd

struct pamd_mlp {
    int N = 0, P = 0, Pp = 0, H = 0, nparts = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool broken = false;
    long long launches = 0;
    // FP32 master parameters: W1 [H][Pp] (columns >= P zero), b1 [H],
    // W2 [H][H], b2 [H], w3 [H], b3 (one float, padded to 4)
    size_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, ow3 = 0, ob3 = 0, n_params = 0;
    float* params = nullptr;
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    long long adam_t = 0;
    float* mu = nullptr;         // [Pp]
    float* sd = nullptr;         // [Pp]
    float* inv_sd = nullptr;     // [Pp]
    double mu_E = 0.0, sigma_E = 1.0;
    __nv_bfloat16* W1b = nullptr;   // [H][Pp]
    __nv_bfloat16* W1Tb = nullptr;  // [Pp][H]
    __nv_bfloat16* W2b = nullptr;   // [H][H]
    __nv_bfloat16* W2Tb = nullptr;  // [H][H]
    ushort2* pairs = nullptr;       // [Pp]
    int* status = nullptr;
    double* scratch = nullptr;      // [4] loss and statistics
    void* base = nullptr;           // allocation holding the members above
    pamd::MlpWork w;
    long long work_gen = 0;         // incremented whenever the workspace is reallocated
    int* loop_ctr = nullptr;        // step index of a captured MD loop (device int)
    cudaStream_t body_stream = nullptr;  // captures the body of that loop
};

namespace pamd {
// Queue the surrogate's energy and force evaluation (features, four GEMMs)
// and the step kernels of theta BAOAB steps on stream s; used by the
// propagate launcher of a context with a force model.
int mlp_propagate(pamd_mlp* m, float* state, double* E, double* ke, double* rg, float* fout,
                  const float* masses, int* status, const uint32_t* dev_counters, long long R,
                  int Np, int theta, double dt, double T, double gamma, unsigned long long seed,
                  uint32_t step0, uint32_t purpose_mol, cudaStream_t s, long long* launches);
int mlp_ensure_work(pamd_mlp* m, long long M, bool train);
// The theta steps of mlp_propagate as one WHILE node of the graph being
// captured on stream s (needs mlp_prepare_capture).
int mlp_loop_captured(pamd_mlp* m, MlpStepParams p, int theta, int M, cudaStream_t s, int* status);
// Everything a capture of mlp_propagate needs allocated or configured before
// the capture starts (loop counter, body stream, tensor-core GEMM set-up).
int mlp_prepare_capture(pamd_mlp* m);
// GEMMs of one evaluation of the M configurations whose features are in
// m->w.a: layers 1 and 2 (energy partial sums), and with forces the two
// backward products (de/da in m->w.ga).  Tensor-core timeouts are recorded
// in *status.
int mlp_gemms(pamd_mlp* m, int M, bool forces, cudaStream_t s, int* status);
}  // namespace pamd
