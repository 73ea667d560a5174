// pamd_internal.h -- definitions shared by libpamd's translation units
// (host context, kernel parameter blocks, launcher entry points).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pamd.h"

namespace pamd {

constexpr double kBoltzmann = 0.008314462618;  // kJ/mol/K

// Largest block of the single-replica propagate kernel with B atoms per lane
// (its launch bounds): 5 atoms per lane run 128-thread blocks, three per SM.
__host__ __device__ constexpr int prop_max_threads(int B) { return B == 5 ? 128 : 256; }
constexpr double kCoulomb = 138.935458;        // kJ mol^-1 nm e^-2
constexpr int kNumBins = 64;                   // family bins for jackknife errors
constexpr uint32_t kPurposeNoise = 0u, kPurposeInit = 1u, kPurposeResample = 2u;
constexpr int kMaxColors = 64;                 // colour classes per bonded term type
constexpr size_t kPairTableMaxBytes = 48 * 1024;  // largest pair-parameter table kept in shared memory

// Bonded terms as laid out in the topology blob (16-byte aligned records).
struct BondRec { int32_t i, j; float r0, k; };
struct AngleRec { int32_t i, j, k, pad; float t0, kk, pad1, pad2; };
struct DihRec { int32_t i, j, k, l; float kd, n, cos_ph, sin_ph; };
struct Pair14Rec { int32_t i, j; float s_lj, s_c; };

// Byte layout of the per-molecule table the propagate kernel copies to
// shared memory once per CTA.  All offsets are multiples of 16.
struct TopoLayout {
    int n_atoms, n_pad;        // N and Np = round_up(N, 4) (global state stride)
    int lanes, per_lane;       // L lanes per replica (1..32), B atoms per lane (1..8)
    int block_stride;          // B rounded up to odd (smem atoms per lane block)
    int nk;                    // L * block_stride smem atom slots
    int off_params;            // float4 [nk]: {sigma/2, sqrt(24 eps), q sqrt(k_e), 1/m}
    int off_masks;             // uint64 [(L/2+1) * L]: excluded and scaled 1-4 pairs per tile
    int off_m14;               // uint64 [(L/2+1) * L]: the scaled 1-4 pairs among them
    int far_masks;             // 1 if a tile at ring step t >= 2 has a masked pair
    int std_chain;             // chain whose excluded pairs are exactly (i, i+1) and (i, i+2)
    int off_bonds, n_bonds;
    int off_angles, n_angles;
    int off_dihs, n_dihs;
    int off_p14, n_p14;
    int off_colors;            // int32 [4][kMaxColors+1] colour start offsets
    int n_colors[4];           // bonds, angles, dihedrals, 1-4 pairs
    int chain;                 // 1: linear-chain bonded layout (B >= 3)
    int off_cbond;             // chain: float2 [N-1] {r0, k} of bond (d, d+1)
    int off_cangle;            // chain: float2 [N-2] {theta0, k} of angle (d, d+1, d+2)
    int off_cdih;              // chain: float4 [N-3] {k, n, cos phase, sin phase} of (d..d+3)
    float s14_lj, s14_c;       // chain: 1-4 scale factors
    int paired;                // launch: 1 = two replicas per lane group (packed FP32x2)
    int packed;                // launch: 1 = own-atom pairs in packed FP32x2 (chain, B = 3..8)
    int ptab, off_ptab;        // chain: 1 if float4 [L/2][B][B][L] {sigma_ij^2, eps_ij, qq_ij, 0}
                               //   of the half-ring tiles follows (entry ((t-1) B^2 + b B + a) L + g)
    int bytes;                 // total, multiple of 16
};

// Shared memory of the packed-pair propagate kernel: the topology table
// without the pair-parameter table; the duplicated mixing parameters
// {sigma/2, sigma/2, sqrt(24 eps), sqrt(24 eps)} (float4) and the integrator
// constants {dt/(2m), noise scale} (float2) of the nk atom slots; then per
// replica slot posA[nk] {x,x,y,y}, posB[nk] {z,z,q,q} and vel[nk] {vx,vy,vz,0}
// (+1 float4 to spread the replicas over the banks).
__host__ __device__ inline int x2_topo_bytes(const TopoLayout& lay) {
    return lay.ptab ? lay.off_ptab : lay.bytes;
}
__host__ __device__ inline int x2_table_f4(const TopoLayout& lay) { return lay.nk + (lay.nk + 1) / 2; }
__host__ __device__ inline int x2_slot_f4(const TopoLayout& lay) { return 3 * lay.nk + 1; }

struct PropParams {
    const float* state_in;     // [R][6][Np]
    float* state_out;          // may equal state_in
    double* E;                 // [R]
    double* ke;                // [R]
    double* rg;                // [R]
    float* fout;               // [R][3][Np] or null (force dump)
    const float* masses;       // [Np] (0 for padding)
    const unsigned char* topo; // TopoLayout.bytes
    int* status;               // [2]: code, replica
    const uint32_t* dev_counters;  // null, or {step, resample index} base
    const uint32_t* live;      // null, or the live size of a variable population (R = capacity)
    TopoLayout lay;
    long long R;
    int theta;
    float hdt;                 // dt / 2
    float c1;                  // exp(-gamma dt)
    float c2kT;                // sqrt((1 - c1^2) k_B T)
    unsigned long long seed;
    uint32_t step0;            // added to dev_counters[0] (or absolute when null)
    uint32_t purpose_mol;      // mol << 8
};

// Device tables of the all-FP64 mode (PAMD_PREC_FP64); pointers into one
// device allocation.
struct TopoF64 {
    int n_atoms;
    const double* sigma_half;   // [N]
    const double* epsilon;      // [N]
    const double* charge;       // [N]
    const double* inv_mass;     // [N]
    const double* x0;           // [3][Np] recentred start geometry
    const unsigned char* kind;  // [N][N]: 0 full, 1 excluded, 2 scaled 1-4 pair
    double s14_lj, s14_c;
    int n_bonds, n_angles, n_dihs;
    const int* bond;            // [nb][2]
    const double* bond_p;       // [nb][2] r0, k
    const int* angle;           // [na][3]
    const double* angle_p;      // [na][2] theta0, k
    const int* dih;             // [nd][4]
    const double* dih_p;        // [nd][4] k, n, cos phase, sin phase
};

struct PropF64Params {
    double* state;              // [R][6][Np], updated in place
    double* E;
    double* ke;
    double* rg;
    double* fout;               // [R][3][Np] or null
    int* status;
    const uint32_t* dev_counters;
    TopoF64 top;
    int n_pad;
    long long R;
    int theta;
    double dt, T, gamma;
    unsigned long long seed;
    uint32_t step0;
    uint32_t purpose_mol;
};

// Batched propagate (propagate_batch.cu): one launch for many molecules.
constexpr int kBatchThreads = 128;  // 4 warps per block
constexpr int kMaxBatchMols = 64;
struct BatchParams {
    int n_items;
    const int4* items;  // {molecule, first replica, end replica, 0}
    int* queue;         // work counter, zero at launch
    PropParams mol[kMaxBatchMols];
};

struct DevScalars {
    double m;                  // max a_j
    double S;                  // sum exp(a_j - m)
    double lnQ;
    double sum_lnQ;
    unsigned long long C_total;
    int max_copies;
    int status;                // PAMD status code set by kernels (0 = ok)
    int bad_replica;
    int pad_;
    long long R_new;           // size of the population a resampling produces
};

struct Buffers {
    float* state = nullptr;
    float* state_alt = nullptr;
    double* E = nullptr;
    double* E_alt = nullptr;
    int32_t* fam = nullptr;
    int32_t* fam_alt = nullptr;
    double* ke = nullptr;
    double* rg = nullptr;
    float* masses = nullptr;
    unsigned char* topo = nullptr;
    float* x0 = nullptr;          // [3][Np] recentred start geometry
    // resampling scratch
    unsigned long long* W = nullptr;
    unsigned long long* C = nullptr;
    int32_t* cnt = nullptr;
    int32_t* cnt_incl = nullptr;
    unsigned long long* blk_u64 = nullptr;
    double* blk_f64 = nullptr;
    int32_t* blk_i32 = nullptr;
    unsigned char* flags = nullptr;
    double* obs_part = nullptr;
    DevScalars* scal = nullptr;
    uint32_t* counters = nullptr;
    pamd_obs* obs = nullptr;      // [obs_cap]
    float* fout = nullptr;        // [R][3][Np] allocated on demand
};

struct GraphKey {
    int K = -1, theta = -1, resample = -1;
    double dt = 0;
    std::vector<double> T;
    const double* rec = nullptr;  // energy recording target (pamd_record_energies)
    int rec_rows = 0;
    // force model: which one, the generation of its workspace, its energy scale
    const void* model = nullptr;
    long long model_gen = 0;
    double mu_E = 0, sigma_E = 0;
    bool operator==(const GraphKey& o) const {
        return K == o.K && theta == o.theta && resample == o.resample && dt == o.dt && T == o.T &&
               rec == o.rec && rec_rows == o.rec_rows && model == o.model && model_gen == o.model_gen &&
               mu_E == o.mu_E && sigma_E == o.sigma_E;
    }
};

}  // namespace pamd

namespace pamd {
// Copy of the caller's topology, kept so that the launch shape can be
// re-chosen (autotuning) after pamd_init returned.
struct HostTopology {
    int32_t n_atoms = 0;
    std::vector<double> mass, charge, sigma, epsilon, x0, bond_r0, bond_k, angle_t0, angle_k,
        dih_k, dih_phase;
    std::vector<int32_t> bond, angle, dihedral, dih_n, excl, pair14;
    double scale14_lj = 0, scale14_coul = 0;
    void assign(const pamd_topology* t) {
        auto cp = [](auto& v, const auto* p, size_t n) { v.assign(p, p + (p ? n : 0)); };
        const size_t N = (size_t)t->n_atoms;
        n_atoms = t->n_atoms;
        cp(mass, t->mass, N); cp(charge, t->charge, N); cp(sigma, t->sigma, N);
        cp(epsilon, t->epsilon, N); cp(x0, t->x0, 3 * N);
        cp(bond, t->bond, 2 * (size_t)t->n_bonds); cp(bond_r0, t->bond_r0, (size_t)t->n_bonds);
        cp(bond_k, t->bond_k, (size_t)t->n_bonds);
        cp(angle, t->angle, 3 * (size_t)t->n_angles); cp(angle_t0, t->angle_t0, (size_t)t->n_angles);
        cp(angle_k, t->angle_k, (size_t)t->n_angles);
        cp(dihedral, t->dihedral, 4 * (size_t)t->n_dihedrals); cp(dih_n, t->dih_n, (size_t)t->n_dihedrals);
        cp(dih_k, t->dih_k, (size_t)t->n_dihedrals); cp(dih_phase, t->dih_phase, (size_t)t->n_dihedrals);
        cp(excl, t->excl, 2 * (size_t)t->n_excl); cp(pair14, t->pair14, 2 * (size_t)t->n_pair14);
        scale14_lj = t->scale14_lj;
        scale14_coul = t->scale14_coul;
    }
    pamd_topology view() const {
        pamd_topology t{};
        t.n_atoms = n_atoms;
        t.mass = mass.data(); t.charge = charge.data(); t.sigma = sigma.data();
        t.epsilon = epsilon.data(); t.x0 = x0.data();
        t.n_bonds = (int32_t)bond_r0.size(); t.bond = bond.data(); t.bond_r0 = bond_r0.data();
        t.bond_k = bond_k.data();
        t.n_angles = (int32_t)angle_t0.size(); t.angle = angle.data(); t.angle_t0 = angle_t0.data();
        t.angle_k = angle_k.data();
        t.n_dihedrals = (int32_t)dih_k.size(); t.dihedral = dihedral.data(); t.dih_n = dih_n.data();
        t.dih_k = dih_k.data(); t.dih_phase = dih_phase.data();
        t.n_excl = (int32_t)(excl.size() / 2); t.excl = excl.data();
        t.n_pair14 = (int32_t)(pair14.size() / 2); t.pair14 = pair14.data();
        t.scale14_lj = scale14_lj;
        t.scale14_coul = scale14_coul;
        return t;
    }
};
}  // namespace pamd

struct pamd_mlp;

struct pamd_ctx {
    long long R = 0;
    int N = 0, Np = 0;
    pamd::TopoLayout lay{};
    int warps_per_block = 4;
    int rpb = 0;               // replicas per block
    int grid_prop = 0;         // persistent grid size for propagate
    int num_sms = 0;
    int precision = PAMD_PREC_MIXED;
    double gamma = 1.0;
    unsigned long long seed = 0;
    int mol = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* (*dev_alloc)(size_t, void*) = nullptr;
    void (*dev_free)(void*, void*) = nullptr;
    void* alloc_user = nullptr;
    pamd::Buffers b;
    std::vector<void*> allocations;
    int n_blk = 0;             // blocks of the 1024-element scans
    int obs_cap = 0;
    uint32_t step = 0;
    uint32_t resample_index = 0;
    long long launches = 0;
    long long graph_kernels = 0;  // kernel launches inside the cached anneal graph
    bool broken = false;
    cudaGraphExec_t graph_exec = nullptr;
    pamd::GraphKey graph_key;
    bool cur_is_alt = false;   // population currently in state_alt
    std::vector<double> host_mass;
    pamd::HostTopology host_top;
    int lanes_req = 0;
    size_t topo_cap = 0;          // bytes allocated for the device topology table
    pamd::TopoF64 top64{};        // all-FP64 mode tables (precision == PAMD_PREC_FP64)
    // batch context (pamd_init_batch): one sub-context per molecule
    std::vector<pamd_ctx*> subs;
    int4* items = nullptr;        // device work lists of the batched propagate, group by group
    int n_items = 0;
    int* queue = nullptr;         // device work counters, one per group
    struct BatchGroup {           // molecules sharing one atoms-per-lane count B and pair arithmetic
        int B, first_item, n_items, grid;
        size_t smem;
        bool packed;
    };
    std::vector<BatchGroup> groups;
    std::vector<cudaStream_t> group_streams;  // one per group (launches overlap)
    std::vector<cudaEvent_t> group_events;    // completion of each group's launch
    cudaEvent_t fork_event = nullptr;         // the groups start after this
    unsigned char* top64_blob = nullptr;
    pamd_mlp* mlp = nullptr;      // force model replacing the exact forces (pamd_set_force_model)
    double* rec_E = nullptr;      // caller's [rec_rows][R] energy record of pamd_anneal, or null
    int rec_rows = 0;
    void* ov_work = nullptr;      // scratch of the adaptive temperature step (allocated on first use)
    int resample_rule = PAMD_RESAMPLE_MULTINOMIAL;
    int pair_arith = PAMD_PAIRS_AUTO;  // pamd_options.pair_arith
    // variable population (nearest-integer or Poisson resampling): R is the
    // capacity of the buffers, R_target the size the copy numbers aim at, and
    // the live size is device counter word 2
    bool variable = false;
    long long R_target = 0;
};

namespace pamd {

// propagate kernels, one function per atoms-per-lane count B (two per
// translation unit).  With p == null they only report how many blocks of that
// shape fit on one SM.
#define PAMD_DECLARE_PROPAGATE(B)                                                            \
    cudaError_t propagate_b##B(const PropParams* p, bool chain, bool table, int warps, int grid, \
                               size_t smem, cudaStream_t s, int* blocks_per_sm);
PAMD_DECLARE_PROPAGATE(1)
PAMD_DECLARE_PROPAGATE(2)
PAMD_DECLARE_PROPAGATE(3)
PAMD_DECLARE_PROPAGATE(4)
PAMD_DECLARE_PROPAGATE(5)
PAMD_DECLARE_PROPAGATE(6)
PAMD_DECLARE_PROPAGATE(7)
PAMD_DECLARE_PROPAGATE(8)
#undef PAMD_DECLARE_PROPAGATE
// kernels with the pair arithmetic in packed FP32x2 (own atoms in register
// pairs; linear chains, 3..8 atoms per lane)
cudaError_t propagate_x2_dispatch(int B, const PropParams* p, int warps, int grid, size_t smem,
                                  cudaStream_t s, int* blocks_per_sm);
// launch variants of the single-molecule propagate kernel
constexpr int kVarScalar = 0, kVarPaired = 1, kVarPacked = 2;
constexpr int kPackedMaxThreads = 128;  // block-size cap of the packed-pair kernel
// paired kernels (two replicas per lane group), 2..4 atoms per lane
cudaError_t propagate2_b2(const PropParams* p, bool chain, int warps, int grid, size_t smem,
                          cudaStream_t s, int* blocks_per_sm);
cudaError_t propagate2_b3(const PropParams* p, bool chain, int warps, int grid, size_t smem,
                          cudaStream_t s, int* blocks_per_sm);
cudaError_t propagate2_b4(const PropParams* p, bool chain, int warps, int grid, size_t smem,
                          cudaStream_t s, int* blocks_per_sm);

// BF16 tensor-core GEMM (mlp_gemm.cu): C = A . B^T with A [M x K], B [N x K]
// row-major BF16 (K contiguous), FP32 accumulation, and a fused epilogue on
// z = acc (+ bias[n]):
//   kEpiStore  C = z, Cb = bf16(z)                       (each output optional)
//   kEpiSilu   C = z, Cs = silu'(z), Cb = bf16(silu(z)), CbT = Cb transposed
//   kEpiHead   C = z, Cs = silu'(z), Cb = bf16(vec[n] silu'(z)), CbT, and
//              part[m * 2 ntiles + 2 tile + h] = sum over the n of half h of
//              the tile of vec[n] silu(z), ntiles = ceil(N / kGemmTileN)
//   kEpiMul    C = z, Cb = bf16(z * mul[m, n]) (mul FP32, leading dim ldc), CbT
enum GemmEpi { kEpiStore = 0, kEpiSilu = 1, kEpiHead = 2, kEpiMul = 3 };
constexpr int kGemmTileN = 256;   // output columns per tile
constexpr int kGemmHeadParts = 2;  // kEpiHead partial sums per tile (part[] has 2 ceil(N / kGemmTileN) columns)
struct GemmArgs {
    const void* A;             // __nv_bfloat16 [M][lda]
    const void* B;             // __nv_bfloat16 [N][ldb]
    float* C;                  // [M][ldc] or null
    float* Cs;                 // [M][ldc] or null
    void* Cb;                  // __nv_bfloat16 [M][ldcb] or null
    void* CbT;                 // __nv_bfloat16 [N][ldt] or null
    const float* bias;         // [N] or null
    const float* vec;          // [N] (kEpiHead)
    const float* mul;          // [M][ldc] (kEpiMul)
    float* part;               // [M][kGemmHeadParts ceil(N / kGemmTileN)] (kEpiHead)
    int* status;               // PAMD status word (timeouts)
    int M, N, K, lda, ldb, ldc, ldcb, ldt, epi;
    int vec_ok;                // set by the launcher: 1 FP32 rows, 2 BF16 rows 16-byte aligned
};
cudaError_t launch_gemm_bf16(const GemmArgs& g, cudaStream_t s);

// Raise the dynamic shared-memory limit of kernel `fn` on the current device
// to at least `bytes` (the attribute belongs to the device's context; the
// largest value asked for so far is kept per kernel and device; thread-safe).
cudaError_t ensure_dyn_smem(const void* fn, size_t bytes);
// the GEMM's once-per-device set-up (kernel attribute, resident clusters) for
// the current device, so that a later launch can be captured in a graph
cudaError_t gemm_prepare_device();

// message returned by pamd_last_error() on this thread (capi.cu)
void set_last_error(const std::string& msg);
// Adaptive temperature step (adaptive.cu): scratch size, argument check and
// the search on device energies E [R]; synchronises s.
size_t overlap_work_bytes(long long R);
int overlap_check_args(long long R, double T_prev, double T_final, double alpha_target);
int overlap_step(cudaStream_t s, const double* E, long long R, double T_prev, double T_final,
                 double alpha_target, void* work, int num_sms, double* T_next, double* alpha_out,
                 long long* launches);

// resampling kernels defined in resample.cu, also launched by noalloc.cu;
// `live`, when not null, holds the live size of a variable population (R is
// then the capacity of the buffers)
__global__ void reset_scalars_kernel(DevScalars* s);
__global__ void amax_kernel(const double* E, long long R, double dbeta, double* blk_max,
                            const uint32_t* live);
__global__ void max_top_kernel(const double* blk_max, int nblk, DevScalars* s);
__global__ void weights_top_kernel(unsigned long long* blk_w, const double* blk_e, int nblk,
                                   long long R, DevScalars* s, const uint32_t* live);
__global__ void scan_local_u64_kernel(unsigned long long* W, long long R,
                                      const unsigned long long* blk_off, unsigned long long* C,
                                      const uint32_t* live);
__global__ void counts_kernel(const unsigned long long* C, long long R, const DevScalars* s,
                              unsigned long long seed, const uint32_t* dev_counters,
                              uint32_t ridx_off, uint32_t purpose, int do_resample, int32_t* cnt,
                              const uint32_t* live);

// resampling / observables / init kernels (resample.cu)
cudaError_t launch_init(pamd_ctx* c, double T0);
cudaError_t launch_resample(pamd_ctx* c, double T_prev, double T_next, int do_resample,
                            const uint32_t* dev_counters, uint32_t resample_offset);
cudaError_t launch_observe(pamd_ctx* c, double T, pamd_obs* dst);
cudaError_t launch_set_counters(pamd_ctx* c, uint32_t step, uint32_t ridx);

// one launch of the batched kernel for atoms-per-lane B (3..7)
cudaError_t launch_propagate_batch(const BatchParams& bp, int B, int grid, size_t smem, cudaStream_t s);
cudaError_t propagate_batch_occupancy(int B, size_t smem, int* blocks_per_sm);
// the same for molecules in the packed FP32x2 layout (propagate_batch_x2.cu)
cudaError_t launch_propagate_batch_x2(const BatchParams& bp, int B, int grid, size_t smem, cudaStream_t s);
cudaError_t propagate_batch_x2_occupancy(int B, size_t smem, int* blocks_per_sm);

// all-FP64 mode (propagate_f64.cu)
cudaError_t launch_propagate_f64(pamd_ctx* c, double* state, double* E, double* ke, double* rg,
                                 int theta, double dt, double T, const uint32_t* dev_ctr,
                                 uint32_t step0, double* fout);
cudaError_t launch_init_f64(pamd_ctx* c, double T0);
cudaError_t launch_gather_f64(pamd_ctx* c, const double* src, double* dst, const double* Ein,
                              double* Eout, const int32_t* fin, int32_t* fout, double vscale);


}  // namespace pamd
