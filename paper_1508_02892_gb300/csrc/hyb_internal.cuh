// hyb_internal.cuh -- device-side state and helpers shared by the kernels and
// the host runtime of the GB300 electron PIC/MCC library (arXiv 1508.02892).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hybrid1d.h"

namespace hyb {

// CODATA 2018 (e and k_B exact)
constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kKb = 1.380649e-23;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kAmu = 1.66053906660e-27;
constexpr double kTwoPi = 6.283185307179586476925286766559;

constexpr int32_t kDeadCell = INT32_MIN;  // cell index of a removed split-mode particle
constexpr int kMaxNodes = HYB_MAX_CELLS + 1;
// Particle kernels split each instance's slots into chunks of kChunk slots;
// prefix arrays hold chunk counts of the running instances.
constexpr int kChunk = 256;

__host__ __device__ __forceinline__ int64_t chunks_of(int64_t n) { return (n + kChunk - 1) / kChunk; }

// Particle store, structure of arrays.  Split mode uses c/o/vxf..; FP64 mode
// uses z/vxd..; id is shared.
struct PartBuf {
    int32_t *c;
    float *o, *vxf, *vyf, *vzf;
    double *z, *vxd, *vyd, *vzd;
    uint64_t *id;
};

// Constants of the field step, formed on the host at admission (the same
// expressions a per-step evaluation would use)
struct FieldK {
    double h, qdt_m, h_m, c_in, c_wall, gs_in, gs_wall;   // split-mode fluid
    double hdt, tfac, inv_ngas_td, inv_qe, inv2dz;        // split-mode transport
    double dt_dz, dt_2dz, h_mion;                         // FP64-mode fluid
    double w_in, w_wall, c_src, inv_dz, half_inv_dz, c_gauss;  // split-mode Poisson
};

// Columns of a transport-table row in the split-mode field kernel: E/N, mu,
// d mu/d(E/N), u, nu, d nu/du and two of padding (rows of 64 bytes)
constexpr int kTabCols = 8;

// Largest cross-section table of a split-mode discharge: the particle step
// stages it with its segment slopes in shared memory (32 bytes an entry)
constexpr int kMaxSplitXs = 4096;

// Everything a kernel needs about one discharge.  Lives in device memory; the
// host writes it at admission and the kernels update the mutable tail.
struct InstDev {
    // ---- constant after admission
    int32_t precision, n_cells, G, ion_model, n_xs, n_tab, eedf_bins, pad0;
    int64_t capacity;
    double L, dz, dt, ngas, w, m_gas, m_ion, qm, nu_max, p_max, n_floor, bin_w;
    double e_lo, e_hi, inv_dlog, e_exc, e_iz, two_mM, gamma_see, see_speed;
    double v_rf, f_rf, v_dc, mu_const, kT_gas;
    double inv_gm1;  // 1 / (G - 1)
    FieldK fk;
    uint32_t seed_lo, seed_hi;
    // FP32 copies for the split-mode electron kernel
    float f_dt_dz, f_qm_dt, f_half_m_q, f_two_q_m, f_pmax, f_e_lo, f_e_hi, f_inv_e_lo, f_inv_dlog;
    float f_e_exc, f_e_iz, f_two_mM, f_bin_inv;
    // tables (device)
    const double *xs;    // [n_xs][4] {E, sigma_el, sigma_exc, sigma_ion}
    const float4 *xsf;   // [n_xs] {E, N sigma_el/nu_max, N sigma_exc/nu_max, N sigma_ion/nu_max}
    const double *tab;   // [n_tab][4] {E/N (Td), mu, nu, u = mu E}
    const double *tabx;  // [n_tab][kTabCols] the same with segment slopes (the split-mode field kernel's layout)
    const float *tabf;   // [2][n_tab] FP32 copies of the E/N and u columns
    // particles (double-buffered for the cell sort)
    PartBuf buf[2];
    // grids, n_nodes entries
    double *ni, *gam, *phi, *E, *ne, *gsrc;
    float *Ef;
    double *dep_n, *dep_e, *s_iz;                     // per-step sums, cleared by the field kernel
    double *acc_ne, *acc_ni, *acc_gi, *acc_wn, *acc_we; // time sums
    unsigned long long *eedf;                         // eedf_bins + 1 counts
    int32_t *cell_cnt;                                // n_cells + 1, sort scratch
    // ---- mutable
    int32_t active, cur;
    int64_t step, target_step;
    unsigned long long n_slots;       // slots in use (atomic append)
    int64_t n_slots_step;             // slots processed by the current step
    int64_t n_samples;
    double flux_in[2];
    unsigned long long ctr[14];       // births_iz, see0, see1, loss0, loss1, el, exc, iz, null, clamps, pushes, rec,
                                      // Penning births, pooling births
    int64_t n_base;                   // live count = n_base + births - losses
    unsigned int status;
    int32_t init_pending;             // field kernel runs in initial-solve mode
    // power control (Eq. 2.9); v_rf above is the current amplitude
    double pw_target, pw_alpha;       // P0 per m^2 (0: fixed amplitude), alpha
    double pw_acc, pw_last;           // sum of V J dt in the running period; P_abs of the last one
    int64_t pw_steps, pw_count, pw_periods;
    unsigned long long pw_loss0;      // electrons absorbed at z = 0 up to the last step
    // electron-ion recombination (Sec. II.D)
    int32_t rec_on, pad1;
    double rec_svmax;                 // bound of sigma_rec v over the table
    const double *xs_rec;             // [n_xs] sigma_rec (FP64 mode)
    const float *xs_recf;             // [n_xs] sigma_rec / rec_svmax (split mode)
    float *nif;                       // [G] n_i / max n_i, written by the field kernel (split mode)
    double rec_numax, rec_pmax;       // max n_i * rec_svmax and 1 - exp(-rec_numax dt), for the next step
    float f_rec_pmax, pad2;
    // kinetic ions (HYB_ION_KINETIC): the ion population lives in a second
    // descriptor of this layout (particles in the batch's precision, its own
    // sort buffers and counters) that points back to the electron one
    InstDev *ion;                     // electron descriptor: its ions (NULL: fluid ions)
    InstDev *elec;                    // ion descriptor: its electrons
    double *dep_ni, *dep_gi;          // per-step CIC sums of the ions: count and v_z
    double mi_red, nu_max_i, p_max_i, vt_gas;
    // FP32 copies for the split-mode ion kernel: (e/M) dt, N, 0.5 M_r / e,
    // the collision bound, P_max, gas thermal speed, M/(M+m), m/(M+m), and
    // N Q_m g in the limit g -> 0
    float fi_qm_dt, fi_ngas, fi_half_mr_q, fi_numax, fi_pmax, fi_vt, fi_cm_a, fi_cm_b, fi_nu0, pad4;
    // metastables and the ionization they cause (Sec. II.D)
    int32_t met_on, pad3;
    double met_D, met_kp, met_kq;     // D, R_P n_N, R_pool
    double met_rp, met_nn;            // R_P and n_N
    double met_sp[2];                 // speeds of Penning and pooling electrons
    double gamma_met;
    double *met, *s_met, *acc_met;    // [G] n_m, this step's CIC excitation sums, time sum of n_m
    double flux_met[2];               // metastables into each wall in the last step, m^-2 s^-1
    unsigned long long ion_loss_prev[2];
};

enum { C_BIRTH_IZ = 0, C_SEE0, C_SEE1, C_LOSS0, C_LOSS1, C_EL, C_EXC, C_IZ, C_NULL, C_CLAMP, C_PUSH, C_REC, C_PEN, C_POOL };

// ------------------------------------------------------------ self-checks
// Every dynamic index of the kernels is guarded: the first failed guard of a
// translation unit is recorded (site, index, bound) and the access is skipped.
// The guards cost a compare each; the recording path is out of line.
static __device__ unsigned long long g_hyb_check[3];
__device__ __noinline__ static bool hyb_check_fail(int site, long long a, long long b)
{
    if (atomicCAS(&g_hyb_check[0], 0ull, (unsigned long long)site) == 0ull) {
        g_hyb_check[1] = (unsigned long long)a;
        g_hyb_check[2] = (unsigned long long)b;
    }
    return false;
}
#define HYB_CHECK(cond, site, a, b) ((cond) ? true : hyb_check_fail((site), (long long)(a), (long long)(b)))

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Draw `call` of particle
// `id` at step `step` in a discharge seeded (seed_lo, seed_hi) is the
// generator's block at counter (step, id_lo, call, id_hi) under key (seed_lo,
// seed_hi).  The key is the same for every particle of a discharge, so a
// thread's round keys are shared by all the draws it forms (and stay out of
// the per-particle instruction stream), and the words the first round
// multiplies (step and call) are the same for every particle: PhiloxPre holds
// the products of the step and the key.
struct PhiloxPre {
    uint32_t hi0, lo0;  // 0xD2511F53 * step, high and low words
    uint2 key;          // (seed_lo, seed_hi)
};

__device__ __forceinline__ PhiloxPre philox_pre(uint32_t step, uint32_t seed_lo, uint32_t seed_hi)
{
    return PhiloxPre{__umulhi(0xD2511F53u, step), 0xD2511F53u * step, make_uint2(seed_lo, seed_hi)};
}

// the state after the first round (the call's products fold to constants
// where `call` is a literal)
__device__ __forceinline__ uint4 philox_first(const PhiloxPre &pre, uint64_t id, uint32_t call)
{
    return make_uint4(__umulhi(0xCD9E8D57u, call) ^ (uint32_t)id ^ pre.key.x, 0xCD9E8D57u * call,
                      pre.hi0 ^ (uint32_t)(id >> 32) ^ pre.key.y, pre.lo0);
}

// round r (1..9) of the later rounds: the key bumped r times by the Weyl
// constants, then the S-box
__device__ __forceinline__ void philox_round(uint4 &c, uint2 kr)
{
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ kr.x, lo1, hi0 ^ c.w ^ kr.y, lo0);
}

__device__ __forceinline__ uint2 philox_round_key(uint2 k, uint32_t r)
{
    return make_uint2(k.x + 0x9E3779B9u * r, k.y + 0xBB67AE85u * r);
}

// Philox4x32-10 of counter (step, id_lo, call, id_hi) under key (seed_lo, seed_hi)
__device__ __forceinline__ uint4 draw_pre(const PhiloxPre &pre, uint64_t id, uint32_t call)
{
    uint4 c = philox_first(pre, id, call);
#pragma unroll
    for (uint32_t r = 1; r < 10; ++r) philox_round(c, philox_round_key(pre.key, r));
    return c;
}

__device__ __forceinline__ uint4 draw(uint64_t id, uint32_t step, uint32_t seed_lo, uint32_t seed_hi, uint32_t call)
{
    return draw_pre(philox_pre(step, seed_lo, seed_hi), id, call);
}

// the same draw for N particles at once, the rounds interleaved across them
template <int N>
__device__ __forceinline__ void draw_n(const PhiloxPre &pre, const uint64_t *ids, uint32_t call, uint4 *out)
{
#pragma unroll
    for (int j = 0; j < N; ++j) out[j] = philox_first(pre, ids[j], call);
#pragma unroll
    for (uint32_t r = 1; r < 10; ++r) {
        const uint2 kr = philox_round_key(pre.key, r);
#pragma unroll
        for (int j = 0; j < N; ++j) philox_round(out[j], kr);
    }
}

// (k + 1/2) 2^-23 from the top 23 bits: the same value in float and double.
// In float it is formed without a conversion: the bits of 1 + k 2^-23 less
// 1 - 2^-24 (both exact, and so is their difference).
__device__ __forceinline__ float u01f_bits(uint32_t x) { return __uint_as_float((x >> 9) | 0x3F800000u); }
__device__ __forceinline__ float u01f(uint32_t x) { return u01f_bits(x) - 0.999999940395355224609375f; }
__device__ __forceinline__ double u01d(uint32_t x) { return ((double)(x >> 9) + 0.5) * 1.1920928955078125e-07; }

// SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t child_id(uint64_t parent, uint32_t step)
{
    return mix64(parent ^ ((uint64_t)step * 0x9E3779B97F4A7C15ull)) | (1ull << 63);
}

__host__ __device__ __forceinline__ uint64_t see_id(int wall, uint32_t step, uint32_t k)
{
    return (1ull << 62) | ((uint64_t)wall << 60) | ((uint64_t)step << 20) | (uint64_t)k;
}

// ------------------------------------------------------- launch helpers
// Work decomposition shared by the particle kernels: prefix[i]..prefix[i+1]
// are instance i's chunks of kChunk slots; each block takes a contiguous run
// of chunks.

// Chunk prefix over the running instances, computed by all threads of one
// block (blockDim >= n_max <= HYB_MAX_INSTANCES); s_buf holds n_max int64.
// Reads other blocks' writes, so the caller must order them (kernel boundary
// or fence + ticket).
__device__ __forceinline__ void block_chunk_prefix(InstDev *insts, int n_max, int64_t *prefix, int64_t *s_buf)
{
    const int t = threadIdx.x;
    if (t < n_max) {
        const volatile InstDev *K = &insts[t];
        s_buf[t] = K->active ? chunks_of(K->n_slots_step) : 0;
    }
    __syncthreads();
    for (int d = 1; d < n_max; d <<= 1) {
        int64_t v = 0;
        if (t < n_max && t >= d) v = s_buf[t - d];
        __syncthreads();
        if (t < n_max) s_buf[t] += v;
        __syncthreads();
    }
    if (t == 0) prefix[0] = 0;
    if (t < n_max) prefix[t + 1] = s_buf[t];
}

// Opt a kernel in to all the dynamic shared memory a block may have beside
// its static shared memory (the opt-in limit counts both)
template <typename Kern>
inline void allow_max_dynamic_smem(Kern kernel)
{
    int dev = 0, optin = 0;
    cudaFuncAttributes a;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&a, (const void *)kernel) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (cudaFuncSetAttribute((const void *)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)a.sharedSizeBytes) != cudaSuccess)
        cudaGetLastError();
}

struct LaunchCfg {
    int grid, block;
    size_t smem;
    int ppt;  // particles per thread of the default split-mode electron step (2 or 4)
};

// electron kernels (hyb_electron.cu)
cudaError_t launch_electron_step(InstDev *inst, int n_max, const int64_t *prefix, int precision, LaunchCfg cfg,
                                 cudaStream_t s,
                                 bool chem = false, bool kin = false);
// kinetic ions (hyb_ion.cu): initial load, the per-step snapshot prefix over a
// lane's ion descriptors, and the ion step (mode 0) or deposit alone (mode 1)
cudaError_t launch_load_ions(InstDev *ion, int64_t n, cudaStream_t s);
double swarm_nu_bound(double ngas, double m_red, double eps_max);
cudaError_t launch_ion_prefix(InstDev *ions, int n_max, int64_t *prefix, cudaStream_t s);
cudaError_t launch_ion_step(InstDev *ions, int n_max, const int64_t *prefix, int mode, int grid, int max_nodes,
                            int precision, cudaStream_t s);
void configure_ion_kernels();
void read_checks_ion(unsigned long long out[3]);
cudaError_t launch_deposit_init(InstDev *inst, int n_max, const int64_t *prefix, int precision, LaunchCfg cfg,
                                cudaStream_t s);
cudaError_t launch_load(InstDev *inst, int64_t n, double vth, int precision, cudaStream_t s);
cudaError_t launch_sort(InstDev *inst, int n_max, int64_t *prefix, int precision, LaunchCfg cfg, cudaStream_t s);
cudaError_t launch_prefix(InstDev *inst, int n_max, int64_t *prefix, cudaStream_t s);
cudaError_t launch_prefix_one(InstDev *inst, int64_t *prefix, cudaStream_t s);
cudaError_t launch_set_active(InstDev *inst, int active, int64_t target_step, cudaStream_t s);
size_t electron_smem_bytes(int precision, int max_nodes, int eedf_bins, int threads = 256, int n_xs = 0);

// field kernel (hyb_field.cu)
cudaError_t launch_field(InstDev *inst, int n_max, int64_t *prefix, unsigned int *ticket, bool fast, int max_nodes,
                         int threads, cudaStream_t s, int csize = 0, bool early = false);
size_t field_smem_bytes(int max_nodes, int threads);
void configure_field_kernel();

// first failed self-check of each translation unit (zeros in the normal build)
void read_checks_electron(unsigned long long out[3]);
void read_checks_sort(unsigned long long out[3]);
void read_checks_field(unsigned long long out[3]);

// sets the message hyb_last_error() returns (hyb_api.cu)
void set_last_error(const char *msg);

// one-time kernel attributes and occupancy (hyb_electron.cu)
void configure_kernels();
int electron_blocks_per_sm(int precision, size_t smem, int threads = 256, int ppt = 2);

}  // namespace hyb
