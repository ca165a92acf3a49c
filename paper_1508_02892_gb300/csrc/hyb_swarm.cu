// hyb_swarm.cu -- the auxiliary ion-swarm Monte Carlo of arXiv 1508.02892,
// Sec. II.C: one ion species in a prescribed constant field E0 (along z) and a
// homogeneous, periodic domain, colliding with the neutral gas at T_N by the
// null-collision method, isotropic scattering in the centre-of-mass frame on
// Q_m = Q_i + 2 Q_b with the He+/He fits quoted with Tables 2/3.  The mean ion
// velocity after a relaxation window is the drift u; the mobility is u/E0 and
// Eq. 2.6 gives the momentum-exchange frequency e/(M mu).  The tables of
// mobility and exchange frequency that the ion fluid uses are built from runs
// at many field values at once.
//
// Every ion is independent (no field solve, no deposit), so one thread owns
// one ion for the whole run and keeps it in registers: the kernel reads and
// writes no particle memory, and its bound is the ALU rate (two Philox4x32-10
// draws on a candidate step, one otherwise).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "hyb_internal.cuh"

namespace hyb {

namespace {

constexpr int kSwarmBlock = 256;
constexpr unsigned kFull = 0xFFFFFFFFu;

struct SwarmConst {
    double M, mn, m_red, ngas, nu_max, p_max, vt0, vtn;
    int64_t n_ions, n_steps, n_relax;
    int n_fields, xs_model;
    uint32_t seed_lo, seed_hi;
};

// the math functions in the precision of the build; the FP32 build takes the
// hardware approximations (relative error near 2^-21, far below the Monte
// Carlo noise), the FP64 build the accurate library functions
__device__ __forceinline__ float m_pow(float a, float b) { return __powf(a, b); }
__device__ __forceinline__ double m_pow(double a, double b) { return pow(a, b); }
__device__ __forceinline__ float m_sqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double m_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float m_log(float a) { return __logf(a); }
__device__ __forceinline__ double m_log(double a) { return log(a); }
__device__ __forceinline__ float m_fmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double m_fmax(double a, double b) { return fmax(a, b); }

// Q_b of the He+/He fit at relative energy eps > 0 (eV)
template <typename T>
__device__ __forceinline__ T q_back(T eps)
{
    return T(1e-19) / (m_pow(eps / T(1000), T(0.15)) * m_pow(T(1) + eps / T(1000), T(0.25)) *
                       m_pow(T(1) + T(5) / eps, T(0.15)));
}

// the instance constants of the collision frequency in the build's precision
template <typename T>
struct NuConst {
    T ngas, m_red, limit;  // limit: the g -> 0 value N Q_i g (Q_b g -> 0)
    int xs_model;
};

// N Q_m(eps(g)) g, eps = M_r g^2 / 2 in eV
template <typename T>
__device__ __forceinline__ T swarm_nu(const NuConst<T> &c, T g)
{
    const T e = T(1.602176634e-19);
    if (!(g > T(0))) return c.limit;
    const T eps = T(0.5) * c.m_red * g * g / e;
    T q = T(7.63e-20) / m_sqrt(eps);
    if (c.xs_model == HYB_SWARM_QM) q += T(2) * q_back(eps);
    return c.ngas * q * g;
}

template <typename T>
__device__ __forceinline__ T u01(uint32_t x);
template <>
__device__ __forceinline__ double u01<double>(uint32_t x) { return u01d(x); }
template <>
__device__ __forceinline__ float u01<float>(uint32_t x) { return u01f(x); }

__device__ __forceinline__ void sin_cos(double x, double *s, double *c) { sincos(x, s, c); }
__device__ __forceinline__ void sin_cos(float x, float *s, float *c) { __sincosf(x, s, c); }

template <typename T>
__device__ __forceinline__ void box_muller(T u1, T u2, T &g1, T &g2)
{
    const T r = m_sqrt(T(-2) * m_log(u1));
    T s, c;
    sin_cos(T(6.283185307179586476925286766559) * u2, &s, &c);
    g1 = r * c;
    g2 = r * s;
}

// One thread per ion of one field value: ion i of field f has id f n_ions + i.
// acc[f] = (e E_f / M) dt.  sums: per field the sums of v_z and v^2 over the
// averaging window; counts: candidates, real collisions, overruns of nu_max.
template <typename T>
__global__ void __launch_bounds__(kSwarmBlock) k_swarm(SwarmConst c, const double *__restrict__ acc_f,
                                                       double *__restrict__ sums, unsigned long long *__restrict__ counts,
                                                       double *__restrict__ v_out)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = c.n_ions * (int64_t)c.n_fields;
    const bool have = tid < total;
    const int f = have ? (int)(tid / c.n_ions) : 0;
    const uint64_t id = (uint64_t)(have ? tid : 0);
    double s_vz = 0.0, s_v2 = 0.0;
    unsigned long long n_cand = 0, n_coll = 0, n_over = 0;
    if (have) {  // f = tid / n_ions < n_fields
        const T acc = T(acc_f[f]);
        const T vt0 = T(c.vt0), vtn = T(c.vtn);
        const T M = T(c.M), mn = T(c.mn);
        const T nu_max = T(c.nu_max), p_max = T(c.p_max);
        NuConst<T> nc;
        nc.ngas = T(c.ngas);
        nc.m_red = T(c.m_red);
        nc.limit = T(c.ngas) * T(7.63e-20) * m_sqrt(T(2) * T(1.602176634e-19) / T(c.m_red));
        nc.xs_model = c.xs_model;
        const T mt = M + mn;
        T vx, vy, vz;
        T p_vz = T(0), p_v2 = T(0);
        int run = 0;
        {   // initial Maxwellian at T_i0, drawn at the reserved step
            const uint4 r = draw(id, 0xFFFFFFFFu, c.seed_lo, c.seed_hi, 0);
            T g1, g2, g3, g4;
            box_muller(u01<T>(r.x), u01<T>(r.y), g1, g2);
            box_muller(u01<T>(r.z), u01<T>(r.w), g3, g4);
            vx = vt0 * g1;
            vy = vt0 * g2;
            vz = vt0 * g3;
        }
        for (int64_t n = 0; n < c.n_steps; ++n) {
            vz += acc;
            const PhiloxPre pre = philox_pre((uint32_t)n, c.seed_lo, c.seed_hi);
            const uint4 r = draw_pre(pre, id, 0u);
            if (u01<T>(r.x) < p_max) {
                ++n_cand;
                const uint4 w = draw_pre(pre, id, 1u);
                T a1, a2, a3, a4;
                box_muller(u01<T>(r.z), u01<T>(r.w), a1, a2);
                box_muller(u01<T>(w.x), u01<T>(w.y), a3, a4);
                const T Vx = vtn * a1, Vy = vtn * a2, Vz = vtn * a3;
                const T gx = vx - Vx, gy = vy - Vy, gz = vz - Vz;
                const T g = m_sqrt(gx * gx + gy * gy + gz * gz);
                const T nu = swarm_nu<T>(nc, g);
                n_over += nu > nu_max ? 1ull : 0ull;
                if (u01<T>(r.y) * nu_max < nu) {
                    ++n_coll;
                    // isotropic in the centre-of-mass frame
                    const T ct = T(1) - T(2) * u01<T>(w.z);
                    const T st = m_sqrt(m_fmax(T(0), T(1) - ct * ct));
                    T sn, cs;
                    sin_cos(T(6.283185307179586476925286766559) * u01<T>(w.w), &sn, &cs);
                    const T fg = mn / mt * g;
                    vx = (M * vx + mn * Vx) / mt + fg * (st * cs);
                    vy = (M * vy + mn * Vy) / mt + fg * (st * sn);
                    vz = (M * vz + mn * Vz) / mt + fg * ct;
                }
            }
            if (n >= c.n_relax) {
                // window sums: FP64 directly in the FP64 build; the FP32 build sums
                // runs of 256 steps in FP32 and adds them to the FP64 totals (an
                // FP64 add per step would bound it on this part's FP64 rate)
                p_vz += vz;
                p_v2 += vx * vx + vy * vy + vz * vz;
                if (sizeof(T) == 8 || ++run == 256) {
                    s_vz += (double)p_vz;
                    s_v2 += (double)p_v2;
                    p_vz = p_v2 = T(0);
                    run = 0;
                }
            }
        }
        s_vz += (double)p_vz;
        s_v2 += (double)p_v2;
        if (v_out) {
            v_out[3 * tid] = (double)vx;
            v_out[3 * tid + 1] = (double)vy;
            v_out[3 * tid + 2] = (double)vz;
        }
    }
    // per-field sums: a warp whose lanes all hold ions of one field reduces by
    // shuffles first; a warp across two fields (or the ragged end) adds per lane
    const unsigned same = __match_any_sync(kFull, have ? f : -1);
    if (same == kFull) {
        for (int d = 16; d; d >>= 1) {
            s_vz += __shfl_xor_sync(kFull, s_vz, d);
            s_v2 += __shfl_xor_sync(kFull, s_v2, d);
            n_cand += __shfl_xor_sync(kFull, n_cand, d);
            n_coll += __shfl_xor_sync(kFull, n_coll, d);
            n_over += __shfl_xor_sync(kFull, n_over, d);
        }
        if ((threadIdx.x & 31) != 0 || !have) return;
    } else if (!have) {
        return;
    }
    atomicAdd(&sums[2 * f], s_vz);
    atomicAdd(&sums[2 * f + 1], s_v2);
    atomicAdd(&counts[3 * f], n_cand);
    atomicAdd(&counts[3 * f + 1], n_coll);
    atomicAdd(&counts[3 * f + 2], n_over);
}

// ---------------------------------------------------------------- host side

// the bound nu_max: the largest N Q_m g over relative energies up to eps_max,
// on a dense logarithmic grid, with a relative margin of 1e-6
double nu_bound(double ngas, double m_red, int xs_model, double eps_max)
{
    const double e = kQe;
    double best = 0.0;
    const int n = 200000;
    for (int i = 0; i <= n; ++i) {
        const double eps = 1e-8 * pow(eps_max / 1e-8, (double)i / n);
        const double g = sqrt(2.0 * e * eps / m_red);
        double q = 7.63e-20 / sqrt(eps);
        if (xs_model == HYB_SWARM_QM)
            q += 2.0 * 1e-19 / (pow(eps / 1000.0, 0.15) * pow(1.0 + eps / 1000.0, 0.25) * pow(1.0 + 5.0 / eps, 0.15));
        const double v = ngas * q * g;
        if (v > best) best = v;
    }
    return best * (1.0 + 1e-6);
}

int swarm_fail(int code, const char *msg)
{
    set_last_error(msg);
    return code;
}

}  // namespace

// the same bound for the kinetic ions of a discharge (Q_m = Q_i + 2 Q_b)
double swarm_nu_bound(double ngas, double m_red, double eps_max) { return nu_bound(ngas, m_red, HYB_SWARM_QM, eps_max); }

}  // namespace hyb

using namespace hyb;

extern "C" int hyb_swarm_run(const hyb_swarm_params *p, int32_t n_fields, const double *e_field, hyb_swarm_result *out,
                             double *v_out, void *stream)
{
    if (!p || !e_field || !out) return swarm_fail(HYB_ERR_ARG, "NULL argument");
    if (n_fields < 1 || n_fields > 65536) return swarm_fail(HYB_ERR_ARG, "n_fields must be in [1, 65536]");
    if (p->n_ions < 1 || p->n_steps < 1 || p->n_relax < 0 || p->n_relax >= p->n_steps)
        return swarm_fail(HYB_ERR_ARG, "need n_ions >= 1 and 0 <= n_relax < n_steps");
    if (p->n_steps > 0xFFFFFFFFll) return swarm_fail(HYB_ERR_ARG, "n_steps must fit the 32-bit step counter");
    if (p->n_ions > (int64_t)1 << 40 || p->n_ions * (int64_t)n_fields > ((int64_t)1 << 40))
        return swarm_fail(HYB_ERR_ARG, "n_ions * n_fields must be below 2^40");
    if (!(p->dt_s > 0) || !(p->pressure_pa > 0) || !(p->gas_temp_k > 0) || !(p->ion_temp0_k >= 0) || p->nu_max < 0 ||
        p->eps_max_ev < 0 || p->gas_mass_amu < 0 || p->ion_mass_amu < 0)
        return swarm_fail(HYB_ERR_ARG, "dt, pressure and gas temperature must be positive, the rest non-negative");
    if (p->xs_model != HYB_SWARM_QM && p->xs_model != HYB_SWARM_QI_ONLY)
        return swarm_fail(HYB_ERR_ARG, "unknown cross-section model");
    if (p->precision != HYB_FP64 && p->precision != HYB_FP32_SPLIT) return swarm_fail(HYB_ERR_ARG, "unknown precision");
    for (int f = 0; f < n_fields; ++f)
        if (!isfinite(e_field[f])) return swarm_fail(HYB_ERR_NONFINITE, "non-finite field value");

    const double mg = p->gas_mass_amu > 0 ? p->gas_mass_amu : 4.002602;
    SwarmConst c{};
    c.M = (p->ion_mass_amu > 0 ? p->ion_mass_amu : mg) * kAmu;
    c.mn = mg * kAmu;
    c.m_red = c.M * c.mn / (c.M + c.mn);
    c.ngas = p->pressure_pa / (kKb * p->gas_temp_k);
    c.nu_max = p->nu_max > 0 ? p->nu_max
                             : nu_bound(c.ngas, c.m_red, p->xs_model, p->eps_max_ev > 0 ? p->eps_max_ev : 100.0);
    c.p_max = -expm1(-c.nu_max * p->dt_s);
    c.vt0 = sqrt(kKb * p->ion_temp0_k / c.M);
    c.vtn = sqrt(kKb * p->gas_temp_k / c.mn);
    c.n_ions = p->n_ions;
    c.n_steps = p->n_steps;
    c.n_relax = p->n_relax;
    c.n_fields = n_fields;
    c.xs_model = p->xs_model;
    c.seed_lo = (uint32_t)p->seed;
    c.seed_hi = (uint32_t)(p->seed >> 32);

    std::vector<double> acc(n_fields);
    for (int f = 0; f < n_fields; ++f) acc[f] = kQe * e_field[f] / c.M * p->dt_s;
    cudaStream_t s = (cudaStream_t)stream;
    char *mem = nullptr;
    const size_t bytes = sizeof(double) * (size_t)n_fields * 3 + sizeof(unsigned long long) * (size_t)n_fields * 3;
    cudaError_t e = cudaMallocAsync((void **)&mem, bytes, s);
    if (e != cudaSuccess) return swarm_fail(HYB_ERR_OOM, cudaGetErrorString(e));
    double *d_acc = (double *)mem;
    double *d_sums = d_acc + n_fields;
    unsigned long long *d_counts = (unsigned long long *)(d_sums + 2 * (size_t)n_fields);
    std::vector<double> h_sums(2 * (size_t)n_fields);
    std::vector<unsigned long long> h_counts(3 * (size_t)n_fields);
    e = cudaMemcpyAsync(d_acc, acc.data(), sizeof(double) * n_fields, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_sums, 0, bytes - sizeof(double) * n_fields, s);
    if (e == cudaSuccess) {
        const int64_t total = c.n_ions * (int64_t)n_fields;
        const unsigned grid = (unsigned)((total + kSwarmBlock - 1) / kSwarmBlock);
        if (p->precision == HYB_FP64)
            k_swarm<double><<<grid, kSwarmBlock, 0, s>>>(c, d_acc, d_sums, d_counts, v_out);
        else
            k_swarm<float><<<grid, kSwarmBlock, 0, s>>>(c, d_acc, d_sums, d_counts, v_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_sums.data(), d_sums, sizeof(double) * 2 * n_fields, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_counts.data(), d_counts, sizeof(unsigned long long) * 3 * n_fields, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(mem, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return swarm_fail(HYB_ERR_CUDA, cudaGetErrorString(e));

    const double ns = (double)c.n_ions * (double)(c.n_steps - c.n_relax);
    for (int f = 0; f < n_fields; ++f) {
        hyb_swarm_result &r = out[f];
        r.e_field = e_field[f];
        r.drift = h_sums[2 * f] / ns;
        r.mean_energy_ev = 0.5 * c.M * h_sums[2 * f + 1] / ns / kQe;
        r.mobility = e_field[f] != 0.0 ? r.drift / e_field[f] : 0.0;
        r.nu_exchange = r.mobility != 0.0 ? kQe / (c.M * r.mobility) : 0.0;
        r.nu_max = c.nu_max;
        r.p_max = c.p_max;
        r.candidates = (int64_t)h_counts[3 * f];
        r.collisions = (int64_t)h_counts[3 * f + 1];
        r.overruns = (int64_t)h_counts[3 * f + 2];
    }
    int over = 0;
    for (int f = 0; f < n_fields; ++f) over |= out[f].overruns > 0;
    if (over) {
        set_last_error("collision frequency exceeded nu_max (raise eps_max_ev or nu_max)");
        return HYB_WARN_NU_MAX;
    }
    return HYB_OK;
}

// Mobility and exchange-frequency tables over E/N for the ion fluid: one
// swarm run per table point, all at once; at E/N = 0 the table takes the
// values of the lowest positive field (the drift vanishes with E there).
extern "C" int hyb_swarm_tables(const hyb_swarm_params *p, int32_t n, const double *eon_td, double *tab_mu,
                                double *tab_nu, void *stream)
{
    if (!p || !eon_td || !tab_mu || !tab_nu || n < 2) return swarm_fail(HYB_ERR_ARG, "NULL argument or n < 2");
    for (int k = 0; k < n; ++k)
        if (!(eon_td[k] >= 0) || (k && !(eon_td[k] > eon_td[k - 1])))
            return swarm_fail(HYB_ERR_ARG, "E/N must be non-negative and increasing");
    const double ngas = p->pressure_pa / (kKb * p->gas_temp_k);
    std::vector<double> E;
    std::vector<int> src(n);
    for (int k = 0; k < n; ++k) {
        if (eon_td[k] > 0) {
            src[k] = (int)E.size();
            E.push_back(eon_td[k] * 1e-21 * ngas);
        }
    }
    if (E.empty()) return swarm_fail(HYB_ERR_ARG, "no positive E/N");
    for (int k = 0; k < n; ++k)
        if (!(eon_td[k] > 0)) src[k] = 0;
    std::vector<hyb_swarm_result> r(E.size());
    const int rc = hyb_swarm_run(p, (int32_t)E.size(), E.data(), r.data(), nullptr, stream);
    if (rc < 0) return rc;
    for (int k = 0; k < n; ++k) {
        tab_mu[k] = r[src[k]].mobility;
        tab_nu[k] = r[src[k]].nu_exchange;
    }
    return rc;
}
