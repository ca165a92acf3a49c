// hyb_api.cu -- host runtime behind the C ABI of include/hybrid1d.h: parameter
// validation and derived constants (arXiv 1508.02892, Secs. II.A-II.D),
// instance slots with one device allocation each, the HBM cap of a batch, the
// initial load, CUDA-graph chunks of steps, reads and writes of the state.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "hyb_internal.cuh"

using namespace hyb;

namespace {
thread_local std::string g_err;
}

void hyb::set_last_error(const char *msg) { g_err = msg ? msg : ""; }

namespace {

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(expr)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (expr);                                                                  \
        if (e_ != cudaSuccess) return fail(HYB_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

constexpr int kDefaultSort = 20;
constexpr int kElectronBlock = 256;
constexpr int kMaxLanes = 16;
constexpr int kDefaultLanes = 4;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t part_bytes, grid_off, total;
    size_t off[64];
    int n;
};

struct Slot {
    bool used = false;
    bool reported = false;
    hyb_params p{};
    InstDev h{};
    InstDev hi{};  // kinetic ions: the ion descriptor
    void *mem = nullptr;
    int64_t bytes = 0;
    int64_t target = 0;
    int64_t admit_after = 0;  // snapshots queued before the admission (they do not show it)
    int64_t admission = 0;    // the batch's admission count when this discharge was admitted
};

double mass_gas_amu(const hyb_params &p)
{
    if (p.gas_mass_amu > 0) return p.gas_mass_amu;
    return p.gas == HYB_GAS_AR ? 39.948 : 4.002602;
}

int bins_of(const hyb_params &p) { return p.eedf_bins > 0 ? p.eedf_bins : 256; }

int64_t capacity_of(const hyb_params &p)
{
    const double f = p.capacity_factor > 0 ? p.capacity_factor : 2.0;
    int64_t c = (int64_t)ceil(f * (double)p.n_particles);
    c = c < 4096 ? 4096 : c;
    return (c + 255) & ~(int64_t)255;
}

bool finite_all(const double *x, int n)
{
    for (int i = 0; i < n; ++i)
        if (!isfinite(x[i])) return false;
    return true;
}

// linear interpolation in (x, y), x increasing, clamped at the ends
double interp_clamped(const double *x, const double *y, int n, double v)
{
    if (v <= x[0]) return y[0];
    if (v >= x[n - 1]) return y[n - 1];
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (x[mid] <= v)
            lo = mid;
        else
            hi = mid;
    }
    return y[lo] + (v - x[lo]) / (x[lo + 1] - x[lo]) * (y[lo + 1] - y[lo]);
}

int validate(const hyb_params *p)
{
    if (!p) return fail(HYB_ERR_ARG, "params is NULL");
    if (!(p->gap_m > 0) || !(p->dt_s > 0) || !(p->pressure_pa > 0) || !(p->gas_temp_k > 0))
        return fail(HYB_ERR_ARG, "gap, dt, pressure and gas temperature must be positive");
    if (p->n_cells < 2 || p->n_cells > HYB_MAX_CELLS)
        return fail(HYB_ERR_ARG, "n_cells must be in [2, %d]", HYB_MAX_CELLS);
    if (p->gas != HYB_GAS_HE && p->gas != HYB_GAS_AR) return fail(HYB_ERR_ARG, "unknown gas");
    if (p->n_particles < 0 || p->n0_m3 < 0 || p->te0_ev < 0 || p->weight < 0 || p->gamma_see < 0)
        return fail(HYB_ERR_ARG, "negative particle count, density, temperature, weight or gamma");
    if (p->precision != HYB_FP64 && p->precision != HYB_FP32_SPLIT) return fail(HYB_ERR_ARG, "unknown precision");
    if (p->ion_model < HYB_ION_DD_CONST || p->ion_model > HYB_ION_KINETIC) return fail(HYB_ERR_ARG, "unknown ion model");
    if (p->ion_model == HYB_ION_KINETIC && p->xs_rec)
        return fail(HYB_ERR_ARG, "recombination is built for the fluid ion models only");
    if (p->eedf_bins < 0 || p->eedf_bins > 4096) return fail(HYB_ERR_ARG, "eedf_bins must be in [0, 4096]");
    if (!p->xs_ev || !p->xs_el || !p->xs_exc || !p->xs_ion || p->n_xs < 2)
        return fail(HYB_ERR_ARG, "cross-section tables missing");
    // the split-mode particle step keeps the table and its segment slopes in
    // shared memory (32 bytes an entry)
    if (p->precision == HYB_FP32_SPLIT && p->n_xs > kMaxSplitXs)
        return fail(HYB_ERR_ARG, "n_xs must be at most %d in split mode", kMaxSplitXs);
    if (!finite_all(p->xs_ev, p->n_xs) || !finite_all(p->xs_el, p->n_xs) || !finite_all(p->xs_exc, p->n_xs) ||
        !finite_all(p->xs_ion, p->n_xs))
        return fail(HYB_ERR_NONFINITE, "non-finite cross-section table entry");
    if (!(p->xs_ev[0] > 0)) return fail(HYB_ERR_ARG, "cross-section energies must be positive");
    for (int i = 1; i < p->n_xs; ++i)
        if (!(p->xs_ev[i] > p->xs_ev[i - 1])) return fail(HYB_ERR_ARG, "cross-section energies must increase");
    for (int i = 0; i < p->n_xs; ++i)
        if (p->xs_el[i] < 0 || p->xs_exc[i] < 0 || p->xs_ion[i] < 0)
            return fail(HYB_ERR_ARG, "negative cross section");
    if (p->e_exc_ev < 0 || p->e_iz_ev < 0) return fail(HYB_ERR_ARG, "negative threshold");
    if (p->ion_model == HYB_ION_DD_TABLE || p->ion_model == HYB_ION_FULL) {
        if (!p->tab_eon_td || !p->tab_mu || !p->tab_nu || p->n_tab < 2 || p->n_tab > 256)
            return fail(HYB_ERR_ARG, "ion transport tables missing or longer than 256");
        if (!finite_all(p->tab_eon_td, p->n_tab) || !finite_all(p->tab_mu, p->n_tab) ||
            !finite_all(p->tab_nu, p->n_tab))
            return fail(HYB_ERR_NONFINITE, "non-finite ion transport table entry");
        for (int k = 1; k < p->n_tab; ++k)
            if (!(p->tab_eon_td[k] > p->tab_eon_td[k - 1])) return fail(HYB_ERR_ARG, "E/N table must increase");
        if (p->ion_model == HYB_ION_FULL)
            for (int k = 1; k < p->n_tab; ++k)
                if (!(p->tab_mu[k] * p->tab_eon_td[k] > p->tab_mu[k - 1] * p->tab_eon_td[k - 1]))
                    return fail(HYB_ERR_ARG, "drift speed mu E must increase along the table");
    } else if (!(p->mu_const >= 0)) {
        return fail(HYB_ERR_ARG, "mu_const must be non-negative");
    }
    if (!isfinite(p->v_rf_amp_v) || !isfinite(p->f_rf_hz) || !isfinite(p->v_dc_v))
        return fail(HYB_ERR_NONFINITE, "non-finite drive");
    if (!(p->power_w_m2 >= 0) || !(p->power_alpha >= 0) || !isfinite(p->power_w_m2) || !isfinite(p->power_alpha))
        return fail(HYB_ERR_ARG, "power target and alpha must be finite and non-negative");
    if (p->xs_rec) {
        if (!finite_all(p->xs_rec, p->n_xs)) return fail(HYB_ERR_NONFINITE, "non-finite recombination cross section");
        for (int i = 0; i < p->n_xs; ++i)
            if (p->xs_rec[i] < 0) return fail(HYB_ERR_ARG, "negative recombination cross section");
    }
    if (p->ion_model == HYB_ION_DD_CONST || p->ion_model == HYB_ION_DD_TABLE) {
        // explicit drift-diffusion (Eq. 2.5 at level n into Eq. 2.4): the
        // centred scheme needs u^2 dt <= 2 D and D dt / dz^2 <= 1/2, checked at
        // the field of the drive across the empty gap, (|V_dc| + |V_rf|) / L,
        // with D from Eq. 2.7 (Eq. 2.8 temperature for the tabulated model)
        const double e = (fabs(p->v_dc_v) + fabs(p->v_rf_amp_v)) / p->gap_m;
        const double kT = kKb * p->gas_temp_k;
        double mu = p->mu_const, T = kT;
        if (p->ion_model == HYB_ION_DD_TABLE) {
            const double eon = e / (p->pressure_pa / kT) * 1e21;
            mu = interp_clamped(p->tab_eon_td, p->tab_mu, p->n_tab, eon);
            const double mn = mass_gas_amu(*p) * kAmu;
            const double mi = p->ion_mass_amu > 0 ? p->ion_mass_amu * kAmu : mn;
            const double ud = mu * e;
            T = kT + (mi + mn) / (5.0 * mi + 3.0 * mn) * mn * ud * ud;
        }
        const double D = mu * T / kQe, u = mu * e, dz = p->gap_m / p->n_cells;
        if (u * u * p->dt_s > 2.0 * D || D * p->dt_s > 0.5 * dz * dz)
            return fail(HYB_ERR_UNSTABLE, "drift-diffusion: u^2 dt > 2 D or D dt/dz^2 > 1/2 at the drive's field");
    }
    if (p->metastables != 0 && p->metastables != 1) return fail(HYB_ERR_ARG, "metastables must be 0 or 1");
    if (!(p->gamma_met >= 0) || !isfinite(p->gamma_met)) return fail(HYB_ERR_ARG, "gamma_met must be finite and >= 0");
    if (p->metastables) {
        if (p->ion_model == HYB_ION_KINETIC)
            return fail(HYB_ERR_ARG, "metastables are built for the fluid ion models only");
        const double v[7] = {p->met_diff_m2s,      p->met_n0_m3,        p->penning_rate_m3s, p->penning_target_m3,
                             p->penning_energy_ev, p->pooling_rate_m3s, p->pooling_energy_ev};
        for (double x : v)
            if (!(x >= 0) || !isfinite(x)) return fail(HYB_ERR_ARG, "metastable parameters must be finite and >= 0");
        // explicit diffusion: D dt / dz^2 <= 1/2
        if (p->met_diff_m2s * p->dt_s * p->n_cells * p->n_cells > 0.5 * p->gap_m * p->gap_m)
            return fail(HYB_ERR_UNSTABLE, "metastable diffusion: D dt/dz^2 > 1/2");
    }
    return HYB_OK;
}

Layout layout_of(const hyb_params &p)
{
    Layout L{};
    const int64_t cap = capacity_of(p);
    const int G = p.n_cells + 1;
    const int nb = bins_of(p);
    size_t o = 0;
    auto add = [&](size_t bytes) {
        L.off[L.n++] = o;
        o += align256(bytes);
    };
    // particle buffers x2
    for (int b = 0; b < 2; ++b) {
        if (p.precision == HYB_FP32_SPLIT) {
            add(4 * cap);  // c
            add(4 * cap);  // o
            add(4 * cap);  // vx
            add(4 * cap);  // vy
            add(4 * cap);  // vz
        } else {
            add(8 * cap);  // z
            add(8 * cap);
            add(8 * cap);
            add(8 * cap);
        }
        add(8 * cap);  // id
    }
    L.part_bytes = o;
    L.grid_off = o;
    for (int k = 0; k < 14; ++k) add(8 * (size_t)G);  // ni gam phi E ne gsrc dep_n dep_e s_iz acc x5
    add(4 * (size_t)G);                                 // Ef
    add(4 * (size_t)G);                                 // cell_cnt (n_cells + 1)
    add(8 * (size_t)(nb + 1));                          // eedf
    add(32 * (size_t)p.n_xs);                           // xs
    add(16 * (size_t)p.n_xs);                           // xsf
    add((32 + 8 * kTabCols + 8) * (size_t)(p.n_tab > 0 ? p.n_tab : 1));  // tab, tabx, tabf
    add(8 * (size_t)p.n_xs);                            // xs_rec
    add(4 * (size_t)p.n_xs);                            // xs_recf
    add(4 * (size_t)G);                                 // nif
    if (p.metastables) {
        add(8 * (size_t)G);                             // met
        add(8 * (size_t)G);                             // s_met
        add(8 * (size_t)G);                             // acc_met
    }
    if (p.ion_model == HYB_ION_KINETIC) {
        for (int b = 0; b < 2; ++b) {                   // ion buffers in the batch's precision
            if (p.precision == HYB_FP32_SPLIT)
                for (int k = 0; k < 5; ++k) add(4 * cap);  // c, o, vx, vy, vz
            else
                for (int k = 0; k < 4; ++k) add(8 * cap);  // z, vx, vy, vz
            add(8 * cap);                                  // id
        }
        add(4 * (size_t)G);                             // ion cell counts
        add(8 * (size_t)G);                             // dep_ni
        add(8 * (size_t)G);                             // dep_gi
    }
    L.total = o;
    return L;
}

// sigma_k(E) with the log-index, linear-in-energy lookup and the thresholds.
void xs_eval_host(const hyb_params &p, double e_lo, double e_hi, double inv_dlog, double en, double sig[3])
{
    const int n = p.n_xs;
    int i;
    double f;
    if (en <= e_lo) {
        i = 0;
        f = 0.0;
    } else if (en >= e_hi) {
        i = n - 2;
        f = 1.0;
    } else {
        const double x = log(en / e_lo) * inv_dlog;
        i = (int)floor(x);
        if (i < 0) i = 0;
        if (i > n - 2) i = n - 2;
        f = (en - p.xs_ev[i]) / (p.xs_ev[i + 1] - p.xs_ev[i]);
    }
    sig[0] = p.xs_el[i] + f * (p.xs_el[i + 1] - p.xs_el[i]);
    sig[1] = p.xs_exc[i] + f * (p.xs_exc[i + 1] - p.xs_exc[i]);
    sig[2] = p.xs_ion[i] + f * (p.xs_ion[i + 1] - p.xs_ion[i]);
    if (en < p.e_exc_ev) sig[1] = 0.0;
    if (en < p.e_iz_ev) sig[2] = 0.0;
}

// Derived constants of Secs. II.A-II.D; fills K (pointers excluded) and the
// host copies of the tables.
void derive(const hyb_params &p, InstDev &K, std::vector<double> &xs, std::vector<float4> &xsf,
            std::vector<double> &tab)
{
    memset(&K, 0, sizeof K);
    K.precision = p.precision;
    K.n_cells = p.n_cells;
    K.G = p.n_cells + 1;
    K.ion_model = p.ion_model;
    K.n_xs = p.n_xs;
    K.n_tab = (p.ion_model == HYB_ION_DD_TABLE || p.ion_model == HYB_ION_FULL) ? p.n_tab : 0;
    K.eedf_bins = bins_of(p);
    K.capacity = capacity_of(p);
    K.L = p.gap_m;
    K.dz = p.gap_m / p.n_cells;
    K.inv_gm1 = 1.0 / (double)p.n_cells;
    K.dt = p.dt_s;
    K.ngas = p.pressure_pa / (kKb * p.gas_temp_k);
    K.w = p.weight > 0 ? p.weight : (p.n_particles > 0 ? p.n0_m3 * p.gap_m / (double)p.n_particles : 0.0);
    const double mg = mass_gas_amu(p);
    K.m_gas = mg * kAmu;
    K.m_ion = (p.ion_mass_amu > 0 ? p.ion_mass_amu : mg) * kAmu;
    K.qm = kQe / kMe;
    K.n_floor = 1e-6 * p.n0_m3;
    K.bin_w = (p.eedf_max_ev > 0 ? p.eedf_max_ev : 64.0) / K.eedf_bins;
    K.e_lo = p.xs_ev[0];
    K.e_hi = p.xs_ev[p.n_xs - 1];
    K.inv_dlog = (p.n_xs - 1) / log(K.e_hi / K.e_lo);
    K.e_exc = p.e_exc_ev;
    K.e_iz = p.e_iz_ev;
    K.two_mM = 2.0 * (kMe / K.m_gas);
    K.gamma_see = p.gamma_see;
    K.see_speed = sqrt(2.0 * kQe * (p.see_energy_ev > 0 ? p.see_energy_ev : 1.0) / kMe);
    K.v_rf = p.v_rf_amp_v;
    K.pw_target = p.power_w_m2;
    K.pw_alpha = p.power_alpha;
    K.pw_steps = p.f_rf_hz > 0 ? llround(1.0 / (p.f_rf_hz * p.dt_s)) : 0;
    if (K.pw_steps < 1) K.pw_steps = INT64_MAX;  // no RF period: no update
    K.f_rf = p.f_rf_hz;
    K.v_dc = p.v_dc_v;
    K.mu_const = p.mu_const;
    K.kT_gas = kKb * p.gas_temp_k;
    K.seed_lo = (uint32_t)p.seed;
    K.seed_hi = (uint32_t)(p.seed >> 32);
    {
        // field-step constants (Secs. II.B-II.D)
        FieldK &f = K.fk;
        const double dz = K.dz, dt = K.dt, w = K.w, mi = K.m_ion, mn = K.m_gas;
        f.h = dt / (2.0 * dz);
        f.qdt_m = kQe * dt / mi;
        f.h_m = f.h / mi;
        f.c_in = dt / (2.0 * dz);
        f.c_wall = dt / dz;
        f.gs_in = w / (dz * dt);
        f.gs_wall = w / (0.5 * dz * dt);
        f.hdt = 0.5 * dt;
        f.tfac = (mi + mn) / (5.0 * mi + 3.0 * mn) * mn;
        f.inv_ngas_td = 1e21 / K.ngas;
        f.inv_qe = 1.0 / kQe;
        f.inv2dz = 1.0 / (2.0 * dz);
        f.dt_dz = dt / dz;
        f.dt_2dz = dt / (2.0 * dz);
        f.h_mion = f.h / mi;
        f.w_in = w / dz;
        f.w_wall = 2.0 * w / dz;
        f.c_src = dz * dz / kEps0;
        f.inv_dz = 1.0 / dz;
        f.half_inv_dz = 0.5 / dz;
        f.c_gauss = dz / (2.0 * kEps0);
    }
    // nu_max over the table nodes and P_max (Sec. II.A)
    double nu_max = 0.0;
    for (int i = 0; i < p.n_xs; ++i) {
        double sig[3];
        xs_eval_host(p, K.e_lo, K.e_hi, K.inv_dlog, p.xs_ev[i], sig);
        const double v = sqrt(2.0 * kQe * p.xs_ev[i] / kMe);
        const double nu = K.ngas * (sig[0] + sig[1] + sig[2]) * v;
        if (nu > nu_max) nu_max = nu;
    }
    K.nu_max = nu_max;
    K.p_max = 1.0 - exp(-nu_max * K.dt);
    // FP32 copies
    K.f_dt_dz = (float)(K.dt / K.dz);
    K.f_qm_dt = (float)(K.qm * K.dt);
    K.f_half_m_q = (float)(0.5 * kMe / kQe);
    K.f_two_q_m = (float)(2.0 * kQe / kMe);
    K.f_pmax = (float)K.p_max;
    K.f_e_lo = (float)K.e_lo;
    K.f_e_hi = (float)K.e_hi;
    K.f_inv_e_lo = (float)(1.0 / K.e_lo);
    K.f_inv_dlog = (float)K.inv_dlog;
    K.f_e_exc = (float)K.e_exc;
    K.f_e_iz = (float)K.e_iz;
    K.f_two_mM = (float)K.two_mM;
    K.f_bin_inv = (float)(1.0 / K.bin_w);
    xs.resize(4 * (size_t)p.n_xs);
    xsf.resize(p.n_xs);
    const double scale = nu_max > 0 ? K.ngas / nu_max : 0.0;
    for (int i = 0; i < p.n_xs; ++i) {
        xs[4 * i + 0] = p.xs_ev[i];
        xs[4 * i + 1] = p.xs_el[i];
        xs[4 * i + 2] = p.xs_exc[i];
        xs[4 * i + 3] = p.xs_ion[i];
        xsf[i] = make_float4((float)p.xs_ev[i], (float)(scale * p.xs_el[i]), (float)(scale * p.xs_exc[i]),
                             (float)(scale * p.xs_ion[i]));
    }
    // kinetic ions: the collision bound of the auxiliary Monte Carlo over
    // relative energies up to 100 eV, and the gas Maxwellian
    if (p.ion_model == HYB_ION_KINETIC) {
        K.mi_red = K.m_ion * K.m_gas / (K.m_ion + K.m_gas);
        K.nu_max_i = swarm_nu_bound(K.ngas, K.mi_red, 100.0);
        K.p_max_i = -expm1(-K.nu_max_i * K.dt);
        K.vt_gas = sqrt(kKb * p.gas_temp_k / K.m_gas);
        K.fi_qm_dt = (float)(kQe / K.m_ion * K.dt);
        K.fi_ngas = (float)K.ngas;
        K.fi_half_mr_q = (float)(0.5 * K.mi_red / kQe);
        K.fi_numax = (float)K.nu_max_i;
        K.fi_pmax = (float)K.p_max_i;
        K.fi_vt = (float)K.vt_gas;
        K.fi_cm_a = (float)(K.m_ion / (K.m_ion + K.m_gas));
        K.fi_cm_b = (float)(K.m_gas / (K.m_ion + K.m_gas));
        K.fi_nu0 = (float)(K.ngas * 7.63e-20 * sqrt(2.0 * kQe / K.mi_red));
    }
    // recombination (Sec. II.D): sigma_rec v bounded on each table segment by the
    // larger endpoint cross section times the speed at the upper end
    K.rec_on = p.xs_rec != nullptr;
    K.rec_svmax = 0.0;
    if (K.rec_on)
        for (int i = 0; i + 1 < p.n_xs; ++i) {
            const double sg = fmax(p.xs_rec[i], p.xs_rec[i + 1]);
            const double v = sqrt(2.0 * kQe * p.xs_ev[i + 1] / kMe);
            if (sg * v > K.rec_svmax) K.rec_svmax = sg * v;
        }
    // metastables and their reactions (Sec. II.D)
    K.met_on = p.metastables ? 1 : 0;
    K.met_D = p.met_diff_m2s;
    K.met_rp = p.penning_rate_m3s;
    K.met_nn = p.penning_target_m3;
    K.met_kp = p.penning_rate_m3s * p.penning_target_m3;
    K.met_kq = p.pooling_rate_m3s;
    K.met_sp[0] = sqrt(2.0 * kQe * p.penning_energy_ev / kMe);
    K.met_sp[1] = sqrt(2.0 * kQe * p.pooling_energy_ev / kMe);
    K.gamma_met = p.gamma_met;
    const int nt = K.n_tab > 0 ? K.n_tab : 1;
    // the table as given, then the split-mode layout (with the slope of each
    // segment, formed once here), then the FP32 abscissae (two per double)
    tab.assign((4 + kTabCols + 1) * (size_t)nt, 0.0);
    for (int k = 0; k < K.n_tab; ++k) {
        tab[4 * k + 0] = p.tab_eon_td[k];
        tab[4 * k + 1] = p.tab_mu[k];
        tab[4 * k + 2] = p.tab_nu[k];
        tab[4 * k + 3] = p.tab_mu[k] * p.tab_eon_td[k] * 1e-21 * K.ngas;
    }
    double *x = tab.data() + 4 * (size_t)nt;
    float *xf = reinterpret_cast<float *>(x + kTabCols * (size_t)nt);
    for (int k = 0; k < K.n_tab; ++k) {
        const double *a = tab.data() + 4 * k;
        double *o = x + kTabCols * k;
        o[0] = a[0];
        o[1] = a[1];
        o[3] = a[3];
        o[4] = a[2];
        o[2] = k + 1 < K.n_tab ? (a[5] - a[1]) / (a[4] - a[0]) : 0.0;
        o[5] = k + 1 < K.n_tab ? (a[6] - a[2]) / (a[7] - a[3]) : 0.0;
        xf[k] = (float)a[0];
        xf[K.n_tab + k] = (float)a[3];
    }
}

void bind_pointers(const hyb_params &p, const Layout &L, char *base, InstDev &K, InstDev *ion_out)
{
    int k = 0;
    for (int b = 0; b < 2; ++b) {
        PartBuf &B = K.buf[b];
        memset(&B, 0, sizeof B);
        if (p.precision == HYB_FP32_SPLIT) {
            B.c = (int32_t *)(base + L.off[k++]);
            B.o = (float *)(base + L.off[k++]);
            B.vxf = (float *)(base + L.off[k++]);
            B.vyf = (float *)(base + L.off[k++]);
            B.vzf = (float *)(base + L.off[k++]);
        } else {
            B.z = (double *)(base + L.off[k++]);
            B.vxd = (double *)(base + L.off[k++]);
            B.vyd = (double *)(base + L.off[k++]);
            B.vzd = (double *)(base + L.off[k++]);
        }
        B.id = (uint64_t *)(base + L.off[k++]);
    }
    double **grids[14] = {&K.ni, &K.gam, &K.phi, &K.E, &K.ne, &K.gsrc, &K.dep_n, &K.dep_e,
                          &K.s_iz, &K.acc_ne, &K.acc_ni, &K.acc_gi, &K.acc_wn, &K.acc_we};
    for (int g = 0; g < 14; ++g) *grids[g] = (double *)(base + L.off[k++]);
    K.Ef = (float *)(base + L.off[k++]);
    K.cell_cnt = (int32_t *)(base + L.off[k++]);
    K.eedf = (unsigned long long *)(base + L.off[k++]);
    K.xs = (const double *)(base + L.off[k++]);
    K.xsf = (const float4 *)(base + L.off[k++]);
    K.tab = (const double *)(base + L.off[k++]);
    {
        const size_t nt = (size_t)(p.n_tab > 0 ? p.n_tab : 1);
        K.tabx = K.tab + 4 * nt;
        K.tabf = (const float *)(K.tabx + kTabCols * nt);
    }
    K.xs_rec = (const double *)(base + L.off[k++]);
    K.xs_recf = (const float *)(base + L.off[k++]);
    K.nif = (float *)(base + L.off[k++]);
    if (p.metastables) {
        K.met = (double *)(base + L.off[k++]);
        K.s_met = (double *)(base + L.off[k++]);
        K.acc_met = (double *)(base + L.off[k++]);
    }
    if (p.ion_model == HYB_ION_KINETIC) {
        // the ion descriptor starts as a copy of this one; here the ion buffers
        // go to I (its fields buf and cell_cnt), the shared sums to K
        InstDev &I = *ion_out;
        for (int b = 0; b < 2; ++b) {
            PartBuf &B = I.buf[b];
            memset(&B, 0, sizeof B);
            if (p.precision == HYB_FP32_SPLIT) {
                B.c = (int32_t *)(base + L.off[k++]);
                B.o = (float *)(base + L.off[k++]);
                B.vxf = (float *)(base + L.off[k++]);
                B.vyf = (float *)(base + L.off[k++]);
                B.vzf = (float *)(base + L.off[k++]);
            } else {
                B.z = (double *)(base + L.off[k++]);
                B.vxd = (double *)(base + L.off[k++]);
                B.vyd = (double *)(base + L.off[k++]);
                B.vzd = (double *)(base + L.off[k++]);
            }
            B.id = (uint64_t *)(base + L.off[k++]);
        }
        I.cell_cnt = (int32_t *)(base + L.off[k++]);
        K.dep_ni = (double *)(base + L.off[k++]);
        K.dep_gi = (double *)(base + L.off[k++]);
    }
}

}  // namespace

// Lanes: the slots are split into `lanes` contiguous groups, each advanced by
// its own chain of launches (electron step, field, periodic sort) with its own
// chunk prefix and field ticket.  Inside a captured chunk the chains are
// parallel branches, so that the field kernels of one lane (one CTA per
// instance, bound by that SM's FP64 rate) run beside the electron kernels of
// the others instead of leaving most SMs idle.
struct hyb_batch {
    int max_inst = 0;
    int precision = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    InstDev *d_inst = nullptr;
    int64_t *d_prefix = nullptr;   // kMaxLanes x (max_inst + 1)
    int64_t *d_prefix1 = nullptr;
    unsigned *d_ticket = nullptr;  // kMaxLanes field tickets, then the single-instance one
    unsigned *d_ticket1 = nullptr;
    int lanes = 1, per_lane = 1;
    cudaStream_t lstream[kMaxLanes] = {};  // lane k > 0 (lane 0 uses `stream`)
    cudaEvent_t ev_fork = nullptr, ev_join[kMaxLanes] = {};
    int blocks_per_sm = 0;                 // electron grid = SMs x this (0: occupancy limit)
    int field_threads = 256;               // threads of each CTA of an instance's field step
    int field_cluster = 0;                 // CTAs per instance's field step (0: from the largest grid)
    int electron_threads = 256;            // threads of the default split-mode electron block
    int electron_ppt = 2;                  // particles per thread of the default split-mode electron step
    bool any_chem = false;                 // some admitted discharge has recombination or metastables
    bool any_kin = false;                  // some admitted discharge has kinetic ions
    bool field_split = false;              // FP64 batch whose field step takes the split-mode arithmetic
    InstDev *d_inst_ion = nullptr;         // ion descriptors, slot for slot (zero: none)
    int64_t *d_prefix_ion = nullptr;       // kMaxLanes x (max_inst + 1)
    int64_t *d_prefix1_ion = nullptr;
    int occ_per_sm = 0;
    std::vector<Slot> slots;
    int64_t hbm_cap = 0, hbm_used = 0;
    int max_nodes = 0, max_bins = 0, max_xs = 0;
    LaunchCfg cfg{};
    int sort_interval = kDefaultSort;
    int since_sort = 0;
    cudaGraphExec_t graph = nullptr;
    int num_sms = 0;
    InstDev *h_stage = nullptr;  // pinned, max_inst entries
    // launch accounting and optional per-kernel timing
    int64_t launches = 0, steps = 0;
    bool profiling = false;
    bool pending = false;         // events of the last graph launch not read yet
    std::vector<cudaEvent_t> ev;  // per lane: 3 per step + 2 per sort of a chunk
    double ms[4] = {0, 0, 0, 0};  // electron, field, sort, ion
    int64_t nt[4] = {0, 0, 0, 0};
    // serving without host waits on the batch's stream: status snapshots taken
    // in stream order (a ring, consumed oldest first), a side stream for reads
    // of finished slots, pinned staging buffers for admissions
    static constexpr int kSnaps = 4;
    InstDev *h_snap[kSnaps] = {};      // pinned, max_inst entries each
    InstDev *h_snap_ion[kSnaps] = {};  // pinned, the ion descriptors
    cudaEvent_t ev_snap[kSnaps] = {};
    int snap_head = 0, snap_count = 0;  // next to consume, snapshots in flight
    int snap_last = -1;                 // the snapshot last consumed (kept until the next poll)
    int64_t snap_issued = 0;            // snapshots ever queued
    int64_t snap_seq[kSnaps] = {};      // sequence number of each ring entry
    cudaStream_t rstream = nullptr;
    // moments snapshots (hyb_batch_snapshot_moments): every taken slot's time
    // sums packed by one kernel and copied to pinned memory in stream order,
    // two entries used in turn
    struct MomentSnap {
        int64_t *h_off = nullptr;   // pinned, max_inst + 1 offsets (doubles) into the packed data
        std::vector<int64_t> who;   // per slot: the admission it held when the snapshot was queued
        double *h = nullptr;        // pinned, the packed data
        size_t cap = 0;             // doubles h holds
        cudaEvent_t ev = nullptr;
        bool queued = false;
    };
    MomentSnap msnap[2];
    int msnap_cur = -1;             // the entry last queued
    int64_t admissions = 0;         // discharges ever admitted
    int64_t *d_moff = nullptr;      // device copy of the offsets
    double *d_mpack = nullptr;      // device packed data
    size_t mpack_cap = 0;
    struct Staging {
        char *p = nullptr;
        size_t n = 0;
        cudaEvent_t ev = nullptr;
        bool used = false;
    };
    std::vector<Staging> stage;
};

struct hyb_discharge {
    hyb_batch *b;
    int slot;
};

namespace {

int64_t live_count(const InstDev &K)
{
    return K.n_base + (int64_t)(K.ctr[C_BIRTH_IZ] + K.ctr[C_SEE0] + K.ctr[C_SEE1] + K.ctr[C_PEN] + K.ctr[C_POOL]) -
           (int64_t)(K.ctr[C_LOSS0] + K.ctr[C_LOSS1] + K.ctr[C_REC]);
}

int fetch_inst(hyb_batch *b, int slot)
{
    CK(cudaMemcpyAsync(&b->h_stage[slot], &b->d_inst[slot], sizeof(InstDev), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return HYB_OK;
}

int status_code(unsigned st)
{
    if (st & HYB_STATUS_NONFINITE) return fail(HYB_ERR_NONFINITE, "non-finite field or ion density");
    if (st & HYB_STATUS_CAPACITY) return fail(HYB_ERR_CAPACITY, "particle store full: births dropped");
    if (st & HYB_STATUS_UNSTABLE) return fail(HYB_ERR_UNSTABLE, "ion-fluid update outside its stability range");
    return HYB_OK;
}

int drop_graph(hyb_batch *b)
{
    if (b->graph) {
        CK(cudaGraphExecDestroy(b->graph));
        b->graph = nullptr;
    }
    return HYB_OK;
}

// threads of an electron-kernel block: the tuning's for the default split
// step, 256 for the FP64 path and the reaction and ion-birth variants
int electron_threads_of(const hyb_batch *b)
{
    return (b->precision != HYB_FP32_SPLIT || b->any_chem || b->any_kin) ? kElectronBlock : b->electron_threads;
}

// particles per electron thread: the tuning's for the default split step, 2
// for the others
int electron_ppt_of(const hyb_batch *b)
{
    return (b->precision != HYB_FP32_SPLIT || b->any_chem || b->any_kin) ? 2 : b->electron_ppt;
}

// electron launch shape (block, shared memory, grid) for the current grids,
// EEDF and block size
int reconfigure(hyb_batch *b)
{
    const int th = electron_threads_of(b);
    const int ppt = electron_ppt_of(b);
    b->cfg.block = th;
    b->cfg.ppt = ppt;
    // the deposit pass at admission and the reaction variants run 256-thread
    // blocks with this shared memory: room for at least 256 threads' rows
    b->cfg.smem = electron_smem_bytes(b->precision, b->max_nodes, b->max_bins, std::max(th, kElectronBlock), b->max_xs);
    int per_sm = electron_blocks_per_sm(b->precision, b->cfg.smem, th, ppt);
    if (per_sm < 1) return fail(HYB_ERR_ARG, "grid too large for the electron kernel's shared memory");
    b->occ_per_sm = per_sm;
    b->cfg.grid = b->num_sms * (b->blocks_per_sm > 0 ? b->blocks_per_sm : per_sm);
    return drop_graph(b);
}

int configure(hyb_batch *b, int nodes, int bins, int xs)
{
    if (nodes <= b->max_nodes && bins <= b->max_bins && xs <= b->max_xs) return HYB_OK;
    b->max_nodes = std::max(b->max_nodes, nodes);
    b->max_bins = std::max(b->max_bins, bins);
    b->max_xs = std::max(b->max_xs, xs);
    return reconfigure(b);
}

int lane_first(const hyb_batch *b, int k) { return k * b->per_lane; }
// the field step takes the split mode's arithmetic (reciprocals, table slopes)
bool field_fast(const hyb_batch *b) { return b->precision == HYB_FP32_SPLIT || b->field_split; }
// CTAs per instance's field step: the tuning's, or automatic; with several
// lanes at most 8, which the GPU co-schedules beside other lanes' electron
// blocks more readily than 16 (measured on the 64-discharge mix)
int field_cluster_of(const hyb_batch *b) { return b->field_cluster > 0 ? b->field_cluster : (b->lanes > 1 ? -8 : 0); }
InstDev *lane_inst_ion(const hyb_batch *b, int k);
int64_t *lane_prefix_ion(const hyb_batch *b, int k);
int lane_count(const hyb_batch *b, int k) { return std::max(0, std::min(b->per_lane, b->max_inst - k * b->per_lane)); }
int64_t *lane_prefix(const hyb_batch *b, int k) { return b->d_prefix + (size_t)k * (b->max_inst + 1); }
unsigned *lane_ticket(const hyb_batch *b, int k) { return b->d_ticket + k; }
cudaStream_t lane_stream(const hyb_batch *b, int k) { return k == 0 ? b->stream : b->lstream[k]; }
InstDev *lane_inst(const hyb_batch *b, int k) { return b->d_inst + lane_first(b, k); }
InstDev *lane_inst_ion(const hyb_batch *b, int k) { return b->d_inst_ion + lane_first(b, k); }
int64_t *lane_prefix_ion(const hyb_batch *b, int k) { return b->d_prefix_ion + (size_t)k * (b->max_inst + 1); }

// Chunk prefixes of every lane (after an admission, eviction or relayout).
int prefix_all(hyb_batch *b)
{
    for (int k = 0; k < b->lanes; ++k)
        if (lane_count(b, k) > 0) CK(launch_prefix(lane_inst(b, k), lane_count(b, k), lane_prefix(b, k), b->stream));
    return HYB_OK;
}

constexpr int kSortKernels = 5;
constexpr int kChunkTarget = 100;  // steps per captured graph (a multiple of the sort interval)

// kernels per lane of a step and of a sort
int step_kernels(const hyb_batch *b) { return 2 + (b->any_kin ? 2 : 0); }
int sort_kernels(const hyb_batch *b) { return kSortKernels + (b->any_kin ? 1 + kSortKernels : 0); }

int chunk_len(const hyb_batch *b)
{
    const int k = b->sort_interval;
    const int m = kChunkTarget / k > 0 ? kChunkTarget / k : 1;
    return k * m;
}

size_t events_per_lane(const hyb_batch *b)
{
    const int GL = chunk_len(b);
    return 4 * (size_t)GL + 2 * (size_t)(GL / b->sort_interval);
}

int ensure_events(hyb_batch *b)
{
    const size_t need = events_per_lane(b) * (size_t)b->lanes;
    while (b->ev.size() < need) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        b->ev.push_back(e);
    }
    return HYB_OK;
}

// Timing event on a lane's stream; inside a stream capture it must become an
// event-record node of the graph (cudaEventRecordExternal).
int record(cudaStream_t s, cudaEvent_t e)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &st));
    if (st == cudaStreamCaptureStatusActive)
        CK(cudaEventRecordWithFlags(e, s, cudaEventRecordExternal));
    else
        CK(cudaEventRecord(e, s));
    return HYB_OK;
}

cudaEvent_t lane_event(const hyb_batch *b, int lane, size_t i) { return b->ev[(size_t)lane * events_per_lane(b) + i]; }

// One step of one lane on stream s; with profiling, the lane's events
// 4k..4k+3 bracket the electron kernel, the ion kernels (kinetic ions) and
// the field kernel.
int launch_step(hyb_batch *b, int k, int lane, cudaStream_t s)
{
    int rc;
    const int n = lane_count(b, lane);
    const size_t e = 4 * (size_t)k;
    if (b->profiling && (rc = record(s, lane_event(b, lane, e)))) return rc;
    CK(launch_electron_step(lane_inst(b, lane), n, lane_prefix(b, lane), b->precision, b->cfg, s, b->any_chem,
                            b->any_kin));
    if (b->profiling && (rc = record(s, lane_event(b, lane, e + 1)))) return rc;
    if (b->any_kin) {  // the ions of the step, after the electrons' births
        CK(launch_ion_prefix(lane_inst_ion(b, lane), n, lane_prefix_ion(b, lane), s));
        CK(launch_ion_step(lane_inst_ion(b, lane), n, lane_prefix_ion(b, lane), 0, b->cfg.grid, b->max_nodes,
                           b->precision, s));
    }
    if (b->profiling && (rc = record(s, lane_event(b, lane, e + 2)))) return rc;
    // with one lane the field step may start while the particle kernel's last
    // blocks finish (with several, the other lanes fill that time and early
    // field CTAs would hold SMs they need)
    const bool early = b->lanes == 1 && !b->profiling && !b->any_kin;
    CK(launch_field(lane_inst(b, lane), n, lane_prefix(b, lane), lane_ticket(b, lane), field_fast(b),
                    b->max_nodes, b->field_threads, s, field_cluster_of(b), early));
    if (b->profiling && (rc = record(s, lane_event(b, lane, e + 3)))) return rc;
    return HYB_OK;
}

// The cell sort of one lane; with profiling, sort j of a chunk is bracketed
// by two of the lane's events.
int launch_sort_all(hyb_batch *b, int j, int lane, cudaStream_t s)
{
    int rc;
    const size_t s0 = 4 * (size_t)chunk_len(b) + 2 * (size_t)j;
    if (b->profiling && (rc = record(s, lane_event(b, lane, s0)))) return rc;
    CK(launch_sort(lane_inst(b, lane), lane_count(b, lane), lane_prefix(b, lane), b->precision, b->cfg, s));
    if (b->any_kin) {  // compaction and cell sort of the ions (the batch's layout)
        CK(launch_ion_prefix(lane_inst_ion(b, lane), lane_count(b, lane), lane_prefix_ion(b, lane), s));
        CK(launch_sort(lane_inst_ion(b, lane), lane_count(b, lane), lane_prefix_ion(b, lane), b->precision, b->cfg, s));
    }
    if (b->profiling && (rc = record(s, lane_event(b, lane, s0 + 1)))) return rc;
    return HYB_OK;
}

// Sum the device times of `steps` profiled steps and `sorts` sorts of every
// lane (lanes that overlap each count their own launch's duration).
int collect_times(hyb_batch *b, int steps, int sorts)
{
    CK(cudaStreamSynchronize(b->stream));
    const size_t s0 = 4 * (size_t)chunk_len(b);
    for (int lane = 0; lane < b->lanes; ++lane) {
        for (int k = 0; k < steps; ++k) {
            const size_t e = 4 * (size_t)k;
            float t0 = 0.f, ti = 0.f, t1 = 0.f;
            CK(cudaEventElapsedTime(&t0, lane_event(b, lane, e), lane_event(b, lane, e + 1)));
            CK(cudaEventElapsedTime(&ti, lane_event(b, lane, e + 1), lane_event(b, lane, e + 2)));
            CK(cudaEventElapsedTime(&t1, lane_event(b, lane, e + 2), lane_event(b, lane, e + 3)));
            b->ms[0] += t0;
            b->ms[1] += t1;
            b->nt[0] += 1;
            b->nt[1] += 1;
            if (b->any_kin) {
                b->ms[3] += ti;
                b->nt[3] += 1;
            }
        }
        for (int j = 0; j < sorts; ++j) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, lane_event(b, lane, s0 + 2 * (size_t)j),
                                    lane_event(b, lane, s0 + 2 * (size_t)j + 1)));
            b->ms[2] += t;
            b->nt[2] += 1;
        }
    }
    return HYB_OK;
}

int flush_pending(hyb_batch *b)
{
    if (!b->pending) return HYB_OK;
    b->pending = false;
    const int GL = chunk_len(b);
    return collect_times(b, GL, GL / b->sort_interval);
}

// Split the slots into n lanes; streams and fork/join events are created on
// first use.  Waits for the batch's stream.
int set_lanes(hyb_batch *b, int n)
{
    if (n < 1 || n > kMaxLanes || n > b->max_inst) return fail(HYB_ERR_ARG, "lanes must be in [1, %d]",
                                                               std::min(kMaxLanes, b->max_inst));
    int rc = flush_pending(b);
    if (rc) return rc;
    CK(cudaStreamSynchronize(b->stream));
    for (int k = 1; k < n; ++k)
        if (!b->lstream[k]) CK(cudaStreamCreateWithFlags(&b->lstream[k], cudaStreamNonBlocking));
    for (int k = 0; k < n; ++k)
        if (!b->ev_join[k]) CK(cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming));
    if (!b->ev_fork) CK(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    rc = drop_graph(b);
    if (rc) return rc;
    b->lanes = n;
    b->per_lane = (b->max_inst + n - 1) / n;
    b->lanes = (b->max_inst + b->per_lane - 1) / b->per_lane;  // no empty trailing lane
    return prefix_all(b);
}


// Graph of one chunk: per lane, sort_interval-long runs of steps, each
// followed by the cell sort; lanes are parallel branches forked from and
// joined back into the batch's stream.
int build_graph(hyb_batch *b)
{
    if (b->profiling) {
        int rc0 = ensure_events(b);
        if (rc0) return rc0;
    }
    const int GL = chunk_len(b);
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = HYB_OK;
    cudaError_t e = cudaSuccess;
    if (b->lanes > 1) {
        e = cudaEventRecord(b->ev_fork, b->stream);
        for (int lane = 1; lane < b->lanes && e == cudaSuccess; ++lane)
            e = cudaStreamWaitEvent(b->lstream[lane], b->ev_fork, 0);
        if (e != cudaSuccess) rc = fail(HYB_ERR_CUDA, "fork: %s", cudaGetErrorString(e));
    }
    for (int lane = 0; lane < b->lanes && rc == HYB_OK; ++lane) {
        const cudaStream_t s = lane_stream(b, lane);
        for (int k = 0; k < GL && rc == HYB_OK; ++k) {
            rc = launch_step(b, k, lane, s);
            if (rc == HYB_OK && (k + 1) % b->sort_interval == 0)
                rc = launch_sort_all(b, (k + 1) / b->sort_interval - 1, lane, s);
        }
    }
    for (int lane = 1; lane < b->lanes && rc == HYB_OK; ++lane) {
        e = cudaEventRecord(b->ev_join[lane], b->lstream[lane]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_join[lane], 0);
        if (e != cudaSuccess) rc = fail(HYB_ERR_CUDA, "join: %s", cudaGetErrorString(e));
    }
    e = cudaStreamEndCapture(b->stream, &g);
    if (rc != HYB_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    CK(e);
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return HYB_OK;
}

// (Re)initialise one slot's field from its particles: deposit, Poisson at the
// current time, then a cell sort of that instance alone.
int reinit_slot(hyb_batch *b, int slot, bool sort)
{
    InstDev *K = &b->d_inst[slot];
    CK(launch_prefix_one(K, b->d_prefix1, b->stream));
    CK(launch_deposit_init(K, 1, b->d_prefix1, b->precision, b->cfg, b->stream));
    if (b->slots[slot].h.ion) {  // kinetic ions: their charge assignment first
        InstDev *I = &b->d_inst_ion[slot];
        CK(launch_prefix_one(I, b->d_prefix1_ion, b->stream));
        CK(launch_ion_step(I, 1, b->d_prefix1_ion, 1, b->cfg.grid, b->max_nodes, b->precision, b->stream));
    }
    CK(launch_field(K, 1, b->d_prefix1, b->d_ticket1, field_fast(b), b->max_nodes, b->field_threads,
                    b->stream, field_cluster_of(b)));
    if (sort) {
        CK(launch_prefix_one(K, b->d_prefix1, b->stream));
        CK(launch_sort(K, 1, b->d_prefix1, b->precision, b->cfg, b->stream));
    }
    return HYB_OK;
}

int set_mutable(hyb_batch *b, int slot, int64_t n_slots, int init_pending)
{
    // write n_slots / n_slots_step / init_pending of the device struct
    Slot &S = b->slots[slot];
    CK(cudaStreamSynchronize(b->stream));
    int rc = fetch_inst(b, slot);
    if (rc) return rc;
    InstDev h = b->h_stage[slot];
    if (init_pending == 1 && (int64_t)h.n_slots != n_slots) {
        // a new particle set: keep live = n_base + births - losses equal to it
        h.n_base = n_slots - (live_count(h) - h.n_base);
    }
    h.n_slots = (unsigned long long)n_slots;
    h.n_slots_step = n_slots;
    h.init_pending = init_pending;
    CK(cudaMemcpyAsync(&b->d_inst[slot], &h, sizeof h, cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    (void)S;
    return HYB_OK;
}

// A pinned staging buffer of at least `need` bytes whose earlier copies have
// completed (a new one if none is free); stage_release records the copies
// queued from it.
int stage_acquire(hyb_batch *b, size_t need, char **out)
{
    for (auto &x : b->stage) {
        if (x.used || x.n < need) continue;
        const cudaError_t q = cudaEventQuery(x.ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return fail(HYB_ERR_CUDA, "staging event: %s", cudaGetErrorString(q));
        x.used = true;
        *out = x.p;
        return HYB_OK;
    }
    hyb_batch::Staging x;
    x.n = need > ((size_t)256 << 10) ? need : ((size_t)256 << 10);
    CK(cudaHostAlloc((void **)&x.p, x.n, cudaHostAllocDefault));
    CK(cudaEventCreateWithFlags(&x.ev, cudaEventDisableTiming));
    x.used = true;
    b->stage.push_back(x);
    *out = x.p;
    return HYB_OK;
}

int stage_release(hyb_batch *b, char *p)
{
    for (auto &x : b->stage)
        if (x.p == p) {
            x.used = false;
            CK(cudaEventRecord(x.ev, b->stream));
        }
    return HYB_OK;
}

int admit(hyb_batch *b, const hyb_params *p, int64_t n_steps, int *slot_out)
{
    int rc = validate(p);
    if (rc) return rc;
    if (p->precision != b->precision) return fail(HYB_ERR_ARG, "precision differs from the batch's");
    // a free slot in the lane holding the fewest initial particles, so that
    // the lanes' chains stay about equally long
    int slot = -1;
    double best_load = 0.0;
    for (int k = 0; k < b->lanes; ++k) {
        double load = 0.0;
        int free_i = -1;
        for (int i = lane_first(b, k); i < lane_first(b, k) + lane_count(b, k); ++i) {
            if (b->slots[i].used)
                load += (double)b->slots[i].p.n_particles;
            else if (free_i < 0)
                free_i = i;
        }
        if (free_i >= 0 && (slot < 0 || load < best_load)) {
            slot = free_i;
            best_load = load;
        }
    }
    if (slot < 0) return fail(HYB_ERR_OOM, "no free slot in the batch");
    const Layout L = layout_of(*p);
    if (b->hbm_cap > 0 && b->hbm_used + (int64_t)L.total > b->hbm_cap)
        return fail(HYB_ERR_OOM, "HBM cap: %lld + %lld > %lld bytes", (long long)b->hbm_used, (long long)L.total,
                    (long long)b->hbm_cap);
    rc = configure(b, p->n_cells + 1, bins_of(*p) + 1, p->n_xs);
    if (rc) return rc;

    Slot &S = b->slots[slot];
    std::vector<double> xs, tab;
    std::vector<float4> xsf;
    derive(*p, S.h, xs, xsf, tab);
    void *mem = nullptr;
    cudaError_t e = cudaMallocAsync(&mem, L.total, b->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HYB_ERR_OOM, "cudaMallocAsync(%zu): %s", L.total, cudaGetErrorString(e));
    }
    char *base = (char *)mem;
    bind_pointers(*p, L, base, S.h, &S.hi);
    CK(cudaMemsetAsync(base + L.grid_off, 0, L.total - L.grid_off, b->stream));
    const int G = S.h.G;
    std::vector<double> xr(p->n_xs, 0.0);
    std::vector<float> xrf(p->n_xs, 0.0f);
    if (p->xs_rec)
        for (int i = 0; i < p->n_xs; ++i) {
            xr[i] = p->xs_rec[i];
            xrf[i] = S.h.rec_svmax > 0 ? (float)(p->xs_rec[i] / S.h.rec_svmax) : 0.0f;
        }
    S.h.active = 0;
    S.h.cur = 0;
    S.h.step = 0;
    S.h.target_step = n_steps > 0 ? n_steps : 0;
    S.h.n_slots = (unsigned long long)p->n_particles;
    S.h.n_slots_step = p->n_particles;
    S.h.n_base = p->n_particles;
    S.h.init_pending = 1;
    if (p->n_particles > S.h.capacity) return fail(HYB_ERR_CAPACITY, "n_particles exceeds capacity");
    const bool kin = p->ion_model == HYB_ION_KINETIC;
    if (kin) {
        // the ion descriptor: the electron one's constants and grids, the ion
        // buffers bound above, particles in the batch's precision, its own counts
        InstDev I = S.h;
        I.buf[0] = S.hi.buf[0];
        I.buf[1] = S.hi.buf[1];
        I.cell_cnt = S.hi.cell_cnt;
        I.precision = p->precision;
        I.cur = 0;
        I.n_slots = (unsigned long long)p->n_particles;
        I.n_slots_step = p->n_particles;
        I.n_base = p->n_particles;
        I.init_pending = 0;
        I.ion = nullptr;
        I.elec = &b->d_inst[slot];
        S.hi = I;
        S.h.ion = &b->d_inst_ion[slot];
    } else {
        S.h.ion = nullptr;
    }
    // every host input goes through one pinned staging buffer, so that the
    // copies are queued without the host waiting for the work already queued
    const size_t sz_grid = 8 * (size_t)G;
    const size_t need = 2 * sz_grid + 8 * xs.size() + 16 * xsf.size() + 8 * tab.size() + 8 * xr.size() +
                        4 * xrf.size() + 2 * sizeof(InstDev) + 8 * 16;
    char *st = nullptr;
    int rc2 = stage_acquire(b, need, &st);
    if (rc2) return rc2;
    size_t off = 0;
    auto put = [&](void *dev, const void *src, size_t n) -> cudaError_t {
        off = (off + 15) & ~(size_t)15;
        memcpy(st + off, src, n);
        const cudaError_t e2 = cudaMemcpyAsync(dev, st + off, n, cudaMemcpyHostToDevice, b->stream);
        off += n;
        return e2;
    };
    {
        std::vector<double> ni(G, p->n0_m3);
        CK(put(S.h.ni, ni.data(), sz_grid));
    }
    CK(put((void *)S.h.xs, xs.data(), 8 * xs.size()));
    CK(put((void *)S.h.xsf, xsf.data(), 16 * xsf.size()));
    CK(put((void *)S.h.tab, tab.data(), 8 * tab.size()));
    CK(put((void *)S.h.xs_rec, xr.data(), 8 * xr.size()));
    CK(put((void *)S.h.xs_recf, xrf.data(), 4 * xrf.size()));
    if (p->metastables) {
        std::vector<double> met0(G, p->met_n0_m3);  // metastables: n0 inside, 0 at the electrodes
        met0[0] = met0[G - 1] = 0.0;
        CK(put(S.h.met, met0.data(), sz_grid));
    }
    if (kin)
        CK(put(&b->d_inst_ion[slot], &S.hi, sizeof(InstDev)));
    else
        CK(cudaMemsetAsync(&b->d_inst_ion[slot], 0, sizeof(InstDev), b->stream));
    CK(put(&b->d_inst[slot], &S.h, sizeof(InstDev)));
    rc2 = stage_release(b, st);
    if (rc2) return rc2;
    if (kin) CK(launch_load_ions(&b->d_inst_ion[slot], p->n_particles, b->stream));
    const double vth = sqrt(kQe * p->te0_ev / kMe);
    CK(launch_load(&b->d_inst[slot], p->n_particles, vth, p->precision, b->stream));
    rc = reinit_slot(b, slot, true);
    if (rc) return rc;
    CK(launch_set_active(&b->d_inst[slot], 1, S.h.target_step, b->stream));
    rc = prefix_all(b);
    if (rc) return rc;
    S.used = true;
    S.reported = false;
    S.p = *p;
    S.p.tab_eon_td = S.p.tab_mu = S.p.tab_nu = nullptr;
    S.p.xs_ev = S.p.xs_el = S.p.xs_exc = S.p.xs_ion = S.p.xs_rec = nullptr;
    if ((S.h.rec_on || S.h.met_on) && !b->any_chem) {
        // the electron step switches to its variant with recombination and the metastable source
        b->any_chem = true;
        rc = reconfigure(b);
        if (rc) return rc;
    }
    if (kin && !b->any_kin) {  // from now on every step also runs the ion kernels
        b->any_kin = true;
        rc = reconfigure(b);
        if (rc) return rc;
    }
    S.mem = mem;
    S.bytes = (int64_t)L.total;
    S.target = S.h.target_step;
    S.admit_after = b->snap_issued;
    S.admission = ++b->admissions;
    b->hbm_used += S.bytes;
    *slot_out = slot;
    if (S.h.nu_max * S.h.dt > 0.1) {
        fail(HYB_WARN_DT_NULLCOLL, "nu_max*dt = %.3g exceeds 0.1", S.h.nu_max * S.h.dt);
        return HYB_WARN_DT_NULLCOLL;
    }
    return HYB_OK;
}

int advance(hyb_batch *b, int64_t n)
{
    if (n < 0) return fail(HYB_ERR_ARG, "negative step count");
    int rc;
    if (b->profiling) {
        rc = ensure_events(b);
        if (rc) return rc;
    }
    const int GL = chunk_len(b);
    while (n > 0) {
        rc = flush_pending(b);
        if (rc) return rc;
        if (b->since_sort == 0 && n >= GL) {
            if (!b->graph) {
                rc = build_graph(b);
                if (rc) return rc;
            }
            CK(cudaGraphLaunch(b->graph, b->stream));
            b->launches += b->lanes * (step_kernels(b) * (int64_t)GL + sort_kernels(b) * (int64_t)(GL / b->sort_interval));
            b->steps += GL;
            n -= GL;
            b->pending = b->profiling;
            continue;
        }
        // a single step: the lanes one after the other on the batch's stream
        const bool sort_now = b->since_sort + 1 == b->sort_interval;
        for (int lane = 0; lane < b->lanes; ++lane) {
            rc = launch_step(b, 0, lane, b->stream);
            if (rc) return rc;
            if (sort_now && (rc = launch_sort_all(b, 0, lane, b->stream))) return rc;
        }
        b->launches += b->lanes * (step_kernels(b) + (sort_now ? sort_kernels(b) : 0));
        b->steps += 1;
        --n;
        b->since_sort = sort_now ? 0 : b->since_sort + 1;
        if (b->profiling) {
            rc = collect_times(b, 1, sort_now ? 1 : 0);
            if (rc) return rc;
        }
    }
    return HYB_OK;
}

int64_t total_pushes(hyb_batch *b)
{
    int64_t n = 0;
    for (int i = 0; i < b->max_inst; ++i)
        if (b->slots[i].used) n += (int64_t)b->h_stage[i].ctr[C_PUSH];
    return n;
}

int fetch_all(hyb_batch *b)
{
    CK(cudaMemcpyAsync(b->h_stage, b->d_inst, sizeof(InstDev) * (size_t)b->max_inst, cudaMemcpyDeviceToHost,
                       b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return HYB_OK;
}

int set_tuning(hyb_batch *b, const hyb_tuning &t)
{
    if (t.sort_interval < 1 || t.sort_interval > 1000) return fail(HYB_ERR_ARG, "sort_interval must be in [1, 1000]");
    if (t.blocks_per_sm < 0 || t.blocks_per_sm > 64) return fail(HYB_ERR_ARG, "blocks_per_sm must be in [0, 64]");
    if (t.field_threads != 256 && t.field_threads != 512 && t.field_threads != 1024)
        return fail(HYB_ERR_ARG, "field_threads must be 256, 512 or 1024");
    if (t.field_cluster < 0 || t.field_cluster > 16) return fail(HYB_ERR_ARG, "field_cluster must be in [0, 16]");
    const int eth = t.electron_threads == 0 ? kElectronBlock : t.electron_threads;
    if (eth != 128 && eth != 256 && eth != 512) return fail(HYB_ERR_ARG, "electron_threads must be 0, 128, 256 or 512");
    const int ppt = t.particles_per_thread == 0 ? 2 : t.particles_per_thread;
    if (ppt != 2 && ppt != 4) return fail(HYB_ERR_ARG, "particles_per_thread must be 0, 2 or 4");
    int rc = flush_pending(b);
    if (rc) return rc;
    if (t.lanes != b->lanes && (rc = set_lanes(b, t.lanes))) return rc;
    if (t.sort_interval != b->sort_interval) {
        if ((rc = drop_graph(b))) return rc;
        b->sort_interval = t.sort_interval;
        b->since_sort = 0;
    }
    if (t.field_threads != b->field_threads) {
        if ((rc = drop_graph(b))) return rc;
        b->field_threads = t.field_threads;
    }
    if (t.field_cluster != b->field_cluster) {
        if ((rc = drop_graph(b))) return rc;
        b->field_cluster = t.field_cluster;
    }
    if (eth != b->electron_threads || ppt != b->electron_ppt) {
        b->electron_threads = eth;
        b->electron_ppt = ppt;
        if (b->max_nodes > 0 && (rc = reconfigure(b))) return rc;
    }
    if (t.blocks_per_sm != b->blocks_per_sm) {
        b->blocks_per_sm = t.blocks_per_sm;
        b->cfg.grid = b->num_sms * (t.blocks_per_sm > 0 ? t.blocks_per_sm : b->occ_per_sm);
        if ((rc = drop_graph(b))) return rc;
    }
    return HYB_OK;
}

hyb_tuning get_tuning(const hyb_batch *b)
{
    hyb_tuning t{};
    t.lanes = b->lanes;
    t.sort_interval = b->sort_interval;
    t.blocks_per_sm = b->blocks_per_sm;
    t.field_threads = b->field_threads;
    t.field_cluster = b->field_cluster;
    t.electron_threads = b->electron_threads;
    t.particles_per_thread = b->electron_ppt;
    t.rate = 0.0;
    return t;
}

// Particle-steps/s of `steps` steps (whole chunks) under tuning t, after one
// untimed chunk that builds the graph.  The steps are real steps of every
// running discharge.
int measure(hyb_batch *b, const hyb_tuning &t, int64_t steps, cudaEvent_t e0, cudaEvent_t e1, double *rate)
{
    int rc = set_tuning(b, t);
    if (rc) return rc;
    if ((rc = advance(b, chunk_len(b)))) return rc;
    if ((rc = fetch_all(b))) return rc;
    const int64_t p0 = total_pushes(b);
    CK(cudaEventRecord(e0, b->stream));
    if ((rc = advance(b, steps))) return rc;
    CK(cudaEventRecord(e1, b->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if ((rc = fetch_all(b))) return rc;
    *rate = ms > 0.f ? (double)(total_pushes(b) - p0) / (ms * 1e-3) : 0.0;
    return HYB_OK;
}

// Coordinate search over lanes, then the sort interval, then the electron
// grid, each trial timed on the batch's own running discharges.
int autotune(hyb_batch *b, int32_t trial_steps, hyb_tuning *out)
{
    if (trial_steps < 1) return fail(HYB_ERR_ARG, "trial_steps must be positive");
    if (b->profiling) return fail(HYB_ERR_ARG, "switch profiling off before tuning");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    hyb_tuning best = get_tuning(b);
    best.rate = -1.0;
    int rc = HYB_OK;
    // every trial's layout and rate, for the final re-timing of the leaders
    std::vector<hyb_tuning> tried;
    auto same = [](const hyb_tuning &x, const hyb_tuning &y) {
        return x.lanes == y.lanes && x.sort_interval == y.sort_interval && x.blocks_per_sm == y.blocks_per_sm &&
               x.field_threads == y.field_threads && x.field_cluster == y.field_cluster &&
               x.electron_threads == y.electron_threads && x.particles_per_thread == y.particles_per_thread;
    };
    auto trial = [&](hyb_tuning t) {
        if (rc) return;
        const int64_t GL = chunk_len(b);
        const int64_t steps = ((trial_steps + GL - 1) / GL) * GL;
        double r = 0.0;
        rc = measure(b, t, steps, e0, e1, &r);
        if (rc != HYB_OK) return;
        t.rate = r;
        bool seen = false;
        for (auto &x : tried)
            if (same(x, t)) {
                x.rate = std::max(x.rate, r);
                seen = true;
            }
        if (!seen) tried.push_back(t);
        if (r > best.rate) best = t;
    };
    const int lane_opts[5] = {1, 2, 4, 8, 16};
    for (int l : lane_opts) {
        if (l > std::min(kMaxLanes, b->max_inst)) break;
        hyb_tuning t = best;
        t.lanes = l;
        if (l == best.lanes && best.rate >= 0) continue;
        trial(t);
    }
    const int sort_opts[4] = {10, 20, 50, 100};
    const hyb_tuning after_lanes = best;
    for (int k : sort_opts) {
        if (k == after_lanes.sort_interval) continue;
        hyb_tuning t = after_lanes;
        t.sort_interval = k;
        trial(t);
    }
    const hyb_tuning after_sort = best;
    {
        hyb_tuning t = after_sort;
        t.blocks_per_sm = after_sort.blocks_per_sm == 0 ? 2 * b->occ_per_sm : 0;
        trial(t);
    }
    const hyb_tuning after_grid = best;
    const int field_opts[3] = {256, 512, 1024};
    for (int f : field_opts) {
        if (f == after_grid.field_threads) continue;
        hyb_tuning t = after_grid;
        t.field_threads = f;
        trial(t);
    }
    const hyb_tuning after_field = best;
    const int cluster_opts[6] = {0, 1, 2, 4, 8, 16};
    for (int c : cluster_opts) {
        if (c == after_field.field_cluster) continue;
        hyb_tuning t = after_field;
        t.field_cluster = c;
        trial(t);
    }
    if (b->precision == HYB_FP32_SPLIT && !b->any_chem && !b->any_kin) {
        // the default split step's block size and particles per thread
        const hyb_tuning after_cluster = best;
        const int thread_opts[3] = {128, 256, 512};
        const int ppt_opts[2] = {2, 4};
        for (int th : thread_opts)
            for (int v : ppt_opts) {
                if (th == after_cluster.electron_threads && v == after_cluster.particles_per_thread) continue;
                hyb_tuning t = after_cluster;
                t.electron_threads = th;
                t.particles_per_thread = v;
                trial(t);
            }
    }
    // the lane count once more, with everything else as chosen (how well the
    // lanes overlap depends on the block sizes)
    const hyb_tuning after_threads = best;
    for (int l : lane_opts) {
        if (l > std::min(kMaxLanes, b->max_inst)) break;
        if (l == after_threads.lanes) continue;
        hyb_tuning t = after_threads;
        t.lanes = l;
        trial(t);
    }
    // the three fastest layouts once more, each over twice the trial length:
    // single trials differ by about a per cent from run to run, as much as
    // the leading layouts differ from each other
    if (rc == HYB_OK && tried.size() > 1) {
        std::sort(tried.begin(), tried.end(), [](const hyb_tuning &x, const hyb_tuning &y) { return x.rate > y.rate; });
        const int64_t GL = chunk_len(b);
        const int64_t steps = 2 * (((trial_steps + GL - 1) / GL) * GL);
        hyb_tuning win = best;
        double win_rate = -1.0;
        for (size_t i = 0; i < tried.size() && i < 3 && rc == HYB_OK; ++i) {
            double r = 0.0;
            rc = measure(b, tried[i], steps, e0, e1, &r);
            if (rc == HYB_OK && r > win_rate) {
                win = tried[i];
                win_rate = r;
            }
        }
        if (rc == HYB_OK) {
            best = win;
            best.rate = win_rate;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    rc = set_tuning(b, best);
    if (rc) return rc;
    if (out) *out = best;
    return HYB_OK;
}

int sync_status(hyb_batch *b, int slot)
{
    CK(cudaStreamSynchronize(b->stream));
    int rc = fetch_inst(b, slot);
    if (rc) return rc;
    return status_code(b->h_stage[slot].status);
}

int check_slot(hyb_batch *b, int slot)
{
    if (!b) return fail(HYB_ERR_ARG, "NULL batch");
    if (slot < 0 || slot >= b->max_inst || !b->slots[slot].used) return fail(HYB_ERR_ARG, "no discharge in slot %d", slot);
    return HYB_OK;
}

// time-averaged moments of a discharge with descriptor K, copied on stream s
// Pack each slot's time sums (n_e, n_i, Gamma_i, electron weight, weight x
// energy), its EEDF counts and its sample count into one buffer: slot i's
// block is out[off[i] .. off[i + 1]), 5 G + nb + 2 doubles (the counts as their
// bit patterns), or empty for a slot not taken.  A block whose size does not
// match the slot's descriptor gets a NaN sample count.
__global__ void k_pack_moments(const InstDev *insts, const int64_t *off, double *out)
{
    const int slot = blockIdx.x;
    const int64_t a = off[slot], n = off[slot + 1] - a;
    if (n <= 0) return;
    const InstDev &K = insts[slot];
    const int G = K.G, nb = K.eedf_bins;
    double *o = out + a;
    if (n != 5 * (int64_t)G + nb + 2) {
        if (threadIdx.x == 0) o[n - 1] = __longlong_as_double(0x7FF8000000000000ll);
        return;
    }
    const double *src[5] = {K.acc_ne, K.acc_ni, K.acc_gi, K.acc_wn, K.acc_we};
    for (int k = 0; k < 5; ++k)
        for (int j = threadIdx.x; j < G; j += blockDim.x) o[(size_t)k * G + j] = src[k][j];
    for (int j = threadIdx.x; j <= nb; j += blockDim.x) o[5 * (size_t)G + j] = __longlong_as_double((long long)K.eedf[j]);
    if (threadIdx.x == 0) o[5 * (size_t)G + nb + 1] = __longlong_as_double((long long)K.n_samples);
}

// The time averages of hyb_read_moments from the time sums acc (5 G: n_e,
// n_i, Gamma_i, electron weight, weight x energy), the EEDF counts and the
// sample count
void moments_from_sums(const double *acc, const unsigned long long *eedf, int64_t ns, int G, int nb, double bin_w,
                       hyb_moments *out)
{
    out->n_samples = ns;
    for (int j = 0; j < G; ++j) {
        if (out->ne) out->ne[j] = ns ? acc[j] / ns : 0.0;
        if (out->ni) out->ni[j] = ns ? acc[G + j] / ns : 0.0;
        if (out->gamma_i) out->gamma_i[j] = ns ? acc[2 * G + j] / ns : 0.0;
        if (out->mean_energy_ev) out->mean_energy_ev[j] = acc[3 * G + j] > 0 ? acc[4 * G + j] / acc[3 * G + j] : 0.0;
    }
    if (out->eedf) {
        double tot = 0.0;
        for (int k = 0; k <= nb; ++k) tot += (double)eedf[k];
        for (int k = 0; k < nb; ++k) out->eedf[k] = tot > 0 ? (double)eedf[k] / (tot * bin_w) : 0.0;
        out->eedf[nb] = tot > 0 ? (double)eedf[nb] / tot : 0.0;
    }
}

int moments_of(const InstDev &K, cudaStream_t s, hyb_moments *out)
{
    const int G = K.G, nb = K.eedf_bins;
    std::vector<double> acc(5 * (size_t)G);
    std::vector<unsigned long long> eedf(nb + 1);
    double *src[5] = {K.acc_ne, K.acc_ni, K.acc_gi, K.acc_wn, K.acc_we};
    for (int k = 0; k < 5; ++k)
        CK(cudaMemcpyAsync(acc.data() + (size_t)k * G, src[k], 8 * (size_t)G, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(eedf.data(), K.eedf, 8 * (size_t)(nb + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    moments_from_sums(acc.data(), eedf.data(), K.n_samples, G, nb, K.bin_w, out);
    return HYB_OK;
}

int read_moments(hyb_batch *b, int slot, hyb_moments *out)
{
    int rc = check_slot(b, slot);
    if (rc) return rc;
    if (!out) return fail(HYB_ERR_ARG, "NULL output");
    rc = sync_status(b, slot);
    const int r2 = moments_of(b->h_stage[slot], b->stream, out);
    return r2 ? r2 : rc;
}

// counters from a discharge's descriptor (and its ion descriptor, if any)
void fill_counters(const InstDev &K, const InstDev *I, hyb_counters *c)
{
    c->step = K.step;
    c->births_ionization = (int64_t)K.ctr[C_BIRTH_IZ];
    c->births_see[0] = (int64_t)K.ctr[C_SEE0];
    c->births_see[1] = (int64_t)K.ctr[C_SEE1];
    c->losses[0] = (int64_t)K.ctr[C_LOSS0];
    c->losses[1] = (int64_t)K.ctr[C_LOSS1];
    c->collisions[0] = (int64_t)K.ctr[C_EL];
    c->collisions[1] = (int64_t)K.ctr[C_EXC];
    c->collisions[2] = (int64_t)K.ctr[C_IZ];
    c->collisions[3] = (int64_t)K.ctr[C_NULL];
    c->clamps = (int64_t)K.ctr[C_CLAMP];
    c->pushes = (int64_t)K.ctr[C_PUSH];
    c->status = K.status;
    c->particles = live_count(K);
    c->v_rf_amp_v = K.v_rf;
    c->power_last_w_m2 = K.pw_last;
    c->power_periods = K.pw_periods;
    c->recombinations = (int64_t)K.ctr[C_REC];
    c->births_penning = (int64_t)K.ctr[C_PEN];
    c->births_pooling = (int64_t)K.ctr[C_POOL];
    c->ions = c->ion_losses[0] = c->ion_losses[1] = c->ion_collisions = c->ion_pushes = 0;
    if (I) {
        c->ion_losses[0] = (int64_t)I->ctr[C_LOSS0];
        c->ion_losses[1] = (int64_t)I->ctr[C_LOSS1];
        c->ion_collisions = (int64_t)I->ctr[C_EL];
        c->ion_pushes = (int64_t)I->ctr[C_PUSH];
        c->ions = I->n_base + (int64_t)K.ctr[C_BIRTH_IZ] - c->ion_losses[0] - c->ion_losses[1];
    }
}

int read_counters(hyb_batch *b, int slot, hyb_counters *c)
{
    int rc = check_slot(b, slot);
    if (rc) return rc;
    if (!c) return fail(HYB_ERR_ARG, "NULL output");
    rc = sync_status(b, slot);
    InstDev I{};
    const bool kin = b->slots[slot].h.ion != nullptr;
    if (kin) {
        CK(cudaMemcpyAsync(&I, &b->d_inst_ion[slot], sizeof I, cudaMemcpyDeviceToHost, b->stream));
        CK(cudaStreamSynchronize(b->stream));
    }
    fill_counters(b->h_stage[slot], kin ? &I : nullptr, c);
    return rc;
}

int gather_sorted(const InstDev &K, int64_t ns, double *z, double *vx, double *vy, double *vz, uint64_t *id,
                  int64_t cap, int64_t *n, const char *what)
{
    const PartBuf P = K.buf[K.cur];
    std::vector<double> hz(ns), hx(ns), hy(ns), hv(ns);
    std::vector<uint64_t> hid(ns);
    std::vector<char> alive(ns, 0);
    if (ns > 0) {
        CK(cudaMemcpy(hid.data(), P.id, 8 * (size_t)ns, cudaMemcpyDeviceToHost));
        if (K.precision == HYB_FP32_SPLIT) {
            std::vector<int32_t> c(ns);
            std::vector<float> o(ns), fx(ns), fy(ns), fz(ns);
            CK(cudaMemcpy(c.data(), P.c, 4 * (size_t)ns, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(o.data(), P.o, 4 * (size_t)ns, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(fx.data(), P.vxf, 4 * (size_t)ns, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(fy.data(), P.vyf, 4 * (size_t)ns, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(fz.data(), P.vzf, 4 * (size_t)ns, cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < ns; ++i) {
                alive[i] = c[i] >= 0;
                hz[i] = ((double)c[i] + (double)o[i]) * K.dz;
                hx[i] = fx[i];
                hy[i] = fy[i];
                hv[i] = fz[i];
            }
        } else {
            CK(cudaMemcpy(hz.data(), P.z, 8 * (size_t)ns, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(hx.data(), P.vxd, 8 * (size_t)ns, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(hy.data(), P.vyd, 8 * (size_t)ns, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(hv.data(), P.vzd, 8 * (size_t)ns, cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < ns; ++i) alive[i] = hz[i] >= 0.0;
        }
    }
    std::vector<int64_t> idx;
    idx.reserve(ns);
    for (int64_t i = 0; i < ns; ++i)
        if (alive[i]) idx.push_back(i);
    std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t c) { return hid[a] < hid[c]; });
    *n = (int64_t)idx.size();
    if (*n > cap) return fail(HYB_ERR_ARG, "%lld %s exceed the buffers (%lld)", (long long)*n, what, (long long)cap);
    for (size_t k = 0; k < idx.size(); ++k) {
        const int64_t i = idx[k];
        if (z) z[k] = hz[i];
        if (vx) vx[k] = hx[i];
        if (vy) vy[k] = hy[i];
        if (vz) vz[k] = hv[i];
        if (id) id[k] = hid[i];
    }
    return HYB_OK;
}

int read_particles(hyb_batch *b, int slot, double *z, double *vx, double *vy, double *vz, uint64_t *id, int64_t cap,
                   int64_t *n)
{
    int rc = check_slot(b, slot);
    if (rc) return rc;
    rc = sync_status(b, slot);
    const InstDev &K = b->h_stage[slot];
    const int rg = gather_sorted(K, (int64_t)K.n_slots, z, vx, vy, vz, id, cap, n, "live particles");
    return rg ? rg : rc;
}

// the kinetic ions of a slot, alive ones sorted by id
int read_ions(hyb_batch *b, int slot, double *z, double *vx, double *vy, double *vz, uint64_t *id, int64_t cap,
              int64_t *n)
{
    int rc = check_slot(b, slot);
    if (rc) return rc;
    if (!b->slots[slot].h.ion) return fail(HYB_ERR_STATE, "the discharge has fluid ions");
    rc = sync_status(b, slot);
    InstDev I{};
    CK(cudaMemcpy(&I, &b->d_inst_ion[slot], sizeof I, cudaMemcpyDeviceToHost));
    const int rg = gather_sorted(I, std::min((int64_t)I.n_slots, I.capacity), z, vx, vy, vz, id, cap, n, "ions");
    return rg ? rg : rc;
}

// the metastable density, its time average and the last wall fluxes of a slot
int read_metastables(hyb_batch *b, int slot, double *met, double *avg, double *flux)
{
    int rc = check_slot(b, slot);
    if (rc) return rc;
    if (!b->slots[slot].h.met_on) return fail(HYB_ERR_STATE, "the discharge has no metastables");
    rc = sync_status(b, slot);
    const InstDev &K = b->h_stage[slot];
    const int G = K.G;
    if (met) CK(cudaMemcpy(met, K.met, 8 * (size_t)G, cudaMemcpyDeviceToHost));
    if (avg) {
        CK(cudaMemcpy(avg, K.acc_met, 8 * (size_t)G, cudaMemcpyDeviceToHost));
        for (int j = 0; j < G; ++j) avg[j] = K.n_samples ? avg[j] / (double)K.n_samples : 0.0;
    }
    if (flux) {
        flux[0] = K.flux_met[0];
        flux[1] = K.flux_met[1];
    }
    return rc;
}

int free_slot(hyb_batch *b, int slot)
{
    Slot &S = b->slots[slot];
    if (!S.used) return HYB_OK;
    CK(launch_set_active(&b->d_inst[slot], 0, 0, b->stream));
    CK(cudaMemsetAsync(&b->d_inst_ion[slot], 0, sizeof(InstDev), b->stream));  // before its buffers go
    int rc = prefix_all(b);
    if (rc) return rc;
    CK(cudaFreeAsync(S.mem, b->stream));  // in stream order: later admissions allocate after it
    b->hbm_used -= S.bytes;
    S = Slot{};
    return HYB_OK;
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

const char *hyb_last_error(void) { return g_err.c_str(); }

int hyb_footprint(const hyb_params *p, int64_t *bytes)
{
    int rc = validate(p);
    if (rc) return rc;
    if (!bytes) return fail(HYB_ERR_ARG, "NULL output");
    *bytes = (int64_t)layout_of(*p).total;
    return HYB_OK;
}

int hyb_batch_create(int32_t max_instances, int32_t precision, int64_t hbm_cap_bytes, void *stream, hyb_batch **out)
{
    if (!out) return fail(HYB_ERR_ARG, "NULL output");
    *out = nullptr;
    if (max_instances < 1 || max_instances > HYB_MAX_INSTANCES)
        return fail(HYB_ERR_ARG, "max_instances must be in [1, %d]", HYB_MAX_INSTANCES);
    if (precision != HYB_FP64 && precision != HYB_FP32_SPLIT) return fail(HYB_ERR_ARG, "unknown precision");
    int dev = 0;
    CK(cudaGetDevice(&dev));
    hyb::configure_kernels();
    hyb_batch *b = new hyb_batch();
    b->max_inst = max_instances;
    b->precision = precision;
    b->hbm_cap = hbm_cap_bytes > 0 ? hbm_cap_bytes : 0;
    b->slots.resize(max_instances);
    CK(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev));
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        CK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        b->own_stream = true;
    }
    CK(cudaMalloc(&b->d_inst, sizeof(InstDev) * (size_t)max_instances));
    CK(cudaMemset(b->d_inst, 0, sizeof(InstDev) * (size_t)max_instances));
    const size_t np = (size_t)kMaxLanes * (size_t)(max_instances + 1);
    CK(cudaMalloc(&b->d_prefix, sizeof(int64_t) * np));
    CK(cudaMemset(b->d_prefix, 0, sizeof(int64_t) * np));
    CK(cudaMalloc(&b->d_prefix1, sizeof(int64_t) * 2));
    CK(cudaMalloc(&b->d_ticket, sizeof(unsigned) * (kMaxLanes + 1)));
    CK(cudaMemset(b->d_ticket, 0, sizeof(unsigned) * (kMaxLanes + 1)));
    b->d_ticket1 = b->d_ticket + kMaxLanes;
    CK(cudaMallocHost(&b->h_stage, sizeof(InstDev) * (size_t)max_instances));
    CK(cudaMalloc(&b->d_inst_ion, sizeof(InstDev) * (size_t)max_instances));
    CK(cudaMemset(b->d_inst_ion, 0, sizeof(InstDev) * (size_t)max_instances));
    CK(cudaMalloc(&b->d_prefix_ion, sizeof(int64_t) * np));
    CK(cudaMemset(b->d_prefix_ion, 0, sizeof(int64_t) * np));
    CK(cudaMalloc(&b->d_prefix1_ion, sizeof(int64_t) * 2));
    int rc = configure(b, 3, 2, 2);
    if (rc) return rc;
    rc = set_lanes(b, std::min(kDefaultLanes, max_instances));
    if (rc) return rc;
    *out = b;
    return HYB_OK;
}

int hyb_batch_admit(hyb_batch *b, const hyb_params *p, int64_t n_steps, int32_t *slot)
{
    if (!b || !slot) return fail(HYB_ERR_ARG, "NULL argument");
    int s = -1;
    int rc = admit(b, p, n_steps, &s);
    *slot = s;
    return rc;
}

int hyb_batch_advance(hyb_batch *b, int64_t n_steps)
{
    if (!b) return fail(HYB_ERR_ARG, "NULL batch");
    return advance(b, n_steps);
}

int hyb_batch_poll(hyb_batch *b, int32_t *done, int32_t cap, int32_t *n_done)
{
    if (!b || !n_done) return fail(HYB_ERR_ARG, "NULL argument");
    CK(cudaMemcpyAsync(b->h_stage, b->d_inst, sizeof(InstDev) * (size_t)b->max_inst, cudaMemcpyDeviceToHost,
                       b->stream));
    CK(cudaStreamSynchronize(b->stream));
    int k = 0;
    int rc = HYB_OK;
    for (int i = 0; i < b->max_inst; ++i) {
        Slot &S = b->slots[i];
        if (!S.used || S.reported) continue;
        const InstDev &K = b->h_stage[i];
        const bool finished = S.target > 0 && K.step >= S.target && !K.active;
        const bool failed = (K.status & (HYB_STATUS_NONFINITE | HYB_STATUS_CAPACITY | HYB_STATUS_UNSTABLE)) != 0;
        if (finished || failed) {
            if (k < cap && done) done[k] = i;
            ++k;
            S.reported = true;
            if (failed && rc == HYB_OK) rc = status_code(K.status);
        }
    }
    *n_done = k < cap ? k : cap;
    return rc;
}

int hyb_batch_wait(hyb_batch *b, double timeout_s)
{
    if (!b) return fail(HYB_ERR_ARG, "NULL batch");
    if (!(timeout_s >= 0)) return fail(HYB_ERR_ARG, "timeout must be non-negative");
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t q = cudaStreamQuery(b->stream);
        if (q == cudaSuccess) return HYB_OK;
        if (q != cudaErrorNotReady) return fail(HYB_ERR_CUDA, "cudaStreamQuery: %s", cudaGetErrorString(q));
        const double waited = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (waited >= timeout_s)
            return fail(HYB_ERR_TIMEOUT, "the batch's queued work did not finish within %.3g s", timeout_s);
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

int hyb_batch_snapshot(hyb_batch *b)
{
    if (!b) return fail(HYB_ERR_ARG, "NULL batch");
    // one entry stays for the snapshot last polled, which reads may still use
    if (b->snap_count >= hyb_batch::kSnaps - 1)
        return fail(HYB_ERR_STATE, "%d snapshots not yet polled", b->snap_count);
    const int k = (b->snap_head + b->snap_count) % hyb_batch::kSnaps;
    if (!b->h_snap[k]) {
        CK(cudaHostAlloc((void **)&b->h_snap[k], sizeof(InstDev) * (size_t)b->max_inst, cudaHostAllocDefault));
        CK(cudaHostAlloc((void **)&b->h_snap_ion[k], sizeof(InstDev) * (size_t)b->max_inst, cudaHostAllocDefault));
        CK(cudaEventCreateWithFlags(&b->ev_snap[k], cudaEventDisableTiming));
    }
    CK(cudaMemcpyAsync(b->h_snap[k], b->d_inst, sizeof(InstDev) * (size_t)b->max_inst, cudaMemcpyDeviceToHost,
                       b->stream));
    if (b->any_kin)
        CK(cudaMemcpyAsync(b->h_snap_ion[k], b->d_inst_ion, sizeof(InstDev) * (size_t)b->max_inst,
                           cudaMemcpyDeviceToHost, b->stream));
    CK(cudaEventRecord(b->ev_snap[k], b->stream));
    b->snap_seq[k] = b->snap_issued++;
    ++b->snap_count;
    return HYB_OK;
}

int hyb_batch_poll_snapshot(hyb_batch *b, int32_t *done, int32_t cap, int32_t *n_done)
{
    if (!b || !n_done) return fail(HYB_ERR_ARG, "NULL argument");
    if (b->snap_count == 0) return fail(HYB_ERR_STATE, "no snapshot to poll");
    const int k = b->snap_head;
    CK(cudaEventSynchronize(b->ev_snap[k]));
    b->snap_head = (k + 1) % hyb_batch::kSnaps;
    --b->snap_count;
    b->snap_last = k;
    int m = 0;
    int rc = HYB_OK;
    for (int i = 0; i < b->max_inst; ++i) {
        Slot &S = b->slots[i];
        if (!S.used || S.reported) continue;
        if (b->snap_seq[k] < S.admit_after) continue;  // admitted after the snapshot was queued
        const InstDev &K = b->h_snap[k][i];
        const bool finished = S.target > 0 && K.step >= S.target && !K.active;
        const bool failed = (K.status & (HYB_STATUS_NONFINITE | HYB_STATUS_CAPACITY | HYB_STATUS_UNSTABLE)) != 0;
        if (finished || failed) {
            if (m < cap && done) done[m] = i;
            ++m;
            S.reported = true;
            if (failed && rc == HYB_OK) rc = status_code(K.status);
        }
    }
    *n_done = m < cap ? m : cap;
    return rc;
}

int hyb_batch_read_finished(hyb_batch *b, int32_t slot, hyb_counters *counters, hyb_moments *moments)
{
    if (!b) return fail(HYB_ERR_ARG, "NULL batch");
    if (slot < 0 || slot >= b->max_inst || !b->slots[slot].used) return fail(HYB_ERR_ARG, "no discharge in slot %d", slot);
    if (b->snap_last < 0 || !b->slots[slot].reported)
        return fail(HYB_ERR_STATE, "slot %d was not reported by hyb_batch_poll_snapshot", slot);
    const InstDev &K = b->h_snap[b->snap_last][slot];
    if (K.active) return fail(HYB_ERR_STATE, "slot %d is still running", slot);
    if (counters)
        fill_counters(K, b->slots[slot].h.ion ? &b->h_snap_ion[b->snap_last][slot] : nullptr, counters);
    if (moments) {
        if (!b->rstream) CK(cudaStreamCreateWithFlags(&b->rstream, cudaStreamNonBlocking));
        // the slot has been idle on the GPU since the snapshot: read it beside
        // the chunks queued after it
        CK(cudaStreamWaitEvent(b->rstream, b->ev_snap[b->snap_last], 0));
        const int rc = moments_of(K, b->rstream, moments);
        if (rc) return rc;
    }
    return status_code(K.status);
}

int hyb_batch_snapshot_moments(hyb_batch *b)
{
    if (!b) return fail(HYB_ERR_ARG, "NULL batch");
    const int k = (b->msnap_cur + 1) % 2;
    hyb_batch::MomentSnap &M = b->msnap[k];
    if (!M.ev) {
        CK(cudaEventCreateWithFlags(&M.ev, cudaEventDisableTiming));
        CK(cudaHostAlloc((void **)&M.h_off, sizeof(int64_t) * ((size_t)b->max_inst + 1), cudaHostAllocDefault));
    }
    // the entry's previous copies (two snapshots back) are done before its
    // buffers are written again
    if (M.queued) CK(cudaEventSynchronize(M.ev));
    int64_t total = 0;
    M.who.assign((size_t)b->max_inst, 0);
    for (int i = 0; i < b->max_inst; ++i) {
        M.h_off[i] = total;
        const Slot &S = b->slots[i];
        if (S.used) {
            total += 5 * (int64_t)S.h.G + S.h.eedf_bins + 2;
            M.who[i] = S.admission;
        }
    }
    M.h_off[b->max_inst] = total;
    if ((size_t)total > b->mpack_cap) {
        // a larger packing buffer: wait for the work that may still use the old one
        CK(cudaStreamSynchronize(b->stream));
        cudaFree(b->d_mpack);
        b->d_mpack = nullptr;
        b->mpack_cap = 0;
        CK(cudaMalloc((void **)&b->d_mpack, 8 * (size_t)total));
        b->mpack_cap = (size_t)total;
    }
    if (!b->d_moff) CK(cudaMalloc((void **)&b->d_moff, sizeof(int64_t) * ((size_t)b->max_inst + 1)));
    if ((size_t)total > M.cap) {
        if (M.h) cudaFreeHost(M.h);
        M.h = nullptr;
        M.cap = 0;
        CK(cudaHostAlloc((void **)&M.h, 8 * (size_t)total, cudaHostAllocDefault));
        M.cap = (size_t)total;
    }
    CK(cudaMemcpyAsync(b->d_moff, M.h_off, sizeof(int64_t) * ((size_t)b->max_inst + 1), cudaMemcpyHostToDevice,
                       b->stream));
    if (total > 0) {
        k_pack_moments<<<b->max_inst, 256, 0, b->stream>>>(b->d_inst, b->d_moff, b->d_mpack);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(M.h, b->d_mpack, 8 * (size_t)total, cudaMemcpyDeviceToHost, b->stream));
    }
    CK(cudaEventRecord(M.ev, b->stream));
    M.queued = true;
    b->msnap_cur = k;
    return HYB_OK;
}

int hyb_batch_read_snapshot_moments(hyb_batch *b, int32_t slot, hyb_moments *out)
{
    if (!b || !out) return fail(HYB_ERR_ARG, "NULL argument");
    if (slot < 0 || slot >= b->max_inst) return fail(HYB_ERR_ARG, "slot %d out of range", slot);
    if (b->msnap_cur < 0) return fail(HYB_ERR_STATE, "no moments snapshot queued");
    hyb_batch::MomentSnap &M = b->msnap[b->msnap_cur];
    const int64_t a = M.h_off[slot], n = M.h_off[slot + 1] - a;
    if (n <= 0) return fail(HYB_ERR_STATE, "slot %d was empty when the snapshot was queued", slot);
    if (!b->slots[slot].used || b->slots[slot].admission != M.who[slot])
        return fail(HYB_ERR_STATE, "slot %d holds another discharge than when the snapshot was queued", slot);
    CK(cudaEventSynchronize(M.ev));
    const double *d = M.h + a;
    const int64_t ns_bits = (int64_t)__builtin_bit_cast(uint64_t, d[n - 1]);
    const int nb = b->slots[slot].used ? b->slots[slot].h.eedf_bins : -1;
    const int G = b->slots[slot].used ? b->slots[slot].h.G : -1;
    if (d[n - 1] != d[n - 1] || nb < 0 || n != 5 * (int64_t)G + nb + 2)
        return fail(HYB_ERR_STATE, "slot %d changed since the snapshot was queued", slot);
    std::vector<unsigned long long> eedf(nb + 1);
    memcpy(eedf.data(), d + 5 * (size_t)G, 8 * (size_t)(nb + 1));
    moments_from_sums(d, eedf.data(), ns_bits, G, nb, b->slots[slot].h.bin_w, out);
    return HYB_OK;
}

int hyb_batch_read_moments(hyb_batch *b, int32_t slot, hyb_moments *out) { return read_moments(b, slot, out); }

int hyb_batch_read_counters(hyb_batch *b, int32_t slot, hyb_counters *out) { return read_counters(b, slot, out); }

int hyb_batch_read_particles(hyb_batch *b, int32_t slot, double *z, double *vx, double *vy, double *vz, uint64_t *id,
                             int64_t cap, int64_t *n)
{
    return read_particles(b, slot, z, vx, vy, vz, id, cap, n);
}

int hyb_batch_read_metastables(hyb_batch *b, int32_t slot, double *met, double *avg, double *flux)
{
    return read_metastables(b, slot, met, avg, flux);
}

int hyb_batch_read_ions(hyb_batch *b, int32_t slot, double *z, double *vx, double *vy, double *vz, uint64_t *id,
                        int64_t cap, int64_t *n)
{
    if (!n) return fail(HYB_ERR_ARG, "NULL argument");
    return read_ions(b, slot, z, vx, vy, vz, id, cap, n);
}

int hyb_batch_evict(hyb_batch *b, int32_t slot)
{
    int rc = check_slot(b, slot);
    if (rc) return rc;
    return free_slot(b, slot);
}

int hyb_batch_stats(hyb_batch *b, int32_t *running, int64_t *particles, int64_t *bytes)
{
    if (!b) return fail(HYB_ERR_ARG, "NULL batch");
    CK(cudaMemcpyAsync(b->h_stage, b->d_inst, sizeof(InstDev) * (size_t)b->max_inst, cudaMemcpyDeviceToHost,
                       b->stream));
    CK(cudaStreamSynchronize(b->stream));
    int r = 0;
    int64_t np = 0;
    for (int i = 0; i < b->max_inst; ++i) {
        if (!b->slots[i].used) continue;
        if (b->h_stage[i].active) {
            ++r;
            np += b->h_stage[i].n_slots_step;
        }
    }
    if (running) *running = r;
    if (particles) *particles = np;
    if (bytes) *bytes = b->hbm_used;
    return HYB_OK;
}

int hyb_batch_destroy(hyb_batch *b)
{
    if (!b) return HYB_OK;
    cudaStreamSynchronize(b->stream);
    for (int i = 0; i < b->max_inst; ++i)
        if (b->slots[i].used) cudaFreeAsync(b->slots[i].mem, b->stream);
    cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    for (int k = 0; k < kMaxLanes; ++k) {
        if (b->lstream[k]) cudaStreamDestroy(b->lstream[k]);
        if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    cudaFree(b->d_inst);
    cudaFree(b->d_prefix);
    cudaFree(b->d_prefix1);
    cudaFree(b->d_ticket);
    cudaFree(b->d_inst_ion);
    cudaFree(b->d_prefix_ion);
    cudaFree(b->d_prefix1_ion);
    cudaFreeHost(b->h_stage);
    for (int k = 0; k < hyb_batch::kSnaps; ++k) {
        if (b->h_snap[k]) cudaFreeHost(b->h_snap[k]);
        if (b->h_snap_ion[k]) cudaFreeHost(b->h_snap_ion[k]);
        if (b->ev_snap[k]) cudaEventDestroy(b->ev_snap[k]);
    }
    for (auto &x : b->stage) {
        cudaFreeHost(x.p);
        cudaEventDestroy(x.ev);
    }
    for (auto &m : b->msnap) {
        if (m.h_off) cudaFreeHost(m.h_off);
        if (m.h) cudaFreeHost(m.h);
        if (m.ev) cudaEventDestroy(m.ev);
    }
    cudaFree(b->d_moff);
    cudaFree(b->d_mpack);
    if (b->rstream) cudaStreamDestroy(b->rstream);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return HYB_OK;
}

int hyb_batch_get_tuning(hyb_batch *b, hyb_tuning *out)
{
    if (!b || !out) return fail(HYB_ERR_ARG, "NULL argument");
    *out = get_tuning(b);
    return HYB_OK;
}

int hyb_batch_set_tuning(hyb_batch *b, const hyb_tuning *t)
{
    if (!b || !t) return fail(HYB_ERR_ARG, "NULL argument");
    return set_tuning(b, *t);
}

int hyb_batch_autotune(hyb_batch *b, int32_t trial_steps, hyb_tuning *chosen)
{
    if (!b) return fail(HYB_ERR_ARG, "NULL batch");
    return autotune(b, trial_steps, chosen);
}

int hyb_batch_set_profiling(hyb_batch *b, int32_t on)
{
    if (!b) return fail(HYB_ERR_ARG, "NULL batch");
    if ((on != 0) != b->profiling) {
        int rc = flush_pending(b);
        if (rc) return rc;
        CK(cudaStreamSynchronize(b->stream));
        rc = drop_graph(b);
        if (rc) return rc;
        b->profiling = on != 0;
    }
    return HYB_OK;
}

int hyb_batch_profile(hyb_batch *b, hyb_profile *out, int32_t reset)
{
    if (!b || !out) return fail(HYB_ERR_ARG, "NULL argument");
    int rc = flush_pending(b);
    if (rc) return rc;
    CK(cudaStreamSynchronize(b->stream));
    out->kernel_launches = b->launches;
    out->steps = b->steps;
    out->ms_electron = b->ms[0];
    out->ms_field = b->ms[1];
    out->ms_sort = b->ms[2];
    out->n_electron = b->nt[0];
    out->n_field = b->nt[1];
    out->n_sort = b->nt[2];
    out->ms_ion = b->ms[3];
    out->n_ion = b->nt[3];
    if (reset) {
        b->ms[0] = b->ms[1] = b->ms[2] = b->ms[3] = 0.0;
        b->nt[0] = b->nt[1] = b->nt[2] = b->nt[3] = 0;
    }
    return HYB_OK;
}

hyb_batch *hyb_discharge_batch(hyb_discharge *h) { return h ? h->b : nullptr; }

int hyb_batch_set_field_arith(hyb_batch *b, int32_t split)
{
    if (!b) return fail(HYB_ERR_ARG, "NULL batch");
    if (split != 0 && split != 1) return fail(HYB_ERR_ARG, "split must be 0 or 1");
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(HYB_ERR_CUDA, "stream synchronisation failed");
    b->field_split = split == 1;
    return drop_graph(b);
}

int hyb_debug_checks(uint64_t out[6])
{
    if (!out) return fail(HYB_ERR_ARG, "NULL output");
    unsigned long long e[3], f[3], g[3], h[3];
    read_checks_electron(e);
    read_checks_sort(h);
    read_checks_ion(g);
    // the particle kernels: electrons first, then the sort, then the ions
    if (e[0] == 0 && e[1] == 0 && e[2] == 0)
        for (int k = 0; k < 3; ++k) e[k] = h[k];
    if (e[0] == 0 && e[1] == 0 && e[2] == 0)
        for (int k = 0; k < 3; ++k) e[k] = g[k];
    read_checks_field(f);
    for (int k = 0; k < 3; ++k) {
        out[k] = e[k];
        out[3 + k] = f[k];
    }
    return HYB_OK;
}

// ------------------------------------------------------------- single run

int hyb_create_discharge(const hyb_params *p, void *stream, hyb_discharge **out)
{
    if (!out) return fail(HYB_ERR_ARG, "NULL output");
    *out = nullptr;
    int rc = validate(p);
    if (rc) return rc;
    hyb_batch *b = nullptr;
    rc = hyb_batch_create(1, p->precision, 0, stream, &b);
    if (rc) return rc;
    if (p->sort_interval > 0) b->sort_interval = p->sort_interval > 1000 ? 1000 : p->sort_interval;
    int slot = -1;
    rc = admit(b, p, 0, &slot);
    if (rc < 0) {
        std::string msg = g_err;
        hyb_batch_destroy(b);
        g_err = msg;
        return rc;
    }
    hyb_discharge *h = new hyb_discharge{b, slot};
    *out = h;
    return rc;
}

int hyb_advance(hyb_discharge *h, int64_t n_steps)
{
    if (!h) return fail(HYB_ERR_ARG, "NULL handle");
    return advance(h->b, n_steps);
}

int hyb_sync(hyb_discharge *h)
{
    if (!h) return fail(HYB_ERR_ARG, "NULL handle");
    return sync_status(h->b, h->slot);
}

int hyb_read_moments(hyb_discharge *h, hyb_moments *out)
{
    if (!h) return fail(HYB_ERR_ARG, "NULL handle");
    return read_moments(h->b, h->slot, out);
}

int hyb_read_counters(hyb_discharge *h, hyb_counters *out)
{
    if (!h) return fail(HYB_ERR_ARG, "NULL handle");
    return read_counters(h->b, h->slot, out);
}

int hyb_read_fields(hyb_discharge *h, hyb_fields *out)
{
    if (!h || !out) return fail(HYB_ERR_ARG, "NULL argument");
    hyb_batch *b = h->b;
    int rc = sync_status(b, h->slot);
    const InstDev &K = b->h_stage[h->slot];
    const size_t bytes = 8 * (size_t)K.G;
    double *dst[6] = {out->ne, out->ni, out->gamma_i, out->phi, out->efield, out->ion_source};
    const double *src[6] = {K.ne, K.ni, K.gam, K.phi, K.E, K.gsrc};
    for (int k = 0; k < 6; ++k)
        if (dst[k]) CK(cudaMemcpyAsync(dst[k], src[k], bytes, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return rc;
}

int hyb_get_info(hyb_discharge *h, hyb_info *out)
{
    if (!h || !out) return fail(HYB_ERR_ARG, "NULL argument");
    const Slot &S = h->b->slots[h->slot];
    out->n_nodes = S.h.G;
    out->eedf_bins = S.h.eedf_bins;
    out->weight = S.h.w;
    out->gas_density = S.h.ngas;
    out->nu_max = S.h.nu_max;
    out->p_max = S.h.p_max;
    out->dz = S.h.dz;
    out->capacity = S.h.capacity;
    out->device_bytes = S.bytes;
    return HYB_OK;
}

int hyb_reset_moments(hyb_discharge *h)
{
    if (!h) return fail(HYB_ERR_ARG, "NULL handle");
    hyb_batch *b = h->b;
    int rc = fetch_inst(b, h->slot);
    if (rc) return rc;
    InstDev K = b->h_stage[h->slot];
    const size_t bytes = 8 * (size_t)K.G;
    double *acc[5] = {K.acc_ne, K.acc_ni, K.acc_gi, K.acc_wn, K.acc_we};
    for (int k = 0; k < 5; ++k) CK(cudaMemsetAsync(acc[k], 0, bytes, b->stream));
    if (K.met_on) CK(cudaMemsetAsync(K.acc_met, 0, bytes, b->stream));
    CK(cudaMemsetAsync(K.eedf, 0, 8 * (size_t)(K.eedf_bins + 1), b->stream));
    K.n_samples = 0;
    CK(cudaMemcpyAsync(&b->d_inst[h->slot], &K, sizeof K, cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return HYB_OK;
}

int hyb_read_particles(hyb_discharge *h, double *z, double *vx, double *vy, double *vz, uint64_t *id, int64_t cap,
                       int64_t *n)
{
    if (!h || !n) return fail(HYB_ERR_ARG, "NULL argument");
    return read_particles(h->b, h->slot, z, vx, vy, vz, id, cap, n);
}

int hyb_write_particles(hyb_discharge *h, int64_t n, const double *z, const double *vx, const double *vy,
                        const double *vz, const uint64_t *id)
{
    if (!h) return fail(HYB_ERR_ARG, "NULL handle");
    if (n < 0 || (n > 0 && (!z || !vx || !vy || !vz || !id))) return fail(HYB_ERR_ARG, "bad particle arrays");
    hyb_batch *b = h->b;
    const Slot &S = b->slots[h->slot];
    if (n > S.h.capacity) return fail(HYB_ERR_CAPACITY, "%lld particles exceed capacity %lld", (long long)n,
                                      (long long)S.h.capacity);
    for (int64_t i = 0; i < n; ++i) {
        if (!(z[i] >= 0.0 && z[i] < S.h.L)) return fail(HYB_ERR_ARG, "particle %lld outside [0, L)", (long long)i);
        if (!isfinite(vx[i]) || !isfinite(vy[i]) || !isfinite(vz[i]))
            return fail(HYB_ERR_NONFINITE, "non-finite velocity of particle %lld", (long long)i);
    }
    int rc = fetch_inst(b, h->slot);
    if (rc) return rc;
    const InstDev K = b->h_stage[h->slot];
    const PartBuf P = K.buf[K.cur];
    if (n > 0) {
        CK(cudaMemcpy(P.id, id, 8 * (size_t)n, cudaMemcpyHostToDevice));
        if (K.precision == HYB_FP32_SPLIT) {
            std::vector<int32_t> c(n);
            std::vector<float> o(n), fx(n), fy(n), fz(n);
            for (int64_t i = 0; i < n; ++i) {
                const double x = z[i] / K.dz;
                const double f = floor(x);
                int ci = (int)f;
                double oi = x - f;
                if (ci >= K.n_cells) {
                    ci = K.n_cells - 1;
                    oi = 1.0;
                }
                c[i] = ci;
                o[i] = (float)oi;
                fx[i] = (float)vx[i];
                fy[i] = (float)vy[i];
                fz[i] = (float)vz[i];
            }
            CK(cudaMemcpy(P.c, c.data(), 4 * (size_t)n, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(P.o, o.data(), 4 * (size_t)n, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(P.vxf, fx.data(), 4 * (size_t)n, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(P.vyf, fy.data(), 4 * (size_t)n, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(P.vzf, fz.data(), 4 * (size_t)n, cudaMemcpyHostToDevice));
        } else {
            CK(cudaMemcpy(P.z, z, 8 * (size_t)n, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(P.vxd, vx, 8 * (size_t)n, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(P.vyd, vy, 8 * (size_t)n, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(P.vzd, vz, 8 * (size_t)n, cudaMemcpyHostToDevice));
        }
    }
    rc = set_mutable(b, h->slot, n, 1);
    if (rc) return rc;
    rc = reinit_slot(b, h->slot, true);
    if (rc) return rc;
    rc = prefix_all(b);
    if (rc) return rc;
    CK(cudaStreamSynchronize(b->stream));
    return HYB_OK;
}

int hyb_read_ions(hyb_discharge *h, double *z, double *vx, double *vy, double *vz, uint64_t *id, int64_t cap,
                  int64_t *n)
{
    if (!h || !n) return fail(HYB_ERR_ARG, "NULL argument");
    return read_ions(h->b, h->slot, z, vx, vy, vz, id, cap, n);
}

int hyb_read_metastables(hyb_discharge *h, double *met, double *avg, double *flux)
{
    if (!h) return fail(HYB_ERR_ARG, "NULL handle");
    return read_metastables(h->b, h->slot, met, avg, flux);
}

int hyb_write_metastables(hyb_discharge *h, const double *met)
{
    if (!h || !met) return fail(HYB_ERR_ARG, "NULL argument");
    hyb_batch *b = h->b;
    const InstDev &K = b->slots[h->slot].h;
    if (!K.met_on) return fail(HYB_ERR_STATE, "the discharge has no metastables");
    const int G = K.G;
    for (int j = 0; j < G; ++j)
        if (!(met[j] >= 0.0) || !isfinite(met[j])) return fail(HYB_ERR_ARG, "metastable density %d invalid", j);
    if (met[0] != 0.0 || met[G - 1] != 0.0) return fail(HYB_ERR_ARG, "the electrode nodes must be 0");
    CK(cudaStreamSynchronize(b->stream));
    CK(cudaMemcpy(K.met, met, 8 * (size_t)G, cudaMemcpyHostToDevice));
    return HYB_OK;
}

int hyb_write_ion_density(hyb_discharge *h, const double *ni)
{
    if (!h || !ni) return fail(HYB_ERR_ARG, "NULL argument");
    if (h->b->slots[h->slot].h.ion) return fail(HYB_ERR_STATE, "kinetic ions: the ion density follows the ions");
    hyb_batch *b = h->b;
    const Slot &S = b->slots[h->slot];
    if (!finite_all(ni, S.h.G)) return fail(HYB_ERR_NONFINITE, "non-finite ion density");
    CK(cudaStreamSynchronize(b->stream));
    CK(cudaMemcpy(S.h.ni, ni, 8 * (size_t)S.h.G, cudaMemcpyHostToDevice));
    int rc = fetch_inst(b, h->slot);
    if (rc) return rc;
    rc = set_mutable(b, h->slot, (int64_t)b->h_stage[h->slot].n_slots, 1);
    if (rc) return rc;
    rc = reinit_slot(b, h->slot, false);
    if (rc) return rc;
    rc = prefix_all(b);
    if (rc) return rc;
    CK(cudaStreamSynchronize(b->stream));
    return HYB_OK;
}

int hyb_destroy(hyb_discharge *h)
{
    if (!h) return HYB_OK;
    hyb_batch_destroy(h->b);
    delete h;
    return HYB_OK;
}

}  // extern "C"
