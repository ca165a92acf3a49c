// hyb_field.cu -- the per-instance FP64 grid kernel of each step (arXiv
// 1508.02892, Secs. II.B-II.D): electron density from the CIC sums, the ion
// fluid update (drift-diffusion, Eqs. 2.5-2.8, or the full model, Eq. 2.3,
// then continuity, Eq. 2.4), the Poisson solve and field, the time sums, and
// the gamma secondaries that will take part in the next step.
//
// One CTA of 1024 threads per instance, all node arrays in shared memory
// (7 x n_nodes doubles), thread t owning a contiguous run of nodes.
//   * Poisson: the constant-coefficient tridiagonal system is solved in closed
//     form by two block prefix scans (phi = linear part + discrete double
//     integral of the charge) instead of the serial Thomas recursion.
//   * Full-model flux: the tridiagonal system of Eq. 2.3 is diagonally
//     dominant with ratio r = max (|a|+|c|)/b (a Courant number); it is solved
//     by Jacobi sweeps, ceil(ln 2^-60 / ln r) of them, which bounds the error
//     by 2^-60 of the initial one.  r >= 1/2 is reported as unstable.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hyb_internal.cuh"

namespace hyb {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kArrays = 7;

struct Red {
    double w[32];
    double total;
    int flag;
    int iters;
    unsigned long long count;
};

// Instance constants of the field step, formed once per block by thread 0
// (each the same expression the per-node code would evaluate, so results do
// not change; FP64 division, sin and log are long instruction sequences on
// this part's FP64 rate).
struct FieldConsts {
    double h, inv2dz, qdt_m, h_m, c_in, c_wall, gs_in, gs_wall;  // split-mode fluid
    double dt_dz, dt_2dz, h_mion;                                // FP64-mode fluid
    double w_in, w_wall, c_src, inv_dz, half_inv_dz, c_gauss;    // split-mode Poisson
    double phi0;
    float inv_ngas_td, tfac;
};

// Exclusive block scan of one double per thread; *total gets the sum.
__device__ double block_exscan(double v, Red &r, double *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const double y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) r.w[wid] = x;
    __syncthreads();
    if (wid == 0) {
        double t = lane < nw ? r.w[lane] : 0.0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const double y = __shfl_up_sync(kFull, t, d);
            if (lane >= d) t += y;
        }
        r.w[lane] = t;
    }
    __syncthreads();
    const double off = wid ? r.w[wid - 1] : 0.0;
    if (total) *total = r.w[nw - 1];
    __syncthreads();
    return off + x - v;
}

__device__ double block_max(double v, Red &r)
{
#pragma unroll
    for (int d = 16; d; d >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, d));
    if ((threadIdx.x & 31) == 0) r.w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double m = threadIdx.x < (blockDim.x >> 5) ? r.w[threadIdx.x] : 0.0;
#pragma unroll
        for (int d = 16; d; d >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, d));
        if (threadIdx.x == 0) r.total = fmax(m, 0.0);
    }
    __syncthreads();
    const double m = r.total;
    __syncthreads();
    return m;
}

// Jacobi sweeps for a contraction ratio r: ceil(ln 2^-60 / ln r), 1..64,
// formed by thread 0 and shared
__device__ int jacobi_iters(double r, Red &red)
{
    if (threadIdx.x == 0) {
        int iters = 1;
        if (r > 1e-300) iters = (int)ceil(-41.58883083359672 / log(r));
        red.iters = iters < 1 ? 1 : (iters > 64 ? 64 : iters);
    }
    __syncthreads();
    return red.iters;
}

// linear interpolation in a 4-column table, clamped at the ends
__device__ double interp_lin(const double *tab, int n, int cx, int cy, double v)
{
    if (v <= tab[cx]) return tab[cy];
    if (v >= tab[4 * (n - 1) + cx]) return tab[4 * (n - 1) + cy];
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (tab[4 * mid + cx] <= v)
            lo = mid;
        else
            hi = mid;
    }
    const double f = (v - tab[4 * lo + cx]) / (tab[4 * (lo + 1) + cx] - tab[4 * lo + cx]);
    return tab[4 * lo + cy] + f * (tab[4 * (lo + 1) + cy] - tab[4 * lo + cy]);
}

struct Fluid {
    int model, n_tab;
    const double *tab;
    double mu_const, ngas, kT, mi, mn;

    // ion mobility at |E| (Sec. II.C, tabulated Tables 2/4)
    __device__ double mobility(double e_abs) const
    {
        if (model == HYB_ION_DD_CONST) return mu_const;
        const double eon_td = e_abs / ngas * 1e21;
        return interp_lin(tab, n_tab, 0, 1, eon_td);
    }
    // ion temperature (J): gas temperature, or Eq. 2.8
    __device__ double temp(double mu, double e_abs) const
    {
        if (model == HYB_ION_DD_CONST) return kT;
        const double ud = mu * e_abs;
        return kT + (mi + mn) / (5.0 * mi + 3.0 * mn) * mn * ud * ud;
    }
    // momentum-exchange frequency at |u| (Sec. II.B, tabulated Tables 3/5)
    __device__ double exch(double u_abs) const { return interp_lin(tab, n_tab, 3, 2, u_abs); }
    // field-driven wall flux with the alpha switch of Sec. II.C
    __device__ double wall(int w, double n, double E) const
    {
        const bool into = w == 0 ? (E < 0.0) : (E > 0.0);
        if (!into) return 0.0;
        return mobility(fabs(E)) * n * E;
    }
};

__device__ __forceinline__ double node_volume(int j, int G, double dz) { return (j == 0 || j == G - 1) ? 0.5 * dz : dz; }

// FP32 copy of the transport coefficients for the split mode: the table is
// staged in shared memory and mu(E), T_i, nu(u) are evaluated in FP32; the
// state (n, Gamma) and every difference of neighbouring values stay FP64.
constexpr int kMaxTab = 256;

__device__ __forceinline__ float interp_linf(const float *tab, int n, int cx, int cy, float v)
{
    if (v <= tab[cx]) return tab[cy];
    if (v >= tab[4 * (n - 1) + cx]) return tab[4 * (n - 1) + cy];
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tab[4 * mid + cx] <= v)
            lo = mid;
        else
            hi = mid;
    }
    const float f = __fdividef(v - tab[4 * lo + cx], tab[4 * (lo + 1) + cx] - tab[4 * lo + cx]);
    return tab[4 * lo + cy] + f * (tab[4 * (lo + 1) + cy] - tab[4 * lo + cy]);
}

struct FluidF {
    int model, n_tab;
    const float *tab;  // shared memory
    float mu_const, inv_ngas_td, kT, tfac;

    __device__ float mobility(float e_abs) const
    {
        if (model == HYB_ION_DD_CONST) return mu_const;
        return interp_linf(tab, n_tab, 0, 1, e_abs * inv_ngas_td);
    }
    __device__ float temp(float mu, float e_abs) const
    {
        if (model == HYB_ION_DD_CONST) return kT;
        const float ud = mu * e_abs;
        return kT + tfac * ud * ud;
    }
    __device__ float exch(float u_abs) const { return interp_linf(tab, n_tab, 3, 2, u_abs); }
    __device__ double wall(int w, double n, double E) const
    {
        const bool into = w == 0 ? (E < 0.0) : (E > 0.0);
        if (!into) return 0.0;
        return (double)mobility(fabsf((float)E)) * n * E;
    }
};

// Metastables and the ionization they cause (Sec. II.D), from n_m^n at the
// start of the step:
//  - Penning (Delta N_e = R_P n_N n_m dt dz) and pooling (R_pool n_m^2 dt dz)
//    electrons per interior node j: the integer part of Delta N_e / N_p/sp plus
//    one with the probability of the fraction (call 3 of the key of the process
//    and j); numbered k = 0, 1, ... in node order per process, each placed
//    uniformly in [z_j - dz/2, z_j + dz/2) at the process's energy with an
//    isotropic direction (call 7 of its id), appended after this step's
//    children, its ion added to the ion source (CIC);
//  - the explicit update n_m += dt (D n_m'' + S_m - R_P n_N n_m - 2 R_pool n_m^2)
//    at the interior nodes, n_m = 0 at the electrodes, and the flux into each
//    wall (D n_m(next node)/dz plus the excitation sources on the wall node).
// Delta N_e of one node: R_P n_m n_N dt dz (Penning) or R_pool n_m^2 dt dz (pooling)
__device__ __forceinline__ double birth_mean(const InstDev *K, int proc, double nm, double dt, double dz)
{
    return proc == 0 ? K->met_rp * nm * K->met_nn * dt * dz : K->met_kq * nm * nm * dt * dz;
}

// old, cnt0, cnt1: G doubles each of shared scratch (n_m at the start of the
// step, the per-node Penning and pooling counts).  The split mode multiplies by
// reciprocals where the FP64 mode divides as the oracle does (an FP64 division
// is a long instruction sequence at this part's FP64 rate).
template <bool FAST>
__device__ void metastable_step(InstDev *K, double *old, double *cnt0, double *cnt1, Red &red, int j0, int j1)
{
    const int G = K->G;
    const double dz = K->dz, dt = K->dt, w = K->w;
    const uint32_t n = (uint32_t)K->step;
    const double kp = K->met_kp, kq = K->met_kq;
    const double inv_w = w > 0.0 ? 1.0 / w : 0.0;
    __shared__ unsigned long long s_base;
    __shared__ int64_t s_tot[2];
    int64_t mine[2] = {0, 0};
    // counts per node, kept in the scratch row until the update below
    for (int j = j0; j < j1; ++j) {
        const double nm = K->met[j];
        old[j] = nm;
    }
    double part[2] = {0.0, 0.0};
    for (int proc = 0; proc < 2; ++proc) {
        double *cnt = proc == 0 ? cnt0 : cnt1;
        const double r = proc == 0 ? kp : kq;
        for (int j = j0; j < j1; ++j) {
            double c = 0.0;
            double m = 0.0;
            if (j >= 1 && j <= G - 2 && r > 0.0 && w > 0.0)
                m = FAST ? birth_mean(K, proc, old[j], dt, dz) * inv_w : birth_mean(K, proc, old[j], dt, dz) / w;
            if (m > 0.0) {
                const double fl = floor(m);
                const uint4 u = draw(0xFFFFFFFF00000000ull | ((uint64_t)(proc + 1) << 24) | (uint64_t)j, n,
                                     K->seed_lo, K->seed_hi, 3);
                c = fl + (u01d(u.x) < m - fl ? 1.0 : 0.0);
            }
            cnt[j] = c;
            part[proc] += c;
        }
    }
    double tot[2];
    const double off0 = block_exscan(part[0], red, &tot[0]);
    const double off1 = block_exscan(part[1], red, &tot[1]);
    const int64_t cap = (1 << 20) - 1;
    if (threadIdx.x == 0) {
        s_tot[0] = (int64_t)tot[0] < cap ? (int64_t)tot[0] : cap;
        s_tot[1] = (int64_t)tot[1] < cap ? (int64_t)tot[1] : cap;
        if ((int64_t)tot[0] > cap || (int64_t)tot[1] > cap) K->status |= HYB_STATUS_EMIT_CAP;
        s_base = K->n_slots;
        K->n_slots = s_base + (unsigned long long)(s_tot[0] + s_tot[1]);
        K->ctr[C_PEN] += (unsigned long long)s_tot[0];
        K->ctr[C_POOL] += (unsigned long long)s_tot[1];
    }
    __syncthreads();
    mine[0] = (int64_t)off0;
    mine[1] = (int64_t)off1;
    const PartBuf P = K->buf[K->cur];
    for (int proc = 0; proc < 2; ++proc) {
        if (part[proc] == 0.0) continue;
        const double *cnts = proc == 0 ? cnt0 : cnt1;
        const double sp = K->met_sp[proc];
        int64_t k = mine[proc];
        for (int j = max(j0, 1); j < min(j1, G - 1) && k < s_tot[proc]; ++j) {
            const int64_t cnt = (int64_t)cnts[j];
            for (int64_t b = 0; b < cnt && k < s_tot[proc]; ++b, ++k) {
                const uint64_t id = (1ull << 62) | ((uint64_t)(2 + proc) << 60) | ((uint64_t)n << 20) | (uint64_t)k;
                const uint4 v = draw(id, n, K->seed_lo, K->seed_hi, 7);
                const double z = ((double)j - 0.5 + u01d(v.x)) * dz;
                const double ct = 1.0 - 2.0 * u01d(v.y);
                const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
                const double ph = kTwoPi * u01d(v.z);
                const double vx = sp * st * cos(ph), vy = sp * st * sin(ph), vz = sp * ct;
                // the ion of the event (CIC), as for an impact ionization
                const double x = z / dz;
                const double f = floor(x);
                int c = (int)f;
                double o = x - f;
                if (c >= K->n_cells) {
                    c = K->n_cells - 1;
                    o = 1.0;
                }
                if (HYB_CHECK(c >= 0 && c + 1 < G, 21, c, G)) {
                    atomicAdd(&K->s_iz[c], 1.0 - o);
                    atomicAdd(&K->s_iz[c + 1], o);
                }
                const unsigned long long slot = s_base + (unsigned long long)(proc == 0 ? k : s_tot[0] + k);
                if (slot >= (unsigned long long)K->capacity) {
                    atomicOr(&K->status, (unsigned)HYB_STATUS_CAPACITY);
                    continue;
                }
                P.id[slot] = id;
                if (K->precision == HYB_FP32_SPLIT) {
                    P.c[slot] = c;
                    P.o[slot] = (float)o;
                    P.vxf[slot] = (float)vx;
                    P.vyf[slot] = (float)vy;
                    P.vzf[slot] = (float)vz;
                } else {
                    P.z[slot] = z;
                    P.vxd[slot] = vx;
                    P.vyd[slot] = vy;
                    P.vzd[slot] = vz;
                }
            }
        }
    }
    __syncthreads();
    // the density update from the old values
    const double D = K->met_D;
    const double c_src = w / (dz * dt), c_lap = D / (dz * dz);
    unsigned long long clamps = 0;
    for (int j = j0; j < j1; ++j) {
        double nn = 0.0;
        if (j >= 1 && j <= G - 2) {
            const double src = FAST ? K->s_met[j] * c_src : w * K->s_met[j] / (dz * dt);
            const double lap = FAST ? c_lap * (old[j + 1] - 2.0 * old[j] + old[j - 1])
                                    : D * (old[j + 1] - 2.0 * old[j] + old[j - 1]) / (dz * dz);
            const double loss = kp * old[j] + 2.0 * kq * old[j] * old[j];
            nn = old[j] + dt * (lap + src - loss);
            if (nn < 0.0) {
                nn = 0.0;
                ++clamps;
            }
        }
        K->met[j] = nn;
        K->acc_met[j] += nn;
    }
    if (clamps) atomicAdd(&red.count, clamps);
    __syncthreads();
    if (threadIdx.x == 0) {
        K->flux_met[0] = D * old[1] / dz + w * K->s_met[0] / dt;
        K->flux_met[1] = D * old[G - 2] / dz + w * K->s_met[G - 1] / dt;
    }
    __syncthreads();
    for (int j = j0; j < j1; ++j) K->s_met[j] = 0.0;
}

template <bool FAST>
__device__ void field_body(InstDev *K, double *sm, Red &red, float *s_tabf, FieldConsts &fc)
{
    const int G = K->G;
    const int T = blockDim.x;
    const int t = threadIdx.x;
    const int per = (G + T - 1) / T;
    const int j0 = min(t * per, G), j1 = min(j0 + per, G);
    const double dz = K->dz, dt = K->dt, w = K->w;
    const bool init = K->init_pending != 0;

    double *s_ni = sm;
    double *s_E = sm + G;
    double *s_g = sm + 2 * G;
    double *s_A = sm + 3 * G;
    double *s_ib = sm + 4 * G;
    double *s_d = sm + 5 * G;
    double *s_x = sm + 6 * G;

    for (int j = j0; j < j1; ++j) {
        s_ni[j] = K->ni[j];
        s_E[j] = K->E[j];
        s_g[j] = K->gam[j];
    }
    if (t == 0) {
        red.flag = 0;
        red.count = 0ull;
        const double mi = K->m_ion, mn = K->m_gas;
        fc.h = dt / (2.0 * dz);
        fc.inv2dz = 1.0 / (2.0 * dz);
        fc.qdt_m = kQe * dt / mi;
        fc.h_m = fc.h / mi;
        fc.c_in = dt * fc.inv2dz;
        fc.c_wall = dt / dz;
        fc.gs_in = w / (dz * dt);
        fc.gs_wall = w / (0.5 * dz * dt);
        fc.dt_dz = dt / dz;
        fc.dt_2dz = dt / (2.0 * dz);
        fc.h_mion = fc.h / K->m_ion;
        fc.w_in = w / dz;
        fc.w_wall = 2.0 * w / dz;
        fc.c_src = dz * dz / kEps0;
        fc.inv_dz = 1.0 / dz;
        fc.half_inv_dz = 0.5 / dz;
        fc.c_gauss = dz / (2.0 * kEps0);
        fc.phi0 = K->v_dc + K->v_rf * sin(kTwoPi * K->f_rf * ((double)(K->step + (init ? 0 : 1)) * dt));
        fc.inv_ngas_td = (float)(1e21 / K->ngas);
        fc.tfac = (float)((mi + mn) / (5.0 * mi + 3.0 * mn) * mn);
    }
    __syncthreads();

    if (K->met_on && !init) metastable_step<FAST>(K, s_d, s_x, s_ib, red, j0, j1);

    const Fluid F{K->ion_model, K->n_tab, K->tab, K->mu_const, K->ngas, K->kT_gas, K->m_ion, K->m_gas};
    double *gfin = s_g;
    const bool kin = K->ion_model == HYB_ION_KINETIC;
    if (kin) {
        // kinetic ions: n_i and Gamma_i from the ions' charge assignment of this
        // step (at initialisation, of the loaded ions)
        for (int j = j0; j < j1; ++j) {
            const double vol = node_volume(j, G, dz);
            const double nn = w * K->dep_ni[j] / vol;
            const double gg = w * K->dep_gi[j] / vol;
            s_ni[j] = nn;
            s_g[j] = gg;
            K->ni[j] = nn;
            K->gam[j] = gg;
            K->dep_ni[j] = 0.0;
            K->dep_gi[j] = 0.0;
            if (!init) {
                K->gsrc[j] = w * K->s_iz[j] / (vol * dt);
                K->acc_ni[j] += nn;
                K->acc_gi[j] += gg;
            }
        }
        __syncthreads();
    }
    if (FAST && !init && !kin) {
        // ------------------------------------ ion fluid, FP32 coefficients
        for (int j = t; j < 4 * K->n_tab; j += T) s_tabf[j] = (float)K->tab[j];
        __syncthreads();
        const FluidF FF{K->ion_model, K->n_tab, s_tabf, (float)K->mu_const, fc.inv_ngas_td, (float)K->kT_gas,
                        fc.tfac};
        const double h = fc.h;
        const double inv2dz = fc.inv2dz;
        if (K->ion_model == HYB_ION_FULL) {
            const double qdt_m = fc.qdt_m, h_m = fc.h_m;
            const float hdt = (float)(0.5 * dt);
            for (int j = j0; j < j1; ++j) {
                const double nj = s_ni[j];
                const float A = nj >= K->n_floor ? (float)s_g[j] / (float)nj : 0.f;
                s_A[j] = h * (double)A;  // h Gamma/n, the advection coefficient
                const float ea = fabsf((float)s_E[j]);
                s_x[j] = nj * (double)FF.temp(FF.mobility(ea), ea);
            }
            __syncthreads();
            float rmax = 0.f;
            for (int j = j0; j < j1; ++j) {
                if (j == 0 || j == G - 1) continue;
                const float nu = FF.exch(fabsf((float)(s_A[j] / h)));
                const float ib = 1.f / (1.f + nu * hdt);
                s_d[j] = s_g[j] * (double)(1.f - nu * hdt) + qdt_m * s_ni[j] * s_E[j] - h_m * (s_x[j + 1] - s_x[j - 1]);
                s_ib[j] = (double)ib;
                rmax = fmaxf(rmax, (fabsf((float)s_A[j - 1]) + fabsf((float)s_A[j + 1])) * ib);
            }
            const double r = block_max((double)rmax, red);
            if (t == 0) {
                const double g0 = FF.wall(0, s_ni[0], s_E[0]);
                const double gN = FF.wall(1, s_ni[G - 1], s_E[G - 1]);
                s_g[0] = g0;
                s_x[0] = g0;
                s_g[G - 1] = gN;
                s_x[G - 1] = gN;
                if (r >= 0.5) atomicOr(&K->status, (unsigned)HYB_STATUS_UNSTABLE);
            }
            const int iters = jacobi_iters(r, red);
            double *X = s_g, *Y = s_x;
            for (int it = 0; it < iters; ++it) {
                for (int j = j0; j < j1; ++j) {
                    if (j == 0 || j == G - 1) continue;
                    Y[j] = (s_d[j] + s_A[j - 1] * X[j - 1] - s_A[j + 1] * X[j + 1]) * s_ib[j];
                }
                __syncthreads();
                double *tmp = X;
                X = Y;
                Y = tmp;
            }
            gfin = X;
        } else {
            for (int j = j0; j < j1; ++j) {
                if (j == 0) {
                    s_x[j] = FF.wall(0, s_ni[0], s_E[0]);
                } else if (j == G - 1) {
                    s_x[j] = FF.wall(1, s_ni[G - 1], s_E[G - 1]);
                } else {
                    const float ea = fabsf((float)s_E[j]);
                    const float mu = FF.mobility(ea);
                    const float D = mu * FF.temp(mu, ea) * (float)(1.0 / kQe);
                    s_x[j] = (double)mu * s_ni[j] * s_E[j] - (double)D * ((s_ni[j + 1] - s_ni[j - 1]) * inv2dz);
                }
            }
            __syncthreads();
            gfin = s_x;
        }
        unsigned long long clamps = 0;
        const double c_in = fc.c_in, c_wall = fc.c_wall;
        const double gs_in = fc.gs_in, gs_wall = fc.gs_wall;
        for (int j = j0; j < j1; ++j) {
            const bool wall = j == 0 || j == G - 1;
            const double gs = K->s_iz[j] * (wall ? gs_wall : gs_in);
            double nn;
            if (j == 0)
                nn = s_ni[0] - c_wall * (gfin[1] - gfin[0]) + dt * gs;
            else if (j == G - 1)
                nn = s_ni[G - 1] - c_wall * (gfin[G - 1] - gfin[G - 2]) + dt * gs;
            else
                nn = s_ni[j] - c_in * (gfin[j + 1] - gfin[j - 1]) + dt * gs;
            if (nn < 0.0) {
                nn = 0.0;
                ++clamps;
            }
            s_ni[j] = nn;
            K->ni[j] = nn;
            K->gam[j] = gfin[j];
            K->gsrc[j] = gs;
            K->acc_ni[j] += nn;
            K->acc_gi[j] += gfin[j];
        }
        if (clamps) atomicAdd(&red.count, clamps);
        __syncthreads();
    }
    if (!FAST && !init && !kin) {
        // ---------------------------------------------------------- ion fluid
        if (K->ion_model == HYB_ION_FULL) {
            // Eq. 2.3: nu at u^n = Gamma^{n-1/2}/n^n, advection semi-implicit
            for (int j = j0; j < j1; ++j) {
                const double nj = s_ni[j];
                s_A[j] = nj >= K->n_floor ? s_g[j] / nj : 0.0;
                const double ea = fabs(s_E[j]);
                s_x[j] = nj * F.temp(F.mobility(ea), ea);
            }
            __syncthreads();
            const double h = fc.h;
            double rmax = 0.0;
            for (int j = j0; j < j1; ++j) {
                if (j == 0 || j == G - 1) continue;
                const double nu = F.exch(fabs(s_A[j]));
                const double b = 1.0 + nu * dt / 2.0;
                s_d[j] = s_g[j] * (1.0 - nu * dt / 2.0) + kQe * s_ni[j] * s_E[j] * dt / K->m_ion -
                         fc.h_mion * (s_x[j + 1] - s_x[j - 1]);
                s_ib[j] = 1.0 / b;
                rmax = fmax(rmax, (fabs(h * s_A[j - 1]) + fabs(h * s_A[j + 1])) / b);
            }
            const double r = block_max(rmax, red);
            // Dirichlet wall rows (field-driven wall flux), both Jacobi buffers
            if (t == 0) {
                const double g0 = F.wall(0, s_ni[0], s_E[0]);
                const double gN = F.wall(1, s_ni[G - 1], s_E[G - 1]);
                s_g[0] = g0;
                s_x[0] = g0;
                s_g[G - 1] = gN;
                s_x[G - 1] = gN;
                if (r >= 0.5) atomicOr(&K->status, (unsigned)HYB_STATUS_UNSTABLE);
            }
            const int iters = jacobi_iters(r, red);
            double *X = s_g, *Y = s_x;
            for (int it = 0; it < iters; ++it) {
                for (int j = j0; j < j1; ++j) {
                    if (j == 0 || j == G - 1) continue;
                    Y[j] = (s_d[j] + h * s_A[j - 1] * X[j - 1] - h * s_A[j + 1] * X[j + 1]) * s_ib[j];
                }
                __syncthreads();
                double *tmp = X;
                X = Y;
                Y = tmp;
            }
            gfin = X;
        } else {
            // Eq. 2.5 at level n (explicit drift-diffusion)
            for (int j = j0; j < j1; ++j) {
                if (j == 0) {
                    s_x[j] = F.wall(0, s_ni[0], s_E[0]);
                } else if (j == G - 1) {
                    s_x[j] = F.wall(1, s_ni[G - 1], s_E[G - 1]);
                } else {
                    const double ea = fabs(s_E[j]);
                    const double mu = F.mobility(ea);
                    const double D = mu * F.temp(mu, ea) / kQe;
                    s_x[j] = mu * s_ni[j] * s_E[j] - D * (s_ni[j + 1] - s_ni[j - 1]) / (2.0 * dz);
                }
            }
            __syncthreads();
            gfin = s_x;
        }
        // ------------------------------------- continuity, Eq. 2.4 (G^n source)
        unsigned long long clamps = 0;
        for (int j = j0; j < j1; ++j) {
            const double gs = w * K->s_iz[j] / (node_volume(j, G, dz) * dt);
            double nn;
            if (j == 0)
                nn = s_ni[0] - fc.dt_dz * (gfin[1] - gfin[0]) + dt * gs;
            else if (j == G - 1)
                nn = s_ni[G - 1] - fc.dt_dz * (gfin[G - 1] - gfin[G - 2]) + dt * gs;
            else
                nn = s_ni[j] - fc.dt_2dz * (gfin[j + 1] - gfin[j - 1]) + dt * gs;
            if (nn < 0.0) {
                nn = 0.0;
                ++clamps;
            }
            s_ni[j] = nn;
            K->ni[j] = nn;
            K->gam[j] = gfin[j];
            K->gsrc[j] = gs;
            K->acc_ni[j] += nn;
            K->acc_gi[j] += gfin[j];
        }
        if (clamps) atomicAdd(&red.count, clamps);
        __syncthreads();
    }

    if (K->rec_on) {
        // bound of the next electron step's recombination test (Sec. II.D):
        // nu_rec,max = max_z n_i * max sigma_rec v; the split mode reads n_i / max n_i
        double m = 0.0;
        for (int j = j0; j < j1; ++j) m = fmax(m, s_ni[j]);
        const double nimax = block_max(m, red);
        if (t == 0) {
            K->rec_numax = nimax * K->rec_svmax;
            K->rec_pmax = -expm1(-K->rec_numax * dt);
            K->f_rec_pmax = (float)K->rec_pmax;
        }
        const double inv = nimax > 0.0 ? 1.0 / nimax : 0.0;
        for (int j = j0; j < j1; ++j) K->nif[j] = (float)(s_ni[j] * inv);
    }

    // ------------------------------------------------------------- Poisson
    const double phi0 = fc.phi0;
    double *s_rho = s_A;
    double *s_S = s_ib;
    double *s_phi = s_d;
    double part = 0.0;
    // the split mode multiplies by reciprocals where the FP64 mode divides (as
    // the oracle does); FP64 division is a long instruction sequence here
    const double w_in = fc.w_in, w_wall = fc.w_wall, c_src = fc.c_src;
    for (int j = j0; j < j1; ++j) {
        const double ne = FAST ? K->dep_n[j] * ((j == 0 || j == G - 1) ? w_wall : w_in)
                               : w * K->dep_n[j] / node_volume(j, G, dz);
        K->ne[j] = ne;
        const double rho = kQe * (s_ni[j] - ne);
        s_rho[j] = rho;
        const double sj = (j >= 1 && j <= G - 2) ? (FAST ? rho * c_src : dz * dz * rho / kEps0) : 0.0;
        part += sj;
        s_S[j] = part;  // local inclusive
        if (!init) {
            K->acc_ne[j] += ne;
            K->acc_wn[j] += K->dep_n[j];
            K->acc_we[j] += K->dep_e[j];
        }
        K->dep_n[j] = 0.0;
        K->dep_e[j] = 0.0;
        K->s_iz[j] = 0.0;
    }
    // S_j = sum_{k=1..j} s_k
    const double off = block_exscan(part, red, nullptr);
    double ssum = 0.0;
    for (int j = j0; j < j1; ++j) {
        s_S[j] += off;
        if (j <= G - 2) ssum += s_S[j];
    }
    double stot;
    block_exscan(ssum, red, &stot);
    // d_0 = (phi_N - phi_0 + sum_{j=0}^{G-2} S_j)/(G-1); d_j = d_0 - S_j
    const double d0 = FAST ? (0.0 - phi0 + stot) * K->inv_gm1 : (0.0 - phi0 + stot) / (double)(G - 1);
    double dpart = 0.0;
    for (int j = j0; j < j1; ++j) {
        const double dj = j <= G - 2 ? d0 - s_S[j] : 0.0;
        s_phi[j] = dpart;  // local exclusive
        dpart += dj;
    }
    const double doff = block_exscan(dpart, red, nullptr);
    for (int j = j0; j < j1; ++j) s_phi[j] = phi0 + doff + s_phi[j];
    __syncthreads();
    if (t == 0) s_phi[G - 1] = 0.0;
    __syncthreads();
    int bad = 0;
    const double inv_dz = fc.inv_dz, half_inv_dz = fc.half_inv_dz, c_gauss = fc.c_gauss;
    for (int j = j0; j < j1; ++j) {
        double e;
        if (FAST) {
            if (j == 0)
                e = -d0 * inv_dz - s_rho[0] * c_gauss;
            else if (j == G - 1)
                e = -(d0 - s_S[G - 2]) * inv_dz + s_rho[G - 1] * c_gauss;
            else
                e = -((d0 - s_S[j]) + (d0 - s_S[j - 1])) * half_inv_dz;
        } else if (j == 0) {
            e = -d0 / dz - s_rho[0] * dz / (2.0 * kEps0);
        } else if (j == G - 1) {
            e = -(d0 - s_S[G - 2]) / dz + s_rho[G - 1] * dz / (2.0 * kEps0);
        } else {
            e = -((d0 - s_S[j]) + (d0 - s_S[j - 1])) / (2.0 * dz);
        }
        K->E[j] = e;
        K->Ef[j] = (float)e;
        K->phi[j] = s_phi[j];
        if (!isfinite(e) || !isfinite(s_ni[j])) bad = 1;
    }
    if (bad) red.flag = 1;
    __syncthreads();
    if (red.flag && t == 0) atomicOr(&K->status, (unsigned)HYB_STATUS_NONFINITE);

    if (init) {
        if (t == 0) {
            K->n_slots_step = (int64_t)K->n_slots;
            K->init_pending = 0;
        }
        return;
    }

    // ------------------------------------------- bookkeeping, gamma emission
    __shared__ int s_cnt[2];
    __shared__ unsigned long long s_base;
    if (t == 0) {
        if (red.count) K->ctr[C_CLAMP] += red.count;
        K->n_samples += 1;
        const double v_old = K->v_dc + K->v_rf * sin(kTwoPi * K->f_rf * ((double)K->step * dt));
        if (kin) {  // the ions removed at each wall this step
            const InstDev *I = K->ion;
            const unsigned long long l0 = I->ctr[C_LOSS0], l1 = I->ctr[C_LOSS1];
            K->flux_in[0] = (double)(l0 - K->ion_loss_prev[0]) * w / dt;
            K->flux_in[1] = (double)(l1 - K->ion_loss_prev[1]) * w / dt;
            K->ion_loss_prev[0] = l0;
            K->ion_loss_prev[1] = l1;
        } else {
            const double g0 = gfin[0], gN = gfin[G - 1];
            K->flux_in[0] = g0 < 0.0 ? -g0 : 0.0;
            K->flux_in[1] = gN > 0.0 ? gN : 0.0;
        }
        K->step += 1;
        const uint32_t n = (uint32_t)K->step;
        s_cnt[0] = s_cnt[1] = 0;
        if ((K->gamma_see > 0.0 || K->gamma_met > 0.0) && w > 0.0) {
            for (int wall = 0; wall < 2; ++wall) {
                // ions and metastables striking the wall (Sec. II.D)
                const double ns = (K->gamma_see * K->flux_in[wall] + K->gamma_met * K->flux_met[wall]) * dt / w;
                if (!(ns > 0.0)) continue;
                const double k = floor(ns);
                const double frac = ns - k;
                const uint4 r = draw(0xFFFFFFFFFFFFFF00ull | (uint64_t)wall, n, K->seed_lo, K->seed_hi, 3);
                int64_t c = (int64_t)k + (u01d(r.x) < frac ? 1 : 0);
                if (c > (1 << 20) - 1) {
                    c = (1 << 20) - 1;
                    K->status |= HYB_STATUS_EMIT_CAP;
                }
                s_cnt[wall] = (int)c;
            }
        }
        s_base = K->n_slots;
        const unsigned long long tot = (unsigned long long)(s_cnt[0] + s_cnt[1]);
        K->n_slots = s_base + tot;
        K->ctr[C_SEE0] += s_cnt[0];
        K->ctr[C_SEE1] += s_cnt[1];
        // Absorbed power (Eq. 2.9): V J dt per step at the driven electrode, V at
        // mid-step, J along +z = ion flux + electrons absorbed (+) and emitted (-)
        // there + displacement current; at the end of an RF period P_abs and the
        // amplitude of the next period
        const unsigned long long l0 = K->ctr[C_LOSS0];
        const int64_t d_loss0 = (int64_t)(l0 - K->pw_loss0), d_see0 = s_cnt[0];
        K->pw_loss0 = l0;
        const double v_mid = 0.5 * (v_old + fc.phi0);
        const double jz = kQe * gfin[0] + kQe * w * (double)(d_loss0 - d_see0) / dt + kEps0 * (K->E[0] - s_E[0]) / dt;
        K->pw_acc += v_mid * jz * dt;
        if (++K->pw_count == K->pw_steps) {
            K->pw_last = K->pw_acc / ((double)K->pw_steps * dt);
            if (K->pw_target > 0.0 && K->pw_alpha > 0.0)
                K->v_rf = K->v_rf * (1.0 - K->pw_alpha * (K->pw_last - K->pw_target) / K->pw_target);
            K->pw_acc = 0.0;
            K->pw_count = 0;
            K->pw_periods += 1;
        }
    }
    __syncthreads();
    const int ntot = s_cnt[0] + s_cnt[1];
    if (ntot) {
        const PartBuf P = K->buf[K->cur];
        const uint32_t n = (uint32_t)K->step;
        const double sp = K->see_speed, L = K->L;
        for (int k = t; k < ntot; k += T) {
            const int wall = k < s_cnt[0] ? 0 : 1;
            const uint32_t j = (uint32_t)(wall == 0 ? k : k - s_cnt[0]);
            const uint64_t id = see_id(wall, n, j);
            const uint4 r = draw(id, n, K->seed_lo, K->seed_hi, 7);
            const double ct = sqrt(u01d(r.x));
            const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
            const double ph = kTwoPi * u01d(r.y);
            const double vn = sp * ct;
            const double vx = sp * st * cos(ph), vy = sp * st * sin(ph);
            double vz, z;
            if (wall == 0) {
                vz = vn;
                z = u01d(r.z) * vn * dt;
            } else {
                vz = -vn;
                z = L - u01d(r.z) * vn * dt;
            }
            const unsigned long long slot = s_base + (unsigned long long)k;
            if (slot >= (unsigned long long)K->capacity) {
                atomicOr(&K->status, (unsigned)HYB_STATUS_CAPACITY);
                continue;
            }
            P.id[slot] = id;
            if (K->precision == HYB_FP32_SPLIT) {
                const double x = z / dz;
                const double f = floor(x);
                int c = (int)f;
                double o = x - f;
                if (c >= K->n_cells) {
                    c = K->n_cells - 1;
                    o = 1.0;
                }
                P.c[slot] = c;
                P.o[slot] = (float)o;
                P.vxf[slot] = (float)vx;
                P.vyf[slot] = (float)vy;
                P.vzf[slot] = (float)vz;
            } else {
                P.z[slot] = z;
                P.vxd[slot] = vx;
                P.vyd[slot] = vy;
                P.vzd[slot] = vz;
            }
        }
    }
    __syncthreads();
    if (t == 0) {
        unsigned long long ns = K->n_slots;
        if (ns > (unsigned long long)K->capacity) {
            K->status |= HYB_STATUS_CAPACITY;
            ns = (unsigned long long)K->capacity;
            K->n_slots = ns;
        }
        K->n_slots_step = (int64_t)ns;
        if (K->target_step > 0 && K->step >= K->target_step) K->active = 0;
    }
}

template <bool FAST, int THREADS>
__global__ void __launch_bounds__(THREADS) k_field(InstDev *insts, int n_max, int64_t *prefix, unsigned *ticket,
                                                   int max_nodes)
{
    extern __shared__ __align__(16) double sm[];
    __shared__ Red red;
    __shared__ float s_tabf[FAST ? 4 * kMaxTab : 1];
    __shared__ FieldConsts fc;
    InstDev *K = &insts[blockIdx.x];
    const bool run = K->active || K->init_pending;
    if (run && HYB_CHECK(K->G >= 3 && K->G <= max_nodes && K->n_tab <= kMaxTab, 20, K->G, max_nodes))
        field_body<FAST>(K, sm, red, s_tabf, fc);
    // the last block to finish computes the chunk prefix of the next step
    __shared__ bool s_last;
    __shared__ int64_t s_buf[HYB_MAX_INSTANCES];
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        if (s_last) __threadfence();
    }
    __syncthreads();
    if (s_last) {
        block_chunk_prefix(insts, n_max, prefix, s_buf);
        if (threadIdx.x == 0) *ticket = 0u;
    }
}

}  // namespace

size_t field_smem_bytes(int max_nodes) { return (size_t)kArrays * 8 * (size_t)max_nodes; }

void read_checks_field(unsigned long long out[3])
{
    if (cudaMemcpyFromSymbol(out, g_hyb_check, sizeof(unsigned long long) * 3) != cudaSuccess)
        out[0] = out[1] = out[2] = 0ull;
}

void configure_field_kernel()
{
    const int sm = (int)field_smem_bytes(kMaxNodes);
    cudaFuncSetAttribute(k_field<false, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_field<true, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_field<false, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_field<true, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_field<false, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_field<true, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

template <bool FAST>
cudaError_t launch_field_t(InstDev *inst, int n_max, int64_t *prefix, unsigned *ticket, int max_nodes, int threads,
                           cudaStream_t s)
{
    const size_t smem = field_smem_bytes(max_nodes);
    if (threads == 256)
        k_field<FAST, 256><<<n_max, 256, smem, s>>>(inst, n_max, prefix, ticket, max_nodes);
    else if (threads == 512)
        k_field<FAST, 512><<<n_max, 512, smem, s>>>(inst, n_max, prefix, ticket, max_nodes);
    else if (threads == 1024)
        k_field<FAST, 1024><<<n_max, 1024, smem, s>>>(inst, n_max, prefix, ticket, max_nodes);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// `fast`: FP32 transport coefficients (split mode); FP64 throughout otherwise.
// max_nodes bounds the node count of every instance launched (shared memory
// is sized for it; a larger instance is skipped by the device guard);
// threads: 256, 512 or 1024 per instance's block.
cudaError_t launch_field(InstDev *inst, int n_max, int64_t *prefix, unsigned *ticket, bool fast, int max_nodes,
                         int threads, cudaStream_t s)
{
    if (max_nodes < 3 || max_nodes > kMaxNodes || n_max > HYB_MAX_INSTANCES || n_max > threads)
        return cudaErrorInvalidValue;
    return fast ? launch_field_t<true>(inst, n_max, prefix, ticket, max_nodes, threads, s)
                : launch_field_t<false>(inst, n_max, prefix, ticket, max_nodes, threads, s);
}

}  // namespace hyb
