/*
 * oracle.c -- plain, slow FP64 CPU reference of the kinetic-electron PIC/MCC step
 * of the 1D hybrid scheme of Eremin, Hemke and Mussenbrock, "A New Hybrid Scheme
 * for Simulations of Highly Collisional RF-Driven Plasmas" (arXiv 1508.02892).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only the tests, the package's smoke check and the benchmark's
 * CPU-baseline arm use it.  It shares no code, header, table or constant with
 * the CUDA library: every formula below is written again from the paper.
 *
 * Step order follows Sec. II.A (pusher with boundary processes -> removal ->
 * charge assignment -> Monte Carlo collisions), then the coupling of Sec. II.D
 * (fluid ions, Poisson).  Where the paper is silent the readings are:
 *   - work per unit electrode area, S = 1 m^2 (Eq. 1.2);
 *   - 1D3V velocities, leapfrog start v^{-1/2} = v^0;
 *   - gamma secondaries for step n are born from the ion wall flux of step n-1,
 *     at the end of step n-1 (so they are part of the particle set between
 *     steps);
 *   - deposit before MCC, so ionization children enter n_e one step later;
 *   - boundary rows of Eqs. 2.3/2.4 by half-cell integration with a Dirichlet
 *     wall flux alpha*mu*n*E (Sec. II.C wall condition) at the wall nodes;
 *   - isotropic lab-frame scattering for every process, cold background gas;
 *   - counter-based Philox4x32-10 (Salmon et al., SC'11) replaces the paper's
 *     xorshift128 (Sec. II.A): a particle's draws are the generator's blocks
 *     at counter (step, id_lo, call, id_hi) under the discharge's seed as key,
 *     a function of (seed, particle id, step, call) alone, so that results do
 *     not depend on particle order.
 * Beyond the step itself the oracle carries the rest of Secs. II.C-II.D: the
 * auxiliary ion-swarm Monte Carlo (mobility and exchange-frequency tables),
 * the power-controlled voltage (Eq. 2.9), electron-ion recombination as a
 * null-collision process on the non-uniform ion density, metastables with
 * Penning and pooling ionization, and the fully kinetic ions of the paper's
 * comparison model.
 * Each function below names the passage it follows.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018 (e and k_B exact) */
#define Q_E 1.602176634e-19
#define M_E 9.1093837015e-31
#define K_B 1.380649e-23
#define EPS0 8.8541878128e-12
#define AMU 1.66053906660e-27
#define TWO_PI 6.283185307179586476925286766559

#define ION_DD_CONST 0
#define ION_DD_TABLE 1
#define ION_FULL 2
#define ION_KINETIC 3   /* ions as macroparticles (the paper's fully kinetic comparison model) */

/* test-only switches of the oracle */
#define FLAG_THERMAL_GAS 2  /* elastic scattering off a Maxwellian target at T_g */

typedef struct orc_params {
    double gap_m;
    int32_t n_cells;
    int32_t gas;            /* 0 He, 1 Ar: neutral mass when gas_mass_amu == 0 */
    double pressure_pa;
    double gas_temp_k;
    double v_rf_amp_v;
    double f_rf_hz;
    double v_dc_v;
    double dt_s;
    int64_t n_particles;
    double n0_m3;
    double te0_ev;
    double weight;          /* 0: n0 * gap / n_particles (Eq. 1.2 with S = 1) */
    double gamma_see;
    double see_energy_ev;
    int32_t ion_model;
    double ion_mass_amu;    /* 0: same as the neutral */
    double gas_mass_amu;    /* 0: by gas */
    double mu_const;
    const double *tab_eon_td, *tab_mu, *tab_nu;
    int32_t n_tab;
    const double *xs_ev, *xs_el, *xs_exc, *xs_ion;
    int32_t n_xs;
    double e_exc_ev, e_iz_ev;
    uint64_t seed;
    int32_t eedf_bins;
    double eedf_max_ev;
    int32_t flags;
    double power_w_m2;      /* prescribed absorbed power P0 per m^2 (Eq. 2.9); 0: fixed amplitude */
    double power_alpha;     /* the relaxation parameter alpha of Eq. 2.9 */
    const double *xs_rec;   /* electron-ion recombination cross section at xs_ev (NULL: none) */
    int32_t metastables;    /* 1: a metastable density fed by the excitation events (Sec. II.D) */
    double met_diff_m2s;    /* diffusion coefficient of the metastables */
    double met_n0_m3;       /* initial metastable density at the interior nodes */
    double penning_rate_m3s;  /* R of Penning ionization of the admixture by the metastables */
    double penning_target_m3; /* n_N, density of the admixture the metastables ionize */
    double penning_energy_ev; /* energy of a Penning electron, E_* - E_I */
    double pooling_rate_m3s;  /* R of metastable pooling (two metastables -> ion + electron) */
    double pooling_energy_ev; /* energy of a pooling electron */
    double gamma_met;       /* secondary-electron yield of metastables at the electrodes */
} orc_params;

typedef struct part {
    double z, vx, vy, vz;
    uint64_t id;
} part;

typedef struct orc_sim {
    orc_params p;
    /* owned copies of the tables */
    double *tab_eon, *tab_mu, *tab_nu, *tab_u;
    double *xs_ev, *xs_el, *xs_exc, *xs_ion, *xs_rec;
    /* derived */
    int G;                  /* nodes */
    double L, dz, dt, ngas, w, m_gas, m_ion, e_lo, e_hi, inv_dlog, nu_max, p_max;
    double n_floor, bin_w;
    /* particles */
    part *pp;
    int64_t np, cap;
    /* grids */
    double *ni, *gam, *phi, *E, *ne, *dep_n, *dep_e, *s_iz, *gsrc;
    /* moments */
    double *acc_ne, *acc_ni, *acc_gi, *acc_wn, *acc_we, *eedf;
    int64_t n_samples;
    /* bookkeeping */
    int64_t step;
    int64_t births_iz, births_see[2], losses[2], coll[4], n_clamp, recomb;
    double rec_svmax;       /* bound of sigma_rec(E) v(E) over the table */
    int64_t status;
    double flux_in[2];      /* ion flux into each wall, from the last fluid update */
    /* power control (Eq. 2.9) */
    double u_rf;            /* current RF amplitude U^N */
    double pw_acc;          /* sum over the period so far of V J dt */
    double pw_last;         /* P_abs of the last finished period */
    int64_t pw_steps;       /* steps per RF period */
    int64_t pw_count, pw_periods;
    /* kinetic ions */
    part *ip;
    int64_t nip, icap;
    double *dep_ni, *dep_gi;
    double mi_red, nu_max_i, p_max_i, vt_gas;
    int64_t ion_losses[2], ion_coll, ion_cand;
    /* metastables and their reactions (Sec. II.D) */
    double *met, *s_met, *acc_met;
    double flux_met[2];     /* metastables reaching each wall per m^2 and s in the last step */
    int64_t births_pen, births_pool;
} orc_sim;

double orc_swarm_nu(double ngas, double m_red, int xs_model, double g);
double orc_swarm_nu_bound(double ngas, double m_red, int xs_model, double eps_max);

/* ---------------------------------------------------------------- RNG ---- */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 5): ten rounds of two
 * 32x32->64 multiplications; the key is bumped by the Weyl constants between
 * rounds. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* uniform in (0,1) from the top 23 bits: (k + 1/2) 2^-23, exact in float and double */
double orc_u01(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* The draws of particle `id` at step `step`, call number `call`: counter
 * (step, id_lo, call, id_hi), key (seed_lo, seed_hi). */
static void draws(const orc_sim *s, uint64_t id, uint32_t step, uint32_t call, double u[4])
{
    uint32_t ctr[4] = {step, (uint32_t)id, call, (uint32_t)(id >> 32)};
    uint32_t key[2] = {(uint32_t)s->p.seed, (uint32_t)(s->p.seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    for (int i = 0; i < 4; ++i) u[i] = orc_u01(r[i]);
}

/* SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014). */
uint64_t orc_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Id of the electron ejected by an ionization of `parent` at `step`; the top bit
 * marks ionization children. */
uint64_t orc_child_id(uint64_t parent, uint32_t step)
{
    return orc_mix64(parent ^ ((uint64_t)step * 0x9E3779B97F4A7C15ull)) | (1ull << 63);
}

/* Id of the k-th gamma secondary at wall `wall` born for step `step`. */
uint64_t orc_see_id(int wall, uint32_t step, uint32_t k)
{
    return (1ull << 62) | ((uint64_t)wall << 60) | ((uint64_t)step << 20) | (uint64_t)k;
}

/* ------------------------------------------------------ cross sections ---- */

/* sigma_k(energy) from the log-spaced tables: index from the logarithm, linear
 * in energy between the bracketing nodes, clamped outside the table, and zero
 * below each inelastic threshold (Sec. II.A, "energy resolved cross-sections"). */
void orc_xs_eval(const orc_sim *s, double en, double out[3])
{
    int n = s->p.n_xs;
    int i;
    double f;
    if (en <= s->e_lo) {
        i = 0;
        f = 0.0;
    } else if (en >= s->e_hi) {
        i = n - 2;
        f = 1.0;
    } else {
        double x = log(en / s->e_lo) * s->inv_dlog;
        i = (int)floor(x);
        if (i < 0) i = 0;
        if (i > n - 2) i = n - 2;
        f = (en - s->xs_ev[i]) / (s->xs_ev[i + 1] - s->xs_ev[i]);
    }
    out[0] = s->xs_el[i] + f * (s->xs_el[i + 1] - s->xs_el[i]);
    out[1] = s->xs_exc[i] + f * (s->xs_exc[i + 1] - s->xs_exc[i]);
    out[2] = s->xs_ion[i] + f * (s->xs_ion[i + 1] - s->xs_ion[i]);
    if (en < s->p.e_exc_ev) out[1] = 0.0;
    if (en < s->p.e_iz_ev) out[2] = 0.0;
}

double orc_nu_max(const orc_sim *s) { return s->nu_max; }
double orc_p_max(const orc_sim *s) { return s->p_max; }
double orc_weight(const orc_sim *s) { return s->w; }
double orc_ngas(const orc_sim *s) { return s->ngas; }

/* ---------------------------------------------------- transport tables ---- */

static double interp_lin(const double *x, const double *y, int n, double v)
{
    if (v <= x[0]) return y[0];
    if (v >= x[n - 1]) return y[n - 1];
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (x[mid] <= v)
            lo = mid;
        else
            hi = mid;
    }
    double f = (v - x[lo]) / (x[lo + 1] - x[lo]);
    return y[lo] + f * (y[lo + 1] - y[lo]);
}

/* Ion mobility at field |E| (Sec. II.C, Tables 2/4 as tabulated input). */
static double mobility(const orc_sim *s, double e_abs)
{
    if (s->p.ion_model == ION_DD_CONST) return s->p.mu_const;
    double eon_td = e_abs / s->ngas * 1e21;
    return interp_lin(s->tab_eon, s->tab_mu, s->p.n_tab, eon_td);
}

/* Ion temperature in joules: T_N for the constant-mobility model (Einstein
 * relation at the gas temperature), Eq. 2.8 otherwise. */
static double ion_temp(const orc_sim *s, double mu, double e_abs)
{
    double t = K_B * s->p.gas_temp_k;
    if (s->p.ion_model == ION_DD_CONST) return t;
    double mi = s->m_ion, mn = s->m_gas;
    double ud = mu * e_abs;
    return t + (mi + mn) / (5.0 * mi + 3.0 * mn) * mn * ud * ud;
}

/* Momentum-exchange frequency at drift speed |u| (Sec. II.B, Tables 3/5 as
 * tabulated input, abscissa u_k = mu_k E_k). */
static double exch_freq(const orc_sim *s, double u_abs)
{
    return interp_lin(s->tab_u, s->tab_nu, s->p.n_tab, u_abs);
}

/* The transport coefficients the fluid update takes at field |E| and drift
 * speed |u|: out = {mu (Sec. II.C), T_i in J (Eq. 2.8), D = mu T_i / e
 * (Eq. 2.7), nu (Sec. II.B)}.  Read by the tests. */
void orc_ion_transport(const orc_sim *s, double e_abs, double u_abs, double out[4])
{
    double mu = mobility(s, e_abs);
    double t = ion_temp(s, mu, e_abs);
    out[0] = mu;
    out[1] = t;
    out[2] = mu * t / Q_E;
    out[3] = exch_freq(s, u_abs);
}

/* ------------------------------------------------------------ Poisson ---- */

/* -eps0 phi'' = rho on the uniform grid, 3-point differences, Dirichlet ends,
 * solved by the Thomas algorithm (Sec. II.D).  E at interior nodes by central
 * difference; at the wall nodes by Gauss's law over the half cell. */
void orc_poisson(int G, double dz, const double *rho, double phi0, double phiN, double *phi, double *E)
{
    int m = G - 2; /* unknowns phi_1 .. phi_{G-2} */
    phi[0] = phi0;
    phi[G - 1] = phiN;
    if (m > 0) {
        double *cp = (double *)malloc(sizeof(double) * m);
        double *dp = (double *)malloc(sizeof(double) * m);
        /* row j (1..G-2): phi_{j-1} - 2 phi_j + phi_{j+1} = -dz^2 rho_j / eps0 */
        for (int k = 0; k < m; ++k) {
            int j = k + 1;
            double a = 1.0, b = -2.0, c = 1.0;
            double d = -dz * dz * rho[j] / EPS0;
            if (j == 1) d -= phi0;
            if (j == G - 2) d -= phiN;
            if (k == 0) {
                cp[k] = c / b;
                dp[k] = d / b;
            } else {
                double den = b - a * cp[k - 1];
                cp[k] = c / den;
                dp[k] = (d - a * dp[k - 1]) / den;
            }
        }
        phi[m] = dp[m - 1];
        for (int k = m - 2; k >= 0; --k) phi[k + 1] = dp[k] - cp[k] * phi[k + 2];
        free(cp);
        free(dp);
    }
    for (int j = 1; j < G - 1; ++j) E[j] = -(phi[j + 1] - phi[j - 1]) / (2.0 * dz);
    E[0] = -(phi[1] - phi[0]) / dz - rho[0] * dz / (2.0 * EPS0);
    E[G - 1] = -(phi[G - 1] - phi[G - 2]) / dz + rho[G - 1] * dz / (2.0 * EPS0);
}

/* Thomas algorithm for a general tridiagonal system a x_{j-1} + b x_j + c x_{j+1} = d. */
static void thomas(int m, const double *a, const double *b, const double *c, const double *d, double *x)
{
    double *cp = (double *)malloc(sizeof(double) * m);
    double *dp = (double *)malloc(sizeof(double) * m);
    cp[0] = c[0] / b[0];
    dp[0] = d[0] / b[0];
    for (int k = 1; k < m; ++k) {
        double den = b[k] - a[k] * cp[k - 1];
        cp[k] = c[k] / den;
        dp[k] = (d[k] - a[k] * dp[k - 1]) / den;
    }
    x[m - 1] = dp[m - 1];
    for (int k = m - 2; k >= 0; --k) x[k] = dp[k] - cp[k] * x[k + 1];
    free(cp);
    free(dp);
}

/* --------------------------------------------------------- ion fluid ---- */

static double wall_flux(const orc_sim *s, int wall, double n, double E)
{
    /* alpha switch of Sec. II.C: the field-driven flux counts only when E
     * points into the electrode (E < 0 at z = 0, E > 0 at z = L). */
    int into = wall == 0 ? (E < 0.0) : (E > 0.0);
    if (!into) return 0.0;
    return mobility(s, fabs(E)) * n * E;
}

/* One ion-fluid update from level n to n+1 given E^n and the source G^n.
 * Drift-diffusion (Eqs. 2.5-2.8) explicit at level n, or the full model
 * (Eq. 2.3 for the flux at n+1/2, Thomas), then continuity (Eq. 2.4) with the
 * half-cell rows at the walls.  ni and gam are updated in place; flux_in gets
 * the ion flux into each wall; returns the number of clamped negative
 * densities. */
int64_t orc_fluid_update(orc_sim *s, const double *E, const double *gsrc, double *ni, double *gam, double flux_in[2])
{
    int G = s->G;
    double dz = s->dz, dt = s->dt;
    double *gnew = (double *)calloc(G, sizeof(double));
    if (s->p.ion_model == ION_FULL) {
        /* Eq. 2.3: tridiagonal in Gamma^{n+1/2}; nu at u^n = Gamma^{n-1/2}/n^n. */
        double *A = (double *)calloc(G, sizeof(double));
        double *T = (double *)calloc(G, sizeof(double));
        for (int j = 0; j < G; ++j) {
            A[j] = ni[j] >= s->n_floor ? gam[j] / ni[j] : 0.0;
            double mu = mobility(s, fabs(E[j]));
            T[j] = ion_temp(s, mu, fabs(E[j]));
        }
        gnew[0] = wall_flux(s, 0, ni[0], E[0]);
        gnew[G - 1] = wall_flux(s, 1, ni[G - 1], E[G - 1]);
        int m = G - 2;
        if (m > 0) {
            double *a = (double *)malloc(sizeof(double) * m), *b = (double *)malloc(sizeof(double) * m);
            double *c = (double *)malloc(sizeof(double) * m), *d = (double *)malloc(sizeof(double) * m);
            double *x = (double *)malloc(sizeof(double) * m);
            double h = dt / (2.0 * dz);
            for (int k = 0; k < m; ++k) {
                int j = k + 1;
                double nu = exch_freq(s, fabs(A[j]));
                a[k] = -h * A[j - 1];
                b[k] = 1.0 + nu * dt / 2.0;
                c[k] = h * A[j + 1];
                d[k] = gam[j] * (1.0 - nu * dt / 2.0) + Q_E * ni[j] * E[j] * dt / s->m_ion -
                       h / s->m_ion * (ni[j + 1] * T[j + 1] - ni[j - 1] * T[j - 1]);
            }
            d[0] -= a[0] * gnew[0];
            d[m - 1] -= c[m - 1] * gnew[G - 1];
            a[0] = 0.0;
            c[m - 1] = 0.0;
            thomas(m, a, b, c, d, x);
            for (int k = 0; k < m; ++k) gnew[k + 1] = x[k];
            free(a);
            free(b);
            free(c);
            free(d);
            free(x);
        }
        free(A);
        free(T);
    } else {
        /* Eq. 2.5 at level n: Gamma = mu n E - D dn/dz, D = mu T / e (Eq. 2.7). */
        for (int j = 1; j < G - 1; ++j) {
            double mu = mobility(s, fabs(E[j]));
            double D = mu * ion_temp(s, mu, fabs(E[j])) / Q_E;
            gnew[j] = mu * ni[j] * E[j] - D * (ni[j + 1] - ni[j - 1]) / (2.0 * dz);
        }
        gnew[0] = wall_flux(s, 0, ni[0], E[0]);
        gnew[G - 1] = wall_flux(s, 1, ni[G - 1], E[G - 1]);
    }
    /* Eq. 2.4 with G^{n+1/2} -> G^n; half-cell rows at the walls. */
    int64_t clamps = 0;
    double *nnew = (double *)malloc(sizeof(double) * G);
    for (int j = 1; j < G - 1; ++j)
        nnew[j] = ni[j] - dt / (2.0 * dz) * (gnew[j + 1] - gnew[j - 1]) + dt * gsrc[j];
    nnew[0] = ni[0] - dt / dz * (gnew[1] - gnew[0]) + dt * gsrc[0];
    nnew[G - 1] = ni[G - 1] - dt / dz * (gnew[G - 1] - gnew[G - 2]) + dt * gsrc[G - 1];
    for (int j = 0; j < G; ++j) {
        if (nnew[j] < 0.0) {
            nnew[j] = 0.0;
            ++clamps;
        }
        ni[j] = nnew[j];
        gam[j] = gnew[j];
    }
    flux_in[0] = gnew[0] < 0.0 ? -gnew[0] : 0.0;
    flux_in[1] = gnew[G - 1] > 0.0 ? gnew[G - 1] : 0.0;
    free(nnew);
    free(gnew);
    return clamps;
}

/* ---------------------------------------------------------- particles ---- */

static void push_particle(orc_sim *s, const part *q)
{
    if (s->np == s->cap) {
        s->cap = s->cap ? 2 * s->cap : 1024;
        s->pp = (part *)realloc(s->pp, sizeof(part) * (size_t)s->cap);
    }
    s->pp[s->np++] = *q;
}

static void push_ion(orc_sim *s, const part *q)
{
    if (s->nip == s->icap) {
        s->icap = s->icap ? 2 * s->icap : 1024;
        s->ip = (part *)realloc(s->ip, sizeof(part) * (size_t)s->icap);
    }
    s->ip[s->nip++] = *q;
}

/* Cell index and CIC offset of position z (Eq. 1.1 with CIC shape). */
static void locate(const orc_sim *s, double z, int *c, double *o)
{
    double x = z / s->dz;
    double f = floor(x);
    int ci = (int)f;
    double oo = x - f;
    if (ci >= s->p.n_cells) {
        ci = s->p.n_cells - 1;
        oo = 1.0;
    }
    *c = ci;
    *o = oo;
}

static double energy_ev(const part *q)
{
    return 0.5 * M_E * (q->vx * q->vx + q->vy * q->vy + q->vz * q->vz) / Q_E;
}

static void iso_dir(double u_cos, double u_phi, double d[3])
{
    double ct = 1.0 - 2.0 * u_cos;
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double ph = TWO_PI * u_phi;
    d[0] = st * cos(ph);
    d[1] = st * sin(ph);
    d[2] = ct;
}

/* Box-Muller on two uniforms. */
static void gauss2(double u1, double u2, double *g1, double *g2)
{
    double r = sqrt(-2.0 * log(u1));
    double ph = TWO_PI * u2;
    *g1 = r * cos(ph);
    *g2 = r * sin(ph);
}

enum { OUT_NONE = 0, OUT_ELASTIC = 1, OUT_EXC = 2, OUT_ION = 3, OUT_NULL = 4, OUT_LOST0 = 5, OUT_LOST1 = 6 };

/* Pusher, boundary check and removal for one particle (Sec. II.A): CIC gather
 * of E^n, leapfrog v^{n-1/2} -> v^{n+1/2}, z^n -> z^{n+1}.  Returns 0 if the
 * particle stays in (0, L), else 1 + wall index. */
static int push_one(const orc_sim *s, const double *E, part *q)
{
    int c;
    double o;
    locate(s, q->z, &c, &o);
    double ep = (1.0 - o) * E[c] + o * E[c + 1];
    q->vz = q->vz - (Q_E / M_E) * ep * s->dt;
    q->z = q->z + q->vz * s->dt;
    if (q->z < 0.0) return 1;
    if (q->z >= s->L) return 2;
    return 0;
}

/* Modified null-collision MCC for one particle at step n (Sec. II.A, Mertmann
 * et al.; ionization births and ion source of Sec. II.D).  Every particle draws
 * R1 and is a candidate if R1 < P_max; the process is the first k with
 * R2 nu_max < sum_{i<=k} nu_i(E).  Returns the outcome; fills *child on an
 * ionization. */
static int mcc_one(const orc_sim *s, uint32_t n, part *q, part *child)
{
    double u[4];
    draws(s, q->id, n, 0, u);
    if (!(u[0] < s->p_max)) return OUT_NONE;
    double en = energy_ev(q);
    double speed = sqrt(q->vx * q->vx + q->vy * q->vy + q->vz * q->vz);
    double sig[3];
    orc_xs_eval(s, en, sig);
    double nu_el = s->ngas * sig[0] * speed;
    double nu_ex = s->ngas * sig[1] * speed;
    double nu_iz = s->ngas * sig[2] * speed;
    double r = u[1] * s->nu_max;
    double d[3];
    iso_dir(u[2], u[3], d);
    if (r < nu_el) {
        if (s->p.flags & FLAG_THERMAL_GAS) {
            /* test-only: elastic collision with a Maxwellian target at T_g,
             * isotropic in the centre-of-mass frame */
            double g[4], V[3];
            draws(s, q->id, n, 2, g);
            double vt = sqrt(K_B * s->p.gas_temp_k / s->m_gas);
            double a1, a2, a3, a4;
            gauss2(g[0], g[1], &a1, &a2);
            gauss2(g[2], g[3], &a3, &a4);
            V[0] = vt * a1;
            V[1] = vt * a2;
            V[2] = vt * a3;
            double mt = M_E + s->m_gas;
            double vc[3] = {(M_E * q->vx + s->m_gas * V[0]) / mt, (M_E * q->vy + s->m_gas * V[1]) / mt,
                            (M_E * q->vz + s->m_gas * V[2]) / mt};
            double gx = q->vx - V[0], gy = q->vy - V[1], gz = q->vz - V[2];
            double gm = sqrt(gx * gx + gy * gy + gz * gz);
            double f = s->m_gas / mt * gm;
            q->vx = vc[0] + f * d[0];
            q->vy = vc[1] + f * d[1];
            q->vz = vc[2] + f * d[2];
            return OUT_ELASTIC;
        }
        /* elastic: energy loss (2m/M)(1 - cos chi) of the energy, chi the
         * angle between old and new directions */
        double cchi = (q->vx * d[0] + q->vy * d[1] + q->vz * d[2]) / speed;
        double sp = speed * sqrt(1.0 - 2.0 * (M_E / s->m_gas) * (1.0 - cchi));
        q->vx = sp * d[0];
        q->vy = sp * d[1];
        q->vz = sp * d[2];
        return OUT_ELASTIC;
    }
    if (r < nu_el + nu_ex) {
        double sp = sqrt(2.0 * Q_E * (en - s->p.e_exc_ev) / M_E);
        q->vx = sp * d[0];
        q->vy = sp * d[1];
        q->vz = sp * d[2];
        return OUT_EXC;
    }
    if (r < nu_el + nu_ex + nu_iz) {
        double v2[4];
        draws(s, q->id, n, 1, v2);
        double de = en - s->p.e_iz_ev;
        double e_ej = v2[0] * de;
        double e_sc = de - e_ej;
        double sp = sqrt(2.0 * Q_E * e_sc / M_E);
        double dj[3];
        iso_dir(v2[1], v2[2], dj);
        double sj = sqrt(2.0 * Q_E * e_ej / M_E);
        child->z = q->z;
        child->vx = sj * dj[0];
        child->vy = sj * dj[1];
        child->vz = sj * dj[2];
        child->id = orc_child_id(q->id, n);
        q->vx = sp * d[0];
        q->vy = sp * d[1];
        q->vz = sp * d[2];
        return OUT_ION;
    }
    return OUT_NULL;
}

/* Recombination test of one electron after its charge assignment (Sec. II.D):
 * candidate if R3 < P_rec = 1 - exp(-nu_rec,max dt), real if R4 nu_rec,max <
 * n_i(z) sigma_rec(E) v with n_i interpolated (CIC) at the electron.  A
 * recombined electron is removed and its ion leaves the ion density through
 * the source term of Eq. 2.4 (a CIC sink in s_iz).  Draws: call 2, (R3, R4). */
static int recombine(orc_sim *s, uint32_t n, const part *q, double rec_numax, double rec_pmax)
{
    double u[4];
    draws(s, q->id, n, 2, u);
    if (!(u[0] < rec_pmax)) return 0;
    int c;
    double o;
    locate(s, q->z, &c, &o);
    double nil = (1.0 - o) * s->ni[c] + o * s->ni[c + 1];
    double en = energy_ev(q);
    double speed = sqrt(q->vx * q->vx + q->vy * q->vy + q->vz * q->vz);
    int i;
    double f;
    if (en <= s->e_lo) {
        i = 0;
        f = 0.0;
    } else if (en >= s->e_hi) {
        i = s->p.n_xs - 2;
        f = 1.0;
    } else {
        double x = log(en / s->e_lo) * s->inv_dlog;
        i = (int)floor(x);
        if (i < 0) i = 0;
        if (i > s->p.n_xs - 2) i = s->p.n_xs - 2;
        f = (en - s->xs_ev[i]) / (s->xs_ev[i + 1] - s->xs_ev[i]);
    }
    double sig = s->xs_rec[i] + f * (s->xs_rec[i + 1] - s->xs_rec[i]);
    if (!(u[1] * rec_numax < nil * sig * speed)) return 0;
    s->recomb++;
    s->s_iz[c] -= 1.0 - o;
    s->s_iz[c + 1] -= o;
    return 1;
}

/* One particle through the whole per-particle part of step n, given E^n:
 * push, wall test, MCC.  Exposed for sampled checks of large runs. */
int orc_particle_step_one(const orc_sim *s, const double *E, uint32_t n, const double in[4], uint64_t id,
                          double out[4], double child_out[4], uint64_t *child_id)
{
    part q = {in[0], in[1], in[2], in[3], id};
    int w = push_one(s, E, &q);
    if (w) {
        out[0] = q.z;
        out[1] = q.vx;
        out[2] = q.vy;
        out[3] = q.vz;
        return w == 1 ? OUT_LOST0 : OUT_LOST1;
    }
    part ch;
    int oc = mcc_one(s, n, &q, &ch);
    out[0] = q.z;
    out[1] = q.vx;
    out[2] = q.vy;
    out[3] = q.vz;
    if (oc == OUT_ION) {
        child_out[0] = ch.z;
        child_out[1] = ch.vx;
        child_out[2] = ch.vy;
        child_out[3] = ch.vz;
        *child_id = ch.id;
    }
    return oc;
}

/* CIC charge assignment of one particle (Sec. II.A) plus its energy moment and
 * EEDF sample. */
static void deposit_one(orc_sim *s, const part *q, int sample)
{
    int c;
    double o;
    locate(s, q->z, &c, &o);
    s->dep_n[c] += 1.0 - o;
    s->dep_n[c + 1] += o;
    if (!sample) return;
    double en = energy_ev(q);
    s->dep_e[c] += (1.0 - o) * en;
    s->dep_e[c + 1] += o * en;
    int b = (int)(en / s->bin_w);
    if (b > s->p.eedf_bins || b < 0) b = s->p.eedf_bins;
    s->eedf[b] += 1.0;
}

/* gamma secondaries (Sec. II.D): per wall, (gamma_i Gamma_i + gamma_* Gamma_*)
 * S dt / N_p/sp superparticles (ions and metastables striking the wall), integer
 * part plus one more with the probability of the fractional part.  Born with energy see_energy_ev, Lambertian direction,
 * a random fraction of one push inside the wall. */
static void emit_secondaries(orc_sim *s, uint32_t n)
{
    if ((s->p.gamma_see <= 0.0 && s->p.gamma_met <= 0.0) || s->w <= 0.0) return;
    for (int wall = 0; wall < 2; ++wall) {
        /* heavy particles of both kinds (ions, metastables) hitting the wall */
        double ns = (s->p.gamma_see * s->flux_in[wall] + s->p.gamma_met * s->flux_met[wall]) * s->dt / s->w;
        if (!(ns > 0.0)) continue;
        double k = floor(ns);
        double frac = ns - k;
        uint64_t wid = 0xFFFFFFFFFFFFFF00ull | (uint64_t)wall;
        double u[4];
        draws(s, wid, n, 3, u);
        int64_t cnt = (int64_t)k + (u[0] < frac ? 1 : 0);
        if (cnt > (1 << 20) - 1) {
            cnt = (1 << 20) - 1;
            s->status |= 8;
        }
        double sp = sqrt(2.0 * Q_E * s->p.see_energy_ev / M_E);
        for (int64_t j = 0; j < cnt; ++j) {
            part q;
            q.id = orc_see_id(wall, n, (uint32_t)j);
            double v[4];
            draws(s, q.id, n, 7, v);
            double ct = sqrt(v[0]);
            double st = sqrt(fmax(0.0, 1.0 - ct * ct));
            double ph = TWO_PI * v[1];
            double vn = sp * ct;
            q.vx = sp * st * cos(ph);
            q.vy = sp * st * sin(ph);
            if (wall == 0) {
                q.vz = vn;
                q.z = v[2] * vn * s->dt;
            } else {
                q.vz = -vn;
                q.z = s->L - v[2] * vn * s->dt;
            }
            push_particle(s, &q);
            s->births_see[wall]++;
        }
    }
}

static double drive(const orc_sim *s, double t)
{
    return s->p.v_dc_v + s->u_rf * sin(TWO_PI * s->p.f_rf_hz * t);
}

/* Absorbed power and the amplitude update of Eq. 2.9.  Per step the power per
 * m^2 delivered through the driven electrode (z = 0) is V J, with V at mid-step
 * and J the total current density along +z there: the ion flux e Gamma_i(0),
 * the electrons absorbed at and emitted from that electrode (+e and -e times
 * their number x w / dt), and the displacement current eps0 (E_0^{n+1} -
 * E_0^n)/dt.  Summed over an RF period of round(1/(f dt)) steps and divided
 * by its duration this is P_abs^N; then U^{N+1} = U^N (1 - alpha (P_abs^N -
 * P0)/P0) holds for the next period. */
static void power_step(orc_sim *s, double v_old, double v_new, double e0_old, double e0_new, int64_t d_loss0,
                       int64_t d_see0)
{
    const double v_mid = 0.5 * (v_old + v_new);
    const double j = Q_E * s->gam[0] + Q_E * s->w * (double)(d_loss0 - d_see0) / s->dt +
                     EPS0 * (e0_new - e0_old) / s->dt;
    s->pw_acc += v_mid * j * s->dt;
    if (++s->pw_count == s->pw_steps) {
        s->pw_last = s->pw_acc / ((double)s->pw_steps * s->dt);
        if (s->p.power_w_m2 > 0.0 && s->p.power_alpha > 0.0)
            s->u_rf = s->u_rf * (1.0 - s->p.power_alpha * (s->pw_last - s->p.power_w_m2) / s->p.power_w_m2);
        s->pw_acc = 0.0;
        s->pw_count = 0;
        s->pw_periods++;
    }
}

static double node_volume(const orc_sim *s, int j)
{
    return (j == 0 || j == s->G - 1) ? 0.5 * s->dz : s->dz;
}

/* Electron density from the node sums, then Poisson at time t. */
static void solve_field(orc_sim *s, double t)
{
    int G = s->G;
    double *rho = (double *)malloc(sizeof(double) * G);
    for (int j = 0; j < G; ++j) {
        s->ne[j] = s->w * s->dep_n[j] / node_volume(s, j);
        rho[j] = Q_E * (s->ni[j] - s->ne[j]);
    }
    orc_poisson(G, s->dz, rho, drive(s, t), 0.0, s->phi, s->E);
    free(rho);
}

/* Ion density (and flux) from the ions' CIC charge assignment. */
static void ion_grids(orc_sim *s)
{
    for (int j = 0; j < s->G; ++j) {
        s->ni[j] = s->w * s->dep_ni[j] / node_volume(s, j);
        s->gam[j] = s->w * s->dep_gi[j] / node_volume(s, j);
    }
}

/* Deposit the current particles and solve for E at the current time (start of
 * a run, or after the particles were replaced). */
void orc_init_field(orc_sim *s)
{
    memset(s->dep_n, 0, sizeof(double) * s->G);
    for (int64_t i = 0; i < s->np; ++i) deposit_one(s, &s->pp[i], 0);
    if (s->p.ion_model == ION_KINETIC) {
        memset(s->dep_ni, 0, sizeof(double) * s->G);
        memset(s->dep_gi, 0, sizeof(double) * s->G);
        for (int64_t i = 0; i < s->nip; ++i) {
            int c;
            double o;
            locate(s, s->ip[i].z, &c, &o);
            s->dep_ni[c] += 1.0 - o;
            s->dep_ni[c + 1] += o;
            s->dep_gi[c] += (1.0 - o) * s->ip[i].vz;
            s->dep_gi[c + 1] += o * s->ip[i].vz;
        }
        ion_grids(s);
    }
    solve_field(s, (double)s->step * s->dt);
    memset(s->dep_n, 0, sizeof(double) * s->G);
}

/* One ion's push in E (CIC gather, leapfrog); 1 or 2 if it left through
 * z = 0 or z = L (then it is removed), else 0. */
static int ion_push(const orc_sim *s, const double *E, part *q)
{
    int c;
    double o;
    locate(s, q->z, &c, &o);
    double ep = (1.0 - o) * E[c] + o * E[c + 1];
    q->vz = q->vz + (Q_E / s->m_ion) * ep * s->dt;
    q->z = q->z + q->vz * s->dt;
    if (q->z < 0.0) return 1;
    if (q->z >= s->L) return 2;
    return 0;
}

/* One ion's collision with the gas in step n (Sec. II.C): null-collision test
 * R < P_max (call 5), a neutral from the gas Maxwellian (Box-Muller on calls 5
 * and 6), acceptance on R' nu_max < N Q_m(eps) g, isotropic scattering in the
 * centre-of-mass frame.  0: no candidate, 1: null collision, 2: collided. */
static int ion_collide(const orc_sim *s, uint32_t n, part *q)
{
    const double M = s->m_ion, mn = s->m_gas;
    double u[4], w[4];
    draws(s, q->id, n, 5, u);
    if (!(u[0] < s->p_max_i)) return 0;
    draws(s, q->id, n, 6, w);
    double b1, b2, b3, b4;
    gauss2(u[2], u[3], &b1, &b2);
    gauss2(w[0], w[1], &b3, &b4);
    double V[3] = {s->vt_gas * b1, s->vt_gas * b2, s->vt_gas * b3};
    double v[3] = {q->vx, q->vy, q->vz};
    double gx = v[0] - V[0], gy = v[1] - V[1], gz = v[2] - V[2];
    double g = sqrt(gx * gx + gy * gy + gz * gz);
    double nu = orc_swarm_nu(s->ngas, s->mi_red, 0, g);
    if (!(u[1] * s->nu_max_i < nu)) return 1;
    double d[3];
    iso_dir(w[2], w[3], d);
    for (int k = 0; k < 3; ++k) v[k] = (M * v[k] + mn * V[k]) / (M + mn) + mn / (M + mn) * g * d[k];
    q->vx = v[0];
    q->vy = v[1];
    q->vz = v[2];
    return 2;
}

/* One ion's part of step n from `in` (z, vx, vy, vz) in the field E, for the
 * tests that step sampled ions of a large run one by one: OUT_LOST0/1 if it
 * left, else 0 (no candidate), 1 (null collision) or 2 (collided); out gets
 * the new state. */
int orc_ion_step_one(const orc_sim *s, const double *E, uint32_t n, const double in[4], uint64_t id,
                     double out[4])
{
    part q = {in[0], in[1], in[2], in[3], id};
    const int w = ion_push(s, E, &q);
    int oc = w ? (w == 1 ? OUT_LOST0 : OUT_LOST1) : ion_collide(s, n, &q);
    out[0] = q.z;
    out[1] = q.vx;
    out[2] = q.vy;
    out[3] = q.vz;
    return oc;
}

/* The kinetic-ion part of step n (the paper's fully kinetic comparison model,
 * with the ion-neutral collisions of the auxiliary Monte Carlo, Sec. II.C):
 * every ionization of this step adds an ion at the child electron's position
 * (id = the child's id) with a velocity from the gas Maxwellian (call 4 at
 * step n); then every ion is pushed in E^n (CIC gather, leapfrog), removed at
 * the walls (the count per wall is that wall's ion flux for gamma emission),
 * assigned (CIC) to the ion density and flux, and collides with the gas:
 * null-collision with a neutral from the gas Maxwellian, acceptance on
 * N Q_m(eps) g, Q_m = Q_i + 2 Q_b, isotropic in the centre-of-mass frame
 * (calls 5 and 6 at step n). */
static void ion_step(orc_sim *s, uint32_t n, const double *kz, const uint64_t *kid, int64_t nk)
{
    for (int64_t i = 0; i < nk; ++i) {
        part q;
        q.id = kid[i];
        q.z = kz[i];
        double a[4], g1, g2, g3, g4;
        draws(s, q.id, n, 4, a);
        gauss2(a[0], a[1], &g1, &g2);
        gauss2(a[2], a[3], &g3, &g4);
        q.vx = s->vt_gas * g1;
        q.vy = s->vt_gas * g2;
        q.vz = s->vt_gas * g3;
        push_ion(s, &q);
    }
    const int G = s->G;
    memset(s->dep_ni, 0, sizeof(double) * G);
    memset(s->dep_gi, 0, sizeof(double) * G);
    int64_t lost[2] = {0, 0}, keep = 0;
    for (int64_t i = 0; i < s->nip; ++i) {
        part q = s->ip[i];
        const int w = ion_push(s, s->E, &q);
        if (w) {
            lost[w - 1]++;
            continue;
        }
        int c;
        double o;
        locate(s, q.z, &c, &o);
        s->dep_ni[c] += 1.0 - o;
        s->dep_ni[c + 1] += o;
        s->dep_gi[c] += (1.0 - o) * q.vz;
        s->dep_gi[c + 1] += o * q.vz;
        const int oc = ion_collide(s, n, &q);
        if (oc >= 1) s->ion_cand++;
        if (oc == 2) s->ion_coll++;
        s->ip[keep++] = q;
    }
    s->nip = keep;
    s->ion_losses[0] += lost[0];
    s->ion_losses[1] += lost[1];
    s->flux_in[0] = (double)lost[0] * s->w / s->dt;
    s->flux_in[1] = (double)lost[1] * s->w / s->dt;
    ion_grids(s);
}

/* Metastables and the ionization they cause (Sec. II.D).  Every excitation
 * event of the step adds N_p/sp/dV to the metastable density n_m (CIC at the
 * electron); here, from the density n_m^n at the start of the step:
 *  - Penning ionization of the admixture, Delta N_e = R_P n_m n_N dt dV, and
 *    metastable pooling, Delta N_e = R_pool n_m^2 dt dV, per interior node j
 *    (dV = dz S): Delta N_e / N_p/sp superparticles, the integer part plus one
 *    with the probability of the fraction (the Bernoulli draw indexed by the
 *    process and j, call 3); each new electron is placed uniformly in the
 *    node's cell [z_j - dz/2, z_j + dz/2) with the process's energy and an
 *    isotropic direction (call 7 of its own id), and its ion enters the ion
 *    source (CIC) as an ionization's would;
 *  - then the explicit update of the metastable density,
 *    n_m^{n+1} = n_m + dt [D d2n_m/dz2 + S_m - R_P n_N n_m - 2 R_pool n_m^2]
 *    at the interior nodes, n_m = 0 at the electrodes (absorbing walls); the
 *    flux into a wall is D n_m(next node)/dz plus what the excitation events
 *    put on the wall node, and it drives gamma emission with gamma_m.
 * Ids of the new electrons: bit 62 set, process 2 (Penning) or 3 (pooling) in
 * bits 60-61, the step in bits 20-51, the running index k in bits 0-19. */
static void metastable_step(orc_sim *s, uint32_t n)
{
    const int G = s->G;
    const double dz = s->dz, dt = s->dt, w = s->w;
    const double rate[2] = {s->p.penning_rate_m3s, s->p.pooling_rate_m3s};
    const double energy[2] = {s->p.penning_energy_ev, s->p.pooling_energy_ev};
    for (int proc = 0; proc < 2; ++proc) {
        if (!(rate[proc] > 0.0) || !(w > 0.0)) continue;
        const double sp = sqrt(2.0 * Q_E * energy[proc] / M_E);
        int64_t k = 0;
        for (int j = 1; j <= G - 2; ++j) {
            const double nm = s->met[j];
            const double dn = proc == 0 ? rate[0] * nm * s->p.penning_target_m3 * dt * dz
                                        : rate[1] * nm * nm * dt * dz;
            const double m = dn / w;
            if (!(m > 0.0)) continue;
            const double fl = floor(m);
            double u[4];
            draws(s, 0xFFFFFFFF00000000ull | ((uint64_t)(proc + 1) << 24) | (uint64_t)j, n, 3, u);
            int64_t cnt = (int64_t)fl + (u[0] < m - fl ? 1 : 0);
            for (int64_t b = 0; b < cnt; ++b) {
                if (k >= (1 << 20) - 1) {
                    s->status |= 8;
                    break;
                }
                part q;
                q.id = (1ull << 62) | ((uint64_t)(2 + proc) << 60) | ((uint64_t)n << 20) | (uint64_t)k;
                double v[4];
                draws(s, q.id, n, 7, v);
                q.z = ((double)j - 0.5 + v[0]) * dz;
                double ct = 1.0 - 2.0 * v[1];
                double st = sqrt(fmax(0.0, 1.0 - ct * ct));
                double ph = TWO_PI * v[2];
                q.vx = sp * st * cos(ph);
                q.vy = sp * st * sin(ph);
                q.vz = sp * ct;
                push_particle(s, &q);
                int c;
                double o;
                locate(s, q.z, &c, &o);
                s->s_iz[c] += 1.0 - o;
                s->s_iz[c + 1] += o;
                if (proc == 0)
                    s->births_pen++;
                else
                    s->births_pool++;
                ++k;
            }
        }
    }
    double *old = (double *)malloc(sizeof(double) * G);
    memcpy(old, s->met, sizeof(double) * G);
    const double D = s->p.met_diff_m2s;
    const double kp = s->p.penning_rate_m3s * s->p.penning_target_m3, kq = s->p.pooling_rate_m3s;
    for (int j = 1; j <= G - 2; ++j) {
        const double src = w * s->s_met[j] / (dz * dt);
        const double lap = D * (old[j + 1] - 2.0 * old[j] + old[j - 1]) / (dz * dz);
        const double loss = kp * old[j] + 2.0 * kq * old[j] * old[j];
        double nn = old[j] + dt * (lap + src - loss);
        if (nn < 0.0) {
            nn = 0.0;
            s->n_clamp++;
        }
        s->met[j] = nn;
    }
    s->met[0] = s->met[G - 1] = 0.0;
    s->flux_met[0] = D * old[1] / dz + w * s->s_met[0] / dt;
    s->flux_met[1] = D * old[G - 2] / dz + w * s->s_met[G - 1] / dt;
    free(old);
}

/* One full step n -> n+1 (Secs. II.A and II.D), ending with the gamma
 * secondaries that will take part in step n+1. */
static void step_once(orc_sim *s)
{
    int G = s->G;
    uint32_t n = (uint32_t)s->step;
    const double e0_old = s->E[0];
    const double v_old = drive(s, (double)s->step * s->dt);
    const int64_t loss0_before = s->losses[0], see0_before = s->births_see[0];
    memset(s->dep_n, 0, sizeof(double) * G);
    memset(s->dep_e, 0, sizeof(double) * G);
    memset(s->s_iz, 0, sizeof(double) * G);
    if (s->met) memset(s->s_met, 0, sizeof(double) * G);
    int64_t n0 = s->np;
    /* electron-ion recombination (Sec. II.D): a null-collision procedure of its
     * own on the non-uniform ion density, nu_rec,max = max_z n_i * max sigma v */
    double rec_numax = 0.0, rec_pmax = 0.0;
    if (s->xs_rec) {
        double nimax = 0.0;
        for (int j = 0; j < G; ++j)
            if (s->ni[j] > nimax) nimax = s->ni[j];
        rec_numax = nimax * s->rec_svmax;
        rec_pmax = -expm1(-rec_numax * s->dt);
    }
    part *kids = NULL;
    int64_t nk = 0, ck = 0;
    int64_t keep = 0;
    for (int64_t i = 0; i < n0; ++i) {
        part q = s->pp[i];
        int w = push_one(s, s->E, &q);
        if (w) {
            s->losses[w - 1]++;
            continue;
        }
        deposit_one(s, &q, 1);
        if (s->xs_rec && recombine(s, n, &q, rec_numax, rec_pmax)) continue;
        part ch;
        int oc = mcc_one(s, n, &q, &ch);
        if (oc == OUT_ELASTIC) s->coll[0]++;
        if (oc == OUT_EXC) {
            s->coll[1]++;
            if (s->met) {  /* a metastable at the electron's position */
                int c;
                double o;
                locate(s, q.z, &c, &o);
                s->s_met[c] += 1.0 - o;
                s->s_met[c + 1] += o;
            }
        }
        if (oc == OUT_NULL) s->coll[3]++;
        if (oc == OUT_ION) {
            s->coll[2]++;
            s->births_iz++;
            int c;
            double o;
            locate(s, ch.z, &c, &o);
            s->s_iz[c] += 1.0 - o;
            s->s_iz[c + 1] += o;
            if (nk == ck) {
                ck = ck ? 2 * ck : 256;
                kids = (part *)realloc(kids, sizeof(part) * (size_t)ck);
            }
            kids[nk++] = ch;
        }
        s->pp[keep++] = q;
    }
    s->np = keep;
    double *kids_z = (double *)malloc(sizeof(double) * (size_t)(nk ? nk : 1));
    uint64_t *kids_id = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nk ? nk : 1));
    for (int64_t i = 0; i < nk; ++i) {
        kids_z[i] = kids[i].z;
        kids_id[i] = kids[i].id;
        push_particle(s, &kids[i]);
    }
    free(kids);

    if (s->met) metastable_step(s, n);
    /* coupling: ion source, fluid ions, Poisson */
    for (int j = 0; j < G; ++j) s->gsrc[j] = s->w * s->s_iz[j] / (node_volume(s, j) * s->dt);
    if (s->p.ion_model == ION_KINETIC)
        ion_step(s, n, kids_z, kids_id, nk);
    else
        s->n_clamp += orc_fluid_update(s, s->E, s->gsrc, s->ni, s->gam, s->flux_in);
    solve_field(s, (double)(s->step + 1) * s->dt);

    for (int j = 0; j < G; ++j) {
        s->acc_ne[j] += s->ne[j];
        s->acc_ni[j] += s->ni[j];
        s->acc_gi[j] += s->gam[j];
        s->acc_wn[j] += s->dep_n[j];
        s->acc_we[j] += s->dep_e[j];
        if (s->met) s->acc_met[j] += s->met[j];
    }
    free(kids_z);
    free(kids_id);
    s->n_samples++;
    const double v_new = drive(s, (double)(s->step + 1) * s->dt);
    s->step++;
    /* secondaries of the next step, from the ion wall flux just computed */
    emit_secondaries(s, (uint32_t)s->step);
    power_step(s, v_old, v_new, e0_old, s->E[0], s->losses[0] - loss0_before, s->births_see[0] - see0_before);
}

int orc_step(orc_sim *s, int64_t nsteps)
{
    for (int64_t i = 0; i < nsteps; ++i) step_once(s);
    return (int)s->status;
}

/* ---------------------------------------------------------- lifecycle ---- */

static double *dup(const double *x, int n)
{
    double *y = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    if (n > 0) memcpy(y, x, sizeof(double) * n);
    return y;
}

/* Initial load: uniform positions and a Maxwellian at te0 (Box-Muller), ids
 * 0..N-1, draws at the reserved step 0xFFFFFFFF. */
static void load_particles(orc_sim *s)
{
    double vth = sqrt(Q_E * s->p.te0_ev / M_E);
    for (int64_t j = 0; j < s->p.n_particles; ++j) {
        part q;
        q.id = (uint64_t)j;
        double a[4], b[4];
        draws(s, q.id, 0xFFFFFFFFu, 0, a);
        draws(s, q.id, 0xFFFFFFFFu, 1, b);
        q.z = a[0] * s->L;
        double g1, g2, g3, g4;
        gauss2(a[1], a[2], &g1, &g2);
        gauss2(a[3], b[0], &g3, &g4);
        q.vx = vth * g1;
        q.vy = vth * g2;
        q.vz = vth * g3;
        push_particle(s, &q);
    }
}

/* Kinetic ions: n_particles ions, ids 2^61 + i, uniform in [0, L), Maxwellian
 * at the gas temperature, drawn at step 0xFFFFFFFF with calls 4 (position and
 * a Box-Muller pair) and 5 (a second pair). */
static void load_ions(orc_sim *s)
{
    for (int64_t j = 0; j < s->p.n_particles; ++j) {
        part q;
        q.id = (1ull << 61) + (uint64_t)j;
        double a[4], b[4];
        draws(s, q.id, 0xFFFFFFFFu, 4, a);
        draws(s, q.id, 0xFFFFFFFFu, 5, b);
        q.z = a[0] * s->L;
        double g1, g2, g3, g4;
        gauss2(a[1], a[2], &g1, &g2);
        gauss2(b[0], b[1], &g3, &g4);
        q.vx = s->vt_gas * g1;
        q.vy = s->vt_gas * g2;
        q.vz = s->vt_gas * g3;
        push_ion(s, &q);
    }
}

orc_sim *orc_create(const orc_params *p)
{
    if (p->n_cells < 2 || p->n_xs < 2 || p->gap_m <= 0 || p->dt_s <= 0) return NULL;
    /* metastables: explicit diffusion stable (D dt/dz^2 <= 1/2), fluid ions only */
    if (p->metastables && (p->ion_model == ION_KINETIC || p->met_diff_m2s < 0 ||
                           p->met_diff_m2s * p->dt_s * p->n_cells * p->n_cells > 0.5 * p->gap_m * p->gap_m))
        return NULL;
    /* explicit drift-diffusion (Eq. 2.5 into Eq. 2.4): u^2 dt <= 2 D and
     * D dt / dz^2 <= 1/2 at the drive's field across the empty gap */
    if (p->ion_model == ION_DD_CONST || p->ion_model == ION_DD_TABLE) {
        double e = (fabs(p->v_dc_v) + fabs(p->v_rf_amp_v)) / p->gap_m;
        double kt = K_B * p->gas_temp_k, mu = p->mu_const, t = kt;
        if (p->ion_model == ION_DD_TABLE) {
            mu = interp_lin(p->tab_eon_td, p->tab_mu, p->n_tab, e / (p->pressure_pa / kt) * 1e21);
            double mn = (p->gas_mass_amu > 0 ? p->gas_mass_amu : (p->gas == 1 ? 39.948 : 4.002602)) * AMU;
            double mi = p->ion_mass_amu > 0 ? p->ion_mass_amu * AMU : mn;
            t = kt + (mi + mn) / (5.0 * mi + 3.0 * mn) * mn * (mu * e) * (mu * e);
        }
        double d = mu * t / Q_E, u = mu * e, dz = p->gap_m / p->n_cells;
        if (u * u * p->dt_s > 2.0 * d || d * p->dt_s > 0.5 * dz * dz) return NULL;
    }
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->p = *p;
    s->xs_ev = dup(p->xs_ev, p->n_xs);
    s->xs_el = dup(p->xs_el, p->n_xs);
    s->xs_exc = dup(p->xs_exc, p->n_xs);
    s->xs_ion = dup(p->xs_ion, p->n_xs);
    s->xs_rec = p->xs_rec ? dup(p->xs_rec, p->n_xs) : NULL;
    s->tab_eon = dup(p->tab_eon_td, p->n_tab);
    s->tab_mu = dup(p->tab_mu, p->n_tab);
    s->tab_nu = dup(p->tab_nu, p->n_tab);
    s->p.xs_ev = s->p.xs_el = s->p.xs_exc = s->p.xs_ion = s->p.xs_rec = NULL;
    s->p.tab_eon_td = s->p.tab_mu = s->p.tab_nu = NULL;
    if (s->p.eedf_bins <= 0) s->p.eedf_bins = 256;
    if (s->p.eedf_max_ev <= 0) s->p.eedf_max_ev = 64.0;
    if (s->p.see_energy_ev <= 0) s->p.see_energy_ev = 1.0;
    s->u_rf = p->v_rf_amp_v;
    s->pw_steps = p->f_rf_hz > 0 ? llround(1.0 / (p->f_rf_hz * p->dt_s)) : 0;
    if (s->pw_steps < 1) s->pw_steps = INT64_MAX;  /* no RF period: no update */

    s->G = p->n_cells + 1;
    s->L = p->gap_m;
    s->dz = p->gap_m / p->n_cells;
    s->dt = p->dt_s;
    s->ngas = p->pressure_pa / (K_B * p->gas_temp_k);
    s->w = p->weight > 0 ? p->weight : (p->n_particles > 0 ? p->n0_m3 * p->gap_m / (double)p->n_particles : 0.0);
    double mg = p->gas_mass_amu > 0 ? p->gas_mass_amu : (p->gas == 1 ? 39.948 : 4.002602);
    s->m_gas = mg * AMU;
    s->m_ion = (p->ion_mass_amu > 0 ? p->ion_mass_amu : mg) * AMU;
    s->n_floor = 1e-6 * p->n0_m3;
    s->bin_w = s->p.eedf_max_ev / s->p.eedf_bins;

    /* u abscissa of the exchange-frequency table: u_k = mu_k E_k */
    s->tab_u = (double *)malloc(sizeof(double) * (p->n_tab > 0 ? p->n_tab : 1));
    for (int k = 0; k < p->n_tab; ++k) s->tab_u[k] = s->tab_mu[k] * s->tab_eon[k] * 1e-21 * s->ngas;

    /* cross-section table lookup constants and nu_max (Sec. II.A) */
    s->e_lo = s->xs_ev[0];
    s->e_hi = s->xs_ev[p->n_xs - 1];
    s->inv_dlog = (p->n_xs - 1) / log(s->e_hi / s->e_lo);
    s->nu_max = 0.0;
    for (int i = 0; i < p->n_xs; ++i) {
        double sig[3];
        orc_xs_eval(s, s->xs_ev[i], sig);
        double v = sqrt(2.0 * Q_E * s->xs_ev[i] / M_E);
        double nu = s->ngas * (sig[0] + sig[1] + sig[2]) * v;
        if (nu > s->nu_max) s->nu_max = nu;
    }
    s->p_max = 1.0 - exp(-s->nu_max * s->dt);
    /* recombination: sigma_rec v is bounded on each table segment by the larger
     * endpoint cross section times the speed at the upper end (the lookup is
     * linear in energy between nodes) */
    s->rec_svmax = 0.0;
    if (s->xs_rec) {
        for (int i = 0; i + 1 < p->n_xs; ++i) {
            double sg = fmax(s->xs_rec[i], s->xs_rec[i + 1]);
            double v = sqrt(2.0 * Q_E * s->xs_ev[i + 1] / M_E);
            if (sg * v > s->rec_svmax) s->rec_svmax = sg * v;
        }
    }

    int G = s->G;
    s->ni = (double *)calloc(G, sizeof(double));
    s->gam = (double *)calloc(G, sizeof(double));
    s->phi = (double *)calloc(G, sizeof(double));
    s->E = (double *)calloc(G, sizeof(double));
    s->ne = (double *)calloc(G, sizeof(double));
    s->dep_n = (double *)calloc(G, sizeof(double));
    s->dep_e = (double *)calloc(G, sizeof(double));
    s->s_iz = (double *)calloc(G, sizeof(double));
    s->gsrc = (double *)calloc(G, sizeof(double));
    s->acc_ne = (double *)calloc(G, sizeof(double));
    s->acc_ni = (double *)calloc(G, sizeof(double));
    s->acc_gi = (double *)calloc(G, sizeof(double));
    s->acc_wn = (double *)calloc(G, sizeof(double));
    s->acc_we = (double *)calloc(G, sizeof(double));
    s->eedf = (double *)calloc(s->p.eedf_bins + 1, sizeof(double));
    for (int j = 0; j < G; ++j) s->ni[j] = p->n0_m3;
    if (p->metastables) {
        s->met = (double *)calloc(G, sizeof(double));
        s->s_met = (double *)calloc(G, sizeof(double));
        s->acc_met = (double *)calloc(G, sizeof(double));
        for (int j = 1; j <= G - 2; ++j) s->met[j] = p->met_n0_m3;
    }

    if (p->ion_model == ION_KINETIC) {
        s->dep_ni = (double *)calloc(G, sizeof(double));
        s->dep_gi = (double *)calloc(G, sizeof(double));
        s->mi_red = s->m_ion * s->m_gas / (s->m_ion + s->m_gas);
        s->nu_max_i = orc_swarm_nu_bound(s->ngas, s->mi_red, 0, 100.0);
        s->p_max_i = -expm1(-s->nu_max_i * s->dt);
        s->vt_gas = sqrt(K_B * p->gas_temp_k / s->m_gas);
        load_ions(s);
    }
    load_particles(s);
    orc_init_field(s);
    return s;
}

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    double *bufs[] = {s->tab_eon, s->tab_mu, s->tab_nu, s->tab_u, s->xs_ev, s->xs_el, s->xs_exc, s->xs_ion, s->xs_rec,
                      s->dep_ni, s->dep_gi,
                      s->ni, s->gam, s->phi, s->E, s->ne, s->dep_n, s->dep_e, s->s_iz, s->gsrc,
                      s->acc_ne, s->acc_ni, s->acc_gi, s->acc_wn, s->acc_we, s->eedf, s->met, s->s_met, s->acc_met};
    for (size_t i = 0; i < sizeof(bufs) / sizeof(bufs[0]); ++i) free(bufs[i]);
    free(s->pp);
    free(s->ip);
    free(s);
}

/* ----------------------------------------------------------- accessors ---- */

int64_t orc_num_particles(const orc_sim *s) { return s->np; }
int orc_num_nodes(const orc_sim *s) { return s->G; }

static int by_id(const void *a, const void *b)
{
    uint64_t x = ((const part *)a)->id, y = ((const part *)b)->id;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Particles sorted by id. */
void orc_get_particles(orc_sim *s, double *z, double *vx, double *vy, double *vz, uint64_t *id)
{
    qsort(s->pp, (size_t)s->np, sizeof(part), by_id);
    for (int64_t i = 0; i < s->np; ++i) {
        z[i] = s->pp[i].z;
        vx[i] = s->pp[i].vx;
        vy[i] = s->pp[i].vy;
        vz[i] = s->pp[i].vz;
        id[i] = s->pp[i].id;
    }
}

void orc_set_particles(orc_sim *s, int64_t n, const double *z, const double *vx, const double *vy,
                       const double *vz, const uint64_t *id)
{
    s->np = 0;
    for (int64_t i = 0; i < n; ++i) {
        part q = {z[i], vx[i], vy[i], vz[i], id[i]};
        push_particle(s, &q);
    }
    orc_init_field(s);
}

/* which: 0 n_e, 1 n_i, 2 Gamma_i, 3 phi, 4 E, 5 ion source G */
void orc_get_grid(const orc_sim *s, int which, double *out)
{
    const double *src[] = {s->ne, s->ni, s->gam, s->phi, s->E, s->gsrc};
    memcpy(out, src[which], sizeof(double) * s->G);
}

void orc_set_grid(orc_sim *s, int which, const double *in)
{
    double *dst[] = {s->ne, s->ni, s->gam, s->phi, s->E, s->gsrc};
    memcpy(dst[which], in, sizeof(double) * s->G);
}

/* Time averages over the recorded steps: n_e, n_i, Gamma_i, mean energy per
 * node (CIC-weighted), EEDF normalised to unit area over the in-range bins
 * plus the overflow fraction in the last entry. */
int64_t orc_get_moments(const orc_sim *s, double *ne, double *ni, double *gi, double *ebar, double *eedf)
{
    int64_t ns = s->n_samples;
    for (int j = 0; j < s->G; ++j) {
        ne[j] = ns ? s->acc_ne[j] / ns : 0.0;
        ni[j] = ns ? s->acc_ni[j] / ns : 0.0;
        gi[j] = ns ? s->acc_gi[j] / ns : 0.0;
        ebar[j] = s->acc_wn[j] > 0 ? s->acc_we[j] / s->acc_wn[j] : 0.0;
    }
    double tot = 0.0;
    for (int b = 0; b <= s->p.eedf_bins; ++b) tot += s->eedf[b];
    for (int b = 0; b < s->p.eedf_bins; ++b) eedf[b] = tot > 0 ? s->eedf[b] / (tot * s->bin_w) : 0.0;
    eedf[s->p.eedf_bins] = tot > 0 ? s->eedf[s->p.eedf_bins] / tot : 0.0;
    return ns;
}

/* raw EEDF counts (bins + overflow) */
void orc_get_eedf_counts(const orc_sim *s, double *out)
{
    memcpy(out, s->eedf, sizeof(double) * (s->p.eedf_bins + 1));
}

/* counters: step, particles, births_iz, births_see0, births_see1, losses0,
 * losses1, elastic, excitation, ionization, null, clamps, status,
 * recombinations, Penning births, pooling births */
void orc_get_counters(const orc_sim *s, int64_t out[16])
{
    out[0] = s->step;
    out[1] = s->np;
    out[2] = s->births_iz;
    out[3] = s->births_see[0];
    out[4] = s->births_see[1];
    out[5] = s->losses[0];
    out[6] = s->losses[1];
    out[7] = s->coll[0];
    out[8] = s->coll[1];
    out[9] = s->coll[2];
    out[10] = s->coll[3];
    out[11] = s->n_clamp;
    out[12] = s->status;
    out[13] = s->recomb;
    out[14] = s->births_pen;
    out[15] = s->births_pool;
}

/* metastables: the density now, its time average, and the wall fluxes of the
 * last step */
void orc_get_metastables(const orc_sim *s, double *met, double *avg, double flux[2])
{
    for (int j = 0; j < s->G; ++j) {
        met[j] = s->met ? s->met[j] : 0.0;
        avg[j] = (s->met && s->n_samples) ? s->acc_met[j] / s->n_samples : 0.0;
    }
    flux[0] = s->flux_met[0];
    flux[1] = s->flux_met[1];
}

void orc_set_metastables(orc_sim *s, const double *met)
{
    if (s->met) memcpy(s->met, met, sizeof(double) * s->G);
}

void orc_get_flux_in(const orc_sim *s, double out[2])
{
    out[0] = s->flux_in[0];
    out[1] = s->flux_in[1];
}

void orc_set_flux_in(orc_sim *s, const double in[2])
{
    s->flux_in[0] = in[0];
    s->flux_in[1] = in[1];
}

/* Emit the secondaries of step `n` alone (for the emission-statistics pin). */
int64_t orc_emit_only(orc_sim *s, uint32_t n)
{
    int64_t before = s->np;
    emit_secondaries(s, n);
    return s->np - before;
}

/* ------------------------------------------------------------------------
 * Auxiliary ion-swarm Monte Carlo (Sec. II.C).  One ion species is followed
 * in a prescribed constant field E0 (along z) in a homogeneous, periodic
 * domain, so positions play no part; collisions with the neutral gas at T_N
 * are sampled by the null-collision method and scatter isotropically in the
 * centre-of-mass frame on Q_m = Q_i + 2 Q_b (the Phelps prescription the
 * paper adopts).  The He+/He cross sections are the ones quoted with
 * Tables 2/3: Q_i = 7.63e-20 / sqrt(eps), Q_b = 1e-19 / [(eps/1000)^0.15
 * (1 + eps/1000)^0.25 (1 + 5/eps)^0.15] m^2, eps = M_r g^2 / 2 in eV with g the
 * relative speed.  The ensemble's mean velocity after the relaxation window is
 * the drift u; the mobility is u/E0 and Eq. 2.6 gives the momentum-exchange
 * frequency nu = e/(M mu).  xs_model 1 keeps Q_i only: then N Q g does not
 * depend on g (a Maxwell-molecule gas), which gives a closed form to test
 * against.
 */
typedef struct orc_swarm_params {
    double gas_mass_amu, ion_mass_amu, pressure_pa, gas_temp_k, ion_temp0_k;
    double dt_s, e_field, nu_max, eps_max_ev;
    int64_t n_ions, n_steps, n_relax, id_base;
    int32_t xs_model;
    uint64_t seed;
} orc_swarm_params;

typedef struct orc_swarm_result {
    double drift, mean_energy_ev, mobility, nu_exchange, nu_max, p_max;
    int64_t candidates, collisions, overruns;
} orc_swarm_result;

/* Q_i and Q_b of the He+/He fits, eps > 0 in eV */
double orc_swarm_qi(double eps) { return 7.63e-20 / sqrt(eps); }
double orc_swarm_qb(double eps)
{
    return 1e-19 / (pow(eps / 1000.0, 0.15) * pow(1.0 + eps / 1000.0, 0.25) * pow(1.0 + 5.0 / eps, 0.15));
}

/* collision frequency N Q_m(eps(g)) g at relative speed g */
double orc_swarm_nu(double ngas, double m_red, int xs_model, double g)
{
    if (!(g > 0.0)) {  /* the g -> 0 limits: Q_i g finite, Q_b g -> 0 */
        return ngas * 7.63e-20 * sqrt(2.0 * Q_E / m_red);
    }
    double eps = 0.5 * m_red * g * g / Q_E;
    double q = orc_swarm_qi(eps);
    if (xs_model == 0) q += 2.0 * orc_swarm_qb(eps);
    return ngas * q * g;
}

/* the bound nu_max: the largest N Q_m g over relative energies up to eps_max
 * (a dense logarithmic grid, then a relative margin of 1e-6) */
double orc_swarm_nu_bound(double ngas, double m_red, int xs_model, double eps_max)
{
    double best = 0.0;
    const int n = 200000;
    for (int i = 0; i <= n; ++i) {
        double eps = 1e-8 * pow(eps_max / 1e-8, (double)i / n);
        double g = sqrt(2.0 * Q_E * eps / m_red);
        double v = orc_swarm_nu(ngas, m_red, xs_model, g);
        if (v > best) best = v;
    }
    return best * (1.0 + 1e-6);
}

static void swarm_draws(const orc_swarm_params *p, uint64_t id, uint32_t step, uint32_t call, double u[4])
{
    uint32_t ctr[4] = {step, (uint32_t)id, call, (uint32_t)(id >> 32)};
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    for (int i = 0; i < 4; ++i) u[i] = orc_u01(r[i]);
}

/* One run at one field value.  Ion i (id id_base + i) starts from a
 * Maxwellian at T_i0 drawn at step 0xFFFFFFFF; each step n: v_z += (e E0/M) dt,
 * then R1 < P_max makes it a candidate, a neutral velocity is drawn from the
 * Maxwellian at T_N, and R2 nu_max < N Q_m(eps) g makes the collision real.
 * The velocities of every ion after the last step go to v_out (3 per ion, may
 * be NULL). */
void orc_swarm_run(const orc_swarm_params *p, orc_swarm_result *res, double *v_out)
{
    const double mg = p->gas_mass_amu > 0 ? p->gas_mass_amu : 4.002602;
    const double M = (p->ion_mass_amu > 0 ? p->ion_mass_amu : mg) * AMU;
    const double mn = mg * AMU;
    const double m_red = M * mn / (M + mn);
    const double ngas = p->pressure_pa / (K_B * p->gas_temp_k);
    const double nu_max = p->nu_max > 0 ? p->nu_max
                                        : orc_swarm_nu_bound(ngas, m_red, p->xs_model,
                                                             p->eps_max_ev > 0 ? p->eps_max_ev : 100.0);
    const double p_max = -expm1(-nu_max * p->dt_s);
    const double acc = Q_E * p->e_field / M * p->dt_s;
    const double vt0 = sqrt(K_B * p->ion_temp0_k / M);
    const double vtn = sqrt(K_B * p->gas_temp_k / mn);
    double sum_vz = 0.0, sum_en = 0.0;
    int64_t cand = 0, coll = 0, over = 0;
    for (int64_t i = 0; i < p->n_ions; ++i) {
        const uint64_t id = (uint64_t)(p->id_base + i);
        double u[4], w[4], g1, g2, g3, g4;
        swarm_draws(p, id, 0xFFFFFFFFu, 0, u);
        gauss2(u[0], u[1], &g1, &g2);
        gauss2(u[2], u[3], &g3, &g4);
        double v[3] = {vt0 * g1, vt0 * g2, vt0 * g3};
        for (int64_t n = 0; n < p->n_steps; ++n) {
            v[2] += acc;
            swarm_draws(p, id, (uint32_t)n, 0, u);
            if (u[0] < p_max) {
                ++cand;
                swarm_draws(p, id, (uint32_t)n, 1, w);
                double a1, a2, a3, a4;
                gauss2(u[2], u[3], &a1, &a2);
                gauss2(w[0], w[1], &a3, &a4);
                const double V[3] = {vtn * a1, vtn * a2, vtn * a3};
                const double gv[3] = {v[0] - V[0], v[1] - V[1], v[2] - V[2]};
                const double g = sqrt(gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2]);
                const double nu = orc_swarm_nu(ngas, m_red, p->xs_model, g);
                if (nu > nu_max) ++over;
                if (u[1] * nu_max < nu) {
                    ++coll;
                    double d[3];
                    iso_dir(w[2], w[3], d);
                    for (int k = 0; k < 3; ++k) {
                        const double vc = (M * v[k] + mn * V[k]) / (M + mn);
                        v[k] = vc + mn / (M + mn) * g * d[k];
                    }
                }
            }
            if (n >= p->n_relax) {
                sum_vz += v[2];
                sum_en += 0.5 * M * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / Q_E;
            }
        }
        if (v_out) {
            v_out[3 * i] = v[0];
            v_out[3 * i + 1] = v[1];
            v_out[3 * i + 2] = v[2];
        }
    }
    const double ns = (double)p->n_ions * (double)(p->n_steps - p->n_relax);
    res->drift = ns > 0 ? sum_vz / ns : 0.0;
    res->mean_energy_ev = ns > 0 ? sum_en / ns : 0.0;
    res->mobility = p->e_field != 0.0 ? res->drift / p->e_field : 0.0;
    res->nu_exchange = res->mobility != 0.0 ? Q_E / (M * res->mobility) : 0.0;
    res->nu_max = nu_max;
    res->p_max = p_max;
    res->candidates = cand;
    res->collisions = coll;
    res->overruns = over;
}

/* power control state: the current amplitude, the last period's absorbed
 * power, the finished periods and the steps per period */
void orc_get_power(const orc_sim *s, double out[2], int64_t iout[2])
{
    out[0] = s->u_rf;
    out[1] = s->pw_last;
    iout[0] = s->pw_periods;
    iout[1] = s->pw_steps;
}

/* kinetic ions: number, losses at z = 0 and z = L, candidates, real collisions */
void orc_get_ion_counters(const orc_sim *s, int64_t out[5])
{
    out[0] = s->nip;
    out[1] = s->ion_losses[0];
    out[2] = s->ion_losses[1];
    out[3] = s->ion_cand;
    out[4] = s->ion_coll;
}

static int ion_by_id(const void *a, const void *b)
{
    uint64_t x = ((const part *)a)->id, y = ((const part *)b)->id;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* the ions, sorted by id */
void orc_get_ions(orc_sim *s, double *z, double *vx, double *vy, double *vz, uint64_t *id)
{
    part *t = (part *)malloc(sizeof(part) * (size_t)(s->nip ? s->nip : 1));
    memcpy(t, s->ip, sizeof(part) * (size_t)s->nip);
    qsort(t, (size_t)s->nip, sizeof(part), ion_by_id);
    for (int64_t i = 0; i < s->nip; ++i) {
        z[i] = t[i].z;
        vx[i] = t[i].vx;
        vy[i] = t[i].vy;
        vz[i] = t[i].vz;
        id[i] = t[i].id;
    }
    free(t);
}

