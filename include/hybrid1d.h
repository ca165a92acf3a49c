/*
 * hybrid1d.h -- C ABI of the GB300 kinetic-electron PIC/MCC library.
 *
 * The library advances the electron part of the 1D hybrid scheme of Eremin,
 * Hemke and Mussenbrock (arXiv 1508.02892) on one GPU: electron
 * macroparticles (Sec. II.A, Eqs. 1.1-1.2) pushed by leapfrog in the
 * CIC-interpolated field, removed at the walls, CIC-deposited, and collided
 * with the background gas by the modified null-collision method; impact
 * ionization births and gamma secondary emission (Sec. II.D); coupled every
 * step to the ion fluid (drift-diffusion, Eqs. 2.5-2.8, or the full model,
 * Eqs. 2.3-2.4) and to the Poisson equation (Sec. II.D).
 *
 * Units are SI unless a name says otherwise (_ev, _amu, _td).  The geometry is
 * planar: quantities are per unit electrode area (S = 1 m^2 in Eq. 1.2), so
 * the macroparticle weight is in m^-2 and fluxes in m^-2 s^-1.
 *
 * Conventions for every call:
 *   - returns HYB_OK (0), a positive warning, or a negative HYB_ERR_*; on an
 *     error hyb_last_error() gives a thread-local message;
 *   - pointers marked "host" are read or written by the call before it
 *     returns and stay owned by the caller; the library owns all device
 *     memory it allocates and frees it in the matching destroy call;
 *   - a handle is not thread-safe; distinct handles are independent;
 *   - device work is enqueued on the stream given at creation (NULL: the
 *     library creates its own); advance calls return before the GPU is done,
 *     read/sync calls wait for it.
 */
#ifndef HYBRID1D_H
#define HYBRID1D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define HYB_OK 0
#define HYB_WARN_DT_NULLCOLL 1  /* nu_max*dt > 0.1: coarser than the time-step rule of Sec. II.A */
#define HYB_WARN_NU_MAX 2       /* ion swarm: a collision frequency exceeded nu_max (result biased) */
#define HYB_ERR_ARG (-1)        /* invalid argument or parameter */
#define HYB_ERR_OOM (-2)        /* device memory, or the batch's HBM cap, exhausted */
#define HYB_ERR_CAPACITY (-3)   /* particle store full: births were dropped */
#define HYB_ERR_NONFINITE (-4)  /* NaN/Inf in an input table or in the fields */
#define HYB_ERR_TIMEOUT (-5)    /* a bounded device wait gave up */
#define HYB_ERR_CUDA (-6)       /* a CUDA runtime call failed */
#define HYB_ERR_UNSTABLE (-7)   /* the ion-fluid update left its stability range */
#define HYB_ERR_STATE (-8)      /* call not valid in the handle's current state */

/* ---------------------------------------------------------------- choices */
#define HYB_GAS_HE 0            /* background gas mass 4.002602 u */
#define HYB_GAS_AR 1            /* background gas mass 39.948 u */

#define HYB_ION_DD_CONST 0      /* drift-diffusion, constant mobility, T_i = T_gas (Eqs. 2.5-2.7) */
#define HYB_ION_DD_TABLE 1      /* drift-diffusion, mu(E) table, T_i from Eq. 2.8 */
#define HYB_ION_FULL 2          /* momentum equation with inertia, Eq. 2.3, nu(u) table */
#define HYB_ION_KINETIC 3       /* ions as macroparticles (the paper's fully kinetic comparison model):
                                   He+ with the electrons' weight, pushed in E every step, removed at
                                   the walls, colliding with the gas as in the auxiliary Monte Carlo of
                                   Sec. II.C (Q_m = Q_i + 2 Q_b, thermal target); one new ion per
                                   ionization, at the new electron's position; the ions take the
                                   precision of the discharge (FP64 or split); not combined with
                                   recombination or metastables (HYB_ERR_ARG) */

#define HYB_FP64 0              /* particles and grids in FP64 */
#define HYB_FP32_SPLIT 1        /* particles as (cell, FP32 offset) + FP32 velocity; FP64 grids */

#define HYB_MAX_CELLS 4000      /* largest grid a discharge may have */
#define HYB_MAX_INSTANCES 256   /* largest batch */

/* Problem statement of one discharge (Secs. II and III).  Copied at creation;
 * the table pointers are host pointers read during the call. */
typedef struct hyb_params {
    double gap_m;               /* electrode distance L; powered electrode at z = 0 */
    int32_t n_cells;            /* uniform grid, n_cells + 1 nodes, 2..HYB_MAX_CELLS */
    int32_t gas;                /* HYB_GAS_* */
    double pressure_pa;         /* background gas, uniform and frozen (Sec. II.A) */
    double gas_temp_k;
    double v_rf_amp_v;          /* phi(0, t) = v_dc_v + v_rf_amp_v sin(2 pi f_rf_hz t), phi(L) = 0 */
    double f_rf_hz;
    double v_dc_v;
    double dt_s;                /* time step shared by electrons and ions */
    int64_t n_particles;        /* initial electron macroparticles */
    double n0_m3;               /* initial uniform electron and ion density */
    double te0_ev;              /* initial Maxwellian temperature of the electrons */
    double weight;              /* real electrons per m^2 per macroparticle; 0: n0 L / n_particles (Eq. 1.2, S = 1) */
    double gamma_see;           /* ion-induced secondary emission coefficient (Sec. II.D) */
    double see_energy_ev;       /* energy of an emitted secondary; 0: 1 eV */
    int32_t ion_model;          /* HYB_ION_* */
    double ion_mass_amu;        /* 0: the gas mass */
    double gas_mass_amu;        /* 0: set by `gas` */
    double mu_const;            /* mobility for HYB_ION_DD_CONST, m^2/(V s) */
    const double *tab_eon_td;   /* host, n_tab increasing E/N values (Td) */
    const double *tab_mu;       /* host, n_tab mobilities at tab_eon_td */
    const double *tab_nu;       /* host, n_tab exchange frequencies at u = mu E (Sec. II.C) */
    int32_t n_tab;              /* 0 allowed for HYB_ION_DD_CONST */
    const double *xs_ev;        /* host, n_xs log-spaced energies (eV) */
    const double *xs_el;        /* host, elastic cross section (m^2) at xs_ev */
    const double *xs_exc;       /* host, excitation cross section */
    const double *xs_ion;       /* host, ionization cross section */
    int32_t n_xs;               /* >= 2; at most 4096 in HYB_FP32_SPLIT (staged in shared memory) */
    double e_exc_ev;            /* excitation threshold / energy loss */
    double e_iz_ev;             /* ionization threshold / energy loss */
    uint64_t seed;              /* Philox key: a particle's draws are the blocks at
                                   counter (step, id_lo, call, id_hi) under key
                                   (seed_lo, seed_hi) */
    int32_t eedf_bins;          /* 0: 256 */
    double eedf_max_ev;         /* 0: 64 eV */
    int32_t precision;          /* HYB_FP64 or HYB_FP32_SPLIT */
    double capacity_factor;     /* particle store = factor * n_particles (min 4096); 0: 2 */
    int32_t sort_interval;      /* steps between cell sorts; 0: library default */
    double power_w_m2;          /* prescribed absorbed power P0 per m^2 of electrode (Eq. 2.9); 0: fixed amplitude */
    double power_alpha;         /* alpha of Eq. 2.9: after each RF period U <- U (1 - alpha (P_abs - P0)/P0) */
    const double *xs_rec;       /* host, NULL or the electron-ion recombination cross section (m^2) at
                                   xs_ev: a null-collision process of its own on the ion density
                                   (Sec. II.D); a recombined electron is removed and its ion leaves
                                   n_i through the source term of Eq. 2.4 */
    /* Metastables and the ionization they cause (Sec. II.D).  With metastables = 1
     * every excitation event adds N_p/sp/dV to a metastable density n_m (CIC at
     * the electron).  Per step, from n_m at the start of the step, each interior
     * node j yields Delta N_e / N_p/sp new electrons (integer part plus a
     * Bernoulli draw on the fraction), with Delta N_e = R_P n_m n_N dt dz for
     * Penning ionization and R_pool n_m^2 dt dz for pooling.  They are placed
     * uniformly in [z_j - dz/2, z_j + dz/2), isotropic, at the process's
     * energy, and their ions enter the ion source.  Then
     *   n_m <- n_m + dt (D n_m'' + S_m - R_P n_N n_m - 2 R_pool n_m^2),
     * with n_m = 0 at the electrodes.  The metastables reaching the walls emit
     * secondaries with gamma_met.  Fluid ion models only; D dt/dz^2 <= 1/2. */
    int32_t metastables;        /* 0: off, 1: on */
    double met_diff_m2s;        /* D of the metastables, m^2/s */
    double met_n0_m3;           /* initial n_m at the interior nodes */
    double penning_rate_m3s;    /* R_P, Penning ionization of the admixture */
    double penning_target_m3;   /* n_N, density of the admixture */
    double penning_energy_ev;   /* energy of a Penning electron (E_* - E_I) */
    double pooling_rate_m3s;    /* R_pool, two metastables -> ion + electron */
    double pooling_energy_ev;   /* energy of a pooling electron */
    double gamma_met;           /* secondary yield of a metastable striking an electrode */
} hyb_params;

/* Time averages since creation or the last hyb_reset_moments (Sec. III
 * diagnostics).  Caller-owned host buffers: n_nodes = n_cells + 1 entries for
 * the profiles, eedf_bins + 1 for the EEDF (last entry = fraction above
 * eedf_max_ev; the others are normalised so that sum f dE + last = 1).  Any
 * pointer may be NULL to skip that quantity. */
typedef struct hyb_moments {
    double *ne;                 /* electron density, m^-3 */
    double *ni;                 /* ion density, m^-3 */
    double *gamma_i;            /* ion flux, m^-2 s^-1 */
    double *mean_energy_ev;     /* CIC-weighted mean electron energy per node */
    double *eedf;               /* eV^-1 */
    int64_t n_samples;          /* out: steps averaged */
} hyb_moments;

/* Instantaneous grids after the last completed step; host buffers of n_nodes
 * doubles, any may be NULL. */
typedef struct hyb_fields {
    double *ne, *ni, *gamma_i, *phi, *efield, *ion_source;
} hyb_fields;

/* Integer bookkeeping since creation. */
typedef struct hyb_counters {
    int64_t step;
    int64_t particles;          /* live macroparticles */
    int64_t births_ionization;
    int64_t births_see[2];      /* gamma secondaries at z = 0 and z = L */
    int64_t losses[2];          /* absorbed at z = 0 and z = L */
    int64_t collisions[4];      /* elastic, excitation, ionization, null (candidates without a real collision) */
    int64_t clamps;             /* ion densities clamped at zero */
    int64_t pushes;             /* particle pushes done (particle-steps) */
    uint32_t status;            /* bit set of HYB_STATUS_* below */
    double v_rf_amp_v;          /* current RF amplitude (changes under power control) */
    double power_last_w_m2;     /* absorbed power per m^2 of the last finished RF period (Eq. 2.9):
                                   mean over round(1/(f dt)) steps of V J, V at mid-step, J the total
                                   current density along +z at the driven electrode (ions, electrons
                                   absorbed and emitted there, displacement) */
    int64_t power_periods;      /* finished RF periods */
    int64_t recombinations;     /* electrons removed by electron-ion recombination */
    int64_t ions;               /* kinetic ions: live ion macroparticles (0 for the fluid models) */
    int64_t ion_losses[2];      /* kinetic ions removed at z = 0 and z = L */
    int64_t ion_collisions;     /* real ion-neutral collisions of the kinetic ions */
    int64_t births_penning;     /* electrons born by Penning ionization */
    int64_t births_pooling;     /* electrons born by metastable pooling */
    int64_t ion_pushes;         /* kinetic ions: ion-steps advanced (pushes), for throughput */
} hyb_counters;

#define HYB_STATUS_CAPACITY 1u
#define HYB_STATUS_NONFINITE 2u
#define HYB_STATUS_UNSTABLE 4u
#define HYB_STATUS_EMIT_CAP 8u

/* Derived constants of a discharge. */
typedef struct hyb_info {
    int32_t n_nodes, eedf_bins;
    double weight, gas_density, nu_max, p_max, dz;
    int64_t capacity;
    int64_t device_bytes;
} hyb_info;

typedef struct hyb_discharge hyb_discharge;
typedef struct hyb_batch hyb_batch;

/* ----------------------------------------------------- single discharge */

/* Create a discharge: validate, derive the constants of Secs. II.A-II.D
 * (gas density p/(k_B T), weight of Eq. 1.2, nu_max over the table nodes,
 * P_max = 1 - exp(-nu_max dt)), load n_particles electrons (uniform positions,
 * Maxwellian at te0_ev, drawn from Philox at step 0xFFFFFFFF), deposit them
 * and solve the initial field.  `stream` is a cudaStream_t or NULL.  Returns
 * HYB_WARN_DT_NULLCOLL (handle valid) when nu_max dt > 0.1. */
int hyb_create_discharge(const hyb_params *p, void *stream, hyb_discharge **out);

/* Enqueue n_steps full steps (push, wall removal, deposit, MCC and births;
 * ion fluid; Poisson; moments; secondaries for the next step). */
int hyb_advance(hyb_discharge *h, int64_t n_steps);

/* Wait for the enqueued work; returns the first error the device flagged. */
int hyb_sync(hyb_discharge *h);

int hyb_read_moments(hyb_discharge *h, hyb_moments *out);
int hyb_read_fields(hyb_discharge *h, hyb_fields *out);
int hyb_read_counters(hyb_discharge *h, hyb_counters *out);
int hyb_get_info(hyb_discharge *h, hyb_info *out);
int hyb_reset_moments(hyb_discharge *h);

/* Copy the live particles, sorted by id, into host arrays of `cap` entries
 * (position z in m, velocity in m/s, FP64 whatever the precision); *n gets
 * the live count (HYB_ERR_ARG if it exceeds cap). */
int hyb_read_particles(hyb_discharge *h, double *z, double *vx, double *vy, double *vz, uint64_t *id,
                       int64_t cap, int64_t *n);

/* Replace the whole particle set (including secondaries already born for the
 * next step) with n host particles and re-solve the field for the current
 * time.  Positions must lie in [0, L). */
int hyb_write_particles(hyb_discharge *h, int64_t n, const double *z, const double *vx, const double *vy,
                        const double *vz, const uint64_t *id);

/* Kinetic ions (HYB_ION_KINETIC): the live ions sorted by id into host arrays
 * of cap entries (any may be NULL), *n their number; HYB_ERR_STATE for the
 * fluid ion models, HYB_ERR_ARG if they do not fit. */
int hyb_read_ions(hyb_discharge *h, double *z, double *vx, double *vy, double *vz, uint64_t *id, int64_t cap,
                  int64_t *n);

/* Metastables (metastables = 1): host buffers of n_nodes values for the density
 * after the last step and its time average (either may be NULL), and flux[2],
 * the metastables that reached z = 0 and z = L per m^2 and s in the last step
 * (may be NULL).  HYB_ERR_STATE without metastables. */
int hyb_read_metastables(hyb_discharge *h, double *met, double *avg, double *flux);

/* Overwrite the metastable density (host, n_nodes values; the electrode nodes
 * must be 0).  HYB_ERR_STATE without metastables, HYB_ERR_ARG for negative or
 * non-finite values or a non-zero electrode node. */
int hyb_write_metastables(hyb_discharge *h, const double *met);

/* Overwrite the ion density (host, n_nodes values) and re-solve the field
 * (fluid ion models; HYB_ERR_STATE for kinetic ions). */
int hyb_write_ion_density(hyb_discharge *h, const double *ni);

int hyb_destroy(hyb_discharge *h);

/* ------------------------------------------------ batches and serving */

/* A batch advances up to max_instances independent discharges of one
 * precision in lockstep launches (one electron kernel over all instances'
 * particles, one field block per instance).  hbm_cap_bytes bounds the device
 * memory of admitted instances (0: no cap). */
int hyb_batch_create(int32_t max_instances, int32_t precision, int64_t hbm_cap_bytes, void *stream,
                     hyb_batch **out);

/* Device bytes an instance with these parameters would hold. */
int hyb_footprint(const hyb_params *p, int64_t *bytes);

/* Admit a discharge into a free slot; it runs for n_steps steps of later
 * hyb_batch_advance calls (n_steps <= 0: until evicted) and then stops by
 * itself.  HYB_ERR_OOM when the cap or the slots are exhausted. */
int hyb_batch_admit(hyb_batch *b, const hyb_params *p, int64_t n_steps, int32_t *slot);

/* Enqueue n_steps steps of every running instance. */
int hyb_batch_advance(hyb_batch *b, int64_t n_steps);

/* Wait, then report in done[0..*n_done) the slots that reached their step
 * count since the last poll (cap entries at most). */
int hyb_batch_poll(hyb_batch *b, int32_t *done, int32_t cap, int32_t *n_done);

/* Serving without host waits on the batch's stream.  hyb_batch_snapshot
 * queues, in stream order after the work queued so far, a copy of every
 * slot's status and counters to pinned host memory (at most 3 not yet
 * polled).  hyb_batch_poll_snapshot waits for the oldest such snapshot only
 * (not for work queued after it) and reports, like hyb_batch_poll, the slots
 * that had finished or failed by then (a slot admitted after a snapshot was
 * queued is not in it).  hyb_batch_read_finished gives such a slot's counters
 * from that snapshot and its time-averaged moments, read on a side stream
 * beside whatever the batch's stream runs meanwhile (a finished slot is idle
 * on the GPU); either output may be NULL; the slot is then evicted as usual.
 * Admission and eviction queue their copies and kernels without waiting for
 * the stream, so a request loop can keep one chunk queued ahead of the one
 * whose results it reads.  Errors: HYB_ERR_STATE (no snapshot, too many
 * queued, slot not reported or still running), HYB_ERR_ARG, HYB_ERR_CUDA, and
 * the slot's own error code (HYB_ERR_CAPACITY, HYB_ERR_NONFINITE,
 * HYB_ERR_UNSTABLE) when it failed. */
int hyb_batch_snapshot(hyb_batch *b);
/* Waits at most timeout_s seconds (host clock) for the work queued on the
 * batch's stream: HYB_OK when it has finished, HYB_ERR_TIMEOUT when the limit
 * passed first (the work goes on; the caller may wait again or give up on the
 * batch).  It polls the stream, so no call of this library blocks a request
 * loop longer than the loop allows.  Errors: HYB_ERR_ARG, HYB_ERR_CUDA. */
int hyb_batch_wait(hyb_batch *b, double timeout_s);
int hyb_batch_poll_snapshot(hyb_batch *b, int32_t *done, int32_t cap, int32_t *n_done);
int hyb_batch_read_finished(hyb_batch *b, int32_t slot, hyb_counters *counters, hyb_moments *moments);

/* Moments of running discharges without a host wait on the batch's stream.
 * hyb_batch_snapshot_moments queues, in stream order after the work queued so
 * far, a copy of every taken slot's time sums (n_e, n_i, Gamma_i, the
 * electron-weighted energy), EEDF counts and sample count: one packing kernel
 * and one device-to-host copy into pinned memory owned by the batch (two
 * snapshots are kept in turn; queueing a third waits for the copies of the
 * first, long done in a chunked loop).  hyb_batch_read_snapshot_moments fills
 * `out` (the layout of hyb_read_moments) for `slot` from the snapshot queued
 * last, waiting for that snapshot's copy only, not for the work queued after
 * it; so a loop can queue chunk n + 1 and then read chunk n's moments while
 * the GPU runs.  Errors: HYB_ERR_ARG; HYB_ERR_STATE when no snapshot was queued,
 * the slot was empty then, or it has been evicted or re-admitted since;
 * HYB_ERR_CUDA. */
int hyb_batch_snapshot_moments(hyb_batch *b);
int hyb_batch_read_snapshot_moments(hyb_batch *b, int32_t slot, hyb_moments *out);

/* Per-slot reads (wait for the GPU first). */
int hyb_batch_read_moments(hyb_batch *b, int32_t slot, hyb_moments *out);
int hyb_batch_read_counters(hyb_batch *b, int32_t slot, hyb_counters *out);
int hyb_batch_read_particles(hyb_batch *b, int32_t slot, double *z, double *vx, double *vy, double *vz,
                             uint64_t *id, int64_t cap, int64_t *n);
/* The same reads for the discharge in `slot` as hyb_read_metastables and
 * hyb_read_ions (same buffers, layout and errors; HYB_ERR_ARG for an empty
 * slot). */
int hyb_batch_read_metastables(hyb_batch *b, int32_t slot, double *met, double *avg, double *flux);
int hyb_batch_read_ions(hyb_batch *b, int32_t slot, double *z, double *vx, double *vy, double *vz, uint64_t *id,
                        int64_t cap, int64_t *n);

/* Free a slot and its memory (waits for the GPU). */
int hyb_batch_evict(hyb_batch *b, int32_t slot);

/* Running slots, live particles over them, device bytes held. */
int hyb_batch_stats(hyb_batch *b, int32_t *running, int64_t *particles, int64_t *bytes);

int hyb_batch_destroy(hyb_batch *b);

/* Launch accounting and per-kernel device time.  With profiling on, every
 * kernel of a step (also inside the captured graphs) is bracketed by CUDA
 * events on the batch's stream and hyb_batch_advance waits for each chunk to
 * read them; times are summed until read. */
typedef struct hyb_profile {
    int64_t kernel_launches;    /* kernels enqueued since creation */
    int64_t steps;              /* lockstep steps enqueued */
    double ms_electron, ms_field, ms_sort; /* summed device time of the timed launches */
    int64_t n_electron, n_field, n_sort;   /* timed launches */
    double ms_ion;              /* kinetic ions: summed device time of the per-step ion kernels */
    int64_t n_ion;              /* timed ion steps */
} hyb_profile;

int hyb_batch_set_profiling(hyb_batch *b, int32_t on);
int hyb_batch_profile(hyb_batch *b, hyb_profile *out, int32_t reset);

/* Launch configuration of a batch.  It decides how the work is laid out on
 * the GPU, not what is computed (beyond the order of floating-point sums):
 *   lanes          the slots are split into this many contiguous groups, each
 *                  advanced by its own chain of launches; inside a captured
 *                  chunk the chains run as parallel graph branches, so the
 *                  field kernels of one group overlap the electron kernels of
 *                  the others (1..16 and at most max_instances; a batch starts
 *                  with min(4, max_instances));
 *   sort_interval  steps between cell sorts (1..1000, default 20);
 *   blocks_per_sm  electron-kernel blocks per SM (0: the occupancy limit);
 *   field_threads  threads of each CTA of an instance's field step: 256, 512
 *                  or 1024 (default 256);
 *   field_cluster  CTAs (a thread-block cluster) over which each instance's
 *                  field step is split: 1..16; 0 (default) picks about one
 *                  computed node (a CTA's run of the grid and 10 halo nodes
 *                  on each side) per half warp for the batch's largest grid
 *                  (at most 8 CTAs when the batch has several lanes), as
 *                  many as let every instance's cluster be resident at once;
 *   electron_threads  threads of an electron-kernel block in split mode: 128,
 *                  256 or 512 (0 or 256: default); the FP64 path and the
 *                  variants with reactions or ion births keep 256;
 *   particles_per_thread  consecutive particles each electron thread takes in
 *                  split mode: 2 or 4 (0 or 2: default); the same variants
 *                  keep 2.
 * rate is filled by hyb_batch_autotune with the particle-steps/s it measured
 * for the returned choice, and is ignored by hyb_batch_set_tuning. */
typedef struct hyb_tuning {
    int32_t lanes;
    int32_t sort_interval;
    int32_t blocks_per_sm;
    int32_t field_threads;
    int32_t field_cluster;
    int32_t electron_threads;
    int32_t particles_per_thread;
    double rate;
} hyb_tuning;

int hyb_batch_get_tuning(hyb_batch *b, hyb_tuning *out);
/* Waits for the GPU; the next chunk re-captures its graph. */
int hyb_batch_set_tuning(hyb_batch *b, const hyb_tuning *t);

/* Time candidate configurations on the batch's own running discharges and
 * keep the fastest: lanes in {1, 2, 4, 8, 16}, then the sort interval in
 * {10, 20, 50, 100}, then the electron grid at the occupancy limit or twice it,
 * then the field block size in {256, 512, 1024}, then the field cluster in
 * {automatic, 1, 2, 4, 8, 16}, then (split mode, no reaction or ion-birth
 * variant) the electron block size in {128, 256, 512} with the particles per
 * thread in {2, 4}, then the lanes again; finally the three fastest layouts
 * once more over twice the trial length, the fastest of those kept.  Each
 * trial advances every running discharge by one untimed chunk and then by
 * trial_steps rounded up to whole chunks (100 steps): those are real steps of
 * the runs.  Profiling must be off.  *chosen may be NULL. */
int hyb_batch_autotune(hyb_batch *b, int32_t trial_steps, hyb_tuning *chosen);

/* The batch behind a single discharge (for profiling and statistics). */
hyb_batch *hyb_discharge_batch(hyb_discharge *h);

/* Test hook: split = 1 makes the field step of an FP64 batch take the split
 * mode's arithmetic (reciprocals of the instance constants, table slopes,
 * Newton reciprocals), everything else staying FP64, so that the rounding of
 * that arithmetic can be measured against the FP64 mode alone; split = 0
 * restores the batch's own.  A split-mode batch always takes it.  Waits for
 * the GPU; the next chunk re-captures its graph.  Errors: HYB_ERR_ARG. */
int hyb_batch_set_field_arith(hyb_batch *b, int32_t split);

/* First failed device index guard since load: out[0] = guard site (0:
 * none), out[1] = index, out[2] = bound, for the electron, sort and load
 * kernels; out[3..5] the same for the field kernel.  A failed guard skips the
 * access it protects, so a nonzero site means results are not to be trusted. */
int hyb_debug_checks(uint64_t out[6]);

/* ------------------------------------------------ auxiliary ion swarm
 *
 * The auxiliary Monte Carlo of Sec. II.C that gives the ion mobility and the
 * momentum-exchange frequency of the fluid model: ions of one species move in
 * a prescribed constant field E0 (along z) through a homogeneous, periodic
 * domain and collide with the neutral gas at T_N by the null-collision method
 * (a neutral velocity drawn from the Maxwellian at T_N for every candidate,
 * acceptance R2 nu_max < N Q_m(eps) g), scattering isotropically in the
 * centre-of-mass frame on Q_m = Q_i + 2 Q_b.  The cross sections are the
 * He+/He fits quoted with Tables 2/3: Q_i = 7.63e-20/sqrt(eps),
 * Q_b = 1e-19/[(eps/1000)^0.15 (1+eps/1000)^0.25 (1+5/eps)^0.15] m^2, with eps
 * = M_r g^2/2 in eV and g the relative speed.  HYB_SWARM_QI_ONLY keeps Q_i
 * alone (N Q g independent of g: a Maxwell-molecule gas).  The drift u is the
 * ensemble mean of v_z over steps n_relax..n_steps-1; mobility = u/E0 and, by
 * Eq. 2.6, nu = e/(M mobility).
 *
 * Random numbers: Philox4x32-10 under key (seed_lo, seed_hi) at counter
 * (step, id_lo, call, id_hi) for the ion id (ion i of field f has id
 * f*n_ions + i): call 0 = (R1, R2,
 * two Box-Muller uniforms), call 1 = (two Box-Muller uniforms, the scattering
 * direction cos and phi); the initial Maxwellian at T_i0 is drawn at step
 * 0xFFFFFFFF. */
#define HYB_SWARM_QM 0       /* Q_m = Q_i + 2 Q_b (the paper's prescription) */
#define HYB_SWARM_QI_ONLY 1  /* Q_i only: constant collision frequency */

typedef struct hyb_swarm_params {
    double gas_mass_amu;   /* 0: helium, 4.002602 */
    double ion_mass_amu;   /* 0: the gas mass */
    double pressure_pa, gas_temp_k;
    double ion_temp0_k;    /* initial Maxwellian of the ions */
    double dt_s;
    double nu_max;         /* null-collision bound, s^-1 (0: the largest N Q_m g up to eps_max_ev) */
    double eps_max_ev;     /* relative energy covered by the computed bound (0: 100 eV) */
    int64_t n_ions;        /* ions per field value */
    int64_t n_steps;       /* steps per run (< 2^32) */
    int64_t n_relax;       /* steps before the averaging window */
    int32_t xs_model;      /* HYB_SWARM_QM or HYB_SWARM_QI_ONLY */
    int32_t precision;     /* HYB_FP64 (FP64 velocities and arithmetic) or HYB_FP32_SPLIT (FP32) */
    uint64_t seed;
} hyb_swarm_params;

typedef struct hyb_swarm_result {
    double e_field;        /* V/m, as given */
    double drift;          /* m/s: mean v_z over the window */
    double mean_energy_ev; /* mean kinetic energy over the window */
    double mobility;       /* drift / e_field (0 at zero field) */
    double nu_exchange;    /* e / (M mobility), Eq. 2.6 (0 at zero field) */
    double nu_max, p_max;  /* the bound used and 1 - exp(-nu_max dt) */
    int64_t candidates, collisions, overruns; /* overruns: candidates with N Q_m g > nu_max */
} hyb_swarm_result;

/* Run the swarm at n_fields field values (host array, V/m) at once; out[f]
 * (host, n_fields entries) receives the results.  v_out: NULL, or a device
 * array of 3*n_ions*n_fields doubles that receives every ion's final
 * velocity (ion i of field f at 3*(f*n_ions + i)).  Allocates and frees its
 * own small device scratch; synchronous on `stream`.  Returns
 * HYB_WARN_NU_MAX (> 0, results filled) when some candidate's collision
 * frequency exceeded nu_max. */
int hyb_swarm_run(const hyb_swarm_params *p, int32_t n_fields, const double *e_field, hyb_swarm_result *out,
                  double *v_out, void *stream);

/* Transport tables for the ion fluid (the tab_eon_td / tab_mu / tab_nu of
 * hyb_params) from swarm runs at E = (E/N) N for the n increasing E/N values
 * (Td, host); at E/N = 0 the table takes the values of the lowest positive
 * point.  tab_mu, tab_nu: host arrays of n values. */
int hyb_swarm_tables(const hyb_swarm_params *p, int32_t n, const double *eon_td, double *tab_mu, double *tab_nu,
                     void *stream);

/* The field of a particle set, computed without allocating device memory.
 * The paper has no counterpart: this is a service for callers that cannot
 * call cudaMalloc, such as applications that reserve all device memory up
 * front and hand out fixed buffers, or that must not let an allocation
 * synchronise the device under other work.  It does what hyb_write_particles
 * followed by hyb_read_fields does for a discharge of these parameters: CIC
 * charge assignment of the n electrons at positions z, electron density, and
 * the Poisson solve with the ion density ni and the drive at time t
 * (phi(0) = v_dc_v + v_rf_amp_v sin(2 pi f_rf_hz t), phi(L) = 0).  Uses
 * gap_m, n_cells, weight (or n0_m3, n_particles) and the drive of p; the rest
 * of p is ignored, power_w_m2 and power_alpha included: for a power-controlled
 * discharge (Eq. 2.9) pass its current amplitude (hyb_counters.v_rf) in
 * v_rf_amp_v.
 *   z:      device, n positions (m), FP64; positions outside [0, L) and
 *           non-finite ones add no charge, z within rounding below L lands on
 *           the last node
 *   ni:     device, n_cells + 1 ion densities (m^-3)
 *   ne, phi, efield: device outputs, n_cells + 1 doubles each
 *   stream: cudaStream_t or NULL; the call returns before the GPU is done.
 * The node sums go to one file-scope device array of HYB_MAX_CELLS + 1 doubles
 * (32 KB, held by every GPU that loads the library until the process exits);
 * n_cells above HYB_MAX_CELLS is rejected with HYB_ERR_ARG.  The first call on
 * a device looks up that array's device address and sets a kernel attribute
 * for the device's current context, so make that first call before any
 * stream capture, and do not use the call across a cudaDeviceReset of that
 * device in the same process.  Every call clears the array and then uses it:
 * calls whose GPU work overlaps (other streams, other threads) race. */
int hyb_field_from_particles_noalloc(const hyb_params *p, int64_t n, const double *z, const double *ni, double t,
                                     double *ne, double *phi, double *efield, void *stream);

/* Thread-local message of the last error. */
const char *hyb_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HYBRID1D_H */
