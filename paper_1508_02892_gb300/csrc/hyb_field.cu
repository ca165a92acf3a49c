// hyb_field.cu -- the per-instance FP64 grid step of each step (arXiv
// 1508.02892, Secs. II.B-II.D): electron density from the CIC sums, the ion
// fluid update (drift-diffusion, Eqs. 2.5-2.8, or the full model, Eq. 2.3,
// then continuity, Eq. 2.4), the Poisson solve and field, the time sums, and
// the gamma secondaries that will take part in the next step.
//
// Each instance's grid is split over a thread-block cluster of up to 16 CTAs
// (one GPU): CTA r of the cluster owns a contiguous run of nodes and keeps it,
// with one halo node on each side, in shared memory (8 node arrays).  The FP64
// work of a step (about a hundred FP64 instructions per node at this part's
// FP64 rate of two FMA per cycle per SM) is so spread over several SMs.
//   * Each CTA keeps kHalo + 1 nodes beyond its run on each side, loaded from
//     global memory (the inputs of the step), and computes the drift-diffusion
//     fluxes and the Jacobi sweeps of the full model on that wider range
//     itself: a sweep spoils one node per side, so up to kHalo - 1 sweeps need
//     no exchange between CTAs at all.  Above that the remaining sweeps pass
//     the edge values into the neighbours' shared memory (distributed shared
//     memory) with a cluster barrier each.
//   * Block scans and maxima combine the CTAs' totals through distributed
//     shared memory; every CTA combines them in the same order, so all of
//     them hold the same bits.
//   * Poisson: the constant-coefficient tridiagonal system is solved in closed
//     form: phi = linear part + discrete double integral of the charge, the
//     running sum S and the running sum of S formed by one associative scan
//     instead of the serial Thomas recursion.
//   * Full-model flux: the tridiagonal system of Eq. 2.3 is diagonally
//     dominant with ratio r = max (|a|+|c|)/b (a Courant number); it is solved
//     by Jacobi sweeps, ceil(ln 2^-60 / ln r) of them, which bounds the error
//     by 2^-60 of the initial one.  r >= 1/2 is reported as unstable.
//   * The instance constants are formed on the host; the drive sin(2 pi f t)
//     by one thread beside the others' work.
// All transport coefficients (mu, T_i, D, nu) and both solves are FP64 in
// both precision modes; the split mode multiplies by reciprocals of the
// instance constants where the FP64 mode divides as a plain program would.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <utility>

#include "hyb_internal.cuh"

namespace cg = cooperative_groups;

namespace hyb {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kArrays = 8;
constexpr int kMaxCluster = 16;  // non-portable cluster size (a GB300 GPC holds 19 SMs)
constexpr int kSlots = 16;    // reductions across the cluster per step (at most 8 are used)
constexpr int kMaxTab = 256;  // rows of a transport table staged in shared memory
constexpr size_t kMaxDynSmem = 160 * 1024;  // node arrays of one CTA, at most
constexpr int kHalo = 10;     // nodes computed beyond a CTA's run on each side (plus one input node)

struct Red {
    double w[32], wx[32];            // warp totals and their block prefixes
    double p[3][32], px[3][32];      // the same for the Poisson pair scan
    double before, all;              // cluster offset and total of the last reduction
    double cpre[3], ctot[3];         // cluster prefix and total of the pair scan
    double phi0, v_old;              // drive at the end and at the start of the step
    double gN;                       // Gamma_i at z = L, written by the CTA that owns node G - 1 (into rank 0's copy)
    double E0;                       // E at z = 0 after the step (rank 0)
    int flag;
    unsigned long long count;
};

// What rank 0's bookkeeping at the end of the step reads of the descriptor,
// loaded at the start of the step beside the other CTAs' work: all of it is
// written only by that bookkeeping (previous steps), by earlier kernels or by
// the host before the launch.  The metastable fluxes and the slot count, which
// the metastable step of this launch may change, are read again after it.
struct Book {
    int64_t step, n_samples, pw_count, pw_steps, pw_periods, capacity, target_step;
    unsigned long long n_slots, see0, see1, loss0, pw_loss0, ion_l0, ion_l1, ion_prev0, ion_prev1;
    double gamma_see, gamma_met, flux_met0, flux_met1, pw_acc, pw_target, pw_alpha, v_rf, see_speed, L;
    uint32_t seed_lo, seed_hi;
    int precision, n_cells, met_on;
    PartBuf P;
};


// This CTA's place in its instance's cluster.  Ranks 0..nown-1 own nodes
// [rank P, min(G, (rank + 1) P)); higher ranks own none and only take part in
// the barriers.
struct Clu {
    int rank, size, nown, P, c0, c1;
};

__device__ __forceinline__ void cl_sync() { cg::this_cluster().sync(); }
// Wait until the kernel this launch programmatically depends on (the step's
// particle kernel, when the launch allows an early start) has finished and its
// writes are visible; returns at once otherwise
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// the two halves of a cluster barrier, for work between them
__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ T *cl_remote(T *p, int rank)
{
    return cg::this_cluster().map_shared_rank(p, (unsigned)rank);
}

// Cluster-wide exclusive scan (or max, MAX = true) of one double per thread:
// the block result is published in this CTA's slot, and after the cluster
// barrier the first warp reads every CTA's slot and combines them with the
// same butterfly in every CTA.  Slots are used once per launch, so no CTA can
// overwrite a slot another one is still reading.  Two block barriers and one
// cluster barrier.
template <bool MAX>
__device__ double cl_reduce(double v, Red &r, const Clu &cu, double *slots, int &ph, double *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        if (MAX) {
            x = fmax(x, __shfl_xor_sync(kFull, x, d));
        } else {
            const double y = __shfl_up_sync(kFull, x, d);
            if (lane >= d) x += y;
        }
    }
    if (lane == 31) r.w[wid] = x;
    __syncthreads();
    const int s = ph++;
    if (wid == 0) {
        double y = lane < nw ? r.w[lane] : 0.0;
        if (MAX) {
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) y = fmax(y, __shfl_xor_sync(kFull, y, d));
            if (lane == 0) slots[s] = y;
        } else {
            double inc = y;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const double z = __shfl_up_sync(kFull, inc, d);
                if (lane >= d) inc += z;
            }
            r.wx[lane] = inc - y;
            if (lane == 31) slots[s] = inc;
        }
    }
    cl_sync();
    if (wid == 0) {
        const int q = lane;
        double c = q < cu.size ? *cl_remote(&slots[s], q) : 0.0;
        double cb = q < cu.rank ? c : 0.0;
#pragma unroll
        for (int d = 16; d; d >>= 1) {
            if (MAX) {
                c = fmax(c, __shfl_xor_sync(kFull, c, d));
            } else {
                c += __shfl_xor_sync(kFull, c, d);
                cb += __shfl_xor_sync(kFull, cb, d);
            }
        }
        if (lane == 0) {
            r.before = cb;
            r.all = c;
        }
    }
    __syncthreads();
    if (total) *total = r.all;
    return MAX ? r.all : r.wx[wid] + (x - v) + r.before;
}

// Element of the Poisson scan over a run of nodes: the sum of the sources s,
// the sum over the run of the running sums of s, and the node count.  Runs
// combine associatively: (a then b) = (s_a + s_b, t_a + t_b + m_b s_a, m_a + m_b).
struct Pair {
    double s, t, m;
};

__device__ __forceinline__ Pair pcomb(const Pair &a, const Pair &b) { return Pair{a.s + b.s, a.t + b.t + b.m * a.s, a.m + b.m}; }

__device__ __forceinline__ Pair pshfl_up(const Pair &x, int d)
{
    return Pair{__shfl_up_sync(kFull, x.s, d), __shfl_up_sync(kFull, x.t, d), __shfl_up_sync(kFull, x.m, d)};
}

__device__ __forceinline__ Pair pshfl(const Pair &x, int src)
{
    return Pair{__shfl_sync(kFull, x.s, src), __shfl_sync(kFull, x.t, src), __shfl_sync(kFull, x.m, src)};
}

// Exclusive scan of one Pair per thread over the instance's nodes (threads in
// order within a CTA, CTAs in rank order); *tot gets the total.  Uses three
// slots; two block barriers and one cluster barrier.
__device__ Pair pair_scan(Pair v, Red &r, const Clu &cu, double *slots, int &ph, Pair *tot)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const Pair zero{0.0, 0.0, 0.0};
    Pair x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const Pair y = pshfl_up(x, d);
        if (lane >= d) x = pcomb(y, x);
    }
    Pair xe = pshfl_up(x, 1);
    if (lane == 0) xe = zero;
    if (lane == 31) {
        r.p[0][wid] = x.s;
        r.p[1][wid] = x.t;
        r.p[2][wid] = x.m;
    }
    __syncthreads();
    const int s = ph;
    ph += 3;
    if (wid == 0) {
        Pair y = lane < nw ? Pair{r.p[0][lane], r.p[1][lane], r.p[2][lane]} : zero;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const Pair z = pshfl_up(y, d);
            if (lane >= d) y = pcomb(z, y);
        }
        Pair ye = pshfl_up(y, 1);
        if (lane == 0) ye = zero;
        r.px[0][lane] = ye.s;
        r.px[1][lane] = ye.t;
        r.px[2][lane] = ye.m;
        if (lane == 31) {
            slots[s] = y.s;
            slots[s + 1] = y.t;
            slots[s + 2] = y.m;
        }
    }
    cl_sync();
    if (wid == 0) {
        const int q = lane;
        Pair c = q < cu.size ? Pair{*cl_remote(&slots[s], q), *cl_remote(&slots[s + 1], q), *cl_remote(&slots[s + 2], q)}
                             : zero;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const Pair z = pshfl_up(c, d);
            if (lane >= d) c = pcomb(z, c);
        }
        Pair ce = pshfl_up(c, 1);
        if (lane == 0) ce = zero;
        const Pair pre = pshfl(ce, cu.rank), all = pshfl(c, 31);
        if (lane == 0) {
            r.cpre[0] = pre.s, r.cpre[1] = pre.t, r.cpre[2] = pre.m;
            r.ctot[0] = all.s, r.ctot[1] = all.t, r.ctot[2] = all.m;
        }
    }
    __syncthreads();
    *tot = Pair{r.ctot[0], r.ctot[1], r.ctot[2]};
    return pcomb(Pair{r.cpre[0], r.cpre[1], r.cpre[2]}, pcomb(Pair{r.px[0][wid], r.px[1][wid], r.px[2][wid]}, xe));
}

// Jacobi sweeps for a contraction ratio r: ceil(ln 2^-60 / ln r), 1..64 (the
// same in every thread and CTA: the same r and instructions)
__device__ __forceinline__ int sweeps_for(double r)
{
    const float lr = logf(fminf((float)r, 0.999f));
    const int it = (int)ceilf(-41.58883f / lr);
    return it < 1 ? 1 : (it > 64 ? 64 : it);
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
    const double *tab;  // shared-memory copy of the instance's table
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

// Split mode: the same coefficients in FP64 with fewer FP64 instructions (this
// part issues FP64 at two FMA per cycle per SM): the table comes with the
// slope of every segment (kTabCols columns: E/N, mu, d mu/d(E/N), u, nu,
// d nu/du, formed at admission), so a lookup is the search and one FMA, and
// reciprocals start from the FP32 reciprocal with two Newton steps.  Values
// differ from the FP64 mode's by rounding only.

__device__ __forceinline__ double lookup_slope(const double *tab, const float *xf, int n, int cx, int cy, int cs,
                                              double v)
{
    if (v <= tab[cx]) return tab[cy];
    if (v >= tab[kTabCols * (n - 1) + cx]) return tab[kTabCols * (n - 1) + cy];
    // bracket on the FP32 copy of the abscissa, then exact FP64 checks against
    // the neighbouring nodes, so that x_lo <= v < x_lo+1 in FP64
    const float vf = (float)v;
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (xf[mid] <= vf)
            lo = mid;
        else
            hi = mid;
    }
    while (lo > 0 && v < tab[kTabCols * lo + cx]) --lo;
    while (lo < n - 2 && v >= tab[kTabCols * (lo + 1) + cx]) ++lo;
    return tab[kTabCols * lo + cy] + (v - tab[kTabCols * lo + cx]) * tab[kTabCols * lo + cs];
}

// 1/x for a normal positive x in the FP32 range: FP32 reciprocal, then two
// Newton steps r <- r (2 - x r), each squaring the relative error
__device__ __forceinline__ double rcp_nr(double x)
{
    double r = (double)(1.0f / (float)x);
    r = r * (2.0 - x * r);
    r = r * (2.0 - x * r);
    return r;
}

struct FluidFast {
    int model, n_tab;
    const double *tab;  // kTabCols columns
    const float *xf;    // FP32 copies of the E/N column, then of the u column
    double mu_const, kT, tfac, inv_ngas_td;

    __device__ double mobility(double e_abs) const
    {
        if (model == HYB_ION_DD_CONST) return mu_const;
        return lookup_slope(tab, xf, n_tab, 0, 1, 2, e_abs * inv_ngas_td);
    }
    __device__ double temp(double mu, double e_abs) const
    {
        if (model == HYB_ION_DD_CONST) return kT;
        const double ud = mu * e_abs;
        return kT + tfac * ud * ud;
    }
    __device__ double exch(double u_abs) const { return lookup_slope(tab, xf + kMaxTab, n_tab, 3, 4, 5, u_abs); }
    __device__ double wall(int w, double n, double E) const
    {
        const bool into = w == 0 ? (E < 0.0) : (E > 0.0);
        if (!into) return 0.0;
        return mobility(fabs(E)) * n * E;
    }
};

// Stage an instance's table in shared memory: {E/N, mu, nu, u} as it is (FP64
// mode), or the split-mode layout with the segment slopes and the FP32
// abscissae (16-byte copies).  Read after the next block barrier.
template <bool FAST>
__device__ void stage_table(const InstDev *K, int n, double *s_tab, float *s_tabf)
{
    if constexpr (!FAST) {
        const double *tab = K->tab;
        for (int j = threadIdx.x; j < 4 * n; j += blockDim.x) s_tab[j] = tab[j];
    } else {
        const double2 *src = reinterpret_cast<const double2 *>(K->tabx);
        const float *srcf = K->tabf;
        double2 *dst = reinterpret_cast<double2 *>(s_tab);
        for (int j = threadIdx.x; j < kTabCols / 2 * n; j += blockDim.x) dst[j] = src[j];
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            s_tabf[k] = srcf[k];
            s_tabf[kMaxTab + k] = srcf[n + k];
        }
    }
}

__device__ __forceinline__ double node_volume(int j, int G, double dz) { return (j == 0 || j == G - 1) ? 0.5 * dz : dz; }

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

// old, cnt0, cnt1: node arrays (global node index) used as scratch: n_m at the
// start of the step on the loaded range [L0, L1), the per-node Penning and
// pooling counts of the thread's run [j0, j1).  The split mode multiplies by
// reciprocals where the FP64 mode divides as the oracle does.
template <bool FAST>
__device__ void metastable_step(InstDev *K, double *old, double *cnt0, double *cnt1, Red &red, const Clu &cu,
                                double *slots, int &ph, int j0, int j1, int L0, int L1)
{
    const int G = K->G;
    const int T = blockDim.x, t = threadIdx.x;
    const double dz = K->dz, dt = K->dt, w = K->w;
    const uint32_t n = (uint32_t)K->step;
    const double kp = K->met_kp, kq = K->met_kq;
    const double inv_w = w > 0.0 ? 1.0 / w : 0.0;
    __shared__ unsigned long long s_base;
    __shared__ int64_t s_tot[2];
    // the slot base, read by rank 0 before its update below and by the other
    // ranks from rank 0's shared memory after the cluster barriers
    if (t == 0 && cu.rank == 0) s_base = K->n_slots;
    // n_m at the start of the step (the neighbours write theirs only after
    // the cluster barriers below)
    for (int j = L0 + t; j < L1; j += T) old[j] = K->met[j];
    __syncthreads();
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
    const double off0 = cl_reduce<false>(part[0], red, cu, slots, ph, &tot[0]);
    const double off1 = cl_reduce<false>(part[1], red, cu, slots, ph, &tot[1]);
    const int64_t cap = (1 << 20) - 1;
    if (t == 0) {
        s_tot[0] = (int64_t)tot[0] < cap ? (int64_t)tot[0] : cap;
        s_tot[1] = (int64_t)tot[1] < cap ? (int64_t)tot[1] : cap;
        if (cu.rank == 0) {
            if ((int64_t)tot[0] > cap || (int64_t)tot[1] > cap) atomicOr(&K->status, (unsigned)HYB_STATUS_EMIT_CAP);
            K->n_slots = s_base + (unsigned long long)(s_tot[0] + s_tot[1]);
            K->ctr[C_PEN] += (unsigned long long)s_tot[0];
            K->ctr[C_POOL] += (unsigned long long)s_tot[1];
        } else {
            s_base = *cl_remote(&s_base, 0);
        }
    }
    __syncthreads();
    const int64_t mine[2] = {(int64_t)off0, (int64_t)off1};
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
                const double ph2 = kTwoPi * u01d(v.z);
                const double vx = sp * st * cos(ph2), vy = sp * st * sin(ph2), vz = sp * ct;
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
        // the flux into each wall, by the thread that owns the wall node
        if (j == 0) K->flux_met[0] = D * old[1] / dz + w * K->s_met[0] / dt;
        if (j == G - 1) K->flux_met[1] = D * old[G - 2] / dz + w * K->s_met[G - 1] / dt;
    }
    if (clamps) atomicAdd(&red.count, clamps);
    __syncthreads();
    for (int j = j0; j < j1; ++j) K->s_met[j] = 0.0;
}

template <bool FAST>
__device__ void field_body(InstDev *K, double *sm, int lw, Red &red, const double *s_tab, const float *s_tabf,
                           const Clu &cu, double *slots)
{
    const int G = K->G;
    const int T = blockDim.x;
    const int t = threadIdx.x;
    const int c0 = cu.c0, c1 = cu.c1;
    const bool own = c1 > c0;
    // the thread's contiguous run of the CTA's nodes (for the scans)
    const int pt = own ? (c1 - c0 + T - 1) / T : 0;
    const int j0 = min(c0 + t * pt, c1), j1 = min(j0 + pt, c1);
    // nodes loaded from global memory, and the wider range computed here
    const int L0 = own ? max(0, c0 - kHalo - 1) : c0, L1 = own ? min(G, c1 + kHalo + 1) : c0;
    const int e0 = own ? max(0, c0 - kHalo) : c0, e1 = own ? min(G, c1 + kHalo) : c0;
    const FieldK &fk = K->fk;
    const double dz = K->dz, dt = K->dt, w = K->w;
    const bool init = K->init_pending != 0;
    const bool kin = K->ion_model == HYB_ION_KINETIC;
    int ph = 0;

    // node arrays: base pointers (local index 0 = node c0 - kHalo - 1) and
    // views indexed by the global node number
    double *b_ni = sm, *b_E = sm + lw, *b_g = sm + 2 * lw, *b_A = sm + 3 * lw;
    double *b_ib = sm + 4 * lw, *b_d = sm + 5 * lw, *b_x = sm + 6 * lw, *b_cp = sm + 7 * lw;
    const int sh = kHalo + 1 - c0;
    double *s_ni = b_ni + sh, *s_E = b_E + sh, *s_g = b_g + sh, *s_A = b_A + sh;
    double *s_ib = b_ib + sh, *s_d = b_d + sh, *s_x = b_x + sh, *s_cp = b_cp + sh;

    // the drive at the end of the step (and at its start, for the absorbed
    // power), by the last thread beside the others' work
    __shared__ Book bk;
    if (t == T - 1) {
        red.flag = 0;
        red.count = 0ull;
        red.phi0 = K->v_dc + K->v_rf * sin(kTwoPi * K->f_rf * ((double)(K->step + (init ? 0 : 1)) * dt));
        red.v_old = (cu.rank == 0 && !init) ? K->v_dc + K->v_rf * sin(kTwoPi * K->f_rf * ((double)K->step * dt)) : 0.0;
    }
    // inputs of the step (every write of these globals comes after at least
    // one cluster barrier)
    if (!kin) {
        for (int j = L0 + t; j < L1; j += T) {
            s_ni[j] = K->ni[j];
            s_E[j] = K->E[j];
            s_g[j] = K->gam[j];
        }
    } else {
        for (int j = c0 + t; j < c1; j += T) s_E[j] = K->E[j];
    }
    // everything above comes from the previous field step or the host; the
    // electron sums, counters and slot counts below from this step's particle
    // kernel, which a launch allowed to start early (one lane) waits for here
    grid_dep_wait();
    if (t == T - 2 && cu.rank == 0 && !init) {
        bk.step = K->step;
        bk.n_samples = K->n_samples;
        bk.pw_count = K->pw_count;
        bk.pw_steps = K->pw_steps;
        bk.pw_periods = K->pw_periods;
        bk.capacity = K->capacity;
        bk.target_step = K->target_step;
        bk.n_slots = K->n_slots;
        bk.see0 = K->ctr[C_SEE0];
        bk.see1 = K->ctr[C_SEE1];
        bk.loss0 = K->ctr[C_LOSS0];
        bk.pw_loss0 = K->pw_loss0;
        if (kin) {
            const InstDev *I = K->ion;
            bk.ion_l0 = I->ctr[C_LOSS0];
            bk.ion_l1 = I->ctr[C_LOSS1];
            bk.ion_prev0 = K->ion_loss_prev[0];
            bk.ion_prev1 = K->ion_loss_prev[1];
        }
        bk.gamma_see = K->gamma_see;
        bk.gamma_met = K->gamma_met;
        bk.flux_met0 = K->flux_met[0];
        bk.flux_met1 = K->flux_met[1];
        bk.pw_acc = K->pw_acc;
        bk.pw_target = K->pw_target;
        bk.pw_alpha = K->pw_alpha;
        bk.v_rf = K->v_rf;
        bk.see_speed = K->see_speed;
        bk.L = K->L;
        bk.seed_lo = K->seed_lo;
        bk.seed_hi = K->seed_hi;
        bk.precision = K->precision;
        bk.n_cells = K->n_cells;
        bk.met_on = K->met_on;
        bk.P = K->buf[K->cur];
    }
    __syncthreads();

    if (K->met_on && !init) {
        metastable_step<FAST>(K, s_d, s_x, s_ib, red, cu, slots, ph, j0, j1, L0, L1);
        // the metastables' ionization adds to the ion source also at the
        // neighbouring CTAs' edge nodes, which read it in the continuity pass:
        // a cluster barrier orders those additions before (the drift-diffusion
        // path has none of its own in between)
        cl_sync();
    }

    const Fluid F{K->ion_model, K->n_tab, s_tab, K->mu_const, K->ngas, K->kT_gas, K->m_ion, K->m_gas};
    const FluidFast FF{K->ion_model, K->n_tab, s_tab, s_tabf, K->mu_const, K->kT_gas, fk.tfac, fk.inv_ngas_td};
    double *gfin = s_g;
    if (kin) {
        // kinetic ions: n_i and Gamma_i from the ions' charge assignment of this
        // step (at initialisation, of the loaded ions)
        for (int j = c0 + t; j < c1; j += T) {
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
    if (!init && !kin) {
        // ---------------------------------------------------------- ion fluid
        if (K->ion_model == HYB_ION_FULL) {
            // Eq. 2.3: nu at u^n = Gamma^{n-1/2}/n^n, advection semi-implicit;
            // A = Gamma/n and n T on the loaded range
            for (int j = L0 + t; j < L1; j += T) {
                const double nj = s_ni[j];
                const double ea = fabs(s_E[j]);
                if (FAST) {
                    s_A[j] = nj >= K->n_floor ? s_g[j] * rcp_nr(nj) : 0.0;
                    s_x[j] = nj * FF.temp(FF.mobility(ea), ea);
                } else {
                    s_A[j] = nj >= K->n_floor ? s_g[j] / nj : 0.0;
                    s_x[j] = nj * F.temp(F.mobility(ea), ea);
                }
            }
            __syncthreads();
            const double h = fk.h;
            double rmax = 0.0;
            for (int j = e0 + t; j < e1; j += T) {
                if (j == 0 || j == G - 1) continue;
                double q;
                if (FAST) {
                    // the row divided by its diagonal: Y_j = dd_j + cm_j X_{j-1} - cp_j X_{j+1}
                    const double nu = FF.exch(fabs(s_A[j]));
                    const double ib = rcp_nr(1.0 + nu * fk.hdt);
                    const double d = s_g[j] * (1.0 - nu * fk.hdt) + fk.qdt_m * s_ni[j] * s_E[j] -
                                     fk.h_m * (s_x[j + 1] - s_x[j - 1]);
                    const double cm = h * s_A[j - 1] * ib, cp = h * s_A[j + 1] * ib;
                    s_d[j] = d * ib;
                    s_ib[j] = cm;
                    s_cp[j] = cp;
                    q = fabs(cm) + fabs(cp);
                } else {
                    const double nu = F.exch(fabs(s_A[j]));
                    const double b = 1.0 + nu * dt / 2.0;
                    s_d[j] = s_g[j] * (1.0 - nu * dt / 2.0) + kQe * s_ni[j] * s_E[j] * dt / K->m_ion -
                             fk.h_mion * (s_x[j + 1] - s_x[j - 1]);
                    s_ib[j] = 1.0 / b;
                    q = (fabs(h * s_A[j - 1]) + fabs(h * s_A[j + 1])) / b;
                }
                if (j >= c0 && j < c1) rmax = fmax(rmax, q);
            }
            const double r = cl_reduce<true>(rmax, red, cu, slots, ph, nullptr);
            // both sweep buffers start from Gamma^{n-1/2}, with the Dirichlet
            // wall rows (field-driven wall flux); the nodes at the ends of the
            // loaded range keep their value through the local sweeps
            for (int j = L0 + t; j < L1; j += T) {
                double v = s_g[j];
                if (j == 0 || j == G - 1) {
                    const int wl = j == 0 ? 0 : 1;
                    v = FAST ? FF.wall(wl, s_ni[j], s_E[j]) : F.wall(wl, s_ni[j], s_E[j]);
                }
                s_g[j] = v;
                s_x[j] = v;
            }
            if (t == 0 && cu.rank == 0 && r >= 0.5) atomicOr(&K->status, (unsigned)HYB_STATUS_UNSTABLE);
            const int iters = sweeps_for(r);
            const int nloc = min(iters, kHalo - 1);
            __syncthreads();
            double *X = s_g, *Y = s_x;
            double *bX = b_g, *bY = b_x;
            // local sweeps over the computed range: after k of them the k
            // nodes at each end are spoiled, the CTA's run and one node on
            // each side are exact
            for (int it = 0; it < iters; ++it) {
                const bool local = it < nloc;
                const int a = local ? e0 : c0, b = local ? e1 : c1;
                for (int j = a + t; j < b; j += T) {
                    if (j == 0 || j == G - 1) continue;
                    if (FAST)
                        Y[j] = s_d[j] + s_ib[j] * X[j - 1] - s_cp[j] * X[j + 1];
                    else
                        Y[j] = (s_d[j] + h * s_A[j - 1] * X[j - 1] - h * s_A[j + 1] * X[j + 1]) * s_ib[j];
                }
                if (local) {
                    __syncthreads();
                } else {
                    // beyond kHalo - 1 sweeps: the CTA's edge values go to the
                    // neighbours' halo nodes each sweep
                    __syncthreads();
                    if (t == 0 && own && cu.rank > 0) *cl_remote(&bY[cu.P + kHalo + 1], cu.rank - 1) = Y[c0];
                    if (t == 1 && own && cu.rank + 1 < cu.nown) *cl_remote(&bY[kHalo], cu.rank + 1) = Y[c1 - 1];
                    cl_sync();
                }
                double *tmp = X;
                X = Y;
                Y = tmp;
                tmp = bX;
                bX = bY;
                bY = tmp;
            }
            gfin = X;
        } else {
            // Eq. 2.5 at level n (explicit drift-diffusion), on the CTA's run
            // and one node beyond it on each side; the centred explicit scheme
            // holds while u^2 dt <= 2 D and D dt <= dz^2 / 2 (checked on the run)
            const int a = own ? max(0, c0 - 1) : c0, b = own ? min(G, c1 + 1) : c0;
            bool unstable = false;
            for (int j = a + t; j < b; j += T) {
                if (j == 0 || j == G - 1) {
                    const int wl = j == 0 ? 0 : 1;
                    s_x[j] = FAST ? FF.wall(wl, s_ni[j], s_E[j]) : F.wall(wl, s_ni[j], s_E[j]);
                    continue;
                }
                const double ea = fabs(s_E[j]);
                double mu, D;
                if (FAST) {
                    mu = FF.mobility(ea);
                    D = mu * FF.temp(mu, ea) * fk.inv_qe;
                    s_x[j] = mu * s_ni[j] * s_E[j] - D * ((s_ni[j + 1] - s_ni[j - 1]) * fk.inv2dz);
                } else {
                    mu = F.mobility(ea);
                    D = mu * F.temp(mu, ea) / kQe;
                    s_x[j] = mu * s_ni[j] * s_E[j] - D * (s_ni[j + 1] - s_ni[j - 1]) / (2.0 * dz);
                }
                const double u = mu * ea;
                if (j >= c0 && j < c1 && (u * u * dt > 2.0 * D || D * dt > 0.5 * dz * dz)) unstable = true;
            }
            if (unstable) atomicOr(&K->status, (unsigned)HYB_STATUS_UNSTABLE);
            __syncthreads();
            gfin = s_x;
        }
        // ------------------------------------- continuity, Eq. 2.4 (G^n source)
        unsigned long long clamps = 0;
        for (int j = c0 + t; j < c1; j += T) {
            const bool wall = j == 0 || j == G - 1;
            const double gs = FAST ? K->s_iz[j] * (wall ? fk.gs_wall : fk.gs_in)
                                   : w * K->s_iz[j] / (node_volume(j, G, dz) * dt);
            double nn;
            if (j == 0)
                nn = s_ni[0] - (FAST ? fk.c_wall : fk.dt_dz) * (gfin[1] - gfin[0]) + dt * gs;
            else if (j == G - 1)
                nn = s_ni[G - 1] - (FAST ? fk.c_wall : fk.dt_dz) * (gfin[G - 1] - gfin[G - 2]) + dt * gs;
            else
                nn = s_ni[j] - (FAST ? fk.c_in : fk.dt_2dz) * (gfin[j + 1] - gfin[j - 1]) + dt * gs;
            if (nn < 0.0) {
                nn = 0.0;
                ++clamps;
            }
            s_ni[j] = nn;
            K->ni[j] = nn;
            K->gam[j] = gfin[j];
            if (j == G - 1) *cl_remote(&red.gN, 0) = gfin[j];
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
        for (int j = c0 + t; j < c1; j += T) m = fmax(m, s_ni[j]);
        const double nimax = cl_reduce<true>(m, red, cu, slots, ph, nullptr);
        if (t == 0 && cu.rank == 0) {
            K->rec_numax = nimax * K->rec_svmax;
            K->rec_pmax = -expm1(-K->rec_numax * dt);
            K->f_rec_pmax = (float)K->rec_pmax;
        }
        const double inv = nimax > 0.0 ? 1.0 / nimax : 0.0;
        for (int j = c0 + t; j < c1; j += T) K->nif[j] = (float)(s_ni[j] * inv);
    }

    // ------------------------------------------------------------- Poisson
    // -eps0 phi'' = e (n_i - n_e): with s_j = dz^2 rho_j / eps0 (interior),
    // S_j = sum_{k<=j} s_k and T_j = sum_{k<j} S_k,
    //   d_0 = (phi_N - phi_0 + T_{G-1})/(G-1),  d_j = d_0 - S_j,
    //   phi_j = phi_0 + j d_0 - T_j,  E from the d_j (Gauss at the walls)
    double *s_rho = s_A;
    double *s_s = s_ib;
    Pair mine{0.0, 0.0, (double)(j1 - j0)};
    {
        double loc = 0.0;
        for (int j = j0; j < j1; ++j) {
            const double ne = FAST ? K->dep_n[j] * ((j == 0 || j == G - 1) ? fk.w_wall : fk.w_in)
                                   : w * K->dep_n[j] / node_volume(j, G, dz);
            K->ne[j] = ne;
            const double rho = kQe * (s_ni[j] - ne);
            s_rho[j] = rho;
            const double sj = (j >= 1 && j <= G - 2) ? (FAST ? rho * fk.c_src : dz * dz * rho / kEps0) : 0.0;
            s_s[j] = sj;
            loc += sj;
            mine.t += loc;
            if (!init) {
                K->acc_ne[j] += ne;
                K->acc_wn[j] += K->dep_n[j];
                K->acc_we[j] += K->dep_e[j];
            }
            K->dep_n[j] = 0.0;
            K->dep_e[j] = 0.0;
            K->s_iz[j] = 0.0;
        }
        mine.s = loc;
    }
    Pair all;
    const Pair pre = pair_scan(mine, red, cu, slots, ph, &all);
    // this CTA reads no other CTA's shared memory from here on
    cl_arrive();
    const double phi0 = red.phi0;
    const double d0 = FAST ? (0.0 - phi0 + (all.t - all.s)) * K->inv_gm1 : (0.0 - phi0 + (all.t - all.s)) / (double)(G - 1);
    int bad = 0;
    double S = pre.s, Tx = pre.t;
    for (int j = j0; j < j1; ++j) {
        const double Sprev = S, Tj = Tx;
        S += s_s[j];
        Tx += S;
        double e;
        if (FAST) {
            if (j == 0)
                e = -d0 * fk.inv_dz - s_rho[0] * fk.c_gauss;
            else if (j == G - 1)
                e = -(d0 - Sprev) * fk.inv_dz + s_rho[G - 1] * fk.c_gauss;
            else
                e = -((d0 - S) + (d0 - Sprev)) * fk.half_inv_dz;
        } else if (j == 0) {
            e = -d0 / dz - s_rho[0] * dz / (2.0 * kEps0);
        } else if (j == G - 1) {
            e = -(d0 - Sprev) / dz + s_rho[G - 1] * dz / (2.0 * kEps0);
        } else {
            e = -((d0 - S) + (d0 - Sprev)) / (2.0 * dz);
        }
        K->E[j] = e;
        K->Ef[j] = (float)e;
        if (j == 0) red.E0 = e;
        K->phi[j] = j == G - 1 ? 0.0 : phi0 + (double)j * d0 - Tj;
        if (!isfinite(e) || !isfinite(s_ni[j])) bad = 1;
    }
    if (bad) red.flag = 1;
    __syncthreads();
    if (t == 0) {
        if (red.flag) atomicOr(&K->status, (unsigned)HYB_STATUS_NONFINITE);
        if (red.count && !init) atomicAdd(&K->ctr[C_CLAMP], red.count);
    }

    if (init) {
        if (t == 0 && cu.rank == 0) {
            K->n_slots_step = (int64_t)K->n_slots;
            K->init_pending = 0;
        }
        return;
    }
    // rank 0 finishes the step: the other CTAs' writes it reads (the wall
    // flux at z = L, the metastable flux there) came before the cluster
    // barrier of the Poisson scan
    if (cu.rank != 0) return;

    // ------------------------------------------- bookkeeping, gamma emission
    // (the descriptor's values from the prefetch bk, written back here).  The
    // two walls' emission counts and the displacement-current term run on
    // three warps side by side: this part issues FP64 at a low rate per SM
    // sub-partition, so one thread's dependent FP64 chain is slow.
    __shared__ int s_cnt[2];
    __shared__ unsigned long long s_base;
    __shared__ double s_disp;
    const int64_t step = bk.step + 1;
    const uint32_t n_step = (uint32_t)step;
    if ((t & 31) == 0 && t < 64) {
        // wall t / 32: flux of ions into it, then the electrons that ions and
        // metastables striking it emit (Sec. II.D)
        const int wall = t >> 5;
        double f_in;
        if (kin) {  // the ions removed at the wall this step
            const unsigned long long l = wall == 0 ? bk.ion_l0 : bk.ion_l1;
            f_in = (double)(l - (wall == 0 ? bk.ion_prev0 : bk.ion_prev1)) * w / dt;
            K->ion_loss_prev[wall] = l;
        } else {
            const double g = wall == 0 ? gfin[0] : red.gN;
            f_in = wall == 0 ? (g < 0.0 ? -g : 0.0) : (g > 0.0 ? g : 0.0);
        }
        K->flux_in[wall] = f_in;
        int cnt = 0;
        if ((bk.gamma_see > 0.0 || bk.gamma_met > 0.0) && w > 0.0) {
            const double f_met = bk.met_on ? K->flux_met[wall] : (wall == 0 ? bk.flux_met0 : bk.flux_met1);
            const double ns = (bk.gamma_see * f_in + bk.gamma_met * f_met) * dt / w;
            if (ns > 0.0) {
                const double k = floor(ns);
                const double frac = ns - k;
                const uint4 r = draw(0xFFFFFFFFFFFFFF00ull | (uint64_t)wall, n_step, bk.seed_lo, bk.seed_hi, 3);
                int64_t c = (int64_t)k + (u01d(r.x) < frac ? 1 : 0);
                if (c > (1 << 20) - 1) {
                    c = (1 << 20) - 1;
                    atomicOr(&K->status, (unsigned)HYB_STATUS_EMIT_CAP);
                }
                cnt = (int)c;
            }
        }
        s_cnt[wall] = cnt;
    } else if (t == 64) {
        s_disp = kEps0 * (red.E0 - s_E[0]) / dt;
    } else if (t == 96) {
        K->n_samples = bk.n_samples + 1;
        K->step = step;
    }
    __syncthreads();
    if (t == 0) {
        const unsigned long long base = bk.met_on ? K->n_slots : bk.n_slots;
        s_base = base;
        const unsigned long long tot = (unsigned long long)(s_cnt[0] + s_cnt[1]);
        K->n_slots = base + tot;
        K->ctr[C_SEE0] = bk.see0 + s_cnt[0];
        K->ctr[C_SEE1] = bk.see1 + s_cnt[1];
        // Absorbed power (Eq. 2.9): V J dt per step at the driven electrode, V at
        // mid-step, J along +z = ion flux + electrons absorbed (+) and emitted (-)
        // there + displacement current; at the end of an RF period P_abs and the
        // amplitude of the next period
        const unsigned long long l0 = bk.loss0;
        const int64_t d_loss0 = (int64_t)(l0 - bk.pw_loss0), d_see0 = s_cnt[0];
        K->pw_loss0 = l0;
        const double v_mid = 0.5 * (red.v_old + phi0);
        const double jz = kQe * gfin[0] + kQe * w * (double)(d_loss0 - d_see0) / dt + s_disp;
        const double acc = bk.pw_acc + v_mid * jz * dt;
        const int64_t cnt = bk.pw_count + 1;
        if (cnt == bk.pw_steps) {
            const double last = acc / ((double)bk.pw_steps * dt);
            K->pw_last = last;
            if (bk.pw_target > 0.0 && bk.pw_alpha > 0.0)
                K->v_rf = bk.v_rf * (1.0 - bk.pw_alpha * (last - bk.pw_target) / bk.pw_target);
            K->pw_acc = 0.0;
            K->pw_count = 0;
            K->pw_periods = bk.pw_periods + 1;
        } else {
            K->pw_acc = acc;
            K->pw_count = cnt;
        }
    }
    __syncthreads();
    const int ntot = s_cnt[0] + s_cnt[1];
    if (ntot) {
        const PartBuf P = bk.P;
        const uint32_t n = n_step;
        const double sp = bk.see_speed, L = bk.L;
        for (int k = t; k < ntot; k += T) {
            const int wall = k < s_cnt[0] ? 0 : 1;
            const uint32_t j = (uint32_t)(wall == 0 ? k : k - s_cnt[0]);
            const uint64_t id = see_id(wall, n, j);
            const uint4 r = draw(id, n, bk.seed_lo, bk.seed_hi, 7);
            const double ct = sqrt(u01d(r.x));
            const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
            const double phw = kTwoPi * u01d(r.y);
            const double vn = sp * ct;
            const double vx = sp * st * cos(phw), vy = sp * st * sin(phw);
            double vz, z;
            if (wall == 0) {
                vz = vn;
                z = u01d(r.z) * vn * dt;
            } else {
                vz = -vn;
                z = L - u01d(r.z) * vn * dt;
            }
            const unsigned long long slot = s_base + (unsigned long long)k;
            if (slot >= (unsigned long long)bk.capacity) {
                atomicOr(&K->status, (unsigned)HYB_STATUS_CAPACITY);
                continue;
            }
            P.id[slot] = id;
            if (bk.precision == HYB_FP32_SPLIT) {
                const double x = z / dz;
                const double f = floor(x);
                int c = (int)f;
                double o = x - f;
                if (c >= bk.n_cells) {
                    c = bk.n_cells - 1;
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
    if (t == 0) {
        unsigned long long ns = s_base + (unsigned long long)ntot;
        if (ns > (unsigned long long)bk.capacity) {
            atomicOr(&K->status, (unsigned)HYB_STATUS_CAPACITY);
            ns = (unsigned long long)bk.capacity;
            K->n_slots = ns;
        }
        K->n_slots_step = (int64_t)ns;
        if (bk.target_step > 0 && bk.step + 1 >= bk.target_step) K->active = 0;
    }
}


// grid (cluster size, instances); cluster (cluster size, 1, 1); lw = doubles
// of one node array (nodes per owning CTA + 2 kHalo + 2)
template <bool FAST, int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS == 256 ? 3 : 1) k_field(InstDev *insts, int n_max, int64_t *prefix, unsigned *ticket,
                                                   int max_nodes, int lw)
{
    extern __shared__ __align__(16) double sm[];
    __shared__ Red red;
    __shared__ double s_slots[kSlots];
    __shared__ __align__(16) double s_tab[kTabCols * kMaxTab];
    __shared__ float s_tabf[FAST ? 2 * kMaxTab : 1];
    InstDev *K = &insts[blockIdx.y];
    // the descriptor's fields read here, loaded together
    const int act = K->active, ini = K->init_pending, G = K->G, n_tab = K->n_tab;
    const bool run = (act | ini) != 0;
    // every CTA of the cluster takes the same branch (one instance per cluster)
    bool body = false;
    if (run && HYB_CHECK(G >= 3 && G <= max_nodes && n_tab <= kMaxTab, 20, G, max_nodes)) {
        Clu cu;
        cu.rank = (int)cg::this_cluster().block_rank();
        cu.size = (int)gridDim.x;
        // at least two nodes per owning CTA, and no more than the arrays hold
        int nown = min(cu.size, max(1, G / 2));
        int P = (G + nown - 1) / nown;
        nown = (G + P - 1) / P;
        cu.nown = nown;
        cu.P = P;
        cu.c0 = min(cu.rank * P, G);
        cu.c1 = cu.rank < nown ? min(cu.c0 + P, G) : cu.c0;
        if (HYB_CHECK(P + 2 * kHalo + 2 <= lw, 22, P, lw)) {
            stage_table<FAST>(K, n_tab, s_tab, s_tabf);
            field_body<FAST>(K, sm, lw, red, s_tab, s_tabf, cu, s_slots);
            body = true;
        }
    }
    // no CTA leaves while another may still read its shared memory: the body
    // arrived at the cluster barrier after its last read of another CTA's
    // shared memory; the other paths arrive here
    if (!body) cl_arrive();
    cl_wait();
    grid_dep_wait();  // a CTA without a body still writes the prefix below
    if (n_max == 1) {
        // one instance: the chunk prefix of the next step from what rank 0's
        // thread 0 itself wrote at the end of the step
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            prefix[0] = 0;
            prefix[1] = K->active ? chunks_of(K->n_slots_step) : 0;
        }
        return;
    }
    // the last block to finish computes the chunk prefix of the next step
    __shared__ bool s_last;
    __shared__ int64_t s_buf[HYB_MAX_INSTANCES];
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x * gridDim.y - 1;
        if (s_last) __threadfence();
    }
    __syncthreads();
    if (s_last) {
        block_chunk_prefix(insts, n_max, prefix, s_buf);
        if (threadIdx.x == 0) *ticket = 0u;
    }
}

// CTAs per instance's cluster for a launch: the nodes a CTA computes (its run
// and kHalo on each side) about one per half warp of its threads, so that with
// 256 threads each SM sub-partition's FP64 pipe serves one warp of nodes (the
// FP64 work of a CTA grows with its nodes at this part's FP64 rate); at most
// 16; 1 for small grids
int cluster_size(int max_nodes, int threads)
{
    const int per = threads / 2 - 2 * kHalo;
    const int c = (max_nodes + per - 1) / per;
    return c < 1 ? 1 : (c > kMaxCluster ? kMaxCluster : c);
}

int array_len(int max_nodes, int csize) { return (max_nodes + csize - 1) / csize + 2 * kHalo + 4; }

}  // namespace

size_t field_smem_bytes(int max_nodes, int threads)
{
    return (size_t)kArrays * 8 * (size_t)array_len(max_nodes, cluster_size(max_nodes, threads));
}

void read_checks_field(unsigned long long out[3])
{
    if (cudaMemcpyFromSymbol(out, g_hyb_check, sizeof(unsigned long long) * 3) != cudaSuccess)
        out[0] = out[1] = out[2] = 0ull;
}

namespace {
template <bool FAST, int THREADS>
void configure_one()
{
    cudaFuncSetAttribute(k_field<FAST, THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxDynSmem);
    cudaFuncSetAttribute(k_field<FAST, THREADS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}
}  // namespace

void configure_field_kernel()
{
    configure_one<false, 256>();
    configure_one<true, 256>();
    configure_one<false, 512>();
    configure_one<true, 512>();
    configure_one<false, 1024>();
    configure_one<true, 1024>();
}

namespace {

template <bool FAST, int THREADS>
cudaLaunchConfig_t field_cfg(int n_max, int lw, int csize, cudaStream_t s, cudaLaunchAttribute *at, bool early = false)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)csize, (unsigned)n_max, 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = (size_t)kArrays * 8 * (size_t)lw;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (early) {
        // programmatic dependent launch: the CTAs may start while the
        // preceding particle kernel finishes, and wait in the kernel
        at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.numAttrs = 2;
    }
    return cfg;
}

// Clusters of csize CTAs that the GPU holds at once (cached per shape)
template <bool FAST, int THREADS>
int active_clusters(int lw, int csize)
{
    static std::mutex mu;
    static std::map<std::pair<int, int>, int> memo;
    std::lock_guard<std::mutex> g(mu);
    const auto key = std::make_pair(lw, csize);
    auto it = memo.find(key);
    if (it != memo.end()) return it->second;
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = field_cfg<FAST, THREADS>(1, lw, csize, nullptr, at);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_field<FAST, THREADS>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    memo[key] = n;
    return n;
}

template <bool FAST, int THREADS>
cudaError_t launch_cl(InstDev *inst, int n_max, int64_t *prefix, unsigned *ticket, int max_nodes, int csize,
                      cudaStream_t s, bool early)
{
    if (csize <= 0) {
        // about one node per half warp (at most -csize when csize < 0), but
        // no more CTAs per instance than lets every instance's cluster be
        // resident at once (one wave)
        const int cap = csize < 0 ? -csize : kMaxCluster;
        csize = cluster_size(max_nodes, THREADS);
        if (csize > cap) csize = cap;
        while (csize > 1 && active_clusters<FAST, THREADS>(array_len(max_nodes, csize), csize) < n_max) --csize;
    }
    // at least as many CTAs as the node arrays need to fit in shared memory
    while (csize < kMaxCluster && (size_t)kArrays * 8 * (size_t)array_len(max_nodes, csize) > kMaxDynSmem) ++csize;
    if (csize > kMaxCluster || (size_t)kArrays * 8 * (size_t)array_len(max_nodes, csize) > kMaxDynSmem)
        return cudaErrorInvalidValue;
    const int lw = array_len(max_nodes, csize);
    cudaLaunchAttribute at[2];
    const cudaLaunchConfig_t cfg = field_cfg<FAST, THREADS>(n_max, lw, csize, s, at, early);
    return cudaLaunchKernelEx(&cfg, k_field<FAST, THREADS>, inst, n_max, prefix, ticket, max_nodes, lw);
}

template <bool FAST>
cudaError_t launch_field_t(InstDev *inst, int n_max, int64_t *prefix, unsigned *ticket, int max_nodes, int threads,
                           int csize, cudaStream_t s, bool early)
{
    if (threads == 256) return launch_cl<FAST, 256>(inst, n_max, prefix, ticket, max_nodes, csize, s, early);
    if (threads == 512) return launch_cl<FAST, 512>(inst, n_max, prefix, ticket, max_nodes, csize, s, early);
    if (threads == 1024) return launch_cl<FAST, 1024>(inst, n_max, prefix, ticket, max_nodes, csize, s, early);
    return cudaErrorInvalidValue;
}

}  // namespace

// `fast`: reciprocals of the instance constants (split mode); divisions as a
// plain FP64 program writes them otherwise.  max_nodes bounds the node count
// of every instance launched (shared memory is sized for it; a larger
// instance is skipped by the device guard); threads: 256, 512 or 1024 per
// CTA; csize: CTAs per instance (1..16; raised until the node arrays fit in
// shared memory), 0 = about one node per half warp, as many as fit in one
// wave of clusters; -m the same with at most m.  early: the launch may start
// while the stream's preceding kernel (the step's particle kernel, which
// signals it) finishes; the kernel waits for it before reading its results.
cudaError_t launch_field(InstDev *inst, int n_max, int64_t *prefix, unsigned *ticket, bool fast, int max_nodes,
                         int threads, cudaStream_t s, int csize, bool early)
{
    if (max_nodes < 3 || max_nodes > kMaxNodes || n_max > HYB_MAX_INSTANCES || n_max > threads ||
        csize > kMaxCluster || csize < -kMaxCluster)
        return cudaErrorInvalidValue;
    return fast ? launch_field_t<true>(inst, n_max, prefix, ticket, max_nodes, threads, csize, s, early)
                : launch_field_t<false>(inst, n_max, prefix, ticket, max_nodes, threads, csize, s, early);
}

}  // namespace hyb
