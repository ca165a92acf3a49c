// hyb_electron.cu -- the per-particle kernels of the electron PIC/MCC step
// (arXiv 1508.02892, Sec. II.A): leapfrog push in the CIC-interpolated field,
// wall removal, CIC charge assignment with the energy moment and EEDF sample,
// modified null-collision MCC with ionization births (Sec. II.D), plus the
// initial load (the periodic cell sort is in hyb_sort.cu).
//
// Work decomposition: the running instances' slot ranges are concatenated and
// each block takes one contiguous chunk (particles are kept sorted by cell, so
// a chunk covers a narrow range of cells).  Deposits go to shared memory: in
// split mode per-warp rows of 32-bit fixed-point sums over a window of cells,
// flushed into the FP64 global sums; in FP64 mode block-private FP64 arrays,
// summed over the warp when all lanes share a cell, flushed over the touched
// node range.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hyb_device.cuh"

namespace hyb {

namespace {

// Per-thread event counts; the split kernel packs two 16-bit counts per word
// (a thread handles far fewer than 65536 particles of one segment).
struct SegCounters {
    unsigned el = 0, exc = 0, iz = 0, nul = 0, loss0 = 0, loss1 = 0, overflow = 0, push = 0, rec = 0;
    int cmin = INT32_MAX, cmax = -1;
};

struct PackedCounters {
    unsigned el_exc = 0, iz_nul = 0, loss = 0, push_ovf = 0, rec = 0;
    int cmin = INT32_MAX, cmax = -1;
    __device__ void unpack(SegCounters &s) const
    {
        s.el = el_exc & 0xFFFFu;
        s.exc = el_exc >> 16;
        s.iz = iz_nul & 0xFFFFu;
        s.nul = iz_nul >> 16;
        s.loss0 = loss & 0xFFFFu;
        s.loss1 = loss >> 16;
        s.push = push_ovf & 0xFFFFu;
        s.overflow = push_ovf >> 16;
        s.rec = rec;
        s.cmin = cmin;
        s.cmax = cmax;
    }
};

// Append children with one atomic per warp; all 32 lanes must call this.
template <typename T>
__device__ __forceinline__ void append_children(InstDev *K, const PartBuf &P, int64_t capacity, bool has, int cc, T co,
                                                double cz, T cvx, T cvy, T cvz, uint64_t cid, unsigned &overflow);

template <>
__device__ __forceinline__ void append_children<float>(InstDev *K, const PartBuf &P, int64_t capacity, bool has,
                                                       int cc, float co, double, float cvx, float cvy, float cvz,
                                                       uint64_t cid, unsigned &overflow)
{
    const unsigned m = __ballot_sync(kFull, has);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&K->n_slots, (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (has) {
        const unsigned long long slot = base + __popc(m & lanemask_lt());
        if (slot < (unsigned long long)capacity) {
            P.c[slot] = cc;
            P.o[slot] = co;
            P.vxf[slot] = cvx;
            P.vyf[slot] = cvy;
            P.vzf[slot] = cvz;
            P.id[slot] = cid;
        } else {
            overflow = 1;
        }
    }
}

template <>
__device__ __forceinline__ void append_children<double>(InstDev *K, const PartBuf &P, int64_t capacity, bool has, int,
                                                        double, double cz, double cvx, double cvy, double cvz,
                                                        uint64_t cid, unsigned &overflow)
{
    const unsigned m = __ballot_sync(kFull, has);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&K->n_slots, (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (has) {
        const unsigned long long slot = base + __popc(m & lanemask_lt());
        if (slot < (unsigned long long)capacity) {
            P.z[slot] = cz;
            P.vxd[slot] = cvx;
            P.vyd[slot] = cvy;
            P.vzd[slot] = cvz;
            P.id[slot] = cid;
        } else {
            overflow = 1;
        }
    }
}

// Kinetic ions: one new ion per ionization, at the new electron's position
// (z, or its cell and offset in split mode), id = the new electron's id,
// velocity from the gas Maxwellian (draw call 4 at the step); one atomic per
// warp on the ion descriptor.  All lanes call.  The ions are in the batch's
// precision: FP64 beside FP64 electrons, split beside split ones.
template <int PREC>
__device__ __forceinline__ void append_ion(InstDev *K, bool has, int c, float o, double z, uint64_t cid,
                                           uint32_t step)
{
    InstDev *I = K->ion;
    if (!I) return;  // a discharge with fluid ions in a batch that has kinetic ones
    const unsigned m = __ballot_sync(kFull, has);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&I->n_slots, (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (!has) return;
    const unsigned long long slot = base + __popc(m & lanemask_lt());
    if (slot >= (unsigned long long)I->capacity) {
        atomicOr(&K->status, (unsigned)HYB_STATUS_CAPACITY);
        return;
    }
    const uint4 a = draw(cid, step, K->seed_lo, K->seed_hi, 4);
    const PartBuf P = I->buf[I->cur];
    P.id[slot] = cid;
    if (PREC == HYB_FP32_SPLIT) {
        float s1, c1;
        const float r1 = sqrtf(-2.f * __logf(u01f(a.x)));
        __sincosf(6.283185307179586f * u01f(a.y), &s1, &c1);
        const float r2 = sqrtf(-2.f * __logf(u01f(a.z)));
        const float vt = K->fi_vt;
        P.c[slot] = c;
        P.o[slot] = o;
        P.vxf[slot] = vt * (r1 * c1);
        P.vyf[slot] = vt * (r1 * s1);
        P.vzf[slot] = vt * (r2 * __cosf(6.283185307179586f * u01f(a.w)));
    } else {
        double g1, g2, g3, g4;
        gauss_pair(u01d(a.x), u01d(a.y), g1, g2);
        gauss_pair(u01d(a.z), u01d(a.w), g3, g4);
        P.z[slot] = z;
        P.vxd[slot] = K->vt_gas * g1;
        P.vyd[slot] = K->vt_gas * g2;
        P.vzd[slot] = K->vt_gas * g3;
    }
}

// ------------------------------------------------------------ FP32 split
//
// Position = (cell c, offset o in [0,1)).  Constants are the f_* copies.
// Each thread takes V consecutive particles (V = 2 or 4, a tuning choice; one
// vector load and store per array), pushes them, deposits them into its
// warp's row of fixed-point cell sums in shared memory (below) and collides
// them, the V chains side by side.

constexpr int kVec = 2;  // particles per thread of the default step

// Per-warp deposit rows in shared memory: for kWin cells starting at `base`,
// 32-bit fixed-point sums of the particle count, the CIC weight to the upper
// node, the energy moment and its part to the upper node (to the lower node:
// count minus upper weight, energy minus upper part).  Every particle adds
// with native integer shared atomics; the warp flushes its row into the FP64
// global sums every kFlushIters iterations (which bounds the fixed-point
// range), when the warp moves past the row, and at the end of the segment.
// A fixed-point value v (0 <= v < 2^22) is formed without a conversion: one
// fused multiply-add gives the float v + 1.5 x 2^23, rounded to the nearest
// integer because floats in [2^23, 2^24) are spaced by 1, and its bits,
// 0x4B400000 + v, are what is added; the flush takes n x 0x4B400000 (mod
// 2^32) off each sum of n such adds.
constexpr int kWin = 64;
constexpr int kFlushParticles = 1024;  // a warp flushes its row after this many particles per lane group
constexpr float kFixW = 1048576.0f;    // 2^20: CIC weight, 1024 x 2^20 = 2^30
constexpr float kFixE = 1024.0f;       // 2^10: weight x energy (eV), 1024 x 2047 x 2^10 < 2^31
constexpr float kMaxFixE = 2047.0f;
constexpr float kFixBias = 12582912.0f;       // 1.5 x 2^23
constexpr unsigned kFixBiasBits = 0x4B400000u;  // its bit pattern

// a[k] and a[k] = v for a run-time k of a register array (selects, no local
// memory)
template <typename T, int N>
__device__ __forceinline__ T pick(const T (&a)[N], int k)
{
    T r = a[0];
#pragma unroll
    for (int j = 1; j < N; ++j) r = k == j ? a[j] : r;
    return r;
}
template <typename T, int N>
__device__ __forceinline__ void put(T (&a)[N], int k, T v)
{
#pragma unroll
    for (int j = 0; j < N; ++j)
        if (k == j) a[j] = v;
}

// V consecutive 4-byte values as one vector access (V = 2: 8 bytes, 4: 16)
template <int V, typename T>
__device__ __forceinline__ void load_vec(const T *p, T (&out)[V])
{
    static_assert(sizeof(T) == 4 && (V == 2 || V == 4), "4-byte values, 2 or 4 of them");
    if constexpr (V == 2) {
        const uint2 u = __ldcs(reinterpret_cast<const uint2 *>(p));
        out[0] = __builtin_bit_cast(T, u.x), out[1] = __builtin_bit_cast(T, u.y);
    } else {
        const uint4 u = __ldcs(reinterpret_cast<const uint4 *>(p));
        out[0] = __builtin_bit_cast(T, u.x), out[1] = __builtin_bit_cast(T, u.y);
        out[2] = __builtin_bit_cast(T, u.z), out[3] = __builtin_bit_cast(T, u.w);
    }
}
template <int V, typename T>
__device__ __forceinline__ void store_vec(T *p, const T (&v)[V])
{
    if constexpr (V == 2) {
        __stcs(reinterpret_cast<uint2 *>(p), make_uint2(__builtin_bit_cast(uint32_t, v[0]), __builtin_bit_cast(uint32_t, v[1])));
    } else {
        __stcs(reinterpret_cast<uint4 *>(p), make_uint4(__builtin_bit_cast(uint32_t, v[0]), __builtin_bit_cast(uint32_t, v[1]),
                                                        __builtin_bit_cast(uint32_t, v[2]), __builtin_bit_cast(uint32_t, v[3])));
    }
}

struct WarpRow {
    unsigned n[kWin], a1[kWin], e[kWin], e1[kWin];
};

__device__ __forceinline__ void add_global(InstDev *K, int c, double w0, double w1, double e0, double e1, int G)
{
    if (HYB_CHECK(c >= 0 && c + 1 < G, 4, c, G)) {
        atomicAdd(&K->dep_n[c], w0);
        atomicAdd(&K->dep_n[c + 1], w1);
        atomicAdd(&K->dep_e[c], e0);
        atomicAdd(&K->dep_e[c + 1], e1);
    }
}

__device__ __forceinline__ void row_flush(WarpRow &row, int base, InstDev *K, int G)
{
    __syncwarp();
    for (int j = threadIdx.x & 31; j < kWin; j += 32) {
        const unsigned n = row.n[j];
        if (n) {
            const unsigned bias = n * kFixBiasBits;
            const unsigned a1i = row.a1[j] - bias, ei = row.e[j] - bias, e1i = row.e1[j] - bias;
            const double a1 = (double)a1i * (1.0 / kFixW);
            add_global(K, base + j, (double)n - a1, a1, (double)(ei - e1i) * (1.0 / kFixE),
                       (double)e1i * (1.0 / kFixE), G);
            row.n[j] = row.a1[j] = row.e[j] = row.e1[j] = 0u;
        }
    }
    __syncwarp();
}

// Deposit one particle per lane (key < 0: none); warp-collective.
__device__ __forceinline__ void row_deposit(WarpRow &row, int &base, InstDev *K, int key, float o, float en, int G)
{
    if (key >= 0 && !(en < kMaxFixE)) {  // outside the fixed-point range
        add_global(K, key, 1.0 - o, o, (1.0 - o) * en, (double)o * en, G);
        key = -1;
    }
    if (__any_sync(kFull, key >= 0 && (unsigned)(key - base) >= (unsigned)kWin)) {
        row_flush(row, base, K, G);
        base = __reduce_min_sync(kFull, key >= 0 ? key : INT32_MAX) - kWin / 4;
        if (key >= 0 && (unsigned)(key - base) >= (unsigned)kWin) {  // a warp spread over more than the row
            add_global(K, key, 1.0 - o, o, (1.0 - o) * en, (double)o * en, G);
            return;
        }
    }
    if (key < 0) return;
    const int j = key - base;
    atomicAdd(&row.n[j], 1u);
    atomicAdd(&row.a1[j], __float_as_uint(fmaf(o, kFixW, kFixBias)));
    atomicAdd(&row.e[j], __float_as_uint(fmaf(en, kFixE, kFixBias)));
    atomicAdd(&row.e1[j], __float_as_uint(fmaf(o * en, kFixE, kFixBias)));
}

template <int MODE, bool CHEM, bool KIN, int V = kVec>
__device__ void segment_split(InstDev *K, int64_t a, int64_t b, unsigned char *smem, PackedCounters &cnt)
{
    static_assert(V == 2 || V == 4, "2 or 4 particles per thread");
    constexpr int kFlushIters = kFlushParticles / (32 * V);
    const int nc = K->n_cells;
    const int G = K->G;
    const int nb = K->eedf_bins;
    const uint32_t step = (uint32_t)K->step;
    const uint32_t sl = K->seed_lo, sh = K->seed_hi;
    const PartBuf P = K->buf[K->cur];
    const int64_t capacity = K->capacity;
    const float *__restrict__ gEf = K->Ef;
    const float4 *__restrict__ gxs = K->xsf;
    const int nxs = K->n_xs;
    const float dt_dz = K->f_dt_dz, qm_dt = K->f_qm_dt, half_m_q = K->f_half_m_q, two_q_m = K->f_two_q_m;
    const float pmax = K->f_pmax, e_lo = K->f_e_lo, e_hi = K->f_e_hi, inv_e_lo = K->f_inv_e_lo;
    const float inv_dlog = K->f_inv_dlog, e_exc = K->f_e_exc, e_iz = K->f_e_iz, two_mM = K->f_two_mM;
    const float bin_inv = K->f_bin_inv;
    const float inv_dlog2 = inv_dlog * 0.693147180559945309f;  // segments per octave of energy
    const PhiloxPre pre = philox_pre(step, sl, sh);

    // shared memory: EEDF histogram, one deposit row per warp, then (full
    // step) the field at the nodes, the cross-section table and the slopes of
    // its segments (formed once per block and discharge, so that a lookup is
    // one multiply-add per process)
    unsigned *s_eedf = reinterpret_cast<unsigned *>(smem);
    WarpRow *rows = reinterpret_cast<WarpRow *>(smem + 4 * (((nb + 2) + 3) & ~3));
    float *s_ef = reinterpret_cast<float *>(rows + (blockDim.x >> 5));
    float4 *s_xs = reinterpret_cast<float4 *>(s_ef + ((G + 3) & ~3));
    float4 *s_xsl = s_xs + nxs;
    if (!HYB_CHECK(b <= capacity && a >= 0 && (a & (V - 1)) == 0, 10, b, capacity)) b = a;
    {
        // the histogram and one deposit row per warp must fit in the launch's
        // dynamic shared memory
        unsigned dyn;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        const size_t need = 4 * (size_t)(((nb + 2) + 3) & ~3) + sizeof(WarpRow) * (size_t)(blockDim.x >> 5) +
                            (MODE == 0 ? 4 * (size_t)((G + 3) & ~3) + 32 * (size_t)nxs : 0);
        if (!HYB_CHECK(need <= (size_t)dyn, 13, need, dyn)) return;
    }
    if (MODE == 0) {
        for (int j = threadIdx.x; j < G; j += blockDim.x) s_ef[j] = gEf[j];
        for (int j = threadIdx.x; j < nxs; j += blockDim.x) {
            const float4 a = gxs[j];
            s_xs[j] = a;
            if (j + 1 < nxs) {
                const float4 b = gxs[j + 1];
                const float inv = 1.f / (b.x - a.x);
                s_xsl[j] = make_float4(0.f, (b.y - a.y) * inv, (b.z - a.z) * inv, (b.w - a.w) * inv);
            }
        }
    }
    const float *Ef = s_ef;
    const float4 *xs = s_xs;
    const float4 *xsl = s_xsl;
    for (int j = threadIdx.x; j <= nb + 1; j += blockDim.x) s_eedf[j] = 0u;
    {
        unsigned *r = reinterpret_cast<unsigned *>(rows);
        for (int j = threadIdx.x; j < 4 * kWin * (int)(blockDim.x >> 5); j += blockDim.x) r[j] = 0u;
    }
    __syncthreads();

    // each warp sweeps a contiguous part of [a, b) in groups of 32 * V
    const int nwarps = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t per = (((b - a) + nwarps - 1) / nwarps + 32 * V - 1) / (32 * V) * (32 * V);
    const int64_t wa = a + per * wid;
    const int64_t wb = wa + per < b ? wa + per : b;
    WarpRow &row = rows[wid];
    int rbase = INT32_MIN / 2;
    int iter = 0;
    for (int64_t base = wa; base < wb; base += 32 * V) {
        const int64_t i0 = base + (int64_t)lane * V;
        const bool full = i0 + V <= wb;
        int cc[V];
        float oo[V], vx[V], vy[V], vz[V];
        uint64_t ids[V];
        if (full) {
            // streaming (evict-first) loads and stores: the particle state is
            // touched once per step and should not displace the field, the
            // cross-section table or the deposit rows in L1 and L2
            load_vec<V>(P.c + i0, cc);
            load_vec<V>(P.o + i0, oo);
            load_vec<V>(P.vxf + i0, vx);
            load_vec<V>(P.vyf + i0, vy);
            load_vec<V>(P.vzf + i0, vz);
            if (MODE == 0) {
#pragma unroll
                for (int k = 0; k < V; k += 2) {
                    const ulonglong2 d0 = __ldcs(reinterpret_cast<const ulonglong2 *>(P.id + i0 + k));
                    ids[k] = d0.x, ids[k + 1] = d0.y;
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const bool in = i0 + k < wb;
                cc[k] = in ? P.c[i0 + k] : kDeadCell;
                oo[k] = in ? P.o[i0 + k] : 0.f;
                vx[k] = in ? P.vxf[i0 + k] : 0.f;
                vy[k] = in ? P.vyf[i0 + k] : 0.f;
                vz[k] = in ? P.vzf[i0 + k] : 0.f;
                ids[k] = (MODE == 0 && in) ? P.id[i0 + k] : 0ull;
            }
        }

        {
            // the warp's next group of particles into L1 while this one is
            // pushed (a prefetch holds no registers)
            const int64_t inx = i0 + 32 * V;
            if (inx + V <= wb) {
                asm volatile("prefetch.global.L1 [%0];" ::"l"(P.c + inx));
                asm volatile("prefetch.global.L1 [%0];" ::"l"(P.o + inx));
                asm volatile("prefetch.global.L1 [%0];" ::"l"(P.vxf + inx));
                asm volatile("prefetch.global.L1 [%0];" ::"l"(P.vyf + inx));
                asm volatile("prefetch.global.L1 [%0];" ::"l"(P.vzf + inx));
                if (MODE == 0) asm volatile("prefetch.global.L1 [%0];" ::"l"(P.id + inx));
            }
        }
        unsigned coll = 0u;      // bit k: slot k ionized (handled in the warp pass below)
        uint2 ru[V];          // direction draws of the colliding particles
        float ens[V];         // kinetic energies (eV) after the push
        bool live[V];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            // leapfrog with the CIC-gathered field (Sec. II.A), formed for every
            // lane and kept for the live ones; the gather index is clamped so
            // that no out-of-range address is formed
            int c = cc[k];
            float o = oo[k];
            bool alive = c >= 0 && c < nc;
            if (MODE == 0) {
                const int cg = min(max(c, 0), nc - 1);
                const float oi = alive ? o : 0.f;
                const float e0 = Ef[cg];
                const float ep = fmaf(oi, Ef[cg + 1] - e0, e0);
                const float vzn = vz[k] - qm_dt * ep;
                float on = oi + vzn * dt_dz;
                const float fl = floorf(on);
                int cn = cg + (int)fl;
                on -= fl;
                const bool wrap = on >= 1.f;
                on = wrap ? on - 1.f : on;
                cn = wrap ? cn + 1 : cn;
                const bool gone = cn < 0 || cn >= nc;  // absorbed by an electrode and removed
                cnt.push_ovf += alive ? 1u : 0u;
                cnt.loss += (alive && gone) ? (cn < 0 ? 1u : (1u << 16)) : 0u;
                vz[k] = alive ? vzn : vz[k];
                o = alive ? on : o;
                c = cn;
                alive = alive && !gone;
            }
            ens[k] = half_m_q * (vx[k] * vx[k] + vy[k] * vy[k] + vz[k] * vz[k]);
            live[k] = alive;
            cc[k] = alive ? c : kDeadCell;
            oo[k] = o;
        }
        // CIC charge assignment and energy moment, then the EEDF sample
#pragma unroll
        for (int k = 0; k < V; ++k)
            row_deposit(row, rbase, K, live[k] ? cc[k] : -1, oo[k], MODE == 0 ? ens[k] : 0.f, G);
        if (MODE == 0) {
            // EEDF sample: bin nb is the overflow (also NaN), bin nb + 1 takes the
            // removed particles and is never read
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const float en = ens[k];
                int bin = (int)(en * bin_inv);
                bin = ((unsigned)bin > (unsigned)nb || !(en >= 0.f)) ? nb : bin;
                atomicAdd(&s_eedf[live[k] ? bin : nb + 1], 1u);
            }
        }
        if (MODE == 0) {
            // modified null-collision method: every particle draws R1 < P_max;
            // the process is the first k with R2 nu_max < sum_{i<=k} nu_i.  The
            // V particles' draws are formed together (independent chains).
            uint4 rk[V];
            draw_n<V>(pre, ids, 0u, rk);
            uint4 rq[V] = {};
            if (CHEM && K->rec_on) draw_n<V>(pre, ids, 2u, rq);
#pragma unroll
            for (int k = 0; k < V; ++k) {
                // computed for every lane without branches, so that the V
                // chains interleave; only candidates keep their outcome
                const float en = ens[k];
                bool cand = cc[k] >= 0 && cc[k] < nc && u01f(rk[k].x) < pmax;
                const float speed = sqrtf(vx[k] * vx[k] + vy[k] * vy[k] + vz[k] * vz[k]);
                // table segment: below the table the first node's values,
                // above it the last node's
                int kk = (int)(__log2f(fmaxf(en, e_lo) * inv_e_lo) * inv_dlog2);
                kk = kk < 0 ? 0 : (kk > nxs - 2 ? nxs - 2 : kk);
                // sigma_i(E) = sigma_i(E_k) + (E - E_k) slope_i with E clamped to
                // the table: below it the first node's values, above the last's
                const float4 lo = xs[kk];
                const float4 slope = xsl[kk];
                const bool below = en <= e_lo, above = en >= e_hi;
                const float dd = fminf(fmaxf(en, e_lo), e_hi) - lo.x;
                const float s_el = lo.y + dd * slope.y;
                const float s_ex = en < e_exc ? 0.f : lo.z + dd * slope.z;
                const float s_iz = en < e_iz ? 0.f : lo.w + dd * slope.w;
                const float4 hi = CHEM ? xs[kk + 1] : lo;
                const float f = (below || !CHEM) ? 0.f : __fdividef(en - lo.x, hi.x - lo.x);
                if (CHEM && cc[k] >= 0 && cc[k] < nc && u01f(rq[k].x) < K->f_rec_pmax) {
                    // electron-ion recombination (Sec. II.D), in units of nu_rec,max:
                    // R4 < (n_i / max n_i)(sigma_rec / max sigma_rec v) v
                    const int cr = cc[k];
                    const float rl = __ldg(&K->xs_recf[kk]), rh = __ldg(&K->xs_recf[kk + 1]);
                    const float sr = above ? rh : rl + f * (rh - rl);
                    const float nr = (1.f - oo[k]) * __ldg(&K->nif[cr]) + oo[k] * __ldg(&K->nif[cr + 1]);
                    if (u01f(rq[k].y) < nr * sr * speed) {
                        cnt.rec += 1u;
                        cand = false;
                        cc[k] = kDeadCell;
                        if (HYB_CHECK(cr >= 0 && cr + 1 < G, 4, cr, G)) {
                            atomicAdd(&K->s_iz[cr], -(1.0 - (double)oo[k]));
                            atomicAdd(&K->s_iz[cr + 1], -(double)oo[k]);
                        }
                    }
                }
                const float t0 = s_el * speed, t1 = t0 + s_ex * speed, t2 = t1 + s_iz * speed;
                const float r2 = u01f(rk[k].y);
                const bool hit = cand && r2 < t2;
                const unsigned kind = r2 < t0 ? 1u : (r2 < t1 ? 2u : 3u);
                // elastic (lab-frame isotropic, energy loss (2m/M)(1 - cos chi))
                // and excitation (E - E_exc) scatter in place, formed for every
                // lane and kept where they happened; ionizations, which eject
                // an electron, go to the warp pass below
                const float v2 = vx[k] * vx[k] + vy[k] * vy[k] + vz[k] * vz[k];
                // cos chi = 1 - 2u and phi = 2 pi u, each one fused multiply-add
                // of the bits 1 + k 2^-23 that u01f forms (u = those less
                // 1 - 2^-24), rounded once
                const float ct = fmaf(u01f_bits(rk[k].z), -2.f, 3.f);
                const float st = sqrtf(fmaxf(0.f, 1.f - ct * ct));
                float sn, cs;
                __sincosf(fmaf(u01f_bits(rk[k].w), 6.283185307179586f, -6.283185307179586f * 0.999999940395355224609375f),
                          &sn, &cs);
                const float dx = st * cs, dy = st * sn, dzz = ct;
                const float rs = rsqrtf(v2);
                const float cchi = (vx[k] * dx + vy[k] * dy + vz[k] * dzz) * rs;
                // the squared speed after either process; one square root
                // for the one that happened
                const float q_el = v2 * (1.f - two_mM * (1.f - cchi));
                const float q_ex = two_q_m * (en - e_exc);
                const bool scat = hit && kind != 3u;
                const float sp = sqrtf(kind == 1u ? q_el : q_ex);
                vx[k] = scat ? sp * dx : vx[k];
                vy[k] = scat ? sp * dy : vy[k];
                vz[k] = scat ? sp * dzz : vz[k];
                cnt.el_exc += scat ? (kind == 1u ? 1u : (1u << 16)) : 0u;
                if (CHEM && scat && kind == 2u && K->met_on) {
                    // a metastable at the electron (Sec. II.D), CIC
                    const int cm = cc[k];
                    if (HYB_CHECK(cm >= 0 && cm + 1 < G, 4, cm, G)) {
                        atomicAdd(&K->s_met[cm], 1.0 - (double)oo[k]);
                        atomicAdd(&K->s_met[cm + 1], (double)oo[k]);
                    }
                }
                coll |= (hit && kind == 3u) ? (1u << k) : 0u;
                ru[k] = make_uint2(rk[k].z, rk[k].w);
                cnt.iz_nul += (cand && !hit) ? (1u << 16) : 0u;
            }
        }
        if (++iter == kFlushIters) {
            row_flush(row, rbase, K, G);
            iter = 0;
        }
        if (MODE == 0) {
            // ionizations of the warp, one particle per lane per pass: split
            // E - E_iz between the scattered and the ejected electron, both
            // isotropic, the child appended with its ion source (Sec. II.D)
            while (__any_sync(kFull, coll != 0u)) {
                const int k = coll ? __ffs(coll) - 1 : 0;
                bool has_child = false;
                float cvx = 0.f, cvy = 0.f, cvz = 0.f;
                uint64_t cid = 0;
                int ck = 0;
                float ok = 0.f;
                if (coll) {
                    const float px = pick(vx, k), py = pick(vy, k), pz = pick(vz, k);
                    const uint2 rr = pick(ru, k);
                    const uint64_t pid = pick(ids, k);
                    ck = pick(cc, k);
                    ok = pick(oo, k);
                    const float en = half_m_q * (px * px + py * py + pz * pz);
                    const float ct = 1.f - 2.f * u01f(rr.x);
                    const float st = sqrtf(fmaxf(0.f, 1.f - ct * ct));
                    float sn, cs;
                    __sincosf(6.283185307179586f * u01f(rr.y), &sn, &cs);
                    const uint4 r1 = draw_pre(pre, pid, 1u);
                    const float de = en - e_iz;
                    const float e_ej = u01f(r1.x) * de;
                    const float sp = sqrtf(two_q_m * (de - e_ej));
                    const float cj = 1.f - 2.f * u01f(r1.y);
                    const float sj = sqrtf(fmaxf(0.f, 1.f - cj * cj));
                    float snj, csj;
                    __sincosf(6.283185307179586f * u01f(r1.z), &snj, &csj);
                    const float spj = sqrtf(two_q_m * e_ej);
                    cvx = spj * sj * csj;
                    cvy = spj * sj * snj;
                    cvz = spj * cj;
                    cid = child_id(pid, step);
                    has_child = true;
                    cnt.iz_nul += 1u;
                    if (HYB_CHECK(ck >= 0 && ck + 1 < G, 4, ck, G)) {
                        atomicAdd(&K->s_iz[ck], 1.0 - ok);
                        atomicAdd(&K->s_iz[ck + 1], (double)ok);
                    }
                    put(vx, k, sp * (st * cs));
                    put(vy, k, sp * (st * sn));
                    put(vz, k, sp * ct);
                }
                unsigned ovf = 0;
                append_children<float>(K, P, capacity, has_child, ck, ok, 0.0, cvx, cvy, cvz, cid, ovf);
                if (KIN) append_ion<HYB_FP32_SPLIT>(K, has_child, ck, ok, 0.0, cid, step);
                cnt.push_ovf |= ovf << 16;
                coll &= ~(1u << k);
            }
        }
        if (MODE == 0) {
            if (full) {
                store_vec<V>(P.c + i0, cc);
                store_vec<V>(P.o + i0, oo);
                store_vec<V>(P.vxf + i0, vx);
                store_vec<V>(P.vyf + i0, vy);
                store_vec<V>(P.vzf + i0, vz);
            } else {
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    if (i0 + k < wb) {
                        P.c[i0 + k] = cc[k];
                        P.o[i0 + k] = oo[k];
                        P.vxf[i0 + k] = vx[k];
                        P.vyf[i0 + k] = vy[k];
                        P.vzf[i0 + k] = vz[k];
                    }
                }
            }
        }
    }
    row_flush(row, rbase, K, G);
}

// ------------------------------------------------------------------ FP64
//
// Same step in FP64 with the position z, written in the same order of
// operations as a plain FP64 program would use, so the two agree to rounding.

// sigma_rec(E) with the same log-index, linear-in-energy lookup
__device__ __forceinline__ double xs_rec_d(const double *__restrict__ xr, const double *__restrict__ xs, int n,
                                           double e_lo, double e_hi, double inv_dlog, double en)
{
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
        f = (en - xs[4 * i]) / (xs[4 * (i + 1)] - xs[4 * i]);
    }
    return xr[i] + f * (xr[i + 1] - xr[i]);
}

__device__ __forceinline__ void xs_eval_d(const double *__restrict__ xs, int n, double e_lo, double e_hi,
                                          double inv_dlog, double e_exc, double e_iz, double en, double sig[3])
{
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
        f = (en - xs[4 * i]) / (xs[4 * (i + 1)] - xs[4 * i]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) sig[k] = xs[4 * i + 1 + k] + f * (xs[4 * (i + 1) + 1 + k] - xs[4 * i + 1 + k]);
    if (en < e_exc) sig[1] = 0.0;
    if (en < e_iz) sig[2] = 0.0;
}

template <int MODE, bool CHEM, bool KIN>
__device__ void segment_fp64(InstDev *K, int64_t a, int64_t b, unsigned char *smem, SegCounters &cnt)
{
    const int nc = K->n_cells;
    const int G = K->G;
    const int nb = K->eedf_bins;
    const uint32_t step = (uint32_t)K->step;
    const uint32_t sl = K->seed_lo, sh = K->seed_hi;
    const PartBuf P = K->buf[K->cur];
    const int64_t capacity = K->capacity;
    const double *__restrict__ E = K->E;
    const double *__restrict__ xs = K->xs;
    const int nxs = K->n_xs;
    const double dz = K->dz, dt = K->dt, L = K->L, qm = K->qm, ngas = K->ngas, nu_max = K->nu_max;
    const double pmax = K->p_max, e_lo = K->e_lo, e_hi = K->e_hi, inv_dlog = K->inv_dlog;
    const double e_exc = K->e_exc, e_iz = K->e_iz, two_mM = K->two_mM, bin_w = K->bin_w;

    double *sd_n = reinterpret_cast<double *>(smem);
    double *sd_e = sd_n + G;
    double *sd_iz = sd_e + G;
    unsigned *s_eedf = reinterpret_cast<unsigned *>(sd_iz + G);
    if (!HYB_CHECK(b <= capacity && a >= 0, 10, b, capacity)) b = a;
    for (int j = threadIdx.x; j < 3 * G; j += blockDim.x) sd_n[j] = 0.0;
    for (int j = threadIdx.x; j <= nb; j += blockDim.x) s_eedf[j] = 0u;
    __syncthreads();

    for (int64_t base = a; base < b; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        double z = i < b ? P.z[i] : -1.0;
        bool alive = z >= 0.0 && z < L;  // also false for NaN
        double vx = 0.0, vy = 0.0, vz = 0.0;
        uint64_t id = 0;
        if (alive) {
            vx = P.vxd[i];
            vy = P.vyd[i];
            vz = P.vzd[i];
            if (MODE == 0) id = P.id[i];
        }
        int c = 0;
        double o = 0.0;
        if (MODE == 0 && alive) {
            ++cnt.push;
            locate_d(z, dz, nc, c, o);
            const double ep = (1.0 - o) * E[c] + o * E[c + 1];
            vz = vz - qm * ep * dt;
            z = z + vz * dt;
            if (!(z >= 0.0 && z < L)) {
                if (z < 0.0)
                    ++cnt.loss0;
                else
                    ++cnt.loss1;
                alive = false;
                P.z[i] = -1.0;
            }
        }
        if (alive) locate_d(z, dz, nc, c, o);
        const double en = 0.5 * kMe * (vx * vx + vy * vy + vz * vz) / kQe;
        deposit_pair<double>(sd_n, alive, c, 1.0 - o, o, G);
        if (MODE == 0) {
            deposit_pair<double>(sd_e, alive, c, (1.0 - o) * en, o * en, G);
            if (alive) {
                int bin = (int)(en / bin_w);
                if (bin > nb || bin < 0 || !(en >= 0.0)) bin = nb;  // overflow bin (also NaN)
                atomicAdd(&s_eedf[bin], 1u);
            }
        }
        if (alive) {
            cnt.cmin = min(cnt.cmin, c);
            cnt.cmax = max(cnt.cmax, c);
        }

        if (CHEM && MODE == 0 && alive && K->rec_on) {
            // electron-ion recombination (Sec. II.D): candidate if R3 < P_rec,
            // real if R4 nu_rec,max < n_i(z) sigma_rec(E) v; the electron is
            // removed and its ion leaves through a CIC sink in the ion source
            const uint4 rq = draw(id, step, sl, sh, 2);
            if (u01d(rq.x) < K->rec_pmax) {
                const double nil = (1.0 - o) * K->ni[c] + o * K->ni[c + 1];
                const double speed = sqrt(vx * vx + vy * vy + vz * vz);
                const double sig = xs_rec_d(K->xs_rec, xs, nxs, e_lo, e_hi, inv_dlog, en);
                if (u01d(rq.y) * K->rec_numax < nil * sig * speed) {
                    ++cnt.rec;
                    alive = false;
                    P.z[i] = -1.0;
                    atomicAdd(&sd_iz[c], -(1.0 - o));
                    atomicAdd(&sd_iz[c + 1], -o);
                }
            }
        }
        bool has_child = false;
        double cvx = 0.0, cvy = 0.0, cvz = 0.0;
        uint64_t cid = 0;
        if (MODE == 0 && alive) {
            const uint4 r = draw(id, step, sl, sh, 0);
            if (u01d(r.x) < pmax) {
                const double speed = sqrt(vx * vx + vy * vy + vz * vz);
                double sig[3];
                xs_eval_d(xs, nxs, e_lo, e_hi, inv_dlog, e_exc, e_iz, en, sig);
                const double nu_el = ngas * sig[0] * speed;
                const double nu_ex = ngas * sig[1] * speed;
                const double nu_iz = ngas * sig[2] * speed;
                const double rr = u01d(r.y) * nu_max;
                double d[3];
                iso_dir_d(u01d(r.z), u01d(r.w), d);
                if (rr < nu_el) {
                    const double cchi = (vx * d[0] + vy * d[1] + vz * d[2]) / speed;
                    const double sp = speed * sqrt(1.0 - two_mM * (1.0 - cchi));
                    vx = sp * d[0];
                    vy = sp * d[1];
                    vz = sp * d[2];
                    ++cnt.el;
                } else if (rr < nu_el + nu_ex) {
                    const double sp = sqrt(2.0 * kQe * (en - e_exc) / kMe);
                    vx = sp * d[0];
                    vy = sp * d[1];
                    vz = sp * d[2];
                    ++cnt.exc;
                    if (CHEM && K->met_on) {  // a metastable at the electron (Sec. II.D), CIC
                        atomicAdd(&K->s_met[c], 1.0 - o);
                        atomicAdd(&K->s_met[c + 1], o);
                    }
                } else if (rr < nu_el + nu_ex + nu_iz) {
                    const uint4 r1 = draw(id, step, sl, sh, 1);
                    const double de = en - e_iz;
                    const double e_ej = u01d(r1.x) * de;
                    const double e_sc = de - e_ej;
                    const double sp = sqrt(2.0 * kQe * e_sc / kMe);
                    double dj[3];
                    iso_dir_d(u01d(r1.y), u01d(r1.z), dj);
                    const double sj = sqrt(2.0 * kQe * e_ej / kMe);
                    cvx = sj * dj[0];
                    cvy = sj * dj[1];
                    cvz = sj * dj[2];
                    cid = child_id(id, step);
                    has_child = true;
                    vx = sp * d[0];
                    vy = sp * d[1];
                    vz = sp * d[2];
                    ++cnt.iz;
                    atomicAdd(&sd_iz[c], 1.0 - o);
                    atomicAdd(&sd_iz[c + 1], o);
                } else {
                    ++cnt.nul;
                }
            }
        }
        if (MODE == 0) {
            append_children<double>(K, P, capacity, has_child, 0, 0.0, z, cvx, cvy, cvz, cid, cnt.overflow);
            if (KIN) append_ion<HYB_FP64>(K, has_child, 0, 0.f, z, cid, step);
            if (alive) {
                P.z[i] = z;
                P.vxd[i] = vx;
                P.vyd[i] = vy;
                P.vzd[i] = vz;
            }
        }
    }
}

// Reduce the per-thread counters, then flush the block-private sums over the
// touched node range into the global FP64 sums (FP64 mode).
__device__ __forceinline__ double sum_value(double q) { return q; }

// Split mode: the node sums went to global memory already; flush the EEDF
// histogram and the counters.
template <int MODE>
__device__ void flush_segment_split(InstDev *K, unsigned char *smem, const SegCounters &cnt)
{
    __shared__ unsigned s_ctr2[9];
    if (threadIdx.x < 9) s_ctr2[threadIdx.x] = 0u;
    __syncthreads();
    const unsigned v[9] = {cnt.el, cnt.exc, cnt.iz, cnt.nul, cnt.loss0, cnt.loss1, cnt.overflow, cnt.push, cnt.rec};
    unsigned tot[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) tot[k] = __reduce_add_sync(kFull, v[k]);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if (tot[k]) atomicAdd(&s_ctr2[k], tot[k]);
    }
    __syncthreads();
    if (MODE == 0) {
        const int nb = K->eedf_bins;
        const unsigned *s_eedf = reinterpret_cast<const unsigned *>(smem);
        for (int j = threadIdx.x; j <= nb; j += blockDim.x)
            if (s_eedf[j]) atomicAdd(&K->eedf[j], (unsigned long long)s_eedf[j]);
        if (threadIdx.x == 0) {
            const int map[6] = {C_EL, C_EXC, C_IZ, C_NULL, C_LOSS0, C_LOSS1};
#pragma unroll
            for (int k = 0; k < 6; ++k)
                if (s_ctr2[k]) atomicAdd(&K->ctr[map[k]], (unsigned long long)s_ctr2[k]);
            if (s_ctr2[2]) atomicAdd(&K->ctr[C_BIRTH_IZ], (unsigned long long)s_ctr2[2]);
            if (s_ctr2[6]) atomicOr(&K->status, (unsigned)HYB_STATUS_CAPACITY);
            if (s_ctr2[7]) atomicAdd(&K->ctr[C_PUSH], (unsigned long long)s_ctr2[7]);
            if (s_ctr2[8]) atomicAdd(&K->ctr[C_REC], (unsigned long long)s_ctr2[8]);
        }
    }
    __syncthreads();
}

template <typename S, int MODE>
__device__ void flush_segment(InstDev *K, unsigned char *smem, const SegCounters &cnt)
{
    __shared__ unsigned s_ctr[9];
    __shared__ int s_cmin, s_cmax;
    if (threadIdx.x < 9) s_ctr[threadIdx.x] = 0u;
    if (threadIdx.x == 0) {
        s_cmin = INT32_MAX;
        s_cmax = -1;
    }
    __syncthreads();
    const unsigned v[9] = {cnt.el, cnt.exc, cnt.iz, cnt.nul, cnt.loss0, cnt.loss1, cnt.overflow, cnt.push, cnt.rec};
    const int mn = __reduce_min_sync(kFull, cnt.cmin);
    const int mx = __reduce_max_sync(kFull, cnt.cmax);
    unsigned tot[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) tot[k] = __reduce_add_sync(kFull, v[k]);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if (tot[k]) atomicAdd(&s_ctr[k], tot[k]);
        atomicMin(&s_cmin, mn);
        atomicMax(&s_cmax, mx);
    }
    __syncthreads();
    const int G = K->G;
    const int nb = K->eedf_bins;
    S *sd_n = reinterpret_cast<S *>(smem);
    S *sd_e = sd_n + G;
    S *sd_iz = sd_e + G;
    unsigned *s_eedf = reinterpret_cast<unsigned *>(sd_iz + G);
    int jlo = s_cmin, jhi = s_cmax < 0 ? -1 : min(s_cmax + 1, G - 1);
    if (jhi >= 0 && !HYB_CHECK(jlo >= 0 && jlo <= jhi, 6, jlo, jhi)) jhi = -1;
    for (int j = (jhi < 0 ? 0 : jlo) + (int)threadIdx.x; j <= jhi; j += blockDim.x) {
        const S a = sd_n[j];
        if (a != S(0)) atomicAdd(&K->dep_n[j], sum_value(a));
        if (MODE == 0) {
            const S e = sd_e[j];
            if (e != S(0)) atomicAdd(&K->dep_e[j], sum_value(e));
            const S s = sd_iz[j];
            if (s != S(0)) atomicAdd(&K->s_iz[j], sum_value(s));
        }
    }
    if (MODE == 0) {
        for (int j = threadIdx.x; j <= nb; j += blockDim.x)
            if (s_eedf[j]) atomicAdd(&K->eedf[j], (unsigned long long)s_eedf[j]);
        if (threadIdx.x == 0) {
            const int map[6] = {C_EL, C_EXC, C_IZ, C_NULL, C_LOSS0, C_LOSS1};
#pragma unroll
            for (int k = 0; k < 6; ++k)
                if (s_ctr[k]) atomicAdd(&K->ctr[map[k]], (unsigned long long)s_ctr[k]);
            if (s_ctr[2]) atomicAdd(&K->ctr[C_BIRTH_IZ], (unsigned long long)s_ctr[2]);
            if (s_ctr[6]) atomicOr(&K->status, (unsigned)HYB_STATUS_CAPACITY);
            if (s_ctr[7]) atomicAdd(&K->ctr[C_PUSH], (unsigned long long)s_ctr[7]);
            if (s_ctr[8]) atomicAdd(&K->ctr[C_REC], (unsigned long long)s_ctr[8]);
        }
    }
    __syncthreads();
}

// Blocks per SM the register budget is set for: 80 registers a thread with two
// particles per thread (a third of the file at 256 threads), 128 with four
constexpr int electron_min_blocks(int prec, int threads, int ppt)
{
    return ppt == 4 ? (threads == 128 ? 4 : (threads == 512 ? 1 : 2))
                    : (threads == 128 ? 6 : (threads == 512 ? 1 : (prec == HYB_FP32_SPLIT ? 3 : 2)));
}

// THREADS: 256 for every variant; the default split-mode step is also built
// for 128 and 512 (a tuning choice), and with four particles per thread (PPT)
template <int PREC, int MODE, bool CHEM = false, bool KIN = false, int THREADS = kBlock, int PPT = kVec>
__global__ void __launch_bounds__(THREADS, electron_min_blocks(PREC, THREADS, PPT))
    k_electron(InstDev *__restrict__ insts, int n_max, const int64_t *__restrict__ prefix)
{
    extern __shared__ __align__(16) unsigned char smem[];
    // a field step launched to start early may be scheduled once every block
    // of this grid has started (it waits for this grid's end before reading
    // any of its results)
    asm volatile("griddepcontrol.launch_dependents;");
    for_block_runs(insts, n_max, prefix, [&](InstDev *K, int64_t a, int64_t b) {
        SegCounters cnt;
        if (PREC == HYB_FP32_SPLIT) {
            PackedCounters pc;
            segment_split<MODE, CHEM, KIN, PPT>(K, a, b, smem, pc);
            pc.unpack(cnt);
            flush_segment_split<MODE>(K, smem, cnt);
        } else {
            segment_fp64<MODE, CHEM, KIN>(K, a, b, smem, cnt);
            flush_segment<double, MODE>(K, smem, cnt);
        }
    });
}

// ------------------------------------------------------------- initial load
// Uniform positions and a Maxwellian (Box-Muller), ids 0..n-1, drawn at the
// reserved step 0xFFFFFFFF.
__global__ void k_load(InstDev *K, int64_t n, double vth, int prec)
{
    const PartBuf P = K->buf[K->cur];
    const double L = K->L, dz = K->dz;
    const int nc = K->n_cells;
    if (!HYB_CHECK(n <= K->capacity, 9, n, K->capacity)) return;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t id = (uint64_t)j;
        const uint4 a = draw(id, 0xFFFFFFFFu, K->seed_lo, K->seed_hi, 0);
        const uint4 b = draw(id, 0xFFFFFFFFu, K->seed_lo, K->seed_hi, 1);
        const double z = u01d(a.x) * L;
        const double r1 = sqrt(-2.0 * log(u01d(a.y)));
        const double p1 = kTwoPi * u01d(a.z);
        const double r2 = sqrt(-2.0 * log(u01d(a.w)));
        const double p2 = kTwoPi * u01d(b.x);
        const double vx = vth * (r1 * cos(p1)), vy = vth * (r1 * sin(p1)), vz = vth * (r2 * cos(p2));
        P.id[j] = id;
        if (prec == HYB_FP32_SPLIT) {
            int c;
            double o;
            locate_d(z, dz, nc, c, o);
            P.c[j] = c;
            P.o[j] = (float)o;
            P.vxf[j] = (float)vx;
            P.vyf[j] = (float)vy;
            P.vzf[j] = (float)vz;
        } else {
            P.z[j] = z;
            P.vxd[j] = vx;
            P.vyd[j] = vy;
            P.vzd[j] = vz;
        }
    }
}

__global__ void __launch_bounds__(HYB_MAX_INSTANCES) k_prefix(InstDev *insts, int n_max, int64_t *prefix)
{
    __shared__ int64_t s_buf[HYB_MAX_INSTANCES];
    block_chunk_prefix(insts, n_max, prefix, s_buf);
}

// prefix over one instance that is being (re)initialised
__global__ void k_prefix_one(InstDev *K, int64_t *prefix)
{
    if (threadIdx.x != 0) return;
    prefix[0] = 0;
    prefix[1] = chunks_of((int64_t)K->n_slots);
    K->n_slots_step = (int64_t)K->n_slots;
}

__global__ void k_set_active(InstDev *K, int active, int64_t target_step)
{
    if (threadIdx.x != 0) return;
    K->active = active;
    K->target_step = target_step;
}

template <int PREC, int MODE, bool CHEM = false, bool KIN = false, int THREADS = kBlock, int PPT = kVec>
cudaError_t launch_k(InstDev *inst, int n_max, const int64_t *prefix, LaunchCfg cfg, cudaStream_t s)
{
    k_electron<PREC, MODE, CHEM, KIN, THREADS, PPT><<<cfg.grid, THREADS, cfg.smem, s>>>(inst, n_max, prefix);
    return cudaGetLastError();
}

}  // namespace

void read_checks_electron(unsigned long long out[3])
{
    if (cudaMemcpyFromSymbol(out, g_hyb_check, sizeof(unsigned long long) * 3) != cudaSuccess)
        out[0] = out[1] = out[2] = 0ull;
}

void configure_kernels()
{
    // opt in to all the shared memory a block may have
    allow_max_dynamic_smem(k_electron<HYB_FP32_SPLIT, 0>);
    allow_max_dynamic_smem(k_electron<HYB_FP32_SPLIT, 1>);
    allow_max_dynamic_smem(k_electron<HYB_FP64, 0>);
    allow_max_dynamic_smem(k_electron<HYB_FP64, 1>);
    allow_max_dynamic_smem(k_electron<HYB_FP32_SPLIT, 0, true>);
    allow_max_dynamic_smem(k_electron<HYB_FP64, 0, true>);
    allow_max_dynamic_smem(k_electron<HYB_FP32_SPLIT, 0, false, true>);
    allow_max_dynamic_smem(k_electron<HYB_FP64, 0, false, true>);
    allow_max_dynamic_smem(k_electron<HYB_FP32_SPLIT, 0, true, true>);
    allow_max_dynamic_smem(k_electron<HYB_FP64, 0, true, true>);
    allow_max_dynamic_smem(k_electron<HYB_FP32_SPLIT, 0, false, false, 128>);
    allow_max_dynamic_smem(k_electron<HYB_FP32_SPLIT, 0, false, false, 512>);
    allow_max_dynamic_smem(k_electron<HYB_FP32_SPLIT, 0, false, false, 128, 4>);
    allow_max_dynamic_smem(k_electron<HYB_FP32_SPLIT, 0, false, false, 256, 4>);
    allow_max_dynamic_smem(k_electron<HYB_FP32_SPLIT, 0, false, false, 512, 4>);
    configure_ion_kernels();
    configure_field_kernel();
}

int electron_blocks_per_sm(int precision, size_t smem, int threads, int ppt)
{
    int n = 0;
    if (precision == HYB_FP32_SPLIT && ppt == 4) {
        if (threads == 128)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_electron<HYB_FP32_SPLIT, 0, false, false, 128, 4>, 128,
                                                          smem);
        else if (threads == 512)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_electron<HYB_FP32_SPLIT, 0, false, false, 512, 4>, 512,
                                                          smem);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_electron<HYB_FP32_SPLIT, 0, false, false, 256, 4>, 256,
                                                          smem);
    } else if (precision == HYB_FP32_SPLIT && threads == 128)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_electron<HYB_FP32_SPLIT, 0, false, false, 128>, 128, smem);
    else if (precision == HYB_FP32_SPLIT && threads == 512)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_electron<HYB_FP32_SPLIT, 0, false, false, 512>, 512, smem);
    else if (precision == HYB_FP32_SPLIT)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_electron<HYB_FP32_SPLIT, 0>, kBlock, smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_electron<HYB_FP64, 0>, kBlock, smem);
    return n;
}

size_t electron_smem_bytes(int precision, int max_nodes, int eedf_bins, int threads, int n_xs)
{
    if (precision == HYB_FP32_SPLIT)  // EEDF histogram, one deposit row per warp, field and table
        return 4 * (size_t)(((eedf_bins + 2) + 3) & ~3) + sizeof(WarpRow) * (size_t)(threads / 32) +
               4 * (size_t)((max_nodes + 3) & ~3) + 32 * (size_t)n_xs + 16;
    const size_t el = 8;
    return 3 * el * (size_t)max_nodes + 4 * (size_t)(eedf_bins + 1) + 16;
}

cudaError_t launch_electron_step(InstDev *inst, int n_max, const int64_t *prefix, int precision, LaunchCfg cfg,
                                 cudaStream_t s, bool chem, bool kin)
{
    // the variants with the reactions of Sec. II.D beyond the neutral MCC
    // (recombination test, metastable source) and with ion births, when some
    // discharge of the batch needs them
    const bool sp = precision == HYB_FP32_SPLIT;
    if (chem && kin)
        return sp ? launch_k<HYB_FP32_SPLIT, 0, true, true>(inst, n_max, prefix, cfg, s)
                  : launch_k<HYB_FP64, 0, true, true>(inst, n_max, prefix, cfg, s);
    if (kin)
        return sp ? launch_k<HYB_FP32_SPLIT, 0, false, true>(inst, n_max, prefix, cfg, s)
                  : launch_k<HYB_FP64, 0, false, true>(inst, n_max, prefix, cfg, s);
    if (chem)
        return sp ? launch_k<HYB_FP32_SPLIT, 0, true>(inst, n_max, prefix, cfg, s)
                  : launch_k<HYB_FP64, 0, true>(inst, n_max, prefix, cfg, s);
    if (sp && cfg.ppt == 4) {
        if (cfg.block == 128) return launch_k<HYB_FP32_SPLIT, 0, false, false, 128, 4>(inst, n_max, prefix, cfg, s);
        if (cfg.block == 512) return launch_k<HYB_FP32_SPLIT, 0, false, false, 512, 4>(inst, n_max, prefix, cfg, s);
        return launch_k<HYB_FP32_SPLIT, 0, false, false, 256, 4>(inst, n_max, prefix, cfg, s);
    }
    if (sp && cfg.block == 128) return launch_k<HYB_FP32_SPLIT, 0, false, false, 128>(inst, n_max, prefix, cfg, s);
    if (sp && cfg.block == 512) return launch_k<HYB_FP32_SPLIT, 0, false, false, 512>(inst, n_max, prefix, cfg, s);
    return sp ? launch_k<HYB_FP32_SPLIT, 0>(inst, n_max, prefix, cfg, s) : launch_k<HYB_FP64, 0>(inst, n_max, prefix, cfg, s);
}

cudaError_t launch_deposit_init(InstDev *inst, int n_max, const int64_t *prefix, int precision, LaunchCfg cfg,
                                cudaStream_t s)
{
    return precision == HYB_FP32_SPLIT ? launch_k<HYB_FP32_SPLIT, 1>(inst, n_max, prefix, cfg, s)
                                       : launch_k<HYB_FP64, 1>(inst, n_max, prefix, cfg, s);
}

cudaError_t launch_load(InstDev *inst, int64_t n, double vth, int precision, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int grid = (int)((n + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    k_load<<<grid, 256, 0, s>>>(inst, n, vth, precision);
    return cudaGetLastError();
}

cudaError_t launch_prefix(InstDev *inst, int n_max, int64_t *prefix, cudaStream_t s)
{
    k_prefix<<<1, HYB_MAX_INSTANCES, 0, s>>>(inst, n_max, prefix);
    return cudaGetLastError();
}

cudaError_t launch_prefix_one(InstDev *inst, int64_t *prefix, cudaStream_t s)
{
    k_prefix_one<<<1, 32, 0, s>>>(inst, prefix);
    return cudaGetLastError();
}

cudaError_t launch_set_active(InstDev *inst, int active, int64_t target_step, cudaStream_t s)
{
    k_set_active<<<1, 32, 0, s>>>(inst, active, target_step);
    return cudaGetLastError();
}

}  // namespace hyb
