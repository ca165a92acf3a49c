// hyb_ion.cu -- the kinetic ions of the paper's fully kinetic comparison model
// (Sec. I and Sec. III): He+ macroparticles with the electrons' weight, in a
// second descriptor per discharge that shares the electrons' grids.  Each
// step, after the electron kernel has appended this step's ions (one per
// ionization): push in E^n (CIC gather, leapfrog), removal at the walls (their
// counts are the wall fluxes), CIC assignment of the ion density and flux,
// and collisions with the gas as in the auxiliary Monte Carlo of Sec. II.C:
// null collision against a neutral from the gas Maxwellian, acceptance on
// N Q_m(eps) g with Q_m = Q_i + 2 Q_b, isotropic scattering in the
// centre-of-mass frame (draw calls 5 and 6 at the step).
//
// Two layouts, as for the electrons: FP64 positions and velocities (the
// parity path, every formula in FP64), and the split mode's cell + FP32
// offset with FP32 velocities and FP32 collision arithmetic (fast
// log2/exp2 for the Q_b fit), which reads and writes 48 B per ion-step.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hyb_device.cuh"

namespace hyb {

namespace {

// N Q_m(eps) g for He+ on He; eps = M_r g^2 / 2 in eV
__device__ __forceinline__ double ion_nu(double ngas, double m_red, double g)
{
    if (!(g > 0.0)) return ngas * 7.63e-20 * sqrt(2.0 * kQe / m_red);
    const double eps = 0.5 * m_red * g * g / kQe;
    double q = 7.63e-20 / sqrt(eps);
    q += 2.0 * (1e-19 / (pow(eps / 1000.0, 0.15) * pow(1.0 + eps / 1000.0, 0.25) * pow(1.0 + 5.0 / eps, 0.15)));
    return ngas * q * g;
}

// ions [a, b) of ion descriptor I; ctr: losses at z = 0, at z = L,
// collision candidates, real collisions, pushes.  MODE 1: charge assignment only.
template <int MODE>
__device__ void segment_ion_fp64(InstDev *I, int64_t a, int64_t b, unsigned char *smem, unsigned ctr[5])
{
    InstDev *K = I->elec;
    const int G = K->G, nc = K->n_cells;
    const double dz = K->dz, dt = K->dt, L = K->L;
    const double *__restrict__ E = K->E;
    const uint32_t step = (uint32_t)K->step;
    const uint32_t sl = K->seed_lo, sh = K->seed_hi;
    const double M = K->m_ion, mn = K->m_gas, ngas = K->ngas, mr = K->mi_red;
    const double numax = K->nu_max_i, pmax = K->p_max_i, vt = K->vt_gas;
    const PartBuf P = I->buf[I->cur];
    double *sd_n = reinterpret_cast<double *>(smem);
    double *sd_g = sd_n + G;
    if (!HYB_CHECK(b <= I->capacity && a >= 0, 14, b, I->capacity)) b = a;
    for (int j = threadIdx.x; j < 2 * G; j += blockDim.x) sd_n[j] = 0.0;
    __syncthreads();
    for (int64_t base = a; base < b; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        double z = i < b ? P.z[i] : -1.0;
        bool alive = z >= 0.0 && z < L;
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
            ++ctr[4];
            locate_d(z, dz, nc, c, o);
            const double ep = (1.0 - o) * E[c] + o * E[c + 1];
            vz = vz + (kQe / M) * ep * dt;
            z = z + vz * dt;
            if (!(z >= 0.0 && z < L)) {
                ctr[0] += z < 0.0 ? 1u : 0u;
                ctr[1] += z < 0.0 ? 0u : 1u;
                alive = false;
                P.z[i] = -1.0;
            }
        }
        if (alive) locate_d(z, dz, nc, c, o);
        deposit_pair<double>(sd_n, alive, c, 1.0 - o, o, G);
        deposit_pair<double>(sd_g, alive, c, (1.0 - o) * vz, o * vz, G);
        if (MODE == 0 && alive) {
            const uint4 u = draw(id, step, sl, sh, 5);
            if (u01d(u.x) < pmax) {
                ++ctr[2];
                const uint4 w = draw(id, step, sl, sh, 6);
                double b1, b2, b3, b4;
                gauss_pair(u01d(u.z), u01d(u.w), b1, b2);
                gauss_pair(u01d(w.x), u01d(w.y), b3, b4);
                const double Vx = vt * b1, Vy = vt * b2, Vz = vt * b3;
                const double gx = vx - Vx, gy = vy - Vy, gz = vz - Vz;
                const double g = sqrt(gx * gx + gy * gy + gz * gz);
                if (u01d(u.y) * numax < ion_nu(ngas, mr, g)) {
                    ++ctr[3];
                    double d[3];
                    iso_dir_d(u01d(w.z), u01d(w.w), d);
                    vx = (M * vx + mn * Vx) / (M + mn) + mn / (M + mn) * g * d[0];
                    vy = (M * vy + mn * Vy) / (M + mn) + mn / (M + mn) * g * d[1];
                    vz = (M * vz + mn * Vz) / (M + mn) + mn / (M + mn) * g * d[2];
                }
            }
            P.z[i] = z;
            P.vxd[i] = vx;
            P.vyd[i] = vy;
            P.vzd[i] = vz;
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < G; j += blockDim.x) {
        if (sd_n[j] != 0.0) atomicAdd(&K->dep_ni[j], sd_n[j]);
        if (sd_g[j] != 0.0) atomicAdd(&K->dep_gi[j], sd_g[j]);
    }
    __syncthreads();
}

// N Q_m(eps) g in FP32: Q_i = 7.63e-20 / sqrt(eps), Q_b = 1e-19 / ((eps/1000)^0.15
// (1 + eps/1000)^0.25 (1 + 5/eps)^0.15) with eps = M_r g^2 / 2 in eV, the powers
// through one exp2 of a sum of log2s
__device__ __forceinline__ float ion_nu_f(const InstDev *K, float g)
{
    if (!(g > 0.f)) return K->fi_nu0;
    const float eps = K->fi_half_mr_q * g * g;
    const float x = eps * 1e-3f;
    const float l = 0.15f * __log2f(x) + 0.25f * __log2f(1.f + x) + 0.15f * __log2f(1.f + __fdividef(5.f, eps));
    const float q = 7.63e-20f * rsqrtf(eps) + 2e-19f * exp2f(-l);
    return K->fi_ngas * q * g;
}

// CIC of two values per lane into the FP64 global sums: value v_k of the
// lane's ion k (k = 0, 1; ion k in cell c_k with offset o_k) adds (1 - o_k) v_k
// to node c_k and o_k v_k to node c_k + 1.  When the warp's live ions lie in
// one cell or two neighbouring ones (the usual case, ions being sorted by cell
// and barely moving between sorts) the three touched nodes are summed over the
// warp in FP32 and lane 0 adds them; otherwise every lane adds its own.  (A
// block-private FP32 row in shared memory was slower: a shared-memory FP32
// atomic add is a compare-and-swap loop, and the block's warps, in step over
// neighbouring ions, contended on the same nodes.)
__device__ __forceinline__ void deposit_two(double *arr, const bool on[2], const int c[2], const float o[2],
                                            const float v[2], int G)
{
    bool ok[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) ok[k] = on[k] && HYB_CHECK(c[k] >= 0 && c[k] + 1 < G, 4, c[k], G);
    const int lo = min(ok[0] ? c[0] : INT32_MAX, ok[1] ? c[1] : INT32_MAX);
    const int hi = max(ok[0] ? c[0] : -1, ok[1] ? c[1] : -1);
    const int kmin = __reduce_min_sync(kFull, lo);
    const int kmax = __reduce_max_sync(kFull, hi);
    if (kmax < 0) return;
    if (kmax - kmin <= 1) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;  // nodes kmin, kmin + 1, kmin + 2
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (!ok[k]) continue;
            const float a = (1.f - o[k]) * v[k], b = o[k] * v[k];
            if (c[k] == kmin) {
                s0 += a;
                s1 += b;
            } else {
                s1 += a;
                s2 += b;
            }
        }
        s0 = WarpSum<float>::run(s0);
        s1 = WarpSum<float>::run(s1);
        if (kmax > kmin) s2 = WarpSum<float>::run(s2);
        if ((threadIdx.x & 31) == 0) {
            if (s0 != 0.f) atomicAdd(&arr[kmin], (double)s0);
            if (s1 != 0.f) atomicAdd(&arr[kmin + 1], (double)s1);
            if (kmax > kmin && s2 != 0.f) atomicAdd(&arr[kmin + 2], (double)s2);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (ok[k]) {
                atomicAdd(&arr[c[k]], (double)((1.f - o[k]) * v[k]));
                atomicAdd(&arr[c[k] + 1], (double)(o[k] * v[k]));
            }
    }
}

// split-mode ions [a, b): cell + FP32 offset, FP32 velocities, two ions per
// thread (8- and 16-byte vector accesses; a is a multiple of the chunk size, so
// the pair is aligned) whose Philox chains and pushes interleave, each warp
// sweeping its own contiguous part of [a, b); the ion density and flux go to
// the FP64 global sums (summed per warp when the lanes share a cell)
template <int MODE>
__device__ void segment_ion_split(InstDev *I, int64_t a, int64_t b, unsigned ctr[5])
{
    InstDev *K = I->elec;
    const int G = K->G, nc = K->n_cells;
    const float *__restrict__ Ef = K->Ef;
    const uint32_t step = (uint32_t)K->step;
    const uint32_t sl = K->seed_lo, sh = K->seed_hi;
    const float qm_dt = K->fi_qm_dt, dt_dz = K->f_dt_dz;
    const float numax = K->fi_numax, pmax = K->fi_pmax, vt = K->fi_vt, ca = K->fi_cm_a, cb = K->fi_cm_b;
    const PartBuf P = I->buf[I->cur];
    double *dep_n = K->dep_ni, *dep_g = K->dep_gi;
    if (!HYB_CHECK(b <= I->capacity && a >= 0 && (a & 1) == 0, 14, b, I->capacity)) b = a;
    const PhiloxPre pre = philox_pre(step, sl, sh);
    const int nwarps = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t per = (((b - a) + nwarps - 1) / nwarps + 63) / 64 * 64;
    const int64_t wa = a + per * wid;
    const int64_t wb = wa + per < b ? wa + per : b;
    for (int64_t base = wa; base < wb; base += 64) {
        const int64_t i0 = base + 2 * (int64_t)lane;
        const bool full = i0 + 1 < wb;
        int c[2];
        float o[2], vx[2], vy[2], vz[2];
        uint64_t id[2];
        if (full) {  // streaming (evict-first) accesses, as the electron kernel
            const int2 c2 = __ldcs(reinterpret_cast<const int2 *>(P.c + i0));
            const float2 o2 = __ldcs(reinterpret_cast<const float2 *>(P.o + i0));
            const float2 x2 = __ldcs(reinterpret_cast<const float2 *>(P.vxf + i0));
            const float2 y2 = __ldcs(reinterpret_cast<const float2 *>(P.vyf + i0));
            const float2 z2 = __ldcs(reinterpret_cast<const float2 *>(P.vzf + i0));
            c[0] = c2.x, c[1] = c2.y, o[0] = o2.x, o[1] = o2.y;
            vx[0] = x2.x, vx[1] = x2.y, vy[0] = y2.x, vy[1] = y2.y, vz[0] = z2.x, vz[1] = z2.y;
            if (MODE == 0) {
                const ulonglong2 d2 = __ldcs(reinterpret_cast<const ulonglong2 *>(P.id + i0));
                id[0] = d2.x, id[1] = d2.y;
            } else {
                id[0] = id[1] = 0ull;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const bool in = i0 + k < wb;
                c[k] = in ? P.c[i0 + k] : kDeadCell;
                o[k] = in ? P.o[i0 + k] : 0.f;
                vx[k] = in ? P.vxf[i0 + k] : 0.f;
                vy[k] = in ? P.vyf[i0 + k] : 0.f;
                vz[k] = in ? P.vzf[i0 + k] : 0.f;
                id[k] = (MODE == 0 && in) ? P.id[i0 + k] : 0ull;
            }
        }
        bool alive[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            alive[k] = c[k] >= 0 && c[k] < nc;
            if (MODE == 0 && alive[k]) {
                ++ctr[4];
                const float ep = (1.f - o[k]) * __ldg(&Ef[c[k]]) + o[k] * __ldg(&Ef[c[k] + 1]);
                vz[k] = vz[k] + qm_dt * ep;
                float on = o[k] + vz[k] * dt_dz;
                const float fl = floorf(on);
                int cn = c[k] + (int)fl;
                on -= fl;
                if (on >= 1.f) {
                    on -= 1.f;
                    cn += 1;
                }
                if (cn < 0 || cn >= nc) {  // absorbed by an electrode and removed
                    ctr[0] += cn < 0 ? 1u : 0u;
                    ctr[1] += cn < 0 ? 0u : 1u;
                    alive[k] = false;
                    c[k] = kDeadCell;
                } else {
                    c[k] = cn;
                    o[k] = on;
                }
            }
        }
        const float one[2] = {1.f, 1.f};
        deposit_two(dep_n, alive, c, o, one, G);
        deposit_two(dep_g, alive, c, o, vz, G);
        if (MODE == 0) {
            uint4 u[2];
            draw_n<2>(pre, id, 5u, u);
            // collision candidates (R < P_max), then one warp pass per
            // candidate a lane holds: the lanes' candidates are handled
            // together instead of one slot after the other
            unsigned cand = 0u;
#pragma unroll
            for (int k = 0; k < 2; ++k) cand |= (alive[k] && u01f(u[k].x) < pmax) ? (1u << k) : 0u;
            ctr[2] += __popc(cand);
            while (__any_sync(kFull, cand != 0u)) {
                if (cand) {
                    const int k = (cand & 1u) ? 0 : 1;
                    cand &= cand - 1u;
                    const uint4 uk = k ? u[1] : u[0];
                    const float px = k ? vx[1] : vx[0], py = k ? vy[1] : vy[0], pz = k ? vz[1] : vz[0];
                    const uint4 w = draw_pre(pre, k ? id[1] : id[0], 6u);
                    // neutral from the gas Maxwellian (Box-Muller), as the FP64 path
                    float s1, c1;
                    const float r1 = sqrtf(-2.f * __logf(u01f(uk.z)));
                    __sincosf(6.283185307179586f * u01f(uk.w), &s1, &c1);
                    const float r2 = sqrtf(-2.f * __logf(u01f(w.x)));
                    const float Vx = vt * (r1 * c1), Vy = vt * (r1 * s1);
                    const float Vz = vt * (r2 * __cosf(6.283185307179586f * u01f(w.y)));
                    const float gx = px - Vx, gy = py - Vy, gz = pz - Vz;
                    const float g = sqrtf(gx * gx + gy * gy + gz * gz);
                    if (u01f(uk.y) * numax < ion_nu_f(K, g)) {
                        ++ctr[3];
                        const float ct = 1.f - 2.f * u01f(w.z);
                        const float st = sqrtf(fmaxf(0.f, 1.f - ct * ct));
                        float sp, cp;
                        __sincosf(6.283185307179586f * u01f(w.w), &sp, &cp);
                        const float cg = cb * g;
                        const float nx = ca * px + cb * Vx + cg * (st * cp);
                        const float ny = ca * py + cb * Vy + cg * (st * sp);
                        const float nz = ca * pz + cb * Vz + cg * ct;
                        if (k) {
                            vx[1] = nx, vy[1] = ny, vz[1] = nz;
                        } else {
                            vx[0] = nx, vy[0] = ny, vz[0] = nz;
                        }
                    }
                }
            }
            if (full) {
                __stcs(reinterpret_cast<int2 *>(P.c + i0), make_int2(c[0], c[1]));
                __stcs(reinterpret_cast<float2 *>(P.o + i0), make_float2(o[0], o[1]));
                __stcs(reinterpret_cast<float2 *>(P.vxf + i0), make_float2(vx[0], vx[1]));
                __stcs(reinterpret_cast<float2 *>(P.vyf + i0), make_float2(vy[0], vy[1]));
                __stcs(reinterpret_cast<float2 *>(P.vzf + i0), make_float2(vz[0], vz[1]));
            } else {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (i0 + k < wb) {
                        P.c[i0 + k] = c[k];
                        P.o[i0 + k] = o[k];
                        P.vxf[i0 + k] = vx[k];
                        P.vyf[i0 + k] = vy[k];
                        P.vzf[i0 + k] = vz[k];
                    }
                }
            }
        }
    }
}

template <int PREC, int MODE>
__global__ void __launch_bounds__(kBlock, PREC == HYB_FP32_SPLIT ? 3 : 2) k_ion(InstDev *__restrict__ ions, int n_max, const int64_t *__restrict__ prefix)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned s_c[5];
    for_block_runs(ions, n_max, prefix, [&](InstDev *I, int64_t a, int64_t b) {
        unsigned ctr[5] = {0u, 0u, 0u, 0u, 0u};
        if (threadIdx.x < 5) s_c[threadIdx.x] = 0u;
        if (PREC == HYB_FP32_SPLIT)
            segment_ion_split<MODE>(I, a, b, ctr);
        else
            segment_ion_fp64<MODE>(I, a, b, smem, ctr);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const unsigned t = __reduce_add_sync(kFull, ctr[k]);
            if ((threadIdx.x & 31) == 0 && t) atomicAdd(&s_c[k], t);
        }
        __syncthreads();
        if (threadIdx.x == 0 && MODE == 0) {
            const int map[5] = {C_LOSS0, C_LOSS1, C_NULL, C_EL, C_PUSH};
#pragma unroll
            for (int k = 0; k < 5; ++k)
                if (s_c[k]) atomicAdd(&I->ctr[map[k]], (unsigned long long)s_c[k]);
        }
        __syncthreads();
    });
}

// ions 0..n-1 of a discharge: ids 2^61 + i, uniform in [0, L), gas
// Maxwellian; draws at step 0xFFFFFFFF, calls 4 and 5 (FP64 arithmetic in both
// layouts; the split layout stores the cell, offset and FP32 velocities)
__global__ void k_load_ions(InstDev *I, int64_t n)
{
    const PartBuf P = I->buf[I->cur];
    if (!HYB_CHECK(n <= I->capacity, 9, n, I->capacity)) return;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t id = (1ull << 61) + (uint64_t)j;
        const uint4 a = draw(id, 0xFFFFFFFFu, I->seed_lo, I->seed_hi, 4);
        const uint4 b = draw(id, 0xFFFFFFFFu, I->seed_lo, I->seed_hi, 5);
        double g1, g2, g3, g4;
        gauss_pair(u01d(a.y), u01d(a.z), g1, g2);
        gauss_pair(u01d(b.x), u01d(b.y), g3, g4);
        const double z = u01d(a.x) * I->L;
        P.id[j] = id;
        if (I->precision == HYB_FP32_SPLIT) {
            int c;
            double o;
            locate_d(z, I->dz, I->n_cells, c, o);
            P.c[j] = c;
            P.o[j] = (float)o;
            P.vxf[j] = (float)(I->vt_gas * g1);
            P.vyf[j] = (float)(I->vt_gas * g2);
            P.vzf[j] = (float)(I->vt_gas * g3);
        } else {
            P.z[j] = z;
            P.vxd[j] = I->vt_gas * g1;
            P.vyd[j] = I->vt_gas * g2;
            P.vzd[j] = I->vt_gas * g3;
        }
    }
}

// the ions to step now are all slots in use (including this step's births),
// and an ion descriptor runs while its discharge does
__global__ void __launch_bounds__(HYB_MAX_INSTANCES) k_ion_prefix(InstDev *ions, int n_max, int64_t *prefix)
{
    __shared__ int64_t s_buf[HYB_MAX_INSTANCES];
    const int t = threadIdx.x;
    if (t < n_max) {
        InstDev *I = &ions[t];
        if (I->elec) {
            I->active = I->elec->active;
            const int64_t n = (int64_t)I->n_slots;
            I->n_slots_step = n < I->capacity ? n : I->capacity;
        } else {
            I->active = 0;
        }
    }
    __syncthreads();
    block_chunk_prefix(ions, n_max, prefix, s_buf);
}

}  // namespace

void read_checks_ion(unsigned long long out[3])
{
    if (cudaMemcpyFromSymbol(out, g_hyb_check, sizeof(unsigned long long) * 3) != cudaSuccess)
        out[0] = out[1] = out[2] = 0ull;
}

void configure_ion_kernels()
{
    allow_max_dynamic_smem(k_ion<HYB_FP64, 0>);
    allow_max_dynamic_smem(k_ion<HYB_FP64, 1>);
    allow_max_dynamic_smem(k_ion<HYB_FP32_SPLIT, 0>);
    allow_max_dynamic_smem(k_ion<HYB_FP32_SPLIT, 1>);
}

cudaError_t launch_load_ions(InstDev *ion, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int grid = (int)((n + 255) / 256);
    if (grid > 4096) grid = 4096;
    k_load_ions<<<grid, 256, 0, s>>>(ion, n);
    return cudaGetLastError();
}

cudaError_t launch_ion_prefix(InstDev *ions, int n_max, int64_t *prefix, cudaStream_t s)
{
    k_ion_prefix<<<1, HYB_MAX_INSTANCES, 0, s>>>(ions, n_max, prefix);
    return cudaGetLastError();
}

cudaError_t launch_ion_step(InstDev *ions, int n_max, const int64_t *prefix, int mode, int grid, int max_nodes,
                            int precision, cudaStream_t s)
{
    if (precision == HYB_FP32_SPLIT) {  // no shared rows: the deposit goes to the global sums
        if (mode == 0)
            k_ion<HYB_FP32_SPLIT, 0><<<grid, kBlock, 0, s>>>(ions, n_max, prefix);
        else
            k_ion<HYB_FP32_SPLIT, 1><<<grid, kBlock, 0, s>>>(ions, n_max, prefix);
    } else {
        const size_t smem = 16 * (size_t)max_nodes;
        if (mode == 0)
            k_ion<HYB_FP64, 0><<<grid, kBlock, smem, s>>>(ions, n_max, prefix);
        else
            k_ion<HYB_FP64, 1><<<grid, kBlock, smem, s>>>(ions, n_max, prefix);
    }
    return cudaGetLastError();
}

}  // namespace hyb
