// hyb_sort.cu -- the periodic cell sort of the particle stores (electrons and
// kinetic ions): a counting sort by cell every K steps that removes the dead
// slots (particles absorbed at the walls, recombined), folds the births
// appended since the last sort into cell order, and restores the cell
// locality the deposit rows of the particle steps rely on (Sec. II.A: removal
// at the walls; the order itself is free, every draw being a function of the
// particle id, not of its slot).
//
// Four launches over a lane's instances: count, an exclusive scan of the
// counts per instance, scatter into the other buffer of the double-buffered
// store, and a finish that flips the buffers and sets the slot counts; then
// the chunk prefix of the next step.  Count and scatter take the block's run
// of slots in tiles of four consecutive slots per thread (one 16-byte load per
// array): a tile counts its cells in shared memory (one shared atomic per run
// of equal cells a thread holds) and makes one global atomic per cell it
// holds, which in the scatter returns the tile's first destination in that
// cell; a slot's destination is that plus its rank within the tile.  (The
// store is sorted at the previous sort and drifts by a few cells between
// sorts, so a tile holds a few cells: the global atomics on the per-cell
// counters, which every warp of a neighbourhood used to contend for, drop
// from one or more per 32 slots to a few per 1024.)
#include <cuda_runtime.h>
#include <stdint.h>

#include "hyb_device.cuh"

namespace hyb {

namespace {

constexpr int kSortE = 4;  // consecutive slots per thread in a tile

// four consecutive values from a slot index that is a multiple of four (16-byte
// aligned for 4-byte values, two 16-byte loads for 8-byte ones), streaming
__device__ __forceinline__ void ld4(const int32_t *p, int32_t (&v)[4])
{
    const int4 u = __ldcs(reinterpret_cast<const int4 *>(p));
    v[0] = u.x, v[1] = u.y, v[2] = u.z, v[3] = u.w;
}
__device__ __forceinline__ void ld4(const float *p, float (&v)[4])
{
    const float4 u = __ldcs(reinterpret_cast<const float4 *>(p));
    v[0] = u.x, v[1] = u.y, v[2] = u.z, v[3] = u.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&v)[4])
{
    const double2 u = __ldcs(reinterpret_cast<const double2 *>(p));
    const double2 w = __ldcs(reinterpret_cast<const double2 *>(p + 2));
    v[0] = u.x, v[1] = u.y, v[2] = w.x, v[3] = w.y;
}
__device__ __forceinline__ void ld4(const uint64_t *p, uint64_t (&v)[4])
{
    const ulonglong2 u = __ldcs(reinterpret_cast<const ulonglong2 *>(p));
    const ulonglong2 w = __ldcs(reinterpret_cast<const ulonglong2 *>(p + 2));
    v[0] = u.x, v[1] = u.y, v[2] = w.x, v[3] = w.y;
}
// the first n (< 4) of them, the rest `fill`
template <typename T>
__device__ __forceinline__ void ld4_part(const T *p, int n, T (&v)[4], T fill)
{
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = j < n ? __ldcs(p + j) : fill;
}
template <typename T>
__device__ __forceinline__ void ld4_any(const T *p, int n, T (&v)[4], T fill)
{
    if (n >= 4)
        ld4(p, v);
    else
        ld4_part(p, n, v, fill);
}

// What a tile moves: the particle state of the store's layout.
template <int PREC>
struct SortTile;

template <>
struct SortTile<HYB_FP32_SPLIT> {
    int32_t c[kSortE];
    float o[kSortE], vx[kSortE], vy[kSortE], vz[kSortE];
    uint64_t id[kSortE];
    __device__ void load_cells(const PartBuf &S, int64_t i, int n, double, int, bool (&al)[kSortE])
    {
        ld4_any(S.c + i, n, c, kDeadCell);
#pragma unroll
        for (int j = 0; j < kSortE; ++j) al[j] = c[j] >= 0;
    }
    __device__ void load_rest(const PartBuf &S, int64_t i, int n)
    {
        ld4_any(S.o + i, n, o, 0.f);
        ld4_any(S.vxf + i, n, vx, 0.f);
        ld4_any(S.vyf + i, n, vy, 0.f);
        ld4_any(S.vzf + i, n, vz, 0.f);
        ld4_any(S.id + i, n, id, (uint64_t)0);
    }
    __device__ void store(const PartBuf &D, int j, int64_t pos) const
    {
        __stcs(&D.id[pos], id[j]);
        __stcs(&D.c[pos], c[j]);
        __stcs(&D.o[pos], o[j]);
        __stcs(&D.vxf[pos], vx[j]);
        __stcs(&D.vyf[pos], vy[j]);
        __stcs(&D.vzf[pos], vz[j]);
    }
};

template <>
struct SortTile<HYB_FP64> {
    int32_t c[kSortE];
    double z[kSortE], vx[kSortE], vy[kSortE], vz[kSortE];
    uint64_t id[kSortE];
    __device__ void load_cells(const PartBuf &S, int64_t i, int n, double dz, int nc, bool (&al)[kSortE])
    {
        ld4_any(S.z + i, n, z, -1.0);
#pragma unroll
        for (int j = 0; j < kSortE; ++j) {
            al[j] = z[j] >= 0.0;
            double o;
            locate_d(al[j] ? z[j] : 0.0, dz, nc, c[j], o);
        }
    }
    __device__ void load_rest(const PartBuf &S, int64_t i, int n)
    {
        ld4_any(S.vxd + i, n, vx, 0.0);
        ld4_any(S.vyd + i, n, vy, 0.0);
        ld4_any(S.vzd + i, n, vz, 0.0);
        ld4_any(S.id + i, n, id, (uint64_t)0);
    }
    __device__ void store(const PartBuf &D, int j, int64_t pos) const
    {
        __stcs(&D.id[pos], id[j]);
        __stcs(&D.z[pos], z[j]);
        __stcs(&D.vxd[pos], vx[j]);
        __stcs(&D.vyd[pos], vy[j]);
        __stcs(&D.vzd[pos], vz[j]);
    }
};

template <int PREC, int PHASE>  // PHASE 0: count, 1: scatter
__global__ void __launch_bounds__(kBlock) k_sort_pass(InstDev *__restrict__ insts, int n_max,
                                                      const int64_t *__restrict__ prefix)
{
    // by cell: the tile's counts, then (scatter) its first destinations; only
    // the tile's span of cells is cleared and read
    __shared__ int32_t s_cnt[kMaxNodes];
    __shared__ int32_t s_wlo[kBlock / 32], s_whi[kBlock / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for_block_runs(insts, n_max, prefix, [&](InstDev *K, int64_t a, int64_t b) {
        const PartBuf S = K->buf[K->cur];
        const PartBuf D = K->buf[K->cur ^ 1];
        const int64_t capacity = K->capacity;
        const int nc = K->n_cells;
        // block-uniform checks (a has the alignment of a chunk start)
        if (!HYB_CHECK(b <= capacity && nc < kMaxNodes && (a & (kSortE - 1)) == 0, 11, b, capacity)) return;
        int32_t *cnt = K->cell_cnt;
        const double dz = K->dz;
        for (int64_t t0 = a; t0 < b; t0 += (int64_t)kSortE * blockDim.x) {
            const int64_t i0 = t0 + (int64_t)kSortE * threadIdx.x;
            const int n = i0 < b ? (int)(b - i0 < kSortE ? b - i0 : kSortE) : 0;
            SortTile<PREC> T;
            bool al[kSortE];
            T.load_cells(S, i0, n, dz, nc, al);
            if (PHASE == 1) T.load_rest(S, i0, n);  // in flight while the tile's counts form
            int lo = INT32_MAX, hi = -1;
#pragma unroll
            for (int j = 0; j < kSortE; ++j) {
                if (al[j] && !HYB_CHECK(T.c[j] < nc, 7, T.c[j], nc)) al[j] = false;
                lo = al[j] && T.c[j] < lo ? T.c[j] : lo;
                hi = al[j] && T.c[j] > hi ? T.c[j] : hi;
            }
            lo = __reduce_min_sync(kFull, lo);
            hi = __reduce_max_sync(kFull, hi);
            __syncthreads();  // the previous tile is done with s_cnt and the spans
            if (lane == 0) s_wlo[wid] = lo, s_whi[wid] = hi;
            __syncthreads();
            int tlo = s_wlo[0], thi = s_whi[0];
            for (int w = 1; w < nw; ++w) {
                tlo = s_wlo[w] < tlo ? s_wlo[w] : tlo;
                thi = s_whi[w] > thi ? s_whi[w] : thi;
            }
            if (thi >= tlo)
                for (int d = tlo + (int)threadIdx.x; d <= thi; d += blockDim.x) s_cnt[d] = 0;
            __syncthreads();
            // runs of equal cells among the thread's slots: one shared add per
            // run, which returns the run's rank within the tile's cell
            int rank[kSortE];
            int run_off = 0, run_start = 0;
#pragma unroll
            for (int j = 0; j < kSortE; ++j) {
                rank[j] = 0;
                if (!al[j]) continue;
                if (j == 0 || !al[j - 1] || T.c[j] != T.c[j - 1]) {
                    int len = 1;
                    bool go = true;
#pragma unroll
                    for (int q = j + 1; q < kSortE; ++q) {
                        go = go && al[q] && T.c[q] == T.c[j];
                        len += go ? 1 : 0;
                    }
                    if (PHASE == 0)
                        atomicAdd(&s_cnt[T.c[j]], len);
                    else
                        run_off = atomicAdd(&s_cnt[T.c[j]], len);
                    run_start = j;
                }
                rank[j] = run_off + (j - run_start);
            }
            __syncthreads();
            // one global atomic per cell of the tile; in the scatter it turns
            // the tile's count into the tile's first destination in that cell
            if (thi >= tlo) {
                for (int d = tlo + (int)threadIdx.x; d <= thi; d += blockDim.x) {
                    const int v = s_cnt[d];
                    if (PHASE == 0) {
                        if (v) atomicAdd(&cnt[d], v);
                    } else {
                        s_cnt[d] = v ? atomicAdd(&cnt[d], v) : 0;
                    }
                }
            }
            if (PHASE == 1) {
                __syncthreads();
#pragma unroll
                for (int j = 0; j < kSortE; ++j) {
                    if (!al[j]) continue;
                    const int64_t pos = (int64_t)s_cnt[T.c[j]] + rank[j];
                    if (!HYB_CHECK(pos >= 0 && pos < capacity, 8, pos, capacity)) continue;
                    T.store(D, j, pos);
                }
            }
        }
    });
}

// Exclusive scan of the cell counts, one CTA per sorted instance; the total
// goes to cell_cnt[n_cells].
__global__ void __launch_bounds__(1024) k_sort_scan(InstDev *insts, const int64_t *prefix)
{
    InstDev *K = &insts[blockIdx.x];
    if (prefix[blockIdx.x + 1] == prefix[blockIdx.x]) return;
    int32_t *cnt = K->cell_cnt;
    const int nc = K->n_cells;
    __shared__ int32_t s_warp[32];
    __shared__ int32_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < nc; base += blockDim.x) {
        const int j = base + threadIdx.x;
        const int32_t v = j < nc ? cnt[j] : 0;
        int32_t x = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, x, d);
            if ((threadIdx.x & 31) >= d) x += y;
        }
        if ((threadIdx.x & 31) == 31) s_warp[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            int32_t w = threadIdx.x < (blockDim.x >> 5) ? s_warp[threadIdx.x] : 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t y = __shfl_up_sync(kFull, w, d);
                if ((int)threadIdx.x >= d) w += y;
            }
            s_warp[threadIdx.x] = w;
        }
        __syncthreads();
        const int32_t warp_off = (threadIdx.x >> 5) ? s_warp[(threadIdx.x >> 5) - 1] : 0;
        const int32_t carry = s_carry;
        if (j < nc) cnt[j] = carry + warp_off + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = carry + warp_off + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) cnt[nc] = s_carry;
}

// After the scatter: flip the buffers, set the slot counts, clear the counts.
__global__ void k_sort_finish(InstDev *insts, const int64_t *prefix)
{
    InstDev *K = &insts[blockIdx.x];
    if (prefix[blockIdx.x + 1] == prefix[blockIdx.x]) return;
    __shared__ int32_t total;
    if (threadIdx.x == 0) total = K->cell_cnt[K->n_cells];
    __syncthreads();
    for (int j = threadIdx.x; j <= K->n_cells; j += blockDim.x) K->cell_cnt[j] = 0;
    if (threadIdx.x == 0) {
        K->cur ^= 1;
        K->n_slots = (unsigned long long)total;
        K->n_slots_step = total;
    }
}

}  // namespace

void read_checks_sort(unsigned long long out[3])
{
    if (cudaMemcpyFromSymbol(out, g_hyb_check, sizeof(unsigned long long) * 3) != cudaSuccess)
        out[0] = out[1] = out[2] = 0ull;
}

cudaError_t launch_sort(InstDev *inst, int n_max, int64_t *prefix, int precision, LaunchCfg cfg, cudaStream_t s)
{
    if (precision == HYB_FP32_SPLIT) {
        k_sort_pass<HYB_FP32_SPLIT, 0><<<cfg.grid, kBlock, 0, s>>>(inst, n_max, prefix);
    } else {
        k_sort_pass<HYB_FP64, 0><<<cfg.grid, kBlock, 0, s>>>(inst, n_max, prefix);
    }
    k_sort_scan<<<n_max, 1024, 0, s>>>(inst, prefix);
    if (precision == HYB_FP32_SPLIT) {
        k_sort_pass<HYB_FP32_SPLIT, 1><<<cfg.grid, kBlock, 0, s>>>(inst, n_max, prefix);
    } else {
        k_sort_pass<HYB_FP64, 1><<<cfg.grid, kBlock, 0, s>>>(inst, n_max, prefix);
    }
    k_sort_finish<<<n_max, 256, 0, s>>>(inst, prefix);
    const cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : launch_prefix(inst, n_max, prefix, s);
}

}  // namespace hyb
