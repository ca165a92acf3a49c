// hyb_sort.cu -- the periodic cell sort of the particle stores (electrons and
// kinetic ions): a counting sort by cell every K steps that removes the dead
// slots (particles absorbed at the walls, recombined), folds the births
// appended since the last sort into cell order, and restores the cell
// locality the deposit rows of the particle steps rely on (Sec. II.A: removal
// at the walls; the order itself is free, every draw being keyed by particle
// id).
//
// Four launches over a lane's instances: count (one atomic per cell a warp
// holds), an exclusive scan of the counts per instance, scatter into the other
// buffer of the double-buffered store (one atomic per cell a warp holds, which
// returns the group's first destination), and a finish that flips the buffers
// and sets the slot counts; then the chunk prefix of the next step.  (Runs of
// equal cells found with a shuffle and a ballot instead of the lanes grouped by
// cell with match_any: 6 % slower, more atomics once the order has drifted.)
#include <cuda_runtime.h>
#include <stdint.h>

#include "hyb_device.cuh"

namespace hyb {

namespace {

template <int PREC>
__device__ __forceinline__ bool cell_of(const PartBuf &P, int64_t i, double dz, int nc, int &c)
{
    if (PREC == HYB_FP32_SPLIT) {
        c = P.c[i];
        return c >= 0;
    }
    const double z = P.z[i];
    if (z < 0.0) return false;
    double o;
    locate_d(z, dz, nc, c, o);
    return true;
}

template <int PREC, int PHASE>  // PHASE 0: count, 1: scatter
__global__ void __launch_bounds__(kBlock) k_sort_pass(InstDev *__restrict__ insts, int n_max,
                                                      const int64_t *__restrict__ prefix)
{
    const int lane = threadIdx.x & 31;
    for_block_runs(insts, n_max, prefix, [&](InstDev *K, int64_t a, int64_t b) {
        const PartBuf S = K->buf[K->cur];
        const PartBuf D = K->buf[K->cur ^ 1];
        if (!HYB_CHECK(b <= K->capacity, 11, b, K->capacity)) return;
        int32_t *cnt = K->cell_cnt;
        const double dz = K->dz;
        const int nc = K->n_cells;
        for (int64_t base = a; base < b; base += blockDim.x) {
            const int64_t i = base + threadIdx.x;
            int c = -1;
            bool alive = i < b && cell_of<PREC>(S, i, dz, nc, c);
            if (alive && !HYB_CHECK(c < nc, 7, c, nc)) alive = false;
            const unsigned act = __ballot_sync(kFull, alive);
            if (!alive) continue;
            const unsigned peers = __match_any_sync(act, c);
            const int leader = __ffs(peers) - 1;
            int pos = 0;
            if (lane == leader) pos = atomicAdd(&cnt[c], __popc(peers));
            if (PHASE == 1) {
                pos = __shfl_sync(peers, pos, leader) + __popc(peers & lanemask_lt());
                if (!HYB_CHECK(pos >= 0 && pos < K->capacity, 8, pos, K->capacity)) continue;
                // streaming (evict-first) accesses: the particle state is read
                // and written once, and should not displace the tables
                __stcs(&D.id[pos], __ldcs(&S.id[i]));
                if (PREC == HYB_FP32_SPLIT) {
                    __stcs(&D.c[pos], c);
                    __stcs(&D.o[pos], __ldcs(&S.o[i]));
                    __stcs(&D.vxf[pos], __ldcs(&S.vxf[i]));
                    __stcs(&D.vyf[pos], __ldcs(&S.vyf[i]));
                    __stcs(&D.vzf[pos], __ldcs(&S.vzf[i]));
                } else {
                    __stcs(&D.z[pos], __ldcs(&S.z[i]));
                    __stcs(&D.vxd[pos], __ldcs(&S.vxd[i]));
                    __stcs(&D.vyd[pos], __ldcs(&S.vyd[i]));
                    __stcs(&D.vzd[pos], __ldcs(&S.vzd[i]));
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
