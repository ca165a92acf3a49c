// hyb_device.cuh -- device helpers shared by the particle kernels (electrons
// and kinetic ions): warp sums, the CIC pair deposit into block-private shared
// rows, the FP64 cell location, Box-Muller pairs, isotropic directions, and
// the split of the running instances' chunks over the blocks of a launch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hyb_internal.cuh"

namespace hyb {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kBlock = 256;

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
struct WarpSum;

template <>
struct WarpSum<double> {
    __device__ static double run(double v)
    {
#pragma unroll
        for (int d = 16; d; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
        return v;
    }
};

template <>
struct WarpSum<float> {
    __device__ static float run(float v)
    {
#pragma unroll
        for (int d = 16; d; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
        return v;
    }
};

// Add (w0 at node c, w1 at node c+1) for every lane that has `on`; when every
// participating lane has the same c, sum over the warp first.
template <typename T>
__device__ __forceinline__ void deposit_pair(T *arr, bool on, int c, T w0, T w1, int G)
{
    if (on && !HYB_CHECK(c >= 0 && c + 1 < G, 4, c, G)) on = false;
    const int kmin = __reduce_min_sync(kFull, on ? c : INT32_MAX);
    const int kmax = __reduce_max_sync(kFull, on ? c : -1);
    if (kmin == kmax) {
        T a = WarpSum<T>::run(on ? w0 : T(0));
        T b = WarpSum<T>::run(on ? w1 : T(0));
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&arr[kmin], a);
            atomicAdd(&arr[kmin + 1], b);
        }
    } else if (on) {
        atomicAdd(&arr[c], w0);
        atomicAdd(&arr[c + 1], w1);
    }
}

__device__ __forceinline__ void locate_d(double z, double dz, int nc, int &c, double &o)
{
    const double x = z / dz;
    const double f = floor(x);
    c = (int)f;
    o = x - f;
    if (c >= nc) {
        c = nc - 1;
        o = 1.0;
    }
}

__device__ __forceinline__ void gauss_pair(double u1, double u2, double &g1, double &g2)
{
    const double r = sqrt(-2.0 * log(u1));
    const double ph = kTwoPi * u2;
    g1 = r * cos(ph);
    g2 = r * sin(ph);
}

__device__ __forceinline__ void iso_dir_d(double u_cos, double u_phi, double d[3])
{
    const double ct = 1.0 - 2.0 * u_cos;
    const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    const double ph = kTwoPi * u_phi;
    d[0] = st * cos(ph);
    d[1] = st * sin(ph);
    d[2] = ct;
}

// This block's contiguous run of kChunk-slot chunks, split by instance:
// fn(K, a, b) for each instance touched, with a a multiple of kChunk.  The
// chunks are dealt as evenly as they divide: every block gets floor or ceil of
// total / grid, so no block idles while others take an extra chunk or more.
template <class F>
__device__ __forceinline__ void for_block_runs(InstDev *__restrict__ insts, int n_max,
                                               const int64_t *__restrict__ prefix, F &&fn)
{
    const int64_t total = prefix[n_max];
    if (total <= 0) return;
    const int64_t c0 = total * (int64_t)blockIdx.x / (int64_t)gridDim.x;
    const int64_t c1 = total * ((int64_t)blockIdx.x + 1) / (int64_t)gridDim.x;
    if (c0 >= c1) return;
    int lo = 0, hi = n_max;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= c0)
            lo = mid;
        else
            hi = mid;
    }
    int64_t ch = c0;
    for (int i = lo; i < n_max && ch < c1; ++i) {
        const int64_t p0 = prefix[i], p1 = prefix[i + 1];
        if (p1 <= ch) continue;
        const int64_t e = c1 < p1 ? c1 : p1;
        InstDev *K = &insts[i];
        const int64_t n = K->n_slots_step;
        const int64_t a = (ch - p0) * kChunk;
        const int64_t b = (e - p0) * kChunk < n ? (e - p0) * kChunk : n;
        if (HYB_CHECK(p1 - p0 == chunks_of(n) && (K->cur & ~1) == 0, 12, i, p1 - p0)) fn(K, a, b);
        ch = e;
    }
}

}  // namespace

}  // namespace hyb
