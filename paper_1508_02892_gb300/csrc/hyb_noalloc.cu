// hyb_noalloc.cu -- the field of a particle set (CIC charge assignment, then
// the Poisson solve) computed without any device allocation, for callers that
// cannot call cudaMalloc: the intermediate node sums live in a file-scope
// device array of fixed size.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "hyb_internal.cuh"

using namespace hyb;

namespace {

constexpr int kNaMaxNodes = HYB_MAX_CELLS + 1;  // 4001 nodes, 32 KB
constexpr int kNaThreads = 1024;
constexpr int kNaMaxDevices = 64;
// k_na_field keeps at most 8 nodes per thread in a local array
static_assert((kNaMaxNodes + kNaThreads - 1) / kNaThreads <= 8, "raise the local array of k_na_field");

// Scratch shared by every call on a device: the CIC node sums.  Its host-side
// name is only a stand-in; kernels get the device address looked up below.
static __device__ __align__(256) double g_na_sums[kNaMaxNodes];

double *g_na_ptr[kNaMaxDevices] = {};
std::mutex g_na_mutex;

__global__ void k_na_deposit(const double *__restrict__ z, int64_t n, double L, double dz, int nc, double *sums)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double zi = z[i];
        if (!(zi >= 0.0 && zi < L)) continue;  // outside the gap: no charge
        const double x = zi / dz;
        const double f = floor(x);
        int c = (int)f;
        double o = x - f;
        if (c >= nc) {
            c = nc - 1;
            o = 1.0;
        }
        atomicAdd(&sums[c], 1.0 - o);
        atomicAdd(&sums[c + 1], o);
    }
}

// Exclusive block scan of one double per thread (1024 threads).
__device__ double na_exscan(double v, double *warp_tot, double *total)
{
    const unsigned full = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double x = v;
    for (int d = 1; d < 32; d <<= 1) {
        const double y = __shfl_up_sync(full, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        double s = lane < nw ? warp_tot[lane] : 0.0;
        for (int d = 1; d < 32; d <<= 1) {
            const double y = __shfl_up_sync(full, s, d);
            if (lane >= d) s += y;
        }
        warp_tot[lane] = s;
    }
    __syncthreads();
    const double off = wid ? warp_tot[wid - 1] : 0.0;
    if (total) *total = warp_tot[nw - 1];
    __syncthreads();
    return off + x - v;
}

// n_e from the node sums, then -eps0 phi'' = e (n_i - n_e) with
// phi(0) = phi0, phi(L) = 0 in closed form (two prefix scans), E by central
// differences inside and Gauss's law over the half cells at the walls.
__global__ void __launch_bounds__(kNaThreads) k_na_field(const double *__restrict__ sums, const double *__restrict__ ni,
                                                         int G, double dz, double w, double phi0, double *ne,
                                                         double *phi, double *E)
{
    extern __shared__ double na_sm[];
    __shared__ double warp_tot[32];
    double *s_rho = na_sm;
    double *s_S = na_sm + G;
    const int T = blockDim.x, t = threadIdx.x;
    const int per = (G + T - 1) / T;
    const int j0 = min(t * per, G), j1 = min(j0 + per, G);
    double part = 0.0;
    for (int j = j0; j < j1; ++j) {
        const double dv = (j == 0 || j == G - 1) ? 0.5 * dz : dz;
        const double nej = w * sums[j] / dv;
        ne[j] = nej;
        const double rho = kQe * (ni[j] - nej);
        s_rho[j] = rho;
        part += (j >= 1 && j <= G - 2) ? dz * dz * rho / kEps0 : 0.0;
        s_S[j] = part;
    }
    const double off = na_exscan(part, warp_tot, nullptr);
    double ssum = 0.0;
    for (int j = j0; j < j1; ++j) {
        s_S[j] += off;
        if (j <= G - 2) ssum += s_S[j];
    }
    double stot;
    na_exscan(ssum, warp_tot, &stot);
    const double d0 = (stot - phi0) / (double)(G - 1);
    double dpart = 0.0;
    double loc[8];
    for (int j = j0; j < j1; ++j) {
        loc[j - j0] = dpart;
        dpart += j <= G - 2 ? d0 - s_S[j] : 0.0;
    }
    const double doff = na_exscan(dpart, warp_tot, nullptr);
    for (int j = j0; j < j1; ++j) {
        phi[j] = j == G - 1 ? 0.0 : phi0 + doff + loc[j - j0];
        double e;
        if (j == 0)
            e = -d0 / dz - s_rho[0] * dz / (2.0 * kEps0);
        else if (j == G - 1)
            e = -(d0 - s_S[G - 2]) / dz + s_rho[G - 1] * dz / (2.0 * kEps0);
        else
            e = -((d0 - s_S[j]) + (d0 - s_S[j - 1])) / (2.0 * dz);
        E[j] = e;
    }
}

// Device address of the scratch array for the current device, looked up once
// per device with that device current.
int na_scratch(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_last_error("cudaGetDevice failed");
        return HYB_ERR_CUDA;
    }
    if (dev < 0 || dev >= kNaMaxDevices) {
        set_last_error("device index out of range");
        return HYB_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_na_sums);
        if (e != cudaSuccess) {
            set_last_error(cudaGetErrorString(e));
            return HYB_ERR_CUDA;
        }
        e = cudaFuncSetAttribute(k_na_field, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(2 * sizeof(double) * kNaMaxNodes));
        if (e != cudaSuccess) {
            set_last_error(cudaGetErrorString(e));
            return HYB_ERR_CUDA;
        }
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return HYB_OK;
}

}  // namespace

extern "C" int hyb_field_from_particles_noalloc(const hyb_params *p, int64_t n, const double *z, const double *ni,
                                                double t, double *ne, double *phi, double *efield, void *stream)
{
    if (!p || (n > 0 && !z) || !ni || !ne || !phi || !efield) {
        set_last_error("NULL argument");
        return HYB_ERR_ARG;
    }
    if (p->n_cells < 2 || p->n_cells > HYB_MAX_CELLS) {
        set_last_error("n_cells must be in [2, 4000]: the scratch holds at most 4001 node sums");
        return HYB_ERR_ARG;
    }
    if (!(p->gap_m > 0) || n < 0) {
        set_last_error("gap must be positive and n non-negative");
        return HYB_ERR_ARG;
    }
    double *sums = nullptr;
    int rc = na_scratch(&sums);
    if (rc) return rc;
    const int G = p->n_cells + 1;
    const double L = p->gap_m, dz = p->gap_m / p->n_cells;
    const double w = p->weight > 0 ? p->weight
                                   : (p->n_particles > 0 ? p->n0_m3 * p->gap_m / (double)p->n_particles : 0.0);
    const double phi0 = p->v_dc_v + p->v_rf_amp_v * sin(kTwoPi * p->f_rf_hz * t);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(double) * G, s);  // clear the previous call's sums
    if (e == cudaSuccess && n > 0) {
        int grid = (int)((n + 255) / 256);
        if (grid > 152 * 8) grid = 152 * 8;
        k_na_deposit<<<grid, 256, 0, s>>>(z, n, L, dz, p->n_cells, sums);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_na_field<<<1, kNaThreads, 2 * sizeof(double) * G, s>>>(sums, ni, G, dz, w, phi0, ne, phi, efield);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return HYB_ERR_CUDA;
    }
    return HYB_OK;
}
