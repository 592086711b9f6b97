// pairs_noalloc.cu -- neighbour-pair search that allocates no device memory.
//
// The same question as prs_find_pairs (all pairs p < q closer than a cutoff,
// minimum image on periodic axes), asked without a context: the cell list it
// needs lives in one fixed array in this file, so a call makes no cudaMalloc,
// cudaFree or other allocating call. Callers that manage every byte of device
// memory themselves (a fixed memory budget, a pool that must not be bypassed)
// or that cannot afford the device synchronisation that cudaFree implies use
// this entry point.
//
// The array is shared by every call in the process on a given device. The
// cell counters that must start at zero are cleared at the start of every
// call, so a call never depends on an earlier one; but two calls whose work
// can overlap on the device (different streams, different host threads without
// ordering) use the same array at the same time and give wrong results.
//
// Steps (all on the caller's stream): clear the counters, count spheres per
// cell, scan the counts into cell starts (one block), scatter sphere ids into
// cell order, then test each sphere against the spheres of its own and the
// neighbouring cells.

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "pr_sed.h"

namespace prs {
void set_error(const char *fmt, ...);
}

namespace {

constexpr int kMaxP = PRS_NOALLOC_MAX_PARTICLES;
constexpr int kMaxCells = PRS_NOALLOC_MAX_CELLS;
constexpr int kMaxDevices = 64;
constexpr int kScanThreads = 1024;

// scratch layout, in ints: count[kMaxCells] | start[kMaxCells + 1] |
// cell of each sphere[kMaxP] | sphere ids in cell order[kMaxP]
constexpr size_t kOffCount = 0;
constexpr size_t kOffStart = kOffCount + kMaxCells;
constexpr size_t kOffCell = kOffStart + kMaxCells + 1;
constexpr size_t kOffSorted = kOffCell + kMaxP;
constexpr size_t kWords = kOffSorted + kMaxP;

static __device__ __align__(256) int g_pair_scratch[kWords];

struct Cells {
    int nc[3];
    double cs[3];
    double L[3];
    int periodic[3];
};

std::mutex g_mu;
int *g_scratch_ptr[kMaxDevices] = {};

__global__ void k_clear(int *__restrict__ count, int ncell,
                        unsigned long long *__restrict__ n_found)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x)
        count[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *n_found = 0ULL;
}

__device__ __forceinline__ int cell_of(const double *__restrict__ x, int n_p, int p,
                                       const Cells &g)
{
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int i = (int)floor(x[a * n_p + p] / g.cs[a]);
        c[a] = min(max(i, 0), g.nc[a] - 1);
    }
    return c[0] + g.nc[0] * (c[1] + g.nc[1] * c[2]);
}

__global__ void k_count(const double *__restrict__ x, int n_p, Cells g, int *__restrict__ pcell,
                        int *__restrict__ count)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_p)
        return;
    const int key = cell_of(x, n_p, p, g);
    pcell[p] = key;
    atomicAdd(&count[key], 1);
}

// exclusive scan of count[0, ncell) into start[0, ncell]; one block, each
// thread owns a contiguous chunk
__global__ void __launch_bounds__(kScanThreads)
k_scan(const int *__restrict__ count, int *__restrict__ start, int ncell)
{
    __shared__ int warp_sum[kScanThreads / 32];
    const int tid = threadIdx.x;
    const int chunk = (ncell + kScanThreads - 1) / kScanThreads;
    const int b = min(tid * chunk, ncell), e = min(b + chunk, ncell);
    int s = 0;
    for (int i = b; i < e; i++)
        s += count[i];
    // inclusive scan of the chunk sums: within the warp, then across warps
    const int lane = tid & 31, wid = tid >> 5;
    int v = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += t;
    }
    if (lane == 31)
        warp_sum[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int w = warp_sum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o)
                w += t;
        }
        warp_sum[lane] = w;
    }
    __syncthreads();
    int run = v - s + (wid > 0 ? warp_sum[wid - 1] : 0);
    for (int i = b; i < e; i++) {
        start[i] = run;
        run += count[i];
    }
    if (tid == kScanThreads - 1)
        start[ncell] = run;
}

// each sphere takes a slot of its cell; the counters end at zero again
__global__ void k_scatter(int n_p, const int *__restrict__ pcell, const int *__restrict__ start,
                          int *__restrict__ count, int *__restrict__ sorted)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_p)
        return;
    const int key = pcell[p];
    sorted[start[key] + atomicSub(&count[key], 1) - 1] = p;
}

// neighbouring cell indices along one axis, each listed once
__device__ __forceinline__ int neighbours(const Cells &g, int a, int c, int idx[3])
{
    const int nc = g.nc[a];
    int k = 0;
    if (g.periodic[a] && nc >= 3) {
        idx[k++] = c == 0 ? nc - 1 : c - 1;
        idx[k++] = c;
        idx[k++] = c == nc - 1 ? 0 : c + 1;
    } else if (g.periodic[a]) {
        for (int i = 0; i < nc; i++)
            idx[k++] = i;
    } else {
        for (int i = max(c - 1, 0); i <= min(c + 1, nc - 1); i++)
            idx[k++] = i;
    }
    return k;
}

// centre distance of spheres p < q: q minus p per axis, shifted by one box
// length on a periodic axis when it exceeds half of it; every operation
// rounded separately (no fused multiply-add)
__device__ __forceinline__ double distance(const double xp[3], const double xq[3], const Cells &g)
{
    double d[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        double s = __dsub_rn(xq[a], xp[a]);
        if (g.periodic[a]) {
            const double half = 0.5 * g.L[a];
            if (s > half)
                s = __dsub_rn(s, g.L[a]);
            else if (s < -half)
                s = __dadd_rn(s, g.L[a]);
        }
        d[a] = s;
    }
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])),
                                __dmul_rn(d[2], d[2]));
    return sqrt(d2);
}

__global__ void k_pairs(const double *__restrict__ x, int n_p, const int *__restrict__ pcell,
                        const int *__restrict__ start, const int *__restrict__ sorted, Cells g,
                        double cutoff, int *__restrict__ out, long long max_pairs,
                        unsigned long long *__restrict__ n_found)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_p)
        return;
    double xp[3];
#pragma unroll
    for (int a = 0; a < 3; a++)
        xp[a] = x[a * n_p + p];
    const int key = pcell[p];
    const int c0 = key % g.nc[0], c1 = (key / g.nc[0]) % g.nc[1], c2 = key / (g.nc[0] * g.nc[1]);
    int ix[3], iy[3], iz[3];
    const int nx = neighbours(g, 0, c0, ix), ny = neighbours(g, 1, c1, iy),
              nz = neighbours(g, 2, c2, iz);
    for (int kz = 0; kz < nz; kz++)
        for (int ky = 0; ky < ny; ky++)
            for (int kx = 0; kx < nx; kx++) {
                const int cell = ix[kx] + g.nc[0] * (iy[ky] + g.nc[1] * iz[kz]);
                const int j1 = start[cell + 1];
                for (int j = start[cell]; j < j1; j++) {
                    const int q = sorted[j];
                    if (q <= p)
                        continue;
                    double xq[3];
#pragma unroll
                    for (int a = 0; a < 3; a++)
                        xq[a] = x[a * n_p + q];
                    if (distance(xp, xq, g) < cutoff) {
                        const unsigned long long slot = atomicAdd(n_found, 1ULL);
                        if ((long long)slot < max_pairs) {
                            out[2 * slot] = p;
                            out[2 * slot + 1] = q;
                        }
                    }
                }
            }
}

// cells wider than the cutoff by a relative 1e-10 (so that rounding of x / cs
// never moves two spheres closer than the cutoff two cells apart), coarsened
// along the longest count until the total fits the fixed array (wider cells
// find the same pairs)
Cells make_cells(const double L[3], const int periodic[3], double cutoff)
{
    Cells g{};
    for (int a = 0; a < 3; a++) {
        const double r = std::floor(L[a] / (cutoff * (1.0 + 1e-10)));
        g.nc[a] = r < 1.0 ? 1 : (r > (double)kMaxCells ? kMaxCells : (int)r);
        g.L[a] = L[a];
        g.periodic[a] = periodic[a] ? 1 : 0;
    }
    while ((long long)g.nc[0] * g.nc[1] * g.nc[2] > kMaxCells) {
        int a = 0;
        for (int k = 1; k < 3; k++)
            if (g.nc[k] > g.nc[a])
                a = k;
        g.nc[a] = g.nc[a] / 2 > 0 ? g.nc[a] / 2 : 1;
    }
    for (int a = 0; a < 3; a++)
        g.cs[a] = L[a] / g.nc[a];
    return g;
}

// the device address of the scratch array on the current device, looked up
// once per device
prs_status scratch_for_current_device(int **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        prs::set_error("prs_find_pairs_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
        return PRS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        prs::set_error("prs_find_pairs_noalloc: device %d beyond the %d supported", dev,
                       kMaxDevices);
        return PRS_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_pair_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            prs::set_error("prs_find_pairs_noalloc: cudaGetSymbolAddress: %s",
                           cudaGetErrorString(e));
            return PRS_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<int *>(p);
    }
    *out = g_scratch_ptr[dev];
    return PRS_OK;
}

}  // namespace

extern "C" prs_status prs_find_pairs_noalloc(const double *x, int n_p, const double *L,
                                             const int *periodic, double cutoff, int *pairs,
                                             long long max_pairs, unsigned long long *n_pairs,
                                             void *stream)
{
    if (!L || !periodic || !n_pairs || (n_p > 0 && !x) || (max_pairs > 0 && !pairs) ||
        max_pairs < 0 || n_p < 0) {
        prs::set_error("prs_find_pairs_noalloc: bad arguments");
        return PRS_ERR_ARG;
    }
    if (n_p > kMaxP) {
        prs::set_error("prs_find_pairs_noalloc: %d spheres exceed the fixed scratch limit of %d",
                       n_p, kMaxP);
        return PRS_ERR_ARG;
    }
    if (!(cutoff > 0.0) || !std::isfinite(cutoff)) {
        prs::set_error("prs_find_pairs_noalloc: cutoff must be positive and finite");
        return PRS_ERR_ARG;
    }
    for (int a = 0; a < 3; a++)
        if (!(L[a] > 0.0) || !std::isfinite(L[a])) {
            prs::set_error("prs_find_pairs_noalloc: box lengths must be positive and finite");
            return PRS_ERR_ARG;
        }
    // an error left pending by earlier, unrelated work is reported as such
    // (and cleared) instead of being taken for a failure of this call
    const cudaError_t pending = cudaGetLastError();
    if (pending != cudaSuccess) {
        prs::set_error("prs_find_pairs_noalloc: a CUDA error was pending before the call: %s",
                       cudaGetErrorString(pending));
        return PRS_ERR_CUDA;
    }
    int *scratch = nullptr;
    prs_status st = scratch_for_current_device(&scratch);
    if (st)
        return st;
    const Cells g = make_cells(L, periodic, cutoff);
    const int ncell = g.nc[0] * g.nc[1] * g.nc[2];
    int *count = scratch + kOffCount, *start = scratch + kOffStart;
    int *pcell = scratch + kOffCell, *sorted = scratch + kOffSorted;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int clear_blocks = (ncell + 255) / 256 < 1024 ? (ncell + 255) / 256 : 1024;
    auto launched = [](const char *kernel) -> prs_status {
        const cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            return PRS_OK;
        prs::set_error("prs_find_pairs_noalloc: launch of %s: %s", kernel, cudaGetErrorString(e));
        return PRS_ERR_CUDA;
    };
    k_clear<<<clear_blocks, 256, 0, s>>>(count, ncell, n_pairs);
    if ((st = launched("k_clear")))
        return st;
    if (n_p > 0) {
        const int nb = (n_p + 255) / 256;
        k_count<<<nb, 256, 0, s>>>(x, n_p, g, pcell, count);
        if ((st = launched("k_count")))
            return st;
        k_scan<<<1, kScanThreads, 0, s>>>(count, start, ncell);
        if ((st = launched("k_scan")))
            return st;
        k_scatter<<<nb, 256, 0, s>>>(n_p, pcell, start, count, sorted);
        if ((st = launched("k_scatter")))
            return st;
        k_pairs<<<(n_p + 127) / 128, 128, 0, s>>>(x, n_p, pcell, start, sorted, g, cutoff, pairs,
                                                  max_pairs, n_pairs);
        if ((st = launched("k_pairs")))
            return st;
    }
    return PRS_OK;
}
