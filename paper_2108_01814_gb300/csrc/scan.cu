// Exclusive prefix sum of int arrays (reduce-then-scan over blocks of 1024,
// recursive on the block totals). Integer arithmetic: deterministic.
#include "prs_internal.cuh"

namespace prs {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanBlock = 4 * kScanThreads;

__device__ __forceinline__ int warp_incl_scan(int v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += t;
    }
    return v;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_blocks(const int *__restrict__ in, int *__restrict__ out, int n, int *__restrict__ sums,
              const int *__restrict__ enable)
{
    if (enable && !*enable)
        return;
    __shared__ int warp_tot[kScanThreads / 32];
    const long long base = (long long)blockIdx.x * kScanBlock + 4LL * threadIdx.x;
    int v[4];
    int tsum = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        long long i = base + k;
        v[k] = i < n ? in[i] : 0;
        tsum += v[k];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = warp_incl_scan(tsum);
    if (lane == 31)
        warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        t = warp_incl_scan(t);
        if (lane < kScanThreads / 32)
            warp_tot[lane] = t;
    }
    __syncthreads();
    int excl = incl - tsum + (wid > 0 ? warp_tot[wid - 1] : 0);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        long long i = base + k;
        if (i < n)
            out[i] = excl;
        excl += v[k];
    }
    if (sums && threadIdx.x == kScanThreads - 1)
        sums[blockIdx.x] = excl;
}

__global__ void k_scan_add(int *__restrict__ out, int n, const int *__restrict__ offs,
                           const int *__restrict__ enable)
{
    if (enable && !*enable)
        return;
    long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    int add = offs[blockIdx.x];
#pragma unroll
    for (int k = 0; k < 4; k++, i += kScanThreads)
        if (i < n)
            out[i] += add;
}

}  // namespace

size_t exclusive_scan_tmp_ints(int n)
{
    size_t t = 0;
    while (n > kScanBlock) {
        int nb = (n + kScanBlock - 1) / kScanBlock;
        t += 2 * (size_t)nb;
        n = nb;
    }
    return t + 1;
}

int exclusive_scan(const int *in, int *out, int n, int *tmp, cudaStream_t s, const int *enable)
{
    if (n <= 0)
        return 0;
    int nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb == 1) {
        k_scan_blocks<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, enable);
        return 1;
    }
    int *sums = tmp;
    int *sums_scanned = tmp + nb;
    k_scan_blocks<<<nb, kScanThreads, 0, s>>>(in, out, n, sums, enable);
    int k = exclusive_scan(sums, sums_scanned, nb, tmp + 2 * nb, s, enable);
    k_scan_add<<<nb, kScanThreads, 0, s>>>(out, n, sums_scanned, enable);
    return k + 2;
}

}  // namespace prs
