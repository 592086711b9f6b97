// Direct-forcing immersed boundary kernels (Sec. 2.1 and 3.3 of the paper).
//
// Markers are never stored: every kernel regenerates X_l = x_p + R t_l from
// the particle and the shared template (Sec. 3.5). Work is organised by
// tiles of kTileX x kTileY x kTileZ grid cells; a marker belongs to the tile
// that holds its nearest grid point (its "bin").
//
//   k_marker_bin     counting sort of the markers by (tile, face class).
//   k_particle_tiles counting sort of the spheres into the tiles their
//                    markers' stencils can reach (the spread's lists).
//   k_interp_tma     persistent, warp-specialised: a producer warp stages
//                    u, v, w of a tile plus a halo in shared memory with TMA
//                    tensor copies, two tiles deep, while eight consumer
//                    warps process the staged tiles; for every marker it
//                    interpolates the fluid velocity with the 3-point
//                    regularised delta and forms the direct-forcing marker
//                    force F_l (stored per marker), and records the tile's
//                    largest |F_l| per component.
//   k_interp_tiles   the same for the tiles at a periodic end, whose halo
//                    wraps, with cp.async staging.
//   k_particle_sums  four lanes per particle: F_h = -rho_f sum F_l dV and
//                    T_h = -rho_f sum (X_l - x_p) x F_l dV (Kahan sums).
//   k_spread_tiles   collects the markers whose stencils reach the tile
//                    (from its sphere list, or the face-class ranges of its
//                    neighbours) and adds F_l phi phi phi dV/h^3 for each
//                    stencil cell inside the tile to fixed-point shared
//                    accumulators with integer atomics: integer addition is
//                    associative, so repeated runs give bit-identical fields.
//                    It then adds the sum to f and alpha dt times it to u.
//
// Precision: T = double (FP64 form) or float (FP32 form). Particle
// positions enter as an FP64 grid index plus a remainder in [0, 1), so the
// FP32 form keeps full accuracy on large grids.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <utility>
#include <climits>
#include <cstdio>

#include "prs_internal.cuh"

namespace prs {
namespace {

constexpr int TX = kTileX, TY = kTileY, TZ = kTileZ;
constexpr int kCells = TX * TY * TZ;
constexpr int kThreads = 256;
constexpr int kCellsPerThread = kCells / kThreads;
static_assert(kCells % kThreads == 0, "cells per thread");
static_assert(kCells % kThreads == 0, "tile cells must be a multiple of the block size");

template <typename T>
struct TileArgs {
    const PartPrep<T> *prep;
    const PartFast<T> *pfast;
    unsigned long long l_magic;
    const T *tR;  // [3][n_l] R/h t_l
    const T *rR;  // [3][n_l] R t_l
    const T *fld[3];
    T *out_f[3];
    T *out_u[3];
    T *Fl, *dFl;  // [n_m][4] marker force and latest increment
    unsigned long long *red;
    // per tile max |dF| per component (bits): written by the interpolation,
    // read by the spread (null: the spread takes the global maxima in red)
    unsigned long long *tile_fmax;
    int *err;
    const int *key_start, *mlist;
    // per tile, the spheres whose markers' stencils can reach it (null: the
    // spread takes the (neighbour, class) ranges of the binned markers)
    const int *pt_start, *pt_list;
    int n[3];
    int periodic[3];
    int nt[3];
    int n_p, n_l;
    int tile0;  // first tile of the launch (block b handles tile tile0 + b)
    const int *tiles;  // or tile tiles[b] (null: tile0 + b)
    int pass, probe;
    T inv_adt;
    double adt;
    double dVh3;
};

// ------------------------------------------------------------------ small helpers
// Weights of the 3-point kernel (Roma, Peskin & Berger 1999) along one axis
// for a point at grid coordinate q: i0 = nearest index, w[d] = weight of
// index i0 - 1 + d. With r1 = i0 - q in [-1/2, 1/2] all three branches of
// the kernel share the root sqrt(1 - 3 r1^2).
template <typename T>
__device__ __forceinline__ void axis_weights(T q, int &i0, T w[3])
{
    T f = floor(q + T(0.5));
    i0 = (int)f;
    T r1 = f - q;
    T S = sqrt(T(1) - T(3) * r1 * r1);
    const T third = T(1) / T(3), sixth = T(1) / T(6);
    w[1] = (T(1) + S) * third;
    w[0] = (T(2) + T(3) * r1 - S) * sixth;
    w[2] = (T(2) - T(3) * r1 - S) * sixth;
}

__device__ __forceinline__ unsigned long long max_bits(float v)
{
    return (unsigned long long)__float_as_uint(v);
}
__device__ __forceinline__ unsigned long long max_bits(double v)
{
    return (unsigned long long)__double_as_longlong(v);
}

// warp maximum of a non-negative value, as max_bits gives it
__device__ __forceinline__ unsigned long long warp_max_bits(float v)
{
    return (unsigned long long)__reduce_max_sync(0xffffffffu, __float_as_uint(v));
}
__device__ __forceinline__ unsigned long long warp_max_bits(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return max_bits(v);
}

template <typename T>
__device__ __forceinline__ T from_bits_t(unsigned long long b);
template <>
__device__ __forceinline__ float from_bits_t<float>(unsigned long long b)
{
    return __uint_as_float((unsigned)b);
}
template <>
__device__ __forceinline__ double from_bits_t<double>(unsigned long long b)
{
    return __longlong_as_double((long long)b);
}

template <typename T>
struct KSum {  // compensated sum, value = s - c
    T s, c;
    __device__ void init() { s = T(0); c = T(0); }
    __device__ void add(T x)
    {
        T y = x - c;
        T t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ void merge(T s2, T c2)
    {
        T t = s + s2;
        T bp = t - s;
        T e = (s - (t - bp)) + (s2 - bp);
        s = t;
        c = (c + c2) - e;
    }
};

__device__ __forceinline__ void store4(float *b, long long m, float x, float y, float z)
{
    reinterpret_cast<float4 *>(b)[m] = make_float4(x, y, z, 0.f);
}
__device__ __forceinline__ void store4(double *b, long long m, double x, double y, double z)
{
    double2 *q = reinterpret_cast<double2 *>(b) + 2 * m;
    q[0] = make_double2(x, y);
    q[1] = make_double2(z, 0.0);
}
__device__ __forceinline__ void load4(const float *b, long long m, float v[3])
{
    float4 t = reinterpret_cast<const float4 *>(b)[m];
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
}
__device__ __forceinline__ void load4(const double *b, long long m, double v[3])
{
    const double2 *q = reinterpret_cast<const double2 *>(b) + 2 * m;
    double2 a = q[0], c = q[1];
    v[0] = a.x;
    v[1] = a.y;
    v[2] = c.x;
}

// block-wide exclusive scan of one int per thread; returns the exclusive
// prefix and writes the total to *total (all threads)
__device__ int block_excl_scan(int v, int *tmp, int *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o)
            x += t;
    }
    if (lane == 31)
        tmp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < kThreads / 32 ? tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o)
                t += u;
        }
        if (lane < kThreads / 32)
            tmp[lane] = t;
    }
    __syncthreads();
    int excl = x - v + (wid > 0 ? tmp[wid - 1] : 0);
    *total = tmp[kThreads / 32 - 1];
    __syncthreads();
    return excl;
}

// The 27 tiles around a tile (offsets -1, 0, 1 per axis; periodic images
// get the shift that maps the neighbour's grid indices next to this tile).
struct Nb {
    int key[27];       // tile index, -1 if outside a bounded axis
    int shift[27][3];  // image shift in cells
    int ext[27][3];    // cells of the neighbour tile per axis
};

template <typename A>
__device__ void gather_neighbours(const A &a, const int tc[3], Nb &nb)
{
    const int te[3] = {TX, TY, TZ};
    for (int t = threadIdx.x; t < 27; t += blockDim.x) {
        const int d[3] = {t % 3 - 1, (t / 3) % 3 - 1, t / 9 - 1};
        int ok = 1, key = 0, mul = 1;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            int q = tc[k] + d[k];
            int sh = 0;
            if (q < 0 || q >= a.nt[k]) {
                if (!a.periodic[k]) {
                    ok = 0;
                } else if (q < 0) {
                    q += a.nt[k];
                    sh = -a.n[k];
                } else {
                    q -= a.nt[k];
                    sh = a.n[k];
                }
            }
            key += q * mul;
            mul *= a.nt[k];
            nb.shift[t][k] = sh;
            nb.ext[t][k] = min(te[k], a.n[k] - q * te[k]);
        }
        nb.key[t] = ok ? key : -1;
    }
    __syncthreads();
}

// Grid index (component 0) of the nearest grid point of marker l of a
// particle, per axis, wrapped into [0, n) on periodic axes and clamped into
// it on bounded ones; from the particle's compact record (two 16-byte loads).
template <typename T>
__device__ __forceinline__ void marker_bin(const PartFast<T> &rec, const T *tR, int n_l, int l,
                                           const int n[3], const int periodic[3], int wb[3])
{
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
        const T q = rec.fr[ax] + __ldg(tR + ax * n_l + l);
        const int b = rec.b[ax] + (int)floor(q + T(0.5));
        if (periodic[ax])
            wb[ax] = b < 0 ? b + n[ax] : (b >= n[ax] ? b - n[ax] : b);
        else
            wb[ax] = min(max(b, 0), n[ax] - 1);
    }
}

// Face class of a grid index inside a tile of ext cells along one axis:
// 0 = within W of the low face, 2 = within W of the high face, 1 = interior
// (low wins when a tile is too thin for both).
__device__ __forceinline__ int face_class(int local, int ext, int W)
{
    return local < W ? 0 : (local >= ext - W ? 2 : 1);
}
__device__ __forceinline__ void class_range(int cls, int ext, int W, int &lo, int &hi)
{
    const int a = min(W, ext), b = max(W, ext - W);
    lo = cls == 0 ? 0 : (cls == 1 ? a : b);
    hi = cls == 0 ? a : (cls == 1 ? b : ext);
}

// ------------------------------------------------------------------ prep
template <typename T>
__global__ void k_prep(const double *__restrict__ x, const double *__restrict__ up,
                       const double *__restrict__ om, int n_p, GridDesc g,
                       PartPrep<T> *__restrict__ prep, PartFast<T> *__restrict__ fast)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_p)
        return;
    PartPrep<T> pp;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        // FP64 divisions are slow here: x / 1 is x, and a centre already in
        // [0, n) needs no wrap (n floor(xs / n) is then 0), so both are taken
        // only when they change the value
        double xs = x[a * n_p + p];
        if (g.h != 1.0)
            xs /= g.h;
        if (g.periodic[a]) {
            // one periodic image for all components: xs in [0, n)
            const double n = (double)g.n[a];
            if (xs < 0.0 || xs >= n) {
                xs -= n * floor(xs / n);
                if (xs >= n)
                    xs = 0.0;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; c++) {
            double s = xs - g.off[c * 3 + a];
            double b = floor(s);
            pp.base[c * 3 + a] = (int)b;  // in [-1, n) on periodic axes
            pp.frac[c * 3 + a] = (T)(s - b);
        }
        pp.up[a] = (T)up[a * n_p + p];
        pp.om[a] = (T)om[a * n_p + p];
    }
    prep[p] = pp;
    PartFast<T> f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        f.fr[a] = pp.frac[a];
        f.up[a] = pp.up[a];
        f.om[a] = pp.om[a];
        f.b[a] = pp.base[a];
    }
    f.fr[3] = f.up[3] = f.om[3] = T(0);
    f.b[3] = 0;
    fast[p] = f;
}

// ------------------------------------------------------------------ marker binning
// Every marker gets the key (tile of its component-0 nearest grid point) *
// 27 + face class; a counting sort by key lists the markers of every
// (tile, class). Warp-aggregated atomics: the 32 markers a warp takes at a
// time belong to one or two particles and share few keys. Pass 0 counts,
// pass 1 scatters (taking positions by decrementing the counts, which end at
// zero). A warp takes kBinGroups such groups of 32 markers at once, so that
// in the scatter pass their atomics' round trips overlap.
constexpr int kBinGroups = 4;
template <typename T>
__global__ void __launch_bounds__(256)
k_marker_bin(const PartFast<T> *__restrict__ pf, const T *__restrict__ tR, int n_p, int n_l,
             unsigned long long l_magic, int n0, int n1, int n2, int per0, int per1, int per2,
             int nt0, int nt1, int W,
             int scatter, int *__restrict__ count, const int *__restrict__ start,
             int *__restrict__ list)
{
    const long long n_m = (long long)n_p * n_l;
    const int lane = threadIdx.x & 31;
    const long long warp_g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n[3] = {n0, n1, n2}, periodic[3] = {per0, per1, per2};
    const int te[3] = {TX, TY, TZ};
    int key[kBinGroups];
    unsigned peers[kBinGroups];
#pragma unroll
    for (int j = 0; j < kBinGroups; j++) {
        const long long m = (warp_g * kBinGroups + j) * 32 + lane;
        const bool valid = m < n_m;
        const unsigned act = __ballot_sync(0xffffffffu, valid);
        key[j] = -1;
        peers[j] = 0u;
        if (valid) {
            const int p = (int)__umul64hi((unsigned long long)m, l_magic);  // m / n_l
            const int l = (int)(m - (long long)p * n_l);
            int wb[3];
            marker_bin(pf[p], tR, n_l, l, n, periodic, wb);
            int t[3], cls[3];
#pragma unroll
            for (int ax = 0; ax < 3; ax++) {
                t[ax] = (int)((unsigned)wb[ax] / (unsigned)te[ax]);  // wb >= 0
                const int ext = min(te[ax], n[ax] - t[ax] * te[ax]);
                cls[ax] = face_class(wb[ax] - t[ax] * te[ax], ext, W);
            }
            key[j] = (t[0] + nt0 * (t[1] + nt1 * t[2])) * 27 + cls[0] + 3 * (cls[1] + 3 * cls[2]);
            peers[j] = __match_any_sync(act, key[j]);
        }
    }
    const unsigned below = (1u << lane) - 1u;
    if (!scatter) {
#pragma unroll
        for (int j = 0; j < kBinGroups; j++)
            if (peers[j] && lane == __ffs(peers[j]) - 1)
                atomicAdd(&count[key[j]], __popc(peers[j]));
        return;
    }
    // the groups' atomics first, all in flight, then their positions
    int base[kBinGroups];
#pragma unroll
    for (int j = 0; j < kBinGroups; j++) {
        base[j] = 0;
        if (peers[j] && lane == __ffs(peers[j]) - 1)
            base[j] = atomicSub(&count[key[j]], __popc(peers[j])) - __popc(peers[j]);
    }
#pragma unroll
    for (int j = 0; j < kBinGroups; j++) {
        if (!peers[j])
            continue;
        const int b = __shfl_sync(peers[j], base[j], __ffs(peers[j]) - 1);
        const long long m = (warp_g * kBinGroups + j) * 32 + lane;
        list[start[key[j]] + b + __popc(peers[j] & below)] = (int)m;
    }
}

__device__ __forceinline__ int floor_div(int a, int b)
{
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

// Sphere -> tiles for the spread: the tiles whose cells the stencils of
// the sphere's markers can reach (component-0 nearest indices of the
// markers lie in [floor(q - R/h + 1/2), floor(q + R/h + 1/2)] per axis, q
// the centre in index space; a tile takes bins within W cells of it).
// Pass 0 counts per tile, pass 1 scatters (counts return to zero).
template <typename T>
__global__ void __launch_bounds__(256)
k_particle_tiles(const PartFast<T> *__restrict__ pf, int n_p, double Rh, int n0, int n1,
                 int n2, int per0, int per1, int per2, int nt0, int nt1, int nt2, int W,
                 int scatter, int *__restrict__ count, const int *__restrict__ start,
                 int *__restrict__ list)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_p)
        return;
    const int n[3] = {n0, n1, n2}, per[3] = {per0, per1, per2}, nt[3] = {nt0, nt1, nt2};
    const int te[3] = {TX, TY, TZ};
    const PartFast<T> r = pf[p];
    int lo[3], hi[3];
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
        const double q = (double)r.b[ax] + (double)r.fr[ax];
        const int bmin = (int)floor(q - Rh + 0.5), bmax = (int)floor(q + Rh + 0.5);
        lo[ax] = floor_div(bmin - W, te[ax]);
        hi[ax] = floor_div(bmax + W, te[ax]);
        if (!per[ax]) {
            lo[ax] = max(lo[ax], 0);
            hi[ax] = min(hi[ax], nt[ax] - 1);
        }
        (void)n;
    }
    for (int tz = lo[2]; tz <= hi[2]; tz++)
        for (int ty = lo[1]; ty <= hi[1]; ty++)
            for (int tx = lo[0]; tx <= hi[0]; tx++) {
                const int wx = (tx % nt0 + nt0) % nt0, wy = (ty % nt1 + nt1) % nt1,
                          wz = (tz % nt2 + nt2) % nt2;
                const int key = wx + nt0 * (wy + nt1 * wz);
                if (!scatter)
                    atomicAdd(&count[key], 1);
                else
                    list[start[key] + atomicSub(&count[key], 1) - 1] = p;
            }
}

__global__ void k_set_int2(int *ptr, int v) { *ptr = v; }

// ------------------------------------------------------------------ interpolation + forcing
template <typename T, bool SAME>
struct SmemInterp {
    static constexpr int H = SAME ? 1 : 2;               // stencil halo in cells
    static constexpr int VW = 16 / sizeof(T);             // elements per 16-byte vector
    static constexpr int XO = (H + VW - 1) / VW * VW;     // staged x margin, vector aligned
    static constexpr int RX = TX + 2 * XO, RY = TY + 2 * H, RZ = TZ + 2 * H;
    static constexpr int RN = RX * RY * RZ;
    T fld[3][RN];
    T red[4][kThreads / 32];
    // the marker template follows: tR[3][n_l], rR[3][n_l]
};

// root of the shared kernel term: FP32 uses the hardware reciprocal square
// root (argument in [1/4, 1]), FP64 the IEEE square root
__device__ __forceinline__ float kernel_root(float x) { return x * rsqrtf(x); }
__device__ __forceinline__ double kernel_root(double x) { return sqrt(x); }

template <typename T>
__device__ __forceinline__ void axis_weights_fast(T q, int &i0, T w[3])
{
    T f = floor(q + T(0.5));
    i0 = (int)f;
    T r1 = f - q;
    T S = kernel_root(T(1) - T(3) * r1 * r1);
    const T third = T(1) / T(3), sixth = T(1) / T(6);
    w[1] = (T(1) + S) * third;
    w[0] = (T(2) + T(3) * r1 - S) * sixth;
    w[2] = (T(2) - T(3) * r1 - S) * sixth;
}

// cp.async of 16 bytes global -> shared (bypassing L1); with valid = false
// no byte is read and the 16 bytes are zero-filled
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(n)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}


// Interpolation of u, v, w at one marker from the staged block (all
// components on the same grid points). CLIP: the stencil may leave the
// staged block beyond a bounded wall; EDGE: the particle may sit on the
// other side of a periodic boundary.
template <typename T, typename Sm, bool CLIP, bool EDGE>
__device__ __forceinline__ void gather_fast(const TileArgs<T> &a, const T (&fld)[3][Sm::RN],
                                            const PartFast<T> rec, const T rt[3],
                                            const int org[3], T U[3], T up[3], T om[3])
{
    constexpr int H = Sm::H, XO = Sm::XO, RX = Sm::RX, RY = Sm::RY, RZ = Sm::RZ;
    const int lo_off[3] = {XO, H, H};
    const int rdim[3] = {RX, RY, RZ};
    int off[3] = {0, 0, 0};
    if (EDGE) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            if (!a.periodic[k])
                continue;
            const int ub = rec.b[k] + (int)floor(rec.fr[k] + rt[k] + T(0.5));
            off[k] = ub < 0 ? a.n[k] : (ub >= a.n[k] ? -a.n[k] : 0);
        }
    }
    int ix[3][3];
    T w[3][3];
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
        int i0;
        axis_weights_fast(rec.fr[ax] + rt[ax], i0, w[ax]);
        const int lo = rec.b[ax] + off[ax] - org[ax] + i0 - 1 + lo_off[ax];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            int q = lo + d;
            if (CLIP && (q < 0 || q >= rdim[ax])) {  // beyond a bounded wall
                w[ax][d] = T(0);
                q = 0;
            }
            ix[ax][d] = q;
        }
    }
    T acc0 = T(0), acc1 = T(0), acc2 = T(0);
#pragma unroll
    for (int dz = 0; dz < 3; dz++) {
#pragma unroll
        for (int dy = 0; dy < 3; dy++) {
            const int row = (ix[2][dz] * RY + ix[1][dy]) * RX;
            const T wyz = w[1][dy] * w[2][dz];
            const int i0 = row + ix[0][0], i1 = row + ix[0][1], i2 = row + ix[0][2];
            acc0 += wyz * (w[0][0] * fld[0][i0] + w[0][1] * fld[0][i1] +
                           w[0][2] * fld[0][i2]);
            acc1 += wyz * (w[0][0] * fld[1][i0] + w[0][1] * fld[1][i1] +
                           w[0][2] * fld[1][i2]);
            acc2 += wyz * (w[0][0] * fld[2][i0] + w[0][1] * fld[2][i1] +
                           w[0][2] * fld[2][i2]);
        }
    }
    U[0] = acc0;
    U[1] = acc1;
    U[2] = acc2;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        up[k] = rec.up[k];
        om[k] = rec.om[k];
    }
}

// Interpolation and direct forcing at the markers binned in one tile (ids
// ml[0 .. n), in global or shared memory), from the tile's staged u, v, w
// block; accumulates the largest slip and |dF| per component.
template <typename T, bool SAME>
__device__ __forceinline__ void interp_tile_markers(const TileArgs<T> &a,
                                                   const T (&fld)[3][SmemInterp<T, SAME>::RN],
                                                   const int *ml, int n, const int org[3],
                                                   bool edge, bool clip, const T *tRs,
                                                   const T *rRs, T &res, T (&fmax)[3])
{
    using Sm = SmemInterp<T, SAME>;
    constexpr int H = Sm::H, XO = Sm::XO, RX = Sm::RX, RY = Sm::RY;
    const int lo_off[3] = {XO, H, H};
    const int rdim[3] = {Sm::RX, Sm::RY, Sm::RZ};
    const int tid = threadIdx.x;
    const int n_l = a.n_l;
    const PartFast<T> *__restrict__ pf = a.pfast;
    for (int j = tid; j < n; j += kThreads) {
        const int m = ml[j];
        const int p = (int)__umul64hi((unsigned long long)m, a.l_magic);
        const int l = m - p * n_l;
        T rt[3], rr[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            rt[k] = tRs[k * n_l + l];
            rr[k] = rRs[k * n_l + l];
        }
        T up[3], om[3];
        T U[3];
        if (SAME) {
            if (clip) {
                if (edge)
                    gather_fast<T, Sm, true, true>(a, fld, pf[p], rt, org, U, up, om);
                else
                    gather_fast<T, Sm, true, false>(a, fld, pf[p], rt, org, U, up, om);
            } else {
                if (edge)
                    gather_fast<T, Sm, false, true>(a, fld, pf[p], rt, org, U, up, om);
                else
                    gather_fast<T, Sm, false, false>(a, fld, pf[p], rt, org, U, up, om);
            }
        } else {
            const PartPrep<T> &pp = a.prep[p];
            int off[3] = {0, 0, 0};
            if (edge) {
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    if (!a.periodic[k])
                        continue;
                    const int ub = pp.base[k] + (int)floor(pp.frac[k] + rt[k] + T(0.5));
                    off[k] = ub < 0 ? a.n[k] : (ub >= a.n[k] ? -a.n[k] : 0);
                }
            }
#pragma unroll
            for (int c = 0; c < 3; c++) {
                int ix[3][3];
                T w[3][3];
#pragma unroll
                for (int ax = 0; ax < 3; ax++) {
                    int i0;
                    axis_weights_fast(pp.frac[c * 3 + ax] + rt[ax], i0, w[ax]);
                    const int lo = pp.base[c * 3 + ax] + off[ax] - org[ax] + i0 - 1 + lo_off[ax];
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        int q = lo + d;
                        if (q < 0 || q >= rdim[ax]) {
                            w[ax][d] = T(0);
                            q = 0;
                        }
                        ix[ax][d] = q;
                    }
                }
                T acc = T(0);
#pragma unroll
                for (int dz = 0; dz < 3; dz++) {
#pragma unroll
                    for (int dy = 0; dy < 3; dy++) {
                        const int row = (ix[2][dz] * RY + ix[1][dy]) * RX;
                        acc += w[1][dy] * w[2][dz] *
                               (w[0][0] * fld[c][row + ix[0][0]] +
                                w[0][1] * fld[c][row + ix[0][1]] +
                                w[0][2] * fld[c][row + ix[0][2]]);
                    }
                }
                U[c] = acc;
                up[c] = pp.up[c];
                om[c] = pp.om[c];
            }
        }
        // rigid-body velocity of the surface point, U_d = u_p + omega_p x r
        T Ud[3];
        Ud[0] = up[0] + (om[1] * rr[2] - om[2] * rr[1]);
        Ud[1] = up[1] + (om[2] * rr[0] - om[0] * rr[2]);
        Ud[2] = up[2] + (om[0] * rr[1] - om[1] * rr[0]);
        T dF[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            T slip = Ud[c] - U[c];
            res = max(res, fabs(slip));
            dF[c] = slip * a.inv_adt;
            fmax[c] = max(fmax[c], fabs(dF[c]));
        }
        if (a.probe)
            continue;
        if (a.pass == 0) {
            store4(a.Fl, m, dF[0], dF[1], dF[2]);
        } else {
            T F[3];
            load4(a.Fl, m, F);
            store4(a.Fl, m, F[0] + dF[0], F[1] + dF[1], F[2] + dF[2]);
            store4(a.dFl, m, dF[0], dF[1], dF[2]);
        }
    }
}

// block maxima of the slip and of |dF| per component, into the device words
// and (|dF|) the tile's words
template <typename T>
__device__ __forceinline__ void interp_block_max(const TileArgs<T> &a, T (&red)[4][kThreads / 32],
                                                 T res, T (&fmax)[3], int tile)
{
    const int tid = threadIdx.x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        res = max(res, __shfl_xor_sync(0xffffffffu, res, o));
#pragma unroll
        for (int c = 0; c < 3; c++)
            fmax[c] = max(fmax[c], __shfl_xor_sync(0xffffffffu, fmax[c], o));
    }
    if ((tid & 31) == 0) {
#pragma unroll
        for (int c = 0; c < 3; c++)
            red[c][tid >> 5] = fmax[c];
        red[3][tid >> 5] = res;
    }
    __syncthreads();
    if (tid < 4) {
        T r = T(0);
        for (int k = 0; k < kThreads / 32; k++)
            r = max(r, red[tid][k]);
        if (tid == kRedRes) {
            atomicMax(&a.red[kRedRes], max_bits(r));
        } else if (!a.probe) {
            atomicMax(&a.red[tid], max_bits(r));
            if (a.tile_fmax)
                a.tile_fmax[tile * 3 + tid] = max_bits(r);
        }
    }
}

template <typename T, bool SAME>
__global__ void __launch_bounds__(kThreads) k_interp_tiles(TileArgs<T> a)
{
    using Sm = SmemInterp<T, SAME>;
    constexpr int H = Sm::H, XO = Sm::XO, RX = Sm::RX, RY = Sm::RY, RZ = Sm::RZ, VW = Sm::VW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sm &sm = *reinterpret_cast<Sm *>(smem_raw);
    T *tRs = reinterpret_cast<T *>(smem_raw + sizeof(Sm));
    T *rRs = tRs + 3 * a.n_l;
    const int tid = threadIdx.x;
    const int tile = a.tiles ? a.tiles[blockIdx.x] : a.tile0 + (int)blockIdx.x;
    const int beg = a.key_start[tile * 27], end = a.key_start[tile * 27 + 27];
    if (beg == end)
        return;
    const int tc[3] = {tile % a.nt[0], (tile / a.nt[0]) % a.nt[1], tile / (a.nt[0] * a.nt[1])};
    const int te[3] = {TX, TY, TZ};
    int org[3];
    bool edge = false, clip = false;  // periodic image shifts / cells beyond a wall possible
#pragma unroll
    for (int k = 0; k < 3; k++) {
        org[k] = tc[k] * te[k];
        const bool at_end = tc[k] == 0 || tc[k] == a.nt[k] - 1;
        edge = edge || (at_end && a.periodic[k]);
        clip = clip || (at_end && !a.periodic[k]);
    }
    const int n_l = a.n_l;
    for (int i = tid; i < 3 * n_l; i += kThreads) {
        tRs[i] = a.tR[i];
        rRs[i] = a.rR[i];
    }

    // stage u, v, w on [org - margin, org + tile + margin) (zero beyond walls)
    const long long nx = a.n[0], nxy = (long long)a.n[0] * a.n[1];
    const int x0 = org[0] - XO;
    if (x0 >= 0 && x0 + RX <= a.n[0] && a.n[0] % VW == 0) {
        constexpr int RV = RX / VW;
        for (int v = tid; v < 3 * RZ * RY * RV; v += kThreads) {
            const int row = v / RV, xv = v - row * RV;
            const int c = row / (RZ * RY), rr = row - c * RZ * RY;
            const int z = rr / RY, y = rr - z * RY;
            int gy = org[1] - H + y, gz = org[2] - H + z;
            bool ok = true;
            if (gy < 0 || gy >= a.n[1]) {
                if (a.periodic[1])
                    gy = ((gy % a.n[1]) + a.n[1]) % a.n[1];
                else
                    ok = false;
            }
            if (gz < 0 || gz >= a.n[2]) {
                if (a.periodic[2])
                    gz = ((gz % a.n[2]) + a.n[2]) % a.n[2];
                else
                    ok = false;
            }
            // asynchronous 16-byte copy; rows beyond a wall are zero-filled
            T *dst = &sm.fld[c][(z * RY + y) * RX + xv * VW];
            const T *src = ok ? a.fld[c] + gz * nxy + gy * nx + x0 + xv * VW : a.fld[c];
            cp_async16(dst, src, ok);
        }
        cp_async_wait_all();
    } else {
        for (int i = tid; i < 3 * Sm::RN; i += kThreads) {
            const int c = i / Sm::RN;
            const int r = i - c * Sm::RN;
            const int rx = r % RX, ry = (r / RX) % RY, rz = r / (RX * RY);
            int g[3] = {x0 + rx, org[1] + ry - H, org[2] + rz - H};
            bool ok = true;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (g[k] < 0 || g[k] >= a.n[k]) {
                    if (a.periodic[k])
                        g[k] = ((g[k] % a.n[k]) + a.n[k]) % a.n[k];
                    else
                        ok = false;
                }
            }
            sm.fld[c][r] = ok ? __ldg(a.fld[c] + g[2] * nxy + g[1] * nx + g[0]) : T(0);
        }
    }
    __syncthreads();

    T res = T(0), fmax[3] = {T(0), T(0), T(0)};
    interp_tile_markers<T, SAME>(a, sm.fld, a.mlist + beg, end - beg, org, edge, clip, tRs, rRs,
                                 res, fmax);
    interp_block_max(a, sm.red, res, fmax, tile);
}

// ------------------------------------------------------------------ interpolation, TMA-staged
// Tiles whose staged block needs no periodic wrap (every tile not at the end
// of a periodic axis) go to a persistent kernel. Its blocks take the list of
// such tiles with markers in turn; one thread loads the next tile's u, v, w
// blocks with TMA tensor copies (cp.async.bulk.tensor, zero fill beyond the
// walls) into the second of two buffers while the block interpolates the
// current tile, so the copy latency hides behind the gathers. Every wait on
// the copies is bounded: on timeout the block sets ERRB_TMA_TIMEOUT, waits
// (bounded) for its copies in flight and stops.
struct FieldMaps {
    CUtensorMap m[3];  // u, v, w as 3-D tensors, boxes of the staged block
};

constexpr long long kTmaSpin = 1LL << 22;

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = smem_addr(bar);
    for (long long it = 0; it < kTmaSpin; it++) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok)
            return true;
        if (it > 16)
            __nanosleep(32);
    }
    return false;
}

// the three field boxes of `tile` into buffer `fld`; completion on `bar`
template <typename T, bool SAME>
__device__ __forceinline__ void tma_stage(const FieldMaps &fm, const TileArgs<T> &a, int tile,
                                          T (&fld)[3][SmemInterp<T, SAME>::RN], uint64_t *bar,
                                          uint32_t extra_bytes = 0)
{
    using Sm = SmemInterp<T, SAME>;
    const int tx = tile % a.nt[0], ty = (tile / a.nt[0]) % a.nt[1],
              tz = tile / (a.nt[0] * a.nt[1]);
    const int x0 = tx * TX - Sm::XO, y0 = ty * TY - Sm::H, z0 = tz * TZ - Sm::H;
    const uint32_t b = smem_addr(bar);
    const uint32_t bytes = 3u * Sm::RN * sizeof(T) + extra_bytes;  // + other copies on bar
    // the buffer was last read by generic loads of the block
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes)
                 : "memory");
#pragma unroll
    for (int c = 0; c < 3; c++)
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(&fld[c][0])),
            "l"(reinterpret_cast<uint64_t>(&fm.m[c])), "r"(x0), "r"(y0), "r"(z0), "r"(b)
            : "memory");
}

// One producer warp issues the copies; eight consumer warps interpolate.
// Buffer b has a "full" barrier (the tensor copies' bytes) and an "empty"
// barrier (one arrival per consumer warp once it has read the buffer), so
// the warps never wait for each other at a tile's end: a warp that finishes
// its share of a tile goes on to the next one as soon as its data is in.
constexpr int kTmaConsumerWarps = kThreads / 32;
constexpr int kTmaThreads = kThreads + 32;

template <typename T, bool SAME>
struct SmemInterpTma {
    using B = SmemInterp<T, SAME>;
    T fld[2][3][B::RN];  // two staged blocks (each component 128-byte aligned)
    // the tile's marker ids, copied with the fields when they fit (the
    // copy starts at the 16-byte boundary at or below the tile's first id)
    static constexpr int kIdCap = 1536;
    int ids[2][kIdCap];
    int id_off[2], id_n[2], id_beg[2];  // offset into ids (-1: read them from global), count, first
    uint64_t full[2], empty[2];
    int issued[2];       // copies issued into each buffer
    int wr[2];           // the launch's positions [wr[0], wr[1]) in the tile list
    T red[4][kTmaConsumerWarps];
    volatile int abort;
    // the marker template follows: tR[3][n_l], rR[3][n_l]
};

__device__ __forceinline__ void mbar_init_count(uint64_t *bar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// bounded wait that also gives up once another warp has aborted
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t *bar, uint32_t parity,
                                                   volatile int *abort)
{
    const uint32_t a = smem_addr(bar);
    for (long long it = 0; it < kTmaSpin; it++) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok)
            return true;
        if (*abort)
            return false;
        if (it > 16)
            __nanosleep(32);
    }
    return false;
}

template <typename T, bool SAME>
__global__ void __launch_bounds__(kTmaThreads)
k_interp_tma(TileArgs<T> a, const __grid_constant__ FieldMaps fm, const int *__restrict__ list,
             const int *__restrict__ count, int t_lo, int t_hi)
{
    using Sm = SmemInterpTma<T, SAME>;
    static_assert((SmemInterp<T, SAME>::RN * sizeof(T)) % 128 == 0, "128-byte aligned boxes");
    extern __shared__ __align__(128) unsigned char smem_tma[];
    Sm &sm = *reinterpret_cast<Sm *>(smem_tma);
    T *tRs = reinterpret_cast<T *>(smem_tma + sizeof(Sm));
    T *rRs = tRs + 3 * a.n_l;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        // the listed tiles in [t_lo, t_hi): the list is in ascending order
        const int n = *count;
        for (int e = 0; e < 2; e++) {
            const int t = e ? t_hi : t_lo;
            int lo = 0, hi = n;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (list[mid] < t)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            sm.wr[e] = lo;
        }
    }
    __syncthreads();
    const int w_lo = sm.wr[0], n_work = sm.wr[1];
    if (w_lo + (int)blockIdx.x >= n_work)
        return;
    for (int i = tid; i < 3 * a.n_l; i += kTmaThreads) {
        tRs[i] = a.tR[i];
        rRs[i] = a.rR[i];
    }
    if (tid == 0) {
        for (int b = 0; b < 2; b++) {
            mbar_init_count(&sm.full[b], 1);
            mbar_init_count(&sm.empty[b], kTmaConsumerWarps);
            sm.issued[b] = 0;
        }
        sm.abort = 0;
    }
    __syncthreads();
    T res = T(0), fmax[3] = {T(0), T(0), T(0)};
    if (warp == kTmaConsumerWarps) {
        // producer: tile i goes to buffer i & 1 once the consumers are done
        // with tile i - 2
        if (lane == 0) {
            int i = 0;
            for (int w = w_lo + blockIdx.x; w < n_work && !sm.abort; w += gridDim.x, i++) {
                const int buf = i & 1;
                if (i >= 2 && !mbar_wait_or_abort(&sm.empty[buf], ((i - 2) >> 1) & 1, &sm.abort)) {
                    if (!sm.abort)
                        atomicOr(a.err, ERRB_TMA_TIMEOUT);
                    sm.abort = 1;
                    break;
                }
                const int tile = list[w];
                const int beg = a.key_start[tile * 27], end = a.key_start[tile * 27 + 27];
                const int a0 = beg & ~3, a1 = (end + 3) & ~3;  // mlist is padded by 4 ids
                const bool fit = a1 - a0 <= Sm::kIdCap;
                sm.id_off[buf] = fit ? beg - a0 : -1;
                sm.id_n[buf] = end - beg;
                sm.id_beg[buf] = beg;
                tma_stage<T, SAME>(fm, a, tile, sm.fld[buf], &sm.full[buf],
                                   fit ? (uint32_t)(4 * (a1 - a0)) : 0u);
                if (fit && a1 > a0)
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes"
                        " [%0], [%1], %2, [%3];" ::"r"(smem_addr(&sm.ids[buf][0])),
                        "l"(a.mlist + a0), "r"(4 * (a1 - a0)), "r"(smem_addr(&sm.full[buf]))
                        : "memory");
                sm.issued[buf] += 1;
            }
        }
    } else {
        int i = 0;
        for (int w = w_lo + blockIdx.x; w < n_work; w += gridDim.x, i++) {
            const int buf = i & 1;
            // every lane waits (acquiring the copied bytes); the warp goes on
            // only if all of them saw the copy complete
            const bool got = mbar_wait_or_abort(&sm.full[buf], (i >> 1) & 1, &sm.abort);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0 && !sm.abort)
                    atomicOr(a.err, ERRB_TMA_TIMEOUT);
                sm.abort = 1;
                break;
            }
            const int tile = list[w];
            const int tc[3] = {tile % a.nt[0], (tile / a.nt[0]) % a.nt[1],
                               tile / (a.nt[0] * a.nt[1])};
            const int te[3] = {TX, TY, TZ};
            int org[3];
            bool clip = false;  // listed tiles sit at no periodic end
#pragma unroll
            for (int k = 0; k < 3; k++) {
                org[k] = tc[k] * te[k];
                clip = clip || ((tc[k] == 0 || tc[k] == a.nt[k] - 1) && !a.periodic[k]);
            }
            const int off = sm.id_off[buf];
            const int *ml = off >= 0 ? &sm.ids[buf][off] : a.mlist + sm.id_beg[buf];
            T ft[3] = {T(0), T(0), T(0)};
            interp_tile_markers<T, SAME>(a, sm.fld[buf], ml, sm.id_n[buf], org, false, clip,
                                         tRs, rRs, res, ft);
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&sm.empty[buf]);
            // the tile's maxima: one atomic per warp and component (the bit
            // patterns of non-negative values order like the values)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                fmax[c] = max(fmax[c], ft[c]);
                const unsigned long long b = warp_max_bits(ft[c]);
                if (lane == 0 && a.tile_fmax && !a.probe && b != 0ULL)
                    atomicMax(&a.tile_fmax[tile * 3 + c], b);
            }
        }
    }
    __syncthreads();
    if (sm.abort) {
        // no copy into this block's shared memory may outlive it: wait
        // (bounded) for the last one issued into each buffer
        if (tid == 0)
            for (int b = 0; b < 2; b++)
                if (sm.issued[b] > 0)
                    mbar_wait_bounded(&sm.full[b], (uint32_t)((sm.issued[b] - 1) & 1));
        return;
    }
    // block maxima over the consumer warps
    if (warp < kTmaConsumerWarps) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            res = max(res, __shfl_xor_sync(0xffffffffu, res, o));
#pragma unroll
            for (int c = 0; c < 3; c++)
                fmax[c] = max(fmax[c], __shfl_xor_sync(0xffffffffu, fmax[c], o));
        }
        if (lane == 0) {
#pragma unroll
            for (int c = 0; c < 3; c++)
                sm.red[c][warp] = fmax[c];
            sm.red[3][warp] = res;
        }
    }
    __syncthreads();
    if (tid < 4) {
        T r = T(0);
        for (int k = 0; k < kTmaConsumerWarps; k++)
            r = max(r, sm.red[tid][k]);
        if (tid == kRedRes)
            atomicMax(&a.red[kRedRes], max_bits(r));
        else if (!a.probe)
            atomicMax(&a.red[tid], max_bits(r));
    }
}

// Non-empty tiles split for the two interpolation kernels: the tiles at no
// periodic end go, in tile order, into `list` (so that the persistent
// kernel's blocks work on neighbouring tiles together and share their halos
// in L2); the others are the static edge list. Pass 0 writes a flag per
// tile, an exclusive scan gives the positions, pass 1 scatters.
__global__ void k_tile_list(const int *__restrict__ key_start, int ntile, int nt0, int nt1,
                            int nt2, int per0, int per1, int per2, int pass,
                            int *__restrict__ flag, const int *__restrict__ pos,
                            int *__restrict__ list, int *__restrict__ count)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > ntile)
        return;
    if (pass == 1) {
        if (t == ntile)
            *count = pos[ntile];
        else if (flag[t])
            list[pos[t]] = t;
        return;
    }
    bool take = false;
    if (t < ntile) {
        const int tx = t % nt0, ty = (t / nt0) % nt1, tz = t / (nt0 * nt1);
        const bool edge = (per0 && (tx == 0 || tx == nt0 - 1)) ||
                          (per1 && (ty == 0 || ty == nt1 - 1)) ||
                          (per2 && (tz == 0 || tz == nt2 - 1));
        take = !edge && key_start[t * 27] < key_start[t * 27 + 27];
    }
    flag[t] = take ? 1 : 0;
}

// ------------------------------------------------------------------ per-particle sums
// kSumLanes lanes per particle, each with compensated sums over every
// kSumLanes-th marker, merged in a fixed order: few shuffles per particle,
// and each group of lanes reads consecutive marker records.
constexpr int kSumLanes = 4;

template <typename T>
__global__ void __launch_bounds__(256)
k_particle_sums(const T *__restrict__ Fl, const T *__restrict__ rR, int n_p, int n_l,
                double neg_rho_dV, double *__restrict__ Fh, double *__restrict__ Th)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int p = (int)(g / kSumLanes);
    const int sub = (int)(g - (long long)p * kSumLanes);
    const bool valid = p < n_p;  // the others join the shuffles only
    KSum<T> fs[3], ts[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        fs[k].init();
        ts[k].init();
    }
    for (int l = sub; valid && l < n_l; l += kSumLanes) {
        T F[3];
        load4(Fl, (long long)p * n_l + l, F);
        T r0 = __ldg(rR + l), r1 = __ldg(rR + n_l + l), r2 = __ldg(rR + 2 * n_l + l);
        fs[0].add(F[0]);
        fs[1].add(F[1]);
        fs[2].add(F[2]);
        ts[0].add(r1 * F[2] - r2 * F[1]);
        ts[1].add(r2 * F[0] - r0 * F[2]);
        ts[2].add(r0 * F[1] - r1 * F[0]);
    }
#pragma unroll
    for (int o = kSumLanes / 2; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            T s2 = __shfl_xor_sync(0xffffffffu, fs[k].s, o);
            T c2 = __shfl_xor_sync(0xffffffffu, fs[k].c, o);
            fs[k].merge(s2, c2);
            s2 = __shfl_xor_sync(0xffffffffu, ts[k].s, o);
            c2 = __shfl_xor_sync(0xffffffffu, ts[k].c, o);
            ts[k].merge(s2, c2);
        }
    }
    if (valid && sub == 0) {
        const T f = (T)neg_rho_dV;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            Fh[k * n_p + p] = (double)(f * (fs[k].s - fs[k].c));
            Th[k * n_p + p] = (double)(f * (ts[k].s - ts[k].c));
        }
    }
}

template <typename T>
void particle_sums_launch(Ctx &c, cudaStream_t s)
{
    k_particle_sums<T><<<(int)(((long long)c.n_p * kSumLanes + 255) / 256), 256, 0, s>>>(
        (const T *)c.Fl, (const T *)c.rR, c.n_p, c.n_l, -c.rho_f * c.dV, c.Fh, c.Th);
    c.n_launch += 1;
}

// ------------------------------------------------------------------ spreading
// A tile needs the markers whose stencils reach it: its own markers and,
// from each of the 26 neighbours, the face classes next to it (bins within
// one cell, two on staggered grids). Every such marker adds
// F phi phi phi dV / h^3 for each of its stencil cells inside the tile to a
// shared-memory accumulator in fixed point (32-bit integers for the FP32
// form, 64-bit for FP64). Integer addition is associative, so the sums, and
// the fields written from them, are bit-identical whatever the order in
// which threads and markers arrive: deterministic spreading without
// floating-point atomics. The fixed-point scale is a power of two chosen per
// tile from the largest force of the markers binned in the tile and its 26
// neighbours (recorded per tile by the interpolation) and from the bin
// count, so no sum can overflow. Being local, the bound lets the lower tile
// layers be spread before the upper ones are interpolated.
// Fixed point: every contribution is scaled by a power of two 2^s and
// rounded to an integer. FP32 form: one 32-bit word per cell and component,
// s chosen from the tile's largest bin count so that no cell's sum can reach
// 2^30. FP64 form: one 64-bit word (64-bit shared atomics are slower, but the
// FP64 form is bound by FP64 arithmetic), every contribution below 2^(62 - K)
// with K bits for the tile's marker count.

template <typename T, bool SAME>
struct SmemSpread {
    static constexpr int W = SAME ? 1 : 2;   // face class width (component-0 bins)
    static constexpr int kRanges = 27 * 27;
    static constexpr int BX = TX + 2 * W, BY = TY + 2 * W, BZ = TZ + 2 * W;
    static constexpr int NB = BX * BY * BZ;  // component-0 bins around the tile
    // accumulators with padded rows and planes: the stencil cells of the
    // markers that run side by side in a warp spread over more banks
    static constexpr int PY = 19, PZ = 153, PC = PZ * TZ;
    static constexpr bool W64 = sizeof(T) == 8;
    int acc32[W64 ? 1 : 3 * PC];             // FP32 form
    long long acc64[W64 ? 3 * PC : 1];       // FP64 form
    int binc[NB];
    int sh[3];      // fixed-point exponent per component
    T cscale[3];    // 2^sh dV/h^3 per component
    T tfmax[3];     // max |F| per component over the markers binned in the 27 tiles around
    int org[3];     // the tile's first cell (read from here in the loops: registers are short)
    int scan_tmp[kThreads / 32];
    static constexpr int kVisCap = 2048;  // markers kept by the first pass (sphere lists)
    int vis[kVisCap];
    int nvis;
    static constexpr int kSphCap = 160;
    union {
        // (neighbour, class) ranges of the binned markers (no sphere lists)
        struct {
            int rbeg[kRanges], roff[kRanges + 1];
            Nb nb;
        };
        // the tile's spheres (sphere lists): id, component-0 base and
        // remainder, and the marker range [l0, l1) whose bins can lie in the
        // tile's z-range
        struct {
            int sph_p[kSphCap];
            int sph_b[kSphCap][3];
            T sph_fr[kSphCap][3];
            int sph_l[kSphCap][2];
        };
    };
    // the marker template follows: tR[3][n_l]
};

template <typename T, bool SAME>
__device__ __forceinline__ void particle_base(const TileArgs<T> &a, int p, int cp, int b[3],
                                              T fr[3])
{
    if (SAME) {
        const PartFast<T> rec = a.pfast[p];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            b[k] = rec.b[k];
            fr[k] = rec.fr[k];
        }
    } else {
        const PartPrep<T> &pp = a.prep[p];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            b[k] = pp.base[cp * 3 + k];
            fr[k] = pp.frac[cp * 3 + k];
        }
    }
}

template <typename T, bool SAME>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 5 : 2) k_spread_tiles(TileArgs<T> a)
{
    using Sm = SmemSpread<T, SAME>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sm &sm = *reinterpret_cast<Sm *>(smem_raw);
    T *tRs = reinterpret_cast<T *>(smem_raw + sizeof(Sm));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = a.tile0 + blockIdx.x;
    const int tc[3] = {tile % a.nt[0], (tile / a.nt[0]) % a.nt[1], tile / (a.nt[0] * a.nt[1])};
    const int te[3] = {TX, TY, TZ};
    const int bdim[3] = {Sm::BX, Sm::BY, Sm::BZ};
    int org[3], ext[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        org[k] = tc[k] * te[k];
        ext[k] = min(te[k], a.n[k] - org[k]);
    }
    if (tid == 0) {
        sm.org[0] = org[0];
        sm.org[1] = org[1];
        sm.org[2] = org[2];
    }
    // the markers whose stencils can reach this tile: the markers of the
    // spheres in its list, or the (neighbour, class) ranges of the binned lists
    const bool vis = a.pt_start != nullptr;
    int vbase = 0, nsph = 0;
    if (vis) {
        vbase = a.pt_start[tile];
        nsph = a.pt_start[tile + 1] - vbase;
    } else {
        gather_neighbours(a, tc, sm.nb);
    }
    for (int r = tid; r < (vis ? 0 : Sm::kRanges); r += kThreads) {
        const int k = r / 27, cls = r - k * 27;
        const int key = sm.nb.key[k];
        int beg = 0, cnt = 0;
        if (key >= 0) {
            const int d[3] = {k % 3 - 1, (k / 3) % 3 - 1, k / 9 - 1};
            const int cc[3] = {cls % 3, (cls / 3) % 3, cls / 9};
            bool use = true;
#pragma unroll
            for (int ax = 0; ax < 3; ax++) {
                int lo, hi;
                class_range(cc[ax], sm.nb.ext[k][ax], Sm::W, lo, hi);
                if (lo >= hi)
                    use = false;
                else if (d[ax] < 0)   // neighbour below: its top W layers
                    use = use && hi > sm.nb.ext[k][ax] - Sm::W;
                else if (d[ax] > 0)   // neighbour above: its bottom W layers
                    use = use && lo < Sm::W;
            }
            if (use) {
                beg = a.key_start[key * 27 + cls];
                cnt = a.key_start[key * 27 + cls + 1] - beg;
            }
        }
        sm.rbeg[r] = beg;
        sm.roff[r] = cnt;  // counts first, offsets below
    }
    __syncthreads();
    if (!vis) {
        constexpr int per = (Sm::kRanges + kThreads - 1) / kThreads;
        const int r0 = tid * per;
        int cnt[per];
        int s = 0;
#pragma unroll
        for (int q = 0; q < per; q++) {
            cnt[q] = r0 + q < Sm::kRanges ? sm.roff[r0 + q] : 0;
            s += cnt[q];
        }
        int total;
        int excl = block_excl_scan(s, sm.scan_tmp, &total);
#pragma unroll
        for (int q = 0; q < per; q++)
            if (r0 + q < Sm::kRanges) {
                sm.roff[r0 + q] = excl;
                excl += cnt[q];
            }
        if (tid == 0)
            sm.roff[Sm::kRanges] = total;
    }
    __syncthreads();
    int total = vis ? nsph * a.n_l : sm.roff[Sm::kRanges];
    T fmax[3];
#pragma unroll
    for (int c = 0; c < 3; c++)
        fmax[c] = from_bits_t<T>(a.red[c]);  // all |dF| so far: zero means nothing to add
    if (total == 0 || !(max(fmax[0], max(fmax[1], fmax[2])) > T(0)))
        return;
    constexpr bool W64 = Sm::W64;
    const int n_l = a.n_l;
    // sphere lists with few enough spheres: their records go to shared memory
    const bool staged = vis && nsph <= Sm::kSphCap;
    for (int i = tid; i < 3 * n_l; i += kThreads)
        tRs[i] = a.tR[i];
    for (int i = tid; i < 3 * Sm::PC; i += kThreads) {
        if (W64)
            sm.acc64[W64 ? i : 0] = 0LL;
        else
            sm.acc32[W64 ? 0 : i] = 0;
    }
    for (int i = tid; i < Sm::NB; i += kThreads)
        sm.binc[i] = 0;
    if (staged) {
        for (int j = tid; j < nsph; j += kThreads) {
            const int p = a.pt_list[vbase + j];
            const PartFast<T> rec = a.pfast[p];
            sm.sph_p[j] = p;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                sm.sph_b[j][k] = rec.b[k];
                sm.sph_fr[j][k] = rec.fr[k];
            }
        }
    }
    // bound of the marker forces that can reach this tile: the maxima of the
    // markers binned in it and its 26 neighbours (a marker reaches the tile
    // only from a bin within W < tile size of it); by the last warp, which
    // stages no sphere record when the records are staged
    if (warp == kThreads / 32 - 1 && a.tile_fmax) {
        T m[3] = {T(0), T(0), T(0)};
        if (lane < 27) {
            const int d[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
            int t[3];
            bool in = true;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                t[k] = tc[k] + d[k];
                if (t[k] < 0 || t[k] >= a.nt[k]) {
                    if (a.periodic[k])
                        t[k] = t[k] < 0 ? t[k] + a.nt[k] : t[k] - a.nt[k];
                    else
                        in = false;
                }
            }
            if (in) {
                const long long q = 3LL * (t[0] + a.nt[0] * (t[1] + a.nt[1] * t[2]));
#pragma unroll
                for (int c = 0; c < 3; c++)
                    m[c] = from_bits_t<T>(a.tile_fmax[q + c]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < 3; c++)
                m[c] = max(m[c], __shfl_xor_sync(0xffffffffu, m[c], o));
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < 3; c++)
                sm.tfmax[c] = m[c];
    }
    if (tid == 0)
        sm.nvis = 0;
    __syncthreads();

    const T *Fsrc = a.pass == 0 ? a.Fl : a.dFl;
    // shift that maps the marker's grid index ub to tile coordinates, on
    // the periodic image next to the tile
    auto tile_shift = [&](int k, int ax, int ub) -> int {
        if (vis) {
            int r = ub - sm.org[ax];
            if (a.periodic[ax]) {
                if (r < -Sm::W)
                    r += a.n[ax];
                else if (r >= ext[ax] + Sm::W)
                    r -= a.n[ax];
            }
            return r - ub;
        }
        int s2 = sm.nb.shift[k][ax] - sm.org[ax];
        if (a.periodic[ax])
            s2 += ub < 0 ? a.n[ax] : (ub >= a.n[ax] ? -a.n[ax] : 0);
        return s2;
    };
    // component-0 bin of marker l around the tile (bins of the tile and its
    // W-wide margin are [0, B) per axis)
    auto bins = [&](const int (&pb0)[3], const T (&fr0)[3], int l, int k, int (&bb)[3]) -> bool {
        bool in = true;
#pragma unroll
        for (int ax = 0; ax < 3; ax++) {
            const int ub = pb0[ax] + (int)floor(fr0[ax] + tRs[ax * n_l + l] + T(0.5));
            bb[ax] = ub + tile_shift(k, ax, ub) + Sm::W;
            in = in && bb[ax] >= 0 && bb[ax] < bdim[ax];
        }
        return in;
    };
    auto staged_sphere = [&](int j, int (&pb0)[3], T (&fr0)[3]) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            pb0[k] = sm.sph_b[j][k];
            fr0[k] = sm.sph_fr[j][k];
        }
    };
    if (staged) {
        // Markers of a sphere whose bins can lie in the tile's z-range: the
        // template's z-components fall with l, so on a bounded z-axis the
        // bins do too and the range is an interval [l0, l1) of l.
        for (int j = tid; j < nsph; j += kThreads) {
            int l0 = 0, l1 = n_l;
            if (!a.periodic[2]) {
                const int b0 = sm.sph_b[j][2] - org[2] + Sm::W;
                const T f0 = sm.sph_fr[j][2];
                auto bz = [&](int l) { return b0 + (int)floor(f0 + tRs[2 * n_l + l] + T(0.5)); };
                int lo = 0, hi = n_l;  // first l with bz(l) < BZ
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (bz(mid) < Sm::BZ)
                        hi = mid;
                    else
                        lo = mid + 1;
                }
                l0 = lo;
                hi = n_l;  // first l with bz(l) < 0
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (bz(mid) < 0)
                        hi = mid;
                    else
                        lo = mid + 1;
                }
                l1 = lo;
            }
            sm.sph_l[j][0] = l0;
            sm.sph_l[j][1] = l1;
        }
        __syncthreads();
    }
    // Bound of every cell's sum. A marker in bin b (the cell nearest to it
    // in component-0 coordinates) reaches cell j of any component only if
    // each |b - j| <= 1 (<= 2 on staggered grids), with a weight per axis of
    // at most 1/2, 2/3, 1/2 over those offsets (1/6, 2/3, 2/3, 1/6 on a
    // half-cell shifted axis): 5/3 per axis in both cases. So with maxbin
    // markers in the fullest bin, |sum_c| <= maxbin (5/3)^3 fmax_c dV/h^3.
    int maxbin = 0;
    auto keep_marker = [&](bool in, const int (&bb)[3], unsigned act, int entry) {
        if (in && !W64)
            atomicAdd(&sm.binc[(bb[2] * Sm::BY + bb[1]) * Sm::BX + bb[0]], 1);
        // warp-aggregated slot in the list of kept markers
        const unsigned keep = __ballot_sync(act, in);
        const int lead = __ffs(act) - 1;
        int base = 0;
        if (lane == lead && keep)
            base = atomicAdd(&sm.nvis, __popc(keep));
        base = __shfl_sync(act, base, lead);
        const int slot = base + __popc(keep & ((1u << lane) - 1u));
        if (in && slot < Sm::kVisCap)
            sm.vis[slot] = entry;
    };
    if (staged) {
        // one warp per sphere; a kept marker is recorded as (j << 16) | l
        for (int j = warp; j < nsph; j += kThreads / 32) {
            int pb0[3];
            T fr0[3];
            staged_sphere(j, pb0, fr0);
            const int l0 = sm.sph_l[j][0], l1 = sm.sph_l[j][1];
            for (int l = l0 + lane; l - lane < l1; l += 32) {
                int bb[3];
                const bool in = l < l1 && bins(pb0, fr0, l, 13, bb);
                keep_marker(in, bb, 0xffffffffu, (j << 16) | l);
            }
        }
    } else if (!W64 || vis) {
        for (int g = tid; g < total; g += kThreads) {
            int m, k = 13;
            if (vis) {
                const int j = (int)__umul64hi((unsigned long long)g, a.l_magic);
                m = a.pt_list[vbase + j] * n_l + (g - j * n_l);
            } else {
                int lo = 0, hi = Sm::kRanges;  // last range with roff <= g
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (sm.roff[mid] <= g)
                        lo = mid;
                    else
                        hi = mid;
                }
                m = a.mlist[sm.rbeg[lo] + (g - sm.roff[lo])];
                k = lo / 27;
            }
            const int p = (int)__umul64hi((unsigned long long)m, a.l_magic);
            const int l = m - p * n_l;
            int pb0[3];
            T fr0[3];
            particle_base<T, SAME>(a, p, 0, pb0, fr0);
            int bb[3];
            const bool in = bins(pb0, fr0, l, k, bb);
            if (vis)
                keep_marker(in, bb, __activemask(), m);
            else if (in && !W64)
                atomicAdd(&sm.binc[(bb[2] * Sm::BY + bb[1]) * Sm::BX + bb[0]], 1);
        }
    }
    __syncthreads();
    if (!W64) {
        for (int i = tid; i < Sm::NB; i += kThreads)
            maxbin = max(maxbin, sm.binc[i]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            maxbin = max(maxbin, __shfl_xor_sync(0xffffffffu, maxbin, o));
        if (lane == 0)
            sm.scan_tmp[warp] = maxbin;
        __syncthreads();
        maxbin = 0;
        if (tid < 3)
            for (int k = 0; k < kThreads / 32; k++)
                maxbin = max(maxbin, sm.scan_tmp[k]);
    }
    const int nvis = sm.nvis;
    const bool compact = vis && nvis <= Sm::kVisCap;
    // the scales, in FP64 by one thread per component (FP64 is slow here)
    if (tid < 3) {
        const int c = tid;
        const T fm = a.tile_fmax ? sm.tfmax[c] : fmax[c];
        int ex;
        if (W64) {
            // 64-bit words: every contribution below 2^(62 - K), K bits for the markers
            const int K = 32 - __clz(vis ? nvis : total);
            frexp((8.0 / 27.0) * (double)fm * a.dVh3, &ex);
            sm.sh[c] = 62 - K - ex;
        } else {
            frexp((125.0 / 27.0) * (double)max(maxbin, 1) * (double)fm * a.dVh3, &ex);
            sm.sh[c] = 30 - ex;
        }
        sm.cscale[c] = fm > T(0) ? (T)ldexp(a.dVh3, sm.sh[c]) : T(0);
    }
    __syncthreads();
    // the scales stay in shared memory (broadcast reads): registers are the
    // accumulation loop's limit
    // contributions of marker m = p n_l + l (component-0 base pb0, fr0),
    // reaching the tile through neighbour k
    auto accumulate = [&](long long m, int p, int l, int k, const int (&pb0)[3],
                          const T (&fr0)[3]) {
        T rt[3];
#pragma unroll
        for (int ax = 0; ax < 3; ax++)
            rt[ax] = tRs[ax * n_l + l];
        int shift[3];
#pragma unroll
        for (int ax = 0; ax < 3; ax++) {
            // image of the particle that holds this marker next to the tile
            const int ub = pb0[ax] + (int)floor(fr0[ax] + rt[ax] + T(0.5));
            shift[ax] = tile_shift(k, ax, ub);
        }
        T F[3];
        load4(Fsrc, m, F);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            int pb[3];
            T fr[3];
            if (SAME) {
                if (c > 0)
                    break;
#pragma unroll
                for (int ax = 0; ax < 3; ax++) {
                    pb[ax] = pb0[ax];
                    fr[ax] = fr0[ax];
                }
            } else {
                particle_base<T, SAME>(a, p, c, pb, fr);
            }
            int lo3[3];
            T w[3][3];
#pragma unroll
            for (int ax = 0; ax < 3; ax++) {
                int i0;
                axis_weights_fast(fr[ax] + rt[ax], i0, w[ax]);
                lo3[ax] = pb[ax] + shift[ax] + i0 - 1;
            }
            const int c0 = SAME ? 0 : c, c1 = SAME ? 3 : c + 1;
            T Fs[3];
#pragma unroll
            for (int q = 0; q < 3; q++)
                Fs[q] = F[q] * sm.cscale[q];
#pragma unroll
            for (int dz = 0; dz < 3; dz++) {
                const int z = lo3[2] + dz;
                if (z < 0 || z >= ext[2])
                    continue;
#pragma unroll
                for (int dy = 0; dy < 3; dy++) {
                    const int y = lo3[1] + dy;
                    if (y < 0 || y >= ext[1])
                        continue;
                    const T wyz = w[1][dy] * w[2][dz];
#pragma unroll
                    for (int dx = 0; dx < 3; dx++) {
                        const int x = lo3[0] + dx;
                        if (x < 0 || x >= ext[0])
                            continue;
                        const int cell = z * Sm::PZ + y * Sm::PY + x;
                        const T wgt = wyz * w[0][dx];
                        for (int cc = c0; cc < c1; cc++) {
                            if (W64)
                                atomicAdd(reinterpret_cast<unsigned long long *>(
                                              &sm.acc64[W64 ? cc * Sm::PC + cell : 0]),
                                          (unsigned long long)__double2ll_rn(
                                              (double)(Fs[cc] * wgt)));
                            else
                                atomicAdd(&sm.acc32[W64 ? 0 : cc * Sm::PC + cell],
                                          __float2int_rn((float)(Fs[cc] * wgt)));
                        }
                    }
                }
            }
        }
    };
    if (compact) {
        for (int g = tid; g < nvis; g += kThreads) {
            const int e = sm.vis[g];
            int pb0[3];
            T fr0[3];
            int p, l;
            if (staged) {
                const int j = e >> 16;
                l = e & 0xffff;
                p = sm.sph_p[j];
                staged_sphere(j, pb0, fr0);
            } else {
                p = (int)__umul64hi((unsigned long long)e, a.l_magic);
                l = e - p * n_l;
                particle_base<T, SAME>(a, p, 0, pb0, fr0);
            }
            accumulate((long long)p * n_l + l, p, l, 13, pb0, fr0);
        }
    } else if (staged) {
        // more kept markers than the list holds: test them again
        for (int j = warp; j < nsph; j += kThreads / 32) {
            int pb0[3];
            T fr0[3];
            staged_sphere(j, pb0, fr0);
            const int p = sm.sph_p[j];
            for (int l = sm.sph_l[j][0] + lane; l < sm.sph_l[j][1]; l += 32) {
                int bb[3];
                if (bins(pb0, fr0, l, 13, bb))
                    accumulate((long long)p * n_l + l, p, l, 13, pb0, fr0);
            }
        }
    } else {
        for (int g = tid; g < total; g += kThreads) {
            int m, k = 13;
            if (vis) {
                const int j = (int)__umul64hi((unsigned long long)g, a.l_magic);
                m = a.pt_list[vbase + j] * n_l + (g - j * n_l);
            } else {
                int lo = 0, hi = Sm::kRanges;  // last range with roff <= g
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (sm.roff[mid] <= g)
                        lo = mid;
                    else
                        hi = mid;
                }
                m = a.mlist[sm.rbeg[lo] + (g - sm.roff[lo])];
                k = lo / 27;
            }
            const int p = (int)__umul64hi((unsigned long long)m, a.l_magic);
            const int l = m - p * n_l;
            int pb0[3];
            T fr0[3];
            particle_base<T, SAME>(a, p, 0, pb0, fr0);
            int bb[3];
            // sphere lists cover some markers out of reach: skip them
            if (!vis || bins(pb0, fr0, l, k, bb))
                accumulate(m, p, l, k, pb0, fr0);
        }
    }
    __syncthreads();

    // read-modify-write of f and u on the cells with a nonzero sum (the
    // others would not change): all loads of a thread's cells first, so
    // that they are in flight together, then the stores
    const long long nx = a.n[0], nxy = (long long)a.n[0] * a.n[1];
    const T adt = (T)a.adt;
    T vf[kCellsPerThread][3], vu[kCellsPerThread][3], dv[kCellsPerThread][3];
    long long gi[kCellsPerThread];
    bool on[kCellsPerThread][3];
#pragma unroll
    for (int q = 0; q < kCellsPerThread; q++) {
        const int cell = tid + q * kThreads;
        const int cx = cell % TX, cy = (cell / TX) % TY, cz = cell / (TX * TY);
        const int pc = cz * Sm::PZ + cy * Sm::PY + cx;
        const bool inside = cx < ext[0] && cy < ext[1] && cz < ext[2];
        gi[q] = (sm.org[2] + cz) * nxy + (sm.org[1] + cy) * nx + (sm.org[0] + cx);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            long long iv;
            if (W64)
                iv = sm.acc64[W64 ? c * Sm::PC + pc : 0];
            else
                iv = sm.acc32[W64 ? 0 : c * Sm::PC + pc];
            on[q][c] = inside && iv != 0;
            dv[q][c] = W64 ? (T)ldexp((double)iv, -sm.sh[c]) : ldexp((T)(int)iv, -sm.sh[c]);
            if (on[q][c]) {
                vf[q][c] = a.out_f[c][gi[q]];
                vu[q][c] = a.out_u[c][gi[q]];
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kCellsPerThread; q++)
#pragma unroll
        for (int c = 0; c < 3; c++)
            if (on[q][c]) {
                a.out_f[c][gi[q]] = vf[q][c] + dv[q][c];
                a.out_u[c][gi[q]] = vu[q][c] + adt * dv[q][c];
            }
}

// ------------------------------------------------------------------ spreading, bank-bucketed
// FP32 form with all components on the cell centres. A block takes a
// super-tile of 2 x 2 x 1 tiles (32 x 16 x 8 cells) and every marker whose
// stencil can reach it: the markers binned in its own tiles and, from the
// tiles around it, those in the face classes next to it. Its shared
// accumulators cover x in [-2, 32) with rows of 34 words, y in [-1, 17)
// with planes of 18 rows, z in [-1, 9), plus guard words at both ends: every
// stencil cell of a marker whose nearest cell lies within one cell of the
// super-tile falls in the array, outside the super-tile only in padding
// (rows that leave it wrap into the padding of the next row or plane). So
// every marker adds all 81 contributions without a test; the padding is
// never written back. A stencil offset moves every cell of a warp by the same
// amount, and the bank of a cell is its index modulo 32. The markers are
// bucketed by the bank of their nearest cell; lane b of a warp takes the
// k-th marker of bucket b, so each of the warp's 81 integer atomic adds per
// marker touches 32 distinct banks (one shared-memory wavefront). The few
// markers beyond a full bucket are spread after the batches. Each contribution is rounded to fixed point by one
// fused multiply-add: F w 2^s + 1.5 2^23 is formed and rounded once, and for
// |F w 2^s| < 2^22 its bit pattern minus that of 1.5 2^23 is the rounded
// integer. Integer addition is associative, so the sums, and the fields
// written from them, are bit-identical whatever the order of the atomics.
constexpr int kSX = 2 * TX, kSY = 2 * TY, kSZ = TZ;  // super-tile extent in cells
constexpr int kSCells = kSX * kSY * kSZ;
constexpr int kSpreadThreads = 512;
constexpr int kSpreadWarps = kSpreadThreads / 32;
constexpr int kBankCap = 144;                        // markers per bank bucket
constexpr int kZCap = 48;                            // per bank bucket of plane markers
constexpr int kSpillCap = 512;                       // markers beyond a full bucket
constexpr int kRow = kSX + 2;                        // x in [-2, 32)
constexpr int kPlane = kRow * (kSY + 2);             // y in [-1, 17)
constexpr int kGuard = 64;                           // words before and after the planes
constexpr int kAccPlanes = kSZ + 2;                  // z in [-1, 9)
constexpr int kAccC = (kGuard * 2 + kPlane * kAccPlanes + 31) / 32 * 32;  // per component
// index of cell (x, y, z) of the super-tile in one component's array
__device__ __forceinline__ int acc_index(int x, int y, int z)
{
    return kGuard + (x + 2) + kRow * (y + 1) + kPlane * (z + 1);
}
// coarse bins (2 x 2 x 2 cells) of the nearest cells in [-1, ext]: their
// largest count bounds the markers of any single bin
constexpr int kCBX = (kSX + 3) / 2, kCBY = (kSY + 3) / 2, kCBZ = (kSZ + 3) / 2;
constexpr int kCBins = kCBX * kCBY * kCBZ;
constexpr int kNbTiles = 4 * 4 * 3;  // tiles of the super-tile and around it (x, y: 4; z: 3)
constexpr int kSlots = kNbTiles * 9;  // (tile, y class, z class): one run of keys each
constexpr int kChunkCap = 256;        // 32-marker chunks with a tabled run
static_assert(kAccC % 32 == 0, "the components share one bank layout");
static_assert(kGuard >= kRow + 2, "a row beyond the first or last plane stays in the guard");
static_assert(kSCells % kSpreadThreads == 0, "cells per thread");
constexpr unsigned kMagicBits = 0x4B400000u;  // bit pattern of 1.5 * 2^23
constexpr float kMagic = 12582912.0f;         // 1.5 * 2^23

struct SmemSpreadBank {
    int acc[3 * kAccC];
    int binc[kCBins];  // markers per coarse bin
    int sorted[32 * kBankCap];
    int zsorted[32 * kZCap];  // plane markers (nearest cell one plane above or below)
    int bcnt[32];
    int zcnt[32];
    int spill[kSpillCap];
    int nspill;
    int rbeg[kSlots];      // the non-empty runs of keys, in slot order: first binned
    int roff[kSlots + 1];  // position, and offset in their concatenation
    int crun[kChunkCap];   // run of the first marker of each 32-marker chunk
    int nrun;
    int red_tmp[kSpreadWarps];
    int sh[3];
    float cscale[3];
    int over;
    int nb, nzb;
    // the marker template follows: tR[3][n_l]
};

// compile-time loop: f(std::integral_constant<int, i>) for i = 0 .. N-1
template <int... I, class F>
__device__ __forceinline__ void static_for_impl(std::integer_sequence<int, I...>, F &&f)
{
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F &&f)
{
    static_for_impl(std::make_integer_sequence<int, N>{}, f);
}

// shared-memory integer add without a result, at a constant byte offset
// from a 32-bit shared address
template <int OFF>
__device__ __forceinline__ void red_shared_add(unsigned addr, int v)
{
    asm volatile("red.shared.add.s32 [%0+%2], %1;" ::"r"(addr), "r"(v), "n"(OFF));
}

// Local nearest cell of marker l of a sphere, relative to the super-tile
// origin: the actual cell on bounded axes, on periodic ones the image that
// lands in [-1, ext] (unique: the launcher requires n >= ext + 3 there).
__device__ __forceinline__ void bank_local_base(const TileArgs<float> &a, const PartFast<float> &rec,
                                                const float *tRs, int n_l, int l,
                                                const int (&org)[3], const int (&ext)[3],
                                                int (&lc)[3], int (&i0)[3], float (&q)[3])
{
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
        q[ax] = rec.fr[ax] + tRs[ax * n_l + l];
        i0[ax] = (int)floorf(q[ax] + 0.5f);
        int ub = rec.b[ax] + i0[ax];
        if (a.periodic[ax]) {
            const int n = a.n[ax];
            ub = ub < 0 ? ub + n : (ub >= n ? ub - n : ub);
            int r = ub - org[ax];
            r = r < -1 ? r + n : (r > ext[ax] ? r - n : r);
            lc[ax] = r;
        } else {
            lc[ax] = ub - org[ax];
        }
    }
}

// The same from the record's position part only (fractional offset, base).
__device__ __forceinline__ void bank_local_base(const TileArgs<float> &a, const float4 &fr,
                                                const int4 &b, const float *tRs, int n_l, int l,
                                                const int (&org)[3], const int (&ext)[3],
                                                int (&lc)[3], int (&i0)[3], float (&q)[3])
{
    PartFast<float> rec;
    rec.fr[0] = fr.x;
    rec.fr[1] = fr.y;
    rec.fr[2] = fr.z;
    rec.b[0] = b.x;
    rec.b[1] = b.y;
    rec.b[2] = b.z;
    bank_local_base(a, rec, tRs, n_l, l, org, ext, lc, i0, q);
}

// The plan of a super-tile's spread, made by a kernel of its own before
// the spread (small blocks, many per SM, so that the latency of the key
// lookups is hidden): the runs of (tile, y class, z class) keys whose
// markers can reach the super-tile, compacted in slot order with the offset
// of each in their concatenation, and the bound of their forces. Header
// per super-tile: {number of runs, markers, |F| bits x, y, z}; runs
// [kSlots + 1][2]: {first binned, offset}, entry nrun = {0, markers}.
constexpr int kPlanHdr = 8;
constexpr int kPlanThreads = 128;
constexpr int kPlanPer = (kSlots + kPlanThreads - 1) / kPlanThreads;

// The run of slot `slot` (tile * 9 + y class + 3 z class over the 4 x 4 x 3
// tiles around the super-tile): its first binned marker and count, and the
// tile whose force bound it adds (-1: none).
__device__ __forceinline__ void spread_slot(const TileArgs<float> &a, const int (&o0)[3],
                                            const int (&o1)[3], int slot, int &beg, int &cnt,
                                            int &ftile)
{
    const int t48 = slot / 9, j = slot - t48 * 9;
    const int ii[3] = {t48 & 3, (t48 >> 2) & 3, t48 >> 4};
    const int cj[2] = {j % 3, j / 3};  // y class, z class of this run
    int tix[3], clo[3], chi[3];
    bool ok = true;
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
        int qq = o0[ax] - 1 + ii[ax];
        if (ii[ax] == 0) {
            clo[ax] = chi[ax] = 2;             // the tile below: its high face
        } else if (qq < o1[ax]) {
            clo[ax] = 0;                       // an own tile: every class
            chi[ax] = 2;
        } else if (qq == o1[ax]) {
            clo[ax] = chi[ax] = 0;             // the tile above: its low face
        } else {
            ok = false;
        }
        if (qq < 0 || qq >= a.nt[ax]) {
            if (a.periodic[ax])
                qq = qq < 0 ? qq + a.nt[ax] : qq - a.nt[ax];
            else
                ok = false;
        }
        tix[ax] = qq;
    }
    const int tile = tix[0] + a.nt[0] * (tix[1] + a.nt[1] * tix[2]);
    ftile = ok && j == 0 ? tile : -1;
    ok = ok && cj[0] >= clo[1] && cj[0] <= chi[1] && cj[1] >= clo[2] && cj[1] <= chi[2];
    beg = 0;
    cnt = 0;
    if (ok) {
        const int k0 = tile * 27 + clo[0] + 3 * cj[0] + 9 * cj[1];
        const int k1 = tile * 27 + chi[0] + 3 * cj[0] + 9 * cj[1];
        beg = a.key_start[k0];
        cnt = a.key_start[k1 + 1] - beg;
    }
}

__global__ void __launch_bounds__(kPlanThreads) k_spread_plan(TileArgs<float> a, int sz0,
                                                              int *__restrict__ hdr,
                                                              int2 *__restrict__ runs)
{
    __shared__ int s_tot[kPlanThreads / 32], s_nr[kPlanThreads / 32];
    __shared__ unsigned s_fm[3];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nsx = (a.nt[0] + 1) / 2, nsy = (a.nt[1] + 1) / 2;
    const int sx = blockIdx.x % nsx, sy = (blockIdx.x / nsx) % nsy;
    const int tz = sz0 + blockIdx.x / (nsx * nsy);
    const long long st = (long long)blockIdx.x + (long long)sz0 * nsx * nsy;
    const int o0[3] = {2 * sx, 2 * sy, tz};
    const int o1[3] = {min(2 * sx + 2, a.nt[0]), min(2 * sy + 2, a.nt[1]), tz + 1};
    if (tid < 3)
        s_fm[tid] = 0u;
    int beg[kPlanPer], cnt[kPlanPer];
    unsigned fm[3] = {0u, 0u, 0u};
    int sum = 0, nr = 0;
#pragma unroll
    for (int i = 0; i < kPlanPer; i++) {
        const int slot = tid * kPlanPer + i;
        int ft = -1;
        beg[i] = cnt[i] = 0;
        if (slot < kSlots)
            spread_slot(a, o0, o1, slot, beg[i], cnt[i], ft);
        if (ft >= 0 && a.tile_fmax)
#pragma unroll
            for (int c = 0; c < 3; c++)
                fm[c] = max(fm[c], (unsigned)a.tile_fmax[(long long)ft * 3 + c]);
        sum += cnt[i];
        nr += cnt[i] > 0 ? 1 : 0;
    }
    // exclusive scans over the threads (slot order) of the counts and of
    // the non-empty runs; maxima of the force bounds
    int isum = sum, inr = nr;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t1 = __shfl_up_sync(0xffffffffu, isum, o);
        const int t2 = __shfl_up_sync(0xffffffffu, inr, o);
        if (lane >= o) {
            isum += t1;
            inr += t2;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; c++)
        fm[c] = __reduce_max_sync(0xffffffffu, fm[c]);
    if (lane == 31) {
        s_tot[warp] = isum;
        s_nr[warp] = inr;
    }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 3; c++)
            atomicMax(&s_fm[c], fm[c]);
    int wsum = 0, wnr = 0, tot = 0, ntr = 0;
#pragma unroll
    for (int w = 0; w < kPlanThreads / 32; w++) {
        if (w < warp) {
            wsum += s_tot[w];
            wnr += s_nr[w];
        }
        tot += s_tot[w];
        ntr += s_nr[w];
    }
    int off = wsum + isum - sum, pos = wnr + inr - nr;
    int2 *r = runs + st * (kSlots + 1);
#pragma unroll
    for (int i = 0; i < kPlanPer; i++)
        if (cnt[i] > 0) {
            r[pos] = make_int2(beg[i], off);
            off += cnt[i];
            pos++;
        }
    __syncthreads();
    if (tid == 0) {
        r[ntr] = make_int2(0, tot);
        int *h = hdr + st * kPlanHdr;
        h[0] = ntr;
        h[1] = tot;
        for (int c = 0; c < 3; c++)
            h[2 + c] = a.tile_fmax ? (int)s_fm[c] : (int)(unsigned)a.red[c];
    }
}

__global__ void __launch_bounds__(kSpreadThreads, 2) k_spread_bank(TileArgs<float> a, int sz0,
                                                                  const int *__restrict__ hdr,
                                                                  const int2 *__restrict__ runs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemSpreadBank &sm = *reinterpret_cast<SmemSpreadBank *>(smem_raw);
    float *tRs = reinterpret_cast<float *>(smem_raw + sizeof(SmemSpreadBank));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nsx = (a.nt[0] + 1) / 2, nsy = (a.nt[1] + 1) / 2;
    const int sx = blockIdx.x % nsx, sy = (blockIdx.x / nsx) % nsy;
    const int tz = sz0 + blockIdx.x / (nsx * nsy);
    const int org[3] = {sx * kSX, sy * kSY, tz * kSZ};
    const int ext[3] = {min(kSX, a.n[0] - org[0]), min(kSY, a.n[1] - org[1]),
                        min(kSZ, a.n[2] - org[2])};
    const int n_l = a.n_l;

    // the plan: the runs of binned markers that can reach the super-tile
    const long long st = (long long)blockIdx.x + (long long)sz0 * nsx * nsy;
    const int *h = hdr + st * kPlanHdr;
    const int nrun = h[0], total = h[1];
    float fm[3];
#pragma unroll
    for (int c = 0; c < 3; c++)
        fm[c] = __uint_as_float((unsigned)h[2 + c]);
    if (total == 0 || !(fmaxf(fm[0], fmaxf(fm[1], fm[2])) > 0.f))
        return;  // block-uniform
    for (int i = tid; i <= nrun; i += kSpreadThreads) {
        const int2 r = runs[st * (kSlots + 1) + i];
        if (i < nrun)
            sm.rbeg[i] = r.x;
        sm.roff[i] = r.y;
    }
    if (tid == 0)
        sm.nrun = nrun;
    const long long nx = a.n[0], nxy = (long long)a.n[0] * a.n[1];
    // the rows of f and u that the write-back reads, into L2 while the
    // markers are sorted and spread
    for (int r = tid; r < 6 * kSY * kSZ; r += kSpreadThreads) {
        const int f = r / (kSY * kSZ), yz = r - f * (kSY * kSZ), y = yz % kSY, z = yz / kSY;
        if (y < ext[1] && z < ext[2]) {
            const float *row = (f < 3 ? a.out_f[f] : a.out_u[f - 3]) +
                               ((org[2] + z) * nxy + (org[1] + y) * nx + org[0]);
            asm volatile("prefetch.global.L2 [%0];" ::"l"(row));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(row + ext[0] - 1));
        }
    }
    for (int i = tid; i < 3 * n_l; i += kSpreadThreads)
        tRs[i] = a.tR[i];
    for (int i = tid; i < 3 * kAccC / 4; i += kSpreadThreads)
        reinterpret_cast<int4 *>(sm.acc)[i] = make_int4(0, 0, 0, 0);
    for (int i = tid; i < kCBins; i += kSpreadThreads)
        sm.binc[i] = 0;
    if (tid < 32) {
        sm.bcnt[tid] = 0;
        sm.zcnt[tid] = 0;
    }
    if (tid == 0) {
        sm.over = 0;
        sm.nspill = 0;
    }
    __syncthreads();

    // the run of the first marker of every 32-marker chunk (one thread per
    // run writes the chunks that start in it)
    for (int r = tid; r < nrun; r += kSpreadThreads) {
        const int e = min(sm.roff[r + 1], 32 * kChunkCap);
        for (int g = (sm.roff[r] + 31) & ~31; g < e; g += 32)
            sm.crun[g >> 5] = r;
    }
    __syncthreads();

    const PartFast<float> *__restrict__ pf = a.pfast;
    // marker g0 + lane of the concatenated runs (g0 a multiple of 32, common
    // to the warp): the run of g0 from the chunk table (beyond it by a
    // binary search), then a few steps forward
    auto marker_of = [&](int g0, int g) -> int {
        int lo;
        if ((g0 >> 5) < kChunkCap) {
            lo = sm.crun[g0 >> 5];
        } else {
            lo = 0;
            int hi = sm.nrun;  // last run with roff <= g0
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (sm.roff[mid] <= g0)
                    lo = mid;
                else
                    hi = mid;
            }
        }
        while (sm.roff[lo + 1] <= g)
            lo++;
        return a.mlist[sm.rbeg[lo] + (g - sm.roff[lo])];
    };
    // pass A: bins and bank buckets, four candidates of a lane at a time
    // (their dependent loads, list entry then sphere record, in flight together)
    auto bucket = [&](int m, const float4 &fr, const int4 &b) {
        const int p = (int)__umul64hi((unsigned long long)m, a.l_magic);
        int lc[3], i0[3];
        float q[3];
        bank_local_base(a, fr, b, tRs, n_l, m - p * n_l, org, ext, lc, i0, q);
        const bool in = lc[0] >= -1 && lc[0] <= ext[0] && lc[1] >= -1 && lc[1] <= ext[1] &&
                        lc[2] >= -1 && lc[2] <= ext[2];
        if (!in)
            return;  // beyond a wall by more than a cell: reaches no cell here
        atomicAdd(&sm.binc[(((lc[2] + 1) >> 1) * kCBY + ((lc[1] + 1) >> 1)) * kCBX +
                           ((lc[0] + 1) >> 1)], 1);
        if (lc[2] < 0 || lc[2] >= ext[2]) {
            // nearest cell one plane below or above the super-tile: only one
            // plane of its stencil lies in it (bucketed by the bank of that
            // plane's first stencil cell)
            const int zb = acc_index(lc[0] - 1, lc[1] - 1, lc[2] < 0 ? 0 : ext[2] - 1) & 31;
            const int rz = atomicAdd(&sm.zcnt[zb], 1);
            if (rz < kZCap) {
                sm.zsorted[rz * 32 + zb] = m;
                return;
            }
        }
        const int bank = acc_index(lc[0], lc[1], lc[2]) & 31;
        const int r = atomicAdd(&sm.bcnt[bank], 1);
        if (r < kBankCap) {
            sm.sorted[r * 32 + bank] = m;  // [rank][bank]: a warp's reads hit 32 banks
        } else {
            const int s2 = atomicAdd(&sm.nspill, 1);
            if (s2 < kSpillCap)
                sm.spill[s2] = m;
            else
                sm.over = 1;
        }
    };
    constexpr int kCand = 4;
    for (int g0 = warp * 32; g0 < total; g0 += kCand * kSpreadThreads) {
        int mc[kCand];
        float4 frc[kCand];
        int4 bc[kCand];
#pragma unroll
        for (int j = 0; j < kCand; j++) {
            const int gj0 = g0 + j * kSpreadThreads, gj = gj0 + lane;
            mc[j] = (gj0 < total && gj < total) ? marker_of(gj0, gj) : -1;
        }
#pragma unroll
        for (int j = 0; j < kCand; j++) {
            frc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            bc[j] = make_int4(0, 0, 0, 0);
            if (mc[j] >= 0) {
                const float4 *rp = reinterpret_cast<const float4 *>(
                    pf + (int)__umul64hi((unsigned long long)mc[j], a.l_magic));
                frc[j] = __ldg(rp);
                bc[j] = __ldg(reinterpret_cast<const int4 *>(rp + 3));
            }
        }
#pragma unroll
        for (int j = 0; j < kCand; j++)
            if (mc[j] >= 0)
                bucket(mc[j], frc[j], bc[j]);
    }
    __syncthreads();
    // the fullest bin bounds every cell's sum
    int mb = 0;
    for (int i = tid; i < kCBins; i += kSpreadThreads)
        mb = max(mb, sm.binc[i]);
    mb = __reduce_max_sync(0xffffffffu, mb);
    if (lane == 0)
        sm.red_tmp[warp] = mb;
    if (warp == 0) {
        const int nb = __reduce_max_sync(0xffffffffu, min(sm.bcnt[lane], kBankCap));
        const int nzb = __reduce_max_sync(0xffffffffu, min(sm.zcnt[lane], kZCap));
        if (lane == 0) {
            sm.nb = nb;
            sm.nzb = nzb;
        }
    }
    __syncthreads();
    if (tid < 3) {
        int maxbin = 0;
        for (int k = 0; k < kSpreadWarps; k++)
            maxbin = max(maxbin, sm.red_tmp[k]);
        const int c = tid;
        // every contribution below 2^21 (margin for the rounding of the
        // magic-constant sum), every cell's sum below 2^30: a marker in bin b
        // reaches a cell j only if each |b - j| <= 1, with a weight per axis
        // of at most 1/2, 2/3, 1/2 over those offsets (5/3 in sum, at most
        // 2/3 for one)
        int ex1, ex2;
        frexp((8.0 / 27.0) * (double)fm[c] * a.dVh3, &ex1);
        frexp((125.0 / 27.0) * (double)max(maxbin, 1) * (double)fm[c] * a.dVh3, &ex2);
        const int s = min(21 - ex1, 30 - ex2);
        sm.sh[c] = s;
        sm.cscale[c] = fm[c] > 0.f ? (float)ldexp(a.dVh3, s) : 0.f;
    }
    __syncthreads();

    const float *__restrict__ Fsrc = a.pass == 0 ? a.Fl : a.dFl;
    // the loads of a marker: its sphere's position part and its force
    struct Loaded {
        float4 fr, F4;
        int4 b;
        int l;
    };
    auto load = [&](int m) {
        Loaded d;
        const int p = (int)__umul64hi((unsigned long long)m, a.l_magic);
        d.l = m - p * n_l;
        const float4 *rp = reinterpret_cast<const float4 *>(pf + p);
        d.fr = __ldg(rp);
        d.b = __ldg(reinterpret_cast<const int4 *>(rp + 3));
        d.F4 = __ldg(reinterpret_cast<const float4 *>(Fsrc) + m);
        return d;
    };
    auto accumulate_loaded = [&](const Loaded &d) {
        int lc[3], i0[3];
        float q[3];
        bank_local_base(a, d.fr, d.b, tRs, n_l, d.l, org, ext, lc, i0, q);
        const float4 F4 = d.F4;
        float w[3][3];
#pragma unroll
        for (int ax = 0; ax < 3; ax++) {
            const float r1 = (float)i0[ax] - q[ax];
            const float S = kernel_root(1.f - 3.f * r1 * r1);
            w[ax][1] = (1.f + S) * (1.f / 3.f);
            w[ax][0] = (2.f + 3.f * r1 - S) * (1.f / 6.f);
            w[ax][2] = (2.f - 3.f * r1 - S) * (1.f / 6.f);
        }
        const float Fc[3] = {F4.x * sm.cscale[0], F4.y * sm.cscale[1], F4.z * sm.cscale[2]};
        float Fw[3][3];
#pragma unroll
        for (int c = 0; c < 3; c++)
#pragma unroll
            for (int d = 0; d < 3; d++)
                Fw[c][d] = Fc[c] * w[0][d];
        // the stencil's first cell (lc - 1 per axis), one base per plane; a
        // plane below z = -1 or above z = 8 (nearest cell at z = -1 or 8) is
        // folded into the first 32 words of the padding plane next to it,
        // which keeps the bank of every cell
        int bz[3];
        bz[0] = acc_index(lc[0] - 1, lc[1] - 1, lc[2] - 1);
        bz[1] = bz[0] + kPlane;
        bz[2] = bz[0] + 2 * kPlane;
        if (lc[2] - 1 < -1) {
            const int p0 = acc_index(-2, -1, -1);
            bz[0] = p0 + ((bz[0] - p0) & 31);
        }
        if (lc[2] + 1 > kSZ) {
            const int p9 = acc_index(-2, -1, kSZ);
            bz[2] = p9 + ((bz[2] - p9) & 31);
        }
        const unsigned acc_s = (unsigned)__cvta_generic_to_shared(sm.acc);
        const unsigned rb[3] = {acc_s + 4u * (unsigned)bz[0], acc_s + 4u * (unsigned)bz[1],
                                acc_s + 4u * (unsigned)bz[2]};
        float wyz[9];
#pragma unroll
        for (int i = 0; i < 9; i++)
            wyz[i] = w[1][i % 3] * w[2][i / 3];
        // the 81 adds at constant offsets from one register per plane
        static_for<81>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int c = i % 3, dx = (i / 3) % 3, dy = (i / 9) % 3, dz = i / 27;
            const int v = (int)(__float_as_uint(fmaf(Fw[c][dx], wyz[dy + 3 * dz], kMagic)) -
                                kMagicBits);
            red_shared_add<4 * (dx + kRow * dy + c * kAccC)>(rb[dz], v);
        });
    };
    auto accumulate = [&](int m) { accumulate_loaded(load(m)); };
    // a plane marker: the 27 adds of its one stencil plane in the super-tile
    // (the same rounded contributions as the full stencil's for that plane)
    auto accumulate_plane = [&](const Loaded &d) {
        int lc[3], i0[3];
        float q[3];
        bank_local_base(a, d.fr, d.b, tRs, n_l, d.l, org, ext, lc, i0, q);
        const float4 F4 = d.F4;
        float w[3][3];
#pragma unroll
        for (int ax = 0; ax < 3; ax++) {
            const float r1 = (float)i0[ax] - q[ax];
            const float S = kernel_root(1.f - 3.f * r1 * r1);
            w[ax][1] = (1.f + S) * (1.f / 3.f);
            w[ax][0] = (2.f + 3.f * r1 - S) * (1.f / 6.f);
            w[ax][2] = (2.f - 3.f * r1 - S) * (1.f / 6.f);
        }
        const bool below = lc[2] < 0;
        const float wz = below ? w[2][2] : w[2][0];
        const float Fc[3] = {F4.x * sm.cscale[0], F4.y * sm.cscale[1], F4.z * sm.cscale[2]};
        float Fw[3][3];
#pragma unroll
        for (int c = 0; c < 3; c++)
#pragma unroll
            for (int dd = 0; dd < 3; dd++)
                Fw[c][dd] = Fc[c] * w[0][dd];
        float wyz[3];
#pragma unroll
        for (int dy = 0; dy < 3; dy++)
            wyz[dy] = w[1][dy] * wz;
        const unsigned rb = (unsigned)__cvta_generic_to_shared(sm.acc) +
                            4u * (unsigned)acc_index(lc[0] - 1, lc[1] - 1, below ? 0 : ext[2] - 1);
        static_for<27>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int c = i % 3, dx = (i / 3) % 3, dy = i / 9;
            const int v =
                (int)(__float_as_uint(fmaf(Fw[c][dx], wyz[dy], kMagic)) - kMagicBits);
            red_shared_add<4 * (dx + kRow * dy + c * kAccC)>(rb, v);
        });
    };
    if (sm.over) {
        // the spill list overflowed: every marker
        // in turn, with bank conflicts but the same sums
        for (int g0 = warp * 32; g0 < total; g0 += kSpreadThreads) {
            const int g = g0 + lane;
            if (g >= total)
                break;
            const int m = marker_of(g0, g);
            const int p = (int)__umul64hi((unsigned long long)m, a.l_magic);
            int lc[3], i0[3];
            float q[3];
            bank_local_base(a, pf[p], tRs, n_l, m - p * n_l, org, ext, lc, i0, q);
            if (lc[0] >= -1 && lc[0] <= ext[0] && lc[1] >= -1 && lc[1] <= ext[1] &&
                lc[2] >= -1 && lc[2] <= ext[2])
                accumulate(m);
        }
    } else {
        const int nb = sm.nb;
        const int mine = min(sm.bcnt[lane], kBankCap);
        for (int k = warp; k < nb; k += kSpreadWarps)
            if (k < mine) {
                // the force of this lane's next marker towards L2 (most
                // forces come from DRAM): no registers held across the adds
                if (k + kSpreadWarps < mine)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(
                        reinterpret_cast<const float4 *>(Fsrc) +
                        sm.sorted[(k + kSpreadWarps) * 32 + lane]));
                accumulate(sm.sorted[k * 32 + lane]);
            }
        const int nzb = sm.nzb, minez = min(sm.zcnt[lane], kZCap);
        for (int k = warp; k < nzb; k += kSpreadWarps)
            if (k < minez)
                accumulate_plane(load(sm.zsorted[k * 32 + lane]));
        for (int j = tid; j < min(sm.nspill, kSpillCap); j += kSpreadThreads)
            accumulate(sm.spill[j]);
    }
    __syncthreads();

    // read-modify-write of f and u on the cells with a nonzero sum, four
    // cells of a thread at a time (their loads in flight together)
    const float adt = (float)a.adt;
    float scl[3];
#pragma unroll
    for (int c = 0; c < 3; c++)
        scl[c] = ldexpf(1.f, -sm.sh[c]);
    constexpr int kPer = kSCells / kSpreadThreads;
#pragma unroll
    for (int h = 0; h < kPer; h += 4) {
        float vf[4][3], vu[4][3], dv[4][3];
        long long gi[4];
        bool on[4][3];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int cell = tid + (h + q) * kSpreadThreads;
            const int cx = cell & (kSX - 1), cy = (cell / kSX) % kSY, cz = cell / (kSX * kSY);
            const bool inside = cx < ext[0] && cy < ext[1] && cz < ext[2];
            gi[q] = (org[2] + cz) * nxy + (org[1] + cy) * nx + (org[0] + cx);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const int iv = sm.acc[c * kAccC + acc_index(cx, cy, cz)];
                on[q][c] = inside && iv != 0;
                dv[q][c] = (float)iv * scl[c];
                if (on[q][c]) {
                    vf[q][c] = a.out_f[c][gi[q]];
                    vu[q][c] = a.out_u[c][gi[q]];
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; q++)
#pragma unroll
            for (int c = 0; c < 3; c++)
                if (on[q][c]) {
                    a.out_f[c][gi[q]] = vf[q][c] + dv[q][c];
                    a.out_u[c][gi[q]] = vu[q][c] + adt * dv[q][c];
                }
    }
}

// ------------------------------------------------------------------ interpolation, bank-bucketed
// FP32 form with all components on the cell centres. A block takes the
// markers binned in one super-tile (2 x 2 x 1 tiles, 32 x 16 x 8 cells). One
// thread stages u, v, w on x in [-4, 36), y in [-1, 17), z in [-1, 9) around
// it with TMA tensor copies (zero fill beyond walls; cp.async with periodic
// wrap at a periodic end) while the block buckets the markers by the bank
// of their nearest cell in the staged layout. Lane b of a warp takes the
// k-th marker of bucket b, so each of the warp's 81 shared loads per marker
// reads 32 distinct banks. For each marker it interpolates the fluid
// velocity with the 3-point regularised delta and forms the direct-forcing
// force F_l = (U_d - U) / (alpha dt). Markers whose stencil leaves the
// staged block (beyond a wall) take a clipped path after the batches.
constexpr int kIX = kSX + 8, kIY = kSY + 2, kIZ = kSZ + 2;  // staged block
constexpr int kIN = kIX * kIY * kIZ;
constexpr int kIThreads = kSpreadThreads;
constexpr int kIWarps = kIThreads / 32;
constexpr int kIBankCap = 128;
constexpr int kISpill = 256;
static_assert(kIN % 32 == 0 && (kIN * 4) % 128 == 0, "component blocks share banks, TMA-aligned");

struct SmemInterpBank {
    float fld[3][kIN];
    int sorted[kIBankCap * 32];
    int spill[kISpill];  // markers beyond a full bucket
    int clip[kISpill];   // markers whose stencil leaves the staged block
    int bcnt[32];
    int nspill, nclip, over, nb;
    int rbeg[4], roff[5];
    uint64_t bar;
    float red[4][kIWarps];
    // the marker template follows: tR[3][n_l], rR[3][n_l]
};

// A sphere's 64-byte record as two 32-byte loads (read-only path): one load
// per sector, half the requests of four 16-byte loads when the lanes of a
// warp gather different spheres' records.
__device__ __forceinline__ PartFast<float> load_rec32(const PartFast<float> *rp)
{
    float v[16];
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
                   "=f"(v[6]), "=f"(v[7])
                 : "l"(rp));
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8+32];"
                 : "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]),
                   "=f"(v[14]), "=f"(v[15])
                 : "l"(rp));
    PartFast<float> r;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        r.fr[k] = v[k];
        r.up[k] = v[4 + k];
        r.om[k] = v[8 + k];
        r.b[k] = __float_as_int(v[12 + k]);
    }
    return r;
}
static_assert(sizeof(PartFast<float>) == 64 && alignof(PartFast<float>) == 16,
              "record layout: fr, up, om, b");

// staged index of the stencil's first cell (nearest cell - 1 per axis)
__device__ __forceinline__ int staged_first(int l0, int l1, int l2)
{
    return (l0 + 3) + kIX * l1 + kIX * kIY * l2;
}

__global__ void __launch_bounds__(kIThreads, 2)
k_interp_bank(TileArgs<float> a, const __grid_constant__ FieldMaps fm, int use_tma, int sz0)
{
    extern __shared__ __align__(128) unsigned char smem_ib[];
    SmemInterpBank &sm = *reinterpret_cast<SmemInterpBank *>(smem_ib);
    float *tRs = reinterpret_cast<float *>(smem_ib + sizeof(SmemInterpBank));
    const int n_l = a.n_l;
    float *rRs = tRs + 3 * n_l;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nsx = (a.nt[0] + 1) / 2, nsy = (a.nt[1] + 1) / 2;
    const int sx = blockIdx.x % nsx, sy = (blockIdx.x / nsx) % nsy;
    const int tz = sz0 + blockIdx.x / (nsx * nsy);
    const int org[3] = {sx * kSX, sy * kSY, tz * kSZ};
    const int ext[3] = {min(kSX, a.n[0] - org[0]), min(kSY, a.n[1] - org[1]),
                        min(kSZ, a.n[2] - org[2])};
    // the own tiles' markers: up to four contiguous runs of the binned list
    if (tid == 0) {
        int off = 0;
        for (int j = 0; j < 4; j++) {
            const int tx = 2 * sx + (j & 1), ty = 2 * sy + (j >> 1);
            int beg = 0, cnt = 0;
            if (tx < a.nt[0] && ty < a.nt[1]) {
                const int t = tx + a.nt[0] * (ty + a.nt[1] * tz);
                beg = a.key_start[t * 27];
                cnt = a.key_start[t * 27 + 27] - beg;
            }
            sm.rbeg[j] = beg;
            sm.roff[j] = off;
            off += cnt;
        }
        sm.roff[4] = off;
        sm.nspill = sm.nclip = sm.over = 0;
    }
    if (tid < 32)
        sm.bcnt[tid] = 0;
    __syncthreads();
    const int total = sm.roff[4];
    if (total == 0)
        return;  // block-uniform
    // staging: TMA unless a periodic axis wraps around the staged block
    const int lo_s[3] = {org[0] - 4, org[1] - 1, org[2] - 1};
    const int hi_s[3] = {org[0] + kIX - 4, org[1] + kIY - 1, org[2] + kIZ - 1};
    bool wrap = false;
#pragma unroll
    for (int k = 0; k < 3; k++)
        wrap = wrap || (a.periodic[k] && (lo_s[k] < 0 || hi_s[k] > a.n[k]));
    const bool tma = use_tma && !wrap;
    if (tma) {
        if (tid == 0) {
            mbar_init_count(&sm.bar, 1);
            const uint32_t b = smem_addr(&sm.bar);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
                         "r"((uint32_t)(3 * kIN * sizeof(float)))
                         : "memory");
#pragma unroll
            for (int c = 0; c < 3; c++)
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::"
                    "bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(&sm.fld[c][0])),
                    "l"(reinterpret_cast<uint64_t>(&fm.m[c])), "r"(lo_s[0]), "r"(lo_s[1]),
                    "r"(lo_s[2]), "r"(b)
                    : "memory");
        }
    } else {
        // 16-byte copies where rows allow them (x start and n_x multiples of
        // four values), single values otherwise; zero beyond a wall
        const long long nx = a.n[0], nxy = (long long)a.n[0] * a.n[1];
        const bool vec = (a.n[0] & 3) == 0 &&
                         ((reinterpret_cast<uintptr_t>(a.fld[0]) | reinterpret_cast<uintptr_t>(a.fld[1]) |
                           reinterpret_cast<uintptr_t>(a.fld[2])) & 15) == 0;
        const int per_row = vec ? kIX / 4 : kIX;
        for (int i = tid; i < 3 * kIY * kIZ * per_row; i += kIThreads) {
            const int row = i / per_row, ch = i - row * per_row;
            const int c = row / (kIY * kIZ), yz = row - c * (kIY * kIZ);
            const int sy2 = yz % kIY, sz2 = yz / kIY;
            int g[3] = {lo_s[0] + (vec ? 4 * ch : ch), lo_s[1] + sy2, lo_s[2] + sz2};
            bool ok = true;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (g[k] < 0 || g[k] >= a.n[k]) {
                    if (a.periodic[k])
                        g[k] = g[k] < 0 ? g[k] + a.n[k] : g[k] - a.n[k];
                    else
                        ok = false;
                }
            }
            float *dst = &sm.fld[c][(sz2 * kIY + sy2) * kIX + (vec ? 4 * ch : ch)];
            const float *src = a.fld[c] + (g[2] * nxy + g[1] * nx + g[0]);
            if (vec)
                cp_async16(dst, ok ? src : a.fld[c], ok);
            else
                *dst = ok ? __ldg(src) : 0.f;
        }
    }
    for (int i = tid; i < 3 * n_l; i += kIThreads) {
        tRs[i] = a.tR[i];
        rRs[i] = a.rR[i];
    }
    __syncthreads();  // template staged (and the barrier initialised)

    const PartFast<float> *__restrict__ pf = a.pfast;
    auto marker_of = [&](int g) -> int {
        int j = 0;
        while (sm.roff[j + 1] <= g)
            j++;
        return a.mlist[sm.rbeg[j] + (g - sm.roff[j])];
    };
    // nearest cell of marker m relative to the super-tile (its bin lies in
    // it: periodic axes need no image; on a bounded axis a marker beyond a
    // wall keeps its actual cell, outside the super-tile)
    auto local_cell = [&](const PartFast<float> &rec, int l, int (&lc)[3], int (&i0)[3],
                          float (&q)[3]) {
#pragma unroll
        for (int ax = 0; ax < 3; ax++) {
            q[ax] = rec.fr[ax] + tRs[ax * n_l + l];
            i0[ax] = (int)floorf(q[ax] + 0.5f);
            int ub = rec.b[ax] + i0[ax];
            if (a.periodic[ax])
                ub = ub < 0 ? ub + a.n[ax] : (ub >= a.n[ax] ? ub - a.n[ax] : ub);
            lc[ax] = ub - org[ax];
        }
    };
    // pass A: bank buckets, two candidates of a thread at a time (their
    // dependent loads, list entry then sphere record, in flight together)
    auto bucket = [&](int m, const float4 &fr, const int4 &b) {
        const int p = (int)__umul64hi((unsigned long long)m, a.l_magic);
        PartFast<float> rec;
        rec.fr[0] = fr.x, rec.fr[1] = fr.y, rec.fr[2] = fr.z;
        rec.b[0] = b.x, rec.b[1] = b.y, rec.b[2] = b.z;
        int lc[3], i0[3];
        float q[3];
        local_cell(rec, m - p * n_l, lc, i0, q);
        const bool inside = lc[0] >= 0 && lc[0] < ext[0] && lc[1] >= 0 && lc[1] < ext[1] &&
                            lc[2] >= 0 && lc[2] < ext[2];
        if (!inside) {
            const int s2 = atomicAdd(&sm.nclip, 1);
            if (s2 < kISpill)
                sm.clip[s2] = m;
            else
                sm.over = 1;
            return;
        }
        const int bank = staged_first(lc[0], lc[1], lc[2]) & 31;
        const int r = atomicAdd(&sm.bcnt[bank], 1);
        if (r < kIBankCap) {
            sm.sorted[r * 32 + bank] = m;
        } else {
            const int s2 = atomicAdd(&sm.nspill, 1);
            if (s2 < kISpill)
                sm.spill[s2] = m;
            else
                sm.over = 1;
        }
    };
    for (int g = tid; g < total; g += 2 * kIThreads) {
        const int gb = g + kIThreads;
        const int ma = marker_of(g);
        const int mb = gb < total ? marker_of(gb) : -1;
        const float4 *rpa = reinterpret_cast<const float4 *>(
            pf + (int)__umul64hi((unsigned long long)ma, a.l_magic));
        const float4 fra = __ldg(rpa);
        const int4 ba = __ldg(reinterpret_cast<const int4 *>(rpa + 3));
        float4 frb{};
        int4 bb{};
        if (mb >= 0) {
            const float4 *rp = reinterpret_cast<const float4 *>(
                pf + (int)__umul64hi((unsigned long long)mb, a.l_magic));
            frb = __ldg(rp);
            bb = __ldg(reinterpret_cast<const int4 *>(rp + 3));
        }
        bucket(ma, fra, ba);
        if (mb >= 0)
            bucket(mb, frb, bb);
    }
    // the staged fields
    bool staged = true;
    if (tma) {
        staged = mbar_wait_bounded(&sm.bar, 0);
        if (!staged && lane == 0)
            atomicOr(a.err, ERRB_TMA_TIMEOUT);
    } else {
        cp_async_wait_all();
    }
    __syncthreads();  // every marker bucketed
    if (warp == 0) {
        const int nb = __reduce_max_sync(0xffffffffu, min(sm.bcnt[lane], kIBankCap));
        if (lane == 0)
            sm.nb = nb;
    }
    __syncthreads();
    if (!__syncthreads_and(staged)) {
        // a timed-out copy: nothing is read (the flag is set); wait once more,
        // bounded, so that no copy into this block's memory outlives it
        if (tid == 0)
            mbar_wait_bounded(&sm.bar, 0);
        return;
    }

    const float inv_adt = a.inv_adt;
    float res = 0.f, fmx[3] = {0.f, 0.f, 0.f};
    // interpolation and forcing of marker m; CLIP: stencil cells outside the
    // staged block get weight zero (they lie beyond a wall)
    auto force_rec = [&](int m, const PartFast<float> &rec, bool clip) {
        const int p = (int)__umul64hi((unsigned long long)m, a.l_magic);
        const int l = m - p * n_l;
        int lc[3], i0[3];
        float q[3];
        local_cell(rec, l, lc, i0, q);
        float w[3][3];
#pragma unroll
        for (int ax = 0; ax < 3; ax++) {
            const float r1 = (float)i0[ax] - q[ax];
            const float S = kernel_root(1.f - 3.f * r1 * r1);
            w[ax][1] = (1.f + S) * (1.f / 3.f);
            w[ax][0] = (2.f + 3.f * r1 - S) * (1.f / 6.f);
            w[ax][2] = (2.f - 3.f * r1 - S) * (1.f / 6.f);
        }
        float U[3] = {0.f, 0.f, 0.f};
        if (!clip) {
            const float *f0 = &sm.fld[0][staged_first(lc[0], lc[1], lc[2])];
#pragma unroll
            for (int dz = 0; dz < 3; dz++)
#pragma unroll
                for (int dy = 0; dy < 3; dy++) {
                    const float wyz = w[1][dy] * w[2][dz];
                    const int o = kIX * dy + kIX * kIY * dz;
#pragma unroll
                    for (int c = 0; c < 3; c++)
                        U[c] += wyz * (w[0][0] * f0[c * kIN + o] + w[0][1] * f0[c * kIN + o + 1] +
                                       w[0][2] * f0[c * kIN + o + 2]);
                }
        } else {
            const int sdim[3] = {kIX, kIY, kIZ};
            const int soff[3] = {4, 1, 1};
            int ix[3][3];
#pragma unroll
            for (int ax = 0; ax < 3; ax++)
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    int s = lc[ax] - 1 + d + soff[ax];
                    if (s < 0 || s >= sdim[ax]) {
                        w[ax][d] = 0.f;
                        s = 0;
                    }
                    ix[ax][d] = s;
                }
#pragma unroll
            for (int dz = 0; dz < 3; dz++)
#pragma unroll
                for (int dy = 0; dy < 3; dy++) {
                    const float wyz = w[1][dy] * w[2][dz];
                    const int row = (ix[2][dz] * kIY + ix[1][dy]) * kIX;
#pragma unroll
                    for (int c = 0; c < 3; c++)
                        U[c] += wyz * (w[0][0] * sm.fld[c][row + ix[0][0]] +
                                       w[0][1] * sm.fld[c][row + ix[0][1]] +
                                       w[0][2] * sm.fld[c][row + ix[0][2]]);
                }
        }
        // rigid-body velocity of the surface point, U_d = u_p + omega_p x r
        const float rr[3] = {rRs[l], rRs[n_l + l], rRs[2 * n_l + l]};
        float Ud[3];
        Ud[0] = rec.up[0] + (rec.om[1] * rr[2] - rec.om[2] * rr[1]);
        Ud[1] = rec.up[1] + (rec.om[2] * rr[0] - rec.om[0] * rr[2]);
        Ud[2] = rec.up[2] + (rec.om[0] * rr[1] - rec.om[1] * rr[0]);
        float dF[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float slip = Ud[c] - U[c];
            res = fmaxf(res, fabsf(slip));
            dF[c] = slip * inv_adt;
            fmx[c] = fmaxf(fmx[c], fabsf(dF[c]));
        }
        if (a.probe)
            return;
        if (a.pass == 0) {
            store4(a.Fl, m, dF[0], dF[1], dF[2]);
        } else {
            float F[3];
            load4(a.Fl, m, F);
            store4(a.Fl, m, F[0] + dF[0], F[1] + dF[1], F[2] + dF[2]);
            store4(a.dFl, m, dF[0], dF[1], dF[2]);
        }
    };
    auto force = [&](int m, bool clip) {
        const int p = (int)__umul64hi((unsigned long long)m, a.l_magic);
        force_rec(m, pf[p], clip);
    };
    if (sm.over) {
        // a list overflowed: every marker in turn, clipped where needed
        for (int g = tid; g < total; g += kIThreads)
            force(marker_of(g), true);
    } else {
        // software-pipelined: the next batch's sphere record is in flight
        // while this batch interpolates
        const int nb = sm.nb, mine = min(sm.bcnt[lane], kIBankCap);
        int k = warp;
        int m = k < mine ? sm.sorted[k * 32 + lane] : -1;
        PartFast<float> rec{};
        if (m >= 0)
            rec = load_rec32(pf + (int)__umul64hi((unsigned long long)m, a.l_magic));
        for (; k < nb; k += kIWarps) {
            const int kn = k + kIWarps;
            const int mn = kn < mine ? sm.sorted[kn * 32 + lane] : -1;
            PartFast<float> recn{};
            if (mn >= 0)
                recn = load_rec32(pf + (int)__umul64hi((unsigned long long)mn, a.l_magic));
            if (m >= 0)
                force_rec(m, rec, false);
            m = mn;
            rec = recn;
        }
        for (int j = tid; j < sm.nspill; j += kIThreads)
            force(sm.spill[j], false);
        for (int j = tid; j < sm.nclip; j += kIThreads)
            force(sm.clip[j], true);
    }
    // block maxima: the residual and |dF| per component (device words), and
    // |dF| as the bound of the super-tile's four tiles for the spread
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        res = fmaxf(res, __shfl_xor_sync(0xffffffffu, res, o));
#pragma unroll
        for (int c = 0; c < 3; c++)
            fmx[c] = fmaxf(fmx[c], __shfl_xor_sync(0xffffffffu, fmx[c], o));
    }
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < 3; c++)
            sm.red[c][warp] = fmx[c];
        sm.red[3][warp] = res;
    }
    __syncthreads();
    if (tid < 4) {
        float r = 0.f;
        for (int k = 0; k < kIWarps; k++)
            r = fmaxf(r, sm.red[tid][k]);
        if (tid == kRedRes) {
            atomicMax(&a.red[kRedRes], max_bits(r));
        } else if (!a.probe) {
            atomicMax(&a.red[tid], max_bits(r));
            if (a.tile_fmax)
                for (int j = 0; j < 4; j++) {
                    const int tx = 2 * sx + (j & 1), ty = 2 * sy + (j >> 1);
                    if (tx < a.nt[0] && ty < a.nt[1])
                        a.tile_fmax[3LL * (tx + a.nt[0] * (ty + a.nt[1] * tz)) + tid] = max_bits(r);
                }
        }
    }
}

template <typename T>
__global__ void k_unpack(const T *__restrict__ Fl, long long n_m, T *__restrict__ out)
{
    long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_m)
        return;
    T v[3];
    load4(Fl, m, v);
    out[m] = v[0];
    out[n_m + m] = v[1];
    out[2 * n_m + m] = v[2];
}

template <typename T>
TileArgs<T> tile_args(const Ctx &c)
{
    TileArgs<T> a{};
    a.prep = (const PartPrep<T> *)c.prep;
    a.pfast = (const PartFast<T> *)c.pfast;
    a.l_magic = c.l_magic;
    a.pt_start = c.pt_count ? c.pt_start : nullptr;
    a.pt_list = c.pt_count ? c.pt_list : nullptr;
    a.tR = (const T *)c.tR;
    a.rR = (const T *)c.rR;
    a.Fl = (T *)c.Fl;
    a.dFl = (T *)c.dFl;
    a.red = c.d_red;
    a.tile_fmax = c.tile_fmax;
    a.err = c.d_err;
    a.key_start = c.key_start;
    a.mlist = c.mlist;
    for (int k = 0; k < 3; k++) {
        a.n[k] = c.g.n[k];
        a.periodic[k] = c.g.periodic[k];
        a.nt[k] = c.nt[k];
    }
    a.n_p = c.n_p;
    a.n_l = c.n_l;
    a.dVh3 = c.dV / (c.g.h * c.g.h * c.g.h);
    return a;
}

template <typename K>
void set_smem(K kernel, size_t bytes)
{
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

size_t ibm_smem_bytes(int precision, int same_off)
{
    if (precision == PRS_FP64)
        return same_off ? std::max(sizeof(SmemInterp<double, true>), sizeof(SmemSpread<double, true>))
                        : std::max(sizeof(SmemInterp<double, false>),
                                   sizeof(SmemSpread<double, false>));
    return same_off ? std::max(sizeof(SmemInterp<float, true>), sizeof(SmemSpread<float, true>))
                    : std::max(sizeof(SmemInterp<float, false>), sizeof(SmemSpread<float, false>));
}

void ibm_unpack_forces(const Ctx &c, void *dst, cudaStream_t s)
{
    const long long n_m = (long long)c.n_p * c.n_l;
    const int blocks = (int)((n_m + 255) / 256);
    if (c.precision == PRS_FP64)
        k_unpack<double><<<blocks, 256, 0, s>>>((const double *)c.Fl, n_m, (double *)dst);
    else
        k_unpack<float><<<blocks, 256, 0, s>>>((const float *)c.Fl, n_m, (float *)dst);
    c.n_launch += 1;
}

template <typename T>
void ibm_prep(Ctx &c, cudaStream_t s)
{
    k_prep<T><<<(c.n_p + 255) / 256, 256, 0, s>>>(c.x[c.cur], c.u[c.cur], c.om[c.cur], c.n_p,
                                                  c.g, (PartPrep<T> *)c.prep,
                                                  (PartFast<T> *)c.pfast);
    c.n_launch += 1;
}

template <typename T>
static void marker_bin_t(Ctx &c, cudaStream_t s)
{
    const long long n_m = (long long)c.n_p * c.n_l;
    const long long per_block = 256LL * kBinGroups;
    const int blocks = (int)((n_m + per_block - 1) / per_block);
    const int nkeys = c.ntile * 27;
    const int W = c.g.same_off ? 1 : 2;
    for (int pass = 0; pass < 2; pass++) {
        k_marker_bin<T><<<blocks, 256, 0, s>>>((const PartFast<T> *)c.pfast, (const T *)c.tR,
                                               c.n_p, c.n_l, c.l_magic, c.g.n[0], c.g.n[1],
                                               c.g.n[2],
                                               c.g.periodic[0], c.g.periodic[1],
                                               c.g.periodic[2], c.nt[0], c.nt[1], W, pass,
                                               c.key_count, c.key_start, c.mlist);
        if (pass == 0) {
            int k = exclusive_scan(c.key_count, c.key_start, nkeys, c.key_scan_tmp, s);
            k_set_int2<<<1, 1, 0, s>>>(c.key_start + nkeys, (int)n_m);
            c.n_launch += k + 1;
        }
    }
    c.n_launch += 2;
}

template <typename T>
static void particle_tiles_t(Ctx &c, cudaStream_t s)
{
    const int blocks = (c.n_p + 255) / 256;
    const int W = c.g.same_off ? 1 : 2;
    for (int pass = 0; pass < 2; pass++) {
        k_particle_tiles<T><<<blocks, 256, 0, s>>>(
            (const PartFast<T> *)c.pfast, c.n_p, c.R / c.g.h, c.g.n[0], c.g.n[1], c.g.n[2],
            c.g.periodic[0], c.g.periodic[1], c.g.periodic[2], c.nt[0], c.nt[1], c.nt[2], W,
            pass, c.pt_count, c.pt_start, c.pt_list);
        if (pass == 0)
            c.n_launch += exclusive_scan(c.pt_count, c.pt_start, c.ntile + 1, c.pt_scan_tmp, s);
    }
    c.n_launch += 2;
}

// ints of the spread plans of every super-tile
size_t spread_plan_ints(const Ctx &c)
{
    return (size_t)c.nsuper * (kPlanHdr + 2 * (kSlots + 1));
}

// The bank-bucketed spread serves the FP32 form with all components on
// the cell centres, when every periodic axis is long enough that a marker
// reaches a super-tile through one periodic image only.
bool spread_bank_ok(const Ctx &c)
{
    if (c.precision != PRS_FP32 || !c.g.same_off)
        return false;
    const int ext[3] = {kSX, kSY, kSZ};
    for (int k = 0; k < 3; k++)
        if (c.g.periodic[k] && c.g.n[k] < ext[k] + 3)
            return false;
    return true;
}

void ibm_marker_bin(Ctx &c, cudaStream_t s)
{
    if (c.pt_count && !spread_bank_ok(c)) {
        if (c.precision == PRS_FP64)
            particle_tiles_t<double>(c, s);
        else
            particle_tiles_t<float>(c, s);
    }
    if (c.precision == PRS_FP64)
        marker_bin_t<double>(c, s);
    else
        marker_bin_t<float>(c, s);
    // the interpolation's list of non-empty tiles at no periodic end, in order
    // (the bank-bucketed kernels take the super-tiles directly)
    if (spread_bank_ok(c))
        return;
    const int tb = (c.ntile + 1 + 255) / 256;
    for (int pass = 0; pass < 2; pass++) {
        k_tile_list<<<tb, 256, 0, s>>>(c.key_start, c.ntile, c.nt[0], c.nt[1], c.nt[2],
                                       c.g.periodic[0], c.g.periodic[1], c.g.periodic[2], pass,
                                       c.tile_flag, c.tile_pos, c.tma_list, c.tma_count);
        if (pass == 0)
            c.n_launch += exclusive_scan(c.tile_flag, c.tile_pos, c.ntile + 1, c.tile_scan_tmp, s);
    }
    c.n_launch += 2;
}

// TMA descriptors of u, v, w for the staged block of SmemInterp<T, SAME>;
// false when the fields or the marker list do not meet TMA's alignment rules
// (16-byte base and rows) or the driver lacks the encoder: the caller then
// stages with cp.async
template <typename T, bool SAME>
bool field_maps(const Ctx &c, const T *u, const T *v, const T *w, FieldMaps &fm)
{
    using Sm = SmemInterp<T, SAME>;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = []() {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        cudaGetLastError();
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    // the marker ids are bulk-copied in 16-byte units as well
    if (!encode || !c.tma_list || reinterpret_cast<uintptr_t>(c.mlist) % 16 != 0)
        return false;
    const T *f[3] = {u, v, w};
    const cuuint64_t dim[3] = {(cuuint64_t)c.g.n[0], (cuuint64_t)c.g.n[1], (cuuint64_t)c.g.n[2]};
    const cuuint64_t stride[2] = {dim[0] * sizeof(T), dim[0] * dim[1] * sizeof(T)};
    if (stride[0] % 16 != 0)
        return false;
    const cuuint32_t box[3] = {(cuuint32_t)Sm::RX, (cuuint32_t)Sm::RY, (cuuint32_t)Sm::RZ};
    const cuuint32_t estride[3] = {1, 1, 1};
    for (int k = 0; k < 3; k++) {
        if (reinterpret_cast<uintptr_t>(f[k]) % 16 != 0)
            return false;
        const CUresult r = encode(&fm.m[k],
                                  sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                                 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                  3, const_cast<T *>(f[k]), dim, stride, box, estride,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return false;
    }
    return true;
}

// TMA descriptors of u, v, w (FP32) with boxes of bx x by x bz values;
// false when the fields do not meet TMA's alignment rules (16-byte base and
// rows) or the driver lacks the encoder
bool field_maps_box(const float *u, const float *v, const float *w, const int n[3],
                    FieldMaps &fm, int bx, int by, int bz)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = []() {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        cudaGetLastError();
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    if (!encode)
        return false;
    const float *f[3] = {u, v, w};
    const cuuint64_t dim[3] = {(cuuint64_t)n[0], (cuuint64_t)n[1], (cuuint64_t)n[2]};
    const cuuint64_t stride[2] = {dim[0] * sizeof(float), dim[0] * dim[1] * sizeof(float)};
    if (stride[0] % 16 != 0)
        return false;
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t estride[3] = {1, 1, 1};
    for (int k = 0; k < 3; k++) {
        if (reinterpret_cast<uintptr_t>(f[k]) % 16 != 0)
            return false;
        const CUresult r = encode(&fm.m[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                                  const_cast<float *>(f[k]), dim, stride, box, estride,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return false;
    }
    return true;
}

template <typename T, bool SAME>
void interp_tiles_launch(Ctx &c, TileArgs<T> a, const int *tiles, int n, cudaStream_t s)
{
    if (n <= 0)
        return;
    a.tiles = tiles;
    const size_t sm = sizeof(SmemInterp<T, SAME>) + 6 * sizeof(T) * (size_t)c.n_l;
    set_smem(k_interp_tiles<T, SAME>, sm);
    k_interp_tiles<T, SAME><<<n, kThreads, sm, s>>>(a);
    c.n_launch += 1;
}

// tiles at a periodic end with cp.async staging, the others with the
// persistent TMA kernel (one block per resident slot); tiles [t_lo, t_hi)
template <typename T, bool SAME>
void interp_tma_launch(Ctx &c, const TileArgs<T> &a, const FieldMaps &fm, cudaStream_t s,
                       int t_lo, int t_hi)
{
    {
        const auto &e = c.edge_host;
        const int i0 = (int)(std::lower_bound(e.begin(), e.end(), t_lo) - e.begin());
        const int i1 = (int)(std::lower_bound(e.begin(), e.end(), t_hi) - e.begin());
        if (c.edge_tiles)
            interp_tiles_launch<T, SAME>(c, a, c.edge_tiles + i0, i1 - i0, s);
    }
    const size_t sm = sizeof(SmemInterpTma<T, SAME>) + 6 * sizeof(T) * (size_t)c.n_l;
    set_smem(k_interp_tma<T, SAME>, sm);
    static int grid = 0;  // per instantiation: resident blocks on all SMs
    if (!grid) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_interp_tma<T, SAME>, kTmaThreads,
                                                      sm);
        grid = std::max(1, per) * std::max(1, sms);
    }
    k_interp_tma<T, SAME><<<grid, kTmaThreads, sm, s>>>(a, fm, c.tma_list, c.tma_count, t_lo,
                                                         t_hi);
    c.n_launch += 1;
}

template <typename T>
void ibm_interp_force(Ctx &c, const T *u, const T *v, const T *w, int pass, double inv_adt,
                      int probe, cudaStream_t s, int tz_lo, int tz_hi, bool sums)
{
    TileArgs<T> a = tile_args<T>(c);
    const int per_layer = c.nt[0] * c.nt[1];
    int t_lo = 0, t_hi = c.ntile;
    if (tz_hi >= tz_lo) {
        t_lo = tz_lo * per_layer;
        t_hi = (tz_hi + 1) * per_layer;
    }
    a.tile0 = t_lo;
    a.fld[0] = u;
    a.fld[1] = v;
    a.fld[2] = w;
    a.pass = pass;
    a.probe = probe;
    a.inv_adt = (T)inv_adt;
    phase_begin(c, PRS_PHASE_INTERP);
    if (c.delta_kernel == 4) {
        ibm4_interp_force<T>(c, u, v, w, pass, inv_adt, probe, s);
        if (!probe && sums)
            particle_sums_launch<T>(c, s);
        phase_end(c);
        return;
    }
    FieldMaps fm;
    if constexpr (sizeof(T) == 4) {
        if (spread_bank_ok(c)) {
            const bool tma = field_maps_box(u, v, w, c.g.n, fm, kIX, kIY, kIZ);
            const int layers = tz_hi >= tz_lo ? tz_hi - tz_lo + 1 : c.nt[2];
            const int sz0 = tz_hi >= tz_lo ? tz_lo : 0;
            const int blocks = ((c.nt[0] + 1) / 2) * ((c.nt[1] + 1) / 2) * layers;
            const size_t sm = sizeof(SmemInterpBank) + 6 * sizeof(float) * (size_t)c.n_l;
            set_smem(k_interp_bank, sm);
            cudaFuncSetAttribute(k_interp_bank, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 100);
            k_interp_bank<<<blocks, kIThreads, sm, s>>>(a, fm, tma ? 1 : 0, sz0);
            c.n_launch += 1;
            if (!probe && sums)
                particle_sums_launch<T>(c, s);
            phase_end(c);
            return;
        }
    }
    if (c.g.same_off) {
        if (field_maps<T, true>(c, u, v, w, fm))
            interp_tma_launch<T, true>(c, a, fm, s, t_lo, t_hi);
        else
            interp_tiles_launch<T, true>(c, a, nullptr, t_hi - t_lo, s);
    } else {
        if (field_maps<T, false>(c, u, v, w, fm))
            interp_tma_launch<T, false>(c, a, fm, s, t_lo, t_hi);
        else
            interp_tiles_launch<T, false>(c, a, nullptr, t_hi - t_lo, s);
    }
    if (!probe && sums) {
        particle_sums_launch<T>(c, s);
    }
    phase_end(c);
}

template <typename T>
void ibm_spread(Ctx &c, T *u, T *v, T *w, T *fx, T *fy, T *fz, int pass, double adt,
                cudaStream_t s, int tz_lo, int tz_hi)
{
    TileArgs<T> a = tile_args<T>(c);
    // tiles of z-layers [tz_lo, tz_hi] only (all tiles when tz_hi < tz_lo)
    int ntiles = c.ntile;
    if (tz_hi >= tz_lo) {
        a.tile0 = tz_lo * c.nt[0] * c.nt[1];
        ntiles = (tz_hi - tz_lo + 1) * c.nt[0] * c.nt[1];
    }
    if (c.spread_global)
        a.tile_fmax = nullptr;
    a.out_f[0] = fx;
    a.out_f[1] = fy;
    a.out_f[2] = fz;
    a.out_u[0] = u;
    a.out_u[1] = v;
    a.out_u[2] = w;
    a.pass = pass;
    a.adt = adt;
    phase_begin(c, PRS_PHASE_SPREAD);
    if (c.delta_kernel == 4) {
        ibm4_spread<T>(c, u, v, w, fx, fy, fz, pass, adt, s);
        phase_end(c);
        return;
    }
    const size_t tmpl = 3 * sizeof(T) * (size_t)c.n_l;
    if constexpr (sizeof(T) == 4) {
        if (spread_bank_ok(c)) {
            const int layers = tz_hi >= tz_lo ? tz_hi - tz_lo + 1 : c.nt[2];
            const int sz0 = tz_hi >= tz_lo ? tz_lo : 0;
            const int blocks = ((c.nt[0] + 1) / 2) * ((c.nt[1] + 1) / 2) * layers;
            const size_t sm = sizeof(SmemSpreadBank) + tmpl;
            set_smem(k_spread_bank, sm);
            cudaFuncSetAttribute(k_spread_bank, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 100);
            int2 *runs = reinterpret_cast<int2 *>(c.sp_plan + (size_t)kPlanHdr * c.nsuper);
            k_spread_plan<<<blocks, kPlanThreads, 0, s>>>(a, sz0, c.sp_plan, runs);
            k_spread_bank<<<blocks, kSpreadThreads, sm, s>>>(a, sz0, c.sp_plan, runs);
            phase_end(c);
            c.n_launch += 2;
            return;
        }
    }
    if (c.g.same_off) {
        const size_t sm = sizeof(SmemSpread<T, true>) + tmpl;
        set_smem(k_spread_tiles<T, true>, sm);
        cudaFuncSetAttribute(k_spread_tiles<T, true>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        k_spread_tiles<T, true><<<ntiles, kThreads, sm, s>>>(a);
    } else {
        const size_t sm = sizeof(SmemSpread<T, false>) + tmpl;
        set_smem(k_spread_tiles<T, false>, sm);
        cudaFuncSetAttribute(k_spread_tiles<T, false>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        k_spread_tiles<T, false><<<ntiles, kThreads, sm, s>>>(a);
    }
    phase_end(c);
    c.n_launch += 1;
}

template void ibm_prep<float>(Ctx &, cudaStream_t);
template void ibm_prep<double>(Ctx &, cudaStream_t);
// z cells that the markers' stencils of any sphere can reach: [floor((z -
// R)/h) - 3, floor((z + R)/h) + 3] over all spheres (3 cells cover the
// stencil and a staggered component offset)
__global__ void k_zrange(const double *__restrict__ x, int n_p, double h, double R,
                         int *__restrict__ zr)
{
    int lo = INT_MAX, hi = INT_MIN;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_p; p += gridDim.x * blockDim.x) {
        const double z = x[2 * n_p + p];
        lo = min(lo, (int)floor((z - R) / h) - 3);
        hi = max(hi, (int)floor((z + R) / h) + 3);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&zr[0], lo);
        atomicMax(&zr[1], hi);
    }
}

// A bounded wait on a shared-memory barrier that nothing completes: the
// wait runs out after `polls` polls and latches the timeout bit, as every
// bounded wait of the library does when its copies never arrive.
__global__ void k_wait_probe(int *err, long long polls)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0)
        mbar_init_count(&bar, 1);
    __syncthreads();
    const uint32_t a = smem_addr(&bar);
    uint32_t ok = 0;
    for (long long it = 0; it < polls && !ok; it++)
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(a), "r"(0u)
            : "memory");
    if (!ok && threadIdx.x == 0)
        atomicOr(err, ERRB_TMA_TIMEOUT);
}

void wait_probe(Ctx &c, long long polls)
{
    k_wait_probe<<<1, 32, 0, c.stream>>>(c.d_err, polls);
    c.n_launch += 1;
}

void particle_zrange(Ctx &c, int zr[2], cudaStream_t s)
{
    const int init[2] = {INT_MAX, INT_MIN};
    cudaMemcpyAsync(c.d_zr, init, sizeof(init), cudaMemcpyHostToDevice, s);
    k_zrange<<<std::min((c.n_p + 255) / 256, 1024), 256, 0, s>>>(c.x[c.cur], c.n_p, c.g.h, c.R,
                                                                c.d_zr);
    c.n_launch += 1;
    cudaMemcpyAsync(zr, c.d_zr, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
}

template <typename T>
void ibm_particle_sums(Ctx &c, cudaStream_t s)
{
    particle_sums_launch<T>(c, s);
}

template void ibm_particle_sums<float>(Ctx &, cudaStream_t);
template void ibm_particle_sums<double>(Ctx &, cudaStream_t);
template void ibm_interp_force<float>(Ctx &, const float *, const float *, const float *, int,
                                      double, int, cudaStream_t, int, int, bool);
template void ibm_interp_force<double>(Ctx &, const double *, const double *, const double *,
                                       int, double, int, cudaStream_t, int, int, bool);
template void ibm_spread<float>(Ctx &, float *, float *, float *, float *, float *, float *,
                                int, double, cudaStream_t, int, int);
template void ibm_spread<double>(Ctx &, double *, double *, double *, double *, double *,
                                 double *, int, double, cudaStream_t, int, int);

}  // namespace prs
