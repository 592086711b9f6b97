// Direct forcing with Peskin's 4-point kernel (Peskin 2002), the wider
// variant of the regularised delta of Sec. 3.3: per axis the four grid
// points within 2h of a marker, phi(r) = (3 - 2|r| + sqrt(1 + 4|r| - 4r^2))/8
// for |r| <= 1 and (5 - 2|r| - sqrt(-7 + 12|r| - 4r^2))/8 for 1 <= |r| <= 2.
//
//   k_interp4   one thread per marker: U(X_l) from the 64 grid points of each
//               component (read from the field in global memory), the
//               direct-forcing force F_l = (U_d - U)/(alpha dt), the largest
//               slip and |F_l| per component.
//   k_spread4   one thread per marker: F_l phi phi phi dV/h^3 scaled by a
//               power of two and rounded to a 64-bit integer, added to the
//               cell's integer in a scratch grid. Integer addition is
//               associative: the sums do not depend on the order.
//   k_spread4_box  the same sums, one block per sphere and component: the
//               contributions meet first in a box of cells in shared memory
//               (used when the box fits in 48 KB)
//   k_apply4    one thread per cell: f += sum, u += alpha dt sum, and the
//               scratch back to zero.
//
// The scale 2^s of a component is chosen on the device from the pass's
// largest |F_l|: every contribution stays below 2^50 (FP64) or 2^40 (FP32),
// so a cell can take 2^13 contributions without overflow.

#include <cmath>
#include <cstdint>

#include "prs_internal.cuh"

namespace prs {
namespace {

template <typename T>
__device__ __forceinline__ T phi4(T r)
{
    const T a = fabs(r);
    if (a <= T(1))
        return (T(3) - T(2) * a + sqrt(T(1) + T(4) * a - T(4) * a * a)) * T(0.125);
    if (a <= T(2))
        return (T(5) - T(2) * a - sqrt(T(-7) + T(12) * a - T(4) * a * a)) * T(0.125);
    return T(0);
}

__device__ __forceinline__ unsigned long long bits_of(float v)
{
    return (unsigned long long)__float_as_uint(v);
}
__device__ __forceinline__ unsigned long long bits_of(double v)
{
    return (unsigned long long)__double_as_longlong(v);
}
template <typename T>
__device__ __forceinline__ T from_bits(unsigned long long b);
template <>
__device__ __forceinline__ float from_bits<float>(unsigned long long b)
{
    return __uint_as_float((unsigned)b);
}
template <>
__device__ __forceinline__ double from_bits<double>(unsigned long long b)
{
    return __longlong_as_double((long long)b);
}

template <typename T>
struct Args4 {
    const PartPrep<T> *prep;
    const T *tR, *rR;  // [3][n_l]: R/h t_l and R t_l
    const T *fld[3];
    T *Fl, *dFl;       // [n_m][4]
    unsigned long long *red;   // max |dF| per component, max slip (bits)
    unsigned long long *acc;   // [3][cells]
    T *out_f[3], *out_u[3];
    int n[3], periodic[3];
    int n_l;
    long long n_m;
    unsigned long long l_magic;
    int pass, probe;
    T inv_adt;
    double adt, dVh3;
    int *err;  // latched error bits
    int same_off;  // all components at the same offsets: one stencil serves all
};

// the four grid indices (or -1 beyond a wall) and weights along one axis for
// a point at index coordinate b + q
template <typename T>
__device__ __forceinline__ void stencil4(int b, T q, int n, int periodic, int (&i)[4], T (&w)[4])
{
    const T f = floor(q);
#pragma unroll
    for (int d = 0; d < 4; d++) {
        const T r = f - T(1) + T(d) - q;
        w[d] = phi4(r);
        int k = b + (int)f - 1 + d;
        if (periodic) {
            // a few cells out at most: wrapped by additions, not a division
            while (k < 0)
                k += n;
            while (k >= n)
                k -= n;
        } else if (k < 0 || k >= n) {
            k = -1;
        }
        i[d] = k;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_interp4(Args4<T> a)
{
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    T res = T(0), fm[3] = {T(0), T(0), T(0)};
    if (m < a.n_m) {
        const int p = (int)__umul64hi((unsigned long long)m, a.l_magic);
        const int l = (int)(m - (long long)p * a.n_l);
        const PartPrep<T> &pp = a.prep[p];
        const long long nx = a.n[0], nxy = (long long)a.n[0] * a.n[1];
        T U[3];
        int ix[3][4];
        T w[3][4];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            if (c == 0 || !a.same_off)
#pragma unroll
                for (int ax = 0; ax < 3; ax++)
                    stencil4<T>(pp.base[c * 3 + ax], pp.frac[c * 3 + ax] + a.tR[ax * a.n_l + l],
                                a.n[ax], a.periodic[ax], ix[ax], w[ax]);
            T acc = T(0);
            for (int dz = 0; dz < 4; dz++) {
                if (ix[2][dz] < 0)
                    continue;
                for (int dy = 0; dy < 4; dy++) {
                    if (ix[1][dy] < 0)
                        continue;
                    const long long row = ix[2][dz] * nxy + ix[1][dy] * nx;
                    T s = T(0);
#pragma unroll
                    for (int dx = 0; dx < 4; dx++)
                        if (ix[0][dx] >= 0)
                            s += w[0][dx] * a.fld[c][row + ix[0][dx]];
                    acc += w[1][dy] * w[2][dz] * s;
                }
            }
            U[c] = acc;
        }
        // rigid-body velocity of the surface point, U_d = u_p + omega_p x r
        const T rr[3] = {a.rR[l], a.rR[a.n_l + l], a.rR[2 * a.n_l + l]};
        T Ud[3];
        Ud[0] = pp.up[0] + (pp.om[1] * rr[2] - pp.om[2] * rr[1]);
        Ud[1] = pp.up[1] + (pp.om[2] * rr[0] - pp.om[0] * rr[2]);
        Ud[2] = pp.up[2] + (pp.om[0] * rr[1] - pp.om[1] * rr[0]);
        T dF[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const T slip = Ud[c] - U[c];
            res = max(res, fabs(slip));
            dF[c] = slip * a.inv_adt;
            fm[c] = max(fm[c], fabs(dF[c]));
        }
        if (!a.probe) {
            T *F = a.Fl + 4 * m;
            if (a.pass == 0) {
#pragma unroll
                for (int c = 0; c < 3; c++)
                    F[c] = dF[c];
            } else {
                T *D = a.dFl + 4 * m;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    F[c] = F[c] + dF[c];
                    D[c] = dF[c];
                }
            }
        }
    }
    // block maxima (non-negative values: their bit patterns order alike)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        res = max(res, __shfl_xor_sync(0xffffffffu, res, o));
#pragma unroll
        for (int c = 0; c < 3; c++)
            fm[c] = max(fm[c], __shfl_xor_sync(0xffffffffu, fm[c], o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&a.red[kRedRes], bits_of(res));
        if (!a.probe)
#pragma unroll
            for (int c = 0; c < 3; c++)
                atomicMax(&a.red[c], bits_of(fm[c]));
    }
}

// the power of two of component c: largest contribution below 2^B
template <typename T>
__device__ __forceinline__ int scale_exp(const Args4<T> &a, int c)
{
    const double fm = (double)from_bits<T>(a.red[c]) * a.dVh3;
    if (!(fm > 0.0))
        return 0;
    int e;
    frexp(fm, &e);  // fm < 2^e
    return (sizeof(T) == 8 ? 50 : 40) - e;
}

// x rounded to the nearest 64-bit integer (ties to even), by integer
// operations on its bits: the conversion instructions run on the FP64 pipe,
// which is slow on this GPU. |x| < 2^62 (the spread keeps it below 2^40).
__device__ __forceinline__ long long f32_round_ll(float x)
{
    const unsigned b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xFFu);
    if (e < 126 || e > 188)
        return 0;  // |x| < 1/2 (or out of the stated range)
    const unsigned long long m = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u);
    const int sh = e - 150;  // x = m 2^sh
    unsigned long long r;
    if (sh >= 0) {
        r = m << sh;
    } else {
        const int k = -sh;  // 1 .. 24
        const unsigned long long q = m >> k, rem = m & ((1ULL << k) - 1ULL),
                                 half = 1ULL << (k - 1);
        r = q + ((rem > half || (rem == half && (q & 1ULL))) ? 1ULL : 0ULL);
    }
    return (b >> 31) ? -(long long)r : (long long)r;
}

// The rounded contribution of one stencil point at the scratch grid's scale
template <typename T>
__device__ __forceinline__ long long contribution4(double Fc, T wyz, T wx)
{
    if (sizeof(T) == 4)
        return f32_round_ll((float)Fc * ((float)wyz * (float)wx));
    return __double2ll_rn(Fc * ((double)wyz * (double)wx));
}

template <typename T>
__global__ void __launch_bounds__(256) k_spread4(Args4<T> a)
{
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= a.n_m)
        return;
    const int p = (int)__umul64hi((unsigned long long)m, a.l_magic);
    const int l = (int)(m - (long long)p * a.n_l);
    const PartPrep<T> &pp = a.prep[p];
    const T *Fsrc = (a.pass == 0 ? a.Fl : a.dFl) + 4 * m;
    const long long nx = a.n[0], nxy = (long long)a.n[0] * a.n[1];
    const long long cells = nxy * a.n[2];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const double scale = ldexp(a.dVh3, scale_exp(a, c));
        const double Fc = (double)Fsrc[c] * scale;
        if (Fc == 0.0)
            continue;
        int ix[3][4];
        T w[3][4];
#pragma unroll
        for (int ax = 0; ax < 3; ax++)
            stencil4<T>(pp.base[c * 3 + ax], pp.frac[c * 3 + ax] + a.tR[ax * a.n_l + l], a.n[ax],
                        a.periodic[ax], ix[ax], w[ax]);
        unsigned long long *acc = a.acc + c * cells;
        for (int dz = 0; dz < 4; dz++) {
            if (ix[2][dz] < 0)
                continue;
            for (int dy = 0; dy < 4; dy++) {
                if (ix[1][dy] < 0)
                    continue;
                const long long row = ix[2][dz] * nxy + ix[1][dy] * nx;
                const T wyz = w[1][dy] * w[2][dz];
                for (int dx = 0; dx < 4; dx++) {
                    if (ix[0][dx] < 0)
                        continue;
                    atomicAdd(acc + row + ix[0][dx],
                              (unsigned long long)contribution4<T>(Fc, wyz, w[0][dx]));
                }
            }
        }
    }
}

// The box's integers: in the FP32 form 32-bit (native shared atomics), the
// contributions rounded 2^16 coarser than the scratch grid's and shifted
// into the grid's scale on the way out; in the FP64 form 64-bit, at the
// grid's scale. Bound: at the grid's scale every |F| dV/h^3 is below 2^40
// and a stencil weight per axis is at most phi(0) = 1/2, so one
// contribution is below 2^37 (2^21 in the box: in range of the rounding by
// a magic-constant FFMA) and the sum of up to 512 markers' contributions
// below 2^30.
template <typename T>
struct Box4Acc {
    using type = unsigned long long;
    static constexpr int shift = 0;
};
template <>
struct Box4Acc<float> {
    using type = int;
    static constexpr int shift = 16;
};
constexpr int kBox4MaxMarkers32 = 512;

// One block per sphere and component: the sphere's markers add their
// rounded contributions into a box of (2 rh + 6)^3 cells around it in shared
// memory (integers), and the box's non-zero sums then go to the
// scratch grid with one global atomic each. A sphere's 4 x 4 x 4 stencils
// overlap heavily, so this takes several times fewer global atomics than
// one per stencil point. Integer sums: deterministic (in the FP32 form the
// box rounds 2^16 coarser than k_spread4, within the form's tolerance).
constexpr int kBox4Threads = 128;
template <typename T>
__global__ void __launch_bounds__(kBox4Threads) k_spread4_box(Args4<T> a, int rh)
{
    using Acc = typename Box4Acc<T>::type;
    constexpr int kShift = Box4Acc<T>::shift;
    extern __shared__ __align__(16) unsigned char box_raw[];
    Acc *box = reinterpret_cast<Acc *>(box_raw);
    const int p = blockIdx.x, c = blockIdx.y;
    // the box starts rh + 2 cells below the sphere's base index: a marker's
    // first stencil point lies at most rh + 1 below it (one more for the
    // rounding of R t_l), its last at most rh + 3 above
    const int B = 2 * rh + 6, B3 = B * B * B;
    const PartPrep<T> &pp = a.prep[p];
    for (int i = threadIdx.x; i < B3; i += kBox4Threads)
        box[i] = Acc(0);
    __syncthreads();
    const double scale = ldexp(a.dVh3, scale_exp(a, c) - kShift);
    const T *F0 = a.pass == 0 ? a.Fl : a.dFl;
    // a warp takes every fourth marker: its lanes' stencils spread over the
    // whole sphere instead of one cap of it, and collide less in the box
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarps = kBox4Threads / 32;
    for (int j = lane; j * kWarps + warp < a.n_l; j += 32) {
        const int l = j * kWarps + warp;
        const long long m = (long long)p * a.n_l + l;
        const double Fc = (double)F0[4 * m + c] * scale;
        if (Fc == 0.0)
            continue;
        int lo[3];
        T w[3][4];
        bool ok[3][4];
#pragma unroll
        for (int ax = 0; ax < 3; ax++) {
            const T q = pp.frac[c * 3 + ax] + a.tR[ax * a.n_l + l];
            const T f = floor(q);
            lo[ax] = (int)f + rh + 1;  // local index of the first stencil point
#pragma unroll
            for (int d = 0; d < 4; d++) {
                w[ax][d] = phi4(f - T(1) + T(d) - q);
                const int k = pp.base[c * 3 + ax] + (int)f - 1 + d;
                ok[ax][d] = a.periodic[ax] || (k >= 0 && k < a.n[ax]);
            }
        }
        if (lo[0] < 0 || lo[1] < 0 || lo[2] < 0 || lo[0] + 4 > B || lo[1] + 4 > B ||
            lo[2] + 4 > B) {
            // outside the box (not possible for markers on the sphere): the
            // contribution is not lost silently, the call reports it
            atomicOr(a.err, ERRB_CAPACITY);
            continue;
        }
        for (int dz = 0; dz < 4; dz++) {
            if (!ok[2][dz])
                continue;
            for (int dy = 0; dy < 4; dy++) {
                if (!ok[1][dy])
                    continue;
                const T wyz = w[1][dy] * w[2][dz];
                const int row = ((lo[2] + dz) * B + lo[1] + dy) * B + lo[0];
#pragma unroll
                for (int dx = 0; dx < 4; dx++) {
                    if (!ok[0][dx])
                        continue;
                    if (sizeof(T) == 4) {
                        // |F w 2^s| < 2^21: rounded by one fused add of 1.5 2^23
                        const float x = fmaf((float)Fc, (float)wyz * (float)w[0][dx],
                                             12582912.0f);
                        atomicAdd(&box[row + dx], (Acc)(int)(__float_as_uint(x) - 0x4B400000u));
                    } else {
                        atomicAdd(&box[row + dx],
                                  (Acc)contribution4<T>(Fc, wyz, w[0][dx]));
                    }
                }
            }
        }
    }
    __syncthreads();
    const long long nx = a.n[0], nxy = (long long)a.n[0] * a.n[1];
    unsigned long long *acc = a.acc + (long long)c * nxy * a.n[2];
    for (int i = threadIdx.x; i < B3; i += kBox4Threads) {
        const Acc b = box[i];
        if (b == Acc(0))
            continue;
        const unsigned long long v = (unsigned long long)((long long)b * (1LL << kShift));
        const int loc[3] = {i % B, (i / B) % B, i / (B * B)};
        long long g[3];
        bool in = true;
#pragma unroll
        for (int ax = 0; ax < 3; ax++) {
            int k = pp.base[c * 3 + ax] - rh - 2 + loc[ax];
            if (a.periodic[ax]) {
                while (k < 0)
                    k += a.n[ax];
                while (k >= a.n[ax])
                    k -= a.n[ax];
            } else {
                in = in && k >= 0 && k < a.n[ax];
            }
            g[ax] = k;
        }
        if (in)
            atomicAdd(acc + g[2] * nxy + g[1] * nx + g[0], v);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_apply4(Args4<T> a)
{
    const long long cells = (long long)a.n[0] * a.n[1] * a.n[2];
    const T adt = (T)a.adt;
    double unit[3];
#pragma unroll
    for (int c = 0; c < 3; c++)
        unit[c] = ldexp(1.0, -scale_exp(a, c));
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cells;
         i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const long long v = (long long)a.acc[c * cells + i];
            if (v == 0)
                continue;
            const T d = (T)((double)v * unit[c]);
            a.out_f[c][i] = a.out_f[c][i] + d;
            a.out_u[c][i] = a.out_u[c][i] + adt * d;
            a.acc[c * cells + i] = 0ULL;
        }
    }
}

template <typename T>
Args4<T> args4(const Ctx &c)
{
    Args4<T> a{};
    a.prep = (const PartPrep<T> *)c.prep;
    a.tR = (const T *)c.tR;
    a.rR = (const T *)c.rR;
    a.Fl = (T *)c.Fl;
    a.dFl = (T *)c.dFl;
    a.red = c.d_red;
    a.acc = c.acc4;
    a.err = c.d_err;
    a.same_off = c.g.same_off ? 1 : 0;
    for (int k = 0; k < 3; k++) {
        a.n[k] = c.g.n[k];
        a.periodic[k] = c.g.periodic[k];
    }
    a.n_l = c.n_l;
    a.n_m = (long long)c.n_p * c.n_l;
    a.l_magic = c.l_magic;
    a.dVh3 = c.dV / (c.g.h * c.g.h * c.g.h);
    return a;
}

}  // namespace

template <typename T>
void ibm4_interp_force(Ctx &c, const T *u, const T *v, const T *w, int pass, double inv_adt,
                       int probe, cudaStream_t s)
{
    Args4<T> a = args4<T>(c);
    a.fld[0] = u;
    a.fld[1] = v;
    a.fld[2] = w;
    a.pass = pass;
    a.probe = probe;
    a.inv_adt = (T)inv_adt;
    const int blocks = (int)((a.n_m + 255) / 256);
    k_interp4<T><<<blocks, 256, 0, s>>>(a);
    c.n_launch += 1;
}

template <typename T>
void ibm4_spread(Ctx &c, T *u, T *v, T *w, T *fx, T *fy, T *fz, int pass, double adt,
                 cudaStream_t s)
{
    Args4<T> a = args4<T>(c);
    a.pass = pass;
    a.adt = adt;
    T *f[3] = {fx, fy, fz}, *uu[3] = {u, v, w};
    for (int k = 0; k < 3; k++) {
        a.out_f[k] = f[k];
        a.out_u[k] = uu[k];
    }
    // per sphere in shared memory when its box fits, else per marker
    const int rh = (int)std::ceil(c.R / c.g.h);
    const bool small = sizeof(T) == 8 || c.n_l <= kBox4MaxMarkers32;
    const size_t box = (sizeof(T) == 4 ? sizeof(int) : sizeof(unsigned long long)) *
                       (size_t)(2 * rh + 6) * (2 * rh + 6) * (2 * rh + 6);
    if (small && box <= 48 * 1024) {
        k_spread4_box<T><<<dim3((unsigned)c.n_p, 3), kBox4Threads, box, s>>>(a, rh);
    } else {
        const int blocks = (int)((a.n_m + 255) / 256);
        k_spread4<T><<<blocks, 256, 0, s>>>(a);
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_apply4<T><<<8 * sms, 256, 0, s>>>(a);
    c.n_launch += 2;
}

template void ibm4_interp_force<float>(Ctx &, const float *, const float *, const float *, int,
                                       double, int, cudaStream_t);
template void ibm4_interp_force<double>(Ctx &, const double *, const double *, const double *,
                                        int, double, int, cudaStream_t);
template void ibm4_spread<float>(Ctx &, float *, float *, float *, float *, float *, float *, int,
                                 double, cudaStream_t);
template void ibm4_spread<double>(Ctx &, double *, double *, double *, double *, double *,
                                  double *, int, double, cudaStream_t);

}  // namespace prs
