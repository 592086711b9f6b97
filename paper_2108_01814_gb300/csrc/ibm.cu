// Direct-forcing immersed boundary kernels (Sec. 2.1 and 3.3 of the paper):
// markers generated on the fly from the shared template (Sec. 3.5),
// interpolation of the fluid velocity with the 3-point regularised delta,
// direct forcing, per-particle force/torque sums, and a deterministic
// spreading of the marker forces back to the grid.
//
// Precision: T = double (FP64 form) or float (FP32 form). Positions are
// kept as an FP64 grid index plus a remainder in [0, 1), so the FP32 form
// loses no accuracy on large grids.
#include <cstdio>

#include "prs_internal.cuh"

namespace prs {
namespace {

constexpr int kInterpThreads = 256;
constexpr int kMaxNb = 125;  // neighbour tiles for a reach of up to 2 tiles

template <typename T>
struct IbmArgs {
    const PartPrep<T> *prep;
    const T *tR;  // [3][n_l] R/h t_l
    const T *rR;  // [3][n_l] R t_l
    const T *u, *v, *w;
    T *Fl, *dFl;
    double *Fh, *Th;
    unsigned long long *red;
    int n[3];
    int periodic[3];
    int n_p, n_l;
    int pass;
    int probe;  // 1: only measure the slip max |U_d - U|, write nothing else
    T inv_adt;
    double neg_rho_dV;
};

template <typename T>
struct SpreadArgs {
    const PartPrep<T> *prep;
    const T *tR;
    const T *F;  // the force increment being spread, [3][n_m]
    T *f[3];
    T *uvw[3];
    const int *tile_start, *tile_list;
    const unsigned long long *red;
    int n[3];
    int periodic[3];
    int nt[3];
    int reach;
    int n_p, n_l;
    double dVh3;
    double adt;
};

// Weights of the 3-point kernel (Roma, Peskin & Berger 1999) along one
// axis for a point at grid coordinate q: i0 = nearest index, w[d] is the
// weight of index i0 - 1 + d. With r1 = i0 - q in [-1/2, 1/2], all three
// branches share the root sqrt(1 - 3 r1^2).
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

// compensated (Kahan) sum: value = s - c
template <typename T>
struct KSum {
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

template <typename T>
__global__ void k_prep(const double *__restrict__ x, const double *__restrict__ up,
                       const double *__restrict__ om, int n_p, GridDesc g,
                       PartPrep<T> *__restrict__ prep)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_p)
        return;
    PartPrep<T> pp;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        double xs = x[a * n_p + p] / g.h;
        if (g.periodic[a]) {
            // one periodic image for all components: xs in [0, n)
            const double n = (double)g.n[a];
            xs -= n * floor(xs / n);
            if (xs >= n)
                xs = 0.0;
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
}

// ------------------------------------------------------------------ interp + force
template <typename T, bool SAME>
__global__ void __launch_bounds__(kInterpThreads) k_interp_force(IbmArgs<T> a)
{
    const int lane = threadIdx.x & 31;
    const int p = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (p >= a.n_p)
        return;
    const PartPrep<T> &pp = a.prep[p];
    const int n_l = a.n_l;
    const long long n_m = (long long)a.n_p * n_l;
    const long long nx = a.n[0], nxy = (long long)a.n[0] * a.n[1];
    const T *fld[3] = {a.u, a.v, a.w};

    KSum<T> fs[3], ts[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        fs[k].init();
        ts[k].init();
    }
    T res = T(0), fmax = T(0);

    for (int l = lane; l < n_l; l += 32) {
        T rt[3], rr[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            rt[k] = a.tR[k * n_l + l];
            rr[k] = a.rR[k * n_l + l];
        }
        T U[3];
        long long idx[3][3];
        T w[3][3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            if (c == 0 || !SAME) {
#pragma unroll
                for (int ax = 0; ax < 3; ax++) {
                    int i0;
                    axis_weights(pp.frac[c * 3 + ax] + rt[ax], i0, w[ax]);
                    const int n = a.n[ax];
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        int gi = pp.base[c * 3 + ax] + i0 - 1 + d;
                        if (a.periodic[ax]) {
                            if (gi < 0)
                                gi += n;
                            else if (gi >= n)
                                gi -= n;
                        } else if (gi < 0 || gi >= n) {
                            w[ax][d] = T(0);
                            gi = 0;
                        }
                        idx[ax][d] = gi;
                    }
                }
            }
            const T *__restrict__ f = fld[c];
            T acc = T(0);
#pragma unroll
            for (int dz = 0; dz < 3; dz++) {
#pragma unroll
                for (int dy = 0; dy < 3; dy++) {
                    const T wyz = w[1][dy] * w[2][dz];
                    const long long row = idx[2][dz] * nxy + idx[1][dy] * nx;
#pragma unroll
                    for (int dx = 0; dx < 3; dx++)
                        acc += __ldg(f + row + idx[0][dx]) * (w[0][dx] * wyz);
                }
            }
            U[c] = acc;
        }
        // rigid-body velocity of the surface point, U_d = u_p + omega_p x r
        T Ud[3];
        Ud[0] = pp.up[0] + (pp.om[1] * rr[2] - pp.om[2] * rr[1]);
        Ud[1] = pp.up[1] + (pp.om[2] * rr[0] - pp.om[0] * rr[2]);
        Ud[2] = pp.up[2] + (pp.om[0] * rr[1] - pp.om[1] * rr[0]);
        if (a.probe) {
#pragma unroll
            for (int c = 0; c < 3; c++)
                res = max(res, fabs(Ud[c] - U[c]));
            continue;
        }
        T F[3];
        const long long m = (long long)p * n_l + l;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            T slip = Ud[c] - U[c];
            res = max(res, fabs(slip));
            T dF = slip * a.inv_adt;
            fmax = max(fmax, fabs(dF));
            if (a.pass == 0) {
                F[c] = dF;
            } else {
                F[c] = a.Fl[c * n_m + m] + dF;
                a.dFl[c * n_m + m] = dF;
            }
            a.Fl[c * n_m + m] = F[c];
        }
        // per-particle sums (modification (2) of Sec. 3.3)
#pragma unroll
        for (int c = 0; c < 3; c++)
            fs[c].add(F[c]);
        ts[0].add(rr[1] * F[2] - rr[2] * F[1]);
        ts[1].add(rr[2] * F[0] - rr[0] * F[2]);
        ts[2].add(rr[0] * F[1] - rr[1] * F[0]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            T s2 = __shfl_xor_sync(0xffffffffu, fs[k].s, o);
            T c2 = __shfl_xor_sync(0xffffffffu, fs[k].c, o);
            fs[k].merge(s2, c2);
            s2 = __shfl_xor_sync(0xffffffffu, ts[k].s, o);
            c2 = __shfl_xor_sync(0xffffffffu, ts[k].c, o);
            ts[k].merge(s2, c2);
        }
        res = max(res, __shfl_xor_sync(0xffffffffu, res, o));
        fmax = max(fmax, __shfl_xor_sync(0xffffffffu, fmax, o));
    }
    if (lane == 0) {
        if (!a.probe) {
#pragma unroll
            for (int k = 0; k < 3; k++) {
                a.Fh[k * a.n_p + p] = a.neg_rho_dV * ((double)fs[k].s - (double)fs[k].c);
                a.Th[k * a.n_p + p] = a.neg_rho_dV * ((double)ts[k].s - (double)ts[k].c);
            }
            atomicMax(&a.red[0], max_bits(fmax));
        }
        atomicMax(&a.red[1], max_bits(res));
    }
}

// ------------------------------------------------------------------ tile binning
__global__ void k_tile_count(const int *__restrict__ base0, int stride, int n_p, GridDesc g,
                             int nt0, int nt1, int nt2, int *__restrict__ ptile,
                             int *__restrict__ count)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_p)
        return;
    const int *b = base0 + (long long)p * stride;
    int nt[3] = {nt0, nt1, nt2};
    int t[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        int ti = b[a] >= 0 ? b[a] / kTile : -1;
        t[a] = min(max(ti, 0), nt[a] - 1);
    }
    int key = t[0] + nt0 * (t[1] + nt1 * t[2]);
    ptile[p] = key;
    atomicAdd(&count[key], 1);
}

__global__ void k_tile_scatter(int n_p, const int *__restrict__ ptile,
                               const int *__restrict__ start, int *__restrict__ count,
                               int *__restrict__ list)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_p)
        return;
    int key = ptile[p];
    list[start[key] + atomicSub(&count[key], 1) - 1] = p;
}

__global__ void k_set_int2(int *ptr, int v) { *ptr = v; }

// ------------------------------------------------------------------ spread
// One CTA per tile of 8^3 cells. Every marker whose 27-point stencil
// reaches the tile adds its contributions F phi phi phi dV / h^3 to a
// shared-memory accumulator in 64-bit fixed point. Integer addition is
// associative, so the sums, and the fields written from them, do not depend
// on the order in which threads arrive: the spread is bit-reproducible
// without floating-point atomics.
template <typename T, bool SAME>
__global__ void __launch_bounds__(kSpreadThreads) k_spread(SpreadArgs<T> a)
{
    __shared__ unsigned long long acc[3][kTileCells];
    __shared__ unsigned char touched[3][kTileCells];
    __shared__ int nb_beg[kMaxNb], nb_cnt[kMaxNb], nb_off[kMaxNb + 1];
    __shared__ int nb_shift[kMaxNb][3];
    __shared__ int cand_p[kMaxCand];
    __shared__ int cand_rel[kMaxCand][3];
    __shared__ int s_nnb;

    const int tid = threadIdx.x;
    int tile = blockIdx.x;
    int tc[3];
    tc[0] = tile % a.nt[0];
    tc[1] = (tile / a.nt[0]) % a.nt[1];
    tc[2] = tile / (a.nt[0] * a.nt[1]);
    int org[3], ext[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        org[k] = tc[k] * kTile;
        ext[k] = min(kTile, a.n[k] - org[k]);
    }
    const int span = 2 * a.reach + 1;
    const int nnb = span * span * span;

    // neighbour tiles (with periodic images) and their particle counts
    if (tid < nnb) {
        int d[3] = {tid % span - a.reach, (tid / span) % span - a.reach,
                    tid / (span * span) - a.reach};
        int ok = 1, key = 0, mul = 1;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            int t = tc[k] + d[k];
            int sh = 0;
            if (t < 0 || t >= a.nt[k]) {
                if (!a.periodic[k]) {
                    ok = 0;
                } else if (t < 0) {
                    t += a.nt[k];
                    sh = -a.n[k];
                } else {
                    t -= a.nt[k];
                    sh = a.n[k];
                }
            }
            key += t * mul;
            mul *= a.nt[k];
            nb_shift[tid][k] = sh;
        }
        // with fewer tiles than the span along a periodic axis the same tile
        // appears as several images; each is a distinct translate and is kept
        nb_beg[tid] = ok ? a.tile_start[key] : 0;
        nb_cnt[tid] = ok ? a.tile_start[key + 1] - a.tile_start[key] : 0;
    }
    __syncthreads();
    if (tid == 0) {
        int s = 0;
        for (int k = 0; k < nnb; k++) {
            nb_off[k] = s;
            s += nb_cnt[k];
        }
        nb_off[nnb] = s;
        s_nnb = nnb;
    }
    __syncthreads();
    const int total = nb_off[s_nnb];
    const T fmax = from_bits<T>(a.red[0]);
    if (total == 0 || !(fmax > T(0)))
        return;

    // fixed-point scale: a power of two such that the sum of magnitudes of
    // all contributions to one cell stays below 2^61
    const double bound = (double)total * a.n_l * (8.0 / 27.0) * (double)fmax * a.dVh3;
    int e;
    frexp(bound, &e);
    const double scale = ldexp(1.0, 61 - e);
    const double inv_scale = ldexp(1.0, e - 61);
    const T cscale = (T)(a.dVh3 * scale);

    for (int i = tid; i < 3 * kTileCells; i += blockDim.x) {
        (&acc[0][0])[i] = 0ULL;
        (&touched[0][0])[i] = 0;
    }

    const int n_l = a.n_l;
    const long long n_m = (long long)a.n_p * n_l;
    for (int c0 = 0; c0 < total; c0 += kMaxCand) {
        const int nc = min(kMaxCand, total - c0);
        __syncthreads();
        for (int j = tid; j < nc; j += blockDim.x) {
            int gj = c0 + j;
            int k = 0;
            while (nb_off[k + 1] <= gj)
                k++;
            int p = a.tile_list[nb_beg[k] + (gj - nb_off[k])];
            cand_p[j] = p;
#pragma unroll
            for (int ax = 0; ax < 3; ax++)
                cand_rel[j][ax] = nb_shift[k][ax] - org[ax];
        }
        __syncthreads();
        const int work = nc * n_l;
        for (int it = tid; it < work; it += blockDim.x) {
            const int j = it / n_l;
            const int l = it - j * n_l;
            const int p = cand_p[j];
            const PartPrep<T> &pp = a.prep[p];
            T rt[3];
#pragma unroll
            for (int k = 0; k < 3; k++)
                rt[k] = a.tR[k * n_l + l];
            const long long m = (long long)p * n_l + l;
            int lo[3];
            T w[3][3];
            bool inside = false;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                if (c == 0 || !SAME) {
                    inside = true;
#pragma unroll
                    for (int ax = 0; ax < 3; ax++) {
                        int i0;
                        axis_weights(pp.frac[c * 3 + ax] + rt[ax], i0, w[ax]);
                        lo[ax] = pp.base[c * 3 + ax] + cand_rel[j][ax] + i0 - 1;
                        inside = inside && lo[ax] >= -2 && lo[ax] < ext[ax];
                    }
                }
                if (!inside)
                    continue;
                const T Fc = a.F[c * n_m + m] * cscale;
#pragma unroll
                for (int dz = 0; dz < 3; dz++) {
                    const int cz = lo[2] + dz;
                    if (cz < 0 || cz >= ext[2])
                        continue;
#pragma unroll
                    for (int dy = 0; dy < 3; dy++) {
                        const int cy = lo[1] + dy;
                        if (cy < 0 || cy >= ext[1])
                            continue;
                        const T fyz = Fc * (w[1][dy] * w[2][dz]);
#pragma unroll
                        for (int dx = 0; dx < 3; dx++) {
                            const int cx = lo[0] + dx;
                            if (cx < 0 || cx >= ext[0])
                                continue;
                            const int cell = cx + kTile * (cy + kTile * cz);
                            const long long v = llrint((double)(fyz * w[0][dx]));
                            atomicAdd(&acc[c][cell], (unsigned long long)v);
                            touched[c][cell] = 1;
                        }
                    }
                }
            }
        }
    }
    __syncthreads();

    const long long nx = a.n[0], nxy = (long long)a.n[0] * a.n[1];
    for (int cell = tid; cell < kTileCells; cell += blockDim.x) {
        const int cx = cell % kTile, cy = (cell / kTile) % kTile, cz = cell / (kTile * kTile);
        if (cx >= ext[0] || cy >= ext[1] || cz >= ext[2])
            continue;
        const long long gidx = (org[2] + cz) * nxy + (org[1] + cy) * nx + (org[0] + cx);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            if (!touched[c][cell])
                continue;
            const double sv = (double)(long long)acc[c][cell] * inv_scale;
            a.f[c][gidx] += (T)sv;
            a.uvw[c][gidx] += (T)(a.adt * sv);
        }
    }
}

}  // namespace

template <typename T>
void ibm_prep(Ctx &c, cudaStream_t s)
{
    k_prep<T><<<(c.n_p + 255) / 256, 256, 0, s>>>(c.x[c.cur], c.u[c.cur], c.om[c.cur], c.n_p,
                                                  c.g, (PartPrep<T> *)c.prep);
    c.n_launch += 1;
}

void ibm_tile_bin(Ctx &c, cudaStream_t s)
{
    const int nb = (c.n_p + 255) / 256;
    // component 0 base indices: first 3 ints of each PartPrep record
    const int stride = c.precision == PRS_FP64 ? (int)(sizeof(PartPrep<double>) / sizeof(int))
                                               : (int)(sizeof(PartPrep<float>) / sizeof(int));
    k_tile_count<<<nb, 256, 0, s>>>((const int *)c.prep, stride, c.n_p, c.g, c.nt[0], c.nt[1],
                                    c.nt[2], c.ptile, c.tile_count);
    int k = exclusive_scan(c.tile_count, c.tile_start, c.ntile, c.tile_scan_tmp, s);
    k_set_int2<<<1, 1, 0, s>>>(c.tile_start + c.ntile, c.n_p);
    k_tile_scatter<<<nb, 256, 0, s>>>(c.n_p, c.ptile, c.tile_start, c.tile_count, c.tile_list);
    c.n_launch += 3 + k;
}

template <typename T>
void ibm_interp_force(Ctx &c, const T *u, const T *v, const T *w, int pass,
                      double inv_adt, int probe, cudaStream_t s)
{
    IbmArgs<T> a;
    a.probe = probe;
    a.prep = (const PartPrep<T> *)c.prep;
    a.tR = (const T *)c.tR;
    a.rR = (const T *)c.rR;
    a.u = u;
    a.v = v;
    a.w = w;
    a.Fl = (T *)c.Fl;
    a.dFl = (T *)c.dFl;
    a.Fh = c.Fh;
    a.Th = c.Th;
    a.red = c.d_red;
    for (int k = 0; k < 3; k++) {
        a.n[k] = c.g.n[k];
        a.periodic[k] = c.g.periodic[k];
    }
    a.n_p = c.n_p;
    a.n_l = c.n_l;
    a.pass = pass;
    a.inv_adt = (T)inv_adt;
    a.neg_rho_dV = -c.rho_f * c.dV;
    const long long threads = (long long)c.n_p * 32;
    const int blocks = (int)((threads + kInterpThreads - 1) / kInterpThreads);
    phase_begin(c, 1);
    if (c.g.same_off)
        k_interp_force<T, true><<<blocks, kInterpThreads, 0, s>>>(a);
    else
        k_interp_force<T, false><<<blocks, kInterpThreads, 0, s>>>(a);
    phase_end(c);
    c.n_launch += 1;
}

template <typename T>
void ibm_spread(Ctx &c, T *u, T *v, T *w, T *fx, T *fy, T *fz, int pass, double adt,
                cudaStream_t s)
{
    SpreadArgs<T> a;
    a.prep = (const PartPrep<T> *)c.prep;
    a.tR = (const T *)c.tR;
    a.F = (const T *)(pass == 0 ? c.Fl : c.dFl);
    a.f[0] = fx;
    a.f[1] = fy;
    a.f[2] = fz;
    a.uvw[0] = u;
    a.uvw[1] = v;
    a.uvw[2] = w;
    a.tile_start = c.tile_start;
    a.tile_list = c.tile_list;
    a.red = c.d_red;
    for (int k = 0; k < 3; k++) {
        a.n[k] = c.g.n[k];
        a.periodic[k] = c.g.periodic[k];
        a.nt[k] = c.nt[k];
    }
    a.reach = c.reach;
    a.n_p = c.n_p;
    a.n_l = c.n_l;
    a.dVh3 = c.dV / (c.g.h * c.g.h * c.g.h);
    a.adt = adt;
    phase_begin(c, 2);
    if (c.g.same_off)
        k_spread<T, true><<<c.ntile, kSpreadThreads, 0, s>>>(a);
    else
        k_spread<T, false><<<c.ntile, kSpreadThreads, 0, s>>>(a);
    phase_end(c);
    c.n_launch += 1;
}

template void ibm_prep<float>(Ctx &, cudaStream_t);
template void ibm_prep<double>(Ctx &, cudaStream_t);
template void ibm_interp_force<float>(Ctx &, const float *, const float *, const float *, int,
                                      double, int, cudaStream_t);
template void ibm_interp_force<double>(Ctx &, const double *, const double *, const double *,
                                       int, double, int, cudaStream_t);
template void ibm_spread<float>(Ctx &, float *, float *, float *, float *, float *, float *,
                                int, double, cudaStream_t);
template void ibm_spread<double>(Ctx &, double *, double *, double *, double *, double *,
                                 double *, int, double, cudaStream_t);

}  // namespace prs
