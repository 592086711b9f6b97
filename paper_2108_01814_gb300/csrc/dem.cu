// Soft-sphere DEM on the GPU: cell-list contact search, contact history with
// at most 12 slots per sphere (Sec. 3.4), linear spring-dashpot forces with a
// Coulomb cap (Sec. 2.1, Eq. 9-10, Appendix A.1-A.11) and the semi-implicit
// Newton-Euler update of Eq. 7-8 in rigid-body form.
//
// One sub-step is two kernels:
//   k_dem_contacts  every sphere finds its contacts (ascending ids); for the
//                   pairs where it has the lower id it evaluates the pair
//                   force once, in canonical orientation, and keeps the pair's
//                   history (impact velocity, tangential displacement) and
//                   force in its own slots;
//   k_dem_update    every sphere sums its pair forces in ascending partner
//                   order (reading the partner's slot, negated, where the
//                   partner has the lower id), adds wall contacts and
//                   integrates.
//
// Precision. FP64 form: everything FP64, evaluated as written (this unit is
// compiled with --fmad=false), so contact decisions and contact forces are
// reproducible bit for bit from a given state. FP32 form: the sphere state
// and the stored tangential displacement stay FP64; the spring-dashpot
// arithmetic and the accelerations are FP32, their increments added to the
// FP64 values; the rotation of the stored displacement onto the new tangent
// plane (A.9-A.10) is an FP32 correction to the FP64 value. Positions are
// also held as unevaluated FP32 pairs (x = xf + xl), from which the overlap
// takes d^2 - 4R^2 in pair arithmetic with FP64 accuracy. Contact decisions
// match the FP64 form exactly: the FP32 distance where it is clear, the pair
// arithmetic within its error bound, the FP64 distance inside that bound. On
// GB300 FP64 arithmetic and FP64/FP32 conversions share a slow pipe, so the
// FP32 form converts with integer operations.
#include <cstdio>

#include <algorithm>
#include <cmath>

#include "prs_internal.cuh"

namespace prs {
namespace {

constexpr int kDemThreads = 128;
// both sub-step kernels wait on dependent gathers: in the FP32 form the
// contact kernel keeps 12 resident blocks per SM (40 registers, a few
// spills; 10 blocks were 2 % slower on the million-sphere bed) and the
// update 10 (48 registers; 12 were slower); the FP64 form keeps 6 (up to
// 80 registers, no spills)
constexpr int kDemMinBlocksContacts = 12;
constexpr int kDemMinBlocksUpdate = 10;
constexpr int S = PRS_MAX_CONTACTS;

struct HistPtrs {
    int *cnt;       // lower-id pair slots in use
    int *pid;       // partner id (ascending)
    double *uin;    // impact velocity
    double *dlt;    // tangential displacement [3]
    unsigned char *wact;
    double *wuin;
    double *wdlt;
};

template <typename T>
struct DemArgs {
    const double *x, *u, *om;
    const float *xf, *uf, *omf;      // FP32 copies of x, u, omega
    const float *xl;                 // FP32 remainders x - xf
    double *xn, *un, *omn;
    float *xfn, *ufn, *omfn, *xln;
    const double *Fh, *Th;
    double *Fc, *Tc;
    HistPtrs ho, hn;
    T *pairFT;                       // [S][n_p][6]: force on the lower id, torque
    int *ccnt, *clist;               // owned contacts per sphere; clist is not read here (its storage holds inc)
    const int *sorted, *start, *pcell;
    CellGeom cg;
    DemParams dp;
    double dt_p;
    double inv_m, inv_J;
    float cut2_f32;   // (2R + eps)^2: beyond it in FP32 a pair cannot touch
    float in2_f32;    // (2R - eps)^2: below it in FP32 a pair surely touches
    float halfL[3], Lf[3];
    const float *xb;  // positions at the last cell-list build
    float move2_f32;  // (skin/2 - eps)^2: moving further forces a rebuild
    float wall_f32;   // R + eps: an FP32 wall distance beyond it cannot touch
    int *rebuild;
    int n_p;
    int *err;
    double four_R2;   // 4 R^2
    float four_R2h, four_R2l;  // 4 R^2 as an unevaluated FP32 pair
    float band_D;     // error bound of d^2 - 4R^2 in pair arithmetic
    float two_Rf;     // 2 R
    float Rf;         // R
    // FP32 copies of the contact constants: sphere-sphere, sphere-wall
    float kn_pp, dn_pp, kt_pp, dt_pp, kn_pw, dn_pw, kt_pw, dt_pw, mu, dtp_f;
    // FP32 form: FP32 hydrodynamic load, collision outputs and constants
    const float *Fhf, *Thf;
    float *Fcf, *Tcf;
    float inv_m_f, inv_J_f, dt_f, g_f[3];
    int last;  // last sub-step of the call: the collision force is kept
    const int *nlist, *ncnt;  // neighbour list [ncap][n_p], ascending ids
    const int *nlo;           // its leading entries with ids below the sphere's
    int *inc, *inc_cnt;       // pairs owned by lower ids: [S][n_p] (id * 16 + slot), counts
    const double *flub;       // lubrication force per sphere [3][n_p], or null (off)
};

// finite test on the exponent bits (integer pipe)
__device__ __forceinline__ bool finite_bits(double v)
{
    return (__double2hiint(v) & 0x7ff00000) != 0x7ff00000;
}

// Conversions between FP64 and FP32 by integer operations. The conversion
// instructions share the FP64 pipe, which is slow on this GPU, and the FP32
// form of the contact kernels is bound by it.
// FP64 -> FP32 rounded toward zero (error below 1 ulp of the FP32 result);
// magnitudes below 2^-126 give a signed zero, overflow, infinity and NaN
// give NaN.
__device__ __forceinline__ float f32_rz(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned bits = e <= 0 ? sign : (e >= 255 ? (sign | 0x7fc00000u)
                                                     : (sign | ((unsigned)e << 23) | m));
    return __uint_as_float(bits);
}
// FP32 -> FP64, exact for normal numbers and zero (FP32 subnormals become
// zero), infinity and NaN kept
__device__ __forceinline__ double f64_of(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u, ex = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    unsigned hi = sign, lo = 0u;
    if (ex == 255u) {
        hi = sign | 0x7ff00000u | (m >> 3);
        lo = m << 29;
    } else if (ex != 0u) {
        hi = sign | ((ex + 896u) << 20) | (m >> 3);
        lo = m << 29;
    }
    return __hiloint2double((int)hi, (int)lo);
}

// s + err = a + b exactly, s = fl(a + b) (Knuth's TwoSum)
__device__ __forceinline__ float two_sum(float a, float b, float &err)
{
    const float s = a + b;
    const float bb = s - a;
    err = (a - (s - bb)) + (b - bb);
    return s;
}

__device__ __forceinline__ void cell_coords(int key, const CellGeom &cg, int c[3])
{
    c[0] = key % cg.nc[0];
    int r = key / cg.nc[0];
    c[1] = r % cg.nc[1];
    c[2] = r / cg.nc[1];
}

// neighbour cell offsets along one axis, without repeats
__device__ __forceinline__ int axis_offsets(const CellGeom &cg, int a, int c, int idx[3])
{
    const int nc = cg.nc[a];
    int k = 0;
    if (cg.periodic[a]) {
        if (nc >= 3) {
            idx[k++] = (c + nc - 1) % nc;
            idx[k++] = c;
            idx[k++] = (c + 1) % nc;
        } else {
            for (int i = 0; i < nc; i++)
                idx[k++] = i;
        }
    } else {
        for (int d = -1; d <= 1; d++) {
            int i = c + d;
            if (i >= 0 && i < nc)
                idx[k++] = i;
        }
    }
    return k;
}

// separation lo -> hi with minimum image and its length (Eq. A.1, A.3)
__device__ __forceinline__ double pair_vector(const DemParams &dp, const double xl[3],
                                              const double xh[3], double dx[3])
{
#pragma unroll
    for (int k = 0; k < 3; k++) {
        double s = xh[k] - xl[k];
        if (dp.periodic[k]) {
            double L = dp.L[k];
            if (s > 0.5 * L)
                s -= L;
            else if (s < -0.5 * L)
                s += L;
        }
        dx[k] = s;
    }
    double d2 = (dx[0] * dx[0] + dx[1] * dx[1]) + dx[2] * dx[2];
    return sqrt(d2);
}

// FP32 squared distance with minimum image; its error is a few ulp of the
// domain size, and callers compare it with cutoffs widened by that bound
__device__ __forceinline__ float pair_dist2_f32(const float a[3], const float b[3],
                                                const int periodic[3], const float halfL[3],
                                                const float L[3])
{
    float d2 = 0.f;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        float s = b[k] - a[k];
        if (periodic[k]) {
            if (s > halfL[k])
                s -= L[k];
            else if (s < -halfL[k])
                s += L[k];
        }
        d2 = __fmaf_rn(s, s, d2);
    }
    return d2;
}

template <typename T>
__device__ __forceinline__ void cross3(const T a[3], const T b[3], T c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// A pair's force and torque: one entry of six contiguous values per slot and
// sphere, moved as three 2-vectors, so a gather of a partner's entry touches
// one or two 32-byte sectors instead of six.
template <typename T>
struct Vec2Of;
template <>
struct Vec2Of<float> {
    using type = float2;
};
template <>
struct Vec2Of<double> {
    using type = double2;
};

template <typename T>
__device__ __forceinline__ T *pair_entry(T *base, int slot, int sphere, int n_p)
{
    return base + ((long long)slot * n_p + sphere) * 6;
}

template <typename T>
__device__ __forceinline__ void load_pair(const T *e, T (&v)[6])
{
    using V = typename Vec2Of<T>::type;
    const V *q = reinterpret_cast<const V *>(e);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const V t = q[i];
        v[2 * i] = t.x;
        v[2 * i + 1] = t.y;
    }
}

template <typename T>
__device__ __forceinline__ void store_pair(T *e, const T (&F)[3], const T (&Tq)[3])
{
    using V = typename Vec2Of<T>::type;
    V *q = reinterpret_cast<V *>(e);
    q[0] = V{F[0], F[1]};
    q[1] = V{F[2], Tq[0]};
    q[2] = V{Tq[1], Tq[2]};
}

template <typename T>
__device__ __forceinline__ T dot3(const T a[3], const T b[3])
{
    return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

// FP64 contact force (A.7-A.11 and the spring-dashpot law), seen from the
// particle with contact velocity ucp.
// model 1 (adaptive collision time): kn holds m_eff tau^(-5/2), the
// contact's stiffness is kn / sqrt(vin) with vin = max(|u_in|, u_min), and
// the spring is Hertzian, kn / sqrt(vin) |delta_n|^(3/2)
__device__ __forceinline__ void contact_force64(const double n[3], double delta_n,
                                                const double ucp[3], const double dprev[3],
                                                double kn, double dn, double kt, double dtc,
                                                double mu, double dt_p, bool clip, int model,
                                                double vin, double Fn[3], double Ft[3],
                                                double dnew[3])
{
    double un = dot3(ucp, n);
    double ucpt[3];
#pragma unroll
    for (int k = 0; k < 3; k++)
        ucpt[k] = ucp[k] - un * n[k];
    double dd = dot3(dprev, n);
    double dtil[3];
#pragma unroll
    for (int k = 0; k < 3; k++)
        dtil[k] = dprev[k] - dd * n[k];
    double nprev = sqrt(dot3(dprev, dprev));
    double ntil = sqrt(dot3(dtil, dtil));
#pragma unroll
    for (int k = 0; k < 3; k++) {
        double dhat = (ntil > 0.0) ? (nprev / ntil) * dtil[k] : 0.0;
        dnew[k] = dhat + dt_p * ucpt[k];
    }
    double s = kn * delta_n - dn * un;
    if (model) {
        const double k = kn / sqrt(vin);
        const double ov = -delta_n;
        s = -(k * (ov * sqrt(ov))) - dn * un;
    }
    if (clip && s > 0.0)  // repulsive only (s < 0 pushes the sphere away along -n)
        s = 0.0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        Fn[k] = s * n[k];
        Ft[k] = -(kt * dnew[k]) - dtc * ucpt[k];
    }
    double fn = fabs(s);
    double ft = sqrt(dot3(Ft, Ft));
    if (ft > mu * fn) {
        double scale = mu * fn / ft;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            Ft[k] = scale * Ft[k];
            dnew[k] = -(Ft[k] + dtc * ucpt[k]) / kt;
        }
    }
}

// The same law for the FP32 form: FP32 forces from FP64 overlap and FP64
// stored displacement. A.9-A.10 rotate the stored displacement onto the
// plane normal to n keeping its length: with dd = delta.n and
// e = dd^2 / |delta|^2 the rotated vector is delta + r1 delta - (1 + r1) dd n,
// r1 = e / (sqrt(1 - e) (1 + sqrt(1 - e))). This correction and the A.11
// increment dt_p u_cp,t are small; they are formed in FP32 and added to the
// FP64 value, so the stored displacement keeps FP64 accuracy.
__device__ __forceinline__ void contact_force_mixed(const float n[3], float delta_n,
                                                    const float ucp[3], const double dprev[3],
                                                    float kn, float dn, float kt, float dtc,
                                                    float mu, float dt_p, bool clip, int model,
                                                    float vin, float Fn[3], float Ft[3],
                                                    double dnew[3])
{
    float un = dot3(ucp, n);
    float ucpt[3];
#pragma unroll
    for (int k = 0; k < 3; k++)
        ucpt[k] = ucp[k] - un * n[k];
    float dp[3] = {f32_rz(dprev[0]), f32_rz(dprev[1]), f32_rz(dprev[2])};
    float dd = dot3(dp, n);
    float p2 = dot3(dp, dp);
    float corr[3] = {0.f, 0.f, 0.f};
    if (p2 > 0.f) {
        float e = dd * dd / p2;
        if (e < 1.f) {
            float sq = sqrtf(1.f - e);
            float r1 = e / (sq * (1.f + sq));
#pragma unroll
            for (int k = 0; k < 3; k++)
                corr[k] = r1 * dp[k] - (1.f + r1) * dd * n[k];
        } else {
#pragma unroll
            for (int k = 0; k < 3; k++)
                corr[k] = -dp[k];
        }
    }
    float dnf[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float inc = corr[k] + dt_p * ucpt[k];
        dnew[k] = dprev[k] + f64_of(inc);
        dnf[k] = dp[k] + inc;  // the force needs FP32 only
    }
    float s = kn * delta_n - dn * un;
    if (model) {
        const float ov = -delta_n;
        s = -((kn * rsqrtf(vin)) * (ov * sqrtf(ov))) - dn * un;
    }
    if (clip && s > 0.f)
        s = 0.f;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        Fn[k] = s * n[k];
        Ft[k] = -(kt * dnf[k]) - dtc * ucpt[k];
    }
    float fn = fabsf(s);
    float ft = sqrtf(dot3(Ft, Ft));
    if (ft > mu * fn) {
        float scale = mu * fn / ft;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            Ft[k] = scale * Ft[k];
            dnew[k] = f64_of(-(Ft[k] + dtc * ucpt[k]) / kt);
        }
    }
}

__global__ void k_cell_count(const double *__restrict__ x, int n_p, CellGeom cg,
                             int *__restrict__ pcell, int *__restrict__ count,
                             float *__restrict__ xb, const int *__restrict__ enable)
{
    if (enable && !*enable)
        return;
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_p)
        return;
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double xa = x[a * n_p + p];
        if (xb)
            xb[a * n_p + p] = (float)xa;
        int i = (int)floor(xa / cg.cs[a]);
        c[a] = min(max(i, 0), cg.nc[a] - 1);
    }
    int key = c[0] + cg.nc[0] * (c[1] + cg.nc[1] * c[2]);
    pcell[p] = key;
    atomicAdd(&count[key], 1);
}

// count[] returns to zero: each particle takes its slot with a decrement
__global__ void k_cell_scatter(int n_p, const int *__restrict__ pcell,
                               const int *__restrict__ start, int *__restrict__ count,
                               int *__restrict__ sorted, const int *__restrict__ enable)
{
    if (enable && !*enable)
        return;
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_p)
        return;
    int key = pcell[p];
    int pos = start[key] + atomicSub(&count[key], 1) - 1;
    sorted[pos] = p;
}

__global__ void k_set_int(int *ptr, int v) { *ptr = v; }

// clears the rebuild flag once the cell list has been rebuilt
__global__ void k_clear(int *flag) { *flag = 0; }

// Grid-wide barrier of a cooperative launch (every block resident):
// arrival counter and generation word, bounded wait. Returns false (and
// latches ERRB_CAPACITY's sibling bit) if the wait ran out.
__device__ bool grid_barrier(unsigned *bar, int *err)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        ok = 1;
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            bar[0] = 0;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long it = 0;
            while (*gen == g) {
                if (++it > (1LL << 26)) {
                    atomicOr(err, ERRB_BARRIER_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

struct RebuildArgs {
    const double *x;
    const float *xf;
    int n_p, ncell;
    CellGeom cg;
    int *pcell, *count, *start, *sorted;
    float *xb;
    float3 halfL, Lf;
    float cut2;
    int *nlist, *ncnt, *nlo;
    int ncap;
    int *flag, *err;
    int *blocksum;  // [gridDim.x]
    unsigned *bar;  // arrival count, generation
};

__device__ void neigh_list_one(const RebuildArgs &a, int p);

// Neighbour (Verlet) list of sphere p: in ascending id order, the spheres
// whose FP32 centre distance is below 2R + skin (+ the FP32 error bound).
// Until the next build no sphere moves more than skin/2, so every pair that
// comes into contact is on the list.
__device__ void neigh_list_one(const RebuildArgs &a, int p)
{
    const int n_p = a.n_p;
    const float *xf = a.xf;
    int *nlist = a.nlist;
    const float xp[3] = {xf[p], xf[n_p + p], xf[2 * n_p + p]};
    const float hl[3] = {a.halfL.x, a.halfL.y, a.halfL.z}, ll[3] = {a.Lf.x, a.Lf.y, a.Lf.z};
    int cc[3];
    cell_coords(__ldcg(a.pcell + p), a.cg, cc);
    int ox[3], oy[3], oz[3];
    const int nx = axis_offsets(a.cg, 0, cc[0], ox);
    const int ny = axis_offsets(a.cg, 1, cc[1], oy);
    const int nz = axis_offsets(a.cg, 2, cc[2], oz);
    int n = 0, lo = 0;
    bool over = false;
    for (int kz = 0; kz < nz; kz++)
        for (int ky = 0; ky < ny; ky++)
            for (int kx = 0; kx < nx; kx++) {
                const int cell = ox[kx] + a.cg.nc[0] * (oy[ky] + a.cg.nc[1] * oz[kz]);
                const int j1 = __ldcg(a.start + cell + 1);
                for (int j = __ldcg(a.start + cell); j < j1; j++) {
                    const int q = __ldcg(a.sorted + j);
                    if (q == p)
                        continue;
                    const float xq[3] = {xf[q], xf[n_p + q], xf[2 * n_p + q]};
                    if (pair_dist2_f32(xp, xq, a.cg.periodic, hl, ll) > a.cut2)
                        continue;
                    if (n == a.ncap) {
                        over = true;
                        continue;
                    }
                    // insert q keeping the list ascending
                    lo += q < p ? 1 : 0;
                    int pos = n++;
                    while (pos > 0 && nlist[(pos - 1) * n_p + p] > q) {
                        nlist[pos * n_p + p] = nlist[(pos - 1) * n_p + p];
                        pos--;
                    }
                    nlist[pos * n_p + p] = q;
                }
            }
    a.ncnt[p] = n;
    a.nlo[p] = lo;
    if (over)
        atomicOr(a.err, ERRB_CAPACITY);
}

// The cell list and the neighbour list in one cooperative launch per
// sub-step. Nothing happens unless the rebuild flag is set (the common
// case costs one launch instead of the nine of the separate kernels).
// Phases: cell of every sphere and counts; exclusive scan of the counts
// (per-block chunks, then the block totals); scatter into cell order;
// neighbour lists; the flag is cleared last.
__global__ void __launch_bounds__(256) k_rebuild(RebuildArgs a)
{
    if (!*a.flag)
        return;
    const int nth = gridDim.x * blockDim.x;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_p = a.n_p;
    for (int p = gtid; p < n_p; p += nth) {
        int c[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const double xd = a.x[d * n_p + p];
            a.xb[d * n_p + p] = (float)xd;
            const int i = (int)floor(xd / a.cg.cs[d]);
            c[d] = min(max(i, 0), a.cg.nc[d] - 1);
        }
        const int key = c[0] + a.cg.nc[0] * (c[1] + a.cg.nc[1] * c[2]);
        a.pcell[p] = key;
        atomicAdd(&a.count[key], 1);
    }
    if (!grid_barrier(a.bar, a.err))
        return;
    // exclusive scan of the counts: block b owns cells [b*chunk, (b+1)*chunk)
    __shared__ int wsum[8];
    __shared__ int btot;
    const int chunk = (a.ncell + gridDim.x - 1) / gridDim.x;
    const int c0 = min(blockIdx.x * chunk, a.ncell), c1 = min(c0 + chunk, a.ncell);
    const int per = (chunk + blockDim.x - 1) / blockDim.x;
    const int t0 = min(c0 + threadIdx.x * per, c1), t1 = min(t0 + per, c1);
    int sum = 0;
    for (int i = t0; i < t1; i++)
        sum += a.count[i];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int v = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += u;
    }
    if (lane == 31)
        wsum[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < 8; w++) {
            const int t = wsum[w];
            wsum[w] = run;
            run += t;
        }
        btot = run;
    }
    __syncthreads();
    int run = v - sum + wsum[wid];
    for (int i = t0; i < t1; i++) {
        a.start[i] = run;
        run += a.count[i];
    }
    if (threadIdx.x == 0)
        a.blocksum[blockIdx.x] = btot;
    if (!grid_barrier(a.bar, a.err))
        return;
    // offsets of the blocks (each block sums the totals before it)
    {
        int off = 0;
        for (int b = threadIdx.x; b < (int)blockIdx.x; b += blockDim.x)
            off += __ldcg(a.blocksum + b);  // written by other blocks in this launch
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            off += __shfl_xor_sync(0xffffffffu, off, o);
        if (lane == 0)
            wsum[wid] = off;
        __syncthreads();
        off = 0;
        for (int w = 0; w < 8; w++)
            off += wsum[w];
        for (int i = t0; i < t1; i++)
            a.start[i] += off;
        if (gtid == 0)
            a.start[a.ncell] = n_p;
    }
    if (!grid_barrier(a.bar, a.err))
        return;
    // scatter into cell order (counts return to zero)
    for (int p = gtid; p < n_p; p += nth) {
        const int key = a.pcell[p];
        a.sorted[__ldcg(a.start + key) + atomicSub(&a.count[key], 1) - 1] = p;
    }
    if (!grid_barrier(a.bar, a.err))
        return;
    for (int i = gtid; i < n_p; i += nth)
        neigh_list_one(a, __ldcg(a.sorted + i));
    if (!grid_barrier(a.bar, a.err))
        return;
    if (gtid == 0)
        *a.flag = 0;
}


__global__ void k_shadow(const double *__restrict__ x, const double *__restrict__ u,
                         const double *__restrict__ om, float *__restrict__ xf,
                         float *__restrict__ uf, float *__restrict__ omf, long long n,
                         const double *__restrict__ Fh, const double *__restrict__ Th,
                         float *__restrict__ Fhf, float *__restrict__ Thf,
                         float *__restrict__ xl)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const float h = (float)x[i];
        xf[i] = h;
        xl[i] = f32_rz(x[i] - f64_of(h));
        uf[i] = (float)u[i];
        omf[i] = (float)om[i];
        if (Fhf) {
            Fhf[i] = (float)Fh[i];
            Thf[i] = (float)Th[i];
        }
    }
}

// ------------------------------------------------------------------ contacts
// d^2 - 4R^2 for the pair (p, q) of the FP32 form, from positions held as
// unevaluated FP32 pairs xf + xl. The separation is formed as a pair dh + dl
// (exact differences by TwoSum; the periodic image is chosen on the FP32
// separation, which for a pair within 2R + skin cannot be near L/2), and the
// cancelling difference d^2 - 4R^2 in pair arithmetic (exact squares by FMA):
// FP64 accuracy without the FP64 pipe. Also returns dh and |d| in FP32. The
// result is the same, bit for bit, from either sphere of the pair.
template <typename T>
__device__ __forceinline__ float pair_overlap2(const DemArgs<T> &a, int q, const float xpf[3],
                                               const float xpl[3], float dh[3], float &dist_f)
{
    const int n_p = a.n_p;
    float dl[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        float e1, e2 = 0.f;
        float s1 = two_sum(a.xf[k * n_p + q], -xpf[k], e1);
        if (a.dp.periodic[k]) {
            if (s1 > a.halfL[k])
                s1 = two_sum(s1, -a.Lf[k], e2);
            else if (s1 < -a.halfL[k])
                s1 = two_sum(s1, a.Lf[k], e2);
        }
        const float lo = (e1 + e2) + (a.xl[k * n_p + q] - xpl[k]);
        dh[k] = s1 + lo;
        dl[k] = lo - (dh[k] - s1);
    }
    float sq[3], er[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        sq[k] = dh[k] * dh[k];
        er[k] = __fmaf_rn(dh[k], dh[k], -sq[k]);
    }
    float f1, f2, f3;
    float t = two_sum(sq[0], sq[1], f1);
    t = two_sum(t, sq[2], f2);
    dist_f = sqrtf(t);
    t = two_sum(t, -a.four_R2h, f3);
    const float cross = (dh[0] * dl[0] + dh[1] * dl[1]) + dh[2] * dl[2];
    const float low = (((f1 + f2) + f3) + ((er[0] + er[1]) + er[2])) +
                      ((cross + cross) - a.four_R2l);
    return t + low;
}

template <typename T, bool MIXED>
__global__ void __launch_bounds__(kDemThreads, MIXED ? kDemMinBlocksContacts : 6) k_dem_contacts(DemArgs<T> a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_p)
        return;
    const int n_p = a.n_p;
    const int p = i;
    const DemParams &dp = a.dp;
    const double R = dp.R;
    double xp[3];
    float xpf[3], xpl[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        // the FP32 form needs the FP64 position only for the rare exact test
        xp[k] = MIXED ? 0.0 : a.x[k * n_p + p];
        xpf[k] = a.xf[k * n_p + p];
        xpl[k] = MIXED ? a.xl[k * n_p + p] : 0.f;
    }
    // the partner ids of the old history, loaded together (they do not
    // depend on the contact search) into this thread's column of shared
    // memory, where the matching below walks them
    __shared__ int s_pid[S][kDemThreads];
    const int old_cnt = a.ho.cnt[p];
#pragma unroll
    for (int s2 = 0; s2 < S; s2++)
        if (s2 < old_cnt)
            s_pid[s2][threadIdx.x] = a.ho.pid[s2 * n_p + p];

    // the contacts p owns (higher partner ids, ascending); in the FP32 form
    // a pair whose FP32 distance is clearly below 2R needs no FP64 test
    // (pairs within the FP32 error band of 2R are decided exactly, as in the
    // FP64 form). Candidates: the neighbour list, already in ascending id
    // order. A sphere's contacts with lower ids are found by their owners;
    // the update checks the total against the 12 slots.
    int cand[S];
    int nc = 0;
    bool overflow = false;
    {
        // neighbours in batches of four: their ids, then their positions, are
        // loaded together so that the gathers overlap
        // the list is ascending: its higher ids start after the nlo lower ones
        const int nn = a.ncnt[p];
        for (int j0 = a.nlo[p]; j0 < nn && !overflow; j0 += 4) {
            int qq[4];
            float xq4[4][3];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                // a lower id evaluates its pair with p: only higher ids are
                // tested here (-1 also past the end of the list)
                const int q = j0 + u < nn ? a.nlist[(j0 + u) * n_p + p] : -1;
                qq[u] = q > p ? q : -1;
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int k = 0; k < 3; k++)
                    xq4[u][k] = qq[u] >= 0 ? a.xf[k * n_p + qq[u]] : 0.f;
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int q = qq[u];
                if (overflow)
                    break;
                if (q < 0)
                    continue;
                const float d2f = pair_dist2_f32(xpf, xq4[u], dp.periodic, a.halfL, a.Lf);
                if (d2f > a.cut2_f32)
                    continue;
                bool exact = !(MIXED && d2f < a.in2_f32);
                if (MIXED && exact) {
                    // within the FP32 band around 2R: the pair arithmetic
                    // decides unless d^2 - 4R^2 is within its own error bound
                    float dh[3], df;
                    const float D = pair_overlap2(a, q, xpf, xpl, dh, df);
                    if (D > a.band_D)
                        continue;
                    exact = !(D < -a.band_D);
                }
                if (exact) {
                    // exact decision, in canonical orientation (Eq. A.3)
                    double xq[3], dx[3];
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        xq[k] = a.x[k * n_p + q];
                        if (MIXED)
                            xp[k] = a.x[k * n_p + p];
                    }
                    const double dist =
                        p < q ? pair_vector(dp, xp, xq, dx) : pair_vector(dp, xq, xp, dx);
                    if (!(dist < R + R))
                        continue;
                }
                if (nc == S) {  // the 12 lowest ids are kept, the rest flagged
                    overflow = true;
                    break;
                }
                cand[nc++] = q;  // the owned contacts, ascending
            }
        }
    }
    if (overflow)
        atomicOr(a.err, ERRB_CONTACT_OVERFLOW);
    a.ccnt[p] = nc;

    // pair forces where p has the lower id, history matched against M_temp
    int so = 0, sn = 0;
    for (int s = 0; s < nc; s++) {
        const int q = cand[s];
        if (q < p)
            continue;
        double dx[3];
        double dist = 0.0, delta_n = 0.0;
        float dist_f = 0.f, delta_f = 0.f;
        float dh[3];
        if (MIXED) {
            const float D = pair_overlap2(a, q, xpf, xpl, dh, dist_f);
            delta_f = D / (dist_f + a.two_Rf);   // Eq. A.3
        } else {
            double xq[3];
#pragma unroll
            for (int k = 0; k < 3; k++)
                xq[k] = a.x[k * n_p + q];
            dist = pair_vector(dp, xp, xq, dx);
            delta_n = dist - R - R;                       // Eq. A.3
        }
        while (so < old_cnt && s_pid[so][threadIdx.x] < q)
            so++;
        const bool existing = so < old_cnt && s_pid[so][threadIdx.x] == q;
        double dprev[3] = {0.0, 0.0, 0.0};
        if (existing) {                                   // existing event (Sec. 3.4)
#pragma unroll
            for (int k = 0; k < 3; k++)
                dprev[k] = a.ho.dlt[(so * 3 + k) * n_p + p];
        }
        double uin;
        T F[3], Tq[3];
        double dnew[3];
        if (MIXED) {
            const float inv = 1.0f / dist_f;
            float n[3], ul[3], uh[3], ol[3], oh[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                n[k] = dh[k] * inv;                       // Eq. A.1
                ul[k] = a.uf[k * n_p + p];
                uh[k] = a.uf[k * n_p + q];
                ol[k] = a.omf[k * n_p + p];
                oh[k] = a.omf[k * n_p + q];
            }
            const float Rf = a.Rf;
            float cl[3], ch[3], ucp[3];
            cross3(ol, n, cl);
            cross3(oh, n, ch);
#pragma unroll
            for (int k = 0; k < 3; k++)                   // Eq. A.5
                ucp[k] = ((ul[k] - uh[k]) + Rf * cl[k]) + Rf * ch[k];
            uin = existing ? a.ho.uin[so * n_p + p] : f64_of(dot3(ucp, n));
            float Fn[3], Ft[3];
            contact_force_mixed(n, delta_f, ucp, dprev, a.kn_pp, a.dn_pp, a.kt_pp, a.dt_pp, a.mu,
                                a.dtp_f, a.dp.clip_n, a.dp.model,
                                fmaxf(fabsf((float)uin), (float)a.dp.u_min), Fn, Ft, dnew);
            float tq[3];
            cross3(n, Ft, tq);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                F[k] = (T)(Fn[k] + Ft[k]);
                Tq[k] = (T)(Rf * tq[k]);
            }
        } else {
            double n[3];
#pragma unroll
            for (int k = 0; k < 3; k++)
                n[k] = dx[k] / dist;                      // Eq. A.1
            double ul[3], uh[3], ol[3], oh[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                ul[k] = a.u[k * n_p + p];
                uh[k] = a.u[k * n_p + q];
                ol[k] = a.om[k * n_p + p];
                oh[k] = a.om[k * n_p + q];
            }
            double cl[3], ch[3], ucp[3];
            cross3(ol, n, cl);
            cross3(oh, n, ch);
#pragma unroll
            for (int k = 0; k < 3; k++)                   // Eq. A.5
                ucp[k] = ((ul[k] - uh[k]) + R * cl[k]) + R * ch[k];
            uin = existing ? a.ho.uin[so * n_p + p] : dot3(ucp, n);
            double Fn[3], Ft[3];
            contact_force64(n, delta_n, ucp, dprev, dp.kn_pp, dp.dn_pp, dp.kt_pp, dp.dt_pp,
                            dp.mu, a.dt_p, dp.clip_n, dp.model, fmax(fabs(uin), dp.u_min), Fn,
                            Ft, dnew);
            double tq[3];
            cross3(n, Ft, tq);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                F[k] = (T)(Fn[k] + Ft[k]);
                Tq[k] = (T)(R * tq[k]);
            }
        }
        a.hn.pid[sn * n_p + p] = q;
        a.hn.uin[sn * n_p + p] = uin;
        {
            // the higher id finds the pair through its incoming list (p, slot)
            const int k = atomicAdd(&a.inc_cnt[q], 1);
            if (k < S)
                a.inc[k * n_p + q] = p * 16 + sn;
        }
#pragma unroll
        for (int k = 0; k < 3; k++)
            a.hn.dlt[(sn * 3 + k) * n_p + p] = dnew[k];
        store_pair(pair_entry(a.pairFT, sn, p, n_p), F, Tq);
        sn++;
    }
    a.hn.cnt[p] = sn;
}

// ------------------------------------------------------------------ update
// small-gap Stokes amplification of the normal resistance (eps = gap / R):
// two equal spheres (Jeffrey 1982), a sphere and a wall (Cox & Brenner 1967)
__device__ __forceinline__ double lub_lambda(bool wall, double eps)
{
    const double l = log(eps);
    return wall ? 1.0 / eps - 0.2 * l - eps * l / 21.0 + 0.9713
                : 0.5 / eps - 0.45 * l - 3.0 * eps * l / 56.0 + 1.346;
}

// Lubrication (Sec. 2.1, two-parameter model): per sphere, the normal force
// from every neighbour whose gap lies in [0, eps_d R) and from the walls,
// in FP64 from the FP64 state. A pair is evaluated in canonical orientation
// (lower id to higher) and its force negated for the higher id, so the two
// spheres receive exactly opposite forces without sharing any storage.
__global__ void __launch_bounds__(256) k_dem_lub(const double *__restrict__ x,
                                                 const double *__restrict__ u,
                                                 const int *__restrict__ nlist,
                                                 const int *__restrict__ ncnt, int n_p,
                                                 DemParams dp, double *__restrict__ flub)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_p)
        return;
    const double R = dp.R;
    double F[3] = {0.0, 0.0, 0.0};
    const int nn = ncnt[p];
    for (int j = 0; j < nn; j++) {
        const int q = nlist[j * n_p + p];
        const int lo = min(p, q), hi = max(p, q);
        double dx[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            double s = __dsub_rn(x[k * n_p + hi], x[k * n_p + lo]);
            if (dp.periodic[k]) {
                const double L = dp.L[k];
                if (s > 0.5 * L)
                    s = __dsub_rn(s, L);
                else if (s < -0.5 * L)
                    s = __dadd_rn(s, L);
            }
            dx[k] = s;
        }
        const double d = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx[0], dx[0]), __dmul_rn(dx[1], dx[1])),
                                         __dmul_rn(dx[2], dx[2])));
        const double gap = __dsub_rn(__dsub_rn(d, R), R);
        if (!(gap >= 0.0 && gap < dp.eps_d_pp * R))
            continue;
        double eps = gap / R;
        if (eps < dp.eps_s)
            eps = dp.eps_s;
        const double f = dp.lub_pp * (lub_lambda(false, eps) - dp.lam_d_pp);
        double nv[3], un = 0.0;
#pragma unroll
        for (int k = 0; k < 3; k++)
            nv[k] = dx[k] / d;
#pragma unroll
        for (int k = 0; k < 3; k++)
            un = __dadd_rn(un, __dmul_rn(__dsub_rn(u[k * n_p + lo], u[k * n_p + hi]), nv[k]));
        const double fu = __dmul_rn(f, un);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const double fk = -__dmul_rn(fu, nv[k]);
            F[k] = p == lo ? __dadd_rn(F[k], fk) : __dsub_rn(F[k], fk);
        }
    }
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
        if (dp.periodic[ax])
            continue;
        for (int side = 0; side < 2; side++) {
            const double xa = x[ax * n_p + p];
            const double gap = __dsub_rn(side == 0 ? xa : __dsub_rn(dp.L[ax], xa), R);
            if (!(gap >= 0.0 && gap < dp.eps_d_pw * R))
                continue;
            double eps = gap / R;
            if (eps < dp.eps_s)
                eps = dp.eps_s;
            const double f = dp.lub_pw * (lub_lambda(true, eps) - dp.lam_d_pw);
            const double nw = side == 0 ? -1.0 : 1.0;
            const double un = __dmul_rn(u[ax * n_p + p], nw);
            F[ax] = __dadd_rn(F[ax], -__dmul_rn(__dmul_rn(f, un), nw));
        }
    }
#pragma unroll
    for (int k = 0; k < 3; k++)
        flub[k * n_p + p] = F[k];
}

template <typename T, bool MIXED>
__global__ void __launch_bounds__(kDemThreads, MIXED ? kDemMinBlocksUpdate : 6) k_dem_update(DemArgs<T> a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_p)
        return;
    const int n_p = a.n_p;
    const int p = i;
    const DemParams &dp = a.dp;
    const double R = dp.R;
    double xp[3], upv[3], opv[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        xp[k] = a.x[k * n_p + p];
        upv[k] = a.u[k * n_p + p];
        opv[k] = a.om[k * n_p + p];
    }
    // pair forces in ascending partner order (Eq. 9-10): a pair evaluated by
    // p itself, or by the lower-id partner and negated (the torque R n x F_t
    // is the same for both spheres)
    T Fc[3] = {T(0), T(0), T(0)}, Tc[3] = {T(0), T(0), T(0)};
    {
        // pairs owned by lower ids: entries (partner * 16 + slot), loaded
        // together into this thread's column of shared memory, then sorted
        // ascending there so the sum runs in ascending partner order
        __shared__ int s_in[S][kDemThreads];
        const int tx = threadIdx.x;
        const int n_inc = a.inc_cnt[p];
        const int nin = min(n_inc, S);
        int e_in[S];
#pragma unroll
        for (int s = 0; s < S; s++)
            if (s < nin)
                e_in[s] = a.inc[s * n_p + p];
#pragma unroll
        for (int s = 0; s < S; s++) {
            if (s >= nin)
                break;
            const int e = e_in[s];
            int pos = s;
            while (pos > 0 && s_in[pos - 1][tx] > e) {
                s_in[pos][tx] = s_in[pos - 1][tx];
                pos--;
            }
            s_in[pos][tx] = e;
        }
        a.inc_cnt[p] = 0;
        // two entries' gathers in flight at a time (four spill), summed in list
        // order
        constexpr int kB = 2;
        static_assert(S % kB == 0, "batches cover the slots");
        for (int s0 = 0; s0 < nin; s0 += kB) {
            T v[kB][6];
#pragma unroll
            for (int b = 0; b < kB; b++)
                if (s0 + b < nin) {
                    const int e = s_in[s0 + b][tx];
                    load_pair(pair_entry<const T>(a.pairFT, e & 15, e >> 4, n_p), v[b]);
                }
#pragma unroll
            for (int b = 0; b < kB; b++)
                if (s0 + b < nin) {
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        Fc[k] -= v[b][k];
                        Tc[k] += v[b][3 + k];
                    }
                }
        }
        // then the pairs p owns (higher ids, ascending)
        const int own = a.hn.cnt[p];
        if (n_inc + own > S)  // more than 12 contacts in all
            atomicOr(a.err, ERRB_CONTACT_OVERFLOW);
        for (int s0 = 0; s0 < own; s0 += kB) {
            T v[kB][6];
#pragma unroll
            for (int b = 0; b < kB; b++)
                if (s0 + b < own)
                    load_pair(pair_entry<const T>(a.pairFT, s0 + b, p, n_p), v[b]);
#pragma unroll
            for (int b = 0; b < kB; b++)
                if (s0 + b < own) {
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        Fc[k] += v[b][k];
                        Tc[k] += v[b][3 + k];
                    }
                }
        }
    }

    // walls on bounded axes, low side then high side (Eq. A.2, A.4, A.6)
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
        for (int side = 0; side < 2; side++) {
            const int wslot = 2 * ax + side;
            const int ws = wslot * n_p + p;
            if (dp.periodic[ax]) {
                a.hn.wact[ws] = 0;
                continue;
            }
            // FP32 form: spheres clearly away from the wall skip the FP64 test
            const float xpf = a.xf[ax * n_p + p];
            if (MIXED && (side == 0 ? xpf : a.Lf[ax] - xpf) > a.wall_f32) {
                a.hn.wact[ws] = 0;
                continue;
            }
            const double dist = side == 0 ? xp[ax] : dp.L[ax] - xp[ax];
            const double delta_n = dist - R;
            if (!(delta_n < 0.0)) {
                a.hn.wact[ws] = 0;
                continue;
            }
            const bool existing = a.ho.wact[ws];
            double dprev[3] = {0.0, 0.0, 0.0};
            if (existing) {
#pragma unroll
                for (int k = 0; k < 3; k++)
                    dprev[k] = a.ho.wdlt[(wslot * 3 + k) * n_p + p];
            }
            double uin, dnew[3];
            if (MIXED) {
                float n[3] = {0.f, 0.f, 0.f};
                n[ax] = side == 0 ? -1.f : 1.f;
                float o[3], uu[3], cw[3], ucp[3];
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    o[k] = a.omf[k * n_p + p];
                    uu[k] = a.uf[k * n_p + p];
                }
                cross3(o, n, cw);
                const float Rf = a.Rf;
#pragma unroll
                for (int k = 0; k < 3; k++)
                    ucp[k] = uu[k] + Rf * cw[k];
                uin = existing ? a.ho.wuin[ws] : f64_of(dot3(ucp, n));
                float Fn[3], Ft[3];
                contact_force_mixed(n, f32_rz(delta_n), ucp, dprev, a.kn_pw, a.dn_pw, a.kt_pw,
                                    a.dt_pw, a.mu, a.dtp_f, a.dp.clip_n, a.dp.model,
                                    fmaxf(fabsf((float)uin), (float)a.dp.u_min), Fn, Ft, dnew);
                float tq[3];
                cross3(n, Ft, tq);
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    Fc[k] += (T)(Fn[k] + Ft[k]);
                    Tc[k] += (T)(Rf * tq[k]);
                }
            } else {
                double n[3] = {0.0, 0.0, 0.0};
                n[ax] = side == 0 ? -1.0 : 1.0;
                double cw[3], ucp[3];
                cross3(opv, n, cw);
#pragma unroll
                for (int k = 0; k < 3; k++)
                    ucp[k] = upv[k] + R * cw[k];
                uin = existing ? a.ho.wuin[ws] : dot3(ucp, n);
                double Fn[3], Ft[3];
                contact_force64(n, delta_n, ucp, dprev, dp.kn_pw, dp.dn_pw, dp.kt_pw, dp.dt_pw,
                                dp.mu, a.dt_p, dp.clip_n, dp.model, fmax(fabs(uin), dp.u_min),
                                Fn, Ft, dnew);
                double tq[3];
                cross3(n, Ft, tq);
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    Fc[k] += (T)(Fn[k] + Ft[k]);
                    Tc[k] += (T)(R * tq[k]);
                }
            }
            a.hn.wact[ws] = 1;
            a.hn.wuin[ws] = uin;
#pragma unroll
            for (int k = 0; k < 3; k++)
                a.hn.wdlt[(wslot * 3 + k) * n_p + p] = dnew[k];
        }
    }

    if (a.flub) {
#pragma unroll
        for (int k = 0; k < 3; k++)
            Fc[k] += (T)a.flub[k * n_p + p];
    }
    // Newton-Euler, semi-implicit Euler. The update multiplies by the
    // precomputed inverse inertia and fuses multiply-adds: within a rounding
    // or two of the plain formula, with a third of its FP64 operations.
    // In the FP32 form the accelerations are FP32 (like the forces) and
    // only their increments enter the FP64 velocities and positions.
    bool finite = true;
    float xnf[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        double un, on;
        if (MIXED) {
            const float accf = fmaf(a.Fhf[k * n_p + p] + (float)Fc[k], a.inv_m_f, a.g_f[k]);
            const float angf = (a.Thf[k * n_p + p] + (float)Tc[k]) * a.inv_J_f;
            un = upv[k] + f64_of(a.dt_f * accf);
            on = opv[k] + f64_of(a.dt_f * angf);
            if (a.last) {
                a.Fcf[k * n_p + p] = (float)Fc[k];
                a.Tcf[k * n_p + p] = (float)Tc[k];
            }
        } else {
            const double fc = (double)Fc[k], tc = (double)Tc[k];
            const double acc = __fma_rn(a.Fh[k * n_p + p] + fc, a.inv_m, dp.g[k]);
            un = __fma_rn(a.dt_p, acc, upv[k]);
            const double ang = (a.Th[k * n_p + p] + tc) * a.inv_J;
            on = __fma_rn(a.dt_p, ang, opv[k]);
            if (a.last) {
                a.Fc[k * n_p + p] = fc;
                a.Tc[k * n_p + p] = tc;
            }
        }
        double xn = __fma_rn(a.dt_p, un, xp[k]);
        float xf = MIXED ? f32_rz(xn) : (float)xn;
        // the exact FP64 wrap only when the FP32 value is at or past a face
        if (dp.periodic[k] && !(xf > 0.f && xf < a.Lf[k])) {
            const double L = dp.L[k];
            if (xn < 0.0) {
                xn += L;
                if (xn >= L)
                    xn = 0.0;
            } else if (xn >= L) {
                xn -= L;
            }
            xf = MIXED ? f32_rz(xn) : (float)xn;
        }
        finite = finite && finite_bits(xn) && finite_bits(un) && finite_bits(on);
        a.un[k * n_p + p] = un;
        a.omn[k * n_p + p] = on;
        a.xn[k * n_p + p] = xn;
        a.xfn[k * n_p + p] = xf;
        if (MIXED)
            a.xln[k * n_p + p] = f32_rz(xn - f64_of(xf));
        a.ufn[k * n_p + p] = MIXED ? f32_rz(un) : (float)un;
        a.omfn[k * n_p + p] = MIXED ? f32_rz(on) : (float)on;
        xnf[k] = xf;
    }
    if (!finite)
        atomicOr(a.err, ERRB_NONFINITE);
    // displacement since the last cell-list build
    float xbp[3];
#pragma unroll
    for (int k = 0; k < 3; k++)
        xbp[k] = a.xb[k * n_p + p];
    if (pair_dist2_f32(xbp, xnf, dp.periodic, a.halfL, a.Lf) > a.move2_f32 || !finite)
        atomicOr(a.rebuild, 1);
}

__global__ void k_pairs(const double *__restrict__ x, int n_p, const int *__restrict__ sorted,
                        const int *__restrict__ start, const int *__restrict__ pcell,
                        CellGeom cg, DemParams dp, double cutoff, int *__restrict__ out,
                        long long max_pairs, unsigned long long *__restrict__ n_out)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_p)
        return;
    double xp[3];
#pragma unroll
    for (int k = 0; k < 3; k++)
        xp[k] = x[k * n_p + p];
    int cc[3];
    cell_coords(pcell[p], cg, cc);
    int ox[3], oy[3], oz[3];
    int nx = axis_offsets(cg, 0, cc[0], ox);
    int ny = axis_offsets(cg, 1, cc[1], oy);
    int nz = axis_offsets(cg, 2, cc[2], oz);
    for (int kz = 0; kz < nz; kz++)
        for (int ky = 0; ky < ny; ky++)
            for (int kx = 0; kx < nx; kx++) {
                int cell = ox[kx] + cg.nc[0] * (oy[ky] + cg.nc[1] * oz[kz]);
                int j1 = start[cell + 1];
                for (int j = start[cell]; j < j1; j++) {
                    int q = sorted[j];
                    if (q <= p)
                        continue;
                    double xq[3], dx[3];
#pragma unroll
                    for (int k = 0; k < 3; k++)
                        xq[k] = x[k * n_p + q];
                    double dist = pair_vector(dp, xp, xq, dx);
                    if (dist < cutoff) {
                        unsigned long long slot = atomicAdd(n_out, 1ULL);
                        if ((long long)slot < max_pairs) {
                            out[2 * slot] = p;
                            out[2 * slot + 1] = q;
                        }
                    }
                }
            }
}

template <typename T, bool MIXED>
void substep_t(Ctx &c, double dt_p, bool last, cudaStream_t s)
{
    const int cur = c.cur, nxt = 1 - c.cur;
    const int ho = c.hcur, hn = 1 - c.hcur;
    phase_begin(c, PRS_PHASE_DEM_CELLS);
    dem_rebuild(c, s);
    phase_end(c);
    DemArgs<T> a;
    a.x = c.x[cur];
    a.u = c.u[cur];
    a.om = c.om[cur];
    a.xf = c.xf[cur];
    a.xl = c.xl[cur];
    a.xln = c.xl[nxt];
    a.uf = c.uf[cur];
    a.omf = c.omf[cur];
    a.xn = c.x[nxt];
    a.un = c.u[nxt];
    a.omn = c.om[nxt];
    a.xfn = c.xf[nxt];
    a.ufn = c.uf[nxt];
    a.omfn = c.omf[nxt];
    a.Fh = c.Fh;
    a.Th = c.Th;
    a.Fc = c.Fc;
    a.Tc = c.Tc;
    a.ho = HistPtrs{c.hcnt[ho], c.hpid[ho], c.huin[ho], c.hdlt[ho], c.wact[ho], c.wuin[ho],
                    c.wdlt[ho]};
    a.hn = HistPtrs{c.hcnt[hn], c.hpid[hn], c.huin[hn], c.hdlt[hn], c.wact[hn], c.wuin[hn],
                    c.wdlt[hn]};
    a.pairFT = (T *)c.pairFT;
    a.ccnt = c.ccnt;
    a.clist = c.clist;
    a.sorted = c.cell_sorted;
    a.start = c.cell_start;
    a.pcell = c.pcell;
    a.cg = c.cg;
    a.dp = c.dp;
    a.dt_p = dt_p;
    a.last = last ? 1 : 0;
    a.n_p = c.n_p;
    a.err = c.d_err;
    double Lmax = 0.0;
    for (int k = 0; k < 3; k++) {
        a.halfL[k] = (float)(0.5 * c.dp.L[k]);
        a.Lf[k] = (float)c.dp.L[k];
        Lmax = fmax(Lmax, c.dp.L[k]);
    }
    // rounding of x to FP32 and of the FP32 differences: < 8 ulp(L) per axis
    const double eps = 16.0 * Lmax * 5.96e-8 + 1e-6;
    const double cut = 2.0 * c.dp.R + eps, in = 2.0 * c.dp.R - eps;
    a.cut2_f32 = (float)(cut * cut * (1.0 + 1e-6));
    a.in2_f32 = (float)(in > 0.0 ? in * in * (1.0 - 1e-6) : 0.0);
    const double mv = 0.5 * c.skin - eps;
    a.move2_f32 = (float)(mv > 0.0 ? mv * mv : 0.0);
    a.wall_f32 = (float)(c.dp.R + eps);
    a.xb = c.xb;
    a.rebuild = c.d_rebuild;
    a.inv_m = 1.0 / c.dp.m;
    a.inv_J = 1.0 / c.dp.J;
    a.Fhf = c.Fhf;
    a.Thf = c.Thf;
    a.Fcf = c.Fcf;
    a.Tcf = c.Tcf;
    a.inv_m_f = (float)a.inv_m;
    a.inv_J_f = (float)a.inv_J;
    a.dt_f = (float)dt_p;
    for (int k = 0; k < 3; k++)
        a.g_f[k] = (float)c.dp.g[k];
    a.four_R2 = 4.0 * c.dp.R * c.dp.R;
    a.four_R2h = (float)a.four_R2;
    a.four_R2l = (float)(a.four_R2 - (double)a.four_R2h);
    // positions as FP32 pairs carry < 2^-46 Lmax, the separation < 2^-44
    // Lmax, d^2 - 4R^2 < 6 (2R + skin) 2^-44 Lmax; a factor 16 of margin
    a.band_D = (float)(16.0 * 6.0 * (2.0 * c.dp.R + c.skin) * std::ldexp(Lmax, -44));
    a.two_Rf = (float)(2.0 * c.dp.R);
    a.Rf = (float)c.dp.R;
    a.kn_pp = (float)c.dp.kn_pp;
    a.dn_pp = (float)c.dp.dn_pp;
    a.kt_pp = (float)c.dp.kt_pp;
    a.dt_pp = (float)c.dp.dt_pp;
    a.kn_pw = (float)c.dp.kn_pw;
    a.dn_pw = (float)c.dp.dn_pw;
    a.kt_pw = (float)c.dp.kt_pw;
    a.dt_pw = (float)c.dp.dt_pw;
    a.mu = (float)c.dp.mu;
    a.dtp_f = (float)dt_p;
    a.nlist = c.nlist;
    a.ncnt = c.ncnt;
    a.nlo = c.nlo;
    a.inc = c.clist;
    a.inc_cnt = c.inc_cnt;
    a.flub = c.dp.mu_f > 0.0 ? c.flub : nullptr;
    const int blocks = (c.n_p + kDemThreads - 1) / kDemThreads;
    phase_begin(c, PRS_PHASE_DEM_CONTACTS);
    k_dem_contacts<T, MIXED><<<blocks, kDemThreads, 0, s>>>(a);
    if (a.flub) {
        k_dem_lub<<<(c.n_p + 255) / 256, 256, 0, s>>>(c.x[c.cur], c.u[c.cur], c.nlist, c.ncnt,
                                                       c.n_p, c.dp, c.flub);
        c.n_launch += 1;
    }
    phase_end(c);
    phase_begin(c, PRS_PHASE_DEM_UPDATE);
    k_dem_update<T, MIXED><<<blocks, kDemThreads, 0, s>>>(a);
    phase_end(c);
    c.n_launch += 2;
}

}  // namespace

__global__ void k_f2d(const float *__restrict__ a, double *__restrict__ b, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        b[i] = (double)a[i];
}

void dem_forces_f2d(const Ctx &c, const float *src, double *dst, cudaStream_t s)
{
    const long long n = 3LL * c.n_p;
    k_f2d<<<(int)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
    c.n_launch += 1;
}

void dem_shadow(Ctx &c, cudaStream_t s)
{
    const long long n = 3LL * c.n_p;
    k_shadow<<<(int)((n + 255) / 256), 256, 0, s>>>(c.x[c.cur], c.u[c.cur], c.om[c.cur],
                                                    c.xf[c.cur], c.uf[c.cur], c.omf[c.cur], n,
                                                    c.Fh, c.Th, c.Fhf, c.Thf, c.xl[c.cur]);
    c.n_launch += 1;
}

CellGeom make_cell_geom(const DemParams &dp, double cutoff)
{
    CellGeom cg{};
    for (int a = 0; a < 3; a++) {
        int nc = (int)floor(dp.L[a] / cutoff);
        if (nc < 1)
            nc = 1;
        cg.nc[a] = nc;
        cg.cs[a] = dp.L[a] / nc;
        cg.periodic[a] = dp.periodic[a];
        cg.L[a] = dp.L[a];
    }
    return cg;
}

void dem_rebuild(const Ctx &c, cudaStream_t s)
{
    const CellGeom &cg = c.cg;
    RebuildArgs ra;
    ra.x = c.x[c.cur];
    ra.xf = c.xf[c.cur];
    ra.n_p = c.n_p;
    ra.ncell = cg.nc[0] * cg.nc[1] * cg.nc[2];
    ra.cg = cg;
    ra.pcell = c.pcell;
    ra.count = c.cell_count;
    ra.start = c.cell_start;
    ra.sorted = c.cell_sorted;
    ra.xb = c.xb;
    double Lmax = 0.0;
    for (int d = 0; d < 3; d++)
        Lmax = fmax(Lmax, cg.L[d]);
    const double eps = 16.0 * Lmax * 5.96e-8 + 1e-6;
    const double lc = 2.0 * c.R + c.skin + c.lub_reach + eps;
    ra.halfL = make_float3((float)(0.5 * cg.L[0]), (float)(0.5 * cg.L[1]),
                           (float)(0.5 * cg.L[2]));
    ra.Lf = make_float3((float)cg.L[0], (float)cg.L[1], (float)cg.L[2]);
    ra.cut2 = (float)(lc * lc * (1.0 + 1e-6));
    ra.nlist = c.nlist;
    ra.ncnt = c.ncnt;
    ra.nlo = c.nlo;
    ra.ncap = c.ncap;
    ra.flag = c.d_rebuild;
    ra.err = c.d_err;
    ra.blocksum = c.coop_blocksum;
    ra.bar = c.coop_bar;
    void *args[] = {&ra};
    cudaLaunchCooperativeKernel((void *)k_rebuild, dim3(c.coop_grid), dim3(256), args, 0, s);
    c.n_launch += 1;
}

int dem_rebuild_grid()
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rebuild, 256, 0);
    return std::max(1, std::min(per, 4)) * std::max(sms, 1);
}

void dem_cells_build(const Ctx &c, const CellGeom &cg, const double *x, cudaStream_t s,
                     const int *enable)
{
    const int n_p = c.n_p;
    const int ncell = cg.nc[0] * cg.nc[1] * cg.nc[2];
    const int nb = (n_p + 255) / 256;
    k_cell_count<<<nb, 256, 0, s>>>(x, n_p, cg, c.pcell, c.cell_count, enable ? c.xb : nullptr,
                                    enable);
    int k = exclusive_scan(c.cell_count, c.cell_start, ncell, c.cell_scan_tmp, s, enable);
    k_set_int<<<1, 1, 0, s>>>(c.cell_start + ncell, n_p);
    k_cell_scatter<<<nb, 256, 0, s>>>(n_p, c.pcell, c.cell_start, c.cell_count, c.cell_sorted,
                                      enable);
    c.n_launch += 3 + k;
    if (enable) {
        k_clear<<<1, 1, 0, s>>>(c.d_rebuild);
        c.n_launch += 1;
    }
}

void dem_substep(Ctx &c, double dt_p, bool last, cudaStream_t s)
{
    if (c.precision == PRS_FP64)
        substep_t<double, false>(c, dt_p, last, s);
    else
        substep_t<float, true>(c, dt_p, last, s);
}

void dem_pairs(const Ctx &c, const CellGeom &cg, double cutoff, int *d_pairs,
               long long max_pairs, cudaStream_t s)
{
    dem_cells_build(c, cg, c.x[c.cur], s);
    cudaMemsetAsync(c.d_pairs_n, 0, sizeof(long long), s);
    DemParams geo = c.dp;
    for (int a = 0; a < 3; a++) {
        geo.L[a] = cg.L[a];
        geo.periodic[a] = cg.periodic[a];
    }
    k_pairs<<<(c.n_p + 127) / 128, 128, 0, s>>>(
        c.x[c.cur], c.n_p, c.cell_sorted, c.cell_start, c.pcell, cg, geo, cutoff, d_pairs,
        max_pairs, reinterpret_cast<unsigned long long *>(c.d_pairs_n));
    c.n_launch += 1;
}

}  // namespace prs
