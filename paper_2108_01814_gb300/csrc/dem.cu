// Soft-sphere DEM on the GPU: cell-list contact search, 12-slot contact
// history (Sec. 3.4), linear spring-dashpot forces with Coulomb cap
// (Sec. 2.1, Eq. 9-10, Appendix A.1-A.11) and the semi-implicit
// Newton-Euler update of Eq. 7-8 in rigid-body form.
//
// Compiled with --fmad=false: every FP64 expression below is evaluated as
// written (no fused multiply-add), so that contact decisions and contact
// forces are reproducible bit for bit from a given state.
#include <cstdio>

#include "prs_internal.cuh"

namespace prs {
namespace {

constexpr int kDemThreads = 128;

struct HistPtrs {
    int *cnt;
    int *pid;
    double *uin;
    double *dlt;
    unsigned char *wact;
    double *wuin;
    double *wdlt;
};

struct DemArgs {
    const double *x, *u, *om;
    const float *xf;   // FP32 copy of x, for a conservative distance pre-filter
    double *xn, *un, *omn;
    float *xfn;
    const double *Fh, *Th;
    double *Fc, *Tc;
    HistPtrs ho, hn;
    const int *sorted, *start, *pcell;
    CellGeom cg;
    DemParams dp;
    double dt_p;
    float cut2_f32;    // (2R + eps)^2: pairs beyond it in FP32 cannot touch
    float halfL[3], Lf[3];
    double inv_m, inv_J;
    const float *xb;   // positions at the last cell-list build
    float move2_f32;   // (skin/2 - eps)^2: moving further forces a rebuild
    int *rebuild;
    int n_p;
    int *err;
};

// FP32 pre-filter: squared distance with minimum image, in FP32. Its error
// is bounded by a few ulp of the domain size; the caller compares it with a
// cutoff enlarged by that bound, so no pair the exact FP64 test would keep
// is ever rejected.
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

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ double dot3(const double a[3], const double b[3])
{
    return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

// Tangential displacement (A.9-A.11) and spring-dashpot force of one
// contact, seen from the particle with contact velocity ucp.
__device__ __forceinline__ void contact_force(const double n[3], double delta_n,
                                              const double ucp[3], const double dprev[3],
                                              double kn, double dn, double kt, double dtc,
                                              double mu, double dt_p, double Fn[3],
                                              double Ft[3], double dnew[3])
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

__global__ void k_shadow(const double *__restrict__ x, float *__restrict__ xf, long long n)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        xf[i] = (float)x[i];
}

__global__ void __launch_bounds__(kDemThreads)
k_dem_substep(DemArgs a)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_p)
        return;
    const int n_p = a.n_p;
    const int p = a.sorted[i];
    const DemParams &dp = a.dp;
    const double R = dp.R;
    double xp[3], upv[3], opv[3];
    float xpf[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        xp[k] = a.x[k * n_p + p];
        upv[k] = a.u[k * n_p + p];
        opv[k] = a.om[k * n_p + p];
        xpf[k] = a.xf[k * n_p + p];
    }

    // contact partners, ascending ids
    int cand[PRS_MAX_CONTACTS];
    int nc = 0;
    bool overflow = false;
    {
        int cc[3];
        cell_coords(a.pcell[p], a.cg, cc);
        int ox[3], oy[3], oz[3];
        int nx = axis_offsets(a.cg, 0, cc[0], ox);
        int ny = axis_offsets(a.cg, 1, cc[1], oy);
        int nz = axis_offsets(a.cg, 2, cc[2], oz);
        for (int kz = 0; kz < nz; kz++)
            for (int ky = 0; ky < ny; ky++)
                for (int kx = 0; kx < nx; kx++) {
                    int cell = ox[kx] + a.cg.nc[0] * (oy[ky] + a.cg.nc[1] * oz[kz]);
                    int j1 = a.start[cell + 1];
                    for (int j = a.start[cell]; j < j1; j++) {
                        int q = a.sorted[j];
                        if (q == p)
                            continue;
                        float xqf[3];
#pragma unroll
                        for (int k = 0; k < 3; k++)
                            xqf[k] = a.xf[k * n_p + q];
                        if (pair_dist2_f32(xpf, xqf, dp.periodic, a.halfL, a.Lf) > a.cut2_f32)
                            continue;
                        double xq[3], dx[3];
#pragma unroll
                        for (int k = 0; k < 3; k++)
                            xq[k] = a.x[k * n_p + q];
                        double dist = p < q ? pair_vector(dp, xp, xq, dx)
                                            : pair_vector(dp, xq, xp, dx);
                        if (!(dist < R + R))
                            continue;
                        int pos;
                        if (nc == PRS_MAX_CONTACTS) {  // keep the 12 lowest ids, flag the rest
                            overflow = true;
                            if (cand[PRS_MAX_CONTACTS - 1] < q)
                                continue;
                            pos = PRS_MAX_CONTACTS - 1;
                        } else {
                            pos = nc++;
                        }
                        while (pos > 0 && cand[pos - 1] > q) {
                            cand[pos] = cand[pos - 1];
                            pos--;
                        }
                        cand[pos] = q;
                    }
                }
    }
    if (overflow)
        atomicOr(a.err, ERRB_CONTACT_OVERFLOW);

    double Fc[3] = {0.0, 0.0, 0.0}, Tc[3] = {0.0, 0.0, 0.0};
    const int old_cnt = a.ho.cnt[p];
    int so = 0;  // merge cursor into the old (sorted) slots
    for (int s = 0; s < nc; s++) {
        const int q = cand[s];
        const int lo = p < q ? p : q, hi = p < q ? q : p;
        double xl[3], xh[3], ul[3], uh[3], ol[3], oh[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            xl[k] = a.x[k * n_p + lo];
            xh[k] = a.x[k * n_p + hi];
            ul[k] = a.u[k * n_p + lo];
            uh[k] = a.u[k * n_p + hi];
            ol[k] = a.om[k * n_p + lo];
            oh[k] = a.om[k * n_p + hi];
        }
        double dx[3];
        double dist = pair_vector(dp, xl, xh, dx);
        double n[3];
#pragma unroll
        for (int k = 0; k < 3; k++)
            n[k] = dx[k] / dist;
        double delta_n = dist - R - R;
        double cl[3], ch[3], ucp[3];
        cross3(ol, n, cl);
        cross3(oh, n, ch);
#pragma unroll
        for (int k = 0; k < 3; k++)
            ucp[k] = ((ul[k] - uh[k]) + R * cl[k]) + R * ch[k];

        while (so < old_cnt && a.ho.pid[so * n_p + p] < q)
            so++;
        double uin, dprev[3];
        if (so < old_cnt && a.ho.pid[so * n_p + p] == q) {  // existing event
            uin = a.ho.uin[so * n_p + p];
#pragma unroll
            for (int k = 0; k < 3; k++)
                dprev[k] = a.ho.dlt[(so * 3 + k) * n_p + p];
        } else {                                              // new event
            uin = dot3(ucp, n);
            dprev[0] = dprev[1] = dprev[2] = 0.0;
        }
        double Fn[3], Ft[3], dnew[3];
        contact_force(n, delta_n, ucp, dprev, dp.kn_pp, dp.dn_pp, dp.kt_pp, dp.dt_pp, dp.mu,
                      a.dt_p, Fn, Ft, dnew);
        a.hn.pid[s * n_p + p] = q;
        a.hn.uin[s * n_p + p] = uin;
#pragma unroll
        for (int k = 0; k < 3; k++)
            a.hn.dlt[(s * 3 + k) * n_p + p] = dnew[k];
        double tq[3];
        cross3(n, Ft, tq);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            double f = Fn[k] + Ft[k];
            if (p == lo)
                Fc[k] += f;
            else
                Fc[k] -= f;
            Tc[k] += R * tq[k];
        }
    }
    a.hn.cnt[p] = nc;

    // walls on bounded axes, low side then high side
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
        for (int side = 0; side < 2; side++) {
            const int ws = (2 * ax + side) * n_p + p;
            if (dp.periodic[ax]) {
                a.hn.wact[ws] = 0;
                continue;
            }
            double dist = side == 0 ? xp[ax] : dp.L[ax] - xp[ax];
            double delta_n = dist - R;
            if (!(delta_n < 0.0)) {  // no wall contact: slot released
                a.hn.wact[ws] = 0;
                continue;
            }
            double n[3] = {0.0, 0.0, 0.0};
            n[ax] = side == 0 ? -1.0 : 1.0;
            double c[3], ucp[3];
            cross3(opv, n, c);
#pragma unroll
            for (int k = 0; k < 3; k++)
                ucp[k] = upv[k] + R * c[k];
            double uin, dprev[3];
            const int wslot = 2 * ax + side;
            if (a.ho.wact[ws]) {
                uin = a.ho.wuin[ws];
#pragma unroll
                for (int k = 0; k < 3; k++)
                    dprev[k] = a.ho.wdlt[(wslot * 3 + k) * n_p + p];
            } else {
                uin = dot3(ucp, n);
                dprev[0] = dprev[1] = dprev[2] = 0.0;
            }
            double Fn[3], Ft[3], dnew[3];
            contact_force(n, delta_n, ucp, dprev, dp.kn_pw, dp.dn_pw, dp.kt_pw, dp.dt_pw,
                          dp.mu, a.dt_p, Fn, Ft, dnew);
            a.hn.wact[ws] = 1;
            a.hn.wuin[ws] = uin;
#pragma unroll
            for (int k = 0; k < 3; k++)
                a.hn.wdlt[(wslot * 3 + k) * n_p + p] = dnew[k];
            double tq[3];
            cross3(n, Ft, tq);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                Fc[k] += Fn[k] + Ft[k];
                Tc[k] += R * tq[k];
            }
        }
    }

    // Newton-Euler, semi-implicit Euler. The update multiplies by the
    // precomputed inverse inertia and fuses multiply-adds: within a rounding
    // or two of the plain formula, and with a third of its FP64 operations,
    // which are slow on this GPU.
    bool finite = true;
    float xnf[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        double acc = __fma_rn(a.Fh[k * n_p + p] + Fc[k], a.inv_m, dp.g[k]);
        double un = __fma_rn(a.dt_p, acc, upv[k]);
        double ang = (a.Th[k * n_p + p] + Tc[k]) * a.inv_J;
        double on = __fma_rn(a.dt_p, ang, opv[k]);
        double xn = __fma_rn(a.dt_p, un, xp[k]);
        if (dp.periodic[k]) {
            double L = dp.L[k];
            if (xn < 0.0) {
                xn += L;
                if (xn >= L)
                    xn = 0.0;
            } else if (xn >= L) {
                xn -= L;
            }
        }
        finite = finite && isfinite(xn) && isfinite(un) && isfinite(on);
        a.un[k * n_p + p] = un;
        a.omn[k * n_p + p] = on;
        a.xn[k * n_p + p] = xn;
        a.xfn[k * n_p + p] = (float)xn;
        xnf[k] = (float)xn;
        a.Fc[k * n_p + p] = Fc[k];
        a.Tc[k * n_p + p] = Tc[k];
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

}  // namespace

void dem_shadow(Ctx &c, cudaStream_t s)
{
    const long long n = 3LL * c.n_p;
    k_shadow<<<(int)((n + 255) / 256), 256, 0, s>>>(c.x[c.cur], c.xf[c.cur], n);
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

void dem_substep(Ctx &c, double dt_p, cudaStream_t s)
{
    const int cur = c.cur, nxt = 1 - c.cur;
    const int ho = c.hcur, hn = 1 - c.hcur;
    phase_begin(c, 3);
    dem_cells_build(c, c.cg, c.x[cur], s, c.d_rebuild);
    phase_end(c);
    DemArgs a;
    a.x = c.x[cur];
    a.u = c.u[cur];
    a.om = c.om[cur];
    a.xn = c.x[nxt];
    a.un = c.u[nxt];
    a.omn = c.om[nxt];
    a.Fh = c.Fh;
    a.Th = c.Th;
    a.Fc = c.Fc;
    a.Tc = c.Tc;
    a.ho = HistPtrs{c.hcnt[ho], c.hpid[ho], c.huin[ho], c.hdlt[ho], c.wact[ho], c.wuin[ho],
                    c.wdlt[ho]};
    a.hn = HistPtrs{c.hcnt[hn], c.hpid[hn], c.huin[hn], c.hdlt[hn], c.wact[hn], c.wuin[hn],
                    c.wdlt[hn]};
    a.sorted = c.cell_sorted;
    a.start = c.cell_start;
    a.pcell = c.pcell;
    a.cg = c.cg;
    a.dp = c.dp;
    a.dt_p = dt_p;
    a.n_p = c.n_p;
    a.err = c.d_err;
    a.xf = c.xf[cur];
    a.xfn = c.xf[nxt];
    {
        double Lmax = 0.0;
        for (int k = 0; k < 3; k++) {
            a.halfL[k] = (float)(0.5 * c.dp.L[k]);
            a.Lf[k] = (float)c.dp.L[k];
            Lmax = fmax(Lmax, c.dp.L[k]);
        }
        // rounding of x to FP32 and of the FP32 differences: < 8 ulp(L) per axis
        const double eps = 16.0 * Lmax * 5.96e-8 + 1e-6;
        const double cut = 2.0 * c.dp.R + eps;
        a.cut2_f32 = (float)(cut * cut * (1.0 + 1e-6));
        const double mv = 0.5 * c.skin - eps;
        a.move2_f32 = (float)(mv > 0.0 ? mv * mv : 0.0);
    }
    a.xb = c.xb;
    a.rebuild = c.d_rebuild;
    a.inv_m = 1.0 / c.dp.m;
    a.inv_J = 1.0 / c.dp.J;
    phase_begin(c, 4);
    k_dem_substep<<<(c.n_p + kDemThreads - 1) / kDemThreads, kDemThreads, 0, s>>>(a);
    phase_end(c);
    c.n_launch += 1;
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
