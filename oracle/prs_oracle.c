/*
 * prs_oracle.c -- plain, slow, FP64 CPU oracle for the particle-side hot path
 * of particle-resolved sediment transport (Zhu, Hu, Lei, Shen, Zheng,
 * arXiv 2108.01814).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this file's library. The GPU product path never
 * links, calls or includes it, and it includes nothing of the GPU path.
 *
 * Everything is FP64, compiled with -ffp-contract=off, written as nested
 * loops in a fixed order: particles ascending, markers ascending, stencil
 * z -> y -> x, contact partners ascending.
 *
 * What each part follows:
 *   - Newton-Euler equations, sphere volume and inertia: Sec. 2.1, Eq. 7-8.
 *   - Collision force and torque sums: Sec. 2.1, Eq. 9-10 (lubrication is
 *     not part of this path).
 *   - Contact geometry and tangential displacement: Appendix A, Eq. A.1-A.11.
 *   - Contact history with at most 12 slots, new / existing / finished
 *     events: Sec. 3.4.
 *   - Direct forcing, interpolation and spreading with a regularised delta
 *     function: Sec. 2.1 (tilde-u = hat-u + alpha dt f) and Sec. 3.3.
 *   - Markers generated per particle from one template: Sec. 3.5.
 *
 * Where the paper names a method without printing it, this oracle takes the
 * following readings (each is pinned by the CPU tests):
 *   - delta kernel: the 3-point kernel of Roma, Peskin & Berger (1999), or
 *     as an option Peskin's 4-point kernel (Peskin 2002);
 *   - marker count and marker volume: the thin-shell rule of Uhlmann (2005),
 *     N_L = round(pi/3 (12 R^2/h^2 + 1)), dV = pi h (12 R^2 + h^2)/(3 N_L),
 *     which gives the 315 markers quoted for D/h = 10 in Sec. 3.5;
 *   - marker positions: the golden-angle (Fibonacci) spiral;
 *   - hydrodynamic load: the rigid-body form of Uhlmann (2005),
 *     (rho_p - rho_f) V_p du/dt = -rho_f sum F_l dV + (rho_p - rho_f) V_p g + F_c;
 *   - collision: a linear spring-dashpot calibrated on the collision time
 *     T_c and the restitution coefficients (the ACTM family of Sec. 2.1),
 *     with a Coulomb cap on the tangential force; as an option, the
 *     adaptive collision time model of Kempe & Froehlich (2012) cited in
 *     Sec. 2.1: a Hertzian spring k |delta_n|^(3/2) and a dashpot d u_n
 *     whose constants are set per contact from its impact speed u_in
 *     (recorded at the contact's first sub-step, Sec. 3.4) so that the
 *     contact lasts T_c and rebounds with e_n;
 *   - lubrication, as an option: the two-parameter model of Costa et al.
 *     (2015) cited in Sec. 2.1, a normal force from the small-gap Stokes
 *     resistance (Jeffrey 1982 for two equal spheres, Cox & Brenner 1967
 *     for a sphere and a wall), active for gaps below eps_d R and held at
 *     its value at eps_s R below that;
 *   - integrator: semi-implicit Euler per particle sub-step.
 *
 * Threads (orc_set_threads, one by default): when the library is built with
 * OpenMP, the loops over particles and markers run on several host threads.
 * Each such loop writes only its own particle's or marker's outputs, and the
 * spreading splits the grid into slabs of z-planes, each slab owned by one
 * thread that visits the markers in ascending order. Every output therefore
 * receives the same terms in the same order as with one thread, and the
 * results are bit-identical for any thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "prs_oracle.h"

static int orc_nt = 1;

int orc_set_threads(int n)
{
#ifdef _OPENMP
    orc_nt = n < 1 ? 1 : n;
    return orc_nt;
#else
    (void)n;
    return 1;
#endif
}

#define PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Regularised delta function (Sec. 3.3): Roma-Peskin-Berger 3-point.   */
/* ------------------------------------------------------------------ */
double orc_phi(double r)
{
    double a = fabs(r);
    if (a <= 0.5)
        return (1.0 + sqrt(1.0 - 3.0 * a * a)) / 3.0;
    if (a <= 1.5) {
        double b = 1.0 - a;
        return (5.0 - 3.0 * a - sqrt(1.0 - 3.0 * b * b)) / 6.0;
    }
    return 0.0;
}

/* Peskin's 4-point kernel (Peskin 2002, Acta Numerica), a wider variant of
 * the regularised delta: with the zeroth and first moments it keeps
 * sum_j phi(x - j)^2 = 3/8 for every x. */
double orc_phi4(double r)
{
    double a = fabs(r);
    if (a <= 1.0)
        return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    if (a <= 2.0)
        return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
    return 0.0;
}

/* ------------------------------------------------------------------ */
/* Marker template (Sec. 3.5: markers generated per particle from one  */
/* stored set of points).                                              */
/* ------------------------------------------------------------------ */
int orc_marker_count(double R, double h)
{
    double q = R / h;
    return (int)floor(PI / 3.0 * (12.0 * q * q + 1.0) + 0.5);
}

double orc_marker_volume(double R, double h, int n_l)
{
    /* volume of the shell R-h/2 .. R+h/2, shared equally by the markers */
    return PI * h * (12.0 * R * R + h * h) / (3.0 * (double)n_l);
}

void orc_template(int n_l, double *t)
{
    double golden = PI * (3.0 - sqrt(5.0));
    for (int l = 0; l < n_l; l++) {
        double z = 1.0 - (2.0 * l + 1.0) / (double)n_l;
        double rho = sqrt(1.0 - z * z);
        double ang = (double)l * golden;
        t[0 * n_l + l] = rho * cos(ang);
        t[1 * n_l + l] = rho * sin(ang);
        t[2 * n_l + l] = z;
    }
}

/* ------------------------------------------------------------------ */
/* Grid stencil                                                         */
/* ------------------------------------------------------------------ */
/* Grid points of component c sit at ((i + off[c][a]) h) along axis a.
 * For a point X the stencil along axis a is, for the 3-point kernel, the
 * nearest grid index and its two neighbours, for the 4-point kernel the
 * four indices within 2h; r is (x_i - X)/h. Returns in idx the (wrapped)
 * index, or -1 where a non-periodic axis has no such grid point, and the
 * number of points. */
static int stencil_first(const orc_grid *g, int c, int a, double X)
{
    double s = X / g->h - g->off[c][a];
    return g->kernel == 4 ? (int)floor(s) - 1 : (int)floor(s + 0.5) - 1;
}

static int stencil_axis(const orc_grid *g, int c, int a, double X,
                        int idx[4], double w[4])
{
    const int four = g->kernel == 4;
    const int np = four ? 4 : 3;
    const int i0 = stencil_first(g, c, a, X);
    for (int d = 0; d < np; d++) {
        int i = i0 + d;
        double r = ((double)i + g->off[c][a]) - X / g->h;
        w[d] = four ? orc_phi4(r) : orc_phi(r);
        int n = g->n[a];
        if (g->periodic[a]) {
            int m = i % n;
            if (m < 0)
                m += n;
            idx[d] = m;
        } else {
            idx[d] = (i >= 0 && i < n) ? i : -1;
        }
    }
    return np;
}

/* Interpolation U(X) = sum_ijk u(x_ijk) delta_d(x_ijk - X) h^3 (Sec. 3.3). */
void orc_interp(const orc_grid *g, int c, const double *field, long n_m,
                const double *X, double *U)
{
    long nx = g->n[0], ny = g->n[1];
#pragma omp parallel for schedule(static) num_threads(orc_nt) if (orc_nt > 1)
    for (long m = 0; m < n_m; m++) {
        int ix[4], iy[4], iz[4];
        double wx[4], wy[4], wz[4];
        const int np = stencil_axis(g, c, 0, X[0 * n_m + m], ix, wx);
        stencil_axis(g, c, 1, X[1 * n_m + m], iy, wy);
        stencil_axis(g, c, 2, X[2 * n_m + m], iz, wz);
        double acc = 0.0;
        for (int k = 0; k < np; k++) {
            if (iz[k] < 0)
                continue;
            for (int j = 0; j < np; j++) {
                if (iy[j] < 0)
                    continue;
                for (int i = 0; i < np; i++) {
                    if (ix[i] < 0)
                        continue;
                    long cell = ix[i] + nx * (iy[j] + ny * (long)iz[k]);
                    acc += field[cell] * (wx[i] * wy[j] * wz[k]);
                }
            }
        }
        U[m] = acc;
    }
}

/* Spreading f(x_ijk) += sum_l F_l delta_d(x_ijk - X_l) dV_l (Sec. 3.3).
 * Thread t of T owns the z-planes [t nz / T, (t + 1) nz / T) and adds, in
 * ascending marker order, only the terms that fall on its planes. */
void orc_spread(const orc_grid *g, int c, double *field, long n_m,
                const double *X, const double *F, double dV)
{
    long nx = g->n[0], ny = g->n[1];
    double h3 = g->h * g->h * g->h;
#pragma omp parallel num_threads(orc_nt) if (orc_nt > 1)
    {
        int T = 1, t = 0;
#ifdef _OPENMP
        T = omp_get_num_threads();
        t = omp_get_thread_num();
#endif
        const int nz = g->n[2];
        const int z0 = (int)((long)nz * t / T), z1 = (int)((long)nz * (t + 1) / T);
        const int np_z = g->kernel == 4 ? 4 : 3;
        for (long m = 0; m < n_m; m++) {
            /* skip markers whose z-stencil misses this thread's planes */
            const int i0 = stencil_first(g, c, 2, X[2 * n_m + m]);
            int hit = 0;
            for (int d = 0; d < np_z && !hit; d++) {
                int i = i0 + d;
                if (g->periodic[2]) {
                    i %= nz;
                    if (i < 0)
                        i += nz;
                }
                hit = i >= z0 && i < z1;
            }
            if (!hit)
                continue;
            int ix[4], iy[4], iz[4];
            double wx[4], wy[4], wz[4];
            const int np = stencil_axis(g, c, 0, X[0 * n_m + m], ix, wx);
            stencil_axis(g, c, 1, X[1 * n_m + m], iy, wy);
            stencil_axis(g, c, 2, X[2 * n_m + m], iz, wz);
            for (int k = 0; k < np; k++) {
                if (iz[k] < z0 || iz[k] >= z1)
                    continue;
                for (int j = 0; j < np; j++) {
                    if (iy[j] < 0)
                        continue;
                    for (int i = 0; i < np; i++) {
                        if (ix[i] < 0)
                            continue;
                        long cell = ix[i] + nx * (iy[j] + ny * (long)iz[k]);
                        field[cell] += F[m] * (wx[i] * wy[j] * wz[k]) * dV / h3;
                    }
                }
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* One direct-forcing IBM step (Sec. 2.1 and 3.3).                      */
/* ------------------------------------------------------------------ */
int orc_ibm_step(const orc_grid *g, int n_p, double R, double rho_f,
                 int n_l, const double *t, double dV,
                 const double *x, const double *up, const double *om,
                 double *u, double *v, double *w,
                 double *fx, double *fy, double *fz,
                 double dt, double alpha, int n_mdf_max, double tol,
                 double *F_h, double *T_h, double *F_l, double *res_out)
{
    return orc_ibm_step_warm(g, n_p, R, rho_f, n_l, t, dV, x, up, om, u, v, w, fx, fy, fz,
                             dt, alpha, n_mdf_max, tol, NULL, F_h, T_h, F_l, res_out);
}

/* The same step with a warm start: the first forcing increment is
 * (U_d - U)/(alpha dt) + dF0 instead of the plain one; every later pass is
 * plain. dF0 is [3][n_p * n_l] (force units) or NULL. */
int orc_ibm_step_warm(const orc_grid *g, int n_p, double R, double rho_f,
                      int n_l, const double *t, double dV,
                      const double *x, const double *up, const double *om,
                      double *u, double *v, double *w,
                      double *fx, double *fy, double *fz,
                      double dt, double alpha, int n_mdf_max, double tol,
                      const double *dF0,
                      double *F_h, double *T_h, double *F_l, double *res_out)
{
    long n_m = (long)n_p * n_l;
    double *X = malloc(sizeof(double) * 3 * n_m);
    double *Ud = malloc(sizeof(double) * 3 * n_m);
    double *U = malloc(sizeof(double) * 3 * n_m);
    double *F = calloc(3 * n_m, sizeof(double));
    double *dF = malloc(sizeof(double) * 3 * n_m);
    double *dFs = malloc(sizeof(double) * 3 * n_m);
    if (!X || !Ud || !U || !F || !dF || !dFs) {
        free(X); free(Ud); free(U); free(F); free(dF); free(dFs);
        return -1;
    }
    double *fld[3] = {u, v, w};
    double *frc[3] = {fx, fy, fz};

    /* markers X_l = x_p + R t_l and rigid-body velocity
     * U_d = u_p + omega_p x (X_l - x_p) */
#pragma omp parallel for schedule(static) num_threads(orc_nt) if (orc_nt > 1)
    for (int p = 0; p < n_p; p++) {
        for (int l = 0; l < n_l; l++) {
            long m = (long)p * n_l + l;
            double r[3];
            for (int a = 0; a < 3; a++) {
                r[a] = R * t[a * n_l + l];
                X[a * n_m + m] = x[a * n_p + p] + r[a];
            }
            double ox = om[0 * n_p + p], oy = om[1 * n_p + p], oz = om[2 * n_p + p];
            Ud[0 * n_m + m] = up[0 * n_p + p] + (oy * r[2] - oz * r[1]);
            Ud[1 * n_m + m] = up[1 * n_p + p] + (oz * r[0] - ox * r[2]);
            Ud[2 * n_m + m] = up[2 * n_p + p] + (ox * r[1] - oy * r[0]);
        }
    }

    /* multi-direct forcing: interpolate, force, spread, repeat */
    int it = 0;
    double res = 0.0;
    for (;;) {
        for (int c = 0; c < 3; c++)
            orc_interp(g, c, fld[c], n_m, X, U + c * n_m);
        res = 0.0;
#pragma omp parallel for schedule(static) reduction(max : res) num_threads(orc_nt) if (orc_nt > 1)
        for (long i = 0; i < 3 * n_m; i++) {
            double e = fabs(Ud[i] - U[i]);
            if (e > res)
                res = e;
        }
        if (tol > 0.0 && res < tol)
            break;
        if (it >= n_mdf_max)
            break;
#pragma omp parallel for schedule(static) num_threads(orc_nt) if (orc_nt > 1)
        for (long i = 0; i < 3 * n_m; i++) {
            dF[i] = (Ud[i] - U[i]) / (alpha * dt);
            if (dF0 && it == 0)
                dF[i] += dF0[i];
            F[i] += dF[i];
        }
        /* f += spread(dF) and u += alpha dt spread(dF): tilde-u = hat-u + alpha dt f */
#pragma omp parallel for schedule(static) num_threads(orc_nt) if (orc_nt > 1)
        for (long i = 0; i < 3 * n_m; i++)
            dFs[i] = alpha * dt * dF[i];
        for (int c = 0; c < 3; c++) {
            orc_spread(g, c, frc[c], n_m, X, dF + c * n_m, dV);
            orc_spread(g, c, fld[c], n_m, X, dFs + c * n_m, dV);
        }
        it++;
    }

    /* hydrodynamic force and torque on each particle:
     * F_h = -rho_f sum_l F_l dV, T_h = -rho_f sum_l (X_l - x_p) x F_l dV */
#pragma omp parallel for schedule(static) num_threads(orc_nt) if (orc_nt > 1)
    for (int p = 0; p < n_p; p++) {
        double sf[3] = {0, 0, 0}, st[3] = {0, 0, 0};
        for (int l = 0; l < n_l; l++) {
            long m = (long)p * n_l + l;
            double r[3], f[3];
            for (int a = 0; a < 3; a++) {
                r[a] = R * t[a * n_l + l];
                f[a] = F[a * n_m + m] * dV;
            }
            sf[0] += f[0];
            sf[1] += f[1];
            sf[2] += f[2];
            st[0] += r[1] * f[2] - r[2] * f[1];
            st[1] += r[2] * f[0] - r[0] * f[2];
            st[2] += r[0] * f[1] - r[1] * f[0];
        }
        for (int a = 0; a < 3; a++) {
            F_h[a * n_p + p] = -rho_f * sf[a];
            T_h[a * n_p + p] = -rho_f * st[a];
        }
    }
    if (F_l)
        memcpy(F_l, F, sizeof(double) * 3 * n_m);
    if (res_out)
        *res_out = res;
    free(X); free(Ud); free(U); free(F); free(dF); free(dFs);
    return it;
}

/* ------------------------------------------------------------------ */
/* Soft-sphere DEM (Sec. 2.1 Eq. 7-10, Sec. 3.4, Appendix A).           */
/* ------------------------------------------------------------------ */
void orc_dem_params(orc_dem *d, double R, double rho_p, double rho_f,
                    double e_n, double e_t, double mu, double T_c,
                    const double g[3], const double L[3], const int per[3])
{
    double Vp = 4.0 / 3.0 * PI * R * R * R;
    d->R = R;
    d->m = (rho_p - rho_f) * Vp;          /* inertia of Eq. 7 in rigid-body form */
    d->J = 0.4 * d->m * R * R;            /* I_p (1 - rho_f/rho_p), Eq. 8 */
    double ln_n = log(e_n), ln_t = log(e_t);
    double me[2] = {0.5 * d->m, d->m};    /* P-P (two equal spheres), P-W */
    double *kn[2] = {&d->kn_pp, &d->kn_pw}, *dn[2] = {&d->dn_pp, &d->dn_pw};
    double *kt[2] = {&d->kt_pp, &d->kt_pw}, *dtg[2] = {&d->dt_pp, &d->dt_pw};
    for (int s = 0; s < 2; s++) {
        *kn[s] = me[s] * (PI * PI + ln_n * ln_n) / (T_c * T_c);
        *dn[s] = -2.0 * me[s] * ln_n / T_c;
        *kt[s] = (2.0 / 7.0) * me[s] * (PI * PI + ln_t * ln_t) / (T_c * T_c);
        *dtg[s] = -(2.0 / 7.0) * 2.0 * me[s] * ln_t / T_c;
    }
    d->mu = mu;
    d->clip_normal = 0;
    d->model = 0;
    d->e_n = e_n;
    d->T_c = T_c;
    d->actm_beta = 0.0;
    d->actm_S = 0.0;
    d->u_min = 0.0;
    d->mu_f = 0.0;
    d->eps_d_pp = 0.05;
    d->eps_d_pw = 0.05;
    d->eps_s = 0.001;
    for (int a = 0; a < 3; a++) {
        d->g[a] = g[a];
        d->L[a] = L[a];
        d->periodic[a] = per[a];
    }
}

/* Adaptive collision time model, in units of the impact: with the overlap
 * x = z / (v tau) and t = s tau, tau = (m / (k sqrt(v)))^(2/5), the contact
 * m z'' + d z' + k z^(3/2) = 0, z(0) = 0, z'(0) = v becomes
 * x'' + beta x' + x^(3/2) = 0, x(0) = 0, x'(0) = 1 with beta = d tau / m:
 * its duration S and restitution e = -x'(S) depend on beta alone. Classical
 * fourth-order Runge-Kutta with a fixed step; the exit x(S) = 0 by a
 * shorter last step whose length the secant method finds. */
static void actm_rhs(double beta, double x, double v, double *dx, double *dv)
{
    *dx = v;
    *dv = -beta * v - (x > 0.0 ? x * sqrt(x) : 0.0);
}

/* one Runge-Kutta step of length h from (x, v) */
static void actm_step(double beta, double h, double *x, double *v)
{
    double k1x, k1v, k2x, k2v, k3x, k3v, k4x, k4v;
    actm_rhs(beta, *x, *v, &k1x, &k1v);
    actm_rhs(beta, *x + 0.5 * h * k1x, *v + 0.5 * h * k1v, &k2x, &k2v);
    actm_rhs(beta, *x + 0.5 * h * k2x, *v + 0.5 * h * k2v, &k3x, &k3v);
    actm_rhs(beta, *x + h * k3x, *v + h * k3v, &k4x, &k4v);
    *x += h / 6.0 * (k1x + 2.0 * k2x + 2.0 * k3x + k4x);
    *v += h / 6.0 * (k1v + 2.0 * k2v + 2.0 * k3v + k4v);
}

void orc_actm_unit(double beta, double *S, double *e)
{
    const double h = 1e-5;
    double x = 0.0, v = 1.0;
    for (long it = 0; it < 10000000; it++) {
        double xn = x, vn = v;
        actm_step(beta, h, &xn, &vn);
        if (it > 0 && xn <= 0.0) {
            /* the exit inside this step: the length s of a shorter step that
             * lands on x = 0, by the secant method from s = 0 and s = h */
            double s0 = 0.0, f0 = x, s1 = h, f1 = xn;
            for (int k = 0; k < 60 && f1 != f0; k++) {
                const double s2 = s1 - f1 * (s1 - s0) / (f1 - f0);
                double xs = x, vs = v;
                actm_step(beta, s2, &xs, &vs);
                s0 = s1;
                f0 = f1;
                s1 = s2;
                f1 = xs;
                if (fabs(s1 - s0) < 1e-18)
                    break;
            }
            double xs = x, vs = v;
            actm_step(beta, s1, &xs, &vs);
            *S = (double)it * h + s1;
            *e = -vs;
            return;
        }
        x = xn;
        v = vn;
    }
    *S = 1e7 * h;
    *e = 0.0;
}

/* the damping beta whose unit collision rebounds with e_n (e decreases as
 * beta grows; bisection) and that collision's duration */
void orc_actm_calibrate(double e_n, double *beta, double *S)
{
    double lo = 0.0, hi = 1.0, Sx, ex;
    for (;;) {
        orc_actm_unit(hi, &Sx, &ex);
        if (ex < e_n || hi > 64.0)
            break;
        hi *= 2.0;
    }
    for (int it = 0; it < 60; it++) {
        const double mid = 0.5 * (lo + hi);
        orc_actm_unit(mid, &Sx, &ex);
        if (ex > e_n)
            lo = mid;
        else
            hi = mid;
    }
    *beta = 0.5 * (lo + hi);
    orc_actm_unit(*beta, S, &ex);
}

/* Stokes amplification of the normal resistance at the dimensionless gap
 * eps = delta_n / R: two equal spheres approaching each other (wall = 0;
 * the force on each is 6 pi mu R (u_n / 2) lambda, u_n their relative normal
 * speed; Jeffrey 1982), a sphere approaching a wall (wall = 1; 6 pi mu R u_n
 * lambda; Cox & Brenner 1967). */
double orc_lub_lambda(int wall, double eps)
{
    const double le = log(eps);
    if (wall)
        return 1.0 / eps - 0.2 * le - (1.0 / 21.0) * eps * le + 0.9713;
    return 1.0 / (2.0 * eps) - (9.0 / 20.0) * le - (3.0 / 56.0) * eps * le + 1.346;
}

/* normal lubrication force factor: F = -6 pi mu R w lambda-term u_n n on the
 * sphere, w = 1/2 between two spheres and 1 against a wall; zero in contact
 * (delta_n < 0) and beyond eps_d R; lambda held at its eps_s value below */
static double lub_factor(const orc_dem *d, int wall, double delta_n)
{
    const double eps_d = wall ? d->eps_d_pw : d->eps_d_pp;
    if (d->mu_f <= 0.0 || delta_n < 0.0 || !(delta_n < eps_d * d->R))
        return 0.0;
    double eps = delta_n / d->R;
    if (eps < d->eps_s)
        eps = d->eps_s;
    const double w = wall ? 1.0 : 0.5;
    return 6.0 * PI * d->mu_f * d->R * w * (orc_lub_lambda(wall, eps) - orc_lub_lambda(wall, eps_d));
}

/* separation vector from particle a to particle b, minimum image on
 * periodic axes, and its length */
static double pair_vector(const orc_dem *d, int n_p, const double *x,
                          int a, int b, double dx[3])
{
    for (int k = 0; k < 3; k++) {
        double s = x[k * n_p + b] - x[k * n_p + a];
        if (d->periodic[k]) {
            double L = d->L[k];
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

long orc_pairs(const orc_dem *d, int n_p, const double *x, double cutoff,
               int *pairs, long max_pairs)
{
    long n = 0;
    for (int p = 0; p < n_p; p++) {
        for (int q = p + 1; q < n_p; q++) {
            double dx[3];
            double dist = pair_vector(d, n_p, x, p, q, dx);
            if (dist < cutoff) {
                if (n < max_pairs) {
                    pairs[2 * n] = p;
                    pairs[2 * n + 1] = q;
                }
                n++;
            }
        }
    }
    return n;
}

static void cross(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot(const double a[3], const double b[3])
{
    return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

/* Tangential displacement and contact force for one contact, seen from
 * the particle whose relative contact velocity is ucp (Appendix A).
 * Inputs: n, delta_n, ucp, the previous displacement (A.9-A.11), spring
 * and damping constants. Outputs: normal and tangential force on that
 * particle, the new displacement. */
static void contact_force(const orc_dem *d, double m_eff, double uin,
                          const double n[3], double delta_n, const double ucp[3],
                          const double dprev[3], double kn, double dn,
                          double kt, double dtc, double mu, double dt_p, int clip,
                          double Fn[3], double Ft[3], double dnew[3])
{
    double un = dot(ucp, n);                                   /* A.7 */
    double ucpt[3];
    for (int k = 0; k < 3; k++)
        ucpt[k] = ucp[k] - un * n[k];                          /* A.8 */
    double dd = dot(dprev, n);
    double dtil[3];
    for (int k = 0; k < 3; k++)
        dtil[k] = dprev[k] - dd * n[k];                        /* A.9 */
    double nprev = sqrt(dot(dprev, dprev));
    double ntil = sqrt(dot(dtil, dtil));
    double dhat[3];
    for (int k = 0; k < 3; k++)                                /* A.10 */
        dhat[k] = (ntil > 0.0) ? (nprev / ntil) * dtil[k] : 0.0;
    for (int k = 0; k < 3; k++)
        dnew[k] = dhat[k] + dt_p * ucpt[k];                    /* A.11 */
    double s = kn * delta_n - dn * un;      /* Eq. 9: s < 0 pushes the particle along -n */
    if (d->model == 1) {
        /* ACTM: k and d of the unit collision scaled to this contact's impact
         * speed, tau = T_c / S: k = m tau^(-5/2) v^(-1/2), d = beta m / tau */
        const double v = fabs(uin) > d->u_min ? fabs(uin) : d->u_min;
        const double tau = d->T_c / d->actm_S;
        const double k = m_eff / (tau * tau * sqrt(tau) * sqrt(v));
        const double dd_ = d->actm_beta * m_eff / tau;
        const double ov = -delta_n;
        s = -(k * (ov * sqrt(ov))) - dd_ * un;
    }
    if (clip && s > 0.0)                     /* clipped variant: never attractive */
        s = 0.0;
    for (int k = 0; k < 3; k++) {
        Fn[k] = s * n[k];
        Ft[k] = -(kt * dnew[k]) - dtc * ucpt[k];
    }
    double fn = fabs(s);
    double ft = sqrt(dot(Ft, Ft));
    if (ft > mu * fn) {
        double scale = mu * fn / ft;
        for (int k = 0; k < 3; k++) {
            Ft[k] = scale * Ft[k];
            dnew[k] = -(Ft[k] + dtc * ucpt[k]) / kt;
        }
    }
}

int orc_dem_substep(const orc_dem *d, int n_p, double dt_p,
                    const double *x, const double *up, const double *om,
                    const double *F_h, const double *T_h,
                    const orc_hist *old, orc_hist *neu,
                    double *x_out, double *u_out, double *om_out,
                    double *F_c, double *T_c)
{
    double R = d->R;
    int status = 0;
#pragma omp parallel for schedule(static) reduction(max : status) num_threads(orc_nt) if (orc_nt > 1)
    for (int p = 0; p < n_p; p++) {
        double Fc[3] = {0, 0, 0}, Tc[3] = {0, 0, 0};
        int cnt = 0;
        /* particle-particle contacts, partners ascending */
        for (int q = 0; q < n_p; q++) {
            if (q == p)
                continue;
            int lo = p < q ? p : q, hi = p < q ? q : p;
            double dx[3];
            double dist = pair_vector(d, n_p, x, lo, hi, dx);
            if (!(dist < R + R)) {
                /* lubrication across the gap (normal only, no torque),
                 * in canonical orientation, negated for the higher id */
                const double lf = lub_factor(d, 0, dist - R - R);
                if (lf != 0.0) {
                    double nl[3], un = 0.0;
                    for (int k = 0; k < 3; k++)
                        nl[k] = dx[k] / dist;
                    for (int k = 0; k < 3; k++)
                        un += (up[k * n_p + lo] - up[k * n_p + hi]) * nl[k];
                    for (int k = 0; k < 3; k++) {
                        const double f = -(lf * un) * nl[k];
                        if (p == lo)
                            Fc[k] += f;
                        else
                            Fc[k] -= f;
                    }
                }
                continue;
            }
            double n[3];
            for (int k = 0; k < 3; k++)
                n[k] = dx[k] / dist;                            /* A.1 */
            double delta_n = dist - R - R;                      /* A.3 */
            double ol[3] = {om[0 * n_p + lo], om[1 * n_p + lo], om[2 * n_p + lo]};
            double oh[3] = {om[0 * n_p + hi], om[1 * n_p + hi], om[2 * n_p + hi]};
            double cl[3], ch[3], ucp[3];
            cross(ol, n, cl);
            cross(oh, n, ch);
            for (int k = 0; k < 3; k++)                         /* A.5 */
                ucp[k] = ((up[k * n_p + lo] - up[k * n_p + hi]) + R * cl[k]) + R * ch[k];
            /* history lookup in M_temp (Sec. 3.4) */
            double uin = 0.0, dprev[3] = {0, 0, 0};
            int found = -1;
            for (int s = 0; s < old->cnt[p]; s++) {
                if (old->pid[p * ORC_MAX_PP + s] == q) {
                    found = s;
                    break;
                }
            }
            if (found >= 0) {                                   /* existing event */
                uin = old->uin[p * ORC_MAX_PP + found];
                for (int k = 0; k < 3; k++)
                    dprev[k] = old->dlt[(p * ORC_MAX_PP + found) * 3 + k];
            } else {                                            /* new event */
                uin = dot(ucp, n);
            }
            double Fn[3], Ft[3], dnew[3];
            contact_force(d, 0.5 * d->m, uin, n, delta_n, ucp, dprev, d->kn_pp, d->dn_pp, d->kt_pp,
                          d->dt_pp, d->mu, dt_p, d->clip_normal, Fn, Ft, dnew);
            if (cnt < ORC_MAX_PP) {
                neu->pid[p * ORC_MAX_PP + cnt] = q;
                neu->uin[p * ORC_MAX_PP + cnt] = uin;
                for (int k = 0; k < 3; k++)
                    neu->dlt[(p * ORC_MAX_PP + cnt) * 3 + k] = dnew[k];
            } else {
                status = 1; /* more than 12 contacts: slot overflow */
            }
            cnt++;
            double tq[3];
            cross(n, Ft, tq);
            for (int k = 0; k < 3; k++) {
                double f = Fn[k] + Ft[k];
                if (p == lo)
                    Fc[k] += f;
                else
                    Fc[k] -= f;
                Tc[k] += R * tq[k];
            }
        }
        neu->cnt[p] = cnt < ORC_MAX_PP ? cnt : ORC_MAX_PP;
        /* finished events are the old slots not copied to M_p: dropped */

        /* particle-wall contacts on non-periodic axes: low wall then high */
        for (int a = 0; a < 3; a++) {
            if (d->periodic[a])
                continue;
            for (int side = 0; side < 2; side++) {
                int wslot = 2 * a + side;
                double dist = side == 0 ? x[a * n_p + p] : d->L[a] - x[a * n_p + p];
                double delta_n = dist - R;                      /* A.4 */
                int ws = p * ORC_MAX_WALL + wslot;
                if (!(delta_n < 0.0)) {
                    const double lf = lub_factor(d, 1, delta_n);
                    if (lf != 0.0) {
                        const double nw = side == 0 ? -1.0 : 1.0;
                        const double un = up[a * n_p + p] * nw;
                        Fc[a] += -(lf * un) * nw;
                    }
                    neu->wact[ws] = 0;
                    neu->wuin[ws] = 0.0;
                    for (int k = 0; k < 3; k++)
                        neu->wdlt[ws * 3 + k] = 0.0;
                    continue;
                }
                double n[3] = {0, 0, 0};
                n[a] = side == 0 ? -1.0 : 1.0;                  /* A.2 */
                double o[3] = {om[0 * n_p + p], om[1 * n_p + p], om[2 * n_p + p]};
                double c[3], ucp[3];
                cross(o, n, c);
                for (int k = 0; k < 3; k++)                     /* A.6 */
                    ucp[k] = up[k * n_p + p] + R * c[k];
                double uin = 0.0, dprev[3] = {0, 0, 0};
                if (old->wact[ws]) {
                    uin = old->wuin[ws];
                    for (int k = 0; k < 3; k++)
                        dprev[k] = old->wdlt[ws * 3 + k];
                } else {
                    uin = dot(ucp, n);
                }
                double Fn[3], Ft[3], dnew[3];
                contact_force(d, d->m, uin, n, delta_n, ucp, dprev, d->kn_pw, d->dn_pw, d->kt_pw,
                              d->dt_pw, d->mu, dt_p, d->clip_normal, Fn, Ft, dnew);
                neu->wact[ws] = 1;
                neu->wuin[ws] = uin;
                for (int k = 0; k < 3; k++)
                    neu->wdlt[ws * 3 + k] = dnew[k];
                double tq[3];
                cross(n, Ft, tq);
                for (int k = 0; k < 3; k++) {
                    Fc[k] += Fn[k] + Ft[k];
                    Tc[k] += R * tq[k];
                }
            }
        }
        for (int a = 0; a < 6; a++) {
            if (d->periodic[a / 2]) {
                int ws = p * ORC_MAX_WALL + a;
                neu->wact[ws] = 0;
                neu->wuin[ws] = 0.0;
                for (int k = 0; k < 3; k++)
                    neu->wdlt[ws * 3 + k] = 0.0;
            }
        }

        /* Newton-Euler, semi-implicit Euler (Eq. 7-8, rigid-body form) */
        for (int k = 0; k < 3; k++) {
            double acc = (F_h[k * n_p + p] + Fc[k]) / d->m + d->g[k];
            double un = up[k * n_p + p] + dt_p * acc;
            double ang = (T_h[k * n_p + p] + Tc[k]) / d->J;
            double on = om[k * n_p + p] + dt_p * ang;
            double xn = x[k * n_p + p] + dt_p * un;
            if (d->periodic[k]) {
                double L = d->L[k];
                if (xn < 0.0) {
                    xn += L;
                    if (xn >= L)
                        xn = 0.0;
                } else if (xn >= L) {
                    xn -= L;
                }
            }
            u_out[k * n_p + p] = un;
            om_out[k * n_p + p] = on;
            x_out[k * n_p + p] = xn;
            if (F_c)
                F_c[k * n_p + p] = Fc[k];
            if (T_c)
                T_c[k * n_p + p] = Tc[k];
        }
    }
    return status;
}
