/*
 * prs_oracle.h -- declarations of the FP64 CPU oracle (test infrastructure
 * only; see prs_oracle.c). Shares nothing with the GPU library.
 *
 * Array conventions: particle vectors are [3][n_p] (all x components, then
 * all y, then all z). Grid fields are [n_z][n_y][n_x] with x fastest.
 */
#ifndef PRS_ORACLE_H
#define PRS_ORACLE_H

#define ORC_MAX_PP 12  /* contact slots per equal sphere (Sec. 3.4) */
#define ORC_MAX_WALL 6 /* one slot per wall: x-lo, x-hi, y-lo, y-hi, z-lo, z-hi */

typedef struct {
    int n[3];          /* cells per axis */
    double h;          /* uniform spacing */
    int periodic[3];   /* 1 = periodic axis, 0 = bounded by walls */
    double off[3][3];  /* off[c][a]: component c lives at (i + off) h on axis a */
    int kernel;        /* regularised delta: 3 (Roma et al. 1999; also 0) or 4 (Peskin 2002) */
} orc_grid;

typedef struct {
    double R, m, J;                     /* radius, translational and rotational inertia */
    double kn_pp, dn_pp, kt_pp, dt_pp;  /* particle-particle spring/dashpot */
    double kn_pw, dn_pw, kt_pw, dt_pw;  /* particle-wall spring/dashpot */
    double mu;                          /* Coulomb friction coefficient */
    double g[3];                        /* gravity */
    double L[3];                        /* domain size */
    int periodic[3];
    int clip_normal;                    /* 1: normal force clipped to be repulsive */
    /* collision model: 0 = linear spring-dashpot; 1 = adaptive collision
     * time model with a Hertzian spring, whose stiffness and damping are
     * calibrated per contact from its impact speed u_in (Sec. 2.1, 3.4) */
    int model;
    double e_n, T_c;                    /* calibration targets */
    double actm_beta, actm_S;           /* dimensionless damping, contact duration */
    double u_min;                       /* smallest impact speed of the calibration */
    /* lubrication (Sec. 2.1, two-parameter model): off when mu_f = 0 */
    double mu_f, eps_d_pp, eps_d_pw, eps_s;
} orc_dem;

/* Contact history M_p / M_temp of Sec. 3.4, per particle:
 * cnt[p] active slots, pid/uin/dlt of slot s at [p*12 + s] (dlt has 3
 * components), partner ids ascending. Wall slots at [p*6 + w]. */
typedef struct {
    int *cnt;
    int *pid;
    double *uin;
    double *dlt;
    unsigned char *wact;
    double *wuin;
    double *wdlt;
} orc_hist;

/* host threads for the particle, marker and grid-slab loops; returns the
 * count in use (1 without OpenMP). Results are bit-identical for any count. */
int orc_set_threads(int n);

double orc_phi(double r);
double orc_phi4(double r);
int orc_marker_count(double R, double h);
double orc_marker_volume(double R, double h, int n_l);
void orc_template(int n_l, double *t);

void orc_interp(const orc_grid *g, int c, const double *field, long n_m,
                const double *X, double *U);
void orc_spread(const orc_grid *g, int c, double *field, long n_m,
                const double *X, const double *F, double dV);

int orc_ibm_step(const orc_grid *g, int n_p, double R, double rho_f,
                 int n_l, const double *t, double dV,
                 const double *x, const double *up, const double *om,
                 double *u, double *v, double *w,
                 double *fx, double *fy, double *fz,
                 double dt, double alpha, int n_mdf_max, double tol,
                 double *F_h, double *T_h, double *F_l, double *res_out);
int orc_ibm_step_warm(const orc_grid *g, int n_p, double R, double rho_f,
                      int n_l, const double *t, double dV,
                      const double *x, const double *up, const double *om,
                      double *u, double *v, double *w,
                      double *fx, double *fy, double *fz,
                      double dt, double alpha, int n_mdf_max, double tol,
                      const double *dF0,
                      double *F_h, double *T_h, double *F_l, double *res_out);

void orc_dem_params(orc_dem *d, double R, double rho_p, double rho_f,
                    double e_n, double e_t, double mu, double T_c,
                    const double g[3], const double L[3], const int per[3]);
void orc_actm_unit(double beta, double *S, double *e);
void orc_actm_calibrate(double e_n, double *beta, double *S);
double orc_lub_lambda(int wall, double eps);
long orc_pairs(const orc_dem *d, int n_p, const double *x, double cutoff,
               int *pairs, long max_pairs);
int orc_dem_substep(const orc_dem *d, int n_p, double dt_p,
                    const double *x, const double *up, const double *om,
                    const double *F_h, const double *T_h,
                    const orc_hist *old, orc_hist *neu,
                    double *x_out, double *u_out, double *om_out,
                    double *F_c, double *T_c);

#endif
