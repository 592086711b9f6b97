/*
 * pr_sed.h -- C ABI of the GB300 particle-side hot path of particle-resolved
 * sediment transport (Zhu, Hu, Lei, Shen, Zheng, arXiv 2108.01814).
 *
 * One context holds one Eulerian grid description and one population of
 * equal spheres. Per fluid (Runge-Kutta) sub-step the caller runs
 *   prs_ibm_step  -- markers from the shared template (Sec. 3.5), velocity
 *                    interpolation with the regularised delta (Sec. 3.3),
 *                    direct forcing (Sec. 2.1, tilde-u = hat-u + alpha dt f),
 *                    spreading back to the grid (Sec. 3.3), per-particle
 *                    force and torque sums (Sec. 3.3 modification 2);
 *   prs_dem_step  -- n_sub particle sub-steps (Sec. 2.1: dt_p = dt_f / 50) of
 *                    cell-list contact search, 12-slot contact history
 *                    (Sec. 3.4), spring-dashpot contact forces (Eq. 9-10,
 *                    Appendix A) and the Newton-Euler update (Eq. 7-8).
 *
 * Conventions
 *   - Grid fields are [nz][ny][nx], x fastest, in the context's precision
 *     (double for PRS_FP64, float for PRS_FP32). Component c of the velocity
 *     lives at ((i + offset[c][0]) h, (j + offset[c][1]) h, (k + offset[c][2]) h).
 *   - Particle vectors are [3][n_p] doubles (all x, then all y, then all z).
 *     Particle state is FP64 in both precisions.
 *   - `where` arguments are PRS_HOST or PRS_DEVICE and say where a pointer
 *     lives. Device pointers must come from the current CUDA device.
 *   - All calls are asynchronous on the context's stream, except the
 *     prs_read_* calls and prs_sync, which synchronise it.
 *   - Every call returns a prs_status: 0 = success, > 0 warning, < 0 error.
 *     prs_last_error_string() describes the last non-zero status of the
 *     calling thread. Errors found by kernels (slot overflow, non-finite
 *     state, capacity) are latched in a device error word and reported by the
 *     next prs_sync / prs_read_* call.
 *   - Ownership: the caller owns grid fields and all arrays it passes; the
 *     context owns particle state, contact history, marker forces and all
 *     scratch, allocated through the prs_allocator given at creation (or
 *     cudaMalloc when it is NULL) and released by prs_destroy.
 */
#ifndef PR_SED_H
#define PR_SED_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct prs_ctx prs_ctx;
typedef int prs_status;

enum {
    PRS_OK = 0,
    PRS_WARN_NOT_CONVERGED = 1,   /* forcing passes ran out before the slip tolerance */
    PRS_ERR_ARG = -1,             /* invalid argument */
    PRS_ERR_OOM = -2,             /* allocator returned NULL */
    PRS_ERR_CUDA = -3,            /* a CUDA runtime call failed */
    PRS_ERR_STATE = -4,           /* call out of order (e.g. no particles yet) */
    PRS_ERR_CONTACT_OVERFLOW = -5,/* a sphere had more than 12 particle contacts */
    PRS_ERR_NONFINITE = -6,       /* NaN or Inf in the particle state */
    PRS_ERR_CAPACITY = -7,        /* a fixed-size buffer was too small */
    PRS_ERR_TIMEOUT = -8          /* a bounded device-side wait ran out */
};

enum { PRS_FP64 = 0, PRS_FP32 = 1 };
enum { PRS_HOST = 0, PRS_DEVICE = 1 };

#define PRS_MAX_CONTACTS 12  /* equal spheres touch at most 12 others (Sec. 3.4) */
#define PRS_MAX_WALLS 6      /* x-lo, x-hi, y-lo, y-hi, z-lo, z-hi */

/* Device memory provider. alloc returns device memory of at least `bytes`
 * bytes usable on `stream` (NULL on failure), aligned to 256 bytes like
 * cudaMalloc's (a pointer that is not is freed again and the call fails
 * with PRS_ERR_OOM: the kernels load vectors and tensor-map tiles from
 * these buffers); free releases it. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, void *stream, void *user);
    void *user;
} prs_allocator;

/* Options of prs_ibm_step (Sec. 2.1 and 3.3). */
typedef struct {
    int n_mdf_max;      /* forcing passes (multi-direct forcing), >= 1 */
    double tol;         /* stop early once max_l |U_d - U(X_l)| < tol; <= 0 never */
    int grid_where;     /* PRS_DEVICE, or PRS_HOST: u..fz are host arrays, copied in and out */
    int final_residual; /* 1: interpolate once more after the last pass to report the slip */
    int learned;        /* 1: warm-start the first pass with the context's network
                           (prs_mlp_*; no counterpart in the paper) */
    int host_async;     /* with PRS_HOST: 1 = return once the work is queued; the
                           arrays hold the result after the next prs_sync or
                           prs_read_* call, and the caller leaves them alone until
                           then (later calls may run while the copies finish) */
    int delta_kernel;   /* regularised delta of Sec. 3.3: 3 (Roma, Peskin & Berger
                           1999; also 0, the default) or 4 (Peskin's 4-point
                           kernel, Peskin 2002, a wider variant); the 4-point
                           kernel takes device fields, no warm start and no
                           training-pair collection, and spreads through a
                           fixed-point scratch grid the context allocates on
                           first use (8 bytes per cell and component) */
} prs_ibm_opts;

/* Options of prs_dem_step: linear spring-dashpot calibrated on the
 * collision time T_c (Sec. 2.1: T_c = 10 dt_f) and the normal / tangential
 * restitution coefficients, Coulomb friction mu, gravity g. Fields left at
 * zero take the defaults stated beside them. */
typedef struct {
    double e_n, e_t, mu, T_c;
    double g[3];
    int clip_normal; /* 1: the normal force (spring + dashpot) is clipped to be
                        repulsive, so a contact exerts no pull while the spheres
                        separate; 0: the plain law of Eq. 9 (default) */
    int model;       /* normal law: PRS_CONTACT_LINEAR (default), or
                        PRS_CONTACT_ACTM, the adaptive collision time model
                        cited in Sec. 2.1 (Kempe & Froehlich 2012): a Hertzian
                        spring k |delta_n|^(3/2) and a dashpot d u_n whose
                        constants each contact takes from its impact speed
                        u_in (recorded at its first sub-step, Sec. 3.4), so that
                        every contact lasts T_c and rebounds with e_n */
    double u_min;    /* ACTM: impact speeds below it are taken as u_min
                        (0: |g| T_c, or 1e-3 R / T_c without gravity) */
    double mu_f;     /* dynamic viscosity of the fluid; > 0 adds the
                        two-parameter lubrication force cited in Sec. 2.1
                        (Costa et al. 2015) to Eq. 9: normal, between spheres
                        6 pi mu_f R (u_n / 2) [lambda(eps) - lambda(eps_d)] and
                        against a wall 6 pi mu_f R u_n [...], at the gap
                        eps = delta_n / R below eps_d and above zero, held at
                        its eps_s value below eps_s (lambda: Jeffrey 1982 for
                        two equal spheres, Cox & Brenner 1967 for a wall) */
    double eps_d_pp, eps_d_pw; /* lubrication range over R (0: 0.05; at most 0.1) */
    double eps_s;              /* lubrication saturation over R (0: 0.001) */
} prs_dem_opts;

enum { PRS_CONTACT_LINEAR = 0, PRS_CONTACT_ACTM = 1 };

/* Counters of the last calls. */
typedef struct {
    int mdf_passes;            /* forcing passes of the last prs_ibm_step */
    double residual;           /* max |U_d - U| of the last interpolation */
    long long n_markers;       /* n_p * n_l */
    long long n_contacts;      /* particle-particle contact slots after the last sub-step */
    long long n_wall_contacts; /* wall slots in use after the last sub-step */
    int error_word;            /* latched device error bits */
    long long n_launches;      /* kernels this context has launched so far */
    long long h2d_bytes;       /* host->device bytes of the last prs_ibm_step (host fields) */
    long long d2h_bytes;       /* device->host bytes of the last prs_ibm_step (host fields) */
    int dem_graph;             /* 1: the last prs_dem_step ran its sub-steps as a CUDA graph */
} prs_stats;

/* Phases timed by prs_set_profiling / prs_read_profile. */
enum {
    PRS_PHASE_IBM_BIN = 0,     /* per-particle preparation and tile binning */
    PRS_PHASE_INTERP = 1,      /* interpolation + direct forcing + particle sums */
    PRS_PHASE_SPREAD = 2,      /* spreading to the grid */
    PRS_PHASE_DEM_CELLS = 3,   /* cell-list build of the contact search */
    PRS_PHASE_DEM_CONTACTS = 4,/* contacts, history, pair forces */
    PRS_PHASE_DEM_UPDATE = 5,  /* force sums, wall contacts, integration */
    PRS_PHASE_MLP = 6,         /* warm-start network: inference, training, features */
    PRS_NPHASES = 7
};

/* Creates a context for an nx x ny x nz grid of spacing h.
 *   periodic[3]: 1 = periodic axis, 0 = bounded by walls at 0 and n h.
 *   offset: 9 doubles offset[c*3 + a], grid point of velocity component c on
 *           axis a sits at (i + offset) h; NULL = 0.5 everywhere (cell centres).
 *   precision: PRS_FP64 or PRS_FP32 (grid fields and marker arithmetic).
 *   alloc: device memory provider, or NULL for cudaMalloc / cudaFree.
 *   stream: cudaStream_t for all work (NULL = legacy default stream).
 * Errors: PRS_ERR_ARG for non-positive sizes or spacing. */
prs_status prs_create_grid(int nx, int ny, int nz, double h, const int periodic[3],
                           const double *offset, int precision, const prs_allocator *alloc,
                           void *stream, prs_ctx **out);

/* Adds n_p equal spheres of radius R and densities rho_p, rho_f (Eq. 7-8).
 * n_markers = 0 picks the thin-shell rule round(pi/3 (12 R^2/h^2 + 1)),
 * which gives the 315 markers of Sec. 3.5 at R = 5h. Allocates the state,
 * contact history and marker buffers. Sets the state to zero; call
 * prs_write_state next. Errors: PRS_ERR_ARG, PRS_ERR_OOM. */
prs_status prs_create_particles(prs_ctx *ctx, int n_p, double R, double rho_p,
                                double rho_f, int n_markers);

/* Particle state x, u, omega, each [3][n_p] doubles. Writing clears the
 * contact history. */
prs_status prs_write_state(prs_ctx *ctx, const double *x, const double *u,
                           const double *omega, int where);
prs_status prs_read_state(prs_ctx *ctx, double *x, double *u, double *omega, int where);

/* One direct-forcing step. u, v, w: fluid velocity (in: hat-u, out:
 * tilde-u = hat-u + alpha dt f_ib on the cells the markers touch);
 * fx, fy, fz: accumulated, f += f_ib. dt: fluid step; alpha: Runge-Kutta
 * coefficient alpha_k. Also sets the per-particle hydrodynamic force and
 * torque F_h = -rho_f sum_l F_l dV, T_h = -rho_f sum_l (X_l - x_p) x F_l dV.
 * The spread is deterministic: repeated calls give bit-identical fields.
 * With grid_where = PRS_HOST the six arrays are host memory (pinned memory
 * copies fastest): the z-slab of planes that marker stencils can reach is
 * copied in and out on two streams the context creates for this (one per
 * direction), overlapped with the kernels; a one-pass step on a grid with
 * walls in z runs as a pipeline over z-chunks of the slab, so that chunks
 * go out while later ones come in. The call returns once the arrays hold
 * the result (host_async = 0) or once the work is queued (host_async = 1).
 * Returns PRS_WARN_NOT_CONVERGED when tol > 0 and the passes ran out. */
prs_status prs_ibm_step(prs_ctx *ctx, void *u, void *v, void *w, void *fx, void *fy,
                        void *fz, double dt, double alpha, const prs_ibm_opts *opts);

/* Predictor of a Runge-Kutta fluid sub-step (Sec. 2.1) with an explicit
 * viscous stand-in for H: H = nu lap_h(u), the second-order central 7-point
 * Laplacian, no convection and no pressure. For velocity component
 * `component` (0..2; its grid offsets set the wall rule):
 *   u_out = u_in + dt (alpha H(u_in) - beta H),  then H <- H(u_in),
 * so that with the paper's RK2 coefficients (alpha_1 = 1, beta_1 = 0;
 * alpha_2 = beta_2 = 1/2) H carries H^{k-1} into sub-step k + 1. H is not
 * read when beta = 0. Walls (non-periodic axes, no-slip): points half a cell
 * off the walls (offset 1/2) see the mirrored ghost -u; points on the walls
 * (offset 0) keep their value at the lower wall and see 0 at the upper one.
 * u_in, u_out, H: device fields [nz][ny][nx] in the context's precision;
 * u_out may not be u_in. Asynchronous on the context's stream.
 * Errors: PRS_ERR_ARG for NULL or aliased fields, a bad component, nu < 0,
 * dt <= 0, or a wall-bounded axis whose offset is neither 0 nor 1/2. */
prs_status prs_predict(prs_ctx *ctx, int component, const void *u_in, void *u_out, void *H,
                       double nu, double dt, double alpha, double beta);

/* n_sub particle sub-steps of length dt_p with F_h, T_h of the last
 * prs_ibm_step held fixed (zero before the first one). */
prs_status prs_dem_step(prs_ctx *ctx, double dt_p, int n_sub, const prs_dem_opts *opts);

/* Per-particle hydrodynamic force/torque and the collision force/torque of
 * the last sub-step, each [3][n_p] doubles; any pointer may be NULL. */
prs_status prs_read_forces(prs_ctx *ctx, double *F_h, double *T_h, double *F_c,
                           double *T_c, int where);

/* Marker forces F_l of the last prs_ibm_step, [3][n_p * n_l] in the
 * context's precision (marker index p * n_l + l). */
prs_status prs_read_marker_forces(prs_ctx *ctx, void *F_l, int where);

/* Marker template: t [3][n_l] unit vectors (may be NULL), marker volume dV
 * and count n_l (may be NULL). */
prs_status prs_read_template(prs_ctx *ctx, double *t, double *dV, int *n_l);

/* Contact history M_p of Sec. 3.4 after the last sub-step, host arrays in
 * per-particle layout: cnt[n_p]; pid[n_p][12] (partner ids ascending, -1
 * unused); uin[n_p][12] (impact velocity); dlt[n_p][12][3] (tangential
 * displacement); wall_act[n_p][6]; wall_uin[n_p][6]; wall_dlt[n_p][6][3].
 * prs_write_history takes the same layout (checkpoint / resume). */
prs_status prs_read_history(prs_ctx *ctx, int *cnt, int *pid, double *uin, double *dlt,
                            unsigned char *wall_act, double *wall_uin, double *wall_dlt);
prs_status prs_write_history(prs_ctx *ctx, const int *cnt, const int *pid,
                             const double *uin, const double *dlt,
                             const unsigned char *wall_act, const double *wall_uin,
                             const double *wall_dlt);

/* All pairs p < q of the current state with centre distance < cutoff
 * (minimum image on periodic axes, Eq. A.1 and A.3), found with the same
 * cell list as the contact search, sorted lexicographically. pairs is a
 * host array of 2 * max_pairs ints; *n_pairs receives the total count (the
 * first min(total, max_pairs) pairs are written). */
prs_status prs_find_pairs(prs_ctx *ctx, double cutoff, int *pairs, long long max_pairs,
                          long long *n_pairs);

/* The pair search of prs_find_pairs without a context and without any
 * device allocation. This entry point has no counterpart in the paper; it
 * serves callers that must not allocate device memory: those that account
 * for every byte through their own pool or a fixed budget, and those whose
 * loop cannot absorb the device-wide synchronisation that cudaFree implies.
 * Its cell list lives in one fixed array inside the library (about 2.6 MB per
 * device), sized for PRS_NOALLOC_MAX_PARTICLES spheres; the cells are widened
 * as needed to fit PRS_NOALLOC_MAX_CELLS.
 *
 *   x         device, [3][n_p] doubles, centres inside [0, L) per axis; a
 *             centre outside that range is put in the nearest edge cell and
 *             its pairs are undefined (the library's own state is always
 *             wrapped into the box before it is searched)
 *   L         host, 3 box lengths; periodic: host, 3 flags (minimum image)
 *   cutoff    pairs p < q with centre distance < cutoff are reported
 *   pairs     device, [max_pairs][2] ints (p, q), order unspecified; the
 *             first min(total, max_pairs) found are written
 *   n_pairs   device, one unsigned long long: receives the total count
 *   stream    CUDA stream (NULL = legacy default); the call is asynchronous
 *
 * Errors (checked before any device work): PRS_ERR_ARG for NULL pointers,
 * negative sizes, a non-positive cutoff or box length, or n_p above
 * PRS_NOALLOC_MAX_PARTICLES; PRS_ERR_CUDA if a CUDA error was already
 * pending when the call began (reported and cleared, nothing launched), or
 * if a launch fails (the message names the kernel).
 * The first call on each device looks up the array's device address (a
 * runtime call on that device, made once); make that first call before any
 * stream capture begins. Every call on a device shares the one array: the
 * counters it needs at zero are cleared at the start of each call, but calls
 * that may run on the device at the same time (other streams, other threads)
 * race on it and give wrong results, so order them on one stream. */
#define PRS_NOALLOC_MAX_PARTICLES 65536
#define PRS_NOALLOC_MAX_CELLS 262144
prs_status prs_find_pairs_noalloc(const double *x, int n_p, const double *L,
                                  const int *periodic, double cutoff, int *pairs,
                                  long long max_pairs, unsigned long long *n_pairs,
                                  void *stream);

/* ---------------------------------------------------------------------
 * Bed and flying spheres, saltation events (Sec. 4.3.1, steps 1-3). The
 * vertical axis is z and the bottom is z = 0.
 *
 * prs_bed_detect classifies the current state. The bottom layer is the
 * spheres whose centre lies below one diameter, z < 2R. Bed spheres are the
 * bottom layer and every sphere in contact (d < 2R, minimum image) with a
 * bed sphere, directly or through other bed spheres; all others fly.
 *   flags: n_p bytes, 1 = bed, 0 = flying, host or device per `where`
 *          (may be NULL); n_bed: receives the count (may be NULL).
 * Synchronises. Errors: PRS_ERR_CAPACITY when the contacts exceed
 * 6 n_p pairs. */
prs_status prs_bed_detect(prs_ctx *ctx, unsigned char *flags, long long *n_bed, int where);

/* One closed impact event of a saltating sphere. */
typedef struct {
    int particle;               /* sphere index */
    int rebound;                /* 1: it departed less than t_cir after the impact */
    double t_impact;            /* time of the first state seen in the bed */
    double t_departure;         /* time of the first state seen flying again */
    double u_impact[3], omega_impact[3];        /* velocities at t_impact */
    double u_departure[3], omega_departure[3];  /* velocities at t_departure */
} prs_event;

/* prs_track_saltation advances every sphere by one observed state, the
 * current one, at time t (call it after each prs_dem_step, for example):
 *   - a departure (bed -> flying) starts a flight at the centre height;
 *   - a flying sphere whose centre rises more than h_r above that height is
 *     saltating (the paper takes h_r = D/2), otherwise it rolls;
 *   - an impact (flying -> bed) of a saltating sphere opens an event;
 *   - the sphere's next departure closes it, as a rebound if it comes less
 *     than t_cir after the impact (the paper takes t_cir = 5 T_c), as an
 *     entrainment after enduring contact otherwise.
 * The events this state closes are written in sphere order to
 * events[0 .. min(n, max_events)), host or device per `where`, and their
 * number n to *n_events. The first call after prs_create_particles or
 * prs_reset_saltation records the states and closes nothing. Synchronises.
 * Errors: PRS_ERR_ARG (h_r or t_cir negative, NULL n_events), and
 * PRS_ERR_CAPACITY when n > max_events (the first max_events are written,
 * the others are lost). */
prs_status prs_track_saltation(prs_ctx *ctx, double t, double h_r, double t_cir,
                               prs_event *events, long long max_events, long long *n_events,
                               int where);
/* Forgets the tracked states: the next prs_track_saltation starts afresh. */
prs_status prs_reset_saltation(prs_ctx *ctx);

/* ---------------------------------------------------------------------
 * Learned warm start of the direct forcing. This part has no counterpart in
 * the paper. A per-marker network 9 -> 64 -> 64 -> 3 with ReLU,
 *   y = W3 relu(W2 relu(W1 x + b1) + b2) + b3,
 * maps the features
 *   x = [U_d - U (slip at the first interpolation),
 *        omega x (X_l - x_p), t_l (outward normal)]
 * to y. With prs_ibm_opts.learned = 1, the first forcing increment becomes
 * (U_d - U + y)/(alpha dt); every later pass stays plain.
 *
 * Training pairs come from the plain solver (prs_mlp_collect). The target
 * is y* = (F_K - F_1) alpha dt, the marker force after K plain passes minus
 * that of the first pass. Loss: mean over markers and components of
 * (y - y*)^2; optimiser: Adam.
 *
 * Inference and training run on the tensor cores with BF16 weights and
 * activations and FP32 accumulation; the master weights and Adam moments
 * are FP32. Parameters cross the ABI as one float vector of PRS_MLP_NPARAM
 * values: W1 [64][9], b1 [64], W2 [64][64], b2 [64], W3 [3][64], b3 [3],
 * row-major.
 *
 * feats, targets and out are device arrays: [n][9], [n][3] and [n][3]
 * floats. The context owns the weights. PRS_ERR_STATE is returned before
 * prs_mlp_set_params; PRS_ERR_TIMEOUT if a tensor-core wait ran out. */
#define PRS_MLP_NPARAM 4995

typedef struct {
    double lr, beta1, beta2, eps;
} prs_adam_opts;

/* Sets the parameters (host array) and clears the Adam state. */
prs_status prs_mlp_set_params(prs_ctx *ctx, const float *params);
/* Current FP32 master parameters into a host array; synchronises. */
prs_status prs_mlp_get_params(prs_ctx *ctx, float *params);
/* out = network(feats) for n rows; asynchronous. */
prs_status prs_mlp_forward(prs_ctx *ctx, const float *feats, long long n, float *out);
/* Loss and gradient (host, PRS_MLP_NPARAM floats, same layout as the
 * parameters) over n rows; synchronises. Either output may be NULL. */
prs_status prs_mlp_grad(prs_ctx *ctx, const float *feats, const float *targets, long long n,
                        float *grad, float *loss);
/* One Adam step on the full batch of n rows. If loss is not NULL it
 * receives the loss before the step, and the call synchronises;
 * otherwise it is asynchronous. */
prs_status prs_mlp_train_step(prs_ctx *ctx, const float *feats, const float *targets,
                              long long n, const prs_adam_opts *opts, float *loss);
/* One Adam step on a minibatch drawn from n_total training pairs without
 * copying them: batch row i (0 <= i < n) is pair (start + i stride) mod
 * n_total. A stride coprime with n_total makes the n rows distinct and,
 * when it is large, spreads them over the whole set, so that a batch of
 * marker-ordered pairs is not a run of neighbouring markers. Requires
 * 1 <= n <= n_total <= 2^40, 0 <= start < n_total, 1 <= stride <= 2^22 and
 * gcd(stride, n_total) = 1, else PRS_ERR_ARG. Otherwise as
 * prs_mlp_train_step, which is the case start = 0, stride = 1, n = n_total. */
prs_status prs_mlp_train_step_sampled(prs_ctx *ctx, const float *feats, const float *targets,
                                      long long n_total, long long n, long long start,
                                      long long stride, const prs_adam_opts *opts,
                                      float *loss);
/* A plain prs_ibm_step (opts.learned is ignored) that also writes the
 * training pairs of every marker: feats [n_p * n_l][9] at the first
 * interpolation and targets [n_p * n_l][3] after the last pass (device
 * arrays, marker index p * n_l + l). */
prs_status prs_mlp_collect(prs_ctx *ctx, void *u, void *v, void *w, void *fx, void *fy,
                           void *fz, double dt, double alpha, const prs_ibm_opts *opts,
                           float *feats, float *targets);

prs_status prs_get_stats(prs_ctx *ctx, prs_stats *stats);

/* Per-phase timing with CUDA events recorded on the context's stream around
 * every launch of a phase (on = 1 starts, 0 stops recording). prs_read_profile
 * synchronises and returns, per phase, the summed milliseconds and the
 * number of timed launches since the last read (arrays of PRS_NPHASES), then
 * clears the record. Either pointer may be NULL. */
prs_status prs_set_profiling(prs_ctx *ctx, int on);
/* The particle sub-steps of prs_dem_step as a CUDA graph (on = 1, the
 * default): the sequence of launches of a call is captured once and
 * replayed by later calls with the same sub-step count, step, options and
 * stream. The graph holds the same kernels in the same order as the
 * launches it replaces, so results are identical; launches are used
 * instead while prs_set_profiling is on, on the legacy default stream, or
 * if the capture is refused; after two graphs in a row that no later call
 * replayed (a caller that changes the step or the options every call) the
 * context also goes back to launches. Either way graphs then stay off for
 * the context until prs_set_graphs(ctx, 1). */
prs_status prs_set_graphs(prs_ctx *ctx, int on);
prs_status prs_read_profile(prs_ctx *ctx, double *ms, long long *launches);
prs_status prs_set_stream(prs_ctx *ctx, void *stream);
/* Waits for the context's stream and reports latched device errors. */
prs_status prs_sync(prs_ctx *ctx);
/* Diagnostics of the device-side waits; the paper has no counterpart.
 * Every wait inside the library's kernels (on a tensor copy, a grid barrier,
 * the tensor cores) is bounded: when it runs out the kernel latches an error
 * bit in the context and returns, the context stays usable for reads, and
 * the next synchronising call (prs_sync, prs_read_*) returns
 * PRS_ERR_TIMEOUT. This call exercises that path without any fault: it
 * launches one block on the context's stream that waits, with the same
 * bounded wait, on a shared-memory barrier that nothing completes, polling
 * at most `polls` times (1 .. 2^24). The latched bit stays set for the
 * context's lifetime. Errors: PRS_ERR_ARG for a NULL context or polls out
 * of range; PRS_ERR_CUDA if the launch fails. */
prs_status prs_probe_wait(prs_ctx *ctx, long long polls);
void prs_destroy(prs_ctx *ctx);
const char *prs_last_error_string(void);

#ifdef __cplusplus
}
#endif

#endif /* PR_SED_H */
