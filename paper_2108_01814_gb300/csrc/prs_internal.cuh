// Internal declarations shared by the translation units of the GB300 library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "pr_sed.h"

namespace prs {

// device error bits (latched in Ctx::d_err)
enum : int {
    ERRB_CONTACT_OVERFLOW = 1,
    ERRB_NONFINITE = 2,
    ERRB_CAPACITY = 4,
    ERRB_MLP_TIMEOUT = 8,  // a tensor-core wait of the warm-start network ran out
    ERRB_BARRIER_TIMEOUT = 16,  // a grid barrier of the cell-list rebuild ran out
    ERRB_TMA_TIMEOUT = 32,      // a wait on the interpolation's tensor copies ran out
};

// Adam hyper-parameters of one step, with the bias corrections
// c1 = 1/(1 - beta1^k) and c2 = 1/(1 - beta2^k)
struct MlpAdam {
    double lr, b1, b2, eps, c1, c2;
};

// IBM tiles: kTileX x kTileY x kTileZ cells (x fastest)
constexpr int kRedWords = 4;  // words of Ctx::d_red
constexpr int kRedRes = 3;    // the residual word
constexpr int kTileX = 16, kTileY = 8, kTileZ = 8;

// Per-particle data computed once per IBM step: for velocity component c
// and axis a, base[c*3+a] = floor(x_a/h - off[c][a]) and frac = the rest in
// [0, 1) (computed in FP64, stored in the marker precision), plus the
// particle velocity and spin in the marker precision.
template <typename T>
struct PartPrep {
    int base[9];
    T frac[9];
    T up[3];
    T om[3];
};

// The same, compact and 16-byte aligned for vector loads, when all velocity
// components share grid offsets (only component 0 is needed).
template <typename T>
struct alignas(16) PartFast {
    T fr[4];   // frac of component 0 (x, y, z), pad
    T up[4];   // particle velocity, pad
    T om[4];   // angular velocity, pad
    int b[4];  // base of component 0 (x, y, z), pad
};

struct GridDesc {
    int n[3];
    int periodic[3];
    double h;
    double off[9];
    int same_off;  // all components share offsets
};

struct DemParams {
    double R, m, J;
    double kn_pp, dn_pp, kt_pp, dt_pp;
    double kn_pw, dn_pw, kt_pw, dt_pw;
    double mu;
    double g[3];
    double L[3];
    int periodic[3];
    int clip_n;  // normal force clipped to be repulsive
    // adaptive collision time model: kn_* and dn_* then hold m_eff tau^(-5/2)
    // and beta m_eff / tau, the stiffness being kn / sqrt(max(|u_in|, u_min))
    int model;
    double u_min;
    // lubrication (off when mu_f = 0): force factors 6 pi mu_f R w, ranges
    // and saturation over R, and lambda at the range's end
    double mu_f, lub_pp, lub_pw, eps_d_pp, eps_d_pw, eps_s, lam_d_pp, lam_d_pw;
};

struct CellGeom {
    int nc[3];
    double cs[3];  // cell edge per axis (>= the search cutoff)
    int periodic[3];
    double L[3];
};

// All device buffers of one context. Particle vectors are [3][n_p];
// history slot s of particle p sits at s * n_p + p (structure of arrays).
struct Ctx {
    GridDesc g;
    int precision;
    prs_allocator alloc;
    int have_alloc;
    cudaStream_t stream;

    // particles
    int n_p = 0;
    double R = 0, rho_p = 0, rho_f = 0, dV = 0;
    int n_l = 0;
    double *x[2] = {}, *u[2] = {}, *om[2] = {};
    float *xf[2] = {};  // FP32 copies of x (contact pre-filter), u and omega
    float *xl[2] = {};  // FP32 remainders x - xf: x as an unevaluated FP32 pair
    float *uf[2] = {}, *omf[2] = {};
    int cur = 0;
    double *Fh = nullptr, *Th = nullptr, *Fc = nullptr, *Tc = nullptr;
    // FP32 form: FP32 copies of F_h, T_h for the sub-steps and the FP32
    // collision force and torque they produce
    float *Fhf = nullptr, *Thf = nullptr, *Fcf = nullptr, *Tcf = nullptr;

    // marker template: unit vectors (FP64), R/h t and R t in marker precision
    double *t64 = nullptr;
    float *t32 = nullptr;  // t_l rounded to FP32 (network features)
    void *tR = nullptr;
    void *rR = nullptr;
    void *prep = nullptr;  // PartPrep<T>[n_p]
    void *pfast = nullptr; // PartFast<T>[n_p]
    unsigned long long l_magic = 0;  // ceil(2^64 / n_l): p = umulhi(m, l_magic)
    void *Fl = nullptr;    // [n_m][4] marker force (x, y, z, unused)
    void *dFl = nullptr;   // [n_m][4] increment of the latest pass (passes > 1)

    // IBM tiles and the markers binned by (tile, face class): key = tile * 27 + class
    int nt[3] = {}, ntile = 0;
    int *key_count = nullptr, *key_start = nullptr, *mlist = nullptr, *key_scan_tmp = nullptr;
    // per tile, the spheres whose markers' stencils can reach it (null when a
    // sphere could reach one tile through two periodic images)
    int *pt_count = nullptr, *pt_start = nullptr, *pt_list = nullptr, *pt_scan_tmp = nullptr;
    // interpolation work lists: non-empty tiles at no periodic end (TMA-staged
    // persistent kernel; count on the device) and all tiles at a periodic end
    int *tma_list = nullptr, *tma_count = nullptr;
    int *tile_flag = nullptr, *tile_pos = nullptr, *tile_scan_tmp = nullptr;  // its scan
    // bank-bucketed spread: super-tiles of 2 x 2 x 1 tiles and their plans
    int nsuper = 0;
    int *sp_plan = nullptr;

    // bed / flying classification and saltation tracking (allocated on first
    // use): contact pairs, union-find parents, root marks, flags; per-sphere
    // tracker states and the scan that orders the events
    int *bed_pairs = nullptr;
    long long bed_cap = 0;
    int *bed_parent = nullptr;
    unsigned char *bed_root = nullptr, *bed_flags = nullptr;
    unsigned long long *bed_count = nullptr;
    unsigned char *trk_prev = nullptr, *trk_salt = nullptr, *trk_pend = nullptr;
    double *trk_dep_z = nullptr, *trk_t_imp = nullptr, *trk_u_imp = nullptr,
           *trk_om_imp = nullptr;
    int *trk_flag = nullptr, *trk_pos = nullptr, *trk_scan_tmp = nullptr;
    int trk_started = 0;
    int *edge_tiles = nullptr, n_edge = 0;
    std::vector<int> edge_host;  // the same list on the host (ascending)

    // device reductions: bit patterns of max |dF| and max slip
    unsigned long long *d_red = nullptr;  // [0..2] = max |dF| per component, [3] = residual (bits)
    // per tile, max |dF| per component over the markers binned in it (bits);
    // the spread bounds a tile's sums by the maxima of its 27 neighbours
    unsigned long long *tile_fmax = nullptr;  // [ntile][3]
    bool spread_global = false;  // bound by d_red instead (marker forces changed since)

    // contact history, double buffered; a pair is kept only by its lower id
    int *hcnt[2] = {}, *hpid[2] = {};
    double *huin[2] = {}, *hdlt[2] = {};
    unsigned char *wact[2] = {};
    double *wuin[2] = {}, *wdlt[2] = {};
    int hcur = 0;
    void *pairFT = nullptr;  // [12][n_p][6] pair force and torque, working precision
    int *ccnt = nullptr;   // contacts of every sphere
    int *clist = nullptr;  // [12][n_p] pairs owned by lower ids (id * 16 + slot)
    int *inc_cnt = nullptr;  // their number (returned to zero by the update)

    // cell list of the contact search: cells of edge >= 2R + skin, rebuilt
    // only when some particle has moved more than skin/2 since the last build
    // (device flag d_rebuild, set by the sub-step kernel)
    double skin = 0.0;
    int *d_rebuild = nullptr;
    float *xb = nullptr;  // FP32 positions at the last build
    CellGeom cg{};
    int cell_cap = 0;
    int *cell_count = nullptr, *cell_start = nullptr, *cell_sorted = nullptr;
    int *pcell = nullptr, *cell_scan_tmp = nullptr;
    int *nlist = nullptr, *ncnt = nullptr;  // neighbour list [ncap][n_p], counts
    int *nlo = nullptr;  // per sphere: neighbours with lower ids (they lead its list)
    int ncap = 0;
    // cooperative rebuild: grid size, per-block totals, barrier words
    int coop_grid = 0;
    int *coop_blocksum = nullptr;
    unsigned *coop_bar = nullptr;
    long long *d_pairs_n = nullptr;

    DemParams dp{};
    int dp_valid = 0;
    // adaptive collision model: the unit collision's damping and duration
    // for the restitution e_n they were calibrated on (0: none yet)
    double actm_e = 0.0, actm_beta = 0.0, actm_S = 0.0;
    // regularised delta of the IBM step (3 or 4 points) and, for the
    // 4-point kernel, the fixed-point spreading scratch [3][cells]
    int delta_kernel = 3;
    unsigned long long *acc4 = nullptr;
    // lubrication: per-sphere force of the last sub-step, [3][n_p]; the
    // neighbour list's extra reach it was last built with
    double *flub = nullptr;
    double lub_reach = 0.0;
    double cell_margin = 0.0;  // extra cell width reserved for that reach
    int *d_err = nullptr;

    // learned warm start: FP32 master weights and Adam moments (padded
    // layout), the BF16 image staged by the tensor-core kernels, partial
    // gradients of the training CTAs, and device scratch for a gradient and a loss
    void *mlp_pack = nullptr;
    float *mlp_w = nullptr, *mlp_m = nullptr, *mlp_v = nullptr;
    float *mlp_part = nullptr;
    int mlp_part_cap = 0;
    float *mlp_dev = nullptr;
    long long mlp_step = 0;
    int mlp_ready = 0;

    // host-resident grid staging (prs_ibm_opts.grid_where == PRS_HOST), and
    // the z-range of cells the markers can reach
    void *stage[6] = {};
    int *d_zr = nullptr;
    long long last_h2d = 0, last_d2h = 0;
    // copies of the host path run on their own streams (in and out), ordered
    // against the kernels by events: u, v, w in; fx, fy, fz in (or all six by
    // z-chunks); the spread's z-chunks out
    cudaStream_t copy_stream = nullptr, copy_out = nullptr;
    static constexpr int kHostChunks = 16;
    cudaEvent_t ev_start = nullptr, ev_uvw = nullptr, ev_f = nullptr;
    cudaEvent_t ev_chunk[kHostChunks] = {};
    cudaEvent_t ev_in[kHostChunks] = {};
    // an asynchronous host step's copies out may still run (ev_out_done marks
    // their end); the next synchronising call waits for them
    cudaEvent_t ev_out_done = nullptr;
    bool host_pending = false;

    // counters
    int last_passes = 0;
    double last_res = 0.0;
    mutable long long n_launch = 0;  // kernels launched by this context

    // optional per-phase CUDA-event timing (prs_set_profiling)
    int profiling = 0;
    // the DEM sub-step loop as a CUDA graph (prs_set_graphs): the executable
    // and what it was captured for
    int graphs = 1;
    cudaGraphExec_t dg_exec = nullptr;
    int dg_nsub = -1, dg_cur = -1, dg_hcur = -1;
    double dg_dt = 0.0;
    DemParams dg_dp{};
    const void *dg_flub = nullptr;
    cudaStream_t dg_stream = nullptr;
    long long dg_launches = 0;
    int dg_used = 0;  // the last prs_dem_step ran its sub-steps as the graph
    int dg_replays = 0;   // replays of the current graph
    int dg_wasted = 0;    // graphs in a row captured and never replayed
    struct Mark {
        int phase;
        cudaEvent_t a, b;
    };
    Mark *marks = nullptr;
    int n_marks = 0, cap_marks = 0;
    cudaEvent_t *pool = nullptr;
    int n_pool = 0, cap_pool = 0;
    int open_phase = -1;
    cudaEvent_t open_event = nullptr;
};

// phase timing helpers (no-ops unless profiling is on)
void phase_begin(Ctx &c, int phase);
void phase_end(Ctx &c);

void *ctx_alloc(Ctx &c, size_t bytes);
void ctx_free(Ctx &c, void *p);

// ------------------------------------------------------------------ IBM
template <typename T>
void ibm_prep(Ctx &c, cudaStream_t s);
// interpolation and forcing of one pass over the tiles of z-layers
// [tz_lo, tz_hi] (all tiles when tz_hi < tz_lo), then (sums) the
// per-particle loads
template <typename T>
void ibm_interp_force(Ctx &c, const T *u, const T *v, const T *w, int pass,
                      double inv_adt, int probe, cudaStream_t s, int tz_lo = 0,
                      int tz_hi = -1, bool sums = true);
// spread of one forcing pass over the tiles of z-layers [tz_lo, tz_hi]
// (all tiles when tz_hi < tz_lo)
bool spread_bank_ok(const Ctx &c);
size_t spread_plan_ints(const Ctx &c);
template <typename T>
void ibm_spread(Ctx &c, T *u, T *v, T *w, T *fx, T *fy, T *fz, int pass,
                double adt, cudaStream_t s, int tz_lo = 0, int tz_hi = -1);
void ibm_marker_bin(Ctx &c, cudaStream_t s);
// the 4-point kernel's interpolation and forcing (one pass) and spreading
template <typename T>
void ibm4_interp_force(Ctx &c, const T *u, const T *v, const T *w, int pass, double inv_adt,
                       int probe, cudaStream_t s);
template <typename T>
void ibm4_spread(Ctx &c, T *u, T *v, T *w, T *fx, T *fy, T *fz, int pass, double adt,
                 cudaStream_t s);
size_t ibm_smem_bytes(int precision, int same_off);
void ibm_unpack_forces(const Ctx &c, void *dst, cudaStream_t s);
// [lo, hi] z cells the stencils of any sphere can reach; synchronises
void particle_zrange(Ctx &c, int zr[2], cudaStream_t s);
// a bounded wait that runs out (prs_probe_wait)
void wait_probe(Ctx &c, long long polls);

// ------------------------------------------------------------------ warm-start network
int mlp_npad();                // padded parameter count (master / gradient layout)
int mlp_pack_elems();          // BF16 elements of the staged image
int mlp_pad_index(int q);      // padded index of natural parameter q
void mlp_pack(Ctx &c, cudaStream_t s);
// gradient (and, with adam, one optimiser step); returns -1 if out of memory
// (stride > 0: batch row i is row (start + i stride) mod n_total of the pairs)
int mlp_grad_launch(Ctx &c, const float *feats, const float *targets, long long n,
                    float *grad, float *loss, const MlpAdam *adam, cudaStream_t s,
                    long long n_total = 0, long long start = 0, long long stride = 0);
void mlp_forward_launch(Ctx &c, const float *feats, long long n, float *out, cudaStream_t s);
template <typename T>
void mlp_warm_launch(Ctx &c, double adt, cudaStream_t s);
template <typename T>
void mlp_features_launch(Ctx &c, double adt, float *feats, cudaStream_t s);
template <typename T>
void mlp_targets_launch(Ctx &c, double adt, const float *feats, float *targets,
                        cudaStream_t s);
template <typename T>
void ibm_particle_sums(Ctx &c, cudaStream_t s);

// ------------------------------------------------------------------ DEM
CellGeom make_cell_geom(const DemParams &dp, double cutoff);
void dem_cells_build(const Ctx &c, const CellGeom &cg, const double *x, cudaStream_t s,
                     const int *enable = nullptr);
// one sub-step; `last`: the call's final one, whose collision force is kept
void dem_substep(Ctx &c, double dt_p, bool last, cudaStream_t s);
int dem_rebuild_grid();

// ------------------------------------------------------------------ bed and saltation
// bed flags (c.bed_flags) and their count (c.bed_count) from the contact
// pairs in `pairs` (count in c.d_pairs_n, at most cap written)
void bed_classify(Ctx &c, const int *pairs, long long cap, cudaStream_t s);

// ------------------------------------------------------------------ fluid sub-step stand-in
// predictor of one velocity component with H = nu lap_h(u) (prs_predict)
void fluid_predict(Ctx &c, int comp, const void *u_in, void *u_out, void *H, double nu,
                   double dt, double alpha, double beta, cudaStream_t s);
// one tracked state at time t; events to out[0 .. cap), count in c.trk_pos[n_p]
void track_saltation(Ctx &c, double t, double h_r, double t_cir, prs_event *out,
                     long long cap, cudaStream_t s);
// cell list and neighbour list when the device flag asks for it (one
// cooperative launch)
void dem_rebuild(const Ctx &c, cudaStream_t s);
void dem_shadow(Ctx &c, cudaStream_t s);
void dem_forces_f2d(const Ctx &c, const float *src, double *dst, cudaStream_t s);
void dem_pairs(const Ctx &c, const CellGeom &cg, double cutoff, int *d_pairs,
               long long max_pairs, cudaStream_t s);

// ------------------------------------------------------------------ utilities
// returns the number of kernels launched; with `enable`, every kernel does
// nothing unless *enable is non-zero (a device-side condition)
int exclusive_scan(const int *in, int *out, int n, int *tmp, cudaStream_t s,
                   const int *enable = nullptr);
size_t exclusive_scan_tmp_ints(int n);

}  // namespace prs
