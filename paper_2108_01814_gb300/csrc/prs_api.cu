// C ABI of the GB300 particle-side hot path (declared in include/pr_sed.h):
// argument checks, memory management and the sequencing of the kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "prs_internal.cuh"

namespace prs {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void *ctx_alloc(Ctx &c, size_t bytes)
{
    if (bytes == 0)
        bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void *p = nullptr;
    if (c.have_alloc) {
        p = c.alloc.alloc(bytes, (void *)c.stream, c.alloc.user);
        if (p && ((uintptr_t)p & 255u)) {
            // vector loads and tensor maps need the alignment cudaMalloc gives
            c.alloc.free(p, (void *)c.stream, c.alloc.user);
            p = nullptr;
        }
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void ctx_free(Ctx &c, void *p)
{
    if (!p)
        return;
    if (c.have_alloc)
        c.alloc.free(p, (void *)c.stream, c.alloc.user);
    else
        cudaFree(p);
}

void phase_begin(Ctx &c, int phase)
{
    if (!c.profiling)
        return;
    if (c.n_pool == 0) {
        if (c.cap_pool == 0) {
            c.cap_pool = 64;
            c.pool = new cudaEvent_t[c.cap_pool];
        }
        cudaEventCreate(&c.pool[c.n_pool++]);
    }
    c.open_event = c.pool[--c.n_pool];
    c.open_phase = phase;
    cudaEventRecord(c.open_event, c.stream);
}

void phase_end(Ctx &c)
{
    if (!c.profiling || c.open_phase < 0)
        return;
    cudaEvent_t b;
    if (c.n_pool > 0)
        b = c.pool[--c.n_pool];
    else
        cudaEventCreate(&b);
    cudaEventRecord(b, c.stream);
    if (c.n_marks == c.cap_marks) {
        int cap = c.cap_marks ? 2 * c.cap_marks : 256;
        Ctx::Mark *m = new Ctx::Mark[cap];
        for (int i = 0; i < c.n_marks; i++)
            m[i] = c.marks[i];
        delete[] c.marks;
        c.marks = m;
        c.cap_marks = cap;
    }
    c.marks[c.n_marks++] = Ctx::Mark{c.open_phase, c.open_event, b};
    c.open_phase = -1;
}

static void pool_return(Ctx &c, cudaEvent_t e)
{
    if (c.n_pool == c.cap_pool) {
        int cap = c.cap_pool ? 2 * c.cap_pool : 64;
        cudaEvent_t *p = new cudaEvent_t[cap];
        for (int i = 0; i < c.n_pool; i++)
            p[i] = c.pool[i];
        delete[] c.pool;
        c.pool = p;
        c.cap_pool = cap;
    }
    c.pool[c.n_pool++] = e;
}

static void profile_clear(Ctx &c, double *ms, long long *cnt)
{
    for (int i = 0; i < c.n_marks; i++) {
        const Ctx::Mark &m = c.marks[i];
        if (ms || cnt) {
            float t = 0.f;
            cudaEventElapsedTime(&t, m.a, m.b);
            if (ms && m.phase >= 0 && m.phase < PRS_NPHASES)
                ms[m.phase] += t;
            if (cnt && m.phase >= 0 && m.phase < PRS_NPHASES)
                cnt[m.phase] += 1;
        }
        pool_return(c, m.a);
        pool_return(c, m.b);
    }
    c.n_marks = 0;
}

static void profile_destroy(Ctx &c)
{
    profile_clear(c, nullptr, nullptr);
    for (int i = 0; i < c.n_pool; i++)
        cudaEventDestroy(c.pool[i]);
    delete[] c.pool;
    delete[] c.marks;
    c.pool = nullptr;
    c.marks = nullptr;
    c.n_pool = c.cap_pool = 0;
}

}  // namespace prs

using namespace prs;

struct prs_ctx {
    Ctx c;
    std::vector<void *> owned;
};

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kNeighCap = 32;  // neighbour-list slots per sphere (2R + skin)

prs_status fail(prs_status st, const char *msg)
{
    set_error("%s", msg);
    return st;
}

prs_status cuda_check(const char *where)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s: %s", where, cudaGetErrorString(e));
        return PRS_ERR_CUDA;
    }
    return PRS_OK;
}

template <typename P>
bool alloc_into(prs_ctx *h, P *&ptr, size_t bytes)
{
    void *p = ctx_alloc(h->c, bytes);
    if (!p)
        return false;
    h->owned.push_back(p);
    ptr = (P *)p;
    return true;
}

size_t prec_bytes(const Ctx &c) { return c.precision == PRS_FP64 ? 8 : 4; }

cudaMemcpyKind kind_to_dev(int where)
{
    return where == PRS_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
}
cudaMemcpyKind kind_from_dev(int where)
{
    return where == PRS_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
}

prs_status latched_errors(Ctx &c)
{
    if (c.host_pending) {
        // copies out of an asynchronous host step
        c.host_pending = false;
        if (cudaStreamSynchronize(c.copy_out) != cudaSuccess)
            return cuda_check("synchronise (host copies)");
    }
    int err = 0;
    if (cudaMemcpyAsync(&err, c.d_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c.stream) != cudaSuccess)
        return cuda_check("synchronise");
    if (err & ERRB_CONTACT_OVERFLOW)
        return fail(PRS_ERR_CONTACT_OVERFLOW, "a sphere had more than 12 particle contacts");
    if (err & ERRB_NONFINITE)
        return fail(PRS_ERR_NONFINITE, "non-finite particle state");
    if (err & ERRB_CAPACITY)
        return fail(PRS_ERR_CAPACITY, "internal buffer capacity exceeded");
    if (err & ERRB_BARRIER_TIMEOUT)
        return fail(PRS_ERR_TIMEOUT, "a grid barrier of the cell-list rebuild ran out");
    if (err & ERRB_MLP_TIMEOUT)
        return fail(PRS_ERR_TIMEOUT, "a tensor-core wait of the warm-start network ran out");
    if (err & ERRB_TMA_TIMEOUT)
        return fail(PRS_ERR_TIMEOUT, "a wait on the interpolation's tensor copies ran out");
    return PRS_OK;
}

// marker template: thin-shell count rule and golden-angle spiral
int marker_count_rule(double R, double h)
{
    double q = R / h;
    return (int)std::floor(kPi / 3.0 * (12.0 * q * q + 1.0) + 0.5);
}

void spiral(int n_l, std::vector<double> &t)
{
    t.assign(3 * (size_t)n_l, 0.0);
    const double golden = kPi * (3.0 - std::sqrt(5.0));
    for (int l = 0; l < n_l; l++) {
        double z = 1.0 - (2.0 * l + 1.0) / (double)n_l;
        double rho = std::sqrt(1.0 - z * z);
        double ang = (double)l * golden;
        t[l] = rho * std::cos(ang);
        t[n_l + l] = rho * std::sin(ang);
        t[2 * n_l + l] = z;
    }
}

// spring-dashpot constants calibrated on T_c and the restitution
// coefficients; inertia (rho_p - rho_f) V_p of the rigid-body Eq. 7
// Adaptive collision time model, scaled: a contact m z'' + d z' + k z^(3/2)
// = 0 entered at speed v becomes, with z = v tau x and t = tau s,
// tau = (m / (k sqrt(v)))^(2/5), the unit collision x'' + beta x' +
// x^(3/2) = 0, x(0) = 0, x'(0) = 1, beta = d tau / m. Its duration and exit
// speed depend on beta alone. Fourth-order Runge-Kutta with a fixed step;
// the exit x = 0 is found by Newton steps on the length of a last partial
// Runge-Kutta step.
static void unit_rk4(double beta, double h, double &x, double &v)
{
    auto acc = [beta](double xx, double vv) { return -beta * vv - (xx > 0.0 ? xx * std::sqrt(xx) : 0.0); };
    const double a1 = acc(x, v);
    const double x2 = x + 0.5 * h * v, v2 = v + 0.5 * h * a1;
    const double a2 = acc(x2, v2);
    const double x3 = x + 0.5 * h * v2, v3 = v + 0.5 * h * a2;
    const double a3 = acc(x3, v3);
    const double x4 = x + h * v3, v4 = v + h * a3;
    const double a4 = acc(x4, v4);
    x += h / 6.0 * (v + 2.0 * v2 + 2.0 * v3 + v4);
    v += h / 6.0 * (a1 + 2.0 * a2 + 2.0 * a3 + a4);
}

static void unit_collision(double beta, double &dur, double &rest)
{
    const double h = 5e-6;
    double x = 0.0, v = 1.0, t = 0.0;
    for (long k = 0; k < 20000000; k++) {
        double xn = x, vn = v;
        unit_rk4(beta, h, xn, vn);
        if (k > 0 && xn <= 0.0) {
            double s = h * x / (x - xn);
            double xs = x, vs = v;
            for (int it = 0; it < 40; it++) {
                xs = x;
                vs = v;
                unit_rk4(beta, s, xs, vs);
                const double ds = xs / vs;
                s -= ds;
                if (std::fabs(ds) < 1e-17)
                    break;
            }
            xs = x;
            vs = v;
            unit_rk4(beta, s, xs, vs);
            dur = t + s;
            rest = -vs;
            return;
        }
        x = xn;
        v = vn;
        t = (double)(k + 1) * h;  // not a running sum: no rounding drift
    }
    dur = t;
    rest = 0.0;
}

// beta with exit speed e_n (it falls as beta grows): bracketing, then the
// Illinois variant of regula falsi on e(beta) - e_n
static void actm_calibrate(double e_n, double &beta, double &dur)
{
    double lo = 0.0, hi = 0.5, d_, e_lo, e_hi;
    unit_collision(lo, d_, e_lo);
    unit_collision(hi, d_, e_hi);
    while (e_hi > e_n && hi < 100.0) {
        lo = hi;
        e_lo = e_hi;
        hi *= 2.0;
        unit_collision(hi, d_, e_hi);
    }
    double f_lo = e_lo - e_n, f_hi = e_hi - e_n;
    int side = 0;
    double b = lo;
    for (int it = 0; it < 200; it++) {
        b = (lo * f_hi - hi * f_lo) / (f_hi - f_lo);
        double eb;
        unit_collision(b, d_, eb);
        const double fb = eb - e_n;
        if (fb == 0.0 || std::fabs(hi - lo) < 1e-15 * std::max(1.0, std::fabs(b)))
            break;
        if ((fb > 0.0) == (f_lo > 0.0)) {
            lo = b;
            f_lo = fb;
            if (side == -1)
                f_hi *= 0.5;
            side = -1;
        } else {
            hi = b;
            f_hi = fb;
            if (side == 1)
                f_lo *= 0.5;
            side = 1;
        }
        if (std::fabs(fb) < 1e-15)
            break;
    }
    beta = b;
    double e_;
    unit_collision(beta, dur, e_);
}

// small-gap Stokes amplification of the normal resistance (eps = gap / R):
// two equal spheres (Jeffrey 1982), a sphere and a wall (Cox & Brenner 1967)
static double lub_lambda(bool wall, double eps)
{
    const double l = std::log(eps);
    return wall ? 1.0 / eps - 0.2 * l - eps * l / 21.0 + 0.9713
                : 0.5 / eps - 0.45 * l - 3.0 * eps * l / 56.0 + 1.346;
}

void dem_constants(Ctx &c, const prs_dem_opts &o, DemParams &d)
{
    const double R = c.R;
    double Vp = 4.0 / 3.0 * kPi * R * R * R;
    d.R = R;
    d.m = (c.rho_p - c.rho_f) * Vp;
    d.J = 0.4 * d.m * R * R;
    double ln_n = std::log(o.e_n), ln_t = std::log(o.e_t);
    double me[2] = {0.5 * d.m, d.m};
    double *kn[2] = {&d.kn_pp, &d.kn_pw}, *dn[2] = {&d.dn_pp, &d.dn_pw};
    double *kt[2] = {&d.kt_pp, &d.kt_pw}, *dtg[2] = {&d.dt_pp, &d.dt_pw};
    for (int s = 0; s < 2; s++) {
        *kn[s] = me[s] * (kPi * kPi + ln_n * ln_n) / (o.T_c * o.T_c);
        *dn[s] = -2.0 * me[s] * ln_n / o.T_c;
        *kt[s] = (2.0 / 7.0) * me[s] * (kPi * kPi + ln_t * ln_t) / (o.T_c * o.T_c);
        *dtg[s] = -(2.0 / 7.0) * 2.0 * me[s] * ln_t / o.T_c;
    }
    d.mu = o.mu;
    d.clip_n = o.clip_normal ? 1 : 0;
    for (int a = 0; a < 3; a++) {
        d.g[a] = o.g[a];
        d.L[a] = c.g.n[a] * c.g.h;
        d.periodic[a] = c.g.periodic[a];
    }
    d.model = o.model == PRS_CONTACT_ACTM ? 1 : 0;
    if (d.model) {
        if (c.actm_e != o.e_n) {
            actm_calibrate(o.e_n, c.actm_beta, c.actm_S);
            c.actm_e = o.e_n;
        }
        const double tau = o.T_c / c.actm_S;
        for (int s = 0; s < 2; s++) {
            *kn[s] = me[s] / (tau * tau * std::sqrt(tau));
            *dn[s] = c.actm_beta * me[s] / tau;
        }
        const double gm = std::sqrt(o.g[0] * o.g[0] + o.g[1] * o.g[1] + o.g[2] * o.g[2]);
        d.u_min = o.u_min > 0.0 ? o.u_min : (gm > 0.0 ? gm * o.T_c : 1e-3 * R / o.T_c);
    }
    d.mu_f = o.mu_f > 0.0 ? o.mu_f : 0.0;
    d.eps_d_pp = o.eps_d_pp > 0.0 ? o.eps_d_pp : 0.05;
    d.eps_d_pw = o.eps_d_pw > 0.0 ? o.eps_d_pw : 0.05;
    d.eps_s = o.eps_s > 0.0 ? o.eps_s : 0.001;
    d.lub_pp = 6.0 * kPi * d.mu_f * R * 0.5;
    d.lub_pw = 6.0 * kPi * d.mu_f * R;
    d.lam_d_pp = lub_lambda(false, d.eps_d_pp);
    d.lam_d_pw = lub_lambda(true, d.eps_d_pw);
}

// the next sub-step rebuilds the contact cell list
void force_rebuild(Ctx &c)
{
    static const int one = 1;
    cudaMemcpyAsync(c.d_rebuild, &one, sizeof(int), cudaMemcpyHostToDevice, c.stream);
}

void geometry_only(const Ctx &c, DemParams &d)
{
    d.R = c.R;
    for (int a = 0; a < 3; a++) {
        d.L[a] = c.g.n[a] * c.g.h;
        d.periodic[a] = c.g.periodic[a];
    }
}

}  // namespace

namespace {

// Host-resident fields (prs_ibm_opts.grid_where == PRS_HOST). Copies in
// run on the context's copy stream, copies out on a second one, so the two
// directions overlap; events order them against the kernels.
// - A step of one forcing pass on a z-bounded grid runs as a pipeline over
//   z-chunks of tile layers (pipelined_pass): each chunk's six fields come
//   in, chunk k is interpolated once chunks k and k + 1 are in, chunk k - 1
//   is spread right after it and goes back while later chunks come in.
// - Otherwise u, v, w come in first, then fx, fy, fz; the kernels wait for
//   u, v, w before the first interpolation and for the forces before the
//   first spread. The last pass's spread runs in z-chunks whose planes go
//   back while the next chunk is spread.
// Tiles write only their own cells, so a chunk's planes are final once its
// tiles are spread.
struct HostPipe {
    void *host[6];
    void *dev[6];
    int zlo = 0, zhi = 0;  // planes copied in and out, [zlo, zhi)
    size_t plane = 0;      // bytes per z-plane
    bool uvw_in = false, f_in = false, out_done = false;
    int chunks = 0;        // > 0: pipelined over this many z-chunks
    int tz_lo = 0, layers = 0;  // tile layers [tz_lo, tz_lo + layers) hold the slab
    int layer_lo(int k, int K) const { return tz_lo + layers * k / K; }
    int layer_hi(int k, int K) const { return tz_lo + layers * (k + 1) / K - 1; }
    int plane_lo(int k, int K) const { return std::max(zlo, layer_lo(k, K) * kTileZ); }
    int plane_hi(int k, int K) const { return std::min(zhi, (layer_hi(k, K) + 1) * kTileZ); }
};

void host_copy_planes(const HostPipe &hp, int z0, int z1, cudaMemcpyKind kind, int i0, int i1,
                      cudaStream_t cs)
{
    if (z1 <= z0)
        return;
    const size_t off = hp.plane * (size_t)z0, len = hp.plane * (size_t)(z1 - z0);
    for (int i = i0; i < i1; i++) {
        const bool in = kind == cudaMemcpyHostToDevice;
        cudaMemcpyAsync((char *)(in ? hp.dev[i] : hp.host[i]) + off,
                        (const char *)(in ? hp.host[i] : hp.dev[i]) + off, len, kind, cs);
    }
}

// spread of tile layers [a, b], then its planes back to the host on the
// copy-out stream (event slot k)
template <typename T>
void spread_chunk_out(Ctx &c, const HostPipe &hp, T *u, T *v, T *w, T *fx, T *fy, T *fz,
                      int pass, double adt, cudaStream_t s, int a, int b, int k)
{
    ibm_spread<T>(c, u, v, w, fx, fy, fz, pass, adt, s, a, b);
    cudaEventRecord(c.ev_chunk[k], s);
    cudaStreamWaitEvent(c.copy_out, c.ev_chunk[k], 0);
    host_copy_planes(hp, std::max(hp.zlo, a * kTileZ), std::min(hp.zhi, (b + 1) * kTileZ),
                     cudaMemcpyDeviceToHost, 0, 6, c.copy_out);
}

template <typename T>
void spread_and_copy_out(Ctx &c, HostPipe &hp, T *u, T *v, T *w, T *fx, T *fy, T *fz,
                         int pass, double adt, cudaStream_t s)
{
    const int tz_lo = hp.zlo / kTileZ, tz_hi = (hp.zhi - 1) / kTileZ;
    const int layers = tz_hi - tz_lo + 1;
    const int K = std::min(Ctx::kHostChunks, layers);
    for (int k = 0; k < K; k++) {
        const int a = tz_lo + layers * k / K, b = tz_lo + layers * (k + 1) / K - 1;
        spread_chunk_out<T>(c, hp, u, v, w, fx, fy, fz, pass, adt, s, a, b, k);
    }
    hp.out_done = true;
}

// One forcing pass over the z-chunks of a host step (the copies in were
// issued chunk by chunk, event ev_in[k] after chunk k). The interpolation
// of chunk k reads a halo of at most two planes into chunk k + 1; the
// spread of chunk k - 1 takes markers binned up to two cells into chunk k,
// whose forces and per-tile bounds are then final, and it runs after the
// interpolation of chunk k has read the planes it overwrites.
template <typename T>
void pipelined_pass(Ctx &c, HostPipe &hp, T *u, T *v, T *w, T *fx, T *fy, T *fz,
                    double inv_adt, double adt, cudaStream_t s)
{
    const int K = hp.chunks;
    for (int k = 0; k < K; k++) {
        cudaStreamWaitEvent(s, c.ev_in[std::min(k + 1, K - 1)], 0);
        ibm_interp_force<T>(c, u, v, w, 0, inv_adt, 0, s, hp.layer_lo(k, K), hp.layer_hi(k, K),
                            false);
        if (k > 0)
            spread_chunk_out<T>(c, hp, u, v, w, fx, fy, fz, 0, adt, s, hp.layer_lo(k - 1, K),
                                hp.layer_hi(k - 1, K), k - 1);
    }
    phase_begin(c, PRS_PHASE_INTERP);
    ibm_particle_sums<T>(c, s);
    phase_end(c);
    spread_chunk_out<T>(c, hp, u, v, w, fx, fy, fz, 0, adt, s, hp.layer_lo(K - 1, K),
                        hp.layer_hi(K - 1, K), K - 1);
    hp.out_done = true;
}

// the maxima the interpolation accumulates: global words and per tile
void reset_maxima(Ctx &c, cudaStream_t s)
{
    cudaMemsetAsync(c.d_red, 0, kRedWords * sizeof(unsigned long long), s);
    if (c.tile_fmax)
        cudaMemsetAsync(c.tile_fmax, 0, 3 * sizeof(unsigned long long) * (size_t)c.ntile, s);
}

template <typename T>
prs_status ibm_step_t(prs_ctx *h, T *u, T *v, T *w, T *fx, T *fy, T *fz, double dt,
                             double alpha, const prs_ibm_opts &o, float *feats = nullptr,
                             float *targets = nullptr, HostPipe *hp = nullptr)
{
    Ctx &c = h->c;
    cudaStream_t s = c.stream;
    auto need_uvw = [&]() {
        if (hp && !hp->uvw_in) {
            cudaStreamWaitEvent(s, c.ev_uvw, 0);
            hp->uvw_in = true;
        }
    };
    auto need_f = [&]() {
        if (hp && !hp->f_in) {
            cudaStreamWaitEvent(s, c.ev_f, 0);
            hp->f_in = true;
        }
    };
    const double adt = alpha * dt;
    const double inv_adt = 1.0 / adt;
    phase_begin(c, PRS_PHASE_IBM_BIN);
    ibm_prep<T>(c, s);
    ibm_marker_bin(c, s);
    phase_end(c);
    int passes = 0;
    double res = 0.0;
    auto read_res = [&]() -> double {
        unsigned long long b[kRedWords];
        cudaMemcpyAsync(b, c.d_red, sizeof(b), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        if (c.precision == PRS_FP64) {
            double d;
            std::memcpy(&d, &b[kRedRes], sizeof(d));
            return d;
        }
        unsigned u32 = (unsigned)b[kRedRes];
        float f;
        std::memcpy(&f, &u32, sizeof(f));
        return (double)f;
    };
    bool converged = false;
    if (hp && hp->chunks > 0) {
        // one pass, pipelined with the host copies
        reset_maxima(c, s);
        pipelined_pass<T>(c, *hp, u, v, w, fx, fy, fz, inv_adt, adt, s);
        passes = 1;
    }
    for (; !(hp && hp->chunks > 0);) {
        if (o.tol > 0.0) {
            cudaMemsetAsync(c.d_red, 0, kRedWords * sizeof(unsigned long long), s);
            need_uvw();
            ibm_interp_force<T>(c, u, v, w, passes, inv_adt, 1, s);
            res = read_res();
            if (res < o.tol) {
                converged = true;
                break;
            }
        }
        if (passes >= o.n_mdf_max)
            break;
        reset_maxima(c, s);
        need_uvw();
        ibm_interp_force<T>(c, u, v, w, passes, inv_adt, 0, s);
        if (passes == 0 && feats)
            mlp_features_launch<T>(c, adt, feats, s);
        if (passes == 0 && o.learned) {
            // first increment += network output / (alpha dt); the sums and
            // the spread's force bound follow the new F_l
            phase_begin(c, PRS_PHASE_MLP);
            mlp_warm_launch<T>(c, adt, s);
            phase_end(c);
            phase_begin(c, PRS_PHASE_INTERP);
            ibm_particle_sums<T>(c, s);
            phase_end(c);
        }
        need_f();
        // the network changed the marker forces after the per-tile maxima
        // were taken; its kernel updated the global ones
        c.spread_global = passes == 0 && o.learned;
        if (hp && o.tol <= 0.0 && passes + 1 >= o.n_mdf_max && hp->zhi > hp->zlo)
            spread_and_copy_out<T>(c, *hp, u, v, w, fx, fy, fz, passes, adt, s);
        else
            ibm_spread<T>(c, u, v, w, fx, fy, fz, passes, adt, s);
        c.spread_global = false;
        passes++;
        if (o.tol <= 0.0 && passes >= o.n_mdf_max)
            break;
    }
    if (o.tol <= 0.0) {
        if (o.final_residual) {
            cudaMemsetAsync(c.d_red, 0, kRedWords * sizeof(unsigned long long), s);
            ibm_interp_force<T>(c, u, v, w, passes, inv_adt, 1, s);
        }
        res = -1.0;  // read lazily by prs_get_stats
    }
    if (targets)
        mlp_targets_launch<T>(c, adt, feats, targets, s);
    c.last_passes = passes;
    c.last_res = res;
    prs_status st = cuda_check("prs_ibm_step");
    if (st)
        return st;
    if (o.tol > 0.0 && !converged)
        return fail(PRS_WARN_NOT_CONVERGED, "prs_ibm_step: forcing passes ran out");
    return PRS_OK;
}

}  // namespace

extern "C" {

const char *prs_last_error_string(void) { return g_err; }

prs_status prs_create_grid(int nx, int ny, int nz, double h, const int periodic[3],
                           const double *offset, int precision, const prs_allocator *alloc,
                           void *stream, prs_ctx **out)
{
    if (!out)
        return fail(PRS_ERR_ARG, "prs_create_grid: out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || !(h > 0.0) || !periodic)
        return fail(PRS_ERR_ARG, "prs_create_grid: sizes and spacing must be positive");
    if ((long long)nx * ny * nz > (1LL << 40))
        return fail(PRS_ERR_ARG, "prs_create_grid: grid too large");
    if (precision != PRS_FP64 && precision != PRS_FP32)
        return fail(PRS_ERR_ARG, "prs_create_grid: precision must be PRS_FP64 or PRS_FP32");
    if (alloc && (!alloc->alloc || !alloc->free))
        return fail(PRS_ERR_ARG, "prs_create_grid: allocator needs alloc and free");
    prs_ctx *hnd = new (std::nothrow) prs_ctx();
    if (!hnd)
        return fail(PRS_ERR_OOM, "prs_create_grid: host allocation failed");
    Ctx &c = hnd->c;
    c.g.n[0] = nx;
    c.g.n[1] = ny;
    c.g.n[2] = nz;
    c.g.h = h;
    for (int a = 0; a < 3; a++)
        c.g.periodic[a] = periodic[a] ? 1 : 0;
    for (int i = 0; i < 9; i++) {
        double o = offset ? offset[i] : 0.5;
        if (!(o >= 0.0 && o < 1.0)) {
            delete hnd;
            return fail(PRS_ERR_ARG, "prs_create_grid: offsets must lie in [0, 1)");
        }
        c.g.off[i] = o;
    }
    c.g.same_off = 1;
    for (int cc = 1; cc < 3; cc++)
        for (int a = 0; a < 3; a++)
            if (c.g.off[cc * 3 + a] != c.g.off[a])
                c.g.same_off = 0;
    c.precision = precision;
    c.have_alloc = alloc ? 1 : 0;
    if (alloc)
        c.alloc = *alloc;
    c.stream = (cudaStream_t)stream;
    const int te[3] = {kTileX, kTileY, kTileZ};
    for (int a = 0; a < 3; a++)
        c.nt[a] = (c.g.n[a] + te[a] - 1) / te[a];
    c.ntile = c.nt[0] * c.nt[1] * c.nt[2];
    c.nsuper = ((c.nt[0] + 1) / 2) * ((c.nt[1] + 1) / 2) * c.nt[2];
    if (!alloc_into(hnd, c.d_err, sizeof(int)) || !alloc_into(hnd, c.d_zr, 2 * sizeof(int)) ||
        !alloc_into(hnd, c.d_red, kRedWords * sizeof(unsigned long long))) {
        prs_destroy(hnd);
        return fail(PRS_ERR_OOM, "prs_create_grid: device allocation failed");
    }
    cudaMemsetAsync(c.d_err, 0, sizeof(int), c.stream);
    cudaMemsetAsync(c.d_red, 0, kRedWords * sizeof(unsigned long long), c.stream);
    prs_status st = cuda_check("prs_create_grid");
    if (st) {
        prs_destroy(hnd);
        return st;
    }
    *out = hnd;
    return PRS_OK;
}

prs_status prs_create_particles(prs_ctx *h, int n_p, double R, double rho_p, double rho_f,
                                int n_markers)
{
    if (!h)
        return fail(PRS_ERR_ARG, "prs_create_particles: NULL context");
    Ctx &c = h->c;
    if (c.n_p)
        return fail(PRS_ERR_STATE, "prs_create_particles: particles already created");
    if (n_p < 1 || !(R > 0.0) || !(rho_p > rho_f) || rho_f < 0.0 || n_markers < 0)
        return fail(PRS_ERR_ARG,
                    "prs_create_particles: need n_p >= 1, R > 0, rho_p > rho_f >= 0");
    for (int a = 0; a < 3; a++) {
        double L = c.g.n[a] * c.g.h;
        if (L < 2.0 * R)
            return fail(PRS_ERR_ARG, "prs_create_particles: domain narrower than a sphere");
        if (c.g.periodic[a] && c.g.n[a] < (int)std::ceil(R / c.g.h) + 4)
            return fail(PRS_ERR_ARG,
                        "prs_create_particles: periodic axis shorter than R/h + 4 cells");
    }
    const int n_l = n_markers ? n_markers : marker_count_rule(R, c.g.h);
    if (n_l < 1 || (long long)n_p * n_l > (1LL << 31) - 1)
        return fail(PRS_ERR_ARG, "prs_create_particles: marker count out of range");
    c.n_p = n_p;
    c.R = R;
    c.rho_p = rho_p;
    c.rho_f = rho_f;
    c.n_l = n_l;
    c.dV = kPi * c.g.h * (12.0 * R * R + c.g.h * c.g.h) / (3.0 * (double)n_l);
    if ((long long)c.ntile * 27 >= (1LL << 31) - 1) {
        c.n_p = 0;
        return fail(PRS_ERR_ARG, "prs_create_particles: grid has too many tiles");
    }
    const size_t pb = prec_bytes(c);
    const size_t n_m = (size_t)n_p * n_l;
    const size_t vec = 3 * sizeof(double) * (size_t)n_p;

    DemParams geo{};
    geometry_only(c, geo);
    c.skin = 0.5 * c.g.h;
    // cells reserve 0.1 R beyond 2R + skin for the lubrication range
    c.cell_margin = 0.1 * R;
    c.cg = make_cell_geom(geo, 2.0 * R + c.skin + c.cell_margin);
    c.cell_cap = c.cg.nc[0] * c.cg.nc[1] * c.cg.nc[2];
    const size_t prep_bytes = c.precision == PRS_FP64 ? sizeof(PartPrep<double>)
                                                      : sizeof(PartPrep<float>);
    bool ok = true;
    for (int b = 0; b < 2; b++) {
        ok = ok && alloc_into(h, c.x[b], vec) && alloc_into(h, c.u[b], vec) &&
             alloc_into(h, c.om[b], vec) && alloc_into(h, c.xf[b], vec / 2) &&
             alloc_into(h, c.xl[b], vec / 2) &&
             alloc_into(h, c.uf[b], vec / 2) && alloc_into(h, c.omf[b], vec / 2);
        ok = ok && alloc_into(h, c.hcnt[b], sizeof(int) * n_p) &&
             alloc_into(h, c.hpid[b], sizeof(int) * PRS_MAX_CONTACTS * n_p) &&
             alloc_into(h, c.huin[b], sizeof(double) * PRS_MAX_CONTACTS * n_p) &&
             alloc_into(h, c.hdlt[b], sizeof(double) * 3 * PRS_MAX_CONTACTS * n_p) &&
             alloc_into(h, c.wact[b], PRS_MAX_WALLS * (size_t)n_p) &&
             alloc_into(h, c.wuin[b], sizeof(double) * PRS_MAX_WALLS * n_p) &&
             alloc_into(h, c.wdlt[b], sizeof(double) * 3 * PRS_MAX_WALLS * n_p);
    }
    ok = ok && alloc_into(h, c.pairFT, 6 * PRS_MAX_CONTACTS * pb * n_p) &&
         alloc_into(h, c.ccnt, sizeof(int) * n_p) &&
         alloc_into(h, c.clist, sizeof(int) * PRS_MAX_CONTACTS * n_p) &&
         alloc_into(h, c.inc_cnt, sizeof(int) * n_p);
    ok = ok && alloc_into(h, c.Fh, vec) && alloc_into(h, c.Th, vec) &&
         alloc_into(h, c.Fc, vec) && alloc_into(h, c.Tc, vec);
    if (c.precision == PRS_FP32)
        ok = ok && alloc_into(h, c.Fhf, vec / 2) && alloc_into(h, c.Thf, vec / 2) &&
             alloc_into(h, c.Fcf, vec / 2) && alloc_into(h, c.Tcf, vec / 2);
    ok = ok && alloc_into(h, c.t64, 3 * sizeof(double) * n_l) &&
         alloc_into(h, c.t32, 3 * sizeof(float) * n_l) &&
         alloc_into(h, c.tR, 3 * pb * n_l) && alloc_into(h, c.rR, 3 * pb * n_l);
    const size_t fast_bytes = c.precision == PRS_FP64 ? sizeof(PartFast<double>)
                                                      : sizeof(PartFast<float>);
    ok = ok && alloc_into(h, c.prep, prep_bytes * n_p) && alloc_into(h, c.Fl, 4 * pb * n_m) &&
         alloc_into(h, c.pfast, fast_bytes * n_p);
    c.l_magic = ~0ULL / (unsigned long long)n_l + 1ULL;
    const int nkeys = c.ntile * 27;
    ok = ok && alloc_into(h, c.key_count, sizeof(int) * nkeys) &&
         alloc_into(h, c.key_start, sizeof(int) * (nkeys + 1)) &&
         alloc_into(h, c.mlist, sizeof(int) * (n_m + 4)) &&  // + 4: 16-byte copies
         alloc_into(h, c.key_scan_tmp, sizeof(int) * exclusive_scan_tmp_ints(nkeys));
    if (ok && spread_bank_ok(c))
        ok = alloc_into(h, c.sp_plan, sizeof(int) * spread_plan_ints(c));
    {
        // tiles a sphere's stencils can reach, per axis (bins within R/h of
        // the centre, plus W); lists only when no periodic axis could wrap
        // onto the same tile
        const int W = c.g.same_off ? 1 : 2;
        const int te[3] = {kTileX, kTileY, kTileZ};
        long long per_p = 1;
        bool lists = true;
        for (int a = 0; a < 3; a++) {
            const int span = (int)std::ceil(2.0 * R / c.g.h) + 2 + 2 * W;
            const int tiles = span / te[a] + 2;
            per_p *= tiles;
            if (c.g.periodic[a] && tiles >= c.nt[a])
                lists = false;
        }
        if (ok && lists && per_p * n_p < 2147483647LL) {
            ok = alloc_into(h, c.pt_count, sizeof(int) * (c.ntile + 1)) &&
                 alloc_into(h, c.pt_start, sizeof(int) * (c.ntile + 1)) &&
                 alloc_into(h, c.pt_list, sizeof(int) * per_p * n_p) &&
                 alloc_into(h, c.pt_scan_tmp,
                            sizeof(int) * exclusive_scan_tmp_ints(c.ntile + 1));
        }
    }
    {
        // interpolation work lists: tiles at a periodic end are static
        std::vector<int> edge;
        for (int t = 0; t < c.ntile; t++) {
            const int tc[3] = {t % c.nt[0], (t / c.nt[0]) % c.nt[1], t / (c.nt[0] * c.nt[1])};
            bool e = false;
            for (int a = 0; a < 3; a++)
                e = e || (c.g.periodic[a] && (tc[a] == 0 || tc[a] == c.nt[a] - 1));
            if (e)
                edge.push_back(t);
        }
        c.n_edge = (int)edge.size();
        c.edge_host = edge;
        ok = ok && alloc_into(h, c.tma_list, sizeof(int) * c.ntile) &&
             alloc_into(h, c.tile_fmax, sizeof(unsigned long long) * 3 * (size_t)c.ntile) &&
             alloc_into(h, c.tma_count, sizeof(int)) &&
             alloc_into(h, c.tile_flag, sizeof(int) * (c.ntile + 1)) &&
             alloc_into(h, c.tile_pos, sizeof(int) * (c.ntile + 1)) &&
             alloc_into(h, c.tile_scan_tmp,
                        sizeof(int) * exclusive_scan_tmp_ints(c.ntile + 1)) &&
             (edge.empty() || alloc_into(h, c.edge_tiles, sizeof(int) * edge.size()));
        if (ok && !edge.empty())
            cudaMemcpy(c.edge_tiles, edge.data(), sizeof(int) * edge.size(),
                       cudaMemcpyHostToDevice);
    }
    ok = ok && alloc_into(h, c.cell_count, sizeof(int) * c.cell_cap) &&
         alloc_into(h, c.cell_start, sizeof(int) * (c.cell_cap + 1)) &&
         alloc_into(h, c.cell_sorted, sizeof(int) * n_p) &&
         alloc_into(h, c.pcell, sizeof(int) * n_p) &&
         alloc_into(h, c.cell_scan_tmp, sizeof(int) * exclusive_scan_tmp_ints(c.cell_cap)) &&
         alloc_into(h, c.d_pairs_n, sizeof(long long)) &&
         alloc_into(h, c.d_rebuild, sizeof(int)) && alloc_into(h, c.xb, vec / 2);
    c.ncap = kNeighCap;
    ok = ok && alloc_into(h, c.nlist, sizeof(int) * (size_t)c.ncap * n_p) &&
         alloc_into(h, c.ncnt, sizeof(int) * n_p) && alloc_into(h, c.nlo, sizeof(int) * n_p);
    c.coop_grid = dem_rebuild_grid();
    ok = ok && alloc_into(h, c.coop_blocksum, sizeof(int) * (size_t)c.coop_grid) &&
         alloc_into(h, c.coop_bar, 2 * sizeof(unsigned));
    if (!ok) {
        c.n_p = 0;
        return fail(PRS_ERR_OOM, "prs_create_particles: device allocation failed");
    }
    cudaStream_t s = c.stream;
    for (int b = 0; b < 2; b++) {
        cudaMemsetAsync(c.x[b], 0, vec, s);
        cudaMemsetAsync(c.u[b], 0, vec, s);
        cudaMemsetAsync(c.om[b], 0, vec, s);
        cudaMemsetAsync(c.hcnt[b], 0, sizeof(int) * n_p, s);
        cudaMemsetAsync(c.wact[b], 0, PRS_MAX_WALLS * (size_t)n_p, s);
    }
    for (double *p : {c.Fh, c.Th, c.Fc, c.Tc})
        cudaMemsetAsync(p, 0, vec, s);
    for (float *p : {c.Fhf, c.Thf, c.Fcf, c.Tcf})
        if (p)
            cudaMemsetAsync(p, 0, vec / 2, s);
    cudaMemsetAsync(c.ccnt, 0, sizeof(int) * n_p, s);
    cudaMemsetAsync(c.ncnt, 0, sizeof(int) * n_p, s);
    cudaMemsetAsync(c.nlo, 0, sizeof(int) * n_p, s);
    cudaMemsetAsync(c.inc_cnt, 0, sizeof(int) * n_p, s);
    cudaMemsetAsync(c.Fl, 0, 4 * pb * n_m, s);
    cudaMemsetAsync(c.key_count, 0, sizeof(int) * nkeys, s);
    if (c.pt_count)
        cudaMemsetAsync(c.pt_count, 0, sizeof(int) * (c.ntile + 1), s);
    cudaMemsetAsync(c.cell_count, 0, sizeof(int) * c.cell_cap, s);
    cudaMemsetAsync(c.coop_bar, 0, 2 * sizeof(unsigned), s);
    {
        const int one = 1;
        cudaMemcpy(c.d_rebuild, &one, sizeof(int), cudaMemcpyHostToDevice);
    }

    // template: unit vectors, R/h t and R t in the marker precision
    std::vector<double> t;
    spiral(n_l, t);
    std::vector<double> tr(3 * (size_t)n_l), rr(3 * (size_t)n_l);
    for (size_t i = 0; i < t.size(); i++) {
        tr[i] = (R / c.g.h) * t[i];
        rr[i] = R * t[i];
    }
    cudaMemcpy(c.t64, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice);
    {
        std::vector<float> t32(t.begin(), t.end());
        cudaMemcpy(c.t32, t32.data(), sizeof(float) * t32.size(), cudaMemcpyHostToDevice);
    }
    if (c.precision == PRS_FP64) {
        cudaMemcpy(c.tR, tr.data(), sizeof(double) * tr.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(c.rR, rr.data(), sizeof(double) * rr.size(), cudaMemcpyHostToDevice);
    } else {
        std::vector<float> trf(tr.begin(), tr.end()), rrf(rr.begin(), rr.end());
        cudaMemcpy(c.tR, trf.data(), sizeof(float) * trf.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(c.rR, rrf.data(), sizeof(float) * rrf.size(), cudaMemcpyHostToDevice);
    }
    return cuda_check("prs_create_particles");
}

prs_status prs_write_state(prs_ctx *h, const double *x, const double *u, const double *omega,
                           int where)
{
    if (!h || !h->c.n_p)
        return fail(PRS_ERR_STATE, "prs_write_state: no particles");
    if (!x || !u || !omega || (where != PRS_HOST && where != PRS_DEVICE))
        return fail(PRS_ERR_ARG, "prs_write_state: bad arguments");
    Ctx &c = h->c;
    const size_t vec = 3 * sizeof(double) * (size_t)c.n_p;
    cudaMemcpyAsync(c.x[c.cur], x, vec, kind_to_dev(where), c.stream);
    cudaMemcpyAsync(c.u[c.cur], u, vec, kind_to_dev(where), c.stream);
    cudaMemcpyAsync(c.om[c.cur], omega, vec, kind_to_dev(where), c.stream);
    cudaMemsetAsync(c.hcnt[c.hcur], 0, sizeof(int) * c.n_p, c.stream);
    cudaMemsetAsync(c.wact[c.hcur], 0, PRS_MAX_WALLS * (size_t)c.n_p, c.stream);
    force_rebuild(c);
    if (where == PRS_HOST)
        cudaStreamSynchronize(c.stream);
    return cuda_check("prs_write_state");
}

prs_status prs_read_state(prs_ctx *h, double *x, double *u, double *omega, int where)
{
    if (!h || !h->c.n_p)
        return fail(PRS_ERR_STATE, "prs_read_state: no particles");
    if (where != PRS_HOST && where != PRS_DEVICE)
        return fail(PRS_ERR_ARG, "prs_read_state: bad where");
    Ctx &c = h->c;
    const size_t vec = 3 * sizeof(double) * (size_t)c.n_p;
    if (x)
        cudaMemcpyAsync(x, c.x[c.cur], vec, kind_from_dev(where), c.stream);
    if (u)
        cudaMemcpyAsync(u, c.u[c.cur], vec, kind_from_dev(where), c.stream);
    if (omega)
        cudaMemcpyAsync(omega, c.om[c.cur], vec, kind_from_dev(where), c.stream);
    prs_status st = cuda_check("prs_read_state");
    if (st)
        return st;
    return latched_errors(c);
}

static prs_status ibm_step_entry(prs_ctx *h, void *u, void *v, void *w, void *fx, void *fy,
                                 void *fz, double dt, double alpha, const prs_ibm_opts *opts,
                                 float *feats, float *targets)
{
    if (!h || !h->c.n_p)
        return fail(PRS_ERR_STATE, "prs_ibm_step: no particles");
    Ctx &c = h->c;
    prs_ibm_opts o{1, 0.0, PRS_DEVICE, 0, 0, 0, 0};
    if (opts)
        o = *opts;
    if (o.delta_kernel != 0 && o.delta_kernel != 3 && o.delta_kernel != 4)
        return fail(PRS_ERR_ARG, "prs_ibm_step: delta_kernel must be 3 or 4");
    if (o.delta_kernel == 4 && (o.grid_where != PRS_DEVICE || o.learned || feats || targets))
        return fail(PRS_ERR_ARG,
                    "prs_ibm_step: the 4-point kernel takes device fields, no warm start");
    c.delta_kernel = o.delta_kernel == 4 ? 4 : 3;
    if (c.delta_kernel == 4 && !c.acc4) {
        const size_t cells = (size_t)c.g.n[0] * c.g.n[1] * c.g.n[2];
        if (!alloc_into(h, c.acc4, 3 * sizeof(unsigned long long) * cells))
            return fail(PRS_ERR_OOM, "prs_ibm_step: device allocation failed");
        cudaMemsetAsync(c.acc4, 0, 3 * sizeof(unsigned long long) * cells, c.stream);
    }
    if (o.learned && !c.mlp_ready)
        return fail(PRS_ERR_STATE, "prs_ibm_step: learned warm start without network parameters");
    if (!u || !v || !w || !fx || !fy || !fz)
        return fail(PRS_ERR_ARG, "prs_ibm_step: NULL field");
    if (!(dt > 0.0) || !(alpha > 0.0) || o.n_mdf_max < 1 ||
        (o.grid_where != PRS_HOST && o.grid_where != PRS_DEVICE))
        return fail(PRS_ERR_ARG, "prs_ibm_step: need dt > 0, alpha > 0, n_mdf_max >= 1");
    if (o.n_mdf_max > 1 && !c.dFl) {
        if (!alloc_into(h, c.dFl, 4 * prec_bytes(c) * (size_t)c.n_p * c.n_l))
            return fail(PRS_ERR_OOM, "prs_ibm_step: device allocation failed");
    }
    void *fld[6] = {u, v, w, fx, fy, fz};
    const size_t bytes = prec_bytes(c) * (size_t)c.g.n[0] * c.g.n[1] * c.g.n[2];
    const bool host = o.grid_where == PRS_HOST;
    // host fields: only the z-slab the markers' stencils can reach is copied
    // in and out (the step changes no other cell)
    HostPipe hp;
    if (host) {
        for (int i = 0; i < 6; i++) {
            if (!c.stage[i]) {
                if (!alloc_into(h, c.stage[i], bytes))
                    return fail(PRS_ERR_OOM, "prs_ibm_step: staging allocation failed");
                cudaMemsetAsync(c.stage[i], 0, bytes, c.stream);
            }
        }
        if (!c.copy_stream) {
            bool ok = cudaStreamCreateWithFlags(&c.copy_stream, cudaStreamNonBlocking) ==
                          cudaSuccess &&
                      cudaStreamCreateWithFlags(&c.copy_out, cudaStreamNonBlocking) ==
                          cudaSuccess;
            cudaEvent_t *ev[4] = {&c.ev_start, &c.ev_uvw, &c.ev_f, &c.ev_out_done};
            for (int i = 0; i < 4; i++)
                ok = ok && cudaEventCreateWithFlags(ev[i], cudaEventDisableTiming) == cudaSuccess;
            for (int i = 0; i < Ctx::kHostChunks; i++)
                ok = ok &&
                     cudaEventCreateWithFlags(&c.ev_chunk[i], cudaEventDisableTiming) ==
                         cudaSuccess &&
                     cudaEventCreateWithFlags(&c.ev_in[i], cudaEventDisableTiming) == cudaSuccess;
            if (!ok)
                return cuda_check("prs_ibm_step (copy streams)");
        }
        int zlo = 0, zhi = c.g.n[2];
        if (!c.g.periodic[2]) {
            int zr[2];
            particle_zrange(c, zr, c.stream);  // synchronises
            zlo = std::max(0, zr[0]);
            zhi = std::min(c.g.n[2], zr[1] + 1);
            if (zhi <= zlo)
                zlo = zhi = 0;
        }
        hp.zlo = zlo;
        hp.zhi = zhi;
        hp.plane = prec_bytes(c) * (size_t)c.g.n[0] * c.g.n[1];
        for (int i = 0; i < 6; i++) {
            hp.host[i] = fld[i];
            hp.dev[i] = c.stage[i];
        }
        // the copies start after the context stream's earlier work
        cudaEventRecord(c.ev_start, c.stream);
        cudaStreamWaitEvent(c.copy_stream, c.ev_start, 0);
        cudaStreamWaitEvent(c.copy_out, c.ev_start, 0);
        if (c.host_pending)  // an earlier asynchronous step may still write the arrays
            cudaStreamWaitEvent(c.copy_stream, c.ev_out_done, 0);
        const bool pipe = !c.g.periodic[2] && zhi > zlo && c.tile_fmax && o.tol <= 0.0 &&
                          o.n_mdf_max == 1 && !o.learned && !feats && !targets;
        if (pipe) {
            hp.tz_lo = zlo / kTileZ;
            hp.layers = (zhi - 1) / kTileZ - hp.tz_lo + 1;
            hp.chunks = std::min(Ctx::kHostChunks, hp.layers);
            hp.uvw_in = hp.f_in = true;
            for (int k = 0; k < hp.chunks; k++) {
                host_copy_planes(hp, hp.plane_lo(k, hp.chunks), hp.plane_hi(k, hp.chunks),
                                 cudaMemcpyHostToDevice, 0, 6, c.copy_stream);
                cudaEventRecord(c.ev_in[k], c.copy_stream);
            }
        } else {
            host_copy_planes(hp, zlo, zhi, cudaMemcpyHostToDevice, 0, 3, c.copy_stream);
            cudaEventRecord(c.ev_uvw, c.copy_stream);
            host_copy_planes(hp, zlo, zhi, cudaMemcpyHostToDevice, 3, 6, c.copy_stream);
            cudaEventRecord(c.ev_f, c.copy_stream);
        }
    }
    c.last_h2d = c.last_d2h = host ? 6 * (long long)(hp.plane * (size_t)(hp.zhi - hp.zlo)) : 0;
    void *d[6];
    for (int i = 0; i < 6; i++)
        d[i] = host ? c.stage[i] : fld[i];
    HostPipe *hpp = host ? &hp : nullptr;
    prs_status st;
    if (c.precision == PRS_FP64)
        st = ibm_step_t<double>(h, (double *)d[0], (double *)d[1], (double *)d[2],
                                (double *)d[3], (double *)d[4], (double *)d[5], dt, alpha, o,
                                feats, targets, hpp);
    else
        st = ibm_step_t<float>(h, (float *)d[0], (float *)d[1], (float *)d[2], (float *)d[3],
                               (float *)d[4], (float *)d[5], dt, alpha, o, feats, targets, hpp);
    if (host) {
        if (st >= 0 && !hp.out_done) {
            // the whole slab once the step's kernels are done
            cudaEventRecord(c.ev_chunk[0], c.stream);
            cudaStreamWaitEvent(c.copy_out, c.ev_chunk[0], 0);
            host_copy_planes(hp, hp.zlo, hp.zhi, cudaMemcpyDeviceToHost, 0, 6, c.copy_out);
        }
        if (st >= 0 && o.host_async) {
            // the copies in are done once the kernels that wait for them are;
            // the copies out are waited for by the next synchronising call
            cudaEventRecord(c.ev_out_done, c.copy_out);
            c.host_pending = true;
            return cuda_check("prs_ibm_step (host copies)");
        }
        // no copy into or out of the caller's buffers outlives the call
        cudaStreamSynchronize(c.copy_stream);
        cudaStreamSynchronize(c.copy_out);
        cudaStreamSynchronize(c.stream);
        c.host_pending = false;
        if (st < 0)
            return st;
        prs_status e = cuda_check("prs_ibm_step (host copies)");
        if (e)
            return e;
    }
    return st;
}

prs_status prs_ibm_step(prs_ctx *h, void *u, void *v, void *w, void *fx, void *fy, void *fz,
                        double dt, double alpha, const prs_ibm_opts *opts)
{
    return ibm_step_entry(h, u, v, w, fx, fy, fz, dt, alpha, opts, nullptr, nullptr);
}

prs_status prs_predict(prs_ctx *h, int component, const void *u_in, void *u_out, void *H,
                       double nu, double dt, double alpha, double beta)
{
    if (!h)
        return fail(PRS_ERR_ARG, "prs_predict: NULL context");
    Ctx &c = h->c;
    if (!u_in || !u_out || !H || u_in == u_out || u_out == H || u_in == H)
        return fail(PRS_ERR_ARG, "prs_predict: NULL or aliased fields");
    if (component < 0 || component > 2 || !(nu >= 0.0) || !(dt > 0.0) ||
        !std::isfinite(alpha) || !std::isfinite(beta))
        return fail(PRS_ERR_ARG, "prs_predict: need component 0..2, nu >= 0, dt > 0");
    for (int a = 0; a < 3; a++) {
        const double off = c.g.off[component * 3 + a];
        if (!c.g.periodic[a] && off != 0.0 && off != 0.5)
            return fail(PRS_ERR_ARG, "prs_predict: wall-bounded axis with offset not 0 or 1/2");
    }
    fluid_predict(c, component, u_in, u_out, H, nu, dt, alpha, beta, c.stream);
    return cuda_check("prs_predict");
}

prs_status prs_mlp_collect(prs_ctx *h, void *u, void *v, void *w, void *fx, void *fy, void *fz,
                           double dt, double alpha, const prs_ibm_opts *opts, float *feats,
                           float *targets)
{
    if (!feats || !targets)
        return fail(PRS_ERR_ARG, "prs_mlp_collect: NULL feats or targets");
    prs_ibm_opts o{1, 0.0, PRS_DEVICE, 0, 0, 0, 0};
    if (opts)
        o = *opts;
    o.learned = 0;
    return ibm_step_entry(h, u, v, w, fx, fy, fz, dt, alpha, &o, feats, targets);
}

static prs_status mlp_ready(prs_ctx *h, const char *who)
{
    if (!h)
        return fail(PRS_ERR_ARG, who);
    if (!h->c.mlp_ready) {
        set_error("%s: no network parameters (prs_mlp_set_params first)", who);
        return PRS_ERR_STATE;
    }
    return PRS_OK;
}

prs_status prs_mlp_set_params(prs_ctx *h, const float *params)
{
    if (!h || !params)
        return fail(PRS_ERR_ARG, "prs_mlp_set_params: NULL argument");
    Ctx &c = h->c;
    const int npad = mlp_npad();
    if (!c.mlp_w) {
        if (!alloc_into(h, c.mlp_w, sizeof(float) * npad) ||
            !alloc_into(h, c.mlp_m, sizeof(float) * npad) ||
            !alloc_into(h, c.mlp_v, sizeof(float) * npad) ||
            !alloc_into(h, c.mlp_pack, 2 * (size_t)mlp_pack_elems()) ||
            !alloc_into(h, c.mlp_dev, sizeof(float) * (npad + 1)))
            return fail(PRS_ERR_OOM, "prs_mlp_set_params: device allocation failed");
    }
    std::vector<float> w(npad, 0.0f);
    for (int q = 0; q < PRS_MLP_NPARAM; q++)
        w[mlp_pad_index(q)] = params[q];
    cudaStream_t s = c.stream;
    cudaMemcpyAsync(c.mlp_w, w.data(), sizeof(float) * npad, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(c.mlp_m, 0, sizeof(float) * npad, s);
    cudaMemsetAsync(c.mlp_v, 0, sizeof(float) * npad, s);
    cudaMemsetAsync(c.mlp_pack, 0, 2 * (size_t)mlp_pack_elems(), s);
    mlp_pack(c, s);
    cudaStreamSynchronize(s);  // the host vector goes out of scope
    c.mlp_step = 0;
    c.mlp_ready = 1;
    return cuda_check("prs_mlp_set_params");
}

prs_status prs_mlp_get_params(prs_ctx *h, float *params)
{
    prs_status st = mlp_ready(h, "prs_mlp_get_params");
    if (st)
        return st;
    if (!params)
        return fail(PRS_ERR_ARG, "prs_mlp_get_params: NULL params");
    Ctx &c = h->c;
    std::vector<float> w(mlp_npad());
    cudaMemcpyAsync(w.data(), c.mlp_w, sizeof(float) * w.size(), cudaMemcpyDeviceToHost,
                    c.stream);
    cudaStreamSynchronize(c.stream);
    for (int q = 0; q < PRS_MLP_NPARAM; q++)
        params[q] = w[mlp_pad_index(q)];
    st = cuda_check("prs_mlp_get_params");
    return st ? st : latched_errors(c);
}

prs_status prs_mlp_forward(prs_ctx *h, const float *feats, long long n, float *out)
{
    prs_status st = mlp_ready(h, "prs_mlp_forward");
    if (st)
        return st;
    if (n < 0 || (n > 0 && (!feats || !out)))
        return fail(PRS_ERR_ARG, "prs_mlp_forward: bad arguments");
    phase_begin(h->c, PRS_PHASE_MLP);
    mlp_forward_launch(h->c, feats, n, out, h->c.stream);
    phase_end(h->c);
    return cuda_check("prs_mlp_forward");
}

prs_status prs_mlp_grad(prs_ctx *h, const float *feats, const float *targets, long long n,
                        float *grad, float *loss)
{
    prs_status st = mlp_ready(h, "prs_mlp_grad");
    if (st)
        return st;
    if (n < 1 || !feats || !targets)
        return fail(PRS_ERR_ARG, "prs_mlp_grad: bad arguments");
    Ctx &c = h->c;
    const int npad = mlp_npad();
    if (mlp_grad_launch(c, feats, targets, n, c.mlp_dev, c.mlp_dev + npad, nullptr, c.stream))
        return fail(PRS_ERR_OOM, "prs_mlp_grad: device allocation failed");
    std::vector<float> g(npad + 1);
    cudaMemcpyAsync(g.data(), c.mlp_dev, sizeof(float) * g.size(), cudaMemcpyDeviceToHost,
                    c.stream);
    cudaStreamSynchronize(c.stream);
    st = cuda_check("prs_mlp_grad");
    if (!st)
        st = latched_errors(c);
    if (st)
        return st;
    if (grad)
        for (int q = 0; q < PRS_MLP_NPARAM; q++)
            grad[q] = g[mlp_pad_index(q)];
    if (loss)
        *loss = g[npad];
    return PRS_OK;
}

static prs_status mlp_train(prs_ctx *h, const char *who, const float *feats,
                            const float *targets, long long n, long long n_total,
                            long long start, long long stride, const prs_adam_opts *opts,
                            float *loss)
{
    prs_status st = mlp_ready(h, who);
    if (st)
        return st;
    if (n < 1 || !feats || !targets || !opts || !(opts->lr > 0.0) ||
        !(opts->beta1 >= 0.0 && opts->beta1 < 1.0) || !(opts->beta2 >= 0.0 && opts->beta2 < 1.0) ||
        !(opts->eps > 0.0))
        return fail(PRS_ERR_ARG, (std::string(who) + ": bad arguments").c_str());
    Ctx &c = h->c;
    const int npad = mlp_npad();
    const long long k = c.mlp_step + 1;
    MlpAdam ad{opts->lr, opts->beta1, opts->beta2, opts->eps,
               1.0 / (1.0 - std::pow(opts->beta1, (double)k)),
               1.0 / (1.0 - std::pow(opts->beta2, (double)k))};
    phase_begin(c, PRS_PHASE_MLP);
    const int r = mlp_grad_launch(c, feats, targets, n, nullptr, c.mlp_dev + npad, &ad, c.stream,
                                  n_total, start, stride);
    phase_end(c);
    if (r)
        return fail(PRS_ERR_OOM, (std::string(who) + ": device allocation failed").c_str());
    c.mlp_step = k;
    if (loss) {
        cudaMemcpyAsync(loss, c.mlp_dev + npad, sizeof(float), cudaMemcpyDeviceToHost, c.stream);
        cudaStreamSynchronize(c.stream);
        st = cuda_check(who);
        return st ? st : latched_errors(c);
    }
    return cuda_check(who);
}

prs_status prs_mlp_train_step(prs_ctx *h, const float *feats, const float *targets,
                              long long n, const prs_adam_opts *opts, float *loss)
{
    return mlp_train(h, "prs_mlp_train_step", feats, targets, n, n, 0, 0, opts, loss);
}

static long long gcd_ll(long long a, long long b)
{
    while (b) {
        const long long t = a % b;
        a = b;
        b = t;
    }
    return a;
}

prs_status prs_mlp_train_step_sampled(prs_ctx *h, const float *feats, const float *targets,
                                      long long n_total, long long n, long long start,
                                      long long stride, const prs_adam_opts *opts, float *loss)
{
    const char *who = "prs_mlp_train_step_sampled";
    if (!h)
        return fail(PRS_ERR_ARG, "prs_mlp_train_step_sampled: no context");
    if (n_total < 1 || n < 1 || n > n_total || start < 0 || start >= n_total || stride < 1 ||
        gcd_ll(stride, n_total) != 1 || n_total > (1LL << 40) || stride > (1LL << 22))
        return fail(PRS_ERR_ARG, "prs_mlp_train_step_sampled: need 1 <= n <= n_total, "
                                 "0 <= start < n_total and a stride in [1, 2^22] coprime "
                                 "with n_total");
    return mlp_train(h, who, feats, targets, n, n_total, start, stride, opts, loss);
}

// The n_sub sub-steps as one CUDA graph: captured on first use, replayed
// while the sub-step count, the step, the parameters, the buffer parity and
// the stream stay the same. The graph holds the same launches in the same
// order as the loop, so the results are the same bit for bit. Returns false,
// with nothing queued, when graphs are off, when the phases are being timed
// (the timing events are recorded per launch), on the legacy default
// stream, or when the capture fails (graphs are then turned off for the
// context).
static bool dem_graph_run(Ctx &c, double dt_p, int n_sub)
{
    if (!c.graphs || c.profiling || !c.stream || n_sub < 1)
        return false;
    const void *flub = c.dp.mu_f > 0.0 ? c.flub : nullptr;
    const bool same = c.dg_exec && c.dg_nsub == n_sub && c.dg_dt == dt_p &&
                      c.dg_cur == c.cur && c.dg_hcur == c.hcur && c.dg_stream == c.stream &&
                      c.dg_flub == flub && std::memcmp(&c.dg_dp, &c.dp, sizeof(DemParams)) == 0;
    if (!same) {
        if (c.dg_exec) {
            // a caller that changes the step or the options on every call
            // would pay a capture per call: after two graphs in a row that
            // were never replayed, launches are used for the context
            c.dg_wasted = c.dg_replays == 0 ? c.dg_wasted + 1 : 0;
            cudaGraphExecDestroy(c.dg_exec);
            c.dg_exec = nullptr;
            if (c.dg_wasted >= 2) {
                c.graphs = 0;
                return false;
            }
        }
        const int cur0 = c.cur, hcur0 = c.hcur;
        const long long l0 = c.n_launch;
        if (cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            c.graphs = 0;
            return false;
        }
        for (int k = 0; k < n_sub; k++) {
            dem_substep(c, dt_p, k == n_sub - 1, c.stream);
            c.cur = 1 - c.cur;
            c.hcur = 1 - c.hcur;
        }
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c.stream, &g);
        c.cur = cur0;  // nothing has run yet
        c.hcur = hcur0;
        const long long nl = c.n_launch - l0;
        c.n_launch = l0;
        cudaGraphExec_t ex = nullptr;
        if (e != cudaSuccess || !g || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
            if (g)
                cudaGraphDestroy(g);
            cudaGetLastError();
            c.graphs = 0;
            return false;
        }
        cudaGraphDestroy(g);
        c.dg_exec = ex;
        c.dg_nsub = n_sub;
        c.dg_dt = dt_p;
        c.dg_cur = c.cur;
        c.dg_hcur = c.hcur;
        c.dg_stream = c.stream;
        c.dg_flub = flub;
        c.dg_dp = c.dp;
        c.dg_launches = nl;
        c.dg_replays = -1;  // the launch below is the capture's own
    }
    if (cudaGraphLaunch(c.dg_exec, c.stream) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (n_sub & 1) {
        c.cur = 1 - c.cur;
        c.hcur = 1 - c.hcur;
    }
    c.n_launch += c.dg_launches;
    c.dg_replays++;
    return true;
}

prs_status prs_dem_step(prs_ctx *h, double dt_p, int n_sub, const prs_dem_opts *opts)
{
    if (!h || !h->c.n_p)
        return fail(PRS_ERR_STATE, "prs_dem_step: no particles");
    if (!opts || !(dt_p > 0.0) || n_sub < 0)
        return fail(PRS_ERR_ARG, "prs_dem_step: need options, dt_p > 0, n_sub >= 0");
    const prs_dem_opts &o = *opts;
    if (!(o.e_n > 0.0 && o.e_n <= 1.0) || !(o.e_t > 0.0 && o.e_t <= 1.0) || !(o.mu >= 0.0) ||
        !(o.T_c > 0.0))
        return fail(PRS_ERR_ARG, "prs_dem_step: need 0 < e_n, e_t <= 1, mu >= 0, T_c > 0");
    if (o.model != PRS_CONTACT_LINEAR && o.model != PRS_CONTACT_ACTM)
        return fail(PRS_ERR_ARG, "prs_dem_step: unknown contact model");
    if (o.model == PRS_CONTACT_ACTM && !(o.e_n < 1.0))
        return fail(PRS_ERR_ARG, "prs_dem_step: the adaptive model needs e_n < 1");
    if (!(o.u_min >= 0.0) || !(o.mu_f >= 0.0) || !(o.eps_d_pp >= 0.0 && o.eps_d_pp <= 0.1) ||
        !(o.eps_d_pw >= 0.0 && o.eps_d_pw <= 0.1) || !(o.eps_s >= 0.0))
        return fail(PRS_ERR_ARG,
                    "prs_dem_step: need u_min, mu_f, eps_s >= 0 and lubrication ranges in [0, 0.1]");
    Ctx &c = h->c;
    dem_constants(c, o, c.dp);
    if (c.dp.eps_s >= c.dp.eps_d_pp || c.dp.eps_s >= c.dp.eps_d_pw)
        return fail(PRS_ERR_ARG, "prs_dem_step: the saturation gap must lie below the ranges");
    c.dp_valid = 1;
    // lubrication reaches gaps up to eps_d R beyond contact: the neighbour
    // list is widened by that much (within the cells' reserved margin)
    const double reach = c.dp.mu_f > 0.0 ? c.dp.eps_d_pp * c.R : 0.0;
    if (c.dp.mu_f > 0.0 && !c.flub && !alloc_into(h, c.flub, 3 * sizeof(double) * (size_t)c.n_p))
        return fail(PRS_ERR_OOM, "prs_dem_step: device allocation failed");
    if (reach != c.lub_reach) {
        c.lub_reach = reach;
        force_rebuild(c);
    }
    if (n_sub > 0)
        dem_shadow(c, c.stream);
    c.dg_used = dem_graph_run(c, dt_p, n_sub) ? 1 : 0;
    if (!c.dg_used) {
        for (int k = 0; k < n_sub; k++) {
            dem_substep(c, dt_p, k == n_sub - 1, c.stream);
            c.cur = 1 - c.cur;
            c.hcur = 1 - c.hcur;
        }
    }
    return cuda_check("prs_dem_step");
}

prs_status prs_read_forces(prs_ctx *h, double *F_h, double *T_h, double *F_c, double *T_c,
                           int where)
{
    if (!h || !h->c.n_p)
        return fail(PRS_ERR_STATE, "prs_read_forces: no particles");
    if (where != PRS_HOST && where != PRS_DEVICE)
        return fail(PRS_ERR_ARG, "prs_read_forces: bad where");
    Ctx &c = h->c;
    const size_t vec = 3 * sizeof(double) * (size_t)c.n_p;
    if (c.Fcf) {
        // FP32 form: the collision force and torque are kept in FP32
        dem_forces_f2d(c, c.Fcf, c.Fc, c.stream);
        dem_forces_f2d(c, c.Tcf, c.Tc, c.stream);
    }
    double *dst[4] = {F_h, T_h, F_c, T_c};
    double *src[4] = {c.Fh, c.Th, c.Fc, c.Tc};
    for (int i = 0; i < 4; i++)
        if (dst[i])
            cudaMemcpyAsync(dst[i], src[i], vec, kind_from_dev(where), c.stream);
    prs_status st = cuda_check("prs_read_forces");
    return st ? st : latched_errors(c);
}

prs_status prs_read_marker_forces(prs_ctx *h, void *F_l, int where)
{
    if (!h || !h->c.n_p)
        return fail(PRS_ERR_STATE, "prs_read_marker_forces: no particles");
    if (!F_l || (where != PRS_HOST && where != PRS_DEVICE))
        return fail(PRS_ERR_ARG, "prs_read_marker_forces: bad arguments");
    Ctx &c = h->c;
    const size_t bytes = 3 * prec_bytes(c) * (size_t)c.n_p * c.n_l;
    if (where == PRS_DEVICE) {
        ibm_unpack_forces(c, F_l, c.stream);
    } else {
        void *tmp = ctx_alloc(c, bytes);
        if (!tmp)
            return fail(PRS_ERR_OOM, "prs_read_marker_forces: device allocation failed");
        ibm_unpack_forces(c, tmp, c.stream);
        cudaMemcpyAsync(F_l, tmp, bytes, cudaMemcpyDeviceToHost, c.stream);
        cudaStreamSynchronize(c.stream);
        ctx_free(c, tmp);
    }
    prs_status st = cuda_check("prs_read_marker_forces");
    return st ? st : latched_errors(c);
}

prs_status prs_read_template(prs_ctx *h, double *t, double *dV, int *n_l)
{
    if (!h || !h->c.n_p)
        return fail(PRS_ERR_STATE, "prs_read_template: no particles");
    Ctx &c = h->c;
    if (t) {
        cudaMemcpyAsync(t, c.t64, 3 * sizeof(double) * c.n_l, cudaMemcpyDeviceToHost, c.stream);
        cudaStreamSynchronize(c.stream);
    }
    if (dV)
        *dV = c.dV;
    if (n_l)
        *n_l = c.n_l;
    return cuda_check("prs_read_template");
}

prs_status prs_read_history(prs_ctx *h, int *cnt, int *pid, double *uin, double *dlt,
                            unsigned char *wall_act, double *wall_uin, double *wall_dlt)
{
    if (!h || !h->c.n_p)
        return fail(PRS_ERR_STATE, "prs_read_history: no particles");
    if (!cnt || !pid || !uin || !dlt || !wall_act || !wall_uin || !wall_dlt)
        return fail(PRS_ERR_ARG, "prs_read_history: NULL output");
    Ctx &c = h->c;
    const int n = c.n_p, b = c.hcur;
    const int S = PRS_MAX_CONTACTS, W = PRS_MAX_WALLS;
    std::vector<int> hc(n), hp((size_t)S * n);
    std::vector<double> hu((size_t)S * n), hd((size_t)3 * S * n), wu((size_t)W * n),
        wd((size_t)3 * W * n);
    std::vector<unsigned char> wa((size_t)W * n);
    cudaMemcpyAsync(hc.data(), c.hcnt[b], sizeof(int) * n, cudaMemcpyDeviceToHost, c.stream);
    cudaMemcpyAsync(hp.data(), c.hpid[b], sizeof(int) * hp.size(), cudaMemcpyDeviceToHost,
                    c.stream);
    cudaMemcpyAsync(hu.data(), c.huin[b], sizeof(double) * hu.size(), cudaMemcpyDeviceToHost,
                    c.stream);
    cudaMemcpyAsync(hd.data(), c.hdlt[b], sizeof(double) * hd.size(), cudaMemcpyDeviceToHost,
                    c.stream);
    cudaMemcpyAsync(wa.data(), c.wact[b], wa.size(), cudaMemcpyDeviceToHost, c.stream);
    cudaMemcpyAsync(wu.data(), c.wuin[b], sizeof(double) * wu.size(), cudaMemcpyDeviceToHost,
                    c.stream);
    cudaMemcpyAsync(wd.data(), c.wdlt[b], sizeof(double) * wd.size(), cudaMemcpyDeviceToHost,
                    c.stream);
    prs_status st = cuda_check("prs_read_history");
    if (st)
        return st;
    st = latched_errors(c);
    if (st)
        return st;
    // the device keeps each pair once, at its lower id: give it to both
    std::vector<std::vector<int>> slots(n);
    for (int p = 0; p < n; p++)
        for (int s = 0; s < hc[p]; s++) {
            const int q = hp[(size_t)s * n + p];
            slots[p].push_back((int)((size_t)s * n + p));
            if (q >= 0 && q < n)
                slots[q].push_back((int)((size_t)s * n + p));
        }
    for (int p = 0; p < n; p++) {
        auto &v = slots[p];
        // slot k = s * n + owner; seen from sphere p its partner is hp[k]
        // when p owns it, else the owner; list partners ascending
        auto partner = [&](int k) {
            const int owner = (int)((size_t)k % n);
            return owner == p ? hp[(size_t)k] : owner;
        };
        std::sort(v.begin(), v.end(), [&](int x, int y) { return partner(x) < partner(y); });
        const int m = (int)std::min<size_t>(v.size(), S);
        cnt[p] = m;
        for (int s = 0; s < S; s++) {
            size_t o = (size_t)p * S + s;
            if (s < m) {
                const int k = v[s];
                const int owner = (int)((size_t)k % n);
                const int sl = (int)((size_t)k / n);
                pid[o] = partner(k);
                uin[o] = hu[k];
                for (int d = 0; d < 3; d++)
                    dlt[o * 3 + d] = hd[((size_t)sl * 3 + d) * n + owner];
            } else {
                pid[o] = -1;
                uin[o] = 0.0;
                for (int d = 0; d < 3; d++)
                    dlt[o * 3 + d] = 0.0;
            }
        }
        for (int wsl = 0; wsl < W; wsl++) {
            bool on = wa[(size_t)wsl * n + p] != 0;
            size_t o = (size_t)p * W + wsl;
            wall_act[o] = on ? 1 : 0;
            wall_uin[o] = on ? wu[(size_t)wsl * n + p] : 0.0;
            for (int k = 0; k < 3; k++)
                wall_dlt[o * 3 + k] = on ? wd[((size_t)wsl * 3 + k) * n + p] : 0.0;
        }
    }
    return PRS_OK;
}

prs_status prs_write_history(prs_ctx *h, const int *cnt, const int *pid, const double *uin,
                             const double *dlt, const unsigned char *wall_act,
                             const double *wall_uin, const double *wall_dlt)
{
    if (!h || !h->c.n_p)
        return fail(PRS_ERR_STATE, "prs_write_history: no particles");
    if (!cnt || !pid || !uin || !dlt || !wall_act || !wall_uin || !wall_dlt)
        return fail(PRS_ERR_ARG, "prs_write_history: NULL input");
    Ctx &c = h->c;
    const int n = c.n_p, b = c.hcur;
    const int S = PRS_MAX_CONTACTS, W = PRS_MAX_WALLS;
    std::vector<int> hp((size_t)S * n, -1);
    std::vector<double> hu((size_t)S * n), hd((size_t)3 * S * n), wu((size_t)W * n),
        wd((size_t)3 * W * n);
    std::vector<unsigned char> wa((size_t)W * n);
    std::vector<int> lc(n, 0);
    for (int p = 0; p < n; p++) {
        if (cnt[p] < 0 || cnt[p] > S)
            return fail(PRS_ERR_ARG, "prs_write_history: slot count out of range");
        for (int s = 0; s < cnt[p]; s++) {
            size_t o = (size_t)p * S + s;
            if (pid[o] < 0 || pid[o] >= n || pid[o] == p || (s > 0 && pid[o] <= pid[o - 1]))
                return fail(PRS_ERR_ARG,
                            "prs_write_history: partner ids must be ascending and valid");
            if (pid[o] < p)
                continue;  // the device keeps each pair at its lower id
            const int sl = lc[p]++;
            hp[(size_t)sl * n + p] = pid[o];
            hu[(size_t)sl * n + p] = uin[o];
            for (int k = 0; k < 3; k++)
                hd[((size_t)sl * 3 + k) * n + p] = dlt[o * 3 + k];
        }
        for (int wsl = 0; wsl < W; wsl++) {
            size_t o = (size_t)p * W + wsl;
            wa[(size_t)wsl * n + p] = wall_act[o] ? 1 : 0;
            wu[(size_t)wsl * n + p] = wall_uin[o];
            for (int k = 0; k < 3; k++)
                wd[((size_t)wsl * 3 + k) * n + p] = wall_dlt[o * 3 + k];
        }
    }
    cudaMemcpyAsync(c.hcnt[b], lc.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c.stream);
    cudaMemcpyAsync(c.hpid[b], hp.data(), sizeof(int) * hp.size(), cudaMemcpyHostToDevice,
                    c.stream);
    cudaMemcpyAsync(c.huin[b], hu.data(), sizeof(double) * hu.size(), cudaMemcpyHostToDevice,
                    c.stream);
    cudaMemcpyAsync(c.hdlt[b], hd.data(), sizeof(double) * hd.size(), cudaMemcpyHostToDevice,
                    c.stream);
    cudaMemcpyAsync(c.wact[b], wa.data(), wa.size(), cudaMemcpyHostToDevice, c.stream);
    cudaMemcpyAsync(c.wuin[b], wu.data(), sizeof(double) * wu.size(), cudaMemcpyHostToDevice,
                    c.stream);
    cudaMemcpyAsync(c.wdlt[b], wd.data(), sizeof(double) * wd.size(), cudaMemcpyHostToDevice,
                    c.stream);
    cudaStreamSynchronize(c.stream);
    return cuda_check("prs_write_history");
}

prs_status prs_find_pairs(prs_ctx *h, double cutoff, int *pairs, long long max_pairs,
                          long long *n_pairs)
{
    if (!h || !h->c.n_p)
        return fail(PRS_ERR_STATE, "prs_find_pairs: no particles");
    if (!(cutoff > 0.0) || max_pairs < 0 || (max_pairs > 0 && !pairs) || !n_pairs)
        return fail(PRS_ERR_ARG, "prs_find_pairs: bad arguments");
    Ctx &c = h->c;
    DemParams geo{};
    geometry_only(c, geo);
    // never more cells than the contact cell list was sized for
    CellGeom cg = make_cell_geom(geo, std::max(cutoff, 2.0 * c.R + c.skin + c.cell_margin));
    int *d_pairs = nullptr;
    void *buf = nullptr;
    if (max_pairs > 0) {
        buf = ctx_alloc(c, sizeof(int) * 2 * (size_t)max_pairs);
        if (!buf)
            return fail(PRS_ERR_OOM, "prs_find_pairs: device allocation failed");
        d_pairs = (int *)buf;
    }
    dem_pairs(c, cg, cutoff, d_pairs, max_pairs, c.stream);
    force_rebuild(c);
    long long total = 0;
    cudaMemcpyAsync(&total, c.d_pairs_n, sizeof(long long), cudaMemcpyDeviceToHost, c.stream);
    cudaStreamSynchronize(c.stream);
    prs_status st = cuda_check("prs_find_pairs");
    if (!st && max_pairs > 0) {
        long long k = std::min(total, max_pairs);
        std::vector<int> hp(2 * (size_t)k);
        cudaMemcpy(hp.data(), d_pairs, sizeof(int) * hp.size(), cudaMemcpyDeviceToHost);
        std::vector<std::pair<int, int>> v((size_t)k);
        for (long long i = 0; i < k; i++)
            v[i] = {hp[2 * i], hp[2 * i + 1]};
        std::sort(v.begin(), v.end());
        for (long long i = 0; i < k; i++) {
            pairs[2 * i] = v[i].first;
            pairs[2 * i + 1] = v[i].second;
        }
        st = cuda_check("prs_find_pairs (copy)");
    }
    if (buf) {
        cudaStreamSynchronize(c.stream);
        ctx_free(c, buf);
    }
    *n_pairs = total;
    return st;
}

// bed arrays on first use
static bool ensure_bed(prs_ctx *h)
{
    Ctx &c = h->c;
    if (c.bed_parent)
        return true;
    const size_t n = (size_t)c.n_p;
    c.bed_cap = 6LL * c.n_p + 64;  // at most 12 contacts a sphere
    return alloc_into(h, c.bed_pairs, sizeof(int) * 2 * (size_t)c.bed_cap) &&
           alloc_into(h, c.bed_parent, sizeof(int) * n) && alloc_into(h, c.bed_root, n) &&
           alloc_into(h, c.bed_flags, n) &&
           alloc_into(h, c.bed_count, sizeof(unsigned long long));
}

static bool ensure_tracker(prs_ctx *h)
{
    Ctx &c = h->c;
    if (c.trk_prev)
        return true;
    const size_t n = (size_t)c.n_p;
    return alloc_into(h, c.trk_prev, n) && alloc_into(h, c.trk_salt, n) &&
           alloc_into(h, c.trk_pend, n) && alloc_into(h, c.trk_dep_z, sizeof(double) * n) &&
           alloc_into(h, c.trk_t_imp, sizeof(double) * n) &&
           alloc_into(h, c.trk_u_imp, 3 * sizeof(double) * n) &&
           alloc_into(h, c.trk_om_imp, 3 * sizeof(double) * n) &&
           alloc_into(h, c.trk_flag, sizeof(int) * (n + 1)) &&
           alloc_into(h, c.trk_pos, sizeof(int) * (n + 1)) &&
           alloc_into(h, c.trk_scan_tmp, sizeof(int) * exclusive_scan_tmp_ints(c.n_p + 1));
}

// contact pairs of the current state, then the bed flags; synchronises
static prs_status run_bed(Ctx &c, const char *who)
{
    DemParams geo{};
    geometry_only(c, geo);
    CellGeom cg = make_cell_geom(geo, 2.0 * c.R + c.skin + c.cell_margin);
    dem_pairs(c, cg, 2.0 * c.R, c.bed_pairs, c.bed_cap, c.stream);
    force_rebuild(c);  // the contact search's cell list was reused
    bed_classify(c, c.bed_pairs, c.bed_cap, c.stream);
    long long total = 0;
    cudaMemcpyAsync(&total, c.d_pairs_n, sizeof(long long), cudaMemcpyDeviceToHost, c.stream);
    cudaStreamSynchronize(c.stream);
    prs_status st = cuda_check(who);
    if (st)
        return st;
    if (total > c.bed_cap)
        return fail(PRS_ERR_CAPACITY, "bed detection: more than 6 n_p contact pairs");
    return latched_errors(c);
}

prs_status prs_bed_detect(prs_ctx *h, unsigned char *flags, long long *n_bed, int where)
{
    if (!h || !h->c.n_p)
        return fail(PRS_ERR_STATE, "prs_bed_detect: no particles");
    if (where != PRS_HOST && where != PRS_DEVICE)
        return fail(PRS_ERR_ARG, "prs_bed_detect: bad where");
    Ctx &c = h->c;
    if (!ensure_bed(h))
        return fail(PRS_ERR_OOM, "prs_bed_detect: device allocation failed");
    prs_status st = run_bed(c, "prs_bed_detect");
    if (st)
        return st;
    if (flags)
        cudaMemcpyAsync(flags, c.bed_flags, (size_t)c.n_p, kind_from_dev(where), c.stream);
    unsigned long long cnt = 0;
    cudaMemcpyAsync(&cnt, c.bed_count, sizeof(cnt), cudaMemcpyDeviceToHost, c.stream);
    cudaStreamSynchronize(c.stream);
    if (n_bed)
        *n_bed = (long long)cnt;
    return cuda_check("prs_bed_detect (copy)");
}

prs_status prs_track_saltation(prs_ctx *h, double t, double h_r, double t_cir,
                               prs_event *events, long long max_events, long long *n_events,
                               int where)
{
    if (!h || !h->c.n_p)
        return fail(PRS_ERR_STATE, "prs_track_saltation: no particles");
    if (!(h_r >= 0.0) || !(t_cir >= 0.0) || max_events < 0 || !n_events ||
        (max_events > 0 && !events) || (where != PRS_HOST && where != PRS_DEVICE))
        return fail(PRS_ERR_ARG, "prs_track_saltation: bad arguments");
    Ctx &c = h->c;
    if (!ensure_bed(h) || !ensure_tracker(h))
        return fail(PRS_ERR_OOM, "prs_track_saltation: device allocation failed");
    prs_status st = run_bed(c, "prs_track_saltation");
    if (st)
        return st;
    const long long cap = std::min<long long>(max_events, c.n_p);
    prs_event *out = where == PRS_DEVICE ? events : nullptr;
    void *tmp = nullptr;
    if (where == PRS_HOST && cap > 0) {
        tmp = ctx_alloc(c, sizeof(prs_event) * (size_t)cap);
        if (!tmp)
            return fail(PRS_ERR_OOM, "prs_track_saltation: device allocation failed");
        out = (prs_event *)tmp;
    }
    track_saltation(c, t, h_r, t_cir, out, out ? cap : 0, c.stream);
    int n = 0;
    cudaMemcpyAsync(&n, c.trk_pos + c.n_p, sizeof(int), cudaMemcpyDeviceToHost, c.stream);
    cudaStreamSynchronize(c.stream);
    if (tmp) {
        const long long k = std::min<long long>(n, cap);
        if (k > 0)
            cudaMemcpy(events, tmp, sizeof(prs_event) * (size_t)k, cudaMemcpyDeviceToHost);
        ctx_free(c, tmp);
    }
    *n_events = n;
    st = cuda_check("prs_track_saltation");
    if (st)
        return st;
    if (n > max_events)
        return fail(PRS_ERR_CAPACITY, "prs_track_saltation: more events than max_events");
    return latched_errors(c);
}

prs_status prs_reset_saltation(prs_ctx *h)
{
    if (!h)
        return fail(PRS_ERR_ARG, "prs_reset_saltation: NULL context");
    h->c.trk_started = 0;
    return PRS_OK;
}

prs_status prs_probe_wait(prs_ctx *h, long long polls)
{
    if (!h)
        return fail(PRS_ERR_ARG, "prs_probe_wait: NULL context");
    if (polls < 1 || polls > (1LL << 24))
        return fail(PRS_ERR_ARG, "prs_probe_wait: polls must lie in [1, 2^24]");
    wait_probe(h->c, polls);
    return cuda_check("prs_probe_wait");
}

prs_status prs_get_stats(prs_ctx *h, prs_stats *out)
{
    if (!h || !out)
        return fail(PRS_ERR_ARG, "prs_get_stats: NULL argument");
    Ctx &c = h->c;
    std::memset(out, 0, sizeof(*out));
    out->mdf_passes = c.last_passes;
    out->n_markers = (long long)c.n_p * c.n_l;
    cudaStreamSynchronize(c.stream);
    int err = 0;
    cudaMemcpy(&err, c.d_err, sizeof(int), cudaMemcpyDeviceToHost);
    out->error_word = err;
    out->n_launches = c.n_launch;
    out->h2d_bytes = c.last_h2d;
    out->d2h_bytes = c.last_d2h;
    out->dem_graph = c.dg_used;
    if (c.last_res >= 0.0) {
        out->residual = c.last_res;
    } else {
        unsigned long long b[kRedWords];
        cudaMemcpy(b, c.d_red, sizeof(b), cudaMemcpyDeviceToHost);
        if (c.precision == PRS_FP64) {
            std::memcpy(&out->residual, &b[kRedRes], sizeof(double));
        } else {
            unsigned u32 = (unsigned)b[kRedRes];
            float f;
            std::memcpy(&f, &u32, sizeof(f));
            out->residual = f;
        }
    }
    if (c.n_p) {
        std::vector<int> hc(c.n_p);
        std::vector<unsigned char> wa((size_t)PRS_MAX_WALLS * c.n_p);
        cudaMemcpy(hc.data(), c.ccnt, sizeof(int) * c.n_p, cudaMemcpyDeviceToHost);
        cudaMemcpy(wa.data(), c.wact[c.hcur], wa.size(), cudaMemcpyDeviceToHost);
        // each pair is counted by its owner (the lower id): twice that is
        // the number of occupied contact slots over both spheres
        for (int v : hc)
            out->n_contacts += 2 * v;
        for (unsigned char v : wa)
            out->n_wall_contacts += v;
    }
    return cuda_check("prs_get_stats");
}

prs_status prs_set_stream(prs_ctx *h, void *stream)
{
    if (!h)
        return fail(PRS_ERR_ARG, "prs_set_stream: NULL context");
    cudaStreamSynchronize(h->c.stream);
    h->c.stream = (cudaStream_t)stream;
    return cuda_check("prs_set_stream");
}

prs_status prs_sync(prs_ctx *h)
{
    if (!h)
        return fail(PRS_ERR_ARG, "prs_sync: NULL context");
    prs_status st = cuda_check("prs_sync");
    return st ? st : latched_errors(h->c);
}

prs_status prs_set_graphs(prs_ctx *h, int on)
{
    if (!h)
        return fail(PRS_ERR_ARG, "prs_set_graphs: NULL context");
    h->c.graphs = on ? 1 : 0;
    h->c.dg_wasted = 0;
    if (!on && h->c.dg_exec) {
        cudaGraphExecDestroy(h->c.dg_exec);
        h->c.dg_exec = nullptr;
    }
    return PRS_OK;
}

prs_status prs_set_profiling(prs_ctx *h, int on)
{
    if (!h)
        return fail(PRS_ERR_ARG, "prs_set_profiling: NULL context");
    h->c.profiling = on ? 1 : 0;
    return PRS_OK;
}

prs_status prs_read_profile(prs_ctx *h, double *ms, long long *launches)
{
    if (!h)
        return fail(PRS_ERR_ARG, "prs_read_profile: NULL context");
    cudaStreamSynchronize(h->c.stream);
    if (ms)
        for (int i = 0; i < PRS_NPHASES; i++)
            ms[i] = 0.0;
    if (launches)
        for (int i = 0; i < PRS_NPHASES; i++)
            launches[i] = 0;
    profile_clear(h->c, ms, launches);
    return cuda_check("prs_read_profile");
}

void prs_destroy(prs_ctx *h)
{
    if (!h)
        return;
    cudaStreamSynchronize(h->c.stream);
    if (h->c.dg_exec)
        cudaGraphExecDestroy(h->c.dg_exec);
    if (h->c.copy_stream) {
        cudaStreamSynchronize(h->c.copy_stream);
        cudaStreamDestroy(h->c.copy_stream);
        if (h->c.copy_out) {
            cudaStreamSynchronize(h->c.copy_out);
            cudaStreamDestroy(h->c.copy_out);
        }
        cudaEvent_t ev[4] = {h->c.ev_start, h->c.ev_uvw, h->c.ev_f, h->c.ev_out_done};
        for (cudaEvent_t e : ev)
            if (e)
                cudaEventDestroy(e);
        for (cudaEvent_t e : h->c.ev_chunk)
            if (e)
                cudaEventDestroy(e);
        for (cudaEvent_t e : h->c.ev_in)
            if (e)
                cudaEventDestroy(e);
    }
    profile_destroy(h->c);
    if (h->c.mlp_part)
        ctx_free(h->c, h->c.mlp_part);
    for (void *p : h->owned)
        ctx_free(h->c, p);
    delete h;
}

}  // extern "C"
