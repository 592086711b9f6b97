// Bed and flying spheres, and the impact / rebound events of saltating
// spheres (Sec. 4.3.1 of the paper, steps 1-3).
//
// Step 1. The paper sweeps over the spheres until the number of bed spheres
// stops changing: a sphere is a bed sphere if it touches one. The fixed
// point is the set of spheres connected, through contacts, to the bottom
// layer (centre below one diameter). Here it is found as connected
// components of the contact graph:
//   k_uf_init / k_uf_link / k_uf_compress  lock-free union-find over the
//                   contact pairs (every link hooks the larger root under the
//                   smaller with atomicCAS, so parents only decrease and no
//                   cycle can form); the components, and so the flags, do not
//                   depend on the order in which links land;
//   k_bed_seed      marks the root of every bottom-layer sphere;
//   k_bed_flags     a sphere is a bed sphere if its root is marked.
// Steps 2-3. k_track advances every sphere's state by one observed state:
// departures start a flight at the current height, a rise above h_r makes
// the flight a saltation, the impact of a saltating sphere opens an event
// that its next departure closes (a rebound if within t_cir). Pass 0 only
// flags the spheres that close an event; a scan of the flags gives each its
// slot, and pass 1 writes the events in sphere order and updates the states.
#include "prs_internal.cuh"

namespace prs {
namespace {

constexpr long long kUfSteps = 1LL << 24;  // bound of every find / link loop

__device__ __forceinline__ int uf_find(volatile int *parent, int i)
{
    for (long long it = 0; it < kUfSteps; it++) {
        const int p = parent[i];
        if (p == i)
            return i;
        const int g = parent[p];
        if (g != p)
            parent[i] = g;  // path halving: i is no root, g an ancestor
        i = p;
    }
    return -1;
}

__global__ void k_uf_init(int *parent, unsigned char *root_bed, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        parent[i] = i;
        root_bed[i] = 0;
    }
}

__global__ void k_uf_link(const int *__restrict__ pairs,
                          const unsigned long long *__restrict__ n_pairs, long long cap,
                          int *parent, int *err)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)*n_pairs;
    if (e >= (n < cap ? n : cap))
        return;
    volatile int *vp = parent;
    int a = pairs[2 * e], b = pairs[2 * e + 1];
    for (long long it = 0; it < kUfSteps; it++) {
        a = uf_find(vp, a);
        b = uf_find(vp, b);
        if (a < 0 || b < 0)
            break;
        if (a == b)
            return;
        const int hi = a > b ? a : b, lo = a > b ? b : a;
        const int old = atomicCAS(parent + hi, hi, lo);
        if (old == hi)
            return;
        a = old;  // hi was hooked meanwhile: continue from its new parent
        b = lo;
    }
    atomicOr(err, ERRB_CAPACITY);
}

__global__ void k_uf_compress(int *parent, int n, int *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const int r = uf_find(parent, i);
    if (r < 0)
        atomicOr(err, ERRB_CAPACITY);
    else
        parent[i] = r;
}

// bottom layer: centre height below one diameter
__global__ void k_bed_seed(const double *__restrict__ x, int n, double D,
                           const int *__restrict__ parent, unsigned char *root_bed)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && x[2 * (long long)n + i] < D)
        root_bed[parent[i]] = 1;
}

__global__ void k_bed_flags(const int *__restrict__ parent,
                            const unsigned char *__restrict__ root_bed, int n,
                            unsigned char *__restrict__ flags, unsigned long long *count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool bed = i < n && root_bed[parent[i]];
    if (i < n)
        flags[i] = bed ? 1 : 0;
    const unsigned m = __ballot_sync(0xffffffffu, bed);
    if ((threadIdx.x & 31) == 0 && m)
        atomicAdd(count, (unsigned long long)__popc(m));
}

struct TrackArgs {
    const unsigned char *bed;  // this state's flags
    const double *x, *u, *om;  // [3][n]
    unsigned char *prev, *salt, *pend;
    double *dep_z, *t_imp, *u_imp, *om_imp;  // [n], [n], [3][n], [3][n]
    int *flag;                 // pass 0: 1 where an event closes
    const int *pos;            // pass 1: its slot
    prs_event *out;
    long long cap;
    int n, started, pass;
    double t, h_r, t_cir;
};

__global__ void k_track(TrackArgs a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > a.n)
        return;
    if (p == a.n) {  // the scan's last entry
        if (a.pass == 0)
            a.flag[p] = 0;
        return;
    }
    const int n = a.n;
    const unsigned char now = a.bed[p];
    const double z = a.x[2 * (long long)n + p];
    if (!a.started) {
        if (a.pass == 0) {
            a.flag[p] = 0;
        } else {
            a.prev[p] = now;
            a.dep_z[p] = z;
            a.salt[p] = 0;
            a.pend[p] = 0;
        }
        return;
    }
    const unsigned char was = a.prev[p];
    const bool closes = was && !now && a.pend[p];
    if (a.pass == 0) {
        a.flag[p] = closes ? 1 : 0;
        return;
    }
    if (!was && !now) {
        if (z - a.dep_z[p] > a.h_r)
            a.salt[p] = 1;
    } else if (!was && now) {
        if (a.salt[p]) {
            a.pend[p] = 1;
            a.t_imp[p] = a.t;
            for (int k = 0; k < 3; k++) {
                a.u_imp[k * n + p] = a.u[k * n + p];
                a.om_imp[k * n + p] = a.om[k * n + p];
            }
        }
        a.salt[p] = 0;
    } else if (was && !now) {
        if (closes && a.pos[p] < a.cap) {
            prs_event e;
            e.particle = p;
            e.rebound = a.t - a.t_imp[p] < a.t_cir ? 1 : 0;
            e.t_impact = a.t_imp[p];
            e.t_departure = a.t;
            for (int k = 0; k < 3; k++) {
                e.u_impact[k] = a.u_imp[k * n + p];
                e.omega_impact[k] = a.om_imp[k * n + p];
                e.u_departure[k] = a.u[k * n + p];
                e.omega_departure[k] = a.om[k * n + p];
            }
            a.out[a.pos[p]] = e;
        }
        a.pend[p] = 0;
        a.dep_z[p] = z;
        a.salt[p] = 0;
    }
    a.prev[p] = now;
}

}  // namespace

void bed_classify(Ctx &c, const int *pairs, long long cap, cudaStream_t s)
{
    const int n = c.n_p;
    const int b = (n + 255) / 256;
    k_uf_init<<<b, 256, 0, s>>>(c.bed_parent, c.bed_root, n);
    const int bl = (int)((cap + 255) / 256);
    k_uf_link<<<bl, 256, 0, s>>>(pairs, reinterpret_cast<const unsigned long long *>(c.d_pairs_n),
                                 cap, c.bed_parent, c.d_err);
    k_uf_compress<<<b, 256, 0, s>>>(c.bed_parent, n, c.d_err);
    k_bed_seed<<<b, 256, 0, s>>>(c.x[c.cur], n, 2.0 * c.R, c.bed_parent, c.bed_root);
    cudaMemsetAsync(c.bed_count, 0, sizeof(unsigned long long), s);
    k_bed_flags<<<b, 256, 0, s>>>(c.bed_parent, c.bed_root, n, c.bed_flags, c.bed_count);
    c.n_launch += 5;
}

void track_saltation(Ctx &c, double t, double h_r, double t_cir, prs_event *out,
                     long long cap, cudaStream_t s)
{
    TrackArgs a{};
    const int n = c.n_p;
    a.bed = c.bed_flags;
    a.x = c.x[c.cur];
    a.u = c.u[c.cur];
    a.om = c.om[c.cur];
    a.prev = c.trk_prev;
    a.salt = c.trk_salt;
    a.pend = c.trk_pend;
    a.dep_z = c.trk_dep_z;
    a.t_imp = c.trk_t_imp;
    a.u_imp = c.trk_u_imp;
    a.om_imp = c.trk_om_imp;
    a.flag = c.trk_flag;
    a.pos = c.trk_pos;
    a.out = out;
    a.cap = cap;
    a.n = n;
    a.started = c.trk_started;
    a.t = t;
    a.h_r = h_r;
    a.t_cir = t_cir;
    const int b = (n + 1 + 255) / 256;
    a.pass = 0;
    k_track<<<b, 256, 0, s>>>(a);
    c.n_launch += 1 + exclusive_scan(c.trk_flag, c.trk_pos, n + 1, c.trk_scan_tmp, s);
    a.pass = 1;
    k_track<<<b, 256, 0, s>>>(a);
    c.n_launch += 1;
    c.trk_started = 1;
}

}  // namespace prs
