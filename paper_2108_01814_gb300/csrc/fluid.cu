// Predictor of a Runge-Kutta fluid sub-step with an explicit viscous
// stand-in (Sec. 2.1). The paper forms, for sub-step k of its RK2 scheme,
//   hat-u^k = u^{k-1} + dt_f [alpha_k H^{k-1} - beta_k (H^{k-2} - grad p^{k-2} / rho_f)]
// with H = -div(uu) + nu lap(u). The stand-in keeps the viscous part of H
// and no pressure: H = nu lap_h(u), the second-order central 7-point
// Laplacian, so per grid point
//   u_out = u_in + dt (alpha H(u_in) - beta H_prev),   H_prev <- H(u_in).
// The direct forcing then adds alpha_k dt f (prs_ibm_step with alpha_k).
//
// Boundaries: periodic axes wrap. On an axis bounded by no-slip walls at 0
// and n h, a component whose points sit half a cell off the walls (offset
// 1/2) takes the mirrored ghost value -u beyond each wall; a component whose
// points sit on the faces (offset 0) has its point 0 on the lower wall,
// held (H = 0, u_out = u_in), and the upper wall point n (not stored) is 0.
//
// One thread per (x, y) column over kPredZ planes, unrolled so that the
// loads of all of them are in flight together (the kernel is bound by HBM
// bandwidth only if enough lines are outstanding per SM); the x and y
// neighbours come from the threads beside it (L1), the z neighbours from
// the same thread's other planes, so DRAM sees each field about once: 4
// words per point (u_in and H read, u_out and H written).
#include <cuda_runtime.h>

#include "prs_internal.cuh"

namespace prs {
namespace {

constexpr int kPredX = 32, kPredY = 8, kPredZ = 8;

template <typename T>
struct PredictArgs {
    int n[3];
    int periodic[3];
    int node[3];  // bounded axis whose points sit on the walls (offset 0)
    T c_lap;      // nu / h^2
    T dt_alpha, dt_beta;
};

// neighbours of index i along one axis: indices and the factors their values
// enter with (1, -1 for the mirrored ghost, 0 for the upper wall point);
// hold: i is a wall point
template <typename T>
__device__ __forceinline__ void axis_nb(int i, int n, int per, int node, int &im, T &fm,
                                        int &ip, T &fp, bool &hold)
{
    im = i - 1;
    ip = i + 1;
    fm = T(1);
    fp = T(1);
    if (i == 0) {
        if (per) {
            im = n - 1;
        } else if (node) {
            hold = true;
            im = 0;
        } else {
            im = 0;
            fm = T(-1);
        }
    }
    if (i == n - 1) {
        if (per) {
            ip = 0;
        } else {
            ip = i;
            fp = node ? T(0) : T(-1);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kPredX *kPredY)
k_predict(const T *__restrict__ u_in, T *__restrict__ u_out, T *__restrict__ H, PredictArgs<T> a)
{
    const int ix = blockIdx.x * kPredX + (threadIdx.x % kPredX);
    const int iy = blockIdx.y * kPredY + (threadIdx.x / kPredX);
    if (ix >= a.n[0] || iy >= a.n[1])
        return;
    const int z0 = blockIdx.z * kPredZ, nzb = min(kPredZ, a.n[2] - z0);
    const long long nx = a.n[0], sxy = (long long)a.n[0] * a.n[1];
    int xm, xp, ym, yp;
    T fxm, fxp, fym, fyp;
    bool hold_xy = false;
    axis_nb(ix, a.n[0], a.periodic[0], a.node[0], xm, fxm, xp, fxp, hold_xy);
    axis_nb(iy, a.n[1], a.periodic[1], a.node[1], ym, fym, yp, fyp, hold_xy);
    const long long col = iy * nx + ix;
    const long long oxm = iy * nx + xm, oxp = iy * nx + xp;
    const long long oym = ym * nx + ix, oyp = yp * nx + ix;
#pragma unroll
    for (int j = 0; j < kPredZ; j++) {
        const int iz = z0 + j;
        if (j >= nzb)  // predicated, so the loads of all planes can issue together
            continue;
        int zm, zp;
        T fzm, fzp;
        bool hold = hold_xy;
        axis_nb(iz, a.n[2], a.periodic[2], a.node[2], zm, fzm, zp, fzp, hold);
        const long long pz = iz * sxy;
        const T uc = __ldg(u_in + pz + col);
        T Hn = T(0);
        if (!hold) {
            const T sx = fxm * __ldg(u_in + pz + oxm) + fxp * __ldg(u_in + pz + oxp);
            const T sy = fym * __ldg(u_in + pz + oym) + fyp * __ldg(u_in + pz + oyp);
            const T sz = fzm * __ldg(u_in + zm * sxy + col) + fzp * __ldg(u_in + zp * sxy + col);
            Hn = a.c_lap * (((sx + sy) + sz) - T(6) * uc);
        }
        // beta = 0 (first sub-step): H_prev is not read, whatever it holds
        const T Hp = a.dt_beta != T(0) ? H[pz + col] : T(0);
        u_out[pz + col] = hold ? uc : uc + (a.dt_alpha * Hn - a.dt_beta * Hp);
        H[pz + col] = Hn;
    }
}

// 16-byte vectors of V points along x (float: 4, double: 2)
template <typename T>
struct Vec;
template <>
struct Vec<float> {
    static constexpr int V = 4;
    using type = float4;
};
template <>
struct Vec<double> {
    static constexpr int V = 2;
    using type = double2;
};

template <typename T, int V>
__device__ __forceinline__ void ld_vec(const T *p, T (&v)[V])
{
    using VT = typename Vec<T>::type;
    const VT q = __ldg(reinterpret_cast<const VT *>(p));
    const T *e = reinterpret_cast<const T *>(&q);
#pragma unroll
    for (int k = 0; k < V; k++)
        v[k] = e[k];
}

template <typename T, int V>
__device__ __forceinline__ void st_vec(T *p, const T (&v)[V])
{
    using VT = typename Vec<T>::type;
    VT q;
    T *e = reinterpret_cast<T *>(&q);
#pragma unroll
    for (int k = 0; k < V; k++)
        e[k] = v[k];
    *reinterpret_cast<VT *>(p) = q;
}

// The same with V points along x per thread, 16-byte loads and stores
// (nx a multiple of V, 16-byte aligned fields). The centre and H vectors of
// all kPredZV planes are loaded first, so that a warp has 2 kPredZV 512-byte
// requests to DRAM in flight; the neighbour loads that follow hit L1 / L2.
constexpr int kPredZV = 4;

template <typename T>
__global__ void __launch_bounds__(kPredX *kPredY)
k_predict_vec(const T *__restrict__ u_in, T *__restrict__ u_out, T *__restrict__ H,
              PredictArgs<T> a)
{
    constexpr int V = Vec<T>::V;
    const int tx = blockIdx.x * kPredX + (threadIdx.x % kPredX);
    const int iy = blockIdx.y * kPredY + (threadIdx.x / kPredX);
    const int x0 = tx * V;
    if (x0 >= a.n[0] || iy >= a.n[1])
        return;
    const int z0 = blockIdx.z * kPredZV, nzb = min(kPredZV, a.n[2] - z0);
    const long long nx = a.n[0], sxy = (long long)a.n[0] * a.n[1];
    // x: neighbours of the vector's first and last points
    int xm, xp, dum;
    T fxm, fxp, fdum;
    bool hold_x0 = false, hold_dum = false;
    axis_nb(x0, a.n[0], a.periodic[0], a.node[0], xm, fxm, dum, fdum, hold_x0);
    axis_nb(x0 + V - 1, a.n[0], a.periodic[0], a.node[0], dum, fdum, xp, fxp, hold_dum);
    int ym, yp;
    T fym, fyp;
    bool hold_y = false;
    axis_nb(iy, a.n[1], a.periodic[1], a.node[1], ym, fym, yp, fyp, hold_y);
    const long long col = iy * nx + x0;
    T c[kPredZV][V], hp[kPredZV][V];
#pragma unroll
    for (int j = 0; j < kPredZV; j++) {
        if (j < nzb) {
            const long long pz = (z0 + j) * sxy;
            ld_vec<T, V>(u_in + pz + col, c[j]);
            if (a.dt_beta != T(0))
                ld_vec<T, V>(H + pz + col, hp[j]);
            else
#pragma unroll
                for (int k = 0; k < V; k++)
                    hp[j][k] = T(0);
        }
    }
#pragma unroll
    for (int j = 0; j < kPredZV; j++) {
        if (j >= nzb)
            continue;
        const int iz = z0 + j;
        int zm, zp;
        T fzm, fzp;
        bool hold_z = false;
        axis_nb(iz, a.n[2], a.periodic[2], a.node[2], zm, fzm, zp, fzp, hold_z);
        const long long pz = iz * sxy;
        T um[V], up[V], ys[V], yn[V];
        ld_vec<T, V>(u_in + zm * sxy + col, um);
        ld_vec<T, V>(u_in + zp * sxy + col, up);
        ld_vec<T, V>(u_in + pz + ym * nx + x0, ys);
        ld_vec<T, V>(u_in + pz + yp * nx + x0, yn);
        const T left = fxm * __ldg(u_in + pz + iy * nx + xm);
        const T right = fxp * __ldg(u_in + pz + iy * nx + xp);
        T uo[V], Hn[V];
#pragma unroll
        for (int k = 0; k < V; k++) {
            const T sx = (k == 0 ? left : c[j][k - 1]) + (k == V - 1 ? right : c[j][k + 1]);
            const T sy = fym * ys[k] + fyp * yn[k];
            const T sz = fzm * um[k] + fzp * up[k];
            const bool hold = hold_y || hold_z || (k == 0 && hold_x0);
            Hn[k] = hold ? T(0) : a.c_lap * (((sx + sy) + sz) - T(6) * c[j][k]);
            uo[k] = hold ? c[j][k] : c[j][k] + (a.dt_alpha * Hn[k] - a.dt_beta * hp[j][k]);
        }
        st_vec<T, V>(u_out + pz + col, uo);
        st_vec<T, V>(H + pz + col, Hn);
    }
}

template <typename T>
void predict_t(Ctx &c, int comp, const void *u_in, void *u_out, void *H, double nu, double dt,
               double alpha, double beta, cudaStream_t s)
{
    PredictArgs<T> a;
    for (int k = 0; k < 3; k++) {
        a.n[k] = c.g.n[k];
        a.periodic[k] = c.g.periodic[k];
        a.node[k] = !c.g.periodic[k] && c.g.off[comp * 3 + k] == 0.0;
    }
    a.c_lap = (T)(nu / (c.g.h * c.g.h));
    a.dt_alpha = (T)(dt * alpha);
    a.dt_beta = (T)(dt * beta);
    constexpr int V = Vec<T>::V;
    const bool vec = c.g.n[0] % V == 0 && reinterpret_cast<uintptr_t>(u_in) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(u_out) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(H) % 16 == 0;
    if (vec) {
        const dim3 grid((c.g.n[0] / V + kPredX - 1) / kPredX, (c.g.n[1] + kPredY - 1) / kPredY,
                        (c.g.n[2] + kPredZV - 1) / kPredZV);
        k_predict_vec<T><<<grid, kPredX * kPredY, 0, s>>>((const T *)u_in, (T *)u_out, (T *)H,
                                                          a);
    } else {
        const dim3 grid((c.g.n[0] + kPredX - 1) / kPredX, (c.g.n[1] + kPredY - 1) / kPredY,
                        (c.g.n[2] + kPredZ - 1) / kPredZ);
        k_predict<T><<<grid, kPredX * kPredY, 0, s>>>((const T *)u_in, (T *)u_out, (T *)H, a);
    }
    c.n_launch += 1;
}

}  // namespace

void fluid_predict(Ctx &c, int comp, const void *u_in, void *u_out, void *H, double nu,
                   double dt, double alpha, double beta, cudaStream_t s)
{
    if (c.precision == PRS_FP64)
        predict_t<double>(c, comp, u_in, u_out, H, nu, dt, alpha, beta, s);
    else
        predict_t<float>(c, comp, u_in, u_out, H, nu, dt, alpha, beta, s);
}

}  // namespace prs
