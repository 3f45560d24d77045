// FP64 kernels of the adjoint path (Sec. 6.1): the equilibrium residual of
// Eq. g for the Newton steps, the Hessian product of Eq. adjoint_state_solve
// for the refinement of the adjoint state, and the parameter sensitivity
// dL/dgamma = -lambda^T dg/dgamma of Eq. adjoint_state, all evaluated at an
// FP64 state with FP64 rest operators (rows of Dm^-1), volumes and weights.
//
// Why FP64 here: dg/dgamma_e = V_e (F - R(F)) g_c is the strain itself, and
// at strains of 1e-3 the FP32 rounding of positions stored in absolute
// coordinates (1e-8 m on a 0.2 m mesh with 1 cm elements) already moves
// F - R by 1e-4 relative.  The state therefore stays in FP64 through the
// Newton steps (FP64 residual, FP32 preconditioned CG for the correction:
// iterative refinement), and every per-tet term that contracts with the
// adjoint state is formed in FP64.  The linear solves themselves stay FP32
// (the PD subspace solve as preconditioner).
//
// Vectors of 3 doubles per vertex in the library's vertex order; per-tet
// corner terms force64[(4 e + c) * 3 + i]; geo64 holds 12 doubles per tet:
// g1, g2, g3 (rows of Dm^-1), w_s = V_e gamma_s, w_v = V_e gamma_v, V_e.
#include <algorithm>

#include "pd_internal.h"
#include "proj3_64.cuh"

namespace pdg {

namespace {

using namespace proj64;

inline int nb64(int n, int b) { return (n + b - 1) / b; }

struct Tet64 {
    int4 tv;
    double g[4][3];
    double ws, wv, vol;
};

__device__ __forceinline__ void load_tet64(int e, const int4* __restrict__ tets, const double* __restrict__ geo64,
                                           Tet64& T) {
    T.tv = tets[e];
    const double* q = geo64 + 12 * (int64_t)e;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) T.g[k + 1][j] = q[3 * k + j];
#pragma unroll
    for (int j = 0; j < 3; ++j) T.g[0][j] = -(T.g[1][j] + T.g[2][j] + T.g[3][j]);
    T.ws = q[9];
    T.wv = q[10];
    T.vol = q[11];
}

// F = sum_{k>=1} (x_k - x_0) (outer) g_k from an FP64 vertex array
__device__ __forceinline__ void grad64(const Tet64& T, const double* __restrict__ x, double (&F)[3][3]) {
    const int v[4] = {T.tv.x, T.tv.y, T.tv.z, T.tv.w};
    double e[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) e[k][i] = x[3 * (int64_t)v[k + 1] + i] - x[3 * (int64_t)v[0] + i];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F[i][j] = e[0][i] * T.g[1][j] + e[1][i] * T.g[2][j] + e[2][i] * T.g[3][j];
}

// same from an FP32 float4 vertex array (a direction, or the adjoint state)
__device__ __forceinline__ void grad64(const Tet64& T, const float4* __restrict__ x, double (&F)[3][3]) {
    const float4 x0 = x[T.tv.x], x1 = x[T.tv.y], x2 = x[T.tv.z], x3 = x[T.tv.w];
    const double e[3][3] = {{(double)x1.x - x0.x, (double)x1.y - x0.y, (double)x1.z - x0.z},
                            {(double)x2.x - x0.x, (double)x2.y - x0.y, (double)x2.z - x0.z},
                            {(double)x3.x - x0.x, (double)x3.y - x0.y, (double)x3.z - x0.z}};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F[i][j] = e[0][i] * T.g[1][j] + e[1][i] * T.g[2][j] + e[2][i] * T.g[3][j];
}

__device__ __forceinline__ void store_corners64(const double (&P)[3][3], const Tet64& T, double* __restrict__ out) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int i = 0; i < 3; ++i)
            out[3 * c + i] = P[i][0] * T.g[c][0] + P[i][1] * T.g[c][1] + P[i][2] * T.g[c][2];
}

// per-tet elastic force terms of Eq. g: (w_s (F - R) + w_v (F - V)) g_c
__global__ void __launch_bounds__(128) k_grad_local64(int n_t, const int4* __restrict__ tets,
                                                      const double* __restrict__ geo64, const double* __restrict__ x,
                                                      double* __restrict__ force) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_t) return;
    Tet64 T;
    load_tet64(e, tets, geo64, T);
    double F[3][3], U[3][3], W[3][3], s[3], d[3], P[3][3];
    grad64(T, x, F);
    svd3(F, U, s, W);
    volume_targets(s, d);
    const double c[3] = {T.ws * (s[0] - 1.0) + T.wv * (s[0] - d[0]), T.ws * (s[1] - 1.0) + T.wv * (s[1] - d[1]),
                         T.ws * (s[2] - 1.0) + T.wv * (s[2] - d[2])};
    udwt(U, c, W, P);
    store_corners64(P, T, force + 12 * (int64_t)e);
}

// per-tet terms of the Hessian product: d^2E_e[v] = dP(F; dF(v)) g_c
__global__ void __launch_bounds__(128) k_hvp_local64(int n_t, const int4* __restrict__ tets,
                                                     const double* __restrict__ geo64, const double* __restrict__ x,
                                                     const float4* __restrict__ v, double* __restrict__ force) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_t) return;
    Tet64 T;
    load_tet64(e, tets, geo64, T);
    double F[3][3], dF[3][3], U[3][3], W[3][3], s[3], d[3], dP[3][3];
    grad64(T, x, F);
    grad64(T, v, dF);
    svd3(F, U, s, W);
    volume_targets(s, d);
    stress_derivative(U, s, W, d, T.ws, T.wv, dF, dP);
    store_corners64(dP, T, force + 12 * (int64_t)e);
}

// Newton right-hand side: out_i = -float((M/dt^2)(x_i - y_i) + sum_inc force),
// y = xprev + h vprev + h^2 g (free vertices, fixed incidence order)
__global__ void __launch_bounds__(256) k_residual_rhs64(int n_free, const int* __restrict__ inc_ptr,
                                                        const int* __restrict__ inc, const double* __restrict__ force,
                                                        const double* __restrict__ mh2, const double* __restrict__ x,
                                                        const double* __restrict__ xprev,
                                                        const double* __restrict__ vprev, double h, double gx,
                                                        double gy, double gz, float4* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_free) return;
    const double gr[3] = {gx, gy, gz};
    double a[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int64_t q = 3 * (int64_t)i + k;
        a[k] = mh2[i] * ((x[q] - xprev[q]) - h * vprev[q] - h * h * gr[k]);
    }
    for (int k = inc_ptr[i]; k < inc_ptr[i + 1]; ++k) {
        const double* f = force + 3 * (int64_t)inc[k];
        a[0] += f[0];
        a[1] += f[1];
        a[2] += f[2];
    }
    out[i] = make_float4((float)-a[0], (float)-a[1], (float)-a[2], 0.f);
}

// refinement residual of H lambda = rhs: out_i = float(rhs_i - (M/dt^2) lambda_i - sum_inc force)
__global__ void __launch_bounds__(256) k_hvp_residual64(int n_free, const int* __restrict__ inc_ptr,
                                                        const int* __restrict__ inc, const double* __restrict__ force,
                                                        const double* __restrict__ mh2,
                                                        const float4* __restrict__ lam,
                                                        const float4* __restrict__ rhs, float4* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_free) return;
    const float4 l = lam[i], r = rhs[i];
    double a[3] = {(double)r.x - mh2[i] * l.x, (double)r.y - mh2[i] * l.y, (double)r.z - mh2[i] * l.z};
    for (int k = inc_ptr[i]; k < inc_ptr[i + 1]; ++k) {
        const double* f = force + 3 * (int64_t)inc[k];
        a[0] -= f[0];
        a[1] -= f[1];
        a[2] -= f[2];
    }
    out[i] = make_float4((float)a[0], (float)a[1], (float)a[2], 0.f);
}

// dL/dgs[user] -= V_e <F - R, Lambda>, dL/dgv[user] -= V_e <F - V, Lambda>, Lambda = sum_c lambda_c (outer) g_c
__global__ void __launch_bounds__(128) k_grad_gamma64(int n_t, const int4* __restrict__ tets,
                                                      const double* __restrict__ geo64, const double* __restrict__ x,
                                                      const float4* __restrict__ lam,
                                                      const int* __restrict__ user_of_tet, float* __restrict__ gs,
                                                      float* __restrict__ gv) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_t) return;
    Tet64 T;
    load_tet64(e, tets, geo64, T);
    double F[3][3], L[3][3], U[3][3], W[3][3], s[3], d[3];
    grad64(T, x, F);
    grad64(T, lam, L);
    svd3(F, U, s, W);
    volume_targets(s, d);
    // <U diag(c) W^T, L> = sum_i c_i (U^T L W)_ii
    double fs = 0.0, fv = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        double m = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) m += U[a][i] * L[a][b] * W[b][i];
        fs += (s[i] - 1.0) * m;
        fv += (s[i] - d[i]) * m;
    }
    const int u = user_of_tet[e];
    gs[u] = (float)((double)gs[u] - T.vol * fs);
    gv[u] = (float)((double)gv[u] - T.vol * fv);
}

// x64 (+)= float4 -> double, first n entries
__global__ void k_f4_to_d(int n, const float4* __restrict__ a, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 v = a[i];
    out[3 * (int64_t)i] = v.x;
    out[3 * (int64_t)i + 1] = v.y;
    out[3 * (int64_t)i + 2] = v.z;
}

__global__ void k_d_to_f4(int n, const double* __restrict__ a, float4* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = make_float4((float)a[3 * (int64_t)i], (float)a[3 * (int64_t)i + 1], (float)a[3 * (int64_t)i + 2], 0.f);
}

// Newton update on the free vertices: x64 += dx, x32 = float(x64)
__global__ void k_newton_update64(int n_free, const float4* __restrict__ dx, double* __restrict__ x64,
                                  float4* __restrict__ x32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_free) return;
    const float4 d = dx[i];
    double* p = x64 + 3 * (int64_t)i;
    p[0] += d.x;
    p[1] += d.y;
    p[2] += d.z;
    x32[i] = make_float4((float)p[0], (float)p[1], (float)p[2], 0.f);
}

// v64 = (x64 - xprev64) / h; FP32 copies of both (every vertex)
__global__ void k_velocity64(int n_v, const double* __restrict__ x64, const double* __restrict__ xprev64, double ih,
                             double* __restrict__ v64, float4* __restrict__ x32, float4* __restrict__ v32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_v) return;
    double v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int64_t q = 3 * (int64_t)i + k;
        v[k] = (x64[q] - xprev64[q]) * ih;
        v64[q] = v[k];
    }
    x32[i] = make_float4((float)x64[3 * (int64_t)i], (float)x64[3 * (int64_t)i + 1], (float)x64[3 * (int64_t)i + 2],
                         0.f);
    v32[i] = make_float4((float)v[0], (float)v[1], (float)v[2], 0.f);
}

// caller order <-> library order (old_of_new: library vertex -> caller vertex)
__global__ void k_gather64(int n_v, const int* __restrict__ old_of_new, const double* __restrict__ src,
                           double* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_v) return;
    const int64_t o = old_of_new[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) dst[3 * (int64_t)i + k] = src[3 * o + k];
}

__global__ void k_scatter64(int n_v, const int* __restrict__ old_of_new, const double* __restrict__ src,
                            double* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_v) return;
    const int64_t o = old_of_new[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) dst[3 * o + k] = src[3 * (int64_t)i + k];
}

// lam += dlam on the free vertices
__global__ void k_add_f4(int n, const float4* __restrict__ d, float4* __restrict__ x) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = d[i];
    float4 b = x[i];
    b.x += a.x;
    b.y += a.y;
    b.z += a.z;
    x[i] = b;
}

}  // namespace

void launch_grad_local64(const pd_mesh* m, const double* geo64, const double* x64, double* force64, cudaStream_t s) {
    if (m->n_t <= 0) return;
    k_grad_local64<<<nb64(m->n_t, 128), 128, 0, s>>>(m->n_t, m->d_tets.p, geo64, x64, force64);
    PDG_CHECK_LAUNCH();
}

void launch_residual_rhs64(const pd_mesh* m, const double* force64, const double* mh2, const double* x64,
                           const double* xprev64, const double* vprev64, double h, const float g[3], float4* out,
                           cudaStream_t s) {
    if (m->n_free <= 0) return;
    k_residual_rhs64<<<nb64(m->n_free, 256), 256, 0, s>>>(m->n_free, m->d_inc_ptr.p, m->d_inc.p, force64, mh2, x64,
                                                           xprev64, vprev64, h, (double)g[0], (double)g[1],
                                                           (double)g[2], out);
    PDG_CHECK_LAUNCH();
}

void launch_hvp_residual64(const pd_mesh* m, const double* geo64, const double* x64, const float4* lam,
                           const double* mh2, const float4* rhs, double* force64, float4* out, cudaStream_t s) {
    if (m->n_t > 0) {
        k_hvp_local64<<<nb64(m->n_t, 128), 128, 0, s>>>(m->n_t, m->d_tets.p, geo64, x64, lam, force64);
        PDG_CHECK_LAUNCH();
    }
    if (m->n_free <= 0) return;
    k_hvp_residual64<<<nb64(m->n_free, 256), 256, 0, s>>>(m->n_free, m->d_inc_ptr.p, m->d_inc.p, force64, mh2, lam,
                                                           rhs, out);
    PDG_CHECK_LAUNCH();
}

void launch_grad_gamma64(const pd_mesh* m, const double* geo64, const int* user_of_tet, const double* x64,
                         const float4* lam, float* gs, float* gv, cudaStream_t s) {
    if (m->n_t <= 0) return;
    k_grad_gamma64<<<nb64(m->n_t, 128), 128, 0, s>>>(m->n_t, m->d_tets.p, geo64, x64, lam, user_of_tet, gs, gv);
    PDG_CHECK_LAUNCH();
}

void launch_f4_to_d(int n, const float4* a, double* out, cudaStream_t s) {
    if (n <= 0) return;
    k_f4_to_d<<<nb64(n, 256), 256, 0, s>>>(n, a, out);
    PDG_CHECK_LAUNCH();
}

void launch_d_to_f4(int n, const double* a, float4* out, cudaStream_t s) {
    if (n <= 0) return;
    k_d_to_f4<<<nb64(n, 256), 256, 0, s>>>(n, a, out);
    PDG_CHECK_LAUNCH();
}

void launch_newton_update64(int n_free, const float4* dx, double* x64, float4* x32, cudaStream_t s) {
    if (n_free <= 0) return;
    k_newton_update64<<<nb64(n_free, 256), 256, 0, s>>>(n_free, dx, x64, x32);
    PDG_CHECK_LAUNCH();
}

void launch_velocity64(int n_v, const double* x64, const double* xprev64, double h, double* v64, float4* x32,
                       float4* v32, cudaStream_t s) {
    if (n_v <= 0) return;
    k_velocity64<<<nb64(n_v, 256), 256, 0, s>>>(n_v, x64, xprev64, 1.0 / h, v64, x32, v32);
    PDG_CHECK_LAUNCH();
}

void launch_gather64(const pd_mesh* m, const double* src, double* dst, cudaStream_t s) {
    k_gather64<<<nb64(m->n_v, 256), 256, 0, s>>>(m->n_v, m->d_old_of_new.p, src, dst);
    PDG_CHECK_LAUNCH();
}

void launch_scatter64(const pd_mesh* m, const double* src, double* dst, cudaStream_t s) {
    k_scatter64<<<nb64(m->n_v, 256), 256, 0, s>>>(m->n_v, m->d_old_of_new.p, src, dst);
    PDG_CHECK_LAUNCH();
}

void launch_add_f4(int n, const float4* d, float4* x, cudaStream_t s) {
    if (n <= 0) return;
    k_add_f4<<<nb64(n, 256), 256, 0, s>>>(n, d, x);
    PDG_CHECK_LAUNCH();
}

}  // namespace pdg
