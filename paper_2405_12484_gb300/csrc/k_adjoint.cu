// Kernels of the adjoint path (Sec. 6.1: Eq. g, Eq. pxpgamma,
// Eq. adjoint_state, Eq. adjoint_state_solve), all per tet or per vertex:
//
//  * k_grad_local / k_assemble_residual: g = (M/dt^2)(x - y) + grad E(x),
//    the equilibrium residual of Eq. g, with per-tet contributions
//    (ws (F - R) + wv (F - V)) g_c = U diag(ws (s - 1) + wv (s - d)) W^T g_c;
//  * k_hvp_local / k_assemble_hvp: H v = (M/dt^2) v + sum_e d^2E_e[v], with
//    d^2E_e/dF^2 = V_e [gs (I - dR/dF) + gv (I - dV/dF)] from the derivative
//    of an isotropic matrix function P = U diag(f(s)) W^T:  A = U^T dF W,
//    (U^T dP W)_ii = sum_k (df_i/ds_k) A_kk and, for i != j,
//    alpha_ij (A_ij + A_ji)/2 + beta_ij (A_ij - A_ji)/2 with
//    alpha_ij = (f_i - f_j)/(s_i - s_j), beta_ij = (f_i + f_j)/(s_i + s_j);
//  * k_grad_gamma: dL/dgamma_e -= V_e <F - R, Lambda_e> (and <F - V, .>),
//    Lambda_e = sum_c lambda_c (outer) g_c (the adjoint's own gradient);
//  * deterministic FP64 dot products and the PCG vector updates.
#include <algorithm>

#include "pd_internal.h"
#include "proj3.cuh"

namespace pdg {

namespace {

using namespace proj;

struct Tet {
    int4 tv;
    float g[4][3];   // corner vectors, g0 = -(g1 + g2 + g3)
    float ws, wv;
};

__device__ __forceinline__ Tet load_tet(int e, int n_t, const int4* __restrict__ tets, const float4* __restrict__ geo) {
    Tet T;
    T.tv = __ldg(&tets[e]);
    const float4 r1 = __ldg(&geo[e]);
    const float4 r2 = __ldg(&geo[n_t + e]);
    const float4 r3 = __ldg(&geo[2 * (int64_t)n_t + e]);
    T.g[1][0] = r1.x; T.g[1][1] = r1.y; T.g[1][2] = r1.z;
    T.g[2][0] = r2.x; T.g[2][1] = r2.y; T.g[2][2] = r2.z;
    T.g[3][0] = r3.x; T.g[3][1] = r3.y; T.g[3][2] = r3.z;
#pragma unroll
    for (int j = 0; j < 3; ++j) T.g[0][j] = -(T.g[1][j] + T.g[2][j] + T.g[3][j]);
    T.ws = r1.w;
    T.wv = r2.w;
    return T;
}

// F = sum_c x_c (outer) g_c, evaluated as sum_{k>=1} (x_k - x_0) (outer) g_k
__device__ __forceinline__ void tet_grad(const Tet& T, const float4* __restrict__ x, float (&F)[3][3]) {
    const float4 x0 = x[T.tv.x], x1 = x[T.tv.y], x2 = x[T.tv.z], x3 = x[T.tv.w];
    const float e1[3] = {x1.x - x0.x, x1.y - x0.y, x1.z - x0.z};
    const float e2[3] = {x2.x - x0.x, x2.y - x0.y, x2.z - x0.z};
    const float e3[3] = {x3.x - x0.x, x3.y - x0.y, x3.z - x0.z};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F[i][j] = e1[i] * T.g[1][j] + e2[i] * T.g[2][j] + e3[i] * T.g[3][j];
}

__device__ __forceinline__ void store_corners(const float (&P)[3][3], const Tet& T, float4* __restrict__ out) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float f[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) f[i] = P[i][0] * T.g[c][0] + P[i][1] * T.g[c][1] + P[i][2] * T.g[c][2];
        out[c] = make_float4(f[0], f[1], f[2], 0.f);
    }
}

__global__ void __launch_bounds__(128) k_grad_local(int n_t, const int4* __restrict__ tets,
                                                    const float4* __restrict__ geo, const float4* __restrict__ x,
                                                    float4* __restrict__ force) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_t) return;
    const Tet T = load_tet(e, n_t, tets, geo);
    float F[3][3], U[3][3], W[3][3], s[3], d[3], P[3][3];
    tet_grad(T, x, F);
    svd3(F, U, s, W);
    volume_targets(s, d);
    const float c[3] = {T.ws * (s[0] - 1.f) + T.wv * (s[0] - d[0]), T.ws * (s[1] - 1.f) + T.wv * (s[1] - d[1]),
                        T.ws * (s[2] - 1.f) + T.wv * (s[2] - d[2])};
    udwt(U, c, W, P);
    store_corners(P, T, force + 4 * (int64_t)e);
}

// Jacobian J = dd/ds of the volume targets on the free (unclamped) set.
__device__ __forceinline__ void volume_jacobian(const float (&s)[3], const float (&d)[3], float (&J)[3][3],
                                                bool (&fr)[3], float (&sq)[3]) {
    float a[3], S = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        fr[i] = d[i] > kClamp * (1.f + 1e-5f);
        sq[i] = 2.f * d[i] - s[i];   // + branch: sqrt(s^2 + 4 mu) > 0, - branch: < 0
        float den = sq[i];
        if (fabsf(den) < 1e-12f) den = copysignf(1e-12f, den);
        a[i] = fr[i] ? 1.f / den : 0.f;
        S += fr[i] ? a[i] / d[i] : 0.f;
    }
    const float iS = (S != 0.f) ? 1.f / S : 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) J[i][k] = (fr[i] && fr[k]) ? ((i == k ? a[i] * d[i] : 0.f) - a[i] * a[k] * iS) : 0.f;
}

__global__ void __launch_bounds__(128) k_hvp_local(int n_t, const int4* __restrict__ tets,
                                                   const float4* __restrict__ geo, const float4* __restrict__ x,
                                                   const float4* __restrict__ v, float4* __restrict__ force) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_t) return;
    const Tet T = load_tet(e, n_t, tets, geo);
    float F[3][3], U[3][3], W[3][3], s[3], d[3], dF[3][3];
    tet_grad(T, x, F);
    tet_grad(T, v, dF);
    svd3(F, U, s, W);
    volume_targets(s, d);
    float J[3][3], sq[3];
    bool fr[3];
    volume_jacobian(s, d, J, fr, sq);
    // A = U^T dF W
    float A[3][3], T1[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) T1[i][j] = dF[i][0] * W[0][j] + dF[i][1] * W[1][j] + dF[i][2] * W[2][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) A[i][j] = U[0][i] * T1[0][j] + U[1][i] * T1[1][j] + U[2][i] * T1[2][j];
    // B = ws B_R + wv B_V (in the singular frame)
    float B[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float diag = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) diag += J[i][k] * A[k][k];
        B[i][i] = T.wv * diag;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (i == j) continue;
            const float sym = 0.5f * (A[i][j] + A[j][i]);
            const float skw = 0.5f * (A[i][j] - A[j][i]);
            float ssum = s[i] + s[j];
            if (fabsf(ssum) < 1e-6f) ssum = copysignf(1e-6f, ssum);
            const float betaR = 2.f / ssum;
            const float betaV = (d[i] + d[j]) / ssum;
            float alphaV;
            if (fr[i] && fr[j] && sq[i] > 0.f && sq[j] > 0.f) {
                // both on the + branch: (d_i - d_j)/(s_i - s_j) without cancellation
                alphaV = 0.5f * (1.f + (s[i] + s[j]) / (sq[i] + sq[j]));
            } else if (fabsf(s[i] - s[j]) > 1e-6f * fmaxf(1.f, fabsf(s[i]))) {
                alphaV = (d[i] - d[j]) / (s[i] - s[j]);
            } else {
                alphaV = J[i][i] - J[i][j];
            }
            B[i][j] = T.ws * (betaR * skw) + T.wv * (alphaV * sym + betaV * skw);
        }
    // dP = (ws + wv) dF - U B W^T
    float UB[3][3], dP[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) UB[i][j] = U[i][0] * B[0][j] + U[i][1] * B[1][j] + U[i][2] * B[2][j];
    const float wsum = T.ws + T.wv;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            dP[i][j] = wsum * dF[i][j] - (UB[i][0] * W[j][0] + UB[i][1] * W[j][1] + UB[i][2] * W[j][2]);
    store_corners(dP, T, force + 4 * (int64_t)e);
}

// out_i = sign * (mh2_i * (x_i - y_i) + sum_inc force), y_i = xprev_i + h vprev_i + h^2 g (free vertices)
__global__ void __launch_bounds__(256) k_assemble_residual(int n_free, const int* __restrict__ inc_ptr,
                                                           const int* __restrict__ inc,
                                                           const float4* __restrict__ force,
                                                           const float* __restrict__ mh2,
                                                           const float4* __restrict__ x,
                                                           const float4* __restrict__ xprev,
                                                           const float4* __restrict__ vprev, float h, float gx,
                                                           float gy, float gz, float sign, float4* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_free) return;
    const float4 xi = x[i], xp = xprev[i], vp = vprev[i];
    const float h2 = h * h;
    const float m = mh2[i];
    // x - y = (x - x*) - h v* - h^2 g
    float ax = m * ((xi.x - xp.x) - h * vp.x - h2 * gx);
    float ay = m * ((xi.y - xp.y) - h * vp.y - h2 * gy);
    float az = m * ((xi.z - xp.z) - h * vp.z - h2 * gz);
    for (int k = inc_ptr[i]; k < inc_ptr[i + 1]; ++k) {
        const float4 f = force[inc[k]];
        ax += f.x; ay += f.y; az += f.z;
    }
    out[i] = make_float4(sign * ax, sign * ay, sign * az, 0.f);
}

// out_i = mh2_i v_i + sum_inc force (free vertices)
__global__ void __launch_bounds__(256) k_assemble_hvp(int n_free, const int* __restrict__ inc_ptr,
                                                      const int* __restrict__ inc, const float4* __restrict__ force,
                                                      const float* __restrict__ mh2, const float4* __restrict__ v,
                                                      float4* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_free) return;
    const float4 vi = v[i];
    const float m = mh2[i];
    float ax = m * vi.x, ay = m * vi.y, az = m * vi.z;
    for (int k = inc_ptr[i]; k < inc_ptr[i + 1]; ++k) {
        const float4 f = force[inc[k]];
        ax += f.x; ay += f.y; az += f.z;
    }
    out[i] = make_float4(ax, ay, az, 0.f);
}

// dL/dgs[t_user] -= V_e <F - R, Lambda>, dL/dgv[t_user] -= V_e <F - V, Lambda>
__global__ void __launch_bounds__(128) k_grad_gamma(int n_t, const int4* __restrict__ tets,
                                                    const float4* __restrict__ geo, const float* __restrict__ vol,
                                                    const float4* __restrict__ x, const float4* __restrict__ lam,
                                                    const int* __restrict__ user_of_tet, float* __restrict__ gs,
                                                    float* __restrict__ gv) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_t) return;
    const Tet T = load_tet(e, n_t, tets, geo);
    float F[3][3], L[3][3], U[3][3], W[3][3], s[3], d[3];
    tet_grad(T, x, F);
    tet_grad(T, lam, L);
    svd3(F, U, s, W);
    volume_targets(s, d);
    // <U diag(c) W^T, L> = sum_i c_i (U^T L W)_ii
    float fs = 0.f, fv = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float m = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) m += U[a][i] * L[a][b] * W[b][i];
        fs += (s[i] - 1.f) * m;
        fv += (s[i] - d[i]) * m;
    }
    const int u = user_of_tet[e];
    gs[u] -= vol[e] * fs;
    gv[u] -= vol[e] * fv;
}

// ---- deterministic FP64 dot product over the free vertices (x, y, z components)
constexpr int kDotBlocks = 512;

__global__ void __launch_bounds__(256) k_dot_partial(int n, const float4* __restrict__ a, const float4* __restrict__ b,
                                                     double* __restrict__ partial) {
    __shared__ double sm[256];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 u = a[i], v = b[i];
        acc += (double)u.x * v.x + (double)u.y * v.y + (double)u.z * v.z;
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

// mode 0: sc[dst] = sum; mode 1: alpha = sc[0] / sum (sc[1] = sum, sc[2] = alpha);
// mode 2: beta = sum / sc[0], sc[0] = sum (sc[3] = beta)
__global__ void __launch_bounds__(256) k_dot_final(int nb, const double* __restrict__ partial, double* __restrict__ sc,
                                                   int mode, int dst) {
    __shared__ double sm[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double v = sm[0];
    if (mode == 0) {
        sc[dst] = v;
    } else if (mode == 1) {
        sc[1] = v;
        sc[2] = (fabs(v) > 1e-300) ? sc[0] / v : 0.0;
    } else {
        sc[3] = (fabs(sc[0]) > 1e-300) ? v / sc[0] : 0.0;
        sc[0] = v;
    }
}

// x += alpha p ; r -= alpha Ap  (alpha = sc[2])
__global__ void k_cg_update(int n, const double* __restrict__ sc, const float4* __restrict__ p,
                            const float4* __restrict__ Ap, float4* __restrict__ x, float4* __restrict__ r) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float al = (float)sc[2];
    const float4 pi = p[i], api = Ap[i];
    float4 xi = x[i], ri = r[i];
    xi.x += al * pi.x; xi.y += al * pi.y; xi.z += al * pi.z;
    ri.x -= al * api.x; ri.y -= al * api.y; ri.z -= al * api.z;
    x[i] = xi;
    r[i] = ri;
}

// p = z + beta p (beta = sc[3]); beta_zero: p = z
__global__ void k_cg_direction(int n, const double* __restrict__ sc, const float4* __restrict__ z,
                               float4* __restrict__ p, int beta_zero) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float be = beta_zero ? 0.f : (float)sc[3];
    const float4 zi = z[i], pi = p[i];
    p[i] = make_float4(zi.x + be * pi.x, zi.y + be * pi.y, zi.z + be * pi.z, 0.f);
}

// rhs = dLdx + mh2 (2 lam1 - lam2)  (free vertices)
__global__ void k_adj_rhs(int n, const float4* __restrict__ dldx, const float* __restrict__ mh2,
                          const float4* __restrict__ lam1, const float4* __restrict__ lam2, float4* __restrict__ rhs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float m = mh2[i];
    const float4 a = dldx[i], l1 = lam1[i], l2 = lam2[i];
    rhs[i] = make_float4(a.x + m * (2.f * l1.x - l2.x), a.y + m * (2.f * l1.y - l2.y), a.z + m * (2.f * l1.z - l2.z),
                         0.f);
}

// ---- Gauss-Newton (Sec. 6.2, Eq. gn / Eq. agn): dg/dgamma and its transpose
// With x fixed, the columns of B = dg/dgamma of element e are
// V_e (F - R) g_c (gamma_s) and V_e (F - V) g_c (gamma_v) at its corners c.
// k_gn_setup stores Ts = V_e (F - R), Tv = V_e (F - V) once per direction
// (9 planes of n_t floats each, plane k = row-major entry k), so that every
// product B v and B^T nu is a memory-bound pass without an SVD.
__global__ void __launch_bounds__(128) k_gn_setup(int n_t, const int4* __restrict__ tets,
                                                  const float4* __restrict__ geo, const float* __restrict__ vol,
                                                  const float4* __restrict__ x, float* __restrict__ Ts,
                                                  float* __restrict__ Tv) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_t) return;
    const Tet T = load_tet(e, n_t, tets, geo);
    float F[3][3], U[3][3], W[3][3], s[3], d[3], Ps[3][3], Pv[3][3];
    tet_grad(T, x, F);
    svd3(F, U, s, W);
    volume_targets(s, d);
    const float ve = vol[e];
    const float cs[3] = {ve * (s[0] - 1.f), ve * (s[1] - 1.f), ve * (s[2] - 1.f)};
    const float cv[3] = {ve * (s[0] - d[0]), ve * (s[1] - d[1]), ve * (s[2] - d[2])};
    udwt(U, cs, W, Ps);
    udwt(U, cv, W, Pv);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            Ts[(int64_t)(3 * i + j) * n_t + e] = Ps[i][j];
            Tv[(int64_t)(3 * i + j) * n_t + e] = Pv[i][j];
        }
}

// corner forces of B v: (v_s Ts + v_v Tv) g_c; v = [v_s | v_v] in the caller's tet order.
__global__ void __launch_bounds__(128) k_gn_bv(int n_t, const float4* __restrict__ geo, const float* __restrict__ Ts,
                                               const float* __restrict__ Tv, const int* __restrict__ user_of_tet,
                                               const float* __restrict__ v, float4* __restrict__ force) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_t) return;
    Tet T;
    const float4 r1 = __ldg(&geo[e]);
    const float4 r2 = __ldg(&geo[n_t + e]);
    const float4 r3 = __ldg(&geo[2 * (int64_t)n_t + e]);
    T.g[1][0] = r1.x; T.g[1][1] = r1.y; T.g[1][2] = r1.z;
    T.g[2][0] = r2.x; T.g[2][1] = r2.y; T.g[2][2] = r2.z;
    T.g[3][0] = r3.x; T.g[3][1] = r3.y; T.g[3][2] = r3.z;
#pragma unroll
    for (int j = 0; j < 3; ++j) T.g[0][j] = -(T.g[1][j] + T.g[2][j] + T.g[3][j]);
    const int u = user_of_tet[e];
    const float vs = v[u], vv = v[n_t + u];
    float P[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            P[i][j] = vs * Ts[(int64_t)(3 * i + j) * n_t + e] + vv * Tv[(int64_t)(3 * i + j) * n_t + e];
    store_corners(P, T, force + 4 * (int64_t)e);
}

// out_i = sum_inc force (free vertices)
__global__ void __launch_bounds__(256) k_assemble_sum(int n_free, const int* __restrict__ inc_ptr,
                                                         const int* __restrict__ inc, const float4* __restrict__ force,
                                                         float4* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_free) return;
    float ax = 0.f, ay = 0.f, az = 0.f;
    for (int k = inc_ptr[i]; k < inc_ptr[i + 1]; ++k) {
        const float4 f = force[inc[k]];
        ax += f.x; ay += f.y; az += f.z;
    }
    out[i] = make_float4(ax, ay, az, 0.f);
}

// x *= 1 / sqrt(sc[idx]) (x = 0 when sc[idx] <= 0); free vertices
__global__ void k_normalize_f4(int n, const double* __restrict__ sc, int idx, float4* __restrict__ x) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double nn = sc[idx];
    const float f = nn > 0.0 ? (float)(1.0 / sqrt(nn)) : 0.f;
    float4 a = x[i];
    x[i] = make_float4(a.x * f, a.y * f, a.z * f, 0.f);
}

// B^T nu: out_s[u] = c <Ts, N>, out_v[u] = c <Tv, N>, N = sum_c nu_c (outer) g_c,
// c = gs * sqrt(sc[i1] sc[i2]); entries of inactive parameters are 0.
__global__ void __launch_bounds__(128) k_gn_btv(int n_t, const int4* __restrict__ tets, const float4* __restrict__ geo,
                                                const float* __restrict__ Ts, const float* __restrict__ Tv,
                                                const int* __restrict__ user_of_tet, const float4* __restrict__ nu,
                                                const uint8_t* __restrict__ active, const double* __restrict__ sc,
                                                int i1, int i2, float gs, float* __restrict__ out) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_t) return;
    const Tet T = load_tet(e, n_t, tets, geo);
    float N[3][3];
    tet_grad(T, nu, N);
    float as = 0.f, av = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            as += Ts[(int64_t)(3 * i + j) * n_t + e] * N[i][j];
            av += Tv[(int64_t)(3 * i + j) * n_t + e] * N[i][j];
        }
    const double p = sc[i1] * sc[i2];
    const float c = gs * (p > 0.0 ? (float)sqrt(p) : 0.f);
    const int u = user_of_tet[e];
    out[u] = (active && !active[u]) ? 0.f : c * as;
    out[n_t + u] = (active && !active[n_t + u]) ? 0.f : c * av;
}

// ---- parameter-space vectors (2 n_t floats) of the outer CG and the fitting loop
// Scalars (FP64, one array): see GnScalar.
enum GnScalar : int { G_RR = 0, G_PAP, G_ALPHA, G_BETA, G_KAPPA, G_GG, G_N1, G_N2, G_TMP, G_MAX, G_COUNT };

constexpr int kPBlocks = 256;

// partial sums of a.b (FP64) or, with mode 1, of max_j |a_j| / b_j over b_j > 0
__global__ void __launch_bounds__(256) k_pdot_partial(int n, const float* __restrict__ a, const float* __restrict__ b,
                                                      const uint8_t* __restrict__ mask, int mode,
                                                      double* __restrict__ partial) {
    __shared__ double sm[256];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (mask && !mask[i]) continue;
        if (mode == 0) {
            acc += (double)a[i] * (double)b[i];
        } else {
            const double r = b[i] > 0.f ? fabs((double)a[i]) / (double)b[i] : 0.0;
            acc = r > acc ? r : acc;
        }
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            sm[threadIdx.x] = mode == 0 ? sm[threadIdx.x] + sm[threadIdx.x + w]
                                        : (sm[threadIdx.x + w] > sm[threadIdx.x] ? sm[threadIdx.x + w] : sm[threadIdx.x]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

// op 0: sc[dst] = v; op 1 (alpha): sc[PAP] = v, sc[ALPHA] = sc[RR] / v (0 unless v > 0);
// op 2 (beta): sc[BETA] = v / sc[RR] (0 unless sc[RR] > 0), sc[RR] = v;
// op 3 (kappa): sc[KAPPA] = kr * v / sc[RR] (0 unless sc[RR] > 0)
__global__ void __launch_bounds__(256) k_pdot_final(int nb, const double* __restrict__ partial, int mode, int op,
                                                    int dst, double kr, double* __restrict__ sc) {
    __shared__ double sm[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const double v = partial[i];
        acc = mode == 0 ? acc + v : (v > acc ? v : acc);
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            sm[threadIdx.x] = mode == 0 ? sm[threadIdx.x] + sm[threadIdx.x + w]
                                        : (sm[threadIdx.x + w] > sm[threadIdx.x] ? sm[threadIdx.x + w] : sm[threadIdx.x]);
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double v = sm[0];
    if (op == 0) {
        sc[dst] = v;
    } else if (op == 1) {
        sc[G_PAP] = v;
        sc[G_ALPHA] = (v > 0.0 && isfinite(v)) ? sc[G_RR] / v : 0.0;
    } else if (op == 2) {
        sc[G_BETA] = sc[G_RR] > 0.0 ? v / sc[G_RR] : 0.0;
        sc[G_RR] = v;
    } else if (op == 4) {
        sc[dst] += v;   // accumulated (a loss summed over time steps)
    } else {
        sc[G_KAPPA] = sc[G_RR] > 0.0 ? kr * v / sc[G_RR] : 0.0;
    }
}

// tied parameterisation gamma_s = theta, gamma_v = ratio theta:
// dL/dtheta = scale (dL/dgamma_s + ratio dL/dgamma_v), in FP64, scale from the device (or 1)
__global__ void k_tied_gradient(int n, const float* __restrict__ gs, const float* __restrict__ gv, double ratio,
                                const double* __restrict__ scale, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double f = scale ? scale[0] : 1.0;
    out[i] = (float)(((double)gs[i] + ratio * (double)gv[i]) * f);
}

// r = p = -g / |g| on the active parameters (0 elsewhere); d = 0
__global__ void k_gn_init(int n, const float* __restrict__ g, const uint8_t* __restrict__ active,
                          const double* __restrict__ sc, float* __restrict__ r, float* __restrict__ p,
                          float* __restrict__ d) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double gg = sc[G_GG];
    const float f = gg > 0.0 ? (float)(-1.0 / sqrt(gg)) : 0.f;
    const float v = (active && !active[i]) ? 0.f : f * g[i];
    r[i] = v;
    p[i] = v;
    d[i] = 0.f;
}

// Ap = q + kappa p
__global__ void k_gn_ap(int n, const double* __restrict__ sc, const float* __restrict__ q, const float* __restrict__ p,
                        float* __restrict__ ap) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    ap[i] = q[i] + (float)sc[G_KAPPA] * p[i];
}

// d += alpha p ; r -= alpha Ap
__global__ void k_gn_update(int n, const double* __restrict__ sc, const float* __restrict__ p,
                            const float* __restrict__ ap, float* __restrict__ d, float* __restrict__ r) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float al = (float)sc[G_ALPHA];
    d[i] += al * p[i];
    r[i] -= al * ap[i];
}

// p = r + beta p
__global__ void k_gn_pdir(int n, const double* __restrict__ sc, const float* __restrict__ r, float* __restrict__ p) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    p[i] = r[i] + (float)sc[G_BETA] * p[i];
}

// x *= sqrt(sc[idx]) (mode 0) or x *= -1 / sc[idx] (mode 1, 0 when sc[idx] <= 0); masked entries -> 0
__global__ void k_pscale(int n, const double* __restrict__ sc, int idx, int mode, const uint8_t* __restrict__ active,
                         const float* __restrict__ src, float* __restrict__ x) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = sc[idx];
    const float f = mode == 0 ? (v > 0.0 ? (float)sqrt(v) : 0.f) : (v > 0.0 ? (float)(-1.0 / v) : 0.f);
    x[i] = (active && !active[i]) ? 0.f : f * src[i];
}

// d = raw, with components of cached (clamped) parameters that would decrease set to 0
__global__ void k_clamp_dir(int n, const float* __restrict__ raw, const uint8_t* __restrict__ clamped,
                            float* __restrict__ d) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float r = raw[i];
    d[i] = (clamped[i] && r < 0.f) ? 0.f : r;
}

// trial = gamma + alpha d; negative components -> floor, neg = 1 there
__global__ void k_project(int n, const float* __restrict__ gamma, const float* __restrict__ d, float alpha, float fl,
                          float* __restrict__ trial, uint8_t* __restrict__ neg) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float t = gamma[i] + alpha * d[i];
    const bool ng = t < 0.f;
    trial[i] = ng ? fl : t;
    neg[i] = ng ? 1 : 0;
}

// gamma = trial; clamped |= neg
__global__ void k_accept(int n, const float* __restrict__ trial, const uint8_t* __restrict__ neg,
                         float* __restrict__ gamma, uint8_t* __restrict__ clamped) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    gamma[i] = trial[i];
    clamped[i] = (clamped[i] || neg[i]) ? 1 : 0;
}

// pivot candidate: clamped, not pivoted, raw < 0, gamma at the floor; key = gamma + raw.
// Partial argmin per block (ties -> smaller index); index -1 when none.
__global__ void __launch_bounds__(256) k_pivot_partial(int n, const float* __restrict__ gamma,
                                                       const float* __restrict__ raw,
                                                       const uint8_t* __restrict__ clamped,
                                                       const uint8_t* __restrict__ active, float fl,
                                                       double* __restrict__ pval, int* __restrict__ pidx) {
    __shared__ double sv[256];
    __shared__ int si[256];
    double best = 0.0;
    int bi = -1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const bool cand = clamped[i] && active[i] && raw[i] < 0.f && gamma[i] <= fl * (1.f + 1e-6f);
        if (!cand) continue;
        const double key = (double)gamma[i] + (double)raw[i];
        if (bi < 0 || key < best || (key == best && i < bi)) {
            best = key;
            bi = i;
        }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const int j = si[threadIdx.x + w];
            const int k = si[threadIdx.x];
            if (j >= 0 && (k < 0 || sv[threadIdx.x + w] < sv[threadIdx.x] ||
                           (sv[threadIdx.x + w] == sv[threadIdx.x] && j < k))) {
                sv[threadIdx.x] = sv[threadIdx.x + w];
                si[threadIdx.x] = j;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        pval[blockIdx.x] = sv[0];
        pidx[blockIdx.x] = si[0];
    }
}

__global__ void __launch_bounds__(256) k_pivot_final(int nb, const double* __restrict__ pval,
                                                     const int* __restrict__ pidx, int* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double best = 0.0;
    int bi = -1;
    for (int b = 0; b < nb; ++b) {
        const int j = pidx[b];
        if (j < 0) continue;
        if (bi < 0 || pval[b] < best || (pval[b] == best && j < bi)) {
            best = pval[b];
            bi = j;
        }
    }
    *out = bi;
}

// out[i] = sign * a[i], 0 on inactive parameters (parameter vectors)
__global__ void k_pcopy(int n, float sign, const float* __restrict__ a, const uint8_t* __restrict__ active,
                        float* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = (active && !active[i]) ? 0.f : sign * a[i];
}

// pose misfit: diff = x - xhat on free vertices -> dL/dx = 2 diff, partial sums of |diff|^2
__global__ void __launch_bounds__(256) k_misfit(int n_free, const float4* __restrict__ x,
                                                const float4* __restrict__ xhat, float4* __restrict__ dldx,
                                                double* __restrict__ partial) {
    __shared__ double sm[256];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_free; i += gridDim.x * blockDim.x) {
        const float4 a = x[i], b = xhat[i];
        const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
        if (dldx) dldx[i] = make_float4(2.f * dx, 2.f * dy, 2.f * dz, 0.f);
        acc += (double)dx * dx + (double)dy * dy + (double)dz * dz;
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

// ---- reduced coordinates gamma = diag(H, H) q (Eq. q2gamma); H column-major n_t x r
// out[b] = sum_t H[k][t] w[half n_t + t], b = half r + k; one block per output, fixed order
__global__ void __launch_bounds__(256) k_basis_t(int n_t, int r, const float* __restrict__ H,
                                                 const float* __restrict__ w, double* __restrict__ out) {
    __shared__ double sm[256];
    const int b = blockIdx.x, half = b / r, k = b % r;
    const float* h = H + (int64_t)k * n_t;
    const float* v = w + (int64_t)half * n_t;
    double acc = 0.0;
    for (int t = threadIdx.x; t < n_t; t += blockDim.x) acc += (double)h[t] * (double)v[t];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[b] = sm[0];
}

// out[half n_t + t] = sum_k H[k][t] q[half r + k]
__global__ void k_basis_apply(int n_t, int r, const float* __restrict__ H, const double* __restrict__ q,
                              float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * n_t) return;
    const int half = i / n_t, t = i % n_t;
    double acc = 0.0;
    for (int k = 0; k < r; ++k) acc += (double)H[(int64_t)k * n_t + t] * q[half * r + k];
    out[i] = (float)acc;
}

// out = column j of diag(H, H)
__global__ void k_basis_col(int n_t, int r, const float* __restrict__ H, int j, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * n_t) return;
    const int half = i / n_t, t = i % n_t;
    out[i] = (half == j / r) ? H[(int64_t)(j % r) * n_t + t] : 0.f;
}

// *count += number of a[i] < fl
__global__ void k_count_below(int n, const float* __restrict__ a, float fl, int* __restrict__ count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool below = i < n && a[i] < fl;
    const unsigned m = __ballot_sync(0xffffffffu, below);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(count, __popc(m));
}

inline int nb(int n, int b) { return (n + b - 1) / b; }

}  // namespace

void launch_grad_local(const pd_mesh* m, const float4* x, float4* force, cudaStream_t s) {
    k_grad_local<<<nb(m->n_t, 128), 128, 0, s>>>(m->n_t, m->d_tets.p, m->d_geo.p, x, force);
    PDG_CHECK_LAUNCH();
}

void launch_assemble_residual(const pd_mesh* m, const float4* force, const float4* x, const float4* xprev,
                              const float4* vprev, float h, const float g[3], float sign, float4* out,
                              cudaStream_t s) {
    if (m->n_free <= 0) return;
    k_assemble_residual<<<nb(m->n_free, 256), 256, 0, s>>>(m->n_free, m->d_inc_ptr.p, m->d_inc.p, force, m->d_mh2.p,
                                                           x, xprev, vprev, h, g[0], g[1], g[2], sign, out);
    PDG_CHECK_LAUNCH();
}

void launch_hvp(const pd_mesh* m, const float4* x, const float4* v, float4* force, float4* out, cudaStream_t s) {
    k_hvp_local<<<nb(m->n_t, 128), 128, 0, s>>>(m->n_t, m->d_tets.p, m->d_geo.p, x, v, force);
    PDG_CHECK_LAUNCH();
    if (m->n_free <= 0) return;
    k_assemble_hvp<<<nb(m->n_free, 256), 256, 0, s>>>(m->n_free, m->d_inc_ptr.p, m->d_inc.p, force, m->d_mh2.p, v,
                                                      out);
    PDG_CHECK_LAUNCH();
}

void launch_grad_gamma(const pd_mesh* m, const float* vol, const int* user_of_tet, const float4* x,
                       const float4* lam, float* gs, float* gv, cudaStream_t s) {
    k_grad_gamma<<<nb(m->n_t, 128), 128, 0, s>>>(m->n_t, m->d_tets.p, m->d_geo.p, vol, x, lam, user_of_tet, gs, gv);
    PDG_CHECK_LAUNCH();
}

int dot_blocks() { return kDotBlocks; }

void launch_dot(int n, const float4* a, const float4* b, double* partial, double* sc, int mode, int dst,
                cudaStream_t s) {
    const int blocks = std::max(1, std::min(kDotBlocks, nb(n, 256)));
    k_dot_partial<<<blocks, 256, 0, s>>>(n, a, b, partial);
    PDG_CHECK_LAUNCH();
    k_dot_final<<<1, 256, 0, s>>>(blocks, partial, sc, mode, dst);
    PDG_CHECK_LAUNCH();
}

void launch_cg_update(int n, const double* sc, const float4* p, const float4* Ap, float4* x, float4* r,
                      cudaStream_t s) {
    if (n <= 0) return;
    k_cg_update<<<nb(n, 256), 256, 0, s>>>(n, sc, p, Ap, x, r);
    PDG_CHECK_LAUNCH();
}

void launch_cg_direction(int n, const double* sc, const float4* z, float4* p, int beta_zero, cudaStream_t s) {
    if (n <= 0) return;
    k_cg_direction<<<nb(n, 256), 256, 0, s>>>(n, sc, z, p, beta_zero);
    PDG_CHECK_LAUNCH();
}

void launch_adj_rhs(int n, const float4* dldx, const float* mh2, const float4* lam1, const float4* lam2, float4* rhs,
                    cudaStream_t s) {
    if (n <= 0) return;
    k_adj_rhs<<<nb(n, 256), 256, 0, s>>>(n, dldx, mh2, lam1, lam2, rhs);
    PDG_CHECK_LAUNCH();
}

// ---- Gauss-Newton launchers
int gn_scalar_count() { return G_COUNT; }
int gn_partial_blocks() { return kPBlocks; }

void launch_gn_setup(const pd_mesh* m, const float* vol, const float4* x, float* Ts, float* Tv, cudaStream_t s) {
    k_gn_setup<<<nb(m->n_t, 128), 128, 0, s>>>(m->n_t, m->d_tets.p, m->d_geo.p, vol, x, Ts, Tv);
    PDG_CHECK_LAUNCH();
}

// out (free vertices) = B v
void launch_gn_bv(const pd_mesh* m, const float* Ts, const float* Tv, const int* user_of_tet, const float* v,
                  float4* force, float4* out, cudaStream_t s) {
    k_gn_bv<<<nb(m->n_t, 128), 128, 0, s>>>(m->n_t, m->d_geo.p, Ts, Tv, user_of_tet, v, force);
    PDG_CHECK_LAUNCH();
    if (m->n_free <= 0) return;
    k_assemble_sum<<<nb(m->n_free, 256), 256, 0, s>>>(m->n_free, m->d_inc_ptr.p, m->d_inc.p, force, out);
    PDG_CHECK_LAUNCH();
}

void launch_normalize_f4(int n, const double* sc, int idx, float4* x, cudaStream_t s) {
    if (n <= 0) return;
    k_normalize_f4<<<nb(n, 256), 256, 0, s>>>(n, sc, idx, x);
    PDG_CHECK_LAUNCH();
}

void launch_gn_btv(const pd_mesh* m, const float* Ts, const float* Tv, const int* user_of_tet, const float4* nu,
                   const uint8_t* active, const double* sc, int i1, int i2, float gs, float* out, cudaStream_t s) {
    k_gn_btv<<<nb(m->n_t, 128), 128, 0, s>>>(m->n_t, m->d_tets.p, m->d_geo.p, Ts, Tv, user_of_tet, nu, active, sc,
                                             i1, i2, gs, out);
    PDG_CHECK_LAUNCH();
}

// parameter-space reduction into sc: op as k_pdot_final; mode 0 = dot, 1 = max |a|/b
void launch_pdot(int n, const float* a, const float* b, const uint8_t* mask, int mode, int op, int dst, double kr,
                 double* partial, double* sc, cudaStream_t s) {
    const int blocks = std::max(1, std::min(kPBlocks, nb(n, 256)));
    k_pdot_partial<<<blocks, 256, 0, s>>>(n, a, b, mask, mode, partial);
    PDG_CHECK_LAUNCH();
    k_pdot_final<<<1, 256, 0, s>>>(blocks, partial, mode, op, dst, kr, sc);
    PDG_CHECK_LAUNCH();
}

void launch_gn_init(int n, const float* g, const uint8_t* active, const double* sc, float* r, float* p, float* d,
                    cudaStream_t s) {
    k_gn_init<<<nb(n, 256), 256, 0, s>>>(n, g, active, sc, r, p, d);
    PDG_CHECK_LAUNCH();
}

void launch_gn_ap(int n, const double* sc, const float* q, const float* p, float* ap, cudaStream_t s) {
    k_gn_ap<<<nb(n, 256), 256, 0, s>>>(n, sc, q, p, ap);
    PDG_CHECK_LAUNCH();
}

void launch_gn_update(int n, const double* sc, const float* p, const float* ap, float* d, float* r, cudaStream_t s) {
    k_gn_update<<<nb(n, 256), 256, 0, s>>>(n, sc, p, ap, d, r);
    PDG_CHECK_LAUNCH();
}

void launch_gn_pdir(int n, const double* sc, const float* r, float* p, cudaStream_t s) {
    k_gn_pdir<<<nb(n, 256), 256, 0, s>>>(n, sc, r, p);
    PDG_CHECK_LAUNCH();
}

void launch_pscale(int n, const double* sc, int idx, int mode, const uint8_t* active, const float* src, float* x,
                   cudaStream_t s) {
    k_pscale<<<nb(n, 256), 256, 0, s>>>(n, sc, idx, mode, active, src, x);
    PDG_CHECK_LAUNCH();
}

void launch_clamp_dir(int n, const float* raw, const uint8_t* clamped, float* d, cudaStream_t s) {
    k_clamp_dir<<<nb(n, 256), 256, 0, s>>>(n, raw, clamped, d);
    PDG_CHECK_LAUNCH();
}

void launch_project(int n, const float* gamma, const float* d, float alpha, float fl, float* trial, uint8_t* neg,
                    cudaStream_t s) {
    k_project<<<nb(n, 256), 256, 0, s>>>(n, gamma, d, alpha, fl, trial, neg);
    PDG_CHECK_LAUNCH();
}

void launch_accept(int n, const float* trial, const uint8_t* neg, float* gamma, uint8_t* clamped, cudaStream_t s) {
    k_accept<<<nb(n, 256), 256, 0, s>>>(n, trial, neg, gamma, clamped);
    PDG_CHECK_LAUNCH();
}

void launch_pick_pivot(int n, const float* gamma, const float* raw, const uint8_t* clamped, const uint8_t* active,
                       float fl, double* pval, int* pidx, int* out, cudaStream_t s) {
    const int blocks = std::max(1, std::min(kPBlocks, nb(n, 256)));
    k_pivot_partial<<<blocks, 256, 0, s>>>(n, gamma, raw, clamped, active, fl, pval, pidx);
    PDG_CHECK_LAUNCH();
    k_pivot_final<<<1, 32, 0, s>>>(blocks, pval, pidx, out);
    PDG_CHECK_LAUNCH();
}

void launch_pcopy(int n, float sign, const float* a, const uint8_t* active, float* out, cudaStream_t s) {
    k_pcopy<<<nb(n, 256), 256, 0, s>>>(n, sign, a, active, out);
    PDG_CHECK_LAUNCH();
}

void launch_basis_t(int n_t, int r, const float* H, const float* w, double* out, cudaStream_t s) {
    k_basis_t<<<2 * r, 256, 0, s>>>(n_t, r, H, w, out);
    PDG_CHECK_LAUNCH();
}

void launch_basis_apply(int n_t, int r, const float* H, const double* q, float* out, cudaStream_t s) {
    k_basis_apply<<<nb(2 * n_t, 256), 256, 0, s>>>(n_t, r, H, q, out);
    PDG_CHECK_LAUNCH();
}

void launch_basis_col(int n_t, int r, const float* H, int j, float* out, cudaStream_t s) {
    k_basis_col<<<nb(2 * n_t, 256), 256, 0, s>>>(n_t, r, H, j, out);
    PDG_CHECK_LAUNCH();
}

void launch_count_below(int n, const float* a, float fl, int* count, cudaStream_t s) {
    PDG_CUDA(cudaMemsetAsync(count, 0, sizeof(int), s));
    k_count_below<<<nb(n, 256), 256, 0, s>>>(n, a, fl, count);
    PDG_CHECK_LAUNCH();
}

// loss partial sums into partial[0..blocks), then sc[dst] = loss (or += loss when accumulate)
void launch_misfit(int n_free, const float4* x, const float4* xhat, float4* dldx, double* partial, double* sc, int dst,
                   cudaStream_t s, bool accumulate) {
    const int blocks = std::max(1, std::min(kPBlocks, nb(n_free, 256)));
    k_misfit<<<blocks, 256, 0, s>>>(n_free, x, xhat, dldx, partial);
    PDG_CHECK_LAUNCH();
    k_pdot_final<<<1, 256, 0, s>>>(blocks, partial, 0, accumulate ? 4 : 0, dst, 0.0, sc);
    PDG_CHECK_LAUNCH();
}

void launch_tied_gradient(int n, const float* gs, const float* gv, double ratio, const double* scale, float* out,
                          cudaStream_t s) {
    if (n <= 0) return;
    k_tied_gradient<<<nb(n, 256), 256, 0, s>>>(n, gs, gv, ratio, scale, out);
    PDG_CHECK_LAUNCH();
}

}  // namespace pdg
