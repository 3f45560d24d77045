// PD local step on sm_103a: per-tet deformation gradient, 3x3 SVD, rotation
// and volume targets, and the per-corner right-hand-side contributions.
//
// Paper: Sec. 7.1 (local step; R by polar decomposition through the SVD
// F = U Sigma W^T; V through the three-unknown problem of Eq. vol_pre with
// targets clamped to >= 0.01), Eq. pd_local, Eq. energy (per-element
// gamma_s, gamma_v).
//
// SVD: cyclic Jacobi eigen-decomposition of F^T F (Golub & Van Loan,
// "Matrix Computations", the two-sided symmetric Schur rotation), sorted
// eigenvectors W in SO(3), then a Givens QR of F W (the structure used by
// McAdams et al. 2011, "Computing the SVD of 3x3 matrices with minimal
// branching") so that U in SO(3) and the last singular value carries the
// sign of det F.
//
// Volume target: minimise sum (d_i - s_i)^2 s.t. prod d = 1, d_i >= 0.01.
// KKT: (d_i - s_i) d_i = mu for the free targets.  The smallest target
// t = d_3 parameterises every candidate root: mu = t (t - s_3) and
// d_{1,2} = (s_i + sqrt(s_i^2 + 4 mu)) / 2.  On t >= s_3/2 the product is
// increasing (all roots on the + branch: safeguarded Newton); on
// [0.01, s_3/2) d_3 is the - root of its quadratic (bisection on the sign
// change).  If neither holds, d_3 is clamped to 0.01 and the same
// construction solves d_1 d_2 = 100; failing that d = (1e4, 0.01, 0.01).
#include "pd_internal.h"
#include "proj3.cuh"

namespace pdg {

namespace {

using namespace proj;

__global__ void __launch_bounds__(256) k_project(const float* __restrict__ Fin, int n, float* __restrict__ Rout,
                                                 float* __restrict__ Vout, float* __restrict__ sout) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F[i][j] = Fin[9 * (int64_t)e + 3 * i + j];
    float U[3][3], W[3][3], s[3], d[3], P[3][3];
    svd3(F, U, s, W);
    if (sout) {
        sout[3 * (int64_t)e] = s[0];
        sout[3 * (int64_t)e + 1] = s[1];
        sout[3 * (int64_t)e + 2] = s[2];
    }
    if (Rout) {
        const float one[3] = {1.f, 1.f, 1.f};
        udwt(U, one, W, P);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Rout[9 * (int64_t)e + 3 * i + j] = P[i][j];
    }
    if (Vout) {
        volume_targets(s, d);
        udwt(U, d, W, P);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Vout[9 * (int64_t)e + 3 * i + j] = P[i][j];
    }
}

// geo holds three float4 rows per tet in SoA blocks:
// geo[t] = (g1, ws), geo[n_t + t] = (g2, wv), geo[2 n_t + t] = (g3, 0), with
// g_k the rows of Dm^-1 and ws = V_e gamma_s, wv = V_e gamma_v.
// Output: force[4 t + c] = (ws R + wv V) g_c, g_0 = -(g1 + g2 + g3).
struct LocalIn {
    float4 r1, r2, r3, x0, x1, x2, x3;
};

__device__ __forceinline__ void local_tet(const LocalIn& L, float4* __restrict__ out) {
    const float e1[3] = {L.x1.x - L.x0.x, L.x1.y - L.x0.y, L.x1.z - L.x0.z};
    const float e2[3] = {L.x2.x - L.x0.x, L.x2.y - L.x0.y, L.x2.z - L.x0.z};
    const float e3[3] = {L.x3.x - L.x0.x, L.x3.y - L.x0.y, L.x3.z - L.x0.z};
    const float g1[3] = {L.r1.x, L.r1.y, L.r1.z};
    const float g2[3] = {L.r2.x, L.r2.y, L.r2.z};
    const float g3[3] = {L.r3.x, L.r3.y, L.r3.z};
    float F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F[i][j] = e1[i] * g1[j] + e2[i] * g2[j] + e3[i] * g3[j];
    float U[3][3], W[3][3], s[3], d[3], P[3][3];
    svd3(F, U, s, W);
    volume_targets(s, d);
    const float ws = L.r1.w, wv = L.r2.w;
    const float c[3] = {ws + wv * d[0], ws + wv * d[1], ws + wv * d[2]};
    udwt(U, c, W, P);
    float f1[3], f2[3], f3[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        f1[i] = P[i][0] * g1[0] + P[i][1] * g1[1] + P[i][2] * g1[2];
        f2[i] = P[i][0] * g2[0] + P[i][1] * g2[1] + P[i][2] * g2[2];
        f3[i] = P[i][0] * g3[0] + P[i][1] * g3[1] + P[i][2] * g3[2];
    }
    out[0] = make_float4(-(f1[0] + f2[0] + f3[0]), -(f1[1] + f2[1] + f3[1]), -(f1[2] + f2[2] + f3[2]), 0.f);
    out[1] = make_float4(f1[0], f1[1], f1[2], 0.f);
    out[2] = make_float4(f2[0], f2[1], f2[2], 0.f);
    out[3] = make_float4(f3[0], f3[1], f3[2], 0.f);
}

// kLocalTpt tets per thread (e, e + blockDim.x, ...) in the block's chunk: the
// independent per-tet chains (SVD, volume solve) interleave in one thread.
#ifndef PDG_LOCAL_TPT
#define PDG_LOCAL_TPT 1
#endif
constexpr int kLocalTpt = PDG_LOCAL_TPT;

__global__ void __launch_bounds__(128) k_local(int n_t, const int4* __restrict__ tets,
                                               const float4* __restrict__ geo, const float4* __restrict__ x,
                                               float4* __restrict__ force) {
    pdl_trigger();
    const int base = blockIdx.x * blockDim.x * kLocalTpt + threadIdx.x;
    LocalIn L[kLocalTpt];
    int4 tv[kLocalTpt];
#pragma unroll
    for (int u = 0; u < kLocalTpt; ++u) {
        const int e = min(base + u * (int)blockDim.x, n_t - 1);
        tv[u] = __ldg(&tets[e]);
        L[u].r1 = __ldg(&geo[e]);
        L[u].r2 = __ldg(&geo[n_t + e]);
        L[u].r3 = __ldg(&geo[2 * (int64_t)n_t + e]);
    }
    pdl_wait();   // x comes from the previous solve
#pragma unroll
    for (int u = 0; u < kLocalTpt; ++u) {
        L[u].x0 = x[tv[u].x];
        L[u].x1 = x[tv[u].y];
        L[u].x2 = x[tv[u].z];
        L[u].x3 = x[tv[u].w];
    }
#pragma unroll
    for (int u = 0; u < kLocalTpt; ++u) {
        const int e = base + u * (int)blockDim.x;
        if (e < n_t) local_tet(L[u], force + 4 * (int64_t)e);
    }
}

}  // namespace

void launch_project(const float* F, int n, float* R, float* V, float* sig, cudaStream_t s) {
    if (n <= 0) return;
    k_project<<<(n + 255) / 256, 256, 0, s>>>(F, n, R, V, sig);
    PDG_CHECK_LAUNCH();
}

void launch_local(const pd_mesh* m, const float4* x, float4* force, cudaStream_t s) {
    if (m->n_t <= 0) return;
    launch_pdl(k_local, dim3((m->n_t + 128 * kLocalTpt - 1) / (128 * kLocalTpt)), dim3(128), 0, s, m->n_t, m->d_tets.p,
               m->d_geo.p, x, force);
    PDG_CHECK_LAUNCH();
}

}  // namespace pdg
