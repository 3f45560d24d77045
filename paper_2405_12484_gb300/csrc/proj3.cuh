// Device functions of the per-tet projections (Sec. 7.1, Eq. pd_local,
// Eq. vol_pre), shared by the local step and the adjoint kernels.
//
// SVD: cyclic Jacobi eigen-decomposition of F^T F (Golub & Van Loan,
// "Matrix Computations", the two-sided symmetric Schur rotation), sorted
// eigenvectors W in SO(3), then a Givens QR of F W (the structure used by
// McAdams et al. 2011, "Computing the SVD of 3x3 matrices with minimal
// branching") so that U in SO(3) and the last singular value carries the
// sign of det F; a final one-sided Jacobi rotation of the trailing 2x2 block
// keeps the two smallest singular values accurate when sigma_1 / sigma_3 is
// beyond the FP32 resolution of F^T F.
//
// Volume target: minimise sum (d_i - s_i)^2 s.t. prod d = 1, d_i >= 0.01.
// KKT: (d_i - s_i) d_i = mu for the free targets.  The smallest target
// t = d_3 parameterises every candidate root: mu = t (t - s_3) and
// d_{1,2} = (s_i + sqrt(s_i^2 + 4 mu)) / 2.  On t >= s_3/2 the product is
// increasing (all roots on the + branch: safeguarded Newton); on
// [0.01, s_3/2) d_3 is the - root of its quadratic (scan and bisection of
// every sign change, only where a bound of the product allows a root).  The
// cheapest candidate is kept; the face with d_3 clamped to 0.01 (d_1 d_2 = 100,
// the same construction) is tried when the first face has no feasible point
// or a - root under the clamp; failing both, d = (1e4, 0.01, 0.01).
#pragma once

#include <cuda_runtime.h>

namespace pdg {
namespace proj {

constexpr float kClamp = 0.01f;

// The Jacobi sweeps of the SVD stop after this many (of four) once the
// off-diagonal of F^T F is below the rounding of its diagonal (0: always four)
#ifndef PDG_SVD_EARLY_SWEEP
#define PDG_SVD_EARLY_SWEEP 3
#endif

static __device__ __forceinline__ void jacobi_pair(float& app, float& aqq, float& apq, float& arp, float& arq,
                                            float (&v)[3][3], int p, int q) {
    if (fabsf(apq) < 1e-30f) return;
    float tau = (aqq - app) / (2.0f * apq);
    float t;
    if (fabsf(tau) > 1e18f) {
        t = 0.5f / tau;
    } else {
        t = copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
    }
    float c = rsqrtf(1.0f + t * t);
    float s = t * c;
    app -= t * apq;
    aqq += t * apq;
    apq = 0.0f;
    float rp = c * arp - s * arq;
    float rq = s * arp + c * arq;
    arp = rp;
    arq = rq;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float vp = v[k][p], vq = v[k][q];
        v[k][p] = c * vp - s * vq;
        v[k][q] = s * vp + c * vq;
    }
}

static __device__ __forceinline__ void swap_cols(float (&v)[3][3], int i, int j) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float a = v[k][i];
        v[k][i] = -v[k][j];   // negate one column: det stays +1
        v[k][j] = a;
    }
}

static __device__ __forceinline__ void givens_rows(float (&b)[3][3], float (&u)[3][3], int i, int j, int col) {
    float a = b[i][col], c_ = b[j][col];
    float r2 = a * a + c_ * c_;
    if (r2 <= 1e-38f) return;
    float ir = rsqrtf(r2);
    float c = a * ir, s = c_ * ir;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float bi = b[i][k], bj = b[j][k];
        b[i][k] = c * bi + s * bj;
        b[j][k] = -s * bi + c * bj;
    }
    // U <- U G^T
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float ui = u[k][i], uj = u[k][j];
        u[k][i] = c * ui + s * uj;
        u[k][j] = -s * ui + c * uj;
    }
}

// F = U diag(s) W^T, U, W in SO(3), |s0| >= |s1| >= |s2|, s0, s1 >= 0.
static __device__ __forceinline__ void svd3(const float (&F)[3][3], float (&U)[3][3], float (&s)[3], float (&W)[3][3]) {
    // A = F^T F (symmetric)
    float a00 = 0.f, a01 = 0.f, a02 = 0.f, a11 = 0.f, a12 = 0.f, a22 = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a00 += F[k][0] * F[k][0];
        a01 += F[k][0] * F[k][1];
        a02 += F[k][0] * F[k][2];
        a11 += F[k][1] * F[k][1];
        a12 += F[k][1] * F[k][2];
        a22 += F[k][2] * F[k][2];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) W[i][j] = (i == j) ? 1.f : 0.f;
    // four cyclic sweeps reach FP32 rounding (quadratic convergence); after
    // the third the sweep loop ends once converged (nearly every element),
    // which keeps most warps convergent
#pragma unroll 1
    for (int sweep = 0; sweep < 4; ++sweep) {
        jacobi_pair(a00, a11, a01, a02, a12, W, 0, 1);   // pair (0,1), r = 2
        jacobi_pair(a00, a22, a02, a01, a12, W, 0, 2);   // pair (0,2), r = 1
        jacobi_pair(a11, a22, a12, a01, a02, W, 1, 2);   // pair (1,2), r = 0
#if PDG_SVD_EARLY_SWEEP > 0
        // converged to FP32: the off-diagonal is below rounding of the diagonal
        if (sweep + 1 >= PDG_SVD_EARLY_SWEEP &&
            a01 * a01 + a02 * a02 + a12 * a12 <= 1e-15f * (a00 * a00 + a11 * a11 + a22 * a22))
            break;
#endif
    }
    float l0 = a00, l1 = a11, l2 = a22;
    if (l0 < l1) { float t = l0; l0 = l1; l1 = t; swap_cols(W, 0, 1); }
    if (l0 < l2) { float t = l0; l0 = l2; l2 = t; swap_cols(W, 0, 2); }
    if (l1 < l2) { float t = l1; l1 = l2; l2 = t; swap_cols(W, 1, 2); }
    // B = F W, then QR by Givens rotations: B = U R
    float B[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) B[i][j] = F[i][0] * W[0][j] + F[i][1] * W[1][j] + F[i][2] * W[2][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) U[i][j] = (i == j) ? 1.f : 0.f;
    givens_rows(B, U, 0, 1, 0);
    givens_rows(B, U, 0, 2, 0);
    givens_rows(B, U, 1, 2, 1);
    // When sigma_1 / sigma_3 exceeds ~1e3 the two smallest eigenvalues of F^T F
    // fall below its FP32 rounding, so the Jacobi sweeps leave their
    // eigenvectors mixed and B keeps a trailing 2x2 block.  One-sided Jacobi on
    // that block's two columns (their Gram matrix is free of sigma_1) makes them
    // orthogonal, a Givens rotation re-triangularises, and the pair is re-sorted.
    // (skipped when the off-diagonal is negligible: its effect on s is second order)
    if (fabsf(B[1][2]) > 1e-5f * (fabsf(B[1][1]) + fabsf(B[2][2]))) {
        const float al = B[1][1] * B[1][1], be = B[1][2] * B[1][2] + B[2][2] * B[2][2], ga = B[1][1] * B[1][2];
        const float zeta = (be - al) / (2.f * ga);
        const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
        const float c = rsqrtf(1.f + t * t), sn = c * t;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float b1 = B[k][1], b2 = B[k][2];
            B[k][1] = c * b1 - sn * b2;
            B[k][2] = sn * b1 + c * b2;
            const float w1 = W[k][1], w2 = W[k][2];
            W[k][1] = c * w1 - sn * w2;
            W[k][2] = sn * w1 + c * w2;
        }
        givens_rows(B, U, 1, 2, 1);
        if (fabsf(B[2][2]) > B[1][1]) {
            // swap the pair (one column of each negated keeps both in SO(3)): diag becomes (b22, b11)
            swap_cols(U, 1, 2);
            swap_cols(W, 1, 2);
            const float b11 = B[1][1], b22 = B[2][2];
            B[1][1] = b22;
            B[2][2] = b11;
            if (b22 < 0.f) {   // keep s1 >= 0: flip both columns of U
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    U[k][1] = -U[k][1];
                    U[k][2] = -U[k][2];
                }
                B[1][1] = -B[1][1];
                B[2][2] = -B[2][2];
            }
        }
    }
    s[0] = B[0][0];
    s[1] = B[1][1];
    s[2] = B[2][2];
}

// psi(t) = ln t + sum_k ln r+(sh_k, t (t - st)) - logp, and its derivative.
template <int K>
static __device__ __forceinline__ bool face_eval(const float (&sh)[2], float st, float logp, float t, float& val,
                                          float& dval, float (&d)[2]) {
    float mu = t * (t - st);
    val = logf(t) - logp;
    dval = 1.0f / t;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float disc = fmaxf(sh[k] * sh[k] + 4.0f * mu, 0.0f);
        float sq = sqrtf(disc);
        float dk = 0.5f * (sh[k] + sq);
        ok = ok && (dk >= kClamp);
        d[k] = dk;
        val += logf(fmaxf(dk, 1e-30f));
        if (sq > 0.f) dval += (2.0f * t - st) / (sq * dk);
    }
    return ok;
}

// The "-" roots of the smallest target (rare: strong stretch), out of line so
// that the common path keeps its registers.  Updates the best candidate.
template <int K>
static __device__ __noinline__ void minus_branch(const float (&sh)[2], float st, float logp, float tm, float& best,
                                                 float& t_out, float (&d)[2], bool& have, bool& below) {
    float dv, dd[2];
    auto keep = [&](float t, const float (&dk)[2]) {
        float c = (t - st) * (t - st);
#pragma unroll
        for (int k = 0; k < K; ++k) c += (dk[k] - sh[k]) * (dk[k] - sh[k]);
        if (c < best) {
            best = c;
            t_out = t;
#pragma unroll
            for (int k = 0; k < K; ++k) d[k] = dk[k];
            have = true;
        }
    };
    if (0.5f * st > kClamp) {
        {
            // "-" branch: geometric grid on [0.01, tm], every sign change bisected
            constexpr int kScan = 24;
            const float ratio = powf(tm / kClamp, 1.0f / (kScan - 1));
            float ta = kClamp, va;
            bool oka = face_eval<K>(sh, st, logp, ta, va, dv, dd);
            below = oka && va > 0.0f;
#pragma unroll 1
            for (int j = 1; j < kScan; ++j) {
                const float tb = (j == kScan - 1) ? tm : ta * ratio;
                float vb;
                const bool okb = face_eval<K>(sh, st, logp, tb, vb, dv, dd);
                if (oka && okb && (va <= 0.0f) != (vb <= 0.0f)) {
                    float a = ta, b = tb;
                    const bool a_neg = va <= 0.0f;
#pragma unroll 1
                    for (int it = 0; it < 40 && b - a > 1e-7f * b; ++it) {
                        const float mid = 0.5f * (a + b);
                        float vm;
                        face_eval<K>(sh, st, logp, mid, vm, dv, dd);
                        if ((vm <= 0.0f) == a_neg) a = mid; else b = mid;
                    }
                    const float t = 0.5f * (a + b);
                    float vt;
                    if (face_eval<K>(sh, st, logp, t, vt, dv, dd)) keep(t, dd);
                }
                ta = tb;
                va = vb;
                oka = okb;
            }
        }
    } else if (st > 0.0f) {
        // the whole "-" branch (0, st/2] lies under the clamp: a root there if psi > 0 at its top
        float vf;
        face_eval<K>(sh, st, logp, 0.5f * st, vf, dv, dd);
        below = vf > 0.0f;
    }
}

// One face of the feasible set: free targets sh[0..K) plus the smallest
// target t, product exp(logp).  Candidates (KKT points): the all-"+" root
// (psi increasing on [tm, inf): safeguarded Newton) and the "-" roots of the
// smallest target on [0.01, st/2) (scan of psi and bisection of every sign
// change); the cheapest feasible one is returned in (d, t_out) with its cost.
// The "-" branch is scanned only when psi can reach 0 there: its "+"
// partners are largest at t = 0.01 and t <= st/2, which bounds psi.
// below: psi > 0 at the lower end of the "-" branch, so a "-" root lies
// under the clamp (the optimum may then sit on the face with t clamped).
template <int K>
static __device__ __forceinline__ bool solve_face(const float (&sh)[2], float st, float logp, float t_hi,
                                                  float (&d)[2], float& t_out, float& cost_out, bool& below) {
    float v, dv, dd[2];
    const float tm = fmaxf(0.5f * st, kClamp);
    // at t = tm every + root is >= max(st/2, 0.01) >= 0.01 (equal for a tie sh_k = st), and the
    // + roots grow with t: the + branch is feasible whatever rounding says at the bracket end
    face_eval<K>(sh, st, logp, tm, v, dv, dd);
    bool have = false;
    below = false;
    float best = 3.4e38f;
    auto keep = [&](float t, const float (&dk)[2]) {
        float c = (t - st) * (t - st);
#pragma unroll
        for (int k = 0; k < K; ++k) c += (dk[k] - sh[k]) * (dk[k] - sh[k]);
        if (c < best) {
            best = c;
            t_out = t;
#pragma unroll
            for (int k = 0; k < K; ++k) d[k] = dk[k];
            have = true;
        }
    };
    if (v <= 0.0f) {
        // + branch: bracket [a, b], Newton safeguarded by bisection.  One fixed step from the
        // uniform-scaling guess (no divergence inside a warp; near rest that guess is within
        // O(strain^2) of the root), then the bracketed loop continues, to the tolerance, only
        // for elements not yet converged.
        float a = tm, b = fmaxf(t_hi, tm);
        float prod = st;
#pragma unroll
        for (int k = 0; k < K; ++k) prod *= sh[k];
        float t = (st > 0.f && prod > 0.f) ? st * expf((logp - logf(prod)) / (K + 1)) : 0.5f * (a + b);
        t = fminf(fmaxf(t, a), b);
#pragma unroll 1
        for (int it = 0; it < 1; ++it) {
            face_eval<K>(sh, st, logp, t, v, dv, dd);
            if (v <= 0.0f) a = t; else b = t;
            float tn = t - v / dv;
            if (!(tn > a && tn < b)) tn = 0.5f * (a + b);
            t = tn;
        }
        face_eval<K>(sh, st, logp, t, v, dv, dd);
#pragma unroll 1
        for (int it = 0; it < 40 && fabsf(v) > 2e-6f && (b - a) > 1e-7f * t; ++it) {
            if (v <= 0.0f) a = t; else b = t;
            float tn = t - v / dv;
            if (!(tn > a && tn < b)) tn = 0.5f * (a + b);
            t = tn;
            face_eval<K>(sh, st, logp, t, v, dv, dd);
        }
        keep(t, dd);
    }
    // the "-" branch only where psi can reach 0 on it (strong stretch), or lies under the clamp
    bool scan = st > 0.0f && 0.5f * st <= kClamp;
    if (0.5f * st > kClamp) {
        float bound = logf(0.5f * st) - logp;
        const float mu_top = kClamp * kClamp - st * kClamp;
#pragma unroll
        for (int k = 0; k < K; ++k)
            bound += logf(fmaxf(0.5f * (sh[k] + sqrtf(fmaxf(sh[k] * sh[k] + 4.0f * mu_top, 0.0f))), 1e-30f));
        scan = bound >= 0.0f;
    }
    if (scan) minus_branch<K>(sh, st, logp, tm, best, t_out, d, have, below);
    cost_out = best;
    return have;
}

static __device__ __forceinline__ void volume_targets(const float (&s)[3], float (&dd)[3]) {
    float d[2], t, c2 = 3.4e38f, c1 = 3.4e38f;
    bool below2 = false, below1 = false;
    const float sh2[2] = {s[0], s[1]};
    const bool f2 = solve_face<2>(sh2, s[2], 0.0f, fmaxf(1.0f, s[2] + 1.0f), d, t, c2, below2);
    if (f2) {
        dd[0] = d[0]; dd[1] = d[1]; dd[2] = t;
    }
    // the face with the smallest target clamped: when the unclamped face has no feasible KKT
    // point, or when it has an infeasible "-" root under the clamp
    if (!f2 || below2) {
        const float sh1[2] = {s[0], 0.f};
        const float logp = -logf(kClamp);
        float d1[2], t1;
        if (solve_face<1>(sh1, s[1], logp, fmaxf(10.0f, s[1] + 10.0f), d1, t1, c1, below1)) {
            c1 += (kClamp - s[2]) * (kClamp - s[2]);
            if (!f2 || c1 < c2) {
                dd[0] = d1[0]; dd[1] = t1; dd[2] = kClamp;
                return;
            }
        }
    }
    if (f2) return;
    dd[0] = 1.0f / (kClamp * kClamp);
    dd[1] = kClamp;
    dd[2] = kClamp;
}

// P = U diag(c) W^T
static __device__ __forceinline__ void udwt(const float (&U)[3][3], const float (&c)[3], const float (&W)[3][3],
                                     float (&P)[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            P[i][j] = U[i][0] * c[0] * W[j][0] + U[i][1] * c[1] * W[j][1] + U[i][2] * c[2] * W[j][2];
}

}  // namespace proj
}  // namespace pdg
