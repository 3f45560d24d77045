// FP64 per-tet projections and their derivatives for the adjoint path
// (Sec. 6.1: the equilibrium residual of Eq. g, the Hessian of the elastic
// energy in Eq. adjoint_state_solve and the parameter sensitivity of
// Eq. pxpgamma), at the accuracy the adjoint gradient needs: with strains of
// 1e-3 and below, F - R(F) carries the strain itself, which FP32 rounding of
// F, R or the singular values would cover with relative errors of 1e-4 and
// more.
//
// Same constructions as the FP32 local step (proj3.cuh), in double and run
// to FP64 convergence:
//  * SVD: cyclic Jacobi eigen-decomposition of F^T F (Golub & Van Loan, the
//    two-sided symmetric Schur rotation) until its off-diagonal is below
//    FP64 rounding of the diagonal, eigenvectors W sorted and kept in SO(3),
//    then Givens QR of F W, so U in SO(3) and s_3 carries sign(det F);
//  * volume target (Eq. vol_pre): minimise sum (d_i - s_i)^2 s.t.
//    prod d = 1, d_i >= 0.01, through the KKT roots (d_i - s_i) d_i = mu
//    parameterised by the smallest target t: on the unclamped face the all-"+"
//    root (safeguarded Newton) and every "-" root of d_3 (scan + bisection),
//    the cheapest kept; the face with d_3 clamped to 0.01 (d_1 d_2 = 100, the
//    same way) when the first has no feasible point or a "-" root under the
//    clamp; else (1e4, 0.01, 0.01);
//  * derivative of the isotropic matrix functions R(F) and V(F)
//    (P = U diag(f(s)) W^T): with A = U^T dF W the singular-frame entries
//    are sum_k J_ik A_kk on the diagonal and
//    alpha_ij (A_ij + A_ji)/2 + beta_ij (A_ij - A_ji)/2 off it,
//    alpha_ij = (f_i - f_j)/(s_i - s_j), beta_ij = (f_i + f_j)/(s_i + s_j);
//    J = dd/ds from differentiating the KKT conditions on the free targets.
// Every function is __host__ __device__ and uses only <cmath> operations.
#pragma once

#include <cmath>

#include <cuda_runtime.h>

namespace pdg {
namespace proj64 {

constexpr double kClamp = 0.01;

__host__ __device__ inline void jacobi_pair(double& app, double& aqq, double& apq, double& arp, double& arq,
                                            double (&v)[3][3], int p, int q) {
    if (apq == 0.0) return;
    const double tau = (aqq - app) / (2.0 * apq);
    double t;
    if (fabs(tau) > 1e150) {
        t = 0.5 / tau;
    } else {
        t = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
    }
    const double c = 1.0 / sqrt(1.0 + t * t);
    const double s = t * c;
    app -= t * apq;
    aqq += t * apq;
    apq = 0.0;
    const double rp = c * arp - s * arq;
    const double rq = s * arp + c * arq;
    arp = rp;
    arq = rq;
    for (int k = 0; k < 3; ++k) {
        const double vp = v[k][p], vq = v[k][q];
        v[k][p] = c * vp - s * vq;
        v[k][q] = s * vp + c * vq;
    }
}

__host__ __device__ inline void swap_cols(double (&v)[3][3], int i, int j) {
    for (int k = 0; k < 3; ++k) {
        const double a = v[k][i];
        v[k][i] = -v[k][j];   // one column negated: det stays +1
        v[k][j] = a;
    }
}

__host__ __device__ inline void givens_rows(double (&b)[3][3], double (&u)[3][3], int i, int j, int col) {
    const double a = b[i][col], c_ = b[j][col];
    const double r = hypot(a, c_);
    if (r == 0.0) return;
    const double c = a / r, s = c_ / r;
    for (int k = 0; k < 3; ++k) {
        const double bi = b[i][k], bj = b[j][k];
        b[i][k] = c * bi + s * bj;
        b[j][k] = -s * bi + c * bj;
    }
    for (int k = 0; k < 3; ++k) {   // U <- U G^T
        const double ui = u[k][i], uj = u[k][j];
        u[k][i] = c * ui + s * uj;
        u[k][j] = -s * ui + c * uj;
    }
}

// F = U diag(s) W^T with U, W in SO(3), |s0| >= |s1| >= |s2|, s0, s1 >= 0.
__host__ __device__ inline void svd3(const double (&F)[3][3], double (&U)[3][3], double (&s)[3], double (&W)[3][3]) {
    double a00 = 0.0, a01 = 0.0, a02 = 0.0, a11 = 0.0, a12 = 0.0, a22 = 0.0;
    for (int k = 0; k < 3; ++k) {
        a00 += F[k][0] * F[k][0];
        a01 += F[k][0] * F[k][1];
        a02 += F[k][0] * F[k][2];
        a11 += F[k][1] * F[k][1];
        a12 += F[k][1] * F[k][2];
        a22 += F[k][2] * F[k][2];
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) W[i][j] = (i == j) ? 1.0 : 0.0;
    // quadratic convergence: a handful of sweeps reach FP64 rounding
    for (int sweep = 0; sweep < 12; ++sweep) {
        const double off = a01 * a01 + a02 * a02 + a12 * a12;
        if (off <= 1e-34 * (a00 * a00 + a11 * a11 + a22 * a22)) break;
        jacobi_pair(a00, a11, a01, a02, a12, W, 0, 1);
        jacobi_pair(a00, a22, a02, a01, a12, W, 0, 2);
        jacobi_pair(a11, a22, a12, a01, a02, W, 1, 2);
    }
    double l0 = a00, l1 = a11, l2 = a22;
    if (l0 < l1) { const double t = l0; l0 = l1; l1 = t; swap_cols(W, 0, 1); }
    if (l0 < l2) { const double t = l0; l0 = l2; l2 = t; swap_cols(W, 0, 2); }
    if (l1 < l2) { const double t = l1; l1 = l2; l2 = t; swap_cols(W, 1, 2); }
    double B[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) B[i][j] = F[i][0] * W[0][j] + F[i][1] * W[1][j] + F[i][2] * W[2][j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) U[i][j] = (i == j) ? 1.0 : 0.0;
    givens_rows(B, U, 0, 1, 0);
    givens_rows(B, U, 0, 2, 0);
    givens_rows(B, U, 1, 2, 1);
    // trailing 2x2 block left by eigenvalues of F^T F below its rounding
    // (sigma_1 / sigma_3 beyond ~1e8): one-sided Jacobi on its two columns,
    // a Givens rotation, and the pair re-sorted
    if (B[1][2] != 0.0) {
        const double al = B[1][1] * B[1][1], be = B[1][2] * B[1][2] + B[2][2] * B[2][2], ga = B[1][1] * B[1][2];
        const double zeta = (be - al) / (2.0 * ga);
        const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
        for (int k = 0; k < 3; ++k) {
            const double b1 = B[k][1], b2 = B[k][2];
            B[k][1] = c * b1 - sn * b2;
            B[k][2] = sn * b1 + c * b2;
            const double w1 = W[k][1], w2 = W[k][2];
            W[k][1] = c * w1 - sn * w2;
            W[k][2] = sn * w1 + c * w2;
        }
        givens_rows(B, U, 1, 2, 1);
        if (fabs(B[2][2]) > B[1][1]) {
            swap_cols(U, 1, 2);
            swap_cols(W, 1, 2);
            const double b11 = B[1][1], b22 = B[2][2];
            B[1][1] = b22;
            B[2][2] = b11;
            if (b22 < 0.0) {
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

// psi(t) = ln t + sum_k ln r+(sh_k, t (t - st)) - logp and its derivative; d[k] = the + roots.
template <int K>
__host__ __device__ inline bool face_eval(const double (&sh)[2], double st, double logp, double t, double& val,
                                          double& dval, double (&d)[2]) {
    const double mu = t * (t - st);
    val = log(t) - logp;
    dval = 1.0 / t;
    bool ok = true;
    for (int k = 0; k < K; ++k) {
        const double disc = fmax(sh[k] * sh[k] + 4.0 * mu, 0.0);
        const double sq = sqrt(disc);
        const double dk = 0.5 * (sh[k] + sq);
        ok = ok && (dk >= kClamp);
        d[k] = dk;
        val += log(fmax(dk, 1e-300));
        if (sq > 0.0) dval += (2.0 * t - st) / (sq * dk);
    }
    return ok;
}

// One face: free targets sh[0..K) plus the smallest target t, product
// exp(logp).  Candidates: the all-"+" root (psi increasing on [tm, inf):
// safeguarded Newton) and the "-" roots of the smallest target on
// [0.01, st/2) (geometric scan of psi, bisection of every sign change), the
// "-" branch only when the bound of psi there (its "+" partners are largest
// at t = 0.01, t <= st/2) reaches 0.  The cheapest is returned with its cost;
// below: a "-" root lies under the clamp.
template <int K>
__host__ __device__ inline bool solve_face(const double (&sh)[2], double st, double logp, double t_hi, double (&d)[2],
                                           double& t_out, double& cost_out, bool& below) {
    double v, dv, dd[2];
    const double tm = fmax(0.5 * st, kClamp);
    // at t = tm every + root is >= max(st/2, 0.01) >= 0.01 (equal for a tie sh_k = st), and the
    // + roots grow with t: the + branch is feasible whatever rounding says at the bracket end
    face_eval<K>(sh, st, logp, tm, v, dv, dd);
    bool have = false;
    below = false;
    double best = 1e300;
    auto keep = [&](double t, const double (&dk)[2]) {
        double c = (t - st) * (t - st);
        for (int k = 0; k < K; ++k) c += (dk[k] - sh[k]) * (dk[k] - sh[k]);
        if (c < best) {
            best = c;
            t_out = t;
            for (int k = 0; k < K; ++k) d[k] = dk[k];
            have = true;
        }
    };
    if (v <= 0.0) {
        double a = tm, b = fmax(t_hi, tm);
        double prod = st;
        for (int k = 0; k < K; ++k) prod *= sh[k];
        double t = (st > 0.0 && prod > 0.0) ? st * exp((logp - log(prod)) / (K + 1)) : 0.5 * (a + b);
        t = fmin(fmax(t, a), b);
        face_eval<K>(sh, st, logp, t, v, dv, dd);
        for (int it = 0; it < 200 && fabs(v) > 1e-15 && (b - a) > 1e-16 * t; ++it) {
            if (v <= 0.0) a = t; else b = t;
            double tn = t - v / dv;
            if (!(tn > a && tn < b)) tn = 0.5 * (a + b);
            t = tn;
            face_eval<K>(sh, st, logp, t, v, dv, dd);
        }
        keep(t, dd);
    }
    if (0.5 * st > kClamp) {
        double bound = log(0.5 * st) - logp;
        const double mu_top = kClamp * kClamp - st * kClamp;
        for (int k = 0; k < K; ++k)
            bound += log(fmax(0.5 * (sh[k] + sqrt(fmax(sh[k] * sh[k] + 4.0 * mu_top, 0.0))), 1e-300));
        if (bound >= 0.0) {
            const int kScan = 64;
            const double ratio = pow(tm / kClamp, 1.0 / (kScan - 1));
            double ta = kClamp, va;
            bool oka = face_eval<K>(sh, st, logp, ta, va, dv, dd);
            below = oka && va > 0.0;
            for (int j = 1; j < kScan; ++j) {
                const double tb = (j == kScan - 1) ? tm : ta * ratio;
                double vb;
                const bool okb = face_eval<K>(sh, st, logp, tb, vb, dv, dd);
                if (oka && okb && (va <= 0.0) != (vb <= 0.0)) {
                    double a = ta, b = tb;
                    const bool a_neg = va <= 0.0;
                    for (int it = 0; it < 200 && b - a > 1e-16 * b; ++it) {
                        const double mid = 0.5 * (a + b);
                        double vm;
                        face_eval<K>(sh, st, logp, mid, vm, dv, dd);
                        if ((vm <= 0.0) == a_neg) a = mid; else b = mid;
                    }
                    const double t = 0.5 * (a + b);
                    double vt;
                    if (face_eval<K>(sh, st, logp, t, vt, dv, dd)) keep(t, dd);
                }
                ta = tb;
                va = vb;
                oka = okb;
            }
        }
    } else if (st > 0.0) {
        double vf;
        face_eval<K>(sh, st, logp, 0.5 * st, vf, dv, dd);
        below = vf > 0.0;
    }
    cost_out = best;
    return have;
}

__host__ __device__ inline void volume_targets(const double (&s)[3], double (&dd)[3]) {
    double d[2], t, c2 = 1e300, c1 = 1e300;
    bool below2 = false, below1 = false;
    const double sh2[2] = {s[0], s[1]};
    const bool f2 = solve_face<2>(sh2, s[2], 0.0, fmax(1.0, s[2] + 1.0), d, t, c2, below2);
    if (f2) {
        dd[0] = d[0]; dd[1] = d[1]; dd[2] = t;
    }
    if (!f2 || below2) {
        const double sh1[2] = {s[0], 0.0};
        const double logp = -log(kClamp);
        double d1[2], t1;
        if (solve_face<1>(sh1, s[1], logp, fmax(10.0, s[1] + 10.0), d1, t1, c1, below1)) {
            c1 += (kClamp - s[2]) * (kClamp - s[2]);
            if (!f2 || c1 < c2) {
                dd[0] = d1[0]; dd[1] = t1; dd[2] = kClamp;
                return;
            }
        }
    }
    if (f2) return;
    dd[0] = 1.0 / (kClamp * kClamp);
    dd[1] = kClamp;
    dd[2] = kClamp;
}

// P = U diag(c) W^T
__host__ __device__ inline void udwt(const double (&U)[3][3], const double (&c)[3], const double (&W)[3][3],
                                     double (&P)[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            P[i][j] = U[i][0] * c[0] * W[j][0] + U[i][1] * c[1] * W[j][1] + U[i][2] * c[2] * W[j][2];
}

// J = dd/ds of the volume targets on the free (unclamped) set; sq_i = 2 d_i - s_i
// (> 0 on the + branch of d_i's quadratic, < 0 on the - branch).
__host__ __device__ inline void volume_jacobian(const double (&s)[3], const double (&d)[3], double (&J)[3][3],
                                                bool (&fr)[3], double (&sq)[3]) {
    double a[3], S = 0.0;
    for (int i = 0; i < 3; ++i) {
        fr[i] = d[i] > kClamp * (1.0 + 1e-9);
        sq[i] = 2.0 * d[i] - s[i];
        double den = sq[i];
        if (fabs(den) < 1e-300) den = copysign(1e-300, den);
        a[i] = fr[i] ? 1.0 / den : 0.0;
        S += fr[i] ? a[i] / d[i] : 0.0;
    }
    const double iS = (S != 0.0) ? 1.0 / S : 0.0;
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) J[i][k] = (fr[i] && fr[k]) ? ((i == k ? a[i] * d[i] : 0.0) - a[i] * a[k] * iS) : 0.0;
}

// Directional derivative of the elastic stress P(F) = ws (F - R) + wv (F - V)
// along dF: dP = (ws + wv) dF - U [ws B_R + wv B_V] W^T (singular frame B).
__host__ __device__ inline void stress_derivative(const double (&U)[3][3], const double (&s)[3],
                                                  const double (&W)[3][3], const double (&d)[3], double ws, double wv,
                                                  const double (&dF)[3][3], double (&dP)[3][3]) {
    double J[3][3], sq[3];
    bool fr[3];
    volume_jacobian(s, d, J, fr, sq);
    double T1[3][3], A[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T1[i][j] = dF[i][0] * W[0][j] + dF[i][1] * W[1][j] + dF[i][2] * W[2][j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A[i][j] = U[0][i] * T1[0][j] + U[1][i] * T1[1][j] + U[2][i] * T1[2][j];
    double B[3][3];
    for (int i = 0; i < 3; ++i) {
        double diag = 0.0;
        for (int k = 0; k < 3; ++k) diag += J[i][k] * A[k][k];
        B[i][i] = wv * diag;   // dR has no diagonal part in the singular frame
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            if (i == j) continue;
            const double sym = 0.5 * (A[i][j] + A[j][i]);
            const double skw = 0.5 * (A[i][j] - A[j][i]);
            double ssum = s[i] + s[j];
            if (fabs(ssum) < 1e-300) ssum = copysign(1e-300, ssum);
            const double betaR = 2.0 / ssum;
            const double betaV = (d[i] + d[j]) / ssum;
            double alphaV;
            if (fr[i] && fr[j] && sq[i] > 0.0 && sq[j] > 0.0) {
                // both targets on the + branch: (d_i - d_j)/(s_i - s_j) without cancellation
                alphaV = 0.5 * (1.0 + (s[i] + s[j]) / (sq[i] + sq[j]));
            } else if (fabs(s[i] - s[j]) > 1e-12 * fmax(1.0, fabs(s[i]))) {
                alphaV = (d[i] - d[j]) / (s[i] - s[j]);
            } else {
                alphaV = J[i][i] - J[i][j];
            }
            B[i][j] = ws * (betaR * skw) + wv * (alphaV * sym + betaV * skw);
        }
    double UB[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) UB[i][j] = U[i][0] * B[0][j] + U[i][1] * B[1][j] + U[i][2] * B[2][j];
    const double wsum = ws + wv;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            dP[i][j] = wsum * dF[i][j] - (UB[i][0] * W[j][0] + UB[i][1] * W[j][1] + UB[i][2] * W[j][2]);
}

}  // namespace proj64
}  // namespace pdg
