// Harmonic material basis (Sec. 6, "Harmonic Initialization", Eq. q2gamma):
// the r lowest eigenvectors of the graph Laplacian of the tets' face
// adjacency (L = D - A; two tets are adjacent when they share a face),
// computed on the device in FP64 by Chebyshev-filtered subspace iteration
// (Zhou & Saad, "Self-consistent-field calculations using Chebyshev-filtered
// subspace iteration", 2007): a block of q = r + 8 vectors is repeatedly
// multiplied by a Chebyshev polynomial of L that damps the interval
// [a, lambda_max] and amplifies the eigenvalues below a, re-orthonormalised
// (Cholesky QR, twice) and rotated onto Ritz vectors (Rayleigh-Ritz).  Only
// the q x q Gram and projected matrices go to the host.
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <tuple>
#include <vector>

#include "pd_internal.h"

namespace pdg {

namespace {

// Y = L X for a block stored row-major (n x q): Y[t][j] = deg_t X[t][j] - sum_nbr X[nbr][j]
__global__ void k_lap_block(int n, int q, const int4* __restrict__ nbr, const double* __restrict__ X,
                            double* __restrict__ Y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * q) return;
    const int t = (int)(i / q), j = (int)(i % q);
    const int4 nb = nbr[t];
    double deg = 0.0, acc = 0.0;
    if (nb.x >= 0) { deg += 1.0; acc += X[(int64_t)nb.x * q + j]; }
    if (nb.y >= 0) { deg += 1.0; acc += X[(int64_t)nb.y * q + j]; }
    if (nb.z >= 0) { deg += 1.0; acc += X[(int64_t)nb.z * q + j]; }
    if (nb.w >= 0) { deg += 1.0; acc += X[(int64_t)nb.w * q + j]; }
    Y[i] = deg * X[i] - acc;
}

// out = a (W - c Y) + b X   (elementwise over n x q)
__global__ void k_cheb_combine(int64_t N, const double* __restrict__ W, const double* __restrict__ Y,
                               const double* __restrict__ X, double a, double c, double b, double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    out[i] = a * (W[i] - c * Y[i]) + (X ? b * X[i] : 0.0);
}

// per column j: out[j] = sum_t (A[t][j] - theta_j B[t][j])^2 (B may be null); one block per column, fixed order
__global__ void __launch_bounds__(256) k_col_norm2(int n, int q, const double* __restrict__ A,
                                                   const double* __restrict__ B, const double* __restrict__ theta,
                                                   double* __restrict__ out) {
    __shared__ double sm[256];
    const int j = blockIdx.x;
    const double th = theta ? theta[j] : 0.0;
    double acc = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const double v = A[(int64_t)t * q + j] - (B ? th * B[(int64_t)t * q + j] : 0.0);
        acc += v * v;
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = sm[0];
}

// X[t][j] *= s[j]
__global__ void k_col_scale(int n, int q, const double* __restrict__ s, double* __restrict__ X) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * q) return;
    X[i] *= s[i % q];
}

// H (column-major, n x r, float) from the first r columns of X (row-major n x q)
__global__ void k_store_basis(int n, int q, int r, const double* __restrict__ X, const float* __restrict__ sign,
                              float* __restrict__ H) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * r) return;
    const int k = (int)(i / n), t = (int)(i % n);
    H[i] = sign[k] * (float)X[(int64_t)t * q + k];
}

inline unsigned grid(int64_t N, int b = 256) { return (unsigned)((N + b - 1) / b); }

}  // namespace

}  // namespace pdg

using namespace pdg;

static pd_status hfail(pd_status c, const char* msg) {
    set_error(msg);
    return c;
}

// Face adjacency of the tets, in the caller's tet order (-1 = no neighbour).
static std::vector<int4> face_neighbours(const pd_mesh* m) {
    const int n_t = m->n_t;
    std::vector<int4> nb(n_t, make_int4(-1, -1, -1, -1));
    std::vector<std::tuple<int32_t, int32_t, int32_t, int32_t>> faces;   // (a, b, c, user tet), a < b < c
    faces.reserve((size_t)4 * n_t);
    for (int t = 0; t < n_t; ++t) {
        const int32_t* v = &m->tets_new[(size_t)4 * t];
        const int32_t u = m->tet_old_of_new[t];
        for (int skip = 0; skip < 4; ++skip) {
            int32_t f[3], k = 0;
            for (int c = 0; c < 4; ++c)
                if (c != skip) f[k++] = v[c];
            std::sort(f, f + 3);
            faces.emplace_back(f[0], f[1], f[2], u);
        }
    }
    std::sort(faces.begin(), faces.end());
    std::vector<int> cnt(n_t, 0);
    auto add = [&](int32_t a, int32_t b) {
        int* slot = &nb[a].x;
        if (cnt[a] < 4) slot[cnt[a]++] = b;
    };
    for (size_t i = 0; i + 1 < faces.size(); ++i) {
        const auto& A = faces[i];
        const auto& B = faces[i + 1];
        if (std::get<0>(A) == std::get<0>(B) && std::get<1>(A) == std::get<1>(B) && std::get<2>(A) == std::get<2>(B)) {
            add(std::get<3>(A), std::get<3>(B));
            add(std::get<3>(B), std::get<3>(A));
        }
    }
    // fixed neighbour order (ascending) so that the sums are reproducible
    for (int t = 0; t < n_t; ++t) {
        int* s = &nb[t].x;
        std::sort(s, s + cnt[t]);
    }
    return nb;
}

extern "C" {

pd_status pd_harmonic_basis(pd_mesh* m, int32_t r, float* H, double* lambda, int32_t* iterations) {
    if (!m || !H) return hfail(PD_ERR_INVALID_ARG, "null argument");
    if (r < 1 || r > 56 || r > m->n_t) return hfail(PD_ERR_INVALID_ARG, "r out of range [1, min(56, n_t)]");
    cudaStream_t s = m->stream;
    const int n = m->n_t;
    const int q = std::min(r + 8, n);
    const int64_t N = (int64_t)n * q;
    try {
        const std::vector<int4> hnb = face_neighbours(m);
        int max_deg = 0;
        for (const int4& v : hnb) max_deg = std::max(max_deg, (v.x >= 0) + (v.y >= 0) + (v.z >= 0) + (v.w >= 0));
        const double b_up = std::max(2.0 * max_deg, 1.0);   // Gershgorin bound of lambda_max
        DBuf<int4> dnb;
        upload(dnb, hnb, s);
        // start: the constant vector and deterministic pseudo-random columns
        std::vector<double> hx((size_t)N);
        uint64_t st = 0x2545f4914f6cdd1dull;
        for (int t = 0; t < n; ++t)
            for (int j = 0; j < q; ++j) {
                st = st * 6364136223846793005ull + 1442695040888963407ull;
                hx[(size_t)t * q + j] = j == 0 ? 1.0 : (double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
            }
        // block rows padded with zeros to whole chunks of kChunk rows: the Gram
        // matrices A^T B are batched over the chunks and summed in a fixed order
        constexpr int kChunk = 2048;
        const int nch = (n + kChunk - 1) / kChunk;
        const int64_t Npad = (int64_t)nch * kChunk * q;
        DBuf<double> X, Y, W, Z, G, Gp, cn;
        for (auto* b : {&X, &Y, &W, &Z}) {
            b->alloc(Npad);
            PDG_CUDA(cudaMemsetAsync(b->p, 0, sizeof(double) * Npad, s));
        }
        PDG_CUDA(cudaMemcpyAsync(X.p, hx.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
        G.alloc((size_t)q * q);
        Gp.alloc((size_t)nch * q * q);
        cn.alloc(q);
        std::vector<double> hG((size_t)q * q), hGp((size_t)nch * q * q), Rinv, hs(q), T, w, V, hn(q);
        // hG = A^T B (q x q)
        auto gram = [&](const double* A, const double* B) {
            dense_gemm(true, false, q, q, kChunk, 1.0, A, q, (int64_t)kChunk * q, B, q, (int64_t)kChunk * q, 0.0,
                       Gp.p, q, (int64_t)q * q, nch, false, s);
            PDG_CUDA(cudaMemcpyAsync(hGp.data(), Gp.p, sizeof(double) * hGp.size(), cudaMemcpyDeviceToHost, s));
            PDG_CUDA(cudaStreamSynchronize(s));
            std::fill(hG.begin(), hG.end(), 0.0);
            for (int c = 0; c < nch; ++c)
                for (size_t i = 0; i < hG.size(); ++i) hG[i] += hGp[(size_t)c * q * q + i];
        };

        auto lap = [&](const double* src, double* dst) {
            k_lap_block<<<grid(N), 256, 0, s>>>(n, q, dnb.p, src, dst);
            PDG_CHECK_LAUNCH();
        };
        // normalise the columns of A, then Cholesky-QR twice into A
        auto orthonormalise = [&](double* A) {
            k_col_norm2<<<q, 256, 0, s>>>(n, q, A, nullptr, nullptr, cn.p);
            PDG_CHECK_LAUNCH();
            PDG_CUDA(cudaMemcpyAsync(hn.data(), cn.p, sizeof(double) * q, cudaMemcpyDeviceToHost, s));
            PDG_CUDA(cudaStreamSynchronize(s));
            for (int j = 0; j < q; ++j) hs[j] = hn[j] > 0.0 ? 1.0 / std::sqrt(hn[j]) : 0.0;
            PDG_CUDA(cudaMemcpyAsync(cn.p, hs.data(), sizeof(double) * q, cudaMemcpyHostToDevice, s));
            k_col_scale<<<grid(N), 256, 0, s>>>(n, q, cn.p, A);
            PDG_CHECK_LAUNCH();
            for (int pass = 0; pass < 2; ++pass) {
                gram(A, A);
                if (!chol_upper_inverse(hG.data(), q, q, Rinv)) throw Fail{PD_ERR_NOT_SPD};
                PDG_CUDA(cudaMemcpyAsync(G.p, Rinv.data(), sizeof(double) * q * q, cudaMemcpyHostToDevice, s));
                dense_gemm(false, false, n, q, q, 1.0, A, q, 0, G.p, q, 0, 0.0, Z.p, q, 0, 1, false, s);
                PDG_CUDA(cudaMemcpyAsync(A, Z.p, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
            }
        };
        std::vector<double> theta(q);
        // Rayleigh-Ritz on the orthonormal block A: A <- A V (ascending Ritz values in theta)
        auto rayleigh_ritz = [&](double* A) {
            lap(A, W.p);
            gram(A, W.p);
            T.assign((size_t)q * q, 0.0);
            for (int i = 0; i < q; ++i)
                for (int j = 0; j < q; ++j) T[(size_t)i * q + j] = 0.5 * (hG[(size_t)i * q + j] + hG[(size_t)j * q + i]);
            jacobi_eig(T, q, w, V);
            std::vector<int> idx(q);
            std::iota(idx.begin(), idx.end(), 0);
            std::sort(idx.begin(), idx.end(), [&](int a, int b) { return w[a] < w[b]; });
            std::vector<double> Vs((size_t)q * q);
            for (int j = 0; j < q; ++j) {
                theta[j] = w[idx[j]];
                for (int i = 0; i < q; ++i) Vs[(size_t)i * q + j] = V[(size_t)i * q + idx[j]];
            }
            PDG_CUDA(cudaMemcpyAsync(G.p, Vs.data(), sizeof(double) * q * q, cudaMemcpyHostToDevice, s));
            dense_gemm(false, false, n, q, q, 1.0, A, q, 0, G.p, q, 0, 0.0, Z.p, q, 0, 1, false, s);
            PDG_CUDA(cudaMemcpyAsync(A, Z.p, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        };
        // largest residual |L x_j - theta_j x_j| over the first r Ritz pairs
        DBuf<double> dth;
        dth.alloc(q);
        auto residual = [&](const double* A) {
            lap(A, W.p);
            PDG_CUDA(cudaMemcpyAsync(dth.p, theta.data(), sizeof(double) * q, cudaMemcpyHostToDevice, s));
            k_col_norm2<<<q, 256, 0, s>>>(n, q, W.p, A, dth.p, cn.p);
            PDG_CHECK_LAUNCH();
            PDG_CUDA(cudaMemcpyAsync(hn.data(), cn.p, sizeof(double) * q, cudaMemcpyDeviceToHost, s));
            PDG_CUDA(cudaStreamSynchronize(s));
            double e = 0.0;
            for (int j = 0; j < r; ++j) e = std::max(e, std::sqrt(std::max(hn[j], 0.0)));
            return e;
        };

        orthonormalise(X.p);
        rayleigh_ritz(X.p);
        const double tol = 1e-9 * b_up;
        constexpr int kMaxIter = 500;
        int it = 0;
        double res = residual(X.p);
        while (res > tol) {
            if (++it > kMaxIter) throw Fail{PD_ERR_TIMEOUT};
            // filter: damp [a, b_up], a = the largest Ritz value of the block; scaled three-term
            // recurrence with the lower spectrum bound 0 (L is positive semi-definite)
            const double a = std::min(std::max(theta[q - 1], 1e-12 * b_up), 0.9 * b_up);
            const double e = 0.5 * (b_up - a), c = 0.5 * (b_up + a);
            // degree: the filter grows by about e^3 from a down to 0 (T_m(x) ~ cosh(m acosh x))
            const int degree = std::min(400, std::max(8, (int)std::ceil(3.0 / std::acosh(1.0 + 2.0 * a / (b_up - a)))));
            double sigma = e / (0.0 - c);
            const double sigma1 = sigma, tau = 2.0 / sigma1;
            lap(X.p, W.p);
            k_cheb_combine<<<grid(N), 256, 0, s>>>(N, W.p, X.p, nullptr, sigma1 / e, c, 0.0, Y.p);   // Y = p1(L) X
            PDG_CHECK_LAUNCH();
            double* prev = X.p;
            double* cur = Y.p;
            double* nxt = Z.p;
            for (int k = 2; k <= degree; ++k) {
                const double sigma2 = 1.0 / (tau - sigma);
                lap(cur, W.p);
                k_cheb_combine<<<grid(N), 256, 0, s>>>(N, W.p, cur, prev, 2.0 * sigma2 / e, c, -sigma * sigma2, nxt);
                PDG_CHECK_LAUNCH();
                double* old = prev;
                prev = cur;
                cur = nxt;
                nxt = old;
                sigma = sigma2;
            }
            if (cur != X.p) PDG_CUDA(cudaMemcpyAsync(X.p, cur, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
            orthonormalise(X.p);
            rayleigh_ritz(X.p);
            res = residual(X.p);
        }
        // sign: the entry of largest magnitude of each basis vector is positive
        std::vector<double> hxf((size_t)N);
        PDG_CUDA(cudaMemcpyAsync(hxf.data(), X.p, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
        PDG_CUDA(cudaStreamSynchronize(s));
        std::vector<float> sg(r, 1.f);
        for (int k = 0; k < r; ++k) {
            double best = 0.0;
            for (int t = 0; t < n; ++t) {
                const double v = hxf[(size_t)t * q + k];
                if (std::fabs(v) > std::fabs(best) * (1.0 + 1e-9)) best = v;
            }
            sg[k] = best < 0.0 ? -1.f : 1.f;
        }
        DBuf<float> dsg;
        upload(dsg, sg, s);
        k_store_basis<<<grid((int64_t)n * r), 256, 0, s>>>(n, q, r, X.p, dsg.p, H);
        PDG_CHECK_LAUNCH();
        PDG_CUDA(cudaStreamSynchronize(s));
        if (lambda)
            for (int k = 0; k < r; ++k) lambda[k] = theta[k];
        if (iterations) *iterations = it;
    } catch (const Fail& f) {
        cudaStreamSynchronize(s);
        if (f.code == PD_ERR_NOT_SPD) set_error("harmonic subspace lost rank");
        if (f.code == PD_ERR_TIMEOUT) set_error("harmonic basis did not converge in 500 filter iterations");
        return f.code;
    }
    return PD_OK;
}

}  // extern "C"
