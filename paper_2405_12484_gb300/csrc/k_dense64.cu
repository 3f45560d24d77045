// FP64 dense kernels of the prefactorisation (Sec. 7.2: Eq. cms_boundary
// and the reduced system of Eq. global_subspace / Eq. dd, computed on the
// device): batched blocked Cholesky, inverse of an SPD matrix from its
// factor, and a batched FP64 GEMM.  Row-major storage throughout; matrices
// handed to the blocked routines are padded to a multiple of the 64-wide
// block with identity rows/columns.
#include "pd_internal.h"

namespace pdg {

namespace {

constexpr int NB = 64;   // diagonal block size of the blocked algorithms

// C = alpha op(A) op(B) + beta C, 64x64 tile per block, k-step 16, 4x4 outputs per
// thread (rows ty + 16 i, columns tx + 16 j).  lower_only: skip tiles above the
// diagonal and write only entries with row >= column.
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int K, double alpha, const double* __restrict__ A,
                                               int lda, int64_t sA, int ta, const double* __restrict__ B, int ldb,
                                               int64_t sB, int tb, double beta, double* __restrict__ C, int ldc,
                                               int64_t sC, int lower_only) {
    const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
    if (lower_only && row0 + 63 < col0) return;
    A += (int64_t)blockIdx.z * sA;
    B += (int64_t)blockIdx.z * sB;
    C += (int64_t)blockIdx.z * sC;
    __shared__ double As[16][65];
    __shared__ double Bs[16][65];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int l = threadIdx.x; l < 1024; l += 256) {
            int i, k;
            if (!ta) { i = l / 16; k = l % 16; } else { k = l / 64; i = l % 64; }
            const int gi = row0 + i, gk = k0 + k;
            double v = 0.0;
            if (gi < M && gk < K) v = ta ? A[(int64_t)gk * lda + gi] : A[(int64_t)gi * lda + gk];
            As[k][i] = v;
        }
        for (int l = threadIdx.x; l < 1024; l += 256) {
            int k, j;
            if (!tb) { k = l / 64; j = l % 64; } else { j = l / 16; k = l % 16; }
            const int gk = k0 + k, gj = col0 + j;
            double v = 0.0;
            if (gk < K && gj < N) v = tb ? B[(int64_t)gj * ldb + gk] : B[(int64_t)gk * ldb + gj];
            Bs[k][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gi = row0 + ty + 16 * i;
        if (gi >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gj = col0 + tx + 16 * j;
            if (gj >= N || (lower_only && gj > gi)) continue;
            double* c = C + (int64_t)gi * ldc + gj;
            *c = (beta == 0.0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *c);
        }
    }
}

// Factor the 64x64 diagonal block at (k0, k0) in place (lower) and write the
// inverse of the factor to Linv.  One block per batch item.  Shared memory
// holds L in the lower triangle and the strictly-lower part of X = L^-1
// transposed into the upper triangle (diagonal of X kept apart): 34 KB.
__global__ void __launch_bounds__(256) k_potrf_diag(double* __restrict__ A, int lda, int64_t sA, int k0,
                                                    double* __restrict__ Linv, int64_t sLinv, int* __restrict__ err) {
    A += (int64_t)blockIdx.x * sA;
    Linv += (int64_t)blockIdx.x * sLinv;
    __shared__ double L[NB][NB + 1];
    __shared__ double xd[NB];
    __shared__ int bad;
    const int tid = threadIdx.x;
    if (tid == 0) bad = 0;
    for (int l = tid; l < NB * NB; l += blockDim.x) {
        int i = l / NB, j = l % NB;
        L[i][j] = (j <= i) ? A[(int64_t)(k0 + i) * lda + k0 + j] : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < NB; ++j) {
        if (tid == 0) {
            double d = L[j][j];
            if (!(d > 0.0) || !isfinite(d)) {
                bad = 1;
                d = 1.0;
            }
            L[j][j] = sqrt(d);
        }
        __syncthreads();
        const double djj = L[j][j];
        for (int i = j + 1 + tid; i < NB; i += blockDim.x) L[i][j] /= djj;
        __syncthreads();
        const int w = NB - 1 - j;
        for (int idx = tid; idx < w * w; idx += blockDim.x) {
            const int i = j + 1 + idx / w, k = j + 1 + idx % w;
            if (k <= i) L[i][k] -= L[i][j] * L[k][j];
        }
        __syncthreads();
    }
    // column c of X = L^-1 by forward substitution; X[i][c] (i > c) is kept at L[c][i]
    if (tid < NB) {
        const int c = tid;
        const double xcc = 1.0 / L[c][c];
        xd[c] = xcc;
        for (int i = c + 1; i < NB; ++i) {
            double s = L[i][c] * xcc;
            for (int k = c + 1; k < i; ++k) s = fma(L[i][k], L[c][k], s);
            L[c][i] = -s / L[i][i];
        }
    }
    __syncthreads();
    for (int l = tid; l < NB * NB; l += blockDim.x) {
        int i = l / NB, j = l % NB;
        if (j <= i) A[(int64_t)(k0 + i) * lda + k0 + j] = L[i][j];
        Linv[l] = (i > j) ? L[j][i] : ((i == j) ? xd[i] : 0.0);
    }
    if (tid == 0 && bad) atomicOr(err, ERR_NOT_SPD);
}

__global__ void k_copy2d(const double* __restrict__ src, int lds, int64_t sS, double* __restrict__ dst, int ldd,
                         int64_t sD, int rows, int cols) {
    const int64_t n = (int64_t)rows * cols;
    src += (int64_t)blockIdx.y * sS;
    dst += (int64_t)blockIdx.y * sD;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        int r = (int)(l / cols), c = (int)(l % cols);
        dst[(int64_t)r * ldd + c] = src[(int64_t)r * lds + c];
    }
}

__global__ void k_set_identity(double* __restrict__ A, int n, int lda, int64_t sA) {
    A += (int64_t)blockIdx.y * sA;
    const int64_t tot = (int64_t)n * n;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < tot; l += (int64_t)gridDim.x * blockDim.x) {
        int r = (int)(l / n), c = (int)(l % n);
        A[(int64_t)r * lda + c] = (r == c) ? 1.0 : 0.0;
    }
}

inline int grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (int)(b < 65535 ? (b > 0 ? b : 1) : 65535);
}

void copy2d(const double* src, int lds, int64_t sS, double* dst, int ldd, int64_t sD, int rows, int cols, int batch,
            cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return;
    dim3 g(grid_for((int64_t)rows * cols), batch);
    k_copy2d<<<g, 256, 0, s>>>(src, lds, sS, dst, ldd, sD, rows, cols);
    PDG_CHECK_LAUNCH();
}

}  // namespace

void dense_gemm(bool ta, bool tb, int M, int N, int K, double alpha, const double* A, int lda, int64_t sA,
                const double* B, int ldb, int64_t sB, double beta, double* C, int ldc, int64_t sC, int batch,
                bool lower_only, cudaStream_t s) {
    if (M <= 0 || N <= 0 || batch <= 0) return;
    dim3 g((N + 63) / 64, (M + 63) / 64, batch);
    k_dgemm<<<g, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, ta ? 1 : 0, B, ldb, sB, tb ? 1 : 0, beta, C, ldc, sC,
                              lower_only ? 1 : 0);
    PDG_CHECK_LAUNCH();
}

void dense_set_identity(double* A, int n, int lda, int64_t strideA, int batch, cudaStream_t s) {
    dim3 g(grid_for((int64_t)n * n), batch);
    k_set_identity<<<g, 256, 0, s>>>(A, n, lda, strideA);
    PDG_CHECK_LAUNCH();
}

// Right-looking blocked Cholesky, n a multiple of 64.  Linv: batch x (n/64) x 64 x 64.
// W: workspace of batch x n x 64 doubles.
static void cholesky_blocked(double* A, int n, int lda, int64_t sA, int batch, double* Linv, double* W, int* err,
                             cudaStream_t s) {
    const int nblk = n / NB;
    const int64_t sLinv = (int64_t)nblk * NB * NB;
    const int64_t sW = (int64_t)n * NB;
    for (int kb = 0; kb < nblk; ++kb) {
        const int k0 = kb * NB;
        k_potrf_diag<<<batch, 256, 0, s>>>(A, lda, sA, k0, Linv + (int64_t)kb * NB * NB, sLinv, err);
        PDG_CHECK_LAUNCH();
        const int rem = n - k0 - NB;
        if (rem <= 0) continue;
        double* P = A + (int64_t)(k0 + NB) * lda + k0;
        // panel: L_ik = A_ik L_kk^-T
        dense_gemm(false, true, rem, NB, NB, 1.0, P, lda, sA, Linv + (int64_t)kb * NB * NB, NB, sLinv, 0.0, W, NB,
                   sW, batch, false, s);
        copy2d(W, NB, sW, P, lda, sA, rem, NB, batch, s);
        // trailing update (lower part only)
        dense_gemm(false, true, rem, rem, NB, -1.0, P, lda, sA, P, lda, sA, 1.0, P + NB, lda, sA, batch, true, s);
    }
}

// X = (L L^T)^-1 from the factor (forward then backward substitution on the identity).
static void inverse_from_factor(const double* L, int n, int lda, int64_t sL, const double* Linv, double* X, int ldx,
                                int64_t sX, int batch, double* W, cudaStream_t s) {
    const int nblk = n / NB;
    const int64_t sLinv = (int64_t)nblk * NB * NB;
    const int64_t sW = (int64_t)n * NB;
    dense_set_identity(X, n, ldx, sX, batch, s);
    for (int kb = 0; kb < nblk; ++kb) {
        const int k0 = kb * NB;
        const int cols = k0 + NB;   // the forward solution of the identity is lower triangular
        double* Xk = X + (int64_t)k0 * ldx;
        dense_gemm(false, false, NB, cols, NB, 1.0, Linv + (int64_t)kb * NB * NB, NB, sLinv, Xk, ldx, sX, 0.0, W,
                   cols, sW, batch, false, s);
        copy2d(W, cols, sW, Xk, ldx, sX, NB, cols, batch, s);
        const int rem = n - k0 - NB;
        if (rem > 0)
            dense_gemm(false, false, rem, cols, NB, -1.0, L + (int64_t)(k0 + NB) * lda + k0, lda, sL, Xk, ldx, sX,
                       1.0, X + (int64_t)(k0 + NB) * ldx, ldx, sX, batch, false, s);
    }
    for (int kb = nblk - 1; kb >= 0; --kb) {
        const int k0 = kb * NB;
        double* Xk = X + (int64_t)k0 * ldx;
        dense_gemm(true, false, NB, n, NB, 1.0, Linv + (int64_t)kb * NB * NB, NB, sLinv, Xk, ldx, sX, 0.0, W, n, sW,
                   batch, false, s);
        copy2d(W, n, sW, Xk, ldx, sX, NB, n, batch, s);
        if (k0 > 0)
            dense_gemm(true, false, k0, n, NB, -1.0, L + (int64_t)k0 * lda, lda, sL, Xk, ldx, sX, 1.0, X, ldx, sX,
                       batch, false, s);
    }
}

// In-place Cholesky of A (batched, n multiple of 64) and X = A^-1.
void dense_spd_inverse(double* A, int n, int lda, int64_t sA, double* X, int ldx, int64_t sX, int batch, int* d_err,
                       cudaStream_t s) {
    const int nblk = n / NB;
    double* Linv = nullptr;
    double* W = nullptr;
    PDG_CUDA(cudaMallocAsync((void**)&Linv, sizeof(double) * (size_t)batch * nblk * NB * NB, s));
    cudaError_t e = cudaMallocAsync((void**)&W, sizeof(double) * (size_t)batch * n * NB, s);
    if (e != cudaSuccess) {
        cudaFreeAsync(Linv, s);
        PDG_CUDA(e);
    }
    try {
        cholesky_blocked(A, n, lda, sA, batch, Linv, W, d_err, s);
        inverse_from_factor(A, n, lda, sA, Linv, X, ldx, sX, batch, W, s);
    } catch (...) {
        cudaFreeAsync(Linv, s);
        cudaFreeAsync(W, s);
        throw;
    }
    PDG_CUDA(cudaFreeAsync(Linv, s));
    PDG_CUDA(cudaFreeAsync(W, s));
}

int dense_block() { return NB; }

}  // namespace pdg

// ---------------------------------------------------------------- prefactor helpers
namespace pdg {

namespace {

__global__ void k_scatter_coo(double* __restrict__ S, int ld, const int* __restrict__ r, const int* __restrict__ c,
                              const double* __restrict__ v, int n) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    S[(int64_t)r[k] * ld + c[k]] = v[k];   // each (row, col) appears once
}

// S[bidx[a], bidx[b]] += Sd[a, b]; one launch per domain keeps the sum order fixed
__global__ void k_add_block(double* __restrict__ S, int ldS, const double* __restrict__ Sd, int ldSd,
                            const int* __restrict__ bidx, int nb) {
    const int64_t n = (int64_t)nb * nb;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        int a = (int)(l / nb), b = (int)(l % nb);
        S[(int64_t)bidx[a] * ldS + bidx[b]] += Sd[(int64_t)a * ldSd + b];
    }
}

__device__ __forceinline__ float round_tf32(float x) {
    uint32_t y;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
    return __uint_as_float(y);
}

// dst[r, c] = src[r, c] (or src[c, r] when transposed), converted to the storage precision
__global__ void k_cast_block(const double* __restrict__ src, int lds, int rows, int cols, int transpose, int prec,
                             float* __restrict__ d32, __nv_bfloat16* __restrict__ d16, int64_t off, int ldd) {
    const int64_t n = (int64_t)rows * cols;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        int r = (int)(l / cols), c = (int)(l % cols);
        double v = transpose ? src[(int64_t)c * lds + r] : src[(int64_t)r * lds + c];
        int64_t o = off + (int64_t)r * ldd + c;
        if (prec == PD_PREC_BF16) d16[o] = __double2bfloat16(v);
        else if (prec == PD_PREC_TF32) d32[o] = round_tf32((float)v);
        else d32[o] = (float)v;
    }
}

// the same cast into the tiled axpy layout (ax_tile_width), chunks of CW outputs
__global__ void k_cast_tiled(const double* __restrict__ src, int lds, int rows, int cols, int transpose, int prec,
                             float* __restrict__ d32, __nv_bfloat16* __restrict__ d16, int64_t off, int CW, int VN) {
    const int64_t n = (int64_t)rows * cols;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        int r = (int)(l / cols), c = (int)(l % cols);
        double v = transpose ? src[(int64_t)c * lds + r] : src[(int64_t)r * lds + c];
        const int o0 = c / CW * CW;
        const int64_t o = off + (int64_t)o0 * rows + (int64_t)r * ax_tile_width(cols, o0, CW, VN) + (c - o0);
        if (prec == PD_PREC_BF16) d16[o] = __double2bfloat16(v);
        else if (prec == PD_PREC_TF32) d32[o] = round_tf32((float)v);
        else d32[o] = (float)v;
    }
}

// BF16 tile in the tensor-core fragment order (rows padded to 16; see k_axpy_mma):
// element (r, c) of chunk o0 = c - c % CW lands in its 16 x 8 block at the
// lane and register the mma B operand reads it from.
__global__ void k_cast_frag16(const double* __restrict__ src, int lds, int rows, int cols, int transpose,
                              __nv_bfloat16* __restrict__ d16, int64_t off, int CW) {
    const int64_t n = (int64_t)rows * cols;
    const int kp = (rows + 15) & ~15;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(l / cols), c = (int)(l % cols);
        const double v = transpose ? src[(int64_t)c * lds + r] : src[(int64_t)r * lds + c];
        const int o0 = c / CW * CW;
        const int w = ax_tile_width(cols, o0, CW, 8);
        const int kb = r >> 4, kk = r & 15, cc = c - o0, nb = cc >> 3, nn = cc & 7;
        const int q = (kk & 7) >> 1, j = (kk & 1) + ((kk >> 3) << 1);
        d16[off + (int64_t)o0 * kp + ((int64_t)kb * (w >> 3) + nb) * 128 + (4 * nn + q) * 4 + j] =
            __double2bfloat16(v);
    }
}

// TF32 tile (rows padded to 8) in the register order of the B operand of
// mma.m16n8k8 (tf32): 8 x 8 blocks, lane 4 n + (k mod 4) holding rows k mod 4
// and k mod 4 + 4 of output n; values rounded to TF32.
__global__ void k_cast_frag32(const double* __restrict__ src, int lds, int rows, int cols, int transpose,
                              float* __restrict__ d32, int64_t off, int CW) {
    const int64_t n = (int64_t)rows * cols;
    const int kp = (rows + 7) & ~7;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(l / cols), c = (int)(l % cols);
        const double v = transpose ? src[(int64_t)c * lds + r] : src[(int64_t)r * lds + c];
        const int o0 = c / CW * CW;
        const int w = ax_tile_width(cols, o0, CW, 8);
        const int kb = r >> 3, kk = r & 7, cc = c - o0, nb = cc >> 3, nn = cc & 7;
        d32[off + (int64_t)o0 * kp + ((int64_t)kb * (w >> 3) + nb) * 64 + (4 * nn + (kk & 3)) * 2 + (kk >> 2)] =
            round_tf32((float)v);
    }
}

// BF16 row-form block in the tensor-core fragment order (rows and columns
// padded to 16, see k_rowdot_mma): element (r, c) lands in 16 x 16 block
// (r / 16, c / 16) at the lane and register of the mma A operand.
__global__ void k_cast_rowfrag16(const double* __restrict__ src, int lds, int rows, int cols, int transpose,
                                 __nv_bfloat16* __restrict__ d16, int64_t off, int Kp) {
    const int64_t n = (int64_t)rows * cols;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(l / cols), c = (int)(l % cols);
        const double v = transpose ? src[(int64_t)c * lds + r] : src[(int64_t)r * lds + c];
        const int rb = r >> 4, kb = c >> 4, rr = r & 15, kk = c & 15;
        const int g = rr & 7, rhi = rr >> 3, q = (kk & 7) >> 1, j = kk & 1, khi = kk >> 3;
        d16[off + ((int64_t)rb * (Kp >> 4) + kb) * 256 + (4 * g + q) * 8 + (rhi + 2 * khi) * 2 + j] =
            __double2bfloat16(v);
    }
}

// dst[i][k] = S[r0 + i][cols ? c0 + cols[k] : c0 + k]
__global__ void k_copy_block_idx(const double* __restrict__ S, int ldS, int r0, int nr, const int* __restrict__ cols,
                                 int c0, int nc, double* __restrict__ dst, int ldd) {
    const int64_t n = (int64_t)nr * nc;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(l / nc), k = (int)(l % nc);
        const int c = c0 + (cols ? cols[k] : k);
        dst[(int64_t)i * ldd + k] = S[(int64_t)(r0 + i) * ldS + c];
    }
}

inline int grid_of(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (int)(b < 65535 ? (b > 0 ? b : 1) : 65535);
}

}  // namespace

void launch_prefactor_helpers_scatter_coo(double* S, int ld, const int* r, const int* c, const double* v, int n,
                                          cudaStream_t s) {
    if (n <= 0) return;
    k_scatter_coo<<<(n + 255) / 256, 256, 0, s>>>(S, ld, r, c, v, n);
    PDG_CHECK_LAUNCH();
}

void launch_prefactor_add_block(double* S, int ldS, const double* Sd, int ldSd, const int* bidx, int nb,
                                cudaStream_t s) {
    if (nb <= 0) return;
    k_add_block<<<grid_of((int64_t)nb * nb), 256, 0, s>>>(S, ldS, Sd, ldSd, bidx, nb);
    PDG_CHECK_LAUNCH();
}

void launch_copy_block_idx(const double* S, int ldS, int r0, int nr, const int* cols, int c0, int nc, double* dst,
                           int ldd, cudaStream_t s) {
    if (nr <= 0 || nc <= 0) return;
    k_copy_block_idx<<<grid_of((int64_t)nr * nc), 256, 0, s>>>(S, ldS, r0, nr, cols, c0, nc, dst, ldd);
    PDG_CHECK_LAUNCH();
}

void launch_cast_block(const double* src, int lds, int rows, int cols, int transpose, int prec, float* dst32,
                       __nv_bfloat16* dst16, int64_t dst_off, int ldd, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return;
    k_cast_block<<<grid_of((int64_t)rows * cols), 256, 0, s>>>(src, lds, rows, cols, transpose, prec, dst32, dst16,
                                                                dst_off, ldd);
    PDG_CHECK_LAUNCH();
}

void launch_cast_frag32(const double* src, int lds, int rows, int cols, int transpose, float* dst32,
                        int64_t dst_off, int CW, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return;
    k_cast_frag32<<<grid_of((int64_t)rows * cols), 256, 0, s>>>(src, lds, rows, cols, transpose, dst32, dst_off, CW);
    PDG_CHECK_LAUNCH();
}

void launch_cast_rowfrag16(const double* src, int lds, int rows, int cols, int transpose, __nv_bfloat16* dst16,
                           int64_t dst_off, int Kp, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return;
    k_cast_rowfrag16<<<grid_of((int64_t)rows * cols), 256, 0, s>>>(src, lds, rows, cols, transpose, dst16, dst_off,
                                                                    Kp);
    PDG_CHECK_LAUNCH();
}

void launch_cast_frag16(const double* src, int lds, int rows, int cols, int transpose, __nv_bfloat16* dst16,
                        int64_t dst_off, int CW, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return;
    k_cast_frag16<<<grid_of((int64_t)rows * cols), 256, 0, s>>>(src, lds, rows, cols, transpose, dst16, dst_off, CW);
    PDG_CHECK_LAUNCH();
}

void launch_cast_tiled(const double* src, int lds, int rows, int cols, int transpose, int prec, float* dst32,
                       __nv_bfloat16* dst16, int64_t dst_off, int CW, int VN, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return;
    k_cast_tiled<<<grid_of((int64_t)rows * cols), 256, 0, s>>>(src, lds, rows, cols, transpose, prec, dst32, dst16,
                                                                dst_off, CW, VN);
    PDG_CHECK_LAUNCH();
}

}  // namespace pdg
