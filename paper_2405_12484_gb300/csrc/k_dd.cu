// Per-iteration domain-decomposed subspace solve (Sec. 7.2) on sm_103a.
//
// With the internal/boundary split of every domain d (Eq. dd) and the
// boundary modes Psi_d = -K_ii^-1 K_ib (Eq. cms_boundary), the Galerkin
// projection onto the subspace of Eq. global_subspace with the full set of
// internal modes gives the exact solution of K x = b in four phases:
//   condense : [t_d; c_d] = [K_ii^-1; Psi_d^T] b_i            (per domain)
//   gather   : c = b_B + sum_d E_d c_d                          (per interface vertex, fixed order)
//   coarse   : x_B = S^-1 c,  S = K_BB + sum_d K_bi Psi_d       (reduced interface system)
//   backsub  : x_i = t_d + Psi_d x_B(d)                         (per domain)
// Every product is a dense matrix times three right-hand sides (x, y, z
// share the scalar matrix, K = K_s (x) I_3): HBM-bound streaming of the
// matrices (bulk asynchronous copies of whole tiles or rows into a
// shared-memory ring, or 16-byte loads in the fallback kernels), FP32
// accumulation, vectors staged in shared memory, fixed-order reductions
// (deterministic), no atomics.
#include <algorithm>
#include <type_traits>

#include "pd_internal.h"
#include "tma.cuh"

namespace pdg {

void launch_stream_solve(const StreamPlan& P, FusedArgs F, cudaStream_t s);

// Test hook: bytes the next first stage of block 0 of a tile-streaming launch
// expects beyond what its copy delivers (0 = none; consumed once).
__device__ int g_test_copy_extra = 0;

namespace {

template <class T>
struct VecN;
template <>
struct VecN<float> {
    static constexpr int N = 4;
};
template <>
struct VecN<__nv_bfloat16> {
    static constexpr int N = 8;
};

__device__ __forceinline__ void load_vec(const float* p, float (&v)[4]) {
    float4 a = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}

__device__ __forceinline__ void load_vec(const __nv_bfloat16* p, float (&v)[8]) {
    uint4 a = __ldcs(reinterpret_cast<const uint4*>(p));
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&a);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float2 f = __bfloat1622float2(h[k]);
        v[2 * k] = f.x;
        v[2 * k + 1] = f.y;
    }
}

__device__ __forceinline__ void load_vec_shared(const float* p, float (&v)[4]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}

__device__ __forceinline__ void load_vec_shared(const __nv_bfloat16* p, float (&v)[8]) {
    const uint4 a = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&a);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float2 f = __bfloat1622float2(h[k]);
        v[2 * k] = f.x;
        v[2 * k + 1] = f.y;
    }
}

// Staging of a product's x vector in shared memory with many loads in flight:
// each thread issues kStageU independent loads (indices first when indexed,
// then values) before it stores any of them, so staging costs one or two
// memory latencies per kStageU entries instead of one per entry.
constexpr int kStageU = 8;

// xs[k] = x[idx ? idx[k] : k] for k < n
__device__ __forceinline__ void stage_f4(float4* __restrict__ xs, int n, const float4* __restrict__ x,
                                         const int* __restrict__ idx, int tid, int nthreads) {
    for (int base = tid; base < n; base += nthreads * kStageU) {
        int id[kStageU];
#pragma unroll
        for (int u = 0; u < kStageU; ++u) {
            const int k = base + u * nthreads;
            id[u] = k < n ? (idx ? idx[k] : k) : -1;
        }
        float4 v[kStageU];
#pragma unroll
        for (int u = 0; u < kStageU; ++u) v[u] = id[u] >= 0 ? x[id[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < kStageU; ++u) {
            const int k = base + u * nthreads;
            if (k < n) xs[k] = v[u];
        }
    }
}

// stage_f4 in two parts around the wait for the predecessor: the indices of
// the first kStageU entries per thread (constant) before it, the values after.
struct StageIdx {
    int id[kStageU];
};

__device__ __forceinline__ void stage_f4_indices(StageIdx& S, int n, const int* __restrict__ idx, int tid,
                                                 int nthreads) {
#pragma unroll
    for (int u = 0; u < kStageU; ++u) {
        const int k = tid + u * nthreads;
        S.id[u] = k < n ? (idx ? idx[k] : k) : -1;
    }
}

__device__ __forceinline__ void stage_f4_values(float4* __restrict__ xs, int n, const float4* __restrict__ x,
                                                const int* __restrict__ idx, const StageIdx& S, int tid,
                                                int nthreads) {
    float4 v[kStageU];
#pragma unroll
    for (int u = 0; u < kStageU; ++u) v[u] = S.id[u] >= 0 ? x[S.id[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < kStageU; ++u) {
        const int k = tid + u * nthreads;
        if (k < n) xs[k] = v[u];
    }
    // entries beyond the first kStageU per thread (not on the shell's meshes)
    if (n > nthreads * kStageU) {
        for (int base = tid + nthreads * kStageU; base < n; base += nthreads * kStageU) {
            int id[kStageU];
#pragma unroll
            for (int u = 0; u < kStageU; ++u) {
                const int k = base + u * nthreads;
                id[u] = k < n ? (idx ? idx[k] : k) : -1;
            }
            float4 w[kStageU];
#pragma unroll
            for (int u = 0; u < kStageU; ++u) w[u] = id[u] >= 0 ? x[id[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < kStageU; ++u) {
                const int k = base + u * nthreads;
                if (k < n) xs[k] = w[u];
            }
        }
    }
}

// three float planes x0/x1/x2[k] = x[idx ? idx[k] : k] for k < n_valid, 0 for n_valid <= k < n
__device__ __forceinline__ void stage_planes(float* __restrict__ x0, float* __restrict__ x1, float* __restrict__ x2,
                                             int n_valid, int n, const float4* __restrict__ x,
                                             const int* __restrict__ idx, int tid, int nthreads) {
    for (int base = tid; base < n; base += nthreads * kStageU) {
        int id[kStageU];
#pragma unroll
        for (int u = 0; u < kStageU; ++u) {
            const int k = base + u * nthreads;
            id[u] = k < n_valid ? (idx ? idx[k] : k) : -1;
        }
        float4 v[kStageU];
#pragma unroll
        for (int u = 0; u < kStageU; ++u) v[u] = id[u] >= 0 ? x[id[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < kStageU; ++u) {
            const int k = base + u * nthreads;
            if (k < n) {
                x0[k] = v[u].x;
                x1[k] = v[u].y;
                x2[k] = v[u].z;
            }
        }
    }
}

// y[r] = add[r] + A[r, 0:cols] . xs  for r < rows; groups of LPR lanes own
// two rows at a time; 256 threads.
template <class T, int LPR, int NT>
__device__ __forceinline__ void block_rows_n(const T* __restrict__ A, int rows, int ld, int cols,
                                             const float4* __restrict__ xs, float4* __restrict__ y,
                                             const float4* __restrict__ add) {
    constexpr int VN = VecN<T>::N;
    constexpr int G = NT / LPR;
    const int lane = threadIdx.x % LPR;
    const int grp = threadIdx.x / LPR;
    // the trip count is uniform across the block so every lane reaches the shuffles
    for (int base = 0; base < rows; base += 2 * G) {
        const int r0 = base + 2 * grp;
        const bool one = r0 < rows;
        const bool two = (r0 + 1) < rows;
        const T* a0 = A + (int64_t)(one ? r0 : 0) * ld;
        const T* a1 = A + (int64_t)(two ? r0 + 1 : (one ? r0 : 0)) * ld;
        const int ncol = one ? cols : 0;
        float s00 = 0.f, s01 = 0.f, s02 = 0.f, s10 = 0.f, s11 = 0.f, s12 = 0.f;
#pragma unroll 4
        for (int c = lane * VN; c < ncol; c += LPR * VN) {
            float v0[VN], v1[VN];
            load_vec(a0 + c, v0);
            load_vec(a1 + c, v1);
#pragma unroll
            for (int j = 0; j < VN; ++j) {
                float4 xv = xs[c + j];
                s00 = fmaf(v0[j], xv.x, s00);
                s01 = fmaf(v0[j], xv.y, s01);
                s02 = fmaf(v0[j], xv.z, s02);
                s10 = fmaf(v1[j], xv.x, s10);
                s11 = fmaf(v1[j], xv.y, s11);
                s12 = fmaf(v1[j], xv.z, s12);
            }
        }
#pragma unroll
        for (int off = LPR / 2; off > 0; off >>= 1) {
            s00 += __shfl_xor_sync(0xffffffffu, s00, off, LPR);
            s01 += __shfl_xor_sync(0xffffffffu, s01, off, LPR);
            s02 += __shfl_xor_sync(0xffffffffu, s02, off, LPR);
            s10 += __shfl_xor_sync(0xffffffffu, s10, off, LPR);
            s11 += __shfl_xor_sync(0xffffffffu, s11, off, LPR);
            s12 += __shfl_xor_sync(0xffffffffu, s12, off, LPR);
        }
        if (lane == 0 && one) {
            float4 a = add ? add[r0] : make_float4(0.f, 0.f, 0.f, 0.f);
            y[r0] = make_float4(a.x + s00, a.y + s01, a.z + s02, 0.f);
            if (two) {
                float4 b = add ? add[r0 + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
                y[r0 + 1] = make_float4(b.x + s10, b.y + s11, b.z + s12, 0.f);
            }
        }
    }
}

// Same product with RPG rows per lane group sharing every x value read from
// shared memory (shared-memory bytes per matrix byte = VN / RPG).
template <class T, int LPR>
__device__ __forceinline__ void block_rows(const T* __restrict__ A, int rows, int ld, int cols,
                                           const float4* __restrict__ xs, float4* __restrict__ y,
                                           const float4* __restrict__ add) {
    block_rows_n<T, LPR, 256>(A, rows, ld, cols, xs, y, add);
}

constexpr int kMaxSubCols = 2048;   // largest per-domain internal / boundary count handled in shared memory

// Column-oriented per-domain products ("axpy form"): y = add + sum_k A[k, :] x_k
// with A stored so that each output is a column (rows k of A are contiguous).
// One block = one output chunk of one domain matrix: each lane owns VN
// consecutive outputs, the kAxWarps warps split k into equal ranges, x_k is a
// shared-memory broadcast, and the warps' partial sums are combined in a
// fixed order (deterministic).  No cross-lane reductions, fully coalesced
// 16-byte row loads.
#ifndef PDG_AX_WARPS
#define PDG_AX_WARPS 8
#endif
#ifndef PDG_AX_UNROLL
#define PDG_AX_UNROLL 4
#endif
#ifndef PDG_ROW_UNROLL
#define PDG_ROW_UNROLL 4
#endif
#ifndef PDG_ROW_WARPS
#define PDG_ROW_WARPS 16
#endif
#ifndef PDG_ROW_BPS
#define PDG_ROW_BPS 2
#endif
#ifndef PDG_ROW_RU32
#define PDG_ROW_RU32 1
#endif
#ifndef PDG_COARSE_BPS
#define PDG_COARSE_BPS 2
#endif
#ifndef PDG_AX_M
#define PDG_AX_M 1
#endif
constexpr int kRowWarps = PDG_ROW_WARPS;
constexpr int kRowBps = PDG_ROW_BPS;
constexpr int kRowRu32 = PDG_ROW_RU32;
constexpr int kCoarseBps = PDG_COARSE_BPS;
constexpr int kAxM = PDG_AX_M;
constexpr int kAxWarps = PDG_AX_WARPS;
constexpr int kAxUnroll = PDG_AX_UNROLL;
constexpr int kRowUnroll = PDG_ROW_UNROLL;

template <class T, bool BATCHED>
__global__ void __launch_bounds__(32 * kAxWarps) k_axpy_form(const AxDesc* __restrict__ descs,
                                                              const AxBlock* __restrict__ blocks, AxBases single,
                                                              const AxBases* __restrict__ multi) {
    constexpr int VN = VecN<T>::N;
    constexpr int SW = 32 * VN;          // outputs of one warp-wide sub-chunk
    constexpr int OW = SW * kAxM;        // outputs of the block
    extern __shared__ float4 xs[];   // K_max entries (dynamic)
    __shared__ float red[kAxWarps - 1][OW][3];
    const AxBlock bk = blocks[blockIdx.x];
    const AxDesc D = descs[bk.desc];
    const AxBases B = BATCHED ? multi[D.slot] : single;
    const T* A = reinterpret_cast<const T*>(B.pool) + D.a_off;
    stage_f4(xs, D.K, B.x + D.x_off, D.bidx_off >= 0 ? B.bidx + D.bidx_off : nullptr, threadIdx.x, blockDim.x);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k0 = D.K * warp / kAxWarps, k1 = D.K * (warp + 1) / kAxWarps;
    float acc[kAxM][VN][3];
#pragma unroll
    for (int j = 0; j < kAxM; ++j)
#pragma unroll
        for (int i = 0; i < VN; ++i) acc[j][i][0] = acc[j][i][1] = acc[j][i][2] = 0.f;
    // row stride: the matrix's ld, or the width of this block's tile (chunk width in ld)
    const int ldr = D.tiled ? ax_tile_width(D.n_out, bk.o0, D.ld, VN) : D.ld;
    bool valid[kAxM];
#pragma unroll
    for (int j = 0; j < kAxM; ++j)
        valid[j] = bk.o0 + j * SW + lane * VN < D.n_out && (!D.tiled || j * SW + lane * VN < ldr);
    if (valid[0]) {
        const T* a = A + (D.tiled ? (int64_t)bk.o0 * D.K : (int64_t)bk.o0) + lane * VN;
#pragma unroll kAxUnroll
        for (int k = k0; k < k1; ++k) {
            const float4 xk = xs[k];
#pragma unroll
            for (int j = 0; j < kAxM; ++j) {
                if (!valid[j]) continue;
                float v[VN];
                load_vec(a + (int64_t)k * ldr + j * SW, v);
#pragma unroll
                for (int i = 0; i < VN; ++i) {
                    acc[j][i][0] = fmaf(v[i], xk.x, acc[j][i][0]);
                    acc[j][i][1] = fmaf(v[i], xk.y, acc[j][i][1]);
                    acc[j][i][2] = fmaf(v[i], xk.z, acc[j][i][2]);
                }
            }
        }
    }
    if (warp > 0) {
#pragma unroll
        for (int j = 0; j < kAxM; ++j)
#pragma unroll
            for (int i = 0; i < VN; ++i) {
                red[warp - 1][j * SW + lane * VN + i][0] = acc[j][i][0];
                red[warp - 1][j * SW + lane * VN + i][1] = acc[j][i][1];
                red[warp - 1][j * SW + lane * VN + i][2] = acc[j][i][2];
            }
    }
    __syncthreads();
    if (warp == 0) {
        float4* out = B.out + D.out_off;
        const float4* add = (D.add_off >= 0) ? B.add + D.add_off : nullptr;
#pragma unroll
        for (int j = 0; j < kAxM; ++j)
#pragma unroll
            for (int i = 0; i < VN; ++i) {
                const int oi = bk.o0 + j * SW + lane * VN + i;
                // outputs past this block's tile belong to the next block
                if (oi >= D.n_out || (D.tiled && j * SW + lane * VN + i >= ldr)) break;
                float r0 = acc[j][i][0], r1 = acc[j][i][1], r2 = acc[j][i][2];
#pragma unroll
                for (int w = 0; w < kAxWarps - 1; ++w) {
                    r0 += red[w][j * SW + lane * VN + i][0];
                    r1 += red[w][j * SW + lane * VN + i][1];
                    r2 += red[w][j * SW + lane * VN + i][2];
                }
                const float4 b = add ? add[oi] : make_float4(0.f, 0.f, 0.f, 0.f);
                out[oi] = make_float4(b.x + r0, b.y + r1, b.z + r2, 0.f);
            }
    }
}

// The same product streamed through shared memory with bulk asynchronous
// copies (tiled layout only): one producer lane copies the block's tile in
// stages of kAxtRows rows (one cp.async.bulk per stage, a ring of kAxtStages
// stages of kAxtRows x w elements, completion counted in bytes on an
// mbarrier), so the copies in flight do not depend on what the compute
// warps do.  kAxtWarps consumer warps take the rows of a stage in turn (row
// r to warp r mod kAxtWarps), each lane owning VN consecutive outputs with
// x_k a shared-memory broadcast; after the last stage the warps' partial
// sums go through the (then idle) ring and are added in warp order
// (deterministic).  Every wait is bounded (1 s or the CTA's abort flag): a
// wait that runs out sets ERR_TIMEOUT in `err`, the producer stops issuing
// and drains the copies it has in flight.
#ifndef PDG_AXT_STAGES
#define PDG_AXT_STAGES 3
#endif
#ifndef PDG_AXT_ROWS
#define PDG_AXT_ROWS 32
#endif
#ifndef PDG_AXT_WARPS
#define PDG_AXT_WARPS 4
#endif
constexpr int kAxtStages = PDG_AXT_STAGES;
constexpr int kAxtRows = PDG_AXT_ROWS;
constexpr int kAxtWarps = PDG_AXT_WARPS;
static_assert(kAxM == 1, "the tiled layout has one output chunk per block");

// ring bytes of a launch whose widest tile has wmax outputs (a multiple of VN)
template <class T>
inline size_t axt_ring_bytes(int wmax) {
    const size_t ring = (size_t)kAxtStages * kAxtRows * wmax * sizeof(T);
    const size_t red = (size_t)(kAxtWarps - 1) * wmax * 3 * sizeof(float);
    return (std::max(ring, red) + 15) / 16 * 16;
}

template <class T, bool BATCHED>
__global__ void __launch_bounds__(32 * (kAxtWarps + 1)) k_axpy_tma(const AxDesc* __restrict__ descs,
                                                                   const AxBlock* __restrict__ blocks,
                                                                   AxBases single,
                                                                   const AxBases* __restrict__ multi,
                                                                   int ring_bytes, int* __restrict__ err) {
    using namespace tma;
    constexpr int VN = VecN<T>::N;
    constexpr int S = kAxtStages, R = kAxtRows;
    extern __shared__ __align__(128) unsigned char axt_smem[];
    T* ring = reinterpret_cast<T*>(axt_smem);
    float* red = reinterpret_cast<float*>(axt_smem);     // reused after the last stage
    float4* xs = reinterpret_cast<float4*>(axt_smem + ring_bytes);
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ int abort_flag;
    const AxBlock bk = blocks[blockIdx.x];
    const AxDesc D = descs[bk.desc];
    const AxBases B = BATCHED ? multi[D.slot] : single;   // serving: the request's own arrays
    const int w = ax_tile_width(D.n_out, bk.o0, D.ld, VN);
    const T* tile = reinterpret_cast<const T*>(B.pool) + D.a_off + (int64_t)bk.o0 * D.K;
    const int n_st = (D.K + R - 1) / R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    pdl_trigger();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < S; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kAxtWarps);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();   // barriers initialised: the producer starts at once, the consumers stage x meanwhile
    if (warp == kAxtWarps) {
        // producer
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < n_st; ++i) {
                const int slot = i % S;
                if (i >= S && !mbar_wait(&empty[slot], ((i / S) - 1) & 1, &abort_flag)) {
                    abort_flag = 1;
                    atomicOr(err, ERR_TIMEOUT);
                    break;
                }
                const int rows = min(R, D.K - i * R);
                const uint32_t bytes = (uint32_t)(rows * w * (int)sizeof(T));
                uint32_t expect = bytes;
                if (blockIdx.x == 0 && i == 0 && *reinterpret_cast<volatile int*>(&g_test_copy_extra) > 0)
                    expect += (uint32_t)max(atomicExch(&g_test_copy_extra, 0), 0);
                mbar_arrive_expect_tx(&full[slot], expect);
                bulk_g2s(ring + (size_t)slot * R * w, tile + (int64_t)i * R * w, bytes, &full[slot]);
                issued = i + 1;
            }
            // every copy issued has landed before the CTA may exit
            for (int i = max(0, issued - S); i < issued; ++i)
                if (!mbar_wait(&full[i % S], (i / S) & 1)) atomicOr(err, ERR_TIMEOUT);
        }
        return;
    }
    // consumers (the producer streams the constant tile without waiting for the predecessor)
    {
        const int* xi = D.bidx_off >= 0 ? B.bidx + D.bidx_off : nullptr;
        StageIdx si;
        stage_f4_indices(si, D.K, xi, threadIdx.x, 32 * kAxtWarps);   // constant: before the wait
        pdl_wait();
        stage_f4_values(xs, D.K, B.x + D.x_off, xi, si, threadIdx.x, 32 * kAxtWarps);
    }
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kAxtWarps) : "memory");
    float acc[VN][3];
#pragma unroll
    for (int i = 0; i < VN; ++i) acc[i][0] = acc[i][1] = acc[i][2] = 0.f;
    const int my = lane * VN;
    const bool act = my < w;
    for (int i = 0; i < n_st; ++i) {
        const int slot = i % S;
        if (!mbar_wait(&full[slot], (i / S) & 1, &abort_flag)) {
            if (lane == 0) {
                abort_flag = 1;
                atomicOr(err, ERR_TIMEOUT);
            }
            break;
        }
        const int rows = min(R, D.K - i * R);
        const T* st = ring + (size_t)slot * R * w;
        if (act) {
#pragma unroll 2
            for (int r = warp; r < rows; r += kAxtWarps) {
                const float4 xk = xs[i * R + r];
                float v[VN];
                load_vec_shared(st + r * w + my, v);
#pragma unroll
                for (int j = 0; j < VN; ++j) {
                    acc[j][0] = fmaf(v[j], xk.x, acc[j][0]);
                    acc[j][1] = fmaf(v[j], xk.y, acc[j][1]);
                    acc[j][2] = fmaf(v[j], xk.z, acc[j][2]);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
    }
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kAxtWarps) : "memory");   // every consumer is past the ring
    if (warp > 0 && act) {
#pragma unroll
        for (int j = 0; j < VN; ++j) {
            float* r = red + ((size_t)(warp - 1) * w + my + j) * 3;
            r[0] = acc[j][0];
            r[1] = acc[j][1];
            r[2] = acc[j][2];
        }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kAxtWarps) : "memory");
    if (warp == 0 && act) {
        float4* out = B.out + D.out_off;
        const float4* add = (D.add_off >= 0) ? B.add + D.add_off : nullptr;
#pragma unroll
        for (int j = 0; j < VN; ++j) {
            const int oi = bk.o0 + my + j;
            if (oi >= D.n_out) break;
            float r0 = acc[j][0], r1 = acc[j][1], r2 = acc[j][2];
            for (int q = 0; q < kAxtWarps - 1; ++q) {
                const float* r = red + ((size_t)q * w + my + j) * 3;
                r0 += r[0];
                r1 += r[1];
                r2 += r[2];
            }
            const float4 b = add ? add[oi] : make_float4(0.f, 0.f, 0.f, 0.f);
            out[oi] = make_float4(b.x + r0, b.y + r1, b.z + r2, 0.f);
        }
    }
}

// BF16 tiles on the tensor cores.  A BF16 axpy-form tile is stored with its
// rows padded to a multiple of 16 and cut into 16 x 8 (rows k x outputs n)
// blocks in row-block-major order, each block in the register order of the
// B operand of mma.m16n8k16 (lane 4 n + q holds rows 2q, 2q+1, 2q+8, 2q+9 of
// column n), so a bulk-copied stage is consumed with one 8-byte shared load
// per lane and block, free of bank conflicts.  The A operand is the
// right-hand sides: rows 0..2 hold x, y, z rounded to BF16 and rows 8..10
// their BF16 remainders (x - bf16(x)), so the FP32 accumulators of the
// product carry x to about 16 bits while the matrix is BF16.  Output n of
// right-hand side c is D[c][n] + D[c + 8][n].  The consumer warps own
// disjoint output columns (no cross-warp reduction); the copy ring, the
// producer lane and the bounded waits are those of k_axpy_tma.  (The tiles
// are written in this order by k_cast_frag16 at prefactorisation.)

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint4& a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

constexpr int kAxmNb = 8;   // n8 blocks per consumer warp (tile width <= 8 * 8 * kAxtWarps = 256)
// stages of 64 BF16 rows: the bytes of the FP32 kernel's 32-row stages (measured: 64-row
// stages 1.88 ms per frame against 1.93 ms with 32; the FP32 kernel is fastest at 32)
#ifndef PDG_AXM_ROWS
#define PDG_AXM_ROWS 64
#endif
constexpr int kAxmRows = PDG_AXM_ROWS;
constexpr int kAxmStages = kAxtStages;
static_assert(kAxmNb * 8 * kAxtWarps >= 256, "one consumer warp per output column group");

// TF32 tiles: stages of 32 FP32-sized rows (the FP32 kernel's stage), 8-row k-blocks
constexpr int kAxfRows = kAxtRows;
// lanes whose A operand is not zero: groups 0..2 (x, y, z in rows g and g + 8)
constexpr int kAxmFragLanes = 12;

inline size_t axm_ring_bytes(int wmax, bool tf32 = false) {
    const size_t b = tf32 ? (size_t)kAxmStages * kAxfRows * wmax * sizeof(float)
                          : (size_t)kAxmStages * kAxmRows * wmax * sizeof(__nv_bfloat16);
    return (b + 15) / 16 * 16;
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t y;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void mma_tf32_1688(float (&d)[4], const uint4& a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// TF32 = true: the same product from FP32-sized TF32 tiles with mma.m16n8k8
// (8-row k-blocks; B fragment b0 = row q, b1 = row q + 4 of output g; the A
// operand holds x, y, z rounded to TF32 in rows 0-2 and their TF32
// remainders in rows 8-10, so x again carries about twice the storage
// precision).
template <bool TF32>
__global__ void __launch_bounds__(32 * (kAxtWarps + 1)) k_axpy_mma(const AxDesc* __restrict__ descs,
                                                                   const AxBlock* __restrict__ blocks, AxBases B,
                                                                   int ring_bytes, int* __restrict__ err) {
    using namespace tma;
    using E = typename std::conditional<TF32, float, __nv_bfloat16>::type;
    constexpr int KB = TF32 ? 8 : 16;   // matrix rows per mma k-block
    constexpr int S = kAxmStages, R = TF32 ? kAxfRows : kAxmRows;
    static_assert(R % KB == 0, "stages hold whole k-blocks");
    extern __shared__ __align__(128) unsigned char axm_smem[];
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ int abort_flag;
    const AxBlock bk = blocks[blockIdx.x];
    const AxDesc D = descs[bk.desc];
    const int w = ax_tile_width(D.n_out, bk.o0, D.ld, 8);
    const int Kp = (D.K + KB - 1) / KB * KB;
    E* ring = reinterpret_cast<E*>(axm_smem);
    // A operands of lanes 0..11 only (rows 0-2 and 8-10: the lanes of groups 3..7 hold zeros)
    uint4* frag = reinterpret_cast<uint4*>(axm_smem + ring_bytes);   // Kp / KB x 12 lanes
    float4* xs = reinterpret_cast<float4*>(axm_smem + ring_bytes + (size_t)(Kp / KB) * kAxmFragLanes * sizeof(uint4));
    const E* tile = reinterpret_cast<const E*>(B.pool) + D.a_off + (int64_t)bk.o0 * Kp;
    const int n_st = (Kp + R - 1) / R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    pdl_trigger();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < S; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kAxtWarps);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (warp == kAxtWarps) {
        // producer: whole 16-row blocks per stage, one bulk copy each
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < n_st; ++i) {
                const int slot = i % S;
                if (i >= S && !mbar_wait(&empty[slot], ((i / S) - 1) & 1, &abort_flag)) {
                    abort_flag = 1;
                    atomicOr(err, ERR_TIMEOUT);
                    break;
                }
                const int rows = min(R, Kp - i * R);
                const uint32_t bytes = (uint32_t)(rows * w * (int)sizeof(E));
                uint32_t expect = bytes;
                if (blockIdx.x == 0 && i == 0 && *reinterpret_cast<volatile int*>(&g_test_copy_extra) > 0)
                    expect += (uint32_t)max(atomicExch(&g_test_copy_extra, 0), 0);
                mbar_arrive_expect_tx(&full[slot], expect);
                bulk_g2s(ring + (size_t)slot * R * w, tile + (int64_t)i * R * w, bytes, &full[slot]);
                issued = i + 1;
            }
            for (int i = max(0, issued - S); i < issued; ++i)
                if (!mbar_wait(&full[i % S], (i / S) & 1)) atomicOr(err, ERR_TIMEOUT);
        }
        return;
    }
    // consumers: stage x, then the A operands of every k-block (hi rows 0..2, remainders 8..10)
    {
        const int* xi = D.bidx_off >= 0 ? B.bidx + D.bidx_off : nullptr;
        StageIdx si;
        stage_f4_indices(si, D.K, xi, threadIdx.x, 32 * kAxtWarps);   // constant: before the wait
        pdl_wait();
        stage_f4_values(xs, D.K, B.x + D.x_off, xi, si, threadIdx.x, 32 * kAxtWarps);
    }
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kAxtWarps) : "memory");
    if (TF32) {
        // a0 = (row g, k q), a1 = (row g + 8, k q), a2 = (row g, k q + 4), a3 = (row g + 8, k q + 4)
        for (int f = threadIdx.x; f < (Kp / KB) * kAxmFragLanes; f += 32 * kAxtWarps) {
            const int kb = f / kAxmFragLanes, l = f % kAxmFragLanes, g = l >> 2, q = l & 3;
            uint32_t a[4] = {0u, 0u, 0u, 0u};
            {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = kb * 8 + q + 4 * h;
                    float v = 0.f;
                    if (k < D.K) {
                        const float4 xv = xs[k];
                        v = g == 0 ? xv.x : (g == 1 ? xv.y : xv.z);
                    }
                    const uint32_t hi = to_tf32(v);
                    a[2 * h] = hi;
                    a[2 * h + 1] = to_tf32(v - __uint_as_float(hi));
                }
            }
            frag[f] = make_uint4(a[0], a[1], a[2], a[3]);
        }
    } else
    for (int f = threadIdx.x; f < (Kp >> 4) * kAxmFragLanes; f += 32 * kAxtWarps) {
        const int kb = f / kAxmFragLanes, l = f % kAxmFragLanes, g = l >> 2, q = l & 3;
        uint32_t hv[4] = {0u, 0u, 0u, 0u}, lv[4] = {0u, 0u, 0u, 0u};   // (a0, a2) hi, (a1, a3) lo
        {
#pragma unroll
            for (int h = 0; h < 2; ++h) {       // h = 0: rows 2q, 2q+1; h = 1: rows 2q+8, 2q+9
                __nv_bfloat16 hi[2], lo[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int k = kb * 16 + 2 * q + 8 * h + e;
                    float v = 0.f;
                    if (k < D.K) {
                        const float4 xv = xs[k];
                        v = g == 0 ? xv.x : (g == 1 ? xv.y : xv.z);
                    }
                    hi[e] = __float2bfloat16_rn(v);
                    lo[e] = __float2bfloat16_rn(v - __bfloat162float(hi[e]));
                }
                hv[h] = pack_bf16(hi[0], hi[1]);
                lv[h] = pack_bf16(lo[0], lo[1]);
            }
        }
        frag[f] = make_uint4(hv[0], lv[0], hv[1], lv[1]);
    }
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kAxtWarps) : "memory");
    const int nb8 = w >> 3;
    float acc[kAxmNb][4];
#pragma unroll
    for (int j = 0; j < kAxmNb; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (int i = 0; i < n_st; ++i) {
        const int slot = i % S;
        if (!mbar_wait(&full[slot], (i / S) & 1, &abort_flag)) {
            if (lane == 0) {
                abort_flag = 1;
                atomicOr(err, ERR_TIMEOUT);
            }
            break;
        }
        const int kbs = min(R, Kp - i * R) / KB;
        const uint2* st = reinterpret_cast<const uint2*>(ring + (size_t)slot * R * w);
        for (int kk = 0; kk < kbs; ++kk) {
            const uint4 a = lane < kAxmFragLanes ? frag[(i * (R / KB) + kk) * kAxmFragLanes + lane]
                                                 : make_uint4(0u, 0u, 0u, 0u);
            const uint2* blk = st + (size_t)kk * nb8 * 32;   // a k-block x 8-output block: 32 lanes x 8 bytes
#pragma unroll
            for (int j = 0; j < kAxmNb; ++j) {
                const int nb = warp + kAxtWarps * j;
                if (nb < nb8) {
                    const uint2 bv = blk[nb * 32 + lane];
                    if (TF32) mma_tf32_1688(acc[j], a, bv.x, bv.y);
                    else mma_bf16_16816(acc[j], a, bv.x, bv.y);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
    }
    // epilogue: lanes 0..3 gather x, y, z of outputs 2q, 2q+1 from lanes q, q+4, q+8
    const int q = lane & 3;
    float4* out = B.out + D.out_off;
    const float4* add = (D.add_off >= 0) ? B.add + D.add_off : nullptr;
#pragma unroll
    for (int j = 0; j < kAxmNb; ++j) {
        const int nb = warp + kAxtWarps * j;
        if (nb >= nb8) break;   // uniform across the warp
        const float v0 = acc[j][0] + acc[j][2], v1 = acc[j][1] + acc[j][3];
        const float y0 = __shfl_sync(0xffffffffu, v0, q + 4), y1 = __shfl_sync(0xffffffffu, v1, q + 4);
        const float z0 = __shfl_sync(0xffffffffu, v0, q + 8), z1 = __shfl_sync(0xffffffffu, v1, q + 8);
        if (lane < 4) {
            const int o = bk.o0 + nb * 8 + 2 * q;
            if (o < D.n_out) {
                const float4 b = add ? add[o] : make_float4(0.f, 0.f, 0.f, 0.f);
                out[o] = make_float4(b.x + v0, b.y + y0, b.z + z0, 0.f);
            }
            if (o + 1 < D.n_out) {
                const float4 b = add ? add[o + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
                out[o + 1] = make_float4(b.x + v1, b.y + y1, b.z + z1, 0.f);
            }
        }
    }
}

// gather: c_B[j] = b_B[j] + sum over the domains touching j of their c_d entry (fixed order)
__global__ void k_gather(int n_B, const int* __restrict__ ptr, const int* __restrict__ rows,
                         const float4* __restrict__ bB, const float4* __restrict__ tc, float4* __restrict__ cB) {
    pdl_trigger();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_B) return;
    // the index lists are constant: read them (the first four entries) before
    // the wait for the predecessor, so only the sums' own loads follow it
    constexpr int kPre = 4;
    const int k0 = ptr[j], k1 = ptr[j + 1];
    int r[kPre];
#pragma unroll
    for (int q = 0; q < kPre; ++q) r[q] = (k0 + q < k1) ? rows[k0 + q] : -1;
    pdl_wait();
    float4 acc = bB[j];
#pragma unroll
    for (int q = 0; q < kPre; ++q) {
        if (r[q] >= 0) {
            const float4 c = tc[r[q]];
            acc.x += c.x; acc.y += c.y; acc.z += c.z;
        }
    }
    for (int k = k0 + kPre; k < k1; ++k) {
        const float4 c = tc[rows[k]];
        acc.x += c.x; acc.y += c.y; acc.z += c.z;
    }
    cB[j] = acc;
}

constexpr int kCoarseChunk = 2048;

// coarse: block (rb, ch) forms rows [rb*RPC, +RPC) of S^-1 times the column chunk ch of c_B
template <class T>
__global__ void __launch_bounds__(256) k_coarse(const T* __restrict__ S, int n_B, int ld, int rpc,
                                                const float4* __restrict__ cB, float4* __restrict__ part) {
    __shared__ float4 xs[kCoarseChunk];
    const int c0 = blockIdx.y * kCoarseChunk;
    const int ncol = min(kCoarseChunk, ld - c0);   // ld is a multiple of the vector width
    for (int k = threadIdx.x; k < ncol; k += blockDim.x) {
        int c = c0 + k;
        xs[k] = (c < n_B) ? cB[c] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const int r0 = blockIdx.x * rpc;
    const int rows = min(rpc, n_B - r0);
    if (rows <= 0) return;
    block_rows<T, 32>(S + (int64_t)r0 * ld + c0, rows, ld, ncol, xs, part + (int64_t)blockIdx.y * n_B + r0,
                      nullptr);
}

// coarse, balanced form: one 512-thread block per SM holds all of c_B in
// shared memory (three float planes); the (row pair, 2048-column chunk) units
// of S^-1 are split into equal contiguous ranges, one per warp, so every warp
// streams the same number of bytes.  Each unit's partial sums go to
// part[chunk][row].
constexpr int kCoarseWarps = 16;

template <class T>
struct CoarseRows;
template <>
struct CoarseRows<float> {
    static constexpr int R = 2;
};
template <>
struct CoarseRows<__nv_bfloat16> {
    static constexpr int R = 4;
};

template <class T>
__global__ void __launch_bounds__(512, kCoarseBps) k_coarse_bal(const T* __restrict__ S, int n_B, int ld, int cols, int nch,
                                                        const float4* __restrict__ cB, float4* __restrict__ part) {
    extern __shared__ float xsm[];
    float* x0 = xsm;
    float* x1 = xsm + cols;
    float* x2 = xsm + 2 * cols;
    pdl_trigger();
    pdl_wait();
    stage_planes(x0, x1, x2, n_B, cols, cB, nullptr, threadIdx.x, blockDim.x);
    __syncthreads();
    constexpr int VN = VecN<T>::N;
    constexpr int RU = CoarseRows<T>::R;   // rows per unit: x values reused RU times
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kCoarseWarps + (threadIdx.x >> 5);
    const int64_t W = (int64_t)gridDim.x * kCoarseWarps;
    const int n_rg = (n_B + RU - 1) / RU;
    const int64_t U = (int64_t)n_rg * nch;
    const int64_t u0 = U * gw / W, u1 = U * (gw + 1) / W;
    for (int64_t u = u0; u < u1; ++u) {
        const int rg = (int)(u / nch), ch = (int)(u % nch);
        const int r0 = RU * rg;
        const T* a[RU];
#pragma unroll
        for (int k = 0; k < RU; ++k) a[k] = S + (int64_t)((r0 + k < n_B) ? r0 + k : r0) * ld;
        const int cb = ch * kCoarseChunk, ce = min(cols, cb + kCoarseChunk);
        float acc[RU][3];
#pragma unroll
        for (int k = 0; k < RU; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0.f;
#pragma unroll 4
        for (int c = cb + lane * VN; c < ce; c += 32 * VN) {
            float v[RU][VN];
#pragma unroll
            for (int k = 0; k < RU; ++k) load_vec(a[k] + c, v[k]);
#pragma unroll
            for (int j = 0; j < VN; j += 4) {
                const float4 p0 = *reinterpret_cast<const float4*>(x0 + c + j);
                const float4 p1 = *reinterpret_cast<const float4*>(x1 + c + j);
                const float4 p2 = *reinterpret_cast<const float4*>(x2 + c + j);
                const float q0[4] = {p0.x, p0.y, p0.z, p0.w};
                const float q1[4] = {p1.x, p1.y, p1.z, p1.w};
                const float q2[4] = {p2.x, p2.y, p2.z, p2.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int k = 0; k < RU; ++k) {
                        acc[k][0] = fmaf(v[k][j + i], q0[i], acc[k][0]);
                        acc[k][1] = fmaf(v[k][j + i], q1[i], acc[k][1]);
                        acc[k][2] = fmaf(v[k][j + i], q2[i], acc[k][2]);
                    }
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int k = 0; k < RU; ++k) {
                acc[k][0] += __shfl_xor_sync(0xffffffffu, acc[k][0], off);
                acc[k][1] += __shfl_xor_sync(0xffffffffu, acc[k][1], off);
                acc[k][2] += __shfl_xor_sync(0xffffffffu, acc[k][2], off);
            }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < RU; ++k)
                if (r0 + k < n_B) part[(int64_t)ch * n_B + r0 + k] = make_float4(acc[k][0], acc[k][1], acc[k][2], 0.f);
        }
    }
}

// Batched coarse products: the (row pair, chunk) units of every slot's S^-1
// are concatenated; block c takes units [U c / C, U (c+1) / C), stages each
// overlapped slot's c_B in shared memory and splits that piece evenly over
// its warps.  Each unit is computed exactly as in k_coarse_bal.
__global__ void __launch_bounds__(512, 1) k_coarse_b(const CoarseDescB* __restrict__ cd, int n_desc, int64_t U,
                                                      int max_cols) {
    extern __shared__ float xsm[];
    float* x0 = xsm;
    float* x1 = xsm + max_cols;
    float* x2 = xsm + 2 * max_cols;
    constexpr int VN = 4;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t b0 = U * blockIdx.x / gridDim.x, b1 = U * (blockIdx.x + 1) / gridDim.x;
    for (int di = 0; di < n_desc; ++di) {
        const CoarseDescB D = cd[di];
        const int64_t nu = (int64_t)((D.n_B + 1) / 2) * D.nch;
        const int64_t lo = b0 > D.u0 ? b0 : D.u0;
        const int64_t hi = b1 < D.u0 + nu ? b1 : D.u0 + nu;
        if (hi <= lo) continue;
        __syncthreads();
        for (int k = threadIdx.x; k < D.ld; k += blockDim.x) {
            float4 v = (k < D.n_B) ? D.cB[k] : make_float4(0.f, 0.f, 0.f, 0.f);
            x0[k] = v.x;
            x1[k] = v.y;
            x2[k] = v.z;
        }
        __syncthreads();
        const int64_t n = hi - lo;
        const int64_t w0 = lo + n * warp / kCoarseWarps, w1 = lo + n * (warp + 1) / kCoarseWarps;
        for (int64_t u = w0; u < w1; ++u) {
            const int64_t ul = u - D.u0;
            const int rp = (int)(ul / D.nch), ch = (int)(ul % D.nch);
            const int r0 = 2 * rp;
            const bool two = (r0 + 1) < D.n_B;
            const float* a0 = D.S + (int64_t)r0 * D.ld;
            const float* a1 = D.S + (int64_t)(two ? r0 + 1 : r0) * D.ld;
            const int cb = ch * kCoarseChunk, ce = min(D.ld, cb + kCoarseChunk);
            float acc[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll 4
            for (int c = cb + lane * VN; c < ce; c += 32 * VN) {
                float v[2][VN];
                load_vec(a0 + c, v[0]);
                load_vec(a1 + c, v[1]);
                const float4 p0 = *reinterpret_cast<const float4*>(x0 + c);
                const float4 p1 = *reinterpret_cast<const float4*>(x1 + c);
                const float4 p2 = *reinterpret_cast<const float4*>(x2 + c);
                const float q0[4] = {p0.x, p0.y, p0.z, p0.w};
                const float q1[4] = {p1.x, p1.y, p1.z, p1.w};
                const float q2[4] = {p2.x, p2.y, p2.z, p2.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        acc[k][0] = fmaf(v[k][i], q0[i], acc[k][0]);
                        acc[k][1] = fmaf(v[k][i], q1[i], acc[k][1]);
                        acc[k][2] = fmaf(v[k][i], q2[i], acc[k][2]);
                    }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    acc[k][0] += __shfl_xor_sync(0xffffffffu, acc[k][0], off);
                    acc[k][1] += __shfl_xor_sync(0xffffffffu, acc[k][1], off);
                    acc[k][2] += __shfl_xor_sync(0xffffffffu, acc[k][2], off);
                }
            if (lane == 0) {
                D.part[(int64_t)ch * D.n_B + r0] = make_float4(acc[0][0], acc[0][1], acc[0][2], 0.f);
                if (two) D.part[(int64_t)ch * D.n_B + r0 + 1] = make_float4(acc[1][0], acc[1][1], acc[1][2], 0.f);
            }
        }
    }
}

// Row-oriented products of many dense blocks in one balanced launch
// ("row form"): out[r] = add[r] + A[r, 0:cols] . x for every row r of every
// descriptor, x being the descriptor's contiguous or gathered slice of B.x.
// The RU-row units of all descriptors are concatenated; block b takes the
// units [blk_u[b], blk_u[b+1]) (cut on the host so every block streams about
// the same number of matrix bytes), stages each overlapped descriptor's x in
// shared memory as three float planes and splits its piece evenly over its
// warps.  A unit is a full row dot product: lanes stride the row with 16-byte
// loads, a fixed-order shuffle tree combines them (deterministic).
template <class T>
struct RowRows {
    static constexpr int R = 4;
};
template <>
struct RowRows<float> {
    static constexpr int R = kRowRu32;
};

template <class T>
__global__ void __launch_bounds__(32 * kRowWarps, kRowBps) k_rowdot(const RowDesc* __restrict__ descs, int n_desc,
                                                                const int64_t* __restrict__ blk_u, AxBases B,
                                                                int xcap) {
    extern __shared__ float xsm[];
    float* x0 = xsm;
    float* x1 = xsm + xcap;
    float* x2 = xsm + 2 * xcap;
    constexpr int VN = VecN<T>::N;
    constexpr int RU = RowRows<T>::R;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t b0 = blk_u[blockIdx.x], b1 = blk_u[blockIdx.x + 1];
    const T* pool = reinterpret_cast<const T*>(B.pool);
    for (int di = 0; di < n_desc; ++di) {
        const RowDesc D = descs[di];
        const int64_t nu = (D.rows + RU - 1) / RU;
        const int64_t lo = b0 > D.u0 ? b0 : D.u0;
        const int64_t hi = b1 < D.u0 + nu ? b1 : D.u0 + nu;
        if (hi <= lo) continue;
        __syncthreads();
        if (D.xidx_off >= 0) stage_planes(x0, x1, x2, D.cols, D.ld, B.x, B.bidx + D.xidx_off, threadIdx.x, blockDim.x);
        else stage_planes(x0, x1, x2, D.cols, D.ld, B.x + D.x_off, nullptr, threadIdx.x, blockDim.x);
        __syncthreads();
        const int64_t n = hi - lo;
        const int64_t w0 = lo + n * warp / kRowWarps, w1 = lo + n * (warp + 1) / kRowWarps;
        for (int64_t u = w0; u < w1; ++u) {
            const int r0 = RU * (int)(u - D.u0);
            const T* a[RU];
#pragma unroll
            for (int k = 0; k < RU; ++k) a[k] = pool + D.a_off + (int64_t)((r0 + k < D.rows) ? r0 + k : r0) * D.ld;
            float acc[RU][3];
#pragma unroll
            for (int k = 0; k < RU; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0.f;
#pragma unroll kRowUnroll
            for (int c = lane * VN; c < D.ld; c += 32 * VN) {
                float v[RU][VN];
#pragma unroll
                for (int k = 0; k < RU; ++k) load_vec(a[k] + c, v[k]);
#pragma unroll
                for (int j = 0; j < VN; j += 4) {
                    const float4 p0 = *reinterpret_cast<const float4*>(x0 + c + j);
                    const float4 p1 = *reinterpret_cast<const float4*>(x1 + c + j);
                    const float4 p2 = *reinterpret_cast<const float4*>(x2 + c + j);
                    const float q0[4] = {p0.x, p0.y, p0.z, p0.w};
                    const float q1[4] = {p1.x, p1.y, p1.z, p1.w};
                    const float q2[4] = {p2.x, p2.y, p2.z, p2.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int k = 0; k < RU; ++k) {
                            acc[k][0] = fmaf(v[k][j + i], q0[i], acc[k][0]);
                            acc[k][1] = fmaf(v[k][j + i], q1[i], acc[k][1]);
                            acc[k][2] = fmaf(v[k][j + i], q2[i], acc[k][2]);
                        }
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                for (int k = 0; k < RU; ++k) {
                    acc[k][0] += __shfl_xor_sync(0xffffffffu, acc[k][0], off);
                    acc[k][1] += __shfl_xor_sync(0xffffffffu, acc[k][1], off);
                    acc[k][2] += __shfl_xor_sync(0xffffffffu, acc[k][2], off);
                }
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < RU; ++k) {
                    const int r = r0 + k;
                    if (r >= D.rows) break;
                    const float4 ad = (D.add_off >= 0) ? B.add[D.add_off + r] : make_float4(0.f, 0.f, 0.f, 0.f);
                    B.out[D.out_off + r] = make_float4(ad.x + acc[k][0], ad.y + acc[k][1], ad.z + acc[k][2], 0.f);
                }
            }
        }
    }
}

// reduce: x_B[j] = sum over chunks (fixed order) of part[ch][j]
__global__ void k_reduce(int n_B, int n_chunks, const float4* __restrict__ part, float4* __restrict__ xB) {
    pdl_trigger();
    pdl_wait();
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_B) return;
    float4 acc = part[j];
    for (int c = 1; c < n_chunks; ++c) {
        float4 p = part[(int64_t)c * n_B + j];
        acc.x += p.x; acc.y += p.y; acc.z += p.z;
    }
    xB[j] = make_float4(acc.x, acc.y, acc.z, 0.f);
}

// r = b - K x over free vertices with FP64 accumulation (refinement residual)
__global__ void k_residual(int n_free, const int* __restrict__ ptr, const int* __restrict__ col,
                           const double* __restrict__ val, const float4* __restrict__ b, const float4* __restrict__ x,
                           float4* __restrict__ r) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_free) return;
    float4 bb = b[i];
    double ax = bb.x, ay = bb.y, az = bb.z;
    for (int k = ptr[i]; k < ptr[i + 1]; ++k) {
        double kv = val[k];
        float4 xv = x[col[k]];
        ax -= kv * (double)xv.x;
        ay -= kv * (double)xv.y;
        az -= kv * (double)xv.z;
    }
    r[i] = make_float4((float)ax, (float)ay, (float)az, 0.f);
}

__global__ void k_axpy(int n, const float4* __restrict__ dx, float4* __restrict__ x) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 a = x[i], d = dx[i];
    x[i] = make_float4(a.x + d.x, a.y + d.y, a.z + d.z, a.w);
}

// One Jacobi sweep with Chebyshev weight omega over the free vertices:
// x_hat = x + D^-1 (b - K x) (FP64 accumulation), out = omega (x_hat - x_prev) + x_prev.
__global__ void k_cheb_jacobi(int n_free, const int* __restrict__ ptr, const int* __restrict__ col,
                              const double* __restrict__ val, const double* __restrict__ dinv,
                              const float4* __restrict__ b, const float4* __restrict__ x,
                              const float4* __restrict__ x_prev, float omega, float4* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_free) return;
    const float4 bb = b[i];
    double rx = bb.x, ry = bb.y, rz = bb.z;
    for (int k = ptr[i]; k < ptr[i + 1]; ++k) {
        const double kv = val[k];
        const float4 xv = x[col[k]];
        rx -= kv * (double)xv.x;
        ry -= kv * (double)xv.y;
        rz -= kv * (double)xv.z;
    }
    const float4 xi = x[i], xp = x_prev[i];
    const double di = dinv[i];
    const float hx = (float)((double)xi.x + di * rx), hy = (float)((double)xi.y + di * ry),
                hz = (float)((double)xi.z + di * rz);
    out[i] = make_float4(fmaf(omega, hx - xp.x, xp.x), fmaf(omega, hy - xp.y, xp.y), fmaf(omega, hz - xp.z, xp.z), 0.f);
}

// Row-form products streamed through shared memory with bulk asynchronous
// copies.  A block's rows of one descriptor are contiguous in the pool (row
// stride ld), so one cp.async.bulk moves a whole stage of RS rows
// (RS = kRowtStageBytes / row bytes); a ring of kRowtStages stages keeps them
// in flight.  The rows go to the consumer warps in pairs (pair p to warp
// p mod kRowtWarps), so every x value read from shared memory serves two
// rows: lanes stride the rows with 16-byte shared-memory loads against x
// staged as three float planes, a fixed-order shuffle tree combines them
// (deterministic).  Every wait is bounded, as in k_axpy_tma.
#ifndef PDG_ROWT_STAGE_BYTES
#define PDG_ROWT_STAGE_BYTES 24576
#endif
#ifndef PDG_ROWT_STAGES
#define PDG_ROWT_STAGES 3
#endif
#ifndef PDG_ROWT_WARPS
#define PDG_ROWT_WARPS 8
#endif
constexpr int kRowtStageBytes = PDG_ROWT_STAGE_BYTES;
constexpr int kRowtStages = PDG_ROWT_STAGES;
constexpr int kRowtWarps = PDG_ROWT_WARPS;

// BATCHED (serving): descriptor D works on the arrays of request D.slot,
// multi[D.slot]; otherwise on B.
template <class T, bool BATCHED>
__global__ void __launch_bounds__(32 * (kRowtWarps + 1)) k_rowdot_tma(const RowDesc* __restrict__ descs, int n_desc,
                                                                      const int64_t* __restrict__ blk_u, AxBases B,
                                                                      const AxBases* __restrict__ multi, int xcap,
                                                                      int* __restrict__ err) {
    using namespace tma;
    constexpr int VN = VecN<T>::N;
    constexpr int RU = RowRows<T>::R;
    constexpr int S = kRowtStages;
    constexpr int SE = kRowtStageBytes / (int)sizeof(T);   // elements of one stage
    extern __shared__ __align__(128) unsigned char rt_smem[];
    T* ring = reinterpret_cast<T*>(rt_smem);
    float* x0 = reinterpret_cast<float*>(rt_smem + (size_t)S * kRowtStageBytes);
    float* x1 = x0 + xcap;
    float* x2 = x1 + xcap;
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ int abort_flag;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t b0 = blk_u[blockIdx.x], b1 = blk_u[blockIdx.x + 1];
    const T* pool = reinterpret_cast<const T*>(B.pool);
    pdl_trigger();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < S; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kRowtWarps);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (warp == kRowtWarps) {
        if (lane == 0) {
            int g = 0, issued = 0;
            bool ok = true;
            for (int di = 0; di < n_desc && ok; ++di) {
                const RowDesc D = descs[di];
                const int64_t nu = (D.rows + RU - 1) / RU;
                const int64_t lo = b0 > D.u0 ? b0 : D.u0;
                const int64_t hi = b1 < D.u0 + nu ? b1 : D.u0 + nu;
                if (hi <= lo) continue;
                const int r_lo = (int)(lo - D.u0) * RU;
                const int r_hi = min((int)(hi - D.u0) * RU, D.rows);
                const int RS = max(1, SE / D.ld);
                for (int r = r_lo; r < r_hi; r += RS, ++g) {
                    const int slot = g % S;
                    if (g >= S && !mbar_wait(&empty[slot], ((g / S) - 1) & 1, &abort_flag)) {
                        abort_flag = 1;
                        atomicOr(err, ERR_TIMEOUT);
                        ok = false;
                        break;
                    }
                    const int rows = min(RS, r_hi - r);
                    const uint32_t bytes = (uint32_t)rows * (uint32_t)D.ld * (uint32_t)sizeof(T);
                    mbar_arrive_expect_tx(&full[slot], bytes);
                    const T* pl = BATCHED ? reinterpret_cast<const T*>(multi[D.slot].pool) : pool;
                    bulk_g2s(ring + (size_t)slot * SE, pl + D.a_off + (int64_t)r * D.ld, bytes, &full[slot]);
                    issued = g + 1;
                }
            }
            for (int i = max(0, issued - S); i < issued; ++i)
                if (!mbar_wait(&full[i % S], (i / S) & 1)) atomicOr(err, ERR_TIMEOUT);
        }
        return;
    }
    // after an abort every consumer warp still runs every segment's barriers
    // (no warp may leave a barrier short); the stages are skipped
    pdl_wait();   // x comes from the predecessor; the producer streams the constant rows meanwhile
    int g = 0, pc = 0;
    for (int di = 0; di < n_desc; ++di) {
        const RowDesc D = descs[di];
        const int64_t nu = (D.rows + RU - 1) / RU;
        const int64_t lo = b0 > D.u0 ? b0 : D.u0;
        const int64_t hi = b1 < D.u0 + nu ? b1 : D.u0 + nu;
        if (hi <= lo) continue;
        const int r_lo = (int)(lo - D.u0) * RU;
        const int r_hi = min((int)(hi - D.u0) * RU, D.rows);
        const int RS = max(1, SE / D.ld);
        asm volatile("bar.sync 1, %0;" ::"n"(32 * kRowtWarps) : "memory");   // the previous x is no longer read
        const AxBases Bd = BATCHED ? multi[D.slot] : B;
        if (D.xidx_off >= 0) stage_planes(x0, x1, x2, D.cols, D.ld, Bd.x, Bd.bidx + D.xidx_off, threadIdx.x, 32 * kRowtWarps);
        else stage_planes(x0, x1, x2, D.cols, D.ld, Bd.x + D.x_off, nullptr, threadIdx.x, 32 * kRowtWarps);
        asm volatile("bar.sync 1, %0;" ::"n"(32 * kRowtWarps) : "memory");
        for (int r = r_lo; r < r_hi; r += RS, ++g) {
            const int slot = g % S;
            if (*reinterpret_cast<volatile int*>(&abort_flag)) break;
            if (!mbar_wait(&full[slot], (g / S) & 1, &abort_flag)) {
                if (lane == 0) {
                    abort_flag = 1;
                    atomicOr(err, ERR_TIMEOUT);
                }
                break;
            }
            const int rows = min(RS, r_hi - r);
            const T* st = ring + (size_t)slot * SE;
            // rows in pairs sharing every x read; pair pc goes to warp pc mod kRowtWarps
            const int np = (rows + 1) / 2;
            for (int q = 0; q < np; ++q, ++pc) {
                if (pc % kRowtWarps != warp) continue;
                const int j0 = 2 * q;
                const bool two = j0 + 1 < rows;
                const T* a0 = st + (size_t)j0 * D.ld;
                const T* a1 = two ? a0 + D.ld : a0;
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, t0 = 0.f, t1 = 0.f, t2 = 0.f;
#pragma unroll 2
                for (int c = lane * VN; c < D.ld; c += 32 * VN) {
                    float v[VN], u[VN];
                    load_vec_shared(a0 + c, v);
                    load_vec_shared(a1 + c, u);
#pragma unroll
                    for (int q4 = 0; q4 < VN; q4 += 4) {
                        const float4 p0 = *reinterpret_cast<const float4*>(x0 + c + q4);
                        const float4 p1 = *reinterpret_cast<const float4*>(x1 + c + q4);
                        const float4 p2 = *reinterpret_cast<const float4*>(x2 + c + q4);
                        s0 = fmaf(v[q4], p0.x, fmaf(v[q4 + 1], p0.y, fmaf(v[q4 + 2], p0.z, fmaf(v[q4 + 3], p0.w, s0))));
                        s1 = fmaf(v[q4], p1.x, fmaf(v[q4 + 1], p1.y, fmaf(v[q4 + 2], p1.z, fmaf(v[q4 + 3], p1.w, s1))));
                        s2 = fmaf(v[q4], p2.x, fmaf(v[q4 + 1], p2.y, fmaf(v[q4 + 2], p2.z, fmaf(v[q4 + 3], p2.w, s2))));
                        t0 = fmaf(u[q4], p0.x, fmaf(u[q4 + 1], p0.y, fmaf(u[q4 + 2], p0.z, fmaf(u[q4 + 3], p0.w, t0))));
                        t1 = fmaf(u[q4], p1.x, fmaf(u[q4 + 1], p1.y, fmaf(u[q4 + 2], p1.z, fmaf(u[q4 + 3], p1.w, t1))));
                        t2 = fmaf(u[q4], p2.x, fmaf(u[q4 + 1], p2.y, fmaf(u[q4 + 2], p2.z, fmaf(u[q4 + 3], p2.w, t2))));
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    s0 += __shfl_xor_sync(0xffffffffu, s0, off);
                    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
                    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
                    t0 += __shfl_xor_sync(0xffffffffu, t0, off);
                    t1 += __shfl_xor_sync(0xffffffffu, t1, off);
                    t2 += __shfl_xor_sync(0xffffffffu, t2, off);
                }
                if (lane == 0) {
                    const int row = r + j0;
                    const float4 ad = (D.add_off >= 0) ? Bd.add[D.add_off + row] : make_float4(0.f, 0.f, 0.f, 0.f);
                    Bd.out[D.out_off + row] = make_float4(ad.x + s0, ad.y + s1, ad.z + s2, 0.f);
                    if (two) {
                        const float4 ae = (D.add_off >= 0) ? Bd.add[D.add_off + row + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
                        Bd.out[D.out_off + row + 1] = make_float4(ae.x + t0, ae.y + t1, ae.z + t2, 0.f);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
        }
    }
}

// Row-form BF16 products on the tensor cores: out[r] = add[r] + A[r, :] . x
// with A stored as 16 x 16 blocks in the register order of the A operand of
// mma.m16n8k16 (rows and columns padded to 16; a 16-row block-row is one
// contiguous range), so one 16-byte shared load per lane feeds one mma.
// The B operand is x: columns 0..2 hold x, y, z rounded to BF16, columns
// 3..5 their BF16 remainders.  A CTA streams whole 16-row block-rows of its
// unit range in stages of up to kRowmStageBytes with bulk copies; the 16-col
// blocks of a stage go to the consumer warps in turn, each warp accumulating
// its own 16 x 8 tile, and the warps' tiles are added in warp order
// (deterministic) before the 16 outputs of the block-row are written.  The
// blocks are written in this order by k_cast_rowfrag16 at prefactorisation.
__device__ __forceinline__ void mma_bf16_rowform(float (&d)[4], const uint4& a, const uint2& b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y));
}

#ifndef PDG_ROWM_STAGE_BYTES
#define PDG_ROWM_STAGE_BYTES 16384
#endif
#ifndef PDG_ROWM_STAGES
#define PDG_ROWM_STAGES 3
#endif
constexpr int kRowmStageBytes = PDG_ROWM_STAGE_BYTES;   // a multiple of 512 (whole 16 x 16 blocks)
constexpr int kRowmStages = PDG_ROWM_STAGES;

// ring, B fragments (16 B per padded column), the warps' tiles
inline size_t rowm_smem_bytes(int xcap) {
    const int kp = (std::max(xcap, 1) + 15) & ~15;
    return (size_t)kRowmStages * kRowmStageBytes + sizeof(uint2) * 2 * (size_t)kp + sizeof(float) * 4 * 32 * kRowtWarps;
}

__global__ void __launch_bounds__(32 * (kRowtWarps + 1)) k_rowdot_mma(const RowDesc* __restrict__ descs, int n_desc,
                                                                      const int64_t* __restrict__ blk_u, AxBases B,
                                                                      int xcap, int* __restrict__ err) {
    using namespace tma;
    constexpr int S = kRowmStages;
    constexpr int SB = kRowmStageBytes / 512;   // 16 x 16 blocks of one stage
    extern __shared__ __align__(128) unsigned char rm_smem[];
    const int kcap = (xcap + 15) & ~15;
    __nv_bfloat16* ring = reinterpret_cast<__nv_bfloat16*>(rm_smem);
    uint2* bfr = reinterpret_cast<uint2*>(rm_smem + (size_t)S * kRowmStageBytes);   // kcap / 16 blocks x 32 lanes
    float* red = reinterpret_cast<float*>(bfr + 2 * kcap);                           // kRowtWarps x 32 lanes x 4
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ int abort_flag;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t b0 = blk_u[blockIdx.x], b1 = blk_u[blockIdx.x + 1];
    const __nv_bfloat16* pool = reinterpret_cast<const __nv_bfloat16*>(B.pool);
    pdl_trigger();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < S; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kRowtWarps);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (warp == kRowtWarps) {
        // producer: every block-row of the range, in stages of up to SB blocks
        if (lane == 0) {
            int g = 0, issued = 0;
            bool ok = true;
            for (int di = 0; di < n_desc && ok; ++di) {
                const RowDesc D = descs[di];
                const int64_t nu = (D.rows + 15) / 16;
                const int64_t lo = b0 > D.u0 ? b0 : D.u0;
                const int64_t hi = b1 < D.u0 + nu ? b1 : D.u0 + nu;
                const int nkb = D.ld >> 4;
                for (int64_t u = lo; u < hi && ok; ++u) {
                    const __nv_bfloat16* row = pool + D.a_off + (u - D.u0) * 16 * (int64_t)D.ld;
                    for (int kb0 = 0; kb0 < nkb; kb0 += SB, ++g) {
                        const int slot = g % S;
                        if (g >= S && !mbar_wait(&empty[slot], ((g / S) - 1) & 1, &abort_flag)) {
                            abort_flag = 1;
                            atomicOr(err, ERR_TIMEOUT);
                            ok = false;
                            break;
                        }
                        const uint32_t bytes = (uint32_t)min(SB, nkb - kb0) * 512u;
                        mbar_arrive_expect_tx(&full[slot], bytes);
                        bulk_g2s(ring + (size_t)slot * (SB * 256), row + (int64_t)kb0 * 256, bytes, &full[slot]);
                        issued = g + 1;
                    }
                }
            }
            for (int i = max(0, issued - S); i < issued; ++i)
                if (!mbar_wait(&full[i % S], (i / S) & 1)) atomicOr(err, ERR_TIMEOUT);
        }
        return;
    }
    pdl_wait();   // x comes from the predecessor; the producer streams the constant rows meanwhile
    int g = 0;
    for (int di = 0; di < n_desc; ++di) {
        const RowDesc D = descs[di];
        const int64_t nu = (D.rows + 15) / 16;
        const int64_t lo = b0 > D.u0 ? b0 : D.u0;
        const int64_t hi = b1 < D.u0 + nu ? b1 : D.u0 + nu;
        if (hi <= lo) continue;
        const int nkb = D.ld >> 4;
        // the B operands of this block's x, one thread per column k: B[k][n] for
        // n = 0..2 is x, y, z rounded to BF16, n = 3..5 their BF16 remainders,
        // n = 6, 7 and the padded columns are zero.  In the mma B layout, k lies
        // in block k / 16 at lane 4 n + ((k mod 8) / 2), register (k mod 16) / 8,
        // half k mod 2.
        asm volatile("bar.sync 1, %0;" ::"n"(32 * kRowtWarps) : "memory");   // the previous B is no longer read
        {
            __nv_bfloat16* bh = reinterpret_cast<__nv_bfloat16*>(bfr);
            for (int k = threadIdx.x; k < nkb * 16; k += 32 * kRowtWarps) {
                float v[3] = {0.f, 0.f, 0.f};
                if (k < D.cols) {
                    const float4 xv = D.xidx_off >= 0 ? B.x[B.bidx[D.xidx_off + k]] : B.x[D.x_off + k];
                    v[0] = xv.x;
                    v[1] = xv.y;
                    v[2] = xv.z;
                }
                const int kb = k >> 4, kk = k & 15, q = (kk & 7) >> 1, h = kk >> 3, e = kk & 1;
                __nv_bfloat16* col = bh + (size_t)kb * 32 * 4 + q * 4 + h * 2 + e;   // lane 4 n + q: + 16 n halves
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const __nv_bfloat16 vh = __float2bfloat16_rn(v[c]);
                    col[16 * c] = vh;
                    col[16 * (c + 3)] = __float2bfloat16_rn(v[c] - __bfloat162float(vh));
                }
                col[16 * 6] = __float2bfloat16_rn(0.f);
                col[16 * 7] = __float2bfloat16_rn(0.f);
            }
        }
        asm volatile("bar.sync 1, %0;" ::"n"(32 * kRowtWarps) : "memory");
        for (int64_t u = lo; u < hi; ++u) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            for (int kb0 = 0; kb0 < nkb; kb0 += SB, ++g) {
                const int slot = g % S;
                if (*reinterpret_cast<volatile int*>(&abort_flag)) break;
                if (!mbar_wait(&full[slot], (g / S) & 1, &abort_flag)) {
                    if (lane == 0) {
                        abort_flag = 1;
                        atomicOr(err, ERR_TIMEOUT);
                    }
                    break;
                }
                const int nb = min(SB, nkb - kb0);
                const uint4* st = reinterpret_cast<const uint4*>(ring + (size_t)slot * (SB * 256));
                for (int kb = warp; kb < nb; kb += kRowtWarps)
                    mma_bf16_rowform(acc, st[kb * 32 + lane], bfr[(kb0 + kb) * 32 + lane]);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
            }
            // the warps' 16 x 8 tiles, added in warp order
#pragma unroll
            for (int i = 0; i < 4; ++i) red[(warp * 32 + lane) * 4 + i] = acc[i];
            asm volatile("bar.sync 1, %0;" ::"n"(32 * kRowtWarps) : "memory");
            if (warp == 0) {
                float d[4] = {0.f, 0.f, 0.f, 0.f};
                for (int w = 0; w < kRowtWarps; ++w)
#pragma unroll
                    for (int i = 0; i < 4; ++i) d[i] += red[(w * 32 + lane) * 4 + i];
                // lane 4 r + q holds columns 2q, 2q + 1 of rows r (d0, d1) and r + 8 (d2, d3):
                // x = col 0 + col 3, y = col 1 + col 4, z = col 2 + col 5
                const int base = lane & ~3;
                float o1[4], o2[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    o1[i] = __shfl_sync(0xffffffffu, d[i], base + 1);
                    o2[i] = __shfl_sync(0xffffffffu, d[i], base + 2);
                }
                if ((lane & 3) == 0) {
                    const int r0 = (int)(u - D.u0) * 16 + (lane >> 2);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int r = r0 + 8 * h;
                        if (r < D.rows) {
                            const float x = d[2 * h] + o1[2 * h + 1];
                            const float y = d[2 * h + 1] + o2[2 * h];
                            const float z = o1[2 * h] + o2[2 * h + 1];
                            const float4 ad = (D.add_off >= 0) ? B.add[D.add_off + r] : make_float4(0.f, 0.f, 0.f, 0.f);
                            B.out[D.out_off + r] = make_float4(ad.x + x, ad.y + y, ad.z + z, 0.f);
                        }
                    }
                }
            }
            asm volatile("bar.sync 1, %0;" ::"n"(32 * kRowtWarps) : "memory");   // red is free again
        }
    }
}

inline int nblk(int n, int b) { return (n + b - 1) / b; }

template <class T>
void launch_coarse(pd_mesh* m, const T* pool, const float4* cin, float4* part, cudaStream_t s) {
    if (m->coarse_blocks > 0) {
        const size_t smem = sizeof(float) * 3 * (size_t)m->ld_S;
        k_coarse_bal<T><<<m->coarse_blocks, 32 * kCoarseWarps, smem, s>>>(pool + m->off_S, m->cs_n, m->ld_S, m->ld_S,
                                                                          m->coarse_nchunks, cin, part);
    } else {
        dim3 grid(nblk(m->cs_n, m->coarse_rows_per_cta), m->coarse_nchunks);
        k_coarse<T><<<grid, 256, 0, s>>>(pool + m->off_S, m->cs_n, m->ld_S, m->coarse_rows_per_cta, cin, part);
    }
    PDG_CHECK_LAUNCH();
}

template <class T>
int axt_smem_limit() {
    static const int lim = std::min(allow_max_dynamic_smem(k_axpy_tma<T, false>),
                                    allow_max_dynamic_smem(k_axpy_tma<T, true>));
    return lim;
}

int axm_smem_limit() {
    static const int lim = std::min(allow_max_dynamic_smem(k_axpy_mma<false>), allow_max_dynamic_smem(k_axpy_mma<true>));
    return lim;
}

template <class T>
void launch_ax(const AxDesc* descs, const AxBlock* blocks, int n_blocks, int k_max, const AxBases& B, cudaStream_t s,
               int* tma_err = nullptr, int w_max = 0, bool pdl = false, bool tf32 = false) {
    if (n_blocks <= 0) return;
    const bool bf16 = std::is_same<T, __nv_bfloat16>::value;
    if (tma_err && (bf16 || tf32)) {
        // BF16 or TF32 tiles in the tensor-core fragment layout (k-blocks of 16 or 8 rows;
        // the A operands take 16 bytes per k-block for each of lanes 0..11)
        const int kb = bf16 ? 16 : 8;
        const int kp = (std::max(k_max, 1) + kb - 1) / kb * kb;
        const size_t ring = axm_ring_bytes(w_max, !bf16);
        const size_t smem = ring + (size_t)(kp / kb) * kAxmFragLanes * sizeof(uint4) + sizeof(float4) * std::max(k_max, 1);
        if ((int)smem > axm_smem_limit()) throw Fail{PD_ERR_UNSUPPORTED};
        auto kern = bf16 ? k_axpy_mma<false> : k_axpy_mma<true>;
        if (pdl)
            launch_pdl(kern, dim3(n_blocks), dim3(32 * (kAxtWarps + 1)), smem, s, descs, blocks, B, (int)ring,
                       tma_err);
        else
            kern<<<n_blocks, 32 * (kAxtWarps + 1), smem, s>>>(descs, blocks, B, (int)ring, tma_err);
    } else if (tma_err) {
        // tiled matrices: the bulk-copy streaming kernel
        const size_t ring = axt_ring_bytes<T>(w_max);
        const size_t smem = ring + sizeof(float4) * std::max(k_max, 1);
        if ((int)smem > axt_smem_limit<T>()) throw Fail{PD_ERR_UNSUPPORTED};
        if (pdl)
            launch_pdl(k_axpy_tma<T, false>, dim3(n_blocks), dim3(32 * (kAxtWarps + 1)), smem, s, descs, blocks, B,
                       (const AxBases*)nullptr, (int)ring, tma_err);
        else
            k_axpy_tma<T, false><<<n_blocks, 32 * (kAxtWarps + 1), smem, s>>>(descs, blocks, B, nullptr, (int)ring,
                                                                              tma_err);
    } else {
        k_axpy_form<T, false><<<n_blocks, 32 * kAxWarps, sizeof(float4) * std::max(k_max, 1), s>>>(descs, blocks, B,
                                                                                                 nullptr);
    }
    PDG_CHECK_LAUNCH();
}

template <class T>
void launch_rowdot(const RowPlan& P, const AxBases& B, cudaStream_t s, int* tma_err = nullptr) {
    if (P.n_blocks <= 0) return;
    if (P.mma && tma_err) {
        k_rowdot_mma<<<P.n_blocks, 32 * (kRowtWarps + 1), rowm_smem_bytes(P.xcap), s>>>(P.descs.p, P.n_desc, P.blk_u.p,
                                                                                     B, P.xcap, tma_err);
    } else if (P.tma && tma_err) {
        const size_t smem = (size_t)kRowtStages * kRowtStageBytes + sizeof(float) * 3 * (size_t)P.xcap;
        k_rowdot_tma<T, false><<<P.n_blocks, 32 * (kRowtWarps + 1), smem, s>>>(P.descs.p, P.n_desc, P.blk_u.p, B,
                                                                              nullptr, P.xcap, tma_err);
    } else {
        k_rowdot<T><<<P.n_blocks, 32 * kRowWarps, sizeof(float) * 3 * (size_t)P.xcap, s>>>(P.descs.p, P.n_desc,
                                                                                             P.blk_u.p, B, P.xcap);
    }
    PDG_CHECK_LAUNCH();
}

struct DDBufs {
    float4 *tc, *cB, *part, *tc2, *cT, *xg2, *xgB, *pm, *jx1, *jx2;
};

// One subspace solve: x (free vertices of xout) = K_ff^-1 b.
// The same solve as one fused streaming launch (every product, both levels).
void dd_solve_stream(pd_mesh* m, const float4* b, float4* xout, const DDBufs& w, cudaStream_t s) {
    FusedArgs F{};
    F.b = b;
    F.x = xout;
    F.tc = w.tc;
    F.tc2 = w.tc2;
    F.gat_ptr = m->d_gat_ptr.p;
    F.gat = m->d_gat.p;
    F.gat2_ptr = m->d_gat2_ptr.p;
    F.gat2 = m->d_gat2.p;
    F.bidx = m->d_bidx.p;
    F.bidx2 = m->d_bidx2.p;
    F.cB = w.cB;
    F.cT = w.cT;
    F.xg2 = w.xg2;
    F.xgB = w.xgB;
    F.invB_ptr = m->d_invB_ptr.p;
    F.invB = m->d_invB.p;
    F.inv2_ptr = m->d_inv2_ptr.p;
    F.inv2 = m->d_inv2.p;
    F.cb0 = m->d_cb0.p;
    F.ct0 = m->d_ct0.p;
    F.n_cb0 = m->n_cb0;
    F.n_ct0 = m->n_ct0;
    F.cnt_cb = m->st_solve.cnt_cb.p;
    F.cnt_ct = m->st_solve.cnt_ct.p;
    F.err = m->d_err.p;
    F.n_int = m->n_int;
    F.T0 = m->n_B - m->n_top;
    phase_begin(m, PH_SOLVE, s);
    launch_stream_solve(m->st_solve, F, s);
    phase_end(m, s);
}

template <class T>
void dd_solve_impl(pd_mesh* m, const T* pool, const float4* b, float4* xout, const DDBufs& w, cudaStream_t s) {
    // the interior part t = K_ii^-1 b_i runs on a side stream beside the
    // interface solve and is joined before the back-substitution
    const bool fork1 = m->ax_blocks_int > 0 || m->ax_blocks_m1 > 0;
    if (fork1) {
        PDG_CUDA(cudaEventRecord(m->ev_fork[0], s));
        PDG_CUDA(cudaStreamWaitEvent(m->side[0], m->ev_fork[0], 0));
        if (m->modal) {
            // t = (Phi Lambda^-1)(Phi^T b_i): the truncated interior response
            phase_begin(m, PH_MODAL, m->side[0]);
            launch_ax<T>(m->d_ax_desc_m1.p, m->d_ax_blk_m1.p, m->ax_blocks_m1, m->ax_kmax_m1,
                         AxBases{pool, b, nullptr, nullptr, w.pm}, m->side[0]);
            launch_ax<T>(m->d_ax_desc_m2.p, m->d_ax_blk_m2.p, m->ax_blocks_m2, m->ax_kmax_m2,
                         AxBases{pool, w.pm, nullptr, nullptr, w.tc}, m->side[0]);
            phase_end(m, m->side[0]);
        } else {
            // In two launches when it has more than three blocks per SM: one launch of all its
            // tiles fills every SM with interior blocks, and the interface chain's blocks wait
            // for slots (measured on the 390K shell: 800 tiles in two launches 2.126 ms/frame,
            // one 2.197, three 2.236)
            const int nb = m->ax_blocks_int, parts = nb > 3 * m->sms ? 2 : 1, per = (nb + parts - 1) / parts;
            for (int b0 = 0; b0 < nb; b0 += per) {
                phase_begin(m, PH_INTERIOR, m->side[0]);   // (timed per launch)
                launch_ax<T>(m->d_ax_desc_int.p, m->d_ax_blk_int.p + b0, std::min(per, nb - b0), m->ax_kmax_int,
                             AxBases{pool, b, nullptr, nullptr, w.tc}, m->side[0], m->ax_tiled ? m->d_err.p : nullptr,
                             m->ax_wmax_int, false, m->ax_tf32);
                phase_end(m, m->side[0]);
            }
        }
        PDG_CUDA(cudaEventRecord(m->ev_join[0], m->side[0]));
    }
    if (m->ax_blocks_cond > 0) {
        phase_begin(m, PH_CONDENSE, s);
        launch_ax<T>(m->d_ax_desc_cond.p, m->d_ax_blk_cond.p, m->ax_blocks_cond, m->ax_kmax_cond,
                     AxBases{pool, b, nullptr, nullptr, w.tc}, s, m->ax_tiled ? m->d_err.p : nullptr, m->ax_wmax_cond,
                     true, m->ax_tf32);
        phase_end(m, s);
    }
    if (m->n_B > 0) {
        phase_begin(m, PH_GATHER, s);
        launch_pdl(k_gather, dim3(nblk(m->n_B, 256)), dim3(256), 0, s, m->n_B, m->d_gat_ptr.p, m->d_gat.p,
                   b + m->n_int, w.tc, w.cB);
        PDG_CHECK_LAUNCH();
        phase_end(m, s);
        const float4* cin = w.cB;
        float4* xcs = xout + m->n_int;
        const int T0 = m->n_B - m->n_top;
        bool fork2 = false;
        if (m->two_level) {
            fork2 = m->rows_int2.n_blocks > 0;
            if (fork2) {
                PDG_CUDA(cudaEventRecord(m->ev_fork[1], s));
                PDG_CUDA(cudaStreamWaitEvent(m->side[1], m->ev_fork[1], 0));
                phase_begin(m, PH_INTERIOR2, m->side[1]);
                launch_rowdot<T>(m->rows_int2, AxBases{pool, w.cB, nullptr, nullptr, w.tc2}, m->side[1], m->d_err.p);
                phase_end(m, m->side[1]);
                PDG_CUDA(cudaEventRecord(m->ev_join[1], m->side[1]));
            }
            phase_begin(m, PH_CONDENSE2, s);
            launch_rowdot<T>(m->rows_cond2, AxBases{pool, w.cB, nullptr, nullptr, w.tc2}, s, m->d_err.p);
            phase_end(m, s);
            phase_begin(m, PH_GATHER2, s);
            launch_pdl(k_gather, dim3(nblk(m->n_top, 256)), dim3(256), 0, s, m->n_top, m->d_gat2_ptr.p, m->d_gat2.p,
                       w.cB + T0, w.tc2, w.cT);
            PDG_CHECK_LAUNCH();
            phase_end(m, s);
            cin = w.cT;
            xcs = xout + m->n_int + T0;
        }
        if (m->rows_coarse.n_blocks > 0) {
            // BF16 on the tensor cores: whole block-rows, written straight to x
            phase_begin(m, PH_COARSE, s);
            launch_rowdot<T>(m->rows_coarse, AxBases{pool, cin, nullptr, nullptr, xcs}, s, m->d_err.p);
            phase_end(m, s);
        } else {
            phase_begin(m, PH_COARSE, s);
            launch_coarse<T>(m, pool, cin, w.part, s);
            phase_end(m, s);
            phase_begin(m, PH_REDUCE, s);
            launch_pdl(k_reduce, dim3(nblk(m->cs_n, 256)), dim3(256), 0, s, m->cs_n, m->coarse_nchunks, w.part,
                       xcs);
            PDG_CHECK_LAUNCH();
            phase_end(m, s);
        }
        if (m->two_level) {
            if (fork2) PDG_CUDA(cudaStreamWaitEvent(s, m->ev_join[1], 0));
            phase_begin(m, PH_BACKSUB2, s);
            launch_rowdot<T>(m->rows_back2, AxBases{pool, xout + m->n_int + T0, m->d_bidx2.p, w.tc2, xout + m->n_int},
                             s, m->d_err.p);
            phase_end(m, s);
        }
    }
    if (fork1) PDG_CUDA(cudaStreamWaitEvent(s, m->ev_join[0], 0));
    if (m->ax_blocks_back > 0) {
        phase_begin(m, PH_BACKSUB, s);
        launch_ax<T>(m->d_ax_desc_back.p, m->d_ax_blk_back.p, m->ax_blocks_back, m->ax_kmax_back,
                     AxBases{pool, xout + m->n_int, m->d_bidx.p, w.tc, xout}, s, m->ax_tiled ? m->d_err.p : nullptr,
                     m->ax_wmax_back, true, m->ax_tf32);
        phase_end(m, s);
    }
    const int S = (int)m->jacobi_omega.size();
    if (S > 0 && m->n_free > 0) {
        // full-space Chebyshev-weighted Jacobi sweeps; iterate k+1 goes to buffer
        // (k+1) mod 3 of {xout, jx1, jx2}, the last one is copied back to xout
        float4* buf[3] = {xout, w.jx1, w.jx2};
        phase_begin(m, PH_JACOBI, s);
        for (int k = 1; k <= S; ++k) {
            const float4* cur = buf[(k - 1) % 3];
            const float4* prev = buf[(k >= 2 ? k - 2 : 0) % 3];
            k_cheb_jacobi<<<nblk(m->n_free, 256), 256, 0, s>>>(m->n_free, m->d_K_ptr.p, m->d_K_col.p, m->d_K_val.p,
                                                              m->d_Dinv.p, b, cur, prev, m->jacobi_omega[k - 1],
                                                              buf[k % 3]);
            PDG_CHECK_LAUNCH();
        }
        if (S % 3 != 0)
            PDG_CUDA(cudaMemcpyAsync(xout, buf[S % 3], sizeof(float4) * (size_t)m->n_free, cudaMemcpyDeviceToDevice,
                                     s));
        phase_end(m, s);
    }
}

}  // namespace

void launch_dd_solve_scratch(pd_mesh* m, const float4* b, float4* xout, float4* tc, float4* cB, float4* part,
                             float4* tc2, float4* cT, float4* xg2, float4* xgB, float4* pm, float4* jx1, float4* jx2,
                             cudaStream_t s) {
    const DDBufs w{tc, cB, part, tc2, cT, xg2, xgB, pm, jx1, jx2};
    if (m->use_stream) {
        dd_solve_stream(m, b, xout, w, s);
    } else if (m->prec == PD_PREC_BF16) dd_solve_impl<__nv_bfloat16>(m, m->d_mat16.p, b, xout, w, s);
    else dd_solve_impl<float>(m, m->d_mat32.p, b, xout, w, s);
}

// Serving batches: every resident request's tiled products in one launch of
// the bulk-copy kernel (each block reads its request's arrays from `bases`).
void launch_axpy_b(const AxDesc* descs, const AxBlock* blocks, const AxBases* bases, int n_blocks, int k_max,
                   int w_max, int* err, cudaStream_t s) {
    if (n_blocks <= 0) return;
    const size_t ring = axt_ring_bytes<float>(w_max);
    const size_t smem = ring + sizeof(float4) * std::max(k_max, 1);
    if ((int)smem > axt_smem_limit<float>()) throw Fail{PD_ERR_UNSUPPORTED};
    k_axpy_tma<float, true><<<n_blocks, 32 * (kAxtWarps + 1), smem, s>>>(descs, blocks, AxBases{}, bases, (int)ring,
                                                                          err);
    PDG_CHECK_LAUNCH();
}

int ax_outputs_per_block(int prec) { return 32 * kAxM * (prec == PD_PREC_BF16 ? 8 : 4); }

// Outputs of one tile of the tiled (bulk-copy) layout, one CTA each: 128 in
// FP32; the BF16 tiles of the tensor cores keep 128 outputs too, so that a
// launch has as many CTAs streaming (each with half the bytes), not half as
// many.
#ifndef PDG_AXM_CW
#define PDG_AXM_CW 128
#endif
int ax_tile_outputs(int prec) { return prec == PD_PREC_BF16 ? PDG_AXM_CW : 32 * 4; }

void test_set_copy_extra(int bytes, cudaStream_t s) {
    PDG_CUDA(cudaMemcpyToSymbolAsync(g_test_copy_extra, &bytes, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    PDG_CUDA(cudaStreamSynchronize(s));
}

// raise the dynamic shared-memory limit of the bulk-copy kernel (outside any capture)
void ax_prepare_tma(int prec) {
    if (prec == PD_PREC_BF16 || prec == PD_PREC_TF32) (void)axm_smem_limit();   // the tensor-core tile kernels
    if (prec != PD_PREC_BF16) (void)axt_smem_limit<float>();
}

// Returns false when the largest interface vector does not fit in shared memory.
bool configure_coarse_b(int max_cols) {
    const size_t smem = sizeof(float) * 3 * (size_t)max_cols;
    return smem <= (size_t)allow_max_dynamic_smem(k_coarse_b);
}

void launch_coarse_b(const CoarseDescB* cd, int n_desc, int64_t U, int max_cols, int blocks, cudaStream_t s) {
    if (blocks <= 0 || U <= 0) return;
    k_coarse_b<<<blocks, 32 * kCoarseWarps, sizeof(float) * 3 * (size_t)max_cols, s>>>(cd, n_desc, U, max_cols);
    PDG_CHECK_LAUNCH();
}

int dd_max_sub_cols() { return kMaxSubCols; }

// Number of blocks of the balanced coarse kernel (one per SM), or 0 when the
// interface vector does not fit in shared memory and the chunked kernel is used.
int dd_configure_coarse(int ld_S) {
    const size_t smem = sizeof(float) * 3 * (size_t)ld_S;
    int dev = 0, sms = 0;
    PDG_CUDA(cudaGetDevice(&dev));
    PDG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int optin = std::min(allow_max_dynamic_smem(k_coarse_bal<float>),
                               allow_max_dynamic_smem(k_coarse_bal<__nv_bfloat16>));
    if (smem > (size_t)optin || sms <= 0) return 0;
    const int bps = (smem * kCoarseBps <= (size_t)optin) ? kCoarseBps : 1;
    return sms * bps;
}
int dd_coarse_chunk() { return kCoarseChunk; }

int rowdot_rows_per_unit(int prec) { return prec == PD_PREC_BF16 ? RowRows<__nv_bfloat16>::R : RowRows<float>::R; }

// Unit numbering and block cuts of a row-form launch: block b gets the units
// whose cumulative cost (matrix columns streamed plus a fixed per-unit cost)
// starts in [W b / C, W (b+1) / C), C = one block per SM.
bool rowdot_row_fits_stage(int ld, int elem_bytes) { return (int64_t)ld * elem_bytes <= kRowtStageBytes; }

bool rowdot_mma_fits(int xcap) {
    static const int optin_m = allow_max_dynamic_smem(k_rowdot_mma);
    return rowm_smem_bytes(xcap) <= (size_t)optin_m;
}

void build_row_plan(RowPlan& P, std::vector<RowDesc> descs, int prec, cudaStream_t s, bool mma) {
    const int RU = mma ? 16 : rowdot_rows_per_unit(prec);
    int64_t u = 0;
    int xcap = 8;
    double W = 0.0;
    for (auto& d : descs) {
        d.u0 = u;
        const int64_t nu = (d.rows + RU - 1) / RU;
        u += nu;
        xcap = std::max(xcap, d.ld);
        W += (double)nu * (RU * (double)d.ld + 64.0);
    }
    P.n_desc = (int)descs.size();
    P.xcap = xcap;
    P.n_blocks = 0;
    if (u == 0) return;
    int dev = 0, sms = 0;
    PDG_CUDA(cudaGetDevice(&dev));
    PDG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int bps = kRowBps;
    if (mma && rowdot_mma_fits(xcap)) {
        // as many blocks as are resident at once (its shared memory grows with x)
        int occ = 0;
        PDG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rowdot_mma, 32 * (kRowtWarps + 1),
                                                               rowm_smem_bytes(xcap)));
        bps = std::max(1, std::min(bps, occ));
    }
    const int C = std::max(1, sms) * bps;
    std::vector<int64_t> cut(C + 1, u);
    cut[0] = 0;
    double acc = 0.0;
    int b = 1;
    for (const auto& d : descs) {
        const int64_t nu = (d.rows + RU - 1) / RU;
        const double cu = RU * (double)d.ld + 64.0;
        for (int64_t k = 0; k < nu; ++k) {
            while (b < C && acc >= W * b / C) cut[b++] = d.u0 + k;
            acc += cu;
        }
    }
    const size_t smem = sizeof(float) * 3 * (size_t)xcap;
    const int optin = std::min(allow_max_dynamic_smem(k_rowdot<float>), allow_max_dynamic_smem(k_rowdot<__nv_bfloat16>));
    if (!mma && smem > (size_t)optin) {
        set_error("row-form product: the x vector does not fit in shared memory");
        throw Fail{PD_ERR_UNSUPPORTED};
    }
    // bulk-copy streaming when a whole row fits in one stage (16-byte aligned rows: ld % 8 == 0)
    const int es = (prec == PD_PREC_BF16) ? 2 : 4;
    const int optin_t = (prec == PD_PREC_BF16) ? allow_max_dynamic_smem(k_rowdot_tma<__nv_bfloat16, false>)
                                               : std::min(allow_max_dynamic_smem(k_rowdot_tma<float, false>),
                                                          allow_max_dynamic_smem(k_rowdot_tma<float, true>));
    P.tma = (size_t)kRowtStages * kRowtStageBytes + smem <= (size_t)optin_t;
    for (const auto& d : descs) P.tma = P.tma && d.ld * es <= kRowtStageBytes && d.ld % 8 == 0 && d.a_off % 8 == 0;
    P.mma = false;
    if (mma) {
        // BF16 fragment layout: whole 16-row block-rows, columns padded to 16
        if (!rowdot_mma_fits(xcap)) {
            set_error("row-form tensor-core product: the x vector does not fit in shared memory");
            throw Fail{PD_ERR_UNSUPPORTED};
        }
        for (const auto& d : descs)
            if (d.ld % 16 != 0 || d.a_off % 8 != 0) {
                set_error("row-form tensor-core product: block not in the fragment layout");
                throw Fail{PD_ERR_UNSUPPORTED};
            }
        P.mma = true;
    }
    upload(P.descs, descs, s);
    upload(P.blk_u, cut, s);
    PDG_CUDA(cudaStreamSynchronize(s));
    P.host = std::move(descs);
    P.n_blocks = C;
}

// Serving: one row-form launch over the descriptors of several requests (each
// descriptor's slot selects its request's arrays); FP32 rows streamed by bulk
// copies, so every row must fit one stage (checked when the plan is built).
void launch_rowdot_b(const RowPlan& P, const AxBases* multi, int* err, cudaStream_t s) {
    if (P.n_blocks <= 0) return;
    if (!P.tma) throw Fail{PD_ERR_UNSUPPORTED};
    const size_t smem = (size_t)kRowtStages * kRowtStageBytes + sizeof(float) * 3 * (size_t)P.xcap;
    k_rowdot_tma<float, true><<<P.n_blocks, 32 * (kRowtWarps + 1), smem, s>>>(P.descs.p, P.n_desc, P.blk_u.p,
                                                                             AxBases{}, multi, P.xcap, err);
    PDG_CHECK_LAUNCH();
}

void launch_dd_solve(pd_mesh* m, const float4* b, float4* xout, cudaStream_t s, bool /*timed*/) {
    launch_dd_solve_scratch(m, b, xout, m->d_tc.p, m->d_cB.p, m->d_part.p, m->d_tc2.p, m->d_cT.p, m->d_xg2.p,
                            m->d_xgB.p, m->d_pm.p, m->d_jx1.p, m->d_jx2.p, s);
}

void launch_residual(const pd_mesh* m, const float4* b, const float4* x, float4* r, cudaStream_t s) {
    if (m->n_free <= 0) return;
    k_residual<<<nblk(m->n_free, 256), 256, 0, s>>>(m->n_free, m->d_K_ptr.p, m->d_K_col.p, m->d_K_val.p, b, x, r);
    PDG_CHECK_LAUNCH();
}

void launch_axpy_free(const pd_mesh* m, const float4* dx, float4* x, cudaStream_t s) {
    if (m->n_free <= 0) return;
    k_axpy<<<nblk(m->n_free, 256), 256, 0, s>>>(m->n_free, dx, x);
    PDG_CHECK_LAUNCH();
}

}  // namespace pdg
