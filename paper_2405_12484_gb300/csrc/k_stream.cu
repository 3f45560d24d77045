// Streaming row-form products of the subspace solve (Sec. 7.2) on sm_103a:
// out[r] = add[r] + A[r, 0:cols] . x for every row of a list of dense blocks
// (RowDesc), x being three right-hand sides (K = K_s (x) I_3).
//
// The matrices are read once per solve and are far larger than L2, so the
// launch is bound by HBM.  Plain per-warp loads leave too few bytes in flight
// (long-scoreboard stalls); here one producer thread per CTA streams
// contiguous row tiles into a shared-memory ring with bulk asynchronous copies
// (cp.async.bulk, completion counted in bytes on an mbarrier), so up to
// kStages x kStageBytes per SM are in flight independently of the compute
// warps.  Eight consumer warps take (row, column chunk) units of a tile, dot
// them with x staged in shared memory as three float planes, and combine the
// lanes with a fixed shuffle tree; the chunk sums of a row are added in chunk
// order.  Results are bitwise reproducible and do not depend on the tile
// schedule.  One CTA per SM; the host cuts the tile list into equal byte
// ranges, one per CTA.
//
// Every wait is bounded: a wait that runs out sets ERR_TIMEOUT in the mesh's
// error word, marks the CTA aborted (no further copies are issued, consumers
// stop waiting), and the producer waits, again bounded, for its copies in
// flight before the CTA exits.
#include <algorithm>

#include "pd_internal.h"

namespace pdg {

namespace {

constexpr int kStreamWarps = 8;                           // consumer warps
constexpr int kStreamThreads = 32 * (kStreamWarps + 1);   // + one producer warp
constexpr int kStages = 4;
constexpr int kStageBytes = 32 * 1024;
constexpr int kMaxTileRows = 256;
constexpr int kMaxUnits = 512;                            // (row, chunk) units of one tile
constexpr int kChunkLoads = 4;                            // 16-byte loads per lane per unit
constexpr long long kWaitLimit = 1LL << 24;               // try_wait polls before giving up

template <class T>
struct SVec;
template <>
struct SVec<float> {
    static constexpr int N = 4;
};
template <>
struct SVec<__nv_bfloat16> {
    static constexpr int N = 8;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; false when the limit ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (long long k = 0; k < kWaitLimit; ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void consumer_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kStreamWarps) : "memory");
}

__device__ __forceinline__ void vec_from_smem(const float* p, float (&v)[4]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}

__device__ __forceinline__ void vec_from_smem(const __nv_bfloat16* p, float (&v)[8]) {
    const uint4 a = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&a);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 f = __bfloat1622float2(h[k]);
        v[2 * k] = f.x;
        v[2 * k + 1] = f.y;
    }
}

template <class T>
__global__ void __launch_bounds__(kStreamThreads, 1)
    k_stream_rows(const RowDesc* __restrict__ descs, const StreamTile* __restrict__ tiles,
                  const int32_t* __restrict__ cta_tiles, AxBases B, int xcap, int* __restrict__ err) {
    constexpr int VN = SVec<T>::N;
    constexpr int CW = 32 * VN * kChunkLoads;   // columns of one unit
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char* ring = sm;
    float* x0 = reinterpret_cast<float*>(sm + (size_t)kStages * kStageBytes);
    float* x1 = x0 + xcap;
    float* x2 = x1 + xcap;
    float* part = x2 + xcap;                                            // [kMaxUnits][3]
    uint64_t* full = reinterpret_cast<uint64_t*>(part + 3 * kMaxUnits);  // [kStages]
    uint64_t* empty = full + kStages;                                   // [kStages]
    __shared__ int abort_flag;

    const int t0 = cta_tiles[blockIdx.x], t1 = cta_tiles[blockIdx.x + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int k = 0; k < kStages; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kStreamWarps);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (t1 <= t0) return;
    const T* pool = reinterpret_cast<const T*>(B.pool);

    if (warp == kStreamWarps) {
        // ---- producer: one thread issues the bulk copies of this CTA's tiles
        if (lane != 0) return;
        int issued = 0;
        for (int i = 0; i < t1 - t0; ++i) {
            if (*reinterpret_cast<volatile int*>(&abort_flag)) break;
            const int slot = i % kStages;
            if (i >= kStages && !mbar_wait(&empty[slot], (uint32_t)((i / kStages) - 1) & 1u)) {
                atomicOr(err, ERR_TIMEOUT);
                atomicExch(&abort_flag, 1);
                break;
            }
            const StreamTile tl = tiles[t0 + i];
            const RowDesc D = descs[tl.desc];
            const uint32_t bytes = (uint32_t)tl.nr * (uint32_t)D.ld * (uint32_t)sizeof(T);
            mbar_arrive_expect_tx(&full[slot], bytes);
            bulk_g2s(ring + (size_t)slot * kStageBytes, pool + D.a_off + (int64_t)tl.r0 * D.ld, bytes, &full[slot]);
            issued = i + 1;
        }
        // before exit: every issued copy has landed (normally already consumed)
        for (int i = (issued > kStages ? issued - kStages : 0); i < issued; ++i)
            if (!mbar_wait(&full[i % kStages], (uint32_t)(i / kStages) & 1u)) atomicOr(err, ERR_TIMEOUT);
        return;
    }

    // ---- consumers (warps 0 .. kStreamWarps-1)
    int cur_desc = -1;
    for (int i = 0; i < t1 - t0; ++i) {
        const StreamTile tl = tiles[t0 + i];
        const RowDesc D = descs[tl.desc];
        if (tl.desc != cur_desc) {
            // the previous tile ended with a consumer barrier: nobody reads the old x
            for (int k = threadIdx.x; k < D.ld; k += 32 * kStreamWarps) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (k < D.cols) v = (D.xidx_off >= 0) ? B.x[B.bidx[D.xidx_off + k]] : B.x[D.x_off + k];
                x0[k] = v.x;
                x1[k] = v.y;
                x2[k] = v.z;
            }
            cur_desc = tl.desc;
            consumer_sync();
        }
        const int slot = i % kStages;
        if (!*reinterpret_cast<volatile int*>(&abort_flag) && !mbar_wait(&full[slot], (uint32_t)(i / kStages) & 1u)) {
            atomicOr(err, ERR_TIMEOUT);
            atomicExch(&abort_flag, 1);
        }
        const T* A = reinterpret_cast<const T*>(ring + (size_t)slot * kStageBytes);
        const int units = tl.nr * tl.q;
        for (int u = warp; u < units; u += kStreamWarps) {
            const int r = u / tl.q, ch = u - r * tl.q;
            const T* row = A + (int64_t)r * D.ld;
            const int cb = ch * CW, ce = min(D.ld, cb + CW);
            float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
            for (int l = 0; l < kChunkLoads; ++l) {
                const int c = cb + (l * 32 + lane) * VN;
                if (c < ce) {
                    float v[VN];
                    vec_from_smem(row + c, v);
#pragma unroll
                    for (int j = 0; j < VN; j += 4) {
                        const float4 p0 = *reinterpret_cast<const float4*>(x0 + c + j);
                        const float4 p1 = *reinterpret_cast<const float4*>(x1 + c + j);
                        const float4 p2 = *reinterpret_cast<const float4*>(x2 + c + j);
                        a0 = fmaf(v[j], p0.x, a0); a0 = fmaf(v[j + 1], p0.y, a0);
                        a0 = fmaf(v[j + 2], p0.z, a0); a0 = fmaf(v[j + 3], p0.w, a0);
                        a1 = fmaf(v[j], p1.x, a1); a1 = fmaf(v[j + 1], p1.y, a1);
                        a1 = fmaf(v[j + 2], p1.z, a1); a1 = fmaf(v[j + 3], p1.w, a1);
                        a2 = fmaf(v[j], p2.x, a2); a2 = fmaf(v[j + 1], p2.y, a2);
                        a2 = fmaf(v[j + 2], p2.z, a2); a2 = fmaf(v[j + 3], p2.w, a2);
                    }
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                a0 += __shfl_xor_sync(0xffffffffu, a0, off);
                a1 += __shfl_xor_sync(0xffffffffu, a1, off);
                a2 += __shfl_xor_sync(0xffffffffu, a2, off);
            }
            if (lane == 0) {
                part[3 * u] = a0;
                part[3 * u + 1] = a1;
                part[3 * u + 2] = a2;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);   // this warp is done with the tile's bytes
        consumer_sync();                             // every unit's partial sum is in part[]
        for (int r = threadIdx.x; r < tl.nr; r += 32 * kStreamWarps) {
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
            for (int ch = 0; ch < tl.q; ++ch) {
                s0 += part[3 * (r * tl.q + ch)];
                s1 += part[3 * (r * tl.q + ch) + 1];
                s2 += part[3 * (r * tl.q + ch) + 2];
            }
            const int gr = tl.r0 + r;
            const float4 ad = (D.add_off >= 0) ? B.add[D.add_off + gr] : make_float4(0.f, 0.f, 0.f, 0.f);
            B.out[D.out_off + gr] = make_float4(ad.x + s0, ad.y + s1, ad.z + s2, 0.f);
        }
        consumer_sync();                             // part[] free for the next tile
    }
}

size_t stream_smem_bytes(int xcap) {
    return (size_t)kStages * kStageBytes + sizeof(float) * (3 * (size_t)xcap + 3 * (size_t)kMaxUnits) +
           sizeof(uint64_t) * 2 * kStages;
}

}  // namespace

// Tiles of whole rows (at most kStageBytes, kMaxTileRows rows and kMaxUnits
// units each) for every descriptor in order, and the cut of the tile list into
// one contiguous range per CTA with about the same number of bytes.  Returns
// false (plan left empty) when a row does not fit in one stage or x does not
// fit in shared memory.
bool build_stream_plan(StreamPlan& P, std::vector<RowDesc> descs, int prec, cudaStream_t s) {
    P.n_ctas = 0;
    P.host.clear();
    const int es = (prec == PD_PREC_BF16) ? 2 : 4;
    const int VN = (prec == PD_PREC_BF16) ? 8 : 4;
    const int CW = 32 * VN * kChunkLoads;
    int xcap = 8;
    std::vector<StreamTile> tiles;
    std::vector<int64_t> tbytes;
    for (int d = 0; d < (int)descs.size(); ++d) {
        const RowDesc& D = descs[d];
        if (D.rows <= 0) continue;
        const int64_t row_bytes = (int64_t)D.ld * es;
        if (row_bytes > kStageBytes || D.ld % 8 != 0 || D.a_off % 8 != 0) return false;
        xcap = std::max(xcap, D.ld);
        const int q = (D.ld + CW - 1) / CW;
        int nr = (int)std::min<int64_t>(kStageBytes / row_bytes, kMaxTileRows);
        nr = std::max(1, std::min(nr, kMaxUnits / q));
        for (int r0 = 0; r0 < D.rows; r0 += nr) {
            const int n = std::min(nr, D.rows - r0);
            tiles.push_back(StreamTile{d, r0, n, q});
            tbytes.push_back((int64_t)n * row_bytes + 1024);   // + a fixed per-tile cost
        }
    }
    int dev = 0, sms = 0;
    PDG_CUDA(cudaGetDevice(&dev));
    PDG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int lim = std::min(allow_max_dynamic_smem(k_stream_rows<float>),
                             allow_max_dynamic_smem(k_stream_rows<__nv_bfloat16>));
    const size_t smem = stream_smem_bytes(xcap);
    if (smem > (size_t)lim) return false;
    if (tiles.empty()) {
        P.xcap = xcap;
        return true;
    }
    const int C = std::max(1, sms);
    int64_t W = 0;
    for (auto b : tbytes) W += b;
    std::vector<int32_t> cut(C + 1, (int32_t)tiles.size());
    cut[0] = 0;
    int64_t acc = 0;
    int c = 1;
    for (int t = 0; t < (int)tiles.size(); ++t) {
        while (c < C && acc * C >= W * c) cut[c++] = t;
        acc += tbytes[t];
    }
    upload(P.descs, descs, s);
    upload(P.tiles, tiles, s);
    upload(P.cta_tiles, cut, s);
    PDG_CUDA(cudaStreamSynchronize(s));
    P.host = std::move(descs);
    P.xcap = xcap;
    P.n_ctas = C;
    P.smem = smem;
    return true;
}

void launch_stream_rows(const StreamPlan& P, int prec, const void* pool, const float4* x, const int* xidx,
                        const float4* add, float4* out, int* err, cudaStream_t s) {
    if (P.n_ctas <= 0) return;
    const AxBases B{pool, x, xidx, add, out};
    if (prec == PD_PREC_BF16)
        k_stream_rows<__nv_bfloat16><<<P.n_ctas, kStreamThreads, P.smem, s>>>(P.descs.p, P.tiles.p, P.cta_tiles.p, B,
                                                                              P.xcap, err);
    else
        k_stream_rows<float><<<P.n_ctas, kStreamThreads, P.smem, s>>>(P.descs.p, P.tiles.p, P.cta_tiles.p, B, P.xcap,
                                                                      err);
    PDG_CHECK_LAUNCH();
}

}  // namespace pdg
