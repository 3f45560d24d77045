// Streaming products of the subspace solve (Sec. 7.2) on sm_103a in the
// column ("axpy") form: out[o] = add[o] + sum_k A[k][o] x_k for o < n_out,
// the rows k of A contiguous in memory, x_k three right-hand sides
// (K = K_s (x) I_3).  Every product of the solve has this form with the
// factors the pool holds: K_ii^-1 (symmetric), Psi_d, Psi_d^T, and the same
// for the second level and the coarse inverse.
//
// The matrices are read once per solve and are far larger than L2: the
// launch is bound by HBM.  One producer thread per CTA streams whole-row
// tiles into a shared-memory ring with bulk asynchronous copies
// (cp.async.bulk, completion counted in bytes on an mbarrier), keeping
// kStages x kStageBytes per SM in flight whatever the compute warps do; a
// second warp loads the x slice of the next piece (gathered where the block
// says so) into a double buffer.  Sixteen consumer warps own (output slab,
// row group) pairs: a warp adds
// A[k][slab] * x_k for the rows k of its group, with x_k a shared-memory
// broadcast and the accumulators in registers (no cross-lane reductions).
// The row groups of a slab are combined in group order through shared memory.
//
// Work split: the rows of all blocks are cut into pieces, one contiguous
// byte range of about the same size per CTA (a block may span CTAs).  A block
// cut into several pieces writes per-piece partial sums; the CTA that
// finishes the block's last piece (an atomic counter, no waiting) adds them in
// piece order.  Results are bitwise reproducible for a given plan.
//
// Every wait is bounded: a wait that runs out sets ERR_TIMEOUT in the mesh's
// error word and marks the CTA aborted (no further copies are issued,
// consumers stop waiting); the producer waits, again bounded, for its copies
// in flight before it exits.
#include <algorithm>

#include "pd_internal.h"

namespace pdg {

namespace {

constexpr int kColWarps = 16;                            // consumer warps
constexpr int kColThreads = 32 * (kColWarps + 2);        // + copy producer and x loader warps
constexpr int kStages = 4;
constexpr int kStageBytes = 24 * 1024;
constexpr int kMaxGroups = 8;                            // row groups per slab
constexpr int kMaxPieceRows = 1024;                      // x slice of a piece in shared memory
constexpr long long kWaitLimit = 1LL << 24;              // try_wait polls before giving up

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
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kColWarps) : "memory");
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

// outputs of one warp's slab: M sub-slabs of 32 lanes x VN consecutive outputs
template <class T>
struct Slab {
    static constexpr int VN = SVec<T>::N;
    static constexpr int M = (VN == 4) ? 2 : 1;
    static constexpr int OUT = 32 * VN * M;
};

__host__ __device__ inline int col_rows_per_tile(int ld, int es) {
    const int r = kStageBytes / (ld * es);
    return r > 0 ? r : 1;
}

__host__ __device__ inline void col_layout(int n_out, int slab_out, int& S, int& G) {
    S = (n_out + slab_out - 1) / slab_out;
    if (S < 1) S = 1;
    G = kColWarps / S;
    if (G > kMaxGroups) G = kMaxGroups;
    if (G < 1) G = 1;
}

// largest (G - 1) * S over the slab counts S (the row-group partials kept in red[])
__host__ __device__ constexpr int red_slabs() {
    int best = 0;
    for (int S = 1; S <= kColWarps; ++S) {
        int G = kColWarps / S;
        if (G > kMaxGroups) G = kMaxGroups;
        if (G < 1) G = 1;
        if ((G - 1) * S > best) best = (G - 1) * S;
    }
    return best;
}

template <class T>
__global__ void __launch_bounds__(kColThreads, 1)
    k_stream_cols(const ColDesc* __restrict__ descs, const ColPiece* __restrict__ pieces,
                  const int32_t* __restrict__ cta_pieces, AxBases B, float4* __restrict__ part,
                  int* __restrict__ cnt, int* __restrict__ err) {
    constexpr int VN = Slab<T>::VN, M = Slab<T>::M, SO = Slab<T>::OUT;
    constexpr int ES = (int)sizeof(T);
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char* ring = sm;
    float4* xs = reinterpret_cast<float4*>(sm + (size_t)kStages * kStageBytes);    // [2][kMaxPieceRows]
    float* red = reinterpret_cast<float*>(xs + 2 * kMaxPieceRows);                  // [red_slabs()][SO][3]
    uint64_t* full = reinterpret_cast<uint64_t*>(red + (size_t)red_slabs() * SO * 3);
    uint64_t* empty = full + kStages;
    uint64_t* xfull = empty + kStages;   // [2]
    uint64_t* xempty = xfull + 2;        // [2]
    __shared__ int abort_flag, last_flag;

    const int p0 = cta_pieces[blockIdx.x], p1 = cta_pieces[blockIdx.x + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int k = 0; k < kStages; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kColWarps);
        }
        for (int k = 0; k < 2; ++k) {
            mbar_init(&xfull[k], 1);
            mbar_init(&xempty[k], kColWarps);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (p1 <= p0) return;
    const T* pool = reinterpret_cast<const T*>(B.pool);

    if (warp == kColWarps) {
        // ---- producer: one thread issues the bulk copies of every tile of this CTA
        if (lane != 0) return;
        int i = 0, issued = 0;
        bool stop = false;
        for (int p = p0; p < p1 && !stop; ++p) {
            const ColPiece pc = pieces[p];
            const ColDesc D = descs[pc.desc];
            const int rpt = col_rows_per_tile(D.ld, ES);
            for (int k = pc.k0; k < pc.k1; k += rpt, ++i) {
                if (*reinterpret_cast<volatile int*>(&abort_flag)) {
                    stop = true;
                    break;
                }
                const int slot = i % kStages;
                if (i >= kStages && !mbar_wait(&empty[slot], (uint32_t)((i / kStages) - 1) & 1u)) {
                    atomicOr(err, ERR_TIMEOUT);
                    atomicExch(&abort_flag, 1);
                    stop = true;
                    break;
                }
                const int nr = min(rpt, pc.k1 - k);
                const uint32_t bytes = (uint32_t)nr * (uint32_t)D.ld * (uint32_t)ES;
                mbar_arrive_expect_tx(&full[slot], bytes);
                bulk_g2s(ring + (size_t)slot * kStageBytes, pool + D.a_off + (int64_t)k * D.ld, bytes, &full[slot]);
                issued = i + 1;
            }
        }
        for (int j = (issued > kStages ? issued - kStages : 0); j < issued; ++j)
            if (!mbar_wait(&full[j % kStages], (uint32_t)(j / kStages) & 1u)) atomicOr(err, ERR_TIMEOUT);
        return;
    }
    if (warp == kColWarps + 1) {
        // ---- x loader: the x slice of every piece (gathered where the block says
        // so) into a double buffer, ahead of the consumers
        for (int p = p0; p < p1; ++p) {
            const int pp = p - p0, buf = pp & 1;
            if (pp >= 2) {
                bool ok = true;
                if (lane == 0) ok = mbar_wait(&xempty[buf], (uint32_t)((pp / 2) - 1) & 1u);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) {
                    if (lane == 0) {
                        atomicOr(err, ERR_TIMEOUT);
                        atomicExch(&abort_flag, 1);
                    }
                    return;
                }
            }
            const ColPiece pc = pieces[p];
            const ColDesc D = descs[pc.desc];
            float4* xb = xs + buf * kMaxPieceRows;
            for (int k = lane; k < pc.k1 - pc.k0; k += 32) {
                const int kk = pc.k0 + k;
                xb[k] = (D.xidx_off >= 0) ? B.x[B.bidx[D.xidx_off + kk]] : B.x[D.x_off + kk];
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&xfull[buf]);   // release: the warp's writes above
        }
        return;
    }

    // ---- consumers
    const int tid = threadIdx.x;
    int i = 0;   // tile counter (same sequence as the producer's)
    for (int p = p0; p < p1; ++p) {
        const int pp = p - p0, buf = pp & 1;
        const ColPiece pc = pieces[p];
        const ColDesc D = descs[pc.desc];
        const int rpt = col_rows_per_tile(D.ld, ES);
        int S, G;
        col_layout(D.n_out, SO, S, G);
        if (!*reinterpret_cast<volatile int*>(&abort_flag) && !mbar_wait(&xfull[buf], (uint32_t)(pp / 2) & 1u)) {
            atomicOr(err, ERR_TIMEOUT);
            atomicExch(&abort_flag, 1);
        }
        const float4* xb = xs + buf * kMaxPieceRows;
        const bool active = warp < S * G;
        const int slab = warp % S, grp = warp / S;
        const int o_base = slab * SO + lane * VN;
        float acc[M][VN][3];
#pragma unroll
        for (int mm = 0; mm < M; ++mm)
#pragma unroll
            for (int j = 0; j < VN; ++j) acc[mm][j][0] = acc[mm][j][1] = acc[mm][j][2] = 0.f;
        bool valid[M];
#pragma unroll
        for (int mm = 0; mm < M; ++mm) valid[mm] = active && (o_base + mm * 32 * VN < D.n_out);
        for (int k = pc.k0; k < pc.k1; k += rpt, ++i) {
            const int slot = i % kStages;
            if (!*reinterpret_cast<volatile int*>(&abort_flag) &&
                !mbar_wait(&full[slot], (uint32_t)(i / kStages) & 1u)) {
                atomicOr(err, ERR_TIMEOUT);
                atomicExch(&abort_flag, 1);
            }
            const T* A = reinterpret_cast<const T*>(ring + (size_t)slot * kStageBytes);
            const int nr = min(rpt, pc.k1 - k);
            if (valid[0]) {
                // rows r of the tile with (k - k0 + r) = grp (mod G)
                int r = grp - ((k - pc.k0) % G);
                if (r < 0) r += G;
#pragma unroll 2
                for (; r < nr; r += G) {
                    const float4 xk = xb[k - pc.k0 + r];
                    const T* a = A + (int64_t)r * D.ld + o_base;
#pragma unroll
                    for (int mm = 0; mm < M; ++mm) {
                        if (!valid[mm]) continue;
                        float v[VN];
                        vec_from_smem(a + mm * 32 * VN, v);
#pragma unroll
                        for (int j = 0; j < VN; ++j) {
                            acc[mm][j][0] = fmaf(v[j], xk.x, acc[mm][j][0]);
                            acc[mm][j][1] = fmaf(v[j], xk.y, acc[mm][j][1]);
                            acc[mm][j][2] = fmaf(v[j], xk.z, acc[mm][j][2]);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&xempty[buf]);   // this warp no longer reads the x slice
        // combine the row groups of each slab in group order
        if (active && grp > 0) {
            float* rb = red + ((size_t)(grp - 1) * S + slab) * SO * 3;
#pragma unroll
            for (int mm = 0; mm < M; ++mm)
#pragma unroll
                for (int j = 0; j < VN; ++j) {
                    const int lo = mm * 32 * VN + lane * VN + j;
                    rb[3 * lo] = acc[mm][j][0];
                    rb[3 * lo + 1] = acc[mm][j][1];
                    rb[3 * lo + 2] = acc[mm][j][2];
                }
        }
        if (G > 1) consumer_sync();
        const bool single = D.n_pieces == 1;
        if (active && grp == 0) {
#pragma unroll
            for (int mm = 0; mm < M; ++mm)
#pragma unroll
                for (int j = 0; j < VN; ++j) {
                    const int lo = mm * 32 * VN + lane * VN + j;
                    const int o = slab * SO + lo;
                    if (o >= D.n_out) continue;
                    float s0 = acc[mm][j][0], s1 = acc[mm][j][1], s2 = acc[mm][j][2];
                    for (int g = 1; g < G; ++g) {
                        const float* rb = red + ((size_t)(g - 1) * S + slab) * SO * 3;
                        s0 += rb[3 * lo];
                        s1 += rb[3 * lo + 1];
                        s2 += rb[3 * lo + 2];
                    }
                    if (single) {
                        const float4 ad =
                            (D.add_off >= 0) ? B.add[D.add_off + o] : make_float4(0.f, 0.f, 0.f, 0.f);
                        B.out[D.out_off + o] = make_float4(ad.x + s0, ad.y + s1, ad.z + s2, 0.f);
                    } else {
                        part[D.part_off + (int64_t)pc.piece * D.n_out + o] = make_float4(s0, s1, s2, 0.f);
                    }
                }
        }
        if (!single) {
            // the CTA that completes the block's last piece adds the pieces in
            // order: one release (fence + counter) per CTA after a CTA barrier,
            // an acquire fence on the counter's result
            consumer_sync();
            if (tid == 0) {
                asm volatile("fence.acq_rel.gpu;" ::: "memory");
                const int prev = atomicAdd(&cnt[pc.desc], 1);
                asm volatile("fence.acq_rel.gpu;" ::: "memory");
                last_flag = (prev == D.n_pieces - 1);
            }
            consumer_sync();
            if (last_flag) {
                for (int o = tid; o < D.n_out; o += 32 * kColWarps) {
                    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
                    for (int q = 0; q < D.n_pieces; ++q) {
                        const float4 v = __ldcg(&part[D.part_off + (int64_t)q * D.n_out + o]);
                        s0 += v.x;
                        s1 += v.y;
                        s2 += v.z;
                    }
                    const float4 ad = (D.add_off >= 0) ? B.add[D.add_off + o] : make_float4(0.f, 0.f, 0.f, 0.f);
                    B.out[D.out_off + o] = make_float4(ad.x + s0, ad.y + s1, ad.z + s2, 0.f);
                }
                if (tid == 0) cnt[pc.desc] = 0;   // ready for the next launch
            }
        }
        if (G > 1 || !single) consumer_sync();   // red[] (and last_flag) free for the next piece
    }
}

template <class T>
size_t col_smem_bytes() {
    return (size_t)kStages * kStageBytes + sizeof(float4) * 2 * kMaxPieceRows +
           sizeof(float) * (size_t)red_slabs() * Slab<T>::OUT * 3 + sizeof(uint64_t) * (2 * kStages + 4);
}

}  // namespace

// Pieces of whole rows for every block in order, cut so that every CTA gets a
// contiguous range of about the same number of bytes (at most kMaxPieceRows
// rows per piece).  Returns false (plan left empty) when a row does not fit in
// one stage or a block has more outputs than the consumer warps cover.
bool build_stream_plan(StreamPlan& P, std::vector<ColDesc> descs, int prec, cudaStream_t s) {
    P.n_ctas = 0;
    P.host.clear();
    const int es = (prec == PD_PREC_BF16) ? 2 : 4;
    const int SO = (prec == PD_PREC_BF16) ? Slab<__nv_bfloat16>::OUT : Slab<float>::OUT;
    int dev = 0, sms = 0;
    PDG_CUDA(cudaGetDevice(&dev));
    PDG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int C = std::max(1, sms);
    int64_t W = 0;
    for (const auto& D : descs) {
        if ((int64_t)D.ld * es > kStageBytes || D.ld % 8 != 0 || D.a_off % 8 != 0) return false;
        if ((D.n_out + SO - 1) / SO > kColWarps) return false;
        W += (int64_t)D.K * D.ld * es + (int64_t)D.n_out * 64;
    }
    // walk the blocks, closing a CTA's range when its byte budget is reached
    std::vector<ColPiece> pcs;
    std::vector<int32_t> cut(1, 0);
    int64_t acc = 0;
    int c = 0;
    for (int d = 0; d < (int)descs.size(); ++d) {
        ColDesc& D = descs[d];
        const int64_t row_b = (int64_t)D.ld * es;
        int k = 0, piece = 0;
        acc += (int64_t)D.n_out * 64;
        do {
            // rows that fit in what is left of this CTA's budget
            const int64_t budget = W * (c + 1) / C - acc;
            int take = (int)std::min<int64_t>(D.K - k, std::max<int64_t>(1, budget / std::max<int64_t>(row_b, 1)));
            take = std::min(take, kMaxPieceRows);
            if (D.K == 0) take = 0;
            pcs.push_back(ColPiece{d, k, k + take, piece++});
            k += take;
            acc += (int64_t)take * row_b;
            if (c + 1 < C && acc * C >= W * (c + 1)) {
                cut.push_back((int32_t)pcs.size());
                ++c;
            }
        } while (k < D.K);
        D.n_pieces = piece;
    }
    while ((int)cut.size() < C + 1) cut.push_back((int32_t)pcs.size());
    int64_t po = 0;
    for (auto& D : descs) {
        D.part_off = po;
        if (D.n_pieces > 1) po += (int64_t)D.n_pieces * D.n_out;
    }
    const size_t smem = (prec == PD_PREC_BF16) ? col_smem_bytes<__nv_bfloat16>() : col_smem_bytes<float>();
    const int lim = std::min(allow_max_dynamic_smem(k_stream_cols<float>),
                             allow_max_dynamic_smem(k_stream_cols<__nv_bfloat16>));
    if (smem > (size_t)lim) return false;
    upload(P.descs, descs, s);
    upload(P.pieces, pcs, s);
    upload(P.cta_pieces, cut, s);
    P.part.alloc((size_t)std::max<int64_t>(po, 1));
    P.cnt.alloc(std::max<size_t>(descs.size(), 1));
    PDG_CUDA(cudaMemsetAsync(P.cnt.p, 0, P.cnt.bytes(), s));
    PDG_CUDA(cudaStreamSynchronize(s));
    P.host = std::move(descs);
    P.n_ctas = pcs.empty() ? 0 : C;
    P.smem = smem;
    return true;
}

void launch_stream_cols(const StreamPlan& P, int prec, const void* pool, const float4* x, const int* xidx,
                        const float4* add, float4* out, int* err, cudaStream_t s) {
    if (P.n_ctas <= 0) return;
    const AxBases B{pool, x, xidx, add, out};
    if (prec == PD_PREC_BF16)
        k_stream_cols<__nv_bfloat16><<<P.n_ctas, kColThreads, P.smem, s>>>(P.descs.p, P.pieces.p, P.cta_pieces.p, B,
                                                                           P.part.p, P.cnt.p, err);
    else
        k_stream_cols<float><<<P.n_ctas, kColThreads, P.smem, s>>>(P.descs.p, P.pieces.p, P.cta_pieces.p, B, P.part.p,
                                                                   P.cnt.p, err);
    PDG_CHECK_LAUNCH();
}

// After a wait ran out the block counters may be left mid-count: clear them.
void reset_stream_plan(StreamPlan& P, cudaStream_t s) {
    if (P.cnt.p) PDG_CUDA(cudaMemsetAsync(P.cnt.p, 0, P.cnt.bytes(), s));
}

}  // namespace pdg
