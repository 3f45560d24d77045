// Streaming products of the subspace solve (Sec. 7.2) on sm_103a in the
// column ("axpy") form: out[o] = add[o] + sum_k A[k][o] x_k for o < n_out,
// x_k three right-hand sides (K = K_s (x) I_3).  Every product of the solve
// has this form with the factors of the pool: K_ii^-1 (symmetric), Psi_d,
// Psi_d^T, and the same for the second level.
//
// Layout: the plan copies each block into column panels of at most 256
// outputs, every panel contiguous (rows k of the panel back to back), so a
// unit of work (a panel, or a range of its rows) is one contiguous stream.
//
// The matrices are read once per solve and are far larger than L2: the
// launch is bound by HBM.  One producer thread per CTA streams whole-row
// tiles into a shared-memory ring with bulk asynchronous copies
// (cp.async.bulk, completion counted in bytes on an mbarrier), keeping
// kStages x kStageBytes per SM in flight whatever the compute warps do; a
// second warp loads the x slice of the next piece (one bulk copy, or
// gathered loads where the block says so) into a double buffer.  Sixteen
// consumer warps split the rows of a tile (row groups); each lane owns a few
// outputs of the panel and adds A[k][o] x_k with x_k a shared-memory
// broadcast and paired FMAs, accumulators in registers, no cross-lane
// reductions.  At the end of a piece all consumer threads add the row
// groups in group order through shared memory.
//
// Work split: the panels' rows are cut into pieces, one contiguous byte range
// of about the same size per CTA (a panel may span CTAs).  A panel cut into
// several pieces writes per-piece partial sums; the CTA that finishes the
// panel's last piece (an atomic counter, no waiting) adds them in piece
// order.  Results are bitwise reproducible for a given plan.
//
// Every wait is bounded: a wait that runs out sets ERR_TIMEOUT in the mesh's
// error word and marks the CTA aborted (no further copies are issued,
// consumers stop waiting); the producer and the x loader wait, again
// bounded, for their copies in flight before they exit.
#include <algorithm>

#include "pd_internal.h"
#include "tma.cuh"

namespace pdg {

namespace {

using namespace tma;

constexpr int kColWarps = 16;                            // consumer warps
constexpr int kEpiWarps = 4;                             // epilogue warps
constexpr int kColThreads = 32 * (kColWarps + 2 + kEpiWarps);   // + copy producer, x loader, epilogue
constexpr int kPanel = 256;                              // outputs of one panel
constexpr int kStages = 3;
constexpr int kStageBytes = 32 * 1024;
constexpr int kMaxGroups = 16;                           // row groups per slab
constexpr int kMaxPieceRows = 512;                       // x slice of a piece in shared memory
constexpr int kMaxCtaPieces = 64;                        // piece records of one CTA in shared memory
static_assert(sizeof(ColPieceRec) % 16 == 0, "piece records are copied in 16-byte words");

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

__device__ __forceinline__ void epi_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory");
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
    static constexpr int M = 1;
    static constexpr int OUT = 32 * VN * M;
    static constexpr int RB = (OUT <= 128) ? 3 : 2;   // row-group partial buffers (epilogue lag in pieces)
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

__device__ __forceinline__ float4 f4add(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, 0.f); }

__device__ __forceinline__ const float4* xvec_of(const FusedArgs& F, int kind) {
    switch (kind) {
        case XK_B: return F.b;
        case XK_CB: return F.cB;
        case XK_CT: return F.cT;
        case XK_G2: return F.xg2;
        default: return F.xgB;
    }
}

// atomic add with acquire-release semantics at gpu scope (publishes this
// thread's earlier stores; the last contributor sees everyone's)
__device__ __forceinline__ int atom_add_acq_rel(int* p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// what follows the store of a final output v at index o of a block
__device__ __forceinline__ void post_output(const FusedArgs& F, const ColDesc& D, int o, float4 v) {
    switch (D.post_kind) {
        case PK_CB: {
            const int j = __ldg(F.bidx + D.post_off + o);
            const int q0 = __ldg(F.gat_ptr + j), q1 = __ldg(F.gat_ptr + j + 1);
            if (atom_add_acq_rel(F.cnt_cb + j, 1) == q1 - q0 - 1) {
                float4 acc = F.b[F.n_int + j];
                for (int q = q0; q < q1; ++q) acc = f4add(acc, __ldcg(F.tc + __ldg(F.gat + q)));
                F.cB[j] = acc;
                F.cnt_cb[j] = 0;   // ready for the next launch
            }
            break;
        }
        case PK_CT: {
            const int t = __ldg(F.bidx2 + D.post_off + o);
            const int q0 = __ldg(F.gat2_ptr + t), q1 = __ldg(F.gat2_ptr + t + 1);
            if (atom_add_acq_rel(F.cnt_ct + t, 1) == q1 - q0 - 1) {
                float4 acc = __ldcg(F.cB + F.T0 + t);
                for (int q = q0; q < q1; ++q) acc = f4add(acc, __ldcg(F.tc2 + __ldg(F.gat2 + q)));
                F.cT[t] = acc;
                F.cnt_ct[t] = 0;
            }
            break;
        }
        case PK_XT: {
            const int t = D.post_off + o;
            for (int q = __ldg(F.inv2_ptr + t), e = __ldg(F.inv2_ptr + t + 1); q < e; ++q) F.xg2[__ldg(F.inv2 + q)] = v;
            const int j = F.T0 + t;
            for (int q = __ldg(F.invB_ptr + j), e = __ldg(F.invB_ptr + j + 1); q < e; ++q) F.xgB[__ldg(F.invB + q)] = v;
            break;
        }
        case PK_XB: {
            const int j = D.post_off + o;
            for (int q = __ldg(F.invB_ptr + j), e = __ldg(F.invB_ptr + j + 1); q < e; ++q) F.xgB[__ldg(F.invB + q)] = v;
            break;
        }
        default: break;
    }
}

__device__ __forceinline__ float4* vec_of(const FusedArgs& F, int kind) {
    return kind == VK_TC ? F.tc : (kind == VK_TC2 ? F.tc2 : F.x);
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// bounded wait for every CTA to have completed phase ph (false when it ran
// out, 1 s, or the CTA was marked aborted)
__device__ __forceinline__ bool phase_wait(const FusedArgs& F, int ph, const int* abort) {
    const unsigned long long t0 = gtime_ns();
    for (;;) {
        if (ld_acquire(F.phase_cnt + ph) >= F.n_ctas) return true;
        if (*reinterpret_cast<const volatile int*>(abort)) return false;
        if (gtime_ns() - t0 > kWaitNs) return false;
        __nanosleep(64);
    }
}

__device__ __forceinline__ void phase_arrive(const FusedArgs& F, int ph) {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    atomicAdd(F.phase_cnt + ph, 1);
}

// the final count: every CTA's x loader (past all its waits) and epilogue
// (past all its stores); the last of the 2 n_ctas arrivals clears the
// counters for the next launch
__device__ __forceinline__ void final_arrive(const FusedArgs& F) {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    if (atomicAdd(F.phase_cnt + F.n_phases, 1) == 2 * F.n_ctas - 1)
        for (int k = 0; k <= F.n_phases; ++k) F.phase_cnt[k] = 0;
}

// Work of CTA 0's epilogue threads before it signals phase ph: the entries
// of c_B (phase 0) and c_T (phase 1, after every CTA completed phase 0) that
// no block contributes to.
__device__ __forceinline__ void epi_extra(const FusedArgs& F, int ph, int et, const int* abort) {
    if (blockIdx.x != 0) return;
    if (ph == 0) {
        for (int k = et; k < F.n_cb0; k += 32 * kEpiWarps) {
            const int j = __ldg(F.cb0 + k);
            F.cB[j] = F.b[F.n_int + j];
        }
    } else if (ph == 1 && F.n_ct0 > 0) {
        bool ok = true;
        if (et == 0) ok = phase_wait(F, 0, abort);
        if (et == 0 && !ok) atomicOr(F.err, ERR_TIMEOUT);
        epi_sync();
        for (int k = et; k < F.n_ct0; k += 32 * kEpiWarps) {
            const int t = __ldg(F.ct0 + k);
            F.cT[t] = __ldcg(F.cB + F.T0 + t);
        }
    }
}

// One launch runs the products of the solve as phases: the copy producer
// streams every tile of this CTA's pieces in order (the matrices do not
// depend on the solve's data, so the stream runs ahead across phases); the x
// loader of a piece in phase p waits until every CTA has completed phase
// p - 1; the epilogue warps signal the completion of each phase.  Launched
// cooperatively (all CTAs resident).
template <class T>
__global__ void __launch_bounds__(kColThreads, 1) k_stream_solve(const ColPieceRec* __restrict__ recs,
                                                                 const int32_t* __restrict__ cta_pieces,
                                                                 FusedArgs F) {
    constexpr int VN = Slab<T>::VN, M = Slab<T>::M, SO = Slab<T>::OUT;
    constexpr int ES = (int)sizeof(T);
    constexpr int RB = Slab<T>::RB;
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char* ring = sm;
    float4* xs = reinterpret_cast<float4*>(sm + (size_t)kStages * kStageBytes);    // [2][kMaxPieceRows]
    float* red = reinterpret_cast<float*>(xs + 2 * kMaxPieceRows);                  // [RB][kColWarps][SO][3]
    uint64_t* full = reinterpret_cast<uint64_t*>(red + (size_t)RB * kColWarps * SO * 3);
    uint64_t* empty = full + kStages;
    uint64_t* xfull = empty + kStages;   // [2]
    uint64_t* xempty = xfull + 2;        // [2]
    uint64_t* rfull = xempty + 2;        // [RB]
    uint64_t* rempty = rfull + RB;       // [RB]
    __shared__ int abort_flag, last_flag;
    __shared__ __align__(16) ColPieceRec srec[kMaxCtaPieces];

    const int p0 = cta_pieces[blockIdx.x], p1 = cta_pieces[blockIdx.x + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    {
        // every piece record of this CTA into shared memory (16-byte words)
        const int nw = (p1 - p0) * (int)(sizeof(ColPieceRec) / 16);
        const int4* src = reinterpret_cast<const int4*>(recs + p0);
        int4* dst = reinterpret_cast<int4*>(srec);
        for (int k = threadIdx.x; k < nw; k += blockDim.x) dst[k] = src[k];
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < kStages; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kColWarps);
        }
        for (int k = 0; k < 2; ++k) {
            mbar_init(&xfull[k], 1);
            mbar_init(&xempty[k], kColWarps);
        }
        for (int k = 0; k < RB; ++k) {
            mbar_init(&rfull[k], kColWarps);
            mbar_init(&rempty[k], 1);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (p1 <= p0) {
        // no work here: complete every phase and the final count at once
        if (threadIdx.x < 32 * kEpiWarps) {
            for (int ph = 0; ph < F.n_phases; ++ph) {
                epi_extra(F, ph, threadIdx.x, &abort_flag);
                epi_sync();
                if (threadIdx.x == 0) phase_arrive(F, ph);
            }
            if (threadIdx.x == 0) {
                final_arrive(F);
                final_arrive(F);
            }
        }
        return;
    }
    const T* pool = reinterpret_cast<const T*>(F.pool);

    if (warp == kColWarps) {
        // ---- producer: one thread issues the bulk copies of every tile of this CTA
        if (lane != 0) return;
        int i = 0, issued = 0;
        bool stop = false;
        for (int p = p0; p < p1 && !stop; ++p) {
            const ColPiece pc = srec[p - p0].p;
            const ColDesc D = srec[p - p0].d;
            const int rpt = col_rows_per_tile(D.ld, ES);
            for (int k = pc.k0; k < pc.k1; k += rpt, ++i) {
                if (*reinterpret_cast<volatile int*>(&abort_flag)) {
                    stop = true;
                    break;
                }
                const int slot = i % kStages;
                if (i >= kStages && !mbar_wait(&empty[slot], (uint32_t)((i / kStages) - 1) & 1u, &abort_flag)) {
                    atomicOr(F.err, ERR_TIMEOUT);
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
            if (!mbar_wait(&full[j % kStages], (uint32_t)(j / kStages) & 1u)) atomicOr(F.err, ERR_TIMEOUT);
        return;
    }
    if (warp == kColWarps + 1) {
        // ---- x loader: the x slice of every piece into a double buffer, ahead
        // of the consumers; before the first piece of a phase p > 0 it waits
        // until every CTA has completed phase p - 1
        int bulk_mask = 0;   // bit b: the last slice written to buffer b came by bulk copy
        int done = 0;        // pieces whose slice was issued
        int ready = 0;       // phases whose inputs are known complete
        for (int p = p0; p < p1; ++p) {
            const int pp = p - p0, buf = pp & 1;
            const ColPiece pc = srec[pp].p;
            const ColDesc D = srec[pp].d;
            bool ok = true;
            if (pp >= 2 && lane == 0) ok = mbar_wait(&xempty[buf], (uint32_t)((pp / 2) - 1) & 1u, &abort_flag);
            if (ok && D.phase > ready) {
                if (lane == 0 && !*reinterpret_cast<volatile int*>(&abort_flag)) {
                    ok = phase_wait(F, D.phase - 1, &abort_flag);
                    // the bulk copies below read what other CTAs stored (generic proxy)
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                }
                ready = D.phase;
            }
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            __syncwarp();   // orders every lane's loads below after lane 0's acquire
            if (!ok) {
                if (lane == 0) {
                    atomicOr(F.err, ERR_TIMEOUT);
                    atomicExch(&abort_flag, 1);
                }
                break;
            }
            float4* xb = xs + buf * kMaxPieceRows;
            const int n = pc.k1 - pc.k0;
            if (n > 0) {
                // contiguous slice of a vector: one bulk copy, completion counted on xfull
                if (lane == 0) {
                    const uint32_t bytes = (uint32_t)n * 16u;
                    mbar_arrive_expect_tx(&xfull[buf], bytes);
                    bulk_g2s(xb, xvec_of(F, D.xkind) + D.x_off + pc.k0, bytes, &xfull[buf]);
                }
                bulk_mask |= 1 << buf;
            } else {
                bulk_mask &= ~(1 << buf);
                if (lane == 0) mbar_arrive(&xfull[buf]);
            }
            done = pp + 1;
        }
        // before exit: the last bulk copies have landed (normally long since consumed)
        for (int pp = (done > 2 ? done - 2 : 0); pp < done; ++pp)
            if (lane == 0 && (bulk_mask >> (pp & 1) & 1) && !mbar_wait(&xfull[pp & 1], (uint32_t)(pp / 2) & 1u))
                atomicOr(F.err, ERR_TIMEOUT);
        if (lane == 0) final_arrive(F);
        return;
    }
    if (warp >= kColWarps + 2) {
        // ---- epilogue warps: add the row groups of every output in group order,
        // write the outputs or the piece's partial sums (a panel cut into several
        // pieces is completed by the CTA finishing its last piece, adding the
        // pieces in order), and signal the completion of each phase
        const int et = threadIdx.x - 32 * (kColWarps + 2);
        int arrived = 0;   // phases signalled
        for (int p = p0; p < p1; ++p) {
            const int pp = p - p0, rbuf = pp % RB;
            const ColPiece pc = srec[pp].p;
            const ColDesc D = srec[pp].d;
            // all of this CTA's pieces of earlier phases are done
            for (; arrived < D.phase; ++arrived) {
                epi_extra(F, arrived, et, &abort_flag);
                epi_sync();
                if (et == 0) phase_arrive(F, arrived);
            }
            int S, G;
            col_layout(D.n_out, SO, S, G);
            if (et == 0 && !*reinterpret_cast<volatile int*>(&abort_flag) &&
                !mbar_wait(&rfull[rbuf], (uint32_t)(pp / RB) & 1u, &abort_flag)) {
                atomicOr(F.err, ERR_TIMEOUT);
                atomicExch(&abort_flag, 1);
            }
            epi_sync();
            const float* rb = red + (size_t)rbuf * kColWarps * SO * 3;
            const bool single = D.n_pieces == 1;
            float4* outv = vec_of(F, D.okind);
            const float4* addv = (D.akind == VK_NONE) ? nullptr : vec_of(F, D.akind);
            for (int o = et; o < D.n_out; o += 32 * kEpiWarps) {
                const int sl = o / SO, lo = o - sl * SO;
                float s0 = 0.f, s1 = 0.f, s2 = 0.f;
                for (int g = 0; g < G; ++g) {
                    const float* q = rb + ((size_t)(g * S + sl) * SO + lo) * 3;
                    s0 += q[0];
                    s1 += q[1];
                    s2 += q[2];
                }
                if (single) {
                    const float4 ad = addv ? __ldcg(addv + D.add_off + o) : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 v = make_float4(ad.x + s0, ad.y + s1, ad.z + s2, 0.f);
                    outv[D.out_off + o] = v;
                    post_output(F, D, o, v);
                } else {
                    F.part[D.part_off + (int64_t)pc.piece * D.n_out + o] = make_float4(s0, s1, s2, 0.f);
                }
            }
            epi_sync();   // red[rbuf] read by every epilogue thread
            if (et == 0) mbar_arrive(&rempty[rbuf]);
            if (!single) {
                if (et == 0) {
                    asm volatile("fence.acq_rel.gpu;" ::: "memory");
                    const int prev = atomicAdd(&F.cnt[pc.desc], 1);
                    asm volatile("fence.acq_rel.gpu;" ::: "memory");
                    last_flag = (prev == D.n_pieces - 1);
                }
                epi_sync();
                if (last_flag) {
                    for (int o = et; o < D.n_out; o += 32 * kEpiWarps) {
                        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll 4
                        for (int q = 0; q < D.n_pieces; ++q) {
                            const float4 v = __ldcg(&F.part[D.part_off + (int64_t)q * D.n_out + o]);
                            s0 += v.x;
                            s1 += v.y;
                            s2 += v.z;
                        }
                        const float4 ad = addv ? __ldcg(addv + D.add_off + o) : make_float4(0.f, 0.f, 0.f, 0.f);
                        const float4 v = make_float4(ad.x + s0, ad.y + s1, ad.z + s2, 0.f);
                        outv[D.out_off + o] = v;
                        post_output(F, D, o, v);
                    }
                    if (et == 0) F.cnt[pc.desc] = 0;   // ready for the next launch
                }
                epi_sync();   // last_flag free for the next piece
            }
        }
        for (; arrived < F.n_phases; ++arrived) {
            epi_extra(F, arrived, et, &abort_flag);
            epi_sync();
            if (et == 0) phase_arrive(F, arrived);
        }
        if (et == 0) final_arrive(F);
        return;
    }

    // ---- consumers: hand the row-group partials of a piece to the epilogue
    // warps and go on with the next piece
    int i = 0;   // tile counter (same sequence as the producer's)
    for (int p = p0; p < p1; ++p) {
        const int pp = p - p0, buf = pp & 1;
        const ColPiece pc = srec[pp].p;
        const ColDesc D = srec[pp].d;
        const int rpt = col_rows_per_tile(D.ld, ES);
        int S, G;
        col_layout(D.n_out, SO, S, G);
        if (!*reinterpret_cast<volatile int*>(&abort_flag) && !mbar_wait(&xfull[buf], (uint32_t)(pp / 2) & 1u, &abort_flag)) {
            atomicOr(F.err, ERR_TIMEOUT);
            atomicExch(&abort_flag, 1);
        }
        const float4* xb = xs + buf * kMaxPieceRows;
        const bool active = warp < S * G;
        const int slab = warp % S, grp = warp / S;
        const int o_base = slab * SO + lane * VN;
        // accumulators of output pairs (2jp, 2jp+1), one per right-hand side:
        // paired FMAs (FFMA2), each lane of the pair rounded like fmaf
        float2 acc[M][VN / 2][3];
#pragma unroll
        for (int mm = 0; mm < M; ++mm)
#pragma unroll
            for (int j = 0; j < VN / 2; ++j) acc[mm][j][0] = acc[mm][j][1] = acc[mm][j][2] = make_float2(0.f, 0.f);
        bool valid[M];
#pragma unroll
        for (int mm = 0; mm < M; ++mm) valid[mm] = active && (o_base + mm * 32 * VN < D.n_out);
        int ph = 0;   // (k - k0) mod G at the start of the tile
        for (int k = pc.k0; k < pc.k1; k += rpt, ++i) {
            const int slot = i % kStages;
            if (lane == 0 && !*reinterpret_cast<volatile int*>(&abort_flag) &&
                !mbar_wait(&full[slot], (uint32_t)(i / kStages) & 1u, &abort_flag)) {
                atomicOr(F.err, ERR_TIMEOUT);
                atomicExch(&abort_flag, 1);
            }
            __syncwarp();
            const T* A = reinterpret_cast<const T*>(ring + (size_t)slot * kStageBytes);
            const int nr = min(rpt, pc.k1 - k);
            if (valid[0]) {
                // rows r of the tile with (k - k0 + r) = grp (mod G)
                int r = grp - ph;
                if (r < 0) r += G;
#pragma unroll 2
                for (; r < nr; r += G) {
                    const float4 xk = xb[k - pc.k0 + r];
                    const float2 xx = make_float2(xk.x, xk.x), xy = make_float2(xk.y, xk.y);
                    const float2 xz = make_float2(xk.z, xk.z);
                    const T* a = A + r * D.ld + o_base;
#pragma unroll
                    for (int mm = 0; mm < M; ++mm) {
                        if (!valid[mm]) continue;
                        float v[VN];
                        vec_from_smem(a + mm * 32 * VN, v);
#pragma unroll
                        for (int j = 0; j < VN / 2; ++j) {
                            const float2 vv = make_float2(v[2 * j], v[2 * j + 1]);
                            acc[mm][j][0] = __ffma2_rn(vv, xx, acc[mm][j][0]);
                            acc[mm][j][1] = __ffma2_rn(vv, xy, acc[mm][j][1]);
                            acc[mm][j][2] = __ffma2_rn(vv, xz, acc[mm][j][2]);
                        }
                    }
                }
            }
            ph += nr;
            while (ph >= G) ph -= G;
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&xempty[buf]);   // this warp no longer reads the x slice
        const int rbuf = pp % RB;
        if (pp >= RB) {
            // red[rbuf] was last filled for piece pp - RB: the epilogue must be done with it
            if (lane == 0 && !*reinterpret_cast<volatile int*>(&abort_flag) &&
                !mbar_wait(&rempty[rbuf], (uint32_t)((pp / RB) - 1) & 1u, &abort_flag)) {
                atomicOr(F.err, ERR_TIMEOUT);
                atomicExch(&abort_flag, 1);
            }
            __syncwarp();
        }
        if (active) {
            float* rb = red + ((size_t)rbuf * kColWarps + (size_t)(grp * S + slab)) * SO * 3;
#pragma unroll
            for (int mm = 0; mm < M; ++mm)
#pragma unroll
                for (int j = 0; j < VN; ++j) {
                    const int lo = mm * 32 * VN + lane * VN + j;
                    rb[3 * lo] = (j & 1) ? acc[mm][j / 2][0].y : acc[mm][j / 2][0].x;
                    rb[3 * lo + 1] = (j & 1) ? acc[mm][j / 2][1].y : acc[mm][j / 2][1].x;
                    rb[3 * lo + 2] = (j & 1) ? acc[mm][j / 2][2].y : acc[mm][j / 2][2].x;
                }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&rfull[rbuf]);   // release: this warp's partials
    }
}

// Panel copies: dst panel (K rows x width, zero beyond `valid` columns) from
// columns [c0, c0 + valid) of a row-major block of the pool.
struct PanelCopy {
    int64_t src_off, dst_off;
    int32_t K, src_ld, c0, width, valid, pad;
};

template <class T>
__global__ void k_copy_panels(const PanelCopy* __restrict__ pc, const T* __restrict__ src, T* __restrict__ dst) {
    const PanelCopy P = pc[blockIdx.x];
    const int64_t n = (int64_t)P.K * P.width;
    for (int64_t l = threadIdx.x; l < n; l += blockDim.x) {
        const int k = (int)(l / P.width), j = (int)(l - (int64_t)k * P.width);
        dst[P.dst_off + l] = (j < P.valid) ? src[P.src_off + (int64_t)k * P.src_ld + P.c0 + j] : T(0.f);
    }
}

template <class T>
size_t col_smem_bytes() {
    return (size_t)kStages * kStageBytes + sizeof(float4) * 2 * kMaxPieceRows +
           sizeof(float) * (size_t)Slab<T>::RB * kColWarps * Slab<T>::OUT * 3 +
           sizeof(uint64_t) * (2 * kStages + 4 + 2 * Slab<T>::RB);
}

}  // namespace

// Builds the fused solve: copies every block (a_off into the row-major pool
// src; phase, x/add/out kinds set by the caller) into the plan's own pool as
// contiguous column panels of at most kPanel outputs, cuts the rows of each
// phase's panels into pieces so that every CTA gets a contiguous range of
// about the same number of bytes of every phase (at most kMaxPieceRows rows
// per piece), and lays out each CTA's pieces phase by phase.  Returns false
// (plan left empty) when a panel row does not fit in one stage or a CTA would
// hold more than kMaxCtaPieces pieces.
bool build_stream_plan(StreamPlan& P, const std::vector<ColDesc>& blocks, int prec, const void* src, cudaStream_t s) {
    P.n_ctas = 0;
    P.n_phases = 0;
    P.host.clear();
    const int es = (prec == PD_PREC_BF16) ? 2 : 4;
    int n_ph = 0;
    for (const auto& D : blocks) n_ph = std::max(n_ph, D.phase + 1);
    // panels, phase by phase
    std::vector<ColDesc> descs;
    std::vector<PanelCopy> copies;
    std::vector<std::vector<int>> ph_descs(n_ph);
    int64_t pool = 0;
    for (const auto& D : blocks) {
        if (D.n_out <= 0) continue;
        for (int c0 = 0; c0 < D.n_out; c0 += kPanel) {
            const int valid = std::min(kPanel, D.n_out - c0);
            const int width = (valid + 7) / 8 * 8;
            if ((int64_t)width * es > kStageBytes) return false;
            ColDesc p = D;
            p.a_off = pool;
            p.ld = width;
            p.n_out = valid;
            p.out_off = D.out_off + c0;
            p.add_off = (D.akind != VK_NONE) ? D.add_off + c0 : -1;
            p.post_off = D.post_off + c0;
            p.n_pieces = 1;
            ph_descs[D.phase].push_back((int)descs.size());
            descs.push_back(p);
            if (D.K > 0) copies.push_back(PanelCopy{D.a_off, pool, D.K, D.ld, c0, width, valid, 0});
            pool += (int64_t)D.K * width;
        }
    }
    int dev = 0, sms = 0;
    PDG_CUDA(cudaGetDevice(&dev));
    PDG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int C = std::max(1, sms);
    // per phase: walk its panels, closing a CTA's range when its byte budget is reached
    std::vector<std::vector<ColPiece>> per_cta(C);
    for (int ph = 0; ph < n_ph; ++ph) {
        int64_t W = 0;
        for (int d : ph_descs[ph]) W += (int64_t)descs[d].K * descs[d].ld * es + (int64_t)descs[d].n_out * 64;
        int64_t acc = 0;
        int c = 0;
        for (int d : ph_descs[ph]) {
            ColDesc& D = descs[d];
            const int64_t row_b = (int64_t)D.ld * es;
            int k = 0, piece = 0;
            acc += (int64_t)D.n_out * 64;
            do {
                const int64_t budget = W * (c + 1) / C - acc;
                int take =
                    (int)std::min<int64_t>(D.K - k, std::max<int64_t>(1, budget / std::max<int64_t>(row_b, 1)));
                take = std::min(take, kMaxPieceRows);
                if (D.K == 0) take = 0;
                per_cta[c].push_back(ColPiece{d, k, k + take, piece++});
                k += take;
                acc += (int64_t)take * row_b;
                if (c + 1 < C && acc * C >= W * (c + 1)) ++c;
            } while (k < D.K);
            D.n_pieces = piece;
        }
    }
    std::vector<int32_t> cut(C + 1, 0);
    std::vector<ColPiece> pcs;
    for (int c = 0; c < C; ++c) {
        if ((int)per_cta[c].size() > kMaxCtaPieces) return false;
        cut[c] = (int32_t)pcs.size();
        pcs.insert(pcs.end(), per_cta[c].begin(), per_cta[c].end());
    }
    cut[C] = (int32_t)pcs.size();
    int64_t po = 0;
    for (auto& D : descs) {
        D.part_off = po;
        if (D.n_pieces > 1) po += (int64_t)D.n_pieces * D.n_out;
    }
    std::vector<ColPieceRec> recs(pcs.size());
    for (size_t q = 0; q < pcs.size(); ++q) recs[q] = ColPieceRec{descs[pcs[q].desc], pcs[q]};
    const size_t smem = (prec == PD_PREC_BF16) ? col_smem_bytes<__nv_bfloat16>() : col_smem_bytes<float>();
    const int lim = std::min(allow_max_dynamic_smem(k_stream_solve<float>),
                             allow_max_dynamic_smem(k_stream_solve<__nv_bfloat16>));
    if (smem > (size_t)lim) return false;
    // all CTAs resident at once (the phases wait on one another)
    int per_sm = 0;
    if (prec == PD_PREC_BF16)
        PDG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_solve<__nv_bfloat16>, kColThreads,
                                                               smem));
    else
        PDG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_solve<float>, kColThreads, smem));
    if (per_sm < 1) return false;
    // the panel pool
    P.pan32.free();
    P.pan16.free();
    DBuf<PanelCopy> dcp;
    upload(dcp, copies, s);
    if (prec == PD_PREC_BF16) {
        P.pan16.alloc((size_t)std::max<int64_t>(pool, 8));
        if (!copies.empty())
            k_copy_panels<__nv_bfloat16><<<(int)copies.size(), 256, 0, s>>>(
                dcp.p, static_cast<const __nv_bfloat16*>(src), P.pan16.p);
    } else {
        P.pan32.alloc((size_t)std::max<int64_t>(pool, 8));
        if (!copies.empty())
            k_copy_panels<float><<<(int)copies.size(), 256, 0, s>>>(dcp.p, static_cast<const float*>(src), P.pan32.p);
    }
    PDG_CHECK_LAUNCH();
    upload(P.recs, recs, s);
    upload(P.cta_pieces, cut, s);
    P.part.alloc((size_t)std::max<int64_t>(po, 1));
    P.cnt.alloc(std::max<size_t>(descs.size(), 1));
    PDG_CUDA(cudaMemsetAsync(P.cnt.p, 0, P.cnt.bytes(), s));
    P.phase_cnt.alloc((size_t)n_ph + 1);
    PDG_CUDA(cudaMemsetAsync(P.phase_cnt.p, 0, P.phase_cnt.bytes(), s));
    PDG_CUDA(cudaStreamSynchronize(s));
    P.host = std::move(descs);
    P.prec = prec;
    P.n_phases = n_ph;
    P.n_ctas = pcs.empty() ? 0 : C;
    P.smem = smem;
    return true;
}

// One fused solve: every phase of the plan in one cooperative launch.
void launch_stream_solve(const StreamPlan& P, FusedArgs F, cudaStream_t s) {
    if (P.n_ctas <= 0) return;
    F.pool = (P.prec == PD_PREC_BF16) ? (const void*)P.pan16.p : (const void*)P.pan32.p;
    F.part = P.part.p;
    F.cnt = P.cnt.p;
    F.phase_cnt = P.phase_cnt.p;
    F.n_phases = P.n_phases;
    F.n_ctas = P.n_ctas;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P.n_ctas);
    cfg.blockDim = dim3(kColThreads);
    cfg.dynamicSmemBytes = P.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const ColPieceRec* recs = P.recs.p;
    const int32_t* cuts = P.cta_pieces.p;
    if (P.prec == PD_PREC_BF16) PDG_CUDA(cudaLaunchKernelEx(&cfg, k_stream_solve<__nv_bfloat16>, recs, cuts, F));
    else PDG_CUDA(cudaLaunchKernelEx(&cfg, k_stream_solve<float>, recs, cuts, F));
}

// After a wait ran out the counters may be left mid-count: clear them.
void reset_stream_plan(StreamPlan& P, cudaStream_t s) {
    if (P.cnt.p) PDG_CUDA(cudaMemsetAsync(P.cnt.p, 0, P.cnt.bytes(), s));
    if (P.phase_cnt.p) PDG_CUDA(cudaMemsetAsync(P.phase_cnt.p, 0, P.phase_cnt.bytes(), s));
    if (P.cnt_cb.p) PDG_CUDA(cudaMemsetAsync(P.cnt_cb.p, 0, P.cnt_cb.bytes(), s));
    if (P.cnt_ct.p) PDG_CUDA(cudaMemsetAsync(P.cnt_ct.p, 0, P.cnt_ct.bytes(), s));
}

}  // namespace pdg
