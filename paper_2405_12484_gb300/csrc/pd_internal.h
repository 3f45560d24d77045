// Internal declarations of libpdgb300: mesh object, device buffers, kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>
#include <map>
#include <memory>

#include "../../include/pd.h"

namespace pdg {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);

struct Fail {
    pd_status code;
};

#define PDG_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            ::pdg::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));              \
            (void)cudaGetLastError(); /* reported here: not left for the next check */          \
            throw ::pdg::Fail{e_ == cudaErrorMemoryAllocation ? PD_ERR_NO_MEMORY : PD_ERR_CUDA}; \
        }                                                                                     \
    } while (0)

#define PDG_CHECK_LAUNCH() PDG_CUDA(cudaGetLastError())

// Lets a kernel use all the dynamic shared memory the device allows per block
// (the attribute is per kernel and shared by every mesh and plan).  Returns
// that limit in bytes.
template <class K>
inline int allow_max_dynamic_smem(K* kernel) {
    int dev = 0, optin = 0;
    PDG_CUDA(cudaGetDevice(&dev));
    PDG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    PDG_CUDA(cudaFuncGetAttributes(&fa, kernel));
    const int lim = optin - (int)fa.sharedSizeBytes;
    PDG_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    return lim;
}

// Programmatic dependent launch (sm_90 and later): a kernel launched with
// launch_pdl may be scheduled while its stream predecessor is still running
// (once every block of the predecessor has started or called pdl_trigger);
// it must call pdl_wait() before it reads anything a predecessor wrote or
// writes anything a predecessor reads.  Constant data (the prefactored
// matrices, the topology) may be fetched before the wait.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    PDG_CUDA(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...));
}

// Device error flag bits (d_err).
enum : int { ERR_NONFINITE = 1, ERR_NOT_SPD = 2, ERR_TIMEOUT = 4 };

// ---------------------------------------------------------------- device buffer
// Allocation stream of the calling thread (set by AllocStreamScope): buffers
// allocated while one is set are stream-ordered (cudaMallocAsync on it) and
// freed on it (cudaFreeAsync, after the work queued there), so neither the
// allocation nor the free waits for the whole device.  cudaFree does: while
// one thread's prefactorisation freed a temporary, another thread's frames
// stalled until every queued kernel of that prefactorisation had finished.
// Without a scope (or while the stream is being captured) plain
// cudaMalloc / cudaFree.  Every use of a stream-ordered buffer is ordered
// after its allocation on that stream (the same stream, or a graph or a
// joined fork launched there), and its last use precedes the free there.
inline cudaStream_t& alloc_stream() {
    static thread_local cudaStream_t s = nullptr;
    return s;
}
struct AllocStreamScope {
    cudaStream_t prev;
    explicit AllocStreamScope(cudaStream_t s) : prev(alloc_stream()) { alloc_stream() = s; }
    ~AllocStreamScope() { alloc_stream() = prev; }
    AllocStreamScope(const AllocStreamScope&) = delete;
    AllocStreamScope& operator=(const AllocStreamScope&) = delete;
};

template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaStream_t owner = nullptr;   // stream-ordered: allocated and freed on this stream
    bool ordered = false;
    void alloc(size_t count) {
        free();
        if (count == 0) count = 1;
        void* q = nullptr;
        cudaStream_t s = alloc_stream();
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (s) PDG_CUDA(cudaStreamIsCapturing(s, &cs));
        if (s && cs == cudaStreamCaptureStatusNone) {
            PDG_CUDA(cudaMallocAsync(&q, count * sizeof(T), s));
            owner = s;
            ordered = true;
        } else {
            PDG_CUDA(cudaMalloc(&q, count * sizeof(T)));
            owner = nullptr;
            ordered = false;
        }
        p = static_cast<T*>(q);
        n = count;
    }
    void free() {
        if (p) {
            if (ordered) cudaFreeAsync(p, owner);
            else cudaFree(p);
        }
        p = nullptr;
        n = 0;
        ordered = false;
    }
    size_t bytes() const { return n * sizeof(T); }
    ~DBuf() { free(); }
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
};

// Host vector -> new device buffer (asynchronous on s; pageable sources are
// staged before the call returns).
template <class T>
inline void upload(DBuf<T>& d, const std::vector<T>& h, cudaStream_t s) {
    d.alloc(h.size());
    if (!h.empty()) PDG_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
}

// Column-oriented per-domain product y[o] = add[o] + sum_k A[k][o] x_k: base
// pointers of one launch (or of one serving slot) and the offsets of one
// domain matrix into them.
struct AxBases {
    const void* pool;      // matrix pool (float or bf16)
    const float4* x;       // vector source
    const int* bidx;       // gather list (boundary products) or null
    const float4* add;     // added to the result, or null
    float4* out;
};
struct AxDesc {
    int64_t a_off;         // pool offset of row 0
    int32_t x_off;         // x offset (contiguous source)
    int32_t bidx_off;      // >= 0: x_k = x[bidx[bidx_off + k]]
    int32_t add_off;       // >= 0: add offset
    int32_t out_off;
    int32_t K, ld, n_out;  // rows, row stride, outputs
    int32_t slot;          // serving slot (batched launches)
    int32_t tiled;         // 1: output-chunk tiles (see ax_tile_width); ld then holds the chunk width
    int32_t pad_[3];
};

// Tiled layout of an axpy-form matrix (K rows x n_out outputs cut into
// chunks of CW outputs, CW a multiple of VN, one chunk per block): the chunk
// with first output o0 (a multiple of CW) is a contiguous K x w tile at
// a_off + o0 K, row k at + k w, w = min(CW, n_out - o0 rounded up to VN).
__host__ __device__ inline int ax_tile_width(int n_out, int o0, int CW, int VN) {
    const int w = (n_out - o0 + VN - 1) / VN * VN;
    return w < CW ? w : CW;
}

// Balanced chunk width: the fewest chunks of at most OW outputs, equal widths
// (rounded up to VN).
__host__ __device__ inline int ax_chunk_width(int n_out, int OW, int VN) {
    const int c = (n_out + OW - 1) / OW;
    const int w = (n_out + c - 1) / c;
    return (w + VN - 1) / VN * VN;
}
struct AxBlock {
    int32_t desc, o0;      // descriptor and first output of one block
};

// Row-oriented product out[r] = add[r] + A[r, 0:cols] . x of one dense block
// (offsets into AxBases, as for AxDesc); u0 = first unit of the block in the
// concatenated unit list of its launch.
struct RowDesc {
    int64_t a_off;         // pool offset of row 0
    int64_t u0;
    int32_t rows, cols, ld;
    int32_t x_off;         // x offset (contiguous source)
    int32_t xidx_off;      // >= 0: x_k = x[bidx[xidx_off + k]]
    int32_t add_off;       // >= 0: add offset
    int32_t out_off;
    int32_t slot;          // serving batches: the request whose arrays the descriptor uses
};
// One row-form launch: its descriptors and the unit range of every block.
struct RowPlan {
    DBuf<RowDesc> descs;
    DBuf<int64_t> blk_u;
    int n_desc = 0, n_blocks = 0, xcap = 8;
    bool tma = false;              // rows streamed by bulk copies (k_rowdot_tma)
    bool mma = false;              // BF16 fragment layout on the tensor cores (k_rowdot_mma)
    std::vector<RowDesc> host;     // host copy (byte accounting)
};

// Streaming column-form product out[o] = add[o] + sum_k A[k][o] x_k of one
// dense block (a column panel of a factor), and a piece of its rows.  The
// fused solve runs several such products as phases of one launch; x, add
// and out name vectors of the solve (XK_*, VK_*) plus offsets into them.
enum : int32_t {
    XK_B = 0,      // x_k = b[x_off + k]      (input of the solve)
    XK_CB = 1,     // x_k = c_B[x_off + k]    (interface right-hand side)
    XK_CT = 2,     // x_k = c_T[x_off + k]    (top-level right-hand side)
    XK_G2 = 3,     // x_k = xg2[x_off + k]    (x_T gathered per group)
    XK_GB = 4,     // x_k = xgB[x_off + k]    (x_B gathered per domain)
};
enum : int32_t { VK_NONE = -1, VK_TC = 0, VK_TC2 = 1, VK_X = 2 };
// what the epilogue does with a final output besides storing it
enum : int32_t {
    PK_NONE = 0,
    PK_CB = 1,     // contribution to c_B[bidx[post_off + o]]: the last contributor forms the entry
    PK_CT = 2,     // contribution to c_T[bidx2[post_off + o]]: likewise
    PK_XT = 3,     // x_T[post_off + o]: copies into xg2 and xgB
    PK_XB = 4,     // x_B[post_off + o]: copies into xgB
};
struct ColDesc {
    int64_t a_off;         // pool offset of row 0
    int64_t part_off;      // partial-sum offset (blocks cut into several pieces)
    int32_t K, n_out, ld;  // rows, outputs, row stride
    int32_t x_off;         // offset of x_0 in the XK_* vector
    int32_t xidx_off;      // (unused by the fused solve)
    int32_t add_off;       // >= 0: add offset (into the add vector)
    int32_t out_off;
    int32_t n_pieces;
    int32_t phase;         // phase of the fused solve (0 = first)
    int32_t xkind;         // XK_*
    int32_t akind, okind;  // VK_* of the add and out vectors
    int32_t post_kind;     // PK_*
    int32_t post_off;
    int32_t pad0, pad1;
};
struct ColPiece {
    int32_t desc, k0, k1, piece;
};
// A piece with a copy of its block's descriptor: a CTA loads all of its
// records into shared memory once.
struct ColPieceRec {
    ColDesc d;
    ColPiece p;
};
// Vectors and index lists of one fused solve (kernel argument).
struct FusedArgs {
    const void* pool;
    const float4* b;
    float4* x;
    float4* tc;
    float4* tc2;
    float4* cB;
    float4* cT;
    float4* xg2;
    float4* xgB;
    float4* part;
    const int* gat_ptr;    // c_B[j] = b_B[j] + sum tc[gat[gat_ptr[j] ..]]
    const int* gat;
    const int* gat2_ptr;   // c_T[t] = c_B[T0 + t] + sum tc2[gat2[gat2_ptr[t] ..]]
    const int* gat2;
    const int* bidx;       // interface index of every (domain, boundary mode)
    const int* bidx2;      // top index of every (group, boundary mode)
    const int* invB_ptr;   // positions q with bidx[q] = j
    const int* invB;
    const int* inv2_ptr;   // positions q with bidx2[q] = t
    const int* inv2;
    const int* cb0;        // interface entries without a contribution
    const int* ct0;        // top entries without a contribution
    int* cnt;              // per panel: pieces done
    int* cnt_cb;           // per c_B entry: contributions done
    int* cnt_ct;           // per c_T entry
    int* phase_cnt;        // per phase: CTAs done; [n_phases]: final count (loaders and epilogues)
    int* err;
    int n_int, T0, n_phases, n_ctas, n_cb0, n_ct0;
};
// One fused streaming solve: piece records, the piece range of every CTA,
// partial sums, counters and the panel pool.
struct StreamPlan {
    DBuf<ColPieceRec> recs;
    DBuf<int32_t> cta_pieces;
    DBuf<float4> part;
    DBuf<int32_t> cnt;
    DBuf<int32_t> phase_cnt;
    DBuf<int32_t> cnt_cb, cnt_ct;
    DBuf<float> pan32;             // the blocks as column panels (the plan's own copy)
    DBuf<__nv_bfloat16> pan16;
    int prec = 0;
    int n_ctas = 0;
    int n_phases = 0;
    size_t smem = 0;
    std::vector<ColDesc> host;
};

// Tets per block of the fused local step and RHS assembly.
#ifndef PDG_LA_TETS
#define PDG_LA_TETS 128
#endif

// Arguments of the fused local step and assembly (see k_local.cu).
struct LocalAsmArgs {
    int n_t;
    const int4* tets;
    const float4* geo;
    const float4* x;
    const float4* by0;     // RHS form: (m/dt^2) y - K_fp x_p
    const float4* y;       // residual form: the inertial target
    const float* mh2;
    float4* b;             // RHS or residual (free vertices)
    const int *vptr, *vert, *slot, *cptr;
    const uint16_t* corner;
    const int *sh_ptr, *sh_vert;
    float4* part;
};

// One resident request of the serving loop, as the batched kernels see it.
struct BatchSlot {
    const int4* tets;
    const float4* geo;
    float4 *x, *xprev, *v, *by0, *b, *pin_tgt;
    const float4* pin_rest;
    const float* mh2;
    const int *kfp_ptr, *kfp_col;
    const float* kfp_val;
    float4 *tc, *cB, *part;
    const int *gat_ptr, *gat;
    // second level (two-level interface solve): c_T = c_B[T0:] - gathered t2 entries
    const int *gat2_ptr, *gat2;
    float4 *tc2, *cT;
    int n_top, two_level;
    int* err;
    int* frame;          // frames completed (device counter)
    // plan of the fused local step + assembly (see LocalAsmArgs)
    const int *la_vptr, *la_vert, *la_slot, *la_cptr, *la_sh_ptr, *la_sh_vert;
    const uint16_t* la_corner;
    float4* la_part;
    int la_shared;
    int n_t, n_v, n_free, n_pin, n_int, n_B, nch;
    float h, gx, gy, gz;
    float drive_amp, drive_w;
    int drive_axis;
};

// The slot of a block of a batched launch: the last s with off[s] <= b
// (off[0] = 0, off increasing).
__device__ __forceinline__ int batch_find_slot(const int* __restrict__ off, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The interface matrix S^-1 of one slot in the batched coarse kernel.
struct CoarseDescB {
    const float* S;
    const float4* cB;
    float4* part;
    int64_t u0;            // first unit of this slot in the concatenated unit list
    int32_t n_B, ld, nch, pad;
};

enum Phase : int {
    PH_INERTIA = 0, PH_LOCAL, PH_ASSEMBLE, PH_CONDENSE, PH_GATHER, PH_COARSE, PH_REDUCE,
    PH_BACKSUB, PH_RESIDUAL, PH_VELOCITY, PH_CONDENSE2, PH_GATHER2, PH_BACKSUB2, PH_INTERIOR, PH_INTERIOR2,
    PH_SOLVE, PH_MODAL, PH_JACOBI, PH_COUNT
};

// ---------------------------------------------------------------- mesh
struct pd_mesh_impl;

}  // namespace pdg

struct pd_mesh {
    // sizes
    int32_t n_v = 0, n_t = 0, n_dom = 0, n_pin = 0, n_free = 0, n_int = 0, n_B = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs (high priority)
    bool node_priority = true;          // instantiate frames with the captured per-node priorities
    bool ax_tiled = false;              // axpy-form matrices stored as tiles, streamed by bulk copies
    bool ax_tf32 = false;               // TF32 tiles in the tensor-core fragment layout (k_axpy_mma<true>)
    // side streams of the subspace solve: the interior parts of the two
    // condensations run beside the interface solve (fork/join by events)
    cudaStream_t side[2] = {nullptr, nullptr};
    cudaEvent_t ev_fork[2] = {nullptr, nullptr}, ev_join[2] = {nullptr, nullptr};

    // host-side topology (new vertex numbering: [domain internals][interface][pinned])
    std::vector<int32_t> new_of_old, old_of_new;  // vertex maps
    std::vector<int32_t> tet_old_of_new;          // tet order: sorted by domain
    std::vector<int32_t> tets_new;                // n_t x 4, new vertex ids
    std::vector<int32_t> tet_dom;                 // domain of each (sorted) tet
    std::vector<double> vol;                      // rest volume of each (sorted) tet
    std::vector<double> Dminv;                    // n_t x 9 (sorted tets)
    std::vector<double> mass;                     // n_v (new numbering)
    std::vector<int32_t> dom_int_off, dom_n_int;  // per domain: first internal vertex, count
    std::vector<std::vector<int32_t>> dom_bnd;    // per domain: interface ids (0..n_B) coupled to its internals
    // two-level interface solve: groups of domains, interface block ordered as
    // [group 0 internal | ... | group G-1 internal | top level]
    int32_t n_groups = 0, n_top = 0;
    std::vector<int32_t> grp_of_dom, grp_n2;
    std::vector<uint64_t> top_mask;                         // per top-level vertex (interface order): group bits
    std::vector<std::pair<int32_t, uint64_t>> top_groups_of_old;   // (caller vertex id, group bits)
    // CSR of the scalar matrix over free vertices (new numbering) and of the free-pinned block
    std::vector<int32_t> K_rowptr, K_col;         // n_free rows, columns < n_free
    std::vector<int32_t> Kfp_rowptr, Kfp_col;     // n_free rows, columns = pinned slot (0..n_pin)
    std::vector<double> K_val, Kfp_val;
    std::vector<float> gamma_s, gamma_v;          // sorted tet order

    // device: geometry and state
    pdg::DBuf<int4> d_tets;         // n_t
    pdg::DBuf<float4> d_geo;        // 3 * n_t: rows g1|g2|g3 (xyz) + (ws, wv, 0) in .w
    pdg::DBuf<float4> d_x, d_xprev, d_v;   // n_v each
    pdg::DBuf<float4> d_force;      // 4 * n_t
    pdg::DBuf<float4> d_by0;        // n_free
    pdg::DBuf<float4> d_b;          // n_free
    pdg::DBuf<float4> d_pin_tgt;    // n_pin
    pdg::DBuf<float> d_mh2;         // n_free: m / dt^2
    pdg::DBuf<int32_t> d_inc_ptr, d_inc;   // free-vertex -> (tet*4+corner) CSR
    pdg::DBuf<float4> d_y;                 // inertial target of the free vertices (residual form)
    // fused local step + assembly: per block the free vertices it touches
    // (vptr over blocks; vertex, slot or -1, corner CSR of block-local corner
    // ids), the shared vertices (sh_vert) with their slots (sh_ptr) and the
    // partial sums of the slots
    pdg::DBuf<int32_t> d_la_vptr, d_la_vert, d_la_slot, d_la_cptr, d_la_sh_ptr, d_la_sh_vert;
    pdg::DBuf<uint16_t> d_la_corner;
    pdg::DBuf<float4> d_la_part;
    int32_t la_blocks = 0, la_entries = 0, la_corners = 0, la_slots = 0, la_shared = 0;
    pdg::DBuf<int32_t> d_kfp_ptr, d_kfp_col;
    pdg::DBuf<float> d_kfp_val;
    pdg::DBuf<int32_t> d_old_of_new;       // n_v
    pdg::DBuf<int32_t> d_err;              // device error flags

    // device: subspace solve (per-iteration data)
    int32_t prec = PD_PREC_FP32;
    int32_t refine = 0;
    bool correction = false;                // PD_SOLVE_CORRECTION
    pdg::DBuf<float> d_mat32;               // matrix pool (FP32 or TF32-rounded)
    pdg::DBuf<__nv_bfloat16> d_mat16;       // matrix pool (BF16)
    int64_t off_S = 0;                      // pool offset of S^-1
    int32_t ld_S = 0;
    // per-domain products (axpy form): boundary modes, interior part, back-substitution
    pdg::DBuf<pdg::AxDesc> d_ax_desc_cond, d_ax_desc_int, d_ax_desc_back;
    pdg::DBuf<pdg::AxBlock> d_ax_blk_cond, d_ax_blk_int, d_ax_blk_back;
    int32_t ax_blocks_cond = 0, ax_blocks_int = 0, ax_blocks_back = 0;
    int32_t ax_kmax_cond = 1, ax_kmax_int = 1, ax_kmax_back = 1;   // largest K (shared-memory vector size)
    int32_t ax_wmax_cond = 1, ax_wmax_int = 1, ax_wmax_back = 1;   // largest tile width (tiled layout)
    // second level (groups of domains): condensation onto the top-level interface
    bool two_level = false;
    int32_t cs_n = 0;                                       // rows of the dense coarse inverse in the pool
    pdg::RowPlan rows_cond2, rows_back2;   // row-form launches of the second level
    pdg::RowPlan rows_int2;                // second-level interior part S_II^-1 c_I
    pdg::RowPlan rows_coarse;              // BF16 tensor cores: the coarse product as a row-form product
    // the fused streaming solve (one cooperative launch per solve); used when it
    // could be planned (every panel row fits one pipeline stage)
    bool use_stream = false;
    // the paper's own global step (PD_SOLVE_MODAL): rank-r interior response
    // t = (Phi Lambda^-1)(Phi^T b_i), then Chebyshev-weighted Jacobi sweeps
    bool modal = false;
    int32_t modes = 0, jacobi_sweeps = 0;
    double jacobi_rho = 0.0;
    double modal_lambda_min = 0.0;          // smallest kept normal-mode eigenvalue (diagnostics)
    pdg::DBuf<pdg::AxDesc> d_ax_desc_m1, d_ax_desc_m2;
    pdg::DBuf<pdg::AxBlock> d_ax_blk_m1, d_ax_blk_m2;
    int32_t ax_blocks_m1 = 0, ax_blocks_m2 = 0, ax_kmax_m1 = 1, ax_kmax_m2 = 1;
    pdg::DBuf<float4> d_pm;                 // modal coordinates p (sum of the domains' r)
    int32_t n_pm = 0;
    pdg::DBuf<double> d_Dinv;               // 1 / diag K_ff
    pdg::DBuf<float4> d_jx1, d_jx2;         // Jacobi iterates
    std::vector<float> jacobi_omega;        // Chebyshev weights of the sweeps
    bool batched_only = false;             // set by the serving loop: no streaming plans
    int32_t sms = 1;                       // multiprocessors of the mesh's device
    pdg::StreamPlan st_solve;
    pdg::DBuf<int32_t> d_bidx2, d_gat2_ptr, d_gat2;
    pdg::DBuf<float4> d_tc2, d_cT;
    // fused solve: gathered copies of x_T (per group) and x_B (per domain), the
    // inverse gather lists, and the entries without any contribution
    pdg::DBuf<float4> d_xg2, d_xgB;
    pdg::DBuf<int32_t> d_invB_ptr, d_invB, d_inv2_ptr, d_inv2, d_cb0, d_ct0;
    int32_t n_cb0 = 0, n_ct0 = 0, n_xg2 = 0, n_xgB = 0;
    int32_t n_tc2 = 0, n_gat2 = 0;
    std::vector<pdg::AxDesc> h_ax_desc_cond, h_ax_desc_back;   // host copies (serving batches)
    pdg::DBuf<float4> d_tc;                 // stacked [t_d; c_d] rows of every domain
    int32_t n_tc = 0;
    pdg::DBuf<int32_t> d_bidx;              // concatenated per-domain boundary index lists
    pdg::DBuf<int32_t> d_gat_ptr, d_gat;    // interface vertex -> rows of tc holding its c_d pieces
    pdg::DBuf<float4> d_cB;                 // n_B condensed interface RHS
    pdg::DBuf<float4> d_part;               // coarse partial sums: n_chunks x n_B
    int32_t coarse_chunk = 0, coarse_nchunks = 0, coarse_rows_per_cta = 0;
    int32_t coarse_blocks = 0;              // > 0: balanced coarse kernel with this many blocks
    // FP64 residual for refinement
    pdg::DBuf<int32_t> d_K_ptr, d_K_col;
    pdg::DBuf<double> d_K_val;
    pdg::DBuf<float4> d_r, d_dx;             // refinement residual / correction (n_free)

    // generations of the FP32 state (pd_set_state, pd_step) and of the
    // materials (pd_set_materials): the adjoint workspace's FP64 state and
    // FP64 per-tet weights follow them
    uint64_t state_gen = 0, mat_gen = 0;
    // state flags
    bool materials_set = false;
    bool prefactored = false;
    double dt = 0.0;
    bool use_graphs = true;
    double prefactor_seconds = 0.0;
    int64_t phase_bytes[24] = {0};
    int32_t phase_launches[24] = {0};   // launches of each phase per PD iteration (or per frame)
    int32_t launches_per_iter = 0;

    // per-phase timing: the event pairs recorded by one captured graph (or by
    // the plain launches); each graph owns its set, so replaying one graph never
    // reads events that another graph's capture assigned to other phases
    struct TimingSet {
        std::vector<cudaEvent_t> ev;      // pairs (start, stop)
        std::vector<int32_t> phase;       // phase of each pair
        int32_t used = 0;
        ~TimingSet() {
            for (auto e : ev) cudaEventDestroy(e);
        }
    };

    // graphs: key = (n_iter, gravity bits, refinement steps, timing mask)
    struct GraphEntry {
        cudaGraphExec_t exec = nullptr;
        std::shared_ptr<TimingSet> timing;
    };
    std::map<std::vector<uint32_t>, GraphEntry> graphs;

    int32_t timing_mask = 0;
    int32_t timing_iter = -1;   // >= 0: loop phases timed in this iteration only
    int32_t cur_iter = -1;      // the iteration being recorded (-1 outside the loop)
    TimingSet* ev_rec = nullptr;                  // set being recorded into (during capture / plain launches)
    std::shared_ptr<TimingSet> ev_plain;          // set of the plain launches
    std::shared_ptr<TimingSet> ev_last;           // set of the last frame launched (read by pd_phase_times)
    bool timing_armed = false;
    bool ev_open = false;

    ~pd_mesh();
};

// Workspace of the adjoint path (equilibrium steps, adjoint steps, Gauss-Newton).
struct pd_adjoint {
    pd_mesh* mesh = nullptr;
    int32_t cg_iters = 30;
    pdg::DBuf<float4> xeq, vprev, g, rhs, lam, lam1, lam2, r, z, p, Ap, dx;
    pdg::DBuf<double> partial, sc;
    pdg::DBuf<float> vol;
    pdg::DBuf<int32_t> user_of_tet;
    // Gauss-Newton (allocated on first use): per-tet V_e (F - R), V_e (F - V)
    // (9 planes of n_t each), parameter-space CG vectors (2 n_t), vertex
    // vectors of the two inner solves, and the outer scalars.
    pdg::DBuf<float> gn_Ts, gn_Tv, gn_r, gn_p, gn_q, gn_ap, gn_tmp;
    pdg::DBuf<float4> gn_b, gn_mu, gn_nu;
    pdg::DBuf<double> gn_sc, gn_partial;
    pdg::DBuf<int32_t> gn_ipartial;
    bool gn_ready = false;
    // FP64 state of the equilibrium steps (3 doubles per vertex, library
    // order): x, v, the state the step started from, the state given to the
    // adjoint step; FP64 per-tet operators (12 doubles per tet), M/dt^2,
    // corner terms; the adjoint refinement vectors
    pdg::DBuf<double> x64, v64, xprev64, vprev64, xa64, geo64, mh2_64, force64;
    pdg::DBuf<float4> rhs2, dlam;
    uint64_t gen64 = ~uint64_t(0);       // mesh state generation x64/v64 belong to
    uint64_t mat_gen64 = ~uint64_t(0);   // material generation of geo64
    double dt64 = 0.0;                   // dt of mh2_64
};

namespace pdg {

void adjoint_pcg(pd_mesh* m, pd_adjoint* a, const float4* x_lin, const float4* b, float4* x, cudaStream_t s);

// Small dense FP64 helpers (host, q up to ~100; row-major q x q with leading dimension ld):
// Cholesky G = R^T R and R^-1 (false if G is not SPD); cyclic Jacobi eigen-decomposition
// (A overwritten, eigenvalues in w unsorted, eigenvectors in the columns of V).
bool chol_upper_inverse(const double* G, int q, int ld, std::vector<double>& Rinv);
void jacobi_eig(std::vector<double>& A, int q, std::vector<double>& w, std::vector<double>& V);

// ---------------------------------------------------------------- kernels (launchers)
void launch_project(const float* F, int n, float* R, float* V, float* sig, cudaStream_t s);
void build_local_plan(pd_mesh* m, const std::vector<int32_t>& inc_ptr, const std::vector<int32_t>& inc,
                      cudaStream_t s);
// fused local step + assembly: b = by0 + sum (RHS form) or b = (M/dt^2)(y - x) + sum (residual form)
void launch_local_assemble(const pd_mesh* m, const float4* x, const float4* by0, const float4* y, float4* b,
                           bool residual, cudaStream_t s);
void launch_inertia(const pd_mesh* m, float h, float gx, float gy, float gz, cudaStream_t s);
void launch_velocity(const pd_mesh* m, float inv_h, cudaStream_t s);
void launch_pin_copy(const pd_mesh* m, const float* user_targets, cudaStream_t s);
void launch_pin_hold(const pd_mesh* m, cudaStream_t s);
void launch_scatter_out(const pd_mesh* m, const float4* src, float* dst, int free_only, cudaStream_t s);
void launch_gather_in(const pd_mesh* m, const float* src, float4* dst, cudaStream_t s);
void launch_by0_from_y(const pd_mesh* m, const float4* y, float4* by0, cudaStream_t s);

// subspace solve: b (free, new order) -> x positions of free vertices written into `xout`
// (float4 array indexed by new vertex id).
void launch_dd_solve(pd_mesh* m, const float4* b, float4* xout, cudaStream_t s, bool timed);
void launch_residual(const pd_mesh* m, const float4* b, const float4* x, float4* r, cudaStream_t s);
void launch_axpy_free(const pd_mesh* m, const float4* dx, float4* x, cudaStream_t s);

// FP64 dense factorisations (device), used by the prefactorisation.
void dense_gemm(bool ta, bool tb, int M, int N, int K, double alpha, const double* A, int lda,
                int64_t sA, const double* B, int ldb, int64_t sB, double beta, double* C, int ldc,
                int64_t sC, int batch, bool lower_only, cudaStream_t s);
void dense_set_identity(double* A, int n, int lda, int64_t strideA, int batch, cudaStream_t s);

// Resolves the fixed scratch array of pd_solve_noalloc on the current device
// (loads its module; called by pd_prefactor while allocation is allowed).
pd_status noalloc_prepare_device();

// timing helpers (no-ops unless the phase is in the mesh's timing mask)
void phase_begin(pd_mesh* m, int phase, cudaStream_t s);
void phase_end(pd_mesh* m, cudaStream_t s);

}  // namespace pdg
