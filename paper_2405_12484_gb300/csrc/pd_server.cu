// Serving loop of the C ABI: continuous batching of garment simulations on
// one GPU.  Requests (one mesh each) are admitted by a worker thread while
// the HBM budget and the slots allow: it builds the mesh and runs the FP64
// prefactorisation on its own low-priority stream, so the requests already
// resident keep advancing meanwhile.  Every resident request advances one
// frame per pd_server_tick in shared batched launches (one CUDA graph per
// set of resident requests); a newly prepared request joins at the next
// tick.  Retired meshes are freed by the worker too, so the tick thread
// never waits on a device-wide free.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <system_error>
#include <thread>
#include <vector>

#include "pd_internal.h"

namespace pdg {

void launch_b_drive(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s);
void launch_b_inertia(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s);
void launch_b_local_assemble(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s);
void launch_b_assemble_shared(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s);
void launch_b_gather(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s);
void launch_b_reduce(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s);
void launch_b_gather2(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s);
void launch_rowdot_b(const RowPlan& P, const AxBases* multi, int* err, cudaStream_t s);
void build_row_plan(RowPlan& P, std::vector<RowDesc> descs, int prec, cudaStream_t s, bool mma);
void launch_b_velocity(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s);
void launch_axpy_b(const AxDesc* descs, const AxBlock* blocks, const AxBases* bases, int n_blocks, int k_max,
                   int w_max, int* err, cudaStream_t s);
int ax_outputs_per_block(int prec);
bool configure_coarse_b(int max_cols);
void launch_coarse_b(const CoarseDescB* cd, int n_desc, int64_t U, int max_cols, int blocks, cudaStream_t s);

}  // namespace pdg

using namespace pdg;

namespace {

struct Request {
    pd_request_id id = 0;
    std::vector<double> rest;
    std::vector<int32_t> tets, dom;
    std::vector<uint8_t> pinned;
    std::vector<float> gs, gv;
    int32_t n_v = 0, n_t = 0, n_dom = 1, n_frames = 0;
    double density = 300.0, dt = 1.0 / 150.0;
    float g[3] = {0.f, 0.f, -9.81f};
    float amp = 0.f, freq = 0.f;
    int32_t axis = 0;
    int32_t state = PD_REQ_QUEUED;
    pd_mesh* mesh = nullptr;
    int64_t steady_bytes = 0;
    // device-memory estimate from the first build of the mesh (kept while the
    // request waits, so that it is not rebuilt at every tick)
    bool estimated = false;
    int64_t est_steady = 0, est_transient = 0;
    DBuf<float4> pin_rest;
    DBuf<int32_t> frame;
    int32_t frames_done = 0;
    // per-frame latency seen by the request: wall time from its admission (or
    // its previous frame) to the completion of the frame, stalls included
    std::chrono::steady_clock::time_point t_last;
    std::vector<float> frame_ms, x_final;
    ~Request() {
        if (mesh) pd_destroy_mesh(mesh);
    }
};

using Clock = std::chrono::steady_clock;

enum { PH_DRIVE = 0, PH_INER, PH_LOC, PH_ASM, PH_GAT, PH_RED, PH_VEL, PH_GAT2, PH_NB };

}  // namespace

// A stream destroyed with its owner.  Declared first in pd_server, so that it
// outlives every member buffer freed on it (members are destroyed in reverse
// order, after the destructor's body).
struct OwnedStream {
    cudaStream_t s = nullptr;
    ~OwnedStream() {
        if (s) cudaStreamDestroy(s);
    }
};

struct pd_server {
    OwnedStream frame_stream;              // the frames' stream (highest priority)
    int64_t budget = 0;
    int32_t max_slots = 0, n_iter = 20;
    int device = 0;
    cudaStream_t user = nullptr;           // the caller's stream: each tick is ordered after its prior work
    cudaStream_t stream = nullptr, cap = nullptr;   // stream = frame_stream.s
    cudaEvent_t e_user = nullptr;
    int32_t* h_err = nullptr;              // pinned copy of d_err
    cudaStream_t adm = nullptr;            // admission stream (lowest priority)
    std::vector<cudaStream_t> adm_streams; // one per admission thread (lowest priority)
    pd_request_id next_id = 1;
    // shared with the admission worker (under mu)
    std::mutex mu;
    std::condition_variable cv;            // work for the worker
    std::condition_variable cv_ready;      // a request became ready (or failed)
    std::map<pd_request_id, std::unique_ptr<Request>> reqs;
    std::deque<pd_request_id> queue;       // waiting for admission, in arrival order
    std::deque<pd_request_id> ready;       // prepared by the worker, joining at the next tick
    std::vector<std::pair<pd_mesh*, int64_t>> retired;   // meshes the worker frees, with their budgeted bytes
    int32_t n_active = 0;                  // resident requests (read by the workers)
    int32_t n_preparing = 0;               // requests taken from the queue by a worker
    bool stop = false;
    int64_t used = 0, reserved = 0, peak = 0;
    uint64_t freed_gen = 0;                // bumps whenever memory or a slot is returned
    std::vector<std::thread> workers;      // admission threads (mesh set-up is host work: several in parallel)
    std::mutex prefactor_mu;               // one FP64 prefactorisation on the GPU at a time beside the frames
    // tick thread only
    std::vector<pd_request_id> active;
    bool dirty = true;
    cudaGraphExec_t graph = nullptr;
    int sms = 0;
    // batch descriptors (capacity grows, never shrinks: no free on the tick thread)
    DBuf<BatchSlot> d_slots;
    DBuf<int32_t> d_off[PH_NB];
    int blocks[PH_NB] = {0};
    DBuf<AxDesc> d_axc, d_axb;
    DBuf<AxBlock> d_blkc, d_blkb;
    DBuf<AxBases> d_basc, d_basb;
    // two-level requests: the second level's row-form products over every such request
    RowPlan rows_r2, rows_co, rows_b2;      // S_II^-1 and Psi2^T rows; S2^-1 rows; Psi2 rows
    DBuf<AxBases> d_basr2, d_basco, d_basb2;
    int blocks_c = 0, blocks_b = 0, kmax_c = 1, kmax_b = 1, wmax_c = 1, wmax_b = 1;
    DBuf<CoarseDescB> d_cd;
    int n_cd = 0, max_cols = 0, coarse_blocks = 0;
    int64_t units = 0;
    DBuf<float> d_out;                     // final positions of a retiring request
    DBuf<int32_t> d_err;                   // bounded-wait flag of the batched products
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~pd_server() {
        if (graph) cudaGraphExecDestroy(graph);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (e_user) cudaEventDestroy(e_user);
        if (h_err) cudaFreeHost(h_err);
        if (cap) cudaStreamDestroy(cap);
        if (adm) cudaStreamDestroy(adm);
        for (auto st : adm_streams)
            if (st) cudaStreamDestroy(st);
    }
};

static pd_status sfail(pd_status c, const std::string& m) {
    set_error(m);
    return c;
}

// Device memory of a resident request (after pd_prefactor) and the extra
// transient memory of its FP64 prefactorisation, from the mesh sizes.
static void estimate(pd_mesh* m, int64_t& steady, int64_t& transient) {
    pd_mesh_info in{};
    pd_get_info(m, &in);
    const int64_t NI = (in.max_domain_internal + 63) / 64 * 64, NB = (in.max_domain_boundary + 7) / 8 * 8;
    const int64_t nB = in.n_interface, nBp = (nB + 63) / 64 * 64, nd = in.n_domains;
    const int64_t pool = nd * ((NI + NB) * NI + NI * NB) * 4 + nB * ((nB + 7) / 8 * 8) * 4;
    const int64_t small = (int64_t)in.n_tets * 64 + (int64_t)in.n_vertices * 96 + nd * (NI + NB) * 16 +
                          nB * 16 * ((nB + 2047) / 2048 + 1);
    steady = in.device_bytes + pool + small;
    transient = nd * (2 * NI * NI + 2 * NI * NB + NB * NB) * 8 + 2 * nBp * nBp * 8 + nBp * 64 * 8 * 2;
}

// Copies a host vector into a device buffer whose capacity only grows (a
// reallocation, the only free here, happens when a larger resident set first
// appears).
template <class T>
static void put(DBuf<T>& d, const std::vector<T>& h, cudaStream_t s) {
    if (h.size() > d.n) d.alloc(std::max(h.size(), 2 * d.n));
    if (!h.empty()) PDG_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
}

static void rebuild(pd_server* S) {
    const int n = (int)S->active.size();
    if (S->graph) {
        cudaGraphExecDestroy(S->graph);
        S->graph = nullptr;
    }
    S->dirty = false;
    if (n == 0) return;
    std::vector<BatchSlot> slots(n);
    std::vector<int32_t> off[PH_NB];
    for (auto& o : off) o.assign(n + 1, 0);
    std::vector<AxDesc> axc, axb;
    std::vector<AxBlock> blkc, blkb;
    std::vector<AxBases> basc(n), basb(n);
    std::vector<CoarseDescB> cd;
    std::vector<RowDesc> r2, co, b2;
    std::vector<AxBases> basr2(n), basco(n), basb2(n);
    int64_t units = 0;
    int max_cols = 0;
    for (int k = 0; k < n; ++k) {
        Request& R = *S->reqs[S->active[k]];
        pd_mesh* m = R.mesh;
        BatchSlot& b = slots[k];
        b.tets = m->d_tets.p;
        b.geo = m->d_geo.p;
        b.x = m->d_x.p;
        b.xprev = m->d_xprev.p;
        b.v = m->d_v.p;
        b.by0 = m->d_by0.p;
        b.b = m->d_b.p;
        b.pin_tgt = m->d_pin_tgt.p;
        b.pin_rest = R.pin_rest.p;
        b.mh2 = m->d_mh2.p;
        b.kfp_ptr = m->d_kfp_ptr.p;
        b.kfp_col = m->d_kfp_col.p;
        b.kfp_val = m->d_kfp_val.p;
        b.tc = m->d_tc.p;
        b.cB = m->d_cB.p;
        b.part = m->d_part.p;
        b.gat_ptr = m->d_gat_ptr.p;
        b.gat = m->d_gat.p;
        b.err = m->d_err.p;
        b.frame = R.frame.p;
        b.la_vptr = m->d_la_vptr.p;
        b.la_vert = m->d_la_vert.p;
        b.la_slot = m->d_la_slot.p;
        b.la_cptr = m->d_la_cptr.p;
        b.la_corner = m->d_la_corner.p;
        b.la_sh_ptr = m->d_la_sh_ptr.p;
        b.la_sh_vert = m->d_la_sh_vert.p;
        b.la_part = m->d_la_part.p;
        b.la_shared = m->la_shared;
        b.two_level = m->two_level ? 1 : 0;
        b.n_top = m->two_level ? m->n_top : 0;
        b.gat2_ptr = m->d_gat2_ptr.p;
        b.gat2 = m->d_gat2.p;
        b.tc2 = m->d_tc2.p;
        b.cT = m->d_cT.p;
        b.n_t = m->n_t;
        b.n_v = m->n_v;
        b.n_free = m->n_free;
        b.n_pin = m->n_pin;
        b.n_int = m->n_int;
        b.n_B = m->n_B;
        b.nch = m->coarse_nchunks;
        b.h = (float)m->dt;
        b.gx = R.g[0];
        b.gy = R.g[1];
        b.gz = R.g[2];
        b.drive_amp = R.amp;
        b.drive_w = 2.0f * 3.14159265358979f * R.freq;
        b.drive_axis = R.axis;
        // (the fused local step: one block per plan block; the finish of the shared vertices)
        // (two levels: no partial sums to reduce, the second-level gather instead)
        const int cnt[PH_NB] = {(m->n_pin + 255) / 256, (m->n_v + 255) / 256, m->la_blocks,
                                (m->la_shared + 255) / 256, (m->n_B + 255) / 256,
                                m->two_level ? 0 : (m->n_B + 255) / 256, (m->n_v + 255) / 256,
                                m->two_level ? (m->n_top + 255) / 256 : 0};
        for (int p = 0; p < PH_NB; ++p) off[p][k + 1] = off[p][k] + cnt[p];
        const float* pool = m->d_mat32.p;
        basc[k] = AxBases{pool, m->d_b.p, nullptr, nullptr, m->d_tc.p};
        basb[k] = AxBases{pool, m->d_x.p + m->n_int, m->d_bidx.p, m->d_tc.p, m->d_x.p};
        // the meshes' products are tiled (bulk-copy layout): one block per output chunk of ld outputs
        for (AxDesc a : m->h_ax_desc_cond) {
            a.slot = k;
            for (int32_t o0 = 0; o0 < a.n_out; o0 += a.ld) blkc.push_back(AxBlock{(int32_t)axc.size(), o0});
            axc.push_back(a);
        }
        for (AxDesc a : m->h_ax_desc_back) {
            a.slot = k;
            for (int32_t o0 = 0; o0 < a.n_out; o0 += a.ld) blkb.push_back(AxBlock{(int32_t)axb.size(), o0});
            axb.push_back(a);
        }
        if (m->two_level) {
            // the single-mesh frame's second-level row plans, on this request's arrays
            const int T0 = m->n_B - m->n_top;
            basr2[k] = AxBases{pool, m->d_cB.p, nullptr, nullptr, m->d_tc2.p};
            basco[k] = AxBases{pool, m->d_cT.p, nullptr, nullptr, m->d_x.p + m->n_int + T0};
            basb2[k] = AxBases{pool, m->d_x.p + m->n_int + T0, m->d_bidx2.p, m->d_tc2.p, m->d_x.p + m->n_int};
            for (const RowPlan* P : {&m->rows_int2, &m->rows_cond2})
                for (RowDesc d : P->host) {
                    d.slot = k;
                    r2.push_back(d);
                }
            for (RowDesc d : m->rows_coarse.host) {
                d.slot = k;
                co.push_back(d);
            }
            for (RowDesc d : m->rows_back2.host) {
                d.slot = k;
                b2.push_back(d);
            }
        } else if (m->n_B > 0) {
            CoarseDescB c{};
            c.S = pool + m->off_S;
            c.cB = m->d_cB.p;
            c.part = m->d_part.p;
            c.u0 = units;
            c.n_B = m->n_B;
            c.ld = m->ld_S;
            c.nch = m->coarse_nchunks;
            cd.push_back(c);
            units += (int64_t)((m->n_B + 1) / 2) * m->coarse_nchunks;
            max_cols = std::max(max_cols, m->ld_S);
        }
    }
    put(S->d_slots, slots, S->stream);
    for (int p = 0; p < PH_NB; ++p) {
        put(S->d_off[p], off[p], S->stream);
        S->blocks[p] = off[p][n];
    }
    put(S->d_axc, axc, S->stream);
    put(S->d_axb, axb, S->stream);
    put(S->d_blkc, blkc, S->stream);
    put(S->d_blkb, blkb, S->stream);
    put(S->d_basc, basc, S->stream);
    put(S->d_basb, basb, S->stream);
    S->blocks_c = (int)blkc.size();
    S->blocks_b = (int)blkb.size();
    S->kmax_c = S->kmax_b = S->wmax_c = S->wmax_b = 1;
    for (const auto& a : axc) {
        S->kmax_c = std::max(S->kmax_c, a.K);
        S->wmax_c = std::max(S->wmax_c, a.ld);
    }
    for (const auto& a : axb) {
        S->kmax_b = std::max(S->kmax_b, a.K);
        S->wmax_b = std::max(S->wmax_b, a.ld);
    }
    put(S->d_cd, cd, S->stream);
    S->n_cd = (int)cd.size();
    put(S->d_basr2, basr2, S->stream);
    put(S->d_basco, basco, S->stream);
    put(S->d_basb2, basb2, S->stream);
    build_row_plan(S->rows_r2, r2, PD_PREC_FP32, S->stream, false);
    build_row_plan(S->rows_co, co, PD_PREC_FP32, S->stream, false);
    build_row_plan(S->rows_b2, b2, PD_PREC_FP32, S->stream, false);
    S->units = units;
    S->max_cols = max_cols;
    S->coarse_blocks = 0;
    if (units > 0) {
        if (!configure_coarse_b(max_cols)) throw Fail{PD_ERR_UNSUPPORTED};
        S->coarse_blocks = S->sms;
    }
    PDG_CUDA(cudaStreamSynchronize(S->stream));
    // capture one batched frame
    cudaGraph_t g = nullptr;
    cudaStream_t c = S->cap;
    PDG_CUDA(cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal));
    try {
        const BatchSlot* sl = S->d_slots.p;
        launch_b_drive(sl, S->d_off[PH_DRIVE].p, n, S->blocks[PH_DRIVE], c);
        launch_b_inertia(sl, S->d_off[PH_INER].p, n, S->blocks[PH_INER], c);
        for (int it = 0; it < S->n_iter; ++it) {
            launch_b_local_assemble(sl, S->d_off[PH_LOC].p, n, S->blocks[PH_LOC], c);
            launch_b_assemble_shared(sl, S->d_off[PH_ASM].p, n, S->blocks[PH_ASM], c);
            launch_axpy_b(S->d_axc.p, S->d_blkc.p, S->d_basc.p, S->blocks_c, S->kmax_c, S->wmax_c, S->d_err.p, c);
            launch_b_gather(sl, S->d_off[PH_GAT].p, n, S->blocks[PH_GAT], c);
            launch_rowdot_b(S->rows_r2, S->d_basr2.p, S->d_err.p, c);
            launch_b_gather2(sl, S->d_off[PH_GAT2].p, n, S->blocks[PH_GAT2], c);
            if (S->n_cd > 0) launch_coarse_b(S->d_cd.p, S->n_cd, S->units, S->max_cols, S->coarse_blocks, c);
            launch_rowdot_b(S->rows_co, S->d_basco.p, S->d_err.p, c);
            launch_b_reduce(sl, S->d_off[PH_RED].p, n, S->blocks[PH_RED], c);
            launch_rowdot_b(S->rows_b2, S->d_basb2.p, S->d_err.p, c);
            launch_axpy_b(S->d_axb.p, S->d_blkb.p, S->d_basb.p, S->blocks_b, S->kmax_b, S->wmax_b, S->d_err.p, c);
        }
        launch_b_velocity(sl, S->d_off[PH_VEL].p, n, S->blocks[PH_VEL], c);
    } catch (...) {
        cudaStreamEndCapture(c, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    PDG_CUDA(cudaStreamEndCapture(c, &g));
    cudaError_t e = cudaGraphInstantiate(&S->graph, g, 0);
    cudaGraphDestroy(g);
    PDG_CUDA(e);
}

// ---------------------------------------------------------------- admission workers
constexpr int kAdmissionWorkers = 4;

// Takes the request at the head of the queue and builds and prefactors it on
// the admission stream when the budget and the slots allow.  Under lk except
// while it works on the host or the device.  A request that must wait for
// memory goes back to the head of the queue.
static void prepare_head(pd_server* S, std::unique_lock<std::mutex>& lk, cudaStream_t adm) {
    AllocStreamScope alloc_scope(adm);   // the request's own buffers: allocated and freed on its admission stream
    const pd_request_id id = S->queue.front();
    Request& R = *S->reqs[id];
    auto nothing_resident = [&]() {
        return S->n_active == 0 && S->ready.empty() && S->retired.empty() && S->n_preparing == 0;
    };
    auto fail_it = [&]() {
        R.state = PD_REQ_FAILED;
        S->cv_ready.notify_all();
    };
    // a request seen before waits on its cached estimate without being rebuilt
    if (R.estimated && S->used + S->reserved + R.est_steady + R.est_transient > S->budget) {
        if (nothing_resident()) {
            S->queue.pop_front();
            fail_it();   // it can never fit
        }
        return;
    }
    S->queue.pop_front();
    ++S->n_preparing;
    lk.unlock();
    pd_mesh* m = nullptr;
    pd_status st = pd_create_mesh(R.rest.data(), R.n_v, R.tets.data(), R.n_t, nullptr, R.density,
                                  R.dom.empty() ? nullptr : R.dom.data(), R.n_dom,
                                  R.pinned.empty() ? nullptr : R.pinned.data(), adm, &m);
    int64_t steady = 0, transient = 0;
    if (st == PD_OK) estimate(m, steady, transient);
    lk.lock();
    if (st != PD_OK) {
        --S->n_preparing;
        fail_it();
        return;
    }
    R.estimated = true;
    R.est_steady = steady;
    R.est_transient = transient;
    if (S->used + S->reserved + steady + transient > S->budget) {
        --S->n_preparing;
        const bool never = nothing_resident();
        lk.unlock();
        pd_destroy_mesh(m);
        lk.lock();
        if (never) fail_it();
        else S->queue.push_front(id);   // waits at the head for memory
        S->cv.notify_all();
        return;
    }
    S->reserved += steady + transient;
    S->peak = std::max(S->peak, S->used + S->reserved);
    lk.unlock();
    st = pd_set_materials(m, R.gs.data(), R.gv.data());
    // FP32; two interface levels where the prefactorisation chooses them and the batched
    // row-form kernels can stream their rows (every row within one stage), else one level
    pd_solver_opts o{PD_PREC_FP32, 0, 0, 0};
    m->batched_only = true;   // the serving loop runs its own batched kernels: no streaming copies
    if (st == PD_OK) {
        // the FP64 factorisation shares the GPU with the resident requests' frames: one at a time
        std::lock_guard<std::mutex> pk(S->prefactor_mu);
        st = pd_prefactor(m, R.dt, &o);
        auto streamable = [](const RowPlan& P) { return P.n_blocks == 0 || P.tma; };
        if (st == PD_OK && m->two_level &&
            !(m->rows_coarse.n_blocks > 0 && streamable(m->rows_coarse) && streamable(m->rows_int2) &&
              streamable(m->rows_cond2) && streamable(m->rows_back2))) {
            o.flags = PD_SOLVE_SINGLE_LEVEL;
            st = pd_prefactor(m, R.dt, &o);
        }
    }
    if (st == PD_OK) {
        try {
            // pinned rest positions (increasing vertex id) and the frame counter
            std::vector<float4> pr;
            for (int32_t v = 0; v < R.n_v; ++v)
                if (!R.pinned.empty() && R.pinned[v])
                    pr.push_back(make_float4((float)R.rest[3 * (size_t)v], (float)R.rest[3 * (size_t)v + 1],
                                             (float)R.rest[3 * (size_t)v + 2], 0.f));
            R.pin_rest.alloc(std::max<size_t>(pr.size(), 1));
            if (!pr.empty())
                PDG_CUDA(cudaMemcpyAsync(R.pin_rest.p, pr.data(), pr.size() * sizeof(float4),
                                         cudaMemcpyHostToDevice, adm));
            R.frame.alloc(1);
            PDG_CUDA(cudaMemsetAsync(R.frame.p, 0, sizeof(int32_t), adm));
            PDG_CUDA(cudaStreamSynchronize(adm));
        } catch (const Fail& f) {
            st = f.code;
        } catch (const std::bad_alloc&) {
            st = PD_ERR_NO_MEMORY;
        }
    }
    if (st != PD_OK) {
        R.pin_rest.free();
        R.frame.free();
        pd_destroy_mesh(m);
        lk.lock();
        --S->n_preparing;
        S->reserved -= steady + transient;
        fail_it();
        S->cv.notify_all();
        return;
    }
    lk.lock();
    --S->n_preparing;
    S->reserved -= steady + transient;
    S->used += steady;
    R.mesh = m;
    R.steady_bytes = steady;
    R.t_last = Clock::now();
    S->ready.push_back(id);
    S->cv_ready.notify_all();
    S->cv.notify_all();
}

static void worker_main(pd_server* S, int index) {
    cudaSetDevice(S->device);
    cudaStream_t adm = S->adm_streams[index];
    std::unique_lock<std::mutex> lk(S->mu);
    uint64_t seen_gen = ~uint64_t(0);
    for (;;) {
        // free the meshes the tick thread retired (worker 0)
        while (index == 0 && !S->retired.empty()) {
            std::vector<std::pair<pd_mesh*, int64_t>> dead;
            dead.swap(S->retired);
            lk.unlock();
            for (auto& d : dead) pd_destroy_mesh(d.first);
            lk.lock();
            for (auto& d : dead) S->used -= d.second;   // returned to the budget once actually freed
            ++S->freed_gen;
            S->cv.notify_all();
        }
        if (S->stop) break;
        const bool slot_free = S->n_active + (int32_t)S->ready.size() + S->n_preparing < S->max_slots;
        if (!S->queue.empty() && slot_free) {
            const Request& R = *S->reqs[S->queue.front()];
            // a request waiting on the budget is retried only after memory was returned
            if (!(R.estimated && seen_gen == S->freed_gen &&
                  S->used + S->reserved + R.est_steady + R.est_transient > S->budget)) {
                seen_gen = S->freed_gen;
                prepare_head(S, lk, adm);
                continue;
            }
        }
        S->cv.wait(lk);
    }
}

extern "C" {

pd_status pd_server_create(int64_t hbm_budget_bytes, int32_t max_slots, int32_t n_iter, void* stream,
                           pd_server** out) {
    if (!out || hbm_budget_bytes <= 0 || max_slots < 1 || max_slots > 1024 || n_iter < 1 || n_iter > 1000)
        return sfail(PD_ERR_INVALID_ARG, "bad server arguments");
    *out = nullptr;
    pd_server* S = new (std::nothrow) pd_server();
    if (!S) return sfail(PD_ERR_NO_MEMORY, "host allocation failed");
    try {
        S->budget = hbm_budget_bytes;
        S->max_slots = max_slots;
        S->n_iter = n_iter;
        S->user = static_cast<cudaStream_t>(stream);
        PDG_CUDA(cudaGetDevice(&S->device));
        PDG_CUDA(cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking));
        int prio_low = 0, prio_high = 0;
        PDG_CUDA(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
        // the frames ahead of the admission work (FP64 prefactorisations) whenever an SM frees up
        PDG_CUDA(cudaStreamCreateWithPriority(&S->frame_stream.s, cudaStreamNonBlocking, prio_high));
        S->stream = S->frame_stream.s;
        PDG_CUDA(cudaEventCreateWithFlags(&S->e_user, cudaEventDisableTiming));
        PDG_CUDA(cudaMallocHost((void**)&S->h_err, sizeof(int32_t)));
        *S->h_err = 0;
        AllocStreamScope alloc_scope(S->stream);
        PDG_CUDA(cudaStreamCreateWithPriority(&S->adm, cudaStreamNonBlocking, prio_low));
        S->adm_streams.assign(kAdmissionWorkers, nullptr);
        for (auto& st : S->adm_streams) PDG_CUDA(cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio_low));
        PDG_CUDA(cudaEventCreate(&S->e0));
        PDG_CUDA(cudaEventCreate(&S->e1));
        PDG_CUDA(cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->device));
        S->d_err.alloc(1);
        PDG_CUDA(cudaMemsetAsync(S->d_err.p, 0, sizeof(int32_t), S->stream));
        PDG_CUDA(cudaStreamSynchronize(S->stream));
        for (int k = 0; k < kAdmissionWorkers; ++k) S->workers.emplace_back(worker_main, S, k);
    } catch (const Fail& f) {
        delete S;
        return f.code;
    } catch (const std::system_error&) {
        delete S;
        return sfail(PD_ERR_NO_MEMORY, "could not start the admission thread");
    }
    *out = S;
    return PD_OK;
}

void pd_server_destroy(pd_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    for (auto& t : S->workers)
        if (t.joinable()) t.join();
    cudaStreamSynchronize(S->stream);
    for (auto& d : S->retired) pd_destroy_mesh(d.first);
    S->retired.clear();
    S->reqs.clear();   // resident and prepared meshes, while their streams still exist
    delete S;
}

pd_status pd_submit(pd_server* S, const pd_request* q, pd_request_id* id) {
    if (!S || !q || !id || !q->rest_xyz || !q->tets || !q->gamma_s || !q->gamma_v || q->n_v <= 0 || q->n_t <= 0 ||
        q->n_frames < 1 || !(q->dt > 0.0) || q->n_domains <= 0)
        return sfail(PD_ERR_INVALID_ARG, "bad request");
    try {
        auto R = std::make_unique<Request>();
        R->n_v = q->n_v;
        R->n_t = q->n_t;
        R->n_dom = q->n_domains;
        R->rest.assign(q->rest_xyz, q->rest_xyz + 3 * (size_t)q->n_v);
        R->tets.assign(q->tets, q->tets + 4 * (size_t)q->n_t);
        if (q->tet_domain) R->dom.assign(q->tet_domain, q->tet_domain + q->n_t);
        if (q->pinned) R->pinned.assign(q->pinned, q->pinned + q->n_v);
        R->gs.assign(q->gamma_s, q->gamma_s + q->n_t);
        R->gv.assign(q->gamma_v, q->gamma_v + q->n_t);
        R->density = q->density;
        R->dt = q->dt;
        R->n_frames = q->n_frames;
        for (int k = 0; k < 3; ++k) R->g[k] = q->gravity[k];
        R->amp = q->drive_amp;
        R->freq = q->drive_freq;
        R->axis = q->drive_axis;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            R->id = S->next_id++;
            *id = R->id;
            S->queue.push_back(R->id);
            S->reqs[R->id] = std::move(R);
        }
        S->cv.notify_all();
    } catch (const std::bad_alloc&) {
        return sfail(PD_ERR_NO_MEMORY, "host allocation failed");
    }
    return PD_OK;
}

pd_status pd_server_tick(pd_server* S, int32_t* n_active, float* frame_ms) {
    if (!S) return sfail(PD_ERR_INVALID_ARG, "server is NULL");
    try {
        AllocStreamScope alloc_scope(S->stream);   // the batch descriptors: allocated and freed on the frame stream
        // this tick after the caller's prior work on its own stream.  Not on the legacy
        // default stream: an event recorded there waited 12-50 ms for the driver while an
        // admission thread was inside a prefactorisation (requests and results are host
        // arrays, so the frames need no ordering with it).
        if (S->user) {
            PDG_CUDA(cudaEventRecord(S->e_user, S->user));
            PDG_CUDA(cudaStreamWaitEvent(S->stream, S->e_user, 0));
        }
        // retire finished requests: read back their positions, hand their meshes to the worker
        std::vector<std::pair<pd_mesh*, int64_t>> dead;
        for (size_t k = 0; k < S->active.size();) {
            Request* R;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                R = S->reqs[S->active[k]].get();
            }
            if (R->frames_done >= R->n_frames) {
                const size_t n3 = 3 * (size_t)R->n_v;
                R->x_final.resize(n3);
                if (n3 > S->d_out.n) S->d_out.alloc(std::max(n3, 2 * S->d_out.n));
                launch_scatter_out(R->mesh, R->mesh->d_x.p, S->d_out.p, 0, S->stream);
                PDG_CUDA(cudaMemcpyAsync(R->x_final.data(), S->d_out.p, sizeof(float) * n3, cudaMemcpyDeviceToHost,
                                         S->stream));
                PDG_CUDA(cudaStreamSynchronize(S->stream));
                std::lock_guard<std::mutex> lk(S->mu);
                dead.emplace_back(R->mesh, R->steady_bytes);
                R->mesh = nullptr;
                R->state = PD_REQ_DONE;
                S->active.erase(S->active.begin() + k);
                S->n_active = (int32_t)S->active.size();
                S->dirty = true;
            } else {
                ++k;
            }
        }
        bool wait_for_ready = false;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (auto& d : dead) S->retired.push_back(d);
            // nothing to run yet but requests on their way: wait (bounded) for the first to be ready
            wait_for_ready = S->active.empty() && S->ready.empty() && (!S->queue.empty() || S->n_preparing > 0);
            if (wait_for_ready) {
                S->cv.notify_all();
                S->cv_ready.wait_for(lk, std::chrono::milliseconds(5));
            }
            // requests prepared by the worker join the batch
            while (!S->ready.empty()) {
                const pd_request_id id = S->ready.front();
                S->ready.pop_front();
                S->reqs[id]->state = PD_REQ_ACTIVE;
                S->active.push_back(id);
                S->dirty = true;
            }
            S->n_active = (int32_t)S->active.size();
        }
        S->cv.notify_all();   // slots or memory may have been returned
        if (S->dirty) rebuild(S);
        if (n_active) *n_active = (int32_t)S->active.size();
        float ms = 0.f;
        if (!S->active.empty() && S->graph) {
            PDG_CUDA(cudaEventRecord(S->e0, S->stream));
            PDG_CUDA(cudaGraphLaunch(S->graph, S->stream));
            PDG_CUDA(cudaEventRecord(S->e1, S->stream));
            PDG_CUDA(cudaMemcpyAsync(S->h_err, S->d_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, S->stream));
            PDG_CUDA(cudaStreamSynchronize(S->stream));
            PDG_CUDA(cudaEventElapsedTime(&ms, S->e0, S->e1));
            const auto now = Clock::now();
            std::lock_guard<std::mutex> lk(S->mu);
            for (auto id : S->active) {
                Request& R = *S->reqs[id];
                R.frames_done++;
                R.frame_ms.push_back(std::chrono::duration<float, std::milli>(now - R.t_last).count());
                R.t_last = now;
            }
        }
        if (frame_ms) *frame_ms = ms;
        if (*S->h_err) {
            *S->h_err = 0;
            PDG_CUDA(cudaMemsetAsync(S->d_err.p, 0, sizeof(int32_t), S->stream));
            PDG_CUDA(cudaStreamSynchronize(S->stream));
            return sfail(PD_ERR_TIMEOUT, "pd_server_tick: a bounded wait of the batched products ran out");
        }
    } catch (const Fail& f) {
        return f.code;
    } catch (const std::bad_alloc&) {
        return sfail(PD_ERR_NO_MEMORY, "pd_server_tick: host allocation failed");
    } catch (...) {
        return sfail(PD_ERR_CUDA, "pd_server_tick: unexpected host exception");
    }
    return PD_OK;
}

static bool outstanding(pd_server* S) {
    std::lock_guard<std::mutex> lk(S->mu);
    return !S->queue.empty() || !S->ready.empty() || S->n_preparing > 0 || !S->active.empty();
}

pd_status pd_server_run(pd_server* S, int32_t max_ticks, int32_t* ticks) {
    if (!S) return sfail(PD_ERR_INVALID_ARG, "server is NULL");
    if (max_ticks < 1) return sfail(PD_ERR_INVALID_ARG, "max_ticks must be >= 1");
    int32_t t = 0;
    for (; t < max_ticks && outstanding(S); ++t) {
        const pd_status st = pd_server_tick(S, nullptr, nullptr);
        if (st != PD_OK) {
            if (ticks) *ticks = t;
            return st;
        }
    }
    if (ticks) *ticks = t;
    if (outstanding(S))
        return sfail(PD_ERR_TIMEOUT, "pd_server_run: max_ticks ticks ran and requests are still queued or resident");
    return PD_OK;
}

pd_status pd_poll(pd_server* S, pd_request_id id, int32_t* state, int32_t* frames_done) {
    if (!S) return sfail(PD_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return sfail(PD_ERR_INVALID_ARG, "unknown request id");
    if (state) *state = it->second->state;
    if (frames_done) *frames_done = it->second->frames_done;
    return PD_OK;
}

pd_status pd_fetch(pd_server* S, pd_request_id id, float* x_out, float* frame_ms) {
    if (!S) return sfail(PD_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return sfail(PD_ERR_INVALID_ARG, "unknown request id");
    Request& R = *it->second;
    if (R.state != PD_REQ_DONE) return sfail(PD_ERR_INVALID_ARG, "request not done");
    if (x_out) std::copy(R.x_final.begin(), R.x_final.end(), x_out);
    if (frame_ms) std::copy(R.frame_ms.begin(), R.frame_ms.end(), frame_ms);
    return PD_OK;
}

pd_status pd_release(pd_server* S, pd_request_id id) {
    if (!S) return sfail(PD_ERR_INVALID_ARG, "server is NULL");
    std::unique_ptr<Request> gone;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(id);
        if (it == S->reqs.end()) return sfail(PD_ERR_INVALID_ARG, "unknown request id");
        if (it->second->state == PD_REQ_ACTIVE || it->second->state == PD_REQ_QUEUED)
            return sfail(PD_ERR_INVALID_ARG, "request still queued or active");
        gone = std::move(it->second);
        S->reqs.erase(it);
    }
    return PD_OK;
}

pd_status pd_server_stats(pd_server* S, int32_t* n_queued, int32_t* n_active, int64_t* used_bytes,
                          int64_t* peak_bytes) {
    if (!S) return sfail(PD_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    if (n_queued) *n_queued = (int32_t)S->queue.size() + S->n_preparing;
    if (n_active) *n_active = (int32_t)(S->active.size() + S->ready.size());
    if (used_bytes) *used_bytes = S->used;
    if (peak_bytes) *peak_bytes = S->peak;
    return PD_OK;
}

}  // extern "C"
