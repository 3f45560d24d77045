// Serving loop of the C ABI: requests (one garment mesh each) are admitted
// while the HBM budget allows, stay resident on the device, and advance one
// frame per pd_server_tick in shared batched launches (one CUDA graph per
// set of resident requests).  Requests that arrive while others run are
// admitted at the next tick as memory and slots free up.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <memory>
#include <vector>

#include "pd_internal.h"

namespace pdg {

void launch_b_drive(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s);
void launch_b_inertia(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s);
void launch_b_local(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s);
void launch_b_assemble(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s);
void launch_b_gather(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s);
void launch_b_reduce(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s);
void launch_b_velocity(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s);
void launch_axpy_b(const AxDesc* descs, const AxBlock* blocks, const AxBases* bases, int n_blocks, int k_max,
                   cudaStream_t s);
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
    std::vector<float> frame_ms, x_final;
    ~Request() {
        if (mesh) pd_destroy_mesh(mesh);
    }
};

enum { PH_DRIVE = 0, PH_INER, PH_LOC, PH_ASM, PH_GAT, PH_RED, PH_VEL, PH_NB };

}  // namespace

struct pd_server {
    int64_t budget = 0;
    int32_t max_slots = 0, n_iter = 20;
    cudaStream_t stream = nullptr, cap = nullptr;
    pd_request_id next_id = 1;
    std::map<pd_request_id, std::unique_ptr<Request>> reqs;
    std::deque<pd_request_id> queue;
    std::vector<pd_request_id> active;
    int64_t used = 0, peak = 0;
    bool dirty = true;
    cudaGraphExec_t graph = nullptr;
    int sms = 0;
    // batch descriptors
    DBuf<BatchSlot> d_slots;
    DBuf<int32_t> d_off[PH_NB];
    int blocks[PH_NB] = {0};
    DBuf<AxDesc> d_axc, d_axb;
    DBuf<AxBlock> d_blkc, d_blkb;
    DBuf<AxBases> d_basc, d_basb;
    int blocks_c = 0, blocks_b = 0, kmax_c = 1, kmax_b = 1;
    DBuf<CoarseDescB> d_cd;
    int n_cd = 0, max_cols = 0, coarse_blocks = 0;
    int64_t units = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~pd_server() {
        if (graph) cudaGraphExecDestroy(graph);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (cap) cudaStreamDestroy(cap);
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
    int64_t units = 0;
    const int OW = ax_outputs_per_block(PD_PREC_FP32);
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
        b.force = m->d_force.p;
        b.by0 = m->d_by0.p;
        b.b = m->d_b.p;
        b.pin_tgt = m->d_pin_tgt.p;
        b.pin_rest = R.pin_rest.p;
        b.mh2 = m->d_mh2.p;
        b.inc_ptr = m->d_inc_ptr.p;
        b.inc = m->d_inc.p;
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
        const int cnt[PH_NB] = {(m->n_pin + 255) / 256, (m->n_v + 255) / 256, (m->n_t + 127) / 128,
                                (m->n_free + 255) / 256, (m->n_B + 255) / 256, (m->n_B + 255) / 256,
                                (m->n_v + 255) / 256};
        for (int p = 0; p < PH_NB; ++p) off[p][k + 1] = off[p][k] + cnt[p];
        const float* pool = m->d_mat32.p;
        basc[k] = AxBases{pool, m->d_b.p, nullptr, nullptr, m->d_tc.p};
        basb[k] = AxBases{pool, m->d_x.p + m->n_int, m->d_bidx.p, m->d_tc.p, m->d_x.p};
        for (AxDesc a : m->h_ax_desc_cond) {
            a.slot = k;
            const int32_t cw = a.tiled ? a.ld : OW;   // tiled: one block per chunk of ld outputs
            for (int32_t o0 = 0; o0 < a.n_out; o0 += cw) blkc.push_back(AxBlock{(int32_t)axc.size(), o0});
            axc.push_back(a);
        }
        for (AxDesc a : m->h_ax_desc_back) {
            a.slot = k;
            const int32_t cw = a.tiled ? a.ld : OW;
            for (int32_t o0 = 0; o0 < a.n_out; o0 += cw) blkb.push_back(AxBlock{(int32_t)axb.size(), o0});
            axb.push_back(a);
        }
        if (m->n_B > 0) {
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
    auto up = [&](auto& dbuf, const auto& h) {
        dbuf.alloc(h.size());
        if (!h.empty())
            PDG_CUDA(cudaMemcpyAsync(dbuf.p, h.data(), h.size() * sizeof(h[0]), cudaMemcpyHostToDevice, S->stream));
    };
    up(S->d_slots, slots);
    for (int p = 0; p < PH_NB; ++p) {
        up(S->d_off[p], off[p]);
        S->blocks[p] = off[p][n];
    }
    up(S->d_axc, axc);
    up(S->d_axb, axb);
    up(S->d_blkc, blkc);
    up(S->d_blkb, blkb);
    up(S->d_basc, basc);
    up(S->d_basb, basb);
    S->blocks_c = (int)blkc.size();
    S->blocks_b = (int)blkb.size();
    S->kmax_c = S->kmax_b = 1;
    for (const auto& a : axc) S->kmax_c = std::max(S->kmax_c, a.K);
    for (const auto& a : axb) S->kmax_b = std::max(S->kmax_b, a.K);
    up(S->d_cd, cd);
    S->n_cd = (int)cd.size();
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
            launch_b_local(sl, S->d_off[PH_LOC].p, n, S->blocks[PH_LOC], c);
            launch_b_assemble(sl, S->d_off[PH_ASM].p, n, S->blocks[PH_ASM], c);
            launch_axpy_b(S->d_axc.p, S->d_blkc.p, S->d_basc.p, S->blocks_c, S->kmax_c, c);
            launch_b_gather(sl, S->d_off[PH_GAT].p, n, S->blocks[PH_GAT], c);
            launch_coarse_b(S->d_cd.p, S->n_cd, S->units, S->max_cols, S->coarse_blocks, c);
            launch_b_reduce(sl, S->d_off[PH_RED].p, n, S->blocks[PH_RED], c);
            launch_axpy_b(S->d_axb.p, S->d_blkb.p, S->d_basb.p, S->blocks_b, S->kmax_b, c);
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

// Admits the request at the head of the queue if the budget allows.  Returns
// true when the request leaves the queue (admitted, or failed: it can never
// fit, or its mesh or factorisation failed), false when it must wait for
// resident requests to retire.
static bool admit(pd_server* S, Request& R) {
    // a request seen before waits on its cached estimate without being rebuilt
    if (R.estimated && S->used + R.est_steady + R.est_transient > S->budget) {
        if (!S->active.empty()) return false;
        R.state = PD_REQ_FAILED;
        return true;
    }
    pd_mesh* m = nullptr;
    pd_status st = pd_create_mesh(R.rest.data(), R.n_v, R.tets.data(), R.n_t, nullptr, R.density,
                                  R.dom.empty() ? nullptr : R.dom.data(), R.n_dom,
                                  R.pinned.empty() ? nullptr : R.pinned.data(), S->stream, &m);
    if (st != PD_OK) {
        R.state = PD_REQ_FAILED;
        return true;
    }
    R.mesh = m;   // owned by the request from here on (destroyed with it on any failure)
    int64_t steady = 0, transient = 0;
    estimate(m, steady, transient);
    R.estimated = true;
    R.est_steady = steady;
    R.est_transient = transient;
    if (S->used + steady + transient > S->budget) {
        pd_destroy_mesh(m);
        R.mesh = nullptr;
        if (!S->active.empty()) return false;   // waits for resident requests to retire
        // nothing is resident and it still does not fit: it never will
        R.state = PD_REQ_FAILED;
        return true;
    }
    st = pd_set_materials(m, R.gs.data(), R.gv.data());
    pd_solver_opts o{PD_PREC_FP32, 0, 0, PD_SOLVE_SINGLE_LEVEL};  // the batched coarse kernel is single-level
    m->batched_only = true;   // the serving loop runs its own batched kernels: no streaming copies
    if (st == PD_OK) st = pd_prefactor(m, R.dt, &o);
    if (st != PD_OK) {
        pd_destroy_mesh(m);
        R.mesh = nullptr;
        R.state = PD_REQ_FAILED;
        return true;
    }
    R.steady_bytes = steady;
    S->peak = std::max(S->peak, S->used + steady + transient);
    S->used += steady;
    R.state = PD_REQ_ACTIVE;   // resident: retired (and its bytes returned) like any other from here on
    // pinned rest positions (increasing vertex id) and the frame counter
    std::vector<float4> pr;
    for (int32_t v = 0; v < R.n_v; ++v)
        if (!R.pinned.empty() && R.pinned[v])
            pr.push_back(make_float4((float)R.rest[3 * (size_t)v], (float)R.rest[3 * (size_t)v + 1],
                                     (float)R.rest[3 * (size_t)v + 2], 0.f));
    R.pin_rest.alloc(std::max<size_t>(pr.size(), 1));
    if (!pr.empty())
        PDG_CUDA(cudaMemcpyAsync(R.pin_rest.p, pr.data(), pr.size() * sizeof(float4), cudaMemcpyHostToDevice,
                                 S->stream));
    R.frame.alloc(1);
    PDG_CUDA(cudaMemsetAsync(R.frame.p, 0, sizeof(int32_t), S->stream));
    return true;
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
        S->stream = static_cast<cudaStream_t>(stream);
        PDG_CUDA(cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking));
        PDG_CUDA(cudaEventCreate(&S->e0));
        PDG_CUDA(cudaEventCreate(&S->e1));
        int dev = 0;
        PDG_CUDA(cudaGetDevice(&dev));
        PDG_CUDA(cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, dev));
    } catch (const Fail& f) {
        delete S;
        return f.code;
    }
    *out = S;
    return PD_OK;
}

void pd_server_destroy(pd_server* S) {
    if (!S) return;
    cudaStreamSynchronize(S->stream);
    delete S;
}

pd_status pd_submit(pd_server* S, const pd_request* q, pd_request_id* id) {
    if (!S || !q || !id || !q->rest_xyz || !q->tets || !q->gamma_s || !q->gamma_v || q->n_v <= 0 || q->n_t <= 0 ||
        q->n_frames < 1 || !(q->dt > 0.0) || q->n_domains <= 0)
        return sfail(PD_ERR_INVALID_ARG, "bad request");
    try {
        auto R = std::make_unique<Request>();
        R->id = S->next_id++;
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
        *id = R->id;
        S->queue.push_back(R->id);
        S->reqs[R->id] = std::move(R);
    } catch (const std::bad_alloc&) {
        return sfail(PD_ERR_NO_MEMORY, "host allocation failed");
    }
    return PD_OK;
}

pd_status pd_server_tick(pd_server* S, int32_t* n_active, float* frame_ms) {
    if (!S) return sfail(PD_ERR_INVALID_ARG, "server is NULL");
    try {
        // retire finished requests
        for (size_t k = 0; k < S->active.size();) {
            Request& R = *S->reqs[S->active[k]];
            if (R.frames_done >= R.n_frames) {
                R.x_final.resize(3 * (size_t)R.n_v);
                DBuf<float> tmp;
                tmp.alloc(3 * (size_t)R.n_v);
                launch_scatter_out(R.mesh, R.mesh->d_x.p, tmp.p, 0, S->stream);
                PDG_CUDA(cudaMemcpyAsync(R.x_final.data(), tmp.p, sizeof(float) * 3 * R.n_v, cudaMemcpyDeviceToHost,
                                         S->stream));
                PDG_CUDA(cudaStreamSynchronize(S->stream));
                pd_destroy_mesh(R.mesh);
                R.mesh = nullptr;
                R.pin_rest.free();
                R.frame.free();
                S->used -= R.steady_bytes;
                R.state = PD_REQ_DONE;
                S->active.erase(S->active.begin() + k);
                S->dirty = true;
            } else {
                ++k;
            }
        }
        // admit in arrival order while slots and memory allow
        while (!S->queue.empty() && (int)S->active.size() < S->max_slots) {
            Request& R = *S->reqs[S->queue.front()];
            if (!admit(S, R)) break;
            S->queue.pop_front();
            if (R.state == PD_REQ_ACTIVE) {
                S->active.push_back(R.id);
                S->dirty = true;
            }
        }
        if (S->dirty) rebuild(S);
        if (n_active) *n_active = (int32_t)S->active.size();
        float ms = 0.f;
        if (!S->active.empty() && S->graph) {
            PDG_CUDA(cudaEventRecord(S->e0, S->stream));
            PDG_CUDA(cudaGraphLaunch(S->graph, S->stream));
            PDG_CUDA(cudaEventRecord(S->e1, S->stream));
            PDG_CUDA(cudaEventSynchronize(S->e1));
            PDG_CUDA(cudaEventElapsedTime(&ms, S->e0, S->e1));
            for (auto id : S->active) {
                Request& R = *S->reqs[id];
                R.frames_done++;
                R.frame_ms.push_back(ms);
            }
        }
        if (frame_ms) *frame_ms = ms;
    } catch (const Fail& f) {
        return f.code;
    } catch (const std::bad_alloc&) {
        return sfail(PD_ERR_NO_MEMORY, "pd_server_tick: host allocation failed");
    } catch (...) {
        return sfail(PD_ERR_CUDA, "pd_server_tick: unexpected host exception");
    }
    return PD_OK;
}

pd_status pd_server_run(pd_server* S, int32_t max_ticks, int32_t* ticks) {
    if (!S) return sfail(PD_ERR_INVALID_ARG, "server is NULL");
    if (max_ticks < 1) return sfail(PD_ERR_INVALID_ARG, "max_ticks must be >= 1");
    int32_t t = 0;
    for (; t < max_ticks && (!S->queue.empty() || !S->active.empty()); ++t) {
        const pd_status st = pd_server_tick(S, nullptr, nullptr);
        if (st != PD_OK) {
            if (ticks) *ticks = t;
            return st;
        }
    }
    if (ticks) *ticks = t;
    if (!S->queue.empty() || !S->active.empty())
        return sfail(PD_ERR_TIMEOUT, "pd_server_run: max_ticks ticks ran and requests are still queued or resident");
    return PD_OK;
}

pd_status pd_poll(pd_server* S, pd_request_id id, int32_t* state, int32_t* frames_done) {
    if (!S) return sfail(PD_ERR_INVALID_ARG, "server is NULL");
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return sfail(PD_ERR_INVALID_ARG, "unknown request id");
    if (state) *state = it->second->state;
    if (frames_done) *frames_done = it->second->frames_done;
    return PD_OK;
}

pd_status pd_fetch(pd_server* S, pd_request_id id, float* x_out, float* frame_ms) {
    if (!S) return sfail(PD_ERR_INVALID_ARG, "server is NULL");
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
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return sfail(PD_ERR_INVALID_ARG, "unknown request id");
    if (it->second->state == PD_REQ_ACTIVE || it->second->state == PD_REQ_QUEUED)
        return sfail(PD_ERR_INVALID_ARG, "request still queued or active");
    S->reqs.erase(it);
    return PD_OK;
}

pd_status pd_server_stats(pd_server* S, int32_t* n_queued, int32_t* n_active, int64_t* used_bytes,
                          int64_t* peak_bytes) {
    if (!S) return sfail(PD_ERR_INVALID_ARG, "server is NULL");
    if (n_queued) *n_queued = (int32_t)S->queue.size();
    if (n_active) *n_active = (int32_t)S->active.size();
    if (used_bytes) *used_bytes = S->used;
    if (peak_bytes) *peak_bytes = S->peak;
    return PD_OK;
}

}  // extern "C"
