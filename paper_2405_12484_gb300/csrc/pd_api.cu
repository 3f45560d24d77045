// C ABI of libpdgb300: mesh set-up, prefactorisation orchestration, frame
// stepping with CUDA graphs, diagnostics.  Declarations and argument
// contracts are in include/pd.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <utility>

#include "pd_internal.h"

namespace pdg {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

// defined in the kernel translation units
void launch_weights_raw(int n_t, const float* vol, const float* gs, const float* gv, float4* geo, cudaStream_t s);
void dense_spd_inverse(double* A, int n, int lda, int64_t sA, double* X, int ldx, int64_t sX, int batch, int* d_err,
                       cudaStream_t s);
int dense_block();
int dd_max_sub_cols();
int dd_coarse_chunk();
int dd_configure_coarse(int ld_S);
int ax_outputs_per_block(int prec);
int ax_tile_outputs(int prec);
void build_row_plan(RowPlan& P, std::vector<RowDesc> descs, int prec, cudaStream_t s, bool mma = false);
bool rowdot_mma_fits(int xcap);
bool rowdot_row_fits_stage(int ld, int elem_bytes);
void launch_cast_frag32(const double* src, int lds, int rows, int cols, int transpose, float* dst32,
                        int64_t dst_off, int CW, cudaStream_t s);
void launch_cast_rowfrag16(const double* src, int lds, int rows, int cols, int transpose, __nv_bfloat16* dst16,
                           int64_t dst_off, int Kp, cudaStream_t s);
bool build_stream_plan(StreamPlan& P, const std::vector<ColDesc>& blocks, int prec, const void* src,
                       cudaStream_t s);
void reset_stream_plan(StreamPlan& P, cudaStream_t s);
void launch_prefactor_helpers_scatter_coo(double* S, int ld, const int* r, const int* c, const double* v, int n,
                                          cudaStream_t s);
void launch_prefactor_add_block(double* S, int ldS, const double* Sd, int ldSd, const int* bidx, int nb,
                                cudaStream_t s);
void launch_cast_block(const double* src, int lds, int rows, int cols, int transpose, int prec, float* dst32,
                       __nv_bfloat16* dst16, int64_t dst_off, int ldd, cudaStream_t s);
void launch_cast_frag16(const double* src, int lds, int rows, int cols, int transpose, __nv_bfloat16* dst16,
                        int64_t dst_off, int CW, cudaStream_t s);
void launch_cast_tiled(const double* src, int lds, int rows, int cols, int transpose, int prec, float* dst32,
                       __nv_bfloat16* dst16, int64_t dst_off, int OW, int VN, cudaStream_t s);
void ax_prepare_tma(int prec);
void test_set_copy_extra(int bytes, cudaStream_t s);
void launch_copy_block_idx(const double* S, int ldS, int r0, int nr, const int* cols, int c0, int nc, double* dst,
                           int ldd, cudaStream_t s);

static int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// ---- small dense helpers (q x q, q <= 64, FP64) of the modal prefactorisation and
// the harmonic basis

// G = R^T R (R upper triangular) and the inverse of R; false if G is not SPD.
bool chol_upper_inverse(const double* G, int q, int ld, std::vector<double>& Rinv) {
    std::vector<double> R((size_t)q * q, 0.0);
    for (int j = 0; j < q; ++j) {
        double s = G[(size_t)j * ld + j];
        for (int k = 0; k < j; ++k) s -= R[(size_t)k * q + j] * R[(size_t)k * q + j];
        if (!(s > 0.0)) return false;
        const double rjj = std::sqrt(s);
        R[(size_t)j * q + j] = rjj;
        for (int i = j + 1; i < q; ++i) {
            double t = G[(size_t)j * ld + i];
            for (int k = 0; k < j; ++k) t -= R[(size_t)k * q + j] * R[(size_t)k * q + i];
            R[(size_t)j * q + i] = t / rjj;
        }
    }
    // back substitution on the identity: R X = I, X upper triangular
    Rinv.assign((size_t)q * q, 0.0);
    for (int c = 0; c < q; ++c)
        for (int i = c; i >= 0; --i) {
            double t = (i == c) ? 1.0 : 0.0;
            for (int k = i + 1; k <= c; ++k) t -= R[(size_t)i * q + k] * Rinv[(size_t)k * q + c];
            Rinv[(size_t)i * q + c] = t / R[(size_t)i * q + i];
        }
    return true;
}

// Cyclic Jacobi eigenvalue algorithm for a symmetric q x q matrix (Golub &
// Van Loan, Sec. 8.5): A is overwritten; on return w holds the eigenvalues and
// the columns of V the eigenvectors (unsorted).
void jacobi_eig(std::vector<double>& A, int q, std::vector<double>& w, std::vector<double>& V) {
    V.assign((size_t)q * q, 0.0);
    for (int i = 0; i < q; ++i) V[(size_t)i * q + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < q; ++i)
            for (int j = 0; j < q; ++j) {
                const double a = A[(size_t)i * q + j];
                tot += a * a;
                if (i != j) off += a * a;
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < q - 1; ++p)
            for (int r = p + 1; r < q; ++r) {
                const double apr = A[(size_t)p * q + r];
                if (apr == 0.0) continue;
                const double theta = (A[(size_t)r * q + r] - A[(size_t)p * q + p]) / (2.0 * apr);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < q; ++k) {   // A <- J^T A J
                    const double akp = A[(size_t)k * q + p], akr = A[(size_t)k * q + r];
                    A[(size_t)k * q + p] = c * akp - sn * akr;
                    A[(size_t)k * q + r] = sn * akp + c * akr;
                }
                for (int k = 0; k < q; ++k) {
                    const double apk = A[(size_t)p * q + k], ark = A[(size_t)r * q + k];
                    A[(size_t)p * q + k] = c * apk - sn * ark;
                    A[(size_t)r * q + k] = sn * apk + c * ark;
                }
                for (int k = 0; k < q; ++k) {
                    const double vkp = V[(size_t)k * q + p], vkr = V[(size_t)k * q + r];
                    V[(size_t)k * q + p] = c * vkp - sn * vkr;
                    V[(size_t)k * q + r] = sn * vkp + c * vkr;
                }
            }
    }
    w.resize(q);
    for (int i = 0; i < q; ++i) w[i] = A[(size_t)i * q + i];
}

void phase_begin(pd_mesh* m, int phase, cudaStream_t s) {
    if (!m->timing_armed || !m->ev_rec || !(m->timing_mask & (1 << phase))) return;
    if (m->timing_iter >= 0 && m->cur_iter >= 0 && m->cur_iter != m->timing_iter) return;
    pd_mesh::TimingSet& T = *m->ev_rec;
    size_t k = (size_t)T.used;
    if (2 * k + 1 >= T.ev.size()) {
        cudaEvent_t a, b;
        PDG_CUDA(cudaEventCreate(&a));
        T.ev.push_back(a);
        PDG_CUDA(cudaEventCreate(&b));
        T.ev.push_back(b);
    }
    if (T.phase.size() <= k) T.phase.resize(k + 1);
    T.phase[k] = phase;
    cudaStreamCaptureStatus st;
    PDG_CUDA(cudaStreamIsCapturing(s, &st));
    unsigned flags = (st == cudaStreamCaptureStatusActive) ? cudaEventRecordExternal : cudaEventRecordDefault;
    PDG_CUDA(cudaEventRecordWithFlags(T.ev[2 * k], s, flags));
    m->ev_open = true;
}

void phase_end(pd_mesh* m, cudaStream_t s) {
    if (!m->timing_armed || !m->ev_open || !m->ev_rec) return;   // only close a pair opened by phase_begin
    m->ev_open = false;
    pd_mesh::TimingSet& T = *m->ev_rec;
    size_t k = (size_t)T.used;
    cudaStreamCaptureStatus st;
    PDG_CUDA(cudaStreamIsCapturing(s, &st));
    unsigned flags = (st == cudaStreamCaptureStatusActive) ? cudaEventRecordExternal : cudaEventRecordDefault;
    PDG_CUDA(cudaEventRecordWithFlags(T.ev[2 * k + 1], s, flags));
    T.used++;
}

}  // namespace pdg

using namespace pdg;

pd_mesh::~pd_mesh() {
    for (auto& kv : graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    graphs.clear();   // the graphs' event sets after their executables
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (int k = 0; k < 2; ++k) {
        if (side[k]) cudaStreamDestroy(side[k]);
        if (ev_fork[k]) cudaEventDestroy(ev_fork[k]);
        if (ev_join[k]) cudaEventDestroy(ev_join[k]);
    }
}

#define PD_API_BEGIN try {
#define PD_API_END                                   \
    }                                                \
    catch (const pdg::Fail& f) {                     \
        return f.code;                               \
    }                                                \
    catch (const std::bad_alloc&) {                  \
        pdg::set_error("host allocation failed");    \
        return PD_ERR_NO_MEMORY;                     \
    }                                                \
    catch (...) {                                    \
        pdg::set_error("unexpected host exception"); \
        return PD_ERR_CUDA;                          \
    }

static pd_status fail(pd_status code, const std::string& msg) {
    set_error(msg);
    return code;
}


static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Recursive coordinate bisection of domain centroids into `parts` groups.
static void rcb(const std::vector<double>& c, std::vector<int32_t> ids, int parts, int32_t first,
                std::vector<int32_t>& out) {
    if (parts <= 1 || ids.size() <= 1) {
        for (int32_t d : ids) out[d] = first;
        return;
    }
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int32_t d : ids)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], c[3 * (size_t)d + k]);
            hi[k] = std::max(hi[k], c[3 * (size_t)d + k]);
        }
    int ax = 0;
    for (int k = 1; k < 3; ++k)
        if (hi[k] - lo[k] > hi[ax] - lo[ax]) ax = k;
    std::stable_sort(ids.begin(), ids.end(),
                     [&](int32_t a, int32_t b) { return c[3 * (size_t)a + ax] < c[3 * (size_t)b + ax]; });
    const int left = parts / 2;
    const size_t cut = ids.size() * left / parts;
    std::vector<int32_t> a(ids.begin(), ids.begin() + cut), b(ids.begin() + cut, ids.end());
    rcb(c, a, left, first, out);
    rcb(c, b, parts - left, first + left, out);
}

// Chooses the domain groups of the two-level interface solve (or none) and
// classifies every interface vertex: iface_class[v] = its group when all its
// domains lie in that group, n_groups for the top-level interface.
static void plan_groups(pd_mesh* m, const double* rest, const std::vector<int32_t>& T,
                        const std::vector<int32_t>& tdom, const std::vector<int32_t>& vdom,
                        const std::vector<uint8_t>& multi, const std::vector<uint8_t>& pin,
                        std::vector<int32_t>& iface_class) {
    const int32_t n_v = m->n_v, n_t = m->n_t, n_dom = m->n_dom;
    m->n_groups = 0;
    m->grp_of_dom.assign(n_dom, 0);
    for (int32_t v = 0; v < n_v; ++v) iface_class[v] = (!pin[v] && multi[v]) ? 0 : -1;
    if (m->n_B <= 4096 || n_dom < 8) return;
    std::vector<double> cen(3 * (size_t)n_dom, 0.0);
    std::vector<int32_t> cnt(n_dom, 0);
    for (int32_t t = 0; t < n_t; ++t)
        for (int k = 0; k < 4; ++k) {
            const int32_t v = T[4 * (size_t)t + k];
            for (int c = 0; c < 3; ++c) cen[3 * (size_t)tdom[t] + c] += rest[3 * (size_t)v + c];
            cnt[tdom[t]]++;
        }
    for (int32_t d = 0; d < n_dom; ++d)
        for (int c = 0; c < 3; ++c) cen[3 * (size_t)d + c] /= std::max(cnt[d], 1);
    std::vector<int32_t> ids(n_dom);
    std::iota(ids.begin(), ids.end(), 0);
    for (int G = 8; G <= 64 && G <= n_dom / 2; G *= 2) {
        std::vector<int32_t> gd(n_dom, 0);
        rcb(cen, ids, G, 0, gd);
        // group set of every vertex (bit mask, G <= 64)
        std::vector<uint64_t> mask(n_v, 0);
        for (int32_t t = 0; t < n_t; ++t)
            for (int k = 0; k < 4; ++k) mask[T[4 * (size_t)t + k]] |= uint64_t(1) << gd[tdom[t]];
        std::vector<int32_t> n2(G, 0), nb2(G, 0);
        int32_t n_top = 0;
        for (int32_t v = 0; v < n_v; ++v) {
            if (pin[v] || !multi[v]) continue;
            if ((mask[v] & (mask[v] - 1)) == 0) {
                n2[__builtin_ctzll(mask[v])]++;
            } else {
                n_top++;
                for (int g = 0; g < G; ++g)
                    if (mask[v] >> g & 1) nb2[g]++;
            }
        }
        const int32_t mx2 = *std::max_element(n2.begin(), n2.end());
        const int32_t mxb = *std::max_element(nb2.begin(), nb2.end());
        if (mx2 > 2048 || mxb > 2048) continue;
        if (n_top == 0 || n_top > 16384 || 2 * n_top > m->n_B) return;   // no worthwhile split
        m->n_groups = G;
        m->grp_of_dom = gd;
        m->top_mask.clear();
        for (int32_t v = 0; v < n_v; ++v) {
            if (pin[v] || !multi[v]) continue;
            iface_class[v] = ((mask[v] & (mask[v] - 1)) == 0) ? __builtin_ctzll(mask[v]) : G;
        }
        m->grp_n2 = n2;
        m->n_top = n_top;
        m->top_groups_of_old.clear();
        for (int32_t v = 0; v < n_v; ++v)
            if (!pin[v] && multi[v] && iface_class[v] == G) m->top_groups_of_old.emplace_back(v, mask[v]);
        return;
    }
}

extern "C" {

const char* pd_status_string(pd_status s) {
    switch (s) {
        case PD_OK: return "ok";
        case PD_ERR_INVALID_ARG: return "invalid argument";
        case PD_ERR_BAD_MESH: return "bad mesh";
        case PD_ERR_BAD_MATERIAL: return "bad material (gamma must be finite and >= 0)";
        case PD_ERR_NOT_PREFACTORED: return "not prefactored";
        case PD_ERR_NOT_SPD: return "matrix not positive definite";
        case PD_ERR_NO_MEMORY: return "out of memory";
        case PD_ERR_NONFINITE: return "non-finite state";
        case PD_ERR_TIMEOUT: return "timeout";
        case PD_ERR_CUDA: return "CUDA error";
        case PD_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

const char* pd_last_error(void) { return g_last_error.c_str(); }

static const char* kPhaseNames[PH_COUNT] = {"inertia",      "local",      "assemble",   "dd_condense", "dd_gather",
                                            "dd_coarse",    "dd_reduce",  "dd_backsub", "residual",    "velocity",
                                            "dd_condense2", "dd_gather2", "dd_backsub2", "dd_interior",
                                            "dd_interior2", "dd_solve", "dd_modal", "dd_jacobi"};

const char* pd_phase_name(int32_t k) { return (k >= 0 && k < PH_COUNT) ? kPhaseNames[k] : "?"; }

void pd_destroy_mesh(pd_mesh* m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    delete m;
}

pd_status pd_create_mesh(const double* rest_xyz, int32_t n_v, const int32_t* tets, int32_t n_t,
                         const double* vertex_mass, double density, const int32_t* tet_domain, int32_t n_domains,
                         const uint8_t* pinned, void* cuda_stream, pd_mesh** out) {
    if (!out) return fail(PD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!rest_xyz || !tets || n_v <= 0 || n_t <= 0 || n_domains <= 0 || n_domains > n_t)
        return fail(PD_ERR_INVALID_ARG, "null input or size out of range");
    if (!vertex_mass && !(density > 0.0 && std::isfinite(density)))
        return fail(PD_ERR_INVALID_ARG, "density must be > 0 when vertex_mass is NULL");
    pd_mesh* m = new (std::nothrow) pd_mesh();
    if (!m) return fail(PD_ERR_NO_MEMORY, "host allocation failed");
    PD_API_BEGIN
    struct Guard {
        pd_mesh* m;
        bool keep = false;
        ~Guard() {
            if (!keep) delete m;
        }
    } guard{m};
    m->n_v = n_v;
    m->n_t = n_t;
    m->n_dom = n_domains;
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    pdg::AllocStreamScope alloc_scope(m->stream);

    // ---- validate tets, rest operators (Dm^-1, V_e); fix orientation
    std::vector<int32_t> T(tets, tets + 4 * (size_t)n_t);
    std::vector<double> dminv_old(9 * (size_t)n_t), vol_old(n_t);
    for (int32_t t = 0; t < n_t; ++t) {
        int32_t* q = &T[4 * (size_t)t];
        for (int k = 0; k < 4; ++k)
            if (q[k] < 0 || q[k] >= n_v) return fail(PD_ERR_BAD_MESH, "tet vertex index out of range");
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b)
                if (q[a] == q[b]) return fail(PD_ERR_BAD_MESH, "tet with a repeated vertex");
        auto X = [&](int k, int c) { return rest_xyz[3 * (size_t)q[k] + c]; };
        double D[3][3];
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 3; ++k) D[c][k] = X(k + 1, c) - X(0, c);   // columns = edges
        double det = D[0][0] * (D[1][1] * D[2][2] - D[1][2] * D[2][1]) -
                     D[0][1] * (D[1][0] * D[2][2] - D[1][2] * D[2][0]) +
                     D[0][2] * (D[1][0] * D[2][1] - D[1][1] * D[2][0]);
        if (det < 0) {
            std::swap(q[2], q[3]);
            for (int c = 0; c < 3; ++c) std::swap(D[c][1], D[c][2]);
            det = -det;
        }
        double e2 = 0;
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 3; ++k) e2 = std::max(e2, D[c][k] * D[c][k]);
        if (!(det > 1e-12 * e2 * std::sqrt(e2)) || !std::isfinite(det))
            return fail(PD_ERR_BAD_MESH, "degenerate tet (rest volume <= 0)");
        double inv[3][3];
        inv[0][0] = (D[1][1] * D[2][2] - D[1][2] * D[2][1]) / det;
        inv[0][1] = (D[0][2] * D[2][1] - D[0][1] * D[2][2]) / det;
        inv[0][2] = (D[0][1] * D[1][2] - D[0][2] * D[1][1]) / det;
        inv[1][0] = (D[1][2] * D[2][0] - D[1][0] * D[2][2]) / det;
        inv[1][1] = (D[0][0] * D[2][2] - D[0][2] * D[2][0]) / det;
        inv[1][2] = (D[0][2] * D[1][0] - D[0][0] * D[1][2]) / det;
        inv[2][0] = (D[1][0] * D[2][1] - D[1][1] * D[2][0]) / det;
        inv[2][1] = (D[0][1] * D[2][0] - D[0][0] * D[2][1]) / det;
        inv[2][2] = (D[0][0] * D[1][1] - D[0][1] * D[1][0]) / det;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) dminv_old[9 * (size_t)t + 3 * i + j] = inv[i][j];
        vol_old[t] = det / 6.0;
    }

    // ---- domains
    std::vector<int32_t> tdom(n_t);
    if (tet_domain) {
        for (int32_t t = 0; t < n_t; ++t) {
            if (tet_domain[t] < 0 || tet_domain[t] >= n_domains)
                return fail(PD_ERR_INVALID_ARG, "tet_domain out of range");
            tdom[t] = tet_domain[t];
        }
    } else {
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int32_t v = 0; v < n_v; ++v)
            for (int c = 0; c < 3; ++c) {
                lo[c] = std::min(lo[c], rest_xyz[3 * (size_t)v + c]);
                hi[c] = std::max(hi[c], rest_xyz[3 * (size_t)v + c]);
            }
        int ax = 0;
        for (int c = 1; c < 3; ++c)
            if (hi[c] - lo[c] > hi[ax] - lo[ax]) ax = c;
        std::vector<std::pair<double, int32_t>> key(n_t);
        for (int32_t t = 0; t < n_t; ++t) {
            double s = 0;
            for (int k = 0; k < 4; ++k) s += rest_xyz[3 * (size_t)T[4 * (size_t)t + k] + ax];
            key[t] = {s, t};
        }
        std::stable_sort(key.begin(), key.end());
        for (int32_t r = 0; r < n_t; ++r) tdom[key[r].second] = (int32_t)((int64_t)r * n_domains / n_t);
    }

    // ---- vertex classes
    std::vector<int32_t> vdom(n_v, -1);
    std::vector<uint8_t> multi(n_v, 0);
    for (int32_t t = 0; t < n_t; ++t)
        for (int k = 0; k < 4; ++k) {
            int32_t v = T[4 * (size_t)t + k];
            if (vdom[v] < 0) vdom[v] = tdom[t];
            else if (vdom[v] != tdom[t]) multi[v] = 1;
        }
    std::vector<uint8_t> pin(n_v, 0);
    if (pinned)
        for (int32_t v = 0; v < n_v; ++v) pin[v] = pinned[v] ? 1 : 0;
    for (int32_t v = 0; v < n_v; ++v)
        if (vdom[v] < 0 && !pin[v]) return fail(PD_ERR_BAD_MESH, "vertex not used by any tet (and not pinned)");

    // ---- new numbering: [domain internals][interface][pinned], each in increasing old id
    m->dom_n_int.assign(n_domains, 0);
    int32_t n_pin = 0, n_B = 0;
    for (int32_t v = 0; v < n_v; ++v) {
        if (pin[v]) n_pin++;
        else if (multi[v]) n_B++;
        else m->dom_n_int[vdom[v]]++;
    }
    m->dom_int_off.assign(n_domains, 0);
    int32_t acc = 0;
    for (int32_t d = 0; d < n_domains; ++d) {
        m->dom_int_off[d] = acc;
        acc += m->dom_n_int[d];
    }
    m->n_int = acc;
    m->n_B = n_B;
    m->n_pin = n_pin;
    m->n_free = acc + n_B;
    // ---- super-domains for the two-level interface solve: the interface vertices
    // whose domains all lie in one group of domains form that group's internal
    // set (S is block-diagonal on them); the rest form the top-level interface.
    std::vector<int32_t> iface_class(n_v, -1);   // group of an internal-interface vertex, n_groups = top
    plan_groups(m, rest_xyz, T, tdom, vdom, multi, pin, iface_class);
    m->new_of_old.assign(n_v, -1);
    m->old_of_new.assign(n_v, -1);
    {
        std::vector<int32_t> fill(m->dom_int_off);
        // interface block ordered by (group class, vertex id)
        std::vector<int32_t> ifill(m->n_groups + 1, 0);
        {
            std::vector<int32_t> cnt(m->n_groups + 1, 0);
            for (int32_t v = 0; v < n_v; ++v)
                if (!pin[v] && multi[v]) cnt[iface_class[v]]++;
            int32_t a = m->n_int;
            for (int32_t g = 0; g <= m->n_groups; ++g) {
                ifill[g] = a;
                a += cnt[g];
            }
        }
        int32_t np = m->n_free;
        for (int32_t v = 0; v < n_v; ++v) {
            int32_t nv;
            if (pin[v]) nv = np++;
            else if (multi[v]) nv = ifill[iface_class[v]]++;
            else nv = fill[vdom[v]]++;
            m->new_of_old[v] = nv;
            m->old_of_new[nv] = v;
        }
    }

    if (m->n_groups > 0) {
        m->top_mask.assign(m->n_top, 0);
        const int32_t T0 = m->n_int + m->n_B - m->n_top;
        for (const auto& pr : m->top_groups_of_old) m->top_mask[m->new_of_old[pr.first] - T0] = pr.second;
        m->top_groups_of_old.clear();
    }

    // ---- tets sorted by domain (stable), in new vertex ids
    m->tet_old_of_new.resize(n_t);
    std::iota(m->tet_old_of_new.begin(), m->tet_old_of_new.end(), 0);
    std::stable_sort(m->tet_old_of_new.begin(), m->tet_old_of_new.end(),
                     [&](int32_t a, int32_t b) { return tdom[a] < tdom[b]; });
    m->tets_new.resize(4 * (size_t)n_t);
    m->tet_dom.resize(n_t);
    m->vol.resize(n_t);
    m->Dminv.resize(9 * (size_t)n_t);
    for (int32_t t = 0; t < n_t; ++t) {
        int32_t o = m->tet_old_of_new[t];
        for (int k = 0; k < 4; ++k) m->tets_new[4 * (size_t)t + k] = m->new_of_old[T[4 * (size_t)o + k]];
        m->tet_dom[t] = tdom[o];
        m->vol[t] = vol_old[o];
        for (int k = 0; k < 9; ++k) m->Dminv[9 * (size_t)t + k] = dminv_old[9 * (size_t)o + k];
    }

    // ---- masses (new order)
    m->mass.assign(n_v, 0.0);
    if (vertex_mass) {
        for (int32_t v = 0; v < n_v; ++v) {
            if (!(vertex_mass[v] > 0.0) || !std::isfinite(vertex_mass[v]))
                return fail(PD_ERR_INVALID_ARG, "vertex_mass must be finite and > 0");
            m->mass[m->new_of_old[v]] = vertex_mass[v];
        }
    } else {
        for (int32_t t = 0; t < n_t; ++t)
            for (int k = 0; k < 4; ++k) m->mass[m->tets_new[4 * (size_t)t + k]] += density * m->vol[t] / 4.0;
    }

    // ---- per-domain boundary lists: interface vertices sharing a tet with an internal vertex of d
    m->dom_bnd.assign(n_domains, {});
    {
        std::vector<int32_t> mark(n_B, -1);
        for (int32_t t = 0; t < n_t; ++t) {
            const int32_t d = m->tet_dom[t];
            const int32_t* q = &m->tets_new[4 * (size_t)t];
            bool has_int = false;
            for (int k = 0; k < 4; ++k) has_int |= (q[k] < m->n_int);
            if (!has_int) continue;
            for (int k = 0; k < 4; ++k) {
                int32_t v = q[k];
                if (v >= m->n_int && v < m->n_free) {
                    int32_t j = v - m->n_int;
                    if (mark[j] != d) {
                        mark[j] = d;
                        m->dom_bnd[d].push_back(j);
                    }
                }
            }
        }
        for (auto& b : m->dom_bnd) {
            std::sort(b.begin(), b.end());
            b.erase(std::unique(b.begin(), b.end()), b.end());
        }
    }
    int32_t max_ni = 0, max_nb = 0;
    for (int32_t d = 0; d < n_domains; ++d) {
        max_ni = std::max(max_ni, m->dom_n_int[d]);
        max_nb = std::max(max_nb, (int32_t)m->dom_bnd[d].size());
    }
    if (max_ni > dd_max_sub_cols() || max_nb > dd_max_sub_cols())
        return fail(PD_ERR_UNSUPPORTED, "a domain has more than 2048 internal or boundary vertices; use more domains");

    // ---- CSR patterns of K_ff and K_fp; vertex -> (tet, corner) incidences
    {
        std::vector<std::vector<int32_t>> rows(m->n_free), prow(m->n_free);
        for (int32_t t = 0; t < n_t; ++t) {
            const int32_t* q = &m->tets_new[4 * (size_t)t];
            for (int a = 0; a < 4; ++a) {
                if (q[a] >= m->n_free) continue;
                for (int b = 0; b < 4; ++b) {
                    if (q[b] < m->n_free) rows[q[a]].push_back(q[b]);
                    else prow[q[a]].push_back(q[b] - m->n_free);
                }
            }
        }
        m->K_rowptr.assign(m->n_free + 1, 0);
        m->Kfp_rowptr.assign(m->n_free + 1, 0);
        for (int32_t i = 0; i < m->n_free; ++i) {
            auto& r = rows[i];
            std::sort(r.begin(), r.end());
            r.erase(std::unique(r.begin(), r.end()), r.end());
            auto& p = prow[i];
            std::sort(p.begin(), p.end());
            p.erase(std::unique(p.begin(), p.end()), p.end());
            m->K_rowptr[i + 1] = m->K_rowptr[i] + (int32_t)r.size();
            m->Kfp_rowptr[i + 1] = m->Kfp_rowptr[i] + (int32_t)p.size();
        }
        m->K_col.resize(m->K_rowptr.back());
        m->Kfp_col.resize(m->Kfp_rowptr.back());
        for (int32_t i = 0; i < m->n_free; ++i) {
            std::copy(rows[i].begin(), rows[i].end(), m->K_col.begin() + m->K_rowptr[i]);
            std::copy(prow[i].begin(), prow[i].end(), m->Kfp_col.begin() + m->Kfp_rowptr[i]);
        }
    }
    std::vector<int32_t> inc_ptr(m->n_free + 1, 0), inc;
    {
        for (int32_t t = 0; t < n_t; ++t)
            for (int k = 0; k < 4; ++k) {
                int32_t v = m->tets_new[4 * (size_t)t + k];
                if (v < m->n_free) inc_ptr[v + 1]++;
            }
        for (int32_t i = 0; i < m->n_free; ++i) inc_ptr[i + 1] += inc_ptr[i];
        inc.resize(inc_ptr.back());
        std::vector<int32_t> fill(inc_ptr.begin(), inc_ptr.end() - 1);
        for (int32_t t = 0; t < n_t; ++t)
            for (int k = 0; k < 4; ++k) {
                int32_t v = m->tets_new[4 * (size_t)t + k];
                if (v < m->n_free) inc[fill[v]++] = 4 * t + k;   // increasing (t, corner) order
            }
    }

    // ---- device uploads: topology, geometry, state (first CUDA call of the set-up)
    // Priorities: the frame is captured on a high-priority stream and the
    // off-critical-path interior products on low-priority side streams, so
    // that (with per-node priorities at instantiation) the blocks of the
    // interface chain are scheduled ahead of the interior products they
    // run beside.
    int prio_low = 0, prio_high = 0;
    PDG_CUDA(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
    PDG_CUDA(cudaStreamCreateWithPriority(&m->cap_stream, cudaStreamNonBlocking, prio_high));
    for (int k = 0; k < 2; ++k) {
        PDG_CUDA(cudaStreamCreateWithPriority(&m->side[k], cudaStreamNonBlocking, prio_low));
        PDG_CUDA(cudaEventCreateWithFlags(&m->ev_fork[k], cudaEventDisableTiming));
        PDG_CUDA(cudaEventCreateWithFlags(&m->ev_join[k], cudaEventDisableTiming));
    }
    cudaStream_t s = m->stream;
    std::vector<int4> ht(n_t);
    std::vector<float4> hg(3 * (size_t)n_t);
    for (int32_t t = 0; t < n_t; ++t) {
        const int32_t* q = &m->tets_new[4 * (size_t)t];
        ht[t] = make_int4(q[0], q[1], q[2], q[3]);
        const double* D = &m->Dminv[9 * (size_t)t];
        for (int r = 0; r < 3; ++r)
            hg[(size_t)r * n_t + t] = make_float4((float)D[3 * r], (float)D[3 * r + 1], (float)D[3 * r + 2], 0.f);
    }
    upload(m->d_tets, ht, s);
    upload(m->d_geo, hg, s);
    upload(m->d_inc_ptr, inc_ptr, s);
    upload(m->d_inc, inc, s);
    build_local_plan(m, inc_ptr, inc, s);
    upload(m->d_old_of_new, m->old_of_new, s);
    std::vector<float4> hx(n_v);
    for (int32_t i = 0; i < n_v; ++i) {
        int32_t o = m->old_of_new[i];
        hx[i] = make_float4((float)rest_xyz[3 * (size_t)o], (float)rest_xyz[3 * (size_t)o + 1],
                            (float)rest_xyz[3 * (size_t)o + 2], 0.f);
    }
    upload(m->d_x, hx, s);
    m->d_xprev.alloc(n_v);
    m->d_v.alloc(n_v);
    PDG_CUDA(cudaMemsetAsync(m->d_v.p, 0, sizeof(float4) * n_v, s));
    PDG_CUDA(cudaMemcpyAsync(m->d_xprev.p, m->d_x.p, sizeof(float4) * n_v, cudaMemcpyDeviceToDevice, s));
    m->d_force.alloc(4 * (size_t)n_t);
    m->d_by0.alloc(std::max(m->n_free, 1));
    m->d_b.alloc(std::max(m->n_free, 1));
    m->d_y.alloc(std::max(m->n_free, 1));
    m->d_pin_tgt.alloc(std::max(n_pin, 1));
    m->d_r.alloc(std::max(m->n_free, 1));
    m->d_dx.alloc(n_v);
    PDG_CUDA(cudaMemsetAsync(m->d_dx.p, 0, sizeof(float4) * n_v, s));
    m->d_err.alloc(1);
    PDG_CUDA(cudaMemsetAsync(m->d_err.p, 0, sizeof(int32_t), s));
    PDG_CUDA(cudaStreamSynchronize(s));
    guard.keep = true;
    *out = m;
    return PD_OK;
    PD_API_END
}

pd_status pd_set_materials(pd_mesh* m, const float* gamma_s, const float* gamma_v) {
    if (!m || !gamma_s || !gamma_v) return fail(PD_ERR_INVALID_ARG, "null argument");
    PD_API_BEGIN
    pdg::AllocStreamScope alloc_scope(m->stream);
    const int32_t n_t = m->n_t;
    std::vector<float> gs(n_t), gv(n_t);
    auto fetch = [&](const float* src, std::vector<float>& dst) {
        if (is_device_ptr(src)) {
            PDG_CUDA(cudaMemcpyAsync(dst.data(), src, sizeof(float) * n_t, cudaMemcpyDeviceToHost, m->stream));
            PDG_CUDA(cudaStreamSynchronize(m->stream));
        } else {
            std::memcpy(dst.data(), src, sizeof(float) * n_t);
        }
    };
    fetch(gamma_s, gs);
    fetch(gamma_v, gv);
    for (int32_t t = 0; t < n_t; ++t)
        if (!(gs[t] >= 0.f) || !(gv[t] >= 0.f) || !std::isfinite(gs[t]) || !std::isfinite(gv[t]))
            return fail(PD_ERR_BAD_MATERIAL, "gamma must be finite and >= 0");
    m->gamma_s.resize(n_t);
    m->gamma_v.resize(n_t);
    std::vector<float> vol(n_t);
    for (int32_t t = 0; t < n_t; ++t) {
        m->gamma_s[t] = gs[m->tet_old_of_new[t]];
        m->gamma_v[t] = gv[m->tet_old_of_new[t]];
        vol[t] = (float)m->vol[t];
    }
    DBuf<float> dvol, dgs, dgv;
    upload(dvol, vol, m->stream);
    upload(dgs, m->gamma_s, m->stream);
    upload(dgv, m->gamma_v, m->stream);
    launch_weights_raw(n_t, dvol.p, dgs.p, dgv.p, m->d_geo.p, m->stream);
    PDG_CUDA(cudaStreamSynchronize(m->stream));
    m->materials_set = true;
    m->prefactored = false;
    ++m->mat_gen;
    return PD_OK;
    PD_API_END
}

pd_status pd_prefactor(pd_mesh* m, double dt, const pd_solver_opts* opts) {
    if (!m) return fail(PD_ERR_INVALID_ARG, "mesh is NULL");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(PD_ERR_INVALID_ARG, "dt must be > 0");
    if (!m->materials_set) return fail(PD_ERR_BAD_MATERIAL, "materials not set");
    pd_solver_opts o{PD_PREC_FP32, 0, 1, 0};
    if (opts) o = *opts;
    if ((o.flags & PD_SOLVE_CORRECTION) && o.refine_steps > 0)
        return fail(PD_ERR_INVALID_ARG, "the correction form refines every PD iteration itself: refine_steps must be 0");
    if (o.precision < PD_PREC_FP32 || o.precision > PD_PREC_TF32 || o.refine_steps < 0 || o.refine_steps > 2 ||
        (o.flags & ~(PD_SOLVE_CORRECTION | PD_SOLVE_SINGLE_LEVEL | PD_SOLVE_STREAMING | PD_SOLVE_MODAL)) != 0)
        return fail(PD_ERR_INVALID_ARG, "bad solver options");
    if ((o.flags & PD_SOLVE_MODAL) &&
        ((o.flags & PD_SOLVE_STREAMING) || o.modes < 0 || o.modes > 64 || o.jacobi_sweeps < 0 ||
         o.jacobi_sweeps > 1000 || !(o.jacobi_rho < 1.0) || !std::isfinite(o.jacobi_rho)))
        return fail(PD_ERR_INVALID_ARG, "bad modal-solve options");
    PD_API_BEGIN
    pdg::AllocStreamScope alloc_scope(m->stream);
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = m->stream;
    m->prefactored = false;
    {
        int dev = 0;
        PDG_CUDA(cudaGetDevice(&dev));
        PDG_CUDA(cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, dev));
    }
    for (auto& kv : m->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    m->graphs.clear();
    const int32_t n_free = m->n_free, n_int = m->n_int, n_B = m->n_B, n_dom = m->n_dom;
    const double inv_h2 = 1.0 / (dt * dt);

    // ---- scalar K over free vertices and the free-pinned block (FP64, host, fixed order)
    m->K_val.assign(m->K_col.size(), 0.0);
    m->Kfp_val.assign(m->Kfp_col.size(), 0.0);
    auto addK = [&](int32_t a, int32_t b, double v) {
        if (b < n_free) {
            auto beg = m->K_col.begin() + m->K_rowptr[a], end = m->K_col.begin() + m->K_rowptr[a + 1];
            m->K_val[std::lower_bound(beg, end, b) - m->K_col.begin()] += v;
        } else {
            int32_t p = b - n_free;
            auto beg = m->Kfp_col.begin() + m->Kfp_rowptr[a], end = m->Kfp_col.begin() + m->Kfp_rowptr[a + 1];
            m->Kfp_val[std::lower_bound(beg, end, p) - m->Kfp_col.begin()] += v;
        }
    };
    for (int32_t t = 0; t < m->n_t; ++t) {
        const double* D = &m->Dminv[9 * (size_t)t];
        double g[4][3];
        for (int c = 0; c < 3; ++c) {
            g[1][c] = D[c];
            g[2][c] = D[3 + c];
            g[3][c] = D[6 + c];
            g[0][c] = -(D[c] + D[3 + c] + D[6 + c]);
        }
        const double w = m->vol[t] * ((double)m->gamma_s[t] + (double)m->gamma_v[t]);
        const int32_t* q = &m->tets_new[4 * (size_t)t];
        for (int a = 0; a < 4; ++a) {
            if (q[a] >= n_free) continue;
            for (int b = 0; b < 4; ++b)
                addK(q[a], q[b], w * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]));
        }
    }
    for (int32_t i = 0; i < n_free; ++i) addK(i, i, m->mass[i] * inv_h2);

    // per-iteration small arrays
    {
        std::vector<float> mh2(std::max(n_free, 1));
        for (int32_t i = 0; i < n_free; ++i) mh2[i] = (float)(m->mass[i] * inv_h2);
        upload(m->d_mh2, mh2, s);
        upload(m->d_kfp_ptr, m->Kfp_rowptr, s);
        std::vector<int32_t> kc(m->Kfp_col);
        std::vector<float> kv(m->Kfp_val.size());
        for (size_t k = 0; k < kv.size(); ++k) kv[k] = (float)m->Kfp_val[k];
        upload(m->d_kfp_col, kc, s);
        upload(m->d_kfp_val, kv, s);
        upload(m->d_K_ptr, m->K_rowptr, s);
        upload(m->d_K_col, m->K_col, s);
        upload(m->d_K_val, m->K_val, s);
    }

    // ---- per-domain dense blocks K_ii (padded with identity) and K_ib
    const int nb64 = dense_block();
    int32_t max_ni = 1, max_nb = 1;
    for (int32_t d = 0; d < n_dom; ++d) {
        max_ni = std::max(max_ni, m->dom_n_int[d]);
        max_nb = std::max(max_nb, (int32_t)m->dom_bnd[d].size());
    }
    const int NI = (int)round_up(max_ni, nb64);
    const int NBp = (int)round_up(max_nb, 8);
    const int64_t sKii = (int64_t)NI * NI, sKib = (int64_t)NI * NBp, sSd = (int64_t)NBp * NBp;
    std::vector<double> hKii((size_t)n_dom * sKii, 0.0), hKib((size_t)n_dom * sKib, 0.0);
    {
        std::vector<int32_t> pos(std::max(n_B, 1), -1);
        for (int32_t d = 0; d < n_dom; ++d) {
            double* Kii = &hKii[(size_t)d * sKii];
            double* Kib = &hKib[(size_t)d * sKib];
            const auto& bl = m->dom_bnd[d];
            for (int32_t k = 0; k < (int32_t)bl.size(); ++k) pos[bl[k]] = k;
            const int32_t off = m->dom_int_off[d], ni = m->dom_n_int[d];
            for (int32_t r = ni; r < NI; ++r) Kii[(size_t)r * NI + r] = 1.0;
            for (int32_t r = 0; r < ni; ++r) {
                const int32_t i = off + r;
                for (int32_t k = m->K_rowptr[i]; k < m->K_rowptr[i + 1]; ++k) {
                    const int32_t c = m->K_col[k];
                    if (c >= off && c < off + ni) Kii[(size_t)r * NI + (c - off)] = m->K_val[k];
                    else if (c >= n_int) Kib[(size_t)r * NBp + pos[c - n_int]] = m->K_val[k];
                    else return fail(PD_ERR_BAD_MESH, "internal vertex coupled to another domain's internal vertex");
                }
            }
            for (int32_t k = 0; k < (int32_t)bl.size(); ++k) pos[bl[k]] = -1;
        }
    }
    DBuf<double> dKii, dXii, dKib, dPsi, dSd;
    upload(dKii, hKii, s);
    upload(dKib, hKib, s);
    hKii.clear(); hKii.shrink_to_fit();
    hKib.clear(); hKib.shrink_to_fit();
    dXii.alloc((size_t)n_dom * sKii);
    dPsi.alloc((size_t)n_dom * sKib);
    dSd.alloc((size_t)n_dom * sSd);
    PDG_CUDA(cudaMemsetAsync(m->d_err.p, 0, sizeof(int32_t), s));
    dense_spd_inverse(dKii.p, NI, NI, sKii, dXii.p, NI, sKii, n_dom, m->d_err.p, s);
    // Psi = -K_ii^-1 K_ib ;  S_d = K_ib^T Psi = -K_bi K_ii^-1 K_ib
    dense_gemm(false, false, NI, NBp, NI, -1.0, dXii.p, NI, sKii, dKib.p, NBp, sKib, 0.0, dPsi.p, NBp, sKib, n_dom,
               false, s);
    dense_gemm(true, false, NBp, NBp, NI, 1.0, dKib.p, NBp, sKib, dPsi.p, NBp, sKib, 0.0, dSd.p, NBp, sSd, n_dom,
               false, s);
    dKii.free();
    dKib.free();

    // ---- the paper's normal modes (PD_SOLVE_MODAL): per domain the r
    // eigenvectors of K_ii with the smallest eigenvalues (the largest of
    // K_ii^-1), by subspace iteration with K_ii^-1 (batched FP64 GEMMs on the
    // device) re-orthonormalised by Cholesky QR, then Rayleigh-Ritz; only the
    // q x q Gram and Ritz matrices (q <= 64) are factored on the host.
    const bool modal = (o.flags & PD_SOLVE_MODAL) != 0;
    const int r_req = modal ? (o.modes > 0 ? o.modes : 20) : 0;
    const int NR = modal ? (int)round_up(r_req, 8) : 8;
    std::vector<int32_t> r_dom(n_dom, 0);
    DBuf<double> dPhi, dPhiS;   // Phi and Phi Lambda^-1, n_dom blocks of NI x NR
    if (modal) {
        const int NQ = (int)round_up(std::min(r_req + 8, 64), 8);
        const int64_t sZ = (int64_t)NI * NQ, sG = (int64_t)NQ * NQ, sP = (int64_t)NI * NR, sV = (int64_t)NQ * NR;
        std::vector<int32_t> q_dom(n_dom, 0);
        for (int32_t d = 0; d < n_dom; ++d) {
            q_dom[d] = std::min(NQ, m->dom_n_int[d]);
            r_dom[d] = std::min(r_req, m->dom_n_int[d]);
        }
        // start block: fixed pseudo-random entries (64-bit LCG) on each domain's
        // rows and first q columns, zero elsewhere
        std::vector<double> hz((size_t)n_dom * sZ, 0.0);
        uint64_t st = 0x9e3779b97f4a7c15ull;
        for (int32_t d = 0; d < n_dom; ++d)
            for (int32_t k = 0; k < m->dom_n_int[d]; ++k)
                for (int j = 0; j < q_dom[d]; ++j) {
                    st = st * 6364136223846793005ull + 1442695040888963407ull;
                    hz[(size_t)d * sZ + (size_t)k * NQ + j] = (double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
                }
        DBuf<double> dZ, dY, dG;
        upload(dZ, hz, s);
        dY.alloc((size_t)n_dom * sZ);
        dG.alloc((size_t)n_dom * sG);
        std::vector<double> hG((size_t)n_dom * sG), hR((size_t)n_dom * sG);
        std::vector<double> Rinv;
        constexpr int kModalIters = 60;
        for (int it = 0; it <= kModalIters; ++it) {
            dense_gemm(false, false, NI, NQ, NI, 1.0, dXii.p, NI, sKii, dZ.p, NQ, sZ, 0.0, dY.p, NQ, sZ, n_dom, false,
                       s);
            if (it == kModalIters) break;
            dense_gemm(true, false, NQ, NQ, NI, 1.0, dY.p, NQ, sZ, dY.p, NQ, sZ, 0.0, dG.p, NQ, sG, n_dom, false, s);
            PDG_CUDA(cudaMemcpyAsync(hG.data(), dG.p, sizeof(double) * hG.size(), cudaMemcpyDeviceToHost, s));
            PDG_CUDA(cudaStreamSynchronize(s));
            std::fill(hR.begin(), hR.end(), 0.0);
            for (int32_t d = 0; d < n_dom; ++d) {
                const int q = q_dom[d];
                if (q == 0) continue;
                if (!chol_upper_inverse(&hG[(size_t)d * sG], q, NQ, Rinv))
                    return fail(PD_ERR_NOT_SPD, "modal subspace iteration lost rank");
                for (int i = 0; i < q; ++i)
                    for (int j = 0; j < q; ++j) hR[(size_t)d * sG + (size_t)i * NQ + j] = Rinv[(size_t)i * q + j];
            }
            PDG_CUDA(cudaMemcpyAsync(dG.p, hR.data(), sizeof(double) * hR.size(), cudaMemcpyHostToDevice, s));
            dense_gemm(false, false, NI, NQ, NQ, 1.0, dY.p, NQ, sZ, dG.p, NQ, sG, 0.0, dZ.p, NQ, sZ, n_dom, false, s);
        }
        // Rayleigh-Ritz with K_ii^-1: T = Z^T (K_ii^-1 Z), eigenvalues mu = 1 / lambda
        dense_gemm(true, false, NQ, NQ, NI, 1.0, dZ.p, NQ, sZ, dY.p, NQ, sZ, 0.0, dG.p, NQ, sG, n_dom, false, s);
        PDG_CUDA(cudaMemcpyAsync(hG.data(), dG.p, sizeof(double) * hG.size(), cudaMemcpyDeviceToHost, s));
        PDG_CUDA(cudaStreamSynchronize(s));
        std::vector<double> hV((size_t)n_dom * sV, 0.0), hVs((size_t)n_dom * sV, 0.0), T, w, V;
        m->modal_lambda_min = 1e300;
        for (int32_t d = 0; d < n_dom; ++d) {
            const int q = q_dom[d];
            if (q == 0) continue;
            T.assign((size_t)q * q, 0.0);
            for (int i = 0; i < q; ++i)
                for (int j = 0; j < q; ++j)
                    T[(size_t)i * q + j] =
                        0.5 * (hG[(size_t)d * sG + (size_t)i * NQ + j] + hG[(size_t)d * sG + (size_t)j * NQ + i]);
            jacobi_eig(T, q, w, V);
            std::vector<int> idx(q);
            std::iota(idx.begin(), idx.end(), 0);
            std::sort(idx.begin(), idx.end(), [&](int a, int b) { return w[a] > w[b]; });
            for (int j = 0; j < r_dom[d]; ++j) {
                const double mu = w[idx[j]];
                if (!(mu > 0.0)) return fail(PD_ERR_NOT_SPD, "modal Rayleigh-Ritz value not positive");
                m->modal_lambda_min = std::min(m->modal_lambda_min, 1.0 / mu);
                for (int i = 0; i < q; ++i) {
                    hV[(size_t)d * sV + (size_t)i * NR + j] = V[(size_t)i * q + idx[j]];
                    hVs[(size_t)d * sV + (size_t)i * NR + j] = V[(size_t)i * q + idx[j]] * mu;   // / lambda
                }
            }
        }
        DBuf<double> dV, dVs;
        upload(dV, hV, s);
        upload(dVs, hVs, s);
        dPhi.alloc((size_t)n_dom * sP);
        dPhiS.alloc((size_t)n_dom * sP);
        dense_gemm(false, false, NI, NR, NQ, 1.0, dZ.p, NQ, sZ, dV.p, NR, sV, 0.0, dPhi.p, NR, sP, n_dom, false, s);
        dense_gemm(false, false, NI, NR, NQ, 1.0, dZ.p, NQ, sZ, dVs.p, NR, sV, 0.0, dPhiS.p, NR, sP, n_dom, false, s);
        PDG_CUDA(cudaStreamSynchronize(s));
    }

    // ---- boundary index lists and the reduced interface matrix S = K_BB + sum_d S_d
    std::vector<int32_t> sbidx_off(n_dom + 1, 0), sbidx;
    for (int32_t d = 0; d < n_dom; ++d) sbidx_off[d + 1] = sbidx_off[d] + (int32_t)m->dom_bnd[d].size();
    sbidx.reserve(sbidx_off.back());
    for (int32_t d = 0; d < n_dom; ++d) sbidx.insert(sbidx.end(), m->dom_bnd[d].begin(), m->dom_bnd[d].end());
    DBuf<int32_t> d_sbidx;
    upload(d_sbidx, sbidx, s);
    const int nBp = (int)round_up(std::max(n_B, 1), nb64);
    DBuf<double> dS, dXS;
    const bool two = m->n_groups > 0 && n_B > 0 && !(o.flags & PD_SOLVE_SINGLE_LEVEL);
    if (n_B > 0) {
        dS.alloc((size_t)nBp * nBp);
        dense_set_identity(dS.p, nBp, nBp, 0, 1, s);
        std::vector<int32_t> cr, cc;
        std::vector<double> cv;
        for (int32_t j = 0; j < n_B; ++j) {
            const int32_t i = n_int + j;
            for (int32_t k = m->K_rowptr[i]; k < m->K_rowptr[i + 1]; ++k)
                if (m->K_col[k] >= n_int) {
                    cr.push_back(j);
                    cc.push_back(m->K_col[k] - n_int);
                    cv.push_back(m->K_val[k]);
                }
        }
        // diagonal entries of the padding stay 1; real diagonal entries are overwritten
        DBuf<int32_t> dcr, dcc;
        DBuf<double> dcv;
        upload(dcr, cr, s);
        upload(dcc, cc, s);
        upload(dcv, cv, s);
        launch_prefactor_helpers_scatter_coo(dS.p, nBp, dcr.p, dcc.p, dcv.p, (int)cv.size(), s);
        for (int32_t d = 0; d < n_dom; ++d) {
            const int nbd = (int)m->dom_bnd[d].size();
            if (nbd == 0 || m->dom_n_int[d] == 0) continue;
            launch_prefactor_add_block(dS.p, nBp, dSd.p + (size_t)d * sSd, NBp, d_sbidx.p + sbidx_off[d], nbd, s);
        }
        PDG_CUDA(cudaStreamSynchronize(s));
        if (!two) {
            dXS.alloc((size_t)nBp * nBp);
            dense_spd_inverse(dS.p, nBp, nBp, 0, dXS.p, nBp, 0, 1, m->d_err.p, s);
        }
    }
    dSd.free();

    // ---- second level: the interface vertices internal to each group of domains
    // (S_II block-diagonal over groups) are condensed onto the top-level
    // interface T: S2 = S_TT + sum_g S_TI S_II^-1 S_IT (the same construction as
    // the first level, applied to S).
    const int G = two ? m->n_groups : 0;
    const int32_t nT = two ? m->n_top : 0, T0 = n_B - nT;
    std::vector<int32_t> i2_off(G + 1, 0), b2_off(G + 1, 0), b2all;
    std::vector<std::vector<int32_t>> b2(G);
    int NI2 = 64, NB2 = 8, nTp = 64;
    DBuf<double> dX2ii, dPsi2, dX2;
    if (two) {
        for (int g = 0; g < G; ++g) i2_off[g + 1] = i2_off[g] + m->grp_n2[g];
        for (int32_t k = 0; k < nT; ++k)
            for (int g = 0; g < G; ++g)
                if (m->top_mask[k] >> g & 1) b2[g].push_back(k);
        int32_t mx2 = 1, mxb = 1;
        for (int g = 0; g < G; ++g) {
            mx2 = std::max(mx2, m->grp_n2[g]);
            mxb = std::max(mxb, (int32_t)b2[g].size());
            b2_off[g + 1] = b2_off[g] + (int32_t)b2[g].size();
            b2all.insert(b2all.end(), b2[g].begin(), b2[g].end());
        }
        NI2 = (int)round_up(mx2, nb64);
        NB2 = (int)round_up(mxb, 8);
        nTp = (int)round_up(std::max(nT, 1), nb64);
        const int64_t s2ii = (int64_t)NI2 * NI2, s2it = (int64_t)NI2 * NB2, s2d = (int64_t)NB2 * NB2;
        DBuf<int32_t> d_b2;
        upload(d_b2, b2all, s);
        DBuf<double> dS2ii, dS2it, dS2d, dS2;
        dS2ii.alloc((size_t)G * s2ii);
        dS2it.alloc((size_t)G * s2it);
        dX2ii.alloc((size_t)G * s2ii);
        dPsi2.alloc((size_t)G * s2it);
        dS2d.alloc((size_t)G * s2d);
        dense_set_identity(dS2ii.p, NI2, NI2, s2ii, G, s);
        PDG_CUDA(cudaMemsetAsync(dS2it.p, 0, sizeof(double) * G * s2it, s));
        for (int g = 0; g < G; ++g) {
            const int r0 = i2_off[g], n2 = m->grp_n2[g], nb = (int)b2[g].size();
            if (n2 == 0) continue;
            launch_copy_block_idx(dS.p, nBp, r0, n2, nullptr, r0, n2, dS2ii.p + g * s2ii, NI2, s);
            if (nb > 0)
                launch_copy_block_idx(dS.p, nBp, r0, n2, d_b2.p + b2_off[g], T0, nb, dS2it.p + g * s2it, NB2, s);
        }
        dense_spd_inverse(dS2ii.p, NI2, NI2, s2ii, dX2ii.p, NI2, s2ii, G, m->d_err.p, s);
        dense_gemm(false, false, NI2, NB2, NI2, -1.0, dX2ii.p, NI2, s2ii, dS2it.p, NB2, s2it, 0.0, dPsi2.p, NB2, s2it,
                   G, false, s);
        dense_gemm(true, false, NB2, NB2, NI2, 1.0, dS2it.p, NB2, s2it, dPsi2.p, NB2, s2it, 0.0, dS2d.p, NB2, s2d, G,
                   false, s);
        dS2.alloc((size_t)nTp * nTp);
        dX2.alloc((size_t)nTp * nTp);
        dense_set_identity(dS2.p, nTp, nTp, 0, 1, s);
        launch_copy_block_idx(dS.p, nBp, T0, nT, nullptr, T0, nT, dS2.p, nTp, s);
        for (int g = 0; g < G; ++g) {
            const int nb = (int)b2[g].size();
            if (nb == 0 || m->grp_n2[g] == 0) continue;
            launch_prefactor_add_block(dS2.p, nTp, dS2d.p + g * s2d, NB2, d_b2.p + b2_off[g], nb, s);
        }
        dense_spd_inverse(dS2.p, nTp, nTp, 0, dX2.p, nTp, 0, 1, m->d_err.p, s);
        PDG_CUDA(cudaStreamSynchronize(s));
    }
    dS.free();
    m->two_level = two;

    // ---- per-iteration matrix pool.  Per domain: H_d = [K_ii^-1 | Psi_d]
    // (n_i x (n_i + n_bd), row k holds the coefficients of b_k for every
    // output of the condensation, K_ii^-1 being symmetric) and Psi_d^T
    // (n_bd x n_i, row j holds the coefficients of x_B[j] for every internal
    // output of the back-substitution); then S^-1 (n_B x n_B).
    m->prec = o.precision;
    m->refine = o.refine_steps;
    m->correction = (o.flags & PD_SOLVE_CORRECTION) != 0;
    m->use_graphs = o.use_graphs != 0;
    // per domain: K_ii^-1 (n_i x n_i), Psi_d (n_i x n_bd, row k = coefficients of
    // b_k for every boundary mode) and Psi_d^T (n_bd x n_i); row strides rounded
    // to 8 entries so every row starts on a 16-byte boundary
    std::vector<int64_t> h_off(n_dom), p_off(n_dom), t_off(n_dom), m1_off(n_dom), m2_off(n_dom);
    std::vector<int32_t> ldH(n_dom), ldP(n_dom), ldT(n_dom), tc_off(n_dom), pm_off(n_dom);
    // BF16 tiles for the tensor cores hold their rows padded to a multiple of 16
    const bool frag16 = !(o.flags & PD_SOLVE_STREAMING) && m->prec == PD_PREC_BF16;
    auto krows = [&](int32_t k) { return frag16 ? (int64_t)round_up(k, 16) : (int64_t)k; };
    // TF32 tiles for the tensor cores: rows padded to a multiple of 8 (the row-form blocks stay row-major)
    const bool fragT = !(o.flags & PD_SOLVE_STREAMING) && m->prec == PD_PREC_TF32;
    auto kax = [&](int32_t k) { return fragT ? (int64_t)round_up(k, 8) : krows(k); };
    int64_t pool = 0;
    int32_t tcr = 0, pmr = 0;
    for (int32_t d = 0; d < n_dom; ++d) {
        const int32_t ni = m->dom_n_int[d], nbd = (int32_t)m->dom_bnd[d].size();
        ldH[d] = (int32_t)round_up(std::max(ni, 1), 8);
        ldP[d] = (int32_t)round_up(std::max(nbd, 1), 8);
        ldT[d] = ldH[d];
        h_off[d] = pool;
        if (modal) {
            // Phi (n_i x r) and (Phi Lambda^-1)^T (r x n_i) in place of K_ii^-1
            m1_off[d] = pool;
            pool += (int64_t)ni * NR;
            m2_off[d] = pool;
            pool += (int64_t)r_dom[d] * ldH[d];
            pm_off[d] = pmr;
            pmr += r_dom[d];
        } else {
            pool += kax(ni) * ldH[d];
        }
        p_off[d] = pool;
        pool += kax(ni) * ldP[d];
        t_off[d] = pool;
        pool += kax(nbd) * ldT[d];
        tc_off[d] = tcr;
        tcr += ni + nbd;
    }
    // second level, row form: per group [S_II^-1; Psi2^T] ((n2 + nb) x n2, row o
    // holds the coefficients of every c_I entry for output o) and Psi2 (n2 x nb)
    std::vector<int64_t> h2_off(G), t2_off(G);
    std::vector<int32_t> ldH2(G), ldT2(G), tc2_off(G);
    int32_t tc2r = 0;
    // (BF16 on the tensor cores: rows and columns padded to 16, 16 x 16 blocks
    // in the mma operand order, the Psi2^T rows starting a block-row of their own)
    std::vector<int32_t> psi2_row(G);   // first row of Psi2^T in the stacked block
    for (int g = 0; g < G; ++g) {
        const int32_t n2 = m->grp_n2[g], nb = (int32_t)b2[g].size();
        ldH2[g] = (int32_t)round_up(std::max(n2, 1), frag16 ? 16 : 8);
        ldT2[g] = (int32_t)round_up(std::max(nb, 1), frag16 ? 16 : 8);
        psi2_row[g] = (int32_t)krows(n2);
        h2_off[g] = pool;
        pool += (krows(n2) + krows(nb)) * ldH2[g];
        t2_off[g] = pool;
        pool += krows(n2) * ldT2[g];
        pool = round_up(pool, 8);
        tc2_off[g] = tc2r;
        tc2r += n2 + nb;
    }
    m->cs_n = two ? nT : n_B;
    // the coarse block too, where its x fits in shared memory beside the stages
    const bool coarse_frag = frag16 && rowdot_mma_fits((int)round_up(std::max(m->cs_n, 1), 16));
    m->off_S = pool;
    m->ld_S = (int32_t)round_up(std::max(m->cs_n, 1), coarse_frag ? 16 : 8);
    pool += (coarse_frag ? krows(m->cs_n) : (int64_t)m->cs_n) * m->ld_S;
    pool = std::max<int64_t>(pool, 8);
    m->d_mat32.free();
    m->d_mat16.free();
    if (m->prec == PD_PREC_BF16) {
        m->d_mat16.alloc(pool);
        PDG_CUDA(cudaMemsetAsync(m->d_mat16.p, 0, sizeof(__nv_bfloat16) * pool, s));
    } else {
        m->d_mat32.alloc(pool);
        PDG_CUDA(cudaMemsetAsync(m->d_mat32.p, 0, sizeof(float) * pool, s));
    }
    // the per-domain axpy-form matrices are stored as output-chunk tiles
    // (streamed by bulk copies), except for the fused streaming solve, whose
    // plan copies row-major blocks into its own panels
    const bool tiled = !(o.flags & PD_SOLVE_STREAMING);
    const int OWt = ax_tile_outputs(m->prec), VNt = (m->prec == PD_PREC_BF16 || fragT) ? 8 : 4;
    m->ax_tiled = tiled;
    m->ax_tf32 = fragT;
    if (tiled) ax_prepare_tma(m->prec);
    auto cast_ax = [&](const double* src, int lds, int rows, int cols, int transpose, int64_t off, int ld) {
        if (frag16)
            launch_cast_frag16(src, lds, rows, cols, transpose, m->d_mat16.p, off, ax_chunk_width(cols, OWt, VNt),
                               s);
        else if (fragT)
            launch_cast_frag32(src, lds, rows, cols, transpose, m->d_mat32.p, off, ax_chunk_width(cols, OWt, VNt), s);
        else if (tiled)
            launch_cast_tiled(src, lds, rows, cols, transpose, m->prec, m->d_mat32.p, m->d_mat16.p, off,
                              ax_chunk_width(cols, OWt, VNt), VNt, s);
        else
            launch_cast_block(src, lds, rows, cols, transpose, m->prec, m->d_mat32.p, m->d_mat16.p, off, ld, s);
    };
    for (int32_t d = 0; d < n_dom; ++d) {
        const int32_t ni = m->dom_n_int[d], nbd = (int32_t)m->dom_bnd[d].size();
        if (ni == 0) continue;
        const double* Xd = dXii.p + (size_t)d * sKii;
        const double* Pd = dPsi.p + (size_t)d * sKib;
        if (modal) {
            const int64_t sP = (int64_t)NI * NR;
            if (r_dom[d] > 0) {
                launch_cast_block(dPhi.p + d * sP, NR, ni, r_dom[d], 0, m->prec, m->d_mat32.p, m->d_mat16.p, m1_off[d],
                                  NR, s);
                launch_cast_block(dPhiS.p + d * sP, NR, r_dom[d], ni, 1, m->prec, m->d_mat32.p, m->d_mat16.p, m2_off[d],
                                  ldH[d], s);
            }
        } else {
            cast_ax(Xd, NI, ni, ni, 0, h_off[d], ldH[d]);
        }
        if (nbd > 0) {
            cast_ax(Pd, NBp, ni, nbd, 0, p_off[d], ldP[d]);
            cast_ax(Pd, NBp, nbd, ni, 1, t_off[d], ldT[d]);
        }
    }
    // row-form blocks: row-major, or the BF16 fragment layout of the tensor cores
    auto cast_row = [&](const double* src, int lds, int rows, int cols, int transpose, int64_t off, int ld,
                        bool frag) {
        if (frag) launch_cast_rowfrag16(src, lds, rows, cols, transpose, m->d_mat16.p, off, ld, s);
        else launch_cast_block(src, lds, rows, cols, transpose, m->prec, m->d_mat32.p, m->d_mat16.p, off, ld, s);
    };
    if (n_B > 0 && !two) cast_row(dXS.p, nBp, n_B, n_B, 0, m->off_S, m->ld_S, coarse_frag);
    if (two) {
        const int64_t s2ii = (int64_t)NI2 * NI2, s2it = (int64_t)NI2 * NB2;
        for (int g = 0; g < G; ++g) {
            const int32_t n2 = m->grp_n2[g], nb = (int32_t)b2[g].size();
            if (n2 == 0) continue;
            cast_row(dX2ii.p + g * s2ii, NI2, n2, n2, 0, h2_off[g], ldH2[g], frag16);
            if (nb > 0) {
                cast_row(dPsi2.p + g * s2it, NB2, nb, n2, 1, h2_off[g] + (int64_t)psi2_row[g] * ldH2[g], ldH2[g],
                         frag16);
                cast_row(dPsi2.p + g * s2it, NB2, n2, nb, 0, t2_off[g], ldT2[g], frag16);
            }
        }
        cast_row(dX2.p, nTp, nT, nT, 0, m->off_S, m->ld_S, coarse_frag);
    }

    // ---- descriptors of the per-domain products: one block per output chunk
    const int VN = (m->prec == PD_PREC_BF16 || m->ax_tf32) ? 8 : 4;
    std::vector<int32_t> bidx_off(n_dom + 1, 0), bidx;
    for (int32_t d = 0; d < n_dom; ++d) bidx_off[d + 1] = bidx_off[d] + (int32_t)m->dom_bnd[d].size();
    bidx.reserve(bidx_off.back());
    for (int32_t d = 0; d < n_dom; ++d) bidx.insert(bidx.end(), m->dom_bnd[d].begin(), m->dom_bnd[d].end());
    upload(m->d_bidx, bidx, s);
    {
        // condensation split in two launches: the boundary modes c_d = Psi_d^T b_i
        // (on the path to the interface solve) and the interior part
        // t_d = K_ii^-1 b_i (needed only by the back-substitution)
        const int OW = ax_outputs_per_block(m->prec);
        // tiled descriptors: ld = the chunk width, one block per chunk
        auto tile_desc = [&](AxDesc& a) {
            if (!a.tiled) return OW;
            a.ld = ax_chunk_width(a.n_out, OWt, VN);
            return (int)a.ld;
        };
        std::vector<AxDesc> dc, di, db, dm1, dm2;
        std::vector<AxBlock> bc, bi, bb, bm1, bm2;
        for (int32_t d = 0; d < n_dom; ++d) {
            const int32_t ni = m->dom_n_int[d], nbd = (int32_t)m->dom_bnd[d].size();
            if (ni == 0) continue;
            AxDesc c{};
            c.a_off = p_off[d];
            c.x_off = m->dom_int_off[d];
            c.bidx_off = -1;
            c.add_off = -1;
            c.out_off = tc_off[d] + ni;
            c.K = ni;
            c.ld = ldP[d];
            c.n_out = nbd;
            c.tiled = tiled ? 1 : 0;
            if (nbd > 0) {
                const int cw = tile_desc(c);
                for (int32_t o0 = 0; o0 < c.n_out; o0 += cw) bc.push_back(AxBlock{(int32_t)dc.size(), o0});
                dc.push_back(c);
            }
            if (!modal) {
                AxDesc t = c;
                t.a_off = h_off[d];
                t.out_off = tc_off[d];
                t.ld = ldH[d];
                t.n_out = ni;
                const int cw = tile_desc(t);
                for (int32_t o0 = 0; o0 < t.n_out; o0 += cw) bi.push_back(AxBlock{(int32_t)di.size(), o0});
                di.push_back(t);
            } else if (r_dom[d] > 0) {
                // p = Phi^T b_i (rows k of Phi), then t = (Phi Lambda^-1) p (rows j of its transpose)
                AxDesc a1{};
                a1.a_off = m1_off[d];
                a1.x_off = m->dom_int_off[d];
                a1.bidx_off = -1;
                a1.add_off = -1;
                a1.out_off = pm_off[d];
                a1.K = ni;
                a1.ld = NR;
                a1.n_out = r_dom[d];
                a1.tiled = 0;
                for (int32_t o0 = 0; o0 < a1.n_out; o0 += OW) bm1.push_back(AxBlock{(int32_t)dm1.size(), o0});
                dm1.push_back(a1);
                AxDesc a2{};
                a2.a_off = m2_off[d];
                a2.x_off = pm_off[d];
                a2.bidx_off = -1;
                a2.add_off = -1;
                a2.out_off = tc_off[d];
                a2.K = r_dom[d];
                a2.ld = ldH[d];
                a2.n_out = ni;
                a2.tiled = 0;
                for (int32_t o0 = 0; o0 < a2.n_out; o0 += OW) bm2.push_back(AxBlock{(int32_t)dm2.size(), o0});
                dm2.push_back(a2);
            }
            AxDesc b{};
            b.a_off = t_off[d];
            b.x_off = 0;
            b.bidx_off = bidx_off[d];
            b.add_off = tc_off[d];
            b.out_off = m->dom_int_off[d];
            b.K = nbd;
            b.ld = ldT[d];
            b.n_out = ni;
            b.tiled = tiled ? 1 : 0;
            const int cwb = tile_desc(b);
            for (int32_t o0 = 0; o0 < b.n_out; o0 += cwb) bb.push_back(AxBlock{(int32_t)db.size(), o0});
            db.push_back(b);
        }
        upload(m->d_ax_desc_cond, dc, s);
        upload(m->d_ax_desc_int, di, s);
        upload(m->d_ax_desc_back, db, s);
        upload(m->d_ax_blk_cond, bc, s);
        upload(m->d_ax_blk_int, bi, s);
        upload(m->d_ax_blk_back, bb, s);
        m->ax_blocks_cond = (int32_t)bc.size();
        m->ax_blocks_int = (int32_t)bi.size();
        m->ax_blocks_back = (int32_t)bb.size();
        // host copies for the serving batches: both condensation parts in one launch
        m->h_ax_desc_cond = dc;
        m->h_ax_desc_cond.insert(m->h_ax_desc_cond.end(), di.begin(), di.end());
        m->h_ax_desc_back = db;
        upload(m->d_ax_desc_m1, dm1, s);
        upload(m->d_ax_desc_m2, dm2, s);
        upload(m->d_ax_blk_m1, bm1, s);
        upload(m->d_ax_blk_m2, bm2, s);
        m->ax_blocks_m1 = (int32_t)bm1.size();
        m->ax_blocks_m2 = (int32_t)bm2.size();
        m->ax_kmax_m1 = m->ax_kmax_m2 = 1;
        for (const auto& a : dm1) m->ax_kmax_m1 = std::max(m->ax_kmax_m1, a.K);
        for (const auto& a : dm2) m->ax_kmax_m2 = std::max(m->ax_kmax_m2, a.K);
        m->ax_kmax_cond = m->ax_kmax_int = m->ax_kmax_back = 1;
        for (const auto& a : dc) m->ax_kmax_cond = std::max(m->ax_kmax_cond, a.K);
        for (const auto& a : di) m->ax_kmax_int = std::max(m->ax_kmax_int, a.K);
        for (const auto& a : db) m->ax_kmax_back = std::max(m->ax_kmax_back, a.K);
        m->ax_wmax_cond = m->ax_wmax_int = m->ax_wmax_back = 1;
        for (const auto& a : dc) m->ax_wmax_cond = std::max(m->ax_wmax_cond, a.tiled ? a.ld : OW);
        for (const auto& a : di) m->ax_wmax_int = std::max(m->ax_wmax_int, a.tiled ? a.ld : OW);
        for (const auto& a : db) m->ax_wmax_back = std::max(m->ax_wmax_back, a.tiled ? a.ld : OW);
        (void)VN;
    }
    m->n_tc = tcr;
    m->modal = modal;
    m->modes = r_req;
    m->jacobi_sweeps = modal ? o.jacobi_sweeps : 0;
    m->n_pm = pmr;
    m->d_pm.alloc(std::max(pmr, 1));
    m->jacobi_omega.clear();
    if (modal && m->jacobi_sweeps > 0) {
        // the Jacobi diagonal and the Chebyshev weights (Wang 2015) for the
        // spectral radius rho of I - D^-1 K (given, or from 300 power
        // iterations on the similar symmetric I - D^-1/2 K D^-1/2, raised by 1 %)
        std::vector<double> dinv(std::max(n_free, 1), 1.0), sq(std::max(n_free, 1), 1.0);
        for (int32_t i = 0; i < n_free; ++i)
            for (int32_t k = m->K_rowptr[i]; k < m->K_rowptr[i + 1]; ++k)
                if (m->K_col[k] == i) {
                    dinv[i] = 1.0 / m->K_val[k];
                    sq[i] = std::sqrt(dinv[i]);
                }
        upload(m->d_Dinv, dinv, s);
        double rho = o.jacobi_rho;
        if (!(rho > 0.0)) {
            std::vector<double> v(n_free), w(n_free);
            uint64_t st = 0x2545f4914f6cdd1dull;
            for (auto& e : v) {
                st = st * 6364136223846793005ull + 1442695040888963407ull;
                e = (double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
            }
            double lam = 0.0;
            for (int it = 0; it < 300; ++it) {
                double nrm = 0.0;
                for (int32_t i = 0; i < n_free; ++i) {
                    double kv = 0.0;
                    for (int32_t k = m->K_rowptr[i]; k < m->K_rowptr[i + 1]; ++k)
                        kv += m->K_val[k] * sq[m->K_col[k]] * v[m->K_col[k]];
                    w[i] = v[i] - sq[i] * kv;
                    nrm += w[i] * w[i];
                }
                nrm = std::sqrt(nrm);
                if (!(nrm > 0.0)) break;
                lam = nrm;   // |v| = 1 after the first iteration: ||A v|| -> |lambda|max
                for (int32_t i = 0; i < n_free; ++i) v[i] = w[i] / nrm;
            }
            rho = std::min(0.9999, 1.01 * lam);
        }
        if (!(rho < 1.0)) return fail(PD_ERR_UNSUPPORTED, "Jacobi sweeps do not converge on this matrix");
        m->jacobi_rho = rho;
        double om = 1.0;
        for (int k = 1; k <= m->jacobi_sweeps; ++k) {
            om = (k == 1) ? 1.0 : (k == 2 ? 2.0 / (2.0 - rho * rho) : 4.0 / (4.0 - rho * rho * om));
            m->jacobi_omega.push_back((float)om);
        }
        m->d_jx1.alloc(std::max(n_free, 1));
        m->d_jx2.alloc(std::max(n_free, 1));
    }
    m->d_tc.alloc(std::max(tcr, 1));
    m->rows_cond2.n_blocks = m->rows_int2.n_blocks = m->rows_back2.n_blocks = 0;
    m->rows_cond2.host.clear();
    m->rows_int2.host.clear();
    m->rows_back2.host.clear();
    if (two) {
        // [S_II^-1; Psi2^T] split by rows: the Psi2^T rows give the top-level
        // condensation c2 (on the path to the coarse solve), the S_II^-1 rows
        // the interior part t2 (needed only by the second-level back-substitution)
        std::vector<RowDesc> dc, di, db;
        for (int g = 0; g < G; ++g) {
            const int32_t n2 = m->grp_n2[g], nb = (int32_t)b2[g].size();
            if (n2 == 0) continue;
            RowDesc t{};
            t.a_off = h2_off[g];
            t.rows = n2;
            t.cols = n2;
            t.ld = ldH2[g];
            t.x_off = i2_off[g];
            t.xidx_off = -1;
            t.add_off = -1;
            t.out_off = tc2_off[g];
            di.push_back(t);
            if (nb == 0) continue;
            RowDesc c = t;
            c.a_off = h2_off[g] + (int64_t)psi2_row[g] * ldH2[g];
            c.rows = nb;
            c.out_off = tc2_off[g] + n2;
            dc.push_back(c);
            RowDesc b{};
            b.a_off = t2_off[g];
            b.rows = n2;
            b.cols = nb;
            b.ld = ldT2[g];
            b.x_off = 0;
            b.xidx_off = b2_off[g];
            b.add_off = tc2_off[g];
            b.out_off = i2_off[g];
            db.push_back(b);
        }
        build_row_plan(m->rows_cond2, dc, m->prec, s, frag16);
        build_row_plan(m->rows_int2, di, m->prec, s, frag16);
        build_row_plan(m->rows_back2, db, m->prec, s, frag16);
        upload(m->d_bidx2, b2all, s);
        // top-level gather lists (groups in increasing order)
        std::vector<int32_t> gp(nT + 1, 0), gl;
        std::vector<std::vector<int32_t>> lists(nT);
        for (int g = 0; g < G; ++g) {
            if (m->grp_n2[g] == 0) continue;
            for (int32_t k = 0; k < (int32_t)b2[g].size(); ++k) lists[b2[g][k]].push_back(tc2_off[g] + m->grp_n2[g] + k);
        }
        for (int32_t k = 0; k < nT; ++k) {
            gp[k + 1] = gp[k] + (int32_t)lists[k].size();
            gl.insert(gl.end(), lists[k].begin(), lists[k].end());
        }
        upload(m->d_gat2_ptr, gp, s);
        upload(m->d_gat2, gl, s);
        m->n_tc2 = tc2r;
        m->d_tc2.alloc(std::max(tc2r, 1));
        m->d_cT.alloc(std::max(nT, 1));
        m->n_gat2 = (int32_t)gl.size();
    }
    // interface gather lists (domains in increasing order)
    {
        std::vector<int32_t> gp(n_B + 1, 0), gl;
        std::vector<std::vector<int32_t>> lists(n_B);
        for (int32_t d = 0; d < n_dom; ++d) {
            const int32_t ni = m->dom_n_int[d];
            if (ni == 0) continue;
            const auto& bl = m->dom_bnd[d];
            for (int32_t k = 0; k < (int32_t)bl.size(); ++k) lists[bl[k]].push_back(tc_off[d] + ni + k);
        }
        for (int32_t j = 0; j < n_B; ++j) {
            gp[j + 1] = gp[j] + (int32_t)lists[j].size();
            gl.insert(gl.end(), lists[j].begin(), lists[j].end());
        }
        upload(m->d_gat_ptr, gp, s);
        upload(m->d_gat, gl, s);
    }
    m->d_cB.alloc(std::max(n_B, 1));
    m->coarse_rows_per_cta = 64;
    m->coarse_chunk = dd_coarse_chunk();
    m->coarse_nchunks = (int32_t)((m->ld_S + m->coarse_chunk - 1) / m->coarse_chunk);
    m->d_part.alloc((size_t)std::max(m->cs_n, 1) * m->coarse_nchunks);
    m->coarse_blocks = (m->cs_n > 0) ? dd_configure_coarse(m->ld_S) : 0;
    // The coarse product as a row-form product of whole rows (no split into
    // column chunks, no partial sums to reduce): BF16 on the tensor cores, FP32
    // and TF32 where a row fits one bulk-copy stage; otherwise the balanced split kernel.
    m->rows_coarse.n_blocks = 0;
    m->rows_coarse.host.clear();
    const bool coarse_rows =
        coarse_frag || ((m->prec == PD_PREC_FP32 || m->prec == PD_PREC_TF32) && !(o.flags & PD_SOLVE_STREAMING) &&
                        rowdot_row_fits_stage(m->ld_S, 4));
    if (coarse_rows && m->cs_n > 0) {
        RowDesc c{};
        c.a_off = m->off_S;
        c.rows = m->cs_n;
        c.cols = m->cs_n;
        c.ld = m->ld_S;
        c.x_off = 0;
        c.xidx_off = -1;
        c.add_off = -1;
        c.out_off = 0;
        build_row_plan(m->rows_coarse, std::vector<RowDesc>{c}, m->prec, s, coarse_frag);
        if (!m->rows_coarse.mma && !m->rows_coarse.tma) m->rows_coarse.n_blocks = 0;   // rows too long
    }

    // ---- fused streaming solve (column form), phase by phase:
    //   0: c_d = Psi_d^T b_i over the rows of Psi_d, t_d = K_ii^-1 b_i over the rows of K_ii^-1
    //   1: (two levels) c2, t2 over the rows of Psi2 and S_II^-1, x = c_B formed on the fly
    //   2: x_T = S2^-1 c_T (or x_B = S^-1 c_B on one level), S symmetric
    //   3: (two levels) x_I = t2 + Psi2 x_T over the rows of Psi2^T
    //   4: x_i = t_d + Psi_d x_B over the rows of Psi_d^T
    {
        auto col = [](int phase, int64_t a_off, int32_t K, int32_t n_out, int32_t ld, int32_t xkind, int32_t x_off,
                      int32_t xidx_off, int32_t akind, int32_t add_off, int32_t okind, int32_t out_off) {
            ColDesc c{};
            c.a_off = a_off;
            c.K = K;
            c.n_out = n_out;
            c.ld = ld;
            c.x_off = x_off;
            c.xidx_off = xidx_off;
            c.add_off = add_off;
            c.out_off = out_off;
            c.n_pieces = 1;
            c.phase = phase;
            c.xkind = xkind;
            c.akind = akind;
            c.okind = okind;
            return c;
        };
        auto post = [](ColDesc c, int32_t kind, int32_t off) {
            c.post_kind = kind;
            c.post_off = off;
            return c;
        };
        std::vector<ColDesc> bl;
        for (int32_t d = 0; d < n_dom; ++d) {
            const int32_t ni = m->dom_n_int[d], nbd = (int32_t)m->dom_bnd[d].size();
            if (ni == 0) continue;
            if (nbd > 0)
                bl.push_back(post(col(0, p_off[d], ni, nbd, ldP[d], XK_B, m->dom_int_off[d], -1, VK_NONE, -1, VK_TC,
                                      tc_off[d] + ni),
                                  PK_CB, bidx_off[d]));
            bl.push_back(col(0, h_off[d], ni, ni, ldH[d], XK_B, m->dom_int_off[d], -1, VK_NONE, -1, VK_TC, tc_off[d]));
        }
        const int ph_coarse = two ? 2 : 1, ph_back = two ? 4 : (n_B > 0 ? 2 : 1);
        if (two) {
            for (int g = 0; g < G; ++g) {
                const int32_t n2 = m->grp_n2[g], nb = (int32_t)b2[g].size();
                if (n2 == 0) continue;
                if (nb > 0)
                    bl.push_back(post(col(1, t2_off[g], n2, nb, ldT2[g], XK_CB, i2_off[g], -1, VK_NONE, -1, VK_TC2,
                                          tc2_off[g] + n2),
                                      PK_CT, b2_off[g]));
                bl.push_back(col(1, h2_off[g], n2, n2, ldH2[g], XK_CB, i2_off[g], -1, VK_NONE, -1, VK_TC2, tc2_off[g]));
            }
            bl.push_back(post(col(2, m->off_S, nT, nT, m->ld_S, XK_CT, 0, -1, VK_NONE, -1, VK_X, n_int + T0), PK_XT, 0));
            for (int g = 0; g < G; ++g) {
                const int32_t n2 = m->grp_n2[g], nb = (int32_t)b2[g].size();
                if (n2 == 0 || nb == 0) continue;
                bl.push_back(post(col(3, h2_off[g] + (int64_t)n2 * ldH2[g], nb, n2, ldH2[g], XK_G2, b2_off[g], -1,
                                      VK_TC2, tc2_off[g], VK_X, n_int + i2_off[g]),
                                  PK_XB, i2_off[g]));
            }
        } else if (n_B > 0) {
            bl.push_back(post(col(ph_coarse, m->off_S, n_B, n_B, m->ld_S, XK_CB, 0, -1, VK_NONE, -1, VK_X, n_int), PK_XB,
                              0));
        }
        for (int32_t d = 0; d < n_dom; ++d) {
            const int32_t ni = m->dom_n_int[d], nbd = (int32_t)m->dom_bnd[d].size();
            if (ni == 0) continue;
            bl.push_back(col(ph_back, t_off[d], nbd, ni, ldT[d], XK_GB, bidx_off[d], -1, VK_TC, tc_off[d], VK_X,
                             m->dom_int_off[d]));
        }
        // inverse gather lists (positions of every interface / top entry in the
        // per-domain and per-group lists) and the entries nobody contributes to
        {
            const int32_t nq = (int32_t)bidx.size();
            std::vector<int32_t> ip(n_B + 1, 0), il(nq);
            for (int32_t q = 0; q < nq; ++q) ip[bidx[q] + 1]++;
            for (int32_t j = 0; j < n_B; ++j) ip[j + 1] += ip[j];
            std::vector<int32_t> fill(ip.begin(), ip.end() - 1);
            for (int32_t q = 0; q < nq; ++q) il[fill[bidx[q]]++] = q;
            upload(m->d_invB_ptr, ip, s);
            upload(m->d_invB, il, s);
            m->n_xgB = nq;
            m->d_xgB.alloc(std::max(nq, 1));
            // c_B entries: the contributing domains are those with internal vertices
            std::vector<int32_t> ncb(std::max(n_B, 1), 0);
            for (int32_t d = 0; d < n_dom; ++d)
                if (m->dom_n_int[d] > 0)
                    for (int32_t j : m->dom_bnd[d]) ncb[j]++;
            std::vector<int32_t> z;
            for (int32_t j = 0; j < n_B; ++j)
                if (ncb[j] == 0) z.push_back(j);
            upload(m->d_cb0, z, s);
            m->n_cb0 = (int32_t)z.size();
            const int32_t nq2 = two ? (int32_t)b2all.size() : 0;
            std::vector<int32_t> ip2(nT + 1, 0), il2(std::max(nq2, 0));
            for (int32_t q = 0; q < nq2; ++q) ip2[b2all[q] + 1]++;
            for (int32_t t = 0; t < nT; ++t) ip2[t + 1] += ip2[t];
            std::vector<int32_t> fill2(ip2.begin(), ip2.end() - 1);
            for (int32_t q = 0; q < nq2; ++q) il2[fill2[b2all[q]]++] = q;
            upload(m->d_inv2_ptr, ip2, s);
            upload(m->d_inv2, il2, s);
            m->n_xg2 = nq2;
            m->d_xg2.alloc(std::max(nq2, 1));
            std::vector<int32_t> z2;
            if (two) {
                // the contributing groups are those with internal interface vertices
                std::vector<int32_t> nct(std::max(nT, 1), 0);
                for (int g = 0; g < G; ++g)
                    if (m->grp_n2[g] > 0)
                        for (int32_t t : b2[g]) nct[t]++;
                for (int32_t t = 0; t < nT; ++t)
                    if (nct[t] == 0) z2.push_back(t);
            }
            upload(m->d_ct0, z2, s);
            m->n_ct0 = (int32_t)z2.size();
        }
        const void* src = (m->prec == PD_PREC_BF16) ? (const void*)m->d_mat16.p : (const void*)m->d_mat32.p;
        m->use_stream = (o.flags & PD_SOLVE_STREAMING) && !m->batched_only &&
                        build_stream_plan(m->st_solve, bl, m->prec, src, s);
        if (!m->use_stream) {
            // release what an earlier streaming plan held
            m->st_solve.pan32.free();
            m->st_solve.pan16.free();
            m->st_solve.n_ctas = 0;
        }
        if (m->use_stream) {
            m->st_solve.cnt_cb.alloc(std::max(n_B, 1));
            PDG_CUDA(cudaMemsetAsync(m->st_solve.cnt_cb.p, 0, m->st_solve.cnt_cb.bytes(), s));
            m->st_solve.cnt_ct.alloc(std::max(nT, 1));
            PDG_CUDA(cudaMemsetAsync(m->st_solve.cnt_ct.p, 0, m->st_solve.cnt_ct.bytes(), s));
        }
    }

    // ---- algorithmic bytes per launch of each phase (each array counted once)
    {
        const int64_t es = (m->prec == PD_PREC_BF16) ? 2 : 4;
        int64_t mat_c = 0, mat_i = 0, mat_b = 0, nbd_tot = 0;
        for (int32_t d = 0; d < n_dom; ++d) {
            const int64_t ni = m->dom_n_int[d], nbd = (int64_t)m->dom_bnd[d].size();
            if (ni == 0) continue;
            mat_c += ni * round_up(nbd, VN) * es;
            mat_i += ni * round_up(ni, VN) * es;
        }
        for (const auto& a : m->h_ax_desc_back) mat_b += (int64_t)a.K * round_up(a.n_out, VN) * es;
        for (int32_t d = 0; d < n_dom; ++d)
            if (m->dom_n_int[d] > 0) nbd_tot += (int64_t)m->dom_bnd[d].size();
        const int64_t nv = m->n_v, nf = n_free, nt = m->n_t, ninc = (int64_t)4 * nt;
        const int64_t nkfp = (int64_t)m->Kfp_col.size(), nk = (int64_t)m->K_col.size();
        const int64_t ngat = nbd_tot;
        const int64_t colsS = (int64_t)round_up(std::max(m->cs_n, 1), VN);
        // (tensor-core layout: whole 16-row block-rows are streamed)
        auto plan_bytes = [&](const RowPlan& P) {
            int64_t b = 0;
            for (const auto& d : P.host) b += (int64_t)(P.mma ? round_up(d.rows, 16) : d.rows) * d.ld * es;
            return b;
        };
        const int64_t mat_c2 = plan_bytes(m->rows_cond2), mat_i2 = plan_bytes(m->rows_int2),
                      mat_b2 = plan_bytes(m->rows_back2);
        for (int k = 0; k < 24; ++k) m->phase_bytes[k] = 0;
        m->phase_bytes[PH_INERTIA] = nv * 48 + nf * (16 + 4 + 16 + 4) + nkfp * 8 + (int64_t)m->n_pin * 16;
        // fused local step + assembly: tets and rest operators, x once, by0 (or y and m/dt^2) and b per
        // free vertex, the block plan (16 B per block-vertex entry, 2 B per corner), partial sums of the
        // shared vertices written and read, their counters
        m->phase_bytes[PH_LOCAL] = nt * (16 + 48) + nv * 16 + nf * (m->correction ? 16 + 4 + 16 : 16 + 16) +
                                   (int64_t)m->la_entries * 12 + (int64_t)m->la_corners * 2 +
                                   (int64_t)m->la_slots * 32 + (int64_t)m->la_shared * 8 +
                                   (int64_t)(m->la_blocks + 1) * 4;
        m->phase_bytes[PH_ASSEMBLE] = 0;
        (void)ninc;
        m->phase_bytes[PH_CONDENSE] = mat_c + (int64_t)n_int * 16 + nbd_tot * 16;
        // (per launch: the interior product goes out in two launches when it has more than
        // three tiles per SM, see the solve)
        m->phase_bytes[PH_INTERIOR] = (mat_i + (int64_t)n_int * 32) / (m->ax_blocks_int > 3 * m->sms ? 2 : 1);
        if (modal) {
            int64_t mb = 0;
            for (int32_t d = 0; d < n_dom; ++d)
                mb += ((int64_t)m->dom_n_int[d] * NR + (int64_t)r_dom[d] * ldH[d]) * es;
            m->phase_bytes[PH_INTERIOR] = 0;
            m->phase_bytes[PH_MODAL] = mb + (int64_t)n_int * 32 + (int64_t)pmr * 32;
            m->phase_bytes[PH_JACOBI] = (int64_t)m->jacobi_omega.size() *
                                        ((int64_t)m->K_col.size() * (4 + 8 + 16) + (int64_t)n_free * (4 + 8 + 16 * 4));
        }

        m->phase_bytes[PH_GATHER] = (int64_t)n_B * (4 + 16 + 16) + ngat * (4 + 16);
        const int64_t ncs = m->cs_n;
        if (m->rows_coarse.n_blocks > 0) {
            m->phase_bytes[PH_COARSE] = plan_bytes(m->rows_coarse) + ncs * 16 + ncs * 16;
            m->phase_bytes[PH_REDUCE] = 0;
        } else {
            m->phase_bytes[PH_COARSE] = ncs * colsS * es + ncs * 16 + (int64_t)m->coarse_nchunks * ncs * 16;
            m->phase_bytes[PH_REDUCE] = (int64_t)m->coarse_nchunks * ncs * 16 + ncs * 16;
        }
        if (two) {
            m->phase_bytes[PH_CONDENSE2] = mat_c2 + (int64_t)(n_B - nT) * 16 + (int64_t)b2all.size() * 16;
            m->phase_bytes[PH_INTERIOR2] = mat_i2 + (int64_t)(n_B - nT) * 32;

            m->phase_bytes[PH_GATHER2] = (int64_t)nT * (4 + 16 + 16) + (int64_t)m->n_gat2 * (4 + 16);
            m->phase_bytes[PH_BACKSUB2] = mat_b2 + (int64_t)b2all.size() * (4 + 16) + (int64_t)(n_B - nT) * 32;
        }
        m->phase_bytes[PH_BACKSUB] = mat_b + nbd_tot * (4 + 16) + (int64_t)n_int * 32;
        m->phase_bytes[PH_RESIDUAL] = nk * (4 + 8 + 16) + nf * (4 + 16 + 16);
        m->phase_bytes[PH_VELOCITY] = nv * 48;
        if (m->use_stream) {
            // matrices once, every x slice read, every output written (and its add read)
            int64_t sb = 0;
            for (const auto& D : m->st_solve.host)
                sb += (int64_t)D.K * D.ld * es + (int64_t)D.K * 16 + (int64_t)D.n_out * (D.akind >= 0 ? 32 : 16);
            m->phase_bytes[PH_SOLVE] = sb;
        }
        int dd = (m->ax_blocks_cond > 0 ? 1 : 0) + (m->ax_blocks_int > 0 ? (m->ax_blocks_int > 3 * m->sms ? 2 : 1) : 0) +
                 (n_B > 0 ? (m->rows_coarse.n_blocks > 0 ? 2 : 3) : 0) + (m->ax_blocks_back > 0 ? 1 : 0);
        if (modal) dd += (m->ax_blocks_m1 > 0 ? 2 : 0) + (int)m->jacobi_omega.size();
        if (two)
            dd += (m->rows_cond2.n_blocks > 0 ? 1 : 0) + (m->rows_int2.n_blocks > 0 ? 1 : 0) + (nT > 0 ? 1 : 0) +
                  (m->rows_back2.n_blocks > 0 ? 1 : 0);
        if (m->use_stream) dd = 1;   // the fused solve
        m->launches_per_iter = 1 + (m->la_shared > 0 ? 1 : 0) + dd + (m->correction ? 1 : 0) + m->refine * (2 + dd);
        for (int k = 0; k < 24; ++k) m->phase_launches[k] = m->phase_bytes[k] > 0 ? 1 : 0;
        if (m->phase_bytes[PH_INTERIOR] > 0 && m->ax_blocks_int > 3 * m->sms) m->phase_launches[PH_INTERIOR] = 2;
        if (m->phase_bytes[PH_RESIDUAL] > 0) m->phase_launches[PH_RESIDUAL] = m->refine;
    }

    // (the flag is read on the mesh's stream, never through the legacy default stream)
    int32_t herr = 0;
    PDG_CUDA(cudaMemcpyAsync(&herr, m->d_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PDG_CUDA(cudaStreamSynchronize(s));
    if (herr & ERR_NOT_SPD) {
        PDG_CUDA(cudaMemsetAsync(m->d_err.p, 0, sizeof(int32_t), s));
        PDG_CUDA(cudaStreamSynchronize(s));
        return fail(PD_ERR_NOT_SPD, "a Cholesky pivot was not positive");
    }
    // load the fixed scratch array of pd_solve_noalloc on this device now,
    // while allocation is allowed (the runtime loads device modules lazily)
    {
        const pd_status ns = noalloc_prepare_device();
        if (ns != PD_OK) return ns;
    }
    m->dt = dt;
    m->prefactored = true;
    m->prefactor_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return PD_OK;
    PD_API_END
}

pd_status pd_set_state(pd_mesh* m, const float* x, const float* v) {
    if (!m) return fail(PD_ERR_INVALID_ARG, "mesh is NULL");
    PD_API_BEGIN
    pdg::AllocStreamScope alloc_scope(m->stream);
    if (x) launch_gather_in(m, x, m->d_x.p, m->stream);
    if (v) launch_gather_in(m, v, m->d_v.p, m->stream);
    ++m->state_gen;
    return PD_OK;
    PD_API_END
}

pd_status pd_get_state(pd_mesh* m, float* x, float* v) {
    if (!m) return fail(PD_ERR_INVALID_ARG, "mesh is NULL");
    PD_API_BEGIN
    pdg::AllocStreamScope alloc_scope(m->stream);
    if (x) launch_scatter_out(m, m->d_x.p, x, 0, m->stream);
    if (v) launch_scatter_out(m, m->d_v.p, v, 0, m->stream);
    return PD_OK;
    PD_API_END
}

}  // extern "C"

static void run_frame(pd_mesh* m, int n_iter, const float g[3], cudaStream_t s) {
    const float h = (float)m->dt;
    phase_begin(m, PH_INERTIA, s);
    launch_inertia(m, h, g[0], g[1], g[2], s);
    phase_end(m, s);
    for (int it = 0; it < n_iter; ++it) {
        m->cur_iter = it;
        // fused local step and assembly: the RHS b, or in the correction form
        // the residual b - K x itself (formed per tet without cancellation)
        phase_begin(m, PH_LOCAL, s);
        launch_local_assemble(m, m->d_x.p, m->d_by0.p, m->d_y.p, m->d_b.p, m->correction, s);
        phase_end(m, s);
        if (m->correction) {
            launch_dd_solve(m, m->d_b.p, m->d_dx.p, s, false);
            launch_axpy_free(m, m->d_dx.p, m->d_x.p, s);
        } else {
            launch_dd_solve(m, m->d_b.p, m->d_x.p, s, false);
        }
        for (int r = 0; r < m->refine; ++r) {
            phase_begin(m, PH_RESIDUAL, s);
            launch_residual(m, m->d_b.p, m->d_x.p, m->d_r.p, s);
            phase_end(m, s);
            launch_dd_solve(m, m->d_r.p, m->d_dx.p, s, false);
            launch_axpy_free(m, m->d_dx.p, m->d_x.p, s);
        }
    }
    m->cur_iter = -1;
    phase_begin(m, PH_VELOCITY, s);
    launch_velocity(m, 1.0f / h, s);
    phase_end(m, s);
}

extern "C" {

pd_status pd_step(pd_mesh* m, const float* pin_targets, const float* gravity, int32_t n_iter, float* x_out) {
    if (!m) return fail(PD_ERR_INVALID_ARG, "mesh is NULL");
    if (!m->prefactored) return fail(PD_ERR_NOT_PREFACTORED, "pd_prefactor has not run since the last change");
    if (n_iter < 1 || n_iter > 1000) return fail(PD_ERR_INVALID_ARG, "n_iter out of range");
    PD_API_BEGIN
    pdg::AllocStreamScope alloc_scope(m->stream);
    float g[3] = {0.f, 0.f, -9.81f};
    if (gravity) {
        g[0] = gravity[0];
        g[1] = gravity[1];
        g[2] = gravity[2];
    }
    cudaStream_t s = m->stream;
    ++m->state_gen;
    if (pin_targets) launch_pin_copy(m, pin_targets, s);
    else launch_pin_hold(m, s);
    if (m->use_graphs) {
        std::vector<uint32_t> key(6);
        key[0] = (uint32_t)n_iter;
        std::memcpy(&key[1], g, sizeof(g));
        key[4] = (uint32_t)m->refine;
        key[5] = (uint32_t)m->timing_mask;
        key.push_back((uint32_t)(m->timing_iter + 1));
        auto it = m->graphs.find(key);
        if (it == m->graphs.end()) {
            cudaGraph_t graph = nullptr;
            auto ts = std::make_shared<pd_mesh::TimingSet>();
            m->timing_armed = m->timing_mask != 0;
            m->ev_rec = ts.get();
            m->ev_open = false;
            PDG_CUDA(cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal));
            try {
                run_frame(m, n_iter, g, m->cap_stream);
            } catch (...) {
                cudaStreamEndCapture(m->cap_stream, &graph);
                if (graph) cudaGraphDestroy(graph);
                m->timing_armed = false;
                m->ev_rec = nullptr;
                throw;
            }
            m->timing_armed = false;
            m->ev_rec = nullptr;
            PDG_CUDA(cudaStreamEndCapture(m->cap_stream, &graph));
            cudaGraphExec_t exec = nullptr;
            cudaError_t e = cudaGraphInstantiate(&exec, graph, m->node_priority ? cudaGraphInstantiateFlagUseNodePriority : 0);
            cudaGraphDestroy(graph);
            PDG_CUDA(e);
            it = m->graphs.emplace(key, pd_mesh::GraphEntry{exec, ts}).first;
        }
        PDG_CUDA(cudaGraphLaunch(it->second.exec, s));
        m->ev_last = it->second.timing;
    } else {
        if (!m->ev_plain) m->ev_plain = std::make_shared<pd_mesh::TimingSet>();
        m->ev_plain->used = 0;
        m->timing_armed = m->timing_mask != 0;
        m->ev_rec = m->ev_plain.get();
        m->ev_open = false;
        try {
            run_frame(m, n_iter, g, s);
        } catch (...) {
            m->timing_armed = false;
            m->ev_rec = nullptr;
            throw;
        }
        m->timing_armed = false;
        m->ev_rec = nullptr;
        m->ev_last = m->ev_plain;
    }
    if (x_out) launch_scatter_out(m, m->d_x.p, x_out, 0, s);
    return PD_OK;
    PD_API_END
}

pd_status pd_sync(pd_mesh* m) {
    if (!m) return fail(PD_ERR_INVALID_ARG, "mesh is NULL");
    PD_API_BEGIN
    pdg::AllocStreamScope alloc_scope(m->stream);
    int32_t herr = 0;
    PDG_CUDA(cudaMemcpyAsync(&herr, m->d_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, m->stream));
    PDG_CUDA(cudaStreamSynchronize(m->stream));
    if (herr) {
        PDG_CUDA(cudaMemsetAsync(m->d_err.p, 0, sizeof(int32_t), m->stream));
        PDG_CUDA(cudaStreamSynchronize(m->stream));
        if (herr & ERR_TIMEOUT) {   // the root cause: the solve's values are not meaningful
            reset_stream_plan(m->st_solve, m->stream);
            PDG_CUDA(cudaStreamSynchronize(m->stream));
            return fail(PD_ERR_TIMEOUT, "a pipeline wait in the subspace solve ran out");
        }
        if (herr & ERR_NONFINITE) return fail(PD_ERR_NONFINITE, "non-finite positions or velocities");
        return fail(PD_ERR_NOT_SPD, "a Cholesky pivot was not positive");
    }
    return PD_OK;
    PD_API_END
}

pd_status pd_get_info(pd_mesh* m, pd_mesh_info* out) {
    if (!m || !out) return fail(PD_ERR_INVALID_ARG, "null argument");
    out->n_vertices = m->n_v;
    out->n_tets = m->n_t;
    out->n_domains = m->n_dom;
    out->n_pinned = m->n_pin;
    out->n_interface = m->n_B;
    out->n_internal = m->n_int;
    int32_t mi = 0, mb = 0;
    for (int32_t d = 0; d < m->n_dom; ++d) {
        mi = std::max(mi, m->dom_n_int[d]);
        mb = std::max(mb, (int32_t)m->dom_bnd[d].size());
    }
    out->max_domain_internal = mi;
    out->max_domain_boundary = mb;
    out->n_groups = m->n_groups;
    out->n_top_interface = m->n_groups > 0 ? m->n_top : 0;
    out->two_level = m->two_level ? 1 : 0;
    int64_t bytes = 0;
    bytes += m->d_tets.bytes() + m->d_geo.bytes() + m->d_x.bytes() + m->d_xprev.bytes() + m->d_v.bytes();
    bytes += m->d_force.bytes() + m->d_by0.bytes() + m->d_b.bytes() + m->d_pin_tgt.bytes() + m->d_mh2.bytes();
    bytes += m->d_inc_ptr.bytes() + m->d_inc.bytes() + m->d_kfp_ptr.bytes() + m->d_kfp_col.bytes();
    bytes += m->d_kfp_val.bytes() + m->d_old_of_new.bytes() + m->d_mat32.bytes() + m->d_mat16.bytes();
    bytes += m->d_ax_desc_cond.bytes() + m->d_ax_desc_back.bytes() + m->d_ax_blk_cond.bytes();
    bytes += m->d_ax_desc_int.bytes() + m->d_ax_blk_int.bytes() + m->rows_int2.descs.bytes() + m->rows_int2.blk_u.bytes();
    bytes += m->d_ax_blk_back.bytes() + m->d_tc.bytes() + m->d_bidx.bytes();
    bytes += m->d_gat_ptr.bytes() + m->d_gat.bytes() + m->d_cB.bytes() + m->d_part.bytes();
    bytes += m->d_K_ptr.bytes() + m->d_K_col.bytes() + m->d_K_val.bytes() + m->d_r.bytes() + m->d_dx.bytes();
    bytes += m->rows_cond2.descs.bytes() + m->rows_cond2.blk_u.bytes() + m->rows_back2.descs.bytes();
    bytes += m->rows_coarse.descs.bytes() + m->rows_coarse.blk_u.bytes();
    bytes += m->rows_back2.blk_u.bytes() + m->d_bidx2.bytes() + m->d_gat2_ptr.bytes() + m->d_gat2.bytes();
    bytes += m->d_tc2.bytes() + m->d_cT.bytes();
    bytes += m->st_solve.pan32.bytes() + m->st_solve.pan16.bytes() + m->st_solve.recs.bytes() +
             m->st_solve.part.bytes() + m->st_solve.cnt.bytes();
    out->device_bytes = bytes;
    out->prefactor_seconds = m->prefactor_seconds;
    out->launches_per_iter = m->launches_per_iter;
    out->launches_per_frame = 3;   // pin copy (or hold), inertia, velocity
    for (int k = 0; k < 24; ++k) out->phase_bytes[k] = m->phase_bytes[k];
    for (int k = 0; k < 24; ++k) out->phase_launches[k] = m->phase_launches[k];
    return PD_OK;
}

pd_status pd_project(const float* F, int32_t n, float* R, float* V, float* sigma, void* stream) {
    if (n < 0 || (n > 0 && !F)) return fail(PD_ERR_INVALID_ARG, "bad arguments");
    PD_API_BEGIN
    launch_project(F, n, R, V, sigma, static_cast<cudaStream_t>(stream));
    return PD_OK;
    PD_API_END
}

pd_status pd_local_rhs(pd_mesh* m, const float* x, const float* y, float* b) {
    if (!m || !x || !y || !b) return fail(PD_ERR_INVALID_ARG, "null argument");
    if (!m->prefactored) return fail(PD_ERR_NOT_PREFACTORED, "pd_prefactor has not run");
    PD_API_BEGIN
    pdg::AllocStreamScope alloc_scope(m->stream);
    cudaStream_t s = m->stream;
    DBuf<float4> xi, yi, by0, bb, frc;
    xi.alloc(m->n_v);
    yi.alloc(m->n_v);
    by0.alloc(std::max(m->n_free, 1));
    bb.alloc(m->n_v);
    frc.alloc(4 * (size_t)m->n_t);
    launch_gather_in(m, x, xi.p, s);
    launch_gather_in(m, y, yi.p, s);
    // pinned positions for the K_fp term come from x
    if (m->n_pin > 0)
        PDG_CUDA(cudaMemcpyAsync(m->d_pin_tgt.p, xi.p + m->n_free, sizeof(float4) * m->n_pin,
                                 cudaMemcpyDeviceToDevice, s));
    launch_by0_from_y(m, yi.p, by0.p, s);
    launch_local_assemble(m, xi.p, by0.p, nullptr, bb.p, false, s);
    launch_scatter_out(m, bb.p, b, 1, s);
    PDG_CUDA(cudaStreamSynchronize(s));
    return PD_OK;
    PD_API_END
}

pd_status pd_solve(pd_mesh* m, const float* r, float* x) {
    if (!m || !r || !x) return fail(PD_ERR_INVALID_ARG, "null argument");
    if (!m->prefactored) return fail(PD_ERR_NOT_PREFACTORED, "pd_prefactor has not run");
    PD_API_BEGIN
    pdg::AllocStreamScope alloc_scope(m->stream);
    cudaStream_t s = m->stream;
    DBuf<float4> ri, xi;
    ri.alloc(m->n_v);
    xi.alloc(m->n_v);
    PDG_CUDA(cudaMemsetAsync(xi.p, 0, sizeof(float4) * m->n_v, s));
    launch_gather_in(m, r, ri.p, s);
    launch_dd_solve(m, ri.p, xi.p, s, false);
    for (int k = 0; k < m->refine; ++k) {
        DBuf<float4> rr, dx;
        rr.alloc(std::max(m->n_free, 1));
        dx.alloc(m->n_v);
        launch_residual(m, ri.p, xi.p, rr.p, s);
        launch_dd_solve(m, rr.p, dx.p, s, false);
        launch_axpy_free(m, dx.p, xi.p, s);
        PDG_CUDA(cudaStreamSynchronize(s));
    }
    launch_scatter_out(m, xi.p, x, 1, s);
    PDG_CUDA(cudaStreamSynchronize(s));
    return PD_OK;
    PD_API_END
}

pd_status pd_enable_timing(pd_mesh* m, int32_t mask) {
    if (!m) return fail(PD_ERR_INVALID_ARG, "mesh is NULL");
    m->timing_mask = mask < 0 ? ((1 << PH_COUNT) - 1) : (mask & ((1 << PH_COUNT) - 1));
    return PD_OK;
}

pd_status pd_set_timing_iteration(pd_mesh* m, int32_t iteration) {
    if (!m) return fail(PD_ERR_INVALID_ARG, "mesh is NULL");
    if (iteration < -1) return fail(PD_ERR_INVALID_ARG, "iteration must be >= -1");
    m->timing_iter = iteration;
    return PD_OK;
}

pd_status pd_test_offset_phase_counter(pd_mesh* m, int32_t phase, int32_t delta) {
    if (!m || !m->use_stream || phase < 0 || phase >= m->st_solve.n_phases)
        return fail(PD_ERR_INVALID_ARG, "no streaming plan or phase out of range");
    PD_API_BEGIN
    pdg::AllocStreamScope alloc_scope(m->stream);
    PDG_CUDA(cudaStreamSynchronize(m->stream));
    int32_t v = 0;
    PDG_CUDA(cudaMemcpy(&v, m->st_solve.phase_cnt.p + phase, sizeof(int32_t), cudaMemcpyDeviceToHost));
    v += delta;
    PDG_CUDA(cudaMemcpy(m->st_solve.phase_cnt.p + phase, &v, sizeof(int32_t), cudaMemcpyHostToDevice));
    return PD_OK;
    PD_API_END
}

pd_status pd_test_inflate_copy(pd_mesh* m, int32_t bytes) {
    if (!m || !m->ax_tiled || bytes < 0 || bytes % 16 != 0)
        return fail(PD_ERR_INVALID_ARG, "no tile-streaming products, or bytes not a non-negative multiple of 16");
    PD_API_BEGIN
    pdg::AllocStreamScope alloc_scope(m->stream);
    test_set_copy_extra(bytes, m->stream);
    return PD_OK;
    PD_API_END
}

pd_status pd_phase_times(pd_mesh* m, float* out, int32_t n_out, int32_t* n_phases) {
    if (!m) return fail(PD_ERR_INVALID_ARG, "mesh is NULL");
    PD_API_BEGIN
    pdg::AllocStreamScope alloc_scope(m->stream);
    if (n_phases) *n_phases = PH_COUNT;
    std::vector<double> sum(PH_COUNT, 0.0);
    std::vector<int> cnt(PH_COUNT, 0);
    PDG_CUDA(cudaStreamSynchronize(m->stream));
    const pd_mesh::TimingSet* T = m->ev_last.get();
    for (int32_t k = 0; T && k < T->used; ++k) {
        float ms = 0.f;
        cudaError_t e = cudaEventElapsedTime(&ms, T->ev[2 * k], T->ev[2 * k + 1]);
        if (e != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        sum[T->phase[k]] += ms;
        cnt[T->phase[k]]++;
    }
    for (int32_t p = 0; p < n_out && p < PH_COUNT; ++p) out[p] = cnt[p] ? (float)(sum[p] / cnt[p]) : 0.f;
    return PD_OK;
    PD_API_END
}

}  // extern "C"
