// Adjoint path of the C ABI: equilibrium time steps (PD iterations followed
// by Newton steps on Eq. g) and the backward adjoint step of Sec. 6.1
// (Eq. adjoint_state_solve, Eq. adjoint_state).  Linear systems with the
// true Hessian are solved by preconditioned CG whose preconditioner is the
// PD subspace solve of the mesh (K^-1 with K the PD matrix), with every CG
// scalar kept on the device.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pd_internal.h"

namespace pdg {

void launch_grad_local(const pd_mesh* m, const float4* x, float4* force, cudaStream_t s);
void launch_assemble_residual(const pd_mesh* m, const float4* force, const float4* x, const float4* xprev,
                              const float4* vprev, float h, const float g[3], float sign, float4* out,
                              cudaStream_t s);
void launch_hvp(const pd_mesh* m, const float4* x, const float4* v, float4* force, float4* out, cudaStream_t s);
void launch_grad_gamma(const pd_mesh* m, const float* vol, const int* user_of_tet, const float4* x,
                       const float4* lam, float* gs, float* gv, cudaStream_t s);
int dot_blocks();
void launch_dot(int n, const float4* a, const float4* b, double* partial, double* sc, int mode, int dst,
                cudaStream_t s);
void launch_cg_update(int n, const double* sc, const float4* p, const float4* Ap, float4* x, float4* r,
                      cudaStream_t s);
void launch_cg_direction(int n, const double* sc, const float4* z, float4* p, int beta_zero, cudaStream_t s);
void launch_adj_rhs(int n, const float4* dldx, const float* mh2, const float4* lam1, const float4* lam2, float4* rhs,
                    cudaStream_t s);
void launch_grad_local64(const pd_mesh* m, const double* geo64, const double* x64, double* force64, cudaStream_t s);
void launch_residual_rhs64(const pd_mesh* m, const double* force64, const double* mh2, const double* x64,
                           const double* xprev64, const double* vprev64, double h, const float g[3], float4* out,
                           cudaStream_t s);
void launch_hvp_residual64(const pd_mesh* m, const double* geo64, const double* x64, const float4* lam,
                           const double* mh2, const float4* rhs, double* force64, float4* out, cudaStream_t s);
void launch_grad_gamma64(const pd_mesh* m, const double* geo64, const int* user_of_tet, const double* x64,
                         const float4* lam, float* gs, float* gv, cudaStream_t s);
void launch_f4_to_d(int n, const float4* a, double* out, cudaStream_t s);
void launch_d_to_f4(int n, const double* a, float4* out, cudaStream_t s);
void launch_newton_update64(int n_free, const float4* dx, double* x64, float4* x32, cudaStream_t s);
void launch_velocity64(int n_v, const double* x64, const double* xprev64, double h, double* v64, float4* x32,
                       float4* v32, cudaStream_t s);
void launch_gather64(const pd_mesh* m, const double* src, double* dst, cudaStream_t s);
void launch_scatter64(const pd_mesh* m, const double* src, double* dst, cudaStream_t s);
void launch_add_f4(int n, const float4* d, float4* x, cudaStream_t s);

}  // namespace pdg

using namespace pdg;

static pd_status afail(pd_status c, const char* msg) {
    set_error(msg);
    return c;
}

namespace pdg {

// x = H(x_lin)^-1 b by PCG (fixed iteration count), preconditioner = PD subspace solve.
void adjoint_pcg(pd_mesh* m, pd_adjoint* a, const float4* x_lin, const float4* b, float4* x, cudaStream_t s) {
    const int n = m->n_free;
    PDG_CUDA(cudaMemsetAsync(x, 0, sizeof(float4) * m->n_v, s));
    if (n <= 0) return;
    PDG_CUDA(cudaMemcpyAsync(a->r.p, b, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s));
    launch_dd_solve(m, a->r.p, a->z.p, s, false);
    launch_cg_direction(n, a->sc.p, a->z.p, a->p.p, 1, s);
    launch_dot(n, a->r.p, a->z.p, a->partial.p, a->sc.p, 0, 0, s);
    for (int k = 0; k < a->cg_iters; ++k) {
        launch_hvp(m, x_lin, a->p.p, m->d_force.p, a->Ap.p, s);
        launch_dot(n, a->p.p, a->Ap.p, a->partial.p, a->sc.p, 1, 0, s);
        launch_cg_update(n, a->sc.p, a->p.p, a->Ap.p, x, a->r.p, s);
        launch_dd_solve(m, a->r.p, a->z.p, s, false);
        launch_dot(n, a->r.p, a->z.p, a->partial.p, a->sc.p, 2, 0, s);
        launch_cg_direction(n, a->sc.p, a->z.p, a->p.p, 0, s);
    }
}

// FP64 side of the workspace: buffers on first use, per-tet operators after
// every material change, M/dt^2 after every change of dt.
static void ensure64(pd_mesh* m, pd_adjoint* a, cudaStream_t s) {
    const size_t nv3 = 3 * (size_t)m->n_v;
    if (!a->x64.p) {
        DBuf<double>* vecs[] = {&a->x64, &a->v64, &a->xprev64, &a->vprev64, &a->xa64};
        for (auto* b : vecs) b->alloc(nv3);
        a->force64.alloc(12 * (size_t)std::max(m->n_t, 1));
        a->rhs2.alloc(m->n_v);
        a->dlam.alloc(m->n_v);
        PDG_CUDA(cudaMemsetAsync(a->dlam.p, 0, sizeof(float4) * m->n_v, s));
    }
    if (a->mat_gen64 != m->mat_gen) {
        std::vector<double> g(12 * (size_t)m->n_t);
        for (int32_t t = 0; t < m->n_t; ++t) {
            double* q = &g[12 * (size_t)t];
            for (int k = 0; k < 9; ++k) q[k] = m->Dminv[9 * (size_t)t + k];
            q[9] = m->vol[t] * (double)m->gamma_s[t];
            q[10] = m->vol[t] * (double)m->gamma_v[t];
            q[11] = m->vol[t];
        }
        upload(a->geo64, g, s);
        PDG_CUDA(cudaStreamSynchronize(s));   // the host vector is released on return
        a->mat_gen64 = m->mat_gen;
    }
    if (a->dt64 != m->dt) {
        std::vector<double> mh2((size_t)std::max(m->n_free, 1), 0.0);
        for (int32_t i = 0; i < m->n_free; ++i) mh2[i] = m->mass[i] / (m->dt * m->dt);
        upload(a->mh2_64, mh2, s);
        PDG_CUDA(cudaStreamSynchronize(s));
        a->dt64 = m->dt;
    }
}

// The FP64 state follows the mesh's FP32 state unless it was set or advanced
// by the adjoint workspace itself since the last change of the FP32 state.
static void sync64(pd_mesh* m, pd_adjoint* a, cudaStream_t s) {
    if (a->gen64 == m->state_gen) return;
    launch_f4_to_d(m->n_v, m->d_x.p, a->x64.p, s);
    launch_f4_to_d(m->n_v, m->d_v.p, a->v64.p, s);
    a->gen64 = m->state_gen;
}

// One backward step at the FP64 state a->xa64 (library order): the adjoint
// state by FP32 PCG plus one FP64 refinement, then the FP64 sensitivities.
static void adjoint_step64(pd_mesh* m, pd_adjoint* a, const float* dL_dx, float* gs, float* gv, cudaStream_t s) {
    launch_d_to_f4(m->n_v, a->xa64.p, a->xeq.p, s);
    launch_gather_in(m, dL_dx, a->g.p, s);
    launch_adj_rhs(m->n_free, a->g.p, m->d_mh2.p, a->lam1.p, a->lam2.p, a->rhs.p, s);
    adjoint_pcg(m, a, a->xeq.p, a->rhs.p, a->lam.p, s);
    // r = rhs - H(x64) lambda with FP64 per-tet terms and sums; lambda += H^-1 r
    launch_hvp_residual64(m, a->geo64.p, a->xa64.p, a->lam.p, a->mh2_64.p, a->rhs.p, a->force64.p, a->rhs2.p, s);
    adjoint_pcg(m, a, a->xeq.p, a->rhs2.p, a->dlam.p, s);
    launch_add_f4(m->n_free, a->dlam.p, a->lam.p, s);
    launch_grad_gamma64(m, a->geo64.p, a->user_of_tet.p, a->xa64.p, a->lam.p, gs, gv, s);
    const size_t bytes = sizeof(float4) * m->n_v;
    PDG_CUDA(cudaMemcpyAsync(a->lam2.p, a->lam1.p, bytes, cudaMemcpyDeviceToDevice, s));
    PDG_CUDA(cudaMemcpyAsync(a->lam1.p, a->lam.p, bytes, cudaMemcpyDeviceToDevice, s));
}

}  // namespace pdg

extern "C" {

pd_status pd_adjoint_create(pd_mesh* m, int32_t cg_iters, pd_adjoint** out) {
    if (!m || !out) return afail(PD_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (cg_iters < 1 || cg_iters > 500) return afail(PD_ERR_INVALID_ARG, "cg_iters out of range [1, 500]");
    pd_adjoint* a = new (std::nothrow) pd_adjoint();
    if (!a) return afail(PD_ERR_NO_MEMORY, "host allocation failed");
    try {
        a->mesh = m;
        a->cg_iters = cg_iters;
        const size_t nv = (size_t)m->n_v;
        DBuf<float4>* bufs[] = {&a->xeq, &a->vprev, &a->g, &a->rhs, &a->lam, &a->lam1, &a->lam2,
                                &a->r, &a->z, &a->p, &a->Ap, &a->dx};
        for (auto* b : bufs) {
            b->alloc(nv);
            PDG_CUDA(cudaMemsetAsync(b->p, 0, sizeof(float4) * nv, m->stream));
        }
        a->partial.alloc(dot_blocks());
        a->sc.alloc(8);
        PDG_CUDA(cudaMemsetAsync(a->sc.p, 0, sizeof(double) * 8, m->stream));
        std::vector<float> vol(m->n_t);
        for (int32_t t = 0; t < m->n_t; ++t) vol[t] = (float)m->vol[t];
        a->vol.alloc(m->n_t);
        a->user_of_tet.alloc(m->n_t);
        PDG_CUDA(cudaMemcpyAsync(a->vol.p, vol.data(), sizeof(float) * m->n_t, cudaMemcpyHostToDevice, m->stream));
        PDG_CUDA(cudaMemcpyAsync(a->user_of_tet.p, m->tet_old_of_new.data(), sizeof(int32_t) * m->n_t,
                                 cudaMemcpyHostToDevice, m->stream));
        PDG_CUDA(cudaStreamSynchronize(m->stream));
    } catch (const Fail& f) {
        delete a;
        return f.code;
    }
    *out = a;
    return PD_OK;
}

void pd_adjoint_destroy(pd_adjoint* a) {
    if (!a) return;
    if (a->mesh) cudaStreamSynchronize(a->mesh->stream);
    delete a;
}

pd_status pd_adjoint_reset(pd_adjoint* a) {
    if (!a) return afail(PD_ERR_INVALID_ARG, "null argument");
    try {
        const size_t nv = (size_t)a->mesh->n_v;
        PDG_CUDA(cudaMemsetAsync(a->lam1.p, 0, sizeof(float4) * nv, a->mesh->stream));
        PDG_CUDA(cudaMemsetAsync(a->lam2.p, 0, sizeof(float4) * nv, a->mesh->stream));
    } catch (const Fail& f) {
        return f.code;
    }
    return PD_OK;
}

pd_status pd_equilibrium_step(pd_mesh* m, pd_adjoint* a, const float* pin_targets, const float* gravity,
                              int32_t n_pd_iter, int32_t n_newton, float* x_out) {
    if (!m || !a || a->mesh != m) return afail(PD_ERR_INVALID_ARG, "bad mesh / workspace");
    if (!m->prefactored) return afail(PD_ERR_NOT_PREFACTORED, "pd_prefactor has not run");
    if (n_newton < 0 || n_newton > 50) return afail(PD_ERR_INVALID_ARG, "n_newton out of range [0, 50]");
    float g[3] = {0.f, 0.f, -9.81f};
    if (gravity) {
        g[0] = gravity[0];
        g[1] = gravity[1];
        g[2] = gravity[2];
    }
    try {
        cudaStream_t s = m->stream;
        ensure64(m, a, s);
        sync64(m, a, s);
        const size_t nv3 = 3 * sizeof(double) * (size_t)m->n_v;
        PDG_CUDA(cudaMemcpyAsync(a->xprev64.p, a->x64.p, nv3, cudaMemcpyDeviceToDevice, s));
        PDG_CUDA(cudaMemcpyAsync(a->vprev64.p, a->v64.p, nv3, cudaMemcpyDeviceToDevice, s));
        // PD iterations in FP32 give the starting point (and the pinned targets)
        pd_status st = pd_step(m, pin_targets, g, n_pd_iter, nullptr);
        if (st != PD_OK) return st;
        launch_f4_to_d(m->n_v, m->d_x.p, a->x64.p, s);
        // Newton on Eq. g: FP64 residual at the FP64 state, FP32 PCG for the
        // correction (preconditioner: the PD subspace solve)
        for (int k = 0; k < n_newton; ++k) {
            launch_grad_local64(m, a->geo64.p, a->x64.p, a->force64.p, s);
            launch_residual_rhs64(m, a->force64.p, a->mh2_64.p, a->x64.p, a->xprev64.p, a->vprev64.p, m->dt, g,
                                  a->rhs.p, s);
            adjoint_pcg(m, a, m->d_x.p, a->rhs.p, a->dx.p, s);
            launch_newton_update64(m->n_free, a->dx.p, a->x64.p, m->d_x.p, s);
        }
        launch_velocity64(m->n_v, a->x64.p, a->xprev64.p, m->dt, a->v64.p, m->d_x.p, m->d_v.p, s);
        a->gen64 = ++m->state_gen;
        if (x_out) launch_scatter_out(m, m->d_x.p, x_out, 0, s);
    } catch (const Fail& f) {
        return f.code;
    }
    return PD_OK;
}

pd_status pd_adjoint_get_state64(pd_adjoint* a, double* x, double* v) {
    if (!a || !a->mesh) return afail(PD_ERR_INVALID_ARG, "null argument");
    pd_mesh* m = a->mesh;
    try {
        cudaStream_t s = m->stream;
        ensure64(m, a, s);
        sync64(m, a, s);
        if (x) launch_scatter64(m, a->x64.p, x, s);
        if (v) launch_scatter64(m, a->v64.p, v, s);
    } catch (const Fail& f) {
        return f.code;
    }
    return PD_OK;
}

pd_status pd_adjoint_set_state64(pd_adjoint* a, const double* x, const double* v) {
    if (!a || !a->mesh || !x || !v) return afail(PD_ERR_INVALID_ARG, "null argument");
    pd_mesh* m = a->mesh;
    try {
        cudaStream_t s = m->stream;
        ensure64(m, a, s);
        launch_gather64(m, x, a->x64.p, s);
        launch_gather64(m, v, a->v64.p, s);
        launch_d_to_f4(m->n_v, a->x64.p, m->d_x.p, s);
        launch_d_to_f4(m->n_v, a->v64.p, m->d_v.p, s);
        a->gen64 = ++m->state_gen;
    } catch (const Fail& f) {
        return f.code;
    }
    return PD_OK;
}

pd_status pd_adjoint_step(pd_mesh* m, pd_adjoint* a, const float* x_n, const float* dL_dx, float* dL_dgamma_s,
                          float* dL_dgamma_v) {
    if (!m || !a || a->mesh != m || !x_n || !dL_dx || !dL_dgamma_s || !dL_dgamma_v)
        return afail(PD_ERR_INVALID_ARG, "null argument or mismatched workspace");
    if (!m->prefactored) return afail(PD_ERR_NOT_PREFACTORED, "pd_prefactor has not run");
    try {
        cudaStream_t s = m->stream;
        ensure64(m, a, s);
        launch_gather_in(m, x_n, a->xeq.p, s);
        launch_f4_to_d(m->n_v, a->xeq.p, a->xa64.p, s);
        adjoint_step64(m, a, dL_dx, dL_dgamma_s, dL_dgamma_v, s);
    } catch (const Fail& f) {
        return f.code;
    }
    return PD_OK;
}

pd_status pd_adjoint_step64(pd_mesh* m, pd_adjoint* a, const double* x_n, const float* dL_dx, float* dL_dgamma_s,
                            float* dL_dgamma_v) {
    if (!m || !a || a->mesh != m || !x_n || !dL_dx || !dL_dgamma_s || !dL_dgamma_v)
        return afail(PD_ERR_INVALID_ARG, "null argument or mismatched workspace");
    if (!m->prefactored) return afail(PD_ERR_NOT_PREFACTORED, "pd_prefactor has not run");
    try {
        cudaStream_t s = m->stream;
        ensure64(m, a, s);
        launch_gather64(m, x_n, a->xa64.p, s);
        adjoint_step64(m, a, dL_dx, dL_dgamma_s, dL_dgamma_v, s);
    } catch (const Fail& f) {
        return f.code;
    }
    return PD_OK;
}

pd_status pd_hessian_vec(pd_mesh* m, const float* x, const float* v, float* Hv) {
    if (!m || !x || !v || !Hv) return afail(PD_ERR_INVALID_ARG, "null argument");
    if (!m->prefactored) return afail(PD_ERR_NOT_PREFACTORED, "pd_prefactor has not run");
    try {
        cudaStream_t s = m->stream;
        DBuf<float4> xi, vi, out;
        xi.alloc(m->n_v);
        vi.alloc(m->n_v);
        out.alloc(m->n_v);
        launch_gather_in(m, x, xi.p, s);
        launch_gather_in(m, v, vi.p, s);
        if (m->n_pin > 0)   // directions vanish on pinned vertices
            PDG_CUDA(cudaMemsetAsync(vi.p + m->n_free, 0, sizeof(float4) * m->n_pin, s));
        launch_hvp(m, xi.p, vi.p, m->d_force.p, out.p, s);
        launch_scatter_out(m, out.p, Hv, 1, s);
        PDG_CUDA(cudaStreamSynchronize(s));
    } catch (const Fail& f) {
        return f.code;
    }
    return PD_OK;
}

pd_status pd_residual(pd_mesh* m, const float* x, const float* x_prev, const float* v_prev, const float* gravity,
                      float* g_out) {
    if (!m || !x || !x_prev || !v_prev || !g_out) return afail(PD_ERR_INVALID_ARG, "null argument");
    if (!m->prefactored) return afail(PD_ERR_NOT_PREFACTORED, "pd_prefactor has not run");
    float g[3] = {0.f, 0.f, -9.81f};
    if (gravity) {
        g[0] = gravity[0];
        g[1] = gravity[1];
        g[2] = gravity[2];
    }
    try {
        cudaStream_t s = m->stream;
        DBuf<float4> xi, xp, vp, out;
        xi.alloc(m->n_v);
        xp.alloc(m->n_v);
        vp.alloc(m->n_v);
        out.alloc(m->n_v);
        launch_gather_in(m, x, xi.p, s);
        launch_gather_in(m, x_prev, xp.p, s);
        launch_gather_in(m, v_prev, vp.p, s);
        launch_grad_local(m, xi.p, m->d_force.p, s);
        launch_assemble_residual(m, m->d_force.p, xi.p, xp.p, vp.p, (float)m->dt, g, 1.f, out.p, s);
        launch_scatter_out(m, out.p, g_out, 1, s);
        PDG_CUDA(cudaStreamSynchronize(s));
    } catch (const Fail& f) {
        return f.code;
    }
    return PD_OK;
}

}  // extern "C"
