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
        PDG_CUDA(cudaMemcpyAsync(a->vprev.p, m->d_v.p, sizeof(float4) * m->n_v, cudaMemcpyDeviceToDevice, s));
        pd_status st = pd_step(m, pin_targets, g, n_pd_iter, nullptr);
        if (st != PD_OK) return st;
        const float h = (float)m->dt;
        for (int k = 0; k < n_newton; ++k) {
            launch_grad_local(m, m->d_x.p, m->d_force.p, s);
            launch_assemble_residual(m, m->d_force.p, m->d_x.p, m->d_xprev.p, a->vprev.p, h, g, -1.f, a->rhs.p, s);
            adjoint_pcg(m, a, m->d_x.p, a->rhs.p, a->dx.p, s);
            launch_axpy_free(m, a->dx.p, m->d_x.p, s);
        }
        launch_velocity(m, 1.0f / h, s);
        if (x_out) launch_scatter_out(m, m->d_x.p, x_out, 0, s);
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
        launch_gather_in(m, x_n, a->xeq.p, s);
        launch_gather_in(m, dL_dx, a->g.p, s);
        launch_adj_rhs(m->n_free, a->g.p, m->d_mh2.p, a->lam1.p, a->lam2.p, a->rhs.p, s);
        adjoint_pcg(m, a, a->xeq.p, a->rhs.p, a->lam.p, s);
        launch_grad_gamma(m, a->vol.p, a->user_of_tet.p, a->xeq.p, a->lam.p, dL_dgamma_s, dL_dgamma_v, s);
        const size_t bytes = sizeof(float4) * m->n_v;
        PDG_CUDA(cudaMemcpyAsync(a->lam2.p, a->lam1.p, bytes, cudaMemcpyDeviceToDevice, s));
        PDG_CUDA(cudaMemcpyAsync(a->lam1.p, a->lam.p, bytes, cudaMemcpyDeviceToDevice, s));
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
