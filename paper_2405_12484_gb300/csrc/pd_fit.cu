// Material fitting of the C ABI: the adjoint Gauss-Newton direction
// (Sec. 6.2: Eq. gn solved through the eliminated block system of Eq. agn,
// with the Levenberg-Marquardt shift) and the two-stage fitting loop with
// line search and the non-negativity projection / pivoting (Sec. 6.3).
//
// Every vector operation runs in the kernels of k_adjoint.cu; the host
// decides only what the loop does next from scalars it reads back (a loss,
// a descent test, a pivot index).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "pd_internal.h"

namespace pdg {

int dot_blocks();
void launch_dot(int n, const float4* a, const float4* b, double* partial, double* sc, int mode, int dst,
                cudaStream_t s);
int gn_scalar_count();
int gn_partial_blocks();
void launch_gn_setup(const pd_mesh* m, const float* vol, const float4* x, float* Ts, float* Tv, cudaStream_t s);
void launch_gn_bv(const pd_mesh* m, const float* Ts, const float* Tv, const int* user_of_tet, const float* v,
                  float4* force, float4* out, cudaStream_t s);
void launch_normalize_f4(int n, const double* sc, int idx, float4* x, cudaStream_t s);
void launch_gn_btv(const pd_mesh* m, const float* Ts, const float* Tv, const int* user_of_tet, const float4* nu,
                   const uint8_t* active, const double* sc, int i1, int i2, float gs, float* out, cudaStream_t s);
void launch_pdot(int n, const float* a, const float* b, const uint8_t* mask, int mode, int op, int dst, double kr,
                 double* partial, double* sc, cudaStream_t s);
void launch_gn_init(int n, const float* g, const uint8_t* active, const double* sc, float* r, float* p, float* d,
                    cudaStream_t s);
void launch_gn_ap(int n, const double* sc, const float* q, const float* p, float* ap, cudaStream_t s);
void launch_gn_update(int n, const double* sc, const float* p, const float* ap, float* d, float* r, cudaStream_t s);
void launch_gn_pdir(int n, const double* sc, const float* r, float* p, cudaStream_t s);
void launch_pscale(int n, const double* sc, int idx, int mode, const uint8_t* active, const float* src, float* x,
                   cudaStream_t s);
void launch_clamp_dir(int n, const float* raw, const uint8_t* clamped, float* d, cudaStream_t s);
void launch_project(int n, const float* gamma, const float* d, float alpha, float fl, float* trial, uint8_t* neg,
                    cudaStream_t s);
void launch_accept(int n, const float* trial, const uint8_t* neg, float* gamma, uint8_t* clamped, cudaStream_t s);
void launch_pick_pivot(int n, const float* gamma, const float* raw, const uint8_t* clamped, const uint8_t* active,
                       float fl, double* pval, int* pidx, int* out, cudaStream_t s);
void launch_pcopy(int n, float sign, const float* a, const uint8_t* active, float* out, cudaStream_t s);
void launch_misfit(int n_free, const float4* x, const float4* xhat, float4* dldx, double* partial, double* sc, int dst,
                   cudaStream_t s, bool accumulate = false);
void launch_tied_gradient(int n, const float* gs, const float* gv, double ratio, const double* scale, float* out,
                          cudaStream_t s);
void launch_basis_t(int n_t, int r, const float* H, const float* w, double* out, cudaStream_t s);
void launch_basis_apply(int n_t, int r, const float* H, const double* q, float* out, cudaStream_t s);
void launch_basis_col(int n_t, int r, const float* H, int j, float* out, cudaStream_t s);
void launch_count_below(int n, const float* a, float fl, int* count, cudaStream_t s);

// indices of the FP64 scalars of the outer CG (k_adjoint.cu, GnScalar)
enum : int { S_RR = 0, S_PAP, S_ALPHA, S_BETA, S_KAPPA, S_GG, S_N1, S_N2, S_TMP, S_MAX };

}  // namespace pdg

using namespace pdg;

static pd_status ffail(pd_status c, const char* msg) {
    set_error(msg);
    return c;
}

// Allocate the Gauss-Newton buffers of a workspace (first use).
static void gn_prepare(pd_mesh* m, pd_adjoint* a) {
    if (a->gn_ready) return;
    const size_t nt = (size_t)m->n_t, np = 2 * nt;
    a->gn_Ts.alloc(9 * nt);
    a->gn_Tv.alloc(9 * nt);
    for (auto* b : {&a->gn_r, &a->gn_p, &a->gn_q, &a->gn_ap, &a->gn_tmp}) b->alloc(np);
    for (auto* b : {&a->gn_b, &a->gn_mu, &a->gn_nu}) {
        b->alloc(m->n_v);
        PDG_CUDA(cudaMemsetAsync(b->p, 0, sizeof(float4) * m->n_v, m->stream));
    }
    a->gn_sc.alloc(gn_scalar_count());
    PDG_CUDA(cudaMemsetAsync(a->gn_sc.p, 0, sizeof(double) * gn_scalar_count(), m->stream));
    a->gn_partial.alloc(std::max(gn_partial_blocks(), dot_blocks()));
    a->gn_ipartial.alloc(gn_partial_blocks() + 1);
    a->gn_ready = true;
}

// Per-tet V_e (F - R), V_e (F - V) at the positions a->xeq (internal order).
static void gn_setup(pd_mesh* m, pd_adjoint* a, cudaStream_t s) {
    launch_gn_setup(m, a->vol.p, a->xeq.p, a->gn_Ts.p, a->gn_Tv.p, s);
}

// out = P v (v already zero on inactive parameters; out masked by `active`).
static void gn_apply(pd_mesh* m, pd_adjoint* a, const float* v, const uint8_t* active, float g_scale, float* out,
                     cudaStream_t s) {
    const int nf = m->n_free;
    double* sc = a->gn_sc.p;
    launch_gn_bv(m, a->gn_Ts.p, a->gn_Tv.p, a->user_of_tet.p, v, m->d_force.p, a->gn_b.p, s);
    launch_dot(nf, a->gn_b.p, a->gn_b.p, a->gn_partial.p, sc, 0, S_N1, s);
    launch_normalize_f4(nf, sc, S_N1, a->gn_b.p, s);
    adjoint_pcg(m, a, a->xeq.p, a->gn_b.p, a->gn_mu.p, s);      // mu / |B v|
    launch_dot(nf, a->gn_mu.p, a->gn_mu.p, a->gn_partial.p, sc, 0, S_N2, s);
    launch_normalize_f4(nf, sc, S_N2, a->gn_mu.p, s);
    adjoint_pcg(m, a, a->xeq.p, a->gn_mu.p, a->gn_nu.p, s);     // nu / (g_scale |B v| |mu|)
    launch_gn_btv(m, a->gn_Ts.p, a->gn_Tv.p, a->user_of_tet.p, a->gn_nu.p, active, sc, S_N1, S_N2, g_scale, out, s);
}

// (P + kappa I) d = -grad on the active set by `iters` CG iterations; a->xeq and
// the per-tet setup must be current.  kappa = kappa_rel g^T P g / g^T g.
static void gn_direction(pd_mesh* m, pd_adjoint* a, const float* grad, const uint8_t* active, double kappa_rel,
                         float g_scale, int iters, float* d, cudaStream_t s) {
    const int np = 2 * m->n_t;
    double* sc = a->gn_sc.p;
    double* part = a->gn_partial.p;
    launch_pdot(np, grad, grad, active, 0, 0, S_GG, 0.0, part, sc, s);
    launch_gn_init(np, grad, active, sc, a->gn_r.p, a->gn_p.p, a->gn_tmp.p, s);   // normalised: |r| = 1
    launch_pdot(np, a->gn_r.p, a->gn_r.p, nullptr, 0, 0, S_RR, 0.0, part, sc, s);
    for (int k = 0; k < iters; ++k) {
        gn_apply(m, a, a->gn_p.p, active, g_scale, a->gn_q.p, s);
        if (k == 0) launch_pdot(np, a->gn_p.p, a->gn_q.p, nullptr, 0, 3, 0, kappa_rel, part, sc, s);
        launch_gn_ap(np, sc, a->gn_q.p, a->gn_p.p, a->gn_ap.p, s);
        launch_pdot(np, a->gn_p.p, a->gn_ap.p, nullptr, 0, 1, 0, 0.0, part, sc, s);
        launch_gn_update(np, sc, a->gn_p.p, a->gn_ap.p, a->gn_tmp.p, a->gn_r.p, s);
        launch_pdot(np, a->gn_r.p, a->gn_r.p, nullptr, 0, 2, 0, 0.0, part, sc, s);
        launch_gn_pdir(np, sc, a->gn_r.p, a->gn_p.p, s);
    }
    launch_pscale(np, sc, S_GG, 0, active, a->gn_tmp.p, d, s);                  // undo the normalisation
}

static bool check_mesh(pd_mesh* m, pd_adjoint* a) { return m && a && a->mesh == m; }

extern "C" {

static pd_status pose_misfit(pd_mesh* m, const float* x, const float* target, float* dL_dx, double* loss,
                             bool accumulate) {
    if (!m || !x || !target || !loss) return ffail(PD_ERR_INVALID_ARG, "null argument");
    try {
        cudaStream_t s = m->stream;
        DBuf<float4> xi, ti, gi;
        DBuf<double> part;
        xi.alloc(m->n_v);
        ti.alloc(m->n_v);
        part.alloc(gn_partial_blocks());
        launch_gather_in(m, x, xi.p, s);
        launch_gather_in(m, target, ti.p, s);
        if (dL_dx) {
            gi.alloc(m->n_v);
            PDG_CUDA(cudaMemsetAsync(gi.p, 0, sizeof(float4) * m->n_v, s));
        }
        launch_misfit(m->n_free, xi.p, ti.p, dL_dx ? gi.p : nullptr, part.p, loss, 0, s, accumulate);
        if (dL_dx) launch_scatter_out(m, gi.p, dL_dx, 0, s);
        PDG_CUDA(cudaStreamSynchronize(s));   // the temporaries are freed on return
    } catch (const Fail& f) {
        return f.code;
    }
    return PD_OK;
}

pd_status pd_pose_misfit(pd_mesh* m, const float* x, const float* target, float* dL_dx, double* loss) {
    return pose_misfit(m, x, target, dL_dx, loss, false);
}

pd_status pd_pose_misfit_accumulate(pd_mesh* m, const float* x, const float* target, float* dL_dx, double* loss) {
    return pose_misfit(m, x, target, dL_dx, loss, true);
}

pd_status pd_tied_gradient(pd_mesh* m, const float* dL_dgamma_s, const float* dL_dgamma_v, double ratio,
                           const double* scale, float* dL_dtheta) {
    if (!m || !dL_dgamma_s || !dL_dgamma_v || !dL_dtheta) return ffail(PD_ERR_INVALID_ARG, "null argument");
    if (!std::isfinite(ratio)) return ffail(PD_ERR_INVALID_ARG, "ratio must be finite");
    try {
        launch_tied_gradient(m->n_t, dL_dgamma_s, dL_dgamma_v, ratio, scale, dL_dtheta, m->stream);
    } catch (const Fail& f) {
        return f.code;
    }
    return PD_OK;
}

pd_status pd_gn_product(pd_mesh* m, pd_adjoint* a, const float* x, const float* v, const uint8_t* active,
                        float g_scale, float* Pv) {
    if (!check_mesh(m, a) || !x || !v || !Pv) return ffail(PD_ERR_INVALID_ARG, "null argument or mismatched workspace");
    if (!m->prefactored) return ffail(PD_ERR_NOT_PREFACTORED, "pd_prefactor has not run");
    if (!(g_scale > 0.f) || !std::isfinite(g_scale)) return ffail(PD_ERR_INVALID_ARG, "g_scale must be > 0");
    try {
        cudaStream_t s = m->stream;
        gn_prepare(m, a);
        launch_gather_in(m, x, a->xeq.p, s);
        gn_setup(m, a, s);
        launch_pcopy(2 * m->n_t, 1.f, v, active, a->gn_p.p, s);
        gn_apply(m, a, a->gn_p.p, active, g_scale, Pv, s);
    } catch (const Fail& f) {
        return f.code;
    }
    return PD_OK;
}

pd_status pd_gn_direction(pd_mesh* m, pd_adjoint* a, const float* x, const float* grad, const uint8_t* active,
                          double kappa_rel, float g_scale, int32_t outer_iters, float* d, double* kappa_out) {
    if (!check_mesh(m, a) || !x || !grad || !d) return ffail(PD_ERR_INVALID_ARG, "null argument or mismatched workspace");
    if (!m->prefactored) return ffail(PD_ERR_NOT_PREFACTORED, "pd_prefactor has not run");
    if (outer_iters < 1 || outer_iters > 1000) return ffail(PD_ERR_INVALID_ARG, "outer_iters out of range [1, 1000]");
    if (!(kappa_rel >= 0.0) || !std::isfinite(kappa_rel)) return ffail(PD_ERR_INVALID_ARG, "kappa_rel must be >= 0");
    if (!(g_scale > 0.f) || !std::isfinite(g_scale)) return ffail(PD_ERR_INVALID_ARG, "g_scale must be > 0");
    try {
        cudaStream_t s = m->stream;
        gn_prepare(m, a);
        launch_gather_in(m, x, a->xeq.p, s);
        gn_setup(m, a, s);
        gn_direction(m, a, grad, active, kappa_rel, g_scale, outer_iters, d, s);
        if (kappa_out)
            PDG_CUDA(cudaMemcpyAsync(kappa_out, a->gn_sc.p + S_KAPPA, sizeof(double), cudaMemcpyDeviceToDevice, s));
    } catch (const Fail& f) {
        return f.code;
    }
    return PD_OK;
}

pd_status pd_fit_pose(pd_mesh* m, pd_adjoint* a, const pd_fit_opts* o, const float* x_prev, const float* v_prev,
                      const float* pin_targets, const float* gravity, const float* target, float* gamma,
                      double* losses, pd_fit_report* report) {
    if (!check_mesh(m, a) || !o || !x_prev || !v_prev || !target || !gamma)
        return ffail(PD_ERR_INVALID_ARG, "null argument or mismatched workspace");
    if (o->n_gd < 0 || o->n_gn < 0 || o->n_gd + o->n_gn > 10000 || !(o->gd_step > 0.f) || !(o->gn_step > 0.f) ||
        !(o->kappa_rel >= 0.0) || !std::isfinite(o->kappa_rel) || !(o->floor > 0.f) || o->max_halvings < 0 ||
        o->max_halvings > 60 || o->max_pivots < 0 || o->outer_iters < 1 || o->outer_iters > 1000 || !(o->dt > 0.0))
        return ffail(PD_ERR_INVALID_ARG, "fit options out of range");
    const auto t0 = std::chrono::steady_clock::now();
    const int n_t = m->n_t, np = 2 * n_t, nv3 = 3 * m->n_v;
    cudaStream_t s = m->stream;
    pd_fit_report rep{};
    try {
        gn_prepare(m, a);
        DBuf<float> gam, trial, grad, raw, dir, x_acc, x_try, dl_acc, dl_try;
        DBuf<uint8_t> clamped, neg, active;
        DBuf<double> loss_dev;
        DBuf<int32_t> piv;
        gam.alloc(np);
        trial.alloc(np);
        grad.alloc(np);
        raw.alloc(np);
        dir.alloc(np);
        for (auto* b : {&x_acc, &x_try, &dl_acc, &dl_try}) b->alloc(nv3);
        clamped.alloc(np);
        neg.alloc(np);
        active.alloc(np);
        loss_dev.alloc(1);
        piv.alloc(1);
        PDG_CUDA(cudaMemcpyAsync(gam.p, gamma, sizeof(float) * np, cudaMemcpyDeviceToDevice, s));
        PDG_CUDA(cudaMemsetAsync(clamped.p, 0, np, s));
        PDG_CUDA(cudaMemsetAsync(active.p, 1, np, s));

        const float* mesh_gamma = nullptr;   // which parameter array the mesh was last factored with
        auto check = [](pd_status st) {
            if (st != PD_OK) throw Fail{st};
        };
        auto use = [&](const float* g) {     // materials + prefactorisation of g
            check(pd_set_materials(m, g, g + n_t));
            check(pd_prefactor(m, o->dt, o->solver));
            mesh_gamma = g;
        };
        // equilibrium of the pose for materials g -> (x, dL/dx), loss
        auto evaluate = [&](const float* g, float* xo, float* dlo) -> double {
            use(g);
            check(pd_set_state(m, x_prev, v_prev));
            check(pd_equilibrium_step(m, a, pin_targets, gravity, o->n_pd_iter, o->n_newton, xo));
            check(pd_pose_misfit(m, xo, target, dlo, loss_dev.p));
            double l = 0.0;
            PDG_CUDA(cudaMemcpyAsync(&l, loss_dev.p, sizeof(double), cudaMemcpyDeviceToHost, s));
            check(pd_sync(m));
            ++rep.trials;
            return l;
        };
        auto read_scalar = [&](int idx) {
            double v = 0.0;
            PDG_CUDA(cudaMemcpyAsync(&v, a->gn_sc.p + idx, sizeof(double), cudaMemcpyDeviceToHost, s));
            PDG_CUDA(cudaStreamSynchronize(s));
            return v;
        };

        double eps = evaluate(gam.p, x_acc.p, dl_acc.p);
        rep.loss0 = eps;
        const int n_it = o->n_gd + o->n_gn;
        if (losses) losses[0] = eps;
        int done = 0;
        for (int it = 0; it < n_it; ++it) {
            if (mesh_gamma != gam.p) use(gam.p);
            // gradient d eps / d gamma = -B^T lambda (one backward adjoint step)
            PDG_CUDA(cudaMemsetAsync(grad.p, 0, sizeof(float) * np, s));
            check(pd_adjoint_reset(a));
            check(pd_adjoint_step(m, a, x_acc.p, dl_acc.p, grad.p, grad.p + n_t));
            const bool use_gn = it >= o->n_gd;
            float alpha;
            if (use_gn) {
                launch_gather_in(m, x_acc.p, a->xeq.p, s);
                gn_setup(m, a, s);
                gn_direction(m, a, grad.p, active.p, o->kappa_rel, 2.f, o->outer_iters, raw.p, s);
                alpha = o->gn_step;
            } else {
                // -grad scaled so that max_j |d_j| / gamma_j = 1 (active parameters)
                launch_pdot(np, grad.p, gam.p, active.p, 1, 0, S_MAX, 0.0, a->gn_partial.p, a->gn_sc.p, s);
                launch_pscale(np, a->gn_sc.p, S_MAX, 1, active.p, grad.p, raw.p, s);
                alpha = o->gd_step;
            }
            launch_clamp_dir(np, raw.p, clamped.p, dir.p, s);
            if (use_gn) {
                for (int k = 0; k < o->max_pivots; ++k) {
                    launch_pdot(np, dir.p, grad.p, nullptr, 0, 0, S_TMP, 0.0, a->gn_partial.p, a->gn_sc.p, s);
                    if (read_scalar(S_TMP) < 0.0) break;
                    launch_pick_pivot(np, gam.p, raw.p, clamped.p, active.p, o->floor, a->gn_partial.p,
                                      a->gn_ipartial.p, piv.p, s);
                    int j = -1;
                    PDG_CUDA(cudaMemcpyAsync(&j, piv.p, sizeof(int), cudaMemcpyDeviceToHost, s));
                    PDG_CUDA(cudaStreamSynchronize(s));
                    if (j < 0 || j >= np) break;
                    PDG_CUDA(cudaMemsetAsync(active.p + j, 0, 1, s));
                    gn_direction(m, a, grad.p, active.p, o->kappa_rel, 2.f, o->outer_iters, raw.p, s);
                    launch_clamp_dir(np, raw.p, clamped.p, dir.p, s);
                }
            }
            bool accepted = false;
            for (int h = 0; h <= o->max_halvings; ++h) {
                launch_project(np, gam.p, dir.p, alpha, o->floor, trial.p, neg.p, s);
                const double et = evaluate(trial.p, x_try.p, dl_try.p);
                if (et < eps) {
                    launch_accept(np, trial.p, neg.p, gam.p, clamped.p, s);
                    PDG_CUDA(cudaMemcpyAsync(x_acc.p, x_try.p, sizeof(float) * nv3, cudaMemcpyDeviceToDevice, s));
                    PDG_CUDA(cudaMemcpyAsync(dl_acc.p, dl_try.p, sizeof(float) * nv3, cudaMemcpyDeviceToDevice, s));
                    mesh_gamma = gam.p;   // the mesh holds the accepted materials (copied from trial)
                    eps = et;
                    accepted = true;
                    break;
                }
                alpha *= 0.5f;
            }
            if (losses) losses[it + 1] = eps;
            if (!accepted) {
                for (int r = it + 1; losses && r < n_it; ++r) losses[r + 1] = eps;
                break;
            }
            ++done;
        }
        if (mesh_gamma != gam.p) use(gam.p);
        PDG_CUDA(cudaMemcpyAsync(gamma, gam.p, sizeof(float) * np, cudaMemcpyDeviceToDevice, s));
        std::vector<uint8_t> hc(np), ha(np);
        PDG_CUDA(cudaMemcpyAsync(hc.data(), clamped.p, np, cudaMemcpyDeviceToHost, s));
        PDG_CUDA(cudaMemcpyAsync(ha.data(), active.p, np, cudaMemcpyDeviceToHost, s));
        PDG_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < np; ++i) {
            rep.clamped += hc[i] ? 1 : 0;
            rep.pivots += ha[i] ? 0 : 1;
        }
        rep.iterations = done;
        rep.loss = eps;
    } catch (const Fail& f) {
        cudaStreamSynchronize(s);
        return f.code;
    }
    rep.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (report) *report = rep;
    return PD_OK;
}

pd_status pd_fit_pose_reduced(pd_mesh* m, pd_adjoint* a, const pd_fit_opts* o, const float* H, int32_t r,
                              const float* x_prev, const float* v_prev, const float* pin_targets, const float* gravity,
                              const float* target, float* gamma, double* losses, pd_fit_report* report) {
    if (!check_mesh(m, a) || !o || !H || !x_prev || !v_prev || !target || !gamma)
        return ffail(PD_ERR_INVALID_ARG, "null argument or mismatched workspace");
    if (r < 1 || r > 56 || r > m->n_t) return ffail(PD_ERR_INVALID_ARG, "r out of range [1, min(56, n_t)]");
    if (o->n_gn < 0 || o->n_gn > 10000 || !(o->gn_step > 0.f) || !(o->kappa_rel >= 0.0) ||
        !std::isfinite(o->kappa_rel) || !(o->floor > 0.f) || o->max_halvings < 0 || o->max_halvings > 60 ||
        !(o->dt > 0.0))
        return ffail(PD_ERR_INVALID_ARG, "fit options out of range");
    const auto t0 = std::chrono::steady_clock::now();
    const int n_t = m->n_t, np = 2 * n_t, nq = 2 * r, nv3 = 3 * m->n_v;
    cudaStream_t s = m->stream;
    pd_fit_report rep{};
    try {
        gn_prepare(m, a);
        DBuf<float> gam, trial, grad, x_acc, x_try, dl_acc, dl_try;
        DBuf<double> loss_dev, dq, Pq;
        DBuf<int32_t> cnt;
        gam.alloc(np);
        trial.alloc(np);
        grad.alloc(np);
        for (auto* b : {&x_acc, &x_try, &dl_acc, &dl_try}) b->alloc(nv3);
        loss_dev.alloc(1);
        dq.alloc(nq);
        Pq.alloc((size_t)nq * nq);
        cnt.alloc(1);
        auto check = [](pd_status st) {
            if (st != PD_OK) throw Fail{st};
        };
        const float* mesh_gamma = nullptr;
        auto use = [&](const float* g) {
            check(pd_set_materials(m, g, g + n_t));
            check(pd_prefactor(m, o->dt, o->solver));
            mesh_gamma = g;
        };
        auto evaluate = [&](const float* g, float* xo, float* dlo) -> double {
            use(g);
            check(pd_set_state(m, x_prev, v_prev));
            check(pd_equilibrium_step(m, a, pin_targets, gravity, o->n_pd_iter, o->n_newton, xo));
            check(pd_pose_misfit(m, xo, target, dlo, loss_dev.p));
            double l = 0.0;
            PDG_CUDA(cudaMemcpyAsync(&l, loss_dev.p, sizeof(double), cudaMemcpyDeviceToHost, s));
            check(pd_sync(m));
            ++rep.trials;
            return l;
        };
        // gamma = D q, and the number of its components below the floor
        auto apply = [&](const std::vector<double>& q, float* out) {
            PDG_CUDA(cudaMemcpyAsync(dq.p, q.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, s));
            launch_basis_apply(n_t, r, H, dq.p, out, s);
            launch_count_below(np, out, o->floor, cnt.p, s);
            int below = 0;
            PDG_CUDA(cudaMemcpyAsync(&below, cnt.p, sizeof(int), cudaMemcpyDeviceToHost, s));
            PDG_CUDA(cudaStreamSynchronize(s));
            return below;
        };
        auto project_t = [&](const float* w, std::vector<double>& out) {   // out = D^T w
            launch_basis_t(n_t, r, H, w, dq.p, s);
            out.resize(nq);
            PDG_CUDA(cudaMemcpyAsync(out.data(), dq.p, sizeof(double) * nq, cudaMemcpyDeviceToHost, s));
            PDG_CUDA(cudaStreamSynchronize(s));
        };

        std::vector<double> q, gq, qt(nq), hP((size_t)nq * nq), Rinv, dlt(nq);
        project_t(gamma, q);
        if (apply(q, gam.p) > 0) throw Fail{PD_ERR_BAD_MATERIAL};
        double eps = evaluate(gam.p, x_acc.p, dl_acc.p);
        rep.loss0 = eps;
        if (losses) losses[0] = eps;
        int done = 0;
        for (int it = 0; it < o->n_gn; ++it) {
            if (mesh_gamma != gam.p) use(gam.p);
            PDG_CUDA(cudaMemsetAsync(grad.p, 0, sizeof(float) * np, s));
            check(pd_adjoint_reset(a));
            check(pd_adjoint_step(m, a, x_acc.p, dl_acc.p, grad.p, grad.p + n_t));
            project_t(grad.p, gq);
            // P_q = D^T P D, one column per basis vector (2 r products)
            launch_gather_in(m, x_acc.p, a->xeq.p, s);
            gn_setup(m, a, s);
            for (int j = 0; j < nq; ++j) {
                launch_basis_col(n_t, r, H, j, a->gn_p.p, s);
                gn_apply(m, a, a->gn_p.p, nullptr, 2.f, a->gn_q.p, s);
                launch_basis_t(n_t, r, H, a->gn_q.p, Pq.p + (size_t)j * nq, s);
            }
            PDG_CUDA(cudaMemcpyAsync(hP.data(), Pq.p, sizeof(double) * nq * nq, cudaMemcpyDeviceToHost, s));
            PDG_CUDA(cudaStreamSynchronize(s));
            // (P_q + kappa I) d = -g_q on the host (2 r <= 112 unknowns), kappa relative as in the full fit
            double gg = 0.0, gPg = 0.0;
            for (int i = 0; i < nq; ++i) {
                gg += gq[i] * gq[i];
                for (int j = 0; j < nq; ++j) gPg += gq[i] * 0.5 * (hP[(size_t)i * nq + j] + hP[(size_t)j * nq + i]) * gq[j];
            }
            const double kappa = gg > 0.0 ? o->kappa_rel * gPg / gg : 0.0;
            std::vector<double> A((size_t)nq * nq);
            for (int i = 0; i < nq; ++i)
                for (int j = 0; j < nq; ++j)
                    A[(size_t)i * nq + j] = 0.5 * (hP[(size_t)i * nq + j] + hP[(size_t)j * nq + i]) + (i == j ? kappa : 0.0);
            if (!chol_upper_inverse(A.data(), nq, nq, Rinv)) throw Fail{PD_ERR_NOT_SPD};
            // d = -R^-1 R^-T g
            std::vector<double> y(nq, 0.0);
            for (int i = 0; i < nq; ++i)
                for (int k = 0; k < nq; ++k) y[i] += Rinv[(size_t)k * nq + i] * gq[k];
            for (int i = 0; i < nq; ++i) {
                double acc = 0.0;
                for (int k = 0; k < nq; ++k) acc += Rinv[(size_t)i * nq + k] * y[k];
                dlt[i] = -acc;
            }
            double alpha = o->gn_step;
            bool accepted = false;
            for (int h = 0; h <= o->max_halvings; ++h) {
                for (int i = 0; i < nq; ++i) qt[i] = q[i] + alpha * dlt[i];
                if (apply(qt, trial.p) == 0) {
                    const double et = evaluate(trial.p, x_try.p, dl_try.p);
                    if (et < eps) {
                        PDG_CUDA(cudaMemcpyAsync(gam.p, trial.p, sizeof(float) * np, cudaMemcpyDeviceToDevice, s));
                        PDG_CUDA(cudaMemcpyAsync(x_acc.p, x_try.p, sizeof(float) * nv3, cudaMemcpyDeviceToDevice, s));
                        PDG_CUDA(cudaMemcpyAsync(dl_acc.p, dl_try.p, sizeof(float) * nv3, cudaMemcpyDeviceToDevice, s));
                        mesh_gamma = gam.p;
                        q = qt;
                        eps = et;
                        accepted = true;
                        break;
                    }
                }
                alpha *= 0.5;
            }
            if (losses) losses[it + 1] = eps;
            if (!accepted) {
                for (int k = it + 1; losses && k < o->n_gn; ++k) losses[k + 1] = eps;
                break;
            }
            ++done;
        }
        if (mesh_gamma != gam.p) use(gam.p);
        PDG_CUDA(cudaMemcpyAsync(gamma, gam.p, sizeof(float) * np, cudaMemcpyDeviceToDevice, s));
        PDG_CUDA(cudaStreamSynchronize(s));
        rep.iterations = done;
        rep.loss = eps;
    } catch (const Fail& f) {
        cudaStreamSynchronize(s);
        if (f.code == PD_ERR_BAD_MATERIAL) set_error("the projection of gamma onto the basis has a component below the floor");
        return f.code;
    }
    rep.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (report) *report = rep;
    return PD_OK;
}

}  // extern "C"
