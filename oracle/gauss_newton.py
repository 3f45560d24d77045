"""FP64 oracle of the adjoint Gauss-Newton material step and of the fitting
loop around it (Sec. 6.2 "Adjoint Gauss-Newton", Eq. hessian, Eq. gn,
Eq. agn; Sec. 6.3 "Linear Search & Non-Negativity Constraint").

TEST INFRASTRUCTURE ONLY: imported by tests/ (and nothing on the product
path).  It shares no code with the CUDA library.

One sample pose is fitted at a time ("sample-by-sample", Sec. 6).  The pose
starts from a known state (x_prev, v_prev), so its inertial target
y = x_prev + dt v_prev + dt^2 g is a known vector and the equilibrium
constraint of Eq. g reads
    g(x, gamma) = (M/dt^2)(x - y) + grad E(x; gamma) = 0,
with gamma = [gamma_s (n_t), gamma_v (n_t)], the 2 n_E material vector.
The pose loss is eps = sum over free vertices of ||x - xhat||^2, so
G = d^2 eps / dx^2 = 2 I.

Quantities (free DOFs only; pinned vertices are Dirichlet):
  H = dg/dx                        the true Hessian (AdjointOracle.hessian)
  B = dg/dgamma                    3 n_free x 2 n_t, column of element e:
                                     gamma_s: V_e (F - R(F)) g_c at its corners
                                     gamma_v: V_e (F - V(F)) g_c
  J = dx/dgamma = -H^-1 B          Eq. pxpgamma
  grad = d eps/d gamma = -B^T lam,  H lam = 2 (x - xhat)    Eq. adjoint_state(_solve)
  P = J^T G J                      the Gauss-Newton matrix (Eq. hessian without
                                   its second term)
  GN direction: (P + kappa I) d = -grad                     Eq. gn with the
                                   Levenberg-Marquardt shift kappa I

Readings taken here (each listed in the design notes):
  * The block system Eq. agn as printed, eliminated row by row
    (mu = H^-1 B d, nu = H^-T G mu, B^T nu = grad), gives P d = +grad: its d
    is the negative of the descent direction of Eq. gn.  The descent
    direction used is Eq. gn's; block_solve returns the printed system's
    (mu, nu, d) so that the two can be compared.
  * The Levenberg-Marquardt shift is placed on the parameter block of
    Eq. agn (the (3,3) block), which is exactly P + kappa I after
    elimination; G = 2 I is already positive definite.
  * Pivoted parameters (Sec. 6.3) are removed from the solve by deleting
    their rows and columns: their direction component is 0.
  * The Levenberg-Marquardt shift is relative: kappa = kappa_rel * g^T P g /
    g^T g (the Gauss-Newton curvature along the gradient), since "a small
    diagonal" has no absolute scale when gamma is in pascals.
  * The gradient-descent step is relative for the same reason: the
    direction -grad is scaled so that its largest component relative to
    its parameter, max_j |d_j| / gamma_j, is 1; the step 0.01 then moves no
    parameter by more than 1 % of its value.
  * Line search (Sec. 6.3): initial step 0.01 for gradient descent, 1.0 for
    Gauss-Newton, halved until the loss decreases; a step that yields a
    negative component sets it to the floor 1e-3 and caches its index; a
    later direction that would lower a cached component further has that
    component zeroed.  If the clamped Gauss-Newton direction is not a
    descent direction, the cached component whose tentative value
    gamma_j + d_j is most negative (among the cached ones still at the
    floor) is pivoted -- fixed at the floor and removed from the solve --
    and the direction (and its relative shift) recomputed, one component
    at a time.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .adjoint import AdjointOracle
from .pd_oracle import deformation_gradient
from .projections import project_both

FLOOR = 1e-3


class GaussNewtonOracle:
    """Gauss-Newton pieces for one pose of an AdjointOracle's mesh."""

    def __init__(self, ao: AdjointOracle, g_scale: float = 2.0):
        self.ao = ao
        self.o = ao.o
        self.g_scale = float(g_scale)

    # ---- dg/dgamma ---------------------------------------------------------------
    def param_jacobian(self, x) -> sp.csr_matrix:
        """B = dg/dgamma on the free DOFs (3 n_free x 2 n_t)."""
        o = self.o
        F = deformation_gradient(x, o.tets, o.g)
        R, V, *_ = project_both(F)
        n_t = o.n_t
        rows, cols, vals = [], [], []
        for which, T in ((0, F - R), (1, F - V)):
            # corner forces V_e T_e g_c  (n_t, 4, 3)
            f = o.vol[:, None, None] * np.einsum("eij,ecj->eci", T, o.g)
            dof = o.tets[:, :, None] * 3 + np.arange(3)[None, None, :]
            rows.append(dof.ravel())
            cols.append(np.repeat(np.arange(n_t) + which * n_t, 12))
            vals.append(f.ravel())
        n = 3 * o.n_v
        Bfull = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                              shape=(n, 2 * n_t)).tocsr()
        return Bfull[self.ao.fdof].tocsr()

    # ---- the pose: equilibrium, loss and gradient ---------------------------------
    def equilibrium(self, x_prev, v_prev, pins, **kw):
        x, _ = self.ao.equilibrium(x_prev, v_prev, pins, **kw)
        return x

    def loss(self, x, target) -> float:
        f = self.o.free
        return float(np.sum((x[f] - target[f]) ** 2))

    def gradient(self, x, target) -> np.ndarray:
        """d eps / d gamma = -B^T lam with H lam = d eps/dx = G (x - xhat) (Eq. adjoint_state_solve)."""
        f = self.o.free
        H = self.ao.hessian(x)
        lam = spla.spsolve(H.tocsc(), 2.0 * (x[f] - target[f]).ravel())
        return -(self.param_jacobian(x).T @ lam)

    # ---- Gauss-Newton ---------------------------------------------------------------
    def sensitivity(self, x) -> np.ndarray:
        """J = dx/dgamma = -H^-1 B (dense, 3 n_free x 2 n_t; small meshes only)."""
        H = self.ao.hessian(x).tocsc()
        B = self.param_jacobian(x).toarray()
        return -spla.spsolve(H, B).reshape(B.shape)

    def gn_matrix(self, x) -> np.ndarray:
        """P = J^T G J with G = g_scale I."""
        J = self.sensitivity(x)
        return self.g_scale * (J.T @ J)

    def gn_product(self, x, v) -> np.ndarray:
        """P v by the two linear solves of the eliminated block system."""
        H = self.ao.hessian(x).tocsc()
        B = self.param_jacobian(x)
        mu = spla.spsolve(H, B @ v)
        nu = spla.spsolve(H, self.g_scale * mu)
        return B.T @ nu

    def kappa(self, x, grad, kappa_rel, active=None) -> float:
        """kappa = kappa_rel * g^T P g / g^T g over the active parameters."""
        g = np.array(grad, np.float64)
        if active is not None:
            g[~np.asarray(active, bool)] = 0.0
        gg = float(g @ g)
        return 0.0 if gg == 0.0 else kappa_rel * float(g @ self.gn_product(x, g)) / gg

    def direction(self, x, grad, kappa, active=None) -> np.ndarray:
        """Descent direction of Eq. gn: (P + kappa I) d = -grad on the active
        parameters, d = 0 on the rest."""
        P = self.gn_matrix(x)
        n = P.shape[0]
        act = np.ones(n, bool) if active is None else np.asarray(active, bool)
        d = np.zeros(n)
        A = P[np.ix_(act, act)] + kappa * np.eye(int(act.sum()))
        d[act] = np.linalg.solve(A, -np.asarray(grad)[act])
        return d

    def block_solve(self, x, grad, kappa, active=None):
        """The sparse block system of Eq. agn, as printed, with kappa I on its
        parameter block; pivoted parameters' rows and columns removed.
        Returns (mu, nu, d) of that system."""
        H = self.ao.hessian(x).tocsr()
        B = self.param_jacobian(x).tocsr()
        n_p = B.shape[1]
        act = np.ones(n_p, bool) if active is None else np.asarray(active, bool)
        Ba = B[:, np.nonzero(act)[0]]
        na = Ba.shape[1]
        n = H.shape[0]
        G = self.g_scale * sp.identity(n, format="csr")
        A = sp.bmat([[G, -H.T, None],
                     [-H, None, Ba],
                     [None, Ba.T, kappa * sp.identity(na)]], format="csc")
        rhs = np.concatenate([np.zeros(2 * n), np.asarray(grad)[act]])
        lu = spla.splu(A)
        sol = lu.solve(rhs)
        for _ in range(3):          # iterative refinement: the blocks differ in scale by many decades
            sol += lu.solve(rhs - A @ sol)
        d = np.zeros(n_p)
        d[act] = sol[2 * n:]
        return sol[:n], sol[n:2 * n], d


def clamp_direction(d, clamped):
    """Cancel refinements that would lower a cached (clamped) component."""
    d = np.array(d, np.float64)
    d[np.asarray(clamped, bool) & (d < 0)] = 0.0
    return d


def project(trial, floor=FLOOR):
    """Negative components are set to the floor; returns (gamma, which were negative)."""
    trial = np.array(trial, np.float64)
    neg = trial < 0
    trial[neg] = floor
    return trial, neg


def pick_pivot(gamma, raw, clamped, pivot, floor=FLOOR):
    """The cached component at the floor, not yet pivoted, whose tentative
    value gamma_j + raw_j is most negative; None if there is none."""
    gamma = np.asarray(gamma, np.float64)
    raw = np.asarray(raw, np.float64)
    cand = np.nonzero(np.asarray(clamped, bool) & ~np.asarray(pivot, bool) & (raw < 0)
                      & (gamma <= floor * (1 + 1e-12)))[0]
    if cand.size == 0:
        return None
    return int(cand[np.argmin(gamma[cand] + raw[cand])])


def fit_pose(rest, tets, pinned, density, dt, x_prev, v_prev, pins, target, gamma_s, gamma_v,
             n_gd=2, n_gn=3, gd_step=0.01, gn_step=1.0, kappa_rel=1e-2, floor=FLOOR, max_halvings=12,
             max_pivots=8, pd_iters=30, gravity=None):
    """The two-stage fitting loop of Sec. 6.3 on one pose: n_gd gradient
    descent iterations, then n_gn Gauss-Newton iterations, each with a
    halving line search and the non-negativity projection / pivoting.
    Returns (gamma_s, gamma_v, losses, records): losses are the accepted
    losses (first entry: before the first iteration), records one dict per
    iteration.  The loop stops early when no step of the line search lowers
    the loss."""
    from .pd_oracle import PDOracle

    gamma = np.concatenate([np.asarray(gamma_s, np.float64), np.asarray(gamma_v, np.float64)])
    n_t = len(gamma_s)
    clamped = np.zeros(2 * n_t, bool)
    pivot = np.zeros(2 * n_t, bool)

    def make(gm):
        o = PDOracle(rest, tets, pinned, gm[:n_t], gm[n_t:], density, dt)
        return GaussNewtonOracle(AdjointOracle(o) if gravity is None else AdjointOracle(o, gravity))

    def solve(gn):
        return gn.equilibrium(x_prev, v_prev, pins, pd_iters=pd_iters)

    gn = make(gamma)
    x = solve(gn)
    eps = gn.loss(x, target)
    losses = [eps]
    records = []
    for it in range(n_gd + n_gn):
        grad = gn.gradient(x, target)
        use_gn = it >= n_gd
        if use_gn:
            kappa = gn.kappa(x, grad, kappa_rel, active=~pivot)
            raw = gn.direction(x, grad, kappa, active=~pivot)
            alpha = gn_step
        else:
            raw = -grad
            raw[pivot] = 0.0
            top = np.max(np.abs(raw) / gamma)
            if top > 0:
                raw /= top
            alpha = gd_step
        d = clamp_direction(raw, clamped)
        pivots_added = 0
        while use_gn and np.dot(d, grad) >= 0 and pivots_added < max_pivots:
            j = pick_pivot(gamma, raw, clamped, pivot, floor)
            if j is None:
                break
            pivot[j] = True
            pivots_added += 1
            kappa = gn.kappa(x, grad, kappa_rel, active=~pivot)
            raw = gn.direction(x, grad, kappa, active=~pivot)
            d = clamp_direction(raw, clamped)
        accepted = False
        for _ in range(max_halvings + 1):
            trial, neg = project(gamma + alpha * d, floor)
            gt = make(trial)
            xt = solve(gt)
            et = gt.loss(xt, target)
            if et < eps:
                gamma, gn, x, eps = trial, gt, xt, et
                clamped |= neg
                accepted = True
                break
            alpha *= 0.5
        records.append(dict(kind="gn" if use_gn else "gd", alpha=alpha if accepted else 0.0, loss=eps,
                            pivots=int(pivot.sum()), clamped=int(clamped.sum()), descent=float(np.dot(d, grad))))
        losses.append(eps)
        if not accepted:
            break
    return gamma[:n_t], gamma[n_t:], losses, records
