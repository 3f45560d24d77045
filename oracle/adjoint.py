"""FP64 oracle of the adjoint gradient of a pose-matching loss with respect to
every per-element material parameter.

TEST INFRASTRUCTURE ONLY (imported by tests/ and bench.py's CPU legs).

Paper passages followed (Sec. 6.1, "Adjoint Gradient Descent"): the
equilibrium constraint g(x, gamma) = 0 of Eq. g, the sensitivity of
Eq. pxpgamma, and the adjoint state of Eq. adjoint_state and
Eq. adjoint_state_solve: dL/dgamma = -lambda^T dg/dgamma with
(dg/dx) lambda = (dL/dx)^T.

Readings taken here:

* each time step n is solved to equilibrium (Sec. 8 applies Newton after PD
  so that Eq. g holds to a small residual):
      g_n(x_n) = (M/dt^2)(x_n - y_n) + grad E(x_n) = 0,
      y_n = x_{n-1} + dt v_{n-1} + dt^2 g_grav,  v_n = (x_n - x_{n-1})/dt,
  with E the elastic energy whose gradient K x - b the PD step uses (the
  factor-1/2 reading of Eq. energy);
* the loss is L = sum_n sum_v ||x_{n,v} - xhat_{n,v}||^2 over the free
  vertices; since y_{n+1} = 2 x_n - x_{n-1} + dt^2 g, x_n also enters g_{n+1}
  and g_{n+2}, which gives the backward recurrence
      H_n lambda_n = 2 (x_n - xhat_n) + (M/dt^2)(2 lambda_{n+1} - lambda_{n+2}),
      dL/dgamma^s_e = -sum_n lambda_n^T dg_n/dgamma^s_e,
      dg_n/dgamma^s_e = V_e (F - R(F)) g_c on the element's corners
  (gamma^v likewise with V(F)), lambda_{N+1} = lambda_{N+2} = 0;
* H_n = M/dt^2 + sum_e d^2E_e/dx^2, the true Hessian:
      d^2E_e/dF^2 = V_e [gamma^s (I - dR/dF) + gamma^v (I - dV/dF)].

The projection derivatives use the derivative of an isotropic matrix
function P(F) = U diag(f(sigma)) W^T: with A = U^T dF W, U^T dP W has
diagonal J_f diag(A) and off-diagonal entries
    (f_i - f_j)/(sigma_i - sigma_j) * (A_ij + A_ji)/2
  + (f_i + f_j)/(sigma_i + sigma_j) * (A_ij - A_ji)/2
(the first ratio replaced by its limit at equal singular values).  For R,
f = 1; for V, f = d(sigma) and J_f follows from differentiating the KKT
conditions (d_i - sigma_i) d_i = mu, prod d = 1 on the free targets.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .pd_oracle import GRAVITY, PDOracle, deformation_gradient
from .projections import CLAMP, project_both


def volume_jacobian(s: np.ndarray, d: np.ndarray, lo: float = CLAMP) -> np.ndarray:
    """J = dd/dsigma (n, 3, 3) of the volume targets at (sigma, d)."""
    n = s.shape[0]
    J = np.zeros((n, 3, 3))
    free = d > lo * (1 + 1e-9)
    a = np.where(free, 1.0 / (2.0 * d - s), 0.0)
    S = np.sum(np.where(free, a / d, 0.0), axis=1)
    for i in range(3):
        for k in range(3):
            J[:, i, k] = np.where(free[:, i] & free[:, k],
                                  (a[:, i] * d[:, i] if i == k else 0.0) - a[:, i] * a[:, k] / S, 0.0)
    return J


def _coefficients(s, f, Jf):
    """alpha_ij, beta_ij (n, 3, 3) of the isotropic-function derivative."""
    n = s.shape[0]
    alpha = np.zeros((n, 3, 3))
    beta = np.zeros((n, 3, 3))
    for i in range(3):
        for j in range(3):
            if i == j:
                continue
            ds = s[:, i] - s[:, j]
            tie = np.abs(ds) < 1e-9 * np.maximum(1.0, np.abs(s[:, i]))
            lim = Jf[:, i, i] - Jf[:, i, j]
            alpha[:, i, j] = np.where(tie, lim, (f[:, i] - f[:, j]) / np.where(tie, 1.0, ds))
            beta[:, i, j] = (f[:, i] + f[:, j]) / (s[:, i] + s[:, j])
    return alpha, beta


class ProjectionDerivative:
    """dR/dF and dV/dF of a batch of deformation gradients, applied to dF."""

    def __init__(self, F: np.ndarray):
        R, V, U, s, W, d = project_both(F)
        self.R, self.V, self.U, self.W, self.s, self.d = R, V, U, W, s, d
        ones = np.ones_like(s)
        self.aR, self.bR = _coefficients(s, ones, np.zeros((s.shape[0], 3, 3)))
        self.JV = volume_jacobian(s, d)
        self.aV, self.bV = _coefficients(s, d, self.JV)

    def _apply(self, dF, alpha, beta, Jf):
        A = np.swapaxes(self.U, 1, 2) @ dF @ self.W
        sym = 0.5 * (A + np.swapaxes(A, 1, 2))
        skw = 0.5 * (A - np.swapaxes(A, 1, 2))
        B = alpha * sym + beta * skw
        diagA = np.einsum("nii->ni", A)
        B[:, [0, 1, 2], [0, 1, 2]] = np.einsum("nik,nk->ni", Jf, diagA)
        return self.U @ B @ np.swapaxes(self.W, 1, 2)

    def dR(self, dF):
        return self._apply(dF, self.aR, self.bR, np.zeros_like(self.JV))

    def dV(self, dF):
        return self._apply(dF, self.aV, self.bV, self.JV)


class AdjointOracle:
    """Equilibrium time stepping, loss and adjoint gradient in FP64."""

    def __init__(self, pd: PDOracle, gravity=GRAVITY):
        self.o = pd
        self.g = np.asarray(gravity, np.float64)
        n_v = pd.n_v
        self.fdof = (pd.free[:, None] * 3 + np.arange(3)[None, :]).ravel()

    # ---- energy gradient and Hessian -------------------------------------------------
    def residual(self, x, y):
        """g(x) = (M/dt^2)(x - y) + grad E(x) on every vertex (n_v, 3)."""
        o = self.o
        F = deformation_gradient(x, o.tets, o.g)
        R, V, *_ = project_both(F)
        P = o.ws[:, None, None] * (F - R) + o.wv[:, None, None] * (F - V)
        g = (o.mass / o.dt ** 2)[:, None] * (x - y)
        np.add.at(g, o.tets.ravel(), np.einsum("eij,ecj->eci", P, o.g).reshape(-1, 3))
        return g

    def hessian(self, x) -> sp.csr_matrix:
        """True Hessian of Q on the free DOFs (3 n_free x 3 n_free)."""
        o = self.o
        F = deformation_gradient(x, o.tets, o.g)
        D = ProjectionDerivative(F)
        n_t = o.n_t
        # d^2 E_e / dF^2 applied to the 9 unit directions
        HF = np.zeros((n_t, 9, 9))
        for k in range(9):
            E = np.zeros((n_t, 3, 3))
            E[:, k // 3, k % 3] = 1.0
            dP = o.ws[:, None, None] * (E - D.dR(E)) + o.wv[:, None, None] * (E - D.dV(E))
            HF[:, :, k] = dP.reshape(n_t, 9)
        # lift: F_ij = sum_c x_{c,i} g_{c,j} -> G[(i,j), (c,i')] = delta_ii' g_{c,j}
        G = np.zeros((n_t, 9, 12))
        for i in range(3):
            for j in range(3):
                for c in range(4):
                    G[:, 3 * i + j, 3 * c + i] = o.g[:, c, j]
        He = np.einsum("eak,eab,ebl->ekl", G, HF, G)
        dofs = (o.tets[:, :, None] * 3 + np.arange(3)[None, None, :]).reshape(n_t, 12)
        rows = np.repeat(dofs, 12, axis=1).ravel()
        cols = np.tile(dofs, (1, 12)).ravel()
        n = 3 * o.n_v
        H = sp.coo_matrix((He.ravel(), (rows, cols)), shape=(n, n)).tocsr()
        H = H + sp.diags(np.repeat(o.mass / o.dt ** 2, 3))
        return H[self.fdof][:, self.fdof].tocsr()

    # ---- forward ---------------------------------------------------------------------
    def equilibrium(self, x_prev, v_prev, pins, pd_iters=30, tol=1e-11, max_newton=25):
        o = self.o
        y = o.inertial_target(x_prev, v_prev, self.g)
        x, _ = o.step(x_prev, v_prev, pins, self.g, pd_iters)
        scale = np.linalg.norm((o.mass[:, None] * self.g[None, :])[o.free])
        for _ in range(max_newton):
            r = self.residual(x, y)[o.free].ravel()
            if np.linalg.norm(r) <= tol * scale:
                break
            H = self.hessian(x)
            dx = spla.spsolve(H.tocsc(), -r)
            step = 1.0
            base = np.linalg.norm(r)
            while step > 1e-4:
                xt = x.copy()
                xt[o.free] += step * dx.reshape(-1, 3)
                if np.linalg.norm(self.residual(xt, y)[o.free]) < base:
                    break
                step *= 0.5
            x = xt
        v = (x - x_prev) / o.dt
        return x, v

    def forward(self, x0, v0, pins_fn, n_steps, **kw):
        xs, vs = [np.asarray(x0, np.float64)], [np.asarray(v0, np.float64)]
        for n in range(n_steps):
            x, v = self.equilibrium(xs[-1], vs[-1], pins_fn(n), **kw)
            xs.append(x)
            vs.append(v)
        return xs, vs

    @staticmethod
    def loss(xs, targets, free):
        return float(sum(np.sum((xs[n][free] - targets[n][free]) ** 2) for n in range(1, len(xs))))

    # ---- backward ----------------------------------------------------------------------
    def gradient(self, xs, targets):
        """(dL/dgamma_s, dL/dgamma_v) for L = sum_{n>=1} ||x_n - xhat_n||^2 (free vertices)."""
        o = self.o
        N = len(xs) - 1
        mh2 = np.repeat(o.mass[o.free] / o.dt ** 2, 3)
        lam1 = np.zeros(len(self.fdof))   # lambda_{n+1}
        lam2 = np.zeros(len(self.fdof))   # lambda_{n+2}
        gs = np.zeros(o.n_t)
        gv = np.zeros(o.n_t)
        for n in range(N, 0, -1):
            x = xs[n]
            rhs = 2.0 * (x[o.free] - targets[n][o.free]).ravel() + mh2 * (2.0 * lam1 - lam2)
            H = self.hessian(x)
            lam = spla.spsolve(H.tocsc(), rhs)
            full = np.zeros((o.n_v, 3))
            full[o.free] = lam.reshape(-1, 3)
            F = deformation_gradient(x, o.tets, o.g)
            R, V, *_ = project_both(F)
            Lam = deformation_gradient(full, o.tets, o.g)       # sum_c lambda_c (outer) g_c
            gs -= o.vol * np.sum((F - R) * Lam, axis=(1, 2))
            gv -= o.vol * np.sum((F - V) * Lam, axis=(1, 2))
            lam2, lam1 = lam1, lam
        return gs, gv
