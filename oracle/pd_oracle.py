"""FP64 oracle: projective-dynamics time stepping with a full sparse Cholesky.

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of bench.py.  It shares no code with the CUDA library
and never calls it.

What it computes (Sec. 7, "Domain-decomposed projective dynamics"):

* implicit Euler with inertial vector a = x - x* - dt v* - dt^2 M^{-1} f
  (Sec. 7 opening equation); the inertial target is y = x* + dt v* + dt^2 g;
* PD local step (Sec. 7.1): per element the rotation target R(F_e) and the
  volume target V(F_e) of Eq. pd_local (see ``oracle.projections``);
* PD global step (Sec. 7.1): K x = b with
      K = M/dt^2 + sum_e V_e (gs_e + gv_e) B_e^T (D^T : D) B_e,
      b = (M/dt^2) y + sum_e V_e gs_e B_e^T (D^T : R_e)
                     + sum_e V_e gv_e B_e^T (D^T : V_e),
  solved with a direct Cholesky of the whole (not decomposed) matrix, since
  the paper's subspace solve (Eq. cms_boundary, Eq. global_subspace) with
  the full internal space reproduces the full solve: the Galerkin system is
  block-diagonal, the interface values solve S x_b = b_b - sum_d K_bi K_ii^-1 b_i
  exactly and the internal values follow as K_ii^-1 (b_i - K_ib x_b).

Readings of the paper taken here:

* the trailing "x" printed after K is a typo: K is the matrix alone;
* b uses the inertial target y (the "a" printed in b contains the unknown);
* the projections in b are evaluated at the current iterate x^k, not at x*
  (with x* the iterations would not change anything);
* K and b are the stationarity conditions of
      Q(x) = 1/(2 dt^2) ||x - y||_M^2
             + sum_e V_e/2 (gs_e ||F_e - R_e||^2 + gv_e ||F_e - V_e||^2),
  i.e. the elastic energy of Eq. energy with a factor 1/2;
* gravity g = (0, 0, -9.81) m/s^2 unless given; first iterate x^0 = y;
  no damping;
* Dirichlet (pinned) vertices are eliminated: K_ff x_f = b_f - K_fp x_p;
* lumped mass m_v = sum over incident tets of rho V_e / 4;
* velocity update v = (x - x*) / dt.

D and B_e in this code: F_e = sum_c x_c (outer) g_c with g_1..g_3 the rows
of Dm^{-1} (Dm = [X1-X0, X2-X0, X3-X0]) and g_0 = -(g_1+g_2+g_3); so
(D^T : D) between corners a, b is (g_a . g_b) I_3 and D^T : P at corner c
is P g_c.  K is therefore K_s (x) I_3 with the scalar matrix K_s.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
from scipy.sparse.csgraph import reverse_cuthill_mckee

from .projections import project_both

GRAVITY = (0.0, 0.0, -9.81)


def rest_shape(rest: np.ndarray, tets: np.ndarray):
    """Rest-shape operators: Dm^{-1} (n_t,3,3), volumes V_e, corner vectors g (n_t,4,3)."""
    X = rest[tets]                                     # (n_t, 4, 3)
    Dm = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)
    vol = np.linalg.det(Dm) / 6.0
    Dm_inv = np.linalg.inv(Dm)
    g = np.empty((tets.shape[0], 4, 3))
    g[:, 1:] = Dm_inv                                  # rows of Dm^{-1}
    g[:, 0] = -Dm_inv.sum(axis=1)
    return Dm_inv, vol, g


def deformation_gradient(x: np.ndarray, tets: np.ndarray, g: np.ndarray) -> np.ndarray:
    """F_e = sum_c x_c (outer) g_c, i.e. D . (B_e x) (Sec. 5, Eq. y2m notation)."""
    return np.einsum("eci,ecj->eij", x[tets], g)


def lumped_mass(n_v: int, tets: np.ndarray, vol: np.ndarray, density: float) -> np.ndarray:
    m = np.zeros(n_v)
    np.add.at(m, tets.ravel(), np.repeat(density * vol / 4.0, 4))
    return m


def stiffness_scalar(n_v, tets, vol, g, gamma_s, gamma_v, mass, dt) -> sp.csr_matrix:
    """Scalar K_s with K = K_s (x) I_3: M/dt^2 + sum_e V_e (gs+gv) (g_a . g_b)."""
    w = vol * (gamma_s + gamma_v)
    blocks = w[:, None, None] * np.einsum("eai,ebi->eab", g, g)        # (n_t,4,4)
    rows = np.repeat(tets, 4, axis=1).ravel()
    cols = np.tile(tets, (1, 4)).ravel()
    K = sp.coo_matrix((blocks.ravel(), (rows, cols)), shape=(n_v, n_v)).tocsr()
    K = K + sp.diags(mass / dt ** 2)
    K.sum_duplicates()
    return K.tocsr()


class BandedCholesky:
    """Direct solver for an SPD sparse matrix: RCM ordering, then LAPACK's
    banded Cholesky (pbtrf/pbtrs through scipy) on the permuted matrix."""

    def __init__(self, A: sp.csr_matrix):
        A = sp.csr_matrix(A)
        n = A.shape[0]
        perm = reverse_cuthill_mckee(A, symmetric_mode=True).astype(np.int64)
        Ap = A[perm][:, perm].tocoo()
        lower = Ap.row >= Ap.col
        r, c, v = Ap.row[lower], Ap.col[lower], Ap.data[lower]
        bw = int((r - c).max()) if r.size else 0
        ab = np.zeros((bw + 1, n))
        ab[r - c, c] = v
        self.perm = perm
        self.bandwidth = bw
        self.n = n
        self.cb = sla.cholesky_banded(ab, lower=True, check_finite=False)

    def solve(self, b: np.ndarray) -> np.ndarray:
        bp = b[self.perm]
        xp = sla.cho_solve_banded((self.cb, True), bp, check_finite=False)
        x = np.empty_like(xp)
        x[self.perm] = xp
        return x


class PDOracle:
    """Plain FP64 projective-dynamics stepper (no domain decomposition)."""

    def __init__(self, rest, tets, pinned, gamma_s, gamma_v, density=300.0, dt=1.0 / 150.0,
                 vertex_mass=None, factor=True):
        self.rest = np.asarray(rest, np.float64)
        self.tets = np.asarray(tets, np.int64)
        self.n_v = self.rest.shape[0]
        self.n_t = self.tets.shape[0]
        self.pinned = np.asarray(pinned, bool)
        self.free = np.nonzero(~self.pinned)[0]
        self.pin_ids = np.nonzero(self.pinned)[0]
        self.dt = float(dt)
        self.Dm_inv, self.vol, self.g = rest_shape(self.rest, self.tets)
        if np.any(self.vol <= 0):
            raise ValueError("degenerate or inverted rest tet")
        self.mass = (lumped_mass(self.n_v, self.tets, self.vol, density) if vertex_mass is None
                     else np.asarray(vertex_mass, np.float64))
        self.set_materials(gamma_s, gamma_v, factor=factor)

    # -- materials / matrix -------------------------------------------------
    def set_materials(self, gamma_s, gamma_v, factor=True):
        self.gamma_s = np.asarray(gamma_s, np.float64).copy()
        self.gamma_v = np.asarray(gamma_v, np.float64).copy()
        if np.any(self.gamma_s < 0) or np.any(self.gamma_v < 0):
            raise ValueError("negative material parameter")
        self.ws = self.vol * self.gamma_s
        self.wv = self.vol * self.gamma_v
        self.K = stiffness_scalar(self.n_v, self.tets, self.vol, self.g, self.gamma_s,
                                  self.gamma_v, self.mass, self.dt)
        self.K_ff = self.K[self.free][:, self.free].tocsr()
        self.K_fp = self.K[self.free][:, self.pin_ids].tocsr()
        self.chol = BandedCholesky(self.K_ff) if factor else None

    # -- PD pieces -----------------------------------------------------------
    def inertial_target(self, x_prev, v_prev, gravity=GRAVITY):
        return x_prev + self.dt * v_prev + self.dt ** 2 * np.asarray(gravity, np.float64)[None, :]

    def local(self, x):
        """Local step: per-element (R_e, V_e) at positions x."""
        F = deformation_gradient(x, self.tets, self.g)
        R, V, *_ = project_both(F)
        return R, V

    def rhs(self, y, R, V):
        """b = (M/dt^2) y + sum_e B_e^T (D^T : (ws_e R_e + wv_e V_e)) for all vertices."""
        P = self.ws[:, None, None] * R + self.wv[:, None, None] * V
        f = np.einsum("eij,ecj->eci", P, self.g)                        # (n_t, 4, 3)
        b = (self.mass / self.dt ** 2)[:, None] * y
        np.add.at(b, self.tets.ravel(), f.reshape(-1, 3))
        return b

    def global_solve(self, b, x_pin):
        """x_f = K_ff^{-1} (b_f - K_fp x_p)."""
        rhs = b[self.free] - self.K_fp @ x_pin
        return self.chol.solve(rhs)

    def step(self, x_prev, v_prev, pin_targets=None, gravity=GRAVITY, n_iter=10, record=None):
        """One implicit-Euler frame with n_iter local/global iterations."""
        x_prev = np.asarray(x_prev, np.float64)
        v_prev = np.asarray(v_prev, np.float64)
        y = self.inertial_target(x_prev, v_prev, gravity)
        x = y.copy()
        x_pin = x_prev[self.pin_ids] if pin_targets is None else np.asarray(pin_targets, np.float64)
        x[self.pin_ids] = x_pin
        for _ in range(n_iter):
            R, V = self.local(x)
            if record is not None:
                record.append(("local", self.objective(x, y, R, V)))
            b = self.rhs(y, R, V)
            x[self.free] = self.global_solve(b, x_pin)
            if record is not None:
                record.append(("global", self.objective(x, y, R, V)))
        v = (x - x_prev) / self.dt
        return x, v

    # -- energies --------------------------------------------------------------
    def objective(self, x, y, R=None, V=None):
        """Q(x; R, V); with R, V omitted the projections of x itself are used."""
        F = deformation_gradient(x, self.tets, self.g)
        if R is None or V is None:
            R, V, *_ = project_both(F)
        inertia = 0.5 / self.dt ** 2 * np.sum(self.mass[:, None] * (x - y) ** 2)
        es = np.sum((F - R) ** 2, axis=(1, 2))
        ev = np.sum((F - V) ** 2, axis=(1, 2))
        return inertia + 0.5 * np.sum(self.ws * es + self.wv * ev)

    def residual(self, x, y):
        """Gradient of Q at x for the free DOFs (zero at a converged frame)."""
        R, V = self.local(x)
        b = self.rhs(y, R, V)
        Kx = (self.K @ x)
        return (Kx - b)[self.free]


def simulate(oracle: PDOracle, x0, v0, pin_targets_fn, n_steps, n_iter, gravity=GRAVITY):
    """Free-running trajectory: list of (x, v) after each step."""
    x, v = np.asarray(x0, np.float64), np.asarray(v0, np.float64)
    out = []
    for n in range(n_steps):
        x, v = oracle.step(x, v, pin_targets_fn(n), gravity, n_iter)
        out.append((x.copy(), v.copy()))
    return out
