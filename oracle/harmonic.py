"""FP64 oracle of the harmonic initialization (Sec. 6, "Harmonic
Initialization", Eq. q2gamma): material vectors restricted to the span of
the lowest eigenvectors of the mesh Laplacian, fitted by Gauss-Newton in the
reduced coordinates, rank by rank (r = 1, 10, 30), before the full fit.

TEST INFRASTRUCTURE ONLY: imported by tests/ (and nothing on the product
path).  It shares no code with the CUDA library.

Readings taken here (listed in the design notes):
  * gamma lives on elements, so "the mesh Laplacian" is the graph Laplacian
    of the element adjacency graph: two tets are adjacent when they share a
    face; L = D - A, unit weights.  Its lowest eigenvector is constant, as
    the paper states for h_1.
  * H = [h_1 .. h_r] orthonormal (eigenvectors of the symmetric L), so the
    projection of a material vector onto the basis is q = diag(H,H)^T gamma.
  * In the reduced coordinates the Gauss-Newton pieces follow by the chain
    rule (the paper's sandwich of its Eq. agn blocks with diag(H, H)):
        grad_q = D^T grad,  P_q = D^T P D,  D = diag(H, H),
    and the direction solves (P_q + kappa I) d_q = -grad_q with the same
    relative shift as the full fit.
  * Each rank runs Gauss-Newton iterations with the halving line search of
    Sec. 6.3; a trial whose gamma = D q has a component below the floor
    (1e-3) counts as a failed trial (gamma must stay in the span of H, so it
    is not clamped).
  * Rank r starts from the projection of the previous gamma onto its basis
    (exact: the bases are nested), rank 1 from the projection of the initial
    guess, i.e. its mean.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .gauss_newton import FLOOR, GaussNewtonOracle


def face_adjacency(tets) -> np.ndarray:
    """Pairs (a, b), a < b, of tets that share a face."""
    tets = np.asarray(tets, np.int64)
    owner = {}
    pairs = []
    for t in range(tets.shape[0]):
        v = tets[t]
        for skip in range(4):
            f = tuple(sorted(np.delete(v, skip)))
            if f in owner:
                pairs.append((owner[f], t))
            else:
                owner[f] = t
    return np.array(sorted(pairs), np.int64).reshape(-1, 2)


def dual_laplacian(tets) -> sp.csr_matrix:
    """L = D - A of the face-adjacency graph of the tets."""
    n = len(tets)
    p = face_adjacency(tets)
    A = sp.coo_matrix((np.ones(2 * len(p)), (np.r_[p[:, 0], p[:, 1]], np.r_[p[:, 1], p[:, 0]])), shape=(n, n)).tocsr()
    return (sp.diags(np.asarray(A.sum(axis=1)).ravel()) - A).tocsr()


def harmonic_basis(tets, r):
    """(lambda (r,), H (n_t, r)): the r smallest eigenpairs of the dual Laplacian."""
    L = dual_laplacian(tets)
    n = L.shape[0]
    r = min(r, n)
    if n <= 4000:
        lam, vec = np.linalg.eigh(L.toarray())
        return lam[:r], vec[:, :r]
    lam, vec = spla.eigsh(L, k=r, sigma=-1e-3, which="LM")
    order = np.argsort(lam)
    return lam[order], vec[:, order]


def basis_matrix(H) -> np.ndarray:
    """D = diag(H, H) (2 n_t x 2 r)."""
    n, r = H.shape
    D = np.zeros((2 * n, 2 * r))
    D[:n, :r] = H
    D[n:, r:] = H
    return D


class ReducedGN:
    """Gauss-Newton in the coordinates q of gamma = D q."""

    def __init__(self, gn: GaussNewtonOracle, H):
        self.gn = gn
        self.D = basis_matrix(H)

    def gradient(self, x, target):
        return self.D.T @ self.gn.gradient(x, target)

    def matrix(self, x):
        return self.D.T @ self.gn.gn_matrix(x) @ self.D

    def direction(self, x, grad_q, kappa_rel):
        Pq = self.matrix(x)
        gg = float(grad_q @ grad_q)
        kappa = 0.0 if gg == 0.0 else kappa_rel * float(grad_q @ Pq @ grad_q) / gg
        return np.linalg.solve(Pq + kappa * np.eye(Pq.shape[0]), -grad_q), kappa


def fit_reduced(rest, tets, pinned, density, dt, x_prev, v_prev, pins, target, gamma, H, n_gn=3, gn_step=1.0,
                kappa_rel=1e-2, floor=FLOOR, max_halvings=12, pd_iters=30, gravity=None):
    """Gauss-Newton iterations in gamma = D q, starting from q = D^T gamma.
    Returns (gamma, losses): losses[0] is the loss at D D^T gamma."""
    from .adjoint import AdjointOracle
    from .pd_oracle import PDOracle

    n_t = len(tets)
    D = basis_matrix(H)

    def make(gm):
        o = PDOracle(rest, tets, pinned, gm[:n_t], gm[n_t:], density, dt)
        return GaussNewtonOracle(AdjointOracle(o) if gravity is None else AdjointOracle(o, gravity))

    q = D.T @ np.asarray(gamma, np.float64)
    g_now = D @ q
    if g_now.min() < floor:
        raise ValueError("the projected initial guess has a component below the floor")
    gn = make(g_now)
    x = gn.equilibrium(x_prev, v_prev, pins, pd_iters=pd_iters)
    eps = gn.loss(x, target)
    losses = [eps]
    for _ in range(n_gn):
        red = ReducedGN(gn, H)
        gq = red.gradient(x, target)
        dq, _ = red.direction(x, gq, kappa_rel)
        alpha = gn_step
        accepted = False
        for _ in range(max_halvings + 1):
            qt = q + alpha * dq
            gt_vec = D @ qt
            if gt_vec.min() >= floor:
                gt = make(gt_vec)
                xt = gt.equilibrium(x_prev, v_prev, pins, pd_iters=pd_iters)
                et = gt.loss(xt, target)
                if et < eps:
                    q, gn, x, eps = qt, gt, xt, et
                    accepted = True
                    break
            alpha *= 0.5
        losses.append(eps)
        if not accepted:
            break
    return D @ q, losses


def harmonic_initialization(rest, tets, pinned, density, dt, x_prev, v_prev, pins, target, gamma, ranks=(1, 10, 30),
                            n_gn=3, **kw):
    """Rank by rank (Sec. 6, Harmonic Initialization): returns (gamma, per-rank losses)."""
    lam, Hfull = harmonic_basis(tets, max(ranks))
    out = []
    g = np.asarray(gamma, np.float64)
    for r in ranks:
        g, losses = fit_reduced(rest, tets, pinned, density, dt, x_prev, v_prev, pins, target, g, Hfull[:, :r],
                                n_gn=n_gn, **kw)
        out.append((r, losses))
    return g, out
